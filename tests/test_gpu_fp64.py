"""Parity of the plain FP64 CUDA path with the CPU oracle (through the C-ABI).

Tolerances: relative Frobenius error <= 1e-10 in D_k after
the stated step count and <= 1e-8 in J(t) over the whole series.
"""
import numpy as np
import pytest

import oracle as O
from paper_2308_09782_gb300 import inputs
from tests._gpu_util import gpu_run, oracle_ground, oracle_run, rel_fro, system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2308_09782_gb300 import vgtb
    vgtb.load()


@pytest.mark.parametrize("name,nsteps", [("si8_pulse", 1000), ("si64_pulse", 2000)])
def test_fp64_matches_oracle_full_run(name, nsteps):
    sysd, A, n = system(name)
    assert nsteps == n
    ref = oracle_run(name, nsteps)
    with gpu_run(name, nsteps) as c:
        J, E, q = c.observables(0)
        D = [c.get_density(0, k) for k in range(len(sysd["wk"]))]
    assert rel_fro(D, ref["D"]) <= 1e-10
    assert rel_fro([J], [ref["J"]]) <= 1e-8
    assert np.abs(E - ref["E"]).max() <= 1e-9 * max(1.0, np.abs(ref["E"]).max())
    assert np.abs(q - ref["q"]).max() <= 1e-10


def test_dense_and_block_sparse_first_product_agree():
    """product1 = DENSE runs the first product W = D H as a dense FP64 GEMM over all
    of H; the default runs it block-sparse over H's nonzero atom blocks.  The two
    differ only in summation order: D and J agree to 1e-12 after 300 steps of the
    64-atom system, and both match the oracle."""
    name, nsteps = "si64_pulse", 300
    ref = oracle_run(name, nsteps)
    with gpu_run(name, nsteps) as a, gpu_run(name, nsteps, product1=1) as b:
        Ja, _, _ = a.observables(0)
        Jb, _, _ = b.observables(0)
        Da = [a.get_density(0, k) for k in range(8)]
        Db = [b.get_density(0, k) for k in range(8)]
    assert rel_fro(Da, Db) <= 1e-12
    assert rel_fro([Ja], [Jb]) <= 1e-12
    assert rel_fro(Db, ref["D"]) <= 1e-10
    assert rel_fro([Jb], [ref["J"]]) <= 1e-8


def test_fp64_512_atoms_gamma_prefix():
    """512-atom Gamma kick (N = 2048): 20 steps element by element vs the oracle."""
    name, nsteps = "si512_kick", 20
    ref = oracle_run(name, nsteps)
    with gpu_run(name, nsteps) as c:
        J, E, q = c.observables(0)
        D = c.get_density(0, 0)
    assert rel_fro([D], ref["D"]) <= 1e-10
    assert rel_fro([J], [ref["J"]]) <= 1e-8
    assert np.abs(E - ref["E"]).max() <= 1e-9 * np.abs(ref["E"]).max()


def test_gpu_ground_state_matches_oracle():
    """The library's own SCC ground state (cuSOLVER + DIIS) equals the oracle's."""
    from paper_2308_09782_gb300 import vgtb
    name = "si64_pulse"
    sysd, A, n = system(name)
    _, gs = oracle_ground(name)
    with vgtb.Context(sysd, precision=vgtb.FP64, init=vgtb.INIT_GROUND) as c:
        c.set_field(0, A[:11])
        c.propagate(0)
        J, E, q = c.observables(0)
        D = [c.get_density(0, k) for k in range(len(sysd["wk"]))]
    assert rel_fro(D, gs["D"]) <= 1e-8
    assert np.abs(q[0] - 4.0 - gs["dq"]).max() <= 1e-9


def test_delta_form_equals_eq6():
    """P-5: the exact delta form dD/dt = R0 - i[S^-1(H dD + dH D0) - h.c.] gives Eq. 6's D."""
    name, nsteps = "si64_pulse", 300
    with gpu_run(name, nsteps) as a, gpu_run(name, nsteps, delta_form=1) as b:
        Ja, _, _ = a.observables(0)
        Jb, _, _ = b.observables(0)
        Da = [a.get_density(0, k) for k in range(8)]
        Db = [b.get_density(0, k) for k in range(8)]
    assert rel_fro(Db, Da) <= 1e-12
    assert rel_fro([Jb], [Ja]) <= 1e-10


def test_hermiticity_bitwise_and_electron_count():
    name, nsteps = "si8_pulse", 400
    sysd, _, _ = system(name)
    ctx, _ = oracle_ground(name)
    with gpu_run(name, nsteps) as c:
        for k in range(8):
            D = c.get_density(0, k)
            assert np.array_equal(D, D.conj().T)
            assert abs(np.trace(D @ ctx["S"][k]).real - sysd["n_electrons"]) < 1e-11
        _, _, q = c.observables(0)
    np.testing.assert_allclose(q.sum(1), sysd["n_electrons"], atol=1e-10)


def test_rerun_and_graph_are_bitwise_identical():
    name, nsteps = "si8_pulse", 100
    with gpu_run(name, nsteps) as a, gpu_run(name, nsteps) as b, gpu_run(name, nsteps, graph_steps=1) as g:
        Ja, Ea, _ = a.observables(0)
        Jb, Eb, _ = b.observables(0)
        Jg, Eg, _ = g.observables(0)
        assert np.array_equal(Ja, Jb) and np.array_equal(Ea, Eb)
        assert np.array_equal(Ja, Jg) and np.array_equal(Ea, Eg)
        assert np.array_equal(a.get_density(0, 3), g.get_density(0, 3))


def _ctx_full_field(name, **opts):
    from paper_2308_09782_gb300 import vgtb
    sysd, A, n = system(name)
    _, gs = oracle_ground(name)
    c = vgtb.Context(sysd, init=vgtb.INIT_USER, **opts)
    for k, D in enumerate(gs["D"]):
        c.set_density(0, k, D)
    c.set_field(0, A)
    return c


def test_checkpoint_resume_bitwise():
    name = "si8_pulse"
    with _ctx_full_field(name) as full:
        full.propagate(150)
        Jf, _, _ = full.observables(0)
        Df = full.get_density(0, 2)
    with _ctx_full_field(name) as a:
        a.propagate(60)
        st = a.get_state()
        a.propagate(90)
        Ja, _, _ = a.observables(0)
        assert np.array_equal(Ja, Jf) and np.array_equal(a.get_density(0, 2), Df)
    with _ctx_full_field(name) as b:
        b.propagate(10)
        b.set_state(st)
        assert b.steps_done == 60
        b.propagate(90)
        assert np.array_equal(b.get_density(0, 2), Df)
        Jb, _, _ = b.observables(0)
        assert np.array_equal(Jb[60:], Jf[60:])


def test_error_codes():
    from paper_2308_09782_gb300 import vgtb
    sysd, A, n = system("si8_pulse")
    _, gs = oracle_ground("si8_pulse")
    # propagate without a density, then without a long enough field
    with vgtb.Context(sysd, init=vgtb.INIT_USER) as c:
        c.set_field(0, A[:5])
        with pytest.raises(vgtb.VgtbError) as e:
            c.propagate(2)
        assert e.value.code == -6
        for k, D in enumerate(gs["D"]):
            c.set_density(0, k, D)
        with pytest.raises(vgtb.VgtbError) as e:
            c.propagate(10)
        assert e.value.code == -6
        c.propagate(4)
        bad = A[:5].copy()
        bad[2, 0] = np.nan
        with pytest.raises(vgtb.VgtbError) as e:
            c.set_field(0, bad)
        assert e.value.code == -1
    # missing mirror block: drop one block with I != J (on-site blocks mirror themselves)
    b = int(np.nonzero(sysd["blk_ijl"][:, 0] != sysd["blk_ijl"][:, 1])[0][0])
    keep = np.ones(len(sysd["blk_ijl"]), bool)
    keep[b] = False
    s2 = dict(sysd)
    s2["blk_ijl"] = sysd["blk_ijl"][keep]
    vals = np.repeat(keep, 16)
    s2["h0"], s2["s"], s2["ds"] = sysd["h0"][vals], sysd["s"][vals], sysd["ds"][:, vals]
    with pytest.raises(vgtb.VgtbError) as e:
        vgtb.Context(s2)
    assert e.value.code == -1
    # overlap that is not positive definite
    s3 = dict(sysd)
    scale = np.repeat(np.where(np.all(sysd["blk_ijl"][:, 2:] == 0, axis=1)
                               & (sysd["blk_ijl"][:, 0] == sysd["blk_ijl"][:, 1]), 1.0, 4.0), 16)
    s3["s"] = sysd["s"] * scale
    s3["ds"] = sysd["ds"] * scale
    with pytest.raises(vgtb.VgtbError) as e:
        vgtb.Context(s3)
    assert e.value.code == -2
    # asymmetric gamma
    s4 = dict(sysd)
    g = sysd["gamma"].copy()
    g[0, 1] += 1e-3
    s4["gamma"] = g
    with pytest.raises(vgtb.VgtbError) as e:
        vgtb.Context(s4)
    assert e.value.code == -1


@pytest.mark.parametrize("graph_steps", [1, 16])
def test_profiling_counts_every_kernel(graph_steps):
    """vgtb_profile: events around every hot kernel, with and without graphs."""
    with _ctx_full_field("si8_pulse", graph_steps=graph_steps) as c:
        c.propagate(5)
        c.profile(True)            # enable and reset the counters
        c.propagate(40)
        st = c.kernel_stats()
    for k, (n, ms) in st.items():
        assert n == 40 and ms > 0.0, (k, n, ms)


@pytest.mark.parametrize("precision", [0, 1])
def test_frozen_scc_shift_matches_oracle(precision):
    """scc = VGTB_SCC_FROZEN: H keeps the shift of D(0) at every step (the oracle's
    eps_fixed).  si64_pulse, 300 steps: FP64 within the FP64 bounds (rho 1e-10,
    J 1e-8), the split form within 1e-4 in J; the self-consistent run differs."""
    from paper_2308_09782_gb300 import vgtb
    name, nsteps = "si64_pulse", 300
    sysd, A, _ = system(name)
    ctx, gs = oracle_ground(name)
    ref = O.propagate(sysd, A, nsteps, gs["D"], ctx=ctx, eps_fixed=gs["eps"])
    ref_scc = oracle_run(name, nsteps)
    with gpu_run(name, nsteps, precision=precision, scc=vgtb.SCC_FROZEN) as c:
        J, E, q = c.observables(0)
        D = [c.get_density(0, k) for k in range(8)]
    err_j = rel_fro([J], [ref["J"]])
    print(f"frozen shift, precision {precision}: J {err_j:.2e}, vs SCC run {rel_fro([J], [ref_scc['J']]):.2e}")
    # freezing the shift changes J by ~2e-5 here: the run must follow the frozen reference
    assert err_j < 0.1 * rel_fro([J], [ref_scc["J"]])
    if precision == 0:
        assert rel_fro(D, ref["D"]) <= 1e-10
        assert err_j <= 1e-8
        assert np.abs(q - ref["q"]).max() <= 1e-10
    else:
        assert err_j <= 1e-4
