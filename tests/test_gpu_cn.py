"""Parity of the Crank-Nicolson coefficient path (Eq. 5) with the CPU oracle.

The library runs the scheme in FP64 with fixed-point sweeps for the linear
system; the oracle solves it directly (LU).  Bounds: J(t) within 1e-8
(relative, whole series), charges within 1e-9, the states C_k within 1e-9.
"""
import functools

import numpy as np
import pytest

import oracle as O
from oracle import crank_nicolson as cn
from paper_2308_09782_gb300 import inputs
from tests._gpu_util import oracle_ground, rel_fro, system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2308_09782_gb300 import vgtb
    vgtb.load()


@functools.lru_cache(maxsize=None)
def si8d():
    """Distorted 8-atom cell (charge transfer present) with a strong pulse."""
    s = inputs.diamond_si(1, sigma=0.3, seed=5, kgrid="mp2", dt=0.2)
    ctx = O.setup(s)
    return s, ctx, O.ground_state(s, ctx=ctx)


def _cn_ctx(sysd, C0, **opts):
    from paper_2308_09782_gb300 import vgtb
    c = vgtb.Context(sysd, precision=vgtb.FP64, init=vgtb.INIT_USER, integrator=vgtb.CRANK_NICOLSON, **opts)
    for k, Ck in enumerate(C0):
        c.set_coefficients(0, k, Ck)
    return c


def _compare(c, ref, sysd, n_occ, j_tol=1e-8):
    J, E, q = c.observables(0)
    Cs = [c.get_coefficients(0, k, n_occ) for k in range(len(sysd["wk"]))]
    assert rel_fro([J], [ref["J"]]) <= j_tol
    assert np.abs(E - ref["E"]).max() <= 1e-9 * max(1.0, np.abs(ref["E"]).max())
    assert np.abs(q - ref["q"]).max() <= 1e-9
    assert rel_fro(Cs, ref["C"]) <= 1e-9
    return J, E, q, Cs


def test_cn_distorted_si8_pulse_vs_oracle():
    s, ctx, gs = si8d()
    n = 400
    A = inputs.pulse_field(n, s["dt"], 0.05, 0.3)
    ref = cn.propagate_cn(s, A, n, gs["C"], ctx=ctx)
    with _cn_ctx(s, gs["C"]) as c:
        c.set_field(0, A)
        c.propagate(n)
        J, _, _, _ = _compare(c, ref, s, gs["C"][0].shape[1])
    assert np.abs(J).max() > 1e-6


def test_cn_si64_pulse_vs_oracle():
    name, n = "si64_pulse", 300
    sysd, A, _ = system(name)
    ctx, gs = oracle_ground(name)
    ref = cn.propagate_cn(sysd, A[:n + 1], n, gs["C"], ctx=ctx)
    with _cn_ctx(sysd, gs["C"]) as c:
        c.set_field(0, A[:n + 1])
        c.propagate(n)
        _compare(c, ref, sysd, gs["C"][0].shape[1])


def test_cn_block_sparse_and_dense_m_agree():
    """M = S^-1 H of every Crank-Nicolson step runs over H's nonzero atom blocks by
    default and as a dense FP64 GEMM with product1 = DENSE: the same products up to
    summation order, so the states agree to 1e-12 after 100 steps (si64, pulse),
    and the dense run is within the oracle bounds too."""
    from paper_2308_09782_gb300 import vgtb
    name, n = "si64_pulse", 100
    sysd, A, _ = system(name)
    ctx, gs = oracle_ground(name)
    n_occ = gs["C"][0].shape[1]
    ref = cn.propagate_cn(sysd, A[:n + 1], n, gs["C"], ctx=ctx)
    with _cn_ctx(sysd, gs["C"]) as a, _cn_ctx(sysd, gs["C"], product1=vgtb.P1_DENSE) as b:
        for c in (a, b):
            c.set_field(0, A[:n + 1])
            c.propagate(n)
        Ca = [a.get_coefficients(0, k, n_occ) for k in range(8)]
        Cb = [b.get_coefficients(0, k, n_occ) for k in range(8)]
        assert rel_fro(Ca, Cb) <= 1e-12
        _compare(b, ref, sysd, n_occ)


def test_cn_512_atoms_gamma_prefix():
    """512-atom Gamma kick (N = 2048, 1024 occupied states): 6 steps vs the oracle."""
    name, n = "si512_kick", 6
    sysd, A, _ = system(name)
    ctx, gs = oracle_ground(name)
    ref = cn.propagate_cn(sysd, A[:n + 1], n, gs["C"], ctx=ctx)
    with _cn_ctx(sysd, gs["C"]) as c:
        c.set_field(0, A[:n + 1])
        c.propagate(n)
        _compare(c, ref, sysd, gs["C"][0].shape[1])


def test_cn_library_ground_state_is_stationary():
    """From the library's own ground state, no field: D_k(t) stays D_k(0)."""
    from paper_2308_09782_gb300 import vgtb
    s, _, _ = si8d()
    n = 60
    with vgtb.Context(s, precision=vgtb.FP64, init=vgtb.INIT_GROUND, integrator=vgtb.CRANK_NICOLSON) as c:
        c.set_field(0, np.zeros((n + 1, 3)))
        c.propagate(n)
        for k in range(len(s["wk"])):
            assert np.abs(c.get_density(0, k) - c.get_initial_density(0, k)).max() <= 1e-10
        _, _, q = c.observables(0)
    assert np.abs(q - q[0]).max() <= 1e-10


def test_cn_graphs_reruns_and_checkpoint_bitwise():
    s, _, gs = si8d()
    n = 90
    A = inputs.pulse_field(n, s["dt"], 0.05, 0.3)
    with _cn_ctx(s, gs["C"], graph_steps=1) as c:
        c.set_field(0, A)
        c.propagate(n)
        J1, E1, q1 = c.observables(0)
    with _cn_ctx(s, gs["C"], graph_steps=16) as c:
        c.set_field(0, A)
        c.propagate(37)
        state = c.get_state()
        c.propagate(n - 37)
        J2, E2, q2 = c.observables(0)
        c.set_state(state)
        c.propagate(n - 37)
        J3, _, _ = c.observables(0)
    assert np.array_equal(J1, J2) and np.array_equal(E1, E2) and np.array_equal(q1, q2)
    assert np.array_equal(J2, J3)


def test_cn_batch_equals_single_runs():
    from paper_2308_09782_gb300 import vgtb
    s8, _, gs8 = si8d()
    s64, A64, _ = system("si64_pulse")
    _, gs64 = oracle_ground("si64_pulse")
    s64 = dict(s64)
    n = 40
    fields = [inputs.pulse_field(n, 0.2, 0.05, 0.3), A64[:n + 1]]
    singles = []
    for sd, g, A in [(s8, gs8, fields[0]), (s64, gs64, fields[1]), (s8, gs8, fields[1])]:
        with _cn_ctx(sd, g["C"]) as c:
            c.set_field(0, A)
            c.propagate(n)
            singles.append(c.observables(0)[0])
    with vgtb.Context([s8, s64], traj_sys=[0, 1, 0], precision=vgtb.FP64, init=vgtb.INIT_USER,
                      integrator=vgtb.CRANK_NICOLSON) as c:
        for si, g in enumerate([gs8, gs64]):
            for k, Ck in enumerate(g["C"]):
                c.set_coefficients(si, k, Ck)
        for t, A in enumerate([fields[0], fields[1], fields[1]]):
            c.set_field(t, A)
        c.propagate(n)
        for t in range(3):
            assert np.array_equal(c.observables(t)[0], singles[t])


def test_cn_too_few_sweeps_is_reported():
    from paper_2308_09782_gb300 import vgtb
    s, _, gs = si8d()
    A = inputs.pulse_field(10, s["dt"], 0.05, 0.3)
    with _cn_ctx(s, gs["C"], cn_iter=3) as c:
        c.set_field(0, A)
        with pytest.raises(vgtb.VgtbError) as e:
            c.propagate(10)
        assert e.value.code == -7 and "Crank-Nicolson" in str(e.value)


def test_cn_argument_errors():
    from paper_2308_09782_gb300 import vgtb
    s, _, gs = si8d()
    with pytest.raises(vgtb.VgtbError):
        vgtb.Context(s, precision=vgtb.SPLIT_BF16X3, integrator=vgtb.CRANK_NICOLSON)
    with pytest.raises(vgtb.VgtbError):
        vgtb.Context(s, precision=vgtb.FP64, integrator=vgtb.CRANK_NICOLSON, cn_iter=1)
    with _cn_ctx(s, gs["C"]) as c:
        with pytest.raises(vgtb.VgtbError):
            c.set_density(0, 0, gs["D"][0])
        with pytest.raises(vgtb.VgtbError):
            c.set_coefficients(0, 0, gs["C"][0][:, :-1])
