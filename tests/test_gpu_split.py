"""The tcgen05 split-precision form against numpy and against the FP64 oracle.

Product-level tolerance: BF16 hi/lo pieces carry ~2^-17 relative precision and
three partial products are accumulated in FP32, so a relative Frobenius error
of 3e-5 bounds one product.  Propagation tolerance of the split-precision form: J(t)
within 1e-4 relative of the FP64 oracle.
"""
import numpy as np
import pytest

from tests._gpu_util import gpu_run, oracle_ground, oracle_run, rel_fro, system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2308_09782_gb300 import vgtb
    vgtb.load()


@pytest.mark.parametrize("n", [128, 200, 384, 1000])
def test_split_products_match_numpy(n):
    from paper_2308_09782_gb300 import vgtb
    rng = np.random.default_rng(n)
    def rnd():
        return rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    a, r, s = rnd(), rnd(), rnd()
    w, x = vgtb.diag_split_chain(a, r, s)
    w_ref = a @ r.conj().T
    assert rel_fro([w], [w_ref]) < 3e-5
    x_ref = s @ w_ref.conj().T
    assert rel_fro([x], [x_ref]) < 6e-5
    # structure: a transposed operand or a lost sign would give O(1) errors
    assert rel_fro([x], [s @ w_ref]) > 0.1


@pytest.mark.parametrize("n", [384, 1000, 2048])
def test_every_tile_variant_matches_numpy(n):
    """Each schedule the autotuner may pick, forced on its own.  At n = 2048 the
    128 pair tiles fill one whole wave of 76 pairs and leave 52 tiles to the
    stream-K part of the mixed schedule."""
    from paper_2308_09782_gb300 import vgtb
    rng = np.random.default_rng(7 + n)
    def rnd():
        return rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    a, r, s = rnd(), rnd(), rnd()
    w_ref = a @ r.conj().T
    x_ref = s @ w_ref.conj().T
    for v in range(vgtb.num_tile_variants()):
        w, x = vgtb.diag_split_chain(a, r, s, variant=v)
        assert rel_fro([w], [w_ref]) < 3e-5, v
        assert rel_fro([x], [x_ref]) < 6e-5, v


@pytest.mark.parametrize("product1", [0, 2])
@pytest.mark.parametrize("name,nsteps", [("si8_pulse", 1000), ("si64_pulse", 2000)])
def test_split_propagation_matches_oracle(name, nsteps, product1):
    """product1 = AUTO (0): the tcgen05 BF16x3 first product over all of
    [dD | D0][H | dH]^dagger (the split form's default); BLOCKS (2): the
    block-sparse FP32 first product on the CUDA cores."""
    from paper_2308_09782_gb300 import vgtb
    ref = oracle_run(name, nsteps)
    with gpu_run(name, nsteps, precision=vgtb.SPLIT_BF16X3, product1=product1) as c:
        J, E, q = c.observables(0)
        D = [c.get_density(0, k) for k in range(8)]
    err_j = rel_fro([J], [ref["J"]])
    err_d = rel_fro(D, ref["D"])
    err_q = np.abs(q - ref["q"]).max()
    err_e = np.abs(E - ref["E"]).max()
    print(f"{name} product1={product1}: J {err_j:.3e}  D {err_d:.3e}  q {err_q:.3e}  E {err_e:.3e}")
    assert err_j <= 1e-4
    assert err_d <= 1e-4
    assert err_q <= 1e-4


def test_bounded_waits_run_out_deterministically():
    """The product kernels' wait routines, on an mbarrier phase that no thread
    completes and on a stream-K flag that no CTA sets, give up after their limit
    (1 ms here) and report it: VGTB_E_TIMEOUT, no hang; the GPU stays usable."""
    from paper_2308_09782_gb300 import vgtb
    lib = vgtb.load()
    for which in (0, 1):
        assert lib.vgtb_diag_bounded_wait(1_000_000, which) == -8, which
    assert lib.vgtb_diag_bounded_wait(0, 0) == -1
    with gpu_run("si8_pulse", 20, precision=vgtb.SPLIT_BF16X3) as ok:
        J, _, _ = ok.observables(0)
    assert np.all(np.isfinite(J))


def test_split_timeout_returns_error_and_context_recovers():
    """A 1 ns wait limit makes the tcgen05 product kernels give up inside
    vgtb_propagate: E_TIMEOUT, no hang; a fresh context afterwards works.  The
    64-atom system with the dense tcgen05 first product (K' = 4 Np) keeps the
    kernels' waits long enough to reach the limit check."""
    from paper_2308_09782_gb300 import vgtb
    name = "si64_pulse"
    sysd, A, _ = system(name)
    _, gs = oracle_ground(name)
    c = vgtb.Context(sysd, precision=vgtb.SPLIT_BF16X3, init=vgtb.INIT_USER, timeout_ns=1, product1=1)
    for k, D in enumerate(gs["D"]):
        c.set_density(0, k, D)
    c.set_field(0, A[:6])
    with pytest.raises(vgtb.VgtbError) as e:
        c.propagate(5)
    assert e.value.code == -8
    c.close()
    with gpu_run(name, 20, precision=vgtb.SPLIT_BF16X3) as ok:
        J, _, _ = ok.observables(0)
    assert np.all(np.isfinite(J))


@pytest.mark.parametrize("variant", [0, 5, 1, 7])
def test_zero_panel_skipping_matches_the_dense_product(variant):
    """Product 1 skips the k-panels in which a tile's rows of H and dH are zero
    (512 atoms, rows of H interleaved Re/Im in blocks of four: 36 of 64 panels remain
    for 256-row tiles, 32 for 128-row tiles).
    Those panels contribute exact zeros, so with a classic schedule (2-SM pair
    256-wide tiles, variant 0; single-CTA 128-wide tiles, variant 5) the
    propagation equals the dense product (product1 = DENSE, same variant) bit for
    bit; with stream-K (variant 1) the k-ranges of the workers move, so the FP32
    partial sums meet in another order, and with planned column widths (variant
    7) the two runs plan their tiles from different costs: J within 1e-6.  50 steps."""
    from paper_2308_09782_gb300 import vgtb
    name, nsteps = "si512_kick", 50
    tv = [variant, 0]
    with gpu_run(name, nsteps, precision=vgtb.SPLIT_BF16X3, tile_variant=tv) as a, \
            gpu_run(name, nsteps, precision=vgtb.SPLIT_BF16X3, tile_variant=tv, product1=vgtb.P1_DENSE) as b:
        assert "zero k-panels skipped" in a.tile_config(1)["schedule"]
        assert "skipped" not in b.tile_config(1)["schedule"]
        Ja, _, _ = a.observables(0)
        Jb, _, _ = b.observables(0)
        if variant in (1, 7):
            assert rel_fro([Ja], [Jb]) <= 1e-6
        else:
            assert np.array_equal(Ja, Jb)
            assert np.array_equal(a.get_density(0, 0), b.get_density(0, 0))


@pytest.mark.parametrize("tv", [[0, 0], [0, 7], [5, 7]])
def test_chained_products_equal_two_launches(tv):
    """Both products in one launch: product 2 tiles start as soon as the 256-row
    blocks of W they read are stored (bounded waits on per-block counts, an epoch
    per launch so nothing is reset).  Same tile variants, so the propagation
    equals two launches bit for bit: 512 atoms, 50 steps (graphs of 50 launches,
    so the epoch advances across replays).  Product 1 on single CTAs (variant 5)
    cannot be chained: the option then keeps two launches."""
    from paper_2308_09782_gb300 import vgtb
    name, nsteps = "si512_kick", 50
    with gpu_run(name, nsteps, precision=vgtb.SPLIT_BF16X3, tile_variant=tv, chain=vgtb.CHAIN_ON,
                 graph_steps=50) as a, \
            gpu_run(name, nsteps, precision=vgtb.SPLIT_BF16X3, tile_variant=tv, chain=vgtb.CHAIN_OFF) as b:
        chained = "one launch" in a.tile_config(1)["schedule"]
        assert chained == (tv[0] != 5)
        assert "one launch" not in b.tile_config(1)["schedule"]
        Ja, Ea, _ = a.observables(0)
        Jb, Eb, _ = b.observables(0)
        assert np.array_equal(Ja, Jb)
        assert np.array_equal(Ea, Eb)
        assert np.array_equal(a.get_density(0, 0), b.get_density(0, 0))


def test_split_rerun_bitwise_and_autotuned_variants_agree():
    """The stream-K fixup sums partials in a fixed order: reruns are bitwise equal.
    The autotuner's choice (stream-K or classic tiles, 128 or 256 wide) stays within
    the product tolerance of the default."""
    from paper_2308_09782_gb300 import vgtb
    name, nsteps = "si64_pulse", 200
    with gpu_run(name, nsteps, precision=vgtb.SPLIT_BF16X3) as a, \
            gpu_run(name, nsteps, precision=vgtb.SPLIT_BF16X3) as b, \
            gpu_run(name, nsteps, precision=vgtb.SPLIT_BF16X3, autotune=1) as c:
        Ja, _, _ = a.observables(0)
        Jb, _, _ = b.observables(0)
        Jc, _, _ = c.observables(0)
        assert np.array_equal(Ja, Jb)
        assert np.array_equal(a.get_density(0, 5), b.get_density(0, 5))
    ref = oracle_run(name, nsteps)
    assert rel_fro([Jc], [ref["J"]]) <= 1e-4
