"""Failure paths and device unit tests (GPU).

* A leapfrog far beyond its stability bound (dt = 20 au, dt times the spectral
  width of S^-1 H is about 20 where the leapfrog needs it below 1) drives the
  density to overflow.  The host-made failure must come back as VGTB_E_UNSTABLE
  (-7) from vgtb_propagate, in both precision forms, and a fresh context must
  work afterwards.
* The integer-bit float <-> double conversions of the split-precision kernels
  agree bit for bit with CUDA's own conversions on ties, near-ties, the largest
  floats, overflow, infinities and NaNs; below 2^-126 they flush to signed zero
  (their stated behaviour; CUDA would give float subnormals there).
"""
import numpy as np
import pytest

from tests._gpu_util import system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2308_09782_gb300 import vgtb
    vgtb.load()


@pytest.mark.parametrize("precision", [0, 1])
def test_unstable_time_step_returns_e_unstable_then_fresh_context_runs(precision):
    from paper_2308_09782_gb300 import inputs, vgtb
    sysd, _, _ = system("si8_pulse")
    bad = dict(sysd)
    bad["dt"] = 20.0
    n = 200
    A = inputs.kick_field(n, 0.001)
    with vgtb.Context(bad, precision=precision, init=vgtb.INIT_GROUND, graph_steps=1) as c:
        c.set_field(0, A)
        with pytest.raises(vgtb.VgtbError) as ei:
            c.propagate(n)
        assert ei.value.code == -7
    with vgtb.Context(sysd, precision=precision, init=vgtb.INIT_GROUND) as c:
        c.set_field(0, inputs.kick_field(40, 0.001))
        c.propagate(40)
        J, E, q = c.observables(0)
        assert np.all(np.isfinite(J)) and np.all(np.isfinite(E))
        assert np.abs(q.sum(axis=1) - sysd["n_electrons"]).max() < 1e-6


def _bits32(x):
    return np.asarray(x, np.float32).view(np.uint32)


def _bits64(x):
    return np.asarray(x, np.float64).view(np.uint64)


def test_bit_conversions_match_cuda():
    from paper_2308_09782_gb300 import vgtb
    rng = np.random.default_rng(2308)
    # doubles over the normal float range, both signs
    d = np.ldexp(rng.uniform(1.0, 2.0, 4000), rng.integers(-125, 127, 4000)) * rng.choice([-1.0, 1.0], 4000)
    # exact ties and near-ties between two neighbouring floats: the 29 dropped bits = 0x10000000 (+-1)
    f = np.ldexp(rng.uniform(1.0, 2.0, 1000), rng.integers(-120, 120, 1000)).astype(np.float32)
    base = f.astype(np.float64).view(np.uint64)
    ties = np.concatenate([base + (1 << 28), base + (1 << 28) - 1, base + (1 << 28) + 1]).view(np.float64)
    fmax = float(np.finfo(np.float32).max)
    ulp_top = 2.0 ** 104
    special = np.array([0.0, -0.0, 1.0, -1.0, fmax, -fmax, fmax + 0.49 * ulp_top, fmax + 0.5 * ulp_top,
                        3.5e38, -3.5e38, 1e300, -1e300, np.inf, -np.inf, 2.0 ** -126, -(2.0 ** -126)])
    dd = np.concatenate([d, ties, special])
    special_f = np.array([0.0, -0.0, 1.0, -1.0, fmax, -fmax, 2.0 ** -126, -(2.0 ** -126),
                          np.inf, -np.inf, 3.0e38, -3.0e38, 1e-30, -1e-30, 65504.0, 1.0 / 3.0], np.float32)
    assert len(special_f) == len(special)
    fi = np.concatenate([dd[:-len(special)].astype(np.float32), special_f])
    fb, fr, db, dr = vgtb.diag_convert(dd, fi)
    assert np.array_equal(_bits32(fb), _bits32(fr))
    assert np.array_equal(_bits64(db), _bits64(dr))
    # NaN: a quiet NaN of the same sign both ways
    nan_d = np.array([np.nan, -np.nan, np.array([0x7ff0000000000001], np.uint64).view(np.float64)[0]])
    nan_f = np.array([np.nan, -np.nan, np.array([0x7f800001], np.uint32).view(np.float32)[0]], np.float32)
    fb, fr, db, dr = vgtb.diag_convert(nan_d, nan_f)
    assert np.all(np.isnan(fb)) and np.array_equal(np.signbit(fb), np.signbit(nan_d))
    assert np.all(np.isnan(db)) and np.array_equal(np.signbit(db), np.signbit(nan_f))
    # below 2^-126: signed zero (CUDA keeps float subnormals there)
    tiny = np.array([1e-39, -1e-39, 2.0 ** -127, -(2.0 ** -149), 1e-300])
    tiny_f = np.array([1e-39, -1e-39, 2.0 ** -127, -(2.0 ** -149), 0.0], np.float32)
    fb, fr, db, dr = vgtb.diag_convert(tiny, tiny_f)
    assert np.all(fb == 0.0) and np.array_equal(np.signbit(fb), np.signbit(tiny))
    assert np.all(db == 0.0) and np.array_equal(np.signbit(db), np.signbit(tiny_f))
    assert np.any(fr != 0.0)  # CUDA itself rounds to subnormals here
