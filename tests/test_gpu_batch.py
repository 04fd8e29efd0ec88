"""Batched form: systems of different size and several fields in one context.

Every k-point of every trajectory advances in the same launches (one product
launch over all items, one CUDA graph per chunk of steps).  The FP64 batch must
reproduce single-system runs bit for bit (items do not interact); the split
form must stay within the J tolerance of the oracle for every trajectory.
"""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2308_09782_gb300 import inputs
from tests._gpu_util import rel_fro

pytestmark = pytest.mark.gpu

NSTEPS = 200


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2308_09782_gb300 import vgtb
    vgtb.load()


@functools.lru_cache(maxsize=None)
def _systems():
    small = inputs.diamond_si(1, 0.05, seed=21, kgrid="mp2")
    big = inputs.diamond_si(2, 0.05, seed=64, kgrid="mp2")
    fields = [inputs.pulse_field(NSTEPS, 0.2, 0.01, 0.1, pol=(1, 0, 0)),
              inputs.pulse_field(NSTEPS, 0.2, 0.01, 0.05, pol=(0, 1, 0))]
    return small, big, fields


@functools.lru_cache(maxsize=None)
def _ground(which):
    small, big, _ = _systems()
    s = small if which == 0 else big
    ctx = O.setup(s)
    return ctx, O.ground_state(s, ctx=ctx)


@functools.lru_cache(maxsize=None)
def _oracle(which, f):
    small, big, fields = _systems()
    ctx, gs = _ground(which)
    return O.propagate(small if which == 0 else big, fields[f], NSTEPS, gs["D"], ctx=ctx)["J"]


def _run(ids, traj_sys, fields, precision):
    """ids: global system ids (0 = 8 atoms, 1 = 64 atoms) of the context's systems."""
    from paper_2308_09782_gb300 import vgtb
    small, big, _ = _systems()
    systems = [small if i == 0 else big for i in ids]
    c = vgtb.Context(systems, traj_sys=traj_sys, precision=precision, init=vgtb.INIT_USER, graph_steps=16)
    for s, gid in enumerate(ids):
        _, gs = _ground(gid)
        for k, D in enumerate(gs["D"]):
            c.set_density(s, k, D)
    for t, f in enumerate(fields):
        c.set_field(t, f)
    c.propagate(NSTEPS)
    out = [c.observables(t, charges=False)[0] for t in range(len(traj_sys))]
    c.close()
    return out


def test_fp64_batch_equals_single_runs_bitwise():
    from paper_2308_09782_gb300 import vgtb
    small, big, fields = _systems()
    traj_sys = [0, 1, 0, 1]
    fl = [fields[0], fields[0], fields[1], fields[1]]
    batch = _run([0, 1], traj_sys, fl, vgtb.FP64)
    for t, (s, f) in enumerate(zip(traj_sys, [0, 0, 1, 1])):
        single = _run([s], [0], [fields[f]], vgtb.FP64)[0]
        assert np.array_equal(batch[t], single), t


def test_split_batch_matches_oracle_per_trajectory():
    from paper_2308_09782_gb300 import vgtb
    small, big, fields = _systems()
    traj_sys = [0, 1, 0, 1]
    fl = [fields[0], fields[0], fields[1], fields[1]]
    batch = _run([0, 1], traj_sys, fl, vgtb.SPLIT_BF16X3)
    for t, (s, f) in enumerate(zip(traj_sys, [0, 0, 1, 1])):
        err = rel_fro([batch[t]], [_oracle(s, f)])
        print(f"trajectory {t} (system {s}, field {f}): J err {err:.2e}")
        assert err <= 1e-4


# ---------------------------------------------------------------------------
# Config-5 sizes: the 216-atom supercell (N = 864, padded to Np = 896, so the
# last tile rows and columns are padding) and the 512-atom supercell on the
# 2x2x2 k-grid (N = 2048, 8 k-points), as two systems of one context.
# Both start from the oracle's non-SCC density (the lowest N_el/2 generalized
# eigenstates of H0_k, occupied twice; one diagonalisation per k instead of an
# SCC loop).  With SCC on, that density is not stationary, so the charges and
# the current move from the first step.
# ---------------------------------------------------------------------------
BIG_STEPS = 20
BIG_ORACLE_STEPS = {0: 20, 1: 4}     # oracle steps per system (the 512-atom 8-k oracle takes ~7 s a step)


@functools.lru_cache(maxsize=None)
def _big_systems():
    s216 = inputs.diamond_si(3, 0.2, seed=216, kgrid="mp2")
    s512 = inputs.diamond_si(4, 0.3, seed=512, kgrid="mp2")
    fields = [inputs.pulse_field(BIG_STEPS, 0.2, 0.01, 0.1, pol=(1, 0, 0), duration=200.0),
              inputs.pulse_field(BIG_STEPS, 0.2, 0.01, 0.05, pol=(0, 1, 0), duration=200.0)]
    return [s216, s512], fields


@functools.lru_cache(maxsize=None)
def _big_start(which):
    """Oracle: S_k, H0_k, S_k^-1 and the non-SCC start density of system `which`."""
    systems, _ = _big_systems()
    s = systems[which]
    ctx = O.setup(s)
    n_occ = int(round(float(s["n_electrons"]) / 2))
    D = [O.density_from_hamiltonian(H0, S, n_occ)[0] for H0, S in zip(ctx["H0"], ctx["S"])]
    return ctx, D


@functools.lru_cache(maxsize=None)
def _big_oracle(which):
    systems, fields = _big_systems()
    ctx, D = _big_start(which)
    return O.propagate(systems[which], fields[which], BIG_ORACLE_STEPS[which], D, ctx=ctx)


def _big_run(ids, precision, nsteps=BIG_STEPS, densities=False, **opts):
    from paper_2308_09782_gb300 import vgtb
    systems, fields = _big_systems()
    c = vgtb.Context([systems[i] for i in ids], traj_sys=list(range(len(ids))), precision=precision,
                     init=vgtb.INIT_USER, graph_steps=10, **opts)
    for s, gid in enumerate(ids):
        _, D = _big_start(gid)
        for k, Dk in enumerate(D):
            c.set_density(s, k, Dk)
    for t, gid in enumerate(ids):
        c.set_field(t, fields[gid][:nsteps + 1])
    c.propagate(nsteps)
    out = []
    for t, gid in enumerate(ids):
        J, E, q = c.observables(t)
        D = [c.get_density(t, k) for k in range(8)] if densities else None
        out.append((J, E, q, D))
    c.close()
    return out


def test_config5_sizes_fp64_batch_vs_oracle_and_single_runs():
    """FP64: the 216- and 512-atom systems in one context equal their single-system
    runs bit for bit over 20 steps, and match the oracle (rho <= 1e-10, J <= 1e-8,
    q <= 1e-10, E <= 1e-9 relative) over 20 steps (216 atoms) and 4 steps (512
    atoms, 8 k)."""
    from paper_2308_09782_gb300 import vgtb
    batch = _big_run([0, 1], vgtb.FP64, densities=True)
    for gid in (0, 1):
        single = _big_run([gid], vgtb.FP64)[0]
        assert np.array_equal(batch[gid][0], single[0]), gid
        assert np.array_equal(batch[gid][2], single[2]), gid
    short = _big_run([0, 1], vgtb.FP64, nsteps=BIG_ORACLE_STEPS[1], densities=True)
    for gid in (0, 1):
        m = BIG_ORACLE_STEPS[gid]
        ref = _big_oracle(gid)
        J, E, q = batch[gid][0][:m + 1], batch[gid][1][:m + 1], batch[gid][2][:m + 1]
        err_j = rel_fro([J], [ref["J"]])
        err_q = np.abs(q - ref["q"]).max()
        err_e = np.abs(E - ref["E"]).max() / np.abs(ref["E"]).max()
        print(f"system {gid}: {m} steps, J {err_j:.2e}  q {err_q:.2e}  E {err_e:.2e}")
        assert err_j <= 1e-8
        assert err_q <= 1e-10
        assert err_e <= 1e-9
    err_d216 = rel_fro(batch[0][3], _big_oracle(0)["D"])
    err_d512 = rel_fro(short[1][3], _big_oracle(1)["D"])
    print(f"rho: 216 atoms {err_d216:.2e} ({BIG_ORACLE_STEPS[0]} steps), 512 atoms 8 k {err_d512:.2e} "
          f"({BIG_ORACLE_STEPS[1]} steps)")
    assert err_d216 <= 1e-10
    assert err_d512 <= 1e-10


def test_config5_sizes_chained_products_equal_two_launches():
    """Split form, 216 atoms (Np = 896: row blocks of 256 with a half-empty last
    one, column tiles across the Re/Im boundary of W) and 512 atoms on 8 k-points
    in one context: both products in one launch (product 2 tiles waiting for the
    rows of W they read) give the same propagation as two launches, bit for bit,
    with the same tile variants (product 2 on planned column widths)."""
    from paper_2308_09782_gb300 import vgtb
    opts = dict(tile_variant=[0, 7])
    one = _big_run([0, 1], vgtb.SPLIT_BF16X3, densities=True, chain=vgtb.CHAIN_ON, **opts)
    two = _big_run([0, 1], vgtb.SPLIT_BF16X3, densities=True, chain=vgtb.CHAIN_OFF, **opts)
    for gid in (0, 1):
        assert np.array_equal(one[gid][0], two[gid][0])
        assert np.array_equal(one[gid][1], two[gid][1])
        for k in (0, 7):
            assert np.array_equal(one[gid][3][k], two[gid][3][k])


def test_config5_sizes_split_batch_vs_oracle_and_fp64():
    """Split form, same context: J within 1e-4 of the oracle (216 atoms, 20 steps;
    512 atoms 8 k, 4 steps) and of the FP64 batch over all 20 steps."""
    from paper_2308_09782_gb300 import vgtb
    split = _big_run([0, 1], vgtb.SPLIT_BF16X3)
    fp64 = _big_run([0, 1], vgtb.FP64)
    for gid in (0, 1):
        m = BIG_ORACLE_STEPS[gid]
        err_o = rel_fro([split[gid][0][:m + 1]], [_big_oracle(gid)["J"]])
        err_f = rel_fro([split[gid][0]], [fp64[gid][0]])
        print(f"system {gid}: J vs oracle {err_o:.2e} ({m} steps), vs FP64 batch {err_f:.2e} ({BIG_STEPS} steps)")
        assert err_o <= 1e-4
        assert err_f <= 1e-4
