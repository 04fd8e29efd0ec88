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
