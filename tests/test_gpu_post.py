"""Device reductions after propagation: spectrum (Eqs. 15, 16) and group charges,
against the oracle's own propagation followed by the oracle's formulas."""
import numpy as np
import pytest

import oracle as O
from oracle import spectrum as OS
from paper_2308_09782_gb300 import inputs
from tests._gpu_util import oracle_ground, system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2308_09782_gb300 import vgtb
    vgtb.load()


def test_spectrum_of_a_kick_matches_oracle():
    from paper_2308_09782_gb300 import vgtb
    sysd, _, _ = system("si8_pulse")
    ctx, gs = oracle_ground("si8_pulse")
    n, a0 = 1500, 0.001
    A = inputs.kick_field(n, a0)
    ref_J = O.propagate(sysd, A, n, gs["D"], ctx=ctx)["J"]
    e0 = -a0 / O.C_LIGHT
    w = np.linspace(0.02, 1.0, 60)
    s_ref = OS.conductivity(ref_J, sysd["dt"], e0, w, 200.0)
    e_ref = OS.dielectric(s_ref, w)
    with vgtb.Context(sysd, init=vgtb.INIT_USER) as c:
        for k, D in enumerate(gs["D"]):
            c.set_density(0, k, D)
        c.set_field(0, A)
        c.propagate(n)
        s, e = c.spectrum(0, e0, w, tau0=200.0)
        s2, _ = c.spectrum(0, e0, w, n0=100, n1=900)
    assert np.abs(s - s_ref).max() <= 1e-8 * np.abs(s_ref).max()
    assert np.abs(e - e_ref).max() <= 1e-8 * np.abs(e_ref).max()
    t = np.arange(801) * sysd["dt"]
    assert np.abs(s2 - OS.conductivity(ref_J[100:901], sysd["dt"], e0, w, 200.0)).max() <= 1e-8 * np.abs(s2).max()
    assert np.abs(s[:, 0]).max() > 10 * np.abs(s[:, 1]).max()   # response along the kick
    del t


def test_group_charges_match_oracle_series():
    from paper_2308_09782_gb300 import vgtb
    sysd, A, _ = system("si64_pulse")
    ctx, gs = oracle_ground("si64_pulse")
    n = 300
    ref_q = O.propagate(sysd, A, n, gs["D"], ctx=ctx)["q"]
    # groups: coordination-like classes from a 5.0 bohr bond cutoff, plus "no group" atoms
    pos, lat = sysd["pos"], sysd["lattice"]
    d = pos[:, None, :] - pos[None, :, :]
    d -= np.round(d / lat[0, 0]) * lat[0, 0]
    coord = ((np.sqrt((d ** 2).sum(-1)) < 5.0).sum(1) - 1)
    group = np.where(coord >= 4, 1, 0).astype(np.int32)
    group[::7] = -1
    with vgtb.Context(sysd, init=vgtb.INIT_USER, obs_stride=3) as c:
        for k, D in enumerate(gs["D"]):
            c.set_density(0, k, D)
        c.set_field(0, A)
        c.propagate(n)
        dq = c.group_charges(0, group, 2)
    lv = np.arange(0, n + 1, 3)
    ref = np.stack([-(ref_q[lv][:, group == g] - ref_q[0, group == g]).sum(1) for g in range(2)], 1)
    assert dq.shape == ref.shape
    assert np.abs(dq - ref).max() <= 1e-10
    assert np.abs(ref).max() > 1e-6


def test_laser_sweep_coordination_charge_transfer_matches_oracle():
    """The laser experiment of Sec. 3.3 in small: three photon energies as three
    trajectories of one context (FP64), charge transfer per coordination class
    (2.85 A bond cut-off) against the oracle's charges of each single run."""
    from paper_2308_09782_gb300 import inputs, vgtb
    sysd = inputs.diamond_si(2, 0.3, seed=64, kgrid="gamma")
    ctx = O.setup(sysd)
    gs = O.ground_state(sysd, ctx=ctx)
    fields, _ = inputs.laser_sweep(sysd["dt"])
    n = 250
    cn = inputs.coordination_numbers(sysd)
    classes = sorted(set(cn.tolist()))
    assert len(classes) >= 2                          # the displacements break some bonds
    group = np.array([classes.index(c) for c in cn], np.int32)
    with vgtb.Context([sysd], traj_sys=[0, 0, 0], init=vgtb.INIT_USER) as c:
        c.set_density(0, 0, gs["D"][0])
        for tr, f in enumerate(fields):
            c.set_field(tr, f[:n + 1])
        c.propagate(n)
        got = [c.group_charges(tr, group, len(classes)) for tr in range(3)]
    moved = []
    for tr, f in enumerate(fields):
        q = O.propagate(sysd, f[:n + 1], n, gs["D"], ctx=ctx)["q"]
        ref = np.stack([-(q[:, group == g] - q[0, group == g]).sum(1) for g in range(len(classes))], 1)
        assert np.abs(got[tr] - ref).max() <= 1e-10
        moved.append(np.abs(ref).max())
    assert min(moved) > 1e-7                          # every pulse moved charge
