"""512-atom kick at the stated step count against the stored oracle run.

tests/golden/si512_kick_oracle.npz is written by tests/golden/make_oracle_reference.py
(oracle only: SCC ground state, then 5000 leapfrog steps; J and E at every level, q every
250 steps, and a record of the final density matrix: its diagonal atom blocks and the
entries at a seeded sample of 16384 positions).  The FP64 path runs all 5000 steps from
the oracle's ground state (targets: rho <= 1e-10 on the stored entries, J <= 1e-8); the
split form runs all 5000 steps from the library's own ground state (J within 1e-4 of
the FP64 oracle, the bound of the split-precision form).
"""
import os

import numpy as np
import pytest

from tests._gpu_util import oracle_ground, rel_fro, system

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "si512_kick_oracle.npz")


@pytest.fixture(scope="module")
def gold():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2308_09782_gb300 import vgtb
    vgtb.load()
    return dict(np.load(GOLD))


def final_density_errors(D, gold, sysd):
    """Relative errors of the final density on the stored entries: the diagonal
    atom blocks and the seeded sample (sqrt(sum |dD|^2) / sqrt(sum |D|^2) each)."""
    off = np.asarray(sysd["orb_offset"])
    diag = np.concatenate([D[off[i]:off[i + 1], off[i]:off[i + 1]].ravel() for i in range(len(off) - 1)])
    samp = D[gold["d_rows"], gold["d_cols"]]
    e_diag = np.linalg.norm(diag - gold["d_diag"]) / np.linalg.norm(gold["d_diag"])
    e_samp = np.linalg.norm(samp - gold["d_sample"]) / np.linalg.norm(gold["d_sample"])
    return e_diag, e_samp


def test_split_512_kick_full_run_vs_stored_oracle(gold):
    from paper_2308_09782_gb300 import vgtb
    sysd, A, n = system("si512_kick")
    assert int(gold["nsteps"]) == n
    with vgtb.Context(sysd, precision=vgtb.SPLIT_BF16X3, init=vgtb.INIT_GROUND, obs_stride=250) as c:
        c.set_field(0, A)
        c.propagate(0)
        _, _, q0 = c.observables(0)
        assert np.abs((q0[0] - sysd["z_ref"]) - gold["dq0"]).max() <= 1e-8
        c.propagate(n)
        J, E, q = c.observables(0)
        D = c.get_density(0, 0)
    err_j = rel_fro([J], [gold["J"]])
    err_e = np.abs(E - gold["E"]).max() / np.abs(gold["E"]).max()
    err_q = np.abs(q - gold["q"]).max()
    nel_drift = np.abs(q.sum(axis=1) - sysd["n_electrons"]).max()
    e_diag, e_samp = final_density_errors(D, gold, sysd)
    print(f"si512_kick split, {n} steps: J {err_j:.2e}  E {err_e:.2e}  q {err_q:.2e}  "
          f"sum q - N_el {nel_drift:.2e}  rho diag {e_diag:.2e}  rho sample {e_samp:.2e}")
    assert err_j <= 1e-4
    assert err_e <= 1e-6
    assert err_q <= 1e-5
    assert nel_drift <= 1e-6
    assert e_diag <= 1e-4 and e_samp <= 1e-4


def test_fp64_512_kick_full_run_vs_stored_oracle(gold):
    """The plain FP64 path over the whole stated run (5000 steps) from the oracle's
    ground state: J, E and q at the stored levels, and the final density matrix on
    its stored entries."""
    from paper_2308_09782_gb300 import vgtb
    sysd, A, n = system("si512_kick")
    _, gs = oracle_ground("si512_kick")
    with vgtb.Context(sysd, precision=vgtb.FP64, init=vgtb.INIT_USER, obs_stride=250) as c:
        c.set_density(0, 0, gs["D"][0])
        c.set_field(0, A)
        c.propagate(n)
        J, E, q = c.observables(0)
        D = c.get_density(0, 0)
    err_j = rel_fro([J], [gold["J"]])
    err_e = np.abs(E - gold["E"]).max() / np.abs(gold["E"]).max()
    err_q = np.abs(q - gold["q"]).max()
    e_diag, e_samp = final_density_errors(D, gold, sysd)
    print(f"si512_kick FP64, {n} steps: J {err_j:.2e}  E {err_e:.2e}  q {err_q:.2e}  "
          f"rho diag {e_diag:.2e}  rho sample {e_samp:.2e}")
    assert err_j <= 1e-8
    assert err_e <= 1e-9
    assert err_q <= 1e-10
    assert e_diag <= 1e-10 and e_samp <= 1e-10
