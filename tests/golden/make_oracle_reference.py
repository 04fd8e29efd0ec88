"""Write stored oracle results for workloads too long to rerun inside a test.

Calls only ``oracle/`` and the seeded input generator.  Usage:

    python tests/golden/make_oracle_reference.py si512_kick [nsteps]

writes ``tests/golden/<config>_oracle.npz`` with the SCC ground-state charges
dq0, the current J(t_n) (n = 0..nsteps, 3 components), the energy E(t_n), the
Mulliken charges q(t_n) every 250 steps and a record of the final density
matrix D(t_nsteps) of the first k-point: its diagonal atom blocks (``d_diag``,
atom by atom, row-major), the entries at a seeded uniform sample of positions
(``d_rows``, ``d_cols``, ``d_sample``) and its Frobenius norm (``d_fro``).
The full N x N matrix is too large to store.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2308_09782_gb300 import inputs  # noqa: E402


def main():
    name = sys.argv[1]
    sysd, A, nsteps = inputs.config(name)
    if len(sys.argv) > 2:
        nsteps = int(sys.argv[2])
    t0 = time.time()
    ctx = O.setup(sysd)
    gs = O.ground_state(sysd, ctx=ctx)
    print(f"ground state: {gs['iters']} iterations, residual {gs['residual']:.2e}, "
          f"gap {gs['gap']:.4f} Ha, {time.time() - t0:.0f} s", flush=True)
    stride = 250
    J, E, qs, qsteps = [], [], [], []
    D, Dp = gs["D"], None
    n = 0
    while n < nsteps:
        m = min(stride, nsteps - n)
        r = O.propagate(sysd, A, m, D, ctx=ctx, D_prev_list=Dp, n0=n)
        J.append(r["J"][:-1])
        E.append(r["E"][:-1])
        qs.append(r["q"][0])
        qsteps.append(n)
        D, Dp = r["D"], r["D_prev"]
        n += m
        print(f"step {n}/{nsteps}  {time.time() - t0:.0f} s  J_x={r['J'][-1][0]:.6e}", flush=True)
    r = O.propagate(sysd, A, 0, D, ctx=ctx, D_prev_list=Dp, n0=n)
    J.append(r["J"])
    E.append(r["E"])
    qs.append(r["q"][0])
    qsteps.append(n)
    Df = np.asarray(D[0])
    off = np.asarray(sysd["orb_offset"])
    d_diag = np.concatenate([Df[off[i]:off[i + 1], off[i]:off[i + 1]].ravel()
                             for i in range(len(off) - 1)])
    rng = np.random.default_rng(20230818)
    n_orb = Df.shape[0]
    rows = rng.integers(0, n_orb, size=16384).astype(np.int32)
    cols = rng.integers(0, n_orb, size=16384).astype(np.int32)
    out = os.environ.get("VGTB_GOLDEN_OUT") or os.path.join(HERE, f"{name}_oracle.npz")
    np.savez_compressed(out, dq0=gs["dq"], J=np.concatenate(J), E=np.concatenate(E),
                        q=np.array(qs), q_steps=np.array(qsteps), nsteps=nsteps,
                        d_diag=d_diag, d_rows=rows, d_cols=cols, d_sample=Df[rows, cols],
                        d_fro=np.linalg.norm(Df))
    print("wrote", out)


if __name__ == "__main__":
    main()
