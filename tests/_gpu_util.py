"""Shared helpers of the GPU parity tests (oracle references, error metrics)."""
import functools

import numpy as np

import oracle as O
from paper_2308_09782_gb300 import inputs


def rel_fro(a_list, b_list):
    """sqrt(sum ||a - b||_F^2) / sqrt(sum ||b||_F^2) over a list of matrices."""
    num = sum(np.linalg.norm(np.asarray(a) - np.asarray(b)) ** 2 for a, b in zip(a_list, b_list))
    den = sum(np.linalg.norm(np.asarray(b)) ** 2 for b in b_list)
    return float(np.sqrt(num / den))


@functools.lru_cache(maxsize=None)
def system(name):
    return inputs.config(name)


@functools.lru_cache(maxsize=None)
def oracle_ground(name):
    sysd, A, n = system(name)
    ctx = O.setup(sysd)
    gs = O.ground_state(sysd, ctx=ctx)
    return ctx, gs


@functools.lru_cache(maxsize=None)
def oracle_run(name, nsteps):
    sysd, A, n = system(name)
    ctx, gs = oracle_ground(name)
    return O.propagate(sysd, A, nsteps, gs["D"], ctx=ctx)


def gpu_run(name, nsteps, precision=0, init_user=True, **opts):
    from paper_2308_09782_gb300 import vgtb
    sysd, A, n = system(name)
    c = vgtb.Context(sysd, precision=precision, init=vgtb.INIT_USER if init_user else vgtb.INIT_GROUND, **opts)
    if init_user:
        _, gs = oracle_ground(name)
        for k, D in enumerate(gs["D"]):
            c.set_density(0, k, D)
    c.set_field(0, A[:nsteps + 1])
    c.propagate(nsteps)
    return c
