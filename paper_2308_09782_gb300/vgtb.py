"""ctypes binding of libvgtb (include/vgtb.h): argument marshalling only.

Every step of the propagation runs inside the library's CUDA kernels; this
module converts numpy arrays and system dictionaries (see ``inputs``) into the
C structs and calls the entry points of the same names.  ``load()`` raises
when the library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvgtb.so")

VGTB_OK = 0
ERRORS = {-1: "E_INVALID", -2: "E_NOT_PD", -3: "E_NO_GAP", -4: "E_CUDA", -5: "E_NOMEM",
          -6: "E_STATE", -7: "E_UNSTABLE", -8: "E_TIMEOUT", -9: "E_NO_CONVERGE",
          -10: "E_UNSUPPORTED"}
FP64 = 0
SPLIT_BF16X3 = 1
INIT_GROUND = 0
INIT_USER = 1
LEAPFROG = 0
CRANK_NICOLSON = 1
P1_AUTO = 0
P1_DENSE = 1
P1_BLOCKS = 2
SCC_ON = 0
SCC_FROZEN = 1
CHAIN_AUTO = 0
CHAIN_OFF = 1
CHAIN_ON = 2
KERNEL_CLASSES = ["obs", "scc", "phase", "gemm1", "gemm2", "leap"]

EXPORTS = ["vgtb_default_options", "vgtb_create", "vgtb_create_batch", "vgtb_set_density",
           "vgtb_set_field", "vgtb_propagate", "vgtb_steps_done", "vgtb_observables",
           "vgtb_get_density", "vgtb_get_initial_density", "vgtb_state_size", "vgtb_get_state", "vgtb_set_state",
           "vgtb_profile", "vgtb_kernel_stats", "vgtb_last_error", "vgtb_destroy",
           "vgtb_diag_split_chain", "vgtb_split_cgemm_noalloc", "vgtb_spectrum", "vgtb_group_charges",
           "vgtb_set_coefficients", "vgtb_get_coefficients", "vgtb_tile_config",
           "vgtb_diag_split_chain_variant", "vgtb_diag_num_variants", "vgtb_diag_convert",
           "vgtb_diag_bounded_wait"]


class VgtbSystem(C.Structure):
    _fields_ = [("lattice", C.c_double * 9), ("n_atoms", C.c_int), ("pos", C.POINTER(C.c_double)),
                ("orb_offset", C.POINTER(C.c_int)), ("z_ref", C.POINTER(C.c_double)),
                ("n_blocks", C.c_int), ("blk_ijl", C.POINTER(C.c_int)),
                ("h0", C.POINTER(C.c_double)), ("s", C.POINTER(C.c_double)),
                ("ds", C.POINTER(C.c_double)), ("gamma", C.POINTER(C.c_double)),
                ("n_k", C.c_int), ("kpt", C.POINTER(C.c_double)), ("wk", C.POINTER(C.c_double)),
                ("n_electrons", C.c_double), ("dt", C.c_double)]


class VgtbOptions(C.Structure):
    _fields_ = [("precision", C.c_int), ("delta_form", C.c_int), ("init", C.c_int),
                ("cuda_stream", C.c_void_p), ("timeout_ns", C.c_longlong),
                ("obs_stride", C.c_int), ("graph_steps", C.c_int), ("autotune", C.c_int),
                ("scc_tol", C.c_double), ("scc_max_iter", C.c_int),
                ("integrator", C.c_int), ("cn_iter", C.c_int), ("cn_tol", C.c_double),
                ("tile_variant", C.c_int * 2), ("product1", C.c_int), ("scc", C.c_int),
                ("chain", C.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libvgtb.so and declare its signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libvgtb.so not found at {path}: build it with "
                           "`python -m paper_2308_09782_gb300.build`")
    lib = C.CDLL(path)
    P, I, D, V = C.POINTER, C.c_int, C.c_double, C.c_void_p
    ctxp = V
    lib.vgtb_default_options.argtypes = [P(VgtbOptions)]
    lib.vgtb_default_options.restype = None
    lib.vgtb_create.argtypes = [P(ctxp), P(VgtbSystem), P(VgtbOptions)]
    lib.vgtb_create_batch.argtypes = [P(ctxp), I, P(VgtbSystem), I, P(I), P(VgtbOptions)]
    lib.vgtb_set_density.argtypes = [ctxp, I, I, P(D)]
    lib.vgtb_set_field.argtypes = [ctxp, I, I, P(D)]
    lib.vgtb_propagate.argtypes = [ctxp, I]
    lib.vgtb_steps_done.argtypes = [ctxp]
    lib.vgtb_observables.argtypes = [ctxp, I, P(D), P(D), P(D)]
    lib.vgtb_get_density.argtypes = [ctxp, I, I, P(D)]
    lib.vgtb_get_initial_density.argtypes = [ctxp, I, I, P(D)]
    lib.vgtb_state_size.argtypes = [ctxp]
    lib.vgtb_state_size.restype = C.c_longlong
    lib.vgtb_get_state.argtypes = [ctxp, V, C.c_longlong]
    lib.vgtb_set_state.argtypes = [ctxp, V, C.c_longlong]
    lib.vgtb_profile.argtypes = [ctxp, I]
    lib.vgtb_kernel_stats.argtypes = [ctxp, P(C.c_longlong), P(D), I]
    lib.vgtb_last_error.argtypes = [ctxp]
    lib.vgtb_last_error.restype = C.c_char_p
    lib.vgtb_destroy.argtypes = [ctxp]
    lib.vgtb_destroy.restype = None
    lib.vgtb_diag_split_chain.argtypes = [I, P(D), P(D), P(D), P(D), P(D)]
    lib.vgtb_split_cgemm_noalloc.argtypes = [I, V, V, V, V]
    lib.vgtb_spectrum.argtypes = [ctxp, I, I, I, D, D, I, P(D), P(D), P(D)]
    lib.vgtb_group_charges.argtypes = [ctxp, I, I, P(I), P(D)]
    lib.vgtb_set_coefficients.argtypes = [ctxp, I, I, I, P(D)]
    lib.vgtb_get_coefficients.argtypes = [ctxp, I, I, P(D)]
    lib.vgtb_tile_config.argtypes = [ctxp, I, P(I)]
    lib.vgtb_diag_split_chain_variant.argtypes = [I, P(D), P(D), P(D), I, P(D), P(D)]
    lib.vgtb_diag_num_variants.argtypes = []
    lib.vgtb_diag_bounded_wait.argtypes = [C.c_longlong, I]
    lib.vgtb_diag_convert.argtypes = [I, P(D), P(C.c_float), P(C.c_float), P(C.c_float), P(D), P(D)]
    for name in EXPORTS:
        if name not in ("vgtb_default_options", "vgtb_last_error", "vgtb_destroy", "vgtb_state_size"):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


class VgtbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def make_system(sysd: dict):
    """Build a VgtbSystem from an input dictionary; returns (struct, keepalive)."""
    keep = {
        "pos": np.ascontiguousarray(sysd["pos"], np.float64),
        "orb": np.ascontiguousarray(sysd["orb_offset"], np.int32),
        "z": np.ascontiguousarray(sysd["z_ref"], np.float64),
        "ijl": np.ascontiguousarray(sysd["blk_ijl"], np.int32),
        "h0": np.ascontiguousarray(sysd["h0"], np.float64),
        "s": np.ascontiguousarray(sysd["s"], np.float64),
        "ds": np.ascontiguousarray(sysd["ds"], np.float64),
        "gamma": np.ascontiguousarray(sysd["gamma"], np.float64),
        "kpt": np.ascontiguousarray(sysd["kpt"], np.float64),
        "wk": np.ascontiguousarray(sysd["wk"], np.float64),
    }
    st = VgtbSystem()
    st.lattice = (C.c_double * 9)(*np.asarray(sysd["lattice"], float).ravel())
    st.n_atoms = len(keep["z"])
    st.pos = _dptr(keep["pos"])
    st.orb_offset = _iptr(keep["orb"])
    st.z_ref = _dptr(keep["z"])
    st.n_blocks = keep["ijl"].shape[0]
    st.blk_ijl = _iptr(keep["ijl"])
    st.h0 = _dptr(keep["h0"])
    st.s = _dptr(keep["s"])
    st.ds = _dptr(keep["ds"])
    st.gamma = _dptr(keep["gamma"])
    st.n_k = keep["kpt"].shape[0]
    st.kpt = _dptr(keep["kpt"])
    st.wk = _dptr(keep["wk"])
    st.n_electrons = float(sysd["n_electrons"])
    st.dt = float(sysd["dt"])
    return st, keep


def default_options(**kw) -> VgtbOptions:
    lib = load()
    o = VgtbOptions()
    lib.vgtb_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        if k == "tile_variant":
            o.tile_variant[0], o.tile_variant[1] = int(v[0]), int(v[1])
        else:
            setattr(o, k, v)
    return o


def diag_split_chain(a, r, s, variant: int = -1):
    """Run the two tcgen05 split-precision products on host matrices:
    W = a r^dagger and X = s W^dagger, with tile variant `variant` (-1 = default).
    Returns (W, X) as complex128 arrays."""
    lib = load()
    a, r, s = (np.ascontiguousarray(x, np.complex128) for x in (a, r, s))
    n = a.shape[0]
    w = np.zeros((n, n), np.complex128)
    x = np.zeros((n, n), np.complex128)
    cp = lambda m: m.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
    rc = lib.vgtb_diag_split_chain_variant(n, cp(a), cp(r), cp(s), int(variant), cp(w), cp(x))
    if rc != VGTB_OK:
        raise VgtbError(rc, "vgtb_diag_split_chain_variant failed")
    return w, x


def diag_convert(d_in, f_in):
    """The library's bit-operation conversions next to CUDA's on the device.
    Returns (d2f_bits(d_in), __double2float_rn(d_in), f2d_bits(f_in), double(f_in))."""
    lib = load()
    d_in = np.ascontiguousarray(d_in, np.float64)
    f_in = np.ascontiguousarray(f_in, np.float32)
    assert d_in.shape == f_in.shape and d_in.ndim == 1
    n = d_in.shape[0]
    fb, fr = np.zeros(n, np.float32), np.zeros(n, np.float32)
    db, dr = np.zeros(n), np.zeros(n)
    fp = lambda m: m.ctypes.data_as(C.POINTER(C.c_float))  # noqa: E731
    rc = lib.vgtb_diag_convert(n, _dptr(d_in), fp(f_in), fp(fb), fp(fr), _dptr(db), _dptr(dr))
    if rc != VGTB_OK:
        raise VgtbError(rc, "vgtb_diag_convert failed")
    return fb, fr, db, dr


def num_tile_variants() -> int:
    return load().vgtb_diag_num_variants()


class Context:
    """One library context (vgtb_ctx) over one or several systems/trajectories."""

    def __init__(self, systems, traj_sys=None, **opts):
        lib = load()
        if isinstance(systems, dict):
            systems = [systems]
        self._sysd = list(systems)
        self.n_traj = len(traj_sys) if traj_sys is not None else 1
        traj_sys = np.ascontiguousarray(traj_sys if traj_sys is not None else [0], np.int32)
        built = [make_system(s) for s in systems]
        arr = (VgtbSystem * len(built))(*[b[0] for b in built])
        self._opt = default_options(**opts)
        h = C.c_void_p()
        rc = lib.vgtb_create_batch(C.byref(h), len(built), arr, len(traj_sys), _iptr(traj_sys),
                                   C.byref(self._opt))
        if rc != VGTB_OK:
            raise VgtbError(rc, lib.vgtb_last_error(None).decode())
        self._h = h
        self._traj_sys = traj_sys
        self.nat = [len(s["z_ref"]) for s in systems]
        self.N = [int(s["orb_offset"][-1]) for s in systems]
        self.nk = [len(s["wk"]) for s in systems]

    def _check(self, rc):
        if rc != VGTB_OK:
            raise VgtbError(rc, load().vgtb_last_error(self._h).decode())

    def set_density(self, sys_index: int, k: int, d0):
        d = np.ascontiguousarray(d0, np.complex128)
        self._check(load().vgtb_set_density(self._h, sys_index, k, d.ctypes.data_as(C.POINTER(C.c_double))))

    def set_coefficients(self, sys_index: int, k: int, c):
        """Crank-Nicolson start: occupied states C_k(0), shape [N, n_occ] (column n = state n)."""
        a = np.ascontiguousarray(c, np.complex128)
        self._check(load().vgtb_set_coefficients(self._h, sys_index, k, a.shape[1],
                                                 a.ctypes.data_as(C.POINTER(C.c_double))))

    def get_coefficients(self, traj: int, k: int, n_occ: int):
        """Crank-Nicolson: C_k(t_n) of trajectory `traj`, shape [N, n_occ]."""
        s = int(self._traj_sys[traj])
        out = np.zeros((self.N[s], n_occ), np.complex128)
        self._check(load().vgtb_get_coefficients(self._h, traj, k, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def set_field(self, traj: int, A):
        a = np.ascontiguousarray(A, np.float64)
        self._check(load().vgtb_set_field(self._h, traj, a.shape[0], _dptr(a)))

    def propagate(self, nsteps: int):
        self._check(load().vgtb_propagate(self._h, int(nsteps)))

    @property
    def steps_done(self) -> int:
        return load().vgtb_steps_done(self._h)

    def observables(self, traj: int = 0, charges: bool = True):
        n = self.steps_done
        s = int(self._traj_sys[traj])
        J = np.zeros((n + 1, 3))
        E = np.zeros(n + 1)
        stride = self._opt.obs_stride
        q = np.zeros((n // stride + 1, self.nat[s])) if charges else None
        self._check(load().vgtb_observables(self._h, traj, _dptr(J), _dptr(E),
                                            _dptr(q) if charges else None))
        return J, E, q

    def observables_into(self, traj: int, J, E, q=None):
        """Copy the series into caller arrays (e.g. pinned host memory)."""
        self._check(load().vgtb_observables(self._h, traj, _dptr(J), _dptr(E),
                                            _dptr(q) if q is not None else None))

    def spectrum(self, traj: int, e0: float, omegas, n0: int = 0, n1: int | None = None, tau0: float = 200.0):
        """sigma(w), eps(w) [n_omega, 3] complex of Eqs. 15-16 from the device J series."""
        w = np.ascontiguousarray(omegas, np.float64)
        n1 = self.steps_done if n1 is None else n1
        sig = np.zeros((len(w), 3), np.complex128)
        eps = np.zeros((len(w), 3), np.complex128)
        cp = lambda m: m.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
        self._check(load().vgtb_spectrum(self._h, traj, n0, n1, float(e0), float(tau0), len(w), _dptr(w),
                                         cp(sig), cp(eps)))
        return sig, eps

    def group_charges(self, traj: int, group, n_groups: int):
        """dQ_g(t_n) = sum_{I in g} (Q_I(t_n) - Q_I(t_0)), Q_I = -(q_I - Z_I), [n_levels, n_groups]."""
        g = np.ascontiguousarray(group, np.int32)
        nlev = self.steps_done // self._opt.obs_stride + 1
        out = np.zeros((nlev, n_groups))
        self._check(load().vgtb_group_charges(self._h, traj, n_groups, _iptr(g), _dptr(out)))
        return out

    def get_initial_density(self, sys_index: int, k: int):
        out = np.zeros((self.N[sys_index], self.N[sys_index]), np.complex128)
        self._check(load().vgtb_get_initial_density(self._h, sys_index, k,
                                                    out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def get_density(self, traj: int, k: int):
        s = int(self._traj_sys[traj])
        out = np.zeros((self.N[s], self.N[s]), np.complex128)
        self._check(load().vgtb_get_density(self._h, traj, k, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def get_state(self) -> bytes:
        lib = load()
        n = lib.vgtb_state_size(self._h)
        buf = C.create_string_buffer(n)
        self._check(lib.vgtb_get_state(self._h, buf, n))
        return buf.raw

    def set_state(self, state: bytes):
        buf = C.create_string_buffer(state, len(state))
        self._check(load().vgtb_set_state(self._h, buf, len(state)))

    def profile(self, enable: bool = True):
        self._check(load().vgtb_profile(self._h, 1 if enable else 0))

    def tile_config(self, product: int):
        """{"tile_n", "stages", "schedule", "pair"} of tcgen05 product 1 or 2 (split contexts)."""
        cfg = (C.c_int * 4)()
        self._check(load().vgtb_tile_config(self._h, int(product), cfg))
        if cfg[2] == 3:
            return {"schedule": "block-sparse", "atoms_per_group": cfg[0], "rows_per_cta": cfg[1]}
        base = ("classic", "stream-K", "classic waves + stream-K")[cfg[2] & 3]
        if cfg[2] & 8:
            base += ", planned column widths"
        if cfg[2] & 4:
            base += ", zero k-panels skipped"
        if cfg[2] & 16:
            base += ", both products in one launch"
        return {"tile_n": cfg[0], "stages": cfg[1], "schedule": base, "pair": bool(cfg[3])}

    def kernel_stats(self):
        n = len(KERNEL_CLASSES)
        la = (C.c_longlong * n)()
        ms = (C.c_double * n)()
        load().vgtb_kernel_stats(self._h, la, ms, n)
        return {k: (int(la[i]), float(ms[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def close(self):
        if getattr(self, "_h", None):
            load().vgtb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
