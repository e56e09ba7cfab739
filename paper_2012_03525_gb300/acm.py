"""Thin ctypes binding of libacm (include/acm.h).  Argument marshalling only:
every step of the solver runs in the library's CUDA kernels.  If the library
has not been built, importing the binding raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libacm.so")

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6
BC_PERIODIC, BC_WALL, BC_LID, BC_HALO, BC_SYMMETRY = 0, 1, 2, 3, 4
FP64, FP32_DEV = 0, 1
SCHEME_SMAMES, SCHEME_MAMES = 0, 1
TUNE_ZCHUNKS, TUNE_T3Y, TUNE_GRAPH_STEPS, TUNE_BLOCKS, TUNE_LINE2D = 1, 2, 3, 4, 5

#: every symbol include/acm.h declares (checked by the CPU tests)
EXPORTS = ["acm_create", "acm_batch_create", "acm_set_stream", "acm_nruns", "acm_set_fields",
           "acm_step", "acm_sync", "acm_fields", "acm_reduce_mass", "acm_set_tuning",
           "acm_step_count", "acm_destroy", "acm_last_error", "acm_get_tuning", "acm_autotune",
           "acm_restrict", "acm_closure_num_params", "acm_closure_create", "acm_closure_set_stream",
           "acm_closure_set_scales", "acm_closure_set_loss_weights", "acm_closure_set_weights", "acm_closure_get_weights",
           "acm_closure_forward", "acm_closure_loss_grad", "acm_closure_train_step",
           "acm_closure_gather", "acm_closure_apply", "acm_closure_destroy",
           "acm_closure_last_error", "acm_reduce_mass_noalloc",
           "acm_noalloc_last_error", "acm_storage_elems", "acm_create_ext",
           "acm_current_buffer", "acm_stability_ratio", "acm_reduce_error",
           "acm_reduce_laplace", "acm_closure_set_input_noise"]


class AcmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libacm status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dt", ctypes.c_double), ("nu", ctypes.c_double), ("rho0", ctypes.c_double),
        ("bc", ctypes.c_int * 6),
        ("lid_u", ctypes.c_double * 3), ("g", ctypes.c_double * 3),
        ("two_phase", ctypes.c_int),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double), ("M", ctypes.c_double),
        ("precision", ctypes.c_int), ("sat_mask", ctypes.c_int),
        ("theta_deg", ctypes.c_double),
        ("scheme", ctypes.c_int),
        ("rho_ratio", ctypes.c_double),
    ]


_lib = None


def load():
    """Load libacm.so (built by ``paper_2012_03525_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2012_03525_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    P = ctypes.POINTER(Params)
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "acm_create": ([P, ctypes.POINTER(H)], ctypes.c_int),
        "acm_batch_create": ([P, ctypes.c_int, ctypes.POINTER(H)], ctypes.c_int),
        "acm_set_stream": ([H, ctypes.c_void_p], ctypes.c_int),
        "acm_nruns": ([H], ctypes.c_int),
        "acm_set_fields": ([H, ctypes.c_int, dp, dp, dp, dp, dp], ctypes.c_int),
        "acm_step": ([H, ctypes.c_int64], ctypes.c_int),
        "acm_sync": ([H], ctypes.c_int),
        "acm_fields": ([H, ctypes.c_int, dp, dp, dp, dp, dp], ctypes.c_int),
        "acm_reduce_mass": ([H, dp], ctypes.c_int),
        "acm_set_tuning": ([H, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "acm_step_count": ([H], ctypes.c_int64),
        "acm_get_tuning": ([H, ctypes.c_int], ctypes.c_int),
        "acm_autotune": ([H, ctypes.c_int, dp], ctypes.c_int),
        "acm_destroy": ([H], ctypes.c_int),
        "acm_last_error": ([H], ctypes.c_char_p),
        "acm_reduce_mass_noalloc": ([ctypes.c_int] * 5 + [ctypes.c_double] +
                                    [ctypes.c_void_p] * 7 +
                                    [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
                                    ctypes.c_int),
        "acm_noalloc_last_error": ([], ctypes.c_char_p),
        "acm_storage_elems": ([P, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "acm_create_ext": ([P, ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                            ctypes.POINTER(H)], ctypes.c_int),
        "acm_current_buffer": ([H], ctypes.c_int),
        "acm_stability_ratio": ([P, dp, dp, dp, ctypes.c_size_t, dp], ctypes.c_int),
        "acm_reduce_error": ([H, ctypes.c_int, dp, dp, dp, dp], ctypes.c_int),
        "acm_reduce_laplace": ([H, dp], ctypes.c_int),
        "acm_restrict": ([H, H, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                          ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "acm_closure_num_params": ([], ctypes.c_size_t),
        "acm_closure_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "acm_closure_set_stream": ([H, ctypes.c_void_p], ctypes.c_int),
        "acm_closure_set_scales": ([H, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "acm_closure_set_loss_weights": ([H, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "acm_closure_set_input_noise": ([H, ctypes.c_float, ctypes.c_uint64], ctypes.c_int),
        "acm_closure_set_weights": ([H, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t],
                                    ctypes.c_int),
        "acm_closure_get_weights": ([H, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t],
                                    ctypes.c_int),
        "acm_closure_forward": ([H, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
        "acm_closure_loss_grad": ([H, ctypes.c_void_p, ctypes.c_void_p, dp,
                                   ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "acm_closure_train_step": ([H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, dp],
                                   ctypes.c_int),
        "acm_closure_gather": ([H, H, ctypes.c_void_p], ctypes.c_int),
        "acm_closure_apply": ([H, H], ctypes.c_int),
        "acm_closure_destroy": ([H], ctypes.c_int),
        "acm_closure_last_error": ([H], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def make_params(shape, dt=1.0, nu=0.01, rho0=1.0, bc=None, lid_u=(0, 0, 0), g=(0, 0, 0),
                two_phase=False, sigma=0.0, W=4.0, M=0.0, precision=FP64, sat_mask=3,
                theta_deg=90.0, scheme=SCHEME_SMAMES, rho_ratio=0.0) -> Params:
    """``shape`` is (ny, nx) for 2D or (nz, ny, nx) for 3D (array order)."""
    p = Params()
    if len(shape) == 2:
        p.dim, p.nz, (p.ny, p.nx) = 2, 1, shape
    else:
        p.dim, (p.nz, p.ny, p.nx) = 3, shape
    p.dt, p.nu, p.rho0 = dt, nu, rho0
    bc = [BC_PERIODIC] * 6 if bc is None else list(bc)
    for i in range(6):
        p.bc[i] = bc[i]
    for i in range(3):
        p.lid_u[i] = lid_u[i]
        p.g[i] = g[i]
    p.two_phase = int(bool(two_phase))
    p.sigma, p.W, p.M = sigma, W, M
    p.precision = precision
    p.sat_mask = sat_mask
    p.theta_deg = theta_deg
    p.scheme = scheme
    p.rho_ratio = rho_ratio
    return p


def subdomain_params(shape, nz_parts, **kw) -> list:
    """Parameters of a 3D periodic grid ``shape`` = (nz, ny, nx) split along z
    into slabs of ``nz_parts`` planes (summing to nz), for
    ``Solver(list_of_params)``: every slab gets ACM_BC_HALO z faces."""
    nz, ny, nx = shape
    if sum(nz_parts) != nz:
        raise ValueError("slab heights must sum to nz")
    out = []
    for n in nz_parts:
        p = make_params((n, ny, nx), **kw)
        p.bc[4] = p.bc[5] = BC_HALO
        out.append(p)
    return out


def _dptr(a):
    if a is None:
        return None
    if isinstance(a, int):  # raw (e.g. pinned) host address
        return ctypes.cast(ctypes.c_void_p(a), ctypes.POINTER(ctypes.c_double))
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def storage_elems(params: Params) -> int:
    """acm_storage_elems: elements per field buffer of a single-grid solver."""
    lib = load()
    n = ctypes.c_size_t(0)
    st = lib.acm_storage_elems(ctypes.byref(params), ctypes.byref(n))
    if st != OK:
        raise AcmError(st, lib.acm_last_error(None).decode())
    return n.value


def stability_ratio(params: Params, u, v, w=None) -> float:
    """acm_stability_ratio on host velocity arrays (> 1: expected to blow up)."""
    lib = load()
    r = ctypes.c_double(0.0)
    st = lib.acm_stability_ratio(ctypes.byref(params), _dptr(np.ascontiguousarray(u, np.float64)),
                                 _dptr(np.ascontiguousarray(v, np.float64)),
                                 None if w is None else _dptr(np.ascontiguousarray(w, np.float64)),
                                 int(np.asarray(u).size), ctypes.byref(r))
    if st != OK:
        raise AcmError(st, lib.acm_last_error(None).decode())
    return r.value


def reduce_mass_noalloc(dim, nx, ny, nz, precision, rho, u, v, w, prev, blocks, out_dev,
                        stream=0, rho0=0.0):
    """acm_reduce_mass_noalloc on caller-owned device buffers (raw device
    addresses as ints; ``prev`` = (u_prev, v_prev, w_prev) addresses or None;
    ``rho`` holds rho - rho0).  Raises AcmError on a non-zero status."""
    lib = load()
    pu, pv, pw = prev if prev is not None else (None, None, None)
    st = lib.acm_reduce_mass_noalloc(dim, nx, ny, nz, precision, float(rho0), rho, u, v, w,
                                     pu, pv, pw, blocks, out_dev, stream)
    if st != OK:
        raise AcmError(st, lib.acm_noalloc_last_error().decode())


class Solver:
    """One handle: a single grid (``Solver(params)``) or a batch
    (``Solver([params, ...])``).  ``ext_fields`` (10 device addresses,
    buffer-major, None for absent fields) and ``stream`` select
    acm_create_ext: the field storage then belongs to the caller."""

    def __init__(self, params, ext_fields=None, stream=0):
        lib = load()
        self._lib = lib
        self._h = ctypes.c_void_p()
        if ext_fields is not None:
            arr = (ctypes.c_void_p * 10)(*[0 if a is None else a for a in ext_fields])
            st = lib.acm_create_ext(ctypes.byref(params), arr, ctypes.c_void_p(stream),
                                    ctypes.byref(self._h))
            self.params = [params]
        elif isinstance(params, (list, tuple)):
            arr = (Params * len(params))(*params)
            st = lib.acm_batch_create(arr, len(params), ctypes.byref(self._h))
            self.params = list(params)
        else:
            st = lib.acm_create(ctypes.byref(params), ctypes.byref(self._h))
            self.params = [params]
        if st != OK:
            raise AcmError(st, lib.acm_last_error(None).decode())

    # -- helpers
    def _check(self, st):
        if st != OK:
            raise AcmError(st, self._lib.acm_last_error(self._h).decode())
        return st

    def shape(self, run=0):
        p = self.params[run]
        return (p.ny, p.nx) if p.dim == 2 else (p.nz, p.ny, p.nx)

    @property
    def nruns(self):
        return self._lib.acm_nruns(self._h)

    # -- API
    def set_stream(self, stream_ptr: int):
        self._check(self._lib.acm_set_stream(self._h, ctypes.c_void_p(stream_ptr)))

    def set_tuning(self, key: int, value: int):
        self._check(self._lib.acm_set_tuning(self._h, key, value))

    def get_tuning(self, key: int) -> int:
        return self._lib.acm_get_tuning(self._h, key)

    def autotune(self, nsteps: int = 20) -> float:
        """Pick the fastest launch shape (fields are left unchanged); returns
        the winner's milliseconds per step."""
        ms = ctypes.c_double(0.0)
        self._check(self._lib.acm_autotune(self._h, int(nsteps), ctypes.byref(ms)))
        return ms.value

    def set_fields(self, rho, u, v, w=None, phi=None, run=0):
        self._check(self._lib.acm_set_fields(self._h, run, _dptr(rho), _dptr(u), _dptr(v),
                                             _dptr(w), _dptr(phi)))

    def step(self, n=1):
        self._check(self._lib.acm_step(self._h, int(n)))

    def sync(self):
        return self._check(self._lib.acm_sync(self._h))

    def fields(self, run=0, out=None):
        """Returns (rho, u, v, w, phi) as float64 arrays (w/phi None when absent)."""
        p = self.params[run]
        shp = self.shape(run)
        if out is None:
            rho, u, v = np.empty(shp), np.empty(shp), np.empty(shp)
            w = np.empty(shp) if p.dim == 3 else None
            phi = np.empty(shp) if p.two_phase else None
        else:
            rho, u, v, w, phi = out
        self._check(self._lib.acm_fields(self._h, run, _dptr(rho), _dptr(u), _dptr(v), _dptr(w),
                                         _dptr(phi)))
        return rho, u, v, w, phi

    def fields_raw(self, run, ptrs):
        """Copy into caller-provided host addresses (ints or None)."""
        self._check(self._lib.acm_fields(self._h, run, *[_dptr(p) for p in ptrs]))

    def set_fields_raw(self, run, ptrs):
        self._check(self._lib.acm_set_fields(self._h, run, *[_dptr(p) for p in ptrs]))

    def reduce(self):
        out = np.zeros(8 * self.nruns)
        self._check(self._lib.acm_reduce_mass(self._h, _dptr(out)))
        return out.reshape(self.nruns, 8) if self.nruns > 1 else out

    def reduce_error(self, u_ref, v_ref, w_ref=None, run=0):
        """Eq. (3.2) relative L2 error of each velocity component against the
        host reference fields (acm_reduce_error); 0 for a None reference."""
        out = np.zeros(3)
        refs = [None if a is None else np.ascontiguousarray(a, np.float64)
                for a in (u_ref, v_ref, w_ref)]
        self._check(self._lib.acm_reduce_error(self._h, run, *[_dptr(a) for a in refs],
                                               _dptr(out)))
        return out

    def reduce_laplace(self):
        """acm_reduce_laplace: per run [A, R_eff, mu_G, mu_in, mu_out,
        p_in - p_out, (dim - 1) sigma / (2 R_eff), n_in]."""
        out = np.zeros(8 * self.nruns)
        self._check(self._lib.acm_reduce_laplace(self._h, _dptr(out)))
        return out.reshape(self.nruns, 8) if self.nruns > 1 else out

    def current_buffer(self):
        return self._lib.acm_current_buffer(self._h)

    def last_error(self):
        return self._lib.acm_last_error(self._h).decode()

    def restrict_to(self, coarse=None, factor=4, out_dev=None, scales=(1.0, 1.0), u_scale=None,
                    rho_scale=None):
        """Box-filter this (fine) handle's runs into ``coarse`` and/or a
        normalised device buffer (acm_restrict); by default the lattice units
        change with delta_x (u / factor, rho' / factor^2)."""
        us = 1.0 / factor if u_scale is None else u_scale
        rs = 1.0 / factor ** 2 if rho_scale is None else rho_scale
        sc = (ctypes.c_float * 3)(scales[0], scales[1], scales[1])
        self._check(self._lib.acm_restrict(self._h, coarse._h if coarse is not None else None,
                                           factor, us, rs,
                                           ctypes.c_void_p(out_dev) if out_dev else None, sc))

    def step_count(self):
        return self._lib.acm_step_count(self._h)

    def close(self):
        if self._h:
            self._lib.acm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Closure:
    """The learned closure (acm_closure_*): device tensors are passed as raw
    device addresses (ints), host weight vectors as NumPy float32 arrays."""

    def __init__(self, nx, ny, batch):
        lib = load()
        self._lib = lib
        self._c = ctypes.c_void_p()
        st = lib.acm_closure_create(nx, ny, batch, ctypes.byref(self._c))
        if st != OK:
            raise AcmError(st, lib.acm_closure_last_error(None).decode())
        self.nx, self.ny, self.batch = nx, ny, batch
        self.nparams = lib.acm_closure_num_params()

    def _check(self, st):
        if st != OK:
            raise AcmError(st, self._lib.acm_closure_last_error(self._c).decode())

    def set_stream(self, stream_ptr):
        self._check(self._lib.acm_closure_set_stream(self._c, ctypes.c_void_p(stream_ptr)))

    def set_scales(self, s_rho, s_u):
        arr = (ctypes.c_float * 3)(s_rho, s_u, s_u)
        self._check(self._lib.acm_closure_set_scales(self._c, arr))

    def set_loss_weights(self, w_rho, w_u):
        arr = (ctypes.c_float * 3)(w_rho, w_u, w_u)
        self._check(self._lib.acm_closure_set_loss_weights(self._c, arr))

    def set_input_noise(self, sigma, seed=0):
        self._check(self._lib.acm_closure_set_input_noise(self._c, float(sigma), int(seed)))

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        self._check(self._lib.acm_closure_set_weights(
            self._c, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), w.size))

    def get_weights(self):
        w = np.empty(self.nparams, dtype=np.float32)
        self._check(self._lib.acm_closure_get_weights(
            self._c, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), w.size))
        return w

    def forward(self, x_dev, net_dev):
        self._check(self._lib.acm_closure_forward(self._c, ctypes.c_void_p(x_dev),
                                                  ctypes.c_void_p(net_dev)))

    def loss_grad(self, x_dev, target_dev):
        loss = ctypes.c_double(0.0)
        g = np.empty(self.nparams, dtype=np.float32)
        self._check(self._lib.acm_closure_loss_grad(
            self._c, ctypes.c_void_p(x_dev), ctypes.c_void_p(target_dev), ctypes.byref(loss),
            g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return loss.value, g

    def train_step(self, x_dev, target_dev, lr, want_loss=True):
        loss = ctypes.c_double(0.0)
        self._check(self._lib.acm_closure_train_step(
            self._c, ctypes.c_void_p(x_dev), ctypes.c_void_p(target_dev), ctypes.c_float(lr),
            ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def gather(self, solver, x_dev):
        self._check(self._lib.acm_closure_gather(self._c, solver._h, ctypes.c_void_p(x_dev)))

    def apply(self, solver):
        self._check(self._lib.acm_closure_apply(self._c, solver._h))

    def close(self):
        if self._c:
            self._lib.acm_closure_destroy(self._c)
            self._c = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
