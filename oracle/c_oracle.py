"""ctypes binding of the C oracle (``acm_oracle.c``).  Test infrastructure only.

The shared object is built with gcc on first use (or by ``build()`` in the
repository's entry module) into ``oracle/_build/``.  Every function here takes
and returns NumPy float64 arrays in [z][y][x] layout (x fastest).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "acm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC, WALL, LID, SYMMETRY = 0, 1, 2, 4


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dt", ctypes.c_double), ("nu", ctypes.c_double), ("rho0", ctypes.c_double),
        ("bc", ctypes.c_int * 6),
        ("lid_u", ctypes.c_double * 3), ("g", ctypes.c_double * 3),
        ("two_phase", ctypes.c_int),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double), ("M", ctypes.c_double),
        ("sat_mask", ctypes.c_int),
        ("theta_deg", ctypes.c_double),
        ("rho_ratio", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FMA contraction off).  Returns the .so path."""
    with _lock:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-shared",
            "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
        return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(OracleParams)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_step.argtypes = [P, dp, dp, dp, dp, dp, ctypes.c_long]
        lib.oracle_step.restype = ctypes.c_int
        lib.oracle_chem_pot.argtypes = [P, dp, dp]
        lib.oracle_chem_pot.restype = ctypes.c_int
        lib.oracle_grad_lap_iso.argtypes = [P, dp, ctypes.c_int, dp, dp]
        lib.oracle_grad_lap_iso.restype = ctypes.c_int
        lib.oracle_step_mames.argtypes = [P, dp, dp, dp, dp, ctypes.c_long]
        lib.oracle_step_mames.restype = ctypes.c_int
        lib.oracle_reduce.argtypes = [P, dp, dp, dp, dp, dp, dp, dp, dp]
        lib.oracle_reduce.restype = ctypes.c_int
        _lib = lib
    return _lib


def make_params(shape, dt=1.0, nu=0.01, rho0=1.0, bc=None, lid_u=(0, 0, 0), g=(0, 0, 0),
                two_phase=False, sigma=0.0, W=4.0, M=0.0, sat_mask=3,
                theta_deg=90.0, rho_ratio=0.0) -> OracleParams:
    """``shape`` is (ny, nx) for 2D or (nz, ny, nx) for 3D (array order)."""
    p = OracleParams()
    if len(shape) == 2:
        p.dim, p.nz, (p.ny, p.nx) = 2, 1, shape
    else:
        p.dim, (p.nz, p.ny, p.nx) = 3, shape
    p.dt, p.nu, p.rho0 = dt, nu, rho0
    bc = [PERIODIC] * 6 if bc is None else list(bc)
    for i in range(6):
        p.bc[i] = bc[i]
    for i in range(3):
        p.lid_u[i] = lid_u[i]
        p.g[i] = g[i]
    p.two_phase = int(bool(two_phase))
    p.sigma, p.W, p.M = sigma, W, M
    p.sat_mask = sat_mask
    p.theta_deg = theta_deg
    p.rho_ratio = rho_ratio
    return p


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def step(p: OracleParams, rho, u, v, w=None, phi=None, nsteps: int = 1):
    """Advance the state IN PLACE by ``nsteps`` steps.  Missing w/phi are zeros."""
    lib = _load()
    shape = rho.shape
    w = np.zeros(shape) if w is None else w
    phi = np.zeros(shape) if phi is None else phi
    rc = lib.oracle_step(ctypes.byref(p), _ptr(rho), _ptr(u), _ptr(v), _ptr(w), _ptr(phi),
                         int(nsteps))
    if rc != 0:
        raise ValueError(f"oracle_step failed with status {rc}")
    return rho, u, v, w, phi


def step_mames(p: OracleParams, rho, u, v, w=None, nsteps: int = 1):
    """Advance IN PLACE by ``nsteps`` steps of the MAMEs predictor-corrector
    (Eqs. 2.6-2.9), periodic single-phase grids only."""
    lib = _load()
    w = np.zeros(rho.shape) if w is None else w
    rc = lib.oracle_step_mames(ctypes.byref(p), _ptr(rho), _ptr(u), _ptr(v), _ptr(w),
                               int(nsteps))
    if rc != 0:
        raise ValueError(f"oracle_step_mames failed with status {rc}")
    return rho, u, v, w


def chem_pot(p: OracleParams, phi):
    lib = _load()
    mu = np.empty_like(phi)
    if lib.oracle_chem_pot(ctypes.byref(p), _ptr(phi), _ptr(mu)) != 0:
        raise ValueError("oracle_chem_pot failed")
    return mu


def grad_lap_iso(p: OracleParams, f, d: int):
    lib = _load()
    gr = np.empty_like(f)
    la = np.empty_like(f)
    if lib.oracle_grad_lap_iso(ctypes.byref(p), _ptr(f), int(d), _ptr(gr), _ptr(la)) != 0:
        raise ValueError("oracle_grad_lap_iso failed")
    return gr, la


def reduce(p: OracleParams, rho, u, v, w=None, prev=None):
    """Returns the 8 diagnostics (see ``oracle_reduce`` in acm_oracle.c)."""
    lib = _load()
    w = np.zeros_like(rho) if w is None else w
    out = (ctypes.c_double * 8)()
    up = vp = wp = None
    if prev is not None:
        up, vp = prev[0], prev[1]
        wp = prev[2] if len(prev) > 2 and prev[2] is not None else np.zeros_like(rho)
    rc = lib.oracle_reduce(ctypes.byref(p), _ptr(rho), _ptr(u), _ptr(v), _ptr(w),
                           _ptr(up), _ptr(vp), _ptr(wp), out)
    if rc != 0:
        raise ValueError("oracle_reduce failed")
    return np.array(list(out))
