"""CPU-side checks of the C ABI: the library loads, exports every symbol that
include/acm.h declares, and rejects invalid parameters before touching a GPU.
No compute call is made here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2012_03525_gb300 import acm, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return acm.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "acm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(acm_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(acm.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_params_struct_layout_matches_header():
    # field order/types of acm_params as declared in include/acm.h
    src = open(os.path.join(ROOT, "include", "acm.h")).read()
    body = src[src.index("typedef struct {"):src.index("} acm_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"(?:int|double)\s+([^;]+);", body)
    flat = []
    for group in names:
        for n in group.split(","):
            flat.append(re.sub(r"\[.*\]", "", n).strip())
    assert flat == [f[0] for f in acm.Params._fields_]


@pytest.mark.parametrize("kw,msg", [
    (dict(shape=(8, 0)), "grid sizes must be >= 1"),     # empty grids
    (dict(shape=(0, 8)), "grid sizes must be >= 1"),
    (dict(shape=(0, 8, 8)), "grid sizes must be >= 1"),
    (dict(shape=(8, 8, 0)), "grid sizes must be >= 1"),
    (dict(shape=(8, 8), dt=0.0), "dt"),
    (dict(shape=(8, 8), nu=-1.0), "nu"),
    (dict(shape=(8, 8), bc=[1, 0, 0, 0, 0, 0]), "periodic"),
    (dict(shape=(3, 8), bc=[0, 0, 1, 1, 0, 0]), "walls"),
    (dict(shape=(4, 8, 8), bc=[1, 1, 0, 0, 0, 0]), "periodic or symmetry x and y"),
    (dict(shape=(4, 8, 8), bc=[4, 4, 0, 0, 0, 0]), "two-phase"),
    (dict(shape=(4, 8, 8), bc=[4, 0, 0, 0, 0, 0], two_phase=True), "paired"),
    (dict(shape=(4, 8, 8), bc=[0, 0, 0, 0, 4, 4], two_phase=True), "x and y faces"),
    (dict(shape=(8, 8), bc=[4, 4, 0, 0, 0, 0], two_phase=True), "3D"),
    (dict(shape=(4, 8, 8), bc=[0, 0, 0, 0, 1, 1]), "two-phase runs only"),
    (dict(shape=(4, 8, 8), bc=[0, 0, 0, 0, 2, 2], two_phase=True), "lid"),
    (dict(shape=(4, 8, 8), bc=[0, 0, 0, 0, 3, 3], two_phase=True), "single-phase only"),
    (dict(shape=(8, 8), two_phase=True, W=0.0), "sigma/W/M"),
    (dict(shape=(8, 8), two_phase=True, theta_deg=float("nan")), "contact angle"),
    (dict(shape=(8, 8), sat_mask=4), "sat_mask"),
    (dict(shape=(8, 8), precision=7), "precision"),
    (dict(shape=(8, 8), bc=[0, 0, 3, 3, 0, 0]), "z faces of 3D"),
    (dict(shape=(4, 8, 8), bc=[0, 0, 0, 0, 3, 0]), "both faces"),
    (dict(shape=(1, 8, 8), bc=[0, 0, 0, 0, 3, 3]), "nz >= 2"),
    (dict(shape=(4, 8, 8), bc=[3, 3, 0, 0, 0, 0]), "z faces of 3D"),
    (dict(shape=(8, 8), scheme=5), "unknown scheme"),
    (dict(shape=(4, 8, 8), scheme=1), "MAMEs"),
    (dict(shape=(8, 8), scheme=1, two_phase=True), "MAMEs"),
    (dict(shape=(8, 8), scheme=1, bc=[1, 1, 0, 0, 0, 0]), "MAMEs"),
    (dict(shape=(8, 8), scheme=1, g=(1e-5, 0, 0)), "MAMEs"),
])
def test_invalid_params_rejected_on_host(lib, kw, msg):
    shape = kw.pop("shape")
    p = acm.make_params(shape, **kw)
    h = ctypes.c_void_p()
    st = lib.acm_create(ctypes.byref(p), ctypes.byref(h))
    assert st == acm.EINVAL
    assert not h.value
    assert msg in lib.acm_last_error(None).decode()


def test_empty_batch_rejected(lib):
    arr = (acm.Params * 1)(acm.make_params((8, 8)))
    h = ctypes.c_void_p()
    assert lib.acm_batch_create(arr, 0, ctypes.byref(h)) == acm.EINVAL
    assert not h.value
    assert "nruns < 1" in lib.acm_last_error(None).decode()


def test_batch_must_share_precision(lib):
    a = acm.make_params((8, 8))
    b = acm.make_params((16, 8), precision=acm.FP32_DEV)
    arr = (acm.Params * 2)(a, b)
    h = ctypes.c_void_p()
    assert lib.acm_batch_create(arr, 2, ctypes.byref(h)) == acm.EINVAL
    assert "share" in lib.acm_last_error(None).decode()


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.acm_step(None, 1) == acm.EINVAL
    assert lib.acm_sync(None) == acm.EINVAL
    assert lib.acm_destroy(None) == acm.OK
    assert lib.acm_nruns(None) == 0


def test_3d_batches_must_be_matching_subdomains(lib):
    # 3D runs without halo faces cannot be batched
    a = acm.make_params((8, 8, 8))
    arr = (acm.Params * 2)(a, a)
    h = ctypes.c_void_p()
    assert lib.acm_batch_create(arr, 2, ctypes.byref(h)) == acm.EINVAL
    assert "sub-domains" in lib.acm_last_error(None).decode()
    # slabs of different x-y size cannot form one grid
    p = acm.subdomain_params((8, 8, 8), (4, 4))
    p[1].nx = 16
    arr = (acm.Params * 2)(*p)
    assert lib.acm_batch_create(arr, 2, ctypes.byref(h)) == acm.EINVAL
    assert "share" in lib.acm_last_error(None).decode()


def test_subdomain_params_split():
    p = acm.subdomain_params((10, 6, 8), (3, 7), nu=0.1)
    assert [q.nz for q in p] == [3, 7]
    assert all(q.bc[4] == q.bc[5] == acm.BC_HALO for q in p)
    with pytest.raises(ValueError):
        acm.subdomain_params((10, 6, 8), (3, 6))


# ---------------------------------------------------------------- host-only calls
def test_storage_elems_layouts(lib):
    """2D storage is the grid itself; 3D is padded by two ghost layers in x
    and y, rows rounded up to 8 elements; each rounded to 32 elements."""
    assert acm.storage_elems(acm.make_params((64, 64))) == 4096
    assert acm.storage_elems(acm.make_params((5, 7))) == 64          # 35 -> 64
    nz, ny, nx = 10, 12, 30
    px = ((nx + 4 + 7) // 8) * 8
    n = px * (ny + 4) * nz
    assert acm.storage_elems(acm.make_params((nz, ny, nx))) == (n + 31) // 32 * 32
    with pytest.raises(acm.AcmError):
        acm.storage_elems(acm.make_params((8, 8), dt=0.0))


def test_stability_ratio_von_neumann(lib):
    """max(|u|^2 dt / (2 nu), 2 dim nu dt): forward Euler with centred
    advection and diffusion.  The decaying-turbulence set-up of the learned
    closure (u_max ~ 0.15, nu = 5e-4) is unstable at dt = 1 and stable at
    dt = 1/30; the 256^3 Taylor-Green case (u0 = 0.05, Re = 1600) is just
    inside; a diffusion number above 1/(2 dim) is caught as well."""
    u = np.array([0.1, -0.15, 0.02])
    v = np.array([0.0, 0.0, 0.05])
    p = acm.make_params((1, 3), dt=1.0, nu=5e-4)
    assert acm.stability_ratio(p, u, v) == pytest.approx(0.15 ** 2 / (2 * 5e-4))
    p = acm.make_params((1, 3), dt=1.0 / 30, nu=5e-4)
    assert acm.stability_ratio(p, u, v) == pytest.approx(0.15 ** 2 / 30 / (2 * 5e-4))
    assert acm.stability_ratio(p, u, v) < 1
    nu = 0.05 * (256 / (2 * math.pi)) / 1600
    p = acm.make_params((1, 1, 1), nu=nu)
    r = acm.stability_ratio(p, np.array([0.05]), np.array([0.0]), np.array([0.0]))
    assert 0.9 < r < 1.0
    p = acm.make_params((1, 1, 1), nu=0.2)  # 2 * 3 * 0.2 = 1.2
    assert acm.stability_ratio(p, np.zeros(1), np.zeros(1), np.zeros(1)) == pytest.approx(1.2)
    p = acm.make_params((1, 2), nu=0.0)
    assert acm.stability_ratio(p, np.array([0.0, 1e-3]), np.zeros(2)) == math.inf
    assert acm.stability_ratio(p, np.zeros(2), np.zeros(2)) == 0.0


@pytest.mark.parametrize("nx,ny,batch", [(8, 16, 1), (16, 8, 1), (24, 16, 1), (32, 40, 1),
                                         (32, 32, 0), (0, 0, 1)])
def test_closure_grid_rejected_before_any_gpu_work(lib, nx, ny, batch):
    """The closure's convolution tiles are 16 x 8 pixels and its staging
    needs both grid sides a multiple of 16: other grids (or an empty batch)
    are refused by acm_closure_create with ACM_EINVAL and a message."""
    c = ctypes.c_void_p()
    st = lib.acm_closure_create(nx, ny, batch, ctypes.byref(c))
    assert st == acm.EINVAL
    assert not c.value
    assert "multiple of 16" in lib.acm_closure_last_error(None).decode()
