"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports every function that
include/vlasov.h declares, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

from paper_1206_3229_gb300 import build as B
from paper_1206_3229_gb300 import vlasov as V

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vlasov.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(vlasov_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return V.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("vlasov_create", "vlasov_step", "vlasov_moments", "vlasov_set_f", "vlasov_get_f", "vlasov_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(V.EXPORTED)


@pytest.mark.parametrize("nx,np_,dt,model,eps,prec", [
    (10, 64, 0.1, V.HMF, 0.0, V.F64),       # Nx not a multiple of 8
    (64, 8, 0.1, V.HMF, 0.0, V.F64),        # Np below 16
    (64, 64, 0.0, V.HMF, 0.0, V.F64),       # dt <= 0
    (64, 64, 0.1, V.RING, 0.0, V.F64),      # ring without softening
    (64, 64, 0.1, 7, 0.0, V.F64),           # unknown model
    (64, 64, 0.1, V.HMF, 0.0, 5),           # unknown precision
    (8200, 64, 0.1, V.HMF, 0.0, V.F64),     # FP64 rows longer than the staged maximum
    (8200, 64, 0.1, V.HMF, 0.0, V.F32),     # FP32 rows longer than the staged maximum
])
def test_create_rejects_bad_arguments_without_gpu(lib, nx, np_, dt, model, eps, prec):
    dom = V.Domain(-3.14, 3.14, -4.0, 4.0, 1, 0, eps, 1.0, prec, None)
    h = ctypes.c_void_p()
    rc = lib.vlasov_create(model, nx, np_, ctypes.byref(dom), dt, ctypes.byref(h))
    assert rc == V.EINVAL and not h.value
    assert lib.vlasov_last_error()


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.vlasov_step(None, 1) == V.EINVAL
    assert lib.vlasov_init_waterbag(None, 1.0, 1.0, 0.0, 0, 0, 0.0) == V.EINVAL
    assert lib.vlasov_set_ring_method(None, V.RING_METHODS["fixed"]) == V.EINVAL
    assert lib.vlasov_ring_method(None) == 0
    assert lib.vlasov_ring_timings(None, 1, None) == V.EINVAL
    assert lib.vlasov_test_expire_wait(None, 1000) == V.EINVAL
    assert lib.vlasov_sync(None) == V.EINVAL
    lib.vlasov_destroy(None)
    assert lib.vlasov_kernels_per_step(None) == 0
    assert lib.vlasov_launches(None, 3) == 0
    assert lib.vlasov_set_fused_x(None, 1) == V.EINVAL
    assert lib.vlasov_fused_x(None) == 0
    assert lib.vlasov_batch_shape_of(None, None) == V.EINVAL
    assert lib.vlasov_batch_autotune(256, V.F32, None, None, None) == V.EINVAL


@pytest.mark.parametrize("rows,tiles", [(0, 8), (16, 0), (5000, 8), (16, 2000)])
def test_batch_shape_is_checked_before_any_device_work(lib, rows, tiles):
    h = ctypes.c_void_p()
    sh = V.BatchShape(rows, tiles)
    rc = lib.vlasov_batch_create_shaped(4, 256, 1 << 28, V.F32, None, ctypes.byref(sh), ctypes.byref(h))
    assert rc == V.EINVAL and not h.value
