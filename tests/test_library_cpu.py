"""The C-ABI library builds, loads and exports every symbol of
include/lbm_elastic.h; argument validation that needs no GPU (no compute
calls are made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_06404_gb300 import build, binding
    build.build()
    return binding.load_library()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_elastic_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    from paper_2009_06404_gb300 import binding
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert set(binding.SYMBOLS) >= declared


def test_library_is_built_for_sm_103a():
    from paper_2009_06404_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def _cfg(**kw):
    from paper_2009_06404_gb300 import binding
    base = dict(nx=16, ny=12, storage="f32")
    base.update(kw)
    return binding.make_config(**base)


@pytest.mark.parametrize("kw", [
    dict(nx=2), dict(ny=0), dict(tau=0.5), dict(tau=float("nan")),
    dict(bc=("periodic", "free", "periodic", "periodic")),
    dict(bc=("free", "rigid", "periodic", "rigid")),
    dict(sponge=(-1, 0, 0, 0)), dict(sponge=(0, 0, 10, 10)),
    dict(max_receivers=-1),
])
def test_invalid_configs_rejected(lib, kw):
    c = _cfg(**kw)
    assert lib.lbm_elastic_workspace_bytes(ctypes.byref(c)) == 0


def test_valid_config_sizes(lib):
    c = _cfg(nx=1024, ny=512)
    n32 = lib.lbm_elastic_workspace_bytes(ctypes.byref(c))
    c64 = _cfg(nx=1024, ny=512, storage="f64")
    n64 = lib.lbm_elastic_workspace_bytes(ctypes.byref(c64))
    # two population buffers of 9 planes dominate: FP64 needs more
    assert n32 > 2 * 9 * 1024 * 512 * 4 and n64 > 2 * 9 * 1024 * 512 * 8 > n32


def test_create_rejects_bad_workspace(lib):
    c = _cfg()
    need = lib.lbm_elastic_workspace_bytes(ctypes.byref(c))
    h = ctypes.c_void_p()
    # checked before any CUDA call: NULL, misaligned, too small
    assert lib.lbm_elastic_create(ctypes.byref(c), None, need, None, ctypes.byref(h)) == -3
    assert lib.lbm_elastic_create(ctypes.byref(c), 4096 + 8, need, None, ctypes.byref(h)) == -3
    assert lib.lbm_elastic_create(ctypes.byref(c), 4096, need - 1, None, ctypes.byref(h)) == -3
    assert b"small" in lib.lbm_elastic_last_error(None)
    bad = _cfg(nx=1)
    assert lib.lbm_elastic_create(ctypes.byref(bad), 4096, need, None, ctypes.byref(h)) == -1
    assert h.value is None


def test_status_strings(lib):
    assert lib.lbm_elastic_status_string(-5) == b"LBM_ERR_NONFINITE"
    assert lib.lbm_elastic_status_string(0) == b"LBM_OK"


def test_handle_less_error_message_is_per_thread(lib):
    """Calls made without a handle keep their failure message per calling
    thread, so two threads failing at once each read their own."""
    import threading
    c = _cfg()
    need = lib.lbm_elastic_workspace_bytes(ctypes.byref(c))
    got = {}
    barrier = threading.Barrier(2)

    def worker(name, ws, size):
        h = ctypes.c_void_p()
        barrier.wait()
        for _ in range(200):
            lib.lbm_elastic_create(ctypes.byref(c), ws, size, None, ctypes.byref(h))
        got[name] = lib.lbm_elastic_last_error(None)

    t1 = threading.Thread(target=worker, args=("null", None, need))
    t2 = threading.Thread(target=worker, args=("small", 4096, need - 1))
    t1.start(); t2.start(); t1.join(); t2.join()
    assert b"NULL" in got["null"] and b"small" not in got["null"]
    assert b"small" in got["small"] and b"NULL" not in got["small"]
