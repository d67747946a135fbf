"""The moment sums without a workspace (lbm_elastic_moment_sums_noalloc).

That entry point is for callers that can neither hand the library a device
workspace nor let it allocate one (their device memory is all reserved by
another allocator, or an allocation at that point could fail or stall the
device): its scratch is a fixed array inside the library.  Here it is called
through the C ABI on caller-held tensors and compared, on two calls in a row,
with the sums the handle-based entry point computes from the same state.
This file is collected last so that a failure here leaves every other test
already run."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2009_06404_gb300 import binding, build
    build.build()
    return binding.load_library()


@pytest.mark.parametrize("storage,code,tdtype,u_fp64", [("f64", 0, torch.float64, 0),
                                                         ("f32", 1, torch.float32, 0),
                                                         ("f32", 1, torch.float32, 1)])
def test_noalloc_sums_match_workspace_sums(lib, storage, code, tdtype, u_fp64):
    import paper_2009_06404_gb300 as pkg
    from paper_2009_06404_gb300 import workloads as wl
    nx, ny = 301, 170
    fs0, u0 = wl.random_state(nx, ny, seed=12)
    sim = pkg.ElasticLBM(nx, ny, storage=storage, u_fp64=bool(u_fp64))
    sim.set_state(fs0, u0)
    ref = sim.moment_sums()
    # caller-held state with a padded row (pitch > nx); the padding holds
    # values that must not enter the sums
    pitch = 320
    udtype = torch.float64 if (u_fp64 or storage == "f64") else tdtype
    f9 = torch.full((9, ny, pitch), 7.0, dtype=tdtype, device="cuda")
    u2 = torch.full((2, ny, pitch), 7.0, dtype=udtype, device="cuda")
    f9[:, :, :nx] = torch.tensor(fs0, dtype=tdtype)
    u2[:, :, :nx] = torch.tensor(u0, dtype=udtype)
    stream = torch.cuda.current_stream().cuda_stream
    scale = np.abs(ref) + 1e-300
    for _ in range(2):
        out = (ctypes.c_double * 7)()
        st = lib.lbm_elastic_moment_sums_noalloc(f9.data_ptr(), u2.data_ptr(), code, u_fp64, nx,
                                                 ny, pitch, ctypes.addressof(out), 0, stream)
        assert st == 0, lib.lbm_elastic_last_error(None)
        got = np.array(out[:])
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (got, ref)
    # device output, written on the stream
    dev_out = torch.zeros(7, dtype=torch.float64, device="cuda")
    for _ in range(2):
        dev_out.zero_()
        st = lib.lbm_elastic_moment_sums_noalloc(f9.data_ptr(), u2.data_ptr(), code, u_fp64, nx,
                                                 ny, pitch, dev_out.data_ptr(), 1, stream)
        assert st == 0
        torch.cuda.synchronize()
        assert np.all(np.abs(dev_out.cpu().numpy() - ref) <= 1e-12 * scale)


def test_noalloc_rejects_bad_sizes(lib):
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = (ctypes.c_double * 7)()
    # pitch < nx, and a grid beyond the maximum of the entry point
    assert lib.lbm_elastic_moment_sums_noalloc(x.data_ptr(), x.data_ptr(), 0, 0, 8, 2, 4,
                                               ctypes.addressof(out), 0, None) == -1
    assert lib.lbm_elastic_moment_sums_noalloc(x.data_ptr(), x.data_ptr(), 0, 0, 65536, 65536,
                                               65536, ctypes.addressof(out), 0, None) == -1
    assert b"maximum" in lib.lbm_elastic_last_error(None)
    assert lib.lbm_elastic_moment_sums_noalloc(x.data_ptr(), x.data_ptr(), 2, 0, 2, 2, 2,
                                               ctypes.addressof(out), 0, None) == -2
