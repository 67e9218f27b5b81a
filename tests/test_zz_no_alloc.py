"""lb_field_stats_static: FP64 field statistics for callers that must not
allocate device memory, checked against the allocating path.

Callers such as a framework whose caching allocator owns the device memory,
or a latency-critical path where cudaMalloc may synchronise the device, use
this entry point.  It keeps its scratch in a fixed __device__ array.  Its
output must match what lb_init followed by lb_diagnostics reports for the same
fields, on consecutive calls that reuse the same array.
"""
import numpy as np
import pytest

from paper_2505_01126_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-6  # both paths sum FP32 per-thread partials in FP64 in the same tiling


@pytest.fixture(scope="module")
def lbgb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_01126_gb300 import build

    build.build()
    from paper_2505_01126_gb300 import lbgb as mod

    return mod


def fields(shape, seed):
    import torch

    nz, ny, nx = shape
    phi = inputs.bubbles((nx, ny, nz), np.array([[nx / 3, ny / 2, nz / 2], [2 * nx / 3, ny / 3, nz / 4]]), 4.0, 3.0)
    u = inputs.solenoidal_velocity(nx, ny, nz, 0.02, seed=seed)
    return (torch.from_numpy(inputs.to_f32(phi)).cuda(), torch.from_numpy(inputs.to_f32(u)).cuda())


@pytest.mark.parametrize("shape", [(40, 13, 37), (32, 32, 32), (70, 24, 48)])
def test_static_stats_match_lb_init_diagnostics(lbgb, shape):
    import torch

    phi, u = fields(shape, seed=sum(shape))
    nz, ny, nx = shape
    box = lbgb.Box(nx, ny, nz, 0.8, 0.1, 3.0, 0.01)
    box.init(phi, u)
    ref = box.diagnostics()
    box.close()
    first = None
    for _ in range(2):  # the second call reuses the array the first one left behind
        out = lbgb.field_stats_static(phi, u)
        np.testing.assert_allclose(out[[0, 1, 3]], ref[[0, 1, 3]], rtol=RTOL)
        assert out[2] == 0.0 and out[4] == 0.0
        if first is None:
            first = out
        else:
            assert np.array_equal(out, first)
    # device output pointer, stream-ordered
    dev_out = torch.zeros(5, dtype=torch.float64, device="cuda")
    rc = lbgb.lib().lb_field_stats_static(phi.data_ptr(), u.data_ptr(), nx, ny, nz, None,
                                          lbgb.ctypes.cast(dev_out.data_ptr(), lbgb.ctypes.POINTER(lbgb.ctypes.c_double)))
    assert rc == lbgb.LB_OK
    torch.cuda.synchronize()
    np.testing.assert_allclose(dev_out.cpu().numpy()[[0, 1, 3]], ref[[0, 1, 3]], rtol=RTOL)


def test_static_stats_reject_boxes_beyond_the_array(lbgb):
    import torch

    phi = torch.zeros(8, device="cuda")
    u = torch.zeros(24, device="cuda")
    out = (lbgb.ctypes.c_double * 5)()
    rc = lbgb.lib().lb_field_stats_static(phi.data_ptr(), u.data_ptr(), 1024, 1024, 1024, None, out)
    assert rc == lbgb.LB_EINVAL
    assert "partial records" in lbgb.lib().lb_last_error().decode()


def test_static_stats_on_a_side_stream_and_after_a_larger_box(lbgb):
    """A larger box leaves more records in the shared array than a smaller one
    writes; the smaller box's result must not see them.  The calls run on a
    side stream, as a caller with its own stream would make them."""
    import torch

    side = torch.cuda.Stream()
    for shape in [(70, 24, 48), (9, 7, 5)]:
        phi, u = fields(shape, seed=3)
        nz, ny, nx = shape
        box = lbgb.Box(nx, ny, nz, 0.8, 0.1, 3.0, 0.01)
        box.init(phi, u)
        ref = box.diagnostics()
        box.close()
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            out = lbgb.field_stats_static(phi, u, stream=side)
        np.testing.assert_allclose(out[[0, 1, 3]], ref[[0, 1, 3]], rtol=RTOL)


def test_static_stats_report_a_nan_with_a_host_result(lbgb):
    phi, u = fields((16, 16, 16), seed=5)
    u[1, 3, 4, 5] = float("nan")
    with pytest.raises(lbgb.LBError) as exc:
        lbgb.field_stats_static(phi, u)
    assert exc.value.code == lbgb.LB_ENONFINITE


def test_static_stats_reject_host_fields(lbgb):
    phi = np.zeros(8, np.float32)
    u = np.zeros(24, np.float32)
    out = (lbgb.ctypes.c_double * 5)()
    rc = lbgb.lib().lb_field_stats_static(phi.ctypes.data, u.ctypes.data, 2, 2, 2, None, out)
    assert rc == lbgb.LB_EINVAL
    assert "device memory" in lbgb.lib().lb_last_error().decode()


def test_static_stats_reject_another_devices_memory(lbgb):
    import torch

    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    phi = torch.zeros(8, device="cuda:1")
    u = torch.zeros(24, device="cuda:1")
    out = (lbgb.ctypes.c_double * 5)()
    with torch.cuda.device(0):
        rc = lbgb.lib().lb_field_stats_static(phi.data_ptr(), u.data_ptr(), 2, 2, 2, None, out)
    assert rc == lbgb.LB_EINVAL
