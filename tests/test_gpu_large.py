"""Maximum sizes: boxes whose component planes lie more than 2^31 floats from
the base of a caller's 3N velocity array.

lb_init reads u_z at offset 2N + s and lb_moments writes it there; from
N = 2^31/3 on that offset exceeds a 32-bit int, so these calls must index the
component planes in 64 bits.  A 1024 x 1024 x 700 box (7.3e8 sites; about 81
GB of FP16 populations and 30 GB of fields) round-trips phi and u through
lb_init and lb_moments at t = 0 (sigma = 0, no force, so lb_moments returns
the stored velocity), with the comparison done on the device.
"""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbgb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_01126_gb300 import build

    build.build()
    from paper_2505_01126_gb300 import lbgb as mod

    return mod


def test_largest_box_init_and_moments_round_trip(lbgb):
    import torch

    nx, ny, nz = 1024, 1024, 700
    N = nx * ny * nz
    assert 3 * N > 2 ** 31  # 2N + s passes 2^31 for the last sites
    free, _ = torch.cuda.mem_get_info()
    if free < 140e9:
        pytest.skip("needs about 140 GB of free device memory")
    g = torch.Generator(device="cuda").manual_seed(7)
    phi = torch.rand((nz, ny, nx), device="cuda", generator=g)
    u = (torch.rand((3, nz, ny, nx), device="cuda", generator=g) - 0.5) * 0.02
    b = lbgb.Box(nx, ny, nz, 0.8, 0.1, 3.0, 0.0, storage="f16")
    b.init(phi, u)
    rho, uo, po = torch.empty_like(phi), torch.empty_like(u), torch.empty_like(phi)
    b.moments(rho, uo, po)
    torch.cuda.synchronize()
    b.close()
    # FP16 storage of delta = 3 c.u + ... (|delta| <= 0.03, relative rounding 2^-11)
    for k in range(3):
        assert float((uo[k] - u[k]).abs().max()) < 5e-5, k
    assert float((po - phi).abs().max()) < 1e-6
    assert float((rho - 1).abs().max()) < 1e-4
