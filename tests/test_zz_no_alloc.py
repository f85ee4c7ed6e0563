"""GPU test of rpk_field_totals_noalloc, the entry point for callers that may
not allocate device memory where they need conserved totals (an application
whose memory manager owns all device memory, or a loop that must not stall on
cudaMalloc). It reduces fields the caller already holds using a static device
scratch array, and must agree with rpk_diagnostics on the same state. This
file is collected last on purpose."""
import numpy as np
import pytest

import paper_2201_05280_gb300 as rpk
import rpk_inputs as I

pytestmark = pytest.mark.gpu

T0 = 0.2948964908710633
RELAX = dict(delta=2.0, tau=0.6, tau1=0.8, b=0.3, k_r=0.9, nsub=2)
CHUNK = 8192  # points reduced by one block of the entry point


@pytest.fixture(scope="module")
def torch_cuda():
    from paper_2201_05280_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch


def _device_fields(torch, lat):
    n = lat.npts
    out = {k: torch.empty(m * n, dtype=torch.float64, device="cuda")
           for k, m in (("rho", 1), ("u", 3), ("T", 1), ("R", 1))}
    lat.read_moments(out)
    return out


def _check_against_diagnostics(torch, lat, out):
    F = _device_fields(torch, lat)
    rpk.field_totals_noalloc(F["rho"], F["u"], F["T"], F["R"], RELAX["delta"], out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    d = lat.diagnostics()
    assert abs(got[0] - d["M"]) <= 1e-12 * d["M"]
    assert np.abs(got[1:4] - d["J"]).max() <= 1e-12 * d["M"]
    assert abs(got[4] - d["E"]) <= 1e-12 * d["E"]


def test_noalloc_totals_match_diagnostics_on_two_calls(torch_cuda):
    torch = torch_cuda
    nx, ny, nz = 30, 8, 6
    f = I.random_smooth(nx, ny, nz, T0, seed=21)
    lat = rpk.Lattice(nx, ny, nz, precision="f64").set_relax(**RELAX)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    for nsteps in (10, 15):  # two calls in a row on two different states
        lat.step(nsteps)
        _check_against_diagnostics(torch, lat, out)
    lat.close()


def test_noalloc_totals_many_blocks_then_fewer(torch_cuda):
    """A lattice of 8.5 blocks' worth of points (the last block partly full),
    then a smaller one: the second call must not read the first call's slots
    left in the shared scratch."""
    torch = torch_cuda
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    for (nx, ny, nz), seed in (((64, 32, 17), 5), ((40, 16, 9), 6)):
        npts = 2 * nx * ny * nz
        f = I.random_smooth(nx, ny, nz, T0, seed=seed)
        lat = rpk.Lattice(nx, ny, nz, precision="f64").set_relax(**RELAX)
        lat.init_fields(f["rho"], f["u"], f["T"], f["R"]).step(4)
        _check_against_diagnostics(torch, lat, out)
        lat.close()
    assert npts < CHUNK * 2 and 2 * 64 * 32 * 17 > 8 * CHUNK


def test_noalloc_totals_reject_sizes_beyond_the_scratch(torch_cuda):
    torch = torch_cuda
    lib = rpk.load_library()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    for n in (0, 8192 * 8192 + 1):
        code = lib.rpk_field_totals_noalloc(p, p, p, p, n, 2.0, None, p)
        assert code == 1
        assert b"npts must lie in" in lib.rpk_last_error()


def test_noalloc_totals_reject_host_memory(torch_cuda):
    """A host array in place of device memory is refused before any launch."""
    torch = torch_cuda
    lib = rpk.load_library()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    h = np.zeros(8)
    p, hp = x.data_ptr(), h.ctypes.data
    code = lib.rpk_field_totals_noalloc(hp, p, p, p, 8, 2.0, None, p)
    assert code == 1
    assert b"device memory of the current device" in lib.rpk_last_error()
    with pytest.raises(ValueError):
        rpk.field_totals_noalloc(torch.zeros(8, dtype=torch.float64), x.repeat(3), x, x, 2.0,
                                 torch.zeros(5, dtype=torch.float64, device="cuda"))
