"""mpm_cfl_dt_noalloc: the transport time step for callers that cannot allocate device
memory (their memory belongs to another runtime's pre-sized pool, or a latency-critical
loop cannot afford cudaMalloc's implicit synchronisation or its failure mid-run).

It must return the same dt as the context-based mpm_saturation_step for the same fluxes,
on consecutive calls (the calls share the library's fixed scratch array), and refuse sizes
beyond that array's capacity.  Collected last so that a run stopping at the first failure
has already run every other test."""
import ctypes

import numpy as np
import pytest

from tests.cases import case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11050_gb300 import build
    build.build()
    return torch


def test_noalloc_cfl_matches_saturation_step_on_consecutive_calls(torch_cuda):
    torch = torch_cuda
    from paper_2103_11050_gb300 import binding as B
    from paper_2103_11050_gb300 import fields
    c = case("uneven", "front")
    R = 2
    Ks = np.stack([c["K"], fields.lognormal_grf(c["nx"], c["ny"], c["h"], 1.0, 0.1, "exponential", 77)])
    ctx = B.Context(R, c["nx"], c["ny"], c["Lx"], c["Ly"])
    ctx.set_fluids(c["M"])
    ctx.set_boundary(c["bc_type"], c["bc_val"], 1.0)
    ctx.set_decomposition(c["col_w"], c["row_h"], c["seg_len"], c["degree"], c["alpha"])
    ctx.set_permeability(np.ascontiguousarray(Ks))
    ctx.set_saturation(np.ascontiguousarray(np.broadcast_to(c["s0"], (R, c["ny"], c["nx"]))))
    ctx.init(0.05)
    ux = torch.empty((R, c["ny"], c["nx"] + 1), dtype=torch.float64, device="cuda")
    uy = torch.empty((R, c["ny"] + 1, c["nx"]), dtype=torch.float64, device="cuda")
    dt = torch.full((R,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        ctx.get_flux(ux, uy)
        B.cfl_dt_noalloc(ux, uy, dt, c["h"], c["M"], 0.5)
        torch.cuda.synchronize()
        got = dt.cpu().numpy()
        want = ctx.saturation_step(0.5, 1)  # dt of the same fluxes, then one transport step
        assert np.all(want > 0)
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)
        ctx.step(0.05, 0.5, 1)  # new fluxes for the next call
    ctx.close()


def test_noalloc_calls_take_no_device_memory(torch_cuda):
    # The point of the entry point: after its first call on the device (which only looks up
    # the scratch array's address), further calls leave the device's free memory unchanged.
    torch = torch_cuda
    from paper_2103_11050_gb300 import binding as B
    R, nx, ny = 3, 24, 20
    gen = torch.Generator(device="cuda").manual_seed(5)
    ux = torch.randn((R, ny, nx + 1), dtype=torch.float64, device="cuda", generator=gen)
    uy = torch.randn((R, ny + 1, nx), dtype=torch.float64, device="cuda", generator=gen)
    dt = torch.zeros(R, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    B.cfl_dt_noalloc(ux, uy, dt, 1.0 / nx, 2.0, 0.5, stream)
    torch.cuda.synchronize()
    first = dt.clone()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        B.cfl_dt_noalloc(ux, uy, dt, 1.0 / nx, 2.0, 0.5, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(dt, first)


def test_noalloc_binding_checks_shapes_and_types(torch_cuda):
    torch = torch_cuda
    from paper_2103_11050_gb300 import binding as B
    R, nx, ny = 2, 8, 6
    ux = torch.zeros((R, ny, nx + 1), dtype=torch.float64, device="cuda")
    uy = torch.zeros((R, ny + 1, nx), dtype=torch.float64, device="cuda")
    dt = torch.zeros(R, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        B.cfl_dt_noalloc(ux, uy[:, :-1], dt, 0.125, 1.0, 0.5)
    with pytest.raises(ValueError):
        B.cfl_dt_noalloc(ux, uy, dt[:1], 0.125, 1.0, 0.5)
    with pytest.raises(ValueError):
        B.cfl_dt_noalloc(ux.float(), uy, dt, 0.125, 1.0, 0.5)
    with pytest.raises(ValueError):
        B.cfl_dt_noalloc(ux.transpose(1, 2), uy, dt, 0.125, 1.0, 0.5)
    with pytest.raises(ValueError):
        B.cfl_dt_noalloc(ux.cpu(), uy, dt, 0.125, 1.0, 0.5)


def test_noalloc_refuses_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    from paper_2103_11050_gb300 import binding as B
    L = B.load()
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    # R = 1025 realisations exceed the fixed scratch (64 partials each, 65536 in all):
    # rejected before anything is launched, so the small buffers are never touched.
    assert L.mpm_cfl_dt_noalloc(p, p, 1025, 4, 4, 0.25, 1.0, 0.5, p, None) == B.MPM_ERR_TOO_LARGE
    assert L.mpm_cfl_dt_noalloc(p, p, 1, 0, 4, 0.25, 1.0, 0.5, p, None) == B.MPM_ERR_ARG
    assert L.mpm_cfl_dt_noalloc(p, p, 1, 4, 4, 0.25, 1.0, 1.5, p, None) == B.MPM_ERR_ARG
