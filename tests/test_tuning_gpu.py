"""Launch shapes (threads per CTA and factor staging of the local solves, transport tile)
change no result beyond rounding, and the autotuner leaves the state of the step it ran on
as it found it."""
import numpy as np
import pytest

from tests.cases import case, rel

pytestmark = pytest.mark.gpu

SHAPES = [dict(local_threads=64, local_stage=0, ds_threads=64, ds_stage=0, transport_rows=8, sweep_terms=4),
          dict(local_threads=128, local_stage=1, ds_threads=128, ds_stage=1, transport_rows=4, sweep_terms=8),
          dict(local_threads=256, local_stage=0, ds_threads=256, ds_stage=0, transport_rows=16, sweep_terms=16),
          dict(local_threads=64, local_stage=1, ds_threads=128, ds_stage=0, transport_rows=4, sweep_terms=4)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11050_gb300 import build
    build.build()


def _ctx(c, prec, R=1):
    from paper_2103_11050_gb300 import binding as B
    ctx = B.Context(R, c["nx"], c["ny"], c["Lx"], c["Ly"])
    ctx.set_precision(prec, 1e-14, 30)
    ctx.set_fluids(c["M"])
    ctx.set_boundary(c["bc_type"], c["bc_val"], 1.0)
    ctx.set_decomposition(c["col_w"], c["row_h"], c["seg_len"], c["degree"], c["alpha"], c["alpha_face"])
    ctx.set_permeability(np.ascontiguousarray(np.broadcast_to(c["K"], (R, c["ny"], c["nx"]))))
    ctx.set_saturation(np.ascontiguousarray(np.broadcast_to(c["s0"], (R, c["ny"], c["nx"]))))
    return ctx


def _run(c, prec, tune, steps=6, eta=0.03):
    ctx = _ctx(c, prec)
    if tune is not None:
        ctx.set_tuning(tune)
    ctx.init(eta)
    for _ in range(steps):
        ctx.step(eta, 0.5, 1)
    ux, uy = ctx.get_flux()
    out = ux, uy, ctx.get_saturation(), ctx.get_stats()["rebuilds"]
    ctx.close()
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_launch_shapes_agree(prec):
    c = case("contrast64", "zero")
    ref = _run(c, prec, None)
    for tune in SHAPES:
        got = _run(c, prec, tune)
        assert got[3] == ref[3]
        assert rel(got[0], ref[0]) <= 1e-12
        assert rel(got[1], ref[1]) <= 1e-12 + 1e-14
        assert rel(got[2], ref[2]) <= 1e-12


def test_invalid_tuning_rejected():
    from paper_2103_11050_gb300 import binding as B
    ctx = _ctx(case("p1_2x2"), 0)
    for bad in (dict(SHAPES[0], local_threads=96), dict(SHAPES[0], ds_stage=2), dict(SHAPES[0], transport_rows=3),
                dict(SHAPES[0], sweep_terms=12)):
        with pytest.raises(B.MPMError) as ei:
            ctx.set_tuning(bad)
        assert ei.value.code == B.MPM_ERR_ARG


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_keeps_the_state(prec):
    # after mpm_autotune the current update reads back the same (up to refinement rounding) and
    # the trajectory continues like that of a context that was never tuned
    c = case("uneven", "zero")
    eta = 0.03
    a, b = _ctx(c, prec), _ctx(c, prec)
    for ctx in (a, b):
        ctx.init(eta)
        for _ in range(2):
            ctx.step(eta, 0.5, 1)
    ux0, uy0 = a.get_flux()
    tune, ms = a.autotune(3)
    assert tune["local_threads"] in (64, 128, 256) and tune["transport_rows"] in (4, 8, 16)
    assert all(m > 0 for m in ms) and tune["sweep_terms"] in (4, 8, 16)
    ux1, uy1 = a.get_flux()
    assert rel(ux1, ux0) <= 1e-12 and rel(uy1, uy0) <= 1e-12 + 1e-14
    np.testing.assert_array_equal(a.get_saturation(), b.get_saturation())
    for _ in range(3):
        for ctx in (a, b):
            ctx.step(eta, 0.5, 1)
    assert rel(a.get_flux()[0], b.get_flux()[0]) <= 1e-10
    assert rel(a.get_saturation(), b.get_saturation()) <= 1e-10
    assert a.get_stats()["rebuilds"] == b.get_stats()["rebuilds"]
