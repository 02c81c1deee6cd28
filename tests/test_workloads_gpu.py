"""GPU path against the oracle on workload-shaped inputs (the seeded fields of fields.py):
the 64^2 rebuild-every-step run in full, the 256^2 benchmark workload at full size, a
channelised contrast-1e4 field, an ensemble of realisations on an uneven decomposition,
and a homogeneous fingering run.  Tolerances as in test_parity_gpu (1e-10 FP64, 1e-8 mixed)."""
import numpy as np
import pytest

from oracle import mpm_oracle as O
from paper_2103_11050_gb300 import fields
from tests.cases import rel

pytestmark = pytest.mark.gpu
TOL = {0: 1e-10, 1: 1e-8, 2: 1e-8}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11050_gb300 import build
    build.build()


def _ctx(R, nx, ny, M, col_w, row_h, K, s0, prec, bc_type=(0, 0, 1, 1), bc_val=(1.0, 0, 0, 0), seg=4, deg=1):
    from paper_2103_11050_gb300 import binding as B
    ctx = B.Context(R, nx, ny, 1.0, ny / nx)
    ctx.set_precision(prec, 1e-14, 30)
    ctx.set_fluids(M)
    ctx.set_boundary(bc_type, bc_val, 1.0)
    ctx.set_decomposition(col_w, row_h, seg, deg, 1.0)
    ctx.set_permeability(np.ascontiguousarray(np.broadcast_to(K, (R, ny, nx))))
    ctx.set_saturation(np.ascontiguousarray(np.broadcast_to(s0, (R, ny, nx))))
    return ctx


def _run_both(K, s0, nx, ny, M, col_w, row_h, eta, steps, prec, **kw):
    prob = O.Problem(nx, ny, 1.0 / nx, kw.get("bc_type", (0, 0, 1, 1)), kw.get("bc_val", (1.0, 0, 0, 0)), M, 1.0)
    dec = O.Decomposition(nx, ny, col_w, row_h, 4, 1, 1.0)
    st = O.simulate_init(K, s0, prob, dec, eta)
    ctx = _ctx(1, nx, ny, M, col_w, row_h, K, s0, prec, **kw)
    ctx.init(eta)
    for _ in range(steps):
        O.simulate_step(st, K, prob, dec, eta, 0.5, 1)
        ctx.step(eta, 0.5, 1)
    return st, ctx, prob


@pytest.mark.parametrize("prec", [0, 1])
def test_gaussian64_rebuild_every_step(prec):
    # 64^2, 4x4 subdomains of 16^2, exponential GRF (ell 0.1, var 1), M = 1, 20 steps, a full
    # MRCM rebuild at every step from the second on (eta < 0; Algorithm 1 starts with
    # epsilon = eta and a strict test, so the first step reuses the initial basis).
    K, s0, w = fields.make_workload("gaussian64")
    st, ctx, prob = _run_both(K, s0, 64, 64, w["M"], [16] * 4, [16] * 4, w["eta"], w["steps"], prec)
    ux, uy = ctx.get_flux()
    n_reb = sum(1 for h in st.history if h["rebuild"])
    assert n_reb == w["steps"] - 1
    assert ctx.get_stats()["rebuilds"] == n_reb + 1
    assert rel(ux[0], st.step.Fx) <= TOL[prec]
    assert rel(uy[0], st.step.Fy) <= TOL[prec] + 1e-12
    assert rel(ctx.get_saturation()[0], st.s) <= TOL[prec]
    assert rel(ctx.get_pressure(0)[0], st.p_m) <= TOL[prec]


def test_gaussian256_benchmark_workload_full_size():
    # The benchmark workload (graph execution, FP32 downscaling + FP64 refinement), the
    # whole arrays compared after the initial solve and 5 Algorithm 1 steps.
    K, s0, w = fields.make_workload("gaussian256")
    st, ctx, prob = _run_both(K, s0, 256, 256, w["M"], [16] * 16, [16] * 16, w["eta"], 5, 1)
    ux, uy = ctx.get_flux()
    assert rel(ux[0], st.step.Fx) <= 1e-8
    assert rel(uy[0], st.step.Fy) <= 1e-8
    assert rel(ctx.get_saturation()[0], st.s) <= 1e-8
    assert rel(ctx.get_pressure(1)[0], st.step.p_down) <= 1e-8
    bal = np.max(np.abs(O.cell_balance(ux[0], uy[0], prob))) / np.max(np.abs(ux[0]))
    assert bal <= 1e-11
    n_reb = sum(1 for h in st.history if h["rebuild"])
    assert ctx.get_stats()["rebuilds"] == n_reb + 1


@pytest.mark.parametrize("prec", [1, 2])
def test_channelised_contrast_1e4(prec):
    # Channelised binary field (sinusoidal channels, 30 % coverage, contrast 1e4) at 128^2 with
    # 8x8 subdomains of 16^2; mixed forms against the oracle and against the FP64 GPU form.
    nx = 128
    K = fields.channelised(nx, nx, 1.0, 1e-4, 0.30, (4, 12), seed=3)
    s0 = np.zeros((nx, nx))
    st, ctx, prob = _run_both(K, s0, nx, nx, 5.0, [16] * 8, [16] * 8, 0.1, 3, prec)
    ux, _ = ctx.get_flux()
    assert rel(ux[0], st.step.Fx) <= 1e-8
    ref = _ctx(1, nx, nx, 5.0, [16] * 8, [16] * 8, K, s0, 0)
    ref.init(0.1)
    for _ in range(3):
        ref.step(0.1, 0.5, 1)
    assert rel(ux[0], ref.get_flux()[0][0]) <= 1e-8


def test_ensemble_uneven_decomposition():
    # 16 realisations of a 128^2 log-normal field (variance 2, correlation lengths drawn in
    # [0.05, 0.2]) on one uneven decomposition (seeded permutations of 8,8,12,12,16,16,16,20,20):
    # one context, one launch per stage for all realisations; two realisations against the
    # oracle, all of them conservative and bounded.
    nx, R = 128, 16
    rng = np.random.default_rng(4)
    ells = rng.uniform(0.05, 0.2, R)
    Ks = np.stack([fields.lognormal_grf(nx, nx, 1.0 / nx, 2.0, ells[r], "exponential", 4 + r) for r in range(R)])
    parts = [8, 8, 12, 12, 16, 16, 16, 20, 20]
    cw, rh = fields.uneven_widths(nx, parts, 11), fields.uneven_widths(nx, parts, 12)
    s0 = np.zeros((nx, nx))
    eta, steps = 0.05, 4
    ctx = _ctx(R, nx, nx, 3.0, cw, rh, Ks, s0, 1)
    ctx.init(eta)
    for _ in range(steps):
        ctx.step(eta, 0.5, 1)
    ux, uy = ctx.get_flux()
    s = ctx.get_saturation()
    prob = O.Problem(nx, nx, 1.0 / nx, (0, 0, 1, 1), (1.0, 0, 0, 0), 3.0, 1.0)
    dec = O.Decomposition(nx, nx, cw, rh, 4, 1, 1.0)
    for r in (0, R - 1):
        st = O.simulate_init(Ks[r], s0, prob, dec, eta)
        for _ in range(steps):
            O.simulate_step(st, Ks[r], prob, dec, eta, 0.5, 1)
        assert rel(ux[r], st.step.Fx) <= 1e-8
        assert rel(s[r], st.s) <= 1e-8
    for r in range(R):
        bal = np.max(np.abs(O.cell_balance(ux[r], uy[r], prob))) / np.max(np.abs(ux[r]))
        assert bal <= 1e-11
        assert s[r].min() >= -1e-14 and s[r].max() <= 1 + 1e-14


def test_fingering_homogeneous():
    # Homogeneous medium, M = 10, water-filled strip at the inlet with 1 % seeded noise
    # (the fingering set-up), 128^2 with 8x8 subdomains, eta = 0.1, 10 steps.
    nx = 128
    K = np.ones((nx, nx))
    s0 = fields.fingering_s0(nx, nx, 0.05, 8, 0.01, seed=5)
    st, ctx, prob = _run_both(K, s0, nx, nx, 10.0, [16] * 8, [16] * 8, 0.1, 10, 1)
    assert rel(ctx.get_flux()[0][0], st.step.Fx) <= 1e-8
    assert rel(ctx.get_saturation()[0], st.s) <= 1e-8
