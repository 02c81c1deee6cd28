"""GPU path (through the C ABI) against the CPU oracle, element by element, on the same
seeded inputs.  Tolerances: relative L2 error <= 1e-10 for the plain FP64 form and
<= 1e-8 for the FP32 factorisation with FP64 refinement (the accuracy targets of the
method's GPU forms); discrete quantities (rebuild decisions) exactly."""
import numpy as np
import pytest

from oracle import mpm_oracle as O
from tests.cases import case, rel

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-8, 2: 1e-8, 3: 1e-8, 4: 1e-8, 5: 1e-8}


def _oracle_setup(c):
    prob = O.Problem(c["nx"], c["ny"], c["h"], tuple(c["bc_type"]), tuple(c["bc_val"]), c["M"], 1.0)
    dec = O.Decomposition(c["nx"], c["ny"], c["col_w"], c["row_h"], c["seg_len"], c["degree"], c["alpha"],
                          c["alpha_face"])
    return prob, dec


def _balance(Fx, Fy, prob):
    """max over cells of |sum of outward fluxes - q h^2|, relative to the largest x-flux."""
    return float(np.max(np.abs(O.cell_balance(Fx, Fy, prob))) / np.max(np.abs(Fx)))


def _gpu(c, prec, R=1, K=None, s0=None):
    from paper_2103_11050_gb300 import binding as B
    ctx = B.Context(R, c["nx"], c["ny"], c["Lx"], c["Ly"])
    ctx.set_precision(prec, 1e-14, 30)
    ctx.set_fluids(c["M"])
    ctx.set_boundary(c["bc_type"], c["bc_val"], 1.0)
    ctx.set_decomposition(c["col_w"], c["row_h"], c["seg_len"], c["degree"], c["alpha"], c["alpha_face"])
    ctx.set_permeability(np.ascontiguousarray(np.broadcast_to(c["K"] if K is None else K, (R, c["ny"], c["nx"]))))
    ctx.set_saturation(np.ascontiguousarray(np.broadcast_to(c["s0"] if s0 is None else s0, (R, c["ny"], c["nx"]))))
    return ctx


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11050_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("name", ["p1_2x2", "uneven", "const_H", "exact_h", "single", "rate_in", "dirichlet4",
                                  "contrast64", "alpha_field", "max_side", "small_sides"])
def test_mrcm_update_parity(name, prec):
    c = case(name)
    prob, dec = _oracle_setup(c)
    kappa = O.mobility(c["s0"], c["M"]) * c["K"]
    step, _, sol = O.mrcm_step(kappa, prob, dec)
    obal = _balance(step.Fx, step.Fy, prob)
    ctx = _gpu(c, prec)
    ctx.init(0.1)
    pm = ctx.get_pressure(0)[0]
    pd = ctx.get_pressure(1)[0]
    ux, uy = ctx.get_flux()
    tol = TOL[prec]
    assert rel(pm, sol.p) <= tol, rel(pm, sol.p)
    assert rel(pd, step.p_down) <= tol, rel(pd, step.p_down)
    assert rel(ux[0], step.Fx) <= tol, rel(ux[0], step.Fx)
    assert rel(uy[0], step.Fy) <= tol + 1e-12, rel(uy[0], step.Fy)
    # conservation of the GPU fluxes in every cell, as tight as the FP64 oracle's own rounding
    bal = _balance(ux[0], uy[0], prob)
    assert bal <= max(4 * obal, 5e-13), (bal, obal)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("name", ["p1_2x2", "uneven", "rate_in", "dirichlet4", "contrast64", "alpha_field",
                                  "max_side", "small_sides"])
def test_mpm_update_parity(name, prec):
    c = case(name)
    prob, dec = _oracle_setup(c)
    s_m = c["s0"]
    s_n = np.clip(s_m + 0.05 * np.random.default_rng(c["seed"]).standard_normal(s_m.shape), 0, 1)
    kap_m = O.mobility(s_m, c["M"]) * c["K"]
    kap_n = O.mobility(s_n, c["M"]) * c["K"]
    _, bs, sol = O.mrcm_step(kap_m, prob, dec)
    step, _ = O.mpm_step(kap_n, bs, sol.p, prob, dec)
    obal = _balance(step.Fx, step.Fy, prob)
    ctx = _gpu(c, prec)
    ctx.init(0.1)
    ctx.set_saturation(np.ascontiguousarray(s_n[None]))
    eps = ctx.eval_epsilon()
    assert eps[0] == pytest.approx(O.epsilon(kap_n, kap_m), rel=1e-12)
    ctx.perturbation_solve()
    ctx.interface_solve()
    ctx.downscale()
    pd = ctx.get_pressure(1)[0]
    ux, uy = ctx.get_flux()
    tol = TOL[prec]
    assert rel(ux[0], step.Fx) <= tol, rel(ux[0], step.Fx)
    assert rel(uy[0], step.Fy) <= tol + 1e-12, rel(uy[0], step.Fy)
    assert rel(pd, step.p_down) <= tol, rel(pd, step.p_down)
    bal = _balance(ux[0], uy[0], prob)
    assert bal <= max(4 * obal, 5e-13), (bal, obal)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["p1_2x2", "uneven", "contrast64", "alpha_field"])
def test_mpm_first_order_update_parity(name, prec):
    # Eq. (mpm_tf_4), l = 1, through the stand-alone calls: epsilon^0 local + interface solve,
    # first-order local + interface solve, downscaling
    c = case(name)
    prob, dec = _oracle_setup(c)
    s_m = c["s0"]
    s_n = np.clip(s_m + 0.05 * np.random.default_rng(c["seed"]).standard_normal(s_m.shape), 0, 1)
    kap_m = O.mobility(s_m, c["M"]) * c["K"]
    kap_n = O.mobility(s_n, c["M"]) * c["K"]
    _, bs, sol = O.mrcm_step(kap_m, prob, dec)
    step, _ = O.mpm_step(kap_n, bs, sol.p, prob, dec, order=1)
    step0, _ = O.mpm_step(kap_n, bs, sol.p, prob, dec, order=0)
    assert rel(step.Fx, step0.Fx) > 1e3 * TOL[prec]  # the first-order term is visible at this tolerance
    obal = _balance(step.Fx, step.Fy, prob)
    ctx = _gpu(c, prec)
    ctx.set_mpm_order(1)
    ctx.init(0.1)
    ctx.set_saturation(np.ascontiguousarray(s_n[None]))
    ctx.eval_epsilon()
    ctx.perturbation_solve()
    ctx.interface_solve()
    ctx.perturbation_correction()
    ctx.interface_solve()
    ctx.downscale()
    pd = ctx.get_pressure(1)[0]
    ux, uy = ctx.get_flux()
    tol = TOL[prec]
    assert rel(ux[0], step.Fx) <= tol, rel(ux[0], step.Fx)
    assert rel(uy[0], step.Fy) <= tol + 1e-12, rel(uy[0], step.Fy)
    assert rel(pd, step.p_down) <= tol, rel(pd, step.p_down)
    bal = _balance(ux[0], uy[0], prob)
    assert bal <= max(4 * obal, 5e-13), (bal, obal)


def test_first_order_correction_needs_order_one():
    from paper_2103_11050_gb300 import binding as B
    c = case("p1_2x2")
    ctx = _gpu(c, 0)
    ctx.init(0.1)
    with pytest.raises(B.MPMError) as ei:
        ctx.perturbation_correction()
    assert ei.value.code == B.MPM_ERR_STATE


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("prec", [0, 1])
def test_algorithm1_first_order_parity(prec, graph):
    c = case("p1_2x2", "zero")
    prob, dec = _oracle_setup(c)
    eta, steps = 0.02, 10
    st = O.simulate_init(c["K"], c["s0"], prob, dec, eta)
    ctx = _gpu(c, prec)
    ctx.set_mpm_order(1)
    ctx.set_execution(graph, True)
    ctx.init(eta)
    for _ in range(steps):
        O.simulate_step(st, c["K"], prob, dec, eta, 0.5, 1, order=1)
        ctx.step(eta, 0.5, 1)
    tol = TOL[prec]
    n_reb = sum(1 for h in st.history if h["rebuild"])
    assert ctx.get_stats()["rebuilds"] == n_reb + 1
    assert 0 < n_reb < steps - 1  # both kinds of update occur
    ux, uy = ctx.get_flux()
    assert rel(ctx.get_saturation()[0], st.s) <= tol
    assert rel(ux[0], st.step.Fx) <= tol, rel(ux[0], st.step.Fx)
    assert rel(uy[0], st.step.Fy) <= tol + 1e-12
    assert rel(ctx.get_pressure(1)[0], st.step.p_down) <= tol


@pytest.mark.parametrize("name", ["p1_2x2", "uneven", "contrast64", "alpha_field"])
def test_bf16_basis_solves_are_right_or_report(name):
    # bf16 operands (8 significant bits) leave the refinement a contraction only where the
    # scaled local problems are well conditioned: the update must then match the oracle, and
    # otherwise the library must say that it did not converge, never return a silent error.
    from paper_2103_11050_gb300 import binding as B
    c = case(name)
    prob, dec = _oracle_setup(c)
    kappa = O.mobility(c["s0"], c["M"]) * c["K"]
    step, _, sol = O.mrcm_step(kappa, prob, dec)
    ctx = _gpu(c, 5)
    ctx.init(0.1)
    try:
        ctx.sync()
    except B.MPMError as e:
        assert e.code == B.MPM_ERR_NOT_CONVERGED
        return
    ux, uy = ctx.get_flux()
    assert rel(ctx.get_pressure(0)[0], sol.p) <= 1e-8
    assert rel(ux[0], step.Fx) <= 1e-8 and rel(uy[0], step.Fy) <= 1e-8 + 1e-12


def test_transport_parity():
    c = case("uneven", "front")
    prob, dec = _oracle_setup(c)
    kappa = O.mobility(c["s0"], c["M"]) * c["K"]
    step, _, _ = O.mrcm_step(kappa, prob, dec)
    ctx = _gpu(c, 0)
    ctx.init(0.1)
    dt = ctx.saturation_step(0.5, 3)
    dt_o = O.cfl_dt(step.Fx, step.Fy, prob, 0.5)
    assert dt[0] == pytest.approx(dt_o, rel=1e-12)
    s = c["s0"]
    for _ in range(3):
        s = O.upwind_step(s, step.Fx, step.Fy, dt_o, prob)
    sg = ctx.get_saturation()[0]
    assert rel(sg, s) <= 1e-12
    assert np.all(sg >= -1e-14) and np.all(sg <= 1 + 1e-14)
    np.testing.assert_allclose(ctx.get_conductivity()[0], O.mobility(s, c["M"]) * c["K"], rtol=1e-11)


@pytest.mark.parametrize("graph,pdl", [(True, True), (False, True), (True, False), (False, False)])
@pytest.mark.parametrize("prec", [0, 1, 2, 4])
@pytest.mark.parametrize("name,eta,steps", [("p1_2x2", 0.02, 12), ("uneven", -1.0, 4), ("contrast64", 0.05, 8),
                                            ("alpha_field", 0.02, 6)])
def test_algorithm1_parity(name, eta, steps, prec, graph, pdl):
    c = case(name, "zero")
    prob, dec = _oracle_setup(c)
    st = O.simulate_init(c["K"], c["s0"], prob, dec, eta)
    ctx = _gpu(c, prec)
    ctx.set_execution(graph, pdl)
    ctx.init(eta)
    tol = TOL[prec]
    for n in range(steps):
        O.simulate_step(st, c["K"], prob, dec, eta, 0.5, 1)
        ctx.step(eta, 0.5, 1)
    s = ctx.get_saturation()[0]
    ux, uy = ctx.get_flux()
    stats = ctx.get_stats()
    n_reb = sum(1 for h in st.history if h["rebuild"])
    assert stats["rebuilds"] == n_reb + 1  # plus the initial build
    assert stats["mpm_updates"] == steps - n_reb
    # the epsilon history: every step's epsilon and decision, oldest first
    eps_h, reb_h = ctx.get_eps_history()
    assert eps_h.shape == (1, steps)
    np.testing.assert_array_equal(reb_h[0], [int(h["rebuild"]) for h in st.history])
    # epsilon is a norm of kappa^n - kappa^m, i.e. of a difference: a relative error of the
    # saturation of order tol grows by 1/epsilon (~1e2) in it, hence 1e2 tol
    np.testing.assert_allclose(eps_h[0], [h["eps"] for h in st.history], rtol=1e2 * tol, atol=0)
    assert rel(s, st.s) <= tol, rel(s, st.s)
    assert rel(ux[0], st.step.Fx) <= tol, rel(ux[0], st.step.Fx)
    assert rel(uy[0], st.step.Fy) <= tol + 1e-12, rel(uy[0], st.step.Fy)
    # pressures: the MRCM-level p^m of the last rebuild and the last downscaled pressure
    assert rel(ctx.get_pressure(0)[0], st.p_m) <= tol, rel(ctx.get_pressure(0)[0], st.p_m)
    assert rel(ctx.get_pressure(1)[0], st.step.p_down) <= tol, rel(ctx.get_pressure(1)[0], st.step.p_down)


_LONG_SEP = {}


def _long_sep_trajectory(eta, steps):
    """Oracle trajectory of the long-separator case (computed once per module)."""
    if not _LONG_SEP:
        c = case("long_sep", "zero")
        prob, dec = _oracle_setup(c)
        st = O.simulate_init(c["K"], c["s0"], prob, dec, eta)
        for _ in range(steps):
            O.simulate_step(st, c["K"], prob, dec, eta, 0.5, 1)
        _LONG_SEP.update(c=c, st=st)
    return _LONG_SEP["c"], _LONG_SEP["st"]


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("prec", [0, 1])
def test_long_separator_levels(prec, graph):
    """Sweep levels longer than the sweep kernels' register-held terms (the top separator of
    288 DOFs and the boundaries of the level below it take the kernels that stage their
    operator tile in shared memory), in the rebuild and the MPM-2P interface solves: 144^2,
    9 x 9 subdomains, init and 6 Algorithm 1 steps with a rebuild among them, against the
    oracle."""
    eta, steps = 0.003, 6
    c, st = _long_sep_trajectory(eta, steps)
    ctx = _gpu(c, prec)
    ctx.set_execution(graph, True)
    ctx.init(eta)
    for _ in range(steps):
        ctx.step(eta, 0.5, 1)
    n_reb = sum(1 for h in st.history if h["rebuild"])
    assert n_reb >= 1
    assert ctx.get_stats()["rebuilds"] == n_reb + 1
    tol = TOL[prec]
    ux, uy = ctx.get_flux()
    assert rel(ctx.get_saturation()[0], st.s) <= tol
    assert rel(ux[0], st.step.Fx) <= tol, rel(ux[0], st.step.Fx)
    assert rel(uy[0], st.step.Fy) <= tol + 1e-12, rel(uy[0], st.step.Fy)
    assert rel(ctx.get_pressure(0)[0], st.p_m) <= tol, rel(ctx.get_pressure(0)[0], st.p_m)
    assert rel(ctx.get_pressure(1)[0], st.step.p_down) <= tol, rel(ctx.get_pressure(1)[0], st.step.p_down)


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_max_side_trajectory(prec):
    """Subdomains with sides at the library's maximum (24 x 24 cells: a 32-wide padded factor of
    24 block rows, read in place because staged it would not fit in shared memory; in the
    tensor-core mode their basis solves take the float32 CUDA-core path) through the step graph:
    init and 8 Algorithm 1 steps with both kinds of update, against the oracle."""
    c = case("max_side", "zero")
    prob, dec = _oracle_setup(c)
    eta, steps = 0.02, 8
    st = O.simulate_init(c["K"], c["s0"], prob, dec, eta)
    ctx = _gpu(c, prec)
    ctx.init(eta)
    for _ in range(steps):
        O.simulate_step(st, c["K"], prob, dec, eta, 0.5, 1)
        ctx.step(eta, 0.5, 1)
    n_reb = sum(1 for h in st.history if h["rebuild"])
    assert 0 < n_reb < steps - 1  # both kinds of update occur
    assert ctx.get_stats()["rebuilds"] == n_reb + 1
    tol = TOL[prec]
    ux, uy = ctx.get_flux()
    assert rel(ctx.get_saturation()[0], st.s) <= tol
    assert rel(ux[0], st.step.Fx) <= tol, rel(ux[0], st.step.Fx)
    assert rel(uy[0], st.step.Fy) <= tol + 1e-12, rel(uy[0], st.step.Fy)
    assert rel(ctx.get_pressure(0)[0], st.p_m) <= tol, rel(ctx.get_pressure(0)[0], st.p_m)
    assert rel(ctx.get_pressure(1)[0], st.step.p_down) <= tol, rel(ctx.get_pressure(1)[0], st.step.p_down)


@pytest.mark.parametrize("name,eta,steps", [("contrast64", 0.05, 20), ("uneven", 0.02, 12)])
def test_downscale_factor_reuse(name, eta, steps):
    """Kept float32 downscaling factors (mpm_set_downscale_reuse): the float64 refinement runs
    against the current operator, so the trajectory matches the oracle at the mixed form's
    tolerance and the every-step refactorisation to the refinement's accuracy, with fewer
    factorisations (the front has not reached most subdomains, whose kappa^n does not change)."""
    c = case(name, "zero")
    prob, dec = _oracle_setup(c)
    st = O.simulate_init(c["K"], c["s0"], prob, dec, eta)
    for _ in range(steps):
        O.simulate_step(st, c["K"], prob, dec, eta, 0.5, 1)
    nsub = len(c["col_w"]) * len(c["row_h"])
    runs = {}
    for tol in (0.0, 0.05):
        ctx = _gpu(c, 1)
        ctx.set_downscale_reuse(tol)
        ctx.init(eta)
        for _ in range(steps):
            ctx.step(eta, 0.5, 1)
        ux, uy = ctx.get_flux()
        runs[tol] = (ux[0], uy[0], ctx.get_saturation()[0], ctx.get_stats())
        ctx.close()
    assert runs[0.0][3]["ds_factorisations"] == nsub * (steps + 1)
    assert runs[0.05][3]["ds_factorisations"] < nsub * (steps + 1)
    for ux, uy, s, _ in runs.values():
        assert rel(ux, st.step.Fx) <= TOL[1], rel(ux, st.step.Fx)
        assert rel(uy, st.step.Fy) <= TOL[1] + 1e-12, rel(uy, st.step.Fy)
        assert rel(s, st.s) <= TOL[1], rel(s, st.s)
        # per-cell balance within the refinement's stopping rule (1e3 ir_tol of the flux scale)
        assert _balance(ux, uy, prob) <= 4e-11
    assert rel(runs[0.05][0], runs[0.0][0]) <= 1e-10
    assert rel(runs[0.05][1], runs[0.0][1]) <= 1e-10


def test_downscale_reuse_rejects_out_of_range():
    c = case("single")
    ctx = _gpu(c, 1)
    for bad in (0.6, float("nan")):
        with pytest.raises(RuntimeError):
            ctx.set_downscale_reuse(bad)
    ctx.set_downscale_reuse(-1.0)  # the default
    ctx.close()


@pytest.mark.parametrize("graph", [True, False])
def test_algorithm1_twenty_transport_substeps(graph):
    # C_n = 20 transport steps between pressure updates (Section 5.1): the pressure step is
    # Delta t_p = C_n Delta t_s with Delta t_s the CFL step of the current fluxes, so it adapts
    # to the flow; the trajectory against the oracle's with the same C_n
    c = case("p1_2x2", "zero")
    prob, dec = _oracle_setup(c)
    eta, steps, n_sub = 0.02, 5, 20
    st = O.simulate_init(c["K"], c["s0"], prob, dec, eta)
    ctx = _gpu(c, 1)
    ctx.set_execution(graph, True)
    ctx.init(eta)
    for _ in range(steps):
        O.simulate_step(st, c["K"], prob, dec, eta, 0.5, n_sub)
        ctx.step(eta, 0.5, n_sub)
    assert ctx.get_stats()["rebuilds"] == 1 + sum(1 for h in st.history if h["rebuild"])
    assert ctx.get_stats()["last_dt_min"] == pytest.approx(st.history[-1]["dt"], rel=1e-8)
    assert rel(ctx.get_saturation()[0], st.s) <= 1e-8
    ux, uy = ctx.get_flux()
    assert rel(ux[0], st.step.Fx) <= 1e-8 and rel(uy[0], st.step.Fy) <= 1e-8 + 1e-12


def test_graph_replay_mixed_branches_across_realisations():
    # R = 3 realisations whose decisions differ step by step: the graph's two conditional
    # bodies both run and each kernel acts only on its own realisations.
    c = case("p1_2x2", "zero")
    prob, dec = _oracle_setup(c)
    from paper_2103_11050_gb300 import fields
    Ks = [fields.lognormal_grf(c["nx"], c["ny"], c["h"], 1.0 + r, 0.2, "exponential", 60 + r) for r in range(3)]
    etas = 0.03
    sts = [O.simulate_init(K, c["s0"], prob, dec, etas) for K in Ks]
    ctx = _gpu(c, 1, R=3, K=np.stack(Ks))
    ctx.init(etas)
    for _ in range(10):
        for r in range(3):
            O.simulate_step(sts[r], Ks[r], prob, dec, etas, 0.5, 1)
        ctx.step(etas, 0.5, 1)
    ux, _ = ctx.get_flux()
    s = ctx.get_saturation()
    reb = sum(sum(1 for h in st.history if h["rebuild"]) for st in sts)
    assert ctx.get_stats()["rebuilds"] == reb + 3
    for r in range(3):
        assert rel(ux[r], sts[r].step.Fx) <= 1e-8
        assert rel(s[r], sts[r].s) <= 1e-8


def test_realisations_are_independent():
    c = case("p1_2x2")
    prob, dec = _oracle_setup(c)
    from paper_2103_11050_gb300 import fields
    Ks = np.stack([fields.lognormal_grf(c["nx"], c["ny"], c["h"], 1.0, 0.2, "exponential", 40 + r) for r in range(3)])
    ctx = _gpu(c, 0, R=3, K=Ks)
    ctx.init(0.1)
    ux, uy = ctx.get_flux()
    for r in range(3):
        step, _, _ = O.mrcm_step(O.mobility(c["s0"], c["M"]) * Ks[r], prob, dec)
        assert rel(ux[r], step.Fx) <= 1e-10


def test_alpha_face_rejects_non_positive_values_on_interface_faces():
    # only interface faces are read: a zero elsewhere is accepted, a zero on an interface face is not
    from paper_2103_11050_gb300 import binding as B
    c = case("uneven")
    ax, ay = np.ones((c["ny"], c["nx"] + 1)), np.ones((c["ny"] + 1, c["nx"]))
    ax[:, 0] = 0.0  # the left boundary: not an interface
    ctx = _gpu(c, 0)
    ctx.set_decomposition(c["col_w"], c["row_h"], c["seg_len"], c["degree"], 1.0, (ax, ay))
    ax[3, c["col_w"][0]] = -1.0  # a face of the first vertical interface
    with pytest.raises(B.MPMError) as ei:
        ctx.set_decomposition(c["col_w"], c["row_h"], c["seg_len"], c["degree"], 1.0, (ax, ay))
    assert ei.value.code == B.MPM_ERR_ARG


def test_decomposition_rejects_out_of_range_geometry():
    # sides beyond 24 cells, sides that are not multiples of seg_len, and linear interface
    # spaces on one-edge segments (whose linear basis function vanishes at the edge midpoint)
    from paper_2103_11050_gb300 import binding as B
    c = case("max_side")
    ctx = _gpu(c, 0)
    for cw, rh, seg, deg in (([28, 28], [24, 24], 4, 1), ([26, 30], [24, 24], 4, 1), (c["col_w"], c["row_h"], 1, 1)):
        with pytest.raises(B.MPMError) as ei:
            ctx.set_decomposition(cw, rh, seg, deg, 1.0)
        assert ei.value.code == B.MPM_ERR_ARG
    ctx.set_decomposition(c["col_w"], c["row_h"], 1, 0, 1.0)  # one-edge constant segments are fine


def test_refinement_cap_reports_not_converged():
    # one refinement sweep cannot reach 1e-15 with an FP32 factor (nor its 1e3 x floor): the library must say so
    from paper_2103_11050_gb300 import binding as B
    c = case("contrast64")
    ctx = _gpu(c, 2)
    ctx.set_precision(2, 1e-15, 1)
    ctx.init(0.1)
    with pytest.raises(B.MPMError) as ei:
        ctx.sync()
    assert ei.value.code == B.MPM_ERR_NOT_CONVERGED


def test_rejected_saturation_leaves_state_unchanged():
    # a saturation outside [0,1] is refused before it replaces the current one: the state read
    # back is unchanged and the next steps match, bit for bit, a context that never saw the call
    from paper_2103_11050_gb300 import binding as B
    c = case("contrast64")
    ctxs = [_gpu(c, 1), _gpu(c, 1)]
    for ctx in ctxs:
        ctx.init(0.1)
        ctx.step(0.1, 0.5, 1)
    before = ctxs[0].get_saturation()
    bad = before.copy()
    bad[0, 7, 9] = 1.5
    with pytest.raises(B.MPMError) as ei:
        ctxs[0].set_saturation(bad)
    assert ei.value.code == B.MPM_ERR_ARG
    assert np.array_equal(ctxs[0].get_saturation(), before)
    for ctx in ctxs:
        ctx.set_saturation(before)
        for _ in range(3):
            ctx.step(0.1, 0.5, 1)
    s0, s1 = ctxs[0].get_saturation(), ctxs[1].get_saturation()
    ux0, _ = ctxs[0].get_flux()
    ux1, _ = ctxs[1].get_flux()
    assert np.array_equal(s0, s1) and np.array_equal(ux0, ux1)


def test_pinned_host_buffers_match_pageable():
    # pinned host buffers take kernel transfers (no copy engine), pageable ones a copy: the
    # same values either way, and the same range check on the way in
    import torch
    from paper_2103_11050_gb300 import binding as B
    c = case("contrast64")
    shape = (1, c["ny"], c["nx"])
    ctxs = [_gpu(c, 1), _gpu(c, 1)]
    for ctx in ctxs:
        ctx.init(0.1)
        ctx.step(0.1, 0.5, 1)
    pinned = torch.empty(shape, dtype=torch.float64).pin_memory().numpy()
    ctxs[0].get_saturation(pinned)
    pageable = ctxs[1].get_saturation()
    assert np.array_equal(pinned, pageable)
    pinned[0, 3, 5] = -0.25
    with pytest.raises(B.MPMError) as ei:
        ctxs[0].set_saturation(pinned)
    assert ei.value.code == B.MPM_ERR_ARG and "index" in str(ei.value)
    pinned[0, 3, 5] = pageable[0, 3, 5]
    ctxs[0].set_saturation(pinned)
    ctxs[1].set_saturation(pageable)
    # the pinned path computes only f(s) on the way in; kappa^n follows on demand
    assert np.array_equal(ctxs[0].get_conductivity(), ctxs[1].get_conductivity())
    for _ in range(3):
        for ctx in ctxs:
            ctx.step(0.1, 0.5, 1)
    ux_p = torch.empty((1, c["ny"], c["nx"] + 1), dtype=torch.float64).pin_memory().numpy()
    uy_p = torch.empty((1, c["ny"] + 1, c["nx"]), dtype=torch.float64).pin_memory().numpy()
    ctxs[0].get_flux(ux_p, uy_p)
    ux, uy = ctxs[1].get_flux()
    assert np.array_equal(ux_p, ux) and np.array_equal(uy_p, uy)
    ctxs[0].get_saturation(pinned)
    assert np.array_equal(pinned, ctxs[1].get_saturation())
