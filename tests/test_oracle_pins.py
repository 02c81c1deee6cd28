"""Pins of the CPU oracle against facts fixed by the paper or by mathematics.

Each test checks the oracle against something other than itself: closed forms,
brute force, special cases the paper states (one subdomain, H_bar = h), exact
identities of the method (static condensation, defect correction), printed
numbers (Section 4.3, Table 1) and invariants (conservation, bounds).
"""
import os

import numpy as np
import pytest

from oracle import mpm_oracle as O
from paper_2103_11050_gb300 import fields

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _prob(nx, ny, M=2.0, bc_type=(O.DIRICHLET, O.DIRICHLET, O.NEUMANN, O.NEUMANN),
          bc_val=(1.0, 0.0, 0.0, 0.0), q=None):
    return O.Problem(nx, ny, 1.0 / nx, tuple(bc_type), tuple(bc_val), M, 1.0, q)


def _field(nx, ny, seed=7, sigma2=1.0):
    return fields.lognormal_grf(nx, ny, 1.0 / nx, sigma2, 0.2, "exponential", seed)


# ---------------------------------------------------------------- coefficients

@pytest.mark.parametrize("M", [0.5, 1.0, 4.0, 5.0, 10.0, 40.0])
def test_max_frac_flow_deriv_bruteforce(M):
    s = np.linspace(0.0, 1.0, 400001)
    sampled = float(np.max(O.frac_flow_deriv(s, M)))
    exact = O.max_frac_flow_deriv(M)
    assert sampled <= exact * (1 + 1e-12)
    assert exact <= sampled * (1 + 1e-8)


def test_max_frac_flow_deriv_M1():
    # M = 1: f = s^2 / (s^2 + (1-s)^2) has its steepest point at s = 1/2, f'(1/2) = 2.
    assert O.max_frac_flow_deriv(1.0) == pytest.approx(2.0, rel=1e-14)


def test_mobility_fraction_endpoints():
    M = 5.0
    assert O.mobility(0.0, M) == 1.0 and O.mobility(1.0, M) == M
    assert O.frac_flow(0.0, M) == 0.0 and O.frac_flow(1.0, M) == 1.0
    # f = lambda_w / lambda with lambda_w = M s^2 (Section 2 and Section 5)
    s = 0.3
    assert O.frac_flow(s, M) == pytest.approx(M * s * s / O.mobility(s, M))


# ---------------------------------------------------------------- fine grid

def test_fine_linear_pressure_homogeneous():
    # Homogeneous medium, p = 1 left / 0 right, no flow top and bottom: p = 1 - x exactly,
    # integrated flux through each x-face = kappa * h * (1 / L) * L = kappa h (unit square).
    nx, ny, kap = 12, 7, 3.7
    prob = O.Problem(nx, ny, 1.0 / nx, (O.DIRICHLET, O.DIRICHLET, O.NEUMANN, O.NEUMANN), (1.0, 0.0, 0.0, 0.0))
    kappa = np.full((ny, nx), kap)
    p = O.fine_solve(kappa, prob)
    x = (np.arange(nx) + 0.5) / nx
    np.testing.assert_allclose(p, np.broadcast_to(1.0 - x, (ny, nx)), atol=1e-13)
    Fx, Fy = O.fine_fluxes(p, kappa, prob)
    np.testing.assert_allclose(Fx, kap * prob.h * np.ones_like(Fx) * nx * prob.h, rtol=1e-12)
    np.testing.assert_allclose(Fy, 0.0, atol=1e-13)


def test_fine_series_resistance_strip():
    # 1-D strip of 3 cells = resistors in series: half-cell 1/(2 k1), faces 1/(2k_i)+1/(2k_{i+1}),
    # half-cell 1/(2 k3).  The flux is (p_left - p_right) / total resistance.
    k = np.array([[1.0, 10.0, 0.1]])
    prob = O.Problem(3, 1, 1.0 / 3, (O.DIRICHLET, O.DIRICHLET, O.NEUMANN, O.NEUMANN), (2.0, -1.0, 0.0, 0.0))
    p = O.fine_solve(k, prob)
    Rtot = 1 / (2 * 1.0) + (1 / 2 + 1 / 20) + (1 / 20 + 1 / 0.2) + 1 / (2 * 0.1)
    flux = 3.0 / Rtot
    Fx, _ = O.fine_fluxes(p, k, prob)
    np.testing.assert_allclose(Fx[0], flux, rtol=1e-13)
    # pressure drop over the left half cell
    assert p[0, 0] == pytest.approx(2.0 - flux / 2.0, rel=1e-13)


def test_fine_solve_minimises_discrete_energy():
    # Brute force on a small heterogeneous grid: the two-point equations are the optimality
    # conditions of the discrete energy
    #   E(p) = 1/2 sum_interior T_f (p_a - p_b)^2 + sum_Dirichlet kappa_c (p_c - g)^2
    #          - sum_c q_c h^2 p_c + sum_Neumann z h p_c,
    # with T_f the series conductance of the two half cells (each 2 kappa).  The energy is
    # written here face by face, independently of the oracle's assembly; its gradient (central
    # differences, exact for a quadratic up to rounding) must vanish at the oracle's solution,
    # and every perturbation must raise it.
    nx, ny, h = 5, 4, 0.25
    rng = np.random.default_rng(11)
    kappa = np.exp(rng.normal(0.0, 1.5, (ny, nx)))
    q = rng.normal(0.0, 1.0, (ny, nx))
    prob = O.Problem(nx, ny, h, (O.DIRICHLET, O.DIRICHLET, O.NEUMANN, O.NEUMANN), (1.3, -0.4, 0.7, -0.2), M=1.0,
                     q=q)
    p_star = O.fine_solve(kappa, prob)

    def energy(p):
        e = 0.0
        for j in range(ny):
            for i in range(nx):
                for (ii, jj) in ((i + 1, j), (i, j + 1)):
                    if ii < nx and jj < ny:
                        t = 1.0 / (1.0 / (2.0 * kappa[j, i]) + 1.0 / (2.0 * kappa[jj, ii]))
                        e += 0.5 * t * (p[j, i] - p[jj, ii]) ** 2
                e -= q[j, i] * h * h * p[j, i]
        for j in range(ny):
            e += kappa[j, 0] * (p[j, 0] - 1.3) ** 2 + kappa[j, nx - 1] * (p[j, nx - 1] + 0.4) ** 2
        for i in range(nx):
            e += 0.7 * h * p[0, i] - 0.2 * h * p[ny - 1, i]
        return e

    step = 1e-3
    grad = np.zeros((ny, nx))
    for j in range(ny):
        for i in range(nx):
            d = np.zeros((ny, nx))
            d[j, i] = step
            grad[j, i] = (energy(p_star + d) - energy(p_star - d)) / (2.0 * step)
    scale = float(np.max(kappa) * np.max(np.abs(p_star)))
    assert np.max(np.abs(grad)) <= 1e-9 * scale
    e0 = energy(p_star)
    for _ in range(5):
        assert energy(p_star + 0.05 * rng.normal(size=(ny, nx))) > e0


def test_fine_matrix_spd():
    prob = _prob(6, 5)
    A, _ = O.fine_system(_field(6, 5), prob)
    A = A.toarray()
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-14)
    assert np.min(np.linalg.eigvalsh(A)) > 0


def test_fine_neumann_rate_bc():
    # Left side Neumann with inflow z = -u.n = 1 (u.n = -1), right Dirichlet 0:
    # p = (L - x) * 1 / kappa and total flux = 1 per unit length.
    nx, ny, kap = 8, 3, 2.0
    prob = O.Problem(nx, ny, 1.0 / nx, (O.NEUMANN, O.DIRICHLET, O.NEUMANN, O.NEUMANN), (-1.0, 0.0, 0.0, 0.0))
    p = O.fine_solve(np.full((ny, nx), kap), prob)
    x = (np.arange(nx) + 0.5) / nx
    np.testing.assert_allclose(p[0], (1.0 - x) / kap, atol=1e-13)


# ---------------------------------------------------------------- MRCM

def _alpha_field(nx, ny, seed, lo=0.1, hi=10.0):
    """A seeded per-face alpha(x) (log-uniform in [lo, hi]): (alpha_x [ny][nx+1], alpha_y [ny+1][nx])."""
    rng = np.random.default_rng(seed)
    return (np.exp(rng.uniform(np.log(lo), np.log(hi), (ny, nx + 1))),
            np.exp(rng.uniform(np.log(lo), np.log(hi), (ny + 1, nx))))


@pytest.mark.parametrize("alpha", [0.5, 1.0, 4.0, "field"])
def test_local_robin_solve_reproduces_linear_pressure(alpha):
    # Local problem (Eq. mrc1) in a homogeneous medium with the Robin data of an exact linear
    # pressure p = 1 + gx x + gy y.  The Robin condition -beta u.n + lambda = g with
    # beta = alpha H / kappa (Eq. beta) and u = -kappa grad p gives g = p(face) +
    # alpha H dp/dn on each interface face; two-point fluxes are exact for linear fields, so
    # the local solve must return the field at the cell centres and the exact integrated
    # outward fluxes.  The subdomain (bottom middle of 3 x 3) has three interface sides and a
    # physical Neumann side carrying the field's outward velocity.
    nx, ny = 24, 18
    h = 1.0 / nx
    kap, gx, gy = 2.5, 0.3, -0.7
    field = lambda x, y: 1.0 + gx * x + gy * y
    # outward normal derivative of p and outward velocity u.n per side (left, right, bottom, top)
    dpdn = {O.LEFT: -gx, O.RIGHT: gx, O.BOTTOM: -gy, O.TOP: gy}
    prob = O.Problem(nx, ny, h, (O.DIRICHLET, O.DIRICHLET, O.NEUMANN, O.NEUMANN),
                     (1.0, 0.0, -kap * dpdn[O.BOTTOM], -kap * dpdn[O.TOP]), M=1.0)
    # alpha is a constant, or (aMRCM) varies face by face: the Robin datum then carries each
    # face's own alpha, and the local solve must still return the linear field
    af = _alpha_field(nx, ny, 17) if alpha == "field" else None
    dec = O.Decomposition(nx, ny, [8, 8, 8], [6, 6, 6], 2, 1, 1.0 if af else alpha, af)
    sd = dec.subs[1]
    assert [side.kind for side in sd.sides] == ["iface", "iface", "phys", "iface"]
    kappa = np.full((ny, nx), kap)
    g_faces = []
    for side in sd.sides:
        g = []
        for (j, i) in side.gcells:
            xf, yf = (i + 0.5) * h, (j + 0.5) * h
            if side.which == O.LEFT:
                xf = i * h
                a_e = af[0][j, i] if af else alpha
            elif side.which == O.RIGHT:
                xf = (i + 1) * h
                a_e = af[0][j, i + 1] if af else alpha
            elif side.which == O.BOTTOM:
                yf = j * h
                a_e = af[1][j, i] if af else alpha
            else:
                yf = (j + 1) * h
                a_e = af[1][j + 1, i] if af else alpha
            g.append(field(xf, yf) + a_e * side.length * h * dpdn[side.which])
        g_faces.append(np.array(g))
    A = O.local_matrix(kappa, prob, dec, sd)
    rhs = O.local_rhs(kappa, prob, dec, sd, np.zeros(sd.m), g_faces)
    p_loc = np.linalg.solve(A, rhs)
    jl, il = np.divmod(np.arange(sd.m), sd.a)
    exact = field((sd.x0 + il + 0.5) * h, (sd.y0 + jl + 0.5) * h)
    np.testing.assert_allclose(p_loc, exact, rtol=1e-12, atol=1e-12)
    for side, tr in zip(sd.sides, O.local_traces(p_loc, kappa, prob, dec, sd, g_faces)):
        np.testing.assert_allclose(tr, h * (-kap * dpdn[side.which]), rtol=1e-11, atol=1e-13)


def test_mrcm_single_subdomain_equals_fine():
    nx, ny = 12, 8
    prob = _prob(nx, ny)
    kappa = _field(nx, ny)
    dec = O.Decomposition(nx, ny, [nx], [ny], seg_len=4, degree=1)
    step, _, _ = O.mrcm_step(kappa, prob, dec)
    p_ref = O.fine_solve(kappa, prob)
    Fx, Fy = O.fine_fluxes(p_ref, kappa, prob)
    np.testing.assert_allclose(step.p_level, p_ref, atol=1e-12)
    np.testing.assert_allclose(step.Fx, Fx, atol=1e-12)
    np.testing.assert_allclose(step.Fy, Fy, atol=1e-12)


@pytest.mark.parametrize("alpha", [0.1, 1.0, 10.0, "field"])
def test_mrcm_hbar_h_equals_fine(alpha):
    # Section 5.4: MRCM with H_bar = h and constant spaces equals the undecomposed solution,
    # for any alpha, also one that varies face by face (aMRCM).
    nx, ny = 12, 10
    prob = _prob(nx, ny, bc_val=(1.0, -0.5, 0.0, 0.0))
    kappa = _field(nx, ny, seed=3, sigma2=2.0)
    af = _alpha_field(nx, ny, 23) if alpha == "field" else None
    dec = O.Decomposition(nx, ny, [4, 8], [6, 4], seg_len=1, degree=0, alpha=1.0 if af else alpha, alpha_face=af)
    step, _, _ = O.mrcm_step(kappa, prob, dec)
    p_ref = O.fine_solve(kappa, prob)
    Fx, Fy = O.fine_fluxes(p_ref, kappa, prob)
    np.testing.assert_allclose(step.p_level, p_ref, atol=1e-11)
    np.testing.assert_allclose(step.Fx, Fx, atol=1e-11)
    np.testing.assert_allclose(step.Fy, Fy, atol=1e-11)


@pytest.mark.parametrize("direction", ["x", "y"])
def test_mrcm_p1_reproduces_linear_pressure(direction):
    # A linear pressure in a homogeneous medium has linear interface traces, which the
    # piecewise-linear spaces contain; constant spaces on 4-edge segments do not.
    nx = ny = 16
    if direction == "x":
        bct, bcv = (O.DIRICHLET, O.DIRICHLET, O.NEUMANN, O.NEUMANN), (1.0, 0.0, 0.0, 0.0)
    else:
        bct, bcv = (O.NEUMANN, O.NEUMANN, O.DIRICHLET, O.DIRICHLET), (0.0, 0.0, 1.0, 0.0)
    prob = O.Problem(nx, ny, 1.0 / nx, bct, bcv)
    kappa = np.full((ny, nx), 2.5)
    p_ref = O.fine_solve(kappa, prob)
    dec1 = O.uniform_decomposition(nx, ny, 2, 2, seg_len=4, degree=1)
    step1, _, _ = O.mrcm_step(kappa, prob, dec1)
    np.testing.assert_allclose(step1.p_level, p_ref, atol=1e-12)
    dec0 = O.uniform_decomposition(nx, ny, 2, 2, seg_len=4, degree=0)
    step0, _, _ = O.mrcm_step(kappa, prob, dec0)
    assert np.max(np.abs(step0.p_level - p_ref)) > 1e-6


@pytest.mark.parametrize("alpha,degree,seg", [(1.0, 1, 4), (0.5, 0, 4), (2.0, 1, 2), ("field", 1, 4)])
def test_mrcm_basis_route_equals_monolithic(alpha, degree, seg):
    nx, ny = 16, 12
    prob = _prob(nx, ny, bc_val=(1.0, 0.0, 0.0, 0.0))
    kappa = _field(nx, ny, seed=11, sigma2=2.0)
    af = _alpha_field(nx, ny, 29) if alpha == "field" else None
    dec = O.Decomposition(nx, ny, [4, 8, 4], [8, 4], seg_len=seg, degree=degree, alpha=1.0 if af else alpha,
                          alpha_face=af)
    sol, _ = O.mrcm_solve(kappa, prob, dec)
    p_mono, c_mono = O.mrcm_monolithic(kappa, prob, dec)
    scale = np.max(np.abs(p_mono))
    np.testing.assert_allclose(sol.p, p_mono, atol=1e-12 * scale)
    np.testing.assert_allclose(sol.coeffs, c_mono, atol=1e-10 * np.max(np.abs(c_mono)))


@pytest.mark.parametrize("col_w,row_h,seg", [([24, 8], [24], 4), ([4, 8, 4], [2, 6, 4], 2)])
def test_mrcm_basis_route_equals_monolithic_extreme_sides(col_w, row_h, seg):
    # the subdomain sides at the extremes of the GPU parity cases (24 cells; 2 cells, one block
    # row pair): the basis-function route still equals the monolithic solve of Eqs. (mrc1)+(mrc2)
    nx, ny = sum(col_w), sum(row_h)
    prob = _prob(nx, ny, bc_val=(1.0, 0.0, 0.0, 0.0))
    kappa = _field(nx, ny, seed=13, sigma2=2.0)
    dec = O.Decomposition(nx, ny, col_w, row_h, seg_len=seg, degree=1, alpha=1.0)
    sol, _ = O.mrcm_solve(kappa, prob, dec)
    p_mono, c_mono = O.mrcm_monolithic(kappa, prob, dec)
    np.testing.assert_allclose(sol.p, p_mono, atol=1e-12 * np.max(np.abs(p_mono)))
    np.testing.assert_allclose(sol.coeffs, c_mono, atol=1e-10 * np.max(np.abs(c_mono)))


@pytest.mark.parametrize("varying", [False, True])
def test_interface_matrix_symmetric(varying):
    # With the flux-weighted rows negated, Eq. (mrc2) tested with the BFs is symmetric (also
    # with alpha varying face by face: both sides of an interface face share its alpha).
    nx, ny = 16, 16
    prob = _prob(nx, ny)
    kappa = _field(nx, ny, seed=5, sigma2=3.0)
    af = _alpha_field(nx, ny, 31) if varying else None
    dec = O.uniform_decomposition(nx, ny, 2, 2, seg_len=4, degree=1, alpha=1.0, alpha_face=af)
    bs = O.build_basis(kappa, prob, dec)
    K = bs.K.toarray()
    assert np.max(np.abs(K - K.T)) <= 1e-11 * np.max(np.abs(K))


def test_n_hat_counts():
    # Section 4.3: 4x4 subdomains with k_U = k_P = 1 give N_hat = 96.
    dec = O.uniform_decomposition(64, 64, 4, 4, seg_len=16, degree=0)
    assert dec.n_hat() == 96
    # Constant spaces on H/2 double it; piecewise linear on 4-edge segments: 16 per interface.
    assert O.uniform_decomposition(64, 64, 4, 4, seg_len=8, degree=0).n_hat() == 192
    assert O.uniform_decomposition(64, 64, 4, 4, seg_len=4, degree=1).n_hat() == 768


def test_rcr_paper_values():
    with open(os.path.join(GOLDEN, "rcr_paper.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            parts = line.split()
            Te, Tm, Nh, N, val, dec = int(parts[0]), int(parts[1]), int(parts[2]), int(parts[3]), float(parts[4]), int(parts[5])
            assert round(O.rcr(Te, Tm, Nh, N), dec) == pytest.approx(val, abs=0.5 * 10 ** -dec)


# ---------------------------------------------------------------- downscaling

def test_downscale_conservative_and_compatible():
    nx, ny = 16, 16
    prob = _prob(nx, ny, M=3.0)
    kappa = _field(nx, ny, seed=2, sigma2=4.0)
    dec = O.uniform_decomposition(nx, ny, 4, 2, seg_len=4, degree=1)
    step, _, sol = O.mrcm_step(kappa, prob, dec)
    bal = O.cell_balance(step.Fx, step.Fy, prob)
    assert np.max(np.abs(bal)) <= 1e-12 * np.max(np.abs(step.Fx))
    # the boundary fluxes given to each Neumann problem are compatible (sum = 0, no source)
    for sd in dec.subs:
        tot = (np.sum(sol.ubar_x[sd.y0:sd.y0 + sd.b, sd.x0 + sd.a]) - np.sum(sol.ubar_x[sd.y0:sd.y0 + sd.b, sd.x0])
               + np.sum(sol.ubar_y[sd.y0 + sd.b, sd.x0:sd.x0 + sd.a]) - np.sum(sol.ubar_y[sd.y0, sd.x0:sd.x0 + sd.a]))
        assert abs(tot) <= 1e-12 * np.max(np.abs(step.Fx))
    # pressure constant: subdomain means of the downscaled and MRCM-level pressure agree
    for sd in dec.subs:
        blk = np.s_[sd.y0:sd.y0 + sd.b, sd.x0:sd.x0 + sd.a]
        assert np.mean(step.p_down[blk]) == pytest.approx(np.mean(step.p_level[blk]), abs=1e-13)


def test_downscale_of_fine_fluxes_is_identity():
    # Given the exact fine fluxes on subdomain boundaries, the Neumann problems return
    # the fine pressure (up to the constant) and the fine interior fluxes.
    nx, ny = 12, 12
    prob = _prob(nx, ny)
    kappa = _field(nx, ny, seed=4)
    dec = O.uniform_decomposition(nx, ny, 3, 2, seg_len=2, degree=1)
    p = O.fine_solve(kappa, prob)
    Fx, Fy = O.fine_fluxes(p, kappa, prob)
    pt, Fx2, Fy2 = O.downscale(kappa, Fx, Fy, p, prob, dec)
    np.testing.assert_allclose(pt, p, atol=1e-12)
    np.testing.assert_allclose(Fx2, Fx, atol=1e-12)
    np.testing.assert_allclose(Fy2, Fy, atol=1e-12)


# ---------------------------------------------------------------- MPM-2P

def test_mpm_exact_when_mrcm_exact_and_kappa_unchanged():
    nx, ny = 12, 12
    prob = _prob(nx, ny, M=4.0)
    K = _field(nx, ny, seed=9, sigma2=2.0)
    dec = O.uniform_decomposition(nx, ny, 3, 3, seg_len=1, degree=0)
    s = np.clip(np.random.default_rng(1).random((ny, nx)), 0, 1)
    kappa = O.mobility(s, prob.M) * K
    step_m, bs, sol = O.mrcm_step(kappa, prob, dec)
    step_n, _ = O.mpm_step(kappa, bs, sol.p, prob, dec)
    p_ref = O.fine_solve(kappa, prob)
    Fx, Fy = O.fine_fluxes(p_ref, kappa, prob)
    np.testing.assert_allclose(step_n.p_level, p_ref, atol=1e-11)
    np.testing.assert_allclose(step_n.Fx, Fx, atol=1e-11)
    np.testing.assert_allclose(step_n.Fy, Fy, atol=1e-11)


def test_mpm_reuse_route_equals_monolithic():
    # The epsilon^0 problem solved with the stored BFs equals a fresh monolithic MRCM solve
    # of Eq. (mpm_tf_3) with kappa^m (source r, homogeneous physical data).
    nx, ny = 16, 12
    prob = _prob(nx, ny, M=5.0)
    K = _field(nx, ny, seed=13, sigma2=2.0)
    dec = O.Decomposition(nx, ny, [8, 8], [4, 8], seg_len=4, degree=1)
    rng = np.random.default_rng(2)
    s_m = 0.5 * rng.random((ny, nx))
    s_n = np.clip(s_m + 0.1 * rng.random((ny, nx)), 0, 1)
    kap_m = O.mobility(s_m, prob.M) * K
    kap_n = O.mobility(s_n, prob.M) * K
    _, bs, sol = O.mrcm_step(kap_m, prob, dec)
    step_n, dsol = O.mpm_step(kap_n, bs, sol.p, prob, dec)
    r = O.fine_residual(kap_n, sol.p, prob)
    dp_mono, _ = O.mrcm_monolithic(kap_m, prob, dec, src=r, homogeneous_bc=True)
    np.testing.assert_allclose(dsol.p, dp_mono, atol=1e-12 * np.max(np.abs(sol.p)))
    bal = O.cell_balance(step_n.Fx, step_n.Fy, prob)
    assert np.max(np.abs(bal)) <= 1e-12 * np.max(np.abs(step_n.Fx))


@pytest.mark.parametrize("seg,degree,order", [(1, 0, 2), (4, 1, 1)])
def test_mpm_error_order_in_epsilon(seg, degree, order):
    # Section 4.1: MPM-2P keeps only the epsilon^0 problem, i.e. it replaces the operator
    # kappa^m + eps kappa_eps of Eq. (mpm_tf_2) by kappa^m.  Solving Eq. (mpm_tf_2) with
    # the full operator kappa^n (BFs rebuilt at kappa^n, same p^m) differs from MPM-2P by
    # O(eps) times the residual r.  With H_bar = h the MRCM is exact, the full-operator route
    # is the fine solution, p^m is exact for kappa^m and r = O(eps): the difference is
    # O(eps^2) (one defect-correction sweep).  With coarse spaces r = O(1): O(eps).
    nx, ny = 16, 16
    prob = _prob(nx, ny)
    kap_m = _field(nx, ny, seed=21)
    dec = O.uniform_decomposition(nx, ny, 2, 2, seg_len=seg, degree=degree)
    _, bs, sol = O.mrcm_step(kap_m, prob, dec)
    pert = 1.0 + np.sin(np.arange(nx * ny).reshape(ny, nx) * 0.37)
    errs = []
    for t in (1e-2, 5e-3, 2.5e-3):
        kap_n = kap_m * (1.0 + t * pert)
        mpm, _ = O.mpm_step(kap_n, bs, sol.p, prob, dec)
        full, _ = O.mpm_step(kap_n, O.build_basis(kap_n, prob, dec), sol.p, prob, dec)
        if seg == 1:
            p_ref = O.fine_solve(kap_n, prob)
            Fx, Fy = O.fine_fluxes(p_ref, kap_n, prob)
            np.testing.assert_allclose(full.Fx, Fx, atol=1e-11)
        errs.append(np.linalg.norm(mpm.Fx - full.Fx) + np.linalg.norm(mpm.Fy - full.Fy))
    assert errs[0] > 1e-9
    for k in range(2):
        assert 0.9 * 2 ** order < errs[k] / errs[k + 1] < 1.1 * 2 ** order


@pytest.mark.parametrize("alpha_field", [False, True])
def test_mpm_first_order_term_raises_the_order(alpha_field):
    # Eq. (mpm_tf_4), l = 1: with H_bar = h the MRCM is the exact fine solve, so the epsilon^0
    # update is one defect-correction sweep with error O(eps^2) (previous pin) and adding the
    # first-order term (source div(kappa_eps grad delta p_0), flux increment
    # u_hat_1 + (kappa^n - kappa^m) grad delta p_0) leaves O(eps^3).  A dropped flux increment
    # or a flipped source sign leaves O(eps^2) and fails the ratio.
    nx, ny = 16, 16
    prob = _prob(nx, ny)
    kap_m = _field(nx, ny, seed=21)
    af = _alpha_field(nx, ny, 37) if alpha_field else None
    dec = O.uniform_decomposition(nx, ny, 2, 2, seg_len=1, degree=0, alpha_face=af)
    _, bs, sol = O.mrcm_step(kap_m, prob, dec)
    pert = 1.0 + np.sin(np.arange(nx * ny).reshape(ny, nx) * 0.37)
    errs0, errs1 = [], []
    for t in (2e-2, 1e-2, 5e-3):
        kap_n = kap_m * (1.0 + t * pert)
        p_ref = O.fine_solve(kap_n, prob)
        Fx, Fy = O.fine_fluxes(p_ref, kap_n, prob)
        m0, _ = O.mpm_step(kap_n, bs, sol.p, prob, dec, order=0)
        m1, _ = O.mpm_step(kap_n, bs, sol.p, prob, dec, order=1)
        errs0.append(np.linalg.norm(m0.Fx - Fx) + np.linalg.norm(m0.Fy - Fy))
        errs1.append(np.linalg.norm(m1.Fx - Fx) + np.linalg.norm(m1.Fy - Fy))
    assert errs1[-1] < 1e-2 * errs0[-1]
    for k in range(2):
        assert 0.9 * 4 < errs0[k] / errs0[k + 1] < 1.1 * 4
        assert 0.85 * 8 < errs1[k] / errs1[k + 1] < 1.15 * 8


# ---------------------------------------------------------------- transport

def test_upwind_hand_step_strip():
    # 3x1 strip, unit integrated flux to the right everywhere, water enters at the left.
    prob = O.Problem(3, 1, 1.0 / 3, (O.DIRICHLET, O.DIRICHLET, O.NEUMANN, O.NEUMANN), (1, 0, 0, 0), M=1.0)
    Fx = np.ones((1, 4))
    Fy = np.zeros((2, 3))
    s = np.array([[0.0, 0.5, 1.0]])
    dt = 0.01
    s1 = O.upwind_step(s, Fx, Fy, dt, prob)
    f = lambda v: v * v / (v * v + (1 - v) ** 2)
    lam = dt / prob.h ** 2
    expect = [0.0 - lam * (f(0.0) - f(1.0)), 0.5 - lam * (f(0.5) - f(0.0)), 1.0 - lam * (f(1.0) - f(0.5))]
    np.testing.assert_allclose(s1[0], expect, rtol=1e-14)


def test_transport_mass_balance_and_bounds():
    nx, ny = 16, 16
    prob = _prob(nx, ny, M=5.0)
    K = _field(nx, ny, seed=8, sigma2=2.0)
    dec = O.uniform_decomposition(nx, ny, 2, 2)
    s = np.zeros((ny, nx))
    step, _, _ = O.mrcm_step(O.mobility(s, prob.M) * K, prob, dec)
    dt = O.cfl_dt(step.Fx, step.Fy, prob, 0.5)
    for _ in range(30):
        s1 = O.upwind_step(s, step.Fx, step.Fy, dt, prob)
        # boundary fluxes decide the change of total water volume
        # (top and bottom carry no flux)
        fl = O.frac_flow
        left = -step.Fx[:, 0]
        right = step.Fx[:, -1]
        bnd = (np.sum(np.where(left > 0, left * fl(s[:, 0], prob.M), left * fl(prob.s_inflow, prob.M)))
               + np.sum(np.where(right > 0, right * fl(s[:, -1], prob.M), right * fl(prob.s_inflow, prob.M))))
        dvol = (np.sum(s1) - np.sum(s)) * prob.h ** 2
        assert dvol == pytest.approx(-dt * bnd, rel=1e-12, abs=1e-15)
        assert np.all(s1 >= -1e-15) and np.all(s1 <= 1 + 1e-15)
        s = s1


def test_transport_constant_state_preserved():
    nx, ny = 10, 10
    prob = _prob(nx, ny)
    kappa = _field(nx, ny, seed=4)
    p = O.fine_solve(kappa, prob)
    Fx, Fy = O.fine_fluxes(p, kappa, prob)
    s = np.ones((ny, nx))  # equal to the injected saturation
    s1 = O.upwind_step(s, Fx, Fy, O.cfl_dt(Fx, Fy, prob, 0.5), prob)
    np.testing.assert_allclose(s1, 1.0, atol=1e-13)


def test_transport_converges_to_buckley_leverett():
    # 1D strip at unit total velocity, s = 0 initially, water (s = 1) injected at x = 0
    # (Eq. BL2D in one dimension).  The exact solution at injected pore volume Q is the
    # Buckley-Leverett profile with the Welge shock: the tangent condition f(s)/s = f'(s)
    # for f = M s^2 / (M s^2 + (1-s)^2) gives (M + 1) s^2 = 1, so s_f = 1/sqrt(M + 1); behind
    # the shock s solves f'(s) = x / Q.  First-order upwind converges to it in L1 (at about
    # half order across the shock), conserving the injected volume exactly.
    M, Q = 5.0, 0.3
    f = lambda v: M * v * v / (M * v * v + (1.0 - v) ** 2)

    def fprime(v, d=1e-6):  # central difference of f (independent of the oracle's f')
        lo, hi = max(v - d, 0.0), min(v + d, 1.0)
        return (f(hi) - f(lo)) / (hi - lo)

    def bisect(g, lo, hi):
        glo = g(lo) > 0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if (g(mid) > 0) == glo:
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)

    s_f = 1.0 / np.sqrt(M + 1.0)
    assert bisect(lambda v: fprime(v) * v - f(v), 1e-3, 1.0) == pytest.approx(s_f, abs=1e-6)
    xi_f = fprime(s_f)

    def exact(x):
        xi = x / Q
        return 0.0 if xi >= xi_f else bisect(lambda v: fprime(v) - xi, s_f, 1.0)

    errs = []
    for nx in (25, 50, 100, 200):
        h = 1.0 / nx
        prob = O.Problem(nx, 1, h, (O.DIRICHLET, O.DIRICHLET, O.NEUMANN, O.NEUMANN), (1, 0, 0, 0), M=M)
        Fx = np.full((1, nx + 1), h)  # integrated face flux h x unit velocity
        Fy = np.zeros((2, nx))
        dt = O.cfl_dt(Fx, Fy, prob, 0.5)
        s, t = np.zeros((1, nx)), 0.0
        while t < Q - 1e-15:
            step = min(dt, Q - t)
            s = O.upwind_step(s, Fx, Fy, step, prob)
            t += step
        assert h * np.sum(s) == pytest.approx(Q, abs=1e-12)  # front still inside: all water stays
        xc = (np.arange(nx) + 0.5) * h
        errs.append(h * float(np.sum(np.abs(s[0] - np.array([exact(x) for x in xc])))))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < errs[0] / 3.0 and errs[-1] < 0.012, errs


# ---------------------------------------------------------------- Algorithm 1

def test_epsilon_relative_l2():
    a = np.array([[1.0, 2.0], [3.0, 4.0]])
    assert O.epsilon(a, a) == 0.0
    assert O.epsilon(2 * a, a) == pytest.approx(1.0)
    assert O.epsilon(7 * (a + 0.1), 7 * a) == pytest.approx(O.epsilon(a + 0.1, a))


def test_algorithm1_decision_logic():
    # Algorithm 1: eps starts at eta and the test is strict, so step 1 reuses the BFs;
    # a rebuild happens one step after eps exceeds eta, and eps = 0 right after it.
    nx, ny = 16, 16
    prob = _prob(nx, ny, M=5.0)
    K = _field(nx, ny, seed=1)
    dec = O.uniform_decomposition(nx, ny, 2, 2)
    eta = 0.02
    st = O.simulate_init(K, np.zeros((ny, nx)), prob, dec, eta)
    for _ in range(12):
        O.simulate_step(st, K, prob, dec, eta, 0.5, 1)
    h = st.history
    assert h[0]["rebuild"] is False
    for k in range(1, len(h)):
        assert h[k]["rebuild"] == (h[k - 1]["eps"] > eta)
        if h[k]["rebuild"]:
            assert h[k]["eps"] == 0.0
    assert any(x["rebuild"] for x in h)
