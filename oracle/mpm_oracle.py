"""FP64 CPU oracle for MRCM and MPM-2P (Rocha, Mankad, Sousa, Pereira, arXiv 2103.11050).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py, never by the product package.

Everything is float64.  Each function cites the passage of the paper it states.
Where the paper is silent the reading taken is written next to the code:

* fine discretisation (Section 3, fluxes in F_h(E_h), P0 per edge): two-point
  flux on square cells, i.e. the lowest-order mixed method with trapezoidal
  quadrature; interior faces carry T = 2 ka kb / (ka + kb), a Dirichlet face
  carries 2 kc, a Neumann face carries its prescribed flux.
* fluxes are stored INTEGRATED over a face (h times the normal velocity);
  Fx[j][i] is the flux through the x-face left of cell (i, j) in +x direction,
  Fy[j][i] through the y-face below cell (i, j) in +y direction.
* mobility (Section 2, Section 5): k_rw = s^2, k_ro = (1 - s)^2, mu_o = 1,
  mu_w = 1 / M, so lambda(s) = M s^2 + (1 - s)^2 and f = M s^2 / lambda.
* Robin faces (Eq. mrc1 with Eq. beta): eliminating the face pressure between the
  half-cell flux and the Robin condition gives the integrated outward flux
  F_e = r_e (p_c - g_e) with r_e = kappa_c / (1/2 + rho_e), rho_e = alpha_e H_e / h
  (alpha constant, or given per interface face: the aMRCM's alpha(x), Section 3.1),
  and the Robin datum g_e = -(rho_e / kappa_c) s U_e + P_e, where U_e is the
  interface flux integrated over the face and s = n_check . n_check^i.
* H_e (the "characteristic size" in Eq. beta) is the length of the interface
  that carries the face.
* interface spaces (Section 3.1): discontinuous polynomials of degree 0 or 1 on
  segments of ``seg_len`` fine edges, Legendre basis {1, 2 xi - 1}, projected on
  P0 per edge by evaluation at the edge midpoints.  n_check is +x on vertical
  and +y on horizontal interfaces.
* interface equations (Eq. mrc2) use edge quadrature; the flux-weighted rows are
  multiplied by -1, which makes the assembled matrix symmetric.
* downscaling (Eq. mpm_upd) is used after MRCM rebuilds too, with the
  interface flux equal to the mean of the two one-sided traces; the pressure
  constant of each Neumann problem is fixed so that its subdomain mean equals the
  subdomain mean of the MRCM-level pressure of the same step.
* MPM residual (Eq. mpm_tf_3): r = b(kappa^n) - A(kappa^n) p^m on the fine grid,
  with p^m the MRCM-level pressure of the last rebuild; the epsilon^0 problem is
  then solved by MRCM with kappa^m, source r and homogeneous physical data.
* epsilon (Section 4.1, Algorithm 1): relative discrete L2 norm
  ||kappa^n - kappa^m|| / ||kappa^m|| per realisation.
* transport (Section 4): explicit Euler, first-order upwind, C_n substeps with
  the flux frozen, dt = cfl h^2 / (max f' * max_c max(sum out, sum in)).

Pins (tests/test_oracle_pins.py) check each building block against closed forms, brute
force, the paper's special cases and printed numbers, and invariants.  Parity unpinned:
simulate_init / simulate_step as whole Algorithm 1 trajectories.  Their components and the
decision logic are pinned one by one, but a multi-step trajectory has no independent
reference, so the GPU path is compared with it directly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

DIRICHLET, NEUMANN = 0, 1
LEFT, RIGHT, BOTTOM, TOP = 0, 1, 2, 3


# ----------------------------------------------------------------------------
# Two-phase coefficients: Section 2 (lambda_j = k_rj / mu_j, f = lambda_w / lambda)
# and Section 5 (k_ro = (1-s)^2, k_rw = s^2, f = M s^2 / (M s^2 + (1-s)^2)).
# ----------------------------------------------------------------------------

def mobility(s, M):
    """Total mobility lambda(s) = k_rw/mu_w + k_ro/mu_o with mu_o = 1, mu_w = 1/M."""
    s = np.asarray(s, dtype=np.float64)
    return M * s * s + (1.0 - s) ** 2


def frac_flow(s, M):
    """Water fractional flow f(s) = M s^2 / (M s^2 + (1 - s)^2) (Section 5)."""
    s = np.asarray(s, dtype=np.float64)
    lw = M * s * s
    return lw / (lw + (1.0 - s) ** 2)


def frac_flow_deriv(s, M):
    """f'(s) = 2 M s (1 - s) / (M s^2 + (1 - s)^2)^2."""
    s = np.asarray(s, dtype=np.float64)
    d = M * s * s + (1.0 - s) ** 2
    return 2.0 * M * s * (1.0 - s) / (d * d)


def max_frac_flow_deriv(M):
    """max_s f'(s).  Setting d/ds log f' = 0 gives 2(M+1)s^3 - 3(M+1)s^2 + 1 = 0,
    which is strictly decreasing on (0,1) from 1 to -M; its root is found by bisection."""
    lo, hi = 0.0, 1.0
    c = M + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if 2.0 * c * mid ** 3 - 3.0 * c * mid ** 2 + 1.0 > 0.0:
            lo = mid
        else:
            hi = mid
    return float(frac_flow_deriv(0.5 * (lo + hi), M))


def harmonic(a, b):
    """Two-point transmissibility 2 a b / (a + b) of a face between conductivities a, b."""
    return 2.0 * a * b / (a + b)


# ----------------------------------------------------------------------------
# Problem and decomposition
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    """Eq. (Darcy) + Eq. (BL2D) data on [0, nx h] x [0, ny h], square cells.

    bc_type[side] in {DIRICHLET, NEUMANN}; bc_val is g (pressure) on Dirichlet
    sides and z (outward normal velocity u.n) on Neumann sides.  Sides are
    LEFT, RIGHT, BOTTOM, TOP.
    """
    nx: int
    ny: int
    h: float
    bc_type: tuple = (DIRICHLET, DIRICHLET, NEUMANN, NEUMANN)
    bc_val: tuple = (1.0, 0.0, 0.0, 0.0)
    M: float = 1.0
    s_inflow: float = 1.0
    q: np.ndarray | None = None  # source per cell (per unit area), [ny][nx]

    def source(self):
        if self.q is None:
            return np.zeros((self.ny, self.nx))
        return np.asarray(self.q, dtype=np.float64)


@dataclass
class Side:
    """One side of a subdomain: a physical boundary side or an interface."""
    kind: str                 # "phys" or "iface"
    which: int                # LEFT/RIGHT/BOTTOM/TOP (side of the subdomain)
    cells: list               # local cell indices along the side, increasing coordinate
    gcells: list              # global (j, i) of those cells
    iface: int = -1           # interface id
    sign: float = 0.0         # s = n_check . n_check^i
    length: int = 0           # interface length in cells (H_e / h)


@dataclass
class Subdomain:
    I: int
    J: int
    x0: int
    y0: int
    a: int   # width in cells
    b: int   # height in cells
    sides: list = field(default_factory=list)

    @property
    def m(self):
        return self.a * self.b


@dataclass
class Interface:
    orient: str      # "v" (normal +x) or "h" (normal +y)
    minus: int       # subdomain index on the side n_check points away from
    plus: int        # subdomain index n_check points into
    length: int      # cells
    dof0: int = 0    # first global DOF
    n_u: int = 0
    n_p: int = 0


class Decomposition:
    """Tensor-product decomposition (column widths x row heights) with the
    interface spaces of Section 3.1 (degree 0/1 on segments of seg_len edges)."""

    def __init__(self, nx, ny, col_w, row_h, seg_len=4, degree=1, alpha=1.0, alpha_face=None):
        # alpha_face: None (the constant alpha on every interface face) or a pair
        # (alpha_x [ny][nx+1], alpha_y [ny+1][nx]) giving alpha(x) of Eq. (beta) per fine face,
        # read on the interface faces only (the aMRCM's spatially varying alpha, Section 3.1)
        col_w = [int(v) for v in col_w]
        row_h = [int(v) for v in row_h]
        if sum(col_w) != nx or sum(row_h) != ny:
            raise ValueError("decomposition does not tile the grid")
        self.nx, self.ny = nx, ny
        self.col_w, self.row_h = col_w, row_h
        self.ncx, self.ncy = len(col_w), len(row_h)
        self.seg_len, self.degree, self.alpha = int(seg_len), int(degree), float(alpha)
        if alpha_face is None:
            self.alpha_x = np.full((ny, nx + 1), self.alpha)
            self.alpha_y = np.full((ny + 1, nx), self.alpha)
        else:
            self.alpha_x = np.asarray(alpha_face[0], dtype=np.float64).reshape(ny, nx + 1)
            self.alpha_y = np.asarray(alpha_face[1], dtype=np.float64).reshape(ny + 1, nx)
        xo = np.concatenate([[0], np.cumsum(col_w)]).astype(int)
        yo = np.concatenate([[0], np.cumsum(row_h)]).astype(int)
        self.subs = []
        for J in range(self.ncy):
            for I in range(self.ncx):
                self.subs.append(Subdomain(I, J, int(xo[I]), int(yo[J]), col_w[I], row_h[J]))
        self.ifaces = []
        vid, hid = {}, {}
        for J in range(self.ncy):
            for I in range(self.ncx - 1):
                vid[(I, J)] = len(self.ifaces)
                self.ifaces.append(Interface("v", J * self.ncx + I, J * self.ncx + I + 1, row_h[J]))
        for J in range(self.ncy - 1):
            for I in range(self.ncx):
                hid[(I, J)] = len(self.ifaces)
                self.ifaces.append(Interface("h", J * self.ncx + I, (J + 1) * self.ncx + I, col_w[I]))
        nb = self.degree + 1
        off = 0
        for itf in self.ifaces:
            if itf.length % self.seg_len:
                raise ValueError("interface length must be a multiple of seg_len")
            nseg = itf.length // self.seg_len
            itf.dof0, itf.n_u, itf.n_p = off, nseg * nb, nseg * nb
            off += itf.n_u + itf.n_p
        self.n_dof = off
        for sd in self.subs:
            a, b = sd.a, sd.b
            left = [jl * a for jl in range(b)]
            right = [jl * a + a - 1 for jl in range(b)]
            bottom = [il for il in range(a)]
            top = [(b - 1) * a + il for il in range(a)]
            spec = [
                (LEFT, left, [(sd.y0 + jl, sd.x0) for jl in range(b)], (sd.I - 1, sd.J), "v", -1.0),
                (RIGHT, right, [(sd.y0 + jl, sd.x0 + a - 1) for jl in range(b)], (sd.I, sd.J), "v", +1.0),
                (BOTTOM, bottom, [(sd.y0, sd.x0 + il) for il in range(a)], (sd.I, sd.J - 1), "h", -1.0),
                (TOP, top, [(sd.y0 + b - 1, sd.x0 + il) for il in range(a)], (sd.I, sd.J), "h", +1.0),
            ]
            for which, cells, gcells, key, orient, sign in spec:
                table = vid if orient == "v" else hid
                if key in table:
                    itf = self.ifaces[table[key]]
                    sd.sides.append(Side("iface", which, cells, gcells, table[key], sign, itf.length))
                else:
                    sd.sides.append(Side("phys", which, cells, gcells))

    def side_alpha(self, side: Side):
        """alpha of Eq. (beta) on each face of a side (in the side's cell order)."""
        if side.which == LEFT:
            return np.array([self.alpha_x[j, i] for (j, i) in side.gcells])
        if side.which == RIGHT:
            return np.array([self.alpha_x[j, i + 1] for (j, i) in side.gcells])
        if side.which == BOTTOM:
            return np.array([self.alpha_y[j, i] for (j, i) in side.gcells])
        return np.array([self.alpha_y[j + 1, i] for (j, i) in side.gcells])

    def basis(self, itf: Interface, t: int, k: int) -> float:
        """Value at edge t (0-based along the interface) of the k-th basis function of one
        of the two spaces on interface ``itf`` (k = seg * (degree+1) + power)."""
        nb = self.degree + 1
        seg, power = divmod(k, nb)
        if t // self.seg_len != seg:
            return 0.0
        xi = ((t % self.seg_len) + 0.5) / self.seg_len
        return 1.0 if power == 0 else 2.0 * xi - 1.0

    def sub_dofs(self, sd: Subdomain):
        """Global DOFs on the interfaces of sd, in side order: list of
        (global dof, side index, 'U'/'P', k)."""
        out = []
        for si, side in enumerate(sd.sides):
            if side.kind != "iface":
                continue
            itf = self.ifaces[side.iface]
            for k in range(itf.n_u):
                out.append((itf.dof0 + k, si, "U", k))
            for k in range(itf.n_p):
                out.append((itf.dof0 + itf.n_u + k, si, "P", k))
        return out

    def n_hat(self) -> int:
        """Total number of homogeneous BFs (Section 4.3): DOFs on the sides of every subdomain."""
        return sum(len(self.sub_dofs(sd)) for sd in self.subs)


def uniform_decomposition(nx, ny, ncx, ncy, seg_len=4, degree=1, alpha=1.0, alpha_face=None):
    return Decomposition(nx, ny, [nx // ncx] * ncx, [ny // ncy] * ncy, seg_len, degree, alpha, alpha_face)


# ----------------------------------------------------------------------------
# Fine grid (Eq. Darcy discretised with P0 edge fluxes)
# ----------------------------------------------------------------------------

def fine_system(kappa, prob: Problem):
    """Global two-point system A p = b for Eq. (Darcy) with conductivity kappa."""
    ny, nx, h = prob.ny, prob.nx, prob.h
    q = prob.source()
    n = nx * ny
    rows, cols, vals = [], [], []
    b = (q * h * h).reshape(-1).copy()
    diag = np.zeros(n)

    def idx(i, j):
        return j * nx + i

    for j in range(ny):
        for i in range(nx):
            c = idx(i, j)
            for (ii, jj) in ((i + 1, j), (i, j + 1)):
                if ii < nx and jj < ny:
                    t = harmonic(kappa[j, i], kappa[jj, ii])
                    d = idx(ii, jj)
                    diag[c] += t
                    diag[d] += t
                    rows += [c, d]
                    cols += [d, c]
                    vals += [-t, -t]
            for side, on in ((LEFT, i == 0), (RIGHT, i == nx - 1), (BOTTOM, j == 0), (TOP, j == ny - 1)):
                if not on:
                    continue
                if prob.bc_type[side] == DIRICHLET:
                    diag[c] += 2.0 * kappa[j, i]
                    b[c] += 2.0 * kappa[j, i] * prob.bc_val[side]
                else:
                    b[c] -= prob.bc_val[side] * h
    rows += list(range(n))
    cols += list(range(n))
    vals += list(diag)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return A, b


def fine_solve(kappa, prob: Problem):
    A, b = fine_system(kappa, prob)
    return spla.spsolve(A.tocsc(), b).reshape(prob.ny, prob.nx)


def fine_fluxes(p, kappa, prob: Problem):
    """Integrated face fluxes of a global cell pressure p (Darcy's law, two-point)."""
    ny, nx, h = prob.ny, prob.nx, prob.h
    Fx = np.zeros((ny, nx + 1))
    Fy = np.zeros((ny + 1, nx))
    Fx[:, 1:nx] = harmonic(kappa[:, :-1], kappa[:, 1:]) * (p[:, :-1] - p[:, 1:])
    Fy[1:ny, :] = harmonic(kappa[:-1, :], kappa[1:, :]) * (p[:-1, :] - p[1:, :])
    for side in (LEFT, RIGHT, BOTTOM, TOP):
        if side == LEFT:
            kc, pc, sl, sgn = kappa[:, 0], p[:, 0], (slice(None), 0), -1.0
            tgt = Fx
        elif side == RIGHT:
            kc, pc, sl, sgn = kappa[:, -1], p[:, -1], (slice(None), nx), 1.0
            tgt = Fx
        elif side == BOTTOM:
            kc, pc, sl, sgn = kappa[0, :], p[0, :], (0, slice(None)), -1.0
            tgt = Fy
        else:
            kc, pc, sl, sgn = kappa[-1, :], p[-1, :], (ny, slice(None)), 1.0
            tgt = Fy
        if prob.bc_type[side] == DIRICHLET:
            out = 2.0 * kc * (pc - prob.bc_val[side])
        else:
            out = np.full_like(pc, prob.bc_val[side] * h)
        tgt[sl] = sgn * out  # outward flux -> +x/+y flux
    return Fx, Fy


def cell_balance(Fx, Fy, prob: Problem):
    """Per-cell residual  sum_faces F_out - q h^2  (zero for a conservative field)."""
    out = Fx[:, 1:] - Fx[:, :-1] + Fy[1:, :] - Fy[:-1, :]
    return out - prob.source() * prob.h ** 2


# ----------------------------------------------------------------------------
# Local Robin problems, Eq. (mrc1) and its split Eqs. (mrc_homogeneous),
# (mrc_non_homogeneous).
# ----------------------------------------------------------------------------

def _robin_coeffs(dec: Decomposition, side: Side, kappa_cells):
    """r_e = kappa_c / (1/2 + rho_e) and beta_hat_e = rho_e / kappa_c, rho_e = alpha_e H_e / h."""
    rho = dec.side_alpha(side) * side.length
    kc = np.asarray(kappa_cells)
    return kc / (0.5 + rho), rho / kc


def local_matrix(kappa, prob: Problem, dec: Decomposition, sd: Subdomain, neumann=False, pin=False):
    """Dense matrix of the local problem on sd: Robin on interfaces (Eq. mrc1) and the
    physical boundary conditions, or (neumann=True) all sides Neumann (Eq. mpm_upd),
    optionally with cell 0 pinned (adds kappa_0 e_0 e_0^T)."""
    a, b = sd.a, sd.b
    kap = kappa[sd.y0:sd.y0 + b, sd.x0:sd.x0 + a]
    A = np.zeros((sd.m, sd.m))
    for jl in range(b):
        for il in range(a):
            c = jl * a + il
            for (ii, jj) in ((il + 1, jl), (il, jl + 1)):
                if ii < a and jj < b:
                    d = jj * a + ii
                    t = harmonic(kap[jl, il], kap[jj, ii])
                    A[c, c] += t
                    A[d, d] += t
                    A[c, d] -= t
                    A[d, c] -= t
    if not neumann:
        for side in sd.sides:
            kc = np.array([kappa[j, i] for (j, i) in side.gcells])
            if side.kind == "iface":
                r, _ = _robin_coeffs(dec, side, kc)
                for c, rv in zip(side.cells, r):
                    A[c, c] += rv
            elif prob.bc_type[side.which] == DIRICHLET:
                for c, kv in zip(side.cells, kc):
                    A[c, c] += 2.0 * kv
    if pin:
        A[0, 0] += kap[0, 0]
    return A


def local_rhs(kappa, prob: Problem, dec: Decomposition, sd: Subdomain, src_cells, g_faces, homogeneous_bc=False):
    """Right-hand side of the local Robin problem: source (integrated over the cell),
    physical data (unless homogeneous_bc) and Robin data g_faces[side index] (array per side)."""
    rhs = src_cells.reshape(-1).astype(np.float64).copy()
    for si, side in enumerate(sd.sides):
        kc = np.array([kappa[j, i] for (j, i) in side.gcells])
        if side.kind == "iface":
            r, _ = _robin_coeffs(dec, side, kc)
            for c, rv, gv in zip(side.cells, r, g_faces[si]):
                rhs[c] += rv * gv
        elif not homogeneous_bc:
            if prob.bc_type[side.which] == DIRICHLET:
                for c, kv in zip(side.cells, kc):
                    rhs[c] += 2.0 * kv * prob.bc_val[side.which]
            else:
                for c in side.cells:
                    rhs[c] -= prob.bc_val[side.which] * prob.h
    return rhs


def local_traces(p_local, kappa, prob: Problem, dec: Decomposition, sd: Subdomain, g_faces, homogeneous_bc=False):
    """Integrated outward fluxes on every side of sd (list of arrays in side order)."""
    out = []
    for si, side in enumerate(sd.sides):
        kc = np.array([kappa[j, i] for (j, i) in side.gcells])
        pc = p_local[side.cells]
        if side.kind == "iface":
            r, _ = _robin_coeffs(dec, side, kc)
            out.append(r * (pc - np.asarray(g_faces[si])))
        elif prob.bc_type[side.which] == DIRICHLET:
            g = 0.0 if homogeneous_bc else prob.bc_val[side.which]
            out.append(2.0 * kc * (pc - g))
        else:
            z = 0.0 if homogeneous_bc else prob.bc_val[side.which]
            out.append(np.full(len(side.cells), z * prob.h))
    return out


def _dof_robin_data(dec: Decomposition, sd: Subdomain, kappa, dof):
    """Robin data per side for one homogeneous BF (Eq. mrc_homogeneous): a U-DOF
    phi_k gives g = -beta_hat s phi_k, a P-DOF psi_k gives g = psi_k, on the DOF's side."""
    _, si_dof, kind, k = dof
    g = []
    for si, side in enumerate(sd.sides):
        if side.kind != "iface" or si != si_dof:
            g.append(np.zeros(len(side.cells)))
            continue
        itf = dec.ifaces[side.iface]
        kc = np.array([kappa[j, i] for (j, i) in side.gcells])
        _, bh = _robin_coeffs(dec, side, kc)
        phi = np.array([dec.basis(itf, t, k) for t in range(len(side.cells))])
        g.append(-bh * side.sign * phi if kind == "U" else phi)
    return g


@dataclass
class BasisSet:
    """The stored set of BFs {Phi^m, Psi^m} of Algorithm 1 for one conductivity."""
    kappa: np.ndarray
    A: list           # local Robin matrices
    dofs: list        # per subdomain DOF lists
    G: list           # per subdomain, per DOF: Robin data per side
    P_hat: list       # per subdomain: m x n_dof BF pressures
    F_hat: list       # per subdomain: list per side of (n_side x n_dof) BF traces
    K: sp.csr_matrix  # assembled interface matrix
    K_lu: object = None  # its sparse LU factorisation, made at the first solve and kept with the BFs


def build_basis(kappa, prob: Problem, dec: Decomposition) -> BasisSet:
    """One homogeneous local solve per interface DOF of every subdomain (the BFs of
    Eq. mrc_homogeneous), their traces, and the interface matrix of Eq. (mrc2)."""
    A_l, dofs_l, G_l, P_l, F_l = [], [], [], [], []
    for sd in dec.subs:
        A = local_matrix(kappa, prob, dec, sd)
        dofs = dec.sub_dofs(sd)
        G = [_dof_robin_data(dec, sd, kappa, d) for d in dofs]
        zero_src = np.zeros(sd.m)
        if dofs:
            R = np.stack([local_rhs(kappa, prob, dec, sd, zero_src, g, homogeneous_bc=True) for g in G], axis=1)
            P = np.linalg.solve(A, R)
        else:
            P = np.zeros((sd.m, 0))
        F = []
        for si, side in enumerate(sd.sides):
            cols = [local_traces(P[:, l], kappa, prob, dec, sd, G[l], homogeneous_bc=True)[si]
                    for l in range(len(dofs))]
            F.append(np.stack(cols, axis=1) if cols else np.zeros((len(side.cells), 0)))
        A_l.append(A)
        dofs_l.append(dofs)
        G_l.append(G)
        P_l.append(P)
        F_l.append(F)
    bs = BasisSet(kappa.copy(), A_l, dofs_l, G_l, P_l, F_l, None)
    bs.K = _assemble_interface_matrix(bs, kappa, dec)
    return bs


def _test_weights(dec: Decomposition, side: Side, kind: str):
    """(n_side x n_test) matrix of interface test functions of one kind on a side."""
    itf = dec.ifaces[side.iface]
    n = itf.n_u if kind == "U" else itf.n_p
    return np.array([[dec.basis(itf, t, k) for k in range(n)] for t in range(len(side.cells))]).reshape(len(side.cells), n)


def _assemble_interface_matrix(bs: BasisSet, kappa, dec: Decomposition):
    """Eq. (mrc2) tested with every psi (flux balance) and phi (negated Robin-weighted
    pressure continuity), with the traces of the BFs substituted for u_h^i."""
    n = dec.n_dof
    rows, cols, vals = [], [], []
    for s_i, sd in enumerate(dec.subs):
        dofs = bs.dofs[s_i]
        if not dofs:
            continue
        gcols = np.array([d[0] for d in dofs])
        for si, side in enumerate(sd.sides):
            if side.kind != "iface":
                continue
            itf = dec.ifaces[side.iface]
            Fh = bs.F_hat[s_i][si]                       # n_side x n_dof
            kc = np.array([kappa[j, i] for (j, i) in side.gcells])
            _, bh = _robin_coeffs(dec, side, kc)
            Wp = _test_weights(dec, side, "P")           # n_side x n_p
            Wu = _test_weights(dec, side, "U")
            # psi rows: sum_e psi(e) F_e
            blk_p = Wp.T @ Fh
            # phi rows (negated): -sum_e bh (F_e - U_e s) phi(e) s
            blk_u = -(Wu * (bh * side.sign)[:, None]).T @ Fh
            # + sum_e bh phi_l(e) phi_k(e) for U-DOFs l of this interface (s^2 = 1)
            own = np.zeros_like(blk_u)
            for l, d in enumerate(dofs):
                if d[1] == si and d[2] == "U":
                    own[:, l] = (Wu * bh[:, None]).T @ Wu[:, d[3]]
            blk_u = blk_u + own
            pr = itf.dof0 + itf.n_u + np.arange(itf.n_p)
            ur = itf.dof0 + np.arange(itf.n_u)
            for blk, rr in ((blk_p, pr), (blk_u, ur)):
                R, C = np.meshgrid(rr, gcols, indexing="ij")
                rows.append(R.ravel())
                cols.append(C.ravel())
                vals.append(blk.ravel())
    if n == 0:
        return sp.csr_matrix((0, 0))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def _interface_rhs(Fbar, kappa, dec: Decomposition):
    """Right-hand side of Eq. (mrc2) from the non-homogeneous traces (moved to the right)."""
    f = np.zeros(dec.n_dof)
    for s_i, sd in enumerate(dec.subs):
        for si, side in enumerate(sd.sides):
            if side.kind != "iface":
                continue
            itf = dec.ifaces[side.iface]
            kc = np.array([kappa[j, i] for (j, i) in side.gcells])
            _, bh = _robin_coeffs(dec, side, kc)
            Fb = Fbar[s_i][si]
            f[itf.dof0 + itf.n_u: itf.dof0 + itf.n_u + itf.n_p] -= _test_weights(dec, side, "P").T @ Fb
            f[itf.dof0: itf.dof0 + itf.n_u] += _test_weights(dec, side, "U").T @ (bh * side.sign * Fb)
    return f


def _solve_interface(bs: BasisSet, f):
    """Solve the interface system of Eq. (mrc2) with matrix bs.K by sparse LU (SuperLU,
    COLAMD column ordering, partial pivoting).  The factorisation is kept with the BFs, so
    the MPM-2P updates that reuse them do not factor again (the same LU spsolve would make)."""
    if f.size == 0:
        return f.copy()
    if bs.K_lu is None:
        bs.K_lu = spla.splu(bs.K.tocsc(), permc_spec="COLAMD")
    return bs.K_lu.solve(f)


@dataclass
class MRCMSolution:
    p: np.ndarray           # MRCM-level cell pressure [ny][nx] (each cell from its own subdomain)
    coeffs: np.ndarray      # interface unknowns (U then P per interface)
    traces: list            # per subdomain, per side: outward integrated flux
    ubar_x: np.ndarray      # Fx on subdomain-boundary faces (mean of one-sided traces), NaN elsewhere
    ubar_y: np.ndarray


def _nonhomogeneous(kappa, prob, dec, bs: BasisSet, src, homogeneous_bc):
    """Non-homogeneous local solves (Eq. mrc_non_homogeneous): zero Robin data."""
    pbar, Fbar = [], []
    for s_i, sd in enumerate(dec.subs):
        g0 = [np.zeros(len(side.cells)) for side in sd.sides]
        rhs = local_rhs(kappa, prob, dec, sd, src[sd.y0:sd.y0 + sd.b, sd.x0:sd.x0 + sd.a], g0, homogeneous_bc)
        pl = np.linalg.solve(bs.A[s_i], rhs)
        pbar.append(pl)
        Fbar.append(local_traces(pl, kappa, prob, dec, sd, g0, homogeneous_bc))
    return pbar, Fbar


def _combine(kappa, prob, dec, bs: BasisSet, pbar, Fbar, c) -> MRCMSolution:
    """u_h^i = ubar^i + sum_l c_l uhat_l, p_h^i likewise (Section 3, additive split)."""
    p = np.zeros((prob.ny, prob.nx))
    traces = []
    for s_i, sd in enumerate(dec.subs):
        cl = np.array([c[d[0]] for d in bs.dofs[s_i]])
        pl = pbar[s_i] + (bs.P_hat[s_i] @ cl if cl.size else 0.0)
        p[sd.y0:sd.y0 + sd.b, sd.x0:sd.x0 + sd.a] = pl.reshape(sd.b, sd.a)
        traces.append([Fbar[s_i][si] + (bs.F_hat[s_i][si] @ cl if cl.size else 0.0)
                       for si in range(len(sd.sides))])
    ux, uy = subdomain_boundary_fluxes(traces, prob, dec)
    return MRCMSolution(p, c, traces, ux, uy)


def subdomain_boundary_fluxes(traces, prob: Problem, dec: Decomposition):
    """Fluxes on every subdomain-boundary face: physical faces take the trace,
    interface faces the mean of the two one-sided traces, in +x/+y direction."""
    ux = np.full((prob.ny, prob.nx + 1), np.nan)
    uy = np.full((prob.ny + 1, prob.nx), np.nan)
    acc_x = np.zeros_like(ux)
    acc_y = np.zeros_like(uy)
    cnt_x = np.zeros_like(ux)
    cnt_y = np.zeros_like(uy)
    for s_i, sd in enumerate(dec.subs):
        for si, side in enumerate(sd.sides):
            F = traces[s_i][si]
            for t, (j, i) in enumerate(side.gcells):
                if side.which == LEFT:
                    acc_x[j, i] -= F[t]; cnt_x[j, i] += 1
                elif side.which == RIGHT:
                    acc_x[j, i + 1] += F[t]; cnt_x[j, i + 1] += 1
                elif side.which == BOTTOM:
                    acc_y[j, i] -= F[t]; cnt_y[j, i] += 1
                else:
                    acc_y[j + 1, i] += F[t]; cnt_y[j + 1, i] += 1
    mx = cnt_x > 0
    my = cnt_y > 0
    ux[mx] = acc_x[mx] / cnt_x[mx]
    uy[my] = acc_y[my] / cnt_y[my]
    return ux, uy


def mrcm_solve(kappa, prob: Problem, dec: Decomposition, bs: BasisSet | None = None):
    """MRCM solution of Eq. (Darcy) with conductivity kappa, BF route (Section 3)."""
    if bs is None:
        bs = build_basis(kappa, prob, dec)
    pbar, Fbar = _nonhomogeneous(kappa, prob, dec, bs, prob.source() * prob.h ** 2, False)
    c = _solve_interface(bs, _interface_rhs(Fbar, kappa, dec))
    return _combine(kappa, prob, dec, bs, pbar, Fbar, c), bs


def mrcm_monolithic(kappa, prob: Problem, dec: Decomposition, src=None, homogeneous_bc=False):
    """Eqs. (mrc1)+(mrc2) as one sparse system in all local cell pressures and all
    interface unknowns (no basis functions): cross-check of the BF route."""
    ny, nx = prob.ny, prob.nx
    if src is None:
        src = prob.source() * prob.h ** 2
    ncell = nx * ny
    n = ncell + dec.n_dof
    rows, cols, vals = [], [], []
    rhs = np.zeros(n)

    def add(r, c, v):
        rows.append(r); cols.append(c); vals.append(v)

    for sd in dec.subs:
        A = local_matrix(kappa, prob, dec, sd)
        gidx = np.array([(sd.y0 + jl) * nx + sd.x0 + il for jl in range(sd.b) for il in range(sd.a)])
        nz = np.nonzero(A)
        for r, c in zip(*nz):
            add(gidx[r], gidx[c], A[r, c])
        g0 = [np.zeros(len(side.cells)) for side in sd.sides]
        rhs[gidx] += local_rhs(kappa, prob, dec, sd, src[sd.y0:sd.y0 + sd.b, sd.x0:sd.x0 + sd.a], g0, homogeneous_bc)
        for si, side in enumerate(sd.sides):
            if side.kind != "iface":
                continue
            itf = dec.ifaces[side.iface]
            kc = np.array([kappa[j, i] for (j, i) in side.gcells])
            r_e, bh = _robin_coeffs(dec, side, kc)
            Wu = _test_weights(dec, side, "U")
            Wp = _test_weights(dec, side, "P")
            # Robin data g_e = -bh s U_e + P_e, U_e = Wu u, P_e = Wp p
            # cell rows: - r_e g_e moves to the left:  -r_e * (-bh s Wu) u - r_e Wp p
            for t, c in enumerate(side.cells):
                for k in range(itf.n_u):
                    add(gidx[c], ncell + itf.dof0 + k, r_e[t] * bh[t] * side.sign * Wu[t, k])
                for k in range(itf.n_p):
                    add(gidx[c], ncell + itf.dof0 + itf.n_u + k, -r_e[t] * Wp[t, k])
            # psi rows: sum_e psi_k(e) r_e (p_c - g_e) = 0
            # phi rows: -sum_e bh (r_e (p_c - g_e) - U_e s) phi_k(e) s = 0
            for t, c in enumerate(side.cells):
                dg_du = -bh[t] * side.sign * Wu[t, :]     # d g_e / d u
                dg_dp = Wp[t, :]
                for k in range(itf.n_p):
                    row = ncell + itf.dof0 + itf.n_u + k
                    w = Wp[t, k]
                    add(row, gidx[c], w * r_e[t])
                    for kk in range(itf.n_u):
                        add(row, ncell + itf.dof0 + kk, -w * r_e[t] * dg_du[kk])
                    for kk in range(itf.n_p):
                        add(row, ncell + itf.dof0 + itf.n_u + kk, -w * r_e[t] * dg_dp[kk])
                for k in range(itf.n_u):
                    row = ncell + itf.dof0 + k
                    w = -bh[t] * Wu[t, k] * side.sign
                    add(row, gidx[c], w * r_e[t])
                    for kk in range(itf.n_u):
                        add(row, ncell + itf.dof0 + kk, -w * r_e[t] * dg_du[kk] - w * Wu[t, kk] * side.sign)
                    for kk in range(itf.n_p):
                        add(row, ncell + itf.dof0 + itf.n_u + kk, -w * r_e[t] * dg_dp[kk])
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    x = spla.spsolve(A.tocsc(), rhs)
    return x[:ncell].reshape(ny, nx), x[ncell:]


# ----------------------------------------------------------------------------
# Downscaling, Eq. (mpm_upd)
# ----------------------------------------------------------------------------

def downscale(kappa, ux_b, uy_b, p_level, prob: Problem, dec: Decomposition):
    """Neumann problem with conductivity kappa on every subdomain, the given fluxes on
    all its boundary faces; the pressure constant makes mean(p~) = mean(p_level) per
    subdomain.  Returns (p~, Fx, Fy) with Fx/Fy conservative on the fine grid."""
    ny, nx, h = prob.ny, prob.nx, prob.h
    q = prob.source()
    pt = np.zeros((ny, nx))
    Fx = ux_b.copy()
    Fy = uy_b.copy()
    for sd in dec.subs:
        a, b = sd.a, sd.b
        A = local_matrix(kappa, prob, dec, sd, neumann=True, pin=True)
        rhs = (q[sd.y0:sd.y0 + b, sd.x0:sd.x0 + a] * h * h).reshape(-1).copy()
        for jl in range(b):
            for il in range(a):
                c = jl * a + il
                j, i = sd.y0 + jl, sd.x0 + il
                if il == 0:
                    rhs[c] += ux_b[j, i]          # inflow through the left face
                if il == a - 1:
                    rhs[c] -= ux_b[j, i + 1]
                if jl == 0:
                    rhs[c] += uy_b[j, i]
                if jl == b - 1:
                    rhs[c] -= uy_b[j + 1, i]
        pl = np.linalg.solve(A, rhs).reshape(b, a)
        pl += np.mean(p_level[sd.y0:sd.y0 + b, sd.x0:sd.x0 + a]) - np.mean(pl)
        pt[sd.y0:sd.y0 + b, sd.x0:sd.x0 + a] = pl
        kap = kappa[sd.y0:sd.y0 + b, sd.x0:sd.x0 + a]
        Fx[sd.y0:sd.y0 + b, sd.x0 + 1:sd.x0 + a] = harmonic(kap[:, :-1], kap[:, 1:]) * (pl[:, :-1] - pl[:, 1:])
        Fy[sd.y0 + 1:sd.y0 + b, sd.x0:sd.x0 + a] = harmonic(kap[:-1, :], kap[1:, :]) * (pl[:-1, :] - pl[1:, :])
    return pt, Fx, Fy


# ----------------------------------------------------------------------------
# MPM-2P, Section 4.1: epsilon^0 problem (Eq. mpm_tf_3) solved by MRCM with the
# stored BFs of kappa^m, then downscaling with kappa^n.
# ----------------------------------------------------------------------------

def fine_residual(kappa_n, p_m, prob: Problem):
    """r = b(kappa^n) - A(kappa^n) p^m: the source of the epsilon^0 problem, i.e.
    q + div(kappa^n grad p^m) integrated over each cell (Eq. mpm_tf_3)."""
    A, b = fine_system(kappa_n, prob)
    return (b - A @ p_m.reshape(-1)).reshape(prob.ny, prob.nx)


@dataclass
class StepResult:
    p_level: np.ndarray     # MRCM-level pressure of this step
    p_down: np.ndarray      # downscaled pressure
    Fx: np.ndarray          # conservative integrated fluxes
    Fy: np.ndarray


def mrcm_step(kappa, prob: Problem, dec: Decomposition):
    """Full MRCM update (rebuild): BFs at kappa, interface solve, downscale."""
    sol, bs = mrcm_solve(kappa, prob, dec)
    pt, Fx, Fy = downscale(kappa, sol.ubar_x, sol.ubar_y, sol.p, prob, dec)
    return StepResult(sol.p, pt, Fx, Fy), bs, sol


def _homogeneous(prob: Problem):
    """The same problem with zero source and zero physical boundary data (the data of the
    perturbation problems, Eq. mpm_tf_4)."""
    return Problem(prob.nx, prob.ny, prob.h, prob.bc_type, (0.0, 0.0, 0.0, 0.0), prob.M, prob.s_inflow, None)


def mpm_step(kappa_n, bs: BasisSet, p_m, prob: Problem, dec: Decomposition, order: int = 0):
    """One MPM-2P update reusing the BFs of kappa^m = bs.kappa (Section 4.1).

    order = 0 solves the epsilon^0 problem (Eq. mpm_tf_3) only, as the paper does.
    order = 1 adds the first-order term of the expansion (Eq. mpm_tf_4 with l = 1): its
    source div(kappa_eps grad delta p_0), with eps kappa_eps = kappa^n - kappa^m, is on the
    fine grid -(A(kappa^n) - A(kappa^m)) delta p_0 (homogeneous data); it is solved with
    the same stored BFs, and eps u_hat_1 = eps delta u_1 + (kappa^n - kappa^m) grad delta p_0
    gives the flux increment u_hat_1 + F_n(delta p_0) - F_m(delta p_0), F_k the fine flux
    under kappa^k.  delta p_0 is the MRCM-level pressure of the epsilon^0 solve."""
    kappa_m = bs.kappa
    r = fine_residual(kappa_n, p_m, prob)
    pbar, Fbar = _nonhomogeneous(kappa_m, prob, dec, bs, r, True)
    c = _solve_interface(bs, _interface_rhs(Fbar, kappa_m, dec))
    dsol = _combine(kappa_m, prob, dec, bs, pbar, Fbar, c)
    # ubar = u^m + delta u^n = uhat_0 - kappa^n grad p^m  (F_n(p^m) below)
    Fnx, Fny = fine_fluxes(p_m, kappa_n, prob)
    ux = dsol.ubar_x + Fnx
    uy = dsol.ubar_y + Fny
    p_level = p_m + dsol.p
    if order >= 1:
        hom = _homogeneous(prob)
        A_n, _ = fine_system(kappa_n, hom)
        A_m, _ = fine_system(kappa_m, hom)
        dp0 = dsol.p.reshape(-1)
        r1 = -((A_n - A_m) @ dp0).reshape(prob.ny, prob.nx)
        pbar1, Fbar1 = _nonhomogeneous(kappa_m, prob, dec, bs, r1, True)
        c1 = _solve_interface(bs, _interface_rhs(Fbar1, kappa_m, dec))
        dsol1 = _combine(kappa_m, prob, dec, bs, pbar1, Fbar1, c1)
        Gnx, Gny = fine_fluxes(dsol.p, kappa_n, hom)
        Gmx, Gmy = fine_fluxes(dsol.p, kappa_m, hom)
        ux = ux + dsol1.ubar_x + (Gnx - Gmx)
        uy = uy + dsol1.ubar_y + (Gny - Gmy)
        p_level = p_level + dsol1.p
    pt, Fx, Fy = downscale(kappa_n, ux, uy, p_level, prob, dec)
    return StepResult(p_level, pt, Fx, Fy), dsol


# ----------------------------------------------------------------------------
# Transport, Eq. (BL2D): explicit Euler + first-order upwind, u frozen.
# ----------------------------------------------------------------------------

def cfl_dt(Fx, Fy, prob: Problem, cfl: float):
    """dt = cfl h^2 / (max f' * max over cells of max(total outflow, total inflow))."""
    fo = np.zeros((prob.ny, prob.nx))
    fi = np.zeros((prob.ny, prob.nx))
    for F_out in (-Fx[:, :-1], Fx[:, 1:], -Fy[:-1, :], Fy[1:, :]):
        fo += np.maximum(F_out, 0.0)
        fi += np.maximum(-F_out, 0.0)
    rate = float(np.max(np.maximum(fo, fi)))
    if rate == 0.0:
        return math.inf
    return cfl * prob.h ** 2 / (max_frac_flow_deriv(prob.M) * rate)


def upwind_step(s, Fx, Fy, dt, prob: Problem):
    """s_c <- s_c - dt/h^2 sum_faces F_out f(s_upwind); boundary inflow carries s_inflow."""
    ny, nx, h, M = prob.ny, prob.nx, prob.h, prob.M
    s_new = s.copy()
    for j in range(ny):
        for i in range(nx):
            acc = 0.0
            faces = ((-Fx[j, i], (j, i - 1) if i > 0 else None),
                     (Fx[j, i + 1], (j, i + 1) if i < nx - 1 else None),
                     (-Fy[j, i], (j - 1, i) if j > 0 else None),
                     (Fy[j + 1, i], (j + 1, i) if j < ny - 1 else None))
            for F_out, nb in faces:
                if F_out > 0.0:
                    acc += F_out * frac_flow(s[j, i], M)
                elif F_out < 0.0:
                    s_up = prob.s_inflow if nb is None else s[nb]
                    acc += F_out * frac_flow(s_up, M)
            s_new[j, i] = s[j, i] - dt / (h * h) * acc
    return s_new


def epsilon(kappa_n, kappa_m):
    """Dimensionless MPM-2P parameter: relative discrete L2 distance (Section 4.1)."""
    return float(np.sqrt(np.sum((kappa_n - kappa_m) ** 2)) / np.sqrt(np.sum(kappa_m ** 2)))


# ----------------------------------------------------------------------------
# Algorithm 1 and the cost model of Section 4.3
# ----------------------------------------------------------------------------

@dataclass
class SimState:
    s: np.ndarray
    bs: BasisSet
    p_m: np.ndarray
    step: StepResult
    eps: float
    n: int = 1
    ell: int = 0
    history: list = field(default_factory=list)


def simulate_init(K, s0, prob: Problem, dec: Decomposition, eta: float) -> SimState:
    """Algorithm 1, initialisation: kappa^0, MRCM solution, store the BFs, eps = eta."""
    kappa0 = mobility(s0, prob.M) * K
    step, bs, sol = mrcm_step(kappa0, prob, dec)
    return SimState(s0.copy(), bs, sol.p.copy(), step, eta)


def simulate_step(st: SimState, K, prob: Problem, dec: Decomposition, eta: float, cfl: float, n_sub: int,
                  order: int = 0):
    """One pass of the while loop of Algorithm 1 (transport substeps, kappa^n,
    rebuild if eps > eta else MPM of the given perturbation order, new eps)."""
    dt = cfl_dt(st.step.Fx, st.step.Fy, prob, cfl)
    for _ in range(n_sub):
        st.s = upwind_step(st.s, st.step.Fx, st.step.Fy, dt, prob)
    kappa_n = mobility(st.s, prob.M) * K
    rebuild = st.eps > eta
    if rebuild:
        st.ell += 1
        st.step, st.bs, sol = mrcm_step(kappa_n, prob, dec)
        st.p_m = sol.p.copy()
    else:
        st.step, _ = mpm_step(kappa_n, st.bs, st.p_m, prob, dec, order)
    st.eps = epsilon(kappa_n, st.bs.kappa)
    st.history.append(dict(n=st.n, rebuild=rebuild, eps=st.eps, dt=dt))
    st.n += 1
    return st


def rcr(T_e, T_m, N_hat, N):
    """Relative Cost Reduction of MPM-2P over MRCM, Section 4.3 (percent)."""
    return (T_e - T_m) / T_e * (1.0 - 2.0 * N / (N_hat + 2.0 * N)) * 100.0
