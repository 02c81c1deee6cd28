"""Seeded problem set shared by the GPU parity tests (inputs only; no method arithmetic)."""
import numpy as np

from paper_2103_11050_gb300 import fields

D, N = 0, 1

# name: (nx, ny, col_w, row_h, seg_len, degree, alpha, cov, sigma2, ell, M, bc_type, bc_val, seed)
CASES = {
    "p1_2x2": (32, 32, [16, 16], [16, 16], 4, 1, 1.0, "exponential", 1.0, 0.2, 2.0, (D, D, N, N), (1, 0, 0, 0), 1),
    "uneven": (40, 36, [8, 12, 20], [12, 8, 16], 4, 1, 1.0, "exponential", 2.0, 0.15, 5.0, (D, D, N, N), (1, 0, 0, 0), 2),
    "const_H": (32, 32, [16, 16], [16, 16], 16, 0, 1.0, "exponential", 1.0, 0.2, 3.0, (D, D, N, N), (1, 0, 0, 0), 3),
    "exact_h": (24, 24, [8, 8, 8], [12, 12], 1, 0, 0.5, "gaussian", 1.0, 0.1, 2.0, (D, D, N, N), (1, 0, 0, 0), 4),
    "single": (16, 12, [16], [12], 4, 1, 1.0, "exponential", 1.0, 0.2, 2.0, (D, D, N, N), (1, 0, 0, 0), 5),
    "rate_in": (32, 16, [16, 16], [16], 4, 1, 2.0, "exponential", 1.0, 0.2, 4.0, (N, D, N, N), (-1.0, 0, 0, 0), 6),
    "dirichlet4": (32, 32, [8, 8, 16], [16, 16], 8, 1, 1.0, "exponential", 1.0, 0.2, 2.0, (D, D, D, D), (1, 0, 0.5, 0.25), 7),
    "contrast64": (64, 64, [16] * 4, [16] * 4, 4, 1, 1.0, "gaussian", 4.0, 0.05, 5.0, (D, D, N, N), (1, 0, 0, 0), 8),
    # alpha varying face by face (aMRCM, Section 3.1): the alpha argument is replaced by a seeded field
    "alpha_field": (40, 36, [8, 12, 20], [12, 8, 16], 4, 1, None, "exponential", 2.0, 0.15, 5.0, (D, D, N, N),
                    (1, 0, 0, 0), 9),
    # 9 x 9 subdomains with 32 interface DOFs per side: the top separator (9 interfaces, 288
    # DOFs) and the boundaries of the level below it are longer than 256
    "long_sep": (144, 144, [16] * 9, [16] * 9, 2, 1, 1.0, "exponential", 1.0, 0.2, 3.0, (D, D, N, N), (1, 0, 0, 0), 10),
    # subdomain sides at the library's maximum (24 cells) beside narrower ones
    "max_side": (56, 48, [24, 8, 24], [24, 24], 4, 1, 1.0, "exponential", 2.0, 0.15, 4.0, (D, D, N, N), (1, 0, 0, 0), 11),
    # short sides: one to four block rows per subdomain, two-cell interfaces
    "small_sides": (16, 12, [4, 8, 4], [2, 6, 4], 2, 1, 1.0, "exponential", 1.0, 0.2, 2.0, (D, D, N, N), (1, 0, 0, 0),
                    12),
}


def alpha_field(nx, ny, seed, lo=0.1, hi=10.0):
    """Seeded per-face alpha(x), log-uniform in [lo, hi]: (alpha_x [ny][nx+1], alpha_y [ny+1][nx])."""
    rng = np.random.default_rng(1000 + seed)
    return (np.exp(rng.uniform(np.log(lo), np.log(hi), (ny, nx + 1))),
            np.exp(rng.uniform(np.log(lo), np.log(hi), (ny + 1, nx))))


def case(name, s_kind="random"):
    nx, ny, cw, rh, seg, deg, alpha, cov, s2, ell, M, bct, bcv, seed = CASES[name]
    h = 1.0 / nx
    K = fields.lognormal_grf(nx, ny, h, s2, ell, cov, seed)
    rng = np.random.default_rng(100 + seed)
    if s_kind == "random":
        s0 = rng.random((ny, nx))
    elif s_kind == "front":
        x = (np.arange(nx) + 0.5) / nx
        s0 = np.broadcast_to(np.clip(1.0 - x / 0.3, 0, 1), (ny, nx)).copy()
    else:
        s0 = np.zeros((ny, nx))
    af = alpha_field(nx, ny, seed) if alpha is None else None
    return dict(nx=nx, ny=ny, Lx=1.0, Ly=ny * h, h=h, col_w=cw, row_h=rh, seg_len=seg, degree=deg,
                alpha=1.0 if alpha is None else alpha, alpha_face=af, M=M, bc_type=bct, bc_val=bcv, K=K,
                s0=np.ascontiguousarray(s0), seed=seed)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
