"""Plain FP64 geometric multigrid with the kappa-cycle (Section 2.1, Algorithm 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Problem (Section 4): 2D rotated anisotropic diffusion on the unit square with
homogeneous Dirichlet boundary, discretised by the nine-point stencil printed in
Section 4, on an n x n interior grid (n = 2^k - 1, h = 1/(n+1)).

Grid convention used by every function here:
  * a grid function is a float64 array of shape (n, n) holding interior points only;
  * index [j, i]: i is the x index, j is the y index, j+1 is "north";
  * Dirichlet boundary values are zero and are never stored.
A stencil is a 3x3 array ``st`` with ``st[1+dy, 1+dx]`` the coefficient that multiplies
v(i+dx, j+dy) in (A v)(i, j).

Precision: FP64 (every input the tests and the bench pass is float64). Work arrays take the dtype
of the function's input, so the same steps run unchanged on float32 data when a test wants the
size of FP32 rounding in this algorithm (a calibration for the FP32 cycle; FP64 results are
unaffected).

Readings of the paper taken here:
  * The operator is A = S / h^2 with S the printed table (the table omits h^2).
  * The top row of the printed table is north (j+1); then the corner entries are
    NW = SE = +(1-eps)CS/2 and NE = SW = -(1-eps)CS/2, which is the standard
    second-difference discretisation of -div(K grad u), K = R(theta) diag(1, eps) R^T.
  * Coarse operators are Galerkin, A^{l+1} = R A^l P, with full weighting R and
    bilinear P (named in Section 4 for the zebra solvers; used here for all solvers); the
    centre of each coarse stencil is evaluated from the exact zero-row-sum identity
    (``zero_row_sum_centre``).
  * Relaxation is damped Jacobi, v <- v + (omega / a0) (f - A v), a0 the stencil centre.
  * The coarsest level is solved exactly (Algorithm 3, first step): v = f / a0 for a
    1x1 grid, a dense Cholesky solve otherwise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np
import scipy.linalg

__all__ = [
    "cos_sin", "fine_stencil", "convection_stencil", "fine_stencil_derivatives", "apply_stencil", "restrict_fw",
    "prolong_bilinear", "galerkin_stencil", "zero_row_sum_centre", "jacobi", "zebra_lines", "relax",
    "restrict_fw_y", "prolong_y", "galerkin_stencil_y", "Hierarchy", "CallRecorder",
    "kcycle", "gamma_cycle", "f_cycle", "kcycle_adjoint", "cycle", "cycle_adjoint",
    "residual", "relres", "solve", "solve_error_reduction", "pcg", "precondition", "param_grads", "level_sizes",
]


# ----------------------------------------------------------------------------------------
# Discretisation (Section 4)
# ----------------------------------------------------------------------------------------

def cos_sin(theta: float):
    """cos(theta) and sin(theta) correctly rounded to FP64.

    Taylor series of cos and sin evaluated in 60-digit decimal arithmetic on the exact value of
    the FP64 argument (|theta| <= 8), then rounded once. Correct rounding makes the result
    independent of any math library, so every implementation that rounds correctly gets the
    same bits. Pinned against math.cos / math.sin (within 1 ulp) in the tests.
    """
    from decimal import Decimal, localcontext
    if not abs(theta) <= 8.0:
        raise ValueError("theta must satisfy |theta| <= 8")
    fr = Fraction(theta)
    with localcontext() as ctx:
        ctx.prec = 60
        x = Decimal(fr.numerator) / Decimal(fr.denominator)
        term, c, s = Decimal(1), Decimal(0), Decimal(0)
        for k in range(160):      # x^k / k!, signs of cos (k even) and sin (k odd)
            if k % 4 == 0:
                c += term
            elif k % 4 == 1:
                s += term
            elif k % 4 == 2:
                c -= term
            else:
                s -= term
            term = term * x / (k + 1)
        return float(Fraction(c)), float(Fraction(s))


def fine_stencil(theta: float, eps: float, n: int) -> np.ndarray:
    """Nine-point stencil of Section 4 for angle theta and anisotropy eps, scaled by 1/h^2.

    Centre 2(1+eps); west/east -(C^2 + eps S^2); south/north -(eps C^2 + S^2);
    NW and SE +(1-eps)CS/2; NE and SW -(1-eps)CS/2; C = cos(theta), S = sin(theta),
    each correctly rounded (``cos_sin``); entries evaluated left to right, then divided by h*h.
    """
    h = 1.0 / (n + 1)
    C, S = cos_sin(theta)
    cross = 0.5 * (1.0 - eps) * C * S
    st = np.zeros((3, 3))
    st[1, 1] = 2.0 * (1.0 + eps)                 # centre
    st[1, 0] = st[1, 2] = -(C * C + eps * S * S)  # west, east
    st[0, 1] = st[2, 1] = -(eps * C * C + S * S)  # south, north
    st[2, 0] = cross                              # north-west
    st[0, 2] = cross                              # south-east
    st[2, 2] = -cross                             # north-east
    st[0, 0] = -cross                             # south-west
    return st / (h * h)


def convection_stencil(st: np.ndarray, bx: float, by: float, n: int) -> np.ndarray:
    """The Section 4 stencil plus first-order upwind convection b . grad u, b = (bx, by): the
    non-symmetric test problem the conclusions suggest (Section 5), -div(K grad u) + b . grad u.
    bx > 0 differences u backwards in x, (u_i - u_(i-1)) / h: centre +bx/h, west -bx/h; bx < 0
    forwards: centre +|bx|/h, east -|bx|/h; likewise in y (south / north). With 1/h = n + 1:
    cx = |bx| (n + 1), cy = |by| (n + 1), centre += (cx + cy), each step rounded once.
    """
    out = st.copy()
    cx = abs(bx) * float(n + 1)
    cy = abs(by) * float(n + 1)
    out[1, 1] = out[1, 1] + (cx + cy)
    if bx > 0:
        out[1, 0] = out[1, 0] - cx
    elif bx < 0:
        out[1, 2] = out[1, 2] - cx
    if by > 0:
        out[0, 1] = out[0, 1] - cy
    elif by < 0:
        out[2, 1] = out[2, 1] - cy
    return out


def fine_stencil_derivatives(theta: float, eps: float, n: int):
    """Derivatives d(stencil)/d(theta) and d(stencil)/d(eps) of ``fine_stencil``.

    Differentiating the Section 4 entries term by term:
      d/dtheta: centre 0; W/E +(1-eps) sin 2theta; S/N -(1-eps) sin 2theta;
                NW/SE +(1-eps) cos 2theta / 2; NE/SW -(1-eps) cos 2theta / 2.
      d/deps:   centre 2; W/E -S^2; S/N -C^2; NW/SE -CS/2; NE/SW +CS/2.
    Both scaled by 1/h^2. Pinned by central differences of ``fine_stencil``.
    """
    h2 = (1.0 / (n + 1)) ** 2
    C, S = math.cos(theta), math.sin(theta)
    s2, c2 = math.sin(2 * theta), math.cos(2 * theta)
    dth = np.zeros((3, 3))
    dth[1, 0] = dth[1, 2] = (1.0 - eps) * s2
    dth[0, 1] = dth[2, 1] = -(1.0 - eps) * s2
    dth[2, 0] = dth[0, 2] = 0.5 * (1.0 - eps) * c2
    dth[2, 2] = dth[0, 0] = -0.5 * (1.0 - eps) * c2
    dep = np.zeros((3, 3))
    dep[1, 1] = 2.0
    dep[1, 0] = dep[1, 2] = -S * S
    dep[0, 1] = dep[2, 1] = -C * C
    dep[2, 0] = dep[0, 2] = -0.5 * C * S
    dep[2, 2] = dep[0, 0] = 0.5 * C * S
    return dth / h2, dep / h2


def apply_stencil(st: np.ndarray, v: np.ndarray) -> np.ndarray:
    """(A v) for a constant 9-point stencil with zero Dirichlet values outside the grid."""
    ny, nx = v.shape
    padded = np.zeros((ny + 2, nx + 2), dtype=v.dtype)
    padded[1:-1, 1:-1] = v
    out = np.zeros_like(v)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out += st[1 + dy, 1 + dx] * padded[1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
    return out


def residual(st: np.ndarray, v: np.ndarray, f: np.ndarray) -> np.ndarray:
    """r = f - A v."""
    return f - apply_stencil(st, v)


# ----------------------------------------------------------------------------------------
# Inter-grid transfers (full weighting and bilinear interpolation, Section 4)
# ----------------------------------------------------------------------------------------

def restrict_fw(r: np.ndarray) -> np.ndarray:
    """Full-weighting restriction (1/16)[1 2 1; 2 4 2; 1 2 1].

    Fine grid (2m+1)^2 -> coarse grid m^2; coarse point (J, I) sits on fine point
    (2J+1, 2I+1), so all nine fine points it reads are interior.
    """
    nf = r.shape[0]
    m = (nf - 1) // 2
    weights = {-1: 1.0, 0: 2.0, 1: 1.0}
    rows = 2 * np.arange(m) + 1
    out = np.zeros((m, m), dtype=r.dtype)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out += (weights[dy] * weights[dx] / 16.0) * r[np.ix_(rows + dy, rows + dx)]
    return out


def prolong_bilinear(vc: np.ndarray) -> np.ndarray:
    """Bilinear interpolation from an m x m coarse grid to the (2m+1)^2 fine grid.

    Coarse values are injected at fine points with both indices odd; fine points with
    one even index average their two coarse neighbours along that axis; fine points
    with both indices even average their four diagonal coarse neighbours. Coarse
    neighbours outside the grid are the zero Dirichlet values.
    """
    m = vc.shape[0]
    nf = 2 * m + 1
    pc = np.zeros((m + 2, m + 2), dtype=vc.dtype)  # coarse grid with its zero boundary ring
    pc[1:-1, 1:-1] = vc                # pc[J+1, I+1] = vc[J, I]
    out = np.zeros((nf, nf), dtype=vc.dtype)
    out[1::2, 1::2] = vc
    out[1::2, 0::2] = 0.5 * (pc[1:-1, :-1] + pc[1:-1, 1:])
    out[0::2, 1::2] = 0.5 * (pc[:-1, 1:-1] + pc[1:, 1:-1])
    out[0::2, 0::2] = 0.25 * (pc[:-1, :-1] + pc[:-1, 1:] + pc[1:, :-1] + pc[1:, 1:])
    return out


def galerkin_stencil(st: np.ndarray) -> np.ndarray:
    """Coarse stencil of A_c = R A P (Section 4, Galerkin coarse-grid operator).

    Written as the definition: apply P, then A, then R to a coarse unit vector e_c far
    from the boundary. R A P e_c is column c of A_c; for a constant-coefficient operator
    the row entry for offset d is A_c[c, c+d] = (R A P e_c)[c - d].
    Evaluated in exact rational arithmetic on the FP64 entries of ``st`` and rounded once to
    FP64 (correct rounding), with plain loops on an 11 x 11 fine / 5 x 5 coarse grid that
    follow ``prolong_bilinear``, ``apply_stencil`` and ``restrict_fw`` rule by rule.
    """
    m, c = 5, 2
    nf = 2 * m + 1
    S = [[Fraction(float(st[a, b])) for b in range(3)] for a in range(3)]
    half = Fraction(1, 2)

    def hat(fine, coarse):  # bilinear weight of coarse point `coarse` at fine index `fine`
        d = abs(fine - (2 * coarse + 1))
        return Fraction(1) if d == 0 else (half if d == 1 else Fraction(0))

    pe = [[hat(j, c) * hat(i, c) for i in range(nf)] for j in range(nf)]          # P e_c
    ape = [[sum((S[1 + dy][1 + dx] * pe[j + dy][i + dx]
                 for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                 if 0 <= j + dy < nf and 0 <= i + dx < nf), Fraction(0))
            for i in range(nf)] for j in range(nf)]                                 # A P e_c
    fw = {-1: 1, 0: 2, 1: 1}
    col = [[sum((Fraction(fw[dy] * fw[dx], 16) * ape[2 * J + 1 + dy][2 * I + 1 + dx]
                 for dy in (-1, 0, 1) for dx in (-1, 0, 1)), Fraction(0))
            for I in range(m)] for J in range(m)]                                   # R A P e_c
    out = np.zeros((3, 3))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out[1 + dy, 1 + dx] = float(col[c - dy][c - dx])
    return out


def restrict_fw_y(r: np.ndarray) -> np.ndarray:
    """Semi-coarsening restriction along y only (Section 4, solvers 5-6): the 1-D full weighting
    (1/4)[1 2 1] across rows; fine rows 2m+1 -> coarse rows m, coarse row J sits on fine row
    2J+1, every column kept."""
    m = (r.shape[0] - 1) // 2
    rows = 2 * np.arange(m) + 1
    return 0.25 * r[rows - 1] + 0.5 * r[rows] + 0.25 * r[rows + 1]


def prolong_y(vc: np.ndarray) -> np.ndarray:
    """Linear interpolation along y only: coarse row J is injected at fine row 2J+1; fine row
    2J averages coarse rows J-1 and J (zero Dirichlet rows outside)."""
    m, nx = vc.shape
    pc = np.zeros((m + 2, nx))
    pc[1:-1] = vc
    out = np.zeros((2 * m + 1, nx))
    out[1::2] = vc
    out[0::2] = 0.5 * (pc[:-1] + pc[1:])
    return out


def galerkin_stencil_y(st: np.ndarray) -> np.ndarray:
    """Coarse stencil of A_c = R_y A P_y for semi-coarsening along y (Section 4, solvers 5-6).

    The definition written out as for ``galerkin_stencil``: P_y, then A, then R_y applied to a
    coarse unit vector far from the boundary, on a 7-column by 11-row fine grid (5 coarse rows),
    in exact rational arithmetic on the FP64 entries, rounded once to FP64.
    """
    m, c, nxg, cx = 5, 2, 7, 3
    nf = 2 * m + 1
    S = [[Fraction(float(st[a, b])) for b in range(3)] for a in range(3)]
    half = Fraction(1, 2)

    def hat(fine, coarse):  # linear weight of coarse row `coarse` at fine row `fine`
        d = abs(fine - (2 * coarse + 1))
        return Fraction(1) if d == 0 else (half if d == 1 else Fraction(0))

    pe = [[hat(j, c) * (1 if i == cx else 0) for i in range(nxg)] for j in range(nf)]      # P_y e_c
    ape = [[sum((S[1 + dy][1 + dx] * pe[j + dy][i + dx]
                 for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                 if 0 <= j + dy < nf and 0 <= i + dx < nxg), Fraction(0))
            for i in range(nxg)] for j in range(nf)]                                        # A P_y e_c
    fw = {-1: Fraction(1, 4), 0: Fraction(1, 2), 1: Fraction(1, 4)}
    col = [[sum((fw[dy] * ape[2 * J + 1 + dy][i] for dy in (-1, 0, 1)), Fraction(0))
            for i in range(nxg)] for J in range(m)]                                         # R_y A P_y e_c
    out = np.zeros((3, 3))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out[1 + dy, 1 + dx] = float(col[c - dy][cx - dx])
    return out


def zero_row_sum_centre(st: np.ndarray) -> np.ndarray:
    """Coarse stencil with its centre evaluated from the zero-row-sum identity.

    The Section 4 stencil annihilates constants (its entries sum to 2(1+eps)(1 - C^2 - S^2) = 0),
    and the Galerkin map keeps the entry sum of a stencil (sum_D p(x - 2D) = 1 and sum_a r(a) = 1)
    while scaling the entries by about 1/4 per level, so every exact coarse stencil sums to zero.
    In FP64 the rounding of that sum would grow fourfold per level relative to the stencil
    (about 1e-10 at level 11); setting centre = -(sum of the eight off-centre entries, summed in
    row-major order) keeps each coarse stencil within a few ulp of the exact Galerkin stencil.
    Pinned against exact rational arithmetic in the tests.
    """
    out = st.copy()
    off = 0.0
    for dy in (0, 1, 2):
        for dx in (0, 1, 2):
            if (dy, dx) != (1, 1):
                off += float(st[dy, dx])
    out[1, 1] = -off
    return out


def jacobi(st: np.ndarray, v: np.ndarray, f: np.ndarray, omega: float, sweeps: int) -> np.ndarray:
    """Damped Jacobi: repeat ``sweeps`` times v <- v + (omega / a0)(f - A v)."""
    w = omega / st[1, 1]
    for _ in range(sweeps):
        v = v + w * (f - apply_stencil(st, v))
    return v


def zebra_lines(st: np.ndarray, v: np.ndarray, f: np.ndarray, axis: str) -> np.ndarray:
    """One zebra line Gauss-Seidel relaxation (Section 4, solvers 3-4): every line is solved
    exactly with its neighbouring lines held fixed, lines of even index first, then lines of odd
    index (using the new even lines). axis 'x': the lines are rows j (unknowns coupled through the
    west/east entries, a tridiagonal system); axis 'y': the lines are columns i (south/north).
    Off-line stencil entries move to the right-hand side with the current neighbouring values."""
    v = v.copy()
    work = v if axis == "x" else v.T                 # work[line, position]
    rhs_f = f if axis == "x" else f.T
    nl, n = work.shape                               # number of lines, points per line
    # stencil as seen along the line: s[dl, dp] multiplies work[line+dl, pos+dp]
    s = st if axis == "x" else st.T
    ab = np.zeros((3, n))                            # banded storage for solve_banded
    ab[0, 1:] = s[1, 2]                              # upper diagonal (position +1)
    ab[1, :] = s[1, 1]                               # diagonal
    ab[2, :-1] = s[1, 0]                             # lower diagonal (position -1)
    for parity in (0, 1):
        lines = np.arange(parity, nl, 2)
        if lines.size == 0:
            continue
        padded = np.zeros((nl + 2, n + 2))
        padded[1:-1, 1:-1] = work
        rhs = rhs_f[lines].copy()
        for dl in (-1, 1):
            for dp in (-1, 0, 1):
                rhs -= s[1 + dl, 1 + dp] * padded[lines + 1 + dl, 1 + dp:1 + dp + n]
        work[lines] = scipy.linalg.solve_banded((1, 1), ab, rhs.T).T
    return v


def relax(h: "Hierarchy", level: int, v: np.ndarray, f: np.ndarray, sweeps: int) -> np.ndarray:
    """The hierarchy's smoother: damped Jacobi; alternating zebra line relaxation ("zebra"), where
    the k-th relaxation runs along x for odd k and along y for even k (so two relaxations are one
    in each direction, x first, as in Section 4, solvers 3-4); or zebra relaxation along x only
    ("xzebra", Section 4, solvers 5-6)."""
    st = h.stencil(level)
    if h.smoother == "jacobi":
        return jacobi(st, v, f, h.omega, sweeps)
    for k in range(sweeps):
        v = zebra_lines(st, v, f, "x" if (k % 2 == 0 or h.smoother == "xzebra") else "y")
    return v


def level_sizes(n: int, levels: int):
    """Grid side per level, finest first: n, (n-1)/2, ... (Table 3: N = (2^n - 1)^2)."""
    sizes = [n]
    for _ in range(levels - 1):
        sizes.append((sizes[-1] - 1) // 2)
    return sizes


# ----------------------------------------------------------------------------------------
# Hierarchy
# ----------------------------------------------------------------------------------------

@dataclass
class Hierarchy:
    """Multigrid hierarchy: per-level stencils (level 1 finest) and cycle parameters."""
    n: int
    levels: int
    theta: float
    eps: float
    nu1: int = 2
    nu2: int = 2
    omega: float = 0.8
    coarse_op: str = "galerkin"   # or "rediscretized": the Section 4 stencil on each coarse grid
    smoother: str = "jacobi"      # or "zebra": alternating zebra line Gauss-Seidel; "xzebra": x lines only
    coarsening: str = "full"      # or "y": semi-coarsening along y only (every level keeps n columns)
    bx: float = 0.0               # convection b = (bx, by), upwind (a non-symmetric operator when nonzero)
    by: float = 0.0
    stencils: list = field(default_factory=list)
    sizes: list = field(default_factory=list)
    _chol: object = None
    _lu: object = None

    def __post_init__(self):
        k = int(round(math.log2(self.n + 1)))
        if self.n < 1 or (1 << k) - 1 != self.n or not (1 <= self.levels <= k):
            raise ValueError("n must be 2^k - 1 and 1 <= levels <= k")
        if self.smoother not in ("jacobi", "zebra", "xzebra"):
            raise ValueError("smoother must be 'jacobi', 'zebra' or 'xzebra'")
        if self.coarsening not in ("full", "y"):
            raise ValueError("coarsening must be 'full' or 'y'")
        if self.coarsening == "y" and (self.coarse_op != "galerkin" or self.levels != k):
            raise ValueError("semi-coarsening uses Galerkin operators down to a single row")
        self.sizes = level_sizes(self.n, self.levels)   # grid side; under "y" the number of rows
        st = fine_stencil(self.theta, self.eps, self.n)
        if self.bx != 0.0 or self.by != 0.0:
            st = convection_stencil(st, self.bx, self.by, self.n)
        self.stencils = [st]
        for lvl in range(1, self.levels):
            if self.coarsening == "y":
                st = zero_row_sum_centre(galerkin_stencil_y(st))
            elif self.coarse_op == "galerkin":
                st = zero_row_sum_centre(galerkin_stencil(st))
            elif self.coarse_op == "rediscretized":
                st = fine_stencil(self.theta, self.eps, self.sizes[lvl])
                if self.bx != 0.0 or self.by != 0.0:
                    st = convection_stencil(st, self.bx, self.by, self.sizes[lvl])
            else:
                raise ValueError("coarse_op must be 'galerkin' or 'rediscretized'")
            self.stencils.append(st)
        if self.coarsening == "y":
            return                     # the coarsest level is one row: a tridiagonal solve
        # coarsest-level operator as a dense SPD matrix, factorised once
        nc = self.sizes[-1]
        dense = np.zeros((nc * nc, nc * nc))
        for col in range(nc * nc):
            e = np.zeros(nc * nc)
            e[col] = 1.0
            dense[:, col] = apply_stencil(self.stencils[-1], e.reshape(nc, nc)).ravel()
        if self.bx != 0.0 or self.by != 0.0:   # non-symmetric: LU
            self._lu = scipy.linalg.lu_factor(dense)
        else:
            self._chol = scipy.linalg.cho_factor(dense, lower=True)

    def stencil(self, level: int) -> np.ndarray:
        return self.stencils[level - 1]

    def restrict(self, r: np.ndarray) -> np.ndarray:
        return restrict_fw_y(r) if self.coarsening == "y" else restrict_fw(r)

    def prolong(self, vc: np.ndarray) -> np.ndarray:
        return prolong_y(vc) if self.coarsening == "y" else prolong_bilinear(vc)

    def coarsest_solve(self, f: np.ndarray) -> np.ndarray:
        """Exact solve on the coarsest level: division for 1x1, dense Cholesky otherwise; under
        semi-coarsening the single remaining row's tridiagonal system (west, centre, east)."""
        if self.coarsening == "y":
            st = self.stencils[-1]
            n = f.shape[1]
            ab = np.zeros((3, n))
            ab[0, 1:], ab[1, :], ab[2, :-1] = st[1, 2], st[1, 1], st[1, 0]
            return scipy.linalg.solve_banded((1, 1), ab, f[0]).reshape(1, n)
        nc = self.sizes[-1]
        if nc == 1:
            return f / self.stencils[-1][1, 1]
        if self.bx != 0.0 or self.by != 0.0:
            return scipy.linalg.lu_solve(self._lu, f.ravel()).reshape(nc, nc)
        return scipy.linalg.cho_solve(self._chol, f.ravel()).reshape(nc, nc)


class CallRecorder:
    """Counts cycle-routine calls per level and the counters seen on the coarsest level."""

    def __init__(self, levels: int):
        self.per_level = [0] * (levels + 1)   # index by level 1..levels
        self.coarsest_counters = []

    def record(self, level: int, counter: int, coarsest: bool):
        self.per_level[level] += 1
        if coarsest:
            self.coarsest_counters.append(counter)


# ----------------------------------------------------------------------------------------
# Cycles: Algorithm 3 (kappa), Algorithm 1 (gamma), Algorithm 2 (F), and the adjoint
# ----------------------------------------------------------------------------------------

def kcycle(h: Hierarchy, level: int, v: np.ndarray, f: np.ndarray, kappa: int,
           rec: CallRecorder | None = None) -> np.ndarray:
    """Algorithm 3: v <- kappa-cycle(v, f, A, level, n, kappa)."""
    last = level == h.levels
    if rec is not None:
        rec.record(level, kappa, last)
    if last:                                              # coarsest: solve and return
        return h.coarsest_solve(f)
    st = h.stencil(level)
    v = relax(h, level, v, f, h.nu1)                      # relax nu1 times
    fc = h.restrict(f - apply_stencil(st, v))             # restrict the residual
    vc = np.zeros_like(fc)                                # v^{l+1} <- 0
    vc = kcycle(h, level + 1, vc, fc, kappa, rec)         # call with counter kappa
    if kappa > 1:
        vc = kcycle(h, level + 1, vc, fc, kappa - 1, rec)  # then with kappa - 1
    v = v + h.prolong(vc)                                  # coarse-grid correction
    v = relax(h, level, v, f, h.nu2)                       # relax nu2 times
    return v


def gamma_cycle(h: Hierarchy, level: int, v: np.ndarray, f: np.ndarray, gamma: int) -> np.ndarray:
    """Algorithm 1: the classical gamma-cycle (gamma=1 V, gamma=2 W)."""
    if level == h.levels:
        return h.coarsest_solve(f)
    st = h.stencil(level)
    v = relax(h, level, v, f, h.nu1)
    fc = h.restrict(f - apply_stencil(st, v))
    vc = np.zeros_like(fc)
    for _ in range(gamma):
        vc = gamma_cycle(h, level + 1, vc, fc, gamma)
    v = v + h.prolong(vc)
    return relax(h, level, v, f, h.nu2)


def f_cycle(h: Hierarchy, level: int, v: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Algorithm 2: the F-cycle (one recursive F-cycle, then one V-cycle)."""
    if level == h.levels:
        return h.coarsest_solve(f)
    st = h.stencil(level)
    v = relax(h, level, v, f, h.nu1)
    fc = h.restrict(f - apply_stencil(st, v))
    vc = np.zeros_like(fc)
    vc = f_cycle(h, level + 1, vc, fc)
    vc = gamma_cycle(h, level + 1, vc, fc, 1)
    v = v + h.prolong(vc)
    return relax(h, level, v, f, h.nu2)


def kcycle_adjoint(h: Hierarchy, level: int, v: np.ndarray, f: np.ndarray, kappa: int) -> np.ndarray:
    """Adjoint of Algorithm 3 (the cycle whose zero-start map is B^T).

    With A symmetric, a constant Jacobi diagonal and R = P^T / 4, transposing the cycle's
    error propagator swaps the pre- and post-smoothing counts and reverses the order of
    the two coarse calls: the call with counter kappa-1 runs first (from zero), then the
    call with counter kappa. Pinned by the dot-product test <x, B y> = <B^T x, y>.
    Damped Jacobi only (the transposed zebra smoother would also reverse its line order).
    """
    if h.smoother != "jacobi" or h.coarsening != "full":
        raise ValueError("the adjoint cycle is defined for damped Jacobi with full coarsening")
    if level == h.levels:
        return h.coarsest_solve(f)
    st = h.stencil(level)
    v = jacobi(st, v, f, h.omega, h.nu2)
    fc = restrict_fw(f - apply_stencil(st, v))
    vc = np.zeros_like(fc)
    if kappa > 1:
        vc = kcycle_adjoint(h, level + 1, vc, fc, kappa - 1)
    vc = kcycle_adjoint(h, level + 1, vc, fc, kappa)
    v = v + prolong_bilinear(vc)
    return jacobi(st, v, f, h.omega, h.nu1)


def cycle(h: Hierarchy, v: np.ndarray, f: np.ndarray, kappa: int, rec: CallRecorder | None = None):
    """One finest-level kappa-cycle."""
    return kcycle(h, 1, v, f, kappa, rec)


def cycle_adjoint(h: Hierarchy, v: np.ndarray, f: np.ndarray, kappa: int):
    """One finest-level adjoint kappa-cycle."""
    return kcycle_adjoint(h, 1, v, f, kappa)


# ----------------------------------------------------------------------------------------
# Solvers (Section 4: stand-alone cycles and CG preconditioned by one cycle)
# ----------------------------------------------------------------------------------------

def relres(h: Hierarchy, v: np.ndarray, f: np.ndarray) -> float:
    """||f - A v||_2 / ||f||_2 over the finest interior points."""
    return float(np.linalg.norm(residual(h.stencil(1), v, f)) / np.linalg.norm(f))


def solve(h: Hierarchy, f: np.ndarray, kappa: int, tol: float, max_cycles: int,
          v0: np.ndarray | None = None, adjoint: bool = False):
    """Stand-alone solver: repeat finest-level cycles until ||f-Av|| / ||f|| <= tol.

    Returns (v, history) with history[k-1] the relative residual after cycle k.
    """
    v = np.zeros_like(f) if v0 is None else v0.copy()
    fnorm = np.linalg.norm(f)
    hist = []
    step = cycle_adjoint if adjoint else cycle
    for _ in range(max_cycles):
        v = step(h, v, f, kappa)
        rho = float(np.linalg.norm(residual(h.stencil(1), v, f)) / fnorm)
        hist.append(rho)
        if rho <= tol:
            break
    return v, hist


def solve_error_reduction(h: Hierarchy, v0: np.ndarray, kappa: int, reduction: float, max_cycles: int):
    """The error-reduction protocol of Section 4: right-hand side zero (so the exact solution is
    zero and the iterate is the error), cycles from the initial guess v0 until
    ||v_k||_2 <= reduction * ||v0||_2. Returns (v, history of ||v_k|| / ||v0||)."""
    f = np.zeros_like(v0)
    v = v0.copy()
    n0 = np.linalg.norm(v0)
    hist = []
    for _ in range(max_cycles):
        v = cycle(h, v, f, kappa)
        hist.append(float(np.linalg.norm(v) / n0))
        if hist[-1] <= reduction:
            break
    return v, hist


def precondition(h: Hierarchy, r: np.ndarray, kappa: int, symmetric: bool = False) -> np.ndarray:
    """z = B r, one kappa-cycle from zero; with ``symmetric`` the symmetrised preconditioner
    z = (B + B^T - B^T A B) r = B r + B^T (r - A B r): the cycle, then the adjoint cycle on the
    remaining residual, so that I - M A = (I - B^T A)(I - B A)."""
    z = cycle(h, np.zeros_like(r), r, kappa)
    if not symmetric:
        return z
    w = r - apply_stencil(h.stencil(1), z)
    return z + cycle_adjoint(h, np.zeros_like(r), w, kappa)


def pcg(h: Hierarchy, b: np.ndarray, kappa: int, tol: float, max_iters: int, flexible: bool = False,
        symmetric: bool = False):
    """Conjugate gradients preconditioned by one kappa-cycle from a zero start (MGCG).

    x0 = 0, r = b, z = B r, p = z; each iteration: q = A p, alpha = (r.z)/(p.q),
    x += alpha p, r -= alpha q, stop when ||r||/||b|| <= tol, z = B r,
    beta = (r_new.z_new)/(r.z) (or (r_new.(z_new - z_old))/(r.z) when ``flexible``),
    p = z + beta p. Returns (x, history) with history[k-1] = ||r_k|| / ||b||.
    """
    st = h.stencil(1)
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    z = precondition(h, r, kappa, symmetric)
    p = z.copy()
    rz = float(np.sum(r * z))
    hist = []
    for _ in range(max_iters):
        q = apply_stencil(st, p)
        alpha = rz / float(np.sum(p * q))
        x = x + alpha * p
        r = r - alpha * q
        rho = float(np.linalg.norm(r) / bnorm)
        hist.append(rho)
        if rho <= tol:
            break
        z_new = precondition(h, r, kappa, symmetric)
        if flexible:
            rz_new = float(np.sum(r * z_new))
            beta = float(np.sum(r * (z_new - z))) / rz
        else:
            rz_new = float(np.sum(r * z_new))
            beta = rz_new / rz
        p = z_new + beta * p
        z = z_new
        rz = rz_new
    return x, hist


def param_grads(theta: float, eps: float, n: int, lam: np.ndarray, u: np.ndarray):
    """dL/dtheta and dL/deps for u = A(theta, eps)^{-1} f and lam = A^{-T} dL/du.

    Differentiating A u = f gives du/dp = -A^{-1} (dA/dp) u, hence
    dL/dp = -lam^T (dA/dp) u with dA/dp the stencil derivative applied to u.
    """
    dth, dep = fine_stencil_derivatives(theta, eps, n)
    return (-float(np.sum(lam * apply_stencil(dth, u))),
            -float(np.sum(lam * apply_stencil(dep, u))))
