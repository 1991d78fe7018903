"""Plain CPU FP64 oracle of one Taylor–Couette DNS time step.

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py``.  It shares no code with the CUDA library.

What it restates (Shi, Rampp, Hof & Avila, "A hybrid MPI-OpenMP parallel implementation
for pseudospectral simulations with application to Taylor–Couette flow"):

* radial nodes                         Sec. 3.1, Eq. nodeDist
* finite-difference weights            Sec. 3.1 (central stencils of n_s = fd_order + 1
                                       points, shortened towards the walls)
* Fourier expansion and 3/2 dealiasing Sec. 3.1, Eq. fourier and the dealiased grid
* nonlinear term N(u) = u . grad u     Sec. 2, Eq. NS_cyl (left-hand sides) and Eq. pp
* mode operators and u_+/u_- variables Sec. 3.1, Eq. modalNS / Eq. modalNSdecoup
* AB2BD2 projection step               Sec. 3.2, Eq. timeScheme, Eq. pressure, Eq. vel,
                                       Eq. correction, Eq. update; consistent Neumann
                                       condition Eq. ppBC; singular (0,0) mode fix Sec. 3.2
* diagnostics: perturbation energy, torque (Sec. 5.4 quasi-Nusselt number), divergence.

Everything is written from the definitions: transforms are explicit DFT matrices applied
by matrix products, the five linear systems per Fourier mode are assembled as dense
matrices and solved by the oracle's own Gaussian elimination with partial pivoting over
their band (``gauss_banded``).  Angles, nodes and finite-difference weights are computed in
long double and rounded once to float64.

Readings where the paper is silent (the same readings bind the CUDA path):
  nodes     N_r nodes j = 0..N_r-1 including both walls (paper's M = N_r - 1);
  stencils  interior row j: centred, half width min(j, N_r-1-j, fd_order/2); wall rows
            (Neumann rows, wall values of the Laplacian, torque): one-sided over the
            fd_order/2 + 1 nodes nearest the wall;
  grid      physical grid P_theta x P_z, default 3M x 3K (only the edge modes alias);
  storage   m = 0..M, k = -K..K; the m = 0 line enters the real-valued inverse transform
            through its real part (u = Re(sum_m c_m f_m e^{i m theta}), c_0 = 1, c_m = 2);
  Neumann   d_r p* = -(2N^i - N^{i-1})_r + (2 (Lap u)^i - (Lap u)^{i-1})_r at both walls;
  (0,0)     Poisson rows for p* and phi use a homogeneous Dirichlet row at r_o;
  start     a cold state first takes one implicit Euler step of size 2 dt / 3 (the scheme
            with u^{-1} = u^0, N^{-1} = N^0) and extrapolates u^{-1} = u^0 - 1.5 (u_E - u^0),
            N^{-1} = N(u^{-1}), so the global error stays second order.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "Params", "Operators", "State", "radial_nodes", "fd_weights", "stencil_nodes",
    "derivative_matrices", "build_operators", "to_physical", "to_spectral",
    "physical_fields", "nonlinear", "mode_matrices", "div_h", "grad_h", "vector_laplacian_r",
    "gauss_banded", "solve_modes", "advance", "start_up", "step", "run", "couette_state",
    "perturbation_energy", "torque", "max_divergence", "cold_state", "nonlinear_tangent",
    "tangent_step", "nonlinear_adjoint", "adjoint_step", "adjoint_advance", "adjoint_start_up",
    "energy_gradient", "gradient_final_energy", "inner",
]

LD = np.longdouble
PI_LD = LD("3.14159265358979323846264338327950288419716939937510")


class Params:
    """Physical and numerical parameters (names follow the C-ABI: N_r nodes, modes
    m = 0..M with fundamental wavenumber m_p, k = -K..K with k_z = 2 pi / L_z)."""

    def __init__(self, N_r, M, K, m_p, eta, Re_i, Re_o, L_z, dt, fd_order=8, alpha=0.5,
                 P_theta=None, P_z=None):
        if fd_order % 2 or fd_order < 2:
            raise ValueError("fd_order must be even and >= 2")
        if N_r < fd_order // 2 + 2:
            raise ValueError("N_r too small for the wall stencil")
        self.N_r, self.M, self.K, self.m_p = int(N_r), int(M), int(K), int(m_p)
        self.eta, self.Re_i, self.Re_o = float(eta), float(Re_i), float(Re_o)
        self.L_z, self.dt, self.fd_order, self.alpha = float(L_z), float(dt), int(fd_order), float(alpha)
        self.P_theta = int(P_theta) if P_theta else 3 * self.M
        self.P_z = int(P_z) if P_z else 3 * self.K
        if self.P_theta < 2 * self.M + 1 or self.P_z < 2 * self.K + 1:
            raise ValueError("physical grid must hold every stored mode")
        self.k_z = 2.0 * math.pi / self.L_z
        self.r_i = self.eta / (1.0 - self.eta)
        self.r_o = 1.0 / (1.0 - self.eta)

    def shape(self):
        return (self.N_r, self.M + 1, 2 * self.K + 1)


# ----------------------------------------------------------------------------------------
# Radial discretisation (Sec. 3.1)
# ----------------------------------------------------------------------------------------

def radial_nodes(N_r, eta, alpha):
    """Eq. nodeDist with j = 0..N_r-1 (paper's M = N_r - 1); alpha = 0 is the Chebyshev
    limit -cos(pi j / M) / 2 of the second term."""
    j = np.arange(N_r, dtype=LD)
    c = np.cos(PI_LD * j / LD(N_r - 1))
    eta_l = LD(eta)
    centre = (LD(1) + eta_l) / (LD(2) * (LD(1) - eta_l))
    if alpha == 0.0:
        s = -c / LD(2)
    else:
        a = LD(alpha)
        s = np.arcsin(-a * c) / (LD(2) * np.arcsin(a))
    return (centre + s).astype(np.float64), (centre + s)


def _solve_ld(A, b):
    """Gaussian elimination with partial pivoting on a small long-double system."""
    n = len(b)
    A = [list(row) for row in A]
    b = list(b)
    for c in range(n):
        p = max(range(c, n), key=lambda i: abs(A[i][c]))
        A[c], A[p] = A[p], A[c]
        b[c], b[p] = b[p], b[c]
        for i in range(c + 1, n):
            f = A[i][c] / A[c][c]
            if f != 0:
                for j in range(c, n):
                    A[i][j] -= f * A[c][j]
                b[i] -= f * b[c]
    x = [LD(0)] * n
    for i in range(n - 1, -1, -1):
        s = b[i]
        for j in range(i + 1, n):
            s -= A[i][j] * x[j]
        x[i] = s / A[i][i]
    return x


def fd_weights(x0, xs, deriv):
    """Weights w with sum_i w_i f(x_i) = f^(deriv)(x0) exactly for polynomials of degree
    < len(xs): the Taylor moment conditions sum_i w_i (x_i - x0)^q / q! = [q == deriv],
    solved in long double on scaled offsets."""
    xs = [LD(x) for x in xs]
    x0 = LD(x0)
    h = max(abs(x - x0) for x in xs)
    t = [(x - x0) / h for x in xs]
    n = len(xs)
    A = [[t[i] ** q / LD(math.factorial(q)) for i in range(n)] for q in range(n)]
    rhs = [LD(1) if q == deriv else LD(0) for q in range(n)]
    w = _solve_ld(A, rhs)
    return [wi / h ** deriv for wi in w]


def stencil_nodes(j, N_r, half):
    """Node indices of row j: one-sided {0..half} / {N_r-1-half..N_r-1} at the walls,
    centred of half width min(j, N_r-1-j, half) inside."""
    if j == 0:
        return list(range(0, half + 1))
    if j == N_r - 1:
        return list(range(N_r - 1 - half, N_r))
    h = min(j, N_r - 1 - j, half)
    return list(range(j - h, j + h + 1))


def derivative_matrices(r_ld, fd_order):
    """Dense first and second radial-derivative matrices D1, D2 (float64)."""
    N = len(r_ld)
    half = fd_order // 2
    D1 = np.zeros((N, N))
    D2 = np.zeros((N, N))
    for j in range(N):
        idx = stencil_nodes(j, N, half)
        xs = [r_ld[i] for i in idx]
        w1 = fd_weights(r_ld[j], xs, 1)
        w2 = fd_weights(r_ld[j], xs, 2) if len(idx) >= 3 else [LD(0)] * len(idx)
        for i, a, b in zip(idx, w1, w2):
            D1[j, i] = float(a)
            D2[j, i] = float(b)
    return D1, D2


# ----------------------------------------------------------------------------------------
# Fourier transforms with zero padding / truncation (Eq. fourier, 3/2 rule)
# ----------------------------------------------------------------------------------------

def _unit_roots(P, idx_prod, sign):
    """exp(sign * 2 pi i * (idx_prod mod P) / P) from long-double angles."""
    q = np.mod(idx_prod, P).astype(LD)
    ang = LD(2) * PI_LD * q / LD(P)
    return (np.cos(ang).astype(np.float64) + 1j * sign * np.sin(ang).astype(np.float64))


class Operators:
    """Everything the oracle precomputes for a parameter set."""

    def __init__(self, prm: Params):
        self.prm = prm
        self.r, self.r_ld = radial_nodes(prm.N_r, prm.eta, prm.alpha)
        self.D1, self.D2 = derivative_matrices(self.r_ld, prm.fd_order)
        M, K, Pt, Pz = prm.M, prm.K, prm.P_theta, prm.P_z
        m = np.arange(M + 1)
        k = np.arange(-K, K + 1)
        a = np.arange(Pt)
        b = np.arange(Pz)
        # inverse z: f(z_b) = sum_k X_k e^{+i k k_z z_b},  z_b = b L_z / P_z
        self.EzT = _unit_roots(Pz, np.outer(k, b), +1)            # (2K+1, P_z)
        # inverse theta: u(theta_a) = Re sum_m c_m f_m e^{+i m m_p theta_a}
        c = np.full(M + 1, 2.0)
        c[0] = 1.0
        self.G = _unit_roots(Pt, np.outer(a, m), +1) * c[None, :]  # (P_theta, M+1)
        # forward transforms, scaled by 1/P
        self.Ft = _unit_roots(Pt, np.outer(m, a), -1) / Pt          # (M+1, P_theta)
        self.FzT = _unit_roots(Pz, np.outer(b, k), -1) / Pz         # (P_z, 2K+1)
        self.mm = prm.m_p * m.astype(np.float64)                    # m m_p
        self.kk = prm.k_z * k.astype(np.float64)                    # k k_z
        self._mats = None

    @property
    def mats(self):
        if self._mats is None:
            self._mats = mode_matrices(self)
        return self._mats


def build_operators(prm):
    return Operators(prm)


def to_physical(ops, a):
    """(..., N_r, M+1, 2K+1) coefficients -> (..., N_r, P_theta, P_z) real field."""
    f = np.matmul(a, ops.EzT)                 # (..., N_r, M+1, P_z)
    return np.real(np.matmul(ops.G, f))       # (..., N_r, P_theta, P_z)


def to_spectral(ops, u):
    """(..., N_r, P_theta, P_z) real field -> coefficients m = 0..M, k = -K..K."""
    g = np.matmul(ops.Ft, u)                  # (..., N_r, M+1, P_z)
    return np.matmul(g, ops.FzT)              # (..., N_r, M+1, 2K+1)


def _dr(ops, a):
    return np.tensordot(ops.D1, a, axes=(1, 0))


def physical_fields(ops, u_hat, rows=None):
    """The twelve physical fields of step 1 of Sec. 3.2: for c in (r, theta, z):
    u_c, d_r u_c, d_theta u_c, d_z u_c (d_theta is the angle derivative).

    rows: radial rows to evaluate (default all).  Each row's fields need only that row and,
    for d_r, the rows of its stencil, so the others are not touched (the same arithmetic)."""
    if rows is None:
        sub, D, sel = u_hat, ops.D1, slice(None)
    else:
        rows = np.atleast_1d(rows)
        need = np.unique(np.concatenate([rows, np.nonzero(np.any(ops.D1[rows] != 0, axis=0))[0]]))
        sub, D, sel = u_hat[:, need], ops.D1[np.ix_(rows, need)], np.searchsorted(need, rows)
    up, um, uz = sub
    comps = [(up + um) / 2.0, (up - um) / 2j, uz]
    im = 1j * ops.mm[None, :, None]
    ik = 1j * ops.kk[None, None, :]
    out = []
    for a in comps:
        ar = a[sel]
        out.append([to_physical(ops, ar), to_physical(ops, np.tensordot(D, a, axes=(1, 0))),
                    to_physical(ops, im * ar), to_physical(ops, ik * ar)])
    return out


def nonlinear(ops, u_hat, rows=None):
    """N(u) = u . grad u with the curvature terms of Eq. NS_cyl, dealiased; returned as
    (N_+, N_-, N_z) coefficients with N_pm = N_r +- i N_theta.  rows: radial rows to evaluate
    (default all); the result then has those rows only."""
    (ur, ur_r, ur_t, ur_z), (ut, ut_r, ut_t, ut_z), (uz, uz_r, uz_t, uz_z) = physical_fields(ops, u_hat, rows)
    r = (ops.r if rows is None else ops.r[np.atleast_1d(rows)])[:, None, None]

    def adv(f_r, f_t, f_z):
        return ur * f_r + (ut / r) * f_t + uz * f_z

    Nr = adv(ur_r, ur_t, ur_z) - ut * ut / r
    Nt = adv(ut_r, ut_t, ut_z) + ut * ur / r
    Nz = adv(uz_r, uz_t, uz_z)
    Nr_h, Nt_h, Nz_h = (to_spectral(ops, f) for f in (Nr, Nt, Nz))
    return np.stack([Nr_h + 1j * Nt_h, Nr_h - 1j * Nt_h, Nz_h])


# ----------------------------------------------------------------------------------------
# Per-mode operators (Eq. modalNSdecoup) and the five systems of Sec. 3.2
# ----------------------------------------------------------------------------------------

def mode_matrices(ops, m=None, ka=None):
    """Dense real matrices indexed [m, |k|]: 'P' Poisson with Neumann wall rows (Dirichlet
    at r_o for (0,0)); 'Hp', 'Hm', 'Hz' = 3/(2 dt) I - L_c with Dirichlet wall rows.
    m, ka: one mode (m, |k|) only (the result then has leading shape (1, 1)); default all."""
    prm = ops.prm
    N, M, K = prm.N_r, prm.M, prm.K
    r = ops.r
    I = np.eye(N)
    ms = np.arange(M + 1) if m is None else np.array([m])
    kas = np.arange(K + 1) if ka is None else np.array([ka])
    mm = ops.mm[ms][:, None, None, None]
    ka = (prm.k_z * kas)[None, :, None, None]
    D1, D2 = ops.D1, ops.D2
    inv_r = (1.0 / r)[:, None]
    inv_r2 = (1.0 / r ** 2)[:, None]
    base = D2 + inv_r * D1                                  # d_rr + (1/r) d_r
    Lh = base[None, None] - mm ** 2 * inv_r2 * I - ka ** 2 * I   # (M+1, K+1, N, N)
    P = Lh.copy()
    P[:, :, 0, :] = D1[0]
    P[:, :, -1, :] = D1[-1]
    if ms[0] == 0 and kas[0] == 0:
        P[0, 0, -1, :] = I[-1]
    c = 3.0 / (2.0 * prm.dt)
    Lp = Lh - inv_r2 * I - 2.0 * mm * inv_r2 * I
    Lm = Lh - inv_r2 * I + 2.0 * mm * inv_r2 * I
    out = {"P": P}
    for name, L in (("Hp", Lp), ("Hm", Lm), ("Hz", Lh)):
        H = c * I - L
        H[:, :, 0, :] = I[0]
        H[:, :, -1, :] = I[-1]
        out[name] = H
    out["Lp"], out["Lm"] = Lp, Lm
    return out


def gauss_banded(A, B, kl=4, ku=4):
    """Solve A x = B by Gaussian elimination with partial pivoting (row interchanges), for
    a batch of real matrices A[..., N, N] with A[i, j] = 0 unless -kl <= j - i <= ku, and
    right-hand sides B[..., N, nrhs].  The paper solves each mode's banded system once per
    step with precomputed LU factors and row interchanges (Sec. 3.2); this is the same
    elimination done afresh, with B carried along.

    Column c: the pivot is the largest |A[i, c]| over rows i = c..c+kl (the rows below
    hold zeros there); rows c and p are interchanged; rows c+1..c+kl subtract multiples of
    row c.  The rows in the active window hold non-zeros only up to column c+kl+ku (row c+kl
    starts with its band edge there, and the pivot row never reaches further), so the
    interchange and the elimination touch columns c..c+kl+ku only.  Back substitution then
    runs over the kl+ku super-diagonals of the triangular result.  The batch is held as the
    last axis so that each step is one array operation over all systems; only the band of
    the input is copied into that layout (an entry outside it raises ValueError)."""
    N = A.shape[-1]
    lead = A.shape[:-2]
    A_in = np.asarray(A, dtype=np.float64).reshape((-1, N, N))
    ii, jj = np.nonzero(np.abs(np.subtract.outer(np.arange(N), np.arange(N))) <= max(kl, ku))
    band = (jj - ii >= -kl) & (jj - ii <= ku)
    ii, jj = ii[band], jj[band]
    A = np.zeros((N, N, A_in.shape[0]))                                 # (N, N, nb)
    A[ii, jj] = A_in[:, ii, jj].T
    if np.count_nonzero(A) != np.count_nonzero(A_in):
        raise ValueError("matrix has entries outside the band")
    B = np.moveaxis(np.array(B, dtype=np.float64).reshape((-1, N, B.shape[-1])), 0, -1).copy()
    ib = np.arange(A.shape[-1])
    for c in range(N):
        last = min(c + kl, N - 1)
        hi = min(c + kl + ku, N - 1) + 1
        p = c + np.argmax(np.abs(A[c:last + 1, c]), axis=0)          # pivot row per system
        cols = np.arange(c, hi)[:, None]
        row_c, row_p = A[c, c:hi].copy(), A[p, cols, ib].copy()
        A[c, c:hi], A[p, cols, ib] = row_p, row_c
        b_c, b_p = B[c].copy(), B[p, :, ib].T.copy()
        B[c], B[p, :, ib] = b_p, b_c.T
        f = A[c + 1:last + 1, c] / A[c, c]                           # (rows, nb)
        A[c + 1:last + 1, c + 1:hi] -= f[:, None] * A[c, None, c + 1:hi]
        A[c + 1:last + 1, c] = 0.0
        B[c + 1:last + 1] -= f[:, None] * B[c, None]
    x = np.zeros_like(B)
    for i in range(N - 1, -1, -1):
        hi = min(i + kl + ku, N - 1) + 1
        s = B[i] - np.sum(A[i, i + 1:hi, None] * x[i + 1:hi], axis=0)
        x[i] = s / A[i, i]
    return np.moveaxis(x, -1, 0).reshape(lead + (N, x.shape[1]))


def solve_modes(ops, A, rhs):
    """Solve A[m, |k|] x[:, m, k] = rhs[:, m, k] for every stored mode: the matrices are
    real, so the real and imaginary parts of the right-hand sides of k = +|k| and -|k| are
    four right-hand sides of one elimination (`gauss_banded`)."""
    K = ops.prm.K
    b = np.moveaxis(rhs, 0, -1)                            # (M+1, 2K+1, N)
    bp, bm = b[:, K:], b[:, K::-1]                         # k = +|k| and k = -|k|
    B = np.stack([bp.real, bp.imag, bm.real, bm.imag], axis=-1)
    x = gauss_banded(A, B)                                 # (M+1, K+1, N, 4)
    out = np.empty(b.shape, np.complex128)
    out[:, K:] = x[..., 0] + 1j * x[..., 1]
    out[:, K::-1] = x[..., 2] + 1j * x[..., 3]
    return np.moveaxis(out, -1, 0)


def div_h(ops, v):
    """Discrete divergence of (v_+, v_-, v_z): D1 v_r + v_r / r + m m_p (v_+ - v_-)/(2r)
    + i k k_z v_z with v_r = (v_+ + v_-)/2 (Eq. NS_cyl, continuity)."""
    vp, vm, vz = v
    r = ops.r[:, None, None]
    vr = (vp + vm) / 2.0
    return (_dr(ops, vr) + vr / r + ops.mm[None, :, None] * (vp - vm) / (2.0 * r)
            + 1j * ops.kk[None, None, :] * vz)


def grad_h(ops, phi):
    """(grad phi)_pm = d_r phi -+ m m_p phi / r, (grad phi)_z = i k k_z phi."""
    r = ops.r[:, None, None]
    d = _dr(ops, phi)
    t = ops.mm[None, :, None] * phi / r
    return np.stack([d - t, d + t, 1j * ops.kk[None, None, :] * phi])


def vector_laplacian_r(ops, u):
    """r component of the vector Laplacian: ((L_+ u_+) + (L_- u_-)) / 2 with
    L_pm = Lap_h - 1/r^2 -+ 2 m m_p / r^2 (Eq. modalNSdecoup), all rows."""
    prm = ops.prm
    r = ops.r[:, None, None]
    mm = ops.mm[None, :, None]
    kk2 = (ops.kk ** 2)[None, None, :]

    def lap_h(a):
        return (np.tensordot(ops.D2, a, axes=(1, 0)) + _dr(ops, a) / r
                - mm ** 2 * a / r ** 2 - kk2 * a)

    up, um = u[0], u[1]
    Lp = lap_h(up) - up / r ** 2 - 2.0 * mm * up / r ** 2
    Lm = lap_h(um) - um / r ** 2 + 2.0 * mm * um / r ** 2
    del prm
    return (Lp + Lm) / 2.0


class State:
    """AB2BD2 state: u^i, u^{i-1}, N^{i-1}, p^i and whether a step has been taken."""

    def __init__(self, u, u_prev=None, N_prev=None, p=None, started=False):
        self.u = np.array(u, dtype=np.complex128)
        self.u_prev = None if u_prev is None else np.array(u_prev, dtype=np.complex128)
        self.N_prev = None if N_prev is None else np.array(N_prev, dtype=np.complex128)
        self.p = np.zeros(self.u.shape[1:], np.complex128) if p is None else np.array(p, np.complex128)
        self.started = bool(started)

    def copy(self):
        return State(self.u, self.u_prev, self.N_prev, self.p, self.started)


def cold_state(u0):
    return State(u0)


def dirichlet_values(ops):
    """Wall values of (u_+, u_-, u_z) (Eq. nsBC): (0,0) mode u_theta = Re_{i,o}."""
    prm = ops.prm
    vals = np.zeros((3, 2, prm.M + 1, 2 * prm.K + 1), np.complex128)
    vals[0, 0, 0, prm.K] = 1j * prm.Re_i
    vals[1, 0, 0, prm.K] = -1j * prm.Re_i
    vals[0, 1, 0, prm.K] = 1j * prm.Re_o
    vals[1, 1, 0, prm.K] = -1j * prm.Re_o
    return vals


def advance(ops, u, u_prev, N, N_prev):
    """Steps 2-5 of Sec. 3.2 given N^i = N and N^{i-1} = N_prev; returns
    (u^{i+1}, p^{i+1}, parts)."""
    prm = ops.prm
    mats = ops.mats
    K, dt = prm.K, prm.dt
    NN = 2.0 * N - N_prev
    # step 2: pressure prediction, Eq. pressure with the Neumann rows of Eq. ppBC
    b = div_h(ops, -NN)
    g = -(NN[0] + NN[1]) / 2.0 + 2.0 * vector_laplacian_r(ops, u) - vector_laplacian_r(ops, u_prev)
    b[0] = g[0]
    b[-1] = g[-1]
    b[-1, 0, K] = 0.0
    p_star = solve_modes(ops, mats["P"], b)
    # step 3: velocity prediction, Eq. vel, Dirichlet rows from Eq. nsBC
    gp = grad_h(ops, p_star)
    rhs = (4.0 * u - u_prev) / (2.0 * dt) - NN - gp
    wall = dirichlet_values(ops)
    rhs[:, 0] = wall[:, 0]
    rhs[:, -1] = wall[:, 1]
    u_star = np.stack([solve_modes(ops, mats[n], rhs[c]) for c, n in enumerate(("Hp", "Hm", "Hz"))])
    # step 4: correction potential, Eq. correction
    b = div_h(ops, u_star)
    b[0] = 0.0
    b[-1] = 0.0
    phi = solve_modes(ops, mats["P"], b)
    # step 5: update, Eq. update
    u_new = u_star - grad_h(ops, phi)
    p_new = p_star + 3.0 * phi / (2.0 * dt)
    return u_new, p_new, dict(p_star=p_star, u_star=u_star, phi=phi)


def start_up(ops, u0):
    """History for the first AB2BD2 step (not stated in the paper).  With u^{-1} = u^0
    and N^{-1} = N^0 the scheme is an implicit Euler step of size 2 dt / 3 (same matrices);
    its result u_E gives d_t u(0) ~ (u_E - u^0) / (2 dt / 3), from which
    u^{-1} = u^0 - 1.5 (u_E - u^0) and N^{-1} = N(u^{-1}) are second-order accurate."""
    N0 = nonlinear(ops, u0)
    u_e, _, _ = advance(ops, u0, u0, N0, N0)
    u_m1 = u0 - 1.5 * (u_e - u0)
    return State(u0, u_m1, nonlinear(ops, u_m1), None, True)


def step(ops, st: State, return_parts=False):
    """One AB2BD2 step, steps 1-5 of Sec. 3.2 (a cold state is first given its history)."""
    if not st.started:
        st = start_up(ops, st.u)
    N = nonlinear(ops, st.u)                                # step 1
    u_new, p_new, parts = advance(ops, st.u, st.u_prev, N, st.N_prev)
    new = State(u_new, st.u, N, p_new, True)
    if return_parts:
        parts["N"] = N
        return new, parts
    return new


def run(ops, st, nsteps):
    for _ in range(nsteps):
        st = step(ops, st)
    return st


# ----------------------------------------------------------------------------------------
# Diagnostics
# ----------------------------------------------------------------------------------------

def couette_state(ops):
    """Analytic circular Couette flow at the nodes (Sec. 5.1) in stored layout, with its
    exact pressure normalised to p(r_o) = 0."""
    prm = ops.prm
    eta, Re_i, Re_o = prm.eta, prm.Re_i, prm.Re_o
    C1 = (Re_o - eta * Re_i) / (1.0 + eta)
    C2 = eta * (Re_i - eta * Re_o) / ((1.0 - eta) * (1.0 - eta * eta))
    r = ops.r
    U = C1 * r + C2 / r

    def pres(x):
        return C1 * C1 * x * x / 2.0 + 2.0 * C1 * C2 * np.log(x) - C2 * C2 / (2.0 * x * x)

    u = np.zeros((3,) + prm.shape(), np.complex128)
    u[0, :, 0, prm.K] = 1j * U
    u[1, :, 0, prm.K] = -1j * U
    p = np.zeros(prm.shape(), np.complex128)
    p[:, 0, prm.K] = pres(r) - pres(prm.r_o)
    return u, p, (C1, C2)


def _trapezoid_weights(r):
    w = np.zeros_like(r)
    d = np.diff(r)
    w[:-1] += d / 2.0
    w[1:] += d / 2.0
    return w


def perturbation_energy(ops, u):
    """J = 1/2 sum_j w_j r_j sum_{m,k} c_m |u'|^2, u' = u - Couette (trapezoid w_j)."""
    base, _, _ = couette_state(ops)
    d = u - base
    dens = 0.5 * (np.abs(d[0]) ** 2 + np.abs(d[1]) ** 2) + np.abs(d[2]) ** 2
    c = np.full(ops.prm.M + 1, 2.0)
    c[0] = 1.0
    per_r = np.einsum("rmk,m->r", dens, c)
    return 0.5 * float(np.sum(_trapezoid_weights(ops.r) * ops.r * per_r))


def torque(ops, u):
    """T = r^3 d_r(U_theta / r) at (r_i, r_o) from the (0,0) mode, wall D1 rows."""
    K = ops.prm.K
    Ut = np.real((u[0, :, 0, K] - u[1, :, 0, K]) / 2j)
    d = ops.D1 @ (Ut / ops.r)
    T = ops.r ** 3 * d
    return float(T[0]), float(T[-1])


def max_divergence(ops, u, interior=True):
    d = np.abs(div_h(ops, u))
    return float(d[1:-1].max() if interior else d.max())


# ----------------------------------------------------------------------------------------
# Tangent-linear and adjoint of one step (differentiation form; not in the paper)
#
# The step maps (u^i, u^{i-1}, N^{i-1}) -> (u^{i+1}, u^i, N^i); p^{i+1} is an output that is
# not fed back.  Everything but N is affine, with the Dirichlet wall values as the only
# constants, so the tangent is the step with N replaced by N'(u) du and zero wall values.
# The adjoint is written with explicit transposes for the Euclidean inner product on the
# stored (Re, Im) pairs: <a, b> = Re sum conj(a) b.
# ----------------------------------------------------------------------------------------

def _bilinear(ops, a_hat, b_hat):
    """B(a, b) = (a . grad) b with the curvature terms, dealiased, so N(u) = B(u, u)."""
    (ar, _, _, _), (at, _, _, _), (az, _, _, _) = physical_fields(ops, a_hat)
    (br, brr, brt, brz), (bt, btr, btt, btz), (bz, bzr, bzt, bzz) = physical_fields(ops, b_hat)
    r = ops.r[:, None, None]
    Nr = ar * brr + (at / r) * brt + az * brz - at * bt / r
    Nt = ar * btr + (at / r) * btt + az * btz + at * br / r
    Nz = ar * bzr + (at / r) * bzt + az * bzz
    Nr_h, Nt_h, Nz_h = (to_spectral(ops, f) for f in (Nr, Nt, Nz))
    return np.stack([Nr_h + 1j * Nt_h, Nr_h - 1j * Nt_h, Nz_h])


def nonlinear_tangent(ops, u, du):
    """N'(u) du = B(du, u) + B(u, du)."""
    return _bilinear(ops, du, u) + _bilinear(ops, u, du)


def _advance_linear(ops, u, u_prev, N, N_prev):
    """Steps 2-5 with zero Dirichlet wall values (the linear part of `advance`)."""
    prm = ops.prm
    mats = ops.mats
    K, dt = prm.K, prm.dt
    NN = 2.0 * N - N_prev
    b = div_h(ops, -NN)
    g = -(NN[0] + NN[1]) / 2.0 + 2.0 * vector_laplacian_r(ops, u) - vector_laplacian_r(ops, u_prev)
    b[0] = g[0]
    b[-1] = g[-1]
    b[-1, 0, K] = 0.0
    p_star = solve_modes(ops, mats["P"], b)
    rhs = (4.0 * u - u_prev) / (2.0 * dt) - NN - grad_h(ops, p_star)
    rhs[:, 0] = 0.0
    rhs[:, -1] = 0.0
    u_star = np.stack([solve_modes(ops, mats[n], rhs[c]) for c, n in enumerate(("Hp", "Hm", "Hz"))])
    b = div_h(ops, u_star)
    b[0] = 0.0
    b[-1] = 0.0
    phi = solve_modes(ops, mats["P"], b)
    return u_star - grad_h(ops, phi)


def tangent_step(ops, st: State, du, du_prev, dN_prev):
    """Tangent of one step of a started state: returns (du^{i+1}, du^i, dN^i)."""
    dN = nonlinear_tangent(ops, st.u, du)
    return _advance_linear(ops, du, du_prev, dN, dN_prev), du, dN


# transposes of the pieces ------------------------------------------------------------

def _dr_T(ops, a):
    return np.tensordot(ops.D1.T, a, axes=(1, 0))


def _div_T(ops, b):
    """Adjoint of div_h (all rows) for (v_+, v_-, v_z)."""
    r = ops.r[:, None, None]
    mm = ops.mm[None, :, None]
    kk = ops.kk[None, None, :]
    t = _dr_T(ops, b) + b / r                       # adjoint of D1 v_r + v_r / r w.r.t. v_r
    vp = 0.5 * t + mm * b / (2.0 * r)
    vm = 0.5 * t - mm * b / (2.0 * r)
    vz = -1j * kk * b
    return np.stack([vp, vm, vz])


def _grad_T(ops, g):
    """Adjoint of grad_h: (g_+, g_-, g_z) -> scalar."""
    r = ops.r[:, None, None]
    mm = ops.mm[None, :, None]
    kk = ops.kk[None, None, :]
    return _dr_T(ops, g[0] + g[1]) - mm * (g[0] - g[1]) / r - 1j * kk * g[2]


def _lap_r_T_rows(ops, w, rows):
    """Adjoint of the wall values ((L_+ u_+) + (L_- u_-))/2 at `rows` (w holds one value per
    row in `rows`): returns (du_+, du_-) fields."""
    prm = ops.prm
    out = np.zeros((2,) + prm.shape(), np.complex128)
    mm = ops.mm[:, None]
    kk2 = (ops.kk ** 2)[None, :]
    for wv, j in zip(w, rows):
        r = ops.r[j]
        for c, sg in ((0, -1.0), (1, 1.0)):
            diag = -mm ** 2 / r ** 2 - kk2 - 1.0 / r ** 2 + sg * 2.0 * mm / r ** 2
            out[c] += 0.5 * (ops.D2[j] + ops.D1[j] / r)[:, None, None] * wv[None]
            out[c, j] += 0.5 * diag * wv
    return out


def _solve_T(ops, A, rhs):
    """x = A^{-T} rhs for every mode (the matrices are real)."""
    return solve_modes(ops, np.swapaxes(A, -1, -2), rhs)


def _to_physical_T(ops, x):
    """Adjoint of to_physical (complex (N_r, M+1, 2K+1) -> real (N_r, P_t, P_z))."""
    g = np.matmul(np.conj(ops.G).T, x)              # (..., M+1, P_z)
    return np.matmul(g, np.conj(ops.EzT).T)          # (..., M+1, 2K+1)


def _to_spectral_T(ops, y):
    """Adjoint of to_spectral: real field Re(Ft^H y FzT^H)."""
    f = np.matmul(y, np.conj(ops.FzT).T)            # (..., M+1, P_z)
    return np.real(np.matmul(np.conj(ops.Ft).T, f))


def nonlinear_adjoint(ops, u, Nbar):
    """(N'(u))^T Nbar."""
    prm = ops.prm
    r = ops.r[:, None, None]
    (ur, urr, urt, urz), (ut, utr, utt, utz), (uz, uzr, uzt, uzz) = physical_fields(ops, u)
    nr = _to_spectral_T(ops, Nbar[0] + Nbar[1])
    nt = _to_spectral_T(ops, -1j * (Nbar[0] - Nbar[1]))
    nz = _to_spectral_T(ops, Nbar[2])
    bar = {
        ("u", 0): nr * urr + nt * (utr + ut / r) + nz * uzr,
        ("u", 1): nr * (urt - 2.0 * ut) / r + nt * (utt + ur) / r + nz * uzt / r,
        ("u", 2): nr * urz + nt * utz + nz * uzz,
        ("r", 0): ur * nr, ("t", 0): ut / r * nr, ("z", 0): uz * nr,
        ("r", 1): ur * nt, ("t", 1): ut / r * nt, ("z", 1): uz * nt,
        ("r", 2): ur * nz, ("t", 2): ut / r * nz, ("z", 2): uz * nz,
    }
    im = 1j * ops.mm[None, :, None]
    ik = 1j * ops.kk[None, None, :]
    comp = []
    for c in range(3):
        a = (_to_physical_T(ops, bar[("u", c)])
             + _dr_T(ops, _to_physical_T(ops, bar[("r", c)]))
             + np.conj(im) * _to_physical_T(ops, bar[("t", c)])
             + np.conj(ik) * _to_physical_T(ops, bar[("z", c)]))
        comp.append(a)
    # (u_r, u_t, u_z) = ((u_+ + u_-)/2, (u_+ - u_-)/(2i), u_z): transpose
    ub = np.empty((3,) + prm.shape(), np.complex128)
    ub[0] = 0.5 * comp[0] + 0.5j * comp[1]
    ub[1] = 0.5 * comp[0] - 0.5j * comp[1]
    ub[2] = comp[2]
    return ub


def adjoint_advance(ops, ubar_new):
    """Adjoint of the linear map (u, u_prev, N, N_prev) -> u^{i+1} of steps 2-5 (zero wall
    values): returns the adjoints (u_b, up_b, N_b, Np_b) of its four inputs."""
    prm = ops.prm
    mats = ops.mats
    K, dt = prm.K, prm.dt
    # u^{i+1} = u* - grad phi
    us_b = ubar_new.copy()
    phi_b = -_grad_T(ops, ubar_new)
    # phi = P^{-1} b, b = div u* on interior rows
    b_b = _solve_T(ops, mats["P"], phi_b)
    b_b[0] = 0.0
    b_b[-1] = 0.0
    us_b += _div_T(ops, b_b)
    # u*_c = H_c^{-1} rhs_c, interior rows of rhs_c = (4u - u_prev)/(2dt) - NN - grad p*
    rhs_b = np.stack([_solve_T(ops, mats[n], us_b[c]) for c, n in enumerate(("Hp", "Hm", "Hz"))])
    rhs_b[:, 0] = 0.0
    rhs_b[:, -1] = 0.0
    u_b = 4.0 / (2.0 * dt) * rhs_b
    up_b = -1.0 / (2.0 * dt) * rhs_b
    NN_b = -rhs_b
    ps_b = -_grad_T(ops, rhs_b)
    # p* = P^{-1} b_p
    bp_b = _solve_T(ops, mats["P"], ps_b)
    wall = bp_b[[0, -1]].copy()
    wall[1, 0, K] = 0.0                                 # (0,0) Dirichlet row at r_o
    inside = bp_b.copy()
    inside[0] = 0.0
    inside[-1] = 0.0
    NN_b += _div_T(ops, -inside)
    # wall rows: -NN_r + 2 Lap_r(u) - Lap_r(u_prev), NN_r = (NN_+ + NN_-)/2
    for i, j in enumerate((0, -1)):
        NN_b[0, j] += -0.5 * wall[i]
        NN_b[1, j] += -0.5 * wall[i]
    L = _lap_r_T_rows(ops, wall, (0, prm.N_r - 1))
    u_b[:2] += 2.0 * L
    up_b[:2] -= L
    # NN = 2N - N_prev
    return u_b, up_b, 2.0 * NN_b, -NN_b


def adjoint_step(ops, st: State, ubar_new, ubar_cur, Nbar_cur):
    """Adjoint of one step of a started state st = (u^i, u^{i-1}, N^{i-1}): given the
    adjoints of (u^{i+1}, u^i, N^i) returns those of (u^i, u^{i-1}, N^{i-1})."""
    u_b, up_b, N_b, Np_b = adjoint_advance(ops, ubar_new)
    u_b = u_b + ubar_cur + nonlinear_adjoint(ops, st.u, N_b + Nbar_cur)
    return u_b, up_b, Np_b


def adjoint_start_up(ops, u0, ubar, upbar, Npbar):
    """Adjoint of the cold-start map u^0 -> (u^0, u^{-1}, N^{-1}) of `start_up`:
    u^{-1} = 2.5 u^0 - 1.5 u_E(u^0), u_E = advance(u^0, u^0, N(u^0), N(u^0)),
    N^{-1} = N(u^{-1})."""
    u_m1 = start_up(ops, u0).u_prev
    m1_b = upbar + nonlinear_adjoint(ops, u_m1, Npbar)
    uE_b = -1.5 * m1_b
    a_u, a_up, a_N, a_Np = adjoint_advance(ops, uE_b)
    return ubar + 2.5 * m1_b + a_u + a_up + nonlinear_adjoint(ops, u0, a_N + a_Np)


def energy_gradient(ops, u):
    """Gradient of perturbation_energy w.r.t. the stored (Re, Im) pairs, as a complex array."""
    base, _, _ = couette_state(ops)
    d = u - base
    w = _trapezoid_weights(ops.r) * ops.r
    c = np.full(ops.prm.M + 1, 2.0)
    c[0] = 1.0
    wc = w[:, None, None] * c[None, :, None]
    return np.stack([0.5 * wc * d[0], 0.5 * wc * d[1], wc * d[2]])


def gradient_final_energy(ops, u0, nsteps):
    """dJ/du^0 of J = perturbation_energy(u^n) after nsteps from the cold state u^0, by the
    adjoint (states of the forward run kept in memory)."""
    states = [start_up(ops, u0)]
    for _ in range(nsteps - 1):
        states.append(step(ops, states[-1]))
    uN = step(ops, states[-1]).u
    ub, upb, Npb = energy_gradient(ops, uN), np.zeros_like(u0), np.zeros_like(u0)
    for st in reversed(states):
        ub, upb, Npb = adjoint_step(ops, st, ub, upb, Npb)
    return adjoint_start_up(ops, u0, ub, upb, Npb), perturbation_energy(ops, uN)


def inner(a, b):
    return float(np.real(np.vdot(a, b)))
