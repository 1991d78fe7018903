"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU).

Each test compares the oracle with something other than itself: closed forms, textbook
finite-difference weights, library FFTs (numpy.fft), brute-force convolution, banded
library solves, manufactured solutions, and the Taylor-vortex onset point.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1311_2481_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _prm(**kw):
    base = dict(N_r=32, M=8, K=16, m_p=1, eta=0.5, Re_i=50.0, Re_o=0.0,
                L_z=2 * math.pi / 3.16, dt=1e-3)
    base.update(kw)
    return O.Params(**base)


# ---------------------------------------------------------------- P1 nodes (Eq. nodeDist)

def test_nodes_endpoints_and_symmetry():
    for eta in (0.5, 0.868, 0.71):
        r, _ = O.radial_nodes(33, eta, 0.5)
        r_i, r_o = eta / (1 - eta), 1 / (1 - eta)
        assert abs(r[0] - r_i) <= 2e-16 * r_o and abs(r[-1] - r_o) <= 2e-16 * r_o
        assert np.all(np.diff(r) > 0)
        np.testing.assert_allclose(r + r[::-1], r_i + r_o, rtol=0, atol=4e-15 * r_o)


def test_nodes_uniform_and_chebyshev_limits():
    N = 17
    r, _ = O.radial_nodes(N, 0.5, 1.0)
    np.testing.assert_allclose(r, 1.0 + np.arange(N) / (N - 1), atol=1e-15)
    r0, _ = O.radial_nodes(N, 0.5, 0.0)
    cheb = 1.5 - np.cos(np.pi * np.arange(N) / (N - 1)) / 2
    np.testing.assert_allclose(r0, cheb, atol=1e-15)
    r_small, _ = O.radial_nodes(N, 0.5, 1e-6)      # alpha -> 0 approaches Chebyshev
    np.testing.assert_allclose(r_small, cheb, atol=1e-12)


# ---------------------------------------------------------------- P2 finite differences

def _frac(v):
    return float(Fraction(v))


def test_fd_weights_match_textbook_on_uniform_grid():
    g = _gold("fd_central_weights.json")
    xs = list(range(-4, 5))
    for n, w in g["central_d1"].items():
        h = int(n) // 2
        got = [float(x) for x in O.fd_weights(0, xs[4 - h:5 + h], 1)]
        np.testing.assert_allclose(got, [_frac(v) for v in w], atol=1e-15)
    for n, w in g["central_d2"].items():
        h = int(n) // 2
        got = [float(x) for x in O.fd_weights(0, xs[4 - h:5 + h], 2)]
        np.testing.assert_allclose(got, [_frac(v) for v in w], atol=1e-14)
    got1 = [float(x) for x in O.fd_weights(0, range(5), 1)]
    got2 = [float(x) for x in O.fd_weights(0, range(5), 2)]
    np.testing.assert_allclose(got1, [_frac(v) for v in g["forward_d1_5"]], atol=1e-14)
    np.testing.assert_allclose(got2, [_frac(v) for v in g["forward_d2_5"]], atol=1e-13)


def test_derivative_matrices_exact_on_polynomials_and_banded():
    prm = _prm(N_r=24)
    ops = O.Operators(prm)
    r = ops.r
    rng = np.random.default_rng(3)
    N = prm.N_r
    half = prm.fd_order // 2
    for j in range(N):
        n = len(O.stencil_nodes(j, N, half))
        c = rng.standard_normal(n)
        x = r - 1.5
        p = sum(c[q] * x ** q for q in range(n))
        dp = sum(q * c[q] * x ** (q - 1) for q in range(1, n))
        d2p = sum(q * (q - 1) * c[q] * x ** (q - 2) for q in range(2, n))
        assert abs(ops.D1[j] @ p - dp[j]) <= 1e-9 * (1 + abs(dp[j]))
        if n >= 3:
            assert abs(ops.D2[j] @ p - d2p[j]) <= 1e-7 * (1 + abs(d2p[j]))
    for D in (ops.D1, ops.D2):
        jj, ii = np.nonzero(D)
        assert np.max(np.abs(ii - jj)) <= half


def test_fd_convergence_order_interior():
    errs = []
    for N in (32, 64):
        ops = O.Operators(_prm(N_r=N, alpha=1.0))
        f = np.sin(3 * ops.r)
        e = np.abs(ops.D1 @ f - 3 * np.cos(3 * ops.r))[4:-4].max()
        errs.append(e)
    slope = math.log(errs[0] / errs[1]) / math.log(2)
    assert slope > 7.5, slope


# ---------------------------------------------------------------- P3 transforms

def _phys_numpy(a, Pt, Pz, K):
    """Reference synthesis with numpy.fft: u = Re(sum_m c_m sum_k a e^{i(..)})."""
    S = np.zeros(a.shape[:-2] + (Pt, Pz), np.complex128)
    M = a.shape[-2] - 1
    c = np.full(M + 1, 2.0)
    c[0] = 1.0
    for kk in range(2 * K + 1):
        S[..., :M + 1, (kk - K) % Pz] = a[..., :, kk] * c
    return np.real(np.fft.ifft2(S) * Pt * Pz)


def _spec_numpy(u, M, K):
    F = np.fft.fft2(u) / (u.shape[-2] * u.shape[-1])
    Pz = u.shape[-1]
    return np.stack([F[..., :M + 1, (k) % Pz] for k in range(-K, K + 1)], axis=-1)


def test_transforms_match_numpy_fft():
    for (M, K, Pt, Pz) in ((8, 16, 24, 48), (5, 7, 16, 22), (4, 4, 13, 13)):
        prm = _prm(N_r=8, M=M, K=K, P_theta=Pt, P_z=Pz)
        ops = O.Operators(prm)
        a = I.random_spectral((3, 8, M + 1, 2 * K + 1), seed=1)
        u = O.to_physical(ops, a)
        ref = _phys_numpy(a, Pt, Pz, K)
        np.testing.assert_allclose(u, ref, atol=1e-12 * np.abs(ref).max())
        v = np.random.default_rng(2).standard_normal((3, 8, Pt, Pz))
        np.testing.assert_allclose(O.to_spectral(ops, v), _spec_numpy(v, M, K), atol=1e-14)


def test_roundtrip_and_parseval():
    prm = _prm(N_r=6)
    ops = O.Operators(prm)
    a = I.random_spectral((6, prm.M + 1, 2 * prm.K + 1), seed=5, hermitian_K=prm.K)
    u = O.to_physical(ops, a)
    np.testing.assert_allclose(O.to_spectral(ops, u), a, atol=1e-13)
    c = np.full(prm.M + 1, 2.0)
    c[0] = 1.0
    lhs = (u ** 2).mean(axis=(1, 2))
    rhs = np.einsum("rmk,m->r", np.abs(a) ** 2, c)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13)


# ---------------------------------------------------------------- P4 dealiasing

def _full_spectrum(a, K):
    """Map stored (m >= 0) coefficients of a real field onto a dict over all (m, k)."""
    M = a.shape[0] - 1
    d = {}
    for m in range(-M, M + 1):
        for k in range(-K, K + 1):
            if m > 0:
                v = a[m, k + K]
            elif m < 0:
                v = np.conj(a[-m, -k + K])
            else:
                v = a[0, k + K].real if k == 0 else (a[0, k + K] if k > 0 else np.conj(a[0, -k + K]))
            d[(m, k)] = v
    return d


def test_dealiased_product_equals_truncated_convolution():
    M, K = 3, 3
    a = I.random_spectral((M + 1, 2 * K + 1), seed=11, hermitian_K=K)
    b = I.random_spectral((M + 1, 2 * K + 1), seed=12, hermitian_K=K)
    A, B = _full_spectrum(a, K), _full_spectrum(b, K)
    exact = np.zeros((M + 1, 2 * K + 1), np.complex128)
    for (m1, k1), va in A.items():
        for (m2, k2), vb in B.items():
            m, k = m1 + m2, k1 + k2
            if 0 <= m <= M and abs(k) <= K:
                exact[m, k + K] += va * vb
    # 3/2 rule with P >= 3M + 1: exact
    ops = O.Operators(_prm(N_r=6, M=M, K=K, P_theta=3 * M + 1, P_z=3 * K + 1))
    got = O.to_spectral(ops, O.to_physical(ops, a[None]) * O.to_physical(ops, b[None]))[0]
    np.testing.assert_allclose(got, exact, atol=1e-13)
    # P = 3M, 3K (default grid): only the edge modes |m| = M or |k| = K may differ
    ops = O.Operators(_prm(N_r=6, M=M, K=K))
    got = O.to_spectral(ops, O.to_physical(ops, a[None]) * O.to_physical(ops, b[None]))[0]
    inner = got[:M, 1:-1] - exact[:M, 1:-1]
    assert np.abs(inner).max() < 1e-13
    assert np.abs(got - exact).max() > 1e-6     # the edge modes do alias on 3M x 3K


# ---------------------------------------------------------------- P5 nonlinear term

@pytest.mark.parametrize("m_p", [1, 6])
def test_nonlinear_manufactured_against_analytic_derivatives(m_p):
    prm = _prm(N_r=16, M=8, K=8, m_p=m_p)
    ops = O.Operators(prm)
    r = ops.r
    M, K = prm.M, prm.K
    rng = np.random.default_rng(21)
    amps, q, dq = [], [], []
    for c in range(3):
        A = I.random_spectral((M + 1, 2 * K + 1), seed=30 + c, hermitian_K=K)
        mm = np.arange(M + 1)[:, None]
        kk = np.arange(-K, K + 1)[None, :]
        A = A * ((mm <= M // 2) & (np.abs(kk) <= K // 2))
        c0, c1, c2 = rng.standard_normal(3)
        amps.append(A)
        q.append(c0 + c1 * (r - 1.5) + c2 * (r - 1.5) ** 2)
        dq.append(c1 + 2 * c2 * (r - 1.5))
    urtz = [q[c][:, None, None] * amps[c][None] for c in range(3)]
    u_hat = np.stack([urtz[0] + 1j * urtz[1], urtz[0] - 1j * urtz[1], urtz[2]])
    Pt, Pz = prm.P_theta, prm.P_z
    im = 1j * prm.m_p * np.arange(M + 1)[None, :, None]
    ik = 1j * prm.k_z * np.arange(-K, K + 1)[None, None, :]
    f = []
    for c in range(3):
        a = urtz[c]
        f.append((_phys_numpy(a, Pt, Pz, K),
                  _phys_numpy(dq[c][:, None, None] * amps[c][None], Pt, Pz, K),
                  _phys_numpy(im * a, Pt, Pz, K), _phys_numpy(ik * a, Pt, Pz, K)))
    (ur, urr, urt, urz), (ut, utr, utt, utz), (uz, uzr, uzt, uzz) = f
    R = r[:, None, None]
    # Eq. NS_cyl, left-hand sides: (u . grad) u_r - u_t^2 / r, (u . grad) u_t + u_t u_r / r
    Nr = ur * urr + ut / R * urt + uz * urz - ut ** 2 / R
    Nt = ur * utr + ut / R * utt + uz * utz + ut * ur / R
    Nz = ur * uzr + ut / R * uzt + uz * uzz
    Nr_h, Nt_h, Nz_h = (_spec_numpy(x, M, K) for x in (Nr, Nt, Nz))
    ref = np.stack([Nr_h + 1j * Nt_h, Nr_h - 1j * Nt_h, Nz_h])
    got = O.nonlinear(ops, u_hat)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    # the row-restricted evaluation (wall rows, a stencil-edge row, an interior row)
    rows = [0, 3, 7, prm.N_r - 1]
    got_rows = O.nonlinear(ops, u_hat, rows=rows)
    assert got_rows.shape == (3, len(rows), M + 1, 2 * K + 1)
    assert np.linalg.norm(got_rows - ref[:, rows]) <= 1e-12 * np.linalg.norm(ref[:, rows])
    assert np.linalg.norm(got_rows - got[:, rows]) <= 1e-14 * np.linalg.norm(got[:, rows])


def test_nonlinear_closed_forms():
    """Couette flow: N = (-U^2/r, 0, 0); spiral vortex u = (a/r, b/r, 0) is irrotational,
    so u . grad u = grad(|u|^2 / 2) = (-(a^2 + b^2)/r^3, 0, 0)."""
    prm = _prm(N_r=64, M=4, K=4, Re_i=50.0, Re_o=200.0)
    ops = O.Operators(prm)
    K, r = prm.K, ops.r
    u, _, (C1, C2) = O.couette_state(ops)
    N = O.nonlinear(ops, u)
    U = C1 * r + C2 / r
    expect = -U ** 2 / r
    np.testing.assert_allclose(N[0, :, 0, K].real, expect, rtol=1e-12)
    np.testing.assert_allclose(N[1, :, 0, K].real, expect, rtol=1e-12)
    N0 = N.copy()
    N0[:2, :, 0, K] -= expect
    assert np.abs(N0).max() < 1e-10 * np.abs(expect).max()
    a, b = 0.7, 1.3
    v = np.zeros_like(u)
    v[0, :, 0, K] = a / r + 1j * b / r
    v[1, :, 0, K] = a / r - 1j * b / r
    N = O.nonlinear(ops, v)
    ex = -(a * a + b * b) / r ** 3
    np.testing.assert_allclose(N[0, :, 0, K].real, ex, rtol=2e-6)   # FD error of row 1
    assert np.abs(N[0, :, 0, K].imag).max() < 1e-5   # N_theta = 0 needs +u_t u_r / r


# ---------------------------------------------------------------- P6, P9 Couette

def _couette_run(N_r, alpha=0.5, steps=100):
    g = _gold("couette_laminar.json")
    prm = _prm(N_r=N_r, M=2, K=2, Re_i=g["Re_i"], Re_o=g["Re_o"], eta=g["eta"], alpha=alpha)
    ops = O.Operators(prm)
    ub, pb, (C1, C2) = O.couette_state(ops)
    np.testing.assert_allclose([C1, C2], [g["C1"], g["C2"]], rtol=1e-14)
    st = O.run(ops, O.cold_state(ub), steps)
    U = np.imag(ub[0, :, 0, prm.K])
    Uh = np.imag(st.u[0, :, 0, prm.K])
    w = np.zeros_like(ops.r)
    w[:-1] += np.diff(ops.r) / 2
    w[1:] += np.diff(ops.r) / 2
    Eu = float(np.sum(w * ops.r * np.abs((Uh - U) / U)))
    p_err = np.abs(st.p[:, 0, prm.K].real - pb[:, 0, prm.K].real).max() / np.abs(pb[:, 0, prm.K]).max()
    return ops, st, Eu, p_err, C2


def test_couette_steady_state_pressure_and_torque():
    ops, st, Eu, p_err, C2 = _couette_run(32)
    assert Eu < 2e-6 and p_err < 3e-6
    mask = np.ones(st.u.shape, bool)
    mask[:2, :, 0, ops.prm.K] = False
    assert np.abs(st.u[mask]).max() < 1e-12 * 200    # no other mode is excited (roundoff)
    Ti, To = O.torque(ops, st.u)
    assert abs(Ti / (-2 * C2) - 1) < 1e-4 and abs(To / (-2 * C2) - 1) < 1e-4
    ops64, st64, Eu64, p64, _ = _couette_run(64)
    Ti, To = O.torque(ops64, st64.u)
    assert abs(Ti - To) / abs(2 * C2) < 1e-5
    slope = math.log(Eu / Eu64) / math.log(2)
    assert slope > 7.0, slope                        # 9-point stencils: order ~8
    assert p64 < 5e-8


# ---------------------------------------------------------------- P7 solves

def _solve_one_mode(ops, name, m, k, f):
    """The oracle's solve of system `name` for the single mode (m, k), through solve_modes
    (a right-hand side that is zero on every other mode)."""
    prm = ops.prm
    rhs = np.zeros(prm.shape(), np.complex128)
    rhs[:, m, k + prm.K] = f
    x = O.solve_modes(ops, ops.mats[name], rhs)
    others = np.ones(prm.shape(), bool)
    others[:, m, k + prm.K] = False
    assert not np.any(x[others])
    return x[:, m, k + prm.K]


@pytest.mark.parametrize("m_p", [1, 6])
def test_helmholtz_and_poisson_manufactured(m_p):
    """Each of the four matrices of Sec. 3.2 against its own analytic operator
    (Eq. modalNSdecoup: L_pm = Lap_h - 1/r^2 -+ 2 m m_p / r^2, L_z = Lap_h with
    Lap_h = d_rr + d_r / r - (m m_p)^2 / r^2 - (k k_z)^2), on a mode with m > 0, for k = +2
    and k = -2, with FD-order convergence in N_r."""
    m = 3
    errs = {}
    for N in (32, 64):
        prm = _prm(N_r=N, M=4, K=4, dt=1e-3, m_p=m_p)
        ops = O.Operators(prm)
        r = ops.r
        x = r - prm.r_i
        mmp = m * prm.m_p
        for k in (2, -2):
            kkz = k * prm.k_z
            # Helmholtz: u = sin(pi x) e^r (complex amplitude), Dirichlet zero at both walls
            u = np.sin(np.pi * x) * np.exp(r) * (1.0 + 0.5j)
            du = (np.pi * np.cos(np.pi * x) + np.sin(np.pi * x)) * np.exp(r) * (1.0 + 0.5j)
            d2u = (2 * np.pi * np.cos(np.pi * x) + (1 - np.pi ** 2) * np.sin(np.pi * x)) * np.exp(r) * (1.0 + 0.5j)
            lap = d2u + du / r - mmp ** 2 * u / r ** 2 - kkz ** 2 * u
            ops_c = {"Hp": lap - u / r ** 2 - 2 * mmp * u / r ** 2,
                     "Hm": lap - u / r ** 2 + 2 * mmp * u / r ** 2,
                     "Hz": lap}
            for name, Lu in ops_c.items():
                f = 1.5 / prm.dt * u - Lu
                f[0] = f[-1] = 0.0
                sol = _solve_one_mode(ops, name, m, k, f)
                errs.setdefault((name, k), []).append(np.abs(sol - u).max() / np.abs(u).max())
            # Poisson with Neumann rows: phi = cos(pi x) (zero slope at both walls)
            phi = np.cos(np.pi * x) * (0.5 - 1.0j)
            lap = (-np.pi ** 2 * np.cos(np.pi * x) - np.pi * np.sin(np.pi * x) / r) * (0.5 - 1.0j) \
                - mmp ** 2 * phi / r ** 2 - kkz ** 2 * phi
            f = lap.copy()
            f[0] = f[-1] = 0.0
            sol = _solve_one_mode(ops, "P", m, k, f)
            errs.setdefault(("P", k), []).append(np.abs(sol - phi).max())
        # (0,0): Neumann at r_i, Dirichlet at r_o: phi = cos(pi x) + 1
        phi = np.cos(np.pi * x) + 1.0
        f = -np.pi ** 2 * np.cos(np.pi * x) - np.pi * np.sin(np.pi * x) / r
        f[0] = 0.0
        f[-1] = 0.0
        sol = _solve_one_mode(ops, "P", 0, 0, f)
        errs.setdefault(("P00", 0), []).append(np.abs(sol - phi).max())
    for key, e in errs.items():
        assert e[1] < 1e-7, (key, e)
        assert math.log(e[0] / e[1], 2) > 5.0, (key, e)


def test_gauss_banded_against_library_dense_solve():
    """The oracle's banded elimination against LAPACK's dense LU (numpy.linalg.solve) on
    random matrices with kl = ku = 4, half of them with a zero diagonal so that every column
    needs a row interchange, and with a band that reaches the last row."""
    rng = np.random.default_rng(8)
    for N in (5, 9, 20, 33):
        A = np.zeros((6, N, N))
        for b in range(6):
            for i in range(N):
                lo, hi = max(0, i - 4), min(N, i + 5)
                A[b, i, lo:hi] = rng.standard_normal(hi - lo)
            if b % 2 == 0:
                A[b][np.arange(N), np.arange(N)] = 0.0
        B = rng.standard_normal((6, N, 3))
        x = O.gauss_banded(A, B)
        ref = np.linalg.solve(A, B)
        for b in range(6):
            cond = np.linalg.cond(A[b])
            assert np.abs(x[b] - ref[b]).max() <= 1e-14 * cond * np.abs(ref[b]).max(), (N, b)
    A = np.eye(9)
    A[0, 5] = 1.0
    with pytest.raises(ValueError):
        O.gauss_banded(A, np.ones((9, 1)))


def test_mode_matrices_are_banded_and_match_library_banded_solve():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    prm = _prm(N_r=20, M=3, K=3)
    ops = O.Operators(prm)
    rng = np.random.default_rng(4)
    for name in ("P", "Hp", "Hm", "Hz"):
        for (m, k) in ((0, 0), (2, 1), (3, 3)):
            A = ops.mats[name][m, k]
            jj, ii = np.nonzero(A)
            assert np.abs(ii - jj).max() <= 4
            ab = np.zeros((9, prm.N_r))
            for j in range(prm.N_r):
                for i in range(max(0, j - 4), min(prm.N_r, j + 5)):
                    ab[4 + j - i, i] = A[j, i]
            b = rng.standard_normal(prm.N_r)
            x = scipy_linalg.solve_banded((4, 4), ab, b)
            rhs = np.zeros((prm.N_r, prm.M + 1, 2 * prm.K + 1), np.complex128)
            rhs[:, m, k + prm.K] = b
            got = O.solve_modes(ops, ops.mats[name], rhs)[:, m, k + prm.K]
            np.testing.assert_allclose(got.real, x, rtol=1e-10, atol=1e-12 * np.abs(x).max())
            # the single-mode form builds the same matrix
            assert np.array_equal(O.mode_matrices(ops, m, k)[name][0, 0], A)


# ---------------------------------------------------------------- P8 divergence

@pytest.mark.parametrize("m_p", [1, 6])
def test_projection_reduces_divergence_and_converges(m_p):
    vals = {}
    for N in (48, 96):
        prm = _prm(N_r=N, M=4, K=4, m_p=m_p)
        ops = O.Operators(prm)
        u0 = I.initial_state(ops.r, prm.M, prm.K, prm.m_p, prm.L_z, prm.eta, prm.Re_i,
                             prm.Re_o, kind="box", amp=1e-3)
        st = O.step(ops, O.cold_state(u0))
        st, parts = O.step(ops, st, return_parts=True)
        vals[N] = (O.max_divergence(ops, parts["u_star"]), O.max_divergence(ops, st.u))
    assert vals[96][1] < 0.05 * vals[96][0]
    assert vals[48][1] / vals[96][1] > 8.0, vals


@pytest.mark.parametrize("m_p", [1, 6])
def test_divergence_of_analytic_solenoidal_field(m_p):
    """The seeded perturbation is the curl of an analytic vector potential (its curl is
    written out per mode, independently of the oracle), so its divergence vanishes; the
    oracle's div_h of it is FD truncation error only.  On the rows with the full 9-point
    stencil (4 <= j <= N_r - 5) that error falls at the stencil order (2^8 per halving)."""
    errs = []
    for N in (48, 96):
        prm = _prm(N_r=N, M=4, K=4, m_p=m_p)
        ops = O.Operators(prm)
        base = I.base_state(ops.r, prm.M, prm.K, prm.eta, prm.Re_i, prm.Re_o)
        u0 = I.initial_state(ops.r, prm.M, prm.K, prm.m_p, prm.L_z, prm.eta, prm.Re_i,
                             prm.Re_o, kind="box", amp=1e-1)
        scale = np.abs(ops.mm[None, :, None] * (u0 - base)[0]).max() / prm.r_i
        d = np.abs(O.div_h(ops, u0))[4:N - 4]
        errs.append(d.max() / scale)
    assert errs[1] < 1e-12, errs
    assert errs[0] / errs[1] > 100.0, errs


# ---------------------------------------------------------------- P10 onset

def _k1_growth(Re):
    prm = _prm(N_r=24, M=2, K=3, Re_i=Re, dt=2e-3)
    ops = O.Operators(prm)
    K = prm.K
    u = I.base_state(ops.r, prm.M, K, prm.eta, prm.Re_i, prm.Re_o)
    c = np.zeros((3, prm.M + 1, 2 * K + 1), complex)
    c[1, 0, K + 1] = c[1, 0, K - 1] = 0.5
    up = I.curl_perturbation(ops.r, prm.M, K, prm.m_p, prm.k_z, prm.eta, c)
    st = O.cold_state(u + up * (1e-6 * Re / I.rms_amplitude(up, K)))
    t, e = [], []
    for i in range(800):
        st = O.step(ops, st)
        if (i + 1) % 50 == 0:
            t.append((i + 1) * prm.dt)
            e.append(np.log(np.sum(np.abs(st.u[:, :, 0, K + 1]) ** 2)))
    h = len(t) // 2
    return np.polyfit(t[h:], e[h:], 1)[0]


def test_taylor_vortex_onset_bracket():
    g = _gold("taylor_vortex_onset.json")
    lo, hi = g["bracket"]
    assert abs(3.16 - g["k_z"]) < 1e-12
    assert _k1_growth(lo) < -0.5
    assert _k1_growth(hi) > 0.5
    assert abs(_k1_growth(g["Re_c"])) < 0.2


# ---------------------------------------------------------------- P11 time order

def test_ab2bd2_second_order_in_time():
    res = {}
    T = 0.04
    for dt in (2e-3, 1e-3, 5e-4):
        prm = _prm(N_r=48, M=4, K=4, dt=dt)
        ops = O.Operators(prm)
        u0 = I.initial_state(ops.r, prm.M, prm.K, prm.m_p, prm.L_z, prm.eta, prm.Re_i,
                             prm.Re_o, kind="box", amp=1e-2, mbox=2, kbox=2)
        res[dt] = O.run(ops, O.cold_state(u0), int(round(T / dt))).u
    e1 = np.linalg.norm(res[2e-3] - res[1e-3])
    e2 = np.linalg.norm(res[1e-3] - res[5e-4])
    assert 3.4 < e1 / e2 < 4.8, e1 / e2
