"""Pins of the oracle's tangent-linear and adjoint step (differentiation form).

The step is quadratic in the state (through N) and affine otherwise, so central finite
differences of the oracle's own nonlinear step are exact up to rounding: they pin the
tangent.  The adjoint is pinned to the tangent by dot-product tests, and the full gradient
of the final perturbation energy (start-up included) is pinned by central differences.
"""
import math

import numpy as np

import oracle as O
from paper_1311_2481_gb300 import inputs as I

CFG = dict(N_r=16, M=4, K=6, m_p=1, eta=0.5, Re_i=50.0, Re_o=0.0, L_z=2 * math.pi / 3.16, dt=1e-3)


def _setup():
    prm = O.Params(**CFG)
    ops = O.Operators(prm)
    u0 = I.initial_state(ops.r, prm.M, prm.K, prm.m_p, prm.L_z, prm.eta, prm.Re_i, prm.Re_o,
                         kind="box", amp=1e-2)
    return prm, ops, u0


def _rnd(rng, shape, K):
    return I.random_spectral(shape, seed=int(rng.integers(1 << 30)), hermitian_K=None)


def test_tangent_matches_central_differences():
    prm, ops, u0 = _setup()
    st = O.step(ops, O.cold_state(u0))
    rng = np.random.default_rng(1)
    sh = (3,) + prm.shape()
    d = [_rnd(rng, sh, prm.K) for _ in range(3)]
    h = 1e-4
    sp = O.State(st.u + h * d[0], st.u_prev + h * d[1], st.N_prev + h * d[2], st.p, True)
    sm = O.State(st.u - h * d[0], st.u_prev - h * d[1], st.N_prev - h * d[2], st.p, True)
    a, b = O.step(ops, sp), O.step(ops, sm)
    fd = [(a.u - b.u) / (2 * h), (a.u_prev - b.u_prev) / (2 * h), (a.N_prev - b.N_prev) / (2 * h)]
    tl = O.tangent_step(ops, st, *d)
    for x, y in zip(fd, tl):
        assert np.linalg.norm(x - y) <= 1e-8 * np.linalg.norm(y)


def test_adjoint_dot_product_tests():
    prm, ops, u0 = _setup()
    st = O.step(ops, O.cold_state(u0))
    rng = np.random.default_rng(2)
    sh = (3,) + prm.shape()
    x = [_rnd(rng, sh, prm.K) for _ in range(3)]
    y = [_rnd(rng, sh, prm.K) for _ in range(3)]
    tl = O.tangent_step(ops, st, *x)
    ad = O.adjoint_step(ops, st, *y)
    lhs = sum(O.inner(a, b) for a, b in zip(y, tl))
    rhs = sum(O.inner(a, b) for a, b in zip(ad, x))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    a, b = x[0], y[0]
    lhs = O.inner(b, O.nonlinear_tangent(ops, st.u, a))
    rhs = O.inner(O.nonlinear_adjoint(ops, st.u, b), a)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_energy_gradient_matches_central_differences():
    prm, ops, u0 = _setup()
    n = 6
    g, J = O.gradient_final_energy(ops, u0, n)
    rng = np.random.default_rng(3)
    h = 1e-7
    for _ in range(4):
        d = I.random_spectral((3,) + prm.shape(), seed=int(rng.integers(1 << 30)), hermitian_K=prm.K)
        d[:, 0] = 0.0
        d[:, -1] = 0.0
        Jp = O.perturbation_energy(ops, O.run(ops, O.cold_state(u0 + h * d), n).u)
        Jm = O.perturbation_energy(ops, O.run(ops, O.cold_state(u0 - h * d), n).u)
        fd = (Jp - Jm) / (2 * h)
        ad = O.inner(g, d)
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-30), (fd, ad)
