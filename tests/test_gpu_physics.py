"""End-to-end physics check of the CUDA step against a number the paper prints: the wave speed
of wavy Taylor vortices (Sec. 5.2, tests/golden/wavy_vortex_wave_speed.json).

The paper's resolution (n_r, n_theta, n_z) = (32, 32, 32) is (M, 2N+1, 2L+1) in its notation
(Sec. 3.1), i.e. N_r = 32 nodes and modes |m| <= 16 (m_p = k_theta = 6), |k| <= 16 here.  The
run starts from Couette flow with a Taylor-vortex perturbation plus seeded noise, steps until
the m = 1 energy and the measured speed stop changing, and then checks that the state is a
rigid rotation and that its speed matches the paper's to 1e-4 relative.  A relative
equilibrium rotating at angular velocity w has u_m(t + s) = u_m(t) exp(-i m m_p w s), so the
phase drift of the m = 1 coefficients over s gives c = w / Omega_i, Omega_i = Re_i / r_i.
"""
import json
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1311_2481_gb300 import build as B  # noqa: E402
from paper_1311_2481_gb300 import inputs as I  # noqa: E402
from paper_1311_2481_gb300 import tc  # noqa: E402

B.build()
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "wavy_vortex_wave_speed.json")))


def wave_speed_run(precision, max_steps=200_000, chunk=20_000, span=500):
    eta, Re_i, m_p, L_z, dt = GOLD["eta"], GOLD["Re_i"], GOLD["k_theta"], GOLD["Gamma"], GOLD["dt"]
    N_r, M, K = 32, 16, 16
    plan = tc.Plan(N_r, M, K, m_p, eta, Re_i, GOLD["Re_o"], L_z, dt, precision=precision, no_adjoint=True)
    r = plan.nodes()
    Om_i = Re_i / (eta / (1.0 - eta))
    u0 = torch.from_numpy(I.initial_state(r, M, K, m_p, L_z, eta, Re_i, GOLD["Re_o"], kind="taylor",
                                          amp=0.01, seed=7)).cuda()
    st = tc.State(plan, u0)

    def speed():
        a = st.u[:, :, 1, :].clone()
        plan.step(st, span)
        b = st.u[:, :, 1, :].clone()
        z = torch.sum(torch.conj(a) * b).item()
        c = -math.atan2(z.imag, z.real) / (m_p * span * dt * Om_i)
        return c, a, b

    steps, prev = 0, None
    while steps < max_steps:
        plan.step(st, chunk)
        c, _, b = speed()
        steps += chunk + span
        e1 = float((b.abs() ** 2).sum())
        if prev is not None and abs(e1 / prev[0] - 1) < 1e-6 and abs(c - prev[1]) < 1e-7:
            break
        prev = (e1, c)
    c, a, b = speed()
    rot = a * complex(math.cos(-m_p * Om_i * c * span * dt), math.sin(-m_p * Om_i * c * span * dt))
    residual = float(torch.linalg.vector_norm(b - rot) / torch.linalg.vector_norm(b))
    e_ratio = float((b.abs() ** 2).sum() / (st.u[:, :, 0, :].abs() ** 2).sum())
    # tangential slip at the inner wall (Sec. 5.3): the correction u = u* - grad phi leaves
    # (u_theta - Re_i, u_z) != 0 there; RMS over the wall, relative to Re_i, by Parseval on the
    # stored coefficients (mean of f^2 = sum_k |f_0k|^2 + 2 sum_{m>0,k} |f_mk|^2)
    w = st.u[:, 0].cpu().numpy()                   # [c][m][k] at r = r_i
    ut = (w[0] - w[1]) / 2j
    ut[0, K] -= Re_i
    cm = np.full((M + 1, 1), 2.0)
    cm[0] = 1.0
    slip = float(np.sqrt(np.sum(cm * (np.abs(ut) ** 2 + np.abs(w[2]) ** 2))) / Re_i)
    return c, residual, e_ratio, steps, slip


def test_wavy_vortex_wave_speed_fp64():
    c, residual, e_ratio, steps, slip = wave_speed_run(tc.TC_FP64)
    print(f"c = {c:.7f} after {steps} steps, rigid-rotation residual {residual:.2e}, relative slip {slip:.2e}")
    assert e_ratio > 1e-3, "no saturated wavy mode"
    assert residual <= 1e-6, residual
    assert abs(c / GOLD["c"] - 1) <= 1e-4, (c, steps)
    # roughly 1e-6 at this resolution and time step (Sec. 5.3): within a decade either way
    assert GOLD["relative_slip_about"] / 10 <= slip <= GOLD["relative_slip_about"] * 10, slip


def test_wavy_vortex_wave_speed_mixed():
    """The mixed form over the same long run.  Without projecting N's m = 0 line onto the
    real-field symmetry, its FP32 rounding seeded a non-real m = 0 part of u that the FP64
    mean-flow terms amplified until the run overflowed (after about one viscous time)."""
    c, residual, e_ratio, steps, slip = wave_speed_run(tc.TC_MIXED)
    print(f"mixed: c = {c:.7f} after {steps} steps, rigid-rotation residual {residual:.2e}, relative slip {slip:.2e}")
    assert e_ratio > 1e-3, "no saturated wavy mode"
    assert residual <= 1e-5, residual
    assert abs(c / GOLD["c"] - 1) <= 1e-4, (c, steps)


ONSET = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "wavy_vortex_onset.json")))


def n1_growth_rate(Re, u_tvf=None, Re_prev=None):
    """Growth rate of an n = 1 disturbance on saturated Taylor vortices.  In the linear regime
    only the axisymmetric base (m = 0) and the disturbance (m = 1) interact, so M = 1 gives the
    paper's azimuthal resolution's answer; N_r = 64 and |k| <= 64 are its radial and axial
    resolution ((n_r, n_z) = (64, 128) = (M, 2L+1) in its notation)."""
    eta, L_z, dt = ONSET["eta"], ONSET["Gamma"], ONSET["dt"]
    N_r, M, K = 64, 1, 64
    plan = tc.Plan(N_r, M, K, ONSET["k_theta"], eta, Re, ONSET["Re_o"], L_z, dt, no_adjoint=True)
    r = plan.nodes()
    base = torch.from_numpy(I.base_state(r, M, K, eta, Re, 0.0)).cuda()
    if u_tvf is None:
        u0 = torch.from_numpy(I.initial_state(r, M, K, 1, L_z, eta, Re, 0.0, kind="taylor", amp=0.02, seed=3)).cuda()
        u0[:, :, 1, :] = 0
    else:   # the previous Reynolds number's vortices on this Reynolds number's Couette flow
        u0 = u_tvf - torch.from_numpy(I.base_state(r, M, K, eta, Re_prev, 0.0)).cuda() + base
    st = tc.State(plan, u0)
    prev = None
    for _ in range(60):
        plan.step(st, 5000)
        e0 = float((st.u[:, :, 0, :].abs() ** 2).sum())
        if prev is not None and abs(e0 / prev - 1) < 1e-12:
            break
        prev = e0
    u_tvf = st.u.clone()
    pert = torch.from_numpy(I.initial_state(r, M, K, 1, L_z, eta, Re, 0.0, kind="box", amp=1e-7, seed=5)).cuda() - base
    u1 = u_tvf.clone()
    u1[:, :, 1, :] = pert[:, :, 1, :]
    st = tc.State(plan, u1)
    span, logs, rates = 5000, [], []
    for _ in range(60):
        plan.step(st, span)
        logs.append(math.log(float((st.u[:, :, 1, :].abs() ** 2).sum())))
        if len(logs) >= 2:
            rates.append((logs[-1] - logs[-2]) / (2 * span * dt))   # energy ~ exp(2 sigma t)
        if len(rates) >= 3 and abs(rates[-1] - rates[-3]) < 1e-7:
            break
    return rates[-1], u_tvf


def test_wavy_vortex_onset():
    lo, hi = 407.6, 408.6
    s_lo, u_tvf = n1_growth_rate(lo)
    s_hi, _ = n1_growth_rate(hi, u_tvf, lo)
    Re_c = lo - s_lo * (hi - lo) / (s_hi - s_lo)
    print(f"sigma({lo}) = {s_lo:.6e}, sigma({hi}) = {s_hi:.6e}, Re_c = {Re_c:.4f}")
    assert s_lo < 0 < s_hi
    a, b = ONSET["Re_c_bracket"]
    assert a - 0.05 <= Re_c <= b + 0.05, Re_c
