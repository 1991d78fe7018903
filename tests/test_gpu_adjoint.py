"""Adjoint of the CUDA step (through the C ABI) against the oracle's adjoint; dot-product
tests to 1e-12 against the CUDA step's own tangent (exact central differences of the
quadratic step) and against the oracle's tangent-linear step; the gradient of the final
perturbation energy against central finite differences (h = 1e-7, 8 directions, <= 1e-6)
at the 20-step parity size and at the adjoint workload (N_r = 96, 200 steps, checkpoint
every 20), and against the oracle."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_1311_2481_gb300 import adjoint as A  # noqa: E402
from paper_1311_2481_gb300 import build as B  # noqa: E402
from paper_1311_2481_gb300 import inputs as I  # noqa: E402
from paper_1311_2481_gb300 import tc  # noqa: E402

B.build()
LZ = 2 * math.pi / 3.16
CFG1 = dict(N_r=32, M=8, K=16, m_p=1, eta=0.5, Re_i=50.0, Re_o=0.0, L_z=LZ, dt=1e-3)
SMALL = dict(N_r=12, M=3, K=4, m_p=1, eta=0.5, Re_i=50.0, Re_o=0.0, L_z=LZ, dt=1e-3)
# adjoint workload: N_r = 96, m = -32..32, k = -64..64, Re_i = 2000, at the stated dt 5e-4
# halved until 200 FP64 steps stay bounded (5e-4 / 64)
CFG3 = dict(N_r=96, M=32, K=64, m_p=1, eta=0.5, Re_i=2000.0, Re_o=0.0, L_z=LZ, dt=5e-4 / 64)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _inner(a, b):
    """Euclidean inner product on stored (Re, Im) pairs."""
    return float(np.real(np.vdot(a, b)))


def setup(cfg, amp=1e-2, seed=42):
    ops = O.Operators(O.Params(**cfg))
    plan = tc.Plan(**cfg)
    prm = ops.prm
    u0 = I.initial_state(ops.r, prm.M, prm.K, prm.m_p, prm.L_z, prm.eta, prm.Re_i, prm.Re_o,
                         kind="box", amp=amp, mbox=min(4, prm.M), kbox=min(4, prm.K), seed=seed)
    return ops, plan, u0


def gpu_state(plan, st_o):
    st = tc.State(plan, dev(st_o.u))
    st.u_prev.copy_(dev(st_o.u_prev))
    st.N_prev.copy_(dev(st_o.N_prev))
    st.started = True
    return st


@pytest.mark.parametrize("cfg", [CFG1, SMALL])
def test_adjoint_step_matches_oracle(cfg):
    ops, plan, u0 = setup(cfg)
    st_o = O.step(ops, O.cold_state(u0))
    sh = (3,) + ops.prm.shape()
    y = [I.random_spectral(sh, seed=s) for s in (11, 12, 13)]
    ref = O.adjoint_step(ops, st_o, *y)
    bar = tc.StateBar(*[dev(v) for v in y])
    plan.adjoint_step(gpu_state(plan, st_o), bar)
    for got, want in zip((bar.u, bar.u_prev, bar.N_prev), ref):
        assert rel(host(got), want) <= 1e-11


@pytest.mark.parametrize("M", [32, 64, 128])
def test_adjoint_step_theta_lengths(M):
    """The length-specialised adjoint theta pass (P_theta = 96, 192, 384) and the generic one
    (explicit theta_zt) both match the oracle's adjoint step."""
    cfg = dict(N_r=12, M=M, K=4, m_p=1, eta=0.5, Re_i=50.0, Re_o=0.0, L_z=LZ, dt=1e-3)
    ops = O.Operators(O.Params(**cfg))
    prm = ops.prm
    u0 = I.initial_state(ops.r, prm.M, prm.K, prm.m_p, prm.L_z, prm.eta, prm.Re_i, prm.Re_o,
                         kind="broadband", amp=1e-2)
    st_o = O.step(ops, O.cold_state(u0))
    sh = (3,) + prm.shape()
    y = [I.random_spectral(sh, seed=s) for s in (31, 32, 33)]
    ref = O.adjoint_step(ops, st_o, *y)
    for zt in (0, 1):
        plan = tc.Plan(**cfg, theta_zt=zt)
        bar = tc.StateBar(*[dev(v) for v in y])
        plan.adjoint_step(gpu_state(plan, st_o), bar)
        for got, want in zip((bar.u, bar.u_prev, bar.N_prev), ref):
            assert rel(host(got), want) <= 1e-11, zt


@pytest.mark.parametrize("K", [32, 64, 128, 256])
def test_adjoint_step_z_lengths(K):
    """The length-specialised adjoint z passes (P_z = 96 ... 768) and the generic ones
    (explicit theta_zt) both match the oracle's adjoint step."""
    cfg = dict(N_r=10, M=4, K=K, m_p=1, eta=0.5, Re_i=50.0, Re_o=0.0, L_z=LZ, dt=1e-3)
    ops = O.Operators(O.Params(**cfg))
    prm = ops.prm
    u0 = I.initial_state(ops.r, prm.M, prm.K, prm.m_p, prm.L_z, prm.eta, prm.Re_i, prm.Re_o,
                         kind="broadband", amp=1e-2)
    st_o = O.step(ops, O.cold_state(u0))
    sh = (3,) + prm.shape()
    y = [I.random_spectral(sh, seed=s) for s in (41, 42, 43)]
    ref = O.adjoint_step(ops, st_o, *y)
    for zt in (0, 1):
        plan = tc.Plan(**cfg, theta_zt=zt)
        bar = tc.StateBar(*[dev(v) for v in y])
        plan.adjoint_step(gpu_state(plan, st_o), bar)
        for got, want in zip((bar.u, bar.u_prev, bar.N_prev), ref):
            assert rel(host(got), want) <= 1e-11, zt


def test_adjoint_start_matches_oracle():
    ops, plan, u0 = setup(CFG1)
    sh = (3,) + ops.prm.shape()
    y = [I.random_spectral(sh, seed=s) for s in (21, 22, 23)]
    ref = O.adjoint_start_up(ops, u0, *y)
    bar = tc.StateBar(*[dev(v) for v in y])
    got = host(plan.adjoint_start(dev(u0), bar))
    assert rel(got, ref) <= 1e-11


def _gpu_tangent(plan, st_o, x):
    """dF(s)[x] of the CUDA step F at the started state s: F is quadratic in (u, u_prev,
    N_prev) (N(u) is its only nonlinear part; p is not fed back) and its wall values cancel,
    so (F(s + x) - F(s - x)) / 2 equals dF(s)[x] exactly up to rounding, for any size of x."""
    outs = []
    for sg in (1.0, -1.0):
        st = tc.State(plan, dev(st_o.u + sg * x[0]))
        st.u_prev.copy_(dev(st_o.u_prev + sg * x[1]))
        st.N_prev.copy_(dev(st_o.N_prev + sg * x[2]))
        st.started = True
        plan.step(st, 1)
        outs.append([host(st.u), host(st.u_prev), host(st.N_prev)])
    return [(a - b) / 2.0 for a, b in zip(*outs)]


@pytest.mark.parametrize("cfg", [CFG1, "CFG3"])
def test_dot_product_tests_to_1e_12(cfg):
    """<ybar, dF(s)[x]> = <F^T ybar, x> to 1e-12 relative, with the CUDA adjoint on the
    right and, on the left, (a) the CUDA step's own tangent (exact central difference of the
    quadratic step, directions scaled to the state's norm so that no term is lost to
    cancellation) and (b) the oracle's tangent-linear step.  Run at the 20-step parity size and
    at the adjoint workload's size (N_r = 96, m = -32..32, k = -64..64, Re_i = 2000)."""
    if cfg == "CFG3":
        cfg = CFG3
        ops, plan, u0 = setup(cfg, amp=1e-4)
    else:
        ops, plan, u0 = setup(cfg)
    st_o = O.step(ops, O.cold_state(u0))
    sh = (3,) + ops.prm.shape()
    fields = (st_o.u, st_o.u_prev, st_o.N_prev)
    x = [I.random_spectral(sh, seed=s) for s in (31, 32, 33)]
    x = [v * (np.linalg.norm(f) / np.linalg.norm(v)) for v, f in zip(x, fields)]
    y = [I.random_spectral(sh, seed=s) for s in (34, 35, 36)]
    bar = tc.StateBar(*[dev(v) for v in y])
    plan.adjoint_step(gpu_state(plan, st_o), bar)
    rhs = sum(_inner(host(a), b) for a, b in zip((bar.u, bar.u_prev, bar.N_prev), x))
    tl_gpu = _gpu_tangent(plan, st_o, x)
    lhs_gpu = sum(_inner(a, b) for a, b in zip(y, tl_gpu))
    tl_o = O.tangent_step(ops, st_o, *x)
    lhs_o = sum(_inner(a, b) for a, b in zip(y, tl_o))
    print("dot products", lhs_gpu, lhs_o, rhs, abs(lhs_gpu / rhs - 1), abs(lhs_o / rhs - 1))
    assert abs(lhs_gpu - rhs) <= 1e-12 * abs(rhs), (lhs_gpu, rhs)
    assert abs(lhs_o - rhs) <= 1e-12 * abs(rhs), (lhs_o, rhs)


def test_energy_gradient_kernel_matches_oracle():
    ops, plan, u0 = setup(CFG1)
    got = host(plan.energy_gradient(dev(u0)))
    assert rel(got, O.energy_gradient(ops, u0)) <= 1e-14


def test_final_energy_gradient_fd_and_oracle():
    """dJ/du0 after 10 steps (checkpoint every 4): central differences with h = 1e-7 on
    8 random directions agree to <= 1e-6; the gradient agrees with the oracle's."""
    ops, plan, u0 = setup(CFG1)
    n = 10
    u = dev(u0).requires_grad_(False)
    x = u.clone().requires_grad_(True)
    J = A.final_energy(x, plan, n, checkpoint=4)
    J.backward()
    g = host(x.grad)
    g_ref, J_ref = O.gradient_final_energy(ops, u0, n)
    assert abs(J.item() / J_ref - 1) <= 1e-10
    assert rel(g, g_ref) <= 1e-9
    # checkpointing does not change the gradient
    x2 = u.clone().requires_grad_(True)
    A.final_energy(x2, plan, n, checkpoint=n).backward()
    assert rel(host(x2.grad), g) <= 1e-13
    rng = np.random.default_rng(5)
    h = 1e-7
    for _ in range(8):
        d = I.random_spectral((3,) + ops.prm.shape(), seed=int(rng.integers(1 << 30)), hermitian_K=ops.prm.K)
        d[:, 0] = 0.0
        d[:, -1] = 0.0
        dd = dev(d)
        with torch.no_grad():
            Jp = A.final_energy(u + h * dd, plan, n, checkpoint=n).item()
            Jm = A.final_energy(u - h * dd, plan, n, checkpoint=n).item()
        fd = (Jp - Jm) / (2 * h)
        ad = _inner(g, d)
        assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)


def test_final_energy_gradient_fd_at_adjoint_workload():
    """The adjoint workload as stated: N_r = 96, m = -32..32, k = -64..64, Re_i = 2000,
    200 steps with a checkpoint every 20, J = final perturbation energy, seeded initial
    perturbation of amplitude 1e-4 (seed 42) on |m|, |k| <= 4.  The gradient from the
    checkpointed adjoint against central differences with h = 1e-7 on 8 random directions in
    the space of that perturbation (|m|, |k| <= 4, walls fixed), <= 1e-6.  Each direction is
    scaled to the norm of the initial state, so h is a relative step: the state carries the
    Couette flow at Re_i = 2000 against a perturbation of 0.2 RMS, and a step of 1e-7 of the
    perturbation alone is resolved only to the rounding of the total field (about 1e-12 of J,
    i.e. 1e-4 of the difference)."""
    ops, plan, u0 = setup(CFG3, amp=1e-4, seed=42)
    n, C = 200, 20
    u = dev(u0)
    x = u.clone().requires_grad_(True)
    J = A.final_energy(x, plan, n, checkpoint=C)
    J.backward()
    g = host(x.grad)
    assert np.isfinite(J.item()) and np.all(np.isfinite(g))
    rng = np.random.default_rng(7)
    h = 1e-7
    worst = 0.0
    for _ in range(8):
        d = I.random_spectral((3,) + ops.prm.shape(), seed=int(rng.integers(1 << 30)), hermitian_K=ops.prm.K)
        d[:, 0] = 0.0
        d[:, -1] = 0.0
        K = ops.prm.K
        d[:, :, 5:] = 0.0
        d[:, :, :, :K - 4] = 0.0
        d[:, :, :, K + 5:] = 0.0
        d *= np.linalg.norm(u0) / np.linalg.norm(d)
        dd = dev(d)
        with torch.no_grad():
            Jp = A.final_energy(u + h * dd, plan, n, checkpoint=n).item()
            Jm = A.final_energy(u - h * dd, plan, n, checkpoint=n).item()
        fd = (Jp - Jm) / (2 * h)
        ad = _inner(g, d)
        worst = max(worst, abs(fd - ad) / abs(fd))
    print("FD vs adjoint, worst relative difference over 8 directions:", worst)
    assert worst <= 1e-6, worst


def _oracle_power_iteration(ops, u_base, delta0, nsteps, energy, iters):
    """The optimal-perturbation power iteration written with the oracle's own primitives
    (gradient_final_energy, energy_gradient): the same algorithm, independent arithmetic."""
    W = np.real(O.energy_gradient(ops, u_base + 1.0) - O.energy_gradient(ops, u_base))

    def E(d):
        return 0.5 * float(np.sum(W * np.abs(d) ** 2))

    def admissible(d):
        d = d.copy()
        pm = 0.5 * (d[0, :, 0, :] + np.conj(d[1, :, 0, ::-1]))
        zz = 0.5 * (d[2, :, 0, :] + np.conj(d[2, :, 0, ::-1]))
        d[0, :, 0, :], d[1, :, 0, :], d[2, :, 0, :] = pm, np.conj(pm[:, ::-1]), zz
        d[:, 0] = 0
        d[:, -1] = 0
        return d

    g0, J0 = O.gradient_final_energy(ops, u_base, nsteps)
    d = admissible(delta0)
    gains = []
    for _ in range(iters):
        d = d * (energy / E(d)) ** 0.5
        g, J = O.gradient_final_energy(ops, u_base + d, nsteps)
        gains.append((J - J0 - O.inner(g0, d)) / energy)
        d = admissible((g - g0) / W)
    return gains


def test_optimal_perturbation_power_iteration_matches_oracle():
    """Power iteration for the optimal initial perturbation of Couette flow (energy norm, 20
    steps): the gains of the iterates do not decrease, and match the same iteration written
    with the oracle's adjoint from the same seeded start."""
    cfg = dict(N_r=16, M=3, K=6, m_p=1, eta=0.5, Re_i=60.0, Re_o=0.0, L_z=LZ, dt=1e-3)
    ops = O.Operators(O.Params(**cfg))
    plan = tc.Plan(**cfg)
    prm = ops.prm
    base = I.base_state(ops.r, prm.M, prm.K, prm.eta, prm.Re_i, prm.Re_o)
    delta0 = I.initial_state(ops.r, prm.M, prm.K, prm.m_p, prm.L_z, prm.eta, prm.Re_i, prm.Re_o,
                             kind="box", amp=1e-3, seed=21, mbox=3, kbox=3) - base
    nsteps, energy, iters = 20, 1e-6, 5
    d, gains = A.optimal_perturbation(plan, dev(base), nsteps, dev(delta0), energy=energy, iters=iters)
    ref = _oracle_power_iteration(ops, base, delta0, nsteps, energy, iters)
    print("gains", gains, "oracle", ref)
    for a, b in zip(gains, ref):
        assert abs(a / b - 1) <= 1e-6, (a, b)
    for a, b in zip(gains, gains[1:]):
        assert b >= a * (1 - 1e-6), gains
    W = host(A.energy_weights(plan, dev(base)))
    assert abs(0.5 * np.sum(W * np.abs(host(d)) ** 2) / energy - 1) <= 1e-12
