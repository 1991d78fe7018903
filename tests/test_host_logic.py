"""Host-side logic that needs no GPU: the real-field projection of the optimal-perturbation
iteration (adjoint.optimal_perturbation) and the iteration itself on a linear map with a known
largest gain, and the checkpoint and slot schedules of adjoint.final_energy and
adjoint.state_gradient, run against stand-ins for the plan."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1311_2481_gb300 import adjoint as A  # noqa: E402


def test_real_field_projection_of_the_m0_line():
    """The m = 0 line of a real vector field satisfies d_+(0,k) = conj d_-(0,-k) and
    d_z(0,k) = conj d_z(0,-k); the projection enforces exactly that, leaves m > 0 alone, is
    idempotent, and keeps a line that already has the symmetry."""
    rng = np.random.default_rng(4)
    shape = (3, 6, 4, 9)   # [c][r][m][k], K = 4
    d = torch.from_numpy(rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    p = A._real_field_m0(d)
    line = p[:, :, 0, :].numpy()
    assert np.array_equal(line[0], np.conj(line[1][:, ::-1]))
    assert np.array_equal(line[2], np.conj(line[2][:, ::-1]))
    assert np.all(line[2][:, 4].imag == 0)
    assert torch.equal(p[:, :, 1:, :], d[:, :, 1:, :])
    assert torch.equal(A._real_field_m0(p), p)
    # the projection is the orthogonal one: the removed part is orthogonal to every symmetric line
    r = (d - p)[:, :, 0, :].numpy()
    q = A._real_field_m0(torch.from_numpy(rng.standard_normal(shape) + 1j * rng.standard_normal(shape)))
    assert abs(np.real(np.vdot(r, q[:, :, 0, :].numpy()))) <= 1e-12 * np.linalg.norm(r) * np.linalg.norm(q.numpy())


class _CountingPlan:
    """Stands in for a plan in adjoint.state_gradient: a step adds 1 to every field, so the
    velocity of forward state j is j; an adjoint step records the velocity it is given."""

    def __init__(self):
        self.steps = 0
        self.read = []

    def step(self, st, n):
        for _ in range(n):
            st.u += 1
            st.u_prev += 1
            st.N_prev += 1
            self.steps += 1

    def diagnostics(self, u):
        return type("D", (), {"energy": float(u.real.sum())})()

    def energy_gradient(self, u):
        return u.clone()

    def adjoint_step(self, fwd, bar):
        self.read.append(int(fwd.u.real.flatten()[0]))


def _counting_state():
    st = type("S", (), {})()
    st.u = torch.zeros((3, 2, 2, 3), dtype=torch.complex128)
    st.u_prev = torch.full_like(st.u, -1.0)
    st.N_prev = torch.full_like(st.u, 5.0)
    st.p = torch.zeros((2, 2, 3), dtype=torch.complex128)
    st.started = True
    return st


@pytest.mark.parametrize("nsteps,checkpoint,slots", [(1, 1, None), (7, 3, None), (7, 3, 2), (10, 10, 1),
                                                     (50, 17, 7), (12, 5, 5), (9, 4, 3)])
def test_state_gradient_reverses_every_step_once(nsteps, checkpoint, slots):
    """adjoint.state_gradient's schedule: the adjoint steps read the forward velocities
    u^{n-1}, ..., u^0 once each and in that order, whatever the checkpoint interval and the
    number of device slots; the final energy is that of u^n; the working state is given back
    with its initial fields; and each segment of C steps reversed in passes of k slots is
    recomputed once per pass."""
    plan, st = _CountingPlan(), _counting_state()
    J, bar = A.state_gradient(plan, st, nsteps, checkpoint=checkpoint, slots=slots, spill=False)
    assert plan.read == list(range(nsteps - 1, -1, -1))
    assert J == float(nsteps * st.u.numel())
    assert torch.equal(bar.u, torch.full_like(st.u, float(nsteps)))
    assert torch.all(st.u == 0) and torch.all(st.u_prev == -1) and torch.all(st.N_prev == 5)
    k = checkpoint if slots is None else max(1, min(slots, checkpoint))
    recompute = 0
    for s0 in range(0, nsteps, checkpoint):
        hi = min(s0 + checkpoint, nsteps)
        while hi > s0:
            recompute += hi - 1 - s0      # steps from the checkpoint to the last state of the pass
            hi = max(s0, hi - k)
    assert plan.steps == nsteps + recompute


def test_state_gradient_refuses_an_unstarted_state_and_oversized_host_checkpoints(monkeypatch):
    plan, st = _CountingPlan(), _counting_state()
    st.started = False
    with pytest.raises(ValueError, match="started"):
        A.state_gradient(plan, st, 3)
    st.started = True
    with pytest.raises(ValueError, match=">= 1"):
        A.state_gradient(plan, st, 3, checkpoint=0)
    monkeypatch.setattr(A, "_host_bytes_available", lambda: 1000)
    with pytest.raises(ValueError, match="host checkpoints"):
        A.state_gradient(plan, st, 30, checkpoint=10, spill=True)
    assert plan.steps == 0


class _CountingColdPlan(_CountingPlan):
    """The counting plan with what adjoint.FinalEnergy also needs: a device, the scalar shape,
    the history step (nsteps = 0) and the adjoint of the cold start (here the identity)."""

    device = "cpu"

    def scalar_shape(self):
        return (2, 2, 3)

    def step(self, st, n):
        st.started = True
        super().step(st, n)

    def adjoint_start(self, u0, bar):
        return bar.u.clone()


@pytest.mark.parametrize("nsteps,checkpoint", [(1, 1), (1, 20), (6, 2), (7, 3), (20, 20), (21, 20), (9, 4)])
def test_final_energy_backward_reverses_every_step_once(nsteps, checkpoint):
    """FinalEnergy's backward pass: the adjoint steps read u^{n-1}, ..., u^0 once each and in
    that order, for any checkpoint interval, and the gradient is what the cold-start adjoint
    returns for the energy gradient of u^n scaled by the incoming gradient."""
    plan = _CountingColdPlan()
    u0 = torch.zeros((3, 2, 2, 3), dtype=torch.complex128, requires_grad=True)
    J = A.final_energy(u0, plan, nsteps, checkpoint=checkpoint)
    assert float(J.detach()) == float(nsteps * u0.numel())
    plan.steps = 0
    (2.0 * J).backward()
    assert plan.read == list(range(nsteps - 1, -1, -1))
    assert torch.equal(u0.grad, torch.full_like(u0, 2.0 * nsteps))
    starts = sorted({0} | {s for s in range(checkpoint, nsteps, checkpoint)})
    ends = starts[1:] + [nsteps]
    assert plan.steps == sum(e - 1 - s for s, e in zip(starts, ends))


class _DiagonalPlan(_CountingColdPlan):
    """A linear step u <- a u (coefficient-wise) with the energy J = 1/2 sum W |u|^2: its
    adjoint step multiplies by conj(a), so every quantity of the power iteration is known in
    closed form."""

    def __init__(self, a, W):
        super().__init__()
        self.a, self.W = a, W

    def step(self, st, n):
        st.started = True
        for _ in range(n):
            st.u = self.a * st.u

    def diagnostics(self, u):
        return type("D", (), {"energy": 0.5 * float((self.W * u.abs() ** 2).sum())})()

    def energy_gradient(self, u):
        return self.W * u

    def adjoint_step(self, fwd, bar):
        bar.u = torch.conj(self.a) * bar.u


def test_optimal_perturbation_finds_the_largest_gain_of_a_linear_map():
    """adjoint.optimal_perturbation on a diagonal linear step: the gain converges to the
    largest |a|^(2n) over the admissible coefficients (interior rows), the iterate to that
    coefficient, and the wall rows stay zero; a larger |a| on a wall row is not admissible."""
    shape = (3, 5, 3, 7)                       # [c][r][m][k], N_r = 5, M = 2, K = 3
    a = torch.full(shape, 0.5, dtype=torch.complex128)
    a[1, 2, 1, 5] = 0.9 * np.exp(0.3j)         # the leading interior coefficient (m = 1)
    a[0, 0, 2, 1] = 0.99                       # larger, but on the inner wall row
    W = 1.0 + torch.arange(5, dtype=torch.float64).reshape(1, 5, 1, 1).expand(shape).contiguous()
    plan = _DiagonalPlan(a, W)
    rng = np.random.default_rng(3)
    d0 = torch.from_numpy(rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    n = 3
    d, gains = A.optimal_perturbation(plan, torch.zeros(shape, dtype=torch.complex128), n, d0,
                                      energy=1e-6, iters=8, checkpoint=2)
    assert abs(gains[-1] - 0.9 ** (2 * n)) <= 1e-9 * 0.9 ** (2 * n)
    assert all(g1 >= g0 - 1e-12 for g0, g1 in zip(gains, gains[1:]))
    assert torch.all(d[:, 0] == 0) and torch.all(d[:, -1] == 0)
    lead = d[1, 2, 1, 5].abs() ** 2
    assert float((d.abs() ** 2).sum() - lead) <= 1e-12 * float(lead)


def test_roofline_arithmetic_at_the_bench_workload():
    """bench.py's per-launch algorithmic figures at N_r = 64, M = 32, K = 64 (P_theta = 96,
    P_z = 192): the theta-pass reads the 9 H1 line sets and writes the 3 H2 ones (77.9 MB)
    and counts 0.32 GFLOP; a launch of 0.4292 ms is then 0.747 TFLOP/s, 0.594 of the FP64
    peak of 152 SMs x 2 DFMA x 2 flop x 2.07 GHz."""
    import bench
    cfg = dict(N_r=64, M=32, K=64)
    H = 64 * 33 * 192
    rf = bench.kernel_rooflines(cfg, {"k_theta": (1, 0.4292), "k_zinv": (1, 0.2052), "k_pc": (2, 0.4926)})
    th = rf["kernels"]["k_theta"]
    assert th["bytes"] == 12 * H * 16 == 77_856_768
    assert abs(th["flops"] - 320.79e6) <= 0.01e6
    assert abs(th["flops"] / 0.4292e-3 / 1e12 - 0.747) <= 0.001
    assert abs(th["fp64_frac"] - 0.594) <= 0.001
    assert bench.FP64_PEAK == pytest.approx(1.25856e12)
    assert rf["kernels"]["k_zinv"]["bytes"] == 3 * 64 * 33 * 129 * 16 + 9 * H * 16
    assert rf["kernels"]["k_pc"]["ms"] == pytest.approx(0.2463)
    assert "flops" not in rf["kernels"]["k_pc"]
