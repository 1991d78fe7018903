"""FP64 transform staging by radial slab (tc_options.stage_rows), the streamed adjoint theta
pass of the long lines (P_theta = 768, 1152), the per-stage transposed steps 2-5 (the adjoint
advance of the split path, large N_r), the workspace a mixed plan shares with its FP64
adjoint, and the host-checkpointed gradient of a run from a started state
(adjoint.state_gradient), all through the C ABI against the oracle.

A row's transforms read no other row's staging, so the forward nonlinear term is bit-identical
for every slab size; the adjoint adds the transposed radial stencil slab by slab, which only
reorders a sum."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def init(ops, kind="box", amp=1e-2, **kw):
    prm = ops.prm
    if kind == "box":
        kw = dict(mbox=min(4, prm.M), kbox=min(4, prm.K), **kw)
    return I.initial_state(ops.r, prm.M, prm.K, prm.m_p, prm.L_z, prm.eta, prm.Re_i, prm.Re_o,
                           kind=kind, amp=amp, **kw)


def gpu_state(plan, st_o):
    st = tc.State(plan, dev(st_o.u))
    st.u_prev.copy_(dev(st_o.u_prev))
    st.N_prev.copy_(dev(st_o.N_prev))
    st.started = True
    return st


@pytest.mark.parametrize("rows", [1, 5, 12, 31])
def test_nonlinear_slabs_bit_identical_and_match_oracle(rows):
    ops = O.Operators(O.Params(**CFG1))
    u = init(ops)
    ref = O.nonlinear(ops, u)
    whole = host(tc.Plan(**CFG1).nonlinear(dev(u)))
    got = host(tc.Plan(**CFG1, stage_rows=rows).nonlinear(dev(u)))
    assert np.array_equal(got, whole)
    assert rel(got, ref) <= 1e-12


@pytest.mark.parametrize("pc_split", [-1, 1])
def test_twenty_steps_slabs_match_oracle(pc_split):
    ops = O.Operators(O.Params(**CFG1))
    u0 = init(ops, amp=1e-3)
    st_o = O.run(ops, O.cold_state(u0), 20)
    plan = tc.Plan(**CFG1, pc_split=pc_split, stage_rows=7)
    st = tc.State(plan, dev(u0))
    plan.step(st, 20)
    for name in ("u", "u_prev", "N_prev", "p"):
        assert rel(host(getattr(st, name)), getattr(st_o, name)) <= 1e-10, name
    plan1 = tc.Plan(**CFG1, pc_split=pc_split)
    st1 = tc.State(plan1, dev(u0))
    plan1.step(st1, 20)
    assert np.array_equal(host(st.u), host(st1.u))


@pytest.mark.parametrize("cfg,rows", [(CFG1, 1), (CFG1, 5), (CFG1, 12), (SMALL, 5)])
def test_adjoint_step_slabs_match_oracle(cfg, rows):
    ops = O.Operators(O.Params(**cfg))
    st_o = O.step(ops, O.cold_state(init(ops)))
    sh = (3,) + ops.prm.shape()
    y = [I.random_spectral(sh, seed=s) for s in (51, 52, 53)]
    ref = O.adjoint_step(ops, st_o, *y)
    outs = []
    for r in (0, rows):
        plan = tc.Plan(**cfg, stage_rows=r)
        bar = tc.StateBar(*[dev(v) for v in y])
        plan.adjoint_step(gpu_state(plan, st_o), bar)
        outs.append([host(b) for b in (bar.u, bar.u_prev, bar.N_prev)])
        for got, want in zip(outs[-1], ref):
            assert rel(got, want) <= 1e-11, (r, rel(got, want))
    for a, b in zip(*outs):          # the slabs only reorder the transposed stencil's sum
        assert rel(a, b) <= 1e-14


def test_adjoint_start_slabs_match_oracle():
    ops = O.Operators(O.Params(**CFG1))
    u0 = init(ops)
    sh = (3,) + ops.prm.shape()
    y = [I.random_spectral(sh, seed=s) for s in (61, 62, 63)]
    ref = O.adjoint_start_up(ops, u0, *y)
    for rows in (0, 7):
        plan = tc.Plan(**CFG1, stage_rows=rows)
        bar = tc.StateBar(*[dev(v) for v in y])
        assert rel(host(plan.adjoint_start(dev(u0), bar)), ref) <= 1e-11, rows


@pytest.mark.parametrize("M,P_theta", [(8, 768), (8, 1152), (256, 768), (384, 1152)])
def test_streamed_adjoint_theta_pass_matches_oracle(M, P_theta):
    """The streamed transposed theta pass (two lines per z resident) at the long lengths,
    with few and with all modes of the line."""
    cfg = dict(N_r=10, M=M, K=4, m_p=1, eta=0.5, Re_i=50.0, Re_o=0.0, L_z=LZ, dt=1e-3)
    ops = O.Operators(O.Params(**cfg, P_theta=P_theta))
    st_o = O.step(ops, O.cold_state(init(ops, kind="broadband")))
    sh = (3,) + ops.prm.shape()
    y = [I.random_spectral(sh, seed=s) for s in (71, 72, 73)]
    ref = O.adjoint_step(ops, st_o, *y)
    plan = tc.Plan(**cfg, P_theta=P_theta, stage_rows=4)
    bar = tc.StateBar(*[dev(v) for v in y])
    plan.adjoint_step(gpu_state(plan, st_o), bar)
    for got, want in zip((bar.u, bar.u_prev, bar.N_prev), ref):
        assert rel(host(got), want) <= 1e-11, rel(host(got), want)


@pytest.mark.parametrize("cfg", [CFG1, SMALL])   # SMALL: the two wall stencils share columns
def test_split_adjoint_advance_matches_oracle(cfg):
    """The per-stage transposed steps 2-5 against the oracle's adjoint step and the fused
    kernel, and its adjoint start-up against the oracle's."""
    ops = O.Operators(O.Params(**cfg))
    u0 = init(ops)
    st_o = O.step(ops, O.cold_state(u0))
    sh = (3,) + ops.prm.shape()
    y = [I.random_spectral(sh, seed=s) for s in (91, 92, 93)]
    ref = O.adjoint_step(ops, st_o, *y)
    outs = []
    for split in (1, -1):
        plan = tc.Plan(**cfg, pc_split=split)
        bar = tc.StateBar(*[dev(v) for v in y])
        plan.adjoint_step(gpu_state(plan, st_o), bar)
        outs.append([host(b) for b in (bar.u, bar.u_prev, bar.N_prev)])
        for got, want in zip(outs[-1], ref):
            assert rel(got, want) <= 1e-11, (split, rel(got, want))
    for a, b in zip(*outs):
        assert rel(a, b) <= 1e-13
    ref0 = O.adjoint_start_up(ops, u0, *y)
    plan = tc.Plan(**cfg, pc_split=1, stage_rows=5)
    bar = tc.StateBar(*[dev(v) for v in y])
    assert rel(host(plan.adjoint_start(dev(u0), bar)), ref0) <= 1e-11


def test_split_adjoint_dot_product_to_1e_12():
    """<ybar, dF(s)[x]> = <F^T ybar, x> with the split forward step's exact central difference
    on the left and the per-stage transposed steps on the right."""
    ops = O.Operators(O.Params(**CFG1))
    st_o = O.step(ops, O.cold_state(init(ops)))
    plan = tc.Plan(**CFG1, pc_split=1)
    sh = (3,) + ops.prm.shape()
    fields = (st_o.u, st_o.u_prev, st_o.N_prev)
    x = [I.random_spectral(sh, seed=s) for s in (101, 102, 103)]
    x = [v * (np.linalg.norm(f) / np.linalg.norm(v)) for v, f in zip(x, fields)]
    y = [I.random_spectral(sh, seed=s) for s in (104, 105, 106)]
    bar = tc.StateBar(*[dev(v) for v in y])
    plan.adjoint_step(gpu_state(plan, st_o), bar)
    rhs = sum(float(np.real(np.vdot(host(a), b))) for a, b in zip((bar.u, bar.u_prev, bar.N_prev), x))
    outs = []
    for sg in (1.0, -1.0):
        st = tc.State(plan, dev(st_o.u + sg * x[0]))
        st.u_prev.copy_(dev(st_o.u_prev + sg * x[1]))
        st.N_prev.copy_(dev(st_o.N_prev + sg * x[2]))
        st.started = True
        plan.step(st, 1)
        outs.append([host(st.u), host(st.u_prev), host(st.N_prev)])
    tl = [(a - b) / 2.0 for a, b in zip(*outs)]
    lhs = sum(float(np.real(np.vdot(a, b))) for a, b in zip(y, tl))
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs), (lhs, rhs)


def test_mixed_plan_adjoint_step_is_the_fp64_adjoint():
    """A mixed plan's adjoint step runs the FP64 kernels on its own workspace layout (FP32
    forward lines, FP64 adjoint slabs, the start-up temporaries over the forward staging):
    bit-identical to the FP64 plan's."""
    ops = O.Operators(O.Params(**CFG1))
    st_o = O.step(ops, O.cold_state(init(ops)))
    sh = (3,) + ops.prm.shape()
    y = [I.random_spectral(sh, seed=s) for s in (81, 82, 83)]
    outs = []
    for prec in (tc.TC_FP64, tc.TC_MIXED):
        plan = tc.Plan(**CFG1, precision=prec, stage_rows=9)
        bar = tc.StateBar(*[dev(v) for v in y])
        plan.adjoint_step(gpu_state(plan, st_o), bar)
        outs.append([host(b) for b in (bar.u, bar.u_prev, bar.N_prev)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_state_gradient_host_checkpoints():
    """adjoint.state_gradient with host checkpoints and two device slots equals the same
    gradient with every state kept (bit for bit: the same steps in the same order), matches
    the oracle's adjoint chain, and agrees with a central difference of J."""
    cfg = CFG1
    ops = O.Operators(O.Params(**cfg))
    u0 = init(ops)
    plan = tc.Plan(**cfg, stage_rows=11)
    n = 12

    def started():
        st = tc.State(plan, dev(u0))
        plan.step(st, 1)
        return st

    st = started()
    s_u, s_up, s_N = host(st.u), host(st.u_prev), host(st.N_prev)
    J1, g1 = A.state_gradient(plan, st, n, checkpoint=5, slots=2, spill=True)
    # st is back at its initial state
    assert np.array_equal(host(st.u), s_u) and np.array_equal(host(st.N_prev), s_N)
    J2, g2 = A.state_gradient(plan, started(), n, checkpoint=n, slots=None, spill=False)
    assert J1 == J2
    for a, b in zip((g1.u, g1.u_prev, g1.N_prev), (g2.u, g2.u_prev, g2.N_prev)):
        assert np.array_equal(host(a), host(b))
    # oracle: forward states, then the adjoint steps back from dJ/du^n
    st_o = O.State(s_u, s_up, s_N, None, True)
    traj = [st_o]
    for _ in range(n):
        traj.append(O.step(ops, traj[-1]))
    ybar = (O.energy_gradient(ops, traj[-1].u), np.zeros_like(s_u), np.zeros_like(s_u))
    for s in reversed(traj[:-1]):
        ybar = O.adjoint_step(ops, s, *ybar)
    for got, want in zip((g1.u, g1.u_prev, g1.N_prev), ybar):
        assert rel(host(got), want) <= 1e-10
    # central difference along a direction in the low modes of u
    prm = ops.prm
    d = (I.initial_state(ops.r, prm.M, prm.K, 1, prm.L_z, prm.eta, prm.Re_i, prm.Re_o, kind="box",
                         amp=1.0, mbox=2, kbox=2, seed=5)
         - I.base_state(ops.r, prm.M, prm.K, prm.eta, prm.Re_i, prm.Re_o))
    h = 1e-6 * np.linalg.norm(s_u) / np.linalg.norm(d)
    Js = []
    for sg in (1.0, -1.0):
        st2 = tc.State(plan, dev(s_u + sg * h * d))
        st2.u_prev.copy_(dev(s_up))
        st2.N_prev.copy_(dev(s_N))
        st2.started = True
        plan.step(st2, n)
        Js.append(plan.diagnostics(st2.u).energy)
    fd = (Js[0] - Js[1]) / (2 * h)
    ad = float(np.real(np.vdot(host(g1.u), d)))
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
