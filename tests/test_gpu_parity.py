"""Parity of the CUDA path (through the C ABI) with the CPU oracle on seeded inputs.

Tolerances: relative L2 over all stored coefficients <= 1e-12 for one nonlinear evaluation
and <= 1e-10 after 20 time steps (config: N_r = 32, m = -8..8, k = -16..16, Re_i = 50,
dt = 1e-3); solves <= 1e-12 relative to the solution norm.  The oracle evaluates the same
discrete method with naive DFT matrices and dense solves, so only rounding order differs.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_1311_2481_gb300 import build as B  # noqa: E402
from paper_1311_2481_gb300 import inputs as I  # noqa: E402
from paper_1311_2481_gb300 import tc  # noqa: E402

B.build()
LZ = 2 * math.pi / 3.16
CFG1 = dict(N_r=32, M=8, K=16, m_p=1, eta=0.5, Re_i=50.0, Re_o=0.0, L_z=LZ, dt=1e-3)
CFG2 = dict(N_r=64, M=32, K=64, m_p=1, eta=0.5, Re_i=1000.0, Re_o=0.0, L_z=LZ, dt=5e-4)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def pair(cfg, **opt):
    prm = O.Params(**cfg, **{k: v for k, v in opt.items() if k in ("alpha", "P_theta", "P_z")})
    ops = O.Operators(prm)
    plan = tc.Plan(**cfg, **opt)
    return ops, plan


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def init(ops, kind="box", amp=1e-3, **kw):
    prm = ops.prm
    return I.initial_state(ops.r, prm.M, prm.K, prm.m_p, prm.L_z, prm.eta, prm.Re_i, prm.Re_o,
                           kind=kind, amp=amp, **kw)


@pytest.mark.parametrize("shape", [
    dict(),                                               # config 1 (3/2 grid 24 x 48)
    dict(N_r=20, M=6, K=9),                               # radix-2/3 only, ragged sizes
    dict(N_r=11, M=4, K=5, P_theta=16, P_z=16),           # explicit grids (exact 3/2+ rule)
    dict(N_r=9, M=1, K=1),                                # smallest: 3 x 3 grid, 9 nodes
])
def test_nonlinear_matches_oracle(shape):
    cfg = {**CFG1, **{k: v for k, v in shape.items() if k in CFG1}}
    opt = {k: v for k, v in shape.items() if k not in CFG1}
    ops, plan = pair(cfg, **opt)
    prm = ops.prm
    for seed, u in ((0, init(ops, amp=1e-2, mbox=min(4, prm.M), kbox=min(4, prm.K))),
                    (1, I.random_spectral((3,) + prm.shape(), seed=7))):
        ref = O.nonlinear(ops, u)
        got = host(plan.nonlinear(dev(u)))
        assert rel(got, ref) <= 1e-12, (seed, rel(got, ref))


def test_nonlinear_full_size_config2():
    ops, plan = pair(CFG2)
    u = init(ops, kind="taylor", amp=1e-2)
    ref = O.nonlinear(ops, u)
    got = host(plan.nonlinear(dev(u)))
    assert rel(got, ref) <= 1e-12
    pert = np.ones(got.shape, bool)
    pert[:, :, 0, ops.prm.K] = False
    assert rel(got[pert], ref[pert]) <= 1e-11


@pytest.mark.parametrize("which,name", [(tc.TC_P_STAR, "P"), (tc.TC_U_PLUS, "Hp"),
                                        (tc.TC_U_MINUS, "Hm"), (tc.TC_U_Z, "Hz"), (tc.TC_PHI, "P")])
def test_banded_solves_match_dense(which, name):
    ops, plan = pair({**CFG1, "N_r": 40})
    prm = ops.prm
    b = I.random_spectral(prm.shape(), seed=100 + which)
    ref = O.solve_modes(ops, ops.mats[name], b)
    got = host(plan.helmholtz_solve(which, dev(b)))
    assert rel(got, ref) <= 1e-12, rel(got, ref)
    x = dev(b)
    plan.helmholtz_solve(which, x, x)          # in place
    assert rel(host(x), ref) <= 1e-12


@pytest.mark.parametrize("pc_split", [-1, 1])      # fused steps-2-5 kernel, split kernels
def test_twenty_steps_match_oracle(pc_split):
    ops, plan = pair(CFG1, pc_split=pc_split)
    u0 = init(ops)
    st_o = O.cold_state(u0)
    st_o = O.run(ops, st_o, 20)
    st = tc.State(plan, dev(u0))
    plan.step(st, 20)
    for name in ("u", "u_prev", "N_prev", "p"):
        got, ref = host(getattr(st, name)), getattr(st_o, name)
        assert rel(got, ref) <= 1e-10, (name, rel(got, ref))
    ref = st_o.u
    pert = np.ones(ref.shape, bool)
    pert[:, :, 0, ops.prm.K] = False
    assert rel(host(st.u)[pert], ref[pert]) <= 1e-9
    # stepping in two calls is the same as one call
    st2 = tc.State(plan, dev(u0))
    plan.step(st2, 7)
    plan.step(st2, 13)
    assert rel(host(st2.u), host(st.u)) <= 1e-14


@pytest.mark.parametrize("case", [
    dict(N_r=20, M=4, K=6, m_p=6, eta=0.868, Re_i=458.1, L_z=2.4, dt=2e-5),   # wavy-vortex parameters
    dict(N_r=24, M=4, K=6, eta=0.71, Re_i=300.0, Re_o=-150.0, dt=2e-4),        # counter-rotation
    dict(N_r=12, M=4, K=4, fd_order=4),                                         # 5-point stencils
    dict(N_r=10, M=3, K=4, fd_order=2),                                         # 3-point stencils
    dict(N_r=18, M=4, K=6, alpha=0.0),                                          # Chebyshev limit of the nodes
    dict(N_r=18, M=4, K=6, alpha=1.0),                                          # uniform nodes
])
def test_twenty_steps_match_oracle_across_parameters(case):
    """The whole step against the oracle over 20 steps away from the default parameters:
    m_p > 1 with the wavy-vortex geometry, a rotating outer cylinder, shorter FD stencils, and
    both limits of the node clustering of Eq. nodeDist; fused and split steps 2-5.  p carries
    3 phi / (2 dt), so its bound grows as the time step falls below the 1e-3 of the 20-step
    gate."""
    cfg = {**CFG1, **{k: v for k, v in case.items() if k in CFG1 or k == "fd_order"}}
    opt = {k: v for k, v in case.items() if k == "alpha"}
    prm = O.Params(**cfg, **opt)
    ops = O.Operators(prm)
    u0 = init(ops, amp=1e-2, mbox=min(3, prm.M), kbox=min(3, prm.K))
    ref = O.run(ops, O.cold_state(u0), 20)
    for pc_split in (-1, 1):
        plan = tc.Plan(**cfg, **opt, pc_split=pc_split)
        st = tc.State(plan, dev(u0))
        plan.step(st, 20)
        for name in ("u", "u_prev", "N_prev", "p"):
            got = host(getattr(st, name))
            tol = 1e-10 * (max(1.0, 1e-3 / cfg["dt"]) if name == "p" else 1.0)
            assert rel(got, getattr(ref, name)) <= tol, (pc_split, name, rel(got, getattr(ref, name)))


@pytest.mark.parametrize("pc_split", [0, 1])
def test_step_full_size_config2(pc_split):
    ops, plan = pair(CFG2, pc_split=pc_split)
    u0 = init(ops, kind="taylor", amp=1e-2)
    st_o = O.run(ops, O.cold_state(u0), 2)
    st = tc.State(plan, dev(u0))
    plan.step(st, 2)
    assert rel(host(st.u), st_o.u) <= 1e-11
    assert rel(host(st.p), st_o.p) <= 1e-10


@pytest.mark.parametrize("N_r", [15, 16, 17, 33])
def test_partitioned_solves_match_oracle(N_r):
    """The fused kernel's two-partition (SPIKE) form of the banded systems, with even, odd and
    ragged cuts (N_r = 15 keeps one partition): 20 steps against the oracle, and against the
    one-partition form of the same kernel to rounding (the forms differ in rounding order, so
    a cut plan's state is not bit-identical to the uncut one)."""
    cfg = dict(CFG1, N_r=N_r)
    ops = O.Operators(O.Params(**cfg))
    u0 = init(ops, kind="broadband", amp=1e-2, seed=12)
    ref = O.run(ops, O.cold_state(u0), 20)
    out = {}
    for parts in (1, 2):
        plan = tc.Plan(**cfg, pc_split=-1, pc_partitions=parts)
        st = tc.State(plan, dev(u0))
        plan.step(st, 20)
        out[parts] = {k: host(getattr(st, k)) for k in ("u", "p")}
        for k in ("u", "p"):
            assert rel(out[parts][k], getattr(ref, k)) <= 1e-10, (parts, k, rel(out[parts][k], getattr(ref, k)))
    for k in ("u", "p"):
        assert rel(out[2][k], out[1][k]) <= 1e-12, (k, rel(out[2][k], out[1][k]))
    assert np.array_equal(out[2]["u"], out[1]["u"]) == (N_r < 16)


@pytest.mark.parametrize("pc_split", [-1, 1])
def test_nonfinite_state_is_reported_by_the_next_step(pc_split):
    """A step that writes a NaN into the state raises the plan's flag (mapped host memory):
    the next tc_step returns TC_ERR_NONFINITE before launching and clears it; tc_step_host
    reports its own steps."""
    ops, plan = pair(CFG1, pc_split=pc_split)
    u0 = init(ops)
    st = tc.State(plan, dev(u0))
    plan.step(st, 2)
    bad = host(st.u).copy()
    bad[0, 5, 1, ops.prm.K] = np.nan
    st.u.copy_(dev(bad))
    plan.step(st, 1)
    torch.cuda.synchronize()
    with pytest.raises(tc.TCError) as e:
        plan.step(st, 1)
    assert e.value.status == tc.TC_ERR_NONFINITE
    st2 = tc.State(plan, dev(u0))
    plan.step(st2, 3)                               # cleared: a finite state steps on
    assert plan.diagnostics(st2.u).finite
    hin = {k: torch.from_numpy(host(getattr(st2, k))).pin_memory() for k in ("u", "u_prev", "N_prev", "p")}
    hin["u"][0, 5, 1, ops.prm.K] = complex("nan")
    hin["started"] = True
    hout = {"u": torch.empty_like(hin["u"]).pin_memory()}
    with pytest.raises(tc.TCError) as e:
        plan.step_host(st2, hin, hout, 1)
    assert e.value.status == tc.TC_ERR_NONFINITE
    hin["u"][0, 5, 1, ops.prm.K] = complex(0.0)
    plan.step_host(st2, hin, hout, 1)               # cleared again


def test_unmapped_buffer_tails_rejected_before_launch():
    """A buffer whose bytes run past mapped device memory is rejected on the host (the
    driver's address-range query, walked over contiguous mappings).  Every call here is
    tc_step with nsteps = 0 on a started state, which launches nothing even when the
    arguments pass, so the test cannot touch device memory either way.  The bogus workspace
    starts on the last 256-byte boundary at least 256 bytes before the end of the mapped run
    that holds the state's u (found with the same driver query), so the 0.2 GB it must hold
    cross into unmapped memory."""
    import ctypes
    try:
        cuda = ctypes.CDLL("libcuda.so.1")
    except OSError:
        pytest.skip("no driver library to locate the end of the mapping")
    get_range = cuda.cuMemGetAddressRange_v2
    get_range.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_size_t), ctypes.c_uint64]
    get_range.restype = ctypes.c_int
    ops, plan = pair(CFG2)
    lib = tc.load_library()
    st = tc.State(plan, dev(init(ops)))
    plan.step(st, 0)
    assert st.started

    def call(u_ptr, ws_ptr):
        cs = tc.tc_state(u_ptr, st.u_prev.data_ptr(), st.N_prev.data_ptr(), st.p.data_ptr(), 1)
        return lib.tc_step(plan.handle, ctypes.byref(cs), 0, ws_ptr, None)

    base, size = ctypes.c_uint64(0), ctypes.c_size_t(0)
    end = st.u.data_ptr()
    for _ in range(100000):   # to the end of the contiguous run of mappings
        if get_range(ctypes.byref(base), ctypes.byref(size), ctypes.c_uint64(end)) != 0 or base.value > end:
            break
        end = base.value + size.value
    ws = plan._ws()
    assert call(st.u.data_ptr(), ws) == tc.TC_OK
    assert call(st.u.data_ptr(), ctypes.c_void_p((end - 256) & ~255)) == tc.TC_ERR_ARG
    assert b"are mapped" in lib.tc_plan_last_error(plan.handle)
    assert call(st.u.data_ptr(), ws) == tc.TC_OK


def test_diagnostics_match_oracle():
    ops, plan = pair(CFG1)
    u = O.run(ops, O.cold_state(init(ops)), 3).u
    d = plan.diagnostics(dev(u))
    assert d.finite == 1
    assert abs(d.energy / O.perturbation_energy(ops, u) - 1) < 1e-12
    Ti, To = O.torque(ops, u)
    assert abs(d.torque_inner / Ti - 1) < 1e-12 and abs(d.torque_outer / To - 1) < 1e-12
    assert abs(d.max_div / O.max_divergence(ops, u) - 1) < 1e-10
    bad = u.copy()
    bad[2, 5, 1, 3] = np.nan
    d = plan.diagnostics(dev(bad))
    assert d.finite == 0


def test_invalid_pointers_rejected():
    ops, plan = pair(CFG1)
    u = dev(init(ops))
    lib = tc.load_library()
    hostbuf = np.zeros(8, np.complex128)
    st = lib.tc_nonlinear(plan.handle, hostbuf.ctypes.data, u.data_ptr(), plan._ws(), None)
    assert st == tc.TC_ERR_ARG
    st = lib.tc_nonlinear(plan.handle, u.data_ptr(), u.data_ptr(), plan._ws(), None)
    assert st == tc.TC_ERR_ARG
    st = lib.tc_helmholtz_solve(plan.handle, 7, u.data_ptr(), u.data_ptr(), plan._ws(), None)
    assert st == tc.TC_ERR_ARG


# ------------------------------------------------------------------ mixed precision form

def _mean_removed(ops, u):
    K = ops.prm.K
    up = u.copy()
    U = np.imag(u[0, :, 0, K] - u[1, :, 0, K]) / 2
    up[0, :, 0, K] -= 1j * U
    up[1, :, 0, K] += 1j * U
    return up


@pytest.mark.parametrize("cfg", [CFG1, CFG2])
def test_mixed_nonlinear_error_is_fp32_level_of_the_perturbation_part(cfg):
    """FP32 transforms of N(u') plus FP64 mean-flow terms: the error against the FP64
    oracle is bounded by a few FP32 roundings of the perturbation part N(u')."""
    ops = O.Operators(O.Params(**cfg))
    plan = tc.Plan(**cfg, precision=tc.TC_MIXED)
    u = init(ops, kind="taylor" if cfg is CFG2 else "box", amp=1e-2)
    ref = O.nonlinear(ops, u)
    ref_pert = O.nonlinear(ops, _mean_removed(ops, u))
    got = host(plan.nonlinear(dev(u)))
    err = np.linalg.norm(got - ref)
    assert err <= 2e-6 * np.linalg.norm(ref_pert), err / np.linalg.norm(ref_pert)
    assert err <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("case", ["bench", "quasi_keplerian"])
def test_mixed_mean_mode_at_fp64_accuracy(case):
    """The mixed form's (m, k) = (0, 0) mode of N, the mean the torque depends on, comes from
    the double-FP32 Parseval sum of the FP64 state: against the oracle to 1e-10 of the
    perturbation's share of that mode (the FP32 transforms alone give 1e-5 there)."""
    if case == "bench":
        cfg, kind, amp = CFG2, "taylor", 1e-2
    else:
        Re = 3e4
        cfg = dict(N_r=24, M=24, K=32, m_p=1, eta=0.5, Re_i=Re, Re_o=math.sqrt(0.5) * Re, L_z=LZ, dt=1e-8)
        kind, amp = "broadband", 0.05
    ops = O.Operators(O.Params(**cfg))
    plan = tc.Plan(**cfg, precision=tc.TC_MIXED)
    u = init(ops, kind=kind, amp=amp)
    K = ops.prm.K
    ref = O.nonlinear(ops, u)[:, :, 0, K]
    base = O.nonlinear(ops, I.base_state(ops.r, ops.prm.M, K, cfg["eta"], cfg["Re_i"], cfg["Re_o"]))[:, :, 0, K]
    got = host(plan.nonlinear(dev(u)))[:, :, 0, K]
    for c in range(3):
        scale = np.linalg.norm(ref[c] - base[c])
        assert np.linalg.norm(got[c] - ref[c]) <= 1e-10 * scale, (c, np.linalg.norm(got[c] - ref[c]) / scale)


def test_mixed_mean_fp32_option_changes_only_the_mean_mode():
    """tc_options.mean_fp32 keeps the FP32 transforms' (0,0) mode of N; every other
    coefficient is bit-identical to the default mixed plan's."""
    ops = O.Operators(O.Params(**CFG1))
    u = init(ops, kind="box", amp=1e-2)
    a = host(tc.Plan(**CFG1, precision=tc.TC_MIXED).nonlinear(dev(u)))
    b = host(tc.Plan(**CFG1, precision=tc.TC_MIXED, mean_fp32=True).nonlinear(dev(u)))
    K = ops.prm.K
    keep = np.ones(a.shape, bool)
    keep[:, :, 0, K] = False
    assert np.array_equal(a[keep], b[keep])
    ref = O.nonlinear(ops, u)
    assert rel(b, ref) <= 2e-6


def test_mixed_nonlinear_m0_line_is_a_real_field():
    """The mixed form's N keeps the m = 0 symmetry of a real field exactly:
    N_+(0,k) = conj N_-(0,-k) and N_z(0,k) = conj N_z(0,-k)."""
    cfg = dict(CFG1, m_p=6, eta=0.868, Re_i=458.1, L_z=2.4, dt=2e-5)
    ops, plan = pair(cfg, precision=tc.TC_MIXED)
    u0 = init(ops, kind="taylor", amp=1e-2, seed=7)
    N = host(plan.nonlinear(dev(u0)))
    K = ops.prm.K
    Np, Nm, Nz = N[0, :, 0, :], N[1, :, 0, :], N[2, :, 0, :]
    assert np.array_equal(Np, np.conj(Nm[:, ::-1]))
    assert np.array_equal(Nz, np.conj(Nz[:, ::-1]))
    assert np.all(Nz[:, K].imag == 0)
    ref = O.nonlinear(ops, u0)
    assert rel(N, ref) <= 2e-6


@pytest.mark.parametrize("M,K", [(16, 8), (32, 8), (64, 8), (128, 8), (256, 4), (384, 4), (512, 4)])
def test_mixed_theta_pass_lengths(M, K):
    """Every length-specialised theta pass (P_theta = 48 ... 1536) against the oracle and
    against the generic theta kernel (selected by an explicit theta_zt), on a broadband state
    with all stored modes excited."""
    cfg = dict(N_r=12, M=M, K=K, m_p=1, eta=0.5, Re_i=1000.0, Re_o=0.0, L_z=LZ, dt=1e-4)
    ops = O.Operators(O.Params(**cfg))
    u = init(ops, kind="broadband", amp=1e-2, seed=5)
    ref = O.nonlinear(ops, u)
    nrm = np.linalg.norm(O.nonlinear(ops, _mean_removed(ops, u)))
    got = {}
    for zt, variant in ((0, 0), (1, 0), (0, 1), (0, 2), (0, 3), (0, 4)):
        plan = tc.Plan(**cfg, precision=tc.TC_MIXED, theta_zt=zt, no_adjoint=True, theta_variant=variant)
        got[zt, variant] = host(plan.nonlinear(dev(u)))
        err = np.linalg.norm(got[zt, variant] - ref)
        assert err <= 2e-6 * nrm, (zt, variant, err / nrm)
    assert np.linalg.norm(got[0, 0] - got[1, 0]) <= 2e-6 * nrm


@pytest.mark.parametrize("M,K", [(32, 8), (64, 8), (128, 8), (256, 4), (384, 4)])
def test_fp64_theta_pass_lengths(M, K):
    """The length-specialised FP64 theta pass (P_theta = 96 ... 1152) and the generic one
    (explicit theta_zt) both match the oracle to 1e-12 on a broadband state."""
    cfg = dict(N_r=12, M=M, K=K, m_p=1, eta=0.5, Re_i=1000.0, Re_o=0.0, L_z=LZ, dt=1e-4)
    ops = O.Operators(O.Params(**cfg))
    u = init(ops, kind="broadband", amp=1e-2, seed=7)
    ref = O.nonlinear(ops, u)
    for zt in (0, 1):
        plan = tc.Plan(**cfg, theta_zt=zt)
        assert rel(host(plan.nonlinear(dev(u))), ref) <= 1e-12, zt


@pytest.mark.parametrize("M,K,P_theta,P_z", [(35, 71, 96, 192), (36, 72, 96, 192),
                                             (32, 64, 96, 192), (24, 48, 96, 192)])
def test_fp64_first_pass_zero_band_both_sides(M, K, P_theta, P_z):
    """The FP64 first inverse radix-8 pass leaves out inputs 3 and 4 of its butterflies only when
    the zero band M < m < P - M holds [3P/8, 5P/8): M = 35 on P = 96 (band 36..60) is the last
    such case, M = 36 (band 37..59) takes the full pass; likewise K = 71 / 72 on P_z = 192.
    Both sides, and the default and a wider band, match the oracle on the same lengths to
    1e-12 (with P < 3M the product is aliased on both sides alike)."""
    cfg = dict(N_r=12, M=M, K=K, m_p=1, eta=0.5, Re_i=1000.0, Re_o=0.0, L_z=LZ, dt=1e-4)
    ops = O.Operators(O.Params(**cfg, P_theta=P_theta, P_z=P_z))
    u = init(ops, kind="broadband", amp=1e-2, seed=9)
    ref = O.nonlinear(ops, u)
    plan = tc.Plan(**cfg, P_theta=P_theta, P_z=P_z)
    assert rel(host(plan.nonlinear(dev(u))), ref) <= 1e-12


@pytest.mark.parametrize("K", [128, 256, 384, 512])
def test_fp64_z_pass_lengths(K):
    """The length-specialised FP64 z passes (P_z = 384 ... 1536) and the generic ones
    (explicit theta_zt) both match the oracle to 1e-12."""
    cfg = dict(N_r=9, M=2, K=K, m_p=1, eta=0.5, Re_i=1000.0, Re_o=0.0, L_z=LZ, dt=1e-4)
    ops = O.Operators(O.Params(**cfg))
    u = init(ops, kind="broadband", amp=1e-2, seed=8)
    ref = O.nonlinear(ops, u)
    for zt in (0, 1):
        plan = tc.Plan(**cfg, theta_zt=zt)
        assert rel(host(plan.nonlinear(dev(u))), ref) <= 1e-12, zt


@pytest.mark.parametrize("K", [128, 256, 384, 512, 768, 1024])
def test_mixed_z_pass_lengths(K):
    """The length-specialised z passes (P_z = 384 ... 3072) against the oracle and against the
    generic z kernels (selected by an explicit theta_zt)."""
    cfg = dict(N_r=9, M=2, K=K, m_p=1, eta=0.5, Re_i=1000.0, Re_o=0.0, L_z=LZ, dt=1e-4)
    ops = O.Operators(O.Params(**cfg))
    u = init(ops, kind="broadband", amp=1e-2, seed=6)
    ref = O.nonlinear(ops, u)
    nrm = np.linalg.norm(O.nonlinear(ops, _mean_removed(ops, u)))
    got = {}
    for zt in (0, 1):
        plan = tc.Plan(**cfg, precision=tc.TC_MIXED, theta_zt=zt, no_adjoint=True)
        got[zt] = host(plan.nonlinear(dev(u)))
        assert np.linalg.norm(got[zt] - ref) <= 2e-6 * nrm, zt
    assert np.linalg.norm(got[0] - got[1]) <= 2e-6 * nrm


def test_mixed_twenty_steps_track_fp64():
    ops = O.Operators(O.Params(**CFG1))
    u0 = init(ops, amp=1e-2)
    ref = O.run(ops, O.cold_state(u0), 20)
    plan = tc.Plan(**CFG1, precision=tc.TC_MIXED)
    st = tc.State(plan, dev(u0))
    plan.step(st, 20)
    got = host(st.u)
    pert = np.ones(got.shape, bool)
    pert[:, :, 0, ops.prm.K] = False
    e_pert = np.linalg.norm(got[pert] - ref.u[pert]) / np.linalg.norm(ref.u[pert])
    assert e_pert <= 1e-5, e_pert
    assert rel(got, ref.u) <= 1e-8


def test_mixed_split_path_stencils():
    """The mixed form's per-stage steps 2-5 (radial stencils in double-FP32) against its fused
    kernel (FP64 stencils) and the oracle, over 20 steps; the wall row N_r = 9 < 32 and the
    tile edges (N_r = 37) included."""
    for cfg in (CFG1, dict(CFG1, N_r=37), dict(CFG1, N_r=9, M=4, K=6)):
        ops = O.Operators(O.Params(**cfg))
        u0 = init(ops, amp=1e-2)
        ref = O.run(ops, O.cold_state(u0), 20)
        outs = []
        for split in (1, -1):
            plan = tc.Plan(**cfg, precision=tc.TC_MIXED, pc_split=split)
            st = tc.State(plan, dev(u0))
            plan.step(st, 20)
            outs.append([host(getattr(st, k)) for k in ("u", "u_prev", "N_prev", "p")])
        for a, b in zip(*outs):
            assert rel(a, b) <= 1e-11, (cfg["N_r"], rel(a, b))
        assert rel(outs[0][0], ref.u) <= 1e-8


def test_mixed_at_the_bench_workload_against_oracle():
    """The mixed form at the bench workload (N_r = 64, m = -32..32, k = -64..64, Re_i = 1000,
    Taylor-vortex-like start) over 20 steps at the largest stable dt (the stated 5e-4 halved
    until 200 FP64 steps stay bounded: 1.5625e-5), against the oracle's FP64 steps: the
    errors of the velocity perturbation, the velocity, the two torques and the largest
    divergence."""
    cfg = {**CFG2, "dt": 5e-4 / 32}
    ops = O.Operators(O.Params(**cfg))
    u0 = init(ops, kind="taylor", amp=1e-2)
    ref = O.run(ops, O.cold_state(u0), 20)
    plan = tc.Plan(**cfg, precision=tc.TC_MIXED)
    st = tc.State(plan, dev(u0))
    plan.step(st, 20)
    got = host(st.u)
    base = I.base_state(ops.r, ops.prm.M, ops.prm.K, 0.5, 1000.0, 0.0)
    d = plan.diagnostics(st.u)
    Ti, To = O.torque(ops, ref.u)
    err = {"velocity_perturbation": rel(got - base, ref.u - base), "velocity": rel(got, ref.u),
           "torque_inner": abs(d.torque_inner / Ti - 1), "torque_outer": abs(d.torque_outer / To - 1),
           "max_div": abs(d.max_div / O.max_divergence(ops, ref.u) - 1)}
    print("mixed vs oracle, bench workload, 20 steps:", err)
    assert err["velocity_perturbation"] <= 1e-6 and err["velocity"] <= 1e-8, err
    assert err["torque_inner"] <= 1e-7 and err["torque_outer"] <= 1e-7, err
    assert err["max_div"] <= 1e-5, err


# ------------------------------------------------------------------ tc_plan_set
@pytest.mark.parametrize("key,value,kw", [(tc.TC_SET_PRECISION, tc.TC_MIXED, dict(precision=tc.TC_MIXED)),
                                          (tc.TC_SET_PC_SPLIT, 1, dict(pc_split=1)),
                                          (tc.TC_SET_ALPHA, 0.7, dict(alpha=0.7)),
                                          (tc.TC_SET_P_Z, 36, dict(P_z=36))])
def test_plan_set_gives_the_created_plan(key, value, kw):
    """A setting changed by tc_plan_set before the first compute call gives the same steps,
    bit for bit, as a plan created with that setting; after a compute call it is refused."""
    cfg = dict(N_r=24, M=8, K=12, m_p=1, eta=0.5, Re_i=100.0, Re_o=0.0, L_z=LZ, dt=1e-4)
    ops = O.Operators(O.Params(**cfg))
    u0 = init(ops, kind="broadband", amp=1e-2, seed=9)
    out = []
    for plan in (tc.Plan(**cfg, **kw), tc.Plan(**cfg)):
        if len(out):
            plan.set(key, value)
        st = tc.State(plan, dev(u0))
        plan.step(st, 4)
        out.append([host(getattr(st, k)) for k in ("u", "u_prev", "N_prev", "p")])
        with pytest.raises(tc.TCError) as e:
            plan.set(key, value)
        assert e.value.status == tc.TC_ERR_STATE
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("T,prec", [(4, tc.TC_FP64), (16, tc.TC_FP64), (4, tc.TC_MIXED), (16, tc.TC_MIXED)])
def test_pc_modes_bit_identical(T, prec):
    """The fused steps-2-5 kernel with 4 or 16 modes per block (128 or 256 threads) gives the
    same state as the default 8, bit for bit: each mode's arithmetic is the same (the mixed
    form's double-FP32 stencils included)."""
    cfg = dict(N_r=32, M=12, K=16, m_p=1, eta=0.5, Re_i=100.0, Re_o=0.0, L_z=LZ, dt=1e-4)
    ops = O.Operators(O.Params(**cfg))
    u0 = init(ops, kind="broadband", amp=1e-2, seed=10)
    out = []
    for modes in (8, T):
        plan = tc.Plan(**cfg, pc_modes=modes, precision=prec)
        st = tc.State(plan, dev(u0))
        plan.step(st, 5)
        out.append([host(getattr(st, k)) for k in ("u", "u_prev", "N_prev", "p")])
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_step_host_matches_device_step():
    """tc_step_host (state in host memory, pinned or pageable) gives the device tc_step's
    result, and refuses device pointers where host memory is expected."""
    ops = O.Operators(O.Params(**CFG1))
    u0 = init(ops)
    plan = tc.Plan(**CFG1)
    ref = tc.State(plan, dev(u0))
    plan.step(ref, 3)
    want = {k: host(getattr(ref, k)) for k in ("u", "u_prev", "N_prev", "p")}
    plan.step(ref, 2)
    want2 = {k: host(getattr(ref, k)) for k in ("u", "p")}
    for pin in (True, False):
        h_in = {k: torch.from_numpy(v.copy()) for k, v in want.items()}
        if pin:
            h_in = {k: v.pin_memory() for k, v in h_in.items()}
        h_in["started"] = True
        h_out = {"u": torch.empty_like(h_in["u"]), "p": torch.empty_like(h_in["p"])}
        work = tc.State(plan, dev(u0))
        plan.step_host(work, h_in, h_out, 2)
        assert np.array_equal(h_out["u"].numpy(), want2["u"])
        assert np.array_equal(h_out["p"].numpy(), want2["p"])
        # a started state's p^i is not read (the update writes p^{i+1}): a NaN there changes nothing
        h_in["p"].fill_(float("nan"))
        h_out = {"u": torch.empty_like(h_in["u"]), "p": torch.empty_like(h_in["p"])}
        plan.step_host(tc.State(plan, dev(u0)), h_in, h_out, 2)
        assert np.array_equal(h_out["u"].numpy(), want2["u"])
        assert np.array_equal(h_out["p"].numpy(), want2["p"])
    # a cold state through host memory: the history is built on the device as tc_step does
    cold_ref = tc.State(plan, dev(u0))
    plan.step(cold_ref, 3)
    h_in = {"u": torch.from_numpy(u0.copy()), "u_prev": torch.zeros_like(torch.from_numpy(u0)),
            "N_prev": torch.zeros_like(torch.from_numpy(u0)), "p": torch.zeros(plan.scalar_shape(), dtype=torch.complex128),
            "started": False}
    h_out = {"u": torch.empty_like(h_in["u"])}
    plan.step_host(tc.State(plan, dev(u0)), h_in, h_out, 3)
    assert np.array_equal(h_out["u"].numpy(), host(cold_ref.u))
    bad = {k: getattr(ref, k) for k in ("u", "u_prev", "N_prev", "p")}   # device tensors
    with pytest.raises(tc.TCError):
        plan.step_host(tc.State(plan, dev(u0)), bad, {}, 1)


@pytest.mark.parametrize("prec", [tc.TC_FP64, tc.TC_MIXED])
def test_step_captured_in_a_cuda_graph(prec):
    """tc_step records into a CUDA graph (the mixed form's second-stream fork and join
    included), and replaying the graph gives the eager steps bit for bit."""
    ops = O.Operators(O.Params(**CFG1))
    plan = tc.Plan(**CFG1, precision=prec)
    u0 = dev(init(ops, amp=1e-2))
    a = tc.State(plan, u0)
    b = tc.State(plan, u0)
    plan.step(a, 1)
    plan.step(b, 1)
    plan.step(a, 3)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.step(b, 1)                      # recorded, not run
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for name in ("u", "u_prev", "N_prev", "p"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name
