"""Benchmark of the Taylor–Couette AB2BD2 time step (libtc on one GB300 per rank).

Workload (one "step" = one full AB2BD2 step, Sec. 3.2 steps 1-5, through the C ABI):
plain FP64 step at N_r = 64 radial nodes, m = -32..32, k = -64..64, 3/2-dealiased physical
grid 64 x 96 x 192, eta = 0.5, Re_i = 1000, outer cylinder at rest, dt = 5e-4, initial state
circular Couette flow plus a seeded Taylor-vortex-like perturbation (amp 1e-2).

Prints one JSON line.  ``--impl reference`` times the CPU oracle (the reference arm of this
benchmark) on the same workload on the host cores.  Under torchrun each rank advances its
own independent simulation (seed 42 + rank); no data-path collective.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# DRAM bytes (read + write) of one FP64 theta-pass launch at the bench workload, from ncu
# (58.44 MB read + 2.99 MB written; the H2 lines stay in L2)
THETA_TRAFFIC = 61.43e6
CFG2 = dict(N_r=64, M=32, K=64, m_p=1, eta=0.5, Re_i=1000.0, Re_o=0.0, L_z=2 * math.pi / 3.16, dt=5e-4)
# mid-size case for profiling (inputs larger than L2, a few GB on the device)
CFG_MID = dict(N_r=128, M=128, K=256, m_p=1, eta=0.5, Re_i=1000.0, Re_o=0.0, L_z=2 * math.pi / 3.16, dt=5e-4)
# N_r beyond the fused steps-2-5 kernel's shared memory, for profiling the per-stage kernels
CFG_SPLIT = dict(N_r=256, M=32, K=64, m_p=1, eta=0.5, Re_i=1000.0, Re_o=0.0, L_z=2 * math.pi / 3.16, dt=5e-4)
# adjoint workload: N_r = 96, m = -32..32, k = -64..64, Re_i = 2000, 200 steps, checkpoint every 20
CFG3 = dict(N_r=96, M=32, K=64, m_p=1, eta=0.5, Re_i=2000.0, Re_o=0.0, L_z=2 * math.pi / 3.16, dt=5e-4)
# mixed vs FP64 at the same size: quasi-Keplerian (Re_o = sqrt(eta) Re_i), 256 x 768 x 1536 grid
CFG4 = dict(N_r=256, M=256, K=512, m_p=1, eta=0.5, Re_i=1e4, Re_o=math.sqrt(0.5) * 1e4,
            L_z=2 * math.pi / 3.16, dt=1e-4)
WORKLOAD = ("FP64 AB2BD2 step: eta=0.5, Re_i=1000, Re_o=0, N_r=64 clustered nodes (alpha=0.5), "
            "m=-32..32 (m_p=1), k=-64..64 (L_z=2pi/3.16), phys grid 64x96x192, dt=5e-4, "
            "init Couette + Taylor-vortex-like perturbation amp 1e-2 (seed 42)")
METRIC = "time-steps/s (FP64 plain AB2BD2 step)"
L2_FLUSH_BYTES = 256 << 20


def gdof(cfg):
    return 3 * cfg["N_r"] * (2 * cfg["M"] + 1) * (2 * cfg["K"] + 1)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def replica_seed(rank):
    """Each rank advances its own independent simulation (weak scaling, no data exchange)."""
    return 42 + rank


def max_over_ranks(dist, value, device):
    """Max of a per-rank float over all ranks (the timed region is as slow as the slowest)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world, steps, max_ms):
    """Whole-job steps/s: all ranks' steps over the slowest rank's time."""
    return world * steps / (max_ms / 1e3)


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (getattr(self, "out", "") or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, v in enumerate(flags) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def theta_flops(cfg, Pt, Pz):
    """Algorithmic FP64 flops of one k_theta launch: 6 inverse and 1.5 forward complex
    transforms of length P_theta per (r, z) at 5 n log2 n, plus 25 flops of products per
    physical point."""
    n = Pt
    per_line = 5.0 * n * math.log2(n)
    return cfg["N_r"] * Pz * (7.5 * per_line + 25.0 * n)


def zpass_flops(cfg, Pz, lines):
    return cfg["N_r"] * (cfg["M"] + 1) * lines * 5.0 * Pz * math.log2(Pz)


def hbm_peak_gbs():
    """Measured HBM copy bandwidth (MEASURED_PEAKS.json), else the recipe's fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# FP64 peak from unit counts and clock: 152 SMs x 2 DFMA/clk/SM (ncu peak_sustained of
# sm__sass_thread_inst_executed_op_dfma_pred_on) x 2 flop x 2.07 GHz
FP64_PEAK = 152 * 2 * 2 * 2.07e9


def kernel_rooflines(cfg, prof):
    """Every traced kernel at this workload: algorithmic bytes (inputs read once, outputs
    written once) and, for the FP64 transforms, algorithmic flops; the fraction of the
    measured HBM bandwidth and of the FP64 peak, and the roof that binds."""
    N, M, K = cfg["N_r"], cfg["M"], cfg["K"]
    Pt, Pz = 3 * M, 3 * K
    S = N * (M + 1) * (2 * K + 1)
    H = N * (M + 1) * Pz
    fac = 4 * N * (M + 1) * (K + 1) * (13 * 8 + 1)        # 4 factor sets, 13 doubles + pivot per row
    state_rw = (4 * 3 * S + S) * 16 + (3 * 3 * S + S) * 16   # N, N_prev, u, u_prev, p in; u, u_prev, N_prev, p out
    table = {
        "k_zinv": (3 * S * 16 + 9 * H * 16, zpass_flops(cfg, Pz, 9) + 36.0 * 3 * S, "alu"),   # + 9-tap stencil
        "k_theta": (9 * H * 16 + 3 * H * 16, theta_flops(cfg, Pt, Pz), "alu"),
        "k_zfwd": (3 * H * 16 + 3 * S * 16, zpass_flops(cfg, Pz, 3), "alu"),
        "k_pc": (fac + state_rw, None, "alu"),
        "k_prep_f32": (3 * S * 16 + 6 * S * 8, None, "hbm"),
        "k_zinv_f32": (6 * S * 8 + 9 * H * 8, None, "hbm"),
        "k_theta_f32": (9 * H * 8 + 3 * H * 8, None, "hbm"),
        "k_zfwd_f32": (3 * H * 8 + 3 * S * 16 + 3 * S * 16, None, "hbm"),
        # the mean mode of N by double-FP32 Parseval sums: u read once (~1250 FP32 operations
        # per (row, mode) make it bound by issue, not bytes)
        "k_mean00_f32": (3 * S * 16, None, "alu"),
    }
    hbm, src = hbm_peak_gbs()
    out = {}
    for name, (n, ms) in prof.items():
        if name not in table or n == 0:
            continue
        t = ms / n / 1e3
        b, f, bound = table[name]
        e = {"ms": ms / n, "bytes": b, "hbm_frac": b / t / (hbm * 1e9), "bound": bound}
        if f:
            e["flops"] = f
            e["fp64_frac"] = f / t / FP64_PEAK
        out[name] = e
    return {"kernels": out, "hbm_peak_gbs": hbm, "hbm_peak_source": src,
            "fp64_peak_tflops": FP64_PEAK / 1e12,
            "note": "k_pc: DP instructions ~380 per (row, mode) in its two-partition form (ncu: 103 M per launch at the bench size), bound by FP64 issue (16 cycles per warp instruction)"}


def cufft_comparison(torch, cfg, dev, reps=20):
    """cuFFT (through torch.fft) on the batch shapes of the four transform passes, FP64 and
    FP32, as a comparison only.  The hand-written passes also apply the radial stencil, the
    products, the real-pair packing and the layout changes; cuFFT here does transforms only,
    each in its natural contiguous layout."""
    N, M, K = cfg["N_r"], cfg["M"], cfg["K"]
    Pt, Pz = 3 * M, 3 * K
    out = {"workload": f"N_r={N}, M={M}, K={K}, P_theta={Pt}, P_z={Pz}",
           "batches": {"z_inverse": f"{9 * N * (M + 1)} complex lines of {Pz}",
                       "theta_inverse": f"{12 * N * Pz} C2R lines of {Pt} from {M + 1} modes",
                       "theta_forward": f"{3 * N * Pz} R2C lines of {Pt}",
                       "z_forward": f"{3 * N * (M + 1)} complex lines of {Pz}"}}
    for name, tc_, tr_ in (("fp64", torch.complex128, torch.float64), ("fp32", torch.complex64, torch.float32)):
        g = torch.Generator(device=dev).manual_seed(1)
        zin = torch.randn(9 * N * (M + 1), Pz, dtype=tc_, device=dev, generator=g)
        thin = torch.randn(12 * N * Pz, M + 1, dtype=tc_, device=dev, generator=g)
        thfw = torch.randn(3 * N * Pz, Pt, dtype=tr_, device=dev, generator=g)
        zfw = torch.randn(3 * N * (M + 1), Pz, dtype=tc_, device=dev, generator=g)
        ops = {"z_inverse": lambda: torch.fft.ifft(zin, dim=-1),
               "theta_inverse": lambda: torch.fft.irfft(thin, n=Pt, dim=-1),
               "theta_forward": lambda: torch.fft.rfft(thfw, dim=-1),
               "z_forward": lambda: torch.fft.fft(zfw, dim=-1)}
        r = {}
        for k, fn in ops.items():
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            r[k + "_ms"] = e0.elapsed_time(e1) / reps
        r["total_ms"] = sum(r.values())
        out[name] = r
        del zin, thin, thfw, zfw
        torch.cuda.empty_cache()
    return out


def tensor_dft_comparison(torch, dev, reps=3):
    """The theta stage of the nonlinear term as dense DFT products on the tensor cores, timed
    with cuBLAS (torch.matmul) as a comparison only, against the hand-written FP32 theta pass.
    The inverse stage is one real product [P_theta x 2(M+1)] x [2(M+1) x 12 N_r P_z] (cos and
    sin columns of the stored modes, 12 physical fields per (r, z)); the forward stage
    [2(M+1) x P_theta] x [P_theta x 3 N_r P_z].  The FP32 error budget of the mixed form needs
    split operands: with FP16 pairs (hi + lo, about 22 bits) three products per stage
    (hi hi, hi lo, lo hi), accumulated in FP32.  Counted here: the products alone, 16-bit
    outputs, no splitting, no assembly and no pointwise products, so the sum is a lower bound
    for any DFT-as-GEMM theta stage."""
    out = {}
    for name, (N_r, M, K) in (("N_r=64, M=32, K=64", (64, 32, 64)), ("N_r=256, M=256, K=512", (256, 256, 512)),
                              ("N_r=384, M=384, K=768", (384, 384, 768))):
        Pt, Pz = 3 * M, 3 * K
        kk = 2 * (M + 1)
        Li, Lf = 12 * N_r * Pz, 3 * N_r * Pz
        g = torch.Generator(device=dev).manual_seed(3)
        Ai = torch.randn(Pt, kk, device=dev, dtype=torch.float16, generator=g)
        Bi = torch.randn(kk, Li, device=dev, dtype=torch.float16, generator=g)
        Af = torch.randn(kk, Pt, device=dev, dtype=torch.float16, generator=g)
        Bf = torch.randn(Pt, Lf, device=dev, dtype=torch.float16, generator=g)
        Ci = torch.empty(Pt, Li, device=dev, dtype=torch.float16)
        Cf = torch.empty(kk, Lf, device=dev, dtype=torch.float16)
        torch.matmul(Ai, Bi, out=Ci)
        torch.matmul(Af, Bf, out=Cf)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        for _ in range(reps):
            torch.matmul(Ai, Bi, out=Ci)
        ev[1].record()
        for _ in range(reps):
            torch.matmul(Af, Bf, out=Cf)
        ev[2].record()
        torch.cuda.synchronize()
        ti, tf = ev[0].elapsed_time(ev[1]) / reps, ev[1].elapsed_time(ev[2]) / reps
        fl = 2.0 * (Pt * kk * Li + kk * Pt * Lf)
        out[name] = {"inverse_gemm_ms": ti, "forward_gemm_ms": tf,
                     "tflops": fl / ((ti + tf) / 1e3) / 1e12,
                     "split_fp16_pairs_lower_bound_ms": 3 * (ti + tf)}
        del Ai, Bi, Af, Bf, Ci, Cf
        torch.cuda.empty_cache()
    return out


def stable_dt(tc, torch, cfg, u0_t, dev, nsteps=200):
    """Stated dt halved until nsteps FP64 steps stay finite with < 10x energy growth."""
    dt = cfg["dt"]
    for _ in range(12):
        plan = tc.Plan(**{**cfg, "dt": dt}, device=dev)
        st = tc.State(plan, u0_t.to(dev))
        e0 = plan.diagnostics(st.u).energy
        plan.step(st, nsteps)
        d = plan.diagnostics(st.u)
        del plan, st
        if d.finite and d.energy < 10.0 * e0:
            return dt
        dt /= 2.0
    return dt


def adjoint_ratio(tc, torch, I, dev):
    """Cost of the checkpointed adjoint of 200 steps (N_r = 96) against the forward run."""
    from paper_1311_2481_gb300 import adjoint as A
    cfg = CFG3
    probe = tc.Plan(**cfg, device=dev)
    r = probe.nodes()
    del probe
    u0 = torch.from_numpy(I.initial_state(r, cfg["M"], cfg["K"], 1, cfg["L_z"], cfg["eta"], cfg["Re_i"],
                                          cfg["Re_o"], kind="box", amp=1e-4, seed=42))
    dt = stable_dt(tc, torch, cfg, u0, dev)
    plan = tc.Plan(**{**cfg, "dt": dt}, device=dev)
    n, C = 200, 20
    x = u0.to(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    xw = x.clone().requires_grad_(True)                       # warm-up: forward and backward
    A.final_energy(xw, plan, 2 * C, checkpoint=C).backward()
    torch.cuda.synchronize()
    del xw
    ev[0].record()
    with torch.no_grad():
        J0 = A.final_energy(x, plan, n, checkpoint=C)
    ev[1].record()
    xg = x.clone().requires_grad_(True)
    ev[2].record()
    J = A.final_energy(xg, plan, n, checkpoint=C)
    J.backward()
    ev[3].record()
    torch.cuda.synchronize()
    t_f = ev[0].elapsed_time(ev[1])
    t_fb = ev[2].elapsed_time(ev[3])
    g = xg.grad
    return {"workload": "N_r=96, m=-32..32, k=-64..64, Re_i=2000, 200 steps, checkpoint every 20, "
                        "J = final perturbation energy, init amp 1e-4 (seed 42)",
            "dt": dt, "forward_ms": t_f, "forward_plus_adjoint_ms": t_fb,
            "backward_ms_per_step": (t_fb - t_f) / n, "forward_ms_per_step": t_f / n,
            # backward (segment recomputation + adjoint steps) over the plain forward run
            "adjoint_to_forward_ratio": (t_fb - t_f) / t_f, "J": float(J0),
            "grad_finite": bool(torch.isfinite(torch.view_as_real(g)).all())}


def cfl_dt(cfg, c=0.25):
    """The stated dt, capped by the azimuthal advection limit of the explicit AB2 term:
    dt * Omega_max * M * m_p <= c, with Omega_max the larger wall angular velocity
    (|Re_i| / r_i, |Re_o| / r_o in viscous units)."""
    r_i = cfg["eta"] / (1.0 - cfg["eta"])
    r_o = 1.0 / (1.0 - cfg["eta"])
    om = max(abs(cfg["Re_i"]) / r_i, abs(cfg["Re_o"]) / r_o)
    return min(cfg["dt"], c / (om * cfg["M"] * cfg["m_p"]))


def _rel(a, b, torch):
    return float(torch.linalg.vector_norm(b - a) / torch.linalg.vector_norm(a))


def large_mixed(tc, torch, I, dev, steps=4, err_steps=100):
    """FP64 plain vs mixed step at N_r = 256, m = -256..256, k = -512..512 (same size), with
    the mixed form's error against the FP64 GPU step after the workload's 100 steps from the
    same initial state (the error against the oracle, at this N_r with fewer modes, is a test)."""
    cfg = {**CFG4, "dt": cfl_dt(CFG4)}
    out = {"workload": "quasi-Keplerian eta=0.5, Re_i=1e4, Re_o=sqrt(eta) Re_i, N_r=256, m=-256..256, "
                       "k=-512..512, phys 256x768x1536, broadband amp 0.05 (seed 42)",
           "gdof": gdof(cfg), "dt_stated": CFG4["dt"], "dt": cfg["dt"]}
    res, keep = {}, {}
    u0h = None
    for name, prec in (("fp64", tc.TC_FP64), ("mixed", tc.TC_MIXED)):
        plan = tc.Plan(**cfg, precision=prec, device=dev)
        r = plan.nodes()
        if u0h is None:
            u0h = torch.from_numpy(I.initial_state(r, cfg["M"], cfg["K"], 1, cfg["L_z"], cfg["eta"],
                                                   cfg["Re_i"], cfg["Re_o"], kind="broadband", amp=0.05,
                                                   seed=42))
        u0 = u0h.to(dev)
        N0 = plan.nonlinear(u0)
        st = tc.State(plan, u0)
        e_start = plan.diagnostics(st.u).energy
        plan.step(st, 2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.step(st, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        plan.profile(True)
        plan.step(st, 1)
        torch.cuda.synchronize()
        kern = {k: v[1] for k, v in plan.profile_read().items()}
        plan.profile(False)
        d_timed = plan.diagnostics(st.u)
        # the error run: err_steps steps from the initial state
        st = tc.State(plan, u0)
        del u0
        plan.step(st, err_steps)
        d = plan.diagnostics(st.u)
        res[name] = ms
        keep[name] = (N0, st.u.clone(), d)
        out[name] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "gdof_steps_per_s": gdof(cfg) / ms / 1e6,
                     "kernels_ms": kern, "state_finite": bool(d_timed.finite and d.finite),
                     "energy_growth": d_timed.energy / e_start,
                     f"energy_growth_{err_steps}_steps": d.energy / e_start}
        del plan, st
        torch.cuda.empty_cache()
    out["mixed_speedup_vs_fp64"] = res["fp64"] / res["mixed"]
    (Na, ua, da), (Nb, ub, db) = keep["fp64"], keep["mixed"]
    base = torch.from_numpy(I.base_state(r, cfg["M"], cfg["K"], cfg["eta"], cfg["Re_i"], cfg["Re_o"])).to(dev)
    out["mixed_error"] = {
        "after_steps": err_steps, "dt": cfg["dt"], "against": "FP64 CUDA step",
        "rel_err_nonlinear_term_initial_state": _rel(Na, Nb, torch),
        "rel_err_velocity_perturbation": _rel(ua - base, ub - base, torch),
        "rel_err_velocity": _rel(ua, ub, torch),
        "rel_err_torque_inner": abs(db.torque_inner / da.torque_inner - 1),
        "rel_err_torque_outer": abs(db.torque_outer / da.torque_outer - 1),
        "max_div_fp64": da.max_div, "max_div_mixed": db.max_div}
    del keep, base
    torch.cuda.empty_cache()
    return out


# the paper's SMALL timing grid (n_r, n_theta, n_z) = (32, 384, 640): m = -192..192,
# k = -320..320; P_z = 972 = 2^2 3^5 >= 3K + 1 (the 3/2 grid 960 has a factor 5)
CFG_SMALL = dict(N_r=32, M=192, K=320, m_p=1, eta=0.5, Re_i=1e3, Re_o=0.0, L_z=2 * math.pi / 3.16,
                 dt=5e-4, P_theta=576, P_z=972)
# its best time in the paper: 0.104 s per step on 32 x 20 Xeon cores (Table of the SMALL run)
PAPER_SMALL_S_PER_STEP = 0.104


def paper_small(tc, torch, I, dev, steps=10):
    """FP64 and mixed step at the paper's SMALL grid, beside its best CPU time (context)."""
    cfg = {**CFG_SMALL, "dt": cfl_dt(CFG_SMALL)}
    out = {"workload": "paper SMALL grid: N_r=32, m=-192..192, k=-320..320, phys 32x576x972, eta=0.5, "
                       "Re_i=1000, broadband amp 0.01 (seed 42)",
           "gdof": gdof(cfg), "dt": cfg["dt"],
           "paper_best_s_per_step": PAPER_SMALL_S_PER_STEP, "paper_cores": 640}
    for name, prec in (("fp64", tc.TC_FP64), ("mixed", tc.TC_MIXED)):
        plan = tc.Plan(**cfg, precision=prec, no_adjoint=True, device=dev)
        r = plan.nodes()
        u0 = torch.from_numpy(I.initial_state(r, cfg["M"], cfg["K"], 1, cfg["L_z"], cfg["eta"], cfg["Re_i"],
                                              cfg["Re_o"], kind="broadband", amp=0.01, seed=42)).to(dev)
        st = tc.State(plan, u0)
        del u0
        plan.step(st, 3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.step(st, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        d = plan.diagnostics(st.u)
        out[name] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "gdof_steps_per_s": gdof(cfg) / ms / 1e6,
                     "vs_paper_best": PAPER_SMALL_S_PER_STEP * 1e3 / ms, "state_finite": bool(d.finite)}
        del plan, st
        torch.cuda.empty_cache()
    return out


# largest single-GPU workload: N_r = 384, m = -384..384, k = -768..768, grid 384 x 1152 x 2304
CFG5 = dict(N_r=384, M=384, K=768, m_p=1, eta=0.5, Re_i=3e4, Re_o=math.sqrt(0.5) * 3e4,
            L_z=2 * math.pi / 3.16, dt=5e-5)


def largest(tc, torch, I, dev, steps=3, err_steps=100):
    """FP64 and mixed step at the largest workload (no adjoint workspace), one after the other
    (the two plans do not fit the device together), and the mixed form's error against the
    FP64 step after the workload's 100 steps from the same initial state.  The FP64 plan
    stages its transforms by radial slab."""
    cfg = {**CFG5, "dt": cfl_dt(CFG5)}
    out = {"workload": "quasi-Keplerian eta=0.5, Re_i=3e4, Re_o=sqrt(eta) Re_i, N_r=384, m=-384..384, "
                       "k=-768..768, phys 384x1152x2304, broadband amp 0.05 (seed 42)",
           "gdof": gdof(cfg), "dt_stated": CFG5["dt"], "dt": cfg["dt"]}
    u0h, keep = None, {}
    for name, prec in (("fp64", tc.TC_FP64), ("mixed", tc.TC_MIXED)):
        torch.cuda.reset_peak_memory_stats()
        t0 = time.perf_counter()
        plan = tc.Plan(**cfg, precision=prec, no_adjoint=True, device=dev)
        t_plan = time.perf_counter() - t0
        r = plan.nodes()
        if u0h is None:
            u0h = torch.from_numpy(I.initial_state(r, cfg["M"], cfg["K"], 1, cfg["L_z"], cfg["eta"], cfg["Re_i"],
                                                   cfg["Re_o"], kind="broadband", amp=0.05, seed=42))
        st = tc.State(plan, u0h.to(dev))
        e_start = plan.diagnostics(st.u).energy
        plan.step(st, 2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.step(st, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        plan.profile(True)
        plan.step(st, 1)
        torch.cuda.synchronize()
        kern = {k: v[1] for k, v in plan.profile_read().items()}
        plan.profile(False)
        mem = torch.cuda.max_memory_allocated() / 1e9
        # the error run: err_steps steps from the initial state
        st = tc.State(plan, u0h.to(dev))
        plan.step(st, err_steps)
        d = plan.diagnostics(st.u)
        keep[name] = (st.u.to("cpu"), d)
        out[name] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "gdof_steps_per_s": gdof(cfg) / ms / 1e6,
                     "kernels_ms": kern, "plan_create_s": t_plan, "torch_device_memory_gb": mem,
                     "state_finite": bool(d.finite), f"energy_growth_{err_steps}_steps": d.energy / e_start}
        del plan, st
        torch.cuda.empty_cache()
    out["mixed_speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    (ua, da), (ub, db) = keep["fp64"], keep["mixed"]
    base = torch.from_numpy(I.base_state(r, cfg["M"], cfg["K"], cfg["eta"], cfg["Re_i"], cfg["Re_o"]))
    ua, ub = ua.to(dev), ub.to(dev)
    bd = base.to(dev)
    del base
    out["mixed_error"] = {
        "after_steps": err_steps, "dt": cfg["dt"], "against": "FP64 CUDA step",
        "rel_err_velocity_perturbation": _rel(ua - bd, ub - bd, torch),
        "rel_err_velocity": _rel(ua, ub, torch),
        "rel_err_torque_inner": abs(db.torque_inner / da.torque_inner - 1),
        "rel_err_torque_outer": abs(db.torque_outer / da.torque_outer - 1),
        "max_div_fp64": da.max_div, "max_div_mixed": db.max_div}
    del keep, ua, ub, bd
    torch.cuda.empty_cache()
    return out


def _free_device_bytes(torch):
    """Device memory free for new tensors: the driver's free bytes plus torch's unused cache."""
    free, _ = torch.cuda.mem_get_info()
    return free + torch.cuda.memory_reserved() - torch.cuda.memory_allocated()


def config5_adjoint(tc, torch, I, dev, n_total=100, n_adj=50, checkpoint=17):
    """The largest workload as stated: the quasi-Keplerian flow at N_r = 384, M = 384,
    K = 768 in the mixed form for n_total steps, and the gradient of the final perturbation
    energy with respect to the state (u, u_prev, N_prev) n_adj steps before the end, through
    the FP64 adjoint (adjoint.state_gradient): checkpoints every `checkpoint` steps in pinned
    host memory, the segments reversed through as many device copies of u as fit.  Then a
    central difference of J along the gradient's u part, through the mixed forward."""
    from paper_1311_2481_gb300 import adjoint as A
    cfg = {**CFG5, "dt": cfl_dt(CFG5)}
    torch.cuda.reset_peak_memory_stats()
    t0 = time.perf_counter()
    plan = tc.Plan(**cfg, precision=tc.TC_MIXED, device=dev)
    t_plan = time.perf_counter() - t0
    r = plan.nodes()
    u0 = torch.from_numpy(I.initial_state(r, cfg["M"], cfg["K"], 1, cfg["L_z"], cfg["eta"], cfg["Re_i"],
                                          cfg["Re_o"], kind="broadband", amp=0.05, seed=42)).to(dev)
    st = tc.State(plan, u0)
    del u0
    field = st.u.numel() * st.u.element_size()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    plan.step(st, n_total - n_adj)
    ev[1].record()
    torch.cuda.synchronize()
    # device copies of u for the segment reversal: what is left after the gradient's three fields
    slots = int(max(1, min(checkpoint, (_free_device_bytes(torch) - 3 * field - (6 << 30)) // field)))
    ev[2].record()
    J, bar = A.state_gradient(plan, st, n_adj, checkpoint=checkpoint, slots=slots, spill=True)
    ev[3].record()
    torch.cuda.synchronize()
    t_fwd = ev[0].elapsed_time(ev[1]) / (n_total - n_adj)
    t_sg = ev[2].elapsed_time(ev[3])
    back = (t_sg - t_fwd * n_adj) / n_adj
    finite = all(bool(torch.isfinite(torch.view_as_real(t)).all()) for t in (bar.u, bar.u_prev, bar.N_prev))
    mem = torch.cuda.max_memory_allocated() / 1e9     # torch's tensors (the plan's factors are not among them)
    free, total = torch.cuda.mem_get_info()
    used = (total - free) / 1e9                       # the whole device, torch's cache at its peak included
    # central difference of J(u + h g_u) along g_u = dJ/du, against <g_u, g_u>
    g = bar.u
    del bar
    s_u, s_up, s_N = st.u.clone(), st.u_prev.clone(), st.N_prev.clone()
    gn2 = float(torch.sum(torch.view_as_real(g) ** 2))
    h = 1e-2 * J / gn2        # J changes by about 1% of itself: above the mixed form's rounding
    Js = []
    for sg in (1.0, -1.0):
        st.u.copy_(s_u)
        st.u.add_(g, alpha=sg * h)
        st.u_prev.copy_(s_up)
        st.N_prev.copy_(s_N)
        st.started = True
        plan.step(st, n_adj)
        Js.append(plan.diagnostics(st.u).energy)
    fd = (Js[0] - Js[1]) / (2 * h)
    return {"workload": f"quasi-Keplerian eta=0.5, Re_i=3e4, Re_o=sqrt(eta) Re_i, N_r=384, m=-384..384, "
                        f"k=-768..768, broadband amp 0.05 (seed 42), mixed form, {n_total} steps; "
                        f"FP64 adjoint of the last {n_adj} (gradient w.r.t. the state {n_adj} steps "
                        f"before the end), checkpoint every {checkpoint} in pinned host memory",
            "dt_stated": CFG5["dt"], "dt": cfg["dt"], "plan_create_s": t_plan,
            "forward_ms_per_step": t_fwd, "state_gradient_ms": t_sg, "backward_ms_per_step": back,
            "adjoint_to_forward_ratio": back / t_fwd, "J": J, "grad_finite": finite,
            "u_slots": slots, "host_checkpoint_gb": -(-n_adj // checkpoint) * 3 * field / 1e9,
            "device_memory_gb": mem, "device_used_gb": used,
            "fd_along_grad": fd, "grad_norm_sq": gn2, "fd_rel_diff": abs(fd - gn2) / gn2,
            "fd_note": "central difference of J through the mixed forward vs <g, g> from the FP64 adjoint"}


def config5_dot_product(tc, torch, I, dev, h_scale=1.0):
    """Dot-product test of the FP64 adjoint step at the largest workload: with s a started
    FP64 state, x and y seeded directions (x scaled to the state's norms), compares
    <y, dF(s)[x]> with <F^T y, x>.  dF(s)[x] = (F(s + x) - F(s - x)) / 2 exactly up to
    rounding, F being quadratic in the state.  s and x are kept in pinned host memory."""
    cfg = {**CFG5, "dt": cfl_dt(CFG5)}
    torch.cuda.reset_peak_memory_stats()
    plan = tc.Plan(**cfg, device=dev)
    r = plan.nodes()
    u0 = torch.from_numpy(I.initial_state(r, cfg["M"], cfg["K"], 1, cfg["L_z"], cfg["eta"], cfg["Re_i"],
                                          cfg["Re_o"], kind="broadband", amp=0.05, seed=42)).to(dev)
    st = tc.State(plan, u0)
    del u0
    plan.step(st, 1)
    names = ("u", "u_prev", "N_prev")
    pin = lambda t: t.to("cpu", non_blocking=False).pin_memory()   # noqa: E731
    s = [pin(getattr(st, k)) for k in names]
    gen = torch.Generator(device=dev)
    x = []
    for i, k in enumerate(names):
        gen.manual_seed(1000 + i)
        v = torch.randn(st.u.shape, dtype=torch.complex128, device=dev, generator=gen)
        v.mul_(h_scale * float(torch.linalg.vector_norm(getattr(st, k))) / float(torch.linalg.vector_norm(v)))
        x.append(pin(v))
        del v
    # F(s + x) -> kept on the device; F(s - x) in st
    fp = []
    for sg in (1.0, -1.0):
        for k, a, b in zip(names, s, x):
            t = getattr(st, k)
            t.copy_(a)
            t.add_(b.to(dev), alpha=sg)
        st.started = True
        plan.step(st, 1)
        if sg > 0:
            fp = [getattr(st, k).clone() for k in names]
    tl = [(a - getattr(st, k)) / 2 for a, k in zip(fp, names)]   # dF(s)[x]
    del fp
    ys = []
    for i in range(3):
        gen.manual_seed(2000 + i)
        ys.append(torch.randn(st.u.shape, dtype=torch.complex128, device=dev, generator=gen))
    lhs = sum(float(torch.sum(torch.view_as_real(a) * torch.view_as_real(b))) for a, b in zip(ys, tl))
    del tl
    for k, a in zip(names, s):
        getattr(st, k).copy_(a)
    st.started = True
    bar = tc.StateBar(*ys)
    plan.adjoint_step(st, bar)
    rhs = sum(float(torch.sum(torch.view_as_real(getattr(bar, k)) * torch.view_as_real(b.to(dev))))
              for k, b in zip(names, x))
    # kernel times of one FP64 adjoint step and one FP64 step at this size (CUDA events)
    plan.profile(True)
    plan.adjoint_step(st, bar)
    torch.cuda.synchronize()
    adj = {k: v[1] for k, v in plan.profile_read().items()}
    plan.profile(False)
    plan.profile(True)
    plan.step(st, 1)
    torch.cuda.synchronize()
    fwd = {k: v[1] for k, v in plan.profile_read().items()}
    plan.profile(False)
    return {"workload": "N_r=384, m=-384..384, k=-768..768, FP64 step and adjoint step at a started "
                        "state (one step from the broadband initial state)",
            "lhs": lhs, "rhs": rhs, "rel_diff": abs(lhs - rhs) / abs(rhs),
            "adjoint_step_kernels_ms": adj, "adjoint_step_ms": sum(adj.values()),
            "fp64_step_kernels_ms": fwd, "fp64_step_ms": sum(fwd.values()),
            "device_memory_gb": torch.cuda.max_memory_allocated() / 1e9}


# profiling case of the long-line transforms: P_theta = 1152, P_z = 192
CFG_LONG = dict(N_r=32, M=384, K=64, m_p=1, eta=0.5, Re_i=1000.0, Re_o=0.0, L_z=2 * math.pi / 3.16, dt=5e-6)


def run_adjoint_case(args):
    """--workload adjoint: K timed FP64 adjoint steps (tc_adjoint_step) at a profiling size,
    after W untimed ones, one JSON line with the per-kernel times (CUDA events)."""
    import torch
    from paper_1311_2481_gb300 import build as B
    from paper_1311_2481_gb300 import inputs as I
    from paper_1311_2481_gb300 import tc
    B.build()
    cfg = {"mid": CFG_MID, "split": CFG_SPLIT, "long": CFG_LONG}.get(args.size, CFG2)
    plan = tc.Plan(**cfg, device="cuda:0")
    r = plan.nodes()
    u0 = torch.from_numpy(I.initial_state(r, cfg["M"], cfg["K"], 1, cfg["L_z"], cfg["eta"], cfg["Re_i"],
                                          cfg["Re_o"], kind="broadband", amp=1e-2, seed=42)).cuda()
    st = tc.State(plan, u0)
    plan.step(st, 1)
    bar = tc.StateBar(u0.clone(), u0.clone(), u0.clone())
    for _ in range(args.warmup):
        plan.adjoint_step(st, bar)
    torch.cuda.synchronize()
    plan.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        plan.adjoint_step(st, bar)
    e1.record()
    torch.cuda.synchronize()
    kern = {k: v[1] / args.steps for k, v in plan.profile_read().items()}
    plan.profile(False)
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"metric": "FP64 adjoint steps/s (profiling case)", "value": 1e3 / ms, "unit": "steps/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": f"FP64 adjoint step at N_r={cfg['N_r']}, M={cfg['M']}, "
                                             f"K={cfg['K']}, P_theta={3 * cfg['M']}, P_z={3 * cfg['K']}"},
                      "kernels_ms_per_step": kern}), flush=True)


def run_ours(args):
    import torch
    from paper_1311_2481_gb300 import build as B
    from paper_1311_2481_gb300 import inputs as I
    from paper_1311_2481_gb300 import tc

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    if rank == 0 or world == 1:
        B.build()
    if dist:
        dist.barrier()
    cfg = {"mid": CFG_MID, "split": CFG_SPLIT}.get(args.size, CFG2)
    main_is_bench = args.size == "bench" and args.workload == "fp64"
    prec = tc.TC_MIXED if args.workload == "mixed" else tc.TC_FP64
    plan = tc.Plan(**cfg, precision=prec, no_adjoint=True, device=f"cuda:{local}")
    r = plan.nodes()
    u0 = I.initial_state(r, cfg["M"], cfg["K"], cfg["m_p"], cfg["L_z"], cfg["eta"], cfg["Re_i"],
                         cfg["Re_o"], kind="taylor", amp=1e-2, seed=replica_seed(rank))
    u0_t = torch.from_numpy(u0)
    st = tc.State(plan, u0_t.cuda())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def gpu_spin():
        # about 100 us of untimed device work before each step's start event, so the events
        # time the step's kernels and not the host's launch latency (the first call of a
        # timed loop enqueued in ~55 us, longer than the L2 flush)
        if hasattr(torch.cuda, "_sleep"):
            torch.cuda._sleep(200_000)
        else:
            flush.fill_(1.0)
            flush.fill_(2.0)

    # At dt = 5e-4 the explicit advection exceeds its stability limit (azimuthal CFL ~ 7.6):
    # from the initial state the energy grows 60x in 9 steps and overflows at step 19.  Every
    # CHUNK steps the state is restored (outside the per-step events), in the warm-up too, and
    # each call starts from its entry state, so no step runs more than 2 CHUNK - 1 steps past
    # the initial state and every timed step runs on finite data (libtc reports a non-finite
    # state on the next tc_step).
    CHUNK = 5

    def timed_steps(plan, st, K, profile=False):
        if not st.started:
            plan.step(st, 0)           # the cold state's history first: the snapshot is a started state
        start = {k: getattr(st, k).clone() for k in ("u", "u_prev", "N_prev", "p")}
        for w in range(args.warmup):
            if w and w % CHUNK == 0:   # a long warm-up restarts from the entry state too
                for k, v in start.items():
                    getattr(st, k).copy_(v)
            plan.step(st, 1)
        # keep the GPU loaded (untimed L2-flush writes) for 0.3 s after the warm-up steps: a GPU
        # left idle drops its clocks, and the first timed step then ran up to 20% slow
        t_end = time.perf_counter() + 0.3
        while time.perf_counter() < t_end:
            flush.fill_(0.0)
            torch.cuda.synchronize()
        torch.cuda.synchronize()
        saved = {k: getattr(st, k).clone() for k in ("u", "u_prev", "N_prev", "p")}
        finite = True
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        prof = {}
        # no garbage-collection pause while the host enqueues a timed step
        gc.collect()
        gc.disable()
        for c0 in range(0, K, CHUNK):
            for k, v in saved.items():
                getattr(st, k).copy_(v)
            if profile:
                plan.profile(True)
            for i in range(c0, min(K, c0 + CHUNK)):
                flush.fill_(float(i))
                gpu_spin()   # the GPU stays busy while the host enqueues the step's launches
                ev[i][0].record(stream)
                plan.step(st, 1)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            if profile:
                for name, (n, ms) in plan.profile_read().items():
                    a = prof.get(name, (0, 0.0))
                    prof[name] = (a[0] + n, a[1] + ms)
                plan.profile(False)
            finite = finite and bool(plan.diagnostics(st.u).finite)
        gc.enable()
        for k, v in start.items():
            getattr(st, k).copy_(v)
        return [a.elapsed_time(b) for a, b in ev], prof, finite

    K = args.steps
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        step_ms, _, finite = timed_steps(plan, st, K)
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    total_ms = max_over_ranks(dist, sum(step_ms), "cuda")
    ms_per_step = total_ms / K
    value = aggregate_value(world, K, total_ms)

    # per-kernel breakdown: a tracing pass over the same number of steps
    _, prof, _ = timed_steps(plan, st, K, profile=True)
    launches = sum(n for n, _ in prof.values())
    NL = ("k_zinv", "k_theta", "k_zfwd")
    nl_ms = sum(prof[k][1] for k in NL if k in prof) / K
    pc_ms = sum(v[1] for k, v in prof.items() if k not in NL) / K
    top = max(prof.items(), key=lambda kv: kv[1][1])
    Pt, Pz = 3 * cfg["M"], 3 * cfg["K"]
    flops = {"k_theta": theta_flops(cfg, Pt, Pz), "k_zinv": zpass_flops(cfg, Pz, 9),
             "k_zfwd": zpass_flops(cfg, Pz, 3)}
    fp64_peak = FP64_PEAK
    # the FP64 FMA rate measured on this device by libtc's probe (8 independent FMA chains per
    # thread, 8 blocks of 256 threads per SM): the achievable counterpart of the unit-count peak
    fp64_measured = tc.fp64_fma_rate()
    roof = None
    if top[0] in flops:
        avg_s = top[1][1] / top[1][0] / 1e3
        ach = flops[top[0]] / avg_s
        roof = {"kernel": top[0], "bound": "alu", "achieved": ach / 1e12, "peak": fp64_peak / 1e12,
                "unit": "TFLOP/s", "frac": ach / fp64_peak,
                # dram__bytes_read.sum + dram__bytes_write.sum of the FP64 theta pass per launch at
                # this workload from one ncu --set full capture; None until the current kernel
                # has been captured
                "traffic": THETA_TRAFFIC if (top[0] == "k_theta" and main_is_bench) else None,
                "peak_source": "152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz (unit counts and max clock)",
                "peak_measured": fp64_measured / 1e12,
                "frac_of_measured": ach / fp64_measured,
                "peak_measured_source": "tc_probe_fp64_fma: 8 independent FMA chains per thread, "
                                        "8 x 256 threads per SM, best of 5 launches (CUDA events)",
                "algorithmic": "7.5 complex FFTs of P_theta at 5 n log2 n + 25 flop/point per (r, z)"}
    else:
        roof = {"kernel": top[0], "bound": "alu", "achieved": None, "peak": fp64_peak / 1e12,
                "unit": "TFLOP/s", "frac": None, "traffic": None, "peak_measured": fp64_measured / 1e12}

    # mixed precision form at the same size: speed and error after CHUNK steps vs FP64
    mplan = tc.Plan(**cfg, precision=tc.TC_MIXED, device=f"cuda:{local}")
    mst = tc.State(mplan, u0_t.cuda())
    m_ms, _, m_finite = timed_steps(mplan, mst, K)
    _, mprof, _ = timed_steps(mplan, mst, K, profile=True)
    # the same with the FP32 transforms' mean mode (tc_options.mean_fp32): the cost of the
    # exact mean mode
    qplan = tc.Plan(**cfg, precision=tc.TC_MIXED, mean_fp32=True, device=f"cuda:{local}")
    qst = tc.State(qplan, u0_t.cuda())
    q_ms, _, _ = timed_steps(qplan, qst, K)
    del qplan, qst
    # error of the mixed form at the largest stable dt (stated dt halved until 200 FP64
    # steps stay finite and the perturbation energy grows by less than 10x)
    base = torch.from_numpy(I.base_state(r, cfg["M"], cfg["K"], cfg["eta"], cfg["Re_i"], cfg["Re_o"])).cuda()
    NERR = 200
    dt_eff = cfg["dt"]
    for _ in range(10):
        tplan = tc.Plan(**{**cfg, "dt": dt_eff}, device=f"cuda:{local}")
        ts = tc.State(tplan, u0_t.cuda())
        e0 = tplan.diagnostics(ts.u).energy
        tplan.step(ts, NERR)
        d = tplan.diagnostics(ts.u)
        del tplan
        if d.finite and d.energy < 10.0 * e0:
            break
        dt_eff /= 2.0
    fplan = tc.Plan(**{**cfg, "dt": dt_eff}, device=f"cuda:{local}")
    eplan = tc.Plan(**{**cfg, "dt": dt_eff}, precision=tc.TC_MIXED, device=f"cuda:{local}")
    a = tc.State(fplan, u0_t.cuda())
    b = tc.State(eplan, u0_t.cuda())
    fplan.step(a, NERR)
    eplan.step(b, NERR)
    da, db = fplan.diagnostics(a.u), eplan.diagnostics(b.u)
    pa, pb = a.u - base, b.u - base
    mixed = {"value": world * K / (sum(m_ms) / 1e3), "unit": "steps/s", "ms_per_step": sum(m_ms) / K,
             "speedup_vs_fp64": (total_ms / K) / (sum(m_ms) / K),
             "dtype": "f32 transforms/products + f64 mean flow, solves, factors",
             "ms_per_step_fp32_mean_mode": sum(q_ms) / K,
             "note": "the (0,0) mode of N from an exact double-FP32 Parseval sum (beside the FP32 "
                     "transforms); ms_per_step_fp32_mean_mode keeps the transforms' value instead",
             "error_dt": dt_eff, "error_after_steps": NERR,
             "rel_err_velocity_perturbation": float(torch.linalg.vector_norm(pb - pa) / torch.linalg.vector_norm(pa)),
             "rel_err_velocity": float(torch.linalg.vector_norm(b.u - a.u) / torch.linalg.vector_norm(a.u)),
             "rel_err_torque_inner": abs(db.torque_inner / da.torque_inner - 1),
             "rel_err_torque_outer": abs(db.torque_outer / da.torque_outer - 1),
             "max_div_fp64": da.max_div, "max_div_mixed": db.max_div,
             "state_finite": m_finite and bool(db.finite)}
    del fplan, eplan
    del mplan

    # end to end through the C ABI with host buffers (tc_step_host): every step copies the
    # state (u, u_prev, N_prev) from pinned host memory, steps it, and copies u and p back;
    # the call returns when the host copies are complete
    host = {k: torch.empty_like(getattr(st, k), device="cpu").pin_memory() for k in ("u", "u_prev", "N_prev", "p")}
    for k in host:
        host[k].copy_(getattr(st, k))
    host["started"] = True
    # a started state's p^i is not read by a step, so tc_step_host copies u, u_prev, N_prev in
    bi = sum(t.numel() * t.element_size() for k, t in host.items() if k in ("u", "u_prev", "N_prev"))
    hout = {"u": torch.empty_like(host["u"]).pin_memory(), "p": torch.empty_like(host["p"]).pin_memory()}
    bo = sum(t.numel() * t.element_size() for t in hout.values())
    for _ in range(args.warmup):
        plan.step_host(st, host, hout, 1, stream=stream)
    torch.cuda.synchronize()
    E = min(K, 20)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(E):
        plan.step_host(st, host, hout, 1, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value = world * E / (e0.elapsed_time(e1) / 1e3)

    out = {
        "metric": METRIC if main_is_bench else METRIC.replace("FP64 plain", args.workload + " " + args.size),
        "value": value, "unit": "steps/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.workload == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if main_is_bench else
                   f"{args.workload} step at N_r={cfg['N_r']}, M={cfg['M']}, K={cfg['K']} (profiling case)",
                   "N_r": cfg["N_r"], "M": cfg["M"], "K": cfg["K"],
                   "P_theta": Pt, "P_z": Pz, "dt": cfg["dt"], "gdof": gdof(cfg),
                   "l2": "flushed before every timed step (256 MiB fill outside the per-step events)",
                   "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
        "gdof_steps_per_s": value * gdof(cfg) / 1e9,
        "phases_ms": {"nonlinear": nl_ms, "predictor_corrector": pc_ms},
        "kernels_ms_per_step": {k: v[1] / K for k, v in sorted(prof.items())},
        "kernel_rooflines": {"fp64": kernel_rooflines(cfg, prof), "mixed": kernel_rooflines(cfg, mprof)},
        "roofline": roof,
        "mixed": mixed,
        "e2e": {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "wall_s_timed_region": wall,
        "state_finite": bool(finite),
    }
    if not args.no_extras:
        nl64 = sum(prof[k][1] for k in ("k_zinv", "k_theta", "k_zfwd") if k in prof) / K
        nl32 = sum(v[1] for k, v in mprof.items() if k.endswith("_f32")) / K
        for key, fn in (("cufft_comparison", lambda: {**cufft_comparison(torch, cfg, f"cuda:{local}"),
                                                      "ours_fp64_nonlinear_ms": nl64,
                                                      "ours_fp32_nonlinear_ms": nl32}),
                        ("tensor_dft_comparison", lambda: tensor_dft_comparison(torch, f"cuda:{local}")),
                        ("adjoint", lambda: adjoint_ratio(tc, torch, I, f"cuda:{local}")),
                        ("large_same_size", lambda: large_mixed(tc, torch, I, f"cuda:{local}")),
                        ("paper_small", lambda: paper_small(tc, torch, I, f"cuda:{local}"))):
            try:
                out[key] = fn()
            except Exception as exc:  # keep the main line even if an extra measurement fails
                out[key] = {"error": repr(exc)[:300]}
            torch.cuda.empty_cache()
    if args.largest:
        for key, fn in (("largest", lambda: largest(tc, torch, I, f"cuda:{local}")),
                        ("config5_adjoint", lambda: config5_adjoint(tc, torch, I, f"cuda:{local}")),
                        ("config5_dot_product", lambda: config5_dot_product(tc, torch, I, f"cuda:{local}"))):
            try:
                out[key] = fn()
            except Exception as exc:
                out[key] = {"error": repr(exc)[:300]}
            torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


ORACLE_CHUNK = 5


def _oracle_steps(seconds, max_steps=None):
    """Time the oracle's step on the benchmark workload for about `seconds` (host cores).
    As in the GPU arm, the stated dt is beyond the advection limit, so the started state is
    restored every ORACLE_CHUNK steps (outside the timed intervals): every timed step runs
    on finite data no more than 2 ORACLE_CHUNK - 1 steps past the initial state."""
    import numpy as np
    import oracle as O
    from paper_1311_2481_gb300 import inputs as I
    ops = O.Operators(O.Params(**CFG2))
    ops.mats
    u0 = I.initial_state(ops.r, CFG2["M"], CFG2["K"], CFG2["m_p"], CFG2["L_z"], CFG2["eta"],
                         CFG2["Re_i"], CFG2["Re_o"], kind="taylor", amp=1e-2, seed=42)
    start = O.step(ops, O.cold_state(u0))       # start-up outside the sample
    st = start
    n, el = 0, 0.0
    with np.errstate(over="raise", invalid="raise"):
        while True:
            if n % ORACLE_CHUNK == 0:
                st = start
            t0 = time.perf_counter()
            st = O.step(ops, st)
            el += time.perf_counter() - t0
            n += 1
            if el >= seconds or (max_steps and n >= max_steps):
                return n, el


def cpu_baseline(seconds):
    n, el = _oracle_steps(seconds)
    return {"value": n / el, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} oracle steps of the benchmark workload after its start-up step, "
                      f"restarted every {ORACLE_CHUNK} steps (numpy FP64, dense DFT matrices, "
                      f"banded Gaussian elimination per mode)"}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    secs = max(1.0, args.cpu_seconds)
    for _ in range(args.warmup):
        _oracle_steps(0.0, max_steps=1)
    n, el = _oracle_steps(secs * max(1, args.steps) / 10.0, max_steps=max(1, args.steps))
    v = n / el
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": world,
           "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * el / n, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD},
           "cpu_baseline": {"value": v, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"{n} oracle steps after the start-up step, restarted every "
                                      f"{ORACLE_CHUNK} steps"},
           "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the adjoint and large-size measurements")
    ap.add_argument("--largest", action="store_true",
                    help="also time the FP64 and mixed steps at N_r = 384 (384 x 1152 x 2304), the mixed "
                         "form there with the FP64 adjoint of its last 50 steps, and one FP64 adjoint step "
                         "with its dot-product test at that size")
    ap.add_argument("--workload", default="fp64", choices=["fp64", "mixed", "adjoint"],
                    help="form of the main timed step: the headline metric is the FP64 step at the "
                         "bench size; mixed (or another --size) names its form and size in the metric; "
                         "adjoint: time the FP64 adjoint step at --size instead (profiling)")
    ap.add_argument("--size", default="bench", choices=["bench", "mid", "split", "long"],
                    help="bench: N_r=64, M=32, K=64; mid: N_r=128, M=128, K=256; split: N_r=256, M=32, "
                         "K=64 (the per-stage steps-2-5 kernels); long: N_r=32, M=384, K=64 (1152-point "
                         "theta lines) -- the last three for profiling")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "adjoint":
        run_adjoint_case(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
