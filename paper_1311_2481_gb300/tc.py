"""Thin ctypes binding of libtc (include/tc.h).  Argument marshalling only: every step of the
time step runs in the library's CUDA kernels.  There is no CPU fallback: importing a function
that needs the library raises if ``_lib/libtc.so`` is missing (build it with
``paper_1311_2481_gb300.build.build()``).

Module-level functions carry the C names (``tc_plan_create``, ``tc_nonlinear``, ...); the
``Plan`` and ``State`` classes wrap them for torch tensors (device memory and streams)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libtc.so")

TC_OK, TC_ERR_ARG, TC_ERR_CUDA, TC_ERR_OOM, TC_ERR_NONFINITE, TC_ERR_TIMEOUT, TC_ERR_STATE = range(7)
TC_P_STAR, TC_U_PLUS, TC_U_MINUS, TC_U_Z, TC_PHI = range(5)
TC_FP64, TC_MIXED = 0, 1
(TC_SET_ALPHA, TC_SET_P_THETA, TC_SET_P_Z, TC_SET_PRECISION, TC_SET_HOST_ONLY, TC_SET_THETA_ZT,
 TC_SET_PC_MODES, TC_SET_NO_ADJOINT, TC_SET_PC_SPLIT, TC_SET_THETA_VARIANT, TC_SET_PC_PARTITIONS,
 TC_SET_STAGE_ROWS, TC_SET_MEAN_FP32) = range(13)

# every symbol include/tc.h declares, in declaration order
SYMBOLS = [
    "tc_plan_create", "tc_plan_create_ex", "tc_plan_destroy", "tc_plan_set", "tc_plan_workspace_bytes",
    "tc_plan_nodes", "tc_plan_fd_weights", "tc_plan_solve_host", "tc_plan_last_error", "tc_status_string",
    "tc_nonlinear", "tc_helmholtz_solve", "tc_step", "tc_step_host", "tc_diagnostics",
    "tc_adjoint_step", "tc_adjoint_start", "tc_energy_gradient",
    "tc_nonlinear_noalloc", "tc_probe_fp64_fma", "tc_profile_enable", "tc_profile_read",
]


class tc_options(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("P_theta", ctypes.c_int), ("P_z", ctypes.c_int),
                ("precision", ctypes.c_int), ("host_only", ctypes.c_int), ("theta_zt", ctypes.c_int),
                ("pc_modes", ctypes.c_int), ("no_adjoint", ctypes.c_int), ("pc_split", ctypes.c_int),
                ("theta_variant", ctypes.c_int), ("pc_partitions", ctypes.c_int),
                ("stage_rows", ctypes.c_int), ("mean_fp32", ctypes.c_int)]


class tc_state(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("u_prev", ctypes.c_void_p), ("N_prev", ctypes.c_void_p),
                ("p", ctypes.c_void_p), ("started", ctypes.c_int)]


class tc_state_bar(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("u_prev", ctypes.c_void_p), ("N_prev", ctypes.c_void_p)]


class tc_diag(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("torque_inner", ctypes.c_double),
                ("torque_outer", ctypes.c_double), ("max_div", ctypes.c_double),
                ("finite", ctypes.c_int), ("nu_omega_inner", ctypes.c_double),
                ("nu_omega_outer", ctypes.c_double)]


class TCError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"libtc status {status} ({_status_text(status)}){': ' + msg if msg else ''}")


_LIB = None


def load_library(path: str = LIB_PATH):
    """Load libtc.so (raises OSError when it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise OSError(f"libtc.so not built at {path}; run paper_1311_2481_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I, D, S = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "tc_plan_create": (I, [ctypes.POINTER(P), I, I, I, I, D, D, D, D, D, I]),
        "tc_plan_create_ex": (I, [ctypes.POINTER(P), I, I, I, I, D, D, D, D, D, I, ctypes.POINTER(tc_options)]),
        "tc_plan_destroy": (None, [P]),
        "tc_plan_set": (I, [P, I, D]),
        "tc_plan_workspace_bytes": (I, [P, ctypes.POINTER(S)]),
        "tc_plan_nodes": (I, [P, ctypes.POINTER(D)]),
        "tc_plan_fd_weights": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(I)]),
        "tc_plan_solve_host": (I, [P, I, I, I, I, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "tc_plan_last_error": (ctypes.c_char_p, [P]),
        "tc_status_string": (ctypes.c_char_p, [I]),
        "tc_nonlinear": (I, [P, P, P, P, P]),
        "tc_helmholtz_solve": (I, [P, I, P, P, P, P]),
        "tc_step": (I, [P, ctypes.POINTER(tc_state), I, P, P]),
        "tc_step_host": (I, [P, ctypes.POINTER(tc_state), ctypes.POINTER(tc_state), ctypes.POINTER(tc_state),
                             I, P, P]),
        "tc_diagnostics": (I, [P, P, ctypes.POINTER(tc_diag), P, P]),
        "tc_adjoint_step": (I, [P, ctypes.POINTER(tc_state), ctypes.POINTER(tc_state_bar), P, P]),
        "tc_adjoint_start": (I, [P, P, ctypes.POINTER(tc_state_bar), P, P, P]),
        "tc_energy_gradient": (I, [P, P, P, P]),
        "tc_nonlinear_noalloc": (I, [P, P, P, P]),
        "tc_probe_fp64_fma": (I, [I, I, I, P, P, ctypes.POINTER(D)]),
        "tc_profile_enable": (I, [P, I]),
        "tc_profile_read": (I, [P, I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(D)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _status_text(s):
    try:
        return load_library().tc_status_string(s).decode()
    except OSError:
        return "?"


def _check(status, plan=None):
    if status != TC_OK:
        msg = ""
        if plan:
            msg = (load_library().tc_plan_last_error(plan) or b"").decode()
        raise TCError(status, msg)


# ------------------------------------------------------------------ C-named functions

def tc_plan_create(N_r, M, K, m_p, eta, Re_i, Re_o, L_z, dt, fd_order=8, options=None):
    lib = load_library()
    h = ctypes.c_void_p()
    if options is None:
        st = lib.tc_plan_create(ctypes.byref(h), N_r, M, K, m_p, eta, Re_i, Re_o, L_z, dt, fd_order)
    else:
        st = lib.tc_plan_create_ex(ctypes.byref(h), N_r, M, K, m_p, eta, Re_i, Re_o, L_z, dt,
                                   fd_order, ctypes.byref(options))
    _check(st)
    return h


def tc_plan_destroy(h):
    load_library().tc_plan_destroy(h)


def tc_plan_set(h, key, value):
    _check(load_library().tc_plan_set(h, key, float(value)), h)


def tc_plan_workspace_bytes(h):
    n = ctypes.c_size_t()
    _check(load_library().tc_plan_workspace_bytes(h, ctypes.byref(n)), h)
    return n.value


def tc_nonlinear(h, u_ptr, N_ptr, ws_ptr, stream_ptr):
    _check(load_library().tc_nonlinear(h, u_ptr, N_ptr, ws_ptr, stream_ptr), h)


def tc_helmholtz_solve(h, which, rhs_ptr, x_ptr, ws_ptr, stream_ptr):
    _check(load_library().tc_helmholtz_solve(h, which, rhs_ptr, x_ptr, ws_ptr, stream_ptr), h)


def tc_step(h, state: tc_state, nsteps, ws_ptr, stream_ptr):
    _check(load_library().tc_step(h, ctypes.byref(state), nsteps, ws_ptr, stream_ptr), h)


def tc_step_host(h, host_in: tc_state, host_out: tc_state, dev: tc_state, nsteps, ws_ptr, stream_ptr):
    _check(load_library().tc_step_host(h, ctypes.byref(host_in), ctypes.byref(host_out), ctypes.byref(dev),
                                       nsteps, ws_ptr, stream_ptr), h)


def tc_diagnostics(h, u_ptr, ws_ptr, stream_ptr):
    d = tc_diag()
    st = load_library().tc_diagnostics(h, u_ptr, ctypes.byref(d), ws_ptr, stream_ptr)
    if st not in (TC_OK, TC_ERR_NONFINITE):
        _check(st, h)
    return d


# ------------------------------------------------------------------ torch convenience layer

def fp64_fma_rate(blocks=None, threads=256, iters=20000, reps=5):
    """Measured FP64 FMA rate of the current device (tc_probe_fp64_fma): flop/s of the best
    of `reps` launches, timed with CUDA events on the current stream."""
    torch = _torch()
    if blocks is None:
        blocks = 8 * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    fl = ctypes.c_double()
    best = None
    for i in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _check(load_library().tc_probe_fp64_fma(blocks, threads, iters, ctypes.c_void_p(sink.data_ptr()),
                                                ctypes.c_void_p(stream.cuda_stream), ctypes.byref(fl)))
        e1.record(stream)
        torch.cuda.synchronize()
        if i:   # the first launch warms up
            rate = fl.value / (e0.elapsed_time(e1) / 1e3)
            best = rate if best is None else max(best, rate)
    return best


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A libtc plan plus a device workspace (torch-allocated)."""

    def __init__(self, N_r, M, K, m_p, eta, Re_i, Re_o, L_z, dt, fd_order=8, alpha=0.5,
                 P_theta=0, P_z=0, precision=TC_FP64, host_only=False, device=None, theta_zt=0,
                 pc_modes=0, no_adjoint=False, pc_split=0, theta_variant=0, pc_partitions=0,
                 stage_rows=0, mean_fp32=0):
        opt = tc_options(alpha if alpha != 0.0 else -1.0, P_theta, P_z, precision, int(host_only),
                         theta_zt, pc_modes, int(no_adjoint), pc_split, theta_variant, pc_partitions,
                         stage_rows, int(mean_fp32))
        self.N_r, self.M, self.K = N_r, M, K
        self.handle = None
        torch = _torch()
        if not host_only:
            dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
            if dev.index is None:
                dev = torch.device("cuda", torch.cuda.current_device())
            torch.cuda.set_device(dev)
            self.device = dev
        self.handle = tc_plan_create(N_r, M, K, m_p, eta, Re_i, Re_o, L_z, dt, fd_order, opt)
        self.host_only = bool(host_only)
        self.ws = None
        self._alloc_ws()

    def _alloc_ws(self):
        self.ws_bytes = tc_plan_workspace_bytes(self.handle)
        self.ws = None
        if not self.host_only:
            self.ws = _torch().empty(self.ws_bytes + 256, dtype=_torch().uint8, device=self.device)

    def set(self, key, value):
        """tc_plan_set (before the plan's first compute call); the workspace is sized anew."""
        self.ws = None
        tc_plan_set(self.handle, key, value)
        if key == TC_SET_HOST_ONLY:
            self.host_only = bool(value)
            if not self.host_only:
                torch = _torch()
                self.device = torch.device("cuda", torch.cuda.current_device())
        self._alloc_ws()

    # shapes
    def vector_shape(self):
        return (3, self.N_r, self.M + 1, 2 * self.K + 1)

    def scalar_shape(self):
        return (self.N_r, self.M + 1, 2 * self.K + 1)

    def _ws(self):
        return ctypes.c_void_p((self.ws.data_ptr() + 255) & ~255)

    def nodes(self):
        import numpy as np
        r = np.zeros(self.N_r)
        _check(load_library().tc_plan_nodes(self.handle, r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), self.handle)
        return r

    def fd_weights(self, deriv):
        import numpy as np
        w = np.zeros((self.N_r, 9))
        c = np.zeros(self.N_r, dtype=np.int32)
        _check(load_library().tc_plan_fd_weights(self.handle, deriv,
                                                 w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                 c.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), self.handle)
        return w, c

    def solve_host(self, which, m, ka, b, partitions=1):
        """Host solve with the stored factors of a host_only plan (inspection)."""
        import numpy as np
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.N_r)
        _check(load_library().tc_plan_solve_host(self.handle, which, m, ka, partitions,
                                                 b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                 x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), self.handle)
        return x

    def nonlinear(self, u, N=None, stream=None):
        torch = _torch()
        if N is None:
            N = torch.empty_like(u)
        tc_nonlinear(self.handle, _ptr(u), _ptr(N), self._ws(), _stream_ptr(stream))
        return N

    def helmholtz_solve(self, which, rhs, x=None, stream=None):
        torch = _torch()
        if x is None:
            x = torch.empty_like(rhs)
        tc_helmholtz_solve(self.handle, which, _ptr(rhs), _ptr(x), self._ws(), _stream_ptr(stream))
        return x

    def step(self, state: "State", nsteps=1, stream=None):
        cs = state.c_struct()
        tc_step(self.handle, cs, nsteps, self._ws(), _stream_ptr(stream))
        state.started = bool(cs.started)
        return state

    def step_host(self, dev: "State", host_in: dict, host_out: dict, nsteps=1, stream=None):
        """tc_step_host: host_in / host_out map 'u', 'u_prev', 'N_prev', 'p' to CPU tensors
        (pinned for full-speed copies; host_out may omit fields); dev is the device working
        state.  Returns when host_out holds the result."""
        def hstate(d, started):
            return tc_state(*[d[k].data_ptr() if k in d else None for k in ("u", "u_prev", "N_prev", "p")],
                            int(started))
        hin, hout = hstate(host_in, host_in.get("started", dev.started)), hstate(host_out, 0)
        cs = dev.c_struct()
        tc_step_host(self.handle, hin, hout, cs, nsteps, self._ws(), _stream_ptr(stream))
        dev.started = bool(cs.started)
        return dev

    def diagnostics(self, u, stream=None):
        return tc_diagnostics(self.handle, _ptr(u), self._ws(), _stream_ptr(stream))

    def adjoint_step(self, fwd: "State", bar: "StateBar", stream=None):
        """In place: bar (adjoints of u^{i+1}, u^i, N^i) -> adjoints of (u^i, u^{i-1}, N^{i-1})."""
        cs = fwd.c_struct()
        cb = bar.c_struct()
        _check(load_library().tc_adjoint_step(self.handle, ctypes.byref(cs), ctypes.byref(cb), self._ws(),
                                              _stream_ptr(stream)), self.handle)
        return bar

    def adjoint_start(self, u0, bar: "StateBar", out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty_like(u0)
        cb = bar.c_struct()
        _check(load_library().tc_adjoint_start(self.handle, _ptr(u0), ctypes.byref(cb), _ptr(out), self._ws(),
                                               _stream_ptr(stream)), self.handle)
        return out

    def energy_gradient(self, u, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty_like(u)
        _check(load_library().tc_energy_gradient(self.handle, _ptr(u), _ptr(out), _stream_ptr(stream)), self.handle)
        return out

    def profile(self, enable=True):
        _check(load_library().tc_profile_enable(self.handle, int(enable)), self.handle)

    def profile_read(self):
        """{kernel name: (launches, total ms)} recorded since profile(True)."""
        lib = load_library()
        out = {}
        i = 0
        while True:
            name = ctypes.c_char_p()
            n = ctypes.c_longlong()
            ms = ctypes.c_double()
            st = lib.tc_profile_read(self.handle, i, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms))
            if st == TC_ERR_ARG:
                break
            _check(st, self.handle)
            if n.value:
                out[name.value.decode()] = (n.value, ms.value)
            i += 1
        return out

    def close(self):
        if self.handle:
            tc_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StateBar:
    """Adjoint state (device tensors): adjoints of u, u_prev, N_prev."""

    def __init__(self, u, u_prev, N_prev):
        self.u, self.u_prev, self.N_prev = u, u_prev, N_prev

    def c_struct(self):
        return tc_state_bar(self.u.data_ptr(), self.u_prev.data_ptr(), self.N_prev.data_ptr())


class State:
    """Caller-owned AB2BD2 state (device tensors): u, u_prev, N_prev (vector fields), p."""

    def __init__(self, plan: Plan, u0):
        torch = _torch()
        self.u = u0.to(device=plan.device, dtype=torch.complex128).contiguous().clone()
        self.u_prev = torch.zeros_like(self.u)
        self.N_prev = torch.zeros_like(self.u)
        self.p = torch.zeros(plan.scalar_shape(), dtype=torch.complex128, device=plan.device)
        self.started = False

    def c_struct(self):
        return tc_state(self.u.data_ptr(), self.u_prev.data_ptr(), self.N_prev.data_ptr(),
                        self.p.data_ptr(), int(self.started))
