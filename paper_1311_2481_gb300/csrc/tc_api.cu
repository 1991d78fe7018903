// C-ABI entry points of libtc that launch work: argument validation on the host, then
// kernels enqueued on the caller's stream.
#include <cmath>
#include <cstring>

#include "tc_internal.cuh"

using namespace tc;

namespace {

tc_status ready(tc_plan* p) {
    if (!p) return TC_ERR_ARG;
    if (p->host_only) {
        snprintf(p->err, sizeof(p->err), "host-only plan");
        return TC_ERR_STATE;
    }
    int dev = -1;
    TC_CUDA(p, cudaGetDevice(&dev));
    if (dev != p->device) {
        snprintf(p->err, sizeof(p->err), "current device %d differs from the plan's device %d", dev, p->device);
        return TC_ERR_STATE;
    }
    p->used = true;
    return TC_OK;
}

tc_status check_ws(tc_plan* p, void* ws) {
    if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
        snprintf(p->err, sizeof(p->err), "workspace must be a 256-byte aligned device pointer");
        return TC_ERR_ARG;
    }
    return check_device_ptr(p, ws, "ws", p->ws.total);
}

// An update kernel of an earlier step wrote a NaN/Inf into the state (flag in mapped host
// memory, read without synchronising): report it once and clear it.
tc_status take_nonfinite(tc_plan* p) {
    volatile int* f = p->h_nonfinite;
    if (f && *f) {
        *f = 0;
        snprintf(p->err, sizeof(p->err), "an earlier step wrote a non-finite value into the state");
        return TC_ERR_NONFINITE;
    }
    return TC_OK;
}

#define TC_TRY(x)                       \
    do {                                \
        tc_status s_ = (x);             \
        if (s_ != TC_OK) return s_;     \
    } while (0)

}  // namespace

extern "C" {

tc_status tc_nonlinear(tc_plan* plan, const void* u_hat, void* N_hat, void* ws, void* stream) {
    TC_TRY(ready(plan));
    const size_t vb = 3 * plan->S * sizeof(double2);
    TC_TRY(check_device_ptr(plan, u_hat, "u_hat", vb));
    TC_TRY(check_device_ptr(plan, N_hat, "N_hat", vb));
    TC_TRY(check_ws(plan, ws));
    if (u_hat == N_hat) return TC_ERR_ARG;
    return launch_nonlinear(plan, static_cast<const double2*>(u_hat), static_cast<double2*>(N_hat),
                            static_cast<char*>(ws), static_cast<cudaStream_t>(stream));
}

tc_status tc_helmholtz_solve(tc_plan* plan, int which, const void* rhs, void* x, void* ws, void* stream) {
    TC_TRY(ready(plan));
    if (which < TC_P_STAR || which > TC_PHI) return TC_ERR_ARG;
    TC_TRY(check_device_ptr(plan, rhs, "rhs", plan->S * sizeof(double2)));
    TC_TRY(check_device_ptr(plan, x, "x", plan->S * sizeof(double2)));
    TC_TRY(check_ws(plan, ws));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (rhs != x)
        TC_CUDA(plan, cudaMemcpyAsync(x, rhs, plan->S * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    const int set = (which == TC_P_STAR || which == TC_PHI) ? kSetP
                  : which == TC_U_PLUS ? kSetHp : which == TC_U_MINUS ? kSetHm : kSetHz;
    return launch_solve(plan, set, static_cast<double2*>(x), 1, s);
}

tc_status tc_step(tc_plan* plan, tc_state* st, int nsteps, void* ws, void* stream) {
    TC_TRY(ready(plan));
    if (!st || nsteps < 0) return TC_ERR_ARG;
    const size_t vb = 3 * plan->S * sizeof(double2), sb = plan->S * sizeof(double2);
    TC_TRY(check_device_ptr(plan, st->u, "u", vb));
    TC_TRY(check_device_ptr(plan, st->u_prev, "u_prev", vb));
    TC_TRY(check_device_ptr(plan, st->N_prev, "N_prev", vb));
    TC_TRY(check_device_ptr(plan, st->p, "p", sb));
    TC_TRY(check_ws(plan, ws));
    const void* ptrs[4] = {st->u, st->u_prev, st->N_prev, st->p};
    for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j)
            if (ptrs[i] == ptrs[j]) return TC_ERR_ARG;
    TC_TRY(take_nonfinite(plan));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    double2* u = static_cast<double2*>(st->u);
    double2* up = static_cast<double2*>(st->u_prev);
    double2* Np = static_cast<double2*>(st->N_prev);
    double2* p = static_cast<double2*>(st->p);
    double2* Nc = reinterpret_cast<double2*>(w + plan->ws.Ncur);
    double2* uE = reinterpret_cast<double2*>(w + plan->ws.uE);
    const size_t n3 = 3 * plan->S;
    if (!st->started) {
        // history for AB2BD2: implicit Euler step of 2dt/3, then u^{-1}, N^{-1}
        TC_TRY(launch_nonlinear(plan, u, Nc, w, s));
        TC_TRY(launch_advance(plan, u, u, Nc, Nc, p, uE, w, false, s));
        TC_TRY(launch_axpby(plan, up, u, 2.5, uE, -1.5, n3, s));
        TC_TRY(launch_nonlinear(plan, up, Np, w, s));
        st->started = 1;
    }
    for (int i = 0; i < nsteps; ++i) {
        TC_TRY(launch_nonlinear(plan, u, Nc, w, s));
        TC_TRY(launch_advance(plan, u, up, Nc, Np, p, nullptr, w, true, s));
    }
    return TC_OK;
}

tc_status tc_step_host(tc_plan* plan, const tc_state* host_in, tc_state* host_out, tc_state* dev,
                       int nsteps, void* ws, void* stream) {
    TC_TRY(ready(plan));
    if (!host_in || !host_out || !dev) return TC_ERR_ARG;
    const void* hin[4] = {host_in->u, host_in->u_prev, host_in->N_prev, host_in->p};
    for (int i = 0; i < 4; ++i) {
        if (!hin[i]) return TC_ERR_ARG;
        cudaPointerAttributes at;
        TC_CUDA(plan, cudaPointerGetAttributes(&at, hin[i]));
        if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
            snprintf(plan->err, sizeof(plan->err), "tc_step_host: host_in field %d is device memory", i);
            return TC_ERR_ARG;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t vb = 3 * plan->S * sizeof(double2), sb = plan->S * sizeof(double2);
    void* dptr[4] = {dev->u, dev->u_prev, dev->N_prev, dev->p};
    const size_t bytes[4] = {vb, vb, vb, sb};
    for (int i = 0; i < 4; ++i) TC_TRY(check_device_ptr(plan, dptr[i], "dev state", bytes[i]));
    if (host_in->started && nsteps >= 1) {
        // A started state: the first step's nonlinear term needs u only, so u_prev and N_prev
        // come in on a second stream while it runs; steps 2-5 wait for them.  p^i is not read
        // by a step (p* is solved afresh and the update writes p^{i+1}), so it is not copied.
        TC_TRY(take_nonfinite(plan));
        TC_CUDA(plan, cudaMemcpyAsync(dptr[0], hin[0], bytes[0], cudaMemcpyHostToDevice, s));
        if (!plan->copy_stream) {
            TC_CUDA(plan, cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking));
            for (cudaEvent_t& e : plan->copy_ev) TC_CUDA(plan, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
        TC_CUDA(plan, cudaEventRecord(plan->copy_ev[0], s));           // after earlier work on dev
        TC_CUDA(plan, cudaStreamWaitEvent(plan->copy_stream, plan->copy_ev[0], 0));
        for (int i = 1; i < 3; ++i)
            TC_CUDA(plan, cudaMemcpyAsync(dptr[i], hin[i], bytes[i], cudaMemcpyHostToDevice, plan->copy_stream));
        TC_CUDA(plan, cudaEventRecord(plan->copy_ev[1], plan->copy_stream));
        char* w = static_cast<char*>(ws);
        double2* Nc = reinterpret_cast<double2*>(w + plan->ws.Ncur);
        double2* u = static_cast<double2*>(dev->u);
        TC_TRY(launch_nonlinear(plan, u, Nc, w, s));
        TC_CUDA(plan, cudaStreamWaitEvent(s, plan->copy_ev[1], 0));
        TC_TRY(launch_advance(plan, u, static_cast<double2*>(dev->u_prev), Nc, static_cast<double2*>(dev->N_prev),
                              static_cast<double2*>(dev->p), nullptr, w, true, s));
        dev->started = 1;
        TC_TRY(tc_step(plan, dev, nsteps - 1, ws, stream));
    } else {
        for (int i = 0; i < 4; ++i)
            TC_CUDA(plan, cudaMemcpyAsync(dptr[i], hin[i], bytes[i], cudaMemcpyHostToDevice, s));
        dev->started = host_in->started;
        TC_TRY(tc_step(plan, dev, nsteps, ws, stream));
    }
    void* hout[4] = {host_out->u, host_out->u_prev, host_out->N_prev, host_out->p};
    for (int i = 0; i < 4; ++i)
        if (hout[i]) TC_CUDA(plan, cudaMemcpyAsync(hout[i], dptr[i], bytes[i], cudaMemcpyDeviceToHost, s));
    TC_CUDA(plan, cudaStreamSynchronize(s));
    host_out->started = dev->started;
    return take_nonfinite(plan);   // this call's own steps (it has synchronised)
}

tc_status tc_diagnostics(tc_plan* plan, const void* u, tc_diag* out, void* ws, void* stream) {
    TC_TRY(ready(plan));
    if (!out) return TC_ERR_ARG;
    TC_TRY(check_device_ptr(plan, u, "u", 3 * plan->S * sizeof(double2)));
    TC_TRY(check_ws(plan, ws));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* red = reinterpret_cast<double*>(static_cast<char*>(ws) + plan->ws.red);
    TC_TRY(launch_diagnostics(plan, static_cast<const double2*>(u), red, s));
    double h[3];
    TC_CUDA(plan, cudaMemcpyAsync(h, red, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    // (0,0) column of u_+ and u_- for the torque
    const int N = plan->N_r;
    std::vector<double2> col(2 * (size_t)N);
    const size_t st = (size_t)plan->nmode;
    const double2* ud = static_cast<const double2*>(u);
    TC_CUDA(plan, cudaMemcpy2DAsync(col.data(), sizeof(double2), ud + plan->K, st * sizeof(double2),
                                    sizeof(double2), N, cudaMemcpyDeviceToHost, s));
    TC_CUDA(plan, cudaMemcpy2DAsync(col.data() + N, sizeof(double2), ud + plan->S + plan->K,
                                    st * sizeof(double2), sizeof(double2), N, cudaMemcpyDeviceToHost, s));
    TC_CUDA(plan, cudaStreamSynchronize(s));
    unsigned long long nbad;
    memcpy(&nbad, &h[2], sizeof(nbad));
    out->energy = h[0];
    out->max_div = h[1];
    out->finite = nbad == 0;
    // T = r^3 d_r(u_theta / r), u_theta^{00} = Im(u_+)... = (u_+ - u_-)/(2i) real part
    auto torque_at = [&](int j) {
        double d = 0.0;
        for (int t = 0; t < kStencil; ++t) {
            int c = plan->col0[j] + t;
            double ut = 0.5 * (col[c].y - col[N + c].y);
            d += plan->w1[(size_t)j * kStencil + t] * ut / plan->r[c];
        }
        double r = plan->r[j];
        return r * r * r * d;
    };
    out->torque_inner = torque_at(0);
    out->torque_outer = torque_at(N - 1);
    // laminar torque r^3 d_r(U / r) = -2 C2 of U = C1 r + C2 / r (Sec. 5.1)
    const double eta = plan->eta;
    const double C2 = eta * (plan->Re_i - eta * plan->Re_o) / ((1.0 - eta) * (1.0 - eta * eta));
    const double T_lam = -2.0 * C2;
    out->nu_omega_inner = T_lam != 0.0 ? out->torque_inner / T_lam : NAN;
    out->nu_omega_outer = T_lam != 0.0 ? out->torque_outer / T_lam : NAN;
    return out->finite ? TC_OK : TC_ERR_NONFINITE;
}

}  // extern "C"
