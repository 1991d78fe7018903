// Linear part of the AB2BD2 step (Sec. 3.2 steps 2-5): right-hand sides, the five banded
// solves per Fourier mode with precomputed LU factors (forward / backward substitution,
// O(N_r) per system), and the update.  One thread per (m, k) system; threads of a warp own
// consecutive k, so every access to a field [r][m][k] or to the factors [j][band][m][|k|]
// is coalesced.
#include "tc_internal.cuh"

namespace tc {

struct Geo {
    int N, M, K, nk, nmode, K1, M1K1;
    size_t S;
    double mp, kz, dt;
};

static Geo geo(const tc_plan* p) {
    Geo g;
    g.N = p->N_r; g.M = p->M; g.K = p->K; g.nk = 2 * p->K + 1; g.nmode = p->nmode;
    g.K1 = p->K + 1; g.M1K1 = (p->M + 1) * (p->K + 1); g.S = p->S;
    g.mp = (double)p->m_p; g.kz = p->k_z; g.dt = p->dt;
    return g;
}

// first and second radial derivative of column `mode` of a scalar field at row j
__device__ __forceinline__ double2 drow(const double2* __restrict__ f, const double* __restrict__ w,
                                        const int* __restrict__ col0, int j, int nmode, int mode) {
    const int c0 = col0[j];
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int t = 0; t < kStencil; ++t) {
        const double wt = __ldg(&w[j * kStencil + t]);
        const double2 v = f[(size_t)(c0 + t) * nmode + mode];
        s.x += wt * v.x;
        s.y += wt * v.y;
    }
    return s;
}

// (Lap u)_r = ((L_+ u_+) + (L_- u_-)) / 2 at row j, L_pm = Lap_h - 1/r^2 -+ 2 m m_p / r^2
__device__ double2 lap_r(const double2* __restrict__ u, const double* __restrict__ w1,
                         const double* __restrict__ w2, const int* __restrict__ col0,
                         double r, int j, int mode, double mm, double kk, const Geo& g) {
    double2 acc = make_double2(0.0, 0.0);
    const double ir = 1.0 / r, ir2 = ir * ir;
    for (int c = 0; c < 2; ++c) {
        const double2* f = u + (size_t)c * g.S;
        const double2 d1 = drow(f, w1, col0, j, g.nmode, mode);
        const double2 d2 = drow(f, w2, col0, j, g.nmode, mode);
        const double2 v = f[(size_t)j * g.nmode + mode];
        const double sgn = c == 0 ? -1.0 : 1.0;
        const double diag = -mm * mm * ir2 - kk * kk - ir2 + sgn * 2.0 * mm * ir2;
        acc.x += d2.x + ir * d1.x + diag * v.x;
        acc.y += d2.y + ir * d1.y + diag * v.y;
    }
    acc.x *= 0.5;
    acc.y *= 0.5;
    return acc;
}

// Step 2 right-hand side: interior rows div_h(-(2N - N_prev)); wall rows the consistent
// Neumann value of Eq. ppBC; (0,0) at r_o the Dirichlet value 0.
__global__ void k_rhs_pressure(const double2* __restrict__ u, const double2* __restrict__ up,
                               const double2* __restrict__ Nc, const double2* __restrict__ Np,
                               double2* __restrict__ b, const double* __restrict__ rn,
                               const double* __restrict__ w1, const double* __restrict__ w2,
                               const int* __restrict__ col0, Geo g) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= g.S) return;
    const int j = (int)(e / g.nmode);
    const int mode = (int)(e - (size_t)j * g.nmode);
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const double mm = g.mp * m, kk = g.kz * k;
    const double r = rn[j], ir = 1.0 / r;
    auto NN = [&](int c, int row) {
        const size_t o = (size_t)c * g.S + (size_t)row * g.nmode + mode;
        const double2 a = Nc[o], q = Np[o];
        return make_double2(2.0 * a.x - q.x, 2.0 * a.y - q.y);
    };
    double2 out;
    if (j == 0 || j == g.N - 1) {
        if (j == g.N - 1 && m == 0 && k == 0) {
            out = make_double2(0.0, 0.0);
        } else {
            const double2 np = NN(0, j), nm = NN(1, j);
            const double2 l0 = lap_r(u, w1, w2, col0, r, j, mode, mm, kk, g);
            const double2 l1 = lap_r(up, w1, w2, col0, r, j, mode, mm, kk, g);
            out.x = -0.5 * (np.x + nm.x) + 2.0 * l0.x - l1.x;
            out.y = -0.5 * (np.y + nm.y) + 2.0 * l0.y - l1.y;
        }
    } else {
        // D1 of NN_r = (NN_+ + NN_-)/2
        const int c0 = col0[j];
        double2 d = make_double2(0.0, 0.0);
#pragma unroll
        for (int t = 0; t < kStencil; ++t) {
            const double wt = __ldg(&w1[j * kStencil + t]);
            const double2 a = NN(0, c0 + t), q = NN(1, c0 + t);
            d.x += wt * 0.5 * (a.x + q.x);
            d.y += wt * 0.5 * (a.y + q.y);
        }
        const double2 np = NN(0, j), nm = NN(1, j), nz = NN(2, j);
        const double2 vr = make_double2(0.5 * (np.x + nm.x), 0.5 * (np.y + nm.y));
        double2 div;
        div.x = d.x + vr.x * ir + mm * (np.x - nm.x) * 0.5 * ir - kk * nz.y;
        div.y = d.y + vr.y * ir + mm * (np.y - nm.y) * 0.5 * ir + kk * nz.x;
        out = make_double2(-div.x, -div.y);
    }
    b[e] = out;
}

// Step 3 right-hand sides: (4u - u_prev)/(2dt) - (2N - N_prev) - grad_h p*; Dirichlet rows.
__global__ void k_rhs_velocity(const double2* __restrict__ u, const double2* __restrict__ up,
                               const double2* __restrict__ Nc, const double2* __restrict__ Np,
                               const double2* __restrict__ ps, double2* __restrict__ rhs,
                               const double* __restrict__ rn, const double* __restrict__ w1,
                               const int* __restrict__ col0, double Re_i, double Re_o, Geo g) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * g.S) return;
    const int c = (int)(e / g.S);
    const size_t es = e - (size_t)c * g.S;
    const int j = (int)(es / g.nmode);
    const int mode = (int)(es - (size_t)j * g.nmode);
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    double2 out;
    if (j == 0 || j == g.N - 1) {
        out = make_double2(0.0, 0.0);
        if (m == 0 && k == 0 && c < 2) {
            const double Re = j == 0 ? Re_i : Re_o;
            out.y = c == 0 ? Re : -Re;  // u_pm = +-i u_theta
        }
    } else {
        const double r = rn[j];
        const double c1 = 1.0 / (2.0 * g.dt);
        const double2 a = u[e], q = up[e], n1 = Nc[e], n0 = Np[e];
        double2 gp;
        const double2 pv = ps[es];
        if (c == 2) {
            const double kk = g.kz * k;
            gp = make_double2(-kk * pv.y, kk * pv.x);
        } else {
            const double2 d = drow(ps, w1, col0, j, g.nmode, mode);
            const double t = (c == 0 ? -1.0 : 1.0) * g.mp * m / r;
            gp = make_double2(d.x + t * pv.x, d.y + t * pv.y);
        }
        out.x = (4.0 * a.x - q.x) * c1 - (2.0 * n1.x - n0.x) - gp.x;
        out.y = (4.0 * a.y - q.y) * c1 - (2.0 * n1.y - n0.y) - gp.y;
    }
    rhs[e] = out;
}

// Step 4 right-hand side: div_h u* on interior rows, homogeneous Neumann / Dirichlet rows.
__global__ void k_rhs_div(const double2* __restrict__ us, double2* __restrict__ b,
                          const double* __restrict__ rn, const double* __restrict__ w1,
                          const int* __restrict__ col0, Geo g) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= g.S) return;
    const int j = (int)(e / g.nmode);
    const int mode = (int)(e - (size_t)j * g.nmode);
    if (j == 0 || j == g.N - 1) { b[e] = make_double2(0.0, 0.0); return; }
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const double mm = g.mp * m, kk = g.kz * k, ir = 1.0 / rn[j];
    const int c0 = col0[j];
    double2 d = make_double2(0.0, 0.0);
#pragma unroll
    for (int t = 0; t < kStencil; ++t) {
        const double wt = __ldg(&w1[j * kStencil + t]);
        const size_t o = (size_t)(c0 + t) * g.nmode + mode;
        const double2 a = us[o], q = us[g.S + o];
        d.x += wt * 0.5 * (a.x + q.x);
        d.y += wt * 0.5 * (a.y + q.y);
    }
    const double2 vp = us[e], vm = us[g.S + e], vz = us[2 * g.S + e];
    double2 div;
    div.x = d.x + 0.5 * (vp.x + vm.x) * ir + mm * (vp.x - vm.x) * 0.5 * ir - kk * vz.y;
    div.y = d.y + 0.5 * (vp.y + vm.y) * ir + mm * (vp.y - vm.y) * 0.5 * ir + kk * vz.x;
    b[e] = div;
}

// Step 5: u^{i+1} = u* - grad_h phi; p^{i+1} = p* + 3 phi / (2 dt).  commit: rotate the
// history in place (u_prev <- u^i, u <- u^{i+1}, N_prev <- N^i, p <- p^{i+1}); otherwise write
// u^{i+1} to u_out only.
__global__ void k_update(double2* __restrict__ u, double2* __restrict__ up, const double2* __restrict__ Nc,
                         double2* __restrict__ Np, double2* __restrict__ p, const double2* __restrict__ us,
                         const double2* __restrict__ ps, const double2* __restrict__ phi,
                         double2* __restrict__ u_out, const double* __restrict__ rn,
                         const double* __restrict__ w1, const int* __restrict__ col0, int commit, Geo g) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * g.S) return;
    const int c = (int)(e / g.S);
    const size_t es = e - (size_t)c * g.S;
    const int j = (int)(es / g.nmode);
    const int mode = (int)(es - (size_t)j * g.nmode);
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const double2 f = phi[es];
    double2 gphi;
    if (c == 2) {
        const double kk = g.kz * k;
        gphi = make_double2(-kk * f.y, kk * f.x);
    } else {
        const double2 d = drow(phi, w1, col0, j, g.nmode, mode);
        const double t = (c == 0 ? -1.0 : 1.0) * g.mp * m / rn[j];
        gphi = make_double2(d.x + t * f.x, d.y + t * f.y);
    }
    const double2 s = us[e];
    const double2 un = make_double2(s.x - gphi.x, s.y - gphi.y);
    if (commit) {
        up[e] = u[e];
        u[e] = un;
        Np[e] = Nc[e];
        if (c == 0) {
            const double q = 3.0 / (2.0 * g.dt);
            const double2 a = ps[es];
            p[es] = make_double2(a.x + q * f.x, a.y + q * f.y);
        }
    } else {
        u_out[e] = un;
    }
}

// Banded substitution with the pivoted LU of Sec. 3.2 (LAPACK band convention): forward
// elimination applying row interchange j <-> j + piv_j then the 4 multipliers of column j,
// backward substitution with the 8 super-diagonals of U and the stored 1/U_jj.
__global__ void k_band_solve(double2* __restrict__ x, const double* __restrict__ fac,
                             const uint8_t* __restrict__ piv, int set0, int nfields, Geo g) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nfields * g.nmode) return;
    const int fld = t / g.nmode;
    const int mode = t - fld * g.nmode;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const int ka = k < 0 ? -k : k;
    const int set = set0 + fld;
    const size_t mk = (size_t)m * g.K1 + ka;
    const size_t per_set = (size_t)g.N * kBands * g.M1K1;
    const double* F = fac + (size_t)set * per_set + mk;
    const uint8_t* P = piv + (size_t)set * g.N * g.M1K1 + mk;
    double2* X = x + (size_t)fld * g.S + mode;
    const int N = g.N;
    const size_t st = g.nmode;
    for (int j = 0; j < N; ++j) {
        const int pj = P[(size_t)j * g.M1K1];
        double2 xj = X[(size_t)j * st];
        if (pj) {
            const double2 xp = X[(size_t)(j + pj) * st];
            X[(size_t)(j + pj) * st] = xj;
            xj = xp;
            X[(size_t)j * st] = xj;
        }
        const double* Fj = F + (size_t)j * kBands * g.M1K1;
#pragma unroll
        for (int q = 1; q <= kKl; ++q) {
            if (j + q < N) {
                const double l = __ldg(&Fj[(size_t)(q - 1) * g.M1K1]);
                double2 v = X[(size_t)(j + q) * st];
                v.x -= l * xj.x;
                v.y -= l * xj.y;
                X[(size_t)(j + q) * st] = v;
            }
        }
    }
    for (int j = N - 1; j >= 0; --j) {
        const double* Fj = F + (size_t)j * kBands * g.M1K1;
        double2 s = X[(size_t)j * st];
#pragma unroll
        for (int q = 1; q <= 2 * kKl; ++q) {
            if (j + q < N) {
                const double uq = __ldg(&Fj[(size_t)(4 + q) * g.M1K1]);
                const double2 v = X[(size_t)(j + q) * st];
                s.x -= uq * v.x;
                s.y -= uq * v.y;
            }
        }
        const double id = __ldg(&Fj[(size_t)4 * g.M1K1]);
        X[(size_t)j * st] = make_double2(s.x * id, s.y * id);
    }
}

__global__ void k_axpby(double2* __restrict__ y, const double2* __restrict__ a, double ca,
                        const double2* __restrict__ b, double cb, size_t n) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double2 x = a[e], z = b[e];
    y[e] = make_double2(ca * x.x + cb * z.x, ca * x.y + cb * z.y);
}

// Diagnostics: red[0] += energy, red[1] = max |div_h u| (as ordered bits), red[2] += non-finite.
__global__ void k_diag(const double2* __restrict__ u, double* __restrict__ red,
                       const double* __restrict__ rn, const double* __restrict__ w1,
                       const int* __restrict__ col0, double C1, double C2, Geo g) {
    __shared__ double s_e[256];
    __shared__ unsigned long long s_d[256];
    __shared__ int s_n[256];
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double en = 0.0, dv = 0.0;
    int bad = 0;
    if (e < g.S) {
        const int j = (int)(e / g.nmode);
        const int mode = (int)(e - (size_t)j * g.nmode);
        const int m = mode / g.nk;
        const int k = mode - m * g.nk - g.K;
        const double r = rn[j];
        double2 a = u[e], b = u[g.S + e], z = u[2 * g.S + e];
        bad = !(isfinite(a.x) && isfinite(a.y) && isfinite(b.x) && isfinite(b.y) && isfinite(z.x) && isfinite(z.y));
        if (m == 0 && k == 0) {
            const double U = C1 * r + C2 / r;
            a.y -= U;
            b.y += U;
        }
        double wr = 0.0;
        if (j > 0) wr += 0.5 * (r - rn[j - 1]);
        if (j < g.N - 1) wr += 0.5 * (rn[j + 1] - r);
        const double cm = m == 0 ? 1.0 : 2.0;
        en = 0.5 * wr * r * cm * (0.5 * (a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y) + z.x * z.x + z.y * z.y);
        if (j > 0 && j < g.N - 1) {
            const int c0 = col0[j];
            double2 d = make_double2(0.0, 0.0);
            for (int t = 0; t < kStencil; ++t) {
                const double wt = w1[j * kStencil + t];
                const size_t o = (size_t)(c0 + t) * g.nmode + mode;
                const double2 p1 = u[o], p2 = u[g.S + o];
                d.x += wt * 0.5 * (p1.x + p2.x);
                d.y += wt * 0.5 * (p1.y + p2.y);
            }
            const double2 vp = u[e], vm = u[g.S + e], vz = u[2 * g.S + e];
            const double mm = g.mp * m, kk = g.kz * k, ir = 1.0 / r;
            const double dx = d.x + 0.5 * (vp.x + vm.x) * ir + mm * (vp.x - vm.x) * 0.5 * ir - kk * vz.y;
            const double dy = d.y + 0.5 * (vp.y + vm.y) * ir + mm * (vp.y - vm.y) * 0.5 * ir + kk * vz.x;
            dv = sqrt(dx * dx + dy * dy);
        }
        if (!isfinite(en)) en = 0.0;
        if (!isfinite(dv)) dv = 0.0;
    }
    s_e[threadIdx.x] = en;
    s_d[threadIdx.x] = (unsigned long long)__double_as_longlong(dv);
    s_n[threadIdx.x] = bad;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s_e[threadIdx.x] += s_e[threadIdx.x + w];
            s_d[threadIdx.x] = max(s_d[threadIdx.x], s_d[threadIdx.x + w]);
            s_n[threadIdx.x] += s_n[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&red[0], s_e[0]);
        atomicMax(reinterpret_cast<unsigned long long*>(&red[1]), s_d[0]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&red[2]), (unsigned long long)s_n[0]);
    }
}

static int blocks_for(size_t n, int bs) { return (int)((n + bs - 1) / bs); }

tc_status launch_solve(tc_plan* p, int set, double2* x, int nfields, cudaStream_t s) {
    Geo g = geo(p);
    const int n = nfields * g.nmode;
    { const int slot_ = prof_begin(p, set == kSetP ? kKSolveP : kKSolveH, s); k_band_solve<<<blocks_for(n, 128), 128, 0, s>>>(x, p->d_fac, p->d_piv, set, nfields, g); prof_end(p, slot_, s); }
    TC_LAUNCHED(p, "k_band_solve");
    return TC_OK;
}

tc_status launch_advance(tc_plan* p, const double2* u, double2* u_prev, const double2* Ncur,
                         double2* N_prev, double2* p_out, double2* u_out, char* ws, bool commit,
                         cudaStream_t s) {
    Geo g = geo(p);
    double2* ps = reinterpret_cast<double2*>(ws + p->ws.pstar);
    double2* us = reinterpret_cast<double2*>(ws + p->ws.ustar);
    double2* phi = reinterpret_cast<double2*>(ws + p->ws.phi);
    const int bs = 256;
    { const int slot_ = prof_begin(p, kKRhsPressure, s); k_rhs_pressure<<<blocks_for(g.S, bs), bs, 0, s>>>(u, u_prev, Ncur, N_prev, ps, p->d_r, p->d_w1, p->d_w2, p->d_col0, g); prof_end(p, slot_, s); }
    TC_LAUNCHED(p, "k_rhs_pressure");
    tc_status st = launch_solve(p, kSetP, ps, 1, s);
    if (st != TC_OK) return st;
    { const int slot_ = prof_begin(p, kKRhsVelocity, s); k_rhs_velocity<<<blocks_for(3 * g.S, bs), bs, 0, s>>>(u, u_prev, Ncur, N_prev, ps, us, p->d_r, p->d_w1, p->d_col0, p->Re_i, p->Re_o, g); prof_end(p, slot_, s); }
    TC_LAUNCHED(p, "k_rhs_velocity");
    st = launch_solve(p, kSetHp, us, 3, s);
    if (st != TC_OK) return st;
    { const int slot_ = prof_begin(p, kKRhsDiv, s); k_rhs_div<<<blocks_for(g.S, bs), bs, 0, s>>>(us, phi, p->d_r, p->d_w1, p->d_col0, g); prof_end(p, slot_, s); }
    TC_LAUNCHED(p, "k_rhs_div");
    st = launch_solve(p, kSetP, phi, 1, s);
    if (st != TC_OK) return st;
    { const int slot_ = prof_begin(p, kKUpdate, s); k_update<<<blocks_for(3 * g.S, bs), bs, 0, s>>>(const_cast<double2*>(u), u_prev, Ncur, N_prev, p_out, us, ps, phi, u_out,
                                                    p->d_r, p->d_w1, p->d_col0, commit ? 1 : 0, g); prof_end(p, slot_, s); }
    TC_LAUNCHED(p, "k_update");
    return TC_OK;
}

tc_status launch_axpby(tc_plan* p, double2* y, const double2* a, double ca, const double2* b,
                       double cb, size_t n, cudaStream_t s) {
    { const int slot_ = prof_begin(p, kKAxpby, s); k_axpby<<<blocks_for(n, 256), 256, 0, s>>>(y, a, ca, b, cb, n); prof_end(p, slot_, s); }
    TC_LAUNCHED(p, "k_axpby");
    return TC_OK;
}

tc_status launch_diagnostics(tc_plan* p, const double2* u, double* red, cudaStream_t s) {
    Geo g = geo(p);
    const double eta = p->eta;
    const double C1 = (p->Re_o - eta * p->Re_i) / (1.0 + eta);
    const double C2 = eta * (p->Re_i - eta * p->Re_o) / ((1.0 - eta) * (1.0 - eta * eta));
    TC_CUDA(p, cudaMemsetAsync(red, 0, 4 * sizeof(double), s));
    { const int slot_ = prof_begin(p, kKDiag, s); k_diag<<<blocks_for(g.S, 256), 256, 0, s>>>(u, red, p->d_r, p->d_w1, p->d_col0, C1, C2, g); prof_end(p, slot_, s); }
    TC_LAUNCHED(p, "k_diag");
    return TC_OK;
}

}  // namespace tc
