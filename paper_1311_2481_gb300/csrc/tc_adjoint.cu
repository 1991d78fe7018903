// Adjoint of the AB2BD2 step (differentiation form; the paper has no adjoint).  The step maps
// (u^i, u^{i-1}, N^{i-1}) -> (u^{i+1}, u^i, N^i) and is affine except for N(u) = u . grad u,
// so its adjoint is the transposed chain of the linear part (steps 2-5 of Sec. 3.2:
// transposed banded solves, transposed stencils) plus the transposed linearised nonlinear
// term about the forward state (transposed forward transforms = unscaled inverse transforms
// and vice versa, the transposed pointwise products, the transposed radial stencil).  The
// inner product is the Euclidean one on the stored (Re, Im) pairs.
#include "tc_fft_core.cuh"
#include "tc_fftc.cuh"
#include "tc_solve_core.cuh"

namespace tc {

static int ablocks(size_t n, int bs) { return (int)((n + bs - 1) / bs); }

// x <- A^{-T} x on one real part of column t of a [N][T] smem array, for A = P L U stored
// as in smem_band_solve: first U^T y = x (forward), then for j = N-1..0 the transposed
// elimination x_j -= sum_q l_q(j) x_{j+q} followed by the row interchange j <-> j + piv_j.
// The factors of the next kPCDepth rows are kept in flight in a register ring (as in
// smem_band_solve).
__device__ __forceinline__ void smem_band_solve_T(double2* col, int T, int t, int part, int N,
                                                  const double* __restrict__ F,
                                                  const uint8_t* __restrict__ P, int M1K1) {
    constexpr int D = kPCDepth;
    double* x = reinterpret_cast<double*>(col) + 2 * t + part;
    const int st = 2 * T;
    // U^T y = b: y_j = (b_j - sum_{q=1..8} U(j-q, j) y_{j-q}) / U_jj, column-oriented: p0..p7
    // hold the partial sums of rows j .. j+7, and y_j is taken out of rows j+1 .. j+8 as soon
    // as it is known, with U(j, j+q) = band 4+q of row j (one FMA and one multiply between
    // consecutive y)
    const size_t rs = (size_t)kBands * M1K1;
    double p0 = N > 0 ? x[0] : 0.0, p1 = N > 1 ? x[(size_t)st] : 0.0, p2 = N > 2 ? x[(size_t)2 * st] : 0.0;
    double p3 = N > 3 ? x[(size_t)3 * st] : 0.0, p4 = N > 4 ? x[(size_t)4 * st] : 0.0;
    double p5 = N > 5 ? x[(size_t)5 * st] : 0.0, p6 = N > 6 ? x[(size_t)6 * st] : 0.0;
    double p7 = N > 7 ? x[(size_t)7 * st] : 0.0;
    double ur[D][9];
#pragma unroll
    for (int d = 0; d < D; ++d)
#pragma unroll
        for (int q = 0; q < 9; ++q) ur[d][q] = d < N ? __ldg(&F[(size_t)d * rs + (size_t)(4 + q) * M1K1]) : 0.0;
    for (int j0 = 0; j0 < N; j0 += D) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int j = j0 + d;
            if (j < N) {
                double u[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) u[q] = ur[d][q];
                if (j + D < N) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) ur[d][q] = __ldg(&F[(size_t)(j + D) * rs + (size_t)(4 + q) * M1K1]);
                }
                const double yj = p0 * u[0];
                x[(size_t)j * st] = yj;
                const double p8 = j + 8 < N ? x[(size_t)(j + 8) * st] : 0.0;
                p0 = fma(-u[1], yj, p1);
                p1 = fma(-u[2], yj, p2);
                p2 = fma(-u[3], yj, p3);
                p3 = fma(-u[4], yj, p4);
                p4 = fma(-u[5], yj, p5);
                p5 = fma(-u[6], yj, p6);
                p6 = fma(-u[7], yj, p7);
                p7 = fma(-u[8], yj, p8);
            }
        }
    }
    // transposed eliminations and interchanges, j = N-1 .. 0; w1..w4 hold x_{j+1..j+4}
    double w1 = 0.0, w2 = 0.0, w3 = 0.0, w4 = 0.0;
    double lr[D][4];
    int pr[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int j = N - 1 - d;
        pr[d] = j >= 0 ? P[(size_t)j * M1K1] : 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) lr[d][q] = j >= 0 ? __ldg(&F[(size_t)j * rs + (size_t)q * M1K1]) : 0.0;
    }
    for (int j0 = N - 1; j0 >= 0; j0 -= D) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int j = j0 - d;
            if (j >= 0) {
                const double l1 = lr[d][0], l2 = lr[d][1], l3 = lr[d][2], l4 = lr[d][3];
                const int pj = pr[d];
                if (j - D >= 0) {
                    pr[d] = P[(size_t)(j - D) * M1K1];
#pragma unroll
                    for (int q = 0; q < 4; ++q) lr[d][q] = __ldg(&F[(size_t)(j - D) * rs + (size_t)q * M1K1]);
                }
                double w0 = x[(size_t)j * st];
                // oldest values first: without an interchange at row j+1 only w1 is new
                w0 = fma(-l4, w4, w0);
                w0 = fma(-l3, w3, w0);
                w0 = fma(-l2, w2, w0);
                w0 = fma(-l1, w1, w0);
                if (pj == 1) { double q = w0; w0 = w1; w1 = q; }
                else if (pj == 2) { double q = w0; w0 = w2; w2 = q; }
                else if (pj == 3) { double q = w0; w0 = w3; w3 = q; }
                else if (pj == 4) { double q = w0; w0 = w4; w4 = q; }
                if (j + 4 < N) x[(size_t)(j + 4) * st] = w4;   // x_{j+4} is final
                w4 = w3; w3 = w2; w2 = w1; w1 = w0;
            }
        }
    }
    // flush the window: x_0..x_3
    if (N > 0) x[0] = w1;
    if (N > 1) x[(size_t)st] = w2;
    if (N > 2) x[(size_t)2 * st] = w3;
    if (N > 3) x[(size_t)3 * st] = w4;
}

// (D1^T v)(c) for column t of smem array C ([N][T]): gather over the rows whose stencil
// holds c, from the host-built table (row, weight) padded with zero weights.
__device__ __forceinline__ double2 sdrowT(const double2* C, const int* __restrict__ trow,
                                          const double* __restrict__ tw, int ntab, int c, int T, int t) {
    double2 s = make_double2(0.0, 0.0);
    for (int e = 0; e < ntab; ++e) {
        const double w = __ldg(&tw[c * ntab + e]);
        const double2 v = C[__ldg(&trow[c * ntab + e]) * T + t];
        s.x = fma(w, v.x, s.x);
        s.y = fma(w, v.y, s.y);
    }
    return s;
}

struct PCAdjArgs {
    const double2* ubar_new;   // adjoint of u^{i+1}
    const double2* ubar_cur;   // adjoint of u^i from the later step (may be null: zero)
    const double2* Nbar_cur;   // adjoint of N^i from the later step (may be null: zero)
    double2* u_out;            // ubar_cur + linear-part adjoint of u^i (nonlinear part added later)
    double2* up_out;           // adjoint of u^{i-1}
    double2* N_out;            // total adjoint of N^i (input of the transposed nonlinear term)
    double2* Np_out;           // adjoint of N^{i-1}
    const double* ir;   // 1 / r_j
    const double* w1;
    const double* w2;
    const int* col0;
    const int* trow;
    const double* tw;
    int ntab;
    const double* fac;
    const uint8_t* piv;
};

// Adjoint of k_pc (steps 2-5 of Sec. 3.2), phases in reverse order.  Shared memory as in
// k_pc: C0 scalar column, C1..C3 vector columns, [N][T] each.
__global__ void __launch_bounds__(256) k_pc_adj(PCAdjArgs a, Geo g, int T) {
    extern __shared__ double2 sm[];
    const int N = g.N;
    const int items = N * T;
    double2* C0 = sm;
    double2* C1 = sm + items;
    double2* C2 = C1 + items;
    double2* C3 = C2 + items;
    double2* Cv[3] = {C1, C2, C3};
    const int mode0 = blockIdx.x * T;
    const int nT = min(T, g.nmode - mode0);
    const size_t per_set = (size_t)N * kBands * g.M1K1;
    const double dt = g.dt;
    auto minfo = [&](int t, int& m, int& k) {
        const int mode = mode0 + t;
        m = mode / g.nk;
        k = mode - m * g.nk - g.K;
    };

    // G': u*bar = ubar_new; phibar = -grad_h^T ubar_new
    for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
        const int j = idx / T, t = idx - (idx / T) * T;
        double2 v0 = make_double2(0.0, 0.0), v1 = v0, v2 = v0;
        if (t < nT) {
            const size_t e = (size_t)j * g.nmode + mode0 + t;
            v0 = a.ubar_new[e];
            v1 = a.ubar_new[g.S + e];
            v2 = a.ubar_new[2 * g.S + e];
        }
        C1[idx] = v0;
        C2[idx] = v1;
        C3[idx] = v2;
    }
    __syncthreads();
    // grad_h^T g = D1^T(g_+ + g_-) - m m_p (g_+ - g_-)/r - i k k_z g_z  (into C0, negated)
    auto gradT = [&](int j, int t) {
        int m, k;
        minfo(t, m, k);
        const double2 dp = sdrowT(C1, a.trow, a.tw, a.ntab, j, T, t);
        const double2 dm = sdrowT(C2, a.trow, a.tw, a.ntab, j, T, t);
        const double2 gp = C1[j * T + t], gm = C2[j * T + t], gz = C3[j * T + t];
        const double mm = g.mp * m * a.ir[j], kk = g.kz * k;
        double2 o;
        o.x = dp.x + dm.x - mm * (gp.x - gm.x) + kk * gz.y;
        o.y = dp.y + dm.y - mm * (gp.y - gm.y) - kk * gz.x;
        return o;
    };
    for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
        const int j = idx / T, t = idx - (idx / T) * T;
        double2 o = make_double2(0.0, 0.0);
        if (t < nT) {
            const double2 q = gradT(j, t);
            o = make_double2(-q.x, -q.y);
        }
        C0[idx] = o;
    }
    __syncthreads();
    // F': bbar = P^{-T} phibar, wall rows carry no dependence
    if (threadIdx.x < 2 * nT) {
        const int t = threadIdx.x >> 1, part = threadIdx.x & 1;
        int m, k;
        minfo(t, m, k);
        const size_t mk = (size_t)m * g.K1 + (k < 0 ? -k : k);
        smem_band_solve_T(C0, T, t, part, N, a.fac + (size_t)kSetP * per_set + mk,
                          a.piv + (size_t)kSetP * N * g.M1K1 + mk, g.M1K1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        C0[t] = make_double2(0.0, 0.0);
        C0[(N - 1) * T + t] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    // E': u*bar += div_h^T bbar:  t = D1^T b + b/r;  +: t/2 + m m_p b/(2r), -: t/2 - .., z: -i k k_z b
    for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
        const int j = idx / T, t = idx - (idx / T) * T;
        if (t >= nT) continue;
        int m, k;
        minfo(t, m, k);
        const double ir = a.ir[j];
        const double2 d = sdrowT(C0, a.trow, a.tw, a.ntab, j, T, t);
        const double2 b = C0[idx];
        const double2 tt = make_double2(d.x + b.x * ir, d.y + b.y * ir);
        const double mm = 0.5 * g.mp * m * ir, kk = g.kz * k;
        double2 v;
        v = C1[idx]; v.x += 0.5 * tt.x + mm * b.x; v.y += 0.5 * tt.y + mm * b.y; C1[idx] = v;
        v = C2[idx]; v.x += 0.5 * tt.x - mm * b.x; v.y += 0.5 * tt.y - mm * b.y; C2[idx] = v;
        v = C3[idx]; v.x += kk * b.y; v.y -= kk * b.x; C3[idx] = v;
    }
    __syncthreads();
    // D': rhsbar_c = H_c^{-T} u*bar_c; wall rows of rhs are constants
    if (threadIdx.x < 6 * nT) {
        const int c = threadIdx.x / (2 * nT), rem = threadIdx.x - c * 2 * nT;
        const int t = rem >> 1, part = rem & 1;
        int m, k;
        minfo(t, m, k);
        const size_t mk = (size_t)m * g.K1 + (k < 0 ? -k : k);
        const int set = kSetHp + c;
        smem_band_solve_T(Cv[c], T, t, part, N, a.fac + (size_t)set * per_set + mk,
                          a.piv + (size_t)set * N * g.M1K1 + mk, g.M1K1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x)
        for (int c = 0; c < 3; ++c) {
            Cv[c][t] = make_double2(0.0, 0.0);
            Cv[c][(N - 1) * T + t] = make_double2(0.0, 0.0);
        }
    __syncthreads();
    // C': ubar += (4/(2dt)) rhsbar, up_bar = -rhsbar/(2dt); p*bar = -grad_h^T rhsbar (C0)
    for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
        const int j = idx / T, t = idx - (idx / T) * T;
        double2 o = make_double2(0.0, 0.0);
        if (t < nT) {
            const size_t e = (size_t)j * g.nmode + mode0 + t;
            for (int c = 0; c < 3; ++c) {
                const size_t ec = (size_t)c * g.S + e;
                const double2 rb = Cv[c][idx];
                double2 ub = a.ubar_cur ? a.ubar_cur[ec] : make_double2(0.0, 0.0);
                ub.x += 2.0 / dt * rb.x;
                ub.y += 2.0 / dt * rb.y;
                a.u_out[ec] = ub;
                a.up_out[ec] = make_double2(-rb.x / (2.0 * dt), -rb.y / (2.0 * dt));
            }
            const double2 q = gradT(j, t);
            o = make_double2(-q.x, -q.y);
        }
        C0[idx] = o;
    }
    __syncthreads();
    // NNbar = -rhsbar (in place)
    for (int idx = threadIdx.x; idx < 3 * items; idx += blockDim.x) {
        double2* C = Cv[idx / items];
        const int r = idx % items;
        C[r] = make_double2(-C[r].x, -C[r].y);
    }
    __syncthreads();
    // B': bpbar = P^{-T} p*bar
    if (threadIdx.x < 2 * nT) {
        const int t = threadIdx.x >> 1, part = threadIdx.x & 1;
        int m, k;
        minfo(t, m, k);
        const size_t mk = (size_t)m * g.K1 + (k < 0 ? -k : k);
        smem_band_solve_T(C0, T, t, part, N, a.fac + (size_t)kSetP * per_set + mk,
                          a.piv + (size_t)kSetP * N * g.M1K1 + mk, g.M1K1);
    }
    __syncthreads();
    // A': interior rows b_p = div_h(-NN): NNbar += div_h^T(-bpbar_interior);
    //     wall rows b_p = -NN_r + 2 Lap_r(u) - Lap_r(u_prev) (not the (0,0) row at r_o)
    for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
        const int j = idx / T, t = idx - (idx / T) * T;
        if (t >= nT) continue;
        int m, k;
        minfo(t, m, k);
        const double ir = a.ir[j];
        // v = -bpbar on interior rows, 0 on wall rows
        double2 d = make_double2(0.0, 0.0);
        for (int e = 0; e < a.ntab; ++e) {
            const int row = __ldg(&a.trow[j * a.ntab + e]);
            if (row == 0 || row == N - 1) continue;
            const double w = __ldg(&a.tw[j * a.ntab + e]);
            const double2 b = C0[row * T + t];
            d.x -= w * b.x;
            d.y -= w * b.y;
        }
        double2 v = make_double2(0.0, 0.0);
        if (j > 0 && j < N - 1) v = make_double2(-C0[idx].x, -C0[idx].y);
        const double2 tt = make_double2(d.x + v.x * ir, d.y + v.y * ir);
        const double mm = 0.5 * g.mp * m * ir, kk = g.kz * k;
        double2 q;
        q = C1[idx]; q.x += 0.5 * tt.x + mm * v.x; q.y += 0.5 * tt.y + mm * v.y;
        if (j == 0 || (j == N - 1 && !(m == 0 && k == 0))) { q.x -= 0.5 * C0[idx].x; q.y -= 0.5 * C0[idx].y; }
        C1[idx] = q;
        q = C2[idx]; q.x += 0.5 * tt.x - mm * v.x; q.y += 0.5 * tt.y - mm * v.y;
        if (j == 0 || (j == N - 1 && !(m == 0 && k == 0))) { q.x -= 0.5 * C0[idx].x; q.y -= 0.5 * C0[idx].y; }
        C2[idx] = q;
        q = C3[idx]; q.x += kk * v.y; q.y -= kk * v.x;
        C3[idx] = q;
    }
    // wall Laplacian transposes: column c of the wall stencils receives, for wall row jw with
    // value w: 1/2 (D2[jw][c] + D1[jw][c]/r_jw) w (+ 1/2 diag_pm w at c = jw), times 2 into
    // ubar and -1 into up_bar.  One thread per (column, mode) of the two wall stencils.
    for (int idx = threadIdx.x; idx < 2 * kStencil * T; idx += blockDim.x) {
        const int side = idx / (kStencil * T);
        const int rem = idx - side * kStencil * T;
        const int q = rem / T, t = rem - (rem / T) * T;
        if (t >= nT) continue;
        int m, k;
        minfo(t, m, k);
        const int jw = side == 0 ? 0 : N - 1;
        if (jw == N - 1 && m == 0 && k == 0) continue;
        const int c = a.col0[jw] + q;
        const double ir = a.ir[jw], ir2 = ir * ir;
        const double wq = 0.5 * (a.w2[jw * kStencil + q] + ir * a.w1[jw * kStencil + q]);
        const double2 w = C0[jw * T + t];
        const double mm = g.mp * m, kk = g.kz * k;
        const size_t e = (size_t)c * g.nmode + mode0 + t;
        for (int cc = 0; cc < 2; ++cc) {
            double coef = wq;
            if (c == jw) {
                const double sgn = cc == 0 ? -1.0 : 1.0;
                coef += 0.5 * (-mm * mm * ir2 - kk * kk - ir2 + sgn * 2.0 * mm * ir2);
            }
            if (coef == 0.0) continue;
            const size_t ec = (size_t)cc * g.S + e;
            // rows of the two wall stencils may share a column only when N_r < 10; the
            // two sides then run in sequence below to keep the read-modify-write race free
            if (side == 1 && N < 2 * kStencil) continue;
            double2 ub = a.u_out[ec], pb = a.up_out[ec];
            ub.x += 2.0 * coef * w.x; ub.y += 2.0 * coef * w.y;
            pb.x -= coef * w.x; pb.y -= coef * w.y;
            a.u_out[ec] = ub;
            a.up_out[ec] = pb;
        }
    }
    __syncthreads();
    if (N < 2 * kStencil) {   // second wall for small N_r, after the first
        for (int idx = threadIdx.x; idx < kStencil * T; idx += blockDim.x) {
            const int q = idx / T, t = idx - (idx / T) * T;
            if (t >= nT) continue;
            int m, k;
            minfo(t, m, k);
            const int jw = N - 1;
            if (m == 0 && k == 0) continue;
            const int c = a.col0[jw] + q;
            const double ir = a.ir[jw], ir2 = ir * ir;
            const double wq = 0.5 * (a.w2[jw * kStencil + q] + ir * a.w1[jw * kStencil + q]);
            const double2 w = C0[jw * T + t];
            const double mm = g.mp * m, kk = g.kz * k;
            const size_t e = (size_t)c * g.nmode + mode0 + t;
            for (int cc = 0; cc < 2; ++cc) {
                double coef = wq;
                if (c == jw) {
                    const double sgn = cc == 0 ? -1.0 : 1.0;
                    coef += 0.5 * (-mm * mm * ir2 - kk * kk - ir2 + sgn * 2.0 * mm * ir2);
                }
                if (coef == 0.0) continue;
                const size_t ec = (size_t)cc * g.S + e;
                double2 ub = a.u_out[ec], pb = a.up_out[ec];
                ub.x += 2.0 * coef * w.x; ub.y += 2.0 * coef * w.y;
                pb.x -= coef * w.x; pb.y -= coef * w.y;
                a.u_out[ec] = ub;
                a.up_out[ec] = pb;
            }
        }
        __syncthreads();
    }
    // NN = 2N - N_prev:  Nbar = Nbar_cur + 2 NNbar,  Np_bar = -NNbar
    for (int idx = threadIdx.x; idx < 3 * items; idx += blockDim.x) {
        const int c = idx / items, rem = idx - c * items;
        const int j = rem / T, t = rem - (rem / T) * T;
        if (t >= nT) continue;
        const size_t ec = (size_t)c * g.S + (size_t)j * g.nmode + mode0 + t;
        const double2 nn = Cv[c][rem];
        double2 nb = a.Nbar_cur ? a.Nbar_cur[ec] : make_double2(0.0, 0.0);
        nb.x += 2.0 * nn.x;
        nb.y += 2.0 * nn.y;
        a.N_out[ec] = nb;
        a.Np_out[ec] = make_double2(-nn.x, -nn.y);
    }
}

// ---------------------------------------------------------------- transposed steps 2-5, per stage
// The same phases as k_pc_adj as one kernel per stage over all modes, for large N_r: each
// column lives in global memory, so every transposed substitution runs on its own thread
// (mode, real / imaginary part) with full warps, where k_pc_adj would hold few modes per
// block.  Scratch: US (3 fields), PH and PS (one each), the forward split path's buffers.
// A wall row of PH, US or PS holds no dependence after its solve and is read as zero.

struct AdjT {
    const double* ir;
    const int* trow;
    const double* tw;
    int ntab;
};

// sum_e D1[row_e][j] f(row_e) over the rows whose stencil holds column j; wall rows of f
// dropped when `walls` is false
__device__ __forceinline__ double2 growT(const double2* __restrict__ f, const AdjT& a, int j, int nmode,
                                         int mode, int N, bool walls) {
    double2 s = make_double2(0.0, 0.0);
    for (int e = 0; e < a.ntab; ++e) {
        const int row = __ldg(&a.trow[j * a.ntab + e]);
        if (!walls && (row == 0 || row == N - 1)) continue;
        const double w = __ldg(&a.tw[j * a.ntab + e]);
        const double2 v = f[(size_t)row * nmode + mode];
        s.x = fma(w, v.x, s.x);
        s.y = fma(w, v.y, s.y);
    }
    return s;
}

// grad_h^T of the vector field v at (j, mode), negated: -(D1^T(v_+ + v_-) - m m_p (v_+ - v_-)/r
// - i k k_z v_z); wall rows of v read as zero unless `walls`
__device__ __forceinline__ double2 neg_gradT(const double2* __restrict__ v, const AdjT& a, const Geo& g, int j,
                                             int mode, bool walls) {
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const double2 dp = growT(v, a, j, g.nmode, mode, g.N, walls);
    const double2 dm = growT(v + g.S, a, j, g.nmode, mode, g.N, walls);
    const bool wall = j == 0 || j == g.N - 1;
    const size_t e = (size_t)j * g.nmode + mode;
    const double2 z0 = make_double2(0.0, 0.0);
    const double2 gp = (walls || !wall) ? v[e] : z0, gm = (walls || !wall) ? v[g.S + e] : z0;
    const double2 gz = (walls || !wall) ? v[2 * g.S + e] : z0;
    const double mm = g.mp * m * a.ir[j], kk = g.kz * k;
    return make_double2(-(dp.x + dm.x - mm * (gp.x - gm.x) + kk * gz.y),
                        -(dp.y + dm.y - mm * (gp.y - gm.y) - kk * gz.x));
}

// G': PH = -grad_h^T ubar_new
__global__ void k_adjT_phi(const double2* __restrict__ ubn, double2* __restrict__ PH, AdjT a, Geo g) {
    const int mode = blockIdx.y * blockDim.x + threadIdx.x;   // x = radial row
    if (mode >= g.nmode) return;
    const int j = blockIdx.x;
    PH[(size_t)j * g.nmode + mode] = neg_gradT(ubn, a, g, j, mode, true);
}

// E': US = ubar_new + div_h^T PH (PH's wall rows zero)
__global__ void k_adjT_ustar(const double2* __restrict__ ubn, const double2* __restrict__ PH,
                             double2* __restrict__ US, AdjT a, Geo g) {
    const int mode = blockIdx.y * blockDim.x + threadIdx.x;
    if (mode >= g.nmode) return;
    const int j = blockIdx.x;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const size_t e = (size_t)j * g.nmode + mode;
    const double ir = a.ir[j];
    const double2 d = growT(PH, a, j, g.nmode, mode, g.N, false);
    const double2 b = (j == 0 || j == g.N - 1) ? make_double2(0.0, 0.0) : PH[e];
    const double2 tt = make_double2(d.x + b.x * ir, d.y + b.y * ir);
    const double mm = 0.5 * g.mp * m * ir, kk = g.kz * k;
    double2 v;
    v = ubn[e]; v.x += 0.5 * tt.x + mm * b.x; v.y += 0.5 * tt.y + mm * b.y; US[e] = v;
    v = ubn[g.S + e]; v.x += 0.5 * tt.x - mm * b.x; v.y += 0.5 * tt.y - mm * b.y; US[g.S + e] = v;
    v = ubn[2 * g.S + e]; v.x += kk * b.y; v.y -= kk * b.x; US[2 * g.S + e] = v;
}

// C': with rb = US (wall rows zero): u_out = ubar_cur + (2/dt) rb, up_out = -rb/(2 dt),
// PS = -grad_h^T rb.  u_out may alias ubar_new (no longer read) and up_out ubar_cur (read
// first, by the same thread).
__global__ void k_adjT_rhs(const double2* __restrict__ US, const double2* ubc, double2* u_out, double2* up_out,
                           double2* __restrict__ PS, AdjT a, Geo g) {
    const int mode = blockIdx.y * blockDim.x + threadIdx.x;
    if (mode >= g.nmode) return;
    const int j = blockIdx.x;
    const size_t e = (size_t)j * g.nmode + mode;
    const bool wall = j == 0 || j == g.N - 1;
    const double dt = g.dt;
    for (int c = 0; c < 3; ++c) {
        const size_t ec = (size_t)c * g.S + e;
        const double2 rb = wall ? make_double2(0.0, 0.0) : US[ec];
        double2 ub = ubc ? ubc[ec] : make_double2(0.0, 0.0);
        ub.x += 2.0 / dt * rb.x;
        ub.y += 2.0 / dt * rb.y;
        u_out[ec] = ub;
        up_out[ec] = make_double2(-rb.x / (2.0 * dt), -rb.y / (2.0 * dt));
    }
    PS[e] = neg_gradT(US, a, g, j, mode, false);
}

// A': NNbar = -rb + div_h^T(-bpbar on interior rows) and the wall-row terms of Eq. ppBC;
// N_out = Nbar_cur + 2 NNbar, Np_out = -NNbar (Np_out may alias Nbar_cur: same thread)
__global__ void k_adjT_nn(const double2* __restrict__ US, const double2* __restrict__ PS, const double2* Nbc,
                          double2* N_out, double2* Np_out, AdjT a, Geo g) {
    const int mode = blockIdx.y * blockDim.x + threadIdx.x;
    if (mode >= g.nmode) return;
    const int j = blockIdx.x;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const size_t e = (size_t)j * g.nmode + mode;
    const int N = g.N;
    const bool wall = j == 0 || j == N - 1;
    const double ir = a.ir[j];
    const double2 dd = growT(PS, a, j, g.nmode, mode, N, false);
    const double2 d = make_double2(-dd.x, -dd.y);
    const double2 bp = PS[e];
    const double2 v = wall ? make_double2(0.0, 0.0) : make_double2(-bp.x, -bp.y);
    const double2 tt = make_double2(d.x + v.x * ir, d.y + v.y * ir);
    const double mm = 0.5 * g.mp * m * ir, kk = g.kz * k;
    const bool wterm = j == 0 || (j == N - 1 && !(m == 0 && k == 0));
    double2 q[3];
    for (int c = 0; c < 3; ++c) {
        const double2 rb = wall ? make_double2(0.0, 0.0) : US[(size_t)c * g.S + e];
        q[c] = make_double2(-rb.x, -rb.y);
    }
    q[0].x += 0.5 * tt.x + mm * v.x; q[0].y += 0.5 * tt.y + mm * v.y;
    q[1].x += 0.5 * tt.x - mm * v.x; q[1].y += 0.5 * tt.y - mm * v.y;
    if (wterm) {
        q[0].x -= 0.5 * bp.x; q[0].y -= 0.5 * bp.y;
        q[1].x -= 0.5 * bp.x; q[1].y -= 0.5 * bp.y;
    }
    q[2].x += kk * v.y; q[2].y -= kk * v.x;
    for (int c = 0; c < 3; ++c) {
        const size_t ec = (size_t)c * g.S + e;
        double2 nb = Nbc ? Nbc[ec] : make_double2(0.0, 0.0);
        nb.x += 2.0 * q[c].x;
        nb.y += 2.0 * q[c].y;
        N_out[ec] = nb;
        Np_out[ec] = make_double2(-q[c].x, -q[c].y);
    }
}

// Wall Laplacian transposes of Eq. ppBC's wall rows (side 0: r_i, 1: r_o; `sides` of them
// from `side0`): column c of the wall stencil receives 1/2 (D2 + D1/r)[jw][c] bpbar(jw)
// (+ the diagonal terms at c = jw), times 2 into u_out and -1 into up_out, for the + and -
// components.  One thread per (side, stencil column, mode); the two sides touch the same
// columns only when N_r < 18, and then run as two launches.
__global__ void k_adjT_wall(const double2* __restrict__ PS, double2* u_out, double2* up_out,
                            const double* __restrict__ w1, const double* __restrict__ w2,
                            const int* __restrict__ col0, AdjT a, Geo g, int side0) {
    const int mode = blockIdx.x * blockDim.x + threadIdx.x;
    if (mode >= g.nmode) return;
    const int q = blockIdx.y;
    const int side = side0 + blockIdx.z;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const int jw = side == 0 ? 0 : g.N - 1;
    if (jw == g.N - 1 && m == 0 && k == 0) return;
    const int c = col0[jw] + q;
    const double ir = a.ir[jw], ir2 = ir * ir;
    const double wq = 0.5 * (w2[jw * kStencil + q] + ir * w1[jw * kStencil + q]);
    const double2 w = PS[(size_t)jw * g.nmode + mode];
    const double mm = g.mp * m, kk = g.kz * k;
    const size_t e = (size_t)c * g.nmode + mode;
    for (int cc = 0; cc < 2; ++cc) {
        double coef = wq;
        if (c == jw) {
            const double sgn = cc == 0 ? -1.0 : 1.0;
            coef += 0.5 * (-mm * mm * ir2 - kk * kk - ir2 + sgn * 2.0 * mm * ir2);
        }
        if (coef == 0.0) continue;
        const size_t ec = (size_t)cc * g.S + e;
        double2 ub = u_out[ec], pb = up_out[ec];
        ub.x += 2.0 * coef * w.x; ub.y += 2.0 * coef * w.y;
        pb.x -= coef * w.x; pb.y -= coef * w.y;
        u_out[ec] = ub;
        up_out[ec] = pb;
    }
}

// x <- A^{-T} x for every mode of nfields consecutive fields (sets set0, set0 + 1, ...):
// thread (field, mode, part) runs the transposed substitution down its global column
__global__ void k_band_solve_gT(double2* __restrict__ x, const double* __restrict__ fac,
                                const uint8_t* __restrict__ piv, int set0, Geo g) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;   // (mode, part); y = field
    if (t >= 2 * g.nmode) return;
    const int part = t & 1;
    const int mode = t >> 1;
    const int fld = blockIdx.y;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const size_t mk = (size_t)m * g.K1 + (k < 0 ? -k : k);
    const size_t per_set = (size_t)g.N * kBands * g.M1K1;
    const int set = set0 + fld;
    smem_band_solve_T(x + (size_t)fld * g.S, g.nmode, mode, part, g.N, fac + (size_t)set * per_set + mk,
                      piv + (size_t)set * g.N * g.M1K1 + mk, g.M1K1);
}

// ---------------------------------------------------------------- transposed nonlinear term
// Transposed forward transform: a physical field x = (1/(P_t P_z)) Re sum_{m>=0,k} w e^{i phi};
// with the C2R convention (weight 2 for m > 0) the lines carry w/2 for m > 0.  Lines per
// (r, m): s_r = (Nbar_+ + Nbar_-), s_t = -i (Nbar_+ - Nbar_-), s_z = Nbar_z.
__global__ void __launch_bounds__(256) k_zinv_adjin(const double2* __restrict__ Nb, double2* __restrict__ H,
                                                    int N_r, int M, int K, double scale,
                                                    const double2* __restrict__ tw, Radices rad, int r0, int nh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Pz = rad.n;
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + (size_t)3 * Pz;
    const int m = blockIdx.x % (M + 1);
    const int rl = blockIdx.x / (M + 1);
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    const size_t o = ((size_t)(r0 + rl) * (M + 1) + m) * nk;
    const double cm = (m == 0 ? 1.0 : 0.5) * scale;
    for (int idx = threadIdx.x; idx < 3 * Pz; idx += blockDim.x) {
        const int l = idx / Pz, q = idx - l * Pz;
        const int k = q <= K ? q : q - Pz;
        double2 v = make_double2(0.0, 0.0);
        if (k >= -K && k <= K) {
            const size_t e = o + (k + K);
            if (l == 0) { const double2 p = Nb[e], n = Nb[S + e]; v = make_double2(p.x + n.x, p.y + n.y); }
            else if (l == 1) { const double2 p = Nb[e], n = Nb[S + e]; v = make_double2(p.y - n.y, -(p.x - n.x)); }
            else v = Nb[2 * S + e];
            v.x *= cm;
            v.y *= cm;
        }
        a[idx] = v;
    }
    __syncthreads();
    double2* res = smem_fft(a, b, 3, tw, true, rad);
    const size_t fstride = (size_t)nh * (M + 1) * Pz;
    for (int idx = threadIdx.x; idx < 3 * Pz; idx += blockDim.x) {
        const int l = idx / Pz, z = idx - l * Pz;
        H[l * fstride + ((size_t)rl * (M + 1) + m) * Pz + z] = res[idx];
    }
}

// Per (r, z tile): recompute the 12 forward physical fields (6 lines per z as in k_theta),
// the 3 adjoint physical fields (1 line (s_r, s_t) per z, s_z two z per line), the
// transposed products, and the transposed inverse theta transform (unscaled forward DFT
// times c_m) of the 12 adjoint fields as 6 paired lines.  Output per (r, m, z), 9 lines in
// the (+, -, z) basis: A (u, with -i m m_p d_theta folded in), R (d_r), Z (d_z).
__global__ void __launch_bounds__(256) k_theta_adj(const double2* __restrict__ H1, const double2* __restrict__ Ha,
                                                   double2* __restrict__ H3, const double* __restrict__ irn,
                                                   int r0, int nh, int M, int Pz, double mp, int zt,
                                                   const double2* __restrict__ tw, Radices rad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Pt = rad.n;
    const int nza = (zt + 1) / 2;
    const int nl = 7 * zt + nza;               // 6 forward + 1 (s_r, s_t) per z + s_z pairs
    const int nbuf = nl > 6 * zt ? nl : 6 * zt;
    double2* A = reinterpret_cast<double2*>(smem_raw);
    double2* B = A + (size_t)nbuf * Pt;
    const int tiles = Pz / zt;
    const int r = blockIdx.x / tiles;   // row within the staged rows r0 .. r0 + nh - 1
    const int z0 = (blockIdx.x % tiles) * zt;
    const size_t fstride = (size_t)nh * (M + 1) * Pz;
    const double2* h = H1 + (size_t)r * (M + 1) * Pz + z0;
    const double2* ha = Ha + (size_t)r * (M + 1) * Pz + z0;

    for (int idx = threadIdx.x; idx < nl * Pt; idx += blockDim.x) A[idx] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < (7 * zt + nza) * (M + 1); idx += blockDim.x) {
        const int m = idx % (M + 1);
        const int L = idx / (M + 1);
        const double mm = mp * m;
        double2* line = A + (size_t)L * Pt;
        if (L < 6 * zt) {   // forward lines, as in k_theta
            const int zi = L / 6, pr = L - 6 * (L / 6);
            const size_t o = (size_t)m * Pz + zi;
            if (pr < 4) {
                const int fa = pr == 0 ? 0 : pr == 1 ? 3 : pr == 2 ? 0 : 6;
                double2 Av = h[fa * fstride + o], Bv = h[(fa + 1) * fstride + o];
                if (pr == 2) { Av = make_double2(-mm * Av.y, mm * Av.x); Bv = make_double2(-mm * Bv.y, mm * Bv.x); }
                if (m == 0) line[0] = make_double2(0.5 * (Av.x + Bv.x), 0.5 * (Av.y - Bv.y));
                else { line[m] = Av; line[Pt - m] = cconj(Bv); }
            } else {
                double2 X, Y;
                if (pr == 4) { X = h[2 * fstride + o]; Y = h[5 * fstride + o]; }
                else { X = h[2 * fstride + o]; X = make_double2(-mm * X.y, mm * X.x); Y = h[8 * fstride + o]; }
                if (m == 0) line[0] = make_double2(X.x, Y.x);
                else {
                    line[m] = make_double2(X.x - Y.y, X.y + Y.x);
                    line[Pt - m] = make_double2(X.x + Y.y, Y.x - X.y);
                }
            }
        } else if (L < 7 * zt) {   // adjoint (s_r, s_t) as two real fields
            const int zi = L - 6 * zt;
            const size_t o = (size_t)m * Pz + zi;
            const double2 X = ha[o], Y = ha[fstride + o];
            if (m == 0) line[0] = make_double2(X.x, Y.x);
            else {
                line[m] = make_double2(X.x - Y.y, X.y + Y.x);
                line[Pt - m] = make_double2(X.x + Y.y, Y.x - X.y);
            }
        } else {                   // s_z of z values 2i and 2i+1
            const int zp = L - 7 * zt;
            const int za = 2 * zp, zb = 2 * zp + 1;
            const double2 X = ha[2 * fstride + (size_t)m * Pz + za];
            const double2 Y = zb < zt ? ha[2 * fstride + (size_t)m * Pz + zb] : make_double2(0.0, 0.0);
            if (m == 0) line[0] = make_double2(X.x, Y.x);
            else {
                line[m] = make_double2(X.x - Y.y, X.y + Y.x);
                line[Pt - m] = make_double2(X.x + Y.y, Y.x - X.y);
            }
        }
    }
    __syncthreads();
    double2* phys = smem_fft(A, B, nl, tw, true, rad);
    double2* out = phys == A ? B : A;
    const double ir = irn[r0 + r];   // 1 / r_j from the plan
    for (int idx = threadIdx.x; idx < zt * Pt; idx += blockDim.x) {
        const int zi = idx / Pt, th = idx - zi * Pt;
        const double2* L0 = phys + (size_t)(zi * 6) * Pt + th;
        const double2 p0 = L0[0], p1 = L0[Pt], p2 = L0[2 * Pt], p3 = L0[3 * Pt], p4 = L0[4 * Pt], p5 = L0[5 * Pt];
        const double2 an = phys[(size_t)(6 * zt + zi) * Pt + th];
        const double2 az = phys[(size_t)(7 * zt + zi / 2) * Pt + th];
        const double nr = an.x, nt = an.y, nz = (zi & 1) ? az.y : az.x;
        const double ur = p0.x, ut = p0.y, uz = p4.x;
        const double urr = p1.x, utr = p1.y, urt = p2.x, utt = p2.y, urz = p3.x, utz = p3.y;
        const double uzr = p4.y, uzt = p5.x, uzz = p5.y;
        const double utr_ = ut * ir;
        const double b_ur = nr * urr + nt * (utr + utr_) + nz * uzr;
        const double b_ut = (nr * (urt - 2.0 * ut) + nt * (utt + ur) + nz * uzt) * ir;
        const double b_uz = nr * urz + nt * utz + nz * uzz;
        double2* o = out + (size_t)(zi * 6) * Pt + th;
        o[0] = make_double2(b_ur, b_ut);                     // pair 0: (u_r, u_t)
        o[Pt] = make_double2(b_uz, ur * nz);                 // pair 1: (u_z, d_r u_z)
        o[2 * Pt] = make_double2(ur * nr, ur * nt);          // pair 2: (d_r u_r, d_r u_t)
        o[3 * Pt] = make_double2(utr_ * nr, utr_ * nt);      // pair 3: (d_t u_r, d_t u_t)
        o[4 * Pt] = make_double2(utr_ * nz, uz * nz);        // pair 4: (d_t u_z, d_z u_z)
        o[5 * Pt] = make_double2(uz * nr, uz * nt);          // pair 5: (d_z u_r, d_z u_t)
    }
    __syncthreads();
    double2* spare = out == A ? B : A;
    double2* spec = smem_fft(out, spare, 6 * zt, tw, false, rad);
    const size_t S9 = fstride;
    for (int idx = threadIdx.x; idx < zt * (M + 1); idx += blockDim.x) {
        const int m = idx / zt, zi = idx - m * zt;
        const double cmw = m == 0 ? 1.0 : 2.0;
        const double mm = mp * m;
        double2 X[6], Y[6];
        for (int pr = 0; pr < 6; ++pr) {
            const double2* Ls = spec + (size_t)(zi * 6 + pr) * Pt;
            const double2 Cp = Ls[m], Cm = cconj(Ls[m ? Pt - m : 0]);
            X[pr] = make_double2(0.5 * cmw * (Cp.x + Cm.x), 0.5 * cmw * (Cp.y + Cm.y));
            Y[pr] = make_double2(0.5 * cmw * (Cp.y - Cm.y), 0.5 * cmw * (Cm.x - Cp.x));
        }
        // A_c = G^T ubar_{u_c} - i m m_p G^T ubar_{d_t u_c}; R_c = G^T ubar_{d_r u_c}; Z_c = G^T ubar_{d_z u_c}
        const double2 Ar = make_double2(X[0].x + mm * X[3].y, X[0].y - mm * X[3].x);
        const double2 At = make_double2(Y[0].x + mm * Y[3].y, Y[0].y - mm * Y[3].x);
        const double2 Az = make_double2(X[1].x + mm * X[4].y, X[1].y - mm * X[4].x);
        const double2 Rr = X[2], Rt = Y[2], Rz = Y[1];
        const double2 Zr = X[5], Zt = Y[5], Zz = Y[4];
        // (r, t, z) -> (+, -, z):  bar_+ = a_r/2 + i a_t/2,  bar_- = a_r/2 - i a_t/2
        auto plus = [](double2 ar, double2 at) { return make_double2(0.5 * (ar.x - at.y), 0.5 * (ar.y + at.x)); };
        auto minus = [](double2 ar, double2 at) { return make_double2(0.5 * (ar.x + at.y), 0.5 * (ar.y - at.x)); };
        const size_t o = ((size_t)r * (M + 1) + m) * Pz + z0 + zi;
        H3[0 * S9 + o] = plus(Ar, At);
        H3[1 * S9 + o] = minus(Ar, At);
        H3[2 * S9 + o] = Az;
        H3[3 * S9 + o] = plus(Rr, Rt);
        H3[4 * S9 + o] = minus(Rr, Rt);
        H3[5 * S9 + o] = Rz;
        H3[6 * S9 + o] = plus(Zr, Zt);
        H3[7 * S9 + o] = minus(Zr, Zt);
        H3[8 * S9 + o] = Zz;
    }
}

// Length-specialised form of k_theta_adj: compile-time radix plans (radices <= 8) over padded
// lines; same fields, products and outputs.
template <int PT, int ZT, int NT>
__global__ void __launch_bounds__(NT) k_theta_adj_s(const double2* __restrict__ H1, const double2* __restrict__ Ha,
                                                   double2* __restrict__ H3, const double* __restrict__ irn,
                                                   int r0, int nh, int M, int Pz, double mp,
                                                   const double2* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int Pt = PT, zt = ZT;
    constexpr int LP = cft::padded<PT>();
    constexpr int nza = (ZT + 1) / 2;
    constexpr int nl = 7 * ZT + nza;           // 6 forward + 1 (s_r, s_t) per z + s_z pairs
    constexpr int nbuf = nl > 6 * ZT ? nl : 6 * ZT;
    double2* A = reinterpret_cast<double2*>(smem_raw);
    double2* B = A + (size_t)nbuf * LP;
    const int tiles = Pz / zt;
    const int r = blockIdx.x / tiles;   // row within the staged rows r0 .. r0 + nh - 1
    const int z0 = (blockIdx.x % tiles) * zt;
    const size_t fstride = (size_t)nh * (M + 1) * Pz;
    const double2* h = H1 + (size_t)r * (M + 1) * Pz + z0;
    const double2* ha = Ha + (size_t)r * (M + 1) * Pz + z0;

    for (int idx = threadIdx.x; idx < nl * LP; idx += NT) A[idx] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < (7 * zt + nza) * (M + 1); idx += NT) {
        const int m = idx % (M + 1);
        const int L = idx / (M + 1);
        const double mm = mp * m;
        double2* line = A + (size_t)L * LP;
        if (L < 6 * zt) {   // forward lines, as in k_theta
            const int zi = L / 6, pr = L - 6 * (L / 6);
            const size_t o = (size_t)m * Pz + zi;
            if (pr < 4) {
                const int fa = pr == 0 ? 0 : pr == 1 ? 3 : pr == 2 ? 0 : 6;
                double2 Av = h[fa * fstride + o], Bv = h[(fa + 1) * fstride + o];
                if (pr == 2) { Av = make_double2(-mm * Av.y, mm * Av.x); Bv = make_double2(-mm * Bv.y, mm * Bv.x); }
                if (m == 0) line[0] = make_double2(0.5 * (Av.x + Bv.x), 0.5 * (Av.y - Bv.y));
                else { line[cft::pd(m)] = Av; line[cft::pd(Pt - m)] = cconj(Bv); }
            } else {
                double2 X, Y;
                if (pr == 4) { X = h[2 * fstride + o]; Y = h[5 * fstride + o]; }
                else { X = h[2 * fstride + o]; X = make_double2(-mm * X.y, mm * X.x); Y = h[8 * fstride + o]; }
                if (m == 0) line[0] = make_double2(X.x, Y.x);
                else {
                    line[cft::pd(m)] = make_double2(X.x - Y.y, X.y + Y.x);
                    line[cft::pd(Pt - m)] = make_double2(X.x + Y.y, Y.x - X.y);
                }
            }
        } else if (L < 7 * zt) {   // adjoint (s_r, s_t) as two real fields
            const int zi = L - 6 * zt;
            const size_t o = (size_t)m * Pz + zi;
            const double2 X = ha[o], Y = ha[fstride + o];
            if (m == 0) line[0] = make_double2(X.x, Y.x);
            else {
                line[cft::pd(m)] = make_double2(X.x - Y.y, X.y + Y.x);
                line[cft::pd(Pt - m)] = make_double2(X.x + Y.y, Y.x - X.y);
            }
        } else {                   // s_z of z values 2i and 2i+1
            const int zp = L - 7 * zt;
            const int za = 2 * zp, zb = 2 * zp + 1;
            const double2 X = ha[2 * fstride + (size_t)m * Pz + za];
            const double2 Y = zb < zt ? ha[2 * fstride + (size_t)m * Pz + zb] : make_double2(0.0, 0.0);
            if (m == 0) line[0] = make_double2(X.x, Y.x);
            else {
                line[cft::pd(m)] = make_double2(X.x - Y.y, X.y + Y.x);
                line[cft::pd(Pt - m)] = make_double2(X.x + Y.y, Y.x - X.y);
            }
        }
    }
    __syncthreads();
    const double2* phys = cft::passes<PT, 0, 1, nl, NT, true, double2, true>(A, B, tw);
    double2* out = phys == A ? B : A;
    const double ir = irn[r0 + r];   // 1 / r_j from the plan
    for (int idx = threadIdx.x; idx < zt * Pt; idx += NT) {
        const int zi = idx / Pt, th = idx - zi * Pt;
        const int pth = cft::pd(th);
        const double2* L0 = phys + (size_t)(zi * 6) * LP + pth;
        const double2 p0 = L0[0], p1 = L0[LP], p2 = L0[2 * LP], p3 = L0[3 * LP], p4 = L0[4 * LP], p5 = L0[5 * LP];
        const double2 an = phys[(size_t)(6 * zt + zi) * LP + pth];
        const double2 az = phys[(size_t)(7 * zt + zi / 2) * LP + pth];
        const double nr = an.x, nt = an.y, nz = (zi & 1) ? az.y : az.x;
        const double ur = p0.x, ut = p0.y, uz = p4.x;
        const double urr = p1.x, utr = p1.y, urt = p2.x, utt = p2.y, urz = p3.x, utz = p3.y;
        const double uzr = p4.y, uzt = p5.x, uzz = p5.y;
        const double utr_ = ut * ir;
        const double b_ur = nr * urr + nt * (utr + utr_) + nz * uzr;
        const double b_ut = (nr * (urt - 2.0 * ut) + nt * (utt + ur) + nz * uzt) * ir;
        const double b_uz = nr * urz + nt * utz + nz * uzz;
        double2* o = out + (size_t)(zi * 6) * LP + pth;
        o[0] = make_double2(b_ur, b_ut);                     // pair 0: (u_r, u_t)
        o[LP] = make_double2(b_uz, ur * nz);                 // pair 1: (u_z, d_r u_z)
        o[2 * LP] = make_double2(ur * nr, ur * nt);          // pair 2: (d_r u_r, d_r u_t)
        o[3 * LP] = make_double2(utr_ * nr, utr_ * nt);      // pair 3: (d_t u_r, d_t u_t)
        o[4 * LP] = make_double2(utr_ * nz, uz * nz);        // pair 4: (d_t u_z, d_z u_z)
        o[5 * LP] = make_double2(uz * nr, uz * nt);          // pair 5: (d_z u_r, d_z u_t)
    }
    __syncthreads();
    double2* spare = out == A ? B : A;
    const double2* spec = cft::passes<PT, 0, 1, 6 * ZT, NT, false, double2, true>(out, spare, tw);
    const size_t S9 = fstride;
    for (int idx = threadIdx.x; idx < zt * (M + 1); idx += NT) {
        const int m = idx / zt, zi = idx - m * zt;
        const double cmw = m == 0 ? 1.0 : 2.0;
        const double mm = mp * m;
        double2 X[6], Y[6];
        for (int pr = 0; pr < 6; ++pr) {
            const double2* Ls = spec + (size_t)(zi * 6 + pr) * LP;
            const double2 Cp = Ls[cft::pd(m)], Cm = cconj(Ls[cft::pd(m ? Pt - m : 0)]);
            X[pr] = make_double2(0.5 * cmw * (Cp.x + Cm.x), 0.5 * cmw * (Cp.y + Cm.y));
            Y[pr] = make_double2(0.5 * cmw * (Cp.y - Cm.y), 0.5 * cmw * (Cm.x - Cp.x));
        }
        // A_c = G^T ubar_{u_c} - i m m_p G^T ubar_{d_t u_c}; R_c = G^T ubar_{d_r u_c}; Z_c = G^T ubar_{d_z u_c}
        const double2 Ar = make_double2(X[0].x + mm * X[3].y, X[0].y - mm * X[3].x);
        const double2 At = make_double2(Y[0].x + mm * Y[3].y, Y[0].y - mm * Y[3].x);
        const double2 Az = make_double2(X[1].x + mm * X[4].y, X[1].y - mm * X[4].x);
        const double2 Rr = X[2], Rt = Y[2], Rz = Y[1];
        const double2 Zr = X[5], Zt = Y[5], Zz = Y[4];
        // (r, t, z) -> (+, -, z):  bar_+ = a_r/2 + i a_t/2,  bar_- = a_r/2 - i a_t/2
        auto plus = [](double2 ar, double2 at) { return make_double2(0.5 * (ar.x - at.y), 0.5 * (ar.y + at.x)); };
        auto minus = [](double2 ar, double2 at) { return make_double2(0.5 * (ar.x + at.y), 0.5 * (ar.y - at.x)); };
        const size_t o = ((size_t)r * (M + 1) + m) * Pz + z0 + zi;
        H3[0 * S9 + o] = plus(Ar, At);
        H3[1 * S9 + o] = minus(Ar, At);
        H3[2 * S9 + o] = Az;
        H3[3 * S9 + o] = plus(Rr, Rt);
        H3[4 * S9 + o] = minus(Rr, Rt);
        H3[5 * S9 + o] = Rz;
        H3[6 * S9 + o] = plus(Zr, Zt);
        H3[7 * S9 + o] = minus(Zr, Zt);
        H3[8 * S9 + o] = Zz;
    }
}

// Per (r, m, component c): unscaled forward DFT along z of A_c, R_c, Z_c, truncation to
// |k| <= K; ubar_c += A_c - i k k_z Z_c;  Rhat_c = R_c (transposed stencil applied next).
// Rhat holds the nh staged rows r0 .. r0 + nh - 1.
__global__ void __launch_bounds__(256) k_zfwd_adj(const double2* __restrict__ H3, double2* __restrict__ ub,
                                                  double2* __restrict__ Rh, int N_r, int M, int K, double kz,
                                                  const double2* __restrict__ tw, Radices rad, int r0, int nh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Pz = rad.n;
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + (size_t)3 * Pz;
    const int c = blockIdx.x % 3;
    const int rm = blockIdx.x / 3;
    const int m = rm % (M + 1), rl = rm / (M + 1);
    const size_t fstride = (size_t)nh * (M + 1) * Pz;
    const double2* h = H3 + ((size_t)rl * (M + 1) + m) * Pz;
    for (int idx = threadIdx.x; idx < 3 * Pz; idx += blockDim.x) {
        const int l = idx / Pz, z = idx - l * Pz;   // l: 0 A, 1 R, 2 Z of component c
        a[idx] = h[(size_t)(3 * l + c) * fstride + z];
    }
    __syncthreads();
    double2* res = smem_fft(a, b, 3, tw, false, rad);
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    const size_t Sh = (size_t)nh * (M + 1) * nk;
    for (int kk = threadIdx.x; kk < nk; kk += blockDim.x) {
        const int k = kk - K;
        const int q = k < 0 ? k + Pz : k;
        const double2 Av = res[q], Rv = res[Pz + q], Zv = res[2 * Pz + q];
        const double kzk = kz * k;
        const size_t e = (size_t)c * S + ((size_t)(r0 + rl) * (M + 1) + m) * nk + kk;
        double2 u = ub[e];
        u.x += Av.x + kzk * Zv.y;
        u.y += Av.y - kzk * Zv.x;
        ub[e] = u;
        Rh[(size_t)c * Sh + ((size_t)rl * (M + 1) + m) * nk + kk] = Rv;
    }
}

// Length-specialised forms of k_zinv_adjin and k_zfwd_adj: compile-time radix plans
// (radices <= 8) over padded lines; same inputs, outputs and arithmetic.
template <int PZ, int NT>
__global__ void __launch_bounds__(NT) k_zinv_adjin_s(const double2* __restrict__ Nb, double2* __restrict__ H,
                                                     int N_r, int M, int K, double scale,
                                                     const double2* __restrict__ tw, int r0, int nh) {
    constexpr int LP = cft::padded<PZ>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + 3 * LP;
    const int m = blockIdx.x % (M + 1);
    const int rl = blockIdx.x / (M + 1);
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    const size_t o = ((size_t)(r0 + rl) * (M + 1) + m) * nk;
    const double cm = (m == 0 ? 1.0 : 0.5) * scale;
    for (int q = threadIdx.x; q < PZ; q += NT) {
        const int k = q <= K ? q : q - PZ;
        if (k < -K) continue;                      // zero band, not read by the first pass
        const size_t e = o + (k + K);
        const double2 p = Nb[e], n = Nb[S + e], zz = Nb[2 * S + e];
        a[cft::pd(q)] = make_double2(cm * (p.x + n.x), cm * (p.y + n.y));
        a[LP + cft::pd(q)] = make_double2(cm * (p.y - n.y), -cm * (p.x - n.x));
        a[2 * LP + cft::pd(q)] = make_double2(cm * zz.x, cm * zz.y);
    }
    __syncthreads();
    const double2* X = cft::passes<PZ, 0, 1, 3, NT, true, double2, true>(a, b, tw, K + 1, PZ - K);
    const size_t fstride = (size_t)nh * (M + 1) * PZ;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        double2* dst = H + l * fstride + ((size_t)rl * (M + 1) + m) * PZ;
        for (int z = threadIdx.x; z < PZ; z += NT) dst[z] = X[l * LP + cft::pd(z)];
    }
}

template <int PZ, int NT>
__global__ void __launch_bounds__(NT) k_zfwd_adj_s(const double2* __restrict__ H3, double2* __restrict__ ub,
                                                   double2* __restrict__ Rh, int N_r, int M, int K, double kz,
                                                   const double2* __restrict__ tw, int r0, int nh) {
    constexpr int LP = cft::padded<PZ>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + 3 * LP;
    const int c = blockIdx.x % 3;
    const int rm = blockIdx.x / 3;
    const int m = rm % (M + 1), rl = rm / (M + 1);
    const size_t fstride = (size_t)nh * (M + 1) * PZ;
    const double2* h = H3 + ((size_t)rl * (M + 1) + m) * PZ;
#pragma unroll
    for (int l = 0; l < 3; ++l)   // l: 0 A, 1 R, 2 Z of component c
        for (int z = threadIdx.x; z < PZ; z += NT) a[l * LP + cft::pd(z)] = h[(size_t)(3 * l + c) * fstride + z];
    __syncthreads();
    const double2* X = cft::passes<PZ, 0, 1, 3, NT, false, double2, true>(a, b, tw);
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    const size_t Sh = (size_t)nh * (M + 1) * nk;
    for (int kk = threadIdx.x; kk < nk; kk += NT) {
        const int k = kk - K;
        const int q = cft::pd(k < 0 ? k + PZ : k);
        const double2 Av = X[q], Rv = X[LP + q], Zv = X[2 * LP + q];
        const double kzk = kz * k;
        const size_t e = (size_t)c * S + ((size_t)(r0 + rl) * (M + 1) + m) * nk + kk;
        double2 u = ub[e];
        u.x += Av.x + kzk * Zv.y;
        u.y += Av.y - kzk * Zv.x;
        ub[e] = u;
        Rh[(size_t)c * Sh + ((size_t)rl * (M + 1) + m) * nk + kk] = Rv;
    }
}

// Streamed form of the transposed theta pass for long lines: two lines per z are resident at
// a time instead of eight, as in the forward k_theta_s, so 1152-point FP64 lines fit a block.
// Inverse phases, two lines per z each:
//   0: (s_r, s_t), (u_r, u_t)        1: (s_z, 0), (u_z, d_r u_z)
//   2: (d_r u_r, d_r u_t), (d_t u_r, d_t u_t)      3: (d_z u_r, d_z u_t), (d_t u_z, d_z u_z)
// Each physical point is owned by one thread in every phase, which keeps there (n_r, n_t),
// (u_r, u_t / r), n_z, u_z and the transposed products that need the gradient lines:
//   b_r = n_r d_r u_r + n_t (d_r u_t + u_t / r) + n_z d_r u_z,
//   r b_t = n_r (d_t u_r - 2 u_t) + n_t (d_t u_t + u_r) + n_z d_t u_z,
//   b_z = n_r d_z u_r + n_t d_z u_t + n_z d_z u_z.
// Forward phases transform the six output pairs of k_theta_adj two per z, grouped so that
// each group alone fixes the H3 fields it writes: (o2, o5) -> R_+-, Z_+-; (o0, o3) -> A_+-;
// (o1, o4) -> A_z, R_z, Z_z.
template <int PT, int ZT, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_theta_adj_st(const double2* __restrict__ H1,
                                                          const double2* __restrict__ Ha,
                                                          double2* __restrict__ H3, const double* __restrict__ irn,
                                                          int r0, int nh, int M, int Pz, double mp,
                                                          const double2* __restrict__ tw) {
    using V = double2;
    constexpr int LP = cft::padded<PT>();
    constexpr int NL = 2 * ZT;   // resident lines
    constexpr int NPT = ZT * PT; // physical points of the block
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* A = reinterpret_cast<V*>(smem_raw);
    V* B = A + NL * LP;
    V* Nv = B + NL * LP;   // (n_r, n_t)
    V* Uu = Nv + NPT;      // (u_r, u_t / r)
    V* Ac = Uu + NPT;      // (b_r, r b_t)
    double* Nz = reinterpret_cast<double*>(Ac + NPT);
    double* Uz = Nz + NPT;
    double* Bz = Uz + NPT;
    const int tiles = Pz / ZT;
    const int r = blockIdx.x / tiles;   // row within the staged rows r0 .. r0 + nh - 1
    const int z0 = (blockIdx.x % tiles) * ZT;
    const size_t fstride = (size_t)nh * (M + 1) * Pz;
    const V* h = H1 + (size_t)r * (M + 1) * Pz + z0;
    const V* ha = Ha + (size_t)r * (M + 1) * Pz + z0;
    const double ir = irn[r0 + r];   // 1 / r_j from the plan
    const int zi = threadIdx.x % ZT;
    const int mstep = NT / ZT;

#pragma unroll 1
    for (int phase = 0; phase < 4; ++phase) {
        V* L0 = A + (2 * zi) * LP;
        V* L1 = L0 + LP;
        for (int m = (int)threadIdx.x / ZT; m <= M; m += mstep) {
            const size_t o = (size_t)m * Pz + zi;
            const double mm = mp * m;
            if (phase == 0) {
                cft::put_real2(L0, PT, m, ha[o], ha[fstride + o]);
                cft::put_pair(L1, PT, m, h[o], h[fstride + o]);
            } else if (phase == 1) {
                cft::put_real2(L0, PT, m, ha[2 * fstride + o], make_double2(0.0, 0.0));
                cft::put_real2(L1, PT, m, h[2 * fstride + o], h[5 * fstride + o]);
            } else if (phase == 2) {
                cft::put_pair(L0, PT, m, h[3 * fstride + o], h[4 * fstride + o]);
                cft::put_pair(L1, PT, m, cft::imul(h[o], mm), cft::imul(h[fstride + o], mm));
            } else {
                cft::put_pair(L0, PT, m, h[6 * fstride + o], h[7 * fstride + o]);
                cft::put_real2(L1, PT, m, cft::imul(h[2 * fstride + o], mm), h[8 * fstride + o]);
            }
        }
        __syncthreads();
        // the band M < p < PT - M of every line is zero: the first pass does not read it
        const V* X = cft::passes<PT, 0, 1, NL, NT, true, V, true>(A, B, tw, M + 1, PT - M);
        for (int pt = threadIdx.x; pt < NPT; pt += NT) {
            const int z = pt / PT;
            const int th = pt - z * PT;
            const V p0 = X[(2 * z) * LP + cft::pd(th)];
            const V p1 = X[(2 * z + 1) * LP + cft::pd(th)];
            if (phase == 0) {          // p0 = (n_r, n_t), p1 = (u_r, u_t)
                const double utr = p1.y * ir;
                Nv[pt] = p0;
                Uu[pt] = make_double2(p1.x, utr);
                Ac[pt] = make_double2(p0.y * utr, p0.y * p1.x - 2.0 * p0.x * p1.y);
            } else if (phase == 1) {   // p0 = (n_z, 0), p1 = (u_z, d_r u_z)
                Nz[pt] = p0.x;
                Uz[pt] = p1.x;
                Ac[pt].x += p0.x * p1.y;
            } else if (phase == 2) {   // p0 = d_r (u_r, u_t), p1 = d_t (u_r, u_t)
                const V n = Nv[pt];
                V c = Ac[pt];
                c.x += n.x * p0.x + n.y * p0.y;
                c.y += n.x * p1.x + n.y * p1.y;
                Ac[pt] = c;
            } else {                   // p0 = d_z (u_r, u_t), p1 = (d_t u_z, d_z u_z)
                const V n = Nv[pt];
                const double nz = Nz[pt];
                Bz[pt] = n.x * p0.x + n.y * p0.y + nz * p1.y;
                Ac[pt].y += nz * p1.x;
            }
        }
        __syncthreads();   // the next fill overwrites the lines
    }

    const size_t S9 = fstride;
    auto plus = [](double2 ar, double2 at) { return make_double2(0.5 * (ar.x - at.y), 0.5 * (ar.y + at.x)); };
    auto minus = [](double2 ar, double2 at) { return make_double2(0.5 * (ar.x + at.y), 0.5 * (ar.y - at.x)); };
#pragma unroll 1
    for (int fp = 0; fp < 3; ++fp) {
        for (int pt = threadIdx.x; pt < NPT; pt += NT) {
            const int z = pt / PT;
            const int th = pt - z * PT;
            const V n = Nv[pt], uu = Uu[pt];
            V a, b;
            if (fp == 0) {
                const double uz = Uz[pt];
                a = make_double2(uu.x * n.x, uu.x * n.y);         // o2: (d_r u_r, d_r u_t)
                b = make_double2(uz * n.x, uz * n.y);             // o5: (d_z u_r, d_z u_t)
            } else if (fp == 1) {
                const V c = Ac[pt];
                a = make_double2(c.x, c.y * ir);                  // o0: (u_r, u_t)
                b = make_double2(uu.y * n.x, uu.y * n.y);         // o3: (d_t u_r, d_t u_t)
            } else {
                const double nz = Nz[pt];
                a = make_double2(Bz[pt], uu.x * nz);              // o1: (u_z, d_r u_z)
                b = make_double2(uu.y * nz, Uz[pt] * nz);         // o4: (d_t u_z, d_z u_z)
            }
            A[(2 * z) * LP + cft::pd(th)] = a;
            A[(2 * z + 1) * LP + cft::pd(th)] = b;
        }
        __syncthreads();
        const V* Y = cft::passes<PT, 0, 1, NL, NT, false, V, true>(A, B, tw);
        for (int idx = threadIdx.x; idx < ZT * (M + 1); idx += NT) {
            const int m = idx / ZT, z = idx - m * ZT;
            const double cmw = m == 0 ? 1.0 : 2.0;
            const double mm = mp * m;
            V Xl[2], Yl[2];
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const V* Ls = Y + (2 * z + l) * LP;
                const V Cp = Ls[cft::pd(m)], Cm = cconj(Ls[cft::pd(m ? PT - m : 0)]);
                Xl[l] = make_double2(0.5 * cmw * (Cp.x + Cm.x), 0.5 * cmw * (Cp.y + Cm.y));
                Yl[l] = make_double2(0.5 * cmw * (Cp.y - Cm.y), 0.5 * cmw * (Cm.x - Cp.x));
            }
            const size_t o = ((size_t)r * (M + 1) + m) * Pz + z0 + z;
            if (fp == 0) {
                H3[3 * S9 + o] = plus(Xl[0], Yl[0]);
                H3[4 * S9 + o] = minus(Xl[0], Yl[0]);
                H3[6 * S9 + o] = plus(Xl[1], Yl[1]);
                H3[7 * S9 + o] = minus(Xl[1], Yl[1]);
            } else if (fp == 1) {
                const V Ar = make_double2(Xl[0].x + mm * Xl[1].y, Xl[0].y - mm * Xl[1].x);
                const V At = make_double2(Yl[0].x + mm * Yl[1].y, Yl[0].y - mm * Yl[1].x);
                H3[0 * S9 + o] = plus(Ar, At);
                H3[1 * S9 + o] = minus(Ar, At);
            } else {
                H3[2 * S9 + o] = make_double2(Xl[0].x + mm * Xl[1].y, Xl[0].y - mm * Xl[1].x);
                H3[5 * S9 + o] = Yl[0];
                H3[8 * S9 + o] = Yl[1];
            }
        }
        __syncthreads();   // the next fill overwrites the lines
    }
}

template <int PZ, int NT>
static tc_status zadj_s(tc_plan* p, const double2* Nbar, double2* Ha, const double2* H3, double2* ubar,
                        double2* Rh, cudaStream_t s, bool inverse, int r0, int nh) {
    const size_t sm = (size_t)2 * 3 * cft::padded<PZ>() * sizeof(double2);
    if (inverse) {
        TC_CUDA(p, cudaFuncSetAttribute(k_zinv_adjin_s<PZ, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const int slot = prof_begin(p, kKZinvAdj, s);
        k_zinv_adjin_s<PZ, NT><<<nh * (p->M + 1), NT, sm, s>>>(Nbar, Ha, p->N_r, p->M, p->K,
                                                               1.0 / ((double)p->P_t * (double)p->P_z), p->d_tw_z,
                                                               r0, nh);
        prof_end(p, slot, s);
        TC_LAUNCHED(p, "k_zinv_adjin_s");
    } else {
        TC_CUDA(p, cudaFuncSetAttribute(k_zfwd_adj_s<PZ, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const int slot = prof_begin(p, kKZfwdAdj, s);
        k_zfwd_adj_s<PZ, NT><<<nh * (p->M + 1) * 3, NT, sm, s>>>(H3, ubar, Rh, p->N_r, p->M, p->K, p->k_z,
                                                                 p->d_tw_z, r0, nh);
        prof_end(p, slot, s);
        TC_LAUNCHED(p, "k_zfwd_adj_s");
    }
    return TC_OK;
}

static bool zadj_ok(const tc_plan* p) {
    return p->theta_zt_forced == 0 &&
           (p->P_z == 48 || p->P_z == 96 || p->P_z == 192 || p->P_z == 384 || p->P_z == 768);
}

// specialised adjoint z passes where P_z has a compile-time plan (TC_ERR_ARG otherwise)
static tc_status zadj_dispatch(tc_plan* p, const double2* Nbar, double2* Ha, const double2* H3, double2* ubar,
                               double2* Rh, cudaStream_t s, bool inverse, int r0, int nh) {
    if (p->theta_zt_forced != 0) return TC_ERR_ARG;
    switch (p->P_z) {
        case 48: return zadj_s<48, 128>(p, Nbar, Ha, H3, ubar, Rh, s, inverse, r0, nh);
        case 96: return zadj_s<96, 128>(p, Nbar, Ha, H3, ubar, Rh, s, inverse, r0, nh);
        case 192: return zadj_s<192, 256>(p, Nbar, Ha, H3, ubar, Rh, s, inverse, r0, nh);
        case 384: return zadj_s<384, 256>(p, Nbar, Ha, H3, ubar, Rh, s, inverse, r0, nh);
        case 768: return zadj_s<768, 256>(p, Nbar, Ha, H3, ubar, Rh, s, inverse, r0, nh);
    }
    return TC_ERR_ARG;
}

// ubar(c, j, mode) += sum over the staged rows i = r0 .. r0 + nh - 1 of D1[i][j] Rhat(c, i, mode)
// for the columns j = j0 .. j0 + gridDim.x - 1 (the columns those rows' stencils reach)
__global__ void k_drT(double2* __restrict__ ub, const double2* __restrict__ Rh, const int* __restrict__ trow,
                      const double* __restrict__ tw, int ntab, Geo g, int r0, int nh, int j0) {
    // grid: x = radial column (fastest: the gathered rows stay in cache), y over modes, z = component
    const int mode = blockIdx.y * blockDim.x + threadIdx.x;
    if (mode >= g.nmode) return;
    const int j = j0 + blockIdx.x, c = blockIdx.z;
    const size_t e = (size_t)c * g.S + (size_t)j * g.nmode + mode;
    const size_t Sh = (size_t)nh * g.nmode;
    double2 s = ub[e];
    for (int q = 0; q < ntab; ++q) {
        const int i = __ldg(&trow[j * ntab + q]) - r0;
        if (i < 0 || i >= nh) continue;
        const double w = __ldg(&tw[j * ntab + q]);
        const double2 v = Rh[(size_t)c * Sh + (size_t)i * g.nmode + mode];
        s.x = fma(w, v.x, s.x);
        s.y = fma(w, v.y, s.y);
    }
    ub[e] = s;
}

tc_status launch_adjoint_advance(tc_plan* p, const double2* ubar_new, const double2* ubar_cur,
                                 const double2* Nbar_cur, double2* u_out, double2* up_out,
                                 double2* N_out, double2* Np_out, char* ws, cudaStream_t s) {
    Geo g = geo(p);
    if (p->pc_split) {
        // per-stage transposed steps 2-5 (the forward split path's scratch)
        double2* PS = reinterpret_cast<double2*>(ws + p->ws.pstar);
        double2* US = reinterpret_cast<double2*>(ws + p->ws.ustar);
        double2* PH = reinterpret_cast<double2*>(ws + p->ws.phi);
        AdjT a{p->d_ir, p->d_d1t_row, p->d_d1t_w, p->d1t_n};
        const dim3 g1(g.N, ablocks(g.nmode, 128));
        auto sgrid = [&](int nf) { return dim3(ablocks((size_t)2 * g.nmode, 128), nf); };
        const int slot = prof_begin(p, kKPCAdj, s);
        k_adjT_phi<<<g1, 128, 0, s>>>(ubar_new, PH, a, g);
        k_band_solve_gT<<<sgrid(1), 128, 0, s>>>(PH, p->d_fac, p->d_piv, kSetP, g);
        k_adjT_ustar<<<g1, 128, 0, s>>>(ubar_new, PH, US, a, g);
        k_band_solve_gT<<<sgrid(3), 128, 0, s>>>(US, p->d_fac, p->d_piv, kSetHp, g);
        k_adjT_rhs<<<g1, 128, 0, s>>>(US, ubar_cur, u_out, up_out, PS, a, g);
        k_band_solve_gT<<<sgrid(1), 128, 0, s>>>(PS, p->d_fac, p->d_piv, kSetP, g);
        k_adjT_nn<<<g1, 128, 0, s>>>(US, PS, Nbar_cur, N_out, Np_out, a, g);
        if (g.N >= 2 * kStencil) {
            k_adjT_wall<<<dim3(ablocks(g.nmode, 128), kStencil, 2), 128, 0, s>>>(PS, u_out, up_out, p->d_w1, p->d_w2,
                                                                                p->d_col0, a, g, 0);
        } else {
            for (int side = 0; side < 2; ++side)
                k_adjT_wall<<<dim3(ablocks(g.nmode, 128), kStencil, 1), 128, 0, s>>>(PS, u_out, up_out, p->d_w1,
                                                                                    p->d_w2, p->d_col0, a, g, side);
        }
        prof_end(p, slot, s);
        TC_LAUNCHED(p, "k_adjT");
        return TC_OK;
    }
    int T = p->pc_modes > 0 ? p->pc_modes : 8;
    while (T > 1 && (size_t)4 * p->N_r * T * sizeof(double2) > 96 * 1024) T /= 2;
    PCAdjArgs a;
    a.ubar_new = ubar_new; a.ubar_cur = ubar_cur; a.Nbar_cur = Nbar_cur;
    a.u_out = u_out; a.up_out = up_out; a.N_out = N_out; a.Np_out = Np_out;
    a.ir = p->d_ir; a.w1 = p->d_w1; a.w2 = p->d_w2; a.col0 = p->d_col0;
    a.trow = p->d_d1t_row; a.tw = p->d_d1t_w; a.ntab = p->d1t_n;
    a.fac = p->d_fac; a.piv = p->d_piv;
    const size_t sm = (size_t)4 * p->N_r * T * sizeof(double2);
    int threads = ((6 * T + 31) / 32) * 32;
    if (threads < 128) threads = 128;
    if (threads > 256) threads = 256;
    TC_CUDA(p, cudaFuncSetAttribute(k_pc_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int slot = prof_begin(p, kKPCAdj, s);
    k_pc_adj<<<ablocks(g.nmode, T), threads, sm, s>>>(a, g, T);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_pc_adj");
    return TC_OK;
}

template <int PT, int ZT, int NT>
static tc_status theta_adj_s(tc_plan* p, const double2* H1, const double2* Ha, double2* H3, cudaStream_t s,
                             int r0, int nh) {
    constexpr int nl = 7 * ZT + (ZT + 1) / 2;
    const size_t sm = (size_t)2 * nl * cft::padded<PT>() * sizeof(double2);
    TC_CUDA(p, cudaFuncSetAttribute(k_theta_adj_s<PT, ZT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int slot = prof_begin(p, kKThetaAdj, s);
    k_theta_adj_s<PT, ZT, NT><<<nh * (p->P_z / ZT), NT, sm, s>>>(H1, Ha, H3, p->d_ir, r0, nh, p->M, p->P_z,
                                                                (double)p->m_p, p->d_tw_t);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_theta_adj_s");
    return TC_OK;
}

template <int PT, int ZT, int NT, int MINB>
static tc_status theta_adj_st(tc_plan* p, const double2* H1, const double2* Ha, double2* H3, cudaStream_t s,
                              int r0, int nh) {
    constexpr int LP = cft::padded<PT>();
    const size_t sm = ((size_t)2 * 2 * ZT * LP + (size_t)3 * ZT * PT) * sizeof(double2) +
                      (size_t)3 * ZT * PT * sizeof(double);
    auto kern = k_theta_adj_st<PT, ZT, NT, MINB>;
    TC_CUDA(p, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int slot = prof_begin(p, kKThetaAdj, s);
    kern<<<nh * (p->P_z / ZT), NT, sm, s>>>(H1, Ha, H3, p->d_ir, r0, nh, p->M, p->P_z, (double)p->m_p, p->d_tw_t);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_theta_adj_st");
    return TC_OK;
}

// adjoint theta pass of the staged rows r0 .. r0 + nh - 1: the streamed kernel for 768 and
// 1152 points, the length-specialised one for 96, 192, 384, the generic one otherwise
static tc_status theta_adj(tc_plan* p, const double2* H1, const double2* Ha, double2* H3, cudaStream_t s,
                           int r0, int nh) {
    const bool spec = p->theta_zt_forced == 0 && 2 * p->M + 1 <= p->P_t;
    if (spec && p->P_t == 1152) return theta_adj_st<1152, 1, 384, 1>(p, H1, Ha, H3, s, r0, nh);
    if (spec && p->P_t == 768) return theta_adj_st<768, 1, 256, 2>(p, H1, Ha, H3, s, r0, nh);
    if (spec && (p->P_t == 96 || p->P_t == 192 || p->P_t == 384) && p->P_z % 2 == 0) {
        switch (p->P_t) {
            case 96: return theta_adj_s<96, 2, 256>(p, H1, Ha, H3, s, r0, nh);
            case 192: return theta_adj_s<192, 2, 256>(p, H1, Ha, H3, s, r0, nh);
            default: return theta_adj_s<384, 2, 256>(p, H1, Ha, H3, s, r0, nh);
        }
    }
    int zt = 4;
    auto smem_for = [&](int z) {
        const int nza = (z + 1) / 2, nl = 7 * z + nza;
        const int nbuf = nl > 6 * z ? nl : 6 * z;
        return (size_t)2 * nbuf * p->P_t * sizeof(double2);
    };
    while (zt > 1 && (smem_for(zt) > 200 * 1024 || p->P_z % zt)) zt /= 2;
    if (smem_for(zt) > 220 * 1024) {
        snprintf(p->err, sizeof(p->err), "adjoint theta pass: P_theta = %d too long for shared memory", p->P_t);
        return TC_ERR_ARG;
    }
    const size_t smt = smem_for(zt);
    TC_CUDA(p, cudaFuncSetAttribute(k_theta_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smt));
    const int slot = prof_begin(p, kKThetaAdj, s);
    k_theta_adj<<<nh * (p->P_z / zt), 256, smt, s>>>(H1, Ha, H3, p->d_ir, r0, nh, p->M, p->P_z,
                                                      (double)p->m_p, zt, p->d_tw_t, p->rad_t);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_theta_adj");
    return TC_OK;
}

// ubar += N'(u)^T Nbar, slab by slab of p->stage_rows radial rows: the transposed transforms of
// a row read only that row's staging, and the transposed radial stencil of a slab's Rhat rows
// is added before the next slab overwrites them
tc_status launch_nonlinear_adjoint(tc_plan* p, const double2* u, const double2* Nbar, double2* ubar,
                                   char* ws, cudaStream_t s) {
    Geo g = geo(p);
    double2* H1 = reinterpret_cast<double2*>(ws + p->ws.H1a);
    double2* Ha = reinterpret_cast<double2*>(ws + p->ws.Ha);
    double2* H3 = reinterpret_cast<double2*>(ws + p->ws.H3);
    double2* Rh = reinterpret_cast<double2*>(ws + p->ws.Rhat);
    const size_t smz = (size_t)2 * 3 * p->P_z * sizeof(double2);
    for (int r0 = 0; r0 < p->N_r; r0 += p->stage_rows) {
        const int nh = p->N_r - r0 < p->stage_rows ? p->N_r - r0 : p->stage_rows;
        // forward lines of u (same kernel as the forward nonlinear term, FP64)
        TC_TRY_STATUS(launch_zinv_fp64(p, u, H1, s, r0, nh));
        int slot;
        if (zadj_ok(p)) {
            TC_TRY_STATUS(zadj_dispatch(p, Nbar, Ha, nullptr, nullptr, nullptr, s, true, r0, nh));
        } else {
            TC_CUDA(p, cudaFuncSetAttribute(k_zinv_adjin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smz));
            slot = prof_begin(p, kKZinvAdj, s);
            k_zinv_adjin<<<nh * (p->M + 1), 256, smz, s>>>(Nbar, Ha, p->N_r, p->M, p->K,
                                                            1.0 / ((double)p->P_t * (double)p->P_z), p->d_tw_z,
                                                            p->rad_z, r0, nh);
            prof_end(p, slot, s);
            TC_LAUNCHED(p, "k_zinv_adjin");
        }
        TC_TRY_STATUS(theta_adj(p, H1, Ha, H3, s, r0, nh));
        if (zadj_ok(p)) {
            TC_TRY_STATUS(zadj_dispatch(p, nullptr, nullptr, H3, ubar, Rh, s, false, r0, nh));
        } else {
            TC_CUDA(p, cudaFuncSetAttribute(k_zfwd_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smz));
            slot = prof_begin(p, kKZfwdAdj, s);
            k_zfwd_adj<<<nh * (p->M + 1) * 3, 256, smz, s>>>(H3, ubar, Rh, p->N_r, p->M, p->K, p->k_z,
                                                              p->d_tw_z, p->rad_z, r0, nh);
            prof_end(p, slot, s);
            TC_LAUNCHED(p, "k_zfwd_adj");
        }
        // columns reached by the stencils of rows r0 .. r0 + nh - 1
        int jlo = p->N_r, jhi = -1;
        for (int i = r0; i < r0 + nh; ++i) {
            jlo = p->col0[i] < jlo ? p->col0[i] : jlo;
            jhi = p->col0[i] + kStencil - 1 > jhi ? p->col0[i] + kStencil - 1 : jhi;
        }
        if (jlo < 0) jlo = 0;
        if (jhi > p->N_r - 1) jhi = p->N_r - 1;
        slot = prof_begin(p, kKDrT, s);
        k_drT<<<dim3(jhi - jlo + 1, ablocks(g.nmode, 128), 3), 128, 0, s>>>(ubar, Rh, p->d_d1t_row, p->d_d1t_w,
                                                                            p->d1t_n, g, r0, nh, jlo);
        prof_end(p, slot, s);
        TC_LAUNCHED(p, "k_drT");
    }
    return TC_OK;
}

// gradient of J = 1/2 sum_j w_j r_j sum c_m (|u'_+|^2/2 + |u'_-|^2/2 + |u'_z|^2), u' = u - Couette
__global__ void k_energy_grad(const double2* __restrict__ u, double2* __restrict__ gr,
                              const double* __restrict__ rn, double C1, double C2, Geo g) {
    const int mode = blockIdx.x * blockDim.x + threadIdx.x;
    if (mode >= g.nmode) return;
    const int j = blockIdx.y, c = blockIdx.z;
    const size_t e = (size_t)c * g.S + (size_t)j * g.nmode + mode;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const double r = rn[j];
    double wr = 0.0;
    if (j > 0) wr += 0.5 * (r - rn[j - 1]);
    if (j < g.N - 1) wr += 0.5 * (rn[j + 1] - r);
    double2 d = u[e];
    if (m == 0 && k == 0 && c < 2) d.y -= (c == 0 ? 1.0 : -1.0) * (C1 * r + C2 / r);
    const double f = wr * r * (m == 0 ? 1.0 : 2.0) * (c < 2 ? 0.5 : 1.0);
    gr[e] = make_double2(f * d.x, f * d.y);
}

tc_status launch_energy_gradient(tc_plan* p, const double2* u, double2* gr, cudaStream_t s) {
    Geo g = geo(p);
    const double eta = p->eta;
    const double C1 = (p->Re_o - eta * p->Re_i) / (1.0 + eta);
    const double C2 = eta * (p->Re_i - eta * p->Re_o) / ((1.0 - eta) * (1.0 - eta * eta));
    k_energy_grad<<<dim3(ablocks(g.nmode, 128), g.N, 3), 128, 0, s>>>(u, gr, p->d_r, C1, C2, g);
    TC_LAUNCHED(p, "k_energy_grad");
    return TC_OK;
}

}  // namespace tc

using namespace tc;

namespace {

tc_status adj_ready(tc_plan* p, void* ws) {
    if (!p) return TC_ERR_ARG;
    if (p->host_only) return TC_ERR_STATE;
    if (!p->adjoint) {
        snprintf(p->err, sizeof(p->err), "plan created with no_adjoint: its workspace has no adjoint regions");
        return TC_ERR_STATE;
    }
    int dev = -1;
    TC_CUDA(p, cudaGetDevice(&dev));
    if (dev != p->device) return TC_ERR_STATE;
    if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 != 0) return TC_ERR_ARG;
    return check_device_ptr(p, ws, "ws", p->ws.total);
}

#define TC_TRY2(x)                   \
    do {                             \
        tc_status s_ = (x);          \
        if (s_ != TC_OK) return s_;  \
    } while (0)

}  // namespace

extern "C" {

tc_status tc_adjoint_step(tc_plan* plan, const tc_state* fwd, tc_state_bar* bar, void* ws, void* stream) {
    TC_TRY2(adj_ready(plan, ws));
    if (!fwd || !bar) return TC_ERR_ARG;
    if (!fwd->started) {
        snprintf(plan->err, sizeof(plan->err), "tc_adjoint_step needs a started forward state (use tc_adjoint_start for the cold start)");
        return TC_ERR_STATE;
    }
    const size_t vb = 3 * plan->S * sizeof(double2);
    TC_TRY2(check_device_ptr(plan, fwd->u, "fwd->u", vb));
    TC_TRY2(check_device_ptr(plan, bar->u, "bar->u", vb));
    TC_TRY2(check_device_ptr(plan, bar->u_prev, "bar->u_prev", vb));
    TC_TRY2(check_device_ptr(plan, bar->N_prev, "bar->N_prev", vb));
    if (bar->u == bar->u_prev || bar->u == bar->N_prev || bar->u_prev == bar->N_prev) return TC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    double2* ub = static_cast<double2*>(bar->u);
    double2* upb = static_cast<double2*>(bar->u_prev);
    double2* Npb = static_cast<double2*>(bar->N_prev);
    double2* Nb = reinterpret_cast<double2*>(w + plan->ws.Nbar);
    TC_TRY2(launch_adjoint_advance(plan, ub, upb, Npb, ub, upb, Nb, Npb, w, s));
    return launch_nonlinear_adjoint(plan, static_cast<const double2*>(fwd->u), Nb, ub, w, s);
}

tc_status tc_adjoint_start(tc_plan* plan, const void* u0, const tc_state_bar* bar, void* u0_bar,
                           void* ws, void* stream) {
    TC_TRY2(adj_ready(plan, ws));
    if (!bar) return TC_ERR_ARG;
    const size_t vb = 3 * plan->S * sizeof(double2);
    TC_TRY2(check_device_ptr(plan, u0, "u0", vb));
    TC_TRY2(check_device_ptr(plan, u0_bar, "u0_bar", vb));
    TC_TRY2(check_device_ptr(plan, bar->u, "bar->u", vb));
    TC_TRY2(check_device_ptr(plan, bar->u_prev, "bar->u_prev", vb));
    TC_TRY2(check_device_ptr(plan, bar->N_prev, "bar->N_prev", vb));
    if (u0_bar == u0 || u0_bar == bar->u_prev || u0_bar == bar->N_prev) return TC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    const size_t n3 = 3 * plan->S;
    const double2* u = static_cast<const double2*>(u0);
    double2* out = static_cast<double2*>(u0_bar);
    double2* Nc = reinterpret_cast<double2*>(w + plan->ws.Ncur);
    double2* uE = reinterpret_cast<double2*>(w + plan->ws.uE);
    double2* Nb = reinterpret_cast<double2*>(w + plan->ws.Nbar);
    double2* um1 = reinterpret_cast<double2*>(w + plan->ws.abar);
    double2* m1b = um1 + n3;
    double2* uEb = m1b + n3;
    // forward recomputation of the start-up: N0 = N(u0), u_E, u^{-1}
    TC_TRY2(launch_nonlinear(plan, u, Nc, w, s));
    TC_TRY2(launch_advance(plan, u, const_cast<double2*>(u), Nc, Nc, nullptr, uE, w, false, s));
    TC_TRY2(launch_axpby(plan, um1, u, 2.5, uE, -1.5, n3, s));
    // m1_bar = ubar_prev + N'(u^{-1})^T Nbar_prev
    TC_CUDA(plan, cudaMemcpyAsync(m1b, bar->u_prev, n3 * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    TC_TRY2(launch_nonlinear_adjoint(plan, um1, static_cast<const double2*>(bar->N_prev), m1b, w, s));
    // u_E bar = -1.5 m1_bar; adjoint of the Euler step (u, u_prev, N, N_prev all = u0 / N0)
    TC_TRY2(launch_axpby(plan, uEb, m1b, -1.5, m1b, 0.0, n3, s));
    double2* a_u = out;   // adjoint of its u input
    double2* a_up = uE;   // adjoint of its u_prev input
    double2* a_N = Nb;    // adjoint of its N input
    double2* a_Np = Nc;   // adjoint of its N_prev input
    TC_TRY2(launch_adjoint_advance(plan, uEb, nullptr, nullptr, a_u, a_up, a_N, a_Np, w, s));
    // u0_bar = ubar + 2.5 m1_bar + a_u + a_up + N'(u0)^T (a_N + a_Np)
    TC_TRY2(launch_axpby(plan, out, out, 1.0, a_up, 1.0, n3, s));
    TC_TRY2(launch_axpby(plan, out, out, 1.0, m1b, 2.5, n3, s));
    TC_TRY2(launch_axpby(plan, out, out, 1.0, static_cast<const double2*>(bar->u), 1.0, n3, s));
    TC_TRY2(launch_axpby(plan, a_N, a_N, 1.0, a_Np, 1.0, n3, s));
    return launch_nonlinear_adjoint(plan, u, a_N, out, w, s);
}

tc_status tc_energy_gradient(tc_plan* plan, const void* u, void* g, void* stream) {
    if (!plan) return TC_ERR_ARG;
    if (plan->host_only) return TC_ERR_STATE;
    TC_TRY2(check_device_ptr(plan, u, "u", 3 * plan->S * sizeof(double2)));
    TC_TRY2(check_device_ptr(plan, g, "g", 3 * plan->S * sizeof(double2)));
    return launch_energy_gradient(plan, static_cast<const double2*>(u), static_cast<double2*>(g),
                                  static_cast<cudaStream_t>(stream));
}

}  // extern "C"
