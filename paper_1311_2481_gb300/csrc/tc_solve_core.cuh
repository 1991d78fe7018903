// Device helpers shared by the forward and adjoint predictor-corrector kernels: geometry,
// radial stencils on global / shared columns, and the banded substitutions with the
// pivoted LU factors of Sec. 3.2.
#pragma once

#include "tc_internal.cuh"

namespace tc {

struct Geo {
    int N, M, K, nk, nmode, K1, M1K1;
    int mlo, mhi;            // modes [mlo, mhi) handled by a launch (default: all)
    int sh;                  // fused steps 2-5: systems cut at row sh into two partitions (0: uncut)
    size_t S;
    double mp, kz, dt, c1;   // c1 = 1 / (2 dt)
};

static inline Geo geo(const tc_plan* p) {
    Geo g;
    g.N = p->N_r; g.M = p->M; g.K = p->K; g.nk = 2 * p->K + 1; g.nmode = p->nmode;
    g.K1 = p->K + 1; g.M1K1 = (p->M + 1) * (p->K + 1); g.S = p->S;
    g.mlo = 0; g.mhi = g.nmode;
    g.sh = 0;
    g.mp = (double)p->m_p; g.kz = p->k_z; g.dt = p->dt; g.c1 = 1.0 / (2.0 * p->dt);
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
static __device__ double2 lap_r(const double2* __restrict__ u, const double* __restrict__ w1,
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

// ---------------------------------------------------------------- fused steps 2-5
// One block owns T consecutive modes (all N_r rows).  Shared memory holds four complex
// columns per mode, row-major [j][t]: C0 = b_p -> p* -> div u* -> phi, C1..C3 = u*_c.
// X = (2N - N_prev)_r (pressure stage) is staged in C1 before C1 receives u*_+.

// In-place banded substitution on one real part (part = 0: re, 1: im) of column t of a
// [N][T] complex smem array, with the pivoted LU of Sec. 3.2 stored for (set, m, |k|).
// The factors of the next D rows are kept in flight in a register ring: the few long
// substitution chains of a block wait on each row's factors otherwise (they come from DRAM:
// a step streams more than L2 holds between two uses), and one row of arithmetic does not
// cover that latency.
template <int D = 1>
__device__ __forceinline__ void smem_band_solve(double2* col, int T, int t, int part, int N,
                                                const double* __restrict__ F, const uint8_t* __restrict__ P,
                                                int M1K1) {
    double* x = reinterpret_cast<double*>(col) + 2 * t + part;   // x[j] at x[2 T j]
    const int st = 2 * T;
    const size_t rs = (size_t)kBands * M1K1;                      // one row of factors
    // forward: rows j .. j+4 live in w0..w4
    double w0 = x[0], w1 = N > 1 ? x[st] : 0.0, w2 = N > 2 ? x[2 * st] : 0.0,
           w3 = N > 3 ? x[3 * st] : 0.0, w4 = N > 4 ? x[4 * st] : 0.0;
    double lr[D][4];
    int pr[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        pr[d] = 0;
        lr[d][0] = lr[d][1] = lr[d][2] = lr[d][3] = 0.0;
        if (d < N) {
            const double* Fr = F + (size_t)d * rs;
            pr[d] = P[(size_t)d * M1K1];
#pragma unroll
            for (int q = 0; q < 4; ++q) lr[d][q] = __ldg(&Fr[(size_t)q * M1K1]);
        }
    }
    for (int j0 = 0; j0 < N; j0 += D) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int j = j0 + d;
            if (j < N) {
                const int pj = pr[d];
                const double l1 = lr[d][0], l2 = lr[d][1], l3 = lr[d][2], l4 = lr[d][3];
                if (j + D < N) {   // refill this slot with row j + D
                    const double* Fr = F + (size_t)(j + D) * rs;
                    pr[d] = P[(size_t)(j + D) * M1K1];
#pragma unroll
                    for (int q = 0; q < 4; ++q) lr[d][q] = __ldg(&Fr[(size_t)q * M1K1]);
                }
                if (pj == 1) { double q = w0; w0 = w1; w1 = q; }
                else if (pj == 2) { double q = w0; w0 = w2; w2 = q; }
                else if (pj == 3) { double q = w0; w0 = w3; w3 = q; }
                else if (pj == 4) { double q = w0; w0 = w4; w4 = q; }
                x[(size_t)j * st] = w0;
                w1 = fma(-l1, w0, w1);
                w2 = fma(-l2, w0, w2);
                w3 = fma(-l3, w0, w3);
                w4 = fma(-l4, w0, w4);
                w0 = w1; w1 = w2; w2 = w3; w3 = w4;
                w4 = (j + 5 < N) ? x[(size_t)(j + 5) * st] : 0.0;
            }
        }
    }
    // backward: x_{j+1..j+8} in v1..v8.  Row-oriented.  A column-oriented variant (each x_j
    // taken out of the rows above at once: two dependent operations per row instead of nine,
    // same results bit for bit) measured slower on GB300 (k_pc 0.547 against 0.286 ms at
    // N_r = 64): each FP64 instruction costs its warp the same issue time whatever the chain,
    // so the substitution is bound by the count of FP64 instructions, not by their latency
    double v1 = 0.0, v2 = 0.0, v3 = 0.0, v4 = 0.0, v5 = 0.0, v6 = 0.0, v7 = 0.0, v8 = 0.0;
    double ur[D][9];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int j = N - 1 - d;
#pragma unroll
        for (int q = 0; q < 9; ++q) ur[d][q] = j >= 0 ? __ldg(&F[(size_t)j * rs + (size_t)(4 + q) * M1K1]) : 0.0;
    }
    for (int j0 = N - 1; j0 >= 0; j0 -= D) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int j = j0 - d;
            if (j >= 0) {
                double uc[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) uc[q] = ur[d][q];
                if (j - D >= 0) {   // refill this slot with row j - D
#pragma unroll
                    for (int q = 0; q < 9; ++q) ur[d][q] = __ldg(&F[(size_t)(j - D) * rs + (size_t)(4 + q) * M1K1]);
                }
                double s = x[(size_t)j * st];
                s = fma(-uc[8], v8, s);
                s = fma(-uc[7], v7, s);
                s = fma(-uc[6], v6, s);
                s = fma(-uc[5], v5, s);
                s = fma(-uc[4], v4, s);
                s = fma(-uc[3], v3, s);
                s = fma(-uc[2], v2, s);
                s = fma(-uc[1], v1, s);
                const double xj = s * uc[0];
                x[(size_t)j * st] = xj;
                v8 = v7; v7 = v6; v6 = v5; v5 = v4; v4 = v3; v3 = v2; v2 = v1; v1 = xj;
            }
        }
    }
}

// D1 of column t of smem array C ([N][T]) at row j
__device__ __forceinline__ double2 sdrow(const double2* C, const double* __restrict__ w1,
                                         const int* __restrict__ col0, int j, int T, int t) {
    const int c0 = col0[j];
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int q = 0; q < kStencil; ++q) {
        const double wq = __ldg(&w1[j * kStencil + q]);
        const double2 v = C[(c0 + q) * T + t];
        s.x = fma(wq, v.x, s.x);
        s.y = fma(wq, v.y, s.y);
    }
    return s;
}

}  // namespace tc
