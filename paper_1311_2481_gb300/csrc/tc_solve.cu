// Linear part of the AB2BD2 step (Sec. 3.2 steps 2-5): right-hand sides, the five banded
// solves per Fourier mode with precomputed LU factors (forward / backward substitution,
// O(N_r) per system), and the update.  Two paths:
//
//   k_pc     (N_r up to 192) one block per T consecutive modes, all five solves and their
//            right-hand sides in shared memory.  Each system is solved in two partitions
//            (rows [0, N_r/2) and [N_r/2, N_r), each with its own pivoted LU factors, on
//            separate threads), coupled through an 8 x 8 reduced system and a fix-up; one
//            real part per thread, consecutive modes on consecutive threads.
//   split    (larger N_r) one kernel per stage; the solves walk one column per thread in
//            global memory with the full-system factors.
//
// Threads of a warp own consecutive k, so every access to a field [r][m][k] or to the
// factors [j][band][m][|k|] is coalesced.
#include <algorithm>

#include "tc_internal.cuh"
#include "tc_solve_core.cuh"
#include "tc_split.cuh"

namespace tc {

struct PCArgs {
    const double2* u;   // u^i
    const double2* up;  // u^{i-1}
    const double2* Nc;  // N^i
    const double2* Np;  // N^{i-1}
    double2* u_out;     // commit: u (in place); otherwise the result u^{i+1} only
    double2* up_out;    // commit: u_prev <- u^i
    double2* Np_out;    // commit: N_prev <- N^i
    double2* p;         // commit: p <- p^{i+1}
    const double* rn;
    const double* ir;   // 1 / r_j
    const double* w1;
    const double* w2;
    const int* col0;
    const double* fac;
    const uint8_t* piv;
    const double* fac2;   // two-partition form (g.sh > 0): factors of the diagonal blocks,
    const uint8_t* piv2;  // spikes [set][j][q][m][ka] and inverse reduced matrices
    const double* spk;    // [set][8 i + l][m][ka]
    const double* rinv;
    int* nonfinite;       // set to 1 when a NaN/Inf is written into the state
    double Re_i, Re_o;
    int commit;
};

// Thread lt of the 4 nT threads of one system solves one half of it for one (mode, part):
// threads [0, 2nT) rows [0, sh), threads [2nT, 4nT) rows [sh, N), each with the pivoted LU
// factors of its diagonal block; the column then holds g = (A1^{-1} b1, A2^{-1} b2).
__device__ __forceinline__ void half_solve(const PCArgs& a, const Geo& g, double2* X, int set, int T, int nT,
                                           int mode0, int lt) {
    const int half = lt >= 2 * nT ? 1 : 0;
    const int r = lt - half * 2 * nT;
    const int t = r >> 1, part = r & 1;
    const int mode = mode0 + t, m = mode / g.nk, k = mode - m * g.nk - g.K;
    const size_t mk = (size_t)m * g.K1 + (k < 0 ? -k : k);
    const size_t per_set = (size_t)g.N * kBands * g.M1K1;
    const int r0 = half ? g.sh : 0, n = half ? g.N - g.sh : g.sh;
    smem_band_solve<kPCDepth>(X + (size_t)r0 * T, T, t, part, n,
                              a.fac2 + (size_t)set * per_set + (size_t)r0 * kBands * g.M1K1 + mk,
                              a.piv2 + ((size_t)set * g.N + r0) * g.M1K1 + mk, g.M1K1);
}

// Couple the halves of nsys systems (columns X0 + s N T, factor sets set0 + s), block-wide:
// the interface unknowns x[sh-4 .. sh+3] = R^{-1} g[sh-4 .. sh+3] per (mode, part) into Xr,
// then x = g - V x[sh .. sh+3] on rows < sh and x = g - W x[sh-4 .. sh-1] on rows >= sh.
// Starts after a barrier that follows the half solves; ends with one.
__device__ __forceinline__ void spike_combine(const PCArgs& a, const Geo& g, double2* X0, int nsys, int set0,
                                              int T, int nT, int mode0, double* Xr) {
    const int N = g.N, h = g.sh, items = N * T, st = 2 * T;
    for (int task = threadIdx.x; task < nsys * nT * 16; task += blockDim.x) {
        const int s = task / (nT * 16), rem = task - s * nT * 16;
        const int t = rem >> 4, part = (rem >> 3) & 1, i = rem & 7;
        const int mode = mode0 + t, m = mode / g.nk, k = mode - m * g.nk - g.K;
        const size_t mk = (size_t)m * g.K1 + (k < 0 ? -k : k);
        const double* x = reinterpret_cast<const double*>(X0 + (size_t)s * items) + 2 * t + part;
        const double* R = a.rinv + ((size_t)(set0 + s) * 64 + 8 * i) * g.M1K1 + mk;
        double acc = 0.0;
#pragma unroll
        for (int l = 0; l < 8; ++l) acc = fma(__ldg(&R[(size_t)l * g.M1K1]), x[(size_t)(h - 4 + l) * st], acc);
        Xr[(s * T + t) * 16 + part * 8 + i] = acc;
    }
    __syncthreads();
    // fix-up: T divides the block size, so a thread's elements all belong to mode t = tid % T;
    // rows step by blockDim / T, four in flight per iteration
    const int t = threadIdx.x % T;
    if (t < nT) {
        const int mode = mode0 + t, m = mode / g.nk, k = mode - m * g.nk - g.K;
        const size_t mk = (size_t)m * g.K1 + (k < 0 ? -k : k);
        const int jstep = blockDim.x / T;
        for (int s = 0; s < nsys; ++s) {
            const double* Vs = a.spk + (size_t)(set0 + s) * N * 4 * g.M1K1 + mk;
            const double* xs = Xr + (s * T + t) * 16;
            double2* Xs = X0 + (size_t)s * items + t;
#pragma unroll 4
            for (int j = threadIdx.x / T; j < N; j += jstep) {
                const double* V = Vs + (size_t)j * 4 * g.M1K1;
                const double* xr = xs + (j < h ? 4 : 0);
                double2 v = Xs[(size_t)j * T];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double w = __ldg(&V[(size_t)q * g.M1K1]);
                    v.x = fma(-w, xr[q], v.x);
                    v.y = fma(-w, xr[8 + q], v.y);
                }
                Xs[(size_t)j * T] = v;
            }
        }
    }
    __syncthreads();
}

// Mixed form: the radial stencil sum_q w_q f_q over the 9 values v[q] of one complex column,
// stored as exact FP32 pairs (hi re, hi im, lo re, lo im), with split weights w: a compensated
// dot product (Ogita-Rump-Oishi), assembled in FP64.  The pairs carry 47 bits of each value,
// so the error is about 2^-46 of sum |w_q f_q|.
__device__ __forceinline__ double2 xs_stencil(const float4* v, int vstride, const float2* w) {
    float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
#pragma unroll
    for (int q = 0; q < kStencil; ++q) {
        const float4 f = v[q * vstride];
        xs::dot_acc(sx, cx, w[q].x, w[q].y, f.x, f.z);
        xs::dot_acc(sy, cy, w[q].x, w[q].y, f.y, f.w);
    }
    return make_double2(xs::f2d_bits(sx) + xs::f2d_bits(cx), xs::f2d_bits(sy) + xs::f2d_bits(cy));
}

// Steps 2-5 of Sec. 3.2 for the T modes of this block: pressure prediction (Eq. pressure
// with the Neumann rows of Eq. ppBC), velocity prediction (Eq. vel), correction potential
// (Eq. correction) and update (Eq. update).
// MX (mixed form): the four radial stencils -- of X, p*, u*_+ + u*_- and phi -- in
// double-FP32: the column is split once into exact FP32 pairs in shared memory (XS, with the
// split weights SW), the stencil is a compensated dot product of the pairs (xs_stencil), the
// result is assembled in FP64; the solves and everything else stay FP64.
// The (0, 0) mode's stencils stay FP64 too (the mean flow, see the per-stage kernels): the
// block that holds it computes that column's stencils in one pass, a row per thread, before
// each phase (D00), so its warps do not diverge into FP64 stencils in the phase itself.
template <int NTH, bool MX>
__global__ void __launch_bounds__(NTH, 512 / NTH) k_pc(PCArgs a, Geo g, int T) {
    extern __shared__ double2 sm[];
    const int N = g.N;
    const int items = N * T;
    double2* C0 = sm;
    double2* C1 = sm + items;
    double2* C2 = C1 + items;
    double2* C3 = C2 + items;
    float4* XS = reinterpret_cast<float4*>(C3 + items) + 3 * T * 16 / 2;   // after the spike scratch
    float2* SW = reinterpret_cast<float2*>(XS + items);
    double2* D00 = reinterpret_cast<double2*>(SW + ((N * kStencil + 1) & ~1));   // 16-byte aligned
    const int mode0 = g.mlo + blockIdx.x * T;
    const int nT = min(T, g.mhi - mode0);
    // column of the (0, 0) mode in this block, or -1
    const int t00 = (g.K >= mode0 && g.K < mode0 + nT) ? g.K - mode0 : -1;
    if (MX) {
        for (int i = threadIdx.x; i < N * kStencil; i += blockDim.x) SW[i] = xs::split_hl(a.w1[i]);
    }
    // XS <- split of the column(s) (F + F2), D00 <- the FP64 stencil of column t00, a barrier
    auto split_cols = [&](const double2* F, const double2* F2) {
        if (t00 >= 0) {
            for (int j = threadIdx.x; j < N; j += blockDim.x) {
                double2 d = sdrow(F, a.w1, a.col0, j, T, t00);
                if (F2) {
                    const double2 d2 = sdrow(F2, a.w1, a.col0, j, T, t00);
                    d.x += d2.x;
                    d.y += d2.y;
                }
                D00[j] = d;
            }
        }
        for (int i = threadIdx.x; i < items; i += blockDim.x) {
            double2 x = F[i];
            if (F2) {
                x.x += F2[i].x;
                x.y += F2[i].y;
            }
            const float2 p = xs::split_hl(x.x), q = xs::split_hl(x.y);
            XS[i] = make_float4(p.x, q.x, p.y, q.y);
        }
        __syncthreads();
    };
    // D1 of the split column at row j, mode t; the (0, 0) column's from D00
    auto xsrow = [&](int j, int t) {
        if (t == t00) return D00[j];
        return xs_stencil(XS + a.col0[j] * T + t, T, SW + j * kStencil);
    };
    const size_t per_set = (size_t)N * kBands * g.M1K1;
    const double c1 = g.c1;   // 1 / (2 dt)
    // T divides the block size, so every element a thread visits in the element loops below
    // belongs to the same mode t = threadIdx.x % T: its row index steps by blockDim / T, and
    // m, k and the FP64 factors m m_p, k k_z are computed once (an int -> double conversion
    // takes the FP64 pipe like an arithmetic instruction)
    const int tq = threadIdx.x % T;
    const int jstep = blockDim.x / T;
    const int modeq = mode0 + tq;
    const int mq = modeq / g.nk;
    const int kq = modeq - mq * g.nk - g.K;
    const double mmq = g.mp * mq, kkq = g.kz * kq;

    // A1: X = (2N - N_prev)_r into C1
    for (int j = threadIdx.x / T; j < N; j += jstep) {
        const int idx = j * T + tq, t = tq;
        double2 x = make_double2(0.0, 0.0);
        if (t < nT) {
            const size_t e = (size_t)j * g.nmode + mode0 + t;
            const double2 n1 = a.Nc[e], n0 = a.Np[e], m1 = a.Nc[g.S + e], m0 = a.Np[g.S + e];
            x.x = 0.5 * ((2.0 * n1.x - n0.x) + (2.0 * m1.x - m0.x));
            x.y = 0.5 * ((2.0 * n1.y - n0.y) + (2.0 * m1.y - m0.y));
        }
        C1[idx] = x;
        if (MX) {
            const float2 p = xs::split_hl(x.x), q = xs::split_hl(x.y);
            XS[idx] = make_float4(p.x, q.x, p.y, q.y);
        }
    }
    __syncthreads();
    if (MX && t00 >= 0) {   // the (0, 0) column's stencil of X in FP64
        for (int j = threadIdx.x; j < N; j += blockDim.x) D00[j] = sdrow(C1, a.w1, a.col0, j, T, t00);
        __syncthreads();
    }
    // A2: pressure right-hand side into C0
    for (int j = threadIdx.x / T; j < N; j += jstep) {
        const int idx = j * T + tq, t = tq;
        double2 out = make_double2(0.0, 0.0);
        if (t < nT) {
            const int mode = modeq, m = mq, k = kq;
            const double mm = mmq, kk = kkq;
            const double r = a.rn[j], ir = a.ir[j];
            const size_t e = (size_t)j * g.nmode + mode;
            if (j == 0 || j == N - 1) {
                if (!(j == N - 1 && m == 0 && k == 0)) {
                    const double2 l0 = lap_r(a.u, a.w1, a.w2, a.col0, r, j, mode, mm, kk, g);
                    const double2 l1 = lap_r(a.up, a.w1, a.w2, a.col0, r, j, mode, mm, kk, g);
                    const double2 X = C1[idx];
                    out.x = -X.x + 2.0 * l0.x - l1.x;
                    out.y = -X.y + 2.0 * l0.y - l1.y;
                }
            } else {
                const double2 d = MX ? xsrow(j, t) : sdrow(C1, a.w1, a.col0, j, T, t);
                const double2 X = C1[idx];
                const double2 n1 = a.Nc[e], n0 = a.Np[e], m1 = a.Nc[g.S + e], m0 = a.Np[g.S + e];
                const double2 z1 = a.Nc[2 * g.S + e], z0 = a.Np[2 * g.S + e];
                const double dpx = (2.0 * n1.x - n0.x) - (2.0 * m1.x - m0.x);
                const double dpy = (2.0 * n1.y - n0.y) - (2.0 * m1.y - m0.y);
                const double nzx = 2.0 * z1.x - z0.x, nzy = 2.0 * z1.y - z0.y;
                out.x = -(d.x + X.x * ir + 0.5 * mm * ir * dpx - kk * nzy);
                out.y = -(d.y + X.y * ir + 0.5 * mm * ir * dpy + kk * nzx);
            }
        }
        C0[idx] = out;
    }
    __syncthreads();
    // B: p* = P^{-1} b_p (real and imaginary parts by separate threads).  Meanwhile the
    // warps without a substitution precompute the part of the velocity right-hand sides that
    // does not depend on p*: (4u - u_prev)/(2dt) - (2N - N_prev), and the Dirichlet rows.
    // With two partitions (g.sh > 0) 4 nT threads solve, two per (mode, part).
    const bool sp = g.sh > 0;
    double* Xr = reinterpret_cast<double*>(C3 + items);
    const int nsolve = (sp ? 4 : 2) * nT;
    const int helper0 = ((nsolve + 31) / 32) * 32;
    if (threadIdx.x < nsolve) {
        if (sp) {
            half_solve(a, g, C0, kSetP, T, nT, mode0, threadIdx.x);
        } else {
            const int t = threadIdx.x >> 1, part = threadIdx.x & 1;
            const int mode = mode0 + t, m = mode / g.nk, k = mode - m * g.nk - g.K;
            const size_t mk = (size_t)m * g.K1 + (k < 0 ? -k : k);
            smem_band_solve<kPCDepth>(C0, T, t, part, N, a.fac + (size_t)kSetP * per_set + mk,
                            a.piv + (size_t)kSetP * N * g.M1K1 + mk, g.M1K1);
        }
    }
    // (with no spare warp the whole block does this after the substitution)
    const bool spare0 = helper0 < (int)blockDim.x;
    if (!spare0) __syncthreads();
    if (spare0 ? threadIdx.x >= helper0 : true) {
        const int first = spare0 ? helper0 : 0;   // a multiple of 32: (threadIdx.x - first) % T == tq
        for (int j = (threadIdx.x - first) / T; j < N; j += ((int)blockDim.x - first) / T) {
            const int idx = j * T + tq, t = tq;
            double2 o[3] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
            if (t < nT) {
                const int mode = modeq, m = mq, k = kq;
                if (j == 0 || j == N - 1) {
                    if (m == 0 && k == 0) {
                        const double Re = j == 0 ? a.Re_i : a.Re_o;
                        o[0].y = Re;
                        o[1].y = -Re;
                    }
                } else {
                    const size_t e = (size_t)j * g.nmode + mode;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const size_t ec = (size_t)c * g.S + e;
                        const double2 uu = a.u[ec], q = a.up[ec], n1 = a.Nc[ec], n0 = a.Np[ec];
                        o[c].x = (4.0 * uu.x - q.x) * c1 - (2.0 * n1.x - n0.x);
                        o[c].y = (4.0 * uu.y - q.y) * c1 - (2.0 * n1.y - n0.y);
                    }
                }
            }
            C1[idx] = o[0];
            C2[idx] = o[1];
            C3[idx] = o[2];
        }
    }
    __syncthreads();
    if (sp) spike_combine(a, g, C0, 1, kSetP, T, nT, mode0, Xr);
    if (MX) split_cols(C0, nullptr);
    // C: velocity right-hand sides: subtract grad_h p* on interior rows; p <- p* (commit)
    for (int j = threadIdx.x / T; j < N && tq < nT; j += jstep) {
        const int idx = j * T + tq, t = tq;
        const int mode = modeq;
        const double2 pv = C0[idx];
        if (a.commit) a.p[(size_t)j * g.nmode + mode] = pv;
        if (j == 0 || j == N - 1) continue;
        const double2 d = MX ? xsrow(j, t) : sdrow(C0, a.w1, a.col0, j, T, t);
        const double tt = mmq * a.ir[j];
        const double kk = kkq;
        double2 v;
        v = C1[idx]; v.x -= d.x - tt * pv.x; v.y -= d.y - tt * pv.y; C1[idx] = v;
        v = C2[idx]; v.x -= d.x + tt * pv.x; v.y -= d.y + tt * pv.y; C2[idx] = v;
        v = C3[idx]; v.x += kk * pv.y; v.y -= kk * pv.x; C3[idx] = v;
    }
    __syncthreads();
    // D: the three Helmholtz solves.  Meanwhile the other warps rotate the history (nothing
    // reads u_prev or N_prev after C): u_prev <- u^i, N_prev <- N^i (commit).
    const int nsolve1 = (sp ? 12 : 6) * nT;
    const int helper1 = ((nsolve1 + 31) / 32) * 32;
    if (threadIdx.x < nsolve1) {
        if (sp) {
            const int c = threadIdx.x / (4 * nT);
            half_solve(a, g, C1 + (size_t)c * items, kSetHp + c, T, nT, mode0, threadIdx.x - c * 4 * nT);
        } else {
            const int c = threadIdx.x / (2 * nT), rem = threadIdx.x - c * 2 * nT;
            const int t = rem >> 1, part = rem & 1;
            const int mode = mode0 + t, m = mode / g.nk, k = mode - m * g.nk - g.K;
            const size_t mk = (size_t)m * g.K1 + (k < 0 ? -k : k);
            const int set = kSetHp + c;
            smem_band_solve<kPCDepth>(C1 + (size_t)c * items, T, t, part, N, a.fac + (size_t)set * per_set + mk,
                            a.piv + (size_t)set * N * g.M1K1 + mk, g.M1K1);
        }
    } else if (a.commit && threadIdx.x >= helper1) {
        for (int idx = threadIdx.x - helper1; idx < 3 * items; idx += blockDim.x - helper1) {
            const int c = idx / items, rem = idx - c * items;
            const int j = rem / T, t = rem - (rem / T) * T;
            if (t >= nT) continue;
            const size_t ec = (size_t)c * g.S + (size_t)j * g.nmode + mode0 + t;
            a.up_out[ec] = a.u[ec];
            a.Np_out[ec] = a.Nc[ec];
        }
    }
    __syncthreads();
    if (sp) spike_combine(a, g, C1, 3, kSetHp, T, nT, mode0, Xr);
    if (a.commit && helper1 >= (int)blockDim.x) {   // no spare warp: rotate here
        for (int idx = threadIdx.x; idx < 3 * items; idx += blockDim.x) {
            const int c = idx / items, rem = idx - c * items;
            const int j = rem / T, t = rem - (rem / T) * T;
            if (t >= nT) continue;
            const size_t ec = (size_t)c * g.S + (size_t)j * g.nmode + mode0 + t;
            a.up_out[ec] = a.u[ec];
            a.Np_out[ec] = a.Nc[ec];
        }
    }
    // E: div_h u* into C0 (homogeneous Neumann / Dirichlet rows)
    if (MX) split_cols(C1, C2);   // the stencil of u*_+ + u*_-
    for (int j = threadIdx.x / T; j < N; j += jstep) {
        const int idx = j * T + tq, t = tq;
        double2 out = make_double2(0.0, 0.0);
        if (t < nT && j > 0 && j < N - 1) {
            const double mm = mmq, kk = kkq, ir = a.ir[j];
            double2 ds;
            if (MX) {
                ds = xsrow(j, t);
            } else {
                const double2 dp = sdrow(C1, a.w1, a.col0, j, T, t), dm = sdrow(C2, a.w1, a.col0, j, T, t);
                ds = make_double2(dp.x + dm.x, dp.y + dm.y);
            }
            const double2 vp = C1[idx], vm = C2[idx], vz = C3[idx];
            out.x = 0.5 * ds.x + 0.5 * (vp.x + vm.x) * ir + 0.5 * mm * ir * (vp.x - vm.x) - kk * vz.y;
            out.y = 0.5 * ds.y + 0.5 * (vp.y + vm.y) * ir + 0.5 * mm * ir * (vp.y - vm.y) + kk * vz.x;
        }
        C0[idx] = out;
    }
    __syncthreads();
    // F: phi = P^{-1} div_h u*
    if (threadIdx.x < nsolve) {
        if (sp) {
            half_solve(a, g, C0, kSetP, T, nT, mode0, threadIdx.x);
        } else {
            const int t = threadIdx.x >> 1, part = threadIdx.x & 1;
            const int mode = mode0 + t, m = mode / g.nk, k = mode - m * g.nk - g.K;
            const size_t mk = (size_t)m * g.K1 + (k < 0 ? -k : k);
            smem_band_solve<kPCDepth>(C0, T, t, part, N, a.fac + (size_t)kSetP * per_set + mk,
                            a.piv + (size_t)kSetP * N * g.M1K1 + mk, g.M1K1);
        }
    }
    __syncthreads();
    if (sp) spike_combine(a, g, C0, 1, kSetP, T, nT, mode0, Xr);
    if (MX) split_cols(C0, nullptr);
    // G: u^{i+1} = u* - grad_h phi, p^{i+1} = p* + 3 phi / (2 dt), history rotation
    bool bad = false;
    for (int j = threadIdx.x / T; j < N && tq < nT; j += jstep) {
        const int idx = j * T + tq, t = tq;
        const size_t e = (size_t)j * g.nmode + modeq;
        const double2 f = C0[idx];
        const double2 d = MX ? xsrow(j, t) : sdrow(C0, a.w1, a.col0, j, T, t);
        const double tt = mmq * a.ir[j];
        const double kk = kkq;
        const double2 gph[3] = {make_double2(d.x - tt * f.x, d.y - tt * f.y),
                                make_double2(d.x + tt * f.x, d.y + tt * f.y),
                                make_double2(-kk * f.y, kk * f.x)};
        const double2 us[3] = {C1[idx], C2[idx], C3[idx]};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t ec = (size_t)c * g.S + e;
            const double2 un = make_double2(us[c].x - gph[c].x, us[c].y - gph[c].y);
            a.u_out[ec] = un;
            bad |= nonfinite2(un);
        }
        if (a.commit) {
            const double q = 3.0 * c1;   // 3 / (2 dt)
            const double2 ps = a.p[e];
            a.p[e] = make_double2(ps.x + q * f.x, ps.y + q * f.y);
        }
    }
    if (bad && a.nonfinite) *a.nonfinite = 1;
}

// ---------------------------------------------------------------- split path (large N_r)
// With few modes per block in shared memory the fused kernel leaves most lanes idle during
// the substitutions; at large N_r there are enough modes to run each stage as its own
// kernel instead: elementwise right-hand sides and update, and one thread per (system,
// mode, real/imaginary part) walking its column in global memory.

// X = (2N - N_prev)_r = ((2N - N_prev)_+ + (2N - N_prev)_-) / 2, once per element (the
// pressure right-hand side applies the radial stencil to it).
__global__ void k_nn_r(const double2* __restrict__ Nc, const double2* __restrict__ Np, double2* __restrict__ X, Geo g) {
    const int mode = g.mlo + blockIdx.y * blockDim.x + threadIdx.x;   // x = radial row
    if (mode >= g.mhi) return;
    const size_t e = (size_t)blockIdx.x * g.nmode + mode;
    const double2 n1 = Nc[e], n0 = Np[e], m1 = Nc[g.S + e], m0 = Np[g.S + e];
    X[e] = make_double2(0.5 * ((2.0 * n1.x - n0.x) + (2.0 * m1.x - m0.x)),
                        0.5 * ((2.0 * n1.y - n0.y) + (2.0 * m1.y - m0.y)));
}

// Step 2 right-hand side on the interior rows: div_h(-(2N - N_prev)) (the wall rows:
// k_rhs_pressure_walls).
__global__ void k_rhs_pressure(const double2* __restrict__ u, const double2* __restrict__ up,
                               const double2* __restrict__ Nc, const double2* __restrict__ Np,
                               const double2* __restrict__ X, double2* __restrict__ b,
                               const double* __restrict__ rn, const double* __restrict__ irn,
                               const double* __restrict__ w1, const double* __restrict__ w2,
                               const int* __restrict__ col0, Geo g) {
    // grid: x = radial row (fastest, so neighbouring rows of a mode range run together and
    // the stencil's rows stay in cache), y over modes
    const int mode = g.mlo + blockIdx.y * blockDim.x + threadIdx.x;
    if (mode >= g.mhi) return;
    const int j = blockIdx.x + 1;   // interior rows (k_rhs_pressure_walls takes the walls)
    const size_t e = (size_t)j * g.nmode + mode;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const double mm = g.mp * m, kk = g.kz * k;
    const double ir = irn[j];
    double2 out = make_double2(0.0, 0.0);
    {
        const double2 d = drow(X, w1, col0, j, g.nmode, mode);
        const double2 x = X[e];
        const double2 n1 = Nc[e], n0 = Np[e], m1 = Nc[g.S + e], m0 = Np[g.S + e];
        const double2 z1 = Nc[2 * g.S + e], z0 = Np[2 * g.S + e];
        const double dpx = (2.0 * n1.x - n0.x) - (2.0 * m1.x - m0.x);
        const double dpy = (2.0 * n1.y - n0.y) - (2.0 * m1.y - m0.y);
        const double nzx = 2.0 * z1.x - z0.x, nzy = 2.0 * z1.y - z0.y;
        out.x = -(d.x + x.x * ir + 0.5 * mm * ir * dpx - kk * nzy);
        out.y = -(d.y + x.y * ir + 0.5 * mm * ir * dpy + kk * nzx);
    }
    b[e] = out;
}

// Step 2 right-hand side on the two wall rows: the consistent Neumann value of Eq. ppBC
// (the wall Laplacian of u and u_prev), or the Dirichlet value 0 for (0,0) at r_o; kept apart
// from the interior rows, whose kernel then needs far fewer registers
__global__ void k_rhs_pressure_walls(const double2* __restrict__ u, const double2* __restrict__ up,
                                     const double2* __restrict__ X, double2* __restrict__ b,
                                     const double* __restrict__ rn, const double* __restrict__ w1,
                                     const double* __restrict__ w2, const int* __restrict__ col0, Geo g) {
    const int mode = g.mlo + blockIdx.x * blockDim.x + threadIdx.x;   // y = wall (0: r_i, 1: r_o)
    if (mode >= g.mhi) return;
    const int j = blockIdx.y == 0 ? 0 : g.N - 1;
    const size_t e = (size_t)j * g.nmode + mode;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    double2 out = make_double2(0.0, 0.0);
    if (!(j == g.N - 1 && m == 0 && k == 0)) {
        const double mm = g.mp * m, kk = g.kz * k;
        const double r = rn[j];
        const double2 x = X[e];
        const double2 l0 = lap_r(u, w1, w2, col0, r, j, mode, mm, kk, g);
        const double2 l1 = lap_r(up, w1, w2, col0, r, j, mode, mm, kk, g);
        out.x = -x.x + 2.0 * l0.x - l1.x;
        out.y = -x.y + 2.0 * l0.y - l1.y;
    }
    b[e] = out;
}

// Step 3 right-hand sides, all three components per (row, mode) so that the radial
// stencil of p* is applied once: (4u - u_prev)/(2dt) - (2N - N_prev) - grad_h p*;
// Dirichlet rows.  commit: p <- p* (p^{i+1} is completed in the update).
__global__ void k_rhs_velocity(const double2* __restrict__ u, const double2* __restrict__ up,
                               const double2* __restrict__ Nc, const double2* __restrict__ Np,
                               const double2* __restrict__ ps, double2* __restrict__ rhs,
                               double2* __restrict__ p_out, const double* __restrict__ irn,
                               const double* __restrict__ w1, const int* __restrict__ col0,
                               double Re_i, double Re_o, Geo g) {
    const int mode = g.mlo + blockIdx.y * blockDim.x + threadIdx.x;   // x = radial row
    if (mode >= g.mhi) return;
    const int j = blockIdx.x;
    const size_t e = (size_t)j * g.nmode + mode;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const double2 pv = ps[e];
    if (p_out) p_out[e] = pv;
    if (j == 0 || j == g.N - 1) {
        const double Re = (m == 0 && k == 0) ? (j == 0 ? Re_i : Re_o) : 0.0;
        rhs[e] = make_double2(0.0, Re);
        rhs[g.S + e] = make_double2(0.0, -Re);
        rhs[2 * g.S + e] = make_double2(0.0, 0.0);
        return;
    }
    const double2 d = drow(ps, w1, col0, j, g.nmode, mode);
    const double tt = g.mp * m * irn[j], kk = g.kz * k;
    const double2 gp[3] = {make_double2(d.x - tt * pv.x, d.y - tt * pv.y),
                           make_double2(d.x + tt * pv.x, d.y + tt * pv.y),
                           make_double2(-kk * pv.y, kk * pv.x)};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t ec = (size_t)c * g.S + e;
        const double2 a = u[ec], q = up[ec], n1 = Nc[ec], n0 = Np[ec];
        rhs[ec] = make_double2((4.0 * a.x - q.x) * g.c1 - (2.0 * n1.x - n0.x) - gp[c].x,
                               (4.0 * a.y - q.y) * g.c1 - (2.0 * n1.y - n0.y) - gp[c].y);
    }
}

// Step 4 right-hand side: div_h u* on interior rows, homogeneous Neumann / Dirichlet rows.
__global__ void k_rhs_div(const double2* __restrict__ us, double2* __restrict__ b,
                          const double* __restrict__ irn, const double* __restrict__ w1,
                          const int* __restrict__ col0, Geo g) {
    const int mode = g.mlo + blockIdx.y * blockDim.x + threadIdx.x;   // x = radial row
    if (mode >= g.mhi) return;
    const int j = blockIdx.x;
    const size_t e = (size_t)j * g.nmode + mode;
    if (j == 0 || j == g.N - 1) { b[e] = make_double2(0.0, 0.0); return; }
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const double mm = g.mp * m, kk = g.kz * k, ir = irn[j];
    const int c0 = col0[j];
    double2 d = make_double2(0.0, 0.0);
#pragma unroll
    for (int t = 0; t < kStencil; ++t) {
        const double wt = __ldg(&w1[j * kStencil + t]);
        const size_t o = (size_t)(c0 + t) * g.nmode + mode;
        const double2 a = us[o], q = us[g.S + o];
        d.x += wt * (a.x + q.x);
        d.y += wt * (a.y + q.y);
    }
    const double2 vp = us[e], vm = us[g.S + e], vz = us[2 * g.S + e];
    b[e] = make_double2(0.5 * d.x + 0.5 * (vp.x + vm.x) * ir + 0.5 * mm * ir * (vp.x - vm.x) - kk * vz.y,
                        0.5 * d.y + 0.5 * (vp.y + vm.y) * ir + 0.5 * mm * ir * (vp.y - vm.y) + kk * vz.x);
}

// Step 5, all components per (row, mode): u^{i+1} = u* - grad_h phi; p^{i+1} = p* + 3 phi/(2dt).
// commit: rotate the history in place (u_prev <- u^i, u <- u^{i+1}, N_prev <- N^i, p += 3 phi/(2dt));
// otherwise write u^{i+1} to u_out only.
__global__ void k_update(double2* u, double2* up, const double2* Nc, double2* Np, double2* p,
                         const double2* __restrict__ us, const double2* __restrict__ phi,
                         double2* __restrict__ u_out, const double* __restrict__ irn,
                         const double* __restrict__ w1, const int* __restrict__ col0, int commit,
                         int* __restrict__ nonfinite, Geo g) {
    const int mode = g.mlo + blockIdx.y * blockDim.x + threadIdx.x;   // x = radial row
    if (mode >= g.mhi) return;
    const int j = blockIdx.x;
    const size_t e = (size_t)j * g.nmode + mode;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const double2 f = phi[e];
    const double2 d = drow(phi, w1, col0, j, g.nmode, mode);
    const double tt = g.mp * m * irn[j], kk = g.kz * k;
    const double2 gph[3] = {make_double2(d.x - tt * f.x, d.y - tt * f.y),
                            make_double2(d.x + tt * f.x, d.y + tt * f.y),
                            make_double2(-kk * f.y, kk * f.x)};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t ec = (size_t)c * g.S + e;
        const double2 s = us[ec];
        const double2 un = make_double2(s.x - gph[c].x, s.y - gph[c].y);
        if (nonfinite2(un) && nonfinite) *nonfinite = 1;
        if (commit) {
            up[ec] = u[ec];
            u[ec] = un;
            Np[ec] = Nc[ec];
        } else {
            u_out[ec] = un;
        }
    }
    if (commit) {
        const double q = 3.0 * g.c1;
        const double2 a = p[e];
        p[e] = make_double2(a.x + q * f.x, a.y + q * f.y);
    }
}

// ---------------------------------------------------------------- split path, mixed form
// The same four per-stage kernels for TC_MIXED plans, with each radial stencil (of X, p*,
// u*_+ + u*_- and phi) in double-FP32 instead of FP64: the FP64 pipe, which bounds these
// kernels, then carries only the rest.  The (0, 0) mode keeps the FP64 stencil: it carries
// the mean flow, a smooth profile some 1e5 times larger near the clustered walls than the
// differences of neighbouring rows its derivative rests on, so the 47 bits of the split
// would cost it 1e-9 of the wall shear (and the torque follows it).  A block takes a tile of 32 modes x 32 rows; the
// tile's window of rows is read once and each value split once into an exact FP32 pair
// (hi, lo) in shared memory, the stencil is a compensated dot product of the pairs (about 44
// significant bits, against FP32 transforms elsewhere in the form), and the result is
// assembled in FP64.  Everything else keeps the FP64 arithmetic of the FP64 kernels.
constexpr int kXsM = 32;                     // modes per tile (one warp row)
constexpr int kXsR = 32;                     // rows per tile
constexpr int kXsWin = kXsR + kStencil - 1;  // window rows

struct XsTile {
    int mode;   // this thread's mode
    bool in;    // mode < g.mhi
    int r0, r1, jlo;
};

__device__ __forceinline__ XsTile xs_tile(const int* __restrict__ col0, const Geo& g) {
    XsTile t;
    t.mode = g.mlo + blockIdx.x * kXsM + threadIdx.x;
    t.in = t.mode < g.mhi;
    t.r0 = blockIdx.y * kXsR;
    t.r1 = min(t.r0 + kXsR, g.N) - 1;
    t.jlo = col0[t.r0];
    return t;
}

// the tile's stencil weights and the window of f (or of f + f2), split once
__device__ __forceinline__ void xs_load(const double2* __restrict__ f, const double2* __restrict__ f2,
                                        const double* __restrict__ w1, const int* __restrict__ col0,
                                        float4* win, float2* sw, const XsTile& t, const Geo& g) {
    const int tid = threadIdx.y * kXsM + threadIdx.x;
    for (int i = tid; i < (t.r1 - t.r0 + 1) * kStencil; i += blockDim.x * blockDim.y)
        sw[i] = xs::split_hl(w1[(size_t)t.r0 * kStencil + i]);
    const int jhi = col0[t.r1] + kStencil - 1;
    for (int j = t.jlo + threadIdx.y; j <= jhi; j += blockDim.y) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t.in) {
            double2 x = f[(size_t)j * g.nmode + t.mode];
            if (f2) {
                const double2 y = f2[(size_t)j * g.nmode + t.mode];
                x.x += y.x;
                x.y += y.y;
            }
            const float2 a = xs::split_hl(x.x), q = xs::split_hl(x.y);
            v = make_float4(a.x, q.x, a.y, q.y);
        }
        win[(j - t.jlo) * kXsM + threadIdx.x] = v;
    }
    __syncthreads();
}

// D1 of the window's field at row r for this thread's mode
__device__ __forceinline__ double2 xs_drow(const float4* win, const float2* sw, const int* __restrict__ col0,
                                           const XsTile& t, int r) {
    const int w0 = (col0[r] - t.jlo) * kXsM + threadIdx.x;
    return xs_stencil(win + w0, kXsM, sw + (r - t.r0) * kStencil);
}

__global__ void __launch_bounds__(256) k_rhs_pressure_mx(const double2* __restrict__ u, const double2* __restrict__ up,
                                                         const double2* __restrict__ Nc, const double2* __restrict__ Np,
                                                         const double2* __restrict__ X, double2* __restrict__ b,
                                                         const double* __restrict__ rn, const double* __restrict__ irn,
                                                         const double* __restrict__ w1, const double* __restrict__ w2,
                                                         const int* __restrict__ col0, Geo g) {
    __shared__ float4 win[kXsWin * kXsM];
    __shared__ float2 sw[kXsR * kStencil];
    const XsTile t = xs_tile(col0, g);
    xs_load(X, nullptr, w1, col0, win, sw, t, g);
    if (!t.in) return;
    const int mode = t.mode;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const bool mode00 = m == 0 && k == 0;
    const double mm = g.mp * m, kk = g.kz * k;
    for (int j = t.r0 + threadIdx.y; j <= t.r1; j += blockDim.y) {
        if (j == 0 || j == g.N - 1) continue;   // k_rhs_pressure_walls
        const size_t e = (size_t)j * g.nmode + mode;
        const double ir = irn[j];
        double2 out = make_double2(0.0, 0.0);
        {
            const double2 d = mode00 ? drow(X, w1, col0, j, g.nmode, mode) : xs_drow(win, sw, col0, t, j);
            const double2 x = X[e];
            const double2 n1 = Nc[e], n0 = Np[e], m1 = Nc[g.S + e], m0 = Np[g.S + e];
            const double2 z1 = Nc[2 * g.S + e], z0 = Np[2 * g.S + e];
            const double dpx = (2.0 * n1.x - n0.x) - (2.0 * m1.x - m0.x);
            const double dpy = (2.0 * n1.y - n0.y) - (2.0 * m1.y - m0.y);
            const double nzx = 2.0 * z1.x - z0.x, nzy = 2.0 * z1.y - z0.y;
            out.x = -(d.x + x.x * ir + 0.5 * mm * ir * dpx - kk * nzy);
            out.y = -(d.y + x.y * ir + 0.5 * mm * ir * dpy + kk * nzx);
        }
        b[e] = out;
    }
}

__global__ void __launch_bounds__(256) k_rhs_velocity_mx(const double2* __restrict__ u, const double2* __restrict__ up,
                                                         const double2* __restrict__ Nc, const double2* __restrict__ Np,
                                                         const double2* __restrict__ ps, double2* __restrict__ rhs,
                                                         double2* __restrict__ p_out, const double* __restrict__ irn,
                                                         const double* __restrict__ w1, const int* __restrict__ col0,
                                                         double Re_i, double Re_o, Geo g) {
    __shared__ float4 win[kXsWin * kXsM];
    __shared__ float2 sw[kXsR * kStencil];
    const XsTile t = xs_tile(col0, g);
    xs_load(ps, nullptr, w1, col0, win, sw, t, g);
    if (!t.in) return;
    const int mode = t.mode;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const bool mode00 = m == 0 && k == 0;
    for (int j = t.r0 + threadIdx.y; j <= t.r1; j += blockDim.y) {
        const size_t e = (size_t)j * g.nmode + mode;
        const double2 pv = ps[e];
        if (p_out) p_out[e] = pv;
        if (j == 0 || j == g.N - 1) {
            const double Re = (m == 0 && k == 0) ? (j == 0 ? Re_i : Re_o) : 0.0;
            rhs[e] = make_double2(0.0, Re);
            rhs[g.S + e] = make_double2(0.0, -Re);
            rhs[2 * g.S + e] = make_double2(0.0, 0.0);
            continue;
        }
        const double2 d = mode00 ? drow(ps, w1, col0, j, g.nmode, mode) : xs_drow(win, sw, col0, t, j);
        const double tt = g.mp * m * irn[j], kk = g.kz * k;
        const double2 gp[3] = {make_double2(d.x - tt * pv.x, d.y - tt * pv.y),
                               make_double2(d.x + tt * pv.x, d.y + tt * pv.y),
                               make_double2(-kk * pv.y, kk * pv.x)};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t ec = (size_t)c * g.S + e;
            const double2 a = u[ec], q = up[ec], n1 = Nc[ec], n0 = Np[ec];
            rhs[ec] = make_double2((4.0 * a.x - q.x) * g.c1 - (2.0 * n1.x - n0.x) - gp[c].x,
                                   (4.0 * a.y - q.y) * g.c1 - (2.0 * n1.y - n0.y) - gp[c].y);
        }
    }
}

__global__ void __launch_bounds__(256) k_rhs_div_mx(const double2* __restrict__ us, double2* __restrict__ b,
                                                    const double* __restrict__ irn, const double* __restrict__ w1,
                                                    const int* __restrict__ col0, Geo g) {
    __shared__ float4 win[kXsWin * kXsM];
    __shared__ float2 sw[kXsR * kStencil];
    const XsTile t = xs_tile(col0, g);
    xs_load(us, us + g.S, w1, col0, win, sw, t, g);   // the stencil of u*_+ + u*_-
    if (!t.in) return;
    const int mode = t.mode;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const bool mode00 = m == 0 && k == 0;
    const double mm = g.mp * m, kk = g.kz * k;
    for (int j = t.r0 + threadIdx.y; j <= t.r1; j += blockDim.y) {
        const size_t e = (size_t)j * g.nmode + mode;
        if (j == 0 || j == g.N - 1) {
            b[e] = make_double2(0.0, 0.0);
            continue;
        }
        const double ir = irn[j];
        double2 d;
        if (mode00) {
            const double2 dp = drow(us, w1, col0, j, g.nmode, mode), dm = drow(us + g.S, w1, col0, j, g.nmode, mode);
            d = make_double2(dp.x + dm.x, dp.y + dm.y);
        } else {
            d = xs_drow(win, sw, col0, t, j);
        }
        const double2 vp = us[e], vm = us[g.S + e], vz = us[2 * g.S + e];
        b[e] = make_double2(0.5 * d.x + 0.5 * (vp.x + vm.x) * ir + 0.5 * mm * ir * (vp.x - vm.x) - kk * vz.y,
                            0.5 * d.y + 0.5 * (vp.y + vm.y) * ir + 0.5 * mm * ir * (vp.y - vm.y) + kk * vz.x);
    }
}

__global__ void __launch_bounds__(256) k_update_mx(double2* u, double2* up, const double2* Nc, double2* Np, double2* p,
                                                   const double2* __restrict__ us, const double2* __restrict__ phi,
                                                   double2* __restrict__ u_out, const double* __restrict__ irn,
                                                   const double* __restrict__ w1, const int* __restrict__ col0,
                                                   int commit, int* __restrict__ nonfinite, Geo g) {
    __shared__ float4 win[kXsWin * kXsM];
    __shared__ float2 sw[kXsR * kStencil];
    const XsTile t = xs_tile(col0, g);
    xs_load(phi, nullptr, w1, col0, win, sw, t, g);
    if (!t.in) return;
    const int mode = t.mode;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const bool mode00 = m == 0 && k == 0;
    bool bad = false;
    for (int j = t.r0 + threadIdx.y; j <= t.r1; j += blockDim.y) {
        const size_t e = (size_t)j * g.nmode + mode;
        const double2 f = phi[e];
        const double2 d = mode00 ? drow(phi, w1, col0, j, g.nmode, mode) : xs_drow(win, sw, col0, t, j);
        const double tt = g.mp * m * irn[j], kk = g.kz * k;
        const double2 gph[3] = {make_double2(d.x - tt * f.x, d.y - tt * f.y),
                                make_double2(d.x + tt * f.x, d.y + tt * f.y),
                                make_double2(-kk * f.y, kk * f.x)};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t ec = (size_t)c * g.S + e;
            const double2 s = us[ec];
            const double2 un = make_double2(s.x - gph[c].x, s.y - gph[c].y);
            bad |= nonfinite2(un);
            if (commit) {
                up[ec] = u[ec];
                u[ec] = un;
                Np[ec] = Nc[ec];
            } else {
                u_out[ec] = un;
            }
        }
        if (commit) {
            const double q = 3.0 * g.c1;
            const double2 a = p[e];
            p[e] = make_double2(a.x + q * f.x, a.y + q * f.y);
        }
    }
    if (bad && nonfinite) *nonfinite = 1;
}

// x <- A^{-1} x for every mode of nfields consecutive fields (system sets set0, set0+1, ...):
// thread (field, mode, part) runs the register-window substitution down its global column.
__global__ void k_band_solve_g(double2* __restrict__ x, const double* __restrict__ fac,
                               const uint8_t* __restrict__ piv, int set0, int nfields, Geo g) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;   // (mode, part); y = field
    if (t >= 2 * (g.mhi - g.mlo)) return;
    const int part = t & 1;
    const int mode = g.mlo + (t >> 1);
    const int fld = blockIdx.y;
    const int m = mode / g.nk;
    const int k = mode - m * g.nk - g.K;
    const size_t mk = (size_t)m * g.K1 + (k < 0 ? -k : k);
    const size_t per_set = (size_t)g.N * kBands * g.M1K1;
    const int set = set0 + fld;
    smem_band_solve(x + (size_t)fld * g.S, g.nmode, mode, part, g.N, fac + (size_t)set * per_set + mk,
                    piv + (size_t)set * g.N * g.M1K1 + mk, g.M1K1);
}

// Stand-alone solve of one system set for all modes (tc_helmholtz_solve): columns staged in
// shared memory, real and imaginary parts by separate threads.
__global__ void __launch_bounds__(256) k_band_solve_s(double2* __restrict__ x, const double* __restrict__ fac,
                                                      const uint8_t* __restrict__ piv, int set, Geo g, int T) {
    extern __shared__ double2 sm[];
    const int N = g.N;
    const int mode0 = g.mlo + blockIdx.x * T;
    const int nT = min(T, g.mhi - mode0);
    for (int idx = threadIdx.x; idx < N * T; idx += blockDim.x) {
        const int j = idx / T, t = idx - (idx / T) * T;
        sm[idx] = t < nT ? x[(size_t)j * g.nmode + mode0 + t] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (threadIdx.x < 2 * nT) {
        const int t = threadIdx.x >> 1, part = threadIdx.x & 1;
        const int mode = mode0 + t, m = mode / g.nk, k = mode - m * g.nk - g.K;
        const size_t mk = (size_t)m * g.K1 + (k < 0 ? -k : k);
        const size_t per_set = (size_t)N * kBands * g.M1K1;
        smem_band_solve<kPCDepth>(sm, T, t, part, N, fac + (size_t)set * per_set + mk, piv + (size_t)set * N * g.M1K1 + mk, g.M1K1);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < N * T; idx += blockDim.x) {
        const int j = idx / T, t = idx - (idx / T) * T;
        if (t < nT) x[(size_t)j * g.nmode + mode0 + t] = sm[idx];
    }
}

__global__ void k_axpby(double2* __restrict__ y, const double2* __restrict__ a, double ca,
                        const double2* __restrict__ b, double cb, size_t n) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double2 x = a[e], z = b[e];
    y[e] = make_double2(ca * x.x + cb * z.x, ca * x.y + cb * z.y);
}

// Diagnostics: red[1] = max |div_h u| (as ordered bits), red[2] += non-finite, and each
// block's energy sum in red[kDiagPartials + block]; k_diag_sum adds those in a fixed order into
// red[0], so the energy does not depend on the order in which blocks finish.
constexpr int kDiagPartials = 8;
__global__ void k_diag(const double2* __restrict__ u, double* __restrict__ red,
                       const double* __restrict__ rn, const double* __restrict__ w1,
                       const int* __restrict__ col0, double C1, double C2, Geo g) {
    __shared__ double s_e[256];
    __shared__ unsigned long long s_d[256];
    __shared__ int s_n[256];
    const int mode = blockIdx.x * blockDim.x + threadIdx.x;   // y = radial row
    const int j = blockIdx.y;
    const size_t e = (size_t)j * g.nmode + mode;
    double en = 0.0, dv = 0.0;
    int bad = 0;
    if (mode < g.nmode) {
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
        red[kDiagPartials + (size_t)blockIdx.y * gridDim.x + blockIdx.x] = s_e[0];
        atomicMax(reinterpret_cast<unsigned long long*>(&red[1]), s_d[0]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&red[2]), (unsigned long long)s_n[0]);
    }
}

// red[0] = sum of the n block partials: each thread a contiguous run, then a tree (one block)
__global__ void __launch_bounds__(1024) k_diag_sum(double* __restrict__ red, int n) {
    __shared__ double s[1024];
    const int per = (n + 1023) / 1024;
    double a = 0.0;
    for (int i = threadIdx.x * per; i < (threadIdx.x + 1) * per && i < n; ++i) a += red[kDiagPartials + i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) red[0] = s[0];
}

static int blocks_for(size_t n, int bs) { return (int)((n + bs - 1) / bs); }

// doubles of the diagnostics reduction buffer: the fixed slots and one partial per k_diag block
size_t diag_red_doubles(const tc_plan* p) {
    return kDiagPartials + (size_t)blocks_for((size_t)p->nmode, 256) * p->N_r;
}

// modes per block of the fused kernel: four complex columns of N_r rows in shared memory
// Modes per block of the fused kernel (a power of two): the most (up to 16) that still give every SM a block,
// within 96 KB of shared memory for the four columns.  Each block's time is its substitution
// chain, so more modes per block cost little while the blocks fit one wave.
static int pc_modes(const tc_plan* p, int nmode) {
    int T = 16;
    if (p->pc_modes > 0)
        while (T > p->pc_modes) T /= 2;   // a power of two: it divides the block size
    else
        while (T > 4 && (nmode + T - 1) / T < p->num_sms) T /= 2;
    while (T > 1 && (size_t)4 * p->N_r * T * sizeof(double2) > 96 * 1024) T /= 2;
    return T;
}

tc_status launch_solve(tc_plan* p, int set, double2* x, int nfields, cudaStream_t s) {
    Geo g = geo(p);
    int T = 32;
    while (T > 1 && (size_t)p->N_r * T * sizeof(double2) > 96 * 1024) T /= 2;
    const size_t sm = (size_t)p->N_r * T * sizeof(double2);
    TC_CUDA(p, cudaFuncSetAttribute(k_band_solve_s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    for (int f = 0; f < nfields; ++f) {
        const int slot = prof_begin(p, set == kSetP ? kKSolveP : kKSolveH, s);
        k_band_solve_s<<<blocks_for(g.nmode, T), 64, sm, s>>>(x + (size_t)f * g.S, p->d_fac, p->d_piv, set + f, g, T);
        prof_end(p, slot, s);
        TC_LAUNCHED(p, "k_band_solve_s");
    }
    return TC_OK;
}

static tc_status launch_advance_split(tc_plan* p, const double2* u, double2* u_prev, const double2* Ncur,
                                      double2* N_prev, double2* p_out, double2* u_out, char* ws, bool commit,
                                      cudaStream_t s, int ma, int mb) {
    Geo g = geo(p);
    g.mlo = ma * g.nk;
    g.mhi = mb * g.nk;
    const int nm = g.mhi - g.mlo;
    double2* ps = reinterpret_cast<double2*>(ws + p->ws.pstar);
    double2* us = reinterpret_cast<double2*>(ws + p->ws.ustar);
    double2* phi = reinterpret_cast<double2*>(ws + p->ws.phi);   // also holds X before phi
    const dim3 g1(g.N, blocks_for(nm, 128));
    auto sgrid = [&](int nf) { return dim3(blocks_for((size_t)2 * nm, 128), nf); };
    // mixed form: the radial stencils in double-FP32 (the *_mx kernels), tiles of 32 x 32
    const bool mx = p->precision == TC_MIXED;
    const dim3 gx(blocks_for(nm, kXsM), blocks_for(g.N, kXsR)), bx(kXsM, 8);
    int slot = prof_begin(p, kKRhsPressure, s);
    k_nn_r<<<g1, 128, 0, s>>>(Ncur, N_prev, phi, g);
    if (mx)
        k_rhs_pressure_mx<<<gx, bx, 0, s>>>(u, u_prev, Ncur, N_prev, phi, ps, p->d_r, p->d_ir, p->d_w1, p->d_w2,
                                            p->d_col0, g);
    else
        k_rhs_pressure<<<dim3(g.N - 2, blocks_for(nm, 128)), 128, 0, s>>>(u, u_prev, Ncur, N_prev, phi, ps, p->d_r,
                                                                        p->d_ir, p->d_w1, p->d_w2, p->d_col0, g);
    k_rhs_pressure_walls<<<dim3(blocks_for(nm, 128), 2), 128, 0, s>>>(u, u_prev, phi, ps, p->d_r, p->d_w1, p->d_w2,
                                                                     p->d_col0, g);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_rhs_pressure");
    slot = prof_begin(p, kKSolveP, s);
    k_band_solve_g<<<sgrid(1), 128, 0, s>>>(ps, p->d_fac, p->d_piv, kSetP, 1, g);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_band_solve_g");
    slot = prof_begin(p, kKRhsVelocity, s);
    if (mx)
        k_rhs_velocity_mx<<<gx, bx, 0, s>>>(u, u_prev, Ncur, N_prev, ps, us, commit ? p_out : nullptr, p->d_ir,
                                            p->d_w1, p->d_col0, p->Re_i, p->Re_o, g);
    else
        k_rhs_velocity<<<g1, 128, 0, s>>>(u, u_prev, Ncur, N_prev, ps, us, commit ? p_out : nullptr, p->d_ir,
                                          p->d_w1, p->d_col0, p->Re_i, p->Re_o, g);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_rhs_velocity");
    slot = prof_begin(p, kKSolveH, s);
    k_band_solve_g<<<sgrid(3), 128, 0, s>>>(us, p->d_fac, p->d_piv, kSetHp, 3, g);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_band_solve_g");
    slot = prof_begin(p, kKRhsDiv, s);
    if (mx)
        k_rhs_div_mx<<<gx, bx, 0, s>>>(us, phi, p->d_ir, p->d_w1, p->d_col0, g);
    else
        k_rhs_div<<<g1, 128, 0, s>>>(us, phi, p->d_ir, p->d_w1, p->d_col0, g);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_rhs_div");
    slot = prof_begin(p, kKSolveP, s);
    k_band_solve_g<<<sgrid(1), 128, 0, s>>>(phi, p->d_fac, p->d_piv, kSetP, 1, g);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_band_solve_g");
    slot = prof_begin(p, kKUpdate, s);
    if (mx)
        k_update_mx<<<gx, bx, 0, s>>>(const_cast<double2*>(u), u_prev, Ncur, N_prev, p_out, us, phi, u_out, p->d_ir,
                                      p->d_w1, p->d_col0, commit ? 1 : 0, p->d_nonfinite, g);
    else
        k_update<<<g1, 128, 0, s>>>(const_cast<double2*>(u), u_prev, Ncur, N_prev, p_out, us, phi, u_out, p->d_ir,
                                    p->d_w1, p->d_col0, commit ? 1 : 0, p->d_nonfinite, g);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_update");
    return TC_OK;
}

tc_status launch_advance(tc_plan* p, const double2* u, double2* u_prev, const double2* Ncur,
                         double2* N_prev, double2* p_out, double2* u_out, char* ws, bool commit,
                         cudaStream_t s, int ma, int mb) {
    if (mb < 0) mb = p->M + 1;
    if (p->pc_split) return launch_advance_split(p, u, u_prev, Ncur, N_prev, p_out, u_out, ws, commit, s, ma, mb);
    Geo g = geo(p);
    g.mlo = ma * g.nk;
    g.mhi = mb * g.nk;
    const int T = pc_modes(p, g.mhi - g.mlo);
    PCArgs a;
    a.u = u; a.up = u_prev; a.Nc = Ncur; a.Np = N_prev;
    a.u_out = commit ? const_cast<double2*>(u) : u_out;
    a.up_out = commit ? u_prev : nullptr;
    a.Np_out = commit ? N_prev : nullptr;
    a.p = commit ? p_out : nullptr;
    a.rn = p->d_r; a.ir = p->d_ir; a.w1 = p->d_w1; a.w2 = p->d_w2; a.col0 = p->d_col0;
    a.fac = p->d_fac; a.piv = p->d_piv;
    a.fac2 = p->d_fac2; a.piv2 = p->d_piv2; a.spk = p->d_spk; a.rinv = p->d_rinv;
    a.nonfinite = p->d_nonfinite;
    a.Re_i = p->Re_i; a.Re_o = p->Re_o;
    a.commit = commit ? 1 : 0;
    // two partitions while the 12 T substitution threads of the Helmholtz phase fit the block
    g.sh = (p->part_h > 0 && 12 * T <= (T <= 8 ? 128 : 256)) ? p->part_h : 0;
    // mixed form: the split column and weights of the double-FP32 stencils after the rest
    const bool mx = p->precision == TC_MIXED;
    const size_t sm = (size_t)4 * p->N_r * T * sizeof(double2) + (size_t)3 * T * 16 * sizeof(double) +
                      (mx ? (size_t)p->N_r * T * sizeof(float4) +
                                (size_t)((p->N_r * kStencil + 1) & ~1) * sizeof(float2) +
                                (size_t)p->N_r * sizeof(double2) : 0);
    // 128 threads up to 8 modes per block, 256 beyond (6T substitution threads plus helpers)
    const int slot = prof_begin(p, kKPC, s);
    auto run = [&](auto kern, int nth) -> tc_status {
        TC_CUDA(p, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        kern<<<blocks_for(g.mhi - g.mlo, T), nth, sm, s>>>(a, g, T);
        return TC_OK;
    };
    if (T <= 8) TC_TRY_STATUS(mx ? run(k_pc<128, true>, 128) : run(k_pc<128, false>, 128));
    else TC_TRY_STATUS(mx ? run(k_pc<256, true>, 256) : run(k_pc<256, false>, 256));
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_pc");
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
    const dim3 grid(blocks_for(g.nmode, 256), g.N);
    const int slot = prof_begin(p, kKDiag, s);
    k_diag<<<grid, 256, 0, s>>>(u, red, p->d_r, p->d_w1, p->d_col0, C1, C2, g);
    k_diag_sum<<<1, 1024, 0, s>>>(red, (int)(grid.x * grid.y));
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_diag");
    return TC_OK;
}

}  // namespace tc
