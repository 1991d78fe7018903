// Length-specialised theta pass (Sec. 3.2 step 1, Eq. NS_cyl) for the common transform
// lengths, FP32 or FP64 lines.  Same input (H1) and output (H2) as k_theta, organised
// differently:
//
//  * the radices of each length are compile-time constants (e.g. 768 = 16 * 16 * 3 for FP32
//    lines), so the Stockham index arithmetic folds and fewer passes are needed;
//  * lines sit in shared memory with one padding slot per 32 entries, which makes the
//    stride-R stores of the first pass and all later accesses bank-conflict free;
//  * the products are streamed: u is transformed first and kept per physical point (in shared
//    memory, each point owned by one thread), then the derivative line pairs go through the
//    transform two lines per z at a time and are accumulated into N.  Only 2 lines per z are
//    resident instead of 6, so a block holds several z values, and the H1 loads and H2 stores
//    of a (field, m) cover 16- or 32-byte runs along z.
#include "tc_internal.cuh"
#include "tc_fftc.cuh"

namespace tc {

using namespace cft;

// H1 fields: f = 3 d + c, c in {+, -, z}, d in {u, d_r u, d_z u}.
// Phase 0: lines (u_r, u_t) and (u_z, d_r u_z); phase 1: (d_r u_r, d_r u_t) and
// (d_t u_r, d_t u_t); phase 2: (d_z u_r, d_z u_t) and (d_t u_z, d_z u_z); then the forward
// transform of N_r + i N_t (one line per z) and of N_z (two z per line).
// FUSE (plans whose last pass is radix 3): the last inverse pass feeds the products from
// registers instead of storing its lines and reading them back: a thread takes the radix-3
// butterfly j of both lines of a z, whose outputs are the points theta = j, j + PT/3,
// j + 2 PT/3 of that z, and those points are its own in every phase.  Likewise the first
// forward pass (NS = 1) reads N_r + i N_t and N_z from the per-point arrays directly.
template <typename V, int PT, int ZT, int NT, int MINB, bool R8, bool FUSE = false>
__global__ void __launch_bounds__(NT, MINB) k_theta_s(const V* __restrict__ H1, V* __restrict__ H2,
                                                      const double* __restrict__ irn, int r0, int nh, int M, int Pz,
                                                      double mp, const V* __restrict__ tw,
                                                      const float* __restrict__ dsc) {
    using T = typename Elem<V>::T;
    constexpr int LP = padded<PT>();
    constexpr int NL = 2 * ZT;             // resident lines in a phase
    constexpr int NLF = ZT + (ZT + 1) / 2;  // lines of the forward transform
    constexpr int NPT = ZT * PT;           // physical points of the block
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NP = Plan<PT, R8>::np;
    static_assert(!FUSE || Plan<PT, R8>::r[NP - 1] == 3, "FUSE needs a plan that ends with radix 3");
    V* A = reinterpret_cast<V*>(smem_raw);
    V* B = A + NL * LP;
    // per physical point: Ua = (u_r, u_t / r), Ub = (u_z, N_z), Nn = (N_r, N_t); each point is
    // owned by one thread in every phase
    V* Ua = B + NL * LP;
    V* Ub = Ua + NPT;
    V* Nn = Ub + NPT;
    // FUSE: the twiddle table in shared memory (PT entries), read by every pass (measured 4-6%
    // faster than the read-only path at P_theta = 384, 768, 1536 and 2% slower at 1152, which
    // keeps the read-only path)
    constexpr bool TWS = FUSE && PT != 1152;
    V* TW = Nn + NPT;
    const V* twp = TWS ? TW : tw;
    const int tiles = Pz / ZT;
    const int r = blockIdx.x / tiles;   // row within the staged rows r0 .. r0 + nh - 1
    const int z0 = (blockIdx.x % tiles) * ZT;
    const size_t fstride = (size_t)nh * (M + 1) * Pz;
    const V* h = H1 + (size_t)r * (M + 1) * Pz + z0;
    const T ir = (T)irn[r0 + r];   // 1 / r_j from the plan
    const T mpf = (T)mp;
    // FP32 lines: d_r u_z enters the (u_z, d_r u_z) line scaled by a power of two, so that
    // its rounding does not swamp u_z near the walls; FP64 lines are not scaled
    const T ds = sizeof(V) == 8 ? (T)dsc[r0 + r] : (T)1, ids = (T)1 / ds;
    const int zi = threadIdx.x % ZT;        // z of this thread in the load and store loops
    const int mstep = NT / ZT;
    if constexpr (TWS) {
        for (int i = threadIdx.x; i < PT; i += NT) TW[i] = tw[i];   // visible after the first fill's barrier
    }
    // one phase's products at point pt from the two physical lines' values p0, p1
    auto products = [&](int phase, int pt, V p0, V p1) {
        if (phase == 0) {
            const T utr = p0.y * ir;
            Ua[pt] = vmk<V>(p0.x, utr);
            Ub[pt] = vmk<V>(p1.x, p0.x * (p1.y * ids));              // N_z = u_r d_r u_z
            Nn[pt] = vmk<V>(-p0.y * utr, utr * p0.x);                // curvature terms
        } else if (phase == 1) {
            const V a = Ua[pt];
            V n = Nn[pt];
            n.x += a.x * p0.x + a.y * p1.x;
            n.y += a.x * p0.y + a.y * p1.y;
            Nn[pt] = n;
        } else {
            const V a = Ua[pt];
            V b = Ub[pt];
            V n = Nn[pt];
            n.x += b.x * p0.x;
            n.y += b.x * p0.y;
            Nn[pt] = n;
            b.y += a.y * p1.x + b.x * p1.y;
            Ub[pt] = b;
        }
    };

#pragma unroll 1
    for (int phase = 0; phase < 3; ++phase) {
        // spectra of the two lines of each z (lines 2 zi and 2 zi + 1)
        if constexpr (sizeof(V) == 16) {
            // FP64 lines: the four fields of the phase for two m values per thread loaded
            // before they are placed (measured faster; 2M+1 <= PT bounds the m values)
            const int fa = phase == 0 ? 0 : phase == 1 ? 3 : 6;
            const int fc = phase == 0 ? 2 : phase == 1 ? 0 : 2;
            const int fd = phase == 0 ? 5 : phase == 1 ? 1 : 8;
            constexpr int MI = (PT / 2 + 1 + NT / ZT - 1) / (NT / ZT);
            constexpr int G = 2;
            V* L0 = A + (2 * zi) * LP;
            V* L1 = L0 + LP;
#pragma unroll
            for (int i0 = 0; i0 < MI; i0 += G) {
                V va[G], vb[G], vc[G], vd[G];
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    const int m = (int)threadIdx.x / ZT + (i0 + i) * mstep;
                    if (i0 + i < MI && m <= M) {
                        const size_t o = (size_t)m * Pz + zi;
                        va[i] = h[fa * fstride + o];
                        vb[i] = h[(fa + 1) * fstride + o];
                        vc[i] = h[fc * fstride + o];
                        vd[i] = h[fd * fstride + o];
                    }
                }
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    const int m = (int)threadIdx.x / ZT + (i0 + i) * mstep;
                    if (i0 + i < MI && m <= M) {
                        const T mm = mpf * (T)m;
                        put_pair(L0, PT, m, va[i], vb[i]);
                        if (phase == 0) put_real2(L1, PT, m, vc[i], vd[i]);
                        else if (phase == 1) put_pair(L1, PT, m, imul(vc[i], mm), imul(vd[i], mm));
                        else put_real2(L1, PT, m, imul(vc[i], mm), vd[i]);
                    }
                }
            }
        } else {
            // FP32 lines: one m value at a time (the extra registers of batched loads cost
            // more than the latency they hide here)
            for (int m = (int)threadIdx.x / ZT; m <= M; m += mstep) {
                const size_t o = (size_t)m * Pz + zi;
                const T mm = mpf * (T)m;
                V* L0 = A + (2 * zi) * LP;
                V* L1 = L0 + LP;
                if (phase == 0) {
                    put_pair(L0, PT, m, h[0 * fstride + o], h[1 * fstride + o]);
                    const V drz = h[5 * fstride + o];
                    put_real2(L1, PT, m, h[2 * fstride + o], vmk<V>(drz.x * ds, drz.y * ds));
                } else if (phase == 1) {
                    put_pair(L0, PT, m, h[3 * fstride + o], h[4 * fstride + o]);
                    put_pair(L1, PT, m, imul(h[0 * fstride + o], mm), imul(h[1 * fstride + o], mm));
                } else {
                    put_pair(L0, PT, m, h[6 * fstride + o], h[7 * fstride + o]);
                    put_real2(L1, PT, m, imul(h[2 * fstride + o], mm), h[8 * fstride + o]);
                }
            }
        }
        __syncthreads();
        // the band M < p < PT - M of every line is zero: the first pass does not read it
        if constexpr (FUSE) {
            // all passes but the last, then the last radix-3 pass (NS = PT/3, unit twiddle
            // step) on both lines of each z with the products taken from its outputs
            const V* X = passes_range<PT, 0, NP - 1, NL, NT, true, V, R8, TWS>(A, B, twp, M + 1, PT - M);
            constexpr int NB3 = PT / 3;
            for (int it = threadIdx.x; it < ZT * NB3; it += NT) {
                const int z = it / NB3;
                const int j = it - z * NB3;
                const V* s0 = X + (2 * z) * LP;
                const V* s1 = s0 + LP;
                V a[3], b[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    a[q] = s0[pd(j + q * NB3)];
                    b[q] = s1[pd(j + q * NB3)];
                }
                if (j) {
#pragma unroll
                    for (int q = 1; q < 3; ++q) {
                        const V w = twiddle<TWS>(twp, q * j);
                        a[q] = vmul(a[q], w);
                        b[q] = vmul(b[q], w);
                    }
                }
                dftR<3, true>(a);
                dftR<3, true>(b);
#pragma unroll
                for (int q = 0; q < 3; ++q) products(phase, z * PT + j + q * NB3, a[q], b[q]);
            }
            __syncthreads();   // the next fill overwrites the lines
        } else {
            const V* X = passes<PT, 0, 1, NL, NT, true, V, R8>(A, B, tw, M + 1, PT - M);
            for (int pt = threadIdx.x; pt < NPT; pt += NT) {
                const int z = pt / PT;
                const int th = pt - z * PT;
                products(phase, pt, X[(2 * z) * LP + pd(th)], X[(2 * z + 1) * LP + pd(th)]);
            }
            if (result_in_first<PT, R8>()) __syncthreads();   // the next fill overwrites X
        }
    }

    // forward transform: line z holds N_r + i N_t, line ZT + z/2 holds N_z of two z values
    const V* Y;
    if constexpr (FUSE) {
        // first forward pass (NS = 1, no twiddles) straight from the per-point arrays
        constexpr int R0 = Plan<PT, R8>::r[0];
        constexpr int NB0 = PT / R0;
        for (int idx = threadIdx.x; idx < NLF * NB0; idx += NT) {
            const int line = idx / NB0;
            const int j = idx - line * NB0;
            V v[R0];
#pragma unroll
            for (int q = 0; q < R0; ++q) {
                const int th = j + q * NB0;
                if (line < ZT) {
                    v[q] = Nn[line * PT + th];
                } else {
                    const int z = 2 * (line - ZT);
                    v[q] = vmk<V>(Ub[z * PT + th].y, z + 1 < ZT ? Ub[(z + 1) * PT + th].y : (T)0);
                }
            }
            dftR<R0, false>(v);
            V* dst = A + line * LP;
#pragma unroll
            for (int q = 0; q < R0; ++q) dst[pd(j * R0 + q)] = v[q];
        }
        __syncthreads();
        Y = passes_range<PT, 1, NP, NLF, NT, false, V, R8, TWS>(A, B, twp);
    } else {
        for (int pt = threadIdx.x; pt < NPT; pt += NT) {
            const int z = pt / PT;
            const int th = pt - z * PT;
            A[z * LP + pd(th)] = Nn[pt];
            T* zl = reinterpret_cast<T*>(A + (ZT + z / 2) * LP + pd(th));
            const T nz = Ub[pt].y;
            if (z & 1) {
                zl[1] = nz;
            } else {
                zl[0] = nz;
                if (z + 1 == ZT) zl[1] = 0;
            }
        }
        __syncthreads();
        Y = passes<PT, 0, 1, NLF, NT, false, V, R8>(A, B, tw);
    }
    for (int m = (int)threadIdx.x / ZT; m <= M; m += mstep) {
        const int mneg = m ? PT - m : 0;
        const V Q = Y[zi * LP + pd(m)];
        const V Qm = Y[zi * LP + pd(mneg)];
        const V* SL = Y + (ZT + zi / 2) * LP;
        const V Sp = SL[pd(m)];
        const V Smc = SL[pd(mneg)];
        const V Sm = vmk<V>(Smc.x, -Smc.y);
        V nz;
        if (zi & 1) nz = vmk<V>((T)0.5 * (Sp.y - Sm.y), (T)0.5 * (Sm.x - Sp.x));   // (S - conj S-)/(2i)
        else nz = vmk<V>((T)0.5 * (Sp.x + Sm.x), (T)0.5 * (Sp.y + Sm.y));
        const size_t o = ((size_t)r * (M + 1) + m) * Pz + z0 + zi;
        H2[o] = Q;
        H2[fstride + o] = vmk<V>(Qm.x, -Qm.y);
        H2[2 * fstride + o] = nz;
    }
}

namespace {

template <typename V, int PT, int ZT, int NT, int MINB, bool R8, bool FUSE = false>
tc_status run_theta_s(tc_plan* p, const V* H1, V* H2, const V* tw, cudaStream_t s, int r0, int nh) {
    constexpr int LP = padded<PT>();
    const size_t sm = ((size_t)2 * 2 * ZT * LP + (size_t)3 * ZT * PT + (FUSE && PT != 1152 ? PT : 0)) * sizeof(V);
    auto kern = k_theta_s<V, PT, ZT, NT, MINB, R8, FUSE>;
    TC_CUDA(p, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int slot = prof_begin(p, sizeof(V) == 8 ? kKTheta32 : kKTheta, s);
    kern<<<nh * (p->P_z / ZT), NT, sm, s>>>(H1, H2, p->d_ir, r0, nh, p->M, p->P_z, (double)p->m_p, tw,
                                             sizeof(V) == 8 ? p->d_dsc : nullptr);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_theta_s");
    return TC_OK;
}

// FP32 launch shapes per length: variant 1 radices <= 16, Z z values per block, 2 blocks per
// SM; variants 2 and 3 radices <= 8 (64 / 76 registers), half the z values per block, 4 / 3
// blocks per SM; variant 4 is variant 1 with the last inverse pass and the first forward
// pass fused into the products (FUSE), for lengths 384 and up.  Default (0): variant 2 up to
// P_theta = 96, where occupancy decides; variant 1 at 192; variant 4 from 384 on, where the
// extra pass of the radix-8 plan costs more (0.057 vs 0.082 ms at P_theta = 96; 14.1 vs
// 18.5 ms at 768) and the fusion saves 4-11% (13.5 -> 12.0 ms at 768, N_r = 256), with
// bit-identical results.

template <int PT, int Z, int NT>
tc_status theta_s32(tc_plan* p, const float2* H1, float2* H2, cudaStream_t s) {
    const float2* tw = p->d_tw_t32;
    constexpr int Zh = Z > 1 ? Z / 2 : 1;
    const int v = p->theta_variant ? p->theta_variant : (PT <= 96 ? 2 : PT >= 384 ? 4 : 1);
    switch (v) {
        case 2: return run_theta_s<float2, PT, Zh, NT, (NT > 256 ? 3 : 4), true>(p, H1, H2, tw, s, 0, p->N_r);
        case 3: return run_theta_s<float2, PT, Zh, NT, (NT > 256 ? 2 : 3), true>(p, H1, H2, tw, s, 0, p->N_r);
        case 4:
            if constexpr (PT >= 384) return run_theta_s<float2, PT, Z, NT, 2, false, true>(p, H1, H2, tw, s, 0, p->N_r);
            return run_theta_s<float2, PT, Z, NT, 2, false>(p, H1, H2, tw, s, 0, p->N_r);
        default: return run_theta_s<float2, PT, Z, NT, 2, false>(p, H1, H2, tw, s, 0, p->N_r);
    }
}

}  // namespace

// z values per block of the streamed theta pass for this plan and line type, 0 if none
int theta_s_zt(const tc_plan* p, bool fp64) {
    int zt = 0;
    if (fp64) {
        switch (p->P_t) {
            case 96: zt = 4; break;
            case 192: case 384: zt = 2; break;
            case 768: case 1152: zt = 1; break;
            default: return 0;
        }
    } else {
        switch (p->P_t) {
            case 48: case 96: zt = 8; break;
            case 192: case 384: zt = 4; break;
            case 768: case 1152: case 1536: zt = 2; break;
            default: return 0;
        }
    }
    if (2 * p->M + 1 > p->P_t || p->P_z % zt) return 0;
    return zt;
}

tc_status launch_theta_s(tc_plan* p, const float2* H1, float2* H2, cudaStream_t s) {
    if (theta_s_zt(p, false) == 0) return TC_ERR_ARG;
    switch (p->P_t) {
        case 48: return theta_s32<48, 8, 128>(p, H1, H2, s);
        case 96: return theta_s32<96, 8, 256>(p, H1, H2, s);
        case 192: return theta_s32<192, 4, 256>(p, H1, H2, s);
        case 384: return theta_s32<384, 4, 256>(p, H1, H2, s);
        case 768: return theta_s32<768, 2, 256>(p, H1, H2, s);
        case 1152: return theta_s32<1152, 2, 384>(p, H1, H2, s);
        case 1536: return theta_s32<1536, 2, 256>(p, H1, H2, s);
    }
    return TC_ERR_ARG;
}

tc_status launch_theta_s64(tc_plan* p, const double2* H1, double2* H2, cudaStream_t s, int r0, int nh) {
    if (theta_s_zt(p, true) == 0) return TC_ERR_ARG;
    const double2* tw = p->d_tw_t;
    // the FUSE form measured no faster with FP64 lines (0.4425 vs 0.4445 ms at the bench size):
    // the FP64 pipe, not shared memory, bounds this kernel
    switch (p->P_t) {
        case 96: return run_theta_s<double2, 96, 4, 128, 3, true>(p, H1, H2, tw, s, r0, nh);
        case 192: return run_theta_s<double2, 192, 2, 128, 3, true>(p, H1, H2, tw, s, r0, nh);
        case 384: return run_theta_s<double2, 384, 2, 256, 2, true>(p, H1, H2, tw, s, r0, nh);
        case 768: return run_theta_s<double2, 768, 1, 256, 2, true>(p, H1, H2, tw, s, r0, nh);
        case 1152: return run_theta_s<double2, 1152, 1, 384, 1, true>(p, H1, H2, tw, s, r0, nh);
    }
    return TC_ERR_ARG;
}

}  // namespace tc
