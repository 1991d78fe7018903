// Mixed-precision form of the nonlinear term (Sec. 3.2 step 1): the transforms and products
// of the perturbation u' = u - U e_theta run in FP32; the radial derivative and the
// mode-diagonal mean-flow terms keep FP64-grade accuracy without the FP64 pipe, which on
// this GPU retires 2 lanes per SM per clock against 128 for FP32.
//
//   k_prep32    per (c, m, 32 k, 32 r): each FP64 coefficient is split once into an FP32 pair
//               (hi, lo) by integer operations; d_r u' is the FD stencil (Sec. 3.1) applied to
//               the differences u_t - u_r = (hi_t - hi_r) + (lo_t - lo_r). The weights of a
//               derivative stencil sum to zero, so this is the same stencil; the differences
//               are O(dr |d_r u|), which keeps the FP32 rounding of each term at the size of
//               the result instead of the size of u / dr.           -> P[d][c][r][m][k]
//   k_zinv_p32  per (r, m): u', d_r u', d_z u' = i k k_z u' of the 3 components, zero-padded
//               inverse z transforms (FP32).                          -> H1[9][r][m][z]
//   k_theta_s   length-specialised theta pass with streamed products (tc_theta_s.cu), or
//               the generic k_theta with FP32 lines for other lengths -> H2[3][r][m][z]
//   k_zfwd32    per (r, m): forward z transforms, truncation, 1/(P_theta P_z), plus the
//               mean-flow terms in double-FP32 arithmetic (error-free products and sums),
//               assembled into FP64 by exact bit conversion and one FP64 add.
//   k_mean00    beside them on a second stream: the (0, 0) mode of N by an exact Parseval
//               sum in double-FP32 (below), which replaces that coefficient at the end.
//
// Mean-flow terms (Eq. NS_cyl with u_theta = U + u'_theta, U = Re u_theta^{(0,0)}):
//   N_pm += (U/r) i m m_p u'_pm + i (U/r)(u'_+ - u'_-) +- (i/2)(d_r U + U/r)(u'_+ + u'_-),
//   N_z  += (U/r) i m m_p u'_z,   and -U^2/r on the (0,0) mode of N_pm.
// Collected per output: N_+ += i (A u'_+ - B u'_-), N_- += i (C u'_- + B u'_+),
// N_z += i t u'_z, with t = (U/r) m m_p, q = (d_r U + U/r)/2, A = t + U/r + q, B = U/r - q,
// C = t - U/r - q.
#include "tc_internal.cuh"
#include "tc_fft_core.cuh"
#include "tc_fftc.cuh"
#include "tc_split.cuh"

namespace tc {

using namespace xs;

namespace {

// (ah + al)(xh + xl) + (bh + bl)(yh + yl) as an unevaluated pair (s, t), |error| ~ 2^-44 of
// the larger product
__device__ __forceinline__ void dot2(float ah, float al, float xh, float xl, float bh, float bl,
                                     float yh, float yl, float& s, float& t) {
    float p1, e1, p2, e2;
    two_prod(ah, xh, p1, e1);
    e1 = __fmaf_rn(ah, xl, __fmaf_rn(al, xh, e1));
    two_prod(bh, yh, p2, e2);
    e2 = __fmaf_rn(bh, yl, __fmaf_rn(bl, yh, e2));
    two_sum(p1, p2, s, t);
    t = __fadd_rn(t, __fadd_rn(e1, e2));
}

// v + (s + t) in FP64: the FP32 sum is formed error-free, then one FP64 add of exact parts
__device__ __forceinline__ double assemble(float v, float s, float t) {
    float a, b;
    two_sum(v, s, a, b);
    b = __fadd_rn(b, t);
    return f2d_bits(a) + f2d_bits(b);
}

constexpr int kPrepK = 32;   // k values per block (one warp row)
constexpr int kPrepR = 32;   // rows per block
constexpr int kPrepWin = kPrepR + kStencil - 1;

}  // namespace

// ---------------------------------------------------------------- u' and d_r u' in FP32
// P[(d * 3 + c) * S + (r (M+1) + m) nk + kk], d = 0: u', d = 1: d_r u'.
__global__ void __launch_bounds__(256) k_prep32(const double2* __restrict__ u, float2* __restrict__ P,
                                                const float* __restrict__ w1f, const int* __restrict__ col0,
                                                int N_r, int M, int K, int nkt, int nrc, int m0, int mcnt) {
    __shared__ float4 win[kPrepWin * kPrepK];
    __shared__ float sw[kPrepR * kStencil];
    int b = blockIdx.x;
    const int kt = b % nkt;
    b /= nkt;
    const int rc = b % nrc;
    b /= nrc;
    const int m = m0 + b % mcnt;
    const int c = b / mcnt;
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    const size_t colstride = (size_t)(M + 1) * nk;
    const int r0 = rc * kPrepR;
    const int r1 = min(r0 + kPrepR, N_r) - 1;
    const int jlo = col0[r0];
    const int jhi = col0[r1] + kStencil - 1;   // window rows jlo..jhi, at most kPrepWin
    const int kk = kt * kPrepK + threadIdx.x;
    const bool kin = kk < nk;
    // u' = u - U e_theta: on the (0,0) mode Im u'_+ = Im u'_- = (Im u_+ + Im u_-) / 2
    const bool sub = m == 0 && kk == K && c < 2;
    const int tid = threadIdx.y * kPrepK + threadIdx.x;
    for (int i = tid; i < (r1 - r0 + 1) * kStencil; i += blockDim.x * blockDim.y)
        sw[i] = w1f[(size_t)r0 * kStencil + i];
    const double2* base = u + (size_t)c * S + (size_t)m * nk + kk;
    const double2* other = u + (size_t)(c == 1 ? 0 : 1) * S + (size_t)m * nk + kk;   // read only if c < 2
    for (int j = jlo + threadIdx.y; j <= jhi; j += blockDim.y) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kin) {
            double2 x = base[(size_t)j * colstride];
            if (sub) x.y = 0.5 * (x.y + other[(size_t)j * colstride].y);
            const float2 a = split_hl(x.x), q = split_hl(x.y);
            v = make_float4(a.x, q.x, a.y, q.y);   // (hi re, hi im, lo re, lo im)
        }
        win[(j - jlo) * kPrepK + threadIdx.x] = v;
    }
    __syncthreads();
    if (!kin) return;
    float2* Pu = P + (size_t)c * S + (size_t)m * nk + kk;
    float2* Pd = P + (size_t)(3 + c) * S + (size_t)m * nk + kk;
    for (int r = r0 + threadIdx.y; r <= r1; r += blockDim.y) {
        const float4 cen = win[(r - jlo) * kPrepK + threadIdx.x];
        const int w0 = (col0[r] - jlo) * kPrepK + threadIdx.x;
        const float* w = sw + (r - r0) * kStencil;
        float dre = 0.f, dim = 0.f;
#pragma unroll
        for (int t = 0; t < kStencil; ++t) {
            const float4 v = win[w0 + t * kPrepK];
            const float ddr = __fadd_rn(__fsub_rn(v.x, cen.x), __fsub_rn(v.z, cen.z));
            const float ddi = __fadd_rn(__fsub_rn(v.y, cen.y), __fsub_rn(v.w, cen.w));
            dre = __fmaf_rn(w[t], ddr, dre);
            dim = __fmaf_rn(w[t], ddi, dim);
        }
        Pu[(size_t)r * colstride] = make_float2(__fadd_rn(cen.x, cen.z), __fadd_rn(cen.y, cen.w));
        Pd[(size_t)r * colstride] = make_float2(dre, dim);
    }
}

// ---------------------------------------------------------------- inverse z-pass, FP32
// Field f of H1: f = 3 d + c, d in {u', d_r u', d_z u'}.  Line q of the padded transform holds
// wavenumber k = q (q <= K) or q - P_z (q >= P_z - K), zero between.
__device__ __forceinline__ float2 zinv_input(const float2* __restrict__ P, size_t S, size_t line, int f,
                                             int q, int K, int Pz, float kzf) {
    const int k = q <= K ? q : q - Pz;
    if (k < -K) return make_float2(0.f, 0.f);
    const int c = f % 3, d = f / 3;
    const float2 x = P[(size_t)((d == 1 ? 3 : 0) + c) * S + line + k];
    if (d != 2) return x;
    const float kk = kzf * (float)k;
    return make_float2(-kk * x.y, kk * x.x);
}

// generic length: runtime radices, L lines per block
__global__ void __launch_bounds__(256) k_zinv_p32(const float2* __restrict__ P, float2* __restrict__ H1,
                                                  int N_r, int M, int K, float kzf, int L,
                                                  const float2* __restrict__ tw, Radices rad, int m0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Pz = rad.n;
    float2* a = reinterpret_cast<float2*>(smem_raw);
    float2* b = a + (size_t)L * Pz;
    const int groups = 9 / L;
    const int g = blockIdx.x % groups;
    const int rm = blockIdx.x / groups;
    const int r = rm % N_r;
    const int m = m0 + rm / N_r;
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    const size_t line = ((size_t)r * (M + 1) + m) * nk + K;
    for (int idx = threadIdx.x; idx < L * Pz; idx += blockDim.x) {
        const int l = idx / Pz;
        const int q = idx - l * Pz;
        a[idx] = zinv_input(P, S, line, g * L + l, q, K, Pz, kzf);
    }
    __syncthreads();
    float2* res = smem_fft(a, b, L, tw, true, rad);
    for (int idx = threadIdx.x; idx < L * Pz; idx += blockDim.x) {
        const int l = idx / Pz;
        const int z = idx - l * Pz;
        const int f = g * L + l;
        H1[(((size_t)f * N_r + r) * (M + 1) + m) * Pz + z] = res[idx];
    }
}

// compile-time length PZ, L lines per block
// blocks per SM the shared memory of L padded FP32 line pairs allows, at most 1024 threads
template <int PZ, int L, int NT>
constexpr int zinv_minb() {
    constexpr int sm = 2 * L * cft::padded<PZ>() * 8 + 1024;
    constexpr int by_smem = (227 * 1024) / sm;
    constexpr int by_threads = 1024 / NT;
    return by_smem < by_threads ? (by_smem > 0 ? by_smem : 1) : by_threads;
}

// FUSE: the last pass (radix 3, NS = PZ/3) writes its outputs z = j, j + PZ/3, j + 2 PZ/3
// straight to H1 instead of to shared memory for a separate store loop.
template <int PZ, int L, int NT, bool FUSE = false, bool TWS = false>
__global__ void __launch_bounds__(NT, zinv_minb<PZ, L, NT>()) k_zinv_s(const float2* __restrict__ P, float2* __restrict__ H1,
                                               int N_r, int M, int K, float kzf, const float2* __restrict__ tw,
                                               int m0) {
    constexpr int LP = cft::padded<PZ>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* a = reinterpret_cast<float2*>(smem_raw);
    float2* b = a + L * LP;
    // TWS: the twiddle table in shared memory after the two line buffers
    float2* tws = b + L * LP;
    if constexpr (TWS) {
        for (int i = threadIdx.x; i < PZ; i += NT) tws[i] = tw[i];   // visible after the fill's barrier
    }
    const float2* twp = TWS ? tws : tw;
    constexpr int groups = 9 / L;
    const int g = blockIdx.x % groups;
    const int rm = blockIdx.x / groups;
    const int r = rm % N_r;
    const int m = m0 + rm / N_r;
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    const size_t line = ((size_t)r * (M + 1) + m) * nk + K;
    // all loads of the thread first (compile-time trip counts), then the shared-memory stores
    constexpr int NQ = (PZ + NT - 1) / NT;
    float2 vals[L][NQ];
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            const int q = threadIdx.x + i * NT;
            vals[l][i] = (q < PZ && (q <= K || q >= PZ - K)) ? zinv_input(P, S, line, g * L + l, q, K, PZ, kzf)
                                                              : make_float2(0.f, 0.f);
        }
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            const int q = threadIdx.x + i * NT;
            if (q < PZ && (q <= K || q >= PZ - K)) a[l * LP + cft::pd(q)] = vals[l][i];
        }
    __syncthreads();
    // the band K < q < PZ - K is zero: the first pass does not read it
    if constexpr (FUSE) {
        constexpr int NP = cft::Plan<PZ, false>::np;
        static_assert(cft::Plan<PZ, false>::r[NP - 1] == 3, "FUSE needs a plan that ends with radix 3");
        const float2* X = cft::passes_range<PZ, 0, NP - 1, L, NT, true, float2, false, TWS>(a, b, twp, K + 1, PZ - K);
        constexpr int NB3 = PZ / 3;
        for (int it = threadIdx.x; it < L * NB3; it += NT) {
            const int l = it / NB3;
            const int j = it - l * NB3;
            const float2* src = X + l * LP;
            float2 v[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) v[q] = src[cft::pd(j + q * NB3)];
            if (j) {
#pragma unroll
                for (int q = 1; q < 3; ++q) v[q] = cft::vmul(v[q], cft::twiddle<TWS>(twp, q * j));
            }
            cft::dftR<3, true>(v);
            float2* dst = H1 + (((size_t)(g * L + l) * N_r + r) * (M + 1) + m) * PZ;
#pragma unroll
            for (int q = 0; q < 3; ++q) dst[j + q * NB3] = v[q];
        }
    } else {
        const float2* X = cft::passes<PZ, 0, 1, L, NT, true, float2, false, TWS>(a, b, twp, K + 1, PZ - K);
#pragma unroll
        for (int l = 0; l < L; ++l) {
            float2* dst = H1 + (((size_t)(g * L + l) * N_r + r) * (M + 1) + m) * PZ;
            for (int z = threadIdx.x; z < PZ; z += NT) dst[z] = X[l * LP + cft::pd(z)];
        }
    }
}

// ---------------------------------------------------------------- forward z-pass, FP32
// thread 0: U/r, q = (d_r U + U/r)/2 and U in FP64 from the (0,0) column; the coefficients
// A, B, C, t of the mean-flow terms as (hi, lo) pairs
__device__ __forceinline__ void mean_flow_coeffs(const double2* __restrict__ u, const double* __restrict__ rnodes,
                                                 const double* __restrict__ w1, const int* __restrict__ col0,
                                                 int r, int m, int M, int K, size_t S, double mp,
                                                 float* s_cf, double* s_mf) {
    const int nk = 2 * K + 1;
    const size_t col = (size_t)(M + 1) * nk;
    const double2* up = u + K;
    const double2* um = u + S + K;
    double dU = 0.0;
    const int c0 = col0[r];
    for (int t = 0; t < kStencil; ++t)
        dU += w1[r * kStencil + t] * 0.5 * (up[(size_t)(c0 + t) * col].y - um[(size_t)(c0 + t) * col].y);
    const double U = 0.5 * (up[(size_t)r * col].y - um[(size_t)r * col].y);
    const double Ur = U / rnodes[r];
    const double q = 0.5 * (dU + Ur);
    const double t = Ur * mp * m;
    const double cf[4] = {t + Ur + q, Ur - q, t - Ur - q, t};
    for (int i = 0; i < 4; ++i) {
        const float2 x = split_hl(cf[i]);
        s_cf[2 * i] = x.x;
        s_cf[2 * i + 1] = x.y;
    }
    s_mf[0] = Ur;
    s_mf[1] = q;
    s_mf[2] = U;
}

// one output coefficient: scale * v plus the mean-flow terms of component c at (r, m, k), e
__device__ __forceinline__ double2 zfwd_coeff(float2 v, float scale, int c, int m, int k, size_t e, size_t S,
                                              const double2* __restrict__ u, const float* s_cf,
                                              const double* s_mf) {
    const float vr = __fmul_rn(v.x, scale), vi = __fmul_rn(v.y, scale);
    double2 o;
    if (m == 0 && k == 0) {
        // (0,0) mode: t = 0; u'_pm with the averaged imaginary part; -U^2/r on N_pm
        o = make_double2(f2d_bits(vr), f2d_bits(vi));
        if (c < 2) {
            const double Ur = s_mf[0], q = s_mf[1], U = s_mf[2];
            double2 ap = u[e], am = u[S + e];
            const double im = 0.5 * (ap.y + am.y);
            ap.y = im;
            am.y = im;
            const double sg = c == 0 ? 1.0 : -1.0;
            const double dx = ap.x - am.x, dy = ap.y - am.y;
            const double sx = ap.x + am.x, sy = ap.y + am.y;
            o.x += -Ur * dy - sg * q * sy - Ur * U;
            o.y += Ur * dx + sg * q * sx;
        }
        return o;
    }
    // N += i (alpha x + beta y)
    float ah, al, bh = 0.f, bl = 0.f;
    double2 x, y = make_double2(0.0, 0.0);
    if (c == 0) {
        ah = s_cf[0]; al = s_cf[1]; bh = -s_cf[2]; bl = -s_cf[3];
        x = u[e]; y = u[S + e];
    } else if (c == 1) {
        ah = s_cf[4]; al = s_cf[5]; bh = s_cf[2]; bl = s_cf[3];
        x = u[S + e]; y = u[e];
    } else {
        ah = s_cf[6]; al = s_cf[7];
        x = u[2 * S + e];
    }
    const float2 xr = split_hl(x.x), xi = split_hl(x.y);
    const float2 yr = split_hl(y.x), yi = split_hl(y.y);
    float s, t;
    dot2(ah, al, xi.x, xi.y, bh, bl, yi.x, yi.y, s, t);   // alpha Im x + beta Im y
    o.x = assemble(vr, -s, -t);
    dot2(ah, al, xr.x, xr.y, bh, bl, yr.x, yr.y, s, t);   // alpha Re x + beta Re y
    o.y = assemble(vi, s, t);
    return o;
}

// generic length
__global__ void __launch_bounds__(256) k_zfwd32(const float2* __restrict__ H2, double2* __restrict__ N,
                                                int N_r, int M, int K, float scale,
                                                const float2* __restrict__ tw, Radices rad,
                                                const double2* __restrict__ u, const double* __restrict__ rnodes,
                                                const double* __restrict__ w1, const int* __restrict__ col0,
                                                double mp, int Lf, int m0, int mcnt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float s_cf[8];    // A, B, C, t as (hi, lo)
    __shared__ double s_mf[3];   // U/r, q, U (the (0,0) mode is assembled in FP64)
    const int Pz = rad.n;
    float2* a = reinterpret_cast<float2*>(smem_raw);
    float2* b = a + (size_t)Lf * Pz;
    const int cg = blockIdx.x % (3 / Lf);
    const int m = m0 + (blockIdx.x / (3 / Lf)) % mcnt;
    const int r = (blockIdx.x / (3 / Lf)) / mcnt;
    const size_t fstride = (size_t)N_r * (M + 1) * Pz;
    const float2* h = H2 + ((size_t)r * (M + 1) + m) * Pz;
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    for (int idx = threadIdx.x; idx < Lf * Pz; idx += blockDim.x) {
        const int l = idx / Pz;
        const int z = idx - l * Pz;
        a[idx] = h[(cg * Lf + l) * fstride + z];
    }
    if (threadIdx.x == 0) mean_flow_coeffs(u, rnodes, w1, col0, r, m, M, K, S, mp, s_cf, s_mf);
    __syncthreads();
    float2* res = smem_fft(a, b, Lf, tw, false, rad);
    for (int idx = threadIdx.x; idx < Lf * nk; idx += blockDim.x) {
        const int l = idx / nk;
        const int kk = idx - l * nk;
        const int k = kk - K;
        const size_t e = ((size_t)r * (M + 1) + m) * nk + kk;
        const int c = cg * Lf + l;
        N[(size_t)c * S + e] = zfwd_coeff(res[(size_t)l * Pz + (k < 0 ? k + Pz : k)], scale, c, m, k, e, S, u, s_cf, s_mf);
    }
}

// compile-time length PZ, LF components per block
// FUSE: the first pass (NS = 1, no twiddles) reads its inputs z = j + q PZ/R straight from H2
// instead of from a separate load into shared memory.
template <int PZ, int LF, int NT, bool FUSE = false, bool TWS = false>
__global__ void __launch_bounds__(NT) k_zfwd_s(const float2* __restrict__ H2, double2* __restrict__ N,
                                               int N_r, int M, int K, float scale, const float2* __restrict__ tw,
                                               const double2* __restrict__ u, const double* __restrict__ rnodes,
                                               const double* __restrict__ w1, const int* __restrict__ col0,
                                               double mp, int m0, int mcnt) {
    constexpr int LP = cft::padded<PZ>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float s_cf[8];
    __shared__ double s_mf[3];
    float2* a = reinterpret_cast<float2*>(smem_raw);
    float2* b = a + LF * LP;
    float2* tws = b + LF * LP;   // TWS: the twiddle table in shared memory
    if constexpr (TWS) {
        for (int i = threadIdx.x; i < PZ; i += NT) tws[i] = tw[i];   // visible after the load barrier
    }
    const float2* twp = TWS ? tws : tw;
    constexpr int groups = 3 / LF;
    const int cg = blockIdx.x % groups;
    const int m = m0 + (blockIdx.x / groups) % mcnt;
    const int r = (blockIdx.x / groups) / mcnt;
    const size_t fstride = (size_t)N_r * (M + 1) * PZ;
    const float2* h = H2 + ((size_t)r * (M + 1) + m) * PZ;
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    constexpr int NQ = (PZ + NT - 1) / NT;
    const float2* X;
    if constexpr (FUSE) {
        constexpr int NP = cft::Plan<PZ, false>::np;
        constexpr int R0 = cft::Plan<PZ, false>::r[0];
        constexpr int NB0 = PZ / R0;
        for (int idx = threadIdx.x; idx < LF * NB0; idx += NT) {
            const int l = idx / NB0;
            const int j = idx - l * NB0;
            const float2* src = h + (size_t)(cg * LF + l) * fstride;
            float2 v[R0];
#pragma unroll
            for (int q = 0; q < R0; ++q) v[q] = src[j + q * NB0];
            cft::dftR<R0, false>(v);
#pragma unroll
            for (int q = 0; q < R0; ++q) a[l * LP + cft::pd(j * R0 + q)] = v[q];
        }
        if (threadIdx.x == 0) mean_flow_coeffs(u, rnodes, w1, col0, r, m, M, K, S, mp, s_cf, s_mf);
        __syncthreads();
        X = cft::passes_range<PZ, 1, NP, LF, NT, false, float2, false, TWS>(a, b, twp);
    } else {
        float2 vals[LF][NQ];
#pragma unroll
        for (int l = 0; l < LF; ++l)
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                const int z = threadIdx.x + i * NT;
                vals[l][i] = z < PZ ? h[(cg * LF + l) * fstride + z] : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int l = 0; l < LF; ++l)
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                const int z = threadIdx.x + i * NT;
                if (z < PZ) a[l * LP + cft::pd(z)] = vals[l][i];
            }
        if (threadIdx.x == 0) mean_flow_coeffs(u, rnodes, w1, col0, r, m, M, K, S, mp, s_cf, s_mf);
        __syncthreads();
        X = cft::passes<PZ, 0, 1, LF, NT, false, float2, false, TWS>(a, b, twp);
    }
    const size_t e0 = ((size_t)r * (M + 1) + m) * nk;
    // one thread per k for all LF components of the block
    for (int kk = threadIdx.x; kk < nk; kk += NT) {
        const int k = kk - K;
        const int z = k < 0 ? k + PZ : k;
#pragma unroll
        for (int l = 0; l < LF; ++l) {
            const int c = cg * LF + l;
            N[(size_t)c * S + e0 + kk] = zfwd_coeff(X[l * LP + cft::pd(z)], scale, c, m, k, e0 + kk, S, u, s_cf, s_mf);
        }
    }
}

namespace {

template <int PZ, int L, int LF, int NT, bool FUSE, bool TWS>
tc_status run_zpasses_f(tc_plan* p, const float2* P, float2* H1, const float2* H2, const double2* u, double2* N,
                        cudaStream_t s, bool inverse, int ma, int mb) {
    constexpr int LP = cft::padded<PZ>();
    const int mc = mb - ma;
    if (inverse) {
        const size_t sm = ((size_t)2 * L * LP + (TWS ? PZ : 0)) * sizeof(float2);
        auto kern = k_zinv_s<PZ, L, NT, FUSE, TWS>;
        TC_CUDA(p, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const int slot = prof_begin(p, kKZinv32, s);
        kern<<<p->N_r * mc * (9 / L), NT, sm, s>>>(P, H1, p->N_r, p->M, p->K, (float)p->k_z, p->d_tw_z32, ma);
        prof_end(p, slot, s);
        TC_LAUNCHED(p, "k_zinv_s");
    } else {
        const size_t sm = ((size_t)2 * LF * LP + (TWS ? PZ : 0)) * sizeof(float2);
        auto kern = k_zfwd_s<PZ, LF, NT, FUSE, TWS>;
        TC_CUDA(p, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const float scale = (float)(1.0 / ((double)p->P_t * (double)p->P_z));
        const int slot = prof_begin(p, kKZfwd32, s);
        kern<<<p->N_r * mc * (3 / LF), NT, sm, s>>>(H2, N, p->N_r, p->M, p->K, scale, p->d_tw_z32, u, p->d_r,
                                                   p->d_w1, p->d_col0, (double)p->m_p, ma, mc);
        prof_end(p, slot, s);
        TC_LAUNCHED(p, "k_zfwd_s");
    }
    return TC_OK;
}

// The inverse pass always writes from its fused last pass (measured 4-12% faster at
// P_z = 384 ... 1536 on GB300, bit-identical).  The forward pass reads through its fused first
// pass only when that pass keeps every thread busy (LF PZ / R0 >= NT: P_z = 1536, 5% faster);
// with fewer butterflies than threads it measured 6-8% slower (P_z = 768).
template <int PZ, int L, int LF, int NT>
tc_status run_zpasses_s(tc_plan* p, const float2* P, float2* H1, const float2* H2, const double2* u, double2* N,
                        cudaStream_t s, bool inverse, int ma, int mb) {
    constexpr bool fuse_fwd = LF * (PZ / cft::Plan<PZ, false>::r[0]) >= NT;
    // the twiddles stay on the read-only path here: a shared-memory table measured 8% slower at
    // P_z = 768 and 26-29% slower at 1536
    constexpr bool tws = false;
    if (inverse) return run_zpasses_f<PZ, L, LF, NT, true, tws>(p, P, H1, H2, u, N, s, true, ma, mb);
    return run_zpasses_f<PZ, L, LF, NT, fuse_fwd, tws>(p, P, H1, H2, u, N, s, false, ma, mb);
}

// length-specialised z passes over m in [ma, mb); TC_ERR_ARG if P_z has no compile-time plan
tc_status zpass_s(tc_plan* p, const float2* P, float2* H1, const float2* H2, const double2* u, double2* N,
                  cudaStream_t s, bool inverse, int ma, int mb) {
    switch (p->P_z) {
        case 12: return run_zpasses_s<12, 9, 3, 64>(p, P, H1, H2, u, N, s, inverse, ma, mb);
        case 24: return run_zpasses_s<24, 9, 3, 64>(p, P, H1, H2, u, N, s, inverse, ma, mb);
        case 48: return run_zpasses_s<48, 9, 3, 128>(p, P, H1, H2, u, N, s, inverse, ma, mb);
        case 96: return run_zpasses_s<96, 9, 3, 128>(p, P, H1, H2, u, N, s, inverse, ma, mb);
        case 192: return run_zpasses_s<192, 9, 3, 256>(p, P, H1, H2, u, N, s, inverse, ma, mb);
        case 384: return run_zpasses_s<384, 3, 3, 128>(p, P, H1, H2, u, N, s, inverse, ma, mb);
        case 768: return run_zpasses_s<768, 3, 3, 256>(p, P, H1, H2, u, N, s, inverse, ma, mb);
        case 1152: return run_zpasses_s<1152, 3, 3, 256>(p, P, H1, H2, u, N, s, inverse, ma, mb);
        case 1536: return run_zpasses_s<1536, 3, 3, 256>(p, P, H1, H2, u, N, s, inverse, ma, mb);
        case 2304: return run_zpasses_s<2304, 1, 1, 256>(p, P, H1, H2, u, N, s, inverse, ma, mb);
        case 3072: return run_zpasses_s<3072, 1, 1, 256>(p, P, H1, H2, u, N, s, inverse, ma, mb);
    }
    return TC_ERR_ARG;
}

bool zpass_s_ok(const tc_plan* p) {
    switch (p->P_z) {
        case 12: case 24: case 48: case 96: case 192: case 384: case 768: case 1152: case 1536: case 2304: case 3072:
            return p->theta_zt_forced == 0;
    }
    return false;
}

}  // namespace

// before the theta pass, for m in [ma, mb): FP32 split and radial derivative, inverse z pass
tc_status launch_nl_pre32(tc_plan* p, const double2* u, char* ws, cudaStream_t s, int ma, int mb) {
    float2* P = reinterpret_cast<float2*>(ws + p->ws.P32);
    float2* H1 = reinterpret_cast<float2*>(ws + p->ws.H1);
    const int mc = mb - ma;
    const int nk = 2 * p->K + 1;
    const int nkt = (nk + kPrepK - 1) / kPrepK;
    const int nrc = (p->N_r + kPrepR - 1) / kPrepR;
    int slot = prof_begin(p, kKPrep32, s);
    k_prep32<<<(unsigned)(nkt * nrc * mc * 3), dim3(kPrepK, 8), 0, s>>>(u, P, p->d_w1f, p->d_col0, p->N_r, p->M, p->K,
                                                                      nkt, nrc, ma, mc);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_prep32");
    // length-specialised kernels where the plan's lengths have compile-time radix plans, unless
    // the plan fixed the generic theta kernel's z tile (tc_options.theta_zt)
    if (zpass_s_ok(p)) return zpass_s(p, P, H1, nullptr, nullptr, nullptr, s, true, ma, mb);
    const int L = p->zinv_lines32;
    const size_t sm1 = (size_t)2 * L * p->P_z * sizeof(float2);
    TC_CUDA(p, cudaFuncSetAttribute(k_zinv_p32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
    slot = prof_begin(p, kKZinv32, s);
    k_zinv_p32<<<p->N_r * mc * (9 / L), 256, sm1, s>>>(P, H1, p->N_r, p->M, p->K, (float)p->k_z, L,
                                                        p->d_tw_z32, p->rad_z, ma);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_zinv_p32");
    return TC_OK;
}

tc_status launch_nl_theta32(tc_plan* p, char* ws, cudaStream_t s) {
    const float2* H1 = reinterpret_cast<const float2*>(ws + p->ws.H1);
    float2* H2 = reinterpret_cast<float2*>(ws + p->ws.H2);
    if (p->theta_zt_forced == 0 && theta_s_zt(p, false) > 0) return launch_theta_s(p, H1, H2, s);
    return launch_theta32(p, H1, H2, s);
}

// after the theta pass, for m in [ma, mb): forward z pass, mean-flow terms, N in FP64
// The m = 0 line of a real field satisfies N_+(0,k) = conj N_-(0,-k) and N_z(0,k) = conj N_z(0,-k).
// The FP32 products keep this only to rounding (about 1e-8 of N); the FP64 mean-flow terms of
// the next evaluation act on the non-real part of u that such a defect seeds, and above the
// Taylor-vortex onset they amplify it, while nothing saturates it (the transforms read only the
// real part of the m = 0 line).  Projecting N's m = 0 line onto the symmetry leaves that part of
// u to decay under the Stokes operator.  One thread per (r, k >= 0).
__global__ void k_sym_m0(double2* __restrict__ N, int N_r, int M, int K, size_t S) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N_r * (K + 1)) return;
    const int r = idx / (K + 1), k = idx - r * (K + 1);
    const size_t line = (size_t)r * (M + 1) * (2 * K + 1);
    const size_t ep = line + K + k, em = line + K - k;
    auto pair = [&](size_t ia, size_t ib) {   // a <- (a + conj b) / 2, b <- conj a
        const double2 a = N[ia], b = N[ib];
        const double2 v = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        N[ia] = v;
        N[ib] = make_double2(v.x, -v.y);
    };
    pair(ep, S + em);                          // N_+(k), N_-(-k)
    if (k > 0) pair(em, S + ep);               // N_+(-k), N_-(k)
    pair(2 * S + ep, 2 * S + em);              // N_z(k), N_z(-k)
}

static tc_status launch_sym_m0(tc_plan* p, double2* N, cudaStream_t s) {
    const int n = p->N_r * (p->K + 1);
    k_sym_m0<<<(n + 127) / 128, 128, 0, s>>>(N, p->N_r, p->M, p->K, p->S);
    TC_LAUNCHED(p, "k_sym_m0");
    return TC_OK;
}

// ---------------------------------------------------------------- the mean mode of N
// The (m, k) = (0, 0) mode of N is the azimuthal and axial mean of u . grad u, and in a
// step the mean flow changes only through it (the wall torque of Sec. 5.4 is its wall
// derivative).  In FP32 it is the small residue of large fluctuating products, and it
// keeps far less relative accuracy than the rest of N.  With P_theta >= 2M+1 and
// P_z >= 2K+1 no product of two retained modes aliases onto (0, 0), so the mean of a product
// of real fields f g is exactly the Parseval sum over the stored modes
//     <f g> = sum_{m >= 0, k} c_m Re(f_mk conj g_mk),  c_0 = 1, c_m = 2,
// and with d_theta = i m m_p, d_z = i k k_z, u_r = (u_+ + u_-)/2, u_t = -i (u_+ - u_-)/2:
//     <N_r> = <u_r D u_r> + (1/r) sum c_m m m_p Im(u_t conj u_r) + sum c_m k k_z Im(u_z conj u_r) - (1/r) <u_t u_t>
//     <N_t> = <u_r D u_t> + sum c_m k k_z Im(u_z conj u_t) + (1/r) <u_r u_t>
//     <N_z> = <u_r D u_z> + (1/r) sum c_m m m_p Im(u_t conj u_z)
// (D: the FD stencil of Sec. 3.1).  k_mean00 evaluates these from the FP64 state in
// double-FP32 arithmetic (each value an unevaluated FP32 pair, error-free products and
// sums, about 44 significant bits), one thread per (row, mode), and writes each
// warp's sum over its 32 modes; k_mean00_fin adds those in FP64 in a fixed order and
// overwrites N's (0, 0) coefficients: N_pm = <N_r> +- i <N_t>, N_z = <N_z>.

struct dfl {
    float h, l;
};
__device__ __forceinline__ dfl df_of(double d) {
    const float2 s = split_hl(d);
    dfl r;
    r.h = s.x;
    r.l = s.y;
    return r;
}
__device__ __forceinline__ dfl df_norm(float s, float t) {   // |t| <= ulp-sized part of s
    dfl r;
    r.h = __fadd_rn(s, t);
    r.l = __fsub_rn(t, __fsub_rn(r.h, s));
    return r;
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    float s, t;
    two_sum(a.h, b.h, s, t);
    t = __fadd_rn(t, __fadd_rn(a.l, b.l));
    return df_norm(s, t);
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    float p, e;
    two_prod(a.h, b.h, p, e);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    return df_norm(p, e);
}
__device__ __forceinline__ dfl df_neg(dfl a) {
    a.h = -a.h;
    a.l = -a.l;
    return a;
}
__device__ __forceinline__ dfl df_half(dfl a) {   // exact
    a.h = __fmul_rn(a.h, 0.5f);
    a.l = __fmul_rn(a.l, 0.5f);
    return a;
}
__device__ __forceinline__ double df_val(dfl a) { return f2d_bits(a.h) + f2d_bits(a.l); }
// Re(f conj g) and Im(f conj g) of complex pairs (fx, fy), (gx, gy)
__device__ __forceinline__ dfl df_re(dfl fx, dfl fy, dfl gx, dfl gy) { return df_add(df_mul(fx, gx), df_mul(fy, gy)); }
__device__ __forceinline__ dfl df_im(dfl fx, dfl fy, dfl gx, dfl gy) {
    return df_add(df_mul(fy, gx), df_neg(df_mul(fx, gy)));
}
__device__ __forceinline__ dfl df_shfl_down(dfl a, int o) {
    a.h = __shfl_down_sync(0xffffffffu, a.h, o);
    a.l = __shfl_down_sync(0xffffffffu, a.l, o);
    return a;
}

constexpr int kMeanK = 32;   // k values per block (one warp row)
constexpr int kMeanR = 8;    // rows per block (one per warp)
constexpr int kMeanWin = kMeanR + kStencil - 1;

// part[(c * N_r + r) * ntile + tile], c = 0: <N_r>, 1: <N_t>, 2: <N_z>
__global__ void __launch_bounds__(256) k_mean00(const double2* __restrict__ u, double* __restrict__ part,
                                                const double* __restrict__ w1, const int* __restrict__ col0,
                                                const double* __restrict__ irn, int N_r, int M, int K, int ntile,
                                                int nrc, double mp, double kz) {
    // window of the three components' rows, each value split once: (hi re, hi im, lo re, lo im)
    __shared__ float4 win[3][kMeanWin * kMeanK];
    __shared__ float2 sw[kMeanR * kStencil];
    // a block takes 32 consecutive modes of the flattened (m, k) index, so no lane idles at
    // the end of an m line
    const int tile = blockIdx.x % ntile;
    const int rc = blockIdx.x / ntile;
    const int nk = 2 * K + 1;
    const int nmode = (M + 1) * nk;
    const size_t S = (size_t)N_r * nmode;
    const int r0 = rc * kMeanR;
    const int r1 = min(r0 + kMeanR, N_r) - 1;
    const int jlo = col0[r0];
    const int jhi = col0[r1] + kStencil - 1;
    const int mode = tile * kMeanK + threadIdx.x;
    const bool kin = mode < nmode;
    const int tid = threadIdx.y * kMeanK + threadIdx.x;
    for (int i = tid; i < (r1 - r0 + 1) * kStencil; i += blockDim.x * blockDim.y)
        sw[i] = split_hl(w1[(size_t)r0 * kStencil + i]);
    for (int c = 0; c < 3; ++c) {
        const double2* base = u + (size_t)c * S + mode;
        for (int j = jlo + threadIdx.y; j <= jhi; j += blockDim.y) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kin) {
                const double2 x = base[(size_t)j * nmode];
                const float2 a = split_hl(x.x), q = split_hl(x.y);
                v = make_float4(a.x, q.x, a.y, q.y);
            }
            win[c][(j - jlo) * kMeanK + threadIdx.x] = v;
        }
    }
    __syncthreads();
    const int m = kin ? mode / nk : 0;
    const int k = kin ? mode - m * nk - K : 0;
    const float cm = m == 0 ? 1.f : 2.f;
    const dfl mm = df_of(mp * m), kzk = df_of(kz * (double)k);   // m m_p and k k_z as in FP64
    const size_t nseg = (size_t)ntile;
    for (int r = r0 + threadIdx.y; r <= r1; r += blockDim.y) {
        dfl tr = {0.f, 0.f}, tt = {0.f, 0.f}, tz = {0.f, 0.f};
        if (kin) {
            dfl x[3], y[3], dx[3], dy[3];   // value and D of (re, im) of u_+, u_-, u_z
            const int w0 = (col0[r] - jlo) * kMeanK + threadIdx.x;
            const float2* w = sw + (r - r0) * kStencil;
            for (int c = 0; c < 3; ++c) {
                const float4 cen = win[c][(r - jlo) * kMeanK + threadIdx.x];
                x[c] = df_norm(cen.x, cen.z);
                y[c] = df_norm(cen.y, cen.w);
                float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
#pragma unroll
                for (int t = 0; t < kStencil; ++t) {
                    const float4 v = win[c][w0 + t * kMeanK];
                    dot_acc(sx, cx, w[t].x, w[t].y, v.x, v.z);
                    dot_acc(sy, cy, w[t].x, w[t].y, v.y, v.w);
                }
                dx[c] = df_norm(sx, cx);
                dy[c] = df_norm(sy, cy);
            }
            // u_r = (u_+ + u_-)/2, u_t = -i (u_+ - u_-)/2 = ((Im u_+ - Im u_-)/2, -(Re u_+ - Re u_-)/2)
            const dfl urx = df_half(df_add(x[0], x[1])), ury = df_half(df_add(y[0], y[1]));
            const dfl utx = df_half(df_add(y[0], df_neg(y[1]))), uty = df_half(df_add(x[1], df_neg(x[0])));
            const dfl drx = df_half(df_add(dx[0], dx[1])), dry = df_half(df_add(dy[0], dy[1]));
            const dfl dtx = df_half(df_add(dy[0], df_neg(dy[1]))), dty = df_half(df_add(dx[1], df_neg(dx[0])));
            const dfl ir = df_of(irn[r]);
            // <N_r>: u_r D u_r + (1/r) m Im(u_t conj u_r) + k Im(u_z conj u_r) - (1/r) |u_t|^2
            dfl a1 = df_re(urx, ury, drx, dry);
            dfl a2 = df_mul(mm, df_im(utx, uty, urx, ury));
            a2 = df_add(a2, df_neg(df_re(utx, uty, utx, uty)));
            tr = df_add(df_add(a1, df_mul(kzk, df_im(x[2], y[2], urx, ury))), df_mul(ir, a2));
            // <N_t>: u_r D u_t + k Im(u_z conj u_t) + (1/r) Re(u_r conj u_t)
            tt = df_add(df_add(df_re(urx, ury, dtx, dty), df_mul(kzk, df_im(x[2], y[2], utx, uty))),
                        df_mul(ir, df_re(urx, ury, utx, uty)));
            // <N_z>: u_r D u_z + (1/r) m Im(u_t conj u_z)
            tz = df_add(df_re(urx, ury, dx[2], dy[2]), df_mul(ir, df_mul(mm, df_im(utx, uty, x[2], y[2]))));
            if (cm != 1.f) {   // exact doubling
                tr.h *= 2.f; tr.l *= 2.f;
                tt.h *= 2.f; tt.l *= 2.f;
                tz.h *= 2.f; tz.l *= 2.f;
            }
        }
        // sum over the warp's 32 modes (fixed tree)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tr = df_add(tr, df_shfl_down(tr, o));
            tt = df_add(tt, df_shfl_down(tt, o));
            tz = df_add(tz, df_shfl_down(tz, o));
        }
        if (threadIdx.x == 0) {
            const size_t seg = (size_t)tile;
            part[((size_t)0 * N_r + r) * nseg + seg] = df_val(tr);
            part[((size_t)1 * N_r + r) * nseg + seg] = df_val(tt);
            part[((size_t)2 * N_r + r) * nseg + seg] = df_val(tz);
        }
    }
}

// per row: the FP64 sum of the row's segments in a fixed order, into N's (0, 0) coefficients
__global__ void __launch_bounds__(256) k_mean00_fin(const double* __restrict__ part, double2* __restrict__ N,
                                                    int N_r, int M, int K, int nseg, size_t S) {
    __shared__ double sh[3][256];
    const int r = blockIdx.x;
    const int per = (nseg + 255) / 256;
    for (int c = 0; c < 3; ++c) {
        const double* q = part + ((size_t)c * N_r + r) * nseg;
        double a = 0.0;
        for (int i = threadIdx.x * per; i < (threadIdx.x + 1) * per && i < nseg; ++i) a += q[i];
        sh[c][threadIdx.x] = a;
    }
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const size_t e = (size_t)r * (M + 1) * (2 * K + 1) + K;   // (m, k) = (0, 0) of row r
        N[e] = make_double2(sh[0][0], sh[1][0]);
        N[S + e] = make_double2(sh[0][0], -sh[1][0]);
        N[2 * S + e] = make_double2(sh[2][0], 0.0);
    }
}

static int mean00_tiles(const tc_plan* p) { return (p->nmode + kMeanK - 1) / kMeanK; }

size_t mean00_part_doubles(const tc_plan* p) { return (size_t)3 * p->N_r * mean00_tiles(p); }

// the segment sums of the mean mode (reads only u and the plan)
tc_status launch_mean00_part(tc_plan* p, const double2* u, char* ws, cudaStream_t s) {
    const int ntile = mean00_tiles(p);
    const int nrc = (p->N_r + kMeanR - 1) / kMeanR;
    double* part = reinterpret_cast<double*>(ws + p->ws.mean);
    const int slot = prof_begin(p, kKMean00, s);
    k_mean00<<<(unsigned)(ntile * nrc), dim3(kMeanK, kMeanR), 0, s>>>(
        u, part, p->d_w1, p->d_col0, p->d_ir, p->N_r, p->M, p->K, ntile, nrc, (double)p->m_p, p->k_z);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_mean00");
    return TC_OK;
}

// N's (0, 0) coefficients from the segment sums (after the forward z pass wrote N)
tc_status launch_mean00_fin(tc_plan* p, double2* N, char* ws, cudaStream_t s) {
    const double* part = reinterpret_cast<const double*>(ws + p->ws.mean);
    k_mean00_fin<<<p->N_r, 256, 0, s>>>(part, N, p->N_r, p->M, p->K, mean00_tiles(p), p->S);
    TC_LAUNCHED(p, "k_mean00_fin");
    return TC_OK;
}


tc_status launch_nl_post32(tc_plan* p, const double2* u, double2* N, char* ws, cudaStream_t s, int ma, int mb) {
    const float2* H2 = reinterpret_cast<const float2*>(ws + p->ws.H2);
    if (zpass_s_ok(p)) {
        TC_TRY_STATUS(zpass_s(p, nullptr, nullptr, H2, u, N, s, false, ma, mb));
        return ma == 0 ? launch_sym_m0(p, N, s) : TC_OK;
    }
    const int Lf = p->zfwd_lines32;
    const size_t sm3 = (size_t)2 * Lf * p->P_z * sizeof(float2);
    TC_CUDA(p, cudaFuncSetAttribute(k_zfwd32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
    const float scale = (float)(1.0 / ((double)p->P_t * (double)p->P_z));
    const int slot = prof_begin(p, kKZfwd32, s);
    k_zfwd32<<<p->N_r * (mb - ma) * (3 / Lf), 256, sm3, s>>>(H2, N, p->N_r, p->M, p->K, scale, p->d_tw_z32,
                                                              p->rad_z, u, p->d_r, p->d_w1, p->d_col0,
                                                              (double)p->m_p, Lf, ma, mb - ma);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_zfwd32");
    return ma == 0 ? launch_sym_m0(p, N, s) : TC_OK;
}

}  // namespace tc
