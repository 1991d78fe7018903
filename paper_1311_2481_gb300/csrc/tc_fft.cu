// Pseudospectral nonlinear term N(u) = u . grad u (Sec. 3.2 step 1, Eq. NS_cyl) on the
// P_theta x P_z dealiased grid (Sec. 3.1).  Three kernels, one device-memory staging area
// between each (the single-GPU counterpart of the paper's global transposes, Sec. 4):
//
//   k_zinv   per (r, m): radial FD derivative (Sec. 3.1 stencils) and d_z = i k k_z fused into
//            the load; 9 zero-padded inverse transforms along z of the u_+, u_-, u_z lines and
//            of their d_r and d_z lines.                                   -> H1[9][r][m][z]
//   k_theta  per (r, z tile): the 12 real physical fields as 6 complex inverse transforms
//            along theta (two real fields per complex line; d_theta = i m m_p applied here),
//            the pointwise products with the curvature terms, and the forward transform
//            of N_r + i N_theta (giving N_+ and N_- directly) and of N_z (two z per line).
//                                                                          -> H2[3][r][m][z]
//   k_zfwd   per (r, m): forward transforms along z, truncation to |k| <= K, 1/(P_theta P_z).
//
// The mixed-precision form (tc_mixed.cu) shares k_theta with FP32 lines.
// The transforms are mixed-radix (4, 2, 3) Stockham passes in shared memory with twiddles
// from a long-double table.
#include "tc_internal.cuh"
#include "tc_fft_core.cuh"
#include "tc_fftc.cuh"

namespace tc {

// ---------------------------------------------------------------- inverse z-pass
// Field f of H1: f = 3 d + c, c in {+, -, z}, d in {u, d_r u, d_z u}.
__global__ void __launch_bounds__(256) k_zinv(const double2* __restrict__ u, double2* __restrict__ H1,
                                              const double* __restrict__ w1, const int* __restrict__ col0,
                                              int N_r, int M, int K, double kz, int L,
                                              const double2* __restrict__ tw, Radices rad, int m0,
                                              int r0, int nh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Pz = rad.n;
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + (size_t)L * Pz;
    const int groups = 9 / L;
    const int g = blockIdx.x % groups;
    const int rm = blockIdx.x / groups;
    const int rl = rm % nh;        // r fastest: blocks sharing stencil rows run together
    const int r = r0 + rl;
    const int m = m0 + rm / nh;
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    const size_t colstride = (size_t)(M + 1) * nk;
    const int c0 = col0[r];
    for (int idx = threadIdx.x; idx < L * Pz; idx += blockDim.x) {
        const int l = idx / Pz;
        const int q = idx - l * Pz;
        const int k = q <= K ? q : q - Pz;
        double2 x = make_double2(0.0, 0.0);
        if (k >= -K && k <= K) {
            const int f = g * L + l;
            const int c = f % 3, d = f / 3;
            const double2* base = u + (size_t)c * S + (size_t)m * nk + (k + K);
            if (d == 1) {
#pragma unroll
                for (int t = 0; t < kStencil; ++t) {
                    const double w = __ldg(&w1[r * kStencil + t]);
                    const double2 y = __ldg(&base[(size_t)(c0 + t) * colstride]);
                    x.x += w * y.x;
                    x.y += w * y.y;
                }
            } else {
                x = __ldg(&base[(size_t)r * colstride]);
                if (d == 2) {
                    const double kk = kz * k;
                    x = make_double2(-kk * x.y, kk * x.x);
                }
            }
        }
        a[idx] = x;
    }
    __syncthreads();
    double2* res = smem_fft(a, b, L, tw, true, rad);
    for (int idx = threadIdx.x; idx < L * Pz; idx += blockDim.x) {
        const int l = idx / Pz;
        const int z = idx - l * Pz;
        const int f = g * L + l;
        H1[(((size_t)f * nh + rl) * (M + 1) + m) * Pz + z] = res[idx];
    }
}

// ---------------------------------------------------------------- theta pass + products
// Line p of a z value (6 per z):  0 (u_r, u_t)  1 (d_r u_r, d_r u_t)  2 (d_t u_r, d_t u_t)
//                                 3 (d_z u_r, d_z u_t)  4 (u_z, d_r u_z)  5 (d_t u_z, d_z u_z)
template <typename V>
__global__ void __launch_bounds__(256) k_theta(const V* __restrict__ H1, V* __restrict__ H2,
                                               const double* __restrict__ irn, int r0, int nh, int M,
                                               int Pz, double mp, int zt,
                                               const V* __restrict__ tw, Radices rad,
                                               const float* __restrict__ dsc) {
    using T = typename Real<V>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Pt = rad.n;
    const int nl = 6 * zt;
    V* a = reinterpret_cast<V*>(smem_raw);
    V* b = a + (size_t)nl * Pt;
    const int tiles = Pz / zt;
    const int r = blockIdx.x / tiles;   // row within the staged rows r0 .. r0 + nh - 1
    const int z0 = (blockIdx.x % tiles) * zt;
    const size_t fstride = (size_t)nh * (M + 1) * Pz;
    const V* h = H1 + (size_t)r * (M + 1) * Pz + z0;
    // FP32 lines: d_r u_z enters line 4 scaled by a power of two (1 for FP64 lines)
    const T ds = sizeof(T) == 4 ? (T)dsc[r0 + r] : (T)1, ids = (T)1 / ds;

    for (int idx = threadIdx.x; idx < nl * Pt; idx += blockDim.x) { a[idx].x = 0; a[idx].y = 0; }
    __syncthreads();
    // spectra of the 6 complex lines per z
    for (int idx = threadIdx.x; idx < 6 * zt * (M + 1); idx += blockDim.x) {
        // z fastest: neighbouring threads read neighbouring z of one (field, m) line
        const int zi = idx % zt;
        const int t = idx / zt;
        const int m = t % (M + 1);
        const int pr = t / (M + 1);
        V* line = a + (size_t)(zi * 6 + pr) * Pt;
        const size_t o = (size_t)m * Pz + zi;
        const T mm = (T)(mp * m);
        if (pr < 4) {  // (+,-) pair: x = c_r + i c_t has spectrum A_m (m>0), conj(B_m) at -m
            const int fa = pr == 0 ? 0 : pr == 1 ? 3 : pr == 2 ? 0 : 6;
            V A = h[fa * fstride + o], B = h[(fa + 1) * fstride + o];
            if (pr == 2) { A = cmuli(A); A.x *= mm; A.y *= mm; B = cmuli(B); B.x *= mm; B.y *= mm; }
            if (m == 0) {
                V c0; c0.x = (T)0.5 * (A.x + B.x); c0.y = (T)0.5 * (A.y - B.y);
                line[0] = c0;
            } else {
                line[m] = A;
                line[Pt - m] = cconj(B);
            }
        } else {       // two real fields x, y: spectrum X_m + i Y_m, conj(X_m) + i conj(Y_m) at -m
            V X, Y;
            if (pr == 4) { X = h[2 * fstride + o]; Y = h[5 * fstride + o]; Y.x *= ds; Y.y *= ds; }
            else { X = h[2 * fstride + o]; X = cmuli(X); X.x *= mm; X.y *= mm; Y = h[8 * fstride + o]; }
            if (m == 0) {
                V c0; c0.x = X.x; c0.y = Y.x;
                line[0] = c0;
            } else {
                V p1; p1.x = X.x - Y.y; p1.y = X.y + Y.x;
                V p2; p2.x = X.x + Y.y; p2.y = Y.x - X.y;
                line[m] = p1;
                line[Pt - m] = p2;
            }
        }
    }
    __syncthreads();
    V* phys = smem_fft(a, b, nl, tw, true, rad);
    V* fw = phys == a ? b : a;
    const int nzl = (zt + 1) / 2;
    const T ir = (T)irn[r0 + r];   // 1 / r_j from the plan
    for (int idx = threadIdx.x; idx < zt * Pt; idx += blockDim.x) {
        const int zi = idx / Pt;
        const int th = idx - zi * Pt;
        const V* L0 = phys + (size_t)(zi * 6) * Pt + th;
        const V p0 = L0[0], p1 = L0[Pt], p2 = L0[2 * Pt], p3 = L0[3 * Pt], p4 = L0[4 * Pt], p5 = L0[5 * Pt];
        const T ur = p0.x, ut = p0.y, uz = p4.x;
        const T utr = ut * ir;
        const T Nr = ur * p1.x + utr * p2.x + uz * p3.x - ut * utr;
        const T Nt = ur * p1.y + utr * p2.y + uz * p3.y + utr * ur;
        const T Nz = ur * (p4.y * ids) + utr * p5.x + uz * p5.y;
        V q; q.x = Nr; q.y = Nt;
        fw[(size_t)zi * Pt + th] = q;
        V* zl = fw + (size_t)(zt + zi / 2) * Pt + th;
        if (zi & 1) zl->y = Nz;
        else { zl->x = Nz; if (zi + 1 == zt) zl->y = 0; }
    }
    __syncthreads();
    V* other = fw == a ? b : a;
    V* spec = smem_fft(fw, other, zt + nzl, tw, false, rad);
    for (int idx = threadIdx.x; idx < zt * (M + 1); idx += blockDim.x) {
        const int m = idx / zt;
        const int zi = idx - m * zt;
        const V Q = spec[(size_t)zi * Pt + m];
        const V Qm = spec[(size_t)zi * Pt + (m ? Pt - m : 0)];
        const V* SL = spec + (size_t)(zt + zi / 2) * Pt;
        const V Sp = SL[m], Sm = cconj(SL[m ? Pt - m : 0]);
        V nz;
        if (zi & 1) { nz.x = (T)0.5 * (Sp.y - Sm.y); nz.y = (T)0.5 * (Sm.x - Sp.x); }  // (S - conj S-)/(2i)
        else        { nz.x = (T)0.5 * (Sp.x + Sm.x); nz.y = (T)0.5 * (Sp.y + Sm.y); }
        const size_t o = ((size_t)r * (M + 1) + m) * Pz + z0 + zi;
        H2[o] = Q;
        H2[fstride + o] = cconj(Qm);
        H2[2 * fstride + o] = nz;
    }
}

// ---------------------------------------------------------------- forward z-pass
__global__ void __launch_bounds__(256) k_zfwd(const double2* __restrict__ H2, double2* __restrict__ N,
                                              int N_r, int M, int K, double scale,
                                              const double2* __restrict__ tw, Radices rad, int Lf,
                                              int m0, int mcnt, int r0, int nh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Pz = rad.n;
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + (size_t)Lf * Pz;
    const int cg = blockIdx.x % (3 / Lf);     // component group (Lf = 3: all three)
    const int m = m0 + (blockIdx.x / (3 / Lf)) % mcnt;
    const int rl = (blockIdx.x / (3 / Lf)) / mcnt;
    const int r = r0 + rl;
    const size_t fstride = (size_t)nh * (M + 1) * Pz;
    const double2* h = H2 + ((size_t)rl * (M + 1) + m) * Pz;
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    for (int idx = threadIdx.x; idx < Lf * Pz; idx += blockDim.x) {
        const int l = idx / Pz;
        const int z = idx - l * Pz;
        a[idx] = h[(cg * Lf + l) * fstride + z];
    }
    __syncthreads();
    double2* res = smem_fft(a, b, Lf, tw, false, rad);
    for (int idx = threadIdx.x; idx < Lf * nk; idx += blockDim.x) {
        const int l = idx / nk;
        const int c = cg * Lf + l;
        const int kk = idx - l * nk;
        const int k = kk - K;
        const double2 v = res[(size_t)l * Pz + (k < 0 ? k + Pz : k)];
        N[(size_t)c * S + ((size_t)r * (M + 1) + m) * nk + kk] = make_double2(v.x * scale, v.y * scale);
    }
}

// ---------------------------------------------------------------- length-specialised z passes
// Same work as k_zinv / k_zfwd with compile-time radix plans (radices <= 8) and padded lines.
__device__ __forceinline__ double2 zinv_value(const double2* __restrict__ u, const double* __restrict__ w1,
                                              int c0, size_t S, size_t colstride, int r, int m, int nk,
                                              int K, int f, int k, double kz) {
    const int c = f % 3, d = f / 3;
    const double2* base = u + (size_t)c * S + (size_t)m * nk + (k + K);
    double2 x = make_double2(0.0, 0.0);
    if (d == 1) {
#pragma unroll
        for (int t = 0; t < kStencil; ++t) {
            const double w = __ldg(&w1[r * kStencil + t]);
            const double2 y = __ldg(&base[(size_t)(c0 + t) * colstride]);
            x.x += w * y.x;
            x.y += w * y.y;
        }
    } else {
        x = __ldg(&base[(size_t)r * colstride]);
        if (d == 2) {
            const double kk = kz * k;
            x = make_double2(-kk * x.y, kk * x.x);
        }
    }
    return x;
}

template <int PZ, int L, int NT>
__global__ void __launch_bounds__(NT, 2) k_zinv_s64(const double2* __restrict__ u, double2* __restrict__ H1,
                                                    const double* __restrict__ w1, const int* __restrict__ col0,
                                                    int N_r, int M, int K, double kz, const double2* __restrict__ tw,
                                                    int m0, int r0, int nh) {
    constexpr int LP = cft::padded<PZ>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + L * LP;
    constexpr int groups = 9 / L;
    const int g = blockIdx.x % groups;
    const int rm = blockIdx.x / groups;
    const int rl = rm % nh;
    const int r = r0 + rl;
    const int m = m0 + rm / nh;
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    const size_t colstride = (size_t)(M + 1) * nk;
    const int c0 = col0[r];
#pragma unroll
    for (int l = 0; l < L; ++l)
        for (int q = threadIdx.x; q < PZ; q += NT) {
            const int k = q <= K ? q : q - PZ;
            if (k >= -K) a[l * LP + cft::pd(q)] = zinv_value(u, w1, c0, S, colstride, r, m, nk, K, g * L + l, k, kz);
        }
    __syncthreads();
    // the band K < q < PZ - K is zero: the first pass does not read it
    const double2* X = cft::passes<PZ, 0, 1, L, NT, true, double2, true>(a, b, tw, K + 1, PZ - K);
#pragma unroll
    for (int l = 0; l < L; ++l) {
        double2* dst = H1 + (((size_t)(g * L + l) * nh + rl) * (M + 1) + m) * PZ;
        for (int z = threadIdx.x; z < PZ; z += NT) dst[z] = X[l * LP + cft::pd(z)];
    }
}

template <int PZ, int LF, int NT>
__global__ void __launch_bounds__(NT, 2) k_zfwd_s64(const double2* __restrict__ H2, double2* __restrict__ N,
                                                    int N_r, int M, int K, double scale,
                                                    const double2* __restrict__ tw, int m0, int mcnt, int r0, int nh) {
    constexpr int LP = cft::padded<PZ>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + LF * LP;
    constexpr int groups = 3 / LF;
    const int cg = blockIdx.x % groups;
    const int m = m0 + (blockIdx.x / groups) % mcnt;
    const int rl = (blockIdx.x / groups) / mcnt;
    const int r = r0 + rl;
    const size_t fstride = (size_t)nh * (M + 1) * PZ;
    const double2* h = H2 + ((size_t)rl * (M + 1) + m) * PZ;
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
#pragma unroll
    for (int l = 0; l < LF; ++l)
        for (int z = threadIdx.x; z < PZ; z += NT) a[l * LP + cft::pd(z)] = h[(cg * LF + l) * fstride + z];
    __syncthreads();
    const double2* X = cft::passes<PZ, 0, 1, LF, NT, false, double2, true>(a, b, tw);
    const size_t e0 = ((size_t)r * (M + 1) + m) * nk;
    for (int kk = threadIdx.x; kk < nk; kk += NT) {
        const int k = kk - K;
        const int z = k < 0 ? k + PZ : k;
#pragma unroll
        for (int l = 0; l < LF; ++l) {
            const double2 v = X[l * LP + cft::pd(z)];
            N[(size_t)(cg * LF + l) * S + e0 + kk] = make_double2(v.x * scale, v.y * scale);
        }
    }
}

namespace {

// The FP64 staging kernels below process the radial rows r0 .. r0 + nh - 1 and address their
// staging lines (H1, H2) as nh rows; the spectral arrays keep all N_r rows.

template <int PZ, int L, int LF, int NT>
tc_status zpass64(tc_plan* p, const double2* u, double2* H1, const double2* H2, double2* N, cudaStream_t s,
                  bool inverse, int ma, int mb, int r0, int nh) {
    constexpr int LP = cft::padded<PZ>();
    const int mc = mb - ma;
    if (inverse) {
        const size_t sm = (size_t)2 * L * LP * sizeof(double2);
        TC_CUDA(p, cudaFuncSetAttribute(k_zinv_s64<PZ, L, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const int slot = prof_begin(p, kKZinv, s);
        k_zinv_s64<PZ, L, NT><<<nh * mc * (9 / L), NT, sm, s>>>(u, H1, p->d_w1, p->d_col0, p->N_r, p->M,
                                                               p->K, p->k_z, p->d_tw_z, ma, r0, nh);
        prof_end(p, slot, s);
        TC_LAUNCHED(p, "k_zinv_s64");
    } else {
        const size_t sm = (size_t)2 * LF * LP * sizeof(double2);
        TC_CUDA(p, cudaFuncSetAttribute(k_zfwd_s64<PZ, LF, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const double scale = 1.0 / ((double)p->P_t * (double)p->P_z);
        const int slot = prof_begin(p, kKZfwd, s);
        k_zfwd_s64<PZ, LF, NT><<<nh * mc * (3 / LF), NT, sm, s>>>(H2, N, p->N_r, p->M, p->K, scale,
                                                                 p->d_tw_z, ma, mc, r0, nh);
        prof_end(p, slot, s);
        TC_LAUNCHED(p, "k_zfwd_s64");
    }
    return TC_OK;
}

// length-specialised FP64 z passes over m in [ma, mb); TC_ERR_ARG if P_z has no compile-time plan
tc_status zpass64_s(tc_plan* p, const double2* u, double2* H1, const double2* H2, double2* N, cudaStream_t s,
                    bool inverse, int ma, int mb, int r0, int nh) {
    switch (p->P_z) {
        case 12: return zpass64<12, 9, 3, 64>(p, u, H1, H2, N, s, inverse, ma, mb, r0, nh);
        case 24: return zpass64<24, 9, 3, 64>(p, u, H1, H2, N, s, inverse, ma, mb, r0, nh);
        case 48: return zpass64<48, 9, 3, 128>(p, u, H1, H2, N, s, inverse, ma, mb, r0, nh);
        case 96: return zpass64<96, 9, 3, 128>(p, u, H1, H2, N, s, inverse, ma, mb, r0, nh);
        case 192: return zpass64<192, 9, 3, 256>(p, u, H1, H2, N, s, inverse, ma, mb, r0, nh);
        case 384: return zpass64<384, 3, 3, 128>(p, u, H1, H2, N, s, inverse, ma, mb, r0, nh);
        // one line per block from 768 on: three FP64 lines would take 76 KB and more
        case 768: return zpass64<768, 3, 1, 256>(p, u, H1, H2, N, s, inverse, ma, mb, r0, nh);
        case 1152: return zpass64<1152, 1, 1, 128>(p, u, H1, H2, N, s, inverse, ma, mb, r0, nh);
        case 1536: return zpass64<1536, 1, 1, 256>(p, u, H1, H2, N, s, inverse, ma, mb, r0, nh);
        case 2304: return zpass64<2304, 1, 1, 256>(p, u, H1, H2, N, s, inverse, ma, mb, r0, nh);
    }
    return TC_ERR_ARG;
}

bool zpass64_ok(const tc_plan* p) {
    switch (p->P_z) {
        case 12: case 24: case 48: case 96: case 192: case 384: case 768: case 1152: case 1536: case 2304:
            return p->theta_zt_forced == 0;
    }
    return false;
}

}  // namespace

// inverse z pass (with the radial stencil) of the lines of m in [ma, mb), rows r0 .. r0 + nh - 1
static tc_status zinv64(tc_plan* p, const double2* u, double2* H1, cudaStream_t s, int ma, int mb, int r0, int nh) {
    if (zpass64_ok(p)) return zpass64_s(p, u, H1, nullptr, nullptr, s, true, ma, mb, r0, nh);
    const int L = p->zinv_lines;
    const size_t sm1 = (size_t)2 * L * p->P_z * sizeof(double2);
    TC_CUDA(p, cudaFuncSetAttribute(k_zinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
    const int slot = prof_begin(p, kKZinv, s);
    k_zinv<<<nh * (mb - ma) * (9 / L), p->thr_zinv, sm1, s>>>(u, H1, p->d_w1, p->d_col0, p->N_r, p->M, p->K,
                                                             p->k_z, L, p->d_tw_z, p->rad_z, ma, r0, nh);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_zinv");
    return TC_OK;
}

// forward z pass of the lines of m in [ma, mb), rows r0 .. r0 + nh - 1, into N
static tc_status zfwd64(tc_plan* p, const double2* H2, double2* N, cudaStream_t s, int ma, int mb, int r0, int nh) {
    if (zpass64_ok(p)) return zpass64_s(p, nullptr, nullptr, H2, N, s, false, ma, mb, r0, nh);
    const int Lf = p->zfwd_lines;
    const size_t sm3 = (size_t)2 * Lf * p->P_z * sizeof(double2);
    TC_CUDA(p, cudaFuncSetAttribute(k_zfwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
    const double scale = 1.0 / ((double)p->P_t * (double)p->P_z);
    const int slot = prof_begin(p, kKZfwd, s);
    k_zfwd<<<nh * (mb - ma) * (3 / Lf), p->thr_zfwd, sm3, s>>>(H2, N, p->N_r, p->M, p->K, scale, p->d_tw_z,
                                                              p->rad_z, Lf, ma, mb - ma, r0, nh);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_zfwd");
    return TC_OK;
}

static tc_status theta64(tc_plan* p, const double2* H1, double2* H2, cudaStream_t s, int r0, int nh) {
    if (p->theta_zt_forced == 0 && theta_s_zt(p, true) > 0) return launch_theta_s64(p, H1, H2, s, r0, nh);
    const int zt = p->zt;
    const size_t sm2 = (size_t)2 * 6 * zt * p->P_t * sizeof(double2);
    TC_CUDA(p, cudaFuncSetAttribute(k_theta<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
    const int slot = prof_begin(p, kKTheta, s);
    k_theta<double2><<<nh * (p->P_z / zt), p->thr_theta, sm2, s>>>(H1, H2, p->d_ir, r0, nh, p->M, p->P_z,
                                                                  (double)p->m_p, zt, p->d_tw_t, p->rad_t,
                                                                  nullptr);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_theta");
    return TC_OK;
}

tc_status launch_zinv_fp64(tc_plan* p, const double2* u, double2* H1, cudaStream_t s, int r0, int nh) {
    return zinv64(p, u, H1, s, 0, p->M + 1, r0, nh);
}

// theta pass of the mixed form with the generic kernel: FP32 lines (H1, H2 in float2), all rows
tc_status launch_theta32(tc_plan* p, const float2* H1, float2* H2, cudaStream_t s) {
    const int zt = p->zt32;
    const size_t sm2 = (size_t)2 * 6 * zt * p->P_t * sizeof(float2);
    TC_CUDA(p, cudaFuncSetAttribute(k_theta<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
    const int slot = prof_begin(p, kKTheta32, s);
    k_theta<float2><<<p->N_r * (p->P_z / zt), 256, sm2, s>>>(H1, H2, p->d_ir, 0, p->N_r, p->M, p->P_z,
                                                             (double)p->m_p, zt, p->d_tw_t32, p->rad_t, p->d_dsc);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_theta");
    return TC_OK;
}

// The nonlinear term.  FP64 lines: the three transforms slab by slab of p->stage_rows radial
// rows (a row's transforms read no other row's staging), so the staging holds 12 line sets of
// stage_rows rows.  Mixed form: FP32 lines of all rows (tc_mixed.cu).
tc_status launch_nonlinear(tc_plan* p, const double2* u, double2* N, char* ws, cudaStream_t s) {
    if (p->precision == TC_MIXED && p->opt.mean_fp32) {
        TC_TRY_STATUS(launch_nl_pre32(p, u, ws, s, 0, p->M + 1));
        TC_TRY_STATUS(launch_nl_theta32(p, ws, s));
        return launch_nl_post32(p, u, N, ws, s, 0, p->M + 1);
    }
    if (p->precision == TC_MIXED) {
        // the mean mode reads only u: it runs on the plan's second stream beside the FP32
        // transforms, and its sums replace N's (0, 0) coefficients after the forward z pass
        TC_CUDA(p, cudaEventRecord(p->mean_ev[0], s));
        TC_CUDA(p, cudaStreamWaitEvent(p->mean_stream, p->mean_ev[0], 0));
        TC_TRY_STATUS(launch_mean00_part(p, u, ws, p->mean_stream));
        TC_CUDA(p, cudaEventRecord(p->mean_ev[1], p->mean_stream));
        TC_TRY_STATUS(launch_nl_pre32(p, u, ws, s, 0, p->M + 1));
        TC_TRY_STATUS(launch_nl_theta32(p, ws, s));
        TC_TRY_STATUS(launch_nl_post32(p, u, N, ws, s, 0, p->M + 1));
        TC_CUDA(p, cudaStreamWaitEvent(s, p->mean_ev[1], 0));
        return launch_mean00_fin(p, N, ws, s);
    }
    double2* H1 = reinterpret_cast<double2*>(ws + p->ws.H1);
    double2* H2 = reinterpret_cast<double2*>(ws + p->ws.H2);
    for (int r0 = 0; r0 < p->N_r; r0 += p->stage_rows) {
        const int nh = p->N_r - r0 < p->stage_rows ? p->N_r - r0 : p->stage_rows;
        TC_TRY_STATUS(zinv64(p, u, H1, s, 0, p->M + 1, r0, nh));
        TC_TRY_STATUS(theta64(p, H1, H2, s, r0, nh));
        TC_TRY_STATUS(zfwd64(p, H2, N, s, 0, p->M + 1, r0, nh));
    }
    return TC_OK;
}

}  // namespace tc
