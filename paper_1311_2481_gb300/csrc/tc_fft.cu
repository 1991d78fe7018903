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
// The transforms are mixed-radix (4, 2, 3) Stockham passes in shared memory with twiddles
// from a long-double table.
#include "tc_internal.cuh"
#include "tc_fft_core.cuh"

namespace tc {

// ---------------------------------------------------------------- inverse z-pass
// Field f of H1: f = 3 d + c, c in {+, -, z}, d in {u, d_r u, d_z u}.
template <typename V>
__global__ void __launch_bounds__(256) k_zinv(const double2* __restrict__ u, V* __restrict__ H1,
                                              const double* __restrict__ w1, const int* __restrict__ col0,
                                              int N_r, int M, int K, double kz, int L, int mean_sub,
                                              const V* __restrict__ tw, Radices rad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Pz = rad.n;
    V* a = reinterpret_cast<V*>(smem_raw);
    V* b = a + (size_t)L * Pz;
    const int groups = 9 / L;
    const int g = blockIdx.x % groups;
    const int rm = blockIdx.x / groups;
    const int r = rm % N_r;        // r fastest: blocks sharing stencil rows run together
    const int m = rm / N_r;
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    const size_t colstride = (size_t)(M + 1) * nk;
    const int c0 = col0[r];
    for (int idx = threadIdx.x; idx < L * Pz; idx += blockDim.x) {
        const int l = idx / Pz;
        const int q = idx - l * Pz;
        const int k = q <= K ? q : q - Pz;
        V val;
        val.x = 0; val.y = 0;
        if (k >= -K && k <= K) {
            const int f = g * L + l;
            const int c = f % 3, d = f / 3;
            const double2* base = u + (size_t)c * S + (size_t)m * nk + (k + K);
            // mixed form: u' = u - U e_theta, i.e. on the (0,0) mode Im u'_+ = Im u'_- =
            // (Im u_+ + Im u_-) / 2 (U = Im(u_+ - u_-) / 2)
            const bool sub = mean_sub && m == 0 && k == 0 && c < 2;
            const double2* other = u + (size_t)(1 - c) * S + (size_t)m * nk + (k + K);
            double2 x;
            if (d == 1) {
                x = make_double2(0.0, 0.0);
#pragma unroll
                for (int t = 0; t < kStencil; ++t) {
                    const double w = __ldg(&w1[r * kStencil + t]);
                    double2 y = __ldg(&base[(size_t)(c0 + t) * colstride]);
                    if (sub) y.y = 0.5 * (y.y + __ldg(&other[(size_t)(c0 + t) * colstride]).y);
                    x.x += w * y.x;
                    x.y += w * y.y;
                }
            } else {
                x = __ldg(&base[(size_t)r * colstride]);
                if (sub) x.y = 0.5 * (x.y + __ldg(&other[(size_t)r * colstride]).y);
                if (d == 2) {
                    const double kk = kz * k;
                    x = make_double2(-kk * x.y, kk * x.x);
                }
            }
            val = from_d2<V>(x);
        }
        a[idx] = val;
    }
    __syncthreads();
    V* res = smem_fft(a, b, L, tw, true, rad);
    for (int idx = threadIdx.x; idx < L * Pz; idx += blockDim.x) {
        const int l = idx / Pz;
        const int z = idx - l * Pz;
        const int f = g * L + l;
        H1[(((size_t)f * N_r + r) * (M + 1) + m) * Pz + z] = res[idx];
    }
}

// ---------------------------------------------------------------- theta pass + products
// Line p of a z value (6 per z):  0 (u_r, u_t)  1 (d_r u_r, d_r u_t)  2 (d_t u_r, d_t u_t)
//                                 3 (d_z u_r, d_z u_t)  4 (u_z, d_r u_z)  5 (d_t u_z, d_z u_z)
template <typename V>
__global__ void __launch_bounds__(256) k_theta(const V* __restrict__ H1, V* __restrict__ H2,
                                               const double* __restrict__ rnodes, int N_r, int M,
                                               int Pz, double mp, int zt,
                                               const V* __restrict__ tw, Radices rad) {
    using T = typename Real<V>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Pt = rad.n;
    const int nl = 6 * zt;
    V* a = reinterpret_cast<V*>(smem_raw);
    V* b = a + (size_t)nl * Pt;
    const int tiles = Pz / zt;
    const int r = blockIdx.x / tiles;
    const int z0 = (blockIdx.x % tiles) * zt;
    const size_t fstride = (size_t)N_r * (M + 1) * Pz;
    const V* h = H1 + (size_t)r * (M + 1) * Pz + z0;

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
            if (pr == 4) { X = h[2 * fstride + o]; Y = h[5 * fstride + o]; }
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
    const T rr = (T)rnodes[r];
    const T ir = (T)(1.0 / rnodes[r]);
    for (int idx = threadIdx.x; idx < zt * Pt; idx += blockDim.x) {
        const int zi = idx / Pt;
        const int th = idx - zi * Pt;
        const V* L0 = phys + (size_t)(zi * 6) * Pt + th;
        const V p0 = L0[0], p1 = L0[Pt], p2 = L0[2 * Pt], p3 = L0[3 * Pt], p4 = L0[4 * Pt], p5 = L0[5 * Pt];
        const T ur = p0.x, ut = p0.y, uz = p4.x;
        const T utr = ut * ir;
        const T Nr = ur * p1.x + utr * p2.x + uz * p3.x - ut * utr;
        const T Nt = ur * p1.y + utr * p2.y + uz * p3.y + utr * ur;
        const T Nz = ur * p4.y + utr * p5.x + uz * p5.y;
        V q; q.x = Nr; q.y = Nt;
        fw[(size_t)zi * Pt + th] = q;
        V* zl = fw + (size_t)(zt + zi / 2) * Pt + th;
        if (zi & 1) zl->y = Nz;
        else { zl->x = Nz; if (zi + 1 == zt) zl->y = 0; }
    }
    (void)rr;
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
// With mean_add (mixed form) the FP64 mode-diagonal terms of the base flow U(r) e_theta,
// U = Re u_theta^{(0,0)}, are added to the transformed N(u'):
//   N_pm += (U/r) i m m_p u'_pm + i (U/r)(u'_+ - u'_-) +- (i/2)(d_r U + U/r)(u'_+ + u'_-),
//   N_z  += (U/r) i m m_p u'_z,   and -U^2/r on the (0,0) mode of N_pm
// (Eq. NS_cyl with u_theta = U + u'_theta; d_r U by the same FD stencil).
template <typename V>
__global__ void __launch_bounds__(256) k_zfwd(const V* __restrict__ H2, double2* __restrict__ N,
                                              int N_r, int M, int K, double scale,
                                              const V* __restrict__ tw, Radices rad,
                                              const double2* __restrict__ u, const double* __restrict__ rnodes,
                                              const double* __restrict__ w1, const int* __restrict__ col0,
                                              double mp, int mean_add, int Lf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double s_mf[2];
    const int Pz = rad.n;
    V* a = reinterpret_cast<V*>(smem_raw);
    V* b = a + (size_t)Lf * Pz;
    const int cg = blockIdx.x % (3 / Lf);     // component group (Lf = 3: all three)
    const int m = (blockIdx.x / (3 / Lf)) % (M + 1);
    const int r = (blockIdx.x / (3 / Lf)) / (M + 1);
    const size_t fstride = (size_t)N_r * (M + 1) * Pz;
    const V* h = H2 + ((size_t)r * (M + 1) + m) * Pz;
    const int nk = 2 * K + 1;
    const size_t S = (size_t)N_r * (M + 1) * nk;
    for (int idx = threadIdx.x; idx < Lf * Pz; idx += blockDim.x) {
        const int l = idx / Pz;
        const int z = idx - l * Pz;
        a[idx] = h[(cg * Lf + l) * fstride + z];
    }
    if (mean_add && threadIdx.x == 0) {
        // U(r)/r and d_r U(r) from the (0,0) column, U = Im(u_+ - u_-)/2
        const size_t col = (size_t)(M + 1) * nk;
        const double2* up = u + K;
        const double2* um = u + S + K;
        double dU = 0.0;
        const int c0 = col0[r];
        for (int t = 0; t < kStencil; ++t)
            dU += w1[r * kStencil + t] * 0.5 * (up[(size_t)(c0 + t) * col].y - um[(size_t)(c0 + t) * col].y);
        const double U = 0.5 * (up[(size_t)r * col].y - um[(size_t)r * col].y);
        s_mf[0] = U / rnodes[r];
        s_mf[1] = dU;
    }
    __syncthreads();
    V* res = smem_fft(a, b, Lf, tw, false, rad);
    double Ur = 0.0, q = 0.0;
    if (mean_add) {
        Ur = s_mf[0];
        q = 0.5 * (s_mf[1] + Ur);
    }
    for (int idx = threadIdx.x; idx < Lf * nk; idx += blockDim.x) {
        const int l = idx / nk;
        const int c = cg * Lf + l;
        const int kk = idx - l * nk;
        const int k = kk - K;
        const V v = res[(size_t)l * Pz + (k < 0 ? k + Pz : k)];
        double2 o = make_double2((double)v.x * scale, (double)v.y * scale);
        if (mean_add) {
            const size_t e = ((size_t)r * (M + 1) + m) * nk + kk;
            const double t = Ur * mp * m;
            if (c == 2) {
                const double2 z = u[2 * S + e];
                o.x -= t * z.y;
                o.y += t * z.x;
            } else {
                double2 ap = u[e], am = u[S + e];
                if (m == 0 && k == 0) {  // u'_pm on the (0,0) mode
                    const double im = 0.5 * (ap.y + am.y);
                    ap.y = im;
                    am.y = im;
                    const double U = Ur * rnodes[r];
                    o.x -= Ur * U;
                }
                const double2 own = c == 0 ? ap : am;
                const double sg = c == 0 ? 1.0 : -1.0;
                const double dx = ap.x - am.x, dy = ap.y - am.y;   // u'_+ - u'_-
                const double sx = ap.x + am.x, sy = ap.y + am.y;   // u'_+ + u'_-
                o.x += -t * own.y - Ur * dy - sg * q * sy;
                o.y += t * own.x + Ur * dx + sg * q * sx;
            }
        }
        N[(size_t)c * S + ((size_t)r * (M + 1) + m) * nk + kk] = o;
    }
}

template <typename V>
static tc_status run_nonlinear(tc_plan* p, const double2* u, double2* N, char* ws, cudaStream_t s,
                               const V* twz, const V* twt) {
    const bool mixed = sizeof(V) == 8;
    V* H1 = reinterpret_cast<V*>(ws + p->ws.H1);
    V* H2 = reinterpret_cast<V*>(ws + p->ws.H2);
    const int L = mixed ? p->zinv_lines32 : p->zinv_lines;
    const int zt = mixed ? p->zt32 : p->zt;
    size_t sm1 = (size_t)2 * L * p->P_z * sizeof(V);
    size_t sm2 = (size_t)2 * 6 * zt * p->P_t * sizeof(V);
    const int Lf = mixed ? p->zfwd_lines32 : p->zfwd_lines;
    size_t sm3 = (size_t)2 * Lf * p->P_z * sizeof(V);
    TC_CUDA(p, cudaFuncSetAttribute(k_zinv<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
    TC_CUDA(p, cudaFuncSetAttribute(k_theta<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
    TC_CUDA(p, cudaFuncSetAttribute(k_zfwd<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
    const int blocks1 = p->N_r * (p->M + 1) * (9 / L);
    int slot = prof_begin(p, sizeof(V) == 16 ? kKZinv : kKZinv32, s);
    k_zinv<V><<<blocks1, mixed ? 256 : p->thr_zinv, sm1, s>>>(u, H1, p->d_w1, p->d_col0, p->N_r, p->M, p->K, p->k_z, L, mixed ? 1 : 0, twz, p->rad_z);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_zinv");
    const int blocks2 = p->N_r * (p->P_z / zt);
    slot = prof_begin(p, sizeof(V) == 16 ? kKTheta : kKTheta32, s);
    k_theta<V><<<blocks2, mixed ? 256 : p->thr_theta, sm2, s>>>(H1, H2, p->d_r, p->N_r, p->M, p->P_z, (double)p->m_p, zt, twt, p->rad_t);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_theta");
    const double scale = 1.0 / ((double)p->P_t * (double)p->P_z);
    slot = prof_begin(p, sizeof(V) == 16 ? kKZfwd : kKZfwd32, s);
    k_zfwd<V><<<p->N_r * (p->M + 1) * (3 / Lf), mixed ? 256 : p->thr_zfwd, sm3, s>>>(H2, N, p->N_r, p->M, p->K, scale, twz, p->rad_z,
                                                     u, p->d_r, p->d_w1, p->d_col0, (double)p->m_p, mixed ? 1 : 0, Lf);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_zfwd");
    return TC_OK;
}

tc_status launch_zinv_fp64(tc_plan* p, const double2* u, double2* H1, cudaStream_t s) {
    const int L = p->zinv_lines;
    const size_t sm1 = (size_t)2 * L * p->P_z * sizeof(double2);
    TC_CUDA(p, cudaFuncSetAttribute(k_zinv<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
    const int slot = prof_begin(p, kKZinv, s);
    k_zinv<double2><<<p->N_r * (p->M + 1) * (9 / L), p->thr_zinv, sm1, s>>>(u, H1, p->d_w1, p->d_col0, p->N_r, p->M, p->K,
                                                                     p->k_z, L, 0, p->d_tw_z, p->rad_z);
    prof_end(p, slot, s);
    TC_LAUNCHED(p, "k_zinv");
    return TC_OK;
}

tc_status launch_nonlinear(tc_plan* p, const double2* u, double2* N, char* ws, cudaStream_t s) {
    if (p->precision == TC_MIXED) return run_nonlinear<float2>(p, u, N, ws, s, p->d_tw_z32, p->d_tw_t32);
    return run_nonlinear<double2>(p, u, N, ws, s, p->d_tw_z, p->d_tw_t);
}

}  // namespace tc
