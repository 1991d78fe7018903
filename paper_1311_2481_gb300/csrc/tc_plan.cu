// Host plan of libtc: radial nodes (Eq. nodeDist), finite-difference weights (Sec. 3.1,
// Fornberg's recursion in long double), twiddle tables, and the banded LU factors with partial
// pivoting of the per-mode Poisson / Helmholtz matrices (Sec. 3.2, factored once), plus their
// two-partition form for the fused steps-2-5 kernel; argument checks shared by the entry
// points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <utility>

#include <cuda.h>

#include "tc_internal.cuh"

namespace tc {

static const long double kPiL = 3.141592653589793238462643383279502884197L;

tc_status cuda_fail(tc_plan* p, cudaError_t e, const char* where) {
    if (p) snprintf(p->err, sizeof(p->err), "%s: %s", where, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return TC_ERR_OOM;
    return TC_ERR_CUDA;
}

// The allocation that contains ptr (base, size), from cuMemGetAddressRange fetched through the
// runtime, so that the library needs no link against the driver library.  False if the query
// is unavailable or fails.
static bool alloc_range(const void* ptr, unsigned long long* base, size_t* size) {
    using Fn = CUresult (*)(CUdeviceptr*, size_t*, CUdeviceptr);
    static const Fn fn = []() -> Fn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<Fn>(f);
    }();
    if (!fn) return false;
    CUdeviceptr b = 0;
    size_t s = 0;
    if (fn(&b, &s, (CUdeviceptr)(uintptr_t)ptr) != CUDA_SUCCESS) return false;
    *base = (unsigned long long)b;
    *size = s;
    return true;
}

tc_status check_device_ptr(tc_plan* p, const void* ptr, const char* name, size_t bytes) {
    if (!ptr) {
        snprintf(p->err, sizeof(p->err), "%s is NULL", name);
        return TC_ERR_ARG;
    }
    if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0) {
        snprintf(p->err, sizeof(p->err), "%s is not 16-byte aligned", name);
        return TC_ERR_ARG;
    }
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        snprintf(p->err, sizeof(p->err), "%s: %s", name, cudaGetErrorString(e));
        return TC_ERR_ARG;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
        snprintf(p->err, sizeof(p->err), "%s is not device memory", name);
        return TC_ERR_ARG;
    }
    // the bytes from ptr must be mapped without a gap: walk the allocations that cover them
    // (contiguous mappings, as in virtual-memory pools, count as one buffer; a buffer that
    // runs into a neighbouring allocation cannot be told from one that does not)
    unsigned long long base = 0;
    size_t size = 0;
    if (bytes > 0 && alloc_range(ptr, &base, &size)) {
        const unsigned long long q = (unsigned long long)(uintptr_t)ptr, end = q + bytes;
        unsigned long long cur = base + size;
        for (int i = 0; i < 4096 && cur < end; ++i) {
            if (!alloc_range(reinterpret_cast<const void*>((uintptr_t)cur), &base, &size) || base != cur) {
                snprintf(p->err, sizeof(p->err), "%s: only %llu of the %zu bytes from this pointer are mapped", name,
                         cur - q, bytes);
                return TC_ERR_ARG;
            }
            cur = base + size;
        }
    }
    return TC_OK;
}

// Fornberg's recursion for the weights of derivatives 0..md at z on nodes x[0..n-1]
// (B. Fornberg, Math. Comp. 51 (1988) 699): c[i * (md+1) + k] is the weight of node i for
// derivative k.
static void fornberg(long double z, const long double* x, int n, int md, long double* c) {
    for (int i = 0; i < n * (md + 1); ++i) c[i] = 0.0L;
    long double c1 = 1.0L, c4 = x[0] - z;
    c[0] = 1.0L;
    for (int i = 1; i < n; ++i) {
        int mn = std::min(i, md);
        long double c2 = 1.0L, c5 = c4;
        c4 = x[i] - z;
        for (int j = 0; j < i; ++j) {
            long double c3 = x[i] - x[j];
            c2 *= c3;
            if (j == i - 1) {
                for (int k = mn; k >= 1; --k)
                    c[i * (md + 1) + k] = c1 * (k * c[(i - 1) * (md + 1) + k - 1] -
                                                c5 * c[(i - 1) * (md + 1) + k]) / c2;
                c[i * (md + 1)] = -c1 * c5 * c[(i - 1) * (md + 1)] / c2;
            }
            for (int k = mn; k >= 1; --k)
                c[j * (md + 1) + k] = (c4 * c[j * (md + 1) + k] - k * c[j * (md + 1) + k - 1]) / c3;
            c[j * (md + 1)] = c4 * c[j * (md + 1)] / c3;
        }
        c1 = c2;
    }
}

static bool factor_radices(int n, Radices& rad) {
    rad.n = n;
    rad.count = 0;
    int m = n;
    while (m % 4 == 0 && rad.count < kMaxRadix) { rad.r[rad.count++] = 4; m /= 4; }
    while (m % 2 == 0 && rad.count < kMaxRadix) { rad.r[rad.count++] = 2; m /= 2; }
    while (m % 3 == 0 && rad.count < kMaxRadix) { rad.r[rad.count++] = 3; m /= 3; }
    return m == 1 && n > 1;
}

static void twiddles(int n, std::vector<double>& tw) {
    tw.resize(2 * (size_t)n);
    for (int j = 0; j < n; ++j) {
        long double a = 2.0L * kPiL * (long double)j / (long double)n;
        tw[2 * j] = (double)cosl(a);
        tw[2 * j + 1] = (double)sinl(a);
    }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Block size for a kernel whose FP64 work is Stockham passes over `lines` transforms of
// length rad.n (plus `lines2` of a second batch): the FP64 pipe is charged per warp
// instruction, so pick the size that wastes the fewest lanes over all passes.
static int choose_threads(const Radices& rad, int lines, int lines2) {
    double best = -1.0;
    int bestT = 256;
    for (int T = 96; T <= 256; T += 32) {
        double items = 0.0, slots = 0.0;
        for (int batch = 0; batch < 2; ++batch) {
            const int L = batch ? lines2 : lines;
            if (L <= 0) continue;
            for (int q = 0; q < rad.count; ++q) {
                const double it = (double)L * rad.n / rad.r[q];
                items += it;
                slots += std::ceil(it / T) * T;
            }
        }
        const double e = items / slots;
        if (e > best + 1e-9 || (std::fabs(e - best) <= 1e-9 && T > bestT)) { best = e; bestT = T; }
    }
    return bestT;
}

// Banded LU with partial pivoting of one matrix given in row windows W[i][t] = A[i][i-kl+t],
// t in [0, 2kl+ku] (kl = ku = 4).  On return W holds the multipliers of step j in
// W[j+q][kl-q] (q = 1..kl, column j of L, LAPACK convention: not permuted by later steps)
// and row j of U in W[j][kl..2kl+ku]; piv[j] = pivot row - j.  Returns false if singular.
static bool band_lu(int n, double* W, uint8_t* piv) {
    const int kl = kKl, w = 3 * kKl + 1;
    auto at = [&](int i, int c) -> double& { return W[(size_t)i * w + (c - i + kl)]; };
    for (int j = 0; j < n; ++j) {
        int last = std::min(n - 1, j + kl);
        int p = j;
        double best = std::fabs(at(j, j));
        for (int i = j + 1; i <= last; ++i)
            if (std::fabs(at(i, j)) > best) { best = std::fabs(at(i, j)); p = i; }
        if (best == 0.0) return false;
        piv[j] = (uint8_t)(p - j);
        int cmax = std::min(n - 1, j + 2 * kl);
        if (p != j)
            for (int c = j; c <= cmax; ++c) std::swap(at(j, c), at(p, c));
        double d = at(j, j);
        for (int i = j + 1; i <= last; ++i) {
            double l = at(i, j) / d;
            at(i, j) = l;
            if (l != 0.0)
                for (int c = j + 1; c <= cmax; ++c) at(i, c) -= l * at(j, c);
        }
    }
    return true;
}

// Assemble the matrix of (set, m, ka) into row windows.
static void assemble(const tc_plan* p, int set, int m, int ka, double* W) {
    const int n = p->N_r, kl = kKl, w = 3 * kKl + 1;
    std::fill(W, W + (size_t)n * w, 0.0);
    auto at = [&](int i, int c) -> double& { return W[(size_t)i * w + (c - i + kl)]; };
    const double mm = (double)m * p->m_p, kk = (double)ka * p->k_z;
    const double c0 = 3.0 / (2.0 * p->dt);
    for (int j = 0; j < n; ++j) {
        const double* w1 = &p->w1[(size_t)j * kStencil];
        const double* w2 = &p->w2[(size_t)j * kStencil];
        const int c0l = p->col0[j];
        const double r = p->r[j], ir = 1.0 / r, ir2 = 1.0 / (r * r);
        bool wall = (j == 0 || j == n - 1);
        if (set == kSetP) {
            if (wall) {
                if (j == n - 1 && m == 0 && ka == 0) { at(j, j) = 1.0; continue; }
                for (int t = 0; t < kStencil; ++t)
                    if (w1[t] != 0.0) at(j, c0l + t) += w1[t];
                continue;
            }
            for (int t = 0; t < kStencil; ++t) {
                double v = w2[t] + ir * w1[t];
                if (v != 0.0) at(j, c0l + t) += v;
            }
            at(j, j) += -mm * mm * ir2 - kk * kk;
        } else {
            if (wall) { at(j, j) = 1.0; continue; }
            for (int t = 0; t < kStencil; ++t) {
                double v = -(w2[t] + ir * w1[t]);
                if (v != 0.0) at(j, c0l + t) += v;
            }
            double diag = c0 + mm * mm * ir2 + kk * kk;
            if (set == kSetHp) diag += ir2 + 2.0 * mm * ir2;
            if (set == kSetHm) diag += ir2 - 2.0 * mm * ir2;
            at(j, j) += diag;
        }
    }
}

static bool build_factors(tc_plan* p) {
    const int n = p->N_r, M1 = p->M + 1, K1 = p->K + 1, w = 3 * kKl + 1;
    const size_t per_set = (size_t)n * kBands * M1 * K1;
    p->fac.assign((size_t)kNumSets * per_set, 0.0);
    p->piv.assign((size_t)kNumSets * n * M1 * K1, 0);
    bool ok = true;
    unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    std::vector<char> good(nth, 1);
    for (unsigned t = 0; t < nth; ++t) {
        th.emplace_back([&, t]() {
            std::vector<double> W((size_t)n * w);
            std::vector<uint8_t> pv(n);
            for (int job = t; job < kNumSets * M1; job += nth) {
                int set = job / M1, m = job % M1;
                for (int ka = 0; ka < K1; ++ka) {
                    assemble(p, set, m, ka, W.data());
                    if (!band_lu(n, W.data(), pv.data())) { good[t] = 0; return; }
                    for (int j = 0; j < n; ++j) {
                        auto dst = [&](int q) -> double& {
                            return p->fac[(size_t)set * per_set + (((size_t)j * kBands + q) * M1 + m) * K1 + ka];
                        };
                        const double* row = &W[(size_t)j * w];
                        for (int q = 1; q <= kKl; ++q)                       // L multipliers
                            dst(q - 1) = (j + q < n) ? W[(size_t)(j + q) * w + (kKl - q)] : 0.0;
                        dst(4) = 1.0 / row[kKl];                            // 1 / U_jj
                        for (int q = 1; q <= 2 * kKl; ++q)                  // U_{j, j+q}
                            dst(4 + q) = (j + q < n) ? row[kKl + q] : 0.0;
                        p->piv[(((size_t)set * n + j) * M1 + m) * K1 + ka] = pv[j];
                    }
                }
            }
        });
    }
    for (auto& x : th) x.join();
    for (char g : good) ok = ok && g;
    return ok;
}

// Solve with the factors band_lu leaves in W (row swap and column-j elimination in the
// order of the factorisation, then back substitution), in place.
static void band_lu_solve(int n, const double* W, const uint8_t* piv, double* b) {
    const int kl = kKl, w = 3 * kKl + 1;
    auto at = [&](int i, int c) { return W[(size_t)i * w + (c - i + kl)]; };
    for (int j = 0; j < n; ++j) {
        const int pj = j + piv[j];
        if (pj != j) std::swap(b[j], b[pj]);
        for (int q = 1; q <= kl && j + q < n; ++q) b[j + q] -= at(j + q, j) * b[j];
    }
    for (int j = n - 1; j >= 0; --j) {
        double s = b[j];
        for (int q = 1; q <= 2 * kl && j + q < n; ++q) s -= at(j, j + q) * b[j + q];
        b[j] = s / at(j, j);
    }
}

// Store the factors of an n-row block whose first row is global row r0 (layout of fac).
static void store_lu(const tc_plan* p, std::vector<double>& fac, std::vector<uint8_t>& piv, int set, int m,
                     int ka, int r0, int n, const double* W, const uint8_t* pv) {
    const int N = p->N_r, M1 = p->M + 1, K1 = p->K + 1, w = 3 * kKl + 1;
    const size_t per_set = (size_t)N * kBands * M1 * K1;
    for (int i = 0; i < n; ++i) {
        const int j = r0 + i;
        auto dst = [&](int q) -> double& { return fac[(size_t)set * per_set + (((size_t)j * kBands + q) * M1 + m) * K1 + ka]; };
        const double* row = &W[(size_t)i * w];
        for (int q = 1; q <= kKl; ++q) dst(q - 1) = (i + q < n) ? W[(size_t)(i + q) * w + (kKl - q)] : 0.0;
        dst(4) = 1.0 / row[kKl];
        for (int q = 1; q <= 2 * kKl; ++q) dst(4 + q) = (i + q < n) ? row[kKl + q] : 0.0;
        piv[(((size_t)set * N + j) * M1 + m) * K1 + ka] = pv[i];
    }
}

// Two-partition (SPIKE) form of every system: A = [A1 B; C A2] cut at row h.  A1 and A2 are
// factored like A; with kl = ku = 4, B has its non-zeros in rows h-4..h-1 of columns h..h+3
// and C in rows h..h+3 of columns h-4..h-1.  The spikes V = A1^{-1} B and W = A2^{-1} C give
// x1 = g1 - V x2[0..3] and x2 = g2 - W x1[h-4..h-1] (g_i = A_i^{-1} b_i), and the eight
// interface unknowns x[h-4..h+3] solve R t = g[h-4..h+3] with R = [I V_b; W_t I] (V_b: rows
// h-4..h-1 of V, W_t: rows 0..3 of W), whose inverse is stored.  Returns false if a block or
// R is singular (the plan then keeps one partition).
static bool build_partitions(tc_plan* p, int h) {
    const int N = p->N_r, M1 = p->M + 1, K1 = p->K + 1, w = 3 * kKl + 1, n2 = N - h;
    const size_t per_set = (size_t)N * kBands * M1 * K1;
    p->fac2.assign((size_t)kNumSets * per_set, 0.0);
    p->piv2.assign((size_t)kNumSets * N * M1 * K1, 0);
    p->spk.assign((size_t)kNumSets * N * 4 * M1 * K1, 0.0);
    p->rinv.assign((size_t)kNumSets * 64 * M1 * K1, 0.0);
    unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    std::vector<char> good(nth, 1);
    for (unsigned t = 0; t < nth; ++t) {
        th.emplace_back([&, t]() {
            std::vector<double> W((size_t)N * w), W1((size_t)h * w), W2((size_t)n2 * w), col(N);
            std::vector<uint8_t> pv1(h), pv2(n2);
            double Bm[4][4], Cm[4][4];   // B[h-4+i][h+q], C[h+i][h-4+q]
            for (int job = t; job < kNumSets * M1; job += nth) {
                const int set = job / M1, m = job % M1;
                for (int ka = 0; ka < K1; ++ka) {
                    assemble(p, set, m, ka, W.data());
                    auto A = [&](int i, int c) -> double {
                        const int d = c - i + kKl;
                        return (d >= 0 && d < w) ? W[(size_t)i * w + d] : 0.0;
                    };
                    std::fill(W1.begin(), W1.end(), 0.0);
                    std::fill(W2.begin(), W2.end(), 0.0);
                    for (int i = 0; i < h; ++i)
                        for (int c = std::max(0, i - kKl); c <= std::min(h - 1, i + kKl); ++c)
                            W1[(size_t)i * w + (c - i + kKl)] = A(i, c);
                    for (int i = 0; i < n2; ++i)
                        for (int c = std::max(0, i - kKl); c <= std::min(n2 - 1, i + kKl); ++c)
                            W2[(size_t)i * w + (c - i + kKl)] = A(h + i, h + c);
                    for (int i = 0; i < 4; ++i)
                        for (int q = 0; q < 4; ++q) {
                            Bm[i][q] = A(h - 4 + i, h + q);
                            Cm[i][q] = A(h + i, h - 4 + q);
                        }
                    if (!band_lu(h, W1.data(), pv1.data()) || !band_lu(n2, W2.data(), pv2.data())) { good[t] = 0; return; }
                    store_lu(p, p->fac2, p->piv2, set, m, ka, 0, h, W1.data(), pv1.data());
                    store_lu(p, p->fac2, p->piv2, set, m, ka, h, n2, W2.data(), pv2.data());
                    long double R[8][16];
                    for (int i = 0; i < 8; ++i)
                        for (int c = 0; c < 16; ++c) R[i][c] = (c == i || c == i + 8) ? 1.0L : 0.0L;
                    auto spk = [&](int j, int q) -> double& { return p->spk[((((size_t)set * N + j) * 4 + q) * M1 + m) * K1 + ka]; };
                    for (int q = 0; q < 4; ++q) {
                        std::fill(col.begin(), col.end(), 0.0);
                        for (int i = 0; i < 4; ++i) col[h - 4 + i] = Bm[i][q];
                        band_lu_solve(h, W1.data(), pv1.data(), col.data());
                        for (int j = 0; j < h; ++j) spk(j, q) = col[j];
                        for (int i = 0; i < 4; ++i) R[i][4 + q] = col[h - 4 + i];
                        std::fill(col.begin(), col.end(), 0.0);
                        for (int i = 0; i < 4; ++i) col[i] = Cm[i][q];
                        band_lu_solve(n2, W2.data(), pv2.data(), col.data());
                        for (int i = 0; i < n2; ++i) spk(h + i, q) = col[i];
                        for (int i = 0; i < 4; ++i) R[4 + i][q] = col[i];
                    }
                    // Gauss-Jordan with partial pivoting on [R | I]
                    for (int c = 0; c < 8; ++c) {
                        int piv = c;
                        for (int i = c + 1; i < 8; ++i)
                            if (std::fabs((double)R[i][c]) > std::fabs((double)R[piv][c])) piv = i;
                        if (R[piv][c] == 0.0L) { good[t] = 0; return; }
                        if (piv != c)
                            for (int e = 0; e < 16; ++e) std::swap(R[c][e], R[piv][e]);
                        const long double d = R[c][c];
                        for (int e = 0; e < 16; ++e) R[c][e] /= d;
                        for (int i = 0; i < 8; ++i) {
                            if (i == c || R[i][c] == 0.0L) continue;
                            const long double f = R[i][c];
                            for (int e = 0; e < 16; ++e) R[i][e] -= f * R[c][e];
                        }
                    }
                    for (int i = 0; i < 8; ++i)
                        for (int l = 0; l < 8; ++l)
                            p->rinv[(((size_t)set * 64 + i * 8 + l) * M1 + m) * K1 + ka] = (double)R[i][8 + l];
                }
            }
        });
    }
    for (auto& x : th) x.join();
    for (char g : good)
        if (!g) return false;
    return true;
}

static tc_status upload(tc_plan* p) {
    TC_CUDA(p, cudaGetDevice(&p->device));
    TC_CUDA(p, cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    TC_CUDA(p, cudaHostAlloc((void**)&p->h_nonfinite, sizeof(int), cudaHostAllocMapped));
    *p->h_nonfinite = 0;
    TC_CUDA(p, cudaHostGetDevicePointer((void**)&p->d_nonfinite, p->h_nonfinite, 0));
    if (p->precision == TC_MIXED) {
        TC_CUDA(p, cudaStreamCreateWithFlags(&p->mean_stream, cudaStreamNonBlocking));
        for (cudaEvent_t& e : p->mean_ev) TC_CUDA(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    auto put = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(dst, bytes);
        if (e != cudaSuccess) return e;
        return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    TC_CUDA(p, put((void**)&p->d_r, p->r.data(), p->r.size() * sizeof(double)));
    std::vector<double> ir(p->r.size());
    for (size_t j = 0; j < ir.size(); ++j) ir[j] = 1.0 / p->r[j];
    TC_CUDA(p, put((void**)&p->d_ir, ir.data(), ir.size() * sizeof(double)));
    TC_CUDA(p, put((void**)&p->d_w1, p->w1.data(), p->w1.size() * sizeof(double)));
    std::vector<float> w1f(p->w1.begin(), p->w1.end());
    TC_CUDA(p, put((void**)&p->d_w1f, w1f.data(), w1f.size() * sizeof(float)));
    {
        // The FP32 theta lines carry u_z and d_r u_z as one complex line, so the transform's
        // rounding is relative to the larger of the two.  Near a no-slip wall u' ~ (r - r_w)
        // d_r u', so d_r u_z is scaled by 2^floor(log2 d), d the distance to the nearer wall
        // (at most 1, the gap width), which keeps both parts of the line at a similar size;
        // the scale is a power of two, so scaling and unscaling are exact.  Wall rows take
        // the scale of their neighbour (u' = 0 there).
        const int N = p->N_r;
        std::vector<float> dsc(N, 1.0f);
        for (int j = 0; j < N; ++j) {
            const int jj = j == 0 ? 1 : (j == N - 1 ? N - 2 : j);
            const double d = std::min(std::min(p->r[jj] - p->r_i, p->r_o - p->r[jj]), 1.0);
            dsc[j] = d > 0.0 ? (float)std::ldexp(1.0, (int)std::floor(std::log2(d))) : 1.0f;
        }
        TC_CUDA(p, put((void**)&p->d_dsc, dsc.data(), dsc.size() * sizeof(float)));
    }
    TC_CUDA(p, put((void**)&p->d_w2, p->w2.data(), p->w2.size() * sizeof(double)));
    TC_CUDA(p, put((void**)&p->d_col0, p->col0.data(), p->col0.size() * sizeof(int)));
    TC_CUDA(p, put((void**)&p->d_d1t_row, p->d1t_row.data(), p->d1t_row.size() * sizeof(int)));
    TC_CUDA(p, put((void**)&p->d_d1t_w, p->d1t_w.data(), p->d1t_w.size() * sizeof(double)));
    TC_CUDA(p, put((void**)&p->d_fac, p->fac.data(), p->fac.size() * sizeof(double)));
    TC_CUDA(p, put((void**)&p->d_piv, p->piv.data(), p->piv.size()));
    if (p->part_h > 0) {
        TC_CUDA(p, put((void**)&p->d_fac2, p->fac2.data(), p->fac2.size() * sizeof(double)));
        TC_CUDA(p, put((void**)&p->d_piv2, p->piv2.data(), p->piv2.size()));
        TC_CUDA(p, put((void**)&p->d_spk, p->spk.data(), p->spk.size() * sizeof(double)));
        TC_CUDA(p, put((void**)&p->d_rinv, p->rinv.data(), p->rinv.size() * sizeof(double)));
    }
    TC_CUDA(p, put((void**)&p->d_tw_z, p->tw_z.data(), p->tw_z.size() * sizeof(double)));
    TC_CUDA(p, put((void**)&p->d_tw_t, p->tw_t.data(), p->tw_t.size() * sizeof(double)));
    std::vector<float> f(p->tw_z.begin(), p->tw_z.end());
    TC_CUDA(p, put((void**)&p->d_tw_z32, f.data(), f.size() * sizeof(float)));
    f.assign(p->tw_t.begin(), p->tw_t.end());
    TC_CUDA(p, put((void**)&p->d_tw_t32, f.data(), f.size() * sizeof(float)));
    return TC_OK;
}

const char* const kKernelNames[kNumKernels] = {
    "k_zinv", "k_theta", "k_zfwd", "k_rhs_pressure", "k_band_solve_P", "k_rhs_velocity",
    "k_band_solve_H", "k_rhs_div", "k_update", "k_axpby", "k_diag", "k_zinv_f32",
    "k_theta_f32", "k_zfwd_f32", "k_pc", "k_pc_adj", "k_zinv_adjin",
    "k_theta_adj", "k_zfwd_adj", "k_drT", "k_prep_f32", "k_mean00_f32"};

int prof_begin(tc_plan* p, int kid, cudaStream_t s) {
    if (!p->prof_on) return -1;
    if (2 * (p->prof_used + 1) > p->prof_ev.size()) {
        size_t grow = std::max<size_t>(256, p->prof_ev.size());
        for (size_t i = 0; i < grow; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return -1; }
            p->prof_ev.push_back(e);
        }
    }
    int slot = (int)p->prof_used++;
    if ((size_t)slot >= p->prof_kid.size()) p->prof_kid.resize(slot + 1);
    p->prof_kid[slot] = kid;
    cudaEventRecord(p->prof_ev[2 * slot], s);
    return slot;
}

void prof_end(tc_plan* p, int slot, cudaStream_t s) {
    if (slot < 0) return;
    cudaEventRecord(p->prof_ev[2 * slot + 1], s);
}

static void free_device(tc_plan* p) {
    for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
    p->prof_ev.clear();
    for (cudaEvent_t& e : p->copy_ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    if (p->copy_stream) {
        cudaStreamDestroy(p->copy_stream);
        p->copy_stream = nullptr;
    }
    for (cudaEvent_t& e : p->mean_ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    if (p->mean_stream) {
        cudaStreamDestroy(p->mean_stream);
        p->mean_stream = nullptr;
    }
    void* ptrs[] = {p->d_r, p->d_ir, p->d_w1, p->d_w1f, p->d_dsc, p->d_w2, p->d_col0, p->d_d1t_row, p->d_d1t_w, p->d_fac, p->d_piv,
                    p->d_fac2, p->d_piv2, p->d_spk, p->d_rinv, p->d_tw_z, p->d_tw_t, p->d_tw_z32, p->d_tw_t32};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (p->h_nonfinite) cudaFreeHost(p->h_nonfinite);
    p->h_nonfinite = p->d_nonfinite = nullptr;
}

}  // namespace tc

using namespace tc;

extern "C" {

const char* tc_status_string(tc_status s) {
    switch (s) {
        case TC_OK: return "ok";
        case TC_ERR_ARG: return "invalid argument";
        case TC_ERR_CUDA: return "CUDA error";
        case TC_ERR_OOM: return "out of memory";
        case TC_ERR_NONFINITE: return "non-finite value in state";
        case TC_ERR_TIMEOUT: return "device wait timed out";
        case TC_ERR_STATE: return "call not allowed in this plan state";
    }
    return "unknown status";
}

const char* tc_plan_last_error(const tc_plan* plan) { return plan ? plan->err : "no plan"; }

tc_status tc_plan_create_ex(tc_plan** out, int N_r, int M, int K, int m_p, double eta,
                            double Re_i, double Re_o, double L_z, double dt, int fd_order,
                            const tc_options* opt) {
    if (!out) return TC_ERR_ARG;
    *out = nullptr;
    tc_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (fd_order < 2 || fd_order > 8 || fd_order % 2) return TC_ERR_ARG;
    if (N_r < fd_order + 1 || N_r > 2048 || M < 1 || K < 1 || m_p < 1) return TC_ERR_ARG;
    if (!(eta > 0.0 && eta < 1.0) || !(L_z > 0.0) || !(dt > 0.0)) return TC_ERR_ARG;
    if (!std::isfinite(Re_i) || !std::isfinite(Re_o) || !std::isfinite(L_z) || !std::isfinite(dt))
        return TC_ERR_ARG;
    if (o.precision != TC_FP64 && o.precision != TC_MIXED) return TC_ERR_ARG;
    double alpha = o.alpha == 0.0 ? 0.5 : (o.alpha < 0.0 ? 0.0 : o.alpha);
    if (alpha > 1.0) return TC_ERR_ARG;
    int Pt = o.P_theta ? o.P_theta : 3 * M;
    int Pz = o.P_z ? o.P_z : 3 * K;
    Radices rz, rt;
    if (Pt < 2 * M + 1 || Pz < 2 * K + 1 || !factor_radices(Pz, rz) || !factor_radices(Pt, rt))
        return TC_ERR_ARG;
    if ((size_t)N_r * (M + 1) * (size_t)(2 * K + 1) > ((size_t)1 << 40)) return TC_ERR_ARG;

    tc_plan* p = new (std::nothrow) tc_plan();
    if (!p) return TC_ERR_OOM;
    p->err[0] = 0;
    p->N_r = N_r; p->M = M; p->K = K; p->m_p = m_p; p->fd_order = fd_order; p->half = fd_order / 2;
    p->P_t = Pt; p->P_z = Pz; p->precision = o.precision;
    p->eta = eta; p->Re_i = Re_i; p->Re_o = Re_o; p->L_z = L_z; p->dt = dt; p->alpha = alpha;
    p->k_z = (double)(2.0L * kPiL / (long double)L_z);
    p->r_i = eta / (1.0 - eta);
    p->r_o = 1.0 / (1.0 - eta);
    p->host_only = o.host_only != 0;
    p->opt = o;
    p->rad_z = rz;
    p->rad_t = rt;
    p->S = (size_t)N_r * (M + 1) * (2 * K + 1);
    p->Hfield = (size_t)N_r * (M + 1) * Pz;
    p->nmode = (M + 1) * (2 * K + 1);
    p->nmode_half = (M + 1) * (K + 1);

    // nodes, Eq. nodeDist with paper-M = N_r - 1, in long double
    p->r.resize(N_r);
    std::vector<long double> rl(N_r);
    long double etal = eta, centre = (1.0L + etal) / (2.0L * (1.0L - etal));
    for (int j = 0; j < N_r; ++j) {
        long double c = cosl(kPiL * (long double)j / (long double)(N_r - 1));
        long double s = alpha == 0.0 ? -c / 2.0L
                                     : asinl(-(long double)alpha * c) / (2.0L * asinl((long double)alpha));
        rl[j] = centre + s;
        p->r[j] = (double)rl[j];
    }
    // FD weights, padded to 9 entries starting at col0
    const int half = p->half;
    p->w1.assign((size_t)N_r * kStencil, 0.0);
    p->w2.assign((size_t)N_r * kStencil, 0.0);
    p->col0.resize(N_r);
    for (int j = 0; j < N_r; ++j) {
        int lo, hi;
        if (j == 0) { lo = 0; hi = half; }
        else if (j == N_r - 1) { lo = N_r - 1 - half; hi = N_r - 1; }
        else { int h = std::min(std::min(j, N_r - 1 - j), half); lo = j - h; hi = j + h; }
        int c0 = std::min(std::max(j - kStencil / 2, 0), N_r - kStencil);
        p->col0[j] = c0;
        int n = hi - lo + 1;
        long double c[kStencil * 3];
        fornberg(rl[j], &rl[lo], n, 2, c);
        for (int i = 0; i < n; ++i) {
            p->w1[(size_t)j * kStencil + (lo + i - c0)] = (double)c[i * 3 + 1];
            p->w2[(size_t)j * kStencil + (lo + i - c0)] = n >= 3 ? (double)c[i * 3 + 2] : 0.0;
        }
    }
    // transposed D1 as a gather table: column c collects w1[j][c - col0[j]] from rows j
    {
        std::vector<std::vector<std::pair<int, double>>> cols(N_r);
        for (int j = 0; j < N_r; ++j)
            for (int t = 0; t < kStencil; ++t) {
                double w = p->w1[(size_t)j * kStencil + t];
                if (w != 0.0) cols[p->col0[j] + t].push_back({j, w});
            }
        int n = 1;
        for (auto& c : cols) n = std::max<int>(n, (int)c.size());
        p->d1t_n = n;
        p->d1t_row.assign((size_t)N_r * n, 0);
        p->d1t_w.assign((size_t)N_r * n, 0.0);
        for (int c = 0; c < N_r; ++c)
            for (size_t e = 0; e < cols[c].size(); ++e) {
                p->d1t_row[(size_t)c * n + e] = cols[c][e].first;
                p->d1t_w[(size_t)c * n + e] = cols[c][e].second;
            }
    }
    twiddles(Pz, p->tw_z);
    twiddles(Pt, p->tw_t);
    if (!build_factors(p)) {
        delete p;
        return TC_ERR_ARG;  // a singular mode matrix (parameters out of range)
    }
    // launch geometry and workspace
    const size_t cplx = sizeof(double2);
    // lines per z-pass block: several blocks per SM (<= 76 KB of shared memory each)
    auto lines_for = [&](size_t esz, int Lmax) {
        int L = Lmax;
        while (L > 1 && (size_t)2 * L * Pz * esz > 76 * 1024) L = L == 9 ? 3 : 1;
        return L;
    };
    // z values per theta block: at most `cap` bytes of shared memory, so that several blocks
    // share an SM (the FP32 lines are latency-bound; three 76 KB blocks fit an SM)
    auto zt_for = [&](size_t esz, int zmax, size_t cap) {
        int zt = zmax;
        while (zt > 1 && (size_t)2 * 6 * zt * Pt * esz > cap) zt /= 2;
        while (zt > 1 && Pz % zt) zt /= 2;
        return zt;
    };
    p->zinv_lines = lines_for(sizeof(double2), 9);
    p->zinv_lines32 = lines_for(sizeof(float2), 9);
    p->zfwd_lines = lines_for(sizeof(double2), 3);
    p->zfwd_lines32 = lines_for(sizeof(float2), 3);
    p->zt = zt_for(sizeof(double2), o.theta_zt > 0 ? o.theta_zt : 4, 200 * 1024);
    p->zt32 = zt_for(sizeof(float2), o.theta_zt > 0 ? o.theta_zt : 8, o.theta_zt > 0 ? 200 * 1024 : 76 * 1024);
    p->pc_modes = o.pc_modes;
    p->theta_zt_forced = o.theta_zt;
    p->theta_variant = o.theta_variant;
    p->thr_zinv = choose_threads(rz, p->zinv_lines, 0);
    p->thr_theta = choose_threads(rt, 6 * p->zt, p->zt + (p->zt + 1) / 2);
    p->thr_zfwd = choose_threads(rz, p->zfwd_lines, 0);
    if (o.theta_zt < 0 || o.theta_zt > 64 || o.pc_modes < 0 || o.pc_modes > 32 || o.pc_split < -1 || o.pc_split > 1 ||
        o.theta_variant < 0 || o.theta_variant > 4 || o.pc_partitions < 0 || o.pc_partitions > 2 ||
        o.stage_rows < 0 || o.mean_fp32 < 0 || o.mean_fp32 > 1) {
        delete p;
        return TC_ERR_ARG;
    }
    {
        // FP64 lines unless the plan is mixed without the (FP64) adjoint
        const size_t lb = (o.precision == TC_MIXED && o.no_adjoint) ? sizeof(float2) : cplx;
        if ((size_t)2 * 3 * Pz * lb > 220 * 1024 || (size_t)2 * 6 * Pt * lb > 220 * 1024) {
            delete p;
            return TC_ERR_ARG;   // transform lines too long for one block's shared memory
        }
    }
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o2 = off; off = align256(off + bytes); return o2; };
    p->adjoint = o.no_adjoint == 0;
    // FP64 staging rows per slab: the FP64 forward lines (12 line sets) and the adjoint's
    // (21 line sets and the Rhat rows) of stage_rows rows
    {
        const size_t hrow = (size_t)(M + 1) * Pz * cplx;
        size_t per_row = p->precision == TC_MIXED ? 0 : 12 * hrow;
        if (p->adjoint) per_row = std::max(per_row, 21 * hrow + 3 * (size_t)p->nmode * cplx);
        const size_t cap = (size_t)4 << 30;
        int rows = N_r;
        if (o.stage_rows > 0) rows = std::min(o.stage_rows, N_r);
        else if (per_row * (size_t)N_r > cap) rows = (int)std::max<size_t>(1, cap / std::max<size_t>(per_row, 1));
        p->stage_rows = rows;
    }
    // forward transform staging: FP64 lines of stage_rows rows, or the mixed form's FP32
    // lines of all rows and its FP32 u', d_r u'
    if (p->precision == TC_MIXED) {
        p->ws.H1 = take(9 * p->Hfield * sizeof(float2));
        p->ws.H2 = take(3 * p->Hfield * sizeof(float2));
        p->ws.P32 = take(6 * p->S * sizeof(float2));
        p->ws.mean = take(mean00_part_doubles(p) * sizeof(double));
    } else {
        const size_t hst = (size_t)p->stage_rows * (M + 1) * Pz;
        p->ws.H1 = take(9 * hst * cplx);
        p->ws.H2 = take(3 * hst * cplx);
        p->ws.P32 = take(0);
        p->ws.mean = take(0);
    }
    const size_t fwd_staging = off;
    p->ws.Ncur = take(3 * p->S * cplx);
    p->ws.uE = take(3 * p->S * cplx);
    // steps 2-5: fused kernel while 8 modes' four columns fit in 96 KB of shared memory,
    // split kernels beyond (tc_options.pc_split forces either)
    p->pc_split = o.pc_split == 1 || (o.pc_split == 0 && (size_t)4 * N_r * 8 * cplx > 96 * 1024);
    // two partitions per system in the fused kernel (a singular diagonal block or reduced
    // matrix keeps one)
    if (!p->pc_split && o.pc_partitions != 1 && N_r >= 16)
        p->part_h = build_partitions(p, N_r / 2) ? N_r / 2 : 0;
    if (p->part_h == 0) {
        std::vector<double>().swap(p->fac2);
        std::vector<double>().swap(p->spk);
        std::vector<double>().swap(p->rinv);
        std::vector<uint8_t>().swap(p->piv2);
    }
    p->ws.red = take(diag_red_doubles(p) * sizeof(double));
    // The split steps-2-5 buffers (scratch of a forward or adjoint advance) and the
    // transposed nonlinear term's staging (which runs after the advance of its call) share
    // one region.
    const size_t shared0 = off;
    if (p->pc_split) {
        p->ws.pstar = take(p->S * cplx);
        p->ws.ustar = take(3 * p->S * cplx);
        p->ws.phi = take(p->S * cplx);
    }
    const size_t split_end = off;
    if (p->adjoint) {
        off = shared0;
        const size_t hst = (size_t)p->stage_rows * (M + 1) * Pz;
        p->ws.H1a = take(9 * hst * cplx);
        p->ws.Ha = take(3 * hst * cplx);
        p->ws.H3 = take(9 * hst * cplx);
        p->ws.Rhat = take(3 * (size_t)p->stage_rows * p->nmode * cplx);
        off = std::max(off, split_end);
        p->ws.Nbar = take(3 * p->S * cplx);   // written by the adjoint advance
        // tc_adjoint_start's temporaries live from u^{-1} = 2.5 u0 - 1.5 u_E on, after its one
        // forward nonlinear evaluation: they take the forward staging when it is large enough
        p->ws.abar = fwd_staging >= 9 * p->S * cplx ? 0 : take(9 * p->S * cplx);
    }
    p->ws.total = off;
    if (!p->host_only) {
        tc_status st = upload(p);
        if (st != TC_OK) {
            free_device(p);
            delete p;
            return st;
        }
        // the device holds the factors now; release the host copy (tens of GB at N_r = 384)
        std::vector<double>().swap(p->fac);
        std::vector<uint8_t>().swap(p->piv);
        std::vector<double>().swap(p->fac2);
        std::vector<double>().swap(p->spk);
        std::vector<double>().swap(p->rinv);
        std::vector<uint8_t>().swap(p->piv2);
    }
    *out = p;
    return TC_OK;
}

tc_status tc_plan_create(tc_plan** out, int N_r, int M, int K, int m_p, double eta, double Re_i,
                         double Re_o, double L_z, double dt, int fd_order) {
    return tc_plan_create_ex(out, N_r, M, K, m_p, eta, Re_i, Re_o, L_z, dt, fd_order, nullptr);
}

tc_status tc_plan_set(tc_plan* plan, int key, double value) {
    if (!plan) return TC_ERR_ARG;
    if (plan->used) {
        snprintf(plan->err, sizeof(plan->err), "tc_plan_set after the plan's first compute call");
        return TC_ERR_STATE;
    }
    if (!plan->host_only) {
        int dev = -1;
        TC_CUDA(plan, cudaGetDevice(&dev));
        if (dev != plan->device) {
            snprintf(plan->err, sizeof(plan->err), "tc_plan_set: current device %d is not the plan's device %d",
                     dev, plan->device);
            return TC_ERR_STATE;
        }
    }
    tc_options o = plan->opt;
    if (key == TC_SET_ALPHA) {
        if (!std::isfinite(value)) return TC_ERR_ARG;
        o.alpha = value;
    } else {
        // every other setting is an integer
        if (!(value >= -1e9 && value <= 1e9) || value != std::floor(value)) return TC_ERR_ARG;
        const int v = (int)value;
        switch (key) {
            case TC_SET_P_THETA: o.P_theta = v; break;
            case TC_SET_P_Z: o.P_z = v; break;
            case TC_SET_PRECISION: o.precision = v; break;
            case TC_SET_HOST_ONLY: o.host_only = v; break;
            case TC_SET_THETA_ZT: o.theta_zt = v; break;
            case TC_SET_PC_MODES: o.pc_modes = v; break;
            case TC_SET_NO_ADJOINT: o.no_adjoint = v; break;
            case TC_SET_PC_SPLIT: o.pc_split = v; break;
            case TC_SET_THETA_VARIANT: o.theta_variant = v; break;
            case TC_SET_PC_PARTITIONS: o.pc_partitions = v; break;
            case TC_SET_STAGE_ROWS: o.stage_rows = v; break;
            case TC_SET_MEAN_FP32: o.mean_fp32 = v; break;
            default: return TC_ERR_ARG;
        }
    }
    // build the replacement completely before touching the plan, so an error leaves it as it was
    tc_plan* np = nullptr;
    tc_status st = tc_plan_create_ex(&np, plan->N_r, plan->M, plan->K, plan->m_p, plan->eta, plan->Re_i,
                                     plan->Re_o, plan->L_z, plan->dt, plan->fd_order, &o);
    if (st != TC_OK) {
        snprintf(plan->err, sizeof(plan->err), "tc_plan_set: rebuilding the plan failed (status %d)", (int)st);
        return st;
    }
    free_device(plan);
    *plan = std::move(*np);   // device pointers move with it; np's destructor frees host vectors only
    delete np;
    return TC_OK;
}

void tc_plan_destroy(tc_plan* plan) {
    if (!plan) return;
    free_device(plan);
    delete plan;
}

tc_status tc_plan_workspace_bytes(const tc_plan* plan, size_t* bytes) {
    if (!plan || !bytes) return TC_ERR_ARG;
    *bytes = plan->ws.total;
    return TC_OK;
}

tc_status tc_plan_nodes(const tc_plan* plan, double* r_host) {
    if (!plan || !r_host) return TC_ERR_ARG;
    memcpy(r_host, plan->r.data(), plan->r.size() * sizeof(double));
    return TC_OK;
}

tc_status tc_profile_enable(tc_plan* plan, int enable) {
    if (!plan) return TC_ERR_ARG;
    if (plan->host_only) return TC_ERR_STATE;
    plan->prof_on = enable != 0;
    plan->prof_used = 0;
    return TC_OK;
}

tc_status tc_profile_read(tc_plan* plan, int index, const char** name, long long* launches,
                          double* total_ms) {
    if (!plan || index < 0 || index >= kNumKernels) return TC_ERR_ARG;
    if (plan->host_only) return TC_ERR_STATE;
    long long n = 0;
    double ms = 0.0;
    for (size_t i = 0; i < plan->prof_used; ++i) {
        if (plan->prof_kid[i] != index) continue;
        TC_CUDA(plan, cudaEventSynchronize(plan->prof_ev[2 * i + 1]));
        float t = 0.0f;
        TC_CUDA(plan, cudaEventElapsedTime(&t, plan->prof_ev[2 * i], plan->prof_ev[2 * i + 1]));
        ms += t;
        ++n;
    }
    if (name) *name = kKernelNames[index];
    if (launches) *launches = n;
    if (total_ms) *total_ms = ms;
    return TC_OK;
}

tc_status tc_plan_fd_weights(const tc_plan* plan, int deriv, double* w_host, int* col0_host) {
    if (!plan || !w_host || (deriv != 1 && deriv != 2)) return TC_ERR_ARG;
    const std::vector<double>& w = deriv == 1 ? plan->w1 : plan->w2;
    memcpy(w_host, w.data(), w.size() * sizeof(double));
    if (col0_host) memcpy(col0_host, plan->col0.data(), plan->col0.size() * sizeof(int));
    return TC_OK;
}

tc_status tc_plan_solve_host(const tc_plan* plan, int which, int m, int ka, int partitions, const double* b,
                             double* x) {
    if (!plan || !b || !x || which < TC_P_STAR || which > TC_PHI || m < 0 || m > plan->M || ka < 0 ||
        ka > plan->K || (partitions != 1 && partitions != 2))
        return TC_ERR_ARG;
    if (!plan->host_only || (partitions == 2 && plan->part_h == 0)) return TC_ERR_STATE;
    const int N = plan->N_r, M1 = plan->M + 1, K1 = plan->K + 1;
    const int set = which == TC_PHI ? kSetP : which;
    const size_t per_set = (size_t)N * kBands * M1 * K1;
    const std::vector<double>& fac = partitions == 2 ? plan->fac2 : plan->fac;
    const std::vector<uint8_t>& piv = partitions == 2 ? plan->piv2 : plan->piv;
    auto F = [&](int j, int q) { return fac[(size_t)set * per_set + (((size_t)j * kBands + q) * M1 + m) * K1 + ka]; };
    auto Pv = [&](int j) { return (int)piv[(((size_t)set * N + j) * M1 + m) * K1 + ka]; };
    for (int j = 0; j < N; ++j) x[j] = b[j];
    // rows [r0, r0 + n) with the stored factors, in the order the device substitution uses
    auto solve_rows = [&](int r0, int n) {
        for (int i = 0; i < n; ++i) {
            const int j = r0 + i, pj = j + Pv(j);
            if (pj != j) std::swap(x[j], x[pj]);
            for (int q = 1; q <= kKl && i + q < n; ++q) x[j + q] -= F(j, q - 1) * x[j];
        }
        for (int i = n - 1; i >= 0; --i) {
            const int j = r0 + i;
            double s = x[j];
            for (int q = 2 * kKl; q >= 1; --q)
                if (i + q < n) s -= F(j, 4 + q) * x[j + q];
            x[j] = s * F(j, 4);
        }
    };
    if (partitions == 1) {
        solve_rows(0, N);
        return TC_OK;
    }
    const int h = plan->part_h;
    solve_rows(0, h);
    solve_rows(h, N - h);
    double t[8];
    for (int i = 0; i < 8; ++i) {
        double acc = 0.0;
        for (int l = 0; l < 8; ++l) acc += plan->rinv[(((size_t)set * 64 + i * 8 + l) * M1 + m) * K1 + ka] * x[h - 4 + l];
        t[i] = acc;
    }
    for (int j = 0; j < N; ++j)
        for (int q = 0; q < 4; ++q)
            x[j] -= plan->spk[((((size_t)set * N + j) * 4 + q) * M1 + m) * K1 + ka] * (j < h ? t[4 + q] : t[q]);
    return TC_OK;
}

}  // extern "C"
