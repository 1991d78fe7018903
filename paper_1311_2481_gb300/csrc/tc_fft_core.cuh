// Shared-memory mixed-radix (4, 2, 3) Stockham transforms used by the forward and adjoint
// nonlinear-term kernels.  Twiddles come from a long-double table exp(+2 pi i j / n).
#pragma once

#include "tc_internal.cuh"

namespace tc {

template <typename V> struct Real;
template <> struct Real<double2> { using type = double; };
template <> struct Real<float2> { using type = float; };

// small DFTs of the Stockham passes; inv selects exp(+2 pi i / R)
template <typename V>
__device__ __forceinline__ void dft2(V& a, V& b) {
    V t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <typename V>
__device__ __forceinline__ void dft3(V& v0, V& v1, V& v2, bool inv) {
    using T = typename Real<V>::type;
    const T s3 = (T)0.866025403784438646763723170752936183L;
    V t1 = cadd(v1, v2), t2 = csub(v1, v2);
    V m1;
    m1.x = v0.x - (T)0.5 * t1.x;
    m1.y = v0.y - (T)0.5 * t1.y;
    V m2;  // (inv ? +i : -i) * s3 * t2
    if (inv) { m2.x = -s3 * t2.y; m2.y = s3 * t2.x; }
    else     { m2.x = s3 * t2.y;  m2.y = -s3 * t2.x; }
    v0 = cadd(v0, t1);
    v1 = cadd(m1, m2);
    v2 = csub(m1, m2);
}

template <typename V>
__device__ __forceinline__ void dft4(V& v0, V& v1, V& v2, V& v3, bool inv) {
    V a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), d = csub(v1, v3);
    V a3;
    if (inv) { a3.x = -d.y; a3.y = d.x; }   // +i d
    else     { a3.x = d.y;  a3.y = -d.x; }  // -i d
    v0 = cadd(a0, a2);
    v2 = csub(a0, a2);
    v1 = cadd(a1, a3);
    v3 = csub(a1, a3);
}

template <int R, typename V>
__device__ __forceinline__ void stockham_pass(const V* in, V* out, int n, int nlines, int Ns,
                                              const V* __restrict__ tw, bool inv) {
    const int nb = n / R;
    const int step = n / (Ns * R);
    for (int idx = threadIdx.x; idx < nb * nlines; idx += blockDim.x) {
        const int line = idx / nb;
        const int j = idx - line * nb;
        const V* src = in + (size_t)line * n;
        V* dst = out + (size_t)line * n;
        const int k = j % Ns;
        V v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = src[j + q * nb];
        if (k) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                V w = __ldg(&tw[q * k * step]);
                if (!inv) w.y = -w.y;
                v[q] = cmul(v[q], w);
            }
        }
        if (R == 2) dft2(v[0], v[1]);
        if (R == 3) dft3(v[0], v[1], v[2 % R], inv);
        if (R == 4) dft4(v[0], v[1], v[2 % R], v[3 % R], inv);
        const int o = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) dst[o + q * Ns] = v[q];
    }
}

// nlines transforms of length rad.n held contiguously in a; b is scratch of equal size.
// Returns the buffer holding the result.  Must be called by every thread of the block.
template <typename V>
__device__ V* smem_fft(V* a, V* b, int nlines, const V* __restrict__ tw, bool inv, const Radices& rad) {
    int Ns = 1;
    const int n = rad.n;
    for (int p = 0; p < rad.count; ++p) {
        const int R = rad.r[p];
        if (R == 4) stockham_pass<4>(a, b, n, nlines, Ns, tw, inv);
        else if (R == 2) stockham_pass<2>(a, b, n, nlines, Ns, tw, inv);
        else stockham_pass<3>(a, b, n, nlines, Ns, tw, inv);
        __syncthreads();
        V* t = a; a = b; b = t;
        Ns *= R;
    }
    return a;
}

}  // namespace tc
