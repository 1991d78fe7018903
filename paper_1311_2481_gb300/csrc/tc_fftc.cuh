// Transforms of compile-time length (FP32 or FP64 lines): radix plans, in-register DFT
// codelets and Stockham passes over lines held in shared memory with one padding slot per
// 32 entries, which keeps the strided accesses of every pass at the minimum number of
// shared-memory wavefronts.  Used by the length-specialised theta and z passes.
#pragma once

#include "tc_internal.cuh"

namespace tc {
namespace cft {

// ---------------------------------------------------------------- radix plans
// Two tables: radices up to 16 (fewer passes) and up to 8 (fewer registers per butterfly:
// a radix-16 butterfly with its twiddles holds ~60 values in registers).
template <int N> struct PlanR16;
template <> struct PlanR16<12> { static constexpr int np = 2; static constexpr int r[6] = {4, 3}; };
template <> struct PlanR16<24> { static constexpr int np = 2; static constexpr int r[6] = {8, 3}; };
template <> struct PlanR16<48> { static constexpr int np = 2; static constexpr int r[6] = {16, 3}; };
template <> struct PlanR16<96> { static constexpr int np = 3; static constexpr int r[6] = {8, 4, 3}; };
template <> struct PlanR16<192> { static constexpr int np = 3; static constexpr int r[6] = {8, 8, 3}; };
template <> struct PlanR16<384> { static constexpr int np = 3; static constexpr int r[6] = {16, 8, 3}; };
template <> struct PlanR16<768> { static constexpr int np = 3; static constexpr int r[6] = {16, 16, 3}; };
template <> struct PlanR16<1152> { static constexpr int np = 4; static constexpr int r[6] = {16, 8, 3, 3}; };
template <> struct PlanR16<1536> { static constexpr int np = 4; static constexpr int r[6] = {16, 16, 2, 3}; };
template <> struct PlanR16<2304> { static constexpr int np = 4; static constexpr int r[6] = {16, 16, 3, 3}; };
template <> struct PlanR16<3072> { static constexpr int np = 4; static constexpr int r[6] = {16, 16, 4, 3}; };
template <int N> struct PlanR8;
template <> struct PlanR8<12> { static constexpr int np = 2; static constexpr int r[6] = {4, 3}; };
template <> struct PlanR8<24> { static constexpr int np = 2; static constexpr int r[6] = {8, 3}; };
template <> struct PlanR8<48> { static constexpr int np = 3; static constexpr int r[6] = {8, 2, 3}; };
template <> struct PlanR8<96> { static constexpr int np = 3; static constexpr int r[6] = {8, 4, 3}; };
template <> struct PlanR8<192> { static constexpr int np = 3; static constexpr int r[6] = {8, 8, 3}; };
template <> struct PlanR8<384> { static constexpr int np = 4; static constexpr int r[6] = {8, 8, 2, 3}; };
template <> struct PlanR8<768> { static constexpr int np = 4; static constexpr int r[6] = {8, 8, 4, 3}; };
template <> struct PlanR8<1152> { static constexpr int np = 5; static constexpr int r[6] = {8, 8, 2, 3, 3}; };
template <> struct PlanR8<1536> { static constexpr int np = 4; static constexpr int r[6] = {8, 8, 8, 3}; };
template <> struct PlanR8<2304> { static constexpr int np = 5; static constexpr int r[6] = {8, 8, 4, 3, 3}; };
template <> struct PlanR8<3072> { static constexpr int np = 5; static constexpr int r[6] = {8, 8, 8, 2, 3}; };
template <int N, bool R8> struct Plan;
template <int N> struct Plan<N, false> : PlanR16<N> {};
template <int N> struct Plan<N, true> : PlanR8<N> {};

__device__ __forceinline__ int pd(int i) { return i + (i >> 5); }
template <int PT> __host__ __device__ constexpr int padded() { return PT + (PT + 31) / 32; }

template <typename V> struct Elem;
template <> struct Elem<float2> { using T = float; };
template <> struct Elem<double2> { using T = double; };

template <typename V> __device__ __forceinline__ V vmk(typename Elem<V>::T x, typename Elem<V>::T y) {
    V v;
    v.x = x;
    v.y = y;
    return v;
}
template <typename V> __device__ __forceinline__ V vadd(V a, V b) { return vmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V vsub(V a, V b) { return vmk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V vmul(V a, V b) {
    return vmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V> __device__ __forceinline__ V rot(V a) {
    return INV ? vmk<V>(-a.y, a.x) : vmk<V>(a.y, -a.x);
}
template <typename V> __device__ __forceinline__ V vneg(V a) { return vmk<V>(-a.x, -a.y); }
// a + b and a - b where ZA / ZB say that a / b is known to be zero at compile time: the sum
// is then the other operand, exactly (up to the sign of a zero result)
template <bool ZA, bool ZB, typename V> __device__ __forceinline__ V zadd(V a, V b) {
    static_assert(!(ZA && ZB), "both operands zero");
    if constexpr (ZB) return a;
    else if constexpr (ZA) return b;
    else return vadd(a, b);
}
template <bool ZA, bool ZB, typename V> __device__ __forceinline__ V zsub(V a, V b) {
    static_assert(!(ZA && ZB), "both operands zero");
    if constexpr (ZB) return a;
    else if constexpr (ZA) return vneg(b);
    else return vsub(a, b);
}
// bits i0, i1, i2, i3 of a zero mask, as the mask of a 4-input codelet
template <unsigned Z, int I0, int I1, int I2, int I3> __host__ __device__ constexpr unsigned sub4() {
    return ((Z >> I0) & 1u) | (((Z >> I1) & 1u) << 1) | (((Z >> I2) & 1u) << 2) | (((Z >> I3) & 1u) << 3);
}

// ---------------------------------------------------------------- in-register DFTs
// X_k = sum_n x_n exp(s 2 pi i n k / R), s = +1 (inverse) or -1 (forward), in natural order.
// The radix-4 and 8 codelets take a compile-time mask Z of inputs known to be zero (bit n for
// x_n; the first pass of an inverse transform over the zero band of a dealiased spectrum):
// the additions with those inputs are left out, which changes no result bit but the sign of
// a zero.
template <bool INV, typename V> __device__ __forceinline__ void dft2(V* v) {
    const V a = v[0];
    v[0] = vadd(a, v[1]);
    v[1] = vsub(a, v[1]);
}
template <bool INV, typename V> __device__ __forceinline__ void dft3(V* v) {
    using T = typename Elem<V>::T;
    const T h = (T)0.866025403784438646763723170752936183L;   // sin(pi/3)
    const V t1 = vadd(v[1], v[2]), t2 = vsub(v[1], v[2]);
    const V m1 = vmk<V>(v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y);
    const V m2 = rot<INV>(vmk<V>(h * t2.x, h * t2.y));
    v[0] = vadd(v[0], t1);
    v[1] = vadd(m1, m2);
    v[2] = vsub(m1, m2);
}
template <bool INV, unsigned Z = 0, typename V> __device__ __forceinline__ void dft4(V* v) {
    constexpr bool z0 = Z & 1u, z1 = (Z >> 1) & 1u, z2 = (Z >> 2) & 1u, z3 = (Z >> 3) & 1u;
    const V a0 = zadd<z0, z2>(v[0], v[2]), a1 = zsub<z0, z2>(v[0], v[2]);
    const V a2 = zadd<z1, z3>(v[1], v[3]), a3 = rot<INV>(zsub<z1, z3>(v[1], v[3]));
    v[0] = vadd(a0, a2);
    v[2] = vsub(a0, a2);
    v[1] = vadd(a1, a3);
    v[3] = vsub(a1, a3);
}
// a * exp(s 2 pi i J / 16) with constant factors, J in {0, 1, 2, 3, 4, 6}
template <bool INV, int J, typename V> __device__ __forceinline__ V w16(V a) {
    using T = typename Elem<V>::T;
    constexpr T c1 = (T)0.923879532511286756128183189396788933L;   // cos(pi/8)
    constexpr T s1 = (T)0.382683432365089771728459984030398866L;   // sin(pi/8)
    constexpr T h = (T)0.707106781186547524400844362104849039L;    // cos(pi/4)
    constexpr T s = INV ? (T)1 : (T)-1;
    static_assert(J == 0 || J == 1 || J == 2 || J == 3 || J == 4 || J == 6, "unsupported W16 power");
    if constexpr (J == 0) return a;
    else if constexpr (J == 1) return vmul(a, vmk<V>(c1, s * s1));
    else if constexpr (J == 2) return vmul(a, vmk<V>(h, s * h));
    else if constexpr (J == 3) return vmul(a, vmk<V>(s1, s * c1));
    else if constexpr (J == 4) return rot<INV>(a);
    else return rot<INV>(vmul(a, vmk<V>(h, s * h)));
}
template <bool INV, unsigned Z = 0, typename V> __device__ __forceinline__ void dft8(V* v) {
    // two DFT-4 of the even and odd samples, then the W8 butterflies
    V e[4] = {v[0], v[2], v[4], v[6]};
    V o[4] = {v[1], v[3], v[5], v[7]};
    dft4<INV, sub4<Z, 0, 2, 4, 6>()>(e);
    dft4<INV, sub4<Z, 1, 3, 5, 7>()>(o);
    o[1] = w16<INV, 2>(o[1]);
    o[2] = rot<INV>(o[2]);
    o[3] = w16<INV, 6>(o[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = vadd(e[k], o[k]);
        v[k + 4] = vsub(e[k], o[k]);
    }
}
template <bool INV, typename V> __device__ __forceinline__ void dft16(V* v) {
    // 16 = 4 x 4: DFT-4 over n1 for each n2, twiddle W16^(n2 k1), DFT-4 over n2
    V y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        V t[4] = {v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]};
        dft4<INV>(t);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = t[k1];
    }
    y[1][1] = w16<INV, 1>(y[1][1]);
    y[1][2] = w16<INV, 2>(y[1][2]);
    y[1][3] = w16<INV, 3>(y[1][3]);
    y[2][1] = w16<INV, 2>(y[2][1]);
    y[2][2] = w16<INV, 4>(y[2][2]);
    y[2][3] = w16<INV, 6>(y[2][3]);
    y[3][1] = w16<INV, 3>(y[3][1]);
    y[3][2] = w16<INV, 6>(y[3][2]);
    // W16^9 = -W16^1
    {
        const V t = w16<INV, 1>(y[3][3]);
        y[3][3] = vmk<V>(-t.x, -t.y);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        V t[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
        dft4<INV>(t);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
    }
}
template <int R, bool INV, unsigned Z = 0, typename V> __device__ __forceinline__ void dftR(V* v) {
    static_assert(Z == 0 || R == 4 || R == 8, "zero masks only for radix 4 and 8");
    if constexpr (R == 2) dft2<INV>(v);
    else if constexpr (R == 3) dft3<INV>(v);
    else if constexpr (R == 4) dft4<INV, Z>(v);
    else if constexpr (R == 8) dft8<INV, Z>(v);
    else dft16<INV>(v);
}

// ---------------------------------------------------------------- Stockham passes
// one radix-R pass over NL lines of length PT: in -> out, Ns = product of earlier radices
// Inputs at positions zlo <= p < zhi are zero and are not read (the dealiasing band of an
// inverse transform's input; only the first pass is given a band).
// twiddle j of the table: from shared memory (TWS, the caller copied the table there) or
// through the read-only path from global memory
template <bool TWS, typename V> __device__ __forceinline__ V twiddle(const V* __restrict__ tw, int j) {
    if constexpr (TWS) return tw[j];
    else return __ldg(&tw[j]);
}

// ZM: inputs q of every butterfly known to be zero (the caller has checked the band)
template <int PT, int R, int NS, int NL, int NT, bool INV, typename V, bool TWS, unsigned ZM>
__device__ __forceinline__ void pass_body(const V* in, V* out, const V* __restrict__ tw, int zlo, int zhi) {
    constexpr int NB = PT / R;
    constexpr int STEP = PT / (NS * R);
    constexpr int LP = padded<PT>();
    for (int idx = threadIdx.x; idx < NL * NB; idx += NT) {
        const int line = idx / NB;
        const int j = idx - line * NB;
        const V* src = in + line * LP;
        V* dst = out + line * LP;
        const int k = j % NS;
        V v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int pos = j + q * NB;
            v[q] = ((ZM >> q) & 1u) || (pos >= zlo && pos < zhi) ? vmk<V>(0, 0) : src[pd(pos)];
        }
        if (NS > 1 && k) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                V w = twiddle<TWS>(tw, q * k * STEP);
                if (!INV) w.y = -w.y;
                v[q] = vmul(v[q], w);
            }
        }
        dftR<R, INV, ZM>(v);
        const int o = (j / NS) * NS * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) dst[pd(o + q * NS)] = v[q];
    }
    __syncthreads();
}
template <int PT, int R, int NS, int NL, int NT, bool INV, typename V, bool TWS = false>
__device__ __forceinline__ void pass(const V* in, V* out, const V* __restrict__ tw, int zlo, int zhi) {
    // A first radix-8 pass reads input q of butterfly j at j + q PT / 8.  When the zero band
    // [zlo, zhi) holds [3 PT / 8, 5 PT / 8) (a dealiased spectrum, |m| <= PT / 3), inputs 3
    // and 4 are zero in every butterfly.  Taken for FP64 lines only, where the FP64 pipe
    // bounds the pass; FP32 lines, bound by latency, ran no faster with it.
    if constexpr (NS == 1 && R == 8 && sizeof(V) == 16) {
        constexpr int NB = PT / 8;
        if (zlo <= 3 * NB && zhi >= 5 * NB) {
            pass_body<PT, R, NS, NL, NT, INV, V, TWS, (1u << 3) | (1u << 4)>(in, out, tw, zlo, zhi);
            return;
        }
    }
    pass_body<PT, R, NS, NL, NT, INV, V, TWS, 0u>(in, out, tw, zlo, zhi);
}

// all passes of the plan; returns the buffer that holds the result
// zlo, zhi: zero band of the input (first pass only); zlo = zhi = PT for none
template <int PT, int P, int NS, int NL, int NT, bool INV, typename V, bool R8 = sizeof(V) == 16, bool TWS = false>
__device__ __forceinline__ V* passes(V* a, V* b, const V* __restrict__ tw, int zlo = PT, int zhi = PT) {
    if constexpr (P == Plan<PT, R8>::np) {
        return a;
    } else {
        constexpr int R = Plan<PT, R8>::r[P];
        if constexpr (P == 0) pass<PT, R, NS, NL, NT, INV, V, TWS>(a, b, tw, zlo, zhi);
        else pass<PT, R, NS, NL, NT, INV, V, TWS>(a, b, tw, PT, PT);
        return passes<PT, P + 1, NS * R, NL, NT, INV, V, R8, TWS>(b, a, tw, PT, PT);
    }
}
template <int PT, bool R8> __host__ __device__ constexpr bool result_in_first() { return Plan<PT, R8>::np % 2 == 0; }

// ---------------------------------------------------------------- partial plans
// product of the radices before pass P (the NS a pass P starts from)
template <int PT, int P, bool R8> __host__ __device__ constexpr int ns_before() {
    int ns = 1;
    for (int i = 0; i < P; ++i) ns *= Plan<PT, R8>::r[i];
    return ns;
}
// passes P .. PEND - 1 of the plan, ping-pong from a; returns the buffer that holds the result
// zlo, zhi: zero band of the input of pass P (used only when P == 0)
template <int PT, int P, int PEND, int NL, int NT, bool INV, typename V, bool R8, bool TWS = false>
__device__ __forceinline__ V* passes_range(V* a, V* b, const V* __restrict__ tw, int zlo = PT, int zhi = PT) {
    if constexpr (P == PEND) {
        return a;
    } else {
        constexpr int R = Plan<PT, R8>::r[P];
        constexpr int NS = ns_before<PT, P, R8>();
        pass<PT, R, NS, NL, NT, INV, V, TWS>(a, b, tw, P == 0 ? zlo : PT, P == 0 ? zhi : PT);
        return passes_range<PT, P + 1, PEND, NL, NT, INV, V, R8, TWS>(b, a, tw, PT, PT);
    }
}

// ---------------------------------------------------------------- spectra of two line kinds
// pair line x = c_r + i c_t from (A, B) = (c_+, c_-): spectrum A_m at m > 0, conj(B_m) at -m,
// (A_0 + conj B_0)/2 at 0.  Real-pair line x + i y from (X, Y): X_m + i Y_m at m, conj(X_m) +
// i conj(Y_m) at -m.
template <typename V>
__device__ __forceinline__ void put_pair(V* line, int PTn, int m, V A, V B) {
    using T = typename Elem<V>::T;
    if (m == 0) {
        line[0] = vmk<V>((T)0.5 * (A.x + B.x), (T)0.5 * (A.y - B.y));
    } else {
        line[pd(m)] = A;
        line[pd(PTn - m)] = vmk<V>(B.x, -B.y);
    }
}
template <typename V>
__device__ __forceinline__ void put_real2(V* line, int PTn, int m, V X, V Y) {
    if (m == 0) {
        line[0] = vmk<V>(X.x, Y.x);
    } else {
        line[pd(m)] = vmk<V>(X.x - Y.y, X.y + Y.x);
        line[pd(PTn - m)] = vmk<V>(X.x + Y.y, Y.x - X.y);
    }
}
template <typename V>
__device__ __forceinline__ V imul(V a, typename Elem<V>::T s) { return vmk<V>(-s * a.y, s * a.x); }

}  // namespace cft
}  // namespace tc
