// Internal declarations of libtc (plan layout, complex helpers, launch helpers).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/tc.h"

namespace tc {

constexpr int kMaxRadix = 16;   // passes of a mixed-radix 2^a 3^b transform
constexpr int kStencil = 9;     // padded FD stencil width (fd_order <= 8)
constexpr int kBands = 13;      // stored doubles per LU row: 4 L multipliers, 1/U_jj, 8 U
constexpr int kKl = 4;          // sub/super diagonals of the mode matrices (fd_order/2 <= 4)
constexpr int kPCDepth = 4;     // rows of LU factors in flight per substitution chain

// Factor sets of Sec. 3.2: Poisson (p*, phi), Helmholtz for u_+, u_-, u_z.
enum FactorSet { kSetP = 0, kSetHp = 1, kSetHm = 2, kSetHz = 3, kNumSets = 4 };

struct Radices {
    int n;
    int count;
    int r[kMaxRadix];
};

// Byte offsets of the workspace regions (all 256-byte aligned).
// Every region is scratch of one library call; regions that no call uses at the same time
// share memory (see tc_plan.cu).
struct Workspace {
    size_t H1;      // inverse z-pass output, 9 line sets [f][r][m][z]: FP64 lines of stage_rows
                    // rows, or the mixed form's FP32 lines of all N_r rows
    size_t H2;      // theta-pass output: 3 line sets, rows and precision as H1
    size_t P32;     // mixed form: u', d_r u' in FP32, 6 x S float2
    size_t mean;    // mixed form: segment sums of the mean mode of N (mean00_part_doubles)
    size_t Ncur;    // N^i: vector field (everything before it is the forward staging)
    size_t uE;      // start-up Euler result: vector field
    size_t pstar;   // split path only: p* (scalar), u* (vector), phi (scalar)
    size_t ustar;
    size_t phi;
    size_t red;     // diagnostics reduction buffer (diag_red_doubles doubles)
    // adjoint regions (absent with tc_options.no_adjoint), FP64 lines of stage_rows rows
    size_t H1a;     // recomputed forward lines of u: 9 line sets
    size_t Ha;      // adjoint lines of Nbar: 3 line sets
    size_t H3;      // adjoint theta-pass output: 9 line sets
    size_t Rhat;    // adjoint d_r lines before the transposed stencil: 3 x stage_rows rows of modes
    size_t Nbar;    // adjoint of N: vector field
    size_t abar;    // start-up adjoint temporaries: 3 vector fields
    size_t total;
};

}  // namespace tc

struct tc_plan {
    // parameters
    int N_r, M, K, m_p, fd_order, half, P_t, P_z, precision;
    double eta, Re_i, Re_o, L_z, dt, alpha, k_z, r_i, r_o;
    bool host_only;
    bool adjoint;    // workspace holds the adjoint regions
    tc_options opt;  // the options the plan was built with (tc_plan_set rebuilds from them)
    bool used = false;  // a compute call has run (tc_plan_set is refused from then on)
    // derived sizes
    size_t S;        // complex entries of a scalar spectral field
    size_t Hfield;   // complex entries of one z-pass line set of all rows: N_r (M+1) P_z
    int stage_rows;  // radial rows per slab of the FP64 transform staging
    int nmode;       // (M+1)(2K+1)
    int nmode_half;  // (M+1)(K+1)
    tc::Radices rad_z, rad_t;
    int zt, zt32;                  // z values per theta-pass block (FP64 / FP32 lines)
    int theta_zt_forced;           // tc_options.theta_zt (> 0: generic transform kernels)
    int theta_variant;             // tc_options.theta_variant (launch shape of the FP32 streamed theta pass)
    int pc_modes;                  // modes per block of the fused steps-2-5 kernel (0: auto)
    int num_sms = 152;             // multiprocessors of the plan's device
    int thr_zinv, thr_theta, thr_zfwd;  // block sizes of the FP64 transform kernels
    bool pc_split;                      // steps 2-5 as separate kernels (large N_r)
    int part_h = 0;                     // fused kernel: systems cut into rows [0, h), [h, N_r) (0: uncut)
    int zinv_lines, zinv_lines32;  // lines per inverse z-pass block (FP64 / FP32 lines)
    int zfwd_lines, zfwd_lines32;  // lines per forward z-pass block (3 or 1)
    tc::Workspace ws;
    // host plan
    std::vector<double> r, w1, w2;   // nodes; weights [N_r][9]
    std::vector<int> col0;           // first node of each padded stencil
    int d1t_n = 0;                   // entries per column of the transposed D1 gather table
    std::vector<int> d1t_row;        // [N_r][d1t_n] rows j with D1[j][col] != 0 (padded)
    std::vector<double> d1t_w;       // [N_r][d1t_n] matching weights D1[j][col] (0 padding)
    std::vector<double> fac;         // [set][j][band][m][ka]
    std::vector<uint8_t> piv;        // [set][j][m][ka] pivot offset 0..4
    // two-partition form (part_h > 0): LU factors of the diagonal blocks at their global
    // rows (layout of fac / piv), spikes [set][j][q][m][ka] (q < 4: V = A1^{-1} B for j < h,
    // W = A2^{-1} C for j >= h) and the inverse reduced matrix [set][8 i + l][m][ka]
    std::vector<double> fac2, spk, rinv;
    std::vector<uint8_t> piv2;
    std::vector<double> tw_z, tw_t;  // interleaved complex exp(+2 pi i j / n)
    // device plan
    double* d_r = nullptr;
    double* d_ir = nullptr;          // 1 / r_j
    double* d_w1 = nullptr;
    float* d_w1f = nullptr;          // FP32 copy of w1 (mixed form)
    float* d_dsc = nullptr;          // mixed form: power-of-two scale of d_r u_z beside u_z in a theta line
    double* d_w2 = nullptr;
    int* d_col0 = nullptr;
    int* d_d1t_row = nullptr;
    double* d_d1t_w = nullptr;
    double* d_fac = nullptr;
    uint8_t* d_piv = nullptr;
    double* d_fac2 = nullptr;
    uint8_t* d_piv2 = nullptr;
    double* d_spk = nullptr;
    double* d_rinv = nullptr;
    double2* d_tw_z = nullptr;
    double2* d_tw_t = nullptr;
    float2* d_tw_z32 = nullptr;
    float2* d_tw_t32 = nullptr;
    // non-finite flag: mapped pinned host memory that the update kernels set when they write
    // a NaN/Inf into the state; tc_step reports and clears it
    int* h_nonfinite = nullptr;
    int* d_nonfinite = nullptr;
    int device = -1;
    char err[512];
    // tc_step_host: a second stream that brings u_prev and N_prev in while the first step's
    // nonlinear term runs on u, with events for the hand-over (created on first use)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev[2] = {nullptr, nullptr};
    // mixed form: a second stream on which the mean mode of N runs beside the FP32
    // transforms, with events for the fork and the join (created with the device plan)
    cudaStream_t mean_stream = nullptr;
    cudaEvent_t mean_ev[2] = {nullptr, nullptr};
    // per-kernel CUDA-event tracing
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;         // event pool, two per record
    std::vector<int> prof_kid;                // kernel id of each record
    size_t prof_used = 0;                     // records in use
};

namespace tc {

// ------------------------------------------------------------------ complex helpers
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { V c; c.x = a.x + b.x; c.y = a.y + b.y; return c; }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { V c; c.x = a.x - b.x; c.y = a.y - b.y; return c; }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
    V c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
template <typename V> __host__ __device__ __forceinline__ V cconj(V a) { a.y = -a.y; return a; }
// i * a
template <typename V> __host__ __device__ __forceinline__ V cmuli(V a) { V c; c.x = -a.y; c.y = a.x; return c; }

// true if either part of v is a NaN or an Inf: exponent bits all set (integer test, no FP64
// instruction)
__device__ __forceinline__ bool nonfinite2(double2 v) {
    return ((__double2hiint(v.x) & 0x7ff00000) == 0x7ff00000) | ((__double2hiint(v.y) & 0x7ff00000) == 0x7ff00000);
}

// ------------------------------------------------------------------ error helpers
tc_status cuda_fail(tc_plan* p, cudaError_t e, const char* where);
#define TC_CUDA(plan, call)                                            \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return tc::cuda_fail(plan, e_, #call);  \
    } while (0)
#define TC_TRY_STATUS(x)                                               \
    do {                                                               \
        tc_status s_ = (x);                                            \
        if (s_ != TC_OK) return s_;                                    \
    } while (0)
#define TC_LAUNCHED(plan, what)                                        \
    do {                                                               \
        cudaError_t e_ = cudaGetLastError();                           \
        if (e_ != cudaSuccess) return tc::cuda_fail(plan, e_, what);   \
    } while (0)

// ptr must be 16-byte aligned device memory; with bytes > 0, the bytes from ptr must be mapped
// without a gap (checked through the driver's address-range query when the driver provides
// it; the check cannot tell a short buffer followed by another allocation from a long one)
tc_status check_device_ptr(tc_plan* p, const void* ptr, const char* name, size_t bytes = 0);

// ------------------------------------------------------------------ tracing
enum KernelId {
    kKZinv = 0, kKTheta, kKZfwd, kKRhsPressure, kKSolveP, kKRhsVelocity, kKSolveH, kKRhsDiv,
    kKUpdate, kKAxpby, kKDiag, kKZinv32, kKTheta32, kKZfwd32, kKPC, kKPCAdj,
    kKZinvAdj, kKThetaAdj, kKZfwdAdj, kKDrT, kKPrep32, kKMean00, kNumKernels
};
extern const char* const kKernelNames[kNumKernels];
int prof_begin(tc_plan* p, int kid, cudaStream_t s);
void prof_end(tc_plan* p, int slot, cudaStream_t s);

// ------------------------------------------------------------------ launchers
tc_status launch_nonlinear(tc_plan* p, const double2* u, double2* N, char* ws, cudaStream_t s);
tc_status launch_zinv_fp64(tc_plan* p, const double2* u, double2* H1, cudaStream_t s, int r0, int nh);
tc_status launch_theta32(tc_plan* p, const float2* H1, float2* H2, cudaStream_t s);
int theta_s_zt(const tc_plan* p, bool fp64);
tc_status launch_theta_s(tc_plan* p, const float2* H1, float2* H2, cudaStream_t s);
tc_status launch_theta_s64(tc_plan* p, const double2* H1, double2* H2, cudaStream_t s, int r0, int nh);
tc_status launch_nl_pre32(tc_plan* p, const double2* u, char* ws, cudaStream_t s, int ma, int mb);
tc_status launch_nl_theta32(tc_plan* p, char* ws, cudaStream_t s);
tc_status launch_nl_post32(tc_plan* p, const double2* u, double2* N, char* ws, cudaStream_t s, int ma, int mb);
size_t mean00_part_doubles(const tc_plan* p);
tc_status launch_mean00_part(tc_plan* p, const double2* u, char* ws, cudaStream_t s);
tc_status launch_mean00_fin(tc_plan* p, double2* N, char* ws, cudaStream_t s);
tc_status launch_solve(tc_plan* p, int set, double2* x, int nfields, cudaStream_t s);
tc_status launch_advance(tc_plan* p, const double2* u, double2* u_prev, const double2* Ncur,
                         double2* N_prev, double2* p_out, double2* u_out, char* ws,
                         bool commit, cudaStream_t s, int ma = 0, int mb = -1);
tc_status launch_axpby(tc_plan* p, double2* y, const double2* a, double ca, const double2* b,
                       double cb, size_t n, cudaStream_t s);
tc_status launch_diagnostics(tc_plan* p, const double2* u, double* red, cudaStream_t s);
size_t diag_red_doubles(const tc_plan* p);
tc_status launch_adjoint_advance(tc_plan* p, const double2* ubar_new, const double2* ubar_cur,
                                 const double2* Nbar_cur, double2* u_out, double2* up_out,
                                 double2* N_out, double2* Np_out, char* ws, cudaStream_t s);
tc_status launch_energy_gradient(tc_plan* p, const double2* u, double2* g, cudaStream_t s);
tc_status launch_nonlinear_adjoint(tc_plan* p, const double2* u, const double2* Nbar, double2* ubar,
                                   char* ws, cudaStream_t s);

}  // namespace tc
