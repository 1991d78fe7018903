/*
 * tc.h -- C ABI of libtc, the GB300 (sm_103a) hot path of one Taylor–Couette DNS time step
 * (Shi, Rampp, Hof & Avila, "A hybrid MPI-OpenMP parallel implementation for pseudospectral
 * simulations with application to Taylor–Couette flow").
 *
 * Discretisation (Sec. 3.1): Fourier–Galerkin in theta and z, high-order finite differences on
 * N_r clustered radial nodes r_j (Eq. nodeDist), time stepping by the AB2BD2 projection scheme
 * of Sec. 3.2 (Eq. timeScheme .. Eq. update).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Spectral arrays are complex128 (interleaved re, im doubles), C order, device memory owned
 *    by the caller.  A vector field is [3][N_r][M+1][2K+1] holding (u_+, u_-, u_z) with
 *    u_+- = u_r +- i u_theta per Fourier mode (Sec. 3.1, before Eq. modalNSdecoup); a scalar
 *    field is [N_r][M+1][2K+1].  Index [c][j][m][k+K] is radial node j, azimuthal mode
 *    m = 0..M (wavenumber m * m_p), axial mode k = -K..K (wavenumber k * k_z, k_z = 2 pi / L_z).
 *    The m < 0 half follows from the reality of the physical fields; in the inverse transform
 *    the m = 0 line of u_r, u_theta, u_z contributes through its real part.
 *  - Physical grid for the nonlinear term: P_theta x P_z points per radial node (default
 *    3M x 3K, the 3/2 rule of Sec. 3.1 / Sec. 3.2 step 1).
 *  - Every call validates its arguments on the host before any launch and returns a
 *    tc_status; nothing aborts.  Device pointers must be 16-byte aligned device memory, and
 *    the array's bytes from the pointer must be mapped without a gap (TC_ERR_ARG otherwise;
 *    a short buffer followed by another allocation cannot be detected).  Kernels are enqueued on the caller's stream (cudaStream_t
 *    passed as void*; NULL = legacy default stream); calls return before the GPU finishes.
 *    Asynchronous CUDA errors surface as TC_ERR_CUDA on a later call.
 *  - ws is caller-owned device scratch of at least tc_plan_workspace_bytes() bytes, 256-byte
 *    aligned; its contents are undefined between calls.  A plan and its workspace may be used
 *    by one stream at a time.  Plans are not thread safe.
 *  - Input and output arrays must not overlap unless stated.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_plan tc_plan; /* opaque; owns nodes, FD weights, twiddles and LU factors */

typedef enum {
    TC_OK = 0,
    TC_ERR_ARG = 1,       /* invalid argument (checked on the host before any launch) */
    TC_ERR_CUDA = 2,      /* a CUDA runtime call failed (see tc_plan_last_error) */
    TC_ERR_OOM = 3,       /* device or host allocation failed */
    TC_ERR_NONFINITE = 4, /* a NaN/Inf was found in the state (tc_diagnostics), or an earlier
                             step wrote one (tc_step, tc_step_host) */
    TC_ERR_TIMEOUT = 5,   /* reserved: a bounded device wait gave up (no such wait exists yet) */
    TC_ERR_STATE = 6      /* call not allowed in this plan state (e.g. host-only plan) */
} tc_status;

/* Which of the five banded systems of Sec. 3.2 (steps 2-4) tc_helmholtz_solve solves. */
typedef enum {
    TC_P_STAR = 0,  /* Eq. pressure: Lap_h p* = rhs, Neumann rows at both walls */
    TC_U_PLUS = 1,  /* Eq. vel, u_+ : (3/(2dt) - L_+) u = rhs, Dirichlet rows */
    TC_U_MINUS = 2, /* Eq. vel, u_- : (3/(2dt) - L_-) u = rhs, Dirichlet rows */
    TC_U_Z = 3,     /* Eq. vel, u_z : (3/(2dt) - Lap_h) u = rhs, Dirichlet rows */
    TC_PHI = 4      /* Eq. correction: same matrix as TC_P_STAR */
} tc_system;

typedef enum { TC_FP64 = 0, TC_MIXED = 1 } tc_precision;

/* Optional plan settings; zero-initialise and set what differs from the defaults. */
typedef struct {
    double alpha;     /* node clustering of Eq. nodeDist; 0 -> default 0.5; use a negative
                         value for the Chebyshev limit alpha -> 0 */
    int P_theta;      /* physical points in theta; 0 -> 3M.  Must be 2^a 3^b >= 2M+1 */
    int P_z;          /* physical points in z;     0 -> 3K.  Must be 2^a 3^b >= 2K+1 */
    int precision;    /* tc_precision; TC_MIXED runs the transforms and products in FP32 */
    int host_only;    /* 1: build the host plan only (no device memory); for inspection */
    int theta_zt;     /* launch tuning: z values per theta-pass block (0: automatic); in the
                         mixed form a value > 0 also selects the generic theta kernel over the
                         length-specialised one */
    int pc_modes;     /* launch tuning: modes per block of the steps-2-5 kernel, rounded down to
                         a power of two, at most 16 (0: automatic) */
    int no_adjoint;   /* 1: size the workspace without the adjoint regions (tc_adjoint_* then
                         return TC_ERR_STATE); a TC_MIXED plan also stages its transforms in FP32 */
    int pc_split;     /* steps 2-5 as one fused kernel (-1) or as separate kernels (1);
                         0: fused while N_r <= 192, separate beyond */
    int theta_variant; /* launch tuning of the mixed form's length-specialised theta pass:
                         0 or 1: radices <= 16, two blocks per SM; 2 and 3: radices <= 8 with
                         half the z values per block, four / three blocks per SM; 4 (lengths
                         384 and up): variant 1 with the last inverse transform pass and the
                         first forward pass fused into the products */
    int pc_partitions; /* the fused steps-2-5 kernel solves each banded system (Sec. 3.2) as
                         two partitions, rows [0, N_r/2) and [N_r/2, N_r), each with its own
                         pivoted LU factors, coupled through an 8 x 8 reduced system (SPIKE
                         form; the two halves run on separate lanes).  0 or 2: when N_r >= 16
                         and the fused kernel runs; 1: one pivoted banded LU per system */
    int stage_rows;   /* radial rows per slab of the FP64 transform staging.  The transforms of
                         the nonlinear term (Sec. 3.2 step 1) and of its adjoint act on each
                         radial row independently, so they run slab by slab and the workspace
                         holds the FP64 lines of one slab: 12 line sets of (M+1) P_z values per
                         row for the FP64 forward term, 21 for the adjoint.  0: all rows while
                         that staging stays within 4 GiB, else the most rows that do; the
                         mixed form's FP32 forward lines always cover all rows */
    int mean_fp32;    /* TC_MIXED only.  0 (default): the (m, k) = (0, 0) mode of N, the mean
                         that drives the mean flow and the wall torque, comes from an exact
                         Parseval sum over the stored modes in double-FP32 arithmetic (alias-
                         free under the 3/2 rule), run beside the FP32 transforms; 1: keep the
                         FP32 transforms' value of that mode (about 6% faster at N_r = 64,
                         inner-wall torque error up to 1e-4 after 100 steps at N_r = 384) */
} tc_options;

/* Keys of tc_plan_set: one per field of tc_options, with the same meaning and range. */
typedef enum {
    TC_SET_ALPHA = 0,
    TC_SET_P_THETA = 1,
    TC_SET_P_Z = 2,
    TC_SET_PRECISION = 3,
    TC_SET_HOST_ONLY = 4,
    TC_SET_THETA_ZT = 5,
    TC_SET_PC_MODES = 6,
    TC_SET_NO_ADJOINT = 7,
    TC_SET_PC_SPLIT = 8,
    TC_SET_THETA_VARIANT = 9,
    TC_SET_PC_PARTITIONS = 10,
    TC_SET_STAGE_ROWS = 11,
    TC_SET_MEAN_FP32 = 12
} tc_plan_key;

/* Step state (Sec. 3.2): u = u^i, u_prev = u^{i-1}, N_prev = N^{i-1} (vector fields), p = p^i
 * (scalar field), started = 0 for a cold state whose history is built by the first step. */
typedef struct {
    void* u;
    void* u_prev;
    void* N_prev;
    void* p;
    int started;
} tc_state;

/* Diagnostics of a velocity field (Sec. 5): perturbation energy about analytic Couette flow
 * J = 1/2 sum_j w_j r_j sum_{m,k} c_m |u - U|^2 (trapezoid weights w_j, c_0 = 1, c_m = 2),
 * torque T = r^3 d_r(u_theta^{00} / r) at r_i and r_o with the wall FD rows, the
 * quasi-Nusselt number Nu_omega = T / T_lam of Sec. 5.4 at each wall (T_lam = -2 C2 is the
 * torque of circular Couette flow U = C1 r + C2 / r, Sec. 5.1; NaN when C2 = 0), max
 * |div_h u| over interior rows, and whether every entry is finite. */
typedef struct {
    double energy;
    double torque_inner;
    double torque_outer;
    double max_div;
    int finite;
    double nu_omega_inner;
    double nu_omega_outer;
} tc_diag;

/* Create a plan: nodes (Eq. nodeDist, paper's M = N_r - 1), FD weights of fd_order + 1 points
 * (Sec. 3.1; shortened centred stencils near the walls, one-sided fd_order/2 + 1 points on
 * the wall rows), twiddles, and the banded LU factors with partial pivoting of the Poisson
 * and three Helmholtz matrices of every mode (m, |k|), factored once before any step
 * (Sec. 3.2).  Requires fd_order + 1 <= N_r <= 2048, M >= 1, K >= 1, m_p >= 1, 0 < eta < 1,
 * L_z > 0, dt > 0, fd_order in {2, 4, 6, 8}.  *out receives the plan or NULL on error. */
tc_status tc_plan_create(tc_plan** out, int N_r, int M, int K, int m_p, double eta,
                         double Re_i, double Re_o, double L_z, double dt, int fd_order);
tc_status tc_plan_create_ex(tc_plan** out, int N_r, int M, int K, int m_p, double eta,
                            double Re_i, double Re_o, double L_z, double dt, int fd_order,
                            const tc_options* opt);
void tc_plan_destroy(tc_plan* plan);
/* Change one plan setting after creation and before the plan's first compute call: the
 * physical grid (P_theta, P_z of the 3/2 rule, Sec. 3.1), the node clustering alpha of
 * Eq. nodeDist, the precision form, or a launch option (key: tc_plan_key; an integer setting
 * takes an integral value).  Everything that depends on the setting (nodes, FD weights,
 * twiddles, the LU factors of Sec. 3.2, the workspace size) is rebuilt as tc_plan_create_ex
 * would build it; on any error the plan is left unchanged.  The workspace size may change:
 * query tc_plan_workspace_bytes again.  TC_ERR_ARG for an unknown key or a value out of
 * range; TC_ERR_STATE once the plan has run a compute call (tc_nonlinear, tc_step, ...) or
 * when the current device is not the plan's.  While the replacement is built, the device
 * holds the constants of both (the factors dominate: 13 doubles per row, mode and set). */
tc_status tc_plan_set(tc_plan* plan, int key, double value);

/* Device scratch needed by every call that takes ws. */
tc_status tc_plan_workspace_bytes(const tc_plan* plan, size_t* bytes);
/* Radial nodes r_j, j = 0..N_r-1, into host memory r_host[N_r]. */
tc_status tc_plan_nodes(const tc_plan* plan, double* r_host);
/* FD weights into host memory: w[N_r][fd_order+1] applied to nodes col0[j] + t
 * (zero-padded), deriv = 1 or 2. */
tc_status tc_plan_fd_weights(const tc_plan* plan, int deriv, double* w_host, int* col0_host);
/* Inspection of the stored factors (host_only plans): x = A^{-1} b on the host for the system
 * `which` of mode (m, |k| = ka), b and x real host arrays of N_r values, with the pivoted
 * banded LU factors (partitions = 1) or the two-partition form the fused steps-2-5 kernel
 * uses (partitions = 2: TC_ERR_STATE if the plan has none).  TC_ERR_STATE on a plan with
 * device memory (its host factors are released after upload). */
tc_status tc_plan_solve_host(const tc_plan* plan, int which, int m, int ka, int partitions, const double* b,
                             double* x);
/* Text of the last CUDA error seen by this plan (static storage inside the plan). */
const char* tc_plan_last_error(const tc_plan* plan);
const char* tc_status_string(tc_status s);

/* Nonlinear term, Sec. 3.2 step 1: N_hat = N(u) = u . grad u with the curvature terms of
 * Eq. NS_cyl, evaluated pseudospectrally on the P_theta x P_z grid (d_r by the FD stencil,
 * d_theta and d_z as mode multiplies, inverse transforms, pointwise products, forward
 * transforms truncated to |m| <= M, |k| <= K).  u_hat, N_hat: device vector fields
 * (N_pm = N_r +- i N_theta). */
tc_status tc_nonlinear(tc_plan* plan, const void* u_hat, void* N_hat, void* ws, void* stream);

/* One of the five banded systems of Sec. 3.2 for every mode: rhs and x are device scalar
 * fields; rows 0 and N_r - 1 of rhs hold the boundary values (Dirichlet value, or the
 * Neumann value d_r x; for (m,k) = (0,0) the Poisson systems take a Dirichlet value at r_o,
 * Sec. 3.2).  x may equal rhs (in place). */
tc_status tc_helmholtz_solve(tc_plan* plan, int which, const void* rhs, void* x, void* ws,
                             void* stream);

/* nsteps AB2BD2 steps (Sec. 3.2 steps 1-5) in place on the caller's state.  A cold state
 * (started == 0) first gets its history: one implicit Euler step of size 2dt/3 (the scheme
 * with u^{-1} = u^0, N^{-1} = N^0, same factors), u^{-1} = u^0 - 1.5 (u_E - u^0),
 * N^{-1} = N(u^{-1}); started is then set to 1.  nsteps = 0 on a cold state builds only
 * that history.  The update kernel raises a flag (in mapped host memory, no synchronisation)
 * when it writes a NaN/Inf into the state; the first tc_step call that finds the flag set
 * returns TC_ERR_NONFINITE before launching anything and clears it, so the caller can
 * restore a state and continue.  Steps still in flight are not waited for: a blow-up is
 * reported by a later call. */
tc_status tc_step(tc_plan* plan, tc_state* st, int nsteps, void* ws, void* stream);

/* tc_step with the state in host memory.  host_in: host copies of u, u_prev, N_prev, p (all
 * four required) and its started flag; dev: caller-owned device buffers of the same shapes,
 * used as the working state; host_out: each non-null field receives the device result after
 * the steps (u, u_prev, N_prev, p; host_out->started is set).  Host buffers may be pinned or
 * pageable; pinned ones let the copies run at full link speed.  The copies and the steps are
 * enqueued on `stream`, which is synchronised before the call returns, so host_out is valid
 * on return.  For a started state and nsteps >= 1, u_prev and N_prev are copied on a second,
 * plan-owned stream while the first step's nonlinear term runs on u, and p is not copied in:
 * no step reads p^i (p* is solved afresh and the update writes p^{i+1}).  host_out fields
 * may alias host_in fields.  Errors: TC_ERR_ARG if a pointer of
 * dev is not device memory, a host pointer is device memory, or dev fields coincide;
 * TC_ERR_NONFINITE if these steps wrote a NaN/Inf into the state (host_out is written). */
tc_status tc_step_host(tc_plan* plan, const tc_state* host_in, tc_state* host_out, tc_state* dev,
                       int nsteps, void* ws, void* stream);

/* Diagnostics of the velocity field u (device vector field); synchronises the stream and
 * writes *out (host).  Returns TC_ERR_NONFINITE if u holds a NaN/Inf. */
tc_status tc_diagnostics(tc_plan* plan, const void* u, tc_diag* out, void* ws, void* stream);

/* Adjoint state: adjoints (w.r.t. the Euclidean inner product on the stored (Re, Im) pairs)
 * of the three vector fields a step carries forward. */
typedef struct {
    void* u;
    void* u_prev;
    void* N_prev;
} tc_state_bar;

/* Adjoint of one AB2BD2 step (differentiation form; the paper has no adjoint).  fwd is the
 * forward state before the step (u^i, u^{i-1}, N^{i-1}; started = 1).  On entry bar holds the
 * adjoints of the step's outputs (u^{i+1}, u^i, N^i); on return those of its inputs
 * (u^i, u^{i-1}, N^{i-1}), in place.  The linear part is the transposed chain of Sec. 3.2
 * steps 2-5 (transposed banded solves and stencils); the nonlinear part is the transposed
 * linearisation of N(u) = u . grad u about fwd->u (recomputed).  Runs in FP64 for every plan
 * precision.  Of fwd only u and started are read (u_prev, N_prev and p may be NULL).  The
 * three bar arrays must be distinct. */
tc_status tc_adjoint_step(tc_plan* plan, const tc_state* fwd, tc_state_bar* bar, void* ws,
                          void* stream);
/* Adjoint of the cold-start map u^0 -> (u^0, u^{-1}, N^{-1}) that tc_step applies to a state
 * with started == 0 (its Euler step is recomputed from u0): given the adjoints in bar of
 * (u^0, u^{-1}, N^{-1}), writes the adjoint of u^0 into u0_bar (distinct from u0 and from
 * bar->u_prev, bar->N_prev). */
tc_status tc_adjoint_start(tc_plan* plan, const void* u0, const tc_state_bar* bar, void* u0_bar,
                           void* ws, void* stream);
/* g = dJ/du for the perturbation energy J of tc_diag (gradient w.r.t. the stored (Re, Im)
 * pairs, as complex numbers); u, g device vector fields. */
tc_status tc_energy_gradient(tc_plan* plan, const void* u, void* g, void* stream);

/* Nonlinear term exactly as tc_nonlinear, for callers that cannot allocate device memory
 * (the paper has no counterpart: it is a packaging choice of this library).  Instead of a
 * caller workspace, the staging lines between the transform kernels live in one static
 * 80 MiB device array that every GPU loading the library keeps until the process exits.
 * The staging a plan needs is its workspace before N^i: for TC_FP64 plans 12 line sets of
 * stage_rows * (M+1) * P_z complex128 values (the transforms run slab by slab of stage_rows
 * radial rows); for TC_MIXED plans 12 line sets of N_r * (M+1) * P_z complex64 values and
 * 6 * N_r * (M+1) * (2K+1) complex64 values of the FP32 split of u and d_r u; each region
 * rounded up to 256 bytes.  Plans that need more than 80 MiB get TC_ERR_ARG before any
 * launch (a smaller stage_rows brings a TC_FP64 plan's need down).  Allocates nothing.  The first call on each device looks up the array's address
 * once (cudaGetSymbolAddress) and keeps it; make that call before any stream capture, and do
 * not call this entry point after a device reset (cudaDeviceReset or a primary-context reset
 * unloads the array and leaves the kept address stale).  All calls share the array: calls
 * whose GPU work overlaps (other streams, unordered plans) race on it. */
tc_status tc_nonlinear_noalloc(tc_plan* plan, const void* u_hat, void* N_hat, void* stream);

/* FP64 FMA rate probe (no counterpart in the paper: it measures the FP64 pipe that bounds the
 * FP64 kernels).  Enqueues one kernel of `blocks` x `threads` threads (threads a multiple of 32,
 * at most 1024), each running 8 independent chains of `iters` dependent FMAs, and writes one
 * double per thread into the device buffer `sink` (blocks * threads doubles, caller-owned;
 * only its type is checked).  *flops (host, may be NULL) receives the flops the launch
 * executes (2 per FMA); time the launch with events on `stream`. */
tc_status tc_probe_fp64_fma(int blocks, int threads, int iters, void* sink, void* stream, double* flops);

/* Tracing (no counterpart in the paper beyond its per-phase timings, Table efficiency):
 * when enabled, every kernel the plan launches is bracketed by CUDA events recorded on the
 * launching stream.  tc_profile_enable(plan, 1) also clears earlier records.
 * tc_profile_read(plan, index, ...) synchronises on the recorded events and reports, for
 * kernel `index` (0 <= index < 15, see name), the launches and total milliseconds recorded
 * since the last enable; TC_ERR_ARG past the last index.  name points to static storage. */
tc_status tc_profile_enable(tc_plan* plan, int enable);
tc_status tc_profile_read(tc_plan* plan, int index, const char** name, long long* launches,
                          double* total_ms);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
