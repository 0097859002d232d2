/*
 * uw.h -- C ABI of libuw: fast products with the N x M section U of the
 * Walsh-Hadamard -> boundary-wavelet change-of-basis matrix and with U^*.
 *
 * Paper: V. Antun, "Recovering wavelet coefficients from binary samples using
 * fast transforms", arXiv 2106.00554.
 *
 *   U_{n,m} = <r_m, w_n>                                  (Sec. 1.2)
 *   y = P_Omega U x,   x = U^* P_Omega^* y                 (Sec. 1.1, Algorithm 1)
 *   2D: alpha = G xi G^*, xi = G^* alpha G                 (Sec. 5, Algorithm 2)
 *
 * with w_n the sequency-ordered Walsh functions (Def. 3.1), r_m the
 * orthonormal Daubechies wavelet basis C_{psi,R} on [0,1]^d with periodic or
 * vanishing-moments-preserving (Cohen-Daubechies-Vial) boundary functions
 * (Sec. 3.2), M = 2^R per dimension and N = 2^{R+q} per dimension.  The
 * product is computed as IDWT -> dyadic upsample-and-convolve with the cell
 * integrals of the scaling function -> sequency FWHT -> selection of Omega,
 * and the adjoint as the same steps transposed, on one GPU.
 *
 * Conventions shared by every entry point:
 *  - All functions return a status (UW_OK = 0) or NULL on error; the status of
 *    the last failing call on the calling thread is kept in uw_last_error()
 *    and a message in uw_last_message().  No C++ exception crosses the ABI.
 *  - Device pointers are CUDA device addresses on the device that was
 *    current when the plan was created; the caller owns them.  Every call
 *    that runs a plan's product must be made with that device current: with
 *    another device current it returns UW_ERR_INVALID_ARG before any lookup
 *    or launch.  Host pointers
 *    are ordinary CPU memory (pinned memory is faster, pageable works).
 *  - Calls are asynchronous and ordered on the given stream (a cudaStream_t
 *    passed as void*; NULL = legacy default stream).  A plan may be used by
 *    one stream at a time: it owns one workspace.
 *  - Layouts are row-major.  1D x: batch x M, coefficients ordered
 *    [phi_{J0,.} | psi_{J0,.} | psi_{J0+1,.} | ... | psi_{R-1,.}].
 *    2D x: batch x M x M in the Mallat square layout (J0 scaling block at the
 *    top-left; at level j the three detail blocks [0:2^j, 2^j:2^{j+1}],
 *    [2^j:2^{j+1}, 0:2^j], [2^j:2^{j+1}, 2^j:2^{j+1}]).
 *    y: batch x m, the samples at the sorted linear sequency indices Omega
 *    (2D linear index n1 * N + n2, n1 = row of alpha).
 *  - Precision: UW_F64 (double in, double out, double arithmetic),
 *    UW_F32 (float in/out, float arithmetic on CUDA cores) and
 *    UW_F32_SPLIT_BF16 (float in/out; the last synthesis level, the
 *    upsample-convolve and the Walsh-Hadamard stages of bits 0-7 of each line
 *    run on the tensor cores with every operand split into three bfloat16
 *    parts and float accumulation -- as accurate as UW_F32; lines shorter
 *    than 512 samples and 1D plans with several levels per line take the
 *    UW_F32 kernels).
 */
#ifndef UW_H
#define UW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct uw_plan uw_plan;

enum { UW_BOUNDARY_PERIODIC = 0, UW_BOUNDARY_VMP = 1 };
/* OR'd into p (uw_plan_create, uw_host_table): the least-asymmetric
 * Daubechies filter (symlet) with p vanishing moments instead of the
 * extremal-phase one (Table 1's sym rows) */
enum { UW_FILTER_SYMLET = 0x100 };
enum { UW_F64 = 0, UW_F32 = 1, UW_F32_SPLIT_BF16 = 2 };
enum {
  UW_OK = 0,
  UW_ERR_INVALID_ARG = 1,  /* bad size, pointer, precision, batch, mask  */
  UW_ERR_UNSUPPORTED = 2,  /* valid request this build does not implement */
  UW_ERR_OOM = 3,          /* device or host allocation failed            */
  UW_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed        */
  UW_ERR_TIMEOUT = 5,      /* a bounded device wait gave up               */
  UW_ERR_INTERNAL = 6      /* a device-side consistency check tripped     */
};

/*
 * uw_plan_create -- build every input-independent table of the method on the
 * host in extended precision and upload it to the current CUDA device.
 *   d        dimension, 1 or 2 (Sec. 4 / Sec. 5)
 *   R        level of the reconstruction space, M = 2^R per dimension
 *   q        oversampling, N = 2^{R+q} per dimension (Remark 4.1), 0..6
 *   p        vanishing moments of the Daubechies wavelet (nu), 1..10;
 *            p | UW_FILTER_SYMLET selects the least-asymmetric filter
 *            (symlet): among the choices of one zero per reciprocal pair
 *            of m0 (Daubechies' construction), the one whose unwrapped
 *            phase is closest to linear in mean square on 256 points of
 *            (0, pi), oriented with its energy in the first half of the
 *            taps (equal to the extremal-phase filter for p <= 3)
 *   boundary UW_BOUNDARY_PERIODIC or UW_BOUNDARY_VMP (Sec. 3.2)
 * Tables (Sec. 4.1 "computed a priori", Sec. 4.3, Prop. 4.4): the filter h,
 * the (2p-1) 2^q cell integrals of phi, the boundary cell-integral rows and
 * the level-independent boundary two-scale blocks.  The coarsest level J0 is
 * the smallest J with 2^J >= 2 (2p - 1) (left and right edge functions
 * disjoint); R must satisfy J0 <= R and d * (R + q) <= 26.
 * Omega defaults to all N^d indices; the workspace to batch 1.
 * Returns NULL on error (uw_last_error() says why).  The plan owns its
 * device memory until uw_plan_destroy.
 */
uw_plan* uw_plan_create(int d, int R, int q, int p, int boundary);

/* uw_plan_set_coarsest -- choose J0 (J0_min(p) <= J0 <= R).  Invalidates
 * nothing else.  UW_ERR_INVALID_ARG if out of range. */
int uw_plan_set_coarsest(uw_plan* plan, int J0);

/*
 * uw_plan_set_mask -- P_Omega of Sec. 1.1.  omega_host: m strictly increasing
 * linear sequency indices in [0, N^d) (host memory, copied; the caller keeps
 * ownership).  omega_host == NULL or m < 0 selects all N^d indices.
 * Synchronous (uploads before returning).  UW_ERR_INVALID_ARG if the list
 * is unsorted, repeats or leaves the range.
 */
int uw_plan_set_mask(uw_plan* plan, const int64_t* omega_host, int64_t m);

/* uw_plan_reserve -- size the workspace for batches up to max_batch (>= 1)
 * in every precision.  The only allocation a plan makes after creation. */
int uw_plan_reserve(uw_plan* plan, int max_batch);

/* Accessors: number of samples m, coefficients per instance M^d,
 * coarsest level J0, N per dimension. */
int64_t uw_plan_num_samples(const uw_plan* plan);
int64_t uw_plan_num_coeffs(const uw_plan* plan);
int     uw_plan_coarsest(const uw_plan* plan);
int64_t uw_plan_n(const uw_plan* plan);

/*
 * uw_forward -- y = P_Omega U x for `batch` instances (Algorithm 1 in 1D,
 * Algorithm 2 in 2D, preceded by the IDWT of Remark 4.2).
 *   precision  UW_F64 / UW_F32 / UW_F32_SPLIT_BF16 (x, y are double for
 *              UW_F64 and float otherwise)
 *   x_dev      device, batch x M^d coefficients (read only)
 *   y_dev      device, batch x m samples (written; must not overlap x)
 *   batch      1 .. reserved max_batch, else UW_ERR_INVALID_ARG
 *   stream     cudaStream_t as void*
 */
int uw_forward(const uw_plan* plan, int precision, const void* x_dev, void* y_dev,
               int batch, void* stream);

/*
 * uw_adjoint -- x = U^* P_Omega^* y (Sec. 4.2 and the transposed Algorithm 2:
 * scatter into zeros, FWHT, transposed upsample-convolve, DWT).
 * Same arguments as uw_forward with the roles of x and y exchanged.
 */
int uw_adjoint(const uw_plan* plan, int precision, const void* y_dev, void* x_dev,
               int batch, void* stream);

/*
 * uw_forward_noalloc -- the same product as uw_forward for a 2D plan, with
 * its intermediate arrays in a fixed 8 MiB scratch array that the library
 * holds in device memory from the moment it is loaded on a device, instead
 * of the plan's reserved workspace.  The paper has no counterpart: this is a
 * service for callers that must not allocate device memory at call time or
 * grow a plan's workspace for a larger batch -- e.g. code whose device memory
 * is handed out entirely by its own pool, where a cudaMalloc would fail or
 * fragment that pool.  The call itself makes no allocation of any kind.
 *   precision  UW_F64 or UW_F32 (UW_F32_SPLIT_BF16: UW_ERR_UNSUPPORTED)
 *   x_dev      device, batch x M^2 coefficients (read only)
 *   y_dev      device, batch x m samples (written; must not overlap x)
 *   batch      >= 1, not limited by the reserved max_batch but by the scratch:
 *              batch x (2 (M/2)^2 + M^2 + 2 M N) elements of the precision
 *              must fit in 8 MiB (e.g. M = 256, N = 512 in FP32: batch <= 5;
 *              M = 512, N = 1024 in FP32: batch 1), else UW_ERR_INVALID_ARG
 *              and nothing is launched
 *   stream     cudaStream_t as void*
 * Errors: UW_ERR_UNSUPPORTED for 1D plans; UW_ERR_INVALID_ARG if the
 * current device is not the plan's device (nothing is looked up or launched);
 * UW_ERR_CUDA if the scratch's device address cannot be found.  The address
 * is looked up once per device and CUDA context (after a device reset the
 * next call looks it up again).
 * All calls on one device share the one scratch array: two calls whose
 * kernels can overlap (different streams, or different host threads without
 * ordering) race on it and give wrong results; order them on one stream.
 * The first call on each device does the one-time address lookup, which may
 * load the library's GPU code: make it before any stream capture begins.
 */
int uw_forward_noalloc(const uw_plan* plan, int precision, const void* x_dev, void* y_dev,
                       int batch, void* stream);

/*
 * uw_forward_host / uw_adjoint_host -- the same products on HOST buffers:
 * the input is copied to the plan's device staging area, the product runs on
 * `stream`, the result is copied back; the call returns once the result is in
 * host memory (it synchronises `stream`, after waiting for the plan's
 * asynchronous host calls).  Staging is part of the reserved workspace.
 */
int uw_forward_host(const uw_plan* plan, int precision, const void* x_host, void* y_host,
                    int batch, void* stream);
int uw_adjoint_host(const uw_plan* plan, int precision, const void* y_host, void* x_host,
                    int batch, void* stream);

/*
 * uw_forward_host_async / uw_adjoint_host_async -- the host-buffer products,
 * stream-ordered, for a sequence of instances whose copies overlap the
 * products.  Each call takes the next of two device staging slots:
 *   1. the input is copied host -> device on the plan's upload stream (after
 *      the product that last read that slot is done);
 *   2. the product runs on `stream` once that copy is done (and once the
 *      download that last read the slot's output is done);
 *   3. the result is copied device -> host on the plan's download stream once
 *      the product is done.
 * The call returns as soon as this is enqueued.  The upload of call k+1 and
 * the download of call k-1 therefore run while the product of call k runs.
 * Products run in call order (they share the plan's workspace).
 *
 * The product of step 2 is launched as a CUDA graph: the first call for a
 * (direction, precision, slot) captures it on a stream of the plan's own and
 * later calls replay it.  A call captures anew when anything the graph was
 * built from differs: the batch, the mask, the coarsest level, the reserved
 * buffers, membership of a plan group, the group tuner's kernel choice, or
 * the UW_* launch switches in the environment.  While the per-kernel
 * profiler is on (uw_plan_profile), or if the driver refuses the capture,
 * the kernels are launched one by one as by uw_forward / uw_adjoint.  The
 * first call of each kind therefore costs a capture: make it before
 * timing, and not while another capture is active on this thread.
 *
 * Host buffers must be pinned for the copies to be asynchronous.  They must
 * stay valid until uw_host_wait returns: inputs unchanged, outputs not read.
 * The same input buffer may be passed to several calls.
 *
 * Errors: the same argument checks as uw_forward_host (UW_ERR_INVALID_ARG);
 * UW_ERR_OOM if the plan's copy or capture streams or events cannot be
 * created; UW_ERR_CUDA if a copy or the graph launch cannot be enqueued.
 */
int uw_forward_host_async(const uw_plan* plan, int precision, const void* x_host, void* y_host,
                          int batch, void* stream);
int uw_adjoint_host_async(const uw_plan* plan, int precision, const void* y_host, void* x_host,
                          int batch, void* stream);

/*
 * uw_host_wait -- block until every result of the plan's asynchronous host
 * calls is in host memory.  Returns UW_ERR_CUDA if a copy or product failed.
 */
int uw_host_wait(const uw_plan* plan);

/*
 * Plan groups -- many independent products (any mix of d, R, q, p, boundary
 * and masks) issued as one unit, e.g. to be captured into one CUDA graph.
 *
 * uw_group_create(plans, n, nstreams): a group over n existing plans (still
 *   owned by the caller; they must outlive the group).  A plan owns one
 *   workspace, so it may appear at most once in a group and belong to at
 *   most one live group: a repeated plan, or one already in another group,
 *   gives NULL with UW_ERR_INVALID_ARG.  While the group
 *   exists, its plans run their coarse 2D levels as one launch per level
 *   (kernels of different instances may then run at the same time; no grid-
 *   wide barrier is shared between them); uw_group_destroy restores the plans'
 *   launch choices.  nstreams in [1, 64]: internal streams.  NULL on error.
 * uw_group_forward / uw_group_adjoint(g, precision, in, out, stream): the
 *   product of instance i on device buffers in[i] -> out[i] (batch 1 each,
 *   layouts as uw_forward / uw_adjoint).  The instances are spread round-robin
 *   over the group's streams, forked from `stream` by an event and joined
 *   back into it, so work later on `stream` sees every result and a capture of
 *   `stream` records one graph with nstreams parallel branches.
 * uw_group_tune(g, precision, x, y, reps, stream): for every instance, times
 *   reps forward + adjoint pairs (on x[i] -> y[i] -> x[i], which it
 *   overwrites) with each line-operator variant the plan supports -- the
 *   specialised kernels that apply to its sizes, or the generic ones -- and
 *   keeps the fastest for that plan.  Synchronises `stream`.
 * FP32 products of a group of 2D plans (M >= 64, at most 1024 instances) run
 *   as ONE persistent launch: a grid of CTAs drains a device-side queue of
 *   tasks (instance, phase, run of items), phase by phase across all
 *   instances; the phases of one instance are the coarse Mallat levels (rows,
 *   then columns, one line per item), the transposes (32 x 32 tiles) and the
 *   two line passes (one line per item).  A task waits, bounded, until the
 *   previous phase of its instance has counted all its items; a wait that gives
 *   up is reported by uw_group_device_status.  Other precisions, or groups that
 *   do not qualify, use the forked streams.
 * uw_group_tune_cached(g, precision, x, y, reps, cache_path, stream): as
 *   uw_group_tune, and for FP32 groups on the persistent launch it also times
 *   the launch's parameters (items per task of the line, coarse-level and
 *   transpose phases; largest radix of the shared-memory Walsh-Hadamard
 *   passes, 16 or 8; CTAs per SM) and the forked streams, and keeps the
 *   fastest.  cache_path (may be NULL): a JSON file of choices keyed by GPU
 *   name, dimension, the instances' N values and precision; a hit skips the
 *   timing, a miss adds the entry.
 * uw_group_params(g, out7): out7[0] 1 if the persistent launch is available,
 *   out7[1] 1 if it is in use for FP32, out7[2..6] its parameters (items per
 *   task of line / coarse / transpose phases, radix, CTAs per SM, 0 = as many
 *   as fit).
 * uw_group_device_status(g): waits for the device and returns
 *   UW_ERR_TIMEOUT (and clears it) if a bounded wait of the persistent launch
 *   gave up since the last query; the affected results are invalid.
 * Errors: UW_ERR_INVALID_ARG (null pointers, n < 1, nstreams out of range,
 *   precision, a plan's own argument checks), UW_ERR_OOM (streams or events),
 *   UW_ERR_CUDA; a failing instance stops the call with its status (the
 *   internal streams are still joined back into `stream`, so a capture of
 *   `stream` can end).
 */
typedef struct uw_group uw_group;
uw_group* uw_group_create(uw_plan* const* plans, int n, int nstreams);
int uw_group_forward(uw_group* group, int precision, const void* const* x, void* const* y, void* stream);
int uw_group_adjoint(uw_group* group, int precision, const void* const* y, void* const* x, void* stream);
int uw_group_tune(uw_group* group, int precision, void* const* x, void* const* y, int reps, void* stream);
int uw_group_tune_cached(uw_group* group, int precision, void* const* x, void* const* y, int reps,
                         const char* cache_path, void* stream);
int uw_group_params(const uw_group* group, int* out7);
int uw_group_device_status(uw_group* group);
void uw_group_destroy(uw_group* group);

/*
 * Solver kernels (element-wise, no plan): the pieces of an l1-regularised
 * recovery  min_x 1/2 ||P_Omega U x - y||^2 + lam ||x||_1  (the
 * compressive-sensing use of the products, Sec. 1.2 and Remark 4.2) that are
 * not products with U: FISTA's proximal step with momentum, its
 * vector-Jacobian product for back-propagation through the iterations, and
 * FP64-accumulated inner products.  precision: UW_F32 or UW_F64 (every array
 * of that type, device memory, n elements each); stream: cudaStream_t.
 *
 * uw_fista_step:  v = z - tau (G - B),  x1 = sign(v) max(|v| - tau lam, 0),
 *                 z1 = x1 + beta (x1 - x0).
 *   With G = U^* P_Omega^* P_Omega U z and B = U^* P_Omega^* y this is one
 *   FISTA iteration with step tau (tau <= 1: ||P_Omega U|| <= 1) and
 *   momentum beta.  x1, z1 must not overlap the inputs.
 */
int uw_fista_step(int precision, int64_t n, const void* z, const void* G, const void* B, const void* x0,
                  double tau, double lam, double beta, void* x1, void* z1, void* stream);

/*
 * uw_fista_step_backward -- given gx1 = dL/dx1 and gz1 = dL/dz1 (either may
 * be NULL: zero), writes dL/dz (gz), dL/dG (gG), dL/dB (gB) and dL/dx0 (gx0,
 * skipped if NULL), and ADDS dL/dlam to the device double *glam (the caller
 * zeroes it; accumulated in FP64).  On the active set |v| > tau lam the step
 * passes w = gx1 + (1 + beta) gz1 to v; elsewhere nothing.
 */
int uw_fista_step_backward(int precision, int64_t n, const void* z, const void* G, const void* B, double tau,
                           double lam, double beta, const void* gx1, const void* gz1, void* gz, void* gG,
                           void* gB, void* gx0, double* glam, void* stream);

/* uw_dot -- *out (device double) = sum_i a_i b_i accumulated in FP64. */
int uw_dot(int precision, int64_t n, const void* a, const void* b, double* out, void* stream);

/* uw_axpby -- out = alpha a + beta b (b may be NULL: out = alpha a). */
int uw_axpby(int precision, int64_t n, double alpha, const void* a, double beta, const void* b, void* out,
             void* stream);

/* uw_plan_destroy -- frees the plan's device and host memory; NULL is a
 * no-op.  The caller must make sure no call using the plan is in flight. */
void uw_plan_destroy(uw_plan* plan);

/* Introspection for tests: copy the host tables into `out` (capacity `cap`
 * doubles); returns the number of doubles the table has (call with cap = 0
 * to size).  which: 0 = h, 1 = cell integrals I_q[t] for t from (-p+1) 2^q,
 * 2 = left edge cell rows (p x (2p-1) 2^q), 3 = right edge cell rows,
 * 4 = left scaling block P_L (p x (3p-1)), 5 = Q_L, 6 = P_R, 7 = Q_R. */
int64_t uw_plan_table(const uw_plan* plan, int which, double* out, int64_t cap);

/* uw_host_table -- the same tables computed on the host only (no CUDA call):
 * what uw_plan_create would upload for (p, q).  Same `which` codes and return
 * convention as uw_plan_table; -1 on invalid p or q. */
int64_t uw_host_table(int p, int q, int which, double* out, int64_t cap);

/* uw_plan_profile -- enable (1) or disable (0) per-kernel timing: while
 * enabled every launch of the plan is bracketed by two CUDA events recorded
 * on the launching stream (no extra synchronisation).  Enabling resets the
 * totals.  Not part of the paper: measurement support. */
int uw_plan_profile(uw_plan* plan, int enable);

/* uw_plan_profile_read -- synchronises the recorded events and reports
 * entry i: kernel name (NUL-terminated, at most cap bytes), total device time
 * in ms, number of launches, and the algorithmic bytes of one launch (each
 * input read once, each output written once).  Returns the number of entries
 * (call with i = -1 to size); 0 if profiling was never enabled. */
int uw_plan_profile_read(uw_plan* plan, int i, char* name, int cap, double* total_ms,
                         int64_t* launches, double* bytes_per_launch);

/*
 * uw_plan_device_status -- waits for the device (cudaDeviceSynchronize on the
 * plan's device) and reports whether a bounded device-side wait of the plan
 * gave up since the last query: the 2D products run all coarse wavelet levels
 * in one cooperative launch whose CTAs meet at grid barriers between levels;
 * each wait polls a bounded number of times (environment variable
 * UW_BARRIER_SPIN_LIMIT, default 2^22 polls with a 32 ns sleep after each)
 * and then records the failure and returns.  Returns UW_OK, UW_ERR_TIMEOUT (the results of the
 * calls since the last query are invalid; the barrier is reset for the next
 * call) or UW_ERR_CUDA (a CUDA error surfaced while synchronising).  Not part
 * of the paper: failure reporting of this implementation.
 */
int uw_plan_device_status(uw_plan* plan);

/* Number of kernel launches the last uw_forward / uw_adjoint issued. */
int uw_plan_last_launches(const uw_plan* plan);

int uw_last_error(void);
const char* uw_last_message(void);
const char* uw_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* UW_H */
