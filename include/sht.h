/*
 * sht.h -- C ABI of the GB300 IDBF associated-Legendre / spherical-harmonic
 * transform library (libsht.so).
 *
 * Method: Bremer, Chen & Yang, "Rapid Application of the Spherical Harmonic
 * Transform via Interpolative Decomposition Butterfly Factorization",
 * arXiv:2004.11346.  Section, equation and algorithm numbers below refer to it.
 *
 * Conventions for every entry point
 *  - N is the transform order: degrees k = 0..2N-1, orders |m| <= 2N-1,
 *    2N Gauss-Legendre nodes x_0 < ... < x_{2N-1} in x = cos(theta) and
 *    M = 4N-1 equispaced phi_j = 2 pi (j + 1/2) / M (Sec. 1, the grid).
 *  - Pbar_k^m is L2-normalised on [-1, 1] with no Condon-Shortley phase.
 *  - Complex numbers are interleaved (re, im) doubles.
 *  - Orders are stored in the sequence m = 0, 1, -1, 2, -2, ..., 2N-1, -(2N-1).
 *      coefficients beta : per field 4N^2 complex; for each order the degrees
 *                          k = |m|..2N-1 are contiguous (first coefficient of
 *                          order m > 0 at 2N(2m-1) - m(m-1); of -m right after
 *                          the 2N-m coefficients of +m).
 *      ALT values g      : per field (4N-1) x 2N complex; row = order in the
 *                          sequence above, column = node index l (ascending x).
 *      grid values f     : per field 2N x (4N-1) complex, theta-major.
 *    F fields are stored one after another (field stride = the per-field size).
 *    F = 0 is a no-op, and the data pointers may then be NULL.
 *  - Data pointers are DEVICE pointers owned by the caller, unless the entry
 *    point says otherwise.  Inputs are never modified.  Outputs must not
 *    overlap inputs.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream: the return value reports
 *    argument and launch errors; errors detected by the device are latched in
 *    the plan and returned by the next call or by sht_sync().
 *  - No entry point falls back to the CPU: without a usable CUDA device the
 *    library returns SHT_ERR_CUDA.
 */
#ifndef SHT_H_
#define SHT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sht_plan_s* sht_plan_t;

typedef enum {
  SHT_OK = 0,
  SHT_ERR_ARG = 1,      /* invalid argument (N, eps, m, F, NULL pointer...) */
  SHT_ERR_OOM = 2,      /* host or device allocation failed                 */
  SHT_ERR_CUDA = 3,     /* CUDA runtime error or no device                  */
  SHT_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up               */
  SHT_ERR_NUMERIC = 5,  /* precomputation failed to reach the tolerance     */
  SHT_ERR_IO = 6,       /* plan file missing, truncated or corrupt          */
  SHT_ERR_UNSUPPORTED = 7
} sht_status;

typedef enum {
  SHT_FP64 = 0,        /* factors and arithmetic in FP64                        */
  SHT_FP32 = 1,        /* factors and arithmetic in FP32 (FP64 I/O)             */
  SHT_MIXED = 2        /* every block product (IDBF levels, low-rank factors and
                          the dense turning-point blocks) on the tensor cores as
                          split-BF16 (3 pieces) with FP32 accumulation; FP64
                          only in the precomputation and the FP64 I/O.  Measured
                          relative error against the FP64 definition: about
                          2e-7 per field at eps = 1e-7, N = 1024               */
} sht_precision;

/* Plan options (Sec. 2.1, 2.3, 3.2, 3.3 and Sec. 5's parameter choices). */
typedef struct {
  double eps;          /* ID / rSVD truncation tolerance, absolute on the scale
                          of the largest matrix entry (Sec. 2.1)               */
  int n0;              /* partition stops once a turning-point block has fewer
                          than n0 rows or columns (Sec. 3.2)                   */
  int n_leaf;          /* IDBF leaf size: depth L = floor(log2(min dim/n_leaf)) */
  int r_k;             /* adaptive-rank bound of the ID (Sec. 2.1)              */
  double oversample;   /* t: the ID samples t * r_k rows (Sec. 2.1)             */
  int rsvd_r;          /* initial rank of the randomized SVD (Sec. 5: 30)       */
  int rsvd_q;          /* its oversampling factor q (Sec. 2.3: 2)               */
  double trim_delta;   /* entries below trim_delta are negligible (Sec. 3.3)    */
  int sampling;        /* 0 = mock-Chebyshev rows, 1 = random rows (Sec. 2.1)   */
  int precision;       /* sht_precision                                          */
  int max_fields;      /* workspace sized for this many fields per call          */
  int flags;           /* SHT_FLAG_* bits                                        */
  uint64_t seed;       /* seed of the randomized choices                         */
} sht_opts;

/* sht_opts.flags */
#define SHT_FLAG_FORCE_FACTOR 1 /* keep factored blocks even when larger than dense */
#define SHT_FLAG_HOST_ONLY 2    /* build the program on the host only: no device
                                   upload; apply calls return SHT_ERR_UNSUPPORTED */
#define SHT_FLAG_DENSE 4        /* no partition, trimming or factorisation: every
                                   parity matrix is applied dense (the O(N^3)
                                   transform, kept as a baseline)                */
#define SHT_FLAG_TIMING 8       /* record CUDA events around every apply kernel
                                   launch (see sht_plan_kernel_time)             */
#define SHT_FLAG_GPU_LEGENDRE 32 /* the plan builder takes each order's Legendre
                                   matrices (Sec. 3.1.2) from the device
                                   recurrence of sht_legendre instead of its
                                   host recurrence; the rest of the
                                   precomputation stays on the host.  Values
                                   agree to rounding, so plans can differ from
                                   host-built ones in the last bits.  Not with
                                   SHT_FLAG_HOST_ONLY (SHT_ERR_ARG)            */
#define SHT_FLAG_DIRECT 16      /* no partition and no factorisation, nothing
                                   stored: alt_forward / alt_inverse (and the
                                   full SHT) apply the dense ALT in FP64 with the
                                   Legendre recurrence run on the fly for every
                                   call (O(N^3) work, any N up to 16384 whose
                                   per-CTA scratch fits, about 16 N^2 bytes per
                                   SM); the phi transform as for other plans.
                                   Single-order calls, batches, the no-allocation
                                   entry point and save return
                                   SHT_ERR_UNSUPPORTED.  Not with
                                   SHT_FLAG_HOST_ONLY (SHT_ERR_ARG)            */

/* Plan statistics (Sec. 5 experiments: block counts, ranks, timings). */
typedef struct {
  int N;
  double eps;
  int64_t n_units;           /* orders |m| = 0..2N-1                            */
  int64_t n_ops;             /* dense block products in the apply program       */
  int64_t n_blocks_idbf, n_blocks_lowrank, n_blocks_dense, n_blocks_dropped;
  int64_t entries_idbf, entries_lowrank, entries_dense; /* stored factor entries */
  int64_t entries_total;
  int64_t entries_matrix;    /* entries of the unfactored parity matrices       */
  int64_t max_rank;          /* largest ID / rSVD rank                          */
  int64_t max_phases;
  int64_t workspace_bytes;
  int64_t factor_bytes;      /* bytes of the factor store in the plan precision */
  double t_factor_s;         /* wall time of the precomputation                 */
  double t_upload_s;         /* wall time of the host->device upload             */
  int threads;               /* host threads used by the precomputation         */
} sht_plan_info;

/* Defaults for order N and tolerance eps (n0, n_leaf scaled with N). */
void sht_opts_default(int N, double eps, sht_opts* out);

/* Build the plan (Sec. 3.2-3.3): Gauss-Legendre rule, Legendre matrices by the
 * three-term recurrence with an extended exponent, block partition along the
 * turning-point curve (Eq. new5, Eq. nb), IDBF of oscillatory blocks (Sec. 2.2),
 * randomized SVD of trimmed non-oscillatory blocks (Alg. 1), trimmed dense
 * turning-point blocks; then upload the packed factors to the current device.
 * N >= 1, eps in (0, 1).  opts may be NULL (defaults).  The plan owns all of
 * its host and device memory until sht_plan_destroy. */
sht_status sht_plan_create(int N, double eps, const sht_opts* opts, sht_plan_t* out);
sht_status sht_plan_destroy(sht_plan_t plan);
sht_status sht_plan_stats(sht_plan_t plan, sht_plan_info* out);

/* The plan's Gauss-Legendre nodes and weights (2N each, ascending), copied to
 * HOST arrays owned by the caller. */
sht_status sht_plan_nodes(sht_plan_t plan, double* x_host, double* w_host);

/* One order's factorisation built on its own (host only, no device needed):
 * the per-order experiments of Sec. 5, and a way to size a plan for a large N
 * from a sample of its orders before building it.  Every field describes
 * exactly what sht_plan_create(N, eps, opts) builds at that order. */
typedef struct {
  int N;
  int am;                    /* |m|                                             */
  int64_t cols_even, cols_odd; /* degrees of each parity (N rows each)         */
  int64_t n_blocks_idbf, n_blocks_lowrank, n_blocks_dense, n_blocks_dropped;
  int64_t entries_idbf, entries_lowrank, entries_dense, entries_total;
  int64_t entries_matrix;    /* N * (cols_even + cols_odd)                      */
  int64_t factor_doubles;    /* the order's FP64 factor store, padding included */
  int64_t image_elems;       /* BF16 elements of the order's tensor-core operand
                                images, both directions (SHT_MIXED plans)       */
  /* the tensor-core kernel's work for one forward apply of one 32-field group:
   * pipeline stages (128-row tiles x 32-wide K chunks), tiles, bytes of the
   * forward operand images and of the activation row groups the stages copy */
  int64_t tc_stages, tc_tiles, tc_image_fwd_bytes, tc_act_bytes;
  int64_t max_rank;
  int64_t n_ops;             /* block products of the order's apply program     */
  int64_t n_phases;
  int64_t rows;              /* rows of the order's vector space                */
  double flops_per_rhs;      /* the schedule's cost estimate                    */
  double t_mat_s;            /* building the two Legendre matrices (recurrence) */
  double t_fac_s;            /* partition, IDs / IDBF / rSVD, trimming, packing */
} sht_order_info;

/* Build the orders m[0..count) (each in [-(2N-1), 2N-1]; -m and m are one
 * order) of the plan sht_plan_create(N, eps, opts) would build, one host
 * thread per order, and describe each in out[0..count) (HOST array owned by
 * the caller).  The factors are discarded.  SHT_ERR_ARG for an argument
 * sht_plan_create would refuse, count < 0, or an order out of range;
 * SHT_ERR_OOM when host memory runs out. */
sht_status sht_order_stats(int N, double eps, const sht_opts* opts, int count, const int* m, sht_order_info* out);

/* Forward ALT of F fields (Eq. sht_lt, Sec. 3.1.2 parity split and fold):
 *   g(m, theta_l) = sum_{k=|m|}^{2N-1} beta_{k,m} Pbar_k^{|m|}(x_l)
 * for every order.  beta: F x 4N^2 complex, g: F x (4N-1) x 2N complex. */
sht_status alt_forward(sht_plan_t plan, const double* beta, double* g, int F, void* stream);

/* Inverse ALT of F fields (Sec. 3.1.1, B = A^T W):
 *   beta_{k,m} = sum_l w_l Pbar_k^{|m|}(x_l) g(m, theta_l). */
sht_status alt_inverse(sht_plan_t plan, const double* g, double* beta, int F, void* stream);

/* The same for one order m in [-(2N-1), 2N-1]: beta_m holds F x (2N-|m|)
 * complex coefficients (degrees |m|..2N-1), g_m holds F x 2N complex values. */
sht_status alt_forward_m(sht_plan_t plan, int m, const double* beta_m, double* g_m, int F, void* stream);
sht_status alt_inverse_m(sht_plan_t plan, int m, const double* g_m, double* beta_m, int F, void* stream);

/* phi direction of the SHT (Eq. sht_fft), for every node and field:
 *   synthesis f(theta_l, phi_j) = sum_{m=-(2N-1)}^{2N-1} g(m, theta_l) e^{i m phi_j},
 *   analysis  g(m, theta_l) = (1/M) sum_j f(theta_l, phi_j) e^{-i m phi_j},
 * phi_j = 2 pi (j + 1/2) / M, M = 4N-1 (exact inverse of each other).  g as
 * for alt_forward (F x (4N-1) x 2N complex), f theta-major (F x 2N x (4N-1)).
 * Arithmetic in FP64 for FP64 plans, else FP32.  Each length-M row is
 * transformed in the shared memory of one CTA, or spread over a cluster of up
 * to 8 CTAs when it is longer; SHT_ERR_UNSUPPORTED when it does not fit 8 CTAs
 * (FP64: M up to about 116,000 values, half that when M has a prime factor
 * above 13, e.g. N = 16384: M = 65535 = 3 5 17 257 is refused in FP64). */
sht_status sht_phi_synthesis(sht_plan_t plan, const double* g, double* f, int F, void* stream);
sht_status sht_phi_analysis(sht_plan_t plan, const double* f, double* g, int F, void* stream);

/* Full SHT (Eq. sht_re): forward = forward ALT then phi synthesis,
 * coefficients beta (F x 4N^2) -> grid values f (F x 2N x (4N-1));
 * inverse = phi analysis then inverse ALT.  The ALT values pass through the
 * plan's workspace, max_fields fields at a time. */
sht_status sht_forward(sht_plan_t plan, const double* beta, double* f, int F, void* stream);
sht_status sht_inverse(sht_plan_t plan, const double* f, double* beta, int F, void* stream);

/* Copy one of the plan's host-side program arrays into dst_host (caller-owned,
 * *bytes long); with dst_host == NULL only *bytes is set to the size needed.
 * Layouts are those of the library's internal program (units, ops, phase
 * table, packed FP64 factors, schedule) and the plan's sht_opts; used to
 * inspect the factorisation. */
typedef enum {
  SHT_EXPORT_UNITS = 0,
  SHT_EXPORT_OPS = 1,
  SHT_EXPORT_PHASES = 2,
  SHT_EXPORT_FACTORS = 3,
  SHT_EXPORT_ORDER = 4,
  SHT_EXPORT_OPTS = 5,
  SHT_EXPORT_UNIT_BLOCKS = 6  /* per order |m|: int32 counts of IDBF, low-rank, dense and dropped
                                blocks (Sec. 5's block counts); empty for plans read from files */
} sht_export_kind;
sht_status sht_plan_export(sht_plan_t plan, int what, void* dst_host, size_t* bytes);

/* The tensor-core operand image of op `op` of the program (the index into
 * SHT_EXPORT_OPS), for inspection; the paper has no counterpart.  The image is
 * what the SHT_MIXED kernel streams: the op's block B (transposed != 0: B^T),
 * split into three BF16 pieces b0 + b1 + b2 (piece p the rounding of what
 * pieces 0..p-1 leave), in tiles of 128 rows x chunks of 32 K columns, each
 * chunk piece by piece in 8 x 8 core matrices (K-outer).  The K side is
 * widened to whole 8-row groups of the vector space, with zero columns where
 * it was widened.  Copies `*count` BF16 values into dst_host (caller-owned);
 * with dst_host == NULL only *count is set.  Works for host-only plans too. */
sht_status sht_plan_op_image(sht_plan_t plan, int64_t op, int transposed, uint16_t* dst_host, size_t* count);

/* Save the plan's precomputation (Sec. 3.2-3.3: nodes, weights, the block
 * factorisation as the packed apply program, options and statistics) to a
 * file, so that later processes skip the factorisation.  The file is written
 * in native byte order with a 64-bit checksum.  SHT_ERR_IO when the file
 * cannot be written. */
sht_status sht_plan_save(sht_plan_t plan, const char* path);

/* Load a plan written by sht_plan_save and upload it to the current device
 * (host-only plans stay host-only).  The file is checked (magic, version,
 * struct sizes, checksum, and the same consistency check every built program
 * passes: unit layouts, op ranges, factor offsets, schedule; statistics that
 * describe that program) before anything reaches the GPU, and no array is
 * allocated larger than the rest of the file could hold: SHT_ERR_IO for a
 * missing, damaged or foreign file, SHT_ERR_CUDA without a device.  The
 * caller owns the new plan. */
sht_status sht_plan_load(const char* path, sht_plan_t* out);

/* Batches of transforms of different orders N in one launch.  Sec. 1 states
 * the SHT for one N; a batch applies several plans (each an order N of its
 * own, e.g. fields of different resolutions) to their own fields at once.  The
 * work items of all plans -- (plan, order |m|, group of 32 fields) -- form one
 * queue in decreasing order of estimated cost, which one persistent launch of
 * the tensor-core kernel works through; each plan's output step follows.
 *  - plans: P distinct SHT_MIXED plans (1 <= P <= 8) on the current device;
 *    fields[q] (>= 0, <= the plan's max_fields) fields go with plans[q].
 *  - The batch owns its work-item table, scratch and counter; it uses each
 *    plan's accumulation rows and ALT-value workspace, so a plan must not run
 *    other calls while a batch that contains it is in flight, and must outlive
 *    the batch (destroy the batch first).
 *  - A batch with no fields at all is valid; its calls do nothing.
 *  - SHT_ERR_UNSUPPORTED for host-only plans or other precisions; SHT_ERR_ARG
 *    for bad counts, repeated plans or plans of another device. */
typedef struct sht_batch_s* sht_batch_t;
sht_status sht_batch_create(int P, const sht_plan_t* plans, const int* fields, sht_batch_t* out);
sht_status sht_batch_destroy(sht_batch_t batch);

/* Forward / inverse ALT of a batch (Eq. sht_lt and Sec. 3.1.1 for each plan).
 * in and out are HOST arrays of P device pointers: plan q's fields[q] fields
 * of beta (F x 4N^2 complex) and g (F x (4N-1) x 2N complex) in the layouts of
 * alt_forward.  Pointers of plans with no fields may be NULL. */
sht_status alt_forward_batch(sht_batch_t batch, const double* const* beta, double* const* g, void* stream);
sht_status alt_inverse_batch(sht_batch_t batch, const double* const* g, double* const* beta, void* stream);

/* Full SHT of a batch (Eq. sht_re for each plan): the batched ALT, then each
 * plan's phi-direction transform (as sht_forward / sht_inverse). */
sht_status sht_forward_batch(sht_batch_t batch, const double* const* beta, double* const* f, void* stream);
sht_status sht_inverse_batch(sht_batch_t batch, const double* const* f, double* const* beta, void* stream);

/* Wait for a batch's work on `stream`; SHT_ERR_TIMEOUT if a bounded device
 * wait gave up. */
sht_status sht_batch_sync(sht_batch_t batch, void* stream);

/* alt_forward_m without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory (a memory
 * pool or arena that owns the device, real-time loops where cudaMalloc/cudaFree
 * would synchronise the device, embedders with their own allocator).  It runs
 * the alt_forward_m computation with its scratch (per-CTA vectors and the
 * work counter) in a fixed 8 MiB array inside the library's device image
 * instead of the plan's workspace, and calls no allocating routine.
 *  - Every GPU that loads libsht.so holds that array until the process exits.
 *  - sht_plan_create / sht_plan_load look the array's device address up
 *    (cudaGetSymbolAddress, with the plan's device current) and keep it in
 *    the plan, so this call does no set-up of its own.  The plan must belong
 *    to the current device, in the context it was created in (a plan does not
 *    survive cudaDeviceReset).
 *  - Plans created with SHT_FLAG_TIMING count its launches in
 *    sht_plan_kernel_time like those of the other apply calls.
 *  - FP64 plans only (SHT_ERR_UNSUPPORTED otherwise: the other precisions do
 *    not keep the FP64 factor store on the device).
 *  - Returns SHT_ERR_ARG when one work item's vectors (the plan's largest
 *    order: rows x 4 doubles) do not fit in the array; otherwise the result is
 *    that of alt_forward_m, with fewer CTAs.
 *  - All calls share the array and it keeps the last call's contents: calls
 *    that may overlap on the GPU race on it and must be serialised. */
sht_status alt_forward_m_noalloc(sht_plan_t plan, int m, const double* beta_m, double* g_m, int F, void* stream);

/* Device time of the plan's apply kernels, for plans created with
 * SHT_FLAG_TIMING (instrumentation; the paper has no counterpart).  Every
 * alt_* call then records CUDA events on its stream around each kernel it
 * launches; this call waits for them and returns, summed over the launches
 * since the last reset (at most the latest 256):
 *  - apply_ms: the block-product kernels (for SHT_MIXED the pre-gather
 *    kernel of the inputs and the tensor-core kernel after it; the whole
 *    apply for SHT_FP64 / SHT_FP32 and direct plans),
 *  - output_ms: the tensor-core path's output kernel (the forward's parity
 *    fold; 0 for the inverse, whose scatter to beta the tensor-core kernel
 *    does as each work item finishes, and for the other precisions),
 *  - launches: the number of launches summed.
 * reset != 0 starts a new sum.  SHT_ERR_UNSUPPORTED without the flag. */
sht_status sht_plan_kernel_time(sht_plan_t plan, int reset, double* apply_ms, double* output_ms, int64_t* launches);

/* Pause (enable = 0) or resume (enable != 0) the event recording of a plan
 * created with SHT_FLAG_TIMING (instrumentation; the paper has no
 * counterpart), e.g. so that a timed loop runs without the extra events and a
 * separate pass collects the per-kernel split.  Launches made while paused
 * are not counted by sht_plan_kernel_time.  SHT_ERR_UNSUPPORTED without the
 * flag. */
sht_status sht_plan_set_timing(sht_plan_t plan, int enable);

/* Self-test of the failure detection (the paper has no counterpart).  Every
 * wait inside the tensor-core kernel is bounded (about a second); when one
 * runs out the kernel stops all its roles, releases its tensor memory, and
 * flags the plan, so that the next sht_sync returns SHT_ERR_TIMEOUT and the
 * plan stays usable.  This call launches that kernel with its item warps
 * publishing no work item, so that the other roles' first waits run out:
 * after it, sht_sync must return SHT_ERR_TIMEOUT.  SHT_MIXED plans only
 * (SHT_ERR_UNSUPPORTED otherwise).  Takes a second or more of GPU time. */
sht_status sht_selftest_timeout(sht_plan_t plan, void* stream);

/* Pbar_k^{|m|}(x_{N+i}) for one order on the device (Sec. 1, the normalised
 * associated Legendre functions without Condon-Shortley phase; the recurrence
 * of Sec. 3's matrices): out[t * N + i] = Pbar_{am+t}^{am}(x_{N+i}) for
 * t < 2N - am, i < N, at the plan's N positive Gauss-Legendre nodes
 * (ascending).  Three-term recurrence in FP64 from Pbar_am^am, carried with a
 * separate binary exponent below the FP64 range; values below 2^-760 are
 * written as 0.  out: caller-owned device array of (2N - am) N doubles.
 * Asynchronous on the stream.  SHT_ERR_ARG for a bad am or NULL out;
 * SHT_ERR_UNSUPPORTED for host-only plans. */
sht_status sht_legendre(sht_plan_t plan, int am, double* out, void* stream);

/* The order in which the apply's persistent CTAs take the orders |m| from
 * the work queue (the m-to-CTA schedule; the paper has no counterpart, one
 * order is one independent ALT, Eq. sht_fft): order[q] = |m| of the q-th
 * unit, a permutation of 0 .. 2N-1 (each field group of a unit follows it).
 * Plans start with the orders by decreasing modelled cost; any permutation
 * gives the same results.  Host array, copied; the plan is synchronised
 * first, so no call on it may be in flight.  SHT_ERR_ARG unless n = 2N and
 * order is a permutation; SHT_ERR_UNSUPPORTED for direct plans. */
sht_status sht_plan_set_order(sht_plan_t plan, const int32_t* order, int n);

/* Self-test of the binary64 <-> binary32 conversions that the FP32 and
 * tensor-core paths apply to every input and output value (integer
 * arithmetic, round to nearest even, subnormals, infinities and NaN per IEEE
 * 754; the paper has no counterpart): f32[i] = (float)f64[i] and
 * back[i] = (double)f32[i], i < n.  Device pointers, caller-owned;
 * SHT_ERR_ARG for n < 0 or a NULL pointer with n > 0. */
sht_status sht_selftest_convert(const double* f64, float* f32, double* back, int64_t n, void* stream);

/* Wait for the plan's work on `stream` and return any latched device error. */
sht_status sht_sync(sht_plan_t plan, void* stream);

const char* sht_status_str(sht_status s);

#ifdef __cplusplus
}
#endif

#endif /* SHT_H_ */
