/*
 * taser.h -- C ABI of the GB300 (sm_103a) TASER detector library (libtaser.so).
 *
 * TASER (Triangular Approximate SEmidefinite Relaxation; Castaneda, Goldstein, Studer,
 * arXiv:1609.01797) detects BPSK/QPSK symbols of many independent problems at once:
 * coherent MU-MIMO (Sec. II-A) and SIMO joint channel estimation and detection (JED,
 * Sec. II-B).  Every entry point works on a batch of independent instances.
 *
 * Conventions shared by all entry points
 *   - Array arguments are DEVICE pointers owned by the caller unless stated otherwise.
 *     The library never allocates, frees or keeps them.
 *   - Calls are asynchronous and ordered on `stream` (a cudaStream_t passed as void*;
 *     NULL means the legacy default stream).  A returned TASER_OK means the work was
 *     enqueued; kernel-side numeric trouble is reported through the per-instance flag
 *     bits below, never as a global failure.
 *   - Invalid arguments return TASER_ERR_INVALID_ARG before anything is launched.
 *     Array pointers must be 16-byte aligned.  batch == 0 is a valid no-op.
 *   - TASER_ERR_CUDA carries the CUDA error seen at launch; taser_last_error() returns
 *     its text (thread-local).
 *   - Matrices are row-major per instance and instances are contiguous:
 *     element (i, j) of instance b of an [batch][N][N] array is at b*N*N + i*N + j.
 *   - The last index N-1 of every real-valued problem is the augmented "1" coordinate
 *     (MIMO) or the pilot slot (JED); decisions are returned for indices 0..N-2.
 */
#ifndef TASER_H
#define TASER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TASER_OK = 0,
    TASER_ERR_INVALID_ARG = 1,
    TASER_ERR_UNSUPPORTED = 2,
    TASER_ERR_CUDA = 3,
    TASER_ERR_TIMEOUT = 4,
    TASER_ERR_NUMERIC = 5
} taser_status;

/* Problem kinds (Sec. II).  N is the size of the real-valued matrix T. */
typedef enum {
    TASER_MIMO_BPSK = 0,     /* N = U + 1,  H complex64 [batch][B][U], y [batch][B]      */
    TASER_MIMO_QPSK = 1,     /* N = 2U + 1, same inputs                                  */
    TASER_SIMO_JED_BPSK = 2, /* N = K,      Y complex64 [batch][B][K], slot 0 = +1 pilot */
    TASER_SIMO_JED_QPSK = 3  /* N = 2K - 1, Y complex64 [batch][B][K], slot 0 = (1+j)/sqrt2
                                pilot; data slots use the effective Y_r/sqrt2 (Sec. II-B) */
} taser_problem;

/* Arithmetic of the iterations.  For the first three the triangular product L~ T^
 * runs at the named precision while the prox (column norms and rescaling) and the
 * master copy of L~ stay FP32.  TASER_FIXED14 is the 14-bit fixed-point datapath of
 * the paper's VLSI designs (Sec. IV-B operation modes, Sec. IV-D fixed-point
 * parameters and inverse square-root LUT), computed exactly in integer arithmetic:
 *   - L~ and V carry 8 fraction bits, 7 in row N; L~_NN is a constant register with 5
 *     (so only TASER_LNN_FIXED exists; TASER_LNN_LITERAL returns TASER_ERR_UNSUPPORTED);
 *   - T^ = 2 tau T~ has 12 fraction bits, quantised from the FP32 product fl(2 tau) T~_ij;
 *     D_j has 8, D_N 5;
 *   - every format saturates to [-2^13, 2^13 - 1] (TASER_FLAG_SATURATED) and rounds
 *     half up; the MAC and the squared column norms are exact;
 *   - 1/||v_j|| comes from a 2^11-entry LUT (13 fraction bits) indexed by the top 11
 *     bits of the normalised squared norm, LUT[i] = round(2^13 / sqrt((i + 1/2)/512)).
 * The results (L~ codes scaled to floats, decisions, flags) are bit-exact and do not
 * depend on the GPU or the launch shape. */
typedef enum {
    TASER_FP32 = 0,      /* FP32 FMA pipe                                              */
    TASER_BF16_TC = 1,   /* tensor cores, BF16 operands, FP32 accumulation             */
    TASER_FP16_TC = 2,   /* tensor cores, FP16 operands, FP32 accumulation; the operands
                            are L~ (|L~_ik| <= D_kk) and -2 tau T~ (|.| <= 2 alpha), so D must
                            stay inside FP16's normal range (about 1e-4 .. 6e4); BF16 has
                            FP32's range                                                */
    TASER_FIXED14 = 3    /* 14-bit fixed point of Sec. IV-D, exact integer emulation   */
} taser_precision;

/* Handling of L~_NN (the prox of Sec. III-C applied to the last column). */
typedef enum {
    TASER_LNN_FIXED = 0,   /* default: L~_NN stays +D_NN (last column is constant)       */
    TASER_LNN_LITERAL = 1  /* L~_NN = D_NN sign(V_NN); decisions multiplied by its sign */
} taser_lnn_mode;

/* Per-instance flag bits (uint32). */
#define TASER_FLAG_ZERO_DIAG   (1u << 0) /* some T_kk == 0; D_kk was replaced by 1       */
#define TASER_FLAG_NONFINITE   (1u << 1) /* a non-finite value reached T or its norm     */
#define TASER_FLAG_ZERO_COLUMN (1u << 2) /* a column of V had zero norm in the prox      */
#define TASER_FLAG_LNN_SIGN    (1u << 3) /* V_NN <= 0 was seen in some iteration         */

#define TASER_FLAG_BAD_ITEM    (1u << 4) /* uneven batch: item with N or t_max out of range */
#define TASER_FLAG_SATURATED   (1u << 5) /* TASER_FIXED14: a value saturated to 14 bits    */
#define TASER_FLAG_ASCENT      (1u << 6) /* taser_detect_monitored: the objective rose      */
#define TASER_FLAG_TIMEOUT     (1u << 7) /* a bounded device wait expired: outputs of the
                                            instance are not written                       */

/* Largest N supported by the detection kernels. */
#define TASER_MAX_N 65

/* Size N of the real-valued problem, or -1 for an unknown kind / non-positive size. */
int taser_problem_size(int kind, int U_or_K);

/* Static text of a status code. */
const char* taser_status_string(int status);

/* Thread-local text of the last error reported by this library ("" if none). */
const char* taser_last_error(void);

/*
 * taser_build_T -- per instance, the real-valued matrix T of Sec. II-A (Eq. 2) or
 * Sec. II-B (Eq. 5), its Jacobi preconditioning D = diag(sqrt|T_kk|),
 * T~ = D^-1 T D^-1 (Sec. III-C), and the step size tau = alpha / ||T~||_2
 * (Sec. III-B, inputs of Algorithm 1).
 *
 *   kind      taser_problem.
 *   batch     number of instances (>= 0).
 *   B         receive antennas (>= 1).
 *   U_or_K    users U (MIMO, 1..32) or slots K including the pilot (JED, 2..33).
 *   H_or_Y    complex64 (interleaved re, im float pairs):
 *               MIMO: H [batch][B][U]; JED: Y [batch][B][K] with column 0 the pilot slot.
 *   y         complex64 [batch][B] (MIMO), must be NULL for JED.
 *   alpha     step-size factor, 0 < alpha < 1 (the paper leaves its value open).
 *   T_tilde   out, float [batch][N][N], full symmetric matrix.
 *   D         out, float [batch][N], D_kk = sqrt(|T_kk|) (1 where T_kk == 0).
 *   tau       out, float [batch]; NULL skips the step size (then call
 *             taser_step_size with structure = kind).
 *   spec_norm out, float [batch] = ||T~||_2, or NULL.
 *   flags     out, uint32 [batch] (overwritten with ZERO_DIAG / NONFINITE bits, or with
 *             TIMEOUT alone, see below), or NULL.
 *
 * QPSK with 16 users and an even B stages its antenna rows with the tensor memory
 * accelerator.  Each wait for a staged chunk is bounded (about a second of SM clock).  An
 * instance whose wait expires gets TASER_FLAG_TIMEOUT and its T~ and D are left unwritten
 * (tau and spec_norm, computed from them afterwards, are then meaningless for it).  This
 * cannot happen on a healthy device; the debug library's taser_debug_drop_copy provokes it
 * for tests.
 *
 * QPSK symbols are taken as (+-1 +-j)/sqrt2: T is built from the effective channel
 * H/sqrt2 (or Y_r/sqrt2) so that the relaxed vector lies in {+-1}^N.  For JED the pilot
 * column is moved to the last index, so decisions 0..N-2 are slots 1..K-1 (BPSK), or
 * the real parts of slots 1..K-1 followed by their imaginary parts (QPSK, pilot
 * s_0 = (1+j)/sqrt2).
 * ||T~||_2 is the largest |eigenvalue|, from an FP32 Householder tridiagonalisation
 * and Sturm-count multisection (not a power iteration, which converges too slowly on
 * MU-MIMO matrices with nearly equal top eigenvalues).
 */
taser_status taser_build_T(int kind, int64_t batch, int B, int U_or_K,
                           const void* H_or_Y, const void* y, float alpha,
                           float* T_tilde, float* D, float* tau, float* spec_norm,
                           uint32_t* flags, void* stream);

/* Structure of T~ known to taser_step_size (a problem kind, or this value). */
#define TASER_GENERIC_SYMMETRIC (-1)

/*
 * taser_step_size -- tau = alpha / ||T~||_2 for symmetric T~ (Sec. III-B; Algorithm 1
 * inputs), ||T~||_2 = largest |eigenvalue|.
 *   T_tilde   float [batch][N][N] (full), N in [2, 65].
 *   structure what is known about T~, which selects a cheaper exact method:
 *               TASER_MIMO_BPSK      positive semidefinite;
 *               TASER_SIMO_JED_BPSK  negative semidefinite;
 *               TASER_MIMO_QPSK      the real form of a complex Hermitian (U+1) x (U+1)
 *                                    matrix with Im(last) deleted (N = 2U + 1), as built by
 *                                    taser_build_T; ||T~|| is computed on that matrix;
 *               TASER_SIMO_JED_QPSK  the same form, negative semidefinite (N = 2K - 1);
 *               TASER_GENERIC_SYMMETRIC  nothing known.
 *   tau       out float [batch]; spec_norm out float [batch] or NULL.
 */
taser_status taser_step_size(int64_t batch, int N, const float* T_tilde, int structure,
                             float alpha, float* tau, float* spec_norm, void* stream);

/*
 * taser_detect -- Algorithm 1 (TASER) for every instance:
 *   L~(0) = D;  for t = 1..t_max:  V = L~ - tril(2 tau L~ T~),  L~ = prox(V)
 * where prox rescales every column k < N-1 to norm D_kk (Sec. III-C) and the last
 * column follows lnn_mode; outputs s_k = sign(L~_{N,k}), k = 0..N-2, sign(0) = +1.
 *
 *   batch     number of instances (>= 0).
 *   N         problem size, 2..65.
 *   T_tilde   float [batch][N][N], full symmetric preconditioned matrix.
 *   D         float [batch][N], positive scaling (D_kk of Sec. III-C).
 *   tau       float [batch], step size.
 *   t_max     iterations, >= 1.
 *   precision taser_precision.  Tensor-core precisions run for N >= 10; below that the
 *             FP32 kernel runs (the product has no dense tile worth a tensor core).
 *   lnn_mode  taser_lnn_mode.
 *   L         out, float [batch][N][N] = L~(t_max) with zeros above the diagonal, or NULL.
 *   s_hat     out, int8 [batch][N-1], values +1 / -1.
 *   flags     in/out, uint32 [batch]; ZERO_COLUMN / LNN_SIGN bits are OR-ed in; or NULL.
 */
taser_status taser_detect(int64_t batch, int N, const float* T_tilde, const float* D,
                          const float* tau, int t_max, int precision, int lnn_mode,
                          float* L, int8_t* s_hat, uint32_t* flags, void* stream);

/*
 * taser_detect_monitored -- taser_detect that also watches the objective the iterations
 * minimise, f(L~) = Tr(L~ T~ L~^T) (Sec. III-B, Eq. 8 after the preconditioning of
 * Sec. III-C).  Prop. 1 (Sec. III-E) makes forward-backward splitting a descent method
 * for a small enough step: with the Lipschitz constant 2||T~||_2 of the gradient
 * tril(2 L~ T~), that is alpha < 1/2; larger alpha (the paper leaves it open) can make f
 * rise in some iteration.  This call flags such instances.
 *
 * f(L~) is the sum over i >= k of L~_ik (L~ T~)_ik, and the gradient step that starts at
 * L~(t) forms exactly that lower part of L~ T~.  On the FP32 path f(L~(t)) is read off
 * the step itself, sum L~_ik (L~_ik - V_ik) / (2 tau) with V = L~ - 2 tau tril(L~ T~).
 * On the tensor cores a single BF16/FP16 product (operand rounding about 2^-9) is too
 * coarse for a check, so each step also forms L~ T~ as a BF16 split (hi hi + hi lo +
 * lo hi, about 2^-16 relative error) into scratch registers; the iteration itself is
 * unchanged.  The sum of an instance is formed in FP32, the ratio, the comparison and
 * the trace in FP64.  One extra gradient step after the last iteration gives
 * f(L~(t_max)).  L~, s_hat and the other flags are those of taser_detect with the same
 * arguments.
 *
 *   ascent_tol  >= 0: TASER_FLAG_ASCENT is OR-ed into flags[b] when, for some t in
 *               1..t_max, f(L~(t)) > f(L~(t-1)) + ascent_tol |f(L~(t-1))|.  A tolerance of
 *               about 1e-5 (FP32) or 1e-4 (tensor cores) stays above the rounding of f.
 *   objective   out, double [batch][t_max + 1] = f(L~(t)) for t = 0..t_max, or NULL.
 *   other arguments as in taser_detect.  Supported: TASER_FP32 for N in [2, 65];
 *               TASER_BF16_TC / TASER_FP16_TC for N <= 33 (N < 10 runs FP32, as in
 *               taser_detect); TASER_ERR_UNSUPPORTED for the tensor-core bucket N > 33
 *               and for TASER_FIXED14.
 */
taser_status taser_detect_monitored(int64_t batch, int N, const float* T_tilde, const float* D,
                                    const float* tau, int t_max, int precision, int lnn_mode,
                                    float ascent_tol, double* objective, float* L, int8_t* s_hat,
                                    uint32_t* flags, void* stream);

/*
 * taser_host_workspace_bytes -- bytes of device workspace taser_run_host needs for
 * `batch` instances of the given problem (0 for invalid arguments).
 */
size_t taser_host_workspace_bytes(int kind, int64_t batch, int B, int U_or_K);

/*
 * taser_run_host -- the whole path from HOST inputs to HOST decisions, ordered on
 * `stream`: copy H and y (or Y) to the device, taser_build_T, taser_detect (no L
 * output), copy s_hat and flags back.  Arguments as in taser_build_T / taser_detect,
 * except:
 *   H_or_Y, y     HOST complex64 buffers (pinned memory gives full copy bandwidth).
 *   workspace     DEVICE buffer of at least taser_host_workspace_bytes(...) bytes,
 *                 256-byte aligned, owned by the caller; its contents are scratch.
 *   s_hat, flags  HOST outputs, int8 [batch][N-1] and uint32 [batch] (flags may be NULL).
 * The call returns once the work is enqueued; synchronize `stream` before reading the
 * host outputs.  Batches above 8,192 instances are pipelined in chunks of 8,192: the
 * host-to-device copies run on a side stream the library creates once per host thread and
 * device, each chunk's kernels wait for its copy on `stream`, and `stream` orders the whole
 * call (the side stream first waits for the work already queued on `stream`, and `stream`
 * waits for every copy), so the call keeps the semantics of one stream-ordered operation,
 * also under CUDA graph capture.
 */
taser_status taser_run_host(int kind, int64_t batch, int B, int U_or_K, const void* H_or_Y,
                            const void* y, float alpha, int t_max, int precision, int lnn_mode,
                            void* workspace, size_t workspace_bytes, int8_t* s_hat,
                            uint32_t* flags, void* stream);

/*
 * taser_unfolded_forward -- unfolded TASER: Algorithm 1 with one step size per
 * iteration, tau_t = alpha_t / ||T~||_2, learnable alpha_t shared by all instances
 * (mode TASER_LNN_FIXED).  Forward pass of the training path.
 *   T_tilde, D  as in taser_detect; N in [2, 33].
 *   inv_norm    float [batch] = 1 / ||T~||_2 (from spec_norm of taser_build_T).
 *   alpha_t     float [t_max].
 *   c           checkpoint spacing, 1 <= c <= t_max (ceil(sqrt(t_max)) balances memory
 *               and recomputation).
 *   precision   TASER_FP32, or TASER_BF16_TC / TASER_FP16_TC: the triangular products on
 *               the tensor cores (operands of -2 tau_t L~ and T~ in BF16/FP16, FP32
 *               accumulation) with the master iterates and the prox in FP32, for
 *               18 <= N <= 33; smaller N runs FP32.  TASER_FIXED14 returns
 *               TASER_ERR_UNSUPPORTED.  Pass the same precision to the backward call.
 *   ckpt        out float [batch][ceil(t_max / c)][N][N]: L~(k c) for k = 0, 1, ..., or
 *               NULL when no backward pass follows.
 *   soft        out float [batch][N-1]: x_k = L~(t_max)_{N,k} / D_k, the last row of the
 *               unit-column factor L = L~ D^-1 (Sec. III-C), in [-1, 1].
 *   s_hat       out int8 [batch][N-1] = sign(x_k), or NULL.
 */
taser_status taser_unfolded_forward(int64_t batch, int N, const float* T_tilde, const float* D,
                                    const float* inv_norm, const float* alpha_t, int t_max, int c,
                                    int precision, float* ckpt, float* soft, int8_t* s_hat,
                                    void* stream);

/*
 * taser_unfolded_backward -- adjoint of taser_unfolded_forward.  Given grad_soft =
 * dloss/dsoft (float [batch][N-1]), writes grad_tau (float [batch][t_max]) =
 * dloss/dtau_t per instance and, if grad_alpha is not NULL, grad_alpha (float [t_max]) =
 * sum_n grad_tau[n][t] inv_norm[n] in a fixed reduction order.  Each segment of c
 * iterations is recomputed from ckpt (same arguments as the forward call) and
 * differentiated in reverse; the gradient flows through the soft last row only.
 * The tensor-core precisions differentiate the tensor-core forward (the products of the
 * recomputed steps and Vbar (2 T~) on the tensor cores, the prox Jacobian in FP32).
 * Shared memory per block (one warp, one instance): FP32, (c + 2) M(NB) floats, NB the
 * bucket of N and M(NB) the packed lower triangle of an (NB + 1)-row matrix whose rows
 * are padded to 4 floats (60 / 180 / 612 at NB = 8 / 16 / 32; c <= 92 at N = 33); tensor
 * cores, 1,280 c + 1,248 floats (c <= 44).  Larger c is rejected.
 */
taser_status taser_unfolded_backward(int64_t batch, int N, const float* T_tilde, const float* D,
                                     const float* inv_norm, const float* alpha_t, int t_max, int c,
                                     int precision, const float* ckpt, const float* grad_soft,
                                     float* grad_tau, float* grad_alpha, void* stream);

/*
 * Uneven batches.  One item per detection problem; the items share pooled buffers.
 */
typedef struct {
    int32_t N;       /* problem size, 2..65 */
    int32_t t_max;   /* iterations, >= 1 */
    int64_t t_off;   /* offset (in floats) of the item's T~ (N x N) in T_pool */
    int64_t d_off;   /* offset (in floats) of its D (N) in D_pool */
    int64_t s_off;   /* offset (in bytes) of its decisions (N - 1) in s_pool */
    int64_t l_off;   /* offset (in floats) of its L~ (N x N) in L_pool, or -1 for none */
} taser_item;

/* Per-bucket launch tuning of taser_detect_uneven (buckets N <= 9, 17, 33, 65). */
typedef struct {
    int32_t blocks_per_sm[4];   /* persistent blocks per SM, 0 = as many as fit */
    int32_t pop[4];             /* items a warp (pair) takes per queue pop, 0 = the
                                   default (tensor cores: 4 at N <= 17, 2 at N <= 33, else
                                   1; FP32: one warp-load); FP32 rounds it up to whole
                                   warp-loads (4 / 2 / 1 / 1 items at N <= 9 / 17 / 33 /
                                   65); the fixed-point path ignores it */
} taser_uneven_tuning;

/* Device workspace (bytes) taser_detect_uneven needs for n_items items. */
size_t taser_uneven_workspace_bytes(int64_t n_items);

/*
 * taser_detect_uneven -- Algorithm 1 on a batch of problems of different sizes and
 * iteration counts (N = 2..65, any t_max >= 1 per item), in one stream-ordered sequence
 * without host synchronisation (capturable in a CUDA graph and replayed with one launch):
 * a counting sort (three short kernels) builds a size-bucketed work queue in `workspace`
 * (items grouped by bucket N <= 9 / 17 / 33 / 65, then by t_max, longest first), and one
 * persistent kernel per bucket takes its items: from an atomic counter, or (the N <= 65
 * tensor-core bucket) at a fixed stride per warp pair over the sorted list.  The bucket
 * kernels run on two internal streams forked from and joined back into `stream` (the
 * N <= 65 bucket at high priority, the others after one another at low priority, filling
 * the SMs the first frees in its tail); calls from one host thread share these streams.
 * Precisions as in taser_detect (tensor cores for N >= 10, FP32 below).
 *   items     device array of n_items taser_item.
 *   T_pool, D_pool, tau (float [n_items]), L_pool (may be NULL), s_pool: device pools
 *             addressed by the items' offsets.
 *   flags     uint32 [n_items] or NULL: OR-ed flag bits; items with N or t_max out of range
 *             are skipped and get TASER_FLAG_BAD_ITEM (the bounds-checked debug build
 *             treats items with a negative offset the same way).
 *   workspace device buffer of taser_uneven_workspace_bytes(n_items) bytes, 256-byte aligned.
 *   tuning    per-bucket launch parameters (from the autotuner), or NULL for defaults.
 * Items are independent: their results do not depend on the queue order.
 */
taser_status taser_detect_uneven(int64_t n_items, const taser_item* items, const float* T_pool,
                                 const float* D_pool, const float* tau, int precision,
                                 int lnn_mode, float* L_pool, int8_t* s_pool, uint32_t* flags,
                                 void* workspace, size_t workspace_bytes,
                                 const taser_uneven_tuning* tuning, void* stream);

/*
 * taser_run_host_static -- taser_run_host without a caller-provided workspace.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory.  Examples are baseband pipelines that reserve every buffer at
 * start-up and must not call cudaMalloc inside a slot (it can synchronise the device and
 * stall a real-time deadline), and plug-ins whose host framework owns the whole device
 * memory pool and hands them none.  Such callers pass only their inputs and outputs.
 *
 * The scratch (device copies of H and y or Y, T~, D, tau, the decisions and flags) lives
 * in one file-scope device array of TASER_STATIC_SCRATCH_BYTES, which every GPU that
 * loads the library holds until the process exits.  A batch whose
 * taser_host_workspace_bytes(kind, batch, B, U_or_K) exceeds that size is rejected with
 * TASER_ERR_INVALID_ARG (split it into smaller calls).  Nothing in the scratch has to
 * start at zero: every intermediate is written before it is read.  The array keeps the
 * last call's contents, and all calls share it: calls whose GPU work overlaps (on
 * different streams, or from several threads) race on it and must be serialised by the
 * caller.  The first call on a device looks up the array's device address for that
 * device (cudaGetSymbolAddress, with that device current) and keeps it for the life of
 * the process; make that first call before any stream capture.  The kept address does
 * not survive a cudaDeviceReset (or any other teardown of the device's primary context):
 * calls after one are not supported.  Arguments and outputs are as in taser_run_host.
 */
#define TASER_STATIC_SCRATCH_BYTES ((size_t)64 << 20)

taser_status taser_run_host_static(int kind, int64_t batch, int B, int U_or_K,
                                   const void* H_or_Y, const void* y, float alpha, int t_max,
                                   int precision, int lnn_mode, int8_t* s_hat,
                                   uint32_t* flags, void* stream);

/*
 * taser_debug_report -- counters of the bounds-checked debug build.
 *
 * libtaser_debug.so is the same library compiled with -DTASER_DEBUG.  The paper has no
 * counterpart: the build stands in for a device memory checker.  Every kernel tests the
 * global and shared-memory indices it computes at run time against the extents its
 * arguments imply (batch x per-instance sizes, the staging slots, the queue list) and
 * against the instance's own N x N, N or N - 1 elements; an access that fails is counted
 * and skipped.  Nothing traps and nothing waits.  Pools of taser_detect_uneven have no
 * stated extent, so there only the offsets' signs and each item's own indices are
 * checked.  The build also counts non-finite output values (T~, D, ||T~||, L~, the
 * decisions' row, the unfolded soft outputs and gradients).
 *   fails      failed index checks since the last report (all kernels, current device)
 *   first      the first recorded failure as (source file number << 56) |
 *              (source line << 32) | (low 32 bits of the index), or 0 if none
 *   nonfinite  non-finite output values since the last report
 * The three pointers are HOST pointers and must not be NULL.  Reading the counters
 * (cudaMemcpyFromSymbol) waits for the device and clears them.  The release library
 * (libtaser.so) returns TASER_ERR_UNSUPPORTED and leaves the outputs unchanged.
 */
taser_status taser_debug_report(uint64_t* fails, uint64_t* first, uint64_t* nonfinite);

/*
 * taser_debug_drop_copy -- fault injection of the bounds-checked debug build (the paper has
 * no counterpart).  Later taser_build_T calls that stage by TMA (QPSK with 16 users, B
 * even) withhold the staging copy of 16-antenna chunk `chunk` of instance `instance`, so
 * the bounded wait for it (about a second of SM clock) expires.  That instance then gets
 * TASER_FLAG_TIMEOUT and its T~ and D are left unwritten; the other instances are not
 * affected.  Nothing faults, because the copy is never issued.  instance < 0 turns the
 * injection off.  The release library returns TASER_ERR_UNSUPPORTED.
 */
taser_status taser_debug_drop_copy(int64_t instance, int chunk);

#ifdef __cplusplus
}
#endif

#endif /* TASER_H */
