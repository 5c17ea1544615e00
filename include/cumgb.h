/*
 * cumgb -- block-structured moment and cumulant tensors on GB300 (sm_103a).
 *
 * C ABI of the library libcumgb.so.  Method: Domino, Gawron, Pawela,
 * "Efficient computation of higher order cumulant tensors" (arXiv 1701.05420).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Data.  X is t samples x n variables (Eq. variable), row-major with row stride
 *   ldx elements (ldx >= n), element type cum_dtype.
 * Blocks.  Variables are grouped into nbar = ceil(n / b) blocks of side b
 *   (Sec. 2.1).  n is zero-padded to nbar * b; a padded variable is an exact
 *   zero column, so every moment or cumulant entry that touches it is 0 --
 *   the same result as the ragged last block b_l of Sec. 2.1.
 *   Only blocks with sorted block indices j_1 <= ... <= j_d are stored
 *   (Sec. 2.1); there are C(nbar + d - 1, d) of them (the count printed in
 *   Sec. 2.1 and 5.2.1 swaps the lower index; the multiset count is meant).
 * Block rank.  A sorted tuple j (0-based) has colex rank
 *   r(j) = sum_{k=1..d} C(j_k + k - 1, k)  (combinatorial number system;
 *   the paper does not fix an order, its Alg. 2 loops j_1 outermost).
 * Tensor layout.  An order-d tensor is one contiguous double array of
 *   cum_num_blocks(nbar, d) * b^d entries.  Block r occupies
 *   [r * b^d, (r + 1) * b^d); inside it, the element with in-block index
 *   (i_1..i_d), 0 <= i_k < b, is at offset sum_k i_k * b^(d-k) (i_1 slowest).
 *   It holds the tensor element at variable indices (j_k * b + i_k)_k.
 *   Diagonal blocks are stored in full (Sec. 5.2.1).
 * Normalisation.  Moments use 1/t (Eq. d::moment), never 1/(t-1).
 * Memory.  Unless stated otherwise, data pointers are DEVICE pointers owned by
 *   the caller.  The library allocates no device memory: scratch comes from a
 *   caller-provided workspace of cum_workspace_size() bytes (256-byte
 *   aligned).  Each call enqueues its kernels on the caller's CUDA stream
 *   (passed as void*, a cudaStream_t; NULL = legacy default stream) and
 *   returns without synchronising; results are ready when the stream is.
 * Errors.  Every int-returning call returns CUM_OK (0) or a cum_status code;
 *   on CUM_ECUDA the CUDA error of the failing call is available from
 *   cum_last_cuda_error() (per host thread).  Argument checks happen before
 *   anything is enqueued.
 */
#ifndef CUMGB_H
#define CUMGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CUM_OK = 0,
    CUM_EINVAL = 1,        /* an argument is out of range or a pointer is NULL   */
    CUM_EUNSUPPORTED = 2,  /* valid request outside this build's limits          */
    CUM_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed        */
    CUM_ETIMEOUT = 4,      /* a bounded device-side wait expired                 */
    CUM_EWORKSPACE = 5     /* workspace NULL, misaligned or smaller than needed  */
} cum_status;

typedef enum { CUM_F32 = 0, CUM_F64 = 1 } cum_dtype;

/* Arithmetic of the moment contraction (Alg. 1-2).  Centring sums, the
 * t-chunk reduction and the cumulant subtraction (Eq. cum_r) are FP64 in
 * every mode.
 *   CUM_PREC_FP64   : FP64 products and sums on the CUDA cores.
 *   CUM_PREC_BF16X3 : each Khatri-Rao operand split x = hi + lo in bf16,
 *                     lo*lo + hi*lo + lo*hi + hi*hi on tcgen05 tensor cores
 *                     (lo*lo only outside batches), FP32 accumulation in
 *                     tensor memory drained to FP64.
 *   CUM_PREC_FP16X3 : as BF16X3 with fp16 parts at the bf16 tensor rate: hi
 *                     is the product rounded to 8 significant bits, lo the
 *                     rest rounded to fp16 (19 bits; the short hi part keeps
 *                     the tensor core's truncating sums less biased).  In
 *                     batches hi carries 8 bits at even orders and 11 at
 *                     odd ones, lo 11.
 *   CUM_PREC_TF32X3 : in batches (cum_batch_*), as BF16X3 with tf32 parts
 *                     (22 significant bits) at half the bf16 tensor rate;
 *                     single datasets run the fp16 parts of FP16X3, which
 *                     are faster and more accurate on these tensor cores.
 * Outside batches every split precision scales each centred variable by a
 * power of two 2^s (max |x| in [16, 32), s clamped to [-60, 60]) so that
 * products of up to three factors stay in fp16 range, and multiplies the
 * results back exactly (in batches, FP16X3 only); variables whose largest
 * centred magnitude lies outside [2^-55, 2^64] lose accuracy to fp16 range
 * limits.  In every split precision, orders 2 to 5 instead take the centred data as
 * a double-float (FP32 X~ plus its FP32 remainder), form each Khatri-Rao
 * product as a double-float and split it into three fp16 parts of 8, 11 and
 * 11 bits (about 30 bits, with the 2^s scaling above and an exact factor
 * 2^(15 - 5 k) on each Khatri-Rao row of k factors); the six part products of
 * weight down to 2^-19 run on the tensor cores.  Two parts leave errors
 * above 1e-6 on odd moments that are small next to their terms; order 6,
 * most of the work, keeps two parts from 8192 samples on (below, three).
 * Batches keep two parts at every order on an FP32 centred array, rounded
 * stochastically (round away from zero with probability equal to the
 * remainder over the ulp, from a counter-based hash of dataset, variable and
 * sample; every run rounds alike): round-to-nearest of x - mean leaves an
 * error that is even in x and biases odd moments in proportion to t.  */
typedef enum {
    CUM_PREC_FP64 = 0,
    CUM_PREC_BF16X3 = 1,
    CUM_PREC_FP16X3 = 2,
    CUM_PREC_TF32X3 = 3
} cum_prec;

/* Largest supported order.  */
#define CUM_MAX_ORDER 6

/* Number of stored blocks C(nbar + d - 1, d) of an order-d tensor (Sec. 2.1).
 * Returns -1 if nbar < 1, d < 1 or the count overflows int64.  Host only. */
int64_t cum_num_blocks(int nbar, int d);

/* Colex rank of the sorted block tuple j[0..d-1] (0-based, non-decreasing).
 * Host pointers.  CUM_EINVAL if j is NULL, unsorted, negative, or d < 1.    */
int cum_block_rank(const int32_t* j, int d, int64_t* rank);

/* Inverse of cum_block_rank: writes the sorted tuple j[0..d-1] of block
 * `rank` among the C(nbar + d - 1, d) blocks.  Host pointers.
 * CUM_EINVAL if rank is out of range or a pointer is NULL.                   */
int cum_block_unrank(int64_t rank, int d, int nbar, int32_t* j);

/* Workspace bytes needed by cum_center / cum_moment_blocks / cum_cumulants
 * for orders up to d_max with these sizes and precision.  Returns 0 if the
 * arguments are invalid or unsupported.  Host only.                          */
size_t cum_workspace_size(int64_t t, int n, int d_max, int b, int prec);

/* Centring (Def. 1.3): mean_out[i] = (1/t) sum_l x_{l,i} (two-pass FP64),
 * and the centred data X~ = X - mean is written into the workspace in the
 * operand layout that `prec` uses (variable-major, zero-padded), where
 * cum_moment_blocks reads it.  X: device, t x n, row stride ldx.
 * mean_out: device, n doubles (may be NULL).  ws: workspace sized by
 * cum_workspace_size(t, n, d, b, prec) for the orders d to be computed.
 * Split precisions store X~ in FP32 with its FP32 remainder (a double-float,
 * for orders 2 to 5), and rounding X - mean to FP32 leaves each column with
 * a small residual mean (about 2^-25 of its scale); the FP64 sums of the
 * stored FP32 columns are kept in `ws` for the moments' correction below.   */
int cum_center(const void* X, int dtype, int64_t t, int n, int64_t ldx, int b, int prec,
               double* mean_out, void* ws, size_t ws_bytes, void* stream);

/* Order-d central moment tensor in block storage (Alg. 1 MOMENTBLOCK over all
 * sorted blocks as in Alg. 2 MOMENT; the t axis is split into chunks summed in
 * FP64 and divided by t once, Alg. 3 / Eq. mapred):
 *   M[i] = (1/t) sum_l prod_k x~_{l, i_k}.
 * Reads X~ left in `ws` by cum_center with the same t, n, b, prec.
 * M_out: device, cum_num_blocks(nbar, d) * b^d doubles.  2 <= d <= CUM_MAX_ORDER.
 * On split precisions with d = 6 and t >= 8192 (read from the FP32 X~ alone) the
 * stored X~'s residual column means m are removed to first order,
 * M[i] -= sum_k m_{i_k} M_{d-1}[i without i_k] (the dropped terms are O(m^2),
 * below FP64 resolution); the call computes the order-5 moments into the
 * workspace for it.  Orders 2 to 5 read the double-float X~, whose residual
 * means are below FP64 resolution, and take no correction.                  */
int cum_moment_blocks(int d, int64_t t, int n, int b, int prec, double* M_out,
                      void* ws, size_t ws_bytes, void* stream);

/* The moment contraction alone (Alg. 1-3) on X~ as stored in `ws`: what
 * cum_moment_blocks computes before the residual-mean correction (for FP64
 * operands the two are the same).  Arguments as for cum_moment_blocks.       */
int cum_moment_contraction(int d, int64_t t, int n, int b, int prec, double* M_out,
                           void* ws, size_t ws_bytes, void* stream);

/* Cumulant correction of Alg. 4 OUTERPRODCUM and Alg. 5 CUMULANT (Eq. cum_r):
 *   C_d = M_d - sum_{sigma=2}^{floor(d/2)} sum_{zeta in P^(2)_sigma(1:d)} (x)_{k in zeta} C_|k|
 * over set partitions of 1:d into parts of size >= 2.  M_d: order-d central
 * moment in block storage; C_lower[k-2] (k = 2..d-2): cumulant tensors of
 * order k in block storage.  C_out may equal M_d (in place).  All device.
 * For d <= 3 this is a copy (C_d = M_d).                                     */
int cum_correct(int d, int n, int b, const double* M_d, const double* const* C_lower,
                double* C_out, void* stream);

/* Order-6 correction in moment form (Eq. cum_r at orders 4 and 6).  The
 * partitions of 1:6 whose part holding position 1 is a pair {1, x} sum, over
 * the ways of splitting the other four positions R, to C_2[1x] M_4[R]: by
 * Eq. cum_r at order 4, C_4[R] plus its three pairings of C_2 C_2 is M_4[R].
 * So
 *   C_6 = M_6 - sum_x C_2[1x] M_4[R_x] - sum_{pairs P not holding 1} C_2[P] C_4[rest]
 *             - sum_{3+3} C_3 C_3,
 * 25 products per entry instead of the 40 of cum_correct, same result up to
 * rounding.  M_6, M_4: the order-6 and order-4 central moments in block
 * storage; C_lower[k-2] (k = 2, 3, 4) as for cum_correct; C_out may equal M_6.
 * All device.  cum_cumulants uses this form whenever d_max >= 6.             */
int cum_correct_m4(int n, int b, const double* M_6, const double* const* C_lower,
                   const double* M_4, double* C_out, void* stream);

/* Cumulant tensors of orders 2..d_max (Alg. 5, applied in increasing order):
 * centring, the moment contraction of each order, then the correction.
 * C_out[d-2] (d = 2..d_max): device, cum_num_blocks(nbar, d) * b^d doubles each
 * (the pointer array itself is a HOST array).  mean_out: device, n doubles
 * (the first cumulant), may be NULL.                                          */
int cum_cumulants(const void* X, int dtype, int64_t t, int n, int64_t ldx, int d_max, int b, int prec,
                  double* const* C_out, double* mean_out, void* ws, size_t ws_bytes, void* stream);

/* ---- Steps of the t-sharded computation (Alg. 3 across processes) --------
 * A caller that splits the samples across processes (one shard of rows each)
 * combines these with an allreduce(sum) of its own:
 *   cum_column_sums -> allreduce -> cum_mean_from_sums      (repeat once with
 *   shift = the first mean for the two-pass mean), cum_center_with_mean,
 *   cum_residual_sums -> allreduce -> cum_set_residual_sums(t_total), then
 *   per order: cum_moment_sums -> allreduce -> cum_finalize(scale = 1/t_total).
 * Each is asynchronous on `stream`; pointers are device pointers.            */

/* sums_out[i] = sum_l (x_{l,i} - shift[i]) over the t rows of X (shift may be
 * NULL), in FP64.  ws as for cum_center.                                       */
int cum_column_sums(const void* X, int dtype, int64_t t, int n, int64_t ldx, int b, int prec, const double* shift,
                    double* sums_out, void* ws, size_t ws_bytes, void* stream);

/* mean_out[i] = shift[i] + sums[i] / t_total (shift may be NULL): Def. 1.3.   */
int cum_mean_from_sums(int n, int64_t t_total, const double* shift, const double* sums, double* mean_out,
                       void* stream);

/* As cum_center, but subtracts the given mean (n doubles) instead of the
 * shard's own: the centred shard of a dataset whose mean is global.  The
 * shard's stored column sums are kept (cum_residual_sums) but not used until
 * cum_set_residual_sums supplies the global ones: without that step the
 * moments carry no residual-mean correction.                                */
int cum_center_with_mean(const void* X, int dtype, int64_t t, int n, int64_t ldx, int b, int prec,
                         const double* mean, void* ws, size_t ws_bytes, void* stream);

/* FP64 sums over this shard's rows of the stored X~ columns (split
 * precisions; zeros for FP64 operands), left in `ws` by cum_center or
 * cum_center_with_mean: sums_out, n doubles, device.  Their allreduce over
 * shards gives the global residual column sums.  ws needs only the centring
 * regions of cum_workspace_size's layout (which depend on n, b, prec).       */
int cum_residual_sums(int n, int b, int prec, double* sums_out, const void* ws, size_t ws_bytes, void* stream);

/* Replaces the residual column sums kept in `ws` by `sums` (n doubles, device:
 * the global sums over all shards) with divisor t_total, so that this shard's
 * cum_moment_sums remove the global residual means.  No-op for FP64.         */
int cum_set_residual_sums(int n, int b, int prec, const double* sums, int64_t t_total, void* ws, size_t ws_bytes,
                          void* stream);

/* As cum_moment_blocks but without the 1/t: S[i] = sum_l prod_k x~_{l, i_k}
 * over this shard's rows (the per-process term of Eq. momentp1), with the
 * residual-mean correction (m = the kept sums / their divisor) applied to the
 * sums: summed over shards it is the global correction.                       */
int cum_moment_sums(int d, int64_t t, int n, int b, int prec, double* S_out, void* ws, size_t ws_bytes,
                    void* stream);

/* C_d = scale * S_d - (Alg. 4 partition products of C_lower), i.e. the 1/t of
 * Eq. momentp1 followed by the correction of Eq. cum_r.  C_out may equal S_d. */
int cum_finalize(int d, int n, int b, double scale, const double* S_d, const double* const* C_lower, double* C_out,
                 void* stream);

/* Execution plan of the moment contraction of order d for these sizes (host
 * only; for diagnostics and benchmarks).  Writes info[0..7]:
 *   [0] active output tiles (tiles holding at least one stored entry),
 *   [1] chunks of the t axis (Alg. 3), [2] work units = [0] * [1],
 *   [3] tile rows, [4] tile columns, [5] samples per chunk,
 *   [6] kernels cum_cumulants enqueues for this order's moments (tile plan,
 *       contraction, t-chunk reduction if split, residual-mean correction
 *       on split precisions for d = 6, t >= 8192; cum_moment_blocks enqueues the
 *       order-(d-1) plan and contraction on top),
 *   [7] kernels cum_center enqueues.
 * CUM_EINVAL / CUM_EUNSUPPORTED as for cum_workspace_size.                    */
int cum_plan_info(int d, int64_t t, int n, int b, int prec, int64_t* info);

/* ---- Batches of independent datasets ---------------------------------------
 * Many datasets (each its own t_i x n_i matrix and block side b_i) through one
 * fixed launch sequence: batched centring (Def. 1.3), then for every order one
 * persistent contraction launch over the work units (output tile x t chunk) of
 * every dataset (Alg. 1-3), the t-chunk reduction, and the correction
 * (Alg. 4-5).  Planning and binding run on the host once; cum_batch_run only
 * enqueues kernels on `stream`, so a run can be captured in a CUDA graph and
 * replayed while the bound buffers stay valid.                                */
typedef struct cum_batch_s* cum_batch;

/* Plans `count` datasets: t[i] samples, n[i] variables, block side b[i], orders
 * 2..d_max, precision `prec`, input element type `dtype` (all host arrays).
 * Writes the plan handle (host memory, released by cum_batch_free) and the
 * device workspace bytes the batch needs.  CUM_EUNSUPPORTED if a dataset is
 * outside the limits of cum_workspace_size.                                   */
int cum_batch_plan(int count, const int64_t* t, const int* n, const int* b, int d_max, int prec, int dtype,
                   cum_batch* plan, size_t* ws_bytes);

/* Binds device buffers (host arrays of device pointers): X[i] (t_i x n_i,
 * row stride ldx[i], or n_i if ldx is NULL); C_out[i * (d_max - 1) + d - 2]
 * (block storage of order d of dataset i, b_i blocks); mean_out[i] (n_i
 * doubles, or mean_out NULL).  Writes the device tables into ws (synchronous:
 * returns after they are on the device).                                      */
int cum_batch_bind(cum_batch plan, const void* const* X, const int64_t* ldx, double* const* C_out,
                   double* const* mean_out, void* ws, size_t ws_bytes, void* stream);

/* Enqueues the batch's kernels on `stream` (asynchronous).                     */
int cum_batch_run(cum_batch plan, void* stream);

/* info[0] datasets, [1] contraction work units, [2] kernel launches per run,
 * [3] workspace bytes.                                                         */
int cum_batch_info(cum_batch plan, int64_t* info);

void cum_batch_free(cum_batch plan);

/* ---- Without device allocation --------------------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory themselves -- for example a plugin whose host
 * application owns every byte of device memory, or code on a path that must
 * not call the allocator -- and therefore cannot hand cum_cumulants a
 * workspace.
 *
 * cum_cumulants_noalloc computes exactly what cum_cumulants computes, with the
 * workspace taken from a fixed device array inside the library of
 * CUM_NOALLOC_WORKSPACE_BYTES (64 MiB).  Every GPU that loads the library
 * holds that array until the process exits.  The caller still provides X,
 * C_out and mean_out (device memory, as for cum_cumulants).
 *  - Requests whose cum_workspace_size(t, n, d_max, b, prec) exceeds
 *    CUM_NOALLOC_WORKSPACE_BYTES are rejected with CUM_EUNSUPPORTED before
 *    anything is enqueued; invalid arguments give CUM_EINVAL.
 *  - The call allocates nothing: no cudaMalloc, no cudaFree, no allocating
 *    library routine.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and keeps it; make that
 *    first call before any stream capture on the device.  The kept address
 *    belongs to the device's current context: after cudaDeviceReset on that
 *    device the library may be loaded at another address, so do not call
 *    this entry point on a device after resetting it in the same process.
 *  - All calls share the one array per device, and it keeps the previous
 *    call's contents (the call clears what must start at zero).  Calls whose
 *    work overlaps on the GPU -- on different streams, or from different host
 *    threads without ordering -- race on the array and give wrong results;
 *    order them (one stream, or events).                                      */
#define CUM_NOALLOC_WORKSPACE_BYTES (64ull << 20)

int cum_cumulants_noalloc(const void* X, int dtype, int64_t t, int n, int64_t ldx, int d_max, int b, int prec,
                          double* const* C_out, double* mean_out, void* stream);

/* Synchronises `stream`, then reads and clears the device status word kept in
 * `ws`: CUM_ETIMEOUT if a bounded wait in a kernel expired since the last
 * check, else CUM_OK (or CUM_ECUDA).                                          */
int cum_device_status(void* ws, size_t ws_bytes, void* stream);

/* Diagnostic of failure detection; the paper has no counterpart.  Launches,
 * on `stream`, one thread that performs the contraction kernels' bounded wait
 * on a barrier nothing arrives at: after the wait limit (about 2 s of GPU
 * clock) it records CUM_ETIMEOUT in the status word of `ws` (256-byte
 * aligned, >= 64 bytes, caller-owned) and returns; nothing stays in flight.
 * cum_device_status then reports the timeout, and the device stays usable.
 * Returns CUM_EWORKSPACE for a missing or misaligned workspace.             */
int cum_probe_bounded_wait(void* ws, size_t ws_bytes, void* stream);

/* Static description of a status code (never NULL).                          */
const char* cum_strerror(int status);

/* CUDA error code (cudaError_t) of the last failing CUDA call in this thread. */
int cum_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CUMGB_H */
