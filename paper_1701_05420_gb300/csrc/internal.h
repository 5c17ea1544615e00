// Internal declarations shared by the translation units of libcumgb.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace cum {

constexpr int64_t kTAlign = 128;        // t is zero-padded to a multiple of this
constexpr size_t kWsAlign = 256;        // alignment of every workspace region
constexpr int kColsumChunks = 512;      // row chunks of the centring sums
constexpr int kMaxPartitions = 48;      // >= F(6) - 1 = 40
constexpr int kMaxParts = 3;            // >= floor(6/2)

// Tile geometry of the two moment kernels.
constexpr int kF64TileM = 64, kF64TileN = 64, kF64KStep = 16;
constexpr int kTcTileM = 128, kTcTileN = 128;
constexpr int kTcMaxCtas = 160;         // >= SM count of a GB300 (152)
constexpr int kTcPlanCtas = 152;        // SM count of a GB300: CTAs the t-axis split is planned for
constexpr int64_t kTcUnitSteps = 24;    // fixed cost of a contraction work unit, in 128-sample steps
constexpr int kTcMaxNPad = 256;         // variables staged per TMA box (box rows <= 256)
// CTA-pair contraction (fp16 / bf16 parts, single dataset): 256 x 128 tiles,
// one cluster of two CTAs per TPC; per CTA a 128 x 128 FP64 scratch tile, as
// for the one-CTA kernel.
constexpr int kPairTileM = 256, kPairTileN = 128;
constexpr int kPairPlanClusters = 76;
constexpr int64_t kPreciseOrder6T = 8192;   // order 6 takes three fp16 parts below this many (padded) samples
constexpr size_t kTcScratchDoubles = (size_t)kTcMaxCtas * 128 * 128;

// Set partitions of 1:d into >= 2 parts, every part of size >= 2 (P^(2)_sigma,
// Def. 3.5), as bit masks of positions.
struct PartTable {
    int count;
    int nparts[kMaxPartitions];
    uint32_t mask[kMaxPartitions][kMaxParts];
};

struct LowerPtrs {
    const double* c[kMaxOrder + 1];     // c[k]: cumulant tensor of order k (k = 2..d-2)
    const double* m4;                   // order-4 moment blocks (layout of c[4]) or NULL: with
                                        // d = 6 the staged correction then takes the moment form
};

// Per-order execution plan of the moment contraction.
struct OrderPlan {
    Shape sh;
    bool pair;               // CTA-pair kernel (moment_pair.cu), else one CTA per tile
    bool precise;            // split precisions, orders 2 and 3: three fp16 parts of the double-float X~ (pair kernel)
    int tile_m, tile_n;
    int64_t row_tiles;       // ceil(rows / tile_m)
    int64_t active_tiles;    // tiles with at least one valid (last <= first) entry
    int splits;              // S: chunks of the t axis (Alg. 3)
    int64_t kchunk;          // samples per chunk (multiple of the k step)
    int64_t units;           // active_tiles * splits
};

struct WsLayout {
    size_t status;           // device status word
    size_t colsum;           // kColsumChunks * n_pad doubles, then mean and correction
    size_t maxabs;           // split precisions: max |x~| per variable (float bits, n_pad uint32)
    size_t vexp;             // split precisions: fp16 power-of-two scale exponent per variable (n_pad int32)
    size_t rsum;             // split precisions: FP64 column sums of the stored X~ (n_pad), then their divisor t
    size_t xt;               // X~ transposed: n_pad rows of t_pad (double or float)
    size_t xlo;              // split precisions: FP32 remainder X~ - xt (same layout), the low word of a double-float X~
    // the regions above are what centring writes; their offsets do not depend on d_max
    size_t prefix;           // row-tile prefix of active tile counts (int64)
    size_t partial;          // S * E_d doubles for split chunks
    size_t scratch;          // tensor-core path: per-CTA FP64 accumulation tiles
    size_t m4;               // order-4 moment blocks: kept for the order-6 correction (d_max >= 6) and,
                             // on split precisions, for the order-5 residual-mean correction (d_max >= 5)
    size_t mlow;             // split precisions: order-(d_max - 1) moments (or sums) for the residual-mean correction
    size_t total;
    int64_t t_pad;
    int n_pad;
    size_t xt_elem;
};

bool prec_is_tc(int prec);
bool prec_is_valid(int prec);
int cuda_fail(cudaError_t e);   // records e for cum_last_cuda_error, returns CUM_ECUDA
int64_t pad_t(int64_t t);
// pair_ok: a single-dataset call, which runs fp16 / bf16 parts on the CTA-pair
// kernel; the batched launch plans for the one-CTA kernel.
OrderPlan make_order_plan(int d, int64_t t, int n, int b, int prec, bool pair_ok = true);
// Largest t-axis split of plan P (chunks of >= 2048 samples, partials <= 1 GiB).
int64_t max_order_splits(const OrderPlan& P, int64_t t, int prec);
// Split the t axis of P into (about) S chunks of whole steps; sets kchunk, splits, units.
void set_order_splits(OrderPlan& P, int64_t t, int prec, int64_t S);
bool layout_ws(int64_t t, int n, int d_max, int b, int prec, WsLayout* L);
PartTable make_part_table(int d);

// Launchers (kernels_fp64.cu).
cudaError_t launch_center(const void* X, int dtype, int64_t t, int n, int64_t ldx, const WsLayout& L,
                          char* ws, int prec, double* mean_out, cudaStream_t st);
cudaError_t launch_plan(const OrderPlan& P, int64_t* prefix, cudaStream_t st);
cudaError_t launch_moment_fp64(const OrderPlan& P, const double* xt, int64_t t_pad, const int64_t* prefix,
                               double* out_or_partial, double scale, cudaStream_t st);
cudaError_t launch_reduce(const double* partial, int S, int64_t E, double scale, double* out, cudaStream_t st);
struct BatchOrder;
struct BatchUnit;
cudaError_t launch_moment_fp64_batch(int dA, int dB, const BatchOrder* orders, const BatchUnit* units, int64_t nunits,
                                     cudaStream_t st);
cudaError_t launch_correct(int d, int b, int nbar, const double* M, double scale, const LowerPtrs& low,
                           const PartTable& pt, double* C, cudaStream_t st);
// Correction with the lower-order blocks staged in shared memory (correct.cu);
// sets *done = false, launching nothing, where it does not apply.
cudaError_t launch_correct_staged(int d, int b, int nbar, const double* M, double scale, const LowerPtrs& low,
                                  double* C, cudaStream_t st, bool* done);
cudaError_t launch_column_sums(const void* X, int dtype, int64_t t, int n, int64_t ldx, const double* shift,
                               const WsLayout& L, char* ws, double* sums, cudaStream_t st);
cudaError_t launch_mean_from_sums(int n, int64_t t_total, const double* shift, const double* sums, double* mean,
                                  cudaStream_t st);
cudaError_t launch_shift_correct(int d, int b, int nbar, const double* Mlow, const double* rsum, int n_pad, double* M,
                                 cudaStream_t st);
cudaError_t launch_center_given(const void* X, int dtype, int64_t t, int n, int64_t ldx, const double* mean,
                                const WsLayout& L, char* ws, int prec, cudaStream_t st);

// Batched tensor-core launch: one descriptor per (dataset, order) and a work
// list of (descriptor, t chunk, row tile, column tile).
struct BatchOrder {
    Shape sh;
    int64_t kchunk;
    int64_t t_pad;
    double* out;               // M_d (S == 1, scaled) or the S partial sums (unscaled)
    double scale;
    int S;
    int box_bytes, slab_bytes;
    const CUtensorMap* map;    // TMA map of the dataset's X~ (device memory, 64-byte aligned)
    const double* xt64;        // the dataset's X~ for the FP64 contraction
    const int* vexp;           // fp16 parts: the dataset's per-variable scale exponents
};

struct BatchUnit {
    int32_t ord, s, I, J;
};

// Per (dataset, order >= 4) of a batch: the correction of Alg. 4-5, in place.
struct BatchCorr {
    double* C;
    const double* M;        // the order-d moments (NULL: in place, read from C)
    const double* low[kMaxOrder + 1];
    int b, nbar;
    int64_t bd, nblocks;
    int64_t block_base;     // prefix of correction blocks (one per stored block)
};

// Largest i with base[i] <= x; `base` is a strided int64 field of an array of
// structs (the prefix counts of the batched kernels' work).
__device__ __forceinline__ int64_t find_segment(const int64_t* base, int64_t count, size_t stride, int64_t x)
{
    int64_t lo = 0, hi = count;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (*(const int64_t*)((const char*)base + mid * stride) <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Batched correction with staged lower-order blocks (correct.cu): `dev` and
// `host` are the same `count` descriptors of one order d, `blocks` their total
// stored blocks.  Sets *done = false, launching nothing, where it does not apply.
cudaError_t launch_batch_correct_staged(int d, const BatchCorr* dev, const BatchCorr* host, int count,
                                        int64_t blocks, cudaStream_t st, bool* done);

int tc_box_rows(int n_pad);
int tc_slab_bytes(int n_pad, int prec);
bool encode_xt_map(CUtensorMap* map, const float* xt, int64_t t_pad, int n_pad);
cudaError_t launch_moment_tc_batch(int prec, int dA, int dB, const BatchOrder* orders, const BatchUnit* units,
                                   int64_t nunits, int max_slab_bytes, double* scratch, int* status, cudaStream_t st);

// CTA-pair launcher (moment_pair.cu): fp16 / bf16 parts, plans with pair set.
cudaError_t launch_moment_pair(const OrderPlan& P, int prec, const float* xt, const float* xlo, int64_t t_pad,
                               const int64_t* prefix, double* out_or_partial, double scale, double* scratch,
                               int* status, const int* vexp, cudaStream_t st);

// One-thread kernel whose bounded wait expires (moment_tc.cu).
cudaError_t launch_bounded_wait_probe(int* status, cudaStream_t st);

// Launcher (moment_tc.cu).
cudaError_t launch_moment_tc(const OrderPlan& P, int prec, const float* xt, int64_t t_pad, const int64_t* prefix,
                             double* out_or_partial, double scale, double* scratch, int* status, const int* vexp,
                             cudaStream_t st);

}  // namespace cum
