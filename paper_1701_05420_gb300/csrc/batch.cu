// Many independent datasets in one fixed launch sequence (batched form of Alg. 5):
// batched centring, one persistent contraction launch per order over the work
// units of every dataset, the t-chunk reduction, and the cumulant correction.
// The plan is built on the host once; cum_batch_run only enqueues kernels, so a
// run can be captured in a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cumgb.h"
#include "internal.h"

namespace cum {

constexpr int64_t kBatchRowsPerChunk = 2048;   // rows per column-sum block
constexpr int kBatchMaxChunks = 256;

// Per-dataset descriptor of the centring kernels.
struct BatchDs {
    const void* X;
    int64_t t, ldx, t_pad;
    int n, n_pad;
    double* partial;        // nchunks x n_pad column-sum partials
    double* mean;           // final mean (n_pad)
    double* mean1;          // first-pass mean (n_pad)
    double* mean_out;       // caller's mean output (may be NULL)
    void* xt;               // X~: n_pad rows of t_pad samples (float or double)
    int64_t rows_per_chunk;
    int nchunks;
    int tiles_n;            // ceil(n_pad / 32)
    int64_t tiles_t;        // t_pad / 32
    int64_t chunk_base;     // prefix over datasets of column-sum blocks
    int64_t tile_base;      // prefix over datasets of transpose blocks
    unsigned* maxabs;       // fp16 parts: max |x~| per variable (float bits), else NULL
    int* vexp;              // fp16 parts: power-of-two scale exponent per variable
    double* rsum;           // split precisions: stored X~ column sums (n_pad), then their divisor t
    int64_t var_base;       // prefix over datasets of padded variables
};

// Per (dataset, order d >= 3) of a split-precision batch: the residual-mean
// correction M -= sum_k m[v_k] Mlow[e without position k] (as in the single
// path's shift_correct_kernel), m = rsum / divisor.
struct BatchShift {
    double* M;              // the order-d moments
    const double* Mlow;     // the order-(d-1) moments
    const double* rsum;
    int b, nbar, n_pad;
    int64_t bd, bdm1;
    int64_t block_base;     // prefix of stored blocks
};

// Per (dataset, order) with split t chunks: partials -> scaled output.
struct BatchRed {
    const double* partial;
    double* out;
    int64_t E;
    double scale;
    int S;
    int64_t block_base;     // prefix of reduction blocks
};


template <typename T>
__global__ void __launch_bounds__(256) batch_colsum_kernel(const BatchDs* __restrict__ ds, int count, int pass)
{
    __shared__ double red[8][33];
    const int64_t i = find_segment(&ds[0].chunk_base, count, sizeof(BatchDs), blockIdx.x);
    const BatchDs& D = ds[i];
    const T* X = (const T*)D.X;
    const int64_t chunk = blockIdx.x - D.chunk_base;
    const int64_t r0 = chunk * D.rows_per_chunk;
    const int64_t r1 = r0 + D.rows_per_chunk < D.t ? r0 + D.rows_per_chunk : D.t;
    for (int c0 = 0; c0 < D.n; c0 += 32) {
        const int c = c0 + threadIdx.x;
        double s = 0.0;
        if (c < D.n) {
            const double m = pass ? D.mean1[c] : 0.0;
            for (int64_t r = r0 + threadIdx.y; r < r1; r += 8) s += (double)X[r * D.ldx + c] - m;
        }
        red[threadIdx.y][threadIdx.x] = s;
        __syncthreads();
        if (threadIdx.y == 0 && c < D.n) {
            double tot = 0.0;
            for (int y = 0; y < 8; ++y) tot += red[y][threadIdx.x];
            D.partial[chunk * D.n_pad + c] = tot;
        }
        __syncthreads();
    }
}

// pass 0: mean1 = sum / t; pass 1: mean = mean1 + sum(x - mean1) / t.
__global__ void batch_mean_kernel(const BatchDs* __restrict__ ds, int pass)
{
    const BatchDs& D = ds[blockIdx.x];
    for (int c = threadIdx.x; c < D.n_pad; c += blockDim.x) {
        double v = 0.0;
        if (c < D.n) {
            double s = 0.0;
            for (int k = 0; k < D.nchunks; ++k) s += D.partial[(int64_t)k * D.n_pad + c];
            v = (pass ? D.mean1[c] : 0.0) + s / (double)D.t;
        }
        if (pass) {
            D.mean[c] = v;
            if (D.mean_out && c < D.n) D.mean_out[c] = v;
        } else {
            D.mean1[c] = v;
            if (D.maxabs) D.maxabs[c] = 0u;
        }
    }
}

// Stochastic rounding of a centred value to FP32 (batched split precisions).
// For float32 input x and an FP64 mean, rounding x - mean to nearest leaves
// the same error for every sample in a binade of |x - mean|, for either sign
// of it: an even function of x.  The residual-mean correction removes its
// average, but its correlation with x^2 biases odd moments by an amount that
// grows like t, against their sampling scale of 1/sqrt(t) (order-3 errors up
// to 1.4e-6 at t near 2e5).  Rounding away from zero with probability
// (v - trunc(v)) / ulp makes the error zero-mean for every sample and
// independent of x.  The uniform variate is a counter-based hash of (dataset,
// variable, sample): a Weyl-sequence key through the 32-bit finaliser of
// Appleby's MurmurHash3, so every run rounds alike.
__device__ __forceinline__ uint32_t mix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ float round_stochastic(double v, uint32_t key)
{
    const float h = __double2float_rz(v);                            // toward zero, the sign of v
    const float r = fabsf((float)(v - (double)h));                   // the remainder, below one ulp
    const float up = __uint_as_float(__float_as_uint(h) + 1u);       // next float away from zero
    const float ulp = fabsf(up - h);                                 // exact: a power of two
    const float u = (float)(mix32(key) >> 8) * 0x1.0p-24f;           // uniform on [0, 1), 24 bits
    return u * ulp < r ? up : h;                                     // away with probability r / ulp
}

template <typename T, typename Tout>
__global__ void __launch_bounds__(256) batch_center_kernel(const BatchDs* __restrict__ ds, int count)
{
    __shared__ double tile[32][33];
    const int64_t i = find_segment(&ds[0].tile_base, count, sizeof(BatchDs), blockIdx.x);
    const BatchDs& D = ds[i];
    const T* X = (const T*)D.X;
    Tout* xt = (Tout*)D.xt;
    const int64_t k = blockIdx.x - D.tile_base;
    const int64_t l0 = (k / D.tiles_n) * 32;
    const int c0 = (int)(k % D.tiles_n) * 32;
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int64_t l = l0 + y;
        const int c = c0 + threadIdx.x;
        double v = 0.0;
        if (l < D.t && c < D.n) v = (double)X[l * D.ldx + c] - D.mean[c];
        tile[y][threadIdx.x] = v;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int c = c0 + y;                       // uniform across the warp
        const int64_t l = l0 + threadIdx.x;
        Tout v;
        if constexpr (std::is_same<Tout, float>::value)
            v = round_stochastic(tile[threadIdx.x][y], (uint32_t)l * 0x9e3779b9u + (uint32_t)c * 0x7f4a7c15u +
                                                           (uint32_t)i * 0x632be5abu);
        else
            v = (Tout)tile[threadIdx.x][y];
        if (c < D.n_pad && l < D.t_pad) xt[(int64_t)c * D.t_pad + l] = v;
        if (D.maxabs) {
            const uint32_t w = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf((float)v)));
            if (threadIdx.x == 0 && c < D.n_pad && w) atomicMax(D.maxabs + c, w);
        }
    }
}

// fp16 parts: X~^T[c][l] *= 2^s_c per 32 x 32 tile (the transpose's tiling);
// tiles at l0 = 0 store s_c.
__global__ void __launch_bounds__(256) batch_scale_kernel(const BatchDs* __restrict__ ds, int count)
{
    const int64_t i = find_segment(&ds[0].tile_base, count, sizeof(BatchDs), blockIdx.x);
    const BatchDs& D = ds[i];
    float* xt = (float*)D.xt;
    const int64_t k = blockIdx.x - D.tile_base;
    const int64_t l0 = (k / D.tiles_n) * 32;
    const int c0 = (int)(k % D.tiles_n) * 32;
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int c = c0 + y;
        if (c >= D.n_pad) break;
        const int s = fp16_scale_exponent(D.maxabs[c]);
        if (l0 == 0 && threadIdx.x == 0) D.vexp[c] = s;
        xt[(int64_t)c * D.t_pad + l0 + threadIdx.x] *= __int_as_float((127 + s) << 23);
    }
}

// Split precisions: column sums (FP64, fixed order) of each dataset's stored
// X~ before any fp16 scaling, one CTA per (dataset, padded variable):
// rsum[c] = sum_l X~^T[c][l], rsum[n_pad] = t.
__global__ void __launch_bounds__(256) batch_resid_kernel(const BatchDs* __restrict__ ds, int count)
{
    __shared__ double red[256];
    const int64_t i = find_segment(&ds[0].var_base, count, sizeof(BatchDs), blockIdx.x);
    const BatchDs& D = ds[i];
    const int c = (int)(blockIdx.x - D.var_base);
    const float4* row = (const float4*)((const float*)D.xt + (int64_t)c * D.t_pad);
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < D.t_pad / 4; k += 256) {
        const float4 v = row[k];
        s += ((double)v.x + (double)v.y) + ((double)v.z + (double)v.w);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        D.rsum[c] = red[0];
        if (c == 0) D.rsum[D.n_pad] = (double)D.t;
    }
}

// One CTA per (dataset, stored block) of order D: the residual-mean correction.
template <int D>
__global__ void __launch_bounds__(256) batch_shift_kernel(const BatchShift* __restrict__ sh, int count)
{
    __shared__ int64_t sub[D];
    __shared__ int jb[D];
    const int64_t i = find_segment(&sh[0].block_base, count, sizeof(BatchShift), blockIdx.x);
    const BatchShift& S = sh[i];
    const int64_t r = blockIdx.x - S.block_base;
    const int b = S.b;
    if (threadIdx.x == 0) {
        int j[D];
        colex_unrank(r, D, S.nbar, j);
        for (int k = 0; k < D; ++k) {
            jb[k] = j[k];
            int js[D];
            int q = 0;
            for (int k2 = 0; k2 < D; ++k2)
                if (k2 != k) js[q++] = j[k2];
            sub[k] = colex_rank(js, D - 1) * S.bdm1;
        }
    }
    __syncthreads();
    const double inv_t = 1.0 / S.rsum[S.n_pad];
    for (int64_t e = threadIdx.x; e < S.bd; e += blockDim.x) {
        int dig[D];
        int64_t x = e;
#pragma unroll
        for (int k = D - 1; k >= 0; --k) {
            dig[k] = (int)(x % b);
            x /= b;
        }
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            int64_t o = 0;
#pragma unroll
            for (int k2 = 0; k2 < D; ++k2)
                if (k2 != k) o = o * b + dig[k2];
            acc += S.rsum[jb[k] * b + dig[k]] * S.Mlow[sub[k] + o];
        }
        S.M[r * S.bd + e] -= acc * inv_t;
    }
}

constexpr int kRedBlock = 256 * 16;   // entries per reduction block

__global__ void __launch_bounds__(256) batch_reduce_kernel(const BatchRed* __restrict__ rd, int count)
{
    const int64_t i = find_segment(&rd[0].block_base, count, sizeof(BatchRed), blockIdx.x);
    const BatchRed& R = rd[i];
    const int64_t e0 = (blockIdx.x - R.block_base) * kRedBlock;
    for (int64_t e = e0 + threadIdx.x; e < e0 + kRedBlock && e < R.E; e += blockDim.x) {
        double acc = 0.0;
        for (int s = 0; s < R.S; ++s) acc += R.partial[(int64_t)s * R.E + e];
        R.out[e] = acc * R.scale;
    }
}

// Correction of one stored block per CTA: C = M - sum over the partitions of
// 1:d into parts of size >= 2 of the products of lower-order cumulants (the
// block-level form of Alg. 4-5, as in correct_kernel).
__global__ void __launch_bounds__(256) batch_correct_kernel(const BatchCorr* __restrict__ cr, int count, int d,
                                                            PartTable pt)
{
    __shared__ int64_t base[kMaxPartitions][kMaxParts];
    __shared__ int plen[kMaxPartitions][kMaxParts];
    const int64_t i = find_segment(&cr[0].block_base, count, sizeof(BatchCorr), blockIdx.x);
    const BatchCorr& K = cr[i];
    const int64_t r = blockIdx.x - K.block_base;
    const int b = K.b;
    int j[kMaxOrder];
    colex_unrank(r, d, K.nbar, j);
    for (int z = threadIdx.x; z < pt.count; z += blockDim.x) {
        for (int q = 0; q < pt.nparts[z]; ++q) {
            int js[kMaxOrder];
            int len = 0;
            for (int k = 0; k < d; ++k)
                if (pt.mask[z][q] & (1u << k)) js[len++] = j[k];
            plen[z][q] = len;
            base[z][q] = colex_rank(js, len) * ipow(b, len);
        }
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < K.bd; e += blockDim.x) {
        int ix[kMaxOrder];
        int64_t rem = e;
        for (int k = d - 1; k >= 0; --k) {
            ix[k] = (int)(rem % b);
            rem /= b;
        }
        double sum = 0.0;
        for (int z = 0; z < pt.count; ++z) {
            double prod = 1.0;
            for (int q = 0; q < pt.nparts[z]; ++q) {
                int64_t off = 0;
                for (int k = 0; k < d; ++k)
                    if (pt.mask[z][q] & (1u << k)) off = off * b + ix[k];
                prod *= K.low[plen[z][q]][base[z][q] + off];
            }
            sum += prod;
        }
        K.C[r * K.bd + e] = (K.M ? K.M : K.C)[r * K.bd + e] - sum;
    }
}

}  // namespace cum

// ---------------------------------------------------------------------- plan object

struct cum_batch_s {
    int count = 0, d_max = 0, prec = 0, dtype = 0;
    std::vector<int64_t> t;
    std::vector<int> n, b;
    // workspace layout (byte offsets)
    size_t off_ds = 0, off_ord = 0, off_red = 0, off_corr = 0, off_shift = 0, off_maps = 0, off_units = 0,
           off_data = 0, off_scratch = 0, total = 0;
    std::vector<size_t> ds_partial, ds_mean, ds_xt, ord_partial;   // per dataset / per (dataset, order)
    std::vector<size_t> ds_m4, ds_m5;   // split precisions: kept order-4 / order-5 moments (0: none)
    std::vector<cum::OrderPlan> plans;                               // per (dataset, order)
    std::vector<size_t> units_off;                                   // per order: byte offset of its unit list
    std::vector<int64_t> units_n;                                    // per order: number of units
    std::vector<std::vector<cum::BatchUnit>> units;                  // per order
    int64_t colsum_blocks = 0, center_blocks = 0;
    int max_slab = 0;
    // bound state
    bool bound = false;
    char* ws = nullptr;
    std::vector<cum::BatchDs> ds_dev;
    std::vector<cum::BatchOrder> ord_dev;
    std::vector<cum::BatchRed> red_dev;
    std::vector<int> red_first;                                      // per order: first index into red_dev
    std::vector<int64_t> red_blocks;                                 // per order: reduction blocks
    std::vector<cum::BatchCorr> corr_dev;
    std::vector<int> corr_first;
    std::vector<int64_t> corr_blocks;
    std::vector<cum::BatchShift> shift_dev;
    std::vector<int> shift_first;
    std::vector<int64_t> shift_blocks;
    int64_t vars = 0;                                                // padded variables of all datasets
    std::vector<CUtensorMap> maps;
};

namespace {

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

int ord_index(const cum_batch_s* B, int i, int d) { return i * (B->d_max - 1) + (d - 2); }

}  // namespace

using namespace cum;

static int batch_run_impl(cum_batch B, void* stream);   // the launch sequence of cum_batch_run

extern "C" {

int cum_batch_plan(int count, const int64_t* t, const int* n, const int* b, int d_max, int prec, int dtype,
                   cum_batch* plan, size_t* ws_bytes)
{
    if (!plan || !ws_bytes || count < 1 || !t || !n || !b || d_max < 2 || d_max > kMaxOrder) return CUM_EINVAL;
    if (dtype != CUM_F32 && dtype != CUM_F64) return CUM_EINVAL;
    if (prec != CUM_PREC_FP64 && prec != CUM_PREC_BF16X3 && prec != CUM_PREC_TF32X3 && prec != CUM_PREC_FP16X3)
        return CUM_EINVAL;
    const bool tc = prec != CUM_PREC_FP64;
    cum_batch_s* B = new cum_batch_s;
    B->count = count;
    B->d_max = d_max;
    B->prec = prec;
    B->dtype = dtype;
    B->t.assign(t, t + count);
    B->n.assign(n, n + count);
    B->b.assign(b, b + count);
    const int nord = d_max - 1;
    for (int i = 0; i < count; ++i) {
        if (cum_workspace_size(t[i], n[i], d_max, b[i], prec) == 0) {
            delete B;
            return CUM_EUNSUPPORTED;
        }
    }
    B->plans.resize((size_t)count * nord);
    B->units.assign(kMaxOrder + 1, {});
    for (int i = 0; i < count; ++i)
        for (int d = 2; d <= d_max; ++d) B->plans[ord_index(B, i, d)] = make_order_plan(d, t[i], n[i], b[i], prec, false);
    if (tc) {
        // The units of all datasets share the CTAs, so each dataset's t axis is
        // split only as far as it takes to keep its units within an eighth of
        // a CTA's average work (a unit costs its 128-sample steps plus about
        // kTcUnitSteps): a dataset planned alone would split to fill the GPU by
        // itself, and pay the per-unit cost many times over.
        for (int d = 2; d <= d_max; ++d) {
            int64_t work = 0;
            for (int i = 0; i < count; ++i)
                work += B->plans[ord_index(B, i, d)].active_tiles * (pad_t(t[i]) / 128 + kTcUnitSteps);
            int64_t cap = (work + 8 * kTcPlanCtas - 1) / (8 * kTcPlanCtas);
            if (cap < 16) cap = 16;
            for (int i = 0; i < count; ++i) {
                OrderPlan& P = B->plans[ord_index(B, i, d)];
                int64_t S = (pad_t(t[i]) / 128 + cap - 1) / cap;
                const int64_t smax = max_order_splits(P, t[i], prec);
                set_order_splits(P, t[i], prec, S < smax ? S : smax);
            }
        }
    }
    for (int i = 0; i < count; ++i) {
        for (int d = 2; d <= d_max; ++d) {
            const OrderPlan& P = B->plans[ord_index(B, i, d)];
            // work units of this (dataset, order): every active tile x every t chunk
            for (int64_t I = 0; I < P.row_tiles; ++I) {
                int j[kMaxHalf];
                colex_unrank((I * P.tile_m) / P.sh.bdA, P.sh.dA, P.sh.nbar, j);
                const int64_t cols = cols_with_first_at_least(j[P.sh.dA - 1], P.sh.dB, P.sh.nbar, P.sh.bdB);
                const int64_t nct = (cols + P.tile_n - 1) / P.tile_n;
                for (int64_t J = 0; J < nct; ++J)
                    for (int s = 0; s < P.splits; ++s)
                        B->units[d].push_back(BatchUnit{ord_index(B, i, d), s, (int32_t)I, (int32_t)J});
            }
        }
    }
    // longest units first (their chunk length), so the persistent CTAs finish together
    for (int d = 2; d <= d_max; ++d) {
        auto& U = B->units[d];
        std::stable_sort(U.begin(), U.end(), [&](const BatchUnit& x, const BatchUnit& y) {
            const OrderPlan& px = B->plans[x.ord];
            const OrderPlan& py = B->plans[y.ord];
            return px.kchunk > py.kchunk;
        });
    }
    // workspace layout
    size_t off = 256;   // status word
    B->off_ds = off;
    off = a256(off + sizeof(BatchDs) * count);
    B->off_ord = off;
    off = a256(off + sizeof(BatchOrder) * count * nord);
    B->off_red = off;
    off = a256(off + sizeof(BatchRed) * count * nord);
    B->off_corr = off;
    off = a256(off + sizeof(BatchCorr) * count * nord);
    B->off_shift = off;
    off = a256(off + sizeof(BatchShift) * count * nord);
    B->off_maps = off;
    off = a256(off + sizeof(CUtensorMap) * count);
    B->units_off.assign(kMaxOrder + 1, 0);
    B->units_n.assign(kMaxOrder + 1, 0);
    for (int d = 2; d <= d_max; ++d) {
        B->units_off[d] = off;
        B->units_n[d] = (int64_t)B->units[d].size();
        off = a256(off + sizeof(BatchUnit) * B->units[d].size());
    }
    B->off_data = off;
    B->ds_partial.resize(count);
    B->ds_mean.resize(count);
    B->ds_xt.resize(count);
    B->colsum_blocks = 0;
    B->center_blocks = 0;
    for (int i = 0; i < count; ++i) {
        const int nbar = (n[i] + b[i] - 1) / b[i];
        const int n_pad = nbar * b[i];
        const int64_t t_pad = pad_t(t[i]);
        int64_t rpc = kBatchRowsPerChunk;
        while ((t[i] + rpc - 1) / rpc > kBatchMaxChunks) rpc *= 2;
        const int nchunks = (int)((t[i] + rpc - 1) / rpc);
        B->ds_partial[i] = off;
        off = a256(off + sizeof(double) * (size_t)nchunks * n_pad);
        B->ds_mean[i] = off;
        // mean, first-pass mean, maxabs and vexp (4 bytes each), residual sums + divisor
        off = a256(off + sizeof(double) * 2 * (size_t)n_pad + 8 * (size_t)n_pad + sizeof(double) * ((size_t)n_pad + 1));
        B->ds_xt[i] = off;
        off = a256(off + (tc ? sizeof(float) : sizeof(double)) * (size_t)n_pad * (size_t)t_pad);
        B->colsum_blocks += nchunks;
        B->center_blocks += (t_pad / 32) * ((n_pad + 31) / 32);
        if (tc) B->max_slab = std::max(B->max_slab, tc_slab_bytes(n_pad, prec));
    }
    B->ds_m4.assign(count, 0);
    B->ds_m5.assign(count, 0);
    if (tc)
        for (int i = 0; i < count; ++i) {
            const int nbar = (n[i] + b[i] - 1) / b[i];
            if (d_max >= 5) {
                B->ds_m4[i] = off;
                off = a256(off + sizeof(double) * (size_t)(num_blocks(nbar, 4) * ipow(b[i], 4)));
            }
            if (d_max >= 6) {
                B->ds_m5[i] = off;
                off = a256(off + sizeof(double) * (size_t)(num_blocks(nbar, 5) * ipow(b[i], 5)));
            }
        }
    B->ord_partial.assign((size_t)count * nord, 0);
    for (int i = 0; i < count; ++i)
        for (int d = 2; d <= d_max; ++d) {
            const OrderPlan& P = B->plans[ord_index(B, i, d)];
            if (P.splits > 1) {
                B->ord_partial[ord_index(B, i, d)] = off;
                off = a256(off + sizeof(double) * (size_t)P.splits * (size_t)P.sh.entries);
            }
        }
    B->off_scratch = off;
    if (tc) off = a256(off + sizeof(double) * (size_t)kTcMaxCtas * kTcTileM * kTcTileN);
    B->total = off;
    *plan = B;
    *ws_bytes = B->total;
    return CUM_OK;
}

int cum_batch_bind(cum_batch B, const void* const* X, const int64_t* ldx, double* const* C_out,
                   double* const* mean_out, void* ws, size_t ws_bytes, void* stream)
{
    if (!B || !X || !C_out || !ws) return CUM_EINVAL;
    if (((uintptr_t)ws % kWsAlign) != 0 || ws_bytes < B->total) return CUM_EWORKSPACE;
    const int count = B->count, nord = B->d_max - 1;
    const bool tc = B->prec != CUM_PREC_FP64;
    char* w = (char*)ws;
    for (int i = 0; i < count; ++i) {
        if (!X[i]) return CUM_EINVAL;
        if (ldx && ldx[i] < B->n[i]) return CUM_EINVAL;
        for (int d = 2; d <= B->d_max; ++d)
            if (!C_out[ord_index(B, i, d)]) return CUM_EINVAL;
    }
    B->ds_dev.assign(count, BatchDs{});
    B->maps.assign(count, CUtensorMap{});
    int64_t chunk_base = 0, tile_base = 0, var_base = 0;
    for (int i = 0; i < count; ++i) {
        BatchDs& D = B->ds_dev[i];
        const int nbar = (B->n[i] + B->b[i] - 1) / B->b[i];
        D.X = X[i];
        D.t = B->t[i];
        D.ldx = ldx ? ldx[i] : B->n[i];
        D.n = B->n[i];
        D.n_pad = nbar * B->b[i];
        D.t_pad = pad_t(B->t[i]);
        int64_t rpc = kBatchRowsPerChunk;
        while ((D.t + rpc - 1) / rpc > kBatchMaxChunks) rpc *= 2;
        D.rows_per_chunk = rpc;
        D.nchunks = (int)((D.t + rpc - 1) / rpc);
        D.partial = (double*)(w + B->ds_partial[i]);
        D.mean = (double*)(w + B->ds_mean[i]);
        D.mean1 = D.mean + D.n_pad;
        D.maxabs = B->prec == CUM_PREC_FP16X3 ? (unsigned*)(D.mean1 + D.n_pad) : nullptr;
        D.vexp = B->prec == CUM_PREC_FP16X3 ? (int*)(D.maxabs + D.n_pad) : nullptr;
        D.rsum = tc ? (double*)((char*)(D.mean1 + D.n_pad) + 8 * (size_t)D.n_pad) : nullptr;
        D.var_base = var_base;
        var_base += D.n_pad;
        D.mean_out = mean_out ? mean_out[i] : nullptr;
        D.xt = w + B->ds_xt[i];
        D.tiles_n = (D.n_pad + 31) / 32;
        D.tiles_t = D.t_pad / 32;
        D.chunk_base = chunk_base;
        D.tile_base = tile_base;
        chunk_base += D.nchunks;
        tile_base += D.tiles_t * D.tiles_n;
        if (tc && !encode_xt_map(&B->maps[i], (const float*)D.xt, D.t_pad, D.n_pad)) return CUM_EUNSUPPORTED;
    }
    CUtensorMap* maps_dev = (CUtensorMap*)(w + B->off_maps);
    B->ord_dev.assign((size_t)count * nord, BatchOrder{});
    B->red_dev.clear();
    B->red_first.assign(kMaxOrder + 2, 0);
    B->red_blocks.assign(kMaxOrder + 1, 0);
    B->vars = var_base;
    B->corr_dev.clear();
    B->corr_first.assign(kMaxOrder + 2, 0);
    B->corr_blocks.assign(kMaxOrder + 1, 0);
    B->shift_dev.clear();
    B->shift_first.assign(kMaxOrder + 2, 0);
    B->shift_blocks.assign(kMaxOrder + 1, 0);
    for (int d = 2; d <= B->d_max; ++d) {
        B->red_first[d] = (int)B->red_dev.size();
        B->corr_first[d] = (int)B->corr_dev.size();
        B->shift_first[d] = (int)B->shift_dev.size();
        int64_t rblocks = 0, cblocks = 0, sblocks = 0;
        for (int i = 0; i < count; ++i) {
            const int k = ord_index(B, i, d);
            const OrderPlan& P = B->plans[k];
            const BatchDs& D = B->ds_dev[i];
            BatchOrder& O = B->ord_dev[k];
            // split precisions keep the raw order-4 (d_max >= 5) and order-5
            // (d_max >= 6) moments: the next order's residual-mean correction reads them
            double* Mdst = C_out[k];
            if (tc && d == 4 && B->ds_m4[i]) Mdst = (double*)(w + B->ds_m4[i]);
            if (tc && d == 5 && B->ds_m5[i]) Mdst = (double*)(w + B->ds_m5[i]);
            O.sh = P.sh;
            O.kchunk = P.kchunk;
            O.t_pad = D.t_pad;
            O.S = P.splits;
            O.scale = P.splits > 1 ? 1.0 : 1.0 / (double)D.t;
            O.out = P.splits > 1 ? (double*)(w + B->ord_partial[k]) : Mdst;
            O.box_bytes = tc ? tc_box_rows(D.n_pad) * 128 : 0;
            O.slab_bytes = tc ? tc_slab_bytes(D.n_pad, B->prec) : 0;
            O.map = tc ? maps_dev + i : nullptr;
            O.xt64 = tc ? nullptr : (const double*)D.xt;
            O.vexp = D.vexp;
            if (P.splits > 1) {
                BatchRed R;
                R.partial = O.out;
                R.out = Mdst;
                R.E = P.sh.entries;
                R.scale = 1.0 / (double)D.t;
                R.S = P.splits;
                R.block_base = rblocks;
                rblocks += (R.E + kRedBlock - 1) / kRedBlock;
                B->red_dev.push_back(R);
            }
            if (d >= 4) {
                BatchCorr K;
                std::memset(&K, 0, sizeof(K));
                K.C = C_out[k];
                K.M = Mdst != C_out[k] ? Mdst : nullptr;
                for (int q = 2; q <= d - 2; ++q) K.low[q] = C_out[ord_index(B, i, q)];
                K.b = B->b[i];
                K.nbar = P.sh.nbar;
                K.bd = P.sh.bd;
                K.nblocks = num_blocks(P.sh.nbar, d);
                K.block_base = cblocks;
                cblocks += K.nblocks;
                B->corr_dev.push_back(K);
            }
            if (tc && d >= 3) {
                BatchShift S;
                std::memset(&S, 0, sizeof(S));
                S.M = Mdst;
                S.Mlow = d == 3 ? C_out[ord_index(B, i, 2)]
                       : d == 4 ? C_out[ord_index(B, i, 3)]
                       : d == 5 ? (const double*)(w + B->ds_m4[i])
                                : (const double*)(w + B->ds_m5[i]);
                S.rsum = D.rsum;
                S.b = B->b[i];
                S.nbar = P.sh.nbar;
                S.n_pad = D.n_pad;
                S.bd = P.sh.bd;
                S.bdm1 = ipow(B->b[i], d - 1);
                S.block_base = sblocks;
                sblocks += num_blocks(P.sh.nbar, d);
                B->shift_dev.push_back(S);
            }
        }
        B->red_blocks[d] = rblocks;
        B->corr_blocks[d] = cblocks;
        B->shift_blocks[d] = sblocks;
    }
    B->red_first[B->d_max + 1] = (int)B->red_dev.size();
    B->corr_first[B->d_max + 1] = (int)B->corr_dev.size();
    B->shift_first[B->d_max + 1] = (int)B->shift_dev.size();
    // upload the tables (host memory owned by the plan; the copy completes before return)
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(w + B->off_ds, B->ds_dev.data(), sizeof(BatchDs) * count,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + B->off_ord, B->ord_dev.data(), sizeof(BatchOrder) * B->ord_dev.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !B->red_dev.empty())
        e = cudaMemcpyAsync(w + B->off_red, B->red_dev.data(), sizeof(BatchRed) * B->red_dev.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !B->corr_dev.empty())
        e = cudaMemcpyAsync(w + B->off_corr, B->corr_dev.data(), sizeof(BatchCorr) * B->corr_dev.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !B->shift_dev.empty())
        e = cudaMemcpyAsync(w + B->off_shift, B->shift_dev.data(), sizeof(BatchShift) * B->shift_dev.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && tc)
        e = cudaMemcpyAsync(w + B->off_maps, B->maps.data(), sizeof(CUtensorMap) * count, cudaMemcpyHostToDevice,
                            st);
    for (int d = 2; d <= B->d_max && e == cudaSuccess; ++d)
        if (!B->units[d].empty())
            e = cudaMemcpyAsync(w + B->units_off[d], B->units[d].data(), sizeof(BatchUnit) * B->units[d].size(),
                                cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    B->ws = w;
    B->bound = true;
    return CUM_OK;
}

int cum_batch_run(cum_batch B, void* stream)
{
    if (!B || !B->bound) return CUM_EINVAL;
    nvtxRangePushA("cum_batch_run");
    const int rc = batch_run_impl(B, stream);
    nvtxRangePop();
    return rc;
}

}  // extern "C"

static int batch_run_impl(cum_batch B, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    char* w = B->ws;
    const int count = B->count;
    const bool tc = B->prec != CUM_PREC_FP64;
    const BatchDs* ds = (const BatchDs*)(w + B->off_ds);
    cudaError_t e = cudaMemsetAsync(w, 0, 256, st);
    if (e != cudaSuccess) return cuda_fail(e);
    const dim3 blk(32, 8);
    const unsigned cs = (unsigned)B->colsum_blocks, cb = (unsigned)B->center_blocks;
    if (B->dtype == CUM_F64) {
        batch_colsum_kernel<double><<<cs, blk, 0, st>>>(ds, count, 0);
        batch_mean_kernel<<<count, 128, 0, st>>>(ds, 0);
        batch_colsum_kernel<double><<<cs, blk, 0, st>>>(ds, count, 1);
        batch_mean_kernel<<<count, 128, 0, st>>>(ds, 1);
        if (tc) batch_center_kernel<double, float><<<cb, blk, 0, st>>>(ds, count);
        else batch_center_kernel<double, double><<<cb, blk, 0, st>>>(ds, count);
    } else {
        batch_colsum_kernel<float><<<cs, blk, 0, st>>>(ds, count, 0);
        batch_mean_kernel<<<count, 128, 0, st>>>(ds, 0);
        batch_colsum_kernel<float><<<cs, blk, 0, st>>>(ds, count, 1);
        batch_mean_kernel<<<count, 128, 0, st>>>(ds, 1);
        if (tc) batch_center_kernel<float, float><<<cb, blk, 0, st>>>(ds, count);
        else batch_center_kernel<float, double><<<cb, blk, 0, st>>>(ds, count);
    }
    if (tc) batch_resid_kernel<<<(unsigned)B->vars, 256, 0, st>>>(ds, count);   // before the fp16 scaling
    if (B->prec == CUM_PREC_FP16X3) batch_scale_kernel<<<cb, blk, 0, st>>>(ds, count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    const BatchOrder* ord = (const BatchOrder*)(w + B->off_ord);
    for (int d = 2; d <= B->d_max; ++d) {
        const int dA = (d + 1) / 2, dB = d / 2;
        const BatchUnit* units = (const BatchUnit*)(w + B->units_off[d]);
        if (tc)
            e = launch_moment_tc_batch(B->prec, dA, dB, ord, units, B->units_n[d], B->max_slab,
                                       (double*)(w + B->off_scratch), (int*)w, st);
        else
            e = launch_moment_fp64_batch(dA, dB, ord, units, B->units_n[d], st);
        if (e != cudaSuccess) return cuda_fail(e);
        const int r0 = B->red_first[d], r1 = B->red_first[d + 1];
        if (r1 > r0) {
            batch_reduce_kernel<<<(unsigned)B->red_blocks[d], 256, 0, st>>>((const BatchRed*)(w + B->off_red) + r0,
                                                                           r1 - r0);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e);
        }
        const int s0 = B->shift_first[d], s1 = B->shift_first[d + 1];
        if (s1 > s0) {
            const BatchShift* shd = (const BatchShift*)(w + B->off_shift) + s0;
            const unsigned nb = (unsigned)B->shift_blocks[d];
            switch (d) {
            case 3: batch_shift_kernel<3><<<nb, 256, 0, st>>>(shd, s1 - s0); break;
            case 4: batch_shift_kernel<4><<<nb, 256, 0, st>>>(shd, s1 - s0); break;
            case 5: batch_shift_kernel<5><<<nb, 256, 0, st>>>(shd, s1 - s0); break;
            default: batch_shift_kernel<6><<<nb, 256, 0, st>>>(shd, s1 - s0); break;
            }
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e);
        }
        if (d >= 4) {
            const int c0 = B->corr_first[d], c1 = B->corr_first[d + 1];
            bool done = false;
            e = launch_batch_correct_staged(d, (const BatchCorr*)(w + B->off_corr) + c0, B->corr_dev.data() + c0,
                                            c1 - c0, B->corr_blocks[d], st, &done);
            if (e != cudaSuccess) return cuda_fail(e);
            if (done) continue;
            PartTable pt = make_part_table(d);
            batch_correct_kernel<<<(unsigned)B->corr_blocks[d], 256, 0, st>>>(
                (const BatchCorr*)(w + B->off_corr) + c0, c1 - c0, d, pt);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e);
        }
    }
    return CUM_OK;
}

extern "C" {

int cum_batch_info(cum_batch B, int64_t* info)
{
    if (!B || !info) return CUM_EINVAL;
    const bool tc = B->prec != CUM_PREC_FP64;
    int64_t units = 0, launches = 5 + (tc ? 1 : 0) + (B->prec == CUM_PREC_FP16X3 ? 1 : 0);
    for (int d = 2; d <= B->d_max; ++d) {
        units += B->units_n[d];
        launches += 1 + (tc && d >= 3 ? 1 : 0);
        if (B->bound && B->red_first[d + 1] > B->red_first[d]) launches += 1;
        if (d >= 4) launches += 1;
    }
    info[0] = B->count;
    info[1] = units;
    info[2] = launches;
    info[3] = (int64_t)B->total;
    return CUM_OK;
}

void cum_batch_free(cum_batch B) { delete B; }

}  // extern "C"
