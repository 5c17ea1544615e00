// Centring (Def. 1.3), tile planning, the FP64 moment contraction (Alg. 1-2 on
// CUDA cores), the t-chunk reduction (Alg. 3, Eq. mapred) and the cumulant
// correction (Alg. 4-5, Eq. cum_r).
#include <climits>
#include <cstring>

#include "cumgb.h"
#include "internal.h"

namespace cum {

// ------------------------------------------------------------------ centring

// Per-chunk column sums of (X - shift) in FP64.  Block (32, 8): x = column in
// a group of 32, y = row lane.  partial: [gridDim.x][n_pad].
template <typename T>
__global__ void __launch_bounds__(256) colsum_kernel(const T* __restrict__ X, int64_t t, int n, int64_t ldx,
                                                     const double* __restrict__ shift, int64_t rows_per_chunk,
                                                     double* __restrict__ partial, int n_pad)
{
    __shared__ double red[8][33];
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
    const int64_t r1 = r0 + rows_per_chunk < t ? r0 + rows_per_chunk : t;
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int c = c0 + threadIdx.x;
        double s = 0.0;
        if (c < n) {
            const double m = shift ? shift[c] : 0.0;
            for (int64_t r = r0 + threadIdx.y; r < r1; r += 8) s += (double)X[r * ldx + c] - m;
        }
        red[threadIdx.y][threadIdx.x] = s;
        __syncthreads();
        if (threadIdx.y == 0 && c < n) {
            double tot = 0.0;
            for (int y = 0; y < 8; ++y) tot += red[y][threadIdx.x];
            partial[(int64_t)blockIdx.x * n_pad + c] = tot;
        }
        __syncthreads();
    }
}

// mean[c] = shift[c] + (sum_chunks partial[chunk][c]) / t   (shift may be NULL)
__global__ void mean_finalize_kernel(const double* __restrict__ partial, int nchunks, int n, int n_pad, int64_t t,
                                     const double* __restrict__ shift, double* __restrict__ mean,
                                     double* __restrict__ mean_out)
{
    for (int c = threadIdx.x; c < n_pad; c += blockDim.x) {
        double v = 0.0;
        if (c < n) {
            double s = 0.0;
            for (int k = 0; k < nchunks; ++k) s += partial[(int64_t)k * n_pad + c];
            v = (shift ? shift[c] : 0.0) + s / (double)t;
        }
        mean[c] = v;
        if (mean_out && c < n) mean_out[c] = v;
    }
}

// X~^T[c][l] = x_{l,c} - mean_c, zero for padded l or c.  Tiles of 32 x 32,
// block (32, 8), grid-stride over the sample axis.  With `maxabs` set, also
// records max_l |X~^T[c][l]| (of the stored value, as float bits) per variable;
// with `xlo` set (FP32 output), also stores the remainder of the FP64 value,
// RN32(x~ - X~^T), so that X~^T + xlo is a double-float X~.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) center_transpose_kernel(const Tin* __restrict__ X, int64_t t, int n,
                                                               int64_t ldx, const double* __restrict__ mean,
                                                               Tout* __restrict__ xt, int64_t t_pad, int n_pad,
                                                               unsigned* __restrict__ maxabs,
                                                               float* __restrict__ xlo)
{
    __shared__ double tile[32][33];
    const int c0 = blockIdx.y * 32;
    uint32_t m[4] = {0u, 0u, 0u, 0u};
    for (int64_t l0 = (int64_t)blockIdx.x * 32; l0 < t_pad; l0 += (int64_t)gridDim.x * 32) {
        for (int y = threadIdx.y; y < 32; y += 8) {
            const int64_t l = l0 + y;
            const int c = c0 + threadIdx.x;
            double v = 0.0;
            if (l < t && c < n) v = (double)X[l * ldx + c] - mean[c];
            tile[y][threadIdx.x] = v;
        }
        __syncthreads();
        for (int y = threadIdx.y, k = 0; y < 32; y += 8, ++k) {
            const int c = c0 + y;
            const int64_t l = l0 + threadIdx.x;
            const double v64 = tile[threadIdx.x][y];
            const Tout v = (Tout)v64;
            if (c < n_pad && l < t_pad) {
                xt[(int64_t)c * t_pad + l] = v;
                if (xlo) xlo[(int64_t)c * t_pad + l] = (float)(v64 - (double)v);
            }
            const uint32_t a = __float_as_uint(fabsf((float)v));
            m[k] = a > m[k] ? a : m[k];
        }
        __syncthreads();
    }
    if (maxabs) {
        for (int y = threadIdx.y, k = 0; y < 32; y += 8, ++k) {
            const int c = c0 + y;                       // uniform across the warp
            const uint32_t w = __reduce_max_sync(0xffffffffu, m[k]);
            if (threadIdx.x == 0 && c < n_pad && w) atomicMax(maxabs + c, w);
        }
    }
}

// s_c = fp16_scale_exponent(maxabs[c]) into vexp[c]; for fp16 parts (apply)
// also X~^T[c][:] *= 2^s_c and xlo[c][:] *= 2^s_c, exact in float.  Grid
// (chunks of the row, n_pad); block x == 0 stores s_c.
__global__ void __launch_bounds__(256) scale_rows_kernel(float* __restrict__ xt, float* __restrict__ xlo, int64_t t_pad,
                                                         const unsigned* __restrict__ maxabs, int* __restrict__ vexp,
                                                         int apply)
{
    const int c = blockIdx.y;
    const int s = fp16_scale_exponent(maxabs[c]);
    if (blockIdx.x == 0 && threadIdx.x == 0) vexp[c] = s;
    if (!apply) return;
    const float f = __int_as_float((127 + s) << 23);
    const int64_t n4 = t_pad / 4;
    for (int k = 0; k < 2; ++k) {
        float4* row = (float4*)((k == 0 ? xt : xlo) + (int64_t)c * t_pad);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
            float4 v = row[i];
            v.x *= f;
            v.y *= f;
            v.z *= f;
            v.w *= f;
            row[i] = v;
        }
    }
}

// Split precisions: column sums (FP64, fixed reduction order) of the centred
// array as stored in FP32, before any fp16 scaling: rsum[c] = sum_l X~^T[c][l],
// and rsum[n_pad] = `divisor`.  Rounding X - mean to FP32 leaves each column
// with a small residual mean rsum[c] / t; shift_correct_kernel removes its
// first-order effect on the moments.  A shard centred by a global mean passes
// divisor 0: its own column sums are not a residual (they hold the shard's
// deviation from the global mean), and the correction waits until the global
// sums are set.  One CTA per variable.
__global__ void __launch_bounds__(256) resid_sum_kernel(const float* __restrict__ xt, int64_t t_pad, int n_pad,
                                                        double divisor, double* __restrict__ rsum)
{
    __shared__ double red[256];
    const int c = blockIdx.x;
    const float4* row = (const float4*)(xt + (int64_t)c * t_pad);
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < t_pad / 4; i += 256) {
        const float4 v = row[i];
        s += ((double)v.x + (double)v.y) + ((double)v.z + (double)v.w);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rsum[c] = red[0];
        if (c == 0) rsum[n_pad] = divisor;
    }
}

// Launch of the transpose (and, for fp16 parts, the per-variable scaling).
template <typename T>
static cudaError_t transpose_to_ws(const T* X, int64_t t, int n, int64_t ldx, const double* mean, const WsLayout& L,
                                   char* ws, int prec, cudaStream_t st, bool own_mean)
{
    const dim3 blk(32, 8);
    const int64_t tiles_t = L.t_pad / 32;
    const unsigned gx = (unsigned)(tiles_t < 2048 ? tiles_t : 2048);
    const dim3 grid(gx, (unsigned)((L.n_pad + 31) / 32));
    if (prec == CUM_PREC_FP64) {
        center_transpose_kernel<T, double><<<grid, blk, 0, st>>>(X, t, n, ldx, mean, (double*)(ws + L.xt), L.t_pad,
                                                                   L.n_pad, nullptr, nullptr);
        return cudaGetLastError();
    }
    // split precisions: every one stores the double-float X~, scaled in place
    // by the fp16 scale exponents (the CTA-pair kinds multiply back exactly)
    unsigned* maxabs = (unsigned*)(ws + L.maxabs);
    cudaError_t e = cudaMemsetAsync(maxabs, 0, sizeof(unsigned) * (size_t)L.n_pad, st);
    if (e != cudaSuccess) return e;
    center_transpose_kernel<T, float><<<grid, blk, 0, st>>>(X, t, n, ldx, mean, (float*)(ws + L.xt), L.t_pad,
                                                              L.n_pad, maxabs, (float*)(ws + L.xlo));
    resid_sum_kernel<<<L.n_pad, 256, 0, st>>>((const float*)(ws + L.xt), L.t_pad, L.n_pad, own_mean ? (double)t : 0.0,
                                              (double*)(ws + L.rsum));
    const int64_t n4 = L.t_pad / 4;
    const int64_t bx = (n4 + 255) / 256;
    const dim3 sg((unsigned)(bx < 64 ? bx : 64), (unsigned)L.n_pad);
    scale_rows_kernel<<<sg, 256, 0, st>>>((float*)(ws + L.xt), (float*)(ws + L.xlo), L.t_pad, maxabs,
                                          (int*)(ws + L.vexp), 1);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t center_impl(const T* X, int64_t t, int n, int64_t ldx, const WsLayout& L, char* ws, int prec,
                               double* mean_out, cudaStream_t st)
{
    double* partial = (double*)(ws + L.colsum);
    double* mean = partial + (size_t)kColsumChunks * L.n_pad;
    double* mean2 = mean + L.n_pad;
    int64_t rpc = (t + kColsumChunks - 1) / kColsumChunks;
    int nchunks = (int)((t + rpc - 1) / rpc);
    dim3 blk(32, 8);
    // pass 1: plain sums
    colsum_kernel<T><<<nchunks, blk, 0, st>>>(X, t, n, ldx, nullptr, rpc, partial, L.n_pad);
    mean_finalize_kernel<<<1, 256, 0, st>>>(partial, nchunks, n, L.n_pad, t, nullptr, mean2, nullptr);
    // pass 2: correction by the mean of the residual
    colsum_kernel<T><<<nchunks, blk, 0, st>>>(X, t, n, ldx, mean2, rpc, partial, L.n_pad);
    mean_finalize_kernel<<<1, 256, 0, st>>>(partial, nchunks, n, L.n_pad, t, mean2, mean, mean_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return transpose_to_ws(X, t, n, ldx, mean, L, ws, prec, st, true);
}

cudaError_t launch_center(const void* X, int dtype, int64_t t, int n, int64_t ldx, const WsLayout& L, char* ws,
                          int prec, double* mean_out, cudaStream_t st)
{
    if (dtype == 1) return center_impl((const double*)X, t, n, ldx, L, ws, prec, mean_out, st);
    return center_impl((const float*)X, t, n, ldx, L, ws, prec, mean_out, st);
}

// ------------------------------------------------------------------ tile plan

// prefix[I] = number of active column tiles of row tiles 0..I-1 (prefix[row_tiles]
// = active_tiles).  Row tile I's first row has the smallest last-block index c
// of the tile; the active columns are the leading C(nbar-c+dB-1, dB) b^dB ones.
__global__ void plan_kernel(Shape sh, int tile_m, int tile_n, int64_t row_tiles, int64_t* __restrict__ prefix)
{
    for (int64_t I = threadIdx.x; I < row_tiles; I += blockDim.x) {
        int j[kMaxHalf];
        colex_unrank((I * tile_m) / sh.bdA, sh.dA, sh.nbar, j);
        int64_t P = cols_with_first_at_least(j[sh.dA - 1], sh.dB, sh.nbar, sh.bdB);
        prefix[I + 1] = (P + tile_n - 1) / tile_n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        prefix[0] = 0;
        for (int64_t I = 0; I < row_tiles; ++I) {
            acc += prefix[I + 1];
            prefix[I + 1] = acc;
        }
    }
}

cudaError_t launch_plan(const OrderPlan& P, int64_t* prefix, cudaStream_t st)
{
    plan_kernel<<<1, 1024, 0, st>>>(P.sh, P.tile_m, P.tile_n, P.row_tiles, prefix);
    return cudaGetLastError();
}

// Work unit u -> (row tile I, column tile J): I = largest with prefix[I] <= u.
__device__ __forceinline__ void unit_to_tile(int64_t u, const int64_t* __restrict__ prefix, int64_t row_tiles,
                                             int64_t* I, int64_t* J)
{
    int64_t lo = 0, hi = row_tiles;  // prefix[lo] <= u < prefix[hi]
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (prefix[mid] <= u) lo = mid; else hi = mid;
    }
    *I = lo;
    *J = u - prefix[lo];
}

// ------------------------------------------------------------------ FP64 moment contraction

// One CTA per (active tile, t chunk): a 64 x 64 tile of
//   S[p, q] = sum_{l in chunk} ZA[l, p] ZB[l, q],  ZA[l,p] = prod_k x~_{l, colA_k(p)}
// with both Khatri-Rao operands built in shared memory from X~ (FP64), 4 x 4
// outputs per thread.  Valid entries (last(p) <= first(q)) are written scaled to
// out[split * E_d + rowOff(p) + colOff(q)].
template <int DA, int DB, bool BATCH>
__global__ void __launch_bounds__(256) moment_fp64_kernel(Shape sh_single, const double* __restrict__ xt_single,
                                                          int64_t t_pad_single, const int64_t* __restrict__ prefix,
                                                          int64_t row_tiles, int S, int64_t kchunk_single,
                                                          double* __restrict__ out_single, double scale_single,
                                                          const BatchOrder* __restrict__ border,
                                                          const BatchUnit* __restrict__ bunit)
{
    constexpr int TM = kF64TileM, TN = kF64TileN, KS = kF64KStep;
    __shared__ __align__(16) double As[KS][TM];
    __shared__ __align__(16) double Bs[KS][TN];
    __shared__ int colA[TM][DA], colB[TN][DB];
    __shared__ int64_t offA[TM], offB[TN];
    __shared__ int lastA[TM], firstB[TN];

    const int64_t w = blockIdx.x;
    int s;
    int64_t I, J, kchunk, t_pad;
    const Shape* shp;
    const double* xt;
    double* out;
    double scale;
    if (BATCH) {
        const BatchUnit bu = bunit[w];
        const BatchOrder* o = border + bu.ord;
        s = bu.s;
        I = bu.I;
        J = bu.J;
        shp = &o->sh;
        kchunk = o->kchunk;
        t_pad = o->t_pad;
        xt = o->xt64;
        out = o->out;
        scale = o->scale;
    } else {
        s = (int)(w % S);
        unit_to_tile(w / S, prefix, row_tiles, &I, &J);
        shp = &sh_single;
        kchunk = kchunk_single;
        t_pad = t_pad_single;
        xt = xt_single;
        out = out_single;
        scale = scale_single;
    }
    const Shape& sh = *shp;
    const int tid = threadIdx.x;
    for (int i = tid; i < TM; i += blockDim.x) {
        const int64_t p = I * TM + i;
        if (p < sh.rows) {
            RowInfo r = decode_row(p, DA, DB, sh.b, sh.nbar, sh.bdA, sh.bdB, sh.bd);
            for (int k = 0; k < DA; ++k) colA[i][k] = r.col[k];
            lastA[i] = r.last;
            offA[i] = r.off;
        } else {
            for (int k = 0; k < DA; ++k) colA[i][k] = 0;
            lastA[i] = INT_MAX;
            offA[i] = 0;
        }
    }
    for (int i = tid; i < TN; i += blockDim.x) {
        const int64_t q = J * TN + i;
        if (q < sh.cols) {
            ColInfo c = decode_col(q, DA, DB, sh.b, sh.nbar, sh.bdB, sh.bd);
            for (int k = 0; k < DB; ++k) colB[i][k] = c.col[k];
            firstB[i] = c.first;
            offB[i] = c.off;
        } else {
            for (int k = 0; k < DB; ++k) colB[i][k] = 0;
            firstB[i] = INT_MIN;
            offB[i] = 0;
        }
    }
    __syncthreads();

    const int tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    const int64_t k0 = (int64_t)s * kchunk;
    const int64_t k1 = k0 + kchunk < t_pad ? k0 + kchunk : t_pad;
    for (int64_t kb = k0; kb < k1; kb += KS) {
        for (int e = tid; e < TM * KS; e += 256) {
            const int row = e / KS, k = e % KS;
            double v = xt[(int64_t)colA[row][0] * t_pad + kb + k];
#pragma unroll
            for (int f = 1; f < DA; ++f) v *= xt[(int64_t)colA[row][f] * t_pad + kb + k];
            As[k][row] = v;
        }
        for (int e = tid; e < TN * KS; e += 256) {
            const int col = e / KS, k = e % KS;
            double v = xt[(int64_t)colB[col][0] * t_pad + kb + k];
#pragma unroll
            for (int f = 1; f < DB; ++f) v *= xt[(int64_t)colB[col][f] * t_pad + kb + k];
            Bs[k][col] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const double2 a01 = *(const double2*)&As[k][ty * 4];
            const double2 a23 = *(const double2*)&As[k][ty * 4 + 2];
            const double2 b01 = *(const double2*)&Bs[k][tx * 4];
            const double2 b23 = *(const double2*)&Bs[k][tx * 4 + 2];
            const double a[4] = {a01.x, a01.y, a23.x, a23.y};
            const double bb[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }

    double* dst = out + (int64_t)s * sh.entries;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int ri = ty * 4 + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cj = tx * 4 + j;
            if (lastA[ri] <= firstB[cj]) dst[offA[ri] + offB[cj]] = acc[i][j] * scale;
        }
    }
}

cudaError_t launch_moment_fp64(const OrderPlan& P, const double* xt, int64_t t_pad, const int64_t* prefix,
                               double* out, double scale, cudaStream_t st)
{
    const int64_t grid = P.units;
    if (grid <= 0) return cudaSuccess;
    if (grid > INT_MAX) return cudaErrorInvalidConfiguration;
#define CUM_F64_CASE(A, B)                                                                                    \
    if (P.sh.dA == A && P.sh.dB == B) {                                                                         \
        moment_fp64_kernel<A, B, false><<<(unsigned)grid, 256, 0, st>>>(P.sh, xt, t_pad, prefix, P.row_tiles,  \
                                                                        P.splits, P.kchunk, out, scale,        \
                                                                        nullptr, nullptr);                     \
        return cudaGetLastError();                                                                             \
    }
    CUM_F64_CASE(1, 1)
    CUM_F64_CASE(2, 1)
    CUM_F64_CASE(2, 2)
    CUM_F64_CASE(3, 2)
    CUM_F64_CASE(3, 3)
#undef CUM_F64_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_moment_fp64_batch(int dA, int dB, const BatchOrder* orders, const BatchUnit* units, int64_t nunits,
                                     cudaStream_t st)
{
    if (nunits <= 0) return cudaSuccess;
    if (nunits > INT_MAX) return cudaErrorInvalidConfiguration;
    Shape none;
    std::memset(&none, 0, sizeof(none));
#define CUM_F64B_CASE(A, B)                                                                                   \
    if (dA == A && dB == B) {                                                                                   \
        moment_fp64_kernel<A, B, true><<<(unsigned)nunits, 256, 0, st>>>(none, nullptr, 0, nullptr, 0, 1, 0,   \
                                                                         nullptr, 1.0, orders, units);         \
        return cudaGetLastError();                                                                             \
    }
    CUM_F64B_CASE(1, 1)
    CUM_F64B_CASE(2, 1)
    CUM_F64B_CASE(2, 2)
    CUM_F64B_CASE(3, 2)
    CUM_F64B_CASE(3, 3)
#undef CUM_F64B_CASE
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ chunk reduction (Alg. 3)

// out[e] = scale * sum_{s < S} partial[s][e], summed in a fixed order (FP64).
__global__ void reduce_splits_kernel(const double* __restrict__ partial, int S, int64_t E, double scale,
                                     double* __restrict__ out)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int s = 0; s < S; ++s) acc += partial[(int64_t)s * E + e];
        out[e] = acc * scale;
    }
}

cudaError_t launch_reduce(const double* partial, int S, int64_t E, double scale, double* out, cudaStream_t st)
{
    int64_t blocks = (E + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    reduce_splits_kernel<<<(unsigned)blocks, 256, 0, st>>>(partial, S, E, scale, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ cumulant correction (Alg. 4-5)

// For every stored block j (sorted) and in-block index i:
//   C[j][i] = M[j][i] - sum_{zeta in P^(2)(1:d), |zeta| >= 2} prod_{k in zeta} C_|k|[j_k][i_k]
// The sub-tuple j_k of a sorted j is sorted, so each factor is a stored block of
// a lower-order tensor (Sec. 3.3), found by its colex rank.
__global__ void __launch_bounds__(256) correct_kernel(int d, int b, int nbar, int64_t bd, int64_t nblocks,
                                                      const double* __restrict__ M, double scale, LowerPtrs low,
                                                      PartTable pt, double* __restrict__ C)
{
    __shared__ int64_t base[kMaxPartitions][kMaxParts];
    __shared__ int plen[kMaxPartitions][kMaxParts];
    for (int64_t r = blockIdx.x; r < nblocks; r += gridDim.x) {
        int j[kMaxOrder];
        colex_unrank(r, d, nbar, j);
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
        for (int64_t e = threadIdx.x; e < bd; e += blockDim.x) {
            int i[kMaxOrder];
            int64_t rem = e;
            for (int k = d - 1; k >= 0; --k) {
                i[k] = (int)(rem % b);
                rem /= b;
            }
            double sum = 0.0;
            for (int z = 0; z < pt.count; ++z) {
                double prod = 1.0;
                for (int q = 0; q < pt.nparts[z]; ++q) {
                    int64_t off = 0;
                    for (int k = 0; k < d; ++k)
                        if (pt.mask[z][q] & (1u << k)) off = off * b + i[k];
                    prod *= low.c[plen[z][q]][base[z][q] + off];
                }
                sum += prod;
            }
            C[r * bd + e] = M[r * bd + e] * scale - sum;
        }
        __syncthreads();
    }
}

__global__ void scale_copy_kernel(const double* __restrict__ src, int64_t E, double scale, double* __restrict__ dst)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = src[e] * scale;
}

cudaError_t launch_correct(int d, int b, int nbar, const double* M, double scale, const LowerPtrs& low,
                           const PartTable& pt, double* C, cudaStream_t st)
{
    const int64_t nblocks = num_blocks(nbar, d);
    const int64_t bd = ipow(b, d);
    if (d <= 3) {
        if (C == M && scale == 1.0) return cudaSuccess;
        int64_t E = nblocks * bd;
        int64_t g = (E + 255) / 256;
        scale_copy_kernel<<<(unsigned)(g > 4096 ? 4096 : (g < 1 ? 1 : g)), 256, 0, st>>>(M, E, scale, C);
        return cudaGetLastError();
    }
    bool done = false;
    cudaError_t e = launch_correct_staged(d, b, nbar, M, scale, low, C, st, &done);
    if (done || e != cudaSuccess) return e;
    int64_t grid = nblocks < 65535 * 8 ? nblocks : 65535 * 8;
    int threads = bd >= 256 ? 256 : (bd >= 128 ? 128 : 64);
    correct_kernel<<<(unsigned)grid, threads, 0, st>>>(d, b, nbar, bd, nblocks, M, scale, low, pt, C);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ pieces of the t-sharded path (Alg. 3)

// sums[c] = sum over chunks of partial[chunk][c] (no division).
__global__ void sum_partials_kernel(const double* __restrict__ partial, int nchunks, int n, int n_pad,
                                    double* __restrict__ sums)
{
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nchunks; ++k) s += partial[(int64_t)k * n_pad + c];
        sums[c] = s;
    }
}

template <typename T>
static cudaError_t column_sums_impl(const T* X, int64_t t, int n, int64_t ldx, const double* shift,
                                    const WsLayout& L, char* ws, double* sums, cudaStream_t st)
{
    double* partial = (double*)(ws + L.colsum);
    int64_t rpc = (t + kColsumChunks - 1) / kColsumChunks;
    int nchunks = (int)((t + rpc - 1) / rpc);
    colsum_kernel<T><<<nchunks, dim3(32, 8), 0, st>>>(X, t, n, ldx, shift, rpc, partial, L.n_pad);
    sum_partials_kernel<<<1, 256, 0, st>>>(partial, nchunks, n, L.n_pad, sums);
    return cudaGetLastError();
}

cudaError_t launch_column_sums(const void* X, int dtype, int64_t t, int n, int64_t ldx, const double* shift,
                               const WsLayout& L, char* ws, double* sums, cudaStream_t st)
{
    if (dtype == 1) return column_sums_impl((const double*)X, t, n, ldx, shift, L, ws, sums, st);
    return column_sums_impl((const float*)X, t, n, ldx, shift, L, ws, sums, st);
}

// mean[c] = shift[c] + sums[c] / t_total   (shift may be NULL)
__global__ void mean_from_sums_kernel(int n, double inv_t, const double* __restrict__ shift,
                                      const double* __restrict__ sums, double* __restrict__ mean)
{
    for (int c = threadIdx.x; c < n; c += blockDim.x) mean[c] = (shift ? shift[c] : 0.0) + sums[c] * inv_t;
}

cudaError_t launch_mean_from_sums(int n, int64_t t_total, const double* shift, const double* sums, double* mean,
                                  cudaStream_t st)
{
    mean_from_sums_kernel<<<1, 256, 0, st>>>(n, 1.0 / (double)t_total, shift, sums, mean);
    return cudaGetLastError();
}

// First-order removal of the residual column means m = rsum[0..n_pad) / rsum[n_pad]
// of the stored split-precision array from its order-D moments (or sums):
//   M[e] -= sum_k m[v_k] * Mlow[e without position k],
// Mlow the order-(D-1) moments (or sums) of the same array.  The expansion of
// the moments of (y - m) in m is exact to second order in m, whose relative size
// is about 2^-25: the dropped terms are below FP64 resolution.  One CTA per
// stored block (grid-stride); the block's D sub-tuples are ranked once.
template <int D>
__global__ void __launch_bounds__(256) shift_correct_kernel(int b, int nbar, int64_t nblocks, int64_t bd,
                                                            int64_t bdm1, const double* __restrict__ Mlow,
                                                            const double* __restrict__ rsum, int n_pad,
                                                            double* __restrict__ M)
{
    __shared__ int64_t sub[D];
    __shared__ int jb[D];
    if (rsum[n_pad] == 0.0) return;   // no residual set (a shard before the global sums)
    const double inv_t = 1.0 / rsum[n_pad];
    for (int64_t r = blockIdx.x; r < nblocks; r += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int j[D];
            colex_unrank(r, D, nbar, j);
            for (int k = 0; k < D; ++k) {
                jb[k] = j[k];
                int s[D];
                int q = 0;
                for (int k2 = 0; k2 < D; ++k2)
                    if (k2 != k) s[q++] = j[k2];
                sub[k] = colex_rank(s, D - 1) * bdm1;
            }
        }
        __syncthreads();
        for (int64_t e = threadIdx.x; e < bd; e += blockDim.x) {
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
                acc += rsum[jb[k] * b + dig[k]] * Mlow[sub[k] + o];
            }
            M[r * bd + e] -= acc * inv_t;
        }
    }
}

cudaError_t launch_shift_correct(int d, int b, int nbar, const double* Mlow, const double* rsum, int n_pad, double* M,
                                 cudaStream_t st)
{
    const int64_t nblocks = num_blocks(nbar, d), bd = ipow(b, d), bdm1 = ipow(b, d - 1);
    const int grid = (int)(nblocks < 8 * kTcMaxCtas ? nblocks : 8 * kTcMaxCtas);
    const int threads = bd < 256 ? (int)((bd + 31) / 32 * 32) : 256;
    switch (d) {
    case 3: shift_correct_kernel<3><<<grid, threads, 0, st>>>(b, nbar, nblocks, bd, bdm1, Mlow, rsum, n_pad, M); break;
    case 4: shift_correct_kernel<4><<<grid, threads, 0, st>>>(b, nbar, nblocks, bd, bdm1, Mlow, rsum, n_pad, M); break;
    case 5: shift_correct_kernel<5><<<grid, threads, 0, st>>>(b, nbar, nblocks, bd, bdm1, Mlow, rsum, n_pad, M); break;
    case 6: shift_correct_kernel<6><<<grid, threads, 0, st>>>(b, nbar, nblocks, bd, bdm1, Mlow, rsum, n_pad, M); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_center_given(const void* X, int dtype, int64_t t, int n, int64_t ldx, const double* mean,
                                const WsLayout& L, char* ws, int prec, cudaStream_t st)
{
    if (dtype == 1) return transpose_to_ws((const double*)X, t, n, ldx, mean, L, ws, prec, st, false);
    return transpose_to_ws((const float*)X, t, n, ldx, mean, L, ws, prec, st, false);
}

}  // namespace cum
