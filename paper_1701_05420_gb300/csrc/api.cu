// C ABI of libcumgb (declared in include/cumgb.h): argument checks, workspace
// layout, per-order plans and the launch sequence of Alg. 5 (centring, moment
// contraction per order, t-chunk reduction, cumulant correction).
#include <cstdio>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cumgb.h"
#include "internal.h"

namespace cum {

// Host-side NVTX range around the launches of one step (header-only NVTX: it
// costs nothing unless a profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

static thread_local int g_last_cuda_error = 0;

int cuda_fail(cudaError_t e)
{
    g_last_cuda_error = (int)e;
    return CUM_ECUDA;
}

bool prec_is_tc(int prec)
{
    return prec == CUM_PREC_BF16X3 || prec == CUM_PREC_TF32X3 || prec == CUM_PREC_FP16X3;
}

bool prec_is_valid(int prec) { return prec == CUM_PREC_FP64 || prec_is_tc(prec); }

int64_t pad_t(int64_t t) { return (t + kTAlign - 1) / kTAlign * kTAlign; }

static size_t align_up(size_t x) { return (x + kWsAlign - 1) / kWsAlign * kWsAlign; }

// Basic range checks shared by all entry points; false if unsupported.
static bool sizes_ok(int64_t t, int n, int b, int d_max)
{
    if (t < 1 || n < 1 || b < 1 || b > 64 || d_max < 2 || d_max > kMaxOrder) return false;
    int nbar = (n + b - 1) / b;
    if ((int64_t)nbar + d_max >= kMaxBinomM) return false;
    if ((int64_t)nbar * b > 65535) return false;
    if (t > ((int64_t)1 << 40)) return false;
    return true;
}

// Samples per split step: the tensor-core chunks are whole 128-sample steps.
static int64_t split_step(int prec) { return prec_is_tc(prec) ? 128 : kF64KStep; }

int64_t max_order_splits(const OrderPlan& P, int64_t t, int prec)
{
    // a chunk keeps at least kMinChunk samples and the partial buffer is capped
    const int64_t kMinChunk = prec_is_tc(prec) ? 2048 : 1024;
    const int64_t kMaxPartialBytes = (int64_t)1 << 30;
    int64_t smax = pad_t(t) / kMinChunk;
    const int64_t smax_mem = kMaxPartialBytes / (8 * P.sh.entries);
    if (smax_mem < smax) smax = smax_mem;
    if (smax > 1024) smax = 1024;
    return smax < 1 ? 1 : smax;
}

void set_order_splits(OrderPlan& P, int64_t t, int prec, int64_t S)
{
    const int64_t kstep = split_step(prec);
    const int64_t steps = (pad_t(t) + kstep - 1) / kstep;
    if (S < 1) S = 1;
    const int64_t steps_per = (steps + S - 1) / S;
    P.kchunk = steps_per * kstep;
    P.splits = (int)((steps + steps_per - 1) / steps_per);
    P.units = P.active_tiles * P.splits;
}

// Split of the t axis for one tensor-core contraction (Alg. 3).  Its `workers`
// (CTAs, one per SM, or CTA pairs) take the work units round robin, so the
// busiest one runs ceil(units / workers) units, each of its chunk's 128-sample steps plus a fixed
// cost of about kTcUnitSteps steps (pipeline fill and drain, the tile
// write-out).  S minimises that CTA's time; the smallest S wins a tie.
static int64_t tc_splits(int64_t tiles, int64_t steps, int64_t smax, int64_t workers)
{
    int64_t best = 1, best_cost = -1;
    for (int64_t S = 1; S <= smax; ++S) {
        const int64_t per = (steps + S - 1) / S;
        if ((steps + per - 1) / per != S) continue;   // same chunks as a smaller S
        const int64_t rounds = (tiles * S + workers - 1) / workers;
        const int64_t cost = rounds * (per + kTcUnitSteps);
        if (best_cost < 0 || cost < best_cost) {
            best = S;
            best_cost = cost;
        }
    }
    return best;
}

OrderPlan make_order_plan(int d, int64_t t, int n, int b, int prec, bool pair_ok)
{
    OrderPlan P;
    P.sh = make_shape(d, n, b);
    const bool tc = prec_is_tc(prec);
    // orders 2 to 5 of every split precision take three fp16 parts of the
    // double-float X~ (two parts are too few for odd moments near zero).
    // Order 6, whose contraction dominates, keeps two parts (19 bits, the
    // short hi part for a smaller truncation bias) from kPreciseOrder6T
    // samples on: their unbiased representation error shrinks like 1/sqrt(t)
    // while the bias does not; below it three parts cost little.
    P.precise = pair_ok && tc && (d <= 5 || pad_t(t) < kPreciseOrder6T);
    // every split precision contracts on CTA pairs outside a batch (TF32X3
    // with fp16 parts: the same arithmetic as FP16X3); batches run the one-CTA
    // kernel with the precision's own parts
    P.pair = pair_ok && tc;
    P.tile_m = P.pair ? kPairTileM : tc ? kTcTileM : kF64TileM;
    P.tile_n = P.pair ? kPairTileN : tc ? kTcTileN : kF64TileN;
    P.row_tiles = (P.sh.rows + P.tile_m - 1) / P.tile_m;
    int64_t active = 0;
    for (int64_t I = 0; I < P.row_tiles; ++I) {
        int j[kMaxHalf];
        colex_unrank((I * P.tile_m) / P.sh.bdA, P.sh.dA, P.sh.nbar, j);
        int64_t cols = cols_with_first_at_least(j[P.sh.dA - 1], P.sh.dB, P.sh.nbar, P.sh.bdB);
        active += (cols + P.tile_n - 1) / P.tile_n;
    }
    P.active_tiles = active;
    const int64_t smax = max_order_splits(P, t, prec);
    int64_t S;
    if (tc) {
        S = tc_splits(active, (pad_t(t) + 127) / 128, smax, P.pair ? kPairPlanClusters : kTcPlanCtas);
    } else {
        // FP64 tiles: split until there are about 8 units per SM
        const int64_t target = 8 * kTcMaxCtas;
        S = (target + active - 1) / active;
        if (S > smax) S = smax;
    }
    set_order_splits(P, t, prec, S);
    return P;
}

bool layout_ws(int64_t t, int n, int d_max, int b, int prec, WsLayout* L)
{
    if (!sizes_ok(t, n, b, d_max) || !prec_is_valid(prec)) return false;
    const bool tc = prec_is_tc(prec);
    const int nbar = (n + b - 1) / b;
    L->n_pad = nbar * b;
    if (tc && L->n_pad > kTcMaxNPad) return false;
    L->t_pad = pad_t(t);
    L->xt_elem = tc ? sizeof(float) : sizeof(double);
    size_t off = 0;
    L->status = off;
    off = align_up(off + 64);
    L->colsum = off;
    off = align_up(off + sizeof(double) * ((size_t)kColsumChunks * L->n_pad + 2 * (size_t)L->n_pad));
    // every region that centring writes (status, sums and mean, the fp16 scale
    // tables, X~) comes before the first one sized by the orders, so a
    // workspace laid out for any d_max holds them at the same offsets: a
    // cum_center call and later cum_moment_blocks calls of any order agree
    L->maxabs = off;
    off = align_up(off + sizeof(uint32_t) * (size_t)L->n_pad);
    L->vexp = off;
    off = align_up(off + sizeof(int32_t) * (size_t)L->n_pad);
    L->rsum = off;
    off = align_up(off + sizeof(double) * ((size_t)L->n_pad + 1));
    L->xt = off;
    off = align_up(off + L->xt_elem * (size_t)L->n_pad * (size_t)L->t_pad);
    L->xlo = off;
    if (tc) off = align_up(off + sizeof(float) * (size_t)L->n_pad * (size_t)L->t_pad);
    int64_t max_row_tiles = 0, max_partial = 0;
    for (int d = 2; d <= d_max; ++d) {
        OrderPlan P = make_order_plan(d, t, n, b, prec);
        if (P.row_tiles > max_row_tiles) max_row_tiles = P.row_tiles;
        if (P.splits > 1 && P.splits * P.sh.entries > max_partial) max_partial = P.splits * P.sh.entries;
    }
    L->prefix = off;
    off = align_up(off + sizeof(int64_t) * (size_t)(max_row_tiles + 1));
    L->partial = off;
    off = align_up(off + sizeof(double) * (size_t)max_partial);
    L->scratch = off;
    if (tc) off = align_up(off + sizeof(double) * kTcScratchDoubles);
    L->m4 = off;
    if (d_max >= 6 || (tc && d_max >= 5)) off = align_up(off + sizeof(double) * (size_t)(num_blocks(nbar, 4) * ipow(b, 4)));
    L->mlow = off;
    if (tc && d_max >= 3)
        off = align_up(off + sizeof(double) * (size_t)(num_blocks(nbar, d_max - 1) * ipow(b, d_max - 1)));
    L->total = off;
    return true;
}

// Set partitions of {0..d-1} with every part of size >= 2 and at least two
// parts.  Generated by choosing, for the smallest unassigned position, every
// subset of the remaining positions that contains it and has >= 2 elements.
static void gen_parts(uint32_t remaining, std::vector<uint32_t>& cur, std::vector<std::vector<uint32_t>>& out)
{
    if (!remaining) {
        out.push_back(cur);
        return;
    }
    const uint32_t low = remaining & (~remaining + 1u);
    const uint32_t rest = remaining & ~low;
    // enumerate subsets `sub` of `rest` (including empty) and take low|sub
    uint32_t sub = rest;
    for (;;) {
        const uint32_t part = low | sub;
        if (__builtin_popcount(part) >= 2) {
            cur.push_back(part);
            gen_parts(remaining & ~part, cur, out);
            cur.pop_back();
        }
        if (sub == 0) break;
        sub = (sub - 1) & rest;
    }
}

PartTable make_part_table(int d)
{
    PartTable pt;
    std::memset(&pt, 0, sizeof(pt));
    std::vector<std::vector<uint32_t>> all;
    std::vector<uint32_t> cur;
    gen_parts((1u << d) - 1u, cur, all);
    for (auto& z : all) {
        if (z.size() < 2) continue;  // sigma = 1 is the moment itself
        if (pt.count >= kMaxPartitions || (int)z.size() > kMaxParts) continue;
        pt.nparts[pt.count] = (int)z.size();
        for (size_t q = 0; q < z.size(); ++q) pt.mask[pt.count][q] = z[q];
        ++pt.count;
    }
    return pt;
}

static bool ws_ok(const void* ws, size_t ws_bytes, const WsLayout& L)
{
    return ws && ((uintptr_t)ws % kWsAlign) == 0 && ws_bytes >= L.total;
}

// Moment contraction of one order into `M_out` (scaled by 1/t, or the plain
// sums with sums_only), of the centred array as stored in the workspace.
static int contract_order(int d, int64_t t, int n, int b, int prec, const WsLayout& L, char* ws, double* M_out,
                          cudaStream_t st, bool sums_only = false)
{
    OrderPlan P = make_order_plan(d, t, n, b, prec);
    int64_t* prefix = (int64_t*)(ws + L.prefix);
    cudaError_t e = launch_plan(P, prefix, st);
    if (e != cudaSuccess) return cuda_fail(e);
    const double scale = sums_only ? 1.0 : 1.0 / (double)t;
    double* partial = (double*)(ws + L.partial);
    double* dst = P.splits > 1 ? partial : M_out;
    const double s1 = P.splits > 1 ? 1.0 : scale;
    if (P.pair)
        e = launch_moment_pair(P, prec, (const float*)(ws + L.xt), (const float*)(ws + L.xlo), L.t_pad, prefix, dst,
                               s1, (double*)(ws + L.scratch), (int*)(ws + L.status), (const int*)(ws + L.vexp), st);
    else if (prec_is_tc(prec))
        e = launch_moment_tc(P, prec, (const float*)(ws + L.xt), L.t_pad, prefix, dst, s1, (double*)(ws + L.scratch),
                             (int*)(ws + L.status), (const int*)(ws + L.vexp), st);
    else
        e = launch_moment_fp64(P, (const double*)(ws + L.xt), L.t_pad, prefix, dst, s1, st);
    if (e != cudaSuccess) return cuda_fail(e);
    if (P.splits > 1) {
        e = launch_reduce(partial, P.splits, P.sh.entries, scale, M_out, st);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return CUM_OK;
}

// Split precisions, order 6 (read from the FP32 X~ alone): removes the first-order effect of the stored
// array's residual column means from its order-d moments (or sums) M, given
// the order-(d-1) moments (or sums) Mlow of the same array.
static int shift_order(int d, int n, int b, const WsLayout& L, char* ws, const double* Mlow, double* M,
                       cudaStream_t st)
{
    const int nbar = (n + b - 1) / b;
    cudaError_t e = launch_shift_correct(d, b, nbar, Mlow, (const double*)(ws + L.rsum), L.n_pad, M, st);
    if (e != cudaSuccess) return cuda_fail(e);
    return CUM_OK;
}

// Split precisions: whether order d contracts the FP32 X~ alone (and so needs
// the residual-mean correction): order 6 from kPreciseOrder6T samples on; the
// other orders use the double-float X~.
static bool needs_shift(int d, int64_t t, int prec)
{
    return prec_is_tc(prec) && d >= 6 && pad_t(t) >= kPreciseOrder6T;
}

// Moments (or sums) of order d of the centred data: the contraction and, on
// split precisions for d = 6, the residual-mean correction, with the
// order-(d-1) contraction computed into the workspace for it.
static int moment_order(int d, int64_t t, int n, int b, int prec, const WsLayout& L, char* ws, double* M_out,
                        cudaStream_t st, bool sums_only = false)
{
    int rc = contract_order(d, t, n, b, prec, L, ws, M_out, st, sums_only);
    if (rc != CUM_OK || !needs_shift(d, t, prec)) return rc;
    double* mlow = (double*)(ws + L.mlow);
    rc = contract_order(d - 1, t, n, b, prec, L, ws, mlow, st, sums_only);
    if (rc != CUM_OK) return rc;
    return shift_order(d, n, b, L, ws, mlow, M_out, st);
}

__global__ void set_divisor_kernel(double* dst, double v) { *dst = v; }

}  // namespace cum

using namespace cum;

extern "C" {

int64_t cum_num_blocks(int nbar, int d)
{
    if (nbar < 1 || d < 1 || (int64_t)nbar + d >= kMaxBinomM || d > 8) return -1;
    return num_blocks(nbar, d);
}

int cum_block_rank(const int32_t* j, int d, int64_t* rank)
{
    if (!j || !rank || d < 1 || d > 8) return CUM_EINVAL;
    int jj[8];
    for (int k = 0; k < d; ++k) {
        if (j[k] < 0 || (k > 0 && j[k] < j[k - 1]) || j[k] + d >= kMaxBinomM) return CUM_EINVAL;
        jj[k] = j[k];
    }
    *rank = colex_rank(jj, d);
    return CUM_OK;
}

int cum_block_unrank(int64_t rank, int d, int nbar, int32_t* j)
{
    if (!j || d < 1 || d > 8 || nbar < 1 || (int64_t)nbar + d >= kMaxBinomM) return CUM_EINVAL;
    if (rank < 0 || rank >= num_blocks(nbar, d)) return CUM_EINVAL;
    int jj[8];
    colex_unrank(rank, d, nbar, jj);
    for (int k = 0; k < d; ++k) j[k] = jj[k];
    return CUM_OK;
}

size_t cum_workspace_size(int64_t t, int n, int d_max, int b, int prec)
{
    WsLayout L;
    if (!layout_ws(t, n, d_max, b, prec, &L)) return 0;
    return L.total;
}

int cum_center(const void* X, int dtype, int64_t t, int n, int64_t ldx, int b, int prec, double* mean_out, void* ws,
               size_t ws_bytes, void* stream)
{
    if (!X || (dtype != CUM_F32 && dtype != CUM_F64) || ldx < n || !prec_is_valid(prec)) return CUM_EINVAL;
    WsLayout L;
    if (!sizes_ok(t, n, b, 2)) return CUM_EINVAL;
    if (!layout_ws(t, n, 2, b, prec, &L)) return CUM_EUNSUPPORTED;
    if (!ws_ok(ws, ws_bytes, L)) return CUM_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync((char*)ws + L.status, 0, 64, st);
    if (e == cudaSuccess) e = launch_center(X, dtype, t, n, ldx, L, (char*)ws, prec, mean_out, st);
    if (e != cudaSuccess) return cuda_fail(e);
    return CUM_OK;
}

int cum_moment_blocks(int d, int64_t t, int n, int b, int prec, double* M_out, void* ws, size_t ws_bytes,
                      void* stream)
{
    if (!M_out || !prec_is_valid(prec) || d < 2 || d > kMaxOrder) return CUM_EINVAL;
    if (!sizes_ok(t, n, b, d)) return CUM_EINVAL;
    WsLayout L;
    if (!layout_ws(t, n, d, b, prec, &L)) return CUM_EUNSUPPORTED;
    if (!ws_ok(ws, ws_bytes, L)) return CUM_EWORKSPACE;
    return moment_order(d, t, n, b, prec, L, (char*)ws, M_out, (cudaStream_t)stream);
}

int cum_correct(int d, int n, int b, const double* M_d, const double* const* C_lower, double* C_out, void* stream)
{
    if (!M_d || !C_out || d < 2 || d > kMaxOrder || n < 1 || b < 1) return CUM_EINVAL;
    if (!sizes_ok(1, n, b, d)) return CUM_EINVAL;
    LowerPtrs low;
    std::memset(&low, 0, sizeof(low));
    if (d >= 4) {
        if (!C_lower) return CUM_EINVAL;
        for (int k = 2; k <= d - 2; ++k) {
            if (!C_lower[k - 2]) return CUM_EINVAL;
            low.c[k] = C_lower[k - 2];
        }
    }
    const int nbar = (n + b - 1) / b;
    PartTable pt = make_part_table(d);
    cudaError_t e = launch_correct(d, b, nbar, M_d, 1.0, low, pt, C_out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    return CUM_OK;
}

int cum_correct_m4(int n, int b, const double* M_6, const double* const* C_lower, const double* M_4, double* C_out,
                   void* stream)
{
    if (!M_6 || !C_out || !C_lower || !M_4 || n < 1 || b < 1) return CUM_EINVAL;
    if (!sizes_ok(1, n, b, 6)) return CUM_EINVAL;
    LowerPtrs low;
    std::memset(&low, 0, sizeof(low));
    for (int k = 2; k <= 4; ++k) {
        if (!C_lower[k - 2]) return CUM_EINVAL;
        low.c[k] = C_lower[k - 2];
    }
    low.m4 = M_4;
    const int nbar = (n + b - 1) / b;
    PartTable pt = make_part_table(6);
    cudaError_t e = launch_correct(6, b, nbar, M_6, 1.0, low, pt, C_out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    return CUM_OK;
}

int cum_cumulants(const void* X, int dtype, int64_t t, int n, int64_t ldx, int d_max, int b, int prec,
                  double* const* C_out, double* mean_out, void* ws, size_t ws_bytes, void* stream)
{
    if (!X || !C_out || (dtype != CUM_F32 && dtype != CUM_F64) || ldx < n || !prec_is_valid(prec)) return CUM_EINVAL;
    if (d_max < 2 || d_max > kMaxOrder || !sizes_ok(t, n, b, d_max)) return CUM_EINVAL;
    for (int d = 2; d <= d_max; ++d)
        if (!C_out[d - 2]) return CUM_EINVAL;
    WsLayout L;
    if (!layout_ws(t, n, d_max, b, prec, &L)) return CUM_EUNSUPPORTED;
    if (!ws_ok(ws, ws_bytes, L)) return CUM_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    NvtxRange range("cum_cumulants");
    cudaError_t e = cudaMemsetAsync((char*)ws + L.status, 0, 64, st);
    if (e == cudaSuccess) {
        NvtxRange r1("centring (Def. 1.3)");
        e = launch_center(X, dtype, t, n, ldx, L, (char*)ws, prec, mean_out, st);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    const int nbar = (n + b - 1) / b;
    const bool tc = prec_is_tc(prec);
    // with orders up to 6 the order-4 moments stay in the workspace: the
    // order-6 correction uses them (moment form, see cum_correct_m4).  On split
    // precisions each order's moments also take the residual-mean correction,
    // which needs the previous order's moments: M_2 and M_3 are C_2 and C_3,
    // M_4 stays in the workspace from d_max = 5 on, and M_5 with d_max = 6
    double* m4 = d_max >= 6 || (tc && d_max >= 5) ? (double*)((char*)ws + L.m4) : nullptr;
    double* m5 = tc && d_max >= 6 ? (double*)((char*)ws + L.mlow) : nullptr;
    for (int d = 2; d <= d_max; ++d) {
        char name[48];
        std::snprintf(name, sizeof(name), "order %d: moment blocks (Alg. 1-3)", d);
        double* M = d == 4 && m4 ? m4 : d == 5 && m5 ? m5 : C_out[d - 2];
        int rc;
        {
            NvtxRange r2(name);
            rc = contract_order(d, t, n, b, prec, L, (char*)ws, M, st);
            if (rc == CUM_OK && needs_shift(d, t, prec)) {
                const double* low = d == 4 ? C_out[1] : d == 5 ? m4 : m5;
                rc = shift_order(d, n, b, L, (char*)ws, low, M, st);
            }
        }
        if (rc != CUM_OK) return rc;
        if (d >= 4) {
            std::snprintf(name, sizeof(name), "order %d: correction (Alg. 4-5)", d);
            NvtxRange r3(name);
            LowerPtrs low;
            std::memset(&low, 0, sizeof(low));
            for (int k = 2; k <= d - 2; ++k) low.c[k] = C_out[k - 2];
            if (d == 6) low.m4 = m4;
            PartTable pt = make_part_table(d);
            e = launch_correct(d, b, nbar, M, 1.0, low, pt, C_out[d - 2], st);
            if (e != cudaSuccess) return cuda_fail(e);
        }
    }
    return CUM_OK;
}

int cum_column_sums(const void* X, int dtype, int64_t t, int n, int64_t ldx, int b, int prec, const double* shift,
                    double* sums_out, void* ws, size_t ws_bytes, void* stream)
{
    if (!X || !sums_out || (dtype != CUM_F32 && dtype != CUM_F64) || ldx < n || !prec_is_valid(prec)) return CUM_EINVAL;
    if (!sizes_ok(t, n, b, 2)) return CUM_EINVAL;
    WsLayout L;
    if (!layout_ws(t, n, 2, b, prec, &L)) return CUM_EUNSUPPORTED;
    if (!ws_ok(ws, ws_bytes, L)) return CUM_EWORKSPACE;
    cudaError_t e = launch_column_sums(X, dtype, t, n, ldx, shift, L, (char*)ws, sums_out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    return CUM_OK;
}

int cum_mean_from_sums(int n, int64_t t_total, const double* shift, const double* sums, double* mean_out,
                       void* stream)
{
    if (n < 1 || t_total < 1 || !sums || !mean_out) return CUM_EINVAL;
    cudaError_t e = launch_mean_from_sums(n, t_total, shift, sums, mean_out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    return CUM_OK;
}

int cum_center_with_mean(const void* X, int dtype, int64_t t, int n, int64_t ldx, int b, int prec,
                         const double* mean, void* ws, size_t ws_bytes, void* stream)
{
    if (!X || !mean || (dtype != CUM_F32 && dtype != CUM_F64) || ldx < n || !prec_is_valid(prec)) return CUM_EINVAL;
    if (!sizes_ok(t, n, b, 2)) return CUM_EINVAL;
    WsLayout L;
    if (!layout_ws(t, n, 2, b, prec, &L)) return CUM_EUNSUPPORTED;
    if (!ws_ok(ws, ws_bytes, L)) return CUM_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync((char*)ws + L.status, 0, 64, st);
    if (e == cudaSuccess) e = launch_center_given(X, dtype, t, n, ldx, mean, L, (char*)ws, prec, st);
    if (e != cudaSuccess) return cuda_fail(e);
    return CUM_OK;
}

int cum_moment_sums(int d, int64_t t, int n, int b, int prec, double* S_out, void* ws, size_t ws_bytes, void* stream)
{
    if (!S_out || !prec_is_valid(prec) || d < 2 || d > kMaxOrder) return CUM_EINVAL;
    if (!sizes_ok(t, n, b, d)) return CUM_EINVAL;
    WsLayout L;
    if (!layout_ws(t, n, d, b, prec, &L)) return CUM_EUNSUPPORTED;
    if (!ws_ok(ws, ws_bytes, L)) return CUM_EWORKSPACE;
    return moment_order(d, t, n, b, prec, L, (char*)ws, S_out, (cudaStream_t)stream, true);
}

int cum_moment_contraction(int d, int64_t t, int n, int b, int prec, double* M_out, void* ws, size_t ws_bytes,
                           void* stream)
{
    if (!M_out || !prec_is_valid(prec) || d < 2 || d > kMaxOrder) return CUM_EINVAL;
    if (!sizes_ok(t, n, b, d)) return CUM_EINVAL;
    WsLayout L;
    if (!layout_ws(t, n, d, b, prec, &L)) return CUM_EUNSUPPORTED;
    if (!ws_ok(ws, ws_bytes, L)) return CUM_EWORKSPACE;
    return contract_order(d, t, n, b, prec, L, (char*)ws, M_out, (cudaStream_t)stream);
}

// Layout of the regions that centring writes, which do not depend on t or the
// orders: the residual sums' calls need only n, b and the precision.
static bool centring_layout(int n, int b, int prec, WsLayout* L)
{
    return layout_ws(1, n, 2, b, prec, L);
}

int cum_residual_sums(int n, int b, int prec, double* sums_out, const void* ws, size_t ws_bytes, void* stream)
{
    if (!sums_out || !prec_is_valid(prec) || n < 1 || !sizes_ok(1, n, b, 2)) return CUM_EINVAL;
    WsLayout L;
    if (!centring_layout(n, b, prec, &L)) return CUM_EUNSUPPORTED;
    if (!ws || ((uintptr_t)ws % kWsAlign) != 0 || ws_bytes < L.rsum + sizeof(double) * ((size_t)L.n_pad + 1))
        return CUM_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (prec_is_tc(prec))
        e = cudaMemcpyAsync(sums_out, (const char*)ws + L.rsum, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice,
                            st);
    else
        e = cudaMemsetAsync(sums_out, 0, sizeof(double) * (size_t)n, st);   // FP64 operands: no residual
    if (e != cudaSuccess) return cuda_fail(e);
    return CUM_OK;
}

int cum_set_residual_sums(int n, int b, int prec, const double* sums, int64_t t_total, void* ws, size_t ws_bytes,
                          void* stream)
{
    if (!sums || !prec_is_valid(prec) || n < 1 || t_total < 1 || !sizes_ok(1, n, b, 2)) return CUM_EINVAL;
    WsLayout L;
    if (!centring_layout(n, b, prec, &L)) return CUM_EUNSUPPORTED;
    if (!ws || ((uintptr_t)ws % kWsAlign) != 0 || ws_bytes < L.rsum + sizeof(double) * ((size_t)L.n_pad + 1))
        return CUM_EWORKSPACE;
    if (!prec_is_tc(prec)) return CUM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    double* rsum = (double*)((char*)ws + L.rsum);
    cudaError_t e = cudaMemcpyAsync(rsum, sums, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        set_divisor_kernel<<<1, 1, 0, st>>>(rsum + L.n_pad, (double)t_total);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(e);
    return CUM_OK;
}

int cum_finalize(int d, int n, int b, double scale, const double* S_d, const double* const* C_lower, double* C_out,
                 void* stream)
{
    if (!S_d || !C_out || d < 2 || d > kMaxOrder || n < 1 || b < 1) return CUM_EINVAL;
    if (!sizes_ok(1, n, b, d)) return CUM_EINVAL;
    LowerPtrs low;
    std::memset(&low, 0, sizeof(low));
    if (d >= 4) {
        if (!C_lower) return CUM_EINVAL;
        for (int k = 2; k <= d - 2; ++k) {
            if (!C_lower[k - 2]) return CUM_EINVAL;
            low.c[k] = C_lower[k - 2];
        }
    }
    const int nbar = (n + b - 1) / b;
    PartTable pt = make_part_table(d);
    cudaError_t e = launch_correct(d, b, nbar, S_d, scale, low, pt, C_out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    return CUM_OK;
}

int cum_plan_info(int d, int64_t t, int n, int b, int prec, int64_t* info)
{
    if (!info || d < 2 || d > kMaxOrder || !prec_is_valid(prec) || !sizes_ok(t, n, b, d)) return CUM_EINVAL;
    WsLayout L;
    if (!layout_ws(t, n, d, b, prec, &L)) return CUM_EUNSUPPORTED;
    OrderPlan P = make_order_plan(d, t, n, b, prec);
    info[0] = P.active_tiles;
    info[1] = P.splits;
    info[2] = P.units;
    info[3] = P.tile_m;
    info[4] = P.tile_n;
    info[5] = P.kchunk;
    // plan, contraction, chunk reduction, residual-mean correction
    info[6] = 2 + (P.splits > 1 ? 1 : 0) + (needs_shift(d, t, prec) ? 1 : 0);
    // two sum passes, two finalisations, transpose (+ residual sums and fp16 scale exponents)
    info[7] = 5 + (prec_is_tc(prec) ? 2 : 0);
    return CUM_OK;
}

int cum_probe_bounded_wait(void* ws, size_t ws_bytes, void* stream)
{
    if (!ws || ws_bytes < 64 || ((uintptr_t)ws % kWsAlign) != 0) return CUM_EWORKSPACE;
    cudaError_t e = launch_bounded_wait_probe((int*)ws, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    return CUM_OK;
}

int cum_device_status(void* ws, size_t ws_bytes, void* stream)
{
    if (!ws || ws_bytes < 64) return CUM_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, ws, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    if (h != 0) {
        e = cudaMemsetAsync(ws, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e);
        return CUM_ETIMEOUT;
    }
    return CUM_OK;
}

const char* cum_strerror(int status)
{
    switch (status) {
    case CUM_OK: return "success";
    case CUM_EINVAL: return "invalid argument";
    case CUM_EUNSUPPORTED: return "unsupported size or precision for this build";
    case CUM_ECUDA: return "CUDA error (see cum_last_cuda_error)";
    case CUM_ETIMEOUT: return "a bounded device-side wait expired";
    case CUM_EWORKSPACE: return "workspace missing, misaligned or too small";
    default: return "unknown status";
    }
}

int cum_last_cuda_error(void) { return g_last_cuda_error; }

}  // extern "C"
