// Tensor-core moment contraction on sm_103a (tcgen05 + TMA + TMEM).
//
// Computes, for one order d, the block-stored sums
//   M[rowOff(p) + colOff(q)] = scale * sum_l ZA[l, p] * ZB[l, q]      (Alg. 1-2)
// over the valid pairs last(p) <= first(q), where ZA / ZB are the Khatri-Rao
// products of dA = ceil(d/2) and dB = floor(d/2) centred columns.  Each CTA is
// persistent and walks work units (128 x 128 output tile, t chunk).
//
// Per stage of 128 bytes of samples (64 bf16 / fp16 samples, or 32 tf32):
//  * warp 0 (one thread) TMA-loads the X~ slab [variables x samples] (fp32,
//    128-byte swizzle) into a ring of shared-memory slots;
//  * warp 1 allocates tensor memory and (one thread) issues lo*lo, hi*lo,
//    lo*hi and then hi*hi MMAs (A from TMEM, B from shared memory) into one of
//    two FP32 TMEM accumulators.  The small terms go first so the
//    accumulator's truncating additions act on a small running sum; lo*lo
//    removes the bias of the dropped product on entries of a column with
//    itself; the accumulator restarts every stage;
//  * warps 2-5 build the A tile (128 Khatri-Rao rows, one per thread), split
//    each product z = hi + lo, and store hi / lo into tensor memory (tcgen05.st);
//    with tf32 parts they also drain a quarter of the accumulator;
//  * warps 6-13 build the B tile (128 Khatri-Rao columns, half a row per
//    thread) the same way into shared memory in the canonical K-major
//    128-byte-swizzle layout, and, two stages behind, drain the accumulator into
//    an FP32 running sum in TMEM.  Each 8-column group of that sum is folded
//    into an FP64 per-CTA scratch tile once every kFoldEvery stages, the groups
//    at staggered stages, with fire-and-forget reductions; at the end of a unit
//    the drainers write the valid entries of the tile.
// The fp16 parts need |z| < 2^15: X~ arrives scaled per variable by a power of
// two (max |x| in [16, 32)), and the write-out multiplies by the inverse.
// Batched launches split fp16 products into an 8-bit hi part at even orders
// and 11 + 11 bits at odd orders (Params::h8); single-dataset launches, which
// run only where the pair kernel cannot, keep 11 + 11 bits.
// All waits are bounded: on expiry the kernel records CUM_ETIMEOUT in the
// workspace status word and every role leaves its loop.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <climits>
#include <cstring>

#include "cumgb.h"
#include "internal.h"
#include "tc_ptx.cuh"

namespace cum {
namespace tc {

constexpr int kWarpTma = 0, kWarpMma = 1, kWarpE0 = 6;
constexpr int kWarpsA = 4, kWarpsE = 8;           // A builders; B builders that also drain
constexpr int kThreads = (kWarpE0 + kWarpsE) * 32;  // 14 warps: at most 4 per SM sub-partition
constexpr int kTileM = kTcTileM, kTileN = kTcTileN;
constexpr int kTmemCols = 512;
constexpr int kAccCols = kTileN;                 // FP32 accumulator columns per buffer
constexpr int kSumBase = 2 * kAccCols;           // FP32 running sum of drained stages (128 columns)
constexpr int kAStageCols = 64;                  // hi 32 + lo 32 columns per stage
constexpr int kATmemBase = kSumBase + kTileN;    // A stages follow the running sum
constexpr int kAStages = (kTmemCols - kATmemBase) / kAStageCols;   // 2
constexpr int kBTileBytes = kTileN * 128;        // one B part (hi or lo) per stage
constexpr int kFoldEvery = 64;                   // accumulator groups between FP64 folds
constexpr int kMaxStages = 4;                    // depth of the B operand ring
// Accumulator columns drained per stage by each A builder thread; each B
// builder thread drains half of the rest.  With fp16 / bf16 parts (64 samples
// per stage) the A builders have no slack for it and the added registers
// spill; with tf32 parts they take 32 of the 128 columns.
template <int KIND>
__host__ __device__ constexpr int drain_cols_a() { return KIND == 1 ? 32 : 0; }
template <int KIND>
__host__ __device__ constexpr int drain_cols_e() { return (kTileN - drain_cols_a<KIND>()) / 2; }
constexpr int kMaxSlabs = 8;                     // depth of the X~ slab ring

struct Params {
    Shape sh;
    const int64_t* prefix;
    int64_t row_tiles;
    int64_t units;
    int S;
    int64_t kchunk;
    int64_t t_pad;
    double* out;
    double scale;
    double* scratch;
    int* status;
    int nstages;
    int slab_bytes;      // bytes of one X~ slab stage
    int box_bytes;       // bytes of one TMA box (box_rows x 128)
    int nboxes;          // boxes per stage (2 for bf16 / fp16, 1 for tf32)
    bool h8;             // fp16 parts: 8-bit hi part (even orders of batches), else 11 + 11 bits
    int nslabs;          // depth of the X~ slab ring (>= nstages)
    int slab_slot_bytes; // stride of the slab ring slots (>= slab_bytes of every unit)
    const BatchOrder* border;   // batched launch: per (dataset, order) descriptors
    const BatchUnit* bunit;     // batched launch: work list
    const int* vexp;            // fp16 parts: power-of-two scale exponent of each variable of X~
};

// What every role needs to know about the work unit it is on.
struct Unit {
    const Shape* sh;
    int s;
    int64_t I, J;
    int64_t k0, nst;
    double* out;
    double scale;
    int box_bytes, slab_bytes;
    const CUtensorMap* map;
    const int* vexp;
};

// K-major, 128-byte swizzle shared-memory matrix descriptor (8-row groups of
// 1024 bytes; the leading offset is unused for this layout).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: FP32 accumulator, A and B of the given format
// (kind::f16: 0 = fp16, 1 = bf16; kind::tf32: 2), both K-major, M = 128, N = 128.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma_tmem_a(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    if (KIND != 1)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
                d),
            "r"(a), "l"(bdesc), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
                d),
            "r"(a), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Chunk `cb` of a Khatri-Rao row within its box (bf16 / fp16: 0..3, two quads
// each; tf32: 0..7, one quad), from the row's factor addresses in that box.
template <int KIND, int NF>
__device__ __forceinline__ void build_chunk_at(const uint32_t* a, int cb, uint32_t* hi, uint32_t* lo, bool h8)
{
    if (KIND == 1) {
        float2 a01, a23;
        kr_quad_at<NF>(a, (uint32_t)cb, a01, a23);
        split_tf32(a01, hi, lo);
        split_tf32(a23, hi + 2, lo + 2);
    } else {
        float2 a01, a23, b01, b23;
        kr_quad_at<NF>(a, (uint32_t)(2 * cb), a01, a23);
        kr_quad_at<NF>(a, (uint32_t)(2 * cb + 1), b01, b23);
        if (KIND == 2 && h8) {
            split_f16_h8(a01, hi[0], lo[0]);
            split_f16_h8(a23, hi[1], lo[1]);
            split_f16_h8(b01, hi[2], lo[2]);
            split_f16_h8(b23, hi[3], lo[3]);
        } else if (KIND == 2) {
            split_f16(a01, hi[0], lo[0]);
            split_f16(a23, hi[1], lo[1]);
            split_f16(b01, hi[2], lo[2]);
            split_f16(b23, hi[3], lo[3]);
        } else {
            split_bf16(a01, hi[0], lo[0]);
            split_bf16(a23, hi[1], lo[1]);
            split_bf16(b01, hi[2], lo[2]);
            split_bf16(b23, hi[3], lo[3]);
        }
    }
}

__device__ __forceinline__ void unit_tile(const Params& P, int64_t w, int* s, int64_t* I, int64_t* J)
{
    *s = (int)(w % P.S);
    const int64_t u = w / P.S;
    int64_t lo = 0, hi = P.row_tiles;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (P.prefix[mid] <= u) lo = mid; else hi = mid;
    }
    *I = lo;
    *J = u - P.prefix[lo];
}

__device__ __forceinline__ int64_t unit_stages(const Params& P, int s, int kstg)
{
    const int64_t k0 = (int64_t)s * P.kchunk;
    const int64_t k1 = k0 + P.kchunk < P.t_pad ? k0 + P.kchunk : P.t_pad;
    return (k1 - k0) / kstg;
}

template <bool BATCH>
__device__ __forceinline__ void get_unit(const Params& P, const CUtensorMap* map, int64_t w, int kstg, Unit& u)
{
    if (BATCH) {
        const BatchUnit bu = P.bunit[w];
        const BatchOrder* o = P.border + bu.ord;
        u.sh = &o->sh;
        u.s = bu.s;
        u.I = bu.I;
        u.J = bu.J;
        u.k0 = (int64_t)bu.s * o->kchunk;
        const int64_t k1 = u.k0 + o->kchunk < o->t_pad ? u.k0 + o->kchunk : o->t_pad;
        u.nst = (k1 - u.k0) / kstg;
        u.out = o->out;
        u.scale = o->scale;
        u.box_bytes = o->box_bytes;
        u.slab_bytes = o->slab_bytes;
        u.map = o->map;
        u.vexp = o->vexp;
    } else {
        u.sh = &P.sh;
        unit_tile(P, w, &u.s, &u.I, &u.J);
        u.k0 = (int64_t)u.s * P.kchunk;
        u.nst = unit_stages(P, u.s, kstg);
        u.out = P.out;
        u.scale = P.scale;
        u.box_bytes = P.box_bytes;
        u.slab_bytes = P.slab_bytes;
        u.map = map;
        u.vexp = P.vexp;
    }
}

// ------------------------------------------------------------------ kernel

// Drain of NG groups of 8 accumulator columns [col0, col0 + 8 NG) of the
// calling thread's tile row (its TMEM lane): after each stage's MMAs the FP32
// stage sum is added into the FP32 running sum in TMEM (columns kSumBase + ...),
// which is folded into this CTA's FP64 scratch tile every kFoldEvery stages
// and at the end of the unit.
template <int NG>
struct Drainer {
    // Each group c of 8 columns keeps its own FP32 running sum and folds it into
    // the FP64 scratch tile once every kFoldEvery stages, after stage k with
    // k mod kFoldEvery = 8c + 7: the groups' folds are spread over the period
    // instead of all falling on one stage.
    static_assert(8 * NG <= kFoldEvery, "one fold phase per group");
    uint32_t tacc;      // TMEM address of column col0 of accumulator buffer 0, this lane
    uint32_t tsum;      // TMEM address of the running sum, column col0, this lane
    double* scratch;    // FP64 scratch tile of this CTA at column col0, this row
    uint32_t hbase;     // accumulator groups of the units before this one (mod 2^32: only
                        // the low two bits -- buffer and phase -- are used)
    int64_t drained;    // stages drained in this unit

    // also zeroes this thread's running sums (the folds zero them again)
    __device__ __forceinline__ void init(uint32_t tmem_lane, int col0, double* tile_row)
    {
        tacc = tmem_lane + (uint32_t)col0;
        tsum = tmem_lane + (uint32_t)(kSumBase + col0);
        scratch = tile_row + (size_t)col0 * kTileM;
        hbase = 0u;
        const uint32_t z[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
        for (int c = 0; c < NG; ++c) tmem_st8(tsum + 8 * c, z);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    __device__ __forceinline__ void begin_unit() { drained = 0; }
    // running sum of group c -> FP64 scratch: the first fold of a unit stores,
    // the later ones add with fire-and-forget reductions (each scratch element
    // belongs to this thread alone, so the order of the additions is fixed, and
    // this thread's later loads see them)
    __device__ __forceinline__ void fold_group(int c, bool first)
    {
        uint32_t v[8];
        tmem_ld8_nowait(tsum + 8 * c, v);
        tmem_wait_ld();
        const uint32_t z[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        tmem_st8(tsum + 8 * c, z);   // the running sum starts again from zero
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            double* x = scratch + (size_t)(8 * c + j) * kTileM;
            const double f = (double)__uint_as_float(v[j]);
            if (first)
                *x = f;
            else
                asm volatile("red.global.add.f64 [%0], %1;" ::"l"(x), "d"(f) : "memory");
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    // the unit's last fold of every group (after its last stage; nst stages)
    __device__ __forceinline__ void fold(int64_t nst)
    {
#pragma unroll
        for (int c = 0; c < NG; ++c) fold_group(c, 8 * c + 7 >= nst - 1);
    }
    // drain the next stage of this unit (of `nst`)
    __device__ __forceinline__ bool step(int64_t nst, uint64_t* accfull, uint64_t* accempty,
                                         volatile int* abort_flag, int* status)
    {
        const int64_t k = drained;
        const uint32_t hg = hbase + (uint32_t)k;
        const int a = (int)(hg & 1u);
        if (!wait_bar(su32(&accfull[a]), (hg >> 1) & 1u, abort_flag, status)) return false;
        fence_after();
        const uint32_t ta = tacc + (uint32_t)(a * kAccCols);
        const uint32_t kp = (uint32_t)k & (kFoldEvery - 1);
        static_assert(NG % 2 == 0, "drain groups come in pairs");
#pragma unroll
        for (int c = 0; c < NG; c += 2) {
            // two groups per tensor-memory round trip
            uint32_t v[16], u[16];
            tmem_ld16_nowait(ta + 8 * c, v);
            tmem_ld16_nowait(tsum + 8 * c, u);
            tmem_wait_ld();
            // scalar adds: the loaded registers need not form aligned pairs
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __float_as_uint(__fadd_rn(__uint_as_float(u[j]), __uint_as_float(v[j])));
            tmem_st16(tsum + 8 * c, v);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        fence_before();
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(su32(&accempty[a]));
        ++drained;
        if ((kp & 7u) == 7u && k + 1 < nst) {
            const int c = (int)(kp >> 3);
            if (c < NG) fold_group(c, k < kFoldEvery);
        }
        return true;
    }
    __device__ __forceinline__ void end_unit(int64_t nst) { hbase += (uint32_t)nst; }
};

// Write-out of columns [col0, col0 + ncols) of tile row `row` from the FP64
// scratch tile: the valid entries (last(p) <= first(q)) go to their block
// storage addresses, times the unit's scale (1/t, or 1 into split partials)
// and, for fp16 parts, times 2^-(sum of the entry's variable exponents).
template <int KIND, int DA, int DB>
__device__ __forceinline__ void write_tile(const Unit& u, int row, int col0, int ncols,
                                           const double* __restrict__ scratch)
{
    const Shape& sh = *u.sh;
    const int64_t p = u.I * kTileM + row;
    if (p >= sh.rows) return;
    const int64_t q0 = u.J * kTileN + col0;
    const int64_t left = sh.cols - q0;
    const int nc = left < ncols ? (int)left : ncols;   // columns of the range inside the matrix
    if (nc <= 0) return;
    const RowInfo r = decode_row(p, DA, DB, sh.b, sh.nbar, sh.bdA, sh.bdB, sh.bd);
    double* __restrict__ dst = u.out + (int64_t)u.s * sh.entries + r.off;
    const int bdB = (int)sh.bdB;
    // column q = tu * bdB + rem: dB-tuple tu, in-block offset rem
    int64_t tu = q0 / bdB;
    int rem = (int)(q0 - tu * bdB);
    int64_t cbase = 0;
    int cfirst = 0;
    // fp16 parts: the entry of variables v_1..v_d was computed from X~ scaled
    // by 2^vexp[v] per variable; undo sum_k vexp[v_k] exactly.  The column's
    // in-block digits advance like an odometer.
    int rexp = 0, cblk[DB], dig[DB];
    decode_col_tuple(tu, DA, DB, sh.nbar, sh.bd, &cbase, &cfirst, KIND == 2 ? cblk : nullptr);
    if (KIND == 2) {
#pragma unroll
        for (int f = 0; f < DA; ++f) rexp += __ldg(u.vexp + r.col[f]);
        int x = rem;
#pragma unroll
        for (int k = DB - 1; k >= 0; --k) {
            dig[k] = x % sh.b;
            x /= sh.b;
        }
    }
    // 16 scratch loads in flight at a time (the range is a multiple of 16
    // columns of the 128-column scratch tile, so all of them are in bounds)
    constexpr int kBatch = 16;
    for (int j0 = 0; j0 < nc; j0 += kBatch) {
        double v[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) v[k] = scratch[(size_t)(j0 + k) * kTileM];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            if (j0 + k >= nc) break;
            if (r.last <= cfirst) {
                double f = u.scale;
                if (KIND == 2) {
                    int e = rexp;
#pragma unroll
                    for (int i = 0; i < DB; ++i) e += __ldg(u.vexp + cblk[i] * sh.b + dig[i]);
                    f *= exp2_neg(e);
                }
                dst[cbase + rem] = v[k] * f;
            }
            if (++rem == bdB) {
                rem = 0;
                ++tu;
                if (j0 + k + 1 < nc)
                    decode_col_tuple(tu, DA, DB, sh.nbar, sh.bd, &cbase, &cfirst, KIND == 2 ? cblk : nullptr);
                if (KIND == 2) {
#pragma unroll
                    for (int i = 0; i < DB; ++i) dig[i] = 0;
                }
            } else if (KIND == 2) {
#pragma unroll
                for (int i = DB - 1; i >= 0; --i) {
                    if (++dig[i] < sh.b) break;
                    dig[i] = 0;
                }
            }
        }
    }
}

template <int KIND, int DA, int DB, bool BATCH>
__global__ void __launch_bounds__(kThreads, 1) moment_tc_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                const __grid_constant__ Params P)
{
    constexpr int KSTG = KIND == 1 ? 32 : 64;   // samples per stage
    constexpr uint32_t IDESC = instr_desc(KIND == 0 ? 1u : KIND == 1 ? 2u : 0u);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int NS = P.nstages;                   // B ring (shared memory)
    const int NX = P.nslabs;                    // X~ slab ring (shared memory)
    uint8_t* slab = smem;
    uint8_t* bhi = slab + NX * P.slab_slot_bytes;
    uint8_t* blo = bhi + NS * kBTileBytes;
    uint64_t* bars = (uint64_t*)(blo + NS * kBTileBytes);
    uint64_t* xfull = bars;
    uint64_t* xempty = bars + kMaxSlabs;
    uint64_t* bfull = bars + 2 * kMaxSlabs;
    uint64_t* bempty = bfull + kMaxStages;
    uint64_t* afull = bempty + kMaxStages;      // A ring (tensor memory), kAStages slots
    uint64_t* aempty = afull + kAStages;
    uint64_t* accfull = aempty + kAStages;
    uint64_t* accempty = accfull + 2;
    uint32_t* tmem_slot = (uint32_t*)(accempty + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NX; ++i) {
            mbar_init(su32(&xfull[i]), 1);
            mbar_init(su32(&xempty[i]), kWarpsA + kWarpsE);
        }
        for (int i = 0; i < NS; ++i) {
            mbar_init(su32(&bfull[i]), kWarpsE);
            mbar_init(su32(&bempty[i]), 1);
        }
        for (int i = 0; i < kAStages; ++i) {
            mbar_init(su32(&afull[i]), kWarpsA);
            mbar_init(su32(&aempty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(su32(&accfull[i]), 1);
            mbar_init(su32(&accempty[i]), (drain_cols_a<KIND>() > 0 ? kWarpsA : 0) + kWarpsE);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kWarpMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == kWarpTma) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
            Ring xr(NX);
            bool ok = true;
            for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
                Unit u;
                get_unit<BATCH>(P, &tmap, w, KSTG, u);
                for (int64_t st = 0; st < u.nst; ++st, xr.next()) {
                    if (!(ok = wait_bar(su32(&xempty[xr.slot]), xr.phase ^ 1u, abort_flag, P.status))) break;
                    mbar_expect_tx(su32(&xfull[xr.slot]), (uint32_t)u.slab_bytes);
                    const int x0 = (int)(u.k0 + st * KSTG);
                    for (int h = 0; h < P.nboxes; ++h)
                        tma_load_2d(su32(slab + xr.slot * P.slab_slot_bytes + h * u.box_bytes), u.map, x0 + 32 * h,
                                    0, su32(&xfull[xr.slot]));
                }
            }
        }
    } else if (warp == kWarpMma) {
        // ---------------------------------------------------------- MMA issuer
        // One stage per accumulator group: wait for the stage's A and B operands
        // and for the accumulator buffer, then issue the 16 MMAs (lo*lo and the
        // cross terms first) and 3 commits as one straight sequence.  Descriptors come from
        // precomputed bases plus slot offsets, so the issuing thread -- which
        // shares its sub-partition with busy builder warps -- runs few other
        // instructions between MMAs.
        if (lane == 0) {
            Ring ar(kAStages), br(NS);
            const uint64_t bh0 = smem_desc(su32(bhi)), bl0 = smem_desc(su32(blo));
            const uint32_t a0 = tmem + (uint32_t)kATmemBase;
            int64_t h = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
                Unit u;
                get_unit<BATCH>(P, &tmap, w, KSTG, u);
                const int64_t nst = u.nst;
                for (int64_t st = 0; st < nst; ++st, ++h, ar.next(), br.next()) {
                    ok = wait_bar(su32(&afull[ar.slot]), ar.phase, abort_flag, P.status) &&
                         wait_bar(su32(&bfull[br.slot]), br.phase, abort_flag, P.status);
                    const int a = (int)(h & 1);
                    if (ok && h >= 2) ok = wait_bar(su32(&accempty[a]), (uint32_t)((h >> 1) & 1) ^ 1u, abort_flag,
                                                   P.status);
                    if (!ok) break;
                    fence_after();
                    const uint32_t d = tmem + (uint32_t)(a * kAccCols);
                    const uint64_t boff = (uint64_t)br.slot * (uint64_t)(kBTileBytes >> 4);
                    const uint64_t bh = bh0 + boff, bl = bl0 + boff;
                    const uint32_t ahi = a0 + (uint32_t)(ar.slot * kAStageCols), alo = ahi + 32u;
                    mma_tmem_a<KIND>(d, alo + 0, bl + 0, IDESC, 0u);
                    mma_tmem_a<KIND>(d, alo + 8, bl + 2, IDESC, 1u);
                    mma_tmem_a<KIND>(d, alo + 16, bl + 4, IDESC, 1u);
                    mma_tmem_a<KIND>(d, alo + 24, bl + 6, IDESC, 1u);
                    mma_tmem_a<KIND>(d, ahi + 0, bl + 0, IDESC, 1u);
                    mma_tmem_a<KIND>(d, ahi + 8, bl + 2, IDESC, 1u);
                    mma_tmem_a<KIND>(d, ahi + 16, bl + 4, IDESC, 1u);
                    mma_tmem_a<KIND>(d, ahi + 24, bl + 6, IDESC, 1u);
                    mma_tmem_a<KIND>(d, alo + 0, bh + 0, IDESC, 1u);
                    mma_tmem_a<KIND>(d, alo + 8, bh + 2, IDESC, 1u);
                    mma_tmem_a<KIND>(d, alo + 16, bh + 4, IDESC, 1u);
                    mma_tmem_a<KIND>(d, alo + 24, bh + 6, IDESC, 1u);
                    mma_tmem_a<KIND>(d, ahi + 0, bh + 0, IDESC, 1u);
                    mma_tmem_a<KIND>(d, ahi + 8, bh + 2, IDESC, 1u);
                    mma_tmem_a<KIND>(d, ahi + 16, bh + 4, IDESC, 1u);
                    mma_tmem_a<KIND>(d, ahi + 24, bh + 6, IDESC, 1u);
                    mma_commit(su32(&aempty[ar.slot]));
                    mma_commit(su32(&bempty[br.slot]));
                    mma_commit(su32(&accfull[a]));
                }
            }
        }
    } else if (warp < kWarpE0) {
        // ---------------------------------------------------------- A builder (TMEM) + drain
        // Each thread builds one Khatri-Rao row of A per stage into tensor
        // memory.  With tf32 parts it also drains columns [0, kDrainColsA) of its
        // row: waiting for the A slot of stage st means MMA(st - 2) has
        // completed, so the drain of that stage's accumulator comes first.
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        constexpr int kDrainColsA = drain_cols_a<KIND>();
        static_assert(kDrainColsA % 8 == 0, "drains move groups of 8 columns");
        static_assert(kDrainColsA % 16 == 0, "the write-out loads 16 columns at a time");
        Drainer<kDrainColsA / 8> dr;
        dr.init(tmem + lane_off, 0, P.scratch + (size_t)blockIdx.x * kTileM * kTileN + row);
        Ring ar(kAStages), xr(NX);
        bool ok = true;
        for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
            Unit u;
            get_unit<BATCH>(P, &tmap, w, KSTG, u);
            const Shape& sh = *u.sh;
            int col[DA];
            const int64_t p = u.I * kTileM + row;
            if (p < sh.rows) {
                const RowInfo r = decode_row(p, DA, DB, sh.b, sh.nbar, sh.bdA, sh.bdB, sh.bd);
#pragma unroll
                for (int f = 0; f < DA; ++f) col[f] = r.col[f];
            } else {
#pragma unroll
                for (int f = 0; f < DA; ++f) col[f] = 0;
            }
            KrRow<DA> kr;
            kr.set(col);
            const int64_t nst = u.nst;
            const uint32_t box_bytes = (uint32_t)u.box_bytes;
            dr.begin_unit();
            for (int64_t st = 0; st < nst; ++st, ar.next(), xr.next()) {
                if (!(ok = wait_bar(su32(&xfull[xr.slot]), xr.phase, abort_flag, P.status))) break;
                if (!(ok = wait_bar(su32(&aempty[ar.slot]), ar.phase ^ 1u, abort_flag, P.status))) break;
                if (kDrainColsA > 0 && st >= 2 && !(ok = dr.step(nst, accfull, accempty, abort_flag, P.status)))
                    break;
                const uint32_t s32 = su32(slab) + (uint32_t)(xr.slot * P.slab_slot_bytes);
                const uint32_t tb = tmem + lane_off + (uint32_t)(kATmemBase + ar.slot * kAStageCols);
                uint32_t ab[2][DA];   // factor addresses in box 0 and box 1
                kr.addresses(s32, ab[0]);
#pragma unroll
                for (int f = 0; f < DA; ++f) ab[1][f] = ab[0][f] + box_bytes;
#pragma unroll
                for (int q = 0; q < 8; q += 2) {
                    uint32_t hw[8], lw[8];
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        if (KIND == 1)
                            build_chunk_at<KIND, DA>(ab[0], q + c, hw + 4 * c, lw + 4 * c, P.h8);
                        else
                            build_chunk_at<KIND, DA>(ab[(q + c) >> 2], (q + c) & 3, hw + 4 * c, lw + 4 * c, P.h8);
                    }
                    tmem_st8(tb + 4 * q, hw);
                    tmem_st8(tb + 32 + 4 * q, lw);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(su32(&xempty[xr.slot]));
                    mbar_arrive(su32(&afull[ar.slot]));
                }
            }
            if (kDrainColsA > 0) {
                while (ok && dr.drained < nst) ok = dr.step(nst, accfull, accempty, abort_flag, P.status);
                if (!ok) break;
                dr.fold(nst);
                Unit uw;   // fetched again rather than kept live across the stage loop
                get_unit<BATCH>(P, &tmap, w, KSTG, uw);
                write_tile<KIND, DA, DB>(uw, row, 0, kDrainColsA, dr.scratch);
                dr.end_unit(nst);
            }
        }
    } else {
        // ---------------------------------------------------------- B builder + drain
        // Each thread builds half (4 chunks) of one B row per stage.  Two stages
        // later it drains kDrainColsE accumulator columns of one row.
        const int e = threadIdx.x - kWarpE0 * 32;     // 0..255
        const int bq = e & (kTileN - 1);               // B tile row
        const int bc0 = (e >> 7) * 4;                  // first chunk of this thread
        const int swz_row = (bq >> 3) * 1024 + (bq & 7) * 128;
        const int quarter = warp & 3;
        const int half = (warp - kWarpE0) >> 2;        // which of the two column ranges is drained here
        const int row = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        constexpr int kDrainColsE = drain_cols_e<KIND>();
        static_assert(kDrainColsE % 8 == 0, "drains move groups of 8 columns");
        static_assert(kDrainColsE % 16 == 0, "the write-out loads 16 columns at a time");
        const int dcol0 = drain_cols_a<KIND>() + half * kDrainColsE;
        Drainer<kDrainColsE / 8> dr;
        dr.init(tmem + lane_off, dcol0, P.scratch + (size_t)blockIdx.x * kTileM * kTileN + row);
        Ring br(NS), xr(NX);
        bool ok = true;
        for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
            Unit u;
            get_unit<BATCH>(P, &tmap, w, KSTG, u);
            const Shape& sh = *u.sh;
            const uint32_t box_bytes = (uint32_t)u.box_bytes;
            int col[DB];
            {
                const int64_t qq = u.J * kTileN + bq;
                if (qq < sh.cols) {
                    const ColInfo c = decode_col(qq, DA, DB, sh.b, sh.nbar, sh.bdB, sh.bd);
#pragma unroll
                    for (int f = 0; f < DB; ++f) col[f] = c.col[f];
                } else {
#pragma unroll
                    for (int f = 0; f < DB; ++f) col[f] = 0;
                }
            }
            KrRow<DB> kr;
            kr.set(col);
            const int64_t nst = u.nst;
            dr.begin_unit();
            for (int64_t st = 0; st < nst; ++st, br.next(), xr.next()) {
                if (!(ok = wait_bar(su32(&xfull[xr.slot]), xr.phase, abort_flag, P.status))) break;
                if (!(ok = wait_bar(su32(&bempty[br.slot]), br.phase ^ 1u, abort_flag, P.status))) break;
                const uint32_t s32 = su32(slab) + (uint32_t)(xr.slot * P.slab_slot_bytes);
                // B row bq in this slot: chunk ch = bc0 + c sits at row base + ((ch ^ (bq & 7)) << 4)
                // = (row base + ((bc0 ^ (bq & 7)) << 4)) ^ (c << 4): row bases keep bits 4-6 clear
                const uint32_t sh =
                    su32(bhi) + (uint32_t)(br.slot * kBTileBytes + swz_row + (((bq & 7) ^ bc0) << 4));
                const uint32_t sl32 = sh + (uint32_t)(blo - bhi);
                uint32_t ab[DB];   // factor addresses in this thread's box (chunks bc0..bc0+3)
                kr.addresses(s32 + (KIND == 1 ? 0u : (uint32_t)(bc0 >> 2) * box_bytes), ab);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int ch = bc0 + c;
                    uint32_t hw[4], lw[4];
                    build_chunk_at<KIND, DB>(ab, KIND == 1 ? ch : c, hw, lw, P.h8);
                    sts128(sh ^ ((uint32_t)c << 4), hw[0], hw[1], hw[2], hw[3]);
                    sts128(sl32 ^ ((uint32_t)c << 4), lw[0], lw[1], lw[2], lw[3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(su32(&xempty[xr.slot]));
                    mbar_arrive(su32(&bfull[br.slot]));
                }
                // drain stage st - 2: the build of the next stages never waits for
                // the drain, and the MMA of stage st needs only the drain of st - 2
                if (st >= 2 && !(ok = dr.step(nst, accfull, accempty, abort_flag, P.status))) break;
            }
            while (ok && dr.drained < nst) ok = dr.step(nst, accfull, accempty, abort_flag, P.status);
            if (!ok) break;
            dr.fold(nst);
            {
                Unit uw;   // fetched again rather than kept live across the stage loop
                get_unit<BATCH>(P, &tmap, w, KSTG, uw);
                write_tile<KIND, DA, DB>(uw, row, dcol0, kDrainColsE, dr.scratch);
            }
            dr.end_unit(nst);
        }
    }

    fence_before();
    __syncthreads();
    if (warp == kWarpMma) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// Diagnostic of the bounded wait: one thread waits on an mbarrier that nothing
// arrives at, until the limit expires and CUM_ETIMEOUT is recorded in `status`.
// Nothing is in flight when it returns, so the context stays usable.
__global__ void bounded_wait_probe_kernel(int* status)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    mbar_init(su32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    wait_bar(su32(&bar), 0u, &abort_flag, status);
}

// ------------------------------------------------------------------ host

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

size_t smem_bytes(int nstages, int nslabs, int slab_bytes)
{
    return 1024 + (size_t)nslabs * slab_bytes + (size_t)nstages * 2 * kBTileBytes +
           8 * (2 * kMaxSlabs + 2 * kMaxStages + 2 * kAStages + 4) + 16;
}

template <int KIND, int DA, int DB, bool BATCH>
static cudaError_t launch_typed(const CUtensorMap& map, const Params& P, int grid, size_t smem, cudaStream_t st)
{
    auto kern = moment_tc_kernel<KIND, DA, DB, BATCH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kThreads, smem, st>>>(map, P);
    return cudaGetLastError();
}

template <int KIND, bool BATCH>
static cudaError_t launch_kind(const CUtensorMap& map, const Params& P, int dA, int dB, int grid, size_t smem,
                               cudaStream_t st)
{
    if (dA == 1 && dB == 1) return launch_typed<KIND, 1, 1, BATCH>(map, P, grid, smem, st);
    if (dA == 2 && dB == 1) return launch_typed<KIND, 2, 1, BATCH>(map, P, grid, smem, st);
    if (dA == 2 && dB == 2) return launch_typed<KIND, 2, 2, BATCH>(map, P, grid, smem, st);
    if (dA == 3 && dB == 2) return launch_typed<KIND, 3, 2, BATCH>(map, P, grid, smem, st);
    if (dA == 3 && dB == 3) return launch_typed<KIND, 3, 3, BATCH>(map, P, grid, smem, st);
    return cudaErrorInvalidValue;
}

// Ring depths, shared memory and grid for slabs of `slab_bytes` (the largest
// slab of the launch) and `units` work units.
static cudaError_t configure(Params& P, int slab_bytes, int64_t units, int* grid, size_t* smem)
{
    int dev = 0, sms = 0, maxsmem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    int ns = kMaxStages;
    while (ns > 2 && smem_bytes(ns, ns, slab_bytes) > (size_t)maxsmem) --ns;
    if (smem_bytes(ns, ns, slab_bytes) > (size_t)maxsmem) return cudaErrorInvalidValue;
    int nx = kMaxSlabs;
    while (nx > ns && smem_bytes(ns, nx, slab_bytes) > (size_t)maxsmem) --nx;
    P.nstages = ns;
    P.nslabs = nx;
    P.slab_slot_bytes = slab_bytes;
    int g = (int)(units < sms ? units : sms);
    if (g > kTcMaxCtas) g = kTcMaxCtas;
    *grid = g;
    *smem = smem_bytes(ns, nx, slab_bytes);
    return cudaSuccess;
}

}  // namespace tc

cudaError_t launch_bounded_wait_probe(int* status, cudaStream_t st)
{
    tc::bounded_wait_probe_kernel<<<1, 1, 0, st>>>(status);
    return cudaGetLastError();
}

int tc_box_rows(int n_pad) { return (n_pad + 7) / 8 * 8; }

int tc_slab_bytes(int n_pad, int prec) { return tc_box_rows(n_pad) * 128 * (prec == CUM_PREC_TF32X3 ? 1 : 2); }

bool encode_xt_map(CUtensorMap* map, const float* xt, int64_t t_pad, int n_pad)
{
    auto enc = tc::encode_fn();
    if (!enc) return false;
    const int box_rows = tc_box_rows(n_pad);
    if (box_rows > kTcMaxNPad) return false;
    cuuint64_t dims[2] = {(cuuint64_t)t_pad, (cuuint64_t)n_pad};
    cuuint64_t strides[1] = {(cuuint64_t)t_pad * sizeof(float)};
    cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)xt, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static int tc_kind(int prec) { return prec == CUM_PREC_TF32X3 ? 1 : prec == CUM_PREC_FP16X3 ? 2 : 0; }

template <bool BATCH>
static cudaError_t launch_prec(int kind, const CUtensorMap& map, const tc::Params& P, int dA, int dB, int grid,
                               size_t smem, cudaStream_t st)
{
    using namespace tc;
    if (kind == 1) return launch_kind<1, BATCH>(map, P, dA, dB, grid, smem, st);
    if (kind == 2) return launch_kind<2, BATCH>(map, P, dA, dB, grid, smem, st);
    return launch_kind<0, BATCH>(map, P, dA, dB, grid, smem, st);
}

cudaError_t launch_moment_tc(const OrderPlan& OP, int prec, const float* xt, int64_t t_pad, const int64_t* prefix,
                             double* out, double scale, double* scratch, int* status, const int* vexp,
                             cudaStream_t st)
{
    using namespace tc;
    if (OP.units <= 0) return cudaSuccess;
    const int kind = tc_kind(prec);
    if (kind == 2 && !vexp) return cudaErrorInvalidValue;
    Params P;
    std::memset(&P, 0, sizeof(P));
    P.sh = OP.sh;
    P.prefix = prefix;
    P.row_tiles = OP.row_tiles;
    P.units = OP.units;
    P.S = OP.splits;
    P.kchunk = OP.kchunk;
    P.t_pad = t_pad;
    P.out = out;
    P.scale = scale;
    P.scratch = scratch;
    P.status = status;
    P.box_bytes = tc_box_rows(OP.sh.n_pad) * 128;
    P.nboxes = kind == 1 ? 1 : 2;
    P.vexp = vexp;
    P.slab_bytes = P.box_bytes * P.nboxes;
    CUtensorMap map;
    if (!encode_xt_map(&map, xt, t_pad, OP.sh.n_pad)) return cudaErrorInvalidValue;
    int grid = 0;
    size_t smem = 0;
    cudaError_t e = configure(P, P.slab_bytes, OP.units, &grid, &smem);
    if (e != cudaSuccess) return e;
    return launch_prec<false>(kind, map, P, OP.sh.dA, OP.sh.dB, grid, smem, st);
}

cudaError_t launch_moment_tc_batch(int prec, int dA, int dB, const BatchOrder* orders, const BatchUnit* units,
                                   int64_t nunits, int max_slab_bytes, double* scratch, int* status, cudaStream_t st)
{
    using namespace tc;
    if (nunits <= 0) return cudaSuccess;
    const int kind = tc_kind(prec);
    Params P;
    std::memset(&P, 0, sizeof(P));
    P.units = nunits;
    P.scratch = scratch;
    P.status = status;
    P.nboxes = kind == 1 ? 1 : 2;
    // fp16 parts of a batch: the 8-bit hi part at even orders, where the
    // truncation bias of the accumulation dominates (it keeps the hi*hi
    // products exact on the tensor core's alignment grid); 11 + 11 bits at odd
    // orders, whose small moments feel the shorter parts' representation error
    // more (512 mixed datasets: order 4 worst 9.0e-7 against 1.06e-6, order 3
    // 3.1e-7 against 6.9e-7)
    P.h8 = (dA + dB) % 2 == 0;
    P.border = orders;
    P.bunit = units;
    CUtensorMap unused;
    std::memset(&unused, 0, sizeof(unused));
    int grid = 0;
    size_t smem = 0;
    cudaError_t e = configure(P, max_slab_bytes, nunits, &grid, &smem);
    if (e != cudaSuccess) return e;
    return launch_prec<true>(kind, unused, P, dA, dB, grid, smem, st);
}

}  // namespace cum
