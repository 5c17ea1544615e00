// Tensor-core moment contraction on CTA pairs (tcgen05 cta_group::2) for the
// fp16 and bf16 split precisions.
//
// Computes, for one order d, the block-stored sums
//   M[rowOff(p) + colOff(q)] = scale * sum_l ZA[l, p] * ZB[l, q]      (Alg. 1-2)
// over the valid pairs last(p) <= first(q), like moment_tc.cu, on output tiles
// of 256 x 256 per pair of CTAs (a cluster of two, one per SM of a TPC):
//  * warp 0 of each CTA TMA-loads its X~ slabs (32 fp32 samples of every
//    variable, 128-byte swizzle);
//  * 8 builder warps of CTA c build, per stage of 32 samples, the Khatri-Rao
//    rows p = 256 I + 128 c + (0..127) of A and, for each quarter k of the
//    tile's columns, the B rows q = 256 J + 64 k + 32 c + (0..31), as
//    fp16/bf16 hi and lo parts in shared memory (K-major, 64-byte swizzle);
//  * one thread of the even CTA issues, per stage and quarter, 8 MMAs of
//    M = 256 (128 rows from each CTA's shared memory), N = 64, K = 16:
//    lo*lo, hi*lo, lo*hi, then hi*hi, over the stage's two K steps, into that
//    quarter's FP32 accumulator in each CTA's tensor memory.  Each accumulator
//    therefore restarts every 32 samples: the tensor core's truncating
//    additions act on chains of two K steps only, and the lo*lo term removes
//    the bias of the dropped product on entries of a column with itself;
//  * 8 drainer warps add each quarter's stage sum into an FP32 running sum in
//    tensor memory while the MMAs of the other quarters run, fold it into an
//    FP64 scratch tile every 4096 samples, and write the valid entries of
//    their tile rows to block storage while the builders start the next unit.
// Per stage a CTA builds 256 Khatri-Rao rows for 128 x 256 outputs, half the
// build work per output of the one-CTA kernel.
// All waits are bounded: on expiry the kernel records CUM_ETIMEOUT in the
// workspace status word and every role leaves its loop.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "cumgb.h"
#include "internal.h"
#include "tc_ptx.cuh"

namespace cum {
namespace pair {
using namespace tc;

constexpr int kWarpTma = 0, kWarpMma = 1, kWarpB0 = 2, kWarpD0 = 10;
constexpr int kBuildWarps = 8, kDrainWarps = 8;
constexpr int kThreads = (kWarpD0 + kDrainWarps) * 32;    // 576: 18 warps
constexpr int kTileM = kPairTileM, kTileN = kPairTileN;   // 256 x 256 per pair
constexpr int kRows = 128;                  // A rows (tensor-memory lanes) per CTA
constexpr int kQuarters = 4;
constexpr int kQN = kTileN / kQuarters;     // accumulator columns per quarter (MMA N = 64)
constexpr int kQB = kQN / 2;                // B rows per CTA per quarter
constexpr int kStage = 32;                  // samples per stage
constexpr int kRowBytes = 64;               // 32 fp16 / bf16 samples
constexpr int kPartBytes = 128 * kRowBytes; // one part (hi or lo) of A or of B: 128 rows
constexpr int kSlotBytes = 4 * kPartBytes;  // A hi, A lo, B hi, B lo
constexpr int kSumBase = kTileN;            // running sum: tensor-memory columns 256..511
constexpr int kTmemCols = 512;
constexpr int kFoldEvery = 128;             // stages between FP64 folds (4096 samples)
constexpr int kMaxSlots = 4, kMaxSlabs = 8;
constexpr int kDrainCols = 32;              // columns of each quarter a drainer thread owns

struct Params {
    Shape sh;
    const int64_t* prefix;   // row tile I -> first work unit of I's active column tiles
    int64_t row_tiles;
    int64_t units;
    int S;
    int64_t kchunk;
    int64_t t_pad;
    double* out;
    double scale;
    double* scratch;         // per CTA: 256 columns x 128 rows of FP64
    int* status;
    int nslots;              // operand ring depth
    int nslabs;              // X~ slab ring depth
    int box_bytes;           // one X~ box: box rows x 128 bytes (32 fp32 samples)
    const int* vexp;         // fp16 parts: power-of-two scale exponent of each variable
};

// ------------------------------------------------------------------ cluster PTX

__device__ __forceinline__ uint32_t cta_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Arrive on the mbarrier at local address `bar` of CTA `cta` of the cluster.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t bar, uint32_t cta)
{
    asm volatile(
        "{\n .reg .b32 ra;\n mapa.shared::cluster.u32 ra, %0, %1;\n"
        " mbarrier.arrive.release.cluster.shared::cluster.b64 _, [ra];\n}\n" ::"r"(bar),
        "r"(cta)
        : "memory");
}

// Arrive with no memory ordering (relaxed, cluster scope) on the mbarrier at
// local address `bar` of CTA `cta`: for signals about tensor memory only, whose
// accesses tcgen05.fence::before_thread_sync already orders before the arrive.
__device__ __forceinline__ void mbar_arrive_remote_relaxed(uint32_t bar, uint32_t cta)
{
    asm volatile(
        "{\n .reg .b32 ra;\n mapa.shared::cluster.u32 ra, %0, %1;\n"
        " mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [ra];\n}\n" ::"r"(bar),
        "r"(cta)
        : "memory");
}

// try_wait with cluster-scope acquire: the phase may have been completed by
// arrivals of the peer CTA, whose shared-memory writes must be visible.
__device__ __forceinline__ bool mbar_try_cluster(uint32_t bar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool wait_cluster(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status)
{
    if (mbar_try_cluster(bar, parity, 0u)) return true;
    const long long t0 = clock64();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_cluster(bar, parity, 20000u)) return true;
        if ((i & 15u) == 0u) {
            if (*abort_flag) return false;
            if (clock64() - t0 > kWaitLimit) {
                *abort_flag = 1;
                atomicExch(status, CUM_ETIMEOUT);
                return false;
            }
        }
    }
}

// K-major, 64-byte swizzle shared-memory matrix descriptor: rows of 64 bytes,
// 8-row groups of 512 bytes (stride), layout type 4.
__device__ __forceinline__ uint64_t smem_desc64(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Instruction descriptor: FP32 accumulator, A and B fp16 (fmt 0) or bf16
// (fmt 1), both K-major, M = 256 (the pair), N = 64 (one quarter).
__host__ __device__ constexpr uint32_t idesc_pair(uint32_t fmt)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kQN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

__device__ __forceinline__ void mma_pair(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// Arrive on the mbarrier at local address `bar` in both CTAs of the pair once
// every tcgen05 operation this thread issued before has completed.
__device__ __forceinline__ void commit_both(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            bar),
        "h"((uint16_t)3)
        : "memory");
}

// CTA-local named barrier of `count` threads (id 1; 0 is __syncthreads)
// that also ORs a flag over them: every thread of the role joins it every
// stage, and all learn together whether any of them failed a bounded wait, so
// they leave their loops together and none is left waiting at the barrier.
__device__ __forceinline__ bool named_sync_any(uint32_t id, uint32_t count, bool flag)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.cta.red.or.pred q, %2, %3, p;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)flag), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// Byte offset of 16-byte chunk `ch` (0..3) of row `r` in a 64-byte-swizzled
// part (the part base is 1024-byte aligned): address bits 4-5 are XORed with
// bits 7-8.
__device__ __forceinline__ uint32_t sw64(int r, int ch) { return (uint32_t)(r * kRowBytes + ((ch ^ ((r >> 1) & 3)) << 4)); }

// ------------------------------------------------------------------ work units

struct Unit {
    int s;              // t chunk
    int64_t I, J;       // 256-row tile, 256-column tile
    int64_t k0, nst;    // first sample, stages of 32 samples
};

__device__ __forceinline__ void get_unit(const Params& P, int64_t w, Unit& u)
{
    u.s = (int)(w % P.S);
    const int64_t v = w / P.S;
    int64_t lo = 0, hi = P.row_tiles;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (P.prefix[mid] <= v) lo = mid; else hi = mid;
    }
    u.I = lo;
    u.J = v - P.prefix[lo];
    u.k0 = (int64_t)u.s * P.kchunk;
    const int64_t k1 = u.k0 + P.kchunk < P.t_pad ? u.k0 + P.kchunk : P.t_pad;
    u.nst = (k1 - u.k0) / kStage;
}

// Write-out of output row p, columns [q0, q0 + ncols) from FP64 scratch
// (`scr`: column j at scr[j * kRows]): the valid entries (last(p) <= first(q))
// go to their block-storage addresses, times the unit's scale (1/t, or 1 into
// split partials) and, for fp16 parts, times 2^-(sum of the entry's variable
// exponents).  ncols is a multiple of 16.
template <int KIND, int DA, int DB>
__device__ __forceinline__ void write_segment(const Params& P, const Unit& u, int64_t p, int64_t q0, int ncols,
                                              const double* __restrict__ scr)
{
    const Shape& sh = P.sh;
    if (p >= sh.rows) return;
    const int64_t left = sh.cols - q0;
    const int nc = left < ncols ? (int)left : ncols;
    if (nc <= 0) return;
    const RowInfo r = decode_row(p, DA, DB, sh.b, sh.nbar, sh.bdA, sh.bdB, sh.bd);
    double* __restrict__ dst = P.out + (int64_t)u.s * sh.entries + r.off;
    const int bdB = (int)sh.bdB;
    int64_t tu = q0 / bdB;
    int rem = (int)(q0 - tu * bdB);
    int64_t cbase = 0;
    int cfirst = 0;
    int rexp = 0, cblk[DB], dig[DB];
    decode_col_tuple(tu, DA, DB, sh.nbar, sh.bd, &cbase, &cfirst, KIND == 2 ? cblk : nullptr);
    if (KIND == 2) {
#pragma unroll
        for (int f = 0; f < DA; ++f) rexp += __ldg(P.vexp + r.col[f]);
        int x = rem;
#pragma unroll
        for (int k = DB - 1; k >= 0; --k) {
            dig[k] = x % sh.b;
            x /= sh.b;
        }
    }
    constexpr int kBatch = 16;
    for (int j0 = 0; j0 < nc; j0 += kBatch) {
        double v[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) v[k] = scr[(size_t)(j0 + k) * kRows];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            if (j0 + k >= nc) break;
            if (r.last <= cfirst) {
                double f = P.scale;
                if (KIND == 2) {
                    int e = rexp;
#pragma unroll
                    for (int i = 0; i < DB; ++i) e += __ldg(P.vexp + cblk[i] * sh.b + dig[i]);
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

// One 8-sample chunk `cb` (0..3) of a Khatri-Rao row of NF factors in the
// stage's box, split into packed hi / lo parts (element 0 in the low half).
template <int KIND, int NF>
__device__ __forceinline__ void build_chunk(const uint32_t* a, int cb, uint32_t* hi, uint32_t* lo)
{
    float2 z01, z23, w01, w23;
    kr_quad_at<NF>(a, (uint32_t)(2 * cb), z01, z23);
    kr_quad_at<NF>(a, (uint32_t)(2 * cb + 1), w01, w23);
    if (KIND == 2) {
        split_f16(z01, hi[0], lo[0]);
        split_f16(z23, hi[1], lo[1]);
        split_f16(w01, hi[2], lo[2]);
        split_f16(w23, hi[3], lo[3]);
    } else {
        split_bf16(z01, hi[0], lo[0]);
        split_bf16(z23, hi[1], lo[1]);
        split_bf16(w01, hi[2], lo[2]);
        split_bf16(w23, hi[3], lo[3]);
    }
}

// ------------------------------------------------------------------ kernel

template <int KIND, int DA, int DB>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    moment_pair_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ Params P)
{
    constexpr uint32_t IDESC = idesc_pair(KIND == 0 ? 1u : 0u);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int NS = P.nslots, NX = P.nslabs;
    uint8_t* slots = smem;                                   // NS x (A hi, A lo, B hi, B lo)
    uint8_t* slab = slots + NS * kSlotBytes;                 // NX x one X~ box
    uint64_t* bars = (uint64_t*)(slab + NX * P.box_bytes);
    uint64_t* xfull = bars;
    uint64_t* xempty = xfull + kMaxSlabs;
    uint64_t* opfull = xempty + kMaxSlabs;       // used in the even CTA: both CTAs' builders arrive
    uint64_t* opempty = opfull + kMaxSlots;      // completed by the MMA commits, in both CTAs
    uint64_t* accfull = opempty + kMaxSlots;     // per quarter, in both CTAs
    uint64_t* accempty = accfull + kQuarters;    // per quarter, in the even CTA: both CTAs' drainers arrive
    uint64_t* mmadone = accempty + kQuarters;
    uint32_t* tmem_slot = (uint32_t*)(mmadone + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const uint32_t cta = cta_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        // each role gathers its warps on a named barrier and one thread then
        // arrives for the CTA: one cluster-scope release per CTA and event
        for (int i = 0; i < NX; ++i) {
            mbar_init(su32(&xfull[i]), 1);
            mbar_init(su32(&xempty[i]), 1);
        }
        for (int i = 0; i < NS; ++i) {
            mbar_init(su32(&opfull[i]), 2);
            mbar_init(su32(&opempty[i]), 1);
        }
        for (int q = 0; q < kQuarters; ++q) {
            mbar_init(su32(&accfull[q]), 1);
            mbar_init(su32(&accempty[q]), 2 * kDrainWarps);
        }
        mbar_init(su32(mmadone), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kWarpMma) {
        // one warp of each CTA of the pair allocates, collectively
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    fence_before();
    __syncwarp();
    cluster_sync();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t pair_id = blockIdx.x >> 1, npairs = gridDim.x >> 1;

    if (warp == kWarpTma) {
        // ---------------------------------------------------------- TMA producer (each CTA its own slabs)
        if (lane == 0) {
            Ring xr(NX);
            bool ok = true;
            for (int64_t w = pair_id; w < P.units && ok; w += npairs) {
                Unit u;
                get_unit(P, w, u);
                for (int64_t st = 0; st < u.nst; ++st, xr.next()) {
                    if (!(ok = wait_bar(su32(&xempty[xr.slot]), xr.phase ^ 1u, abort_flag, P.status))) break;
                    mbar_expect_tx(su32(&xfull[xr.slot]), (uint32_t)P.box_bytes);
                    tma_load_2d(su32(slab + xr.slot * P.box_bytes), &tmap, (int)(u.k0 + st * kStage), 0,
                                su32(&xfull[xr.slot]));
                }
            }
        }
    } else if (warp == kWarpMma) {
        // ---------------------------------------------------------- MMA issuer (even CTA)
        // Per stage, quarter by quarter: wait for the quarter's drain of the
        // previous stage, then 8 MMAs (lo*lo, hi*lo, lo*hi, hi*hi over two K
        // steps) and a commit; the drain of quarter q overlaps the MMAs of the
        // other three.
        if (cta == 0 && lane == 0) {
            const uint32_t sbase = su32(slots);
            const uint64_t ah0 = smem_desc64(sbase), al0 = smem_desc64(sbase + kPartBytes);
            const uint64_t bh0 = smem_desc64(sbase + 2 * kPartBytes), bl0 = smem_desc64(sbase + 3 * kPartBytes);
            Ring orr(NS);
            uint64_t g = 0;
            bool ok = true;
            for (int64_t w = pair_id; w < P.units && ok; w += npairs) {
                Unit u;
                get_unit(P, w, u);
                for (int64_t st = 0; st < u.nst; ++st, ++g, orr.next()) {
                    if (!(ok = wait_cluster(su32(&opfull[orr.slot]), orr.phase, abort_flag, P.status))) break;
                    const uint64_t so = (uint64_t)orr.slot * (kSlotBytes >> 4);
#pragma unroll
                    for (int q = 0; q < kQuarters; ++q) {
                        if (g > 0 && !(ok = wait_cluster(su32(&accempty[q]), (uint32_t)((g - 1) & 1), abort_flag,
                                                         P.status)))
                            break;
                        fence_after();
                        const uint32_t d = tmem + (uint32_t)(q * kQN);
                        const uint64_t bo = (uint64_t)q * ((kQB * kRowBytes) >> 4);   // this quarter's B rows
                        const uint64_t ah = ah0 + so, al = al0 + so, bh = bh0 + so + bo, bl = bl0 + so + bo;
                        mma_pair(d, al, bl, IDESC, 0u);
                        mma_pair(d, al + 2, bl + 2, IDESC, 1u);
                        mma_pair(d, ah, bl, IDESC, 1u);
                        mma_pair(d, ah + 2, bl + 2, IDESC, 1u);
                        mma_pair(d, al, bh, IDESC, 1u);
                        mma_pair(d, al + 2, bh + 2, IDESC, 1u);
                        mma_pair(d, ah, bh, IDESC, 1u);
                        mma_pair(d, ah + 2, bh + 2, IDESC, 1u);
                        commit_both(su32(&accfull[q]));
                    }
                    if (!ok) break;
                    commit_both(su32(&opempty[orr.slot]));
                }
            }
            // every MMA issued above has completed before the pair tears down
            commit_both(su32(mmadone));
            wait_bar(su32(mmadone), 0u, abort_flag, P.status);
        }
    } else if (warp < kWarpD0) {
        // ---------------------------------------------------------- builders: one Khatri-Rao row each
        const int r = (warp - kWarpB0) * 32 + lane;   // A rows 0..127, B rows 128..255
        const bool isA = r < kRows;
        const int prow = isA ? r : r - kRows;          // row within the part
        const uint32_t part_hi = (uint32_t)(isA ? 0 : 2 * kPartBytes);
        Ring orr(NS), xr(NX);
        bool ok = true;
        for (int64_t w = pair_id; w < P.units && ok; w += npairs) {
            Unit u;
            get_unit(P, w, u);
            const Shape& sh = P.sh;
            KrRow<DA> kra;
            KrRow<DB> krb;
            if (isA) {
                const int64_t p = u.I * kTileM + (int64_t)cta * kRows + prow;
                int col[DA];
                if (p < sh.rows) {
                    const RowInfo ri = decode_row(p, DA, DB, sh.b, sh.nbar, sh.bdA, sh.bdB, sh.bd);
#pragma unroll
                    for (int f = 0; f < DA; ++f) col[f] = ri.col[f];
                } else {
#pragma unroll
                    for (int f = 0; f < DA; ++f) col[f] = 0;
                }
                kra.set(col);
            } else {
                // B row prow of this CTA: quarter prow / 32, the CTA's 32 of its 64 columns
                const int64_t q = u.J * kTileN + (int64_t)(prow >> 5) * kQN + (int64_t)cta * kQB + (prow & 31);
                int col[DB];
                if (q < sh.cols) {
                    const ColInfo ci = decode_col(q, DA, DB, sh.b, sh.nbar, sh.bdB, sh.bd);
#pragma unroll
                    for (int f = 0; f < DB; ++f) col[f] = ci.col[f];
                } else {
#pragma unroll
                    for (int f = 0; f < DB; ++f) col[f] = 0;
                }
                krb.set(col);
            }
            for (int64_t st = 0; st < u.nst; ++st, orr.next(), xr.next()) {
                bool okw = wait_bar(su32(&xfull[xr.slot]), xr.phase, abort_flag, P.status) &&
                           wait_bar(su32(&opempty[orr.slot]), orr.phase ^ 1u, abort_flag, P.status);
                okw = __all_sync(0xffffffffu, okw);
                if (!okw) {
                    // leave together with the other builders (see named_sync_any)
                    named_sync_any(1, kBuildWarps * 32, true);
                    ok = false;
                    break;
                }
                const uint32_t s32 = su32(slab) + (uint32_t)(xr.slot * P.box_bytes);
                const uint32_t hi_base = su32(slots) + (uint32_t)(orr.slot * kSlotBytes) + part_hi;
                const uint32_t lo_base = hi_base + kPartBytes;
                if (isA) {
                    uint32_t a[DA];
                    kra.addresses(s32, a);
#pragma unroll
                    for (int cb = 0; cb < 4; ++cb) {
                        uint32_t h[4], l[4];
                        build_chunk<KIND, DA>(a, cb, h, l);
                        const uint32_t off = sw64(prow, cb);
                        sts128(hi_base + off, h[0], h[1], h[2], h[3]);
                        sts128(lo_base + off, l[0], l[1], l[2], l[3]);
                    }
                } else {
                    uint32_t a[DB];
                    krb.addresses(s32, a);
#pragma unroll
                    for (int cb = 0; cb < 4; ++cb) {
                        uint32_t h[4], l[4];
                        build_chunk<KIND, DB>(a, cb, h, l);
                        const uint32_t off = sw64(prow, cb);
                        sts128(hi_base + off, h[0], h[1], h[2], h[3]);
                        sts128(lo_base + off, l[0], l[1], l[2], l[3]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (named_sync_any(1, kBuildWarps * 32, false)) {
                    ok = false;
                    break;
                }
                if (warp == kWarpB0 && lane == 0) {
                    mbar_arrive(su32(&xempty[xr.slot]));
                    mbar_arrive_remote(su32(&opfull[orr.slot]), 0u);
                }
            }
        }
    } else {
        // ---------------------------------------------------------- drainers: running sums, folds, write-out
        const int di = warp - kWarpD0;                 // 0..7
        const int q4 = warp & 3, dh = di >> 2;         // lane quarter; which 32 of each quarter's 64 columns
        const int drow = q4 * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
        const uint32_t tD = tmem + lane_off + (uint32_t)(dh * kDrainCols);
        const uint32_t tRun = tmem + lane_off + (uint32_t)(kSumBase + dh * kDrainCols);
        double* scr = P.scratch + (size_t)blockIdx.x * kRows * kTileN + drow;   // column c at scr[c * kRows]
        {
            const uint32_t z[32] = {};
#pragma unroll
            for (int q = 0; q < kQuarters; ++q) tmem_st32(tRun + q * kQN, z);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        // running sum of quarter q -> FP64 scratch: the unit's first fold
        // stores, later ones add with fire-and-forget reductions (each scratch
        // element belongs to this thread, so the order is fixed and its later
        // loads see them); the running sum restarts from zero
        auto fold = [&](int q, bool first) {
            uint32_t v[32];
            tmem_ld32_nowait(tRun + q * kQN, v);
            tmem_wait_ld();
            const uint32_t z[32] = {};
            tmem_st32(tRun + q * kQN, z);
            double* x0 = scr + (size_t)(q * kQN + dh * kDrainCols) * kRows;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                double* x = x0 + (size_t)j * kRows;
                const double f = (double)__uint_as_float(v[j]);
                if (first)
                    *x = f;
                else
                    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(x), "d"(f) : "memory");
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        };
        uint64_t g = 0;
        bool ok = true;
        for (int64_t w = pair_id; w < P.units && ok; w += npairs) {
            Unit u;
            get_unit(P, w, u);
            const int64_t nst = u.nst;
            for (int64_t k = 0; k < nst && ok; ++k, ++g) {
#pragma unroll 1
                for (int q = 0; q < kQuarters; ++q) {
                    // the running sum does not depend on the MMA: its load is in
                    // flight while this quarter's accumulator completes
                    uint32_t v[32], sm[32];
                    tmem_ld32_nowait(tRun + q * kQN, sm);
                    const bool okw = __all_sync(0xffffffffu, wait_bar(su32(&accfull[q]), (uint32_t)(g & 1),
                                                                      abort_flag, P.status));
                    if (!okw) {
                        tmem_wait_ld();
                        ok = false;
                        break;
                    }
                    fence_after();
                    tmem_ld32_nowait(tD + q * kQN, v);
                    tmem_wait_ld();
                    // scalar adds: the loaded registers need not form aligned pairs
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = __float_as_uint(__fadd_rn(__uint_as_float(sm[j]), __uint_as_float(v[j])));
                    // the store to the running sum needs no wait here: the MMAs
                    // write only the accumulator, and this thread waits for its
                    // stores once per stage, before it reads the sums again
                    tmem_st32(tRun + q * kQN, v);
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive_remote_relaxed(su32(&accempty[q]), 0u);
                    // quarter q folds after the stages k = 32 q + 31 (mod 128)
                    if ((k & (kFoldEvery - 1)) == 32 * q + 31 && k + 1 < nst) {
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        fold(q, k < kFoldEvery);
                    }
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            if (!ok) break;
#pragma unroll 1
            for (int q = 0; q < kQuarters; ++q) fold(q, 32 * q + 31 >= nst - 1);
#pragma unroll 1
            for (int q = 0; q < kQuarters; ++q)
                write_segment<KIND, DA, DB>(P, u, u.I * kTileM + (int64_t)cta * kRows + drow,
                                            u.J * kTileN + (int64_t)q * kQN + dh * kDrainCols, kDrainCols,
                                            scr + (size_t)(q * kQN + dh * kDrainCols) * kRows);
        }
    }

    fence_before();
    __syncwarp();
    cluster_sync();
    if (warp == kWarpMma) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// ------------------------------------------------------------------ host

static size_t smem_bytes(int nslots, int nslabs, int box_bytes)
{
    return 1024 + (size_t)nslots * kSlotBytes + (size_t)nslabs * box_bytes +
           8 * (2 * kMaxSlabs + 2 * kMaxSlots + 2 * kQuarters + 1) + 16;
}

template <int KIND, int DA, int DB>
static cudaError_t launch_typed(const CUtensorMap& map, const Params& P, size_t smem, cudaStream_t st)
{
    auto kern = moment_pair_kernel<KIND, DA, DB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(sms / 2 * 2), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, (void*)kern, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    int64_t pairs = P.units < clusters ? P.units : clusters;
    if (pairs > kTcMaxCtas / 2) pairs = kTcMaxCtas / 2;
    kern<<<(unsigned)(2 * pairs), kThreads, smem, st>>>(map, P);
    return cudaGetLastError();
}

template <int KIND>
static cudaError_t launch_kind(const CUtensorMap& map, const Params& P, size_t smem, cudaStream_t st)
{
    const int dA = P.sh.dA, dB = P.sh.dB;
    if (dA == 1 && dB == 1) return launch_typed<KIND, 1, 1>(map, P, smem, st);
    if (dA == 2 && dB == 1) return launch_typed<KIND, 2, 1>(map, P, smem, st);
    if (dA == 2 && dB == 2) return launch_typed<KIND, 2, 2>(map, P, smem, st);
    if (dA == 3 && dB == 2) return launch_typed<KIND, 3, 2>(map, P, smem, st);
    if (dA == 3 && dB == 3) return launch_typed<KIND, 3, 3>(map, P, smem, st);
    return cudaErrorInvalidValue;
}

}  // namespace pair

cudaError_t launch_moment_pair(const OrderPlan& OP, int prec, const float* xt, int64_t t_pad, const int64_t* prefix,
                               double* out, double scale, double* scratch, int* status, const int* vexp,
                               cudaStream_t st)
{
    using namespace pair;
    if (OP.units <= 0) return cudaSuccess;
    if (prec != CUM_PREC_FP16X3 && prec != CUM_PREC_BF16X3) return cudaErrorInvalidValue;
    if (prec == CUM_PREC_FP16X3 && !vexp) return cudaErrorInvalidValue;
    if (OP.tile_m != kTileM || OP.tile_n != kTileN) return cudaErrorInvalidValue;
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
    P.vexp = vexp;
    P.box_bytes = tc_box_rows(OP.sh.n_pad) * 128;
    if (OP.kchunk % kStage || t_pad % kStage) return cudaErrorInvalidValue;
    int dev = 0, maxsmem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    int ns = kMaxSlots, nx = kMaxSlabs;
    while (nx > 2 && smem_bytes(ns, nx, P.box_bytes) > (size_t)maxsmem) --nx;
    while (ns > 2 && smem_bytes(ns, nx, P.box_bytes) > (size_t)maxsmem) --ns;
    if (smem_bytes(ns, nx, P.box_bytes) > (size_t)maxsmem) return cudaErrorInvalidValue;
    P.nslots = ns;
    P.nslabs = nx;
    CUtensorMap map;
    if (!encode_xt_map(&map, xt, t_pad, OP.sh.n_pad)) return cudaErrorInvalidValue;
    const size_t smem = smem_bytes(ns, nx, P.box_bytes);
    if (prec == CUM_PREC_FP16X3) return launch_kind<2>(map, P, smem, st);
    return launch_kind<0>(map, P, smem, st);
}

}  // namespace cum
