// Tensor-core moment contraction on CTA pairs (tcgen05 cta_group::2) for the
// fp16 and bf16 split precisions.
//
// Computes, for one order d, the block-stored sums
//   M[rowOff(p) + colOff(q)] = scale * sum_l ZA[l, p] * ZB[l, q]      (Alg. 1-2)
// over the valid pairs last(p) <= first(q), like moment_tc.cu, on output tiles
// of 256 x 128 per pair of CTAs (a cluster of two, one per SM of a TPC):
//  * one builder thread of each CTA TMA-loads its X~ slabs (32 fp32 samples
//    of every variable, 128-byte swizzle), NX stages ahead;
//  * 6 builder warps of CTA c build, per stage of 32 samples, the Khatri-Rao
//    rows p = 256 I + 128 c + (0..127) of A and the B rows
//    q = 128 J + 64 c + (0..63), as fp16/bf16 hi and lo parts: A into the
//    CTA's tensor memory (row = lane, tcgen05.st), B into shared memory
//    (K-major, 64-byte swizzle);
//  * two threads of the even CTA, on alternate stages, issue 8 MMAs of M = 256 (128
//    A rows from each CTA's tensor memory), N = 128 (64 B rows from each
//    CTA's shared memory), K = 16: lo*lo, hi*lo, lo*hi, then hi*hi, over the
//    stage's two K steps, into one of three FP32 accumulator buffers in each
//    CTA's tensor memory.  Each accumulator therefore restarts every 32
//    samples: the tensor core's truncating additions act on chains of two K
//    steps only, and the lo*lo term removes the bias of the dropped product
//    on entries of a column with itself;
//  * 8 drainer warps add each stage's accumulator, while the MMAs of the next
//    stages fill the other buffers, into FP32 running sums held in registers
//    (tensor memory is read once per element and stage), fold them into an
//    FP64 scratch tile every 4096 samples, and write the valid entries of
//    their tile rows to block storage while the builders start the next unit.
// Per stage a CTA builds 192 Khatri-Rao rows for 128 x 128 outputs (the
// one-CTA kernel builds 256).
// All waits are bounded: on expiry the kernel records CUM_ETIMEOUT in the
// workspace status word and every role leaves its loop.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <type_traits>

#include "cumgb.h"
#include "internal.h"
#include "tc_ptx.cuh"

namespace cum {
namespace pair {
using namespace tc;

constexpr int kWarpMma0 = 0, kWarpMma = 1, kWarpB0 = 2, kWarpBB0 = 6, kWarpD0 = 8;   // A builders 2-5, B 6-7
constexpr int kBuildWarps = 6, kDrainWarps = 8;
constexpr int kThreads = (kWarpD0 + kDrainWarps) * 32;    // 512: 16 warps, 128 registers each
constexpr int kTileM = kPairTileM, kTileN = kPairTileN;   // 256 x 128 per pair
constexpr int kRows = 128;                  // A rows (tensor-memory lanes) per CTA
constexpr int kBRows = kTileN / 2;          // B rows per CTA (its half of N)
constexpr int kStage = 32;                  // samples per stage
constexpr int kRowBytes = 64;               // 32 fp16 / bf16 samples
constexpr int kBPartBytes = kBRows * kRowBytes;   // one part (hi or lo) of B
constexpr int kSlotBytes = 2 * kBPartBytes;       // B hi, B lo (A lives in tensor memory)
// Tensor memory: 3 accumulator buffers of 128 columns, then 4 A stages of 32
// columns (hi 16 + lo 16: 32 fp16 samples per row).  The tensor core reads its
// shared-memory operands at about 64 bytes per cycle, which B alone fills at
// the MMA rate; A read from shared memory as well halved the MMA rate.
constexpr int kAccBufs = 3;
constexpr int kAStageCols = 32;
constexpr int kABase = kAccBufs * kTileN;
constexpr int kTmemCols = 512;
constexpr int kFoldEvery = 128;             // stages between FP64 folds (4096 samples)
constexpr int kMaxSlots = 4, kMaxSlabs = 8;   // operand stages: A in tensor memory, B in shared memory
static_assert(kABase + kMaxSlots * kAStageCols == kTmemCols, "tensor memory map");
constexpr int kDrainCols = 64;              // accumulator columns a drainer thread owns

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
    double* scratch;         // per CTA: 128 columns x 128 rows of FP64
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

// Arrive on the mbarrier at local address `bar` of CTA `cta` of the cluster,
// with the default semantics (release at CTA scope).  The builders' operand
// stores are made visible to the tensor core by fence.proxy.async before the
// arrive; a cluster-scope release on top of that measured about 900 cycles per
// stage, most of the stage.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t bar, uint32_t cta)
{
    asm volatile(
        "{\n .reg .b32 ra;\n mapa.shared::cluster.u32 ra, %0, %1;\n"
        " mbarrier.arrive.shared::cluster.b64 _, [ra];\n}\n" ::"r"(bar),
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

// test_wait (never suspends), default semantics (acquire at CTA scope): the
// waits of the MMA thread, whose consumers are the tensor core's operand reads
// (made visible by the producers' proxy fences) and accumulator writes
__device__ __forceinline__ bool mbar_test_cluster(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait that polls without suspending (the same limit and abort
// handling as wait_cluster).
__device__ __forceinline__ bool wait_cluster_spin(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status)
{
    if (mbar_test_cluster(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t i = 1;; ++i) {
        if (mbar_test_cluster(bar, parity)) return true;
        if ((i & 255u) == 0u) {
            if (*abort_flag) return false;
            if (clock64() - t0 > kWaitLimit) {
                *abort_flag = 1;
                atomicExch(status, CUM_ETIMEOUT);
                return false;
            }
        }
    }
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
// (fmt 1), both K-major, M = 256 (the pair), N = 128.
__host__ __device__ constexpr uint32_t idesc_pair(uint32_t fmt)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

// 32 accumulator columns of this warp's lanes, waited for and returned as 16
// packed pairs (column 2i in the low half), ready for packed FP32 adds.
__device__ __forceinline__ void tmem_ld32_pairs(uint32_t taddr, uint64_t* p)
{
    asm volatile(
        "{\n .reg .b32 r<32>;\n"
        " tcgen05.ld.sync.aligned.32x32b.x32.b32 {r0, r1, r2, r3, r4, r5, r6, r7, r8, r9, r10, r11, r12, r13, r14, "
        "r15, r16, r17, r18, r19, r20, r21, r22, r23, r24, r25, r26, r27, r28, r29, r30, r31}, [%16];\n"
        " tcgen05.wait::ld.sync.aligned;\n"
        " mov.b64 %0, {r0, r1};\n mov.b64 %1, {r2, r3};\n mov.b64 %2, {r4, r5};\n mov.b64 %3, {r6, r7};\n"
        " mov.b64 %4, {r8, r9};\n mov.b64 %5, {r10, r11};\n mov.b64 %6, {r12, r13};\n mov.b64 %7, {r14, r15};\n"
        " mov.b64 %8, {r16, r17};\n mov.b64 %9, {r18, r19};\n mov.b64 %10, {r20, r21};\n mov.b64 %11, {r22, r23};\n"
        " mov.b64 %12, {r24, r25};\n mov.b64 %13, {r26, r27};\n mov.b64 %14, {r28, r29};\n mov.b64 %15, {r30, r31};\n"
        "}\n"
        : "=l"(p[0]), "=l"(p[1]), "=l"(p[2]), "=l"(p[3]), "=l"(p[4]), "=l"(p[5]), "=l"(p[6]), "=l"(p[7]),
          "=l"(p[8]), "=l"(p[9]), "=l"(p[10]), "=l"(p[11]), "=l"(p[12]), "=l"(p[13]), "=l"(p[14]), "=l"(p[15])
        : "r"(taddr)
        : "memory");
}

// a + b on packed FP32 pairs, round to nearest
__device__ __forceinline__ uint64_t add_pair(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// A from tensor memory (each CTA's 128 rows in its own lanes), B from shared memory.
__device__ __forceinline__ void mma_pair(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
            d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(acc));
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

// Lane 0's result of a barrier wait, given to the whole warp.  Only lane 0
// polls the mbarrier (32 lanes polling one barrier cost the builders and
// drainers several hundred cycles a stage); __syncwarp then orders the other
// lanes' later accesses after lane 0's acquire.
__device__ __forceinline__ bool warp_agree(bool ok)
{
    const bool r = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    __syncwarp();
    return r;
}

// Byte offset of 16-byte chunk `ch` (0..3) of row `r` in a 64-byte-swizzled
// part (the part base is 1024-byte aligned): address bits 4-5 are XORed with
// bits 7-8.
__device__ __forceinline__ uint32_t sw64(int r, int ch) { return (uint32_t)(r * kRowBytes + ((ch ^ ((r >> 1) & 3)) << 4)); }

// ------------------------------------------------------------------ work units

struct Unit {
    int s;              // t chunk
    int64_t I, J;       // 256-row tile, 128-column tile
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

// The sample coordinate of each stage of the pair's units, in order: unit
// w = pair_id, pair_id + npairs, ..., stages 0 .. nst-1 of each.
struct StageIter {
    int64_t w;
    int st, nst, k;     // stage in the unit, its stages, its first sample (t_pad < 2^31)
    bool have;
    __device__ __forceinline__ StageIter(const Params& P, int64_t pair_id, int64_t npairs)
        : w(pair_id - npairs), st(0), nst(0), k(0), have(true)
    {
        unit(P, npairs);
    }
    __device__ __forceinline__ void unit(const Params& P, int64_t npairs)
    {
        do {
            w += npairs;
            have = w < P.units;
            if (!have) return;
            Unit u;
            get_unit(P, w, u);
            nst = (int)u.nst;
            k = (int)u.k0;
        } while (nst <= 0);
        st = 0;
    }
    __device__ __forceinline__ void next(const Params& P, int64_t npairs)
    {
        if (++st < nst) k += kStage;
        else unit(P, npairs);
    }
};

// Wait for phase `parity` of the mbarrier at `bar` with a time limit only (no
// early exit on the abort flag): for the copies and MMAs a CTA must see land
// before it releases shared and tensor memory.  On expiry the status word
// records CUM_ETIMEOUT.
__device__ __forceinline__ void wait_bar_bounded(uint32_t bar, uint32_t parity, int* status)
{
    if (mbar_try(bar, parity)) return;
    const long long t0 = clock64();
    while (!mbar_try_sleep(bar, parity, 20000u)) {
        if (clock64() - t0 > kWaitLimit) {
            atomicExch(status, CUM_ETIMEOUT);
            return;
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
    uint8_t* slots = smem;                                   // NS x (B hi, B lo)
    uint8_t* slab = slots + NS * kSlotBytes;                 // NX x one X~ box
    uint64_t* bars = (uint64_t*)(slab + NX * P.box_bytes);
    uint64_t* xfull = bars;
    uint64_t* opfull = xfull + kMaxSlabs;        // used in the even CTA: one arrival per CTA
    uint64_t* opempty = opfull + kMaxSlots;      // completed by the MMA commits, in both CTAs
    uint64_t* accfull = opempty + kMaxSlots;     // per accumulator buffer, in both CTAs
    uint64_t* accempty = accfull + kAccBufs;     // per buffer, in the even CTA: both CTAs' drainers arrive
    uint64_t* mmadone = accempty + kAccBufs;     // one per MMA issuer
    uint32_t* tmem_slot = (uint32_t*)(mmadone + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const uint32_t cta = cta_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        // the builders gather on a named barrier and one thread arrives for
        // the CTA (one cluster-scope release per CTA and stage); each drainer
        // warp arrives for itself (a relaxed arrive: tensor memory only)
        for (int i = 0; i < NX; ++i) mbar_init(su32(&xfull[i]), 1);
        for (int i = 0; i < NS; ++i) {
            mbar_init(su32(&opfull[i]), 2);
            mbar_init(su32(&opempty[i]), 1);
        }
        for (int i = 0; i < kAccBufs; ++i) {
            mbar_init(su32(&accfull[i]), 1);
            mbar_init(su32(&accempty[i]), 2 * kDrainWarps);
        }
        mbar_init(su32(&mmadone[0]), 1);
        mbar_init(su32(&mmadone[1]), 1);
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

    if (warp == kWarpMma0 || warp == kWarpMma) {
        // ---------------------------------------------------------- MMA issuers (even CTA)
        // Stage g accumulates into accumulator buffer g mod 3: 8 MMAs (lo*lo,
        // hi*lo, lo*hi, hi*hi over two K steps; A from tensor memory, B from
        // shared memory) once the stage's operands are built and the buffer's
        // previous stage is drained.  Two threads in two warps take alternate
        // stages: an mbarrier wait issued behind a thread's own MMAs returns only
        // after they have been taken by the tensor core, so one issuing thread
        // left the pipe idle for about 280 cycles of each 512-cycle stage; with
        // two, one waits while the other's MMAs run.  The parity waits stay
        // exact: builders and drainers finish stages in order, and each thread
        // has seen stage g - 2 complete before it waits for stage g.
        if (cta == 0 && lane == 0) {
            const int mine = warp == kWarpMma ? 0 : 1;
            const uint64_t bh0 = smem_desc64(su32(slots)), bl0 = smem_desc64(su32(slots) + kBPartBytes);
            Ring orr(NS), dr(kAccBufs);
            int64_t g = 0;
            bool ok = true;
            for (int64_t w = pair_id; w < P.units && ok; w += npairs) {
                Unit u;
                get_unit(P, w, u);
                for (int64_t st = 0; st < u.nst; ++st, ++g, orr.next(), dr.next()) {
                    if ((int)(g & 1) != mine) continue;
                    ok = wait_cluster(su32(&opfull[orr.slot]), orr.phase, abort_flag, P.status) &&
                         wait_cluster(su32(&accempty[dr.slot]), dr.phase ^ 1u, abort_flag, P.status);
                    if (!ok) break;
                    fence_after();
                    const uint32_t d = tmem + (uint32_t)(dr.slot * kTileN);
                    const uint32_t ah = tmem + (uint32_t)(kABase + orr.slot * kAStageCols), al = ah + 16u;
                    const uint64_t so = (uint64_t)orr.slot * (kSlotBytes >> 4);
                    const uint64_t bh = bh0 + so, bl = bl0 + so;
                    mma_pair(d, al, bl, IDESC, 0u);
                    mma_pair(d, al + 8, bl + 2, IDESC, 1u);
                    mma_pair(d, ah, bl, IDESC, 1u);
                    mma_pair(d, ah + 8, bl + 2, IDESC, 1u);
                    mma_pair(d, al, bh, IDESC, 1u);
                    mma_pair(d, al + 8, bh + 2, IDESC, 1u);
                    mma_pair(d, ah, bh, IDESC, 1u);
                    mma_pair(d, ah + 8, bh + 2, IDESC, 1u);
                    commit_both(su32(&accfull[dr.slot]));
                    commit_both(su32(&opempty[orr.slot]));
                }
            }
            // every MMA this thread issued has completed before the pair tears down
            commit_both(su32(&mmadone[mine]));
            wait_bar_bounded(su32(&mmadone[mine]), 0u, P.status);
        }
    } else if (warp < kWarpD0) {
        // ---------------------------------------------------------- builders: one Khatri-Rao row each
        // A rows: row = tensor-memory lane, so warp w builds the rows of lane
        // quarter w mod 4 and stores them with tcgen05.st; B rows: 64 per CTA
        // into the shared-memory slot.  One builder thread also issues the
        // CTA's X~ loads: the load of stage g + NX goes into stage g's slab
        // once the builders' barrier of stage g has passed (every read of the
        // slab is done by then).
        const bool isA = warp < kWarpBB0;
        const bool loader = warp == kWarpB0 && lane == 0;
        const int prow = isA ? (warp & 3) * 32 + lane : (warp - kWarpBB0) * 32 + lane;
        const uint32_t a_lane = (uint32_t)((warp & 3) * 32) << 16;
        StageIter ld(P, pair_id, npairs);
        int64_t issued = 0, g = 0;
        if (loader) {
            for (int i = 0; i < NX && ld.have; ++i, ++issued, ld.next(P, npairs)) {
                mbar_expect_tx(su32(&xfull[i]), (uint32_t)P.box_bytes);
                tma_load_2d(su32(slab + i * P.box_bytes), &tmap, (int)ld.k, 0, su32(&xfull[i]));
            }
        }
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
                // B row prow of CTA c: tile column 64 c + prow (the MMA takes CTA 0's rows first)
                const int64_t q = u.J * kTileN + (int64_t)cta * kBRows + prow;
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
            for (int64_t st = 0; st < u.nst; ++st, ++g, orr.next(), xr.next()) {
                bool okw = true;
                if (lane == 0)
                    okw = wait_bar(su32(&xfull[xr.slot]), xr.phase, abort_flag, P.status) &&
                          wait_bar(su32(&opempty[orr.slot]), orr.phase ^ 1u, abort_flag, P.status);
                okw = warp_agree(okw);
                if (!okw) {
                    // leave together with the other builders (see named_sync_any)
                    named_sync_any(1, kBuildWarps * 32, true);
                    ok = false;
                    break;
                }
                const uint32_t s32 = su32(slab) + (uint32_t)(xr.slot * P.box_bytes);
                if (isA) {
                    fence_after();   // the MMAs that read this A stage before (opempty) have completed
                    uint32_t a[DA];
                    kra.addresses(s32, a);
                    uint32_t h[16], l[16];
#pragma unroll
                    for (int cb = 0; cb < 4; ++cb) build_chunk<KIND, DA>(a, cb, h + 4 * cb, l + 4 * cb);
                    const uint32_t ta = tmem + a_lane + (uint32_t)(kABase + orr.slot * kAStageCols);
                    tmem_st16(ta, h);
                    tmem_st16(ta + 16, l);
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    fence_before();
                } else {
                    const uint32_t hi_base = su32(slots) + (uint32_t)(orr.slot * kSlotBytes);
                    const uint32_t lo_base = hi_base + kBPartBytes;
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
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                }
                if (named_sync_any(1, kBuildWarps * 32, false)) {
                    ok = false;
                    break;
                }
                if (loader) {
                    mbar_arrive_remote(su32(&opfull[orr.slot]), 0u);
                    if (ld.have) {
                        mbar_expect_tx(su32(&xfull[xr.slot]), (uint32_t)P.box_bytes);
                        tma_load_2d(su32(slab + xr.slot * P.box_bytes), &tmap, (int)ld.k, 0, su32(&xfull[xr.slot]));
                        ++issued;
                        ld.next(P, npairs);
                    }
                }
            }
        }
        // loads still in flight after an early exit land before the CTA leaves
        if (loader)
            for (int64_t i = g; i < issued; ++i)
                wait_bar_bounded(su32(&xfull[i % NX]), (uint32_t)((i / NX) & 1), P.status);
    } else {
        // ---------------------------------------------------------- drainers: register running sums
        // Each thread owns 64 accumulator columns of one tile row (its lane):
        // per stage it adds them to FP32 running sums held in registers as
        // packed pairs, folds 16-column groups into the FP64 scratch tile at
        // staggered stages, and at the end of a unit writes its row segment.
        const int di = warp - kWarpD0;                 // 0..7
        const int q4 = warp & 3, dh = di >> 2;         // lane quarter; which 64 of the 128 columns
        const int drow = q4 * 32 + lane;
        const uint32_t tD = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(dh * kDrainCols);
        double* scr = P.scratch + (size_t)blockIdx.x * kRows * kTileN + (size_t)(dh * kDrainCols) * kRows + drow;
        uint64_t run[kDrainCols / 2];
#pragma unroll
        for (int j = 0; j < kDrainCols / 2; ++j) run[j] = 0ull;
        // running sums of 16-column group c -> FP64 scratch: the unit's first
        // fold stores, later ones add with fire-and-forget reductions (each
        // scratch element belongs to this thread, so the order is fixed and
        // its later loads see them); the group restarts from zero
        // (c is compared against unrolled constants so that run[] stays in registers)
        auto fold_group = [&](auto cc, bool first) {
            constexpr int c = decltype(cc)::value;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint64_t pr = run[8 * c + j];
                const double f0 = (double)__uint_as_float((uint32_t)pr);
                const double f1 = (double)__uint_as_float((uint32_t)(pr >> 32));
                double* x = scr + (size_t)(16 * c + 2 * j) * kRows;
                if (first) {
                    x[0] = f0;
                    x[kRows] = f1;
                } else {
                    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(x), "d"(f0) : "memory");
                    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(x + kRows), "d"(f1) : "memory");
                }
                run[8 * c + j] = 0ull;
            }
        };
        auto fold = [&](int c, bool first) {
            if (c == 0) fold_group(std::integral_constant<int, 0>{}, first);
            else if (c == 1) fold_group(std::integral_constant<int, 1>{}, first);
            else if (c == 2) fold_group(std::integral_constant<int, 2>{}, first);
            else fold_group(std::integral_constant<int, 3>{}, first);
        };
        Ring dr(kAccBufs);
        bool ok = true;
        for (int64_t w = pair_id; w < P.units && ok; w += npairs) {
            Unit u;
            get_unit(P, w, u);
            const int64_t nst = u.nst;
            for (int64_t k = 0; k < nst; ++k, dr.next()) {
                const int buf = dr.slot;
                bool okw = true;
                if (lane == 0) okw = wait_bar(su32(&accfull[buf]), dr.phase, abort_flag, P.status);
                if (!(ok = warp_agree(okw)))
                    break;
                fence_after();
                const uint32_t t0 = tD + (uint32_t)(buf * kTileN);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint64_t v[16];
                    tmem_ld32_pairs(t0 + 32 * h, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) run[16 * h + j] = add_pair(run[16 * h + j], v[j]);
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_remote_relaxed(su32(&accempty[buf]), 0u);
                // group c folds after the stages k = 32 c + 31 (mod 128)
                const int kp = (int)(k & (kFoldEvery - 1));
                if ((kp & 31) == 31 && k + 1 < nst) fold(kp >> 5, k < kFoldEvery);
            }
            if (!ok) break;
#pragma unroll
            for (int c = 0; c < kDrainCols / 16; ++c) fold(c, 32 * c + 31 >= nst - 1);
            write_segment<KIND, DA, DB>(P, u, u.I * kTileM + (int64_t)cta * kRows + drow,
                                        u.J * kTileN + (int64_t)dh * kDrainCols, kDrainCols, scr);
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
           8 * (kMaxSlabs + 2 * kMaxSlots + 2 * kAccBufs + 2) + 16;
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
