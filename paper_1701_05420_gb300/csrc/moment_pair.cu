// Tensor-core moment contraction on CTA pairs (tcgen05 cta_group::2) for the
// fp16 and bf16 split precisions.
//
// Computes, for one order d, the block-stored sums
//   M[rowOff(p) + colOff(q)] = scale * sum_l ZA[l, p] * ZB[l, q]      (Alg. 1-2)
// over the valid pairs last(p) <= first(q), like moment_tc.cu, on output tiles
// of 256 x 128 per pair of CTAs (a cluster of two, one per SM of a TPC):
//  * one thread of each CTA TMA-loads its X~ slabs (32 fp32 samples of every
//    variable, 128-byte swizzle);
//  * 12 builder warps of CTA c build, per stage of 32 samples, the Khatri-Rao
//    rows p = 256 I + 128 c + (0..127) of A and the B rows
//    q = 128 J + 64 c + (0..63), as fp16/bf16 hi and lo parts: A into the
//    CTA's tensor memory (row = lane, tcgen05.st), B into shared memory
//    (K-major, 64-byte swizzle).  With two parts each warp builds whole rows
//    of every other stage (six warps a stage); with three, each thread builds
//    16 samples of one row in every stage;
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
// one-CTA kernel builds 256).  The builders are latency-bound: 12 warps, with
// registers moved to the drainers by setmaxnreg, keep more of their work in
// flight than 6 warps of whole rows of every stage, and taking alternate
// stages halves each warp's barrier waits and arrivals per sample.
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

// Warp roles, by warpgroup: 0 = MMA issuers (warps 0, 1 of the even CTA) and
// the X~ loader (warp 2); 1-3 = builders (A: warps 4-11, B: warps 12-15; each
// thread whole Khatri-Rao rows of alternate stages, or half rows of every
// stage); 4-5 = drainers (warps 16-23).
constexpr int kWarpMma0 = 0, kWarpMma = 1, kWarpTma = 2;
constexpr int kWarpA0 = 4, kAWarps = 8, kBWarps = 4;   // B builders: warps 12-15
constexpr int kBuildWarps = kAWarps + kBWarps;
constexpr int kWarpD0 = 16, kDrainWarps = 8;
constexpr int kThreads = (kWarpD0 + kDrainWarps) * 32;    // 768
// Registers: 80 a thread at launch (65536 / 768, in multiples of 8), then
// moved by setmaxnreg from the control and builder warpgroups to the drainers,
// whose running sums take 64 registers.  The shares must not exceed the
// launch's total, or setmaxnreg.inc would wait forever.
constexpr int kLaunchRegs = 80, kRegsCtl = 48, kRegsBuild = 72, kRegsDrain = 104;
static_assert(128 * kRegsCtl + 3 * 128 * kRegsBuild + 2 * 128 * kRegsDrain <= kThreads * kLaunchRegs,
              "register split above the launch allocation");
constexpr int kTileM = kPairTileM, kTileN = kPairTileN;   // 256 x 128 per pair
constexpr int kRows = 128;                  // A rows (tensor-memory lanes) per CTA
constexpr int kBRows = kTileN / 2;          // B rows per CTA (its half of N)
constexpr int kStage = 32;                  // samples per stage
constexpr int kRowBytes = 64;               // 32 fp16 / bf16 samples
constexpr int kBPartBytes = kBRows * kRowBytes;   // one part (hi or lo) of B
// Operand kinds: 0 = bf16 hi/lo, 2 = fp16 hi/lo, 3 = fp16 in three parts of a
// double-float X~ (orders 2 to 5, and order 6 on few samples).
constexpr int kPrecise = 3;
template <int KIND> constexpr int parts_of() { return KIND == kPrecise ? 3 : 2; }
template <int KIND> constexpr int slot_bytes() { return parts_of<KIND>() * kBPartBytes; }   // B parts of one stage
// Tensor memory: 3 accumulator buffers of 128 columns, then 4 A stages of 32
// columns (hi 16 + lo 16: 32 fp16 samples per row).  The tensor core reads its
// shared-memory operands at about 64 bytes per cycle, which B alone fills at
// the MMA rate; A read from shared memory as well halved the MMA rate.
constexpr int kAccBufs = 3;
constexpr int kAStageCols = 32;             // hi 16 + lo 16 columns (32 fp16 samples of each part)
template <int KIND> constexpr int a_stage_cols() { return KIND == kPrecise ? 64 : kAStageCols; }   // 3 x 16, padded
template <int KIND> constexpr int max_slots() { return KIND == kPrecise ? 2 : 4; }
constexpr int kABase = kAccBufs * kTileN;
constexpr int kTmemCols = 512;
constexpr int kFoldEvery = 128;             // stages between FP64 folds (4096 samples)
constexpr int kMaxSlots = 4, kMaxSlabs = 8;   // operand stages (2 for three parts): A in tensor memory, B in shared memory
static_assert(kABase + kMaxSlots * kAStageCols == kTmemCols, "tensor memory map");
static_assert(kABase + max_slots<kPrecise>() * a_stage_cols<kPrecise>() == kTmemCols, "tensor memory map (3 parts)");
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
    int nslots;              // operand ring depth (2 or 4)
    int nslabs;              // X~ slab ring depth (2, 4 or 8)
    int alt_build;           // builders take alternate stages (whole rows) instead of half rows of every stage
    int box_bytes;           // one X~ box: box rows x 128 bytes (32 fp32 samples)
    int slab_bytes;          // one slab of the ring: the hi box, then (3 parts) the lo box
    const int* vexp;         // power-of-two scale exponent of each variable (X~ carries 2^vexp)
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

// 32 accumulator columns of this warp's lanes (two loads of 16, one wait),
// returned as 16 packed pairs (column 2i in the low half), ready for packed
// FP32 adds.
__device__ __forceinline__ void tmem_ld32_pairs(uint32_t taddr, uint64_t* p)
{
    asm volatile(
        "{\n .reg .b32 r<32>;\n"
        " tcgen05.ld.sync.aligned.32x32b.x16.b32 {r0, r1, r2, r3, r4, r5, r6, r7, r8, r9, r10, r11, r12, r13, r14, "
        "r15}, [%16];\n"
        " tcgen05.ld.sync.aligned.32x32b.x16.b32 {r16, r17, r18, r19, r20, r21, r22, r23, r24, r25, r26, r27, r28, "
        "r29, r30, r31}, [%17];\n"
        " tcgen05.wait::ld.sync.aligned;\n"
        " mov.b64 %0, {r0, r1};\n mov.b64 %1, {r2, r3};\n mov.b64 %2, {r4, r5};\n mov.b64 %3, {r6, r7};\n"
        " mov.b64 %4, {r8, r9};\n mov.b64 %5, {r10, r11};\n mov.b64 %6, {r12, r13};\n mov.b64 %7, {r14, r15};\n"
        " mov.b64 %8, {r16, r17};\n mov.b64 %9, {r18, r19};\n mov.b64 %10, {r20, r21};\n mov.b64 %11, {r22, r23};\n"
        " mov.b64 %12, {r24, r25};\n mov.b64 %13, {r26, r27};\n mov.b64 %14, {r28, r29};\n mov.b64 %15, {r30, r31};\n"
        "}\n"
        : "=l"(p[0]), "=l"(p[1]), "=l"(p[2]), "=l"(p[3]), "=l"(p[4]), "=l"(p[5]), "=l"(p[6]), "=l"(p[7]),
          "=l"(p[8]), "=l"(p[9]), "=l"(p[10]), "=l"(p[11]), "=l"(p[12]), "=l"(p[13]), "=l"(p[14]), "=l"(p[15])
        : "r"(taddr), "r"(taddr + 16u)
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
// split partials), times 2^-(sum of the entry's variable exponents) and, for
// three parts, also 2^-(30 - 5 d) (the builders' factors on A and B rows).
// ncols is a multiple of 16.
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
    constexpr bool kScaled = true;   // the centring scales X~ by 2^vexp for every pair kind
    decode_col_tuple(tu, DA, DB, sh.nbar, sh.bd, &cbase, &cfirst, kScaled ? cblk : nullptr);
    if (kScaled) {
        if (KIND == kPrecise) rexp = 30 - 5 * (DA + DB);   // the builders' 2^(15 - 5 NF) on A and on B
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
                if (kScaled) {
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
                    decode_col_tuple(tu, DA, DB, sh.nbar, sh.bd, &cbase, &cfirst, kScaled ? cblk : nullptr);
                if (kScaled) {
#pragma unroll
                    for (int i = 0; i < DB; ++i) dig[i] = 0;
                }
            } else if (kScaled) {
#pragma unroll
                for (int i = DB - 1; i >= 0; --i) {
                    if (++dig[i] < sh.b) break;
                    dig[i] = 0;
                }
            }
        }
    }
}

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
        split_f16_h8(z01, hi[0], lo[0]);
        split_f16_h8(z23, hi[1], lo[1]);
        split_f16_h8(w01, hi[2], lo[2]);
        split_f16_h8(w23, hi[3], lo[3]);
    } else {
        split_bf16(z01, hi[0], lo[0]);
        split_bf16(z23, hi[1], lo[1]);
        split_bf16(w01, hi[2], lo[2]);
        split_bf16(w23, hi[3], lo[3]);
    }
}

// Shared-memory barrier block: byte offsets of each ring's mbarriers (slot i
// at + 8 i), so that every role addresses them from one base register.
constexpr uint32_t kOffXfull = 0;                                  // X~ slab landed (TMA bytes)
constexpr uint32_t kOffXempty = kOffXfull + 8 * kMaxSlabs;         // every builder warp of the CTA arrives
constexpr uint32_t kOffOpfull = kOffXempty + 8 * kMaxSlabs;        // even CTA: every builder warp of both CTAs
constexpr uint32_t kOffOpempty = kOffOpfull + 8 * kMaxSlots;       // MMA commits, in both CTAs
constexpr uint32_t kOffAccfull = kOffOpempty + 8 * kMaxSlots;      // MMA commits, in both CTAs
constexpr uint32_t kOffAccempty = kOffAccfull + 8 * kAccBufs;      // even CTA: both CTAs' drainer warps
constexpr uint32_t kOffMmadone = kOffAccempty + 8 * kAccBufs;      // one per MMA issuer
constexpr uint32_t kOffTmemSlot = kOffMmadone + 16;
constexpr uint32_t kOffAbort = kOffTmemSlot + 4;
constexpr uint32_t kBarBytes = kOffAbort + 12;

// What a builder warp needs of the CTA's shared state.
struct Builder {
    uint32_t bb;             // shared address of the barrier block
    uint32_t slab, slots;    // shared addresses of the X~ slab ring and the B operand slots
    uint32_t tA;             // A parts: this thread's lane and half in the first A stage of tensor memory
    volatile int* abort_flag;
    int lg_ns, lg_nx;        // log2 of the ring depths
    int half, prow;          // which 16 samples of each stage; row within the CTA's A or B rows
    int par;                 // -1: every stage, half a row; 0 / 1: stages of this parity, whole rows
};

// Builder warp loop.  A rows (IS_A): row = tensor-memory lane, so a warp
// builds rows of its lane quarter and stores them with tcgen05.st; B rows: 64
// per CTA into the shared-memory slot.  Each thread builds samples
// 16 h .. 16 h + 15 of its row (h = B.half) in every stage, or (B.par >= 0)
// all 32 samples of its row in the stages of parity B.par; each warp arrives
// for itself once its part is stored.  The parity waits stay exact in both
// forms: the ring depths are even, so the previous use of a slot or slab was
// a stage this warp itself waited for.
template <int KIND, int DA, int DB, bool IS_A>
__device__ __forceinline__ void build_part(const Params& P, const Builder& B, uint32_t cta, int lane, int64_t pair_id,
                                        int64_t npairs)
{
    constexpr int NF = IS_A ? DA : DB;
    const Shape& sh = P.sh;
    // stage g of the pair uses operand slot g mod NS and slab g mod NX (both
    // powers of two), in lap g / NS and g / NX of their rings
    uint32_t g = 0;
    for (int64_t w = pair_id; w < P.units; w += npairs) {
        Unit u;
        get_unit(P, w, u);
        KrRow<NF> kr;
        int col[NF];
        if (IS_A) {
            const int64_t p = u.I * kTileM + (int64_t)cta * kRows + B.prow;
            if (p < sh.rows) {
                const RowInfo ri = decode_row(p, DA, DB, sh.b, sh.nbar, sh.bdA, sh.bdB, sh.bd);
#pragma unroll
                for (int f = 0; f < NF; ++f) col[f] = ri.col[f];
            } else {
#pragma unroll
                for (int f = 0; f < NF; ++f) col[f] = 0;
            }
        } else {
            // B row prow of CTA c: tile column 64 c + prow (the MMA takes CTA 0's rows first)
            const int64_t q = u.J * kTileN + (int64_t)cta * kBRows + B.prow;
            if (q < sh.cols) {
                const ColInfo ci = decode_col(q, DA, DB, sh.b, sh.nbar, sh.bdB, sh.bd);
#pragma unroll
                for (int f = 0; f < NF; ++f) col[f] = ci.col[f];
            } else {
#pragma unroll
                for (int f = 0; f < NF; ++f) col[f] = 0;
            }
        }
        kr.set(col);
        // three parts: the product of the scaled factors (below 2^5 each)
        // times 2^(15 - 5 NF), exact in FP32: it stays below 2^15, and its
        // second and third parts as far above the fp16 subnormals as that allows
        const float zscale = __int_as_float((127 + 15 - 5 * NF) << 23);
        const int nst = (int)u.nst;
        for (int st = 0; st < nst; ++st, ++g) {
            if (B.par >= 0 && (int)(g & 1u) != B.par) continue;
            const uint32_t os = g & ((1u << B.lg_ns) - 1u), xs = g & ((1u << B.lg_nx) - 1u);
            bool okw = true;
            if (lane == 0)
                okw = wait_bar(B.bb + kOffXfull + 8 * xs, (g >> B.lg_nx) & 1u, B.abort_flag, P.status) &&
                      wait_bar(B.bb + kOffOpempty + 8 * os, ((g >> B.lg_ns) & 1u) ^ 1u, B.abort_flag, P.status);
            if (!warp_agree(okw)) return;
            uint32_t a[NF];
            kr.addresses(B.slab + xs * (uint32_t)P.slab_bytes, a);
            if (KIND == kPrecise) {
                // z = product of the factors (hi + lo) as a double-float, then
                // three fp16 parts of each pair of samples; stored chunk by
                // chunk (8 samples) to keep few registers live
                if (IS_A) fence_after();
                const int h0 = B.par >= 0 ? 0 : B.half, h1 = B.par >= 0 ? 2 : B.half + 1;
#pragma unroll 1
                for (int half = h0; half < h1; ++half) {
                    const uint32_t ta = B.tA + os * (uint32_t)a_stage_cols<KIND>() + 8u * (uint32_t)half;
                    const uint32_t base = B.slots + os * (uint32_t)slot_bytes<KIND>();
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        uint32_t q1[4], q2[4], q3[4];
#pragma unroll
                        for (int qq = 0; qq < 2; ++qq) {
                            const uint32_t lc = (uint32_t)(4 * half + 2 * c + qq);
                            float zh[4], zl[4];
                            {
                                const uint32_t ad = a[0] ^ (lc << 4);
                                const float4 h = lds128(ad), l = lds128(ad + (uint32_t)P.box_bytes);
                                zh[0] = h.x; zh[1] = h.y; zh[2] = h.z; zh[3] = h.w;
                                zl[0] = l.x; zl[1] = l.y; zl[2] = l.z; zl[3] = l.w;
                            }
#pragma unroll
                            for (int f = 1; f < NF; ++f) {
                                const uint32_t ad = a[f] ^ (lc << 4);
                                const float4 h = lds128(ad), l = lds128(ad + (uint32_t)P.box_bytes);
                                const float bh[4] = {h.x, h.y, h.z, h.w};
                                const float bl[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
                                for (int i = 0; i < 4; ++i) {
                                    // TwoProduct of the hi parts plus the cross terms
                                    const float pr = zh[i] * bh[i];
                                    const float er = fmaf(zh[i], bh[i], -pr);
                                    const float cr = fmaf(zh[i], bl[i], zl[i] * bh[i]);
                                    zh[i] = pr;
                                    zl[i] = er + cr;
                                }
                            }
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                zh[i] *= zscale;
                                zl[i] *= zscale;
                            }
                            split3_f16(make_float2(zh[0], zh[1]), make_float2(zl[0], zl[1]), q1[2 * qq], q2[2 * qq],
                                       q3[2 * qq]);
                            split3_f16(make_float2(zh[2], zh[3]), make_float2(zl[2], zl[3]), q1[2 * qq + 1],
                                       q2[2 * qq + 1], q3[2 * qq + 1]);
                        }
                        if (IS_A) {
                            tmem_st4(ta + 4 * c, q1);
                            tmem_st4(ta + 16 + 4 * c, q2);
                            tmem_st4(ta + 32 + 4 * c, q3);
                        } else {
                            const uint32_t off = base + sw64(B.prow, 2 * half + c);
                            sts128(off, q1[0], q1[1], q1[2], q1[3]);
                            sts128(off + kBPartBytes, q2[0], q2[1], q2[2], q2[3]);
                            sts128(off + 2 * kBPartBytes, q3[0], q3[1], q3[2], q3[3]);
                        }
                    }
                }
                if (IS_A) {
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    fence_before();
                } else {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                }
            } else if (IS_A) {
                fence_after();   // the MMAs that read this A stage before (opempty) have completed
                const int h0 = B.par >= 0 ? 0 : B.half, h1 = B.par >= 0 ? 2 : B.half + 1;
#pragma unroll 1
                for (int half = h0; half < h1; ++half) {
                    uint32_t h[8], l[8];
                    build_chunk<KIND, NF>(a, 2 * half, h, l);
                    build_chunk<KIND, NF>(a, 2 * half + 1, h + 4, l + 4);
                    const uint32_t ta = B.tA + os * (uint32_t)a_stage_cols<KIND>() + 8u * (uint32_t)half;
                    tmem_st8(ta, h);
                    tmem_st8(ta + 16, l);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                fence_before();
            } else {
                const uint32_t hi_base = B.slots + os * (uint32_t)slot_bytes<KIND>();
                const int c0 = B.par >= 0 ? 0 : 2 * B.half, c1 = B.par >= 0 ? 4 : 2 * B.half + 2;
#pragma unroll 1
                for (int c = c0; c < c1; ++c) {
                    uint32_t h[4], l[4];
                    build_chunk<KIND, NF>(a, c, h, l);
                    const uint32_t off = hi_base + sw64(B.prow, c);
                    sts128(off, h[0], h[1], h[2], h[3]);
                    sts128(off + kBPartBytes, l[0], l[1], l[2], l[3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(B.bb + kOffXempty + 8 * xs);
                mbar_arrive_remote(B.bb + kOffOpfull + 8 * os, 0u);
            }
        }
    }
}

// ------------------------------------------------------------------ kernel

// Stages of 32 samples in work unit w, and its first sample.
__device__ __forceinline__ int unit_stages(const Params& P, int64_t w)
{
    const int64_t k0 = (w % P.S) * P.kchunk;
    const int64_t k1 = k0 + P.kchunk < P.t_pad ? k0 + P.kchunk : P.t_pad;
    return (int)((k1 - k0) / kStage);
}

template <int KIND, int DA, int DB>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    moment_pair_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap_lo,
                       const __grid_constant__ Params P)
{
    constexpr uint32_t IDESC = idesc_pair(KIND == 0 ? 1u : 0u);
    constexpr int kSlot = slot_bytes<KIND>(), kAStage = a_stage_cols<KIND>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int NS = P.nslots, NX = P.nslabs;
    const uint32_t slots = su32(smem);                                   // NS x (B parts)
    const uint32_t slab = slots + (uint32_t)(NS * kSlot);                // NX x one X~ slab
    uint8_t* bar_ptr = smem + NS * kSlot + NX * P.slab_bytes;
    const uint32_t bb = su32(bar_ptr);
    uint32_t* tmem_slot = (uint32_t*)(bar_ptr + kOffTmemSlot);
    volatile int* abort_flag = (volatile int*)(bar_ptr + kOffAbort);

    const uint32_t cta = cta_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        // builder and drainer warps each arrive for themselves (lane 0, after
        // __syncwarp); drainers with a relaxed arrive (tensor memory only)
        for (int i = 0; i < NX; ++i) {
            mbar_init(bb + kOffXfull + 8 * i, 1);
            mbar_init(bb + kOffXempty + 8 * i, P.alt_build ? kBuildWarps / 2 : kBuildWarps);
        }
        for (int i = 0; i < NS; ++i) {
            mbar_init(bb + kOffOpfull + 8 * i, P.alt_build ? kBuildWarps : 2 * kBuildWarps);
            mbar_init(bb + kOffOpempty + 8 * i, 1);
        }
        for (int i = 0; i < kAccBufs; ++i) {
            mbar_init(bb + kOffAccfull + 8 * i, 1);
            mbar_init(bb + kOffAccempty + 8 * i, 2 * kDrainWarps);
        }
        mbar_init(bb + kOffMmadone, 1);
        mbar_init(bb + kOffMmadone + 8, 1);
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
    // (each role's branch first sets its warpgroup's register count, so that
    // the compiler allocates the code below it within that count)
    if (warp < kWarpA0) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsCtl));
        if (warp == kWarpTma && lane == 0) {
            // ------------------------------------------------------ X~ loads (each CTA its own slabs)
            Ring xr(NX);
            int issued = 0;
            bool ok = true;
            for (int64_t w = pair_id; w < P.units && ok; w += npairs) {
                const int nst = unit_stages(P, w);
                const int k0 = (int)((w % P.S) * P.kchunk);
                for (int st = 0; st < nst; ++st, xr.next()) {
                    if (!(ok = wait_bar(bb + kOffXempty + 8 * xr.slot, xr.phase ^ 1u, abort_flag, P.status))) break;
                    const uint32_t full = bb + kOffXfull + 8 * xr.slot;
                    const uint32_t dst = slab + (uint32_t)(xr.slot * P.slab_bytes);
                    mbar_expect_tx(full, (uint32_t)P.slab_bytes);
                    tma_load_2d(dst, &tmap, k0 + st * kStage, 0, full);
                    if (KIND == kPrecise) tma_load_2d(dst + (uint32_t)P.box_bytes, &tmap_lo, k0 + st * kStage, 0, full);
                    ++issued;
                }
            }
            // the last load into each slab has landed before the CTA leaves
            for (int i = issued > NX ? issued - NX : 0; i < issued; ++i)
                wait_bar_bounded(bb + kOffXfull + 8 * (i % NX), (uint32_t)((i / NX) & 1), P.status);
        } else if ((warp == kWarpMma0 || warp == kWarpMma) && cta == 0 && lane == 0) {
            // ------------------------------------------------------ MMA issuers (even CTA)
            // Stage g accumulates into accumulator buffer g mod 3: 8 MMAs
            // (lo*lo, hi*lo, lo*hi, hi*hi over two K steps; A from tensor
            // memory, B from shared memory) once the stage's operands are
            // built and the buffer's previous stage is drained.  Two threads in
            // two warps take alternate stages: an mbarrier wait issued behind a
            // thread's own MMAs returns only after the tensor core has taken
            // them, so one issuing thread left the pipe idle for about 280
            // cycles of each 512-cycle stage; with two, one waits while the
            // other's MMAs run.  The parity waits stay exact: builders and
            // drainers finish stages in order, and each thread has seen stage
            // g - 2 complete before it waits for stage g.
            const uint32_t mine = warp == kWarpMma ? 0u : 1u;
            const uint64_t bh0 = smem_desc64(slots), bl0 = smem_desc64(slots + kBPartBytes);
            Ring orr(NS), dr(kAccBufs);
            uint32_t g = 0;
            bool ok = true;
            for (int64_t w = pair_id; w < P.units && ok; w += npairs) {
                const int nst = unit_stages(P, w);
                for (int st = 0; st < nst; ++st, ++g, orr.next(), dr.next()) {
                    if ((g & 1u) != mine) continue;
                    ok = wait_cluster(bb + kOffOpfull + 8 * orr.slot, orr.phase, abort_flag, P.status) &&
                         wait_cluster(bb + kOffAccempty + 8 * dr.slot, dr.phase ^ 1u, abort_flag, P.status);
                    if (!ok) break;
                    fence_after();
                    const uint32_t d = tmem + (uint32_t)(dr.slot * kTileN);
                    const uint32_t ah = tmem + (uint32_t)(kABase + orr.slot * kAStage), al = ah + 16u;
                    const uint64_t so = (uint64_t)orr.slot * (kSlot >> 4);
                    const uint64_t bh = bh0 + so, bl = bl0 + so;
                    if (KIND == kPrecise) {
                        // parts 1..3 of A at ah, ah + 16, ah + 32; of B at bh, bl,
                        // bl + one part (8, 11, 11 bits: weights 1, 2^-8, 2^-19):
                        // the six products of weight down to 2^-19 (the dropped
                        // ones weigh 2^-27 and less), smallest first, over the
                        // stage's two K steps
                        const uint32_t a2 = ah + 16u, a3 = ah + 32u;
                        const uint64_t b2 = bl, b3 = bl + (kBPartBytes >> 4);
                        mma_pair(d, a3, bh, IDESC, 0u);
                        mma_pair(d, a3 + 8, bh + 2, IDESC, 1u);
                        mma_pair(d, a2, b2, IDESC, 1u);
                        mma_pair(d, a2 + 8, b2 + 2, IDESC, 1u);
                        mma_pair(d, ah, b3, IDESC, 1u);
                        mma_pair(d, ah + 8, b3 + 2, IDESC, 1u);
                        mma_pair(d, a2, bh, IDESC, 1u);
                        mma_pair(d, a2 + 8, bh + 2, IDESC, 1u);
                        mma_pair(d, ah, b2, IDESC, 1u);
                        mma_pair(d, ah + 8, b2 + 2, IDESC, 1u);
                        mma_pair(d, ah, bh, IDESC, 1u);
                        mma_pair(d, ah + 8, bh + 2, IDESC, 1u);
                        commit_both(bb + kOffAccfull + 8 * dr.slot);
                        commit_both(bb + kOffOpempty + 8 * orr.slot);
                        continue;
                    }
                    mma_pair(d, al, bl, IDESC, 0u);
                    mma_pair(d, al + 8, bl + 2, IDESC, 1u);
                    mma_pair(d, ah, bl, IDESC, 1u);
                    mma_pair(d, ah + 8, bl + 2, IDESC, 1u);
                    mma_pair(d, al, bh, IDESC, 1u);
                    mma_pair(d, al + 8, bh + 2, IDESC, 1u);
                    mma_pair(d, ah, bh, IDESC, 1u);
                    mma_pair(d, ah + 8, bh + 2, IDESC, 1u);
                    commit_both(bb + kOffAccfull + 8 * dr.slot);
                    commit_both(bb + kOffOpempty + 8 * orr.slot);
                }
            }
            // every MMA this thread issued has completed before the pair tears down
            commit_both(bb + kOffMmadone + 8 * mine);
            wait_bar_bounded(bb + kOffMmadone + 8 * mine, 0u, P.status);
        }
    } else if (warp < kWarpD0) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsBuild));
        // ---------------------------------------------------------- builders: Khatri-Rao rows
        const int bw = warp - kWarpA0;
        Builder B;
        B.bb = bb;
        B.slab = slab;
        B.slots = slots;
        B.abort_flag = abort_flag;
        B.lg_ns = 31 - __clz(NS);
        B.lg_nx = 31 - __clz(NX);
        B.par = P.alt_build ? (bw < kAWarps ? bw >> 2 : (bw - kAWarps) >> 1) : -1;
        if (bw < kAWarps) {
            B.half = bw >> 2;
            B.prow = (warp & 3) * 32 + lane;
            B.tA = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)kABase;
            build_part<KIND, DA, DB, true>(P, B, cta, lane, pair_id, npairs);
        } else {
            B.half = (bw - kAWarps) >> 1;
            B.prow = ((bw - kAWarps) & 1) * 32 + lane;
            B.tA = 0;
            build_part<KIND, DA, DB, false>(P, B, cta, lane, pair_id, npairs);
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsDrain));
        // ---------------------------------------------------------- drainers: register running sums
        // Each thread owns 64 accumulator columns of one tile row (its lane):
        // per stage it adds them to FP32 running sums held in registers as
        // packed pairs, folds 16-column groups into the FP64 scratch tile at
        // staggered stages, and at the end of a unit writes its row segment.
        const int q4 = warp & 3, dh = (warp - kWarpD0) >> 2;   // lane quarter; which 64 of the 128 columns
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
            const int nst = unit_stages(P, w);
            for (int k = 0; k < nst; ++k, dr.next()) {
                bool okw = true;
                if (lane == 0) okw = wait_bar(bb + kOffAccfull + 8 * dr.slot, dr.phase, abort_flag, P.status);
                if (!(ok = warp_agree(okw))) break;
                fence_after();
                const uint32_t t0 = tD + (uint32_t)(dr.slot * kTileN);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint64_t v[16];
                    tmem_ld32_pairs(t0 + 32 * h, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) run[16 * h + j] = add_pair(run[16 * h + j], v[j]);
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_remote_relaxed(bb + kOffAccempty + 8 * dr.slot, 0u);
                // group c folds after the stages k = 32 c + 31 (mod 128)
                const int kp = k & (kFoldEvery - 1);
                if ((kp & 31) == 31 && k + 1 < nst) fold(kp >> 5, k < kFoldEvery);
            }
            if (!ok) break;
#pragma unroll
            for (int c = 0; c < kDrainCols / 16; ++c) fold(c, 32 * c + 31 >= nst - 1);
            Unit u;
            get_unit(P, w, u);
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

static size_t smem_bytes(int slot_b, int nslots, int nslabs, int slab_b)
{
    return 1024 + (size_t)nslots * slot_b + (size_t)nslabs * slab_b + kBarBytes;
}

template <int KIND, int DA, int DB>
static cudaError_t launch_typed(const CUtensorMap& map, const CUtensorMap& map_lo, const Params& P, size_t smem,
                                cudaStream_t st)
{
    auto kern = moment_pair_kernel<KIND, DA, DB>;
    // the register shares the warpgroups take with setmaxnreg assume this
    // launch allocation; below it setmaxnreg.inc could wait forever
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if (fa.numRegs < kLaunchRegs) return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
    kern<<<(unsigned)(2 * pairs), kThreads, smem, st>>>(map, map_lo, P);
    return cudaGetLastError();
}

template <int KIND>
static cudaError_t launch_kind(const CUtensorMap& map, const CUtensorMap& map_lo, const Params& P, size_t smem,
                               cudaStream_t st)
{
    const int dA = P.sh.dA, dB = P.sh.dB;
    if constexpr (KIND == kPrecise) {
        if (dA == 1 && dB == 1) return launch_typed<kPrecise, 1, 1>(map, map_lo, P, smem, st);
        if (dA == 2 && dB == 1) return launch_typed<kPrecise, 2, 1>(map, map_lo, P, smem, st);
        if (dA == 2 && dB == 2) return launch_typed<kPrecise, 2, 2>(map, map_lo, P, smem, st);
        if (dA == 3 && dB == 2) return launch_typed<kPrecise, 3, 2>(map, map_lo, P, smem, st);
        if (dA == 3 && dB == 3) return launch_typed<kPrecise, 3, 3>(map, map_lo, P, smem, st);
        return cudaErrorInvalidValue;
    } else {
        if (dA == 1 && dB == 1) return launch_typed<KIND, 1, 1>(map, map_lo, P, smem, st);
        if (dA == 2 && dB == 1) return launch_typed<KIND, 2, 1>(map, map_lo, P, smem, st);
        if (dA == 2 && dB == 2) return launch_typed<KIND, 2, 2>(map, map_lo, P, smem, st);
        if (dA == 3 && dB == 2) return launch_typed<KIND, 3, 2>(map, map_lo, P, smem, st);
        if (dA == 3 && dB == 3) return launch_typed<KIND, 3, 3>(map, map_lo, P, smem, st);
        return cudaErrorInvalidValue;
    }
}

}  // namespace pair

cudaError_t launch_moment_pair(const OrderPlan& OP, int prec, const float* xt, const float* xlo, int64_t t_pad,
                               const int64_t* prefix, double* out, double scale, double* scratch, int* status,
                               const int* vexp, cudaStream_t st)
{
    using namespace pair;
    if (OP.units <= 0) return cudaSuccess;
    const bool precise = OP.precise;
    if (precise) {
        if (!prec_is_tc(prec) || !xlo || !vexp) return cudaErrorInvalidValue;
    } else {
        if (!prec_is_tc(prec) || !vexp) return cudaErrorInvalidValue;
    }
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
    P.slab_bytes = P.box_bytes * (precise ? 2 : 1);
    if (OP.kchunk % kStage || t_pad % kStage) return cudaErrorInvalidValue;
    int dev = 0, maxsmem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    // ring depths are powers of two (the builders index them with masks)
    const int slot_b = precise ? slot_bytes<kPrecise>() : slot_bytes<0>();
    int ns = precise ? max_slots<kPrecise>() : max_slots<0>(), nx = kMaxSlabs;
    while (nx > 2 && smem_bytes(slot_b, ns, nx, P.slab_bytes) > (size_t)maxsmem) nx >>= 1;
    while (ns > 2 && smem_bytes(slot_b, ns, nx, P.slab_bytes) > (size_t)maxsmem) ns >>= 1;
    if (smem_bytes(slot_b, ns, nx, P.slab_bytes) > (size_t)maxsmem) return cudaErrorInvalidValue;
    P.nslots = ns;
    P.nslabs = nx;
    // two parts: each builder warp takes whole rows of every other stage, so
    // it synchronises once per two stages (order 6: 87.6 ms against 89.1 for
    // half rows of every stage); three parts keep half rows: with two operand
    // slots, builders of one parity wait for the MMAs two stages back
    P.alt_build = precise ? 0 : 1;
    CUtensorMap map, map_lo;
    if (!encode_xt_map(&map, xt, t_pad, OP.sh.n_pad)) return cudaErrorInvalidValue;
    if (precise) {
        if (!encode_xt_map(&map_lo, xlo, t_pad, OP.sh.n_pad)) return cudaErrorInvalidValue;
    } else {
        map_lo = map;
    }
    const size_t smem = smem_bytes(slot_b, ns, nx, P.slab_bytes);
    if (precise) return launch_kind<kPrecise>(map, map_lo, P, smem, st);
    if (prec == CUM_PREC_BF16X3) return launch_kind<0>(map, map_lo, P, smem, st);
    return launch_kind<2>(map, map_lo, P, smem, st);   // FP16X3, and TF32X3 outside batches
}

}  // namespace cum
