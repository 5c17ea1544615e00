// Device helpers shared by the tensor-core moment contractions of libcumgb
// (moment_tc.cu: one CTA per tile; moment_pair.cu: CTA pairs): inline PTX for
// mbarriers, bounded waits, TMA and tensor memory, packed FP32 arithmetic, the
// Khatri-Rao row loads from the swizzled X~ slab and the hi/lo splits.
#pragma once

#include <cuda.h>
#include <cstdint>

#include "cumgb.h"
#include "internal.h"

namespace cum {
namespace tc {

constexpr long long kWaitLimit = 4000000000LL;   // clock64 cycles (about 2 s)

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait with a suspend-time hint: a waiting thread sleeps in hardware until
// the phase completes or about `ns` nanoseconds pass, instead of re-polling
// shared memory (the polls of a dozen waiting warps compete with the tensor
// core's operand reads).
__device__ __forceinline__ bool mbar_try_sleep(uint32_t bar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Bounded wait on phase `parity` of an mbarrier.  Returns false (and raises the
// CTA abort flag and the device status word) if the limit expires, or if
// another role has aborted.  The abort flag and the clock are checked every 16
// sleeps only.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_sleep(bar, parity, 20000u)) return true;
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

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t* v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3])
                 : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* v)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

// 16 columns of this warp's lanes, without waiting (pair with tmem_wait_ld).
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t* v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr)
                 : "memory");
}

// 32 columns of this warp's lanes, without waiting (pair with tmem_wait_ld).
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* v)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* f)
{
    uint32_t v[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) f[i] = __uint_as_float(v[i]);
}

// ------------------------------------------------------------------ operand construction

// Packed FP32 pair arithmetic (one instruction for two lanes of work).
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 r;
    asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n mul.rn.f32x2 z, x, y;\n"
        " mov.b64 {%0, %1}, z;\n}\n"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    float2 r;
    asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n add.rn.f32x2 z, x, y;\n"
        " mov.b64 {%0, %1}, z;\n}\n"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 r;
    asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n sub.rn.f32x2 z, x, y;\n"
        " mov.b64 {%0, %1}, z;\n}\n"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// Product over the factors of 4 consecutive samples (quad u of the stage) of
// X~ columns col[0..NF-1], read from the swizzled slab.
// Khatri-Rao row of NF factors, as seen by one thread: the slab rows of its
// factor columns (relative to the slab base) and their 128-byte swizzle keys,
// fixed for a whole work unit.
template <int NF>
struct KrRow {
    uint32_t off[NF];   // column * 128 + ((column & 7) << 4): the row's chunk 0 in the box
    __device__ __forceinline__ void set(const int* col)
    {
#pragma unroll
        for (int f = 0; f < NF; ++f) off[f] = (uint32_t)col[f] * 128u + (((uint32_t)col[f] & 7u) << 4);
    }
    // Shared-memory address of chunk 0 of each factor's row in the box at
    // `box32` (1024-byte aligned): the row's 16-byte chunk lc is then at
    // addr ^ (lc << 4), since the 128-byte swizzle only permutes address
    // bits 4-6 and the box base leaves them clear.
    __device__ __forceinline__ void addresses(uint32_t box32, uint32_t* a) const
    {
#pragma unroll
        for (int f = 0; f < NF; ++f) a[f] = box32 + off[f];
    }
};

// 16-byte shared-memory load (volatile: stays after the barrier waits that
// make the slab valid).
__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ float4 lds128(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}

// Product over the factors of the 4 samples in chunk lc of the row's box,
// from the addresses of KrRow::addresses.
template <int NF>
__device__ __forceinline__ void kr_quad_at(const uint32_t* a, uint32_t lc, float2& z01, float2& z23)
{
    const float4 x0 = lds128(a[0] ^ (lc << 4));
    z01 = make_float2(x0.x, x0.y);
    z23 = make_float2(x0.z, x0.w);
#pragma unroll
    for (int f = 1; f < NF; ++f) {
        const float4 x = lds128(a[f] ^ (lc << 4));
        z01 = mul2(z01, make_float2(x.x, x.y));
        z23 = mul2(z23, make_float2(x.z, x.w));
    }
}

// (z0, z1) -> packed bf16 pairs hi = RN(z), lo = RN(z - hi) (element 0 in the low half).
__device__ __forceinline__ void split_bf16(float2 z, uint32_t& hi, uint32_t& lo)
{
    uint32_t h, l;
    float dx, dy;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(z.y), "f"(z.x));
    // z - hi, exact, from the packed halves: fma(hi, -1, z) with bf16 factors and
    // an f32 addend
    asm("{\n .reg .b16 a, b, m;\n mov.b32 {a, b}, %2;\n mov.b16 m, 0xBF80;\n"
        " fma.rn.f32.bf16 %0, a, m, %3;\n fma.rn.f32.bf16 %1, b, m, %4;\n}\n"
        : "=f"(dx), "=f"(dy)
        : "r"(h), "f"(z.x), "f"(z.y));
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(dy), "f"(dx));
    hi = h;
    lo = l;
}

// (z0, z1) -> packed fp16 hi = RN(z), lo = RN(z - hi); |z| < 2^15 by the scaling of X~.
__device__ __forceinline__ void split_f16(float2 z, uint32_t& hi, uint32_t& lo)
{
    uint32_t h, l;
    float dx, dy;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(z.y), "f"(z.x));
    asm("{\n .reg .f16 a, b, m;\n mov.b32 {a, b}, %2;\n mov.b16 m, 0xBC00;\n"
        " fma.rn.f32.f16 %0, a, m, %3;\n fma.rn.f32.f16 %1, b, m, %4;\n}\n"
        : "=f"(dx), "=f"(dy)
        : "r"(h), "f"(z.x), "f"(z.y));
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(dy), "f"(dx));
    hi = h;
    lo = l;
}

// (z0, z1) -> packed fp16 hi = z rounded to 8 significant bits (through bf16,
// then to fp16), lo = RN16(z - z8) with z8 the 8-bit rounding itself (one
// packed FP32 subtraction, exact): 19 bits of z.  Beside split_f16's 22 bits
// the short hi part keeps the products of hi parts exact on the tensor core's
// alignment grid over a wider range of magnitudes, which cuts the bias of its
// truncating accumulation by about a third; the lost bits are rounded to
// nearest, unbiased, and average out over the samples.  hi equals z8 except
// where z8 is an fp16 subnormal (|z| < 2^-7), and there differs from it by at
// most 2^-25.
__device__ __forceinline__ void split_f16_h8(float2 z, uint32_t& hi, uint32_t& lo)
{
    uint32_t b8, h, l;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(b8) : "f"(z.y), "f"(z.x));
    const float2 z8 = make_float2(__uint_as_float(b8 << 16), __uint_as_float(b8 & 0xffff0000u));
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(z8.y), "f"(z8.x));
    const float2 d = sub2(z, z8);
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(d.y), "f"(d.x));
    hi = h;
    lo = l;
}

// Double-float pairs (zh + zl, element 0 in .x) -> three packed fp16 parts,
// z ~ p1 + p2 + p3: p1 = zh rounded to 8 significant bits (through bf16, then
// exactly to fp16), p2 = RN16((zh - p1) + zl), p3 = RN16(r - p2) with
// r = (zh - p1) + zl.  zh - p1 and r - p2 are exact in FP32; r rounds once,
// at 2^-24 of |zh - p1| <= 2^-8 |zh|, so the parts carry about 30 bits of z.
// The short first part keeps the products of first parts (16 bits) exact on
// the tensor core's alignment grid over a wider range of magnitudes, which
// roughly halves the bias of its truncating accumulation.  Values stay below
// 2^15 by the scaling of X~.
__device__ __forceinline__ void split3_f16(float2 zh, float2 zl, uint32_t& p1, uint32_t& p2, uint32_t& p3)
{
    uint32_t h, m, l, b8;
    float dx, dy, ex, ey;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(b8) : "f"(zh.y), "f"(zh.x));
    const float h0 = __uint_as_float(b8 << 16), h1 = __uint_as_float(b8 & 0xffff0000u);
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(h1), "f"(h0));
    asm("{\n .reg .f16 a, b, m;\n mov.b32 {a, b}, %2;\n mov.b16 m, 0xBC00;\n"
        " fma.rn.f32.f16 %0, a, m, %3;\n fma.rn.f32.f16 %1, b, m, %4;\n}\n"
        : "=f"(dx), "=f"(dy)
        : "r"(h), "f"(zh.x), "f"(zh.y));
    const float rx = dx + zl.x, ry = dy + zl.y;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(m) : "f"(ry), "f"(rx));
    asm("{\n .reg .f16 a, b, m;\n mov.b32 {a, b}, %2;\n mov.b16 m, 0xBC00;\n"
        " fma.rn.f32.f16 %0, a, m, %3;\n fma.rn.f32.f16 %1, b, m, %4;\n}\n"
        : "=f"(ex), "=f"(ey)
        : "r"(m), "f"(rx), "f"(ry));
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(ey), "f"(ex));
    p1 = h;
    p2 = m;
    p3 = l;
}

// (z0, z1) -> tf32 hi = RN(z), lo = RN(z - hi), element by element: rounding
// to nearest (ties away from zero) on the magnitude bits, as cvt.rna does for
// finite normal values.
__device__ __forceinline__ uint32_t tf32_rna(uint32_t x) { return (x + 0x1000u) & 0xffffe000u; }

__device__ __forceinline__ void split_tf32(float2 z, uint32_t* hi, uint32_t* lo)
{
    const uint32_t h0 = tf32_rna(__float_as_uint(z.x)), h1 = tf32_rna(__float_as_uint(z.y));
    const float2 d = sub2(z, make_float2(__uint_as_float(h0), __uint_as_float(h1)));
    hi[0] = h0;
    hi[1] = h1;
    lo[0] = tf32_rna(__float_as_uint(d.x));
    lo[1] = tf32_rna(__float_as_uint(d.y));
}

// Position in a ring of n slots: slot index and the parity of the current lap.
// Waiting on a full barrier uses `phase`; waiting on an empty barrier uses
// phase ^ 1, which a freshly initialised barrier satisfies at once.
struct Ring {
    int slot;
    uint32_t phase;
    int n;
    __device__ __forceinline__ explicit Ring(int n_) : slot(0), phase(0u), n(n_) {}
    __device__ __forceinline__ void next()
    {
        if (++slot == n) {
            slot = 0;
            phase ^= 1u;
        }
    }
};

// Column part of the output address of the first column of dB-tuple u (colex
// rank of its reversed complement), and the tuple's first block index.
// Also returns the tuple's block indices in `blk` unless it is NULL.
__device__ __forceinline__ void decode_col_tuple(int64_t u, int dA, int dB, int nbar, int64_t bd, int64_t* base,
                                                 int* first, int* blk)
{
    int sp[kMaxHalf], s[kMaxHalf];
    colex_unrank(u, dB, nbar, sp);
    for (int k = 0; k < dB; ++k) s[k] = nbar - 1 - sp[dB - 1 - k];
    int64_t rk = 0;
    for (int k = 0; k < dB; ++k) rk += binom(s[k] + dA + k, dA + k + 1);
    *base = rk * bd;
    *first = s[0];
    if (blk)
        for (int k = 0; k < dB; ++k) blk[k] = s[k];
}

// 2^-e as a double, for |e| <= 1000.
__device__ __forceinline__ double exp2_neg(int e) { return __longlong_as_double((long long)(1023 - e) << 52); }

}  // namespace tc
}  // namespace cum
