// Shared host/device helpers of libcumgb: combinatorial number system for the
// block structure of super-symmetric tensors (Sec. 2.1), and the decoding of
// the two Khatri-Rao operand spaces of the moment contraction.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define CUM_HD __host__ __device__ __forceinline__

namespace cum {

constexpr int kMaxOrder = 6;     // largest d
constexpr int kMaxHalf = 3;      // largest dA = ceil(d/2)
constexpr int kMaxBinomM = 320;  // binomials C(m, k) are evaluated for m < kMaxBinomM

// C(m, k), exact in int64 for m < kMaxBinomM and k <= kMaxOrder + 1.
CUM_HD int64_t binom(int64_t m, int k)
{
    if (k < 0 || m < k) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (m - k + i) / i;  // r = C(m-k+i, i) after step i
    return r;
}

CUM_HD int64_t ipow(int64_t b, int e)
{
    int64_t r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

// Colex rank of a sorted (non-decreasing) tuple j[0..q-1]: sum_k C(j_k + k, k + 1)
// (0-based k), i.e. the rank of the strictly increasing set {j_k + k}.
CUM_HD int64_t colex_rank(const int* j, int q)
{
    int64_t r = 0;
    for (int k = 0; k < q; ++k) r += binom(j[k] + k, k + 1);
    return r;
}

// Inverse of colex_rank over tuples with entries in [0, nbar).
CUM_HD void colex_unrank(int64_t r, int q, int nbar, int* j)
{
    for (int k = q; k >= 1; --k) {
        // largest s in [k-1, nbar+k-2] with C(s, k) <= r
        int s = nbar + k - 2;
        while (s > k - 1 && binom(s, k) > r) --s;
        j[k - 1] = s - (k - 1);
        r -= binom(s, k);
    }
}

// Number of stored blocks C(nbar + d - 1, d).
CUM_HD int64_t num_blocks(int nbar, int d) { return binom((int64_t)nbar + d - 1, d); }

// Shape of the moment contraction of order d: M[rowOff(p) + colOff(q)] =
// sum_l ZA[l, p] * ZB[l, q] over the valid pairs last(p) <= first(q).
//  * row space p: sorted dA-tuples in colex order (grouped by their LAST block
//    index, ascending) x in-block indices (b^dA);
//  * col space q: sorted dB-tuples ordered by the colex order of their
//    reversed complement (nbar-1-s_dB, ..., nbar-1-s_1), i.e. grouped by their
//    FIRST block index, descending, x in-block indices (b^dB).
// The colex rank of the concatenated d-tuple splits into a row part and a
// column part, so the output address is separable.
struct Shape {
    int d, dA, dB, b, nbar, n_pad;
    int64_t bd, bdA, bdB;   // b^d, b^dA, b^dB
    int64_t rows, cols;     // E_dA, E_dB
    int64_t entries;        // E_d
};

inline Shape make_shape(int d, int n, int b)
{
    Shape s;
    s.d = d;
    s.dA = (d + 1) / 2;
    s.dB = d / 2;
    s.b = b;
    s.nbar = (n + b - 1) / b;
    s.n_pad = s.nbar * b;
    s.bd = ipow(b, d);
    s.bdA = ipow(b, s.dA);
    s.bdB = ipow(b, s.dB);
    s.rows = num_blocks(s.nbar, s.dA) * s.bdA;
    s.cols = num_blocks(s.nbar, s.dB) * s.bdB;
    s.entries = num_blocks(s.nbar, d) * s.bd;
    return s;
}

struct RowInfo {
    int col[kMaxHalf];   // variable (column of X~) of each factor
    int last;            // last block index of the tuple
    int64_t off;         // row part of the output address
};

CUM_HD RowInfo decode_row(int64_t p, int dA, int dB, int b, int nbar, int64_t bdA, int64_t bdB, int64_t bd)
{
    RowInfo r;
    int64_t tr = p / bdA, ia = p % bdA;
    int j[kMaxHalf];
    colex_unrank(tr, dA, nbar, j);
    int64_t div = bdA / b;
    for (int k = 0; k < dA; ++k) {
        int ik = (int)((ia / div) % b);
        r.col[k] = j[k] * b + ik;
        div /= b;
    }
    for (int k = dA; k < kMaxHalf; ++k) r.col[k] = -1;
    r.last = j[dA - 1];
    r.off = tr * bd + ia * bdB;
    return r;
}

struct ColInfo {
    int col[kMaxHalf];
    int first;           // first block index of the tuple
    int64_t off;         // column part of the output address
};

CUM_HD ColInfo decode_col(int64_t q, int dA, int dB, int b, int nbar, int64_t bdB, int64_t bd)
{
    ColInfo c;
    int64_t u = q / bdB, ib = q % bdB;
    int sp[kMaxHalf], s[kMaxHalf];
    colex_unrank(u, dB, nbar, sp);
    for (int k = 0; k < dB; ++k) s[k] = nbar - 1 - sp[dB - 1 - k];
    int64_t rk = 0;
    for (int k = 0; k < dB; ++k) rk += binom(s[k] + dA + k, dA + k + 1);
    int64_t div = bdB / b;
    for (int k = 0; k < dB; ++k) {
        int ik = (int)((ib / div) % b);
        c.col[k] = s[k] * b + ik;
        div /= b;
    }
    for (int k = dB; k < kMaxHalf; ++k) c.col[k] = -1;
    c.first = s[0];
    c.off = rk * bd + ib;
    return c;
}

// fp16 parts: exponent s of the power-of-two scale 2^s applied to a variable of
// X~ whose largest magnitude has float bits `maxbits`, so that the scaled
// maximum lies in [16, 32) and a product of up to three scaled values stays
// below 2^15 (fp16 holds up to 65504).  s is clamped to [-60, 60], which keeps
// the inverse factor of an order-6 entry, 2^-(s_1 + ... + s_6), a normal double.
CUM_HD int fp16_scale_exponent(uint32_t maxbits)
{
    if (maxbits == 0u) return 0;
    const int e = (int)((maxbits >> 23) & 0xffu) - 127;   // floor(log2 max) for a normal max
    int s = 4 - e;
    if (s > 60) s = 60;
    if (s < -60) s = -60;
    return s;
}

// Number of leading columns (in the column order above) whose first block index
// is >= c: C(nbar - c + dB - 1, dB) * b^dB.
CUM_HD int64_t cols_with_first_at_least(int c, int dB, int nbar, int64_t bdB)
{
    return binom((int64_t)nbar - c + dB - 1, dB) * bdB;
}

}  // namespace cum
