// Cumulant correction of one order with the lower-order factors staged in
// shared memory (Eq. cum_r, Alg. 4-5):
//   C_d[j][i] = scale * M_d[j][i] - sum over the set partitions of 1:d into
//               at least two parts, every part of size >= 2, of the product of
//               (C_|part|)[j_part][i_part].
// One CTA per stored block j (grid-stride).  The order d is a template
// parameter, so the partitions (P^(2), Def. 3.5) and the sub-tuple positions of
// every factor are compile-time constants.  The CTA copies, for every subset S
// of 2..d-2 positions, the block of C_|S| with tuple j_S into shared memory;
// each thread owns the in-block digits L..d-1 of its entries and loops over
// the first L digits, so factors over positions >= L stay in registers across
// the loop.  launch_correct uses this kernel when the staged blocks fit in
// shared memory and b^(d-L) threads make a CTA; the general kernel handles the
// rest.
//
// Moment form of order 6.  Group the partitions of 1:6 by the part that holds
// position 0.  Where that part is a pair {0, x}, the other four positions R
// are either one part (C_4[R]) or split into two pairs (three pairings); their
// sum C_4[R] + sum over the pairings of C_2 C_2 is the order-4 moment M_4[R]
// (Eq. cum_r at order 4, the odd orders' singletons having zero mean).  So
//   C_6 = M_6 - sum_x C_2[0x] M_4[R_x] - sum_{pairs P without 0} C_2[P] C_4[rest]
//             - sum_{3+3} C_3 C_3,
// 25 products instead of the 40 partitions.  Given M_4, the staged kernel reads
// the four-position blocks that leave out position 0 from M_4 instead of C_4.
#include "cumgb.h"
#include "internal.h"

namespace cum {

namespace {

constexpr int kMaxSubsets = 64;   // subsets of {0..5}
constexpr int kStageThreads = 256;

template <int D>
struct CorrTables {
    int nsub;                          // subsets with 2..D-2 elements, ascending masks
    uint32_t sub[kMaxSubsets];
    int npart;                         // partitions into >= 2 parts of >= 2 elements
    int nparts[kMaxPartitions];
    int part[kMaxPartitions][kMaxParts];   // subset index of each part
    // Three-part partitions (d = 6: three pairs) come grouped by their first
    // part, the one holding position 0: the kernel sums the products of the
    // other two parts over a group and multiplies by the shared first part
    // once, 20 FP64 operations for the 15 pairings instead of 30.
    bool gfirst[kMaxPartitions], glast[kMaxPartitions];
    // moment form (d = 6): the factor of subset s comes from M_4, not C_4
    bool from_m[kMaxSubsets];
};

constexpr int popcount_c(uint32_t m)
{
    int c = 0;
    for (; m; m &= m - 1u) ++c;
    return c;
}

// All set partitions of 0..D-1 by restricted growth strings (a[0] = 0,
// a[k] <= 1 + max(a[0..k-1])), kept when every part has >= 2 elements and
// there are >= 2 parts.  MOM (order 6 only): the moment form, which keeps the
// two-part partitions and reads the four-position factors without position 0
// from M_4.
template <int D, bool MOM = false>
constexpr CorrTables<D> make_corr_tables()
{
    static_assert(!MOM || D == 6, "the moment form is the order-6 correction");
    CorrTables<D> t{};
    for (uint32_t m = 0; m < (1u << D); ++m) {
        const int c = popcount_c(m);
        if (c >= 2 && c <= D - 2) {
            t.from_m[t.nsub] = MOM && c == D - 2 && !(m & 1u);
            t.sub[t.nsub++] = m;
        }
    }
    int a[D] = {};
    for (;;) {
        uint32_t mask[D] = {};
        int np = 0;
        for (int k = 0; k < D; ++k) {
            mask[a[k]] |= 1u << k;
            if (a[k] + 1 > np) np = a[k] + 1;
        }
        bool ok = np >= 2;
        for (int p = 0; p < np; ++p) ok = ok && popcount_c(mask[p]) >= 2;
        if (ok && t.npart < kMaxPartitions && np <= kMaxParts) {
            t.nparts[t.npart] = np;
            for (int p = 0; p < np; ++p)
                for (int s = 0; s < t.nsub; ++s)
                    if (t.sub[s] == mask[p]) t.part[t.npart][p] = s;
            ++t.npart;
        }
        // next restricted growth string
        int k = D - 1;
        for (; k >= 1; --k) {
            int mx = 0;
            for (int l = 0; l < k; ++l) mx = a[l] > mx ? a[l] : mx;
            if (a[k] <= mx) break;
        }
        if (k < 1) break;
        ++a[k];
        for (int l = k + 1; l < D; ++l) a[l] = 0;
    }
    // two-part partitions first (in generation order), then the three-part ones
    // grouped by their first part (the part holding position 0)
    CorrTables<D> u = t;
    int n = 0;
    for (int z = 0; z < t.npart; ++z)
        if (t.nparts[z] == 2) {
            u.nparts[n] = 2;
            for (int q = 0; q < kMaxParts; ++q) u.part[n][q] = t.part[z][q];
            ++n;
        }
    for (int g = 0; g < t.nsub && !MOM; ++g)
        for (int z = 0; z < t.npart; ++z)
            if (t.nparts[z] == 3 && t.part[z][0] == g) {
                u.nparts[n] = 3;
                for (int q = 0; q < kMaxParts; ++q) u.part[n][q] = t.part[z][q];
                ++n;
            }
    u.npart = n;
    t = u;
    for (int z = 0; z < t.npart; ++z) {
        const bool three = t.nparts[z] == 3;
        t.gfirst[z] = three && (z == 0 || t.nparts[z - 1] != 3 || t.part[z - 1][0] != t.part[z][0]);
        t.glast[z] = three && (z + 1 == t.npart || t.nparts[z + 1] != 3 || t.part[z + 1][0] != t.part[z][0]);
    }
    return t;
}

// every three-part partition of 1:6 is in a group of 3 (the pairings of the
// four positions left by the first pair), 5 groups
constexpr int count_groups6()
{
    constexpr CorrTables<6> t = make_corr_tables<6>();
    int g = 0, n = 0;
    for (int z = 0; z < t.npart; ++z) {
        g += t.gfirst[z] ? 1 : 0;
        n += t.nparts[z] == 3 ? 1 : 0;
    }
    return g * 100 + n;
}
static_assert(count_groups6() == 5 * 100 + 15, "three-pair partitions of 1:6 in 5 groups");

// F(d) - 1 partitions, as counted in Sec. 5.1: 3, 10 and 40 for d = 4, 5, 6.
static_assert(make_corr_tables<4>().npart == 3, "P^(2) of 1:4");
static_assert(make_corr_tables<5>().npart == 10, "P^(2) of 1:5");
static_assert(make_corr_tables<6>().npart == 40, "P^(2) of 1:6");
// moment form: the 15 {2,4} and 10 {3,3} partitions; 5 of the 15 four-position
// subsets (those without position 0) read M_4
static_assert(make_corr_tables<6, true>().npart == 25, "two-part partitions of 1:6");

constexpr int count_from_m6()
{
    constexpr CorrTables<6> t = make_corr_tables<6, true>();
    int c = 0;
    for (int s = 0; s < t.nsub; ++s) c += t.from_m[s] ? 1 : 0;
    return c;
}
static_assert(count_from_m6() == 5, "four-position subsets of 1:6 without position 0");

template <int D, bool MOM = false>
struct Tables {
    static constexpr CorrTables<D> v = make_corr_tables<D, MOM>();
};

// The same tables in constant memory, for runtime-indexed reads.
__constant__ CorrTables<4> c_tab4 = make_corr_tables<4>();
__constant__ CorrTables<5> c_tab5 = make_corr_tables<5>();
__constant__ CorrTables<6> c_tab6 = make_corr_tables<6>();

template <int D>
__device__ __forceinline__ uint32_t subset_mask(int s)
{
    if constexpr (D == 4) return c_tab4.sub[s];
    else if constexpr (D == 5) return c_tab5.sub[s];
    else return c_tab6.sub[s];
}

// Host-built description of the staged blocks (runtime-indexed, so it lives
// in kernel parameters rather than in the compile-time tables).
struct StageLayout {
    int nsub;
    uint32_t mask[kMaxSubsets];   // subset S (bit k = position k)
    int size[kMaxSubsets];        // |S|
    int off[kMaxSubsets];         // first shared-memory element of its block
    int len[kMaxSubsets];         // b^|S|
    int from_m[kMaxSubsets];      // 1: the block comes from M_4 (moment form)
};

// Factor (C_|S|)[j_S][i_S] of subset number S from the staged block; the
// in-block offset takes the digits of the positions in S, first position most
// significant.
template <int D, int S>
__device__ __forceinline__ double staged_factor(const double* stage, const int* soff, int b, const int* dig)
{
    constexpr uint32_t m = Tables<D>::v.sub[S];
    int off = 0;
#pragma unroll
    for (int k = 0; k < D; ++k)
        if ((m >> k) & 1u) off = off * b + dig[k];
    return stage[soff[S] + off];
}

// Partitions Z, Z+1, ... of the table added into `sum` (compile-time recursion,
// so every partition and part index is a constant).
template <int D, bool MOM, int Z>
__device__ __forceinline__ void partition_terms(const double* stage, const int* soff, int b, const int* dig,
                                                double& sum, double& inner)
{
    constexpr CorrTables<D> T = Tables<D, MOM>::v;
    if constexpr (Z < T.npart) {
        const double f0 = staged_factor<D, T.part[Z][0]>(stage, soff, b, dig);
        const double f1 = staged_factor<D, T.part[Z][1]>(stage, soff, b, dig);
        if constexpr (T.nparts[Z] == 2) {
            sum = fma(f0, f1, sum);
        } else {
            const double f2 = staged_factor<D, T.part[Z][2]>(stage, soff, b, dig);
            if constexpr (T.gfirst[Z])
                inner = f1 * f2;
            else
                inner = fma(f1, f2, inner);
            if constexpr (T.glast[Z]) sum = fma(f0, inner, sum);
        }
        partition_terms<D, MOM, Z + 1>(stage, soff, b, dig, sum, inner);
    }
}

template <int D, int L, bool MOM>
__global__ void __launch_bounds__(kStageThreads) correct_staged_kernel(int b, int nbar, int64_t bd, int64_t nblocks,
                                                                        const double* __restrict__ M, double scale,
                                                                        LowerPtrs low, StageLayout lay,
                                                                        double* __restrict__ C)
{
    extern __shared__ double stage[];
    __shared__ int64_t src_off[kMaxSubsets];
    __shared__ int soff[kMaxSubsets];
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;   // b^(D-L)
    for (int s = tid; s < lay.nsub; s += nthr) soff[s] = lay.off[s];   // ordered by the block loop's barriers
    int dig[D];
    {
        int rem = tid;
#pragma unroll
        for (int k = D - 1; k >= L; --k) {
            dig[k] = rem % b;
            rem /= b;
        }
    }
    int nouter = 1;
#pragma unroll
    for (int k = 0; k < L; ++k) nouter *= b;

    for (int64_t r = blockIdx.x; r < nblocks; r += gridDim.x) {
        int j[D];
        colex_unrank(r, D, nbar, j);
        __syncthreads();   // the previous block's readers are done with the stage
        for (int s = tid; s < lay.nsub; s += nthr) {
            int js[D];
            int len = 0;
            for (int k = 0; k < D; ++k)
                if ((lay.mask[s] >> k) & 1u) js[len++] = j[k];
            src_off[s] = colex_rank(js, len) * (int64_t)lay.len[s];
        }
        __syncthreads();
        for (int s = 0; s < lay.nsub; ++s) {
            const double* src = (MOM && lay.from_m[s] ? low.m4 : low.c[lay.size[s]]) + src_off[s];
            double* dst = stage + lay.off[s];
            for (int x = tid; x < lay.len[s]; x += nthr) dst[x] = src[x];
        }
        __syncthreads();
        const int64_t base = r * bd;
        for (int h = 0; h < nouter; ++h) {
            {
                int rem = h;
#pragma unroll
                for (int k = L - 1; k >= 0; --k) {
                    dig[k] = rem % b;
                    rem /= b;
                }
            }
            double sum = 0.0, inner = 0.0;
            partition_terms<D, MOM, 0>(stage, soff, b, dig, sum, inner);
            const int64_t e = base + (int64_t)h * nthr + tid;
            C[e] = M[e] * scale - sum;
        }
    }
}

template <int D, int L, bool MOM>
cudaError_t launch_staged(int b, int nbar, int64_t nblocks, const double* M, double scale, const LowerPtrs& low,
                          const StageLayout& lay, size_t smem, int threads, double* C, cudaStream_t st)
{
    auto kern = correct_staged_kernel<D, L, MOM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // a few CTAs per SM, each walking many blocks
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t cap = (int64_t)sms * 8;
    const int64_t grid = nblocks < cap ? nblocks : cap;
    kern<<<(unsigned)grid, threads, smem, st>>>(b, nbar, ipow(b, D), nblocks, M, scale, low, lay, C);
    return cudaGetLastError();
}

template <int D, bool MOM>
bool staged_plan(int b, StageLayout* lay, size_t* smem, int* L, int* threads)
{
    constexpr CorrTables<D> T = make_corr_tables<D, MOM>();
    int64_t total = 0;
    lay->nsub = T.nsub;
    for (int s = 0; s < T.nsub; ++s) {
        const int64_t n = ipow(b, popcount_c(T.sub[s]));
        lay->from_m[s] = T.from_m[s] ? 1 : 0;
        lay->mask[s] = T.sub[s];
        lay->size[s] = popcount_c(T.sub[s]);
        lay->off[s] = (int)total;
        lay->len[s] = (int)n;
        total += n;
    }
    *smem = (size_t)total * sizeof(double);
    if (*smem > (size_t)160 * 1024) return false;
    // fewest looped leading digits that keep the CTA within kStageThreads
    for (int l = 0; l <= 3 && l < D; ++l) {
        const int64_t n = ipow(b, D - l);
        if (n <= kStageThreads) {
            if (n < 32) return false;   // too few threads per CTA
            *L = l;
            *threads = (int)n;
            return true;
        }
    }
    return false;
}

template <int D, bool MOM = false>
cudaError_t try_staged(int b, int nbar, const double* M, double scale, const LowerPtrs& low, double* C,
                       cudaStream_t st, bool* done)
{
    StageLayout lay{};
    size_t smem = 0;
    int L = 0, threads = 0;
    *done = false;
    if (!staged_plan<D, MOM>(b, &lay, &smem, &L, &threads)) return cudaSuccess;
    *done = true;
    const int64_t nblocks = num_blocks(nbar, D);
    switch (L) {
    case 0: return launch_staged<D, 0, MOM>(b, nbar, nblocks, M, scale, low, lay, smem, threads, C, st);
    case 1: return launch_staged<D, 1, MOM>(b, nbar, nblocks, M, scale, low, lay, smem, threads, C, st);
    case 2: return launch_staged<D, 2, MOM>(b, nbar, nblocks, M, scale, low, lay, smem, threads, C, st);
    default: return launch_staged<D, 3, MOM>(b, nbar, nblocks, M, scale, low, lay, smem, threads, C, st);
    }
}

// Batched form: one CTA per (dataset, stored block), found by the prefix of
// the descriptors' block counts; the staging layout follows the dataset's b.
template <int D>
__global__ void __launch_bounds__(kStageThreads) batch_correct_staged_kernel(const BatchCorr* __restrict__ cr,
                                                                              int count)
{
    constexpr int NSUB = Tables<D>::v.nsub;
    extern __shared__ double stage[];
    __shared__ int soff[kMaxSubsets];
    __shared__ int64_t src_off[kMaxSubsets];
    const int64_t i = find_segment(&cr[0].block_base, count, sizeof(BatchCorr), blockIdx.x);
    const BatchCorr& K = cr[i];
    const int64_t r = blockIdx.x - K.block_base;
    const int b = K.b;
    const int tid = threadIdx.x, nthr = blockDim.x;
    int j[D];
    colex_unrank(r, D, K.nbar, j);
    if (tid == 0) {
        int tot = 0;
        for (int s = 0; s < NSUB; ++s) {
            soff[s] = tot;
            tot += (int)ipow(b, popcount_c(subset_mask<D>(s)));
        }
    }
    for (int s = tid; s < NSUB; s += nthr) {
        const uint32_t m = subset_mask<D>(s);
        int js[D];
        int len = 0;
        for (int k = 0; k < D; ++k)
            if ((m >> k) & 1u) js[len++] = j[k];
        src_off[s] = colex_rank(js, len) * ipow(b, len);
    }
    __syncthreads();
    for (int s = 0; s < NSUB; ++s) {
        const int len = popcount_c(subset_mask<D>(s));
        const int n = (int)ipow(b, len);
        const double* src = K.low[len] + src_off[s];
        for (int x = tid; x < n; x += nthr) stage[soff[s] + x] = src[x];
    }
    __syncthreads();
    double* C = K.C + r * K.bd;
    const double* M = (K.M ? K.M : K.C) + r * K.bd;
    for (int64_t e = tid; e < K.bd; e += nthr) {
        int dig[D];
        int rem = (int)e;
#pragma unroll
        for (int k = D - 1; k >= 0; --k) {
            dig[k] = rem % b;
            rem /= b;
        }
        double sum = 0.0, inner = 0.0;
        partition_terms<D, false, 0>(stage, soff, b, dig, sum, inner);
        C[e] = M[e] - sum;
    }
}

template <int D>
cudaError_t try_batch_staged(const BatchCorr* dev, const BatchCorr* host, int count, int64_t blocks,
                             cudaStream_t st, bool* done)
{
    constexpr CorrTables<D> T = make_corr_tables<D>();
    size_t smem = 0;
    for (int i = 0; i < count; ++i) {
        int64_t total = 0;
        for (int s = 0; s < T.nsub; ++s) total += ipow(host[i].b, popcount_c(T.sub[s]));
        const size_t bytes = (size_t)total * sizeof(double);
        smem = bytes > smem ? bytes : smem;
    }
    *done = false;
    if (smem > (size_t)160 * 1024) return cudaSuccess;
    *done = true;
    if (blocks <= 0) return cudaSuccess;
    auto kern = batch_correct_staged_kernel<D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)blocks, kStageThreads, smem, st>>>(dev, count);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batch_correct_staged(int d, const BatchCorr* dev, const BatchCorr* host, int count,
                                        int64_t blocks, cudaStream_t st, bool* done)
{
    *done = false;
    if (d == 4) return try_batch_staged<4>(dev, host, count, blocks, st, done);
    if (d == 5) return try_batch_staged<5>(dev, host, count, blocks, st, done);
    if (d == 6) return try_batch_staged<6>(dev, host, count, blocks, st, done);
    return cudaSuccess;
}

cudaError_t launch_correct_staged(int d, int b, int nbar, const double* M, double scale, const LowerPtrs& low,
                                  double* C, cudaStream_t st, bool* done)
{
    *done = false;
    if (d == 4) return try_staged<4>(b, nbar, M, scale, low, C, st, done);
    if (d == 5) return try_staged<5>(b, nbar, M, scale, low, C, st, done);
    if (d == 6 && low.m4) return try_staged<6, true>(b, nbar, M, scale, low, C, st, done);
    if (d == 6) return try_staged<6>(b, nbar, M, scale, low, C, st, done);
    return cudaSuccess;
}

}  // namespace cum
