/*
 * Plain FP64 reference for single entries of moment and cumulant tensors.
 * TEST INFRASTRUCTURE ONLY: called from the tests and from bench.py's CPU
 * baseline, never from the library.  Shares no code with the GPU path.
 *
 * For one multi-index i = (i_1..i_d):
 *   - every subset moment m_{i_B} = (1/t) sum_l prod_{k in B} x~_{l, i_k}
 *     for the 2^d - 1 non-empty subsets B of positions (Def. 1.2, Eq. d::moment),
 *     each summed directly over l;
 *   - the cumulant by the moment-to-cumulant formula over all set partitions
 *     zeta of 1:d (Eq. cumfmom, Sec. 5.3):
 *         c_i = sum_zeta (|zeta|-1)! (-1)^(|zeta|-1) prod_{B in zeta} m_{i_B}.
 * Set partitions are enumerated by restricted growth strings.
 *
 * Xc: centred data, row-major t x n with row stride ldx (doubles).
 * idx: count x d multi-indices (int32, 0-based).  out: count doubles.
 * threads: OpenMP threads (0 = runtime default).  Returns 0, or -1 on bad args.
 */
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXD 8

static double subset_moment(const double* Xc, int64_t t, int64_t ldx, const int32_t* ix, int d, unsigned mask)
{
    int cols[MAXD];
    int nc = 0;
    for (int k = 0; k < d; ++k)
        if (mask & (1u << k)) cols[nc++] = ix[k];
    double s = 0.0;
    for (int64_t l = 0; l < t; ++l) {
        const double* row = Xc + l * ldx;
        double p = 1.0;
        for (int k = 0; k < nc; ++k) p *= row[cols[k]];
        s += p;
    }
    return s / (double)t;
}

static double factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

/* Sum over all set partitions of {0..d-1} via restricted growth strings. */
static double ls_sum(const double* m /* indexed by mask */, int d)
{
    int a[MAXD];
    int mx[MAXD];
    double total = 0.0;
    for (int k = 0; k < d; ++k) { a[k] = 0; mx[k] = 0; }
    for (;;) {
        /* evaluate the partition encoded by a[] */
        unsigned blocks[MAXD];
        int nb = 0;
        for (int k = 0; k < d; ++k) if (a[k] + 1 > nb) nb = a[k] + 1;
        for (int b = 0; b < nb; ++b) blocks[b] = 0u;
        for (int k = 0; k < d; ++k) blocks[a[k]] |= 1u << k;
        double term = factorial(nb - 1) * ((nb - 1) % 2 ? -1.0 : 1.0);
        for (int b = 0; b < nb; ++b) term *= m[blocks[b]];
        total += term;
        /* next restricted growth string: a[0] = 0 always */
        int k = d - 1;
        while (k > 0 && a[k] == mx[k - 1] + 1) --k;
        if (k == 0) break;
        a[k] += 1;
        mx[k] = a[k] > mx[k - 1] ? a[k] : mx[k - 1];
        for (int j = k + 1; j < d; ++j) { a[j] = 0; mx[j] = mx[k]; }
    }
    return total;
}

static int check(const double* Xc, int64_t t, int n, int64_t ldx, int d, int64_t count,
                 const int32_t* idx, const double* out)
{
    if (!Xc || !idx || !out || t <= 0 || n <= 0 || ldx < n || d < 1 || d > MAXD || count < 0) return -1;
    for (int64_t e = 0; e < count * d; ++e)
        if (idx[e] < 0 || idx[e] >= n) return -1;
    return 0;
}

int oracle_cumulant_entries(const double* Xc, int64_t t, int n, int64_t ldx, int d, int64_t count,
                            const int32_t* idx, double* out, int threads)
{
    if (check(Xc, t, n, ldx, d, count, idx, out)) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t e = 0; e < count; ++e) {
        double m[1u << MAXD];
        const int32_t* ix = idx + e * d;
        m[0] = 1.0;
        for (unsigned mask = 1; mask < (1u << d); ++mask)
            m[mask] = subset_moment(Xc, t, ldx, ix, d, mask);
        out[e] = ls_sum(m, d);
    }
    return 0;
}

int oracle_moment_entries(const double* Xc, int64_t t, int n, int64_t ldx, int d, int64_t count,
                          const int32_t* idx, double* out, int threads)
{
    if (check(Xc, t, n, ldx, d, count, idx, out)) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t e = 0; e < count; ++e)
        out[e] = subset_moment(Xc, t, ldx, idx + e * d, d, (1u << d) - 1u);
    return 0;
}
