// Host check of the correction kernel's compile-time partition tables
// (csrc/correct.cu): for orders 4-6, evaluating the tables the way the staged
// kernel does (two-part products, three-pair groups summed inside, the
// order-6 moment form reading M_4) must equal a direct sum over the set
// partitions of 1:d into >= 2 parts of size >= 2 (Eq. cum_r), enumerated here
// independently, on random symmetric lower-order tensors.  Exits 0 when all
// orders and forms agree to rounding.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "correct.cu"

using namespace cum;

namespace {

const int B = 3;   // in-block digits per position

struct Sym {
    std::vector<double> v[7];   // v[k]: a symmetric b^k table
};

double at(const std::vector<double>& v, const int* dig, uint32_t mask, int d)
{
    size_t off = 0;
    for (int q = 0; q < d; ++q)
        if ((mask >> q) & 1u) off = off * B + dig[q];
    return v[off];
}

// all partitions of the positions in `rest` into parts of size >= 2
void parts(uint32_t rest, std::vector<uint32_t>& cur, std::vector<std::vector<uint32_t>>& out)
{
    if (!rest) {
        out.push_back(cur);
        return;
    }
    const uint32_t low = rest & (0u - rest);
    const uint32_t others = rest & ~low;
    for (uint32_t sub = others;; sub = (sub - 1) & others) {
        const uint32_t p = low | sub;
        if (__builtin_popcount(p) >= 2) {
            cur.push_back(p);
            parts(rest & ~p, cur, out);
            cur.pop_back();
        }
        if (!sub) break;
    }
}

template <int D, bool MOM>
double table_sum(const Sym& C, const std::vector<double>& M4, const int* dig)
{
    constexpr CorrTables<D> T = make_corr_tables<D, MOM>();
    auto factor = [&](int s) {
        const uint32_t m = T.sub[s];
        const int k = __builtin_popcount(m);
        return at(T.from_m[s] ? M4 : C.v[k], dig, m, D);
    };
    double sum = 0.0, inner = 0.0;
    for (int z = 0; z < T.npart; ++z) {
        const double f0 = factor(T.part[z][0]), f1 = factor(T.part[z][1]);
        if (T.nparts[z] == 2) {
            sum += f0 * f1;
        } else {
            const double f2 = factor(T.part[z][2]);
            inner = T.gfirst[z] ? f1 * f2 : inner + f1 * f2;
            if (T.glast[z]) sum += f0 * inner;
        }
    }
    return sum;
}

template <int D>
int check(const Sym& C, const std::vector<double>& M4)
{
    std::vector<std::vector<uint32_t>> all;
    std::vector<uint32_t> cur;
    parts((1u << D) - 1u, cur, all);
    int nz = 0;
    for (auto& z : all) nz += z.size() >= 2;
    int bad = nz == make_corr_tables<D>().npart ? 0 : 1;
    double maxd = 0.0, maxv = 0.0;
    int n = 1;
    for (int q = 0; q < D; ++q) n *= B;
    for (int e = 0; e < n; ++e) {
        int dig[D];
        for (int q = D - 1, r = e; q >= 0; --q, r /= B) dig[q] = r % B;
        double direct = 0.0;
        for (auto& z : all) {
            if (z.size() < 2) continue;
            double p = 1.0;
            for (uint32_t m : z) p *= at(C.v[__builtin_popcount(m)], dig, m, D);
            direct += p;
        }
        double a = table_sum<D, false>(C, M4, dig);
        maxd = std::fmax(maxd, std::fabs(a - direct));
        if constexpr (D == 6) maxd = std::fmax(maxd, std::fabs(table_sum<6, true>(C, M4, dig) - direct));
        maxv = std::fmax(maxv, std::fabs(direct));
    }
    if (maxd > 1e-12 * maxv) bad = 1;
    std::printf("d=%d partitions=%d max|diff|=%.3e of %.3e\n", D, nz, maxd, maxv);
    return bad;
}

}  // namespace

int main()
{
    std::mt19937_64 rng(7);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    Sym C;
    for (int k = 2; k <= 4; ++k) {
        size_t n = 1;
        for (int q = 0; q < k; ++q) n *= B;
        std::vector<double> raw(n);
        for (auto& x : raw) x = U(rng);
        C.v[k].resize(n);
        for (size_t i = 0; i < n; ++i) {   // symmetrise: value of the sorted digits
            int dig[4];
            size_t r = i;
            for (int q = k - 1; q >= 0; --q, r /= B) dig[q] = (int)(r % B);
            std::sort(dig, dig + k);
            size_t j = 0;
            for (int q = 0; q < k; ++q) j = j * B + dig[q];
            C.v[k][i] = raw[j];
        }
    }
    // M_4 = C_4 + the three pairings of C_2 C_2 (Eq. cum_r at order 4)
    std::vector<double> M4(C.v[4].size());
    for (size_t i = 0; i < M4.size(); ++i) {
        int g[4];
        size_t r = i;
        for (int q = 3; q >= 0; --q, r /= B) g[q] = (int)(r % B);
        auto c2 = [&](int x, int y) { return C.v[2][g[x] * B + g[y]]; };
        M4[i] = C.v[4][i] + c2(0, 1) * c2(2, 3) + c2(0, 2) * c2(1, 3) + c2(0, 3) * c2(1, 2);
    }
    int bad = check<4>(C, M4) + check<5>(C, M4) + check<6>(C, M4);
    return bad ? 1 : 0;
}
