// Host check of the moment contraction's index mapping (common.cuh): for every
// row p (sorted dA-tuple x in-block digits) and column q (sorted dB-tuple x
// in-block digits) with last(p) <= first(q), the output address
// rowOff(p) + colOff(q) must be the storage address of the entry of variables
// (col(p), col(q)): the colex rank of the sorted block tuple times b^d plus the
// C-order in-block offset (Sec. 2.1).  Every stored entry must be hit exactly
// once, and the tile staircase count must equal a brute-force count of tiles
// holding a valid pair.  With tile 256 (the CTA-pair kernel) it also checks that
// the pair's assignment of B rows -- CTA c, local row r -> column 64 c + r --
// covers the tile's 128 columns once and puts accumulator column j at tile
// column j (the N = 128 MMA takes CTA 0's 64 rows first).
// Usage: mapping_check d n b [tile]; exits 0 when all hold.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "common.cuh"

using namespace cum;

int main(int argc, char** argv)
{
    if (argc != 4 && argc != 5) return 2;
    const int d = atoi(argv[1]), n = atoi(argv[2]), b = atoi(argv[3]);
    const Shape sh = make_shape(d, n, b);
    std::vector<unsigned char> hit((size_t)sh.entries, 0);
    // square tiles of side `tile`, or with `tile` 256 the pair kernel's 256 x 128
    const int64_t tile = argc == 5 ? atoi(argv[4]) : 128;
    int pair_bad = 0;
    const int64_t tile_m = tile, tile_n = tile == 256 ? 128 : tile;
    if (tile == 256) {
        std::vector<int> seen(128, 0);
        for (int c = 0; c < 2; ++c)
            for (int r = 0; r < 64; ++r) {
                const int q = c * 64 + r;          // the kernel's B row -> tile column
                ++seen[q];
                const int acc_col = c * 64 + r;    // N = 128: CTA 0's rows first
                if (acc_col != q) ++pair_bad;
            }
        for (int v : seen)
            if (v != 1) ++pair_bad;
    }
    const int64_t row_tiles = (sh.rows + tile_m - 1) / tile_m, col_tiles = (sh.cols + tile_n - 1) / tile_n;
    std::vector<unsigned char> tile_live((size_t)(row_tiles * col_tiles), 0);
    int bad = 0;
    for (int64_t p = 0; p < sh.rows; ++p) {
        const RowInfo r = decode_row(p, sh.dA, sh.dB, b, sh.nbar, sh.bdA, sh.bdB, sh.bd);
        for (int64_t q = 0; q < sh.cols; ++q) {
            const ColInfo c = decode_col(q, sh.dA, sh.dB, b, sh.nbar, sh.bdB, sh.bd);
            if (r.last > c.first) continue;
            tile_live[(size_t)((p / tile_m) * col_tiles + q / tile_n)] = 1;
            const int64_t addr = r.off + c.off;
            // the entry's variables, in row-then-column order
            int v[kMaxOrder], blk[kMaxOrder];
            for (int k = 0; k < sh.dA; ++k) v[k] = r.col[k];
            for (int k = 0; k < sh.dB; ++k) v[sh.dA + k] = c.col[k];
            for (int k = 0; k < d; ++k) blk[k] = v[k] / b;
            for (int k = 1; k < d; ++k)
                if (blk[k] < blk[k - 1]) ++bad;   // block tuple must be sorted
            int64_t off = 0;
            for (int k = 0; k < d; ++k) off = off * b + v[k] % b;
            const int64_t want = colex_rank(blk, d) * sh.bd + off;
            if (addr != want || addr < 0 || addr >= sh.entries) {
                if (bad < 5) std::printf("p=%lld q=%lld addr=%lld want=%lld\n", (long long)p, (long long)q,
                                         (long long)addr, (long long)want);
                ++bad;
                continue;
            }
            if (hit[(size_t)addr]++) ++bad;
        }
    }
    int64_t missed = 0;
    for (unsigned char h : hit) missed += h == 0;
    // staircase: per row tile, the active column tiles are the leading ones
    // holding a column whose first block is >= the tile's first row's last block
    int64_t active = 0, live = 0;
    for (int64_t I = 0; I < row_tiles; ++I) {
        int j[kMaxHalf];
        colex_unrank((I * tile_m) / sh.bdA, sh.dA, sh.nbar, j);
        const int64_t cols = cols_with_first_at_least(j[sh.dA - 1], sh.dB, sh.nbar, sh.bdB);
        active += (cols + tile_n - 1) / tile_n;
        for (int64_t J = 0; J < col_tiles; ++J) {
            const bool in_stair = J < (cols + tile_n - 1) / tile_n;
            if (tile_live[(size_t)(I * col_tiles + J)] && !in_stair) ++bad;   // a live tile left out
            live += tile_live[(size_t)(I * col_tiles + J)];
        }
    }
    std::printf("d=%d n=%d b=%d entries=%lld missed=%lld bad=%d active=%lld live=%lld\n", d, n, b,
                (long long)sh.entries, (long long)missed, bad, (long long)active, (long long)live);
    if (pair_bad) std::printf("pair assignment: %d failures\n", pair_bad);
    return (bad == 0 && missed == 0 && pair_bad == 0) ? 0 : 1;
}
