// Host check of the single-dataset workspace layout (layout_ws in csrc/api.cu),
// linked against the built library: every region starts on a 256-byte
// boundary, the regions follow one another without overlap, each is at least
// as large as what its users read or write (X~ transposed and, for the split
// precisions, its FP32 remainder; the stored column sums of X~; the row-tile
// prefix, the split partials of every order's plan, the per-CTA scratch tiles,
// the fp16 scale tables, the kept order-4 moments and the order d_max - 1
// moments the residual-mean shift reads), the total is what
// cum_workspace_size reports, and every region that centring writes (status,
// sums and mean, fp16 scale tables, column sums, X~ and its remainder) sits
// at the same offset whatever d_max the workspace was laid out for --
// cum_center lays it out for d_max = 2 and cum_moment_blocks for its own
// order.  Exits 0 when every case holds.
#include <cstdio>

#include "cumgb.h"
#include "internal.h"

using namespace cum;

static int check(int64_t t, int n, int d_max, int b, int prec)
{
    WsLayout L;
    if (!layout_ws(t, n, d_max, b, prec, &L)) return 0;   // unsupported sizes: nothing to check
    int bad = 0;
    const bool tc = prec != CUM_PREC_FP64;
    const int nbar = (n + b - 1) / b;
    int64_t max_rt = 0, max_part = 0;
    for (int d = 2; d <= d_max; ++d) {
        const OrderPlan P = make_order_plan(d, t, n, b, prec);
        if (P.row_tiles > max_rt) max_rt = P.row_tiles;
        if (P.splits > 1 && P.splits * P.sh.entries > max_part) max_part = P.splits * P.sh.entries;
        if (P.kchunk * P.splits < L.t_pad || P.kchunk * (P.splits - 1) >= L.t_pad) ++bad;   // chunks cover t once
    }
    const size_t off[] = {L.status, L.colsum,  L.maxabs,  L.vexp, L.rsum, L.xt,
                          L.xlo,    L.prefix, L.partial, L.scratch, L.m4, L.mlow, L.total};
    const size_t need[] = {
        64,
        sizeof(double) * ((size_t)kColsumChunks * L.n_pad + 2 * (size_t)L.n_pad),
        sizeof(uint32_t) * (size_t)L.n_pad,
        sizeof(int32_t) * (size_t)L.n_pad,
        sizeof(double) * ((size_t)L.n_pad + 1),
        L.xt_elem * (size_t)L.n_pad * (size_t)L.t_pad,
        tc ? sizeof(float) * (size_t)L.n_pad * (size_t)L.t_pad : 0,
        sizeof(int64_t) * (size_t)(max_rt + 1),
        sizeof(double) * (size_t)max_part,
        tc ? sizeof(double) * kTcScratchDoubles : 0,
        d_max >= 6 || (tc && d_max >= 5) ? sizeof(double) * (size_t)(num_blocks(nbar, 4) * ipow(b, 4)) : 0,
        tc && d_max >= 3 ? sizeof(double) * (size_t)(num_blocks(nbar, d_max - 1) * ipow(b, d_max - 1)) : 0,
    };
    const int nreg = (int)(sizeof(need) / sizeof(need[0]));
    for (int i = 0; i < nreg; ++i) {
        if (off[i] % kWsAlign) ++bad;
        if (off[i + 1] < off[i] + need[i]) ++bad;
    }
    if (L.t_pad < t || L.t_pad % kTAlign || L.n_pad != nbar * b) ++bad;
    if (cum_workspace_size(t, n, d_max, b, prec) != L.total) ++bad;
    // the regions centring writes, against the layout cum_center uses (d_max = 2)
    WsLayout C;
    if (!layout_ws(t, n, 2, b, prec, &C)) ++bad;
    else if (C.status != L.status || C.colsum != L.colsum || C.maxabs != L.maxabs || C.vexp != L.vexp ||
             C.rsum != L.rsum || C.xt != L.xt || C.xlo != L.xlo || C.t_pad != L.t_pad || C.n_pad != L.n_pad ||
             C.xt_elem != L.xt_elem)
        ++bad;
    if (bad) std::printf("t=%lld n=%d d_max=%d b=%d prec=%d: %d failures\n", (long long)t, n, d_max, b, prec, bad);
    return bad;
}

int main()
{
    int bad = 0, cases = 0;
    const int64_t ts[] = {1, 127, 129, 2000, 100000, 200000, 1000003};
    const int ns[] = {1, 5, 20, 48, 60, 128, 256};
    const int bs[] = {1, 2, 3, 4, 6, 16};
    for (int prec = 0; prec <= 3; ++prec)
        for (int64_t t : ts)
            for (int n : ns)
                for (int b : bs)
                    for (int d_max = 2; d_max <= 6; ++d_max) {
                        if (n > 64 && d_max > 4) continue;   // keeps the case count small
                        bad += check(t, n, d_max, b, prec);
                        ++cases;
                    }
    std::printf("%d layouts checked, %d failures\n", cases, bad);
    return bad ? 1 : 0;
}
