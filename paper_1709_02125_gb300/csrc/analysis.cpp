// Dependency analysis and tile planning of a queued loop chain (host only).
//
// arXiv 1709.02125, Sec. 3: loops of a chain are delayed; a dependency analysis
// computes a skewed tiling schedule so that all data a tile uses stays in fast
// memory for the whole tile. Sec. 4: the footprint of a tile, its overlap with the
// neighbouring tiles ("left/right edge", "left/right footprint"), and which data
// is uploaded / downloaded; Sec. 4.1: read-only data is not downloaded, write-first
// data is not uploaded, and with the cyclic option write-first data is not
// downloaded either.
//
// Tiling is along the slowest axis only (y in 2-D, z in 3-D). Loop i runs slow rows
// [s_i(t), e_i(t)) in tile t; consecutive tiles of one loop partition its range.
// The ends e_i(t) are computed by a backward sweep over the loops of the tile:
//   RAW  a later reader j of D needs rows up to e_j + rmax_j(D) written first,
//   WAR  a later writer j of D may not overwrite rows that loop i still reads in a
//        later tile (those start at e_i(t) + rmin_i(D)), and
//   WAW  a later writer's rows may not be overwritten later by an earlier writer,
// which gives e_i >= max(b_t, RE[D] for D written, WE[D] for D written,
// WE[D] - rmin_i(D) for D read), clipped to the loop's range, where RE / WE are the
// maxima of e_j + rmax_j(D) over later readers and of e_j over later writers in the
// same tile, and b_t is the nominal boundary of tile t. Every point is computed
// exactly once, from the same inputs as in program order.
//
// Device residency: each dataset gets a cyclic slab of S rows (row y at slot
// (y - y0) mod S) instead of the paper's three slots plus edge copy, so the overlap
// between consecutive tiles never moves. S is the largest span of rows that are
// live in one pipeline phase (see the phase rule in runtime.cu).
#include <algorithm>
#include <climits>
#include <cstring>

#include "../../include/oc.h"
#include "oc_internal.h"

namespace oc {

long long align_up(long long v, long long a) { return (v + a - 1) / a * a; }

static inline uint64_t mix(uint64_t h, uint64_t v)
{
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    return h * 0x100000001b3ull;
}

uint64_t chain_signature(const std::vector<Loop>& loops, const std::vector<Dat>& dats,
                         uint32_t flags)
{
    uint64_t h = 1469598103934665603ull;
    h = mix(h, flags & (OC_FLAG_CYCLIC | OC_FLAG_PREFETCH));
    for (const Loop& lp : loops) {
        h = mix(h, (uint64_t)lp.kernel);
        h = mix(h, lp.params.size());
        for (int a = 0; a < 3; ++a) { h = mix(h, (uint64_t)(uint32_t)lp.lo[a]); h = mix(h, (uint64_t)(uint32_t)lp.hi[a]); }
        for (const Arg& ar : lp.args) {
            h = mix(h, (uint64_t)ar.dat * 16 + ar.access);
            if (ar.access != OC_REDUCE) {
                const Dat& d = dats[ar.dat];
                h = mix(h, (uint64_t)d.dtype * 1315423911ull + (uint64_t)d.nrows);
            }
            for (auto& o : ar.off)
                h = mix(h, ((uint64_t)(uint16_t)o[0]) | ((uint64_t)(uint16_t)o[1] << 16) | ((uint64_t)(uint16_t)o[2] << 32));
        }
    }
    return h;
}

bool full_row_write(const Loop& lp, const Dat& d)
{
    // A write covers whole slow rows if its range spans the full allocated extent of
    // every non-slow axis (halo included), so no old value of the row survives.
    for (int a = 0; a < d.ndim - 1; ++a)
        if (lp.lo[a] > -d.hlo[a] || lp.hi[a] < d.size[a] + d.hhi[a]) return false;
    return true;
}

static inline bool is_read(int acc) { return acc == OC_READ || acc == OC_RW; }
static inline bool is_write(int acc) { return acc == OC_WRITE || acc == OC_RW; }

bool build_plan(const std::vector<Loop>& loops, const std::vector<Dat>& dats,
                const std::vector<int>& red_ops, int h, int depth, uint32_t flags,
                bool incore, Plan& P, std::string& err, const Residency* res)
{
    if (incore || (res && !res->any())) res = nullptr;
    P = Plan();
    const int L = (int)loops.size();
    P.L = L;
    P.depth = depth;
    const int k = depth - 2;  // upload lookahead in tiles
    if (L == 0) { P.valid = true; P.T = 0; return true; }
    const int nd = loops[0].ndim;
    const int sa = nd - 1;

    // datasets used, in first-use order
    P.dat_index.assign(dats.size(), -1);
    for (const Loop& lp : loops)
        for (const Arg& ar : lp.args)
            if (ar.access != OC_REDUCE && P.dat_index[ar.dat] < 0) {
                P.dat_index[ar.dat] = (int)P.dp.size();
                DatPlan dp;
                dp.dat = ar.dat;
                dp.y0 = dats[ar.dat].y0;
                dp.nrows = dats[ar.dat].nrows;
                P.dp.push_back(dp);
            }
    const int ND = (int)P.dp.size();

    int Y0 = INT_MAX, Y1 = INT_MIN;
    for (const Loop& lp : loops) { Y0 = std::min(Y0, lp.lo[sa]); Y1 = std::max(Y1, lp.hi[sa]); }
    P.Y0 = Y0; P.Y1 = Y1;
    const int span = std::max(1, Y1 - Y0);
    if (h <= 0 || incore) h = span;
    P.h = h;
    const int T = (span + h - 1) / h;
    P.T = T;
    P.incore = incore;
    P.se.assign((size_t)T * L * 2, 0);

    // ---- skewed tiling: backward sweep per tile ------------------------------
    std::vector<int> eprev(L);
    for (int i = 0; i < L; ++i) eprev[i] = std::min(loops[i].lo[sa], loops[i].hi[sa]);
    const long long NEG = LLONG_MIN / 4;
    std::vector<long long> RE(ND), WE(ND);
    for (int t = 0; t < T; ++t) {
        std::fill(RE.begin(), RE.end(), NEG);
        std::fill(WE.begin(), WE.end(), NEG);
        const long long b = (t == T - 1) ? (long long)INT_MAX : (long long)Y0 + (long long)(t + 1) * h;
        for (int i = L - 1; i >= 0; --i) {
            const Loop& lp = loops[i];
            long long e = b;
            for (const Arg& ar : lp.args) {
                if (ar.access == OC_REDUCE) continue;
                int d = P.dat_index[ar.dat];
                if (is_write(ar.access)) e = std::max(e, std::max(RE[d], WE[d]));
                if (is_read(ar.access) && WE[d] > NEG) e = std::max(e, WE[d] - ar.rmin[sa]);
            }
            e = std::max(e, (long long)eprev[i]);
            const int lo = std::min(lp.lo[sa], lp.hi[sa]), hi = lp.hi[sa];
            e = std::min(std::max(e, (long long)lo), (long long)hi);
            if (t == T - 1) e = hi;
            P.se[((size_t)t * L + i) * 2] = eprev[i];
            P.se[((size_t)t * L + i) * 2 + 1] = (int)e;
            eprev[i] = (int)e;
            for (const Arg& ar : lp.args) {
                if (ar.access == OC_REDUCE) continue;
                int d = P.dat_index[ar.dat];
                if (is_read(ar.access)) RE[d] = std::max(RE[d], e + ar.rmax[sa]);
                if (is_write(ar.access)) WE[d] = std::max(WE[d], e);
            }
        }
    }

    // ---- per-row first/last tile, upload and download need ----------------------
    for (int d = 0; d < ND; ++d) {
        DatPlan& dp = P.dp[d];
        dp.first.assign(dp.nrows, -1);
        dp.last.assign(dp.nrows, -1);
        dp.need_up.assign(dp.nrows, 0);
        dp.dl.assign(dp.nrows, 0);
    }
    auto mark = [&](DatPlan& dp, int t, long long a, long long b) {
        a = std::max<long long>(a, dp.y0);
        b = std::min<long long>(b, (long long)dp.y0 + dp.nrows);
        for (long long y = a; y < b; ++y) {
            int r = (int)(y - dp.y0);
            if (dp.first[r] < 0) dp.first[r] = t;
            dp.last[r] = t;
        }
    };
    for (int t = 0; t < T; ++t)
        for (int i = 0; i < L; ++i) {
            int s = P.s(t, i), e = P.e(t, i);
            if (s >= e) continue;
            for (const Arg& ar : loops[i].args) {
                if (ar.access == OC_REDUCE) continue;
                DatPlan& dp = P.dp[P.dat_index[ar.dat]];
                if (is_read(ar.access)) mark(dp, t, (long long)s + ar.rmin[sa], (long long)e + ar.rmax[sa]);
                else mark(dp, t, s, e);
            }
        }
    // program-order state per row: 0 untouched, 1 first access a full-row write,
    // 2 first access anything else (a read, or a write that leaves part of the row
    // other than x columns), 3 first access a write over x in [wx0, wx1) and the full
    // extent of the other non-slow axes (only the x columns outside it are uploaded)
    std::vector<std::vector<uint8_t>> state(ND), written(ND);
    // per dataset: 1 if the first loop of the chain that touches it only writes it (a
    // "write-first" dataset, Sec. 4.1: a per-chain temporary under the cyclic option),
    // 2 if that loop reads it
    std::vector<uint8_t> dfirst(ND, 0);
    for (int d = 0; d < ND; ++d) {
        state[d].assign(P.dp[d].nrows, 0);
        written[d].assign(P.dp[d].nrows, 0);
        P.dp[d].wx0.assign(P.dp[d].nrows, 0);
        P.dp[d].wx1.assign(P.dp[d].nrows, 0);
    }
    for (const Loop& lp : loops) {
        int lo = lp.lo[sa], hi = lp.hi[sa];
        if (lo >= hi) continue;
        for (const Arg& ar : lp.args)
            if (ar.access != OC_REDUCE && is_read(ar.access) && !dfirst[P.dat_index[ar.dat]])
                dfirst[P.dat_index[ar.dat]] = 2;
        for (const Arg& ar : lp.args)
            if (ar.access != OC_REDUCE && is_write(ar.access) && !dfirst[P.dat_index[ar.dat]])
                dfirst[P.dat_index[ar.dat]] = 1;
        for (const Arg& ar : lp.args)
            if (ar.access != OC_REDUCE && is_read(ar.access)) {
                int d = P.dat_index[ar.dat];
                const DatPlan& dp = P.dp[d];
                long long a = std::max<long long>((long long)lo + ar.rmin[sa], dp.y0);
                long long b = std::min<long long>((long long)hi + ar.rmax[sa], (long long)dp.y0 + dp.nrows);
                for (long long y = a; y < b; ++y) if (!state[d][y - dp.y0]) state[d][y - dp.y0] = 2;
            }
        for (const Arg& ar : lp.args)
            if (ar.access != OC_REDUCE && is_write(ar.access)) {
                int d = P.dat_index[ar.dat];
                DatPlan& dp = P.dp[d];
                const Dat& dd = dats[ar.dat];
                uint8_t st = full_row_write(lp, dd) ? 1 : 2;
                if (st == 2 && ar.access == OC_WRITE) {
                    bool others_full = true;
                    for (int a = 1; a < dd.ndim - 1; ++a)
                        others_full = others_full && lp.lo[a] <= -dd.hlo[a] && lp.hi[a] >= dd.size[a] + dd.hhi[a];
                    if (others_full) st = 3;
                }
                for (long long y = std::max(lo, dp.y0); y < std::min(hi, dp.y0 + dp.nrows); ++y) {
                    const long long r = y - dp.y0;
                    if (!state[d][r]) {
                        state[d][r] = st;
                        if (st == 3) { dp.wx0[r] = std::max(lp.lo[0], -dd.hlo[0]); dp.wx1[r] = std::min(lp.hi[0], dd.size[0] + dd.hhi[0]); }
                    }
                    written[d][r] = 1;
                }
            }
    }
    const bool cyclic = (flags & OC_FLAG_CYCLIC) != 0;
    for (int d = 0; d < ND; ++d) {
        DatPlan& dp = P.dp[d];
        for (int r = 0; r < dp.nrows; ++r) {
            if (dp.first[r] < 0) continue;
            const uint8_t st = state[d][r];
            dp.need_up[r] = st == 2 ? 1 : (st == 3 ? 2 : 0);
            // cyclic (Sec. 4.1): a write-first dataset is a per-chain temporary, none of
            // its rows go back; any other dataset keeps every row it writes
            dp.dl[r] = written[d][r] && !(cyclic && dfirst[d] == 1);
        }
        // group rows into per-tile intervals (same tile, same copy kind and columns)
        auto group = [&](const std::vector<uint8_t>& need, const std::vector<int>& tile, bool cols,
                         std::vector<Interval>& out) {
            out.clear();
            int r = 0;
            auto key = [&](int q) { return cols && need[q] == 2 ? std::make_pair(dp.wx0[q], dp.wx1[q]) : std::make_pair(0, 0); };
            while (r < dp.nrows) {
                if (!need[r]) { ++r; continue; }
                int t = tile[r], a = r;
                const uint8_t kind = need[r];
                const auto kx = key(r);
                while (r < dp.nrows && need[r] == kind && tile[r] == t && key(r) == kx) ++r;
                Interval iv{t, a + dp.y0, r + dp.y0, kx.first, kx.second};
                out.push_back(iv);
            }
            std::stable_sort(out.begin(), out.end(), [](const Interval& x, const Interval& y) { return x.t < y.t; });
        };
        group(dp.need_up, dp.first, true, dp.up);
        group(dp.dl, dp.last, false, dp.down);
        // a resident dataset stays whole in device memory: no copies, no slab
        if (res && res->off[dp.dat] >= 0) {
            dp.resident = true;
            dp.S = dp.nrows;
            dp.up.clear();
            dp.down.clear();
            continue;
        }

        // slab rows: largest span of rows live in one phase. Phase p computes tile p,
        // uploads tile p + k, downloads tile p - 1. A row is live from the phase of its
        // upload (or first tile) to the phase of its download (or last tile).
        if (incore) { dp.S = dp.nrows; continue; }
        const int NP = T + k + 2;
        std::vector<int> pmin(NP, INT_MAX), pmax(NP, INT_MIN);
        for (int r = 0; r < dp.nrows; ++r) {
            if (dp.first[r] < 0) continue;
            int ps = dp.need_up[r] ? dp.first[r] - k : dp.first[r];
            int pe = dp.dl[r] ? dp.last[r] + 1 : dp.last[r];
            for (int p = ps; p <= pe; ++p) {
                pmin[p + k] = std::min(pmin[p + k], r);
                pmax[p + k] = std::max(pmax[p + k], r);
            }
        }
        int S = 1;
        for (int p = 0; p < NP; ++p)
            if (pmax[p] >= pmin[p]) S = std::max(S, pmax[p] - pmin[p] + 1);
        // Speculative prefetch (Sec. 4.1) uploads the next chain's tile-0 rows while the
        // last tile runs: pick the smallest S >= the minimum for which the slots of those
        // rows (hull R0) and of the rows still live in the last two phases (hull LE) do
        // not meet, so that prefetching never has to wait.
        if ((flags & OC_FLAG_PREFETCH) && T >= 2 && S < dp.nrows) {
            int r0a = INT_MAX, r0b = INT_MIN, lea = INT_MAX, leb = INT_MIN;
            for (int r = 0; r < dp.nrows; ++r) {
                if (dp.first[r] < 0) continue;
                if (dp.need_up[r] && dp.first[r] == 0) { r0a = std::min(r0a, r); r0b = std::max(r0b, r + 1); }
                int pe = dp.dl[r] ? dp.last[r] + 1 : dp.last[r];
                if (pe >= T - 1) { lea = std::min(lea, r); leb = std::max(leb, r + 1); }
            }
            if (r0a < r0b && lea < leb && r0b <= lea) {
                auto disjoint = [&](int Sc) {
                    const long long la = lea % Sc, ll = leb - lea, ra = r0a % Sc, rl = r0b - r0a;
                    if (ll + rl > Sc) return false;
                    // arcs [la, la + ll) and [ra, ra + rl) on a circle of Sc slots
                    const long long d1 = ((ra - la) % Sc + Sc) % Sc;  // start of R0 seen from LE
                    return d1 >= ll && d1 + rl <= Sc;
                };
                const int cap = std::min(dp.nrows, S + 2 * (r0b - r0a) + 64);
                for (int Sc = S; Sc <= cap; ++Sc)
                    if (disjoint(Sc)) { S = Sc; break; }
            }
        }
        dp.S = std::min(S, dp.nrows);
    }

    // ---- reductions: per-row partials, grouped per handle --------------------------
    P.loop_part.assign(L, -1);
    P.loop_chunks.assign(L, 0);
    P.loop_red.assign(L, -1);
    P.loop_param.assign(L, 0);
    std::vector<long long> loop_cnt(L, 0);
    for (int i = 0; i < L; ++i)
        for (const Arg& ar : loops[i].args)
            if (ar.access == OC_REDUCE) {
                int idx = -1;
                for (size_t r = 0; r < P.rp.size(); ++r) if (P.rp[r].handle == ar.dat) idx = (int)r;
                if (idx < 0) {
                    RedPlan rp;
                    rp.handle = ar.dat;
                    rp.op = red_ops[ar.dat];
                    idx = (int)P.rp.size();
                    P.rp.push_back(rp);
                }
                P.loop_red[i] = idx;
                long long plane = 1;
                for (int a = 0; a < nd - 1; ++a) plane *= std::max(0, loops[i].hi[a] - loops[i].lo[a]);
                int chunks = (int)std::max(1LL, (plane + kRedChunk - 1) / kRedChunk);
                P.loop_chunks[i] = chunks;
                loop_cnt[i] = plane > 0 ? (long long)std::max(0, loops[i].hi[sa] - loops[i].lo[sa]) * chunks : 0;
            }
    // ---- arena layout: the resident region first, then the slabs ----------------------
    long long off = res ? res->bytes : 0;
    P.res_bytes = off;
    for (int d = 0; d < ND; ++d) {
        DatPlan& dp = P.dp[d];
        if (dp.resident) {
            dp.off = res->off[dp.dat];
            P.res_dats++;
            continue;
        }
        dp.off = off;
        off += align_up((long long)dp.S * dats[dp.dat].row_bytes(), 256);
    }
    P.slab_bytes = off;
    P.res_level = res ? res->level : 0.0;
    off = 0;
    for (size_t r = 0; r < P.rp.size(); ++r) {
        P.rp[r].part_off = off;
        long long c = 0;
        for (int i = 0; i < L; ++i)
            if (P.loop_red[i] == (int)r) { P.loop_part[i] = off + c * 8; c += loop_cnt[i]; }
        P.rp[r].count = c;
        off += align_up(std::max(1LL, c) * 8, 256);
    }
    int np = 0;
    for (int i = 0; i < L; ++i) { P.loop_param[i] = np; np += (int)loops[i].params.size(); }
    P.nparams = np;
    P.params_off = off;
    off += align_up(std::max(1, np) * 8, 256);
    P.paramsf_off = off;
    off += align_up(std::max(1, np) * 4, 256);
    P.results_off = off;
    off += align_up(std::max<long long>(1, (long long)P.rp.size()) * 8, 256);
    P.scratch_bytes = off;
    P.arena_bytes = P.slab_bytes + P.scratch_bytes;
    P.sig = chain_signature(loops, dats, flags) ^ ((uint64_t)h * 0x9E3779B1u) ^ ((uint64_t)depth << 56)
            ^ (incore ? 0x5555ull : 0);
    if (res) {
        uint64_t r = 0x2545F4914F6CDD1Dull;
        for (size_t k = 0; k < res->off.size(); ++k) r = mix(r, (uint64_t)(res->off[k] + 1) * 31 + k);
        P.sig = mix(P.sig, r);
    }
    P.valid = true;
    (void)err;
    return true;
}

int fit_tile_height(const std::vector<Loop>& loops, const std::vector<Dat>& dats,
                    const std::vector<int>& red_ops, int depth, uint32_t flags,
                    long long budget, std::string& err, const Residency* res)
{
    if (loops.empty()) return 1;
    const int sa = loops[0].ndim - 1;
    int Y0 = INT_MAX, Y1 = INT_MIN;
    for (const Loop& lp : loops) { Y0 = std::min(Y0, lp.lo[sa]); Y1 = std::max(Y1, lp.hi[sa]); }
    const int span = std::max(1, Y1 - Y0);
    Plan P;
    auto fits = [&](int h) {
        build_plan(loops, dats, red_ops, h, depth, flags, false, P, err, res);
        return P.arena_bytes <= budget;
    };
    if (!fits(1)) return 0;
    if (fits(span)) return span;
    int lo = 1, hi = span;  // fits(lo), !fits(hi)
    while (hi - lo > 1) {
        int mid = lo + (hi - lo) / 2;
        if (fits(mid)) lo = mid; else hi = mid;
    }
    // the same number of tiles, evened out: no short last tile (a phase of its own). A
    // plan's size is not monotonic in h (slab rows follow where the skewed tile
    // boundaries fall), so the evened height is used only if its plan fits too.
    const int T = (span + lo - 1) / lo;
    const int even = (span + T - 1) / T;
    return even == lo || fits(even) ? even : lo;
}

Residency choose_residency(const std::vector<Loop>& loops, const std::vector<Dat>& dats,
                           const std::vector<int>& red_ops, uint32_t flags, long long budget,
                           double level)
{
    Residency R;
    R.off.assign(dats.size(), -1);
    R.level = level;
    if (level <= 0 || loops.empty()) return R;
    // bytes each dataset moves per chain without residency (tile height: an eighth of
    // the span, which changes these totals only by the skew of the tile boundaries)
    const int sa = loops[0].ndim - 1;
    int Y0 = INT_MAX, Y1 = INT_MIN;
    for (const Loop& lp : loops) { Y0 = std::min(Y0, lp.lo[sa]); Y1 = std::max(Y1, lp.hi[sa]); }
    Plan P;
    std::string err;
    build_plan(loops, dats, red_ops, std::max(1, (Y1 - Y0) / 8), 3, flags, false, P, err);
    struct Cand { int dat; double traffic, bytes; };
    std::vector<Cand> cand;
    for (const DatPlan& dp : P.dp) {
        const Dat& d = dats[dp.dat];
        double rows = 0;
        for (const Interval& iv : dp.up) if (iv.x0 == iv.x1) rows += iv.b - iv.a;
        for (const Interval& iv : dp.down) rows += iv.b - iv.a;
        if (rows > 0) cand.push_back({dp.dat, rows * (double)d.row_bytes(), (double)d.bytes()});
    }
    std::stable_sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) {
        const double ra = a.traffic / a.bytes, rb = b.traffic / b.bytes;
        if (ra != rb) return ra > rb;
        return a.traffic > b.traffic;
    });
    const long long cap = (long long)(level * (double)budget);
    for (const Cand& c : cand) {
        const long long need = align_up((long long)c.bytes, 256);
        if (R.bytes + need > cap) continue;
        R.off[c.dat] = R.bytes;
        R.bytes += need;
    }
    return R;
}

}  // namespace oc
