// Host planner for tiled passes: lowers a circuit to tile ops, groups them
// into HBM passes (greedy, dependency-respecting) and each pass into
// register segments.  All modes compute the same ordered product of gates
// (Sec. 2); the planner only reorders gates that commute (gates on disjoint
// qubits, or diagonal gates), so the result is the circuit's.
#include <algorithm>
#include <iterator>
#include <cmath>
#include <complex>
#include <cstdlib>

#include "plan.h"
#include "tile.h"

namespace sv {

namespace {

using cd = std::complex<double>;

cd toc(const Cplx &c) { return cd(c.re, c.im); }

int popc(uint64_t x) { return __builtin_popcountll(x); }

// Does U equal c * M_kind for a structured matrix M?  Returns the kind or -1.
int struct_kind(const Cplx *u4, cd *scale) {
    static const cd I(0, 1);
    static const cd M[SK_COUNT][4] = {
        {1, 1, 1, -1},         // H
        {1, -I, -I, 1},        // SX
        {1, I, I, 1},          // SXD
        {1, -1, 1, 1},         // SY
        {1, 1, -1, 1},         // SYD
        {0, 1, 1, 0},          // X
    };
    cd u[4];
    for (int k = 0; k < 4; ++k) u[k] = toc(u4[k]);
    for (int kind = 0; kind < SK_COUNT; ++kind) {
        int piv = -1;
        for (int k = 0; k < 4; ++k)
            if (M[kind][k] != cd(0)) {
                piv = k;
                break;
            }
        const cd c = u[piv] / M[kind][piv];
        if (std::abs(c) == 0) continue;
        bool ok = true;
        for (int k = 0; k < 4 && ok; ++k) ok = std::abs(u[k] - c * M[kind][k]) <= 1e-15 * std::abs(c);
        if (ok) {
            *scale = c;
            return kind;
        }
    }
    return -1;
}

uint64_t full_of(const PGate &g) { return g.kind == 0 ? (uint64_t(1) << g.target) : 0; }
uint64_t diag_of(const PGate &g) { return g.cmask; }

bool conflicts(uint64_t F, uint64_t D, uint64_t bF, uint64_t bD) { return (F & (bF | bD)) || (D & bF); }

}  // namespace

std::vector<PGate> lower_for_tiles(const Circuit &c) {
    std::vector<PGate> out;
    Cplx m[16];
    auto g1 = [&](int t, int ctl, const Cplx *u) {
        PGate g{};
        g.kind = 0;
        g.target = t;
        g.cmask = ctl >= 0 ? (uint64_t(1) << ctl) : 0;
        g.cval = g.cmask;
        for (int k = 0; k < 4; ++k) g.u[k] = u[k];
        g.scale = Cplx{1, 0};
        out.push_back(g);
    };
    auto phase = [&](uint64_t mask, uint64_t val, cd ph) {
        if (ph == cd(1)) return;
        PGate g{};
        g.kind = 1;
        g.target = -1;
        g.cmask = mask;
        g.cval = val;
        g.u[0] = Cplx{ph.real(), ph.imag()};
        g.scale = Cplx{1, 0};
        out.push_back(g);
    };
    for (const Instr &ins : c.instrs) {
        if (ins.nq == 1) {
            gate_matrix(ins.name, ins.p, ins.np, m);
            const bool diag = m[1].re == 0 && m[1].im == 0 && m[2].re == 0 && m[2].im == 0;
            const uint64_t b = uint64_t(1) << ins.q[0];
            if (diag) {
                const cd d0 = toc(m[0]), d1 = toc(m[3]);
                if (d0 == cd(0)) {
                    phase(b, 0, 0);
                    phase(b, b, d1);
                } else {
                    // diag(d0, d1) = d0 * diag(1, d1/d0): the scalar is deferred
                    phase(b, b, d1 / d0);
                    if (d0 != cd(1)) {
                        PGate g{};
                        g.kind = 1;
                        g.target = -1;
                        g.cmask = 0;
                        g.cval = 0;
                        g.u[0] = Cplx{1, 0};
                        g.scale = Cplx{d0.real(), d0.imag()};
                        out.push_back(g);
                    }
                }
            } else {
                g1(ins.q[0], -1, m);
            }
            continue;
        }
        const int a = ins.q[0], b = ins.q[1];
        const uint64_t ab = (uint64_t(1) << a) | (uint64_t(1) << b);
        if (ins.name == "CZ") {
            phase(ab, ab, -1);
        } else if (ins.name == "CP") {
            phase(ab, ab, std::polar(1.0, ins.p[0]));
        } else {
            gate_matrix("X", nullptr, 0, m);
            if (ins.name == "CX") {
                g1(b, a, m);
            } else {  // SWAP
                g1(b, a, m);
                g1(a, b, m);
                g1(b, a, m);
            }
        }
    }
    return out;
}

namespace {

// Shared-memory bank model of the complex64 passes: 8-byte amplitude j of a
// tile lives at element (swz(j >> 1) << 1) | (j & 1), swz(c) = c ^ ((c >> 3 ^
// c >> 6 ^ c >> 9) & 7), the XOR swizzle of the generated kernels.  A warp's
// 8-byte accesses are served per half-warp (lanes 0-15, 16-31); the wavefronts
// of a half-warp are the most distinct 4-byte words any bank receives.  The
// swizzle is linear over XOR, so a register slot's constant offset permutes
// the banks without changing that count: it depends on the lane bits alone.
uint32_t swz_chunk(uint32_t c) { return c ^ (((c >> 3) ^ (c >> 6) ^ (c >> 9)) & 7u); }

int bank_ways64(const int lanes[5]) {
    int worst = 0;
    for (int half = 0; half < 2; ++half) {
        uint32_t words[32];  // the distinct 4-byte words of this half-warp
        int nw = 0;
        for (int l = 0; l < 16; ++l) {
            const int ll = l + 16 * half;
            uint32_t j = 0;
            for (int k = 0; k < 5; ++k)
                if (ll >> k & 1) j |= 1u << lanes[k];
            const uint32_t e = (swz_chunk(j >> 1) << 1) | (j & 1u);
            for (uint32_t w = 2 * e; w < 2 * e + 2; ++w)
                if (std::find(words, words + nw, w) == words + nw) words[nw++] = w;
        }
        int ways[32] = {0};
        for (int i = 0; i < nw; ++i) worst = std::max(worst, ++ways[words[i] & 31u]);
    }
    return worst;
}

// Lanes of a complex64 segment: among the 5-bit subsets of the free tile
// bits (and the choice of which one selects the half-warp) the one with the
// fewest shared-memory wavefronts; with `hbm`, a subset holding tile bits
// 0-2 (whole 32-byte sectors for a direct HBM access) comes first, then one
// holding bit 3 too (whole 128-byte lines).  Warp bits follow, ascending.
void order_thread_bits64(const std::vector<int> &avail, bool hbm, uint8_t *tpos) {
    const int na = int(avail.size());
    int best[5] = {0, 0, 0, 0, 0};
    long best_score = -1;
    for (uint32_t sub = 0; sub < (1u << na); ++sub) {
        if (__builtin_popcount(sub) != 5 || na < 5) continue;
        int pick[5], k = 0;
        for (int i = 0; i < na; ++i)
            if (sub >> i & 1) pick[k++] = avail[size_t(i)];
        uint32_t set = 0;
        for (int i = 0; i < 5; ++i) set |= 1u << pick[i];
        for (int hi = 0; hi < 5; ++hi) {
            int lanes[5], q = 0;
            for (int i = 0; i < 5; ++i)
                if (i != hi) lanes[q++] = pick[i];
            lanes[4] = pick[hi];
            const int ways = bank_ways64(lanes);
            long score = long(16 - ways) * 4;
            if (hbm) score += ((set & 7u) == 7u ? 1000 : 0) + ((set & 15u) == 15u ? 100 : 0);
            score = score * 64 + (63 - pick[hi]);  // ties: the lower sets first
            if (score > best_score) {
                best_score = score;
                std::copy(lanes, lanes + 5, best);
            }
        }
    }
    if (best_score < 0) {  // fewer than 5 free bits (not a complex64 layout)
        for (int i = 0; i < na; ++i) tpos[i] = uint8_t(avail[size_t(i)]);
        return;
    }
    int k = 0;
    for (int i = 0; i < 5; ++i) tpos[k++] = uint8_t(best[i]);
    for (int b : avail)
        if (std::find(best, best + 5, b) == best + 5) tpos[k++] = uint8_t(b);
}

// Lane order for the thread bits of a segment: the first lane bits get tile
// positions whose shared-memory bank contributions are independent under the
// XOR swizzle of k_tile (see phys_chunk there), the rest ascending.
void order_thread_bits(const std::vector<int> &avail, bool c64, uint8_t *tpos) {
    if (c64 && avail.size() >= 5) {
        order_thread_bits64(avail, false, tpos);
        return;
    }
    std::vector<int> rest = avail, lanes;
    auto take = [&](auto pred) {
        for (size_t i = 0; i < rest.size(); ++i)
            if (pred(rest[i])) {
                lanes.push_back(rest[i]);
                rest.erase(rest.begin() + long(i));
                return true;
            }
        return false;
    };
    if (c64) {
        take([](int p) { return p == 0; });
        for (int r = 0; r < 3; ++r) take([r](int p) { return p >= 1 && (p - 1) % 3 == r; });
    } else {
        for (int r = 0; r < 3; ++r) take([r](int p) { return p % 3 == r; });
    }
    std::sort(rest.begin(), rest.end());
    size_t k = 0;
    for (int p : lanes) tpos[k++] = uint8_t(p);
    for (int p : rest) tpos[k++] = uint8_t(p);
}


// Number of pending gates applicable in one pass with tile set T (a gate is
// applicable when its non-diagonal qubit is in T and no earlier pending gate
// it does not commute with stays behind).
int count_applicable(const std::vector<PGate> &G, const std::vector<int> &pending, uint64_t T, uint64_t all) {
    uint64_t bF = 0, bD = 0;
    int cnt = 0;
    for (int idx : pending) {
        const PGate &g = G[size_t(idx)];
        const uint64_t F = full_of(g), D = diag_of(g);
        if (!conflicts(F, D, bF, bD) && (F & ~T) == 0) ++cnt;
        else {
            bF |= F;
            bD |= D;
            if ((bF & all) == all) break;
        }
    }
    return cnt;
}

uint64_t choose_tile(const std::vector<PGate> &G, const std::vector<int> &pending, int n, int m, uint64_t lowmask,
                     uint64_t all) {
    // (a) first-come
    uint64_t Ta = lowmask, bF = 0, bD = 0;
    for (int idx : pending) {
        const PGate &g = G[size_t(idx)];
        const uint64_t F = full_of(g), D = diag_of(g);
        if (conflicts(F, D, bF, bD)) {
            bF |= F;
            bD |= D;
        } else {
            const uint64_t need = F & ~Ta;
            if (popc(Ta | need) <= m) Ta |= need;
            else {
                bF |= F;
                bD |= D;
            }
        }
        if ((bF & all) == all) break;
    }
    for (int q = 0; q < n && popc(Ta) < m; ++q) Ta |= uint64_t(1) << q;
    // (b) greedy growth by applicable-gate count; ties go to the qubit whose
    // first pending non-diagonal gate comes earliest
    std::vector<int> first_use(size_t(n), 1 << 30);
    for (size_t i = 0; i < pending.size(); ++i) {
        const PGate &g = G[size_t(pending[i])];
        if (g.kind == 0 && first_use[size_t(g.target)] > int(i)) first_use[size_t(g.target)] = int(i);
    }
    uint64_t Tb = lowmask;
    while (popc(Tb) < m && popc(Tb) < n) {
        int best_q = -1, best_c = -1;
        for (int q = 0; q < n; ++q) {
            if (Tb >> q & 1) continue;
            const int c = count_applicable(G, pending, Tb | (uint64_t(1) << q), all);
            if (c > best_c || (c == best_c && first_use[size_t(q)] < first_use[size_t(best_q)])) {
                best_c = c;
                best_q = q;
            }
        }
        Tb |= uint64_t(1) << best_q;
    }
    return count_applicable(G, pending, Tb, all) >= count_applicable(G, pending, Ta, all) ? Tb : Ta;
}

// Remove the gates applicable with tile T from `pending` (the pass's gates).
void take_pass(const std::vector<PGate> &G, std::vector<int> &pending, uint64_t T, uint64_t all) {
    std::vector<int> rest;
    rest.reserve(pending.size());
    uint64_t bF = 0, bD = 0;
    for (size_t i = 0; i < pending.size(); ++i) {
        const int idx = pending[i];
        const PGate &g = G[size_t(idx)];
        const uint64_t F = full_of(g), D = diag_of(g);
        if ((bF & all) == all) {
            rest.insert(rest.end(), pending.begin() + long(i), pending.end());
            break;
        }
        if (!conflicts(F, D, bF, bD) && (F & ~T) == 0) continue;
        bF |= F;
        bD |= D;
        rest.push_back(idx);
    }
    pending.swap(rest);
}

int segments_first_fit(const std::vector<PGate> &G, std::vector<int> pending, int rb, uint64_t all);

// Cost of the greedy choice for `pending`: passes, each worth kPassCost
// segments (an HBM round trip of the state against one shared-memory
// transposition of it, as measured), plus the segments first fit needs.
// Passes the greedy choice needs for `pending`.
int greedy_passes(const std::vector<PGate> &G, std::vector<int> pending, int n, int m, uint64_t lowmask, uint64_t all) {
    int np = 0;
    while (!pending.empty()) {
        take_pass(G, pending, choose_tile(G, pending, n, m, lowmask, all), all);
        ++np;
    }
    return np;
}

// Rollout objective of the tile lookahead: 0 = passes alone (ties to the
// greedy choice); c > 0 = c x passes + segments (a pass against the
// shared-memory transpositions it saves).  plan_tiles plans with both and
// keeps the plan with fewer passes, then fewer segments: on the measured
// circuits that is always the faster one, while neither objective alone is.
thread_local int g_pass_cost = 0;
int pass_cost() { return g_pass_cost; }
#define kPassCost pass_cost()
int greedy_cost(const std::vector<PGate> &G, std::vector<int> pending, int n, int m, int rb, uint64_t lowmask,
                uint64_t all) {
    int cost = 0;
    while (!pending.empty()) {
        const std::vector<int> before = pending;
        take_pass(G, pending, choose_tile(G, pending, n, m, lowmask, all), all);
        std::vector<int> ops;
        std::set_difference(before.begin(), before.end(), pending.begin(), pending.end(), std::back_inserter(ops));
        cost += kPassCost + segments_first_fit(G, ops, rb, all);
    }
    return cost;
}

// Tile for the next pass with lookahead: candidates are the greedy choice and
// the greedy growths started from each of the best single qubits; each is
// rolled out with the greedy choice to the end, and the one with the fewest
// passes in total wins (ties: the greedy choice, then more gates now).
uint64_t choose_tile_lookahead(const std::vector<PGate> &G, const std::vector<int> &pending, int n, int m, int rb,
                               uint64_t lowmask, uint64_t all, int width) {
    std::vector<uint64_t> cand;
    cand.push_back(choose_tile(G, pending, n, m, lowmask, all));
    std::vector<std::pair<int, int>> first;  // (applicable count, qubit)
    for (int q = 0; q < n; ++q)
        if (!(lowmask >> q & 1)) first.push_back({count_applicable(G, pending, lowmask | (uint64_t(1) << q), all), q});
    std::sort(first.begin(), first.end(), [](auto a, auto b) { return a.first > b.first || (a.first == b.first && a.second < b.second); });
    for (int i = 0; i < width && i < int(first.size()); ++i) {
        uint64_t Tb = lowmask | (uint64_t(1) << first[size_t(i)].second);
        while (popc(Tb) < m && popc(Tb) < n) {
            int best_q = -1, best_c = -1;
            for (int q = 0; q < n; ++q) {
                if (Tb >> q & 1) continue;
                const int c = count_applicable(G, pending, Tb | (uint64_t(1) << q), all);
                if (c > best_c) {
                    best_c = c;
                    best_q = q;
                }
            }
            Tb |= uint64_t(1) << best_q;
        }
        if (std::find(cand.begin(), cand.end(), Tb) == cand.end()) cand.push_back(Tb);
    }
    uint64_t best = cand[0];
    int best_np = 1 << 30, best_cnt = -1;
    for (uint64_t T : cand) {
        std::vector<int> rest = pending;
        take_pass(G, rest, T, all);
        std::vector<int> ops;
        std::set_difference(pending.begin(), pending.end(), rest.begin(), rest.end(), std::back_inserter(ops));
        const int np = kPassCost == 0 ? 1 + greedy_passes(G, rest, n, m, lowmask, all)
                                      : kPassCost + segments_first_fit(G, ops, rb, all) + greedy_cost(G, rest, n, m, rb, lowmask, all);
        const int cnt = int(pending.size() - rest.size());
        const bool tie_to_greedy = kPassCost == 0;
        if (np < best_np || (np == best_np && !tie_to_greedy) ||
            (np == best_np && cnt > best_cnt && T != cand[0] && best != cand[0])) {
            best_np = np;
            best_cnt = cnt;
            best = T;
        }
    }
    return best;
}

// Register qubits of the next segment, first fit: pending gates in order
// add their non-diagonal qubits while at most rb fit.
uint64_t rset_first_fit(const std::vector<PGate> &G, const std::vector<int> &pending, int rb) {
    uint64_t Rset = 0, bF = 0, bD = 0;
    for (int idx : pending) {
        const PGate &g = G[size_t(idx)];
        const uint64_t F = full_of(g), D = diag_of(g);
        if (conflicts(F, D, bF, bD)) {
            bF |= F;
            bD |= D;
            continue;
        }
        const uint64_t need = F & ~Rset;
        if (popc(Rset | need) <= rb) Rset |= need;
        else {
            bF |= F;
            bD |= D;
        }
    }
    return Rset;
}

// Segments first fit needs for `pending` (diagonal gates count as free).
int segments_first_fit(const std::vector<PGate> &G, std::vector<int> pending, int rb, uint64_t all) {
    int ns = 0;
    for (;;) {
        bool nondiag = false;
        for (int idx : pending) nondiag |= G[size_t(idx)].kind == 0;
        if (!nondiag) return ns;
        take_pass(G, pending, rset_first_fit(G, pending, rb), all);
        ++ns;
    }
}

// Register qubits of the next segment with lookahead: first fit, and greedy
// growth by applicable-gate count started from each of the `width` best
// single qubits; each candidate is rolled out with first fit and the one
// needing the fewest segments wins (ties: first fit, then more gates now).
// avoid: qubits a register set should leave to the lanes when that costs no
// segment (the low tile bits of a segment that loads straight from HBM); the
// greedy growths are then also tried without them.
uint64_t rset_lookahead(const std::vector<PGate> &G, const std::vector<int> &pending, uint64_t T, int rb, uint64_t all,
                        int width, uint64_t avoid = 0) {
    std::vector<uint64_t> cand{rset_first_fit(G, pending, rb)};
    auto grow = [&](uint64_t TT) {
        std::vector<std::pair<int, int>> first;
        for (int q = 0; q < 64; ++q)
            if (TT >> q & 1) first.push_back({count_applicable(G, pending, uint64_t(1) << q, all), q});
        std::sort(first.begin(), first.end(),
                  [](auto a, auto b) { return a.first > b.first || (a.first == b.first && a.second < b.second); });
        for (int i = 0; i < width && i < int(first.size()); ++i) {
            uint64_t R = uint64_t(1) << first[size_t(i)].second;
            while (popc(R) < rb && popc(R) < popc(TT)) {
                int best_q = -1, best_c = -1;
                for (int q = 0; q < 64; ++q) {
                    if (!(TT >> q & 1) || (R >> q & 1)) continue;
                    const int c = count_applicable(G, pending, R | (uint64_t(1) << q), all);
                    if (c > best_c) {
                        best_c = c;
                        best_q = q;
                    }
                }
                R |= uint64_t(1) << best_q;
            }
            if (std::find(cand.begin(), cand.end(), R) == cand.end()) cand.push_back(R);
        }
    };
    grow(T);
    const size_t ngrow = cand.size();
    if (avoid && popc(T & ~avoid) >= rb) grow(T & ~avoid);
    uint64_t best = cand[0];
    int best_ns = 1 << 30, best_cnt = -1;
    bool best_clear = false;
    for (size_t i = 0; i < cand.size(); ++i) {
        const uint64_t R = cand[i];
        std::vector<int> rest = pending;
        take_pass(G, rest, R, all);
        const int ns = 1 + segments_first_fit(G, rest, rb, all);
        const int cnt = int(pending.size() - rest.size());
        const bool clear = avoid && !(R & avoid);
        if (i >= ngrow && !(ns < best_ns || (ns == best_ns && clear && !best_clear))) continue;
        if (ns < best_ns || (ns == best_ns && clear && !best_clear) ||
            (ns == best_ns && clear == best_clear && R != cand[0] && best != cand[0] && cnt > best_cnt)) {
            best_ns = ns;
            best_cnt = cnt;
            best = R;
            best_clear = clear;
        }
    }
    return best;
}

}  // namespace

int seg_lookahead_width() {
    static const int width = std::getenv("SV_SEG_LOOKAHEAD") ? std::atoi(std::getenv("SV_SEG_LOOKAHEAD")) : 4;
    return width;
}

int tile_rb64() {
    const char *e = std::getenv("SV_TILE_RB");
    const int v = e ? std::atoi(e) : kTileRB64;
    return (v >= 4 && v <= 6) ? v : kTileRB64;
}

int plan_lookahead_width() {
    static const int width = std::getenv("SV_PLAN_LOOKAHEAD") ? std::atoi(std::getenv("SV_PLAN_LOOKAHEAD")) : 4;
    return width;
}

int tile_low64() {
    const char *e = std::getenv("SV_TILE_LOW");
    const int v = e ? std::atoi(e) : kTileLow64;
    return (v >= 4 && v <= 10) ? v : kTileLow64;
}

template <typename R>
sv_status plan_tiles_one(const std::vector<PGate> &G, int n, const TileConfig &cfg, TilePlan<R> *out);

template <typename R>
sv_status plan_tiles(const std::vector<PGate> &G, int n, const TileConfig &cfg, TilePlan<R> *out) {
    const char *e = std::getenv("SV_PLAN_PASS_COST");
    if (e) {  // one objective only
        g_pass_cost = std::atoi(e);
        return plan_tiles_one(G, n, cfg, out);
    }
    g_pass_cost = 0;
    sv_status s = plan_tiles_one(G, n, cfg, out);
    if (s || plan_lookahead_width() == 0) return s;
    TilePlan<R> alt;
    g_pass_cost = 4;
    s = plan_tiles_one(G, n, cfg, &alt);
    g_pass_cost = 0;
    if (s) return s;
    if (alt.passes.size() < out->passes.size() ||
        (alt.passes.size() == out->passes.size() && alt.segs.size() < out->segs.size()))
        *out = std::move(alt);
    return SV_OK;
}

template <typename R>
sv_status plan_tiles_one(const std::vector<PGate> &G, int n, const TileConfig &cfg, TilePlan<R> *out) {
    out->passes.clear();
    out->ops.clear();
    out->segs.clear();
    out->lane_ops.clear();
    out->nseg.clear();
    out->m = cfg.m;
    out->rb = cfg.rb;
    out->ctas = cfg.ctas;
    out->direct = cfg.c64 && cfg.direct;
    out->prefetch = cfg.c64 && cfg.direct && cfg.prefetch;
    const int m = cfg.m, rb = cfg.rb, L = cfg.low;
    if (n < m) {
        set_error("tiled mode needs n >= %d", m);
        return SV_ERR_UNSUPPORTED;
    }
    std::vector<int> pending(G.size());
    for (size_t i = 0; i < G.size(); ++i) pending[i] = int(i);
    const uint64_t all = n == 64 ? ~uint64_t(0) : ((uint64_t(1) << n) - 1);
    const uint64_t lowmask = (uint64_t(1) << L) - 1;

    while (!pending.empty()) {
        // ---- choose the tile qubits: the better of (a) first-come (qubits in
        // the order pending gates need them) and (b) greedy growth, adding
        // one qubit at a time the one that makes the most gates applicable;
        // with lookahead, the candidate whose greedy rollout needs the
        // fewest passes
        // lookahead width (SV_PLAN_LOOKAHEAD; 0: the greedy choice alone).
        // Fewer passes, each fuller: 12 -> 11 passes and 5% less time for
        // the 32-qubit depth-24 circuit, 7 -> 6 for QFT-32.
        const int width = plan_lookahead_width();
        const uint64_t T = width > 0 ? choose_tile_lookahead(G, pending, n, m, rb, lowmask, all, width)
                                     : choose_tile(G, pending, n, m, lowmask, all);
        // ---- collect the pass's gates
        std::vector<int> pass_ops, rest;
        uint64_t bF = 0, bD = 0;
        for (size_t i = 0; i < pending.size(); ++i) {
            const int idx = pending[i];
            const PGate &g = G[size_t(idx)];
            const uint64_t F = full_of(g), D = diag_of(g);
            if ((bF & all) == all) {
                rest.insert(rest.end(), pending.begin() + long(i), pending.end());
                break;
            }
            if (!conflicts(F, D, bF, bD) && (F & ~T) == 0) pass_ops.push_back(idx);
            else {
                bF |= F;
                bD |= D;
                rest.push_back(idx);
            }
        }
        pending.swap(rest);

        TilePassArgs pa{};
        pa.n = n;
        pa.m = m;
        int tpos_of[64];
        for (int q = 0; q < 64; ++q) tpos_of[q] = -1;
        {
            int k = 0, o = 0;
            for (int q = 0; q < n; ++q) {
                if (T >> q & 1) {
                    tpos_of[q] = k;
                    pa.tile_pos[k++] = uint8_t(q);
                } else {
                    pa.outer_pos[o++] = uint8_t(q);
                }
            }
            pa.nouter = o;
            int lc = 0;
            while (lc < m && pa.tile_pos[lc] == lc) ++lc;
            pa.lc = lc;
        }
        pa.op_begin = int(out->ops.size());

        // ---- the FP32 work the pass's gates need at least, per amplitude
        {
            double ops = 0.0;
            for (int idx : pass_ops) {
                const PGate &g = G[size_t(idx)];
                const double frac = std::ldexp(1.0, -popc(g.cmask & kQubitBits));
                if (g.kind == 0) {
                    cd c;
                    const int kind = struct_kind(g.u, &c);
                    ops += frac * (kind == SK_X ? 0.0 : kind >= 0 ? 2.0 : 8.0);
                } else if (toc(g.scale) == cd(1)) {
                    const cd ph = toc(g.u[0]);
                    const double ar = std::fabs(ph.real()), ai = std::fabs(ph.imag());
                    if (ph == cd(1) || ph == cd(-1) || ph == cd(0)) continue;
                    ops += frac * (std::fabs(ar - ai) <= 4e-7 * ar ? 2.0 : 4.0);
                }
            }
            out->lane_ops.push_back(ops);
        }
        // ---- segments (list scheduling over register slots)
        std::vector<int> remaining = pass_ops;
        cd scale = 1;
        int since_flush = 0;
        auto flush_scale = [&]() {
            if (std::abs(scale - cd(1)) > 0) {
                TileOp<R> op{};
                op.type = TOP_SCALE;
                op.u[0] = R(scale.real());
                op.u[1] = R(scale.imag());
                out->ops.push_back(op);
            }
            scale = 1;
            since_flush = 0;
        };
        while (!remaining.empty()) {
            const int sw = seg_lookahead_width();
            // the first segment loads straight from HBM when tile bits 0-2 are lanes
            const uint64_t low3 = (cfg.c64 && cfg.direct && remaining.size() == pass_ops.size() && L >= 3)
                                      ? ((uint64_t(1) << pa.tile_pos[0]) | (uint64_t(1) << pa.tile_pos[1]) |
                                         (uint64_t(1) << pa.tile_pos[2]))
                                      : 0;
            uint64_t Rset = sw > 0 ? rset_lookahead(G, remaining, T, rb, all, sw, low3) : rset_first_fit(G, remaining, rb);
            for (int k = m - 1; k >= 0 && popc(Rset) < rb; --k) {
                // fill with the highest tile bits (keeps the low, contiguous
                // ones free for lanes: coalesced HBM access)
                Rset |= uint64_t(1) << pa.tile_pos[k];
            }
            std::vector<int> applicable, rest2;
            bF = bD = 0;
            for (int idx : remaining) {
                const PGate &g = G[size_t(idx)];
                const uint64_t F = full_of(g), D = diag_of(g);
                if (!conflicts(F, D, bF, bD) && (F & ~Rset) == 0) applicable.push_back(idx);
                else {
                    bF |= F;
                    bD |= D;
                    rest2.push_back(idx);
                }
            }
            // Diagonal gates go where they are cheapest: one is emitted now if
            // all its qubits are register qubits here (a compile-time phase or
            // sign), if a later non-diagonal gate of this segment acts on one
            // of its qubits, or if no non-diagonal gate is left for later
            // segments of the pass; otherwise it waits for a later segment.
            bool nondiag_left = false;
            for (int idx : rest2) nondiag_left |= G[size_t(idx)].kind == 0;
            std::vector<int> seg_ops;
            {
                std::vector<char> keep(applicable.size(), 1);
                if (nondiag_left) {
                    uint64_t later_full = 0;
                    for (size_t i = applicable.size(); i-- > 0;) {
                        const PGate &g = G[size_t(applicable[i])];
                        if (g.kind == 0) later_full |= full_of(g);
                        else if (!(diag_of(g) & later_full) && toc(g.scale) == cd(1) && (diag_of(g) & ~Rset))
                            keep[i] = 0;  // defer unless needed now or all its qubits are register qubits
                    }
                }
                std::vector<int> deferred;
                for (size_t i = 0; i < applicable.size(); ++i)
                    (keep[i] ? seg_ops : deferred).push_back(applicable[i]);
                if (!deferred.empty()) {
                    // deferred gates go back in circuit order
                    std::vector<int> merged;
                    merged.reserve(deferred.size() + rest2.size());
                    std::merge(deferred.begin(), deferred.end(), rest2.begin(), rest2.end(), std::back_inserter(merged));
                    rest2.swap(merged);
                }
            }
            remaining.swap(rest2);
            // segment descriptor
            TileSeg sg{};
            int slot_of_tbit[kTileMaxQ];
            for (int k = 0; k < kTileMaxQ; ++k) slot_of_tbit[k] = -1;
            std::vector<int> rpos, avail;
            for (int k = 0; k < m; ++k) {
                if (Rset >> pa.tile_pos[k] & 1) rpos.push_back(k);
                else avail.push_back(k);
            }
            for (size_t s = 0; s < rpos.size(); ++s) {
                sg.rpos[s] = uint8_t(rpos[s]);
                slot_of_tbit[rpos[s]] = int(s);
            }
            order_thread_bits(avail, cfg.c64, sg.tpos);
            TileOp<R> segop{};
            segop.type = TOP_SEG;
            segop.a = int(out->segs.size());
            out->segs.push_back(sg);
            out->ops.push_back(segop);
            // ops of the segment
            for (int idx : seg_ops) {
                const PGate &g = G[size_t(idx)];
                TileOp<R> op{};
                for (int q = 0; q < 64; ++q) {
                    if (!(g.cmask >> q & 1)) continue;
                    const uint64_t want = g.cval >> q & 1;
                    if (q >= kParamBit0) {
                        op.pmask |= 1u << (q - kParamBit0);
                        op.pval |= uint32_t(want) << (q - kParamBit0);
                    } else if (q >= n) {
                        set_error("gate condition on qubit %d of a %d-qubit state", q, n);
                        return SV_ERR_ARG;
                    } else if (tpos_of[q] < 0) {
                        op.gmask |= uint64_t(1) << q;
                        op.gval |= want << q;
                    } else if (slot_of_tbit[tpos_of[q]] >= 0) {
                        op.rmask |= 1u << slot_of_tbit[tpos_of[q]];
                        op.rval |= uint32_t(want) << slot_of_tbit[tpos_of[q]];
                    } else {
                        op.tmask |= 1u << tpos_of[q];
                        op.tval |= uint32_t(want) << tpos_of[q];
                    }
                }
                if (g.kind == 1) {
                    if (toc(g.scale) != cd(1)) {  // a deferred scalar only
                        scale *= toc(g.scale);
                        continue;
                    }
                    const cd ph = toc(g.u[0]);
                    op.type = ph == cd(-1) ? TOP_NEG : TOP_PHASE;
                    op.a = reg_cond_id(op.rmask, op.rval);
                    op.u[0] = R(ph.real());
                    op.u[1] = R(ph.imag());
                    out->ops.push_back(op);
                    continue;
                }
                const int slot = slot_of_tbit[tpos_of[g.target]];
                cd c;
                const int kind = struct_kind(g.u, &c);
                const bool controlled = g.cmask != 0;
                if (kind >= 0 && (!controlled || c == cd(1))) {
                    op.type = TOP_STRUCT;
                    op.a = slot | (kind << 8);
                    if (!controlled) scale *= c;
                    out->ops.push_back(op);
                    if (++since_flush >= 160) flush_scale();  // bounds the deferred growth at 2^80
                } else {
                    op.type = TOP_G1;
                    op.a = slot;
                    for (int k = 0; k < 4; ++k) {
                        op.u[2 * k] = R(g.u[k].re);
                        op.u[2 * k + 1] = R(g.u[k].im);
                    }
                    out->ops.push_back(op);
                }
            }
        }
        flush_scale();
        pa.op_end = int(out->ops.size());
        {
            int ns = 0;
            for (int i = pa.op_begin; i < pa.op_end; ++i) ns += out->ops[size_t(i)].type == TOP_SEG;
            out->nseg.push_back(ns);
        }
        if (cfg.c64 && cfg.direct) {
            // the first and last segments load from and store to HBM straight
            // from registers when tile bits 0-2 are free for lanes: their lanes
            // then take the lowest free tile bits (contiguous amplitudes), so a
            // warp access covers whole sectors; otherwise that end is staged
            // through shared memory and keeps the bank-friendly lane order
            int first = -1, last = -1;
            for (int i = pa.op_begin; i < pa.op_end; ++i)
                if (out->ops[size_t(i)].type == TOP_SEG) {
                    if (first < 0) first = out->ops[size_t(i)].a;
                    last = out->ops[size_t(i)].a;
                }
            for (int sidx : {first, last}) {
                if (sidx < 0) continue;
                TileSeg &sg = out->segs[size_t(sidx)];
                uint32_t reg = 0;
                for (int sl = 0; sl < rb; ++sl) reg |= 1u << sg.rpos[sl];
                if ((reg & 7u) != 0 || L < 3) continue;
                std::vector<int> avail;
                for (int b = 0; b < m; ++b)
                    if (!(reg >> b & 1)) avail.push_back(b);
                order_thread_bits64(avail, true, sg.tpos);
            }
        }
        out->passes.push_back(pa);
    }
    return SV_OK;
}

template sv_status plan_tiles<float>(const std::vector<PGate> &, int, const TileConfig &, TilePlan<float> *);
template sv_status plan_tiles<double>(const std::vector<PGate> &, int, const TileConfig &, TilePlan<double> *);

}  // namespace sv
