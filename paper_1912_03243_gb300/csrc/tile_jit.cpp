// Tiled passes compiled per circuit: the planner's pass programs (tile.h)
// are turned into one straight-line CUDA kernel per pass and compiled with
// NVRTC for sm_103a.
//
// Why compile: in a pass every register slot, segment layout, swizzled
// shared-memory offset, condition mask and matrix entry is known on the host.
// Emitted as constants, the pass becomes straight-line code over 2^RB
// register amplitudes with no op decoding and no branches between ops, so
// the per-amplitude cost of a structured gate is its four FP32 additions.
// (An interpreter that dispatches ops at run time has to reconcile the
// register array at every dispatch point and spends most of its issue slots
// on register moves.)
//
// Generated kernel, per CTA (one 2^M-amplitude tile, NT = 2^(M-RB) threads):
//   load: cp.async 16-byte chunks into an XOR-swizzled shared tile (chunk c
//         stored at c ^ ((c>>3 ^ c>>6 ^ c>>9) & 7)); the global offset and
//         the swizzled address of chunk t + 256 i are a per-thread value XOR
//         a per-i constant (both maps are linear over disjoint bits);
//   per segment: gather 2^RB amplitudes (thread part of the tile index XOR
//         constant register offsets), apply the segment's ops, scatter;
//   store: 16-byte chunks back to HBM.
// Conditions on thread or CTA index bits become selects, not branches.
#include <dlfcn.h>
#include <fcntl.h>
#include <nvrtc.h>
#include <spawn.h>
#include <sys/stat.h>
#include <sys/utsname.h>
#include <sys/wait.h>
#include <unistd.h>

#include <atomic>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <functional>
#include <iterator>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nvrtc_opts.h"
#include "plan.h"
#include "tile.h"

extern char **environ;

namespace sv {

namespace {

std::string lit(float v) {
    char b[48];
    std::snprintf(b, sizeof b, "%.9g", double(v));
    std::string s(b);
    if (s.find_first_of(".eEn") == std::string::npos) s += ".0";
    return s + "f";
}

std::string lit(double v) {
    char b[48];
    std::snprintf(b, sizeof b, "%.17g", v);
    std::string s(b);
    if (s.find_first_of(".eEn") == std::string::npos) s += ".0";
    return s;
}

// Emit "dst |= ((src >> k) & mask) << p" terms mapping source bit k to
// destination position pos[k], grouping runs of consecutive positions.
void emit_deposit(std::ostringstream &o, const char *dst, const char *src, const int *pos, int nbits,
                  const char *type) {
    int k = 0;
    while (k < nbits) {
        int l = 1;
        while (k + l < nbits && pos[k + l] == pos[k] + l) ++l;
        const unsigned long long mask = (l >= 64) ? ~0ull : ((1ull << l) - 1);
        o << "  " << dst << " |= ((" << type << ")((" << src << " >> " << k << ") & " << mask << "ull)) << "
          << pos[k] << ";\n";
        k += l;
    }
}

uint32_t swz_host(uint32_t c) { return c ^ (((c >> 3) ^ (c >> 6) ^ (c >> 9)) & 7u); }

template <typename R>
struct Geo {
    int M, RB, NT, NR, EPC_LOG, NCH;
    explicit Geo(const TilePlan<R> &tp)
        : M(tp.m), RB(tp.rb), NT(1 << (tp.m - tp.rb)), NR(1 << tp.rb), EPC_LOG(sizeof(R) == 4 ? 1 : 0),
          NCH((1 << tp.m) >> (sizeof(R) == 4 ? 1 : 0)) {}
    static uint32_t phys(uint32_t j) {
        if (sizeof(R) == 4) return (swz_host(j >> 1) << 1) | (j & 1u);
        return swz_host(j);
    }
};

// Packed f32x2 additions for the real butterflies (H, SY and adjoints);
// SV_TILE_F32X2=0 emits scalar additions instead.
bool packed_adds_enabled() {
    const char *e = std::getenv("SV_TILE_F32X2");
    return !(e && e[0] == '0');
}



// Which ends of a pass go straight between HBM and registers: direct I/O on,
// complex64, and lanes of the first (last) segment that cover at least the 3
// lowest tile bits (8 lanes x 8 B: whole 32-byte sectors per warp access);
// otherwise that end is staged through shared memory with 16-byte copies.
struct HbmIo {
    bool load, store;
    int nseg;
    bool prefetch;  // persistent CTAs; the next tile's copy overlaps the last segment
};

template <typename R>
HbmIo hbm_io(const TilePlan<R> &tp, size_t pass) {
    const TilePassArgs &pa = tp.passes[pass];
    int first = -1, last = -1, nseg = 0;
    for (int i = pa.op_begin; i < pa.op_end; ++i)
        if (tp.ops[size_t(i)].type == TOP_SEG) {
            if (first < 0) first = tp.ops[size_t(i)].a;
            last = tp.ops[size_t(i)].a;
            ++nseg;
        }
    const bool on = sizeof(R) == 4 && tp.direct && first >= 0;
    auto contiguous = [&](int sidx) {
        const TileSeg &sg = tp.segs[size_t(sidx)];
        uint32_t lanes = 0;
        for (int k = 0; k < 5 && k < tp.m - tp.rb; ++k) lanes |= 1u << sg.tpos[k];
        return (lanes & 7u) == 7u && pa.lc >= 3;
    };
    // prefetch form: the last segment stores straight to HBM, so shared memory
    // is free from its gather on and takes the next tile's copy; the first
    // segment then gathers the copied tile from shared memory
    const bool store = on && contiguous(last);
    const bool prefetch = tp.prefetch && store && first >= 0;
    return HbmIo{on && contiguous(first) && !prefetch, store, nseg, prefetch};
}

template <typename R>
std::string gen_pass(const TilePlan<R> &tp, size_t pass) {
    const Geo<R> G(tp);
    const TilePassArgs &pa = tp.passes[pass];
    const char *RT = sizeof(R) == 4 ? "float" : "double";
    const char *C2T = sizeof(R) == 4 ? "float2" : "double2";
    std::ostringstream o;
    o << "typedef unsigned long long u64;\ntypedef unsigned int u32;\n";
    o << "__device__ __forceinline__ u32 swz(u32 c) { return c ^ (((c >> 3) ^ (c >> 6) ^ (c >> 9)) & 7u); }\n";
    if (sizeof(R) == 4) {
        // packed FP32 pairs: (re, im) of one amplitude as one 64-bit operand
        o << "__device__ __forceinline__ u64 pk(float x, float y) { u64 r; asm(\"mov.b64 %0, {%1, %2};\" : \"=l\"(r) : \"f\"(x), \"f\"(y)); return r; }\n"
             "__device__ __forceinline__ void upk(u64 r, float& x, float& y) { asm(\"mov.b64 {%0, %1}, %2;\" : \"=f\"(x), \"=f\"(y) : \"l\"(r)); }\n"
             "__device__ __forceinline__ u64 add2(u64 a, u64 b) { u64 d; asm(\"add.rn.f32x2 %0, %1, %2;\" : \"=l\"(d) : \"l\"(a), \"l\"(b)); return d; }\n"
             "__device__ __forceinline__ u64 sub2(u64 a, u64 b) { u64 d; asm(\"sub.rn.f32x2 %0, %1, %2;\" : \"=l\"(d) : \"l\"(a), \"l\"(b)); return d; }\n"
             "__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) { u64 d; asm(\"fma.rn.f32x2 %0, %1, %2, %3;\" : \"=l\"(d) : \"l\"(a), \"l\"(b), \"l\"(c)); return d; }\n";
    }
    o << "__device__ __forceinline__ void cpa16(void* s, const void* g) {\n"
         "  u32 sa = (u32)__cvta_generic_to_shared(s);\n"
         "  asm volatile(\"cp.async.cg.shared.global [%0], [%1], 16;\\n\" :: \"r\"(sa), \"l\"(g) : \"memory\");\n}\n";
    const int tbits = G.M - G.RB;  // bits of t
    const int iters = G.NCH / G.NT;
    const unsigned long long tile_bytes = (1ull << G.M) * 2 * sizeof(R);
    // chunk c = t + NT * i: chunk bit k <-> tile bit k + EPC_LOG <-> global tile_pos[k + EPC_LOG]
    std::vector<unsigned long long> gi(static_cast<size_t>(iters));
    std::vector<uint32_t> si(static_cast<size_t>(iters));
    for (int i = 0; i < iters; ++i) {
        const uint32_t c = uint32_t(i) * G.NT;
        unsigned long long g = 0;
        for (int k = 0; k < G.M; ++k)
            if (((c << G.EPC_LOG) >> k) & 1) g |= 1ull << pa.tile_pos[k];
        gi[size_t(i)] = g;
        si[size_t(i)] = swz_host(c);
    }
    int opos[kTileMaxOuter];
    for (int k = 0; k < pa.nouter; ++k) opos[k] = pa.outer_pos[k];
    // global outer-qubit mask -> the same bits of the tile (CTA) number
    auto compress = [&](unsigned long long g) {
        unsigned long long c = 0;
        for (int k = 0; k < pa.nouter; ++k)
            if (g >> opos[k] & 1) c |= 1ull << k;
        return c;
    };
    int tpos[kTileMaxQ];
    for (int k = 0; k < tbits; ++k) tpos[k] = pa.tile_pos[k + G.EPC_LOG];
    const int ctas = tp.pass_ctas.empty() ? tp.ctas : tp.pass_ctas[pass];
    o << "extern \"C\" __global__ void __launch_bounds__(" << G.NT << ", " << ctas << ") svp(" << C2T
      << "* __restrict__ psi, const u64 prm, const u64 ntiles) {\n";
    o << "  extern __shared__ __align__(16) unsigned char smem[];\n";
    o << "  " << C2T << "* sm = reinterpret_cast<" << C2T << "*>(smem);\n";
    // the CTA index is the tile number (persistent CTAs: the loop variable);
    // conditions on outer qubits test its bits, and the global offsets are
    // recomputed for the store (short live ranges leave the registers to the
    // amplitudes)
    o << "  const u32 t = threadIdx.x;\n";
    const HbmIo io = hbm_io(tp, pass);
    // the 16-byte copies of tile `tv` into the swizzled shared tile
    auto emit_tile_copy = [&](const char *tv) {
        o << "  {\n  u64 g0 = 0;\n";
        emit_deposit(o, "g0", tv, opos, pa.nouter, "u64");
        emit_deposit(o, "g0", "t", tpos, tbits, "u64");
        o << "  const u32 s0 = swz(t);\n";
        for (int i = 0; i < iters; ++i)
            o << "  cpa16(smem + ((s0 ^ " << si[size_t(i)] << "u) << 4), psi + (g0 | " << gi[size_t(i)] << "ull));\n";
        o << "  asm volatile(\"cp.async.commit_group;\\n\" ::: \"memory\");\n  }\n";
    };
    if (io.prefetch) {
        o << "  if (u64(blockIdx.x) >= ntiles) return;\n";
        emit_tile_copy("u64(blockIdx.x)");
        o << "  for (u64 cta = blockIdx.x; cta < ntiles; cta += gridDim.x) {\n";
        o << "  asm volatile(\"cp.async.wait_group 0;\\n\" ::: \"memory\");\n  __syncthreads();\n";
    } else {
        o << "  const u64 cta = blockIdx.x;\n";
    }
    if (!io.load && !io.prefetch) {
        o << "  {\n  u64 g0 = 0;\n";
        emit_deposit(o, "g0", "cta", opos, pa.nouter, "u64");
        emit_deposit(o, "g0", "t", tpos, tbits, "u64");
        o << "  const u32 s0 = swz(t);\n";
        for (int i = 0; i < iters; ++i)
            o << "  cpa16(smem + ((s0 ^ " << si[size_t(i)] << "u) << 4), psi + (g0 | " << gi[size_t(i)] << "ull));\n";
        o << "  }\n";
        o << "  asm volatile(\"cp.async.commit_group;\\ncp.async.wait_group 0;\\n\" ::: \"memory\");\n";
        o << "  __syncthreads();\n";
    }
    // Global offset of a segment's registers: the CTA's outer bits and the
    // thread's tile bits (at their global positions) in one per-thread base,
    // plus a constant per register slot (disjoint bits, so + is |).
    auto emit_thread_base = [&](const TileSeg &sg, const char *name) {
        int gpos[kTileMaxQ];
        for (int k = 0; k < tbits; ++k) gpos[k] = pa.tile_pos[sg.tpos[k]];
        o << "  u64 " << name << " = 0;\n";
        emit_deposit(o, name, "cta", opos, pa.nouter, "u64");
        emit_deposit(o, name, "t", gpos, tbits, "u64");
    };
    auto reg_goff = [&](const TileSeg &sg, int v) {
        unsigned long long g = 0;
        for (int sl = 0; sl < G.RB; ++sl)
            if (v >> sl & 1) g |= 1ull << pa.tile_pos[sg.rpos[sl]];
        return g;
    };
    const char *SYNC = "  __syncthreads();\n";
    o << "  " << RT << " xr[" << G.NR << "], xi[" << G.NR << "];\n  u32 jt = 0, pj = 0;\n";
    (void)0;

    int cur_seg = -1;
    bool first_seg = true;
    int seg_index = 0;
    uint32_t pv[kTileMaxRegs] = {0};
    // The stored value of register v is the amplitude divided by
    //   sgn[v] * prod(rsg[v]) * 2^(-me[v] / 2):
    // sgn: compile-time sign (unconditional sign flips such as CZ only flip
    //   it; butterflies fold it into add / sub choices);
    // rsg: runtime signs, a sign flip conditioned on thread / CTA bits
    //   becomes a per-thread factor sg<c> = cond ? -1 : 1 that the register
    //   still owes (equal lists need nothing in a butterfly, otherwise the
    //   relative factor enters as an FMA operand);
    // me: a magnitude exponent.  A phase (+-1 +- i) / sqrt(2) (T and its
    //   adjoint) is applied as the two additions of (+-1 +- i) and the
    //   1 / sqrt(2) is owed: the next butterfly on the register takes the
    //   relative factor 2^((me[v] - me[w]) / 2) as the multiplier of an FMA,
    //   which costs what the plain addition costs, and a scalar op or the
    //   scatter pays what is left.
    // rph: phases conditioned on thread / CTA bits, owed as one per-thread
    //   complex factor per distinct list (the running product of
    //   cond ? phase : 1), paid once per register when the register meets
    //   a register with another list, or at the scatter.
    int sgn[kTileMaxRegs], me[kTileMaxRegs];
    for (int v = 0; v < kTileMaxRegs; ++v) sgn[v] = 1, me[v] = 0;
    std::vector<int> rsg[kTileMaxRegs], rph[kTileMaxRegs];
    std::map<std::vector<int>, std::pair<std::string, std::string>> cph;  // list -> running product (re, im)
    std::map<std::pair<std::vector<int>, std::string>, std::pair<std::string, std::string>> kph;  // times a real factor
    int cph_id = 0;
    std::map<std::vector<int>, std::string> prod_name;
    auto prod = [&](const std::vector<int> &set) -> std::string {  // product of factors (CSE per segment)
        auto it = prod_name.find(set);
        if (it != prod_name.end()) return it->second;
        std::string nm = "rp" + std::to_string(prod_name.size()) + "_" + std::to_string(cur_seg);
        o << "  const " << RT << " " << nm << " = ";
        for (size_t i = 0; i < set.size(); ++i) o << (i ? " * " : "") << "sg" << set[i];
        o << ";\n";
        prod_name.emplace(set, nm);
        return nm;
    };
    std::map<std::pair<std::string, int>, std::string> scaled_name;
    // runtime factor f times the compile-time magnitude 2^(d/2) (CSE per segment)
    auto scaled = [&](const std::string &f, int d) -> std::string {
        if (d == 0) return f;
        auto key = std::make_pair(f, d);
        auto it = scaled_name.find(key);
        if (it != scaled_name.end()) return it->second;
        std::string nm = "rs" + std::to_string(scaled_name.size()) + "_" + std::to_string(cur_seg);
        o << "  const " << RT << " " << nm << " = " << f << " * " << lit(R(std::pow(2.0, d / 2.0)))
          << ";\n";
        scaled_name.emplace(key, nm);
        return nm;
    };
    auto mag = [](int d) { return std::pow(2.0, d / 2.0); };
    auto symdiff = [](const std::vector<int> &a, const std::vector<int> &b) {
        std::vector<int> d;
        std::set_symmetric_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(d));
        return d;
    };
    const bool packed = sizeof(R) == 4 && packed_adds_enabled();
    auto reg = [](const char *a, int v) { return std::string(a) + "[" + std::to_string(v) + "]"; };
    auto materialise = [&](int v) {
        if (!rph[v].empty()) {
            std::string f;  // real factor ("" for 1)
            if (!rsg[v].empty()) f = (sgn[v] < 0 ? "-" : "") + scaled(prod(rsg[v]), -me[v]);
            else if (me[v] != 0 || sgn[v] < 0) f = lit(R(sgn[v] * mag(-me[v])));
            const auto &c = cph.at(rph[v]);
            std::pair<std::string, std::string> k = c;
            if (!f.empty()) {
                auto key = std::make_pair(rph[v], f);
                auto it = kph.find(key);
                if (it == kph.end()) {
                    const std::string nm = "pk" + std::to_string(cph_id++) + "_" + std::to_string(cur_seg);
                    o << "  const " << RT << " " << nm << "r = " << c.first << " * " << f << ", " << nm << "i = "
                      << c.second << " * " << f << ";\n";
                    it = kph.emplace(key, std::make_pair(nm + "r", nm + "i")).first;
                }
                k = it->second;
            }
            const std::string x = reg("xr", v), y = reg("xi", v);
            o << "  { const " << RT << " r = " << x << " * " << k.first << " - " << y << " * " << k.second << "; " << y
              << " = " << x << " * " << k.second << " + " << y << " * " << k.first << "; " << x << " = r; }\n";
        } else if (!rsg[v].empty()) {
            const std::string f = scaled(prod(rsg[v]), -me[v]);
            const char *neg = sgn[v] < 0 ? "-" : "";
            o << "  " << reg("xr", v) << " *= " << neg << f << "; " << reg("xi", v) << " *= " << neg << f << ";\n";
        } else if (me[v] != 0) {
            const std::string f = lit(R(sgn[v] * mag(-me[v])));
            o << "  " << reg("xr", v) << " *= " << f << "; " << reg("xi", v) << " *= " << f << ";\n";
        } else if (sgn[v] < 0) {
            o << "  " << reg("xr", v) << " = -" << reg("xr", v) << "; " << reg("xi", v) << " = -" << reg("xi", v) << ";\n";
        }
        rsg[v].clear();
        rph[v].clear();
        sgn[v] = 1;
        me[v] = 0;
    };
    auto scatter = [&]() {
        for (int v = 0; v < G.NR; ++v) {
            if (!rsg[v].empty() || !rph[v].empty() || me[v] != 0) materialise(v);
            const char *neg = sgn[v] < 0 ? "-" : "";
            o << "  sm[pj ^ " << pv[v] << "u] = make_" << C2T << "(" << neg << "xr[" << v << "], " << neg << "xi[" << v
              << "]);\n";
            sgn[v] = 1;
        }
        prod_name.clear();
        scaled_name.clear();
        cph.clear();
        kph.clear();
    };
    // x + s * m * y with s = +-1 and multiplier string m ("" for 1): an
    // addition, or one FMA
    auto axpy = [&](int sx, const std::string &x, int sy, const std::string &m, const std::string &y) {
        const std::string nx = sx < 0 ? "-" : "";
        if (m.empty()) return (sx < 0 ? "-" + x : x) + (sy < 0 ? " - " : " + ") + y;
        return "fma(" + std::string(sy < 0 ? "-" : "") + m + ", " + y + ", " + nx + x + ")";
    };
    int cond_id = 0;
    for (int i = pa.op_begin; i < pa.op_end; ++i) {
        const TileOp<R> &op = tp.ops[size_t(i)];
        if (op.type == TOP_SEG) {
            if (cur_seg >= 0) {
                scatter();
                o << SYNC;
            }
            cur_seg = op.a;
            const TileSeg &sg = tp.segs[size_t(op.a)];
            int pos[kTileMaxQ];
            for (int k = 0; k < tbits; ++k) pos[k] = sg.tpos[k];
            o << "  jt = 0;\n";
            emit_deposit(o, "jt", "t", pos, tbits, "u32");
            if (sizeof(R) == 4) o << "  pj = (swz(jt >> 1) << 1) | (jt & 1u);\n";
            else o << "  pj = swz(jt);\n";
            const bool from_hbm = io.load && first_seg;
            first_seg = false;
            ++seg_index;
            const bool last_seg = seg_index == io.nseg;
            if (from_hbm) {
                o << "  {\n";
                emit_thread_base(sg, "gq");
            }
            for (int v = 0; v < G.NR; ++v) {
                uint32_t d = 0;
                for (int s = 0; s < G.RB; ++s)
                    if (v >> s & 1) d |= 1u << sg.rpos[s];
                pv[v] = Geo<R>::phys(d);
                if (from_hbm)
                    o << "  { const " << C2T << " a = psi[gq + " << reg_goff(sg, v) << "ull]; xr[" << v
                      << "] = a.x; xi[" << v << "] = a.y; }\n";
                else
                    o << "  { " << C2T << " a = sm[pj ^ " << pv[v] << "u]; xr[" << v << "] = a.x; xi[" << v
                      << "] = a.y; }\n";
            }
            if (from_hbm) o << "  }\n";
            if (io.prefetch && last_seg) {
                // every thread has gathered the tile: shared memory takes the
                // next tile's copy while this segment computes and stores
                o << "  __syncthreads();\n  if (cta + gridDim.x < ntiles) {\n  const u64 nxt = cta + gridDim.x;\n";
                emit_tile_copy("nxt");
                o << "  }\n";
            }
            continue;
        }
        // runtime condition on thread / CTA bits (branch-free select)
        std::string cond;
        int cid = -1;
        if (op.tmask || op.gmask || op.pmask) {
            cid = cond_id++;
            cond = "c" + std::to_string(cid);
            o << "  const bool " << cond << " = ((jt & " << op.tmask << "u) == " << op.tval << "u) && ((cta & "
              << compress(op.gmask) << "ull) == " << compress(op.gval) << "ull)";
            if (op.pmask) o << " && ((prm & " << op.pmask << "ull) == " << op.pval << "ull)";
            o << ";\n";
            if (op.type == TOP_NEG) o << "  const " << RT << " sg" << cid << " = " << cond << " ? " << RT << "(-1) : " << RT << "(1);\n";
        }
        auto sel = [&](const std::string &v_new, const std::string &v_old) {
            return cond.empty() ? v_new : ("(" + cond + " ? " + v_new + " : " + v_old + ")");
        };
        if (op.type == TOP_SCALE) {
            // the scalar, the compile-time sign and the owed magnitude of each
            // register in one multiplication
            for (int v = 0; v < G.NR; ++v) {
                const double f = sgn[v] * mag(-me[v]);
                const R pr = R(double(op.u[0]) * f), pi = R(double(op.u[1]) * f);
                const std::string x = reg("xr", v), y = reg("xi", v);
                if (pi == R(0))
                    o << "  " << x << " *= " << lit(pr) << "; " << y << " *= " << lit(pr) << ";\n";
                else if (pr == R(0))
                    o << "  { const " << RT << " r = " << y << " * " << lit(R(-pi)) << "; " << y << " = " << x << " * "
                      << lit(pi) << "; " << x << " = r; }\n";
                else
                    o << "  { " << RT << " r = " << x << " * " << lit(pr) << " - " << y << " * " << lit(pi) << "; " << y
                      << " = " << x << " * " << lit(pi) << " + " << y << " * " << lit(pr) << "; " << x << " = r; }\n";
                sgn[v] = 1;
                me[v] = 0;
            }
            continue;
        }
        if (op.type == TOP_PHASE || op.type == TOP_NEG) {
            const uint32_t M = uint32_t(op.a) / kTileMaxRegs, V = uint32_t(op.a) % kTileMaxRegs;
            const std::string pr = lit(op.u[0]), pi = lit(op.u[1]);
            // (+-1 +- i) / sqrt(2): two additions, the magnitude is owed
            const double ar = std::fabs(double(op.u[0])), ai = std::fabs(double(op.u[1]));
            const bool eighth = cond.empty() && ar > 0.5 && std::fabs(ar - ai) <= 4e-7 * ar &&
                                std::fabs(ar - std::sqrt(0.5)) <= 4e-7;
            const int s0 = op.u[0] < 0 ? -1 : 1, s1 = op.u[1] < 0 ? -1 : 1;
            if (op.type == TOP_PHASE && !cond.empty()) {
                // per-thread factor; each distinct list of the affected
                // registers gets its running product once
                const std::string ph = "ph" + std::to_string(cid);
                o << "  const " << RT << " " << ph << "r = " << cond << " ? " << RT << "(" << pr << ") : " << RT << "(1), "
                  << ph << "i = " << cond << " ? " << RT << "(" << pi << ") : " << RT << "(0);\n";
                for (int v = 0; v < G.NR; ++v) {
                    if ((uint32_t(v) & M) != V) continue;
                    std::vector<int> nl = rph[v];
                    nl.insert(std::lower_bound(nl.begin(), nl.end(), cid), cid);
                    if (!cph.count(nl)) {
                        if (rph[v].empty()) {
                            cph.emplace(nl, std::make_pair(ph + "r", ph + "i"));
                        } else {
                            const auto &c = cph.at(rph[v]);
                            const std::string nm = "pc" + std::to_string(cph_id++) + "_" + std::to_string(cur_seg);
                            o << "  const " << RT << " " << nm << "r = " << c.first << " * " << ph << "r - " << c.second
                              << " * " << ph << "i, " << nm << "i = " << c.first << " * " << ph << "i + " << c.second
                              << " * " << ph << "r;\n";
                            cph.emplace(nl, std::make_pair(nm + "r", nm + "i"));
                        }
                    }
                    rph[v] = nl;
                }
                continue;
            }
            for (int v = 0; v < G.NR; ++v) {
                if ((uint32_t(v) & M) != V) continue;
                const std::string x = "xr[" + std::to_string(v) + "]", y = "xi[" + std::to_string(v) + "]";
                if (op.type == TOP_NEG) {
                    if (cond.empty()) sgn[v] = -sgn[v];
                    else {
                        auto &r = rsg[v];
                        auto it = std::lower_bound(r.begin(), r.end(), cid);
                        r.insert(it, cid);
                    }
                } else if (eighth) {
                    // (s0 + i s1)(x + i y) = (s0 x - s1 y) + i (s1 x + s0 y)
                    o << "  { const " << RT << " r = " << axpy(s0, x, -s1, "", y) << "; " << y << " = "
                      << axpy(s1, x, s0, "", y) << "; " << x << " = r; }\n";
                    me[v] += 1;
                } else {
                    o << "  { " << RT << " r = " << x << " * " << pr << " - " << y << " * " << pi << "; " << RT
                      << " q = " << x << " * " << pi << " + " << y << " * " << pr << "; " << x << " = "
                      << sel("r", x) << "; " << y << " = " << sel("q", y) << "; }\n";
                }
            }
            continue;
        }
        const int slot = op.type == TOP_STRUCT ? (op.a & 255) : op.a;
        const int kind = op.type == TOP_STRUCT ? (op.a >> 8) : -1;
        for (int v = 0; v < G.NR; ++v) {
            if (v >> slot & 1) continue;
            if ((uint32_t(v) & op.rmask) != op.rval) continue;
            const int w = v | (1 << slot);
            const std::string ar = reg("xr", v), ai = reg("xi", v), br = reg("xr", w), bi = reg("xi", w);
            if (!cond.empty()) {  // runtime condition: plain values, select old / new
                materialise(v);
                materialise(w);
            }
            if (op.type == TOP_G1 && rsg[v] != rsg[w]) {  // general matrices: plain values
                materialise(v);
                materialise(w);
            }
            if (rph[v] != rph[w]) {  // complex relative factors are paid first
                materialise(v);
                materialise(w);
            }
            if (op.type == TOP_STRUCT && kind == SK_X && cond.empty()) {
                o << "  { const " << RT << " t0 = " << ar << ", t1 = " << ai << "; " << ar << " = " << br << "; " << ai
                  << " = " << bi << "; " << br << " = t0; " << bi << " = t1; }\n";
                std::swap(sgn[v], sgn[w]);
                std::swap(rsg[v], rsg[w]);
                std::swap(rph[v], rph[w]);
                std::swap(me[v], me[w]);
                continue;
            }
            const int sa = sgn[v], sb = sgn[w], r = sa * sb;
            // b's stored value times 2^(dm / 2) is on a's magnitude scale
            const int dm = me[v] - me[w];
            // relative runtime factor of b with respect to a ("" when the lists agree)
            const std::vector<int> rel = symdiff(rsg[v], rsg[w]);
            const std::string rf = rel.empty() ? std::string() : prod(rel);
            // multiplier of b: runtime factor and magnitude ("" for 1)
            const std::string mb = rf.empty() ? (dm == 0 ? std::string() : lit(R(mag(dm)))) : scaled(rf, dm);
            if (op.type == TOP_STRUCT && (kind == SK_H || kind == SK_SY || kind == SK_SYD) && cond.empty()) {
                // true a' = sa (m00 A + m01 r B), b' = sa (m10 A + m11 r B); each is
                // +-(A + B) or +-(A - B), one of each
                static const int M[3][4] = {{1, 1, 1, -1}, {1, -1, 1, 1}, {1, 1, -1, 1}};
                const int *m = M[kind == SK_H ? 0 : (kind == SK_SY ? 1 : 2)];
                const bool a_plus = m[0] * m[1] * r > 0;   // A' = m00 (A + e B)
                sgn[v] = sa * m[0];
                sgn[w] = sa * m[2];
                rsg[w] = rsg[v];
                me[w] = me[v];
                if (!mb.empty()) {  // A' = A + e mb B, B' = A - e mb B
                    const std::string e1 = a_plus ? "" : "-";
                    const std::string e2 = a_plus ? "-" : "";
                    if (packed) {
                        o << "  { const u64 a = pk(" << ar << ", " << ai << "), b = pk(" << br << ", " << bi << "); "
                          << "upk(fma2(b, pk(" << e1 << mb << ", " << e1 << mb << "), a), " << ar << ", " << ai << "); "
                          << "upk(fma2(b, pk(" << e2 << mb << ", " << e2 << mb << "), a), " << br << ", " << bi << "); }\n";
                    } else {
                        o << "  { const " << RT << " a0 = " << ar << ", a1 = " << ai << ", b0 = " << br << ", b1 = " << bi
                          << "; " << ar << " = fma(" << e1 << mb << ", b0, a0); " << ai << " = fma(" << e1 << mb
                          << ", b1, a1); " << br << " = fma(" << e2 << mb << ", b0, a0); " << bi << " = fma(" << e2
                          << mb << ", b1, a1); }\n";
                    }
                    continue;
                }
                if (packed) {
                    o << "  { const u64 a = pk(" << ar << ", " << ai << "), b = pk(" << br << ", " << bi << "); upk("
                      << (a_plus ? "add2" : "sub2") << "(a, b), " << ar << ", " << ai << "); upk("
                      << (a_plus ? "sub2" : "add2") << "(a, b), " << br << ", " << bi << "); }\n";
                } else {
                    const char *p1 = a_plus ? " + " : " - ", *p2 = a_plus ? " - " : " + ";
                    o << "  { const " << RT << " a0 = " << ar << ", a1 = " << ai << ", b0 = " << br << ", b1 = " << bi
                      << "; " << ar << " = a0" << p1 << "b0; " << ai << " = a1" << p1 << "b1; " << br << " = a0" << p2
                      << "b0; " << bi << " = a1" << p2 << "b1; }\n";
                }
                continue;
            }
            std::string nar, nai, nbr, nbi;
            if (op.type == TOP_G1) {
                // signs and b's magnitude folded into the constants:
                // a' = u00 sa A + u01 sb mag B, ...
                std::string u[8];
                for (int k = 0; k < 8; ++k) {
                    const bool bcol = !(k == 0 || k == 1 || k == 4 || k == 5);
                    const double f = bcol ? sb * mag(dm) : sa;
                    u[k] = lit(R(f * double(op.u[k])));
                }
                nar = u[0] + "*ar - " + u[1] + "*ai + " + u[2] + "*br - " + u[3] + "*bi";
                nai = u[0] + "*ai + " + u[1] + "*ar + " + u[2] + "*bi + " + u[3] + "*br";
                nbr = u[4] + "*ar - " + u[5] + "*ai + " + u[6] + "*br - " + u[7] + "*bi";
                nbi = u[4] + "*ai + " + u[5] + "*ar + " + u[6] + "*bi + " + u[7] + "*br";
                sgn[v] = sgn[w] = 1;
                rsg[w] = rsg[v];  // equal lists here (else materialised above)
                me[w] = me[v];
            } else {
                // stored results relative to sign sa and magnitude me[v] for
                // both outputs; the b terms carry the multiplier mb
                switch (kind) {
                    case SK_H:
                        nar = axpy(1, "ar", r, mb, "br"); nai = axpy(1, "ai", r, mb, "bi");
                        nbr = axpy(1, "ar", -r, mb, "br"); nbi = axpy(1, "ai", -r, mb, "bi"); break;
                    case SK_SY:
                        nar = axpy(1, "ar", -r, mb, "br"); nai = axpy(1, "ai", -r, mb, "bi");
                        nbr = axpy(1, "ar", r, mb, "br"); nbi = axpy(1, "ai", r, mb, "bi"); break;
                    case SK_SYD:
                        nar = axpy(1, "ar", r, mb, "br"); nai = axpy(1, "ai", r, mb, "bi");
                        nbr = axpy(-1, "ar", r, mb, "br"); nbi = axpy(-1, "ai", r, mb, "bi"); break;
                    case SK_SX:  // (A - i r B, -i A + r B)
                        nar = axpy(1, "ar", r, mb, "bi"); nai = axpy(1, "ai", -r, mb, "br");
                        nbr = axpy(1, "ai", r, mb, "br"); nbi = axpy(-1, "ar", r, mb, "bi"); break;
                    case SK_SXD:  // (A + i r B, i A + r B)
                        nar = axpy(1, "ar", -r, mb, "bi"); nai = axpy(1, "ai", r, mb, "br");
                        nbr = axpy(-1, "ai", r, mb, "br"); nbi = axpy(1, "ar", r, mb, "bi"); break;
                    default:  // X under a runtime condition (plain values here)
                        nar = "br"; nai = "bi"; nbr = "ar"; nbi = "ai"; break;
                }
                sgn[w] = sa;
                rsg[w] = rsg[v];
                me[w] = me[v];
            }
            o << "  { const " << RT << " ar = " << ar << ", ai = " << ai << ", br = " << br << ", bi = " << bi << "; "
              << ar << " = " << sel(nar, "ar") << "; " << ai << " = " << sel(nai, "ai") << "; " << br << " = "
              << sel(nbr, "br") << "; " << bi << " = " << sel(nbi, "bi") << "; }\n";
        }
    }
    if (io.store) {
        // the last segment's registers go straight back to HBM
        if (cur_seg >= 0) {
            const TileSeg &sg = tp.segs[size_t(cur_seg)];
            o << "  {\n";
            emit_thread_base(sg, "gq");
            for (int v = 0; v < G.NR; ++v) {
                if (!rsg[v].empty() || !rph[v].empty() || me[v] != 0) materialise(v);
                const char *neg = sgn[v] < 0 ? "-" : "";
                o << "  psi[gq + " << reg_goff(sg, v) << "ull] = make_" << C2T << "(" << neg << "xr[" << v << "], "
                  << neg << "xi[" << v << "]);\n";
                sgn[v] = 1;
            }
            o << "  }\n";
        }
        if (io.prefetch) o << "  }\n";  // the tile loop
        o << "}\n";
        return o.str();
    }
    if (cur_seg >= 0) {
        scatter();
        o << SYNC;
    }
    o << "  {\n  u64 g0 = 0;\n";
    emit_deposit(o, "g0", "t", tpos, tbits, "u64");
    emit_deposit(o, "g0", "cta", opos, pa.nouter, "u64");
    o << "  const u32 s0 = swz(t);\n";
    for (int i = 0; i < iters; ++i)
        o << "  *reinterpret_cast<int4*>(psi + (g0 | " << gi[size_t(i)] << "ull)) = *reinterpret_cast<const int4*>(smem + ((s0 ^ "
          << si[size_t(i)] << "u) << 4));\n";
    o << "  }\n";
    o << "}\n";
    return o.str();
}

// ---------------------------------------------------------------- NVRTC cache
struct JitEntry {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t fn = nullptr;
};

std::mutex g_jit_mu;
std::unordered_map<std::string, JitEntry> g_jit;  // key: device + source
// per compiled pass: its dynamic shared memory, and for persistent passes the
// CTAs per SM of the grid (0: one CTA per tile)
struct PassLaunch {
    int smem = 0;
    int persistent_ctas = 0;
    int m = 0;  // tile bits
};
std::unordered_map<const void *, PassLaunch> g_jit_smem;

// Shared memory a generated pass uses: the whole tile, unless direct HBM I/O
// leaves it nothing to do (at most one segment).
template <typename R>
int pass_smem_bytes(const TilePlan<R> &tp, size_t pass) {
    const HbmIo io = hbm_io(tp, pass);
    return io.load && io.store && io.nseg <= 1 && !io.prefetch ? 0 : (1 << tp.m) * int(2 * sizeof(R));
}

bool jit_verbose() {
    const char *ve = std::getenv("SV_JIT_VERBOSE");
    return ve && ve[0] == '1';
}

// In-process NVRTC compile of one pass (SV_JIT_VERBOSE=1 prints ptxas
// resource usage, registers and spills, to stderr).
std::string compile_cubin(const std::string &src, std::string *err) {
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "sv_pass.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        *err = "nvrtcCreateProgram failed";
        return {};
    }
    const bool verbose = jit_verbose();
    const nvrtcResult r = nvrtcCompileProgram(prog, verbose ? kPassNvrtcOptsVerbose : kPassNvrtcOptsQuiet,
                                              kPassNvrtcOpts);
    if (verbose) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        nvrtcGetProgramLog(prog, &log[0]);
        std::fprintf(stderr, "%s\n", log.c_str());
    }
    std::string cubin;
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        nvrtcGetProgramLog(prog, &log[0]);
        *err = std::string(nvrtcGetErrorString(r)) + ": " + log.substr(0, 400);
    } else {
        size_t n = 0;
        nvrtcGetCUBINSize(prog, &n);
        cubin.resize(n);
        nvrtcGetCUBIN(prog, &cubin[0]);
    }
    nvrtcDestroyProgram(&prog);
    return cubin;
}

// ---------------------------------------------------------------- compile workers
// NVRTC serialises compilations inside one process (threads do not overlap),
// so passes compile in separate worker processes, several at once: the
// executable sv_nvrtc_worker next to this library (SV_JIT_WORKER overrides
// the path; SV_JIT_PROCS=0 compiles in-process).  The worker runs the same
// NVRTC with the same options, so the cubins are the same.  posix_spawn
// starts it without copying this process (safe with the CUDA context and
// other threads).  If no worker can be started, the compile runs in-process.

void jit_anchor() {}

std::string worker_path() {
    const char *procs = std::getenv("SV_JIT_PROCS");
    if (procs && procs[0] == '0') return std::string();
    if (const char *w = std::getenv("SV_JIT_WORKER")) return std::string(w);
    static const std::string beside_library = [] {
        Dl_info info;
        if (!dladdr(reinterpret_cast<void *>(&jit_anchor), &info) || !info.dli_fname) return std::string();
        const std::string lib = info.dli_fname;
        const size_t slash = lib.rfind('/');
        const std::string dir = slash == std::string::npos ? std::string(".") : lib.substr(0, slash);
        return dir + "/sv_nvrtc_worker";
    }();
    return beside_library;
}

std::string read_file(const std::string &path) {
    std::string out;
    if (FILE *f = std::fopen(path.c_str(), "rb")) {
        char buf[65536];
        size_t n;
        while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) out.append(buf, n);
        std::fclose(f);
    }
    return out;
}

std::string cache_dir();

// Compile src in a worker.  Returns false if no worker could be started (the
// caller compiles in-process); true otherwise, with *cubin set, or empty and
// *err set when the compile itself failed.
bool compile_in_worker(const std::string &src, std::string *cubin, std::string *err) {
    const std::string worker = worker_path();
    if (worker.empty() || access(worker.c_str(), X_OK) != 0) return false;
    // scratch files beside the disk cache when there is one, else in TMPDIR or /tmp
    const std::string cache = cache_dir();
    const char *tmp = std::getenv("TMPDIR");
    std::string dir = (!cache.empty() ? cache : std::string(tmp && tmp[0] ? tmp : "/tmp")) + "/sv_jit_XXXXXX";
    if (!mkdtemp(&dir[0])) return false;
    const std::string src_path = dir + "/pass.cu", out_path = dir + "/pass.cubin", log_path = dir + "/log";
    bool started = false;
    if (FILE *f = std::fopen(src_path.c_str(), "wb")) {
        const bool ok = std::fwrite(src.data(), 1, src.size(), f) == src.size();
        if (std::fclose(f) == 0 && ok) {
            const bool verbose = jit_verbose();
            posix_spawn_file_actions_t fa;
            posix_spawn_file_actions_init(&fa);
            posix_spawn_file_actions_addopen(&fa, 0, "/dev/null", O_RDONLY, 0);
            posix_spawn_file_actions_addopen(&fa, 1, "/dev/null", O_WRONLY, 0);
            if (!verbose) posix_spawn_file_actions_addopen(&fa, 2, log_path.c_str(), O_WRONLY | O_CREAT | O_TRUNC, 0600);
            std::string a0 = worker, a1 = src_path, a2 = out_path, a3 = verbose ? "1" : "0";
            char *argv[] = {&a0[0], &a1[0], &a2[0], &a3[0], nullptr};
            pid_t pid = 0;
            if (posix_spawn(&pid, worker.c_str(), &fa, nullptr, argv, environ) == 0) {
                int status = 0;
                pid_t w;
                do {
                    w = waitpid(pid, &status, 0);
                } while (w < 0 && errno == EINTR);
                if (w == pid) {
                    started = true;
                    if (WIFEXITED(status) && WEXITSTATUS(status) == 0) {
                        *cubin = read_file(out_path);
                        if (cubin->empty()) *err = "the compile worker wrote no cubin";
                    } else {
                        *err = "compile worker failed: " + read_file(log_path).substr(0, 400);
                    }
                }
            }
            posix_spawn_file_actions_destroy(&fa);
        }
    }
    std::remove(src_path.c_str());
    std::remove(out_path.c_str());
    std::remove(log_path.c_str());
    rmdir(dir.c_str());
    return started;
}

// ---------------------------------------------------------------- disk cache
// Compiled passes persist across processes: one file per pass source under
// SV_JIT_CACHE (a directory; "0" turns the cache off), by default the folder
// _jit_cache beside this library.  The file name hashes the host machine,
// the NVRTC version, the options and the source; the file holds the source
// and the cubin, and a load is taken only when the stored source equals the
// current one byte for byte (a hash collision or a damaged file is a miss).
// Files are written under a temporary name and renamed into place, so a
// reader never sees a partial one.

constexpr char kCacheMagic[] = "SVJIT1\n";

std::string cache_dir() {
    const char *e = std::getenv("SV_JIT_CACHE");
    if (e && e[0] == '0' && e[1] == '\0') return std::string();
    std::string dir;
    if (e && e[0]) {
        dir = e;
    } else {
        Dl_info info;
        if (!dladdr(reinterpret_cast<void *>(&jit_anchor), &info) || !info.dli_fname) return std::string();
        const std::string lib = info.dli_fname;
        const size_t slash = lib.rfind('/');
        dir = (slash == std::string::npos ? std::string(".") : lib.substr(0, slash)) + "/_jit_cache";
    }
    // create the directory and its missing parents (0700)
    for (size_t k = 1; k <= dir.size(); ++k)
        if (k == dir.size() || dir[k] == '/') mkdir(dir.substr(0, k).c_str(), 0700);
    struct stat st;
    if (stat(dir.c_str(), &st) != 0 || !S_ISDIR(st.st_mode) || access(dir.c_str(), W_OK | X_OK) != 0)
        return std::string();
    return dir;
}

std::string cache_file(const std::string &dir, const std::string &src) {
    int major = 0, minor = 0;
    nvrtcVersion(&major, &minor);
    struct utsname un;
    std::string tag = std::string(uname(&un) == 0 ? un.machine : "?") + " nvrtc " + std::to_string(major) + "." +
                      std::to_string(minor);
    for (int i = 0; i < kPassNvrtcOptsQuiet; ++i) tag += std::string(" ") + kPassNvrtcOpts[i];
    uint64_t h = 1469598103934665603ull;  // FNV-1a, 64 bits
    const std::string *parts[] = {&tag, &src};
    for (const std::string *part : parts)
        for (unsigned char ch : *part) h = (h ^ ch) * 1099511628211ull;
    char name[40];
    std::snprintf(name, sizeof name, "/%016llx.bin", static_cast<unsigned long long>(h));
    return dir + name;
}

bool cache_load(const std::string &path, const std::string &src, std::string *cubin) {
    const std::string data = read_file(path);
    const std::string head = std::string(kCacheMagic) + std::to_string(src.size()) + "\n";
    if (data.size() <= head.size() + src.size() || data.compare(0, head.size(), head) != 0 ||
        data.compare(head.size(), src.size(), src) != 0)
        return false;
    *cubin = data.substr(head.size() + src.size());
    return true;
}

void cache_store(const std::string &path, const std::string &src, const std::string &cubin) {
    static std::atomic<uint64_t> seq{0};
    const std::string tmp = path + ".tmp" + std::to_string(getpid()) + "." + std::to_string(seq.fetch_add(1));
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;
    const std::string head = std::string(kCacheMagic) + std::to_string(src.size()) + "\n";
    bool ok = std::fwrite(head.data(), 1, head.size(), f) == head.size();
    ok = ok && std::fwrite(src.data(), 1, src.size(), f) == src.size();
    ok = ok && std::fwrite(cubin.data(), 1, cubin.size(), f) == cubin.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) std::remove(tmp.c_str());
}

// Compile one pass: from the disk cache, else in a worker, else in-process.
// SV_JIT_VERBOSE=1 with SV_JIT_DUMP=<file> appends the generated source to
// that file.
std::string compile_pass(const std::string &src, std::string *err) {
    if (jit_verbose() && std::getenv("SV_JIT_DUMP")) {
        static std::mutex dump_mu;
        std::lock_guard<std::mutex> lock(dump_mu);
        if (FILE *f = std::fopen(std::getenv("SV_JIT_DUMP"), "a")) {
            std::fputs(src.c_str(), f);
            std::fclose(f);
        }
    }
    const std::string dir = cache_dir();
    const std::string path = dir.empty() ? std::string() : cache_file(dir, src);
    std::string cubin;
    if (!path.empty() && !jit_verbose() && cache_load(path, src, &cubin)) return cubin;
    if (!compile_in_worker(src, &cubin, err)) cubin = compile_cubin(src, err);
    if (!path.empty() && !cubin.empty()) cache_store(path, src, cubin);
    return cubin;
}

// Compile src[j] for every j in todo, as many at once as there are hardware
// threads; cubin[j] empty and err[j] set for a failure.
void compile_many(const std::vector<std::string> &src, const std::vector<int> &todo, std::vector<std::string> *cubin,
                  std::vector<std::string> *err) {
    const unsigned hw = std::thread::hardware_concurrency();
    const size_t nthreads = std::min<size_t>(todo.size(), hw ? hw : 4);
    std::vector<std::thread> pool;
    size_t next = 0;
    std::mutex qmu;
    for (size_t k = 0; k < nthreads; ++k)
        pool.emplace_back([&]() {
            for (;;) {
                size_t j;
                {
                    std::lock_guard<std::mutex> l(qmu);
                    if (next >= todo.size()) return;
                    j = size_t(todo[next++]);
                }
                (*cubin)[j] = compile_pass(src[j], &(*err)[j]);
            }
        });
    for (auto &th : pool) th.join();
}

template <typename R>
sv_status jit_plan_impl(const TilePlan<R> &tp, std::vector<void *> *fns) {
    // make sure the runtime has made the primary context current
    SV_CUDA_TRY(cudaFree(nullptr));
    int dev = 0;
    SV_CUDA_TRY(cudaGetDevice(&dev));
    const size_t np = tp.passes.size();
    std::vector<std::string> src(np), key(np), cubin(np), err(np);
    std::vector<int> todo;
    fns->assign(np, nullptr);
    {
        std::lock_guard<std::mutex> lock(g_jit_mu);
        for (size_t i = 0; i < np; ++i) {
            src[i] = gen_pass(tp, i);
            key[i] = std::to_string(dev) + "\n" + src[i];
            auto it = g_jit.find(key[i]);
            if (it != g_jit.end()) (*fns)[i] = reinterpret_cast<void *>(it->second.fn);
            else todo.push_back(int(i));
        }
    }
    // compile the misses in parallel (NVRTC programs are independent)
    compile_many(src, todo, &cubin, &err);
    for (int j : todo) {
        if (cubin[size_t(j)].empty()) {
            set_error("NVRTC compile of pass %d failed: %s", j, err[size_t(j)].c_str());
            return SV_ERR_CUDA;
        }
    }
    std::lock_guard<std::mutex> lock(g_jit_mu);
    for (int j : todo) {
        auto it = g_jit.find(key[size_t(j)]);
        if (it == g_jit.end()) {
            JitEntry e;
            cudaError_t ce = cudaLibraryLoadData(&e.lib, cubin[size_t(j)].data(), nullptr, nullptr, 0, nullptr,
                                                 nullptr, 0);
            if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&e.fn, e.lib, "svp");
            const int smem = pass_smem_bytes(tp, size_t(j));
            // a cudaKernel_t is accepted wherever a kernel symbol is
            if (ce == cudaSuccess && smem > 0)
                ce = cudaFuncSetAttribute(reinterpret_cast<const void *>(e.fn),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (ce != cudaSuccess) return cuda_status(ce, "loading a compiled pass");
            it = g_jit.emplace(key[size_t(j)], e).first;
            g_jit_smem[reinterpret_cast<const void *>(e.fn)] =
                PassLaunch{smem,
                           hbm_io(tp, size_t(j)).prefetch ? (tp.pass_ctas.empty() ? tp.ctas : tp.pass_ctas[size_t(j)]) : 0,
                           tp.m};
        }
        (*fns)[size_t(j)] = reinterpret_cast<void *>(it->second.fn);
    }
    return SV_OK;
}

template <typename R>
sv_status compile_check_impl(const TilePlan<R> &tp) {
    const size_t np = tp.passes.size();
    std::vector<std::string> src(np), cubin(np), err(np);
    std::vector<int> todo(np);
    for (size_t i = 0; i < np; ++i) {
        src[i] = gen_pass(tp, i);
        todo[i] = int(i);
    }
    compile_many(src, todo, &cubin, &err);
    for (size_t i = 0; i < np; ++i)
        if (cubin[i].empty()) {
            set_error("NVRTC compile of pass %zu failed: %s", i, err[i].c_str());
            return SV_ERR_CUDA;
        }
    return SV_OK;
}

}  // namespace

// Direct HBM I/O: the first segment loads its register amplitudes straight
// from global memory and the last one stores them straight back, so shared
// memory carries only the transpositions between segments (a one-segment
// pass uses none).  SV_TILE_DIRECT=0 stages the whole tile through shared
// memory with cp.async on the way in and out instead.  complex64 only (the
// complex128 passes keep the staged form).
bool direct_io_enabled() {
    const char *e = std::getenv("SV_TILE_DIRECT");
    return !(e && e[0] == '0');
}

// CTAs per SM the pass kernels are compiled for (register budget); the
// shared tile (64 KiB) allows up to 3, a 2^12 tile (32 KiB) 4 and more.
// SV_TILE_CTAS overrides (1 to 4).
int tile_ctas_per_sm() {
    const char *e = std::getenv("SV_TILE_CTAS");
    const int v = e ? std::atoi(e) : 2;
    return v >= 1 && v <= 4 ? v : 2;
}

// Persistent prefetching passes (SV_TILE_PREFETCH=1; off by default, a
// candidate of the autotuner).
bool prefetch_enabled() {
    const char *e = std::getenv("SV_TILE_PREFETCH");
    return e && e[0] == '1';
}

// Tile bits of complex64 passes (SV_TILE_M overrides, 12 or 13).
int tile_m64() {
    const char *e = std::getenv("SV_TILE_M");
    const int v = e ? std::atoi(e) : kTileM64;
    return v == 12 || v == 13 ? v : kTileM64;
}

TileConfig tile_config64(int rb, int ctas, int direct, int prefetch, int m) {
    TileConfig c{m ? m : tile_m64(), rb ? rb : tile_rb64(), tile_low64(), true};
    c.ctas = ctas ? ctas : tile_ctas_per_sm();
    c.direct = direct < 0 ? direct_io_enabled() : direct != 0;
    c.prefetch = prefetch < 0 ? prefetch_enabled() : prefetch != 0;
    return c;
}

TileConfig tile_config128() {
    TileConfig c{kTileM128, kTileRB128, kTileLow128, false};
    c.ctas = tile_ctas_per_sm();
    c.direct = false;
    return c;
}

std::string tile_config_name(const TileConfig &cfg) {
    return "m=" + std::to_string(cfg.m) + ",rb=" + std::to_string(cfg.rb) + ",low=" + std::to_string(cfg.low) +
           ",ctas=" + std::to_string(cfg.ctas) + ",direct=" + std::to_string(int(cfg.direct)) +
           (cfg.prefetch ? ",prefetch=1" : "");
}

std::string jit_cache_dir() { return cache_dir(); }

std::string tile_codegen_key() {
    return "f32x2=" + std::to_string(int(packed_adds_enabled())) + ",ctas=" + std::to_string(tile_ctas_per_sm()) +
           ",direct=" + std::to_string(int(direct_io_enabled())) + ",prefetch=" + std::to_string(int(prefetch_enabled()));
}

std::string tile_pass_source(const TilePlan<float> &tp, size_t i) { return gen_pass(tp, i); }
std::string tile_pass_source(const TilePlan<double> &tp, size_t i) { return gen_pass(tp, i); }
sv_status jit_tile_plan(const TilePlan<float> &tp, std::vector<void *> *fns) { return jit_plan_impl(tp, fns); }
sv_status jit_tile_plan(const TilePlan<double> &tp, std::vector<void *> *fns) { return jit_plan_impl(tp, fns); }
sv_status jit_compile_check(const TilePlan<float> &tp) { return compile_check_impl(tp); }
sv_status jit_compile_check(const TilePlan<double> &tp) { return compile_check_impl(tp); }

const char *tile_kernel_name(const sv_state *h) {
    static const char *n64[] = {"svp<f32,13,4>", "svp<f32,13,5>", "svp<f32,13,6>"};
    return h->dt == SV_C64 ? n64[tile_rb64() - 4] : "svp<f64,12,4>";
}

cudaError_t launch_jit_pass(sv_state *h, void *fn, int n, int rb, uint64_t param) {
    int M = h->dt == SV_C64 ? kTileM64 : kTileM128;
    size_t tile_bytes = (size_t(1) << M) * (h->dt == SV_C64 ? 8u : 16u);
    int persistent = 0;
    {
        std::lock_guard<std::mutex> lock(g_jit_mu);
        auto it = g_jit_smem.find(fn);
        if (it != g_jit_smem.end()) {
            tile_bytes = size_t(it->second.smem);
            persistent = it->second.persistent_ctas;
            M = it->second.m;
        }
    }
    unsigned long long ntiles = 1ull << (n - M);
    unsigned grid = unsigned(ntiles);
    if (persistent > 0) {  // persistent CTAs: the resident ones, each looping over tiles
        int sms = 0;
        const cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        if (e != cudaSuccess) return e;
        const unsigned long long resident = (unsigned long long)sms * unsigned(persistent);
        grid = unsigned(ntiles < resident ? ntiles : resident);
    }
    void *psi = h->data;
    unsigned long long prm = param;
    void *args[] = {&psi, &prm, &ntiles};
    return cudaLaunchKernel(static_cast<const void *>(fn), dim3(grid), dim3(1u << (M - rb)), args, tile_bytes,
                            h->stream);
}

}  // namespace sv
