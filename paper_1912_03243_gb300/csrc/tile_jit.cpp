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
#include <nvrtc.h>

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

#include "plan.h"
#include "tile.h"

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

// CTAs per SM the pass kernels are compiled for (register budget); the
// shared tile (64 KiB) allows up to 3.  SV_TILE_CTAS overrides.
int tile_ctas_per_sm() {
    const char *e = std::getenv("SV_TILE_CTAS");
    const int v = e ? std::atoi(e) : 2;
    return v >= 1 && v <= 3 ? v : 2;
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
    o << "extern \"C\" __global__ void __launch_bounds__(" << G.NT << ", " << tile_ctas_per_sm() << ") svp(" << C2T
      << "* __restrict__ psi) {\n";
    o << "  extern __shared__ __align__(16) unsigned char smem[];\n";
    o << "  " << C2T << "* sm = reinterpret_cast<" << C2T << "*>(smem);\n";
    o << "  const u32 t = threadIdx.x;\n  const u64 b = blockIdx.x;\n  u64 base = 0;\n";
    {
        int pos[kTileMaxOuter];
        for (int k = 0; k < pa.nouter; ++k) pos[k] = pa.outer_pos[k];
        emit_deposit(o, "base", "b", pos, pa.nouter, "u64");
    }
    // chunk c = t + NT * i: chunk bit k <-> tile bit k + EPC_LOG <-> global tile_pos[k + EPC_LOG]
    const int tbits = G.M - G.RB;  // bits of t
    {
        int pos[kTileMaxQ];
        for (int k = 0; k < tbits; ++k) pos[k] = pa.tile_pos[k + G.EPC_LOG];
        o << "  u64 g0 = base;\n";
        emit_deposit(o, "g0", "t", pos, tbits, "u64");
    }
    o << "  const u32 s0 = swz(t);\n";
    const int iters = G.NCH / G.NT;
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
    for (int i = 0; i < iters; ++i)
        o << "  cpa16(smem + ((s0 ^ " << si[size_t(i)] << "u) << 4), psi + (g0 | " << gi[size_t(i)] << "ull));\n";
    o << "  asm volatile(\"cp.async.commit_group;\\ncp.async.wait_group 0;\\n\" ::: \"memory\");\n";
    o << "  __syncthreads();\n";
    o << "  " << RT << " xr[" << G.NR << "], xi[" << G.NR << "];\n  u32 jt = 0, pj = 0;\n";
    (void)0;

    int cur_seg = -1;
    uint32_t pv[32] = {0};
    // Compile-time sign of each register: the stored value is sgn[v] times
    // the amplitude.  Unconditional sign flips (CZ) only flip sgn; butterflies
    // fold the signs into add / sub choices; the scatter materialises them.
    int sgn[32];
    for (int v = 0; v < 32; ++v) sgn[v] = 1;
    // Runtime signs: a sign flip conditioned on thread / CTA bits becomes a
    // per-thread factor sg<c> = cond ? -1 : 1; rsg[v] lists the factors the
    // stored value still owes.  Butterflies of registers with equal lists
    // need nothing; otherwise the relative factor enters as an FMA operand.
    std::vector<int> rsg[32];
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
    auto symdiff = [](const std::vector<int> &a, const std::vector<int> &b) {
        std::vector<int> d;
        std::set_symmetric_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(d));
        return d;
    };
    const bool packed = sizeof(R) == 4 && packed_adds_enabled();
    auto reg = [](const char *a, int v) { return std::string(a) + "[" + std::to_string(v) + "]"; };
    auto materialise = [&](int v) {
        if (!rsg[v].empty()) {
            const std::string f = prod(rsg[v]);
            const char *neg = sgn[v] < 0 ? "-" : "";
            o << "  " << reg("xr", v) << " *= " << neg << f << "; " << reg("xi", v) << " *= " << neg << f << ";\n";
            rsg[v].clear();
            sgn[v] = 1;
        } else if (sgn[v] < 0) {
            o << "  " << reg("xr", v) << " = -" << reg("xr", v) << "; " << reg("xi", v) << " = -" << reg("xi", v) << ";\n";
            sgn[v] = 1;
        }
    };
    auto scatter = [&]() {
        for (int v = 0; v < G.NR; ++v) {
            if (!rsg[v].empty()) materialise(v);
            const char *neg = sgn[v] < 0 ? "-" : "";
            o << "  sm[pj ^ " << pv[v] << "u] = make_" << C2T << "(" << neg << "xr[" << v << "], " << neg << "xi[" << v
              << "]);\n";
            sgn[v] = 1;
        }
        prod_name.clear();
    };
    int cond_id = 0;
    for (int i = pa.op_begin; i < pa.op_end; ++i) {
        const TileOp<R> &op = tp.ops[size_t(i)];
        if (op.type == TOP_SEG) {
            if (cur_seg >= 0) {
                scatter();
                o << "  __syncthreads();\n";
            }
            cur_seg = op.a;
            const TileSeg &sg = tp.segs[size_t(op.a)];
            int pos[kTileMaxQ];
            for (int k = 0; k < tbits; ++k) pos[k] = sg.tpos[k];
            o << "  jt = 0;\n";
            emit_deposit(o, "jt", "t", pos, tbits, "u32");
            if (sizeof(R) == 4) o << "  pj = (swz(jt >> 1) << 1) | (jt & 1u);\n";
            else o << "  pj = swz(jt);\n";
            for (int v = 0; v < G.NR; ++v) {
                uint32_t d = 0;
                for (int s = 0; s < G.RB; ++s)
                    if (v >> s & 1) d |= 1u << sg.rpos[s];
                pv[v] = Geo<R>::phys(d);
                o << "  { " << C2T << " a = sm[pj ^ " << pv[v] << "u]; xr[" << v << "] = a.x; xi[" << v
                  << "] = a.y; }\n";
            }
            continue;
        }
        // runtime condition on thread / CTA bits (branch-free select)
        std::string cond;
        int cid = -1;
        if (op.tmask || op.gmask) {
            cid = cond_id++;
            cond = "c" + std::to_string(cid);
            o << "  const bool " << cond << " = ((jt & " << op.tmask << "u) == " << op.tval << "u) && ((base & "
              << op.gmask << "ull) == " << op.gval << "ull);\n";
            if (op.type == TOP_NEG) o << "  const " << RT << " sg" << cid << " = " << cond << " ? " << RT << "(-1) : " << RT << "(1);\n";
        }
        auto sel = [&](const std::string &v_new, const std::string &v_old) {
            return cond.empty() ? v_new : ("(" + cond + " ? " + v_new + " : " + v_old + ")");
        };
        if (op.type == TOP_SCALE) {
            const std::string pr = lit(op.u[0]), pi = lit(op.u[1]);
            for (int v = 0; v < G.NR; ++v)
                o << "  { " << RT << " r = xr[" << v << "] * " << pr << " - xi[" << v << "] * " << pi << "; xi[" << v
                  << "] = xr[" << v << "] * " << pi << " + xi[" << v << "] * " << pr << "; xr[" << v << "] = r; }\n";
            continue;
        }
        if (op.type == TOP_PHASE || op.type == TOP_NEG) {
            const uint32_t M = uint32_t(op.a) / 32, V = uint32_t(op.a) % 32;
            const std::string pr = lit(op.u[0]), pi = lit(op.u[1]);
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
            const int sa = sgn[v], sb = sgn[w], r = sa * sb;
            // relative runtime factor of b with respect to a ("" when the lists agree)
            const std::vector<int> rel = symdiff(rsg[v], rsg[w]);
            const std::string rf = rel.empty() ? std::string() : prod(rel);
            if (op.type == TOP_STRUCT && kind == SK_X && cond.empty()) {
                o << "  { const " << RT << " t0 = " << ar << ", t1 = " << ai << "; " << ar << " = " << br << "; " << ai
                  << " = " << bi << "; " << br << " = t0; " << bi << " = t1; }\n";
                std::swap(sgn[v], sgn[w]);
                std::swap(rsg[v], rsg[w]);
                continue;
            }
            if (op.type == TOP_STRUCT && (kind == SK_H || kind == SK_SY || kind == SK_SYD) && cond.empty()) {
                // true a' = sa (m00 A + m01 r B), b' = sa (m10 A + m11 r B); each is
                // +-(A + B) or +-(A - B), one of each
                static const int M[3][4] = {{1, 1, 1, -1}, {1, -1, 1, 1}, {1, 1, -1, 1}};
                const int *m = M[kind == SK_H ? 0 : (kind == SK_SY ? 1 : 2)];
                const bool a_plus = m[0] * m[1] * r > 0;   // A' = m00 (A + e B)
                sgn[v] = sa * m[0];
                sgn[w] = sa * m[2];
                rsg[w] = rsg[v];
                if (!rf.empty()) {  // A' = A + e rf B, B' = A - e rf B
                    const std::string e1 = a_plus ? "" : "-";
                    const std::string e2 = a_plus ? "-" : "";
                    if (packed) {
                        o << "  { const u64 a = pk(" << ar << ", " << ai << "), b = pk(" << br << ", " << bi << "); "
                          << "upk(fma2(b, pk(" << e1 << rf << ", " << e1 << rf << "), a), " << ar << ", " << ai << "); "
                          << "upk(fma2(b, pk(" << e2 << rf << ", " << e2 << rf << "), a), " << br << ", " << bi << "); }\n";
                    } else {
                        o << "  { const " << RT << " a0 = " << ar << ", a1 = " << ai << ", b0 = " << br << ", b1 = " << bi
                          << "; " << ar << " = fma(" << e1 << rf << ", b0, a0); " << ai << " = fma(" << e1 << rf
                          << ", b1, a1); " << br << " = fma(" << e2 << rf << ", b0, a0); " << bi << " = fma(" << e2
                          << rf << ", b1, a1); }\n";
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
            if (op.type == TOP_STRUCT && !rf.empty()) {  // SX / SXD / runtime-conditioned: align b with a
                o << "  " << br << " *= " << rf << "; " << bi << " *= " << rf << ";\n";
                rsg[w] = rsg[v];
            }
            std::string nar, nai, nbr, nbi;
            const std::string rs = r > 0 ? " + " : " - ", rn = r > 0 ? " - " : " + ";
            if (op.type == TOP_G1) {
                // signs folded into the constants: a' = u00 sa A + u01 sb B, ...
                std::string u[8];
                for (int k = 0; k < 8; ++k) {
                    const int colsign = (k == 0 || k == 1 || k == 4 || k == 5) ? sa : sb;
                    u[k] = lit(R(colsign) * op.u[k]);
                }
                nar = u[0] + "*ar - " + u[1] + "*ai + " + u[2] + "*br - " + u[3] + "*bi";
                nai = u[0] + "*ai + " + u[1] + "*ar + " + u[2] + "*bi + " + u[3] + "*br";
                nbr = u[4] + "*ar - " + u[5] + "*ai + " + u[6] + "*br - " + u[7] + "*bi";
                nbi = u[4] + "*ai + " + u[5] + "*ar + " + u[6] + "*bi + " + u[7] + "*br";
                sgn[v] = sgn[w] = 1;
                rsg[w] = rsg[v];  // equal lists here (else materialised above)
            } else {
                // stored results relative to sign sa for both outputs
                switch (kind) {
                    case SK_H: nar = "ar" + rs + "br"; nai = "ai" + rs + "bi"; nbr = "ar" + rn + "br"; nbi = "ai" + rn + "bi"; break;
                    case SK_SY: nar = "ar" + rn + "br"; nai = "ai" + rn + "bi"; nbr = "ar" + rs + "br"; nbi = "ai" + rs + "bi"; break;
                    case SK_SYD: nar = "ar" + rs + "br"; nai = "ai" + rs + "bi"; nbr = "-ar" + rs + "br"; nbi = "-ai" + rs + "bi"; break;
                    case SK_SX:  // (A - i r B, -i A + r B)
                        nar = "ar" + rs + "bi"; nai = "ai" + rn + "br"; nbr = "ai" + rs + "br"; nbi = "-ar" + rs + "bi"; break;
                    case SK_SXD:  // (A + i r B, i A + r B)
                        nar = "ar" + rn + "bi"; nai = "ai" + rs + "br"; nbr = "-ai" + rs + "br"; nbi = "ar" + rs + "bi"; break;
                    default:  // X under a runtime condition (signs are +1 here)
                        nar = "br"; nai = "bi"; nbr = "ar"; nbi = "ai"; break;
                }
                sgn[w] = sa;
                rsg[w] = rsg[v];
            }
            o << "  { const " << RT << " ar = " << ar << ", ai = " << ai << ", br = " << br << ", bi = " << bi << "; "
              << ar << " = " << sel(nar, "ar") << "; " << ai << " = " << sel(nai, "ai") << "; " << br << " = "
              << sel(nbr, "br") << "; " << bi << " = " << sel(nbi, "bi") << "; }\n";
        }
    }
    if (cur_seg >= 0) {
        scatter();
        o << "  __syncthreads();\n";
    }
    for (int i = 0; i < iters; ++i)
        o << "  *reinterpret_cast<int4*>(psi + (g0 | " << gi[size_t(i)] << "ull)) = *reinterpret_cast<const int4*>(smem + ((s0 ^ "
          << si[size_t(i)] << "u) << 4));\n";
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

std::string compile_cubin(const std::string &src, std::string *err) {
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "sv_pass.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        *err = "nvrtcCreateProgram failed";
        return {};
    }
    const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17"};
    const nvrtcResult r = nvrtcCompileProgram(prog, 2, opts);
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
    unsigned hw = std::thread::hardware_concurrency();
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
                cubin[j] = compile_cubin(src[j], &err[j]);
            }
        });
    for (auto &th : pool) th.join();
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
            const int smem = (1 << tp.m) * int(2 * sizeof(R));
            // a cudaKernel_t is accepted wherever a kernel symbol is
            if (ce == cudaSuccess)
                ce = cudaFuncSetAttribute(reinterpret_cast<const void *>(e.fn),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (ce != cudaSuccess) return cuda_status(ce, "loading a compiled pass");
            it = g_jit.emplace(key[size_t(j)], e).first;
        }
        (*fns)[size_t(j)] = reinterpret_cast<void *>(it->second.fn);
    }
    return SV_OK;
}

template <typename R>
sv_status compile_check_impl(const TilePlan<R> &tp) {
    for (size_t i = 0; i < tp.passes.size(); ++i) {
        std::string err;
        if (compile_cubin(gen_pass(tp, i), &err).empty()) {
            set_error("NVRTC compile of pass %zu failed: %s", i, err.c_str());
            return SV_ERR_CUDA;
        }
    }
    return SV_OK;
}

}  // namespace

sv_status jit_tile_plan(const TilePlan<float> &tp, std::vector<void *> *fns) { return jit_plan_impl(tp, fns); }
sv_status jit_tile_plan(const TilePlan<double> &tp, std::vector<void *> *fns) { return jit_plan_impl(tp, fns); }
sv_status jit_compile_check(const TilePlan<float> &tp) { return compile_check_impl(tp); }
sv_status jit_compile_check(const TilePlan<double> &tp) { return compile_check_impl(tp); }

const char *tile_kernel_name(const sv_state *h) {
    static const char *n64[] = {"svp<f32,13,4>", "svp<f32,13,5>"};
    return h->dt == SV_C64 ? n64[tile_rb64() == 5] : "svp<f64,12,4>";
}

cudaError_t launch_jit_pass(sv_state *h, void *fn, int n, int rb) {
    const int M = h->dt == SV_C64 ? kTileM64 : kTileM128;
    const int RB = rb;
    const size_t smem = (size_t(1) << M) * (h->dt == SV_C64 ? 8u : 16u);
    void *psi = h->data;
    void *args[] = {&psi};
    return cudaLaunchKernel(static_cast<const void *>(fn), dim3(1u << (n - M)), dim3(1u << (M - RB)), args, smem,
                            h->stream);
}

}  // namespace sv
