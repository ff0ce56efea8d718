// Tiled multi-gate passes: data structures shared by the host planner
// (tile_plan.cpp) and the pass code generator (tile_jit.cpp).
//
// A pass picks m "tile" qubits.  Each CTA owns one tile: the 2^m amplitudes
// whose other (outer) index bits equal the CTA's number, i.e. 2^(m-L) runs
// of 2^L contiguous amplitudes (the tile always contains the low L qubits so
// every HBM transfer is a contiguous run).  The CTA loads the tile into
// shared memory once, applies every gate of the pass whose non-diagonal
// qubits lie in the tile, and writes it back once: one HBM read and write of
// the state per pass instead of one per gate.  Diagonal gates (T, CZ, CP)
// need no qubit in the tile: an outer bit is a constant per CTA.
//
// Inside a pass, each thread holds 2^RB amplitudes in registers ("register
// qubits"); a segment is a run of ops whose target qubits are register
// qubits, and segments are separated by a shared-memory transposition that
// changes which tile bits are register bits.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "sv_internal.h"

namespace sv {

constexpr int kTileMaxQ = 16;   // max tile bits
constexpr int kTileMaxOuter = 40;

enum TileOpType : int32_t {
    TOP_G1 = 1,      // general 2x2 on register slot `a`
    TOP_STRUCT = 2,  // structured 2x2 (entries 0, +-1, +-i): slot = a & 255, kind = a >> 8
    TOP_PHASE = 3,   // multiply by u[0] + i u[1] where the condition holds; a = register condition id
    TOP_NEG = 4,     // negate where the condition holds; a = register condition id
    TOP_SEG = 5,     // start segment a (shared-memory transposition)
    TOP_SCALE = 6,   // multiply every amplitude by u[0] + i u[1]
};

// Structured kinds: U = c * M with M below; c is deferred to a TOP_SCALE.
enum StructKind : int32_t {
    SK_H = 0,    // [[1, 1], [1, -1]]
    SK_SX = 1,   // [[1, -i], [-i, 1]]
    SK_SXD = 2,  // [[1, i], [i, 1]]
    SK_SY = 3,   // [[1, -1], [1, 1]]
    SK_SYD = 4,  // [[1, 1], [-1, 1]]
    SK_X = 5,    // [[0, 1], [1, 0]]
    SK_COUNT = 6
};

// Planner gate conditions on bits kParamBit0 + j (above every state qubit)
// test bit j of a launch parameter instead of an amplitude index bit: one
// compiled pass then serves every value of those bits (the fixed branch bits
// of a decomposition's branch parts).
constexpr int kParamBit0 = 48;
constexpr int kParamBits = 16;
constexpr uint64_t kQubitBits = (uint64_t(1) << kParamBit0) - 1;

template <typename R>
struct alignas(16) TileOp {
    int32_t type;
    int32_t a;
    uint32_t rmask, rval;  // condition on the register index (TOP_G1 controls)
    uint32_t tmask, tval;  // condition on the thread's tile-index bits
    uint64_t gmask, gval;  // condition on the CTA's outer global index bits
    uint32_t pmask, pval;  // condition on the launch parameter bits
    R u[8];
};

struct TileSeg {
    uint8_t rpos[8];            // tile-bit position of register slot s
    uint8_t tpos[kTileMaxQ];    // tile-bit position of thread-index bit i (lane bits first)
};

struct TilePassArgs {
    int n;
    int m;                      // tile bits
    int lc;                     // contiguous low tile bits (run length 2^lc)
    int nouter;
    uint8_t tile_pos[kTileMaxQ];     // global position of tile bit i (ascending)
    uint8_t outer_pos[kTileMaxOuter];
    int op_begin, op_end;
};

constexpr int kTileMaxRegs = 64;  // register amplitudes per thread (2^rb, rb <= 6)

// Register-condition id used by TOP_PHASE / TOP_NEG: mask * kTileMaxRegs + value with
// at most two mask bits.
constexpr int reg_cond_id(uint32_t mask, uint32_t val) { return int(mask * kTileMaxRegs + val); }

struct TileConfig {
    int m;      // tile bits
    int rb;     // register bits per thread
    int low;    // low qubits always in the tile (contiguous runs of 2^low amplitudes)
    bool c64;
    int ctas = 2;        // CTAs per SM the passes are compiled for (register budget)
    bool direct = true;  // complex64: first / last segment straight between HBM and registers
    bool prefetch = false;  // complex64: persistent CTAs copy the next tile during the last segment
};

template <typename R>
struct TilePlan {
    int m = 0, rb = 0;  // tile bits, register bits per thread
    int ctas = 2;
    bool direct = true;
    bool prefetch = false;
    std::vector<TilePassArgs> passes;
    std::vector<TileOp<R>> ops;
    std::vector<TileSeg> segs;
    // per pass: FP32 lane operations per amplitude its gates need at least
    // (2 per structured butterfly, 1 per T-type phase, 4 per other complex
    // phase or 8 per dense 2x2, times the fraction of amplitudes a control
    // or condition leaves; sign flips and X are free), and its segments
    std::vector<int> pass_ctas;     // CTAs per SM each pass is compiled for (empty: ctas for all)
    std::vector<double> lane_ops;
    std::vector<int> nseg;
};

// A gate in the planner's form.  kind 0: 2x2 update u on `target` where
// the qubits in cmask equal cval (controls; full role on the target);
// kind 1: multiply by u[0] where the qubits in cmask equal cval (diagonal).
// `scale` is a global scalar factor deferred by the lowering (kind 1 with
// cmask = 0 carries only that).
struct PGate {
    int kind;
    int target;
    uint64_t cmask, cval;
    Cplx u[4];
    Cplx scale;
};

// Circuit text -> planner gates (CZ/CP/T/P become diagonal phases, CX a
// controlled X, SWAP three CX).
std::vector<PGate> lower_for_tiles(const Circuit &circ);

template <typename R>
sv_status plan_tiles(const std::vector<PGate> &gates, int n, const TileConfig &cfg, TilePlan<R> *out);
template <typename R>
sv_status plan_tiles(const Circuit &circ, int n, const TileConfig &cfg, TilePlan<R> *out) {
    return plan_tiles<R>(lower_for_tiles(circ), n, cfg, out);
}

// Tile geometry of the kernels: complex64 2^13-amplitude tiles with 32
// amplitudes per thread, complex128 2^12 with 16.
constexpr int kTileM64 = 13, kTileRB64 = 5, kTileLow64 = 4;
constexpr int kTileM128 = 12, kTileRB128 = 4, kTileLow128 = 3;

// The generated CUDA source of pass i of a plan (what jit_tile_plan compiles).
std::string tile_pass_source(const TilePlan<float> &tp, size_t i);
std::string tile_pass_source(const TilePlan<double> &tp, size_t i);
// Compile every pass of a plan into a straight-line kernel (NVRTC, cached
// per device and source); fns receives one CUfunction per pass.
sv_status jit_tile_plan(const TilePlan<float> &tp, std::vector<void *> *fns);
sv_status jit_tile_plan(const TilePlan<double> &tp, std::vector<void *> *fns);
// Compile only (no device needed): NVRTC-compiles every pass, returns status.
sv_status jit_compile_check(const TilePlan<float> &tp);
sv_status jit_compile_check(const TilePlan<double> &tp);
// Register bits per thread of complex64 tile passes (SV_TILE_RB overrides,
// 4 or 5).
int tile_rb64();
// CTAs per SM of the pass kernels (SV_TILE_CTAS overrides, 1 to 3).
int tile_ctas_per_sm();
// The tile configuration of complex64 / complex128 passes: the environment's
// defaults, or the given register bits, CTAs per SM and direct I/O (an
// autotuner's candidate; 0 / -1 keep the default).
TileConfig tile_config64(int rb = 0, int ctas = 0, int direct = -1, int prefetch = -1, int m = 0);
// Tile bits of complex64 passes (SV_TILE_M overrides: 12 or 13).
int tile_m64();
TileConfig tile_config128();
// Folder of the compiled-pass disk cache ("" when there is none).
std::string jit_cache_dir();
// A short text naming a configuration (plan keys, tuning reports).
std::string tile_config_name(const TileConfig &cfg);
// Low qubits always in a complex64 tile (contiguous HBM runs of 2^low
// amplitudes); SV_TILE_LOW overrides (4 to 10).
int tile_low64();
// Launch one compiled pass over the whole state (grid = 2^(n-m) CTAs of
// 2^(m-rb) threads); param: the launch parameter bits (kParamBit0).
cudaError_t launch_jit_pass(sv_state *h, void *fn, int n, int rb, uint64_t param = 0);
const char *tile_kernel_name(const sv_state *h);
// The code-generation switches (environment) that shape a compiled pass, as
// part of a plan-cache key.
std::string tile_codegen_key();
// Direct HBM I/O of complex64 passes (SV_TILE_DIRECT, default on): the first
// segment loads from and the last stores to HBM straight from registers.
bool direct_io_enabled();
// Planner lookahead width (SV_PLAN_LOOKAHEAD, default 4; 0 = greedy).
int plan_lookahead_width();
// Segment (register set) lookahead width (SV_SEG_LOOKAHEAD, default 4; 0 =
// first fit).
int seg_lookahead_width();

}  // namespace sv
