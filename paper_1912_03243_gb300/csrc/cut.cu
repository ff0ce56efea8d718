// Decomposition of entangling gates across partitions (Sec. 4, Eq. 2-3).
//
// Rewrite (host): the qubits fall into P partitions.  Every CZ or CP between
// two partitions becomes a branch slot k; a CX between them is first written
// as H CZ H on its target.  Decomposition forms (a = the gate's first qubit,
// b = its second):
//   projector: CP_ab(th) = P0(a) (x) 1 + P1(a) (x) P(th)(b)   (weight 1)
//   Eq. 2:     CZ_ab = 1/2 sum_{s=+-1} D_s(a) (x) D_s(b),
//              D_s = exp(i sigma^z (x s - pi/4)), cos 2x = i  (weight 1/2 each)
// so the circuit is a sum over s in {0,1}^S of a product of circuits that
// each act on one partition (Sec. 4), and <z|C|0> = sum_s prod_p
// <z_p|W_p(s)|0_p> (Eq. 3).  W_p depends only on the bits of the cuts that
// touch partition p.
//
// Batched simulation (GPU): for each partition p the branch vectors are one
// vector of 2^(n_p + S_p) complex64 amplitudes whose top index bits are the
// S_p branch bits of the cuts touching p.
// A branch operator is then an ordinary diagonal gate coupling a half's qubit
// to branch bit k (the projector zeroes amplitudes where bit a != s_k; P(th)
// and D_s are phases selected by (bit, s_k)).  Branch bits only ever appear
// in diagonal gates, so the tile planner keeps them outside the tiles (a
// constant per CTA) and every pass runs over all branches of a half in one
// launch.  The initial vector has amplitude 1 at index s << n_p for every s
// (or, with branch-prefix sharing, the branches are forked from branch 0 at
// their first operator, see run_half).
//
// Sum (GPU): one warp per output bit string (its partition indices gathered
// from the string's bits by the first P lanes), lanes over s, products of the
// P partitions' amplitudes and the sum in FP64, times the weight.
#include <complex>
#include <cstdlib>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "plan.h"
#include "tile.h"

namespace sv {
namespace {

using cd = std::complex<double>;

__global__ void k_branch_init(float2 *psi, int np, int S) {
    const uint64_t ns = uint64_t(1) << S;
    for (uint64_t s = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < ns; s += uint64_t(gridDim.x) * blockDim.x)
        psi[s << np] = make_float2(1.0f, 0.0f);
}

constexpr int kMaxParts = 16;
constexpr int kMaxPartQubits = 40;  // a partition's state, like any state
constexpr int kMaxCutBits = 24;     // branch bits of one partition
constexpr int kMaxCutQubits = 128;  // qubits of the circuit

struct CutSumArgs {
    int P, Sv, nwords;
    int accumulate;  // add to out (the sum over several branch parts) instead of writing it
    uint64_t m;
    double w;
    const float2 *vec[kMaxParts];
    int nlocal[kMaxParts], nbits[kMaxParts];
    uint8_t cutbit[kMaxParts][kMaxCutBits];      // partition bit j <- batched branch bit cutbit[p][j]
    uint8_t qubit[kMaxParts][kMaxPartQubits];    // partition qubit i <- circuit qubit qubit[p][i]
};

__global__ void k_cut_sum(const uint64_t *__restrict__ z, const CutSumArgs a, double2 *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const size_t warps = size_t(gridDim.x) * (blockDim.x >> 5);
    const uint64_t ns = uint64_t(1) << a.Sv;
    for (size_t j = size_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); j < a.m; j += warps) {
        // lane p < P: the index of z_j inside partition p
        uint64_t mine = 0;
        if (lane < a.P)
            for (int i = 0; i < a.nlocal[lane]; ++i) {
                const int q = a.qubit[lane][i];
                mine |= ((z[j * a.nwords + (q >> 6)] >> (q & 63)) & 1ull) << i;
            }
        uint64_t zl[kMaxParts];
#pragma unroll
        for (int p = 0; p < kMaxParts; ++p) zl[p] = __shfl_sync(0xffffffffu, mine, p);
        double re = 0.0, im = 0.0;
        for (uint64_t s = lane; s < ns; s += 32) {
            double pr = 1.0, pi = 0.0;
            for (int p = 0; p < a.P; ++p) {
                uint64_t sp = 0;
                for (int k = 0; k < a.nbits[p]; ++k) sp |= ((s >> a.cutbit[p][k]) & 1ull) << k;
                const float2 v = a.vec[p][(sp << a.nlocal[p]) | zl[p]];
                const double r = pr * v.x - pi * v.y;
                pi = pr * v.y + pi * v.x;
                pr = r;
            }
            re += pr;
            im += pi;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) {
            double2 v = make_double2(a.w * re, a.w * im);
            if (a.accumulate) {
                const double2 o = out[j];
                v.x += o.x;
                v.y += o.y;
            }
            out[j] = v;
        }
    }
}

// Eq. 2 factor for branch bit value sb (0 <-> s = +1, 1 <-> s = -1):
// exp(i sigma^z phi) = diag(e^{i phi}, e^{-i phi}), phi = x s - pi/4.
void eq2_diag(int sb, cd d[2]) {
    const cd x = std::acos(cd(0.0, 1.0)) / 2.0;  // cos 2x = i, principal branch
    const double s = sb ? -1.0 : 1.0;
    const cd phi = x * s - 3.14159265358979323846 / 4.0;
    d[0] = std::exp(cd(0, 1) * phi);
    d[1] = std::exp(-cd(0, 1) * phi);
}

PGate phase_gate(uint64_t mask, uint64_t val, cd ph) {
    PGate g{};
    g.kind = 1;
    g.target = -1;
    g.cmask = mask;
    g.cval = val;
    g.u[0] = Cplx{ph.real(), ph.imag()};
    g.scale = Cplx{1, 0};
    return g;
}

// Lower one instruction acting inside a half (qubits already local).
void append_lowered(const Instr &ins, std::vector<PGate> *out) {
    Circuit one;
    one.n = 64;
    one.instrs.push_back(ins);
    const std::vector<PGate> g = lower_for_tiles(one);
    out->insert(out->end(), g.begin(), g.end());
}

// One step of a partition's simulation: a stage of compiled tiled passes
// over the low 2^nrun amplitudes, or (branch-prefix sharing) a fork that
// copies the live 2^live amplitudes to the slots above them.
struct HalfStep {
    std::vector<void *> fns;  // compiled passes of a stage; empty for a fork
    int nrun = 0, rb = 0;
    int live = -1;            // fork: live qubits before the copy
};

struct Half {            // one partition
    int nlocal = 0;     // qubits of the partition
    int nbits = 0;      // batched branch bits of the cuts touching it
    int nq = 0;         // qubits of the batched vector (local + branch, padded to a tile)
    std::vector<PGate> gates;
    std::vector<int> qubits;   // circuit qubit of local qubit i
    std::vector<int> cutbits;  // batched branch bit of partition bit j
    float2 *d = nullptr;
    bool init_all = false;     // every branch starts at its own |0> (no prefix sharing)
    std::vector<HalfStep> steps;
};

// Plan and compile `gates` as tiled passes over the low 2^nrun amplitudes.
sv_status plan_stage(std::vector<HalfStep> *steps, const std::vector<PGate> &gates, int nrun) {
    if (gates.empty()) return SV_OK;
    TilePlan<float> tp;
    sv_status s = plan_tiles<float>(gates, nrun, tile_config64(), &tp);
    if (s) return s;
    HalfStep st;
    s = jit_tile_plan(tp, &st.fns);
    if (s) return s;
    st.nrun = nrun;
    st.rb = tp.rb;
    steps->push_back(std::move(st));
    return SV_OK;
}

// Branch-prefix sharing (on unless SV_CUT_PREFIX=0): the gates before the
// first branch operator are the same for every branch, so they run once on
// the 2^n_p amplitudes of branch 0; at the first operator on branch bit k the
// live vector (branches with bits >= k clear, the low 2^(n_p + k) amplitudes)
// is copied to the slots with bit k set, and the following gates run on the
// doubled vector.  Work falls from 2^S G to the sum over stages of
// 2^(n_p + k) G_k.  Amplitudes above the live vector are zero until copied
// to, and gates keep zeros zero, so a stage may run on more qubits (the tile
// size) than it has live.
bool prefix_sharing() {
    const char *e = std::getenv("SV_CUT_PREFIX");
    return !(e && e[0] == '0');
}

// Schedules by partition content (its gates, sizes, branch-bit count and the
// code-generation settings): a repeated decomposition skips the planning, and
// the compiled passes it names stay loaded for the process.
std::mutex g_sched_mu;
std::unordered_map<std::string, std::pair<bool, std::vector<HalfStep>>> g_sched;
constexpr size_t kSchedCacheMax = 256;

std::string schedule_key(const Half &h, int S) {
    std::string k = std::to_string(h.nlocal) + "," + std::to_string(h.nq) + "," + std::to_string(S) + "," +
                    std::to_string(int(prefix_sharing())) + "," + tile_config_name(tile_config64()) + "," +
                    tile_codegen_key() + "," + std::to_string(plan_lookahead_width()) + "|";
    int dev = 0;
    cudaGetDevice(&dev);
    k += std::to_string(dev) + "|";
    for (const PGate &g : h.gates) {
        k.append(reinterpret_cast<const char *>(&g.kind), sizeof g.kind);
        k.append(reinterpret_cast<const char *>(&g.target), sizeof g.target);
        k.append(reinterpret_cast<const char *>(&g.cmask), sizeof g.cmask);
        k.append(reinterpret_cast<const char *>(&g.cval), sizeof g.cval);
        k.append(reinterpret_cast<const char *>(g.u), sizeof g.u);
        k.append(reinterpret_cast<const char *>(&g.scale), sizeof g.scale);
    }
    return k;
}

sv_status plan_half_uncached(Half &h, int S);

// The schedule of a partition: planned and compiled once, then run for every
// branch part (the fixed branch bits of a part are launch parameters).
sv_status plan_half(Half &h, int S) {
    const std::string key = schedule_key(h, S);
    {
        std::lock_guard<std::mutex> lock(g_sched_mu);
        auto it = g_sched.find(key);
        if (it != g_sched.end()) {
            h.init_all = it->second.first;
            h.steps = it->second.second;
            return SV_OK;
        }
    }
    const sv_status s = plan_half_uncached(h, S);
    if (s) return s;
    std::lock_guard<std::mutex> lock(g_sched_mu);
    if (g_sched.size() >= kSchedCacheMax) g_sched.clear();
    g_sched[key] = std::make_pair(h.init_all, h.steps);
    return SV_OK;
}

sv_status plan_half_uncached(Half &h, int S) {
    h.steps.clear();
    h.init_all = !prefix_sharing();
    if (h.init_all) return plan_stage(&h.steps, h.gates, h.nq);
    int live = h.nlocal;  // live amplitudes: 2^live
    std::vector<PGate> stage;
    auto fork = [&]() -> sv_status {
        sv_status s = plan_stage(&h.steps, stage, live > kTileM64 ? live : kTileM64);
        stage.clear();
        if (s) return s;
        HalfStep f;
        f.live = live++;
        h.steps.push_back(f);
        return SV_OK;
    };
    for (const PGate &g : h.gates) {
        // batched branch bits are only ever conditions of diagonal gates
        const uint64_t branch = g.kind == 1 ? ((g.cmask & kQubitBits) >> h.nlocal) : 0;
        while (branch >> (live - h.nlocal)) {
            sv_status s = fork();
            if (s) return s;
        }
        stage.push_back(g);
    }
    while (live < h.nlocal + S) {  // every branch bit has operators; kept for the layout
        sv_status s = fork();
        if (s) return s;
    }
    return plan_stage(&h.steps, stage, h.nq);
}

// Run a partition's schedule for the branch part whose fixed bits are param.
sv_status exec_half(Half &h, cudaStream_t st, int S, uint64_t param) {
    SV_CUDA_TRY(cudaMemsetAsync(h.d, 0, sizeof(float2) << h.nq, st));
    if (h.init_all) k_branch_init<<<64, 256, 0, st>>>(h.d, h.nlocal, S);
    else k_branch_init<<<1, 32, 0, st>>>(h.d, h.nlocal, 0);
    sv_status s = check_launch(cudaGetLastError(), "k_branch_init");
    if (s) return s;
    sv_state tmp;
    tmp.dt = SV_C64;
    tmp.data = h.d;
    tmp.stream = st;
    SV_CUDA_TRY(cudaGetDevice(&tmp.device));
    for (const HalfStep &step : h.steps) {
        if (step.fns.empty()) {
            const size_t bytes = sizeof(float2) << step.live;
            const cudaError_t e =
                cudaMemcpyAsync(reinterpret_cast<char *>(h.d) + bytes, h.d, bytes, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) {
                s = cuda_status(e, "cudaMemcpyAsync (branch fork)");
                break;
            }
            continue;
        }
        tmp.n = step.nrun;
        for (void *fn : step.fns) {
            s = check_launch(launch_jit_pass(&tmp, fn, step.nrun, step.rb, param), "branch pass");
            if (s) break;
        }
        if (s) break;
    }
    tmp.data = nullptr;
    return s;
}

}  // namespace
}  // namespace sv

using namespace sv;

// Sum over the branches s with s mod 2^plog in the list plist (plog = 0,
// plist = {0}: all of them).  For each listed part the low plog branch bits
// are fixed: their branch operators are plain diagonal gates on the
// partitions' qubits, and only the other S - plog bits are batched; the parts
// run one after another on the same device buffers and their sums add up in
// FP64 on the device.  z: m bit strings of nwords 64-bit words (qubit q is bit
// q % 64 of word q / 64).
static sv_status cut_impl(const char *text, int n, const uint8_t *part_of, int P, int form, const uint64_t *plist,
                          size_t nlist, int plog, size_t m, const uint64_t *z, int nwords, double *out, int *n_cut_out,
                          void *stream) {
    if (n < 2 || n > kMaxCutQubits || P < 2 || P > kMaxParts || !part_of || (form != 0 && form != 1) ||
        nwords != (n + 63) / 64 || (m > 0 && (!z || !out))) {
        set_error("bad arguments (n=%d, P=%d, form=%d, nwords=%d)", n, P, form, nwords);
        return SV_ERR_ARG;
    }
    Half parts[kMaxParts];
    int side[kMaxCutQubits], loc[kMaxCutQubits];
    for (int q = 0; q < n; ++q) {
        if (part_of[q] >= P) {
            set_error("qubit %d: partition %d outside 0..%d", q, int(part_of[q]), P - 1);
            return SV_ERR_ARG;
        }
        side[q] = part_of[q];
        loc[q] = parts[side[q]].nlocal++;
        parts[side[q]].qubits.push_back(q);
    }
    for (int p = 0; p < P; ++p)
        if (parts[p].nlocal == 0) {
            set_error("partition %d has no qubits", p);
            return SV_ERR_ARG;
        }
    const int top = n - 64 * (nwords - 1);  // qubits in the last word
    for (size_t j = 0; j < m; ++j)
        if (top < 64 && (z[j * nwords + nwords - 1] >> top)) {
            set_error("bit string %zu has bits above qubit %d", j, n - 1);
            return SV_ERR_ARG;
        }
    Circuit c;
    sv_status s = parse_circuit(text, n, &c);
    if (s) return s;

    // count the decomposed gates first
    int S = 0;
    for (const Instr &ins : c.instrs) {
        if (ins.nq != 2 || side[ins.q[0]] == side[ins.q[1]]) continue;
        if (ins.name == "SWAP") {
            set_error("a SWAP across partitions cannot be decomposed");
            return SV_ERR_UNSUPPORTED;
        }
        if (form == 1 && ins.name == "CP") {
            set_error("the Eq. 2 form decomposes CZ only (CP across partitions)");
            return SV_ERR_UNSUPPORTED;
        }
        ++S;
    }
    if (n_cut_out) *n_cut_out = S;
    if (S - plog > 16) {
        set_error("%d decomposed gates, %d of them batched (at most 16)", S, S - plog);
        return SV_ERR_UNSUPPORTED;
    }
    const int Svar = S > plog ? S - plog : 0;  // batched branch bits
    if (n_cut_out) *n_cut_out = S;
    // the listed parts that hold branches (a part whose low bits exceed every
    // branch index has none)
    std::vector<uint64_t> todo;
    for (size_t i = 0; i < nlist; ++i)
        if (!(S < 64 && (plist[i] >> S) != 0)) todo.push_back(plist[i]);
    if (todo.empty()) {
        for (size_t j = 0; j < 2 * m; ++j) out[j] = 0.0;
        return SV_OK;
    }
    // branch operators: a Z-basis projector (or Eq. 2 phase) on the first
    // qubit's partition, the phase on the second's, conditioned on the cut's
    // branch bit, which each partition holds above its own qubits
    auto build = [&]() -> sv_status {
    for (int p = 0; p < P; ++p) {
        parts[p].gates.clear();
        parts[p].cutbits.clear();
        parts[p].nbits = 0;
    }
    int k = 0;
    for (const Instr &ins0 : c.instrs) {
        Instr ins = ins0;
        if (ins.nq == 1 || side[ins.q[0]] == side[ins.q[1]]) {
            const int p = side[ins.q[0]];
            for (int j = 0; j < ins.nq; ++j) ins.q[j] = loc[ins.q[j]];
            append_lowered(ins, &parts[p].gates);
            continue;
        }
        const int qa = ins.q[0], qb = ins.q[1];
        Half &A = parts[side[qa]], &B = parts[side[qb]];
        const double theta = ins.name == "CP" ? ins.p[0] : 3.14159265358979323846;
        Instr h;
        h.name = "H";
        h.nq = 1;
        if (ins.name == "CX") {  // CX = H_t CZ H_t
            h.q[0] = loc[qb];
            append_lowered(h, &B.gates);
        }
        const uint64_t la = uint64_t(1) << loc[qa], lb = uint64_t(1) << loc[qb];
        // a fixed branch bit (one of the low plog) is a launch parameter bit:
        // the same compiled passes serve every part
        const bool fixed = k < plog;
        uint64_t ka = uint64_t(1) << (kParamBit0 + k), kb = ka;
        if (!fixed) {
            if (A.nbits >= kMaxCutBits || B.nbits >= kMaxCutBits) {
                set_error("a partition touches more than %d batched cuts", kMaxCutBits);
                return SV_ERR_UNSUPPORTED;
            }
            A.cutbits.push_back(k - plog);
            B.cutbits.push_back(k - plog);
            ka = uint64_t(1) << (A.nlocal + A.nbits++);
            kb = uint64_t(1) << (B.nlocal + B.nbits++);
        }
        if (form == 0) {
            A.gates.push_back(phase_gate(la | ka, la, 0.0));  // bit a = 1, s_k = 0: P0 removes it
            A.gates.push_back(phase_gate(la | ka, ka, 0.0));  // bit a = 0, s_k = 1: P1 removes it
            B.gates.push_back(phase_gate(lb | kb, lb | kb, std::polar(1.0, theta)));
        } else {
            for (int sb = 0; sb < 2; ++sb) {
                cd d[2];
                eq2_diag(sb, d);
                const uint64_t sva = sb ? ka : 0, svb = sb ? kb : 0;
                A.gates.push_back(phase_gate(la | ka, sva, d[0]));
                A.gates.push_back(phase_gate(la | ka, la | sva, d[1]));
                B.gates.push_back(phase_gate(lb | kb, svb, d[0]));
                B.gates.push_back(phase_gate(lb | kb, lb | svb, d[1]));
            }
        }
        if (ins.name == "CX") append_lowered(h, &B.gates);
        ++k;
    }
    for (int p = 0; p < P; ++p) {
        Half &h = parts[p];
        h.nq = h.nlocal + h.nbits < kTileM64 ? kTileM64 : h.nlocal + h.nbits;
        if (h.nlocal > kMaxPartQubits || h.nq > kMaxQubits) {
            set_error("partition %d needs %d qubits (local %d + %d branch bits)", p, h.nq, h.nlocal, h.nbits);
            return SV_ERR_UNSUPPORTED;
        }
    }
    return SV_OK;
    };
    s = build();
    if (s) return s;
    if (m == 0) return SV_OK;

    // device memory: the batched vectors + bit strings + results
    size_t bytesV = 0;
    for (int p = 0; p < P; ++p) bytesV += sizeof(float2) << parts[p].nq;
    const size_t bytesZ = m * size_t(nwords) * sizeof(uint64_t), bytesO = m * sizeof(double2);
    size_t free_b = 0, total_b = 0;
    SV_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    if (bytesV + bytesZ + bytesO + (size_t(256) << 20) > free_b) {
        set_error("decomposition needs %zu bytes of device memory, %zu free", bytesV + bytesZ + bytesO, free_b);
        return SV_ERR_OOM;
    }
    if (fault_injected("alloc")) {
        set_error("injected allocation failure");
        return SV_ERR_OOM;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint64_t *dz = nullptr;
    double2 *dout = nullptr;
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (int p = 0; p < P; ++p)
            if (parts[p].d) cudaFree(parts[p].d);
        if (dz) cudaFree(dz);
        if (dout) cudaFree(dout);
    };
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < P && e == cudaSuccess; ++p) e = cudaMalloc(&parts[p].d, sizeof(float2) << parts[p].nq);
    if (e == cudaSuccess) e = cudaMalloc(&dz, bytesZ);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&dout), bytesO);
    if (e != cudaSuccess) {
        release();
        return cuda_status(e, "cudaMalloc (decomposition)");
    }
    if (s == SV_OK) {
        e = cudaMemcpyAsync(dz, z, bytesZ, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = cuda_status(e, "cudaMemcpyAsync");
    }
    for (int p = 0; p < P && s == SV_OK; ++p) s = plan_half(parts[p], parts[p].nbits);
    for (size_t ip = 0; ip < todo.size() && s == SV_OK; ++ip) {
        // every part runs the same compiled passes (its fixed branch bits are
        // the launch parameter) on the same buffers; the stream orders its
        // halves after the previous part's sum
        for (int p = 0; p < P && s == SV_OK; ++p) s = exec_half(parts[p], st, parts[p].nbits, todo[ip]);
        if (s != SV_OK) break;
        CutSumArgs a{};
        a.accumulate = ip > 0;
        a.P = P;
        a.Sv = Svar;
        a.nwords = nwords;
        a.m = m;
        a.w = form == 1 ? std::ldexp(1.0, -S) : 1.0;
        for (int p = 0; p < P; ++p) {
            a.vec[p] = parts[p].d;
            a.nlocal[p] = parts[p].nlocal;
            a.nbits[p] = parts[p].nbits;
            for (int j = 0; j < parts[p].nbits; ++j) a.cutbit[p][j] = uint8_t(parts[p].cutbits[size_t(j)]);
            for (int i = 0; i < parts[p].nlocal; ++i) a.qubit[p][i] = uint8_t(parts[p].qubits[size_t(i)]);
        }
        const size_t blocks = (m + 7) / 8 < 4096 ? (m + 7) / 8 : 4096;
        k_cut_sum<<<unsigned(blocks), 256, 0, st>>>(dz, a, dout);
        s = check_launch(cudaGetLastError(), "k_cut_sum");
    }
    if (s == SV_OK) {
        e = cudaMemcpyAsync(out, dout, bytesO, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) s = cuda_status(e, "cudaMemcpyAsync");
    }
    if (s == SV_OK) s = sync_stream(st, "sv_cut_amplitudes");
    release();
    return s;
}

// Two partitions given by a mask (partition 0 = the mask's qubits).
static sv_status cut_mask(const char *text, int n, uint64_t maskA, int form, const uint64_t *plist, size_t nlist,
                          int plog, size_t m, const uint64_t *z, double *out, int *n_cut_out, void *stream) {
    if (n < 2 || n > 64) {
        set_error("n = %d outside 2..64 (sv_cut_amplitudes_multi takes up to %d qubits)", n, kMaxCutQubits);
        return SV_ERR_ARG;
    }
    const uint64_t all = n == 64 ? ~uint64_t(0) : ((uint64_t(1) << n) - 1);
    if ((maskA & all) == 0 || (maskA & all) == all || (maskA & ~all)) {
        set_error("maskA must select a proper, nonempty subset of the %d qubits", n);
        return SV_ERR_ARG;
    }
    uint8_t part_of[64];
    for (int q = 0; q < n; ++q) part_of[q] = (maskA >> q & 1) ? 0 : 1;
    return cut_impl(text, n, part_of, 2, form, plist, nlist, plog, m, z, 1, out, n_cut_out, stream);
}

// A list of branch parts: each < 2^plog and none repeated.
static sv_status check_parts(const uint64_t *plist, size_t nlist, int plog) {
    if (plog < 0 || plog > 16 || nlist == 0 || nlist > (size_t(1) << plog) || !plist) {
        set_error("bad part list (%zu parts of 2^%d)", nlist, plog);
        return SV_ERR_ARG;
    }
    std::vector<char> seen(size_t(1) << plog, 0);
    for (size_t i = 0; i < nlist; ++i) {
        if ((plist[i] >> plog) != 0 || seen[plist[i]]) {
            set_error("part %llu at position %zu is out of range or repeated (2^%d parts)",
                      (unsigned long long)plist[i], i, plog);
            return SV_ERR_ARG;
        }
        seen[plist[i]] = 1;
    }
    return SV_OK;
}

extern "C" sv_status sv_cut_amplitudes(const char *text, int n, uint64_t maskA, int form, size_t m, const uint64_t *z,
                                       double *out, int *n_cut_out, void *stream) {
    const uint64_t all = 0;
    return cut_mask(text, n, maskA, form, &all, 1, 0, m, z, out, n_cut_out, stream);
}

extern "C" sv_status sv_cut_amplitudes_parts(const char *text, int n, uint64_t maskA, int form, int nparts_log2,
                                             size_t nlist, const uint64_t *parts, size_t m, const uint64_t *z,
                                             double *out, int *n_cut_out, void *stream) {
    sv_status s = check_parts(parts, nlist, nparts_log2);
    return s ? s : cut_mask(text, n, maskA, form, parts, nlist, nparts_log2, m, z, out, n_cut_out, stream);
}

extern "C" sv_status sv_cut_amplitudes_multi_parts(const char *text, int n, const uint8_t *part_of, int P, int form,
                                                   int nparts_log2, size_t nlist, const uint64_t *parts, size_t m,
                                                   const uint64_t *z, double *out, int *n_cut_out, void *stream) {
    sv_status s = check_parts(parts, nlist, nparts_log2);
    return s ? s
             : cut_impl(text, n, part_of, P, form, parts, nlist, nparts_log2, m, z, (n + 63) / 64, out, n_cut_out,
                        stream);
}

extern "C" sv_status sv_cut_amplitudes_part(const char *text, int n, uint64_t maskA, int form, uint64_t part,
                                            int nparts_log2, size_t m, const uint64_t *z, double *out, int *n_cut_out,
                                            void *stream) {
    if (nparts_log2 < 0 || nparts_log2 > 16 || (part >> nparts_log2) != 0) {
        set_error("bad part %llu of 2^%d", (unsigned long long)part, nparts_log2);
        return SV_ERR_ARG;
    }
    return cut_mask(text, n, maskA, form, &part, 1, nparts_log2, m, z, out, n_cut_out, stream);
}

extern "C" sv_status sv_cut_amplitudes_multi(const char *text, int n, const uint8_t *part_of, int P, int form,
                                             uint64_t part, int nparts_log2, size_t m, const uint64_t *z,
                                             double *out, int *n_cut_out, void *stream) {
    if (nparts_log2 < 0 || nparts_log2 > 16 || (part >> nparts_log2) != 0) {
        set_error("bad part %llu of 2^%d", (unsigned long long)part, nparts_log2);
        return SV_ERR_ARG;
    }
    return cut_impl(text, n, part_of, P, form, &part, 1, nparts_log2, m, z, (n + 63) / 64, out, n_cut_out, stream);
}
