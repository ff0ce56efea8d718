// Decomposition of entangling gates across a partition (Sec. 4, Eq. 2-3).
//
// Rewrite (host): qubits in maskA form partition A, the others B.  Every CZ or
// CP between A and B becomes a branch slot k; a CX between them is first
// written as H CZ H on its target.  Decomposition forms:
//   projector: CP_ab(th) = P0(a) (x) 1 + P1(a) (x) P(th)(b)   (weight 1)
//   Eq. 2:     CZ_ab = 1/2 sum_{s=+-1} D_s(a) (x) D_s(b),
//              D_s = exp(i sigma^z (x s - pi/4)), cos 2x = i  (weight 1/2 each)
// so the circuit is a sum over s in {0,1}^S of a product of an A-only and a
// B-only circuit (Sec. 4), and <z|C|0> = sum_s <z_A|W_A(s)|0><z_B|W_B(s)|0>
// (Eq. 3).
//
// Batched simulation (GPU): for each half p the 2^S branch vectors are one
// vector of 2^(n_p + S) complex64 amplitudes whose top S index bits are s.
// A branch operator is then an ordinary diagonal gate coupling a half's qubit
// to branch bit k (the projector zeroes amplitudes where bit a != s_k; P(th)
// and D_s are phases selected by (bit, s_k)).  Branch bits only ever appear
// in diagonal gates, so the tile planner keeps them outside the tiles (a
// constant per CTA) and every pass runs over all branches of a half in one
// launch.  The initial vector has amplitude 1 at index s << n_p for every s
// (or, with branch-prefix sharing, the branches are forked from branch 0 at
// their first operator, see run_half).
//
// Sum (GPU): one warp per output bit string, lanes over s, products and sum
// in FP64, times the weight.
#include <complex>
#include <cstdlib>
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

__global__ void k_branch_sum(const float2 *__restrict__ A, const float2 *__restrict__ B, int nA, int nB, int S,
                             const uint64_t *__restrict__ zA, const uint64_t *__restrict__ zB, size_t m, double w,
                             double2 *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const size_t warps = size_t(gridDim.x) * (blockDim.x >> 5);
    const uint64_t ns = uint64_t(1) << S;
    for (size_t j = size_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); j < m; j += warps) {
        const uint64_t za = zA[j], zb = zB[j];
        double re = 0.0, im = 0.0;
        for (uint64_t s = lane; s < ns; s += 32) {
            const float2 a = A[(s << nA) | za], b = B[(s << nB) | zb];
            const double ar = a.x, ai = a.y, br = b.x, bi = b.y;
            re += ar * br - ai * bi;
            im += ar * bi + ai * br;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) out[j] = make_double2(w * re, w * im);
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

struct Half {
    int nlocal = 0;     // qubits of the partition
    int nq = 0;         // qubits of the batched vector (local + branch, padded to a tile)
    std::vector<PGate> gates;
    float2 *d = nullptr;
};

// Compile and run `gates` as tiled passes over the low 2^nrun amplitudes.
sv_status run_stage(Half &h, cudaStream_t st, const std::vector<PGate> &gates, int nrun) {
    if (gates.empty()) return SV_OK;
    TilePlan<float> tp;
    sv_status s = plan_tiles<float>(gates, nrun, TileConfig{kTileM64, tile_rb64(), tile_low64(), true}, &tp);
    if (s) return s;
    std::vector<void *> fns;
    s = jit_tile_plan(tp, &fns);
    if (s) return s;
    sv_state tmp;
    tmp.n = nrun;
    tmp.dt = SV_C64;
    tmp.data = h.d;
    tmp.stream = st;
    SV_CUDA_TRY(cudaGetDevice(&tmp.device));
    for (void *fn : fns) {
        s = check_launch(launch_jit_pass(&tmp, fn, nrun, tp.rb), "branch pass");
        if (s) break;
    }
    tmp.data = nullptr;
    return s;
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

sv_status run_half(Half &h, cudaStream_t st, int S) {
    SV_CUDA_TRY(cudaMemsetAsync(h.d, 0, sizeof(float2) << h.nq, st));
    if (!prefix_sharing()) {
        k_branch_init<<<64, 256, 0, st>>>(h.d, h.nlocal, S);
        sv_status s = check_launch(cudaGetLastError(), "k_branch_init");
        return s ? s : run_stage(h, st, h.gates, h.nq);
    }
    k_branch_init<<<1, 32, 0, st>>>(h.d, h.nlocal, 0);
    sv_status s = check_launch(cudaGetLastError(), "k_branch_init");
    if (s) return s;
    int live = h.nlocal;  // live amplitudes: 2^live
    std::vector<PGate> stage;
    auto fork = [&]() -> sv_status {
        s = run_stage(h, st, stage, live > kTileM64 ? live : kTileM64);
        stage.clear();
        if (s) return s;
        const size_t bytes = sizeof(float2) << live;
        SV_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<char *>(h.d) + bytes, h.d, bytes, cudaMemcpyDeviceToDevice, st));
        ++live;
        return SV_OK;
    };
    for (const PGate &g : h.gates) {
        // branch bits are only ever conditions of diagonal gates
        const uint64_t branch = g.kind == 1 ? (g.cmask >> h.nlocal) : 0;
        while (branch >> (live - h.nlocal)) {
            s = fork();
            if (s) return s;
        }
        stage.push_back(g);
    }
    while (live < h.nlocal + S) {  // every branch bit has operators; kept for the layout
        s = fork();
        if (s) return s;
    }
    return run_stage(h, st, stage, h.nq);
}

}  // namespace
}  // namespace sv

using namespace sv;

// Sum over the branches s with s mod 2^plog == part (plog = 0: all of them).
// The low plog branch bits are then fixed: their branch operators are plain
// diagonal gates on the halves' qubits, and only the other S - plog bits are
// batched.
static sv_status cut_impl(const char *text, int n, uint64_t maskA, int form, uint64_t part, int plog, size_t m,
                          const uint64_t *z, double *out, int *n_cut_out, void *stream) {
    if (n < 2 || n > 64 || (form != 0 && form != 1) || (m > 0 && (!z || !out))) {
        set_error("bad arguments (n=%d, form=%d)", n, form);
        return SV_ERR_ARG;
    }
    const uint64_t all = n == 64 ? ~uint64_t(0) : ((uint64_t(1) << n) - 1);
    if ((maskA & all) == 0 || (maskA & all) == all || (maskA & ~all)) {
        set_error("maskA must select a proper, nonempty subset of the %d qubits", n);
        return SV_ERR_ARG;
    }
    for (size_t j = 0; j < m; ++j)
        if (z[j] & ~all) {
            set_error("bit string %zu has bits above qubit %d", j, n - 1);
            return SV_ERR_ARG;
        }
    Circuit c;
    sv_status s = parse_circuit(text, n, &c);
    if (s) return s;

    int side[64], loc[64];
    Half half[2];
    for (int q = 0; q < n; ++q) {
        side[q] = (maskA >> q & 1) ? 0 : 1;
        loc[q] = half[side[q]].nlocal++;
    }
    // count the decomposed gates first (branch bits sit above the local qubits)
    int S = 0;
    for (const Instr &ins : c.instrs) {
        if (ins.nq != 2 || side[ins.q[0]] == side[ins.q[1]]) continue;
        if (ins.name == "SWAP") {
            set_error("a SWAP across the partition cannot be decomposed");
            return SV_ERR_UNSUPPORTED;
        }
        if (form == 1 && ins.name == "CP") {
            set_error("the Eq. 2 form decomposes CZ only (CP across the partition)");
            return SV_ERR_UNSUPPORTED;
        }
        ++S;
    }
    if (S > 16) {
        set_error("%d decomposed gates (at most 16)", S);
        return SV_ERR_UNSUPPORTED;
    }
    const int Svar = S > plog ? S - plog : 0;  // batched branch bits
    if (n_cut_out) *n_cut_out = S;
    if (S < 64 && (part >> S) != 0) {  // no branch has these low bits
        for (size_t j = 0; j < 2 * m; ++j) out[j] = 0.0;
        return SV_OK;
    }
    for (int p = 0; p < 2; ++p) {
        half[p].nq = half[p].nlocal + Svar < kTileM64 ? kTileM64 : half[p].nlocal + Svar;
        if (half[p].nq > kMaxQubits) {
            set_error("half %d needs %d qubits (local %d + %d branch bits)", p, half[p].nq, half[p].nlocal, Svar);
            return SV_ERR_UNSUPPORTED;
        }
    }
    int k = 0;
    for (const Instr &ins0 : c.instrs) {
        Instr ins = ins0;
        if (ins.nq == 1 || side[ins.q[0]] == side[ins.q[1]]) {
            const int p = side[ins.q[0]];
            for (int j = 0; j < ins.nq; ++j) ins.q[j] = loc[ins.q[j]];
            append_lowered(ins, &half[p].gates);
            continue;
        }
        const int a = ins.q[0], b = ins.q[1];
        const double theta = ins.name == "CP" ? ins.p[0] : 3.14159265358979323846;
        Instr h;
        h.name = "H";
        h.nq = 1;
        if (ins.name == "CX") {  // CX = H_t CZ H_t
            h.q[0] = loc[b];
            append_lowered(h, &half[side[b]].gates);
        }
        const int qa = side[a] == 0 ? a : b, qb = side[a] == 0 ? b : a;
        const uint64_t la = uint64_t(1) << loc[qa], lb = uint64_t(1) << loc[qb];
        const bool fixed = k < plog;
        const int sfix = int((part >> k) & 1);
        const uint64_t ka = fixed ? 0 : uint64_t(1) << (half[0].nlocal + k - plog);
        const uint64_t kb = fixed ? 0 : uint64_t(1) << (half[1].nlocal + k - plog);
        if (form == 0) {
            if (fixed) {
                half[0].gates.push_back(phase_gate(la, sfix ? 0 : la, 0.0));  // keep bit a == s_k
                if (sfix) half[1].gates.push_back(phase_gate(lb, lb, std::polar(1.0, theta)));
            } else {
                half[0].gates.push_back(phase_gate(la | ka, la, 0.0));  // bit a = 1, s_k = 0: P0 removes it
                half[0].gates.push_back(phase_gate(la | ka, ka, 0.0));  // bit a = 0, s_k = 1: P1 removes it
                half[1].gates.push_back(phase_gate(lb | kb, lb | kb, std::polar(1.0, theta)));
            }
        } else {
            for (int sb = 0; sb < 2; ++sb) {
                if (fixed && sb != sfix) continue;
                cd d[2];
                eq2_diag(sb, d);
                const uint64_t sva = sb ? ka : 0, svb = sb ? kb : 0;
                half[0].gates.push_back(phase_gate(la | ka, sva, d[0]));
                half[0].gates.push_back(phase_gate(la | ka, la | sva, d[1]));
                half[1].gates.push_back(phase_gate(lb | kb, svb, d[0]));
                half[1].gates.push_back(phase_gate(lb | kb, lb | svb, d[1]));
            }
        }
        if (ins.name == "CX") append_lowered(h, &half[side[b]].gates);
        ++k;
    }
    if (m == 0) return SV_OK;

    // device memory: two batched vectors + bit strings + results
    const size_t bytesA = sizeof(float2) << half[0].nq, bytesB = sizeof(float2) << half[1].nq;
    const size_t bytesZ = 2 * m * sizeof(uint64_t), bytesO = m * sizeof(double2);
    size_t free_b = 0, total_b = 0;
    SV_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    if (bytesA + bytesB + bytesZ + bytesO + (size_t(256) << 20) > free_b) {
        set_error("decomposition needs %zu bytes of device memory, %zu free", bytesA + bytesB + bytesZ + bytesO, free_b);
        return SV_ERR_OOM;
    }
    if (fault_injected("alloc")) {
        set_error("injected allocation failure");
        return SV_ERR_OOM;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint64_t *dz = nullptr;
    double2 *dout = nullptr;
    std::vector<uint64_t> zs(2 * m);
    for (size_t j = 0; j < m; ++j) {
        uint64_t za = 0, zb = 0;
        for (int q = 0; q < n; ++q) {
            const uint64_t bit = (z[j] >> q) & 1;
            if (side[q] == 0) za |= bit << loc[q];
            else zb |= bit << loc[q];
        }
        zs[j] = za;
        zs[m + j] = zb;
    }
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (Half &h : half)
            if (h.d) cudaFree(h.d);
        if (dz) cudaFree(dz);
        if (dout) cudaFree(dout);
    };
    cudaError_t e = cudaMalloc(&half[0].d, bytesA);
    if (e == cudaSuccess) e = cudaMalloc(&half[1].d, bytesB);
    if (e == cudaSuccess) e = cudaMalloc(&dz, bytesZ);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&dout), bytesO);
    if (e != cudaSuccess) {
        release();
        return cuda_status(e, "cudaMalloc (decomposition)");
    }
    for (int p = 0; p < 2 && s == SV_OK; ++p) s = run_half(half[p], st, Svar);
    if (s == SV_OK) {
        e = cudaMemcpyAsync(dz, zs.data(), bytesZ, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = cuda_status(e, "cudaMemcpyAsync");
    }
    if (s == SV_OK) {
        const double w = form == 1 ? std::ldexp(1.0, -S) : 1.0;
        const size_t blocks = (m + 7) / 8 < 4096 ? (m + 7) / 8 : 4096;
        k_branch_sum<<<unsigned(blocks), 256, 0, st>>>(half[0].d, half[1].d, half[0].nlocal, half[1].nlocal, Svar, dz,
                                                       dz + m, m, w, dout);
        s = check_launch(cudaGetLastError(), "k_branch_sum");
    }
    if (s == SV_OK) {
        e = cudaMemcpyAsync(out, dout, bytesO, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) s = cuda_status(e, "cudaMemcpyAsync");
    }
    if (s == SV_OK) s = sync_stream(st, "sv_cut_amplitudes");
    release();
    return s;
}

extern "C" sv_status sv_cut_amplitudes(const char *text, int n, uint64_t maskA, int form, size_t m, const uint64_t *z,
                                       double *out, int *n_cut_out, void *stream) {
    return cut_impl(text, n, maskA, form, 0, 0, m, z, out, n_cut_out, stream);
}

extern "C" sv_status sv_cut_amplitudes_part(const char *text, int n, uint64_t maskA, int form, uint64_t part,
                                            int nparts_log2, size_t m, const uint64_t *z, double *out, int *n_cut_out,
                                            void *stream) {
    if (nparts_log2 < 0 || nparts_log2 > 16 || (part >> nparts_log2) != 0) {
        set_error("bad part %llu of 2^%d", (unsigned long long)part, nparts_log2);
        return SV_ERR_ARG;
    }
    return cut_impl(text, n, maskA, form, part, nparts_log2, m, z, out, n_cut_out, stream);
}
