// Circuit plans: the host-side planner output that sv_plan_execute replays.
#pragma once

#include <string>
#include <vector>

#include "enc_run.h"
#include "fused_tc.h"
#include "sv_internal.h"
#include "tile.h"

namespace sv {

constexpr int kMaxFusedQubits = 6;

// Dense k-qubit block (sv_apply_fused); U is 2^k x 2^k complex row-major on
// the host, copied into handle scratch before the launch.  complex64 states
// of at least one tensor-core tile (2^12 amplitudes) run on the tensor cores
// (launch_fused_tc), the rest on the CUDA cores.
cudaError_t launch_fused(sv_state *h, int k, const int *qubits, const double *U);
bool fused_tc_supported(const sv_state *h);
cudaError_t launch_fused_tc(sv_state *h, int k, const int *qubits, const double *U);

// A k-qubit block of a fused plan: the ordered product of the gates it
// absorbed, 2^k x 2^k complex row-major (re, im), local bit j <-> qubits[j].
struct FusedBlock {
    int k = 0;
    int qubits[kMaxFusedQubits] = {0};
    std::vector<double> U;
    int gates = 0;
};

// Greedy fusion of the circuit into blocks of at most kmax qubits; gates are
// reordered only across gates they commute with.  Returns the blocks.
std::vector<FusedBlock> fuse_blocks(const Circuit &c, int kmax);

// Algorithmic HBM bytes of one per-gate update (what the method must move:
// read + write of every amplitude the update changes).
double gate1_bytes(const sv_state *h, const Gate1 &g);

// Name of the kernel launch_gate1 picks for g.
const char *gate1_kernel_name(const sv_state *h, const Gate1 &g);

}  // namespace sv

// One kernel launch of a plan.
struct PlanLaunch {
    int kind;      // 0: per-gate update pergate[index]; 1: compiled tile pass tfns[index];
                   // 2: tensor-core block tcargs[index]; 3: CUDA-core block blocks[index];
                   // 4: run of in-block two-byte-code gates encruns[index]
    int index;
    double bytes;  // algorithmic bytes
    double lane_ops = 0.0;  // compiled tile passes: FP32 lane operations per amplitude (at least)
    int segments = 0;       // compiled tile passes: register segments
};

struct sv_plan_s {
    sv_state *h = nullptr;
    int mode = 0;
    int64_t gates = 0;                     // gates of the circuit text
    std::vector<sv::Gate1> pergate;        // per-gate updates
    struct EncRun {
        int first, count, gates;           // ops d_encops[first .. first + count), circuit gates they apply
    };
    std::vector<EncRun> encruns;           // two-byte code: runs of in-block gates, one pass each
    sv::EncRunOp *d_encops = nullptr;      // their ops (device)
    std::vector<void *> tfns;              // compiled tile passes
    int tile_rb = 0;                       // their register bits per thread
    std::vector<double> tile_lane_ops;     // their FP32 lane operations per amplitude
    std::vector<int> tile_nseg;            // their register segments
    std::string tuning;                    // SV_MODE_AUTO: the measured candidates (JSON), else empty
    std::vector<sv::FusedBlock> blocks;    // fused blocks (CUDA-core kernel)
    std::vector<sv::TcArgs> tcargs;        // fused blocks (tensor-core kernel)
    void *d_tcA = nullptr;                 // their operand images, kTcOperandBytes each
    int fused_k = 0;
    std::vector<PlanLaunch> launches;      // execution order
    double bytes = 0.0;                    // algorithmic bytes of one execution
    // CUDA graph of the launches, from the second execution on: captured on a
    // private stream that joins the handle's stream through two events (the
    // handle's stream may be the legacy default stream, which cannot be
    // captured).  The first execution runs the launches directly and does the
    // one-time set-up they need (error word, kernel attributes).
    int64_t execs = 0;
    bool graph_off = false;                // capture failed or not applicable: direct launches
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec = nullptr;
};

namespace sv {
// Every launch of a plan, in order, on the stream of its handle (no graph).
cudaError_t plan_launch_all(sv_plan_s *p);
// Whether a plan's launches can be captured into a CUDA graph (no host-side
// copies between them).
bool plan_capturable(const sv_plan_s *p);
}  // namespace sv
