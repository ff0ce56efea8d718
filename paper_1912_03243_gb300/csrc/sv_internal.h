// Internal declarations of libsv (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sv.h"

namespace sv {

constexpr int kMaxQubits = 40;
constexpr int kEncBlockLog2 = 8;  // 256 amplitudes per two-byte code block
constexpr int kEncBlock = 1 << kEncBlockLog2;

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
sv_status cuda_status(cudaError_t e, const char *what);
bool fault_injected(const char *what);  // SV_FAULT_INJECT host-side hooks
// Allocate (once) and zero the handle's device error word, which kernels
// with bounded waits set to SV_ERR_TIMEOUT when a wait gives up.
cudaError_t ensure_err_word(::sv_state *h);
// Map a launch result (and the "launch" fault hook) to a status.
sv_status check_launch(cudaError_t e, const char *what);

// Kernel attributes (cudaFuncSetAttribute) belong to a device: one flag bit
// per device records that a kernel family's attributes were set there.
// Setting them twice is harmless, so concurrent first calls need no lock.
inline bool attrs_needed(const std::atomic<uint64_t> &done, int device) {
    return device < 0 || device >= 64 || !((done.load(std::memory_order_acquire) >> device) & 1u);
}
inline void attrs_set(std::atomic<uint64_t> &done, int device) {
    if (device >= 0 && device < 64) done.fetch_or(uint64_t(1) << device, std::memory_order_release);
}
// Synchronise a stream (and honour the "sync" fault hook).
sv_status sync_stream(cudaStream_t st, const char *what);

#define SV_CUDA_TRY(expr)                                            \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return ::sv::cuda_status(_e, #expr); \
    } while (0)

// ---------------------------------------------------------------- gates
struct Cplx {
    double re, im;
};

// A parsed instruction of the circuit text.
struct Instr {
    std::string name;
    int nq = 1;
    int q[2] = {0, 0};
    int np = 0;
    double p[8] = {0};
};

struct Circuit {
    int n = -1;
    std::vector<Instr> instrs;
};

// Parse circuit text; returns SV_OK or SV_ERR_PARSE / SV_ERR_ARG.
sv_status parse_circuit(const char *text, int n_expected, Circuit *out);

// Library gate table: 2x2 (1-qubit) or 4x4 (2-qubit) complex matrices.
int gate_matrix(const std::string &name, const double *p, int np, Cplx *m);

// A single-qubit (optionally controlled) update: the unit the per-gate
// kernels apply.  U is 2x2 row-major.
struct Gate1 {
    int target;
    int control;  // -1: none
    Cplx u[4];
};

// Lower a parsed circuit to controlled single-qubit updates:
// CZ a b -> Z(b | a), CX c t -> X(t | c), CP c t th -> P(th)(t | c),
// SWAP a b -> CX a b, CX b a, CX a b.
std::vector<Gate1> lower_to_gate1(const Circuit &c);

// ---------------------------------------------------------------- state
struct sv_state_impl;

}  // namespace sv

struct sv_state {
    int n = 0;
    sv_dtype dt = SV_C64;
    void *data = nullptr;  // amplitudes (or codes for SV_ENC2B)
    float *scales = nullptr;  // SV_ENC2B only: points into data
    size_t bytes = 0;
    bool owned = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    // scratch (library-owned, small)
    double *d_partials = nullptr;  // norm partial sums
    int partials_cap = 0;
    uint64_t *d_idx = nullptr;     // amplitude gather indices
    double *d_amps = nullptr;      // gathered amplitudes
    size_t gather_cap = 0;
    void *d_mat = nullptr;         // fused-gate matrix upload (64 KB)
    int *d_err = nullptr;          // device error word (bounded waits that gave up)
    double *d_expect = nullptr;    // expectation-value partial sums (per pass and CTA)
    size_t expect_cap = 0;         // their capacity in doubles
    int live_plans = 0;
};

namespace sv {

// ---------------------------------------------------------------- kernels
// All launchers enqueue on `st` and return the launch error (if any).
cudaError_t launch_gate1(sv_state *h, const Gate1 &g);
cudaError_t launch_set_basis(sv_state *h, uint64_t idx);
cudaError_t launch_norm(sv_state *h, double *d_out);  // d_out: device double
cudaError_t launch_gather(sv_state *h, const uint64_t *d_idx, size_t m, double *d_out);
int norm_partials_needed(const sv_state *h);

// two-byte code
cudaError_t launch_enc_gate1(sv_state *h, const Gate1 &g);
cudaError_t launch_encode(const sv_state *src, sv_state *dst);
cudaError_t launch_decode(const sv_state *src, sv_state *dst);
cudaError_t launch_enc_gather(sv_state *h, const uint64_t *d_idx, size_t m, double *d_out);
cudaError_t launch_enc_norm(sv_state *h, double *d_out);

}  // namespace sv
