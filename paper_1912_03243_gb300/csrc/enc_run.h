// Runs of in-block gates on the two-byte code (k_enc.cu): one pass applies a
// run of consecutive gates that each act inside 256-amplitude blocks, or are
// sign flips, in circuit order with the per-gate re-encoding of the code.
#pragma once

#include <cstdint>

#include "sv_internal.h"

namespace sv {

constexpr int kEncRunMaxOps = 64;  // ops of one run (one pass)

struct EncRunOp {
    int kind;                  // 0: 2x2 update on in-block target t; 1: sign flip of the codes
    int t, c;                  // target (< 8), in-block control (-1: none)
    int shape;                 // matrix shape (exact zeros), as the single-gate kernels use it
    uint32_t lo_mask, lo_val;  // flip: in-block index bits of the condition
    uint64_t hi_mask, hi_val;  // block-index bits of the condition (block-level control / flip bits)
    float u[8];
};

// The run op of a gate on an n-qubit two-byte state, or false if the gate is
// not an in-block update or a sign flip (or n < 8).
bool enc_run_op(int n, const Gate1 &g, EncRunOp *op);
// One pass of nops <= kEncRunMaxOps ops (device array) over every block.
cudaError_t launch_enc_run(sv_state *h, const EncRunOp *d_ops, int nops);

}  // namespace sv
