// Tensor-core dense k-qubit blocks (k_fused_tc.cu): launch arguments shared
// with the plan code, which prepares every block of a fused plan once.
#pragma once

#include <cstdint>

#include "sv_internal.h"

namespace sv {

constexpr int kTcM = 12;                            // tile bits (2^12 amplitudes per tile)
constexpr int kTcN = 1 << (kTcM - 6);               // B columns per tile (2^(kTcM + 1) reals / 128)
constexpr size_t kTcOperandBytes = 2 * 128 * 128 * 2;  // A hi + A lo, BF16 (64 KiB)

struct TcArgs {
    int n, k, P;
    int nouter;
    int lc;
    uint64_t ntiles;
    long long timeout_ns;
    int skip_mma;                 // test hook: never issue the MMA (the wait must time out)
    uint8_t epi_mode;             // kernel and epilogue form (k_fused_tc.cu): 0, 1 pipeline; 2 two groups
    // form 0 loads tiles with tensor-map copies: the tile's qubit ranges as
    // the map's dimensions (a dimension starts at qubit tma_start[d] and ends
    // where the next starts; the last ends at n), tma_nbox boxes per tile at
    // global offsets tma_boff[b] (the top tile runs, when there are more than
    // the map's five dimensions can hold)
    uint8_t tma, tma_rank, tma_nbox;
    uint8_t tma_start[5];
    uint64_t tma_boff[4];
    uint8_t tile_pos[kTcM];
    uint8_t outer_pos[40];
    uint16_t offL[64];            // tile index offset of block-local index l
    uint16_t offP[64];            // tile index offset of pack p
    uint16_t offN[kTcN];          // tile index offset of column n
};

// Build the BF16 hi/lo operand image of block U (a_ops: 2 * 128 * 128
// elements) and the launch arguments for an n-qubit state.
void tc_prepare(int n, int k, const int *qubits, const double *U, uint16_t *a_ops, TcArgs *args);
// Launch with operands already in device memory (dA: kTcOperandBytes).
cudaError_t tc_launch(sv_state *h, const TcArgs &args, const void *dA);
// The kernel (and its load form) a launch with these arguments runs.
const char *tc_kernel_name(const TcArgs &a);

}  // namespace sv
