// Dense k-qubit block (Sec. 2: a gate on k qubits is a 2^k x 2^k matrix on
// the amplitudes that differ only in those qubits) on the 5th-generation
// tensor cores, complex64 state.
//
// Real expansion: with amplitudes interleaved (re, im), the complex block U
// acts as the 2d x 2d real matrix Ut, Ut[2r+a][2c+b] = [[Re, -Im], [Im, Re]]
// of U[r][c] (d = 2^k).  A = I_P (x) Ut (P = 64/d copies on the diagonal) is
// always 128 x 128, so one MMA shape (M = 128, N = kTcN = 64, K = 16 per
// instruction) serves every k <= 6; column n of B holds P groups of d
// amplitudes.  For k < 6 most of each product multiplies zeros: harmless
// while the kernel is bound by memory traffic.
//
// Split precision: A = Ah + Al and B = Bh + Bl with BF16 parts (Ah = bf16(A),
// Al = bf16(A - Ah)); D = Ah Bh + Ah Bl + Al Bh accumulates in FP32 in tensor
// memory (relative error about 2^-16 per product instead of 2^-8).
//
// Both kernels keep A in tensor memory (row m in lane m, two BF16 K elements
// per 32-bit column; A_hi in columns 0-63, A_lo in 64-127, written once),
// with two FP32 accumulators of 64 columns after it, and work on tiles of
// 2^12 amplitudes: the k block qubits plus the lowest other qubits, so tile
// bits 0..5 are always state qubits 0..5 and B is 128 x 64.  The host picks
// the kernel per launch from the qubit layout (TcArgs::epi_mode):
//
// k_fused_tc, a warp-specialised pipeline over a ring of four FP32 staging
// tiles, when the accumulator's columns or its rows run along the low
// qubits (every k = 6 block without qubit 0, or with qubits 0..3):
//   loads: tensor-map copies (cp.async.bulk.tensor, 128-byte swizzle) by one
//     thread, counted in bytes on the slot's mbarrier, when the columns run
//     along the low qubits (form 0: the split's lanes along the columns then
//     meet few bank conflicts in the swizzled rows); otherwise 3 loader warps
//     with 16-byte cp.async (the slot's mbarrier counts each loader thread
//     once its copies have landed: cp.async.mbarrier.arrive);
//   converter warps (8): BF16 hi / lo split of a slot into one of two B
//     operands (K-major no-swizzle canonical layout), after which the slot
//     is free for the next load;
//   MMA thread: 3 x 8 tcgen05.mma into one of the two accumulators,
//     committed to the B operand's and the accumulator's mbarriers;
//   epilogue warps (4, one per 32 tensor-memory lanes): tcgen05.ld of the
//     accumulator, re / im of each amplitude joined by one shuffle, then to
//     HBM: through a padded per-warp buffer, half the columns at a time,
//     each store instruction writing rows of 16 columns (form 0: columns
//     0..3 are qubits 0..1, so at least whole 32-byte sectors), or straight
//     from the registers, 8 bytes per lane (form 1: each warp's 16 rows are
//     qubits 0..3).
// In steady state the loads of the next tiles, the split of one, the MMAs
// of another and the epilogue of a third run at once.
//
// k_fused_tc_groups otherwise (k < 6, or qubit 0 in the block among others
// far apart): two groups of 256 threads per CTA, each with its own B
// operand, ring of two staging tiles, accumulator, mbarrier and named
// barrier; per tile and group: the tile's cp.async was issued one tile
// earlier -> split into Bh, Bl -> one thread issues the 3 x 8 MMAs and
// commits -> the group waits (bounded) -> tcgen05.ld, scattered back into
// the staging tile -> coalesced 16-byte stores.
//
// Measured (26 qubits, 6-qubit blocks, per launch): blocks {0..5} 221 us in
// the pipeline (form 1) against 263 us in two groups; {20..25} 221 us (form
// 0, tensor-map loads; 240 with cp.async) against 255; a mixed block whose
// columns start with qubits 0..2 232 (258) against 265.  Alternatives measured and dropped: bulk copies
// (cp.async.bulk) of the tile's 512-byte runs by one producer warp, in and
// out (about 2.1x slower: 64 copies each way per tile kept the copy engine
// busy about 75 cycles per copy); results written back into the slot and
// stored by two loader warps (1.2x slower); six loader and four converter
// warps (1.3x slower: the loads issue sooner but wait longer in the memory
// pipeline); five ring slots with one B operand (1.3x slower: the split then
// waits for each tile's MMAs); for the other layouts, the pipeline with the results written
// through a shared write-back tile and a three-slot ring (about 330 us per
// launch, 1.2-1.3x slower than two groups) or straight from the registers
// (up to 2.6x slower: 8-byte pieces far apart).
// Timeout: every wait is bounded by %globaltimer; the first to run out
// raises a flag that ends every role's loop, the loaders wait for their
// copies in flight, the CTA frees its tensor memory and the host sees
// SV_ERR_TIMEOUT.  The test hook (skip_mma) issues no MMA, so nothing is in
// flight then.  After a real timeout the committed MMAs may still be writing
// the freed tensor memory and may later arrive on an mbarrier in shared
// memory the CTA has released: the state and the CUDA context must then be
// treated as undefined and discarded, not reused.
// B operand layout (K-major, no swizzle): element (row, kk) at byte
// (row%8)*16 + (kk%8)*2 + (kk/8)*128 + (row/8)*2048; leading-dimension byte
// offset 128 (next 8 K-elements), stride-dimension byte offset 2048 (next 8
// rows); the K-slice s of an instruction starts at + 256 s (and at column
// + 8 s of A in tensor memory).
#include <cuda.h>  // CUtensorMap and its encoder's types (the encoder is fetched at run time, not linked)
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "fused_tc.h"
#include "plan.h"

namespace sv {
namespace {

constexpr int kTcACols = 64;                   // TMEM columns of one 128 x 128 BF16 A operand
constexpr int kTcAccs = 2;                     // accumulators (tiles between MMA and epilogue)
// A_hi, A_lo and the accumulators, in an allocation of a power of two
constexpr int kTcCols = 256;
static_assert(2 * kTcACols + kTcAccs * kTcN <= kTcCols, "tensor memory allocation");
constexpr uint32_t kBBytes = kTcN * 128 * 2;   // one BF16 B operand (16 KiB)
constexpr uint32_t kStageBytes = (1u << kTcM) * 8;  // one FP32 staging tile (32 KiB)
// two-group kernel: staging tiles per group (kTcRing - 1 loads in flight);
// two fill the shared memory of two groups.  (2^11-amplitude tiles with a
// ring of five measured slower: the per-tile MMA round trip then dominates.)
constexpr int kTcGroup = 256;                  // threads of one group
constexpr int kTcGroups = 2;                   // groups (tiles in flight) per CTA
constexpr int kTcThreads = kTcGroups * kTcGroup;
static_assert(kTcGroups <= kTcAccs, "one accumulator per group");
constexpr int kTcRing = 2;
constexpr int kChunkIters = (1 << kTcM) / 2 / kTcGroup;  // 16-byte chunks per thread and tile

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g) : "memory");
}
// commit this thread's copies issued since the last commit as one group, then
// wait until at most kTcRing - 1 groups (the newest) are still in flight
__device__ __forceinline__ void cp_async_commit_wait_ring() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group %0;\n" ::"n"(kTcRing - 1) : "memory");
}
// barrier of one 256-thread group (named barrier 1 + g)
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 256;\n" ::"r"(1 + g) : "memory"); }
// Staging tile layout: 16-byte chunk c (amplitudes 2c, 2c+1) lives at chunk
// c ^ ((c>>3 ^ c>>6 ^ c>>9) & 7), which spreads the B-operand reads (lanes
// along group bits, which may lie above the low run) over the banks.
__device__ __forceinline__ uint32_t swz(uint32_t c) { return c ^ (((c >> 3) ^ (c >> 6) ^ (c >> 9)) & 7u); }
__device__ __forceinline__ uint32_t sxpos(uint32_t j) { return (swz(j >> 1) << 1) | (j & 1u); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29),
// SBO >> 4 (32-45), fixed 0b001 at bits 46-48, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = uint64_t((saddr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28 (M = 128, N = kTcN).
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t(kTcN) >> 3) << 17) | ((128u >> 4) << 24);

// D (tensor memory) [+]= A (tensor memory) x B (shared memory descriptor)
__device__ __forceinline__ void mma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t accum) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bdesc), "r"(kIdesc), "r"(accum)
        : "memory");
}

// 64 consecutive 32-bit columns of this warp's 32 lanes <- r
__device__ __forceinline__ void tmem_st64(uint32_t taddr, const uint32_t *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x64.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,"
        "%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63,%64};\n" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
        "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
        "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31]), "r"(r[32]), "r"(r[33]), "r"(r[34]), "r"(r[35]), "r"(r[36]),
        "r"(r[37]), "r"(r[38]), "r"(r[39]), "r"(r[40]), "r"(r[41]), "r"(r[42]), "r"(r[43]), "r"(r[44]), "r"(r[45]),
        "r"(r[46]), "r"(r[47]), "r"(r[48]), "r"(r[49]), "r"(r[50]), "r"(r[51]), "r"(r[52]), "r"(r[53]), "r"(r[54]),
        "r"(r[55]), "r"(r[56]), "r"(r[57]), "r"(r[58]), "r"(r[59]), "r"(r[60]), "r"(r[61]), "r"(r[62]), "r"(r[63])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// kTcN / 2 consecutive columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld_half(uint32_t taddr, float *v) {
    static_assert(kTcN == 32 || kTcN == 64, "read-back written for 32 or 64 accumulator columns");
    uint32_t r[kTcN / 2];
    if constexpr (kTcN == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < kTcN / 2; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kTcThreads, 1) k_fused_tc_groups(float2 *__restrict__ psi, const uint4 *__restrict__ gA,
                                                            int *__restrict__ err, const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[kTcGroups];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag[kTcGroups];
    // index tables in shared memory: lanes read different entries (a kernel-
    // parameter array would serialise on the constant cache)
    __shared__ uint16_t tL[64], tP[64], tN[kTcN];          // swizzled staging offsets of l, p, n
    __shared__ uint16_t tK[64];                            // offset of K elements 2i, 2i + 1 (one amplitude)
    __shared__ uint64_t tB[4][256];                        // global offset of each byte of the tile number
    __shared__ uint64_t gHi[kChunkIters];                  // global offset of the chunk bits above 7
    __shared__ uint16_t sHi[kChunkIters];                  // swizzled chunk of the chunk bits above 7
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = tid / kTcGroup, lt = tid % kTcGroup, gw = warp & 7;  // group, thread and warp in the group
    unsigned char *gbase = smem + size_t(g) * (2 * kBBytes + kTcRing * kStageBytes);
    unsigned char *sBh = gbase, *sBl = gbase + kBBytes;
    unsigned char *sStage = gbase + 2 * kBBytes;  // kTcRing FP32 staging tiles of 2^kTcM amplitudes
    const uint32_t mbar_a = smem_u32(&mbar[g]);

    for (int i = tid; i < 64; i += kTcThreads) {
        if (i < kTcN) tN[i] = uint16_t(sxpos(a.offN[i]));
        tL[i] = uint16_t(sxpos(a.offL[i]));
        tP[i] = uint16_t(sxpos(a.offP[i]));
        {  // K elements 2i, 2i + 1
            const int kk = 2 * i, klg = a.k + 1, rm = (2 << a.k) - 1;
            tK[i] = uint16_t(sxpos(a.offL[(kk & rm) >> 1] ^ a.offP[kk >> klg]));
        }
        if (i < kChunkIters) {  // chunk c = lt + 256 i: tile index bits 9.. of j = 2c
            const uint32_t j = uint32_t(i) << 9;
            uint64_t gg = 0;
            for (int q = 0; q < kTcM; ++q)
                if (j >> q & 1) gg |= uint64_t(1) << a.tile_pos[q];
            gHi[i] = gg;
            sHi[i] = uint16_t(swz(uint32_t(i) << 8));
        }
    }
    // the tile number's outer bits, one table per byte (tile numbers < 2^32)
    for (int i = tid; i < 4 * 256; i += kTcThreads) {
        const int byte = i >> 8, v = i & 255;
        uint64_t off = 0;
        for (int b = 0; b < 8; ++b) {
            const int q = 8 * byte + b;
            if ((v >> b & 1) && q < a.nouter) off |= uint64_t(1) << a.outer_pos[q];
        }
        tB[byte][v] = off;
    }
    // this thread's chunk bits 0..7 (tile index bits 1..8)
    uint64_t gLo = 0;
    for (int q = 1; q <= 8; ++q)
        if ((uint32_t(lt) << 1) >> q & 1) gLo |= uint64_t(1) << a.tile_pos[q];
    const uint32_t sLo = swz(uint32_t(lt));
    if (lt == 0) {
        abort_flag[g] = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();  // tmem_slot
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // the A operands go to tensor memory once: group 0's warp w writes lanes
    // 32 (w % 4) .. +31 of A_hi (w < 4) or A_lo (w >= 4), one row per thread
    // (gA: row-major BF16, A_hi then A_lo)
    if (g == 0) {
        const int q = gw & 3, h = gw >> 2, m = 32 * q + lane;
        uint32_t r[64];
        const uint4 *src = gA + (size_t(h) * 128 * 128 * 2 + size_t(m) * 256) / 16;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const uint4 v = src[i];
            r[4 * i] = v.x;
            r[4 * i + 1] = v.y;
            r[4 * i + 2] = v.z;
            r[4 * i + 3] = v.w;
        }
        tmem_st64(tmem_slot + (uint32_t(32 * q) << 16) + uint32_t(kTcACols * h), r);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot + uint32_t(2 * kTcACols + g * kTcN);  // this group's accumulator columns
    const int klog = a.k + 1, rmask = (2 << a.k) - 1;        // 2d = 2^(k+1)
    // K element kk = 2i, 2i + 1 (re, im of one amplitude): pack p = kk >> klog,
    // real row r = kk & rmask (tables written before the barrier above)
    // per-thread constants of the convert (B row) and of the read-back (D row)
    const uint32_t sn = tN[lt & (kTcN - 1)];
    const int drow = 32 * (gw & 3) + lane;
    const uint32_t srow = tL[(drow & rmask) >> 1] ^ tP[drow >> klog];
    const int dcomp = drow & 1;

    auto tile_base = [&](uint64_t tile) {
        return tB[0][tile & 255] | tB[1][(tile >> 8) & 255] | tB[2][(tile >> 16) & 255] | tB[3][(tile >> 24) & 255];
    };
    // 16-byte chunks c = lt + 256 i (2 amplitudes, tile index 2c); offsets
    // split into a per-thread and a per-i part (disjoint bits)
    auto load_tile = [&](uint64_t tile, int buf) {
        const uint64_t base = tile_base(tile);
        float2 *sx = reinterpret_cast<float2 *>(sStage + buf * kStageBytes);
#pragma unroll
        for (int i = 0; i < kChunkIters; ++i)
            cp_async16(smem_u32(sx + 2 * (sLo ^ sHi[i])), psi + (base | gLo | gHi[i]));
    };

    uint32_t phase = 0;
    int buf = 0;
    const uint64_t stride = uint64_t(kTcGroups) * gridDim.x;
    const uint64_t first = uint64_t(kTcGroups) * blockIdx.x + uint64_t(g);
    // a ring of kTcRing staging tiles: the loads of the next kTcRing - 1
    // tiles are in flight while one is converted, multiplied, read back and
    // stored; one cp.async group per tile (an empty group past the end)
    for (int r = 0; r < kTcRing - 1; ++r) {
        const uint64_t tt = first + uint64_t(r) * stride;
        if (tt < a.ntiles) load_tile(tt, r);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    for (uint64_t tile = first; tile < a.ntiles; tile += stride, buf = buf + 1 == kTcRing ? 0 : buf + 1) {
        // the staging tile before this one in the ring was stored before the
        // last iteration's closing barrier: it takes the load kTcRing - 1 ahead
        const uint64_t ahead = tile + uint64_t(kTcRing - 1) * stride;
        if (ahead < a.ntiles) load_tile(ahead, buf == 0 ? kTcRing - 1 : buf - 1);
        cp_async_commit_wait_ring();
        group_sync(g);
        float2 *sX = reinterpret_cast<float2 *>(sStage + buf * kStageBytes);
        const uint64_t base = tile_base(tile);
        // convert: one task = one B row n and 8 consecutive K elements (16 B
        // of Bh and of Bl); a thread's row n = lt % kTcN is the same in all
        // its tasks
        static_assert(kTcGroup % kTcN == 0, "fixed B row per thread");
#pragma unroll
        for (int t = lt; t < 16 * kTcN; t += kTcGroup) {
            const int nrow = t & (kTcN - 1), q8 = t / kTcN;
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {  // elements kk, kk+1: re and im of one amplitude
                const float2 amp = sX[sn ^ tK[q8 * 4 + (e >> 1)]];
                const __nv_bfloat162 hi = __float22bfloat162_rn(amp);
                const float2 hf = __bfloat1622float2(hi);
                const __nv_bfloat162 lo = __float22bfloat162_rn(make_float2(amp.x - hf.x, amp.y - hf.y));
                hw[e >> 1] = *reinterpret_cast<const uint32_t *>(&hi);
                lw[e >> 1] = *reinterpret_cast<const uint32_t *>(&lo);
            }
            const uint32_t off = uint32_t((nrow & 7) * 16 + q8 * 128 + (nrow >> 3) * 2048);
            *reinterpret_cast<uint4 *>(sBh + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(sBl + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        // generic-proxy writes -> async proxy (the tensor core reads them)
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        group_sync(g);
        if (lt == 0 && !a.skip_mma) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t bh = smem_u32(sBh), bl = smem_u32(sBl);
            uint32_t acc = 0;
#pragma unroll
            for (int pass = 0; pass < 3; ++pass) {
                const uint32_t aa = tmem_slot + uint32_t(pass == 2 ? kTcACols : 0), bb = pass == 1 ? bl : bh;
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    mma_bf16_ts(tmem, aa + 8u * s, sdesc(bb + 256u * s, 128, 2048), acc);
                    acc = 1;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar_a)
                         : "memory");
        }
        // bounded wait for the MMAs (they finish in microseconds)
        {
            const uint64_t t0 = globaltimer();
            uint32_t done = 0;
            while (!done) {
                asm volatile(
                    "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(done)
                    : "r"(mbar_a), "r"(phase)
                    : "memory");
                if (!done && globaltimer() - t0 > uint64_t(a.timeout_ns)) {
                    abort_flag[g] = 1;
                    break;
                }
            }
        }
        group_sync(g);
        if (abort_flag[g]) break;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // read D: warp gw of the group reads lanes 32 (gw % 4) .. +31 and
        // half of the columns (a warp reaches the lanes 32 (warp % 4) .. +31;
        // warp % 4 = gw % 4)
        {
            float *sXf = reinterpret_cast<float *>(sX);
            const int c0 = (kTcN / 2) * (gw >> 2);
            float v[kTcN / 2];
            tmem_ld_half(tmem + (uint32_t(32 * (gw & 3)) << 16) + uint32_t(c0), v);
#pragma unroll
            for (int i = 0; i < kTcN / 2; ++i) sXf[2 * (srow ^ tN[c0 + i]) + dcomp] = v[i];
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        group_sync(g);
        // store
#pragma unroll
        for (int i = 0; i < kChunkIters; ++i)
            *reinterpret_cast<float4 *>(psi + (base | gLo | gHi[i])) =
                *reinterpret_cast<const float4 *>(sX + 2 * (sLo ^ sHi[i]));
        group_sync(g);
    }
    // no copy may still be writing shared memory when the CTA leaves
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (abort_flag[g] && lt == 0) atomicExch(err, int(SV_ERR_TIMEOUT));
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_slot), "r"(kTcCols)
                     : "memory");
    }
}

// ------------------------------------------------------------------------
// The pipeline's shape.  Staging slots use the layout above (XOR-linear in
// the tile index: table entries of disjoint bits combine by XOR).
constexpr int kPipeStages = 4;                      // ring slots
constexpr int kPipeBBufs = 2;                       // B operands (hi + lo each; the indexing assumes two)
// with the MMA warp 16 warps: 4 per SM sub-partition (128 registers)
constexpr int kConvWarps = 8, kEpiWarps = 4, kLoadWarps = 3;
constexpr int kConvThreads = 32 * kConvWarps, kLoadThreads = 32 * kLoadWarps;
constexpr int kPipeThreads = 32 * (kConvWarps + kEpiWarps + kLoadWarps + 1);  // + MMA warp
constexpr int kLoadWarp0 = kConvWarps + kEpiWarps, kMmaWarp = kLoadWarp0 + kLoadWarps;
constexpr int kTileChunks = (1 << kTcM) / 2;        // 16-byte chunks of a tile
constexpr int kLoadIters = (kTileChunks + kLoadThreads - 1) / kLoadThreads;  // per loader thread (the last partly)
constexpr int kEpiRowPitch = 34;                    // float2 per row of the epilogue buffer (16-byte rows, turned banks)
constexpr uint32_t kEpiBufBytes = 16 * kEpiRowPitch * 8;  // 16 rows (amplitudes) of one epilogue warp
constexpr size_t kPipeSmem =
    size_t(kPipeBBufs) * 2 * kBBytes + size_t(kPipeStages) * kStageBytes + size_t(kEpiWarps) * kEpiBufBytes;
static_assert(kTcN == 64, "the pipelined epilogue reads 64 accumulator columns");
static_assert(kConvThreads % kTcN == 0, "fixed B row per converter thread");

// try_wait with a suspend-time hint: the thread sleeps until the phase
// completes or about 20 us pass (no spinning that would take issue slots
// from the working warps), then checks the abort flag and its own limit.
__device__ __forceinline__ bool pipe_wait(uint32_t addr, uint32_t parity, long long timeout_ns, volatile int *abort) {
    const uint64_t t0 = globaltimer();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity), "r"(20000u)
            : "memory");
        if (done) return true;
        if (*abort) return false;
        if (globaltimer() - t0 > uint64_t(timeout_ns)) {
            *abort = 1;
            return false;
        }
    }
}

// Position (in amplitudes) of tile index j in a slot filled by tensor-map
// copies with the 128-byte swizzle: the 16-byte chunk (j bits 1..3) is
// XORed with the 128-byte row modulo 8 (j bits 4..6).  XOR-linear in j.
__host__ __device__ constexpr uint32_t tma_pos(uint32_t j) { return j ^ (((j >> 4) & 7u) << 1); }

// one box of the tensor map at coordinates c into shared memory, counted in
// bytes on the mbarrier
__device__ __forceinline__ void tma_load5(uint32_t dst, const CUtensorMap *map, const int32_t (&c)[5], uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(addr), "r"(bytes)
                 : "memory");
}

// A wait every lane of a warp leaves with the same answer (lane 0 polls):
// the roles that follow use warp-wide (.aligned, shuffle) instructions.
__device__ __forceinline__ bool pipe_wait_warp(uint32_t addr, uint32_t parity, long long timeout_ns,
                                               volatile int *abort, int lane) {
    uint32_t ok = 0;
    if (lane == 0) ok = pipe_wait(addr, parity, timeout_ns, abort) ? 1u : 0u;
    return __shfl_sync(0xffffffffu, ok, 0) != 0u;
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(addr) : "memory");
}
// the barrier counts this thread once all its earlier cp.async have landed
__device__ __forceinline__ void mbar_arrive_on_copies(uint32_t addr) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(addr) : "memory");
}

// 64 consecutive 32-bit columns of this warp's 32 lanes (two loads and the
// wait in one statement: no use of the registers can move above the wait)
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float *v) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%64];\n"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,"
        "%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%65];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
          "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
          "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
          "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
          "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr), "r"(taddr + 32u)
        : "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kPipeThreads, 1) k_fused_tc(float2 *__restrict__ psi, const uint4 *__restrict__ gA,
                                                              int *__restrict__ err, const TcArgs a,
                                                              const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char smem[];
    // mbarriers: full[s], sfree[s] (slots), bfull[b], bempty[b] (B operands),
    // afull[c], aempty[c] (accumulators)
    __shared__ __align__(8) uint64_t mbar[2 * kPipeStages + 8];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ uint16_t tN[kTcN], tK[64];                  // staging positions of n and of K pairs
    __shared__ uint64_t gN[kTcN];                          // global offset of column n
    __shared__ uint64_t tB[4][256];                        // global offset of each byte of the tile number
    __shared__ uint64_t gCL[64], gCH[kTileChunks / 64];    // global offset of chunk bits 0..5 and 6..10
    __shared__ uint16_t sCL[64], sCH[kTileChunks / 64];    // staging chunk of the same
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *sB = smem;                                         // kPipeBBufs x (hi, lo)
    unsigned char *sSlots = smem + size_t(kPipeBBufs) * 2 * kBBytes;  // kPipeStages staging tiles
    unsigned char *sEpi = sSlots + size_t(kPipeStages) * kStageBytes;  // one buffer per epilogue warp
    const uint32_t bar0 = smem_u32(&mbar[0]);
    auto full = [&](int s) { return bar0 + 8u * uint32_t(s); };
    auto sfree = [&](int s) { return bar0 + 8u * uint32_t(kPipeStages + s); };
    auto bfull = [&](int b) { return bar0 + 8u * uint32_t(2 * kPipeStages + b); };
    auto bempty = [&](int b) { return bar0 + 8u * uint32_t(2 * kPipeStages + 2 + b); };
    auto afull = [&](int c) { return bar0 + 8u * uint32_t(2 * kPipeStages + 4 + c); };
    auto aempty = [&](int c) { return bar0 + 8u * uint32_t(2 * kPipeStages + 6 + c); };
    volatile int *abort_p = &abort_flag;

    // global offset of a tile index (its bit q is state qubit tile_pos[q])
    auto gofs = [&](uint32_t j) {
        uint64_t g = 0;
        for (int q = 0; q < kTcM; ++q)
            if (j >> q & 1) g |= uint64_t(1) << a.tile_pos[q];
        return g;
    };
    for (int i = tid; i < 64; i += kPipeThreads) {
        tN[i] = uint16_t(a.tma ? tma_pos(a.offN[i]) : sxpos(a.offN[i]));
        gN[i] = gofs(a.offN[i]);
        const int kk = 2 * i, klg = a.k + 1, rm = (2 << a.k) - 1;  // K elements 2i, 2i + 1
        const uint32_t jk = uint32_t(a.offL[(kk & rm) >> 1] ^ a.offP[kk >> klg]);
        tK[i] = uint16_t(a.tma ? tma_pos(jk) : sxpos(jk));
        gCL[i] = gofs(uint32_t(i) << 1);  // chunk c: amplitudes 2c, 2c + 1
        sCL[i] = uint16_t(swz(uint32_t(i)));
        if (i < kTileChunks / 64) {
            gCH[i] = gofs(uint32_t(i) << 7);
            sCH[i] = uint16_t(swz(uint32_t(i) << 6));
        }
    }
    for (int i = tid; i < 4 * 256; i += kPipeThreads) {  // the tile number's outer bits (tile numbers < 2^32)
        const int byte = i >> 8, v = i & 255;
        uint64_t off = 0;
        for (int b = 0; b < 8; ++b) {
            const int q = 8 * byte + b;
            if ((v >> b & 1) && q < a.nouter) off |= uint64_t(1) << a.outer_pos[q];
        }
        tB[byte][v] = off;
    }
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < kPipeStages; ++s) {
            mbar_init(full(s), a.tma ? 1u : uint32_t(kLoadThreads));
            mbar_init(sfree(s), kConvThreads);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bfull(b), kConvThreads);
            mbar_init(bempty(b), 1);
            mbar_init(afull(b), 1);
            mbar_init(aempty(b), 32 * kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // A operands into tensor memory once: warp w < 8 writes lanes
    // 32 (w % 4) .. +31 of A_hi (w < 4) or A_lo (w >= 4)
    if (warp < 8) {
        const int q = warp & 3, h = warp >> 2, m = 32 * q + lane;
        uint32_t r[64];
        const uint4 *src = gA + (size_t(h) * 128 * 128 * 2 + size_t(m) * 256) / 16;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const uint4 v = src[i];
            r[4 * i] = v.x;
            r[4 * i + 1] = v.y;
            r[4 * i + 2] = v.z;
            r[4 * i + 3] = v.w;
        }
        tmem_st64(tmem_slot + (uint32_t(32 * q) << 16) + uint32_t(kTcACols * h), r);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

    const uint64_t grid = gridDim.x;
    const uint64_t count = (a.ntiles - blockIdx.x + grid - 1) / grid;  // tiles of this CTA (blockIdx.x < ntiles)
    const long long tmo = a.timeout_ns;
    auto tile_base = [&](uint64_t i) {
        const uint64_t tile = blockIdx.x + i * grid;
        return tB[0][tile & 255] | tB[1][(tile >> 8) & 255] | tB[2][(tile >> 16) & 255] | tB[3][(tile >> 24) & 255];
    };

    if (warp < kConvWarps) {
        // ---------------- converters: staging tile -> B operand (BF16 hi, lo)
        const int lt = tid;
        const uint32_t sn = tN[lt & (kTcN - 1)];  // a thread's B row is the same in all its tasks
        for (uint64_t i = 0; i < count; ++i) {
            const int s = int(i % kPipeStages), b = int(i & 1);
            if (!pipe_wait_warp(full(s), uint32_t(i / kPipeStages) & 1u, tmo, abort_p, lane)) break;
            if (i >= 2 && !pipe_wait_warp(bempty(b), uint32_t((i >> 1) - 1) & 1u, tmo, abort_p, lane)) break;
            const float2 *sX = reinterpret_cast<const float2 *>(sSlots + size_t(s) * kStageBytes);
            unsigned char *bh = sB + size_t(b) * 2 * kBBytes, *bl = bh + kBBytes;
#pragma unroll
            for (int t = lt; t < 16 * kTcN; t += kConvThreads) {
                const int nrow = t & (kTcN - 1), q8 = t / kTcN;
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {  // K elements 8 q8 + 2e, +1: re and im of one amplitude
                    const float2 amp = sX[sn ^ tK[q8 * 4 + e]];
                    const __nv_bfloat162 hi = __float22bfloat162_rn(amp);
                    const float2 hf = __bfloat1622float2(hi);
                    const __nv_bfloat162 lo = __float22bfloat162_rn(make_float2(amp.x - hf.x, amp.y - hf.y));
                    hw[e] = *reinterpret_cast<const uint32_t *>(&hi);
                    lw[e] = *reinterpret_cast<const uint32_t *>(&lo);
                }
                const uint32_t off = uint32_t((nrow & 7) * 16 + q8 * 128 + (nrow >> 3) * 2048);
                *reinterpret_cast<uint4 *>(bh + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4 *>(bl + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic writes -> tensor core reads
            mbar_arrive(bfull(b));
            mbar_arrive(sfree(s));
        }
    } else if (warp < kLoadWarp0) {
        // ---------------- epilogue: accumulator -> HBM
        const int eq = warp & 3;  // tensor-memory lanes 32 eq .. +31 (warp % 4)
        const int row = 32 * eq + lane;
        const int klog = a.k + 1, rmask = (2 << a.k) - 1;
        const uint64_t grow = gofs(uint32_t(a.offL[(row & rmask) >> 1] ^ a.offP[row >> klog]));
        const int odd = row & 1;  // odd rows hold Im, even rows Re (of the same amplitude as row ^ 1)
        const int mode = a.epi_mode;
        for (uint64_t i = 0; i < count; ++i) {
            const int c = int(i & 1);
            if (!pipe_wait_warp(afull(c), uint32_t(i >> 1) & 1u, tmo, abort_p, lane)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            float v[64];
            tmem_ld64(tmem_slot + (uint32_t(32 * eq) << 16) + uint32_t(2 * kTcACols + c * kTcN), v);
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            mbar_arrive(aempty(c));
            const uint64_t tb = tile_base(i);
            if (mode == 0) {
                // two rounds of half the columns: the even lane of a pair takes
                // columns 16h + t, the odd lane 32 + 16h + (t ^ 1) (turned: the
                // pair's two 8-byte writes fall in different banks); buffer row
                // r = lane / 2 (the warp's 16 amplitudes), slots 0..15 even, 16..31 odd
                float2 *buf = reinterpret_cast<float2 *>(sEpi + size_t(eq) * kEpiBufBytes);
                const int r = lane >> 1;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        const int ce = 16 * h + t, co = 32 + 16 * h + (t ^ 1);
                        const float got = __shfl_xor_sync(0xffffffffu, odd ? v[ce] : v[co], 1);
                        if (odd)
                            buf[r * kEpiRowPitch + 16 + (t ^ 1)] = make_float2(got, v[co]);
                        else
                            buf[r * kEpiRowPitch + t] = make_float2(v[ce], got);
                    }
                    __syncwarp();
                    // store: lanes 0..15 row 2 ii, lanes 16..31 row 2 ii + 1; lane
                    // L & 15 takes slots 2u, 2u + 1 (u = L & 7), even part for L & 8 = 0
#pragma unroll
                    for (int ii = 0; ii < 8; ++ii) {
                        const int rr = 2 * ii + (lane >> 4), u = lane & 15;
                        const uint64_t gr = __shfl_sync(0xffffffffu, grow, 2 * rr);
                        const float4 val = *reinterpret_cast<const float4 *>(buf + rr * kEpiRowPitch + 2 * u);
                        const int col = (u < 8 ? 16 * h : 32 + 16 * h - 16) + 2 * u;
                        *reinterpret_cast<float4 *>(psi + (tb | gr | gN[col])) = val;
                    }
                    __syncwarp();
                }
            } else {
                float2 *g = psi + (tb | grow);
                const int c0 = odd ? 32 : 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float got = __shfl_xor_sync(0xffffffffu, odd ? v[j] : v[32 + j], 1);
                    g[gN[c0 + j]] = odd ? make_float2(got, v[32 + j]) : make_float2(v[j], got);
                }
            }
        }
    } else if (warp < kMmaWarp) {
        // ---------------- loaders: HBM -> staging tiles
        const int lt = tid - 32 * kLoadWarp0;
        if (a.tma) {
            // one thread: a.tma_nbox tensor-map boxes per tile (each of the
            // map's dimensions holds a range of qubits: the box's coordinate
            // is that range of the box's global offset)
            if (lt == 0) {
                uint64_t issued[kPipeStages] = {0, 0, 0, 0};
                const uint32_t box_bytes = kStageBytes / a.tma_nbox;
                for (uint64_t i = 0; i < count; ++i) {
                    const int s = int(i % kPipeStages);
                    if (i >= kPipeStages && !pipe_wait(sfree(s), uint32_t(i / kPipeStages - 1) & 1u, tmo, abort_p)) break;
                    mbar_expect_tx(full(s), kStageBytes);
                    const uint32_t dst = smem_u32(sSlots + size_t(s) * kStageBytes);
                    const uint64_t tb = tile_base(i);
                    for (int b = 0; b < a.tma_nbox; ++b) {
                        const uint64_t g = tb | a.tma_boff[b];
                        int32_t c[5];
#pragma unroll
                        for (int d = 0; d < 5; ++d) {
                            const int lo = a.tma_start[d], hi = d + 1 < a.tma_rank ? a.tma_start[d + 1] : a.n;
                            c[d] = d < a.tma_rank ? int32_t((g >> lo) & ((uint64_t(1) << (hi - lo)) - 1u)) : 0;
                        }
                        tma_load5(dst + uint32_t(b) * box_bytes, &tmap, c, full(s));
                    }
                    ++issued[s];
                }
                if (*abort_p)  // copies still in flight land before the CTA leaves
                    for (int s = 0; s < kPipeStages; ++s)
                        if (issued[s]) {
                            const uint64_t t0 = globaltimer();
                            uint32_t done = 0;
                            while (!done && globaltimer() - t0 < uint64_t(tmo)) {
                                asm volatile(
                                    "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 "
                                    "%0, 1, 0, p;\n}\n"
                                    : "=r"(done)
                                    : "r"(full(s)), "r"(uint32_t(issued[s] - 1) & 1u)
                                    : "memory");
                            }
                        }
            }
        } else {
            // 16-byte cp.async: chunk c = lt + kLoadThreads r of a tile
            // (amplitudes 2c, 2c + 1); a warp's 32 chunks are 512 contiguous
            // bytes (tile bits 0..5 are state qubits 0..5, and 32 divides
            // kLoadThreads)
            for (uint64_t i = 0; i < count; ++i) {
                const int s = int(i % kPipeStages);
                if (i >= kPipeStages &&
                    !pipe_wait_warp(sfree(s), uint32_t(i / kPipeStages - 1) & 1u, tmo, abort_p, lane))
                    break;
                float2 *sX = reinterpret_cast<float2 *>(sSlots + size_t(s) * kStageBytes);
                const float2 *g = psi + tile_base(i);
#pragma unroll
                for (int r = 0; r < kLoadIters; ++r) {
                    const int c = lt + kLoadThreads * r;
                    if (c < kTileChunks)
                        cp_async16(smem_u32(sX + 2 * (sCL[c & 63] ^ sCH[c >> 6])), g + (gCL[c & 63] | gCH[c >> 6]));
                }
                mbar_arrive_on_copies(full(s));
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");  // no copy still writing when the CTA leaves
        }
    } else if (lane == 0) {
        // ---------------- MMA issue
        const uint32_t tA = tmem_slot;
        for (uint64_t i = 0; i < count; ++i) {
            const int b = int(i & 1), c = int(i & 1);
            if (!pipe_wait(bfull(b), uint32_t(i >> 1) & 1u, tmo, abort_p)) break;
            if (i >= 2 && !pipe_wait(aempty(c), uint32_t((i >> 1) - 1) & 1u, tmo, abort_p)) break;
            if (a.skip_mma) continue;  // test hook: no MMA, no commit (the epilogue's wait runs out)
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t bh = smem_u32(sB + size_t(b) * 2 * kBBytes), bl = bh + kBBytes;
            const uint32_t tD = tA + uint32_t(2 * kTcACols + c * kTcN);
            uint32_t acc = 0;
#pragma unroll
            for (int pass = 0; pass < 3; ++pass) {
                const uint32_t aa = tA + uint32_t(pass == 2 ? kTcACols : 0), bb = pass == 1 ? bl : bh;
#pragma unroll
                for (int ks = 0; ks < 8; ++ks) {
                    mma_bf16_ts(tD, aa + 8u * ks, sdesc(bb + 256u * ks, 128, 2048), acc);
                    acc = 1;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bempty(b))
                         : "memory");
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(afull(c))
                         : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && abort_flag) atomicExch(err, int(SV_ERR_TIMEOUT));
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_slot), "r"(kTcCols)
                     : "memory");
    }
}

uint16_t bf16_rne_host(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return uint16_t(u >> 16);
}

float bf16_to_float_host(uint16_t h) {
    const uint32_t u = uint32_t(h) << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

}  // namespace

bool fused_tc_supported(const sv_state *h) { return h->dt == SV_C64 && h->n >= kTcM; }

void tc_prepare(int n, int k, const int *qubits, const double *U, uint16_t *a_ops, TcArgs *args) {
    const int d = 1 << k, twoD = 2 * d, P = 64 / d;
    // A = I_P (x) Ut, split into BF16 hi / lo, row-major (one row per tensor-memory lane)
    for (int i = 0; i < 2 * 128 * 128; ++i) a_ops[i] = 0;
    for (int m = 0; m < 128; ++m)
        for (int kk = 0; kk < 128; ++kk) {
            double v = 0.0;
            if (m / twoD == kk / twoD) {
                const int rr = (m % twoD) >> 1, ar = m & 1, cc = (kk % twoD) >> 1, bc = kk & 1;
                const double ure = U[2 * (rr * d + cc)], uim = U[2 * (rr * d + cc) + 1];
                v = (ar == bc) ? ure : (ar == 0 ? -uim : uim);
            }
            const uint16_t hi = bf16_rne_host(float(v));
            const uint16_t lo = bf16_rne_host(float(v - double(bf16_to_float_host(hi))));
            const size_t off = size_t(m) * 128 + size_t(kk);  // row-major (tensor-memory rows)
            a_ops[off] = hi;
            a_ops[128 * 128 + off] = lo;
        }
    TcArgs &a = *args;
    a = TcArgs{};
    a.n = n;
    a.k = k;
    a.P = P;
    // tile qubits: the block qubits plus the lowest other qubits
    uint64_t T = 0;
    for (int j = 0; j < k; ++j) T |= uint64_t(1) << qubits[j];
    for (int q = 0; q < n && __builtin_popcountll(T) < kTcM; ++q) T |= uint64_t(1) << q;
    int tpos_of[64];
    int t = 0, o = 0;
    for (int q = 0; q < n; ++q) {
        if (T >> q & 1) {
            tpos_of[q] = t;
            a.tile_pos[t++] = uint8_t(q);
        } else {
            tpos_of[q] = -1;
            a.outer_pos[o++] = uint8_t(q);
        }
    }
    a.nouter = o;
    int lc = 0;
    while (lc < kTcM && a.tile_pos[lc] == lc) ++lc;
    a.lc = lc;
    for (int l = 0; l < d; ++l) {
        uint32_t off = 0;
        for (int j = 0; j < k; ++j)
            if (l >> j & 1) off |= 1u << tpos_of[qubits[j]];
        a.offL[l] = uint16_t(off);
    }
    // group bits: the non-block tile bits ascending; the low log2(P) of them are the pack index
    int gbits[kTcM], ng = 0;
    for (int tb = 0; tb < kTcM; ++tb) {
        bool blk = false;
        for (int j = 0; j < k; ++j) blk |= tpos_of[qubits[j]] == tb;
        if (!blk) gbits[ng++] = tb;
    }
    const int plog = 6 - k;
    for (int p = 0; p < P; ++p) {
        uint32_t off = 0;
        for (int i = 0; i < plog; ++i)
            if (p >> i & 1) off |= 1u << gbits[i];
        a.offP[p] = uint16_t(off);
    }
    for (int nn = 0; nn < kTcN; ++nn) {  // the remaining kTcM - 6 group bits
        uint32_t off = 0;
        for (int i = 0; i < kTcM - 6; ++i)
            if (nn >> i & 1) off |= 1u << gbits[plog + i];
        a.offN[nn] = uint16_t(off);
    }
    a.ntiles = uint64_t(1) << (n - kTcM);
    a.timeout_ns = 2000000000LL;
    // kernel and epilogue form: tile bits 0..3 are state qubits 0..3, so
    // "columns 0..3 are qubits 0..1" means offN[c] = c, and "each epilogue
    // warp's 16 rows are qubits 0..3" means the row amplitudes' tile bits
    // 0..3 count 0..15; with neither, the two-group kernel (epi_mode 2).
    // (Columns 0..7 along qubits 0..2 was the first rule; 0..3 moved three
    // of the 64 blocks of the 32-qubit benchmark's fused plan off the
    // two-group kernel, 270 against about 275 us per 26-qubit launch.)
    bool cols = true, rows = true;
    for (int c = 0; c < 4; ++c) cols = cols && a.offN[c] == c;
    for (int w = 0; w < 4 && rows; ++w)
        for (int r = 0; r < 16; ++r) {
            const int row = 32 * w + 2 * r;
            const uint32_t j = uint32_t(a.offL[(row & (2 * d - 1)) >> 1] ^ a.offP[row >> (k + 1)]);
            rows = rows && (j & 15u) == uint32_t(r);
        }
    a.epi_mode = uint8_t(cols ? 0 : (rows ? 1 : 2));
    // form 0 loads with tensor-map copies: runs of consecutive tile qubits
    // (run 0 starts at qubit 0 and is at least 6 long); the map's dimensions
    // are qubits 0..3 (128 bytes, the 128-byte swizzle's row), the rest of
    // run 0, then one per later run, each reaching up to the next; runs
    // beyond five dimensions (the top ones) are iterated as separate boxes
    if (a.epi_mode == 0) {
        int rs[kTcM], rl[kTcM], nr = 0;
        for (int t = 0; t < kTcM; ++t) {
            if (t > 0 && a.tile_pos[t] == a.tile_pos[t - 1] + 1) {
                ++rl[nr - 1];
            } else {
                rs[nr] = a.tile_pos[t];
                rl[nr++] = 1;
            }
        }
        const int boxed = std::min(nr, 4);  // runs 0 .. boxed-1 in the box (run 0 takes two dimensions)
        int it_bits = 0;
        for (int r = boxed; r < nr; ++r) it_bits += rl[r];
        if (rs[0] == 0 && rl[0] >= 6 && it_bits <= 2) {
            a.tma = 1;
            a.tma_rank = uint8_t(boxed + 1);
            a.tma_start[0] = 0;
            a.tma_start[1] = 4;
            for (int r = 1; r < boxed; ++r) a.tma_start[r + 1] = uint8_t(rs[r]);
            a.tma_nbox = uint8_t(1 << it_bits);
            for (int b = 0; b < a.tma_nbox; ++b) {  // the iterated runs' qubits, ascending, from b's bits
                uint64_t off = 0;
                int bit = 0;
                for (int r = boxed; r < nr; ++r)
                    for (int q = rs[r]; q < rs[r] + rl[r]; ++q, ++bit)
                        if (b >> bit & 1) off |= uint64_t(1) << q;
                a.tma_boff[b] = off;
            }
        }
    }
}

// cuTensorMapEncodeTiled, looked up once through the runtime (the library
// links only the static runtime); nullptr if the driver does not offer it.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn() {
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// The state as a tensor of 8-byte elements whose dimensions are the ranges of
// qubits TcArgs::tma_start sets out (sizes 2^range, strides the products of
// the ones below: the plain layout), padded to five dimensions of size 1; the
// box covers the tile's part of each range; 128-byte swizzle.
void tile_map_dims(int n, const TcArgs &a, uint64_t dim[5], uint64_t stride[4], uint32_t box[5]) {
    uint64_t bytes = 8;  // stride of the current dimension
    for (int d = 0; d < 5; ++d) {
        if (d < a.tma_rank) {
            const int lo = a.tma_start[d], hi = d + 1 < a.tma_rank ? a.tma_start[d + 1] : n;
            dim[d] = uint64_t(1) << (hi - lo);
            int in_tile = 0;  // tile qubits in [lo, hi): qubits 0..3, the rest of run 0, or a run (and iterated ones)
            for (int t = 0; t < kTcM; ++t) in_tile += a.tile_pos[t] >= lo && a.tile_pos[t] < hi;
            box[d] = uint32_t(1) << in_tile;
        } else {
            dim[d] = 1;
            box[d] = 1;
        }
        if (d > 0) stride[d - 1] = bytes;
        bytes *= dim[d];
    }
    // iterated runs lie inside the last range but outside the box
    int it = 0;
    for (int b = a.tma_nbox; b > 1; b >>= 1) ++it;
    box[a.tma_rank - 1] >>= it;
}

cudaError_t encode_tile_map(void *data, int n, const TcArgs &a, CUtensorMap *map) {
    const EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return cudaErrorNotSupported;
    uint64_t dim[5], stride[4];
    uint32_t box[5];
    tile_map_dims(n, a, dim, stride, box);
    cuuint64_t cdim[5], cstride[4];
    cuuint32_t cbox[5], estr[5] = {1, 1, 1, 1, 1};
    for (int d = 0; d < 5; ++d) {
        cdim[d] = dim[d];
        cbox[d] = box[d];
        if (d < 4) cstride[d] = stride[d];
    }
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, data, cdim, cstride, cbox, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", int(r));
        return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t tc_launch(sv_state *h, const TcArgs &args, const void *dA) {
    TcArgs a = args;
    if (fault_injected("tc_wait")) {  // test hook: the MMA wait runs out
        a.skip_mma = 1;
        a.timeout_ns = 1000000LL;
    }
    {
        const cudaError_t e = ensure_err_word(h);
        if (e != cudaSuccess) return e;
    }
    const size_t smem_groups = kTcGroups * (2 * size_t(kBBytes) + kTcRing * size_t(kStageBytes));
    static std::atomic<uint64_t> configured{0};
    if (attrs_needed(configured, h->device)) {
        cudaError_t e = cudaFuncSetAttribute(k_fused_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kPipeSmem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fused_tc_groups, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(smem_groups));
        if (e != cudaSuccess) return e;
        attrs_set(configured, h->device);
    }
    int sms = 0;
    const cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return e;
    if (a.epi_mode <= 1) {  // the pipeline: columns or rows run along the low qubits
        CUtensorMap map;
        std::memset(&map, 0, sizeof(map));
        if (a.tma) {
            const cudaError_t me = encode_tile_map(h->data, h->n, a, &map);
            if (me != cudaSuccess) return me;
        }
        const uint64_t grid = a.ntiles < uint64_t(sms) ? a.ntiles : uint64_t(sms);
        k_fused_tc<<<unsigned(grid), kPipeThreads, kPipeSmem, h->stream>>>(
            static_cast<float2 *>(h->data), static_cast<const uint4 *>(dA), h->d_err, a, map);
    } else {
        const uint64_t sets = (a.ntiles + kTcGroups - 1) / kTcGroups;  // kTcGroups tiles in flight per CTA
        const uint64_t grid = sets < uint64_t(sms) ? sets : uint64_t(sms);
        k_fused_tc_groups<<<unsigned(grid), kTcThreads, smem_groups, h->stream>>>(
            static_cast<float2 *>(h->data), static_cast<const uint4 *>(dA), h->d_err, a);
    }
    return cudaGetLastError();
}

const char *tc_kernel_name(const TcArgs &a) {
    static const char *names[3][7] = {
        {"k_fused_tc<k=0>", "k_fused_tc<k=1>", "k_fused_tc<k=2>", "k_fused_tc<k=3>", "k_fused_tc<k=4>",
         "k_fused_tc<k=5>", "k_fused_tc<k=6>"},
        {"k_fused_tc<k=0,tma>", "k_fused_tc<k=1,tma>", "k_fused_tc<k=2,tma>", "k_fused_tc<k=3,tma>",
         "k_fused_tc<k=4,tma>", "k_fused_tc<k=5,tma>", "k_fused_tc<k=6,tma>"},
        {"k_fused_tc_groups<k=0>", "k_fused_tc_groups<k=1>", "k_fused_tc_groups<k=2>", "k_fused_tc_groups<k=3>",
         "k_fused_tc_groups<k=4>", "k_fused_tc_groups<k=5>", "k_fused_tc_groups<k=6>"}};
    const int form = a.epi_mode > 1 ? 2 : (a.tma ? 1 : 0);
    return names[form][a.k < 0 || a.k > 6 ? 0 : a.k];
}

cudaError_t launch_fused_tc(sv_state *h, int k, const int *qubits, const double *U) {
    static thread_local std::vector<uint16_t> host;
    host.resize(2 * 128 * 128);
    TcArgs a;
    tc_prepare(h->n, k, qubits, U, host.data(), &a);
    if (!h->d_mat) {
        const cudaError_t e = cudaMalloc(&h->d_mat, kTcOperandBytes);
        if (e != cudaSuccess) return e;
    }
    const cudaError_t e = cudaMemcpyAsync(h->d_mat, host.data(), kTcOperandBytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return e;
    return tc_launch(h, a, h->d_mat);
}

}  // namespace sv

using namespace sv;

extern "C" sv_status sv_fused_tc_layout(int n, int k, const int *qubits, char *kernel, size_t cap, int *tile_pos,
                                        int *tma_rank, int *tma_nbox, int *tma_start, uint64_t *tma_boff,
                                        uint64_t *dim, uint64_t *stride, uint32_t *box) {
    if (n < kTcM || n > kMaxQubits || k < 1 || k > 6 || !qubits) {
        set_error("need 12 <= n <= %d, 1 <= k <= 6 and the block's qubits", kMaxQubits);
        return SV_ERR_ARG;
    }
    for (int j = 0; j < k; ++j) {
        bool dup = false;
        for (int i = 0; i < j; ++i) dup = dup || qubits[i] == qubits[j];
        if (qubits[j] < 0 || qubits[j] >= n || dup) {
            set_error("block qubits must be distinct and in [0, n)");
            return SV_ERR_ARG;
        }
    }
    std::vector<double> U(size_t(2) << (2 * k), 0.0);
    for (int i = 0; i < (1 << k); ++i) U[size_t(2) * (size_t(i) * (size_t(1) << k) + size_t(i))] = 1.0;
    std::vector<uint16_t> img(2 * 128 * 128);
    TcArgs a;
    tc_prepare(n, k, qubits, U.data(), img.data(), &a);
    const char *nm = tc_kernel_name(a);
    if (kernel && cap) {
        std::strncpy(kernel, nm, cap - 1);
        kernel[cap - 1] = '\0';
    }
    if (tile_pos)
        for (int t = 0; t < kTcM; ++t) tile_pos[t] = a.tile_pos[t];
    if (tma_rank) *tma_rank = a.tma ? a.tma_rank : 0;
    if (tma_nbox) *tma_nbox = a.tma ? a.tma_nbox : 0;
    uint64_t d5[5] = {0, 0, 0, 0, 0}, s4[4] = {0, 0, 0, 0};
    uint32_t b5[5] = {0, 0, 0, 0, 0};
    if (a.tma) tile_map_dims(n, a, d5, s4, b5);
    for (int d = 0; d < 5; ++d) {
        if (tma_start) tma_start[d] = a.tma && d < a.tma_rank ? a.tma_start[d] : 0;
        if (dim) dim[d] = d5[d];
        if (box) box[d] = b5[d];
        if (stride && d < 4) stride[d] = s4[d];
        if (tma_boff && d < 4) tma_boff[d] = a.tma && d < a.tma_nbox ? a.tma_boff[d] : 0;
    }
    return SV_OK;
}
