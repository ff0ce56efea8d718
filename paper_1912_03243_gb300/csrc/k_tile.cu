// Tiled multi-gate pass (one HBM read + write of the state for many gates).
//
// CTA = one tile of 2^M amplitudes (runs of 2^lc contiguous amplitudes at
// the offsets given by the tile's high qubits).  Phases:
//   1. cp.async 16-byte copies of the runs into shared memory (XOR-swizzled
//      by 16-byte chunk, so register gathers of any bit pattern spread over
//      the banks).
//   2. For each segment: every thread gathers its 2^RB amplitudes (the
//      segment's register qubits) from shared memory, applies the segment's
//      ops in registers, and scatters them back.  Ops are read from global
//      memory (the same address for every thread: a broadcast).
//   3. Copy the tile back to HBM.
// Ops: general 2x2 gates (Eq. 1), structured gates whose entries are
// 0, +-1, +-i (H, SX, SY, X and adjoints: additions only, the scalar factor
// deferred to one multiply per pass), phases and sign flips of diagonal
// gates (T, CZ, CP) with conditions on register, thread and CTA index bits.
#include "tile.h"

namespace sv {
namespace {

template <typename R>
struct CT {
    R re, im;
};

// 16-byte-chunk swizzle: chunk c is stored at chunk c ^ f(c), f folding the
// chunk bits above 3 onto bits 0..2.  Linear over XOR.
__device__ __forceinline__ uint32_t swz(uint32_t c) { return c ^ (((c >> 3) ^ (c >> 6) ^ (c >> 9)) & 7u); }

template <typename R>
__device__ __forceinline__ uint32_t phys(uint32_t j) {
    if constexpr (sizeof(CT<R>) == 8) return (swz(j >> 1) << 1) | (j & 1u);
    else return swz(j);
}

__device__ __forceinline__ void cp_async16(void *smem_ptr, const void *gptr) {
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem_ptr));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gptr) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <typename R>
__device__ __forceinline__ void apply2(const R *u, CT<R> &a, CT<R> &b) {
    const R ar = a.re, ai = a.im, br = b.re, bi = b.im;
    a.re = u[0] * ar - u[1] * ai + u[2] * br - u[3] * bi;
    a.im = u[0] * ai + u[1] * ar + u[2] * bi + u[3] * br;
    b.re = u[4] * ar - u[5] * ai + u[6] * br - u[7] * bi;
    b.im = u[4] * ai + u[5] * ar + u[6] * bi + u[7] * br;
}

template <int S, bool CTL, typename R, int NR>
__device__ __forceinline__ void op_g1(CT<R> *x, const R *u, uint32_t rmask, uint32_t rval) {
#pragma unroll
    for (int v = 0; v < NR; ++v) {
        if (v & (1 << S)) continue;
        if (CTL && (uint32_t(v) & rmask) != rval) continue;
        apply2(u, x[v], x[v | (1 << S)]);
    }
}

template <int K, typename R>
__device__ __forceinline__ void struct2(CT<R> &a, CT<R> &b) {
    const R ar = a.re, ai = a.im, br = b.re, bi = b.im;
    if constexpr (K == SK_H) {
        a = {ar + br, ai + bi};
        b = {ar - br, ai - bi};
    } else if constexpr (K == SK_SX) {  // (a - i b, -i a + b)
        a = {ar + bi, ai - br};
        b = {br + ai, bi - ar};
    } else if constexpr (K == SK_SXD) {  // (a + i b, i a + b)
        a = {ar - bi, ai + br};
        b = {br - ai, bi + ar};
    } else if constexpr (K == SK_SY) {  // (a - b, a + b)
        a = {ar - br, ai - bi};
        b = {ar + br, ai + bi};
    } else if constexpr (K == SK_SYD) {  // (a + b, b - a)
        a = {ar + br, ai + bi};
        b = {br - ar, bi - ai};
    } else {  // X
        a = {br, bi};
        b = {ar, ai};
    }
}

template <int S, int K, bool CTL, typename R, int NR>
__device__ __forceinline__ void op_struct(CT<R> *x, uint32_t rmask, uint32_t rval) {
#pragma unroll
    for (int v = 0; v < NR; ++v) {
        if (v & (1 << S)) continue;
        if (CTL && (uint32_t(v) & rmask) != rval) continue;
        struct2<K>(x[v], x[v | (1 << S)]);
    }
}

template <int M, int V, bool NEG, typename R, int NR>
__device__ __forceinline__ void op_phase(CT<R> *x, R pr, R pi) {
#pragma unroll
    for (int v = 0; v < NR; ++v) {
        if ((v & M) != V) continue;
        if (NEG) {
            x[v].re = -x[v].re;
            x[v].im = -x[v].im;
        } else {
            const R r = x[v].re * pr - x[v].im * pi;
            x[v].im = x[v].re * pi + x[v].im * pr;
            x[v].re = r;
        }
    }
}

template <bool NEG, typename R, int NR>
__device__ __forceinline__ void phase_dispatch(int id, CT<R> *x, R pr, R pi) {
#define SV_PH(Mk, Vk)                                  \
    case (Mk) * 32 + (Vk):                             \
        op_phase<(Mk), (Vk), NEG, R, NR>(x, pr, pi); \
        break;
#define SV_PH1(A) SV_PH(A, 0) SV_PH(A, A)
#define SV_PH2(A, B) SV_PH((A) | (B), 0) SV_PH((A) | (B), A) SV_PH((A) | (B), B) SV_PH((A) | (B), (A) | (B))
    switch (id) {
        SV_PH(0, 0)
        SV_PH1(1) SV_PH1(2) SV_PH1(4) SV_PH1(8) SV_PH1(16)
        SV_PH2(1, 2) SV_PH2(1, 4) SV_PH2(1, 8) SV_PH2(1, 16) SV_PH2(2, 4)
        SV_PH2(2, 8) SV_PH2(2, 16) SV_PH2(4, 8) SV_PH2(4, 16) SV_PH2(8, 16)
        default: break;
    }
#undef SV_PH2
#undef SV_PH1
#undef SV_PH
}

template <bool CTL, typename R, int RB>
__device__ __forceinline__ void struct_dispatch(int a, CT<R> *x, uint32_t rmask, uint32_t rval) {
    constexpr int NR = 1 << RB;
#define SV_ST(S, K)                                                    \
    case (S) | ((K) << 8):                                             \
        if constexpr ((S) < RB) op_struct<(S), (K), CTL, R, NR>(x, rmask, rval); \
        break;
#define SV_STK(S) SV_ST(S, 0) SV_ST(S, 1) SV_ST(S, 2) SV_ST(S, 3) SV_ST(S, 4) SV_ST(S, 5)
    switch (a) {
        SV_STK(0) SV_STK(1) SV_STK(2) SV_STK(3) SV_STK(4)
        default: break;
    }
#undef SV_STK
#undef SV_ST
}

template <bool CTL, typename R, int RB>
__device__ __forceinline__ void g1_dispatch(int s, CT<R> *x, const R *u, uint32_t rmask, uint32_t rval) {
    constexpr int NR = 1 << RB;
    switch (s) {
        case 0: op_g1<0, CTL, R, NR>(x, u, rmask, rval); break;
        case 1: if constexpr (RB > 1) op_g1<1, CTL, R, NR>(x, u, rmask, rval); break;
        case 2: if constexpr (RB > 2) op_g1<2, CTL, R, NR>(x, u, rmask, rval); break;
        case 3: if constexpr (RB > 3) op_g1<3, CTL, R, NR>(x, u, rmask, rval); break;
        case 4: if constexpr (RB > 4) op_g1<4, CTL, R, NR>(x, u, rmask, rval); break;
        default: break;
    }
}

template <typename R, int M, int RB>
__global__ void __launch_bounds__(1 << (M - RB), 2)
    k_tile(CT<R> *__restrict__ psi, const TileOp<R> *__restrict__ ops, const TileSeg *__restrict__ segs,
           const TilePassArgs pa) {
    constexpr int NT = 1 << (M - RB);
    constexpr int NR = 1 << RB;
    constexpr int ELEMS = 1 << M;
    constexpr int EPC = 16 / int(sizeof(CT<R>));  // elements per 16-byte chunk
    constexpr int NCH = ELEMS / EPC;
    extern __shared__ __align__(16) unsigned char smem[];
    CT<R> *sm = reinterpret_cast<CT<R> *>(smem);
    uint64_t *run_off = reinterpret_cast<uint64_t *>(smem + size_t(ELEMS) * sizeof(CT<R>));
    const uint32_t tid = threadIdx.x;

    // global index bits of this CTA's outer qubits
    uint64_t base = 0;
    {
        const uint64_t b = blockIdx.x;
        for (int k = 0; k < pa.nouter; ++k) base |= ((b >> k) & 1ull) << pa.outer_pos[k];
    }
    const int lc = pa.lc;
    const int nruns = 1 << (M - lc);
    for (int r = int(tid); r < nruns; r += NT) {
        uint64_t o = 0;
        for (int k = 0; k < M - lc; ++k)
            if (r >> k & 1) o |= 1ull << pa.tile_pos[lc + k];
        run_off[r] = o;
    }
    __syncthreads();
    const uint32_t lmask = (1u << lc) - 1u;
#pragma unroll 4
    for (int c = int(tid); c < NCH; c += NT) {
        const uint32_t j = uint32_t(c) * EPC;
        const uint64_t g = base | run_off[j >> lc] | (j & lmask);
        cp_async16(smem + size_t(swz(uint32_t(c))) * 16, psi + g);
    }
    cp_async_wait_all();
    __syncthreads();

    CT<R> x[NR];
    uint32_t jt = 0, pjt = 0;
    uint32_t P[RB];
#pragma unroll
    for (int s = 0; s < RB; ++s) P[s] = 0;
    bool started = false;

    auto scatter = [&]() {
#pragma unroll
        for (int v = 0; v < NR; ++v) {
            uint32_t a = pjt;
#pragma unroll
            for (int s = 0; s < RB; ++s)
                if (v >> s & 1) a ^= P[s];
            sm[a] = x[v];
        }
    };
    auto gather = [&]() {
#pragma unroll
        for (int v = 0; v < NR; ++v) {
            uint32_t a = pjt;
#pragma unroll
            for (int s = 0; s < RB; ++s)
                if (v >> s & 1) a ^= P[s];
            x[v] = sm[a];
        }
    };

    for (int i = pa.op_begin; i < pa.op_end; ++i) {
        const TileOp<R> &op = ops[i];
        const int type = op.type;
        if (type == TOP_SEG) {
            if (started) {
                scatter();
                __syncthreads();
            }
            started = true;
            const TileSeg &sg = segs[op.a];
            jt = 0;
#pragma unroll
            for (int k = 0; k < M - RB; ++k) jt |= ((tid >> k) & 1u) << sg.tpos[k];
            pjt = phys<R>(jt);
#pragma unroll
            for (int s = 0; s < RB; ++s) P[s] = phys<R>(1u << sg.rpos[s]);
            gather();
            continue;
        }
        if (type == TOP_SCALE) {
            const R pr = op.u[0], pi = op.u[1];
#pragma unroll
            for (int v = 0; v < NR; ++v) {
                const R r = x[v].re * pr - x[v].im * pi;
                x[v].im = x[v].re * pi + x[v].im * pr;
                x[v].re = r;
            }
            continue;
        }
        const bool pred = ((jt & op.tmask) == op.tval) && ((base & op.gmask) == op.gval);
        if (!pred) continue;
        if (type == TOP_STRUCT) {
            if (op.rmask == 0) struct_dispatch<false, R, RB>(op.a, x, 0, 0);
            else struct_dispatch<true, R, RB>(op.a, x, op.rmask, op.rval);
        } else if (type == TOP_NEG) {
            phase_dispatch<true, R, NR>(op.a, x, R(0), R(0));
        } else if (type == TOP_PHASE) {
            phase_dispatch<false, R, NR>(op.a, x, op.u[0], op.u[1]);
        } else if (type == TOP_G1) {
            R u[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) u[k] = op.u[k];
            if (op.rmask == 0) g1_dispatch<false, R, RB>(op.a, x, u, 0, 0);
            else g1_dispatch<true, R, RB>(op.a, x, u, op.rmask, op.rval);
        }
    }
    if (started) {
        scatter();
        __syncthreads();
    }
#pragma unroll 4
    for (int c = int(tid); c < NCH; c += NT) {
        const uint32_t j = uint32_t(c) * EPC;
        const uint64_t g = base | run_off[j >> lc] | (j & lmask);
        const int4 v = *reinterpret_cast<const int4 *>(smem + size_t(swz(uint32_t(c))) * 16);
        *reinterpret_cast<int4 *>(psi + g) = v;
    }
}

template <typename R, int M, int RB, int LOW>
cudaError_t launch_impl(sv_state *h, const TilePassArgs &pa, const void *d_ops, const TileSeg *d_segs) {
    constexpr int ELEMS = 1 << M;
    // tile + run-offset table (2^(M - lc) entries, lc >= LOW)
    constexpr size_t kMaxSmem = size_t(ELEMS) * sizeof(CT<R>) + sizeof(uint64_t) * (size_t(1) << (M - LOW));
    if (pa.lc < LOW) return cudaErrorInvalidValue;
    const size_t smem = size_t(ELEMS) * sizeof(CT<R>) + sizeof(uint64_t) * (size_t(1) << (M - pa.lc));
    static bool configured = false;
    if (!configured) {
        cudaError_t e =
            cudaFuncSetAttribute(k_tile<R, M, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMaxSmem));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const uint64_t grid = uint64_t(1) << (pa.n - M);
    k_tile<R, M, RB><<<unsigned(grid), 1 << (M - RB), smem, h->stream>>>(
        static_cast<CT<R> *>(h->data), static_cast<const TileOp<R> *>(d_ops), d_segs, pa);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tile_pass(sv_state *h, const TilePassArgs &pa, const void *d_ops, const TileSeg *d_segs) {
    if (h->dt == SV_C64) return launch_impl<float, kTileM64, kTileRB64, kTileLow64>(h, pa, d_ops, d_segs);
    return launch_impl<double, kTileM128, kTileRB128, kTileLow128>(h, pa, d_ops, d_segs);
}

const char *tile_kernel_name(const sv_state *h) {
    return h->dt == SV_C64 ? "k_tile<f32,13,5>" : "k_tile<f64,12,4>";
}

}  // namespace sv
