// Two-byte adaptive amplitude code (Sec. 1 "JUQCS-A"; Sec. 3 on the cost of
// the encoding-decoding operation).
//
// Format (the paper cites but does not give its format; this is the reading
// the library implements): blocks of 256 consecutive amplitudes share one
// FP32 scale s = max over the block of max(|re|, |im|); each component is an
// int8 code q = rint(x * fl(127/s)) clamped to [-127, 127]; decoding gives
// x = sign(q) * fl(s * T[|q|]) with T[k] = fl(k / 127), so +-127 decodes to
// +-s exactly and the uniform superposition is represented exactly.
//
// A gate is one pass: every touched block is decoded into registers, the 2x2
// update runs in FP32 in a fixed fused-multiply-add order, the new block
// scale is a warp max and the block is re-encoded in place.  All arithmetic
// uses explicitly rounded intrinsics (no contraction), so codes are
// reproducible bit for bit by a CPU implementation of the same steps.
//
// Work mapping: one warp per 256-amplitude block, 8 amplitudes (16 code
// bytes, one 16-byte load) per lane.  Target bits 0-2 pair amplitudes inside
// a lane, bits 3-7 pair lanes (register exchange by shuffle), bits >= 8 pair
// two blocks that the same warp holds side by side.  A control bit >= 8
// selects whole blocks; blocks whose control bit is 0 are not touched
// (decode followed by encode with an unchanged scale returns the same codes).
#include "sv_internal.h"

namespace sv {
namespace {

constexpr int kWarpsPerCta = 8;

struct EncGateArgs {
    uint64_t nwork;     // warps of work (blocks or block pairs)
    int t, c;           // target, control (-1 none)
    int ins[2];         // ascending block-index positions where zero bits are inserted
    int nins;
    uint64_t set_mask;  // block-index bits forced to 1 (control >= 8)
    uint64_t tbit;      // block-index bit of the target (t >= 8)
    float u[8];
};

}  // namespace
}  // namespace sv

#include "enc_run.h"

namespace sv {
namespace {

__device__ __forceinline__ uint64_t insert_zero(uint64_t x, int p) {
    const uint64_t lo = x & ((uint64_t(1) << p) - 1);
    return ((x ^ lo) << 1) | lo;
}

// Zero bits inserted at the ascending positions p0, p1 (the first nins of
// them); constant indices keep the launch arguments out of local memory.
__device__ __forceinline__ uint64_t insert_zeros(uint64_t x, int nins, int p0, int p1) {
    if (nins > 0) x = insert_zero(x, p0);
    if (nins > 1) x = insert_zero(x, p1);
    return x;
}

// Signed table, indexed by the code's byte u = (uint8)q: tab[u * 32 + lane] =
// sign(q) fl(|q| / 127), replicated per bank.  fl(s * (-t)) = -fl(s * t), so
// s * tab[u] is exactly sign(q) fl(s T[|q|]).
constexpr int kTabFloats = 256 * 32;
__device__ __forceinline__ void load_table(float *tab) {
    for (int i = threadIdx.x; i < kTabFloats; i += blockDim.x) {
        const int q = int((signed char)(i >> 5));
        const int a = q < 0 ? -q : q;
        const float t = __fdiv_rn(float(a > 127 ? 127 : a), 127.0f);
        tab[i] = q < 0 ? -t : t;
    }
    __syncthreads();
}

__device__ __forceinline__ float dec1(uint32_t u, float s, const float *tab, int lane) {
    return __fmul_rn(s, tab[u * 32 + lane]);
}

// rint(x * fl(127/s)).  No clamp is needed: s is the exact maximum of |x| over
// the block, so |x * fl(127/s)| <= 127 (1 + 2^-24)^2 < 127.5.
__device__ __forceinline__ int enc1(float x, float inv) { return __float2int_rn(__fmul_rn(x, inv)); }

// The same code as a byte, without a float-to-integer conversion: for
// |v| < 2^22 the sum v + 1.5 * 2^23 lies in [2^23, 2^24), where the float
// spacing is 1, so the (round-to-nearest-even) addition yields exactly
// rint(v) + 1.5 * 2^23, whose bit pattern is 0x4B400000 + rint(v).  Its low
// byte is rint(v) mod 256, the two's-complement code byte.  The product is
// rounded on its own first (no contraction), as in enc1.
__device__ __forceinline__ uint32_t enc_bits(float x, float inv) {
    return __float_as_uint(__fadd_rn(__fmul_rn(x, inv), 12582912.0f));
}

__device__ __forceinline__ void gate_pair(const float *u, float &ar, float &ai, float &br, float &bi) {
    const float r0 = __fmaf_rn(u[0], ar, __fmaf_rn(-u[1], ai, __fmaf_rn(u[2], br, -__fmul_rn(u[3], bi))));
    const float i0 = __fmaf_rn(u[0], ai, __fmaf_rn(u[1], ar, __fmaf_rn(u[2], bi, __fmul_rn(u[3], br))));
    const float r1 = __fmaf_rn(u[4], ar, __fmaf_rn(-u[5], ai, __fmaf_rn(u[6], br, -__fmul_rn(u[7], bi))));
    const float i1 = __fmaf_rn(u[4], ai, __fmaf_rn(u[5], ar, __fmaf_rn(u[6], bi, __fmul_rn(u[7], br))));
    ar = r0;
    ai = i0;
    br = r1;
    bi = i1;
}

// Shape of the 2x2 matrix, chosen on the host from exact zeros: the general
// fixed-order update above, or the same update with the terms of zero
// coefficients left out.  A left-out term contributes fmaf(0, x, y) = y up to
// the sign of a zero, and a zero (of either sign) encodes to code 0 and does
// not change a block maximum, so the codes are those of the general form.
enum EncShape { ENC_GENERAL = 0, ENC_REAL = 1, ENC_DIAG = 2, ENC_DIAG1 = 3 };

template <int SHAPE>
__device__ __forceinline__ void gate_pair_s(const float *u, float &ar, float &ai, float &br, float &bi) {
    if constexpr (SHAPE == ENC_REAL) {  // every imaginary part 0 (u[1] = u[3] = u[5] = u[7] = 0)
        const float r0 = __fmaf_rn(u[0], ar, __fmul_rn(u[2], br));
        const float i0 = __fmaf_rn(u[0], ai, __fmul_rn(u[2], bi));
        const float r1 = __fmaf_rn(u[4], ar, __fmul_rn(u[6], br));
        const float i1 = __fmaf_rn(u[4], ai, __fmul_rn(u[6], bi));
        ar = r0;
        ai = i0;
        br = r1;
        bi = i1;
    } else if constexpr (SHAPE == ENC_DIAG || SHAPE == ENC_DIAG1) {  // u01 = u10 = 0
        if constexpr (SHAPE == ENC_DIAG) {  // (u00 = 1: a unchanged)
            const float r0 = __fmaf_rn(u[0], ar, -__fmul_rn(u[1], ai));
            const float i0 = __fmaf_rn(u[0], ai, __fmul_rn(u[1], ar));
            ar = r0;
            ai = i0;
        }
        const float r1 = __fmaf_rn(u[6], br, -__fmul_rn(u[7], bi));
        const float i1 = __fmaf_rn(u[6], bi, __fmul_rn(u[7], br));
        br = r1;
        bi = i1;
    } else {
        gate_pair(u, ar, ai, br, bi);
    }
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

struct Lane8 {
    float re[8], im[8];
};

// Byte k of w, zero-extended (one byte permute).
__device__ __forceinline__ uint32_t byte_of(uint32_t w, int k) { return __byte_perm(w, 0u, 0x4440u | uint32_t(k)); }

__device__ __forceinline__ void decode_lane(const int4 raw, float s, const float *tab, int lane, Lane8 &x) {
    const uint32_t w[4] = {uint32_t(raw.x), uint32_t(raw.y), uint32_t(raw.z), uint32_t(raw.w)};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t word = w[j >> 1];
        const int k = (j & 1) * 2;
        x.re[j] = dec1(byte_of(word, k), s, tab, lane);
        x.im[j] = dec1(byte_of(word, k + 1), s, tab, lane);
    }
}

__device__ __forceinline__ float lane_absmax(const Lane8 &x) {
    float m = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) m = fmaxf(m, fmaxf(fabsf(x.re[j]), fabsf(x.im[j])));
    return m;
}

// Encode a lane's 8 amplitudes with the block scale s (warp-uniform).
__device__ __forceinline__ int4 encode_lane(const Lane8 &x, float s) {
    if (s == 0.0f) return make_int4(0, 0, 0, 0);
    const float inv = __fdiv_rn(127.0f, s);
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // low bytes of the four sums: (re, im) of amplitudes 2k and 2k + 1
        const uint32_t lo = __byte_perm(enc_bits(x.re[2 * k], inv), enc_bits(x.im[2 * k], inv), 0x0040u);
        const uint32_t hi = __byte_perm(enc_bits(x.re[2 * k + 1], inv), enc_bits(x.im[2 * k + 1], inv), 0x0040u);
        w[k] = __byte_perm(lo, hi, 0x5410u);
    }
    return make_int4(int(w[0]), int(w[1]), int(w[2]), int(w[3]));
}

// Does amplitude j of this lane (in-block index lane*8 + j) satisfy the control?
__device__ __forceinline__ bool ctl_ok(int c, int lane, int j) {
    if (c < 0 || c >= kEncBlockLog2) return true;
    const int idx = lane * 8 + j;
    return (idx >> c) & 1;
}

// Pairs inside a lane (target bit TB < 8 of the lane's 8 amplitudes); the
// bit is a compile-time constant so the registers are indexed statically.
template <int SHAPE, int TB>
__device__ __forceinline__ void lane_pairs(const EncGateArgs &a, int lane, Lane8 &x) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j & TB) continue;
        if (!ctl_ok(a.c, lane, j)) continue;
        gate_pair_s<SHAPE>(a.u, x.re[j], x.im[j], x.re[j | TB], x.im[j | TB]);
    }
}

// Target inside the block (t < 8).
template <int SHAPE>
__global__ void __launch_bounds__(32 * kWarpsPerCta) k_enc_gate_in(int4 *__restrict__ codes, float *__restrict__ scales,
                                                                   EncGateArgs a) {
    __shared__ float tab[kTabFloats];
    load_table(tab);
    const int lane = threadIdx.x & 31;
    const uint64_t wid = uint64_t(blockIdx.x) * kWarpsPerCta + (threadIdx.x >> 5);
    const uint64_t nw = uint64_t(gridDim.x) * kWarpsPerCta;
    for (uint64_t w = wid; w < a.nwork; w += nw) {
        uint64_t b = w;
        b = insert_zeros(b, a.nins, a.ins[0], a.ins[1]);
        b |= a.set_mask;
        int4 raw = codes[b * 32 + lane];
        const float s = scales[b];
        Lane8 x;
        decode_lane(raw, s, tab, lane, x);
        if (a.t < 3) {
            if (a.t == 0)
                lane_pairs<SHAPE, 1>(a, lane, x);
            else if (a.t == 1)
                lane_pairs<SHAPE, 2>(a, lane, x);
            else
                lane_pairs<SHAPE, 4>(a, lane, x);
        } else {
            const int lb = 1 << (a.t - 3);
            const bool upper = lane & lb;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float pr = __shfl_xor_sync(0xffffffffu, x.re[j], lb);
                const float pi = __shfl_xor_sync(0xffffffffu, x.im[j], lb);
                if (!ctl_ok(a.c, lane, j)) continue;
                float ar = upper ? pr : x.re[j], ai = upper ? pi : x.im[j];
                float br = upper ? x.re[j] : pr, bi = upper ? x.im[j] : pi;
                gate_pair_s<SHAPE>(a.u, ar, ai, br, bi);
                x.re[j] = upper ? br : ar;
                x.im[j] = upper ? bi : ai;
            }
        }
        const float ns = warp_max(lane_absmax(x));
        codes[b * 32 + lane] = encode_lane(x, ns);
        if (lane == 0) scales[b] = ns;
    }
}

// Target across blocks (t >= 8): the warp holds block b0 and b0 + 2^(t-8).
template <int SHAPE>
__global__ void __launch_bounds__(32 * kWarpsPerCta) k_enc_gate_across(int4 *__restrict__ codes,
                                                                       float *__restrict__ scales, EncGateArgs a) {
    __shared__ float tab[kTabFloats];
    load_table(tab);
    const int lane = threadIdx.x & 31;
    const uint64_t wid = uint64_t(blockIdx.x) * kWarpsPerCta + (threadIdx.x >> 5);
    const uint64_t nw = uint64_t(gridDim.x) * kWarpsPerCta;
    for (uint64_t w = wid; w < a.nwork; w += nw) {
        uint64_t b0 = w;
        b0 = insert_zeros(b0, a.nins, a.ins[0], a.ins[1]);
        b0 |= a.set_mask;
        const uint64_t b1 = b0 | a.tbit;
        int4 r0 = codes[b0 * 32 + lane], r1 = codes[b1 * 32 + lane];
        const float s0 = scales[b0], s1 = scales[b1];
        Lane8 x, y;
        decode_lane(r0, s0, tab, lane, x);
        decode_lane(r1, s1, tab, lane, y);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (!ctl_ok(a.c, lane, j)) continue;
            gate_pair_s<SHAPE>(a.u, x.re[j], x.im[j], y.re[j], y.im[j]);
        }
        const float n0 = warp_max(lane_absmax(x));
        const float n1 = warp_max(lane_absmax(y));
        codes[b0 * 32 + lane] = encode_lane(x, n0);
        codes[b1 * 32 + lane] = encode_lane(y, n1);
        if (lane == 0) {
            scales[b0] = n0;
            scales[b1] = n1;
        }
    }
}

// Diagonal gate with u00 = 1 (T, P, ...) on a target at or above bit 8: the
// blocks with the target bit 0 keep their amplitudes, hence their scale and
// codes (decoding and re-encoding with an unchanged scale is the identity), so
// only the blocks with the target bit 1 are read and rewritten: half the
// traffic of the block-pair kernel, the same codes.
__global__ void __launch_bounds__(32 * kWarpsPerCta) k_enc_phase_blocks(int4 *__restrict__ codes,
                                                                        float *__restrict__ scales, EncGateArgs a) {
    __shared__ float tab[kTabFloats];
    load_table(tab);
    const int lane = threadIdx.x & 31;
    const uint64_t wid = uint64_t(blockIdx.x) * kWarpsPerCta + (threadIdx.x >> 5);
    const uint64_t nw = uint64_t(gridDim.x) * kWarpsPerCta;
    for (uint64_t w = wid; w < a.nwork; w += nw) {
        const uint64_t b = insert_zeros(w, a.nins, a.ins[0], a.ins[1]) | a.set_mask | a.tbit;
        const int4 raw = codes[b * 32 + lane];
        const float s = scales[b];
        Lane8 y;
        decode_lane(raw, s, tab, lane, y);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (!ctl_ok(a.c, lane, j)) continue;
            float ar = 0.0f, ai = 0.0f;  // the lower amplitude is left out (u00 = 1, u01 = u10 = 0)
            gate_pair_s<ENC_DIAG1>(a.u, ar, ai, y.re[j], y.im[j]);
        }
        const float ns = warp_max(lane_absmax(y));
        codes[b * 32 + lane] = encode_lane(y, ns);
        if (lane == 0) scales[b] = ns;
    }
}

// n < 8: one block of 2^n amplitudes, done by one thread in plain order.
__global__ void k_enc_gate_small(signed char *codes, float *scales, int n, EncGateArgs a) {
    __shared__ float re[128], im[128];
    if (threadIdx.x != 0) return;
    const int dim = 1 << n;
    const float s = scales[0];
    for (int i = 0; i < dim; ++i) {
        const int qr = codes[2 * i], qi = codes[2 * i + 1];
        const int ar = qr < 0 ? -qr : qr, ai = qi < 0 ? -qi : qi;
        const float vr = __fmul_rn(s, __fdiv_rn(float(ar), 127.0f));
        const float vi = __fmul_rn(s, __fdiv_rn(float(ai), 127.0f));
        re[i] = qr < 0 ? -vr : vr;
        im[i] = qi < 0 ? -vi : vi;
    }
    for (int i = 0; i < dim; ++i) {
        if ((i >> a.t) & 1) continue;
        if (a.c >= 0 && !((i >> a.c) & 1)) continue;
        const int j = i | (1 << a.t);
        gate_pair(a.u, re[i], im[i], re[j], im[j]);
    }
    float m = 0.0f;
    for (int i = 0; i < dim; ++i) m = fmaxf(m, fmaxf(fabsf(re[i]), fabsf(im[i])));
    scales[0] = m;
    const float inv = m == 0.0f ? 0.0f : __fdiv_rn(127.0f, m);
    for (int i = 0; i < dim; ++i) {
        codes[2 * i] = m == 0.0f ? 0 : (signed char)enc1(re[i], inv);
        codes[2 * i + 1] = m == 0.0f ? 0 : (signed char)enc1(im[i], inv);
    }
}

// c64 -> codes: one warp per block (n >= 8).
__global__ void __launch_bounds__(32 * kWarpsPerCta) k_encode(const float4 *__restrict__ psi, int4 *__restrict__ codes,
                                                              float *__restrict__ scales, uint64_t nblocks) {
    const int lane = threadIdx.x & 31;
    const uint64_t wid = uint64_t(blockIdx.x) * kWarpsPerCta + (threadIdx.x >> 5);
    const uint64_t nw = uint64_t(gridDim.x) * kWarpsPerCta;
    for (uint64_t b = wid; b < nblocks; b += nw) {
        Lane8 x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 v = psi[(b * 256 + lane * 8) / 2 + k];
            x.re[2 * k] = v.x;
            x.im[2 * k] = v.y;
            x.re[2 * k + 1] = v.z;
            x.im[2 * k + 1] = v.w;
        }
        const float s = warp_max(lane_absmax(x));
        codes[b * 32 + lane] = encode_lane(x, s);
        if (lane == 0) scales[b] = s;
    }
}

__global__ void __launch_bounds__(32 * kWarpsPerCta) k_decode(const int4 *__restrict__ codes,
                                                              const float *__restrict__ scales,
                                                              float4 *__restrict__ psi, uint64_t nblocks) {
    __shared__ float tab[kTabFloats];
    load_table(tab);
    const int lane = threadIdx.x & 31;
    const uint64_t wid = uint64_t(blockIdx.x) * kWarpsPerCta + (threadIdx.x >> 5);
    const uint64_t nw = uint64_t(gridDim.x) * kWarpsPerCta;
    for (uint64_t b = wid; b < nblocks; b += nw) {
        Lane8 x;
        decode_lane(codes[b * 32 + lane], scales[b], tab, lane, x);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            psi[(b * 256 + lane * 8) / 2 + k] = make_float4(x.re[2 * k], x.im[2 * k], x.re[2 * k + 1], x.im[2 * k + 1]);
    }
}

__global__ void k_encode_small(const float2 *psi, signed char *codes, float *scales, int n) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int dim = 1 << n;
    float m = 0.0f;
    for (int i = 0; i < dim; ++i) m = fmaxf(m, fmaxf(fabsf(psi[i].x), fabsf(psi[i].y)));
    scales[0] = m;
    const float inv = m == 0.0f ? 0.0f : __fdiv_rn(127.0f, m);
    for (int i = 0; i < dim; ++i) {
        codes[2 * i] = m == 0.0f ? 0 : (signed char)enc1(psi[i].x, inv);
        codes[2 * i + 1] = m == 0.0f ? 0 : (signed char)enc1(psi[i].y, inv);
    }
}

__global__ void k_decode_small(const signed char *codes, const float *scales, float2 *psi, int n) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int dim = 1 << n;
    const float s = scales[0];
    for (int i = 0; i < dim; ++i) {
        const int qr = codes[2 * i], qi = codes[2 * i + 1];
        const float vr = __fmul_rn(s, __fdiv_rn(float(qr < 0 ? -qr : qr), 127.0f));
        const float vi = __fmul_rn(s, __fdiv_rn(float(qi < 0 ? -qi : qi), 127.0f));
        psi[i] = make_float2(qr < 0 ? -vr : vr, qi < 0 ? -vi : vi);
    }
}


// ---------------------------------------------------------------- code-level fast paths
// Exact shortcuts of the decode-gate-encode pass.  Decoding and re-encoding a
// block with an unchanged scale returns its codes (|s T[q] fl(127/s) - q| is
// far below 1/2), and a diagonal gate with entries +-1, or a permutation of
// amplitudes inside a block or of whole blocks, leaves every block maximum
// unchanged; so these gates are sign flips or moves of the codes.

struct EncFlipArgs {
    uint64_t nwork;      // int4 words (8 amplitudes) to visit
    int ins[2], nins;    // ascending block-index positions where bits are inserted
    uint64_t set_mask;   // block-index bits forced to 1
    uint32_t lo_mask;    // in-block index bits of the condition (< 8)
    uint32_t lo_val;
};

// Negate the codes of every amplitude whose in-block bits match (lo_mask, lo_val)
// in the blocks selected by the inserted / forced block bits.
__global__ void __launch_bounds__(256) k_enc_flip(uint4 *__restrict__ codes, EncFlipArgs a) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t w = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < a.nwork; w += stride) {
        uint64_t b = w >> 5;  // selected block number, 32 words per block
        b = insert_zeros(b, a.nins, a.ins[0], a.ins[1]);
        b |= a.set_mask;
        const uint32_t lane = uint32_t(w & 31);
        uint4 v = codes[b * 32 + lane];
        uint32_t *x = reinterpret_cast<uint32_t *>(&v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t bm = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t idx = lane * 8 + 2 * k + h;
                if ((idx & a.lo_mask) == a.lo_val) bm |= 0xFFFFu << (16 * h);
            }
            x[k] = (x[k] & ~bm) | (__vneg4(x[k]) & bm);
        }
        codes[b * 32 + lane] = v;
    }
}

// X on in-block target t (< 8), optional control c: swap amplitude pairs
// inside each selected block; one warp per block.
__global__ void __launch_bounds__(256) k_enc_xin(uint4 *__restrict__ codes, EncGateArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t wid = uint64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
    const uint64_t nw = uint64_t(gridDim.x) * 8;
    for (uint64_t w = wid; w < a.nwork; w += nw) {
        uint64_t b = w;
        b = insert_zeros(b, a.nins, a.ins[0], a.ins[1]);
        b |= a.set_mask;
        const uint4 v = codes[b * 32 + lane];
        uint4 p;
        if (a.t >= 3) {
            const int lb = 1 << (a.t - 3);
            p.x = __shfl_xor_sync(0xffffffffu, v.x, lb);
            p.y = __shfl_xor_sync(0xffffffffu, v.y, lb);
            p.z = __shfl_xor_sync(0xffffffffu, v.z, lb);
            p.w = __shfl_xor_sync(0xffffffffu, v.w, lb);
        } else if (a.t == 0) {
            p = make_uint4(__byte_perm(v.x, 0, 0x1032), __byte_perm(v.y, 0, 0x1032), __byte_perm(v.z, 0, 0x1032),
                           __byte_perm(v.w, 0, 0x1032));
        } else if (a.t == 1) {
            p = make_uint4(v.y, v.x, v.w, v.z);
        } else {
            p = make_uint4(v.z, v.w, v.x, v.y);
        }
        const uint32_t *xv = reinterpret_cast<const uint32_t *>(&v), *xp = reinterpret_cast<const uint32_t *>(&p);
        uint32_t out[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t bm = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (ctl_ok(a.c, lane, 2 * k + h)) bm |= 0xFFFFu << (16 * h);
            out[k] = (xv[k] & ~bm) | (xp[k] & bm);
        }
        codes[b * 32 + lane] = make_uint4(out[0], out[1], out[2], out[3]);
    }
}

// X on a block-level target (>= 8) with no control or a block-level control:
// swap whole blocks (codes and scales); one warp per block pair.
__global__ void __launch_bounds__(256) k_enc_xblocks(uint4 *__restrict__ codes, float *__restrict__ scales,
                                                     EncGateArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t wid = uint64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
    const uint64_t nw = uint64_t(gridDim.x) * 8;
    for (uint64_t w = wid; w < a.nwork; w += nw) {
        uint64_t b0 = w;
        b0 = insert_zeros(b0, a.nins, a.ins[0], a.ins[1]);
        b0 |= a.set_mask;
        const uint64_t b1 = b0 | a.tbit;
        const uint4 v0 = codes[b0 * 32 + lane], v1 = codes[b1 * 32 + lane];
        codes[b0 * 32 + lane] = v1;
        codes[b1 * 32 + lane] = v0;
        if (lane == 0) {
            const float s0 = scales[b0];
            scales[b0] = scales[b1];
            scales[b1] = s0;
        }
    }
}

// ---------------------------------------------------------------- runs of in-block gates
// A run of consecutive gates that each act inside blocks (2x2 updates with a
// target below bit 8, any control) or are sign flips (+-1 diagonals on any
// qubits) is applied in one pass: each warp holds one block's codes and
// scale in registers and goes through the run in circuit order.  A gate is
// the same decode -> FP32 update -> block maximum -> encode as in
// k_enc_gate_in (the same functions, in the same order), and a flip negates
// codes as k_enc_flip does, so every block's codes and scale after the run
// are those of the gates applied one pass at a time: bit-exact.  A gate whose
// block-level control is 0 leaves the block as it is (decoding and
// re-encoding with an unchanged scale is the identity).

template <int SHAPE>
__device__ __forceinline__ void run_gate_in(const EncRunOp &op, int lane, Lane8 &x) {
    EncGateArgs a{};
    a.t = op.t;
    a.c = op.c;
#pragma unroll
    for (int k = 0; k < 8; ++k) a.u[k] = op.u[k];
    if (op.t < 3) {
        if (op.t == 0)
            lane_pairs<SHAPE, 1>(a, lane, x);
        else if (op.t == 1)
            lane_pairs<SHAPE, 2>(a, lane, x);
        else
            lane_pairs<SHAPE, 4>(a, lane, x);
    } else {
        const int lb = 1 << (op.t - 3);
        const bool upper = lane & lb;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float pr = __shfl_xor_sync(0xffffffffu, x.re[j], lb);
            const float pi = __shfl_xor_sync(0xffffffffu, x.im[j], lb);
            if (!ctl_ok(a.c, lane, j)) continue;
            float ar = upper ? pr : x.re[j], ai = upper ? pi : x.im[j];
            float br = upper ? x.re[j] : pr, bi = upper ? x.im[j] : pi;
            gate_pair_s<SHAPE>(a.u, ar, ai, br, bi);
            x.re[j] = upper ? br : ar;
            x.im[j] = upper ? bi : ai;
        }
    }
}

__global__ void __launch_bounds__(32 * kWarpsPerCta) k_enc_run_in(int4 *__restrict__ codes, float *__restrict__ scales,
                                                                  uint64_t nblocks, const EncRunOp *__restrict__ gops,
                                                                  int nops) {
    __shared__ float tab[kTabFloats];
    __shared__ EncRunOp ops[kEncRunMaxOps];
    for (int i = threadIdx.x; i < nops; i += blockDim.x) ops[i] = gops[i];
    load_table(tab);  // (its barrier also publishes the ops)
    const int lane = threadIdx.x & 31;
    const uint64_t wid = uint64_t(blockIdx.x) * kWarpsPerCta + (threadIdx.x >> 5);
    const uint64_t nw = uint64_t(gridDim.x) * kWarpsPerCta;
    for (uint64_t b = wid; b < nblocks; b += nw) {
        int4 raw = codes[b * 32 + lane];
        float s = scales[b];
        for (int i = 0; i < nops; ++i) {
            const EncRunOp &op = ops[i];
            if ((b & op.hi_mask) != op.hi_val) continue;  // block-level condition not met
            if (op.kind == 1) {  // sign flip of the codes whose in-block bits match
                uint32_t *x = reinterpret_cast<uint32_t *>(&raw);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint32_t bm = 0;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t idx = uint32_t(lane) * 8 + 2 * k + h;
                        if ((idx & op.lo_mask) == op.lo_val) bm |= 0xFFFFu << (16 * h);
                    }
                    x[k] = (x[k] & ~bm) | (__vneg4(x[k]) & bm);
                }
                continue;
            }
            Lane8 x;
            decode_lane(raw, s, tab, lane, x);
            switch (op.shape) {
                case ENC_REAL: run_gate_in<ENC_REAL>(op, lane, x); break;
                case ENC_DIAG: run_gate_in<ENC_DIAG>(op, lane, x); break;
                case ENC_DIAG1: run_gate_in<ENC_DIAG1>(op, lane, x); break;
                default: run_gate_in<ENC_GENERAL>(op, lane, x); break;
            }
            s = warp_max(lane_absmax(x));
            raw = encode_lane(x, s);
        }
        codes[b * 32 + lane] = raw;
        if (lane == 0) scales[b] = s;
    }
}

int enc_grid(uint64_t nwork) {
    uint64_t b = (nwork + kWarpsPerCta - 1) / kWarpsPerCta;
    const uint64_t cap = 152ull * 16;
    return int(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

cudaError_t launch_enc_gate1(sv_state *h, const Gate1 &g) {
    EncGateArgs a{};
    for (int k = 0; k < 4; ++k) {
        a.u[2 * k] = float(g.u[k].re);  // round to nearest
        a.u[2 * k + 1] = float(g.u[k].im);
    }
    a.t = g.target;
    a.c = g.control;
    const int n = h->n;
    if (n < kEncBlockLog2) {
        k_enc_gate_small<<<1, 32, 0, h->stream>>>(static_cast<signed char *>(h->data), h->scales, n, a);
        return cudaGetLastError();
    }
    const int nb_log = n - kEncBlockLog2;
    const Cplx *u = g.u;
    auto is = [](const Cplx &z, double re) { return z.re == re && z.im == 0.0; };
    // diagonal with entries +-1 (Z, CZ, ...): sign flips of codes
    if (is(u[1], 0) && is(u[2], 0) && (is(u[0], 1) || is(u[0], -1)) && (is(u[3], 1) || is(u[3], -1))) {
        if (is(u[0], 1) && is(u[3], 1)) return cudaSuccess;  // identity
        uint64_t m = g.control >= 0 ? (uint64_t(1) << g.control) : 0, v = m;
        if (!(is(u[0], -1) && is(u[3], -1))) {  // only one half flips: condition on the target bit
            m |= uint64_t(1) << g.target;
            if (is(u[3], -1)) v |= uint64_t(1) << g.target;
        }
        EncFlipArgs fa{};
        fa.lo_mask = uint32_t(m & 0xFFu);
        fa.lo_val = uint32_t(v & 0xFFu);
        int k = 0;
        for (int bit = kEncBlockLog2; bit < n; ++bit)
            if (m >> bit & 1) {
                fa.ins[k++] = bit - kEncBlockLog2;
                if (v >> bit & 1) fa.set_mask |= uint64_t(1) << (bit - kEncBlockLog2);
            }
        fa.nins = k;
        fa.nwork = (uint64_t(1) << (nb_log - k)) * 32;
        const uint64_t blocks = (fa.nwork + 255) / 256;
        k_enc_flip<<<unsigned(blocks < 152 * 32 ? blocks : 152 * 32), 256, 0, h->stream>>>(static_cast<uint4 *>(h->data),
                                                                                          fa);
        return cudaGetLastError();
    }
    const bool xgate = is(u[0], 0) && is(u[3], 0) && is(u[1], 1) && is(u[2], 1);
    int ins[2], ni = 0;
    if (a.c >= kEncBlockLog2) {
        ins[ni++] = a.c - kEncBlockLog2;
        a.set_mask = uint64_t(1) << (a.c - kEncBlockLog2);
    }
    if (a.t >= kEncBlockLog2) {
        ins[ni++] = a.t - kEncBlockLog2;
        a.tbit = uint64_t(1) << (a.t - kEncBlockLog2);
    }
    if (ni == 2 && ins[0] > ins[1]) {
        const int t = ins[0];
        ins[0] = ins[1];
        ins[1] = t;
    }
    for (int k = 0; k < ni; ++k) a.ins[k] = ins[k];
    a.nins = ni;
    a.nwork = uint64_t(1) << (nb_log - ni);
    int4 *codes = static_cast<int4 *>(h->data);
    if (xgate && a.t < kEncBlockLog2) {  // permutation inside blocks
        k_enc_xin<<<enc_grid(a.nwork), 256, 0, h->stream>>>(reinterpret_cast<uint4 *>(codes), a);
        return cudaGetLastError();
    }
    if (xgate && (a.c < 0 || a.c >= kEncBlockLog2)) {  // whole-block swaps
        k_enc_xblocks<<<enc_grid(a.nwork), 256, 0, h->stream>>>(reinterpret_cast<uint4 *>(codes), h->scales, a);
        return cudaGetLastError();
    }
    // matrix shape from exact zeros of the FP32 entries the kernel uses
    const bool real = a.u[1] == 0.0f && a.u[3] == 0.0f && a.u[5] == 0.0f && a.u[7] == 0.0f;
    const bool diag = a.u[2] == 0.0f && a.u[3] == 0.0f && a.u[4] == 0.0f && a.u[5] == 0.0f;
    const bool one = diag && a.u[0] == 1.0f && a.u[1] == 0.0f;
    const int shape = one ? ENC_DIAG1 : diag ? ENC_DIAG : real ? ENC_REAL : ENC_GENERAL;
    const unsigned grid = enc_grid(a.nwork), block = 32 * kWarpsPerCta;
    if (a.t < kEncBlockLog2) {
        switch (shape) {
            case ENC_REAL: k_enc_gate_in<ENC_REAL><<<grid, block, 0, h->stream>>>(codes, h->scales, a); break;
            case ENC_DIAG: k_enc_gate_in<ENC_DIAG><<<grid, block, 0, h->stream>>>(codes, h->scales, a); break;
            case ENC_DIAG1: k_enc_gate_in<ENC_DIAG1><<<grid, block, 0, h->stream>>>(codes, h->scales, a); break;
            default: k_enc_gate_in<ENC_GENERAL><<<grid, block, 0, h->stream>>>(codes, h->scales, a); break;
        }
    } else {
        switch (shape) {
            case ENC_REAL: k_enc_gate_across<ENC_REAL><<<grid, block, 0, h->stream>>>(codes, h->scales, a); break;
            case ENC_DIAG: k_enc_gate_across<ENC_DIAG><<<grid, block, 0, h->stream>>>(codes, h->scales, a); break;
            case ENC_DIAG1: k_enc_phase_blocks<<<grid, block, 0, h->stream>>>(codes, h->scales, a); break;
            default: k_enc_gate_across<ENC_GENERAL><<<grid, block, 0, h->stream>>>(codes, h->scales, a); break;
        }
    }
    return cudaGetLastError();
}

// The matrix shape of a gate from exact zeros of its FP32 entries.
static int enc_shape(const float *u) {
    const bool real = u[1] == 0.0f && u[3] == 0.0f && u[5] == 0.0f && u[7] == 0.0f;
    const bool diag = u[2] == 0.0f && u[3] == 0.0f && u[4] == 0.0f && u[5] == 0.0f;
    const bool one = diag && u[0] == 1.0f && u[1] == 0.0f;
    return one ? ENC_DIAG1 : diag ? ENC_DIAG : real ? ENC_REAL : ENC_GENERAL;
}

bool enc_run_op(int n, const Gate1 &g, EncRunOp *op) {
    if (n < kEncBlockLog2) return false;
    *op = EncRunOp{};
    const Cplx *u = g.u;
    auto is = [](const Cplx &z, double re) { return z.re == re && z.im == 0.0; };
    if (is(u[1], 0) && is(u[2], 0) && (is(u[0], 1) || is(u[0], -1)) && (is(u[3], 1) || is(u[3], -1))) {
        // +-1 diagonal: a sign flip on any qubits (identity: an empty flip)
        uint64_t m = g.control >= 0 ? (uint64_t(1) << g.control) : 0, v = m;
        if (!(is(u[0], -1) && is(u[3], -1))) {
            m |= uint64_t(1) << g.target;
            if (is(u[3], -1)) v |= uint64_t(1) << g.target;
        }
        op->kind = 1;
        op->lo_mask = uint32_t(m & 0xFFu);
        op->lo_val = uint32_t(v & 0xFFu);
        op->hi_mask = m >> kEncBlockLog2;
        op->hi_val = v >> kEncBlockLog2;
        if (is(u[0], 1) && is(u[3], 1)) {  // identity: a flip that matches no amplitude
            op->lo_mask = 0;
            op->lo_val = 1;
        }
        return true;
    }
    if (g.target >= kEncBlockLog2) return false;
    op->kind = 0;
    op->t = g.target;
    op->c = g.control >= 0 && g.control < kEncBlockLog2 ? g.control : -1;
    if (g.control >= kEncBlockLog2) op->hi_mask = op->hi_val = uint64_t(1) << (g.control - kEncBlockLog2);
    for (int k = 0; k < 4; ++k) {
        op->u[2 * k] = float(g.u[k].re);
        op->u[2 * k + 1] = float(g.u[k].im);
    }
    op->shape = enc_shape(op->u);
    return true;
}

cudaError_t launch_enc_run(sv_state *h, const EncRunOp *d_ops, int nops) {
    const uint64_t nb = uint64_t(1) << (h->n - kEncBlockLog2);
    k_enc_run_in<<<enc_grid(nb), 32 * kWarpsPerCta, 0, h->stream>>>(static_cast<int4 *>(h->data), h->scales, nb,
                                                                    d_ops, nops);
    return cudaGetLastError();
}

cudaError_t launch_encode(const sv_state *src, sv_state *dst) {
    const int n = src->n;
    if (n < kEncBlockLog2) {
        k_encode_small<<<1, 32, 0, dst->stream>>>(static_cast<const float2 *>(src->data),
                                                  static_cast<signed char *>(dst->data), dst->scales, n);
    } else {
        const uint64_t nb = uint64_t(1) << (n - kEncBlockLog2);
        k_encode<<<enc_grid(nb), 32 * kWarpsPerCta, 0, dst->stream>>>(static_cast<const float4 *>(src->data),
                                                                      static_cast<int4 *>(dst->data), dst->scales, nb);
    }
    return cudaGetLastError();
}

cudaError_t launch_decode(const sv_state *src, sv_state *dst) {
    const int n = src->n;
    if (n < kEncBlockLog2) {
        k_decode_small<<<1, 32, 0, dst->stream>>>(static_cast<const signed char *>(src->data), src->scales,
                                                  static_cast<float2 *>(dst->data), n);
    } else {
        const uint64_t nb = uint64_t(1) << (n - kEncBlockLog2);
        k_decode<<<enc_grid(nb), 32 * kWarpsPerCta, 0, dst->stream>>>(static_cast<const int4 *>(src->data), src->scales,
                                                                      static_cast<float4 *>(dst->data), nb);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- read-out
namespace {

__device__ __forceinline__ float dec_plain(int q, float s) {
    const float v = __fmul_rn(s, __fdiv_rn(float(q < 0 ? -q : q), 127.0f));
    return q < 0 ? -v : v;
}

__global__ void k_enc_gather(const char2 *__restrict__ codes, const float *__restrict__ scales, int n,
                             const uint64_t *__restrict__ idx, size_t m, double2 *__restrict__ out) {
    for (size_t j = size_t(blockIdx.x) * blockDim.x + threadIdx.x; j < m; j += size_t(gridDim.x) * blockDim.x) {
        const uint64_t i = idx[j];
        const float s = scales[n < kEncBlockLog2 ? 0 : (i >> kEncBlockLog2)];
        const char2 q = codes[i];
        out[j] = make_double2(dec_plain(q.x, s), dec_plain(q.y, s));
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of |decoded amplitude|^2: one warp per block, 4-amplitude FP32
// partial sums, FP64 beyond; one partial per CTA.
__global__ void __launch_bounds__(256) k_enc_norm(const int4 *__restrict__ codes, const float *__restrict__ scales,
                                                  uint64_t nblocks, double *__restrict__ partials) {
    __shared__ float tab[kTabFloats];
    __shared__ double sh[8];
    load_table(tab);
    const int lane = threadIdx.x & 31;
    const uint64_t wid = uint64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
    const uint64_t nw = uint64_t(gridDim.x) * 8;
    double acc = 0.0;
    for (uint64_t b = wid; b < nblocks; b += nw) {
        Lane8 x;
        decode_lane(codes[b * 32 + lane], scales[b], tab, lane, x);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float s = 0.0f;
#pragma unroll
            for (int j = 4 * h; j < 4 * h + 4; ++j) s = fmaf(x.re[j], x.re[j], fmaf(x.im[j], x.im[j], s));
            acc += double(s);
        }
    }
    acc = warp_sum_d(acc);
    if (lane == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += sh[k];
        partials[blockIdx.x] = t;
    }
}

__global__ void k_enc_norm_small(const signed char *codes, const float *scales, int n, double *partials, int np) {
    if (threadIdx.x != 0) return;
    double acc = 0.0;
    for (int i = 0; i < (1 << n); ++i) {
        const float a = dec_plain(codes[2 * i], scales[0]), b = dec_plain(codes[2 * i + 1], scales[0]);
        acc += double(a) * a + double(b) * b;
    }
    for (int k = 0; k < np; ++k) partials[k] = k == 0 ? acc : 0.0;
}

__global__ void k_sum_partials(const double *__restrict__ partials, int np, double *out) {
    __shared__ double sh[8];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < int(blockDim.x >> 5); ++k) t += sh[k];
        *out = t;
    }
}

}  // namespace

cudaError_t launch_enc_gather(sv_state *h, const uint64_t *d_idx, size_t m, double *d_out) {
    if (m == 0) return cudaSuccess;
    const int blocks = int((m + 255) / 256 < 1024 ? (m + 255) / 256 : 1024);
    k_enc_gather<<<blocks, 256, 0, h->stream>>>(static_cast<const char2 *>(h->data), h->scales, h->n, d_idx, m,
                                                reinterpret_cast<double2 *>(d_out));
    return cudaGetLastError();
}

cudaError_t launch_enc_norm(sv_state *h, double *d_out) {
    const int np = norm_partials_needed(h);
    if (h->n < kEncBlockLog2) {
        k_enc_norm_small<<<1, 32, 0, h->stream>>>(static_cast<const signed char *>(h->data), h->scales, h->n,
                                                  h->d_partials, np);
    } else {
        const uint64_t nb = uint64_t(1) << (h->n - kEncBlockLog2);
        k_enc_norm<<<np, 256, 0, h->stream>>>(static_cast<const int4 *>(h->data), h->scales, nb, h->d_partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_partials<<<1, 256, 0, h->stream>>>(h->d_partials, np, d_out);
    return cudaGetLastError();
}

}  // namespace sv
