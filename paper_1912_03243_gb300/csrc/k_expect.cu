// Expectation values <sigma^alpha_i> of every qubit i (Sec. 3: the
// validation observable <Q_alpha(i)> = (1 - <sigma^alpha_i>)/2), complex64,
// complex128 and the two-byte code.
//
// For qubit k and the pairs (a, b) = (psi_j, psi_{j + 2^k}) with bit k of j
// clear:  <sigma^x_k> = sum 2 Re(conj(a) b),  <sigma^y_k> = sum 2 Im(conj(a) b),
// <sigma^z_k> = sum |a|^2 - |b|^2.  A pass reads the state once in tiles of
// 2^m amplitudes (the low qubits plus chosen ones, as in the tiled gate
// passes) and sums these over every tile qubit; <sigma^z> of the qubits
// outside the tile follows from each tile's total probability, signed by the
// tile number's bits.  Persistent CTAs accumulate in FP32 (FP64 for
// complex128) per tile, or per chunk of 8 tiles in the 13-bit kernel, and in
// FP64 beyond; the host adds the CTAs' partials.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "sv_internal.h"

namespace sv {
namespace {

constexpr int kExThreads = 256;
constexpr int kExWarps = kExThreads / 32;
constexpr int kExMaxM = 13;
constexpr int kExMaxOuter = 40;
constexpr int kExVals = 3 * kExMaxM + kExMaxOuter;  // per-CTA partial: x, y, z per tile bit, z per outer bit

struct ExpArgs {
    int n, m;           // qubits, tile bits
    int nouter;
    int zouter;         // accumulate <sigma^z> of the outer qubits (one pass does)
    uint64_t ntiles;
    uint8_t tile_pos[kExMaxM];
    uint8_t outer_pos[kExMaxOuter];
};

__device__ __forceinline__ uint32_t insert_zero32(uint32_t x, int p) {
    const uint32_t lo = x & ((1u << p) - 1u);
    return ((x ^ lo) << 1) | lo;
}

template <typename C>
struct Real;
template <>
struct Real<float2> {
    using T = float;
};
template <>
struct Real<double2> {
    using T = double;
};

// Tile into shared memory (plain layout, tile index j at sm[j]).
// complex64 / complex128: thread t loads j = t + 256 r; the global offset is a
// per-thread part XOR a per-r part (disjoint bits).
template <typename C>
__device__ void load_tile(const C *__restrict__ psi, C *sm, const ExpArgs &a, uint64_t cta, const uint64_t *gR) {
    uint64_t base = 0;
    for (int o = 0; o < a.nouter; ++o) base |= ((cta >> o) & 1ull) << a.outer_pos[o];
    const int t = threadIdx.x;
    const int tb = a.m < 8 ? a.m : 8;
    uint64_t gT = 0;
    for (int q = 0; q < tb; ++q)
        if (t >> q & 1) gT |= uint64_t(1) << a.tile_pos[q];
    const int size = 1 << a.m;
    for (int r = 0; (r << 8) < size; ++r) {
        const int j = t + (r << 8);
        if (j < size) sm[j] = psi[base | gT | gR[r]];
    }
}

// Two-byte code: whole 256-amplitude blocks (tile bits 0..7 are the in-block
// bits); x = s * tab[u] with the signed table tab[u] = sign(q) fl(|q| / 127).
__device__ void load_tile_enc(const int4 *__restrict__ codes, const signed char *__restrict__ codes8,
                              const float *__restrict__ scales, float2 *sm, const ExpArgs &a, uint64_t cta,
                              const float *tab) {
    if (a.n < 8) {  // one block of 2^n amplitudes, byte codes
        for (int j = threadIdx.x; j < (1 << a.n); j += kExThreads) {
            const float s = scales[0];
            sm[j] = make_float2(__fmul_rn(s, tab[uint8_t(codes8[2 * j])]), __fmul_rn(s, tab[uint8_t(codes8[2 * j + 1])]));
        }
        return;
    }
    uint64_t bbase = 0;  // block index of the tile's outer bits
    for (int o = 0; o < a.nouter; ++o) bbase |= ((cta >> o) & 1ull) << (a.outer_pos[o] - kEncBlockLog2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nblk = 1 << (a.m - kEncBlockLog2);
    for (int bl = warp; bl < nblk; bl += kExWarps) {
        uint64_t b = bbase;
        for (int q = kEncBlockLog2; q < a.m; ++q)
            if (bl >> (q - kEncBlockLog2) & 1) b |= uint64_t(1) << (a.tile_pos[q] - kEncBlockLog2);
        const int4 raw = codes[b * 32 + lane];
        const float s = scales[b];
        const uint32_t w[4] = {uint32_t(raw.x), uint32_t(raw.y), uint32_t(raw.z), uint32_t(raw.w)};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const uint32_t word = w[e >> 1], sh = (e & 1) * 16;
            sm[(bl << kEncBlockLog2) | (lane * 8 + e)] =
                make_float2(__fmul_rn(s, tab[(word >> sh) & 0xFFu]), __fmul_rn(s, tab[(word >> (sh + 8)) & 0xFFu]));
        }
    }
}

template <typename C, bool ENC>
__global__ void __launch_bounds__(kExThreads) k_expect(const void *__restrict__ data, const float *__restrict__ scales,
                                                       const ExpArgs a, double *__restrict__ partials) {
    using R = typename Real<C>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    C *sm = reinterpret_cast<C *>(smem);
    __shared__ double acc[kExVals];
    __shared__ R red[kExWarps][3 * kExMaxM + 1];
    __shared__ uint64_t gR[32];
    __shared__ float tab[256];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int i = t; i < kExVals; i += kExThreads) acc[i] = 0.0;
    if (!ENC) {
        for (int r = t; r < 32; r += kExThreads) {  // tile bits 8.. of j = 256 r
            uint64_t g = 0;
            for (int q = 8; q < a.m; ++q)
                if ((r << 8) >> q & 1) g |= uint64_t(1) << a.tile_pos[q];
            gR[r] = g;
        }
    } else {
        for (int u = t; u < 256; u += kExThreads) {
            const int q = int((signed char)u);
            const int aq = q < 0 ? -q : q;
            const float v = __fdiv_rn(float(aq > 127 ? 127 : aq), 127.0f);
            tab[u] = q < 0 ? -v : v;
        }
    }
    __syncthreads();
    const int half = 1 << (a.m - 1);
    for (uint64_t cta = blockIdx.x; cta < a.ntiles; cta += gridDim.x) {
        if (ENC)
            load_tile_enc(static_cast<const int4 *>(data), static_cast<const signed char *>(data), scales,
                          reinterpret_cast<float2 *>(sm), a, cta, tab);
        else
            load_tile(static_cast<const C *>(data), sm, a, cta, gR);
        __syncthreads();
        R v[3 * kExMaxM + 1];
#pragma unroll
        for (int i = 0; i < 3 * kExMaxM + 1; ++i) v[i] = R(0);
#pragma unroll
        for (int k = 0; k < kExMaxM; ++k) {
            if (k >= a.m) break;
            for (int p = t; p < half; p += kExThreads) {
                const uint32_t j = insert_zero32(uint32_t(p), k);
                const C x = sm[j], y = sm[j | (1u << k)];
                const R pa = x.x * x.x + x.y * x.y, pb = y.x * y.x + y.y * y.y;
                v[3 * k] += x.x * y.x + x.y * y.y;      // Re(conj(a) b)
                v[3 * k + 1] += x.x * y.y - x.y * y.x;  // Im(conj(a) b)
                v[3 * k + 2] += pa - pb;
                if (k == 0) v[3 * kExMaxM] += pa + pb;  // the tile's probability
            }
        }
        // block sums: warps, then FP64 across warps and tiles
#pragma unroll
        for (int i = 0; i < 3 * kExMaxM + 1; ++i) {
            R s = v[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) red[warp][i] = s;
        }
        __syncthreads();
        if (t < 3 * a.m) {
            double s = 0.0;
            for (int w = 0; w < kExWarps; ++w) s += double(red[w][t]);
            acc[t] += (t % 3 == 2) ? s : 2.0 * s;
        } else if (a.zouter && t >= 64 && t < 64 + a.nouter) {
            const int o = t - 64;
            double P = 0.0;
            for (int w = 0; w < kExWarps; ++w) P += double(red[w][3 * kExMaxM]);
            acc[3 * kExMaxM + o] += ((cta >> o) & 1ull) ? -P : P;
        }
        __syncthreads();
    }
    for (int i = t; i < kExVals; i += kExThreads) partials[size_t(blockIdx.x) * kExVals + i] = acc[i];
}

// 2^13-amplitude tiles of complex64 (or decoded codes): each thread holds 32
// amplitudes in registers and takes the pairs of five tile qubits at a time
// (tile bits 8..12, then 3..7, then 0..2), three gathers from shared memory
// instead of one sweep per qubit.  Shared layout j -> xswz(j): the load
// (lanes along tile bits 0..4), the three gathers (lanes along bits 0..4;
// 0,1,2,8,9; 5..9) and the code decode (lanes along bits 3..7) each touch
// every bank the minimum number of times.
__device__ __forceinline__ uint32_t xswz(uint32_t j) { return j ^ ((j >> 5) & 7u) ^ (((j >> 8) & 3u) << 3); }

__device__ __forceinline__ unsigned long long pk2(float x, float y) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float &x, float &y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(r));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Pairs over register bits 0..NB-1: Re and Im of conj(p) q for p = x[r],
// q = x[r + 2^b] (bit b of r clear).  Two packed accumulators per bit whose
// operands are the registers as they stand, or p with its halves swapped
// (one swap per register, shared by all its pairs):
//   A += (p.x q.x, p.y q.y)  ->  Re = A.x + A.y
//   B += (p.y q.x, p.x q.y)  ->  Im = B.y - B.x
template <int NB>
__device__ __forceinline__ void seg_pairs(const float2 (&x)[32], float *re, float *im) {
    unsigned long long A[NB], B[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) A[b] = B[b] = 0ull;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        if ((r & ((1 << NB) - 1)) == (1 << NB) - 1) continue;  // no pair has r as its lower element
        const unsigned long long p = pk2(x[r].x, x[r].y), ps = pk2(x[r].y, x[r].x);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (r >> b & 1) continue;
            const unsigned long long q = pk2(x[r | (1 << b)].x, x[r | (1 << b)].y);
            A[b] = fma2(p, q, A[b]);
            B[b] = fma2(ps, q, B[b]);
        }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        float ax, ay, bx, by;
        upk2(A[b], ax, ay);
        upk2(B[b], bx, by);
        re[b] = ax + ay;
        im[b] = by - bx;
    }
}

// Probability of the 32 register amplitudes.
__device__ __forceinline__ float seg_total(const float2 (&x)[32]) {
    unsigned long long s0 = 0ull, s1 = 0ull;
#pragma unroll
    for (int r = 0; r < 32; r += 2) {
        const unsigned long long p = pk2(x[r].x, x[r].y), q = pk2(x[r + 1].x, x[r + 1].y);
        s0 = fma2(p, p, s0);
        s1 = fma2(q, q, s1);
    }
    float a, b, c, d;
    upk2(s0, a, b);
    upk2(s1, c, d);
    return (a + b) + (c + d);
}

// v with its sign flipped where bit b of the lane index is set.
__device__ __forceinline__ float lane_signed(float v, int lane, int b) {
    return __int_as_float(__float_as_int(v) ^ int(uint32_t(lane >> b & 1) << 31));
}

__device__ __forceinline__ float warp_sum(float s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// One step of a warp reduce-scatter on the value pair (v[i], v[i + H]): the
// lane keeps the member whose index has bit H equal to its own lane bit H and
// adds its partner's copy of it.  After the steps H = 16, 8, 4, 2, 1 over all
// pairs, v[0] of lane l is the warp's sum of v[l].
template <int H>
__device__ __forceinline__ void rs_pair(float (&v)[32], int lane, int i) {
    const bool up = lane & H;
    const float send = up ? v[i] : v[i + H];
    const float keep = up ? v[i + H] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, H);
}

template <int H>
__device__ __forceinline__ void rs_step(float (&v)[32], int lane) {
#pragma unroll
    for (int i = 0; i < H; ++i) rs_pair<H>(v, lane, i);
}

// The tile's global offset from its number (outer qubit o is bit o of the
// tile number): one table lookup per 4-bit nibble of the number.
__device__ __forceinline__ uint64_t tile_base(const uint64_t (*tO)[16], int nnib, uint64_t cta) {
    uint64_t base = 0;
    for (int k = 0; k < nnib; ++k) base |= tO[k][(cta >> (4 * k)) & 15u];
    return base;
}

// complex64: every copy of the tile in flight at once (cp.async, 8 bytes
// each; thread t takes j = t | r << 8).
__device__ __forceinline__ void c64_issue(const float2 *__restrict__ psi, float2 *sm, uint64_t base, uint64_t gT,
                                          const uint64_t *gR, int t) {
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const uint32_t sa = uint32_t(__cvta_generic_to_shared(sm + xswz(uint32_t(t | (r << 8)))));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(psi + (base | gT | gR[r])) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Two-byte code: warp w holds the raw codes of in-tile blocks w, w + 8, w + 16,
// w + 24 (one int4 of 8 amplitudes per lane) and their scales until the
// decode; x = s * tab[u] with the signed table tab[u] = sign(q) fl(|q| / 127).
struct EncRaw {
    int4 raw[4];
    float sc[4];
};

__device__ __forceinline__ void enc_fetch(const int4 *__restrict__ codes, const float *__restrict__ scales,
                                          uint64_t bbase, const uint64_t (&boff)[4], int lane, EncRaw &e) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint64_t b = bbase | boff[i];
        e.raw[i] = codes[b * 32 + lane];
        e.sc[i] = scales[b];
    }
}

__device__ __forceinline__ void enc_decode(const EncRaw &e, float2 *sm, const float *tab, int warp, int lane) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int bl = warp + kExWarps * i;
        const uint32_t w[4] = {uint32_t(e.raw[i].x), uint32_t(e.raw[i].y), uint32_t(e.raw[i].z), uint32_t(e.raw[i].w)};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t word = w[k >> 1], sh = (k & 1) * 16;
            sm[xswz(uint32_t((bl << kEncBlockLog2) | (lane * 8 + k)))] = make_float2(
                __fmul_rn(e.sc[i], tab[(word >> sh) & 0xFFu]), __fmul_rn(e.sc[i], tab[(word >> (sh + 8)) & 0xFFu]));
        }
    }
}

// Per-warp value slots of k_expect13 (each lane accumulates one of the 32
// reduce-scattered values, lanes 0..2 one of the three full warp sums, lane o
// the signed total of outer qubit o):
//   0..12   Re sum of tile bit k            16..28  Im sum of tile bit k
//   13, 14, 15, 29, 30  segment-1 probability signed by lane bit 0..4
//                       (<sigma^z> of tile bits 0..4)
//   31      segment-2 probability signed by lane bit 3  (tile bit 8)
//   32, 33  segment-1 / segment-2 probability (tile bits 5..7 / 10..12 by warp bits; outer qubits)
//   34      segment-2 probability signed by lane bit 4  (tile bit 9)
//   35..66  outer qubit o: the segment-1 probability signed by bit o of the tile number
// Segment 3's six values sit in the pairs (0, 16), (1, 17), (2, 18) of the
// first reduce-scatter step, so the other pairs are reduced before it.
constexpr int kExWSlots = 35 + 32;
constexpr int kExChunk = 8;  // tiles summed in FP32 before an FP64 add

// FIRST: the pass over tile qubits 0..12, every tile bit and <sigma^z> of all
// qubits.  Later passes take only the tile bits above the low ones they share
// with pass 0 (tile bits 3..12 of complex64, 8..12 of the code).  Segment 1
// leaves tile bits 0..7 to the thread index, segment 2 bits 0..2 and 8..12,
// so <sigma^z> of every tile bit follows from two per-thread probabilities
// signed by thread-index bits.  The next tile's load is issued as soon as the
// last gather from shared memory is done, under the rest of the arithmetic.
template <bool ENC, bool FIRST>
__global__ void __launch_bounds__(kExThreads, 2) k_expect13(const void *__restrict__ data,
                                                            const float *__restrict__ scales, const ExpArgs a,
                                                            double *__restrict__ partials) {
    constexpr int kSegs = FIRST ? 3 : (ENC ? 1 : 2);
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *sm = reinterpret_cast<float2 *>(smem);
    __shared__ double wsum[kExWarps][kExWSlots];
    __shared__ uint64_t gR[32];
    __shared__ uint64_t tO[kExMaxOuter / 4][16];
    __shared__ float tab[256];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int r = t; r < 32; r += kExThreads) {  // global offset of tile bits 8..12 of j = 256 r
        uint64_t g = 0;
        for (int q = 8; q < kExMaxM; ++q)
            if ((r << 8) >> q & 1) g |= uint64_t(1) << a.tile_pos[q];
        gR[r] = g;
    }
    const int nnib = (a.nouter + 3) / 4;
    for (int i = t; i < nnib * 16; i += kExThreads) {  // offsets (code: block offsets) of the tile number's nibbles
        uint64_t g = 0;
        for (int b = 0; b < 4; ++b) {
            const int o = 4 * (i >> 4) + b;
            if ((i >> b & 1) && o < a.nouter) g |= uint64_t(1) << (a.outer_pos[o] - (ENC ? kEncBlockLog2 : 0));
        }
        tO[i >> 4][i & 15] = g;
    }
    if (ENC)
        for (int u = t; u < 256; u += kExThreads) {
            const int q = int((signed char)u);
            const int aq = q < 0 ? -q : q;
            const float f = __fdiv_rn(float(aq > 127 ? 127 : aq), 127.0f);
            tab[u] = q < 0 ? -f : f;
        }
    uint64_t gT = 0;  // global offset of tile bits 0..7 (= t)
    for (int q = 0; q < 8; ++q)
        if (t >> q & 1) gT |= uint64_t(1) << a.tile_pos[q];
    uint64_t boff[4] = {0, 0, 0, 0};  // code: block offsets of this warp's in-tile blocks
    if (ENC)
        for (int i = 0; i < 4; ++i)
            for (int q = 0; q < 5; ++q)
                if ((warp + kExWarps * i) >> q & 1) boff[i] |= uint64_t(1) << (a.tile_pos[kEncBlockLog2 + q] - kEncBlockLog2);
    __syncthreads();
    const float2 *psi = static_cast<const float2 *>(data);
    const int4 *codes = static_cast<const int4 *>(data);
    EncRaw raw;
    uint64_t cta = blockIdx.x;
    if (cta < a.ntiles) {
        if (ENC)
            enc_fetch(codes, scales, tile_base(tO, nnib, cta), boff, lane, raw);
        else
            c64_issue(psi, sm, tile_base(tO, nnib, cta), gT, gR, t);
    }
    float cV = 0.f, cE = 0.f, cO = 0.f;
    double dV = 0.0, dE = 0.0, dO = 0.0;
    int cnt = 0;
    for (; cta < a.ntiles; cta += gridDim.x) {
        const uint64_t next = cta + gridDim.x;
        if (ENC)
            enc_decode(raw, sm, tab, warp, lane);
        else
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
        float2 x[32];
        float T1 = 0.f, T2 = 0.f;
        // segment 1: tile bits 8..12 in registers (j = t | r << 8)
#pragma unroll
        for (int r = 0; r < 32; ++r) x[r] = sm[xswz(uint32_t(t | (r << 8)))];
        if (kSegs == 1) __syncthreads();
        seg_pairs<5>(x, v + 8, v + 24);
        if (FIRST) {
            T1 = seg_total(x);
            v[13] = lane_signed(T1, lane, 0);
            v[14] = lane_signed(T1, lane, 1);
            v[15] = lane_signed(T1, lane, 2);
            v[29] = lane_signed(T1, lane, 3);
            v[30] = lane_signed(T1, lane, 4);
        }
        if (kSegs >= 2) {  // segment 2: tile bits 3..7 (j = (t & 7) | r << 3 | (t >> 3) << 8)
#pragma unroll
            for (int r = 0; r < 32; ++r) x[r] = sm[xswz(uint32_t((t & 7) | (r << 3) | ((t >> 3) << 8)))];
            if (kSegs == 2) {
                __syncthreads();
                if (!ENC && next < a.ntiles) c64_issue(psi, sm, tile_base(tO, nnib, next), gT, gR, t);
            }
            seg_pairs<5>(x, v + 3, v + 19);
            if (FIRST) {
                T2 = seg_total(x);
                v[31] = lane_signed(T2, lane, 3);
            }
        }
        if (kSegs == 3) {  // segment 3: tile bits 0..2 (j = r | t << 5; bits 3, 4 were segment 2's)
#pragma unroll
            for (int i = 3; i < 16; ++i) rs_pair<16>(v, lane, i);
#pragma unroll
            for (int r = 0; r < 32; ++r) x[r] = sm[xswz(uint32_t(r | (t << 5)))];
            __syncthreads();
            if (!ENC && next < a.ntiles) c64_issue(psi, sm, tile_base(tO, nnib, next), gT, gR, t);
            seg_pairs<3>(x, v + 0, v + 16);
#pragma unroll
            for (int i = 0; i < 3; ++i) rs_pair<16>(v, lane, i);
        } else {
            rs_step<16>(v, lane);
        }
        if (ENC && next < a.ntiles) enc_fetch(codes, scales, tile_base(tO, nnib, next), boff, lane, raw);
        float e0 = 0.f, e1 = 0.f, e2 = 0.f;
        if (FIRST) {
            e0 = warp_sum(T1);
            e1 = warp_sum(T2);
            e2 = warp_sum(lane_signed(T2, lane, 4));
        }
        rs_step<8>(v, lane);
        rs_step<4>(v, lane);
        rs_step<2>(v, lane);
        rs_step<1>(v, lane);
        cV += v[0];
        if (FIRST) {
            cE += lane == 0 ? e0 : (lane == 1 ? e1 : (lane == 2 ? e2 : 0.f));
            if (lane < a.nouter) cO += ((cta >> lane) & 1ull) ? -e0 : e0;
        }
        if (++cnt == kExChunk) {
            dV += double(cV);
            dE += double(cE);
            dO += double(cO);
            cV = cE = cO = 0.f;
            cnt = 0;
        }
    }
    dV += double(cV);
    dE += double(cE);
    dO += double(cO);
    wsum[warp][lane] = dV;
    if (lane < 3) wsum[warp][32 + lane] = dE;
    wsum[warp][35 + lane] = dO;  // zero where lane >= nouter
    __syncthreads();
    if (t < kExVals) {
        double s = 0.0;
        if (t < 3 * kExMaxM) {
            const int k = t / 3, c = t % 3;
            for (int w = 0; w < kExWarps; ++w) {
                double u;
                if (c == 0)
                    u = 2.0 * wsum[w][k];
                else if (c == 1)
                    u = 2.0 * wsum[w][16 + k];
                else if (!FIRST)
                    u = 0.0;
                else if (k < 3)
                    u = wsum[w][13 + k];
                else if (k < 5)
                    u = wsum[w][26 + k];
                else if (k < 8)
                    u = (w >> (k - 5) & 1) ? -wsum[w][32] : wsum[w][32];
                else if (k == 8)
                    u = wsum[w][31];
                else if (k == 9)
                    u = wsum[w][34];
                else
                    u = (w >> (k - 10) & 1) ? -wsum[w][33] : wsum[w][33];
                s += u;
            }
        } else {
            const int o = t - 3 * kExMaxM;
            if (FIRST && o < 32)
                for (int w = 0; w < kExWarps; ++w) s += wsum[w][35 + o];
        }
        partials[size_t(blockIdx.x) * kExVals + t] = s;
    }
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" sv_status sv_expect_pauli(sv_handle h, double *out) {
    if (!h || !h->data) {
        set_error("NULL handle");
        return SV_ERR_ARG;
    }
    if (!out) {
        set_error("out is NULL");
        return SV_ERR_ARG;
    }
    const int n = h->n;
    const bool enc = h->dt == SV_ENC2B;
    const int m = std::min(n, h->dt == SV_C128 ? 12 : kExMaxM);
    // Qubits every tile keeps (whole code blocks; runs of 2^low amplitudes).
    // The later passes of the 13-bit kernel skip tile bits 0..2 (complex64)
    // or 0..7 (code), so those must be low ones.  Three low qubits make 64-byte
    // runs of complex64 and ten new qubits per pass (three passes at 32 qubits).
    const char *low_env = std::getenv("SV_EXPECT_LOW");
    const int low_c = low_env ? std::max(3, std::min(8, std::atoi(low_env))) : 3;
    const int low = enc ? std::min(n, kEncBlockLog2) : std::min(n, low_c);
    if (n - m > kExMaxOuter) {
        set_error("n = %d is beyond the expectation kernel's %d outer qubits", n, kExMaxOuter);
        return SV_ERR_UNSUPPORTED;
    }
    int sms = 0;
    SV_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    const uint64_t ntiles = uint64_t(1) << (n - m);
    const unsigned grid = unsigned(std::min<uint64_t>(ntiles, uint64_t(2) * uint64_t(sms)));
    const size_t elem = h->dt == SV_C128 ? 16 : 8;
    const size_t smem = (size_t(1) << m) * elem;
    {
        static std::atomic<uint64_t> configured{0};
        if (attrs_needed(configured, h->device)) {
            const int big = (1 << kExMaxM) * 8;  // the largest tile: 64 KiB
            SV_CUDA_TRY(cudaFuncSetAttribute(k_expect<float2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
            SV_CUDA_TRY(cudaFuncSetAttribute(k_expect<double2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
            SV_CUDA_TRY(cudaFuncSetAttribute(k_expect<float2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
            SV_CUDA_TRY(cudaFuncSetAttribute(k_expect13<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
            SV_CUDA_TRY(cudaFuncSetAttribute(k_expect13<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
            SV_CUDA_TRY(cudaFuncSetAttribute(k_expect13<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
            SV_CUDA_TRY(cudaFuncSetAttribute(k_expect13<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
            attrs_set(configured, h->device);
        }
    }
    // The passes' tile sets depend only on which qubits earlier passes
    // covered: plan them all, launch them back to back into one partials
    // buffer, copy it once.
    std::vector<std::vector<int>> tiles;
    {
        std::vector<char> covered(size_t(n), 0);
        for (int pass = 0;; ++pass) {
            // tile qubits: all low ones first, then the low ones plus uncovered ones
            std::vector<int> tile;
            for (int q = 0; q < (pass == 0 ? m : low); ++q) tile.push_back(q);
            for (int q = 0; q < n && int(tile.size()) < m; ++q)
                if (!covered[size_t(q)] && std::find(tile.begin(), tile.end(), q) == tile.end()) tile.push_back(q);
            if (pass > 0 && int(tile.size()) == low) break;  // nothing left to cover
            for (int q : tile) covered[size_t(q)] = 1;
            for (int q = 0; q < n && int(tile.size()) < m; ++q)
                if (std::find(tile.begin(), tile.end(), q) == tile.end()) tile.push_back(q);
            std::sort(tile.begin(), tile.end());
            tiles.push_back(tile);
        }
    }
    const size_t per_pass = size_t(kExVals) * grid;
    if (h->expect_cap < per_pass * tiles.size()) {  // handle scratch, grown on demand
        if (h->d_expect) SV_CUDA_TRY(cudaFree(h->d_expect));
        h->d_expect = nullptr;
        h->expect_cap = 0;
        SV_CUDA_TRY(cudaMalloc(&h->d_expect, sizeof(double) * per_pass * tiles.size()));
        h->expect_cap = per_pass * tiles.size();
    }
    double *d_part = h->d_expect;
    sv_status s = SV_OK;
    for (size_t pass = 0; pass < tiles.size() && s == SV_OK; ++pass) {
        const std::vector<int> &tile = tiles[pass];
        ExpArgs a{};
        a.n = n;
        a.m = m;
        a.zouter = pass == 0;
        a.ntiles = ntiles;
        for (int k = 0; k < m; ++k) a.tile_pos[k] = uint8_t(tile[size_t(k)]);
        for (int q = 0; q < n; ++q)
            if (std::find(tile.begin(), tile.end(), q) == tile.end()) a.outer_pos[a.nouter++] = uint8_t(q);
        const void *data = h->data;
        double *dp = d_part + per_pass * pass;
        if (h->dt != SV_C128 && m == kExMaxM && a.nouter <= 32) {  // register segments (complex64, codes)
            if (h->dt == SV_C64) {
                if (pass == 0)
                    k_expect13<false, true><<<grid, kExThreads, smem, h->stream>>>(data, nullptr, a, dp);
                else
                    k_expect13<false, false><<<grid, kExThreads, smem, h->stream>>>(data, nullptr, a, dp);
            } else if (pass == 0) {
                k_expect13<true, true><<<grid, kExThreads, smem, h->stream>>>(data, h->scales, a, dp);
            } else {
                k_expect13<true, false><<<grid, kExThreads, smem, h->stream>>>(data, h->scales, a, dp);
            }
        } else if (h->dt == SV_C64)
            k_expect<float2, false><<<grid, kExThreads, smem, h->stream>>>(data, nullptr, a, dp);
        else if (h->dt == SV_C128)
            k_expect<double2, false><<<grid, kExThreads, smem, h->stream>>>(data, nullptr, a, dp);
        else
            k_expect<float2, true><<<grid, kExThreads, smem, h->stream>>>(data, h->scales, a, dp);
        s = check_launch(cudaGetLastError(), "sv_expect_pauli");
    }
    std::vector<double> part(per_pass * tiles.size());
    if (s == SV_OK) {
        const cudaError_t e = cudaMemcpyAsync(part.data(), d_part, sizeof(double) * part.size(),
                                              cudaMemcpyDeviceToHost, h->stream);
        s = e != cudaSuccess ? cuda_status(e, "cudaMemcpyAsync") : sync_stream(h->stream, "sv_expect_pauli");
    }
    if (s) return s;
    // x, y of a qubit from the first pass that has it in its tile, z from pass 0
    std::vector<double> x(size_t(n), 0.0), y(size_t(n), 0.0), z(size_t(n), 0.0);
    std::vector<char> covered(size_t(n), 0);
    for (size_t pass = 0; pass < tiles.size(); ++pass) {
        const double *pp = part.data() + per_pass * pass;
        const std::vector<int> &tile = tiles[pass];
        for (int k = 0; k < m; ++k) {
            const int q = tile[size_t(k)];
            if (covered[size_t(q)] && pass > 0) continue;
            double sx = 0, sy = 0, sz = 0;
            for (unsigned b = 0; b < grid; ++b) {
                sx += pp[size_t(b) * kExVals + 3 * k];
                sy += pp[size_t(b) * kExVals + 3 * k + 1];
                sz += pp[size_t(b) * kExVals + 3 * k + 2];
            }
            x[size_t(q)] = sx;
            y[size_t(q)] = sy;
            covered[size_t(q)] = 1;
            if (pass == 0) z[size_t(q)] = sz;
        }
        if (pass == 0) {
            int o = 0;
            for (int q = 0; q < n; ++q) {
                if (std::find(tile.begin(), tile.end(), q) != tile.end()) continue;
                double sz = 0;
                for (unsigned b = 0; b < grid; ++b) sz += pp[size_t(b) * kExVals + 3 * kExMaxM + o];
                z[size_t(q)] = sz;
                ++o;
            }
        }
    }
    for (int q = 0; q < n; ++q) {
        out[3 * q] = x[size_t(q)];
        out[3 * q + 1] = y[size_t(q)];
        out[3 * q + 2] = z[size_t(q)];
    }
    return SV_OK;
}
