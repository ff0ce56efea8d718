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
// tile number's bits.  Persistent CTAs accumulate per tile in FP32 (FP64 for
// complex128) and across tiles in FP64; the host adds the CTAs' partials.
#include <algorithm>
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

// Register bits 0..NB-1 are tile bits B0..: for each, (Re, Im) of conj(p) q
// over the pairs (packed FMAs: p.x (q.x, q.y) + p.y (q.y, -q.x)) into
// v[3k], v[3k+1], and the probability of the registers with the bit set into
// v[3k+2] (<sigma^z> = P - 2 P1 follows in the block sum).
template <int B0, int NB>
__device__ __forceinline__ void reg_pairs(const float2 (&x)[32], float (&v)[3 * kExMaxM + 1], bool total) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        unsigned long long xy = pk2(v[3 * (B0 + b)], v[3 * (B0 + b) + 1]);
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            if (r >> b & 1) continue;
            const float2 p = x[r], q = x[r | (1 << b)];
            xy = fma2(pk2(p.x, p.x), pk2(q.x, q.y), xy);
            xy = fma2(pk2(p.y, p.y), pk2(q.y, -q.x), xy);
        }
        upk2(xy, v[3 * (B0 + b)], v[3 * (B0 + b) + 1]);
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const float pr = x[r].x * x[r].x + x[r].y * x[r].y;
        if (total) v[3 * kExMaxM] += pr;
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (r >> b & 1) v[3 * (B0 + b) + 2] += pr;
    }
}

template <bool ENC>
__global__ void __launch_bounds__(kExThreads, 2) k_expect13(const void *__restrict__ data,
                                                            const float *__restrict__ scales, const ExpArgs a,
                                                            double *__restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *sm = reinterpret_cast<float2 *>(smem);
    __shared__ double acc[kExVals];
    __shared__ float red[kExWarps][3 * kExMaxM + 1];
    __shared__ uint64_t gR[32];
    __shared__ float tab[256];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int i = t; i < kExVals; i += kExThreads) acc[i] = 0.0;
    for (int r = t; r < 32; r += kExThreads) {  // global offset of tile bits 8..12 of j = 256 r
        uint64_t g = 0;
        for (int q = 8; q < kExMaxM; ++q)
            if ((r << 8) >> q & 1) g |= uint64_t(1) << a.tile_pos[q];
        gR[r] = g;
    }
    for (int u = t; u < 256; u += kExThreads) {
        const int q = int((signed char)u);
        const int aq = q < 0 ? -q : q;
        const float f = __fdiv_rn(float(aq > 127 ? 127 : aq), 127.0f);
        tab[u] = q < 0 ? -f : f;
    }
    uint64_t gT = 0;  // global offset of tile bits 0..7 (= t)
    for (int q = 0; q < 8; ++q)
        if (t >> q & 1) gT |= uint64_t(1) << a.tile_pos[q];
    __syncthreads();
    for (uint64_t cta = blockIdx.x; cta < a.ntiles; cta += gridDim.x) {
        if (!ENC) {
            const float2 *psi = static_cast<const float2 *>(data);
            uint64_t base = 0;
            for (int o = 0; o < a.nouter; ++o) base |= ((cta >> o) & 1ull) << a.outer_pos[o];
            // all 32 copies in flight (cp.async, 8 bytes each)
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const uint32_t sa = uint32_t(__cvta_generic_to_shared(sm + xswz(uint32_t(t | (r << 8)))));
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(psi + (base | gT | gR[r]))
                             : "memory");
            }
            asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
        } else {
            const int4 *codes = static_cast<const int4 *>(data);
            uint64_t bbase = 0;
            for (int o = 0; o < a.nouter; ++o) bbase |= ((cta >> o) & 1ull) << (a.outer_pos[o] - kEncBlockLog2);
            for (int bl = warp; bl < 32; bl += kExWarps) {
                uint64_t b = bbase;
                for (int q = 0; q < 5; ++q)
                    if (bl >> q & 1) b |= uint64_t(1) << (a.tile_pos[kEncBlockLog2 + q] - kEncBlockLog2);
                const int4 raw = codes[b * 32 + lane];
                const float sc = scales[b];
                const uint32_t w[4] = {uint32_t(raw.x), uint32_t(raw.y), uint32_t(raw.z), uint32_t(raw.w)};
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint32_t word = w[e >> 1], sh = (e & 1) * 16;
                    sm[xswz(uint32_t((bl << kEncBlockLog2) | (lane * 8 + e)))] =
                        make_float2(__fmul_rn(sc, tab[(word >> sh) & 0xFFu]), __fmul_rn(sc, tab[(word >> (sh + 8)) & 0xFFu]));
                }
            }
        }
        __syncthreads();
        float v[3 * kExMaxM + 1];
#pragma unroll
        for (int i = 0; i < 3 * kExMaxM + 1; ++i) v[i] = 0.0f;
        float2 x[32];
        // tile bits 8..12 in registers (j = t | r << 8); the tile's probability
#pragma unroll
        for (int r = 0; r < 32; ++r) x[r] = sm[xswz(uint32_t(t | (r << 8)))];
        reg_pairs<8, 5>(x, v, true);
        // tile bits 3..7 (j = (t & 7) | r << 3 | (t >> 3) << 8)
#pragma unroll
        for (int r = 0; r < 32; ++r) x[r] = sm[xswz(uint32_t((t & 7) | (r << 3) | ((t >> 3) << 8)))];
        reg_pairs<3, 5>(x, v, false);
        // tile bits 0..2 (j = r | t << 5; register bits 3, 4 were done above)
#pragma unroll
        for (int r = 0; r < 32; ++r) x[r] = sm[xswz(uint32_t(r | (t << 5)))];
        reg_pairs<0, 3>(x, v, false);
#pragma unroll
        for (int i = 0; i < 3 * kExMaxM + 1; ++i) {
            float s = v[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) red[warp][i] = s;
        }
        __syncthreads();
        if (t < 3 * kExMaxM) {
            double s = 0.0;
            for (int w = 0; w < kExWarps; ++w) s += double(red[w][t]);
            if (t % 3 == 2) {  // P - 2 P1
                double P = 0.0;
                for (int w = 0; w < kExWarps; ++w) P += double(red[w][3 * kExMaxM]);
                acc[t] += P - 2.0 * s;
            } else {
                acc[t] += 2.0 * s;
            }
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
    const int low = enc ? std::min(n, kEncBlockLog2) : std::min(n, 4);  // qubits every tile keeps
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
        static bool configured = false;
        if (!configured) {
            const int big = (1 << kExMaxM) * 8;  // the largest tile: 64 KiB
            SV_CUDA_TRY(cudaFuncSetAttribute(k_expect<float2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
            SV_CUDA_TRY(cudaFuncSetAttribute(k_expect<double2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
            SV_CUDA_TRY(cudaFuncSetAttribute(k_expect<float2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
            SV_CUDA_TRY(cudaFuncSetAttribute(k_expect13<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
            SV_CUDA_TRY(cudaFuncSetAttribute(k_expect13<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
            configured = true;
        }
    }
    double *d_part = nullptr;
    SV_CUDA_TRY(cudaMalloc(&d_part, sizeof(double) * kExVals * grid));
    std::vector<double> part(size_t(kExVals) * grid);
    std::vector<double> x(size_t(n), 0.0), y(size_t(n), 0.0), z(size_t(n), 0.0);
    std::vector<char> covered(size_t(n), 0);
    sv_status s = SV_OK;
    for (int pass = 0; s == SV_OK; ++pass) {
        // tile qubits: all low ones first, then the low ones plus uncovered ones
        std::vector<int> tile;
        for (int q = 0; q < (pass == 0 ? m : low); ++q) tile.push_back(q);
        for (int q = 0; q < n && int(tile.size()) < m; ++q)
            if (!covered[size_t(q)] && std::find(tile.begin(), tile.end(), q) == tile.end()) tile.push_back(q);
        if (pass > 0 && int(tile.size()) == low) break;  // nothing left to cover
        for (int q = 0; q < n && int(tile.size()) < m; ++q)
            if (std::find(tile.begin(), tile.end(), q) == tile.end()) tile.push_back(q);
        std::sort(tile.begin(), tile.end());
        ExpArgs a{};
        a.n = n;
        a.m = m;
        a.zouter = pass == 0;
        a.ntiles = ntiles;
        for (int k = 0; k < m; ++k) a.tile_pos[k] = uint8_t(tile[size_t(k)]);
        for (int q = 0; q < n; ++q)
            if (std::find(tile.begin(), tile.end(), q) == tile.end()) a.outer_pos[a.nouter++] = uint8_t(q);
        const void *data = h->data;
        if (h->dt != SV_C128 && m == kExMaxM) {  // register segments (complex64, codes)
            if (h->dt == SV_C64)
                k_expect13<false><<<grid, kExThreads, smem, h->stream>>>(data, nullptr, a, d_part);
            else
                k_expect13<true><<<grid, kExThreads, smem, h->stream>>>(data, h->scales, a, d_part);
        } else if (h->dt == SV_C64)
            k_expect<float2, false><<<grid, kExThreads, smem, h->stream>>>(data, nullptr, a, d_part);
        else if (h->dt == SV_C128)
            k_expect<double2, false><<<grid, kExThreads, smem, h->stream>>>(data, nullptr, a, d_part);
        else
            k_expect<float2, true><<<grid, kExThreads, smem, h->stream>>>(data, h->scales, a, d_part);
        s = check_launch(cudaGetLastError(), "sv_expect_pauli");
        if (s) break;
        cudaError_t e = cudaMemcpyAsync(part.data(), d_part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost,
                                        h->stream);
        if (e != cudaSuccess) {
            s = cuda_status(e, "cudaMemcpyAsync");
            break;
        }
        s = sync_stream(h->stream, "sv_expect_pauli");
        if (s) break;
        for (int k = 0; k < m; ++k) {
            const int q = tile[size_t(k)];
            double sx = 0, sy = 0, sz = 0;
            for (unsigned b = 0; b < grid; ++b) {
                sx += part[size_t(b) * kExVals + 3 * k];
                sy += part[size_t(b) * kExVals + 3 * k + 1];
                sz += part[size_t(b) * kExVals + 3 * k + 2];
            }
            if (!covered[size_t(q)]) {
                x[size_t(q)] = sx;
                y[size_t(q)] = sy;
                covered[size_t(q)] = 1;
            }
            if (pass == 0) z[size_t(q)] = sz;
        }
        if (pass == 0)
            for (int o = 0; o < a.nouter; ++o) {
                double sz = 0;
                for (unsigned b = 0; b < grid; ++b) sz += part[size_t(b) * kExVals + 3 * kExMaxM + o];
                z[a.outer_pos[o]] = sz;
            }
    }
    cudaFree(d_part);
    if (s) return s;
    for (int q = 0; q < n; ++q) {
        out[3 * q] = x[size_t(q)];
        out[3 * q + 1] = y[size_t(q)];
        out[3 * q + 2] = z[size_t(q)];
    }
    return SV_OK;
}
