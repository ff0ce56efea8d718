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

__device__ __forceinline__ uint64_t insert_zero(uint64_t x, int p) {
    const uint64_t lo = x & ((uint64_t(1) << p) - 1);
    return ((x ^ lo) << 1) | lo;
}

// Table T[k] = fl(k/127) replicated per bank: tab[k * 32 + lane].
__device__ __forceinline__ void load_table(float *tab) {
    for (int i = threadIdx.x; i < 128 * 32; i += blockDim.x) tab[i] = __fdiv_rn(float(i >> 5), 127.0f);
    __syncthreads();
}

__device__ __forceinline__ float dec1(int q, float s, const float *tab, int lane) {
    const int a = q < 0 ? -q : q;
    const float v = __fmul_rn(s, tab[a * 32 + lane]);
    return q < 0 ? -v : v;
}

__device__ __forceinline__ signed char enc1(float x, float inv) {
    int r = __float2int_rn(__fmul_rn(x, inv));
    r = r > 127 ? 127 : (r < -127 ? -127 : r);
    return (signed char)r;
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

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

struct Lane8 {
    float re[8], im[8];
};

__device__ __forceinline__ void decode_lane(const int4 raw, float s, const float *tab, int lane, Lane8 &x) {
    const signed char *b = reinterpret_cast<const signed char *>(&raw);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        x.re[j] = dec1(b[2 * j], s, tab, lane);
        x.im[j] = dec1(b[2 * j + 1], s, tab, lane);
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
    int4 raw;
    signed char *b = reinterpret_cast<signed char *>(&raw);
    if (s == 0.0f) {
        raw = make_int4(0, 0, 0, 0);
        return raw;
    }
    const float inv = __fdiv_rn(127.0f, s);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        b[2 * j] = enc1(x.re[j], inv);
        b[2 * j + 1] = enc1(x.im[j], inv);
    }
    return raw;
}

// Does amplitude j of this lane (in-block index lane*8 + j) satisfy the control?
__device__ __forceinline__ bool ctl_ok(int c, int lane, int j) {
    if (c < 0 || c >= kEncBlockLog2) return true;
    const int idx = lane * 8 + j;
    return (idx >> c) & 1;
}

// Target inside the block (t < 8).
__global__ void __launch_bounds__(32 * kWarpsPerCta) k_enc_gate_in(int4 *__restrict__ codes, float *__restrict__ scales,
                                                                   EncGateArgs a) {
    __shared__ float tab[128 * 32];
    load_table(tab);
    const int lane = threadIdx.x & 31;
    const uint64_t wid = uint64_t(blockIdx.x) * kWarpsPerCta + (threadIdx.x >> 5);
    const uint64_t nw = uint64_t(gridDim.x) * kWarpsPerCta;
    for (uint64_t w = wid; w < a.nwork; w += nw) {
        uint64_t b = w;
        for (int k = 0; k < a.nins; ++k) b = insert_zero(b, a.ins[k]);
        b |= a.set_mask;
        int4 raw = codes[b * 32 + lane];
        const float s = scales[b];
        Lane8 x;
        decode_lane(raw, s, tab, lane, x);
        if (a.t < 3) {
            const int tb = 1 << a.t;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j & tb) continue;
                if (!ctl_ok(a.c, lane, j)) continue;
                gate_pair(a.u, x.re[j], x.im[j], x.re[j | tb], x.im[j | tb]);
            }
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
                gate_pair(a.u, ar, ai, br, bi);
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
__global__ void __launch_bounds__(32 * kWarpsPerCta) k_enc_gate_across(int4 *__restrict__ codes,
                                                                       float *__restrict__ scales, EncGateArgs a) {
    __shared__ float tab[128 * 32];
    load_table(tab);
    const int lane = threadIdx.x & 31;
    const uint64_t wid = uint64_t(blockIdx.x) * kWarpsPerCta + (threadIdx.x >> 5);
    const uint64_t nw = uint64_t(gridDim.x) * kWarpsPerCta;
    for (uint64_t w = wid; w < a.nwork; w += nw) {
        uint64_t b0 = w;
        for (int k = 0; k < a.nins; ++k) b0 = insert_zero(b0, a.ins[k]);
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
            gate_pair(a.u, x.re[j], x.im[j], y.re[j], y.im[j]);
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
        codes[2 * i] = m == 0.0f ? 0 : enc1(re[i], inv);
        codes[2 * i + 1] = m == 0.0f ? 0 : enc1(im[i], inv);
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
    __shared__ float tab[128 * 32];
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
        codes[2 * i] = m == 0.0f ? 0 : enc1(psi[i].x, inv);
        codes[2 * i + 1] = m == 0.0f ? 0 : enc1(psi[i].y, inv);
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
    if (a.t < kEncBlockLog2)
        k_enc_gate_in<<<enc_grid(a.nwork), 32 * kWarpsPerCta, 0, h->stream>>>(codes, h->scales, a);
    else
        k_enc_gate_across<<<enc_grid(a.nwork), 32 * kWarpsPerCta, 0, h->stream>>>(codes, h->scales, a);
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
    __shared__ float tab[128 * 32];
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
