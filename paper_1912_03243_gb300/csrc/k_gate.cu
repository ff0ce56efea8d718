// Per-gate kernels: one HBM pass applies one (controlled) single-qubit update
// (Eq. 1) to the whole state.  These are the "plain" per-gate path and the
// building block every other mode is checked against.
//
// Access pattern.  Amplitudes are moved as 16-byte vectors: two complex64
// amplitudes (float4) or one complex128 amplitude (double2).  For a target
// qubit above the vector width the two partners of a pair sit in two
// different vectors 2^(t-W) vectors apart and each thread streams several
// such vector pairs (UNR) so enough bytes are in flight per SM; for the
// complex64 target qubit 0 the pair is inside one float4.  A control qubit
// above the vector width is folded into the work index (only the half with
// the control set is read); a control inside the vector is a per-lane test.
// Diagonal gates with u00 = 1 (T, S, Z, P, CZ, CP) read and write only the
// amplitudes they change.
#include "sv_internal.h"

namespace sv {
namespace {

template <typename R>
struct VecT;
template <>
struct VecT<float> {
    using T = float4;
    static constexpr int W = 1;  // log2 amplitudes per vector
};
template <>
struct VecT<double> {
    using T = double2;
    static constexpr int W = 0;
};

template <typename R>
struct C2 {
    R re, im;
};

template <typename R>
struct GateArgs {
    uint64_t nwork;       // work items
    uint64_t tbit;        // vector-index bit of the target (across kernel)
    uint64_t set_mask;    // vector-index bits forced to 1 (controls, phase mask)
    int ins[3];           // ascending vector-index positions where zero bits are inserted
    int nins;
    int lane_mask;        // amplitude-within-vector bits that must be 1 (W = 1 only)
    R u[8];               // 2x2 row-major (re, im)
};

__device__ __forceinline__ uint64_t insert_zero(uint64_t x, int p) {
    const uint64_t lo = x & ((uint64_t(1) << p) - 1);
    return ((x ^ lo) << 1) | lo;
}

template <typename R>
__device__ __forceinline__ uint64_t expand(uint64_t w, const GateArgs<R> &a) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (k < a.nins) w = insert_zero(w, a.ins[k]);
    return w | a.set_mask;
}

template <typename R>
__device__ __forceinline__ void apply2(const R *u, R &ar, R &ai, R &br, R &bi) {
    const R nar = u[0] * ar - u[1] * ai + u[2] * br - u[3] * bi;
    const R nai = u[0] * ai + u[1] * ar + u[2] * bi + u[3] * br;
    const R nbr = u[4] * ar - u[5] * ai + u[6] * br - u[7] * bi;
    const R nbi = u[4] * ai + u[5] * ar + u[6] * bi + u[7] * br;
    ar = nar;
    ai = nai;
    br = nbr;
    bi = nbi;
}

constexpr int kUnr = 4;
constexpr int kThreads = 256;

// Pair across two vectors (target >= W).
template <typename R>
__global__ void __launch_bounds__(kThreads) k_gate_across(typename VecT<R>::T *__restrict__ v, GateArgs<R> a) {
    using V = typename VecT<R>::T;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t base = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; base < a.nwork; base += stride * kUnr) {
        V x[kUnr], y[kUnr];
        uint64_t i0[kUnr];
#pragma unroll
        for (int k = 0; k < kUnr; ++k) {
            const uint64_t w = base + k * stride;
            if (w < a.nwork) {
                i0[k] = expand(w, a);
                x[k] = v[i0[k]];
                y[k] = v[i0[k] | a.tbit];
            }
        }
#pragma unroll
        for (int k = 0; k < kUnr; ++k) {
            const uint64_t w = base + k * stride;
            if (w < a.nwork) {
                if constexpr (VecT<R>::W == 1) {
                    if (!(a.lane_mask & 1)) apply2(a.u, x[k].x, x[k].y, y[k].x, y[k].y);
                    apply2(a.u, x[k].z, x[k].w, y[k].z, y[k].w);
                } else {
                    apply2(a.u, x[k].x, x[k].y, y[k].x, y[k].y);
                }
                v[i0[k]] = x[k];
                v[i0[k] | a.tbit] = y[k];
            }
        }
    }
}

// complex64 target qubit 0: the pair is the two halves of one float4.
__global__ void __launch_bounds__(kThreads) k_gate_inner(float4 *__restrict__ v, GateArgs<float> a) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t base = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; base < a.nwork; base += stride * kUnr) {
        float4 x[kUnr];
        uint64_t i0[kUnr];
#pragma unroll
        for (int k = 0; k < kUnr; ++k) {
            const uint64_t w = base + k * stride;
            if (w < a.nwork) {
                i0[k] = expand(w, a);
                x[k] = v[i0[k]];
            }
        }
#pragma unroll
        for (int k = 0; k < kUnr; ++k) {
            const uint64_t w = base + k * stride;
            if (w < a.nwork) {
                apply2(a.u, x[k].x, x[k].y, x[k].z, x[k].w);
                v[i0[k]] = x[k];
            }
        }
    }
}

// Diagonal gate with u00 = 1: multiply the amplitudes whose masked bits are
// all set by u11.  Vectors are enumerated with the vector-level mask bits
// forced to 1; lane_mask selects amplitudes inside a float4.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_phase(typename VecT<R>::T *__restrict__ v, GateArgs<R> a) {
    using V = typename VecT<R>::T;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const R pr = a.u[6], pi = a.u[7];
    for (uint64_t base = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; base < a.nwork; base += stride * kUnr) {
        V x[kUnr];
        uint64_t i0[kUnr];
#pragma unroll
        for (int k = 0; k < kUnr; ++k) {
            const uint64_t w = base + k * stride;
            if (w < a.nwork) {
                i0[k] = expand(w, a);
                x[k] = v[i0[k]];
            }
        }
#pragma unroll
        for (int k = 0; k < kUnr; ++k) {
            const uint64_t w = base + k * stride;
            if (w < a.nwork) {
                if constexpr (VecT<R>::W == 1) {
                    if (!(a.lane_mask & 1)) {
                        const R r = x[k].x * pr - x[k].y * pi, i = x[k].x * pi + x[k].y * pr;
                        x[k].x = r;
                        x[k].y = i;
                    }
                    const R r = x[k].z * pr - x[k].w * pi, i = x[k].z * pi + x[k].w * pr;
                    x[k].z = r;
                    x[k].w = i;
                } else {
                    const R r = x[k].x * pr - x[k].y * pi, i = x[k].x * pi + x[k].y * pr;
                    x[k].x = r;
                    x[k].y = i;
                }
                v[i0[k]] = x[k];
            }
        }
    }
}

int grid_for(uint64_t nwork) {
    uint64_t b = (nwork + uint64_t(kThreads) * kUnr - 1) / (uint64_t(kThreads) * kUnr);
    if (b < 1) b = 1;
    const uint64_t cap = 152ull * 32;
    return int(b < cap ? b : cap);
}

void sort_small(int *p, int n) {
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && p[j - 1] > p[j]; --j) {
            int t = p[j];
            p[j] = p[j - 1];
            p[j - 1] = t;
        }
}

template <typename R>
cudaError_t gate1_impl(sv_state *h, const Gate1 &g) {
    using V = typename VecT<R>::T;
    constexpr int W = VecT<R>::W;
    GateArgs<R> a{};
    for (int k = 0; k < 4; ++k) {
        a.u[2 * k] = R(g.u[k].re);
        a.u[2 * k + 1] = R(g.u[k].im);
    }
    const int n = h->n;
    const int nv_log = n - W;  // log2 number of vectors
    V *v = static_cast<V *>(h->data);
    const bool diag = g.u[1].re == 0 && g.u[1].im == 0 && g.u[2].re == 0 && g.u[2].im == 0;
    const bool unit00 = g.u[0].re == 1 && g.u[0].im == 0;
    const int t = g.target, c = g.control;
    if (diag && unit00) {
        // phase on amplitudes with bit t (and bit c) set
        int ins[2], ni = 0;
        uint64_t setm = 0;
        int lane = 0;
        for (int b : {t, c}) {
            if (b < 0) continue;
            if (b >= W) {
                ins[ni++] = b - W;
                setm |= uint64_t(1) << (b - W);
            } else {
                lane |= 1 << b;
            }
        }
        sort_small(ins, ni);
        for (int k = 0; k < ni; ++k) a.ins[k] = ins[k];
        a.nins = ni;
        a.set_mask = setm;
        a.lane_mask = lane;
        a.nwork = uint64_t(1) << (nv_log - ni);
        k_phase<R><<<grid_for(a.nwork), kThreads, 0, h->stream>>>(v, a);
        return cudaGetLastError();
    }
    int ins[2], ni = 0;
    uint64_t setm = 0;
    int lane = 0;
    if (c >= 0) {
        if (c >= W) {
            ins[ni++] = c - W;
            setm |= uint64_t(1) << (c - W);
        } else {
            lane |= 1 << c;
        }
    }
    if (t >= W) {
        ins[ni++] = t - W;
        a.tbit = uint64_t(1) << (t - W);
    }
    sort_small(ins, ni);
    for (int k = 0; k < ni; ++k) a.ins[k] = ins[k];
    a.nins = ni;
    a.set_mask = setm;
    a.lane_mask = lane;
    a.nwork = uint64_t(1) << (nv_log - ni);
    if (t >= W) {
        k_gate_across<R><<<grid_for(a.nwork), kThreads, 0, h->stream>>>(v, a);
    } else {
        if constexpr (W == 1) {
            k_gate_inner<<<grid_for(a.nwork), kThreads, 0, h->stream>>>(reinterpret_cast<float4 *>(v), a);
        }
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- set basis
template <typename R>
__global__ void k_set_one(C2<R> *psi, uint64_t idx) {
    psi[idx].re = R(1);
    psi[idx].im = R(0);
}

__global__ void k_enc_set_one(char2 *codes, float *scales, uint64_t idx) {
    codes[idx] = make_char2(127, 0);
    scales[idx >> kEncBlockLog2] = 1.0f;
}

// ---------------------------------------------------------------- norm
constexpr int kNormBlocks = 152 * 8;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v) {
    __shared__ double sh[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) v = warp_sum(v);
    return v;
}

// complex64: 8 squares (two float4) summed in FP32, then accumulated in FP64.
__global__ void __launch_bounds__(256) k_norm_c64(const float4 *__restrict__ v, uint64_t npairs, uint64_t nvec,
                                                  double *__restrict__ partials) {
    double acc = 0.0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < npairs; i += stride) {
        const float4 x = v[2 * i], y = v[2 * i + 1];
        float s = x.x * x.x;
        s = fmaf(x.y, x.y, s);
        s = fmaf(x.z, x.z, s);
        s = fmaf(x.w, x.w, s);
        s = fmaf(y.x, y.x, s);
        s = fmaf(y.y, y.y, s);
        s = fmaf(y.z, y.z, s);
        s = fmaf(y.w, y.w, s);
        acc += double(s);
    }
    // odd vector count (n = 1): the last float4
    if (blockIdx.x == 0 && threadIdx.x == 0 && (nvec & 1)) {
        const float4 x = v[nvec - 1];
        acc += double(x.x) * x.x + double(x.y) * x.y + double(x.z) * x.z + double(x.w) * x.w;
    }
    const double b = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

__global__ void __launch_bounds__(256) k_norm_c128(const double2 *__restrict__ v, uint64_t namps,
                                                   double *__restrict__ partials) {
    double acc = 0.0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < namps; i += stride) {
        const double2 x = v[i];
        acc = fma(x.x, x.x, acc);
        acc = fma(x.y, x.y, acc);
    }
    const double b = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

// Fixed-order final reduction of the block partials (deterministic).
__global__ void __launch_bounds__(256) k_norm_final(const double *__restrict__ partials, int np, double *out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
    const double b = block_sum(acc);
    if (threadIdx.x == 0) *out = b;
}

// ---------------------------------------------------------------- gather
template <typename R>
__global__ void k_gather(const C2<R> *__restrict__ psi, const uint64_t *__restrict__ idx, size_t m,
                         double2 *__restrict__ out) {
    for (size_t j = size_t(blockIdx.x) * blockDim.x + threadIdx.x; j < m; j += size_t(gridDim.x) * blockDim.x) {
        const C2<R> a = psi[idx[j]];
        out[j] = make_double2(double(a.re), double(a.im));
    }
}

}  // namespace

int norm_partials_needed(const sv_state *) { return kNormBlocks; }

const char *gate1_kernel_name(const sv_state *h, const Gate1 &g) {
    if (h->dt == SV_ENC2B) {
        auto is = [](const Cplx &z, double re) { return z.re == re && z.im == 0.0; };
        const Cplx *u = g.u;
        if (h->n >= kEncBlockLog2) {
            if (is(u[1], 0) && is(u[2], 0) && (is(u[0], 1) || is(u[0], -1)) && (is(u[3], 1) || is(u[3], -1)))
                return "k_enc_flip";
            if (is(u[0], 0) && is(u[3], 0) && is(u[1], 1) && is(u[2], 1)) {
                if (g.target < kEncBlockLog2) return "k_enc_xin";
                if (g.control < 0 || g.control >= kEncBlockLog2) return "k_enc_xblocks";
            }
        }
        if (g.target < kEncBlockLog2 || h->n < kEncBlockLog2) return "k_enc_gate_in";
        // diagonal with u00 = 1 in the FP32 entries the kernels use: only the upper blocks
        auto zero32 = [](const Cplx &z) { return float(z.re) == 0.0f && float(z.im) == 0.0f; };
        if (zero32(u[1]) && zero32(u[2]) && float(u[0].re) == 1.0f && float(u[0].im) == 0.0f)
            return "k_enc_phase_blocks";
        return "k_enc_gate_across";
    }
    const bool diag = g.u[1].re == 0 && g.u[1].im == 0 && g.u[2].re == 0 && g.u[2].im == 0;
    const bool unit00 = g.u[0].re == 1 && g.u[0].im == 0;
    const bool c64 = h->dt == SV_C64;
    if (diag && unit00) return c64 ? "k_phase<f32>" : "k_phase<f64>";
    if (c64 && g.target == 0) return "k_gate_inner<f32>";
    return c64 ? "k_gate_across<f32>" : "k_gate_across<f64>";
}

cudaError_t launch_gate1(sv_state *h, const Gate1 &g) {
    if (h->dt == SV_C64) return gate1_impl<float>(h, g);
    if (h->dt == SV_C128) return gate1_impl<double>(h, g);
    return launch_enc_gate1(h, g);
}

cudaError_t launch_set_basis(sv_state *h, uint64_t idx) {
    cudaError_t e = cudaMemsetAsync(h->data, 0, h->bytes, h->stream);
    if (e != cudaSuccess) return e;
    if (h->dt == SV_C64)
        k_set_one<float><<<1, 1, 0, h->stream>>>(static_cast<C2<float> *>(h->data), idx);
    else if (h->dt == SV_C128)
        k_set_one<double><<<1, 1, 0, h->stream>>>(static_cast<C2<double> *>(h->data), idx);
    else
        k_enc_set_one<<<1, 1, 0, h->stream>>>(static_cast<char2 *>(h->data), h->scales, idx);
    return cudaGetLastError();
}

cudaError_t launch_norm(sv_state *h, double *d_out) {
    const uint64_t namps = uint64_t(1) << h->n;
    if (h->dt == SV_C64) {
        const uint64_t nvec = namps / 2 ? namps / 2 : 1;
        k_norm_c64<<<kNormBlocks, 256, 0, h->stream>>>(static_cast<const float4 *>(h->data), nvec / 2, nvec,
                                                       h->d_partials);
    } else if (h->dt == SV_C128) {
        k_norm_c128<<<kNormBlocks, 256, 0, h->stream>>>(static_cast<const double2 *>(h->data), namps,
                                                        h->d_partials);
    } else {
        return cudaErrorInvalidValue;  // encoded norm goes through launch_enc_norm
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_norm_final<<<1, 256, 0, h->stream>>>(h->d_partials, kNormBlocks, d_out);
    return cudaGetLastError();
}

cudaError_t launch_gather(sv_state *h, const uint64_t *d_idx, size_t m, double *d_out) {
    if (m == 0) return cudaSuccess;
    const int blocks = int((m + 255) / 256 < 1024 ? (m + 255) / 256 : 1024);
    if (h->dt == SV_C64)
        k_gather<float><<<blocks, 256, 0, h->stream>>>(static_cast<const C2<float> *>(h->data), d_idx, m,
                                                       reinterpret_cast<double2 *>(d_out));
    else if (h->dt == SV_C128)
        k_gather<double><<<blocks, 256, 0, h->stream>>>(static_cast<const C2<double> *>(h->data), d_idx, m,
                                                        reinterpret_cast<double2 *>(d_out));
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace sv
