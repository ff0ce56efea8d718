// Dense k-qubit block on the CUDA cores (Sec. 2: a gate on k qubits is a
// 2^k x 2^k matrix acting on the 2^k amplitudes that differ only in those
// qubits).  complex128 runs it in FP64; complex64 in FP32.
//
// A CTA stages kGroupAmps amplitudes (kGroupAmps / 2^k groups) in shared
// memory together with the matrix, each thread computes a few output
// amplitudes as row-times-group dot products, and the CTA writes the groups
// back in place.
#include "plan.h"

namespace sv {
namespace {

template <typename R>
struct C2 {
    R re, im;
};

constexpr int kThreads = 256;
constexpr int kGroupAmps = 1024;

struct FusedArgs {
    int n, k;
    int sorted[kMaxFusedQubits];   // ascending qubit positions
    uint64_t off[1 << kMaxFusedQubits];  // index offset of local index l
    uint64_t ngroups;
};

__device__ __forceinline__ uint64_t insert_zero(uint64_t x, int p) {
    const uint64_t lo = x & ((uint64_t(1) << p) - 1);
    return ((x ^ lo) << 1) | lo;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_fused_dense(C2<R> *__restrict__ psi, const C2<double> *__restrict__ U,
                                                          FusedArgs a) {
    extern __shared__ unsigned char smem_raw[];
    const int d = 1 << a.k;
    C2<R> *um = reinterpret_cast<C2<R> *>(smem_raw);  // d*d
    C2<R> *xs = um + d * d;                            // kGroupAmps
    for (int i = threadIdx.x; i < d * d; i += blockDim.x) um[i] = C2<R>{R(U[i].re), R(U[i].im)};
    const int gpb = kGroupAmps / d;  // groups per batch (>= 16 since d <= 64)
    for (uint64_t g0 = uint64_t(blockIdx.x) * gpb; g0 < a.ngroups; g0 += uint64_t(gridDim.x) * gpb) {
        __syncthreads();
        for (int i = threadIdx.x; i < kGroupAmps; i += blockDim.x) {
            const int gl = i / d, l = i % d;
            const uint64_t g = g0 + gl;
            if (g < a.ngroups) {
                uint64_t base = g;
                for (int j = 0; j < a.k; ++j) base = insert_zero(base, a.sorted[j]);
                xs[i] = psi[base | a.off[l]];
            }
        }
        __syncthreads();
        C2<R> res[kGroupAmps / kThreads];
#pragma unroll
        for (int r = 0; r < kGroupAmps / kThreads; ++r) {
            const int i = threadIdx.x + r * kThreads;
            const int gl = i / d, row = i % d;
            R re = 0, im = 0;
            for (int col = 0; col < d; ++col) {
                const C2<R> u = um[row * d + col], x = xs[gl * d + col];
                re += u.re * x.re - u.im * x.im;
                im += u.re * x.im + u.im * x.re;
            }
            res[r] = C2<R>{re, im};
        }
#pragma unroll
        for (int r = 0; r < kGroupAmps / kThreads; ++r) {
            const int i = threadIdx.x + r * kThreads;
            const int gl = i / d, row = i % d;
            const uint64_t g = g0 + gl;
            if (g < a.ngroups) {
                uint64_t base = g;
                for (int j = 0; j < a.k; ++j) base = insert_zero(base, a.sorted[j]);
                psi[base | a.off[row]] = res[r];
            }
        }
    }
}

}  // namespace

cudaError_t launch_fused(sv_state *h, int k, const int *qubits, const double *U) {
    if (fused_tc_supported(h)) return launch_fused_tc(h, k, qubits, U);
    const int d = 1 << k;
    if (!h->d_mat) {
        cudaError_t e = cudaMalloc(&h->d_mat, sizeof(C2<double>) << (2 * kMaxFusedQubits));
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemcpyAsync(h->d_mat, U, sizeof(C2<double>) * d * d, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return e;
    FusedArgs a{};
    a.n = h->n;
    a.k = k;
    for (int j = 0; j < k; ++j) a.sorted[j] = qubits[j];
    for (int i = 1; i < k; ++i)
        for (int j = i; j > 0 && a.sorted[j - 1] > a.sorted[j]; --j) {
            const int t = a.sorted[j];
            a.sorted[j] = a.sorted[j - 1];
            a.sorted[j - 1] = t;
        }
    for (int l = 0; l < d; ++l) {
        uint64_t o = 0;
        for (int j = 0; j < k; ++j)
            if (l >> j & 1) o |= uint64_t(1) << qubits[j];
        a.off[l] = o;
    }
    a.ngroups = uint64_t(1) << (h->n - k);
    const int gpb = kGroupAmps / d;
    uint64_t blocks = (a.ngroups + gpb - 1) / gpb;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const C2<double> *um = static_cast<const C2<double> *>(h->d_mat);
    if (h->dt == SV_C64) {
        const size_t sm = sizeof(C2<float>) * (size_t(d) * d + kGroupAmps);
        k_fused_dense<float><<<int(blocks), kThreads, sm, h->stream>>>(static_cast<C2<float> *>(h->data), um, a);
    } else {
        const size_t sm = sizeof(C2<double>) * (size_t(d) * d + kGroupAmps);
        if (sm > 48 * 1024) {
            e = cudaFuncSetAttribute(k_fused_dense<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
            if (e != cudaSuccess) return e;
        }
        k_fused_dense<double><<<int(blocks), kThreads, sm, h->stream>>>(static_cast<C2<double> *>(h->data), um, a);
    }
    return cudaGetLastError();
}

}  // namespace sv
