// Amplitude gather that allocates nothing (sv_amplitudes_noalloc).
//
// sv_amplitudes needs a handle, and creating a handle (sv_alloc, sv_attach)
// allocates the handle's device scratch with cudaMalloc.  Some callers cannot
// do that: a host framework whose own allocator owns all device memory, a
// process that has reserved nearly all of HBM for its state, or a latency-
// critical loop that must not run into cudaMalloc's implicit device-wide
// synchronisation or its failure under memory pressure.  This entry point
// works on a raw device pointer to the state and keeps its scratch (the index
// list and the gathered values) in a fixed file-scope device array instead.
//
// The array is sized for kNoAllocMaxAmps indices (24 B each: 1.5 MiB) and,
// like every file-scope __device__ variable, occupies memory on every GPU
// that loads the library until the process exits.  All calls share it.
#include <cuda.h>  // driver types for cuMemGetAddressRange (fetched at run time, not linked)

#include <mutex>

#include "sv_internal.h"

namespace sv {
namespace {

constexpr size_t kNoAllocMaxAmps = 65536;

// [kNoAllocMaxAmps uint64 indices][kNoAllocMaxAmps double2 outputs]
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocMaxAmps * (sizeof(uint64_t) + 2 * sizeof(double))];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, once per device, with that device current.
sv_status scratch_for_current_device(unsigned char **out) {
    int dev = -1;
    SV_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d out of range", dev);
        return SV_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return SV_OK;
}

// cuMemGetAddressRange, looked up once through the runtime (the library links
// only the static runtime); nullptr if the driver does not offer it.
typedef CUresult (*AddrRangeFn)(CUdeviceptr *, size_t *, CUdeviceptr);
AddrRangeFn addr_range_fn() {
    static const AddrRangeFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<AddrRangeFn>(p);
    }();
    return fn;
}

// Host-side checks of the caller's state pointer, before anything touches
// it: aligned for the widest access the gather makes, device memory of the
// current device, and (where the driver reports the allocation's extent)
// large enough for the whole n-qubit layout.  None of these calls allocates.
sv_status check_state_pointer(const void *state, int n, sv_dtype dt) {
    const size_t align = dt == SV_C128 ? 16 : 8;
    if (reinterpret_cast<uintptr_t>(state) % align) {
        set_error("state pointer %p is not %zu-byte aligned", state, align);
        return SV_ERR_ARG;
    }
    int dev = -1;
    SV_CUDA_TRY(cudaGetDevice(&dev));
    cudaPointerAttributes attr{};
    const cudaError_t e = cudaPointerGetAttributes(&attr, state);
    if (e != cudaSuccess) {
        cudaGetLastError();  // an invalid pointer is the caller's error, not a sticky one
        set_error("state pointer %p is not device memory (%s)", state, cudaGetErrorString(e));
        return SV_ERR_ARG;
    }
    if (attr.type != cudaMemoryTypeDevice) {
        set_error("state pointer %p is not device memory (memory type %d)", state, int(attr.type));
        return SV_ERR_ARG;
    }
    if (attr.device != dev) {
        set_error("state pointer %p belongs to device %d, the current device is %d", state, attr.device, dev);
        return SV_ERR_ARG;
    }
    if (AddrRangeFn fn = addr_range_fn()) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (fn(&base, &size, CUdeviceptr(reinterpret_cast<uintptr_t>(state))) == CUDA_SUCCESS) {
            const size_t need = sv_bytes_required(n, dt);
            const size_t avail = size_t(base + size - CUdeviceptr(reinterpret_cast<uintptr_t>(state)));
            if (need > avail) {
                set_error("an n=%d state of dtype %d needs %zu bytes, the allocation holds %zu from %p", n, int(dt),
                          need, avail, state);
                return SV_ERR_ARG;
            }
        }
    }
    return SV_OK;
}

__device__ __forceinline__ float dec_code(int q, float s) {
    const float v = __fmul_rn(s, __fdiv_rn(float(q < 0 ? -q : q), 127.0f));
    return q < 0 ? -v : v;
}

// One thread per requested index; reads the index list and writes the
// values in the static scratch.
__global__ void k_gather_noalloc(const void *__restrict__ state, int n, int dt, const uint64_t *__restrict__ idx,
                                 size_t m, double2 *__restrict__ out) {
    for (size_t j = size_t(blockIdx.x) * blockDim.x + threadIdx.x; j < m; j += size_t(gridDim.x) * blockDim.x) {
        const uint64_t i = idx[j];
        if (dt == SV_C64) {
            const float2 a = static_cast<const float2 *>(state)[i];
            out[j] = make_double2(a.x, a.y);
        } else if (dt == SV_C128) {
            out[j] = static_cast<const double2 *>(state)[i];
        } else {
            const char2 q = static_cast<const char2 *>(state)[i];
            const float *scales = reinterpret_cast<const float *>(static_cast<const char *>(state) + (size_t(2) << n));
            const float s = scales[n < kEncBlockLog2 ? 0 : (i >> kEncBlockLog2)];
            out[j] = make_double2(dec_code(q.x, s), dec_code(q.y, s));
        }
    }
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" sv_status sv_amplitudes_noalloc(const void *state, int n, sv_dtype dt, size_t m, const uint64_t *idx,
                                           double *out, void *stream) {
    if (!state || n < 1 || n > kMaxQubits || (dt != SV_C64 && dt != SV_C128 && dt != SV_ENC2B)) {
        set_error("bad state pointer, n=%d or dtype=%d", n, int(dt));
        return SV_ERR_ARG;
    }
    if (m == 0) return SV_OK;
    if (!idx || !out) {
        set_error("NULL idx/out");
        return SV_ERR_ARG;
    }
    if (m > kNoAllocMaxAmps) {
        set_error("sv_amplitudes_noalloc gathers at most %zu amplitudes per call (got %zu); split the request",
                  kNoAllocMaxAmps, m);
        return SV_ERR_ARG;
    }
    for (size_t j = 0; j < m; ++j)
        if (idx[j] >> n) {
            set_error("index %llu at position %zu >= 2^%d", (unsigned long long)idx[j], j, n);
            return SV_ERR_ARG;
        }
    sv_status s = check_state_pointer(state, n, dt);
    if (s) return s;
    unsigned char *scratch = nullptr;
    s = scratch_for_current_device(&scratch);
    if (s) return s;
    uint64_t *d_idx = reinterpret_cast<uint64_t *>(scratch);
    double2 *d_out = reinterpret_cast<double2 *>(scratch + kNoAllocMaxAmps * sizeof(uint64_t));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Every output slot the copy-back reads is written by the kernel first, so
    // nothing in the shared array needs clearing between calls.
    SV_CUDA_TRY(cudaMemcpyAsync(d_idx, idx, m * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    const int blocks = int((m + 255) / 256 < 256 ? (m + 255) / 256 : 256);
    k_gather_noalloc<<<blocks, 256, 0, st>>>(state, n, int(dt), d_idx, m, d_out);
    s = check_launch(cudaGetLastError(), "sv_amplitudes_noalloc");
    if (s) return s;
    SV_CUDA_TRY(cudaMemcpyAsync(out, d_out, m * 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    return sync_stream(st, "sv_amplitudes_noalloc");
}
