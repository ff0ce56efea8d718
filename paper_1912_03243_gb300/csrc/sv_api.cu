// C ABI of libsv: argument checks, handle lifecycle, dispatch to kernels.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "plan.h"
#include "sv_internal.h"

namespace sv {

namespace {
thread_local std::string g_err;
}

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

sv_status cuda_status(cudaError_t e, const char *what) {
    set_error("CUDA error in %s: %s (%d)", what, cudaGetErrorString(e), int(e));
    return SV_ERR_CUDA;
}

bool fault_injected(const char *what) {
    const char *v = std::getenv("SV_FAULT_INJECT");
    return v && std::strcmp(v, what) == 0;
}

cudaError_t ensure_err_word(sv_state *h) {
    if (h->d_err) return cudaSuccess;
    cudaError_t e = cudaMalloc(&h->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(int));
    return e;
}

sv_status check_launch(cudaError_t e, const char *what) {
    if (fault_injected("launch")) {
        set_error("injected launch failure in %s", what);
        return SV_ERR_CUDA;
    }
    if (e != cudaSuccess) return cuda_status(e, what);
    return SV_OK;
}

sv_status sync_stream(cudaStream_t st, const char *what) {
    if (fault_injected("sync")) {
        set_error("injected synchronisation failure in %s", what);
        return SV_ERR_CUDA;
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, what);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, what);
    return SV_OK;
}

namespace {

// After a successful synchronisation: report (and clear) a bounded device
// wait that gave up.
sv_status check_device_error(sv_state *h) {
    if (!h->d_err) return SV_OK;
    int v = 0;
    SV_CUDA_TRY(cudaMemcpy(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (v == 0) return SV_OK;
    SV_CUDA_TRY(cudaMemset(h->d_err, 0, sizeof(int)));
    set_error("a device-side wait timed out; the state is undefined");
    return sv_status(v);
}

sv_status sync_handle(sv_state *h, const char *what) {
    sv_status s = sync_stream(h->stream, what);
    return s ? s : check_device_error(h);
}

sv_status check_handle(sv_handle h) {
    if (!h) {
        set_error("NULL handle");
        return SV_ERR_ARG;
    }
    if (!h->data) {
        set_error("handle has no storage");
        return SV_ERR_STATE;
    }
    return SV_OK;
}

sv_status init_scratch(sv_state *h) {
    const int np = norm_partials_needed(h) + 1;
    SV_CUDA_TRY(cudaMalloc(&h->d_partials, sizeof(double) * np));
    h->partials_cap = np;
    return SV_OK;
}

sv_status ensure_gather(sv_state *h, size_t m) {
    if (m <= h->gather_cap) return SV_OK;
    if (h->d_idx) cudaFree(h->d_idx);
    if (h->d_amps) cudaFree(h->d_amps);
    h->d_idx = nullptr;
    h->d_amps = nullptr;
    h->gather_cap = 0;
    SV_CUDA_TRY(cudaMalloc(&h->d_idx, sizeof(uint64_t) * m));
    SV_CUDA_TRY(cudaMalloc(&h->d_amps, 2 * sizeof(double) * m));
    h->gather_cap = m;
    return SV_OK;
}

bool valid_n(int n) { return n >= 1 && n <= kMaxQubits; }

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" {

const char *sv_last_error(void) { return g_err.c_str(); }

const char *sv_version(void) { return "libsv 0.1 (sm_103a)"; }

size_t sv_bytes_required(int n, sv_dtype dt) {
    if (!valid_n(n)) return 0;
    const size_t amps = size_t(1) << n;
    switch (dt) {
        case SV_C64: return amps * 8;
        case SV_C128: return amps * 16;
        case SV_ENC2B: {
            const size_t nb = n < kEncBlockLog2 ? 1 : amps >> kEncBlockLog2;
            return amps * 2 + nb * sizeof(float);
        }
    }
    return 0;
}

int sv_num_qubits(sv_handle h) { return h ? h->n : -1; }
int sv_dtype_of(sv_handle h) { return h ? int(h->dt) : -1; }

static sv_status finish_init(sv_state *h) {
    SV_CUDA_TRY(cudaGetDevice(&h->device));
    if (h->dt == SV_ENC2B) h->scales = reinterpret_cast<float *>(static_cast<char *>(h->data) + (size_t(2) << h->n));
    return init_scratch(h);
}

sv_status sv_alloc(int n, sv_dtype dt, void *stream, sv_handle *out) {
    if (!out) {
        set_error("out is NULL");
        return SV_ERR_ARG;
    }
    *out = nullptr;
    if (!valid_n(n) || (dt != SV_C64 && dt != SV_C128 && dt != SV_ENC2B)) {
        set_error("bad n=%d or dtype=%d", n, int(dt));
        return SV_ERR_ARG;
    }
    const size_t bytes = sv_bytes_required(n, dt);
    if (fault_injected("alloc")) {
        set_error("injected allocation failure (%zu bytes)", bytes);
        return SV_ERR_OOM;
    }
    size_t free_b = 0, total_b = 0;
    SV_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    if (bytes + (size_t(64) << 20) > free_b) {
        set_error("state needs %zu bytes, %zu free", bytes, free_b);
        return SV_ERR_OOM;
    }
    sv_state *h = new sv_state;
    h->n = n;
    h->dt = dt;
    h->bytes = bytes;
    h->owned = true;
    h->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMalloc(&h->data, bytes);
    if (e != cudaSuccess) {
        delete h;
        set_error("cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA;
    }
    sv_status s = finish_init(h);
    if (s == SV_OK) s = check_launch(launch_set_basis(h, 0), "sv_alloc");
    if (s != SV_OK) {
        sv_free(h);
        return s;
    }
    *out = h;
    return SV_OK;
}

sv_status sv_attach(int n, sv_dtype dt, void *dev_ptr, size_t bytes, void *stream, sv_handle *out) {
    if (!out || !dev_ptr) {
        set_error("NULL argument");
        return SV_ERR_ARG;
    }
    *out = nullptr;
    if (!valid_n(n) || (dt != SV_C64 && dt != SV_C128 && dt != SV_ENC2B)) {
        set_error("bad n=%d or dtype=%d", n, int(dt));
        return SV_ERR_ARG;
    }
    if (bytes < sv_bytes_required(n, dt)) {
        set_error("buffer of %zu bytes is smaller than the %zu required", bytes, sv_bytes_required(n, dt));
        return SV_ERR_ARG;
    }
    if (reinterpret_cast<uintptr_t>(dev_ptr) % 256) {
        set_error("buffer is not 256-byte aligned");
        return SV_ERR_ARG;
    }
    sv_state *h = new sv_state;
    h->n = n;
    h->dt = dt;
    h->bytes = sv_bytes_required(n, dt);
    h->owned = false;
    h->data = dev_ptr;
    h->stream = static_cast<cudaStream_t>(stream);
    sv_status s = finish_init(h);
    if (s != SV_OK) {
        sv_free(h);
        return s;
    }
    *out = h;
    return SV_OK;
}

sv_status sv_free(sv_handle h) {
    if (!h) return SV_OK;
    if (h->live_plans > 0) {
        set_error("handle still has %d live plans", h->live_plans);
        return SV_ERR_STATE;
    }
    cudaStreamSynchronize(h->stream);
    if (h->owned && h->data) cudaFree(h->data);
    if (h->d_partials) cudaFree(h->d_partials);
    if (h->d_idx) cudaFree(h->d_idx);
    if (h->d_amps) cudaFree(h->d_amps);
    if (h->d_mat) cudaFree(h->d_mat);
    if (h->d_err) cudaFree(h->d_err);
    if (h->d_expect) cudaFree(h->d_expect);
    delete h;
    return SV_OK;
}

sv_status sv_set_basis(sv_handle h, uint64_t idx) {
    sv_status s = check_handle(h);
    if (s) return s;
    if (idx >> h->n) {
        set_error("basis index %llu >= 2^%d", (unsigned long long)idx, h->n);
        return SV_ERR_ARG;
    }
    return check_launch(launch_set_basis(h, idx), "sv_set_basis");
}

sv_status sv_sync(sv_handle h) {
    sv_status s = check_handle(h);
    if (s) return s;
    return sync_handle(h, "sv_sync");
}

sv_status sv_apply_gate(sv_handle h, int target, int control, const double *U) {
    sv_status s = check_handle(h);
    if (s) return s;
    if (!U) {
        set_error("U is NULL");
        return SV_ERR_ARG;
    }
    if (target < 0 || target >= h->n || control < -1 || control >= h->n || control == target) {
        set_error("bad target %d / control %d for n=%d", target, control, h->n);
        return SV_ERR_ARG;
    }
    Gate1 g{};
    g.target = target;
    g.control = control;
    for (int k = 0; k < 4; ++k) g.u[k] = Cplx{U[2 * k], U[2 * k + 1]};
    return check_launch(launch_gate1(h, g), "sv_apply_gate");
}

sv_status sv_apply_fused(sv_handle h, int k, const int *qubits, const double *U) {
    sv_status s = check_handle(h);
    if (s) return s;
    if (!qubits || !U || k < 1 || k > kMaxFusedQubits || k > h->n) {
        set_error("bad fused gate (k=%d)", k);
        return SV_ERR_ARG;
    }
    uint64_t mask = 0;
    for (int j = 0; j < k; ++j) {
        if (qubits[j] < 0 || qubits[j] >= h->n || (mask >> qubits[j] & 1)) {
            set_error("bad or repeated qubit %d", qubits[j]);
            return SV_ERR_ARG;
        }
        mask |= uint64_t(1) << qubits[j];
    }
    if (h->dt == SV_ENC2B) {
        set_error("fused blocks are not defined on the two-byte code");
        return SV_ERR_DTYPE;
    }
    return check_launch(launch_fused(h, k, qubits, U), "sv_apply_fused");
}

sv_status sv_run_circuit(sv_handle h, const char *text, int mode) {
    sv_plan p = nullptr;
    sv_status s = sv_plan_create(h, text, mode, &p);
    if (s) return s;
    s = sv_plan_execute(p);
    const sv_status s2 = sv_plan_free(p);
    return s ? s : s2;
}

sv_status sv_encode2b(sv_handle src, sv_handle dst) {
    sv_status s = check_handle(src);
    if (!s) s = check_handle(dst);
    if (s) return s;
    if (src->dt != SV_C64 || dst->dt != SV_ENC2B) {
        set_error("sv_encode2b needs an SV_C64 source and an SV_ENC2B destination");
        return SV_ERR_DTYPE;
    }
    if (src->n != dst->n) {
        set_error("qubit counts differ (%d vs %d)", src->n, dst->n);
        return SV_ERR_ARG;
    }
    if (src->stream != dst->stream) {
        s = sync_stream(src->stream, "sv_encode2b");
        if (s) return s;
    }
    return check_launch(launch_encode(src, dst), "sv_encode2b");
}

sv_status sv_decode2b(sv_handle src, sv_handle dst) {
    sv_status s = check_handle(src);
    if (!s) s = check_handle(dst);
    if (s) return s;
    if (src->dt != SV_ENC2B || dst->dt != SV_C64) {
        set_error("sv_decode2b needs an SV_ENC2B source and an SV_C64 destination");
        return SV_ERR_DTYPE;
    }
    if (src->n != dst->n) {
        set_error("qubit counts differ (%d vs %d)", src->n, dst->n);
        return SV_ERR_ARG;
    }
    if (src->stream != dst->stream) {
        s = sync_stream(src->stream, "sv_decode2b");
        if (s) return s;
    }
    return check_launch(launch_decode(src, dst), "sv_decode2b");
}

sv_status sv_get_codes(sv_handle h, int8_t *codes, float *scales) {
    sv_status s = check_handle(h);
    if (s) return s;
    if (h->dt != SV_ENC2B) {
        set_error("sv_get_codes needs an SV_ENC2B state");
        return SV_ERR_DTYPE;
    }
    s = sync_handle(h, "sv_get_codes");
    if (s) return s;
    const size_t amps = size_t(1) << h->n;
    const size_t nb = h->n < kEncBlockLog2 ? 1 : amps >> kEncBlockLog2;
    if (codes) SV_CUDA_TRY(cudaMemcpy(codes, h->data, amps * 2, cudaMemcpyDeviceToHost));
    if (scales) SV_CUDA_TRY(cudaMemcpy(scales, h->scales, nb * sizeof(float), cudaMemcpyDeviceToHost));
    return SV_OK;
}

sv_status sv_amplitudes(sv_handle h, size_t m, const uint64_t *idx, double *out) {
    sv_status s = check_handle(h);
    if (s) return s;
    if (m == 0) return SV_OK;
    if (!idx || !out) {
        set_error("NULL idx/out");
        return SV_ERR_ARG;
    }
    for (size_t j = 0; j < m; ++j)
        if (idx[j] >> h->n) {
            set_error("index %llu at position %zu >= 2^%d", (unsigned long long)idx[j], j, h->n);
            return SV_ERR_ARG;
        }
    s = ensure_gather(h, m);
    if (s) return s;
    SV_CUDA_TRY(cudaMemcpyAsync(h->d_idx, idx, m * sizeof(uint64_t), cudaMemcpyHostToDevice, h->stream));
    s = check_launch(h->dt == SV_ENC2B ? launch_enc_gather(h, h->d_idx, m, h->d_amps)
                                       : launch_gather(h, h->d_idx, m, h->d_amps),
                     "sv_amplitudes");
    if (s) return s;
    SV_CUDA_TRY(cudaMemcpyAsync(out, h->d_amps, 2 * m * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return sync_handle(h, "sv_amplitudes");
}

sv_status sv_norm(sv_handle h, double *out) {
    sv_status s = check_handle(h);
    if (s) return s;
    if (!out) {
        set_error("out is NULL");
        return SV_ERR_ARG;
    }
    double *d_out = h->d_partials + (h->partials_cap - 1);
    s = check_launch(h->dt == SV_ENC2B ? launch_enc_norm(h, d_out) : launch_norm(h, d_out), "sv_norm");
    if (s) return s;
    SV_CUDA_TRY(cudaMemcpyAsync(out, d_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return sync_handle(h, "sv_norm");
}

sv_status sv_copy_to_host(sv_handle h, void *dst, size_t bytes) {
    sv_status s = check_handle(h);
    if (s) return s;
    if (!dst || bytes != h->bytes) {
        set_error("need a host buffer of exactly %zu bytes", h->bytes);
        return SV_ERR_ARG;
    }
    SV_CUDA_TRY(cudaMemcpyAsync(dst, h->data, bytes, cudaMemcpyDeviceToHost, h->stream));
    return sync_handle(h, "sv_copy_to_host");
}

sv_status sv_copy_from_host(sv_handle h, const void *src, size_t bytes) {
    sv_status s = check_handle(h);
    if (s) return s;
    if (!src || bytes != h->bytes) {
        set_error("need a host buffer of exactly %zu bytes", h->bytes);
        return SV_ERR_ARG;
    }
    SV_CUDA_TRY(cudaMemcpyAsync(h->data, src, bytes, cudaMemcpyHostToDevice, h->stream));
    return sync_handle(h, "sv_copy_from_host");
}

int sv_gate_matrix(const char *name, const double *params, int n_params, double *out) {
    if (!name || !out || n_params < 0 || n_params > 8) return -1;
    Cplx m[16];
    const int k = gate_matrix(name, params, n_params, m);
    if (k < 0) return -1;
    const int d = k == 1 ? 4 : 16;
    for (int i = 0; i < d; ++i) {
        out[2 * i] = m[i].re;
        out[2 * i + 1] = m[i].im;
    }
    return k;
}

}  // extern "C"
