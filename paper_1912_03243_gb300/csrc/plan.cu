// Plan creation and replay.
#include "plan.h"

namespace sv {

double gate1_bytes(const sv_state *h, const Gate1 &g) {
    const double amps = double(uint64_t(1) << h->n);
    if (h->dt == SV_ENC2B) {
        const double nb = h->n < kEncBlockLog2 ? 1.0 : amps / kEncBlock;
        const double frac = g.control >= 0 ? 0.5 : 1.0;
        return frac * (2.0 * amps * 2.0 + 2.0 * nb * 4.0);
    }
    const double s = h->dt == SV_C64 ? 8.0 : 16.0;
    const bool diag = g.u[1].re == 0 && g.u[1].im == 0 && g.u[2].re == 0 && g.u[2].im == 0;
    const bool unit00 = g.u[0].re == 1 && g.u[0].im == 0;
    double frac = (diag && unit00) ? 0.5 : 1.0;
    if (g.control >= 0) frac *= 0.5;
    return 2.0 * amps * s * frac;
}

}  // namespace sv

using namespace sv;

extern "C" {

sv_status sv_plan_create(sv_handle h, const char *text, int mode, sv_plan *out) {
    if (!out) {
        set_error("out is NULL");
        return SV_ERR_ARG;
    }
    *out = nullptr;
    if (!h || !h->data) {
        set_error("NULL handle");
        return SV_ERR_ARG;
    }
    if (mode != SV_MODE_PERGATE && mode != SV_MODE_TILED && mode != SV_MODE_FUSED) {
        set_error("unknown mode %d", mode);
        return SV_ERR_ARG;
    }
    if (h->dt == SV_ENC2B && mode != SV_MODE_PERGATE) {
        set_error("the two-byte code runs one decode-gate-encode pass per gate (SV_MODE_PERGATE)");
        return SV_ERR_DTYPE;
    }
    Circuit c;
    sv_status s = parse_circuit(text, h->n, &c);
    if (s) return s;
    sv_plan_s *p = new sv_plan_s;
    p->h = h;
    p->mode = mode;
    p->gates = int64_t(c.instrs.size());
    if (mode == SV_MODE_PERGATE) {
        p->pergate = lower_to_gate1(c);
        for (const Gate1 &g : p->pergate) p->bytes += gate1_bytes(h, g);
    } else {
        delete p;
        set_error("mode %d is not available yet", mode);
        return SV_ERR_UNSUPPORTED;
    }
    h->live_plans++;
    *out = p;
    return SV_OK;
}

sv_status sv_plan_execute(sv_plan p) {
    if (!p) {
        set_error("NULL plan");
        return SV_ERR_ARG;
    }
    for (const Gate1 &g : p->pergate) {
        sv_status s = check_launch(launch_gate1(p->h, g), "sv_plan_execute");
        if (s) return s;
    }
    return SV_OK;
}

sv_status sv_plan_info(sv_plan p, int64_t *gates, int64_t *passes, double *bytes) {
    if (!p) {
        set_error("NULL plan");
        return SV_ERR_ARG;
    }
    if (gates) *gates = p->gates;
    if (passes) *passes = int64_t(p->pergate.size());
    if (bytes) *bytes = p->bytes;
    return SV_OK;
}

sv_status sv_plan_execute_timed(sv_plan p, void *const *events, int64_t n_events) {
    if (!p || !events) {
        set_error("NULL argument");
        return SV_ERR_ARG;
    }
    const int64_t passes = int64_t(p->pergate.size());
    if (n_events < passes + 1) {
        set_error("need %lld events, got %lld", (long long)(passes + 1), (long long)n_events);
        return SV_ERR_ARG;
    }
    for (int64_t i = 0; i < passes; ++i) {
        cudaError_t e = cudaEventRecord(static_cast<cudaEvent_t>(events[i]), p->h->stream);
        if (e != cudaSuccess) return cuda_status(e, "cudaEventRecord");
        sv_status s = check_launch(launch_gate1(p->h, p->pergate[size_t(i)]), "sv_plan_execute_timed");
        if (s) return s;
    }
    cudaError_t e = cudaEventRecord(static_cast<cudaEvent_t>(events[passes]), p->h->stream);
    if (e != cudaSuccess) return cuda_status(e, "cudaEventRecord");
    return SV_OK;
}

sv_status sv_plan_free(sv_plan p) {
    if (!p) return SV_OK;
    if (p->h) p->h->live_plans--;
    delete p;
    return SV_OK;
}

}  // extern "C"
