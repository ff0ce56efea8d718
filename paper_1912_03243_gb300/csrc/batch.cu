// Many independent circuits of different sizes run together (the terms of
// Sec. 4 are independent; so are unrelated circuits): sv_batch_*.
//
// Each member circuit gets its own plan on its own state (tiled passes for
// n >= one tile, per-gate updates below that; the plans and their compiled
// passes come from the ordinary planner and its caches).  A small state fills
// only a few CTAs of a pass, so run one after another the members leave the
// GPU mostly idle and are launch-bound.  The batch instead captures all
// members into one CUDA graph in which every member is its own chain of
// launches (a branch forked from and joined to one stream): the chains have
// no edges between them, so the GPU runs the passes of different members at
// the same time, and one graph launch replays the whole batch.  Within a
// chain the passes keep their order (each reads what the previous wrote).
//
// The graph is captured on the second execution (the first runs the launches
// directly and does the plans' one-time set-up) and replayed afterwards.  It
// runs on a private stream (a handle's stream may be the legacy default
// stream, which cannot be captured); events join every member handle's
// stream to it before and after, so work already queued on those streams is
// ordered with the batch.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "plan.h"

struct sv_batch_s {
    std::vector<sv_handle> handles;
    std::vector<sv_plan> plans;
    std::vector<cudaStream_t> branch;      // one private stream per member (capture branches)
    std::vector<cudaStream_t> user;        // the distinct streams of the member handles
    std::vector<cudaEvent_t> ev;           // fork, joins, user-side events
    cudaStream_t main = nullptr;           // private: forks and joins the branches (capturable)
    cudaGraphExec_t gexec = nullptr;
    int64_t gates = 0, launches = 0;
    double bytes = 0.0;
    int64_t execs = 0;
};

namespace sv {
namespace {

void destroy_batch(sv_batch_s *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (sv_plan p : b->plans)
        if (p) sv_plan_free(p);
    for (cudaStream_t s : b->branch)
        if (s) cudaStreamDestroy(s);
    if (b->main) cudaStreamDestroy(b->main);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    delete b;
}

// Run every member's launches on its branch stream, forked from and joined
// to the main stream (direct launches, or recorded into the graph being
// captured on the main stream).
cudaError_t launch_members(sv_batch_s *b) {
    const size_t n = b->plans.size();
    cudaEvent_t fork = b->ev[0];
    cudaError_t e = cudaEventRecord(fork, b->main);
    for (size_t k = 0; k < n && e == cudaSuccess; ++k) {
        sv_plan_s *p = b->plans[k];
        e = cudaStreamWaitEvent(b->branch[k], fork, 0);
        if (e != cudaSuccess) break;
        const cudaStream_t own = p->h->stream;
        p->h->stream = b->branch[k];  // the plan's launches go on the handle's stream
        e = plan_launch_all(p);
        p->h->stream = own;
        if (e == cudaSuccess) e = cudaEventRecord(b->ev[1 + k], b->branch[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->ev[1 + k], 0);
    }
    return e;
}

cudaError_t capture(sv_batch_s *b) {
    cudaError_t e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t le = launch_members(b);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->main, &g);
    e = le != cudaSuccess ? le : ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0ULL);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess && b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return e;
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" sv_status sv_batch_create(const sv_handle *handles, const char *const *texts, int count, sv_batch *out) {
    if (!out) {
        set_error("out is NULL");
        return SV_ERR_ARG;
    }
    *out = nullptr;
    if (!handles || !texts || count < 1 || count > 4096) {
        set_error("bad batch (count = %d)", count);
        return SV_ERR_ARG;
    }
    for (int k = 0; k < count; ++k) {
        if (!handles[k] || !handles[k]->data || !texts[k]) {
            set_error("member %d: NULL handle or circuit", k);
            return SV_ERR_ARG;
        }
        if (handles[k]->dt == SV_ENC2B) {
            set_error("member %d: the two-byte code is not batched", k);
            return SV_ERR_DTYPE;
        }
        if (handles[k]->device != handles[0]->device) {
            set_error("member %d is on device %d, member 0 on %d", k, handles[k]->device, handles[0]->device);
            return SV_ERR_ARG;
        }
        for (int j = 0; j < k; ++j)
            if (handles[j] == handles[k] || handles[j]->data == handles[k]->data) {
                set_error("members %d and %d share a state", j, k);
                return SV_ERR_ARG;
            }
    }
    sv_batch_s *b = new sv_batch_s;
    sv_status s = SV_OK;
    for (int k = 0; k < count && s == SV_OK; ++k) {
        sv_plan p = nullptr;
        s = sv_plan_create(handles[k], texts[k], SV_MODE_TILED, &p);
        if (s) break;
        b->handles.push_back(handles[k]);
        b->plans.push_back(p);
        if (!plan_capturable(p)) {
            set_error("member %d: its plan copies host data between launches", k);
            s = SV_ERR_UNSUPPORTED;
            break;
        }
        b->gates += p->gates;
        b->launches += int64_t(p->launches.size());
        b->bytes += p->bytes;
        if (std::find(b->user.begin(), b->user.end(), handles[k]->stream) == b->user.end())
            b->user.push_back(handles[k]->stream);
    }
    cudaError_t e = s == SV_OK ? cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) : cudaSuccess;
    for (int k = 0; k < count && s == SV_OK && e == cudaSuccess; ++k) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        b->branch.push_back(st);
    }
    // events: the fork, one join per member, one per distinct user stream
    const size_t nev = 1 + size_t(count) + b->user.size();
    for (size_t i = 0; i < nev && s == SV_OK && e == cudaSuccess; ++i) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        b->ev.push_back(ev);
    }
    if (s == SV_OK && e != cudaSuccess) s = cuda_status(e, "sv_batch_create");
    if (s) {
        destroy_batch(b);
        return s;
    }
    *out = b;
    return SV_OK;
}

extern "C" sv_status sv_batch_execute(sv_batch b) {
    if (!b) {
        set_error("NULL batch");
        return SV_ERR_ARG;
    }
    const size_t nu = b->user.size(), base = 1 + b->plans.size();
    // the batch waits for what the member streams already hold
    for (size_t i = 0; i < nu; ++i) {
        SV_CUDA_TRY(cudaEventRecord(b->ev[base + i], b->user[i]));
        SV_CUDA_TRY(cudaStreamWaitEvent(b->main, b->ev[base + i], 0));
    }
    sv_status s = SV_OK;
    const char *g = std::getenv("SV_GRAPH");
    const bool graphs = !(g && g[0] == '0') && !std::getenv("SV_FAULT_INJECT");
    if (b->execs++ == 0 || !graphs) {
        s = check_launch(launch_members(b), "sv_batch_execute");
    } else {
        if (!b->gexec && capture(b) != cudaSuccess) {
            cudaGetLastError();
            s = check_launch(launch_members(b), "sv_batch_execute");
        } else {
            s = check_launch(cudaGraphLaunch(b->gexec, b->main), "sv_batch_execute (graph)");
        }
    }
    if (s) return s;
    // the member streams wait for the batch
    for (size_t i = 0; i < nu; ++i) {
        SV_CUDA_TRY(cudaEventRecord(b->ev[base + i], b->main));
        SV_CUDA_TRY(cudaStreamWaitEvent(b->user[i], b->ev[base + i], 0));
    }
    return SV_OK;
}

extern "C" sv_status sv_batch_info(sv_batch b, int64_t *gates, int64_t *launches, double *bytes, int *uses_graph) {
    if (!b) {
        set_error("NULL batch");
        return SV_ERR_ARG;
    }
    if (gates) *gates = b->gates;
    if (launches) *launches = b->launches;
    if (bytes) *bytes = b->bytes;
    if (uses_graph) *uses_graph = b->gexec != nullptr ? 1 : 0;
    return SV_OK;
}

extern "C" sv_status sv_batch_free(sv_batch b) {
    if (!b) return SV_OK;
    cudaStreamSynchronize(b->main);
    for (cudaStream_t s : b->branch)
        if (s) cudaStreamSynchronize(s);
    destroy_batch(b);
    return SV_OK;
}

extern "C" sv_status sv_run_batch(const sv_handle *handles, const char *const *texts, int count) {
    sv_batch b = nullptr;
    sv_status s = sv_batch_create(handles, texts, count, &b);
    if (s) return s;
    s = sv_batch_execute(b);
    const sv_status f = sv_batch_free(b);
    return s ? s : f;
}
