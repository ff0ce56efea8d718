// Plan creation and replay.
#include <cstdlib>
#include <string>

#include <mutex>
#include <unordered_map>
#include <cstring>

#include "plan.h"

namespace sv {

double gate1_bytes(const sv_state *h, const Gate1 &g) {
    const double amps = double(uint64_t(1) << h->n);
    if (h->dt == SV_ENC2B) {
        const double nb = h->n < kEncBlockLog2 ? 1.0 : amps / kEncBlock;
        const std::string k = gate1_kernel_name(h, g);
        // fraction of blocks a pass visits: block-level condition bits halve it
        int blockbits = 0;
        if (g.control >= kEncBlockLog2) ++blockbits;
        const bool flip = k == "k_enc_flip";
        if (k == "k_enc_phase_blocks") ++blockbits;  // the blocks with the target bit set
        if (flip) {
            const bool both = g.u[0].re == -1 && g.u[3].re == -1;
            if (!both && g.target >= kEncBlockLog2) ++blockbits;
        }
        const double frac = 1.0 / double(1 << blockbits);
        if (flip || k == "k_enc_xin") return frac * 2.0 * amps * 2.0;          // codes only
        return frac * (2.0 * amps * 2.0 + 2.0 * nb * 4.0);                    // codes and scales
    }
    const double s = h->dt == SV_C64 ? 8.0 : 16.0;
    const bool diag = g.u[1].re == 0 && g.u[1].im == 0 && g.u[2].re == 0 && g.u[2].im == 0;
    const bool unit00 = g.u[0].re == 1 && g.u[0].im == 0;
    double frac = (diag && unit00) ? 0.5 : 1.0;
    if (g.control >= 0) frac *= 0.5;
    return 2.0 * amps * s * frac;
}

namespace {

void destroy_plan(sv_plan_s *p) {
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    for (cudaEvent_t e : p->gev)
        if (e) cudaEventDestroy(e);
    if (p->gstream) cudaStreamDestroy(p->gstream);
    if (p->d_tcA) cudaFree(p->d_tcA);
    if (p->d_encops) cudaFree(p->d_encops);
    delete p;
}

// Fused mode: blocks of at most k qubits; without a measured choice
// (kfix = 0) the k in 3..6 with the fewest blocks (each block is one HBM
// pass; ties to the smaller k).
sv_status build_fused_plan(sv_state *h, const Circuit &c, sv_plan_s *p, int kfix = 0) {
    std::vector<FusedBlock> best;
    int bestk = 0;
    const int kmin = kfix ? kfix : (h->n < 3 ? h->n : 3);
    const int kmax = kfix ? kfix : kMaxFusedQubits;
    for (int k = kmin; k <= kmax && k <= h->n; ++k) {
        std::vector<FusedBlock> b = fuse_blocks(c, k);
        if (bestk == 0 || b.size() < best.size()) {
            best.swap(b);
            bestk = k;
        }
    }
    p->fused_k = bestk;
    const double pass_bytes = 2.0 * double(uint64_t(1) << h->n) * (h->dt == SV_C64 ? 8.0 : 16.0);
    if (fused_tc_supported(h) && !best.empty()) {
        std::vector<uint16_t> img(best.size() * (kTcOperandBytes / 2));
        p->tcargs.resize(best.size());
        for (size_t i = 0; i < best.size(); ++i)
            tc_prepare(h->n, best[i].k, best[i].qubits, best[i].U.data(), img.data() + i * (kTcOperandBytes / 2),
                       &p->tcargs[i]);
        SV_CUDA_TRY(cudaMalloc(&p->d_tcA, img.size() * 2));
        SV_CUDA_TRY(cudaMemcpy(p->d_tcA, img.data(), img.size() * 2, cudaMemcpyHostToDevice));
        for (size_t i = 0; i < best.size(); ++i) p->launches.push_back(PlanLaunch{2, int(i), pass_bytes});
    } else {
        p->blocks.swap(best);
        for (size_t i = 0; i < p->blocks.size(); ++i) p->launches.push_back(PlanLaunch{3, int(i), pass_bytes});
    }
    p->bytes = pass_bytes * double(p->launches.size());
    return SV_OK;
}

// Two-byte code: runs of consecutive in-block gates and sign flips become one
// pass each (k_enc_run_in) where the run's gates, one pass each, would move
// more bytes than one pass over the code; the other gates keep their own
// passes.  SV_ENC_RUNS=0 keeps one pass per gate.
bool enc_runs_enabled() {
    const char *e = std::getenv("SV_ENC_RUNS");
    return !(e && e[0] == '0');
}

sv_status build_enc_runs(sv_state *h, sv_plan_s *p) {
    if (h->n < kEncBlockLog2 || !enc_runs_enabled()) return SV_OK;
    const double amps = double(uint64_t(1) << h->n);
    const double pass_bytes = 2.0 * amps * 2.0 + 2.0 * (amps / kEncBlock) * 4.0;
    std::vector<EncRunOp> ops;
    const size_t ng = p->pergate.size();
    size_t i = 0;
    while (i < ng) {
        EncRunOp op;
        size_t j = i;
        double alone = 0.0;
        while (j < ng && j - i < size_t(kEncRunMaxOps) && enc_run_op(h->n, p->pergate[j], &op)) {
            alone += gate1_bytes(h, p->pergate[j]);
            ++j;
        }
        if (j - i >= 2 && alone > pass_bytes) {
            PlanLaunch l{4, int(p->encruns.size()), pass_bytes};
            p->encruns.push_back({int(ops.size()), int(j - i), int(j - i)});
            for (size_t k = i; k < j; ++k) {
                enc_run_op(h->n, p->pergate[k], &op);
                ops.push_back(op);
            }
            p->launches.push_back(l);
            p->bytes += pass_bytes;
            i = j;
            continue;
        }
        const size_t stop = j > i ? j : i + 1;  // the gates of a short run, or one other gate
        for (size_t k = i; k < stop; ++k) {
            const double b = gate1_bytes(h, p->pergate[k]);
            p->launches.push_back(PlanLaunch{0, int(k), b});
            p->bytes += b;
        }
        i = stop;
    }
    if (!ops.empty()) {
        SV_CUDA_TRY(cudaMalloc(&p->d_encops, ops.size() * sizeof(EncRunOp)));
        SV_CUDA_TRY(cudaMemcpy(p->d_encops, ops.data(), ops.size() * sizeof(EncRunOp), cudaMemcpyHostToDevice));
    }
    return SV_OK;
}

template <typename R>
sv_status upload_tile_plan(sv_plan_s *p, const TilePlan<R> &tp) {
    p->tile_lane_ops = tp.lane_ops;
    p->tile_nseg = tp.nseg;
    sv_status s = jit_tile_plan(tp, &p->tfns);
    if (s) return s;
    p->tile_rb = tp.rb;
    const double pass_bytes = 2.0 * double(uint64_t(1) << p->h->n) * (p->h->dt == SV_C64 ? 8.0 : 16.0);
    for (size_t i = 0; i < tp.passes.size(); ++i) {
        PlanLaunch l{1, int(i), pass_bytes};  // compiled pass i
        l.lane_ops = tp.lane_ops[i];
        l.segments = tp.nseg[i];
        p->launches.push_back(l);
        p->bytes += pass_bytes;
    }
    return SV_OK;
}

sv_status build_tile_plan(sv_state *h, const Circuit &c, sv_plan_s *p, const TileConfig &cfg,
                          const std::vector<int> &pass_ctas = std::vector<int>()) {
    if (h->dt == SV_C64) {
        TilePlan<float> tp;
        sv_status s = plan_tiles<float>(c, h->n, cfg, &tp);
        if (!s && !pass_ctas.empty()) {
            if (pass_ctas.size() != tp.passes.size()) {
                set_error("per-pass CTA counts for %zu passes, the plan has %zu", pass_ctas.size(), tp.passes.size());
                return SV_ERR_ARG;
            }
            tp.pass_ctas = pass_ctas;
        }
        return s ? s : upload_tile_plan(p, tp);
    }
    TilePlan<double> tp;
    sv_status s = plan_tiles<double>(c, h->n, tile_config128(), &tp);
    return s ? s : upload_tile_plan(p, tp);
}

cudaError_t launch_one(sv_plan_s *p, const PlanLaunch &l) {
    if (l.kind == 0) return launch_gate1(p->h, p->pergate[size_t(l.index)]);
    if (l.kind == 2)
        return tc_launch(p->h, p->tcargs[size_t(l.index)],
                         static_cast<const char *>(p->d_tcA) + size_t(l.index) * kTcOperandBytes);
    if (l.kind == 3) {
        const FusedBlock &b = p->blocks[size_t(l.index)];
        return launch_fused(p->h, b.k, b.qubits, b.U.data());
    }
    if (l.kind == 4) {
        const sv_plan_s::EncRun &r = p->encruns[size_t(l.index)];
        return launch_enc_run(p->h, p->d_encops + r.first, r.count);
    }
    return launch_jit_pass(p->h, p->tfns[size_t(l.index)], p->h->n, p->tile_rb);
}

const char *launch_name(const sv_plan_s *p, const PlanLaunch &l) {
    if (l.kind == 0) return gate1_kernel_name(p->h, p->pergate[size_t(l.index)]);
    if (l.kind == 2) return tc_kernel_name(p->tcargs[size_t(l.index)]);
    if (l.kind == 3) return p->h->dt == SV_C64 ? "k_fused_dense<f32>" : "k_fused_dense<f64>";
    if (l.kind == 4) return "k_enc_run_in";
    return tile_kernel_name(p->h);
}

}  // namespace

}  // namespace sv

using namespace sv;

extern "C" {

namespace sv {
namespace {

// Tiled plans by circuit text: a repeated circuit skips parsing, planning and
// code generation (its compiled passes stay loaded for the process).  The key
// holds everything the plan depends on: device, dtype, qubit count, tile
// configuration, planner and code-generation settings, and the text.
struct TileCacheEntry {
    std::vector<void *> fns;
    int rb = 0;
    int64_t gates = 0;
    std::vector<double> lane_ops;
    std::vector<int> nseg;
};
std::mutex g_tile_cache_mu;
std::unordered_map<std::string, TileCacheEntry> g_tile_cache;
constexpr size_t kTileCacheMax = 64;

std::string tile_cache_key(const sv_state *h, const TileConfig &cfg, const char *text) {
    return std::to_string(h->device) + "|" + std::to_string(int(h->dt)) + "|" + std::to_string(h->n) + "|" +
           tile_config_name(cfg) + ",look=" + std::to_string(plan_lookahead_width()) + "," + tile_codegen_key() +
           "|" + text;
}

// One candidate execution strategy: a mode, and for the tiled mode the tile
// configuration (and, optionally, the CTAs per SM of each pass), for the
// fused mode the block width (0 = fewest blocks).
struct Strategy {
    int mode = SV_MODE_TILED;
    TileConfig cfg{};
    int k = 0;
    std::vector<int> pass_ctas;
    std::string name() const {
        if (mode == SV_MODE_TILED) {
            std::string nm = "tiled " + tile_config_name(cfg);
            if (!pass_ctas.empty()) {
                nm += ",pass_ctas=";
                for (int v : pass_ctas) nm += char('0' + v);
            }
            return nm;
        }
        if (mode == SV_MODE_FUSED) return "fused k=" + std::to_string(k);
        return "pergate";
    }
};

std::string pass_ctas_key(const std::vector<int> &pc) {
    std::string k;
    for (int v : pc) k += char('0' + v);
    return k;
}

TileConfig default_config(const sv_state *h) { return h->dt == SV_C64 ? tile_config64() : tile_config128(); }

// Build the plan of one strategy for the handle (text already parsed into c).
sv_status create_plan(sv_state *h, const char *text, const Circuit &c, const Strategy &st, sv_plan_s **out) {
    *out = nullptr;
    const int tile_m = st.mode == SV_MODE_TILED ? st.cfg.m : (h->dt == SV_C64 ? kTileM64 : kTileM128);
    const bool tiled = st.mode == SV_MODE_TILED && h->n >= tile_m;
    std::string key;
    if (tiled && text) {
        key = tile_cache_key(h, st.cfg, text) + "|" + pass_ctas_key(st.pass_ctas);
        std::lock_guard<std::mutex> lock(g_tile_cache_mu);
        auto it = g_tile_cache.find(key);
        if (it != g_tile_cache.end()) {
            sv_plan_s *p = new sv_plan_s;
            p->h = h;
            p->mode = st.mode;
            p->gates = it->second.gates;
            p->tfns = it->second.fns;
            p->tile_rb = it->second.rb;
            p->tile_lane_ops = it->second.lane_ops;
            p->tile_nseg = it->second.nseg;
            const double pass_bytes = 2.0 * double(uint64_t(1) << h->n) * (h->dt == SV_C64 ? 8.0 : 16.0);
            for (size_t i = 0; i < p->tfns.size(); ++i) {
                PlanLaunch l{1, int(i), pass_bytes};
                l.lane_ops = i < p->tile_lane_ops.size() ? p->tile_lane_ops[i] : 0.0;
                l.segments = i < p->tile_nseg.size() ? p->tile_nseg[i] : 0;
                p->launches.push_back(l);
                p->bytes += pass_bytes;
            }
            *out = p;
            return SV_OK;
        }
    }
    sv_plan_s *p = new sv_plan_s;
    p->h = h;
    p->mode = st.mode;
    p->gates = int64_t(c.instrs.size());
    sv_status s = SV_OK;
    if (st.mode == SV_MODE_FUSED) {
        s = build_fused_plan(h, c, p, st.k);
    } else if (st.mode == SV_MODE_PERGATE || h->n < tile_m) {
        // per-gate updates (also the tiled mode's path for states smaller than one tile)
        p->pergate = lower_to_gate1(c);
        s = h->dt == SV_ENC2B ? build_enc_runs(h, p) : SV_OK;
        if (!s && p->launches.empty())
            for (size_t i = 0; i < p->pergate.size(); ++i) {
                const double b = gate1_bytes(h, p->pergate[i]);
                p->launches.push_back(PlanLaunch{0, int(i), b});
                p->bytes += b;
            }
    } else {
        s = build_tile_plan(h, c, p, st.cfg, st.pass_ctas);
        if (!s && !key.empty()) {
            std::lock_guard<std::mutex> lock(g_tile_cache_mu);
            if (g_tile_cache.size() >= kTileCacheMax) g_tile_cache.clear();
            g_tile_cache[key] = TileCacheEntry{p->tfns, p->tile_rb, p->gates, p->tile_lane_ops, p->tile_nseg};
        }
    }
    if (s) {
        destroy_plan(p);
        return s;
    }
    *out = p;
    return SV_OK;
}

// ---------------------------------------------------------------- autotuner
// SV_MODE_AUTO measures instead of predicting: every candidate strategy is
// planned (and compiled), run once to warm up and then timed with CUDA events
// on a scratch state of the handle's size and dtype (cudaMalloc'ed for the
// tuning and freed after it; its amplitudes do not change the time of these
// kernels), and the fastest is kept.  The choice is remembered per device,
// dtype, qubit count and circuit text, in the process and in the file
// autotune.txt of the compiled-pass cache folder, so a later plan of the same
// circuit (also in a later process) skips the timing.  Without room for a
// scratch state the planner's own choice (tiled, else fused) is taken.

std::vector<Strategy> candidates(const sv_state *h) {
    std::vector<Strategy> v;
    const int tile_m = h->dt == SV_C64 ? kTileM64 : kTileM128;
    if (h->dt == SV_ENC2B) {
        v.push_back(Strategy{SV_MODE_PERGATE, TileConfig{}, 0});
        return v;
    }
    if (h->n >= tile_m) {
        if (h->dt == SV_C64) {
            // the generator's configurations: register bits, CTAs per SM,
            // direct HBM I/O, prefetching, tile bits
            const int opts[][5] = {{5, 2, 1, 0, 13}, {5, 2, 1, 1, 13}, {5, 2, 0, 0, 13},
                                   {4, 2, 1, 0, 13}, {5, 3, 1, 0, 13}, {5, 4, 1, 0, 12}};
            for (const auto &o : opts)
                if (h->n >= o[4])
                    v.push_back(Strategy{SV_MODE_TILED, tile_config64(o[0], o[1], o[2], o[3], o[4]), 0});
        } else {
            v.push_back(Strategy{SV_MODE_TILED, tile_config128(), 0});
        }
    } else {
        v.push_back(Strategy{SV_MODE_PERGATE, TileConfig{}, 0});
    }
    for (int k = 3; k <= kMaxFusedQubits && k <= h->n; ++k) v.push_back(Strategy{SV_MODE_FUSED, TileConfig{}, k});
    return v;
}

std::mutex g_tune_mu;
std::unordered_map<std::string, std::string> g_tune;  // key -> chosen strategy name

uint64_t fnv1a(const std::string &t) {
    uint64_t x = 1469598103934665603ull;
    for (unsigned char ch : t) x = (x ^ ch) * 1099511628211ull;
    return x;
}

std::string tune_key(const sv_state *h, const char *text) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, h->device);
    char b[96];
    std::snprintf(b, sizeof b, "%d|%d|%016llx", h->n, int(h->dt), static_cast<unsigned long long>(fnv1a(text)));
    std::string name = prop.name;
    for (char &ch : name)
        if (ch == '\t' || ch == '\n') ch = ' ';
    return name + "|" + b + "|" + tile_codegen_key();
}

std::string tune_file() {
    const std::string dir = jit_cache_dir();
    return dir.empty() ? std::string() : dir + "/autotune.txt";
}

// A remembered choice for key ("" if none): the process map, else the file.
std::string tune_lookup(const std::string &key) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
    const std::string path = tune_file();
    if (path.empty()) return std::string();
    std::string found;
    if (FILE *f = std::fopen(path.c_str(), "r")) {
        char line[1024];
        while (std::fgets(line, sizeof line, f)) {
            std::string ln(line);
            while (!ln.empty() && (ln.back() == '\n' || ln.back() == '\r')) ln.pop_back();
            const size_t tab = ln.find('\t');
            if (tab != std::string::npos && ln.compare(0, tab, key) == 0) found = ln.substr(tab + 1);
        }
        std::fclose(f);
    }
    if (!found.empty()) g_tune[key] = found;
    return found;
}

void tune_store(const std::string &key, const std::string &choice) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = choice;
    const std::string path = tune_file();
    if (path.empty()) return;
    if (FILE *f = std::fopen(path.c_str(), "a")) {
        std::fprintf(f, "%s\t%s\n", key.c_str(), choice.c_str());
        std::fclose(f);
    }
}

sv_status execute_direct(sv_plan_s *p);

// Time each candidate on a scratch state; returns the index of the fastest
// and a JSON report of all of them in *report.  Tiled candidates are also
// timed pass by pass; where two of them differ only in the CTAs per SM their
// passes are compiled for, a further candidate takes each pass in its faster
// form (the pass plan does not depend on that count) and is appended to cand
// and timed like the others.
sv_status time_candidates(sv_state *h, const char *text, const Circuit &c, std::vector<Strategy> &cand,
                          size_t *best, std::string *report) {
    size_t free_b = 0, total_b = 0;
    SV_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    if (h->bytes + (size_t(1) << 30) > free_b) {
        *report = "{\"timed\": false, \"reason\": \"no device memory for a scratch state\"}";
        return SV_ERR_OOM;
    }
    sv_state scratch;
    scratch.n = h->n;
    scratch.dt = h->dt;
    scratch.bytes = h->bytes;
    scratch.stream = h->stream;
    scratch.device = h->device;
    SV_CUDA_TRY(cudaMalloc(&scratch.data, h->bytes));
    if (h->dt == SV_ENC2B) scratch.scales = reinterpret_cast<float *>(static_cast<char *>(scratch.data) + (size_t(2) << h->n));
    cudaEvent_t ev[2] = {nullptr, nullptr};
    sv_status s = SV_OK;
    for (int i = 0; i < 2 && s == SV_OK; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) s = SV_ERR_CUDA;
    std::string js = "{\"timed\": true, \"candidates\": [";
    double best_ms = -1.0;
    std::vector<std::vector<double>> pass_ms(cand.size());  // per launch, tiled candidates
    bool mixed_added = false;
    for (size_t i = 0; i < cand.size() && s == SV_OK; ++i) {
        sv_plan_s *p = nullptr;
        sv_status cs = create_plan(&scratch, text, c, cand[i], &p);
        double ms = -1.0;
        if (cs == SV_OK) {
            cs = check_launch(launch_set_basis(&scratch, 0), "autotune");
            if (!cs) cs = execute_direct(p);  // warm-up (module loads, one-time set-up)
            const int reps = 2;
            if (!cs && cudaEventRecord(ev[0], scratch.stream) != cudaSuccess) cs = SV_ERR_CUDA;
            for (int r = 0; r < reps && !cs; ++r) cs = execute_direct(p);
            if (!cs && cudaEventRecord(ev[1], scratch.stream) != cudaSuccess) cs = SV_ERR_CUDA;
            if (!cs) cs = sync_stream(scratch.stream, "autotune");
            float t = 0.0f;
            if (!cs && cudaEventElapsedTime(&t, ev[0], ev[1]) == cudaSuccess) ms = double(t) / reps;
            // pass by pass (tiled plans): one more execution, an event between launches
            const size_t nl = p->launches.size();
            if (!cs && cand[i].mode == SV_MODE_TILED && cand[i].pass_ctas.empty() && nl > 0 &&
                p->launches[0].kind == 1) {
                std::vector<cudaEvent_t> pe(nl + 1, nullptr);
                bool ok = true;
                for (auto &e : pe) ok = ok && cudaEventCreate(&e) == cudaSuccess;
                if (ok) cs = sv_plan_execute_timed(p, reinterpret_cast<void *const *>(pe.data()), int64_t(nl + 1));
                if (ok && !cs) cs = sync_stream(scratch.stream, "autotune");
                if (ok && !cs) {
                    pass_ms[i].resize(nl);
                    for (size_t j = 0; j < nl; ++j) {
                        float tj = 0.0f;
                        cudaEventElapsedTime(&tj, pe[j], pe[j + 1]);
                        pass_ms[i][j] = double(tj);
                    }
                }
                for (auto &e : pe)
                    if (e) cudaEventDestroy(e);
            }
            destroy_plan(p);
        }
        if (cs == SV_ERR_CUDA || cs == SV_ERR_TIMEOUT) s = cs;  // a device fault ends the tuning
        char b[320];
        std::snprintf(b, sizeof b, "%s{\"strategy\": \"%s\", \"ms\": %.6f%s}", i ? ", " : "",
                      cand[i].name().c_str(), ms, cs ? ", \"failed\": true" : "");
        js += b;
        if (ms > 0 && (best_ms < 0 || ms < best_ms)) {
            best_ms = ms;
            *best = i;
        }
        // after the last original candidate: the per-pass mix of two that differ only in CTAs
        if (i + 1 == cand.size() && !mixed_added && s == SV_OK) {
            mixed_added = true;
            for (size_t a2 = 0; a2 < i + 1; ++a2)
                for (size_t a3 = 0; a3 < i + 1; ++a3) {
                    const TileConfig &x = cand[a2].cfg, &y = cand[a3].cfg;
                    if (a2 == a3 || pass_ms[a2].empty() || pass_ms[a2].size() != pass_ms[a3].size() ||
                        x.ctas >= y.ctas || x.m != y.m || x.rb != y.rb || x.low != y.low || x.direct != y.direct ||
                        x.prefetch != y.prefetch || x.c64 != y.c64)
                        continue;
                    Strategy mix = cand[a2];
                    bool both = false, any = false;
                    for (size_t j = 0; j < pass_ms[a2].size(); ++j) {
                        const bool hi = pass_ms[a3][j] < pass_ms[a2][j];
                        mix.pass_ctas.push_back(hi ? y.ctas : x.ctas);
                        any = any || hi;
                        both = both || !hi;
                    }
                    if (any && both && cand.size() < 64) cand.push_back(mix);
                }
        }
    }    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    cudaStreamSynchronize(scratch.stream);
    for (void *d : {static_cast<void *>(scratch.data), static_cast<void *>(scratch.d_partials),
                    static_cast<void *>(scratch.d_idx), static_cast<void *>(scratch.d_amps), scratch.d_mat,
                    static_cast<void *>(scratch.d_err), static_cast<void *>(scratch.d_expect)})
        if (d) cudaFree(d);
    scratch.data = nullptr;
    js += "]";
    if (best_ms > 0) js += ", \"chosen\": \"" + cand[*best].name() + "\"";
    *report = js + "}";
    if (s == SV_OK && best_ms < 0) {
        set_error("autotune: no candidate ran");
        s = SV_ERR_UNSUPPORTED;
    }
    return s;
}

sv_status create_auto_plan(sv_state *h, const char *text, const Circuit &c, sv_plan_s **out) {
    std::vector<Strategy> cand = candidates(h);
    const std::string key = tune_key(h, text);
    const std::string known = tune_lookup(key);
    // a remembered per-pass mix: its base candidate's name, then ",pass_ctas=" and one digit per pass
    const size_t mixed_at = known.find(",pass_ctas=");
    for (const Strategy &base : cand) {
        Strategy st = base;
        if (mixed_at != std::string::npos) {
            if (base.name() != known.substr(0, mixed_at)) continue;
            for (size_t j = mixed_at + 11; j < known.size(); ++j) st.pass_ctas.push_back(known[j] - '0');
        }
        if (!known.empty() && st.name() == known) {
            sv_status s = create_plan(h, text, c, st, out);
            if (!s) (*out)->tuning = "{\"timed\": false, \"remembered\": true, \"chosen\": \"" + known + "\"}";
            return s;
        }
    }
    if (cand.size() == 1) {  // nothing to choose between (the two-byte code)
        sv_status s = create_plan(h, text, c, cand[0], out);
        if (!s)
            (*out)->tuning = "{\"timed\": false, \"reason\": \"one candidate\", \"chosen\": \"" + cand[0].name() + "\"}";
        return s;
    }
    size_t best = 0;
    std::string report;
    sv_status s = time_candidates(h, text, c, cand, &best, &report);
    if (s == SV_ERR_OOM) {
        // no room to time: the planner's own choice
        Strategy st{h->dt == SV_ENC2B ? SV_MODE_PERGATE : SV_MODE_TILED, default_config(h), 0};
        s = create_plan(h, text, c, st, out);
        if (!s) (*out)->tuning = report;
        return s;
    }
    if (s) return s;
    tune_store(key, cand[best].name());
    s = create_plan(h, text, c, cand[best], out);
    if (!s) (*out)->tuning = report;
    return s;
}

}  // namespace
}  // namespace sv

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
    if (mode != SV_MODE_PERGATE && mode != SV_MODE_TILED && mode != SV_MODE_FUSED && mode != SV_MODE_AUTO) {
        set_error("unknown mode %d", mode);
        return SV_ERR_ARG;
    }
    if (h->dt == SV_ENC2B && mode != SV_MODE_PERGATE && mode != SV_MODE_AUTO) {
        set_error("the two-byte code runs one decode-gate-encode pass per gate (SV_MODE_PERGATE)");
        return SV_ERR_DTYPE;
    }
    if (!text) {
        set_error("NULL circuit text");
        return SV_ERR_ARG;
    }
    Circuit c;
    sv_status s = SV_OK;
    // a cached tiled plan needs no parse (the text is part of its key)
    const Strategy st{mode, default_config(h), 0};
    const bool maybe_cached = mode == SV_MODE_TILED;
    if (!maybe_cached) {
        s = parse_circuit(text, h->n, &c);
        if (s) return s;
    }
    sv_plan_s *p = nullptr;
    if (mode == SV_MODE_AUTO) {
        s = create_auto_plan(h, text, c, &p);
    } else {
        if (maybe_cached) {
            std::lock_guard<std::mutex> lock(g_tile_cache_mu);
            if (!g_tile_cache.count(tile_cache_key(h, st.cfg, text))) s = SV_ERR_PARSE;  // not cached: parse below
        }
        if (s == SV_ERR_PARSE) {
            s = parse_circuit(text, h->n, &c);
            if (s) return s;
        }
        s = create_plan(h, text, c, st, &p);
    }
    if (s) return s;
    h->live_plans++;
    *out = p;
    return SV_OK;
}

namespace sv {
namespace {

sv_status execute_direct(sv_plan_s *p) {
    for (const PlanLaunch &l : p->launches) {
        sv_status s = check_launch(launch_one(p, l), "sv_plan_execute");
        if (s) return s;
    }
    return SV_OK;
}

}  // namespace

extern "C++" {
cudaError_t plan_launch_all(sv_plan_s *p) {
    for (const PlanLaunch &l : p->launches) {
        const cudaError_t e = launch_one(p, l);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool plan_capturable(const sv_plan_s *p) {
    for (const PlanLaunch &l : p->launches)
        if (l.kind == 3) return false;  // host matrix copies per launch
    return true;
}
}  // extern "C++"

namespace {

// Graph replay applies to plans of two or more launches that are kernel
// launches only (the CUDA-core dense blocks copy their matrix from host
// memory at launch time), unless SV_GRAPH=0 or a host-side fault injection
// is active (it acts per launch).
bool graph_wanted(const sv_plan_s *p) {
    if (p->graph_off || p->launches.size() < 2) return false;
    const char *g = std::getenv("SV_GRAPH");
    if (g && g[0] == '0') return false;
    if (std::getenv("SV_FAULT_INJECT")) return false;
    for (const PlanLaunch &l : p->launches)
        if (l.kind == 3) return false;
    return true;
}

// Capture the launches on the private stream (thread-local mode: a call that
// is not allowed during capture fails instead of running) and instantiate.
cudaError_t capture_graph(sv_plan_s *p) {
    sv_state *h = p->h;
    cudaError_t e = cudaSuccess;
    if (!p->gstream) e = cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        if (!p->gev[i]) e = cudaEventCreateWithFlags(&p->gev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    const cudaStream_t user = h->stream;
    h->stream = p->gstream;  // the launch functions launch on the handle's stream
    e = cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaSuccess;
        for (const PlanLaunch &l : p->launches) {
            le = launch_one(p, l);
            if (le != cudaSuccess) break;
        }
        cudaGraph_t g = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(p->gstream, &g);
        e = le != cudaSuccess ? le : ee;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&p->gexec, g, 0ULL);
        if (g) cudaGraphDestroy(g);
    }
    h->stream = user;
    if (e != cudaSuccess) {
        if (p->gexec) cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    return e;
}

sv_status execute_graph(sv_plan_s *p) {
    sv_state *h = p->h;
    SV_CUDA_TRY(cudaEventRecord(p->gev[0], h->stream));
    SV_CUDA_TRY(cudaStreamWaitEvent(p->gstream, p->gev[0], 0));
    SV_CUDA_TRY(cudaGraphLaunch(p->gexec, p->gstream));
    SV_CUDA_TRY(cudaEventRecord(p->gev[1], p->gstream));
    SV_CUDA_TRY(cudaStreamWaitEvent(h->stream, p->gev[1], 0));
    return SV_OK;
}

}  // namespace
}  // namespace sv

sv_status sv_plan_execute(sv_plan p) {
    if (!p) {
        set_error("NULL plan");
        return SV_ERR_ARG;
    }
    if (!graph_wanted(p) || p->execs++ == 0) return execute_direct(p);
    if (!p->gexec && capture_graph(p) != cudaSuccess) {
        // not capturable here: clear the error state and launch directly from now on
        cudaGetLastError();
        p->graph_off = true;
        return execute_direct(p);
    }
    return execute_graph(p);
}

sv_status sv_plan_uses_graph(sv_plan p, int *out) {
    if (!p || !out) {
        set_error("NULL argument");
        return SV_ERR_ARG;
    }
    *out = p->gexec != nullptr ? 1 : 0;
    return SV_OK;
}

sv_status sv_plan_info(sv_plan p, int64_t *gates, int64_t *passes, double *bytes) {
    if (!p) {
        set_error("NULL plan");
        return SV_ERR_ARG;
    }
    if (gates) *gates = p->gates;
    if (passes) *passes = int64_t(p->launches.size());
    if (bytes) *bytes = p->bytes;
    return SV_OK;
}

sv_status sv_plan_execute_timed(sv_plan p, void *const *events, int64_t n_events) {
    if (!p || !events) {
        set_error("NULL argument");
        return SV_ERR_ARG;
    }
    const int64_t passes = int64_t(p->launches.size());
    if (n_events < passes + 1) {
        set_error("need %lld events, got %lld", (long long)(passes + 1), (long long)n_events);
        return SV_ERR_ARG;
    }
    for (int64_t i = 0; i < passes; ++i) {
        cudaError_t e = cudaEventRecord(static_cast<cudaEvent_t>(events[i]), p->h->stream);
        if (e != cudaSuccess) return cuda_status(e, "cudaEventRecord");
        sv_status s = check_launch(launch_one(p, p->launches[size_t(i)]), "sv_plan_execute_timed");
        if (s) return s;
    }
    cudaError_t e = cudaEventRecord(static_cast<cudaEvent_t>(events[passes]), p->h->stream);
    if (e != cudaSuccess) return cuda_status(e, "cudaEventRecord");
    return SV_OK;
}

sv_status sv_plan_launch_info(sv_plan p, int64_t i, const char **kernel, double *bytes) {
    if (!p || i < 0 || i >= int64_t(p->launches.size())) {
        set_error("bad plan or launch index");
        return SV_ERR_ARG;
    }
    if (kernel) *kernel = launch_name(p, p->launches[size_t(i)]);
    if (bytes) *bytes = p->launches[size_t(i)].bytes;
    return SV_OK;
}

sv_status sv_plan_stats(const char *text, int n, sv_dtype dt, int compile, int64_t *gates, int64_t *passes,
                        int64_t *segments) {
    if (!text || n < 1 || n > kMaxQubits || (dt != SV_C64 && dt != SV_C128)) {
        set_error("bad arguments");
        return SV_ERR_ARG;
    }
    Circuit c;
    sv_status s = parse_circuit(text, n, &c);
    if (s) return s;
    if (gates) *gates = int64_t(c.instrs.size());
    auto count = [&](auto &tp) -> sv_status {
        int64_t segs = 0;
        for (const auto &op : tp.ops) segs += op.type == TOP_SEG;
        if (passes) *passes = int64_t(tp.passes.size());
        if (segments) *segments = segs;
        return compile ? jit_compile_check(tp) : SV_OK;
    };
    if (dt == SV_C64) {
        if (n < kTileM64) {
            set_error("tiled passes need n >= %d", kTileM64);
            return SV_ERR_UNSUPPORTED;
        }
        TilePlan<float> tp;
        s = plan_tiles<float>(c, n, tile_config64(), &tp);
        return s ? s : count(tp);
    }
    if (n < kTileM128) {
        set_error("tiled passes need n >= %d", kTileM128);
        return SV_ERR_UNSUPPORTED;
    }
    TilePlan<double> tp;
    s = plan_tiles<double>(c, n, tile_config128(), &tp);
    return s ? s : count(tp);
}

sv_status sv_plan_launch_stats(sv_plan p, int64_t i, double *fp32_ops_per_amplitude, int64_t *segments) {
    if (!p || i < 0 || i >= int64_t(p->launches.size())) {
        set_error("bad plan or launch index");
        return SV_ERR_ARG;
    }
    const PlanLaunch &l = p->launches[size_t(i)];
    if (fp32_ops_per_amplitude) *fp32_ops_per_amplitude = l.lane_ops;
    if (segments) *segments = l.segments;
    return SV_OK;
}

sv_status sv_plan_pass_source(const char *text, int n, sv_dtype dt, int64_t pass, char *buf, size_t cap,
                              size_t *len) {
    if (!text || n < 1 || n > kMaxQubits || (dt != SV_C64 && dt != SV_C128) || pass < 0) {
        set_error("bad arguments");
        return SV_ERR_ARG;
    }
    Circuit c;
    sv_status s = parse_circuit(text, n, &c);
    if (s) return s;
    auto emit = [&](auto &tp) -> sv_status {
        if (pass >= int64_t(tp.passes.size())) {
            set_error("pass %lld of a %zu-pass plan", (long long)pass, tp.passes.size());
            return SV_ERR_ARG;
        }
        const std::string src = tile_pass_source(tp, size_t(pass));
        if (len) *len = src.size();
        if (buf && cap > 0) {
            const size_t k = src.size() < cap - 1 ? src.size() : cap - 1;
            std::memcpy(buf, src.data(), k);
            buf[k] = '\0';
        }
        return SV_OK;
    };
    if (dt == SV_C64) {
        if (n < kTileM64) {
            set_error("tiled passes need n >= %d", kTileM64);
            return SV_ERR_UNSUPPORTED;
        }
        TilePlan<float> tp;
        s = plan_tiles<float>(c, n, tile_config64(), &tp);
        return s ? s : emit(tp);
    }
    if (n < kTileM128) {
        set_error("tiled passes need n >= %d", kTileM128);
        return SV_ERR_UNSUPPORTED;
    }
    TilePlan<double> tp;
    s = plan_tiles<double>(c, n, tile_config128(), &tp);
    return s ? s : emit(tp);
}

sv_status sv_plan_tuning(sv_plan p, char *buf, size_t cap, size_t *len) {
    if (!p) {
        set_error("NULL plan");
        return SV_ERR_ARG;
    }
    if (len) *len = p->tuning.size();
    if (buf && cap > 0) {
        const size_t k = p->tuning.size() < cap - 1 ? p->tuning.size() : cap - 1;
        std::memcpy(buf, p->tuning.data(), k);
        buf[k] = '\0';
    }
    return SV_OK;
}

sv_status sv_plan_free(sv_plan p) {
    if (!p) return SV_OK;
    if (p->h) p->h->live_plans--;
    destroy_plan(p);
    return SV_OK;
}

}  // extern "C"
