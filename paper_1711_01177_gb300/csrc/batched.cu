// Batched gather filter (one launch per batch, under a CUDA graph) and its
// autotuner.  The kernels are in gather.cu; this file decides launch
// shapes, captures and caches graphs, and times candidate shapes.
#include <mutex>

#include "grim_internal.cuh"

namespace {

std::mutex g_tune_mu;
grim_tune g_tuned[64][GRIM_MAX_Q + 1];
bool g_has_tuned[64][GRIM_MAX_Q + 1];

grim_tune default_tune() {
    grim_tune t;
    t.warps_per_cta = 8;
    t.reads_per_claim = 1;
    t.ctas_per_sm = 0;
    t.use_graph = 1;
    t.batch_reads = 262144;
    return t;
}

grim_tune normalized(const grim_tune& in) {
    grim_tune t = in;
    const grim_tune d = default_tune();
    if (t.warps_per_cta != 4 && t.warps_per_cta != 8) t.warps_per_cta = d.warps_per_cta;
    if (t.reads_per_claim <= 0) t.reads_per_claim = d.reads_per_claim;
    if (t.reads_per_claim > 64) t.reads_per_claim = 64;
    if (t.ctas_per_sm < 0) t.ctas_per_sm = 0;
    if (t.batch_reads <= 0) t.batch_reads = d.batch_reads;
    t.use_graph = t.use_graph ? 1 : 0;
    return t;
}

bool same_tune(const grim_tune& a, const grim_tune& b) {
    return a.warps_per_cta == b.warps_per_cta && a.reads_per_claim == b.reads_per_claim &&
           a.ctas_per_sm == b.ctas_per_sm && a.batch_reads == b.batch_reads;
}

int check_args(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
               const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, const uint8_t* pass) {
    if (!bank || n_reads < 0) return GRIM_EINVAL;
    if (n_reads == 0) return GRIM_OK;
    if (!reads || !read_offsets || !cand_bins || !cand_offsets || !E || !pass) return GRIM_EINVAL;
    return grim::check_device(bank);
}

}  // namespace

namespace grim {
// The launch shape grim_filter_batched(tune = NULL) would use for this bank.
grim_tune tuned_shape(const grim_bank* bank) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (bank->device >= 0 && bank->device < 64 && g_has_tuned[bank->device][bank->q])
        return g_tuned[bank->device][bank->q];
    return default_tune();
}
}  // namespace grim

extern "C" {

int grim_filter_batched(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                        const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                        uint16_t* sums, const grim_tune* tune, void* stream) {
    int rc = check_args(bank, reads, read_offsets, n_reads, cand_bins, cand_offsets, E, pass);
    if (rc != GRIM_OK || n_reads == 0) return rc;
    grim_tune t = default_tune();
    if (tune) {
        t = normalized(*tune);
    } else {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        if (bank->device >= 0 && bank->device < 64 && g_has_tuned[bank->device][bank->q])
            t = g_tuned[bank->device][bank->q];
    }
    grim::GatherArgs a{reads, read_offsets, n_reads, cand_bins, cand_offsets, E, pass, sums};
    cudaStream_t s = (cudaStream_t)stream;
    grim_bank* mb = const_cast<grim_bank*>(bank);

    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool real_stream = s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
    if (real_stream) GRIM_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (!t.use_graph || !real_stream || cs != cudaStreamCaptureStatusNone)
        return grim::launch_gather_batches(bank, a, t, &mb->counters[0], s);

    const void* key[8] = {reads, read_offsets, cand_bins, cand_offsets, E, pass, sums, nullptr};
    std::vector<grim::GraphEntry>& cache = *mb->graphs;
    for (grim::GraphEntry& g : cache) {
        bool hit = g.n_reads == n_reads && g.stream == s && same_tune(g.tune, t);
        for (int i = 0; hit && i < 8; i++) hit = g.key[i] == key[i];
        if (hit) {
            g.last_use = ++mb->graph_clock;
            GRIM_CUDA_TRY(cudaGraphLaunch(g.exec, s));
            return GRIM_OK;
        }
    }
    // a new graph: take a free counter slot or evict the least recently used
    int slot = (int)cache.size() + 1;
    size_t victim = cache.size();
    if ((int)cache.size() >= grim::kGraphCache) {
        victim = 0;
        for (size_t i = 1; i < cache.size(); i++)
            if (cache[i].last_use < cache[victim].last_use) victim = i;
        slot = cache[victim].slot;
    }
    GRIM_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    rc = grim::launch_gather_batches(bank, a, t, &mb->counters[slot], s);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc != GRIM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) {
        grim::set_last_cuda_error(e);
        return GRIM_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        grim::set_last_cuda_error(e);
        return GRIM_ECUDA;
    }
    grim::GraphEntry g;
    for (int i = 0; i < 8; i++) g.key[i] = key[i];
    g.n_reads = n_reads;
    g.tune = t;
    g.stream = s;
    g.slot = slot;
    g.exec = exec;
    g.last_use = ++mb->graph_clock;
    if (victim < cache.size()) {
        cudaGraphExecDestroy(cache[victim].exec);
        cache[victim] = g;
    } else {
        cache.push_back(g);
    }
    GRIM_CUDA_TRY(cudaGraphLaunch(exec, s));
    return GRIM_OK;
}

int grim_autotune(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                  const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                  grim_tune* out, void* stream) {
    if (!out) return GRIM_EINVAL;
    int rc = check_args(bank, reads, read_offsets, n_reads, cand_bins, cand_offsets, E, pass);
    if (rc != GRIM_OK) return rc;
    *out = default_tune();
    if (n_reads == 0) return GRIM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const grim_tune d = default_tune();
    const int64_t n = n_reads < d.batch_reads ? n_reads : d.batch_reads;
    grim::GatherArgs a{reads, read_offsets, n, cand_bins, cand_offsets, E, pass, nullptr};
    grim_bank* mb = const_cast<grim_bank*>(bank);

    cudaEvent_t e0, e1;
    GRIM_CUDA_TRY(cudaEventCreate(&e0));
    GRIM_CUDA_TRY(cudaEventCreate(&e1));
    const int warps[2] = {8, 4};
    const int claims[3] = {1, 4, 16};
    const int per_sm[2] = {0, 2};
    float best_ms = 1e30f;
    grim_tune best = d;
    for (int w : warps)
        for (int c : claims)
            for (int p : per_sm) {
                grim_tune t = d;
                t.warps_per_cta = w;
                t.reads_per_claim = c;
                t.ctas_per_sm = p;
                t.use_graph = 0;
                rc = grim::launch_gather_batches(bank, a, t, &mb->counters[0], s);  // warm-up
                if (rc != GRIM_OK) break;
                float ms = 1e30f;
                for (int rep = 0; rep < 3 && rc == GRIM_OK; rep++) {
                    cudaEventRecord(e0, s);
                    rc = grim::launch_gather_batches(bank, a, t, &mb->counters[0], s);
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) rc = GRIM_ECUDA;
                    float x = 0;
                    cudaEventElapsedTime(&x, e0, e1);
                    ms = x < ms ? x : ms;
                }
                if (rc != GRIM_OK) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = t;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GRIM_OK) return rc;
    int64_t bounds[2] = {0, 0};
    GRIM_CUDA_TRY(cudaMemcpyAsync(&bounds[0], cand_offsets, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GRIM_CUDA_TRY(cudaMemcpyAsync(&bounds[1], cand_offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GRIM_CUDA_TRY(cudaStreamSynchronize(s));
    if (best_ms > 0 && bounds[1] > bounds[0])
        grim::record_gather_rate(bank, (bounds[1] - bounds[0]) / (best_ms * 1e-3));
    best.use_graph = 1;
    *out = best;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (bank->device >= 0 && bank->device < 64) {
        g_tuned[bank->device][bank->q] = best;
        g_has_tuned[bank->device][bank->q] = true;
    }
    return GRIM_OK;
}

}  // extern "C"
