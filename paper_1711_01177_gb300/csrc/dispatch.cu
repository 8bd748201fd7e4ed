// Per-batch choice between the gather form and the full scan, by candidate
// density.  The gather form costs about n_checks rows; the full scan costs
// n_reads x n_bins contractions no matter how few candidates there are, so
// it only wins when candidate lists cover a large share of the bins.  When
// the scan is chosen, its passing (read, bin) list is turned back into the
// per-candidate mask with a device hash join, so both forms give the same
// bytes.
#include <mutex>
#include <vector>

#include "grim_internal.cuh"

namespace grim {

constexpr int kJoinThreads = 256;

namespace {

std::mutex g_rate_mu;
double g_gather_rate[64][GRIM_MAX_Q + 1];  // measured checks/s, 0 = not measured

constexpr uint64_t kEmpty = ~0ull;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// passing pairs -> open-addressing set of (read << 32 | bin)
// bounds[i] = cand_offsets[min(i * batch_reads, n_reads)] for i <= n_batches:
// every batch's first candidate and the end of the last.
__global__ void batch_bounds_kernel(const int64_t* __restrict__ cand_offsets, int64_t n_reads, int64_t batch_reads,
                                    int64_t n_batches, int64_t* __restrict__ bounds) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n_batches) return;
    const int64_t r = i * batch_reads < n_reads ? i * batch_reads : n_reads;
    bounds[i] = cand_offsets[r];
}

__global__ void join_insert_kernel(const uint32_t* __restrict__ pr, const uint32_t* __restrict__ pb, int64_t n,
                                   uint64_t r0, unsigned long long* __restrict__ table, uint64_t mask) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = ((uint64_t)pr[i] + r0) << 32 | pb[i];
        uint64_t h = mix64(key) & mask;
        for (uint64_t probe = 0; probe <= mask; probe++) {
            const unsigned long long old = atomicCAS(&table[h], (unsigned long long)kEmpty, key);
            if (old == kEmpty || old == key) break;
            h = (h + 1) & mask;
        }
    }
}

// one thread per candidate of the batch: pass = (read, bin) in the set
__global__ void join_lookup_kernel(const int64_t* __restrict__ cand_offsets, int64_t n_reads, int64_t r0,
                                   const uint32_t* __restrict__ cand_bins, int64_t n_bins,
                                   const unsigned long long* __restrict__ table, uint64_t mask,
                                   uint8_t* __restrict__ pass, uint32_t* __restrict__ status) {
    // warp per read
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    uint32_t flags = 0;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_reads; r += warps) {
        const int64_t co = cand_offsets[r], ce = cand_offsets[r + 1];
        for (int64_t c = co + lane; c < ce; c += 32) {
            const uint32_t b = cand_bins[c];
            if ((int64_t)b >= n_bins) {
                flags |= GRIM_FLAG_BAD_BIN;
                pass[c] = 0;
                continue;
            }
            const uint64_t key = ((uint64_t)(r + r0)) << 32 | b;
            uint64_t h = mix64(key) & mask;
            uint8_t hit = 0;
            for (uint64_t probe = 0; probe <= mask; probe++) {
                const unsigned long long v = table[h];
                if (v == key) {
                    hit = 1;
                    break;
                }
                if (v == kEmpty) break;
                h = (h + 1) & mask;
            }
            pass[c] = hit;
        }
    }
    flags = __reduce_or_sync(0xffffffffu, flags);
    if (lane == 0 && flags) atomicOr(status, flags);
}

// Modelled seconds of each form for a batch.
void form_costs(const grim_bank* bank, int64_t n_reads, int64_t n_checks, double* t_gather, double* t_scan) {
    const double row_bytes = (double)bank->row_words * 4.0;
    double rg = 0;
    {
        std::lock_guard<std::mutex> lock(g_rate_mu);
        if (bank->device >= 0 && bank->device < 64) rg = g_gather_rate[bank->device][bank->q];
    }
    if (rg <= 0) {
        // not measured: HBM-bound rows when the bank exceeds L2, else an issue-bound rate
        const double bank_bytes = (double)bank->n_bins * row_bytes;
        rg = bank_bytes > 96e6 ? 6.0e12 / (row_bytes + 5.0) : 3.5e10;
    }
    // full scan: 2 * 4^q flops per check on the FP4 (mxf4) tensor path at ~4.5e15 flops/s
    const double rs = bank->q <= GRIM_MAX_SCAN_Q ? 4.5e15 / (2.0 * (double)(int64_t(1) << (2 * bank->q))) : 0.0;
    *t_gather = (double)n_checks / rg + (double)n_reads * 2e-10;
    *t_scan = rs > 0 ? (double)n_reads * (double)bank->n_bins / rs + 50e-6 : 1e30;
}

}  // namespace

void record_gather_rate(const grim_bank* bank, double checks_per_s) {
    std::lock_guard<std::mutex> lock(g_rate_mu);
    if (bank->device >= 0 && bank->device < 64) g_gather_rate[bank->device][bank->q] = checks_per_s;
}

}  // namespace grim

extern "C" {

int grim_choose_form(const grim_bank* bank, int64_t n_reads, int64_t n_checks, int* form) {
    if (!bank || !form || n_reads < 0 || n_checks < 0) return GRIM_EINVAL;
    double tg, ts;
    grim::form_costs(bank, n_reads, n_checks, &tg, &ts);
    *form = ts < tg ? GRIM_FORM_SCAN : GRIM_FORM_GATHER;
    return GRIM_OK;
}

int grim_filter_auto(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                     const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                     int64_t batch_reads, int64_t* n_scanned, void* stream) {
    if (!bank || n_reads < 0) return GRIM_EINVAL;
    if (n_scanned) *n_scanned = 0;
    if (n_reads == 0) return GRIM_OK;
    if (!reads || !read_offsets || !cand_bins || !cand_offsets || !E || !pass) return GRIM_EINVAL;
    int rc = grim::check_device(bank);
    if (rc != GRIM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (batch_reads <= 0) batch_reads = 262144;
    // the autotuned shape, launched directly (each batch's pointers differ,
    // so a graph per batch would only churn the bank's graph cache)
    grim_tune t = grim::tuned_shape(bank);
    t.use_graph = 0;
    // every batch's candidate count with one copy and one synchronisation
    const int64_t n_batches = (n_reads + batch_reads - 1) / batch_reads;
    std::vector<int64_t> bounds((size_t)n_batches + 1);
    {
        int64_t* bd = nullptr;
        GRIM_CUDA_TRY(grim::scratch_alloc((void**)&bd, (size_t)(n_batches + 1) * 8, s));
        const int64_t nb = (n_batches + 1 + 255) / 256;
        grim::batch_bounds_kernel<<<grim::fault_grid((unsigned)nb), 256, 0, s>>>(cand_offsets, n_reads, batch_reads,
                                                                                n_batches, bd);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bounds.data(), bd, (size_t)(n_batches + 1) * 8, cudaMemcpyDeviceToHost, s);
        cudaFreeAsync(bd, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            grim::set_last_cuda_error(e);
            return GRIM_ECUDA;
        }
    }
    // consecutive gathered batches run as one persistent launch (no tail and
    // no host round trip between them); scanned batches one by one
    int64_t run0 = -1;  // first read of the pending run of gathered batches
    auto flush = [&](int64_t r_end) -> int {
        if (run0 < 0) return GRIM_OK;
        const int64_t n = r_end - run0;
        t.batch_reads = n;
        const int r = grim_filter_batched(bank, reads, read_offsets + run0, n, cand_bins, cand_offsets + run0,
                                          E + run0, pass, nullptr, &t, stream);
        run0 = -1;
        return r;
    };
    for (int64_t b = 0; b < n_batches; b++) {
        const int64_t r0 = b * batch_reads;
        const int64_t n = (n_reads - r0) < batch_reads ? (n_reads - r0) : batch_reads;
        int form = GRIM_FORM_GATHER;
        grim_choose_form(bank, n, bounds[b + 1] - bounds[b], &form);
        bool done = false;
        if (form == GRIM_FORM_SCAN) {
            rc = flush(r0);
            if (rc != GRIM_OK) return rc;
            // scan the batch over every bin; join its pairs back onto the candidates
            const int64_t cap = 1 << 24;
            size_t table_n = 1;
            while (table_n < 2 * (size_t)cap) table_n <<= 1;
            uint8_t* mem = nullptr;
            const size_t bytes = (size_t)cap * 8 + 256 + table_n * 8;
            GRIM_CUDA_TRY(grim::scratch_alloc((void**)&mem, bytes, s));
            uint32_t* pr = (uint32_t*)mem;
            uint32_t* pb = pr + cap;
            int64_t* np_dev = (int64_t*)(mem + (size_t)cap * 8);
            unsigned long long* table = (unsigned long long*)(mem + (size_t)cap * 8 + 256);
            rc = grim_scan(bank, reads, read_offsets + r0, n, E + r0, 0, bank->n_bins, pr, pb, nullptr, cap, np_dev,
                           nullptr, stream);
            int64_t np = 0;
            if (rc == GRIM_OK) {
                cudaMemcpyAsync(&np, np_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
                cudaStreamSynchronize(s);
            }
            if (rc == GRIM_OK && np <= cap) {
                cudaMemsetAsync(table, 0xFF, table_n * 8, s);
                const int64_t ib = (np + grim::kJoinThreads - 1) / grim::kJoinThreads;
                if (np > 0)
                    grim::join_insert_kernel<<<grim::fault_grid((unsigned)(ib < 65535 ? ib : 65535)),
                                               grim::kJoinThreads, 0, s>>>(pr, pb, np, 0, table, table_n - 1);
                const int64_t lb = (n * 32 + grim::kJoinThreads - 1) / grim::kJoinThreads;
                grim::join_lookup_kernel<<<grim::fault_grid((unsigned)(lb < 65535 ? lb : 65535)), grim::kJoinThreads,
                                           0, s>>>(cand_offsets + r0, n, 0, cand_bins, bank->n_bins, table,
                                                   table_n - 1, pass, bank->status);
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) {
                    grim::set_last_cuda_error(e);
                    rc = GRIM_ECUDA;
                }
                done = rc == GRIM_OK;
                if (done && n_scanned) *n_scanned += n;
            }
            cudaFreeAsync(mem, s);
            if (rc != GRIM_OK) return rc;
        }
        // a gathered batch (or a scan whose pairs overflowed) joins the run
        if (!done && run0 < 0) run0 = r0;
    }
    rc = flush(n_reads);
    if (rc != GRIM_OK) return rc;
    return GRIM_OK;
}

}  // extern "C"
