// Host side of the C ABI: argument checks, bank ownership, status word,
// the library's scratch pool.
#include <string.h>

#include <stdlib.h>

#include <atomic>
#include <mutex>

#include "grim_internal.cuh"

namespace grim {

static thread_local int g_last_cuda_error = 0;

void set_last_cuda_error(cudaError_t e) { g_last_cuda_error = (int)e; }

int check_device(const grim_bank* bank) {
    int dev = -1;
    GRIM_CUDA_TRY(cudaGetDevice(&dev));
    return dev == bank->device ? GRIM_OK : GRIM_EINVAL;
}

int device_slot() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    return dev;
}

int sm_count() {
    static DeviceCache cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int n = cached[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cached[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

// Working memory of the entry points comes from one stream-ordered pool per
// device, owned by the library, whose release threshold keeps freed blocks
// cached: the default pool would hand them back to the driver at every
// synchronisation, and calls that allocate gigabytes of scratch would map
// them again each time.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];

static cudaMemPool_t scratch_pool(int dev) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

// Fault injection: one armed fault at a time, counted down by the matching
// events (allocations or kernel launches) of every thread; it fires once.
// GRIM_FAULT=alloc:N or launch:N in the environment arms it when the
// library is first used.
static std::atomic<int> g_fault_kind{-1};  // -1: environment not read yet
static std::atomic<long long> g_fault_left{0};

static void fault_env_once() {
    int expect = -1;
    if (g_fault_kind.load() != -1) return;
    int kind = GRIM_FAULT_NONE;
    long long n = 0;
    const char* v = getenv("GRIM_FAULT");
    if (v) {
        if (!strncmp(v, "alloc:", 6)) kind = GRIM_FAULT_ALLOC, n = atoll(v + 6);
        else if (!strncmp(v, "launch:", 7)) kind = GRIM_FAULT_LAUNCH, n = atoll(v + 7);
        if (n < 1) kind = GRIM_FAULT_NONE, n = 0;
    }
    g_fault_left.store(n);
    g_fault_kind.compare_exchange_strong(expect, kind);
}

static bool fault_hit(int kind) {
    fault_env_once();
    if (g_fault_kind.load(std::memory_order_relaxed) != kind) return false;
    const long long left = g_fault_left.fetch_sub(1) - 1;
    if (left != 0) return false;
    int k = kind;
    g_fault_kind.compare_exchange_strong(k, GRIM_FAULT_NONE);  // fired: disarm
    return true;
}

bool fault_alloc_now() { return fault_hit(GRIM_FAULT_ALLOC); }

unsigned fault_grid(unsigned blocks) { return fault_hit(GRIM_FAULT_LAUNCH) ? 0u : blocks; }

cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t s) {
    if (fault_alloc_now()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = scratch_pool(dev);
    if (!pool) return cudaMallocAsync(p, bytes, s);
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// A bank of the given geometry with unset rows and a cleared status word.
int new_bank(int64_t len, int q, int bin_len, int overlap, cudaStream_t s, grim_bank** out) {
    *out = nullptr;
    if (len < 1 || bin_len < 1 || overlap < 0) return GRIM_EINVAL;
    if (q < 1 || q > GRIM_MAX_Q) return GRIM_ENOTSUP;
    const int64_t n_bins = (len + bin_len - 1) / bin_len;
    if (n_bins > (int64_t)0xFFFFFFFFu) return GRIM_ENOTSUP;
    const int64_t rw = row_words_for(q);
    grim_bank* bank = new grim_bank();
    bank->len = len;
    bank->n_bins = n_bins;
    bank->row_words = rw;
    bank->q = q;
    bank->bin_len = bin_len;
    bank->overlap = overlap;
    if (cudaGetDevice(&bank->device) != cudaSuccess) {
        delete bank;
        return GRIM_ECUDA;
    }
    const size_t bytes = (size_t)n_bins * (size_t)rw * 4;
    const size_t tail = ((bytes + 255) & ~(size_t)255);  // status word, then the work counters
    void* mem = nullptr;
    cudaError_t e = fault_alloc_now() ? cudaErrorMemoryAllocation
                                      : cudaMalloc(&mem, tail + 256 + 8 * (1 + kGraphCache));
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        delete bank;
        return e == cudaErrorMemoryAllocation ? GRIM_ENOMEM : GRIM_ECUDA;
    }
    bank->bits = (uint32_t*)mem;
    bank->status = (uint32_t*)((char*)mem + tail);
    bank->counters = (unsigned long long*)((char*)mem + tail + 256);
    bank->graphs = new std::vector<GraphEntry>();
    bank->graph_clock = 0;
    e = cudaMemsetAsync(bank->status, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        delete_bank(bank);
        return GRIM_ECUDA;
    }
    *out = bank;
    return GRIM_OK;
}

// Releases a bank that no graph has been captured for (creation failures).
void delete_bank(grim_bank* bank) {
    cudaDeviceSynchronize();
    cudaFree(bank->bits);
    delete bank->graphs;
    delete bank;
}

namespace {

// E[r] = floor (or ceil) of num * L_r / den, saturated at 65535; L_r < 0 gives 0.
__global__ void fill_E_rate_kernel(const int64_t* __restrict__ read_offsets, int64_t n, int64_t num, int64_t den,
                                   bool round_up, uint16_t* __restrict__ E) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t L = __ldg(read_offsets + r + 1) - __ldg(read_offsets + r);
        L = L < 0 ? 0 : (L > GRIM_MAX_READ_LEN + 1 ? GRIM_MAX_READ_LEN + 1 : L);  // num * L < 2^48
        const int64_t e = (num * L + (round_up ? den - 1 : 0)) / den;
        E[r] = (uint16_t)(e > 65535 ? 65535 : e);
    }
}

}  // namespace
}  // namespace grim

extern "C" {

int grim_fill_E_rate(const int64_t* read_offsets, int64_t n_reads, int32_t num, int32_t den, int32_t round_up,
                     uint16_t* E, void* stream) {
    if (n_reads < 0 || num < 0 || den < 1) return GRIM_EINVAL;
    if (n_reads == 0) return GRIM_OK;
    if (!read_offsets || !E) return GRIM_EINVAL;
    const int64_t need = (n_reads + 255) / 256;
    const int64_t cap = (int64_t)grim::sm_count() * 8;
    grim::fill_E_rate_kernel<<<grim::fault_grid((unsigned)(need < cap ? need : cap)), 256, 0, (cudaStream_t)stream>>>(
        read_offsets, n_reads, num, den, round_up != 0, E);
    GRIM_CUDA_TRY(cudaGetLastError());
    return GRIM_OK;
}

const char* grim_strerror(int status) {
    switch (status) {
        case GRIM_OK: return "ok";
        case GRIM_EINVAL: return "invalid argument";
        case GRIM_EDATA: return "invalid input data found on the device";
        case GRIM_ENOMEM: return "device allocation failed";
        case GRIM_ECUDA: return "CUDA runtime error";
        case GRIM_EOVERFLOW: return "output capacity exceeded";
        case GRIM_ETIMEOUT: return "bounded device-side wait ran out";
        case GRIM_ENOTSUP: return "parameters not supported by the kernels";
        case GRIM_ESCRATCH: return "request exceeds the fixed scratch of the allocation-free scan";
        case GRIM_EIO: return "bank file could not be written or is not a valid bank file";
        default: return "unknown status";
    }
}

int grim_last_cuda_error(void) { return grim::g_last_cuda_error; }

int grim_fault_inject(int kind, int64_t nth) {
    grim::fault_env_once();
    if (kind == GRIM_FAULT_NONE) {
        grim::g_fault_kind.store(GRIM_FAULT_NONE);
        grim::g_fault_left.store(0);
        return GRIM_OK;
    }
    if ((kind != GRIM_FAULT_ALLOC && kind != GRIM_FAULT_LAUNCH) || nth < 1) return GRIM_EINVAL;
    grim::g_fault_kind.store(GRIM_FAULT_NONE);  // no event counts against a half-armed fault
    grim::g_fault_left.store(nth);
    grim::g_fault_kind.store(kind);
    return GRIM_OK;
}

int grim_fault_pending(int64_t* left) {
    grim::fault_env_once();
    const int kind = grim::g_fault_kind.load();
    if (left) *left = kind == GRIM_FAULT_NONE ? 0 : (int64_t)grim::g_fault_left.load();
    return kind;
}

int grim_wait_selfcheck(unsigned long long limit_ns, void* stream) {
    uint32_t timed_out = 0;
    const int rc = grim::launch_wait_selfcheck(limit_ns, (cudaStream_t)stream, &timed_out);
    if (rc != GRIM_OK) return rc;
    return timed_out ? GRIM_ETIMEOUT : GRIM_OK;
}

int grim_release_scratch(void) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GRIM_ECUDA;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(grim::g_pool_mu);
        if (dev >= 0 && dev < 64) pool = grim::g_pool[dev];
    }
    if (!pool) return GRIM_OK;
    GRIM_CUDA_TRY(cudaDeviceSynchronize());
    GRIM_CUDA_TRY(cudaMemPoolTrimTo(pool, 0));
    return GRIM_OK;
}

int grim_build_bank(const uint8_t* ref2bit, int64_t len, int q, int bin_len, int overlap, void* stream,
                    grim_bank** out) {
    if (!out) return GRIM_EINVAL;
    *out = nullptr;
    if (!ref2bit) return GRIM_EINVAL;
    grim_bank* bank = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = grim::new_bank(len, q, bin_len, overlap, s, &bank);
    if (rc != GRIM_OK) return rc;
    rc = grim::launch_bank_build(ref2bit, bank, s);
    if (rc != GRIM_OK) {
        grim::delete_bank(bank);
        return rc;
    }
    *out = bank;
    return GRIM_OK;
}

int grim_build_bank_into(grim_bank* bank, const uint8_t* ref2bit, void* stream) {
    if (!bank || !ref2bit) return GRIM_EINVAL;
    const int rc = grim::check_device(bank);
    if (rc != GRIM_OK) return rc;
    return grim::launch_bank_build(ref2bit, bank, (cudaStream_t)stream);
}

int grim_bank_info(const grim_bank* bank, int64_t* len, int64_t* n_bins, int* q, int* bin_len, int* overlap,
                   int64_t* row_words, const uint32_t** bits) {
    if (!bank) return GRIM_EINVAL;
    if (len) *len = bank->len;
    if (n_bins) *n_bins = bank->n_bins;
    if (q) *q = bank->q;
    if (bin_len) *bin_len = bank->bin_len;
    if (overlap) *overlap = bank->overlap;
    if (row_words) *row_words = bank->row_words;
    if (bits) *bits = bank->bits;
    return GRIM_OK;
}

int grim_bank_status(grim_bank* bank, void* stream, uint32_t* flags) {
    if (!bank) return GRIM_EINVAL;
    int rc = grim::check_device(bank);
    if (rc != GRIM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t f = 0;
    GRIM_CUDA_TRY(cudaStreamSynchronize(s));
    GRIM_CUDA_TRY(cudaMemcpyAsync(&f, bank->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GRIM_CUDA_TRY(cudaMemsetAsync(bank->status, 0, sizeof(uint32_t), s));
    GRIM_CUDA_TRY(cudaStreamSynchronize(s));
    if (flags) *flags = f;
    if (f & (GRIM_FLAG_BAD_BASE | GRIM_FLAG_BAD_BIN | GRIM_FLAG_BAD_OFFSETS | GRIM_FLAG_LONG_READ))
        return GRIM_EDATA;
    if (f & GRIM_FLAG_OVERFLOW) return GRIM_EOVERFLOW;
    if (f & GRIM_FLAG_TIMEOUT) return GRIM_ETIMEOUT;
    return GRIM_OK;
}

int grim_bank_free(grim_bank* bank) {
    if (!bank) return GRIM_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != bank->device) cudaSetDevice(bank->device);
    cudaError_t e1 = cudaDeviceSynchronize();
    if (bank->graphs) {
        for (grim::GraphEntry& g : *bank->graphs) cudaGraphExecDestroy(g.exec);
        delete bank->graphs;
    }
    cudaError_t e2 = cudaFree(bank->bits);
    if (prev >= 0 && prev != bank->device) cudaSetDevice(prev);
    delete bank;
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        grim::set_last_cuda_error(e1 != cudaSuccess ? e1 : e2);
        return GRIM_ECUDA;
    }
    return GRIM_OK;
}

int grim_filter(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                uint16_t* sums, void* stream) {
    if (!bank || n_reads < 0) return GRIM_EINVAL;
    if (n_reads == 0) return GRIM_OK;
    if (!reads || !read_offsets || !cand_bins || !cand_offsets || !E || !pass) return GRIM_EINVAL;
    int rc = grim::check_device(bank);
    if (rc != GRIM_OK) return rc;
    return grim::launch_gather(bank, reads, read_offsets, n_reads, cand_bins, cand_offsets, E, pass, sums,
                               (cudaStream_t)stream);
}

int grim_scan(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
              const uint16_t* E, int64_t bin_begin, int64_t bin_end, uint32_t* pair_read, uint32_t* pair_bin,
              uint16_t* pair_sum, int64_t cap, int64_t* n_pairs, uint32_t* read_pass, void* stream) {
    if (!bank || n_reads < 0 || cap < 0 || !n_pairs) return GRIM_EINVAL;
    if (bin_begin < 0 || bin_end > bank->n_bins || bin_begin > bin_end) return GRIM_EINVAL;
    if (cap > 0 && (!pair_read || !pair_bin)) return GRIM_EINVAL;
    if (bank->q > GRIM_MAX_SCAN_Q) return GRIM_ENOTSUP;
    if (n_reads > ((int64_t)1 << 30)) return GRIM_ENOTSUP;
    int rc = grim::check_device(bank);
    if (rc != GRIM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_reads == 0 || bin_begin == bin_end) {
        GRIM_CUDA_TRY(cudaMemsetAsync(n_pairs, 0, sizeof(int64_t), s));
        if (read_pass && n_reads > 0) GRIM_CUDA_TRY(cudaMemsetAsync(read_pass, 0, (size_t)n_reads * 4, s));
        return GRIM_OK;
    }
    if (!reads || !read_offsets || !E) return GRIM_EINVAL;
    void* scratch = nullptr;
    GRIM_CUDA_TRY(grim::scratch_alloc(&scratch, grim::scan_scratch_bytes(bank->q, n_reads), s));
    rc = grim::launch_scan(bank, reads, read_offsets, n_reads, E, bin_begin, bin_end, pair_read, pair_bin, pair_sum,
                           cap, n_pairs, read_pass, scratch, s);
    cudaError_t e = cudaFreeAsync(scratch, s);
    if (rc != GRIM_OK) return rc;
    GRIM_CUDA_TRY(e);
    return GRIM_OK;
}

int grim_scan_noalloc(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                      const uint16_t* E, int64_t bin_begin, int64_t bin_end, uint32_t* pair_read, uint32_t* pair_bin,
                      uint16_t* pair_sum, int64_t cap, int64_t* n_pairs, uint32_t* read_pass, void* stream) {
    if (!bank || n_reads < 0 || cap < 0 || !n_pairs) return GRIM_EINVAL;
    if (bin_begin < 0 || bin_end > bank->n_bins || bin_begin > bin_end) return GRIM_EINVAL;
    if (cap > 0 && (!pair_read || !pair_bin)) return GRIM_EINVAL;
    if (bank->q > GRIM_MAX_SCAN_Q) return GRIM_ENOTSUP;
    if (n_reads > ((int64_t)1 << 30)) return GRIM_ESCRATCH;
    int rc = grim::check_device(bank);
    if (rc != GRIM_OK) return rc;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    rc = grim::scan_noalloc_scratch(&scratch, &scratch_bytes);
    if (rc != GRIM_OK) return rc;
    if (grim::scan_scratch_bytes(bank->q, n_reads) > scratch_bytes) return GRIM_ESCRATCH;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_reads == 0 || bin_begin == bin_end) {
        GRIM_CUDA_TRY(cudaMemsetAsync(n_pairs, 0, sizeof(int64_t), s));
        if (read_pass && n_reads > 0) GRIM_CUDA_TRY(cudaMemsetAsync(read_pass, 0, (size_t)n_reads * 4, s));
        return GRIM_OK;
    }
    if (!reads || !read_offsets || !E) return GRIM_EINVAL;
    return grim::launch_scan(bank, reads, read_offsets, n_reads, E, bin_begin, bin_end, pair_read, pair_bin, pair_sum,
                             cap, n_pairs, read_pass, scratch, s);
}

}  // extern "C"
