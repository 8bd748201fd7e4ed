// Internal definitions shared by the CUDA translation units of libgrim.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "grim.h"

namespace grim {
// A captured and instantiated CUDA graph of one batched-filter call.
struct GraphEntry {
    const void* key[8];
    int64_t n_reads;
    grim_tune tune;
    cudaStream_t stream;
    int slot;  // work counter owned by this graph
    cudaGraphExec_t exec;
    uint64_t last_use;
};
constexpr int kGraphCache = 15;  // counters: slot 0 for direct launches, 1..15 for graphs
}  // namespace grim

struct grim_bank {
    int64_t len;        // reference length in bases
    int64_t n_bins;     // ceil(len / bin_len)
    int64_t row_words;  // 32-bit words per bin row (>= 4, 16-byte rows)
    int q, bin_len, overlap;
    int device;
    uint32_t* bits;    // device, n_bins * row_words words, bin-major
    uint32_t* status;  // device, one word of GRIM_FLAG_* bits
    unsigned long long* counters;  // device, 1 + kGraphCache work counters of the batched filter
    std::vector<grim::GraphEntry>* graphs;
    uint64_t graph_clock;
};

namespace grim {

constexpr unsigned kFull = 0xffffffffu;

// Row geometry for token size Q: 4^Q bits per bin, rows padded to 16 bytes.
template <int Q>
struct Geo {
    static constexpr int kBits = 1 << (2 * Q);
    static constexpr int kRowWords = (kBits / 32) < 4 ? 4 : (kBits / 32);
};

// 16 bytes as a 16-bit mask of the nonzero ones (bit i = byte i): a byte
// b is nonzero iff bit 7 of ((b & 0x7F) + 0x7F) | b is set.
__device__ __forceinline__ uint32_t nonzero_bytes16(const uint4& v) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t b = (((w[k] & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w[k]) & 0x80808080u;
        m |= (((b >> 7) & 1u) | ((b >> 14) & 2u) | ((b >> 21) & 4u) | ((b >> 28) & 8u)) << (4 * k);
    }
    return m;
}

inline int64_t row_words_for(int q) {
    int64_t w = (int64_t(1) << (2 * q)) / 32;
    return w < 4 ? 4 : w;
}

// Stream-ordered working memory from the library's pool on the current
// device (freed with cudaFreeAsync; kept cached until grim_release_scratch).
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t s);

// Host-side fault injection (grim_fault_inject).  fault_alloc_now(): true
// when the allocation about to be made is the one armed to fail (the caller
// then allocates nothing and reports cudaErrorMemoryAllocation).
// fault_grid(blocks): the grid size of the launch about to be made -
// `blocks`, or 0 when this launch is the one armed to fail; the runtime
// rejects a zero grid (cudaErrorInvalidConfiguration) before anything runs
// on the device, so the launch's error check takes its real failure path.
bool fault_alloc_now();
unsigned fault_grid(unsigned blocks);

// Records the CUDA error of a failing call for grim_last_cuda_error.
void set_last_cuda_error(cudaError_t e);

// Current device must be the bank's device.
int check_device(const grim_bank* bank);

// A bank of the given geometry (rows unset, status cleared) and its release
// after a failed creation.
int new_bank(int64_t len, int q, int bin_len, int overlap, cudaStream_t s, grim_bank** out);
void delete_bank(grim_bank* bank);

int launch_bank_build(const uint8_t* ref2bit, grim_bank* bank, cudaStream_t stream);
int launch_gather(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                  const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                  uint16_t* sums, cudaStream_t stream);

struct GatherArgs {
    const uint8_t* reads;
    const int64_t* read_offsets;
    int64_t n_reads;
    const uint32_t* cand_bins;
    const int64_t* cand_offsets;
    const uint16_t* E;
    uint8_t* pass;
    uint16_t* sums;
};
// Gather launches over a.n_reads reads in batches of t.batch_reads (0 = one
// launch), shaped by t.warps_per_cta, t.ctas_per_sm and t.reads_per_claim.
// counter == nullptr: each CTA takes a cost-balanced read range; else the
// warps claim reads from *counter, zeroed before every launch.
int launch_gather_batches(const grim_bank* bank, const GatherArgs& a, const grim_tune& t,
                          unsigned long long* counter, cudaStream_t stream);

size_t scan_scratch_bytes(int q, int64_t n_reads);

// The autotuned launch shape for this bank's q on its device (defaults
// when grim_autotune has not run).
grim_tune tuned_shape(const grim_bank* bank);

// Gather rate (checks/s) measured by the autotuner, used by the dispatcher.
void record_gather_rate(const grim_bank* bank, double checks_per_s);
int launch_scan(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                const uint16_t* E, int64_t bin_begin, int64_t bin_end, uint32_t* pair_read, uint32_t* pair_bin,
                uint16_t* pair_sum, int64_t cap, int64_t* n_pairs, uint32_t* read_pass, void* scratch,
                cudaStream_t stream);

// Candidates that n_reads reads are expected to need, from the most per
// read that grim_seed_candidates has produced with this index (0 before
// its first call).
int64_t seed_candidates_hint(const grim_seed_index* idx, int64_t n_reads);

// Device address and size of the fixed scratch of grim_scan_noalloc
// (looked up once per device, with that device current).
int scan_noalloc_scratch(void** ptr, size_t* bytes);

// The full scan's bounded mbarrier wait run for limit_ns on a barrier that
// nothing completes; *timed_out (host) = 1 when it gave up as designed.
int launch_wait_selfcheck(unsigned long long limit_ns, cudaStream_t s, uint32_t* timed_out);

// The current device as an index into per-device caches (kernel attributes
// and occupancy are per device), or -1 when there is none below 64.
int device_slot();

// Number of SMs of the current device (cached per device).
int sm_count();

// Per-device caches of kernel attributes and occupancy are arrays of these:
// several host threads may make their first call on one device at the same
// time, so each entry is atomic (the work behind it is idempotent, and a
// thread that finds 0 simply repeats it).
using DeviceCache = std::atomic<int>;

}  // namespace grim

#define GRIM_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t grim_err_ = (expr);                       \
        if (grim_err_ != cudaSuccess) {                       \
            grim::set_last_cuda_error(grim_err_);             \
            return grim_err_ == cudaErrorMemoryAllocation     \
                       ? GRIM_ENOMEM                          \
                       : GRIM_ECUDA;                          \
        }                                                     \
    } while (0)
