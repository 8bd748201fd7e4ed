// The mapper's path around the filter as one overlapped pipeline: while the
// aligner works on the passing locations of one batch of reads, the filter
// produces the next batch's (the overlap of Sec. 4.2 / 6.1, where sequence
// alignment on the CPU proceeds while the Filter Bitmask Generator moves to
// the next bin window, with a double-buffered bitmask between them).
//
// Two streams and two buffer slots.  For batch k (slot k % 2):
//   filter stream: wait until the aligner has released the slot (batch
//   k - 2); seed candidates -> dispatcher -> Seed Location Checker, whose
//   locations land directly in the caller's output at a running offset;
//   record "filtered(slot)".
//   align stream: wait for "filtered(slot)"; edit distance of every
//   location of the batch; read ids made global; record "aligned(slot)".
// Candidate generation synchronises the filter stream (its scratch is sized
// on the host), so the host runs at most one batch ahead of the aligner.
#include "grim_internal.cuh"

namespace grim {
namespace {

__global__ void add_base_kernel(uint32_t* __restrict__ v, int64_t n, uint32_t base) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] += base;
}

struct Slot {
    uint32_t* cand = nullptr;
    int64_t* co = nullptr;
    uint8_t* pass = nullptr;
    int64_t* n_loc = nullptr;
    int64_t cap = 0;
    cudaEvent_t filtered = nullptr, aligned = nullptr;
};

}  // namespace
}  // namespace grim

extern "C" {

int grim_map(const grim_bank* bank, const grim_seed_index* idx, const uint8_t* ref2bit, const uint8_t* reads,
             const int64_t* read_offsets, int64_t n_reads, const uint16_t* E, int cap, int64_t batch_reads,
             uint32_t* loc_read, uint32_t* loc_bin, uint16_t* loc_dist, int64_t capacity, int64_t* n_loc,
             void* stream, void* align_stream) {
    if (!bank || !idx || !n_loc || n_reads < 0 || cap < 1 || capacity < 0) return GRIM_EINVAL;
    *n_loc = 0;
    if (n_reads == 0) return GRIM_OK;
    if (!ref2bit || !reads || !read_offsets || !E) return GRIM_EINVAL;
    if (capacity > 0 && (!loc_read || !loc_bin || !loc_dist)) return GRIM_EINVAL;
    if (n_reads > (int64_t)0xFFFFFFFFll) return GRIM_ENOTSUP;  // read ids are u32
    int rc = grim::check_device(bank);
    if (rc != GRIM_OK) return rc;
    if (batch_reads <= 0) batch_reads = int64_t(1) << 20;
    cudaStream_t sf = (cudaStream_t)stream;
    cudaStream_t sa = (cudaStream_t)align_stream;
    bool own_sa = false;
    cudaError_t e = cudaSuccess;
    if (!sa) {
        // the aligner's own stream at the lowest priority: the filter's
        // kernels go first when both streams have work
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sa, cudaStreamNonBlocking, least);
        if (e != cudaSuccess) {
            grim::set_last_cuda_error(e);
            return GRIM_ECUDA;
        }
        own_sa = true;
    }
    const int64_t max_nb = n_reads < batch_reads ? n_reads : batch_reads;
    // candidate room per slot: what earlier calls with this index needed
    // (and a quarter more), else 512 per read; a batch that needs more grows
    // the slot and is redone
    const int64_t hint = grim::seed_candidates_hint(idx, max_nb);
    const int64_t slot_cap = hint + hint / 4 > max_nb * 512 ? hint + hint / 4 : max_nb * 512;
    grim::Slot slot[2];
    for (int i = 0; i < 2 && e == cudaSuccess; i++) {
        slot[i].cap = slot_cap;
        e = grim::scratch_alloc((void**)&slot[i].cand, (size_t)slot[i].cap * 4, sf);
        if (e == cudaSuccess) e = grim::scratch_alloc((void**)&slot[i].pass, (size_t)slot[i].cap, sf);
        if (e == cudaSuccess) e = grim::scratch_alloc((void**)&slot[i].co, (size_t)(max_nb + 1) * 8, sf);
        if (e == cudaSuccess) e = grim::scratch_alloc((void**)&slot[i].n_loc, 8, sf);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&slot[i].filtered, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&slot[i].aligned, cudaEventDisableTiming);
    }
    int64_t written = 0;  // locations found so far: the next batch's output offset
    for (int64_t r0 = 0, k = 0; r0 < n_reads && e == cudaSuccess && rc == GRIM_OK; r0 += batch_reads, k++) {
        grim::Slot& sl = slot[k & 1];
        const int64_t nb = (n_reads - r0) < batch_reads ? (n_reads - r0) : batch_reads;
        if (k >= 2) e = cudaStreamWaitEvent(sf, sl.aligned, 0);  // the aligner is done with batch k - 2
        if (e != cudaSuccess) break;
        int64_t n_c = 0;
        rc = grim_seed_candidates(idx, reads, read_offsets + r0, nb, bank->bin_len, bank->n_bins, cap, sl.cand,
                                  sl.cap, sl.co, &n_c, sf);
        if (rc == GRIM_EOVERFLOW) {
            // grow this slot to the batch's need (and, on the first batch, the
            // other slot too, which is not in use yet), then redo the batch
            e = cudaStreamSynchronize(sa);
            for (int g = 0; g < (k == 0 ? 2 : 1) && e == cudaSuccess; g++) {
                grim::Slot& gs = g == 0 ? sl : slot[1];
                cudaFreeAsync(gs.cand, sf);
                cudaFreeAsync(gs.pass, sf);
                gs.cand = nullptr;
                gs.pass = nullptr;
                gs.cap = n_c + n_c / 4;
                e = grim::scratch_alloc((void**)&gs.cand, (size_t)gs.cap * 4, sf);
                if (e == cudaSuccess) e = grim::scratch_alloc((void**)&gs.pass, (size_t)gs.cap, sf);
            }
            if (e != cudaSuccess) break;
            rc = grim_seed_candidates(idx, reads, read_offsets + r0, nb, bank->bin_len, bank->n_bins, cap, sl.cand,
                                      sl.cap, sl.co, &n_c, sf);
        }
        if (rc != GRIM_OK) break;
        rc = grim_filter_auto(bank, reads, read_offsets + r0, nb, sl.cand, sl.co, E + r0, sl.pass, 0, nullptr, sf);
        if (rc != GRIM_OK) break;
        const int64_t room = capacity > written ? capacity - written : 0;
        rc = grim_locate(bank, nullptr, sl.cand, sl.co, nb, n_c, sl.pass, room ? loc_read + written : nullptr,
                         room ? loc_bin + written : nullptr, nullptr, nullptr, nullptr, 0, room, sl.n_loc, sf);
        if (rc != GRIM_OK) break;
        int64_t found = 0;
        e = cudaMemcpyAsync(&found, sl.n_loc, 8, cudaMemcpyDeviceToHost, sf);
        if (e == cudaSuccess) e = cudaEventRecord(sl.filtered, sf);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sf);
        if (e != cudaSuccess) break;
        const int64_t kept = found < room ? found : room;
        // the aligner's share of batch k, behind the filter's
        e = cudaStreamWaitEvent(sa, sl.filtered, 0);
        if (e == cudaSuccess && kept > 0) {
            rc = grim_verify(bank, ref2bit, reads, read_offsets + r0, nb, loc_read + written, loc_bin + written, kept,
                             loc_dist + written, sa);
            if (rc == GRIM_OK && r0 > 0) {
                const int64_t need = (kept + 255) / 256;
                const int64_t grid = (int64_t)grim::sm_count() * 8;
                grim::add_base_kernel<<<grim::fault_grid((unsigned)(need < grid ? need : grid)), 256, 0, sa>>>(
                        loc_read + written, kept, (uint32_t)r0);
                e = cudaGetLastError();
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(sl.aligned, sa);
        written += found;
    }
    cudaError_t e2 = cudaStreamSynchronize(sa);
    if (e == cudaSuccess) e = e2;
    for (int i = 0; i < 2; i++) {
        if (slot[i].cand) cudaFreeAsync(slot[i].cand, sf);
        if (slot[i].pass) cudaFreeAsync(slot[i].pass, sf);
        if (slot[i].co) cudaFreeAsync(slot[i].co, sf);
        if (slot[i].n_loc) cudaFreeAsync(slot[i].n_loc, sf);
    }
    e2 = cudaStreamSynchronize(sf);
    if (e == cudaSuccess) e = e2;
    for (int i = 0; i < 2; i++) {
        if (slot[i].filtered) cudaEventDestroy(slot[i].filtered);
        if (slot[i].aligned) cudaEventDestroy(slot[i].aligned);
    }
    if (own_sa) cudaStreamDestroy(sa);
    if (e != cudaSuccess) {
        grim::set_last_cuda_error(e);
        return e == cudaErrorMemoryAllocation ? GRIM_ENOMEM : GRIM_ECUDA;
    }
    if (rc != GRIM_OK) return rc;
    *n_loc = written;
    return written > capacity ? GRIM_EOVERFLOW : GRIM_OK;
}

}  // extern "C"
