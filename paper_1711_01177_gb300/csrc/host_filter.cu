// grim_filter from host memory: the reads and candidate lists are copied in,
// filtered and the pass bytes copied out in chunks of reads, with three
// streams so that the copies of one chunk overlap the filtering of another.
//
// Two device slots.  For chunk k (slot k % 2):
//   copy-in stream: wait until the filter is done with chunk k - 2 (its
//     inputs); copy bases and candidate bins; record "in(slot)" (the
//     offsets and E of every read are copied once, before the first chunk);
//   filter stream (the caller's): wait "in(slot)" and until chunk k - 2's
//     pass bytes have left (the slot's output); rebase the chunk's offsets
//     to the slot; gather; record "done(slot)";
//   copy-out stream: wait "done(slot)"; copy the pass bytes to the caller's
//     buffer; record "out(slot)".
#include <string.h>

#include <mutex>
#include <vector>

#include "grim_internal.cuh"

namespace grim {
namespace {

// the chunk's offsets, relative to its slot: ro[i] = ro_all[i] - ro_all[0]
__global__ void rebase_kernel(const int64_t* __restrict__ ro_all, const int64_t* __restrict__ co_all,
                              int64_t* __restrict__ ro, int64_t* __restrict__ co, int64_t n1, int64_t ro0,
                              int64_t co0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += (int64_t)gridDim.x * blockDim.x) {
        ro[i] = ro_all[i] - ro0;
        co[i] = co_all[i] - co0;
    }
}

struct HostSlot {
    uint8_t* reads = nullptr;
    int64_t* ro = nullptr;
    int64_t* co = nullptr;
    uint32_t* cb = nullptr;
    uint8_t* pass = nullptr;
    cudaEvent_t in = nullptr, done = nullptr, out = nullptr;
};

// The copy streams and events of one call.  Creating and destroying them
// costs tens of microseconds at both ends of every call, so each device
// keeps one set for reuse; a call that finds it in use (another host thread)
// makes its own.
struct CopyKit {
    cudaStream_t si = nullptr, so = nullptr;
    cudaEvent_t ev[7] = {};  // in, done, out of both slots; "ready"
    cudaError_t create() {
        cudaError_t e = cudaStreamCreateWithFlags(&si, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&so, cudaStreamNonBlocking);
        for (int i = 0; i < 7 && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        return e;
    }
    void destroy() {
        for (cudaEvent_t& v : ev)
            if (v) cudaEventDestroy(v), v = nullptr;
        if (si) cudaStreamDestroy(si), si = nullptr;
        if (so) cudaStreamDestroy(so), so = nullptr;
    }
};

std::mutex g_kit_mu[64];
CopyKit g_kit[64];

}  // namespace
}  // namespace grim

extern "C" {

int grim_filter_host(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                     const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                     int64_t chunk_reads, void* stream) {
    if (!bank || n_reads < 0) return GRIM_EINVAL;
    if (n_reads == 0) return GRIM_OK;
    if (!reads || !read_offsets || !cand_bins || !cand_offsets || !E || !pass) return GRIM_EINVAL;
    if (read_offsets[n_reads] < read_offsets[0] || cand_offsets[n_reads] < cand_offsets[0]) return GRIM_EINVAL;
    int rc = grim::check_device(bank);
    if (rc != GRIM_OK) return rc;
    // chunk boundaries: by default an eighth of the reads each, with the last
    // eighth cut in four so that little filtering is left once the copies in
    // (the critical path) have finished
    std::vector<int64_t> bounds{0};
    if (chunk_reads > 0) {
        for (int64_t r = chunk_reads; r < n_reads; r += chunk_reads) bounds.push_back(r);
    } else {
        const int64_t c = n_reads / 8 > 65536 ? (n_reads + 7) / 8 : 65536;
        int64_t r = 0;
        while (n_reads - r > c) bounds.push_back(r += c);
        const int64_t rest = n_reads - r, q4 = (rest + 3) / 4;
        if (rest >= 4 * 4096)
            for (int k = 1; k < 4; k++) bounds.push_back(r + k * q4);
    }
    bounds.push_back(n_reads);
    const int64_t n_chunks = (int64_t)bounds.size() - 1;
    // the largest chunk, in reads, bases and candidates (offsets are host memory here)
    int64_t max_nr = 1, max_bases = 1, max_cands = 1;
    for (int64_t c = 0; c < n_chunks; c++) {
        const int64_t r0 = bounds[c], r1 = bounds[c + 1];
        const int64_t nb = read_offsets[r1] - read_offsets[r0], nc = cand_offsets[r1] - cand_offsets[r0];
        if (nb < 0 || nc < 0) return GRIM_EINVAL;  // decreasing offsets across a chunk
        max_nr = r1 - r0 > max_nr ? r1 - r0 : max_nr;
        max_bases = nb > max_bases ? nb : max_bases;
        max_cands = nc > max_cands ? nc : max_cands;
    }
    cudaStream_t sf = (cudaStream_t)stream;
    // this device's cached streams and events when free, else a set of our own
    const int slot_dev = grim::device_slot();
    std::unique_lock<std::mutex> kit_lock;
    grim::CopyKit own, *kit = &own;
    cudaError_t e = cudaSuccess;
    if (slot_dev >= 0) {
        kit_lock = std::unique_lock<std::mutex>(grim::g_kit_mu[slot_dev], std::try_to_lock);
        if (kit_lock.owns_lock()) {
            kit = &grim::g_kit[slot_dev];
            if (!kit->si) e = kit->create();
            if (e != cudaSuccess) kit->destroy();
        }
    }
    if (kit == &own) e = own.create();
    cudaStream_t si = kit->si, so = kit->so;
    grim::HostSlot slot[2];
    int64_t *ro_all = nullptr, *co_all = nullptr;
    uint16_t* E_all = nullptr;
    if (e == cudaSuccess) e = grim::scratch_alloc((void**)&ro_all, (size_t)(n_reads + 1) * 8, sf);
    if (e == cudaSuccess) e = grim::scratch_alloc((void**)&co_all, (size_t)(n_reads + 1) * 8, sf);
    if (e == cudaSuccess) e = grim::scratch_alloc((void**)&E_all, (size_t)n_reads * 2, sf);
    for (int i = 0; i < 2 && e == cudaSuccess; i++) {
        grim::HostSlot& s = slot[i];
        e = grim::scratch_alloc((void**)&s.reads, (size_t)max_bases, sf);
        if (e == cudaSuccess) e = grim::scratch_alloc((void**)&s.ro, (size_t)(max_nr + 1) * 8, sf);
        if (e == cudaSuccess) e = grim::scratch_alloc((void**)&s.co, (size_t)(max_nr + 1) * 8, sf);
        if (e == cudaSuccess) e = grim::scratch_alloc((void**)&s.cb, (size_t)max_cands * 4, sf);
        if (e == cudaSuccess) e = grim::scratch_alloc((void**)&s.pass, (size_t)max_cands, sf);
        s.in = kit->ev[3 * i];
        s.done = kit->ev[3 * i + 1];
        s.out = kit->ev[3 * i + 2];
    }
    cudaEvent_t ready = kit->ev[6];  // the slots' memory exists on the filter stream
    if (e == cudaSuccess) e = cudaEventRecord(ready, sf);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(si, ready, 0);
    // every read's offsets and E, once
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ro_all, read_offsets, (size_t)(n_reads + 1) * 8, cudaMemcpyHostToDevice, si);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(co_all, cand_offsets, (size_t)(n_reads + 1) * 8, cudaMemcpyHostToDevice, si);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E_all, E, (size_t)n_reads * 2, cudaMemcpyHostToDevice, si);
    for (int64_t c = 0; c < n_chunks && e == cudaSuccess && rc == GRIM_OK; c++) {
        grim::HostSlot& s = slot[c & 1];
        const int64_t r0 = bounds[c], r1 = bounds[c + 1];
        const int64_t nr = r1 - r0;
        const int64_t ro0 = read_offsets[r0], co0 = cand_offsets[r0];
        const int64_t nb = read_offsets[r1] - ro0, nc = cand_offsets[r1] - co0;
        if (c >= 2) e = cudaStreamWaitEvent(si, s.done, 0);  // chunk c - 2 no longer reads the slot
        if (e == cudaSuccess && nb > 0)
            e = cudaMemcpyAsync(s.reads, reads + ro0, (size_t)nb, cudaMemcpyHostToDevice, si);
        if (e == cudaSuccess && nc > 0)
            e = cudaMemcpyAsync(s.cb, cand_bins + co0, (size_t)nc * 4, cudaMemcpyHostToDevice, si);
        if (e == cudaSuccess) e = cudaEventRecord(s.in, si);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sf, s.in, 0);
        if (e == cudaSuccess && c >= 2) e = cudaStreamWaitEvent(sf, s.out, 0);  // chunk c - 2's bytes have left
        if (e != cudaSuccess) break;
        const int64_t need = (nr + 1 + 255) / 256;
        grim::rebase_kernel<<<grim::fault_grid((unsigned)(need < 1024 ? need : 1024)), 256, 0, sf>>>(
                ro_all + r0, co_all + r0, s.ro, s.co, nr + 1, ro0, co0);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        rc = grim::launch_gather(bank, s.reads, s.ro, nr, s.cb, s.co, E_all + r0, s.pass, nullptr, sf);
        if (rc != GRIM_OK) break;
        e = cudaEventRecord(s.done, sf);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(so, s.done, 0);
        if (e == cudaSuccess && nc > 0) e = cudaMemcpyAsync(pass + co0, s.pass, (size_t)nc, cudaMemcpyDeviceToHost, so);
        if (e == cudaSuccess) e = cudaEventRecord(s.out, so);
    }
    // the caller's stream completes once every copy out has (a slot's "out"
    // event is recorded only when a chunk used the slot)
    for (int64_t i = 0; i < 2 && i < n_chunks; i++)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sf, slot[i].out, 0);
    cudaError_t e2 = so ? cudaStreamSynchronize(so) : cudaSuccess;
    if (e == cudaSuccess) e = e2;
    e2 = si ? cudaStreamSynchronize(si) : cudaSuccess;
    if (e == cudaSuccess) e = e2;
    for (int i = 0; i < 2; i++) {
        grim::HostSlot& s = slot[i];
        void* bufs[5] = {s.reads, s.ro, s.co, s.cb, s.pass};
        for (void* b : bufs)
            if (b) cudaFreeAsync(b, sf);
    }
    if (ro_all) cudaFreeAsync(ro_all, sf);
    if (co_all) cudaFreeAsync(co_all, sf);
    if (E_all) cudaFreeAsync(E_all, sf);
    e2 = cudaStreamSynchronize(sf);
    if (e == cudaSuccess) e = e2;
    // the cached set stays for the next call unless something failed
    if (kit == &own || e != cudaSuccess) kit->destroy();
    if (e != cudaSuccess) {
        grim::set_last_cuda_error(e);
        return e == cudaErrorMemoryAllocation ? GRIM_ENOMEM : GRIM_ECUDA;
    }
    return rc;
}

}  // extern "C"
