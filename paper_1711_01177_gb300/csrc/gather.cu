// Gather-form filter (Sec. 3.2 steps 1-5 for every (read, candidate bin)).
//
// The accumulation sum of read r in bin b is the number of r's token
// positions whose existence bit is set in b.  Grouping equal tokens, it is
// sum_t count_r(t) * bit_b(t): a dot product of the read's token-count
// vector with the bin's bitvector.  Writing the counts in binary,
// count_r(t) = sum_p 2^p * plane_p(t), turns it into
//     Sum(r, b) = sum_p 2^p * popcount(plane_p AND row_b),
// exact integer arithmetic over whole 32-bit words instead of one bit test
// per token.  Reads of 100-150 bases need two or three planes.
//
// One warp per read (grid-stride over reads):
//   1. lanes load 32 bases at a time and roll each lane's token out of the
//      q following bases with warp shuffles (the q-gram window of Sec. 3.2
//      step 1);
//   2. each token is added to the read's bit-sliced count planes in shared
//      memory with a carry chain of atomicXor (bit p flips; a bit that was
//      set carries into plane p+1);
//   3. every lane keeps its 16-byte slice of the first four planes in
//      registers;
//   4. candidate rows are fetched as 16-byte vectors, lanes_per_bin lanes
//      per row (8 for q=5: one 128-byte row per 8 lanes, 4 rows per warp
//      step, 8 steps = 32 rows in flight per warp), ANDed with the planes,
//      popcounted, reduced with xor-shuffles, compared with the threshold;
//   5. the 32 results of a batch are gathered into lane order and stored as
//      one coalesced run of pass bytes (and sums).
#include "grim_internal.cuh"

namespace grim {

constexpr int kGatherWarps = 8;
constexpr int kPlanes = 16;    // sums and counts stay below 2^16
constexpr int kRegPlanes = 4;  // planes held in registers; more go through shared memory

template <int Q>
struct GatherGeo {
    static constexpr int kRowWords = Geo<Q>::kRowWords;
    static constexpr int kLanesPerBin = kRowWords / 4;
    static constexpr int kBinsPerStep = 32 / kLanesPerBin;
    static constexpr int kSteps = (8 * kBinsPerStep) <= 32 ? 8 : (32 / kBinsPerStep);
    static constexpr int kBatch = kSteps * kBinsPerStep;  // <= 32 candidates per batch
    static_assert(kLanesPerBin >= 1 && kLanesPerBin <= 32, "row must fit one warp of 16-byte slices");
};

__device__ __forceinline__ uint32_t and_popc(const uint4& a, const uint4& b) {
    return __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
}

template <int Q>
__global__ void __launch_bounds__(kGatherWarps * 32)
gather_kernel(const uint32_t* __restrict__ bank, int64_t n_bins, const uint8_t* __restrict__ reads,
              const int64_t* __restrict__ read_offsets, int64_t n_reads, const uint32_t* __restrict__ cand_bins,
              const int64_t* __restrict__ cand_offsets, const uint16_t* __restrict__ E,
              uint8_t* __restrict__ pass, uint16_t* __restrict__ sums, uint32_t* __restrict__ status) {
    using G = GatherGeo<Q>;
    constexpr int RW = G::kRowWords;
    extern __shared__ uint4 gather_smem[];  // kGatherWarps x kPlanes x RW words

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int slice = lane % G::kLanesPerBin;  // which 16-byte slice of a row this lane handles
    uint32_t* planes = reinterpret_cast<uint32_t*>(gather_smem) + warp * (kPlanes * RW);
    for (int i = lane; i < kPlanes * RW; i += 32) planes[i] = 0;
    __syncwarp();

    uint32_t flags = 0;
    const int64_t warp_stride = (int64_t)gridDim.x * kGatherWarps;
    for (int64_t r = (int64_t)blockIdx.x * kGatherWarps + warp; r < n_reads; r += warp_stride) {
        const int64_t ro = read_offsets[r], re = read_offsets[r + 1];
        const int64_t co = cand_offsets[r], ce = cand_offsets[r + 1];
        if (ce < co) {  // nothing sensible to write for this read
            flags |= GRIM_FLAG_BAD_OFFSETS;
            continue;
        }
        bool bad_read = false;
        int L = 0;
        if (re < ro) {
            flags |= GRIM_FLAG_BAD_OFFSETS;
            bad_read = true;
        } else if (re - ro > GRIM_MAX_READ_LEN) {
            flags |= GRIM_FLAG_LONG_READ;
            bad_read = true;
        } else {
            L = (int)(re - ro);
        }
        const uint8_t* rd = reads + ro;

        // steps 1-2: tokens into bit-sliced count planes
        uint32_t bad_base = 0;
        int top = -1;  // highest plane this lane set
        uint32_t cur = (lane < L) ? rd[lane] : 0u;
        for (int c0 = 0; c0 < L; c0 += 32) {
            const int i = c0 + lane;
            const uint32_t nxt = (i + 32 < L) ? rd[i + 32] : 0u;
            bad_base |= (uint32_t)((i < L) && (cur > 3u));
            uint32_t tok = 0;
#pragma unroll
            for (int k = 0; k < Q; k++) {
                const int src = lane + k;
                const uint32_t a = __shfl_sync(kFull, cur, src & 31);
                const uint32_t b = __shfl_sync(kFull, nxt, src & 31);
                tok = (tok << 2) | (((src < 32) ? a : b) & 3u);
            }
            if (i + Q <= L) {
                const uint32_t w = tok >> 5, m = 1u << (tok & 31);
                int p = 0;
                while (p < kPlanes) {
                    const uint32_t old = atomicXor(&planes[p * RW + w], m);
                    if (!(old & m)) break;
                    ++p;
                }
                top = p > top ? p : top;
            }
            cur = nxt;
        }
        const int used = (int)__reduce_max_sync(kFull, (unsigned)(top + 1));
        if (__any_sync(kFull, bad_base)) {
            flags |= GRIM_FLAG_BAD_BASE;
            bad_read = true;
        }
        __syncwarp();
        const int P = bad_read ? 0 : used;
        const int n_tok = L - Q + 1 > 0 ? L - Q + 1 : 0;
        const int T = n_tok - Q * (int)E[r];

        // step 3: this lane's slices of the low planes
        uint4 pl[kRegPlanes];
#pragma unroll
        for (int p = 0; p < kRegPlanes; p++)
            pl[p] = (p < P) ? *reinterpret_cast<const uint4*>(&planes[p * RW + 4 * slice]) : make_uint4(0, 0, 0, 0);

        // steps 4-5 over the candidate list
        for (int64_t cb = co; cb < ce; cb += G::kBatch) {
            const int cnt = (ce - cb) < G::kBatch ? (int)(ce - cb) : G::kBatch;
            const uint32_t my_bin = (lane < cnt) ? cand_bins[cb + lane] : 0u;
            uint4 v[G::kSteps];
#pragma unroll
            for (int t = 0; t < G::kSteps; t++) {
                const int j = t * G::kBinsPerStep + lane / G::kLanesPerBin;
                const uint32_t b = __shfl_sync(kFull, my_bin, j & 31);
                v[t] = make_uint4(0, 0, 0, 0);
                if (j < cnt && b < n_bins)
                    v[t] = __ldg(reinterpret_cast<const uint4*>(bank + (size_t)b * RW) + slice);
            }
            uint32_t mine = 0;
#pragma unroll
            for (int t = 0; t < G::kSteps; t++) {
                uint32_t part = 0;
#pragma unroll
                for (int p = 0; p < kRegPlanes; p++)
                    if (p < P) part += and_popc(v[t], pl[p]) << p;
                for (int p = kRegPlanes; p < P; p++)
                    part += and_popc(v[t], *reinterpret_cast<const uint4*>(&planes[p * RW + 4 * slice])) << p;
#pragma unroll
                for (int o = G::kLanesPerBin / 2; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
                const uint32_t got = __shfl_sync(kFull, part, (lane % G::kBinsPerStep) * G::kLanesPerBin);
                if (lane / G::kBinsPerStep == t) mine = got;
            }
            if (lane < cnt) {
                const bool in_range = my_bin < n_bins;
                if (!in_range) flags |= GRIM_FLAG_BAD_BIN;
                const uint32_t sum = (in_range && !bad_read) ? mine : 0u;
                pass[cb + lane] = (in_range && !bad_read && (int)sum >= T) ? 1 : 0;
                if (sums) sums[cb + lane] = (uint16_t)sum;
            }
        }

        // leave the planes zeroed for the warp's next read
        __syncwarp();
        for (int i = lane; i < used * RW; i += 32) planes[i] = 0;
        __syncwarp();
    }
    flags = __reduce_or_sync(kFull, flags);
    if (lane == 0 && flags) atomicOr(status, flags);
}

template <int Q>
static int launch_q(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                    const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                    uint16_t* sums, cudaStream_t s) {
    constexpr size_t smem = (size_t)kGatherWarps * kPlanes * Geo<Q>::kRowWords * 4;
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        if (smem > 48 * 1024)
            GRIM_CUDA_TRY(cudaFuncSetAttribute(gather_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
        int b = 0;
        GRIM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gather_kernel<Q>, kGatherWarps * 32, smem));
        blocks_per_sm = b > 0 ? b : 1;
    }
    const int64_t need = (n_reads + kGatherWarps - 1) / kGatherWarps;
    const int64_t cap = (int64_t)sm_count() * blocks_per_sm * 8;
    const int64_t blocks = need < cap ? need : cap;
    gather_kernel<Q><<<(unsigned)blocks, kGatherWarps * 32, smem, s>>>(bank->bits, bank->n_bins, reads, read_offsets,
                                                                    n_reads, cand_bins, cand_offsets, E, pass, sums,
                                                                    bank->status);
    GRIM_CUDA_TRY(cudaGetLastError());
    return GRIM_OK;
}

int launch_gather(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                  const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                  uint16_t* sums, cudaStream_t s) {
    switch (bank->q) {
        case 1: return launch_q<1>(bank, reads, read_offsets, n_reads, cand_bins, cand_offsets, E, pass, sums, s);
        case 2: return launch_q<2>(bank, reads, read_offsets, n_reads, cand_bins, cand_offsets, E, pass, sums, s);
        case 3: return launch_q<3>(bank, reads, read_offsets, n_reads, cand_bins, cand_offsets, E, pass, sums, s);
        case 4: return launch_q<4>(bank, reads, read_offsets, n_reads, cand_bins, cand_offsets, E, pass, sums, s);
        case 5: return launch_q<5>(bank, reads, read_offsets, n_reads, cand_bins, cand_offsets, E, pass, sums, s);
        case 6: return launch_q<6>(bank, reads, read_offsets, n_reads, cand_bins, cand_offsets, E, pass, sums, s);
        default: return GRIM_ENOTSUP;
    }
}

}  // namespace grim
