// Verification side of the filter (the aligner's check and the paper's
// quality metrics, Sec. 5 and 6.1).
//
// grim_verify: for each location (read r, bin b), the semi-global edit
// distance of r against b's span - the fewest edits that turn r into some
// substring of the span (Sellers' recurrence: free start and end in the
// text).  A location "results in a mapping" when that distance is <= E.
// One thread per location runs Myers' bit-vector form of the recurrence:
// the vertical differences of one text column, for 64 read positions per
// machine word, advance by a handful of word operations per text base.
// Reads of more than 64 bases are split into 64-row blocks that exchange
// only the horizontal difference at their boundary row (Myers, 1999,
// "A fast bit-vector algorithm for approximate string matching based on
// dynamic programming", Sec. 4).  The read's match masks are built once per
// location from its bases; text bases are decoded from the 2-bit reference.
//
// grim_verify_stats: counts of passing / rejected locations with and
// without a mapping, from which the paper's "false negative rate" (passing
// locations without a mapping over all passing locations) and the zero-miss
// property (no rejected location with a mapping) follow.
#include "grim_internal.cuh"

namespace grim {
namespace {

constexpr int kVerifyMaxBlocks = 8;  // reads up to 512 bases

__device__ __forceinline__ uint32_t ref_code(const uint8_t* __restrict__ ref2bit, int64_t i) {
    return (__ldg(ref2bit + (i >> 2)) >> (2 * (i & 3))) & 3u;
}

// One text column for one 64-row block: updates the block's vertical
// differences (Pv: +1 rows, Mv: -1 rows) given the horizontal difference
// hin entering at its top row; returns the horizontal difference at the row
// marked by `top` (the block's last read row).
__device__ __forceinline__ int myers_step(uint64_t& Pv, uint64_t& Mv, uint64_t Eq, int hin, uint64_t top) {
    const uint64_t Xv = Eq | Mv;
    if (hin < 0) Eq |= 1ull;
    const uint64_t Xh = (((Eq & Pv) + Pv) ^ Pv) | Eq;
    uint64_t Ph = Mv | ~(Xh | Pv);
    uint64_t Mh = Pv & Xh;
    const int hout = (Ph & top) ? 1 : ((Mh & top) ? -1 : 0);
    Ph <<= 1;
    Mh <<= 1;
    if (hin < 0) Mh |= 1ull;
    else if (hin > 0) Ph |= 1ull;
    Pv = Mh | ~(Xv | Ph);
    Mv = Ph & Xv;
    return hout;
}

// Semi-global distance of read[0..L) (64 (B-1) < L <= 64 B) against the
// text ref[begin..end).
template <int B>
__device__ uint32_t sellers_distance(const uint8_t* __restrict__ read, int L, const uint8_t* __restrict__ ref2bit,
                                     int64_t begin, int64_t end) {
    uint64_t peq[4][B];
#pragma unroll
    for (int b = 0; b < B; b++) {
        uint64_t p0 = 0, p1 = 0, p2 = 0, p3 = 0;
        const int lo = 64 * b, hi = L < 64 * (b + 1) ? L : 64 * (b + 1);
        for (int i = lo; i < hi; i++) {
            const uint32_t c = __ldg(read + i);
            const uint64_t m = 1ull << (i - lo);
            p0 |= c == 0 ? m : 0ull;
            p1 |= c == 1 ? m : 0ull;
            p2 |= c == 2 ? m : 0ull;
            p3 |= c == 3 ? m : 0ull;  // codes > 3 match nothing
        }
        peq[0][b] = p0;
        peq[1][b] = p1;
        peq[2][b] = p2;
        peq[3][b] = p3;
    }
    uint64_t Pv[B], Mv[B];
#pragma unroll
    for (int b = 0; b < B; b++) {
        Pv[b] = ~0ull;  // column 0: D[i][0] = i, every vertical difference +1
        Mv[b] = 0ull;
    }
    const uint64_t top_last = 1ull << ((L - 1) & 63);
    uint32_t score = (uint32_t)L, best = (uint32_t)L;
    for (int64_t j = begin; j < end; j++) {
        const uint32_t t = ref_code(ref2bit, j);
        int h = 0;  // row 0 of the semi-global table is all zeros
#pragma unroll
        for (int b = 0; b < B; b++) {
            const uint64_t eq = t == 0 ? peq[0][b] : t == 1 ? peq[1][b] : t == 2 ? peq[2][b] : peq[3][b];
            h = myers_step(Pv[b], Mv[b], eq, h, b == B - 1 ? top_last : (1ull << 63));
        }
        score += h;
        best = score < best ? score : best;
    }
    return best;
}

// sellers_distance for a read of nb blocks, K <= nb <= MAXB (0 for nb = 0).
template <int K, int MAXB>
__device__ __forceinline__ uint32_t distance_blocks(int nb, const uint8_t* __restrict__ read, int L,
                                                   const uint8_t* __restrict__ ref2bit, int64_t begin, int64_t end) {
    if constexpr (K > MAXB) {
        return 0;
    } else {
        if (nb == K) return sellers_distance<K>(read, L, ref2bit, begin, end);
        return distance_blocks<K + 1, MAXB>(nb, read, L, ref2bit, begin, end);
    }
}

// Locations whose read spans MINB..MAXB blocks of 64 bases; the MINB == 0
// launch also writes every location it cannot score (bad ids, decreasing
// offsets, reads longer than the largest class).  Splitting by length keeps
// the register budget of short reads small.
template <int MINB, int MAXB>
__global__ void __launch_bounds__(256)
verify_kernel(const uint8_t* __restrict__ ref2bit, int64_t len, int64_t n_bins, int bin_len, int overlap,
              const uint8_t* __restrict__ reads, const int64_t* __restrict__ read_offsets, int64_t n_reads,
              const uint32_t* __restrict__ loc_read, const uint32_t* __restrict__ loc_bin, int64_t n_loc,
              uint16_t* __restrict__ dist, uint32_t* __restrict__ status) {
    uint32_t flags = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_loc; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = loc_read[i], b = loc_bin[i];
        int64_t L = -1;
        if ((int64_t)r < n_reads && (int64_t)b < n_bins) {
            const int64_t ro = read_offsets[r], re = read_offsets[r + 1];
            L = re >= ro ? re - ro : -1;
        }
        const int nb = L <= 0 ? 0 : (int)((L + 63) / 64);
        if (L < 0 || L > 64 * kVerifyMaxBlocks) {
            if (MINB == 0) {
                flags |= (int64_t)b >= n_bins ? GRIM_FLAG_BAD_BIN
                         : L > 64 * kVerifyMaxBlocks ? GRIM_FLAG_LONG_READ : GRIM_FLAG_BAD_OFFSETS;
                dist[i] = 0xFFFF;
            }
            continue;
        }
        if (nb < MINB || nb > MAXB) continue;
        const int64_t begin = (int64_t)b * bin_len;
        const int64_t end = begin + bin_len + overlap < len ? begin + bin_len + overlap : len;
        const uint32_t d = distance_blocks<(MINB > 0 ? MINB : 1), MAXB>(nb, reads + read_offsets[r], (int)L, ref2bit,
                                                                        begin, end);
        dist[i] = (uint16_t)(d < 0xFFFF ? d : 0xFFFF);
    }
    if (flags) atomicOr(status, flags);
}

// counts: [0] passing, [1] passing without a mapping (dist > E),
//         [2] rejected, [3] rejected with a mapping (a miss)
__global__ void verify_stats_kernel(const uint8_t* __restrict__ pass, const uint16_t* __restrict__ dist,
                                    const uint32_t* __restrict__ loc_read, const uint16_t* __restrict__ E,
                                    int64_t n_reads, int64_t n, unsigned long long* __restrict__ counts) {
    unsigned long long c[4] = {0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = loc_read[i];
        const bool mapped = (int64_t)r < n_reads && dist[i] <= E[r];
        if (!pass || pass[i]) {
            c[0]++;
            c[1] += !mapped;
        } else {
            c[2]++;
            c[3] += mapped;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
        unsigned long long v = c[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&counts[k], v);
    }
}

}  // namespace
}  // namespace grim

extern "C" {

int grim_verify(const grim_bank* bank, const uint8_t* ref2bit, const uint8_t* reads, const int64_t* read_offsets,
                int64_t n_reads, const uint32_t* loc_read, const uint32_t* loc_bin, int64_t n_loc, uint16_t* dist,
                void* stream) {
    if (!bank || n_reads < 0 || n_loc < 0) return GRIM_EINVAL;
    if (n_loc == 0) return GRIM_OK;
    if (!ref2bit || !reads || !read_offsets || !loc_read || !loc_bin || !dist) return GRIM_EINVAL;
    int rc = grim::check_device(bank);
    if (rc != GRIM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t need = (n_loc + 255) / 256;
    const int64_t cap = (int64_t)grim::sm_count() * 16;
    const unsigned blocks = (unsigned)(need < cap ? need : cap);
    // reads of up to 128, 129-256 and 257-512 bases
    grim::verify_kernel<0, 2><<<grim::fault_grid(blocks), 256, 0, s>>>(
            ref2bit, bank->len, bank->n_bins, bank->bin_len, bank->overlap, reads, read_offsets, n_reads, loc_read,
            loc_bin, n_loc, dist, bank->status);
    grim::verify_kernel<3, 4><<<grim::fault_grid(blocks), 256, 0, s>>>(
            ref2bit, bank->len, bank->n_bins, bank->bin_len, bank->overlap, reads, read_offsets, n_reads, loc_read,
            loc_bin, n_loc, dist, bank->status);
    grim::verify_kernel<5, 8><<<grim::fault_grid(blocks), 256, 0, s>>>(
            ref2bit, bank->len, bank->n_bins, bank->bin_len, bank->overlap, reads, read_offsets, n_reads, loc_read,
            loc_bin, n_loc, dist, bank->status);
    GRIM_CUDA_TRY(cudaGetLastError());
    return GRIM_OK;
}

int grim_verify_stats(const uint8_t* pass, const uint16_t* dist, const uint32_t* loc_read, const uint16_t* E,
                      int64_t n_reads, int64_t n, unsigned long long* counts, void* stream) {
    if (n < 0 || n_reads < 0 || !counts) return GRIM_EINVAL;
    if (n > 0 && (!dist || !loc_read || !E)) return GRIM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    GRIM_CUDA_TRY(cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long), s));
    if (n == 0) return GRIM_OK;
    const int64_t need = (n + 255) / 256;
    const int64_t cap = (int64_t)grim::sm_count() * 8;
    grim::verify_stats_kernel<<<grim::fault_grid((unsigned)(need < cap ? need : cap)), 256, 0, s>>>(
            pass, dist, loc_read, E, n_reads, n, counts);
    GRIM_CUDA_TRY(cudaGetLastError());
    return GRIM_OK;
}

}  // extern "C"
