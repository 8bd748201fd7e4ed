// The steps either side of the filter in a seed-and-extend mapper.
//
// Before (Sec. 1, Fig. 1 steps 2-3): the read's seeds are looked up in a
// table of reference locations; each location is a potential mapping, and
// the filter checks the bins that hold one (Sec. 3.3).
//   - grim_seed_index_build: a CSR table of the start positions of every
//     k-mer of the reference (count, prefix sum, fill; the order of the
//     positions of one k-mer is not specified);
//   - grim_seed_candidates: non-overlapping k-mer seeds per read; every
//     location p of the seed at offset o votes for the bin whose core holds
//     max(0, p - o); distinct bins are kept, the `cap` most voted when
//     there are more (equal votes: the lower bin), ascending.  Per batch of
//     reads: hits per read (warp per read) -> prefix sum -> votes expanded
//     into scratch -> one CTA per read sorts its votes (stable LSD radix
//     sort, in shared memory up to kDedupSmem votes, else in global
//     scratch), finds the runs, applies the cap (binary search on the vote
//     threshold) and compacts -> prefix sum of the kept counts -> copy into
//     the CSR output.
// After (Sec. 3.3, Fig. 4 steps 2-3): the Seed Location Checker turns the
// filter's bitmask into the list of passing locations and the reference
// segments the aligner receives.
//   - grim_locate: tile counts of passing bytes -> prefix sum -> ordered
//     write of (read, bin, span); optional segment bases copied out of the
//     2-bit reference (one warp per segment).
#include "grim_internal.cuh"

struct grim_seed_index {
    int64_t len;
    int k;
    int device;
    uint32_t* offsets;    // device, 4^k + 1 entries
    uint32_t* positions;  // device, len - k + 1 entries
    // the most candidates per read (x 16, rounded up) that a call has
    // produced: a sizing hint for callers that allocate per batch
    mutable std::atomic<int64_t> per_read_x16{0};
};

namespace grim {

int64_t seed_candidates_hint(const grim_seed_index* idx, int64_t n_reads) {
    return idx->per_read_x16.load() * n_reads / 16;
}

namespace {

// ------------------------------------------------------------ prefix sums

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread (all threads call it);
// *total receives the block's sum.
template <typename T>
__device__ T block_exclusive_scan(T v, T* warp_sums, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    const T before = warp == 0 ? T(0) : warp_sums[warp - 1];
    *total = warp_sums[nw - 1];
    __syncthreads();
    return before + x - v;
}

template <typename T>
__global__ void set_value_kernel(T* p, T v, const T* v_dev) {
    *p = v_dev ? *v_dev : v;
}

// tile sums over the same index sets scan_tiles_kernel uses
template <typename T>
__global__ void tile_sums_kernel(const T* __restrict__ in, int64_t n, T* __restrict__ sums) {
    __shared__ T ws[32];
    const int64_t t0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++)
        if (t0 + i < n) s += in[t0 + i];
    T total;
    block_exclusive_scan<T>(s, ws, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// one block of 1024 threads: sums[b] <- init + sum of sums[0..b), init
// read from init_dev when that is not null
template <typename T>
__global__ void scan_sums_kernel(T* __restrict__ sums, int64_t n_tiles, T init, const T* init_dev) {
    __shared__ T ws[32];
    T carry = init_dev ? *init_dev : init;
    for (int64_t b = 0; b < n_tiles; b += blockDim.x) {
        const int64_t j = b + threadIdx.x;
        const T v = j < n_tiles ? sums[j] : T(0);
        T total;
        const T ex = block_exclusive_scan<T>(v, ws, &total);
        if (j < n_tiles) sums[j] = carry + ex;
        carry += total;
    }
}

// out[i] = tile base + sum of in[tile start .. i); out[n] = the grand total.
// Each thread reads its own items before writing them, so in == out works.
template <typename T>
__global__ void scan_tiles_kernel(const T* in, T* out, int64_t n, const T* __restrict__ sums) {
    __shared__ T ws[32];
    const int64_t t0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = t0 + i < n ? in[t0 + i] : T(0);
        s += v[i];
    }
    T total;
    T run = sums[blockIdx.x] + block_exclusive_scan<T>(s, ws, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        if (t0 + i < n) out[t0 + i] = run;
        run += v[i];
        if (t0 + i == n - 1) out[n] = run;
    }
}

}  // namespace

// out[0..n]: out[i] = init + in[0] + ... + in[i-1]; in == out is allowed.
// init_dev (nullable) supplies init from device memory (it may be out[0]).
template <typename T>
int exclusive_scan(const T* in, T* out, int64_t n, T init, cudaStream_t s, const T* init_dev = nullptr) {
    if (n == 0) {
        set_value_kernel<T><<<grim::fault_grid(1), 1, 0, s>>>(out, init, init_dev);
        GRIM_CUDA_TRY(cudaGetLastError());
        return GRIM_OK;
    }
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    T* sums = nullptr;
    GRIM_CUDA_TRY(grim::scratch_alloc((void**)&sums, (size_t)tiles * sizeof(T), s));
    tile_sums_kernel<T><<<grim::fault_grid((unsigned)tiles), kScanThreads, 0, s>>>(in, n, sums);
    scan_sums_kernel<T><<<grim::fault_grid(1), 1024, 0, s>>>(sums, tiles, init, init_dev);
    scan_tiles_kernel<T><<<grim::fault_grid((unsigned)tiles), kScanThreads, 0, s>>>(in, out, n, sums);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(sums, s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return GRIM_ECUDA;
    }
    return GRIM_OK;
}

namespace {

__device__ __forceinline__ uint32_t ref_base(const uint8_t* __restrict__ ref2bit, int64_t i) {
    return (__ldg(ref2bit + (i >> 2)) >> (2 * (i & 3))) & 3u;
}

// ------------------------------------------------------------- seed index

constexpr int kIndexChunk = 64;  // consecutive positions per thread (rolling key)

// FILL = false: counts[key]++ for every position; true: positions[cursor[key]++] = p.
template <bool FILL>
__global__ void seed_index_kernel(const uint8_t* __restrict__ ref2bit, int64_t npos, int k,
                                  uint32_t* __restrict__ table, uint32_t* __restrict__ positions) {
    const uint32_t mask = (k >= 16) ? 0xFFFFFFFFu : ((1u << (2 * k)) - 1u);
    const int64_t chunks = (npos + kIndexChunk - 1) / kIndexChunk;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p0 = c * kIndexChunk;
        const int64_t p1 = p0 + kIndexChunk < npos ? p0 + kIndexChunk : npos;
        uint32_t key = 0;
        for (int j = 0; j < k - 1; j++) key = (key << 2) | ref_base(ref2bit, p0 + j);
        for (int64_t p = p0; p < p1; p++) {
            key = ((key << 2) | ref_base(ref2bit, p + k - 1)) & mask;
            if (FILL) {
                const uint32_t slot = atomicAdd(&table[key], 1u);
                positions[slot] = (uint32_t)p;
            } else {
                atomicAdd(&table[key], 1u);
            }
        }
    }
}

// ------------------------------------------------------- seed candidates

// Key of the k bases at s (first base most significant); false if one of
// them is not a base code.
__device__ __forceinline__ bool seed_key(const uint8_t* __restrict__ s, int k, uint32_t* key) {
    uint32_t v = 0;
    bool ok = true;
    for (int j = 0; j < k; j++) {
        const uint32_t c = __ldg(s + j);
        ok &= c <= 3u;
        v = (v << 2) | (c & 3u);
    }
    *key = v;
    return ok;
}

__device__ __forceinline__ int64_t n_seeds_of(int64_t L, int k) { return L >= k ? L / k : 0; }

// hits[r] = number of reference locations of read r's seeds (warp per read)
__global__ void seed_hits_kernel(const uint32_t* __restrict__ idx_off, int k, const uint8_t* __restrict__ reads,
                                 const int64_t* __restrict__ read_offsets, int64_t n, int64_t* __restrict__ hits) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        const int64_t ro = read_offsets[r], L = read_offsets[r + 1] - ro;
        const int64_t ns = n_seeds_of(L, k);
        int64_t h = 0;
        for (int64_t sd = lane; sd < ns; sd += 32) {
            uint32_t key;
            if (seed_key(reads + ro + sd * k, k, &key)) h += (int64_t)(idx_off[key + 1] - idx_off[key]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(kFull, h, o);
        if (lane == 0) hits[r] = h;
    }
}

// The batch's votes: read r's bins at H[hit_off[r] - h0 ...] (warp per read;
// seeds in order, each seed's locations spread over the lanes).
__global__ void seed_expand_kernel(const uint32_t* __restrict__ idx_off, const uint32_t* __restrict__ idx_pos, int k,
                                   const uint8_t* __restrict__ reads, const int64_t* __restrict__ read_offsets,
                                   int64_t n, const int64_t* __restrict__ hit_off, int64_t h0, uint32_t bin_len,
                                   uint32_t last_bin, uint32_t* __restrict__ H) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        const int64_t ro = read_offsets[r], L = read_offsets[r + 1] - ro;
        const int64_t ns = n_seeds_of(L, k);
        int64_t w = hit_off[r] - h0;
        for (int64_t g = 0; g < ns; g += 32) {
            // lane sd of this group looks up seed g + sd
            uint32_t a = 0, b = 0;
            if (g + lane < ns) {
                uint32_t key;
                if (seed_key(reads + ro + (g + lane) * k, k, &key)) {
                    a = idx_off[key];
                    b = idx_off[key + 1];
                }
            }
            const int m = ns - g < 32 ? (int)(ns - g) : 32;
            for (int sd = 0; sd < m; sd++) {
                const uint32_t sa = __shfl_sync(kFull, a, sd), sb = __shfl_sync(kFull, b, sd);
                const uint32_t o = (uint32_t)((g + sd) * k);
                for (uint32_t j = sa + lane; j < sb; j += 32) {
                    const uint32_t p = __ldg(idx_pos + j);
                    const uint32_t start = p > o ? p - o : 0u;
                    const uint32_t bin = start / bin_len;
                    H[w + (j - sa)] = bin < last_bin ? bin : last_bin;
                }
                w += sb - sa;
            }
        }
    }
}

constexpr int kDedupThreads = 256;
constexpr int kDedupSmem = 4096;  // votes sorted in shared memory up to this many
constexpr int kDedupItems = 8;    // consecutive entries per thread in the run and cap passes
constexpr int64_t kDedupChunk = (int64_t)kDedupThreads * kDedupItems;
constexpr int kRadixBits = 4;
constexpr int kRadixBuckets = 1 << kRadixBits;
constexpr int kDedupPadded = kDedupSmem + kDedupSmem / 32;
constexpr int kCountWords = kRadixBuckets * kDedupThreads + kRadixBuckets * kDedupThreads / 16;
constexpr size_t kDedupSmemBytes = (2 * (size_t)kDedupPadded + (size_t)kCountWords) * 4;

// Counter (bucket d, thread t) lives at word l + l / 16 for l = d * 256 + t:
// a thread's column (fixed t) and the scan's 16 consecutive counters of a
// thread (l = 16 t' + k, at word 17 t' + k) both spread over the banks.
__device__ __forceinline__ int cnt_at(int l) { return l + (l >> 4); }

// Shared-memory key arrays get one pad word per 32 so that threads reading
// consecutive blocks of keys do not collide on a bank.
template <bool SMEM, typename I>
__device__ __forceinline__ I rx_at(I i) {
    return SMEM ? i + (i >> 5) : i;
}

// Stable ascending LSD radix sort of A[0..n) on `passes` (even) digits of
// kRadixBits, with B as the second buffer; the result ends in A.  Thread t
// owns the contiguous keys [t * ipt, (t + 1) * ipt) and column t of the
// bucket-major counters, so counting and scattering need no atomics and
// keep equal digits in their original order.  I: index type (32-bit for
// the shared-memory case).
template <bool SMEM, typename I>
__device__ __forceinline__ void radix_sort(uint32_t* A, uint32_t* B, I n, int passes, uint32_t* cnt, uint32_t* ws) {
    const int t = threadIdx.x;
    const I ipt = (n + kDedupThreads - 1) / kDedupThreads;
    const I i0 = (I)t * ipt < n ? (I)t * ipt : n;
    const I i1 = i0 + ipt < n ? i0 + ipt : n;
    for (int ps = 0; ps < passes; ps++) {
        const int shift = ps * kRadixBits;
        uint32_t* src = (ps & 1) ? B : A;
        uint32_t* dst = (ps & 1) ? A : B;
#pragma unroll
        for (int b = 0; b < kRadixBuckets; b++) cnt[cnt_at(b * kDedupThreads + t)] = 0;
        for (I i = i0; i < i1; i++)
            cnt[cnt_at((int)((src[rx_at<SMEM>(i)] >> shift) & (kRadixBuckets - 1)) * kDedupThreads + t)]++;
        __syncthreads();
        // exclusive scan of the counters in bucket-major order: thread t owns
        // counters 16 t .. 16 t + 15 of that order (words 17 t .. 17 t + 15)
        uint32_t* mine = cnt + 17 * t;
        uint32_t v[kRadixBuckets];
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < kRadixBuckets; k++) {
            v[k] = mine[k];
            sum += v[k];
        }
        uint32_t tot;
        uint32_t run = block_exclusive_scan<uint32_t>(sum, ws, &tot);
#pragma unroll
        for (int k = 0; k < kRadixBuckets; k++) {
            mine[k] = run;
            run += v[k];
        }
        __syncthreads();
        for (I i = i0; i < i1; i++) {
            const uint32_t key = src[rx_at<SMEM>(i)];
            const uint32_t pos = cnt[cnt_at((int)((key >> shift) & (kRadixBuckets - 1)) * kDedupThreads + t)]++;
            dst[rx_at<SMEM>((I)pos)] = key;
        }
        __syncthreads();
    }
}

constexpr int kBucketBits = 10;  // the shared-memory sort's buckets: the keys' top 10 bits
constexpr int kBuckets = 1 << kBucketBits;
constexpr int kMaxBucket = 256;  // a fuller bucket hands the votes to the radix sort

// Ascending sort of the shared-memory keys A[0..n) (padded layout), all
// below 2^key_bits, into A, with B as the second buffer: the keys go to
// kBuckets buckets by their top bits (one counting pass, one scatter with
// shared atomics), then every key takes its final place in its bucket by
// counting the bucket's keys below it, ties broken by position.  The order
// of equal keys is immaterial here (only the sorted values and their run
// lengths are used).  Returns false, with A unchanged, when a bucket holds
// more than kMaxBucket keys.  cnt: 2 * kBuckets words.
__device__ bool bucket_sort_smem(uint32_t* A, uint32_t* B, int n, int key_bits, uint32_t* cnt, uint32_t* ws32) {
    constexpr int kPer = kBuckets / kDedupThreads;  // buckets per thread
    const int t = threadIdx.x;
    const int shift = key_bits > kBucketBits ? key_bits - kBucketBits : 0;
    uint32_t* start = cnt;              // first slot of each bucket
    uint32_t* cursor = cnt + kBuckets;  // counts, then scatter cursors, then bucket ends
    for (int b = t; b < kBuckets; b += kDedupThreads) cursor[b] = 0;
    __syncthreads();
    for (int i = t; i < n; i += kDedupThreads) atomicAdd(&cursor[A[rx_at<true>(i)] >> shift], 1u);
    __syncthreads();
    uint32_t c[kPer], sum = 0, mx = 0;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        c[k] = cursor[kPer * t + k];
        sum += c[k];
        mx = c[k] > mx ? c[k] : mx;
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan<uint32_t>(sum, ws32, &tot);
    if (__syncthreads_or(mx > (uint32_t)kMaxBucket)) return false;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        start[kPer * t + k] = run;
        cursor[kPer * t + k] = run;
        run += c[k];
    }
    __syncthreads();
    for (int i = t; i < n; i += kDedupThreads) {
        const uint32_t key = A[rx_at<true>(i)];
        B[rx_at<true>((int)atomicAdd(&cursor[key >> shift], 1u))] = key;
    }
    __syncthreads();
    for (int i = t; i < n; i += kDedupThreads) {
        const uint32_t key = B[rx_at<true>(i)];
        const uint32_t bk = key >> shift;
        const int s0 = (int)start[bk], s1 = (int)cursor[bk];
        int rank = s0;
        for (int j = s0; j < s1; j++) {
            const uint32_t o = B[rx_at<true>(j)];
            rank += (o < key) | ((o == key) & (j < i));
        }
        A[rx_at<true>(rank)] = key;
    }
    __syncthreads();
    return true;
}

// Votes of run j of the sorted votes: starts st[0..u), n votes in all.
template <typename I>
__device__ __forceinline__ uint32_t run_votes(const uint32_t* st, I u, I n, I j) {
    return (uint32_t)((j + 1 < u ? (I)st[j + 1] : n) - (I)st[j]);
}

// Block-wide count of runs with at least v votes.
template <typename I>
__device__ int64_t count_votes_at_least(const uint32_t* st, I u, I n, uint32_t v, int64_t* ws) {
    int64_t c = 0;
    for (I j = threadIdx.x; j < u; j += blockDim.x) c += run_votes<I>(st, u, n, j) >= v;
    int64_t total;
    block_exclusive_scan<int64_t>(c, ws, &total);
    return total;
}

// One read's votes A[0..n) (B: second buffer): sort, runs, cap, and the
// kept bins (ascending) to out[0..); returns their number.  st: scratch of
// n u32 for the run starts.  The shared-memory case (SMEM, 32-bit
// indices) reads A through the padded layout; the other case is global
// memory throughout.
template <bool SMEM, typename I>
__device__ __forceinline__ int64_t dedupe_read(uint32_t* A, uint32_t* B, I n, int cap, int passes, int bits,
                                               uint32_t* cnt,
                                               uint32_t* st, uint32_t* out, uint32_t* ws32, int64_t* ws,
                                               unsigned int* max_votes) {
    if (!SMEM || !bucket_sort_smem(A, B, (int)n, bits, cnt, ws32))
        radix_sort<SMEM, I>(A, B, n, passes, cnt, ws32);
    // run starts -> st[0..u), kDedupItems consecutive votes per thread
    I u = 0;
    for (I c0 = 0; c0 < n; c0 += (I)kDedupChunk) {
        const I i0 = c0 + (I)threadIdx.x * kDedupItems;
        uint32_t fl = 0;
#pragma unroll
        for (int k = 0; k < kDedupItems; k++) {
            const I i = i0 + k;
            if (i < n && (i == 0 || A[rx_at<SMEM>(i)] != A[rx_at<SMEM>((I)(i - 1))])) fl |= 1u << k;
        }
        uint32_t tot;
        I o = u + (I)block_exclusive_scan<uint32_t>((uint32_t)__popc(fl), ws32, &tot);
#pragma unroll
        for (int k = 0; k < kDedupItems; k++)
            if ((fl >> k) & 1u) st[o++] = (uint32_t)(i0 + k);
        u += (I)tot;
    }
    __syncthreads();
    int64_t n_keep = 0;
    if (u <= (I)cap) {
        for (I j = threadIdx.x; j < u; j += blockDim.x) out[j] = A[rx_at<SMEM>((I)st[j])];
        n_keep = u;
    } else {
        // the cap: keep votes > v_star, and the first `need` (lowest bins) at v_star
        if (threadIdx.x == 0) *max_votes = 0;
        __syncthreads();
        for (I j = threadIdx.x; j < u; j += blockDim.x) atomicMax(max_votes, run_votes<I>(st, u, n, j));
        __syncthreads();
        uint32_t lo = 1, hi = *max_votes;  // count(votes >= lo) >= cap always holds
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo + 1) / 2;
            if (count_votes_at_least<I>(st, u, n, mid, ws) >= cap) lo = mid;
            else hi = mid - 1;
        }
        const uint32_t v_star = lo;
        const int64_t need = cap - count_votes_at_least<I>(st, u, n, v_star + 1, ws);
        int64_t n_eq = 0;
        for (I c0 = 0; c0 < u; c0 += (I)kDedupChunk) {
            const I j0 = c0 + (I)threadIdx.x * kDedupItems;
            uint32_t gt = 0, eq = 0;
#pragma unroll
            for (int k = 0; k < kDedupItems; k++) {
                const I j = j0 + k;
                if (j < u) {
                    const uint32_t v = run_votes<I>(st, u, n, j);
                    if (v > v_star) gt |= 1u << k;
                    else if (v == v_star) eq |= 1u << k;
                }
            }
            int64_t tot_eq;
            int64_t e = n_eq + block_exclusive_scan<int64_t>(__popc(eq), ws, &tot_eq);
            uint32_t keep = gt;
#pragma unroll
            for (int k = 0; k < kDedupItems; k++)
                if ((eq >> k) & 1u) {
                    if (e < need) keep |= 1u << k;
                    e++;
                }
            int64_t tot_keep;
            int64_t o = n_keep + block_exclusive_scan<int64_t>(__popc(keep), ws, &tot_keep);
#pragma unroll
            for (int k = 0; k < kDedupItems; k++)
                if ((keep >> k) & 1u) out[o++] = A[rx_at<SMEM>((I)st[j0 + k])];
            n_eq += tot_eq;
            n_keep += tot_keep;
        }
    }
    return n_keep;
}

// One CTA per read of the batch: its votes sorted, runs found, the cap
// applied and the kept bins (ascending) written to H[hit_off[r] - h0 ...],
// their number to kept[r].  Reads of up to kDedupSmem votes work in shared
// memory (bucket sort, else radix sort; run starts in the sort's second
// buffer).  Longer reads use S, scratch of 8 bytes per vote, as 2n u32: run
// starts from the front, the back half as the radix sort's second buffer,
// then their list after the starts before it is copied to H.  `passes`:
// radix digits covering every bin id (even); `bits`: bits of the largest bin id.
__global__ void __launch_bounds__(kDedupThreads)
seed_dedupe_kernel(const int64_t* __restrict__ hit_off, int64_t h0, int cap, int passes, int bits,
                   uint32_t* __restrict__ H,
                   unsigned long long* __restrict__ S, int64_t* __restrict__ kept) {
    extern __shared__ uint32_t dedupe_smem[];
    __shared__ int64_t ws[32];
    __shared__ uint32_t ws32[32];
    __shared__ unsigned int max_votes;
    const int64_t r = blockIdx.x;
    const int64_t base = hit_off[r] - h0, n = hit_off[r + 1] - hit_off[r];
    if (n <= 0) {
        if (threadIdx.x == 0) kept[r] = 0;
        return;
    }
    uint32_t* st = reinterpret_cast<uint32_t*>(S + base);  // 2n u32 of scratch
    int64_t n_keep;
    if (n <= kDedupSmem) {
        uint32_t* A_s = dedupe_smem;
        uint32_t* B_s = dedupe_smem + kDedupPadded;
        uint32_t* cnt = dedupe_smem + 2 * kDedupPadded;
        const int ni = (int)n;
        for (int i = threadIdx.x; i < ni; i += blockDim.x) A_s[rx_at<true>(i)] = H[base + i];
        __syncthreads();
        // the run starts go to B_s, free once A_s is sorted
        n_keep = dedupe_read<true, int>(A_s, B_s, ni, cap, passes, bits, cnt, B_s, H + base, ws32, ws, &max_votes);
    } else {
        uint32_t* cnt = dedupe_smem + 2 * kDedupPadded;
        // the list is built after the starts (st + n: the sort's buffer, free by then)
        uint32_t* list = st + n;
        n_keep = dedupe_read<false, int64_t>(H + base, st + n, n, cap, passes, bits, cnt, st, list, ws32, ws,
                                             &max_votes);
        __syncthreads();
        for (int64_t j = threadIdx.x; j < n_keep; j += blockDim.x) H[base + j] = list[j];
    }
    if (threadIdx.x == 0) kept[r] = n_keep;
}

// cand_bins[cand_off[r] ...] <- the kept bins of read r (warp per read),
// entries at or beyond `capacity` dropped.
__global__ void seed_copy_kernel(const uint32_t* __restrict__ H, const int64_t* __restrict__ hit_off, int64_t h0,
                                 const int64_t* __restrict__ cand_off, int64_t n, uint32_t* __restrict__ cand_bins,
                                 int64_t capacity) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        const uint32_t* src = H + (hit_off[r] - h0);
        const int64_t d = cand_off[r], m = cand_off[r + 1] - d;
        for (int64_t j = lane; j < m; j += 32)
            if (d + j < capacity) cand_bins[d + j] = src[j];
    }
}

// next batch [r0, r1): the most reads after r0 whose votes fit `budget`
// (at least one read), at most max_reads.
// out = {hit_off[r0], r1, hit_off[r1], hit_off[n]}.
__global__ void batch_end_kernel(const int64_t* __restrict__ hit_off, int64_t n, int64_t r0, int64_t budget,
                                 int64_t max_reads, int64_t* __restrict__ out) {
    const int64_t h0 = hit_off[r0];
    int64_t lo = r0 + 1, hi = (n - r0) < max_reads ? n : r0 + max_reads;
    while (lo < hi) {  // largest r1 in [r0 + 1, hi] with hit_off[r1] - h0 <= budget (or r0 + 1)
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (hit_off[mid] - h0 <= budget) lo = mid;
        else hi = mid - 1;
    }
    out[0] = h0;
    out[1] = lo;
    out[2] = hit_off[lo];
    out[3] = hit_off[n];
}

// ------------------------------------------------------ seed location checker

constexpr int64_t kLocTile = kScanTile;

// Nonzero pass bytes among this thread's 16 (bit i = byte t0 + i): one
// 16-byte load when the bytes are aligned and in range.
__device__ __forceinline__ uint32_t pass_mask16(const uint8_t* __restrict__ pass, int64_t t0, int64_t n,
                                                bool aligned) {
    if (aligned && t0 + 16 <= n) return nonzero_bytes16(__ldg(reinterpret_cast<const uint4*>(pass + t0)));
    uint32_t m = 0;
    for (int i = 0; i < kScanItems; i++)
        if (t0 + i < n && pass[t0 + i]) m |= 1u << i;
    return m;
}

__global__ void locate_count_kernel(const uint8_t* __restrict__ pass, int64_t n_cands, bool aligned,
                                    int64_t* __restrict__ counts) {
    __shared__ int64_t ws[32];
    const int64_t t0 = (int64_t)blockIdx.x * kLocTile + (int64_t)threadIdx.x * kScanItems;
    const int64_t c = __popc(pass_mask16(pass, t0, n_cands, aligned));
    int64_t total;
    block_exclusive_scan<int64_t>(c, ws, &total);
    if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// Reads holding candidates c0 (lanes 0-15) and c1 (lanes 16-31): the last
// r in [0, n_reads - 1] with cand_offsets[r] <= c, by a 16-ary search per
// half-warp (about log16(n_reads) rounds of parallel loads).  Whole warp.
__device__ int64_t reads_of_half_warps(const int64_t* __restrict__ co, int64_t n_reads, int64_t c0, int64_t c1,
                                       int lane) {
    const int j = lane & 15;
    const int64_t c = lane < 16 ? c0 : c1;
    int64_t lo = 0, hi = n_reads - 1;  // the answer lies in [lo, hi]; co[0] <= c
    while (__any_sync(kFull, hi - lo > 15)) {  // then 16 lanes cover [lo, hi]
        const int64_t p = lo + 1 + (hi - lo - 1 > 0 ? (hi - lo - 1) * j / 15 : 0);  // samples in (lo, hi]
        const bool le = p <= hi && __ldg(co + p) <= c;
        const unsigned b = __ballot_sync(kFull, le);
        const unsigned half = lane < 16 ? b & 0xFFFFu : b >> 16;
        const int k = __popc(half);  // the samples at or below c are a prefix
        const int64_t p_last = __shfl_sync(kFull, p, (lane & 16) + (k > 0 ? k - 1 : 0));
        const int64_t p_next = __shfl_sync(kFull, p, (lane & 16) + (k < 16 ? k : 15));
        if (k > 0) lo = p_last;
        if (k < 16 && p_next - 1 < hi) hi = p_next - 1;
        if (hi < lo) hi = lo;  // only with decreasing (invalid) offsets
    }
    const int64_t p = lo + j;
    const unsigned b = __ballot_sync(kFull, p <= hi && __ldg(co + p) <= c);
    const int cnt = __popc(lane < 16 ? b & 0xFFFFu : b >> 16);
    return cnt > 0 ? lo + cnt - 1 : lo;
}

// read holding candidate c: the last r in [lo, hi] with cand_offsets[r] <= c
__device__ __forceinline__ int64_t read_of(const int64_t* __restrict__ co, int64_t lo, int64_t hi, int64_t c) {
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (co[mid] <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void locate_write_kernel(const uint8_t* __restrict__ pass, bool aligned,
                                    const uint32_t* __restrict__ cand_bins, const int64_t* __restrict__ cand_offsets,
                                    int64_t n_reads, int64_t n_cands, const int64_t* __restrict__ tile_base,
                                    int64_t len, int64_t n_bins, int bin_len, int overlap, int64_t capacity,
                                    uint32_t* __restrict__ loc_read, uint32_t* __restrict__ loc_bin,
                                    int64_t* __restrict__ loc_begin, int64_t* __restrict__ loc_end,
                                    uint32_t* __restrict__ status) {
    __shared__ int64_t ws[32];
    __shared__ int64_t tile_reads[2];
    const int64_t tile0 = (int64_t)blockIdx.x * kLocTile;
    const int64_t t0 = tile0 + (int64_t)threadIdx.x * kScanItems;
    uint32_t m = pass_mask16(pass, t0, n_cands, aligned);
    uint32_t flags = 0;
    if (threadIdx.x == 0 && blockIdx.x == 0 && cand_offsets[n_reads] != n_cands) flags |= GRIM_FLAG_BAD_OFFSETS;
    int64_t total;
    int64_t o = tile_base[blockIdx.x] + block_exclusive_scan<int64_t>(__popc(m), ws, &total);
    if (total == 0) {  // nothing passes in this tile (block-uniform)
        if (flags) atomicOr(status, flags);
        return;
    }
    if (threadIdx.x < 32) {  // the reads of the tile's first and last candidates
        const int64_t last = (tile0 + kLocTile < n_cands ? tile0 + kLocTile : n_cands) - 1;
        const int64_t rr = reads_of_half_warps(cand_offsets, n_reads, tile0, last, threadIdx.x);
        if (threadIdx.x == 0) tile_reads[0] = rr;
        if (threadIdx.x == 16) tile_reads[1] = rr;
    }
    __syncthreads();
    const int64_t tr0 = tile_reads[0], tr1 = tile_reads[1] > tile_reads[0] ? tile_reads[1] : tile_reads[0];
    int64_t r = -1;
    while (m && o < capacity) {
        const int i = __ffs(m) - 1;
        m &= m - 1;
        const int64_t c = t0 + i;
        // the read: one search within the tile's reads, then forward
        if (r < 0) r = read_of(cand_offsets, tr0, tr1, c);
        while (r + 1 < n_reads && cand_offsets[r + 1] <= c) r++;
        const uint32_t b = cand_bins[c];
        int64_t begin = 0, end = 0;
        if ((int64_t)b < n_bins) {
            begin = (int64_t)b * bin_len;
            end = begin + bin_len + overlap < len ? begin + bin_len + overlap : len;
        } else {
            flags |= GRIM_FLAG_BAD_BIN;
        }
        loc_read[o] = (uint32_t)r;
        loc_bin[o] = b;
        if (loc_begin) loc_begin[o] = begin;
        if (loc_end) loc_end[o] = end;
        o++;
    }
    if (flags) atomicOr(status, flags);
}

// segment rows: the span's base codes, then 4 up to the stride (warp per row)
__global__ void locate_segments_kernel(const uint8_t* __restrict__ ref2bit, const int64_t* __restrict__ n_loc,
                                       int64_t capacity, const int64_t* __restrict__ loc_begin,
                                       const int64_t* __restrict__ loc_end, uint8_t* __restrict__ seg,
                                       int64_t stride) {
    const int lane = threadIdx.x & 31;
    const int64_t rows = *n_loc < capacity ? *n_loc : capacity;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows; i += warps) {
        const int64_t b = loc_begin[i], e = loc_end[i];
        uint8_t* row = seg + i * stride;
        for (int64_t j = lane; j < stride; j += 32) row[j] = b + j < e ? (uint8_t)ref_base(ref2bit, b + j) : 4;
    }
}

}  // namespace
}  // namespace grim

extern "C" {

int grim_seed_index_build(const uint8_t* ref2bit, int64_t len, int k, void* stream, grim_seed_index** out) {
    if (!out) return GRIM_EINVAL;
    *out = nullptr;
    if (!ref2bit || k < 1 || k > 15 || len < k || len > (int64_t)0xFFFFFFFFll) return GRIM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nk = int64_t(1) << (2 * k);
    const int64_t npos = len - k + 1;
    grim_seed_index* idx = new grim_seed_index();
    idx->len = len;
    idx->k = k;
    if (cudaGetDevice(&idx->device) != cudaSuccess) {
        delete idx;
        return GRIM_ECUDA;
    }
    uint32_t* cursor = nullptr;
    cudaError_t e = grim::fault_alloc_now() ? cudaErrorMemoryAllocation
                                            : cudaMalloc((void**)&idx->offsets, (size_t)(nk + 1) * 4);
    if (e == cudaSuccess)
        e = grim::fault_alloc_now() ? cudaErrorMemoryAllocation
                                    : cudaMalloc((void**)&idx->positions, (size_t)npos * 4);
    if (e == cudaSuccess) e = grim::scratch_alloc((void**)&cursor, (size_t)nk * 4, s);
    int rc = GRIM_OK;
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, (size_t)nk * 4, s);
    if (e == cudaSuccess) {
        const int blocks = grim::sm_count() * 8;
        grim::seed_index_kernel<false><<<grim::fault_grid(blocks), 256, 0, s>>>(ref2bit, npos, k, cursor, nullptr);
        e = cudaGetLastError();
        if (e == cudaSuccess) rc = grim::exclusive_scan<uint32_t>(cursor, idx->offsets, nk, 0u, s);
        if (e == cudaSuccess && rc == GRIM_OK)
            e = cudaMemcpyAsync(cursor, idx->offsets, (size_t)nk * 4, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && rc == GRIM_OK) {
            grim::seed_index_kernel<true><<<grim::fault_grid(blocks), 256, 0, s>>>(
                    ref2bit, npos, k, cursor, idx->positions);
            e = cudaGetLastError();
        }
    }
    if (cursor) cudaFreeAsync(cursor, s);
    if (e != cudaSuccess || rc != GRIM_OK) {
        if (e != cudaSuccess) {
            grim::set_last_cuda_error(e);
            rc = e == cudaErrorMemoryAllocation ? GRIM_ENOMEM : GRIM_ECUDA;
        }
        cudaStreamSynchronize(s);
        cudaFree(idx->offsets);
        cudaFree(idx->positions);
        delete idx;
        return rc;
    }
    *out = idx;
    return GRIM_OK;
}

int grim_seed_index_info(const grim_seed_index* idx, int64_t* len, int* k, const uint32_t** offsets,
                         const uint32_t** positions) {
    if (!idx) return GRIM_EINVAL;
    if (len) *len = idx->len;
    if (k) *k = idx->k;
    if (offsets) *offsets = idx->offsets;
    if (positions) *positions = idx->positions;
    return GRIM_OK;
}

int grim_seed_index_free(grim_seed_index* idx) {
    if (!idx) return GRIM_OK;
    cudaDeviceSynchronize();
    cudaFree(idx->offsets);
    cudaFree(idx->positions);
    delete idx;
    return GRIM_OK;
}

int grim_seed_candidates(const grim_seed_index* idx, const uint8_t* reads, const int64_t* read_offsets,
                         int64_t n_reads, int bin_len, int64_t n_bins, int cap, uint32_t* cand_bins,
                         int64_t capacity, int64_t* cand_offsets, int64_t* n_cands, void* stream) {
    if (!idx || n_reads < 0 || bin_len < 1 || n_bins < 1 || n_bins > (int64_t)0xFFFFFFFFll || cap < 1 ||
        capacity < 0 || !cand_offsets || !n_cands || (capacity > 0 && !cand_bins))
        return GRIM_EINVAL;
    *n_cands = 0;
    if (n_reads > 0 && (!reads || !read_offsets)) return GRIM_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != idx->device) return GRIM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_reads == 0) return grim::exclusive_scan<int64_t>(nullptr, cand_offsets, 0, 0, s);

    const int threads = 256;
    const int64_t warp_blocks = (n_reads * 32 + threads - 1) / threads;
    const unsigned blocks = (unsigned)(warp_blocks < 65535 ? warp_blocks : 65535);
    int64_t* hit_off = nullptr;
    int64_t* info = nullptr;  // batch bounds
    GRIM_CUDA_TRY(grim::scratch_alloc((void**)&hit_off, (size_t)(n_reads + 1) * 8, s));
    GRIM_CUDA_TRY(grim::scratch_alloc((void**)&info, 64, s));  // batch bounds
    int rc = GRIM_OK;
    grim::seed_hits_kernel<<<grim::fault_grid(blocks), threads, 0, s>>>(
            idx->offsets, idx->k, reads, read_offsets, n_reads, hit_off);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) rc = grim::exclusive_scan<int64_t>(hit_off, hit_off, n_reads, 0, s);

    // radix digits covering bin ids 0 .. n_bins - 1, rounded up to even
    int bits = 0;
    while (bits < 32 && ((n_bins - 1) >> bits) != 0) bits++;
    const int passes = 2 * ((bits + 2 * grim::kRadixBits - 1) / (2 * grim::kRadixBits));
    static grim::DeviceCache smem_set[64];
    if (dev >= 0 && dev < 64 && !smem_set[dev].load()) {
        GRIM_CUDA_TRY(cudaFuncSetAttribute(grim::seed_dedupe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)grim::kDedupSmemBytes));
        smem_set[dev].store(1);
    }
    const int64_t kBudget = int64_t(1) << 28;     // votes per batch
    const int64_t kMaxReads = int64_t(1) << 20;   // reads per batch
    // scratch kept across batches (freeing it would hand it back to the
    // pool at every synchronisation): votes as u32 (H) and 2 u32 per vote (S)
    uint32_t* H = nullptr;
    unsigned long long* S = nullptr;
    int64_t* kept = nullptr;
    int64_t cap_votes = 0;
    if (e == cudaSuccess && rc == GRIM_OK) {
        const int64_t max_nb = n_reads < kMaxReads ? n_reads : kMaxReads;
        e = grim::scratch_alloc((void**)&kept, (size_t)max_nb * 8, s);
        if (e == cudaSuccess) {
            grim::set_value_kernel<int64_t><<<grim::fault_grid(1), 1, 0, s>>>(cand_offsets, 0, nullptr);
            e = cudaGetLastError();
        }
    }
    for (int64_t r0 = 0; r0 < n_reads && e == cudaSuccess && rc == GRIM_OK;) {
        int64_t b[4];
        grim::batch_end_kernel<<<grim::fault_grid(1), 1, 0, s>>>(hit_off, n_reads, r0, kBudget, kMaxReads, info);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(b, info, sizeof(b), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        const int64_t h0 = b[0], r1 = b[1], votes = b[2] - b[0], nb = r1 - r0;
        if (votes > cap_votes) {
            // the first batch sizes it for the largest regular batch
            const int64_t want = votes > kBudget ? votes : (b[3] - h0 < kBudget ? b[3] - h0 : kBudget);
            if (H) cudaFreeAsync(H, s);
            if (S) cudaFreeAsync(S, s);
            H = nullptr;
            S = nullptr;
            e = grim::scratch_alloc((void**)&H, (size_t)(want > 0 ? want : 1) * 4, s);
            if (e == cudaSuccess) e = grim::scratch_alloc((void**)&S, (size_t)(want > 0 ? want : 1) * 8, s);
            if (e != cudaSuccess) break;
            cap_votes = want;
        }
        const int64_t wb = (nb * 32 + threads - 1) / threads;
        const unsigned bb = (unsigned)(wb < 65535 ? wb : 65535);
        if (votes > 0)
            grim::seed_expand_kernel<<<grim::fault_grid(bb), threads, 0, s>>>(
                    idx->offsets, idx->positions, idx->k, reads, read_offsets + r0, nb, hit_off + r0, h0,
                    (uint32_t)bin_len, (uint32_t)(n_bins - 1), H);
        grim::seed_dedupe_kernel<<<grim::fault_grid((unsigned)nb), grim::kDedupThreads, grim::kDedupSmemBytes, s>>>(
            hit_off + r0, h0, cap, passes, bits, H, S, kept);
        e = cudaGetLastError();
        // offsets continue from the previous batch's total in cand_offsets[r0]
        if (e == cudaSuccess) rc = grim::exclusive_scan<int64_t>(kept, cand_offsets + r0, nb, 0, s, cand_offsets + r0);
        if (e == cudaSuccess && rc == GRIM_OK) {
            grim::seed_copy_kernel<<<grim::fault_grid(bb), threads, 0, s>>>(
                    H, hit_off + r0, h0, cand_offsets + r0, nb, cand_bins, capacity);
            e = cudaGetLastError();
        }
        r0 = r1;
    }
    int64_t total = 0;
    if (e == cudaSuccess && rc == GRIM_OK)
        e = cudaMemcpyAsync(&total, cand_offsets + n_reads, 8, cudaMemcpyDeviceToHost, s);
    if (H) cudaFreeAsync(H, s);
    if (S) cudaFreeAsync(S, s);
    if (kept) cudaFreeAsync(kept, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(hit_off, s);
    cudaFreeAsync(info, s);
    if (e != cudaSuccess) {
        grim::set_last_cuda_error(e);
        return e == cudaErrorMemoryAllocation ? GRIM_ENOMEM : GRIM_ECUDA;
    }
    if (rc != GRIM_OK) return rc;
    *n_cands = total;
    const int64_t x16 = (total * 16 + n_reads - 1) / n_reads;
    int64_t seen = idx->per_read_x16.load();
    while (x16 > seen && !idx->per_read_x16.compare_exchange_weak(seen, x16)) {
    }
    return total > capacity ? GRIM_EOVERFLOW : GRIM_OK;
}

int grim_locate(const grim_bank* bank, const uint8_t* ref2bit, const uint32_t* cand_bins,
                const int64_t* cand_offsets, int64_t n_reads, int64_t n_cands, const uint8_t* pass,
                uint32_t* loc_read, uint32_t* loc_bin, int64_t* loc_begin, int64_t* loc_end, uint8_t* segments,
                int64_t seg_stride, int64_t capacity, int64_t* n_loc, void* stream) {
    if (!bank || n_reads < 0 || n_cands < 0 || capacity < 0 || !n_loc || !cand_offsets) return GRIM_EINVAL;
    if (n_cands > 0 && (!cand_bins || !pass)) return GRIM_EINVAL;
    if (capacity > 0 && (!loc_read || !loc_bin)) return GRIM_EINVAL;
    if (segments && (seg_stride <= 0 || !ref2bit || !loc_begin || !loc_end)) return GRIM_EINVAL;
    if (n_cands > 0 && n_reads == 0) return GRIM_EINVAL;
    int rc = grim::check_device(bank);
    if (rc != GRIM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_cands == 0) return grim::exclusive_scan<int64_t>(nullptr, n_loc, 0, 0, s);
    const int64_t tiles = (n_cands + grim::kLocTile - 1) / grim::kLocTile;
    int64_t* counts = nullptr;
    GRIM_CUDA_TRY(grim::scratch_alloc((void**)&counts, (size_t)(tiles + 1) * 8, s));
    const bool aligned = ((uintptr_t)pass & 15) == 0;
    grim::locate_count_kernel<<<grim::fault_grid((unsigned)tiles), grim::kScanThreads, 0, s>>>(
            pass, n_cands, aligned, counts);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) rc = grim::exclusive_scan<int64_t>(counts, counts, tiles, 0, s);
    if (e == cudaSuccess && rc == GRIM_OK)
        e = cudaMemcpyAsync(n_loc, counts + tiles, 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && rc == GRIM_OK) {
        grim::locate_write_kernel<<<grim::fault_grid((unsigned)tiles), grim::kScanThreads, 0, s>>>(
            pass, aligned, cand_bins, cand_offsets, n_reads, n_cands, counts, bank->len, bank->n_bins, bank->bin_len,
            bank->overlap, capacity, loc_read, loc_bin, loc_begin, loc_end, bank->status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && rc == GRIM_OK && segments && capacity > 0) {
        grim::locate_segments_kernel<<<grim::fault_grid(grim::sm_count() * 8), 256, 0, s>>>(
                ref2bit, n_loc, capacity, loc_begin, loc_end, segments, seg_stride);
        e = cudaGetLastError();
    }
    cudaFreeAsync(counts, s);
    if (e != cudaSuccess) {
        grim::set_last_cuda_error(e);
        return GRIM_ECUDA;
    }
    return rc;
}

}  // extern "C"
