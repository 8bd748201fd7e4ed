// Bank build (Sec. 3.1): the 2-bit packed reference -> one 4^q-bit
// existence bitvector per bin, bin-major in HBM.
//
// Main kernel (bank_build_lanes_kernel, q <= 5 and ordinary geometry): one
// thread per bin CORE.  Bin b's token starts are its core's bin_len starts
// followed by the first e = overlap - q + 1 starts after it, i.e. J whole
// following cores and a prefix of r = e mod bin_len starts of the one after
// (J = e / bin_len).  So each thread sets the bits of its own core's tokens
// exactly once, split in two rows: P (the core's first r starts) and R (the
// rest); then
//     row(b) = P_b | R_b | (P|R)_{b+1} | ... | (P|R)_{b+J} | P_{b+J+1}.
// A warp takes 32 consecutive cores and finishes the rows of the first
// 32 - (J + 1), the neighbours' words coming by shuffle, so warps never wait
// for one another.  The rows being built live in shared memory in a
// thread-private transposed layout - word w of lane l's row at w * 32 + l -
// so the bank a thread touches depends on its lane only: a warp's 32
// shared-memory ORs never collide, whatever its tokens.  Tokens come from a
// 64-bit window of the core's bases (reversed to first base most
// significant), one shift per token at a compile-time offset.  The finished
// rows pass through shared memory once more so that each warp stores its
// consecutive rows with whole 512-byte writes.
//
// Fallback kernels (q = 6, very long bins or overlaps, unaligned input): one
// CTA owns a run of consecutive bins and keeps their rows in shared memory;
// its threads walk every token start of the run's spans once and set the
// token's bit in every bin of the run whose span holds it with a
// shared-memory atomicOr; the rows then leave in 16-byte stores.
#include "grim_internal.cuh"

namespace grim {

constexpr int kBuildThreads = 256;
constexpr int kBuildSmemBytes = 16384;    // bin rows per CTA
constexpr int kBuildStageBytes = 32768;   // staged packed reference per CTA

template <int Q>
__global__ void __launch_bounds__(kBuildThreads)
bank_build_kernel(const uint8_t* __restrict__ ref2bit, int64_t len, int bin_len, int overlap, int64_t n_bins,
                  int bins_per_cta, uint32_t* __restrict__ bank) {
    using G = Geo<Q>;
    extern __shared__ uint4 smem4[];
    uint32_t* sbits = reinterpret_cast<uint32_t*>(smem4);

    const int64_t b0 = (int64_t)blockIdx.x * bins_per_cta;
    const int nb = (int)((n_bins - b0) < bins_per_cta ? (n_bins - b0) : bins_per_cta);
    const int row4 = G::kRowWords / 4;

    for (int i = threadIdx.x; i < nb * row4; i += blockDim.x) smem4[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();

    // token starts of the run: the first core base up to the last span end
    const int64_t p0 = b0 * (int64_t)bin_len;
    int64_t pend = (b0 + nb) * (int64_t)bin_len + overlap;
    if (pend > len) pend = len;
    const int64_t b_last = b0 + nb - 1;

    for (int64_t i = p0 + threadIdx.x; i + Q <= pend; i += blockDim.x) {
        uint32_t tok = 0;
#pragma unroll
        for (int k = 0; k < Q; k++) {
            const int64_t x = i + k;
            const uint32_t byte = __ldg(ref2bit + (x >> 2));
            tok = (tok << 2) | ((byte >> (2 * (int)(x & 3))) & 3u);
        }
        // bins b with b*bin_len <= i and i+Q <= b*bin_len + bin_len + overlap
        int64_t bhi = i / bin_len;
        if (bhi > b_last) bhi = b_last;
        const int64_t need = i + Q - (int64_t)bin_len - overlap;
        int64_t blo = need <= 0 ? 0 : (need + bin_len - 1) / bin_len;
        if (blo < b0) blo = b0;
        const uint32_t w = tok >> 5, m = 1u << (tok & 31);
        for (int64_t b = blo; b <= bhi; b++) atomicOr(&sbits[(b - b0) * G::kRowWords + w], m);
    }
    __syncthreads();

    uint4* dst = reinterpret_cast<uint4*>(bank + b0 * G::kRowWords);
    for (int i = threadIdx.x; i < nb * row4; i += blockDim.x) dst[i] = smem4[i];
}

// Fast path: the run's packed reference bytes are staged in shared memory,
// and each thread rolls the token through a contiguous stretch of token
// starts (two instructions per base) while tracking, without divisions, the
// first and last bin whose span holds the current token.
template <int Q>
__global__ void __launch_bounds__(kBuildThreads)
bank_build_staged_kernel(const uint8_t* __restrict__ ref2bit, int64_t len, int bin_len, int overlap, int64_t n_bins,
                         int bins_per_cta, uint32_t* __restrict__ bank) {
    using G = Geo<Q>;
    constexpr uint32_t kMask = (Q == 16) ? 0xffffffffu : ((1u << (2 * Q)) - 1u);
    extern __shared__ uint4 smem4[];
    uint32_t* sbits = reinterpret_cast<uint32_t*>(smem4);
    const int64_t b0 = (int64_t)blockIdx.x * bins_per_cta;
    const int nb = (int)((n_bins - b0) < bins_per_cta ? (n_bins - b0) : bins_per_cta);
    const int row4 = G::kRowWords / 4;
    uint32_t* sref = sbits + (size_t)bins_per_cta * G::kRowWords;  // packed reference, 16 bases per word

    const int64_t p0 = b0 * (int64_t)bin_len;
    int64_t pend = (b0 + nb) * (int64_t)bin_len + overlap;
    if (pend > len) pend = len;
    // packed bytes [4*word0, 4*ceil(pend/16)) of the reference, as words
    const int64_t word0 = p0 >> 4;
    const int64_t byte_end = (pend + 3) >> 2;
    const int nwords = (int)(((pend + 15) >> 4) - word0);
    for (int i = threadIdx.x; i < nb * row4; i += blockDim.x) smem4[i] = make_uint4(0, 0, 0, 0);
    for (int i = threadIdx.x; i < nwords; i += blockDim.x) {
        uint32_t v = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int64_t byte = 4 * (word0 + i) + k;
            if (byte < byte_end) v |= (uint32_t)__ldg(ref2bit + byte) << (8 * k);
        }
        sref[i] = v;
    }
    __syncthreads();

    // token starts i in [p0, pend - Q], split into one stretch per thread
    const int n_starts = (int)(pend - Q + 1 - p0);
    if (n_starts > 0) {
        const int per = (n_starts + blockDim.x - 1) / blockDim.x;
        const int s0 = threadIdx.x * per;
        const int s1 = min(n_starts, s0 + per);
        if (s0 < s1) {
            // bases stream from a one-word buffer: x = position - 16*word0
            int x = (int)(p0 + s0 - 16 * word0);
            uint32_t buf = sref[x >> 4] >> (2 * (x & 15));
            int left = 16 - (x & 15);
            auto next_base = [&]() -> uint32_t {
                if (left == 0) {
                    buf = sref[x >> 4];
                    left = 16;
                }
                const uint32_t b = buf & 3u;
                buf >>= 2;
                --left;
                ++x;
                return b;
            };
            uint32_t tok = 0;
#pragma unroll
            for (int k = 0; k < Q - 1; k++) tok = (tok << 2) | next_base();
            // bin bookkeeping for the first start, then incremental
            const int64_t i_first = p0 + s0;
            int64_t bhi = i_first / bin_len;                           // last bin with b*bin_len <= i
            int64_t next_hi = (bhi + 1) * (int64_t)bin_len;           // i at which bhi grows
            const int64_t need = i_first + Q - (int64_t)bin_len - overlap;
            int64_t blo = need <= 0 ? 0 : (need + bin_len - 1) / bin_len;  // first bin with i+Q <= its span end
            int64_t next_lo = blo * (int64_t)bin_len + bin_len + overlap - Q + 1;  // i at which blo grows
            const int64_t b_last = b0 + nb - 1;
            for (int rel = s0; rel < s1; rel++) {
                const int64_t i = p0 + rel;
                if (i == next_hi) { ++bhi; next_hi += bin_len; }
                if (i == next_lo) { ++blo; next_lo += bin_len; }
                tok = ((tok << 2) | next_base()) & kMask;
                const uint32_t w = tok >> 5, m = 1u << (tok & 31);
                const int lo = (int)((blo > b0 ? blo : b0) - b0);
                const int hi = (int)((bhi < b_last ? bhi : b_last) - b0);
                for (int b = lo; b <= hi; b++) atomicOr(&sbits[b * G::kRowWords + w], m);
            }
        }
    }
    __syncthreads();
    uint4* dst = reinterpret_cast<uint4*>(bank + b0 * G::kRowWords);
    for (int i = threadIdx.x; i < nb * row4; i += blockDim.x) dst[i] = smem4[i];
}


// ------------------------------------------------------------ lane per core

constexpr int kLaneWarps = 4;                  // 128 cores per CTA
constexpr int kLaneCores = kLaneWarps * 32;
constexpr int kLaneMaxBinLen = 1024;           // staged bases per core (two staging buffers)
constexpr int kLaneMaxJ = 16;                  // whole following cores in a span (out_w >= 15)

template <int Q>
struct LaneGeo {
    static constexpr int kRW = Geo<Q>::kRowWords;           // words per row
    static constexpr int kChunks = kRW / 4;                 // 16-byte chunks per row
    static constexpr int kRowSetBytes = kRW * 128;          // 32 rows (one per lane), transposed
    // byte offset of word (token >> 5) within a lane's transposed row, from
    // (token << 2): bits 7 .. 7 + log2(words used) - 1
    static constexpr uint32_t kWordMask = Q >= 3 ? (uint32_t)((1u << (2 * Q - 5)) - 1u) << 7 : 0u;
};

__device__ __forceinline__ void red_or_shared(uint32_t addr, uint32_t v) {
    asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t shared_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// The 16 token starts of one staged word pair.  The 64-bit window hi:lo
// holds 32 bases, first base in bits 63..62; x_t = (hi:lo) >> (64 - 2t - 2Q)
// has token t in its low 2Q bits, and x_{t+1} is token t shifted left by 2
// (the next base below), so the row word of token t comes from x_{t+1} and
// its bit from x_t.  MODE 0: every token into row base0, 1: into base1,
// 2: tokens t < split into base0, the rest into base1.  GUARD: only the
// first `lim` starts exist.

// x_t for a compile-time t: a shift that stays within the high word is a
// multiply-high (the FMA pipe), leaving the ALU pipe to the rest.
template <int Q, int T>
__device__ __forceinline__ uint32_t lane_window(uint32_t hi, uint32_t lo) {
    constexpr int kShift = 64 - 2 * T - 2 * Q;  // right shift of the 64-bit window hi:lo
    if constexpr (kShift > 32) {
        return __umulhi(hi, 1u << (64 - kShift));
    } else if constexpr (kShift == 32) {
        return hi;
    } else {
        return __funnelshift_r(lo, hi, kShift);
    }
}

template <int Q, int MODE, bool GUARD, int T>
__device__ __forceinline__ void lane_token_step(uint32_t hi, uint32_t lo, uint32_t x, uint32_t base0, uint32_t base1,
                                                int split, int lim) {
    if constexpr (T < 16) {
        using LG = LaneGeo<Q>;
        const uint32_t xn = lane_window<Q, T + 1>(hi, lo);
        if (!GUARD || T < lim) {
            const uint32_t tok = Q < 3 ? (x & ((1u << (2 * Q)) - 1u)) : x;  // bit index must not see base t-1
            const uint32_t base = MODE == 0 ? base0 : (MODE == 1 ? base1 : (T < split ? base0 : base1));
            red_or_shared((xn & LG::kWordMask) | base, __funnelshift_l(0u, 1u, tok));  // 1 << (tok & 31)
        }
        lane_token_step<Q, MODE, GUARD, T + 1>(hi, lo, xn, base0, base1, split, lim);
    }
}

template <int Q, int MODE, bool GUARD>
__device__ __forceinline__ void lane_tokens16(uint32_t hi, uint32_t lo, uint32_t base0, uint32_t base1, int split,
                                              int lim) {
    lane_token_step<Q, MODE, GUARD, 0>(hi, lo, lane_window<Q, 0>(hi, lo), base0, base1, split, lim);
}

// Reverses the 2-bit base groups of a packed word: base i (bits 2i, 2i+1)
// moves to bits 31-2i-1 .. 31-2i with its high bit above.
__device__ __forceinline__ uint32_t reverse_bases(uint32_t x) {
    const uint32_t y = __brev(x);
    return ((y >> 1) & 0x55555555u) | ((y & 0x55555555u) << 1);
}

// Staged position of word g of a tile: one pad word after every 32, so that
// the lanes of a warp reading word j of 32 consecutive cores hit distinct banks.
__device__ __forceinline__ int stage_pos(int g) { return g + (g >> 5); }

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Issues the copies of one warp tile's packed words (its 32 cores from c0 and
// the first word after them) into the warp's staging buffer; words past the
// reference are zero-filled by the copy itself.
__device__ __forceinline__ void stage_warp_tile(const uint8_t* __restrict__ ref2bit, int64_t nbytes, int64_t c0,
                                                int wpc, uint32_t stage_s, int lane) {
    const int total = 32 * wpc + 1;
    const int64_t g0 = c0 * (int64_t)wpc;
    if (4 * (g0 + total) <= nbytes) {  // the whole tile lies inside the reference
        const uint8_t* src = ref2bit + 4 * g0;
        for (int i = lane; i < total; i += 32) cp_async4(stage_s + 4u * (uint32_t)stage_pos(i), src + 4 * i, 4);
        return;
    }
    for (int i = lane; i < total; i += 32) {
        const int64_t byte = 4 * (g0 + i);
        const int64_t avail = nbytes - byte;
        const int n = avail >= 4 ? 4 : (avail > 0 ? (int)avail : 0);
        cp_async4(stage_s + 4u * (uint32_t)stage_pos(i), n > 0 ? (const void*)(ref2bit + byte) : (const void*)ref2bit,
                  n);
    }
}

// Persistent, one warp per work unit: warp tile u holds cores
// [u * out_w, u * out_w + 32) and finishes the rows of its first out_w =
// 32 - (J + 1) (the last J + 1 cores only complete their neighbours' rows),
// so a warp never waits for another.  The next warp tile's reference words
// are copied in while the current one is built.
template <int Q>
__global__ void __launch_bounds__(kLaneCores, 4)
bank_build_lanes_kernel(const uint8_t* __restrict__ ref2bit, int64_t len, int bin_len, int r_pref, int J,
                        int64_t n_bins, int64_t n_units, uint32_t* __restrict__ bank) {
    using LG = LaneGeo<Q>;
    constexpr int RW = LG::kRW;
    extern __shared__ uint4 lane_smem4[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int out_w = 32 - (J + 1);   // rows finished per warp tile
    const int wpc = bin_len >> 4;     // packed words per core
    const int stage_words = stage_pos(32 * wpc + 1) + 1;
    const int64_t nbytes = (len + 3) >> 2;

    // rows: the P and R row sets of every warp, aligned so that the word
    // offset bits of a transposed row never meet the base address; then two
    // staging buffers per warp
    const uint32_t raw = shared_addr(lane_smem4);
    const uint32_t pad = ((raw + LG::kRowSetBytes - 1) & ~(uint32_t)(LG::kRowSetBytes - 1)) - raw;
    uint32_t* rows = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(lane_smem4) + pad);
    const uint32_t rows_s = raw + pad;
    uint32_t* my_stage = rows + kLaneWarps * 2 * RW * 32 + warp * 2 * stage_words;
    const uint32_t my_stage_s = rows_s + 4u * (uint32_t)(kLaneWarps * 2 * RW * 32 + warp * 2 * stage_words);
    const uint32_t baseP = rows_s + (uint32_t)((warp * 2) * LG::kRowSetBytes) + 4u * lane;
    const uint32_t baseR = baseP + LG::kRowSetBytes;
    uint32_t* myP = rows + warp * 2 * RW * 32 + lane;  // word w of this lane's P row at myP[32 w]
    uint32_t* myR = myP + RW * 32;
    uint4* my_sets = reinterpret_cast<uint4*>(rows + warp * 2 * RW * 32);

    const int64_t stride = (int64_t)gridDim.x * kLaneWarps;
    int64_t unit = (int64_t)blockIdx.x * kLaneWarps + warp;
    if (unit < n_units) stage_warp_tile(ref2bit, nbytes, unit * out_w, wpc, my_stage_s, lane);
    cp_async_commit();
    // the row sets start zeroed; afterwards every read of them (the rows,
    // then the staged output) swaps in zeros, so no tile needs a clearing pass
#pragma unroll
    for (int i = lane; i < 2 * RW * 8; i += 32) my_sets[i] = make_uint4(0, 0, 0, 0);
    for (int it = 0; unit < n_units; unit += stride, it++) {
        const int64_t c0 = unit * out_w;
        const int buf = it & 1;
        const int64_t next = unit + stride;
        if (next < n_units)
            stage_warp_tile(ref2bit, nbytes, next * out_w, wpc, my_stage_s + 4u * (uint32_t)(stage_words * (buf ^ 1)),
                            lane);
        cp_async_commit();
        cp_async_wait<1>();  // this tile's words have landed (the next tile's may not)
        __syncwarp();

        // token starts of this core: [0, n_lane) (clipped at the reference end)
        {
            const int64_t left = len - Q + 1 - (c0 + lane) * (int64_t)bin_len;
            const int n_lane = left <= 0 ? 0 : (left < bin_len ? (int)left : bin_len);
            const uint32_t* st = my_stage + stage_words * buf;
            const int g = lane * wpc;
            uint32_t hi = reverse_bases(st[stage_pos(g)]);
            for (int j = 0; j < wpc; j++) {
                const uint32_t lo = reverse_bases(st[stage_pos(g + j + 1)]);
                const int s0 = 16 * j;
                const int split = r_pref - s0;  // starts below it go to P (uniform over the warp)
                if (s0 + 16 <= n_lane) {
                    if (split >= 16)
                        lane_tokens16<Q, 0, false>(hi, lo, baseP, baseR, split, 16);
                    else if (split <= 0)
                        lane_tokens16<Q, 1, false>(hi, lo, baseP, baseR, split, 16);
                    else
                        lane_tokens16<Q, 2, false>(hi, lo, baseP, baseR, split, 16);
                } else if (s0 < n_lane) {
                    lane_tokens16<Q, 2, true>(hi, lo, baseP, baseR, split, n_lane - s0);
                }
                hi = lo;
            }
        }
        __syncwarp();

        // this core's bin row: P|R of cores lane .. lane+J, P of core
        // lane+J+1, the neighbours' words by shuffle
        uint32_t v[RW];
#pragma unroll
        for (int w = 0; w < RW; w++) {
            const uint32_t pw = atomicExch(&myP[32 * w], 0u);
            const uint32_t cw = pw | atomicExch(&myR[32 * w], 0u);
            uint32_t x = cw;
            for (int i = 1; i <= J; i++) x |= __shfl_down_sync(kFull, cw, i);
            v[w] = x | __shfl_down_sync(kFull, pw, J + 1);
        }
        __syncwarp();

        // rows through the warp's R row set (free now) in row-major order,
        // 16-byte chunks swizzled by lane, then 512-byte stores
        uint8_t* out_s = reinterpret_cast<uint8_t*>(myR - lane);
#pragma unroll
        for (int c = 0; c < LG::kChunks; c++)
            *reinterpret_cast<uint4*>(out_s + lane * (RW * 4) + 16 * (c ^ (lane & (LG::kChunks - 1)))) =
                make_uint4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        __syncwarp();
        int n_rows = out_w;
        if (c0 + n_rows > n_bins) n_rows = (int)(n_bins - c0);
#pragma unroll
        for (int i = 0; i < LG::kChunks; i++) {
            const int o = (i * 32 + lane) * 16;  // byte offset in the staged rows
            const int r = o / (RW * 4), slot = (o % (RW * 4)) / 16;
            const int c = slot ^ (r & (LG::kChunks - 1));
            unsigned long long* h = reinterpret_cast<unsigned long long*>(out_s + o);
            const unsigned long long lo = atomicExch(h, 0ull), hi = atomicExch(h + 1, 0ull);
            if (r < n_rows)
                reinterpret_cast<uint4*>(bank + (c0 + r) * RW)[c] =
                    make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
        }
        __syncwarp();  // the row sets are cleared before the next tile's tokens
    }
    cp_async_wait<0>();
}

// Shared memory of the lane kernel: row sets (+ alignment slack) and two
// staging buffers per warp.
template <int Q>
constexpr size_t lane_smem_bytes(int bin_len) {
    return (size_t)kLaneWarps * 2 * LaneGeo<Q>::kRowSetBytes + LaneGeo<Q>::kRowSetBytes +
           (size_t)kLaneWarps * 2 * 4 * (size_t)(32 * (bin_len >> 4) + 1 + ((32 * (bin_len >> 4) + 1) >> 5) + 1);
}

template <int Q>
static int launch_lanes(const uint8_t* ref2bit, grim_bank* bank, cudaStream_t s, int r_pref, int J) {
    const int out_w = 32 - (J + 1);
    const int64_t n_units = (bank->n_bins + out_w - 1) / out_w;
    const size_t smem = lane_smem_bytes<Q>(bank->bin_len);
    static DeviceCache attr[64];  // per device: the largest size set so far
    const int slot = device_slot();
    if (slot < 0) return GRIM_ENOTSUP;
    if (attr[slot].load() < (int)smem) {
        GRIM_CUDA_TRY(
            cudaFuncSetAttribute(bank_build_lanes_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr[slot].store((int)smem);
    }
    int per_sm = 0;
    GRIM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bank_build_lanes_kernel<Q>, kLaneCores, smem));
    if (per_sm < 1) return GRIM_ENOTSUP;  // cannot happen below kLaneMaxBinLen
    int64_t blocks = (int64_t)sm_count() * per_sm;
    const int64_t need = (n_units + kLaneWarps - 1) / kLaneWarps;
    if (blocks > need) blocks = need;
    bank_build_lanes_kernel<Q><<<grim::fault_grid((unsigned)blocks), kLaneCores, smem, s>>>(
        ref2bit, bank->len, bank->bin_len, r_pref, J, bank->n_bins, n_units, bank->bits);
    GRIM_CUDA_TRY(cudaGetLastError());
    return GRIM_OK;
}

template <int Q>
static int launch_q(const uint8_t* ref2bit, grim_bank* bank, cudaStream_t s) {
    using G = Geo<Q>;
    // lane-per-core kernel for q <= 5, bins of a multiple of 16 bases, an
    // overlap that holds at least the last token of the core, word-aligned input
    const int64_t e = (int64_t)bank->overlap - Q + 1;  // token starts past the core
    if (Q <= 5 && bank->bin_len % 16 == 0 && bank->bin_len <= kLaneMaxBinLen && e >= 0 &&
        e / bank->bin_len <= kLaneMaxJ && ((uintptr_t)ref2bit & 3) == 0)
        return launch_lanes<Q <= 5 ? Q : 5>(ref2bit, bank, s, (int)(e % bank->bin_len), (int)(e / bank->bin_len));
    const int bins_per_cta = kBuildSmemBytes / (G::kRowWords * 4);
    const int64_t blocks = (bank->n_bins + bins_per_cta - 1) / bins_per_cta;
    if (blocks > 0x7fffffff) return GRIM_ENOTSUP;
    const size_t smem_rows = (size_t)bins_per_cta * G::kRowWords * 4;
    // staged path when a run's packed reference bytes fit beside its rows
    const int64_t span = (int64_t)bins_per_cta * bank->bin_len + bank->overlap;
    const int64_t stage = 4 * (span / 16 + 3);
    if (stage <= kBuildStageBytes) {
        const size_t smem = smem_rows + (size_t)((stage + 15) & ~15LL);
        static DeviceCache attr[64];  // per device
        const int slot = device_slot();
        if (slot < 0) return GRIM_ENOTSUP;
        if (!attr[slot].load() && smem > 48 * 1024) {
            GRIM_CUDA_TRY(cudaFuncSetAttribute(bank_build_staged_kernel<Q>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr[slot].store(1);
        }
        bank_build_staged_kernel<Q><<<grim::fault_grid((unsigned)blocks), kBuildThreads, smem, s>>>(
            ref2bit, bank->len, bank->bin_len, bank->overlap, bank->n_bins, bins_per_cta, bank->bits);
    } else {
        bank_build_kernel<Q><<<grim::fault_grid((unsigned)blocks), kBuildThreads, smem_rows, s>>>(
            ref2bit, bank->len, bank->bin_len, bank->overlap, bank->n_bins, bins_per_cta, bank->bits);
    }
    GRIM_CUDA_TRY(cudaGetLastError());
    return GRIM_OK;
}

int launch_bank_build(const uint8_t* ref2bit, grim_bank* bank, cudaStream_t s) {
    switch (bank->q) {
        case 1: return launch_q<1>(ref2bit, bank, s);
        case 2: return launch_q<2>(ref2bit, bank, s);
        case 3: return launch_q<3>(ref2bit, bank, s);
        case 4: return launch_q<4>(ref2bit, bank, s);
        case 5: return launch_q<5>(ref2bit, bank, s);
        case 6: return launch_q<6>(ref2bit, bank, s);
        default: return GRIM_ENOTSUP;
    }
}

}  // namespace grim
