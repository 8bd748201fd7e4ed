// Bank build (Sec. 3.1): the 2-bit packed reference -> one 4^q-bit
// existence bitvector per bin, bin-major in HBM.
// (Two kernels: a staged fast path for bins of ordinary length, and a
// general one that reads the reference through L1, used when a run's span
// of reference would not fit in shared memory.)
//
// One CTA owns a run of consecutive bins and keeps their rows in shared
// memory.  Its threads walk every token start of the run's spans once
// (consecutive threads on consecutive positions, so the packed reference
// bytes are read coalesced through L1), form the token from its q bases and
// set the token's bit in every bin of the run whose span holds it (one or
// two bins for overlap < bin_len) with a shared-memory atomicOr.  The rows
// then leave in 16-byte stores; each row is written exactly once.
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

template <int Q>
static int launch_q(const uint8_t* ref2bit, grim_bank* bank, cudaStream_t s) {
    using G = Geo<Q>;
    const int bins_per_cta = kBuildSmemBytes / (G::kRowWords * 4);
    const int64_t blocks = (bank->n_bins + bins_per_cta - 1) / bins_per_cta;
    if (blocks > 0x7fffffff) return GRIM_ENOTSUP;
    const size_t smem_rows = (size_t)bins_per_cta * G::kRowWords * 4;
    // staged path when a run's packed reference bytes fit beside its rows
    const int64_t span = (int64_t)bins_per_cta * bank->bin_len + bank->overlap;
    const int64_t stage = 4 * (span / 16 + 3);
    if (stage <= kBuildStageBytes) {
        const size_t smem = smem_rows + (size_t)((stage + 15) & ~15LL);
        static bool attr[64] = {};  // per device
        const int slot = device_slot();
        if (slot < 0) return GRIM_ENOTSUP;
        if (!attr[slot] && smem > 48 * 1024) {
            GRIM_CUDA_TRY(cudaFuncSetAttribute(bank_build_staged_kernel<Q>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr[slot] = true;
        }
        bank_build_staged_kernel<Q><<<(unsigned)blocks, kBuildThreads, smem, s>>>(
            ref2bit, bank->len, bank->bin_len, bank->overlap, bank->n_bins, bins_per_cta, bank->bits);
    } else {
        bank_build_kernel<Q><<<(unsigned)blocks, kBuildThreads, smem_rows, s>>>(
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
