// Bank build (Sec. 3.1): the 2-bit packed reference -> one 4^q-bit
// existence bitvector per bin, bin-major in HBM.
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
constexpr int kBuildSmemBytes = 16384;

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

template <int Q>
static int launch_q(const uint8_t* ref2bit, grim_bank* bank, cudaStream_t s) {
    using G = Geo<Q>;
    const int bins_per_cta = kBuildSmemBytes / (G::kRowWords * 4);
    const int64_t blocks = (bank->n_bins + bins_per_cta - 1) / bins_per_cta;
    if (blocks > 0x7fffffff) return GRIM_ENOTSUP;
    const size_t smem = (size_t)bins_per_cta * G::kRowWords * 4;
    bank_build_kernel<Q><<<(unsigned)blocks, kBuildThreads, smem, s>>>(ref2bit, bank->len, bank->bin_len,
                                                                      bank->overlap, bank->n_bins, bins_per_cta,
                                                                      bank->bits);
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
