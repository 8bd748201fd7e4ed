// Roofline denominators measured on the device the library runs on: the
// L2 read bandwidth (for workloads whose bank stays in L2), the dense
// tcgen05 tensor rates of the MMA kinds the full scan can use, and the
// legacy mma.sync INT8 rate quoted beside them.  None of this computes any
// part of the filter; the benchmark divides its achieved rates by these.
//
//   l2_read_kernel    every thread streams 16-byte L2-only loads (ld.global.cg,
//                     four in flight) over a buffer that fits the L2, pass
//                     after pass, and folds them into one word;
//   tc_peak_kernel    one CTA per SM, one thread issuing back-to-back
//                     tcgen05.mma (M = 128, N = 256) on operands that stay in
//                     shared or tensor memory, one commit at the end;
//   int8_mma_kernel   eight independent mma.sync m16n8k32 s8 chains per warp.
#include "grim_internal.cuh"
#include "tcgen05.cuh"

namespace grim {

// ------------------------------------------------------------ L2 read

__global__ void __launch_bounds__(256) l2_read_kernel(const uint4* __restrict__ buf, int64_t n_vec, int reps,
                                                      uint32_t* __restrict__ out) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t acc = 0;
    for (int r = 0; r < reps; r++) {
        // consecutive passes start at different threads so no SM keeps one
        // slice; four independent loads in flight per thread
        const int64_t shift = ((int64_t)r * 977 * 16) % n_vec;
        int64_t i = tid;
        for (; i + 3 * stride < n_vec; i += 4 * stride) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                int64_t j = i + u * stride + shift;
                j = j >= n_vec ? j - n_vec : j;
                v[u] = __ldcg(buf + j);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        }
        for (; i < n_vec; i += stride) {
            int64_t j = i + shift;
            j = j >= n_vec ? j - n_vec : j;
            const uint4 v = __ldcg(buf + j);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    out[tid] = acc;
}

// ------------------------------------------------------------ tensor rate

constexpr int kPeakM = 128, kPeakN = 256;
constexpr int kPeakABytes = kPeakM * 128;  // one 128-byte K block of A (swizzled K-major)
constexpr int kPeakBBytes = kPeakN * 128;  // and of B
constexpr int kPeakSmem = kPeakABytes + kPeakBBytes + 1024 + 64;

// MODE 0: kind::f8f6f4 e4m3, A smem;  1: kind::mxf4, A smem;
//      2: kind::mxf4, A tmem;         3: kind::f8f6f4 e4m3, A tmem.
// N: the MMA's N (256, or 128 as in the full scan).
// The MMAs cycle over the four 32-byte K slices of one 128-byte block.
template <int MODE, int N>
__global__ void __launch_bounds__(128, 1) tc_peak_kernel(int64_t iters, uint32_t seed, uint32_t* status) {
    extern __shared__ uint8_t peak_smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)peak_smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + kPeakABytes;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sB + kPeakBBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + 3);
    const int warp = threadIdx.x >> 5;
    constexpr bool kMx = MODE == 1 || MODE == 2;
    constexpr bool kTmemA = MODE == 2 || MODE == 3;
    // tensor memory: accumulator [0, 256), scale factors [256, 288) and
    // [288, 320), A slices [320, 352)
    constexpr uint32_t kSfaCol = 256, kSfbCol = 288, kACol = 320;

    // operands: hash-filled bytes (e4m3: bit 3 cleared, so no NaN)
    for (int i = threadIdx.x; i < (kPeakABytes + kPeakBBytes) / 4; i += blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B1u + seed;
        h ^= h >> 15;
        h *= 0x2C1B3C6Du;
        h ^= h >> 12;
        reinterpret_cast<uint32_t*>(smem)[i] = kMx ? h : (h & 0x77777777u);
    }
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, 512);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    if (kMx || kTmemA) {
        // scale factors 1.0 (ue8m0 127 in every byte) and A slices in tensor memory
        uint32_t v[32];
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = 0x7F7F7F7Fu;
        tmem_st32(tmem + lane_base + kSfaCol, v);
        tmem_st32(tmem + lane_base + kSfbCol, v);
#pragma unroll
        for (int i = 0; i < 32; i++) {
            uint32_t h = (uint32_t)(threadIdx.x * 32 + i) * 0x85EBCA6Bu + seed;
            h ^= h >> 13;
            v[i] = kMx ? h : (h & 0x77777777u);
        }
        tmem_st32(tmem + lane_base + kACol, v);
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (threadIdx.x == 0) {
        const uint32_t idesc = kMx ? idesc_mxf4(kPeakM, N) : idesc_f8(kPeakM, N);
        const uint32_t a_s = smem_addr(sA), b_s = smem_addr(sB);
        for (int64_t i = 0; i < iters; i++) {
            const uint32_t kk = (uint32_t)i & 3;
            const uint64_t bdesc = smem_desc_sw128(b_s + kk * 32);
            if (MODE == 0) mma_f8f6f4_smemA(tmem, smem_desc_sw128(a_s + kk * 32), bdesc, idesc, i != 0);
            if (MODE == 1)
                mma_mxf4_smemA(tmem, smem_desc_sw128(a_s + kk * 32), bdesc, idesc, tmem + kSfaCol, tmem + kSfbCol,
                               i != 0);
            if (MODE == 2)
                mma_mxf4_tmemA(tmem, tmem + kACol + kk * 8, bdesc, idesc, tmem + kSfaCol, tmem + kSfbCol, i != 0);
            if (MODE == 3) mma_f8f6f4_tmemA(tmem, tmem + kACol + kk * 8, bdesc, idesc, i != 0);
        }
        mma_commit(bar);
        if (!mbar_wait(bar, 0, abort_flag)) {
            // a second bounded wait for the MMAs before tensor memory is freed
            const unsigned long long t0 = now_ns();
            while (!mbar_try_wait(bar, 0) && now_ns() - t0 < kWaitLimitNs) {
            }
            atomicOr(status, GRIM_FLAG_TIMEOUT);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------ mma.sync INT8

__global__ void __launch_bounds__(256) int8_mma_kernel(int64_t iters, uint32_t seed, int32_t* __restrict__ out) {
    uint32_t a[4], b[2];
    for (int i = 0; i < 4; i++) a[i] = (threadIdx.x + i) * 0x01030507u + seed;
    for (int i = 0; i < 2; i++) b[i] = (threadIdx.x * 3 + i) * 0x0705030Bu ^ seed;
    int32_t c[8][4];
    for (int k = 0; k < 8; k++)
        for (int i = 0; i < 4; i++) c[k][i] = 0;
    for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 8; k++)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                "{%0, %1, %2, %3};"
                : "+r"(c[k][0]), "+r"(c[k][1]), "+r"(c[k][2]), "+r"(c[k][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    int32_t s = 0;
    for (int k = 0; k < 8; k++)
        for (int i = 0; i < 4; i++) s += c[k][i];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace grim

extern "C" {

int grim_peak(int kind, int64_t work, double* units, float* ms, void* stream) {
    if (!units || !ms || work < 1) return GRIM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = grim::sm_count();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    int rc = GRIM_OK;
    double u = 0;
    GRIM_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    if (kind == GRIM_PEAK_L2_READ) {
        // work = buffer bytes (a multiple of 16, at most 64 MiB so it stays in L2)
        if (work % 16 != 0 || work > (64ll << 20)) rc = GRIM_EINVAL;
        const int blocks = sms * 8, threads = 256;
        scratch_bytes = (size_t)work + (size_t)blocks * threads * 4;
        if (rc == GRIM_OK && err == cudaSuccess) err = grim::scratch_alloc(&scratch, scratch_bytes, s);
        if (rc == GRIM_OK && err == cudaSuccess) err = cudaMemsetAsync(scratch, 0x5A, (size_t)work, s);
        const int reps = 40;
        uint32_t* out = reinterpret_cast<uint32_t*>((uint8_t*)scratch + work);
        if (rc == GRIM_OK && err == cudaSuccess) {
            grim::l2_read_kernel<<<grim::fault_grid(blocks), threads, 0, s>>>((const uint4*)scratch, work / 16, 2,
                                                                              out);
            err = cudaGetLastError();
        }
        if (rc == GRIM_OK && err == cudaSuccess) err = cudaEventRecord(e0, s);
        if (rc == GRIM_OK && err == cudaSuccess) {
            grim::l2_read_kernel<<<grim::fault_grid(blocks), threads, 0, s>>>((const uint4*)scratch, work / 16, reps,
                                                                              out);
            err = cudaGetLastError();
        }
        u = (double)work * reps;
    } else if ((kind >= GRIM_PEAK_E4M3 && kind <= GRIM_PEAK_E4M3_TMEM_A) || kind == GRIM_PEAK_MXF4_TMEM_A_N128 ||
               kind == GRIM_PEAK_E4M3_TMEM_A_N128) {
        // work = MMAs per CTA; one CTA per SM
        const size_t smem = grim::kPeakSmem;
        const int mode = kind == GRIM_PEAK_MXF4_TMEM_A_N128 ? 2
                         : kind == GRIM_PEAK_E4M3_TMEM_A_N128 ? 3
                                                              : kind - GRIM_PEAK_E4M3;
        const int k_elems = (mode == 1 || mode == 2) ? 64 : 32;
        const int n_mma = kind >= GRIM_PEAK_MXF4_TMEM_A_N128 ? 128 : grim::kPeakN;
        scratch_bytes = 256;
        if (err == cudaSuccess) err = grim::scratch_alloc(&scratch, scratch_bytes, s);
        if (err == cudaSuccess) err = cudaMemsetAsync(scratch, 0, 4, s);
        const bool n128 = kind >= GRIM_PEAK_MXF4_TMEM_A_N128;
        auto launch = [&](int64_t iters) {
            uint32_t* st = (uint32_t*)scratch;
            const unsigned g = grim::fault_grid(sms);
            switch (mode + (n128 ? 4 : 0)) {
                case 0: grim::tc_peak_kernel<0, 256><<<g, 128, smem, s>>>(iters, 0x1234u, st); break;
                case 1: grim::tc_peak_kernel<1, 256><<<g, 128, smem, s>>>(iters, 0x1234u, st); break;
                case 2: grim::tc_peak_kernel<2, 256><<<g, 128, smem, s>>>(iters, 0x1234u, st); break;
                case 3: grim::tc_peak_kernel<3, 256><<<g, 128, smem, s>>>(iters, 0x1234u, st); break;
                case 6: grim::tc_peak_kernel<2, 128><<<g, 128, smem, s>>>(iters, 0x1234u, st); break;
                default: grim::tc_peak_kernel<3, 128><<<g, 128, smem, s>>>(iters, 0x1234u, st); break;
            }
            return cudaGetLastError();
        };
        const cudaFuncAttribute kSmemAttr = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (err == cudaSuccess) err = cudaFuncSetAttribute(grim::tc_peak_kernel<0, 256>, kSmemAttr, (int)smem);
        if (err == cudaSuccess) err = cudaFuncSetAttribute(grim::tc_peak_kernel<1, 256>, kSmemAttr, (int)smem);
        if (err == cudaSuccess) err = cudaFuncSetAttribute(grim::tc_peak_kernel<2, 256>, kSmemAttr, (int)smem);
        if (err == cudaSuccess) err = cudaFuncSetAttribute(grim::tc_peak_kernel<3, 256>, kSmemAttr, (int)smem);
        if (err == cudaSuccess) err = cudaFuncSetAttribute(grim::tc_peak_kernel<2, 128>, kSmemAttr, (int)smem);
        if (err == cudaSuccess) err = cudaFuncSetAttribute(grim::tc_peak_kernel<3, 128>, kSmemAttr, (int)smem);
        if (err == cudaSuccess) err = launch(work < 64 ? work : 64);  // warm-up
        if (err == cudaSuccess) err = cudaEventRecord(e0, s);
        if (err == cudaSuccess) err = launch(work);
        u = 2.0 * grim::kPeakM * n_mma * k_elems * (double)work * sms;
    } else if (kind == GRIM_PEAK_INT8_MMA_SYNC) {
        // work = loop trips; 8 mma.sync per trip per warp
        const int blocks = sms * 4, threads = 256;
        scratch_bytes = (size_t)blocks * threads * 4;
        if (err == cudaSuccess) err = grim::scratch_alloc(&scratch, scratch_bytes, s);
        if (err == cudaSuccess) {
            grim::int8_mma_kernel<<<grim::fault_grid(blocks), threads, 0, s>>>(work < 16 ? work : 16, 7u,
                                                                               (int32_t*)scratch);
            err = cudaGetLastError();
        }
        if (err == cudaSuccess) err = cudaEventRecord(e0, s);
        if (err == cudaSuccess) {
            grim::int8_mma_kernel<<<grim::fault_grid(blocks), threads, 0, s>>>(work, 7u, (int32_t*)scratch);
            err = cudaGetLastError();
        }
        u = 2.0 * 16 * 8 * 32 * 8 * (double)work * (blocks * threads / 32);
    } else {
        rc = GRIM_EINVAL;
    }
    if (rc == GRIM_OK && err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (rc == GRIM_OK && err == cudaSuccess) err = cudaEventSynchronize(e1);
    float t = 0;
    if (rc == GRIM_OK && err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    uint32_t flags = 0;
    if (rc == GRIM_OK && err == cudaSuccess && kind >= GRIM_PEAK_E4M3 && kind != GRIM_PEAK_INT8_MMA_SYNC)
        err = cudaMemcpy(&flags, scratch, 4, cudaMemcpyDeviceToHost);
    if (scratch) cudaFreeAsync(scratch, s);
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != GRIM_OK) return rc;
    if (err != cudaSuccess) {
        grim::set_last_cuda_error(err);
        return err == cudaErrorMemoryAllocation ? GRIM_ENOMEM : GRIM_ECUDA;
    }
    if (flags & GRIM_FLAG_TIMEOUT) return GRIM_ETIMEOUT;
    *units = u;
    *ms = t;
    return GRIM_OK;
}

}  // extern "C"
