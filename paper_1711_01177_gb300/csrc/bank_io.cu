// Bank files and the packed bitmask.
//
// The bank depends only on the reference and (q, bin_len, overlap); the
// paper builds it once per reference and keeps it (Sec. 3.1, Sec. 6.1).
// grim_bank_save writes it to a file in its device layout behind a 64-byte
// header; grim_bank_load reads it back onto the current device.  The header
// (host byte order; x86-64 and aarch64 are both little-endian):
//   0  char[8]  "GRIMBNK1"          32 int64  n_bins
//   8  uint32   64 (header bytes)   40 int64  row_words
//  12  uint32   q                   48 uint64 payload bytes
//  16  int64    len                 56 uint64 payload checksum
//  24  int32    bin_len, 28 int32 overlap
// The checksum: h = 0x9E3779B97F4A7C15 ^ payload bytes, then for every
// 8-byte word w of the payload h = (h ^ w) * 0x100000001B3.
//
// grim_pack_mask packs the filter's byte mask into the one-bit-per-location
// seed location filter bitmask of Sec. 3.3.
#include <stdio.h>
#include <string.h>

#include "grim_internal.cuh"

namespace grim {
namespace {

constexpr char kMagic[8] = {'G', 'R', 'I', 'M', 'B', 'N', 'K', '1'};
constexpr size_t kChunk = size_t(64) << 20;  // staging bytes per copy

struct BankHeader {
    char magic[8];
    uint32_t header_bytes, q;
    int64_t len;
    int32_t bin_len, overlap;
    int64_t n_bins, row_words;
    uint64_t payload, checksum;
};
static_assert(sizeof(BankHeader) == 64, "bank header layout");

uint64_t checksum_init(uint64_t payload) { return 0x9E3779B97F4A7C15ull ^ payload; }

uint64_t checksum_step(uint64_t h, const unsigned char* p, size_t n) {  // n: multiple of 8
    for (size_t i = 0; i < n; i += 8) {
        uint64_t w;
        memcpy(&w, p + i, 8);
        h = (h ^ w) * 0x100000001B3ull;
    }
    return h;
}

__global__ void pack_mask_kernel(const uint8_t* __restrict__ pass, int64_t n, bool aligned,
                                 uint32_t* __restrict__ bits) {
    const int64_t words = (n + 31) / 32;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b0 = w * 32;
        uint32_t m = 0;
        if (aligned && b0 + 32 <= n) {
            const uint4* v = reinterpret_cast<const uint4*>(pass + b0);
            m = nonzero_bytes16(__ldg(v)) | (nonzero_bytes16(__ldg(v + 1)) << 16);
        } else {
            for (int i = 0; i < 32; i++)
                if (b0 + i < n && pass[b0 + i]) m |= 1u << i;
        }
        bits[w] = m;
    }
}

}  // namespace
}  // namespace grim

extern "C" {

int grim_bank_save(const grim_bank* bank, const char* path, void* stream) {
    if (!bank || !path) return GRIM_EINVAL;
    int rc = grim::check_device(bank);
    if (rc != GRIM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    grim::BankHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, grim::kMagic, 8);
    h.header_bytes = sizeof(h);
    h.q = (uint32_t)bank->q;
    h.len = bank->len;
    h.bin_len = bank->bin_len;
    h.overlap = bank->overlap;
    h.n_bins = bank->n_bins;
    h.row_words = bank->row_words;
    h.payload = (uint64_t)bank->n_bins * (uint64_t)bank->row_words * 4;
    FILE* f = fopen(path, "wb");
    if (!f) return GRIM_EIO;
    unsigned char* stage = nullptr;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = grim::fault_alloc_now() ? cudaErrorMemoryAllocation : cudaMallocHost((void**)&stage, grim::kChunk);
    uint64_t sum = grim::checksum_init(h.payload);
    bool io_ok = fwrite(&h, sizeof(h), 1, f) == 1;  // checksum rewritten at the end
    const unsigned char* src = reinterpret_cast<const unsigned char*>(bank->bits);
    for (uint64_t done = 0; e == cudaSuccess && io_ok && done < h.payload; done += grim::kChunk) {
        const size_t n = (size_t)(h.payload - done < grim::kChunk ? h.payload - done : grim::kChunk);
        e = cudaMemcpyAsync(stage, src + done, n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        sum = grim::checksum_step(sum, stage, n);
        io_ok = fwrite(stage, 1, n, f) == n;
    }
    if (e == cudaSuccess && io_ok) {
        h.checksum = sum;
        io_ok = fseek(f, 0, SEEK_SET) == 0 && fwrite(&h, sizeof(h), 1, f) == 1;
    }
    io_ok = (fclose(f) == 0) && io_ok;
    if (stage) cudaFreeHost(stage);
    if (e != cudaSuccess) {
        grim::set_last_cuda_error(e);
        return e == cudaErrorMemoryAllocation ? GRIM_ENOMEM : GRIM_ECUDA;
    }
    return io_ok ? GRIM_OK : GRIM_EIO;
}

int grim_bank_load(const char* path, void* stream, grim_bank** out) {
    if (!path || !out) return GRIM_EINVAL;
    *out = nullptr;
    // the header and the file's size are checked before any device work
    FILE* f = fopen(path, "rb");
    if (!f) return GRIM_EIO;
    grim::BankHeader h;
    bool ok = fread(&h, sizeof(h), 1, f) == 1 && memcmp(h.magic, grim::kMagic, 8) == 0 &&
              h.header_bytes == sizeof(h) && h.q >= 1 && h.q <= GRIM_MAX_Q && h.len >= 1 && h.bin_len >= 1 &&
              h.overlap >= 0 && h.n_bins == (h.len + h.bin_len - 1) / h.bin_len &&
              h.row_words == grim::row_words_for((int)h.q) &&
              h.payload == (uint64_t)h.n_bins * (uint64_t)h.row_words * 4;
    if (ok) {
        ok = fseek(f, 0, SEEK_END) == 0;
        const long end = ok ? ftell(f) : -1;
        ok = ok && end >= 0 && (uint64_t)end == sizeof(h) + h.payload && fseek(f, sizeof(h), SEEK_SET) == 0;
    }
    if (!ok) {
        fclose(f);
        return GRIM_EIO;
    }
    cudaStream_t s = (cudaStream_t)stream;
    grim_bank* bank = nullptr;
    int rc = grim::new_bank(h.len, (int)h.q, h.bin_len, h.overlap, s, &bank);
    if (rc != GRIM_OK) {
        fclose(f);
        return rc;
    }
    unsigned char* stage = nullptr;
    cudaError_t e =
        grim::fault_alloc_now() ? cudaErrorMemoryAllocation : cudaMallocHost((void**)&stage, grim::kChunk);
    uint64_t sum = grim::checksum_init(h.payload);
    unsigned char* dst = reinterpret_cast<unsigned char*>(bank->bits);
    for (uint64_t done = 0; e == cudaSuccess && ok && done < h.payload; done += grim::kChunk) {
        const size_t n = (size_t)(h.payload - done < grim::kChunk ? h.payload - done : grim::kChunk);
        e = cudaStreamSynchronize(s);  // the staging buffer is free again
        if (e != cudaSuccess) break;
        ok = fread(stage, 1, n, f) == n;
        if (!ok) break;
        sum = grim::checksum_step(sum, stage, n);
        e = cudaMemcpyAsync(dst + done, stage, n, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    fclose(f);
    if (stage) cudaFreeHost(stage);
    if (e != cudaSuccess || !ok || sum != h.checksum) {
        grim::delete_bank(bank);
        if (e != cudaSuccess) {
            grim::set_last_cuda_error(e);
            return e == cudaErrorMemoryAllocation ? GRIM_ENOMEM : GRIM_ECUDA;
        }
        return GRIM_EIO;
    }
    *out = bank;
    return GRIM_OK;
}

int grim_pack_mask(const uint8_t* pass, int64_t n, uint32_t* bits, void* stream) {
    if (n < 0) return GRIM_EINVAL;
    if (n == 0) return GRIM_OK;
    if (!pass || !bits) return GRIM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t words = (n + 31) / 32;
    const int64_t need = (words + 255) / 256;
    const int64_t cap = (int64_t)grim::sm_count() * 16;
    grim::pack_mask_kernel<<<grim::fault_grid((unsigned)(need < cap ? need : cap)), 256, 0, s>>>(
            pass, n, ((uintptr_t)pass & 15) == 0, bits);
    GRIM_CUDA_TRY(cudaGetLastError());
    return GRIM_OK;
}

}  // extern "C"
