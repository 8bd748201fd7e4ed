// Full-scan form: every read of a batch against every bin of a window
// (the filter of Sec. 3.2 applied to all bins, as the paper's bin window of
// Sec. 6.1 checks consecutive bins in lockstep), written as the dense
// contraction it is:
//     Sum[b, r] = sum_t bit_b(t) * count_r(t)        (K = 4^q tokens)
// on the tcgen05 tensor cores, exactly.
//
// Exactness.  sm_103a has no integer tcgen05 kind, so the contraction runs
// on kind::mxf4: e2m1 operands (four-bit floats, two per byte), unit block
// scales, f32 accumulation.  Token t = 32i + 4j + s of a row takes the K
// position 32i + 8s + j, so that one bank word x (tokens 32i .. 32i+31)
// becomes four A words by masking alone: x & 0x11111111 (slot s = 0, a set
// bit reads as e2m1 0.5), x & 0x22222222 (s = 1, 1.0), x & 0x44444444
// (s = 2, 2.0) and (x >> 1) & 0x44444444 (s = 3, 2.0).  B = the read's token
// counts in base-4 digits (count = sum_d 4^d * digit_d, digit_d in 0..3),
// each scaled by the inverse of its slot's A value (2 d, d, d / 2, d / 2 -
// all exact in e2m1), so every product is the digit itself; every digit of
// every read is its own B row, and the epilogue recombines
// Sum = sum_d 4^d * acc_d.  Every partial sum is a small integer, so the f32
// accumulation is exact and the pass decision is bit-identical to counting
// tokens one by one.  Reads whose counts stay below 4 (nearly all) take one
// row; counts up to 15, 255 and 65,535 take 2, 4 and 8; the prep kernel packs
// reads into tiles of 256 rows by digit class (256 x 1, 128 x 2, 64 x 4, 32 x 8).
//
// Data flow per CTA (persistent, one per SM; a work item = one read tile x
// one run of bin tiles):
//   B   : the read tile's 256 digit rows x K/2 bytes, staged once per work
//         item in shared memory in the 128-byte-swizzled K-major layout;
//   bank: tiles of 128 bin rows stream through a 4-deep shared-memory ring
//         by 2-D TMA tensor copies (warp 0), 16-byte chunks swizzled across
//         the banks so that the expanders' row reads never collide;
//   A   : warps 2-5 (one thread per bin = per TMEM lane) mask 512 bits of
//         their bin's row into 512 e2m1 values and store them straight into
//         tensor memory (3 stages of 64 columns, 8 MMAs per stage) - the
//         expanded operand never touches shared memory;
//   MMA : warp 1 issues M=128 (bins) x N=256 (rows) x K=64 tcgen05.mma with A
//         from TMEM, B from shared memory and the unit scale factors from
//         TMEM, accumulating in one 256-column TMEM accumulator (at N=256 an
//         MMA runs at the full rate whatever the commits and operand
//         rotation around it; at N=128 those cost ~40%);
//   out : warps 6-21, four per lane quadrant, each load a quarter of the
//         tile's accumulator columns (64) with tcgen05.ld in one round and
//         hand the accumulator back to the MMAs at once (with one
//         accumulator, the MMAs wait for it), then recombine digits,
//         compare with each read's threshold and append the rare passing
//         (read, bin, sum) triples with warp-aggregated atomics.
// Every wait is an mbarrier try_wait bounded by a time limit; on expiry the
// CTA raises GRIM_FLAG_TIMEOUT, drains and frees its tensor memory.
#include <cuda.h>  // CUtensorMap (encoded through the runtime's driver entry point)
#include <cudaTypedefs.h>

#include <mutex>

#include "grim_internal.cuh"
#include "tcgen05.cuh"
#include "tokens.cuh"

namespace grim {

// Working memory of grim_scan_noalloc: a fixed array in every device image
// of the library, for callers that cannot allocate device memory.  Host code
// must not pass the name itself to a kernel (on the host it is a stand-in,
// not a device address); scan_noalloc_scratch() looks the address up.
static __device__ __align__(256) uint8_t g_scan_scratch[GRIM_SCAN_NOALLOC_SCRATCH_BYTES];

// ------------------------------------------------------------ constants

constexpr int kScanThreads = 704;   // 22 warps: TMA, MMA, 4 expand, 16 epilogue
constexpr int kExpandWarp0 = 2;     // expander warps 2..5, one per TMEM lane quadrant
constexpr int kEpilogueWarp0 = 6;   // epilogue warps 6..21: four per quadrant, each a quarter of the reads
constexpr int kEpilogueWarps = 16;
static_assert(kEpilogueWarp0 == kExpandWarp0 + 4 && kScanThreads == 32 * (kEpilogueWarp0 + kEpilogueWarps),
              "warp roles: TMA, MMA, four expanders, the epilogue");
constexpr int kBinTile = 128;       // bins per MMA tile (M, TMEM lanes)
constexpr int kRowsTile = 256;      // B rows per read tile (N)
constexpr int kBankStages = 4;
constexpr int kAStages = 3;         // A stages in tensor memory, filled by alternate expander groups
constexpr int kAccCol = 0;          // the accumulator: columns [0, 256)
constexpr int kSfCol = 256;         // unit scale factors of A and B: columns [256, 288)
constexpr int kACol = 288;          // A stages: 3 x 64 columns from 288
constexpr int kTmemCols = 512;
constexpr int kPrepWarps = 8;
constexpr int kNumClasses = 4;      // digit classes: 1, 2, 4, 8 base-4 digits
constexpr int kMmaK = 64;           // e2m1 K elements per MMA (32 bytes of a row)

__host__ __device__ constexpr int class_digits(int c) { return 1 << c; }
__host__ __device__ constexpr int class_reads(int c) { return kRowsTile >> c; }

template <int Q>
struct ScanGeo {
    static constexpr int kRowWords = Geo<Q>::kRowWords;
    static constexpr int kRowBytes = kRowWords * 4;
    static constexpr int kK = (1 << (2 * Q)) < 256 ? 256 : (1 << (2 * Q));  // padded token count
    static constexpr int kKBytes = kK / 2;                                   // a B row: two e2m1 per byte
    static constexpr int kChunkTok = kK >= 512 ? 512 : kK;                   // tokens per A stage
    static constexpr int kACols = kChunkTok / 8;                              // TMEM columns per A stage
    static constexpr int kWordsPerChunk = kChunkTok / 32;                     // bank words per A stage
    static constexpr int kMmaPerChunk = kChunkTok / kMmaK;                    // MMAs per A stage
    static constexpr int kChunks = kK / kChunkTok;
    static constexpr int kBBytes = kRowsTile * kKBytes;                       // staged B tile
    static constexpr int kBankTileBytes = kBinTile * kRowBytes;
    // TMA swizzle of the bank tiles: 16-byte chunk bits [4, 7) of a shared
    // address XOR its bits [7, 10) (128-byte rows), bit 4 XOR bit 7 (32-byte
    // rows), none for 16-byte rows
    static constexpr uint32_t kSwzMask = kRowBytes >= 128 ? 7u : (kRowBytes >= 32 ? 1u : 0u);
    static_assert(kRowBytes * 8 <= kK, "a bank row fits the padded K");
    static_assert(kKBytes % 128 == 0 && kACols <= 64, "B rows are whole 128-byte swizzle atoms");
};

// Scratch written by the prep kernel and read by the scan kernel.
struct ScanScratch {
    int32_t* class_count;  // [4] reads per digit class
    int32_t* work;         // [1] work-item counter
    uint8_t* rows[kNumClasses];   // digit rows, tiles of 128 rows x K/2 bytes (e2m1)
    int32_t* T[kNumClasses];      // thresholds per slot (INT_MAX: never passes)
    uint32_t* rid[kNumClasses];   // read index per slot
};

struct ScanOut {
    uint32_t* pair_read;
    uint32_t* pair_bin;
    uint16_t* pair_sum;          // nullable
    int64_t cap;
    unsigned long long* n_pairs;  // device counter
    uint32_t* read_pass;         // nullable, per read
};

// ------------------------------------------------------------ bounded-wait self-check

// The bounded wait above on a barrier that nothing completes: out = 1 when
// it gave up with the abort flag raised, 0 otherwise.
__global__ void wait_selfcheck_kernel(unsigned long long limit_ns, uint32_t* out) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool done = mbar_wait(&bar, 0, &abort_flag, limit_ns);
        *out = (!done && abort_flag) ? 1u : 0u;
    }
}


// e2m1 code of a base-4 digit d in token slot s (t % 4): the B value is the
// digit divided by the slot's A value (0.5, 1, 2, 2), i.e. 2d, d, d/2, d/2:
// codes {0, 4, 6, 7}, {0, 2, 4, 5}, {0, 1, 2, 3} (e2m1: 0, .5, 1, 1.5, 2, 3, 4, 6).
__device__ __forceinline__ uint32_t e2m1_digit(uint32_t s, uint32_t d) {
    constexpr unsigned long long kTab = 0x321054207640ull;  // nibble 4 * (4 * min(s, 2) + d)
    return (uint32_t)(kTab >> (16 * (s < 2 ? s : 2) + 4 * d)) & 0xFu;
}

// A operand: bank word x (tokens 32i .. 32i+31) -> four e2m1 words, slot s
// of token 32i + 4j + s in nibble j of word s.
__device__ __forceinline__ void expand_word_fp4(uint32_t x, uint32_t* v) {
    v[0] = x & 0x11111111u;
    v[1] = x & 0x22222222u;
    v[2] = x & 0x44444444u;
    v[3] = (x >> 1) & 0x44444444u;
}

// ------------------------------------------------------------ prep kernel

// Per read: token counts -> digit class -> digit rows (e2m1), threshold and
// read index at the read's slot in its class.
template <int Q>
__global__ void __launch_bounds__(kPrepWarps * 32)
scan_prep_kernel(const uint8_t* __restrict__ reads, const int64_t* __restrict__ read_offsets, int64_t n_reads,
                 const uint16_t* __restrict__ E, ScanScratch sc, uint32_t* __restrict__ status) {
    using G = ScanGeo<Q>;
    constexpr int kCountWords = (G::kK + 1) / 2;  // u16 counts, two per word
    extern __shared__ uint4 prep_smem[];
    uint16_t* tab = reinterpret_cast<uint16_t*>(prep_smem);
    uint32_t* counts_all = reinterpret_cast<uint32_t*>(prep_smem) + TokenTable<Q>::kWords;
    build_token_table<Q>(tab);
    for (int i = threadIdx.x; i < kPrepWarps * kCountWords; i += blockDim.x) counts_all[i] = 0;
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* counts = counts_all + warp * kCountWords;
    constexpr int kGroups = G::kK / 32;  // 32-token groups of a row: lane i < kGroups writes group i
    uint32_t flags = 0;
    const int64_t stride = (int64_t)gridDim.x * kPrepWarps;
    for (int64_t r = (int64_t)blockIdx.x * kPrepWarps + warp; r < n_reads; r += stride) {
        const int64_t ro = read_offsets[r], re = read_offsets[r + 1];
        bool bad = false;
        int L = 0;
        if (re < ro) {
            flags |= GRIM_FLAG_BAD_OFFSETS;
            bad = true;
        } else if (re - ro > GRIM_MAX_READ_LEN) {
            flags |= GRIM_FLAG_LONG_READ;
            bad = true;
        } else {
            L = (int)(re - ro);
        }
        uint32_t bad_base = 0;
        for_each_token<Q>(reads + ro, L, lane, tab, bad_base, [&](uint32_t tok) {
            atomicAdd(&counts[tok >> 1], 1u << (16 * (tok & 1)));
        });
        if (__any_sync(kFull, bad_base)) {
            flags |= GRIM_FLAG_BAD_BASE;
            bad = true;
        }
        __syncwarp();
        // this lane's tokens: group 32 * lane .. 32 * lane + 31 (lanes past
        // the row's groups hold none)
        uint32_t cnt[32];
        uint32_t mx = 0;
#pragma unroll
        for (int u = 0; u < 32; u++) {
            const int t = 32 * lane + u;
            cnt[u] = (lane < kGroups && !bad) ? (counts[t >> 1] >> (16 * (t & 1))) & 0xFFFFu : 0u;
            mx = cnt[u] > mx ? cnt[u] : mx;
        }
        mx = __reduce_max_sync(kFull, mx);
        const int cls = mx <= 3u ? 0 : (mx <= 15u ? 1 : (mx <= 255u ? 2 : 3));
        int slot = 0;
        if (lane == 0) slot = atomicAdd(&sc.class_count[cls], 1);
        slot = __shfl_sync(kFull, slot, 0);
        const int nD = class_digits(cls), nR = class_reads(cls);
        const int tile = slot / nR, n = slot % nR;
        uint8_t* tile_rows = sc.rows[cls] + (size_t)tile * G::kBBytes;
        for (int d = 0; d < nD; d++) {
            // word s of the group: token 32 * lane + 4j + s in nibble j
            uint4 packed = make_uint4(0, 0, 0, 0);
            uint32_t* pw = reinterpret_cast<uint32_t*>(&packed);
#pragma unroll
            for (int u = 0; u < 32; u++)
                pw[u & 3] |= e2m1_digit(u & 3, (cnt[u] >> (2 * d)) & 3u) << (4 * (u >> 2));
            if (lane < kGroups)
                *reinterpret_cast<uint4*>(tile_rows + (size_t)(d * nR + n) * G::kKBytes + 16 * lane) = packed;
        }
        if (lane == 0) {
            const int n_tok = L - Q + 1 > 0 ? L - Q + 1 : 0;
            sc.T[cls][slot] = bad ? 0x7fffffff : n_tok - Q * (int)E[r];
            sc.rid[cls][slot] = (uint32_t)r;
        }
        __syncwarp();
        for (int i = lane; i < kCountWords; i += 32) counts[i] = 0;
        __syncwarp();
    }
    flags = __reduce_or_sync(kFull, flags);
    if (lane == 0 && flags) atomicOr(status, flags);
}

// ------------------------------------------------------------ scan kernel

template <int Q>
struct ScanSmem {
    using G = ScanGeo<Q>;
    static constexpr size_t kB = 0;                                     // 1024-aligned
    static constexpr size_t kBank = kB + G::kBBytes;                    // 1024-aligned
    static constexpr size_t kT = kBank + (size_t)kBankStages * G::kBankTileBytes;
    static constexpr size_t kTf = kT + 4 * kRowsTile;
    static constexpr size_t kRid = kTf + 4 * kRowsTile;
    static constexpr size_t kBars = kRid + 4 * kRowsTile;
    static constexpr size_t kMisc = kBars + 8 * (2 * kBankStages + 2 * kAStages + 5);
    static constexpr size_t kTotal = kMisc + 64;
    static constexpr size_t kAlloc = kTotal + 1024;  // slack to align the base
};

struct ScanParams {
    const uint32_t* bank;
    int64_t n_bins;
    int64_t bin_begin, bin_end;
    int64_t btiles_per_item;
    ScanScratch sc;
    ScanOut out;
    uint32_t* status;
};

// Appends the passing (read, bin) pairs of one group of reads: sums[i] is
// the sum of read n0 + i for this thread's bin.  Rare path.
template <int NG>
__device__ __forceinline__ void scan_emit(const ScanParams& P, const int* sums, int n0, int valid_reads,
                                          const int32_t* __restrict__ sT, const uint32_t* __restrict__ sRid,
                                          int64_t b, bool bin_ok, int lane) {
    for (int i = 0; i < NG && n0 + i < valid_reads; i++) {
        const int n = n0 + i;
        const int sum = sums[i];
        const bool p = bin_ok && sum >= sT[n];
        const uint32_t bal = __ballot_sync(kFull, p);
        if (!bal) continue;
        const int leader = __ffs(bal) - 1;
        unsigned long long base = 0;
        if (lane == leader) {
            base = atomicAdd(P.out.n_pairs, (unsigned long long)__popc(bal));
            if (P.out.read_pass) atomicAdd(&P.out.read_pass[sRid[n]], (uint32_t)__popc(bal));
        }
        base = __shfl_sync(kFull, base, leader);
        if (p) {
            const unsigned long long idx = base + __popc(bal & ((1u << lane) - 1u));
            if ((long long)idx < P.out.cap) {
                P.out.pair_read[idx] = sRid[n];
                P.out.pair_bin[idx] = (uint32_t)b;
                if (P.out.pair_sum) P.out.pair_sum[idx] = (uint16_t)sum;
            } else {
                atomicOr(P.status, GRIM_FLAG_OVERFLOW);
            }
        }
    }
}

// Epilogue of one work item for reads with D base-4 digits (N = 256 / D
// reads per tile): thread = bin row = TMEM lane of its warp's quadrant; the
// warp takes the GR = 64 / D reads from quarter * N/4, i.e. 64 accumulator
// columns.  Column d*N + n holds the digit-d sum of read n (an exact
// integer in f32); Sum = sum_d 4^d * column d*N + n.  The accumulator is
// handed back as soon as the columns are in registers.
template <int D>
__device__ __forceinline__ void scan_epilogue(const ScanParams& P, uint32_t tmem, uint64_t* acc_full,
                                              uint64_t* acc_empty, volatile int* abort_flag,
                                              const int32_t* __restrict__ sT, const float* __restrict__ sTf,
                                              const uint32_t* __restrict__ sRid, int valid_reads, int64_t bt0,
                                              int64_t bt1, uint32_t& acc_cnt) {
    constexpr int N = kRowsTile / D;
    constexpr int GR = 64 / D;  // reads of this warp: 64, 32, 16, 8
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quad = warp & 3;
    const int quarter = (warp - kEpilogueWarp0) >> 2;
    const int m = quad * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    const uint32_t col0 = tmem + lane_base + kAccCol;
    const int n0 = quarter * GR;  // first read of this warp
    for (int64_t bt = bt0; bt < bt1; bt++) {
        const uint32_t phb = acc_cnt & 1;
        if (!mbar_wait_warp(acc_full, phb, abort_flag)) break;
        tc_fence_after();
        const int64_t b = P.bin_begin + bt * kBinTile + m;
        const bool bin_ok = b < P.bin_end;
        uint32_t v[64];
#pragma unroll
        for (int d = 0; d < D; d++) tmem_ld<GR>(col0 + d * N + n0, v + d * GR);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty);
        if (D == 1) {
            // one digit: the accumulator is the sum; compare it with T in f32
            uint32_t any = 0;
            const float4* t4 = reinterpret_cast<const float4*>(sTf + n0);
#pragma unroll
            for (int i = 0; i < GR / 4; i++) {
                const float4 t = t4[i];  // four thresholds in one shared load
                any |= (uint32_t)(__uint_as_float(v[4 * i]) >= t.x) |
                       (uint32_t)(__uint_as_float(v[4 * i + 1]) >= t.y) |
                       (uint32_t)(__uint_as_float(v[4 * i + 2]) >= t.z) |
                       (uint32_t)(__uint_as_float(v[4 * i + 3]) >= t.w);
            }
            if (__any_sync(kFull, bin_ok && any)) {
                int sums[GR];
#pragma unroll
                for (int i = 0; i < GR; i++) sums[i] = (int)__uint_as_float(v[i]);
                scan_emit<GR>(P, sums, n0, valid_reads, sT, sRid, b, bin_ok, lane);
            }
        } else {
            int acc[GR];
#pragma unroll
            for (int i = 0; i < GR; i++) {
                acc[i] = 0;
#pragma unroll
                for (int d = 0; d < D; d++) acc[i] += (int)__uint_as_float(v[d * GR + i]) << (2 * d);
            }
            uint32_t any = 0;
            const int4* t4 = reinterpret_cast<const int4*>(sT + n0);
#pragma unroll
            for (int i = 0; i < GR / 4; i++) {
                const int4 t = t4[i];
                any |= (uint32_t)(acc[4 * i] >= t.x) | (uint32_t)(acc[4 * i + 1] >= t.y) |
                       (uint32_t)(acc[4 * i + 2] >= t.z) | (uint32_t)(acc[4 * i + 3] >= t.w);
            }
            if (__any_sync(kFull, bin_ok && any)) scan_emit<GR>(P, acc, n0, valid_reads, sT, sRid, b, bin_ok, lane);
        }
        acc_cnt++;
    }
}

template <int Q>
__global__ void __launch_bounds__(kScanThreads, 1) scan_kernel(const __grid_constant__ CUtensorMap tmap, ScanParams P) {
    using G = ScanGeo<Q>;
    using S = ScanSmem<Q>;
    extern __shared__ uint8_t scan_smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)scan_smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sB = smem + S::kB;
    uint8_t* sBank = smem + S::kBank;
    int32_t* sT = reinterpret_cast<int32_t*>(smem + S::kT);
    float* sTf = reinterpret_cast<float*>(smem + S::kTf);
    uint32_t* sRid = reinterpret_cast<uint32_t*>(smem + S::kRid);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::kBars);
    uint64_t* bank_full = bars;
    uint64_t* bank_empty = bars + kBankStages;
    uint64_t* a_full = bars + 2 * kBankStages;
    uint64_t* a_empty = a_full + kAStages;
    uint64_t* acc_full = a_empty + kAStages;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* drain_bar = acc_empty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + S::kMisc);
    volatile int* s_item = reinterpret_cast<volatile int*>(smem + S::kMisc + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + S::kMisc + 8);
    volatile int* s_cls = reinterpret_cast<volatile int*>(smem + S::kMisc + 12);
    volatile int* s_valid = reinterpret_cast<volatile int*>(smem + S::kMisc + 16);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kBankStages; i++) {
            mbar_init(&bank_full[i], 1);
            mbar_init(&bank_empty[i], 4);
        }
        for (int i = 0; i < kAStages; i++) {
            mbar_init(&a_full[i], 4);
            mbar_init(&a_empty[i], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, kEpilogueWarps);
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (warp >= kEpilogueWarp0 && warp < kEpilogueWarp0 + 4) {
        // unit scale factors (ue8m0 127 = 1.0 in every byte) for A and B
        uint32_t v[32];
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = 0x7F7F7F7Fu;
        tmem_st32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + kSfCol, v);
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    // work decomposition: classes' tile counts come from the prep kernel
    int n_tiles[kNumClasses];
    int total_tiles = 0;
    for (int c = 0; c < kNumClasses; c++) {
        const int cnt = P.sc.class_count[c];
        n_tiles[c] = (cnt + class_reads(c) - 1) / class_reads(c);
        total_tiles += n_tiles[c];
    }
    const int64_t n_btiles = (P.bin_end - P.bin_begin + kBinTile - 1) / kBinTile;
    const int64_t n_chunks = (n_btiles + P.btiles_per_item - 1) / P.btiles_per_item;
    const int64_t n_items = (int64_t)total_tiles * n_chunks;
    constexpr uint32_t kIdesc = idesc_mxf4(kBinTile, kRowsTile);

    // running pipeline counters (each role uses its own)
    uint32_t bank_cnt = 0, a_cnt = 0, acc_cnt = 0;

    while (true) {
        if (threadIdx.x == 0) *s_item = atomicAdd(P.sc.work, 1);
        __syncthreads();
        const int64_t item = *s_item;
        if (item >= n_items || *abort_flag) break;
        const int64_t chunk = item / total_tiles;
        int tile = (int)(item % total_tiles);
        int cls = 0;
        while (cls < kNumClasses - 1 && tile >= n_tiles[cls]) tile -= n_tiles[cls++];
        const int nR = class_reads(cls);
        const int valid_reads = min(nR, P.sc.class_count[cls] - tile * nR);
        const int64_t bt0 = chunk * P.btiles_per_item;
        const int64_t bt1 = min(n_btiles, bt0 + P.btiles_per_item);

        // stage the read tile's digit rows (swizzled K-major), thresholds, read ids
        {
            const uint4* src = reinterpret_cast<const uint4*>(P.sc.rows[cls] + (size_t)tile * G::kBBytes);
            constexpr int kChunksPerRow = G::kKBytes / 16;
            for (int i = threadIdx.x; i < kRowsTile * kChunksPerRow; i += kScanThreads) {
                const int row = i / kChunksPerRow, j = i % kChunksPerRow;
                const int kb = j >> 3, cj = j & 7;
                uint4 v = __ldg(src + i);
                *reinterpret_cast<uint4*>(sB + kb * (kRowsTile * 128) + row * 128 + ((cj ^ (row & 7)) << 4)) = v;
            }
            for (int n = threadIdx.x; n < kRowsTile; n += kScanThreads) {
                sT[n] = n < valid_reads ? P.sc.T[cls][tile * nR + n] : 0x7fffffff;
                // T exactly in f32 (|T| < 2^24); "never passes" is +inf
                sTf[n] = sT[n] == 0x7fffffff ? __int_as_float(0x7f800000) : (float)sT[n];
                sRid[n] = n < valid_reads ? P.sc.rid[cls][tile * nR + n] : 0u;
            }
            if (threadIdx.x == 0) {
                *s_cls = cls;
                *s_valid = valid_reads;
            }
            fence_proxy_async_smem();
        }
        __syncthreads();

        if (warp == 0) {
            // ---- TMA producer: bank tiles into the ring
            if (lane == 0) {
                for (int64_t bt = bt0; bt < bt1; bt++) {
                    const uint32_t s = bank_cnt % kBankStages, ph = (bank_cnt / kBankStages) & 1;
                    if (!mbar_wait(&bank_empty[s], ph ^ 1, abort_flag)) break;
                    const int64_t b0 = P.bin_begin + bt * kBinTile;
                    // the whole box arrives; rows past the bank read as zeros
                    mbar_arrive_expect_tx(&bank_full[s], (uint32_t)G::kBankTileBytes);
                    tma_load_2d(sBank + (size_t)s * G::kBankTileBytes, &tmap, 0, (int)b0, &bank_full[s]);
                    bank_cnt++;
                }
            }
        } else if (warp == 1) {
            // ---- MMA issuer
            if (lane == 0) {
                for (int64_t bt = bt0; bt < bt1; bt++) {
                    const uint32_t phb = acc_cnt & 1;
                    if (!mbar_wait(acc_empty, phb ^ 1, abort_flag)) break;
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + kAccCol;
                    bool ok = true;
                    for (int c = 0; c < G::kChunks; c++) {
                        const uint32_t sa = a_cnt % kAStages, pha = (a_cnt / kAStages) & 1;
                        if (!mbar_wait(&a_full[sa], pha, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
#pragma unroll
                        for (int kk = 0; kk < G::kMmaPerChunk; kk++) {
                            const uint32_t a_tmem = tmem + kACol + sa * G::kACols + kk * 8;
                            const int kg = c * G::kMmaPerChunk + kk;  // MMA index within the row
                            const int kb = kg >> 2;                   // 128-byte K block of B (4 MMAs)
                            const uint64_t bdesc =
                                smem_desc_sw128(smem_addr(sB) + kb * (kRowsTile * 128) + (kg & 3) * 32);
                            mma_mxf4_tmemA(d_tmem, a_tmem, bdesc, kIdesc, tmem + kSfCol, tmem + kSfCol,
                                           (c | kk) != 0);
                        }
                        mma_commit(&a_empty[sa]);
                        a_cnt++;
                    }
                    if (!ok) break;
                    mma_commit(acc_full);
                    acc_cnt++;
                }
            }
        } else if (warp < kEpilogueWarp0) {
            // ---- expanders: thread = bin row = TMEM lane
            const int quad = warp & 3;
            const int m = quad * 32 + lane;
            const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
            for (int64_t bt = bt0; bt < bt1; bt++) {
                const uint32_t s = bank_cnt % kBankStages, ph = (bank_cnt / kBankStages) & 1;
                if (!mbar_wait_warp(&bank_full[s], ph, abort_flag)) break;
                const int64_t b0 = P.bin_begin + bt * kBinTile;
                const int rows = (int)((P.bin_end - b0) < kBinTile ? (P.bin_end - b0) : (int64_t)kBinTile);
                const uint32_t tile_off = (uint32_t)s * G::kBankTileBytes + (uint32_t)m * G::kRowBytes;
                bool ok = true;
                for (int c = 0; c < G::kChunks; c++, a_cnt++) {
                    const uint32_t sa = a_cnt % kAStages, pha = (a_cnt / kAStages) & 1;
                    // this stage's bank words (rows shorter than the padded K read as 0)
                    constexpr int kVec = G::kWordsPerChunk / 4;
                    uint4 bits[kVec];
#pragma unroll
                    for (int u = 0; u < kVec; u++) {
                        const int wv = c * kVec + u;  // 16-byte vector of the row
                        const uint32_t a = tile_off + 16u * wv;  // unswizzled offset, then the TMA's pattern
                        const uint32_t off = a ^ (((a >> 7) & G::kSwzMask) << 4);
                        bits[u] = (m < rows && 4 * wv < G::kRowWords) ? *reinterpret_cast<const uint4*>(sBank + off)
                                                                      : make_uint4(0, 0, 0, 0);
                    }
                    if (!mbar_wait_warp(&a_empty[sa], pha ^ 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int u = 0; u < kVec; u += 2) {
                        // 8 bank words -> 32 columns (4 per word)
                        uint32_t v[32];
                        expand_word_fp4(bits[u].x, v);
                        expand_word_fp4(bits[u].y, v + 4);
                        expand_word_fp4(bits[u].z, v + 8);
                        expand_word_fp4(bits[u].w, v + 12);
                        expand_word_fp4(bits[u + 1].x, v + 16);
                        expand_word_fp4(bits[u + 1].y, v + 20);
                        expand_word_fp4(bits[u + 1].z, v + 24);
                        expand_word_fp4(bits[u + 1].w, v + 28);
                        tmem_st32(tmem + lane_base + kACol + sa * G::kACols + u * 16, v);
                    }
                    tmem_wait_st();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&a_full[sa]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&bank_empty[s]);
                bank_cnt++;
                if (!ok) break;
            }
        } else {
            // ---- epilogue: thread = bin row = TMEM lane
            const int cls_now = *s_cls;
            if (cls_now == 0)
                scan_epilogue<1>(P, tmem, acc_full, acc_empty, abort_flag, sT, sTf, sRid, *s_valid, bt0, bt1,
                                 acc_cnt);
            else if (cls_now == 1)
                scan_epilogue<2>(P, tmem, acc_full, acc_empty, abort_flag, sT, sTf, sRid, *s_valid, bt0, bt1,
                                 acc_cnt);
            else if (cls_now == 2)
                scan_epilogue<4>(P, tmem, acc_full, acc_empty, abort_flag, sT, sTf, sRid, *s_valid, bt0, bt1,
                                 acc_cnt);
            else
                scan_epilogue<8>(P, tmem, acc_full, acc_empty, abort_flag, sT, sTf, sRid, *s_valid, bt0, bt1,
                                 acc_cnt);
        }
        __syncthreads();  // the item is drained before B is overwritten
    }

    // drain: no bulk copy or MMA may still target this CTA's memory
    __syncthreads();
    if (*abort_flag) {
        if (threadIdx.x == 0) {
            atomicOr(P.status, GRIM_FLAG_TIMEOUT);
            // the newest copy issued into each ring stage (older ones completed before it was issued)
            for (uint32_t g = bank_cnt > kBankStages ? bank_cnt - kBankStages : 0; g < bank_cnt; g++) {
                const unsigned long long t0 = now_ns();
                while (!mbar_try_wait(&bank_full[g % kBankStages], (g / kBankStages) & 1) &&
                       now_ns() - t0 < kWaitLimitNs) {
                }
            }
        }
        if (threadIdx.x == 32) {  // every MMA this thread issued has finished once drain_bar completes
            mma_commit(drain_bar);
            const unsigned long long t0 = now_ns();
            while (!mbar_try_wait(drain_bar, 0) && now_ns() - t0 < kWaitLimitNs) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ------------------------------------------------------------ host launch

// cuTensorMapEncodeTiled, looked up once through the runtime.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// The bank as a 2-D tensor of n_bins rows x row bytes, read in boxes of
// 128 rows, swizzled as ScanGeo::kSwzMask describes.
template <int Q>
static int bank_tensor_map(const grim_bank* bank, CUtensorMap* map) {
    using G = ScanGeo<Q>;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return GRIM_ENOTSUP;
    const cuuint64_t dims[2] = {(cuuint64_t)G::kRowBytes, (cuuint64_t)bank->n_bins};
    const cuuint64_t strides[1] = {(cuuint64_t)G::kRowBytes};
    const cuuint32_t box[2] = {(cuuint32_t)G::kRowBytes, (cuuint32_t)kBinTile};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle swz = G::kSwzMask == 7u ? CU_TENSOR_MAP_SWIZZLE_128B
                                   : G::kSwzMask == 1u ? CU_TENSOR_MAP_SWIZZLE_32B
                                                       : CU_TENSOR_MAP_SWIZZLE_NONE;
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)bank->bits, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GRIM_OK : GRIM_ECUDA;
}

template <int Q>
static int launch_scan_q(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                         const uint16_t* E, int64_t bin_begin, int64_t bin_end, const ScanOut& out, void* scratch,
                         cudaStream_t s) {
    using G = ScanGeo<Q>;
    // scratch layout (see scan_scratch_bytes)
    uint8_t* p = (uint8_t*)scratch;
    ScanScratch sc;
    sc.class_count = (int32_t*)p;
    sc.work = (int32_t*)(p + 16);
    p += 256;
    for (int c = 0; c < kNumClasses; c++) {
        const int64_t tiles = (n_reads + class_reads(c) - 1) / class_reads(c);
        sc.rows[c] = p;
        p += (size_t)tiles * G::kBBytes;
        sc.T[c] = (int32_t*)p;
        p += ((size_t)tiles * class_reads(c) * 4 + 255) & ~(size_t)255;
        sc.rid[c] = (uint32_t*)p;
        p += ((size_t)tiles * class_reads(c) * 4 + 255) & ~(size_t)255;
    }
    GRIM_CUDA_TRY(cudaMemsetAsync(scratch, 0, 256, s));
    GRIM_CUDA_TRY(cudaMemsetAsync(out.n_pairs, 0, sizeof(unsigned long long), s));
    if (out.read_pass) GRIM_CUDA_TRY(cudaMemsetAsync(out.read_pass, 0, (size_t)n_reads * 4, s));

    {
        constexpr size_t smem = 4 * ((size_t)TokenTable<Q>::kWords + (size_t)kPrepWarps * ((G::kK + 1) / 2));
        const int64_t need = (n_reads + kPrepWarps - 1) / kPrepWarps;
        const int64_t cap = (int64_t)sm_count() * 16;
        const int64_t blocks = need < cap ? need : cap;
        scan_prep_kernel<Q><<<grim::fault_grid((unsigned)blocks), kPrepWarps * 32, smem, s>>>(
                reads, read_offsets, n_reads, E, sc, bank->status);
        GRIM_CUDA_TRY(cudaGetLastError());
    }
    {
        constexpr size_t smem = ScanSmem<Q>::kAlloc;
        static DeviceCache attr[64];  // per device
        const int slot = device_slot();
        if (slot < 0) return GRIM_ENOTSUP;
        if (!attr[slot].load()) {
            GRIM_CUDA_TRY(cudaFuncSetAttribute(scan_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr[slot].store(1);
        }
        ScanParams P;
        P.bank = bank->bits;
        P.n_bins = bank->n_bins;
        P.bin_begin = bin_begin;
        P.bin_end = bin_end;
        const int64_t n_btiles = (bin_end - bin_begin + kBinTile - 1) / kBinTile;
        const int64_t read_tiles = (n_reads + kRowsTile - 1) / kRowsTile;
        const int64_t want_items = 4LL * sm_count();
        int64_t per = (n_btiles * read_tiles + want_items - 1) / want_items;
        per = per < 1 ? 1 : (per > 1024 ? 1024 : per);
        P.btiles_per_item = per;
        P.sc = sc;
        P.out = out;
        P.status = bank->status;
        if (bin_end > (int64_t)0x7fffffff) return GRIM_ENOTSUP;  // TMA row coordinates are 32-bit
        CUtensorMap tmap;
        const int rc = bank_tensor_map<Q>(bank, &tmap);
        if (rc != GRIM_OK) return rc;
        scan_kernel<Q><<<grim::fault_grid(sm_count()), kScanThreads, smem, s>>>(tmap, P);
        GRIM_CUDA_TRY(cudaGetLastError());
    }
    return GRIM_OK;
}

}  // namespace grim

extern "C" const char* grim_scan_mma_kind(void) { return "mxf4"; }

namespace grim {

int scan_noalloc_scratch(void** ptr, size_t* bytes) {
    static std::mutex mu;
    static void* addr[64] = {nullptr};
    int dev = -1;
    GRIM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GRIM_ENOTSUP;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        GRIM_CUDA_TRY(cudaGetSymbolAddress(&p, g_scan_scratch));
        addr[dev] = p;
    }
    *ptr = addr[dev];
    *bytes = sizeof(g_scan_scratch);
    return GRIM_OK;
}

size_t scan_scratch_bytes(int q, int64_t n_reads) {
    const int64_t K = (int64_t(1) << (2 * q)) < 256 ? 256 : (int64_t(1) << (2 * q));  // e2m1: K / 2 bytes a row
    size_t total = 256;
    for (int c = 0; c < kNumClasses; c++) {
        const int64_t tiles = (n_reads + class_reads(c) - 1) / class_reads(c);
        total += (size_t)tiles * kRowsTile * (K / 2);
        total += 2 * (((size_t)tiles * class_reads(c) * 4 + 255) & ~(size_t)255);
    }
    return total;
}

int launch_scan(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                const uint16_t* E, int64_t bin_begin, int64_t bin_end, uint32_t* pair_read, uint32_t* pair_bin,
                uint16_t* pair_sum, int64_t cap, int64_t* n_pairs, uint32_t* read_pass, void* scratch,
                cudaStream_t s) {
    ScanOut out;
    out.pair_read = pair_read;
    out.pair_bin = pair_bin;
    out.pair_sum = pair_sum;
    out.cap = cap;
    out.n_pairs = reinterpret_cast<unsigned long long*>(n_pairs);
    out.read_pass = read_pass;
    switch (bank->q) {
        case 1: return launch_scan_q<1>(bank, reads, read_offsets, n_reads, E, bin_begin, bin_end, out, scratch, s);
        case 2: return launch_scan_q<2>(bank, reads, read_offsets, n_reads, E, bin_begin, bin_end, out, scratch, s);
        case 3: return launch_scan_q<3>(bank, reads, read_offsets, n_reads, E, bin_begin, bin_end, out, scratch, s);
        case 4: return launch_scan_q<4>(bank, reads, read_offsets, n_reads, E, bin_begin, bin_end, out, scratch, s);
        case 5: return launch_scan_q<5>(bank, reads, read_offsets, n_reads, E, bin_begin, bin_end, out, scratch, s);
        default: return GRIM_ENOTSUP;
    }
}

int launch_wait_selfcheck(unsigned long long limit_ns, cudaStream_t s, uint32_t* timed_out) {
    if (limit_ns < 1000000ull || limit_ns > kWaitLimitNs) return GRIM_EINVAL;
    uint32_t* out = nullptr;
    GRIM_CUDA_TRY(scratch_alloc((void**)&out, 4, s));
    wait_selfcheck_kernel<<<1, 32, 0, s>>>(limit_ns, out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(timed_out, out, 4, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return GRIM_ECUDA;
    }
    return GRIM_OK;
}

}  // namespace grim
