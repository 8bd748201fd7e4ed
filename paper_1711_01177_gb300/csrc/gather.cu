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
// One warp per read (warps claim reads; the launch at the end of the file):
//   0. the first candidate rows are requested before anything else, so
//      their latency hides behind the token work;
//   1. each lane packs 5 consecutive bases of a 160-base block (2 bits per
//      base, first base highest), a shuffle brings it the next 5, and its
//      5 tokens are shifts and masks of that 10-base window (the q-gram
//      window of Sec. 3.2 step 1);
//   2. each token is counted in a byte counter in shared memory (one
//      atomic add), and the count planes are cut out of the counters with
//      masks and shifts; for q = 6 and for reads of more than 255 tokens it
//      is added to the bit-sliced planes by a carry chain of atomicXor;
//   3. every lane keeps its slice of the planes in registers (reads with up
//      to three planes, two for q = 6) or reads it from shared memory (more
//      planes);
//   4. candidate rows stream through the warp as 16-byte vectors,
//      lanes_per_row lanes per row (4 lanes x 32 bytes for q=5: 8 rows per
//      warp step); each row is requested one step (q <= 5, with 4 CTAs of
//      64 registers per SM) or three steps (q = 6) before it is scored,
//      its id taken from a prefetched window of 32 candidate ids; rows are
//      ANDed with the planes and popcounted, and the lanes' shares of the
//      window's 32 rows are combined by shuffles as the steps finish
//      (steps 3-4);
//   5. every lane then holds one whole sum of the window, compares it with
//      the threshold and stores its pass byte (and sum): 32 bytes of one
//      window land together (step 5).
#include "grim_internal.cuh"
#include "tokens.cuh"

namespace grim {

constexpr int kGatherWarps = 8;
constexpr int kPlanes = 16;  // sums and counts stay below 2^16

template <int Q>
struct GatherGeo {
    static constexpr int kRowWords = Geo<Q>::kRowWords;
    static constexpr int kRowVecs = kRowWords / 4;             // 16-byte vectors per row
    static constexpr int kVPL = kRowWords >= 32 ? 2 : 1;        // vectors per lane per row
    static constexpr int kLPB = kRowVecs / kVPL;               // lanes per row
    static constexpr int kBPS = 32 / kLPB;                     // rows per warp step
    static constexpr int kPlaneWords = kPlanes * kRowWords;    // per warp
    static_assert(kLPB >= 1 && kLPB <= 32 && 32 % kBPS == 0, "bad gather geometry");
};

template <int Q>
constexpr size_t gather_smem_bytes(int warps = kGatherWarps) {
    return 4 * (size_t)warps * GatherGeo<Q>::kPlaneWords;
}

__device__ __forceinline__ uint32_t and_popc(const uint4& a, const uint4& b) {
    return __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
}

// Carry-save adder over words: bitwise, a + b + c = lo + 2 hi.
__device__ __forceinline__ void csa(uint32_t& hi, uint32_t& lo, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    hi = (a & b) | (u & c);
    lo = u ^ c;
}

// popcount(x AND p0) + 2 popcount(x AND p1) over a lane's 8 words (two
// 16-byte vectors), p1 only when NP == 2.  Full adders first reduce words
// of equal weight (Harley-Seal), so 6 popcounts (4 for one plane) replace
// 16 (8): for rows of 512 bytes the popcount pipe's latency, not issue
// slots, limits the gather.
template <int NP>
__device__ __forceinline__ uint32_t row_sum_csa(const uint4 (&v)[2], const uint4 (&p)[NP][2]) {
    const uint32_t a0 = v[0].x & p[0][0].x, a1 = v[0].y & p[0][0].y, a2 = v[0].z & p[0][0].z,
                   a3 = v[0].w & p[0][0].w, a4 = v[1].x & p[0][1].x, a5 = v[1].y & p[0][1].y,
                   a6 = v[1].z & p[0][1].z, a7 = v[1].w & p[0][1].w;
    uint32_t c1, s1, c2, s2, c3, s3;
    csa(c1, s1, a0, a1, a2);
    csa(c2, s2, a3, a4, a5);
    csa(c3, s3, s1, s2, a6);
    if constexpr (NP == 1) {
        uint32_t d1, s4;
        csa(d1, s4, c1, c2, c3);
        return __popc(s3) + __popc(a7) + 2 * __popc(s4) + 4 * __popc(d1);
    } else {
        const uint32_t b0 = v[0].x & p[1][0].x, b1 = v[0].y & p[1][0].y, b2 = v[0].z & p[1][0].z,
                       b3 = v[0].w & p[1][0].w, b4 = v[1].x & p[1][1].x, b5 = v[1].y & p[1][1].y,
                       b6 = v[1].z & p[1][1].z, b7 = v[1].w & p[1][1].w;
        // weight 2: c1 c2 c3 b0..b7
        uint32_t d1, s4, d2, s5, d3, s6, d4, s7, d5, s8;
        csa(d1, s4, c1, c2, c3);
        csa(d2, s5, b0, b1, b2);
        csa(d3, s6, b3, b4, b5);
        csa(d4, s7, s4, s5, s6);
        csa(d5, s8, s7, b6, b7);
        // weight 4: d1..d5
        uint32_t e1, s9, e2, s10;
        csa(e1, s9, d1, d2, d3);
        csa(e2, s10, s9, d4, d5);
        return __popc(s3) + __popc(a7) + 2 * __popc(s8) + 4 * __popc(s10) + 8 * (__popc(e1) + __popc(e2));
    }
}

// The candidate stream of one read.  Step k scores rows k*BPS .. k*BPS+BPS-1
// (lane group g = lane / LPB takes row k*BPS + g).  Candidate ids arrive in
// windows of 32 (one per lane, the next window prefetched); rows are
// requested kAhead steps before they are scored, into kBufs rotating
// register buffers.  A past-the-end or out-of-range id fetches row 0, which
// is scored but never stored.
template <int Q, bool DEEP>
struct Stream {
    using G = GatherGeo<Q>;
    static constexpr int kWinSteps = 32 / G::kBPS;       // steps per id window
    // row buffers (a divisor of kWinSteps): two for q <= 5 with the bank in
    // L2, whose smaller register budget lets 4 CTAs share an SM; four for
    // q = 6 and for banks read from HBM (DEEP: three steps of rows in flight
    // per warp cover the longer latency)
    static constexpr int kBufs =
        (Q <= 5 && !DEEP && kWinSteps >= 2) ? 2 : (kWinSteps >= 4 ? 4 : kWinSteps);
    static constexpr int kAhead = kBufs - 1;                      // steps a row is requested early
    // q = 6: rows are also prefetched into L2 this many steps ahead (within
    // the two id windows held), which covers more of the DRAM latency than
    // the register buffers alone
    static constexpr int kPrefetch = Q >= 6 ? 8 : 0;
    static_assert(kPrefetch < kWinSteps, "a prefetched id must lie in the next window at most");
    static_assert(kWinSteps % kBufs == 0, "buffer rotation must repeat every window");
    uint32_t win_cur, win_next;  // candidate ids c = base + lane, base + 32 + lane
    uint4 r[kBufs][G::kVPL];
};

__device__ __forceinline__ uint32_t window_id(const uint32_t* __restrict__ cands, int c, int n) {
    return c < n ? __ldg(cands + c) : 0xFFFFFFFFu;
}

// Asks the L2 for the 128-byte lines of a row that will be scored later
// (no register holds it meanwhile): lane s of the row group covers the
// lines holding its vectors when s is a multiple of 8 (8 x 16 bytes).
template <int Q>
__device__ __forceinline__ void prefetch_row(uint32_t id, const uint32_t* __restrict__ bank, uint32_t n_bins32,
                                             int s) {
    using G = GatherGeo<Q>;
    // past the read's end (or an invalid id) there is nothing to fetch; a
    // stand-in row would send every warp's requests to the same lines
    if ((s & 7) != 0 || id >= n_bins32) return;
    const uint4* row = reinterpret_cast<const uint4*>(bank) + (size_t)id * G::kRowVecs + s;
#pragma unroll
    for (int u = 0; u < G::kVPL; u++) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + u * G::kLPB));
}

template <int Q>
__device__ __forceinline__ void fetch_row(uint4 (&r)[GatherGeo<Q>::kVPL], uint32_t id,
                                          const uint32_t* __restrict__ bank, uint32_t n_bins32, int s) {
    using G = GatherGeo<Q>;
    const uint32_t b = id < n_bins32 ? id : 0u;
    const uint4* row = reinterpret_cast<const uint4*>(bank) + (size_t)b * G::kRowVecs + s;
#pragma unroll
    for (int u = 0; u < G::kVPL; u++) r[u] = __ldg(row + u * G::kLPB);
}

// Before the token work: the first two id windows and the first kAhead steps' rows.
template <int Q, bool DEEP>
__device__ __forceinline__ void stream_start(Stream<Q, DEEP>& st, const uint32_t* __restrict__ cands, int n,
                                             const uint32_t* __restrict__ bank, uint32_t n_bins32, int lane) {
    using G = GatherGeo<Q>;
    using S = Stream<Q, DEEP>;
    st.win_cur = window_id(cands, lane, n);
    st.win_next = window_id(cands, 32 + lane, n);
    const int s = lane % G::kLPB, g = lane / G::kLPB;
#pragma unroll
    for (int k = 0; k < S::kAhead; k++) {
        const int idx = k * G::kBPS + g;  // < 64: within the two windows
        const uint32_t id = __shfl_sync(kFull, idx < 32 ? st.win_cur : st.win_next, idx & 31);
        fetch_row<Q>(st.r[k], id, bank, n_bins32, s);
    }
}

// Partial sums of one id window: lane s of a row group holds, for every
// step t of the window, its share of row (t, g); the kLPB lanes of a group
// together hold the kLPB steps.  Steps are combined pairwise as they finish,
// like a binary counter: two step groups that differ in bit l of the step
// index meet across lane bit l, the lane with that bit clear keeping the
// lower group and the other the upper, each adding its partner's share.
// After the last step, lane s holds the whole sum of step s: one shuffle
// per step instead of log2(kLPB), and one row per lane to store.
template <int N>
struct StepReducer {
    static constexpr int kLevels = N >= 16 ? 4 : N >= 8 ? 3 : N >= 4 ? 2 : N >= 2 ? 1 : 0;
    static_assert((1 << kLevels) == N, "steps per window must be a power of two");
    uint32_t stk[kLevels > 0 ? kLevels : 1];
    uint32_t total = 0;
    // T: the step index (a constant once the window loop is unrolled)
    __device__ __forceinline__ void add(int T, uint32_t v, int s) {
#pragma unroll
        for (int l = 0; l < kLevels; l++) {
            if (((T >> l) & 1) == 0) {
                stk[l] = v;
                return;
            }
            const uint32_t lo = stk[l], hi = v;
            const bool upper = (s >> l) & 1;
            const uint32_t send = upper ? lo : hi;
            v = (upper ? hi : lo) + __shfl_xor_sync(kFull, send, 1 << l);
        }
        total = v;
    }
    // The same for a window run as passes of P unrolled steps: step
    // h * P + tl, tl a constant, h the pass (only the levels above log2 P
    // look at it, and only at a pass's last step).
    template <int P>
    __device__ __forceinline__ void add_split(int tl, int h, uint32_t v, int s) {
        constexpr int kPassLevels = P >= 16 ? 4 : P >= 8 ? 3 : P >= 4 ? 2 : P >= 2 ? 1 : 0;
#pragma unroll
        for (int l = 0; l < kLevels; l++) {
            const int bit = l < kPassLevels ? ((tl >> l) & 1) : ((h >> (l - kPassLevels)) & 1);
            if (bit == 0) {
                stk[l] = v;
                return;
            }
            const uint32_t lo = stk[l], hi = v;
            const bool upper = (s >> l) & 1;
            const uint32_t send = upper ? lo : hi;
            v = (upper ? hi : lo) + __shfl_xor_sync(kFull, send, 1 << l);
        }
        total = v;
    }
};

// Score the read's candidates.  NP > 0: NP planes held in registers;
// NP == 0: P planes read from shared memory.  cands / pass / sums point at
// the read's first candidate.
template <int Q, int NP, bool DEEP>
__device__ __forceinline__ void score_read(Stream<Q, DEEP>& st, const uint4* __restrict__ planes, int P, int T,
                                           int n, const uint32_t* __restrict__ cands,
                                           const uint32_t* __restrict__ bank, uint32_t n_bins32,
                                           uint8_t* __restrict__ pass, uint16_t* __restrict__ sums, int lane,
                                           uint32_t& flags) {
    using G = GatherGeo<Q>;
    using S = Stream<Q, DEEP>;
    const int s = lane % G::kLPB, g = lane / G::kLPB;
    uint4 pl[NP > 0 ? NP : 1][G::kVPL];
    if (NP > 0) {
#pragma unroll
        for (int p = 0; p < (NP > 0 ? NP : 1); p++)
#pragma unroll
            for (int u = 0; u < G::kVPL; u++) pl[p][u] = planes[p * G::kRowVecs + s + u * G::kLPB];
    }
    static_assert(S::kWinSteps == G::kLPB, "one step of the window per lane of a row group");
    for (int w0 = 0; w0 < n; w0 += 32) {
        const uint32_t win_after = window_id(cands, w0 + 64 + lane, n);  // two windows ahead
        StepReducer<S::kWinSteps> red;
        // 16-step windows (q = 6) run as two passes of one unrolled 8-step
        // body: half the code of the scoring loop, for the instruction cache
        constexpr int kPass = S::kWinSteps >= 16 ? 8 : S::kWinSteps;
        static_assert(kPass % S::kBufs == 0, "register buffers must rotate within a pass");
#pragma unroll 1
        for (int h = 0; h < S::kWinSteps / kPass; h++) {
#pragma unroll
        for (int tl = 0; tl < kPass; tl++) {
            const int t = h * kPass + tl;
            const int c0 = w0 + t * G::kBPS;
            uint32_t part = 0;
            if (c0 < n) {  // warp-uniform
                // request the rows kAhead steps ahead (window position t + kAhead)
                {
                    const int ahead = t + S::kAhead;
                    const int idx = (ahead % S::kWinSteps) * G::kBPS + g;
                    const uint32_t src = ahead < S::kWinSteps ? st.win_cur : st.win_next;
                    const uint32_t id = __shfl_sync(kFull, src, idx);
                    fetch_row<Q>(st.r[(tl + S::kAhead) % S::kBufs], id, bank, n_bins32, s);
                }
                if constexpr (S::kPrefetch > 0) {
                    const int ahead = t + S::kPrefetch;
                    const int idx = (ahead % S::kWinSteps) * G::kBPS + g;
                    const uint32_t src = ahead < S::kWinSteps ? st.win_cur : st.win_next;
                    const uint32_t id = __shfl_sync(kFull, src, idx);
                    prefetch_row<Q>(id, bank, n_bins32, s);
                }
                // score this step's rows
                const uint4 (&v)[G::kVPL] = st.r[tl % S::kBufs];
                if constexpr (NP > 0 && NP <= 2 && Q >= 6 && G::kVPL == 2) {
                    part = row_sum_csa<NP>(v, pl);
                } else if (NP > 0) {
#pragma unroll
                    for (int p = 0; p < (NP > 0 ? NP : 1); p++) {
                        uint32_t q = 0;
#pragma unroll
                        for (int u = 0; u < G::kVPL; u++) q += and_popc(v[u], pl[p][u]);
                        part += q << p;
                    }
                } else {
                    for (int p = 0; p < P; p++) {
                        uint32_t q = 0;
#pragma unroll
                        for (int u = 0; u < G::kVPL; u++)
                            q += and_popc(v[u], planes[p * G::kRowVecs + s + u * G::kLPB]);
                        part += q << p;
                    }
                }
            }
            if constexpr (kPass == S::kWinSteps) red.add(t, part, s);
            else red.template add_split<kPass>(tl, h, part, s);
        }
        }
        // this lane's row: step s, group g
        const int j = s * G::kBPS + g;
        const int c = w0 + j;
        const uint32_t id = __shfl_sync(kFull, st.win_cur, j);
        if (c < n) {
            const bool in_range = id < n_bins32;
            if (!in_range) flags |= GRIM_FLAG_BAD_BIN;
            const uint32_t sum = in_range ? red.total : 0u;
            pass[c] = (in_range && (int)sum >= T) ? 1 : 0;
            if (sums) sums[c] = (uint16_t)sum;
        }
        st.win_cur = st.win_next;
        st.win_next = win_after;
    }
}

// Outputs of a read whose sum is 0 for every candidate (no tokens, or a
// read rejected for bad data: then nothing passes).
__device__ __forceinline__ void write_constant(int64_t co, int64_t ce, const uint32_t* __restrict__ cand_bins,
                                               int64_t n_bins, bool pass0, uint8_t* __restrict__ pass,
                                               uint16_t* __restrict__ sums, int lane, uint32_t& flags) {
    for (int64_t c = co + lane; c < ce; c += 32) {
        const bool in_range = (int64_t)__ldg(cand_bins + c) < n_bins;
        if (!in_range) flags |= GRIM_FLAG_BAD_BIN;
        pass[c] = (in_range && pass0) ? 1 : 0;
        if (sums) sums[c] = 0;
    }
}

// Reads with at most 255 token positions (q <= 5) count their tokens in bytes: one
// shared atomic add per token, no carries.  The counters sit in the upper
// half of the warp's plane area (planes 8-15, which such reads never use)
// in a transposed order: the counter of token t is byte (t / 8) % 4 of
// counter word k = t % 8 of group w = t / 32, and word k of group w lies at
// 16-byte vector (k / 4) * RW + w, slot k % 4.  Bit 8 b + k of plane word w
// then is bit p of byte b of counter word k, so a plane word is eight
// masked shifts of the group's counter words, with no bit shuffling.
template <int Q>
__device__ __forceinline__ uint32_t counter_word(uint32_t tok) {
    constexpr uint32_t RW = GatherGeo<Q>::kRowWords;
    return 8 * RW + (tok & 4u) * RW + ((tok >> 5) << 2) + (tok & 3u);
}

// Count planes 0 .. used-1 from the byte counters of the warp's reads, which
// are zeroed on the way; returns used (the bit length of the largest count).
// Whole warp, after a __syncwarp that follows the counting.
template <int Q>
__device__ __forceinline__ int planes_from_counters(uint32_t* __restrict__ planes, int lane) {
    constexpr int RW = GatherGeo<Q>::kRowWords;
    uint4* cnt = reinterpret_cast<uint4*>(planes + 8 * RW);
    uint32_t any = 0;  // OR of every count: its bit length is the largest count's
    for (int w = lane; w < RW; w += 32) {
        const uint4 a = cnt[w], b = cnt[RW + w];
        any |= a.x | a.y | a.z | a.w | b.x | b.y | b.z | b.w;
    }
    any |= any >> 16;
    any |= any >> 8;
    const int used = 32 - __clz((int)__reduce_or_sync(kFull, any & 0xFFu));
    for (int w = lane; w < RW; w += 32) {
        const uint4 a = cnt[w], b = cnt[RW + w];
        cnt[w] = make_uint4(0u, 0u, 0u, 0u);
        cnt[RW + w] = make_uint4(0u, 0u, 0u, 0u);
        const uint32_t c[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int p = 0; p < 8; p++) {
            if (p >= used) break;  // warp-uniform
            uint32_t u = 0;
#pragma unroll
            for (int k = 0; k < 8; k++) u |= ((c[k] >> p) & 0x01010101u) << k;
            planes[p * RW + w] = u;
        }
    }
    return used;
}

// Shared-memory set-up of a gather CTA: zeroed count planes.
template <int Q>
__device__ __forceinline__ void gather_cta_setup(uint4* smem, int warps) {
    using G = GatherGeo<Q>;
    uint32_t* planes_all = reinterpret_cast<uint32_t*>(smem);
    for (int i = threadIdx.x; i < warps * G::kPlaneWords; i += blockDim.x) planes_all[i] = 0;
    __syncthreads();
}

// The whole filter for read r, by one warp (steps 0-5 above).  The warp's
// count planes are zero on entry and left zero on exit.
// ro, re: the read's bases; co, ce: its candidates; e: its edit budget.
template <int Q, bool DEEP>
__device__ __forceinline__ void gather_read(int64_t ro, int64_t re, int64_t co, int64_t ce, int e,
                                            const uint32_t* __restrict__ bank, int64_t n_bins,
                                            const uint8_t* __restrict__ reads,
                                            const uint32_t* __restrict__ cand_bins, uint8_t* __restrict__ pass,
                                            uint16_t* __restrict__ sums, uint32_t* __restrict__ planes, int lane,
                                            uint32_t& flags) {
    constexpr int RW = GatherGeo<Q>::kRowWords;
    const uint4* planes4 = reinterpret_cast<const uint4*>(planes);
    if (ce < co) {  // nothing sensible to write for this read
        flags |= GRIM_FLAG_BAD_OFFSETS;
        return;
    }
    // 0. the first candidate rows in flight while the tokens are built
    const uint32_t n_bins32 = (uint32_t)n_bins;  // n_bins < 2^32 (checked when the bank is built)
    const int n_c = (int)(ce - co);
    const uint32_t* cands = cand_bins + co;
    Stream<Q, DEEP> st;
    if (n_c > 0) stream_start<Q, DEEP>(st, cands, n_c, bank, n_bins32, lane);

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

    // 1-2. tokens into bit-sliced count planes
    uint32_t bad_base = 0;
    int used;
    const int n_tok = L - Q + 1 > 0 ? L - Q + 1 : 0;
    // byte counters, then the planes from them (q <= 5); for q = 6 the 4096
    // counters cost more to cut into planes than the carries they save
    if (Q <= 5 && n_tok <= 255) {
        for_each_token5<Q>(rd, L, lane, bad_base,
                           [&](uint32_t tok) { atomicAdd(&planes[counter_word<Q>(tok)], 1u << (tok & 0x18u)); });
        __syncwarp();
        used = planes_from_counters<Q>(planes, lane);
    } else {  // q = 6 and longer reads: a carry chain of atomicXor per token
        int top = -1;  // highest plane this lane set
        for_each_token5<Q>(rd, L, lane, bad_base, [&](uint32_t tok) {
            const uint32_t w = tok >> 5, m = 1u << (tok & 31);
            int p = 0;
            while (p < kPlanes) {
                const uint32_t old = atomicXor(&planes[p * RW + w], m);
                if (!(old & m)) break;
                ++p;
            }
            top = p > top ? p : top;
        });
        used = (int)__reduce_max_sync(kFull, (unsigned)(top + 1));
    }
    if (__any_sync(kFull, bad_base)) {
        flags |= GRIM_FLAG_BAD_BASE;
        bad_read = true;
    }
    __syncwarp();
    const int T = n_tok - Q * e;

    // 3-5. score the candidates
    if (co < ce) {
        if (bad_read || used == 0)
            write_constant(co, ce, cand_bins, n_bins, !bad_read && T <= 0, pass, sums, lane, flags);
        else if (used == 1)
            score_read<Q, 1, DEEP>(st, planes4, used, T, n_c, cands, bank, n_bins32, pass + co, sums ? sums + co : nullptr,
                             lane, flags);
        else if (used == 2)
            score_read<Q, 2, DEEP>(st, planes4, used, T, n_c, cands, bank, n_bins32, pass + co, sums ? sums + co : nullptr,
                             lane, flags);
        else if (Q <= 5 && used == 3)  // for q = 6 three planes stay in shared memory
            score_read<Q, 3, DEEP>(st, planes4, used, T, n_c, cands, bank, n_bins32, pass + co, sums ? sums + co : nullptr,
                             lane, flags);
        else
            score_read<Q, 0, DEEP>(st, planes4, used, T, n_c, cands, bank, n_bins32, pass + co, sums ? sums + co : nullptr,
                             lane, flags);
    }

    // leave the planes zeroed for the warp's next read
    __syncwarp();
    for (int i = lane; i < used * RW; i += 32) planes[i] = 0;
    __syncwarp();
}

// Modelled cost of the reads before r: 8 per candidate, 1 per base, 64 per
// read.  Strictly increasing in r for valid offsets, so equal cost shares
// are contiguous, disjoint read ranges that cover every read.
__device__ __forceinline__ int64_t cost_before(const int64_t* __restrict__ read_offsets,
                                               const int64_t* __restrict__ cand_offsets, int64_t r) {
    return 8 * (__ldg(cand_offsets + r) - __ldg(cand_offsets)) + (__ldg(read_offsets + r) - __ldg(read_offsets)) +
           64 * r;
}

// Smallest r in [0, n] with cost_before(r) >= target, found by a half-warp
// 16-ary search: lanes 0-15 search target0, lanes 16-31 target1.  Every
// lane returns its own half's answer.
__device__ int64_t split_search(const int64_t* __restrict__ read_offsets, const int64_t* __restrict__ cand_offsets,
                                int64_t n, int64_t target0, int64_t target1, int lane) {
    const int j = lane & 15;
    const int64_t target = lane < 16 ? target0 : target1;
    int64_t lo = 0, hi = n;  // the answer lies in [lo, hi]
    while (__any_sync(kFull, hi - lo > 16)) {
        const int64_t p = lo + (hi - lo) * (j + 1) / 17;  // sorted samples inside [lo, hi)
        const unsigned below = __ballot_sync(kFull, cost_before(read_offsets, cand_offsets, p) < target);
        const unsigned half = lane < 16 ? below & 0xFFFFu : below >> 16;
        const int k = __popc(half);  // the samples below target are a prefix
        const int64_t p_last = __shfl_sync(kFull, p, (lane & 16) + (k > 0 ? k - 1 : 0));
        const int64_t p_next = __shfl_sync(kFull, p, (lane & 16) + (k < 16 ? k : 15));
        if (k > 0) lo = p_last + 1;
        if (k < 16) hi = p_next;
        if (lo > hi) lo = hi;  // only with a non-monotone cost (invalid offsets)
    }
    const int64_t p = lo + j;
    const bool below = p < hi && cost_before(read_offsets, cand_offsets, p) < target;
    const unsigned b = __ballot_sync(kFull, below);
    return lo + __popc(lane < 16 ? b & 0xFFFFu : b >> 16);
}

// floor(total * i / n) without overflow, for 0 <= i <= n.
__device__ __forceinline__ int64_t cost_share(int64_t total, int64_t i, int64_t n) {
    return total / n * i + total % n * i / n;
}

// The gather launch: one wave of CTAs of WARPS warps whose warps claim
// `claim` reads at a time, in one of two ways.
//  - counter == nullptr: each CTA owns the contiguous read range of an equal
//    share of the modelled cost and claims from a shared-memory counter.  No
//    device state, so concurrent launches on different streams stay
//    independent (the one-launch filter).
//  - counter != nullptr: every warp claims from that zeroed device counter,
//    which also absorbs speed differences between SMs; the batched filter
//    resets it before each launch of its graph.
template <int Q, int WARPS, bool DEEP>
__global__ void __launch_bounds__(WARPS * 32, (Q >= 6 || DEEP ? 24 : 32) / WARPS)
gather_kernel(const uint32_t* __restrict__ bank, int64_t n_bins, const uint8_t* __restrict__ reads,
              const int64_t* __restrict__ read_offsets, int64_t n_reads, const uint32_t* __restrict__ cand_bins,
              const int64_t* __restrict__ cand_offsets, const uint16_t* __restrict__ E,
              uint8_t* __restrict__ pass, uint16_t* __restrict__ sums, uint32_t* __restrict__ status, int claim,
              unsigned long long* __restrict__ counter) {
    using G = GatherGeo<Q>;
    extern __shared__ uint4 gather_smem[];
    __shared__ unsigned long long next_read;
    __shared__ long long end_read;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (counter == nullptr && warp == 0) {
        const int64_t n_ctas = gridDim.x, b = blockIdx.x;
        const int64_t total = cost_before(read_offsets, cand_offsets, n_reads);
        const int64_t split = split_search(read_offsets, cand_offsets, n_reads, cost_share(total, b, n_ctas),
                                           cost_share(total, b + 1, n_ctas), lane);
        const int64_t r_begin = __shfl_sync(kFull, split, 0);
        const int64_t r_end = __shfl_sync(kFull, split, 16);
        // The ends are pinned so that every read lies in some CTA's range even
        // when decreasing (invalid) offsets break the monotone cost; such
        // reads are then flagged by whichever warp visits them.
        if (lane == 0) {
            next_read = b == 0 ? 0 : (unsigned long long)r_begin;
            end_read = b == n_ctas - 1 ? n_reads : r_end;
        }
    }
    gather_cta_setup<Q>(gather_smem, WARPS);  // ends with a CTA barrier
    uint32_t* planes = reinterpret_cast<uint32_t*>(gather_smem) + warp * G::kPlaneWords;
    const int64_t r_end = counter ? n_reads : end_read;
    unsigned long long* next = counter ? counter : &next_read;

    uint32_t flags = 0;
    while (true) {
        unsigned long long r0 = 0;
        if (lane == 0) r0 = atomicAdd(next, (unsigned long long)claim);
        r0 = __shfl_sync(kFull, r0, 0);
        if ((int64_t)r0 >= r_end) break;
        const int64_t r1 = (int64_t)r0 + claim < r_end ? (int64_t)r0 + claim : r_end;
        for (int64_t r = (int64_t)r0; r < r1; r++)
            gather_read<Q, DEEP>(read_offsets[r], read_offsets[r + 1], cand_offsets[r], cand_offsets[r + 1], E[r],
                                 bank, n_bins, reads, cand_bins, pass, sums, planes, lane, flags);
    }
    flags = __reduce_or_sync(kFull, flags);
    if (lane == 0 && flags) atomicOr(status, flags);
}

// Banks larger than this are read from HBM rather than L2: the gather then
// keeps three steps of rows in flight per warp (the DEEP form).
constexpr double kDeepBankBytes = 96e6;

// One launch over reads [r0, r0 + n) with `per_sm` CTAs per SM (0 = as many
// as fit).
template <int Q, int WARPS, bool DEEP>
static int launch_range(const grim_bank* bank, const GatherArgs& a, int64_t r0, int64_t n, int per_sm, int claim,
                        unsigned long long* counter, cudaStream_t s) {
    constexpr size_t smem = gather_smem_bytes<Q>(WARPS);
    static DeviceCache max_blocks_of[64];  // per device, like the attribute
    const int slot = device_slot();
    if (slot < 0) return GRIM_ENOTSUP;
    if (max_blocks_of[slot].load() == 0) {
        if (smem > 48 * 1024)
            GRIM_CUDA_TRY(cudaFuncSetAttribute(gather_kernel<Q, WARPS, DEEP>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int b = 0;
        GRIM_CUDA_TRY(
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gather_kernel<Q, WARPS, DEEP>, WARPS * 32, smem));
        max_blocks_of[slot].store(b > 0 ? b : 1);
    }
    const int max_blocks = max_blocks_of[slot].load();
    if (per_sm <= 0 || per_sm > max_blocks) per_sm = max_blocks;
    if (claim <= 0) claim = 1;
    int64_t blocks = (int64_t)sm_count() * per_sm;
    const int64_t need = (n + (int64_t)WARPS * claim - 1) / ((int64_t)WARPS * claim);  // a claim per warp at least
    if (need < blocks) blocks = need;
    if (counter) GRIM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    gather_kernel<Q, WARPS, DEEP><<<grim::fault_grid((unsigned)blocks), WARPS * 32, smem, s>>>(
        bank->bits, bank->n_bins, a.reads, a.read_offsets + r0, n, a.cand_bins, a.cand_offsets + r0, a.E + r0,
        a.pass, a.sums, bank->status, claim, counter);
    GRIM_CUDA_TRY(cudaGetLastError());
    return GRIM_OK;
}

template <int Q>
static int launch_batches(const grim_bank* bank, const GatherArgs& a, const grim_tune& t,
                          unsigned long long* counter, cudaStream_t s) {
    const int64_t batch = t.batch_reads > 0 ? t.batch_reads : a.n_reads;
    const bool deep = Q <= 5 && (double)bank->n_bins * (double)bank->row_words * 4.0 > kDeepBankBytes;
    constexpr bool kDeepForm = Q <= 5;  // q = 6 keeps its rows three steps ahead in either form
    for (int64_t r0 = 0; r0 < a.n_reads; r0 += batch) {
        const int64_t n = (a.n_reads - r0) < batch ? (a.n_reads - r0) : batch;
        const int pc = t.ctas_per_sm, rc_ = t.reads_per_claim;
        int rc;
        if (deep)
            rc = t.warps_per_cta == 4 ? launch_range<Q, 4, kDeepForm>(bank, a, r0, n, pc, rc_, counter, s)
                                      : launch_range<Q, 8, kDeepForm>(bank, a, r0, n, pc, rc_, counter, s);
        else
            rc = t.warps_per_cta == 4 ? launch_range<Q, 4, false>(bank, a, r0, n, pc, rc_, counter, s)
                                      : launch_range<Q, 8, false>(bank, a, r0, n, pc, rc_, counter, s);
        if (rc != GRIM_OK) return rc;
    }
    return GRIM_OK;
}

int launch_gather_batches(const grim_bank* bank, const GatherArgs& a, const grim_tune& t,
                          unsigned long long* counter, cudaStream_t s) {
    switch (bank->q) {
        case 1: return launch_batches<1>(bank, a, t, counter, s);
        case 2: return launch_batches<2>(bank, a, t, counter, s);
        case 3: return launch_batches<3>(bank, a, t, counter, s);
        case 4: return launch_batches<4>(bank, a, t, counter, s);
        case 5: return launch_batches<5>(bank, a, t, counter, s);
        case 6: return launch_batches<6>(bank, a, t, counter, s);
        default: return GRIM_ENOTSUP;
    }
}

int launch_gather(const grim_bank* bank, const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                  const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass,
                  uint16_t* sums, cudaStream_t s) {
    const GatherArgs a{reads, read_offsets, n_reads, cand_bins, cand_offsets, E, pass, sums};
    const grim_tune t = {kGatherWarps, 4, 0, 0, 0};  // one launch over every read, 4 reads per claim
    return launch_gather_batches(bank, a, t, nullptr, s);
}

}  // namespace grim
