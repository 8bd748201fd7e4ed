// Warp-level q-gram token rollers (Sec. 3.2 step 1: every token of the read).
//
// for_each_token (full-scan preparation): a warp reads a read 32 bases at a
// time; two ballots per 32 bases give the low and high bits of every base
// code; a funnel shift lines up the q bases starting at a lane's position;
// a table of 4^q entries (built once per CTA in shared memory) maps those 2q
// bits to the token value, first base most significant.
// for_each_token5 (gather): each lane packs 5 bases and takes the next 5 from
// its neighbour; its 5 tokens are shifts and masks of that 10-base window.
#pragma once

#include "grim_internal.cuh"

namespace grim {

template <int Q>
struct TokenTable {
    static constexpr int kEntries = 1 << (2 * Q);
    static constexpr int kWords = (kEntries * 2 + 15) / 16 * 4;  // u16 entries, 16-byte padded
};

// All threads of the CTA; follow with __syncthreads().
template <int Q>
__device__ __forceinline__ void build_token_table(uint16_t* tab) {
    for (int idx = threadIdx.x; idx < TokenTable<Q>::kEntries; idx += blockDim.x) {
        uint32_t tok = 0;
#pragma unroll
        for (int k = 0; k < Q; k++) {
            const uint32_t code = (((idx >> (Q + k)) & 1u) << 1) | ((idx >> k) & 1u);
            tok = (tok << 2) | code;
        }
        tab[idx] = (uint16_t)tok;
    }
}

// Calls f(token) on the lane that owns each token position i (i + Q <= L).
// Whole warp, L warp-uniform.  bad_base collects codes > 3 (then the tokens
// use the code's low two bits; the caller rejects the read).
template <int Q, typename F>
__device__ __forceinline__ void for_each_token(const uint8_t* __restrict__ rd, int L, int lane,
                                               const uint16_t* __restrict__ tab, uint32_t& bad_base, F&& f) {
    constexpr uint32_t kQMask = (1u << Q) - 1;
    for (int s0 = 0; s0 < L; s0 += 256) {
        uint32_t c[9];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const int i = s0 + 32 * k + lane;
            c[k] = (s0 + 32 * k < L && i < L) ? __ldg(rd + i) : 0u;
            bad_base |= (uint32_t)(c[k] > 3u);
        }
        uint32_t lo_c = __ballot_sync(kFull, c[0] & 1u), hi_c = __ballot_sync(kFull, c[0] & 2u);
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (s0 + 32 * k >= L) break;  // warp-uniform
            const uint32_t lo_n = __ballot_sync(kFull, c[k + 1] & 1u);
            const uint32_t hi_n = __ballot_sync(kFull, c[k + 1] & 2u);
            const int i = s0 + 32 * k + lane;
            if (i + Q <= L) {
                const uint32_t xl = __funnelshift_r(lo_c, lo_n, lane) & kQMask;
                const uint32_t xh = __funnelshift_r(hi_c, hi_n, lane) & kQMask;
                f((uint32_t)tab[(xh << Q) | xl]);
            }
            lo_c = lo_n;
            hi_c = hi_n;
        }
    }
}

// Calls f(token) on the lane that owns each token position i (i + Q <= L),
// lane l owning positions 160 b + 5 l .. 160 b + 5 l + 4 of block b: one
// block covers a read of up to 164 bases, with 5 token slots per lane.  Each
// lane packs its 5 bases, 2 bits each with the first base highest; one
// shuffle brings the next lane's 5 (lane 31 takes them from the next block,
// loaded one block ahead); the 20-bit window of 10 bases then holds the
// lane's 5 tokens, each a shift and a mask (Q <= 6).  Whole warp, L
// warp-uniform.  bad_base collects codes > 3 (the tokens then use the
// code's low two bits; the caller rejects the read).
template <int Q, typename F>
__device__ __forceinline__ void for_each_token5(const uint8_t* __restrict__ rd, int L, int lane, uint32_t& bad_base,
                                                F&& f) {
    static_assert(Q >= 1 && Q <= 6, "window of 10 bases");
    constexpr uint32_t kMask = (1u << (2 * Q)) - 1;
    auto pack = [&](int p0) -> uint32_t {
        uint32_t v = 0;
#pragma unroll
        for (int k = 0; k < 5; k++) {
            const int i = p0 + k;
            const uint32_t c = i < L ? (uint32_t)__ldg(rd + i) : 0u;
            bad_base |= (uint32_t)(c > 3u);
            v = (v << 2) | (c & 3u);
        }
        return v;
    };
    if (L <= 0) return;
    uint32_t cur = pack(5 * lane);
    for (int b0 = 0; b0 < L; b0 += 160) {
        const uint32_t nxt = b0 + 160 < L ? pack(b0 + 160 + 5 * lane) : 0u;  // warp-uniform condition
        const uint32_t nb = __shfl_sync(kFull, lane == 0 ? nxt : cur, (lane + 1) & 31);
        const uint32_t w = (cur << 10) | nb;  // bases p .. p + 9 of the read, p = b0 + 5 lane
        const int p = b0 + 5 * lane;
#pragma unroll
        for (int k = 0; k < 5; k++)
            if (p + k + Q <= L) f((w >> (2 * (10 - k - Q))) & kMask);
        cur = nxt;
    }
}

}  // namespace grim
