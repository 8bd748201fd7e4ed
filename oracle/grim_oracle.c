/*
 * GRIM-Filter oracle: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of the seed-location filter of
 * Kim et al., "GRIM-Filter: Fast seed location filtering in DNA read mapping
 * using processing-in-memory technologies" (BMC Genomics 2018, arXiv
 * 1711.01177).  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * table with the CUDA library, and the CUDA library never calls it.
 *
 * Representation choices are deliberately naive: one byte per existence
 * bit, every token recomputed from its bases, every sum recounted from the
 * read's tokens, in the order the paper lists the steps.
 *
 * Conventions (readings of points the paper leaves open):
 *  - base codes A=0, C=1, G=2, T=3; a token's value is its bases read as a
 *    base-4 number, first base most significant (Sec. 3.1 only requires one
 *    bit per possible token; any bijection gives the same filter decisions);
 *  - 2-bit packed reference: base k in bits 2*(k%4) of byte k/4;
 *  - bin b covers the core [b*bin_len, (b+1)*bin_len) and is extended by
 *    `overlap` bases so that a read starting in the core fits (Sec. 3.1,
 *    Fig. 2a: overlapping bins); its span ends at
 *    min(len, b*bin_len + bin_len + overlap); a token belongs to the bin if
 *    all of its bases lie in the span;
 *  - threshold T = (L - q + 1) - q*E for E tolerated edits (Sec. 3.5: token
 *    count minus the worst case of q tokens lost per edit); E is an integer
 *    given per read; T may be <= 0, in which case every location passes;
 *  - a read shorter than q has no tokens and accumulation sum 0.
 *
 * Parity of every function here is pinned by tests/test_oracle_pins.py
 * against brute force, closed forms and the paper's worked examples.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_EDATA (-2)
#define ORACLE_ENOMEM (-3)

/* 2-bit packed reference -> one code per byte. */
void oracle_unpack_ref(const uint8_t* ref2bit, int64_t len, uint8_t* codes) {
    for (int64_t k = 0; k < len; k++) {
        uint8_t byte = ref2bit[k / 4];
        codes[k] = (uint8_t)((byte >> (2 * (k % 4))) & 3);
    }
}

/* Number of bins: ceil(len / bin_len) (Sec. 3.1: the genome is cut into
 * short contiguous bins). */
int64_t oracle_n_bins(int64_t len, int bin_len) {
    if (len <= 0 || bin_len <= 0) return 0;
    return (len + bin_len - 1) / bin_len;
}

/* Span [start, end) of bin b: its core plus the overlap (Sec. 3.1, Fig. 2a). */
void oracle_bin_span(int64_t b, int64_t len, int bin_len, int overlap, int64_t* start, int64_t* end) {
    int64_t s = b * (int64_t)bin_len;
    int64_t e = s + bin_len + overlap;
    if (e > len) e = len;
    *start = s;
    *end = e;
}

/* Token value of q bases (Sec. 3.1: 4^q possible tokens). */
int64_t oracle_token(const uint8_t* s, int q) {
    int64_t v = 0;
    for (int j = 0; j < q; j++) {
        int64_t weight = 1;
        for (int k = 0; k < q - 1 - j; k++) weight *= 4;
        v += (int64_t)s[j] * weight;
    }
    return v;
}

/* Accumulation-sum threshold (Sec. 3.5, Fig. 5a): the read has L-q+1 tokens;
 * each of the E tolerated edits may remove up to q of them. */
int64_t oracle_threshold(int64_t L, int q, int64_t E) {
    int64_t n_tokens = L - q + 1;
    if (n_tokens < 0) n_tokens = 0;
    return n_tokens - (int64_t)q * E;
}

/* Number of existence bits per bin: 4^q. */
int64_t oracle_bits_per_bin(int q) {
    int64_t n = 1;
    for (int k = 0; k < q; k++) n *= 4;
    return n;
}

/*
 * Build the existence bitvectors (Sec. 3.1): scan every bin's span and set
 * bit (b, token) for every token that occurs in it.  bank is
 * n_bins * 4^q bytes, byte b*4^q + t holds bit t of bin b (0 or 1).
 */
int oracle_build_bank(const uint8_t* ref2bit, int64_t len, int q, int bin_len, int overlap,
                      uint8_t* bank) {
    if (len <= 0 || q < 1 || q > 8 || bin_len <= 0 || overlap < 0) return ORACLE_EINVAL;
    int64_t n_bins = oracle_n_bins(len, bin_len);
    int64_t nbits = oracle_bits_per_bin(q);
    uint8_t* codes = (uint8_t*)malloc((size_t)len);
    if (!codes) return ORACLE_ENOMEM;
    oracle_unpack_ref(ref2bit, len, codes);
    memset(bank, 0, (size_t)(n_bins * nbits));
    for (int64_t b = 0; b < n_bins; b++) {
        int64_t s, e;
        oracle_bin_span(b, len, bin_len, overlap, &s, &e);
        for (int64_t i = s; i + q <= e; i++) {
            int64_t t = oracle_token(codes + i, q);
            bank[b * nbits + t] = 1;
        }
    }
    free(codes);
    return ORACLE_OK;
}

/*
 * The filter for one read and one bin (Sec. 3.2, Fig. 3): (1) take every
 * token of the read, (2) use the bin's bitvector, (3) look up each token's
 * existence bit, (4) add the bits up (a token occurring several times in the
 * read counts every time), (5) pass if the sum is >= the threshold.
 * Returns the accumulation sum; -1 if the read holds a code > 3.
 */
int64_t oracle_sum_one(const uint8_t* bank_row, int q, const uint8_t* read, int64_t L) {
    for (int64_t i = 0; i < L; i++)
        if (read[i] > 3) return -1;
    int64_t sum = 0;
    for (int64_t i = 0; i + q <= L; i++) {
        int64_t t = oracle_token(read + i, q);
        sum += bank_row[t];
    }
    return sum;
}

/*
 * Filter Bitmask Generator over a candidate list (Sec. 3.3): one output
 * per (read, candidate bin), 1 = align the location, 0 = discard.
 * sums (nullable) receives the accumulation sums.
 * Returns ORACLE_EDATA on a code > 3 or a bin id >= n_bins.
 */
int oracle_filter(const uint8_t* bank, int64_t n_bins, int q, const uint8_t* reads,
                  const int64_t* read_offsets, int64_t n_reads, const uint32_t* cand_bins,
                  const int64_t* cand_offsets, const uint16_t* E, uint8_t* pass, uint32_t* sums) {
    int64_t nbits = oracle_bits_per_bin(q);
    for (int64_t r = 0; r < n_reads; r++) {
        const uint8_t* read = reads + read_offsets[r];
        int64_t L = read_offsets[r + 1] - read_offsets[r];
        int64_t T = oracle_threshold(L, q, E[r]);
        for (int64_t c = cand_offsets[r]; c < cand_offsets[r + 1]; c++) {
            int64_t b = cand_bins[c];
            if (b >= n_bins) return ORACLE_EDATA;
            int64_t sum = oracle_sum_one(bank + b * nbits, q, read, L);
            if (sum < 0) return ORACLE_EDATA;
            pass[c] = (sum >= T) ? 1 : 0;
            if (sums) sums[c] = (uint32_t)sum;
        }
    }
    return ORACLE_OK;
}

/*
 * Full scan: the filter applied to every bin in [bin_begin, bin_end) for
 * every read (the "bin window" of Sec. 6.1, with every bin checked).
 * Passing pairs are listed read-major, bins ascending, with their sums.
 * Writes at most cap pairs; returns the number of passing pairs (may exceed
 * cap), or a negative error.
 */
int64_t oracle_scan(const uint8_t* bank, int64_t n_bins, int q, const uint8_t* reads,
                    const int64_t* read_offsets, int64_t n_reads, const uint16_t* E, int64_t bin_begin,
                    int64_t bin_end, int64_t cap, uint32_t* pair_read, uint32_t* pair_bin,
                    uint32_t* pair_sum) {
    if (bin_begin < 0 || bin_end > n_bins || bin_begin > bin_end) return ORACLE_EINVAL;
    int64_t nbits = oracle_bits_per_bin(q);
    int64_t n = 0;
    for (int64_t r = 0; r < n_reads; r++) {
        const uint8_t* read = reads + read_offsets[r];
        int64_t L = read_offsets[r + 1] - read_offsets[r];
        int64_t T = oracle_threshold(L, q, E[r]);
        for (int64_t b = bin_begin; b < bin_end; b++) {
            int64_t sum = oracle_sum_one(bank + b * nbits, q, read, L);
            if (sum < 0) return ORACLE_EDATA;
            if (sum >= T) {
                if (n < cap) {
                    pair_read[n] = (uint32_t)r;
                    pair_bin[n] = (uint32_t)b;
                    if (pair_sum) pair_sum[n] = (uint32_t)sum;
                }
                n++;
            }
        }
    }
    return n;
}

/*
 * One bin's bitvector straight from the reference, without a bank: for
 * sampled checks at sizes where the byte-per-bit bank would not fit.
 * row receives 4^q bytes.
 */
int oracle_bin_row(const uint8_t* ref2bit, int64_t len, int q, int bin_len, int overlap, int64_t b,
                   uint8_t* row) {
    if (len <= 0 || q < 1 || q > 8 || bin_len <= 0 || overlap < 0) return ORACLE_EINVAL;
    if (b < 0 || b >= oracle_n_bins(len, bin_len)) return ORACLE_EINVAL;
    int64_t nbits = oracle_bits_per_bin(q);
    int64_t s, e;
    oracle_bin_span(b, len, bin_len, overlap, &s, &e);
    memset(row, 0, (size_t)nbits);
    uint8_t tok[8];
    for (int64_t i = s; i + q <= e; i++) {
        for (int j = 0; j < q; j++) {
            int64_t k = i + j;
            tok[j] = (uint8_t)((ref2bit[k / 4] >> (2 * (k % 4))) & 3);
        }
        row[oracle_token(tok, q)] = 1;
    }
    return ORACLE_OK;
}

/*
 * oracle_filter for a candidate list without a bank: every candidate's
 * bitvector is rebuilt from the reference by oracle_bin_row (Sec. 3.1) and
 * handed to oracle_filter as a one-bin bank (Sec. 3.2 steps 1-5).  For
 * genome-scale references, whose byte-per-bit bank would not fit in memory.
 * Returns ORACLE_EDATA on a code > 3 or a bin id >= n_bins, ORACLE_EINVAL /
 * ORACLE_ENOMEM otherwise on failure.
 */
int oracle_filter_rows(const uint8_t* ref2bit, int64_t len, int q, int bin_len, int overlap,
                       const uint8_t* reads, const int64_t* read_offsets, int64_t n_reads,
                       const uint32_t* cand_bins, const int64_t* cand_offsets, const uint16_t* E,
                       uint8_t* pass, uint32_t* sums) {
    if (len <= 0 || q < 1 || q > 8 || bin_len <= 0 || overlap < 0) return ORACLE_EINVAL;
    int64_t n_bins = oracle_n_bins(len, bin_len);
    uint8_t* row = (uint8_t*)malloc((size_t)oracle_bits_per_bin(q));
    if (!row) return ORACLE_ENOMEM;
    int rc = ORACLE_OK;
    const uint32_t bin0 = 0;
    for (int64_t r = 0; r < n_reads && rc == ORACLE_OK; r++) {
        const uint8_t* read = reads + read_offsets[r];
        const int64_t one_read[2] = {0, read_offsets[r + 1] - read_offsets[r]};
        const int64_t one_cand[2] = {0, 1};
        for (int64_t c = cand_offsets[r]; c < cand_offsets[r + 1] && rc == ORACLE_OK; c++) {
            if (cand_bins[c] >= n_bins) {
                rc = ORACLE_EDATA;
                break;
            }
            oracle_bin_row(ref2bit, len, q, bin_len, overlap, cand_bins[c], row);
            rc = oracle_filter(row, 1, q, read, one_read, 1, &bin0, one_cand, E + r, pass + c, sums ? sums + c : 0);
        }
    }
    free(row);
    return rc;
}

/*
 * Sellers' semi-global edit distance: the fewest substitutions, insertions
 * and deletions that turn the read into some substring of text.  Used by
 * the tests to pin the zero-miss property the paper claims (Sec. 3.2:
 * no location that leads to a correct mapping is rejected).
 */
int64_t oracle_sellers(const uint8_t* read, int64_t L, const uint8_t* text, int64_t n) {
    int64_t* prev = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!prev || !cur) { free(prev); free(cur); return -1; }
    for (int64_t j = 0; j <= n; j++) prev[j] = 0; /* free start anywhere in text */
    for (int64_t i = 1; i <= L; i++) {
        cur[0] = i;
        for (int64_t j = 1; j <= n; j++) {
            int64_t best = prev[j - 1] + (read[i - 1] != text[j - 1] ? 1 : 0);
            if (prev[j] + 1 < best) best = prev[j] + 1;
            if (cur[j - 1] + 1 < best) best = cur[j - 1] + 1;
            cur[j] = best;
        }
        int64_t* t = prev; prev = cur; cur = t;
    }
    int64_t best = prev[0];
    for (int64_t j = 1; j <= n; j++)
        if (prev[j] < best) best = prev[j];
    free(prev);
    free(cur);
    return best;
}

/* ------------------------------------------------ seed locations (Sec. 1, 3.3) */

typedef struct { uint32_t bin; int64_t votes; } oracle_vote;

static int oracle_cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

static int oracle_cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

static int oracle_cmp_votes_desc(const void* a, const void* b) {
    const oracle_vote *x = (const oracle_vote*)a, *y = (const oracle_vote*)b;
    if (x->votes != y->votes) return x->votes > y->votes ? -1 : 1;
    return (x->bin > y->bin) - (x->bin < y->bin);
}

static int oracle_cmp_vote_bin(const void* a, const void* b) {
    const oracle_vote *x = (const oracle_vote*)a, *y = (const oracle_vote*)b;
    return (x->bin > y->bin) - (x->bin < y->bin);
}

/* key of the k bases at s (first base most significant), or -1 if one of
 * them is not a base code 0..3 */
static int64_t oracle_seed_key(const uint8_t* s, int k) {
    int64_t v = 0;
    for (int j = 0; j < k; j++) {
        if (s[j] > 3) return -1;
        v = v * 4 + s[j];
    }
    return v;
}

/* index of key in the sorted array keys[0..n), or -1 */
static int64_t oracle_find_key(const uint64_t* keys, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && keys[lo] == key) ? lo : -1;
}

/*
 * Candidate bins of every read from its exact seed locations, the way a
 * seed-and-extend mapper would hand them to the filter (Sec. 1 / Fig. 1:
 * seeds are looked up in a hash table of reference locations; Sec. 3.3:
 * only the bins that hold a potential seed location are checked).
 * Readings:
 *  - the seeds are the read's non-overlapping k-mers at offsets 0, k, 2k,
 *    ... (o + k <= L); a seed holding a code > 3 has no locations;
 *  - an exact occurrence of the seed at offset o at reference position p
 *    puts the read's start at p - o: it votes for the bin whose core holds
 *    max(0, p - o), clamped to the last bin;
 *  - the distinct voted bins are the candidates; when there are more than
 *    cap, the cap bins with the most votes are kept, equal votes going to
 *    the lower bin id; each read's list is ascending.
 * ref: codes 0..3 (len bases).  Writes cand_offsets[n + 1] always and
 * cand_bins only when the total fits in out_cap; returns the total, or a
 * negative error.
 */
int64_t oracle_seed_candidates(const uint8_t* ref, int64_t len, int k, const uint8_t* reads,
                               const int64_t* read_offsets, int64_t n, int bin_len, int64_t n_bins, int cap,
                               int64_t out_cap, uint32_t* cand_bins, int64_t* cand_offsets) {
    if (k < 1 || k > 15 || bin_len < 1 || n_bins < 1 || cap < 1 || n < 0) return ORACLE_EINVAL;
    /* 1. the seed keys the reads ask for, sorted, without repeats */
    int64_t n_keys = 0;
    for (int64_t r = 0; r < n; r++)
        for (int64_t o = 0; o + k <= read_offsets[r + 1] - read_offsets[r]; o += k) n_keys++;
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n_keys + 1));
    if (!keys) return ORACLE_ENOMEM;
    int64_t m = 0;
    for (int64_t r = 0; r < n; r++)
        for (int64_t o = 0; o + k <= read_offsets[r + 1] - read_offsets[r]; o += k) {
            int64_t key = oracle_seed_key(reads + read_offsets[r] + o, k);
            if (key >= 0) keys[m++] = (uint64_t)key;
        }
    qsort(keys, (size_t)m, sizeof(uint64_t), oracle_cmp_u64);
    int64_t u = 0;
    for (int64_t i = 0; i < m; i++)
        if (u == 0 || keys[u - 1] != keys[i]) keys[u++] = keys[i];
    /* 2. every reference position of each of those keys: one pass over the
     *    reference, recomputing each k-mer from its bases */
    int64_t* count = (int64_t*)calloc((size_t)(u + 1), sizeof(int64_t));
    if (!count) { free(keys); return ORACLE_ENOMEM; }
    for (int64_t p = 0; p + k <= len; p++) {
        int64_t key = oracle_seed_key(ref + p, k);
        int64_t i = key >= 0 ? oracle_find_key(keys, u, (uint64_t)key) : -1;
        if (i >= 0) count[i + 1]++;
    }
    for (int64_t i = 0; i < u; i++) count[i + 1] += count[i];
    int64_t* where = (int64_t*)malloc(sizeof(int64_t) * (size_t)(count[u] + 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(u + 1));
    if (!where || !fill) { free(keys); free(count); free(where); free(fill); return ORACLE_ENOMEM; }
    memcpy(fill, count, sizeof(int64_t) * (size_t)(u + 1));
    for (int64_t p = 0; p + k <= len; p++) {
        int64_t key = oracle_seed_key(ref + p, k);
        int64_t i = key >= 0 ? oracle_find_key(keys, u, (uint64_t)key) : -1;
        if (i >= 0) where[fill[i]++] = p;
    }
    free(fill);
    /* 3. per read: votes, distinct bins with their vote counts, the cap */
    int64_t total = 0;
    cand_offsets[0] = 0;
    for (int64_t r = 0; r < n; r++) {
        const int64_t L = read_offsets[r + 1] - read_offsets[r];
        int64_t* seed_at = (int64_t*)malloc(sizeof(int64_t) * (size_t)(L + 1));  /* seed offsets */
        if (!seed_at) { free(keys); free(count); free(where); return ORACLE_ENOMEM; }
        int64_t n_seeds = 0;
        for (int64_t o = 0; o + k <= L; o += k) seed_at[n_seeds++] = o;
        int64_t n_votes = 0;
        for (int64_t s = 0; s < n_seeds; s++) {
            int64_t key = oracle_seed_key(reads + read_offsets[r] + seed_at[s], k);
            int64_t i = key >= 0 ? oracle_find_key(keys, u, (uint64_t)key) : -1;
            if (i >= 0) n_votes += count[i + 1] - count[i];
        }
        uint32_t* votes = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n_votes + 1));
        oracle_vote* bins = (oracle_vote*)malloc(sizeof(oracle_vote) * (size_t)(n_votes + 1));
        if (!votes || !bins) {
            free(seed_at); free(votes); free(bins); free(keys); free(count); free(where);
            return ORACLE_ENOMEM;
        }
        int64_t v = 0;
        for (int64_t s = 0; s < n_seeds; s++) {
            const int64_t o = seed_at[s];
            int64_t key = oracle_seed_key(reads + read_offsets[r] + o, k);
            int64_t i = key >= 0 ? oracle_find_key(keys, u, (uint64_t)key) : -1;
            if (i < 0) continue;
            for (int64_t j = count[i]; j < count[i + 1]; j++) {
                int64_t start = where[j] - o;
                if (start < 0) start = 0;
                int64_t b = start / bin_len;
                if (b > n_bins - 1) b = n_bins - 1;
                votes[v++] = (uint32_t)b;
            }
        }
        free(seed_at);
        qsort(votes, (size_t)v, sizeof(uint32_t), oracle_cmp_u32);
        int64_t d = 0;
        for (int64_t j = 0; j < v; j++) {
            if (d > 0 && bins[d - 1].bin == votes[j]) {
                bins[d - 1].votes++;
            } else {
                bins[d].bin = votes[j];
                bins[d].votes = 1;
                d++;
            }
        }
        if (d > cap) {
            qsort(bins, (size_t)d, sizeof(oracle_vote), oracle_cmp_votes_desc);
            d = cap;
            qsort(bins, (size_t)d, sizeof(oracle_vote), oracle_cmp_vote_bin);
        }
        for (int64_t j = 0; j < d; j++)
            if (total + j < out_cap && cand_bins) cand_bins[total + j] = bins[j].bin;
        total += d;
        cand_offsets[r + 1] = total;
        free(votes);
        free(bins);
    }
    free(keys);
    free(count);
    free(where);
    return total;
}

/*
 * Seed Location Checker (Sec. 3.3, Fig. 4 steps 2-3): for every candidate
 * whose filter bit is 1, in candidate order, the read, the bin and the
 * reference segment the read mapper would align against: the bin's span
 * [b*bin_len, min(len, b*bin_len + bin_len + overlap)).  When seg is not
 * NULL, the segment's base codes are copied to seg + i*seg_stride (the rest
 * of the row is filled with 4).  Returns the number of passing candidates
 * (outputs written only while below out_cap), or a negative error.
 */
int64_t oracle_locate(const uint8_t* pass, const uint32_t* cand_bins, const int64_t* cand_offsets, int64_t n,
                      const uint8_t* ref, int64_t len, int bin_len, int overlap, int64_t out_cap, uint32_t* out_read,
                      uint32_t* out_bin, int64_t* out_begin, int64_t* out_end, uint8_t* seg, int64_t seg_stride) {
    if (bin_len < 1 || overlap < 0 || n < 0) return ORACLE_EINVAL;
    int64_t m = 0;
    for (int64_t r = 0; r < n; r++)
        for (int64_t c = cand_offsets[r]; c < cand_offsets[r + 1]; c++) {
            if (!pass[c]) continue;
            if (m < out_cap) {
                int64_t b = cand_bins[c], begin, end;
                oracle_bin_span(b, len, bin_len, overlap, &begin, &end);
                out_read[m] = (uint32_t)r;
                out_bin[m] = (uint32_t)b;
                out_begin[m] = begin;
                out_end[m] = end;
                if (seg) {
                    for (int64_t j = 0; j < seg_stride; j++)
                        seg[m * seg_stride + j] = (begin + j < end) ? ref[begin + j] : 4;
                }
            }
            m++;
        }
    return m;
}
