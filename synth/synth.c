/*
 * Seeded synthetic inputs for the seed-location filter: references, reads,
 * candidate bin lists.  Shared by the tests, the oracle checks and the
 * benchmark.  This file holds none of the filter's arithmetic (no q-gram
 * tokens, bitvectors, sums or thresholds); it only draws data.
 *
 * Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), one stream per
 * purpose, seeded by the caller.  Uniform integers use the multiply-shift
 * range reduction (Lemire 2019).  All arithmetic is integer or IEEE double
 * basic operations compiled with -ffp-contract=off, so x86-64 and aarch64
 * produce the same data for the same seed (the log-uniform draw also uses
 * libm exp/log, see synth_cands_random).
 *
 * Base codes: A=0, C=1, G=2, T=3, one byte per base.  The 2-bit packed
 * reference holds base k in bits 2*(k%4) .. 2*(k%4)+1 of byte k/4.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s; } rng_t;

static uint64_t rng_next(rng_t* g) {
    uint64_t z = (g->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static rng_t rng_make(uint64_t seed, uint64_t stream) {
    rng_t g;
    g.s = seed * 0xD1B54A32D192ED03ULL + stream * 0x8CB92BA72F3D8DD7ULL + 1;
    (void)rng_next(&g);
    return g;
}

static uint64_t rng_below(rng_t* g, uint64_t n) {
    return (uint64_t)(((__uint128_t)rng_next(g) * (__uint128_t)n) >> 64);
}

static double rng_unit(rng_t* g) { return (double)(rng_next(g) >> 11) * 0x1.0p-53; }

/* probability p in [0,1] -> 64-bit threshold t with P(rng_next < t) = p */
static uint64_t prob_threshold(double p) {
    if (p <= 0.0) return 0;
    if (p >= 1.0) return UINT64_MAX;
    return (uint64_t)(p * 18446744073709551616.0);
}

/* ---------------------------------------------------------------- refs */

/* i.i.d. uniform ACGT, 32 bases per 64-bit draw. */
void synth_ref_iid(uint64_t seed, int64_t len, uint8_t* codes) {
    rng_t g = rng_make(seed, 11);
    int64_t k = 0;
    while (k < len) {
        uint64_t x = rng_next(&g);
        for (int j = 0; j < 32 && k < len; j++, k++) {
            codes[k] = (uint8_t)(x & 3);
            x >>= 2;
        }
    }
}

/*
 * Overwrite an i.i.d. reference with planted repeat families: n_fam
 * consensus sequences of i.i.d. bases with lengths uniform in
 * [fam_min, fam_max]; copies of a uniformly chosen family go to uniform
 * positions, each copy with its own per-base substitution probability drawn
 * uniformly from [div_lo, div_hi], until at least frac*len bases are covered.
 * Returns the number of copies placed, or -1 on bad arguments / allocation.
 */
int64_t synth_ref_repeats(uint64_t seed, int64_t len, double frac, int n_fam, int fam_min,
                          int fam_max, double div_lo, double div_hi, uint8_t* codes) {
    if (n_fam <= 0 || fam_min <= 0 || fam_max < fam_min || (int64_t)fam_max >= len) return -1;
    rng_t g = rng_make(seed, 23);
    int64_t* fam_len = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_fam);
    int64_t* fam_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_fam + 1));
    if (!fam_len || !fam_off) { free(fam_len); free(fam_off); return -1; }
    fam_off[0] = 0;
    for (int f = 0; f < n_fam; f++) {
        fam_len[f] = fam_min + (int64_t)rng_below(&g, (uint64_t)(fam_max - fam_min + 1));
        fam_off[f + 1] = fam_off[f] + fam_len[f];
    }
    uint8_t* cons = (uint8_t*)malloc((size_t)fam_off[n_fam]);
    uint8_t* covered = (uint8_t*)calloc((size_t)(len / 8 + 1), 1);
    if (!cons || !covered) { free(fam_len); free(fam_off); free(cons); free(covered); return -1; }
    for (int64_t j = 0; j < fam_off[n_fam]; j++) cons[j] = (uint8_t)(rng_next(&g) >> 62);

    int64_t target = (int64_t)(frac * (double)len);
    int64_t n_cov = 0, copies = 0;
    while (n_cov < target) {
        int f = (int)rng_below(&g, (uint64_t)n_fam);
        int64_t fl = fam_len[f];
        int64_t p = (int64_t)rng_below(&g, (uint64_t)(len - fl + 1));
        double d = div_lo + (div_hi - div_lo) * rng_unit(&g);
        uint64_t thr = prob_threshold(d);
        const uint8_t* c = cons + fam_off[f];
        for (int64_t j = 0; j < fl; j++) {
            uint8_t b = c[j];
            if (rng_next(&g) < thr) b = (uint8_t)((b + 1 + rng_below(&g, 3)) & 3);
            int64_t x = p + j;
            codes[x] = b;
            uint8_t bit = (uint8_t)(1u << (x & 7));
            if (!(covered[x >> 3] & bit)) { covered[x >> 3] |= bit; n_cov++; }
        }
        copies++;
    }
    free(fam_len); free(fam_off); free(cons); free(covered);
    return copies;
}

/* 4 bases per byte, base k at bits 2*(k%4). out must hold (len+3)/4 bytes. */
void synth_pack2bit(const uint8_t* codes, int64_t len, uint8_t* out) {
    int64_t nb = (len + 3) / 4;
    memset(out, 0, (size_t)nb);
    for (int64_t k = 0; k < len; k++) out[k >> 2] |= (uint8_t)((codes[k] & 3) << (2 * (k & 3)));
}

/* --------------------------------------------------------------- reads */

/* lengths uniform in [lmin, lmax]; offsets[0]=0, offsets[r+1]=offsets[r]+len_r */
void synth_read_lengths(uint64_t seed, int64_t n, int lmin, int lmax, int64_t* offsets) {
    rng_t g = rng_make(seed, 31);
    offsets[0] = 0;
    for (int64_t r = 0; r < n; r++) {
        int64_t L = lmin + (int64_t)rng_below(&g, (uint64_t)(lmax - lmin + 1));
        offsets[r + 1] = offsets[r] + L;
    }
}

/*
 * Sample reads from the reference.  Read r starts at a uniform position and
 * walks the reference: with probability indel a single-base indel (half
 * insertions of a uniform base, half deletions of the next reference base),
 * otherwise the next reference base, substituted by one of the other three
 * with probability sub.  The walk stops when the read has its length.
 * starts[r] receives the reference start.  Requires len > 2*max length.
 * Returns 0, or -1 if the reference is too short.
 */
int synth_reads(uint64_t seed, const uint8_t* codes, int64_t len, int64_t n, const int64_t* offsets,
                double sub, double indel, uint8_t* bases, int64_t* starts) {
    rng_t g = rng_make(seed, 37);
    uint64_t t_indel = prob_threshold(indel), t_sub = prob_threshold(sub);
    for (int64_t r = 0; r < n; r++) {
        int64_t L = offsets[r + 1] - offsets[r];
        if (len <= 2 * L + 1) return -1;
        int64_t pos = (int64_t)rng_below(&g, (uint64_t)(len - 2 * L - 1));
        starts[r] = pos;
        uint8_t* out = bases + offsets[r];
        int64_t k = 0;
        while (k < L) {
            if (rng_next(&g) < t_indel) {
                if (rng_next(&g) >> 63) out[k++] = (uint8_t)rng_below(&g, 4);
                else pos++;
                continue;
            }
            uint8_t b = codes[pos++];
            if (rng_next(&g) < t_sub) b = (uint8_t)((b + 1 + rng_below(&g, 3)) & 3);
            out[k++] = b;
        }
    }
    return 0;
}

/* ---------------------------------------------------------- candidates */

/* sort u32 ascending: insertion sort for short arrays, else four 8-bit LSD
 * radix passes through tmp (same length) */
static void sort_u32(uint32_t* a, int64_t n, uint32_t* tmp) {
    if (n <= 48) {
        for (int64_t i = 1; i < n; i++) {
            uint32_t x = a[i];
            int64_t j = i - 1;
            while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; j--; }
            a[j + 1] = x;
        }
        return;
    }
    int64_t cnt[257];
    uint32_t* src = a;
    uint32_t* dst = tmp;
    for (int pass = 0; pass < 4; pass++) {
        int sh = 8 * pass;
        memset(cnt, 0, sizeof(cnt));
        for (int64_t i = 0; i < n; i++) cnt[((src[i] >> sh) & 0xFF) + 1]++;
        for (int b = 0; b < 256; b++) cnt[b + 1] += cnt[b];
        for (int64_t i = 0; i < n; i++) dst[cnt[(src[i] >> sh) & 0xFF]++] = src[i];
        uint32_t* t = src; src = dst; dst = t;
    }
    /* four passes: the result is back in a */
}

/* per-read generator, so that reads can be drawn in any order or in parallel */
static rng_t rng_read(uint64_t seed, uint64_t stream, int64_t r) {
    return rng_make(seed * 0x9E3779B97F4A7C15ULL + (uint64_t)r, stream);
}

/*
 * Candidate counts per read: k_fixed > 0 gives k_fixed for every read;
 * otherwise k = floor(exp(U * ln(k_max))) clamped to [1, k_max] (log-uniform).
 * Counts are clamped to n_bins.  Writes cand_offsets[0..n].
 */
void synth_cand_counts(uint64_t seed, int64_t n, int k_fixed, int k_max, int64_t n_bins,
                       int64_t* cand_offsets) {
    cand_offsets[0] = 0;
    double lk = log((double)(k_max > 1 ? k_max : 1));
    for (int64_t r = 0; r < n; r++) {
        int64_t k;
        if (k_fixed > 0) k = k_fixed;
        else {
            rng_t g = rng_read(seed, 41, r);
            k = (int64_t)floor(exp(rng_unit(&g) * lk));
            if (k < 1) k = 1;
            if (k > k_max) k = k_max;
        }
        if (k > n_bins) k = n_bins;
        cand_offsets[r + 1] = cand_offsets[r] + k;
    }
}

/*
 * Candidate bins: the read's true bin floor(start/bin_len) plus distinct
 * uniform others, sorted ascending.  cand_offsets from synth_cand_counts.
 */
int synth_cands_random(uint64_t seed, int64_t n, const int64_t* starts, int bin_len, int64_t n_bins,
                       const int64_t* cand_offsets, uint32_t* cand_bins) {
    int64_t kmax = 1;
    for (int64_t r = 0; r < n; r++)
        if (cand_offsets[r + 1] - cand_offsets[r] > kmax) kmax = cand_offsets[r + 1] - cand_offsets[r];
    int err = 0;
#pragma omp parallel
    {
        uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(2 * kmax + 2));
        if (!tmp) err = 1;
#pragma omp for schedule(dynamic, 256)
        for (int64_t r = 0; r < n; r++) {
            int64_t k = cand_offsets[r + 1] - cand_offsets[r];
            if (k <= 0 || !tmp) continue;
            rng_t g = rng_read(seed, 43, r);
            uint32_t* c = cand_bins + cand_offsets[r];
            int64_t tb = starts[r] / bin_len;
            if (tb >= n_bins) tb = n_bins - 1;
            c[0] = (uint32_t)tb;
            int64_t have = 1;
            while (have < k) {
                int64_t need = k - have;
                for (int64_t j = 0; j < need; j++) c[have + j] = (uint32_t)rng_below(&g, (uint64_t)n_bins);
                int64_t m = have + need;
                sort_u32(c, m, tmp);
                int64_t u = 0;
                for (int64_t j = 0; j < m; j++)
                    if (u == 0 || c[j] != c[u - 1]) c[u++] = c[j];
                have = u;
            }
        }
        free(tmp);
    }
    return err ? -1 : 0;
}

/* ----------------------------------------------- exact k-mer seed index */

static uint64_t kmer_key(const uint8_t* s, int k) {
    uint64_t v = 0;
    for (int j = 0; j < k; j++) v = (v << 2) | (s[j] & 3);
    return v;
}

/*
 * CSR index of every k-mer start position: offsets[4^k + 1] (uint32),
 * positions[len-k+1] (uint32) grouped by key.  Built in parallel; the order
 * of positions within a key is unspecified (the candidate lists drawn from
 * the index do not depend on it: hits are deduplicated and sorted by bin).
 */
int synth_seed_index(const uint8_t* codes, int64_t len, int k, uint32_t* offsets, uint32_t* positions) {
    if (k < 1 || k > 15 || len < k || len > 0xFFFFFFFFLL) return -1;
    uint64_t nk = 1ULL << (2 * k);
    memset(offsets, 0, sizeof(uint32_t) * (size_t)(nk + 1));
    int64_t npos = len - k + 1;
    uint64_t mask = nk - 1;
#pragma omp parallel
    {
#ifdef _OPENMP
        int nt = omp_get_num_threads(), t = omp_get_thread_num();
#else
        int nt = 1, t = 0;
#endif
        int64_t a = npos * t / nt, b = npos * (t + 1) / nt;
        if (a < b) {
            uint64_t v = kmer_key(codes + a, k - 1);
            for (int64_t p = a; p < b; p++) {
                v = ((v << 2) | codes[p + k - 1]) & mask;
#pragma omp atomic
                offsets[v + 1]++;
            }
        }
    }
    for (uint64_t x = 0; x < nk; x++) offsets[x + 1] += offsets[x];
    uint32_t* fill = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nk);
    if (!fill) return -1;
    memcpy(fill, offsets, sizeof(uint32_t) * (size_t)nk);
#pragma omp parallel
    {
#ifdef _OPENMP
        int nt = omp_get_num_threads(), t = omp_get_thread_num();
#else
        int nt = 1, t = 0;
#endif
        int64_t a = npos * t / nt, b = npos * (t + 1) / nt;
        if (a < b) {
            uint64_t v = kmer_key(codes + a, k - 1);
            for (int64_t p = a; p < b; p++) {
                v = ((v << 2) | codes[p + k - 1]) & mask;
                uint32_t slot;
#pragma omp atomic capture
                slot = fill[v]++;
                positions[slot] = (uint32_t)p;
            }
        }
    }
    free(fill);
    return 0;
}

/*
 * The same CSR index restricted to the k-mers set in `needed` (a bitmap of
 * 4^k bits): offsets[4^k + 1] count only needed keys.  Call with
 * positions == NULL to count (returns the number of positions), then with
 * a buffer of that size to fill.  Other keys have empty ranges.
 */
int64_t synth_seed_index_needed(const uint8_t* codes, int64_t len, int k, const uint64_t* needed,
                                uint32_t* offsets, uint32_t* positions) {
    if (k < 1 || k > 15 || len < k || len > 0xFFFFFFFFLL) return -1;
    uint64_t nk = 1ULL << (2 * k);
    int64_t npos = len - k + 1;
    uint64_t mask = nk - 1;
    if (!positions) {
        memset(offsets, 0, sizeof(uint32_t) * (size_t)(nk + 1));
#pragma omp parallel
        {
#ifdef _OPENMP
            int nt = omp_get_num_threads(), t = omp_get_thread_num();
#else
            int nt = 1, t = 0;
#endif
            int64_t a = npos * t / nt, b = npos * (t + 1) / nt;
            if (a < b) {
                uint64_t v = kmer_key(codes + a, k - 1);
                for (int64_t p = a; p < b; p++) {
                    v = ((v << 2) | codes[p + k - 1]) & mask;
                    if ((needed[v >> 6] >> (v & 63)) & 1) {
#pragma omp atomic
                        offsets[v + 1]++;
                    }
                }
            }
        }
        for (uint64_t x = 0; x < nk; x++) offsets[x + 1] += offsets[x];
        return (int64_t)offsets[nk];
    }
    uint32_t* fill = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nk);
    if (!fill) return -1;
    memcpy(fill, offsets, sizeof(uint32_t) * (size_t)nk);
#pragma omp parallel
    {
#ifdef _OPENMP
        int nt = omp_get_num_threads(), t = omp_get_thread_num();
#else
        int nt = 1, t = 0;
#endif
        int64_t a = npos * t / nt, b = npos * (t + 1) / nt;
        if (a < b) {
            uint64_t v = kmer_key(codes + a, k - 1);
            for (int64_t p = a; p < b; p++) {
                v = ((v << 2) | codes[p + k - 1]) & mask;
                if ((needed[v >> 6] >> (v & 63)) & 1) {
                    uint32_t slot;
#pragma omp atomic capture
                    slot = fill[v]++;
                    positions[slot] = (uint32_t)p;
                }
            }
        }
    }
    free(fill);
    return (int64_t)offsets[nk];
}

typedef struct { uint32_t bin, support; } bin_support;

static int cmp_support(const void* a, const void* b) {
    const bin_support *x = (const bin_support*)a, *y = (const bin_support*)b;
    if (x->support != y->support) return (x->support < y->support) - (x->support > y->support);
    return (x->bin > y->bin) - (x->bin < y->bin);
}

static int cmp_bin(const void* a, const void* b) {
    const bin_support *x = (const bin_support*)a, *y = (const bin_support*)b;
    return (x->bin > y->bin) - (x->bin < y->bin);
}

/* distinct voted bins of one read (see synth_cands_seeds); returns the
 * count, bins in (*hits)[0..count) ascending; -1 on allocation failure.
 * bins/tmp: u32 scratch of *hcap entries each (grown with hits). */
static int64_t seed_bins_of_read(const uint32_t* idx_offsets, const uint32_t* idx_positions, int k,
                                 const uint8_t* s, int64_t L, int bin_len, int64_t n_bins, int cap,
                                 bin_support** hits, uint32_t** bins, uint32_t** tmp, int64_t* hcap) {
    int64_t nh = 0;
    for (int64_t o = 0; o + k <= L; o += k) {
        uint64_t key = kmer_key(s + o, k);
        uint32_t a = idx_offsets[key], b = idx_offsets[key + 1];
        if (nh + (int64_t)(b - a) > *hcap) {
            while (nh + (int64_t)(b - a) > *hcap) *hcap *= 2;
            bin_support* h2 = (bin_support*)realloc(*hits, sizeof(bin_support) * (size_t)*hcap);
            uint32_t* b2 = (uint32_t*)realloc(*bins, sizeof(uint32_t) * (size_t)*hcap);
            uint32_t* t2 = (uint32_t*)realloc(*tmp, sizeof(uint32_t) * (size_t)*hcap);
            if (h2) *hits = h2;
            if (b2) *bins = b2;
            if (t2) *tmp = t2;
            if (!h2 || !b2 || !t2) return -1;
        }
        for (uint32_t j = a; j < b; j++) {
            int64_t st = (int64_t)idx_positions[j] - o;
            if (st < 0) st = 0;
            int64_t bin = st / bin_len;
            if (bin >= n_bins) bin = n_bins - 1;
            (*bins)[nh++] = (uint32_t)bin;
        }
    }
    sort_u32(*bins, nh, *tmp);
    bin_support* h = *hits;
    int64_t u = 0;
    for (int64_t j = 0; j < nh; j++) {
        if (u > 0 && h[u - 1].bin == (*bins)[j]) h[u - 1].support++;
        else { h[u].bin = (*bins)[j]; h[u].support = 1; u++; }
    }
    if (u > cap) {
        qsort(h, (size_t)u, sizeof(bin_support), cmp_support);
        u = cap;
        qsort(h, (size_t)u, sizeof(bin_support), cmp_bin);
    }
    return u;
}

/*
 * Seed-hit candidates, as a hash-table read mapper would produce them:
 * non-overlapping k-mers of the read at offsets 0, k, 2k, ...; every exact
 * hit p of the seed at offset o votes for bin floor(max(0, p-o)/bin_len)
 * (clamped to n_bins-1); distinct bins are kept, and if more than cap, the
 * cap most-voted ones (ties to the lower bin id); output sorted ascending.
 * Writes at most cap_total bins; returns the total needed (a return value
 * above cap_total means the output was truncated), or -1 on error.
 */
int64_t synth_cands_seeds(const uint32_t* idx_offsets, const uint32_t* idx_positions, int k,
                          const uint8_t* bases, const int64_t* read_offsets, int64_t n, int bin_len,
                          int64_t n_bins, int cap, int64_t cap_total, uint32_t* cand_bins,
                          int64_t* cand_offsets) {
    int err = 0;
    /* pass 1: counts */
#pragma omp parallel
    {
        int64_t hcap = 1 << 12;
        bin_support* hits = (bin_support*)malloc(sizeof(bin_support) * (size_t)hcap);
        uint32_t* bins = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)hcap);
        uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)hcap);
        if (!hits || !bins || !tmp) err = 1;
#pragma omp for schedule(dynamic, 256)
        for (int64_t r = 0; r < n; r++) {
            if (!hits || !bins || !tmp) continue;
            int64_t u = seed_bins_of_read(idx_offsets, idx_positions, k, bases + read_offsets[r],
                                          read_offsets[r + 1] - read_offsets[r], bin_len, n_bins, cap, &hits, &bins,
                                          &tmp, &hcap);
            if (u < 0) { err = 1; u = 0; }
            cand_offsets[r + 1] = u;
        }
        free(hits); free(bins); free(tmp);
    }
    if (err) return -1;
    cand_offsets[0] = 0;
    for (int64_t r = 0; r < n; r++) cand_offsets[r + 1] += cand_offsets[r];
    int64_t total = cand_offsets[n];
    if (total > cap_total) return total;
    /* pass 2: bins */
#pragma omp parallel
    {
        int64_t hcap = 1 << 12;
        bin_support* hits = (bin_support*)malloc(sizeof(bin_support) * (size_t)hcap);
        uint32_t* bins = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)hcap);
        uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)hcap);
        if (!hits || !bins || !tmp) err = 1;
#pragma omp for schedule(dynamic, 256)
        for (int64_t r = 0; r < n; r++) {
            if (!hits || !bins || !tmp) continue;
            int64_t u = seed_bins_of_read(idx_offsets, idx_positions, k, bases + read_offsets[r],
                                          read_offsets[r + 1] - read_offsets[r], bin_len, n_bins, cap, &hits, &bins,
                                          &tmp, &hcap);
            if (u < 0) { err = 1; continue; }
            for (int64_t j = 0; j < u; j++) cand_bins[cand_offsets[r] + j] = hits[j].bin;
        }
        free(hits); free(bins); free(tmp);
    }
    return err ? -1 : total;
}

/* per-read E = floor(num * L / den) (integer arithmetic) */
void synth_E_rate(const int64_t* read_offsets, int64_t n, int num, int den, uint16_t* E) {
    for (int64_t r = 0; r < n; r++) {
        int64_t L = read_offsets[r + 1] - read_offsets[r];
        E[r] = (uint16_t)((num * L) / den);
    }
}
