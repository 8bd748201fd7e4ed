"""Pins for the CPU oracle, against things other than the oracle itself.

Every check here is either brute force on tiny inputs (substring search,
Sellers edit distance, literal string token lists), a construction whose
answer the paper states (the AAAAA example of Sec. 3.4, the error
propagation of Fig. 5b, the exact-match count of Sec. 3.5), a closed form
the paper prints (footprint, counter width), or an invariant of the method
(zero misses, monotonicity, the sum bound).
"""
import json
import os

import numpy as np
import pytest

import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))

ACGT = "ACGT"


def s_of(codes):
    return "".join(ACGT[int(c)] for c in codes)


def codes_of(s):
    return np.frombuffer(s.translate(str.maketrans("ACGT", "\x00\x01\x02\x03")).encode(), dtype=np.uint8).copy()


def tok_str(t, q):
    """Token index -> bases, first base most significant (base-4 digits)."""
    return np.base_repr(t, 4).zfill(q).translate(str.maketrans("0123", "ACGT"))


def brute_bank(ref_s, q, bin_len, overlap):
    """bit(b, t) = 1 iff the q-mer t occurs as a substring of bin b's span."""
    n = len(ref_s)
    nb = -(-n // bin_len)
    bank = np.zeros((nb, 4 ** q), dtype=np.uint8)
    for b in range(nb):
        span = ref_s[b * bin_len: min(n, b * bin_len + bin_len + overlap)]
        for t in range(4 ** q):
            if tok_str(t, q) in span:
                bank[b, t] = 1
    return bank


def brute_sum(read_s, span_s, q):
    """Number of read positions whose q-mer occurs in the span (duplicates count)."""
    return sum(1 for i in range(len(read_s) - q + 1) if read_s[i:i + q] in span_s)


def levenshtein(a, b):
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j - 1] + (a[i - 1] != b[j - 1]), prev[j] + 1, cur[j - 1] + 1)
        prev = cur
    return prev[-1]


# ------------------------------------------------------------------ encoding

def test_unpack_bit_order(oracle):
    # base k sits in bits 2*(k%4) of byte k/4: 0xE4 = 11 10 01 00 -> A C G T
    assert list(oracle.unpack_ref(np.array([0xE4, 0x1B], dtype=np.uint8), 8)) == [0, 1, 2, 3, 3, 2, 1, 0]
    rng = np.random.default_rng(5)
    codes = rng.integers(0, 4, 1001).astype(np.uint8)
    assert np.array_equal(oracle.unpack_ref(synth.pack2bit(codes), 1001), codes)


def test_token_values(oracle):
    # Sec. 3.1 names GACAG and TTTTT; first base most significant
    g = GOLDEN["token_names"]
    assert oracle.bits_per_bin(g["q"]) == g["bits_per_bin"]
    assert [oracle.token(codes_of(t)) for t in g["tokens"]] == [int("20102", 4), 1023] == [530, 1023]
    assert oracle.token(codes_of("AAAAA")) == 0
    rng = np.random.default_rng(1)
    for q in range(1, 9):
        for _ in range(20):
            c = rng.integers(0, 4, q).astype(np.uint8)
            assert oracle.token(c) == int("".join(str(int(x)) for x in c), 4)
            assert tok_str(oracle.token(c), q) == s_of(c)


def test_bins_closed_forms(oracle):
    # 1 Mbp / 256: 3,907 bins, the last core holds 64 bases
    assert oracle.n_bins(1_000_000, 256) == 3907
    s, e = oracle.bin_span(3906, 1_000_000, 256, 100)
    assert (s, e) == (999_936, 1_000_000)
    assert oracle.n_bins(100_000_000, 256) == 390_625
    assert oracle.n_bins(3_100_000_000, 256) == 12_109_375
    s, e = oracle.bin_span(10, 1_000_000, 256, 100)
    assert (s, e) == (2560, 2560 + 356)


def test_footprint_and_counter_width(oracle):
    # Sec. 6.1: 450 x 2^16 bins of 4^5 bits is about 3.8 GB
    g = GOLDEN["footprint"]
    assert g["bins"] == 450 * 2 ** 16
    nbytes = g["bins"] * oracle.bits_per_bin(g["q"]) // 8
    assert nbytes == 3_774_873_600
    assert round(nbytes / 1e9, 1) == g["gb_rounded"]
    # Sec. 4.2: a seven-bit counter holds the largest sum of a 100 bp read
    g = GOLDEN["counter_width"]
    max_sum = oracle.sum_one(np.ones(1024, dtype=np.uint8), 5, np.zeros(g["L"], dtype=np.uint8))
    assert max_sum == 96 and max_sum < 2 ** g["bits"] and max_sum >= 2 ** (g["bits"] - 1)


# --------------------------------------------------------------- bank build

@pytest.mark.parametrize("q,bin_len,overlap,n", [
    (1, 7, 0, 50), (2, 7, 3, 61), (3, 32, 10, 500), (4, 50, 25, 777), (5, 100, 40, 1500),
    (6, 64, 30, 700), (3, 1000, 5, 300), (4, 17, 0, 4), (5, 16, 16, 3)])
def test_bank_matches_substring_search(oracle, q, bin_len, overlap, n):
    rng = np.random.default_rng(q * 1000 + n)
    codes = rng.integers(0, 4, n).astype(np.uint8)
    bank = oracle.build_bank(synth.pack2bit(codes), n, q, bin_len, overlap)
    assert np.array_equal(bank, brute_bank(s_of(codes), q, bin_len, overlap))


def test_bank_on_repeat_rich_reference(oracle):
    codes = synth.ref_with_repeats(4000, 7, 0.4, n_fam=3, fam_min=50, fam_max=300)
    bank = oracle.build_bank(synth.pack2bit(codes), 4000, 4, 256, 100)
    assert np.array_equal(bank, brute_bank(s_of(codes), 4, 256, 100))


def test_bin_row_matches_bank(oracle):
    codes = synth.ref_iid(3001, 9)
    r2 = synth.pack2bit(codes)
    bank = oracle.build_bank(r2, 3001, 5, 256, 100)
    for b in range(bank.shape[0]):
        assert np.array_equal(oracle.bin_row(r2, 3001, 5, 256, 100, b), bank[b])


# ------------------------------------------------------------------- filter

def test_filter_matches_brute_force(oracle):
    rng = np.random.default_rng(11)
    n, q, bl, ov = 3000, 4, 200, 60
    codes = rng.integers(0, 4, n).astype(np.uint8)
    ref_s = s_of(codes)
    bank = oracle.build_bank(synth.pack2bit(codes), n, q, bl, ov)
    nb = bank.shape[0]
    lens = rng.integers(0, 70, 40)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    reads = rng.integers(0, 4, int(offs[-1])).astype(np.uint8)
    # plant exact copies so that some sums are high
    for r in range(0, 40, 3):
        L = int(lens[r])
        st = int(rng.integers(0, n - L))
        reads[offs[r]:offs[r + 1]] = codes[st:st + L]
    E = rng.integers(0, 6, 40).astype(np.uint16)
    cb = np.concatenate([rng.choice(nb, 6, replace=False) for _ in range(40)]).astype(np.uint32)
    co = np.arange(0, 41 * 6, 6, dtype=np.int64)
    pass_, sums = oracle.filter(bank, q, reads, offs, cb, co, E)
    for r in range(40):
        rs = s_of(reads[offs[r]:offs[r + 1]])
        L = len(rs)
        for c in range(co[r], co[r + 1]):
            b = int(cb[c])
            span = ref_s[b * bl: min(n, b * bl + bl + ov)]
            s = brute_sum(rs, span, q)
            assert sums[c] == s
            # Sec. 3.2 step 5: pass iff the sum reaches the threshold
            n_tok = max(L - q + 1, 0)
            assert pass_[c] == int(s >= n_tok - q * int(E[r]))
    assert sums.max() > 0 and pass_.sum() > 0 and pass_.sum() < len(pass_)
    # the bank-free form rebuilds each candidate's row from the reference:
    # the same bytes, also for a slice of reads with its own offsets
    r2 = synth.pack2bit(codes)
    p2, s2 = oracle.filter_rows(r2, n, q, bl, ov, reads, offs, cb, co, E)
    assert np.array_equal(p2, pass_) and np.array_equal(s2, sums)
    a, z = 5, 20
    p3, s3 = oracle.filter_rows(r2, n, q, bl, ov, reads[offs[a]:offs[z]], offs[a:z + 1], cb[co[a]:co[z]],
                                co[a:z + 1], E[a:z])
    assert np.array_equal(p3, pass_[co[a]:co[z]]) and np.array_equal(s3, sums[co[a]:co[z]])


def test_aaaaa_example(oracle):
    # Sec. 3.4: an all-A read against a bin that is all G except one AAAAA:
    # every token of the read finds that AAAAA (the paper says "100"; a
    # 100 bp read has 96 tokens of size 5).
    ref = ["G"] * 400
    ref[100:105] = "AAAAA"
    codes = codes_of("".join(ref))
    bank = oracle.build_bank(synth.pack2bit(codes), 400, 5, 256, 100)
    g = GOLDEN["all_a_read"]
    read = np.zeros(g["L"], dtype=np.uint8)
    assert oracle.sum_one(bank[0], g["q"], read) == g["sum"]
    p, s = oracle.filter(bank, 5, read, np.array([0, 100]), np.array([0, 1], dtype=np.uint32),
                         np.array([0, 2]), np.array([5], dtype=np.uint16))
    assert list(s) == [g["sum"], 0] and list(p) == [1, 0]


def _distinct_kmer_segment(rng, n, q, tries=1000):
    """A random sequence whose q-mers are all distinct (greedy walk, restarts)."""
    for _ in range(tries):
        c = list(rng.integers(0, 4, q - 1))
        seen = set()
        while len(c) < n:
            for b in rng.permutation(4):
                km = tuple(c[len(c) - q + 1:] + [int(b)])
                if km not in seen:
                    seen.add(km)
                    c.append(int(b))
                    break
            else:
                break
        if len(c) == n:
            return np.array(c, dtype=np.uint8)
    raise RuntimeError("no segment")


def test_fig5b_error_propagation(oracle):
    # Fig. 5b with n = 4: a substitution or deletion removes n tokens of the
    # read from the bin, an insertion n-1 (counted against the error-free read).
    g = GOLDEN["error_propagation"]
    n = g["n"]
    rng = np.random.default_rng(3)
    checked = {"sub": 0, "del": 0, "ins": 0}
    for it in range(400):
        seg = _distinct_kmer_segment(rng, 60, n)
        span_s = s_of(seg)
        bank = oracle.build_bank(synth.pack2bit(seg), 60, n, 60, 0)[0]
        L = 40
        a = int(rng.integers(0, 60 - L))
        read = seg[a:a + L].copy()
        full = L - n + 1
        assert oracle.sum_one(bank, n, read) == full
        k = int(rng.integers(n, L - n))
        kind = ("sub", "del", "ins")[it % 3]
        if kind == "sub":
            mut = read.copy()
            mut[k] = (mut[k] + 1 + rng.integers(0, 3)) % 4
            new = [s_of(mut[i:i + n]) for i in range(k - n + 1, k + 1)]
            expect = full - n
        elif kind == "del":
            mut = np.delete(read, k)
            new = [s_of(mut[i:i + n]) for i in range(k - n + 1, k)]
            expect = (full - 1) - (n - 1)
        else:
            mut = np.insert(read, k, rng.integers(0, 4))
            new = [s_of(mut[i:i + n]) for i in range(k - n + 1, k + 1)]
            expect = full + 1 - n
        if any(t in span_s for t in new):
            continue  # the new tokens must not occur elsewhere in the bin
        got = oracle.sum_one(bank, n, mut)
        assert got == expect, (kind, got, expect)
        assert brute_sum(s_of(mut), span_s, n) == expect
        checked[kind] += 1
    assert min(checked.values()) >= 20
    # the figure's counts: tokens of the error-free read that the edit breaks
    assert full - (full - n) == g["substitution"]          # sub: the n tokens over the base
    assert full - ((full - 1) - (n - 1)) == g["deletion"]  # del: one token fewer, n-1 new
    assert (n - 1) == g["insertion"]                         # ins: n-1 tokens span the gap


def test_exact_match_count(oracle):
    # Sec. 3.5: a read that matches the bin exactly has L-(n-1) tokens present
    codes = synth.ref_iid(2000, 4)
    r2 = synth.pack2bit(codes)
    for q in (3, 4, 5, 6):
        bank = oracle.build_bank(r2, 2000, q, 256, 100)
        for st in (0, 100, 255, 600, 1700):
            b = st // 256
            for L in (q, 20, 100):
                read = codes[st:st + L]
                assert oracle.sum_one(bank[b], q, read) == L - q + 1
                assert oracle.threshold(L, q, 0) == L - q + 1


def test_threshold_is_worst_case_of_spaced_substitutions(oracle):
    # Sec. 3.5: the threshold is the sum left after E worst-case edits, each
    # removing n tokens of its own.  Build exactly that read and compare.
    rng = np.random.default_rng(8)
    n = 4
    done = 0
    for _ in range(600):
        seg = _distinct_kmer_segment(rng, 120, n)
        span_s = s_of(seg)
        bank = oracle.build_bank(synth.pack2bit(seg), 120, n, 120, 0)[0]
        L = 100
        read = seg[10:10 + L].copy()
        E = int(rng.integers(1, 6))
        pos = [n + j * (n + 2) for j in range(E)]
        mut = read.copy()
        ok = True
        for k in pos:  # pick a substitute whose n new tokens are absent from the bin
            for alt in rng.permutation(3):
                mut[k] = (read[k] + 1 + alt) % 4
                ms = s_of(mut)
                if not any(ms[i:i + n] in span_s for i in range(k - n + 1, k + 1)):
                    break
            else:
                ok = False
        if not ok:
            continue
        worst = oracle.sum_one(bank, n, mut)
        assert worst == (L - n + 1) - n * E
        assert oracle.threshold(L, n, E) == worst
        assert oracle.threshold(L, n, E - 1) > worst  # one edit fewer must not pass it
        done += 1
    assert done >= 30


def test_threshold_values(oracle):
    # the five workloads' thresholds, and a non-positive one
    assert oracle.threshold(100, 5, 5) == 71
    assert oracle.threshold(150, 5, 7) == 111
    assert oracle.threshold(50, 6, 2) == 33
    assert oracle.threshold(300, 6, 15) == 205
    assert oracle.threshold(100, 5, 0) == 96
    assert oracle.threshold(10, 5, 2) == -4


def test_short_reads(oracle):
    bank = np.ones((1, 1024), dtype=np.uint8)
    for L in range(0, 5):
        read = np.zeros(L, dtype=np.uint8)
        assert oracle.sum_one(bank[0], 5, read) == 0
        for E in (0, 1):
            p, _ = oracle.filter(bank, 5, read, np.array([0, L]), np.array([0], dtype=np.uint32),
                                 np.array([0, 1]), np.array([E], dtype=np.uint16))
            assert p[0] == 1  # T <= 0 for a read without tokens


def test_invalid_inputs(oracle):
    bank = np.ones((2, 1024), dtype=np.uint8)
    with pytest.raises(ValueError):
        oracle.filter(bank, 5, np.array([0, 1, 4, 2, 0], dtype=np.uint8), np.array([0, 5]),
                      np.array([0], dtype=np.uint32), np.array([0, 1]), np.array([1], dtype=np.uint16))
    with pytest.raises(ValueError):
        oracle.filter(bank, 5, np.zeros(5, dtype=np.uint8), np.array([0, 5]), np.array([2], dtype=np.uint32),
                      np.array([0, 1]), np.array([1], dtype=np.uint16))


# -------------------------------------------- zero misses (q-gram lemma)

def test_sellers_matches_substring_levenshtein(oracle):
    rng = np.random.default_rng(2)
    for _ in range(150):
        a = rng.integers(0, 4, int(rng.integers(0, 7))).astype(np.uint8)
        t = rng.integers(0, 4, int(rng.integers(0, 9))).astype(np.uint8)
        A, T = s_of(a), s_of(t)
        brute = min(levenshtein(A, T[i:j]) for i in range(len(T) + 1) for j in range(i, len(T) + 1))
        assert oracle.sellers(a, t) == brute


@pytest.mark.parametrize("q,E_max,seed", [(3, 3, 0), (4, 4, 1), (5, 3, 2), (6, 2, 3), (5, 5, 4)])
def test_no_miss_within_edit_distance(oracle, q, E_max, seed):
    # Sec. 3.2: no location holding a match within the tolerance is rejected.
    rng = np.random.default_rng(100 + seed)
    n, bl, L_max = 2500, 128, 48
    codes = synth.ref_with_repeats(n, seed, 0.35, n_fam=4, fam_min=60, fam_max=300, div_lo=0.0, div_hi=0.1)
    r2 = synth.pack2bit(codes)
    bank = oracle.build_bank(r2, n, q, bl, L_max + 8)
    nb = bank.shape[0]
    n_reads = 30
    lens = rng.integers(q, L_max + 1, n_reads)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    reads = np.empty(int(offs[-1]), dtype=np.uint8)
    for r in range(n_reads):
        L = int(lens[r])
        st = int(rng.integers(0, n - L - 8))
        seq = list(codes[st:st + L + 8])
        for _ in range(int(rng.integers(0, E_max + 1))):  # random edits
            k = int(rng.integers(0, L))
            kind = rng.integers(0, 3)
            if kind == 0:
                seq[k] = (seq[k] + 1 + int(rng.integers(0, 3))) % 4
            elif kind == 1:
                del seq[k]
            else:
                seq.insert(k, int(rng.integers(0, 4)))
        reads[offs[r]:offs[r + 1]] = np.array(seq[:L], dtype=np.uint8)
    cb = np.tile(np.arange(nb, dtype=np.uint32), n_reads)
    co = np.arange(0, (n_reads + 1) * nb, nb, dtype=np.int64)
    within = 0
    for E in range(0, E_max + 1):
        Ev = np.full(n_reads, E, dtype=np.uint16)
        pass_, sums = oracle.filter(bank, q, reads, offs, cb, co, Ev)
        for r in range(n_reads):
            read = reads[offs[r]:offs[r + 1]]
            for b in range(nb):
                s, e = oracle.bin_span(b, n, bl, L_max + 8)
                if not pass_[r * nb + b]:
                    # rejected: the read must be more than E edits from every substring
                    assert oracle.sellers(read, codes[s:e]) > E
                else:
                    within += 1
    assert within > 0


# --------------------------------------------------------------- invariants

def test_invariants_sum_bound_monotone_scan(oracle):
    w = synth.gather_iid(ref_len=20_000, n_reads=200, L=60, k=8)
    bank = oracle.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    prev = None
    for E in range(0, 6):
        Ev = np.full(w.n_reads, E, dtype=np.uint16)
        p, s = oracle.filter(bank, w.q, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, Ev)
        assert s.max() <= 60 - w.q + 1
        if prev is not None:
            assert np.all(p >= prev)  # more tolerated edits never reject more
        prev = p
    # the true bin of an error-free read always passes at E = 0
    clean = synth.reads(w.codes, w.read_offsets, 77, 0.0, 0.0)
    tb = (clean[1] // w.bin_len).astype(np.uint32)
    p, s = oracle.filter(bank, w.q, clean[0], w.read_offsets, tb, np.arange(w.n_reads + 1, dtype=np.int64),
                         np.zeros(w.n_reads, dtype=np.uint16))
    assert p.all() and np.all(s == 60 - w.q + 1)
    # full scan = filter over every bin
    Ev = np.full(w.n_reads, 5, dtype=np.uint16)
    pr, pb, ps = oracle.scan(bank, w.q, w.bases, w.read_offsets, Ev)
    allb = np.tile(np.arange(w.n_bins, dtype=np.uint32), w.n_reads)
    allo = np.arange(0, (w.n_reads + 1) * w.n_bins, w.n_bins, dtype=np.int64)
    p, s = oracle.filter(bank, w.q, w.bases, w.read_offsets, allb, allo, Ev)
    idx = np.nonzero(p)[0]
    assert np.array_equal(pr, idx // w.n_bins) and np.array_equal(pb, idx % w.n_bins)
    assert np.array_equal(ps, s[idx])
    # window restriction
    pr2, pb2, _ = oracle.scan(bank, w.q, w.bases, w.read_offsets, Ev, 10, 40)
    m = (pb >= 10) & (pb < 40)
    assert np.array_equal(pr2, pr[m]) and np.array_equal(pb2, pb[m])
