"""Pins for the oracle's seed-location functions: candidate bins from exact
seed locations (Sec. 1 Fig. 1 steps 2-3, Sec. 3.3) and the Seed Location
Checker (Sec. 3.3, Fig. 4).  Each pin comes from outside the oracle: a
hand-worked reference with the expected lists written out, brute-force
string search on small inputs, an invariant of exact reads, and the
synthetic generator's independent implementation of the same rule."""
from collections import Counter

import numpy as np
import pytest

import synth

CODE = {"A": 0, "C": 1, "G": 2, "T": 3}


def codes(s):
    return np.array([CODE.get(c, 4) for c in s], dtype=np.uint8)


def csr(reads):
    off = np.zeros(len(reads) + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in reads])
    return np.concatenate([codes(r) for r in reads]) if reads else np.zeros(0, np.uint8), off


# A 30-base reference with planted seeds (k=3, bins of 5):
#   ACG at 2, 12, 21;  TTT at 15, 27;  CCC at 5..9, 18, 24.
HAND_REF = "CCACGCCCCCCCACGTTTCCCACGCCCTTT"


def lists(cb, co):
    return [cb[co[r]:co[r + 1]].tolist() for r in range(len(co) - 1)]


def test_hand_example_votes_cap_and_ties(oracle):
    assert [i for i in range(28) if HAND_REF[i:i + 3] == "ACG"] == [2, 12, 21]
    assert [i for i in range(28) if HAND_REF[i:i + 3] == "TTT"] == [15, 27]
    ref = codes(HAND_REF)
    reads = ["ACGTTT",   # ACG@o0 -> starts 2,12,21; TTT@o3 -> 12,24: bins {0:1, 2:2, 4:2}
             "CCCTTT",   # CCC@o0 -> 5,6,7,8,9,18,24; TTT@o3 -> 12,24: {1:5, 2:1, 3:1, 4:2}
             "AAAACG",   # ACG@o3 -> -1 (clamped to 0), 9, 18: {0:1, 1:1, 3:1}
             "ACGNTT",   # the second seed holds a non-base code: no locations
             "AC",       # shorter than k: no seeds
             "GGGGGGCCA"]  # CCA@o6 at 0, 10, 19 -> starts -6 (a whole bin below 0: clamped), 4, 13: {0:2, 2:1}
    assert [i for i in range(28) if HAND_REF[i:i + 3] == "CCA"] == [0, 10, 19]
    bases, off = csr(reads)
    want = {4: [[0, 2, 4], [1, 2, 3, 4], [0, 1, 3], [0, 2, 4], [], [0, 2]],
            3: [[0, 2, 4], [1, 2, 4], [0, 1, 3], [0, 2, 4], [], [0, 2]],  # CCCTTT: 2 and 3 tie at one vote
            2: [[2, 4], [1, 4], [0, 1], [0, 2], [], [0, 2]],
            1: [[2], [1], [0], [0], [], [0]]}  # ACGTTT: 2 and 4 tie at two votes
    for cap, expect in want.items():
        cb, co = oracle.seed_candidates(ref, 3, bases, off, 5, 6, cap)
        assert lists(cb, co) == expect, cap


def brute_candidates(ref_str, reads, k, bin_len, n_bins, cap):
    out = []
    for r in reads:
        votes = Counter()
        for o in range(0, len(r) - k + 1, k):
            seed = r[o:o + k]
            if any(c not in CODE for c in seed):
                continue
            i = ref_str.find(seed)
            while i >= 0:
                votes[min(max(0, i - o) // bin_len, n_bins - 1)] += 1
                i = ref_str.find(seed, i + 1)
        keep = sorted(votes, key=lambda b: (-votes[b], b))[:cap]
        out.append(sorted(keep))
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_brute_force_string_search(oracle, seed):
    rng = np.random.default_rng(seed)
    n = 4000
    ref_str = "".join(rng.choice(list("ACGT"), n))
    ref_str = ref_str[:1000] + ref_str[200:700] + ref_str[1500:]  # a planted repeat
    reads = []
    for _ in range(60):
        s = int(rng.integers(0, len(ref_str) - 60))
        L = int(rng.integers(3, 60))
        r = list(ref_str[s:s + L])
        for _ in range(int(rng.integers(0, 3))):
            r[int(rng.integers(0, L))] = str(rng.choice(list("ACGTN")))
        reads.append("".join(r))
    k, bin_len = 5, 37
    n_bins = -(-len(ref_str) // bin_len)
    bases, off = csr(reads)
    for cap in (1, 4, 1000):
        cb, co = oracle.seed_candidates(codes(ref_str), k, bases, off, bin_len, n_bins, cap)
        assert lists(cb, co) == brute_candidates(ref_str, reads, k, bin_len, n_bins, cap)


def test_exact_reads_find_their_bin(oracle):
    ref = synth.ref_iid(300_000, 7)
    rng = np.random.default_rng(7)
    starts = rng.integers(0, len(ref) - 100, 500)
    bases = np.concatenate([ref[s:s + 100] for s in starts])
    off = np.arange(0, 501 * 100, 100, dtype=np.int64)
    n_bins = -(-len(ref) // 256)
    cb, co = oracle.seed_candidates(ref, 12, bases, off, 256, n_bins, 10_000)
    for r, s in enumerate(starts):
        got = cb[co[r]:co[r + 1]]
        assert s // 256 in got
        assert np.all(np.diff(got.astype(np.int64)) > 0)


def test_matches_synthetic_generator(oracle):
    """Two independent implementations of the same rule agree: the oracle's
    one-pass scan and the generator's parallel CSR index with radix sorts."""
    codes_ = synth.ref_with_repeats(1_000_000, 11, 0.3, n_fam=30, fam_min=200, fam_max=3000)
    off = synth.read_offsets(3000, 100, 100, 11)
    bases, _ = synth.reads(codes_, off, 11, 0.03, 0.01)
    n_bins = -(-len(codes_) // 256)
    idx = synth.seed_index(codes_, 12)
    for cap in (3, 50, 10_000):
        cb_s, co_s = synth.cands_seeds(idx, bases, off, 256, n_bins, cap, 12)
        cb_o, co_o = oracle.seed_candidates(codes_, 12, bases, off, 256, n_bins, cap)
        assert np.array_equal(co_s, co_o) and np.array_equal(cb_s, cb_o)


def test_locate_hand_example(oracle):
    ref = codes(HAND_REF)
    cb = np.array([0, 2, 4, 5, 1, 3], np.uint32)
    co = np.array([0, 4, 4, 6], np.int64)  # read 0: bins 0,2,4,5; read 1: none; read 2: 1,3
    ps = np.array([1, 0, 1, 1, 0, 1], np.uint8)
    rd, bn, be, en, seg = oracle.locate(ps, cb, co, ref, 5, 3, seg_stride=9)
    assert rd.tolist() == [0, 0, 0, 2]
    assert bn.tolist() == [0, 4, 5, 3]
    assert be.tolist() == [0, 20, 25, 15]
    assert en.tolist() == [8, 28, 30, 23]  # spans of 5 + 3, the last clipped at 30
    assert seg[0].tolist() == codes("CCACGCCC").tolist() + [4]
    assert seg[2].tolist() == codes("CCTTT").tolist() + [4] * 4
    assert seg[3].tolist() == codes("TTTCCCAC").tolist() + [4]
