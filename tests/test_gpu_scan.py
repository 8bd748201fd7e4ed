"""GPU parity of the full-scan form (tcgen05 tensor cores) against the oracle.

The passing (read, bin) set is unique; the kernel emits it in no particular
order, so both sides are compared sorted, with their accumulation sums.
"""
import numpy as np
import pytest
import torch

import paper_1711_01177_gb300 as grim
import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    grim.build()
    grim.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def gpu_pairs(res):
    n = res.n_pairs
    pr = host(res.pair_read[:n], np.uint32)
    pb = host(res.pair_bin[:n], np.uint32)
    ps = host(res.pair_sum[:n], np.uint16)
    o = np.lexsort((pb, pr))
    return pr[o], pb[o], ps[o]


def make_reads(codes, n_reads, rng, lmin=0, lmax=200, planted=0.5, sub=0.02):
    lens = rng.integers(lmin, lmax + 1, n_reads)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    parts = []
    for L in lens:
        if rng.random() < planted:
            st = int(rng.integers(0, len(codes) - L))
            r = codes[st:st + L].copy()
            r ^= (rng.random(L) < sub).astype(np.uint8)
        else:
            r = rng.integers(0, 4, L).astype(np.uint8)
        parts.append(r)
    bases = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
    return bases.astype(np.uint8), offs


def check_scan(oracle, codes, q, bin_len, overlap, bases, offs, E, bin_begin=0, bin_end=None, cap=1 << 20):
    r2 = synth.pack2bit(codes)
    bank = grim.grim_build_bank(dev(r2), len(codes), q, bin_len, overlap)
    res = grim.grim_scan(bank, dev(bases), dev(offs), dev(E), bin_begin, bin_end, cap=cap, with_read_pass=True)
    st, flags = grim.grim_bank_status(bank)
    assert (st, flags) == (grim.GRIM_OK, 0)
    ob = oracle.build_bank(r2, len(codes), q, bin_len, overlap)
    opr, opb, ops = oracle.scan(ob, q, bases, offs, E, bin_begin, bank.n_bins if bin_end is None else bin_end)
    gpr, gpb, gps = gpu_pairs(res)
    assert res.n_pairs == len(opr)
    assert np.array_equal(gpr, opr) and np.array_equal(gpb, opb)
    assert np.array_equal(gps, ops.astype(np.uint16))
    n_reads = len(offs) - 1
    rp = host(res.read_pass[:n_reads], np.uint32)
    assert np.array_equal(rp, np.bincount(opr, minlength=n_reads).astype(np.uint32))
    bank.free()
    return len(opr)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_scan_every_q(oracle, q):
    rng = np.random.default_rng(500 + q)
    codes = synth.ref_with_repeats(60_000, 9 + q, 0.3, n_fam=8, fam_min=100, fam_max=800)
    bases, offs = make_reads(codes, 300, rng, lmax=160)
    E = rng.integers(0, 8, 300).astype(np.uint16)
    n = check_scan(oracle, codes, q, 100, 170, bases, offs, E)
    assert n > 0


def test_scan_plain_workload_sizes(oracle):
    """1 Mbp reference (3,907 bins: a ragged last bin tile), 1,000 reads (ragged read tile)."""
    w = synth.gather_iid(n_reads=1000)
    n = check_scan(oracle, w.codes, w.q, w.bin_len, w.overlap, w.bases, w.read_offsets, w.E)
    assert n >= 500  # most reads pass their own bin


def test_scan_heavy_reads_use_more_digits(oracle):
    """Token counts above 3, 15 and 255 (2, 4 and 8 base-4 digits: every
    digit class of the full scan's B rows)."""
    rng = np.random.default_rng(7)
    codes = synth.ref_iid(30_000, 5)
    codes[3000:3400] = 0                      # poly-A
    codes[8000:8600] = np.tile([0, 1], 300)   # (AC)n
    codes[15000:15900] = np.tile([0, 1, 3], 300)
    reads_l = [np.zeros(300, np.uint8), np.zeros(40, np.uint8), np.tile([0, 1], 150).astype(np.uint8),
               np.tile([0, 1, 3], 100).astype(np.uint8), codes[15000:15300].copy(), codes[100:250].copy(),
               np.zeros(2000, np.uint8)]
    for i in range(200):  # many random reads so tiles of all classes fill partially
        reads_l.append(codes[i * 100:i * 100 + 100].copy() if i % 3 else rng.integers(0, 4, 120).astype(np.uint8))
    offs = np.concatenate([[0], np.cumsum([len(x) for x in reads_l])]).astype(np.int64)
    bases = np.concatenate(reads_l)
    E = rng.integers(0, 6, len(reads_l)).astype(np.uint16)
    E[:7] = [3, 1, 10, 10, 2, 0, 30]
    n = check_scan(oracle, codes, 5, 256, 2100, bases, offs, E)
    assert n > 0


def test_scan_window_and_empty(oracle):
    rng = np.random.default_rng(3)
    codes = synth.ref_iid(80_000, 2)
    bases, offs = make_reads(codes, 150, rng, lmax=120)
    E = np.full(150, 4, np.uint16)
    check_scan(oracle, codes, 4, 64, 130, bases, offs, E, bin_begin=77, bin_end=1001)
    check_scan(oracle, codes, 4, 64, 130, bases, offs, E, bin_begin=500, bin_end=500)
    check_scan(oracle, codes, 4, 64, 130, bases, offs[:1], E[:0])


def test_scan_overflow_counts_all_pairs(oracle):
    codes = synth.ref_iid(20_000, 4)
    rng = np.random.default_rng(1)
    bases, offs = make_reads(codes, 40, rng, lmin=10, lmax=30, planted=0.0)
    E = np.full(40, 50, np.uint16)  # T <= 0: every bin passes
    r2 = synth.pack2bit(codes)
    bank = grim.grim_build_bank(dev(r2), 20_000, 5, 100, 50)
    res = grim.grim_scan(bank, dev(bases), dev(offs), dev(E), cap=1000)
    st, flags = grim.grim_bank_status(bank)
    assert st == grim.GRIM_EOVERFLOW and flags == grim.GRIM_FLAG_OVERFLOW
    assert res.n_pairs == 40 * bank.n_bins
    pr, pb = host(res.pair_read[:1000], np.uint32), host(res.pair_bin[:1000], np.uint32)
    assert pr.max() < 40 and pb.max() < bank.n_bins
    assert len(set(zip(pr.tolist(), pb.tolist()))) == 1000
    bank.free()


def test_scan_agrees_with_gather_on_candidates(oracle):
    w = synth.gather_iid(ref_len=300_000, n_reads=2000, k=16)
    bank = grim.grim_build_bank(dev(w.ref2bit), w.ref_len, w.q, w.bin_len, w.overlap)
    p = host(grim.grim_filter(bank, dev(w.bases), dev(w.read_offsets), dev(w.cand_bins), dev(w.cand_offsets),
                              dev(w.E)), np.uint8)
    res = grim.grim_scan(bank, dev(w.bases), dev(w.read_offsets), dev(w.E))
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    pr, pb, _ = gpu_pairs(res)
    passing = set(zip(pr.tolist(), pb.tolist()))
    read_of = np.repeat(np.arange(w.n_reads), np.diff(w.cand_offsets))
    want = np.array([(int(r), int(b)) in passing for r, b in zip(read_of, w.cand_bins)], dtype=np.uint8)
    assert np.array_equal(p, want)
    bank.free()


def test_scan_bad_reads_never_pass(oracle):
    codes = synth.ref_iid(20_000, 6)
    rng = np.random.default_rng(2)
    bases, offs = make_reads(codes, 64, rng, lmin=50, lmax=80, planted=1.0, sub=0.0)
    bases[offs[5] + 3] = 7
    E = np.full(64, 2, np.uint16)
    r2 = synth.pack2bit(codes)
    bank = grim.grim_build_bank(dev(r2), 20_000, 5, 100, 90)
    res = grim.grim_scan(bank, dev(bases), dev(offs), dev(E), with_read_pass=True)
    st, flags = grim.grim_bank_status(bank)
    assert st == grim.GRIM_EDATA and flags == grim.GRIM_FLAG_BAD_BASE
    rp = host(res.read_pass[:64], np.uint32)
    assert rp[5] == 0 and rp.sum() > 0
    bank.free()


def test_scan_3gbp_batch_sampled(oracle):
    """3.1 Gbp repeat-rich reference (12.1M bins), one batch of 65,536 x 100 bp
    reads: the launch bench.py times, checked on sampled pairs, sampled
    reads x bins, and per-read counts."""
    w = synth.fullscan()
    bank = grim.grim_build_bank(dev(w.ref2bit), w.ref_len, w.q, w.bin_len, w.overlap)
    res = grim.grim_scan(bank, dev(w.bases), dev(w.read_offsets), dev(w.E), cap=1 << 24, with_read_pass=True)
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    n = res.n_pairs
    assert 0 < n <= 1 << 24
    pr = host(res.pair_read[:n], np.uint32)
    pb = host(res.pair_bin[:n], np.uint32)
    ps = host(res.pair_sum[:n], np.uint16)
    rp = host(res.read_pass[:w.n_reads], np.uint32)
    assert np.array_equal(np.bincount(pr, minlength=w.n_reads).astype(np.uint32), rp)
    key = pr.astype(np.int64) * w.n_bins + pb
    assert len(np.unique(key)) == n  # each pair once
    T = (100 - w.q + 1) - w.q * int(w.E[0])
    rng = np.random.default_rng(9)
    row_cache = {}

    def row(b):
        if b not in row_cache:
            row_cache[b] = oracle.bin_row(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap, int(b))
        return row_cache[b]

    for i in rng.integers(0, n, 300):  # every reported pair is a pass with the oracle's sum
        read = w.bases[w.read_offsets[pr[i]]:w.read_offsets[pr[i] + 1]]
        s = oracle.sum_one(row(pb[i]), w.q, read)
        assert s == ps[i] and s >= T
    got = set(key.tolist())
    for r in rng.integers(0, w.n_reads, 4):  # sampled bins of sampled reads: nothing missed, nothing extra
        read = w.bases[w.read_offsets[r]:w.read_offsets[r + 1]]
        true_bin = int(w.starts[r] // w.bin_len)
        bins = set(range(max(0, true_bin - 20), min(w.n_bins, true_bin + 21)))
        bins |= set(rng.integers(0, w.n_bins, 1500).tolist())
        for b in bins:
            passes = oracle.sum_one(row(b), w.q, read) >= T
            assert passes == ((int(r) * w.n_bins + b) in got), (r, b)
    bank.free()


def test_bounded_wait_gives_up_and_the_context_survives(oracle):
    # the scan's mbarrier wait on a barrier that nothing completes: it must
    # give up after its limit with GRIM_ETIMEOUT, not hang, and leave the
    # context usable (a scan right after still matches the oracle)
    import time
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert grim.grim_wait_selfcheck(100_000_000) == grim.GRIM_ETIMEOUT
    dt = time.perf_counter() - t0
    assert 0.1 <= dt < 5.0, dt
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    codes = synth.ref_iid(50_000, 6)
    bases, offs = make_reads(codes, 64, rng, lmax=150)
    check_scan(oracle, codes, 5, 128, 100, bases, offs, np.full(64, 3, np.uint16))
