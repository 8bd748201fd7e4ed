"""GPU parity of the steps either side of the filter: the seed location
table, candidate bins from exact seed locations (Sec. 1 Fig. 1, Sec. 3.3)
and the Seed Location Checker (Sec. 3.3, Fig. 4), bit-exact against the
oracle; at 3.1 Gbp against the synthetic generator's independent
implementation (itself pinned to the oracle on the CPU) for every read and
against the oracle for sampled reads."""
import ctypes

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


def key_pos_pairs(offsets, positions):
    """(key, position) of every table entry, sorted: the table's content
    independent of the order of positions within a key."""
    nk = len(offsets) - 1
    keys = np.repeat(np.arange(nk, dtype=np.int64), np.diff(offsets.astype(np.int64)))
    order = np.lexsort((positions.astype(np.int64), keys))
    return keys[order], positions.astype(np.int64)[order]


@pytest.mark.parametrize("n,k", [(1_000_000, 12), (20_000, 5), (300_000, 13), (40, 3)])
def test_index_matches_generator(n, k):
    codes = synth.ref_with_repeats(n, 5 + k, 0.3 if n > 50_000 else 0.0, n_fam=20, fam_min=100, fam_max=2000)
    idx = grim.grim_seed_index_build(dev(synth.pack2bit(codes)), n, k)
    torch.cuda.synchronize()
    off = host(idx.offsets(), np.uint32)
    pos = host(idx.positions(), np.uint32)
    want_off, want_pos = synth.seed_index(codes, k)
    assert np.array_equal(off, want_off)
    gk, gp = key_pos_pairs(off, pos)
    wk, wp = key_pos_pairs(want_off, want_pos)
    assert np.array_equal(gk, wk) and np.array_equal(gp, wp)
    idx.free()


def seed_reads(codes, n_reads, seed, lmin=100, lmax=100):
    off = synth.read_offsets(n_reads, lmin, lmax, seed)
    bases, starts = synth.reads(codes, off, seed, 0.03, 0.01)
    return bases, off, starts


def with_odd_reads(bases, off):
    """Append reads with a non-base code, shorter than a seed, and empty."""
    extra = [np.concatenate([bases[off[0]:off[0] + 30], [4], bases[off[1]:off[1] + 40]]).astype(np.uint8),
             bases[off[2]:off[2] + 7].copy(), np.zeros(0, np.uint8), bases[off[3]:off[3] + 24].copy()]
    b = np.concatenate([bases] + extra).astype(np.uint8)
    o = np.concatenate([off, off[-1] + np.cumsum([len(x) for x in extra])]).astype(np.int64)
    return b, o


@pytest.mark.parametrize("cap", [3, 50, 10_000])
def test_candidates_match_oracle(oracle, cap):
    n = 1_000_000
    codes = synth.ref_with_repeats(n, 21, 0.3, n_fam=40, fam_min=200, fam_max=4000)
    bases, off, _ = seed_reads(codes, 4000, 21, 20, 300)
    bases, off = with_odd_reads(bases, off)
    n_bins = -(-n // 256)
    idx = grim.grim_seed_index_build(dev(synth.pack2bit(codes)), n, 12)
    cb, co = grim.grim_seed_candidates(idx, dev(bases), dev(off), 256, n_bins, cap)
    ocb, oco = oracle.seed_candidates(codes, 12, bases, off, 256, n_bins, cap)
    assert np.array_equal(host(co, np.int64), oco)
    assert np.array_equal(host(cb, np.uint32), ocb)
    idx.free()


@pytest.mark.parametrize("k,cap", [(4, 7), (6, 1000), (15, 100)])
def test_small_k_many_votes(oracle, k, cap):
    n = 30_000
    codes = synth.ref_iid(n, 31)
    bases, off, _ = seed_reads(codes, 300, 31, 5, 80)
    n_bins = -(-n // 100)
    idx = grim.grim_seed_index_build(dev(synth.pack2bit(codes)), n, k)
    cb, co = grim.grim_seed_candidates(idx, dev(bases), dev(off), 100, n_bins, cap)
    ocb, oco = oracle.seed_candidates(codes, k, bases, off, 100, n_bins, cap)
    assert np.array_equal(host(co, np.int64), oco) and np.array_equal(host(cb, np.uint32), ocb)
    idx.free()


def test_reads_beyond_shared_memory_sort(oracle):
    """A 12-mer planted 12,000 times: reads carrying it at several seed
    offsets collect > 8,192 votes and take the global-memory sort."""
    rng = np.random.default_rng(41)
    n = 1_300_000
    codes = synth.ref_iid(n, 41)
    motif = rng.integers(0, 4, 12).astype(np.uint8)
    for p in rng.choice(n // 100 - 1, 12_000, replace=False) * 100 + 7:
        codes[p:p + 12] = motif
    reads = []
    for r in range(40):
        rd = rng.integers(0, 4, 100).astype(np.uint8)
        for o in range(0, 96, 12)[: 1 + r % 8]:
            rd[o:o + 12] = motif
        reads.append(rd)
    bases = np.concatenate(reads)
    off = np.arange(0, 41 * 100, 100, dtype=np.int64)
    n_bins = -(-n // 256)
    idx = grim.grim_seed_index_build(dev(synth.pack2bit(codes)), n, 12)
    for cap in (100, 5000, 100_000):
        cb, co = grim.grim_seed_candidates(idx, dev(bases), dev(off), 256, n_bins, cap)
        ocb, oco = oracle.seed_candidates(codes, 12, bases, off, 256, n_bins, cap)
        assert np.array_equal(host(co, np.int64), oco) and np.array_equal(host(cb, np.uint32), ocb)
    # read 39 carries the motif at 8 seeds: 96,000 votes, past the shared-memory sort
    assert np.diff(oco)[39] > 1000
    idx.free()


def test_crowded_bin_takes_the_radix_sort(oracle):
    """A 600-base poly-A stretch: a poly-A read's 8 seeds each hit ~590
    positions in two or three bins, so one bin collects several hundred of
    the read's ~4,700 votes.  Reads of that kind (one with 3 seeds, ~1,770
    votes, within shared memory) are sorted by the radix sort instead of the
    bucket sort; the lists must still match the oracle's."""
    rng = np.random.default_rng(43)
    n = 200_000
    codes = synth.ref_iid(n, 43)
    codes[50_000:50_600] = 0
    reads = [np.zeros(36, np.uint8), np.zeros(100, np.uint8), rng.integers(0, 4, 100).astype(np.uint8),
             codes[120_000:120_100].copy()]
    bases = np.concatenate(reads)
    off = np.concatenate([[0], np.cumsum([len(x) for x in reads])]).astype(np.int64)
    n_bins = -(-n // 256)
    idx = grim.grim_seed_index_build(dev(synth.pack2bit(codes)), n, 12)
    for cap in (2, 10_000):
        cb, co = grim.grim_seed_candidates(idx, dev(bases), dev(off), 256, n_bins, cap)
        ocb, oco = oracle.seed_candidates(codes, 12, bases, off, 256, n_bins, cap)
        assert np.array_equal(host(co, np.int64), oco) and np.array_equal(host(cb, np.uint32), ocb)
    idx.free()


def test_overflow_is_reported_then_retried(oracle):
    n = 200_000
    codes = synth.ref_with_repeats(n, 51, 0.3, n_fam=10, fam_min=100, fam_max=2000)
    bases, off, _ = seed_reads(codes, 500, 51)
    n_bins = -(-n // 256)
    idx = grim.grim_seed_index_build(dev(synth.pack2bit(codes)), n, 12)
    ocb, oco = oracle.seed_candidates(codes, 12, bases, off, 256, n_bins, 1000)
    small = torch.empty(10, dtype=torch.int32, device="cuda")
    co = torch.empty(len(off), dtype=torch.int64, device="cuda")
    b_d, o_d = dev(bases), dev(off)  # held until the call has finished
    total = ctypes.c_int64()
    st = grim.load().grim_seed_candidates(idx.handle, ctypes.c_void_p(b_d.data_ptr()),
                                          ctypes.c_void_p(o_d.data_ptr()), len(off) - 1, 256, n_bins, 1000,
                                          ctypes.c_void_p(small.data_ptr()), 10, ctypes.c_void_p(co.data_ptr()),
                                          ctypes.byref(total), grim._stream_ptr(None))
    torch.cuda.synchronize()
    assert st == grim.GRIM_EOVERFLOW and total.value == len(ocb)
    assert np.array_equal(host(co, np.int64), oco) and np.array_equal(host(small, np.uint32), ocb[:10])
    cb, co2 = grim.grim_seed_candidates(idx, dev(bases), dev(off), 256, n_bins, 1000, capacity=16)
    assert np.array_equal(host(cb, np.uint32), ocb)
    idx.free()


def test_candidates_3gbp_match_generator(oracle):
    """3.1 Gbp reference with 40% repeats, 65,536 x 100 bp reads, 12-mer
    seeds capped at 10,000: the full table on the GPU against the
    generator's lists (restricted CPU index, radix sorts) for every read,
    and against the oracle itself (one pass over the whole reference) for
    200 sampled reads."""
    w = synth.mixed_seeds()
    idx = grim.grim_seed_index_build(dev(w.ref2bit), w.ref_len, 12)
    cb, co = grim.grim_seed_candidates(idx, dev(w.bases), dev(w.read_offsets), w.bin_len, w.n_bins, 10_000,
                                       capacity=int(w.n_checks))
    gco, gcb = host(co, np.int64), host(cb, np.uint32)
    assert np.array_equal(gco, w.cand_offsets)
    assert np.array_equal(gcb, w.cand_bins)
    idx.free()
    sample = np.arange(0, w.n_reads, w.n_reads // 200)[:200]
    ro = w.read_offsets
    s_bases = np.concatenate([w.bases[ro[r]:ro[r + 1]] for r in sample])
    s_offs = np.concatenate([[0], np.cumsum([ro[r + 1] - ro[r] for r in sample])]).astype(np.int64)
    ocb, oco = oracle.seed_candidates(w.codes, 12, s_bases, s_offs, w.bin_len, w.n_bins, 10_000)
    for i, r in enumerate(sample):
        assert np.array_equal(gcb[gco[r]:gco[r + 1]], ocb[oco[i]:oco[i + 1]]), r
    assert oco[-1] > 0


def test_locate_matches_oracle(oracle):
    w = synth.gather_iid(ref_len=300_000, n_reads=3000, k=16)
    bank = grim.grim_build_bank(dev(w.ref2bit), w.ref_len, w.q, w.bin_len, w.overlap)
    rng = np.random.default_rng(61)
    ps = (rng.random(w.n_checks) < 0.2).astype(np.uint8)
    ps[-1] = 1  # the last bin's span is clipped at the reference end
    cb = w.cand_bins.copy()
    cb[-1] = bank.n_bins - 1
    stride = w.bin_len + w.overlap + 5
    loc = grim.grim_locate(bank, dev(cb), dev(w.cand_offsets), dev(ps), ref2bit=dev(w.ref2bit), seg_stride=stride)
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    rd, bn, be, en, seg = oracle.locate(ps, cb, w.cand_offsets, w.codes, w.bin_len, w.overlap, stride)
    assert loc.n == len(rd)
    assert np.array_equal(host(loc.read, np.uint32), rd) and np.array_equal(host(loc.bin, np.uint32), bn)
    assert np.array_equal(host(loc.begin, np.int64), be) and np.array_equal(host(loc.end, np.int64), en)
    assert np.array_equal(loc.segments.cpu().numpy(), seg)
    # a short output: the count is complete, the first rows are written
    part = grim.grim_locate(bank, dev(cb), dev(w.cand_offsets), dev(ps), capacity=100)
    assert part.n == len(rd) and np.array_equal(host(part.bin, np.uint32), bn[:100])
    # no passing byte
    none = grim.grim_locate(bank, dev(cb), dev(w.cand_offsets), dev(np.zeros_like(ps)))
    assert none.n == 0
    bank.free()


def test_chain_index_candidates_filter_locate(oracle):
    """The mapper's path around the filter, all on the GPU, against the same
    chain of oracle steps."""
    n = 500_000
    codes = synth.ref_with_repeats(n, 71, 0.3, n_fam=30, fam_min=200, fam_max=3000)
    bases, off, _ = seed_reads(codes, 2000, 71)
    r2 = synth.pack2bit(codes)
    E = np.full(len(off) - 1, 5, np.uint16)
    bank = grim.grim_build_bank(dev(r2), n, 5, 256, 100)
    idx = grim.grim_seed_index_build(dev(r2), n, 12)
    cb, co = grim.grim_seed_candidates(idx, dev(bases), dev(off), 256, bank.n_bins, 1000)
    ps = grim.grim_filter(bank, dev(bases), dev(off), cb, co, dev(E))
    loc = grim.grim_locate(bank, cb, co, ps, ref2bit=dev(r2), seg_stride=356)
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    ocb, oco = oracle.seed_candidates(codes, 12, bases, off, 256, bank.n_bins, 1000)
    ob = oracle.build_bank(r2, n, 5, 256, 100)
    ops, _ = oracle.filter(ob, 5, bases, off, ocb, oco, E)
    rd, bn, be, en, seg = oracle.locate(ops, ocb, oco, codes, 256, 100, 356)
    assert np.array_equal(host(loc.read, np.uint32), rd) and np.array_equal(host(loc.bin, np.uint32), bn)
    assert np.array_equal(loc.segments.cpu().numpy(), seg)
    assert 0 < loc.n < len(ocb)
    bank.free()
    idx.free()
