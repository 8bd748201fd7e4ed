"""GPU parity of the verification side (the aligner's check behind Sec. 5's
metrics): grim_verify's semi-global edit distances against the oracle's
Sellers recurrence, element by element; grim_verify_stats against direct
counts; and the paper's zero-miss guarantee - no location whose read maps
within E edits into the bin's span is rejected - over every candidate."""
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


def span(codes, b, bin_len, overlap):
    s = b * bin_len
    return codes[s:min(len(codes), s + bin_len + overlap)]


def test_distances_match_oracle_at_every_block_boundary(oracle):
    """Reads of 0-512 bases (around each 64-row block boundary), some copied
    from their bin with edits, some random, some with a non-base code;
    bins everywhere including the clipped last one."""
    n = 60_000
    codes = synth.ref_iid(n, 3)
    bin_len, overlap = 256, 300
    n_bins = -(-n // bin_len)
    rng = np.random.default_rng(3)
    lens = [0, 1, 5, 63, 64, 65, 100, 127, 128, 129, 150, 191, 192, 193, 255, 256, 257, 300, 383, 384, 385,
            448, 511, 512]
    reads, loc_r, loc_b = [], [], []
    for r, L in enumerate(lens * 3):
        b = int(rng.integers(0, n_bins))
        sp = span(codes, b, bin_len, overlap)
        if r % 3 == 0 and L <= len(sp):  # a copy of part of the span with a few edits
            o = int(rng.integers(0, len(sp) - L + 1))
            rd = sp[o:o + L].copy()
            for _ in range(int(rng.integers(0, 6))):
                if L:
                    rd[int(rng.integers(0, L))] = rng.integers(0, 4)
        else:
            rd = rng.integers(0, 4, L).astype(np.uint8)
        if r % 7 == 3 and L:
            rd[int(rng.integers(0, L))] = 4
        reads.append(rd.astype(np.uint8))
        for bb in {b, n_bins - 1, int(rng.integers(0, n_bins))}:
            loc_r.append(r)
            loc_b.append(bb)
    off = np.concatenate([[0], np.cumsum([len(x) for x in reads])]).astype(np.int64)
    bases = np.concatenate(reads).astype(np.uint8)
    bank = grim.grim_build_bank(dev(synth.pack2bit(codes)), n, 5, bin_len, overlap)
    lr, lb = np.array(loc_r, np.uint32), np.array(loc_b, np.uint32)
    d = host(grim.grim_verify(bank, dev(synth.pack2bit(codes)), dev(bases), dev(off), dev(lr), dev(lb)), np.uint16)
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    want = [oracle.sellers(bases[off[r]:off[r + 1]], span(codes, b, bin_len, overlap)) for r, b in zip(lr, lb)]
    assert d.tolist() == want
    bank.free()


def test_long_read_and_bad_ids_are_flagged(oracle):
    n = 20_000
    codes = synth.ref_iid(n, 4)
    r2 = synth.pack2bit(codes)
    bank = grim.grim_build_bank(dev(r2), n, 5, 256, 100)
    reads = np.concatenate([codes[:513], codes[1000:1100]]).astype(np.uint8)
    off = np.array([0, 513, 613], np.int64)
    lr = np.array([0, 1, 1, 5], np.uint32)
    lb = np.array([0, 3, bank.n_bins, 3], np.uint32)
    d = host(grim.grim_verify(bank, dev(r2), dev(reads), dev(off), dev(lr), dev(lb)), np.uint16)
    st, flags = grim.grim_bank_status(bank)
    assert st == grim.GRIM_EDATA
    assert flags == grim.GRIM_FLAG_LONG_READ | grim.GRIM_FLAG_BAD_BIN | grim.GRIM_FLAG_BAD_OFFSETS
    assert d[0] == 0xFFFF and d[2] == 0xFFFF and d[3] == 0xFFFF
    assert d[1] == oracle.sellers(reads[513:], span(codes, 3, 256, 100))
    bank.free()


def test_zero_miss_and_false_negative_rate_over_every_candidate(oracle):
    """Seed candidates -> filter -> verify every candidate: no candidate
    whose read maps into its span within E edits is rejected, and the counts
    agree with the distances and pass bytes."""
    n = 500_000
    codes = synth.ref_with_repeats(n, 81, 0.3, n_fam=30, fam_min=200, fam_max=3000)
    off = synth.read_offsets(3000, 100, 100, 81)
    bases, _ = synth.reads(codes, off, 81, 0.03, 0.01)
    r2 = synth.pack2bit(codes)
    E = np.full(len(off) - 1, 5, np.uint16)
    bank = grim.grim_build_bank(dev(r2), n, 5, 256, 100)
    idx = grim.grim_seed_index_build(dev(r2), n, 12)
    cb, co = grim.grim_seed_candidates(idx, dev(bases), dev(off), 256, bank.n_bins, 1000)
    ps = grim.grim_filter(bank, dev(bases), dev(off), cb, co, dev(E))
    every = grim.grim_locate(bank, cb, co, torch.ones_like(ps))
    assert every.n == cb.numel()
    d = grim.grim_verify(bank, dev(r2), dev(bases), dev(off), every.read, every.bin)
    stats = grim.grim_verify_stats(d, every.read, dev(E), pass_=ps)
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    dh, ph, rh = host(d, np.uint16), host(ps, np.uint8), host(every.read, np.uint32)
    mapped = dh <= E[rh]
    assert stats == {"passed": int(ph.sum()), "passed_unmapped": int((ph.astype(bool) & ~mapped).sum()),
                     "rejected": int((ph == 0).sum()), "rejected_mapped": int((~ph.astype(bool) & mapped).sum())}
    assert stats["rejected_mapped"] == 0  # Sec. 3.5: no correct mapping is filtered out
    assert 0 < stats["passed"] and mapped.sum() > 0.5 * 3000  # reads carry ~4 edits on average, E = 5
    sample = np.random.default_rng(8).choice(len(dh), 400, replace=False)
    bins = host(every.bin, np.uint32)
    for i in sample:
        r = rh[i]
        assert dh[i] == oracle.sellers(bases[off[r]:off[r + 1]], span(codes, int(bins[i]), 256, 100))
    bank.free()
    idx.free()


def test_zero_miss_3gbp_first_reads(oracle):
    """The genome-scale mixed workload: every candidate of its first 2,048
    reads verified; none that maps is rejected; sampled distances against
    the oracle."""
    w = synth.mixed_seeds(cand_reads=2048)
    n = len(w.cand_offsets) - 1
    r2 = dev(w.ref2bit)
    bank = grim.grim_build_bank(r2, w.ref_len, w.q, w.bin_len, w.overlap)
    bases_d, off_d = dev(w.bases), dev(w.read_offsets[:n + 1])
    cb_d, co_d = dev(w.cand_bins), dev(w.cand_offsets)
    ps = grim.grim_filter(bank, bases_d, off_d, cb_d, co_d, dev(w.E[:n]))
    every = grim.grim_locate(bank, cb_d, co_d, torch.ones_like(ps))
    d = grim.grim_verify(bank, r2, bases_d, off_d, every.read, every.bin)
    stats = grim.grim_verify_stats(d, every.read, dev(w.E[:n]), pass_=ps)
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    assert stats["rejected_mapped"] == 0 and stats["passed"] > 0
    assert stats["passed"] + stats["rejected"] == len(w.cand_bins)
    dh, rh, bh = host(d, np.uint16), host(every.read, np.uint32), host(every.bin, np.uint32)
    for i in np.random.default_rng(12).choice(len(dh), 200, replace=False):
        r = rh[i]
        assert dh[i] == oracle.sellers(w.bases[w.read_offsets[r]:w.read_offsets[r + 1]],
                                       span(w.codes, int(bh[i]), w.bin_len, w.overlap))
    bank.free()
