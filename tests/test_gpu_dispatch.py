"""GPU parity of the per-batch dispatcher (grim_filter_auto): whichever form
it picks for a batch, the pass bytes equal the oracle's."""
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


def dense_workload(n_reads=10_000, ref_len=256_000, dense_frac=1.0, seed=4, dense_of=None):
    """Every bin as a candidate for the first dense_frac of the reads (or
    the reads r with dense_of(r)), 8 for the rest."""
    rng = np.random.default_rng(seed)
    codes = synth.ref_with_repeats(ref_len, seed, 0.3, n_fam=10, fam_min=100, fam_max=2000)
    off = synth.read_offsets(n_reads, 100, 100, seed)
    bases, starts = synth.reads(codes, off, seed, 0.03, 0.01)
    nb = -(-ref_len // 256)
    n_dense = int(n_reads * dense_frac)
    if dense_of is None:
        dense_of = lambda r: r < n_dense  # noqa: E731
    lists = [np.arange(nb, dtype=np.uint32) if dense_of(r) else
             np.sort(rng.choice(nb, 8, replace=False)).astype(np.uint32) for r in range(n_reads)]
    co = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int64)
    return codes, bases, off, np.concatenate(lists), co, np.full(n_reads, 5, np.uint16)


def run_auto(oracle, codes, bases, off, cb, co, E, batch_reads=262144):
    r2 = synth.pack2bit(codes)
    bank = grim.grim_build_bank(dev(r2), len(codes), 5, 256, 100)
    p, scanned = grim.grim_filter_auto(bank, dev(bases), dev(off), dev(cb), dev(co), dev(E), batch_reads=batch_reads)
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    ob = oracle.build_bank(r2, len(codes), 5, 256, 100)
    op, _ = oracle.filter(ob, 5, bases, off, cb, co, E)
    assert np.array_equal(host(p, np.uint8), op)
    forms = (grim.grim_choose_form(bank, len(off) - 1, len(cb)),)
    bank.free()
    return scanned, forms, op


def test_sparse_candidates_take_the_gather_form(oracle):
    w = synth.gather_iid(ref_len=200_000, n_reads=2000, k=8)
    scanned, forms, op = run_auto(oracle, w.codes, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, w.E)
    assert scanned == 0 and forms == (grim.GRIM_FORM_GATHER,)
    assert 0 < op.sum() < len(op)


def test_dense_candidates_take_the_scan_form(oracle):
    codes, bases, off, cb, co, E = dense_workload()
    scanned, forms, op = run_auto(oracle, codes, bases, off, cb, co, E)
    assert scanned == len(off) - 1 and forms == (grim.GRIM_FORM_SCAN,)
    assert op.sum() > 0


def test_mixed_batches_use_both_forms(oracle):
    codes, bases, off, cb, co, E = dense_workload(n_reads=8_000, ref_len=512_000, dense_frac=0.5, seed=6)
    scanned, _, _ = run_auto(oracle, codes, bases, off, cb, co, E, batch_reads=2000)
    assert scanned == 4000


def test_alternating_batches_run_gathers_between_scans(oracle):
    """Batches of 2,000 reads alternate sparse (gathered) and dense (scanned),
    two sparse batches in a row once, and the last batch is ragged: the
    gathered batches between two scans run as one launch, and every pass byte
    still equals the oracle's."""
    dense = lambda r: (r // 2000) in (1, 4)  # noqa: E731
    codes, bases, off, cb, co, E = dense_workload(n_reads=11_000, ref_len=512_000, seed=8, dense_of=dense)
    scanned, _, _ = run_auto(oracle, codes, bases, off, cb, co, E, batch_reads=2000)
    assert scanned == 4000


def test_dispatch_3gbp_mixed_sampled(oracle):
    """3.1 Gbp reference with 40% repeats at 5-20% divergence, 65,536 reads,
    12-mer seed candidates capped at 10,000: the dispatcher's launch, checked
    on sampled candidates."""
    w = synth.mixed_seeds()
    bank = grim.grim_build_bank(dev(w.ref2bit), w.ref_len, w.q, w.bin_len, w.overlap)
    p, scanned = grim.grim_filter_auto(bank, dev(w.bases), dev(w.read_offsets), dev(w.cand_bins), dev(w.cand_offsets),
                                       dev(w.E))
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    assert scanned == 0  # ~1,700 candidates per read of 12.1M bins: gathering is far cheaper
    p = host(p, np.uint8)
    rng = np.random.default_rng(5)
    read_of = np.searchsorted(w.cand_offsets, np.arange(w.n_checks), side="right") - 1
    T = (100 - w.q + 1) - w.q * 5
    for c in rng.integers(0, w.n_checks, 1500):
        r = int(read_of[c])
        row = oracle.bin_row(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap, int(w.cand_bins[c]))
        s = oracle.sum_one(row, w.q, w.bases[w.read_offsets[r]:w.read_offsets[r + 1]])
        assert p[c] == int(s >= T)
    # the true bin of nearly every read passes (reads carry ~3% substitutions and 1% indels)
    tb = (w.starts // w.bin_len).astype(np.uint32)
    hit = [p[w.cand_offsets[r] + np.searchsorted(w.cand_bins[w.cand_offsets[r]:w.cand_offsets[r + 1]], tb[r])]
           for r in range(0, w.n_reads, 64)
           if tb[r] in w.cand_bins[w.cand_offsets[r]:w.cand_offsets[r + 1]]]
    assert np.mean(hit) > 0.9
    bank.free()


def test_dispatch_3gbp_10m_reads_gpu_candidates_sampled(oracle):
    """The genome-scale mixed workload at its full 10M x 100 bp reads:
    candidates from the GPU seed table, the dispatcher over every read;
    sampled reads' candidate lists against the generator, sampled pass
    bytes against the oracle's per-check sum."""
    w = synth.mixed_seeds(n_reads=10_000_000, cand_reads=0)
    bank = grim.grim_build_bank(dev(w.ref2bit), w.ref_len, w.q, w.bin_len, w.overlap)
    idx = grim.grim_seed_index_build(dev(w.ref2bit), w.ref_len, 12)
    reads_d, offs_d = dev(w.bases), dev(w.read_offsets)
    cb, co = grim.grim_seed_candidates(idx, reads_d, offs_d, w.bin_len, w.n_bins, 10_000,
                                       capacity=w.n_reads * 2048)
    idx.free()
    p, scanned = grim.grim_filter_auto(bank, reads_d, offs_d, cb, co, dev(w.E))
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    assert scanned == 0
    rng = np.random.default_rng(9)
    sample = np.sort(rng.choice(w.n_reads, 200, replace=False))
    co_h = host(co, np.int64)
    sub_off = np.concatenate([[0], np.cumsum(np.diff(w.read_offsets)[sample])]).astype(np.int64)
    sub_bases = np.concatenate([w.bases[w.read_offsets[r]:w.read_offsets[r + 1]] for r in sample])
    want_cb, want_co = synth.cands_seeds(synth.seed_index_for_reads(w.codes, sub_bases, sub_off), sub_bases,
                                         sub_off, w.bin_len, w.n_bins, 10_000)
    for j, r in enumerate(sample):
        got = host(cb[co_h[r]:co_h[r + 1]], np.uint32)
        assert np.array_equal(got, want_cb[want_co[j]:want_co[j + 1]]), r
    T = (100 - w.q + 1) - w.q * 5
    checks = rng.integers(0, int(co_h[-1]), 1500)
    reads_of = np.searchsorted(co_h, checks, side="right") - 1
    bins = host(cb[torch.as_tensor(checks, device="cuda")], np.uint32)
    passes = host(p[torch.as_tensor(checks, device="cuda")], np.uint8)
    for c, r, b, got in zip(checks, reads_of, bins, passes):
        row = oracle.bin_row(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap, int(b))
        assert got == int(oracle.sum_one(row, w.q, w.bases[w.read_offsets[r]:w.read_offsets[r + 1]]) >= T), c
    bank.free()
