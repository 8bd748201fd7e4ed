"""GPU parity of the batched persistent gather (grim_filter_batched) and its
autotuner: every launch shape, multi-batch splits, graph capture and replay
give the oracle's bytes."""
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


def tune(**kw):
    t = grim.GrimTune()
    for k, v in kw.items():
        setattr(t, k, v)
    return t


def small_varlen(q, n_reads=3000, k_max=800):
    return synth.batched_varlen(ref_len=1_000_000, n_reads=n_reads, q=q, k_max=k_max)


@pytest.mark.parametrize("q", [5, 6])
def test_batched_every_shape_matches_oracle(oracle, q):
    w = small_varlen(q)
    bank = grim.grim_build_bank(dev(w.ref2bit), w.ref_len, w.q, w.bin_len, w.overlap)
    ob = oracle.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    op, os_ = oracle.filter(ob, w.q, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, w.E)
    args = [dev(w.bases), dev(w.read_offsets), dev(w.cand_bins), dev(w.cand_offsets), dev(w.E)]
    stream = torch.cuda.Stream()
    shapes = [tune(), tune(warps_per_cta=4), tune(reads_per_claim=16), tune(ctas_per_sm=1),
              tune(batch_reads=700), tune(batch_reads=700, use_graph=1, warps_per_cta=4, reads_per_claim=4),
              tune(use_graph=1)]
    for t in shapes:
        sums = torch.zeros(w.n_checks, dtype=torch.int16, device="cuda")
        with torch.cuda.stream(stream):
            p = grim.grim_filter_batched(bank, *args, sums=sums, tune=t, stream=stream)
        stream.synchronize()
        assert grim.grim_bank_status(bank, stream) == (grim.GRIM_OK, 0)
        assert np.array_equal(host(p, np.uint8), op), t.as_dict()
        assert np.array_equal(host(sums, np.uint16), os_.astype(np.uint16)), t.as_dict()
    bank.free()


def test_batched_graph_replay_reads_current_inputs(oracle):
    w = small_varlen(6, n_reads=2000)
    bank = grim.grim_build_bank(dev(w.ref2bit), w.ref_len, w.q, w.bin_len, w.overlap)
    ob = oracle.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    args = [dev(w.bases), dev(w.read_offsets), dev(w.cand_bins), dev(w.cand_offsets), dev(w.E)]
    out = torch.empty(w.n_checks, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    t = tune(use_graph=1, batch_reads=500)
    for step in range(3):
        E = (w.E + step).astype(np.uint16)
        args[4].copy_(dev(E))  # same buffer, new contents: the replayed graph must see them
        with torch.cuda.stream(stream):
            grim.grim_filter_batched(bank, *args, pass_out=out, tune=t, stream=stream)
        stream.synchronize()
        op, _ = oracle.filter(ob, w.q, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, E)
        assert np.array_equal(host(out, np.uint8), op), step
    assert grim.grim_bank_status(bank, stream) == (grim.GRIM_OK, 0)
    bank.free()


def test_batched_inside_a_caller_graph(oracle):
    w = small_varlen(5, n_reads=1500)
    bank = grim.grim_build_bank(dev(w.ref2bit), w.ref_len, w.q, w.bin_len, w.overlap)
    args = [dev(w.bases), dev(w.read_offsets), dev(w.cand_bins), dev(w.cand_offsets), dev(w.E)]
    out = torch.zeros(w.n_checks, dtype=torch.uint8, device="cuda")
    t = tune(use_graph=1, batch_reads=400)
    grim.grim_filter_batched(bank, *args, pass_out=out, tune=t)  # warm-up outside capture
    torch.cuda.synchronize()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        grim.grim_filter_batched(bank, *args, pass_out=out, tune=t)
    torch.cuda.synchronize()
    assert out.sum().item() == 0  # captured, not run
    g.replay()
    torch.cuda.synchronize()
    ob = oracle.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    op, _ = oracle.filter(ob, w.q, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, w.E)
    assert np.array_equal(host(out, np.uint8), op)
    bank.free()


def test_autotune_then_default_tune(oracle):
    w = small_varlen(6, n_reads=4000)
    bank = grim.grim_build_bank(dev(w.ref2bit), w.ref_len, w.q, w.bin_len, w.overlap)
    args = [dev(w.bases), dev(w.read_offsets), dev(w.cand_bins), dev(w.cand_offsets), dev(w.E)]
    t = grim.grim_autotune(bank, *args)
    assert t.warps_per_cta in (4, 8) and t.reads_per_claim in (1, 4, 16) and t.ctas_per_sm in (0, 2)
    assert t.use_graph == 1 and t.batch_reads == 262144
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        p = grim.grim_filter_batched(bank, *args, stream=stream)
    stream.synchronize()
    ob = oracle.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    op, _ = oracle.filter(ob, w.q, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, w.E)
    assert np.array_equal(host(p, np.uint8), op)
    bank.free()


def test_batched_100mbp_q6_2m_reads_sampled(oracle):
    """100 Mbp repeat-rich reference, q=6, 2M reads of 50-300 bp, log-uniform
    candidate lists (1-5,000): the full launch, checked on sampled pairs."""
    w = synth.batched_varlen()
    bank = grim.grim_build_bank(dev(w.ref2bit), w.ref_len, w.q, w.bin_len, w.overlap)
    sums = torch.empty(w.n_checks, dtype=torch.int16, device="cuda")
    stream = torch.cuda.Stream()
    args = [dev(w.bases), dev(w.read_offsets), dev(w.cand_bins), dev(w.cand_offsets), dev(w.E)]
    with torch.cuda.stream(stream):
        p = grim.grim_filter_batched(bank, *args, sums=sums, tune=tune(use_graph=1), stream=stream)
    stream.synchronize()
    assert grim.grim_bank_status(bank, stream) == (grim.GRIM_OK, 0)
    p, s = host(p, np.uint8), host(sums, np.uint16)
    del args
    rng = np.random.default_rng(77)
    read_of = np.searchsorted(w.cand_offsets, np.arange(w.n_checks), side="right") - 1
    for c in rng.integers(0, w.n_checks, 1500):
        r = int(read_of[c])
        row = oracle.bin_row(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap, int(w.cand_bins[c]))
        read = w.bases[w.read_offsets[r]:w.read_offsets[r + 1]]
        want = oracle.sum_one(row, w.q, read)
        assert s[c] == want
        assert p[c] == int(want >= oracle.threshold(len(read), w.q, int(w.E[r])))
    L = np.diff(w.read_offsets)
    T = (L - w.q + 1) - w.q * w.E.astype(np.int64)
    assert np.array_equal(p, (s.astype(np.int64) >= np.repeat(T, np.diff(w.cand_offsets))).astype(np.uint8))
    bank.free()
