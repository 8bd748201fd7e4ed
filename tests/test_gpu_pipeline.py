"""GPU parity of grim_map, the overlapped pipeline around the filter
(Sec. 4.2 / 6.1): every passing location with its edit distance equals the
chain of oracle steps - seed candidates, filter, Seed Location Checker,
Sellers distance - whatever the batch size and stream arrangement."""
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


def oracle_chain(oracle, codes, q, bin_len, overlap, k, bases, off, E, cap):
    n = len(codes)
    n_bins = -(-n // bin_len)
    cb, co = oracle.seed_candidates(codes, k, bases, off, bin_len, n_bins, cap)
    ob = oracle.build_bank(synth.pack2bit(codes), n, q, bin_len, overlap)
    ps, _ = oracle.filter(ob, q, bases, off, cb, co, E)
    rd, bn, be, en, _ = oracle.locate(ps, cb, co, codes, bin_len, overlap)
    dist = [oracle.sellers(bases[off[r]:off[r + 1]], codes[b0:b1]) for r, b0, b1 in zip(rd, be, en)]
    return rd, bn, np.array(dist, np.uint16)


@pytest.mark.parametrize("k,cap,batch,own_stream", [(12, 1000, 700, True), (12, 1000, 0, False), (5, 1000, 150, False)])
def test_map_matches_oracle_chain(oracle, k, cap, batch, own_stream):
    n = 500_000 if k > 6 else 200_000
    codes = synth.ref_with_repeats(n, 91, 0.3, n_fam=30, fam_min=200, fam_max=3000)
    n_reads = 3000 if k > 6 else 600
    off = synth.read_offsets(n_reads, 50, 200, 91)
    bases, _ = synth.reads(codes, off, 91, 0.03, 0.01)
    E = synth.E_rate(off)
    r2 = dev(synth.pack2bit(codes))
    bank = grim.grim_build_bank(r2, n, 5, 256, 100)
    idx = grim.grim_seed_index_build(r2, n, k)
    align = torch.cuda.Stream() if own_stream else None
    m = grim.grim_map(bank, idx, r2, dev(bases), dev(off), dev(E), cap=cap, batch_reads=batch, align_stream=align)
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    rd, bn, dist = oracle_chain(oracle, codes, 5, 256, 100, k, bases, off, E, cap)
    assert m.n == len(rd) > 0
    assert np.array_equal(host(m.read, np.uint32), rd)
    assert np.array_equal(host(m.bin, np.uint32), bn)
    assert np.array_equal(host(m.dist, np.uint16), dist)
    assert (dist <= E[rd]).sum() > 0  # some passing locations map
    bank.free()
    idx.free()


def test_map_output_overflow(oracle):
    n = 300_000
    codes = synth.ref_with_repeats(n, 93, 0.3, n_fam=20, fam_min=200, fam_max=3000)
    off = synth.read_offsets(1000, 100, 100, 93)
    bases, _ = synth.reads(codes, off, 93, 0.03, 0.01)
    E = np.full(1000, 5, np.uint16)
    r2 = dev(synth.pack2bit(codes))
    bank = grim.grim_build_bank(r2, n, 5, 256, 100)
    idx = grim.grim_seed_index_build(r2, n, 12)
    full = grim.grim_map(bank, idx, r2, dev(bases), dev(off), dev(E), batch_reads=300)
    b_d, o_d, e_d = dev(bases), dev(off), dev(E)
    out = [torch.empty(16, dtype=t, device="cuda") for t in (torch.int32, torch.int32, torch.int16)]
    total = ctypes.c_int64()
    st = grim.load().grim_map(bank.handle, idx.handle, ctypes.c_void_p(r2.data_ptr()),
                              ctypes.c_void_p(b_d.data_ptr()), ctypes.c_void_p(o_d.data_ptr()), 1000,
                              ctypes.c_void_p(e_d.data_ptr()), 10_000, 300,
                              *[ctypes.c_void_p(t.data_ptr()) for t in out],
                              16, ctypes.byref(total), grim._stream_ptr(None), None)
    torch.cuda.synchronize()
    assert st == grim.GRIM_EOVERFLOW and total.value == full.n > 16
    assert torch.equal(out[0], full.read[:16]) and torch.equal(out[1], full.bin[:16])
    assert torch.equal(out[2], full.dist[:16])
    bank.free()
    idx.free()
