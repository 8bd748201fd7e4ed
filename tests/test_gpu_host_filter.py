"""GPU parity of grim_filter_host (the filter called with host buffers,
chunks copied in and out on overlapping streams) against the oracle, for
every chunking, page-locked and pageable buffers, and offsets that do not
start at 0."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1711_01177_gb300 as grim
import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    grim.build()
    grim.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def host(a, pinned):
    a = np.ascontiguousarray(a)
    view = {np.dtype(np.uint32): np.int32, np.dtype(np.uint16): np.int16}.get(a.dtype)
    t = torch.from_numpy(a.view(view) if view else a)
    return t.pin_memory() if pinned else t.clone()


@pytest.fixture(scope="module")
def work(oracle):
    w = synth.gather_iid(ref_len=1_000_000, n_reads=10_000, k=32)
    ob = oracle.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    op, _ = oracle.filter(ob, w.q, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, w.E)
    bank = grim.grim_build_bank(dev(w.ref2bit), w.ref_len, w.q, w.bin_len, w.overlap)
    yield w, op, bank
    bank.free()


@pytest.mark.parametrize("chunk,pinned", [(0, True), (1000, True), (3333, False), (1, True), (10_005, False)])
def test_host_filter_matches_oracle(work, chunk, pinned):
    w, op, bank = work
    ins = [host(w.bases, pinned), host(w.read_offsets, pinned), host(w.cand_bins, pinned),
           host(w.cand_offsets, pinned), host(w.E, pinned)]
    out = torch.full((w.n_checks,), 0xAA, dtype=torch.uint8)
    out = out.pin_memory() if pinned else out
    grim.grim_filter_host(bank, *ins, pass_out=out, chunk_reads=chunk)
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    assert np.array_equal(out.numpy(), op)


def test_host_filter_offsets_not_from_zero(work):
    """Reads 1,234.. with their absolute candidate offsets: pass bytes land at
    the same absolute positions as grim_filter's."""
    w, op, bank = work
    r0 = 1234
    ins = [host(w.bases, True), host(w.read_offsets[r0:], True), host(w.cand_bins, True),
           host(w.cand_offsets[r0:], True), host(w.E[r0:], True)]
    out = torch.full((w.n_checks,), 0xAA, dtype=torch.uint8).pin_memory()
    grim.grim_filter_host(bank, *ins, pass_out=out, chunk_reads=700)
    c0 = int(w.cand_offsets[r0])
    assert np.array_equal(out.numpy()[c0:], op[c0:])
    assert (out.numpy()[:c0] == 0xAA).all()


def test_host_filter_rejects_a_chunk_whose_offsets_run_backwards(work):
    w, _, bank = work
    off = w.read_offsets.copy()
    off[2000] = off[1000] - 5  # the chunk of reads 1,000-1,999 would end before it starts
    out = torch.empty(w.n_checks, dtype=torch.uint8)
    with pytest.raises(grim.GrimError) as e:
        grim.grim_filter_host(bank, host(w.bases, False), host(off, False), host(w.cand_bins, False),
                              host(w.cand_offsets, False), host(w.E, False), pass_out=out, chunk_reads=1000)
    assert e.value.status == grim.GRIM_EINVAL


def test_host_filter_from_two_threads(work):
    """Two host threads at once, each on its own stream: one call takes the
    device's cached copy streams, the other makes its own; both give the
    oracle's bytes, and repeated calls reuse the cached set."""
    import threading
    w, op, bank = work
    ins = [host(w.bases, True), host(w.read_offsets, True), host(w.cand_bins, True),
           host(w.cand_offsets, True), host(w.E, True)]
    outs = [torch.full((w.n_checks,), 0xAA, dtype=torch.uint8).pin_memory() for _ in range(4)]
    errors = []

    def run(k):
        try:
            s = torch.cuda.Stream()
            for rep in range(2):
                grim.grim_filter_host(bank, *ins, pass_out=outs[2 * k + rep], chunk_reads=997, stream=s)
        except Exception as e:  # reported below
            errors.append(e)

    th = [threading.Thread(target=run, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    for o in outs:
        assert np.array_equal(o.numpy(), op)
