"""grim_scan_noalloc gives exactly what grim_scan gives.

grim_scan_noalloc serves callers that cannot allocate device memory when
they call the filter (their device memory belongs to their own pool, or
their footprint is fixed after start-up); it runs the same full scan in the
library's fixed scratch array instead of a cudaMallocAsync'd one.  The test
calls it through the C ABI twice in a row on different read sets - the
second call finds the first call's data in the shared scratch and must not
be affected by it - and compares each result with grim_scan's on the same
inputs: the same set of passing (read, bin) pairs, the same sums, the same
per-read counts (bit-exact, the filter's outputs are integers).  It also
checks that a request beyond the fixed scratch is rejected up front.

This file is collected last so that, if it fails, a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1711_01177_gb300 as grim
import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _scan_c_abi(lib, entry, bank, bases_d, offs_d, E_d, n_reads, cap):
    pr = torch.empty(cap, dtype=torch.int32, device="cuda")
    pb = torch.empty(cap, dtype=torch.int32, device="cuda")
    ps = torch.empty(cap, dtype=torch.int16, device="cuda")
    npairs = torch.zeros(1, dtype=torch.int64, device="cuda")
    rp = torch.empty(max(n_reads, 1), dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, entry)(bank.handle, _ptr(bases_d), _ptr(offs_d), n_reads, _ptr(E_d), 0, bank.n_bins,
                             _ptr(pr), _ptr(pb), _ptr(ps), cap, _ptr(npairs), _ptr(rp), stream)
    assert rc == grim.GRIM_OK, (entry, rc)
    st, flags = grim.grim_bank_status(bank)
    assert (st, flags) == (grim.GRIM_OK, 0), (entry, st, flags)
    n = int(npairs.item())
    assert n <= cap
    a, b, c = host(pr[:n], np.uint32), host(pb[:n], np.uint32), host(ps[:n], np.uint16)
    o = np.lexsort((b, a))
    return a[o], b[o], c[o], host(rp[:n_reads], np.uint32)


def _read_set(codes, n_reads, seed, heavy):
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(n_reads):
        L = int(rng.integers(60, 160))
        if heavy and i % 97 == 0:
            parts.append(np.tile([0, 1], L).astype(np.uint8)[:L] if i % 2 else np.zeros(L, np.uint8))
        elif rng.random() < 0.7:
            st = int(rng.integers(0, len(codes) - L))
            r = codes[st:st + L].copy()
            r ^= (rng.random(L) < 0.03).astype(np.uint8)
            parts.append(r)
        else:
            parts.append(rng.integers(0, 4, L).astype(np.uint8))
    offs = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).astype(np.int64)
    E = rng.integers(0, 8, n_reads).astype(np.uint16)
    return np.concatenate(parts), offs, E


def test_noalloc_scan_matches_scan_on_two_calls():
    grim.build()
    lib = grim.load()
    assert torch.cuda.is_available()
    codes = synth.ref_with_repeats(400_000, 21, 0.3, n_fam=20, fam_min=200, fam_max=3000)
    codes[1000:1500] = 0  # a poly-A stretch so that heavy reads have hits
    bank = grim.grim_build_bank(dev(synth.pack2bit(codes)), len(codes), 5, 256, 170)
    cap = 1 << 20
    for call, (n_reads, seed, heavy) in enumerate([(3000, 1, True), (1200, 2, False)]):
        bases, offs, E = _read_set(codes, n_reads, seed, heavy)
        bd, od, ed = dev(bases), dev(offs), dev(E)
        want = _scan_c_abi(lib, "grim_scan", bank, bd, od, ed, n_reads, cap)
        got = _scan_c_abi(lib, "grim_scan_noalloc", bank, bd, od, ed, n_reads, cap)
        assert len(want[0]) > n_reads // 2, call
        for w_, g_ in zip(want, got):
            assert np.array_equal(w_, g_), call

    # beyond the fixed scratch: rejected before any work is enqueued
    big = 200_000
    offs = torch.zeros(big + 1, dtype=torch.int64, device="cuda")
    E = torch.zeros(big, dtype=torch.int16, device="cuda")
    npairs = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = lib.grim_scan_noalloc(bank.handle, _ptr(offs), _ptr(offs), big, _ptr(E), 0, bank.n_bins, None, None, None,
                               0, _ptr(npairs), None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == grim.GRIM_ESCRATCH
    assert b"fixed scratch" in lib.grim_strerror(rc)
    bank.free()
