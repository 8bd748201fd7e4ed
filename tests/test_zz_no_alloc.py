"""grim_scan_noalloc gives exactly what grim_scan and the oracle give.

grim_scan_noalloc serves callers that cannot allocate device memory when
they call the filter (their device memory belongs to their own pool, or
their footprint is fixed after start-up); it runs the same full scan in the
library's fixed scratch array instead of a cudaMallocAsync'd one.  The test
calls it through the C ABI several times in a row on different read sets -
each call finds the previous call's data in the shared scratch and must not
be affected by it - and compares each result with grim_scan's on the same
inputs and with the oracle's full scan: the same set of passing (read, bin)
pairs, the same sums, the same per-read counts (bit-exact, the filter's
outputs are integers).  The read sets include low-complexity reads whose
token counts need 2, 4 and 8 base-4 digits, so every digit class passes
through the shared array, and a call at q = 4 follows the calls at q = 5.
It also checks the documented limit: the largest accepted request at q = 5
runs, one read more is rejected up front.

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

MAX_READS_Q5 = 8_672  # the largest request the 64 MiB array holds at q = 5


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _scan_c_abi(lib, entry, bank, bases_d, offs_d, E_d, n_reads, cap):
    pr = torch.empty(cap, dtype=torch.int32, device="cuda")
    pb = torch.empty(cap, dtype=torch.int32, device="cuda")
    ps = torch.empty(cap, dtype=torch.int16, device="cuda")
    npairs = torch.zeros(1, dtype=torch.int64, device="cuda")
    rp = torch.empty(max(n_reads, 1), dtype=torch.int32, device="cuda")
    rc = getattr(lib, entry)(bank.handle, _ptr(bases_d), _ptr(offs_d), n_reads, _ptr(E_d), 0, bank.n_bins,
                             _ptr(pr), _ptr(pb), _ptr(ps), cap, _ptr(npairs), _ptr(rp), _stream())
    assert rc == grim.GRIM_OK, (entry, rc)
    st, flags = grim.grim_bank_status(bank)
    assert (st, flags) == (grim.GRIM_OK, 0), (entry, st, flags)
    n = int(npairs.item())
    assert n <= cap
    a, b, c = host(pr[:n], np.uint32), host(pb[:n], np.uint32), host(ps[:n], np.uint16)
    o = np.lexsort((b, a))
    return a[o], b[o], c[o], host(rp[:n_reads], np.uint32)


def _read_set(codes, n_reads, seed, heavy):
    """Reads copied from the reference with 3% substitutions, random reads,
    and (heavy) low-complexity reads: poly-A of 10, 20 and 300 bases (token
    counts 6, 16, 296: 2, 4 and 8 base-4 digits) and a dinucleotide repeat."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(n_reads):
        L = int(rng.integers(60, 160))
        if heavy and i % 97 == 0:
            kind = (i // 97) % 4
            if kind == 0:
                parts.append(np.zeros(10, np.uint8))
            elif kind == 1:
                parts.append(np.zeros(20, np.uint8))
            elif kind == 2:
                parts.append(np.zeros(300, np.uint8))
            else:
                parts.append(np.tile([0, 1], L).astype(np.uint8)[:L])
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


def _oracle_scan(oracle, ob, q, bases, offs, E):
    pr, pb, ps = oracle.scan(ob, q, bases, offs, E)
    rp = np.bincount(pr, minlength=len(offs) - 1).astype(np.uint32)
    return pr, pb, ps.astype(np.uint16), rp


def test_noalloc_scan_matches_scan_and_oracle_on_calls_in_a_row(oracle):
    grim.build()
    lib = grim.load()
    assert torch.cuda.is_available()
    codes = synth.ref_with_repeats(400_000, 21, 0.3, n_fam=20, fam_min=200, fam_max=3000)
    codes[1000:1500] = 0  # a poly-A stretch so that heavy reads have hits
    r2 = synth.pack2bit(codes)
    cap = 1 << 23  # at q = 4 about half of all (read, bin) pairs pass
    calls = [(5, 3000, 1, True), (5, 1200, 2, False), (4, 1500, 3, True)]
    banks = {}
    for call, (q, n_reads, seed, heavy) in enumerate(calls):
        if q not in banks:
            banks[q] = (grim.grim_build_bank(dev(r2), len(codes), q, 256, 300),
                        oracle.build_bank(r2, len(codes), q, 256, 300))
        bank, ob = banks[q]
        bases, offs, E = _read_set(codes, n_reads, seed, heavy)
        bd, od, ed = dev(bases), dev(offs), dev(E)
        want = _scan_c_abi(lib, "grim_scan", bank, bd, od, ed, n_reads, cap)
        got = _scan_c_abi(lib, "grim_scan_noalloc", bank, bd, od, ed, n_reads, cap)
        ora = _oracle_scan(oracle, ob, q, bases, offs, E)
        assert len(want[0]) > n_reads // 2, call
        for w_, g_, o_ in zip(want, got, ora):
            assert np.array_equal(g_, w_), call
            assert np.array_equal(g_, o_), call
    for bank, _ in banks.values():
        bank.free()


def test_noalloc_limit_is_exact():
    grim.build()
    lib = grim.load()
    codes = synth.ref_iid(200_000, 5)
    bank = grim.grim_build_bank(dev(synth.pack2bit(codes)), len(codes), 5, 256, 100)
    rng = np.random.default_rng(9)
    n = MAX_READS_Q5 + 1
    bases = rng.integers(0, 4, 100 * n).astype(np.uint8)
    offs = np.arange(0, 100 * n + 1, 100, dtype=np.int64)
    E = np.full(n, 5, np.uint16)
    bd, od, ed = dev(bases), dev(offs), dev(E)
    # the largest accepted request runs and agrees with grim_scan
    want = _scan_c_abi(lib, "grim_scan", bank, bd, od[:MAX_READS_Q5 + 1], ed, MAX_READS_Q5, 1 << 16)
    got = _scan_c_abi(lib, "grim_scan_noalloc", bank, bd, od[:MAX_READS_Q5 + 1], ed, MAX_READS_Q5, 1 << 16)
    for w_, g_ in zip(want, got):
        assert np.array_equal(g_, w_)
    # one read more is rejected before any work is enqueued
    npairs = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = lib.grim_scan_noalloc(bank.handle, _ptr(bd), _ptr(od), n, _ptr(ed), 0, bank.n_bins, None, None, None, 0,
                               _ptr(npairs), None, _stream())
    assert rc == grim.GRIM_ESCRATCH
    assert b"fixed scratch" in lib.grim_strerror(rc)
    assert int(npairs.item()) == 0
    bank.free()
