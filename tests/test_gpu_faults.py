"""The library's error paths on the GPU, driven by host-side fault
injection (grim_fault_inject): for every entry point, the k-th allocation
(GRIM_ENOMEM) or the k-th kernel launch (GRIM_ECUDA, rejected by the runtime
before it runs) fails, for k = 1, 2, ... until the call makes fewer than k
of them.  Each failing call must return that status and leave the library
usable: the next clean call gives the same bytes as before.  No GPU fault is
ever made; the injected failures happen on the host."""
import os
import tempfile

import numpy as np
import pytest
import torch

import paper_1711_01177_gb300 as grim
import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

ALLOC, LAUNCH, NONE = grim.GRIM_FAULT_ALLOC, grim.GRIM_FAULT_LAUNCH, grim.GRIM_FAULT_NONE
STATUS = {ALLOC: grim.GRIM_ENOMEM, LAUNCH: grim.GRIM_ECUDA}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    grim.build()
    grim.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield
    grim.grim_fault_inject(NONE, 0)


@pytest.fixture(scope="module")
def wl():
    n = 300_000
    codes = synth.ref_with_repeats(n, 17, 0.3, n_fam=20, fam_min=200, fam_max=2000)
    off = synth.read_offsets(1500, 60, 180, 17)
    bases, starts = synth.reads(codes, off, 17, 0.03, 0.01)
    E = synth.E_rate(off)
    n_bins = -(-n // 256)
    cb, co = synth.cands_random(starts, 256, n_bins, 18, k_fixed=32)
    r2 = dev(synth.pack2bit(codes))
    d = dict(n=n, codes=codes, r2=r2, reads=dev(bases), off=dev(off), E=dev(E), cb=dev(cb), co=dev(co),
             h=dict(reads=torch.from_numpy(bases).pin_memory(), off=torch.from_numpy(off).pin_memory(),
                    cb=torch.from_numpy(cb.view(np.int32)).pin_memory(), co=torch.from_numpy(co).pin_memory(),
                    E=torch.from_numpy(E.view(np.int16)).pin_memory()))
    d["bank"] = grim.grim_build_bank(r2, n, 5, 256, 100)
    d["idx"] = grim.grim_seed_index_build(r2, n, 12)
    torch.cuda.synchronize()
    yield d
    d["bank"].free()
    d["idx"].free()


def same(a, b):
    if isinstance(a, (tuple, list)):
        return len(a) == len(b) and all(same(x, y) for x, y in zip(a, b))
    return np.array_equal(a, b)


def sweep(kind, call, max_k=400, expect_events=True):
    """Fail the k-th event of `kind` for k = 1, 2, ...; returns how many
    calls failed (at least one, or none when expect_events is False)."""
    ref = call()
    failed = 0
    for k in range(1, max_k):
        grim.grim_fault_inject(kind, k)
        try:
            out = call()
        except grim.GrimError as e:
            assert e.status == STATUS[kind], (k, str(e))
            assert grim.grim_fault_pending()[0] == NONE, k
            failed += 1
            torch.cuda.synchronize()  # nothing sticky: the context still works
            assert same(call(), ref), f"wrong result after the injected failure at k={k}"
            continue
        still_armed = grim.grim_fault_pending()[0] == kind
        grim.grim_fault_inject(NONE, 0)
        assert same(out, ref), k
        if still_armed:
            break
    else:
        pytest.fail("the call kept making events; raise max_k")
    assert (failed >= 1) if expect_events else (failed == 0)
    return failed


@pytest.mark.parametrize("kind", [ALLOC, LAUNCH])
def test_build_bank(wl, kind):
    def call():
        b = grim.grim_build_bank(wl["r2"], wl["n"], 5, 256, 100)
        out = host(b.bits(), np.uint32).copy()
        b.free()
        return out
    sweep(kind, call)


@pytest.mark.parametrize("kind", [ALLOC, LAUNCH])
def test_seed_index_and_candidates(wl, kind):
    def call():
        idx = grim.grim_seed_index_build(wl["r2"], wl["n"], 12)
        cb, co = grim.grim_seed_candidates(idx, wl["reads"], wl["off"], 256, wl["bank"].n_bins, 100)
        out = (host(cb, np.uint32), host(co, np.int64))
        idx.free()
        return out
    sweep(kind, call)


@pytest.mark.parametrize("kind", [ALLOC, LAUNCH])
def test_filter_forms(wl, kind):
    bank = wl["bank"]
    ins = (wl["reads"], wl["off"], wl["cb"], wl["co"], wl["E"])
    s = torch.cuda.Stream()

    def call():
        with torch.cuda.stream(s):
            a = grim.grim_filter(bank, *ins, stream=s)
            t = grim.GrimTune(use_graph=1)
            b = grim.grim_filter_batched(bank, *ins, tune=t, stream=s)
            c, _ = grim.grim_filter_auto(bank, *ins, stream=s)
        s.synchronize()
        return host(a, np.uint8), host(b, np.uint8), host(c, np.uint8)
    # grim_filter and grim_filter_batched allocate nothing; grim_filter_auto
    # takes its batch-bounds array from the pool, so both kinds can fail
    sweep(kind, call)
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)


@pytest.mark.parametrize("kind", [ALLOC, LAUNCH])
def test_filter_host(wl, kind):
    h = wl["h"]
    out = torch.empty(wl["cb"].numel(), dtype=torch.uint8).pin_memory()

    def call():
        grim.grim_filter_host(wl["bank"], h["reads"], h["off"], h["cb"], h["co"], h["E"], pass_out=out,
                              chunk_reads=400)
        return out.numpy().copy()
    sweep(kind, call)


@pytest.mark.parametrize("kind", [ALLOC, LAUNCH])
def test_scan_locate_verify(wl, kind):
    bank = wl["bank"]
    n = 200
    off = wl["off"][:n + 1]

    def call():
        res = grim.grim_scan(bank, wl["reads"], off, wl["E"][:n])
        m = res.n_pairs
        pairs = sorted(zip(host(res.pair_read[:m], np.uint32).tolist(), host(res.pair_bin[:m], np.uint32).tolist()))
        p = grim.grim_filter(bank, wl["reads"], wl["off"], wl["cb"], wl["co"], wl["E"])
        loc = grim.grim_locate(bank, wl["cb"], wl["co"], p, capacity=int(wl["cb"].numel()))
        d = grim.grim_verify(bank, wl["r2"], wl["reads"], wl["off"], loc.read, loc.bin)
        return (np.array(pairs), host(loc.read, np.uint32), host(loc.bin, np.uint32), host(d, np.uint16))
    sweep(kind, call)


@pytest.mark.parametrize("kind", [ALLOC, LAUNCH])
def test_map(wl, kind):
    def call():
        m = grim.grim_map(wl["bank"], wl["idx"], wl["r2"], wl["reads"], wl["off"], wl["E"], cap=100, batch_reads=600,
                          capacity=200_000)
        return host(m.read, np.uint32), host(m.bin, np.uint32), host(m.dist, np.uint16)
    sweep(kind, call)


def test_bank_file_round_trip(wl):
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "bank.grim")

        def call():
            grim.grim_bank_save(wl["bank"], path)
            b = grim.grim_bank_load(path)
            out = host(b.bits(), np.uint32).copy()
            b.free()
            return out
        sweep(ALLOC, call)
