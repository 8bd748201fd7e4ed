"""Bank files and the packed bitmask (the paper keeps the bank with the
reference, Sec. 3.1; its bitmask holds one bit per location, Sec. 3.3).
The CPU tests check that invalid files are refused before any device work;
the GPU tests round-trip banks and pack masks."""
import ctypes
import struct

import numpy as np
import pytest

import paper_1711_01177_gb300 as grim
import synth


@pytest.fixture(scope="module", autouse=True)
def _lib():
    grim.build()
    grim.load()


def load_status(path):
    h = ctypes.c_void_p()
    return grim.load().grim_bank_load(str(path).encode(), None, ctypes.byref(h)), h.value


def header(q=5, length=1000, bin_len=256, overlap=100, n_bins=None, row_words=None, payload=None, magic=b"GRIMBNK1"):
    n_bins = -(-length // bin_len) if n_bins is None else n_bins
    row_words = max(4, 4 ** q // 32) if row_words is None else row_words
    payload = n_bins * row_words * 4 if payload is None else payload
    return magic + struct.pack("<IIqiiqqQQ", 64, q, length, bin_len, overlap, n_bins, row_words, payload, 0)


def test_invalid_bank_files_are_refused_on_the_host(tmp_path):
    assert load_status(tmp_path / "missing.bank") == (grim.GRIM_EIO, None)
    bad = {
        "garbage": b"not a bank file at all" * 10,
        "short_header": header()[:40],
        "bad_magic": header(magic=b"GRIMBNK0") + bytes(4 * 128 * 4),
        "wrong_n_bins": header(n_bins=5) + bytes(5 * 32 * 4),
        "wrong_row_words": header(row_words=64) + bytes(4 * 64 * 4),
        "q_out_of_range": header(q=9, row_words=4) + bytes(16 * 4),
        "truncated_payload": header() + bytes(100),
        "trailing_bytes": header() + bytes(4 * 32 * 4 + 1),
    }
    for name, data in bad.items():
        p = tmp_path / f"{name}.bank"
        p.write_bytes(data)
        assert load_status(p) == (grim.GRIM_EIO, None), name


@pytest.mark.gpu
@pytest.mark.parametrize("q,n,bin_len,overlap", [(5, 1_000_003, 256, 100), (6, 300_000, 256, 300), (3, 5000, 17, 0),
                                                 (4, 70_000_000, 256, 150)])
def test_bank_round_trip(tmp_path, q, n, bin_len, overlap):
    import torch
    from gpu_util import dev, host
    codes = synth.ref_with_repeats(n, q + 2, 0.2 if n > 50_000 else 0.0, n_fam=20, fam_min=100, fam_max=2000)
    r2 = dev(synth.pack2bit(codes))
    bank = grim.grim_build_bank(r2, n, q, bin_len, overlap)
    path = str(tmp_path / "ref.bank")
    grim.grim_bank_save(bank, path)
    back = grim.grim_bank_load(path)
    assert (back.len, back.n_bins, back.q, back.bin_len, back.overlap, back.row_words) == \
        (bank.len, bank.n_bins, bank.q, bank.bin_len, bank.overlap, bank.row_words)
    assert torch.equal(back.bits(), bank.bits())
    # the loaded bank filters like the built one
    off = synth.read_offsets(2000, 100, 100, 5)
    bases, starts = synth.reads(codes, off, 5, 0.03, 0.01)
    cb, co = synth.cands_random(starts, bin_len, bank.n_bins, 5, k_fixed=8)
    E = np.full(2000, 5, np.uint16)
    ins = [dev(bases), dev(off), dev(cb), dev(co), dev(E)]
    assert torch.equal(grim.grim_filter(bank, *ins), grim.grim_filter(back, *ins))
    assert grim.grim_bank_status(back) == (grim.GRIM_OK, 0)
    back.free()
    # a flipped payload byte fails the checksum; a cut file fails the size check
    raw = bytearray(open(path, "rb").read())
    raw[64 + len(raw) // 3] ^= 0x10
    open(path, "wb").write(bytes(raw))
    assert load_status(path)[0] == grim.GRIM_EIO
    open(path, "wb").write(bytes(raw[:-16]))
    assert load_status(path)[0] == grim.GRIM_EIO
    bank.free()


@pytest.mark.gpu
@pytest.mark.parametrize("n,offset", [(0, 0), (1, 0), (31, 0), (32, 0), (1000, 0), (1000, 3), (3_000_001, 5),
                                      (64 * 100_000, 0)])
def test_pack_mask(n, offset):
    import torch
    from gpu_util import host
    rng = np.random.default_rng(n + offset)
    raw = rng.integers(0, 256, n + offset).astype(np.uint8)
    raw[rng.random(n + offset) < 0.7] = 0
    buf = torch.from_numpy(raw).cuda()
    bits = grim.grim_pack_mask(buf[offset:])
    torch.cuda.synchronize()
    want = np.packbits(raw[offset:] != 0, bitorder="little")
    want = np.concatenate([want, np.zeros((-len(want)) % 4, np.uint8)]).view("<u4")
    assert np.array_equal(host(bits, np.uint32), want)
