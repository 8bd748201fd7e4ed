"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact comparisons on the same seeded inputs: bank rows, pass bytes and
accumulation sums.  Sizes span many tiles, ragged tails and every token size
the kernels implement; the full-size gather workload (100 Mbp, 1M reads)
is compared on sampled outputs the oracle computes one by one.
"""
import numpy as np
import pytest
import torch

import paper_1711_01177_gb300 as grim
import synth
from gpu_util import dev, host, pack_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    grim.build()
    grim.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def gpu_bank(ref2bit, length, q, bin_len, overlap):
    bank = grim.grim_build_bank(dev(ref2bit), length, q, bin_len, overlap)
    st, flags = grim.grim_bank_status(bank)
    assert st == grim.GRIM_OK and flags == 0
    return bank


def run_filter(bank, bases, offs, cb, co, E):
    sums = torch.empty(len(cb), dtype=torch.int16, device="cuda")
    p = grim.grim_filter(bank, dev(bases), dev(offs), dev(cb), dev(co), dev(E), sums=sums)
    st, flags = grim.grim_bank_status(bank)
    return host(p, np.uint8), host(sums, np.uint16), st, flags


# ------------------------------------------------------------- bank build

@pytest.mark.parametrize("q,bin_len,overlap,n", [
    (1, 7, 0, 50), (2, 7, 3, 61), (3, 32, 10, 5000), (4, 50, 25, 7777), (5, 256, 100, 200_003),
    (6, 256, 300, 100_001), (5, 100, 0, 12_345), (5, 1000, 5, 3000), (4, 17, 0, 4), (5, 16, 16, 3),
    (6, 3, 40, 999), (5, 256, 100, 1), (3, 300_000, 7, 1_000_000),
    # geometries of the lane-per-core kernel: whole following cores in a
    # span (J >= 1), no prefix (e = 0), the largest bins, CTA boundaries
    (5, 256, 300, 400_000), (5, 256, 4, 300_001), (4, 64, 700, 100_000), (5, 1024, 100, 500_000),
    (5, 2048, 100, 500_000), (5, 512, 100, 1_000_003),
    (5, 256, 100, 195_840), (3, 48, 2, 9_999), (1, 16, 0, 1000), (5, 16, 4000, 50_000), (2, 32, 45, 7_001),
    (5, 256, 100, 2_000_003)])
def test_bank_matches_oracle(oracle, q, bin_len, overlap, n):
    codes = synth.ref_with_repeats(n, q + n, 0.3 if n > 20_000 else 0.0, n_fam=20, fam_min=100, fam_max=2000)
    r2 = synth.pack2bit(codes)
    bank = gpu_bank(r2, n, q, bin_len, overlap)
    assert bank.n_bins == -(-n // bin_len)
    assert bank.row_words == max(4, 4 ** q // 32)
    want = pack_rows(oracle.build_bank(r2, n, q, bin_len, overlap), bank.row_words)
    got = bank.bits().cpu().numpy().view(np.uint32)
    assert np.array_equal(got, want)
    bank.free()


@pytest.mark.parametrize("bin_len,k", [(19, 1), (16, 2)])
def test_bank_at_bin_counts_multiple_of_2_16(oracle, bin_len, k):
    """Banks of exactly k x 2^16 bins (the paper's banks hold 450 x 2^16,
    Sec. 6.1): a 19-base bin length takes the run-per-CTA build, a 16-base
    one the lane-per-core build; every row against the oracle."""
    n = k * (1 << 16) * bin_len
    codes = synth.ref_with_repeats(n, 77 + k, 0.3, n_fam=20, fam_min=100, fam_max=2000)
    r2 = synth.pack2bit(codes)
    bank = gpu_bank(r2, n, 5, bin_len, 150)
    assert bank.n_bins == k << 16
    want = pack_rows(oracle.build_bank(r2, n, 5, bin_len, 150), bank.row_words)
    assert np.array_equal(bank.bits().cpu().numpy().view(np.uint32), want)
    bank.free()


def test_bank_from_unaligned_reference(oracle):
    """A reference buffer that does not start on a 4-byte boundary takes the
    byte-wise build; the rows are the same."""
    n = 300_001
    codes = synth.ref_with_repeats(n, 77, 0.3, n_fam=20, fam_min=100, fam_max=2000)
    r2 = synth.pack2bit(codes)
    buf = torch.zeros(len(r2) + 1, dtype=torch.uint8, device="cuda")
    buf[1:] = dev(r2)
    bank = grim.grim_build_bank(buf[1:], n, 5, 256, 100)
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    want = pack_rows(oracle.build_bank(r2, n, 5, 256, 100), bank.row_words)
    assert np.array_equal(bank.bits().cpu().numpy().view(np.uint32), want)
    bank.free()


# ---------------------------------------------------------------- filter

def test_filter_plain_gather_workload_full(oracle):
    """1 Mbp i.i.d. reference, 10,000 x 100 bp reads, 32 candidates each: all 320,000 checks."""
    w = synth.gather_iid()
    bank = gpu_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    p, s, st, flags = run_filter(bank, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, w.E)
    assert st == grim.GRIM_OK and flags == 0
    ob = oracle.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    op, os_ = oracle.filter(ob, w.q, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, w.E)
    assert np.array_equal(s, os_.astype(np.uint16))
    assert np.array_equal(p, op)
    assert 0 < p.sum() < len(p)
    bank.free()


@pytest.mark.parametrize("q,ref_len", [(5, 200_000_000), (6, 60_000_000)])
def test_filter_bank_beyond_l2_takes_the_deep_form(oracle, q, ref_len):
    """Banks beyond the L2 (200 Mbp at q=5: 100 MB, read by the gather form
    that keeps three steps of rows in flight; 60 Mbp at q=6: 120 MB); every
    pass byte and sum against the oracle, each candidate's bitvector rebuilt
    from the reference."""
    w = synth.gather_iid(ref_len=ref_len, n_reads=20_000, k=32, q=q)
    bank = gpu_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    assert bank.n_bins * bank.row_words * 4 > 96e6
    p, s, st, flags = run_filter(bank, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, w.E)
    assert st == grim.GRIM_OK and flags == 0
    op, os_ = oracle.filter_rows(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap, w.bases, w.read_offsets,
                                 w.cand_bins, w.cand_offsets, w.E)
    assert np.array_equal(s, os_.astype(np.uint16))
    assert np.array_equal(p, op)
    assert 0 < p.sum() < len(p)
    bank.free()


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6])
def test_filter_every_q_ragged(oracle, q):
    rng = np.random.default_rng(40 + q)
    n = 60_000
    codes = synth.ref_with_repeats(n, 5 + q, 0.3, n_fam=10, fam_min=100, fam_max=1000)
    r2 = synth.pack2bit(codes)
    bin_len, overlap = 200, 320
    bank = gpu_bank(r2, n, q, bin_len, overlap)
    nb = bank.n_bins
    n_reads = 777
    lens = rng.integers(0, 320, n_reads)
    lens[:20] = np.arange(20)  # empty and shorter-than-q reads
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    starts = rng.integers(0, n - 330, n_reads)
    bases = np.concatenate([codes[s:s + L] for s, L in zip(starts, lens)]).astype(np.uint8)
    bases ^= (rng.random(len(bases)) < 0.03).astype(np.uint8)  # sprinkle substitutions
    k = rng.integers(0, 90, n_reads)
    k[::50] = 0  # reads without candidates
    co = np.concatenate([[0], np.cumsum(k)]).astype(np.int64)
    cb = rng.integers(0, nb, int(co[-1])).astype(np.uint32)
    for r in range(n_reads):  # include the true bin and a duplicate when possible
        if k[r] >= 2:
            cb[co[r]] = starts[r] // bin_len
            cb[co[r] + 1] = cb[co[r]]
    E = rng.integers(0, 12, n_reads).astype(np.uint16)
    p, s, st, flags = run_filter(bank, bases, offs, cb, co, E)
    assert st == grim.GRIM_OK and flags == 0
    ob = oracle.build_bank(r2, n, q, bin_len, overlap)
    op, os_ = oracle.filter(ob, q, bases, offs, cb, co, E)
    assert np.array_equal(s, os_.astype(np.uint16))
    assert np.array_equal(p, op)
    bank.free()


def test_filter_low_complexity_and_long_reads(oracle):
    """Counts far above 15 exercise the shared-memory count planes (more than 4 planes)."""
    n = 20_000
    codes = synth.ref_iid(n, 3)
    codes[5000:5600] = 0  # a poly-A stretch
    codes[9000:9800] = np.tile([0, 1], 400)  # (AC)n
    r2 = synth.pack2bit(codes)
    q, bl, ov = 5, 256, 65_600
    bank = gpu_bank(r2, n, q, bl, ov)
    reads_l = [np.zeros(100, np.uint8), np.zeros(5000, np.uint8), np.tile([0, 1], 2000).astype(np.uint8),
               np.zeros(65_535, np.uint8), codes[4900:5700].copy(), codes[100:65535 % n + 100].copy(),
               np.tile([0, 1, 2], 20_000).astype(np.uint8)]
    offs = np.concatenate([[0], np.cumsum([len(x) for x in reads_l])]).astype(np.int64)
    bases = np.concatenate(reads_l)
    cb = np.tile(np.arange(bank.n_bins, dtype=np.uint32), len(reads_l))
    co = np.arange(0, (len(reads_l) + 1) * bank.n_bins, bank.n_bins, dtype=np.int64)
    E = np.array([0, 3, 100, 10, 5, 1000, 7], dtype=np.uint16)
    p, s, st, flags = run_filter(bank, bases, offs, cb, co, E)
    assert st == grim.GRIM_OK and flags == 0
    ob = oracle.build_bank(r2, n, q, bl, ov)
    op, os_ = oracle.filter(ob, q, bases, offs, cb, co, E)
    assert np.array_equal(s, os_.astype(np.uint16))
    assert np.array_equal(p, op)
    assert s.max() > 60_000  # the 65,535-base poly-A read
    bank.free()


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6])
def test_filter_count_path_boundaries(oracle, q):
    """The token-count paths at their edges: reads of 255 token positions
    (byte counters, one of them reaching 255: eight planes) and of 256 (the
    carry chain), lengths around the 160-base blocks of the token roller,
    and random reads with one run giving a top count of 2 .. 8 (one to four
    planes, the register paths and the shared-memory path)."""
    rng = np.random.default_rng(700 + q)
    n = 30_000
    codes = synth.ref_iid(n, 70 + q)
    codes[8000:8400] = 0  # poly-A
    codes[12000:12400] = np.tile([0, 1], 200)  # (AC)n
    r2 = synth.pack2bit(codes)
    bank = gpu_bank(r2, n, q, 256, 120)
    reads_l = []
    for L in (q + 253, q + 254, q + 255, q + 256):  # 254 .. 257 token positions
        reads_l += [np.zeros(L, np.uint8), np.tile([0, 1], L)[:L].astype(np.uint8), codes[7900:7900 + L].copy()]
    for L in (155, 159, 160, 161, 163, 164, 165, 166, 319, 320, 321, 324, 325):
        st = int(rng.integers(0, n - L))
        reads_l.append(codes[st:st + L].copy())
    for run in range(q + 1, q + 8):  # a poly-A run of `run` bases: top count run - q + 1
        st = int(rng.integers(0, n - 150))
        r = codes[st:st + 150].copy()
        r[40:40 + run] = 0
        reads_l.append(r)
    offs = np.concatenate([[0], np.cumsum([len(x) for x in reads_l])]).astype(np.int64)
    bases = np.concatenate(reads_l).astype(np.uint8)
    nr = len(reads_l)
    cb = np.tile(np.arange(bank.n_bins, dtype=np.uint32), nr)
    co = np.arange(0, (nr + 1) * bank.n_bins, bank.n_bins, dtype=np.int64)
    E = rng.integers(0, 20, nr).astype(np.uint16)
    p, s, st, flags = run_filter(bank, bases, offs, cb, co, E)
    assert st == grim.GRIM_OK and flags == 0
    ob = oracle.build_bank(r2, n, q, 256, 120)
    op, os_ = oracle.filter(ob, q, bases, offs, cb, co, E)
    assert np.array_equal(s, os_.astype(np.uint16))
    assert np.array_equal(p, op)
    assert p.any() and (q == 1 or not p.all())  # at q = 1 every bin holds all four tokens
    bank.free()


def test_fill_E_rate_is_the_integer_rule():
    """E = floor(num L / den) (or the ceiling), saturated, 0 for a negative
    length: checked against Python integers and the input generator's rule."""
    rng = np.random.default_rng(5)
    lens = rng.integers(0, 400, 5000)
    lens[:6] = [0, 1, 19, 20, 21, 150]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    offs_d = dev(offs)
    for num, den, up in ((5, 100, False), (5, 100, True), (1, 3, False), (7, 1, True), (0, 9, False)):
        E = host(grim.grim_fill_E_rate(offs_d, num, den, up), np.uint16)
        want = [min(65535, (num * int(L) + (den - 1 if up else 0)) // den) for L in lens]
        assert E.tolist() == want, (num, den, up)
    assert np.array_equal(host(grim.grim_fill_E_rate(offs_d), np.uint16), synth.E_rate(offs))
    odd = dev(np.array([0, 100, 50, 50 + 10_000_000], np.int64))  # decreasing, then very long
    assert host(grim.grim_fill_E_rate(odd, 5, 100), np.uint16).tolist() == [5, 0, 3276]
    assert host(grim.grim_fill_E_rate(odd, 60_000, 1), np.uint16).tolist() == [65535, 0, 65535]


def test_filter_empty_inputs(oracle):
    w = synth.gather_iid(ref_len=50_000, n_reads=64, k=4)
    bank = gpu_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    # no reads at all
    p = grim.grim_filter(bank, dev(w.bases[:0]), dev(np.zeros(1, np.int64)), dev(np.zeros(0, np.uint32)),
                         dev(np.zeros(1, np.int64)), dev(np.zeros(0, np.uint16)))
    assert p.numel() == 0
    # reads but no candidates
    co = np.zeros(w.n_reads + 1, np.int64)
    p = grim.grim_filter(bank, dev(w.bases), dev(w.read_offsets), dev(np.zeros(0, np.uint32)), dev(co), dev(w.E))
    assert p.numel() == 0
    # all reads empty, candidates present: sum 0, threshold <= 0 -> pass
    offs0 = np.zeros(w.n_reads + 1, np.int64)
    pp, s, st, _ = run_filter(bank, w.bases[:0], offs0, w.cand_bins, w.cand_offsets, w.E)
    assert st == grim.GRIM_OK and pp.all() and not s.any()
    bank.free()


def test_filter_bad_data_is_flagged_not_faulted(oracle):
    w = synth.gather_iid(ref_len=100_000, n_reads=300, k=16)
    bank = gpu_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    ob = oracle.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    op, os_ = oracle.filter(ob, w.q, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, w.E)
    bases = w.bases.copy()
    bases[w.read_offsets[7] + 50] = 4  # read 7: a code > 3
    cb = w.cand_bins.copy()
    cb[w.cand_offsets[11] + 3] = bank.n_bins  # read 11: one bin id out of range
    cb[w.cand_offsets[12]] = 0xFFFFFFFF
    p, s, st, flags = run_filter(bank, bases, w.read_offsets, cb, w.cand_offsets, w.E)
    assert st == grim.GRIM_EDATA
    assert flags == grim.GRIM_FLAG_BAD_BASE | grim.GRIM_FLAG_BAD_BIN
    bad = np.zeros(len(cb), bool)
    bad[w.cand_offsets[7]:w.cand_offsets[8]] = True
    bad[w.cand_offsets[11] + 3] = True
    bad[w.cand_offsets[12]] = True
    assert not p[bad].any() and not s[bad].any()
    assert np.array_equal(p[~bad], op[~bad]) and np.array_equal(s[~bad], os_[~bad].astype(np.uint16))
    # the status word was cleared by the read
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    # decreasing read offsets: flagged, outputs of that read discarded
    offs = w.read_offsets.copy()
    offs[20] = offs[21] + 5
    p, s, st, flags = run_filter(bank, w.bases, offs, w.cand_bins, w.cand_offsets, w.E)
    assert st == grim.GRIM_EDATA and flags & grim.GRIM_FLAG_BAD_OFFSETS
    assert not p[w.cand_offsets[20]:w.cand_offsets[21]].any()
    bank.free()


@pytest.mark.parametrize("entry", ["grim_filter", "grim_filter_batched"])
def test_decreasing_offsets_spare_every_other_read(oracle, entry):
    """Decreasing read and candidate offsets in a 20,000-read launch: both
    reads are flagged and every read whose own offsets are intact, on any warp
    of the launch, still gets the oracle's bytes."""
    w = synth.gather_iid(ref_len=400_000, n_reads=20_000, k=16)
    bank = gpu_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    ob = oracle.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    op, os_ = oracle.filter(ob, w.q, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, w.E)
    offs = w.read_offsets.copy()
    offs[5000] = offs[5001] + 2000  # read 4999 grows into later bases, read 5000 decreases
    co = w.cand_offsets.copy()
    co[1000] = co[1001] + 40  # read 999 spills over reads 1000-1003's slots, read 1000 decreases
    spoiled = np.zeros(len(w.cand_bins), bool)
    spoiled[w.cand_offsets[999]:w.cand_offsets[1004]] = True
    spoiled[w.cand_offsets[4999]:w.cand_offsets[5001]] = True
    pass_out = torch.full((len(w.cand_bins),), 0xAA, dtype=torch.uint8, device="cuda")
    sums = torch.full((len(w.cand_bins),), 0x5A5A, dtype=torch.int16, device="cuda")
    getattr(grim, entry)(bank, dev(w.bases), dev(offs), dev(w.cand_bins), dev(co), dev(w.E), pass_out=pass_out,
                         sums=sums)
    st, flags = grim.grim_bank_status(bank)
    assert st == grim.GRIM_EDATA and flags == grim.GRIM_FLAG_BAD_OFFSETS
    p, s = host(pass_out, np.uint8), host(sums, np.uint16)
    assert np.array_equal(p[~spoiled], op[~spoiled])
    assert np.array_equal(s[~spoiled], os_[~spoiled].astype(np.uint16))
    bank.free()


def test_host_errors():
    r2 = dev(synth.pack2bit(synth.ref_iid(1000, 1)))
    with pytest.raises(grim.GrimError) as e:
        grim.grim_build_bank(r2, 1000, 7, 256, 100)
    assert e.value.status == grim.GRIM_ENOTSUP
    with pytest.raises(grim.GrimError) as e:
        grim.grim_build_bank(r2, 1000, 5, 0, 100)
    assert e.value.status == grim.GRIM_EINVAL


# ------------------------------------------------- full-size workload, sampled

def test_filter_100mbp_seed_workload_sampled(oracle):
    """100 Mbp repeat-rich reference, 1M x 150 bp reads, 12-mer seed candidates:
    the full launch bench.py times, checked on a sample of rows and pairs."""
    w = synth.gather_seeds()
    r2 = dev(w.ref2bit)
    bank = grim.grim_build_bank(r2, w.ref_len, w.q, w.bin_len, w.overlap)
    sums = torch.empty(w.n_checks, dtype=torch.int16, device="cuda")
    p = grim.grim_filter(bank, dev(w.bases), dev(w.read_offsets), dev(w.cand_bins), dev(w.cand_offsets), dev(w.E),
                         sums=sums)
    assert grim.grim_bank_status(bank) == (grim.GRIM_OK, 0)
    p, s = host(p, np.uint8), host(sums, np.uint16)
    rng = np.random.default_rng(123)
    bits = bank.bits()
    for b in rng.integers(0, w.n_bins, 200):
        row = oracle.bin_row(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap, int(b))
        assert np.array_equal(bits[int(b)].cpu().numpy().view(np.uint32), pack_rows(row[None, :], bank.row_words)[0])
    read_of = np.searchsorted(w.cand_offsets, np.arange(w.n_checks), side="right") - 1
    for c in rng.integers(0, w.n_checks, 3000):
        r = int(read_of[c])
        b = int(w.cand_bins[c])
        row = oracle.bin_row(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap, b)
        read = w.bases[w.read_offsets[r]:w.read_offsets[r + 1]]
        want = oracle.sum_one(row, w.q, read)
        assert s[c] == want
        assert p[c] == int(want >= oracle.threshold(len(read), w.q, int(w.E[r])))
    # properties that hold at any size
    assert s.max() <= 150 - w.q + 1
    assert np.array_equal(p, (s.astype(np.int64) >= 146 - 5 * 7).astype(np.uint8))
    bank.free()
