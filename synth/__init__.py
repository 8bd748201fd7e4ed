"""Seeded synthetic inputs for the seed-location filter.

Shared by the tests, the oracle checks and the benchmark.  Nothing here
computes any part of the filter (tokens, bitvectors, sums, thresholds); it
draws references, reads and candidate bin lists from splitmix64 streams
(see ``synth.c``) and packs references into the 2-bit format.

The workload recipes at the bottom describe the five synthetic workloads by
what they are (sizes, error model, candidate source) and stand in for the
1000 Genomes read sets and the human reference used in the paper (Sec. 5,
Table 1), which are not available here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile libsynth.so with gcc (portable flags, no FP contraction;
    OpenMP over reads when the compiler has it - the data do not depend on
    the thread count)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        try:
            subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64, U64, I32, D = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        sig = {
            "synth_ref_iid": (None, [U64, I64, P]),
            "synth_ref_repeats": (I64, [U64, I64, D, I32, I32, I32, D, D, P]),
            "synth_pack2bit": (None, [P, I64, P]),
            "synth_read_lengths": (None, [U64, I64, I32, I32, P]),
            "synth_reads": (I32, [U64, P, I64, I64, P, D, D, P, P]),
            "synth_cand_counts": (None, [U64, I64, I32, I32, I64, P]),
            "synth_cands_random": (I32, [U64, I64, P, I32, I64, P, P]),
            "synth_seed_index": (I32, [P, I64, I32, P, P]),
            "synth_seed_index_needed": (I64, [P, I64, I32, P, P, P]),
            "synth_cands_seeds": (I64, [P, P, I32, P, P, I64, I32, I64, I32, I64, P, P]),
            "synth_E_rate": (None, [P, I64, I32, I32, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ primitives

def ref_iid(length: int, seed: int) -> np.ndarray:
    out = np.empty(length, dtype=np.uint8)
    _load().synth_ref_iid(seed, length, _p(out))
    return out


def ref_with_repeats(length: int, seed: int, frac: float, n_fam: int = 200, fam_min: int = 300,
                     fam_max: int = 6000, div_lo: float = 0.10, div_hi: float = 0.20) -> np.ndarray:
    """i.i.d. ACGT with planted repeat families covering >= frac of the bases."""
    codes = ref_iid(length, seed)
    if frac > 0:
        fam_max = min(fam_max, length // 2)
        fam_min = min(fam_min, fam_max)
        n = _load().synth_ref_repeats(seed + 3, length, frac, n_fam, fam_min, fam_max, div_lo, div_hi,
                                      _p(codes))
        if n < 0:
            raise ValueError("synth_ref_repeats: bad arguments")
    return codes


def pack2bit(codes: np.ndarray) -> np.ndarray:
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    out = np.empty((len(codes) + 3) // 4, dtype=np.uint8)
    _load().synth_pack2bit(_p(codes), len(codes), _p(out))
    return out


def read_offsets(n: int, lmin: int, lmax: int, seed: int) -> np.ndarray:
    off = np.empty(n + 1, dtype=np.int64)
    _load().synth_read_lengths(seed, n, lmin, lmax, _p(off))
    return off


def reads(codes: np.ndarray, offsets: np.ndarray, seed: int, sub: float, indel: float):
    """Returns (bases u8, starts i64)."""
    n = len(offsets) - 1
    bases = np.empty(int(offsets[-1]), dtype=np.uint8)
    starts = np.empty(n, dtype=np.int64)
    rc = _load().synth_reads(seed, _p(codes), len(codes), n, _p(offsets), sub, indel, _p(bases), _p(starts))
    if rc != 0:
        raise ValueError("reference too short for the read lengths")
    return bases, starts


def cands_random(starts: np.ndarray, bin_len: int, n_bins: int, seed: int, k_fixed: int = 0,
                 k_max: int = 0):
    """True bin + distinct uniform others; k fixed or log-uniform in [1, k_max]."""
    n = len(starts)
    off = np.empty(n + 1, dtype=np.int64)
    _load().synth_cand_counts(seed, n, k_fixed, k_max, n_bins, _p(off))
    bins = np.empty(int(off[-1]), dtype=np.uint32)
    _load().synth_cands_random(seed, n, _p(np.ascontiguousarray(starts, dtype=np.int64)), bin_len, n_bins,
                               _p(off), _p(bins))
    return bins, off


def seed_index(codes: np.ndarray, k: int = 12):
    offsets = np.empty((1 << (2 * k)) + 1, dtype=np.uint32)
    positions = np.empty(len(codes) - k + 1, dtype=np.uint32)
    if _load().synth_seed_index(_p(codes), len(codes), k, _p(offsets), _p(positions)) != 0:
        raise ValueError("synth_seed_index failed")
    return offsets, positions


def seed_index_for_reads(codes: np.ndarray, bases: np.ndarray, offsets: np.ndarray, k: int = 12):
    """The seed index restricted to the k-mers the reads' non-overlapping
    seeds ask for (same hits for those seeds as the full index)."""
    lib = _load()
    needed = np.zeros((1 << (2 * k)) // 64, dtype=np.uint64)
    L = np.diff(offsets)
    starts = offsets[:-1]
    for o in range(0, int(L.max()) - k + 1, k):
        sel = L >= o + k
        pos = starts[sel] + o
        key = np.zeros(len(pos), dtype=np.uint64)
        for j in range(k):
            key = (key << np.uint64(2)) | bases[pos + j].astype(np.uint64)
        np.bitwise_or.at(needed, key >> np.uint64(6), np.uint64(1) << (key & np.uint64(63)))
    idx_off = np.empty((1 << (2 * k)) + 1, dtype=np.uint32)
    n = lib.synth_seed_index_needed(_p(codes), len(codes), k, _p(needed), _p(idx_off), None)
    if n < 0:
        raise ValueError("synth_seed_index_needed failed")
    positions = np.empty(max(int(n), 1), dtype=np.uint32)
    if lib.synth_seed_index_needed(_p(codes), len(codes), k, _p(needed), _p(idx_off), _p(positions)) < 0:
        raise ValueError("synth_seed_index_needed failed")
    return idx_off, positions


def cands_seeds(index, bases: np.ndarray, offsets: np.ndarray, bin_len: int, n_bins: int, cap: int,
                k: int = 12):
    """Bins of all exact k-mer seed hits (non-overlapping seeds), capped per read."""
    idx_off, idx_pos = index
    n = len(offsets) - 1
    cap_total = max(1024, n * 96)
    lib = _load()
    while True:
        bins = np.empty(cap_total, dtype=np.uint32)
        coff = np.empty(n + 1, dtype=np.int64)
        total = lib.synth_cands_seeds(_p(idx_off), _p(idx_pos), k, _p(bases), _p(offsets), n, bin_len, n_bins,
                                      cap, cap_total, _p(bins), _p(coff))
        if total < 0:
            raise MemoryError("synth_cands_seeds failed")
        if total <= cap_total:
            return bins[:total], coff
        cap_total = int(total)


def E_rate(offsets: np.ndarray, num: int = 5, den: int = 100) -> np.ndarray:
    E = np.empty(len(offsets) - 1, dtype=np.uint16)
    _load().synth_E_rate(_p(offsets), len(offsets) - 1, num, den, _p(E))
    return E


# ------------------------------------------------------------------ workloads

@dataclass
class Workload:
    """One synthetic workload: reference (codes + 2-bit), bin geometry, reads, candidates."""
    name: str
    codes: np.ndarray
    ref2bit: np.ndarray
    q: int
    bin_len: int
    overlap: int
    bases: np.ndarray
    read_offsets: np.ndarray
    starts: np.ndarray
    E: np.ndarray
    cand_bins: np.ndarray | None
    cand_offsets: np.ndarray | None
    meta: dict = field(default_factory=dict)

    @property
    def ref_len(self) -> int:
        return len(self.codes)

    @property
    def n_bins(self) -> int:
        return -(-self.ref_len // self.bin_len)

    @property
    def n_reads(self) -> int:
        return len(self.read_offsets) - 1

    @property
    def n_checks(self) -> int:
        return 0 if self.cand_offsets is None else int(self.cand_offsets[-1])


# Seeds: reference 0, reads 1, candidates 2 (repeats use reference seed + 3).
SEED_REF, SEED_READS, SEED_CANDS = 0, 1, 2


def gather_iid(ref_len: int = 1_000_000, n_reads: int = 10_000, L: int = 100, q: int = 5,
               bin_len: int = 256, overlap: int = 100, E: int = 5, k: int = 32,
               sub: float = 0.03, indel: float = 0.01) -> Workload:
    """i.i.d. uniform reference; fixed-length reads at uniform positions;
    candidates = true bin + (k-1) distinct uniform bins.  Defaults: the
    1 Mbp / 10,000 x 100 bp / 32-candidate plain gather workload."""
    codes = ref_iid(ref_len, SEED_REF)
    off = read_offsets(n_reads, L, L, SEED_READS)
    bases, starts = reads(codes, off, SEED_READS, sub, indel)
    n_bins = -(-ref_len // bin_len)
    cb, co = cands_random(starts, bin_len, n_bins, SEED_CANDS, k_fixed=k)
    return Workload(f"gather_iid_{ref_len}bp_q{q}_L{L}_k{k}", codes, pack2bit(codes), q, bin_len, overlap,
                    bases, off, starts, np.full(n_reads, E, dtype=np.uint16), cb, co,
                    {"sub": sub, "indel": indel, "repeat_frac": 0.0})


def gather_seeds(ref_len: int = 100_000_000, n_reads: int = 1_000_000, L: int = 150, q: int = 5,
                 bin_len: int = 256, overlap: int = 150, E: int = 7, cap: int = 1000, repeat_frac: float = 0.30,
                 div_lo: float = 0.10, div_hi: float = 0.20, sub: float = 0.04, indel: float = 0.01,
                 seed_k: int = 12, read_seed: int = SEED_READS) -> Workload:
    """Repeat-rich reference (i.i.d. + planted families); reads at uniform
    positions; candidates = bins of all exact 12-mer seed hits from a CPU
    index, capped per read.  Defaults: the 100 Mbp / 1M x 150 bp workload."""
    codes = ref_with_repeats(ref_len, SEED_REF, repeat_frac, div_lo=div_lo, div_hi=div_hi)
    off = read_offsets(n_reads, L, L, read_seed)
    bases, starts = reads(codes, off, read_seed, sub, indel)
    n_bins = -(-ref_len // bin_len)
    idx = seed_index_for_reads(codes, bases, off, seed_k)
    cb, co = cands_seeds(idx, bases, off, bin_len, n_bins, cap, seed_k)
    del idx
    return Workload(f"gather_seeds_{ref_len}bp_q{q}_L{L}_cap{cap}", codes, pack2bit(codes), q, bin_len, overlap,
                    bases, off, starts, np.full(n_reads, E, dtype=np.uint16), cb, co,
                    {"sub": sub, "indel": indel, "repeat_frac": repeat_frac, "seed_k": seed_k})


def batched_varlen(ref_len: int = 100_000_000, n_reads: int = 2_000_000, lmin: int = 50, lmax: int = 300,
                   q: int = 6, bin_len: int = 256, overlap: int = 300, k_max: int = 5000,
                   repeat_frac: float = 0.30, sub: float = 0.03, indel: float = 0.01,
                   read_seed: int = SEED_READS) -> Workload:
    """Repeat-rich reference; read lengths uniform in [lmin, lmax]; per-read
    E = floor(0.05 L); candidates = true bin + log-uniform [1, k_max] total."""
    codes = ref_with_repeats(ref_len, SEED_REF, repeat_frac)
    off = read_offsets(n_reads, lmin, lmax, read_seed)
    bases, starts = reads(codes, off, read_seed, sub, indel)
    n_bins = -(-ref_len // bin_len)
    cb, co = cands_random(starts, bin_len, n_bins, SEED_CANDS + read_seed - SEED_READS, k_max=k_max)
    return Workload(f"batched_varlen_{ref_len}bp_q{q}_L{lmin}-{lmax}", codes, pack2bit(codes), q, bin_len,
                    overlap, bases, off, starts, E_rate(off), cb, co,
                    {"sub": sub, "indel": indel, "repeat_frac": repeat_frac})


def mixed_seeds(ref_len: int = 3_100_000_000, n_reads: int = 65_536, L: int = 100, q: int = 5,
                bin_len: int = 256, overlap: int = 100, E: int = 5, cap: int = 10_000, repeat_frac: float = 0.40,
                div_lo: float = 0.05, div_hi: float = 0.20, sub: float = 0.03, indel: float = 0.01, seed_k: int = 12,
                read_seed: int = SEED_READS, cand_reads: int | None = None) -> Workload:
    """Genome-scale reference with 40% repeats at 5-20% divergence; 100 bp
    reads; candidates = bins of all exact 12-mer seed hits, capped at
    10,000 per read (dense for reads from repeat families).  cand_reads
    limits the CPU candidate lists to the first cand_reads reads (0: none;
    None: every read)."""
    codes = ref_with_repeats(ref_len, SEED_REF + 100, repeat_frac, div_lo=div_lo, div_hi=div_hi)
    off = read_offsets(n_reads, L, L, read_seed)
    bases, starts = reads(codes, off, read_seed, sub, indel)
    n_bins = -(-ref_len // bin_len)
    m = n_reads if cand_reads is None else min(cand_reads, n_reads)
    cb = co = None
    if m > 0:
        sub_off = off[:m + 1]
        sub_bases = bases[:sub_off[-1]]
        idx = seed_index_for_reads(codes, sub_bases, sub_off, seed_k)
        cb, co = cands_seeds(idx, sub_bases, sub_off, bin_len, n_bins, cap, seed_k)
        del idx
    return Workload(f"mixed_seeds_{ref_len}bp_q{q}_L{L}_cap{cap}", codes, pack2bit(codes), q, bin_len, overlap,
                    bases, off, starts, np.full(n_reads, E, dtype=np.uint16), cb, co,
                    {"sub": sub, "indel": indel, "repeat_frac": repeat_frac, "seed_k": seed_k,
                     "div": [div_lo, div_hi], "cap": cap})


def fullscan(ref_len: int = 3_100_000_000, n_reads: int = 65_536, L: int = 100, q: int = 5,
             bin_len: int = 256, overlap: int = 100, E: int = 5, repeat_frac: float = 0.30,
             sub: float = 0.03, indel: float = 0.01, read_seed: int = SEED_READS) -> Workload:
    """Genome-scale repeat-rich reference, one read batch, no candidate list
    (every bin is scored)."""
    codes = ref_with_repeats(ref_len, SEED_REF, repeat_frac)
    off = read_offsets(n_reads, L, L, read_seed)
    bases, starts = reads(codes, off, read_seed, sub, indel)
    return Workload(f"fullscan_{ref_len}bp_q{q}_L{L}_batch{n_reads}", codes, pack2bit(codes), q, bin_len, overlap,
                    bases, off, starts, np.full(n_reads, E, dtype=np.uint16), None, None,
                    {"sub": sub, "indel": indel, "repeat_frac": repeat_frac})
