"""GRIM-Filter oracle: TEST INFRASTRUCTURE ONLY.

Python handle on ``grim_oracle.c``, the plain single-threaded CPU statement
of the seed-location filter (bins, existence bitvectors, accumulation sums,
threshold; paper Sec. 3.1-3.5).  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grim_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle with gcc (plain -O2, no vector or math tricks)."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src, "-o", tmp])
        os.replace(tmp, out)
    return out


def _bind(lib):
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    sig = {
        "oracle_unpack_ref": (None, [P, I64, P]),
        "oracle_n_bins": (I64, [I64, I32]),
        "oracle_bin_span": (None, [I64, I64, I32, I32, P, P]),
        "oracle_token": (I64, [P, I32]),
        "oracle_threshold": (I64, [I64, I32, I64]),
        "oracle_bits_per_bin": (I64, [I32]),
        "oracle_build_bank": (I32, [P, I64, I32, I32, I32, P]),
        "oracle_sum_one": (I64, [P, I32, P, I64]),
        "oracle_filter": (I32, [P, I64, I32, P, P, I64, P, P, P, P, P]),
        "oracle_scan": (I64, [P, I64, I32, P, P, I64, P, I64, I64, I64, P, P, P]),
        "oracle_bin_row": (I32, [P, I64, I32, I32, I32, I64, P]),
        "oracle_filter_rows": (I32, [P, I64, I32, I32, I32, P, P, I64, P, P, P, P, P]),
        "oracle_sellers": (I64, [P, I64, P, I64]),
        "oracle_seed_candidates": (I64, [P, I64, I32, P, P, I64, I32, I64, I32, I64, P, P]),
        "oracle_locate": (I64, [P, P, P, I64, P, I64, I32, I32, I64, P, P, P, P, P, I64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(path: str | None = None):
    """The oracle library (built on first use).  ``path`` loads another build
    of the same source (the tests use this for planted-mistake variants)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """Thin wrapper: numpy arrays in, numpy arrays out."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else load()

    def unpack_ref(self, ref2bit: np.ndarray, length: int) -> np.ndarray:
        out = np.empty(length, dtype=np.uint8)
        self.lib.oracle_unpack_ref(_p(np.ascontiguousarray(ref2bit, dtype=np.uint8)), length, _p(out))
        return out

    def n_bins(self, length: int, bin_len: int) -> int:
        return int(self.lib.oracle_n_bins(length, bin_len))

    def bin_span(self, b: int, length: int, bin_len: int, overlap: int):
        s, e = ctypes.c_int64(), ctypes.c_int64()
        self.lib.oracle_bin_span(b, length, bin_len, overlap, ctypes.byref(s), ctypes.byref(e))
        return s.value, e.value

    def token(self, codes) -> int:
        a = np.ascontiguousarray(codes, dtype=np.uint8)
        return int(self.lib.oracle_token(_p(a), len(a)))

    def threshold(self, L: int, q: int, E: int) -> int:
        return int(self.lib.oracle_threshold(L, q, E))

    def bits_per_bin(self, q: int) -> int:
        return int(self.lib.oracle_bits_per_bin(q))

    def build_bank(self, ref2bit: np.ndarray, length: int, q: int, bin_len: int, overlap: int) -> np.ndarray:
        """Byte-per-bit bank, shape (n_bins, 4^q), values 0/1."""
        nb = self.n_bins(length, bin_len)
        bank = np.empty((nb, 4 ** q), dtype=np.uint8)
        rc = self.lib.oracle_build_bank(_p(np.ascontiguousarray(ref2bit, dtype=np.uint8)), length, q, bin_len,
                                        overlap, _p(bank))
        if rc != 0:
            raise ValueError(f"oracle_build_bank: {rc}")
        return bank

    def sum_one(self, bank_row: np.ndarray, q: int, read: np.ndarray) -> int:
        r = np.ascontiguousarray(read, dtype=np.uint8)
        return int(self.lib.oracle_sum_one(_p(np.ascontiguousarray(bank_row)), q, _p(r), len(r)))

    def filter(self, bank: np.ndarray, q: int, reads: np.ndarray, read_offsets: np.ndarray,
               cand_bins: np.ndarray, cand_offsets: np.ndarray, E: np.ndarray):
        """Returns (pass u8, sums u32) aligned with cand_bins."""
        n = len(read_offsets) - 1
        nc = int(cand_offsets[-1]) if n > 0 else 0
        pass_ = np.empty(nc, dtype=np.uint8)
        sums = np.empty(nc, dtype=np.uint32)
        rc = self.lib.oracle_filter(_p(bank), bank.shape[0], q, _p(np.ascontiguousarray(reads, dtype=np.uint8)),
                                    _p(np.ascontiguousarray(read_offsets, dtype=np.int64)), n,
                                    _p(np.ascontiguousarray(cand_bins, dtype=np.uint32)),
                                    _p(np.ascontiguousarray(cand_offsets, dtype=np.int64)),
                                    _p(np.ascontiguousarray(E, dtype=np.uint16)), _p(pass_), _p(sums))
        if rc != 0:
            raise ValueError(f"oracle_filter: {rc}")
        return pass_, sums

    def scan(self, bank: np.ndarray, q: int, reads: np.ndarray, read_offsets: np.ndarray, E: np.ndarray,
             bin_begin: int = 0, bin_end: int | None = None):
        """Returns (pair_read, pair_bin, pair_sum), read-major, bins ascending."""
        n = len(read_offsets) - 1
        if bin_end is None:
            bin_end = bank.shape[0]
        args = [_p(bank), bank.shape[0], q, _p(np.ascontiguousarray(reads, dtype=np.uint8)),
                _p(np.ascontiguousarray(read_offsets, dtype=np.int64)), n,
                _p(np.ascontiguousarray(E, dtype=np.uint16)), bin_begin, bin_end]
        cnt = self.lib.oracle_scan(*args, 0, None, None, None)
        if cnt < 0:
            raise ValueError(f"oracle_scan: {cnt}")
        pr = np.empty(cnt, dtype=np.uint32)
        pb = np.empty(cnt, dtype=np.uint32)
        ps = np.empty(cnt, dtype=np.uint32)
        cnt2 = self.lib.oracle_scan(*args, cnt, _p(pr), _p(pb), _p(ps))
        assert cnt2 == cnt
        return pr, pb, ps

    def filter_rows(self, ref2bit: np.ndarray, length: int, q: int, bin_len: int, overlap: int, reads: np.ndarray,
                    read_offsets: np.ndarray, cand_bins: np.ndarray, cand_offsets: np.ndarray, E: np.ndarray):
        """filter() with every candidate's bitvector rebuilt from the reference
        (no bank).  Returns (pass u8, sums u32) aligned with cand_bins."""
        n = len(read_offsets) - 1
        nc = int(cand_offsets[-1]) - int(cand_offsets[0]) if n > 0 else 0
        co = np.ascontiguousarray(cand_offsets, dtype=np.int64) - int(cand_offsets[0])
        ro = np.ascontiguousarray(read_offsets, dtype=np.int64) - int(read_offsets[0])
        pass_ = np.empty(nc, dtype=np.uint8)
        sums = np.empty(nc, dtype=np.uint32)
        rc = self.lib.oracle_filter_rows(_p(np.ascontiguousarray(ref2bit, dtype=np.uint8)), length, q, bin_len,
                                         overlap, _p(np.ascontiguousarray(reads, dtype=np.uint8)), _p(ro), n,
                                         _p(np.ascontiguousarray(cand_bins, dtype=np.uint32)), _p(co),
                                         _p(np.ascontiguousarray(E, dtype=np.uint16)), _p(pass_), _p(sums))
        if rc != 0:
            raise ValueError(f"oracle_filter_rows: {rc}")
        return pass_, sums

    def bin_row(self, ref2bit: np.ndarray, length: int, q: int, bin_len: int, overlap: int, b: int) -> np.ndarray:
        row = np.empty(4 ** q, dtype=np.uint8)
        rc = self.lib.oracle_bin_row(_p(np.ascontiguousarray(ref2bit, dtype=np.uint8)), length, q, bin_len,
                                     overlap, b, _p(row))
        if rc != 0:
            raise ValueError(f"oracle_bin_row: {rc}")
        return row

    def sellers(self, read: np.ndarray, text: np.ndarray) -> int:
        r = np.ascontiguousarray(read, dtype=np.uint8)
        t = np.ascontiguousarray(text, dtype=np.uint8)
        return int(self.lib.oracle_sellers(_p(r), len(r), _p(t), len(t)))

    def seed_candidates(self, ref_codes: np.ndarray, k: int, reads: np.ndarray, read_offsets: np.ndarray,
                        bin_len: int, n_bins: int, cap: int):
        """Candidate bins from exact seed locations (Sec. 1 Fig. 1, Sec. 3.3).
        Returns (cand_bins u32, cand_offsets i64)."""
        ref = np.ascontiguousarray(ref_codes, dtype=np.uint8)
        rd = np.ascontiguousarray(reads, dtype=np.uint8)
        off = np.ascontiguousarray(read_offsets, dtype=np.int64)
        n = len(off) - 1
        co = np.empty(n + 1, dtype=np.int64)
        args = [_p(ref), len(ref), k, _p(rd), _p(off), n, bin_len, n_bins, cap]
        total = self.lib.oracle_seed_candidates(*args, 0, None, _p(co))
        if total < 0:
            raise ValueError(f"oracle_seed_candidates: {total}")
        cb = np.empty(max(int(total), 1), dtype=np.uint32)
        total2 = self.lib.oracle_seed_candidates(*args, int(total), _p(cb), _p(co))
        assert total2 == total
        return cb[:total], co

    def locate(self, pass_: np.ndarray, cand_bins: np.ndarray, cand_offsets: np.ndarray, ref_codes: np.ndarray,
               bin_len: int, overlap: int, seg_stride: int = 0):
        """Seed Location Checker (Sec. 3.3, Fig. 4): passing candidates with
        their reference segments.  Returns (read, bin, begin, end, segments)."""
        ps = np.ascontiguousarray(pass_, dtype=np.uint8)
        cb = np.ascontiguousarray(cand_bins, dtype=np.uint32)
        co = np.ascontiguousarray(cand_offsets, dtype=np.int64)
        ref = np.ascontiguousarray(ref_codes, dtype=np.uint8)
        n = len(co) - 1
        m = int(np.count_nonzero(ps))
        rd, bn = np.empty(m, np.uint32), np.empty(m, np.uint32)
        be, en = np.empty(m, np.int64), np.empty(m, np.int64)
        seg = np.empty((m, seg_stride), np.uint8) if seg_stride > 0 else None
        got = self.lib.oracle_locate(_p(ps), _p(cb), _p(co), n, _p(ref), len(ref), bin_len, overlap, m, _p(rd),
                                     _p(bn), _p(be), _p(en), _p(seg), seg_stride)
        if got != m:
            raise ValueError(f"oracle_locate: {got}")
        return rd, bn, be, en, seg
