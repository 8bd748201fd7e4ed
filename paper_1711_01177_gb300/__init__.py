"""Python binding of libgrim, the GB300 seed-location filter.

Argument marshalling only: every step of the filter runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current stream.  The
functions carry the C ABI's names (include/grim.h); a failing status raises
GrimError.  There is no CPU fallback: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from ._build import LIB as _LIB_PATH
from ._build import build as _build_lib

(GRIM_OK, GRIM_EINVAL, GRIM_EDATA, GRIM_ENOMEM, GRIM_ECUDA, GRIM_EOVERFLOW, GRIM_ETIMEOUT, GRIM_ENOTSUP,
 GRIM_ESCRATCH, GRIM_EIO) = range(10)
GRIM_SCAN_NOALLOC_SCRATCH_BYTES = 64 << 20
GRIM_FLAG_BAD_BASE = 0x1
GRIM_FLAG_BAD_BIN = 0x2
GRIM_FLAG_BAD_OFFSETS = 0x4
GRIM_FLAG_LONG_READ = 0x8
GRIM_FLAG_OVERFLOW = 0x10
GRIM_FLAG_TIMEOUT = 0x20
GRIM_MAX_Q = 6
GRIM_MAX_SCAN_Q = 5
GRIM_MAX_READ_LEN = 65535

# every symbol include/grim.h declares, with (restype, argtypes)
_P, _I64, _I32, _U32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32
SIGNATURES = {
    "grim_strerror": (ctypes.c_char_p, [_I32]),
    "grim_last_cuda_error": (_I32, []),
    "grim_release_scratch": (_I32, []),
    "grim_wait_selfcheck": (_I32, [ctypes.c_ulonglong, _P]),
    "grim_fill_E_rate": (_I32, [_P, _I64, _I32, _I32, _I32, _P, _P]),
    "grim_build_bank": (_I32, [_P, _I64, _I32, _I32, _I32, _P, ctypes.POINTER(_P)]),
    "grim_bank_info": (_I32, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "grim_build_bank_into": (_I32, [_P, _P, _P]),
    "grim_scan_mma_kind": (ctypes.c_char_p, []),
    "grim_bank_status": (_I32, [_P, _P, ctypes.POINTER(_U32)]),
    "grim_bank_free": (_I32, [_P]),
    "grim_filter": (_I32, [_P, _P, _P, _I64, _P, _P, _P, _P, _P, _P]),
    "grim_scan": (_I32, [_P, _P, _P, _I64, _P, _I64, _I64, _P, _P, _P, _I64, _P, _P, _P]),
    "grim_scan_noalloc": (_I32, [_P, _P, _P, _I64, _P, _I64, _I64, _P, _P, _P, _I64, _P, _P, _P]),
    "grim_filter_batched": (_I32, [_P, _P, _P, _I64, _P, _P, _P, _P, _P, _P, _P]),
    "grim_filter_host": (_I32, [_P, _P, _P, _I64, _P, _P, _P, _P, _I64, _P]),
    "grim_autotune": (_I32, [_P, _P, _P, _I64, _P, _P, _P, _P, _P, _P]),
    "grim_choose_form": (_I32, [_P, _I64, _I64, ctypes.POINTER(_I32)]),
    "grim_filter_auto": (_I32, [_P, _P, _P, _I64, _P, _P, _P, _P, _I64, ctypes.POINTER(_I64), _P]),
    "grim_seed_index_build": (_I32, [_P, _I64, _I32, _P, ctypes.POINTER(_P)]),
    "grim_seed_index_info": (_I32, [_P, _P, _P, _P, _P]),
    "grim_seed_index_free": (_I32, [_P]),
    "grim_seed_candidates": (_I32, [_P, _P, _P, _I64, _I32, _I64, _I32, _P, _I64, _P, ctypes.POINTER(_I64), _P]),
    "grim_locate": (_I32, [_P, _P, _P, _P, _I64, _I64, _P, _P, _P, _P, _P, _P, _I64, _I64, _P, _P]),
    "grim_bank_save": (_I32, [_P, ctypes.c_char_p, _P]),
    "grim_bank_load": (_I32, [ctypes.c_char_p, _P, ctypes.POINTER(_P)]),
    "grim_pack_mask": (_I32, [_P, _I64, _P, _P]),
    "grim_verify": (_I32, [_P, _P, _P, _P, _I64, _P, _P, _I64, _P, _P]),
    "grim_map": (_I32, [_P, _P, _P, _P, _P, _I64, _P, _I32, _I64, _P, _P, _P, _I64, ctypes.POINTER(_I64), _P, _P]),
    "grim_verify_stats": (_I32, [_P, _P, _P, _P, _I64, _I64, _P, _P]),
    "grim_fault_inject": (_I32, [_I32, _I64]),
    "grim_peak": (_I32, [_I32, _I64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float), _P]),
    "grim_fault_pending": (_I32, [ctypes.POINTER(_I64)]),
}
GRIM_FAULT_NONE, GRIM_FAULT_ALLOC, GRIM_FAULT_LAUNCH = 0, 1, 2
(GRIM_PEAK_L2_READ, GRIM_PEAK_E4M3, GRIM_PEAK_MXF4, GRIM_PEAK_MXF4_TMEM_A, GRIM_PEAK_E4M3_TMEM_A,
 GRIM_PEAK_INT8_MMA_SYNC, GRIM_PEAK_MXF4_TMEM_A_N128, GRIM_PEAK_E4M3_TMEM_A_N128) = range(1, 9)
GRIM_FORM_GATHER, GRIM_FORM_SCAN = 0, 1


class GrimTune(ctypes.Structure):
    """Launch shape of grim_filter_batched (zero fields take defaults)."""
    _fields_ = [("warps_per_cta", ctypes.c_int32), ("reads_per_claim", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("batch_reads", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

_lib = None


class GrimError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = load().grim_strerror(status).decode()
        if status in (GRIM_ECUDA, GRIM_ENOMEM):
            msg += f" (cudaError {load().grim_last_cuda_error()})"
        super().__init__(f"{what}: {msg} [status {status}]")


def build(force: bool = False) -> str:
    """Compile libgrim.so for sm_103a (nvcc) next to this file."""
    return _build_lib(force=force)


def load(path: str | None = None):
    """The loaded libgrim (raises if it has not been built)."""
    global _lib
    if _lib is None:
        p = path or _LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libgrim.so is not built ({p}); call paper_1711_01177_gb300.build()")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def grim_wait_selfcheck(limit_ns: int, stream=None) -> int:
    """Status of the bounded-wait diagnostic (GRIM_ETIMEOUT when it works)."""
    return load().grim_wait_selfcheck(limit_ns, _stream_ptr(stream))


def grim_fault_inject(kind: int, nth: int = 1) -> None:
    """Arm the library's host-side fault injection: the nth allocation
    (GRIM_FAULT_ALLOC) or kernel launch (GRIM_FAULT_LAUNCH) from now on
    fails; GRIM_FAULT_NONE disarms."""
    _check(load().grim_fault_inject(kind, nth), "grim_fault_inject")


def grim_fault_pending() -> tuple[int, int]:
    """(armed kind, events left before it fires); (GRIM_FAULT_NONE, 0) once fired."""
    left = ctypes.c_int64(0)
    kind = load().grim_fault_pending(ctypes.byref(left))
    return kind, left.value


def grim_peak(kind: int, work: int, stream=None) -> tuple[float, float]:
    """(units, ms) of one timed peak launch: bytes (GRIM_PEAK_L2_READ) or
    flops / ops (the tensor kinds) and its CUDA-event time."""
    u, t = ctypes.c_double(), ctypes.c_float()
    _check(load().grim_peak(kind, work, ctypes.byref(u), ctypes.byref(t), _stream_ptr(stream)), "grim_peak")
    return u.value, t.value


def grim_release_scratch() -> None:
    """Return the library's cached scratch memory on the current device."""
    _check(load().grim_release_scratch(), "grim_release_scratch")


def _check(status: int, what: str):
    if status != GRIM_OK:
        raise GrimError(status, what)


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


_DUMMY = {}


def _dev_ptr(t: torch.Tensor | None, name: str, elem_size: int | None = None, nullable: bool = False):
    if t is None:
        if nullable:
            return None
        raise ValueError(f"{name} is required")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if elem_size is not None and t.element_size() != elem_size:
        raise ValueError(f"{name} must have {elem_size}-byte elements")
    if t.numel() == 0:  # the C ABI wants a valid pointer even for empty arrays
        key = (t.device.index, elem_size or 1)
        if key not in _DUMMY:
            _DUMMY[key] = torch.zeros(16, dtype=torch.uint8, device=t.device)
        return ctypes.c_void_p(_DUMMY[key].data_ptr())
    return ctypes.c_void_p(t.data_ptr())


class _CudaArray:
    """Minimal __cuda_array_interface__ holder to view library memory."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


class Bank:
    """A built bank: existence bitvectors of every bin, owned by libgrim."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        L, nb, rw = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        q, bl, ov = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        bits = ctypes.c_void_p()
        _check(load().grim_bank_info(handle, ctypes.byref(L), ctypes.byref(nb), ctypes.byref(q), ctypes.byref(bl),
                                     ctypes.byref(ov), ctypes.byref(rw), ctypes.byref(bits)), "grim_bank_info")
        self.len, self.n_bins, self.row_words = L.value, nb.value, rw.value
        self.q, self.bin_len, self.overlap = q.value, bl.value, ov.value
        self.bits_ptr = bits.value

    @property
    def handle(self):
        return self._h

    def bits(self) -> torch.Tensor:
        """Zero-copy int32 view (n_bins, row_words) of the bank in HBM."""
        arr = _CudaArray(self.bits_ptr, (self.n_bins, self.row_words), "<i4")
        return torch.as_tensor(arr, device="cuda")

    def free(self):
        if self._h is not None and self._h.value:
            _check(load().grim_bank_free(self._h), "grim_bank_free")
        self._h = None

    def __del__(self):
        try:
            if self._h is not None and self._h.value and _lib is not None:
                _lib.grim_bank_free(self._h)
        except Exception:
            pass


def grim_build_bank(ref2bit: torch.Tensor, length: int, q: int, bin_len: int, overlap: int, stream=None) -> Bank:
    """Existence bitvectors of every bin of a 2-bit packed reference (Sec. 3.1)."""
    h = ctypes.c_void_p()
    _check(load().grim_build_bank(_dev_ptr(ref2bit, "ref2bit", 1), length, q, bin_len, overlap, _stream_ptr(stream),
                                  ctypes.byref(h)), "grim_build_bank")
    return Bank(h)


def grim_build_bank_into(bank: Bank, ref2bit: torch.Tensor, stream=None) -> None:
    """Recompute the bank's rows from a reference of its length (no allocation)."""
    _check(load().grim_build_bank_into(bank.handle, _dev_ptr(ref2bit, "ref2bit", 1), _stream_ptr(stream)),
           "grim_build_bank_into")


def grim_scan_kind() -> str:
    """The full scan's operand type as named in the peaks: "e4m3" or "mxf4"."""
    k = load().grim_scan_mma_kind().decode()
    return "e4m3" if k == "f8f6f4" else k


def grim_bank_status(bank: Bank, stream=None):
    """Synchronise and read+clear the bank's device flags: (status, flags)."""
    f = ctypes.c_uint32()
    st = load().grim_bank_status(bank.handle, _stream_ptr(stream), ctypes.byref(f))
    return st, f.value


def grim_filter(bank: Bank, reads: torch.Tensor, read_offsets: torch.Tensor, cand_bins: torch.Tensor,
                cand_offsets: torch.Tensor, E: torch.Tensor, pass_out: torch.Tensor | None = None,
                sums: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Seed location filter bitmask (one u8 per candidate) for every
    (read, candidate bin) pair (Sec. 3.2-3.3).  Returns pass_out."""
    n_reads = read_offsets.numel() - 1
    if n_reads < 0:
        raise ValueError("read_offsets needs n_reads + 1 entries")
    if cand_offsets.numel() != n_reads + 1 or E.numel() != n_reads:
        raise ValueError("cand_offsets / E sizes do not match read_offsets")
    if pass_out is None:
        pass_out = torch.empty(cand_bins.numel(), dtype=torch.uint8, device=cand_bins.device)
    _check(load().grim_filter(bank.handle, _dev_ptr(reads, "reads", 1), _dev_ptr(read_offsets, "read_offsets", 8),
                              n_reads, _dev_ptr(cand_bins, "cand_bins", 4), _dev_ptr(cand_offsets, "cand_offsets", 8),
                              _dev_ptr(E, "E", 2), _dev_ptr(pass_out, "pass", 1), _dev_ptr(sums, "sums", 2, True),
                              _stream_ptr(stream)), "grim_filter")
    return pass_out


class ScanResult:
    """Passing (read, bin) pairs of a full scan, in no particular order."""

    def __init__(self, pair_read, pair_bin, pair_sum, n_pairs, read_pass):
        self.pair_read, self.pair_bin, self.pair_sum = pair_read, pair_bin, pair_sum
        self.n_pairs_dev, self.read_pass = n_pairs, read_pass

    @property
    def n_pairs(self) -> int:
        return int(self.n_pairs_dev.item())


def grim_scan(bank: Bank, reads: torch.Tensor, read_offsets: torch.Tensor, E: torch.Tensor, bin_begin: int = 0,
              bin_end: int | None = None, cap: int = 1 << 20, with_sums: bool = True, with_read_pass: bool = False,
              out: ScanResult | None = None, stream=None, _entry: str = "grim_scan") -> ScanResult:
    """Every read against every bin of [bin_begin, bin_end) on the tensor
    cores (Sec. 3.2 over the bin window of Sec. 6.1).  Pairs beyond `cap`
    are counted but not written (GRIM_FLAG_OVERFLOW)."""
    n_reads = read_offsets.numel() - 1
    if n_reads < 0 or E.numel() != n_reads:
        raise ValueError("read_offsets / E sizes do not match")
    if bin_end is None:
        bin_end = bank.n_bins
    dev = read_offsets.device
    if out is None:
        out = ScanResult(torch.empty(max(cap, 1), dtype=torch.int32, device=dev),
                         torch.empty(max(cap, 1), dtype=torch.int32, device=dev),
                         torch.empty(max(cap, 1), dtype=torch.int16, device=dev) if with_sums else None,
                         torch.zeros(1, dtype=torch.int64, device=dev),
                         torch.empty(max(n_reads, 1), dtype=torch.int32, device=dev) if with_read_pass else None)
        cap_eff = cap
    else:
        cap_eff = out.pair_read.numel()
    _check(getattr(load(), _entry)(bank.handle, _dev_ptr(reads, "reads", 1), _dev_ptr(read_offsets, "read_offsets", 8),
                            n_reads, _dev_ptr(E, "E", 2), bin_begin, bin_end, _dev_ptr(out.pair_read, "pair_read", 4),
                            _dev_ptr(out.pair_bin, "pair_bin", 4), _dev_ptr(out.pair_sum, "pair_sum", 2, True), cap_eff,
                            _dev_ptr(out.n_pairs_dev, "n_pairs", 8), _dev_ptr(out.read_pass, "read_pass", 4, True),
                            _stream_ptr(stream)), _entry)
    return out


def grim_scan_noalloc(bank: Bank, reads: torch.Tensor, read_offsets: torch.Tensor, E: torch.Tensor,
                      bin_begin: int = 0, bin_end: int | None = None, cap: int = 1 << 20, with_sums: bool = True,
                      with_read_pass: bool = False, out: ScanResult | None = None, stream=None) -> ScanResult:
    """grim_scan without device allocation, for callers that cannot allocate
    when they call the filter: the library's fixed 64 MiB scratch is used
    instead (GRIM_ESCRATCH beyond it; overlapping calls race on it)."""
    return grim_scan(bank, reads, read_offsets, E, bin_begin, bin_end, cap, with_sums, with_read_pass, out, stream,
                     _entry="grim_scan_noalloc")


def grim_filter_batched(bank: Bank, reads: torch.Tensor, read_offsets: torch.Tensor, cand_bins: torch.Tensor,
                        cand_offsets: torch.Tensor, E: torch.Tensor, pass_out: torch.Tensor | None = None,
                        sums: torch.Tensor | None = None, tune: GrimTune | None = None, stream=None) -> torch.Tensor:
    """grim_filter's outputs from persistent launches, one per batch of reads,
    captured in a CUDA graph that identical later calls replay."""
    n_reads = read_offsets.numel() - 1
    if n_reads < 0 or cand_offsets.numel() != n_reads + 1 or E.numel() != n_reads:
        raise ValueError("read_offsets / cand_offsets / E sizes do not match")
    if pass_out is None:
        pass_out = torch.empty(cand_bins.numel(), dtype=torch.uint8, device=cand_bins.device)
    _check(load().grim_filter_batched(bank.handle, _dev_ptr(reads, "reads", 1),
                                      _dev_ptr(read_offsets, "read_offsets", 8), n_reads,
                                      _dev_ptr(cand_bins, "cand_bins", 4), _dev_ptr(cand_offsets, "cand_offsets", 8),
                                      _dev_ptr(E, "E", 2), _dev_ptr(pass_out, "pass", 1),
                                      _dev_ptr(sums, "sums", 2, True), ctypes.byref(tune) if tune is not None else None,
                                      _stream_ptr(stream)), "grim_filter_batched")
    return pass_out


def grim_autotune(bank: Bank, reads: torch.Tensor, read_offsets: torch.Tensor, cand_bins: torch.Tensor,
                  cand_offsets: torch.Tensor, E: torch.Tensor, pass_out: torch.Tensor | None = None,
                  stream=None) -> GrimTune:
    """Time the batched filter's launch shapes on the first batch; returns the
    fastest (also remembered for grim_filter_batched(tune=None))."""
    n_reads = read_offsets.numel() - 1
    if pass_out is None:
        pass_out = torch.empty(cand_bins.numel(), dtype=torch.uint8, device=cand_bins.device)
    t = GrimTune()
    _check(load().grim_autotune(bank.handle, _dev_ptr(reads, "reads", 1), _dev_ptr(read_offsets, "read_offsets", 8),
                                n_reads, _dev_ptr(cand_bins, "cand_bins", 4),
                                _dev_ptr(cand_offsets, "cand_offsets", 8), _dev_ptr(E, "E", 2),
                                _dev_ptr(pass_out, "pass", 1), ctypes.byref(t), _stream_ptr(stream)), "grim_autotune")
    return t


def grim_choose_form(bank: Bank, n_reads: int, n_checks: int) -> int:
    """GRIM_FORM_GATHER or GRIM_FORM_SCAN for a batch (cost model)."""
    f = ctypes.c_int()
    _check(load().grim_choose_form(bank.handle, n_reads, n_checks, ctypes.byref(f)), "grim_choose_form")
    return f.value


def grim_filter_auto(bank: Bank, reads: torch.Tensor, read_offsets: torch.Tensor, cand_bins: torch.Tensor,
                     cand_offsets: torch.Tensor, E: torch.Tensor, pass_out: torch.Tensor | None = None,
                     batch_reads: int = 262144, stream=None):
    """grim_filter's pass bytes, each batch by the cheaper form; returns
    (pass_out, reads that went through the full scan)."""
    n_reads = read_offsets.numel() - 1
    if n_reads < 0 or cand_offsets.numel() != n_reads + 1 or E.numel() != n_reads:
        raise ValueError("read_offsets / cand_offsets / E sizes do not match")
    if pass_out is None:
        pass_out = torch.empty(cand_bins.numel(), dtype=torch.uint8, device=cand_bins.device)
    scanned = ctypes.c_int64()
    _check(load().grim_filter_auto(bank.handle, _dev_ptr(reads, "reads", 1), _dev_ptr(read_offsets, "read_offsets", 8),
                                   n_reads, _dev_ptr(cand_bins, "cand_bins", 4),
                                   _dev_ptr(cand_offsets, "cand_offsets", 8), _dev_ptr(E, "E", 2),
                                   _dev_ptr(pass_out, "pass", 1), batch_reads, ctypes.byref(scanned),
                                   _stream_ptr(stream)), "grim_filter_auto")
    return pass_out, scanned.value


class SeedIndex:
    """A seed location table (every k-mer's reference positions), owned by libgrim."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        L, k = ctypes.c_int64(), ctypes.c_int()
        off, pos = ctypes.c_void_p(), ctypes.c_void_p()
        _check(load().grim_seed_index_info(handle, ctypes.byref(L), ctypes.byref(k), ctypes.byref(off),
                                           ctypes.byref(pos)), "grim_seed_index_info")
        self.len, self.k = L.value, k.value
        self._off, self._pos = off.value, pos.value

    @property
    def handle(self):
        return self._h

    def offsets(self) -> torch.Tensor:
        """Zero-copy int32 view of the 4^k + 1 CSR offsets (u32 values)."""
        return torch.as_tensor(_CudaArray(self._off, ((1 << (2 * self.k)) + 1,), "<i4"), device="cuda")

    def positions(self) -> torch.Tensor:
        """Zero-copy int32 view of the len - k + 1 positions (u32 values)."""
        return torch.as_tensor(_CudaArray(self._pos, (self.len - self.k + 1,), "<i4"), device="cuda")

    def free(self):
        if self._h is not None and self._h.value:
            _check(load().grim_seed_index_free(self._h), "grim_seed_index_free")
        self._h = None

    def __del__(self):
        try:
            if self._h is not None and self._h.value and _lib is not None:
                _lib.grim_seed_index_free(self._h)
        except Exception:
            pass


def grim_seed_index_build(ref2bit: torch.Tensor, length: int, k: int = 12, stream=None) -> SeedIndex:
    """Reference positions of every k-mer (the mapper's seed table, Sec. 1 Fig. 1)."""
    h = ctypes.c_void_p()
    _check(load().grim_seed_index_build(_dev_ptr(ref2bit, "ref2bit", 1), length, k, _stream_ptr(stream),
                                        ctypes.byref(h)), "grim_seed_index_build")
    return SeedIndex(h)


def grim_seed_candidates(idx: SeedIndex, reads: torch.Tensor, read_offsets: torch.Tensor, bin_len: int,
                         n_bins: int, cap: int, capacity: int | None = None, stream=None):
    """Candidate bins from exact seed locations (Sec. 3.3).  Returns
    (cand_bins u32-as-int32, cand_offsets int64); synchronises the stream."""
    n_reads = read_offsets.numel() - 1
    if n_reads < 0:
        raise ValueError("read_offsets needs n_reads + 1 entries")
    co = torch.empty(n_reads + 1, dtype=torch.int64, device=read_offsets.device)
    if capacity is None:
        capacity = max(1024, n_reads * 64)
    total = ctypes.c_int64()
    for _ in range(2):
        cb = torch.empty(max(capacity, 1), dtype=torch.int32, device=read_offsets.device)
        st = load().grim_seed_candidates(idx.handle, _dev_ptr(reads, "reads", 1),
                                         _dev_ptr(read_offsets, "read_offsets", 8), n_reads, bin_len, n_bins, cap,
                                         _dev_ptr(cb, "cand_bins", 4), capacity, _dev_ptr(co, "cand_offsets", 8),
                                         ctypes.byref(total), _stream_ptr(stream))
        if st == GRIM_EOVERFLOW:
            capacity = total.value
            continue
        _check(st, "grim_seed_candidates")
        return cb[:total.value], co
    raise GrimError(GRIM_EOVERFLOW, "grim_seed_candidates")


class Located:
    """Passing locations from grim_locate: read, bin, span [begin, end) and
    optional segment rows; `n` = number of passing locations."""

    def __init__(self, read, bin_, begin, end, segments, n):
        self.read, self.bin, self.begin, self.end, self.segments, self.n = read, bin_, begin, end, segments, n


def grim_locate(bank: Bank, cand_bins: torch.Tensor, cand_offsets: torch.Tensor, pass_: torch.Tensor,
                ref2bit: torch.Tensor | None = None, seg_stride: int = 0, capacity: int | None = None,
                stream=None) -> Located:
    """Seed Location Checker (Sec. 3.3, Fig. 4): passing locations and their
    reference segments.  capacity defaults to the number of passing bytes."""
    n_reads = cand_offsets.numel() - 1
    n_cands = pass_.numel()
    dev = pass_.device
    if capacity is None:
        capacity = int(torch.count_nonzero(pass_).item()) if n_cands else 0
    rd = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    bn = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    be = torch.empty(max(capacity, 1), dtype=torch.int64, device=dev)
    en = torch.empty(max(capacity, 1), dtype=torch.int64, device=dev)
    seg = torch.empty((max(capacity, 1), seg_stride), dtype=torch.uint8, device=dev) if seg_stride > 0 else None
    n_loc = torch.zeros(1, dtype=torch.int64, device=dev)
    _check(load().grim_locate(bank.handle, _dev_ptr(ref2bit, "ref2bit", 1, True), _dev_ptr(cand_bins, "cand_bins", 4),
                              _dev_ptr(cand_offsets, "cand_offsets", 8), n_reads, n_cands,
                              _dev_ptr(pass_, "pass", 1), _dev_ptr(rd, "loc_read", 4), _dev_ptr(bn, "loc_bin", 4),
                              _dev_ptr(be, "loc_begin", 8), _dev_ptr(en, "loc_end", 8),
                              _dev_ptr(seg, "segments", 1, True), seg_stride, capacity,
                              _dev_ptr(n_loc, "n_loc", 8), _stream_ptr(stream)), "grim_locate")
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()
    n = int(n_loc.item())
    m = min(n, capacity)
    return Located(rd[:m], bn[:m], be[:m], en[:m], seg[:m] if seg is not None else None, n)


def grim_verify(bank: Bank, ref2bit: torch.Tensor, reads: torch.Tensor, read_offsets: torch.Tensor,
                loc_read: torch.Tensor, loc_bin: torch.Tensor, dist: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """Semi-global edit distance of each location's read against its bin's
    span (the aligner's check behind Sec. 5's metrics).  Returns dist (int16
    holding u16 values)."""
    n_loc = loc_read.numel()
    if loc_bin.numel() != n_loc:
        raise ValueError("loc_read and loc_bin differ in length")
    if dist is None:
        dist = torch.empty(n_loc, dtype=torch.int16, device=loc_read.device)
    _check(load().grim_verify(bank.handle, _dev_ptr(ref2bit, "ref2bit", 1), _dev_ptr(reads, "reads", 1),
                              _dev_ptr(read_offsets, "read_offsets", 8), read_offsets.numel() - 1,
                              _dev_ptr(loc_read, "loc_read", 4), _dev_ptr(loc_bin, "loc_bin", 4), n_loc,
                              _dev_ptr(dist, "dist", 2), _stream_ptr(stream)), "grim_verify")
    return dist


def grim_verify_stats(dist: torch.Tensor, loc_read: torch.Tensor, E: torch.Tensor, pass_: torch.Tensor | None = None,
                      stream=None) -> dict:
    """Passing / rejected locations with and without a mapping (Sec. 5):
    {"passed", "passed_unmapped", "rejected", "rejected_mapped"}; the
    paper's false negative rate is passed_unmapped / passed."""
    counts = torch.empty(4, dtype=torch.int64, device=dist.device)
    _check(load().grim_verify_stats(_dev_ptr(pass_, "pass", 1, True), _dev_ptr(dist, "dist", 2),
                                    _dev_ptr(loc_read, "loc_read", 4), _dev_ptr(E, "E", 2), E.numel(), dist.numel(),
                                    _dev_ptr(counts, "counts", 8), _stream_ptr(stream)), "grim_verify_stats")
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()
    c = counts.tolist()
    return {"passed": c[0], "passed_unmapped": c[1], "rejected": c[2], "rejected_mapped": c[3]}


def grim_bank_save(bank: Bank, path: str, stream=None) -> None:
    """Write the bank to a file (built once per reference, Sec. 3.1)."""
    _check(load().grim_bank_save(bank.handle, os.fsencode(path), _stream_ptr(stream)), "grim_bank_save")


def grim_bank_load(path: str, stream=None) -> Bank:
    """A bank read back from grim_bank_save's file onto the current device."""
    h = ctypes.c_void_p()
    _check(load().grim_bank_load(os.fsencode(path), _stream_ptr(stream), ctypes.byref(h)), "grim_bank_load")
    return Bank(h)


def grim_fill_E_rate(read_offsets: torch.Tensor, num: int = 5, den: int = 100, round_up: bool = False,
                     E: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Per-read edit budgets floor(num * L / den) (ceil with round_up), as
    int16 holding u16 (Sec. 3.4, Sec. 6.1)."""
    n = read_offsets.numel() - 1
    if n < 0:
        raise ValueError("read_offsets needs n_reads + 1 entries")
    if E is None:
        E = torch.empty(max(n, 1), dtype=torch.int16, device=read_offsets.device)
    _check(load().grim_fill_E_rate(_dev_ptr(read_offsets, "read_offsets", 8), n, num, den, int(bool(round_up)),
                                   _dev_ptr(E, "E", 2), _stream_ptr(stream)), "grim_fill_E_rate")
    return E[:n]


def grim_pack_mask(pass_: torch.Tensor, bits: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """One bit per location (Sec. 3.3): bit i % 32 of word i / 32 (int32
    tensor holding u32 words)."""
    n = pass_.numel()
    if bits is None:
        bits = torch.empty(max(1, (n + 31) // 32), dtype=torch.int32, device=pass_.device)
    _check(load().grim_pack_mask(_dev_ptr(pass_, "pass", 1), n, _dev_ptr(bits, "bits", 4), _stream_ptr(stream)),
           "grim_pack_mask")
    return bits[:(n + 31) // 32]


class Mapped:
    """grim_map's outputs: every passing location (read, bin) with its edit
    distance; `n` = number of passing locations."""

    def __init__(self, read, bin_, dist, n):
        self.read, self.bin, self.dist, self.n = read, bin_, dist, n


def grim_map(bank: Bank, idx: SeedIndex, ref2bit: torch.Tensor, reads: torch.Tensor, read_offsets: torch.Tensor,
             E: torch.Tensor, cap: int = 10_000, batch_reads: int = 0, capacity: int | None = None, stream=None,
             align_stream=None) -> Mapped:
    """Seed candidates -> filter -> Seed Location Checker -> edit distances,
    batch by batch with alignment overlapping the next batch's filtering
    (Sec. 4.2 / 6.1).  Synchronises both streams."""
    n_reads = read_offsets.numel() - 1
    if capacity is None:
        capacity = max(1024, n_reads * 64)
    n = ctypes.c_int64()
    for _ in range(2):
        rd = torch.empty(max(capacity, 1), dtype=torch.int32, device=reads.device)
        bn = torch.empty(max(capacity, 1), dtype=torch.int32, device=reads.device)
        ds = torch.empty(max(capacity, 1), dtype=torch.int16, device=reads.device)
        st = load().grim_map(bank.handle, idx.handle, _dev_ptr(ref2bit, "ref2bit", 1), _dev_ptr(reads, "reads", 1),
                             _dev_ptr(read_offsets, "read_offsets", 8), n_reads, _dev_ptr(E, "E", 2), cap,
                             batch_reads, _dev_ptr(rd, "loc_read", 4), _dev_ptr(bn, "loc_bin", 4),
                             _dev_ptr(ds, "loc_dist", 2), capacity, ctypes.byref(n), _stream_ptr(stream),
                             ctypes.c_void_p(align_stream.cuda_stream) if align_stream is not None else None)
        if st == GRIM_EOVERFLOW:
            capacity = n.value
            continue
        _check(st, "grim_map")
        return Mapped(rd[:n.value], bn[:n.value], ds[:n.value], n.value)
    raise GrimError(GRIM_EOVERFLOW, "grim_map")


def _host_ptr(t: torch.Tensor, name: str, elem_size: int):
    if t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.element_size() != elem_size:
        raise ValueError(f"{name} must have {elem_size}-byte elements")
    return ctypes.c_void_p(t.data_ptr()) if t.numel() else ctypes.c_void_p(ctypes.addressof(_HOST_DUMMY))


_HOST_DUMMY = ctypes.create_string_buffer(16)


def grim_filter_host(bank: Bank, reads: torch.Tensor, read_offsets: torch.Tensor, cand_bins: torch.Tensor,
                     cand_offsets: torch.Tensor, E: torch.Tensor, pass_out: torch.Tensor | None = None,
                     chunk_reads: int = 0, stream=None) -> torch.Tensor:
    """grim_filter on host tensors (page-locked for overlapped copies):
    chunks of reads copied in, filtered and copied out on overlapping
    streams.  Returns pass_out (host u8); synchronises the stream."""
    n_reads = read_offsets.numel() - 1
    if n_reads < 0:
        raise ValueError("read_offsets needs n_reads + 1 entries")
    if cand_offsets.numel() != n_reads + 1 or E.numel() != n_reads:
        raise ValueError("cand_offsets / E sizes do not match read_offsets")
    if pass_out is None:
        pass_out = torch.empty(cand_bins.numel(), dtype=torch.uint8)
    _check(load().grim_filter_host(bank.handle, _host_ptr(reads, "reads", 1),
                                   _host_ptr(read_offsets, "read_offsets", 8), n_reads,
                                   _host_ptr(cand_bins, "cand_bins", 4),
                                   _host_ptr(cand_offsets, "cand_offsets", 8), _host_ptr(E, "E", 2),
                                   _host_ptr(pass_out, "pass", 1), chunk_reads, _stream_ptr(stream)),
           "grim_filter_host")
    return pass_out
