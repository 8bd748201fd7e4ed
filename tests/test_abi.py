"""The C-ABI library builds for sm_103a, loads on a CPU-only host, and
exports every entry point declared in include/grim.h (no compute calls)."""
import os
import re
import subprocess

import pytest

import paper_1711_01177_gb300 as grim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(grim_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    grim.build()
    return grim.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("grim_build_bank", "grim_filter", "grim_bank_free", "grim_bank_status"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", grim._LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = names - exported
    assert not missing, f"declared but not exported: {missing}"
    # and the Python binding knows every one of them, with the same names
    assert names == set(grim.SIGNATURES), names ^ set(grim.SIGNATURES)
    for n in names:
        assert getattr(lib, n) is not None


def test_strerror_without_gpu(lib):
    assert lib.grim_strerror(grim.GRIM_OK) == b"ok"
    assert b"invalid" in lib.grim_strerror(grim.GRIM_EINVAL)
    assert lib.grim_strerror(12345) == b"unknown status"


def test_host_side_argument_checks_need_no_gpu(lib):
    import ctypes
    h = ctypes.c_void_p()
    # rejected before any CUDA call is made
    assert lib.grim_build_bank(None, 100, 5, 256, 100, None, ctypes.byref(h)) == grim.GRIM_EINVAL
    assert lib.grim_build_bank(ctypes.c_void_p(16), 100, 7, 256, 100, None, ctypes.byref(h)) == grim.GRIM_ENOTSUP
    assert lib.grim_build_bank(ctypes.c_void_p(16), 100, 5, 0, 100, None, ctypes.byref(h)) == grim.GRIM_EINVAL
    assert lib.grim_filter(None, None, None, 0, None, None, None, None, None, None) == grim.GRIM_EINVAL
    assert lib.grim_bank_free(None) == grim.GRIM_OK
    # the entry points around the filter check their arguments first too
    n = ctypes.c_int64()
    fake = ctypes.c_void_p(16)
    assert lib.grim_seed_index_build(None, 100, 12, None, ctypes.byref(h)) == grim.GRIM_EINVAL
    assert lib.grim_seed_index_build(fake, 100, 16, None, ctypes.byref(h)) == grim.GRIM_EINVAL  # k <= 15
    assert lib.grim_seed_index_build(fake, 10, 12, None, ctypes.byref(h)) == grim.GRIM_EINVAL  # len < k
    assert lib.grim_seed_index_free(None) == grim.GRIM_OK
    assert lib.grim_seed_candidates(None, fake, fake, 1, 256, 10, 100, fake, 10, fake, ctypes.byref(n),
                                    None) == grim.GRIM_EINVAL
    assert lib.grim_locate(None, None, fake, fake, 1, 1, fake, fake, fake, None, None, None, 0, 1, fake,
                           None) == grim.GRIM_EINVAL
    assert lib.grim_verify(None, fake, fake, fake, 1, fake, fake, 1, fake, None) == grim.GRIM_EINVAL
    assert lib.grim_verify_stats(None, fake, fake, fake, 1, -1, fake, None) == grim.GRIM_EINVAL
    assert lib.grim_verify_stats(None, fake, fake, fake, 1, 1, None, None) == grim.GRIM_EINVAL
    assert lib.grim_pack_mask(fake, -1, fake, None) == grim.GRIM_EINVAL
    assert lib.grim_pack_mask(None, 5, fake, None) == grim.GRIM_EINVAL
    assert lib.grim_map(None, fake, fake, fake, fake, 1, fake, 100, 0, fake, fake, fake, 1, ctypes.byref(n), None,
                        None) == grim.GRIM_EINVAL
    assert lib.grim_filter_host(None, fake, fake, 1, fake, fake, fake, fake, 0, None) == grim.GRIM_EINVAL
    assert lib.grim_bank_save(None, b"/nonexistent", None) == grim.GRIM_EINVAL
    assert lib.grim_bank_load(None, None, ctypes.byref(h)) == grim.GRIM_EINVAL
    assert lib.grim_strerror(grim.GRIM_EIO) != lib.grim_strerror(12345)
    assert lib.grim_fill_E_rate(fake, 5, 5, 0, 0, fake, None) == grim.GRIM_EINVAL  # den >= 1
    assert lib.grim_fill_E_rate(fake, 5, -1, 100, 0, fake, None) == grim.GRIM_EINVAL  # num >= 0
    assert lib.grim_fill_E_rate(None, 5, 5, 100, 0, fake, None) == grim.GRIM_EINVAL
    assert lib.grim_fill_E_rate(None, 0, 5, 100, 0, None, None) == grim.GRIM_OK  # nothing to do
    # the bounded-wait diagnostic takes a limit of 1 ms .. 2 s
    assert lib.grim_wait_selfcheck(999_999, None) == grim.GRIM_EINVAL
    assert lib.grim_wait_selfcheck(2_000_000_001, None) == grim.GRIM_EINVAL


def test_no_oracle_in_product_path():
    # the package must not import, load or run anything under oracle/
    pkg = os.path.join(ROOT, "paper_1711_01177_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"(import\s+oracle|from\s+oracle|liboracle|grim_oracle|oracle_\w+\()", text), f
