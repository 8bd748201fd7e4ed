"""Host-side fault injection (grim_fault_inject / GRIM_FAULT): arming,
countdown and the environment variable, checked without a GPU.  The error
paths it drives are walked on the GPU in test_gpu_faults.py."""
import os
import subprocess
import sys

import pytest

import paper_1711_01177_gb300 as grim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    grim.build()
    grim.load()
    yield
    grim.grim_fault_inject(grim.GRIM_FAULT_NONE, 0)


def test_arm_and_disarm():
    grim.grim_fault_inject(grim.GRIM_FAULT_ALLOC, 3)
    assert grim.grim_fault_pending() == (grim.GRIM_FAULT_ALLOC, 3)
    grim.grim_fault_inject(grim.GRIM_FAULT_LAUNCH, 7)  # replaces the armed one
    assert grim.grim_fault_pending() == (grim.GRIM_FAULT_LAUNCH, 7)
    grim.grim_fault_inject(grim.GRIM_FAULT_NONE, 0)
    assert grim.grim_fault_pending() == (grim.GRIM_FAULT_NONE, 0)


@pytest.mark.parametrize("kind,nth", [(3, 1), (-1, 1), (grim.GRIM_FAULT_ALLOC, 0), (grim.GRIM_FAULT_LAUNCH, -5)])
def test_bad_arguments_are_rejected(kind, nth):
    lib = grim.load()
    assert lib.grim_fault_inject(kind, nth) == grim.GRIM_EINVAL
    assert grim.grim_fault_pending()[0] == grim.GRIM_FAULT_NONE


def test_calls_rejected_on_the_host_do_not_count():
    # argument checks come first: a rejected call makes no allocation and
    # launches nothing, so the armed fault keeps its countdown
    lib = grim.load()
    grim.grim_fault_inject(grim.GRIM_FAULT_ALLOC, 1)
    import ctypes
    h = ctypes.c_void_p()
    assert lib.grim_build_bank(None, 100, 5, 256, 100, None, ctypes.byref(h)) == grim.GRIM_EINVAL
    assert lib.grim_pack_mask(None, 5, ctypes.c_void_p(16), None) == grim.GRIM_EINVAL
    assert grim.grim_fault_pending() == (grim.GRIM_FAULT_ALLOC, 1)
    grim.grim_fault_inject(grim.GRIM_FAULT_NONE, 0)


@pytest.mark.parametrize("env,expect", [("alloc:4", (1, 4)), ("launch:2", (2, 2)), ("alloc:0", (0, 0)),
                                        ("launch:x", (0, 0)), ("disk:3", (0, 0)), ("", (0, 0))])
def test_environment_variable(env, expect):
    code = ("import sys; sys.path.insert(0, %r); import paper_1711_01177_gb300 as g; g.load(); "
            "print(*g.grim_fault_pending())" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                         env=dict(os.environ, GRIM_FAULT=env))
    assert out.returncode == 0, out.stderr
    assert tuple(int(x) for x in out.stdout.split()) == expect
