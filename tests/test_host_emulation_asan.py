"""Memory safety and undefined behaviour of the library's kernels and host
code on the CPU: the emulated library (tests/emulated_library.py) built with
AddressSanitizer and UndefinedBehaviorSanitizer and driven through its C ABI
by tests/host_emulation/asan_exercise.py in a child process with the
sanitizer's runtime preloaded.  Emulated device buffers are allocated at
their exact size and each CTA's dynamic shared memory is followed by a
poisoned gap, so that an access past either is reported; a misaligned vector
access (a fault on the GPU), an out-of-range index into a fixed-size array
and a signed overflow stop the run.  Runs the operator in FP64, FP32 and
FP16, SAP with the fused cluster sweep and the multi-kernel path (per-column
and block MR, FP64 and FP32), block solves with dummy columns and an initial
guess, SSOR domain solves, the clover term and its Jacobi preconditioning
(operators, SAP with MR and SSOR, block solves of D_c X = B), and the 8-CTA
cluster sweep in a block solve on an 8^4 lattice.  An
off-by-one write and a misaligned float4 load planted in a layout kernel are
each reported by this run."""

import os
import subprocess
import sys

import pytest

import emulated_library

EXERCISE = os.path.join(emulated_library.HERE, "asan_exercise.py")


@pytest.fixture(scope="module")
def asan_lib(tmp_path_factory):
    runtime = emulated_library.asan_runtime()
    if not emulated_library.available() or runtime is None:
        pytest.skip("g++, the CUDA headers or the sanitizer runtimes are missing")
    d = tmp_path_factory.mktemp("asan_library")
    return emulated_library.compile_library(str(d), emulated_library.SANITIZE_FLAGS), runtime


@pytest.mark.slow
def test_library_under_sanitizers(asan_lib):
    so, runtime = asan_lib
    env = dict(os.environ, LD_PRELOAD=runtime, ASAN_OPTIONS="detect_leaks=0:halt_on_error=1:exitcode=23",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    env.pop("MBICG_SAP_FUSED", None)
    r = subprocess.run([sys.executable, EXERCISE, so], env=env, capture_output=True, text=True, timeout=900)
    report = r.stdout[-3000:] + r.stderr[-6000:]
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, report
    assert r.returncode == 0, report
    assert "ok sanitizer" in r.stdout and r.stdout.rstrip().endswith("done"), report
