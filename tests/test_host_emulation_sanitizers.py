"""Memory safety, undefined behaviour and data races of the library's kernels
and host code on the CPU: the emulated library (tests/emulated_library.py)
built twice, with AddressSanitizer plus UndefinedBehaviorSanitizer and with
ThreadSanitizer, each driven through its C ABI by
tests/host_emulation/sanitizer_exercise.py in a child process with the
sanitizer's runtime preloaded.

AddressSanitizer: emulated device buffers are allocated at their exact size
and each CTA's dynamic shared memory is followed by a poisoned gap, so that
an access past either is reported; UndefinedBehaviorSanitizer stops the run
at a misaligned vector access (a fault on the GPU), an out-of-range index
into a fixed-size array or a signed overflow.  ThreadSanitizer: every CUDA
thread is a host thread and the emulated barriers, shuffles, mbarriers and
atomics order their accesses, so a shared- or global-memory access that no
barrier orders against another thread's (a missing __syncthreads or cluster
barrier) is reported as a data race, whatever the schedule of the run.

The exercise runs the operator in FP64, FP32 and FP16 (and the
allocation-free one on emulated device buffers), SAP with the fused
cluster sweep and the multi-kernel path (per-column and block MR, FP64 and
FP32), block solves with dummy columns and an initial guess, every launch
configuration of the operator that the autotuner times, SSOR domain solves,
the clover term and its Jacobi preconditioning (operators, SAP with MR and
SSOR, block solves of D_c X = B), the request server (two solver slots on
host threads, four clients submitting and waiting from host threads at
once), and the 8-CTA cluster sweep alone and (AddressSanitizer) in a block
solve on an 8^4 lattice.  Mistakes
planted in a copy of the sources were each reported: an off-by-one write and
a misaligned float4 load in a layout kernel, and a removed barrier before a
block reduction (a data race)."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import emulated_library

EXERCISE = os.path.join(emulated_library.HERE, "sanitizer_exercise.py")
BUILDS = {"address": ("asan", emulated_library.SANITIZE_FLAGS), "thread": ("tsan", emulated_library.TSAN_FLAGS)}


@pytest.fixture(scope="module")
def sanitized(tmp_path_factory):
    """Both sanitized builds, compiled at once: {sanitizer: (library, runtime)}."""
    if not emulated_library.available():
        pytest.skip("g++ or the CUDA headers are missing")
    runtimes = {k: emulated_library.sanitizer_runtime(rt) for k, (rt, _) in BUILDS.items()}

    def build(k):
        d = tmp_path_factory.mktemp(f"{k}_sanitized_library")
        return emulated_library.compile_library(str(d), BUILDS[k][1])

    todo = [k for k in BUILDS if runtimes[k]]
    with ThreadPoolExecutor(len(todo) or 1) as ex:
        libs = dict(zip(todo, ex.map(build, todo)))
    return {k: (libs[k], runtimes[k]) for k in todo}


def _run(sanitized, which):
    if which not in sanitized:
        pytest.skip(f"gcc's {BUILDS[which][0]} runtime is missing")
    so, runtime = sanitized[which]
    env = dict(os.environ, LD_PRELOAD=runtime, ASAN_OPTIONS="detect_leaks=0:halt_on_error=1:exitcode=23",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1", TSAN_OPTIONS="halt_on_error=1:exitcode=66")
    for k in ("MBICG_SAP_FUSED", "MBICG_AUTOTUNE", "MBICG_TUNE_FILE"):
        env.pop(k, None)
    cmd = [sys.executable, EXERCISE, so, which]
    if which == "thread" and shutil.which("setarch"):
        cmd = ["setarch", "-R"] + cmd  # ThreadSanitizer's fixed shadow layout wants the address space unrandomised
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
    report = r.stdout[-3000:] + r.stderr[-6000:]
    assert "Sanitizer" not in r.stderr and "runtime error" not in r.stderr, report
    assert r.returncode == 0, report
    assert "ok sanitizer" in r.stdout and r.stdout.rstrip().endswith("done"), report


@pytest.mark.slow
def test_address_and_undefined_behaviour(sanitized):
    _run(sanitized, "address")


@pytest.mark.slow
def test_no_data_races(sanitized):
    _run(sanitized, "thread")
