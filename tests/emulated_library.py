"""Builds the test-only emulated library (tests/test_host_emulation_library.py
describes it): every CUDA source of the package as a g++ translation unit on
the threaded emulator, linked with the emulated CUDA runtime.  The package
never builds or loads it."""
import ctypes
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import emulation_sources
import paper_1104_0737_gb300 as mb  # the ctypes structures only; no library is loaded

HERE = os.path.join(emulation_sources.ROOT, "tests", "host_emulation")
CUDA_INCLUDE = "/usr/local/cuda/include"


def available():
    return shutil.which("g++") is not None and os.path.exists(os.path.join(CUDA_INCLUDE, "cuda_runtime.h"))


# AddressSanitizer, and UndefinedBehaviorSanitizer (misaligned vector accesses,
# fixed-size array bounds, signed overflow, shifts) stopping at its first
# report; ThreadSanitizer.  -O0: these builds compile in a fraction of the time
SANITIZE_FLAGS = ["-O0", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer"]
TSAN_FLAGS = ["-O0", "-fsanitize=thread"]


def compile_library(d, extra_flags=()):
    """Compile and link into directory d; returns the path of the library."""
    for f in ("shim_threads.h", "emu_runtime.h"):
        shutil.copy(os.path.join(HERE, f), os.path.join(d, f))
    units = []
    for name in emulation_sources.LIBRARY_SOURCES:
        src = os.path.join(d, name.replace(".cu", ".cpp"))
        with open(src, "w") as f:
            f.write(emulation_sources.library_unit(name))
        units.append(src)
    units.append(os.path.join(HERE, "emu_cudart.cpp"))
    flags = ["g++", "-std=c++20", "-O1", "-fPIC", "-pthread", *extra_flags, "-I", str(d), "-I",
             emulation_sources.CSRC, "-I", CUDA_INCLUDE]

    def compile_one(src):
        obj = os.path.join(d, os.path.basename(src) + ".o")
        subprocess.run(flags + ["-c", src, "-o", obj], check=True)
        return obj

    with ThreadPoolExecutor(len(units)) as ex:
        objs = list(ex.map(compile_one, units))
    so = os.path.join(d, "libmbicg_emu.so")
    # -Bsymbolic: calls bind to the emulated runtime even when the real CUDA
    # runtime (linked into the real library) is loaded in the same process
    subprocess.run(["g++", "-shared", "-pthread", *extra_flags, "-Wl,-Bsymbolic", *objs, "-o", so], check=True)
    return so


def load(so):
    """The library at so, with the argument types of the ABI calls the tests use."""
    lb = ctypes.CDLL(so)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    lb.mbicg_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.c_int, vp]
    lb.mbicg_destroy.argtypes = [vp]
    lb.mbicg_load_gauge.argtypes = [vp, vp]
    lb.mbicg_apply_D.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_int]
    lb.mbicg_sap_precond.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(mb.mbicg_params)]
    lb.mbicg_block_solve.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.POINTER(mb.mbicg_params), ip, dp]
    lb.mbicg_default_params.argtypes = [ctypes.POINTER(mb.mbicg_params)]
    lb.mbicg_get_stats.argtypes = [vp, ctypes.POINTER(mb.mbicg_stats)]
    lb.mbicg_last_error.restype = ctypes.c_char_p
    lb.mbicg_last_error.argtypes = [vp]
    llp = ctypes.POINTER(ctypes.c_longlong)
    lb.mbicg_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double]
    lb.mbicg_server_add_field.argtypes = [vp, ip, vp, ctypes.POINTER(mb.mbicg_params), ctypes.c_int, ip]
    lb.mbicg_server_submit.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, llp]
    lb.mbicg_server_wait.argtypes = [vp, ctypes.c_longlong, vp, ip, dp, ctypes.POINTER(mb.mbicg_request_info)]
    lb.mbicg_server_hold.argtypes = [vp, ctypes.c_int]
    lb.mbicg_server_memory.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), llp]
    lb.mbicg_server_stats.argtypes = [vp, llp, llp, llp, ip]
    lb.mbicg_server_destroy.argtypes = [vp]
    lb.mbicg_apply_D_noalloc.argtypes = [ip, vp, vp, vp, ctypes.c_int, ctypes.c_double, vp]
    lb.mbicg_selftest_bounded_wait.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ip]
    lb.cudaMalloc.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t]
    lb.cudaFree.argtypes = [vp]
    lb.emu_set_owner.argtypes = [vp, ctypes.c_int]
    return lb


def build(d):
    """compile_library then load."""
    return load(compile_library(d))


def sanitizer_runtime(name):
    """Path of gcc's runtime of a sanitizer ("asan", "tsan"), or None."""
    try:
        r = subprocess.run(["gcc", f"-print-file-name=lib{name}.so"], capture_output=True, text=True, check=True)
    except (OSError, subprocess.CalledProcessError):
        return None
    path = r.stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None
