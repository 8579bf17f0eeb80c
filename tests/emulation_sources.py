"""Cuts the kernels and their device helpers out of the CUDA sources for the
host emulation tests (tests/host_emulation/): no launches, and for the
threaded emulation the inline PTX helpers replaced by plain C++ and the
shared-memory declarations bound to the emulated CTA arenas.  Every cut and
replacement is located by a fixed marker or signature and fails loudly when
the source no longer has it."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1104_0737_gb300", "csrc")


def read(name, csrc=CSRC):
    with open(os.path.join(csrc, name)) as f:
        return f.read()


def cut(src, start, end):
    a = src.index(start)
    return src[a + len(start):src.index(end, a)]


def replace_body(src, signature, body):
    """Replace the body of the function whose definition starts with
    `signature` by `body` (braces included)."""
    a = src.index(signature)
    b = src.index("{", a + len(signature) - 1)
    depth, i = 0, b
    while True:
        if src[i] == "{":
            depth += 1
        elif src[i] == "}":
            depth -= 1
            if depth == 0:
                break
        i += 1
    return src[:b] + body + src[i + 1:]


SWEEP_END = "// sets the sweep kernel's shared-memory and cluster attributes"
DSLASH_SEQ_END = "// ---------------------------------------------------------------------------\n// Fused SAP colour sweep"


def _bind_shared(src):
    src = re.sub(r"extern __shared__ ([\w ]+?) (\w+)\[\];",
                 r"\1* \2 = reinterpret_cast<\1*>(emu_dyn_smem());", src)
    return re.sub(r"__shared__ (\w+) (\w+)((?:\[[^\]]+\])+);",
                  r"auto& \2 = *reinterpret_cast<\1(*)\3>(emu_static_smem());", src)


def sweep_parts(csrc=CSRC):
    """common.cuh and the device part of dslash.cu (through the fused sweep
    kernel) for the threaded emulation."""
    common = read("common.cuh", csrc)
    common = replace_body(common, "__device__ __forceinline__ void load_spinor(const cx<float>* p, Spinor<float>& s)",
                          "{ for (int k = 0; k < 12; ++k) (&s.c[0][0])[k] = p[k]; }")
    common = replace_body(common, "__device__ __forceinline__ void store_spinor(cx<float>* p, const Spinor<float>& s)",
                          "{ for (int k = 0; k < 12; ++k) p[k] = (&s.c[0][0])[k]; }")
    ds = cut(read("dslash.cu", csrc), "namespace {", SWEEP_END)
    ds = replace_body(ds, "__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank)",
                      "{ return emu_mapa(local, rank); }")
    ds = replace_body(ds, "__device__ __forceinline__ float4 ld_cluster_f4(uint32_t addr)",
                      "{ return emu_ld_cluster_f4(addr); }")
    ds = _bind_shared(ds)
    return "\n".join(['#include "shim_threads.h"', common, "namespace mbicg {", "namespace emu_dslash {", ds,
                      "}", "}"])
