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


def _split_top(s, sep=","):
    out, depth, cur = [], 0, ""
    for ch in s:
        if ch in "[<(":
            depth += 1
        elif ch in "]>)":
            depth -= 1
        if ch == sep and depth == 0:
            out.append(cur)
            cur = ""
        else:
            cur += ch
    out.append(cur)
    return [x.strip() for x in out]


def bind_shared(src):
    """Dynamic shared memory -> the CTA arena; every static __shared__
    declarator -> its own slot of the arena.  Returns (source, slots used)."""
    src = re.sub(r"extern __shared__ (?:__align__\(\d+\) )?([\w ]+?) (\w+)\[\];",
                 r"\1* \2 = reinterpret_cast<\1*>(emu_dyn_smem());", src)
    slot = 0
    out, pos = [], 0
    for m in re.finditer(r"__shared__ ([^;]+);", src):
        out.append(src[pos:m.start()])
        parts = _split_top(m.group(1))
        first = re.match(r"^(.*?)\s*\b(\w+)\s*((?:\[[^\]]*\])*)$", parts[0])
        ctype = first.group(1).strip()
        decls = [(first.group(2), first.group(3))]
        for p in parts[1:]:
            d = re.match(r"^(\w+)\s*((?:\[[^\]]*\])*)$", p)
            decls.append((d.group(1), d.group(2)))
        stmts = []
        for name, dims in decls:
            t = f"{ctype}{dims}"
            stmts.append(f"static_assert(sizeof({t}) <= EMU_SLOT_BYTES, \"static shared variable too large\"); "
                         f"auto& {name} = *reinterpret_cast<{ctype}(*){dims}>(emu_static_smem_slot({slot}));"
                         if dims else
                         f"auto& {name} = *reinterpret_cast<{ctype}*>(emu_static_smem_slot({slot}));")
            slot += 1
        out.append(" ".join(stmts))
        pos = m.end()
    out.append(src[pos:])
    return "".join(out), slot


def _plain_cp_async(src):
    """The sweep's asynchronous 16-byte copies as plain copies (they complete
    at once on the emulator, so committing and waiting do nothing), and the
    two halves of its cluster barrier on the emulated cluster barrier."""
    src = replace_body(src, "__device__ __forceinline__ void cp_async_16(float4* dst, const float4* src)",
                       "{ *dst = *src; }")
    src = replace_body(src, "__device__ __forceinline__ void cp_async_commit()", "{}")
    src = replace_body(src, "__device__ __forceinline__ void cluster_arrive()", "{ emu_cluster_arrive(); }")
    src = replace_body(src, "__device__ __forceinline__ void cluster_wait()", "{ emu_cluster_wait(); }")
    return replace_body(src, "__device__ __forceinline__ void cp_async_wait_all()", "{}")


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
    ds = _plain_cp_async(ds)
    ds, slots = bind_shared(ds)
    return "\n".join([f"#define EMU_STATIC_SLOTS {max(slots, 1)}", '#include "shim_threads.h"', common,
                      "namespace mbicg {", "namespace emu_dslash {", ds, "}", "}"])


MBAR_BODIES = {
    "__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)":
        "{ emu_mbar_init(bar, (int)count); }",
    "__device__ __forceinline__ void mbar_fence_init()": "{}",
    "__device__ __forceinline__ void mbar_arrive(uint64_t* bar)": "{ emu_mbar_update(bar, 1, 0, 0); }",
    "__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)":
        "{ emu_mbar_update(bar, 1, bytes, 0); }",
    "__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase)":
        "{ return emu_mbar_try(bar, phase); }",
    "__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, int limit = MBAR_SPIN_LIMIT)":
        "{ (void)limit; return emu_mbar_wait(bar, phase); }",
    "__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)":
        "{ memcpy(dst, src, bytes); emu_mbar_update(bar, 0, 0, bytes); }",
}


def blas_parts(csrc=CSRC):
    """common.cuh with the mbarrier and bulk-copy helpers emulated, the
    declarations of internal.h, and the device part of blas.cu."""
    common = read("common.cuh", csrc)
    for sig, body in MBAR_BODIES.items():
        common = replace_body(common, sig, body)
    internal = read("internal.h", csrc).replace('#include "common.cuh"', "")
    bl = cut(read("blas.cu", csrc), "namespace {", "}  // namespace\n")
    # the Gram launcher: the same grid, the kernel run by the emulator
    bl = replace_body(bl, "int launch_gram_t(",
                      "{ (void)ex; using SH = GramShape<R, L, HERM>;"
                      " const long long ntiles = (nsite + SH::TS - 1) / SH::TS;"
                      " const int grid = (int)(ntiles < GRAM_CTAS ? ntiles : GRAM_CTAS);"
                      " emu_launch(grid, 1, NT, SH::smem, [&] { k_gram<R, L, HERM>(nsite, A, B1, B2, flags, part, err); });"
                      " return grid; }")
    bl, slots = bind_shared(bl)
    return "\n".join([f"#define EMU_STATIC_SLOTS {max(slots, 1)}", '#include "shim_threads.h"',
                      common, internal, "namespace mbicg {", "namespace emu_blas {", bl, "}", "}"])


def _split_launch_config(cfg):
    parts = _split_top(cfg)
    while len(parts) < 4:
        parts.append("0")
    return parts


def _match_paren(src, i):
    """Index of the parenthesis closing the one at src[i]."""
    depth = 0
    for j in range(i, len(src)):
        if src[j] == "(":
            depth += 1
        elif src[j] == ")":
            depth -= 1
            if depth == 0:
                return j
    raise ValueError("unbalanced parentheses")


def _kernel_name_start(src, i):
    """Start of the (possibly templated) kernel name that ends at src[i - 1]."""
    j = i
    if src[j - 1] == ">":  # template arguments
        depth = 0
        while True:
            j -= 1
            if src[j] == ">":
                depth += 1
            elif src[j] == "<":
                depth -= 1
                if depth == 0:
                    break
    while j > 0 and (src[j - 1].isalnum() or src[j - 1] in "_:"):
        j -= 1
    return j


def rewrite_launches(src):
    """kernel<<<grid, block, smem, stream>>>(args) -> an emulated launch that
    runs the kernel to completion, and cudaLaunchKernelEx(cfg, kernel, args)
    -> emu_launch_ex(cfg, kernel, args)."""
    while True:
        i = src.find("<<<")
        if i < 0:
            break
        start = _kernel_name_start(src, i)
        k = src.index(">>>", i)
        grid, block, smem, stream = _split_launch_config(src[i + 3:k])
        a = src.index("(", k)
        b = _match_paren(src, a)
        call = f"{src[start:i]}{src[a:b + 1]}"
        src = (src[:start] + f"emu_kernel_launch({grid}, {block}, {smem}, {stream}, [&] {{ {call}; }})" +
               src[b + 1:])
    return src.replace("cudaLaunchKernelEx(", "emu_launch_ex(")


def driver_parts(csrc=CSRC):
    """The SAP driver (sap.cu) and everything it launches (dslash.cu), host
    code included (with the autotuner's table, tune.cu), for the threaded emulation: launches rewritten onto the
    emulator, inline PTX helpers replaced, shared memory bound to the arenas."""
    common = read("common.cuh", csrc)
    common = replace_body(common, "__device__ __forceinline__ void load_spinor(const cx<float>* p, Spinor<float>& s)",
                          "{ for (int k = 0; k < 12; ++k) (&s.c[0][0])[k] = p[k]; }")
    common = replace_body(common, "__device__ __forceinline__ void store_spinor(cx<float>* p, const Spinor<float>& s)",
                          "{ for (int k = 0; k < 12; ++k) p[k] = (&s.c[0][0])[k]; }")
    internal = read("internal.h", csrc).replace('#include "common.cuh"', "")
    # the operator's launch configurations come from the autotuner's table (host code)
    tune = read("tune.h", csrc) + "\n" + read("tune.cu", csrc).replace('#include "tune.h"', "")
    ds = read("dslash.cu", csrc)
    ds = ds[ds.index("namespace mbicg {"):]
    ds = replace_body(ds, "__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank)",
                      "{ return emu_mapa(local, rank); }")
    ds = replace_body(ds, "__device__ __forceinline__ float4 ld_cluster_f4(uint32_t addr)",
                      "{ return emu_ld_cluster_f4(addr); }")
    ds = _plain_cp_async(ds)
    sp = read("sap.cu", csrc)
    sp = sp[sp.index("namespace mbicg {"):]
    body = rewrite_launches(ds + "\n" + sp)
    body, slots = bind_shared(body)
    return "\n".join([f"#define EMU_STATIC_SLOTS {max(slots, 1)}", '#include "shim_threads.h"',
                      "#include <algorithm>", "#include <cstdlib>", "#include <type_traits>",
                      '#include "emu_runtime.h"', common, internal, tune, body])


INCLUDE = os.path.join(ROOT, "include")


def _patched_common(csrc):
    common = read("common.cuh", csrc)
    common = replace_body(common, "__device__ __forceinline__ void load_spinor(const cx<float>* p, Spinor<float>& s)",
                          "{ for (int k = 0; k < 12; ++k) (&s.c[0][0])[k] = p[k]; }")
    common = replace_body(common, "__device__ __forceinline__ void store_spinor(cx<float>* p, const Spinor<float>& s)",
                          "{ for (int k = 0; k < 12; ++k) p[k] = (&s.c[0][0])[k]; }")
    for sig, body in MBAR_BODIES.items():
        common = replace_body(common, sig, body)
    return common


LIBRARY_SOURCES = ["api.cu", "dslash.cu", "sap.cu", "blas.cu", "half.cu", "serve.cu", "noalloc.cu", "selftest.cu", "tune.cu",
                   "clover.cu"]


def library_unit(name, csrc=CSRC):
    """One translation unit of the library for the emulated build: the file
    itself with common.cuh (inline PTX replaced) and internal.h inlined, the
    launches rewritten onto the emulator and shared memory bound to the
    arenas."""
    src = read(name, csrc)
    head = _patched_common(csrc) + "\n" + read("internal.h", csrc).replace('#include "common.cuh"', "")
    src = src.replace('#include "internal.h"', head.replace("#pragma once", ""))
    src = src.replace('#include "../../include/mbicg.h"', f'#include "{os.path.join(INCLUDE, "mbicg.h")}"')
    src = src.replace("#include <cooperative_groups.h>", "")
    if name == "dslash.cu":
        src = replace_body(src, "__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank)",
                           "{ return emu_mapa(local, rank); }")
        src = replace_body(src, "__device__ __forceinline__ float4 ld_cluster_f4(uint32_t addr)",
                           "{ return emu_ld_cluster_f4(addr); }")
        src = _plain_cp_async(src)
    src = rewrite_launches(src)
    src, slots = bind_shared(src)
    return "\n".join([f"#define EMU_STATIC_SLOTS {max(slots, 1)}", '#include "shim_threads.h"',
                      '#include "emu_runtime.h"', src])
