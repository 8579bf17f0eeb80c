#!/usr/bin/env python3
"""Benchmark: RHS solves/s of the mixed-precision modified block BiCGSTAB with
SAP (arXiv:1104.0737, Algorithm 2) to a true relative residual of 1e-10 on
the 32^3 x 64 lattice with L = 12 point sources, on one GB300 per process.

One step = one complete block solve of the 12 right-hand sides (initial
residual, every iteration, the FP64 true residual).  Inputs (B, links) are
resident in HBM before the timed region; each step's blocks are 4.8 GB, far
larger than L2, so no extra flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun as independent replicas (one solve stream per GPU,
no collective on the data path); value is the whole-job RHS solves/s.
--impl reference times the FP64 CPU oracle (the reference arm: the method
written plainly from the paper) on the host cores, on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

# ---------------------------------------------------------------------------
# workloads (synthetic stand-ins for the paper's PACS-CS 32^3 x 64 configurations)
# ---------------------------------------------------------------------------
WORKLOADS = {
    # 32^3 x 64, eps 0.5 links, L = 12 point sources, SAP 8^4, mixed precision.
    # kappa: from a scan of kappa on this field, unpreconditioned BiCGSTAB
    # (L = 1, the first point source) needs 2970 iterations at 0.14774 (1971 at
    # 0.1477, 2947 at 0.14773) and diverges at 0.14775.
    "wilson_32c64_L12": dict(dims=(32, 32, 32, 64), eps=0.5, gauge_seed=1003, L=12, source="point",
                             kappa=0.14774, block=(8, 8, 8, 8), ncycle=4, nmr=4, tol=1e-10),
    # smaller lattices of the same family, for quick runs
    "wilson_16c32_L12": dict(dims=(16, 16, 16, 32), eps=0.5, gauge_seed=1002, L=12, source="point",
                             kappa=0.128, block=(8, 8, 8, 8), ncycle=4, nmr=4, tol=1e-10),
    "wilson_8c16_L12": dict(dims=(8, 8, 8, 16), eps=0.5, gauge_seed=1001, L=12, source="point",
                            kappa=0.125, block=(4, 4, 4, 4), ncycle=4, nmr=4, tol=1e-10),
}
DEFAULT_WORKLOAD = "wilson_32c64_L12"
# Iterations the GPU solver takes on the default workload (measured); the CPU
# baseline extrapolates its per-iteration time with it.
GPU_ITERS = {"wilson_32c64_L12": 50}

METRIC = "RHS solves/s to true rel. residual 1e-10, 32^3x64 L=12; Dslash %HBM; p99 ms"
UNIT = "RHS solves/s"


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# algorithmic bytes and flops per launch (FP32 storage, links counted once)
# ---------------------------------------------------------------------------
# The synthetic fields are SU(3) (exponentials of i times traceless Hermitian
# matrices), so the library's FP32 operator and SAP residual kernel read each
# link as its first two rows (12 reals) and rebuild the third.
FP32_LINK_REALS = 12


def dslash_bytes(V, L, real_bytes=4, link_reals=18):
    # per site: L spinors read + L written (12 complex each), 4 forward links
    # of link_reals reals (18, or 12 when only the first two rows are read)
    return V * (L * 2 * 12 * 2 * real_bytes + 4 * link_reals * real_bytes)


def dslash_flops(V, L):
    return V * L * 1368


def sap_domain_bytes(V, L, real_bytes=4):
    # one MR step on the domains of one colour: half the sites
    return dslash_bytes(V // 2, L, real_bytes)


def sap_sweep_bytes(V, L, real_bytes=4):
    """One colour sweep of the fused SAP kernel: on the sweep's half of the
    sites the colour's residual r and psi read, psi written, and the first two
    rows of the four forward links (staged once per domain)."""
    spinor = 24 * real_bytes
    return (V // 2) * (L * 3 * spinor + 4 * 12 * real_bytes)


def sap_sweep_flops(V, L, nmr, frozen=True):
    """The MR steps of one colour sweep: nmr applications of the Dirichlet
    domain operator (the last one is not needed when the step lengths are
    frozen), x += w r and r -= w q (8 flops per complex multiply-add, 12 per
    spinor: 192 flops, 96 in the last frozen step) and, per column, the two
    dot products (12 flops per complex pair)."""
    if frozen:
        return (V // 2) * L * ((nmr - 1) * 1368 + (nmr - 1) * 192 + 96)
    return (V // 2) * L * (nmr * 1368 + nmr * 192 + nmr * 12 * 12)


def sap_resid_bytes(V, L, block, real_bytes=4, link_reals=18):
    """The residual eta - A psi of one colour, every operand moved once: eta
    and psi of the colour's sites read and r written; psi of the other
    colour's sites next to the colour's domains, which is the whole surface of
    every domain of the other colour (all neighbours of a domain have the
    other colour when the domain counts are even); the four forward links of
    the colour's sites and, for each site on a backward face, the link of its
    neighbour across that face (link_reals reals per link)."""
    spinor = 24 * real_bytes
    link = link_reals * real_bytes
    half = V // 2
    vol = block[0] * block[1] * block[2] * block[3]
    inner = 1
    for b in block:
        inner *= max(b - 2, 0)
    surface = (half // vol) * (vol - inner)  # other-colour sites read for the halo
    back_links = sum(half // b for b in block)
    return half * (3 * L * spinor + 4 * link) + surface * L * spinor + back_links * link


# DRAM bytes per launch of the dominant kernel at the benchmark workload, from one
# ncu capture of dram__bytes_read.sum + dram__bytes_write.sum, valid only for the
# kernel source it was taken on (a hash of csrc/dslash.cu and csrc/common.cuh,
# first 16 hex digits)
NCU_TRAFFIC = {("sap_sweep", "wilson_32c64_L12"): {"bytes": 2743783680 + 1172062720, "source_sha256": "703e40b05b940475"},
               ("sap_resid", "wilson_32c64_L12"): {"bytes": 3848284160 + 1190637312, "source_sha256": "703e40b05b940475"}}


def ncu_traffic(kernel: str, workload: str):
    """The recorded DRAM traffic of the kernel per launch, or None when none was
    recorded or the kernel's source has changed since."""
    import hashlib

    rec = NCU_TRAFFIC.get((kernel, workload))
    if rec is None:
        return None
    h = hashlib.sha256()
    for name in ("dslash.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1104_0737_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return rec["bytes"] if h.hexdigest()[:16] == rec["source_sha256"] else None


def fp32_alu_peak_tflops(sm_mhz, sms=152, lanes=128):
    """FP32 FMA throughput from the unit counts: SMs x FP32 lanes x 2 flops x clock."""
    return sms * lanes * 2 * sm_mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------
# clocks sampler
# ---------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # median under load: samples above half the max clock
        top = max(smax) if smax else max(sm)
        load = [s for s in sm if s > 0.5 * top] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(top), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# serving: a Poisson stream of source blocks on three resident gauge fields
# ---------------------------------------------------------------------------
SERVING = dict(fields=[(8, 8, 8, 16), (16, 16, 16, 32), (24, 24, 24, 48)], eps=0.5, gauge_seed=1004,
               kappas=(0.12, 0.125, 0.128), max_L=12, tol=1e-10, block=(4, 4, 4, 4), ncycle=4, nmr=4,
               requests=64, rates_per_s=(8.0, 128.0), slots=2, seed=2004)


def run_serving(device=0):
    """Requests of 1..12 Gaussian columns arrive as a Poisson stream on three
    resident fields with kappa drawn from `kappas`; the library's server packs
    compatible requests into block solves.  One stream per arrival rate (a
    light load and one that queues); for each: throughput, p50/p99 of
    arrival-to-result latency and the mean width of the block solves."""
    import threading

    import paper_1104_0737_gb300 as mb

    cfg = SERVING
    rng = np.random.default_rng(cfg["seed"])
    srv = mb.mbicg_server_create(device, 120.0)
    phases = []
    try:
        params = mb.mbicg_default_params(block=cfg["block"], ncycle=cfg["ncycle"], nmr=cfg["nmr"],
                                         mr_mode=mb.MBICG_MR_FROZEN, max_iter=5000)
        fids = [mb.mbicg_server_add_field(srv, d, synth.su3_links(d, cfg["eps"], cfg["gauge_seed"] + i), params,
                                          cfg["slots"]) for i, d in enumerate(cfg["fields"])]
        for rate in cfg["rates_per_s"]:
            reqs = []
            for i in range(cfg["requests"]):
                f = int(rng.integers(len(fids)))
                L = int(rng.integers(1, cfg["max_L"] + 1))
                kappa = float(cfg["kappas"][int(rng.integers(len(cfg["kappas"])))])
                reqs.append((f, L, kappa, synth.gaussian_source(cfg["fields"][f], L, seed=int(rng.integers(1 << 30))),
                             float(rng.exponential(1.0 / rate))))
            results = [None] * len(reqs)

            def wait(i, rid, B, L):
                X = np.empty_like(B)
                results[i] = mb.mbicg_server_wait(srv, rid, X, L)

            s0 = mb.mbicg_server_stats(srv)
            threads = []
            t0 = time.perf_counter()
            for i, (f, L, kappa, B, gap) in enumerate(reqs):
                time.sleep(gap)
                rid = mb.mbicg_server_submit(srv, fids[f], B, L, kappa, cfg["tol"])
                th = threading.Thread(target=wait, args=(i, rid, B, L))
                th.start()
                threads.append(th)
            for th in threads:
                th.join()
            wall = time.perf_counter() - t0
            s1 = mb.mbicg_server_stats(srv)
            lat = np.array([r[3]["latency_ms"] for r in results])
            cols = sum(r[1] for r in reqs)
            solves = s1["solves"] - s0["solves"]
            phases.append({
                "rate_per_s": rate, "requests": len(reqs), "rhs": cols,
                "all_converged": all(r[0] == mb.MBICG_OK and max(r[2]) <= cfg["tol"] for r in results),
                "rhs_per_s": cols / wall, "wall_s": wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "block_solves": solves, "mean_block_columns": (s1["columns"] - s0["columns"]) / max(solves, 1)})
        slots = mb.mbicg_server_stats(srv)["slots"]
    finally:
        mb.mbicg_server_destroy(srv)
    return {
        "workload": (f"Poisson streams of {cfg['requests']} requests of 1-{cfg['max_L']} Gaussian columns on fields "
                     + ", ".join('x'.join(map(str, d)) for d in cfg["fields"])
                     + f" (eps {cfg['eps']}), kappa in {list(cfg['kappas'])}, SAP "
                     + 'x'.join(map(str, cfg["block"])) + f", tol {cfg['tol']}, {slots} solver slots"),
        "rates": phases,
    }


# ---------------------------------------------------------------------------
# Table 1 / Fig. 2 of Sec. 3.3: the 12 sources solved as 12/L blocks of L
# ---------------------------------------------------------------------------
def run_table1(ctx, cfg, dB, prec_sap, block_sizes=(1, 2, 3, 4, 6, 12)):
    """Solve the workload's 12 right-hand sides as 12/L block solves of L
    columns each, for every L of Table 1, on the resident gauge field; report
    per L the time for all 12 (CUDA events), the iterations of each block,
    NMVM (operator applications on single vectors in the Krylov loop: 2 L per
    iteration, plus L for the initial residual), RHS solves/s, and the
    recursive residual history of the first block (Fig. 2)."""
    import ctypes

    import torch

    import paper_1104_0737_gb300 as mb

    out = []
    nrhs = dB.shape[-1]
    for L in block_sizes:
        if nrhs % L:
            continue
        hist = (ctypes.c_double * 5000)()
        iters, nmvm, tres = [], 0, 0.0
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record()
        for b in range(nrhs // L):
            p = mb.mbicg_default_params(ncycle=cfg["ncycle"], nmr=cfg["nmr"], block=cfg["block"],
                                        mr_mode=mb.MBICG_MR_FROZEN, prec_D=mb.MBICG_FP32,
                                        prec_sap=prec_sap, max_iter=5000)
            if b == 0:
                p.res_history = hist
                p.res_history_len = 5000
            bb = dB[..., b * L:(b + 1) * L].contiguous()
            xx = torch.empty_like(bb)
            st, it, tr = mb.mbicg_block_solve(ctx, bb, xx, L, cfg["kappa"], cfg["tol"], p)
            if st != mb.MBICG_OK:
                raise RuntimeError(f"table-1 solve failed: L={L} block {b} status {st}")
            iters.append(it)
            nmvm += 2 * L * it + L
            tres = max(tres, max(tr))
        t1.record()
        torch.cuda.synchronize()
        sec = t0.elapsed_time(t1) / 1e3
        k = iters[0]
        out.append({"L": L, "blocks": nrhs // L, "time_s": sec, "rhs_per_s": nrhs / sec, "iters": iters,
                    "nmvm": nmvm, "true_res_max": tres,
                    "history_first_block": [float(hist[i]) for i in range(min(k, 5000))]})
    t_l1 = next((r["time_s"] for r in out if r["L"] == 1), None)
    n_l1 = next((r["nmvm"] for r in out if r["L"] == 1), None)
    for r in out:
        r["time_gain"] = t_l1 / r["time_s"] if t_l1 else None
        r["nmvm_gain"] = n_l1 / r["nmvm"] if n_l1 else None
    return out


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
def oracle_sample(cfg, iters_full, n_iter=2):
    """n_iter iterations of the oracle's Algorithm 1 (FP64, SAP with the same
    domains, cycles, MR steps, kappa and L) on a sub-volume of the lattice with
    two domains in x, y, z and four in t; its time per iteration, scaled by the
    volume ratio and the GPU solver's iteration count, gives RHS solves/s.
    The oracle's work per iteration is proportional to the volume."""
    import oracle

    oracle.build()
    blk = cfg["block"]
    sdims = (2 * blk[0], 2 * blk[1], 2 * blk[2], 4 * blk[3])
    L = cfg["L"]
    U = synth.su3_links(sdims, cfg["eps"], cfg["gauge_seed"] + 7)
    B = synth.point_source(sdims, L)
    t0 = time.perf_counter()
    oracle.block_bicgstab(sdims, U, cfg["kappa"], B, tol=1e-300, max_iter=n_iter, ncycle=cfg["ncycle"],
                          nmr=cfg["nmr"], block=blk, mr_mode=2)
    dt = time.perf_counter() - t0
    scale = np.prod(cfg["dims"]) / np.prod(sdims)
    t_solve = dt / n_iter * scale * iters_full
    return {
        "value": L / t_solve, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
        "sample": (f"{n_iter} iterations of Algorithm 1 (FP64 oracle, SAP {cfg['ncycle']} cycles x "
                   f"{cfg['nmr']} MR on {'x'.join(map(str, blk))} domains, L={L}) on a "
                   f"{'x'.join(map(str, sdims))} sub-volume, {dt:.1f} s, scaled by the volume "
                   f"ratio {scale:.0f} and by the GPU solver's {iters_full} iterations"),
        "sample_seconds": dt,
    }


def run_reference(args, cfg, rank, world):
    """--impl reference: the oracle as it stands, on the host cores."""
    if rank != 0:
        return
    iters = GPU_ITERS.get(args.workload) or 50
    for _ in range(args.warmup):
        oracle_sample(cfg, iters)
    vals, times = [], []
    for _ in range(args.steps):
        s = oracle_sample(cfg, iters)
        vals.append(s["value"])
        times.append(s["sample_seconds"])
    value = float(np.mean(vals))
    cpu = dict(s)
    cpu["value"] = value
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, **_cfg_public(cfg)},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest of `value` over the ranks of the process group (the timed
    region of the slowest replica), or value itself without one."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, L: int, steps: int, seconds: float) -> float:
    """RHS solves per second of the whole job: every replica solved L columns
    per step."""
    return world * L * steps / seconds


def leg_error(name: str, exc: BaseException) -> dict:
    """A side leg of the bench (end to end, CPU baseline, FP64 arm, other
    storage, SSOR, Table 1, serving) that raised: reported on stderr and in
    the line in place of that leg's result, so that the timed solve's line is
    still printed."""
    msg = f"{type(exc).__name__}: {exc}"
    print(f"bench.py: the {name} leg failed: {msg}", file=sys.stderr, flush=True)
    return {"error": msg}


def _cfg_public(cfg):
    return {"lattice": "x".join(map(str, cfg["dims"])), "L": cfg["L"], "source": cfg["source"],
            "kappa": cfg["kappa"], "eps": cfg["eps"], "sap_block": "x".join(map(str, cfg["block"])),
            "ncycle": cfg["ncycle"], "nmr": cfg["nmr"], "tol": cfg["tol"],
            "precision": "FP32 operator/Krylov vectors, SAP FP32 arithmetic with " + cfg.get("sap_storage", "FP32")
                         + " storage, FP64 X, QR, LxL, true residual",
            "l2": "inputs larger than L2 (4.8 GB per block)"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--kappa", type=float, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the Poisson request stream on three resident fields")
    ap.add_argument("--no-fp64-arm", action="store_true",
                    help="skip the plain FP64 one-RHS-at-a-time solve timed on the same GPU")
    ap.add_argument("--prec-sap", default="fp32", choices=["fp32", "fp16"],
                    help="storage of the preconditioner's blocks in the timed solve")
    ap.add_argument("--no-alt-storage", action="store_true",
                    help="skip the line of the other preconditioner storage (FP16 / FP32)")
    ap.add_argument("--kappa-scan", default=None,
                    help="comma-separated kappas: iterations of the unpreconditioned solve (L = 1, the first "
                         "source, FP32 Krylov vectors with reliable updates) on the workload's field, then exit")
    ap.add_argument("--no-ssor-line", action="store_true",
                    help="skip the line with SSOR domain solves (Sec. 2.2) in place of MR")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the library's autotuner (launch shapes of the operator and the SAP sweep)")
    ap.add_argument("--table1", action="store_true",
                    help="also solve the 12 sources as 12/L blocks of L = 1, 2, 3, 4, 6, 12 (Table 1, Fig. 2)")
    args = ap.parse_args()
    cfg = dict(WORKLOADS[args.workload])
    if args.kappa is not None:
        cfg["kappa"] = args.kappa
    cfg["sap_storage"] = args.prec_sap.upper()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, cfg, rank, world)
        return
    import torch

    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    # the library's autotuner: the first (warm-up) solve times the launch
    # shapes that give bit-identical results and keeps the fastest
    tune_file = None
    if not args.no_autotune:
        tune_file = os.path.join(tempfile.mkdtemp(prefix="mbicg_tune_"), "tune.txt")
        os.environ["MBICG_AUTOTUNE"] = "1"
        os.environ["MBICG_TUNE_FILE"] = tune_file
    import paper_1104_0737_gb300 as mb

    dims, L = cfg["dims"], cfg["L"]
    V = int(np.prod(dims))
    U = synth.su3_links(dims, cfg["eps"], cfg["gauge_seed"])
    B = synth.point_source(dims, L) if cfg["source"] == "point" else synth.gaussian_source(dims, L, 2003)
    stream = torch.cuda.Stream()
    ctx = mb.mbicg_create(dims, device=local, stream=stream)
    mb.mbicg_load_gauge(ctx, U)
    del U
    prec_sap = {"fp32": mb.MBICG_FP32, "fp16": mb.MBICG_FP16}[args.prec_sap]
    params = mb.mbicg_default_params(ncycle=cfg["ncycle"], nmr=cfg["nmr"], block=cfg["block"],
                                     mr_mode=mb.MBICG_MR_FROZEN, prec_D=mb.MBICG_FP32,
                                     prec_sap=prec_sap, max_iter=5000)
    dB = torch.from_numpy(B).to(f"cuda:{local}")
    dX = torch.empty_like(dB)
    torch.cuda.synchronize()
    if args.kappa_scan:
        # how hard the workload is without a preconditioner, per kappa
        b1 = dB[..., :1].contiguous()
        x1 = torch.empty_like(b1)
        for kappa in [float(k) for k in args.kappa_scan.split(",")]:
            p0 = mb.mbicg_default_params(ncycle=0, max_iter=12000)
            st, it, tr = mb.mbicg_block_solve(ctx, b1, x1, 1, kappa, cfg["tol"], p0)
            print(json.dumps({"kappa": kappa, "unpreconditioned_iters": it, "status": st, "true_res": tr[0]}),
                  flush=True)
        mb.mbicg_destroy(ctx)
        return

    def solve(b, x):
        st, it, tres = mb.mbicg_block_solve(ctx, b, x, L, cfg["kappa"], cfg["tol"], params)
        if st != mb.MBICG_OK:
            raise RuntimeError(f"solve failed: status {st}, iters {it}, true residual {max(tres)}")
        return it, max(tres)

    for _ in range(args.warmup):
        solve(dB, dX)

    clocks = Clocks(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    iters, tres_max, launches = [], 0.0, 0
    with torch.cuda.stream(stream):
        t_start = torch.cuda.Event(enable_timing=True)
        t_start.record()
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            it, tr = solve(dB, dX)
            e1.record()
            evs.append((e0, e1))
            iters.append(it)
            tres_max = max(tres_max, tr)
            launches += mb.mbicg_get_stats(ctx)["kernel_launches"]
        t_end = torch.cuda.Event(enable_timing=True)
        t_end.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    last_stats = mb.mbicg_get_stats(ctx)
    graph_iters = last_stats["graph_iterations"]
    # per-kernel times from one more solve with CUDA events around every launch
    # group (outside the timed region: profiling runs the loop without its graph)
    mb.mbicg_set_profiling(ctx, True)
    solve(dB, dX)
    prof = mb.mbicg_get_profile(ctx)
    mb.mbicg_set_profiling(ctx, False)
    total_ms = max_over_ranks(total_ms, dist, f"cuda:{local}")
    value = whole_job_rate(world, L, args.steps, total_ms / 1e3)

    # roofline of the dominant kernel class (CUDA events around every launch on
    # the library's stream, over the profiled solve)
    hbm_peak, peak_kind = load_peaks()
    sm_mhz = clk.get("sm_mhz") or 1492.0
    alu_peak = fp32_alu_peak_tflops(sm_mhz)
    models = {
        "sap_sweep": ("alu", sap_sweep_bytes(V, L), sap_sweep_flops(V, L, cfg["nmr"])),
        "sap_resid": ("hbm", sap_resid_bytes(V, L, cfg["block"], link_reals=FP32_LINK_REALS),
                      dslash_flops(V // 2, L)),
        "sap_domain": ("hbm", sap_domain_bytes(V, L), dslash_flops(V // 2, L)),
        "dslash": ("hbm", dslash_bytes(V, L, link_reals=FP32_LINK_REALS), dslash_flops(V, L)),
    }
    dom = max((k for k in models if prof[k][1] > 0), key=lambda k: prof[k][0])
    bound, nbytes, nflops = models[dom]
    avg_ms = prof[dom][0] / prof[dom][1]
    gbs = nbytes / (avg_ms * 1e-3) / 1e9
    tfs = nflops / (avg_ms * 1e-3) / 1e12
    if bound == "alu":
        roofline = {"kernel": dom, "bound": "alu", "achieved": tfs, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": tfs / alu_peak, "traffic": ncu_traffic(dom, args.workload),
                    "peak_kind": f"FP32 FMA units x clock: 152 SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz (sampled)",
                    "algorithmic_flops_per_launch": nflops, "algorithmic_bytes_per_launch": nbytes,
                    "achieved_gbs": gbs, "hbm_frac": gbs / hbm_peak, "avg_launch_ms": avg_ms}
    else:
        roofline = {"kernel": dom, "bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": gbs / hbm_peak, "traffic": ncu_traffic(dom, args.workload), "peak_kind": peak_kind,
                    "algorithmic_bytes_per_launch": nbytes, "avg_launch_ms": avg_ms}
    dsl_ms = prof["dslash"][0] / prof["dslash"][1] if prof["dslash"][1] else None
    dsl_bytes = dslash_bytes(V, L, link_reals=FP32_LINK_REALS)
    dslash_frac = (dsl_bytes / (dsl_ms * 1e-3) / 1e9) / hbm_peak if dsl_ms else None
    res_ms = prof["sap_resid"][0] / prof["sap_resid"][1] if prof["sap_resid"][1] else None
    res_bytes = sap_resid_bytes(V, L, cfg["block"], link_reals=FP32_LINK_REALS)
    resid_frac = (res_bytes / (res_ms * 1e-3) / 1e9) / hbm_peak if res_ms else None

    # end to end through the ABI with pinned host buffers
    e2e = None
    try:
        if not args.no_e2e:
            hB = torch.from_numpy(B).pin_memory()
            hX = torch.empty_like(hB).pin_memory()
            solve(hB, hX)  # untimed: the library's staging buffers for host blocks are allocated here
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                solve(hB, hX)
            t1 = time.perf_counter()
            e2e_s = t1 - t0
            e2e_s = max_over_ranks(e2e_s, dist, f"cuda:{local}")
            nb = B.nbytes
            e2e = {"value": whole_job_rate(world, L, args.steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": nb,
                   "d2h_bytes_per_step": nb}
    except Exception as e:  # a failed side leg ends that leg only
        if dist:
            raise  # the other replicas wait in max_over_ranks: fail the job instead
        e2e = leg_error("e2e", e)

    cpu = None
    try:
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            cpu = oracle_sample(cfg, int(np.median(iters)))
            cpu.pop("sample_seconds", None)
    except Exception as e:  # a failed side leg ends that leg only
        cpu = leg_error("cpu", e)

    # legs without an untimed warm-up solve run untuned (a first solve of a
    # new lattice, L or precision would otherwise time the candidates inside
    # the timed region)
    if tune_file:
        os.environ["MBICG_AUTOTUNE"] = "0"
    fp64_arm = None
    try:
        if not args.no_fp64_arm and rank == 0:
            p64 = mb.mbicg_default_params(ncycle=cfg["ncycle"], nmr=cfg["nmr"], block=cfg["block"],
                                          mr_mode=mb.MBICG_MR_FROZEN, prec_D=mb.MBICG_FP64,
                                          prec_sap=mb.MBICG_FP64, max_iter=5000)
            b1 = dB[..., :1].contiguous()
            x1 = torch.empty_like(b1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, it1, tr1 = mb.mbicg_block_solve(ctx, b1, x1, 1, cfg["kappa"], cfg["tol"], p64)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            fp64_arm = {"value": 1.0 / dt, "unit": UNIT, "iters": it1, "status": st,
                        "sample": "one FP64 L=1 solve (column 0), FP64 operator and SAP"}
    except Exception as e:  # a failed side leg ends that leg only
        fp64_arm = leg_error("fp64_arm", e)

    # the same workload with the preconditioner's blocks in the other storage
    # (FP16 with per-(site, column) scales, or FP32): one warm-up solve and one
    # timed solve, stopped at twice the iterations of the main line (FP16
    # storage does not converge on this workload)
    alt = None
    try:
        if not args.no_alt_storage and rank == 0:
            other = "fp16" if args.prec_sap == "fp32" else "fp32"
            pa = mb.mbicg_default_params(ncycle=cfg["ncycle"], nmr=cfg["nmr"], block=cfg["block"],
                                         mr_mode=mb.MBICG_MR_FROZEN, prec_D=mb.MBICG_FP32,
                                         prec_sap={"fp32": mb.MBICG_FP32, "fp16": mb.MBICG_FP16}[other],
                                         max_iter=2 * max(iters) + 20)
            if tune_file:
                os.environ["MBICG_AUTOTUNE"] = "1"
            st, it_a, tr_a = mb.mbicg_block_solve(ctx, dB, dX, L, cfg["kappa"], cfg["tol"], pa)  # warm-up
            if tune_file:
                os.environ["MBICG_AUTOTUNE"] = "0"
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record()
                st, it_a, tr_a = mb.mbicg_block_solve(ctx, dB, dX, L, cfg["kappa"], cfg["tol"], pa)
                its, trs = [it_a], [max(tr_a)]
                a1.record()
            torch.cuda.synchronize()
            ms = a0.elapsed_time(a1) / len(its)
            alt = {"prec_sap": other, "value": L * 1e3 / ms, "unit": UNIT, "ms_per_step": ms, "iters": its,
                   "true_res_max": max(trs), "status": st}
    except Exception as e:  # a failed side leg ends that leg only
        if tune_file:
            os.environ["MBICG_AUTOTUNE"] = "0"
        alt = leg_error("alt", e)

    # the same workload with the paper's SSOR domain solves (Sec. 2.2: omega 1.26,
    # N_SSOR = 1) in place of the MR steps: one warm-up solve, one timed
    ssor = None
    try:
        if not args.no_ssor_line and rank == 0:
            ps = mb.mbicg_default_params(ncycle=cfg["ncycle"], block=cfg["block"], domain_solver=mb.MBICG_DOMAIN_SSOR,
                                         nssor=1, ssor_omega=1.26, prec_D=mb.MBICG_FP32, prec_sap=mb.MBICG_FP32,
                                         max_iter=2 * max(iters) + 20)
            mb.mbicg_block_solve(ctx, dB, dX, L, cfg["kappa"], cfg["tol"], ps)
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                s0 = torch.cuda.Event(enable_timing=True)
                s1 = torch.cuda.Event(enable_timing=True)
                s0.record()
                st, it_s, tr_s = mb.mbicg_block_solve(ctx, dB, dX, L, cfg["kappa"], cfg["tol"], ps)
                s1.record()
            torch.cuda.synchronize()
            ms = s0.elapsed_time(s1)
            ssor = {"domain_solver": "SSOR omega 1.26, N_SSOR 1", "value": L * 1e3 / ms, "unit": UNIT,
                    "ms_per_step": ms, "iters": it_s, "true_res_max": max(tr_s), "status": st}
    except Exception as e:  # a failed side leg ends that leg only
        ssor = leg_error("ssor", e)

    table1 = None
    try:
        if args.table1 and rank == 0:
            table1 = run_table1(ctx, cfg, dB, prec_sap)
    except Exception as e:  # a failed side leg ends that leg only
        table1 = leg_error("table1", e)

    mb.mbicg_destroy(ctx)
    del dB, dX
    serving = None
    try:
        if rank == 0 and world == 1 and not args.no_serving:
            torch.cuda.empty_cache()
            serving = run_serving(local)
    except Exception as e:  # a failed side leg ends that leg only
        serving = leg_error("serving", e)
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, **_cfg_public(cfg),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "iters": iters, "true_res_max": tres_max, "graph_iterations_last_step": graph_iters,
            "host_syncs_last_step": last_stats["host_syncs"],
            "reliable_updates_last_step": last_stats["reliable_updates"],
            "dslash_hbm_frac": dslash_frac, "sap_resid_hbm_frac": resid_frac,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "kernel_ms": {k: v[0] for k, v in prof.items()},
            "kernel_launch_groups": {k: v[1] for k, v in prof.items()},
        }
        if tune_file and os.path.exists(tune_file):
            # key -> index of the chosen candidate (tune.h: the operator's
            # sites per CTA and CTA order; the sweep's shape 0/1/2 = 8-CTA
            # clusters, 16-CTA clusters with two columns per thread, 16-CTA
            # clusters with one)
            with open(tune_file) as f:
                out["autotuned"] = {k: int(v) for k, v in (line.split() for line in f if line.strip())}
        if fp64_arm:
            out["fp64_one_rhs_arm"] = fp64_arm
        if serving:
            out["serving"] = serving
        if table1:
            out["table1"] = table1
        if alt:
            out["alt_storage_line"] = alt
        if ssor:
            out["ssor_line"] = ssor
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
