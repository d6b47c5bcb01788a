"""Benchmark of the GLS hot path on GB300 (one JSON line on rank 0).

Workload (default): n = 10,000 individuals, p = 4 (intercept + 2 covariates + SNP),
t = 1 phenotype, FP64, SNPs streamed in blocks of 16,384 -- the block stream of a
1,000,000-SNP job. One step = one block through the whole per-block path (H2D of the
dosages for e2e, L^{-1} X_blk fused with the per-SNP reductions, p x p solves).
The per-cohort setup (M, Cholesky, L^{-1}, Xbar_L, ybar, S_TL, bbar_T) runs once
before the timed region and is reported as ``setup_ms``.

``value``: SNPs/s with the dosage blocks already resident in HBM (device entry point).
``e2e``: SNPs/s through ``gwas_solve_block`` from pinned host memory, copies timed.
``--impl reference``: the CPU oracle on the host cores, same metric and config.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLS SNP solves/sec at n=10k-30k, p=4: plain FP64 vs mixed precision (<=1e-6 rel)"
UNIT = "SNP/s"


def parse():
    return _parser().parse_args()


def parse_args_for_test(argv):
    return _parser().parse_args(argv)


def _parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--n", type=int, default=10000)
    ap.add_argument("--m-blk", type=int, default=16384)
    ap.add_argument("--t", type=int, default=1)
    ap.add_argument("--limbs", type=int, default=3)
    ap.add_argument("--pool", type=int, default=4, help="distinct dosage blocks cycled")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision legs (n and n=30000) of an FP64 run")
    ap.add_argument("--mixed-steps", type=int, default=240)
    ap.add_argument("--mixed-n30k-snps", type=int, default=5000000,
                    help="SNPs of the n=30000 mixed leg (default: the whole 5e6-SNP job)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (mixed legs)")
    ap.add_argument("--tile-cfg", type=int, default=None,
                    help="fixed tile configuration for the mixed legs (skips the autotuner)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-cohorts legs (48 cohorts, 16 phenotypes)")
    ap.add_argument("--batch-cohorts", type=int, default=48)
    ap.add_argument("--batch-snps", type=int, default=50000,
                    help="SNPs per cohort in the mixed batched leg")
    ap.add_argument("--batch-tile-cfg", type=int, default=None,
                    help="tile configuration of the batched legs (gwas_opts.tile_cfg)")
    ap.add_argument("--batch-snps-fp64", type=int, default=2048,
                    help="SNPs per cohort per step in the FP64 batched leg")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the REML-fit and db/dh leg (n=10000, FP64)")
    ap.add_argument("--adjoint-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--no-fp64-n30k", action="store_true",
                    help="skip the FP64 leg at n=30000 (blocks of 2048 SNPs)")
    ap.add_argument("--fp64-n30k-steps", type=int, default=3)
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the oracle check of the sampled outputs of every leg")
    ap.add_argument("--cpu-worker", default=None, help=argparse.SUPPRESS)
    return ap


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The largest value of x over the ranks of the process group (x itself for one rank):
    every leg reports the slowest rank's time, as the whole job waits for it."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(units_per_rank: float, world: int, elapsed_s: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time
    (replicas: each rank works on its own SNP blocks, no exchange on the data path)."""
    return world * units_per_rank / elapsed_s


def flops_per_snp(n: int, q: int, t: int) -> float:
    """Algorithmic FP64 flops per SNP: the lower-triangular product L^{-1} x_i
    (n(n+1)/2 multiply-adds) plus the fused reductions (2n(q+1+t))."""
    return n * (n + 1) + 2.0 * n * (q + 1 + t)


def bf16_flops_per_snp(n: int, q: int, t: int, limbs: int) -> float:
    """Algorithmic BF16 tensor flops per SNP of the limb path: `limbs` lower-triangular
    products (n(n+1) flop each) plus the `limbs` x (q+t) linear rows (2n flop each)."""
    return limbs * (n * (n + 1) + 2.0 * n * (q + t))


# DRAM traffic of the dominant kernel per block (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of the bench's own launch shape, summed over
# the block's launches: the limb kernel runs two per block of 1024 SNPs or more), valid only
# while the kernel source is the one captured (code_sha of its file) and, for the limb
# kernel, per L2 group size and layout (CTA pairs or one CTA, fused or separate linear
# rows; the traffic does not depend on the pipeline depth).
TRAFFIC = {
    "k_block_fp64": [
        {"file": "block_fp64.cu", "sha": "9b94cec0bf31ad7a", "n": 10000, "m_blk": 16384,
         "bytes": 2062744832 + 111498752},
        {"file": "block_fp64.cu", "sha": "9b94cec0bf31ad7a", "n": 30000, "m_blk": 2048,
         "bytes": 9495486464 + 60372992}],
    # a mixed block of 16,384 SNPs is two launches of 8,192 (the two halves): bytes per block
    "k_block_mixed<3>": [
        {"file": "block_mixed.cu", "sha": "a98e3058f324fc0e", "n": 10000, "m_blk": 16384,
         "single_cta": False, "fuse": False, "ztail": False,
         "bytes_by_group_mb": {40: 1891798016 + 1898073600 + 10515200 + 7256832,
                               160: 3660850688 + 3656167680 + 9178880 + 6081792}},
        {"file": "block_mixed.cu", "sha": "a98e3058f324fc0e", "n": 10000, "m_blk": 16384,
         "single_cta": False, "fuse": False, "ztail": True,
         "bytes_by_group_mb": {40: 1937885696 + 1941512960 + 10448128 + 7621120,
                               160: 3591771904 + 3586308352 + 8904704 + 6366720}},
        {"file": "block_mixed.cu", "sha": "a98e3058f324fc0e", "n": 30000, "m_blk": 16384,
         "single_cta": False, "fuse": False, "ztail": False,
         "bytes_by_group_mb": {40: 63709729792 + 64894514944 + 27092480 + 23768576,
                               160: 44848629760 + 45610755584 + 27181824 + 23899136}},
        {"file": "block_mixed.cu", "sha": "a98e3058f324fc0e", "n": 30000, "m_blk": 16384,
         "single_cta": False, "fuse": False, "ztail": True,
         "bytes_by_group_mb": {40: 60897200384 + 66171474432 + 27252992 + 24198912,
                               160: 45278907136 + 47682639360 + 27141120 + 23846144}}],
}


def factor_record(stats: dict, n: int, args) -> dict:
    """The per-cohort factor (M, Cholesky, L^{-1}, the setup products) from gwas_factor's
    counters: its CUDA-event time without the upload of Phi, X_L and Y from host memory, at
    2n^3/3 FP64 flops (Cholesky n^3/3 + triangular inverse n^3/3; the n^2 terms are not
    counted), against the measured FP64 fma rate when it was probed."""
    up = float(stats.get("factor_upload_ms", 0.0))
    compute_ms = float(stats["factor_ms"]) - up
    flops = 2.0 * n ** 3 / 3.0
    rec = {"ms": float(stats["factor_ms"]), "upload_ms": up, "compute_ms": compute_ms,
           "launches": int(stats["factor_launches"]), "flops": flops,
           "fp64_tflops": flops / (compute_ms / 1e3) / 1e12 if compute_ms > 0 else None}
    probe = getattr(args, "fp64_probe", None)
    if probe and probe.get("tflops") and rec["fp64_tflops"]:
        rec["frac_of_fma_rate"] = rec["fp64_tflops"] / probe["tflops"]
    return rec


def tile_cfg_fields(tile_cfg) -> dict:
    """The tile_cfg bit fields as the library reads them (a negative value = defaults)."""
    d = {"stages": 0, "group_mb": 40, "single_cta": False, "pair": False, "fuse": False,
         "ztail": False}
    if tile_cfg is not None and tile_cfg >= 0:
        d["stages"] = tile_cfg & 0xF
        d["group_mb"] = ((tile_cfg >> 4) & 0xFF) or 40
        d["single_cta"] = bool((tile_cfg >> 12) & 1)
        d["pair"] = bool((tile_cfg >> 13) & 1)
        d["fuse"] = bool((tile_cfg >> 17) & 1) and not bool((tile_cfg >> 14) & 1)
        d["ztail"] = bool((tile_cfg >> 21) & 1) and not d["fuse"]
    return d


# Relative tolerance on b_i against the FP64 oracle that the parity tests hold each limb
# count to (tests/test_parity_mixed.py).
MIXED_TOL = {2: 1e-4, 3: 1e-6, 4: 1e-9, 5: 1e-10}


def traffic_for(kernel: str, n: int, m_blk: int, tile_cfg=None):
    recs = [r for r in TRAFFIC.get(kernel, []) if r["n"] == n and r["m_blk"] == m_blk]
    f = tile_cfg_fields(tile_cfg)
    # a record per tile layout: the one whose layout flags match tile_cfg's
    recs = [r for r in recs if "bytes_by_group_mb" not in r or
            all(f[k] == r.get(k, False) for k in ("single_cta", "fuse", "ztail"))]
    if not recs:
        return None
    rec = recs[0]
    nbytes = rec.get("bytes")
    if "bytes_by_group_mb" in rec:
        nbytes = rec["bytes_by_group_mb"].get(f["group_mb"])
    path = os.path.join(ROOT, "paper_1304_2272_gb300", "csrc", rec["file"])
    try:
        with open(path, encoding="utf-8") as f:
            sha = code_sha(f.read())
    except OSError:
        return None
    return nbytes if sha == rec["sha"] else None


def code_sha(src: str) -> str:
    """First 16 hex digits of the sha256 of a CUDA source with its comments and blank
    space removed: edits to comments keep a traffic record, any code change drops it."""
    import hashlib
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = re.sub(r"\s+", " ", src).strip()
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def h2d_peak_gbs(pinned, dev) -> float:
    """Host -> device copy rate of one pinned block on its own (cudaMemcpyAsync through
    torch, CUDA events), the denominator of the streaming roofline."""
    import torch
    d = torch.empty(pinned.shape, dtype=pinned.dtype, device=dev)
    s = torch.cuda.Stream(device=dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        d.copy_(pinned, non_blocking=True)          # warm-up
        e0.record(s)
        for _ in range(3):
            d.copy_(pinned, non_blocking=True)
        e1.record(s)
    e1.synchronize()
    nbytes = pinned.numel() * pinned.element_size()
    return 3 * nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9


def pack_2bit_torch(Xd):
    """(mb, n) device dosages in {0,1,2} -> (mb, ceil(n/4)) uint8 2-bit calls, four
    individuals per byte (individual k in bits 2(k%4), 2(k%4)+1 of byte k/4)."""
    import torch
    mb, n = Xd.shape
    nb = -(-n // 4)
    pad = torch.zeros((mb, 4 * nb), dtype=torch.uint8, device=Xd.device)
    pad[:, :n] = Xd.to(torch.uint8)
    q = pad.view(mb, nb, 4)
    return (q[..., 0] | (q[..., 1] << 2) | (q[..., 2] << 4) | (q[..., 3] << 6)).contiguous()


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def fp64_peak_tflops(sm_mhz: float | None) -> tuple[float, str]:
    """FP64 FMA peak from the unit count and the clock: 152 SMs x 2 FP64 FMA/clk/SM
    (1.25 TFLOP/s nominal at 2070 MHz) x 2 flops, at the median SM clock of the run."""
    mhz = sm_mhz if sm_mhz else 2070.0
    return 152 * 2 * 2 * mhz * 1e6 / 1e12, f"152 SM x 2 DFMA/clk x 2 flop x {mhz:.0f} MHz"


# SNPs per oracle call on the host, the same in every CPU leg and in the reference arm
# (the oracle's per-call rate depends on the size of its triangular solves).
CPU_BLOCK = 1024


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline records."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def blas_threads():
    """Threads of the OpenBLAS that numpy loaded (None if it cannot be asked)."""
    import ctypes
    libs = set()
    try:
        with open("/proc/self/maps") as f:
            for ln in f:
                parts = ln.split()
                if len(parts) >= 6 and "openblas" in os.path.basename(parts[-1]).lower() \
                        and ".so" in parts[-1]:
                    libs.add(parts[-1])
    except OSError:
        return None
    for path in sorted(libs):
        try:
            lib = ctypes.CDLL(path)
        except OSError:
            continue
        for sym in ("openblas_get_num_threads", "openblas_get_num_threads64_",
                    "scipy_openblas_get_num_threads64_", "scipy_openblas_get_num_threads"):
            fn = getattr(lib, sym, None)
            if fn is not None:
                fn.restype = ctypes.c_int
                return int(fn())
    return None


def oracle_rate(L, cohort, X_host, block: int, seconds: float, trsv: str = "auto"):
    """SNP/s of the oracle's Algorithm 1 route on blocks of `block` SNPs of X_host, run
    until `seconds` of compute or every column is used. Returns (rate, snps)."""
    import numpy as np
    from oracle import gls as G
    setup = G.setup_hoisted(L, cohort.XL, cohort.Y)
    done, elapsed = 0, 0.0
    while done < X_host.shape[1]:
        Xs = np.asfortranarray(X_host[:, done:done + block])
        t1 = time.perf_counter()
        G.gls_hoisted(L, cohort.XL, cohort.Y, Xs, trsv=trsv, setup=setup)
        elapsed += time.perf_counter() - t1
        done += Xs.shape[1]
        if elapsed >= seconds:
            break
    return done / elapsed, done


def cpu_worker(spec_path: str) -> None:
    """One single-threaded oracle process of the CPU baselines (the parent set the BLAS
    threads to 1): load L (memory-mapped), X_L, Y and a dosage chunk, report "ready",
    wait for "go" on stdin, time the chunk, print one JSON line."""
    import numpy as np
    from oracle import gls as G
    with open(spec_path) as f:
        spec = json.load(f)
    L = np.load(spec["L"], mmap_mode="r")
    d = np.load(spec["data"])
    XL, Y = d["XL"], d["Y"]
    X = np.asfortranarray(d["X"][:, spec["lo"]:spec["hi"]])
    setup = G.setup_hoisted(L, XL, Y)
    print("ready", flush=True)
    sys.stdin.readline()
    t0 = time.perf_counter()
    for c0 in range(0, X.shape[1], spec["block"]):
        G.gls_hoisted(L, XL, Y, np.asfortranarray(X[:, c0:c0 + spec["block"]]),
                      trsv=spec["trsv"], setup=setup)
    print(json.dumps({"snps": int(X.shape[1]), "seconds": time.perf_counter() - t0,
                      "blas_threads": blas_threads()}), flush=True)


def run_workers(L, cohort, X_host, chunks, block: int, trsv: str, deadline_s: float = 300.0) -> dict:
    """Start one single-threaded oracle process per (lo, hi) chunk of X_host, release them
    together and time them on the wall clock until the last one is done. Workers still
    running after deadline_s are killed (their output ends, which raises below)."""
    import tempfile
    import numpy as np
    base = "/dev/shm" if os.path.isdir("/dev/shm") else None
    with tempfile.TemporaryDirectory(dir=base) as tmp:
        np.save(os.path.join(tmp, "L.npy"), L)
        np.savez(os.path.join(tmp, "data.npz"), XL=cohort.XL, Y=cohort.Y, X=X_host)
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1",
                   MKL_NUM_THREADS="1")
        procs = []
        for k, (lo, hi) in enumerate(chunks):
            spec = os.path.join(tmp, f"spec{k}.json")
            with open(spec, "w") as f:
                json.dump({"L": os.path.join(tmp, "L.npy"), "data": os.path.join(tmp, "data.npz"),
                           "lo": lo, "hi": hi, "block": block, "trsv": trsv}, f)
            procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__),
                                           "--cpu-worker", spec], stdin=subprocess.PIPE,
                                          stdout=subprocess.PIPE, text=True, env=env, cwd=ROOT))
        def kill_all():
            for pr in procs:
                if pr.poll() is None:
                    pr.kill()
        watchdog = threading.Timer(deadline_s, kill_all)
        watchdog.start()
        try:
            for pr in procs:
                if pr.stdout.readline().strip() != "ready":
                    raise RuntimeError("a CPU baseline worker failed to start")
            t0 = time.perf_counter()
            for pr in procs:
                pr.stdin.write("go\n")
                pr.stdin.flush()
            lines = [pr.stdout.readline() for pr in procs]
            wall = time.perf_counter() - t0
            if not all(ln.strip() for ln in lines):
                raise RuntimeError("a CPU baseline worker ended without a result")
            outs = [json.loads(ln) for ln in lines]
            for pr in procs:
                pr.wait(timeout=60)
        finally:
            watchdog.cancel()
            kill_all()
    snps = sum(o["snps"] for o in outs)
    return {"value": snps / wall, "snps": snps, "wall_s": round(wall, 3),
            "blas_threads": outs[0]["blas_threads"]}


def cpu_baseline(cohort, X_host, seconds: float, flavours: bool = True) -> tuple[dict, object]:
    """The oracle as it stands, timed on the host cores: Algorithm 1 with multithreaded
    BLAS on blocks of CPU_BLOCK SNPs (the headline CPU number; a blocked dtrsm over SNP
    blocks, the shape of the paper's SMP design), and beside it the same route on one
    thread, the textbook row-loop substitution on one thread, and one single-threaded
    process per core each on its own SNPs (parallel over SNPs). Returns (record, L)."""
    from oracle import gls as G
    cores = os.cpu_count()
    model = cpu_model()
    t0 = time.perf_counter()
    L = G.factor(cohort.phi, cohort.h, cohort.sigma2)
    t_factor = time.perf_counter() - t0
    v, done = oracle_rate(L, cohort, X_host, CPU_BLOCK, seconds)
    threads = blas_threads() or cores
    rec = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{done} SNPs at n={cohort.n} in blocks of {CPU_BLOCK} after a one-off "
                     f"factor of {t_factor:.1f} s; Algorithm 1 route (LAPACK dtrsm), "
                     f"OpenBLAS threads {threads} of {cores} cores",
           "factor_s": round(t_factor, 2), "cpu_model": model, "host_cores": cores}
    if flavours:
        fl = [{"flavour": "algorithm1_blas_all_threads", "value": v, "unit": UNIT,
               "threads": threads, "snps": done}]
        try:
            one = run_workers(L, cohort, X_host, [(0, 256)], 256, "auto")
            fl.append({"flavour": "algorithm1_blas_1_thread", "value": one["value"],
                       "unit": UNIT, "threads": one["blas_threads"] or 1, "snps": one["snps"]})
            plain = run_workers(L, cohort, X_host, [(0, 32)], 32, "plain")
            fl.append({"flavour": "plain_row_loop_substitution_1_thread",
                       "value": plain["value"], "unit": UNIT,
                       "threads": plain["blas_threads"] or 1, "snps": plain["snps"]})
            procs = max(1, min(cores, X_host.shape[1]))
            per = min(256, X_host.shape[1] // procs)
            par = run_workers(L, cohort, X_host, [(k * per, (k + 1) * per) for k in range(procs)],
                              per, "auto")
            fl.append({"flavour": f"processes_over_snps_{procs}x1_thread", "value": par["value"],
                       "unit": UNIT, "threads": procs, "snps": par["snps"]})
        except (OSError, RuntimeError, ValueError, subprocess.SubprocessError) as e:
            fl.append({"flavour": "single-threaded workers", "error": str(e)[:200]})
        rec["flavours"] = fl
    return rec, L


def oracle_errors(L, cohort, sample) -> dict:
    """Largest error of the sampled outputs of a GPU leg against the FP64 oracle
    (Algorithm 1 route): b per SNP and phenotype relative to max_c |b_c| of the oracle,
    the Wald statistic relative to max(W, 1); statuses must agree exactly."""
    import numpy as np
    from oracle import gls as G
    rb, rw, rs = G.gls_hoisted(L, cohort.XL, cohort.Y, sample["X"])
    ok = rs == 0
    same = bool(np.array_equal(rs, sample["status"]))
    b, w = sample["b"][ok], sample["wald"][ok]
    scale = np.maximum(np.max(np.abs(rb[ok]), axis=-1, keepdims=True), 1e-300)
    err_b = float(np.max(np.abs(b - rb[ok]) / scale)) if ok.any() else 0.0
    err_w = float(np.max(np.abs(w - rw[ok]) / np.maximum(rw[ok], 1.0))) if ok.any() else 0.0
    return {"err_b": err_b, "err_wald": err_w, "status_match": same,
            "snps_checked": int(sample["snps"])}


def run_reference(args, rank, world):
    """CPU oracle arm: rank 0 only; each step solves a bounded sample of SNPs."""
    if rank != 0:
        return
    import numpy as np
    import synth
    from oracle import gls as G
    dev = None
    try:
        import torch
        if torch.cuda.is_available():
            dev = "cuda:0"
    except Exception:
        pass
    cohort = synth.make_cohort(0, args.n, t=args.t, device=dev)
    L = G.factor(cohort.phi, cohort.h, cohort.sigma2)
    setup = G.setup_hoisted(L, cohort.XL, cohort.Y)
    # the CPU baseline's block of SNPs per oracle call (scaled by n^2 away from n = 10k)
    per_step = max(8, min(CPU_BLOCK, int(CPU_BLOCK * 1e8 / (args.n * args.n))))
    blocks = [cohort.snps(per_step, stream=s) for s in range(args.warmup + args.steps)]
    for s in range(args.warmup):
        G.gls_hoisted(L, cohort.XL, cohort.Y, blocks[s], setup=setup)
    t0 = time.perf_counter()
    for s in range(args.steps):
        G.gls_hoisted(L, cohort.XL, cohort.Y, blocks[args.warmup + s], setup=setup)
    el = time.perf_counter() - t0
    v = per_step * args.steps / el
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": workload_config(args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": blas_threads() or os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{per_step} SNPs per step at n={args.n} (one oracle call, "
                                       "Algorithm 1 route, LAPACK dtrsm), OpenBLAS threads "
                                       f"{blas_threads()} of {os.cpu_count()} cores",
                             "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args) -> dict:
    prec = "FP64" if args.precision == "fp64" else f"mixed BF16x{args.limbs}"
    return {"workload": f"{prec} GLS, n={args.n}, p=4, t={args.t}, blocks of {args.m_blk} SNPs "
                        f"(block stream of a 1e6-SNP job)",
            "n": args.n, "p": 4, "t": args.t, "m_blk": args.m_blk, "precision": args.precision,
            "parallelism": f"replicas x{args.gpus}",
            "l2": f"inputs larger than L2: L^-1 is {8 * args.n * args.n / 1e6:.0f} MB and each "
                  f"dosage block {args.n * args.m_blk / 1e6:.0f} MB, {args.pool} distinct "
                  "blocks cycled"}


def sample_index(mb: int, k: int = 252, seed: int = 1):
    """The SNPs of a block whose outputs are checked against the oracle: the first and
    last SNP, both sides of the first 128-SNP tile boundary and k seeded others (the
    sample the parity tests use)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    pick = rng.choice(mb, min(k, mb), replace=False)
    return np.unique(np.concatenate([[0, min(127, mb - 1), min(128, mb - 1), mb - 1], pick]))


def measure(args, env, *, n, precision, limbs, steps, warmup, want_e2e=True, mb=None,
            packed_steps=None):
    """Factor one cohort, then time `steps` blocks (device-resident) and, if asked,
    the same blocks end to end from pinned host memory. Returns (result, cohort, pool);
    result["sample"] holds sampled dosages and outputs of the last timed block (host
    arrays) for the oracle check after every GPU leg."""
    import numpy as np
    import torch
    import synth
    from paper_1304_2272_gb300 import gwas

    rank, world, local, dev = env
    mb = args.m_blk if mb is None else mb
    t, p = args.t, 4
    prec = gwas.GWAS_PREC_FP64 if precision == "fp64" else gwas.GWAS_PREC_MIXED
    cohort = synth.make_cohort(0, n, t=t, device=dev)
    ctx = gwas.gwas_init(n, p, t, m_blk=mb, device=local, timing=1, precision=prec,
                         n_limbs=limbs)
    gwas.gwas_factor(ctx, np.asfortranarray(cohort.phi), True, cohort.h, cohort.sigma2,
                     cohort.XL, cohort.Y)
    fst = gwas.gwas_get_stats(ctx)
    setup_ms = fst["factor_ms"]
    factor = factor_record(fst, n, args)
    tune = None
    if precision == "mixed" and args.tile_cfg is not None:
        gwas.gwas_set_tile_cfg(ctx, args.tile_cfg)
        tune = {"tile_cfg": args.tile_cfg, "fixed": True}
    elif precision == "mixed" and not args.no_tune:
        from paper_1304_2272_gb300 import autotune
        t0 = time.perf_counter()
        tune = autotune.tuned_tile_cfg(ctx, n, p, t, prec, limbs, mb)
        tune["tune_s"] = round(time.perf_counter() - t0, 2)
    pool = [synth.genotypes_torch(1000 * rank + s, n, mb, dev) for s in range(args.pool)]
    b = torch.empty((mb, t, p), dtype=torch.float64, device=dev)
    w = torch.empty((mb, t), dtype=torch.float64, device=dev)
    st = torch.empty(mb, dtype=torch.uint8, device=dev)
    stream = torch.cuda.ExternalStream(gwas.gwas_stream(ctx), device=dev)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timing (value) --------------------------------------
    for s in range(warmup):
        gwas.gwas_solve_block_device(ctx, pool[s % args.pool], mb, b, w, st)
    gwas.gwas_sync(ctx)
    gwas.gwas_reset_stats(ctx)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0.record(stream)
    for s in range(steps):
        gwas.gwas_solve_block_device(ctx, pool[s % args.pool], mb, b, w, st)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    el_ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    stats = gwas.gwas_get_stats(ctx)
    status_ok = int((st == 0).sum().item())
    value = job_rate(steps * mb, world, el_ms / 1e3)
    idx = sample_index(mb)
    it = torch.from_numpy(idx).to(dev)
    sample = {"X": np.asfortranarray(pool[(steps - 1) % args.pool][it].cpu().numpy().T),
              "b": b[it].cpu().numpy(), "wald": w[it].cpu().numpy(),
              "status": st[it].cpu().numpy(), "snps": int(idx.size)}

    # ---- end to end from pinned host memory (e2e) ------------------------------
    e2e = None
    if want_e2e:
        hpool = [x.cpu().pin_memory() for x in pool[:2]]
        hb = torch.empty((mb, t, p), dtype=torch.float64).pin_memory()
        hw = torch.empty((mb, t), dtype=torch.float64).pin_memory()
        hs = torch.empty(mb, dtype=torch.uint8).pin_memory()
        for s in range(warmup):
            gwas.gwas_solve_block(ctx, hpool[s % 2], mb, hb, hw, hs)
        gwas.gwas_sync(ctx)
        barrier()
        t0 = time.perf_counter()
        for s in range(steps):
            gwas.gwas_solve_block(ctx, hpool[s % 2], mb, hb, hw, hs)
        gwas.gwas_sync(ctx)
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": job_rate(steps * mb, world, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": n * mb, "d2h_bytes_per_step": mb * (t * p * 8 + t * 8 + 1)}
        # secondary roofline: the dosage stream's H2D rate, and how much of the
        # device-resident rate survives streaming (1.0 = copies fully hidden)
        e2e["h2d_gbs"] = n * mb * steps * world / e2e_s / 1e9
        e2e["streamed_over_resident"] = e2e["value"] / value
        e2e["h2d_peak_gbs"] = h2d_peak_gbs(hpool[0], dev)
        e2e["h2d_frac"] = e2e["h2d_gbs"] / world / e2e["h2d_peak_gbs"]
        # the same stream as 2-bit calls (n/4 bytes per SNP), unpacked on the GPU
        ppool = [pack_2bit_torch(x).cpu().pin_memory() for x in pool[:2]]
        pk_steps = steps if packed_steps is None else max(1, min(steps, packed_steps))
        for s in range(min(warmup, 2)):
            gwas.gwas_solve_block_packed(ctx, ppool[s % 2], mb, gwas.CODE_DOSAGE, hb, hw, hs)
        gwas.gwas_sync(ctx)
        barrier()
        t0 = time.perf_counter()
        for s in range(pk_steps):
            gwas.gwas_solve_block_packed(ctx, ppool[s % 2], mb, gwas.CODE_DOSAGE, hb, hw, hs)
        gwas.gwas_sync(ctx)
        barrier()
        pk_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e["packed_2bit"] = {"value": job_rate(pk_steps * mb, world, pk_s), "unit": UNIT,
                              "steps": pk_steps,
                              "h2d_bytes_per_step": ppool[0].numel(),
                              "d2h_bytes_per_step": e2e["d2h_bytes_per_step"]}

    q = p - 1
    launch_ms = stats["trsm_ms"] / max(1, stats["trsm_launches"])
    if precision == "fp64":
        nominal, how = fp64_peak_tflops(clk.get("sm_mhz"))
        achieved = flops_per_snp(n, q, t) * mb / (launch_ms / 1e3) / 1e12
        probe = args.fp64_probe or {}
        peak = probe.get("tflops") or nominal
        src = ("gwas_fp64_fma_rate: FP64 fma chains timed on this GPU before the timed "
               f"region at a median {probe.get('sm_mhz')} MHz (of measured)") if probe.get(
                   "tflops") else how + " (derived, of nominal)"
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_for("k_block_fp64", n, mb),
                "kernel": "k_block_fp64",
                "launch_ms": launch_ms, "peak_source": src,
                "peak_nominal_derived": nominal, "frac_of_nominal": achieved / nominal,
                "nominal_source": how}
    else:
        pk = measured_peaks()
        long_run = el_ms >= 1000.0
        peak = pk.get("bf16_tflops_sustained" if long_run else "bf16_tflops")
        src = ("MEASURED_PEAKS.json " + ("bf16_tflops_sustained" if long_run else "bf16_tflops")
               + " (of measured)") if peak else "fallback 1700 TFLOP/s sustained (of fallback)"
        peak = peak or 1700.0
        achieved = bf16_flops_per_snp(n, q, t, limbs) * mb / (launch_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": traffic_for(f"k_block_mixed<{limbs}>", n, mb,
                                       (tune or {}).get("tile_cfg")),
                "kernel": f"k_block_mixed<{limbs}>",
                "launch_ms": launch_ms, "peak_source": src,
                "fp64_equivalent_tflops": flops_per_snp(n, q, t) * value / world / 1e12}
    # the clock effect apart from the kernel's efficiency: launch time x median SM clock
    # of the timed region, and the rate scaled to the maximum SM clock (compute-bound
    # kernels run in proportion to the clock)
    mhz, mhz_max = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    if mhz and mhz_max:
        roof["launch_ms_x_sm_ghz"] = launch_ms * mhz / 1e3
        roof["achieved_at_max_clock"] = achieved * mhz_max / mhz
        roof["frac_at_max_clock"] = roof["achieved_at_max_clock"] / roof["peak"]
    res = {"value": value, "ms_per_step": el_ms / steps, "steps": steps, "warmup": warmup,
           "setup_ms": setup_ms, "factor": factor, "roofline": roof, "e2e": e2e,
           "autotune": tune, "gpu_launches": int(stats["kernel_launches"]), "clocks": clk,
           "status_ok_last_block": status_ok, "sample": sample, "m_blk": mb}
    gwas.gwas_finalize(ctx)
    return res, cohort, pool


def measure_batch(args, env, precision, snps, steps, warmup):
    """Batched cohorts: args.batch_cohorts cohorts, n ~ U[1000, 8000], p = 4, 16
    phenotypes, h ~ U(0.2, 0.8), `snps` SNPs per cohort per step; one step = one batched
    solve (one grouped launch of the block kernel, replayed from a CUDA graph)."""
    import numpy as np
    import torch
    import synth
    from paper_1304_2272_gb300 import gwas

    rank, world, local, dev = env
    rng = np.random.default_rng(2026)
    ns = rng.integers(1000, 8001, size=args.batch_cohorts).tolist()
    hs = rng.uniform(0.2, 0.8, size=args.batch_cohorts)
    t, p = 16, 4
    prec = gwas.GWAS_PREC_FP64 if precision == "fp64" else gwas.GWAS_PREC_MIXED
    kw = {} if getattr(args, "batch_tile_cfg", None) is None else {"tile_cfg": args.batch_tile_cfg}
    b = gwas.gwas_batch_init(ns, p, t, precision=prec, m_blk=snps, device=local, timing=1,
                             n_limbs=args.limbs, use_graph=1, **kw)
    for k, n in enumerate(ns):
        c = synth.make_cohort(3000 + k, n, t=t, h=float(hs[k]), device=dev)
        gwas.gwas_batch_factor(b, k, np.asfortranarray(c.phi), True, c.h, c.sigma2, c.XL, c.Y)
        del c
    setup_ms = gwas.gwas_batch_get_stats(b)["factor_ms"]
    X = [synth.genotypes_torch(7000 + 100 * rank + k, n, snps, dev) for k, n in enumerate(ns)]
    bo = [torch.empty((snps, t, p), dtype=torch.float64, device=dev) for _ in ns]
    wo = [torch.empty((snps, t), dtype=torch.float64, device=dev) for _ in ns]
    so = [torch.empty((snps,), dtype=torch.uint8, device=dev) for _ in ns]
    mbs = [snps] * len(ns)
    stream = torch.cuda.ExternalStream(gwas.gwas_batch_stream(b), device=dev)
    torch.cuda.synchronize()
    for _ in range(warmup):
        gwas.gwas_batch_solve_device(b, X, mbs, bo, wo, so)
    gwas.gwas_batch_sync(b)
    gwas.gwas_batch_reset_stats(b)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    for _ in range(steps):
        gwas.gwas_batch_solve_device(b, X, mbs, bo, wo, so)
    ev1.record(stream)
    gwas.gwas_batch_sync(b)
    clk = clocks.stop()
    el_ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    st = gwas.gwas_batch_get_stats(b)
    ok = int(sum(int((x == 0).sum().item()) for x in so))
    gwas.gwas_batch_finalize(b)
    total = world * steps * snps * len(ns)
    work = sum(n * (n + 1) + 2.0 * n * (3 + 1 + t) for n in ns) * snps
    res = {"precision": precision, "cohorts": len(ns), "n_min": min(ns), "n_max": max(ns),
           "phenotypes": t, "snps_per_cohort": snps, "steps": steps,
           "value": total / (el_ms / 1e3), "unit": "cohort-SNP/s",
           "snp_phenotypes_per_s": t * total / (el_ms / 1e3), "ms_per_step": el_ms / steps,
           "fp64_equivalent_tflops": work * steps / (el_ms / 1e3) / 1e12,
           "setup_ms": setup_ms, "graph": True, "gpu_launches": int(st["kernel_launches"]),
           "status_ok": ok, "clocks": clk,
           "workload": f"{len(ns)} cohorts n ~ U[1000, 8000], p=4, {t} phenotypes, {snps} SNPs "
                       "per cohort per step" + ("" if snps >= 50000 else
                                                " (a prefix of the 50,000-SNP cohorts, timed "
                                                "as a rate)")}
    if precision == "mixed":
        bf16 = sum(args.limbs * (n * (n + 1) + 2.0 * n * (3 + t)) for n in ns) * snps
        res["bf16_tflops"] = bf16 * steps / (el_ms / 1e3) / 1e12
    return res


def measure_adjoint(args, env, steps, warmup):
    """REML fit of h from h0 = 0.1 (profiled sigma^2, gradient from the library's
    adjoint) and the gradient pass: b_i and db_i/dh for blocks of m_blk SNPs, n = 10,000,
    FP64 (forward L^-1 x_i plus the recomputed M^-1 x_i of the adjoint)."""
    import numpy as np
    import torch
    import synth
    from paper_1304_2272_gb300 import gwas
    from paper_1304_2272_gb300.reml import REMLEngine, fit_h

    rank, world, local, dev = env
    n, mb, t, p = args.n, args.m_blk, 1, 4
    c = synth.make_cohort(0, n, t=t, h=0.4, device=dev)
    e = REMLEngine(c.phi, c.XL, c.Y, m_blk=mb, device=local, timing=1)
    t0 = time.perf_counter()
    fit = fit_h(e, h0=0.1)
    fit_s = time.perf_counter() - t0
    # the gradient pass at the fitted h
    r = e.eval(fit["h"], fit["sigma2"])
    X = [synth.genotypes_torch(900 + 10 * rank + s, n, mb, dev) for s in range(2)]
    b = torch.empty((mb, t, p), dtype=torch.float64, device=dev)
    st = torch.empty(mb, dtype=torch.uint8, device=dev)
    d = torch.empty((mb, t, p), dtype=torch.float64, device=dev)
    stream = torch.cuda.ExternalStream(gwas.gwas_stream(e.ctx), device=dev)
    torch.cuda.synchronize()
    for s in range(warmup):
        gwas.gwas_solve_block_grad_device(e.ctx, X[s % 2], mb, b, None, st, d)
    gwas.gwas_sync(e.ctx)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    for s in range(steps):
        gwas.gwas_solve_block_grad_device(e.ctx, X[s % 2], mb, b, None, st, d)
    ev1.record(stream)
    gwas.gwas_sync(e.ctx)
    clk = clocks.stop()
    el_ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    ok = int((st == 0).sum().item())
    e.close()
    q = p - 1
    work = (n * (n + 1) + 2.0 * n * n + 4.0 * n * (q + 1 + t)) * mb * steps
    return {"n": n, "m_blk": mb, "steps": steps, "value": world * steps * mb / (el_ms / 1e3),
            "unit": "SNP/s (b_i and db_i/dh)", "ms_per_step": el_ms / steps,
            "fp64_tflops": work / (el_ms / 1e3) / 1e12,
            "reml_fit": {"h0": 0.1, "h": fit["h"], "sigma2": fit["sigma2"], "true_h": 0.4,
                         "loglik": fit["loglik"], "dl_dh": fit["dl_dh"], "evals": fit["evals"],
                         "seconds": round(fit_s, 2)},
            "status_ok": ok, "clocks": clk}


# Relative tolerance on the Wald statistic (against max(W, 1)) that the parity tests hold
# each limb count to (tests/test_parity_mixed.py), and that of the FP64 path.
MIXED_WALD_TOL = {3: 1e-5, 4: 1e-8, 5: 1e-10}
FP64_TOL = {"b": 1e-10, "wald": 1e-10}


def probe_fp64(local: int) -> dict:
    """Measured FP64 fma rate of this GPU (the FP64 roofline), with the clocks it ran at."""
    from paper_1304_2272_gb300 import gwas
    clocks = ClockSampler(local)
    clocks.start()
    r = gwas.gwas_fp64_fma_rate(local)
    clk = clocks.stop()
    return {"tflops": r, "sm_mhz": clk.get("sm_mhz"), "clocks": clk}


def main():
    args = parse()
    if args.cpu_worker:
        return cpu_worker(args.cpu_worker)
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(dev))
    env = (rank, world, local, dev)
    args.fp64_probe = probe_fp64(local) if args.precision == "fp64" else None
    res, cohort, pool = measure(args, env, n=args.n, precision=args.precision,
                                limbs=args.limbs, steps=args.steps, warmup=args.warmup,
                                packed_steps=5)
    cohorts = {args.n: cohort}
    checks = [(res, args.n)]  # (record, n): sampled outputs checked against the oracle
    fp64_legs = []
    if args.precision == "fp64" and not args.no_fp64_n30k:
        # the metric's second FP64 point: n = 30,000 in blocks of 2,048 SNPs (a prefix of
        # the n = 30k job, timed as a rate; each block is ~1.5 s of FP64 work)
        r, c30, _ = measure(args, env, n=30000, precision="fp64", limbs=args.limbs,
                            steps=args.fp64_n30k_steps, warmup=1, want_e2e=False, mb=2048)
        cohorts[30000] = c30
        leg = {"n": 30000, "m_blk": 2048, "precision": "fp64",
               "workload": "FP64 GLS, n=30000, p=4, t=1, blocks of 2048 SNPs (a prefix of the "
                           "n=30k job timed as a rate)",
               "tolerance_rel_b": FP64_TOL["b"], "tolerance_wald": FP64_TOL["wald"],
               "value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"],
               "steps": r["steps"], "setup_ms": r["setup_ms"], "factor": r["factor"],
               "roofline": r["roofline"], "clocks": r["clocks"],
               "gpu_launches": r["gpu_launches"], "sample": r["sample"]}
        fp64_legs.append(leg)
        checks.append((leg, 30000))
    mixed = []
    if args.precision == "fp64" and not args.no_mixed:
        # the metric's mixed legs (3 limbs: b within 1e-6 of FP64), and 5 limbs at n = 10k,
        # whose b agrees with the FP64 oracle to the FP64 path's own 1e-10
        # n = 30k: every block of the 5,000,000-SNP job (4 distinct dosage blocks cycled)
        n30k_steps = max(1, -(-args.mixed_n30k_snps // args.m_blk))
        legs = ((args.n, args.limbs, args.mixed_steps),
                (30000, args.limbs, n30k_steps),
                (args.n, 5, max(1, args.mixed_steps // 2)))
        for n_mx, limbs_mx, steps_mx in legs:
            r, c_mx, _ = measure(args, env, n=n_mx, precision="mixed", limbs=limbs_mx,
                                 steps=steps_mx, warmup=args.warmup, packed_steps=steps_mx)
            cohorts.setdefault(n_mx, c_mx)
            del c_mx
            leg = {"n": n_mx, "limbs": limbs_mx,
                   "workload": f"mixed BF16x{limbs_mx} GLS, n={n_mx}, p=4, t={args.t}, "
                               f"{steps_mx} blocks of {args.m_blk} SNPs"
                               + (f" ({steps_mx * args.m_blk} SNPs: the whole "
                                  f"{args.mixed_n30k_snps}-SNP job, 4 distinct dosage blocks "
                                  "cycled)" if n_mx == 30000 else ""),
                   "tolerance_rel_b": MIXED_TOL.get(limbs_mx),
                   "tolerance_wald": MIXED_WALD_TOL.get(limbs_mx),
                   "value": r["value"], "unit": UNIT,
                   "ms_per_step": r["ms_per_step"], "steps": steps_mx,
                   "setup_ms": r["setup_ms"], "roofline": r["roofline"],
                   "e2e": r["e2e"], "clocks": r["clocks"], "autotune": r["autotune"],
                   "gpu_launches": r["gpu_launches"], "sample": r["sample"]}
            mixed.append(leg)
            checks.append((leg, n_mx))
    adjoint = None
    if args.precision == "fp64" and not args.no_adjoint:
        adjoint = measure_adjoint(args, env, args.adjoint_steps, 1)
    batched = []
    if args.precision == "fp64" and not args.no_batch:
        batched.append(measure_batch(args, env, "mixed", args.batch_snps, 5, 2))
        batched.append(measure_batch(args, env, "fp64", args.batch_snps_fp64, 2, 1))
    if rank == 0:
        line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world,
                "steps": res["steps"], "warmup": res["warmup"], "ms_per_step": res["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else f"bf16x{args.limbs}+f64",
                "data": "synthetic", "config": workload_config(args),
                "setup_ms": res["setup_ms"], "factor": res["factor"],
                "roofline": res["roofline"], "e2e": res["e2e"],
                "gpu_launches": res["gpu_launches"], "clocks": res["clocks"],
                "status_ok_last_block": res["status_ok_last_block"]}
        if args.fp64_probe:
            line["fp64_peak_probe"] = {k: v for k, v in args.fp64_probe.items()}
        if fp64_legs:
            line["fp64"] = fp64_legs
        if mixed:
            line["mixed"] = mixed
        if batched:
            line["batched"] = batched
        if adjoint:
            line["adjoint"] = adjoint
        # CPU work only after every timed GPU leg: the oracle on the host cores
        factors = {}
        if not args.no_cpu_baseline:
            Xh = np.asfortranarray(pool[0][:4096].cpu().numpy().T)
            line["cpu_baseline"], factors[args.n] = cpu_baseline(cohort, Xh, args.cpu_seconds)
        if not args.no_oracle_check:
            from oracle import gls as G
            for rec, n_chk in sorted(checks, key=lambda c: c[1]):
                c = cohorts[n_chk]
                if n_chk not in factors:
                    t0 = time.perf_counter()
                    factors[n_chk] = G.factor(c.phi, c.h, c.sigma2)
                    line.setdefault("oracle_factor_s", {})[str(n_chk)] = round(
                        time.perf_counter() - t0, 1)
                rec["oracle_check"] = oracle_errors(factors[n_chk], c, rec["sample"])
            line["oracle_check"] = res["oracle_check"]
        for rec in [*fp64_legs, *mixed]:
            rec.pop("sample", None)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
