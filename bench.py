#!/usr/bin/env python
"""SP2 time-to-D and effective TFLOP/s on one GB300 (whole SP2ACC expansion per step).

Workload (default): the precision form of the water-like recipe -- 8000
molecules of 24 basis functions, N = 192000, tile b = 32, tau = 1e-5,
Frobenius truncation, parameterless stop.  It is a seeded synthetic stand-in
for the paper's HF/3-21G water clusters.  The headline path is the mixed one:
tcgen05 tensor-core squares on four FP16 slices, with traces, norms, the
polynomial choice and the stop test in FP64.  The FP64 GPU path is timed once
on the same workload, and the difference of the two D's is reported (the
metric compares the two paths at ||D - D_FP64||_F <= 1e-6).
A step is one full pass of the method: sp2_create from the device-resident F
(Gershgorin bounds, schedule, X_0), then sp2_run (every iteration's symbolic
square, tile products with the fused epilogue, reductions, stop test,
truncation and compaction, then Step 3), ending with D on the device.

value = algorithmic FLOP/s of the whole job (2 * 32^3 per (I <= J, K) tile
triplet, summed over every square executed) / device time of the timed steps.
With --gpus N > 1 each rank runs an independent replica (the path runs on one
GPU; value sums all ranks' flops over the slowest rank's time).

--impl reference times the CPU oracle (plain numpy FP64) on a bounded sample of
the same recipe (203 molecules, N = 4872, tau = 1e-5 for the default workload)
on this host's cores.
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
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "SP2 time-to-D & eff. TFLOP/s, mixed vs FP64 GPU path at ||D-Dref||_F<=1e-6"
WORKLOADS = {
    "water192k": dict(key=3, sample="3s",
                      desc="water-like, 8000 molecules x 24 basis functions, N=192000, b=32, tau=1e-5, "
                           "Frobenius truncation, parameterless stop (the precision form)"),
    "water24k": dict(key=2, sample="2s",
                     desc="water-like, 1000 molecules x 24 basis functions, N=24000, b=32, tau=1e-6, "
                          "Frobenius truncation, parameterless stop"),
    "water2k": dict(key="2s", sample="2s", desc="water-like, 101 molecules, N=2424, b=32, tau=1e-6"),
    "water9k": dict(key="2m", sample="2s", desc="water-like, 400 molecules, N=9600, b=32, tau=1e-6"),
    "water24k-t5": dict(key="3m", sample="3s", desc="water-like, 1000 molecules, N=24000, b=32, tau=1e-5"),
    "helix128k": dict(key=4, sample="4s", desc="helix-like chain, 2000 residues x 64, N=128000, tau=1e-6"),
    "dense16k": dict(key=5, sample="5s", desc="dense N=16384, gap 0.05, tau=0, idempotency stop 1e-12"),
    "dense512": dict(key=1, sample=1, desc="dense N=512, tau=0, idempotency stop 1e-12"),
}
DEFAULT_WORKLOAD = "water192k"
PEAK_FP64_TFLOPS = 1.25   # GB300 FP64 nominal (no FP64 tensor path on this chip)

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum, mean bytes per launch) of the
# square kernel from one ncu capture of the default workload, keyed by the hash of the kernel
# code it was taken on (_source_hash); reported only while that code is unchanged.
SQUARE_TC_TRAFFIC = {("water192k", 4): ("27c4977856579cdc", 270.23e9)}


def _source_hash(name: str) -> str:
    """sha256 prefix of a kernel source without its // comments and blank lines
    (a comment edit leaves the captured counters valid; a code edit does not)."""
    import hashlib
    import re
    text = (ROOT / "paper_1909_12533_gb300" / "csrc" / name).read_text()
    code = "\n".join(ln.rstrip() for ln in (re.sub(r"//.*", "", t) for t in text.splitlines()) if ln.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def aggregate_ranks(ms: float, flops: float, world: int, device: str = "cuda") -> tuple[float, float]:
    """Whole-job figures of a replicated run (each rank an independent replica):
    the slowest rank's time and the sum of all ranks' flops (collectives of the
    initialised process group; a single rank returns its own figures)."""
    if world <= 1:
        return ms, flops
    import torch
    import torch.distributed as dist
    mx = torch.tensor([ms], dtype=torch.float64, device=device)
    sm = torch.tensor([flops], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[0])


def measured_peaks() -> dict:
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text())
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "fallback": True}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_oracle_sample(workload: str) -> dict:
    """The CPU oracle as it stands on a bounded sample of the same recipe."""
    import numpy as np
    import oracle.sp2_oracle as O
    from synth import from_dense, make_config, to_dense
    key = WORKLOADS[workload]["sample"]
    c = make_config(key)
    Fb = c["F"] if not isinstance(c["F"], np.ndarray) else from_dense(c["F"])
    F = to_dense(Fb)
    pattern = set(zip(Fb.brow.tolist(), Fb.bcol.tolist()))
    t0 = time.perf_counter()
    r = O.sp2(F, c["nocc"], c["homo_ub"], c["lumo_lb"], tau=c["tau"], stop=c["stop"], input_pattern=pattern)
    dt = time.perf_counter() - t0
    flops = 2.0 * 32 ** 3 * r.tile_triplets
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "seconds": dt, "flops": flops, "iterations": r.n,
            "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": f"one full SP2ACC run of the oracle (dense numpy FP64, BLAS on all host cores) on the "
                      f"same recipe reduced to config '{key}' (N={F.shape[0]}, tau={c['tau']:g})"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_oracle_sample(args.workload)
    samples = [cpu_oracle_sample(args.workload) for _ in range(args.steps)]
    tot_flops = sum(s["flops"] for s in samples)
    tot_s = sum(s["seconds"] for s in samples)
    v = tot_flops / tot_s / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"] + "; timed on the CPU sample: " +
                              samples[0]["sample"], "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": samples[0]["cores"], "kind": "oracle",
                             "sample": samples[0]["sample"]},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _tile_diff_norm(a, b, nb):
    """||A - B||_F of two symmetric tile sets (brow, bcol, val) on the device;
    tiles present in only one of them count in full; off-diagonal tiles twice."""
    import torch
    ka = a[0].long() * nb + a[1].long()
    kb = b[0].long() * nb + b[1].long()
    pos = torch.searchsorted(kb, ka).clamp(max=max(kb.numel() - 1, 0))
    hit = kb[pos] == ka if kb.numel() else torch.zeros_like(ka, dtype=torch.bool)
    wa = torch.where(a[0] == a[1], 1.0, 2.0).to(torch.float64)
    wb = torch.where(b[0] == b[1], 1.0, 2.0).to(torch.float64)
    da = a[2].clone()
    da[hit] -= b[2][pos[hit]]
    tot = (wa * (da * da).sum(dim=(1, 2))).sum()
    inb = torch.zeros(kb.numel(), dtype=torch.bool, device=kb.device)
    inb[pos[hit]] = True
    tot += (wb[~inb] * (b[2][~inb] ** 2).sum(dim=(1, 2))).sum()
    return float(tot.sqrt())


def _trace(D, n):
    import torch
    d = D[0] == D[1]
    idx = torch.arange(32, device=D[2].device)
    diag = D[2][d][:, idx, idx]
    return float(diag.sum())


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="split16", choices=["fp64", "split16"])
    ap.add_argument("--slices", type=int, default=4)
    ap.add_argument("--split-supply", type=int, default=None, choices=[0, 1],
                    help="tensor path: B slices through copy warps (1) or bulk copies only (0); default: library")
    ap.add_argument("--fp64-tail", type=float, default=None,
                    help="tensor path with the idempotency stop: FP64 squares once e_j < this (0: none); "
                         "default: library")
    ap.add_argument("--trunc", default=None, choices=["frobenius", "frobinf", "mixed"],
                    help="truncation norm (default: the library's, Frobenius)")
    ap.add_argument("--part", type=int, default=None, help="Frob-Inf / mixed-norm partition in rows")
    ap.add_argument("--storage", default="symmetric", choices=["symmetric", "general"],
                    help="general: both triangles stored and computed (the paper's general-matrix form)")
    ap.add_argument("--no-fp64-compare", action="store_true", help="skip the timed FP64 reference run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import paper_1909_12533_gb300 as sp2
    from synth import from_dense, make_config

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sp2.load()  # fails loudly if the library is missing

    wl = WORKLOADS[args.workload]
    c = make_config(wl["key"])
    Fh = c["F"] if not isinstance(c["F"], np.ndarray) else from_dense(c["F"])
    nb = Fh.nb

    class Dev:
        n = Fh.n
        brow = torch.from_numpy(Fh.brow).cuda()
        bcol = torch.from_numpy(Fh.bcol).cuda()
        val = torch.from_numpy(Fh.val).cuda()

    stream = torch.cuda.current_stream()
    extra = {} if args.split_supply is None else {"split_supply": args.split_supply}
    if args.fp64_tail is not None:
        extra["fp64_tail"] = args.fp64_tail
    if args.trunc is not None:
        extra["trunc"] = args.trunc
    if args.part is not None:
        extra["frobinf_part"] = args.part

    def step(F, precision, keep_D=False):
        ctx = sp2.SP2(F, c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], stop=c["stop"], precision=precision,
                      slices=args.slices, storage=args.storage, **extra)
        st = ctx.run()
        D = ctx.D_device() if keep_D else None
        ctx.close()
        return st, D

    for _ in range(args.warmup):
        step(Dev, args.precision)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stats = [step(Dev, args.precision)[0] for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    flops = sum(s["alg_flops"] for s in stats)
    sq_ms = sum(s["square_ms"] for s in stats)
    squares = sum(s["squares"] for s in stats)
    hw = sum(s["tc_hw_flops"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)
    ms_max, flops_all = aggregate_ranks(ms, flops, world)
    value = flops_all / (ms_max / 1e3) / 1e12

    e2e = None
    if not args.no_e2e:
        # through the public API from pinned host memory: every step uploads F, runs, and
        # copies D back into pinned host buffers (buffers filled / allocated before timing);
        # measured right after the device-timed steps, before the accuracy and FP64 runs,
        # which keep their D on the device
        class HostF:
            n = Fh.n
            brow = torch.from_numpy(Fh.brow).pin_memory()
            bcol = torch.from_numpy(Fh.bcol).pin_memory()
            val = torch.from_numpy(Fh.val).pin_memory()
        cap = int(stats[-1]["nnzb_final"] * 1.25) + 1024
        Dh = (torch.empty(cap, dtype=torch.int32).pin_memory(), torch.empty(cap, dtype=torch.int32).pin_memory(),
              torch.empty((cap, 32, 32), dtype=torch.float64).pin_memory())

        def e2e_step():
            ctx = sp2.SP2(HostF, c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], stop=c["stop"],
                          precision=args.precision, slices=args.slices, storage=args.storage, **extra)
            st = ctx.run()
            out = ctx.D_host(Dh)
            ctx.close()
            return st, out

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        runs = [e2e_step() for _ in range(args.steps)]
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        st, (brow, bcol, val) = runs[-1]
        h2d = Fh.val.nbytes + Fh.brow.nbytes + Fh.bcol.nbytes
        d2h = val.numel() * 8 + brow.numel() * 4 + bcol.numel() * 4
        e2e = {"value": sum(r[0]["alg_flops"] for r in runs) / args.steps / dt / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "seconds_per_step": dt,
               "host_buffers": "pinned"}

    # accuracy of this path, and the FP64 GPU path timed on the same workload
    st_main, D_main = step(Dev, args.precision, keep_D=True)
    fp64 = None
    err = None
    if args.precision != "fp64" and not args.no_fp64_compare:
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        st64, D64 = step(Dev, "fp64", keep_D=True)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        err = _tile_diff_norm(D_main, D64, nb)
        fp64 = {"time_to_D_ms": ms64, "eff_tflops": st64["alg_flops"] / ms64 / 1e9, "iterations": st64["n"],
                "steps": 1, "warmup": 0, "nnzb_final": st64["nnzb_final"],
                "speedup_of_mixed": ms64 / (ms_max / args.steps)}
    accuracy = {"D_minus_D_fp64_F": err, "trace_minus_nocc": _trace(D_main, Fh.n) - c["nocc"],
                "idempotency_e_n": st_main["e"][st_main["n"]], "iterations": st_main["n"],
                "ref": "FP64 GPU path (itself bit-for-bit parity-tested against the CPU oracle)"}

    if rank != 0:
        return 0
    peaks = measured_peaks()
    per_launch_flops = flops / max(squares, 1)
    per_launch_ms = sq_ms / max(squares, 1)
    achieved = per_launch_flops / (per_launch_ms / 1e3) / 1e12 if per_launch_ms > 0 else 0.0
    if args.precision == "fp64":
        roof = {"bound": "alu", "achieved": achieved, "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / PEAK_FP64_TFLOPS, "traffic": None, "kernel": "k_square_f64",
                "peak_source": "GB300 FP64 nominal 1.25 TFLOP/s (no FP64 tensor path); measured DFMA 1.19"}
    else:
        pk = peaks["bf16_tflops_sustained"]
        hw_ach = hw / (sq_ms / 1e3) / 1e12 if sq_ms > 0 else 0.0
        traffic = None
        ref = SQUARE_TC_TRAFFIC.get((args.workload, args.slices))
        if ref and _source_hash("square_tc.cu") == ref[0]:
            traffic = ref[1]
        roof = {"bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                "traffic": traffic, "kernel": "k_square_tc<%d>" % args.slices,
                "hw_achieved": hw_ach, "hw_frac": hw_ach / pk,
                "note": "achieved/frac count algorithmic flops (2*32^3 per tile triplet); hw_* count the "
                        "FP16 MMAs issued (slice pairs s + t <= %d, pairs that multiply an all-zero panel "
                        "slice skipped, 128x128 super-tile padding included); traffic = DRAM bytes per launch "
                        "from ncu, null when the kernel source differs from the captured one; the binding limit "
                        "is the supply of operand slices into shared memory (ncu on the water-like N=9600 "
                        "case: 6.9 TB/s of L2-to-SM reads, 86%% of the 8.0 TB/s that 8 KB bulk copies reach "
                        "with no compute), not the tensor pipe"
                        % (args.slices - 1),
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured; FP16 = BF16 rate)"}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f16x%d-split+f64" % args.slices,
        "data": "synthetic",
        "config": {"workload": wl["desc"], "precision": args.precision, "storage": args.storage,
                   "trunc": args.trunc or "frobenius", "part": args.part,
                   "slices": args.slices if args.precision == "split16" else None,
                   "l2": "inputs larger than L2 (F alone is %.0f MB)" % (Fh.val.nbytes / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "time_to_D_ms": ms_max / args.steps, "iterations": stats[-1]["n"], "squares": stats[-1]["squares"],
        "alg_flops_per_step": stats[-1]["alg_flops"], "nnzb_final": stats[-1]["nnzb_final"],
        "accuracy": accuracy, "fp64_path": fp64,
        "roofline": roof, "clocks": clk, "gpu_launches": int(launches), "e2e": e2e,
    }
    if not args.no_cpu_baseline and world == 1:
        cb = cpu_oracle_sample(args.workload)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
