#!/usr/bin/env python
"""Throughput benchmark of the PEXSI hot path: pole-solves per second.

Workload (default, --workload fluid): the 3D periodic water-like fluid, 512
"O" atoms (13 orbitals) + 1024 "H" atoms (5 orbitals), n = 11,776, 10 bohr
pair cutoff, beta = 1000 / Ha, a 60-pole expansion, complex FP64; mu at the
centre of the spectral interval and Delta E its half-width + 10%.

One step = one pass of the whole hot path over one pole batch: the pole
table, assembly of H - (z_l + mu) S, supernodal LDL^T, selected inversion,
the DM/EDM/FDM pole sum accumulated over the batch, the Tr[DM S] check, and
the inertia counts of a share of the real shifts (16 shifts per 60 poles).
Successive steps walk through the 60 poles. value = pole-solves / second
with H and S resident on the device; e2e = the same through the host-buffer
call (H, S copied in and DM/EDM/FDM copied out every step, from pinned host
memory).

With --impl reference the CPU oracle is timed instead on the same workload
(a bounded sample per step: the dense LU of one shifted matrix plus a
sample of its columns, extrapolated to one full pole-solve).

Multi-GPU (launched by torch.distributed.run): every rank evaluates its own
pole batches on its own GPU (poles are independent, weak scaling, no
collective on the data path); a barrier and a max over ranks bracket the
timed region.
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
sys.path.insert(0, ROOT)

import nao_synth as ns  # noqa: E402

WORKLOADS = {
    "fluid": dict(make=lambda seed: ns.make_fluid(nmol=512, seed=seed),
                  desc="fluid512: 3D periodic water-like fluid, 512 O (13 orb) + 1024 H (5 orb), n=11776, "
                       "10 bohr pair cutoff, decay 3 bohr, beta=1000/Ha, 60 poles, complex FP64",
                  shifts_per_60=16),
    "sheet": dict(make=lambda seed: ns.make_sheet(ncell=32, seed=seed),
                  desc="sheet32x32: periodic honeycomb sheet, 2048 atoms x 13 orb, n=26624, 8 A pair cutoff, "
                       "decay 3 bohr, beta=2000/Ha, 60 poles, complex FP64",
                  shifts_per_60=16),
    "fluid256": dict(make=lambda seed: ns.make_fluid(nmol=256, seed=seed),
                     desc="fluid256: the fluid recipe at half size (256 O + 512 H), n=5888, box 37.2 bohr, "
                          "beta=1000/Ha, 60 poles (profiling case)",
                     shifts_per_60=16),
    "chain": dict(make=lambda seed: ns.make_chain(seed=seed),
                  desc="chain64: 1D chain 64 atoms x 4 orb, n=256, 6 bohr cutoff, beta=1000/Ha, 40 poles",
                  shifts_per_60=16),
}

# FP64 on GB300 (sm_103): 2 DFMA / clock / SM (the nominal 1.25 TFLOP/s at
# the 2070 MHz maximum SM clock over 152 SMs).
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def prepare(workload: str, seed: int):
    w = WORKLOADS[workload]
    s = w["make"](seed)
    mu, dE = ns.mu_and_delta_e(s)
    return s, mu, dE


# ------------------------------------------------------------------ oracle arm
def oracle_pole_sample(s, mu, dE, pole: int, ncols: int, rng):
    """Time the oracle on one pole: dense LU + ncols column solves; returns
    the extrapolated seconds for one full pole-solve (all n columns)."""
    from oracle import poles, sampled
    tab = poles.pole_table(s.beta, dE, s.n_poles, mu)
    z = tab["z"][pole % s.n_poles]
    cols = np.sort(rng.choice(s.n, ncols, replace=False))
    t0 = time.perf_counter()
    lu = sampled.factor_shifted_dense(s.n, s.colptr, s.rowind, s.H, s.S, z)
    t1 = time.perf_counter()
    sampled.selected_columns_dense(s.n, s.colptr, s.rowind, s.H, s.S, z, cols, lu=lu)
    t2 = time.perf_counter()
    return (t1 - t0) + (t2 - t1) * s.n / ncols, t2 - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    s, mu, dE = prepare(args.workload, args.seed)
    rng = np.random.default_rng(1)
    for i in range(args.warmup):
        oracle_pole_sample(s, mu, dE, i, args.oracle_cols, rng)
    per_pole = []
    wall = 0.0
    for i in range(args.steps):
        est, w = oracle_pole_sample(s, mu, dE, args.warmup + i, args.oracle_cols, rng)
        per_pole.append(est)
        wall += w
    v = 1.0 / float(np.mean(per_pole))
    cores = os.cpu_count()
    sample = (f"per step: dense LU of one {s.n}x{s.n} shifted matrix + {args.oracle_cols} of {s.n} columns "
              f"solved, extrapolated to all columns = one pole-solve")
    line = {"impl": "reference", "metric": "pole-solves/sec", "value": v, "unit": "pole-solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "seed": args.seed},
            "cpu_baseline": {"value": v, "unit": "pole-solves/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "pole-solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_1405_0194_gb300 as px
    from paper_1405_0194_gb300 import build as pxbuild
    pxbuild.build()

    s, mu, dE = prepare(args.workload, args.seed)
    P = s.n_poles
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(device=local,
                                                                              max_batch=args.poles_per_step))
    st = px.pexsi_plan_get_stats(plan)
    dev = torch.device("cuda", local)
    dH = torch.from_numpy(s.H).to(dev)
    dS = torch.from_numpy(s.S).to(dev)
    out = torch.zeros(3, s.nnz, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    B = args.poles_per_step
    Q = max(1, round(WORKLOADS[args.workload]["shifts_per_60"] * B / 60))
    all_shifts = mu + np.linspace(-0.5, 0.5, 16) + 1.0e-4

    def step(i, on_device=True, host=None):
        b0 = ((i * world + rank) * B) % P
        b1 = min(P, b0 + B)
        sh = all_shifts[(i * Q) % 16:(i * Q) % 16 + Q]
        if on_device:
            info = px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, b0, b1, 1,
                                      out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), stream,
                                      want_info=True)
            px.pexsi_inertia_device(plan, dH.data_ptr(), dS.data_ptr(), sh, stream)
        else:
            Hh, Sh, dmh, edmh, fdmh = host
            info = px.pexsi_dm_poles(plan, Hh, Sh, mu, s.beta, P, dE, b0, b1, 0, dmh, edmh, fdmh)
            px.pexsi_inertia(plan, Hh, Sh, sh)
        if info["breakdown_front"] != -1:
            raise RuntimeError(f"breakdown in front {info['breakdown_front']}")
        return b1 - b0

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    for i in range(args.warmup):
        step(i)
    # ---- timed region (device-resident inputs)
    px.pexsi_profile_reset(plan)
    px.pexsi_profile_enable(plan, True)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    solves = 0
    for i in range(args.steps):
        solves += step(args.warmup + i)
    e1.record()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    prof = px.pexsi_profile_read(plan)
    px.pexsi_profile_enable(plan, False)
    total_solves = solves * world
    value = total_solves / (ms / 1000.0)

    # ---- end to end through the host-buffer call, pinned host memory
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    host = (pin(s.H), pin(s.S), pin(np.zeros(s.nnz)), pin(np.zeros(s.nnz)), pin(np.zeros(s.nnz)))
    step(0, on_device=False, host=host)
    barrier()
    t0 = time.perf_counter()
    e2e_solves = 0
    for i in range(args.e2e_steps):
        e2e_solves += step(args.warmup + args.steps + i, on_device=False, host=host)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = e2e_solves * world / e2e_s
    h2d = 2 * 2 * s.nnz * 8          # H and S into the DM call and into the inertia call
    d2h = 3 * s.nnz * 8 + 8 * Q      # DM, EDM, FDM and the counts

    if rank != 0:
        px.pexsi_plan_destroy(plan)
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel (live CUDA-event timings)
    kernels = {p["name"]: p for p in prof}
    dom = max(prof, key=lambda p: p["ms"])
    launches = sum(p["launches"] for p in prof) + kernels["trace"]["launches"]  # trace = 2 kernels
    achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12 if dom["ms"] > 0 else 0.0
    gemm = [kernels[k] for k in ("panel_solve", "schur_update", "selinv_offdiag", "selinv_diag_partial")]
    gemm_tf = sum(k["flops"] for k in gemm) / (sum(k["ms"] for k in gemm) / 1e3) / 1e12
    total_kernel_ms = sum(p["ms"] for p in prof)
    peaks, peak_src = load_peaks()
    traffic = None
    tpath = os.path.join(ROOT, "profiles", f"traffic_{args.workload}.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        if tj.get("kernel") == dom["name"]:
            traffic = tj.get("dram_bytes_per_launch")

    line = {
        "metric": "pole-solves/sec", "value": value, "unit": "pole-solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "poles_per_step": B,
                   "inertia_shifts_per_step": Q, "seed": args.seed, "ordering": "own nested dissection",
                   "nsuper": st["nsuper"], "nnz_L": st["nnz_L"],
                   "gemm_flops_per_pole": st["factor_gemm_flops"] + st["selinv_gemm_flops"],
                   "l2": f"no flush: each step streams {st['front_elems'] * 32 * B / 1e9:.1f} GB of fronts "
                         f"(> 129 MB L2)", "parallelism": "replicas" if world == 1 else f"poles sharded x{world}"},
        "roofline": {"bound": "alu", "kernel": dom["name"], "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                     "peak_source": "derived: FP64 DFMA 2/clk/SM x 152 SMs x 2.07 GHz (nominal 1.25 TFLOP/s)",
                     "launches": dom["launches"], "avg_launch_ms": dom["ms"] / max(1, dom["launches"]),
                     "time_share": dom["ms"] / total_kernel_ms if total_kernel_ms else None},
        "gemm_fraction_fp64": {"achieved_tflops": gemm_tf, "peak_tflops": FP64_PEAK_TFLOPS,
                               "frac": gemm_tf / FP64_PEAK_TFLOPS},
        "kernel_ms": {p["name"]: round(p["ms"], 3) for p in prof},
        "e2e": {"value": e2e_value, "unit": "pole-solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
        "gpu_launches": launches,
        "clocks": clk,
        "peaks_source": peak_src,
    }
    px.pexsi_plan_destroy(plan)
    if world == 1 and not args.no_cpu_baseline:
        rng = np.random.default_rng(1)
        est, wall = oracle_pole_sample(s, mu, dE, 0, args.oracle_cols, rng)
        line["cpu_baseline"] = {
            "value": 1.0 / est, "unit": "pole-solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"1 pole: dense LU of the {s.n}x{s.n} shifted matrix + {args.oracle_cols} of {s.n} columns "
                       f"solved ({wall:.1f} s), extrapolated to all columns = one pole-solve")}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="fluid")
    ap.add_argument("--poles-per-step", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--oracle-cols", type=int, default=64)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
