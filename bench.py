#!/usr/bin/env python
"""Throughput benchmark of the PEXSI hot path: pole-solves per second.

Workload (default, --workload fluid): the 3D periodic water-like fluid, 512
"O" atoms (13 orbitals) + 1024 "H" atoms (5 orbitals), n = 11,776, 10 bohr
pair cutoff, beta = 1000 / Ha, a 60-pole expansion, complex FP64; mu at the
centre of the spectral interval and Delta E its half-width + 10%.

One step = one pass of the whole hot path over one 20-pole batch: the pole
table, assembly of H - (z_l + mu) S, supernodal LDL^T, selected inversion,
the DM/EDM/FDM pole sum accumulated over the batch, the Tr[DM S] check, and
the inertia counts of a share of the real shifts (16 shifts per 60 poles, so
5 per step). All poles of a batch run in the same kernel launches; the batch
is as large as HBM allows because the top of the elimination tree has one
front per pole.
Successive steps walk through the 60 poles. value = pole-solves / second
with H and S resident on the device; e2e = the same through the host-buffer
call (H, S copied in and DM/EDM/FDM copied out every step, from pinned host
memory).

By default (--split 6) all supernode GEMMs (panel solve, Schur update,
Takahashi step, the Y[P,P] product, and the real ones of the inertia LDL^T)
run as exact 6-slice bf16 products on the tcgen05 tensor cores with FP64 in
and out; the D-block inverses and the pole sum are FP64. The plain FP64 path
is timed after it on the same workload ("fp64_path"), with the largest
difference between the two on one identical pole batch.

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


def roofline_of(dom: dict, total_kernel_ms: float, peaks: dict, split: int) -> dict:
    """Roofline entry of the dominant launch class. A class that runs on the
    tensor cores (the split-precision GEMMs) is measured by the bf16 flops its
    MMAs execute against the measured sustained bf16 peak (the class is timed
    inside a seconds-long step); an FP64 class by its algorithmic flops against
    the FP64 DFMA peak (no measured FP64 peak exists)."""
    secs = dom["ms"] / 1e3
    r = {"kernel": dom["name"], "launches": dom["launches"], "avg_launch_ms": dom["ms"] / max(1, dom["launches"]),
         "time_share": dom["ms"] / total_kernel_ms if total_kernel_ms else None}
    if dom.get("tensor_flops", 0) > 0 and secs > 0:
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
        ach = dom["tensor_flops"] / secs / 1e12
        r.update({"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                  "peak_source": "bf16_tflops_sustained of MEASURED_PEAKS.json (of measured)",
                  "fp64_equivalent_tflops": dom["flops"] / secs / 1e12,
                  "note": f"achieved = bf16 flops the tcgen05 MMAs execute: {split * (split + 1) // 2} slice pairs "
                          "x 4 real products x 2 flops per complex multiply-add; fp64_equivalent_tflops counts "
                          "8 flops per complex multiply-add of the FP64 product it replaces"})
    else:
        ach = dom["flops"] / secs / 1e12 if secs > 0 else 0.0
        r.update({"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                  "frac": ach / FP64_PEAK_TFLOPS,
                  "peak_source": "derived: FP64 DFMA 2/clk/SM x 152 SMs x 2.07 GHz (nominal 1.25 TFLOP/s)",
                  "executed_frac": ach * 6.0 / 8.0 / FP64_PEAK_TFLOPS,
                  "note": "achieved counts 8 real flops per complex multiply-add; the tiles execute 3 DFMA "
                          "(6 flops) per complex multiply-add (Gauss form), executed_frac is their DFMA rate"})
    return r


def gemm_rate(kernels: dict) -> dict:
    """FP64-equivalent rate of the four supernode GEMM classes together (and
    the split-precision slicing that feeds them, when present)."""
    names = ["panel_solve", "schur_update", "selinv_offdiag", "selinv_diag_partial", "split_slice"]
    ks = [kernels[k] for k in names if k in kernels]
    ms = sum(k["ms"] for k in ks)
    tf = sum(k["flops"] for k in ks) / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    return {"fp64_equivalent_tflops": tf, "fp64_peak_tflops": FP64_PEAK_TFLOPS, "vs_fp64_peak": tf / FP64_PEAK_TFLOPS}


def fp64_path(px, s, mu, dE, device, dH, dS, stream, args, B, Q, all_shifts, split_dm):
    """The plain FP64 path on the same workload and step (fewer timed steps),
    and the split path's deviation from it on one identical pole batch."""
    import torch
    P = s.n_poles
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind,
                          opts=px.pexsi_opts_default(device=device, max_batch=B, split_slices=0))
    o = torch.zeros(3, s.nnz, dtype=torch.float64, device=dH.device)
    px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, 0, B, 0,
                       o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr(), stream, want_info=True)
    ref = o.cpu().numpy()
    px.pexsi_profile_reset(plan)
    px.pexsi_profile_enable(plan, True)
    torch.cuda.synchronize(dH.device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.fp64_steps):
        b0 = ((1 + i) * B) % P
        px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, b0, min(P, b0 + B), 1,
                           o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr(), stream, want_info=True)
        sh = all_shifts[(i * Q) % 16:(i * Q) % 16 + Q]
        px.pexsi_inertia_device(plan, dH.data_ptr(), dS.data_ptr(), sh, stream)
    e1.record()
    torch.cuda.synchronize(dH.device)
    ms = e0.elapsed_time(e1)
    prof = px.pexsi_profile_read(plan)
    px.pexsi_plan_destroy(plan)
    kern = {p["name"]: p for p in prof}
    dom = max(prof, key=lambda p: p["ms"])
    scale = [float(np.max(np.abs(ref[k]))) for k in range(3)]
    dev = [float(np.max(np.abs(ref[k] - split_dm[k]))) for k in range(3)]
    return {"value": B * args.fp64_steps / (ms / 1e3), "unit": "pole-solves/s", "steps": args.fp64_steps,
            "ms_per_step": ms / args.fp64_steps, "dominant": roofline_of(dom, sum(p["ms"] for p in prof), {}, 0),
            "gemm_rate": gemm_rate(kern),
            "split_vs_fp64_same_batch": {"max_abs": {"dm": dev[0], "edm": dev[1], "fdm": dev[2]},
                                         "max_abs_over_max_entry": {"dm": dev[0] / scale[0], "edm": dev[1] / scale[1],
                                                                    "fdm": dev[2] / scale[2]},
                                         "batch": f"poles 0..{B - 1}"}}


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
                                                                              max_batch=args.poles_per_step,
                                                                              split_slices=args.split))
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

    # ---- roofline of the dominant launch class (live CUDA-event timings)
    kernels = {p["name"]: p for p in prof}
    dom = max(prof, key=lambda p: p["ms"])
    launches = sum(p["launches"] for p in prof) + kernels["trace"]["launches"]  # trace = 2 kernels
    total_kernel_ms = sum(p["ms"] for p in prof)
    peaks, peak_src = load_peaks()
    roofline = roofline_of(dom, total_kernel_ms, peaks, args.split)
    roofline["traffic"] = None
    tpath = os.path.join(ROOT, "profiles", f"traffic_{args.workload}.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        if tj.get("kernel") == dom["name"] and tj.get("split_slices", 0) == args.split:
            roofline["traffic"] = tj.get("dram_bytes_per_launch")

    # split-precision result against the FP64 path on one identical pole batch
    split_dm = None
    if args.split and args.fp64_steps > 0:
        o = torch.zeros(3, s.nnz, dtype=torch.float64, device=dev)
        px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, 0, B, 0,
                           o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr(), stream, want_info=True)
        split_dm = o.cpu().numpy()
        del o

    line = {
        "metric": "pole-solves/sec", "value": value, "unit": "pole-solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": (f"f64 in/out; supernode GEMMs as bf16x{args.split} slices on tcgen05 (exact fp32 / int64 "
                  f"accumulation)" if args.split else "f64"),
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "poles_per_step": B, "split_slices": args.split,
                   "inertia_shifts_per_step": Q, "seed": args.seed, "ordering": "own nested dissection",
                   "nsuper": st["nsuper"], "nnz_L": st["nnz_L"],
                   "gemm_flops_per_pole": st["factor_gemm_flops"] + st["selinv_gemm_flops"],
                   "l2": f"no flush: each step streams {st['front_elems'] * 32 * B / 1e9:.1f} GB of fronts "
                         f"(> 129 MB L2)", "parallelism": "replicas" if world == 1 else f"poles sharded x{world}"},
        "roofline": roofline,
        "gemm_rate": gemm_rate(kernels),
        "kernel_ms": {p["name"]: round(p["ms"], 3) for p in prof},
        "e2e": {"value": e2e_value, "unit": "pole-solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
        "gpu_launches": launches,
        "clocks": clk,
        "peaks_source": peak_src,
    }
    px.pexsi_plan_destroy(plan)
    if args.split and args.fp64_steps > 0:
        line["fp64_path"] = fp64_path(px, s, mu, dE, local, dH, dS, stream, args, B, Q, all_shifts, split_dm)
    if world == 1 and args.serve_requests > 0:
        line["serving"] = serve_trace(px, local, args.serve_rate, args.serve_requests)
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


# ------------------------------------------------------------------ serving trace
SERVE_SYSTEMS = [
    ("sheet8x8", lambda: ns.make_sheet(ncell=8, seed=11)),
    ("fluid64", lambda: ns.make_fluid(nmol=64, seed=12)),
    ("chain256", lambda: ns.make_chain(natoms=256, seed=13, norb=4)),
]


def serve_trace(px, device, rate, n_req, seed=0):
    """Seeded Poisson trace of mu-search-shaped requests (8 inertia shifts then
    one 60-pole DM) over three system sizes with per-request mu and beta
    jitter, through the request server twice: continuous batching (4 slots,
    8-pole device batches) and the plain per-pole path (1 slot, 1 pole per
    batch). Returns p50 / p99 latency and throughput of both."""
    rng = np.random.default_rng(seed)
    systems = []
    for name, make in SERVE_SYSTEMS:
        s = make()
        mu, dE = ns.mu_and_delta_e(s)
        plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(device=device))
        systems.append((name, s, mu, dE, plan))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    picks = rng.integers(0, len(systems), n_req)
    jit_mu = rng.uniform(-0.05, 0.05, n_req)
    jit_beta = rng.uniform(0.9, 1.1, n_req)

    def run(slots, batch):
        server = px.pexsi_server_create(px.pexsi_server_opts_default(device=device, slots=slots, batch=batch))
        reqs = []
        t0 = time.perf_counter()
        for k in range(n_req):
            while time.perf_counter() - t0 < arrivals[k]:
                time.sleep(0.0005)
            name, s, mu, dE, plan = systems[picks[k]]
            m = mu + jit_mu[k]
            r = px.ServerRequest(plan, s.H, s.S, mu=m, beta=s.beta * jit_beta[k], n_poles=60, delta_e=dE + 0.05,
                                 shifts=m + np.linspace(-0.2, 0.2, 8) + 1.0e-4)
            px.pexsi_server_submit(server, r)
            reqs.append(r)
        res = [px.pexsi_server_wait(server, r.ticket) for r in reqs]
        wall = time.perf_counter() - t0
        st = px.pexsi_server_get_stats(server)
        px.pexsi_server_destroy(server)
        lat = np.array([x["latency_ms"] for x in res])
        ok = all(x["status"] == 0 for x in res)
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "throughput_req_s": n_req / wall, "pole_solves_s": 60 * n_req / wall,
                "peak_concurrent": st["peak_concurrent"], "all_ok": ok}, reqs

    cont, r1 = run(4, 8)
    plain, r2 = run(1, 1)
    same = max(float(np.max(np.abs(a.dm - b.dm))) for a, b in zip(r1, r2))
    for *_, plan in systems:
        px.pexsi_plan_destroy(plan)
    return {"workload": "Poisson arrivals, requests = 8 inertia shifts + one 60-pole DM over "
                        + ", ".join(f"{n} (n={s.n})" for n, s, *_ in systems)
                        + "; mu jitter +-0.05 Ha, beta jitter +-10% (sizes scaled down from 4k-50k)",
            "rate_req_s": rate, "requests": n_req, "continuous": cont, "plain_per_pole": plain,
            "max_abs_dm_diff_between_modes": same}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="fluid")
    ap.add_argument("--poles-per-step", type=int, default=20,
                    help="poles per batch (20 x 7.3 GB of fronts on fluid512 fits 60%% of HBM)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--oracle-cols", type=int, default=64)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--split", type=int, default=6,
                    help="bf16 slices of the split-precision supernode GEMMs (0 = FP64 everywhere)")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the plain FP64 path reported beside a split-precision run (0 = skip)")
    ap.add_argument("--serve-requests", type=int, default=24, help="requests of the serving trace (0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=3.0, help="Poisson arrival rate of the serving trace")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
