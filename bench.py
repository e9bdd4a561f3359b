#!/usr/bin/env python
"""Throughput benchmark of the PEXSI hot path: pole-solves per second.

Workload (default, --workload fluid): the 3D periodic water-like fluid, 512
"O" atoms (13 orbitals) + 1024 "H" atoms (5 orbitals), n = 11,776, 10 bohr
pair cutoff, beta = 1000 / Ha, a 60-pole expansion, complex FP64; mu at the
centre of the spectral interval and Delta E its half-width + 10%.

One step = one pass of the whole hot path over one batch of poles (4 by
default): the pole table, assembly of H - (z_l + mu) S, supernodal LDL^T,
selected inversion, the DM/EDM/FDM pole sum accumulated over the batch, the
Tr[DM S] check, and the step's share of the 16 real inertia shifts per 60
poles (cumulatively rounded, so that 15 steps of 4 poles take all 16). All
poles of a batch run in the same kernel launches. Successive steps walk
through the 60 poles. value = pole-solves / second of the plain FP64 path
with H and S resident on the device (no per-launch instrumentation in the
timed region; per-kernel shares come from separate instrumented steps);
e2e = the same steps through the host-buffer calls (H, S copied in and
DM/EDM/FDM copied out every step, from pinned host memory); dm_latency =
the full 60-pole pexsi_dm host call.

Beside it ("split_path", --split-compare 6): all supernode GEMMs (panel
solve, Schur update, Takahashi step, the Y[P,P] product, and the real ones of
the inertia LDL^T) as exact 6-slice bf16 products on the tcgen05 tensor
cores with FP64 in and out (the D-block inverses and the pole sum FP64), in
20-pole steps, with its roofline, its 60-pole call latency, and its error
against the FP64 path and the oracle on the poles that carry the DM.
"oracle_error" states the error of each path against the eigen closed form
of the oracle in sampled columns.

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
        oracle_pole_sample(s, mu, dE, i, args.cpu_cols, rng)
    per_pole = []
    wall = 0.0
    for i in range(args.steps):
        est, w = oracle_pole_sample(s, mu, dE, args.warmup + i, args.cpu_cols, rng)
        per_pole.append(est)
        wall += w
    v = 1.0 / float(np.mean(per_pole))
    cores = os.cpu_count()
    sample = (f"per step: dense LU of one {s.n}x{s.n} shifted matrix + {args.cpu_cols} of {s.n} columns "
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
def shifts_in_step(i: int, B: int, per60: int) -> tuple[int, int]:
    """Inertia shifts [a, b) of the 16-shift grid that step i takes: the
    shifts are spread over the steps in proportion to their poles (per60
    shifts per 60 poles), cumulatively rounded, cycling through the grid."""
    a = (i * B * per60) // 60
    b = ((i + 1) * B * per60) // 60
    return a, b


def make_step(px, plan, s, mu, dE, dH, dS, out, stream, B, per60, all_shifts, world=1, rank=0):
    """One step: a B-pole batch of the P-pole table (walking through the
    table) into the accumulated outputs, with Tr[DM S], and its share of the
    16 inertia shifts; device-resident H and S."""
    P = s.n_poles

    def step(i):
        b0 = ((i * world + rank) * B) % P
        b1 = min(P, b0 + B)
        info = px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, b0, b1, 1,
                                  out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), stream, want_info=True)
        a, b = shifts_in_step(i, B, per60)
        if b > a:
            sh = np.array([all_shifts[k % 16] for k in range(a, b)])
            px.pexsi_inertia_device(plan, dH.data_ptr(), dS.data_ptr(), sh, stream)
        if info["breakdown_front"] != -1:
            raise RuntimeError(f"breakdown in front {info['breakdown_front']}")
        return b1 - b0

    return step


def instrumented(px, plan, step, first, n, dev):
    """Per-kernel-class CUDA-event timings of n steps run after the timed
    region (the timed region itself runs without per-launch events)."""
    import torch
    px.pexsi_profile_reset(plan)
    px.pexsi_profile_enable(plan, True)
    for i in range(n):
        step(first + i)
    torch.cuda.synchronize(dev)
    prof = px.pexsi_profile_read(plan)
    px.pexsi_profile_enable(plan, False)
    return prof


def dm_latency(px, plan, s, mu, dE, calls: int) -> dict:
    """Latency of the full P-pole pexsi_dm host call (H, S in; DM, EDM, FDM
    out; synchronous), p50 / p99 over `calls` calls."""
    pin = lambda a: __import__("torch").from_numpy(a).pin_memory().numpy()
    H, S = pin(s.H), pin(s.S)
    lat = []
    for _ in range(calls):
        t0 = time.perf_counter()
        px.pexsi_dm(plan, H, S, mu, s.beta, s.n_poles, dE)
        lat.append(1e3 * (time.perf_counter() - t0))
    lat = np.array(lat)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "calls": calls, "samples_ms": [round(float(x), 1) for x in lat], "n_poles": s.n_poles,
            "call": "pexsi_dm (host buffers; H, S copied in, DM, EDM, FDM copied out)"}


def oracle_error(s, mu, dE, got: np.ndarray, poles_idx, ncols: int, eig=None) -> dict:
    """Largest error of DM / EDM / FDM in ncols sampled columns against the
    oracle's eigen closed form C (Lambda - z)^-1 C^T summed over poles_idx
    (absolute, and relative to the largest sampled entry)."""
    from oracle import dense, poles
    lam, C = eig if eig is not None else dense.eig_pencil(s.n, s.colptr, s.rowind, s.H, s.S)
    tab = poles.pole_table(s.beta, dE, s.n_poles, mu)
    cols = np.sort(np.random.default_rng(0).choice(s.n, ncols, replace=False))
    ref = dense.dm_columns_eig(lam, C, s.colptr, s.rowind, tab, cols, poles_idx)
    res = {}
    for q, name in enumerate(("dm", "edm", "fdm")):
        err = max(float(np.max(np.abs(got[q, s.colptr[j]:s.colptr[j + 1]] - ref[j][q]))) for j in cols)
        big = max(float(np.max(np.abs(ref[j][q]))) for j in cols)
        res[name] = {"max_abs": err, "rel_to_max_entry": err / big if big else None}
    return res


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
    B = args.poles_per_step or (20 if args.split else 4)
    per60 = WORKLOADS[args.workload]["shifts_per_60"]
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(device=local, max_batch=B,
                                                                              split_slices=args.split))
    st = px.pexsi_plan_get_stats(plan)
    dev = torch.device("cuda", local)
    dH = torch.from_numpy(s.H).to(dev)
    dS = torch.from_numpy(s.S).to(dev)
    out = torch.zeros(3, s.nnz, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    all_shifts = mu + np.linspace(-0.5, 0.5, 16) + 1.0e-4
    step = make_step(px, plan, s, mu, dE, dH, dS, out, stream, B, per60, all_shifts, world, rank)

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
    # ---- timed region (device-resident inputs, no per-launch instrumentation)
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
    total_solves = solves * world
    value = total_solves / (ms / 1000.0)
    # ---- per-kernel classes from separate instrumented steps
    prof = instrumented(px, plan, step, args.warmup + args.steps, args.profile_steps, dev)

    # ---- end to end through the host-buffer calls, pinned host memory
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    Hh, Sh = pin(s.H), pin(s.S)
    dmh, edmh, fdmh = (pin(np.zeros(s.nnz)) for _ in range(3))

    def host_step(i):
        b0 = ((i * world + rank) * B) % P
        b1 = min(P, b0 + B)
        px.pexsi_dm_poles(plan, Hh, Sh, mu, s.beta, P, dE, b0, b1, 0, dmh, edmh, fdmh)
        a, b = shifts_in_step(i, B, per60)
        if b > a:
            px.pexsi_inertia(plan, Hh, Sh, np.array([all_shifts[k % 16] for k in range(a, b)]))
        return b1 - b0, b - a

    host_step(0)
    barrier()
    t0 = time.perf_counter()
    e2e_solves = e2e_shifts = with_shifts = 0
    for i in range(args.e2e_steps):
        a, b = host_step(args.warmup + args.steps + i)
        e2e_solves += a
        e2e_shifts += b
        with_shifts += 1 if b else 0
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = e2e_solves * world / e2e_s
    steps_e2e = max(1, args.e2e_steps)
    # per step (averaged over the e2e steps): H and S into the DM call, and
    # again into the inertia call of a step that has shifts; DM, EDM, FDM and
    # the counts out
    h2d = int(2 * s.nnz * 8 * (steps_e2e + with_shifts) / steps_e2e)
    d2h = int(3 * s.nnz * 8 + 8 * e2e_shifts / steps_e2e)

    if rank != 0:
        px.pexsi_plan_destroy(plan)
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant launch class (CUDA events on the launch stream)
    kernels = {p["name"]: p for p in prof}
    dom = max(prof, key=lambda p: p["ms"])
    per_step_launches = (sum(p["launches"] for p in prof) + kernels["trace"]["launches"]) / max(1, args.profile_steps)
    total_kernel_ms = sum(p["ms"] for p in prof)
    peaks, peak_src = load_peaks()
    roofline = roofline_of(dom, total_kernel_ms, peaks, args.split)
    roofline["traffic"] = traffic_of(args.workload, dom, args.split)

    latency = dm_latency(px, plan, s, mu, dE, args.latency_calls) if args.latency_calls > 0 else None
    # the 16 inertia shifts of a counting cycle (Sec. II.C) in one call
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    px.pexsi_inertia_device(plan, dH.data_ptr(), dS.data_ptr(), all_shifts, stream)
    inertia_ms = 1e3 * (time.perf_counter() - t0)
    line = {
        "metric": "pole-solves/sec", "value": value, "unit": "pole-solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("f64 in/out; supernode GEMMs as bf16x%d slices on tcgen05 (exact fp32 / int64 accumulation)"
                  % args.split) if args.split else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "poles_per_step": B, "split_slices": args.split,
                   "inertia_shifts": f"{per60} per {P} poles, spread over the steps", "seed": args.seed,
                   "ordering": "own nested dissection", "nsuper": st["nsuper"], "nnz_L": st["nnz_L"],
                   "gemm_flops_per_pole": st["factor_gemm_flops"] + st["selinv_gemm_flops"],
                   "l2": f"no flush: each step streams {st['front_elems'] * 32 * B / 1e9:.1f} GB of fronts "
                         f"(> 129 MB L2)", "parallelism": "replicas" if world == 1 else f"poles sharded x{world}"},
        "roofline": roofline,
        "gemm_rate": gemm_rate(kernels),
        "kernels_per_step": per_step(prof, args.profile_steps),
        "e2e": {"value": e2e_value, "unit": "pole-solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
        "dm_latency": latency,
        "inertia_16_shifts": {"ms": inertia_ms, "shifts_per_s": 16 / (inertia_ms / 1e3),
                              "call": "pexsi_inertia_device, 16 shifts in [mu - 0.5, mu + 0.5] Ha"},
        "gpu_launches": int(round(per_step_launches * args.steps)),
        "clocks": clk,
        "peaks_source": peak_src,
    }
    ref_dm = None
    heavy = (max(0, P - 20), P)  # the poles that carry the density matrix
    if args.split_compare > 0 and args.split == 0 and world == 1:
        o = torch.zeros(3, s.nnz, dtype=torch.float64, device=dev)
        px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, heavy[0], heavy[1], 0,
                           o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr(), stream, want_info=True)
        ref_dm = o.cpu().numpy()
        del o
    px.pexsi_plan_destroy(plan)
    eig = None
    if world == 1 and args.oracle_cols > 0 and ref_dm is not None:
        from oracle import dense
        t0 = time.perf_counter()
        eig = dense.eig_pencil(s.n, s.colptr, s.rowind, s.H, s.S)
        eig_s = time.perf_counter() - t0
        line["oracle_error"] = {"batch": f"poles {heavy[0]}..{heavy[1] - 1} (those carrying the DM)",
                                "columns": args.oracle_cols, "oracle": "eigen closed form, sampled columns",
                                "eig_seconds": round(eig_s, 1),
                                "fp64_path": oracle_error(s, mu, dE, ref_dm, range(*heavy), args.oracle_cols, eig)}
    if args.split_compare > 0 and args.split == 0 and world == 1:
        line["split_path"] = split_path(px, s, mu, dE, local, dH, dS, stream, args, per60, all_shifts, ref_dm,
                                        heavy, eig, peaks)
    if world == 1 and args.batched_passes > 0:
        line["batched_split"] = batched_systems(px, local, args.split_compare or 6, args.batched_passes)
        line["batched_split_small"] = batched_systems(px, local, args.split_compare or 6, args.batched_passes,
                                                      which="small")
    if world == 1 and args.serve_requests > 0:
        line["serving"] = serve_trace(px, local, args.serve_rate, args.serve_requests, args.serve_set,
                                      args.serve_fp64_budget, capacity_frac=args.serve_capacity_frac)
    if world == 1 and not args.no_cpu_baseline:
        rng = np.random.default_rng(1)
        est, wall = oracle_pole_sample(s, mu, dE, 0, args.cpu_cols, rng)
        line["cpu_baseline"] = {
            "value": 1.0 / est, "unit": "pole-solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"1 pole: the oracle's dense O(n^3) route, not the sparse method -- LU of the {s.n}x{s.n} "
                       f"shifted matrix + {args.cpu_cols} of {s.n} columns solved ({wall:.1f} s), extrapolated "
                       f"to all columns = one pole-solve")}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def per_step(prof, steps: int) -> dict:
    """Per launch class and step: milliseconds, launches, algorithmic bytes
    and flops (from the library's CUDA-event profiler)."""
    k = max(1, steps)
    return {p["name"]: {"ms": round(p["ms"] / k, 3), "launches": p["launches"] / k, "bytes": p["bytes"] / k,
                        "flops": p["flops"] / k} for p in prof if p["launches"]}


def traffic_of(workload: str, dom: dict, split: int):
    """DRAM bytes per launch of the dominant class from the committed ncu
    summary profiles/traffic_<workload>.json, when it was taken for this
    kernel class and precision: the measured DRAM / algorithmic byte ratio of
    the captured launches times this run's algorithmic bytes per launch."""
    tpath = os.path.join(ROOT, "profiles", f"traffic_{workload}.json")
    if not os.path.exists(tpath):
        return None
    with open(tpath) as f:
        tj = json.load(f)
    if tj.get("kernel_class") != dom["name"] or tj.get("split_slices", 0) != split:
        return None
    ratio = tj.get("dram_over_algorithmic")
    if ratio is None or not dom["launches"]:
        return None
    return ratio * dom["bytes"] / dom["launches"]


def split_path(px, s, mu, dE, device, dH, dS, stream, args, per60, all_shifts, ref_dm, heavy, eig, peaks):
    """The split-precision path (bf16 Ozaki slices on the tcgen05 tensor
    cores) on the same workload: its throughput in 20-pole steps, the
    roofline of its dominant class, the latency of the full P-pole host call,
    and its error against the FP64 GPU path and the oracle on the poles that
    carry the DM."""
    import torch
    P, B = s.n_poles, 20
    S = args.split_compare
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind,
                          opts=px.pexsi_opts_default(device=device, max_batch=B, split_slices=S))
    o = torch.zeros(3, s.nnz, dtype=torch.float64, device=dH.device)
    step = make_step(px, plan, s, mu, dE, dH, dS, o, stream, B, per60, all_shifts)
    for i in range(3):
        step(i)
    torch.cuda.synchronize(dH.device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    solves = 0
    for i in range(args.split_steps):
        solves += step(3 + i)
    e1.record()
    torch.cuda.synchronize(dH.device)
    ms = e0.elapsed_time(e1)
    prof = instrumented(px, plan, step, 3 + args.split_steps, 1, dH.device)
    kern = {p["name"]: p for p in prof}
    dom = max(prof, key=lambda p: p["ms"])
    res = {"value": solves / (ms / 1e3), "unit": "pole-solves/s", "steps": args.split_steps, "poles_per_step": B,
           "ms_per_step": ms / args.split_steps, "split_slices": S,
           "dtype": f"f64 in/out; supernode GEMMs as bf16x{S} slices on tcgen05 (exact fp32 / int64 accumulation)",
           "roofline": roofline_of(dom, sum(p["ms"] for p in prof), peaks, S),
           "gemm_rate": gemm_rate(kern),
           "kernels_per_step": per_step(prof, 1)}
    res["roofline"]["traffic"] = traffic_of(args.workload, dom, S)
    px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, heavy[0], heavy[1], 0,
                       o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr(), stream, want_info=True)
    got = o.cpu().numpy()
    if ref_dm is not None:
        scale = [float(np.max(np.abs(ref_dm[k]))) for k in range(3)]
        dev_ = [float(np.max(np.abs(ref_dm[k] - got[k]))) for k in range(3)]
        res["vs_fp64_path"] = {"batch": f"poles {heavy[0]}..{heavy[1] - 1}",
                               "max_abs": dict(zip(("dm", "edm", "fdm"), dev_)),
                               "rel_to_max_entry": {k: d / sc for k, d, sc in zip(("dm", "edm", "fdm"), dev_, scale)}}
    if eig is not None:
        res["oracle_error"] = oracle_error(s, mu, dE, got, range(*heavy), args.oracle_cols, eig)
    full = px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, 0, P, 0,
                              o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr(), stream, want_info=True)
    res["trace_dm_s_all_poles"] = full["trace_dm_s"]
    if eig is not None:
        from oracle import dense, poles
        tr = dense.trace_eig(eig[0], poles.pole_table(s.beta, dE, P, mu), range(P))
        res["trace_error_all_poles"] = abs(full["trace_dm_s"] - tr[0])
    if args.split_latency_calls > 0:
        res["dm_latency"] = dm_latency(px, plan, s, mu, dE, args.split_latency_calls)
    px.pexsi_plan_destroy(plan)
    return res


# ------------------------------------------------------------------ batched systems
BATCHED_SETS = {
    # the six systems of the batched configuration, n = 2,000 to 30,000
    "config": [("chain500", lambda: ns.make_chain(natoms=500, seed=21)),
               ("fluid96", lambda: ns.make_fluid(nmol=96, seed=22)),
               ("sheet14", lambda: ns.make_sheet(ncell=14, seed=23)),
               ("fluid384", lambda: ns.make_fluid(nmol=384, seed=24)),
               ("sheet23", lambda: ns.make_sheet(ncell=23, seed=25)),
               ("chain7500", lambda: ns.make_chain(natoms=7500, seed=26))],
    # six systems at the small end of the range (n = 1,472 to 4,000), where no
    # single system fills the GPU
    "small": [("chain500", lambda: ns.make_chain(natoms=500, seed=21)),
              ("fluid96", lambda: ns.make_fluid(nmol=96, seed=22)),
              ("sheet8", lambda: ns.make_sheet(ncell=8, seed=27)),
              ("fluid64", lambda: ns.make_fluid(nmol=64, seed=28)),
              ("chain1000", lambda: ns.make_chain(natoms=1000, seed=29)),
              ("sheet12", lambda: ns.make_sheet(ncell=12, seed=30))],
}
BATCHED = BATCHED_SETS["config"]


def batched_systems(px, device, split, passes, P=64, which="config"):
    """Six systems of uneven size (chain, sheet and bulk recipes, n = 2,000
    to 30,000), P = 64 poles each, split precision, in one group: every
    level launch covers the fronts of all six systems for a wave of poles,
    the schedule (wave, Schur block width) chosen by the group's tuner.
    Reported against the same systems run one after another on their own
    plans, with each system's deviation from the FP64 path on the poles next
    to the real axis, and from the oracle's closed form for the two smallest."""
    import torch
    from oracle import dense, poles as opoles
    systems = []
    for name, make in BATCHED_SETS[which]:
        s = make()
        mu, dE = ns.mu_and_delta_e(s)
        systems.append((name, s, mu, dE))
    dev = torch.device("cuda", device)
    dH = [torch.from_numpy(s.H).to(dev) for _, s, _, _ in systems]
    dS = [torch.from_numpy(s.S).to(dev) for _, s, _, _ in systems]
    outs = [torch.zeros(3, s.nnz, dtype=torch.float64, device=dev) for _, s, _, _ in systems]
    st = torch.cuda.current_stream(dev).cuda_stream
    common = ([h.data_ptr() for h in dH], [x.data_ptr() for x in dS], [m for _, _, m, _ in systems],
              [s.beta for _, s, _, _ in systems], P, [d for _, _, _, d in systems])
    ptrs = ([o[0].data_ptr() for o in outs], [o[1].data_ptr() for o in outs], [o[2].data_ptr() for o in outs])

    def group_of(split_):
        plans = [px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(device=-1))
                 for _, s, _, _ in systems]
        g = px.pexsi_group_create(plans, opts=px.pexsi_opts_default(device=device, split_slices=split_))
        for p in plans:
            px.pexsi_plan_destroy(p)
        return g

    g = group_of(split)
    cache = os.path.join(tempfile.gettempdir(), "pexsi_gb300_schedules.txt")
    t0 = time.perf_counter()
    sched = px.pexsi_group_tune(g, *common, cache_path=cache)
    tune_s = time.perf_counter() - t0
    px.pexsi_group_dm_device(g, *common, 0, P, 0, *ptrs, st, want_info=True)  # warm-up pass
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(passes):
        px.pexsi_group_dm_device(g, *common, 0, P, 0, *ptrs, st)
    e1.record()
    torch.cuda.synchronize(dev)
    ms_group = e0.elapsed_time(e1) / passes
    stats = px.pexsi_group_get_stats(g)
    # poles next to the real axis on the occupied side, for the error checks
    lo, hi = P - 4, P
    px.pexsi_group_dm_device(g, *common, lo, hi, 0, *ptrs, st, want_info=True)
    split_near = [o.cpu().numpy() for o in outs]
    px.pexsi_group_destroy(g)
    # the same systems one after another, each on its own plan
    seq_ms = []
    for q, (name, s, mu, dE) in enumerate(systems):
        plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(device=device, split_slices=split))
        o = outs[q]
        args = (plan, dH[q].data_ptr(), dS[q].data_ptr(), mu, s.beta, P, dE)
        px.pexsi_dm_device(*args, 0, min(P, 8), 0, o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr(), st,
                           want_info=True)
        torch.cuda.synchronize(dev)
        e0.record()
        px.pexsi_dm_device(*args, 0, P, 0, o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr(), st)
        e1.record()
        torch.cuda.synchronize(dev)
        seq_ms.append(e0.elapsed_time(e1))
        px.pexsi_plan_destroy(plan)
    # FP64 path on the same poles
    g = group_of(0)
    px.pexsi_group_dm_device(g, *common, lo, hi, 0, *ptrs, st, want_info=True)
    fp64_near = [o.cpu().numpy() for o in outs]
    px.pexsi_group_destroy(g)
    errs = {}
    for q, (name, s, mu, dE) in enumerate(systems):
        d = float(np.max(np.abs(split_near[q] - fp64_near[q])))
        errs[name] = {"n": s.n, "vs_fp64_path_max_abs": d,
                      "rel_to_max_entry": d / float(np.max(np.abs(fp64_near[q][0])))}
        if s.n <= 2300:
            lam, C = dense.eig_pencil(s.n, s.colptr, s.rowind, s.H, s.S)
            tab = opoles.pole_table(s.beta, dE, P, mu)
            cols = np.sort(np.random.default_rng(0).choice(s.n, 8, replace=False))
            ref = dense.dm_columns_eig(lam, C, s.colptr, s.rowind, tab, cols, range(lo, hi))
            errs[name]["vs_oracle_sampled_max_abs"] = max(
                float(np.max(np.abs(split_near[q][k, s.colptr[j]:s.colptr[j + 1]] - ref[j][k])))
                for j in cols for k in range(3))
    solves = P * len(systems)
    return {"workload": "6 systems, 64 poles each: " + ", ".join(f"{nm} (n={s.n})" for nm, s, _, _ in systems),
            "split_slices": split, "pole_solves_per_pass": solves,
            "group": {"value": solves / (ms_group / 1e3), "unit": "pole-solves/s", "ms_per_pass": ms_group,
                      "passes": passes},
            "one_after_another": {"value": solves / (sum(seq_ms) / 1e3), "unit": "pole-solves/s",
                                  "ms_per_system": dict(zip([nm for nm, *_ in systems], [round(x, 1) for x in seq_ms]))},
            "speedup": sum(seq_ms) / ms_group,
            "schedule": sched, "tune_seconds": round(tune_s, 2), "front_elems": stats["front_elems"],
            "batch_capacity": stats["batch"],
            "error_poles": f"{lo}..{hi - 1} of each 64-pole table (occupied side, next to the real axis)",
            "error": errs}


# ------------------------------------------------------------------ serving trace
SERVE_SETS = {
    # the serving sizes: 2D and 3D recipes at n = 3.7k, 12k and 27k
    "config": [("sheet12x12", lambda: ns.make_sheet(ncell=12, seed=11)),
               ("fluid512", lambda: ns.make_fluid(nmol=512, seed=12)),
               ("sheet32x32", lambda: ns.make_sheet(ncell=32, seed=13))],
    # a small set that keeps the default benchmark short
    "small": [("sheet12x12", lambda: ns.make_sheet(ncell=12, seed=11)),
              ("fluid128", lambda: ns.make_fluid(nmol=128, seed=12)),
              ("chain1000", lambda: ns.make_chain(natoms=1000, seed=13, norb=4))],
}


def serve_trace(px, device, rate, n_req, which="small", fp64_budget_s=60.0, seed=0, capacity_frac=None):
    """Seeded Poisson trace of mu-search-shaped requests (8 inertia shifts,
    then one 60-pole DM) over the systems of SERVE_SETS[which], with
    per-request mu (+-0.05 Ha) and beta (+-10%) jitter, through the request
    server twice:
      split  -- continuous batching (4 slots, 8-pole device batches), plans
                with the split-precision GEMMs (6 bf16 slices);
      fp64   -- the plain per-pole FP64 path (1 slot, 1 pole per batch).
    The FP64 arm stops at fp64_budget_s of wall time: requests still queued or
    running are cancelled and enter its p50 / p99 at the budget, so its
    latencies are lower bounds. With capacity_frac the rate is that fraction
    of the split arm's measured capacity (requests/s of a first pass).
    Three requests of the split arm are replayed alone: results identical to
    the mix (deterministic kernels)."""
    rng = np.random.default_rng(seed)
    systems = []
    for name, make in SERVE_SETS[which]:
        s = make()
        mu, dE = ns.mu_and_delta_e(s)
        plans = {k: px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(device=device, split_slices=k))
                 for k in (0, 6)}
        systems.append((name, s, mu, dE, plans))
    gaps = rng.exponential(1.0, n_req)
    picks = rng.integers(0, len(systems), n_req)
    jit_mu = rng.uniform(-0.05, 0.05, n_req)
    jit_beta = rng.uniform(0.9, 1.1, n_req)

    def request(k, split):
        name, s, mu, dE, plans = systems[picks[k]]
        m = mu + jit_mu[k]
        return px.ServerRequest(plans[split], s.H, s.S, mu=m, beta=s.beta * jit_beta[k], n_poles=60,
                                delta_e=dE + 0.05, shifts=m + np.linspace(-0.2, 0.2, 8) + 1.0e-4)

    def run(slots, batch, split, rate_, budget=None, only=None):
        arrivals = np.cumsum(gaps / rate_)
        idx = list(range(n_req)) if only is None else only
        server = px.pexsi_server_create(px.pexsi_server_opts_default(device=device, slots=slots, batch=batch))
        reqs = []
        t0 = time.perf_counter()
        for k in idx:
            if only is None:
                while time.perf_counter() - t0 < arrivals[k]:
                    time.sleep(0.0005)
            r = request(k, split)
            px.pexsi_server_submit(server, r)
            reqs.append(r)
        res = []
        cancelled = False
        for r in reqs:
            while True:
                x = px.pexsi_server_poll(server, r.ticket)
                if x is not None:
                    break
                if budget is not None and not cancelled and time.perf_counter() - t0 > budget:
                    for q in reqs:  # everything unfinished at the budget
                        try:
                            px.pexsi_server_cancel(server, q.ticket)
                        except px.PexsiError:
                            pass  # finished in the meantime
                    cancelled = True
                time.sleep(0.002)
            res.append(x)
        wall = time.perf_counter() - t0
        st = px.pexsi_server_get_stats(server)
        px.pexsi_server_destroy(server)
        done = [x for x in res if x["status"] == 0]
        cut = [x for x in res if x["status"] == -7]
        lat = np.array([x["latency_ms"] if x["status"] == 0 else 1e3 * budget for x in res if x["status"] in (0, -7)])
        return {"p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                "completed": len(done), "cancelled_at_budget": len(cut),
                "failed": len(res) - len(done) - len(cut),
                "throughput_req_s": len(done) / wall, "pole_solves_s": 60 * len(done) / wall, "wall_s": wall,
                "peak_concurrent": st["peak_concurrent"]}, reqs, res

    rate_used = rate
    if capacity_frac:
        probe, _, _ = run(4, 8, 6, 1e6)  # all at once: the split arm's capacity
        rate_used = capacity_frac * probe["throughput_req_s"]
    split, r_split, res_split = run(4, 8, 6, rate_used)
    fp64, r_fp64, res_fp64 = run(1, 1, 0, rate_used, budget=fp64_budget_s)
    # determinism: three split requests replayed alone
    replay = [k for k in range(min(n_req, 3))]
    _, r_alone, _ = run(1, 8, 6, rate_used, only=replay)
    alone_diff = max(float(np.max(np.abs(a.dm - r_split[k].dm))) for a, k in zip(r_alone, replay))
    split_vs_fp64 = [float(np.max(np.abs(a.dm - b.dm))) for a, b, x in zip(r_split, r_fp64, res_fp64)
                     if x["status"] == 0]
    for *_, plans in systems:
        for p in plans.values():
            px.pexsi_plan_destroy(p)
    return {"workload": "Poisson arrivals; request = 8 inertia shifts + one 60-pole DM over "
                        + ", ".join(f"{n} (n={s.n})" for n, s, *_ in systems)
                        + "; mu jitter +-0.05 Ha, beta jitter +-10%",
            "rate_req_s": rate_used, "requests": n_req,
            "split_continuous": split, "fp64_plain_per_pole": fp64, "fp64_budget_s": fp64_budget_s,
            "alone_vs_mix_max_abs_dm": alone_diff,
            "split_vs_fp64_max_abs_dm": max(split_vs_fp64) if split_vs_fp64 else None}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="fluid")
    ap.add_argument("--poles-per-step", type=int, default=0,
                    help="poles per batch (0: 4 for the FP64 path, 20 for a split-precision run)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--profile-steps", type=int, default=2,
                    help="instrumented steps after the timed region (per-kernel CUDA-event timings)")
    ap.add_argument("--latency-calls", type=int, default=1,
                    help="full P-pole pexsi_dm host calls timed for the DM latency of the main path (0 = skip)")
    ap.add_argument("--oracle-cols", type=int, default=8,
                    help="sampled columns of the oracle check of the DM-carrying poles (0 = skip)")
    ap.add_argument("--cpu-cols", type=int, default=64, help="columns solved by the timed CPU oracle sample")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--split", type=int, default=0,
                    help="bf16 slices of the split-precision supernode GEMMs of the main path (0 = FP64)")
    ap.add_argument("--split-compare", type=int, default=6,
                    help="slices of the split-precision path reported beside the FP64 main path (0 = skip)")
    ap.add_argument("--split-steps", type=int, default=6, help="timed 20-pole steps of the split-precision path")
    ap.add_argument("--split-latency-calls", type=int, default=5,
                    help="full P-pole host calls timed for the split path's DM latency")
    ap.add_argument("--batched-passes", type=int, default=2,
                    help="timed passes of the six-system batched split-precision group (0 = skip)")
    ap.add_argument("--serve-requests", type=int, default=16, help="requests of the serving trace (0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=50.0, help="Poisson arrival rate of the serving trace")
    ap.add_argument("--serve-set", choices=sorted(SERVE_SETS), default="small",
                    help="systems of the serving trace (config: n = 3.7k, 12k, 27k)")
    ap.add_argument("--serve-fp64-budget", type=float, default=60.0,
                    help="wall seconds after which the plain FP64 arm's unfinished requests are cancelled")
    ap.add_argument("--serve-capacity-frac", type=float, default=0.0,
                    help="if > 0: arrival rate = this fraction of the split arm's measured capacity")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
