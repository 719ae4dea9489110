#!/usr/bin/env python
"""Benchmark of the short-range MD hot path: atom-timesteps/s on one GB300.

One benchmark step = md_step(inner) velocity-Verlet time steps (neighbour
rebuilds whenever some atom moved more than skin/2, exactly as in a
production run) followed by md_energy_virial (thermodynamic output), on the
2,048,000-atom Lennard-Jones system (80^3 fcc cells, rho* = 0.8442, T* = 0.72,
r_cut = 2.5, skin = 0.3, dt = 0.005), mixed precision, full neighbour lists.

Prints one JSON line (rank 0).  With --impl reference the FP64 CPU oracle is
timed instead, on bounded samples of the same workload.  Under torchrun every
rank runs its own replica (the method has no data exchange between
independent systems), and the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-timesteps/s"
WORKLOADS = {
    "lj_liquid_2048000": dict(n_cells=80, rho=0.8442, T=0.72, seed=2),
    # smaller case of the same kernels for profiler captures (lists still exceed L2)
    "lj_liquid_1048576": dict(n_cells=64, rho=0.8442, T=0.72, seed=2),
    # strongly inhomogeneous: fcc slab (30 % of a 151.2 sigma cube) plus 40 fcc nanoparticles in vacuum
    "slab_nanoparticles_1192114": dict(L=152.0, rho=0.8442, T=0.3, seed=3),
    # the same structure in the literal 300 sigma cube (supplementary row)
    "slab_nanoparticles_7239270": dict(L=300.0, rho=0.8442, T=0.3, seed=3),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--inner", type=int, default=100, help="MD time steps per benchmark step")
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--list", default="full", choices=["full", "half", "half_af"],
                   help="neighbour lists: full, half (8 colours, shared-memory atomics) or half_af (8 colours, "
                        "no atomics)")
    p.add_argument("--workload", default="lj_liquid_2048000", choices=sorted(WORKLOADS))
    p.add_argument("--no-extras", action="store_true", help="skip the FP64 / half-list comparison runs")
    p.add_argument("--cpu-steps", type=int, default=4,
                   help="oracle time steps in the all-cores CPU baseline sample (the single-thread leg times 1)")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--many-body", action="store_true",
                   help="only time the TB-SMA copper system (the many_body extra) and print it")
    p.add_argument("--only", choices=["ensemble", "force-matching"],
                   help="only time that extra (the batch_ensemble or force_matching entry) and print it")
    p.add_argument("--ensemble-steps", type=int, default=200, help="timed steps of the ensemble extra")
    p.add_argument("--no-autotune", action="store_true", help="ensemble extra: keep the default launch shapes")
    return p.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


def make_workload(name):
    from paper_1305_4196_gb300 import workloads as W
    w = WORKLOADS[name]
    if "L" in w:
        return W.slab_nanoparticles(w["L"], rho=w["rho"], T=w["T"], seed=w["seed"])
    return W.lj_fcc(w["n_cells"], rho=w["rho"], T=w["T"], seed=w["seed"])


def config_of(args, sysm, world):
    return {"workload": args.workload, "atoms": sysm.n, "box_sigma": float(sysm.box[0]),
            "rho": WORKLOADS[args.workload]["rho"], "T": WORKLOADS[args.workload]["T"], "r_cut": 2.5,
            "skin": 0.3, "dt": 0.005, "timesteps_per_step": args.inner, "precision": args.precision,
            "neighbour_list": args.list, "parallelism": f"replicas{world}" if world > 1 else "single",
            "l2": "working set > L2 (positions, lists and state exceed 129 MB)"}


def cpu_baseline(sysm, steps):
    """The FP64 oracle as it stands, timed on the host: the all-cores form (full neighbour
    sums, one writer per atom, OpenMP over every host core) over `steps` velocity-Verlet
    steps of the whole workload, and the single-thread serial form over one step.  Each
    timed step is exactly one force evaluation: the forces at the start come from an
    untimed evaluation and are carried from step to step."""
    from oracle import oracle as O
    O.build()
    P = O.LJParams.single()
    f0, _, threads = O.lj_forces_all_cores(sysm.pos, sysm.box, P)
    t0 = time.perf_counter()
    O.run_nve(sysm.pos, sysm.vel, sysm.box, P, 0.005, 0.3, steps, forces=f0, all_cores=True)
    dt_all = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.run_nve(sysm.pos, sysm.vel, sysm.box, P, 0.005, 0.3, 1, forces=f0)
    dt_one = time.perf_counter() - t0
    return {"value": sysm.n * steps / dt_all, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"{steps} velocity-Verlet steps of the full {sysm.n}-atom workload, one force "
                      f"evaluation per step (full neighbour sums), FP64, {threads} host threads "
                      f"(os.cpu_count() = {os.cpu_count()})", "seconds": dt_all,
            "single_thread": {"value": sysm.n / dt_one, "unit": METRIC, "cores": 1, "kind": "oracle",
                              "sample": f"1 velocity-Verlet step of the full {sysm.n}-atom workload (one "
                                        f"Newton-3 force evaluation), FP64, single thread", "seconds": dt_one}}


def run_reference(args):
    """--impl reference: the CPU oracle on every host core, one velocity-Verlet step (one
    force evaluation; the forces are carried from step to step) of the whole workload per
    benchmark step."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    sysm = make_workload(args.workload)
    P = O.LJParams.single()
    x, v = sysm.pos.copy(), sysm.vel.copy()
    img = np.zeros((sysm.n, 3), dtype=np.int32)
    f, _, threads = O.lj_forces_all_cores(x, sysm.box, P)

    def one():
        r = O.run_nve(x, v, sysm.box, P, 0.005, 0.3, 1, image=img, forces=f, all_cores=True)
        return r["pos"], r["vel"], r["image"], r["forces"]

    for _ in range(args.warmup):
        x, v, img, f = one()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        x, v, img, f = one()
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sysm.n * args.steps / total
    cfg = config_of(args, sysm, world)
    cfg["timesteps_per_step"] = 1
    cfg["precision"] = "fp64"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded fcc start, Gaussian velocities)", "config": cfg,
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle",
                             "sample": "1 velocity-Verlet step of the full workload per benchmark step, one "
                                       "force evaluation (full neighbour sums, forces carried from the "
                                       f"previous step), FP64, {threads} host threads "
                                       f"(os.cpu_count() = {os.cpu_count()})"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measured_force_traffic(n, fused):
    """DRAM bytes per launch of the force kernel (fused: with velocity Verlet) from the
    committed ncu capture (profiles/force_traffic.json), scaled to n atoms; None if the
    kernel's source changed since the capture."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "force_traffic.json")))
        src = os.path.join(ROOT, "paper_1305_4196_gb300", "csrc", "k_force.cu")
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["k_force_cu_sha256"]:
            return None
        r = rec["fused" if fused else "force"]
        return (r["dram_read_bytes"] + r["dram_write_bytes"]) * n / rec["atoms"]
    except Exception:
        return None


def algorithmic_force_bytes(n, entries, precision):
    """Algorithmic bytes of one full-list force evaluation, the per-unit figures of the method's
    cost model: per atom its coordinates with species (16 B FP32 / 28 B FP64), a 4 B list
    length and the 24 B force written; per list entry one 4 B neighbour index.  The kernels
    store lists as 2 B tile-local indices with a 2 B length, so the DRAM traffic they cause
    (roofline.traffic, from ncu) is below this figure."""
    per_atom = (16 if precision == "mixed" else 28) + 4 + 24
    return n * per_atom + 4 * entries


def algorithmic_half_bytes(n, entries, precision):
    """The same for a half-list (Newton-3) evaluation: each pair once, and per atom also the
    24 B of force read back when the reactions of a block's tile are added to it."""
    return algorithmic_force_bytes(n, entries, precision) + 24 * n


def algorithmic_fused_bytes(n, entries):
    """The same for the force kernel with the velocity-Verlet updates fused in: the force
    part without the force write (16 + 4 B per atom, 4 B per entry) plus the update's
    positions and velocities read and written (96 B) and its 24 B reference read."""
    return n * (16 + 4 + 96 + 24) + 4 * entries


def job_time_and_value(ms, atoms_per_rank, timesteps, world, device):
    """The slowest rank's time in ms (every rank must call this) and the whole-job
    throughput in atom-timesteps/s: each rank advances its own replica of the workload,
    so the job processed world * atoms * timesteps units in that time."""
    t_max = ms
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    return t_max, world * atoms_per_rank * timesteps / (t_max * 1e-3)


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1305_4196_gb300 import build as B
    B.build()
    from paper_1305_4196_gb300 import mdgb as M

    sysm = make_workload(args.workload)
    # CPU baseline first (rank 0, one GPU only): no GPU context is touched by the oracle
    cpu = cpu_baseline(sysm, args.cpu_steps) if (rank == 0 and world == 1 and args.cpu_steps > 0) else None

    stream = torch.cuda.Stream()
    prec = M.MD_MIXED if args.precision == "mixed" else M.MD_FP64
    lst = {"full": M.MD_LIST_FULL, "half": M.MD_LIST_HALF_COLOUR8, "half_af": M.MD_LIST_HALF_ATOMIC_FREE}[args.list]
    s = M.System(sysm.n, sysm.box, precision=prec, list_kind=lst, stream=stream.cuda_stream)
    s.set_state(sysm.pos, sysm.vel, sysm.species)

    def one_step():
        s.step(args.inner)
        s.energy_virial()

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    info0 = s.info()
    s.set_timing(True)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    info1 = s.info()
    s.set_timing(False)
    timesteps = args.steps * args.inner
    t_max, value = job_time_and_value(ms, sysm.n, timesteps, world, "cuda")
    launches = info1["kernel_launches"] - info0["kernel_launches"]

    # roofline of the dominant kernel (the force evaluation; on the full-list mixed path the
    # force kernel with velocity Verlet fused in), from events around each launch
    fused = args.precision == "mixed" and args.list == "full" and os.environ.get("MDGB_NO_FUSE", "0") in ("", "0")
    f_evals = max(info1["timed_force_evals"], 1)
    f_ms = info1["force_ms"] / f_evals
    peak, peak_kind = load_peaks()
    if fused:
        abytes = algorithmic_fused_bytes(sysm.n, info1["list_entries"])
        kname = "k_force_mixed_full<1, 0, FM_KKD> (forces + velocity Verlet)"
    elif args.list == "full":
        abytes = algorithmic_force_bytes(sysm.n, info1["list_entries"], args.precision)
        kname = "k_force_mixed_full" if args.precision == "mixed" else "k_force_fp64_full"
    else:
        abytes = algorithmic_half_bytes(sysm.n, info1["list_entries"], args.precision)
        kname = {"half": "k_force_mixed_half" if args.precision == "mixed" else "k_force_fp64_half",
                 "half_af": "k_force_half_af"}[args.list] + " (8 colour launches per evaluation)"
    achieved = abytes / (f_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": kname,
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": measured_force_traffic(sysm.n, fused) if args.precision == "mixed" and args.list == "full"
                else None,
                "traffic_note": "ncu dram read+write of a 1,048,576-atom launch scaled by atoms",
                "algorithmic_bytes": abytes, "avg_launch_ms": f_ms, "launches_timed": info1["timed_force_evals"],
                "launches": info1["force_evals"] - info0["force_evals"],
                "force_share_of_step": f_ms * (info1["force_evals"] - info0["force_evals"]) / ms}

    # the force kernel alone (md_forces: no integration), against the force-only cost model
    s.set_timing(True)
    i_f0 = s.info()
    for _ in range(5):
        M.md_forces(s.handle, None)
    torch.cuda.synchronize()
    i_f1 = s.info()
    s.set_timing(False)
    fo_ms = (i_f1["force_ms"] - i_f0["force_ms"]) / max(i_f1["timed_force_evals"] - i_f0["timed_force_evals"], 1)
    fo_bytes = (algorithmic_force_bytes if args.list == "full" else algorithmic_half_bytes)(
        sysm.n, i_f1["list_entries"], args.precision)
    roofline["force_kernel_alone"] = {"avg_launch_ms": fo_ms, "algorithmic_bytes": fo_bytes,
                                      "achieved": fo_bytes / (fo_ms * 1e-3) / 1e9,
                                      "frac": fo_bytes / (fo_ms * 1e-3) / 1e9 / peak,
                                      "traffic": measured_force_traffic(sysm.n, False)
                                      if args.precision == "mixed" and args.list == "full" else None}

    # neighbour-list build (binning + lists) on its own: builds inside graph-launched steps
    # are not bracketed by events, so time a few host-launched ones after the timed region
    s.set_timing(True)
    for _ in range(3):
        s.build_neighbors()
    torch.cuda.synchronize()
    binfo = s.info()
    s.set_timing(False)
    build_ms = binfo["build_ms"] / max(binfo["timed_builds"], 1)

    # end to end through the C ABI with pinned host buffers, copies inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        pos_h = torch.empty((sysm.n, 3), dtype=torch.float64, pin_memory=True).numpy()
        vel_h = torch.empty((sysm.n, 3), dtype=torch.float64, pin_memory=True).numpy()
        img_h = torch.empty((sysm.n, 3), dtype=torch.int32, pin_memory=True).numpy()
        sp_h = torch.empty((sysm.n,), dtype=torch.int32, pin_memory=True).numpy()
        s.get_state()  # warm path
        M.md_get_state(s.handle, pos_h, vel_h, img_h)
        sp_h[:] = sysm.species
        pos_h += img_h * sysm.box
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            M.md_set_state(s.handle, pos_h, vel_h, sp_h)
            s.step(args.inner)
            M.md_get_state(s.handle, pos_h, vel_h, img_h)
            s.energy_virial()
        torch.cuda.synchronize()
        _, e2e_value = job_time_and_value(1e3 * (time.perf_counter() - t0), sysm.n, args.inner * args.e2e_steps,
                                          world, "cuda")
        e2e = {"value": e2e_value, "unit": METRIC,
               "h2d_bytes_per_step": sysm.n * (24 + 24 + 4), "d2h_bytes_per_step": sysm.n * (24 + 24 + 12) + 64}

    extras = {}
    if not args.no_extras and rank == 0 and world == 1:
        extras = comparisons(args, sysm, M, stream, value, info1["list_entries"] / sysm.n,
                             hom={"force_ns_per_atom": f_ms * 1e6 / sysm.n, "build_ns_per_atom": build_ms * 1e6 / sysm.n,
                                  "rebuilds_per_timestep": (info1["n_builds"] - info0["n_builds"]) / timesteps})

    s.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64" if args.precision == "mixed" else "f64",
                "data": "synthetic (seeded fcc start, Gaussian velocities at T*=0.72)",
                "config": config_of(args, sysm, world), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk, "gpu_launches": launches,
                "rebuilds_per_timestep": (info1["n_builds"] - info0["n_builds"]) / timesteps,
                "ns_per_atom_timestep": t_max * 1e6 / (sysm.n * timesteps),
                "build_ms_avg": build_ms}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def comparisons(args, sysm, M, stream, value, list_len_hom, hom=None):
    """Same workload on the FP64 GPU path and on the 8-colour half-list path (short runs), and
    the per-atom cost of the strongly inhomogeneous workload next to this one."""
    import torch
    out = {}
    if args.workload.startswith("lj_liquid"):
        # the strongly inhomogeneous case as its own run: 500 time steps from the prepared
        # state, all timed (the cold slab and particles contract, so lists lengthen as it runs)
        inh = make_workload("slab_nanoparticles_1192114")
        s = M.System(inh.n, inh.box, precision=M.MD_MIXED if args.precision == "mixed" else M.MD_FP64,
                     list_kind={"full": M.MD_LIST_FULL, "half": M.MD_LIST_HALF_COLOUR8,
                                "half_af": M.MD_LIST_HALF_ATOMIC_FREE}[args.list],
                     stream=stream.cuda_stream)
        s.set_state(inh.pos, inh.vel, inh.species)
        s.forces()
        torch.cuda.synchronize()
        s.set_timing(True)  # as in the homogeneous run: events around one force launch per graph
        info0 = s.info()
        steps_inh = 500
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps_inh // 100):
            s.step(100)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        info1 = s.info()
        s.set_timing(False)
        ns_inh = ms * 1e6 / (inh.n * steps_inh)
        ns_hom = 1e9 / value
        f_ms_inh = (info1["force_ms"] - info0["force_ms"]) / max(info1["timed_force_evals"] - info0["timed_force_evals"], 1)
        s.set_timing(True)
        b0 = s.info()
        for _ in range(3):
            s.build_neighbors()
        torch.cuda.synchronize()
        b1 = s.info()
        s.set_timing(False)
        build_ms_inh = (b1["build_ms"] - b0["build_ms"]) / max(b1["timed_builds"] - b0["timed_builds"], 1)
        out["inhomogeneous"] = {"workload": "slab_nanoparticles_1192114", "atoms": inh.n,
                                "box_sigma": float(inh.box[0]), "timesteps": steps_inh,
                                "value": inh.n * steps_inh / (ms * 1e-3), "unit": METRIC,
                                "ns_per_atom_timestep": ns_inh,
                                "rebuilds_per_timestep": (info1["n_builds"] - info0["n_builds"]) / steps_inh,
                                "redos": info1["n_redos"] - info0["n_redos"],
                                "mean_list_length_end": info1["list_entries"] / inh.n,
                                "mean_list_length_homogeneous": list_len_hom,
                                "per_atom_cost_vs_homogeneous": ns_inh / ns_hom,
                                "force_ns_per_atom": f_ms_inh * 1e6 / inh.n,
                                "build_ns_per_atom": build_ms_inh * 1e6 / inh.n,
                                "homogeneous": hom}
        s.close()
    if args.workload.startswith("lj_liquid") and args.precision == "mixed" and args.list == "full":
        out["inhomogeneous_literal"] = literal_inhomogeneous_timing(M, stream, value)
    out["force_matching"] = force_matching_timing(M, stream)
    out["batch_ensemble"] = batch_ensemble_timing(stream)
    out["many_body"] = many_body_timing(M, stream)
    # the paper's dependent wave schedule on the two workloads' cell grids, beside the
    # 8 colour phases (host tool; no GPU work)
    from paper_1305_4196_gb300 import waves as WV
    out["wave_schedule"] = {f"{nc}^3 cells": {f"overlap_{ov}": WV.compare_with_colours(nc, ov) for ov in (27, 18)}
                            for nc in (44, 52)}
    runs = []
    if args.precision == "mixed":
        runs.append(("fp64_gpu", M.MD_FP64, M.MD_LIST_FULL, 100, 2))  # 200 timed steps, with rebuilds
    if args.list == "full":
        runs.append(("half_colour8_mixed", M.MD_MIXED, M.MD_LIST_HALF_COLOUR8, args.inner, 3))
        runs.append(("half_atomic_free_mixed", M.MD_MIXED, M.MD_LIST_HALF_ATOMIC_FREE, args.inner, 3))
    else:
        runs.append(("full_mixed", M.MD_MIXED, M.MD_LIST_FULL, args.inner, 3))
    for name, prec, lst, inner, steps in runs:
        s = M.System(sysm.n, sysm.box, precision=prec, list_kind=lst, stream=stream.cuda_stream)
        s.set_state(sysm.pos, sysm.vel, sysm.species)
        s.step(inner)
        torch.cuda.synchronize()
        s.set_timing(True)
        i0 = s.info()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            s.step(inner)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        info = s.info()
        v = sysm.n * inner * steps / (ms * 1e-3)
        out[name] = {"value": v, "unit": METRIC, "timesteps": inner * steps, "seconds": ms * 1e-3,
                     "rebuilds_per_timestep": (info["n_builds"] - i0["n_builds"]) / (inner * steps),
                     "force_ms_avg": info["force_ms"] / max(info["timed_force_evals"], 1)}
        s.close()
    if "fp64_gpu" in out:
        out["speedup_mixed_vs_fp64_gpu"] = value / out["fp64_gpu"]["value"]
    return {"compare": out}


def batch_ensemble_timing(stream, steps=200, autotune=True):
    """512 independent LJ systems, atom counts log-uniform in 256..32,768, densities
    U(0.7, 0.95), temperatures U(0.5, 1.5), 200 steps, mixed precision, in one persistent
    launch per call (shape autotuned first): small systems one CTA each for all steps,
    larger ones as block tasks shared by all CTAs.  Timed with CUDA events on the stream
    around md_batch_step (one graph launch)."""
    import tempfile
    import torch
    from paper_1305_4196_gb300 import batch as BA
    from paper_1305_4196_gb300 import workloads as W
    systems = W.batch_ensemble(512, seed=4)
    b = BA.from_systems(systems, stream=stream.cuda_stream)
    t_tune = 0.0
    if autotune:
        cache = os.path.join(tempfile.mkdtemp(), "batch_tune.json")
        t0 = time.perf_counter()
        b.autotune(cache)
        t_tune = time.perf_counter() - t0
    path, threads, R = b.layout()
    b.step(20)  # warm-up, including the graph capture of the launch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) * 1e-3
    ntot = sum(s.n for s in systems)
    res = {"systems": len(systems), "atoms_total": ntot, "timesteps": steps, "value": ntot * steps / dt,
           "unit": METRIC, "seconds": dt, "kernel_launches_per_call": 1,
           "one_cta_systems": int((path == 0).sum()), "block_task_systems": int((path == 1).sum()),
           "one_cta_atoms": int(sum(s.n for s, p in zip(systems, path) if p == 0)),
           "largest_one_cta_system": int(max([s.n for s, p in zip(systems, path) if p == 0], default=0)),
           "smallest_block_task_system": int(min([s.n for s, p in zip(systems, path) if p == 1], default=0)),
           "autotune_seconds": t_tune, "tuned_threads": int(threads[0]),
           "tuned_cell_range_by_size": sorted({int(r) for r in R[path == 0]})}
    b.close()
    return res


def many_body_timing(M, stream, steps=200):
    """The paper's bulk copper benchmark size, 1,000,188 atoms (63^3 fcc cells at 3.615 A),
    with the Cleri-Rosato tight-binding second-moment potential (cut between the fifth and
    sixth shells), room-temperature displacements and velocities (0.08 A, kT = 0.02585 eV),
    skin 0.4 A, 1 fs steps: velocity Verlet with the density and force passes launched from
    a CUDA graph per step.  Force time from the library's events (both passes)."""
    import torch
    from paper_1305_4196_gb300 import workloads as W
    P = W.copper_tbsma()
    mass, kT = P["mass"], 0.02585
    pos, box = W.fcc_lattice(63, 63, 63, 3.615)
    pos = W.gaussian_jitter(pos, box, 0.08, 11, stream=2)
    vel = W.thermal_velocities(np.full(len(pos), mass), kT, 11, stream=1)
    s = M.System(len(pos), box, r_cut=P["rc"], skin=0.4, mass=mass, dt=0.0982, precision=M.MD_MIXED,
                 stream=stream.cuda_stream)
    s.set_tbsma(P["A"], P["xi"], P["p"], P["q"], P["r0"], P["rc"])
    s.set_state(pos, vel, np.zeros(len(pos), dtype=np.int32))
    s.step(20)
    torch.cuda.synchronize()
    s.set_timing(True)
    i0 = s.info()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    i1 = s.info()
    s.set_timing(False)
    ms = e0.elapsed_time(e1)
    f_ms = (i1["force_ms"] - i0["force_ms"]) / max(i1["timed_force_evals"] - i0["timed_force_evals"], 1)
    res = {"workload": "fcc Cu 1,000,188 atoms, TB-SMA (Cleri-Rosato), 300 K", "atoms": len(pos),
           "timesteps": steps, "value": len(pos) * steps / (ms * 1e-3), "unit": METRIC,
           "ns_per_atom_timestep": ms * 1e6 / (len(pos) * steps), "force_ms_avg": f_ms,
           "rebuilds_per_timestep": (i1["n_builds"] - i0["n_builds"]) / steps,
           "mean_list_length": i1["list_entries"] / len(pos)}
    s.close()
    return res


def literal_inhomogeneous_timing(M, stream, value_hom, steps=500):
    """The strongly inhomogeneous structure in the literal 300 sigma cube: the fcc slab fills
    30 % of the height and 40 particles sit in the vacuum, 7,239,270 atoms, T* = 0.3, 500 steps
    from the prepared state (supplementary to the 1,192,114-atom row, whose smaller cube has
    more surface per atom)."""
    import torch
    w = make_workload("slab_nanoparticles_7239270")
    s = M.System(w.n, w.box, precision=M.MD_MIXED, stream=stream.cuda_stream)
    s.set_state(w.pos, w.vel, w.species)
    s.forces()
    torch.cuda.synchronize()
    i0 = s.info()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps // 100):
        s.step(100)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    i1 = s.info()
    s.close()
    ns = ms * 1e6 / (w.n * steps)
    return {"workload": "slab_nanoparticles_7239270", "atoms": w.n, "box_sigma": float(w.box[0]),
            "timesteps": steps, "value": w.n * steps / (ms * 1e-3), "unit": METRIC, "ns_per_atom_timestep": ns,
            "rebuilds_per_timestep": (i1["n_builds"] - i0["n_builds"]) / steps,
            "per_atom_cost_vs_homogeneous": ns / (1e9 / value_hom)}


def force_matching_timing(M, stream, n_snap=8):
    """Forward + backward (md_forces, md_forces_backward) of the force-matching loss on
    32,000-atom Kob-Andersen snapshots (fcc sites at rho* = 1.2, 80:20 species shuffle, 0.05
    sigma jitter per snapshot seed), at parameters perturbed by 10 %, FP64 and mixed."""
    import torch
    from paper_1305_4196_gb300 import workloads as W
    eps0 = np.array([[1.0, 1.5], [1.5, 0.5]])
    sig0 = np.array([[1.0, 0.8], [0.8, 0.88]])
    eps1 = eps0 * np.array([[1.1, 0.9], [0.9, 1.1]])
    sig1 = sig0 * np.array([[0.9, 1.1], [1.1, 0.9]])
    snaps = []
    for k in range(n_snap):
        w = W.lj_fcc(20, rho=1.2, seed=100 + k, jitter=0.05)
        snaps.append((torch.as_tensor(w.pos, device="cuda"),
                      torch.as_tensor(W.species_shuffle(w.n, 0.2, 100 + k), dtype=torch.int32, device="cuda")))
    box = w.box
    res = {"workload": "Kob-Andersen 80:20, 32,000 atoms per snapshot", "snapshots": n_snap}
    for name, prec in [("fp64", M.MD_FP64), ("mixed", M.MD_MIXED)]:
        s = M.System(w.n, box, r_cut=2.5 * 1.1, skin=0.3, eps=eps0, sigma=sig0, mass=[1.0, 1.0], precision=prec,
                     rcut=2.5 * sig0 * 1.1, stream=stream.cuda_stream)
        zeros = torch.zeros_like(snaps[0][0])
        F = torch.empty_like(zeros)
        T = torch.empty_like(zeros)
        gpos = torch.empty_like(zeros)

        def one(pos, sp):
            # torch work below runs on the library's stream, so it is ordered with its kernels
            s.set_params(eps0, sig0, 2.5 * sig0)
            s.set_state(pos, zeros, sp)
            s.forces(out=T)
            s.set_params(eps1, sig1, 2.5 * sig1)
            s.forces(out=F)
            G = (2.0 / F.numel()) * (F - T)
            return s.forces_backward(G, gpos)

        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            one(*snaps[0])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for pos, sp in snaps:
                one(pos, sp)
            torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[name] = {"ms_per_snapshot": 1e3 * dt / n_snap,
                     "note": "target forces, perturbed forces and the backward pass per snapshot"}
        s.close()
    return res


def main():
    args = parse()
    if args.many_body:
        import torch
        from paper_1305_4196_gb300 import build as B
        B.build()
        from paper_1305_4196_gb300 import mdgb as M
        stream = torch.cuda.Stream()
        print(json.dumps({"many_body": many_body_timing(M, stream, steps=args.inner)}))
    elif args.only:
        import torch
        from paper_1305_4196_gb300 import build as B
        B.build()
        from paper_1305_4196_gb300 import mdgb as M
        stream = torch.cuda.Stream()
        if args.only == "ensemble":
            res = {"batch_ensemble": batch_ensemble_timing(stream, steps=args.ensemble_steps,
                                                           autotune=not args.no_autotune)}
        else:
            res = {"force_matching": force_matching_timing(M, stream)}
        print(json.dumps(res))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
