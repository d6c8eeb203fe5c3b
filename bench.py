"""Benchmark of the fused SNAP finite-volume step on GB300.

Workload: the 2-D dry density current (25.6 km x 6.4 km, 1024 x 256 cells, theta = 300 K,
-15 K cosine bubble, nu = 75 m^2/s, reflecting walls), seeded and synthetic. A step is one
SSP-RK3 step (three fused stages). Metric: cell-updates per second per RK stage,
cells x 3 x steps / time, FP32 (the headline) with the FP64 step measured beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One JSON line on rank 0. Under torchrun (N > 1) each rank advances an independent replica
(weak scaling, no collective on the data path); time is the max over ranks.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK stage (WENO5+LMARS), FP32 vs FP64, % of HBM roofline"
UNIT = "cell-updates/s"
WORKLOAD = "density_current_1024x256"
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extra", action="store_true",
                   help="leave out the Jovian and ensemble sub-lines of the default line (for "
                        "profiling runs of the headline kernel)")
    p.add_argument("--workload", default=WORKLOAD,
                   choices=[WORKLOAD, "jovian_256x256x128", "jovian_256x256x128_kessler",
                            "jovian_rce_256x256x128",
                            "ensemble_96", "ensemble_96_autotuned", "adjoint_256x256",
                            "bryan_1000s", "density_current_900s", "density_current_slabs"],
                   help="the default is the headline workload; the others print an extra "
                        "measurement line of the same form (3-D moist column, the same with "
                        "Kessler microphysics and falling precipitation, moist ensemble) or "
                        "the adjoint's cost")
    p.add_argument("--adjoint-steps", type=int, default=400,
                   help="steps of the forward and adjoint runs of the adjoint workload")
    return p.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(dtype, name=WORKLOAD):
    import workloads as W
    if name == "jovian_256x256x128":
        return [W.jovian(dtype=dtype)]
    if name == "jovian_256x256x128_kessler":
        # the Kessler constants and precipitation speed of the paper's Jovian simulation
        import dataclasses
        return [dataclasses.replace(W.jovian(dtype=dtype), kessler_k=(1e9, 1e-4, 0.0, 1e-2),
                                    w_term=(0.0, -20.0))]
    if name == "jovian_rce_256x256x128":
        # the radiative-convective setup of Sec. 6: microphysics, falling precipitation,
        # cooling, sponge, and the no-slip floor at a fixed temperature
        return [W.jovian_rce(dtype=dtype)]
    if name.startswith("ensemble_96"):
        return W.ensemble()
    return W.density_current(dtype=dtype)


# Nominal arithmetic peaks from the part's unit counts and its maximum SM clock (152 SMs at
# 2070 MHz): 128 FP32 lanes per SM, one fused multiply-add (2 flop) per lane per clock; the
# FP64 rate is the part's nominal 1.25 TFLOP/s.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def alg_flops_per_cell_stage(D, nmom, nv, visc=False, shared_indicators=False):
    """Floating-point operations one cell-stage of the scheme needs by its definition (an
    addition, multiplication, division, square root or power counts 1; nothing for halo
    recomputation, index arithmetic or the saturation adjustment):
      WENO5, one side of one face for one variable (Sec. 4.2): 3 smoothness indicators 33,
        3 candidates 15, 3 weights 9, normalised combination 8 -> 65; two sides of D faces
        per cell for every one of the nv primitives. With shared_indicators the indicators
        and the squares (eps + beta_k)^2 of a cell's five-point window are counted once for
        the two face states that window gives (the right state of the face below the cell
        and the left state of the face above read the same three sub-stencils): 33 + 6 per
        window plus 3 divisions, 15 candidate and 8 combination operations per state -> 91
        per cell and direction instead of 130;
      LMARS per face (Sec. 4.1): total pressures 2, sound speeds 6, rho c 4, u* 6, p* 6,
        mass flux 1, momentum fluxes nmom + 1, energy flux 2 nmom + 5, and 10 per tracer for
        the tracer fluxes and the mixture gamma;
      primitives per cell (App. B): 3 nmom + 3, plus 8 per tracer for the mixture sums;
      divergence 3 D nv; gravity 7; SSP-RK3 combine 4 nv (stage average);
      viscous fluxes (when present) 6 nmom + 12 per face and 5 per cell."""
    ntr = nv - 2 - nmom  # tracer densities besides rho_d
    weno = D * nv * (91 if shared_indicators else 2 * 65)
    lmars = D * (31 + 3 * nmom + 10 * ntr)
    prim = 3 * nmom + 3 + 8 * ntr
    rest = 3 * D * nv + 7 + 4 * nv
    vis = D * (6 * nmom + 12) + 5 if visc else 0
    return weno + lmars + prim + rest + vis


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_sources_md5(kern="kern_dry2d.cu"):
    """Hash of the sources that define a stage kernel (its template, the structures it reads
    and the file that instantiates it with its tiles); a change in any invalidates the
    committed ncu traffic figure."""
    h = hashlib.md5()
    csrc = os.path.join(ROOT, "paper_1901_02955_gb300", "csrc")
    for f in ("snap_stage.cuh", "snap_internal.h", kern):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()


def ncu_record(name="density_current", kern="kern_dry2d.cu"):
    """The committed ncu record of a stage kernel (DRAM bytes and warp instructions per
    launch), if it was taken on the current kernel sources (else an empty dict)."""
    path = os.path.join(ROOT, "profiles", f"stage_kernel_{name}_traffic.json")
    if not os.path.exists(path):
        return {}
    try:
        d = json.load(open(path))
        if d.get("sources_md5") == kernel_sources_md5(kern):
            return d
    except Exception:
        pass
    return {}


def ncu_traffic():
    """DRAM bytes per launch of the stage kernel (None without a current ncu record)."""
    d = ncu_record()
    return float(d["dram_bytes_per_launch"]) if "dram_bytes_per_launch" in d else None


# Instruction issue limit of the part: 152 SMs x 4 schedulers, one warp instruction each per
# clock at 2070 MHz
ISSUE_PEAK_WARP_INST = 152 * 4 * 2.070e9


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.path = None
        self.index = index

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.path:
            return None
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i] == "Active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_replica(q, barrier, warmup, steps, seconds):
    """One host core: the oracle as it stands stepping its own copy of the workload. Either
    `steps` timed steps, or (steps == 0) as many as fit in `seconds` after one probe step.
    All replicas start their timed loop together (barrier)."""
    import oracle
    w = workload("f64")
    o = oracle.Oracle(w)
    dt = o.dt_cfl(w.Y)
    Y = w.Y
    t0 = time.perf_counter()
    for _ in range(max(1, warmup)):
        Y, _, _ = o.step(Y, 1, dt=dt)
    per = (time.perf_counter() - t0) / max(1, warmup)
    n = steps if steps > 0 else max(1, int(seconds / max(per, 1e-6)))
    barrier.wait()
    t0 = time.perf_counter()
    o.step(Y, n, dt=dt)
    q.put((n, time.perf_counter() - t0))


def oracle_on_host_cores(warmup, steps, seconds=0.0, cores=None):
    """The FP64 oracle, unchanged, on every host core at once: one process per core, each
    stepping its own replica of the full workload (independent problems, like replicas on
    GPUs). Returns (cell-updates/s over all replicas, replicas, steps each, wall seconds of
    the slowest replica). Processes are spawned, never forked (this process may hold a CUDA
    context)."""
    import multiprocessing as mp
    import oracle
    oracle.build()  # compile once before the replicas load it
    n = cores or host_cores()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    barrier = ctx.Barrier(n)
    procs = [ctx.Process(target=_oracle_replica, args=(q, barrier, warmup, steps, seconds))
             for _ in range(n)]
    for p in procs:
        p.start()
    res = [q.get() for _ in procs]
    for p in procs:
        p.join()
    cells = workload("f64").ncells
    wall = max(t for _, t in res)
    work = sum(k for k, _ in res) * cells * 3
    return work / wall, n, min(k for k, _ in res), wall


def cpu_baseline(seconds):
    """The FP64 oracle as it stands on the host: whole steps of the full workload, one
    replica per host core."""
    v, n, k, wall = oracle_on_host_cores(1, 0, seconds)
    return {"value": v, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} processes, one per host core, each {k}+ full SSP-RK3 steps of its "
                      f"own copy of {WORKLOAD} in FP64 ({wall:.1f} s wall)"}


def reference_arm(args, rank):
    if rank != 0:
        return
    v, n, k, wall = oracle_on_host_cores(args.warmup, args.steps)
    w = workload("f64")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": w.ncells, "nfields": w.nv,
                       "parallelism": f"{n} host cores, one replica of the workload each"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": n, "kind": "oracle",
                             "sample": f"{n} replicas x {args.steps} full steps of {WORKLOAD}, "
                                       f"FP64, one process per host core"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def extra_workload(args, local, rank=0, world=1):
    """Measurement line for the 3-D moist column or the moist ensemble (inputs larger than
    L2, so no flush is needed between steps). Under torchrun the ensemble's domains are
    split across the ranks (no exchange between them; strong scaling of the fixed ensemble)
    and the step time is the slowest rank's; other workloads run on rank 0."""
    import torch
    from paper_1901_02955_gb300 import Context
    from paper_1901_02955_gb300.ranks import max_over_ranks, shard_domains
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ws_all = workload("f32", args.workload)
    cells_all = sum(w.ncells for w in ws_all)
    ws = [ws_all[d] for d in shard_domains([w.ncells for w in ws_all], world)[rank]]
    ctx = Context(ws, dtype="f32")
    ctx.set_stream(stream)
    for d, w in enumerate(ws):
        ctx.set_state(w.Y.astype(np.float32), domain=d)
    tuned = None
    if args.workload.endswith("_autotuned"):
        tuned = ctx.autotune(steps=3)
    cells = sum(w.ncells for w in ws)
    nv = ws[0].nv
    for _ in range(args.warmup):
        ctx.step_async(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with Clocks(local) as clk:
        for s_, e_ in ev:
            s_.record(stream)
            ctx.step_async(1)
            e_.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    rc, flags = ctx.check()
    ms = max_over_ranks(float(np.mean([s_.elapsed_time(e_) for s_, e_ in ev])), dist,
                        torch.device("cuda", local))
    peak, src = measured_peaks()
    three_d = ws[0].ny > 1
    roof = stage_rooflines(ms, cells, nv, 3 if three_d else 2, peak, src)
    stage_ms = roof["stage_ms"]
    flops_cell = roof["alu"]["algorithmic_flops_per_cell_stage"]
    tflops = roof["alu"]["achieved"]
    ach = roof["hbm"]["achieved"]
    alg = (8.0 / 3.0) * nv * 4 * cells
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {"metric": METRIC, "value": cells_all * 3 / (ms * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True,
            "scaling": "strong" if args.workload.startswith("ensemble_96") else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "cells": cells_all, "nfields": nv,
                       "domains": len(ws_all), "domains_rank0": len(ws),
                       "cells_rank0": cells, "l2": "inputs larger than L2",
                       "parallelism": f"ensemble domains split over {world} ranks"
                       if world > 1 else "single GPU",
                       "device_checks": {"rc": rc, "flags": flags},
                       "info": ctx.info(), "autotune": tuned},
            "roofline": {"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": tflops / FP32_PEAK_TFLOPS,
                         "traffic": None,
                         "peak_source": "nominal FP32 FMA rate from unit counts and the "
                                        "2070 MHz clock",
                         "stage_ms": stage_ms,
                         "stage_ms_source": "timed step / 3 launches",
                         "algorithmic_flops_per_cell_stage": flops_cell,
                         "frac_shared_indicators": roof["alu"]["frac_shared_indicators"],
                         "note": "saturation adjustment not counted in the flops",
                         "hbm": {"achieved": ach, "peak": peak, "unit": "GB/s",
                                 "frac": ach / peak, "peak_source": src,
                                 "algorithmic_bytes_per_launch": alg}},
            "gpu_launches": 3 * args.steps, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def bryan_workload(args, local):
    """The Bryan moist bubble (Sec. 5) run to 1000 s at 100 m on the GPU, FP64 and FP32, with
    the CFL time step: the largest equivalent-potential-temperature anomaly (against the
    initial state's edge column, the unperturbed background) and the throughput. The paper
    reports 4.4 K at 1000 s (Bryan & Fritsch's reference solution: 4.09 K)."""
    import torch
    import workloads as W
    from paper_1901_02955_gb300 import Context
    torch.cuda.set_device(local)
    w = W.bryan_moist_bubble()
    out = {}
    for dt_name in ("f64", "f32"):
        ctx = Context(w, dtype=dt_name)
        ctx.set_state(w.Y)
        bg = ctx.theta_e()[:, :, :1]
        t, n = 0.0, 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while t < 1000.0 - 1e-9:
            dt = min(ctx.compute_dt(), 1000.0 - t)
            ctx.step(1, dt_fixed=dt)
            t += dt
            n += 1
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        te = ctx.theta_e()
        Y = ctx.get_state()
        out[dt_name] = {"max_theta_e_anomaly_K": float((te - bg).max()),
                        "min_theta_e_anomaly_K": float((te - bg).min()),
                        "max_w_m_s": float((Y[5] / Y[:4].sum(axis=0)).max()),
                        "steps": n, "wall_s": wall,
                        "cell_updates_per_s": w.ncells * 3 * n / wall}
        ctx.close()
    line = {"metric": "max equivalent potential temperature anomaly at 1000 s", "unit": "K",
            "value": out["f64"]["max_theta_e_anomaly_K"], "higher_is_better": None,
            "n_gpus": 1, "vs_baseline": None, "data": "synthetic",
            "config": {"workload": "bryan_moist_bubble_200x100", "t_end_s": 1000.0,
                       "paper_value_K": 4.4, "note": "wall clock includes one host "
                       "round trip per step for the CFL time step", "results": out}}
    print(json.dumps(line), flush=True)


def straka_workload(args, local):
    """The density current (Sec. 5.1, after Straka et al.) run to 900 s at 25 m on the GPU,
    FP64 and FP32, viscous (75 m^2/s) and inviscid, with the CFL time step: the extrema of the
    potential-temperature anomaly against the 300 K background and the position of the front
    (the farthest surface cell colder than -1 K). The paper reports a largest anomaly at 900 s
    of 0.12 K viscous and about 0.3 K inviscid with LMARS (1.84 K and over 12 K with HLLC);
    the minimum starts at -15 K and mixing raises it."""
    import torch
    import workloads as W
    from paper_1901_02955_gb300 import Context
    torch.cuda.set_device(local)
    kappa = (1.4 - 1.0) / 1.4
    out = {}
    runs = (("f64", 75.0), ("f32", 75.0), ("f64_inviscid", 0.0), ("f32_inviscid", 0.0))
    for name, nu in runs:
        w = W.density_current(dtype="f64", nu=nu)
        dt_name = name[:3]
        ctx = Context(w, dtype=dt_name)
        ctx.set_state(w.Y)
        t, n = 0.0, 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while t < 900.0 - 1e-9:
            dt = min(ctx.compute_dt(), 900.0 - t)
            ctx.step(1, dt_fixed=dt)
            t += dt
            n += 1
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        Y = ctx.get_state()
        rho = Y[0]
        p = (w.gamma_d - 1.0) * (Y[3] - 0.5 * (Y[1] ** 2 + Y[2] ** 2) / rho)
        theta = p / (rho * w.R_d) * (1e5 / p) ** kappa
        dth = theta - 300.0
        cold = np.nonzero(dth[0, 0] < -1.0)[0]
        out[name] = {"max_theta_anomaly_K": float(dth.max()),
                        "min_theta_anomaly_K": float(dth.min()),
                        "front_x_m": float((cold.max() + 0.5) * w.dx) if cold.size else 0.0,
                        "steps": n, "wall_s": wall,
                        "cell_updates_per_s": w.ncells * 3 * n / wall}
        ctx.close()
    line = {"metric": "potential temperature anomaly extrema at 900 s", "unit": "K",
            "value": out["f64"]["max_theta_anomaly_K"], "higher_is_better": None,
            "n_gpus": 1, "vs_baseline": None, "data": "synthetic",
            "config": {"workload": "density_current_1024x256", "t_end_s": 900.0,
                       "paper_max_anomaly_K": 0.12, "paper_max_anomaly_inviscid_K": 0.3,
                       "viscosity_m2_s": 75.0,
                       "note": "wall clock includes one host round trip per step for the CFL "
                               "time step", "results": out}}
    print(json.dumps(line), flush=True)


def adjoint_workload(args, local):
    """Forward and discrete-adjoint cost of the 2-D warm bubble at 256 x 256 and of its moist
    variant (cloud forming in the core), 400 steps with a checkpoint every 20 steps or with
    every stage input kept, FP64 and FP32 (fixed time step from the initial CFL)."""
    import torch
    import workloads as W
    from paper_1901_02955_gb300 import Context
    torch.cuda.set_device(local)
    nsteps, every = args.adjoint_steps, 20
    out = {}
    for kind, dt_name in (("dry", "f64"), ("dry", "f32"), ("moist", "f64"), ("moist", "f32")):
        w = W.adjoint_bubble(n=256) if kind == "dry" else W.moist_adjoint_bubble(n=256)
        ctx = Context(w, dtype=dt_name)
        ctx.set_state(w.Y)
        dt = ctx.compute_dt()
        ctx.step(5, dt_fixed=dt)  # warm-up
        ctx.set_state(w.Y)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.step(nsteps, dt_fixed=dt)
        t_fwd = time.perf_counter() - t0
        res = {"forward_ms_per_step": 1e3 * t_fwd / nsteps}
        lam = np.random.default_rng(1).normal(size=w.Y.shape).astype(
            np.float32 if dt_name == "f32" else np.float64)
        lam_d = torch.from_numpy(lam).cuda()
        # every: checkpoints and recomputation; 0: every stage input kept by the record
        for mode, k in (("checkpointed", every), ("stored", 0)):
            ctx.set_state(w.Y)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.record(nsteps, k, dt)
            t_rec = time.perf_counter() - t0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.step_adjoint(nsteps, lam_d)
            torch.cuda.synchronize()
            t_adj = time.perf_counter() - t0
            res[mode] = {"checkpoint_every": k,
                         "record_ms_per_step": 1e3 * t_rec / nsteps,
                         "adjoint_ms_per_step": 1e3 * t_adj / nsteps,
                         "adjoint_over_forward": t_adj / t_fwd}
        out[f"{kind}_{dt_name}"] = res
        ctx.close()
    line = {"metric": "discrete adjoint cost relative to the forward run", "unit": "ratio",
            "value": out["dry_f32"]["checkpointed"]["adjoint_over_forward"],
            "higher_is_better": False,
            "config": {"workload": "adjoint_bubble_256x256", "steps": nsteps,
                       "checkpoint_every": every, "cells": w.ncells,
                       "note": "wall clock incl. host orchestration; value: dry FP32 with "
                               "checkpoints, the adjoint including the segment "
                               "recomputation; 'stored' keeps every stage input instead; "
                               "moist: the moist adjoint bubble (cloud in the core, "
                               "saturation adjustment after every stage)",
                       "results": out}}
    print(json.dumps(line), flush=True)


def slabs_workload(args, local):
    """The density current split along x into 1, 2 and 4 slabs, all domains of one context
    with their boundaries linked (the kernels read a neighbour's columns in place; one CFL
    time step for the group): the cost of the decomposition against the undecomposed grid,
    FP32, L2 flushed before every timed step, and the states after the timed steps compared
    bitwise with the undecomposed run."""
    import torch
    from paper_1901_02955_gb300 import Context
    from paper_1901_02955_gb300.slabs import Decomposition, gather, link_slabs, slab_workload
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    w = workload("f32")
    out, ref = {}, None
    for nslab in (1, 2, 4):
        if nslab == 1:
            ws = [w]
            ctx = Context(ws, dtype="f32")
        else:
            dec = Decomposition(w.nx, nslab, periodic=False)
            ws = [slab_workload(w, dec, s_) for s_ in range(nslab)]
            ctx = Context(ws, dtype="f32")
            ctx.set_tile_variant(0)
            link_slabs(ctx, dec)
        ctx.set_stream(stream)
        for d, ws_ in enumerate(ws):
            ctx.set_state(ws_.Y.astype(np.float32), domain=d)
        for _ in range(args.warmup):
            flush.fill_(1)
            ctx.step_async(1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        torch.cuda.synchronize()
        for s_, e_ in ev:
            flush.fill_(1)
            s_.record(stream)
            ctx.step_async(1)
            e_.record(stream)
        torch.cuda.synchronize()
        rc, flags = ctx.check()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        Y = ctx.get_state() if nslab == 1 else \
            gather(dec, {d: ctx.get_state(domain=d) for d in range(nslab)})
        if ref is None:
            ref = Y
        info = ctx.info()
        out[f"slabs_{nslab}"] = {"ms_per_step": ms, "cell_updates_per_s": w.ncells * 3 / (ms * 1e-3),
                                 "tiles": info["tiles_total"], "device_checks": flags,
                                 "bitwise_equal_to_undecomposed": bool(np.array_equal(Y, ref))}
        ctx.close()
    line = {"metric": "slab decomposition of one domain: step time against the undecomposed grid",
            "unit": "ms", "value": out["slabs_2"]["ms_per_step"], "higher_is_better": False,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
            "config": {"workload": WORKLOAD, "dtype": "f32", "l2": "flushed before every step",
                       "note": "slabs linked in one context; the warm-up and timed steps of "
                               "every run start from the same state", "results": out}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    if args.workload == "adjoint_256x256":
        if rank == 0:
            adjoint_workload(args, local)
        return
    if args.workload == "bryan_1000s":
        if rank == 0:
            bryan_workload(args, local)
        return
    if args.workload == "density_current_900s":
        if rank == 0:
            straka_workload(args, local)
        return
    if args.workload == "density_current_slabs":
        if rank == 0:
            slabs_workload(args, local)
        return
    if args.workload != WORKLOAD:
        if args.workload.startswith("ensemble_96"):
            extra_workload(args, local, rank, world)
        elif rank == 0:
            extra_workload(args, local)
        return
    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        sys.exit(1)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1901_02955_gb300 import Context

    stream = torch.cuda.Stream()  # the library and the events share this stream
    torch.cuda.set_stream(stream)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if not dist:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def device_steps(ctx, steps, warmup):
        """Per-step device time (ms) with the L2 flushed before each step."""
        for _ in range(warmup):
            flush.fill_(1)
            ctx.step_async(1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        barrier()
        for s, e in ev:
            flush.fill_(1)
            s.record(stream)
            ctx.step_async(1)
            e.record(stream)
        barrier()
        rc, flags = ctx.check()
        assert rc == 0, f"device check failed: flags {flags}"
        return [s.elapsed_time(e) for s, e in ev]

    # ---- FP32 fused step (headline) --------------------------------------------------------
    w32 = workload("f32")
    ctx = Context(w32, dtype="f32")
    ctx.set_stream(stream)
    ctx.set_state(w32.Y)
    with Clocks(local) as clk:
        times = device_steps(ctx, args.steps, args.warmup)
    ms32 = max_over_ranks(float(np.sum(times)) / args.steps)
    cells = w32.ncells
    value = world * cells * 3 / (ms32 * 1e-3)
    launches = 3 * args.steps

    # ---- dominant kernel: the stage kernel ---------------------------------------------------
    # Its average launch duration inside the timed step is at most the step time over its three
    # launches (the graph's gaps between them included), which the roofline uses. Launches
    # timed one by one with events around each (a flush before every step) are reported
    # beside it; they carry the launch overhead the graph replay does not pay.
    ctx.set_state(w32.Y)
    dt = ctx.compute_dt()
    nst = max(10, args.steps // 2)
    evs = []
    for i in range(nst + 3):
        flush.fill_(1)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        for st in range(3):
            ctx.stage(st, dt)
            e[st + 1].record(stream)
        if i >= 3:
            evs.append(e)
    torch.cuda.synchronize()
    per_stage = [[e[s].elapsed_time(e[s + 1]) for s in range(3)] for e in evs]
    stage_ms = ms32 / 3.0
    word = 4
    alg_bytes = (8.0 / 3.0) * w32.nv * word * cells  # per launch, averaged over the 3 stages
    peak, peak_src = measured_peaks()
    achieved = alg_bytes / (stage_ms * 1e-3) / 1e9
    traffic = ncu_traffic()
    flops_cell = alg_flops_per_cell_stage(2, 2, w32.nv, visc=w32.nu > 0)
    flops_cell_sh = alg_flops_per_cell_stage(2, 2, w32.nv, visc=w32.nu > 0,
                                             shared_indicators=True)
    alg_flops = flops_cell * cells
    tflops = alg_flops / (stage_ms * 1e-3) / 1e12
    tflops_sh = flops_cell_sh * cells / (stage_ms * 1e-3) / 1e12
    # the stage kernel is bound by arithmetic issue, not by HBM (DRAM a few % busy in ncu):
    # the roofline is the FP32 one; the HBM fraction the metric names is reported beside it
    roofline = {"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": tflops / FP32_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "nominal FP32 FMA rate from unit counts and the 2070 MHz clock",
                "kernel": "snap::stage_kernel<float, dry x-z, viscous>",
                "stage_ms": stage_ms,
                "stage_ms_source": "timed step / 3 launches (graph replay, L2 flushed before "
                                   "each step)",
                "stage_ms_isolated": [float(np.mean([p[s] for p in per_stage]))
                                      for s in range(3)],
                "algorithmic_flops_per_launch": alg_flops,
                "algorithmic_flops_per_cell_stage": flops_cell,
                "shared_indicators": {
                    "algorithmic_flops_per_cell_stage": flops_cell_sh,
                    "achieved": tflops_sh, "frac": tflops_sh / FP32_PEAK_TFLOPS,
                    "note": "the same count with each window's smoothness indicators charged "
                            "once for the two face states that share them"},
                "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "peak_source": f"{peak_src} HBM copy bandwidth",
                        "algorithmic_bytes_per_launch": alg_bytes,
                        "note": "the 4 MB state stays in L2 between the stages of a step"}}
    # the device's achieved fused multiply-add rate (snap_probe_fma), beside the nominal peak
    from paper_1901_02955_gb300 import capi as _capi
    probe32 = _capi.probe_fma("f32", stream.cuda_stream)
    roofline["peak_probe"] = {"value": probe32, "unit": "TFLOP/s",
                              "frac_of_probe": tflops / probe32,
                              "note": "FP32 fused multiply-add chains on every SM, measured "
                                      "before the timed region"}
    inst = ncu_record().get("warp_instructions_per_launch")
    if inst:
        # issued warp instructions per launch (ncu, same sources) over the in-step stage time
        rate = float(inst) / (stage_ms * 1e-3)
        roofline["issue"] = {"achieved": rate, "peak": ISSUE_PEAK_WARP_INST,
                             "unit": "warp instructions/s", "frac": rate / ISSUE_PEAK_WARP_INST,
                             "warp_instructions_per_launch": float(inst),
                             "peak_source": "4 schedulers x 152 SMs x 2070 MHz"}

    # ---- end to end through the C ABI with pinned host buffers --------------------------------
    host_in = torch.from_numpy(w32.Y.astype(np.float32)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    for _ in range(max(2, args.warmup)):
        ctx.step_io(host_in, host_out, nsteps=1)
    barrier()
    step_s = []
    for _ in range(args.steps):
        # L2 flushed between timed steps, outside the timed region
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # one call: the state read from pinned host memory, one step, the result written to
        # pinned host memory; returns when it is there
        ctx.step_io(host_in, host_out, nsteps=1)
        step_s.append(time.perf_counter() - t0)
    barrier()
    e2e_s = max_over_ranks(float(np.mean(step_s)))
    nbytes = host_in.numel() * 4
    e2e = {"value": world * cells * 3 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes,
           "note": "host wall clock per step of snap_step_io: the state read from pinned host "
                   "memory (with its CFL rate), one step, the result written to pinned host "
                   "memory; L2 flushed before each step outside the timed region"}
    ctx.close()

    # ---- FP64 fused step beside it ---------------------------------------------------------
    w64 = workload("f64")
    c64 = Context(w64, dtype="f64")
    c64.set_stream(stream)
    c64.set_state(w64.Y)
    k64 = max(5, args.steps // 4)
    t64 = device_steps(c64, k64, 2)
    ms64 = max_over_ranks(float(np.sum(t64)) / k64)
    v64 = world * cells * 3 / (ms64 * 1e-3)
    c64.close()
    fp64_tflops = flops_cell * cells * 3 / (ms64 * 1e-3) / 1e12

    # ---- the workloads larger than L2, timed in the same run ----------------------------------
    jov = None if args.no_extra else jovian_line(args, stream, peak, peak_src)
    ens = None if args.no_extra else ensemble_line(args, stream, peak, peak_src)

    # ---- one step of the bench input on the GPU, kept for the parity report -----------------
    gpu_steps = parity_gpu_steps(stream)
    jov_windows = None if args.no_extra else jovian_window_steps(stream)

    if rank == 0:
        cpu = None
        parity = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(args.cpu_seconds)
            parity = parity_report(gpu_steps)
            if jov_windows is not None:
                parity["jovian_256x256x128_stage0_windows"] = jovian_window_report(jov_windows)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms32,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": cells, "nfields": w32.nv,
                       "grid": [w32.nx, w32.nz], "viscosity": w32.nu,
                       "l2": "flushed (512 MB write) before every timed step",
                       "fp64_value": v64, "fp64_ms_per_step": ms64, "fp32_over_fp64": value / v64,
                       "fp64_alu": {"achieved": fp64_tflops, "peak": FP64_PEAK_TFLOPS,
                                    "unit": "TFLOP/s", "frac": fp64_tflops / FP64_PEAK_TFLOPS,
                                    "peak_probe": _capi.probe_fma("f64", stream.cuda_stream),
                                    "note": "whole step time, nominal FP64 rate; peak_probe: "
                                            "the device's measured FP64 fused multiply-add rate"},
                       "jovian_256x256x128": jov, "ensemble_96": ens,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "parity": parity, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def timed_steps(ctx, stream, steps, warmup):
    """Mean device time per step (ms) of `steps` graph-replayed steps after `warmup`, CUDA
    events on the launching stream; the inputs are larger than L2, so no flush."""
    import torch
    for _ in range(warmup):
        ctx.step_async(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    for s_, e_ in ev:
        s_.record(stream)
        ctx.step_async(1)
        e_.record(stream)
    torch.cuda.synchronize()
    rc, flags = ctx.check()
    assert rc == 0, f"device check failed: flags {flags}"
    return float(np.mean([s_.elapsed_time(e_) for s_, e_ in ev]))


def stage_rooflines(ms_step, cells, nv, D, peak, peak_src, record=None):
    """ALU and HBM fractions of the stage kernel from the in-step time (step / 3); with a
    current ncu record, its DRAM bytes per launch (traffic) and the warp-instruction issue
    fraction."""
    stage_s = ms_step / 3.0 * 1e-3
    flops = alg_flops_per_cell_stage(D, D, nv)
    flops_sh = alg_flops_per_cell_stage(D, D, nv, shared_indicators=True)
    gbs = (8.0 / 3.0) * nv * 4 * cells / stage_s / 1e9
    out = {"stage_ms": ms_step / 3.0,
           "alu": {"achieved": flops * cells / stage_s / 1e12, "peak": FP32_PEAK_TFLOPS,
                   "unit": "TFLOP/s", "frac": flops * cells / stage_s / 1e12 / FP32_PEAK_TFLOPS,
                   "algorithmic_flops_per_cell_stage": flops,
                   "frac_shared_indicators": flops_sh * cells / stage_s / 1e12 /
                   FP32_PEAK_TFLOPS},
           "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                   "peak_source": f"{peak_src} HBM copy bandwidth",
                   "algorithmic_bytes_per_cell_stage": (8.0 / 3.0) * nv * 4,
                   "traffic": None}}
    if record:
        out["hbm"]["traffic"] = float(record["dram_bytes_per_launch"])
        out["hbm"]["traffic_note"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                      "stage-0 launch (its input is read once: Y_s is Y^n)")
        rate = float(record["warp_instructions_per_launch"]) / stage_s
        out["issue"] = {"achieved": rate, "peak": ISSUE_PEAK_WARP_INST,
                        "unit": "warp instructions/s", "frac": rate / ISSUE_PEAK_WARP_INST}
    return out


def jovian_line(args, stream, peak, peak_src):
    """The 3-D moist Jovian column, 256 x 256 x 128, FP32 (state 369 MB, larger than L2)."""
    from paper_1901_02955_gb300 import Context
    w = workload("f32", "jovian_256x256x128")[0]
    ctx = Context(w, dtype="f32")
    ctx.set_stream(stream)
    ctx.set_state(w.Y.astype(np.float32))
    ms = timed_steps(ctx, stream, max(4, args.steps // 8), 3)
    ctx.close()
    out = {"value": w.ncells * 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "cells": w.ncells, "nfields": w.nv, "l2": "inputs larger than L2"}
    out.update(stage_rooflines(ms, w.ncells, w.nv, 3, peak, peak_src,
                               ncu_record("jovian_256x256x128", "kern_moist3d.cu")))
    return out


def ensemble_line(args, stream, peak, peak_src):
    """The 96-domain moist ensemble (8.36 M cells, FP32): the autotuned launch mode, and the
    persistent one-launch step of the same tile shape."""
    from paper_1901_02955_gb300 import Context
    ws = workload("f32", "ensemble_96")
    ctx = Context(ws, dtype="f32")
    ctx.set_stream(stream)
    for d, w in enumerate(ws):
        ctx.set_state(w.Y.astype(np.float32), domain=d)
    tuned = ctx.autotune(steps=3)
    k = max(4, args.steps // 8)
    ms = timed_steps(ctx, stream, k, 3)
    info = ctx.info()
    ctx.use_persistent(not info["persistent"])
    ms_other = timed_steps(ctx, stream, k, 3)
    pers = ms if info["persistent"] else ms_other
    three = ms_other if info["persistent"] else ms
    ctx.close()
    cells = sum(w.ncells for w in ws)
    out = {"value": cells * 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "cells": cells,
           "domains": len(ws), "nfields": ws[0].nv, "autotune": tuned,
           "tile": list(info["tile"]), "tile_per_size": info.get("tile_per_size"),
           "ms_per_step_persistent": pers, "ms_per_step_three_launches": three,
           "l2": "inputs larger than L2"}
    out.update(stage_rooflines(ms, cells, ws[0].nv, 2, peak, peak_src,
                               ncu_record("ensemble_96", "kern_moist2d.cu")))
    return out


def parity_gpu_steps(stream):
    """One GPU step of the bench input (from rest) and of the same state with a seeded
    velocity field, in FP32 and FP64, at the initial CFL time step: the inputs and results
    (numpy, FP64) for the parity report."""
    import workloads as W
    from paper_1901_02955_gb300 import Context
    out = {}
    for case in ("from_rest", "moving"):
        w = workload("f64")
        if case == "moving":
            w = W.add_random_motion(w)
        for dt_name in ("f32", "f64"):
            Y0 = w.Y.astype(np.float32).astype(np.float64) if dt_name == "f32" else w.Y
            ctx = Context(w, dtype=dt_name)
            ctx.set_stream(stream)
            ctx.set_state(Y0)
            dt = ctx.compute_dt()
            ctx.step(1, dt_fixed=dt)
            out[(case, dt_name)] = (w, Y0, dt, ctx.get_state())
            ctx.close()
    return out


def parity_report(gpu_steps):
    """Relative L2 error of each field of one full-size step against the FP64 oracle on the
    same input (part of the CPU-baseline leg, after the timed regions), against two norms:
      vs_state: the parity tests' reference, the larger of the oracle's and the input's norm
        of the field (the momentum vector for a momentum component, floored at ||rho|| x
        1 m/s: a flow from rest has momenta near zero after one step); bounds 1e-5 FP32,
        1e-12 FP64;
      vs_increment: the norm of the oracle's increment Y_oracle - Y_0 of the field.
    increment_over_state is ||Y_oracle - Y_0|| / ||Y_0||: an FP32 state resolves increments
    only to about 6e-8 of the state, so vs_increment can be no better than 6e-8 over it."""
    import oracle
    oracle.build()
    rep = {}
    for (case, dt_name), (w, Y0, dt, Yg) in gpu_steps.items():
        Yo, _, rc = oracle.Oracle(w).step(Y0, 1, dt=dt)
        names = w.field_names()
        nv = len(names)
        im0 = 1 + w.nvapor * (1 + w.ncond)
        rho_norm = float(np.linalg.norm(Yo[:im0].sum(axis=0)))
        d = {}
        for f, nm in enumerate(names):
            err = float(np.linalg.norm(Yg[f] - Yo[f]))
            ref = list(range(im0, nv - 1)) if im0 <= f < nv - 1 else [f]
            den = max(float(np.linalg.norm(Yo[ref])), float(np.linalg.norm(Y0[ref])))
            if im0 <= f < nv - 1:
                den = max(den, rho_norm)
            inc = float(np.linalg.norm(Yo[f] - Y0[f]))
            d[nm] = {"vs_state": err / max(den, 1e-300),
                     "vs_increment": err / max(inc, 1e-300),
                     "increment_over_state": inc / max(float(np.linalg.norm(Y0[f])), 1e-300)}
        rep.setdefault(case, {})[dt_name] = d
    rep["note"] = ("one SSP-RK3 step of density_current_1024x256 at the initial CFL time step, "
                   "GPU (C ABI) against the FP64 oracle on the same input (FP32: the "
                   "FP32-rounded input on both sides); 'moving' adds a seeded random velocity "
                   "field to the same state")
    return rep


def jovian_window_steps(stream, nsamp=24):
    """Stage 0 of the full Jovian column (256 x 256 x 128) on the GPU in FP32 and FP64, at the
    initial CFL time step; kept: the stage result at seeded sample cells (interior levels) and
    the input on the 7 x 7 x 7 window around each (a stage result depends only on cells within
    3 along each axis; x and y periodic), for the parity report."""
    import torch
    import workloads as W
    from paper_1901_02955_gb300 import Context
    w = W.jovian(dtype="f64")
    rs = np.random.default_rng(3)
    cells = [(int(rs.integers(w.nx)), int(rs.integers(w.ny)), int(rs.integers(3, w.nz - 3)))
             for _ in range(nsamp)]
    ii = torch.tensor([c[0] for c in cells], device="cuda")
    jj = torch.tensor([c[1] for c in cells], device="cuda")
    kk = torch.tensor([c[2] for c in cells], device="cuda")
    e_ref = 0.5 * (w.p_bar_face[:-1] + w.p_bar_face[1:]) / (w.gamma_d - 1.0)
    out = {}
    for dt_name in ("f32", "f64"):
        Y0 = w.Y.astype(np.float32) if dt_name == "f32" else w.Y
        ctx = Context(w, dtype=dt_name)
        ctx.set_stream(stream)
        ctx.set_state(Y0)
        dt = ctx.compute_dt()
        ctx.stage(0, dt_fixed=dt)
        stream.synchronize()
        got = ctx.buffer_view(slot=1)[:, kk, jj, ii].double().cpu().numpy().T.copy()
        ctx.close()
        Yd = Y0.astype(np.float64)
        wins = []
        for n, (i, j, k) in enumerate(cells):
            got[n, -1] += e_ref[k]  # stored energy -> total energy
            xi = [(i + s) % w.nx for s in range(-3, 4)]
            yj = [(j + s) % w.ny for s in range(-3, 4)]
            wins.append(np.ascontiguousarray(Yd[:, k - 3:k + 4][:, :, yj][:, :, :, xi]))
        out[dt_name] = (dt, got, wins)
    return w, cells, out


def jovian_window_report(steps):
    """Per-field errors of the GPU's stage 0 at the sampled cells of the Jovian column against
    the FP64 oracle's stage 0 on each cell's 7 x 7 x 7 window of the same input: the
    relative L2 over the samples against the oracle's values (vs_state; a condensate against
    its vapour's, a momentum component against the momentum vector floored at the density x
    1 m/s, as in the parity tests) and against the oracle's increment over the stage
    (vs_increment; None where the oracle's increment is exactly zero, as for the dry air and
    the energy of a column at rest in hydrostatic balance), the increment over the state, and
    the largest error over the largest magnitude of the same reference (max_vs_state)."""
    import dataclasses
    import oracle
    oracle.build()
    w, cells, out = steps
    names = w.field_names()
    im0 = 1 + w.nvapor * (1 + w.ncond)
    rep = {}
    for dt_name, (dt, got, wins) in out.items():
        want = np.empty_like(got)
        y0 = np.empty_like(got)
        for n, (i, j, k) in enumerate(cells):
            ww = dataclasses.replace(w, nx=7, ny=7, nz=7, Y=wins[n],
                                     rho_bar=w.rho_bar[k - 3:k + 4],
                                     p_bar_face=w.p_bar_face[k - 3:k + 5])
            o, _ = oracle.Oracle(ww).stage(0, ww.Y, ww.Y, dt)
            want[n] = o[:, 3, 3, 3]
            y0[n] = wins[n][:, 3, 3, 3]
        err = got - want
        rho = want[:, :im0].sum(axis=1)
        nmom = len(names) - 1 - im0
        d = {}
        for f, nm in enumerate(names):
            if im0 <= f < len(names) - 1:  # the momentum vector, floored at rho x 1 m/s
                sel = want[:, im0:im0 + nmom]
                ref = max(float(np.linalg.norm(sel)), float(np.linalg.norm(rho)))
                top = max(float(np.abs(sel).max()), float(rho.max()))
            elif 1 + w.nvapor <= f < im0:  # a condensate against its vapour too
                sel = want[:, [f, 1 + (f - 1 - w.nvapor) // w.ncond]]
                ref = max(float(np.linalg.norm(c)) for c in sel.T)
                top = float(np.abs(sel).max())
            else:
                ref = float(np.linalg.norm(want[:, f]))
                top = float(np.abs(want[:, f]).max())
            inc = float(np.linalg.norm(want[:, f] - y0[:, f]))
            e2 = float(np.linalg.norm(err[:, f]))
            d[nm] = {"vs_state": e2 / max(ref, 1e-300),
                     "vs_increment": e2 / inc if inc > 0.0 else None,
                     "increment_over_state": inc / max(ref, 1e-300),
                     "max_vs_state": float(np.abs(err[:, f]).max()) / max(top, 1e-300)}
        rep[dt_name] = d
    rep["note"] = (f"stage 0 of jovian_256x256x128 at {len(cells)} seeded cells, GPU (C ABI) "
                   "against the FP64 oracle on the 7 x 7 x 7 window of the same input around "
                   "each (FP32: the FP32-rounded input on both sides); the column starts at "
                   "rest in hydrostatic balance, so in one stage only the vertical momentum "
                   "(buoyancy) and the species the adjustment moves change by much")
    return rep


if __name__ == "__main__":
    main()
