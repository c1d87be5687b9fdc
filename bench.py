"""Benchmark of the subset-gradient path of RDP-regularised PET reconstruction.

Headline workload (c5, brain-scale TOF): 215x215x71 image (1.3x1.3x2.0 mm), cylindrical
scanner sinogram 357 radial x 224 views x 1293 planes x 13 TOF bins (1.34 G bins, uint16
counts, 3e8 total, 20% smooth background), 25 view subsets (24 of 9 views, 1 of 8),
generated on the device.  One STEP is one SVRG outer loop of Algorithm 1: the harmonic
preconditioner update (eq. 8), a snapshot refresh (25 subset gradients) and 49 inner
iterations (eq. 9 + eq. 6), i.e. 74 subset gradients (TOF forward projection, KL
ratio, backprojection and RDP gradient) per step.  The JSON line also carries the same
measurement on the 3D non-TOF workload (c2: 128x128x47, 250 x 168 x 109, 21 subsets,
62 subset gradients per step) and the time to 1% NRMSE against converged oracle images.

Metric: subset gradients per second (whole job: all ranks).  Multi-GPU runs are
independent replicas (one reconstruction per rank, no collective on the data path).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload c5|c2]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "subset grads/s (fwd+back+RDP) & % HBM roofline; time to 1% NRMSE vs oracle"
UNIT = "subset_grads/s"
WORKLOADS = {
    "c5": ("c5: 3D TOF brain-scale 215x215x71 (1.3x1.3x2 mm), sinogram 357 radial x 224 views x 1293 "
           "planes (36 rings, span 1) x 13 TOF bins (1.34 G bins), uint16 counts (3e8), 25 subsets "
           "(24 of 9 views, 1 of 8), SVRG + harmonic preconditioner"),
    "c2": ("c2: 3D non-TOF 128x128x47 (2x2x2.8 mm), sinogram 250 radial x 168 views x 109 planes "
           "(span-3 segments 0 and +-9), 1e7 counts, 21 subsets, SVRG + harmonic preconditioner"),
}
WORKLOAD = WORKLOADS["c5"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-copy-blocks", type=int, default=8,
                    help="e2e ingest kernel: grid bound of pet_copy_to_device (0: four blocks per SM; 8 "
                         "blocks already move 175 GB/s)")
    ap.add_argument("--e2e-copy", default="engine", choices=["engine", "kernel", "serial"],
                    help="e2e ingest: the next step's data copied during the current step by the copy "
                         "engines (engine) or by pet_copy_to_device (kernel), or copied by "
                         "pet_copy_to_device before each step (serial)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-nrmse", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--mode", default="step", choices=["step", "grad", "configs", "study", "c4", "c5", "update"],
                    help="grad: only the fused subset-gradient op, for profiler captures; "
                         "configs: SVRG outer-loop rates on the 2D, 3D and 3D TOF workloads; "
                         "study: epochs to 1%% NRMSE over algorithm x preconditioner x tau0 (2D)")
    ap.add_argument("--shape", default="auto",
                    help="grad mode: 'auto' (autotuner) or 'K,S' planes per thread, parts per LOR")
    ap.add_argument("--config", default="c2", choices=["c2", "c3", "c5", "c5p"],
                    help="grad mode: c2 (non-TOF, 1e7 counts), c3 (11 TOF bins, 1e6 counts), c5 "
                         "(13 TOF bins, 1.34 G bins, generated on the device) or c5p (c5 with 50 views: "
                         "2 views per subset, for profiler captures)")
    ap.add_argument("--workload", default="c5", choices=["c5", "c2"],
                    help="step mode: the workload of the headline line (the other one is added as a key)")
    ap.add_argument("--no-c2", action="store_true", help="step mode: skip the secondary c2 measurement")
    ap.add_argument("--study-config", default="c1", choices=["c1", "c1b5", "c1b50", "c2", "c2s", "c2s1", "c2s16", "c2sb50", "c3s"],
                    help="study mode: workload with a converged reference image in tests/golden")
    ap.add_argument("--study-nsub", type=int, default=0,
                    help="study mode: number of subsets (0: the workload's own; Sec. 3.2 uses 27)")
    ap.add_argument("--study-plain", action="store_true",
                    help="study mode: the plain form (one launch per kernel, no CUDA graphs)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(pg, seconds, device):
    """The slowest rank's time (all ranks call this; pg None: single process)."""
    if pg is None:
        return seconds
    import torch
    t = torch.tensor([seconds], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t)


def whole_job_rate(units_per_rank, world, seconds):
    """Units processed by all ranks (independent replicas) per second of the slowest rank."""
    return units_per_rank * world / seconds


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_hash(kernel_name):
    """Hash of the sources a fused-gradient kernel is built from: the windowed TOF kernels
    (tof_kernels.cu) or the others (proj_kernels.cu), with the shared headers."""
    files = ("tof_kernels.cu" if kernel_name.startswith("k_grad_tof") else "proj_kernels.cu", "pet_internal.cuh",
             "packed_f32x2.cuh")
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2506_04976_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_instructions(kernel_tag, kernel_name):
    """Warp instructions per launch of the dominant kernel from the committed ncu summary
    (same conditions as ncu_traffic); else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("source_hash") != source_hash(kernel_name):
        return None
    return d.get("warp_instructions_per_launch", {}).get(kernel_name)


def ncu_traffic(kernel_tag, kernel_name):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, if
    it profiled the same kernel variant and the kernel source is unchanged since the
    counters were taken; else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("source_hash") != source_hash(kernel_name):
        return None
    return d.get("dram_bytes_per_launch", {}).get(kernel_name)


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, out):
        self.out = out
        self.p = None

    def __enter__(self):
        try:
            self.f = open(self.out, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()
            self.f.close()

    def summary(self):
        if not self.p or not os.path.exists(self.out):
            return None
        rows = []
        for line in open(self.out):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), util=float(parts[4]),
                                 hw=parts[6], hwt=parts[7], swt=parts[8], pcap=parts[9]))
            except ValueError:
                continue
        if not rows:
            return None
        load = [r for r in rows if r["util"] >= 50] or rows
        reasons = []
        for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                          ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
            if any(r[key].lower() == "active" for r in load):
                reasons.append(name)
        return {"sm_mhz": float(np.median([r["sm"] for r in load])),
                "sm_max_mhz": max(r["smax"] for r in load), "reasons": reasons,
                "samples": len(load)}


def load_workload(cfg, seed, dev):
    """(problem dict, device tensors y, r, mu, sens) of a workload: c5 is generated on the
    device (its 1.34 G TOF bins do not fit the host generator), the others on the host."""
    import torch
    from paper_2506_04976_gb300 import synth
    if cfg in ("c3", "c5", "c5p"):
        p = synth.make_problem_device(cfg, seed, device=dev) if cfg != "c5p" else \
            synth.make_problem_device("c5", seed, device=dev, nview=50)
        dt = dict(y=p["y"], r=p["r"], sens=p["sens"], mu=torch.from_numpy(p["mu"].astype(np.float32)).to(dev))
        torch.cuda.synchronize()
        torch.cuda.empty_cache()  # return the generator's temporaries to the device
    else:
        p = synth.make_problem(cfg, seed)
        y = p["y"].view(np.int16) if p["y"].dtype == np.uint16 else p["y"].astype(np.int32)
        dt = dict(y=torch.from_numpy(y).to(dev), r=torch.from_numpy(p["r"]).to(dev),
                  mu=torch.from_numpy(p["mu"].astype(np.float32)).to(dev),
                  sens=torch.from_numpy(p["sens"].astype(np.float32)).to(dev))
    return p, dt


def algorithmic_bytes_per_grad(p, y_itemsize=2):
    """Fused subset gradient, averaged over the n subsets: counts and background (f32) per
    TOF bin, factors m (f32) per LOR, one read of the image and one write of the gradient."""
    g = p["geom"]
    T = g["ntof"] if g["ntof"] > 1 else 1
    lors = g["nview"] * len(g["z1"]) * g["nrad"] / p["nsub"]
    N = g["nx"] * g["ny"] * g["nz"]
    return lors * (T * (y_itemsize + 4) + 4) + 2 * 4 * N


def cpu_baseline(p, seconds, steps=None):
    """The FP64 oracle, single-threaded, on whole subset gradients of the same workload
    (data gradient of one subset + RDP gradient), repeated for about `seconds`."""
    import oracle as O
    G = O.Geometry(p["geom"])
    m = O.multiplicative(G, p["mu"], p["sens"])
    x = np.maximum(p["x_true"], 0.05 * p["x_true"].max())
    sp = (p["geom"]["dx"], p["geom"]["dy"], p["geom"]["dz"])
    times = []
    s = 0
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        O.data_grad(G, p["nsub"], s % p["nsub"], x, m, p["r"], p["y"])
        O.rdp(x, sp, p["gamma"], p["eps"])
        times.append(time.perf_counter() - t0)
        s += 1
        if steps is not None:
            if s >= steps:
                break
        elif time.perf_counter() - t_start >= seconds:
            break
    return times


def oracle_workers():
    return max(1, min(16, os.cpu_count() or 1))


def oracle_sampled_rate(p, subset=0, planes_every=1, workers=None):
    """The FP64 oracle on a bounded sample of a device-generated workload: the data term
    and gradient of the first view of `subset` over every `planes_every`-th plane, split
    over host processes (oracle.pieces; the slowest worker's compute time), scaled to a
    whole subset by its LOR count, plus one single-threaded RDP gradient of the image."""
    import torch
    import oracle as O
    from oracle import pieces
    g = p["geom"]
    n = p["nsub"]
    workers = workers or oracle_workers()
    views = O.subset_views(g["nview"], n, subset)
    v = int(views[0])
    P = len(g["z1"])
    sel = np.arange(0, P, planes_every)
    gk = dict(g, z1=np.asarray(g["z1"])[sel], z2=np.asarray(g["z2"])[sel])
    si = torch.from_numpy(sel.astype(np.int64)).to(p["y"].device)
    y = p["y"][v].index_select(0, si).cpu().numpy()
    y = y.view(np.uint16) if y.dtype == np.int16 else y
    r = p["r"][v].index_select(0, si).cpu().numpy()
    sens = p["sens"][v].index_select(0, si).cpu().numpy()
    x = np.maximum(p["x_true"], 0.05 * p["x_true"].max()).astype(np.float32)
    timing = {}
    pieces.data_grad_subset(gk, [v], x, p["mu"].astype(np.float32), sens[None], r[None], y[None],
                            workers=workers, chunk=-(-len(sel) // workers), timing=timing)
    t0 = time.perf_counter()
    O.rdp(x.astype(np.float64), (g["dx"], g["dy"], g["dz"]), p["gamma"], p["eps"])
    t_rdp = time.perf_counter() - t0
    frac = len(sel) / (len(views) * P)
    t_grad = timing["seconds"] / frac + t_rdp
    sample = (f"FP64 oracle: data term + gradient of view {v} of subset {subset} over {len(sel)} of {P} planes "
              f"(all {g['nrad']} radial bins x {g['ntof']} TOF bins; {frac:.4f} of the subset's LORs) in "
              f"{timing['workers']} processes ({timing['seconds']:.2f} s, slowest worker), scaled by the LOR "
              f"count, + one single-threaded RDP gradient ({t_rdp:.2f} s)")
    return {"value": 1.0 / t_grad, "unit": UNIT, "cores": timing["workers"], "kind": "oracle", "sample": sample}


def oracle_subset_rate_mp(p, subset=0, workers=None):
    """The FP64 oracle on one whole subset gradient of a host-generated workload, its data
    term split over host processes by view and run of planes (oracle.pieces; the slowest
    worker's compute time), plus one single-threaded RDP gradient."""
    import oracle as O
    from oracle import pieces
    g = p["geom"]
    workers = workers or oracle_workers()
    views = [int(v) for v in O.subset_views(g["nview"], p["nsub"], subset)]
    P = len(g["z1"])
    chunk = max(1, -(-P * len(views) // (2 * workers)))
    x = np.maximum(p["x_true"], 0.05 * p["x_true"].max()).astype(np.float32)
    timing = {}
    pieces.data_grad_subset(g, views, x, p["mu"].astype(np.float32), p["sens"][views], p["r"][views], p["y"][views],
                            workers=workers, chunk=min(chunk, P), timing=timing)
    t0 = time.perf_counter()
    O.rdp(x.astype(np.float64), (g["dx"], g["dy"], g["dz"]), p["gamma"], p["eps"])
    t_rdp = time.perf_counter() - t0
    t = timing["seconds"] + t_rdp
    return {"subset_grads_per_s": 1.0 / t, "cores": timing["workers"],
            "sample": f"one subset gradient, FP64, data term over {timing['workers']} processes "
                      f"({timing['seconds']:.3f} s, slowest worker) + single-threaded RDP ({t_rdp:.3f} s)"}


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle as it stands on the host cores, on a bounded
    sample of the headline workload per step (rank 0 only)."""
    if rank != 0:
        return
    cfg = getattr(args, "workload", "c5")
    if cfg == "c5":
        import torch
        dev = torch.device("cuda", 0)
        from paper_2506_04976_gb300 import synth
        p = synth.make_problem_device("c5", 0, device=dev)
        torch.cuda.synchronize()
        rates = []
        for k in range(args.warmup + args.steps):
            r = oracle_sampled_rate(p, subset=k % p["nsub"], planes_every=2)
            if k >= args.warmup:
                rates.append(r)
        times = [1.0 / r["value"] for r in rates]
        cores = rates[-1]["cores"]
        sample = f"per step: {rates[-1]['sample']}"
    else:
        from paper_2506_04976_gb300 import synth
        p = synth.make_problem(cfg, 0)
        cpu_baseline(p, 0, steps=args.warmup) if args.warmup > 0 else None
        times = cpu_baseline(p, 0, steps=args.steps)
        cores = 1
        sample = f"{len(times)} full-size subset gradients (fwd+back+RDP), FP64, 1 thread"
    total = sum(times)
    value = len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOADS[cfg], "step": "one subset gradient"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_until_nrmse(pet, solver, n, xref, mask, bg, threshold, max_epochs, start_event, marks=(), check_every=20):
    """Runs whole epochs until the NRMSE against xref falls below threshold.  The NRMSE of
    every epoch is computed on the device right after it and an event is recorded there;
    the host reads them every `check_every` epochs (no host round trip per epoch), and the
    time reported runs from start_event to the event of the first epoch below threshold.
    Returns (epochs to threshold or None, seconds, NRMSE at the end, {mark: NRMSE})."""
    import torch
    reached, last, at, seconds = None, None, {}, None
    e = 0
    while e < max_epochs and reached is None:
        block = []
        for _ in range(min(check_every, max_epochs - e)):
            e += 1
            solver.run(n)
            v = pet.nrmse(solver.image(), xref, mask, bg)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record()
            block.append((e, v, ev))
        torch.cuda.synchronize()
        for ee, v, ev in block:
            val = float(v)
            if ee in marks:
                at[ee] = val
            last = val
            if not np.isfinite(val):
                seconds = start_event.elapsed_time(ev) / 1e3
                return None, seconds, val, at
            if val < threshold:
                reached, seconds = ee, start_event.elapsed_time(ev) / 1e3
                last = val
                break
        if reached is None:
            seconds = start_event.elapsed_time(block[-1][2]) / 1e3
    return reached, seconds, last, at


def time_to_nrmse(pet, dev, config, seed=0, threshold=0.01, max_epochs=3000):
    """GPU wall time from the start of the OSEM initialisation (Sec. 3.1) to the first
    epoch whose NRMSE (c19 reading) against the oracle's converged image is below the
    threshold, for the graph form and the plain form (one launch per kernel).  Returns
    None when no reference image has been written for this configuration."""
    import torch
    ref_path = os.path.join(ROOT, "tests", "golden", f"ref_{config}_seed{seed}.npz")
    if not os.path.exists(ref_path):
        return None
    from paper_2506_04976_gb300 import synth
    ref = np.load(ref_path)
    p = synth.make_problem(config, seed)
    n = p["nsub"]
    plan = pet.Plan(p["geom"], n)
    y = p["y"].view(np.int16) if p["y"].dtype == np.uint16 else p["y"].astype(np.int32)
    plan.set_data(torch.from_numpy(y).to(dev), torch.from_numpy(p["r"]).to(dev),
                  torch.from_numpy(p["mu"].astype(np.float32)).to(dev),
                  torch.from_numpy(p["sens"].astype(np.float32)).to(dev))
    plan.autotune()
    xref = torch.from_numpy(ref["x"]).to(dev)
    mask = torch.from_numpy(p["mask"]).to(dev)
    bg = torch.from_numpy(p["bg"]).to(dev)
    # the 2D workload runs the settings it is specified with (SVRG, vanishing steps from
    # tau0 = 1, eta = 0.02, preconditioner in epochs 1-3); the 3D ones the submitted ALG1
    # (its steps end at 0.5 and keep converging on them; ALG2/ALG3 keep a step of 0.7-1
    # after epoch 6, the BB value or its cap in Table 1, and stall on the full-size 3D
    # workload)
    from paper_2506_04976_gb300.presets import petric_solver_kwargs
    if p["geom"]["nz"] == 1:
        kw = dict(algo=pet.SVRG, omega=2, step_rule=pet.STEP_VANISH, tau0=1.0, eta=0.02, precond_kind=1,
                  pc_iters=(0, n, 2 * n))
        method = "SVRG, vanishing steps tau0 = 1, eta = 0.02, harmonic preconditioner in epochs 1-3"
    else:
        kw = petric_solver_kwargs("ALG1", n)
        method = "ALG1 of Table 1 (SVRG, piecewise steps 3/2/1.5/1/0.5, harmonic preconditioner in epochs 1-3)"
    out = {"reference_kkt": float(ref["kkt"]), "threshold": threshold, "method": method}
    for form in ("graph", "plain"):
        solver = pet.Solver(plan, beta=p["beta"], gamma=p["gamma"], eps=p["eps"], seed=77,
                            use_graph=(form == "graph"), **kw)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        a.record()
        x = torch.ones(plan.img_shape, device=dev)
        for s in range(n):
            plan.em_update(x, s)
        solver.set_image(x)
        reached, seconds, val, _ = run_until_nrmse(pet, solver, n, xref, mask, bg, threshold, max_epochs, a)
        out[form] = {"seconds": seconds, "epochs": reached, "final_nrmse": val}
    return out


def svrg_loop_rate(pet, dev, p, steps, warmup, use_graph=True):
    """Subset gradients per second of whole SVRG outer loops (refresh + 2n - 1 inner
    iterations, harmonic preconditioner updated at each loop start), L2 flushed between
    loops, and the average duration of the fused subset-gradient kernel."""
    import torch
    n = p["nsub"]
    plan = pet.Plan(p["geom"], n)
    y = p["y"].view(np.int16) if p["y"].dtype == np.uint16 else p["y"].astype(np.int32)
    keep = [torch.from_numpy(y).to(dev), torch.from_numpy(p["r"]).to(dev),
            torch.from_numpy(p["mu"].astype(np.float32)).to(dev),
            torch.from_numpy(p["sens"].astype(np.float32)).to(dev)]
    plan.set_data(*keep)
    shape = plan.autotune()
    x0 = torch.ones(plan.img_shape, device=dev)
    for s in range(n):
        plan.em_update(x0, s)
    step_len = 2 * n
    pcs = [k * step_len for k in range(steps + warmup + 1)]
    solver = pet.Solver(plan, algo=pet.SVRG, omega=2, step_rule=pet.STEP_VANISH, tau0=1.0, eta=0.02,
                        precond_kind=1, pc_iters=pcs, beta=p["beta"], gamma=p["gamma"], eps=p["eps"],
                        seed=4321, use_graph=use_graph)
    solver.set_image(x0)
    solver.profile(True)
    flush = torch.empty(64 * 1024 * 1024, device=dev)
    for _ in range(warmup):
        solver.run(step_len)
    torch.cuda.synchronize()
    solver.kernel_time()
    total = 0.0
    kms, kn = 0.0, 0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        solver.run(step_len)
        b.record()
        torch.cuda.synchronize()
        total += a.elapsed_time(b) / 1e3
        ms, nl = solver.kernel_time()
        kms += ms
        kn += nl
    units = (3 * n - 1) * steps
    return {"subset_grads_per_s": units / total, "ms_per_outer_loop": 1e3 * total / steps,
            "fused_kernel_ms": kms / max(kn, 1), "grad_shape": list(shape), "graph": use_graph}


def run_configs(args, pet, dev):
    """Rates on the 2D (c1), 3D non-TOF (c2) and 3D TOF (c3) workloads with the roofline
    figures of the fused subset gradient (algorithmic bytes per launch / launch time)."""
    from paper_2506_04976_gb300 import synth
    peak, peak_kind = measured_peaks()
    out = {"mode": "configs", "peak_gbs": peak, "peak_kind": peak_kind, "configs": {}}
    for cfg in ("c1", "c2", "c3"):
        p = synth.make_problem(cfg, 0)
        r = svrg_loop_rate(pet, dev, p, args.steps, args.warmup)
        g = p["geom"]
        T = g["ntof"] if g["ntof"] > 1 else 1
        lors = (g["nview"] // p["nsub"]) * len(g["z1"]) * g["nrad"]
        N = g["nx"] * g["ny"] * g["nz"]
        abytes = lors * T * (p["y"].itemsize + 4) + lors * 4 + 2 * 4 * N
        r["algorithmic_bytes"] = abytes
        r["achieved_gbs"] = abytes / (r["fused_kernel_ms"] * 1e-3) / 1e9
        r["hbm_frac"] = r["achieved_gbs"] / peak
        if T > 1:
            r["tof_bins_per_s"] = lors * T / (r["fused_kernel_ms"] * 1e-3)
        if not args.no_cpu:  # the FP64 oracle on one or two whole subset gradients of the same workload
            times = cpu_baseline(p, 0, steps=1 if T > 1 else 2)
            r["cpu_oracle"] = {"subset_grads_per_s": len(times) / sum(times), "cores": 1,
                               "sample": f"{len(times)} subset gradient(s), FP64, 1 thread"}
            r["cpu_oracle_processes"] = oracle_subset_rate_mp(p)
        out["configs"][cfg] = r
    print(json.dumps(out), flush=True)


def run_study(args, pet, dev, max_epochs=1500):
    """The comparison of Sec. 3.2 (Fig. 2) against a converged oracle image (2D workload by
    default, 3D with --study-config c2 / c2s / c2s16, 3D TOF with c3s): SGD / SAGA / SVRG
    x MLEM / harmonic preconditioner x tau0 in {0.3, 1, 1.5}, vanishing steps (eta = 0.02),
    preconditioner updated in epochs 1-3, subsets without replacement; then the three
    submitted algorithms (Table 1).
    Epochs and GPU seconds from the OSEM start to NRMSE < 1%, and the NRMSE after
    5 ... 500 epochs."""
    import torch
    from paper_2506_04976_gb300 import synth
    cfg = args.study_config
    ref_path = os.path.join(ROOT, "tests", "golden", f"ref_{cfg}_seed0.npz")
    ref = np.load(ref_path)
    p = synth.make_problem(cfg, 0)
    n = args.study_nsub or p["nsub"]  # the objective does not depend on n, so the reference holds
    plan = pet.Plan(p["geom"], n)
    y = p["y"].view(np.int16) if p["y"].dtype == np.uint16 else p["y"].astype(np.int32)
    plan.set_data(torch.from_numpy(y).to(dev), torch.from_numpy(p["r"]).to(dev),
                  torch.from_numpy(p["mu"].astype(np.float32)).to(dev),
                  torch.from_numpy(p["sens"].astype(np.float32)).to(dev))
    plan.autotune()
    xref = torch.from_numpy(ref["x"]).to(dev)
    mask = torch.from_numpy(p["mask"]).to(dev)
    bg = torch.from_numpy(p["bg"]).to(dev)
    x0 = torch.ones(plan.img_shape, device=dev)
    for s in range(n):  # one OSEM epoch (Sec. 3.1)
        plan.em_update(x0, s)
    from paper_2506_04976_gb300.presets import petric_solver_kwargs
    marks = (5, 10, 20, 50, 100, 500)

    def until_1pct(solver):
        solver.set_image(x0)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        a.record()
        reached, seconds, val, at = run_until_nrmse(pet, solver, n, xref, mask, bg, 0.01, max_epochs, a, marks)
        return {"epochs_to_1pct": reached, "seconds": seconds, "final_nrmse": val, "nrmse_at_epoch": at}

    rows = []
    for algo, aname in ((pet.SGD, "SGD"), (pet.SAGA, "SAGA"), (pet.SVRG, "SVRG")):
        for pc, pname in ((0, "MLEM"), (1, "harmonic")):
            for tau0 in (0.3, 1.0, 1.5):
                solver = pet.Solver(plan, algo=algo, omega=2, step_rule=pet.STEP_VANISH, tau0=tau0, eta=0.02,
                                    precond_kind=pc, pc_iters=(0, n, 2 * n), beta=p["beta"], gamma=p["gamma"],
                                    eps=p["eps"], seed=31, use_graph=not args.study_plain)
                rows.append({"algo": aname, "precond": pname, "tau0": tau0, **until_1pct(solver)})
                del solver
    for name in ("ALG1", "ALG2", "ALG3"):  # the submitted algorithms (Table 1) with this n
        solver = pet.Solver(plan, beta=p["beta"], gamma=p["gamma"], eps=p["eps"], seed=31,
                            use_graph=not args.study_plain, **petric_solver_kwargs(name, n))
        rows.append({"algo": name, "precond": "harmonic", "tau0": None, **until_1pct(solver)})
        del solver
    print(json.dumps({"mode": "study", "workload": f"{cfg}, n = {n}, beta = {p['beta']:.4g}", "max_epochs": max_epochs,
                      "form": "plain" if args.study_plain else "graph",
                      "reference_kkt": float(ref["kkt"]), "runs": rows}), flush=True)


def run_batched(args, pet, dev, E=8):
    """32 independent reconstructions of uneven size (c4): SAGA with harmonic
    preconditioner, advanced by the batched driver (one launch per phase, one graph
    per window of E iterations) and, for comparison, by the same solvers run one
    after another.  Units: subset gradients (one per instance per iteration)."""
    import torch
    from paper_2506_04976_gb300 import synth
    t0 = time.perf_counter()
    plans, solvers, keep = [], [], []
    for i, sp in enumerate(synth.batch_specs(0, 32)):
        sp = dict(sp)
        name = sp.pop("name")
        p = synth.make_problem(name, 100 + i, **sp)
        plan = pet.Plan(p["geom"], p["nsub"])
        y = p["y"].view(np.int16) if p["y"].dtype == np.uint16 else p["y"].astype(np.int32)
        tensors = [torch.from_numpy(y).to(dev), torch.from_numpy(p["r"]).to(dev),
                   torch.from_numpy(p["mu"].astype(np.float32)).to(dev),
                   torch.from_numpy(p["sens"].astype(np.float32)).to(dev)]
        plan.set_data(*tensors)
        keep.append(tensors)
        x0 = torch.full(plan.img_shape, float(p["x_true"].mean()), device=dev)
        sv = pet.Solver(plan, algo=pet.SAGA, step_rule=pet.STEP_VANISH, tau0=1.0, eta=0.02, precond_kind=1,
                        pc_iters=(0,), beta=p["beta"], gamma=p["gamma"], eps=p["eps"], seed=500 + i)
        sv.set_image(x0)
        plans.append(plan)
        solvers.append(sv)
    setup_s = time.perf_counter() - t0
    batch = pet.Batch(solvers, iters_per_graph=E)
    shape = batch.autotune()
    batch.run(E * (1 + args.warmup))  # first window is plain (preconditioner update at k = 0)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = pet.launch_count()
    a.record()
    batch.run(E * args.steps)
    b.record()
    torch.cuda.synchronize()
    t_batch = a.elapsed_time(b) / 1e3
    l_batch = pet.launch_count() - l0
    del batch
    for plan in plans:
        plan.autotune()
    for sv in solvers:
        sv.run(E)
    torch.cuda.synchronize()
    l0 = pet.launch_count()
    a.record()
    for _ in range(args.steps):
        for sv in solvers:
            sv.run(E)
    b.record()
    torch.cuda.synchronize()
    t_seq = a.elapsed_time(b) / 1e3
    l_seq = pet.launch_count() - l0
    units = 32 * E * args.steps
    print(json.dumps({"mode": "c4", "workload": "32 SAGA reconstructions, 96..192 px, 1..35 slices, 8..28 subsets",
                      "units": units, "batched": {"subset_grads_per_s": units / t_batch, "seconds": t_batch,
                                                  "launches": l_batch, "grad_shape": shape},
                      "sequential": {"subset_grads_per_s": units / t_seq, "seconds": t_seq, "launches": l_seq},
                      "setup_s": setup_s}), flush=True)


def run_c5(args, pet, dev):
    """Large TOF workload (215x215x71; 357 x 224 x 1293 x 13 TOF bins): subset gradients
    (fused TOF forward, KL ratio, backprojection + RDP) on device-generated data, one
    SVRG outer loop (74 subset gradients) and one SAGA epoch (25)."""
    import torch
    from paper_2506_04976_gb300 import synth
    t0 = time.perf_counter()
    p = synth.make_problem_device("c5", 0, device=dev)
    t1 = time.perf_counter()
    n = p["nsub"]
    plan = pet.Plan(p["geom"], n)
    plan.set_data(p["y"], p["r"], torch.from_numpy(p["mu"].astype(np.float32)).to(dev), p["sens"])
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    shape = plan.autotune()
    x = torch.from_numpy(np.maximum(p["x_true"], 0.05 * p["x_true"].max()).astype(np.float32)).to(dev)
    g = torch.empty_like(x)
    prior = (p["beta"] / n, p["gamma"], p["eps"])
    for s in range(args.warmup):
        plan.objective_grad(x, s, prior=prior, g=g, want_obj=False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for s in range(args.steps):
        plan.objective_grad(x, s % n, prior=prior, g=g, want_obj=False)
    b.record()
    torch.cuda.synchronize()
    t_grad = a.elapsed_time(b) / 1e3 / args.steps
    solver = pet.Solver(plan, algo=pet.SVRG, beta=p["beta"], gamma=p["gamma"], eps=p["eps"],
                        pc_iters=(0,), seed=5)
    solver.set_image(x)
    solver.run(2 * n)  # warm-up outer loop (plain: preconditioner update at k = 0)
    torch.cuda.synchronize()
    solver.profile(True)
    a.record()
    solver.run(2 * n)
    b.record()
    torch.cuda.synchronize()
    t_loop = a.elapsed_time(b) / 1e3
    kms, kn = solver.kernel_time()
    del solver
    saga = pet.Solver(plan, algo=pet.SAGA, beta=p["beta"], gamma=p["gamma"], eps=p["eps"], pc_iters=(0,), seed=6)
    saga.set_image(x)
    saga.run(n)  # table initialisation pass + one epoch (plain: preconditioner update at k = 0)
    torch.cuda.synchronize()
    a.record()
    saga.run(n)
    b.record()
    torch.cuda.synchronize()
    t_saga = a.elapsed_time(b) / 1e3
    del saga
    lors = 9 * 1293 * 357
    samples = lors * 215  # about one bilinear sample per driving plane
    print(json.dumps({"mode": "c5", "generate_s": t1 - t0, "set_data_s": t2 - t1, "grad_shape": shape,
                      "subset_grad_ms": 1e3 * t_grad, "subset_grads_per_s": 1.0 / t_grad,
                      "svrg_outer_loop_s": t_loop, "svrg_subset_grads_per_s": (3 * n - 1) / t_loop,
                      "saga_epoch_s": t_saga, "saga_subset_grads_per_s": n / t_saga,
                      "fused_kernel_ms": kms / max(kn, 1), "fused_launches": kn,
                      "tof_bin_updates_per_s": lors * 13 / (kms / max(kn, 1) * 1e-3),
                      "samples_per_s_fwd_and_back": 2 * samples / (kms / max(kn, 1) * 1e-3)}), flush=True)


def run_update(args, pet, dev):
    """SVRG outer loops on a workload (default c5p: the brain-scale image, whose SVRG table
    of 25 subset gradients, 328 MB, exceeds L2) for captures of the estimator + step + prox
    kernel; prints the loop time."""
    import torch
    cfg = args.config if args.config != "c2" else "c5p"
    p, dt = load_workload(cfg, 0, dev)
    n = p["nsub"]
    plan = pet.Plan(p["geom"], n)
    plan.set_data(dt["y"], dt["r"], dt["mu"], dt["sens"])
    x = torch.from_numpy(np.maximum(p["x_true"], 0.05 * p["x_true"].max()).astype(np.float32)).to(dev)
    solver = pet.Solver(plan, algo=pet.SVRG, beta=p["beta"], gamma=p["gamma"], eps=p["eps"], pc_iters=(0,), seed=9)
    solver.set_image(x)
    solver.run(2 * n * max(args.warmup, 1))
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    solver.run(2 * n * args.steps)
    b.record()
    torch.cuda.synchronize()
    print(json.dumps({"mode": "update", "config": cfg, "ms_per_outer_loop": a.elapsed_time(b) / args.steps}))


def run_grad_only(args, pet, dev):
    """Subset gradients only (objective_grad on successive subsets), for ncu captures."""
    import torch
    from paper_2506_04976_gb300 import synth
    p, dt = load_workload(args.config, 0, dev)
    plan = pet.Plan(p["geom"], p["nsub"])
    plan.set_data(dt["y"], dt["r"], dt["mu"], dt["sens"])
    x = torch.from_numpy(np.maximum(p["x_true"], 0.05 * p["x_true"].max()).astype(np.float32)).to(dev)
    gbuf = torch.empty_like(x)

    def timed(shape):
        if shape == "auto":
            shape = plan.autotune()
        else:
            plan.set_grad_shape(*shape)
        for i in range(args.warmup):
            plan.objective_grad(x, i % p["nsub"], g=gbuf, want_obj=False)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for i in range(args.steps):
            plan.objective_grad(x, i % p["nsub"], g=gbuf, want_obj=False)
        b.record()
        torch.cuda.synchronize()
        return {"shape": list(shape), "ms_per_call": a.elapsed_time(b) / max(args.steps, 1)}

    if args.shape == "all":  # every launch shape the plan accepts, then the autotuner's choice
        rows = []
        for k in (1, 2, 4):
            for sp in (1, 2, 4, 8, 16):
                try:
                    rows.append(timed((k, sp)))
                except pet.PetError:
                    continue
        rows.append(dict(timed("auto"), autotuned=True))
        print(json.dumps({"mode": "grad", "config": args.config, "shapes": rows}))
        return
    r = timed("auto" if args.shape == "auto" else tuple(int(v) for v in args.shape.split(",")))
    print(json.dumps({"mode": "grad", "config": args.config, **r}))


def tof_window(geom):
    """Bins a TOF sample can meet, as the library's windowed TOF kernel counts them (its
    weight table has 1024 rows per bin width); 0 without TOF."""
    T = geom.get("ntof", 1)
    if T <= 1:
        return 0
    w, sig = geom["tof_bin"], geom["tof_sigma"]
    ktab = math.ceil(2.0 * (3.0 * sig + 0.5 * w) / (w / 1024))
    return (ktab - 1) // 1024 + 1


def kernel_name(geom, shape):
    T = geom.get("ntof", 1)
    if T > 1:
        win = tof_window(geom)
        if T <= 16 and win <= 8:
            wk = 4 if win <= 4 else 6 if win <= 6 else 8
            nt = 256 if shape[0] == 4 else 512
            if shape[1] == 1:  # one part per LOR: the persistent form
                return f"k_grad_tofp<{shape[0]},{wk},{nt}>"
            return f"k_grad_tofk<{shape[0]},{wk},{shape[1]},{nt}>"
        return f"k_grad<{16 if T <= 16 else 32},{shape[1]}>"
    return f"k_grad_mp<{shape[0]},{shape[1]}>" if shape[0] > 1 else f"k_grad<1,{shape[1]}>"


def issue_peak():
    """Instruction-issue roofline: 152 SMs x 4 schedulers x 1 warp instruction per cycle at
    the maximum SM clock."""
    sm_max = 2070.0
    mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(mp):
        sm_max = float(json.load(open(mp)).get("sm_max_mhz", sm_max))
    return 152 * 4 * sm_max * 1e6


def measure_svrg(pet, dev, cfg, p, dt, args, rank, world, pg, e2e=True, clk=None):
    """SVRG outer loops (harmonic preconditioner update, refresh of n subset gradients,
    2n - 1 inner iterations) of one workload: device-timed rate with the L2 flushed
    between steps, the fused kernel's live launch time, and the end-to-end rate through
    the C ABI with the step's inputs copied from pinned host memory every step."""
    import torch
    g = p["geom"]
    n = p["nsub"]
    T = g["ntof"] if g["ntof"] > 1 else 1
    step_len = 2 * n                      # one SVRG outer loop (omega = 2)
    grads_per_step = 3 * n - 1            # n at the refresh + (2n - 1) inner iterations
    plan = pet.Plan(g, n)
    plan.set_data(dt["y"], dt["r"], dt["mu"], dt["sens"])
    shape = plan.autotune()
    x0 = torch.ones(plan.img_shape, device=dev)
    for s in range(n):  # one OSEM epoch from a uniform image (Sec. 3.1 initialisation)
        plan.em_update(x0, s)
    total_steps = args.warmup + args.steps + (args.steps if e2e else 0)
    pcs = [k * step_len for k in range(total_steps + 1)]
    solver = pet.Solver(plan, algo=pet.SVRG, omega=2, step_rule=pet.STEP_VANISH, tau0=1.0, eta=0.02,
                        precond_kind=1, alpha=1.0, delta_rel=1e-6, pc_iters=pcs, beta=p["beta"],
                        gamma=p["gamma"], eps=p["eps"], seed=1234 + rank, use_graph=True)
    solver.set_image(x0)
    solver.profile(True)
    flush = torch.empty(64 * 1024 * 1024, device=dev)  # 256 MB > L2 (129 MB)
    for _ in range(args.warmup):
        solver.run(step_len)
    torch.cuda.synchronize()
    solver.kernel_time()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kern_ms, kern_n = 0.0, 0
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    launches0 = pet.launch_count()
    wall0 = time.perf_counter()
    if clk:
        clk.__enter__()
    try:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record()
            solver.run(step_len)
            ev[i][1].record()
            torch.cuda.synchronize()
            ms, nl = solver.kernel_time()
            kern_ms += ms
            kern_n += nl
        torch.cuda.synchronize()
    finally:
        if clk:
            clk.__exit__(None, None, None)
    wall = time.perf_counter() - wall0
    launches = pet.launch_count() - launches0
    if pg:
        pg.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = max_over_ranks(pg, sum(step_ms) / 1e3, dev)
    out = {"value": whole_job_rate(grads_per_step * args.steps, world, t_total),
           "ms_per_step": 1e3 * t_total / args.steps, "wall_s_timed": wall, "gpu_launches": launches,
           "grads_per_step": grads_per_step, "shape": shape, "kernel_ms": kern_ms / max(kern_n, 1),
           "kernel_launches": kern_n, "T": T, "y_itemsize": dt["y"].element_size()}
    if e2e:
        # The same SVRG outer loops as above, one reconstruction started from the pinned host
        # copy of the start image, with every step's counts and background copied from pinned
        # host memory and the image read back after every step.  engine / kernel: the copy
        # of step i + 1 runs on a second stream (the copy engines, or the library's ingest
        # kernel pet_copy_to_device on a few SMs) into the other of two device buffer sets
        # while step i computes, and pet_plan_set_counts binds each set before its step;
        # serial: pet_copy_to_device into the plan's buffers before each step.
        how = getattr(args, "e2e_copy", "engine")
        cblocks = getattr(args, "e2e_copy_blocks", 8)
        y_host = torch.empty(dt["y"].shape, dtype=dt["y"].dtype, pin_memory=True)
        r_host = torch.empty(dt["r"].shape, dtype=dt["r"].dtype, pin_memory=True)
        y_host.copy_(dt["y"])
        r_host.copy_(dt["r"])
        x0_host = x0.cpu().pin_memory()
        x_dev = torch.empty_like(x0)
        xo = torch.empty(plan.img_shape, pin_memory=True)
        main = torch.cuda.current_stream(dev)
        serial = how == "serial"
        cs = main if serial else torch.cuda.Stream(device=dev)
        bufs = [(dt["y"], dt["r"])] * 2 if serial else \
            [(dt["y"], dt["r"]), (torch.empty_like(dt["y"]), torch.empty_like(dt["r"]))]
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        done = [torch.cuda.Event(), torch.cuda.Event()]
        cp = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

        def issue_copy(i):
            j = i % 2
            if i >= 2 and not serial:
                cs.wait_event(done[j])  # step i - 2 has finished with this buffer set
            cp[i][0].record(cs)
            with torch.cuda.stream(cs):
                if how == "engine":
                    bufs[j][0].copy_(y_host, non_blocking=True)
                    bufs[j][1].copy_(r_host, non_blocking=True)
                else:
                    pet.copy_to_device(bufs[j][0], y_host, cblocks)
                    pet.copy_to_device(bufs[j][1], r_host, cblocks)
            cp[i][1].record(cs)
            copied[j].record(cs)

        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        if not serial:
            cs.wait_stream(main)
            issue_copy(0)
        for i in range(args.steps):
            j = i % 2
            if serial:
                issue_copy(i)
            elif i + 1 < args.steps:
                issue_copy(i + 1)
            main.wait_event(copied[j])
            plan.set_counts(*bufs[j])
            if i == 0:
                pet.copy_to_device(x_dev, x0_host)
                solver.set_image(x_dev)
            solver.run(step_len)
            done[j].record(main)
            xo.copy_(solver.image(), non_blocking=True)
        b.record(main)
        torch.cuda.synchronize()
        te = max_over_ranks(pg, a.elapsed_time(b) / 1e3, dev)
        h2d_ms = sum(c0.elapsed_time(c1) for c0, c1 in cp) / args.steps
        out["e2e"] = {"value": whole_job_rate(grads_per_step * args.steps, world, te), "unit": UNIT,
                      "h2d_bytes_per_step": int(y_host.numel() * y_host.element_size() + r_host.numel() * 4 +
                                                x0_host.numel() * 4 / args.steps),
                      "d2h_bytes_per_step": int(xo.numel() * 4), "ms_per_step": 1e3 * te / args.steps,
                      "h2d_ms_per_step": h2d_ms,
                      "h2d_gbs": (y_host.numel() * y_host.element_size() + r_host.numel() * 4) / (h2d_ms * 1e6),
                      "ingest": {"engine": "counts and background of step i + 1 copied by the copy engines on a "
                                           "second stream during step i (two device buffer sets bound by "
                                           "pet_plan_set_counts; the first copy is not hidden); the start image "
                                           "copied by pet_copy_to_device before the first step",
                                 "kernel": "as engine, with pet_copy_to_device (the copy kernel shares the SMs "
                                           f"with the step; grid bound {cblocks or 'four blocks per SM'})",
                                 "serial": "pet_copy_to_device before each step"}[how]}
        plan.set_counts(dt["y"], dt["r"])
        del bufs
        solver.kernel_time()
        del y_host, r_host
    del solver, plan
    return out


def roofline_of(cfg, p, m):
    """Roofline figures of the fused subset-gradient kernel from its live launch time."""
    peak, peak_kind = measured_peaks()
    kavg = m["kernel_ms"]
    abytes = algorithmic_bytes_per_grad(p, m["y_itemsize"])
    achieved = abytes / (kavg * 1e-3) / 1e9
    kname = kernel_name(p["geom"], m["shape"])
    tag = f"k_grad_{cfg}"
    what = "TOF forward, KL ratio, TOF backprojection" if m["T"] > 1 else "forward, KL ratio, backprojection"
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ncu_traffic(tag, kname), "kernel": f"{kname} (fused {what} of one subset)",
            "kernel_ms": kavg, "launches_timed": m["kernel_launches"], "algorithmic_bytes": abytes,
            "peak_kind": f"hbm_gbs {peak_kind}",
            "launch_shape": {"planes_per_thread": m["shape"][0], "parts_per_lor": m["shape"][1]}}
    inst = ncu_instructions(tag, kname)
    if inst is not None:
        ipeak = issue_peak()
        ach = inst / (kavg * 1e-3)
        roof["issue"] = {"achieved": ach, "peak": ipeak, "unit": "warp instructions/s", "frac": ach / ipeak,
                         "instructions_per_launch": inst, "source": "ncu smsp__inst_executed.sum"}
    return roof


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    from paper_2506_04976_gb300 import binding as pet

    if args.mode == "grad":
        return run_grad_only(args, pet, dev)
    if args.mode == "configs":
        return run_configs(args, pet, dev)
    if args.mode == "study":
        return run_study(args, pet, dev)
    if args.mode == "c4":
        return run_batched(args, pet, dev)
    if args.mode == "c5":
        return run_c5(args, pet, dev)
    if args.mode == "update":
        return run_update(args, pet, dev)
    import tempfile
    cfg = args.workload
    p, dt = load_workload(cfg, rank, dev)
    torch.cuda.synchronize()
    clk = Clocks(os.path.join(tempfile.gettempdir(), f"pet_bench_clocks_rank{rank}.csv"))
    m = measure_svrg(pet, dev, cfg, p, dt, args, rank, world, pg, e2e=not args.no_e2e, clk=clk)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        if cfg == "c5":
            cpu = oracle_sampled_rate(p)
        else:
            times = cpu_baseline(p, args.cpu_seconds)
            cpu = {"value": len(times) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{len(times)} full-size {cfg} subset gradients (fwd+back+RDP), FP64, 1 thread"}
    del dt
    other = None
    if not args.no_c2:
        ocfg = "c2" if cfg == "c5" else "c5"
        po, dto = load_workload(ocfg, rank, dev)
        mo = measure_svrg(pet, dev, ocfg, po, dto, args, rank, world, pg, e2e=False)
        other = {"workload": WORKLOADS[ocfg], "value": mo["value"], "unit": UNIT, "ms_per_step": mo["ms_per_step"],
                 "step": f"SVRG outer loop = {mo['grads_per_step']} subset gradients",
                 "roofline": roofline_of(ocfg, po, mo) if rank == 0 else None}
        del dto
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    nrmse_times = {}
    if not args.no_nrmse:
        for c in ("c1", "c2", "c2s", "c3s"):
            t = time_to_nrmse(pet, dev, c)
            if t is not None:
                nrmse_times[c] = t
    n = p["nsub"]
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[cfg],
                   "step": f"SVRG outer loop: precond update + refresh ({n}) + {2 * n - 1} inner iterations = "
                           f"{m['grads_per_step']} subset gradients",
                   "l2": "flushed between steps (256 MB write)", "graph": "one CUDA graph per epoch",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": roofline_of(cfg, p, m), "cpu_baseline": cpu, "e2e": m.get("e2e"),
        "gpu_launches": m["gpu_launches"], "clocks": clk.summary(), "wall_s_timed": m["wall_s_timed"],
        ("c2" if cfg == "c5" else "c5"): other, "time_to_1pct_nrmse": nrmse_times or None,
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
