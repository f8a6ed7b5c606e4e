"""Benchmark of the fused lattice-Boltzmann step on B300.

Headline workload: D3Q19 lid-driven cavity, 512^3 nodes, Re = 1000, lid
u = 0.1, AA single-lattice pattern, FP32 arithmetic on FP32 shifted storage.
A "step" is one time step (one fused stream-collide launch) over the whole
box.  `value` is whole-job GLUPS (nodes x steps / time / 1e9) summed over
ranks, timed with CUDA events on the launching stream; the state (10.2 GB)
is larger than L2, so no flush is needed between steps.

Besides the headline line the same JSON carries: FP16/BF16-shifted storage
and the two-lattice pull scheme on the same cavity, the D3Q27 768^3
FP16-shifted AA cavity, the adjoint/forward time ratio (D3Q19 periodic
128^3, T = 2000, K = 100), the end-to-end rate through the public API with
host buffers, the roofline of the dominant kernel and the FP64 CPU oracle's
rate on the host (a baseline only).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS & % HBM roofline (D3Q19 FP32 vs FP16-shift); adjoint/forward time ratio"
Q_OF = {"d2q9": 9, "d3q19": 19, "d3q27": 27}
BYTES_OF = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}
HEADLINE = dict(lattice="d3q19", n=512, re=1000.0, lid_u=0.1, storage="f32", aa=True,
                job_steps=2000)  # the workload is a 2000-step run


def workload_name(lattice, n, re, storage, aa):
    scheme = "AA single lattice" if aa else "two-lattice pull"
    return (f"{lattice.upper()} lid-driven cavity {n}^3, Re={re:g}, lid u=0.1, {scheme}, "
            f"{storage.upper()} storage, FP{'64' if storage == 'f64' else '32'} arithmetic")


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2201_11330_b300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, name), "rb") as fh:
                h.update(name.encode())
                h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic(kernel_tag):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel_tag and not line.startswith("#"):
            if parts[2] == want:
                return float(parts[1])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

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
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# distributed plumbing (replicas: one independent run per GPU)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_value(nodes_per_rank, steps, max_ms, world):
    """Whole-job node updates per second (GLUPS) of `world` independent
    replicas, timed by the slowest rank."""
    return world * nodes_per_rank * steps / (max_ms * 1e-3) / 1e9


def max_over_ranks(value, world, device):
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# timed runs


def timed_steps(lat, steps, warmup, world, per_launch=True):
    """Run warmup + steps single-step launches; returns total ms (max over
    ranks) and per-launch event durations split by AA parity."""
    import torch
    lat.step(warmup)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    parity = []
    barrier(world)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(steps):
        parity.append(lat.step_count % 2)
        lat.step(1)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    durs = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    total = ev[0].elapsed_time(ev[steps])
    return total, durs, parity


# rates of the MRT benchmark line (bulk, even and odd higher moments)
MRT_RATES = (1.19, 1.4, 1.2)


def make_cavity(lattice, n, re, storage, aa, lid_u=0.1, trt_lambda=None, mrt=None):
    from paper_2201_11330_b300 import workloads as W
    from paper_2201_11330_b300.lbm import Lattice
    c = W.cavity_params(n, re, lid_u)
    lat = Lattice(lattice, n, n, n, c["tau"], "cavity", storage=storage, aa=aa, lid=c["lid"],
                  trt_lambda=trt_lambda, mrt=mrt)
    lat.init()
    return lat


def run_cavity(lattice, n, re, storage, aa, steps, warmup, world, device, trt_lambda=None,
               mrt=None):
    import torch
    lat = make_cavity(lattice, n, re, storage, aa, trt_lambda=trt_lambda, mrt=mrt)
    total, durs, parity = timed_steps(lat, steps, warmup, world)
    total = max_over_ranks(total, world, device)
    N = n ** 3
    glups = replica_value(N, steps, total, world)
    bytes_per_node = 2 * Q_OF[lattice] * BYTES_OF[storage]
    out = {"glups": glups, "ms_per_step": total / steps, "bytes_per_node": bytes_per_node,
           "nodes": N}
    tag = f"{lattice}_{storage}{'_trt' if trt_lambda else ''}{'_mrt' if mrt else ''}"
    if aa:
        g = [d for d, p in zip(durs, parity) if p == 0]
        l = [d for d, p in zip(durs, parity) if p == 1]
        out["gather_ms"] = statistics.mean(g) if g else None
        out["local_ms"] = statistics.mean(l) if l else None
        out["traffic_gather"] = load_traffic(f"{tag}_gather_{n}")
        out["traffic_local"] = load_traffic(f"{tag}_local_{n}")
    else:
        out["pull_ms"] = statistics.mean(durs)
        out["traffic_pull"] = load_traffic(f"{tag}_pull_{n}")
    out["algorithmic_bytes_per_launch"] = N * bytes_per_node
    r = lat.reduce()
    out["mass_rel_drift"] = abs(r["mass"] - N) / N
    out["max_speed"] = r["max_speed"]
    del lat
    torch.cuda.empty_cache()
    return out


def run_sphere(storage, steps, warmup, world, device):
    """The paper's performance workload (Sec. 5-6): D3Q27 flow past a sphere,
    512 x 128 x 128, radius 8 at (64, 64, 64), uniform inlet 0.05 on -x,
    pressure outlet on +x, symmetry planes on y, periodic z; tau 0.53
    (Re = 80 on the diameter).  General step kernel; bytes per node update
    2 Q b + 4 (the link word)."""
    import numpy as np
    import torch
    from paper_2201_11330_b300.lbm import Lattice
    nx, ny, nz = 512, 128, 128
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    solid = ((x - 64) ** 2 + (y - 64) ** 2 + (z - 64) ** 2 <= 64).astype(np.uint8)
    lat = Lattice("d3q27", nx, ny, nz, 0.53,
                  ["inlet", "outflow", "symmetry", "symmetry", "periodic", "periodic"],
                  storage=storage, obstacles=True)
    lat.set_geometry(torch.from_numpy(solid.ravel()).to(device))
    u_in = torch.zeros((3, ny * nz), dtype=torch.float32, device=device)
    u_in[0] = 0.05
    lat.set_inlet(u_in)
    u0 = torch.zeros((3, nx * ny * nz), dtype=torch.float64, device=device)
    u0[0] = 0.05
    u0[:, torch.from_numpy(solid.ravel() != 0).to(device)] = 0
    lat.init(None, u0)
    del u0
    total, durs, _ = timed_steps(lat, steps, warmup, world)
    total = max_over_ranks(total, world, device)
    N = nx * ny * nz
    f = lat.step_force(1)
    bpn = 2 * 27 * BYTES_OF[storage] + 4
    out = {"glups": replica_value(N, steps, total, world), "ms_per_step": total / steps,
           "bytes_per_node": bpn, "nodes": N, "drag_force_x": f[0],
           "traffic_per_step": load_traffic(f"sphere_{storage}")}
    del lat
    torch.cuda.empty_cache()
    return out


def run_config_lines(world, device):
    """Device throughput on the other configurations' workloads: the 64^2
    D2Q9 cavity (FP64, Re 100, 1000 steps), the 512^2 Taylor-Green vortex
    (FP64 and FP32, tau 0.8, 5000 steps) and the 256^3 D3Q19 cavity (Re 1000,
    AA, FP32 and FP16S).  Event-timed lbm_step(n) calls (CUDA-graph replays
    where the library takes them)."""
    import torch
    from paper_2201_11330_b300 import workloads as W
    from paper_2201_11330_b300.lbm import Lattice
    out = {}

    def timed(name, lat, steps, N):
        lat.step(8)
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lat.step(steps)
        e1.record()
        torch.cuda.synchronize()
        barrier(world)
        ms = max_over_ranks(e0.elapsed_time(e1), world, device)
        out[name] = {"glups": N * steps / (ms * 1e-3) / 1e9 * world, "ms": ms, "steps": steps,
                     "us_per_step": ms * 1e3 / steps}

    c = W.cavity_params(64, 100.0, 0.1)
    lat = Lattice("d2q9", 64, 64, 1, c["tau"], "cavity", storage="f64", lid=c["lid"])
    lat.init()
    timed("d2q9_cavity64_re100_f64", lat, 1000, 64 * 64)
    p0, u0 = W.taylor_green_2d(512, 512, 0.05)
    for st in ("f64", "f32"):
        lat = Lattice("d2q9", 512, 512, 1, 0.8, "periodic", storage=st)
        lat.init(torch.from_numpy(p0).to(device), torch.from_numpy(u0).to(device))
        timed(f"d2q9_tgv512_{st}", lat, 5000, 512 * 512)
    c = W.cavity_params(256, 1000.0, 0.1)
    for st in ("f32", "f16s"):
        lat = Lattice("d3q19", 256, 256, 256, c["tau"], "cavity", storage=st, aa=True,
                      lid=c["lid"])
        lat.init()
        timed(f"d3q19_cavity256_re1000_{st}_aa", lat, 200, 256 ** 3)
    del lat
    torch.cuda.empty_cache()
    return out


def run_e2e(n, re, storage, steps, warmup, world, device, per_step_monitor=True):
    """Public API with host buffers, all inside the timed region: pinned-host
    FP32 initial fields -> device, lbm_init_f32, the steps, final FP32
    macroscopic fields -> pinned host.  per_step_monitor: every step is
    lbm_step_reduce(1) (the step with the Monitor fused in; 48 B to the host
    and a stream sync per step); else one lbm_step(steps) call and one
    lbm_reduce at the end."""
    import torch
    from paper_2201_11330_b300 import workloads as W
    from paper_2201_11330_b300.lbm import Lattice
    c = W.cavity_params(n, re, 0.1)
    N = n ** 3
    lat = Lattice("d3q19", n, n, n, c["tau"], "cavity", storage=storage, aa=True, lid=c["lid"])
    p_host = torch.full((N,), 1.0 / 3.0, dtype=torch.float32).pin_memory()
    u_host = torch.zeros((3, N), dtype=torch.float32).pin_memory()
    p_out = torch.empty((N,), dtype=torch.float32).pin_memory()
    u_out = torch.empty((3, N), dtype=torch.float32).pin_memory()
    p_dev = torch.empty((N,), dtype=torch.float32, device=device)
    u_dev = torch.empty((3, N), dtype=torch.float32, device=device)
    p_o = torch.empty((N,), dtype=torch.float32, device=device)
    u_o = torch.empty((3, N), dtype=torch.float32, device=device)
    monitor = {}

    def job(nsteps):
        p_dev.copy_(p_host, non_blocking=True)
        u_dev.copy_(u_host, non_blocking=True)
        lat.init(p_dev, u_dev)
        if per_step_monitor:
            for _ in range(nsteps):
                monitor.update(lat.step_reduce(1))
        else:
            lat.step(nsteps)
            monitor.update(lat.reduce())
        lat.macroscopic_into(p_o, u_o)
        p_out.copy_(p_o, non_blocking=True)
        u_out.copy_(u_o, non_blocking=True)
        torch.cuda.synchronize()

    job(warmup)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    job(steps)
    barrier(world)
    dt = max_over_ranks(time.perf_counter() - t0, world, device)
    h2d = (p_host.numel() + u_host.numel()) * 4
    d2h = (p_out.numel() + u_out.numel()) * 4
    mon_bytes = 48 * (steps if per_step_monitor else 1)
    how = ("per step lbm_step_reduce(1) (the step with the FP64 monitor fused in, 48 B to "
           "host and a stream sync per step)" if per_step_monitor else
           f"one lbm_step({steps}) call, then one lbm_reduce (48 B to host)")
    res = {"value": world * N * steps / dt / 1e9, "unit": "GLUPS",
           "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": (mon_bytes + d2h) / steps,
           "steps": steps, "max_speed": monitor.get("max_speed"),
           "what": f"D3Q19 cavity {n}^3 {storage} AA via paper_2201_11330_b300.lbm.Lattice: "
                   f"pinned-host FP32 initial (p, u) -> device, lbm_init_f32, {how}, "
                   "final FP32 (p, u) -> pinned host"}
    del lat
    torch.cuda.empty_cache()
    return res


def run_adjoint(n, T, K, world, device, warmup=1, reps=3):
    """Adjoint/forward time ratio on the periodic box with a Fourier force.

    One untimed adjoint run first (the adjoint kernels' first launches and the
    workspace allocation stay out of the timing), then `reps` repetitions of
    the plain forward, the checkpointed forward and the backward; each time is
    the median over the repetitions."""
    import torch
    from paper_2201_11330_b300 import workloads as W
    from paper_2201_11330_b300.lbm import Lattice
    F = torch.from_numpy(W.fourier_force(n, n, n, amplitude=1e-5, seed=2201)).to(device)
    lat = Lattice("d3q19", n, n, n, 0.8, "periodic", storage="f32", aa=False, has_force=True)
    lat.set_force(F)
    lat.init()
    lat.step(warmup)
    lat.init()
    lat.adjoint_forward(T, K)
    lat.adjoint_backward()
    fwd, fwd_ck, bwd = [], [], []
    for _ in range(reps):
        lat.init()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.step(T)
        torch.cuda.synchronize()
        fwd.append(time.perf_counter() - t0)
        lat.init()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J = lat.adjoint_forward(T, K)
        fwd_ck.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        g, gU = lat.adjoint_backward()
        torch.cuda.synchronize()
        bwd.append(time.perf_counter() - t0)
        del g
    t_fwd, t_fwd_ck, t_bwd = (statistics.median(v) for v in (fwd, fwd_ck, bwd))
    res = {"config": f"D3Q19 periodic {n}^3 FP32, Fourier force A=1e-5 seed 2201, T={T}, K={K}",
           "forward_s": t_fwd, "forward_checkpointed_s": t_fwd_ck, "backward_s": t_bwd,
           "ratio": t_bwd / t_fwd, "J": J, "reps": reps,
           "ratio_definition": "backward (recompute + adjoint steps) time / plain forward time, "
                               "medians over reps after one untimed adjoint run"}
    del lat
    torch.cuda.empty_cache()
    return res


def cpu_baseline_sample(target_s=12.0):
    """The FP64 oracle, as it stands, on this host's cores: D3Q19 cavity at
    the headline tau on a 96^3 box, enough steps for ~target_s seconds."""
    import oracle
    from paper_2201_11330_b300 import workloads as W
    c = W.cavity_params(HEADLINE["n"], HEADLINE["re"], HEADLINE["lid_u"])
    n = 96
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.run("d3q19", n, n, n, c["tau"], "cavity", 1, lid=c["lid"], threads=cores)
    t1 = time.perf_counter() - t0
    steps = max(2, int(target_s / max(t1, 1e-3)))
    t0 = time.perf_counter()
    oracle.run("d3q19", n, n, n, c["tau"], "cavity", steps, lid=c["lid"], threads=cores)
    dt = time.perf_counter() - t0
    out = {"value": n ** 3 * steps / dt / 1e9, "unit": "GLUPS", "cores": cores,
           "kind": "oracle",
           "sample": f"D3Q19 cavity {n}^3 at the 512^3 workload's tau={c['tau']}, {steps} steps "
                     f"(init + steps + moments timed), {dt:.1f} s, OpenMP threads={cores}"}
    # the oracle on the other configurations' shapes (a few seconds in all)
    cfg = {}

    def timed(name, threads, *a, **kw):
        t0 = time.perf_counter()
        oracle.run(*a, threads=threads, **kw)
        dt = time.perf_counter() - t0
        nx, ny, nz, steps = a[1], a[2], a[3], a[6]
        cfg[name] = {"mlups": nx * ny * nz * steps / dt / 1e6, "threads": threads,
                     "steps": steps, "s": round(dt, 3)}

    c64 = W.cavity_params(64, 100.0, 0.1)
    timed("d2q9_cavity64_re100", cores, "d2q9", 64, 64, 1, c64["tau"], "cavity", 1000,
          lid=c64["lid"])
    p0, u0 = W.taylor_green_2d(512, 512, 0.05)
    timed("d2q9_tgv512", cores, "d2q9", 512, 512, 1, 0.8, "periodic", 20, p0=p0, u0=u0)
    c3 = W.cavity_params(64, 1000.0, 0.1)
    for threads in (1, cores):
        timed(f"d3q19_cavity64_re1000_threads{threads}", threads, "d3q19", 64, 64, 64, c3["tau"],
              "cavity", 10, lid=c3["lid"])
    out["configs"] = cfg
    return out


# ---------------------------------------------------------------------------


def reference_arm(args, world, rank):
    """Oracle arm: each step is a bounded sample of the headline workload."""
    if rank != 0:
        return 0
    import oracle
    from paper_2201_11330_b300 import workloads as W
    c = W.cavity_params(HEADLINE["n"], HEADLINE["re"], HEADLINE["lid_u"])
    n, sub = 64, 2
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.run("d3q19", n, n, n, c["tau"], "cavity", sub, lid=c["lid"], threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run("d3q19", n, n, n, c["tau"], "cavity", sub, lid=c["lid"], threads=cores)
    dt = time.perf_counter() - t0
    value = n ** 3 * sub * args.steps / dt / 1e9
    sample = (f"each step: FP64 oracle D3Q19 cavity {n}^3 at the 512^3 workload's "
              f"tau={c['tau']}, {sub} time steps incl. init and moments")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(**{k: HEADLINE[k] for k in
                                                    ("lattice", "n", "re", "storage", "aa")}),
                       "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--size", type=int, default=HEADLINE["n"],
                    help="cavity side of the headline run (profiling uses smaller boxes)")
    ap.add_argument("--storage", default=HEADLINE["storage"], choices=list(BYTES_OF),
                    help="storage of the headline run (profiling of the other variants)")
    ap.add_argument("--lattice", default=HEADLINE["lattice"], choices=["d3q19", "d3q27"],
                    help="lattice of the headline run (profiling of the D3Q27 kernels)")
    ap.add_argument("--pull", action="store_true",
                    help="two-lattice pull scheme for the headline run (profiling)")
    ap.add_argument("--trt", action="store_true",
                    help="two-relaxation-time collision (Lambda = 3/16) for the headline run "
                         "(profiling)")
    ap.add_argument("--mrt", action="store_true",
                    help="multiple-relaxation-time collision (rates MRT_RATES) for the headline "
                         "run (profiling)")
    ap.add_argument("--e2e", action="store_true",
                    help="with --no-extras: still run the two end-to-end legs (profiling)")
    ap.add_argument("--workload", default="cavity", choices=["cavity", "sphere"],
                    help="sphere: only the paper's D3Q27 sphere flow at --storage (profiling)")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline line only, for profiling (no storage variants, D3Q27, "
                         "adjoint, end-to-end legs, CPU)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init(world, "nccl")
    from paper_2201_11330_b300 import build
    if rank == 0:
        build.build()
    barrier(world)

    if args.workload == "sphere":
        r = run_sphere(args.storage, args.steps, args.warmup, world, device)
        if rank == 0:
            print(json.dumps({"workload": "D3Q27 sphere 512x128x128", "storage": args.storage,
                              "steps": args.steps, "warmup": args.warmup, **r}))
        return 0

    hb = dict(HEADLINE)
    hb["n"] = args.size
    hb["storage"] = args.storage
    hb["lattice"] = args.lattice
    hb["aa"] = not args.pull
    if args.lattice == "d3q27":  # the D3Q27 cavity is quoted at Re 2000
        hb["re"] = 2000.0
    peak, peak_kind = load_peaks()

    # headline, with clocks sampled during its timed region
    sampler = ClockSampler(local)
    sampler.start()
    head = run_cavity(hb["lattice"], hb["n"], hb["re"], hb["storage"], hb["aa"], args.steps,
                      args.warmup, world, device, trt_lambda=3 / 16 if args.trt else None,
                      mrt=MRT_RATES if args.mrt else None)
    clocks = sampler.stop()

    N = head["nodes"]
    bpn = head["bytes_per_node"]
    st_tag = hb["storage"].upper()
    lat_tag = hb["lattice"].upper()
    if hb["aa"]:
        dom_ms = max(head["gather_ms"], head["local_ms"])
        gather_dom = head["gather_ms"] >= head["local_ms"]
        pat = "GATHER" if gather_dom else "LOCAL"
    else:
        dom_ms = head["pull_ms"]
        pat = "PULL"
    dom_name = f"k_step<{lat_tag},{st_tag},{pat}>"
    achieved = N * bpn / (dom_ms * 1e-3) / 1e9
    traffic = load_traffic(f"{hb['lattice']}_{hb['storage']}{'_trt' if args.trt else ''}"
                           f"{'_mrt' if args.mrt else ''}_"
                           f"{pat.lower()}_{hb['n']}")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": dom_name, "peak_kind": f"{peak_kind} copy bandwidth",
                "algorithmic_bytes_per_launch": N * bpn,
                "gather_ms": head.get("gather_ms"), "local_ms": head.get("local_ms"),
                "pull_ms": head.get("pull_ms"),
                "frac_of_8TBs": N * bpn / (dom_ms * 1e-3) / 8e12}

    extras = {}
    if not args.no_extras:
        for st in ("f16s", "bf16s"):
            r = run_cavity("d3q19", hb["n"], hb["re"], st, True, args.steps, args.warmup, world,
                           device)
            r["hbm_frac"] = r["glups"] / world * r["bytes_per_node"] / peak
            extras[f"d3q19_{st}_aa"] = r
        r = run_cavity("d3q19", hb["n"], hb["re"], "f32", False, args.steps, args.warmup, world,
                       device)
        r["hbm_frac"] = r["glups"] / world * r["bytes_per_node"] / peak
        extras["d3q19_f32_pull"] = r
        for st in ("f32", "f16s"):  # two-relaxation-time collision, Lambda = 3/16
            r = run_cavity("d3q19", hb["n"], hb["re"], st, True, args.steps, args.warmup, world,
                           device, trt_lambda=3 / 16)
            r["hbm_frac"] = r["glups"] / world * r["bytes_per_node"] / peak
            extras[f"d3q19_{st}_aa_trt"] = r
        # multiple-relaxation-time collision, FP32 storage
        r = run_cavity("d3q19", hb["n"], hb["re"], "f32", True, args.steps, args.warmup, world,
                       device, mrt=MRT_RATES)
        r["hbm_frac"] = r["glups"] / world * r["bytes_per_node"] / peak
        extras["d3q19_f32_aa_mrt"] = r
        n27 = 768 if hb["n"] == 512 else hb["n"]
        r = run_cavity("d3q27", n27, 2000.0, "f16s", True, max(10, args.steps // 4),
                       args.warmup, world, device)
        r["hbm_frac"] = r["glups"] / world * r["bytes_per_node"] / peak
        extras["d3q27_f16s_aa_768"] = r
        for st in ("f64", "f32", "f16s"):
            r = run_sphere(st, max(10, args.steps // 2), args.warmup, world, device)
            r["hbm_frac"] = r["glups"] / world * r["bytes_per_node"] / peak
            extras[f"sphere_d3q27_512x128x128_{st}"] = r
        extras["configs"] = run_config_lines(world, device)
        try:
            extras["adjoint"] = run_adjoint(128, 2000, 100, world, device)
        except Exception as exc:  # reported, not hidden
            extras["adjoint"] = {"error": str(exc)}
    # end to end through the public API, the whole job of the workload (its
    # 2000 steps, with the host copies of its initial and final fields): the
    # contract's per-step metric read, and the stepping call with one monitor
    # read at the end
    e2e = e2e_step_n = None
    if not args.no_extras or args.e2e:
        e2e_steps = max(HEADLINE["job_steps"], args.steps)
        e2e = run_e2e(hb["n"], hb["re"], hb["storage"], e2e_steps, args.warmup, world, device)
        e2e_step_n = run_e2e(hb["n"], hb["re"], hb["storage"], e2e_steps, args.warmup, world,
                             device, per_step_monitor=False)

    cpu = cpu_baseline_sample() if (rank == 0 and world == 1 and not args.no_extras) else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["glups"], "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if hb["storage"] == "f64" else "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(hb["lattice"], hb["n"], hb["re"], hb["storage"],
                                                 hb["aa"]),
                       "nodes_per_gpu": N, "parallelism": f"replicas x{world}",
                       "l2": "state larger than L2 (no flush needed)"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "e2e_step_n": e2e_step_n,
            "gpu_launches": args.steps,
            "clocks": clocks,
            "mass_rel_drift": head["mass_rel_drift"],
        }
        line.update(extras)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
