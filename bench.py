"""Benchmark: one Lambda iteration of the NLTE problem on the 128^3 regular grid, plus the
irregular-grid workloads.

A step is one pass of the whole hot path: opacity and source function from the populations
(52 wavelengths), the formal solution over 24 directions by short characteristics with J
accumulated over angles, rates and statistical equilibrium, and the convergence read-back.
Metric: point x direction x wavelength updates per second of the step (Gupd/s).

The same JSON line carries the Voronoi-grid measurements (8 atmospheres of 50k-400k sites batched
against plain per-direction launches, seconds per Lambda iteration on the 215k-site grid), the
time to convergence on both grids, the adjoint of the mu = 1 map, and the accuracy of the
32 x 32 x 64 regular and 20k-site Voronoi maps against the 128 x 128 x 256 fine grid.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--extras]
                    [--no-voronoi] [--no-cpu]

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
--extras adds the final synthesis, the small LTE continuum workloads and the accelerated and
Ng-extrapolated iterations.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = NZ = 128
NDIR = 24
SCHEME = "plane"          # regular-grid short characteristics: "plane" or "face"
WORKLOAD = "NLTE Lambda iteration, regular grid 128x128x128, 52 wavelengths, 24 directions"

# DRAM bytes from the ncu captures summarised in profiles/, valid only for the kernel source with
# this hash (kernel_hash: comments and blank lines ignored; else reported as null)
PROFILED_FILE = "paper_2306_01041_gb300/csrc/regular_tile.cu"
PROFILED = {"sc_pipe_kernel": {"file": "paper_2306_01041_gb300/csrc/regular_pipe.cu",
                               "sha1": "d7bff69764e8aa185027c743d3925766b68b993f",
                               "dram_bytes_per_launch": 5.049951488e9 + 14.094347520e9},
            "sc_wave_kernel": {"file": PROFILED_FILE, "sha1": None, "dram_bytes_per_launch": None},
            "sc_tile_kernel": {"file": PROFILED_FILE, "sha1": None, "dram_bytes_per_launch": None},
            "batch_sweep_kernel": {"file": "paper_2306_01041_gb300/csrc/batch.cu",
                                   "sha1": "15c9bee6f032c97d7e7092c3ed8c86d5a5fc8775",
                                   # measured on the first two atmospheres (146 M updates; the
                                   # 8-atmosphere launch is larger than a capture should hold),
                                   # per update, scaled to the launch by its updates
                                   "dram_bytes_per_update": (1.350062e9 + 0.619866e9) / 146.016e6},
            "face_sweep_kernel": {"file": "paper_2306_01041_gb300/csrc/regular_face.cu",
                                  "sha1": "09789e460a0a787c6dc7550acd0ed83fea06e619",
                                  "dram_bytes_per_launch": 25.295442176e9 + 10.433180160e9}}

# Algorithmic FP32 work of one point-direction-wavelength update of the regular sweep, counted in
# lane operations (an FMA counts once): three bilinear interpolations (6 each), dtau (2), interval
# weights (4), intensity (3 FMA) and J (1 FMA); plus two SFU operations (exp, reciprocal) not
# counted.  The bound is one lane operation per FP32 lane per cycle:
# 152 SMs x 128 lanes x 2070 MHz.
OPS_PER_UPDATE = 28
SM_COUNT, LANES, SM_MHZ_MAX = 152, 128, 2070.0
ALU_PEAK_TOPS = SM_COUNT * LANES * SM_MHZ_MAX * 1e6 / 1e12
# Compulsory HBM bytes of one update of the batched Voronoi sweep at 52 wavelengths: alpha, S and
# J per (site, wavelength) over 24 directions, the upwind records over the wavelengths, and the
# intensity written once and gathered twice.
VOR_BYTES_PER_UPDATE = (12.0 + 24.0 * 24.0 / 52.0) / 24.0 + 4.0
PEAKS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")


def hbm_peak():
    """Measured copy bandwidth of the GB300s (GB/s), else the fallback figure."""
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def max_over_ranks(value, device=None):
    """The largest value over the ranks of the default process group (the timed region of the
    slowest replica); the value itself without a group or with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def setup_problem(torch, dev, z_stretch=0.0):
    from synth import make_atmosphere, model_atom, s4_quadrature
    from synth.atmosphere import regular_fields
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(NX, NY, NZ, atm)
    if z_stretch:
        # non-uniform z: u -> u - a sin(2 pi u) / (2 pi), cell heights (1 -+ a) times uniform
        u = (np.arange(NZ) + 0.5) / NZ
        z = atm.zmin + (atm.zmax - atm.zmin) * (u - z_stretch * np.sin(2 * np.pi * u) / (2 * np.pi))
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        f = {k: v.reshape(-1) for k, v in atm.fields(X, Y, Z).items()}
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    dirs, w = s4_quadrature()
    return atm, f, (x, y, z, dx, dy), data, dirs, w


def kernel_hash(path=PROFILED_FILE):
    """SHA-1 of a source file without its // comments and blank lines: what a capture of the
    kernel's counters stays valid for."""
    with open(os.path.join(ROOT, path), encoding="utf-8") as fh:
        lines = [ln.split("//", 1)[0].rstrip() for ln in fh]
    return hashlib.sha1("\n".join(ln for ln in lines if ln).encode()).hexdigest()


def run_gpu(args):
    import torch
    import paper_2306_01041_gb300 as rt

    rank, world, local = _env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    atm, f, (x, y, z, dx, dy), data, dirs, w = setup_problem(torch, dev, args.z_stretch)
    g = rt.RegularGrid(NX, NY, NZ, dx, dy, z, dirs, w, scheme=args.scheme)
    atom = rt.Atom(data, atm.kappa0)
    nlam = atom.nlam
    npt = NX * NY * NZ
    host = {k: torch.tensor(f[k], dtype=torch.float32).pin_memory() for k in ("T", "rho", "ne", "nH")}
    dvc = {k: v.to(dev) for k, v in host.items()}
    atmos = rt.Atmos(dvc["T"], dvc["rho"], dvc["ne"], dvc["nH"])
    pops0 = rt.lte_populations(g, atom, atmos)
    pops = pops0.clone()
    stream = torch.cuda.current_stream()
    alpha = torch.empty((nlam, npt), device=dev)
    S = torch.empty_like(alpha)
    J = torch.empty_like(alpha)

    # One Lambda iteration = source terms -> formal solution (+ J) -> statistical equilibrium ->
    # read-back of max |dn/n|.  The device part is captured once as a CUDA graph and replayed.
    dmax_host = torch.zeros(1, dtype=torch.float32).pin_memory()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def src(st):
        rt.source_terms(g, atom, atmos, pops, stream=st, out=(alpha, S))

    def fs(st):
        rt.formal_solution(g, alpha, S, J=J, stream=st)

    def se(st):
        d = rt.statistical_equilibrium(g, atom, atmos, J, pops, stream=st)
        dmax_host.copy_(d, non_blocking=True)

    # three graphs so that the formal solution can be timed with events between replays
    cap = torch.cuda.Stream(device=dev)
    cap.wait_stream(torch.cuda.current_stream())
    graphs = []
    with torch.cuda.stream(cap):
        for part in (src, fs, se):
            part(cap)                  # allocates the library's scratch before capture
        cap.synchronize()
        launches = []               # library kernel launches recorded into each graph
        for part in (src, fs, se):
            gr = torch.cuda.CUDAGraph()
            n0 = rt.kernel_launches()
            with torch.cuda.graph(gr, stream=cap):
                part(cap)
            launches.append(rt.kernel_launches() - n0)
            graphs.append(gr)
    torch.cuda.current_stream().wait_stream(cap)
    stream = torch.cuda.current_stream()
    fs_times = []

    part_times = []

    def step(record=False):
        ev[2].record(stream)
        graphs[0].replay()
        ev[0].record(stream)
        graphs[1].replay()
        ev[1].record(stream)
        graphs[2].replay()
        ev[3].record(stream)
        stream.synchronize()           # the convergence read-back
        if record:
            fs_times.append(ev[0].elapsed_time(ev[1]))
            part_times.append((ev[2].elapsed_time(ev[0]), ev[1].elapsed_time(ev[3])))
        return float(dmax_host.item())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        step(record=True)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    clk = clocks.stop()
    ms = max_over_ranks(ms, dev)
    updates = npt * NDIR * nlam
    value = updates * world / (ms * 1e-3) / 1e9
    fs_ms = statistics.mean(fs_times)
    # the formal-solution graph is one persistent wavefront launch (sc_pipe_kernel on periodic
    # grids whose tiles its staging covers, else sc_wave_kernel) or, when neither applies, one
    # launch per plane step and hemisphere (sc_tile_kernel) plus the two boundary planes; the
    # achieved rate is the interior updates over the graph's event time
    interior_ops = OPS_PER_UPDATE * NX * NY * (NZ - 1) * NDIR * nlam
    if args.scheme == "face":
        # face_sweep_kernel, then the J pass over the planes it kept (face_j_kernel)
        kname, per_launch_ms = "face_sweep_kernel", fs_ms
    elif launches[1] == 1:
        kname = ("sc_wave_kernel" if os.environ.get("RT_REGULAR_SWEEP", "pipe") != "pipe"
                 else "sc_pipe_kernel")
        per_launch_ms = fs_ms
    else:
        kname, per_launch_ms = "sc_tile_kernel", fs_ms / (2 * (NZ - 1))
    achieved = interior_ops / (fs_ms * 1e-3) / 1e12
    traffic = None
    prof = PROFILED.get(kname)
    if prof and prof["sha1"] == kernel_hash(prof["file"]) and prof["dram_bytes_per_launch"]:
        traffic = prof["dram_bytes_per_launch"]

    # end to end through the public API with host buffers: H2D of the step's inputs (atmosphere
    # and populations), the iteration, D2H of the new populations and the convergence scalar
    pops_host = pops0.cpu().pin_memory()
    out_host = torch.empty_like(pops_host).pin_memory()
    for _ in range(2):
        for k in dvc:
            dvc[k].copy_(host[k], non_blocking=True)
        pops.copy_(pops_host, non_blocking=True)
        step()
        out_host.copy_(pops, non_blocking=True)
    torch.cuda.synchronize()
    e_steps = max(1, min(args.steps, 5))
    te0 = time.perf_counter()
    for _ in range(e_steps):
        for k in dvc:
            dvc[k].copy_(host[k], non_blocking=True)
        pops.copy_(pops_host, non_blocking=True)
        step()
        out_host.copy_(pops, non_blocking=True)
        torch.cuda.synchronize()
    e_ms = (time.perf_counter() - te0) * 1e3 / e_steps
    h2d = sum(v.numel() * 4 for v in host.values()) + pops_host.numel() * 4
    d2h = out_host.numel() * 4 + 4

    res = {
        "metric": "formal-solution Gupdates/s (pt*dir*lambda), NLTE Lambda iteration",
        "value": round(value, 3), "unit": "Gupd/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [NX, NY, NZ], "wavelengths": nlam,
                   "directions": NDIR, "updates_per_step": updates,
                   "l2": "inputs larger than L2 (alpha, S, J: 3 x 436 MB per step)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(updates / (e_ms * 1e-3) / 1e9, 3), "unit": "Gupd/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * sum(launches),
        "launches_per_step": {"source_terms": launches[0], "formal_solution": launches[1],
                              "statistical_equilibrium": launches[2]},
        "roofline": {"bound": "alu", "kernel": kname,
                     "achieved": round(achieved, 3), "peak": round(ALU_PEAK_TOPS, 2),
                     "unit": "TFLOP/s", "frac": round(achieved / ALU_PEAK_TOPS, 4),
                     "traffic": traffic,
                     "per_launch_ms": round(per_launch_ms, 5),
                     "formal_solution_ms": round(fs_ms, 3),
                     "interior_gupd_s": round(interior_ops / OPS_PER_UPDATE / fs_ms / 1e6, 2),
                     "peak_note": "28 FP32 lane operations per update (an FMA counts once) "
                                  "against one per lane per cycle: 152 SMs x 128 lanes x "
                                  "2070 MHz, derived from unit counts and the maximum clock"},
        "clocks": clk,
        "breakdown_ms": {"source_terms": round(statistics.mean(p[0] for p in part_times), 3),
                         "formal_solution": round(fs_ms, 3),
                         "statistical_equilibrium": round(statistics.mean(p[1] for p in part_times), 3)},
    }
    if not args.no_voronoi:
        work = {s: (g, f, k0) for s, g, f, k0 in voronoi_workload()}
        vclk = ClockSampler(local)
        vclk.start()
        res["voronoi"] = run_voronoi(torch, rt, dev, work)
        res["voronoi"]["clocks"] = vclk.stop()
        res["convergence"], conv_pops = convergence_times(torch, rt, dev, work)
        res["adjoint"] = adjoint_timings(torch, rt, dev, work, conv_pops)
        res["accuracy"] = accuracy_maps(torch, rt, dev, work)
    if args.extras:
        res["extras"] = run_extras(torch, rt, dev, None if args.no_voronoi else work)
    if rank == 0 and not args.no_cpu:
        res["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()


CPU_N = 64          # the oracle's sample: full Lambda iterations on the 64^3 grid


class OracleIteration:
    """The oracle's Lambda iteration as it stands (source terms, formal solution over 24
    directions, rates, statistical equilibrium; 52 wavelengths) on the n^3 grid of the
    benchmark's atmosphere, from LTE populations."""

    def __init__(self, n):
        import oracle
        from oracle.physics import Atom
        from oracle.solve import RegularGrid as OrcRegular
        from synth import make_atmosphere, model_atom, s4_quadrature
        from synth.atmosphere import regular_fields
        atm = make_atmosphere(0)
        self.f, (x, y, z, dx, dy) = regular_fields(n, n, n, atm)
        data = model_atom(np.min(self.f["ne"] / np.sqrt(self.f["T"])))
        self.A = Atom(data, atm.kappa0)
        dirs, w = s4_quadrature()
        self.g = OrcRegular(n, n, n, dx, dy, z, dirs, w, scheme=SCHEME)
        self.pops = self.A.lte_pops(self.f["T"], self.f["ne"], self.f["nH"])
        self.nlam = len(data["lam"])
        self.updates = n ** 3 * NDIR * self.nlam
        self.cores = oracle.num_threads()

    def step(self):
        """One iteration; returns its wall time in seconds."""
        f, A = self.f, self.A
        t = time.perf_counter()
        alpha, S = A.alpha_S(f["T"], f["rho"], f["ne"], self.pops)
        J = self.g.formal_solution(alpha, S)
        self.pops = A.statistical_equilibrium(A.rate_matrix(f["T"], f["ne"], J), f["nH"])
        return time.perf_counter() - t


def _cpu_sample_text(n, nlam, cores, reps):
    scheme = ", face-hitting short characteristics" if SCHEME == "face" else ""
    return (f"{'mean of ' + str(reps) + ' ' if reps > 1 else 'one '}full Lambda "
            f"iteration{'s' if reps > 1 else ''} of the oracle (source terms, formal solution, "
            f"rates, statistical equilibrium; {nlam} wavelengths, 24 directions{scheme}) on the "
            f"{n}^3 grid of the same atmosphere from LTE; its C sweep on {cores} OpenMP "
            f"thread{'s' if cores > 1 else ''}, the atom's numpy arithmetic on one core")


def cpu_one_thread(n):
    """One oracle iteration in a subprocess with OMP_NUM_THREADS=1."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-iteration", str(n),
           "--scheme", SCHEME]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        return {"error": (r.stderr or r.stdout).strip().splitlines()[-1:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline():
    """The oracle on this host's cores: the mean of three full Lambda iterations on the 64^3 grid
    (all cores), and one on a single thread."""
    n = min(CPU_N, NX)
    it = OracleIteration(n)
    sec = statistics.mean(it.step() for _ in range(3))
    return {"value": round(it.updates / sec / 1e9, 5), "unit": "Gupd/s", "cores": it.cores,
            "kind": "oracle", "seconds_per_iteration": round(sec, 2),
            "sample": _cpu_sample_text(n, it.nlam, it.cores, 3),
            "one_thread": cpu_one_thread(n)}


def run_cpu_iteration(args):
    it = OracleIteration(args.cpu_iteration)
    sec = it.step()
    print(json.dumps({"value": round(it.updates / sec / 1e9, 5), "unit": "Gupd/s",
                      "cores": it.cores, "seconds_per_iteration": round(sec, 2),
                      "sample": _cpu_sample_text(args.cpu_iteration, it.nlam, it.cores, 1)}))


def run_reference(args):
    rank, world, local = _env_rank()
    if rank != 0:
        return
    n = min(CPU_N, NX)
    it = OracleIteration(n)
    for _ in range(args.warmup):
        it.step()
    secs = [it.step() for _ in range(args.steps)]
    sec = statistics.mean(secs)
    v = it.updates / sec / 1e9
    res = {"impl": "reference",
           "metric": "formal-solution Gupdates/s (pt*dir*lambda), NLTE Lambda iteration",
           "value": round(v, 5), "unit": "Gupd/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "grid": [NX, NY, NZ], "wavelengths": it.nlam,
                      "directions": NDIR, "parallelism": "host cores (OpenMP)",
                      "sample_grid": [n] * 3},
           "cpu_baseline": {"value": round(v, 5), "unit": "Gupd/s", "cores": it.cores,
                            "kind": "oracle",
                            "sample": _cpu_sample_text(n, it.nlam, it.cores, args.steps)},
           "e2e": {"value": round(v, 5), "unit": "Gupd/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


VOR_SIZES = [50000, 67000, 90000, 120000, 160000, 215000, 290000, 400000]


def _make_vor(args):
    """One Voronoi grid of the workloads: site seed s, size n; seeds 1-8 are the batched
    atmospheres (odd rho^0.3, even |dtau/dz|), later seeds use atmosphere 0 and |dtau/dz|."""
    s, n = args
    sys.path.insert(0, ROOT)
    from synth import make_atmosphere, make_voronoi_grid
    atm = make_atmosphere(s if s <= 8 else 0)
    g = make_voronoi_grid(atm, n, "rho03" if (s <= 8 and s % 2) else "dtau", s)
    f = atm.fields(g["xyz"][:, 0], g["xyz"][:, 1], g["xyz"][:, 2])
    return s, g, f, atm.kappa0


def voronoi_workload(sizes=VOR_SIZES, extra=((9, 200000), (10, 20000))):
    """The 8 batched atmospheres (seeds 1-8), plus the 200k-site adjoint grid and the 20k-site LTE
    continuum grid (site seeds 9 and 10, atmosphere seed 0, density from |dtau/dz|), built in
    parallel on the host cores."""
    import multiprocessing as mp
    jobs = list(zip(range(1, len(sizes) + 1), sizes)) + list(extra)
    jobs.sort(key=lambda j: -j[1])              # largest first: the pool finishes sooner
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        return pool.map(_make_vor, jobs, chunksize=1)


def _vgrid(rt, g, dirs, w):
    return rt.VoronoiGrid(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"], dirs, w)


def _atmos(torch, rt, f, dev):
    return rt.Atmos(*[torch.tensor(np.ascontiguousarray(f[k]), dtype=torch.float32, device=dev)
                      for k in ("T", "rho", "ne", "nH")])


def run_voronoi(torch, rt, dev, work):
    """8 atmospheres on Voronoi grids of 50k-400k sites (1.39M), 52 wavelengths, 24 directions:
    plain per-direction, per-level launches against one persistent all-direction launch per grid
    and against the batched persistent sweep of all grids; the batched Lambda iteration as one
    CUDA graph per iteration; seconds per Lambda iteration on the 215k-site grid alone."""
    from paper_2306_01041_gb300.autotune import tune_batch
    from synth import make_atmosphere, model_atom, s4_quadrature
    dirs, w = s4_quadrature()
    seeds = sorted(s for s in work if s <= 8)
    grids = [_vgrid(rt, work[s][0], dirs, w) for s in seeds]
    fs = [work[s][1] for s in seeds]
    # one model atom for the batch: the collisional scale from the smallest n_e / sqrt(T) of all
    # eight atmospheres, the background opacity scale of the recipe's base atmosphere
    data = model_atom(min(np.min(f["ne"] / np.sqrt(f["T"])) for f in fs))
    atom = rt.Atom(data, make_atmosphere(0).kappa0)
    atms = [_atmos(torch, rt, f, dev) for f in fs]
    pops0 = [rt.lte_populations(G, atom, M) for G, M in zip(grids, atms)]
    alphas, Ss = [], []
    for G, M, p in zip(grids, atms, pops0):
        a, sv = rt.source_terms(G, atom, M, p)
        alphas.append(a)
        Ss.append(sv)
    nlam = atom.nlam
    upd = sum(G.npt for G in grids) * NDIR * nlam
    Jp = [torch.empty_like(a) for a in alphas]
    os.environ["RT_VORONOI_SWEEP"] = "levels"      # plain per-direction, per-level launches
    try:
        ms_plain = _events(torch, lambda: [rt.formal_solution(G, a, sv, J=j)
                                           for G, a, sv, j in zip(grids, alphas, Ss, Jp)])
    finally:
        del os.environ["RT_VORONOI_SWEEP"]
    Js = [torch.empty_like(a) for a in alphas]      # one persistent launch per grid, in turn
    ms_single = _events(torch, lambda: [rt.formal_solution(G, a, sv, J=j)
                                        for G, a, sv, j in zip(grids, alphas, Ss, Js)])
    batch, choice = tune_batch(grids, alphas, Ss, nlam)
    Jb = [torch.empty_like(a) for a in alphas]
    ms_batch = _events(torch, lambda: batch.formal_solution(alphas, Ss, Js=Jb), reps=5)
    diff = max(float(((b - p).abs() / p.abs().clamp_min(1e-30)).max()) for b, p in zip(Jb, Jp))
    # the batched Lambda iteration, one CUDA graph per iteration (host-timed, with the read-back
    # of the convergence scalar every iteration)
    pops = [p.clone() for p in pops0]
    batch.lambda_iterate(atom, atms, pops, max_iter=1, tol=0.0)   # graph capture and scratch
    for q, p in zip(pops, pops0):
        q.copy_(p)
    torch.cuda.synchronize()
    t = time.perf_counter()
    it, hist, _ = batch.lambda_iterate(atom, atms, pops, max_iter=5, tol=0.0)
    s_batch_iter = (time.perf_counter() - t) / it
    # the 215k-site grid alone (its own atmosphere's atom)
    k215 = seeds.index(6)
    G6, f6 = grids[k215], fs[k215]
    A6 = rt.Atom(model_atom(np.min(f6["ne"] / np.sqrt(f6["T"]))), work[6][2])
    M6 = atms[k215]
    p6 = rt.lte_populations(G6, A6, M6)
    rt.lambda_iterate(G6, A6, M6, p6, max_iter=1, tol=0.0)
    p6 = rt.lte_populations(G6, A6, M6)
    torch.cuda.synchronize()
    t = time.perf_counter()
    it6, _, _ = rt.lambda_iterate(G6, A6, M6, p6, max_iter=5, tol=0.0)
    s_iter_215 = (time.perf_counter() - t) / it6
    peak, peak_src = hbm_peak()
    achieved = VOR_BYTES_PER_UPDATE * upd / (ms_batch * 1e-3) / 1e9
    traffic = None
    prof = PROFILED.get("batch_sweep_kernel")
    if prof and prof["sha1"] == kernel_hash(prof["file"]) and prof["dram_bytes_per_update"]:
        traffic = prof["dram_bytes_per_update"] * upd
    return {
        "workload": "8 atmospheres on Voronoi grids (sites from rho^0.3 and |dtau/dz|), one model "
                    "atom, 52 wavelengths, 24 directions, populations at LTE",
        "atmospheres": len(grids), "sites": [G.npt for G in grids],
        "levels_max": [G.max_levels for G in grids], "updates_per_formal_solution": upd,
        "plain_ms": round(ms_plain, 3), "plain_gupd_s": round(upd / ms_plain / 1e6, 3),
        "per_grid_persistent_ms": round(ms_single, 3),
        "per_grid_persistent_gupd_s": round(upd / ms_single / 1e6, 3),
        "batched_ms": round(ms_batch, 3), "batched_gupd_s": round(upd / ms_batch / 1e6, 3),
        "speedup_batched_vs_plain": round(ms_plain / ms_batch, 2),
        "max_rel_diff_batched_vs_plain": diff, "autotuned": choice,
        "batched_lambda_iteration_s": round(s_batch_iter, 5),
        "batched_lambda_iteration_note": "rt_batch_lambda_iterate, one CUDA graph per iteration, "
                                         "host wall time per iteration including the read-back",
        "grid_215k": {"sites": G6.npt, "levels_max": G6.max_levels,
                      "s_per_lambda_iteration": round(s_iter_215, 5),
                      "gupd_s": round(G6.npt * NDIR * nlam / s_iter_215 / 1e9, 3)},
        "roofline": {"bound": "hbm", "kernel": "batch_sweep_kernel",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "bytes_per_update": round(VOR_BYTES_PER_UPDATE, 3),
                     "note": f"compulsory bytes per update x updates / event time of the whole "
                             f"batched formal solution (transposes, sweep, J reduction); peak "
                             f"{peak_src} copy bandwidth"},
    }


def run_iterate(args):
    """Time to convergence of the Lambda iteration or the accelerated one on the NX^3 regular
    grid (from LTE, max |dn/n| < --tol or --max-iter iterations).  Prints one JSON line."""
    import torch
    import paper_2306_01041_gb300 as rt
    dev = torch.device("cuda", 0)
    atm, f, (x, y, z, dx, dy), data, dirs, w = setup_problem(torch, dev)
    g = rt.RegularGrid(NX, NY, NZ, dx, dy, z, dirs, w)
    A = rt.Atom(data, atm.kappa0)
    M = rt.Atmos(*[torch.tensor(f[k], dtype=torch.float32, device=dev)
                   for k in ("T", "rho", "ne", "nH")])
    fn = rt.lambda_iterate_ali if args.iterate == "ali" else rt.lambda_iterate
    pops = rt.lte_populations(g, A, M)
    fn(g, A, M, pops, max_iter=1, tol=args.tol, ng_period=args.ng)   # first-call set-up, untimed
    pops = rt.lte_populations(g, A, M)
    torch.cuda.synchronize()
    t = time.perf_counter()
    it, hist, conv = fn(g, A, M, pops, max_iter=args.max_iter, tol=args.tol, ng_period=args.ng)
    dt = time.perf_counter() - t
    ng = f", Ng every {args.ng}" if args.ng else ""
    print(json.dumps({"workload": f"{args.iterate} iteration{ng}, regular grid {NX}x{NY}x{NZ}, "
                                  f"{len(data['lam'])} wavelengths", "iterations": it,
                      "converged": bool(conv), "seconds": round(dt, 4),
                      "ms_per_iteration": round(dt / it * 1e3, 3),
                      "final_change": float(hist[-1])}))


def run_sample(args):
    """Rejection sampling of Voronoi sites on the GPU (rt_sample_sites) from the 500 nm continuum
    opacity on the 128^3 mesh, floored at 1e-3 of its maximum."""
    import torch
    import paper_2306_01041_gb300 as rt
    from synth import make_atmosphere
    from synth.atmosphere import regular_fields
    dev = torch.device("cuda", 0)
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(NX, NY, NZ, atm)
    T = torch.tensor(f["T"], dtype=torch.float32, device=dev)
    rho = torch.tensor(f["rho"], dtype=torch.float32, device=dev)
    a, _ = rt.source_terms_lte(T, rho, atm.kappa0, 500e-9)
    target = torch.clamp(a / a.max(), min=1e-3).reshape(NZ, NY, NX).contiguous()
    box = (0.0, atm.Lx, 0.0, atm.Ly, atm.zmin, atm.zmax)
    n = args.sample
    for _ in range(2):
        rt.sample_sites(target, z, box, n, 1)
    torch.cuda.synchronize()
    times = []
    for s in range(max(1, args.steps)):
        t0 = time.perf_counter()
        _, nprop = rt.sample_sites(target, z, box, n, s + 2)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    ms = statistics.median(times) * 1e3
    print(json.dumps({"workload": f"rejection sampling of {n} sites from the 500 nm continuum "
                                  f"opacity on the {NX}x{NY}x{NZ} mesh", "ms": round(ms, 3),
                      "proposals": nprop, "gproposals_s": round(nprop / ms / 1e6, 3),
                      "msites_s": round(n / ms / 1e3, 3)}))


def run_tables(args):
    """Voronoi upwind tables and levels: grid creation with the host table build
    (RT_VORONOI_TABLES=host) against the default device build, and the device rebuild alone
    (rt_grid_build_tables_device), on an atmosphere grid of args.tables sites."""
    import torch
    import paper_2306_01041_gb300 as rt
    from synth import s4_quadrature
    _, g, _, _ = _make_vor((1, args.tables))
    dirs, w = s4_quadrature()
    mk = lambda: rt.VoronoiGrid(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"],  # noqa: E731
                                g["box"], dirs, w)
    mk()
    torch.cuda.synchronize()

    def timed(fn):
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out
    host, dflt, rebuild = [], [], []
    for _ in range(max(1, args.steps)):
        os.environ["RT_VORONOI_TABLES"] = "host"
        try:
            host.append(timed(mk)[0])
        finally:
            del os.environ["RT_VORONOI_TABLES"]
        t, G = timed(mk)
        dflt.append(t)
        rebuild.append(timed(G.build_tables_device)[0])
    print(json.dumps({"workload": f"Voronoi upwind tables and levels, {args.tables} sites, "
                                  f"{len(dirs)} directions",
                      "grid_create_host_tables_ms": round(statistics.median(host) * 1e3, 2),
                      "grid_create_device_tables_ms": round(statistics.median(dflt) * 1e3, 2),
                      "device_rebuild_ms": round(statistics.median(rebuild) * 1e3, 2),
                      "max_levels": G.max_levels}))


def run_voronoi_batch(args):
    """The batched Voronoi formal solution alone on the first N atmospheres of the 8-atmosphere
    workload (52 wavelengths, 24 directions, populations at LTE): a smaller case of the batched
    kernel for profiling.  Prints one JSON line."""
    import torch
    import paper_2306_01041_gb300 as rt
    from synth import model_atom, s4_quadrature
    dev = torch.device("cuda", 0)
    work = voronoi_workload(VOR_SIZES[:args.voronoi_batch], extra=())
    dirs, w = s4_quadrature()
    grids, alphas, Ss = [], [], []
    for s, g, f, kappa0 in work:
        G = rt.VoronoiGrid(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"], dirs, w)
        A = rt.Atom(model_atom(np.min(f["ne"] / np.sqrt(f["T"]))), kappa0)
        M = rt.Atmos(*[torch.tensor(f[k], dtype=torch.float32, device=dev)
                       for k in ("T", "rho", "ne", "nH")])
        a, sv = rt.source_terms(G, A, M, rt.lte_populations(G, A, M))
        grids.append(G)
        alphas.append(a)
        Ss.append(sv)
    nlam = alphas[0].shape[0]
    batch = rt.Batch(grids, nlam)
    Js = [torch.empty_like(a) for a in alphas]
    ms = _events(torch, lambda: batch.formal_solution(alphas, Ss, Js=Js), reps=args.steps)
    upd = sum(g.npt for g in grids) * NDIR * nlam
    print(json.dumps({"workload": f"batched Voronoi formal solution, {len(grids)} atmospheres",
                      "sites": [g.npt for g in grids], "ms": round(ms, 3),
                      "gupd_s": round(upd / ms / 1e6, 3)}))


def _events(torch, fn, reps=3):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def convergence_times(torch, rt, dev, work):
    """Time to convergence (max |dn/n| < 1e-3 from LTE) of the Lambda iteration and of the
    accelerated one on the 128^3 regular grid and on the 215k-site Voronoi grid; returns the
    timings and the converged populations of the plain iteration."""
    from synth import make_atmosphere, model_atom, s4_quadrature
    from synth.atmosphere import regular_fields
    res, out = {}, {}
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(NX, NY, NZ, atm)
    dirs, w = s4_quadrature()
    g = rt.RegularGrid(NX, NY, NZ, dx, dy, z, dirs, w)
    A = rt.Atom(model_atom(np.min(f["ne"] / np.sqrt(f["T"]))), atm.kappa0)
    M = _atmos(torch, rt, f, dev)
    g6, f6, k6 = work[6]
    G6 = _vgrid(rt, g6, dirs, w)
    A6 = rt.Atom(model_atom(np.min(f6["ne"] / np.sqrt(f6["T"]))), k6)
    M6 = _atmos(torch, rt, f6, dev)
    for name, (G, AA, MM) in ((f"regular_{NX}x{NY}x{NZ}", (g, A, M)),
                              (f"voronoi_{G6.npt}_sites", (G6, A6, M6))):
        for method, fn in (("lambda", rt.lambda_iterate), ("accelerated", rt.lambda_iterate_ali)):
            pops = rt.lte_populations(G, AA, MM)
            fn(G, AA, MM, pops, max_iter=1, tol=1e-3)       # graph capture and scratch, untimed
            pops = rt.lte_populations(G, AA, MM)
            torch.cuda.synchronize()
            t = time.perf_counter()
            it, hist, conv = fn(G, AA, MM, pops, max_iter=300, tol=1e-3)
            dt = time.perf_counter() - t
            res[f"{name}_{method}"] = {"iterations": it, "converged": bool(conv),
                                       "seconds": round(dt, 4),
                                       "s_per_iteration": round(dt / it, 5),
                                       "final_change": float(hist[-1])}
            if method == "lambda":
                out[name] = (G, AA, MM, pops)
    res["note"] = ("from LTE populations until max |dn/n| < 1e-3 (at most 300 iterations); host "
                   "wall time, one CUDA graph per iteration, a read-back every iteration")
    return res, out


def _pick3(atom_data):
    """The line core and the two continuum wavelengths of the atom."""
    lam = np.asarray(atom_data["lam"])
    return [int(np.argmin(np.abs(lam - atom_data["lam0"]))), len(lam) - 2, len(lam) - 1]


def _gradient_timing(torch, rt, G, A, M, pops, pick, stride):
    """Gradient of the sum of the mu = 1 map at three wavelengths with respect to T (through
    alpha and S at fixed populations), alpha and S: emergent map, adjoint sweep, chain rule."""
    alpha, S = rt.source_terms(G, A, M, pops)
    a3, s3 = alpha[pick].contiguous(), S[pick].contiguous()
    gI = torch.ones((3, G.ntop), device=alpha.device)
    ga_full = torch.zeros_like(alpha)
    gs_full = torch.zeros_like(alpha)

    def grad():
        rt.emergent_intensity(G, (0.0, 0.0, 1.0), a3, s3)
        ga, gs = rt.formal_solution_adjoint(G, (0.0, 0.0, 1.0), a3, s3, gI, ckpt_stride=stride)
        ga_full[pick] = ga
        gs_full[pick] = gs
        return rt.source_terms_adjoint(G, A, M, pops, ga_full, gs_full)
    ms = _events(torch, grad)
    ws = rt.lib().rt_adjoint_workspace_size(G.handle, 3, stride)
    return {"ms": round(ms, 3), "checkpoint_stride": stride, "workspace_MB": round(ws / 2 ** 20, 1)}


def adjoint_timings(torch, rt, dev, work, conv):
    """Gradient of the mu = 1 emergent map at the line core and both continua with respect to T,
    alpha and S at every point, populations at their converged NLTE values: the 128^3 regular
    grid and the 200k-site Voronoi grid."""
    from synth import make_atmosphere, model_atom
    res = {}
    name = f"regular_{NX}x{NY}x{NZ}"
    G, A, M, pops = conv[name]
    data = model_atom()
    pick = _pick3(data)
    res[name] = [_gradient_timing(torch, rt, G, A, M, pops, pick, st) for st in (1, 11)]
    from synth import s4_quadrature
    dirs, w = s4_quadrature()
    g9, f9, k9 = work[9]
    G9 = _vgrid(rt, g9, dirs, w)
    A9 = rt.Atom(model_atom(np.min(f9["ne"] / np.sqrt(f9["T"]))), k9)
    M9 = _atmos(torch, rt, f9, dev)
    p9 = rt.lte_populations(G9, A9, M9)
    it, _, conv9 = rt.lambda_iterate(G9, A9, M9, p9, max_iter=300, tol=1e-3)
    res[f"voronoi_{G9.npt}_sites"] = [_gradient_timing(torch, rt, G9, A9, M9, p9, pick, st)
                                      for st in (1, 8)]
    res["voronoi_converged_in"] = it
    res["note"] = ("mu = 1 map forward, adjoint sweep (FP64 on the device), chain rule to T at "
                   "fixed populations; CUDA events")
    return res


def accuracy_maps(torch, rt, dev, work):
    """LTE continuum at 500 nm, mu = 1 maps: the 32 x 32 x 64 regular grid and the 20k-site
    Voronoi grid (sampled from |dtau/dz|) against the 128 x 128 x 256 fine grid, as the RMS of the
    relative difference at the 32 x 32 shared pixels.  The Voronoi grid twice: its emergent-layer
    sites resampled to 32 x 32 pixels by two-nearest inverse-distance weighting, and the paper's
    procedure (the opacity at the sites interpolated back to the fine mesh by two-nearest inverse
    distance weighting, the mesh's own source function, the vertical formal solution there)."""
    from synth import make_atmosphere, s4_quadrature
    from synth.atmosphere import regular_fields
    atm = make_atmosphere(0)
    dirs, w = s4_quadrature()
    mu1 = (0.0, 0.0, 1.0)

    def regular(n):
        f, (x, y, z, dx, dy) = regular_fields(n, n, 2 * n, atm)
        G = rt.RegularGrid(n, n, 2 * n, dx, dy, z, dirs, w)
        a, sv = rt.source_terms_lte(torch.tensor(f["T"], dtype=torch.float32, device=dev),
                                    torch.tensor(f["rho"], dtype=torch.float32, device=dev),
                                    atm.kappa0, 500e-9)
        a, sv = a[None].contiguous(), sv[None].contiguous()
        return G, a, sv, rt.emergent_map(G, mu1, a, sv, n, n)[0].reshape(n, n)
    Gf, af, sf, fine = regular(128)
    _, _, _, m32 = regular(32)
    g10, f10, _ = work[10]
    G10 = _vgrid(rt, g10, dirs, w)
    av, sv = rt.source_terms_lte(torch.tensor(f10["T"], dtype=torch.float32, device=dev),
                                 torch.tensor(f10["rho"], dtype=torch.float32, device=dev),
                                 atm.kappa0, 500e-9)
    av, sv = av[None].contiguous(), sv[None].contiguous()
    native = rt.emergent_map(G10, mu1, av, sv, 32, 32)[0].reshape(32, 32)
    idw = rt.IDW(G10, Gf)
    synth_map = rt.emergent_map(Gf, mu1, idw.interpolate(av), sf, 128, 128)[0].reshape(128, 128)
    ref = fine[::4, ::4]

    def rms(m, r):
        return float(torch.sqrt(torch.mean((m.double() / r.double() - 1.0) ** 2)))
    e_reg, e_nat = rms(m32, ref), rms(native, ref)
    e_fs, e_fs128 = rms(synth_map[::4, ::4], ref), rms(synth_map, fine)
    return {"workload": "LTE continuum at 500 nm, mu = 1 emergent maps",
            "reference": "128x128x256 regular grid", "pixels": [32, 32],
            "rms_rel_diff": {"regular_32x32x64": round(e_reg, 5),
                             "voronoi_20k_native": round(e_nat, 5),
                             "voronoi_20k_final_synthesis": round(e_fs, 5),
                             "voronoi_20k_final_synthesis_128x128": round(e_fs128, 5)},
            "ratio_voronoi_native_to_regular": round(e_nat / e_reg, 3),
            "ratio_voronoi_final_synthesis_to_regular": round(e_fs / e_reg, 3),
            "voronoi_top_sites": G10.ntop,
            "fine_map_rms_contrast": round(float(fine.double().std() / fine.double().mean()), 4)}


def synthesis_timing(torch, rt, dev, g, f, kappa0, dirs, w):
    """The paper's final synthesis from the 200k-site grid (populations at LTE) to the 128^3
    mesh: two-nearest table (host, once), interpolation of the populations, source terms and the
    vertical long-characteristics formal solution on the mesh (52 wavelengths)."""
    from synth import make_atmosphere, model_atom
    from synth.atmosphere import regular_fields
    atm = make_atmosphere(0)
    mf, (x, y, z, dx, dy) = regular_fields(NX, NY, NZ, atm)
    G = _vgrid(rt, g, dirs, w)
    mesh = rt.RegularGrid(NX, NY, NZ, dx, dy, z, dirs, w)
    A = rt.Atom(model_atom(np.min(mf["ne"] / np.sqrt(mf["T"]))), atm.kappa0)
    sv = _atmos(torch, rt, f, dev)
    mv = _atmos(torch, rt, mf, dev)
    site_pops = rt.lte_populations(G, A, sv)
    t = time.perf_counter()
    idw = rt.IDW(G, mesh)
    build_s = time.perf_counter() - t
    return {"sites": G.npt, "mesh": [NX, NY, NZ], "table_build_s": round(build_s, 3),
            "interpolate_ms": round(_events(torch, lambda: idw.interpolate(site_pops)), 3),
            "final_synthesis_ms": round(_events(torch, lambda: rt.final_synthesis(
                idw, mesh, A, mv, site_pops)), 3)}


def lte_continuum_timing(torch, rt, dev, g, f, kappa0, dirs, w):
    """The small LTE continuum workloads (500 nm, 24 directions): 32x32x64 regular and the
    20k-site Voronoi grid; latency-bound (64 planes, or tens of levels per direction)."""
    from synth import make_atmosphere
    from synth.atmosphere import regular_fields
    res = {}
    atm = make_atmosphere(0)
    fr, (x, y, z, dx, dy) = regular_fields(32, 32, 64, atm)
    gr = rt.RegularGrid(32, 32, 64, dx, dy, z, dirs, w)
    G = _vgrid(rt, g, dirs, w)
    for name, grid, ff in (("regular_32x32x64", gr, fr), ("voronoi_20k", G, f)):
        al, S = rt.source_terms_lte(torch.tensor(ff["T"], dtype=torch.float32, device=dev),
                                    torch.tensor(ff["rho"], dtype=torch.float32, device=dev),
                                    atm.kappa0, 500e-9)
        al, S = al[None].contiguous(), S[None].contiguous()
        J = torch.empty_like(al)
        ms = _events(torch, lambda: rt.formal_solution(grid, al, S, J=J), reps=10)
        res[name] = {"formal_solution_ms": round(ms, 4),
                     "gupd_s": round(grid.npt * NDIR / ms / 1e6, 3)}
    return res


def run_extras(torch, rt, dev, work=None):
    """The final synthesis, the small LTE continuum workloads and the Ng-extrapolated
    iterations."""
    from synth import s4_quadrature
    if work is None:
        work = {s: (g, f, k0) for s, g, f, k0 in voronoi_workload()}
    dirs, w = s4_quadrature()
    out = {"final_synthesis": synthesis_timing(torch, rt, dev, *work[9], dirs, w),
           "lte_continuum": lte_continuum_timing(torch, rt, dev, *work[10], dirs, w)}
    from synth import make_atmosphere, model_atom
    from synth.atmosphere import regular_fields
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(NX, NY, NZ, atm)
    g = rt.RegularGrid(NX, NY, NZ, dx, dy, z, dirs, w)
    A = rt.Atom(model_atom(np.min(f["ne"] / np.sqrt(f["T"]))), atm.kappa0)
    M = _atmos(torch, rt, f, dev)
    for name, fn in (("lambda_ng3", rt.lambda_iterate), ("accelerated_ng3", rt.lambda_iterate_ali)):
        pops = rt.lte_populations(g, A, M)
        fn(g, A, M, pops, max_iter=1, tol=1e-3, ng_period=3)
        pops = rt.lte_populations(g, A, M)
        torch.cuda.synchronize()
        t = time.perf_counter()
        it, hist, conv = fn(g, A, M, pops, max_iter=300, tol=1e-3, ng_period=3)
        out[f"regular_{name}"] = {"iterations": it, "converged": bool(conv),
                                  "seconds": round(time.perf_counter() - t, 4)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle's CPU baseline")
    ap.add_argument("--no-voronoi", action="store_true",
                    help="only the regular-grid line (no Voronoi, convergence, adjoint, accuracy)")
    ap.add_argument("--cpu-iteration", type=int, default=0,
                    help="print the oracle's time for one Lambda iteration on an N^3 grid")
    ap.add_argument("--nx", type=int, default=128,
                    help="grid size per axis (profiling uses smaller cases; the benchmark is 128)")
    ap.add_argument("--voronoi-batch", type=int, default=0,
                    help="time only the batched Voronoi formal solution on the first N of the 8 "
                         "atmospheres (a smaller case for profiling)")
    ap.add_argument("--iterate", choices=["lambda", "ali"], default=None,
                    help="time the Lambda iteration or the accelerated one to convergence")
    ap.add_argument("--max-iter", type=int, default=300)
    ap.add_argument("--ng", type=int, default=0, help="Ng extrapolation period (0: off)")
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--tables", type=int, default=0,
                    help="time the Voronoi table build (host and GPU) on a grid of this many sites")
    ap.add_argument("--sample", type=int, default=0,
                    help="time only the rejection sampling of this many Voronoi sites")
    ap.add_argument("--scheme", choices=["plane", "face"], default="plane",
                    help="regular-grid short characteristics: plane to plane (default) or face "
                         "hitting")
    ap.add_argument("--z-stretch", type=float, default=0.0,
                    help="non-uniform z spacing amplitude a in [0, 1) (cell heights (1 -+ a) dz)")
    args = ap.parse_args()
    global NX, NY, NZ, WORKLOAD, SCHEME
    if args.nx != 128:
        NX = NY = NZ = args.nx
        WORKLOAD = WORKLOAD.replace("128x128x128", f"{NX}x{NY}x{NZ}")
    if args.z_stretch:
        WORKLOAD += f", stretched z (a = {args.z_stretch})"
    SCHEME = args.scheme
    if args.scheme == "face":
        WORKLOAD += ", face-hitting short characteristics"
    if args.warmup < 3:
        args.warmup = 3
    if args.cpu_iteration:
        run_cpu_iteration(args)
        return
    if args.voronoi_batch:
        run_voronoi_batch(args)
        return
    if args.sample:
        run_sample(args)
        return
    if args.tables:
        run_tables(args)
        return
    if args.iterate:
        run_iterate(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
