"""Benchmark: one Lambda iteration of the NLTE problem on the 128^3 regular grid.

A step is one pass of the whole hot path: opacity and source function from the populations
(52 wavelengths), the formal solution over 24 directions by short characteristics with J
accumulated over angles, rates and statistical equilibrium, and the convergence read-back.
Metric: point x direction x wavelength updates per second of the step (Gupd/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--extras]

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
--extras adds the batched-vs-plain Voronoi sweep of 8 atmospheres and the adjoint timing.
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

# DRAM bytes per launch of the dominant kernel from the ncu capture summarised in profiles/,
# valid only for the kernel source with this hash (else reported as null)
PROFILED_FILE = "paper_2306_01041_gb300/csrc/regular_tile.cu"
PROFILED = {"sc_wave_kernel": {"sha1": "f4fe1598b1f61e1bc98975ba75fa48d3def31502",
                               "dram_bytes_per_launch": 2.19e9 + 1.23e9},
            "sc_tile_kernel": {"sha1": None, "dram_bytes_per_launch": None}}

# FP32 FLOPs per point-direction-wavelength update of the sweep: three bilinear interpolations
# (4 mul + 3 add each), dtau (add, mul), exp and the interval weights (5), the intensity update
# (2 mul + 2 add + 1), J accumulation (FMA = 2)
FLOP_PER_UPDATE = 21 + 2 + 6 + 5 + 2
# FP32 (non-tensor) peak: 152 SMs x 128 lanes x 2 FLOP (FMA) x 2070 MHz
SM_COUNT, LANES, SM_MHZ_MAX = 152, 128, 2070.0
ALU_PEAK_TFLOPS = SM_COUNT * LANES * 2 * SM_MHZ_MAX * 1e6 / 1e12


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


def kernel_hash():
    with open(os.path.join(ROOT, PROFILED_FILE), "rb") as fh:
        return hashlib.sha1(fh.read()).hexdigest()


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
    # the formal-solution graph is one persistent wavefront launch (sc_wave_kernel) or, when that
    # path does not apply, one launch per plane step and hemisphere (sc_tile_kernel) plus the two
    # boundary planes; the achieved rate is the interior updates over the graph's event time
    interior_flops = FLOP_PER_UPDATE * NX * NY * (NZ - 1) * NDIR * nlam
    if args.scheme == "face":
        # face_sweep_kernel, then the fixed-order sum of the two hemispheres' J partials
        kname, per_launch_ms = "face_sweep_kernel", fs_ms
    elif launches[1] == 1:
        kname, per_launch_ms = "sc_wave_kernel", fs_ms
    else:
        kname, per_launch_ms = "sc_tile_kernel", fs_ms / (2 * (NZ - 1))
    achieved = interior_flops / (fs_ms * 1e-3) / 1e12
    traffic = None
    prof = PROFILED.get(kname)
    if prof and prof["sha1"] == kernel_hash() and prof["dram_bytes_per_launch"]:
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
                     "achieved": round(achieved, 3), "peak": round(ALU_PEAK_TFLOPS, 2),
                     "unit": "TFLOP/s", "frac": round(achieved / ALU_PEAK_TFLOPS, 4),
                     "traffic": traffic,
                     "per_launch_ms": round(per_launch_ms, 5),
                     "formal_solution_ms": round(fs_ms, 3),
                     "peak_note": "FP32 lanes x FMA x max clock (152 x 128 x 2 x 2070 MHz)"},
        "clocks": clk,
        "breakdown_ms": {"source_terms": round(statistics.mean(p[0] for p in part_times), 3),
                         "formal_solution": round(fs_ms, 3),
                         "statistical_equilibrium": round(statistics.mean(p[1] for p in part_times), 3)},
    }
    if args.extras:
        res["extras"] = run_extras(torch, rt, dev)
    if rank == 0 and not args.no_cpu:
        res["cpu_baseline"] = cpu_baseline(min(args.cpu_lams, nlam))
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()


_CPU_INPUTS = {}


def _cpu_inputs():
    """The oracle's FP64 inputs of the benchmark workload (LTE populations), built once."""
    if not _CPU_INPUTS:
        from oracle.physics import Atom
        from synth import make_atmosphere, model_atom, s4_quadrature
        from synth.atmosphere import regular_fields
        atm = make_atmosphere(0)
        f, (x, y, z, dx, dy) = regular_fields(NX, NY, NZ, atm)
        data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
        A = Atom(data, atm.kappa0)
        pops = A.lte_pops(f["T"], f["ne"], f["nH"])
        alpha, S = A.alpha_S(f["T"], f["rho"], f["ne"], pops)
        dirs, w = s4_quadrature()
        _CPU_INPUTS.update(alpha=alpha, S=S, dx=dx, dy=dy, z=z, dirs=dirs, w=w)
    return _CPU_INPUTS


def cpu_baseline(nl):
    """The oracle as it stands on this host's cores: the formal solution (sweep + J) of nl of the
    52 wavelengths on the benchmark's grid (with the benchmark's scheme), the dominant cost of the
    step."""
    import oracle
    c = _cpu_inputs()
    alpha, S, dx, dy, z, dirs, w = (c[k] for k in ("alpha", "S", "dx", "dy", "z", "dirs", "w"))
    pick = np.linspace(0, alpha.shape[0] - 1, nl).astype(int)
    sweep = oracle.sc_regular_face if SCHEME == "face" else oracle.sc_regular
    t = time.perf_counter()
    sweep(NX, NY, NZ, dx, dy, z, dirs, w, alpha[pick], S[pick])
    dt = time.perf_counter() - t
    upd = NX * NY * NZ * NDIR * nl
    scheme = ", face-hitting" if SCHEME == "face" else ""
    return {"value": round(upd / dt / 1e9, 5), "unit": "Gupd/s", "cores": oracle.num_threads(),
            "kind": "oracle", "seconds": round(dt, 2),
            "sample": f"formal solution of {nl} of 52 wavelengths, {NX}x{NY}x{NZ} grid, "
                      f"24 directions{scheme}"}


def run_reference(args):
    rank, world, local = _env_rank()
    if rank != 0:
        return
    nl = min(args.cpu_lams, 52)
    for _ in range(args.warmup):
        cpu_baseline(1)
    vals = [cpu_baseline(nl) for _ in range(args.steps)]
    v = statistics.mean(x["value"] for x in vals)
    sec = statistics.mean(x["seconds"] for x in vals)
    res = {"impl": "reference", "metric": "formal-solution Gupdates/s (pt*dir*lambda), NLTE Lambda iteration",
           "value": round(v, 5), "unit": "Gupd/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "grid": [NX, NY, NZ], "wavelengths": 52,
                      "directions": NDIR, "parallelism": "host cores (OpenMP)"},
           "cpu_baseline": {"value": round(v, 5), "unit": "Gupd/s", "cores": vals[0]["cores"],
                            "kind": "oracle", "sample": vals[0]["sample"]},
           "e2e": {"value": round(v, 5), "unit": "Gupd/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


VOR_SIZES = [50000, 67000, 90000, 120000, 160000, 215000, 290000, 400000]


def _make_vor(args):
    """One batched-workload atmosphere: seed s, size n; odd seeds rho^0.3, even |dtau/dz|."""
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
    parallel."""
    import multiprocessing as mp
    jobs = list(zip(range(1, len(sizes) + 1), sizes)) + list(extra)
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        return pool.map(_make_vor, jobs)


def run_extras(torch, rt, dev):
    """Batched persistent Voronoi sweep of 8 atmospheres (50k-400k sites, 52 wavelengths, 24
    directions) against plain per-direction launches; time to convergence on both grids; the
    adjoint of the mu = 1 emergent intensity."""
    from synth import model_atom, s4_quadrature
    out = {}
    t0 = time.perf_counter()
    work = voronoi_workload()
    out["voronoi_grid_build_s"] = round(time.perf_counter() - t0, 1)
    dirs, w = s4_quadrature()
    extra = {s: (g, f, kappa0) for s, g, f, kappa0 in work if s > 8}
    work = [x for x in work if x[0] <= 8]
    grids, atoms, atmoss, alphas, Ss = [], [], [], [], []
    for s, g, f, kappa0 in work:
        G = rt.VoronoiGrid(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"], dirs, w)
        data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
        A = rt.Atom(data, kappa0)
        M = rt.Atmos(*[torch.tensor(f[k], dtype=torch.float32, device=dev)
                       for k in ("T", "rho", "ne", "nH")])
        pops = rt.lte_populations(G, A, M)
        a, sv = rt.source_terms(G, A, M, pops)
        grids.append(G)
        atoms.append(A)
        atmoss.append((M, pops))
        alphas.append(a)
        Ss.append(sv)
    nlam = alphas[0].shape[0]
    upd = sum(g.npt for g in grids) * NDIR * nlam

    def timeit(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    Jp = [torch.empty_like(a) for a in alphas]
    os.environ["RT_VORONOI_SWEEP"] = "levels"      # plain per-direction, per-level launches
    ms_plain = timeit(lambda: [rt.formal_solution(g, a, sv, J=j)
                               for g, a, sv, j in zip(grids, alphas, Ss, Jp)])
    del os.environ["RT_VORONOI_SWEEP"]
    Js = [torch.empty_like(a) for a in alphas]      # one persistent launch per grid, in turn
    ms_single = timeit(lambda: [rt.formal_solution(g, a, sv, J=j)
                                for g, a, sv, j in zip(grids, alphas, Ss, Js)])
    from paper_2306_01041_gb300.autotune import tune_batch
    batch, choice = tune_batch(grids, alphas, Ss, nlam)
    Jb = [torch.empty_like(a) for a in alphas]
    ms_batch = timeit(lambda: batch.formal_solution(alphas, Ss, Js=Jb))
    diff = max(float(((b - p).abs() / p.abs().clamp_min(1e-30)).max()) for b, p in zip(Jb, Jp))
    out["voronoi_batch"] = {
        "atmospheres": len(grids), "sites": [g.npt for g in grids],
        "levels_max": [g.max_levels for g in grids], "wavelengths": nlam, "directions": NDIR,
        "plain_ms": round(ms_plain, 2), "batched_ms": round(ms_batch, 2),
        "per_grid_persistent_ms": round(ms_single, 2),
        "plain_gupd_s": round(upd / ms_plain / 1e6, 3),
        "per_grid_persistent_gupd_s": round(upd / ms_single / 1e6, 3),
        "batched_gupd_s": round(upd / ms_batch / 1e6, 3),
        "speedup": round(ms_plain / ms_batch, 2), "max_rel_diff_batched_vs_plain": diff,
        "autotuned": choice}
    # one batched Lambda iteration captured as a CUDA graph
    s_cap = torch.cuda.Stream()
    s_cap.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    bufs = [(torch.empty_like(a), torch.empty_like(a)) for a in alphas]

    def iteration(stream):
        for (M, pops), G, A, (ab, sb) in zip(atmoss, grids, atoms, bufs):
            a, sv = rt.source_terms(G, A, M, pops, stream=stream)
            ab.copy_(a)
            sb.copy_(sv)
        batch.formal_solution([b[0] for b in bufs], [b[1] for b in bufs], Js=Jb, stream=stream)
        for (M, pops), G, A, J in zip(atmoss, grids, atoms, Jb):
            rt.statistical_equilibrium(G, A, M, J, pops, stream=stream)
    with torch.cuda.stream(s_cap):
        iteration(s_cap)
        s_cap.synchronize()
        try:
            with torch.cuda.graph(graph, stream=s_cap):
                iteration(s_cap)
            graph_ok = True
        except Exception as exc:   # report, do not fail the benchmark
            graph_ok = repr(exc)
    torch.cuda.current_stream().wait_stream(s_cap)
    if graph_ok is True:
        ms_graph = timeit(lambda: graph.replay())
        out["voronoi_batch"]["graph_iteration_ms"] = round(ms_graph, 2)
    else:
        out["voronoi_batch"]["graph_iteration_error"] = graph_ok
    # time to convergence: the 128^3 regular grid and the 215k-site irregular grid
    out["convergence"] = convergence_times(torch, rt, dev, grids[5], atoms[5], atmoss[5])
    out["adjoint"] = adjoint_timing(torch, rt, dev)
    out["adjoint_voronoi_200k"] = voronoi_adjoint_timing(torch, rt, dev, *extra[9], dirs, w)
    out["lte_continuum"] = lte_continuum_timing(torch, rt, dev, *extra[10], dirs, w)
    out["final_synthesis"] = synthesis_timing(torch, rt, dev, *extra[9], dirs, w)
    return out


def synthesis_timing(torch, rt, dev, g, f, kappa0, dirs, w):
    """The paper's final synthesis from the 200k-site grid (populations at LTE) to the 128^3
    mesh: two-nearest table (host, once), interpolation of the populations, source terms and the
    vertical long-characteristics formal solution on the mesh (52 wavelengths)."""
    from synth import make_atmosphere, model_atom
    from synth.atmosphere import regular_fields
    atm = make_atmosphere(0)
    mf, (x, y, z, dx, dy) = regular_fields(NX, NY, NZ, atm)
    G = rt.VoronoiGrid(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"], dirs, w)
    mesh = rt.RegularGrid(NX, NY, NZ, dx, dy, z, dirs, w)
    A = rt.Atom(model_atom(np.min(mf["ne"] / np.sqrt(mf["T"]))), atm.kappa0)
    sv = rt.Atmos(*[torch.tensor(f[k], dtype=torch.float32, device=dev)
                    for k in ("T", "rho", "ne", "nH")])
    mv = rt.Atmos(*[torch.tensor(mf[k], dtype=torch.float32, device=dev)
                    for k in ("T", "rho", "ne", "nH")])
    site_pops = rt.lte_populations(G, A, sv)
    t = time.perf_counter()
    idw = rt.IDW(G, mesh)
    build_s = time.perf_counter() - t
    res = {"sites": G.npt, "mesh": [NX, NY, NZ], "table_build_s": round(build_s, 3),
           "interpolate_ms": round(_events(torch, lambda: idw.interpolate(site_pops)), 3),
           "final_synthesis_ms": round(_events(torch, lambda: rt.final_synthesis(
               idw, mesh, A, mv, site_pops)), 3)}
    return res


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
    """Voronoi upwind tables and levels: the host build inside rt_grid_create against the GPU
    rebuild (rt_grid_build_tables_device), on an atmosphere grid of args.tables sites."""
    import torch
    import paper_2306_01041_gb300 as rt
    from synth import s4_quadrature
    _, g, _, _ = _make_vor((1, args.tables))
    dirs, w = s4_quadrature()
    mk = lambda: rt.VoronoiGrid(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"],  # noqa: E731
                                g["box"], dirs, w)
    mk()
    torch.cuda.synchronize()
    host, dev = [], []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        G = mk()
        host.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        G.build_tables_device()
        dev.append(time.perf_counter() - t0)
    print(json.dumps({"workload": f"Voronoi upwind tables and levels, {args.tables} sites, "
                                  f"{len(dirs)} directions",
                      "grid_create_with_host_tables_ms": round(statistics.median(host) * 1e3, 2),
                      "device_rebuild_ms": round(statistics.median(dev) * 1e3, 2),
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


def voronoi_adjoint_timing(torch, rt, dev, g, f, kappa0, dirs, w):
    """Emergent mu = 1 intensity and its adjoint at the line core and both continua on the
    200k-site grid, populations at LTE."""
    from synth import model_atom
    G = rt.VoronoiGrid(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"], dirs, w)
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    A = rt.Atom(data, kappa0)
    M = rt.Atmos(*[torch.tensor(f[k], dtype=torch.float32, device=dev)
                   for k in ("T", "rho", "ne", "nH")])
    pops = rt.lte_populations(G, A, M)
    a, sv = rt.source_terms(G, A, M, pops)
    core = int(np.argmin(np.abs(np.asarray(data["lam"]) - data["lam0"])))
    pick = [core, len(data["lam"]) - 2, len(data["lam"]) - 1]
    a3, s3 = a[pick].contiguous(), sv[pick].contiguous()
    gI = torch.ones((3, G.ntop), device=dev)
    res = {"sites": G.npt, "top_sites": G.ntop,
           "emergent_ms": round(_events(torch, lambda: rt.emergent_intensity(
               G, (0.0, 0.0, 1.0), a3, s3)), 3)}
    for stride in (1, 8):
        res[f"adjoint_stride_{stride}_ms"] = round(_events(torch, lambda: rt.formal_solution_adjoint(
            G, (0.0, 0.0, 1.0), a3, s3, gI, ckpt_stride=stride)), 3)
        res[f"adjoint_stride_{stride}_workspace_MB"] = round(
            rt.lib().rt_adjoint_workspace_size(G.handle, 3, stride) / 2 ** 20, 1)
    return res


def lte_continuum_timing(torch, rt, dev, g, f, kappa0, dirs, w):
    """The small LTE continuum workloads (500 nm, 24 directions): 32x32x64 regular and the
    20k-site Voronoi grid; latency-bound (64 planes, or tens of levels per direction)."""
    from synth import make_atmosphere
    from synth.atmosphere import regular_fields
    res = {}
    atm = make_atmosphere(0)
    fr, (x, y, z, dx, dy) = regular_fields(32, 32, 64, atm)
    gr = rt.RegularGrid(32, 32, 64, dx, dy, z, dirs, w)
    G = rt.VoronoiGrid(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"], dirs, w)
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


def convergence_times(torch, rt, dev, vgrid, vatom, vatm):
    from synth import make_atmosphere, model_atom, s4_quadrature
    from synth.atmosphere import regular_fields
    res = {}
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(NX, NY, NZ, atm)
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    dirs, w = s4_quadrature()
    g = rt.RegularGrid(NX, NY, NZ, dx, dy, z, dirs, w)
    A = rt.Atom(data, atm.kappa0)
    M = rt.Atmos(*[torch.tensor(f[k], dtype=torch.float32, device=dev)
                   for k in ("T", "rho", "ne", "nH")])
    for name, (G, AA, MM) in (("regular_128^3", (g, A, M)),
                              ("voronoi_%d_sites" % vgrid.npt, (vgrid, vatom, vatm[0]))):
        for method, fn, ngp in (("lambda", rt.lambda_iterate, 0), ("ali", rt.lambda_iterate_ali, 0),
                                ("lambda_ng", rt.lambda_iterate, 3),
                                ("ali_ng", rt.lambda_iterate_ali, 3)):
            pops = rt.lte_populations(G, AA, MM)
            fn(G, AA, MM, pops, max_iter=1, tol=1e-3, ng_period=ngp)   # first-call set-up
            pops = rt.lte_populations(G, AA, MM)
            torch.cuda.synchronize()
            t = time.perf_counter()
            it, hist, conv = fn(G, AA, MM, pops, max_iter=300, tol=1e-3, ng_period=ngp)
            dt = time.perf_counter() - t
            res[f"{name}_{method}"] = {"iterations": it, "converged": bool(conv),
                                       "seconds": round(dt, 3), "s_per_iteration": round(dt / it, 5),
                                       "final_change": float(hist[-1])}
    return res


def adjoint_timing(torch, rt, dev):
    """Gradient of the mu = 1 emergent map at the line core and both continua on 128^3."""
    from synth import make_atmosphere, model_atom, s4_quadrature
    from synth.atmosphere import regular_fields
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(NX, NY, NZ, atm)
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    dirs, w = s4_quadrature()
    g = rt.RegularGrid(NX, NY, NZ, dx, dy, z, dirs, w)
    A = rt.Atom(data, atm.kappa0)
    M = rt.Atmos(*[torch.tensor(f[k], dtype=torch.float32, device=dev)
                   for k in ("T", "rho", "ne", "nH")])
    pops = rt.lte_populations(g, A, M)
    a, sv = rt.source_terms(g, A, M, pops)
    core = int(np.argmin(np.abs(np.asarray(data["lam"]) - data["lam0"])))
    pick = [core, len(data["lam"]) - 2, len(data["lam"]) - 1]
    a3, s3 = a[pick].contiguous(), sv[pick].contiguous()
    gI = torch.ones((3, g.ntop), device=dev)
    res = {}
    for stride in (1, 11):
        rt.formal_solution_adjoint(g, (0.0, 0.0, 1.0), a3, s3, gI, ckpt_stride=stride)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            rt.formal_solution_adjoint(g, (0.0, 0.0, 1.0), a3, s3, gI, ckpt_stride=stride)
        e1.record()
        torch.cuda.synchronize()
        res[f"stride_{stride}_ms"] = round(e0.elapsed_time(e1) / 3, 3)
        res[f"stride_{stride}_workspace_MB"] = round(
            rt.lib().rt_adjoint_workspace_size(g.handle, 3, stride) / 2 ** 20, 1)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-lams", type=int, default=52)
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
