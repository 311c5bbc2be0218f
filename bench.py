#!/usr/bin/env python
"""Benchmark of the JGS2 hot path: milliseconds per implicit-Euler time step to a 1e-4
relative residual (capped at --max-sweeps), JGS2 sweeps per second, and the dominant sweep
kernel's fraction of the measured HBM bandwidth.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload spheres|beam|cube|batch]
    python bench.py --impl reference ...     # the FP64 CPU oracle on the host cores

One step = one call of jgs2_step (every sweep of the step: contact pass, pool, gather,
correct, line-search energy and update kernels plus the per-step setup) on inputs already
resident in HBM. The default workload is ten voxel spheres (3.47M tets) in a box with the IPC
barrier on. `batch` is 256 seeded voxel blobs of uneven size stepped together in one mesh
(graph-captured sweep chunks, per-scene stopping). With N > 1 (torchrun) every rank steps
its own replica of a single scene (one scene's sweep does not shard across GPUs), while the
batch workload shards the job's N x n_scenes blobs across the ranks by tet count, with no
exchange between them. The time is the maximum over ranks and the value counts every
rank's work.
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

METRIC = "ms/step to 1e-4 rel. residual at 3.5M tets"
_CONTACT_NAME = {0: "contact off", 1: "IPC barrier dhat=1e-3 on", 2: "penalty contact dhat=1e-3 on"}
KIND = ["k_pool", "k_gather", "k_correct", "k_energy", "k_update", "setup", "contact", "k_elem",
        "k_pair_trials", "k_ls_decide", "k_batch_persistent"]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def shard_scenes(sizes, world):
    """Scene indices per rank, balanced by size: largest scene first to the least-loaded
    rank (ties to the lower rank); each rank's list in ascending order. No scene is shared:
    the batch shards with no exchange between ranks."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += sizes[i]
    return [sorted(o) for o in out]


def over_ranks(value, op="max", device=None):
    """A per-rank float reduced over the process group ("max" or "sum"; the value itself
    when there is no group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def build_scenes(args, rank=0, world=1):
    """(list of scenes, description, batch?). The batch workload has n_scenes scenes per
    rank: the job's n_scenes * world seeded blobs are sharded by tet count."""
    import scenes
    w = args.workload
    if w == "spheres":
        s = scenes.spheres_scene(n_spheres=args.n_spheres, contact=args.contact)
        return [s], (f"{args.n_spheres} voxel spheres r=0.1 m, 48 cells across, {s.n_tets:,} tets, "
                     f"box walls, {_CONTACT_NAME[args.contact]}"), False
    if w == "beam":
        return [scenes.beam_scene()], "20x20x100-vertex Kuhn beam 0.02x0.02x0.1 m, 214,434 tets, E=1e7", False
    if w == "cube":
        return [scenes.cube_scene()], "5x5x5-vertex Kuhn cube, 384 tets", False
    if w == "batch":
        n = args.n_scenes * world
        mine = shard_scenes([scenes.blob_tet_target(i, 1e3, 5e4) for i in range(n)], world)[rank]
        ss = [scenes.blob_scene(i, 1e3, 5e4) for i in mine]
        T = sum(s.n_tets for s in ss)
        shard = f", rank {rank}'s shard of {n}" if world > 1 else ""
        return ss, (f"{len(ss)} seeded voxel blobs{shard} (1-6 spheres, 1k-50k tets each, {T:,} tets), "
                    "E log-uniform 1e4-1e7, nu 0.3-0.48, bottom pinned"), True
    raise SystemExit(f"unknown workload {w}")


def concat(ss):
    return (np.concatenate([s.X for s in ss]), np.concatenate([s.v0 for s in ss]),
            np.concatenate([s.tets + o for s, o in zip(ss, np.cumsum([0] + [q.n_vertices for q in ss[:-1]]))]),
            np.concatenate([s.youngs for s in ss]), np.concatenate([s.poisson for s in ss]),
            np.concatenate([s.density for s in ss]), np.concatenate([s.pinned for s in ss]))


def kernel_bytes(V_f, T, n_cub, fp_bytes=4):
    """DRAM bytes each sweep kernel must move per launch that does work (every datum it
    reads or writes counted once), by kernel.

    tet record fields read: 4 corner ids (16 B) + B (9) + F(x_t) (9) + V_e, mu, lam' (3);
    k_elem: tet record fields, the corners' displacements (u, 16 B per vertex) and the
      element record F_e, V_e, mu, lam' (12 scalars) written;
    k_gather: element records and the four corner vectors b_a (4 x 4 scalars) per tet, 4
      incidence entries per tet (16 B); per free vertex u, dz read, m/h^2, the incidence
      count, D_J written (3) and g, H, R written (18 scalars);
    k_correct: per free vertex g, H, R read (18), D written (3), and n_cub cubature slots of
      (pool index 4 B, weight, 36 U_bar entries); the pool's element data stays in L2;
    k_energy, a one-direction pass: tet record fields; per free vertex u, dz, the direction
      (3 each) and m/h^2; a two-direction pass ("k_energy_2") adds the second direction;
    k_update: per free vertex u read and written, one direction read (3 each)."""
    f = fp_bytes
    rec = 16 + 21 * f
    return {
        "k_elem": T * (rec + 12 * f) + V_f * 4 * f,
        "k_gather": T * (12 * f + 16 * f + 16) + V_f * ((3 + 3 + 1 + 3 + 18) * f + 4),
        "k_correct": V_f * ((18 + 3) * f + n_cub * (4 + 37 * f)),
        "k_energy": T * rec + V_f * (10 * f),
        "k_energy_2": T * rec + V_f * (13 * f),
        "k_update": V_f * (9 * f),
    }


def sweep_bytes(V_f, T, n_cub, fp_bytes=4):
    """Algorithmic bytes of one whole sweep in this layout (the method's compulsory
    traffic, each datum once): per tet the corner ids, B, F(x_t), V_e and material (the tet
    record fields) and four incidence entries; per free vertex x read and written, z, m, R
    written, g/H written and read, and the cubature record (pool index, weight, 12x3 U_bar
    per slot)."""
    f = fp_bytes
    per_tet = 16 + 21 * f + 16
    per_vertex = (3 + 3 + 3 + 1) * f + 9 * f + 2 * 9 * f + n_cub * (4 + 37 * f)
    return T * per_tet + V_f * per_vertex


def scope_sweep_bytes(V_f, T, n_cub, fp_bytes=4):
    """The per-unit byte model of the hot-path scope (FP32, each datum once): 76 B per tet
    (corner ids 16, B 36, V_e 4, E 4, incidence 16) and, per free vertex, x read and
    written, z and m (40 B), R written (36), g/H written and read (72) and the cubature
    record (n_cub x (4 + 4 + 144) = 608 B at n_cub = 4): 756 B. Scalars scale with the
    precision; ids do not."""
    f = fp_bytes
    per_tet = 16 + 9 * f + f + f + 16
    per_vertex = 10 * f + 9 * f + 18 * f + n_cub * (4 + f + 36 * f)
    return T * per_tet + V_f * per_vertex


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture of
# one launch each, FP32, 4 voxel spheres: 1,388,544 tets, 253,652 free vertices, synthetic
# cubature; k_energy is its one-direction pass). It grows in proportion to the tets (the
# vertices grow with them), so a launch on another mesh of the same kind is credited with
# traffic x T / 1,388,544. Only kernels whose code has not changed since their capture are
# listed.
NCU_TRAFFIC_TETS = 1388544
NCU_TRAFFIC = {"k_gather": 198.486528e6 + 19.848448e6, "k_elem": 159.587840e6 + 35.314944e6,
               "k_correct": 175.108096e6 + 5.450752e6, "k_energy": 171.836160e6 + 3.512576e6}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [q.strip() for q in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_units(args):
    """The workload as independent bodies the oracle can sweep one at a time (no exchange
    between them): (builder, argument) pairs, built inside the worker process."""
    if args.workload == "spheres":
        return [("sphere", k) for k in range(args.n_spheres)]
    if args.workload == "batch":
        return [("blob", i) for i in range(args.n_scenes)]
    return [(args.workload, 0)]


def _oracle_sweep_sample(unit, n_sweeps=1, seed=0):
    """One process: builds one body of the workload and times n_sweeps full oracle sweeps
    (FP64 numpy, one thread: the JGS2 direction of every free vertex, sweep.direction, and
    the global line search, sweep.line_search) from x_t. Cubature records are the seeded
    synthetic ones (the oracle cannot train a 63k-vertex body: its precompute is dense), so
    the line search's D_J pass is not triggered. Returns (tets, seconds per sweep)."""
    import scenes
    from oracle import fem, precompute, sweep
    kind, arg = unit
    if kind == "sphere":
        s = scenes.sphere_of_scene(arg)
    elif kind == "blob":
        s = scenes.blob_scene(arg, 1e3, 5e4)
    elif kind == "beam":
        s = scenes.beam_scene()
    else:
        s = scenes.cube_scene()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    elem, w, u = scenes.random_cubature(s.X, s.tets, s.pinned, 4, seed=seed, w_max=0.5, u_sigma=0.2)
    cub = precompute.Cubature(elem, w, u, np.zeros(len(s.X)))
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    x = s.X.copy()
    t0 = time.perf_counter()
    for _ in range(n_sweeps):
        D, DJ, g = sweep.direction(m, x, z, s.dt, cub)
        x = x + sweep.line_search(m, x, z, s.dt, D, DJ, g)
    return s.n_tets, (time.perf_counter() - t0) / n_sweeps


def _oracle_pool(units, procs):
    """Times one sweep of every unit, `procs` single-threaded processes at a time (spawned:
    the parent has already used the GPU). Returns [(tets, seconds)] in unit order."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(processes=procs) as pool:
            return pool.map(_oracle_sweep_sample, units, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def makespan(times, procs):
    """Wall time of independent jobs on `procs` workers, longest job first to the least
    loaded worker."""
    load = [0.0] * max(1, procs)
    for t in sorted(times, reverse=True):
        i = min(range(len(load)), key=lambda q: load[q])
        load[i] += t
    return max(load)


def cpu_baseline(args, sweeps_per_step):
    """The oracle as it stands on the host cores: one full sweep of every body of the
    workload (contact off: the oracle's pair search is all-pairs), the bodies in parallel
    on up to min(cores, bodies) single-threaded processes. The workload's sweep on those
    cores takes the makespan of the measured per-body sweeps; a step is that times the GPU
    step's sweeps (+1 for the final residual evaluation). No other extrapolation."""
    units = oracle_units(args)
    cores = os.cpu_count() or 1
    procs = max(1, min(cores, len(units)))
    res = _oracle_pool(units, procs)
    per = [r[1] for r in res]
    wall = makespan(per, procs)
    n_sw = sweeps_per_step + 1
    return {"value": wall * n_sw * 1e3, "unit": "ms/step", "cores": procs, "kind": "oracle",
            "host_cores": cores,
            "single_thread_ms_per_step": sum(per) * n_sw * 1e3,
            "sweep_s_per_body": {"min": round(min(per), 3), "median": round(float(np.median(per)), 3),
                                 "max": round(max(per), 3)},
            "sample": (f"one full FP64 oracle sweep (direction + global line search, contact off, synthetic "
                       f"cubature records) of each of the {len(units)} bodies ({sum(r[0] for r in res):,} tets), "
                       f"{procs} bodies at a time on single-threaded processes; scene sweep = makespan "
                       f"{wall:.2f} s, times {n_sw:.0f} sweeps per step")}


def run_reference(args, rank, world):
    """The oracle as the reference arm: every step is one full oracle sweep of one body of
    the workload (single-threaded), scaled to the whole step by bodies and sweeps. The
    K + W samples run concurrently on the host cores (spawned processes) so the run takes
    a few minutes; each sample is timed inside its own process."""
    if rank != 0:
        return None
    units = oracle_units(args)
    n = args.warmup + args.steps
    cores = os.cpu_count() or 1
    procs = max(1, min(cores, n))
    res = _oracle_pool([units[q % len(units)] for q in range(n)], procs)
    tets_total = sum(_unit_tets(args))
    per_body = [r[1] for r in res][args.warmup:]
    # the whole workload on one core: each body's sweep in turn (bodies of one workload
    # differ in size only in the batch, where the sample's tets scale it)
    vals = [r[1] * tets_total / r[0] * (args.ref_sweeps + 1) * 1e3 for r in res[args.warmup:]]
    v = float(np.median(vals))
    desc = build_desc(args)
    cb = {"value": v, "unit": "ms/step", "cores": 1, "kind": "oracle", "host_cores": cores,
          "sample": (f"per step, one full FP64 oracle sweep (direction + global line search, contact off, "
                     f"synthetic cubature records) of one body; scaled by tets ({tets_total:,} in the workload) "
                     f"and {args.ref_sweeps + 1:.0f} sweeps per step; {n} samples, {procs} at a time on "
                     f"single-threaded processes; median body sweep {np.median(per_body):.2f} s")}
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms/step", "higher_is_better": False,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "scene": desc, "tets": tets_total,
                       "sweeps_per_step": args.ref_sweeps},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "ms/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _unit_tets(args):
    import scenes
    if args.workload == "spheres":
        return [scenes.sphere_of_scene(0).n_tets] * args.n_spheres
    if args.workload == "batch":
        return [scenes.blob_scene(i, 1e3, 5e4).n_tets for i in range(args.n_scenes)]
    if args.workload == "beam":
        return [scenes.beam_scene().n_tets]
    return [scenes.cube_scene().n_tets]


def build_desc(args):
    return {"spheres": f"{args.n_spheres} voxel spheres r=0.1 m, 48 cells across, box walls",
            "beam": "20x20x100-vertex Kuhn beam 0.02x0.02x0.1 m, 214,434 tets, E=1e7",
            "cube": "5x5x5-vertex Kuhn cube, 384 tets",
            "batch": f"{args.n_scenes} seeded voxel blobs (1-6 spheres, 1k-50k tets each)"}.get(args.workload, "")


def split_cubature(elem, w, u, ss):
    """Per-scene cubature records from a batch mesh's export (tet ids made scene-local)."""
    out, vo, to = [], 0, 0
    for s in ss:
        e = elem[vo:vo + s.n_vertices]
        out.append((np.where(e >= 0, e - to, -1), w[vo:vo + s.n_vertices], u[vo:vo + s.n_vertices]))
        vo += s.n_vertices
        to += s.n_tets
    return out


def timed_steps(mesh, x, v, opts, n, stream, gs=False):
    """n steps (Gauss-Seidel steps with gs) between CUDA events on the launching stream;
    (ms, [report dicts])."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    reps = []
    for _ in range(n):
        r = mesh.step_gs(x, v, opts, stream) if gs else mesh.step(x, v, opts, stream)
        reps.append({"sweeps": r.sweeps, "converged": r.converged, "rel": r.rel_residual,
                     "kms": list(r.kernel_ms), "kl": list(r.kernel_launches), "launches": r.launches,
                     "fallback": r.fallback, "rejects": r.ls_rejects, "dj": r.dj_steps,
                     "rebuilds": r.contact_rebuilds, "cand": r.contact_candidates, "near": r.contact_near,
                     "psw": r.profiled_sweeps, "passes": list(r.ls_passes), "stopped_dx": r.stopped_dx,
                     "last_dx": r.last_dx})
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), reps


def length_scale(args, X):
    """L of the paper's unit-cube normalisation (Sec. 8): the 1 x 1 x 2 m box of the spheres
    scene, else the rest positions' largest extent."""
    if args.workload == "spheres":
        return 2.0
    return float(np.max(X.max(axis=0) - X.min(axis=0)))


def run_jgs2(args, rank, world, local_rank):
    import torch
    import paper_2506_06494_b300 as p

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    ss, desc, batch = build_scenes(args, rank, world)
    X, V0, tets, _, _, _, pin = concat(ss)
    T = sum(s.n_tets for s in ss)
    Vf = int((~pin.astype(bool)).sum())
    t0 = time.perf_counter()
    if args.friction > 0 and (batch or not ss[0].contact):
        raise SystemExit("--friction needs a single scene with contact (the spheres workload)")
    mesh = p.Mesh.batch(ss) if batch else p.Mesh.from_scene(ss[0], friction_mu=args.friction)
    gs = bool(args.gs)
    if gs and (batch or (args.workload == "spheres" and args.contact)):
        raise SystemExit("--gs takes a single scene without contact")
    if args.cubature == "precompute":
        mesh.precompute(n_cub=args.n_cub, gs=int(gs), gpu=int(args.precompute_gpu))
    else:
        # seeded synthetic records: same kernel work, no convergence meaning (profiling only)
        import scenes
        mesh.precompute_import(*scenes.random_cubature(X, tets, pin, args.n_cub, seed=0, w_max=0.5, u_sigma=0.2))
    t_pre = time.perf_counter() - t0
    prec = p.FP32 if args.precision == "fp32" else p.FP64
    corr = {"asm": p.CORR_ASM, "elem": p.CORR_ELEM, "off": p.CORR_OFF}[args.correction]
    stream = torch.cuda.current_stream()
    alu = {"fp32_gflops": p.alu_peak(p.FP32, stream), "fp64_gflops": p.alu_peak(p.FP64, stream)}
    # chunks of 16 sweeps (the library's default), fewer when the cap is lower: the timed
    # (last) sweep of a chunk must fall inside the step
    chunk = max(1, min(16, args.max_sweeps + 1))
    opts = p.step_opts(precision=prec, correction=corr, max_sweeps=args.max_sweeps, rel_tol=1e-4, profile=1,
                       check_every=chunk, persistent=int(args.persistent and batch),
                       contact_coupling=int(args.coupling))
    x0 = torch.tensor(X, dtype=torch.float64, device=dev)
    v0 = torch.tensor(V0, dtype=torch.float64, device=dev)
    mesh.autotune(x0, v0, opts)
    gbs, gtpv, cbs, cpf = mesh.launch_config(prec)
    bs = {"gather_block": gbs, "gather_threads_per_vertex": gtpv, "correct_block": cbs,
          "correct_slot_prefetch": cpf}
    x, v = x0.clone(), v0.clone()
    for _ in range(args.warmup):
        mesh.step_gs(x, v, opts, stream) if gs else mesh.step(x, v, opts, stream)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    gidx = vis.split(",")[local_rank] if vis else str(local_rank)
    clocks = Clocks(gidx)
    ms_total, reps = timed_steps(mesh, x, v, opts, args.steps, stream, gs)
    ck = clocks.stop()
    scene_sweeps = None
    if batch:
        sw, cv, rr = mesh.batch_report()
        scene_sweeps = {"min": int(sw.min()), "median": float(np.median(sw)), "max": int(sw.max()),
                        "converged_scenes_last_step": int(cv.sum()), "max_rel_residual": float(rr.max())}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        ms_total = over_ranks(ms_total, "max", dev)
    sweeps = np.array([q["sweeps"] for q in reps])
    kms = np.sum([q["kms"] for q in reps], axis=0)
    kl = np.sum([q["kl"] for q in reps], axis=0)
    passes = np.sum([q["passes"] for q in reps], axis=0)
    launches = int(sum(q["launches"] for q in reps))
    # time per step of the whole job: every rank advances its own scene (replica) or shard by
    # one step in that time, the slowest rank setting it; aggregate throughput is reported
    # separately (scene steps and sweeps per second over all ranks)
    ms_step = ms_total / args.steps
    # end to end: host buffers through jgs2_step_host, copies inside the timed region
    xh, vh = X.copy(), V0.copy()
    opts_e2e = p.step_opts(precision=prec, correction=corr, max_sweeps=args.max_sweeps, rel_tol=1e-4,
                           check_every=chunk, persistent=int(args.persistent and batch),
                           contact_coupling=int(args.coupling))
    torch.cuda.synchronize()
    # (the host-array entry point runs Jacobi steps; the Gauss-Seidel form has no e2e leg)
    n_e2e = 0 if (args.no_e2e or gs) else args.steps
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        mesh.step_host(xh, vh, opts_e2e, stream)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / max(n_e2e, 1) if n_e2e else None
    if e2e_ms is not None and world > 1:
        e2e_ms = over_ranks(e2e_ms, "max", dev)
    hbm, peak_kind = peaks()
    n_cub = args.n_cub if corr != p.CORR_OFF else 0
    fpb = 4 if prec == p.FP32 else 8
    kb = kernel_bytes(Vf, T, n_cub, fpb)
    out = {
        "metric": METRIC, "value": ms_step, "unit": "ms/step", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == p.FP32 else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "scene": desc, "cubature": args.cubature, "tets": T,
                   "vertices": int(len(X)), "free_vertices": Vf,
                   "contact": bool(args.contact) if args.workload == "spheres" else False,
                   "contact_form": ({1: "ipc", 2: "penalty"}.get(args.contact)
                                    if args.workload == "spheres" else None),
                   "correction": args.correction, "line_search": True, "n_cub": args.n_cub, "rel_tol": 1e-4,
                   "parallelisation": "Gauss-Seidel (greedy colouring, group subspaces)" if gs else "Jacobi",
                   "contact_coupling": bool(args.coupling),
                   "wall_friction_mu": args.friction,
                   "max_sweeps": args.max_sweeps, "block_size": bs,
                   "batch_launch": ("persistent cooperative launch per chunk" if args.persistent else
                                    "one launch per kernel, graph-captured chunks") if batch else None,
                   "parallelism": f"{'scene shards' if batch else 'replicas'} x{world}",
                   "l2": "per-sweep working set larger than L2 (126 MB); no flush"},
        "sweeps_per_step": float(sweeps.mean()),
        "sweeps_per_s": over_ranks(float(sweeps.sum()), "sum", dev if world > 1 else None) / (ms_total * 1e-3),
        "aggregate": {"scene_steps_per_s": world * args.steps / (ms_total * 1e-3),
                      "note": "every rank steps its own replica or shard; value is the time per step of one"},
        "converged_steps": int(sum(q["converged"] for q in reps)),
        "max_rel_residual": float(max(q["rel"] for q in reps)),
        "line_search_per_step": {"dj_steps": float(np.mean([q["dj"] for q in reps])),
                                 "rejects": float(np.mean([q["rejects"] for q in reps])),
                                 "fallback_vertex_solves": float(np.mean([q["fallback"] for q in reps])),
                                 "passes_D": float(passes[0]) / args.steps,
                                 "passes_DJ_after_D_failed": float(passes[1]) / args.steps,
                                 "passes_both": float(passes[2]) / args.steps},
        "contact_rebuilds_per_step": float(np.mean([q["rebuilds"] for q in reps])),
        "contact_pairs_last_step": {"candidates": int(reps[-1]["cand"]), "within_rc_last_sweep": int(reps[-1]["near"])},
        "precompute_s": round(t_pre, 2),
        "precompute_solves": (("GPU (FP32 substitutions, FP64 refinement) for bodies of 20k vertices and "
                               "more; smaller bodies, when several, host FP64 side by side")
                              if args.precompute_gpu else "host FP64")
        if args.cubature == "precompute" else None,
        "e2e": {"value": e2e_ms, "unit": "ms/step", "h2d_bytes_per_step": int(xh.nbytes + vh.nbytes),
                "d2h_bytes_per_step": int(xh.nbytes + vh.nbytes)},
        "gpu_launches": launches,
        "clocks": ck,
        "alu_peak_measured": {k: round(val, 1) for k, val in alu.items()},
    }
    # whole sweep: algorithmic bytes per sweep over the step time per sweep, on this
    # layout's model and on the scope's per-unit model
    sw_tot = max(int(sweeps.sum()), 1)
    ms_sweep = ms_total / sw_tot
    for key, b in (("sweep_roofline", sweep_bytes(Vf, T, n_cub, fpb)),
                   ("sweep_roofline_scope_model", scope_sweep_bytes(Vf, T, n_cub, fpb))):
        gbs = b / (ms_sweep * 1e-3) / 1e9
        out[key] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(gbs / hbm, 4), "bytes_per_sweep": b, "ms_per_sweep": round(ms_sweep, 5),
                    "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    if batch:
        out["scene_sweeps"] = scene_sweeps
    # kernel times: CUDA events, inside the timed steps, around every kernel launch of the
    # last sweep of each replayed chunk of the sweep graph (one sweep in check_every is
    # sampled; the per-step setup kernels are timed in full). A sweep kernel's time per
    # sweep is its sampled time over the sampled sweeps; its time per step, that times the
    # sweeps per step.
    psw = max(int(sum(q["psw"] for q in reps)), 1)
    per_sweep_ms = {}
    for q, name in enumerate(KIND):
        per_sweep_ms[name] = float(kms[q] / args.steps if name == "setup" else kms[q] / psw)
    est_step = {n: per_sweep_ms[n] * (1.0 if n == "setup" else sw_tot / args.steps) for n in KIND}
    tot = max(sum(est_step.values()), 1e-12)
    share = {n: round(est_step[n] / tot, 4) for n in KIND}
    # launches that did work per sweep: one each, except the line search's energy pass,
    # which runs one or two of its three variants
    n_pass = float(passes.sum())
    work = {n: 1.0 for n in ("k_elem", "k_gather", "k_correct", "k_update")}
    per_kernel = {}
    for q, name in enumerate(KIND):
        if kl[q] == 0 or per_sweep_ms[name] <= 0:
            continue
        if name == "k_energy" and n_pass > 0:
            # bytes per working launch: one- and two-direction passes in their measured mix
            b_launch = (kb["k_energy"] * (passes[0] + passes[1]) + kb["k_energy_2"] * passes[2]) / n_pass
            launches_per_sweep = n_pass / sw_tot
        elif name in work and name in kb:
            b_launch = kb[name]
            launches_per_sweep = 1.0
        else:
            per_kernel[name] = {"ms_per_sweep": round(per_sweep_ms[name], 5)}
            continue
        t_launch = per_sweep_ms[name] / launches_per_sweep
        gbs = b_launch / (t_launch * 1e-3) / 1e9
        per_kernel[name] = {"ms_per_sweep": round(per_sweep_ms[name], 5),
                            "working_launches_per_sweep": round(launches_per_sweep, 3),
                            "avg_launch_ms": round(t_launch, 5), "bytes_per_launch": int(b_launch),
                            "GB_s": round(gbs, 1), "frac": round(gbs / hbm, 4)}
    out["profiled_sweeps"] = psw
    out["kernel_ms_per_step"] = {n: round(est_step[n], 4) for n in KIND}
    out["kernel_launches_per_step"] = {KIND[q]: int(kl[q] // args.steps) for q in range(len(KIND))}
    out["kernel_share"] = share
    out["kernels"] = per_kernel
    roofed = [n for n in per_kernel if "GB_s" in per_kernel[n]]
    if roofed:
        dom = max(roofed, key=lambda n: share[n])
        pk = per_kernel[dom]
        traffic = NCU_TRAFFIC.get(dom)
        if traffic is not None and prec == p.FP32 and not batch:
            traffic = int(traffic * T / NCU_TRAFFIC_TETS)
        else:
            traffic = None
        out["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": pk["GB_s"], "peak": hbm,
                           "unit": "GB/s", "frac": pk["frac"], "traffic": traffic,
                           "bytes_per_launch": pk["bytes_per_launch"], "avg_launch_ms": pk["avg_launch_ms"],
                           "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        # every step stopped before the timed last sweep of its first chunk
        out["roofline"] = None
    if not batch and not gs and not args.no_paper_criterion:
        out["paper_criterion"] = paper_criterion(args, p, mesh, x0, v0, stream, prec, corr, X)
    if gs:
        if not args.no_compare:
            out["comparisons"] = compare_gs(args, p, mesh, x0, v0, stream, corr, prec)
    elif not args.no_compare:
        out["comparisons"] = compare(args, p, mesh, ss, batch, x0, v0, stream, corr, prec)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, float(sweeps.mean()))
    return out if rank == 0 else None


def paper_criterion(args, p, mesh, x0, v0, stream, prec, corr, X):
    """The paper's own stopping test (Sec. 8): the scene normalised into a unit cube, stop
    when the positions change by less than 1e-3 between two consecutive sweeps (2-norm over
    the free DOFs), the residual test still on at 1e-4; same step, cap and GPU. Steps from
    the same initial state as the timed run, CUDA events around them."""
    L = length_scale(args, X)
    o = p.step_opts(precision=prec, correction=corr, max_sweeps=args.max_sweeps, rel_tol=1e-4,
                    dx_tol=args.dx_tol, length_scale=L)
    x, v = x0.clone(), v0.clone()
    n = max(1, min(args.steps, 5))
    mesh.step(x.clone(), v.clone(), o, stream)
    ms, reps = timed_steps(mesh, x, v, o, n, stream)
    return {"dx_tol": args.dx_tol, "length_scale_m": L, "steps": n, "ms_per_step": round(ms / n, 3),
            "sweeps_per_step": float(np.mean([q["sweeps"] for q in reps])),
            "stopped_dx": int(sum(q["stopped_dx"] for q in reps)),
            "converged_rel_1e-4": int(sum(q["converged"] for q in reps)),
            "rel_residual_max": float(max(q["rel"] for q in reps)),
            "ls_rejects_per_step": float(np.mean([q["rejects"] for q in reps]))}


def compare(args, p, mesh, ss, batch, x0, v0, stream, corr, prec):
    """The same step on the same GPU in the forms the method is measured against: the FP64
    single-scene form and uncorrected Jacobi (one step each, CUDA events); for the batch, a
    sequential FP64 loop over the scenes one mesh at a time."""
    import torch
    res = {}
    if not batch:
        for name, o in [("fp64_single_scene", p.step_opts(precision=p.FP64, correction=corr,
                                                           max_sweeps=args.max_sweeps, rel_tol=1e-4)),
                        ("jacobi_uncorrected", p.step_opts(precision=prec, correction=p.CORR_OFF,
                                                           max_sweeps=args.max_sweeps, rel_tol=1e-4))]:
            x, v = x0.clone(), v0.clone()
            ms, reps = timed_steps(mesh, x, v, o, 1, stream)
            res[name] = {"ms_per_step": round(ms, 3), "sweeps": int(reps[0]["sweeps"]),
                         "converged": int(reps[0]["converged"]), "rel_residual": float(reps[0]["rel"]),
                         "ms_per_sweep": round(ms / max(reps[0]["sweeps"], 1), 5)}
        return res
    elem, w, u, _ = mesh.precompute_export()
    cubs = split_cubature(elem, w, u.reshape(len(elem), -1), ss)
    o = p.step_opts(precision=p.FP64, correction=corr, max_sweeps=args.max_sweeps, rel_tol=1e-4)
    tot, sweeps, conv = 0.0, [], 0
    for s, c in zip(ss, cubs):
        g = p.Mesh.from_scene(s)
        g.precompute_import(*c)
        x = torch.tensor(s.X, dtype=torch.float64, device=x0.device)
        v = torch.tensor(s.v0, dtype=torch.float64, device=x0.device)
        g.step(x.clone(), v.clone(), o, stream)   # first use: device buffers
        ms, reps = timed_steps(g, x, v, o, 1, stream)
        tot += ms
        sweeps.append(reps[0]["sweeps"])
        conv += reps[0]["converged"]
        g.close()
    res["fp64_per_scene_loop"] = {"ms_per_step": round(tot, 3), "scenes": len(ss), "converged_scenes": conv,
                                  "sweeps_median": float(np.median(sweeps)), "sweeps_max": int(max(sweeps))}
    return res


def compare_gs(args, p, mesh, x0, v0, stream, corr, prec):
    """The Gauss-Seidel step against its FP64 form and its uncorrected form on the same GPU
    (one step each)."""
    res = {}
    for name, o in [("gs_fp64", p.step_opts(precision=p.FP64, correction=corr, max_sweeps=args.max_sweeps,
                                            rel_tol=1e-4)),
                    ("gs_uncorrected", p.step_opts(precision=prec, correction=p.CORR_OFF,
                                                   max_sweeps=args.max_sweeps, rel_tol=1e-4))]:
        x, v = x0.clone(), v0.clone()
        ms, reps = timed_steps(mesh, x, v, o, 1, stream, gs=True)
        res[name] = {"ms_per_step": round(ms, 3), "gs_sweeps": int(reps[0]["sweeps"]),
                     "converged": int(reps[0]["converged"]), "rel_residual": float(reps[0]["rel"])}
    return res


def run_cloth(args, rank, world, local_rank):
    """The cloth workload (reading R26): a square StVK cloth with quadratic bending, held at
    two corners and released under gravity, stepped by jgs2_cloth_step to rel_tol 1e-4
    (capped). Default size: 1001 x 1001 vertices, 2M triangles (the scale of the paper's cloth
    example). No correction and no contact (the cloth path has neither)."""
    import torch
    import paper_2506_06494_b300 as p
    import scenes
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n = args.cloth_n
    s = scenes.cloth_scene(n=n, size=1.0)
    c = p.Cloth.from_scene(s)
    prec = p.FP32 if args.precision == "fp32" else p.FP64
    opts = p.step_opts(precision=prec, max_sweeps=args.max_sweeps, rel_tol=1e-4, check_every=16)
    stream = torch.cuda.current_stream()
    x = torch.tensor(s.X, dtype=torch.float64, device=dev)
    v = torch.tensor(s.v0, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        c.step(x, v, opts, stream)
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    clocks = Clocks(vis.split(",")[local_rank] if vis else str(local_rank))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = [c.step(x, v, opts, stream) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    sweeps = np.array([r.sweeps for r in reps], dtype=float)
    # e2e: host state, copies inside the timed region
    xh = torch.tensor(s.X, dtype=torch.float64).pin_memory()
    vh = torch.tensor(s.v0, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xd, vd = xh.to(dev, non_blocking=True), vh.to(dev, non_blocking=True)
        c.step(xd, vd, opts, stream)
        xh.copy_(xd)
        vh.copy_(vd)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    V, F, H = s.X.shape[0], s.tris.shape[0], c.n_hinges
    fb = 4 if prec == p.FP32 else 8
    # records read by the gather and the line-search pass (triangles 20, hinges 12 words),
    # per-vertex state through gather (u, dz, m/h^2, D written), pass and update
    bytes_sweep = 2 * (F * 20 * fb + H * 12 * fb) + V * (15 * fb + 13 * fb + 12 * fb)
    ms_sweep = ms / max(1.0, float(np.mean(sweeps)))
    hbm, hkind = peaks()
    return {
        "metric": METRIC, "value": ms, "unit": "ms/step", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == p.FP32 else "f64", "data": "synthetic",
        "config": {"workload": "cloth", "scene": f"{n}x{n}-vertex square cloth, 1 m, two corners held, gravity",
                   "vertices": V, "triangles": F, "hinges": H, "rel_tol": 1e-4, "max_sweeps": args.max_sweeps,
                   "correction": "none (cloth path)", "line_search": True, "parallelism": f"replicas x{world}",
                   "l2": "per-sweep working set larger than L2 (126 MB); no flush"},
        "sweeps_per_step": float(np.mean(sweeps)), "converged_steps": int(sum(r.converged for r in reps)),
        "max_rel_residual": float(max(r.rel_residual for r in reps)),
        "e2e": {"value": e2e_ms, "unit": "ms/step", "h2d_bytes_per_step": 2 * V * 24, "d2h_bytes_per_step": 2 * V * 24},
        "gpu_launches": int(sum(4 * r.sweeps + 6 for r in reps)),
        "clocks": ck,
        "sweep_roofline": {"bound": "hbm", "achieved": round(bytes_sweep / ms_sweep / 1e6, 1), "peak": hbm,
                           "unit": "GB/s", "frac": round(bytes_sweep / ms_sweep / 1e6 / hbm, 4),
                           "bytes_per_sweep": int(bytes_sweep), "ms_per_sweep": round(ms_sweep, 5),
                           "peak_source": f"{hkind} (MEASURED_PEAKS.json hbm_gbs)"},
    }


def run_adjoint(args, rank, world, local_rank):
    """Differentiation workload: a rollout of the 20x20x100-vertex beam (214,434 tets) with
    per-element Young's moduli E_e = 1e7 U(0.5, 1.5) (seed 0), loss = sum |x_n - xbar_n|^2
    against a rollout with uniform E = 1e7, gradient dL/dE through jgs2_step_adjoint with
    state checkpoints every 5 steps (segments recomputed in the backward pass). Timed: the
    backward pass per step (recomputation + adjoint solve + parameter derivative), with the
    forward rollout reported beside it. Forward and adjoint run at --precision (vectors and
    kernels; reductions FP64-class either way)."""
    import torch
    import paper_2506_06494_b300 as p
    from paper_2506_06494_b300 import autograd as AG
    import scenes
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    s = scenes.beam_scene()
    mesh = p.Mesh.from_scene(s)
    if args.cubature == "precompute":
        mesh.precompute(n_cub=args.n_cub, gpu=int(args.precompute_gpu))
    else:
        mesh.precompute_import(*scenes.random_cubature(s.X, s.tets, s.pinned, args.n_cub, seed=0, w_max=0.5,
                                                       u_sigma=0.2))
    prec = p.FP32 if args.precision == "fp32" else p.FP64
    opts = p.step_opts(precision=prec, max_sweeps=args.max_sweeps, rel_tol=1e-4)
    aopts = p.adjoint_opts(precision=prec, max_iters=5000, rel_tol=1e-6)
    n = args.rollout_steps
    x0 = torch.tensor(s.X, dtype=torch.float64, device=dev)
    v0 = torch.tensor(s.v0, dtype=torch.float64, device=dev)
    E0 = torch.full((s.n_tets,), 1e7, dtype=torch.float64, device=dev)
    with torch.no_grad():
        xbar, _ = AG.rollout(mesh, x0, v0, E0, n, 5, opts, aopts)
    rng = np.random.default_rng(0)
    E = torch.tensor(1e7 * rng.uniform(0.5, 1.5, s.n_tets), dtype=torch.float64, device=dev, requires_grad=True)
    fwd, bwd, gnorm = [], [], None
    for rep in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xn, _ = AG.rollout(mesh, x0, v0, E, n, 5, opts, aopts)
        loss = ((xn - xbar) ** 2).sum()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        E.grad = None
        loss.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if rep >= args.warmup:
            fwd.append((t1 - t0) * 1e3 / n)
            bwd.append((t2 - t1) * 1e3 / n)
        gnorm = float(E.grad.norm())
    ms_b = float(np.median(bwd))
    return {"metric": "adjoint ms per rollout step (backward: recompute + adjoint + dL/dE)", "value": ms_b,
            "unit": "ms/step", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision.replace("fp", "f"), "data": "synthetic",
            "config": {"workload": "adjoint", "scene": "20x20x100-vertex Kuhn beam 0.02x0.02x0.1 m, 214,434 tets, "
                       "E_e = 1e7 U(0.5,1.5)", "rollout_steps": n, "checkpoint_every": 5,
                       "cubature": args.cubature, "max_sweeps": args.max_sweeps, "adjoint_rel_tol": 1e-6},
            "forward_ms_per_step": float(np.median(fwd)), "loss": float(loss), "grad_norm": gnorm}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="jgs2", choices=["jgs2", "reference"])
    ap.add_argument("--workload", default="spheres", choices=["spheres", "beam", "cube", "batch", "adjoint", "cloth"])
    ap.add_argument("--rollout-steps", type=int, default=30, help="adjoint workload: steps of the rollout")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--correction", default="asm", choices=["asm", "elem", "off"])
    ap.add_argument("--n-cub", type=int, default=4)
    ap.add_argument("--max-sweeps", type=int, default=2000)
    ap.add_argument("--ref-sweeps", type=float, default=2000.0,
                    help="sweeps per step assumed by the reference arm's scaling")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-paper-criterion", action="store_true")
    ap.add_argument("--coupling", type=int, default=0,
                    help="1: contact-aware correction (Sec. 7 two-way coupling across bodies in contact)")
    ap.add_argument("--gs", type=int, default=0,
                    help="1: Gauss-Seidel steps (greedy colouring, group precompute) on a single scene without contact")
    ap.add_argument("--persistent", type=int, default=0,
                    help="batch workload: one persistent cooperative launch per chunk of sweeps (1) or one launch "
                         "per kernel in graph-captured chunks (0, the faster on B300)")
    ap.add_argument("--dx-tol", type=float, default=1e-3,
                    help="the paper's position-change tolerance on the unit-normalised scene")
    ap.add_argument("--friction", type=float, default=0.0,
                    help="wall friction coefficient on the spheres workload (lagged IPC friction; 0 = none)")
    ap.add_argument("--precompute-gpu", type=int, default=1, choices=[0, 1],
                    help="1: the precompute's multi-RHS solves run on the GPU (FP32 substitutions, FP64 refinement)")
    ap.add_argument("--cloth-n", type=int, default=1001, help="cloth workload: vertices per side")
    ap.add_argument("--n-spheres", type=int, default=10)
    ap.add_argument("--contact", type=int, default=1, choices=[0, 1, 2],
                    help="spheres workload: 0 no contact, 1 IPC log barrier, 2 quadratic penalty")
    ap.add_argument("--n-scenes", type=int, default=256)
    ap.add_argument("--cubature", default="precompute", choices=["precompute", "synthetic"],
                    help="synthetic: seeded random records instead of the precompute (kernel profiling only)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    runner = {"adjoint": run_adjoint, "cloth": run_cloth}.get(args.workload, run_jgs2)
    out = runner(args, rank, world, local_rank)
    if out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
