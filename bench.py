#!/usr/bin/env python
"""Timesteps per second of the multilevel elastodynamics timestep on GB300.

One "step" is one implicit-Euler timestep of the whole scene: the complete
Newton loop (element evaluation, assembly, Galerkin coarse operator and its
Cholesky, preconditioned CG, filtered line search) until the Newton step
tolerance is met.  The workload is the seeded random voxel lattice (41^3
grid, p = 0.55, largest component: 224,226 tets, 72,931 vertices) dropped
at 1 m/s from 0.05 m onto a ground plane with the point-plane barrier; it
reaches the plane during the third step, and warm-up steps advance the same
trajectory, so the timed steps are in contact.

Arms:
  ours (default)     mixed precision (FP32 H and PCG, FP64 gradient, norms,
                     energies and coarse Cholesky) with the two-level
                     preconditioner built from the SMS basis.  Also reported:
                     the plain FP64 block-Jacobi PCG path on the same state,
                     the per-step displacement error between the two, the
                     end-to-end rate through the host-pointer entry point, the
                     dominant kernel's roofline and the oracle's CPU rate.
  --impl reference   the FP64 CPU oracle timed on the host cores on a bounded
                     sample of the same workload (see cpu_sample()).

Multi-GPU: the timestep does not shard across GPUs here, so N > 1 runs N
independent replicas (one per rank) and reports their summed rate.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2508_13386_gb300.replicas import lpt_shards, max_over_ranks  # noqa: E402

# Newton count of the FP64 block-Jacobi GPU path on this workload's steps,
# used to scale the oracle's Newton iteration in the reference arm (the main
# arm measures it live)
REF_NEWTON = 11
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, one
# cold-cache ncu capture inside the timed step) of the dominant kernel on the
# 41^3 lattice, keyed by (kernel, precision); valid for the kernel version it
# was taken on and reported as null for anything else
MEASURED_TRAFFIC = {("k_pcg_spmv", "fp32", 41): 46753792}
METRIC = "timesteps/s at 220K tets: plain FP64 vs mixed+learned PCG at 1e-4 disp error"
UNIT = "timesteps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=41, help="lattice grid size (41: ~224K tets, 48: ~360K)")
    ap.add_argument("--handles", type=int, default=160)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--cycle", default="multiplicative", choices=["additive", "multiplicative"])
    ap.add_argument("--omega", type=float, default=0.0,
                    help="block-Jacobi damping in the cycle (0: 0.9 x 2 / the Lanczos estimate of lambda_max(D^-1 H))")
    ap.add_argument("--coarse-refresh", type=int, default=1000,
                    help="rebuild U^T H U every k Newton iterations (>= the Newton count: once per step)")
    ap.add_argument("--coarse-lag", type=int, default=7,
                    help="timesteps a coarse factor may be reused at a step's first Newton iteration (0: rebuilt every step)")
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="plain FP64 steps timed for comparison (the mixed step error is checked on each)")
    ap.add_argument("--newton-tol", type=float, default=1e-3,
                    help="Newton step tolerance of the mixed arm (the FP64 arm uses 1e-10); the per-step "
                         "displacement error against the FP64 arm is measured and reported")
    ap.add_argument("--pcg-rtol", type=float, default=1e-2,
                    help="PCG relative tolerance cap of the mixed arm (the forcing term can only tighten it)")
    ap.add_argument("--pcg-check-every", type=int, default=8,
                    help="PCG iterations launched between host convergence checks")
    ap.add_argument("--batch-pcg-rtol", type=float, default=1e-2,
                    help="batch64: PCG relative tolerance cap (the per-mesh FP64 check is reported)")
    ap.add_argument("--paper-steps", type=int, default=3,
                    help="steps timed with the paper's inexact direction (20 CG refinement iterations, 1e-3 m/s)")
    ap.add_argument("--learned-steps", type=int, default=480,
                    help="training timesteps of the learned warm start (seeded drops of the same lattice, 40 steps "
                         "each; 0 skips the learned arm)")
    ap.add_argument("--contact-steps", type=int, default=4,
                    help="steps timed on the two-lattice stack with mesh-mesh contact (0 skips the arm)")
    ap.add_argument("--contact-grid", type=int, default=24, help="lattice grid of each body of the stack")
    ap.add_argument("--cubature-steps", type=int, default=0,
                    help="steps timed with the cubature coarse operator (Sec. 3.8; its host precompute takes "
                         "minutes on the lattice, so the default run leaves it out)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-pointer end-to-end pass")
    ap.add_argument("--persistent", type=int, default=0, choices=[0, 1],
                    help="1: PCG iterations in one persistent cooperative kernel per solve")
    ap.add_argument("--blocks-per-sm", type=int, default=0, help="persistent kernel blocks per SM (0: library default)")
    ap.add_argument("--workload", default="lattice", choices=["lattice", "batch64", "stack"],
                    help="lattice: the 220K-tet scene (the metric); batch64: 64 independent lattices "
                         "of 2K-60K tets in one batched solve; stack: the two-lattice stack with mesh-mesh "
                         "contact alone (--steps timed steps)")
    ap.add_argument("--batch-precond", default="two_level", choices=["two_level", "jacobi"],
                    help="batch64: per-mesh SMS bases with the two-level cycle, or block Jacobi")
    ap.add_argument("--profile-run", action="store_true",
                    help="only warm-up and timed steps (for ncu: the timed steps sit in NVTX range 'mls_timed')")
    return ap.parse_args()


def workload(grid):
    import synth
    return synth.lattice_scene(n=grid, seed=3, v_down=1.0)


def workload_desc(args, scene):
    return (f"lattice{args.grid}^3 p=0.55 seed 3: {scene.n_tets} tets, {scene.n_verts} verts, "
            f"E log-uniform 1e5-1e8 (32 Voronoi cells), ground barrier dhat=1e-3 kappa=1e5, "
            f"implicit Euler h=1/60, dropped at 1 m/s from 0.05 m (timed steps {args.warmup}..)")


def cpu_sample(scene, x_t, v_t, newton_iters, threads, pcg_iters_known=None, pcg_cap=1000):
    """Time the oracle on the host cores on a bounded sample of one timestep,
    from the state the timed GPU steps start from: its first Newton iteration
    in full -- E, gradient and PSD-projected Hessian with the element loops on
    ``threads`` threads, the Jacobi-PCG solve of H d = -g to the oracle's own
    tolerance (relative residual 1e-13), and the filtered line search.  The
    timestep estimate is ``newton_iters`` such iterations (the Newton count of
    the FP64 GPU path on the same step: the same projected Newton iteration).
    The element evaluation is also timed on one thread.  With
    ``pcg_iters_known`` (the iteration count of a full solve from the same
    state, measured earlier) the solve runs ``pcg_cap`` iterations and its
    time is scaled to that count.  Returns a dict."""
    from oracle import ip, newton, pcg
    t_all = time.perf_counter()
    p = ip.Problem(scene, x_t=x_t, v_t=v_t, threads=threads)
    x = newton.initial_guess(p)
    ta = time.perf_counter()
    E0 = p.energy(x)
    g = p.gradient(x)
    H = p.hessian(x)
    tb = time.perf_counter()
    diag = H.diagonal()
    cap = 200000 if pcg_iters_known is None else min(pcg_cap, pcg_iters_known)
    d, info = pcg.pcg(lambda v: H @ v, -g.ravel(), lambda r: r / diag, rtol=1e-13, max_iter=cap)
    tc = time.perf_counter()
    if pcg_iters_known is not None and info["iters"] > 0:
        tc = tb + (tc - tb) * pcg_iters_known / info["iters"]
        info = dict(info, iters=pcg_iters_known)
    d = d.reshape(-1, 3)
    d[p.pinned] = 0.0
    t_ls = time.perf_counter()
    newton.line_search(p, x, d, g, E0)
    td = tc + (time.perf_counter() - t_ls)
    p1 = ip.Problem(scene, x_t=x_t, v_t=v_t, threads=1)
    te = time.perf_counter()
    p1.energy(x)
    p1.gradient(x)
    p1.hessian(x)
    t_eval1 = time.perf_counter() - te
    it_s = td - ta
    step_s = newton_iters * it_s
    desc = (f"oracle, first Newton iteration of the timed start state on the full {scene.n_tets}-tet lattice: "
            f"E, gradient and projected Hessian {tb - ta:.2f}s on {threads} threads ({t_eval1:.2f}s on one), "
            f"Jacobi-PCG to 1e-13 {tc - tb:.2f}s ({info['iters']} iterations, converged {info['converged']}), "
            f"line search {td - tc:.2f}s; timestep = {newton_iters:g} such iterations (the FP64 GPU path's "
            f"Newton count on the same step)")
    return {"value": 1.0 / step_s, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
            "newton_iteration_s": it_s, "eval_s_threads": tb - ta, "eval_s_one_thread": t_eval1,
            "pcg_iters": int(info["iters"]), "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "spent_s": time.perf_counter() - t_all}


def cpu_model():
    """The host CPU's model name (or architecture) for the report."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_error_estimate(scene, x_t, v_t, x1, threads):
    """Displacement error of a GPU step x1 from (x_t, v_t) against the
    oracle's minimiser, estimated by the oracle's Newton correction at x1:
    |H^-1 g(x1)| / |x1 - x_t| with the oracle's gradient and projected Hessian
    (Jacobi-PCG to 1e-3 relative residual), as the full-size parity test
    does."""
    from oracle import ip, pcg
    p = ip.Problem(scene, x_t=x_t, v_t=v_t, threads=threads)
    if not p.feasible(x1):
        return float("inf")
    g = p.gradient(x1).ravel()
    H = p.hessian(x1)
    diag = H.diagonal()
    e, _ = pcg.pcg(lambda u: H @ u, g, lambda r: r / diag, rtol=1e-3, max_iter=5000)
    return float(np.linalg.norm(e) / np.linalg.norm(x1 - x_t))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.samples = []
        self.proc = None
        self.index = index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi's start-up (driver and NVML initialisation) stalls the
            # GPU host API for up to ~0.1 s: let it finish before timing starts
            t_end = time.perf_counter() + 10.0
            while not self.samples and time.perf_counter() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if len(s) > 2 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) > 2 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def spmv_bytes(solver_meta, precision):
    """Algorithmic bytes of one launch of the PCG product kernel: H's blocks
    (9 values + a 4-byte column index each), the row lengths, z read once and
    p, q each read and written (3 components per vertex)."""
    nnzb, n = solver_meta["nnzb"], solver_meta["n"]
    sv = 8 if precision == "fp64" else 4
    sm = {"fp64": 8, "fp32": 4, "bf16": 2}[precision]
    return nnzb * (9 * sm + 4) + 4 * n + 5 * 3 * n * sv


def pcg_iteration_bytes(meta, precision, cycle):
    """Algorithmic bytes of one PCG iteration of the persistent kernel: every
    array each phase must touch, once (products: H's blocks, column indices
    and row lengths, the gathered vector counted once; restriction and
    prolongation: one 4-coefficient row and an index per vertex-handle pair;
    the coarse solve: both triangular factors)."""
    n, nnzb, nb, rc = meta["n"], meta["nnzb"], meta["basis_nnz"], meta["rc"]
    sv = 8 if precision == "fp64" else 4
    sm = {"fp64": 8, "fp32": 4, "bf16": 2}[precision]
    H = nnzb * (9 * sm + 4) + 4 * n
    vec = 3 * sv * n
    dinv = 9 * sv * n
    restrict = nb * (7 * sv + 4) + (n + 1) * 4
    prolong = nb * (4 * sv + 4) + (n + 1) * 4
    coarse = rc * (rc + 1) * sv
    if cycle == "jacobi":
        return H + 5 * vec + 7 * vec + dinv
    if cycle == "additive":
        return H + 5 * vec + 7 * vec + dinv + restrict + coarse + prolong + 3 * vec
    return 3 * H + 5 * vec + (7 * vec + dinv) + 3 * vec + restrict + coarse + prolong + 2 * vec + (3 * vec + dinv)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    scene = workload(args.grid)
    vals = []
    threads = os.cpu_count() or 1
    known = None
    for k in range(args.warmup + args.steps):
        # the first sample solves in full; later ones run 1000 PCG iterations
        # and scale to the first one's count (same state, same system)
        res = cpu_sample(scene, scene.x0, scene.v0, newton_iters=REF_NEWTON, threads=threads,
                         pcg_iters_known=known)
        known = res["pcg_iters"]
        if k >= args.warmup:
            vals.append(res["value"])
        desc = res["sample"] + ("; PCG time of later samples scaled from 1000 iterations" if k else "")
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(args, scene)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    print(json.dumps(line))


def _sms_job(job):
    """One mesh's SMS basis (a spawned worker builds it serially)."""
    from paper_2508_13386_gb300 import basis as sms
    X, tets, E, m, seed = job
    B = sms.build_sms_basis(X, tets, E, m, seed=seed, workers=1)
    return {k: B[k] for k in ("origins", "vrow", "handle", "phi")}


def run_batch(args):
    """The 64-mesh workload: one step advances every mesh (one graph launch).
    Two-level PCG with per-mesh SMS bases (m = max(4, round(tets / 1400))
    handles each) or block Jacobi, in the chosen precision; reported per
    whole batch."""
    import torch
    import torch.distributed as dist
    import synth
    import paper_2508_13386_gb300 as mls
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    scenes = synth.batched_lattice_scenes()
    # several GPUs: each rank advances its share of the meshes (longest-
    # processing-time by tet count), no exchange during a step
    n_all, tets_all = len(scenes), sum(sc.n_tets for sc in scenes)
    scenes = [scenes[i] for i in lpt_shards([sc.n_tets for sc in scenes], world)[rank]]
    for sc in scenes:
        sc.x0 = sc.x0 - np.array([0.0, 0.0, 0.0495])   # start just above the plane: contact from step 1
    basis_s = 0.0
    bases = None
    if args.batch_precond == "two_level":
        import multiprocessing as mp
        jobs = [(sc.X, sc.tets, sc.E, max(4, int(round(sc.n_tets / 1400))), 1) for sc in scenes]
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
            bases = pool.map(_sms_job, jobs)
        basis_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    omega_b = args.omega if args.omega > 0 else 0.5   # the automatic damping is a single-mesh option
    b = mls.Batch(precision=args.precision, preconditioner=args.batch_precond, omega=omega_b,
                  newton_tol=args.newton_tol if args.precision != "fp64" else 1e-10,
                  pcg_rtol=args.batch_pcg_rtol if args.precision != "fp64" else 1e-4, stream=stream)
    b.upload_scenes(scenes)
    if bases is not None:
        b.upload_bases(bases)
    x = torch.as_tensor(np.concatenate([sc.x0 for sc in scenes]), device=dev).contiguous()
    v = torch.zeros_like(x)
    dx = torch.empty_like(x)
    h = scenes[0].dt
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        b.step(x, v, h, dx=dx)
        v.copy_(dx / h)
        x.add_(dx)
    torch.cuda.synchronize()
    x_s, v_s = x.clone(), v.clone()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos, stats = [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clocks:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            _, st, info = b.step(x, v, h, dx=dx)
            ev[k][1].record(stream)
            infos.append(info)
            stats.append(st)
            v.copy_(dx / h)
            x.add_(dx)
        torch.cuda.synchronize()
    total_s = sum(a.elapsed_time(c) for a, c in ev) / 1e3
    total_s = max_over_ranks(total_s, dist if world > 1 else None, dev)
    # accuracy of the timed settings: the step from the post-warm-up state
    # against an FP64 batch solved to Newton tolerance 1e-10, per mesh
    disp_err = None
    if args.precision != "fp64":
        ref = mls.Batch(precision="fp64", preconditioner=args.batch_precond, omega=omega_b, newton_tol=1e-10,
                        pcg_rtol=1e-4, stream=stream)
        ref.upload_scenes(scenes)
        if bases is not None:
            ref.upload_bases(bases)
        dxm, dxr = torch.empty_like(x), torch.empty_like(x)
        b.step(x_s.clone(), v_s.clone(), h, dx=dxm)
        ref.step(x_s.clone(), v_s.clone(), h, dx=dxr)
        dm, dr = dxm.cpu().numpy(), dxr.cpu().numpy()
        vo = b.vert_offsets
        errs = [float(np.linalg.norm(dm[vo[m]:vo[m + 1]] - dr[vo[m]:vo[m + 1]])
                      / max(np.linalg.norm(dr[vo[m]:vo[m + 1]]), 1e-300)) for m in range(len(vo) - 1)]
        disp_err = {"max": max(errs), "mean": float(np.mean(errs)), "meshes": len(errs), "steps": 1}
        ref.close()
    if rank != 0:
        if world > 1:
            dist.barrier()
        return
    tets = tets_all
    line = {
        "metric": "timesteps/s of a 64-mesh batch (every mesh advanced per step)", "value": args.steps / total_s,
        "unit": "timesteps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32+f64", "bf16": "bf16+f32+f64", "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"64 seeded lattices, {tets} tets total (2K-60K each), E in {{1e5, 1e9}}, ground "
                               f"barrier, IE h=1/60, started 0.5 mm above the plane",
                   "solver": (f"{args.precision} two-level PCG per mesh (SMS bases, "
                              f"{sum(len(B['origins']) for B in bases)} handles in all, multiplicative cycle), "
                              if bases is not None else f"{args.precision} block-Jacobi PCG per mesh, ")
                             + f"Newton step tolerance {args.newton_tol:g}, PCG tolerance cap {args.batch_pcg_rtol:g}, "
                               f"omega {omega_b:g}, one graph launch per step",
                   "l2": "flushed (256 MB write) before every timed step"},
        "mesh_steps_per_s": n_all * args.steps / total_s,
        "newton_rounds_per_step": float(np.mean([i["newton_rounds"] for i in infos])),
        "pcg_rounds_per_step": float(np.mean([i["pcg_rounds"] for i in infos])),
        "pcg_iters_per_step_sum_over_meshes": float(np.mean([sum(m["pcg_iters"] for m in st) for st in stats])),
        "mesh_status_ok": int(sum(all(m["status"] == 0 for m in st) for st in stats)),
        "disp_err_vs_fp64": disp_err,
        "gpu_launches": int(sum(i["kernel_launches"] for i in infos)),
        "graph_launches": int(sum(i["graph_launches"] for i in infos)),
        "tuned": {"spmv_lanes": infos[-1]["spmv_lanes"], "row_threads": infos[-1]["row_threads"],
                  "rows_per_thread": infos[-1]["rows_per_thread"], "tune_ms": infos[-1]["tune_ms"]},
        "clocks": clocks.summary(),
        "setup": {"basis_build_s": basis_s},
        "sharding": f"{n_all} meshes over {world} GPU(s), longest-processing-time by tet count"
                    if world > 1 else None,
    }
    print(json.dumps(line))
    if world > 1:
        dist.barrier()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "stack":
        return run_stack(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2508_13386_gb300 as mls
    from paper_2508_13386_gb300 import basis as sms

    scene = workload(args.grid)
    t0 = time.perf_counter()
    B = sms.build_sms_basis(scene.X, scene.tets, scene.E, args.handles, dirichlet=scene.dirichlet, seed=1)
    basis_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)

    def make(precision, precond):
        s = mls.Solver(precision=precision, preconditioner=precond, cycle=args.cycle, omega=args.omega,
                       newton_tol=args.newton_tol if precision != "fp64" else 1e-10,
                       pcg_rtol=args.pcg_rtol if precision != "fp64" else 1e-4, pcg_check_every=args.pcg_check_every,
                       coarse_refresh=args.coarse_refresh, persistent=bool(args.persistent),
                       persist_blocks_per_sm=args.blocks_per_sm, stream=stream, coarse_lag_steps=args.coarse_lag)
        s.setup_scene(scene)
        if precond == "two_level":
            s.upload_basis(B["origins"], B["vrow"], B["handle"], B["phi"])
        return s

    ours = make(args.precision, "two_level")
    h = scene.dt
    x = torch.as_tensor(scene.x0, device=dev).contiguous()
    v = torch.as_tensor(scene.v0, device=dev).contiguous()
    dx = torch.empty_like(x)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    def advance(solver, x, v):
        _, st = solver.newton_step(x, v, h, dx=dx)
        v.copy_(dx / h)
        x.add_(dx)
        return st

    x_prev, v_prev = x.clone(), v.clone()
    for _ in range(args.warmup):
        x_prev.copy_(x)
        v_prev.copy_(v)
        advance(ours, x, v)
    torch.cuda.synchronize()
    # every measured pass below (timed mixed steps, plain FP64 steps, the
    # end-to-end pass, the breakdown) starts from this state
    x_s, v_s = x.clone(), v.clone()
    # parity of the mixed step against the FP64 GPU path from the same state
    disp_err = None
    fp64 = None
    if not args.profile_run:
        fp64 = make("fp64", "jacobi")
        x_chk, v_chk = x.clone(), v.clone()
        dx64, st64 = fp64.newton_step(x_chk, v_chk, h)
        dxm, stm = ours.newton_step(x_chk, v_chk, h)
        disp_err = float(torch.linalg.norm(dxm - dx64) / torch.linalg.norm(dx64))
    torch.cuda.synchronize()
    # each measured pass of the mixed solver starts with a fresh coarse factor
    # (built at its first step, then reused as the settings allow), so the
    # passes see the same rebuild pattern
    ours.set_options()
    # timed region (no per-kernel events inside: they would split the chained
    # PCG launches)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.nvtx.range_push("mls_timed")
            ev[k][0].record(stream)
            _, st = ours.newton_step(x, v, h, dx=dx)
            ev[k][1].record(stream)
            torch.cuda.nvtx.range_pop()
            v.copy_(dx / h)
            x.add_(dx)
            stats.append(st)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # the dominant kernel's launches timed with CUDA events on the library's
    # stream over a replay of the timed steps (same start state, same inputs)
    x_end, v_end = x.clone(), v.clone()
    x.copy_(x_s)
    v.copy_(v_s)
    ours.set_options()
    ours.profile_enable(["spmv", "pcg_fused"])
    replay = []
    for k in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        advance(ours, x, v)
        e1.record(stream)
        replay.append((e0, e1))
    torch.cuda.synchronize()
    prof = ours.profile_read()
    ours.profile_enable([])
    replay_ms = float(np.mean([a.elapsed_time(b) for a, b in replay]))
    x.copy_(x_end)
    v.copy_(v_end)
    total_s = sum(step_ms) / 1e3
    total_s = max_over_ranks(total_s, dist if world > 1 else None, dev)
    value = world * args.steps / total_s
    # per kernel-class breakdown on one extra (untimed) step from the start state
    breakdown = None
    if not args.profile_run:
        ours.profile_enable(["elements", "assemble", "spmv", "pcg_update", "precond", "galerkin", "cholesky",
                             "linesearch", "pcg_fused"])
        xb, vb = x_s.clone(), v_s.clone()
        _, st_b = ours.newton_step(xb, vb, h)
        breakdown = {k: {"ms": round(ms, 3), "launches": n} for k, (ms, n) in ours.profile_read().items() if n}
        ours.profile_enable([])
    learned_res = None
    if not args.profile_run and args.learned_steps > 0:
        learned_res = learned_arm(args, scene, B, make, dev, stream, x_prev, v_prev, x_s, v_s, flush, fp64)
    # plain FP64 block-Jacobi PCG over the first steps of the same segment
    # and, from each of its states, the mixed step: the per-step relative
    # displacement error of the mixed arm against the plain FP64 step
    fp64_ms = []
    fp64_stats = []
    step_errs = []
    x.copy_(x_s)
    v.copy_(v_s)
    for k in range(0 if args.profile_run else args.fp64_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = fp64.newton_step(x, v, h, dx=dx)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_ms.append(e0.elapsed_time(e1))
        fp64_stats.append(st)
        dxm, _ = ours.newton_step(x.clone(), v.clone(), h)
        step_errs.append(float(torch.linalg.norm(dxm - dx) / torch.linalg.norm(dx)))
        v.copy_(dx / h)
        x.add_(dx)
    if step_errs:
        disp_err = max([disp_err] + step_errs) if disp_err is not None else max(step_errs)
    # the paper's inexact direction (Alg. 1, Alg. 2) over the first steps of
    # the same segment, and its error against the plain FP64 step
    paper = None
    if not args.profile_run and args.paper_steps > 0:
        pap = mls.Solver(precision=args.precision, preconditioner="two_level", cycle=args.cycle, omega=args.omega,
                         coarse_refresh=args.coarse_refresh, direction="paper", refine_iters=20, paper_tol=1e-3,
                         stream=stream)
        pap.setup_scene(scene)
        pap.upload_basis(B["origins"], B["vrow"], B["handle"], B["phi"])
        xp, vp = x_s.clone(), v_s.clone()
        dxp, _ = pap.newton_step(x_s.clone(), v_s.clone(), h)
        dx64, _ = fp64.newton_step(x_s.clone(), v_s.clone(), h)
        perr = float(torch.linalg.norm(dxp - dx64) / torch.linalg.norm(dx64))
        pms, pst = [], []
        for k in range(args.paper_steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st = pap.newton_step(xp, vp, h, dx=dx)
            e1.record(stream)
            torch.cuda.synchronize()
            pms.append(e0.elapsed_time(e1))
            pst.append(st)
            vp.copy_(dx / h)
            xp.add_(dx)
        paper = {"value": 1e3 / float(np.mean(pms)), "unit": UNIT, "ms_per_step": float(np.mean(pms)),
                 "steps": len(pms), "newton_iters_per_step": float(np.mean([s["newton_iters"] for s in pst])),
                 "cg_iters_per_step": float(np.mean([s["pcg_iters"] for s in pst])),
                 "disp_err_vs_fp64_first_step": perr,
                 "settings": "subspace direction from the factored Galerkin operator + 20 block-Jacobi CG "
                             "iterations; stop when sum_v |d_s,v| / (h n) < 1e-3 m/s"}
        # Alg. 2 as printed: affine level, block-Jacobi subspace PCG to 1e-4
        # with matrix-free products, the refinement count from the partitions'
        # edge hops (Sec. 3.7.2) and the lagged elastic Hessian
        hops, _, n_cg = sms.refinement_cg_iterations(scene.tets, B["partition"], B["handle_vertex"])
        lit = mls.Solver(precision=args.precision, preconditioner="two_level", cycle=args.cycle, omega=args.omega,
                         coarse_refresh=args.coarse_refresh, direction="paper_literal", refine_iters=n_cg,
                         paper_tol=1e-3, sub_rtol=1e-4, hessian_lag=True, stream=stream)
        lit.setup_scene(scene)
        lit.upload_basis(B["origins"], B["vrow"], B["handle"], B["phi"])
        dxl, _ = lit.newton_step(x_s.clone(), v_s.clone(), h)
        lerr = float(torch.linalg.norm(dxl - dx64) / torch.linalg.norm(dx64))
        xp, vp = x_s.clone(), v_s.clone()
        lms, lst = [], []
        for k in range(args.paper_steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st = lit.newton_step(xp, vp, h, dx=dx)
            e1.record(stream)
            torch.cuda.synchronize()
            lms.append(e0.elapsed_time(e1))
            lst.append(st)
            vp.copy_(dx / h)
            xp.add_(dx)
        paper["literal_alg2"] = {
            "value": 1e3 / float(np.mean(lms)), "unit": UNIT, "ms_per_step": float(np.mean(lms)), "steps": len(lms),
            "newton_iters_per_step": float(np.mean([s["newton_iters"] for s in lst])),
            "subspace_pcg_iters_per_step": float(np.mean([s["subspace_iters"] for s in lst])),
            "refine_cg_iters_per_step": float(np.mean([s["pcg_iters"] for s in lst])),
            "hessian_refreshes_per_step": float(np.mean([s["hessian_refreshes"] for s in lst])),
            "disp_err_vs_fp64_first_step": lerr,
            "settings": f"affine level + 12x12 block-Jacobi subspace PCG to 1e-4 (matrix-free U^T(H(Uq))), "
                        f"{n_cg} refinement CG iterations (mean partition edge hops {hops:.1f}), lagged elastic "
                        f"Hessian (refresh: step start, mean of 3 step sizes < 0.5, at most every 5 iterations); "
                        f"stop when sum_v |d_s,v| / (h n) < 1e-3 m/s"}
        lit.close()
    # end to end through the host-pointer entry point, the timed segment again:
    # state in pinned host memory, copied in and the step copied out by the
    # library every step, the state advanced on the host in place
    xh = torch.empty(x_s.shape, dtype=torch.float64, pin_memory=True).numpy()
    vh = torch.empty(v_s.shape, dtype=torch.float64, pin_memory=True).numpy()
    dxh = torch.empty(x_s.shape, dtype=torch.float64, pin_memory=True).numpy()
    xh[...] = x_s.cpu().numpy()
    vh[...] = v_s.cpu().numpy()
    e2e_steps = 0 if (args.no_e2e or args.profile_run) else args.steps
    e2e_stats, e2e_step_s = [], []
    ours.set_options()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        t1 = time.perf_counter()
        _, st = ours.newton_step_host(xh, vh, h, dx=dxh)
        np.divide(dxh, h, out=vh)
        np.add(xh, dxh, out=xh)
        e2e_step_s.append(time.perf_counter() - t1)
        e2e_stats.append(st)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * e2e_steps / e2e_s if e2e_steps else None
    # roofline of the dominant kernel: the persistent PCG kernel (or, with
    # one launch per phase, the PCG product)
    meta = {"nnzb": int(ours_meta_nnzb(ours)), "n": scene.n_verts, "basis_nnz": int(len(B["handle"])),
            "rc": 12 * len(B["origins"])}
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("hbm_gbs", 6800.0))
    pcg_total = sum(s["pcg_iters"] for s in stats)
    if args.persistent:
        k_ms, k_n = prof["pcg_fused"]
        per_iter = pcg_iteration_bytes(meta, args.precision, args.cycle)
        total_bytes = per_iter * pcg_total
        roof = {"kernel": "k_pcg_persistent", "bytes_per_iteration": per_iter, "iterations": pcg_total,
                "bytes_per_launch": total_bytes / max(k_n, 1)}
    else:
        k_ms, k_n = prof["spmv"]
        total_bytes = spmv_bytes(meta, args.precision) * k_n
        roof = {"kernel": "k_pcg_spmv", "bytes_per_launch": spmv_bytes(meta, args.precision)}
    achieved = total_bytes / (k_ms / 1e3) / 1e9 if k_n else None
    traffic = MEASURED_TRAFFIC.get((roof["kernel"], args.precision, args.grid))
    roof.update({"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                 "frac": (achieved / peak) if achieved else None, "traffic": traffic, "launches": k_n,
                 "avg_launch_us": 1e3 * k_ms / max(k_n, 1), "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                 "timing": "CUDA events around each launch over a replay of the timed steps",
                 "replay_ms_per_step": replay_ms})
    if rank != 0:
        if world > 1:
            dist.barrier()
        return
    cpu = None
    oracle_err = None
    if world == 1 and not args.no_cpu and not args.profile_run:
        nit = float(np.mean([s["newton_iters"] for s in fp64_stats])) if fp64_stats else REF_NEWTON
        threads = os.cpu_count() or 1
        xs_h, vs_h = x_s.cpu().numpy(), v_s.cpu().numpy()
        cpu = cpu_sample(scene, xs_h, vs_h, nit, threads)
        # the mixed step from the timed start state against the oracle
        dxm, _ = ours.newton_step(x_s.clone(), v_s.clone(), h)
        oracle_err = oracle_error_estimate(scene, xs_h, vs_h, xs_h + dxm.cpu().numpy(), threads)
    cub_res = None
    if not args.profile_run and args.cubature_steps > 0 and rank == 0:
        cub_res = cubature_arm(args, scene, B, make, x_s, v_s, flush, fp64, stream)
    contact_res = None
    if not args.profile_run and args.contact_steps > 0 and rank == 0:
        contact_res = contact_arm(args, dev, stream, flush)
    headline = "mixed two-level PCG (the learned start is reported in 'learned' and loses or does not gain)"
    ms_per_step = total_s * 1e3 / args.steps
    # the learned arm heads the line only if its start was taken and it is faster within the gate
    if (learned_res is not None and learned_res["warm_start_used"] > 0 and world * learned_res["value"] > value
            and learned_res["disp_err_vs_fp64"] is not None and learned_res["disp_err_vs_fp64"] <= 1e-4):
        headline = "mixed two-level PCG with the learned warm start"
        value = world * learned_res["value"]
        ms_per_step = learned_res["ms_per_step"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32+f64", "bf16": "bf16+f32+f64", "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": workload_desc(args, scene),
                   "solver": f"{args.precision} two-level PCG ({args.cycle}, "
                             + (f"omega {args.omega:g}), " if args.omega > 0 else "omega 0.9 x 2 / Lanczos lambda_max(D^-1 H)), ")
                             + f"SMS basis m={len(B['origins'])} "
                             f"(r={12 * len(B['origins'])}), coarse refresh every {args.coarse_refresh}"
                             + (f" and reused over {args.coarse_lag} further steps, " if args.coarse_lag else ", ")
                             + f"Newton step tolerance {args.newton_tol:g}, PCG tolerance cap {args.pcg_rtol:g}, "
                             + ("persistent PCG kernel" if args.persistent
                                else f"one launch per PCG phase, host check every {args.pcg_check_every}")
                             + "; each measured pass starts with a fresh coarse factor",
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "pcg_iters_per_s": pcg_total / total_s,
        "newton_iters_per_step": float(np.mean([s["newton_iters"] for s in stats])),
        "pcg_iters_per_step": pcg_total / args.steps,
        "coarse_builds_per_step": float(np.mean([s["coarse_builds"] for s in stats])),
        "step_ms": [round(t, 3) for t in step_ms],
        "smoother": dict(zip(("omega", "lambda_max_estimate"), ours.smoother_omega())),
        "disp_err_vs_fp64": disp_err,
        "disp_err_vs_fp64_steps": step_errs,
        "disp_err_vs_oracle_estimate": oracle_err,
        "headline_arm": headline,
        "learned": learned_res,
        "paper_direction": paper,
        "mesh_contact": contact_res,
        "cubature": cub_res,
        "fp64_plain": {"value": 1e3 / float(np.mean(fp64_ms)) if fp64_ms else None, "unit": UNIT,
                       "ms_per_step": float(np.mean(fp64_ms)) if fp64_ms else None,
                       "steps": len(fp64_ms),
                       "pcg_iters_per_step": float(np.mean([s["pcg_iters"] for s in fp64_stats])) if fp64_stats else None,
                       "newton_iters_per_step": float(np.mean([s["newton_iters"] for s in fp64_stats])) if fp64_stats else None},
        "e2e_detail": {"step_ms": [round(1e3 * t, 3) for t in e2e_step_s],
                       "pcg_iters_per_step": float(np.mean([s["pcg_iters"] for s in e2e_stats])) if e2e_stats else None,
                       "coarse_builds_per_step": float(np.mean([s["coarse_builds"] for s in e2e_stats]))
                       if e2e_stats else None},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 3 * 8 * scene.n_verts,
                "d2h_bytes_per_step": 3 * 8 * scene.n_verts},
        "roofline": roof,
        "clocks": clocks.summary(),
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "cpu_baseline": cpu,
        "setup": {"basis_build_s": basis_s},
        "breakdown_one_step": breakdown,
    }
    print(json.dumps(line))
    if world > 1:
        dist.barrier()


def cubature_arm(args, scene, B, make, x_s, v_s, flush, fp64, stream):
    """The headline arm's settings with the coarse operator built from the
    cubature H (Sec. 3.8; cubature.build_cubature: modal moment fitting,
    Alg. 3) on the same steps: host precompute time, elements kept, ms per
    step, kernel classes of one step with a coarse build, and the first
    step's displacement error against the FP64 GPU path."""
    import torch
    from paper_2508_13386_gb300 import cubature
    t0 = time.perf_counter()
    C = cubature.build_cubature(scene.X, scene.tets, B, seed=0)
    build_s = time.perf_counter() - t0
    sol = make(args.precision, "two_level")
    sol.upload_cubature(C["scale"])
    h = scene.dt
    x, v = x_s.clone(), v_s.clone()
    dx = torch.empty_like(x)
    dxc, _ = sol.newton_step(x_s.clone(), v_s.clone(), h)
    err, dx64 = None, None
    if fp64 is not None:
        dx64, _ = fp64.newton_step(x_s.clone(), v_s.clone(), h)
        err = float(torch.linalg.norm(dxc - dx64) / torch.linalg.norm(dx64))
    sol.set_options()
    ms, stats = [], []
    for k in range(args.cubature_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = sol.newton_step(x, v, h, dx=dx)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        stats.append(st)
        v.copy_(dx / h)
        x.add_(dx)
    sol.set_options()
    sol.profile_enable(["galerkin", "cholesky"])
    sol.newton_step(x_s.clone(), v_s.clone(), h)
    torch.cuda.synchronize()
    prof = sol.profile_read()
    sol.profile_enable([])
    sol.close()
    # the paper's own direction (Alg. 1, Alg. 2) solves with the coarse
    # operator: the same steps with and without the cubature
    import paper_2508_13386_gb300 as mls
    paper = {}
    for tag, use in (("without", False), ("with", True)):
        pap = mls.Solver(precision=args.precision, preconditioner="two_level", cycle=args.cycle, omega=args.omega,
                         coarse_refresh=args.coarse_refresh, direction="paper", refine_iters=20, paper_tol=1e-3,
                         stream=stream)
        pap.setup_scene(scene)
        pap.upload_basis(B["origins"], B["vrow"], B["handle"], B["phi"])
        if use:
            pap.upload_cubature(C["scale"])
        dxp, _ = pap.newton_step(x_s.clone(), v_s.clone(), h)
        perr = float(torch.linalg.norm(dxp - dx64) / torch.linalg.norm(dx64)) if fp64 is not None else None
        xp, vp = x_s.clone(), v_s.clone()
        pms, pst = [], []
        for k in range(args.cubature_steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st = pap.newton_step(xp, vp, h, dx=dx)
            e1.record(stream)
            torch.cuda.synchronize()
            pms.append(e0.elapsed_time(e1))
            pst.append(st)
            vp.copy_(dx / h)
            xp.add_(dx)
        pap.close()
        paper[tag] = {"value": 1e3 / float(np.mean(pms)), "ms_per_step": float(np.mean(pms)),
                      "newton_iters_per_step": float(np.mean([s["newton_iters"] for s in pst])),
                      "cg_iters_per_step": float(np.mean([s["pcg_iters"] for s in pst])),
                      "disp_err_vs_fp64_first_step": perr}
    return {"value": 1e3 / float(np.mean(ms)), "unit": UNIT, "ms_per_step": float(np.mean(ms)),
            "step_ms": [round(t, 3) for t in ms], "steps": len(ms),
            "paper_direction": paper,
            "elements": int(len(C["elem"])), "of_tets": int(scene.n_tets), "host_build_s": build_s,
            "pcg_iters_per_step": float(np.mean([s["pcg_iters"] for s in stats])),
            "newton_iters_per_step": float(np.mean([s["newton_iters"] for s in stats])),
            "disp_err_vs_fp64_first_step": err,
            "coarse_build_ms": {k: round(t, 3) for k, (t, n) in prof.items() if n}}


def run_stack(args):
    """The mesh-mesh contact workload alone (contact_arm with --steps timed
    steps after one warm-up step): one JSON line.  Rank 0 runs it; other
    ranks exit (the stack is one scene)."""
    import torch
    if int(os.environ.get("RANK", "0")) != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    args.contact_steps = args.steps
    r = contact_arm(args, dev, stream, flush)
    line = {"metric": "timesteps/s, two-lattice stack with mesh-mesh contact", "value": r["value"], "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32+f64", "bf16": "bf16+f32+f64", "fp64": "f64"}[args.precision],
            "data": "synthetic", "config": {"workload": r["workload"], "l2": "flushed before every timed step"},
            "mesh_contact": r}
    print(json.dumps(line))


def contact_arm(args, dev, stream, flush):
    """Mesh-mesh contact (the barrier between bodies and its CCD filter) on
    the two-lattice stack (synth.lattice_stack_scene): the upper lattice
    falls onto the lower one, which rests on the ground.  Same solver
    settings as the headline arm, with an SMS basis per body (64 handles
    each).  The first step is warm-up (the bodies meet during it); the
    next ``--contact-steps`` are timed with CUDA events, L2 flushed before
    each, then one more step is taken with the kernel-class timers on."""
    import torch
    import synth
    import paper_2508_13386_gb300 as mls
    from paper_2508_13386_gb300 import basis as sms
    scene, body = synth.lattice_stack_scene(args.contact_grid)
    origins, vrow, handle, phi = [], [0], [], []
    m0 = 0
    parts = []
    for b in (0, 1):
        vid = np.nonzero(body == b)[0]
        remap = -np.ones(scene.n_verts, np.int64)
        remap[vid] = np.arange(len(vid))
        keep = np.all(body[scene.tets] == b, axis=1)
        Bb = sms.build_sms_basis(scene.X[vid], remap[scene.tets[keep]], scene.E[keep], 64, seed=1)
        parts.append((vid, Bb, m0))
        m0 += len(Bb["origins"])
    # merge: vertex rows in global order, handle indices offset per body
    rows = [None] * scene.n_verts
    for vid, Bb, off in parts:
        for k, v in enumerate(vid):
            lo, hi = Bb["vrow"][k], Bb["vrow"][k + 1]
            rows[v] = (Bb["handle"][lo:hi] + off, Bb["phi"][lo:hi])
        origins.append(Bb["origins"])
    for v in range(scene.n_verts):
        handle.extend(rows[v][0].tolist())
        phi.extend(rows[v][1].tolist())
        vrow.append(len(handle))
    origins = np.vstack(origins)
    sol = mls.Solver(precision=args.precision, preconditioner="two_level", cycle=args.cycle, omega=args.omega,
                     newton_tol=args.newton_tol, pcg_rtol=args.pcg_rtol, pcg_check_every=args.pcg_check_every,
                     coarse_refresh=args.coarse_refresh, stream=stream, coarse_lag_steps=args.coarse_lag)
    sol.setup_scene(scene)
    sol.set_bodies(body, scene.dhat, scene.kappa)
    sol.upload_basis(origins, np.asarray(vrow, np.int32), np.asarray(handle, np.int32), np.asarray(phi))
    h = scene.dt
    x = torch.as_tensor(scene.x0, device=dev).contiguous()
    v = torch.as_tensor(scene.v0, device=dev).contiguous()
    dx = torch.empty_like(x)

    def step():
        _, st = sol.newton_step(x, v, h, dx=dx)
        v.copy_(dx / h)
        x.add_(dx)
        return st

    step()
    torch.cuda.synchronize()
    ms, stats = [], []
    for k in range(args.contact_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        stats.append(st)
    sol.profile_enable(["elements", "assemble", "spmv", "pcg_update", "precond", "galerkin", "cholesky",
                        "linesearch"])
    step()
    torch.cuda.synchronize()
    prof = sol.profile_read()
    sol.profile_enable([])
    gap = float((x[body == 1, 2].min() - x[body == 0, 2].max()).item())
    out = {"value": 1e3 / float(np.mean(ms)), "unit": UNIT, "ms_per_step": float(np.mean(ms)),
           "step_ms": [round(t, 3) for t in ms], "steps": len(ms),
           "workload": f"two {args.contact_grid}^3 lattices (seeds 3, 4): {scene.n_tets} tets, {scene.n_verts} "
                       f"verts; upper falls at 1 m/s from 5 mm onto the lower one resting on the ground; "
                       f"mesh-mesh and ground barrier dhat=1e-3 kappa=1e5; SMS basis 64 handles per body",
           "newton_iters_per_step": float(np.mean([s["newton_iters"] for s in stats])),
           "pcg_iters_per_step": float(np.mean([s["pcg_iters"] for s in stats])),
           "contact_pairs_last_assembly": [int(s["contact_pairs"]) for s in stats],
           "gap_after_m": gap,
           "breakdown_one_step": {k: {"ms": round(t, 3), "launches": n} for k, (t, n) in prof.items() if n}}
    sol.close()
    return out


def learned_arm(args, scene, B, make, dev, stream, x_prev, v_prev, x_s, v_s, flush, fp64):
    """The learned warm start on the benchmark segment.  Training data: seeded
    drops of the same lattice (learned.drop_loads: tilted gravity, random
    linear and angular velocity), 40 steps each, recorded by the solver
    itself; the network 3r -> 256 -> 256 -> r is trained on the GPU by the
    library's kernels.  Held out: the benchmark trajectory.  The warm-started
    solver takes the last warm-up step untimed (to fill its coarse-state
    history) and then the K timed steps from the main arm's start state,
    under the same protocol (L2 flush, CUDA events); its first step is
    compared with the FP64 step from the same state."""
    import torch
    import synth
    import paper_2508_13386_gb300 as mls
    from paper_2508_13386_gb300 import learned as L
    h = scene.dt
    gen = make(args.precision, "two_level")
    gen.warm_start_enable(True, record=True)
    n_traj = max(1, args.learned_steps // 40)
    t0 = time.perf_counter()
    X, T, _ = L.collect(gen, scene, n_traj=n_traj, n_steps=40, seed=7, device=dev)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    r = 12 * gen.m
    sizes = [3 * r, 256, 256, r]
    net = mls.MLP(sizes, synth.mlp_init(sizes, 0), max_batch=256, stream=stream)
    t0 = time.perf_counter()
    losses = L.train(net, X, T, epochs=80, batch=128, lr=1e-3, seed=1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    gen.close()
    ws = make(args.precision, "two_level")
    ws.set_forces(tuple(scene.gravity), scene.contact, scene.plane_n, scene.plane_o, scene.dhat, scene.kappa)
    ws.warm_start_enable(True)
    ws.warm_start_attach(net)
    x, v = x_prev.clone(), v_prev.clone()
    dx = torch.empty_like(x)
    ws.newton_step(x, v, h, dx=dx)   # fills the history q^t, q^{t-1}
    x.copy_(x_s)
    v.copy_(v_s)
    dx64, _ = fp64.newton_step(x_s.clone(), v_s.clone(), h)
    ws.set_options()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    first_err = None
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        _, st = ws.newton_step(x, v, h, dx=dx)
        ev[k][1].record(stream)
        if k == 0:
            first_err = float(torch.linalg.norm(dx - dx64) / torch.linalg.norm(dx64))
        v.copy_(dx / h)
        x.add_(dx)
        stats.append(st)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    return {"value": 1e3 * len(ms) / sum(ms), "unit": UNIT, "ms_per_step": sum(ms) / len(ms),
            "step_ms": [round(t, 3) for t in ms],
            "newton_iters_per_step": float(np.mean([st["newton_iters"] for st in stats])),
            "pcg_iters_per_step": float(np.mean([st["pcg_iters"] for st in stats])),
            "warm_start_used": int(sum(st["warm_start_used"] for st in stats)), "steps": len(ms),
            "disp_err_vs_fp64": first_err,
            "training": {"samples": int(X.shape[0]), "trajectories": n_traj, "epochs": 80,
                         "loss_first": losses[0], "loss_last": losses[-1], "data_s": round(t_data, 2),
                         "train_s": round(t_train, 2), "network": sizes,
                         "data": "seeded drops of the same lattice (tilted gravity, random linear and angular "
                                 "velocity), held out: the benchmark trajectory"}}


def ours_meta_nnzb(solver):
    return solver.get_hessian_nnzb()


if __name__ == "__main__":
    main()
