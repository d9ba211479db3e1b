"""Benchmark of the GPU finite-volume hot path: one streamer step = one Poisson solve to
relative residual 1e-8 + least-squares field + upwind/diamond transport update of n_e
and n_i, on the 3D electron drift-diffusion + Poisson workload of the learned-warm-start
configuration (unit cube, 100^3 jittered hexes x 6 Kuhn tetrahedra = 6,000,000 cells),
timed in the FP64 plain method (CG from the previous potential); beside it, on the same
mesh from the same state to the same residual, mixed precision, the learned warm start
(network trained on 2,000 solver-generated pairs from 20 seed positions) and the other
variants, with their errors against the FP64 run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0). --impl reference times the CPU oracle (the plain FP64
reference implementation of the method) on a bounded sample of the same workload.
Multi-GPU runs are independent replicas (the path does not shard; no collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per FV step + Poisson, learned vs plain CG at rel. residual 1e-8"
UNIT = "cell-updates/s"
K_MESH = 100                # 6 * 100^3 = 6,000,000 cells
MESH_SEED = 301
K_SMALL, SMALL_SEED = 50, 201   # the 750,000-cell FP64 workload, run as a labelled variant
RTOL = 1e-8
INNER_RTOL = 0.5            # inner CG reduction per outer step (Jacobi-scaled CG: measured fastest of
                            # 0.1-0.6 over 20 steps of this workload, FP64 and mixed)
ENSEMBLE_INNER_RTOL = 0.2   # the ensemble's: each outer step of its graph loop costs more (64 parts'
                            # tests); 0.5 measured 193 against 142 ms per step
ORACLE_SAMPLE_K = 12        # 10,368 cells, same recipe
N_SEEDS, N_HELD_OUT, TRAIN_STEPS = 20, 2, 100   # 20 x 100 = 2,000 (charge, phi) pairs
HELD_OUT_STEPS = 40
WORKLOAD = ("3D electron drift-diffusion + Poisson, FP64 plain method, on the 6M-cell mesh of the "
            "learned-warm-start workload: unit cube, 100^3 jittered hexes x 6 Kuhn tets (6,000,000 "
            "cells, mesh seed 301), seed at (0.5,0.5,0.9), V = 12.5 kV, Poisson to rel. residual 1e-8 "
            "each step (FP64 defect correction + FP64 inner CG on the Jacobi-scaled two-point operator "
            "halving its residual per outer step, warm start from the previous potential)")


def workload_text(args):
    text = WORKLOAD
    if args.inner > 0:
        text = text.replace("FP64 inner CG on the Jacobi-scaled two-point operator halving its residual "
                            "per outer step",
                            f"{args.inner} multigrid V-cycles per outer step")
    if args.prec == "mixed":
        text = text.replace("FP64 plain method", "mixed precision (FP32 transport and inner solve, "
                                                 "FP64 refinement), autotuned launch shapes")
        text = text.replace("FP64 inner CG", "FP32 inner CG")
    return text


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-transport", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip training the learned warm start (and its variants)")
    ap.add_argument("--headline-only", action="store_true",
                    help="time the headline step only (no variants, e2e, ensemble, transport or "
                         "CPU baseline); for profiling")
    ap.add_argument("--inner", type=int, default=0,
                    help="inner solve of the headline run: 0 conjugate gradients (default), "
                         "k > 0 k multigrid V-cycles per outer step")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "mixed"],
                    help="precision of the headline run: fp64 (the plain method, default) or mixed "
                         "(FP32 transport and inner CG, FP64 refinement to the same residual)")
    ap.add_argument("--transport-only", default=None, choices=["fp32", "fp64", "both"],
                    help="time only the transport kernels on the 6M-cell mesh (for profiling)")
    ap.add_argument("--cg-fixed", default=None,
                    help="comma-separated CG iteration counts: one Poisson solve on the 6M-cell FP64 mesh "
                         "per count, its single CG launch running exactly that many iterations (for "
                         "profiling the CG kernel's traffic per iteration)")
    ap.add_argument("--network-only", type=int, default=None, metavar="K",
                    help="time the learned start's training step and prediction on the K^3 x 6 mesh "
                         "(random inputs; for profiling the network kernels)")
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------------------
# CPU oracle (baseline leg and the reference arm): a plain single-threaded FP64 run
# ---------------------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from synth.workloads import StreamerCase, streamer_mesh
from oracle.geometry import Geometry
from oracle import streamer
k, steps, warm = {k}, {steps}, {warm}
m = streamer_mesh(k, seed={seed}); c = StreamerCase()
g = Geometry(m.dim, m.xyz, m.cells, m.bface_vert, m.bface_tag)
p = streamer.Params(V=c.V, mu=c.mu, A=c.A, B=c.B, De=c.De, centre=c.centre, sigma=c.sigma,
                    peak=c.peak, background=c.background)
ne, ni = c.initial(m); dt = c.dt(1.0 / k)
times = []
for s in range(warm + steps):
    t0 = time.perf_counter()
    ne, ni, phi, E, S = streamer.step(g, p, ne, ni, dt)
    t1 = time.perf_counter()
    if s >= warm:
        times.append(t1 - t0)
print(json.dumps({{"cells": int(g.n_cell), "times": times}}))
"""


def run_oracle(k, steps, warm):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    code = ORACLE_SNIPPET.format(root=ROOT, k=k, steps=steps, warm=warm, seed=MESH_SEED)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_sample_text(k, steps, cells):
    return (f"{steps} streamer step(s) of the same recipe on the k={k} mesh ({cells} cells) "
            f"by the CPU oracle (numpy/scipy FP64, SuperLU Poisson solve), one thread")


def reference_arm(args, world, rank):
    if rank != 0:
        return
    res = run_oracle(ORACLE_SAMPLE_K, args.steps, args.warmup)
    total = sum(res["times"])
    value = res["cells"] * len(res["times"]) / total
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / len(res["times"]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "sample_cells": res["cells"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": oracle_sample_text(ORACLE_SAMPLE_K, args.steps, res["cells"])},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="fvgb_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1])); smax.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash(*names):
    h = hashlib.sha256()
    for n in names:
        h.update(open(os.path.join(ROOT, "paper_2203_00925_gb300", "csrc", n), "rb").read())
    return h.hexdigest()[:16]


def cg_fixed(capi, device, torch, counts, mixed=False):
    """One Poisson solve per count on the 6M-cell workload mesh (FP64, or mixed: FP32 inner
    CG), whose single CG launch runs exactly that many iterations (tolerances that cannot be
    met, one outer step)."""
    from synth.workloads import StreamerCase, streamer_mesh
    case = StreamerCase()
    mesh = streamer_mesh(K_MESH, MESH_SEED)
    dm = device.DeviceMesh(mesh, [case.bc_ne(), case.bc_phi()], prec="mixed" if mixed else "fp64")
    ne0, ni0 = case.initial(mesh)
    e_over_eps0 = 1.602176634e-19 / 8.8541878128e-12
    f = dm.to_device(-e_over_eps0 * (ni0 * 1.001 - ne0), torch.float64)
    out = {}
    for its in counts:
        phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
        opts = capi.solve_opts(rtol=1e-30, inner_rtol=1e-30, maxit_inner=its, maxit_outer=1,
                               prec=capi.FVGB_FP32 if mixed else capi.FVGB_FP64)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, info = capi.fvgb_poisson_solve(dm.handle, 1, f, phi, opts, check=False)
        e1.record()
        torch.cuda.synchronize()
        out[str(its)] = {"inner_its": info.inner_its_total, "solve_ms": e0.elapsed_time(e1)}
    dm.free()
    return out


def network_only(capi, device, torch, k, reps=3):
    """Training step and prediction of the learned start on the k^3 x 6 mesh (random
    inputs), for the multilevel and the local architecture."""
    from paper_2203_00925_gb300 import learned
    from synth.workloads import StreamerCase, streamer_mesh
    case = StreamerCase()
    mesh = streamer_mesh(k, MESH_SEED)
    dm = device.DeviceMesh(mesh, [case.bc_ne(), case.bc_phi()], prec="mixed")
    g = torch.Generator(device="cuda").manual_seed(0)
    dq = torch.randn(dm.n_cell, dtype=torch.float64, device="cuda", generator=g) * 1e9
    ph = torch.randn(dm.n_cell, dtype=torch.float64, device="cuda", generator=g) * 1e3
    tg = torch.randn(dm.n_cell, dtype=torch.float64, device="cuda", generator=g) * 1e-2
    pred = torch.empty_like(dq)
    out = {"cells": dm.n_cell}
    for arch, ml in (("multilevel", True), ("local", False)):
        net = capi.fvgb_mpnn_create(dm.handle, 1, multilevel=ml)
        capi.fvgb_mpnn_set_params(net, learned.init_params(0, ml))
        capi.fvgb_mpnn_set_scales(net, case.V, 1e-6, 0.58, 1.4e-6)
        for name, fn in (("train_step", lambda: capi.fvgb_mpnn_train_step(net, dq, ph, tg, 1e-3)),
                         ("predict", lambda: capi.fvgb_mpnn_predict(net, dq, ph, pred))):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            out[f"{arch}_{name}_ms"] = e0.elapsed_time(e1) / reps
        capi.fvgb_mpnn_free(net)
    dm.free()
    return out


def profile_traffic(kernel, shash):
    """DRAM traffic of the kernel from the committed ncu summary, if it is for this source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
        e = d.get(kernel)
        if e and e.get("source_hash") == shash:
            return e
    except (OSError, ValueError):
        pass
    return None


TRANSPORT_K = 100          # 6 * 100^3 = 6,000,000 cells: every array well above L2
TRANSPORT_SEED = 301


def transport_kernels(capi, device, torch, stream, flush, precs, meshes=None, reps=10, warm=3):
    """The transport operators on the 6M-cell mesh, each timed alone between CUDA events
    with L2 flushed before every repetition; achieved GB/s from the algorithmic bytes
    (each array element counted once, gathered neighbour values as cache hits).
    ``meshes`` ({"fp32": ..., "fp64": ...}) reuses uploaded meshes of that mesh."""
    import numpy as np
    from synth.workloads import StreamerCase, streamer_mesh
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    hbm = float(peaks["hbm_gbs"])
    case = StreamerCase()
    mesh = streamer_mesh(TRANSPORT_K, TRANSPORT_SEED)
    out = {"mesh": f"unit cube, {TRANSPORT_K}^3 x 6 Kuhn tets, seed {TRANSPORT_SEED}",
           "peak_GBps": hbm, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
           "l2": "flushed before each repetition (256 MiB write, untimed)"}
    meshes = meshes or {}
    for prec in precs:
        own = prec not in meshes
        dm = device.DeviceMesh(mesh, [case.bc_ne(), case.bc_phi()], prec=prec) if own else meshes[prec]
        N, F, V, NN = dm.n_cell, dm.n_face, dm.n_vert, dm.n_nbr
        w = 8 if prec == "fp64" else 4
        rng = np.random.default_rng(1)
        cen = mesh.vertex_mean()
        u = dm.to_device(np.sin(cen @ np.array([2.1, 1.3, 2.9])) + 0.1 * rng.random(N) + 1.0)
        vel = dm.to_device(rng.normal(size=(3, N)))
        src = dm.to_device(rng.normal(size=N))
        g, uv, res = dm.empty(3, N), dm.empty(V), dm.empty(N)
        tc = capi.tcoef(vel=vel, diff=0.1, src=src, bcset=0)
        tcm = capi.tcoef(vel=vel, diff=0.1, src=src, bcset=0, recon=1)
        res_bytes = (4 * N * (4 + w) + N * w + V * w + F * (20 + 7 * w) + V * w
                     + N * (16 + 7 * w) + F * w)
        calls = {
            # node-neighbour indices + u + M^-1 (6) + centre (3) + gradient out (3)
            "gradient": (lambda: capi.fvgb_gradient(dm.handle, 1, u, g),
                         4 * NN + N * 13 * w),
            # star indices + weights (4 per cell) + u + vertex values out
            "vertex_values": (lambda: capi.fvgb_vertex_values(dm.handle, 0, u, uv),
                              4 * N * (4 + w) + N * w + V * w),
            # multiplicity-weighted variant: records (value, centre) + per-vertex sums over the
            # stars (star indices, 5 sums out) + per cell its vertices' sums and geometry
            "gradient_vertex": (lambda: capi.fvgb_gradient_vertex(dm.handle, 1, u, g),
                                N * (4 * w) + 4 * N * 4 + V * (4 + 3 * w + 5 * w)
                                + N * (16 + 6 * w + 3 * w) + V * (3 * w + 5 * w)),
            # vertex values, then per face L, R, A, B, C + 3 coefficients + area vector
            # (3) + flux, then cell_face (4) + fluxes + u, velocity (3), source, 1/mu, out
            "fv_residual": (lambda: capi.fvgb_fv_residual(dm.handle, tc, u, res), res_bytes),
            # MUSCL + Barth-Jespersen: + gradient, + limiter (cell_face, u, gradient in and
            # out, face centroids), + the reconstruction's gradient and centre reads
            "fv_residual_muscl": (lambda: capi.fvgb_fv_residual(dm.handle, tcm, u, res),
                                  res_bytes + 4 * NN + N * 13 * w
                                  + N * (16 + 7 * w) + 3 * w * F + 6 * w * N),
        }
        r = {"cells": N, "faces": F, "vertices": V, "node_neighbour_entries": NN}
        t_end = time.time() + 0.5                 # bring the clocks up before timing
        while time.time() < t_end:
            for fn, _ in calls.values():
                fn()
            torch.cuda.synchronize()
        for name, (fn, nbytes) in calls.items():
            for _ in range(warm):
                fn()
            ms = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            med = statistics.median(ms)
            r[name] = {"ms": med, "algorithmic_bytes": nbytes, "GBps": nbytes / med / 1e6,
                       "frac_of_measured_hbm": nbytes / med / 1e6 / hbm}
        out[prec] = r
        if own:
            dm.free()
    return out


ENSEMBLE_MESHES, ENSEMBLE_SEED, ENSEMBLE_STEPS = 64, 5000, 50


def ensemble_block(capi, device, torch, stream, warm, nets):
    """64 independent meshes (cell counts log-uniform in 20k-1M, own seed position and
    voltage each) packed into one index space and advanced together: mixed precision,
    autotuned launch shapes, each step one CUDA graph; every part's solve to 1e-8."""
    import numpy as np
    from synth.workloads import ensemble_cases, streamer_mesh
    cases = ensemble_cases(ENSEMBLE_MESHES, seed=ENSEMBLE_SEED)
    t0 = time.time()
    meshes = [streamer_mesh(k, seed) for k, seed, _ in cases]
    dm = device.DeviceMesh(meshes, [[c.bc_ne(), c.bc_phi()] for _, _, c in cases], prec="mixed",
                           ensemble=True)
    upload_s = time.time() - t0
    capi.fvgb_autotune(dm.handle)
    ne0 = np.concatenate([c.initial(m)[0] for m, (_, _, c) in zip(meshes, cases)])
    c0 = cases[0][2]
    dt = min(c.dt(1.0 / k) for k, _, c in cases)
    out = {"meshes": len(cases), "cells": dm.n_cell, "faces": dm.n_face,
           "cells_min_max": [int(min(m.n_cell for m in meshes)), int(max(m.n_cell for m in meshes))],
           "steps": ENSEMBLE_STEPS, "warmup": warm, "dt": dt, "build_and_upload_s": upload_s}
    runs = {"mixed_graph": (None, False, 0), "extrapolated_mixed_graph": (None, True, 0),
            "multigrid_extrapolated_mixed_graph": (None, True, 2)}
    if nets is not None:
        runs["learned_extrapolated_mixed_graph"] = (nets[True], True, 0)
    for name, (theta_sc, extrap, inner) in runs.items():
        net = None
        if theta_sc is not None:
            net = capi.fvgb_mpnn_create(dm.handle, 1, multilevel=theta_sc[2])
            capi.fvgb_mpnn_set_params(net, theta_sc[0])
            capi.fvgb_mpnn_set_scales(net, c0.V, *theta_sc[1])
        sp = capi.streamer_params(mu=c0.mu, A=c0.A, B=c0.B, De=c0.De, dt=dt, warm=net,
                                  extrapolate=extrap,
                                  solve=capi.solve_opts(rtol=RTOL, inner_rtol=ENSEMBLE_INNER_RTOL,
                                                        prec=capi.FVGB_FP32, inner=inner))
        ne, ni = dm.to_device(ne0), dm.to_device(ne0)
        phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
        capi.fvgb_streamer_reset(dm.handle)
        capi.fvgb_set_graph_mode(dm.handle, True)
        capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, warm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, ENSEMBLE_STEPS)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        rel, _, _ = capi.fvgb_solve_parts(dm.handle, dm.n_part)
        out[name] = {"ms_per_step": ms / ENSEMBLE_STEPS, "value": dm.n_cell * ENSEMBLE_STEPS / (ms / 1e3),
                     "max_rel_res_last_step_over_parts": float(np.max(rel)),
                     "max_rel_res": max(i["rel_res"] for i in infos),
                     "outer_its_per_step": sum(i["outer_its"] for i in infos) / len(infos),
                     "inner_cg_its_per_step_max_part": sum(i["inner_its_total"] for i in infos) / len(infos)}
        capi.fvgb_set_graph_mode(dm.handle, False)
        if net:
            capi.fvgb_mpnn_free(net)
    dm.free()
    return out


def gpu_arm(args, world, rank, local):
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2203_00925_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2203_00925_gb300 import capi, device
    from synth.workloads import StreamerCase, streamer_mesh

    if args.cg_fixed:
        print(json.dumps(cg_fixed(capi, device, torch, [int(x) for x in args.cg_fixed.split(",")],
                                  mixed=args.prec == "mixed")), flush=True)
        return
    if args.network_only:
        print(json.dumps(network_only(capi, device, torch, args.network_only)), flush=True)
        return
    if args.transport_only:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        precs = ["fp32", "fp64"] if args.transport_only == "both" else [args.transport_only]
        print(json.dumps(transport_kernels(capi, device, torch, torch.cuda.current_stream(),
                                           flush, precs)), flush=True)
        return
    t_start = time.time()

    def log(msg):
        print(f"[bench {time.time() - t_start:7.1f} s] {msg}", file=sys.stderr, flush=True)

    case = StreamerCase()
    mesh = streamer_mesh(K_MESH, MESH_SEED)
    mixed = args.prec == "mixed"
    bcs = [case.bc_ne(), case.bc_phi()]
    meshes = {}

    def mesh_for(prec):
        """The workload mesh uploaded once per precision ("fp64" or "mixed")."""
        if prec not in meshes:
            meshes[prec] = device.DeviceMesh(mesh, bcs, prec=prec)
            if prec != "fp64":
                capi.fvgb_autotune(meshes[prec].handle)
            log(f"uploaded the {prec} mesh")
        return meshes[prec]

    dm = mesh_for("mixed" if mixed else "fp64")
    N = dm.n_cell
    ne0, ni0 = case.initial(mesh)
    dt = case.dt(1.0 / K_MESH)
    sp = capi.streamer_params(mu=case.mu, A=case.A, B=case.B, De=case.De, dt=dt,
                              solve=capi.solve_opts(rtol=RTOL, inner_rtol=INNER_RTOL,
                                                    prec=capi.FVGB_FP32 if mixed else capi.FVGB_FP64,
                                                    inner=args.inner))
    ne, ni = dm.to_device(ne0), dm.to_device(ni0)
    phi = torch.zeros(N, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    capi.fvgb_streamer_reset(dm.handle)
    for _ in range(args.warmup):
        capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, 1)
    capi.fvgb_stats_enable(dm.handle, True)
    capi.fvgb_stats_get(dm.handle, reset=True)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    infos = []
    for s in range(args.steps):
        flush.zero_()                                   # evict L2 between steps (not timed)
        ev[s][0].record(stream)
        infos += capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, 1)
        ev[s][1].record(stream)
    barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    stats = capi.fvgb_stats_get(dm.handle, reset=True)
    capi.fvgb_stats_enable(dm.handle, False)
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * N * args.steps / (total_ms / 1e3)
    log(f"headline {total_ms / args.steps:.2f} ms/step")

    # ---- roofline of the dominant kernel: the persistent CG kernel ------------------------
    # Per CG iteration and cell: the p/q phase (ELL-4 indices 16 B, 4 coefficients of the
    # unit-diagonal scaled operator, r and its 4 neighbours as cache hits, p, q and x read and
    # written) and the r phase (r, q read, r written): 14 w + 16 bytes; flops 8 (operator) +
    # 12 (four updates, two dots). Per launch add the initial pass (r = D^-1/2 rhs, zeroed p,
    # q, x), the first operator apply and the final pass (x = D^-1/2 x): 13 w + 24 bytes and
    # 14 flops.
    # At 6M cells the iteration's working set (~860 MB FP64) is far above L2, so both the HBM
    # and the FP64-pipe views apply; the line reports the one with the larger fraction as the
    # bound and the other beside it.
    w = 4 if mixed else 8
    its, launches = stats["cg_iterations"], max(stats["cg_launches"], 1)
    per_launch_its = its / launches
    flops_per_launch = N * (per_launch_its * 20 + 14)
    bytes_per_launch = N * (per_launch_its * (14 * w + 16) + 13 * w + 24)
    avg_launch_s = stats["cg_ms"] / 1e3 / launches
    props = torch.cuda.get_device_properties(local)
    peak_tflops = props.multi_processor_count * 2 * 2 * 2.070e9 / 1e12
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    hbm = float(peaks["hbm_gbs"])
    ok = avg_launch_s > 0 and args.inner == 0          # multigrid runs launch no CG kernel
    achieved_tf = flops_per_launch / avg_launch_s / 1e12 if ok else None
    achieved_gbs = bytes_per_launch / avg_launch_s / 1e9 if ok else None
    kname = "k_cg<float,4>" if mixed else "k_cg<double,4>"
    # traffic: DRAM bytes of ncu captures of this kernel source on this mesh, launches with
    # fixed iteration counts giving a fixed part and a part per iteration, evaluated at this
    # run's average iterations per launch
    prof = profile_traffic(kname, source_hash("solver.cu"))
    traffic = (prof["dram_bytes_fixed"] + per_launch_its * prof["dram_bytes_per_iteration"]
               if prof and ok else None)
    common = {"kernel": kname, "traffic": traffic,
              "traffic_source": prof.get("source") if prof else None,
              "avg_launch_ms": avg_launch_s * 1e3, "iterations_per_launch": per_launch_its,
              "cg_share_of_step": stats["cg_ms"] / total_ms if world == 1 else None,
              "timing": "CUDA events on the launching stream around every CG launch of the timed steps"}
    hbm_view = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                "frac": achieved_gbs / hbm if ok else None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                "algorithmic_bytes_per_launch": bytes_per_launch}
    alu_view = {"bound": "alu", "achieved": achieved_tf, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved_tf / peak_tflops if ok else None,
                "peak_source": "derived FP64 peak: SMs x 2 FMA/clk x 2 flop x 2.07 GHz (nominal rate; "
                               "MEASURED_PEAKS.json has no FP64 figure)",
                "flops_per_launch": flops_per_launch}
    if mixed or not ok or hbm_view["frac"] >= alu_view["frac"]:
        roofline = {**hbm_view, **common, "alu_view": None if mixed else alu_view}
    else:
        roofline = {**alu_view, **common, "hbm_view": hbm_view}

    headline_only = args.headline_only
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))

    # ---- learned warm start (config: 2,000 (charge, phi) pairs from 20 seeded streamer
    # runs of the plain solver on this mesh; 18 seed positions train, 2 are held out) -------
    nets, learned_info = None, None
    want_learned = world == 1 and not args.no_variants and not args.no_learned and not headline_only
    if want_learned:
        from paper_2203_00925_gb300 import learned
        t_train0 = time.time()
        rng = np.random.default_rng(4000)
        seeds = [StreamerCase(centre=(rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7), rng.uniform(0.8, 0.95)))
                 for _ in range(N_SEEDS)]
        train_cases, held_out = seeds[:N_SEEDS - N_HELD_OUT], seeds[N_SEEDS - N_HELD_OUT:]
        dmx = mesh_for("mixed")
        gen = capi.solve_opts(rtol=RTOL, inner_rtol=INNER_RTOL, prec=capi.FVGB_FP32, inner=2)
        nets, learned_info = learned.train_streaming(
            dmx, mesh, train_cases, dt, TRAIN_STEPS, gen, case.V, log=log)
        learned_info["pairs_generated"] = N_SEEDS * TRAIN_STEPS
        learned_info["seed_positions"] = {"train": len(train_cases), "held_out": len(held_out),
                                          "stream": "numpy default_rng(4000), uniform [0.3,0.7]^2 x [0.8,0.95]"}
        learned_info["train_s"] = time.time() - t_train0
        log(f"trained the networks in {learned_info['train_s']:.1f} s")
        # held-out seed positions: the solves started from the learned guess against the same
        # starts without it (mixed precision, host-driven steps, every solve to 1e-8)
        ho = {}
        for name, kw in (("previous_phi", {}), ("learned", {"net": nets[False]}),
                         ("extrapolated", {"extrapolate": True}),
                         ("learned_extrapolated", {"net": nets[True], "extrapolate": True})):
            tot = {"inner": 0, "outer": 0, "ms": 0.0, "max_rel_res": 0.0, "accepted_steps": 0, "steps": 0}
            for c in held_out:
                r = learned.held_out_run(dmx, mesh, c, dt, HELD_OUT_STEPS, capi.solve_opts(
                    rtol=RTOL, inner_rtol=INNER_RTOL, prec=capi.FVGB_FP32), V=case.V, **kw)
                for key in ("inner", "outer", "ms", "accepted_steps", "steps"):
                    tot[key] += r[key]
                tot["max_rel_res"] = max(tot["max_rel_res"], r["max_rel_res"])
            ho[name] = tot
        ho["inner_ratio_learned_vs_previous_phi"] = ho["learned"]["inner"] / max(ho["previous_phi"]["inner"], 1)
        ho["inner_ratio_learned_extrapolated_vs_extrapolated"] = (
            ho["learned_extrapolated"]["inner"] / max(ho["extrapolated"]["inner"], 1))
        ho["note"] = (f"{len(held_out)} held-out seed positions x {HELD_OUT_STEPS} steps (steps 3.. counted), "
                      "mixed precision, host-driven; inner = CG iterations of the inner solves; "
                      "accepted_steps = steps whose learned start passed the residual check")
        learned_info["held_out"] = ho
        log("held-out evaluation done")

    # ---- variants on the same workload, same steps from the same initial state, all to the
    # same rtol; errors against the plain FP64 run -----------------------------------------
    variants = None
    if world == 1 and not args.no_variants and not headline_only:
        ref_ne = dm.to_host(ne)
        ref_phi = dm.to_host(phi)
        ref_ne_total = capi.fvgb_integral(dm.handle, ne)
        ref_q = capi.fvgb_integral(dm.handle, ni) - ref_ne_total
        plain_inner = sum(i["inner_its_total"] for i in infos) / len(infos)

        def run_variant(prec, graph, warm=None, extrap=False, inner=0, recon=0, stages=1,
                        dmv=None, meshv=None, casev=None, dtv=None):
            dmv = dmv or mesh_for(prec)
            meshv, casev, dtv = meshv or mesh, casev or case, dtv or dt
            net = None
            if warm is not None:
                theta, scales, ml = nets[extrap]
                net = capi.fvgb_mpnn_create(dmv.handle, 1, multilevel=ml)
                capi.fvgb_mpnn_set_params(net, theta)
                capi.fvgb_mpnn_set_scales(net, casev.V, *scales)
            spv = capi.streamer_params(
                mu=casev.mu, A=casev.A, B=casev.B, De=casev.De, dt=dtv, warm=net, extrapolate=extrap,
                recon=recon, stages=stages,
                solve=capi.solve_opts(rtol=RTOL, inner_rtol=INNER_RTOL, inner=inner,
                                      prec=capi.FVGB_FP64 if prec == "fp64" else capi.FVGB_FP32))
            a0, b0 = casev.initial(meshv)
            nev, niv = dmv.to_device(a0), dmv.to_device(b0)
            phiv = torch.zeros(dmv.n_cell, dtype=torch.float64, device="cuda")
            capi.fvgb_streamer_reset(dmv.handle)
            capi.fvgb_set_graph_mode(dmv.handle, graph)
            capi.fvgb_streamer_step(dmv.handle, spv, nev, niv, phiv, None, args.warmup)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infv = capi.fvgb_streamer_step(dmv.handle, spv, nev, niv, phiv, None, args.steps)
            e1.record(stream)
            barrier()
            ms = e0.elapsed_time(e1)
            capi.fvgb_set_graph_mode(dmv.handle, False)
            out = {"ms_per_step": ms / args.steps, "value": dmv.n_cell * args.steps / (ms / 1e3),
                   "max_rel_res": max(i["rel_res"] for i in infv),
                   "outer_its_per_step": sum(i["outer_its"] for i in infv) / len(infv),
                   "inner_its_per_step": sum(i["inner_its_total"] for i in infv) / len(infv)}
            if meshv is mesh:
                q = capi.fvgb_integral(dmv.handle, niv) - capi.fvgb_integral(dmv.handle, nev)
                out["speedup_vs_plain_fp64"] = total_ms / ms
                out["rel_err_vs_plain_fp64"] = {
                    "n_e": rel(dmv.to_host(nev), ref_ne), "phi": rel(dmv.to_host(phiv), ref_phi),
                    "total_charge_over_total_electrons": abs(q - ref_q) / abs(ref_ne_total)}
            if net:
                capi.fvgb_mpnn_free(net)
            log(f"variant {prec} graph={graph} warm={warm is not None} extrap={extrap} inner={inner}: "
                f"{out['ms_per_step']:.2f} ms/step")
            return out

        variants = {
            "note": ("same initial state and step count as the headline run, every Poisson solve to "
                     "rel. residual 1e-8; each variant times all its steps in one call between CUDA "
                     "events (no L2 flush between steps; the 6M-cell arrays are far above L2); "
                     "'mixed': FP32 transport and inner CG, FP64 refinement; 'graph': each step one "
                     "CUDA graph; 'extrapolated': the solve starts from 2 phi^{n-1} - phi^{n-2}; "
                     "'learned': the network's correction of the start (from the previous potential, "
                     "or of the extrapolation), kept per part only where it lowers the FP64 residual; "
                     "'multigrid': 2 smoothed-aggregation V-cycles per outer step instead of the inner "
                     "CG; 'muscl': MUSCL reconstruction with the Barth-Jespersen limiter; 'rk3': three "
                     "Runge-Kutta stages, a Poisson solve each"),
            "plain_fp64_inner_cg_its_per_step": plain_inner,
            "mixed": run_variant("mixed", False),
            "mixed_graph": run_variant("mixed", True),
            "extrapolated_fp64": run_variant("fp64", False, extrap=True),
            "extrapolated_mixed_graph": run_variant("mixed", True, extrap=True),
            "multigrid_extrapolated_mixed_graph": run_variant("mixed", True, extrap=True, inner=2),
            "muscl_multigrid_extrapolated_mixed_graph": run_variant("mixed", True, extrap=True, inner=2, recon=1),
            "rk3_multigrid_extrapolated_mixed": run_variant("mixed", False, extrap=True, inner=2, stages=3),
        }
        if nets is not None:
            variants.update({
                "learned_fp64": run_variant("fp64", False, warm=True),
                "learned_mixed_graph": run_variant("mixed", True, warm=True),
                "learned_extrapolated_fp64": run_variant("fp64", False, warm=True, extrap=True),
                "learned_extrapolated_mixed_graph": run_variant("mixed", True, warm=True, extrap=True),
            })
        # the 750,000-cell FP64 workload (the small 3D configuration; its arrays fit in L2)
        small = streamer_mesh(K_SMALL, SMALL_SEED)
        dms = device.DeviceMesh(small, bcs, prec="fp64")
        variants["plain_fp64_750k"] = run_variant("fp64", False, dmv=dms, meshv=small,
                                                  dtv=case.dt(1.0 / K_SMALL))
        variants["plain_fp64_750k"]["mesh"] = (f"unit cube, {K_SMALL}^3 x 6 Kuhn tets (750,000 cells), "
                                               f"seed {SMALL_SEED}; its working set fits in L2")
        dms.free()

    # ---- end to end through the public API with host buffers ------------------------------
    e2e = None
    if not args.no_e2e and not headline_only:
        rt = dm.real
        hne = torch.from_numpy(ne0.copy()).to(rt).pin_memory()
        hni = torch.from_numpy(ni0.copy()).to(rt).pin_memory()
        hphi = torch.zeros(N, dtype=torch.float64).pin_memory()
        u_ne, u_ni, i_ne, i_ni = (torch.empty(N, dtype=rt, device="cuda") for _ in range(4))
        u_phi, i_phi = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(2))
        triples = ((hne, u_ne, i_ne), (hni, u_ni, i_ni), (hphi, u_phi, i_phi))
        io_bytes = sum(h.numel() * h.element_size() for h, _, _ in triples)

        def e2e_step():
            for h, u, i in triples:
                u.copy_(h, non_blocking=True)
                capi.fvgb_permute(dm.handle, u, i, 1, u.element_size(), True)
            capi.fvgb_streamer_step(dm.handle, sp, i_ne, i_ni, i_phi, None, 1)
            for h, u, i in triples:
                capi.fvgb_permute(dm.handle, i, u, 1, u.element_size(), False)
                h.copy_(u, non_blocking=True)

        capi.fvgb_streamer_reset(dm.handle)
        for _ in range(args.warmup):
            e2e_step()
        barrier()
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for s in range(args.steps):
            flush.zero_()
            ev2[s][0].record(stream)
            e2e_step()
            ev2[s][1].record(stream)
        barrier()
        e2e_ms = sum(a.elapsed_time(b) for a, b in ev2)
        if world > 1:
            t = torch.tensor([e2e_ms], device="cuda", dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_ms = float(t.item())
        e2e = {"value": world * N * args.steps / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes}
        log("e2e done")

    ensemble = None
    if world == 1 and not args.no_ensemble and not headline_only:
        ensemble = ensemble_block(capi, device, torch, stream, args.warmup,
                                  nets if variants is not None else None)
        log("ensemble done")

    transport = None
    if world == 1 and not args.no_transport and not headline_only:
        transport = transport_kernels(capi, device, torch, stream, flush, ["fp32", "fp64"],
                                      meshes={"fp32": mesh_for("mixed"), "fp64": mesh_for("fp64")})
        log("transport kernels done")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not headline_only:
        steps_cpu = 5
        res = run_oracle(ORACLE_SAMPLE_K, steps_cpu, 0)
        v = res["cells"] * len(res["times"]) / sum(res["times"])
        cpu = {"value": v, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
               "sample": oracle_sample_text(ORACLE_SAMPLE_K, steps_cpu, res["cells"])}
        log("CPU baseline done")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32" if mixed else "f64",
            "data": "synthetic", "config": {"workload": workload_text(args),
                       "cells": N, "faces": dm.n_face,
                       "node_neighbour_entries": dm.n_nbr, "poisson_rtol": RTOL,
                       "l2": "flushed between timed steps (256 MiB write, untimed); the 6M-cell arrays "
                             "are far above L2",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "outer_its_per_step": sum(i["outer_its"] for i in infos) / len(infos),
                       "inner_cg_its_per_step": sum(i["inner_its_total"] for i in infos) / len(infos),
                       "max_rel_res": max(i["rel_res"] for i in infos)},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "learned": learned_info,
            "variants": variants,
            "ensemble": ensemble,
            "transport_kernels": transport,
            "gpu_launches": stats["kernel_launches"],
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    for d in meshes.values():
        d.free()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        reference_arm(args, world, rank)
    else:
        gpu_arm(args, world, rank, local)


if __name__ == "__main__":
    main()
