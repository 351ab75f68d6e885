"""Benchmark of the nonlinear-damage ADER-DG step on GB300.

One bench step = one time step of the whole method (predictor, corrector with
volume/source/face terms and update, point source, receivers) over the
196,608-tet N=4 jittered two-layer periodic cube with a dip-slip point source
and 64 receivers (synthetic, seeded).  Metric: element-updates/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N>1 (torchrun, one process per GPU) runs N independent replicas of the
workload (the method is not sharded across GPUs here); value = all ranks'
element updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

# The CPU baseline (the FP64 oracle) runs on one host thread: BLAS thread pools
# are pinned before numpy loads so that the reported core count is exact.
for _var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "element-updates/s (FP32, N=4)"
UNIT = "element-updates/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def n_modes(N):
    return (N + 1) * (N + 2) * (N + 3) // 6


def algorithmic_flops(N):
    """FLOPs per element update of each kernel of the method as this library
    formulates it (FMA = 2 flops): Taylor terms on their nonzero modes (degree
    <= N-i), (N+1)^3 volume nodes, (N+1)^2 face nodes and N+1 time nodes, each
    interior face's flux once (a closed mesh has 2 faces per element).
    Returns {"predictor", "faces", "corrector"}."""
    L, NQ, NF, NT = n_modes(N), (N + 1) ** 3, (N + 1) ** 2, N + 1
    LR = [n_modes(N - i) for i in range(N + 1)]
    SH = sum(LR[1:])
    pred = (2 * 6 * NQ * L + 20 * NQ + 2 * NQ * L                       # damage rate at t_n, projection
            + sum(2 * 27 * LR[i] * LR[i - 1] + 192 * LR[i] for i in range(1, N + 1)))   # CK
    per_face = (2 * NF * 2 * (11 * L + 9 * SH)                          # traces, both sides, all orders
                + 2 * NF * NT * (18 * N + 2)                            # Taylor sums at the time nodes
                + NF * NT * 165)                                        # two normal fluxes + Rusanov
    faces = 2 * per_face
    corr = (2 * NQ * (8 * L + 6 * SH) + 2 * NQ * NT * (6 * N + 1)       # strains, damage at the nodes
            + NQ * NT * 50 + NQ * 63                                    # CDM stress/rate, stress terms
            + 20 * L * NQ                                               # volume and source projections
            + 18 * L * L + 63 * L + 6 * (L + SH)                        # strain rows (modal)
            + 2 * L * 4 * NF * 9 + 10 * L)                              # face projection, update
    return {"predictor": pred, "faces": faces, "corrector": corr}


def algorithmic_bytes(N):
    """Minimum HBM bytes per element update: read and write the FP32 state
    (10 L floats each) plus 176 B of geometry, material and connectivity."""
    return 8 * 10 * n_modes(N) + 176


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
               "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
               "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self._proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self._proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self._proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_baseline(workload, steps=1, max_seconds=None):
    """The FP64 oracle, as it stands, on a bounded sample of the workload: one
    z-layer of hexahedral cells (6 n^2 elements) advanced one step from a
    seeded state on the full mesh.  Returns (element-updates/s, sample text, threads)."""
    from oracle import Oracle
    mesh, mat, N = workload["mesh"], workload["material"], workload["order"]
    n = mesh.cells[0]
    rows = np.arange(6 * n * n * (n // 2), 6 * n * n * (n // 2 + 1))      # one z-layer of cells
    t_setup = time.perf_counter()
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat, face_rows=rows)
    o.set_sources(workload["sources"])
    setup = time.perf_counter() - t_setup
    rng = np.random.default_rng(0)
    Q = rng.normal(size=(mesh.n_elem, o.L, 10)) * 1e-6
    dt = o.cfl_dt()
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step(Q, dt, t=0.3, rows=rows)
    el = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        threads = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:          # threadpoolctl absent: the pinned BLAS thread count
        threads = int(os.environ.get("OPENBLAS_NUM_THREADS", "1"))
    sample = (f"{rows.size} elements (one z-layer of cells of the {mesh.n_elem}-tet mesh), "
              f"{steps} step(s), numpy FP64 with {threads} BLAS thread(s); setup {setup:.1f}s excluded")
    return rows.size * steps / el, sample, threads, el


def cpu_adjoint_baseline():
    """The FP64 oracle's forward step and its discrete adjoint (oracle.adjoint,
    as it stands) timed on a bounded sample of the adjoint workload: its jittered
    cube at 4 cells per side (384 tets) and degree 3, one step each from a seeded
    damaged state.  Returns (adjoint element-steps/s, forward element-steps/s,
    sample text, threads)."""
    import math
    from oracle import Oracle, mode_list
    from oracle.adjoint import step_vjp
    from synthetic import workload_adjoint
    w = workload_adjoint(n=4, order=3, steps=1)
    mesh, N = w["mesh"], w["order"]
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, w["material"])
    rng = np.random.default_rng(0)
    deg = np.array([sum(m) for m in mode_list(N)])
    Q = rng.normal(size=(mesh.n_elem, o.L, 10)) * (0.5 ** deg)[None, :, None]
    Q[..., :6] *= 2e-4
    Q[..., 6:9] *= 0.6
    Q[..., 9] = 0.0
    Q[:, 0, 9] = 0.03 / math.sqrt(6.0)
    lam = rng.normal(size=Q.shape)
    dt = 0.5 * o.cfl_dt()
    t0 = time.perf_counter()
    o.step(Q, dt)
    t1 = time.perf_counter()
    step_vjp(o, Q, dt, lam)
    t2 = time.perf_counter()
    try:
        from threadpoolctl import threadpool_info
        threads = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:          # threadpoolctl absent: the pinned BLAS thread count
        threads = int(os.environ.get("OPENBLAS_NUM_THREADS", "1"))
    sample = (f"{mesh.n_elem} tets of the adjoint workload's cube at n = 4, N = {N}, one forward step and one "
              f"adjoint step, numpy FP64 with {threads} BLAS thread(s)")
    return mesh.n_elem / (t2 - t1), mesh.n_elem / (t1 - t0), sample, threads


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from synthetic import workload_c2
    w = workload_c2(n=args.n, order=args.order)
    vals, total = [], 0.0
    for _ in range(args.warmup):
        cpu_baseline(w, steps=1)
    for _ in range(args.steps):
        v, sample, threads, el = cpu_baseline(w, steps=1)
        vals.append(v)
        total += el
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * w["mesh"].n_elem / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(w, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _config(w, args):
    return {"workload": w["name"], "elements": w["mesh"].n_elem, "order": w["order"],
            "modes": n_modes(w["order"]), "fields": 10, "sources": len(w["sources"]),
            "receivers": int(len(w["receivers"])), "l2_policy": "inputs larger than L2 "
            "(state 2x and predictor buffers > 129 MB at N=4); no flush", "parallelism": f"replicas{args.gpus}",
            "predictor": f"picard{args.picard_iterations}" if getattr(args, "picard_iterations", 0) > 0 else "ck"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=32, help="cells per cube side (32 -> 196,608 tets)")
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3"],
                    help="c2: 196,608-tet two-layer cube (the benchmark); c3: ~4.35 M-tet regional-shaped box")
    ap.add_argument("--ensemble-members", type=int, default=0,
                    help="also time the ensemble workload (N=3, this many members) against one member")
    ap.add_argument("--adjoint-steps", type=int, default=800,
                    help="steps of the adjoint workload (82,944 tets, N=3, 40 snapshots) whose gradient is "
                         "timed against its forward step; 0 skips it")
    ap.add_argument("--adjoint-n", type=int, default=24,
                    help="cells per cube side of the adjoint workload (24 -> 82,944 tets)")
    ap.add_argument("--picard-iterations", type=int, default=0,
                    help="run the Picard predictor with this many iterations after the CK one (0: CK alone); "
                         "the flop counts stay the CK step's")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    import paper_2502_09714_gb300 as dgpkg
    from synthetic import workload_c2

    rank, world, local = _dist()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dgpkg.build()
    if args.workload == "c3":
        from synthetic.regional import workload_c3
        w = workload_c3(order=args.order)
    else:
        w = workload_c2(n=args.n, order=args.order)
    mesh, mat, N = w["mesh"], w["material"], w["order"]
    E, L = mesh.n_elem, n_modes(N)
    stream = torch.cuda.current_stream()
    bc = mesh.face_bc if np.any(mesh.face_bc != 0) else None
    s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, face_bc=bc, cfl=w["cfl"], stream=stream)
    s.set_material(mat)
    if args.picard_iterations > 0:
        s.set_predictor("picard", args.picard_iterations)
    s.set_sources(w["sources"])
    s.set_receivers(w["receivers"])
    s.set_state(np.zeros((E, 10, L), np.float32), 0.0)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    s.step(args.warmup)
    barrier()
    s.profile(True)
    launches0 = s.stats()["kernel_launches"]
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(args.steps)
    ev1.record(stream)
    barrier()
    clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = s.profile_read()
    s.profile(False)
    launches = s.stats()["kernel_launches"] - launches0
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * E * args.steps / (ms_max * 1e-3)

    # end to end through the public API: pinned host state in, one step, state out
    hq = torch.zeros((E, 10, L), dtype=torch.float32).pin_memory()
    hq_np = hq.numpy()
    out = torch.empty_like(hq).pin_memory()
    out_np = out.numpy()
    s.get_state(out=out_np)
    hq_np[...] = out_np
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        s.step_host(hq_np, out_np)        # upload, one step, download (transfers overlap the step)
    barrier()
    e2e_s = time.perf_counter() - t0
    te = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = world * E * args.e2e_steps / float(te.item())

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    peaks, peak_kind = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12    # TFLOP/s
    flops = algorithmic_flops(N)
    kavg = {k: v["total_ms"] / max(1, v["launches"]) for k, v in prof.items()}
    dom = max(("predictor", "faces", "corrector"), key=lambda k: prof[k]["total_ms"])
    dom_ms = kavg[dom]
    achieved = flops[dom] * E / (dom_ms * 1e-3) / 1e12
    traffic = _traffic_per_launch(dom, N, E)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(w, args),
        "roofline": {"kernel": _kernel_name(dom, N), "bound": "alu", "achieved": achieved,
                     "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                     "traffic": traffic,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (recipe unit counts, max clock)",
                     "flops_per_element": flops[dom], "avg_ms": dom_ms},
        "kernels": {k: {"launches": v["launches"], "avg_ms": kavg[k],
                        "tflops": (flops[k] * E / (kavg[k] * 1e-3) / 1e12) if k in flops and kavg[k] > 0 else None}
                    for k, v in prof.items()},
        "hbm": {"algorithmic_bytes_per_element": algorithmic_bytes(N),
                "achieved_gbs": algorithmic_bytes(N) * value / world / 1e9,
                "peak_gbs": peaks.get("hbm_gbs"),
                "frac": algorithmic_bytes(N) * value / world / 1e9 / float(peaks.get("hbm_gbs", 6800.0))},
        "step_flops": dict(flops, per_element_total=sum(flops.values()),
                           achieved_tflops=sum(flops.values()) * value / world / 1e12),
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(hq.numel() * 4),
                "d2h_bytes_per_step": int(out.numel() * 4), "steps": args.e2e_steps},
    }
    if args.ensemble_members > 1:
        line["ensemble"] = run_ensemble(args, dgpkg, torch, stream)
    if args.adjoint_steps > 0:
        line["adjoint"] = run_adjoint(args, dgpkg, torch, stream)
        if not args.no_cpu_baseline and world == 1:
            va, vf, sample, threads = cpu_adjoint_baseline()
            line["adjoint"]["cpu_baseline"] = {
                "value": va, "unit": "element-adjoint-steps/s", "forward_value": vf,
                "adjoint_to_forward_step": vf / va, "cores": threads, "kind": "oracle", "sample": sample}
    if not args.no_cpu_baseline and world == 1:
        v, sample, threads, _ = cpu_baseline(w, steps=1)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}
    print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_ensemble(args, dgpkg, torch, stream, steps=10, warmup=3):
    """Per-member throughput of the ensemble form (all members advance in one
    set of launches per step) against the same mesh run with one member."""
    from synthetic import workload_c4
    w = workload_c4(n=args.n, members=args.ensemble_members)
    mesh, mat, N, M = w["mesh"], w["material"], w["order"], w["members"]
    E, L = mesh.n_elem, n_modes(N)
    rate = {}
    for members in (1, M):
        s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, cfl=w["cfl"], stream=stream, members=members)
        if members == 1:
            m1 = mat.copy()
            m1[:, 4:6] = w["member_xi0_cd"][0]
            s.set_material(m1)
        else:
            s.set_material(mat, w["member_xi0_cd"])
        s.set_sources(w["sources"])
        s.set_receivers(w["receivers"])
        shape = (E, 10, L) if members == 1 else (members, E, 10, L)
        q = torch.zeros(shape, dtype=torch.float32, device="cuda")
        s.set_state(q, 0.0)
        s.step(warmup)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        rate[members] = E * members * steps / (ev0.elapsed_time(ev1) * 1e-3)
        s.close()
        del q
    return {"workload": w["name"], "members": M, "order": N, "elements": E, "steps": steps,
            "member_updates_per_s": rate[M], "single_member_updates_per_s": rate[1],
            "per_member_ratio": rate[M] / rate[1]}


def run_adjoint(args, dgpkg, torch, stream, snapshots=40, fwd_steps=50):
    """Cost of the receiver-misfit gradient (discrete adjoint with binomial
    checkpointing) on the adjoint workload against the forward step of the same
    mesh: the reference traces come from an untimed run with the perturbed
    parameters; the forward step is timed over fwd_steps steps, the gradient as
    one dg_adjoint_gradient call after a short warm-up call."""
    from synthetic import workload_adjoint
    n = args.adjoint_steps
    w = workload_adjoint(n=args.adjoint_n, steps=n)
    mesh, N = w["mesh"], w["order"]
    E, L = mesh.n_elem, n_modes(N)
    s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, cfl=w["cfl"], stream=stream)
    zero = np.zeros((E, 10, L), np.float32)
    s.set_material(w["material_ref"])
    s.set_sources(w["sources"])
    s.set_receivers(w["receivers"])
    s.set_state(zero, 0.0)
    dt = s.dt
    s.step(n, dt)
    ref = s.read_receivers()[:n]
    s.set_material(w["material"])
    s.set_state(zero, 0.0)
    s.step(5, dt)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(fwd_steps, dt)
    ev1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = ev0.elapsed_time(ev1) / fwd_steps
    s.set_state(zero, 0.0)
    k = min(n, 20)
    s.adjoint_gradient(ref[:k], k, dt, snapshots=min(snapshots, k))
    torch.cuda.synchronize()
    ev0.record(stream)
    J, gx, gc, info = s.adjoint_gradient(ref, n, dt, snapshots=snapshots, info=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    total = ev0.elapsed_time(ev1)
    # the whole history kept in HBM (n + 1 states): no forward step is recomputed
    store_all = None
    state_bytes = E * 4 * ((10 * L + 3) // 4 * 4)
    free, _ = torch.cuda.mem_get_info()
    if (n + 4) * state_bytes < 0.8 * free:
        s.set_state(zero, 0.0)
        torch.cuda.synchronize()
        ev0.record(stream)
        J2, _, _, info2 = s.adjoint_gradient(ref, n, dt, snapshots=n + 1, info=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        store_all = {"snapshots": n + 1, "state_gb": (n + 1) * state_bytes / 1e9,
                     "gradient_ms": ev0.elapsed_time(ev1),
                     "gradient_to_forward_run": ev0.elapsed_time(ev1) / (n * fwd_ms),
                     "forward_steps_run": info2["forward_steps"], "misfit": J2}
    s.close()
    adj = info["adjoint_ms"] / info["adjoint_steps"]
    return {"workload": w["name"], "elements": E, "order": N, "steps": n, "snapshots": snapshots,
            "forward_ms_per_step": fwd_ms, "adjoint_ms_per_step": adj, "adjoint_to_forward_step": adj / fwd_ms,
            "forward_steps_run": info["forward_steps"], "snapshot_copy_ms": info["copy_ms"],
            "gradient_ms": total, "gradient_to_forward_run": total / (n * fwd_ms), "misfit": J,
            "max_abs_grad_xi0": float(np.abs(gx).max()), "max_abs_grad_cd": float(np.abs(gc).max()),
            "store_all": store_all}


def _kernel_name(kind, N):
    """Name of the CUDA kernel that runs `kind` at degree N under the CDM (the
    kernels' last template argument 0: compiled for the CDM alone).  The
    corrector's volume evaluation runs on the tensor cores for 2 <= N <= 4
    unless bit 3 of DG_KERNEL_VARIANT selects the all-SIMT corrector."""
    variant = int(os.environ.get("DG_KERNEL_VARIANT", "1"))
    if kind == "corrector" and 2 <= N <= 4 and not (variant & 8):
        return f"k_corrector_tc<{N}, 0>"
    return f"k_{kind}<{N}, 0>"


def _kernel_source_digest():
    import hashlib
    p = os.path.join(ROOT, "paper_2502_09714_gb300", "csrc", "dg_step_kernels.cuh")
    with open(p, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _traffic_per_launch(kernel, N, E):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled
    to E elements; None when no capture exists or the kernel source changed
    since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("order") != N or d.get("kernel_source_sha256_16") != _kernel_source_digest():
        return None
    per = d.get("dram_bytes_per_element", {}).get(kernel)
    return None if per is None else per * E


if __name__ == "__main__":
    sys.exit(main())
