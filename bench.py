"""Benchmark of the nonlinear-damage ADER-DG step on GB300.

One bench step = one time step of the whole method (predictor, face fluxes,
corrector with the volume, damage-source and face terms and the update, point
sources, receivers).  The headline workload is the regional-shaped box: a
120 x 80 x 40 km graded tetrahedral mesh of about 4.35 M elements at degree 4,
with a soft ellipsoidal basin, a layered background, a free surface on top and
absorbing faces elsewhere, about 6000 sub-fault point sources of a planar
dipping fault and 64 surface receivers (synthetic, seeded).  Metric:
element-updates/s.  The line also carries, as extra objects, the 196,608-tet
jittered two-layer cube at degree 4 with one point source ("c2"), the 32-member
ensemble on that cube at degree 3 ("ensemble") and the receiver-misfit gradient
on the 82,944-tet cube at degree 3 ("adjoint").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N>1 (torchrun, one process per GPU) runs N independent replicas of the
workload (the method is not sharded across GPUs here); value = all ranks'
element updates / max-over-ranks time.  --impl reference times the FP64 CPU
oracle (the method has no other implementation) on all host cores, on a
bounded sample of the same workload per step.
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

# The CPU baselines (the FP64 oracle) run one BLAS thread per process: the
# thread pools are pinned before numpy loads so that the reported core counts
# are exact; the all-core baseline runs one process per core.
for _var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "element-updates/s (FP32, N=4)"
UNIT = "element-updates/s"
FP32_LANES_PER_SM = 128


def n_modes(N):
    return (N + 1) * (N + 2) * (N + 3) // 6


def algorithmic_flops(N):
    """FLOPs per element update of each kernel as this library formulates it
    (FMA = 2 flops): Taylor terms on their nonzero modes (degree <= N-i),
    (N+1)^3 volume nodes, (N+1)^2 face nodes and N+1 time nodes, each interior
    face's flux once (a closed mesh has 2 faces per element).  An informational
    count; the roofline uses the dense count of hot_path_terms()."""
    L, NQ, NF, NT = n_modes(N), (N + 1) ** 3, (N + 1) ** 2, N + 1
    LR = [n_modes(N - i) for i in range(N + 1)]
    SH = sum(LR[1:])
    pred = (2 * 6 * NQ * L + 20 * NQ + 2 * NQ * L                       # damage rate at t_n, projection
            + sum(2 * 27 * LR[i] * LR[i - 1] + 192 * LR[i] for i in range(1, N + 1)))   # CK
    per_face = (2 * NF * 2 * (11 * L + 9 * SH)                          # traces, both sides, all orders
                + 2 * NF * (18 * (N + 1) + NT * (12 * N + 2))           # time-integrated trace; strain, alpha
                + NF * (NT * 2 * 61 + 2 * 30))                          # stress n at the time nodes; linear part
    faces = 2 * per_face
    corr = (2 * NQ * (8 * L + 6 * SH) + 2 * NQ * NT * (6 * N + 1)       # strains, damage at the nodes
            + NQ * NT * 50 + NQ * 63                                    # CDM stress/rate, stress terms
            + 20 * L * NQ                                               # volume and source projections
            + 18 * L * L + 63 * L + 6 * (L + SH)                        # strain rows (modal)
            + 2 * L * 4 * NF * 9 + 10 * L)                              # face projection, update
    return {"predictor": pred, "faces": faces, "corrector": corr}


def hot_path_terms(N):
    """Dense FLOP count per element update of each term of the step (FMA = 2;
    reference matrices dense, time nodes and face traces once per element, each
    interior Rusanov flux once per face pair), split into its contraction part
    (products against reference matrices shared by all elements: dense GEMMs when
    batched over elements, tensor-core work) and its pointwise part (FP32 ALU
    work), and assigned to the kernel of this library that computes it.
    Terms (L modes, Nq = (N+1)^3 volume nodes, Nf = (N+1)^2 face nodes,
    Nt = N+1 time nodes):
      CK predictor (Appendix A.1)            3N (20 L^2 + 200 L)
      damage source at i = 1                 16 Nq L + 40 Nq
      volume evaluation (A.2, 3rd term)      14 Nq L Nt + 14 L (N+1) Nt + 94 Nq Nt
      volume projection                      20 L Nq + 54 Nq
      face traces (A.2, 2nd term)            80 Nf L Nt
      Rusanov flux                           580 Nf Nt
      face projection                        80 L Nf
      strain rows (linear in v)              18 L^2
      time integration                       20 L (N+1)
    Returns {term: (kernel, contraction flops, pointwise flops)}."""
    L, NQ, NF, NT = n_modes(N), (N + 1) ** 3, (N + 1) ** 2, N + 1
    return {
        "ck_predictor": ("predictor", 3 * N * 20 * L * L, 3 * N * 200 * L),
        "damage_source_i1": ("predictor", 16 * NQ * L, 40 * NQ),
        "volume_evaluation": ("corrector", 14 * NQ * L * NT, 14 * L * (N + 1) * NT + 94 * NQ * NT),
        "volume_projection": ("corrector", 20 * L * NQ, 54 * NQ),
        "face_traces": ("faces", 80 * NF * L * NT, 0),
        "rusanov_flux": ("faces", 0, 580 * NF * NT),
        "face_projection": ("corrector", 80 * L * NF, 0),
        "strain_rows": ("corrector", 18 * L * L, 0),
        "time_integration": ("corrector", 0, 20 * L * (N + 1)),
    }


def kernel_flops(N):
    """{kernel: (contraction flops, pointwise flops)} per element update."""
    out = {}
    for k, c, p in hot_path_terms(N).values():
        a, b = out.get(k, (0, 0))
        out[k] = (a + c, b + p)
    return out


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


def roofline_peaks(sm_count):
    """The composite roofline's three denominators: the 3xTF32 tensor rate (the
    measured bf16 burst rate x the nominal TF32:BF16 ratio of 1:2, / 3 for the
    three TF32 products of one FP32-accurate product), the FP32 ALU rate (SMs x
    128 lanes x 2 flops x the maximum SM clock) and the measured HBM copy rate."""
    peaks, kind = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    return {"tensor_3xtf32_tflops": float(peaks["bf16_tflops"]) / 2.0 / 3.0,
            "alu_fp32_tflops": sm_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12,
            "hbm_gbs": float(peaks["hbm_gbs"]), "kind": kind,
            "source": (f"tensor: {kind} bf16 burst {peaks['bf16_tflops']} TFLOP/s / 2 (TF32) / 3 (3xTF32); "
                       f"ALU: {sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz; "
                       f"HBM: {kind} copy {peaks['hbm_gbs']} GB/s")}


def composite(contraction, pointwise, n_units, ms, pk, bytes_=0.0):
    """t_min = contraction / P_tensor + pointwise / P_ALU + bytes / BW_HBM for
    n_units element updates, against the measured time ms."""
    t_c = contraction * n_units / (pk["tensor_3xtf32_tflops"] * 1e12)
    t_p = pointwise * n_units / (pk["alu_fp32_tflops"] * 1e12)
    t_b = bytes_ * n_units / (pk["hbm_gbs"] * 1e9)
    t_min = t_c + t_p + t_b
    return {"t_min_ms": 1e3 * t_min, "ms": ms, "frac": 1e3 * t_min / ms if ms > 0 else None,
            "t_tensor_ms": 1e3 * t_c, "t_alu_ms": 1e3 * t_p, "t_hbm_ms": 1e3 * t_b,
            "contraction_flops_per_element": contraction, "pointwise_flops_per_element": pointwise,
            "bytes_per_element": bytes_}


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


def max_over_ranks(values, world, device="cpu"):
    """The per-rank timings reduced to their maximum over the ranks (the job
    ends when its slowest replica does); identity for one rank."""
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(world, units_per_rank, steps, ms):
    """Element updates per second of the whole job: every rank advances its own
    replica of units_per_rank elements for `steps` steps in at most ms."""
    return world * units_per_rank * steps / (ms * 1e-3)


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def load_workload(name, args):
    if name == "c3":
        from synthetic.regional import workload_c3
        return workload_c3(order=args.order)
    from synthetic import workload_c2
    return workload_c2(n=args.n, order=args.order)


# ---------------------------------------------------------------------------
# CPU baselines: the FP64 oracle, as it stands, on bounded samples of a workload
# ---------------------------------------------------------------------------

def _face_index(mesh, rows):
    """The faces of every element that shares a vertex with the sample rows,
    keyed by their sorted vertex-id triple (host bookkeeping only)."""
    vid = np.asarray(mesh.elem_vid)
    cand = np.nonzero(np.isin(vid, np.unique(vid[rows])).any(axis=1))[0]
    owner = {}
    for e in cand.tolist():
        v = vid[e].tolist()
        for f in range(4):
            owner.setdefault(tuple(sorted(v[:f] + v[f + 1:])), []).append(e)
    return owner


def _face_key(vid, e, f):
    v = vid[e].tolist()
    return tuple(sorted(v[:f] + v[f + 1:]))


def _sample_spec(w, rows, owner):
    """The sub-mesh of the sample rows and their face neighbours (faces leaving it
    tagged absorbing: they enter only the neighbours' own updates, which are not
    timed), the sources inside it, and the rows' positions."""
    mesh = w["mesh"]
    vid = np.asarray(mesh.elem_vid)
    nb = [x for e in rows.tolist() for f in range(4) for x in owner[_face_key(vid, e, f)] if x != e]
    elems = np.unique(np.concatenate([rows, np.asarray(nb, dtype=np.int64)]))
    pos = -np.ones(mesh.n_elem, dtype=np.int64)
    pos[elems] = np.arange(elems.size)
    bc = np.array(mesh.face_bc[elems], dtype=np.int8)
    for k, e in enumerate(elems.tolist()):
        for f in range(4):
            if bc[k, f] == 0 and not any(x != e and pos[x] >= 0 for x in owner[_face_key(vid, e, f)]):
                bc[k, f] = 2
    lo, hi = mesh.elem_xyz[elems].min(axis=(0, 1)), mesh.elem_xyz[elems].max(axis=(0, 1))
    srcs = [s for s in w["sources"] if np.all(s["x"] >= lo) and np.all(s["x"] <= hi)]
    return {"xyz": mesh.elem_xyz[elems], "vid": mesh.elem_vid[elems], "bc": bc, "order": w["order"],
            "mat": w["material"][elems], "cfl": w["cfl"], "sources": srcs, "rows": pos[rows]}


def _sample_oracle(spec):
    from oracle import MeshError, Oracle
    o = Oracle(spec["xyz"], spec["vid"], spec["order"], spec["mat"], face_bc=spec["bc"], cfl=spec["cfl"],
               face_rows=spec["rows"])
    kept = []
    for s in spec["sources"]:
        try:
            o.locate(s["x"])
            kept.append(s)
        except MeshError:
            pass
    if kept:
        o.set_sources(kept)
    rng = np.random.default_rng(0)
    Q = rng.normal(size=(o.E, o.L, 10)) * 1e-6
    Q[..., 9] = 0.0
    return o, Q


_WORKER = None


def _worker_init(spec):
    global _WORKER
    o, Q = _sample_oracle(spec)
    _WORKER = (o, Q, spec["rows"], o.cfl_dt())


def _worker_step(_):
    o, Q, rows, dt = _WORKER
    t0 = time.perf_counter()
    o.step(Q, dt, t=0.8, rows=rows)
    return time.perf_counter() - t0


def _sample_rows(w, total):
    E = w["mesh"].n_elem
    start = max(0, E // 2 - total // 2)
    return np.arange(start, min(E, start + total))


class OraclePool:
    """The oracle stepping `workers` disjoint chunks of `chunk` elements of a
    workload, one chunk per process (started with "spawn": a process forked from
    one that has used CUDA can hang; one BLAS thread each).  Set-up (the
    sub-meshes and their reference tables) is outside the timed steps."""

    def __init__(self, w, workers, chunk):
        import concurrent.futures as cf
        import multiprocessing as mp
        rows = _sample_rows(w, workers * chunk)
        owner = _face_index(w["mesh"], rows)
        self.chunks = np.array_split(np.arange(rows.size), workers)
        specs = [_sample_spec(w, rows[c], owner) for c in self.chunks]
        self.rows = rows.size
        self.workers = workers
        ctx = mp.get_context("spawn")
        self.ex = [cf.ProcessPoolExecutor(1, mp_context=ctx, initializer=_worker_init, initargs=(sp,))
                   for sp in specs]
        for f in [ex.submit(_worker_step, 0) for ex in self.ex]:     # builds the oracles, untimed
            f.result()

    def step(self):
        """One step of every chunk, in parallel; returns the wall time in s."""
        t0 = time.perf_counter()
        for f in [ex.submit(_worker_step, 0) for ex in self.ex]:
            f.result()
        return time.perf_counter() - t0

    def close(self):
        for ex in self.ex:
            ex.shutdown()


def cpu_baseline_one_core(w, chunk=1024, steps=2):
    """The oracle on one host core: `chunk` elements of the workload (and their
    face neighbours' predictors), `steps` steps from a seeded state."""
    rows = _sample_rows(w, chunk)
    spec = _sample_spec(w, rows, _face_index(w["mesh"], rows))
    o, Q = _sample_oracle(spec)
    dt = o.cfl_dt()
    o.step(Q, dt, t=0.8, rows=spec["rows"])                        # warm-up
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step(Q, dt, t=0.8, rows=spec["rows"])
    el = time.perf_counter() - t0
    sample = (f"{rows.size} contiguous elements of the {w['mesh'].n_elem}-element mesh (plus their face "
              f"neighbours' predictors), {steps} step(s), numpy FP64, 1 process with 1 BLAS thread")
    return rows.size * steps / el, sample, 1, el


def cpu_baseline_all_cores(w, chunk=512, steps=2):
    """The oracle on every host core: one process per core, each stepping its own
    chunk of `chunk` contiguous elements of the workload."""
    cores = _host_cores()
    pool = OraclePool(w, cores, chunk)
    try:
        el = sum(pool.step() for _ in range(steps))
    finally:
        pool.close()
    sample = (f"{pool.rows} contiguous elements of the {w['mesh'].n_elem}-element mesh in {cores} chunks of "
              f"{chunk} (plus their face neighbours' predictors), {steps} step(s), numpy FP64, {cores} processes "
              f"with 1 BLAS thread each")
    return pool.rows * steps / el, sample, cores, el


def cpu_adjoint_baseline():
    """The FP64 oracle's forward step and its discrete adjoint (oracle.adjoint,
    as it stands) timed on a bounded sample of the adjoint workload: its jittered
    cube at 4 cells per side (384 tets) and degree 3, one step each from a seeded
    damaged state.  Returns (adjoint element-steps/s, forward element-steps/s,
    sample text, threads)."""
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
    sample = (f"{mesh.n_elem} tets of the adjoint workload's cube at n = 4, N = {N}, one forward step and one "
              f"adjoint step, numpy FP64, 1 process with 1 BLAS thread")
    return mesh.n_elem / (t2 - t1), mesh.n_elem / (t1 - t0), sample, 1


def run_reference(args):
    """The oracle on all host cores: each step is one step of a bounded sample
    of the workload (one chunk of `--ref-chunk` contiguous elements per core)."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    w = load_workload(args.workload, args)
    cores = _host_cores()
    # about four minutes of oracle work for the whole run at a conservative 300
    # element updates/s per core, within [64, 1024] elements per core and step
    chunk = args.ref_chunk or int(min(1024, max(64, 240.0 / (args.steps + args.warmup) * 300.0)) // 64 * 64)
    pool = OraclePool(w, cores, chunk)
    try:
        for _ in range(args.warmup):
            pool.step()
        times = [pool.step() for _ in range(args.steps)]
    finally:
        pool.close()
    total = sum(times)
    value = pool.rows * args.steps / total
    sample = (f"per step: {pool.rows} contiguous elements of the {w['mesh'].n_elem}-element mesh in {cores} "
              f"chunks of {chunk} (plus their face neighbours' predictors), numpy FP64, {cores} "
              f"processes with 1 BLAS thread each")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "ms_per_step_is": "one step of the sample timed",
            "ms_per_full_mesh_step_extrapolated": 1e3 * w["mesh"].n_elem / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(w, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _config(w, args):
    return {"workload": w["name"], "elements": w["mesh"].n_elem, "order": w["order"],
            "modes": n_modes(w["order"]), "fields": 10, "sources": len(w["sources"]),
            "receivers": int(len(w["receivers"])), "l2_policy": "inputs larger than L2 "
            "(the state's two buffers and the predictor output exceed 129 MB); no flush",
            "parallelism": f"replicas{args.gpus}",
            "predictor": f"picard{args.picard_iterations}" if getattr(args, "picard_iterations", 0) > 0 else "ck"}


# ---------------------------------------------------------------------------
# GPU runs
# ---------------------------------------------------------------------------

def run_forward(w, args, dgpkg, torch, stream, steps, warmup, e2e_steps, world=1, barrier=None, clocks_index=None):
    """Time `steps` steps of the workload after `warmup` (CUDA events on the
    library's stream, per-kernel events inside the library) and, if e2e_steps,
    the end-to-end step through dg_step_host with pinned host buffers."""
    mesh, mat, N = w["mesh"], w["material"], w["order"]
    E, L = mesh.n_elem, n_modes(N)
    bc = mesh.face_bc if np.any(mesh.face_bc != 0) else None
    s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, face_bc=bc, cfl=w["cfl"], stream=stream)
    s.set_material(mat)
    if getattr(args, "picard_iterations", 0) > 0:
        s.set_predictor("picard", args.picard_iterations)
    s.set_sources(w["sources"])
    s.set_receivers(w["receivers"])
    s.set_state(np.zeros((E, 10, L), np.float32), 0.0)
    barrier = barrier or torch.cuda.synchronize
    s.step(warmup)
    barrier()
    s.profile(True)
    launches0 = s.stats()["kernel_launches"]
    clocks = ClockSampler(clocks_index) if clocks_index is not None else None
    if clocks:
        clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    barrier()
    if clocks:
        clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = s.profile_read()
    s.profile(False)
    out = {"E": E, "N": N, "ms": ms, "prof": prof, "launches": s.stats()["kernel_launches"] - launches0,
           "clocks": clocks.summary() if clocks else None}
    if e2e_steps > 0:
        # end to end through the public API: pinned host state in, one step, state out
        hq = torch.zeros((E, 10, L), dtype=torch.float32).pin_memory()
        hq_np = hq.numpy()
        res = torch.empty_like(hq).pin_memory()
        res_np = res.numpy()
        s.get_state(out=res_np)
        hq_np[...] = res_np
        # W untimed calls, like the device run: the first call allocates the staging buffer,
        # and the first transfers after the device run are slow
        for _ in range(warmup):
            s.step_host(hq_np, res_np)
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            s.step_host(hq_np, res_np)       # upload, one step, download (transfers overlap the step)
        barrier()
        out["e2e_s"] = time.perf_counter() - t0
        out["e2e_bytes"] = (int(hq.numel() * 4), int(res.numel() * 4))
        del hq, res
    s.close()
    return out


def forward_report(r, pk, steps, world=1):
    """Rates, per-kernel times and the composite roofline of a forward run."""
    E, N, prof = r["E"], r["N"], r["prof"]
    value = whole_job_rate(world, E, steps, r["ms"])
    kavg = {k: v["total_ms"] / max(1, v["launches"]) for k, v in prof.items()}
    kf = kernel_flops(N)
    lib_flops = algorithmic_flops(N)
    kernels = {}
    for k, v in prof.items():
        d = {"launches": v["launches"], "avg_ms": kavg[k]}
        if k in kf and kavg[k] > 0:
            c, p = kf[k]
            d["roofline"] = composite(c, p, E, kavg[k], pk)
            d["library_flops_per_element"] = lib_flops[k]
        kernels[k] = d
    ms_step = r["ms"] / steps
    c_all = sum(c for c, _ in kf.values())
    p_all = sum(p for _, p in kf.values())
    step_roof = composite(c_all, p_all, E, ms_step, pk, algorithmic_bytes(N))
    return value, kernels, step_roof, kavg


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c2", "c3"],
                    help="c3: the ~4.35 M-tet regional-shaped box (headline); c2: the 196,608-tet two-layer cube")
    ap.add_argument("--n", type=int, default=32, help="cells per cube side of the two-layer cube (32 -> 196,608)")
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cube-steps", type=int, default=200,
                    help="steps of the two-layer cube timed as the extra 'c2' object (0 skips it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-chunk", type=int, default=0,
                    help="elements per host core in each step of --impl reference (0: sized from the steps so "
                         "that the run takes a few minutes)")
    ap.add_argument("--ensemble-members", type=int, default=32,
                    help="members of the ensemble workload (two-layer cube at N=3) timed against one member; "
                         "0 skips it")
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

    rank, world, local = _dist()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dgpkg.build()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    pk = roofline_peaks(sm_count)
    stream = torch.cuda.current_stream()
    w = load_workload(args.workload, args)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    r = run_forward(w, args, dgpkg, torch, stream, args.steps, args.warmup, args.e2e_steps, world, barrier,
                    clocks_index=local)
    r["ms"], e2e_s = max_over_ranks([r["ms"], r.get("e2e_s", 0.0)], world, device="cuda")
    E, N = r["E"], r["N"]
    value, kernels, step_roof, kavg = forward_report(r, pk, args.steps, world)
    e2e_value = whole_job_rate(world, E, args.e2e_steps, 1e3 * e2e_s) if e2e_s > 0 else None

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    peaks, _ = _peaks()
    dom = max(("predictor", "faces", "corrector"), key=lambda k: r["prof"][k]["total_ms"])
    dr = kernels[dom]["roofline"]
    flops_dom = dr["contraction_flops_per_element"] + dr["pointwise_flops_per_element"]
    achieved = flops_dom * E / (kavg[dom] * 1e-3) / 1e12
    peak_eff = flops_dom * E / (dr["t_min_ms"] * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(w, args),
        "roofline": {"kernel": _kernel_name(dom, N),
                     "bound": "tensor" if dr["t_tensor_ms"] >= dr["t_alu_ms"] else "alu",
                     "achieved": achieved, "peak": peak_eff, "unit": "TFLOP/s", "frac": achieved / peak_eff,
                     "traffic": _traffic_per_launch(dom, N, E),
                     "peak_is": ("composite: the kernel's dense flops / (contraction flops / P_tensor(3xTF32) + "
                                 "pointwise flops / P_ALU(FP32)); frac = t_min / measured launch time"),
                     "peak_source": pk["source"], "avg_ms": kavg[dom],
                     "contraction_flops_per_element": dr["contraction_flops_per_element"],
                     "pointwise_flops_per_element": dr["pointwise_flops_per_element"],
                     "t_min_ms": dr["t_min_ms"]},
        "step_roofline": step_roof,
        "kernels": kernels,
        "hbm": {"algorithmic_bytes_per_element": algorithmic_bytes(N),
                "achieved_gbs": algorithmic_bytes(N) * value / world / 1e9,
                "peak_gbs": peaks.get("hbm_gbs"),
                "frac": algorithmic_bytes(N) * value / world / 1e9 / float(peaks.get("hbm_gbs", 6800.0))},
        "sm_count": sm_count,
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": r.get("e2e_bytes", (0, 0))[0],
                "d2h_bytes_per_step": r.get("e2e_bytes", (0, 0))[1], "steps": args.e2e_steps},
    }
    if args.workload == "c3" and args.cube_steps > 0:
        wc = load_workload("c2", args)
        rc = run_forward(wc, args, dgpkg, torch, stream, args.cube_steps, args.warmup, 0)
        vc, kc, sc, _ = forward_report(rc, pk, args.cube_steps)
        line["c2"] = {"workload": wc["name"], "elements": rc["E"], "order": rc["N"], "steps": args.cube_steps,
                      "value": vc, "unit": UNIT, "ms_per_step": rc["ms"] / args.cube_steps,
                      "step_roofline": sc, "kernels": kc, "gpu_launches": rc["launches"]}
        del wc
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
        v1, s1, c1, _ = cpu_baseline_one_core(w)
        va, sa, ca, _ = cpu_baseline_all_cores(w)
        line["cpu_baseline"] = {"value": va, "unit": UNIT, "cores": ca, "kind": "oracle", "sample": sa,
                                "one_core": {"value": v1, "unit": UNIT, "cores": c1, "kind": "oracle",
                                             "sample": s1}}
    print(json.dumps(line), flush=True)
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
    t_start = w["t_start"]
    s.set_material(w["material_ref"])
    s.set_sources(w["sources"])
    s.set_receivers(w["receivers"])
    s.set_state(zero, t_start)
    dt = s.dt
    s.step(n, dt)
    ref = s.read_receivers()[:n]
    s.set_material(w["material"])
    s.set_state(zero, t_start)
    s.step(5, dt)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(fwd_steps, dt)
    ev1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = ev0.elapsed_time(ev1) / fwd_steps
    s.set_state(zero, t_start)
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
        s.set_state(zero, t_start)
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
    # size of the residual behind J against the traces: J = dt/2 sum |v - v_ref|^2
    res_rms = math.sqrt(2.0 * J / (dt * ref.size)) if J > 0 else 0.0
    ref_rms = float(np.sqrt(np.mean(ref.astype(np.float64) ** 2)))
    return {"workload": w["name"], "elements": E, "order": N, "steps": n, "snapshots": snapshots,
            "forward_ms_per_step": fwd_ms, "adjoint_ms_per_step": adj, "adjoint_to_forward_step": adj / fwd_ms,
            "forward_steps_run": info["forward_steps"], "snapshot_copy_ms": info["copy_ms"],
            "gradient_ms": total, "gradient_to_forward_run": total / (n * fwd_ms), "misfit": J,
            "t_start": t_start, "reference_trace_rms": ref_rms, "residual_rms": res_rms,
            "residual_to_trace_rms": res_rms / ref_rms if ref_rms > 0 else None,
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


def _kernel_source_digest(path=None):
    """Digest of the step kernels' code: comments and spacing are left out, so that
    a change of wording keeps the DRAM counters taken on the same code."""
    import hashlib
    import re
    p = path or os.path.join(ROOT, "paper_2502_09714_gb300", "csrc", "dg_step_kernels.cuh")
    with open(p, encoding="utf-8") as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = " ".join(src.split())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


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
