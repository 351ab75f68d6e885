"""Thin ctypes binding of libdg (include/dg.h): argument marshalling only.

Every step of the method runs in the CUDA kernels of libdg.  If the library is
not built this module raises on use; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB_PATH

STATUS = {
    0: "DG_OK", 1: "DG_E_ARG", 2: "DG_E_MESH", 3: "DG_E_ORDER", 4: "DG_E_OOM", 5: "DG_E_CUDA",
    6: "DG_E_STATE", 7: "DG_E_NONFINITE", 8: "DG_E_NONHYPERBOLIC", 9: "DG_E_OUTSIDE",
    10: "DG_E_UNSUPPORTED",
}

# every entry point declared in include/dg.h
EXPORTS = (
    "dg_mesh_create", "dg_set_material", "dg_set_source", "dg_set_state", "dg_set_state_f32",
    "dg_set_state_device", "dg_get_state", "dg_get_state_f32", "dg_get_state_device", "dg_step",
    "dg_receivers", "dg_receivers_read", "dg_dt", "dg_time", "dg_n_modes", "dg_get_stats",
    "dg_profile_enable", "dg_profile_read", "dg_reference_table", "dg_last_error", "dg_destroy",
    "dg_step_noalloc", "dg_set_rheology", "dg_set_predictor", "dg_set_wait_limit", "dg_step_host",
    "dg_adjoint_gradient", "dg_revolve_plan", "dg_revolve_cost", "dg_host_chunks",
)


class DGError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {message}")


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class MeshDesc(C.Structure):
    _fields_ = [("n_elem", C.c_int64), ("elem_xyz", C.POINTER(C.c_double)),
                ("elem_vid", C.POINTER(C.c_int64)), ("face_bc", C.POINTER(C.c_int8)),
                ("order", C.c_int), ("members", C.c_int), ("cfl", C.c_double),
                ("cuda_stream", C.c_void_p), ("alloc", C.POINTER(Allocator))]


class PointSource(C.Structure):
    _fields_ = [("x", C.c_double * 3), ("m", C.c_double * 6), ("stf", C.c_int),
                ("f0_or_sigma", C.c_double), ("t0", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("kernel_launches", C.c_int64), ("element_updates", C.c_int64)]


class KernelTime(C.Structure):
    _fields_ = [("launches", C.c_int64), ("total_ms", C.c_double)]


class AdjointInfo(C.Structure):
    _fields_ = [("forward_steps", C.c_int64), ("adjoint_steps", C.c_int64), ("forward_ms", C.c_double),
                ("adjoint_ms", C.c_double), ("copy_ms", C.c_double)]


_LIB = None


def load_library(path: str | None = None) -> C.CDLL:
    """Load libdg.so (built in-tree by paper_2502_09714_gb300.build.build())."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libdg is not built ({p} missing); run paper_2502_09714_gb300.build.build()")
    lib = C.CDLL(p)
    vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
    sig = {
        "dg_mesh_create": ([C.POINTER(MeshDesc), C.POINTER(vp)], C.c_int),
        "dg_set_material": ([vp, C.POINTER(dbl), C.POINTER(dbl)], C.c_int),
        "dg_set_rheology": ([vp, C.c_int], C.c_int),
        "dg_set_predictor": ([vp, C.c_int, C.c_int], C.c_int),
        "dg_set_wait_limit": ([vp, i64], C.c_int),
        "dg_step_host": ([vp, vp, vp, C.c_double], C.c_int),
        "dg_host_chunks": ([i64, vp, C.c_int], C.c_int),
        "dg_set_source": ([vp, C.POINTER(PointSource), i64], C.c_int),
        "dg_set_state": ([vp, C.POINTER(dbl), dbl], C.c_int),
        "dg_set_state_f32": ([vp, C.POINTER(C.c_float), dbl], C.c_int),
        "dg_set_state_device": ([vp, vp, dbl], C.c_int),
        "dg_get_state": ([vp, C.POINTER(dbl), C.POINTER(dbl)], C.c_int),
        "dg_get_state_f32": ([vp, C.POINTER(C.c_float), C.POINTER(dbl)], C.c_int),
        "dg_get_state_device": ([vp, vp, C.POINTER(dbl)], C.c_int),
        "dg_step": ([vp, i64, dbl], C.c_int),
        "dg_receivers": ([vp, C.POINTER(dbl), i64], C.c_int),
        "dg_receivers_read": ([vp, C.POINTER(C.c_float), i64, C.POINTER(i64)], C.c_int),
        "dg_dt": ([vp], dbl),
        "dg_time": ([vp], dbl),
        "dg_n_modes": ([C.c_int], i64),
        "dg_get_stats": ([vp, C.POINTER(Stats)], C.c_int),
        "dg_profile_enable": ([vp, C.c_int], C.c_int),
        "dg_profile_read": ([vp, C.POINTER(KernelTime), C.c_int, C.POINTER(C.c_int)], C.c_int),
        "dg_reference_table": ([C.c_int, C.c_int, C.POINTER(dbl), i64, C.POINTER(i64)], C.c_int),
        "dg_last_error": ([vp], C.c_char_p),
        "dg_destroy": ([vp], None),
        "dg_step_noalloc": ([vp, vp, vp, dbl], C.c_int),
        "dg_adjoint_gradient": ([vp, i64, dbl, C.POINTER(C.c_float), C.c_int, C.POINTER(dbl), C.POINTER(dbl),
                                 C.POINTER(dbl), C.POINTER(dbl), C.POINTER(AdjointInfo)], C.c_int),
        "dg_revolve_plan": ([i64, C.c_int, C.POINTER(i64), C.POINTER(i64), i64, C.POINTER(i64)], C.c_int),
        "dg_revolve_cost": ([i64, C.c_int], i64),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path is None:
        _LIB = lib
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def n_modes(order: int) -> int:
    return (order + 1) * (order + 2) * (order + 3) // 6


def reference_table(order: int, which: int) -> np.ndarray:
    lib = load_library()
    count = C.c_int64(0)
    _check(lib, None, lib.dg_reference_table(order, which, None, 0, C.byref(count)))
    out = np.empty(count.value)
    _check(lib, None, lib.dg_reference_table(order, which, _ptr(out, C.c_double), out.size, C.byref(count)))
    return out


def revolve_plan(n_steps: int, snapshots: int):
    """(forward steps, actions [n, 3] of (kind, a, b)) of the checkpointing plan
    (kind 0 advance a -> b, 1 store slot a <- step b, 2 restore slot a (step b),
    3 adjoint of step a)."""
    lib = load_library()
    fw, n = C.c_int64(0), C.c_int64(0)
    _check(lib, None, lib.dg_revolve_plan(int(n_steps), int(snapshots), C.byref(fw), None, 0, C.byref(n)))
    acts = np.empty((n.value, 3), dtype=np.int64)
    _check(lib, None, lib.dg_revolve_plan(int(n_steps), int(snapshots), C.byref(fw), _ptr(acts, C.c_int64),
                                          n.value, C.byref(n)))
    return fw.value, acts


def revolve_cost(n_steps: int, snapshots: int) -> int:
    return int(load_library().dg_revolve_cost(int(n_steps), int(snapshots)))


def host_chunks(n_elem: int):
    """Chunk boundaries [count + 1] of the host-to-host step on a mesh of n_elem
    elements (chunk k holds elements [b[k], b[k + 1]))."""
    lib = load_library()
    n = lib.dg_host_chunks(int(n_elem), None, 0)
    if n < 0:
        raise DGError(1, "dg_host_chunks: n_elem must be >= 1")
    b = np.empty(n + 1, dtype=np.int64)
    lib.dg_host_chunks(int(n_elem), b.ctypes.data_as(C.c_void_p), n + 1)
    return b


def _check(lib, ctx, status):
    if status != 0:
        msg = lib.dg_last_error(ctx)
        raise DGError(status, msg.decode() if msg else "")


def torch_allocator():
    """An Allocator that draws device memory from torch's caching allocator."""
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream or torch.cuda.current_stream().cuda_stream)
        except RuntimeError:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a = Allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    a._keep = (_alloc, _free)
    return a


class Solver:
    """One libdg context: a mesh, its material, state, sources and receivers."""

    def __init__(self, elem_xyz, elem_vid, order, face_bc=None, cfl=0.5, stream=None,
                 allocator=None, members=1, law="cdm"):
        self.lib = load_library()
        xyz = np.ascontiguousarray(elem_xyz, dtype=np.float64)
        vid = np.ascontiguousarray(elem_vid, dtype=np.int64)
        self.E = int(xyz.shape[0])
        self.M = int(members)
        self.order = int(order)
        self.L = n_modes(self.order)
        bc = None if face_bc is None else np.ascontiguousarray(face_bc, dtype=np.int8)
        if stream is None:
            stream_ptr = None
        elif isinstance(stream, int):
            stream_ptr = stream
        else:
            stream_ptr = stream.cuda_stream
        self._allocator = allocator
        desc = MeshDesc(self.E, _ptr(xyz, C.c_double), _ptr(vid, C.c_int64),
                        _ptr(bc, C.c_int8) if bc is not None else None, self.order, members,
                        float(cfl), stream_ptr, C.pointer(allocator) if allocator is not None else None)
        self.ctx = C.c_void_p()
        _check(self.lib, None, self.lib.dg_mesh_create(C.byref(desc), C.byref(self.ctx)))
        if law != "cdm":
            self.set_rheology(law)

    def set_rheology(self, law):
        """law: "cdm" (Eq. "cdb-model"), "ivm" (Eq. "ivm-model") or "nlshear" (the
        nonlinear shear law of the 1-D Riemann verification); set the material after."""
        self._chk(self.lib.dg_set_rheology(self.ctx, {"cdm": 0, "ivm": 1, "nlshear": 2}[law]))

    def set_predictor(self, kind="ck", iterations=0):
        """kind: "ck" (the linearised Cauchy-Kovalevskaya procedure) or "picard"
        (`iterations` discrete Picard sweeps after it, Sec. 5.1's extension)."""
        self._chk(self.lib.dg_set_predictor(self.ctx, {"ck": 0, "picard": 1}[kind], int(iterations)))

    def set_wait_limit(self, polls=-1):
        """Polls per bounded wait of the tensor-core corrector (negative: default)."""
        self._chk(self.lib.dg_set_wait_limit(self.ctx, int(polls)))

    # ------------------------------------------------------------------
    def _chk(self, status):
        _check(self.lib, self.ctx, status)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.dg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------
    def set_material(self, mat, member_xi0_cd=None):
        """mat [E,6] = (rho, lambda0, mu0, gamma_r, xi0, C_d); member_xi0_cd
        [M,E,2] per-member (xi0, C_d) or None."""
        m = np.ascontiguousarray(mat, dtype=np.float64).reshape(self.E, 6)
        mp = None
        if member_xi0_cd is not None:
            mp = np.ascontiguousarray(member_xi0_cd, dtype=np.float64).reshape(self.M, self.E, 2)
        self._chk(self.lib.dg_set_material(self.ctx, _ptr(m, C.c_double),
                                           _ptr(mp, C.c_double) if mp is not None else None))

    def set_sources(self, sources):
        arr = (PointSource * max(1, len(sources)))()
        for i, s in enumerate(sources):
            arr[i].x[:] = [float(v) for v in s["x"]]
            arr[i].m[:] = [float(v) for v in s["m"]]
            arr[i].stf = int(s.get("stf", 0))
            arr[i].f0_or_sigma = float(s.get("f0", s.get("sigma", 1.0)))
            arr[i].t0 = float(s.get("t0", 0.0))
        self._chk(self.lib.dg_set_source(self.ctx, arr, len(sources)))

    def _shape(self):
        return (self.E, 10, self.L) if self.M == 1 else (self.M, self.E, 10, self.L)

    def set_state(self, q, t=0.0):
        """q: [E,10,L] ([M,E,10,L] with several members) host array (float64 or
        float32) or a CUDA float32 torch tensor."""
        if hasattr(q, "is_cuda") and q.is_cuda:
            assert q.dtype.__str__() == "torch.float32" and q.is_contiguous()
            assert tuple(q.shape) == self._shape()
            self._chk(self.lib.dg_set_state_device(self.ctx, C.c_void_p(q.data_ptr()), float(t)))
            return
        if hasattr(q, "numpy"):
            q = q.numpy()
        if q.dtype == np.float32:
            a = np.ascontiguousarray(q).reshape(self._shape())
            self._chk(self.lib.dg_set_state_f32(self.ctx, _ptr(a, C.c_float), float(t)))
        else:
            a = np.ascontiguousarray(q, dtype=np.float64).reshape(self._shape())
            self._chk(self.lib.dg_set_state(self.ctx, _ptr(a, C.c_double), float(t)))

    def get_state(self, dtype=np.float64, out=None):
        """Returns (q [E,10,L] or [M,E,10,L], t).  `out` may be a host array of
        matching dtype or a CUDA float32 torch tensor."""
        t = C.c_double(0.0)
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            self._chk(self.lib.dg_get_state_device(self.ctx, C.c_void_p(out.data_ptr()), C.byref(t)))
            return out, t.value
        if out is None:
            out = np.empty(self._shape(), dtype=dtype)
        a = out.numpy() if hasattr(out, "numpy") else out
        if a.dtype == np.float32:
            self._chk(self.lib.dg_get_state_f32(self.ctx, _ptr(a, C.c_float), C.byref(t)))
        else:
            self._chk(self.lib.dg_get_state(self.ctx, _ptr(a, C.c_double), C.byref(t)))
        return out, t.value

    def step(self, n_steps=1, dt=0.0):
        self._chk(self.lib.dg_step(self.ctx, int(n_steps), float(dt)))

    def step_host(self, q_in, q_out, dt=0.0):
        """One step from the host state q_in to the host state q_out (float32
        arrays [E,10,L], [M,E,10,L] with several members; page-locked memory,
        e.g. numpy views of pinned torch tensors, lets the transfers overlap the
        step)."""
        a = q_in.numpy() if hasattr(q_in, "numpy") else q_in
        b = q_out.numpy() if hasattr(q_out, "numpy") else q_out
        assert a.dtype == np.float32 and b.dtype == np.float32
        assert a.flags.c_contiguous and b.flags.c_contiguous and b.flags.writeable
        assert tuple(a.shape) == self._shape() and tuple(b.shape) == self._shape()
        self._chk(self.lib.dg_step_host(self.ctx, C.c_void_p(a.ctypes.data), C.c_void_p(b.ctypes.data), float(dt)))

    def step_noalloc(self, q_in, q_out, dt=0.0):
        """One step from q_in to q_out (CUDA float32 tensors [E,10,L], or raw
        device pointers) without any allocation: for callers that cannot
        allocate device memory while they step.  Scratch lives in a fixed
        16 MiB device array shared by all calls (small meshes only; calls that
        overlap on the GPU race).  The context's own state is not touched."""
        pin = q_in if isinstance(q_in, int) else q_in.data_ptr()
        pout = q_out if isinstance(q_out, int) else q_out.data_ptr()
        self._chk(self.lib.dg_step_noalloc(self.ctx, C.c_void_p(pin), C.c_void_p(pout), float(dt)))

    def set_receivers(self, xyz):
        x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        self.R = x.shape[0]
        self._chk(self.lib.dg_receivers(self.ctx, _ptr(x, C.c_double), x.shape[0]))

    def read_receivers(self):
        n = C.c_int64(0)
        self._chk(self.lib.dg_receivers_read(self.ctx, None, 0, C.byref(n)))
        out = np.empty((n.value, self.R, 3) if self.M == 1 else (n.value, self.M, self.R, 3), dtype=np.float32)
        if n.value:
            self._chk(self.lib.dg_receivers_read(self.ctx, _ptr(out, C.c_float), n.value, C.byref(n)))
        return out

    @property
    def dt(self):
        return self.lib.dg_dt(self.ctx)

    @property
    def time(self):
        return self.lib.dg_time(self.ctx)

    def stats(self):
        s = Stats()
        self._chk(self.lib.dg_get_stats(self.ctx, C.byref(s)))
        return {"steps": s.steps, "kernel_launches": s.kernel_launches, "element_updates": s.element_updates}

    def adjoint_gradient(self, ref, n_steps, dt=0.0, snapshots=40, grad_state=False, info=False):
        """Receiver misfit J of n_steps steps from the current state against
        ref [n_steps, R, 3] and its gradient by the discrete adjoint with
        binomial checkpointing (`snapshots` state copies; 0 keeps as many as the
        free device memory holds, up to the whole history).  Returns
        (J, dJ/dxi0 [E], dJ/dC_d [E]) plus dJ/dQ^0 [E, 10, L] with grad_state and
        the run's counts and device times (a dict) with info.  The state, time and
        traces of the solver are left unchanged."""
        r = np.ascontiguousarray(ref, dtype=np.float32)
        assert r.shape == (int(n_steps), self.R, 3), r.shape
        J = C.c_double(0.0)
        gx = np.empty(self.E)
        gc = np.empty(self.E)
        gq = np.empty((self.E, 10, self.L)) if grad_state else None
        inf = AdjointInfo()
        self._chk(self.lib.dg_adjoint_gradient(self.ctx, int(n_steps), float(dt), _ptr(r, C.c_float), int(snapshots),
                                               C.byref(J), _ptr(gx, C.c_double), _ptr(gc, C.c_double),
                                               _ptr(gq, C.c_double) if gq is not None else None,
                                               C.byref(inf) if info else None))
        out = [J.value, gx, gc]
        if grad_state:
            out.append(gq)
        if info:
            out.append({"forward_steps": inf.forward_steps, "adjoint_steps": inf.adjoint_steps,
                        "forward_ms": inf.forward_ms, "adjoint_ms": inf.adjoint_ms, "copy_ms": inf.copy_ms})
        return tuple(out)

    def profile(self, on=True):
        self._chk(self.lib.dg_profile_enable(self.ctx, int(on)))

    def profile_read(self):
        out = (KernelTime * 5)()
        n = C.c_int(0)
        self._chk(self.lib.dg_profile_read(self.ctx, out, 5, C.byref(n)))
        names = ("predictor", "corrector", "source", "receivers", "faces")
        return {names[k]: {"launches": out[k].launches, "total_ms": out[k].total_ms} for k in range(n.value)}


def misfit_function():
    """torch.autograd.Function of the receiver misfit in the per-element damage
    parameters: MisfitFn.apply(xi0, cd, solver, material, ref, n_steps, dt,
    snapshots) sets rows 4 and 5 of `material` [E, 6] from the tensors xi0 [E]
    and cd [E] (FP64), runs dg_adjoint_gradient from the solver's current state
    and returns J as a 0-d FP64 tensor; backward gives grad_J * dJ/dxi0 and
    grad_J * dJ/dC_d.  The gradient is computed with J (one call of the adjoint),
    so backward only scales it."""
    import torch

    class MisfitFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, xi0, cd, solver, material, ref, n_steps, dt, snapshots):
            mat = np.array(material, dtype=np.float64, copy=True)
            mat[:, 4] = xi0.detach().cpu().numpy()
            mat[:, 5] = cd.detach().cpu().numpy()
            solver.set_material(mat)
            J, gx, gc = solver.adjoint_gradient(ref, n_steps, dt, snapshots)
            ctx.save_for_backward(torch.from_numpy(gx).to(xi0.device), torch.from_numpy(gc).to(cd.device))
            return torch.tensor(J, dtype=torch.float64, device=xi0.device)

        @staticmethod
        def backward(ctx, grad):
            gx, gc = ctx.saved_tensors
            return grad * gx, grad * gc, None, None, None, None, None, None

    return MisfitFn
