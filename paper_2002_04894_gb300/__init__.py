"""GB300 balanced-tree FMM (Bull & Engblom, arXiv:2002.04894) -- Python binding.

A thin ctypes layer over the C ABI declared in ``include/fmm.h``; every
function below has the name of the C entry point it marshals arguments for.
All computation runs in the CUDA library ``lib/libfmm_<arch>.so``; there is no
CPU fallback: if the library cannot be built or loaded, :func:`load` raises.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays (host). Device
memory for plans comes from PyTorch's caching allocator unless
``allocator=None`` is given (then the library uses cudaMallocAsync).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

FMM_F64, FMM_F32 = 0, 1
FMM_PREC_FP64, FMM_PREC_MIXED = 0, 1
FMM_MAX_LEVELS, FMM_MAX_P = 24, 20
FMM_FLAG_PROFILE = 1
FMM_FLAG_ETA = 2
FMM_FLAG_TC_M2L = 4
FMM_FLAG_TIGHT = 8
FMM_FLAG_ROOT_CELL = 16
STAGES = ("tree", "lists", "p2m", "m2m", "m2l", "l2l", "l2p", "p2p")
STATUS = {0: "FMM_OK", -1: "FMM_EINVAL", -2: "FMM_ENOMEM", -3: "FMM_ENONFINITE",
          -4: "FMM_ECAPACITY", -5: "FMM_ETIMEDOUT", -6: "FMM_ECUDA", -7: "FMM_EINTERNAL"}


class FmmError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = _LIB.fmm_strerror(status).decode() if _LIB is not None else STATUS.get(status, "?")
        super().__init__(f"{what}: {STATUS.get(status, status)} ({msg})")


class fmm_opts(C.Structure):
    _fields_ = [("levels", C.c_int), ("p", C.c_int), ("theta", C.c_double),
                ("prec", C.c_int), ("flags", C.c_int), ("eta", C.c_double),
                ("bisections_per_level", C.c_int), ("root_lo", C.c_double * 3),
                ("root_hi", C.c_double * 3)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class fmm_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class fmm_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("nbox", C.c_int64), ("nleaf", C.c_int64),
                ("levels", C.c_int), ("p", C.c_int), ("prec", C.c_int), ("dtype", C.c_int),
                ("theta", C.c_double), ("weak_pairs", C.c_int64),
                ("strong_leaf_pairs", C.c_int64), ("p2p_interactions", C.c_int64),
                ("weak_pairs_level", C.c_int64 * (FMM_MAX_LEVELS + 1)),
                ("p2p_units", C.c_int64), ("p2p_partial_slots", C.c_int64)]


_LIB = None
EXPORTS = ("fmm_plan", "fmm_eval", "fmm_destroy", "fmm_direct", "fmm_plan_stats",
           "fmm_plan_tree", "fmm_plan_list", "fmm_eval_expansions", "fmm_strerror",
           "fmm_last_cuda_error", "fmm_stage_times", "fmm_kernel_launches",
           "fmm_orb_order_noalloc", "fmm_batch_create", "fmm_batch_launch", "fmm_batch_destroy", "fmm_batch_info",
           "fmm_eval_check", "fmm_pool_trim", "fmm_set_list_capacity", "fmm_measure_peak",
           "fmm_theta_test", "fmm_eval_upward", "fmm_plan_multipoles", "fmm_plan_add_locals",
           "fmm_m2l_external", "fmm_plan_leaf_points", "fmm_p2p_external", "fmm_eval_downward",
           "fmm_translate", "fmm_set_wait_limit")
FMM_NOALLOC_MAX_POINTS, FMM_NOALLOC_MAX_LEVELS = 4096, 12


def ncoef_of(p: int) -> int:
    """Stored coefficients (n, m), 0 <= m <= n <= p, of one expansion."""
    return (p + 1) * (p + 2) // 2


def lib_path() -> str:
    return _build.lib_path()


def load(build: bool = True) -> C.CDLL:
    """Load (building first if missing or stale) the CUDA library. Raises if
    it cannot be built or loaded -- there is no fallback path."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build else _build.lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libfmm not built: {path}")
    lib = C.CDLL(path)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    lib.fmm_plan.argtypes = [vp, i64, i32, C.POINTER(fmm_opts), C.POINTER(fmm_allocator), vp,
                             C.POINTER(vp)]
    lib.fmm_plan.restype = i32
    lib.fmm_eval.argtypes = [vp, vp, vp, vp, vp]
    lib.fmm_eval.restype = i32
    lib.fmm_destroy.argtypes = [vp]
    lib.fmm_destroy.restype = None
    lib.fmm_direct.argtypes = [vp, vp, i64, i32, vp, i64, vp, vp, vp]
    lib.fmm_direct.restype = i32
    lib.fmm_plan_stats.argtypes = [vp, C.POINTER(fmm_stats)]
    lib.fmm_plan_stats.restype = i32
    lib.fmm_plan_tree.argtypes = [vp] * 10
    lib.fmm_plan_tree.restype = i32
    lib.fmm_plan_list.argtypes = [vp, i32, i32, vp, vp]
    lib.fmm_plan_list.restype = i32
    lib.fmm_eval_expansions.argtypes = [vp, i32, vp]
    lib.fmm_eval_expansions.restype = i32
    lib.fmm_eval_check.argtypes = [vp]
    lib.fmm_eval_check.restype = i32
    lib.fmm_strerror.argtypes = [i32]
    lib.fmm_strerror.restype = C.c_char_p
    lib.fmm_last_cuda_error.restype = i32
    lib.fmm_pool_trim.argtypes = [i32]
    lib.fmm_pool_trim.restype = i32
    lib.fmm_stage_times.argtypes = [vp, vp]
    lib.fmm_stage_times.restype = i32
    lib.fmm_kernel_launches.argtypes = []
    lib.fmm_kernel_launches.restype = i64
    lib.fmm_orb_order_noalloc.argtypes = [vp, i64, i32, i32, vp, vp]
    lib.fmm_orb_order_noalloc.restype = i32
    lib.fmm_batch_create.argtypes = [vp, i32, vp, vp, vp, i32, vp, C.POINTER(vp)]
    lib.fmm_batch_create.restype = i32
    lib.fmm_batch_launch.argtypes = [vp, vp]
    lib.fmm_batch_launch.restype = i32
    lib.fmm_batch_destroy.argtypes = [vp]
    lib.fmm_batch_destroy.restype = None
    lib.fmm_batch_info.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(i32)]
    lib.fmm_batch_info.restype = i32
    for name, args in (("fmm_theta_test", [C.c_double, i64, vp, vp, vp, vp, vp, vp]),
                       ("fmm_eval_upward", [vp, vp, vp]),
                       ("fmm_plan_multipoles", [vp, i32, i64, vp, vp, vp]),
                       ("fmm_plan_add_locals", [vp, i32, i64, vp, vp, vp]),
                       ("fmm_m2l_external", [vp, i32, i64, vp, vp, vp, vp]),
                       ("fmm_plan_leaf_points", [vp, i64, vp, vp, vp, vp]),
                       ("fmm_p2p_external", [vp, i64, vp, vp, vp, vp]),
                       ("fmm_eval_downward", [vp, vp, vp, vp]),
                       ("fmm_translate", [i32, i32, i64, vp, vp, vp, vp, vp])):
        getattr(lib, name).argtypes = args
        getattr(lib, name).restype = i32
    lib.fmm_set_wait_limit.argtypes = [i64, i64]
    lib.fmm_set_wait_limit.restype = i64
    lib.fmm_measure_peak.argtypes = [i32, i64, vp, vp, vp]
    lib.fmm_measure_peak.restype = i32
    lib.fmm_set_list_capacity.argtypes = [i64]
    lib.fmm_set_list_capacity.restype = i64
    _LIB = lib
    return lib


def _check(status: int, what: str) -> None:
    if status != 0:
        raise FmmError(status, what)


# ---------------------------------------------------------------------------
# argument marshalling
# ---------------------------------------------------------------------------
def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(pointer, keep-alive) for a contiguous torch tensor or numpy array."""
    if a is None:
        return None, None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a)
    return arr.ctypes.data, arr


def _dtype_code(a) -> int:
    name = str(a.dtype)
    if name.endswith("float64"):
        return FMM_F64
    if name.endswith("float32"):
        return FMM_F32
    raise TypeError(f"points/charges must be float64 or float32, got {a.dtype}")


def _stream(stream):
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


def _torch_allocator():
    import torch

    dev = torch.cuda.current_device()

    def alloc(nbytes, ctx, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
        except Exception:
            return None

    def free(ptr, nbytes, ctx, stream):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC_FN(alloc), FREE_FN(free)
    return fmm_allocator(a, f, None), (a, f)


class Plan:
    """Owning handle of an fmm_plan_t (released by fmm_destroy or on GC)."""

    def __init__(self, handle, n, dtype, opts, keep):
        self.handle, self.n, self.dtype, self.opts, self._keep = handle, n, dtype, opts, keep

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.fmm_destroy(self.handle)
            self.handle = None

    @property
    def levels(self):
        return self.opts.levels

    @property
    def p(self):
        return self.opts.p

    @property
    def theta(self):
        return self.opts.theta


# ---------------------------------------------------------------------------
# the C ABI, one function each
# ---------------------------------------------------------------------------
def fmm_plan(points, levels: int, p: int, theta: float, prec: int = FMM_PREC_FP64,
             stream=None, allocator="torch", profile: bool = False, eta: float = 1.0,
             bisections_per_level: int = 1, tc_m2l: bool = False, tight: bool = False,
             root_cell=None) -> Plan:
    """Build the tree and connectivity for n x 3 `points`; eta in [0, 1] is
    the split adaptivity (1: balanced median splits, 0: cell bisection);
    bisections_per_level = 3 makes octree levels (`levels` counts bisections);
    tight = True takes box centres and radii from the boxes' own points;
    root_cell = (lo[3], hi[3]) fixes the root cell (it must hold every point)."""
    lib = load()
    ptr, keep = _ptr(points)
    n = int(points.shape[0])
    dt = _dtype_code(points)
    flags = ((FMM_FLAG_PROFILE if profile else 0) | (FMM_FLAG_ETA if float(eta) != 1.0 else 0)
             | (FMM_FLAG_TC_M2L if tc_m2l else 0) | (FMM_FLAG_TIGHT if tight else 0)
             | (FMM_FLAG_ROOT_CELL if root_cell is not None else 0))
    opts = fmm_opts(int(levels), int(p), float(theta), int(prec), flags, float(eta),
                    int(bisections_per_level))
    if root_cell is not None:
        opts.root_lo[:] = [float(v) for v in root_cell[0]]
        opts.root_hi[:] = [float(v) for v in root_cell[1]]
    alloc, cbs = (None, None)
    if allocator == "torch":
        alloc, cbs = _torch_allocator()
    h = C.c_void_p()
    st = fmm_plan_raw(lib, ptr, n, dt, opts, alloc, _stream(stream), h)
    _check(st, "fmm_plan")
    return Plan(h.value, n, dt, opts, (alloc, cbs, keep))


def fmm_plan_raw(lib, ptr, n, dt, opts, alloc, stream, handle) -> int:
    return lib.fmm_plan(ptr, n, dt, C.byref(opts), C.byref(alloc) if alloc is not None else None,
                        stream, C.byref(handle))


def fmm_eval(plan: Plan, charges, potentials=None, fields=None, stream=None, want_fields=True):
    """One FMM evaluation; returns (potentials, fields) in input order.
    Outputs default to new tensors on the charges' device (or numpy arrays)."""
    lib = load()
    if potentials is None:
        potentials, fields = _alloc_outputs(charges, plan.n, want_fields)
    qp, qk = _ptr(charges)
    pp, pk = _ptr(potentials)
    fp, fk = _ptr(fields)
    _check(lib.fmm_eval(plan.handle, qp, pp, fp, _stream(stream)), "fmm_eval")
    return potentials, fields


def _alloc_outputs(like, n, want_fields):
    if _is_torch(like):
        import torch
        pot = torch.empty(n, dtype=like.dtype, device=like.device)
        fld = torch.empty((n, 3), dtype=like.dtype, device=like.device) if want_fields else None
        return pot, fld
    dt = np.asarray(like).dtype
    return np.empty(n, dt), (np.empty((n, 3), dt) if want_fields else None)


def fmm_destroy(plan: Plan) -> None:
    if plan.handle:
        load().fmm_destroy(plan.handle)
        plan.handle = None


def fmm_direct(points, charges, targets, potentials=None, fields=None, stream=None):
    """Exact Eq. 2.1 sum at `targets` (int64 indices) on the GPU in FP64."""
    lib = load()
    n = int(points.shape[0])
    dt = _dtype_code(points)
    if _is_torch(targets):
        import torch
        targets = targets.to(torch.int64).contiguous()
    else:
        targets = np.ascontiguousarray(targets, np.int64)
    nt = int(targets.shape[0])
    if potentials is None:
        potentials, fields = _alloc_outputs(charges, nt, True)
    a, ak = _ptr(points)
    b, bk = _ptr(charges)
    t, tk = _ptr(targets)
    pp, pk = _ptr(potentials)
    fp, fk = _ptr(fields)
    _check(lib.fmm_direct(a, b, n, dt, t, nt, pp, fp, _stream(stream)), "fmm_direct")
    return potentials, fields


def fmm_plan_stats(plan: Plan) -> dict:
    s = fmm_stats()
    _check(load().fmm_plan_stats(plan.handle, C.byref(s)), "fmm_plan_stats")
    out = {k: getattr(s, k) for k, _ in fmm_stats._fields_ if k != "weak_pairs_level"}
    out["weak_pairs_level"] = list(s.weak_pairs_level)[: s.levels + 1]
    return out


def fmm_plan_tree(plan: Plan) -> dict:
    nb = (2 << plan.levels) - 1
    out = dict(perm=np.zeros(plan.n, np.int64), begin=np.zeros(nb, np.int64),
               count=np.zeros(nb, np.int64), lo=np.zeros((nb, 3)), hi=np.zeros((nb, 3)),
               centre=np.zeros((nb, 3)), radius=np.zeros(nb), axis=np.zeros(nb, np.int32),
               plane=np.zeros(nb))
    args = [out[k].ctypes.data for k in ("perm", "begin", "count", "lo", "hi", "centre",
                                         "radius", "axis", "plane")]
    _check(load().fmm_plan_tree(plan.handle, *args), "fmm_plan_tree")
    return out


def fmm_plan_list(plan: Plan, level: int, kind: str):
    """CSR (ptr int64, src int32) of the 'weak' or 'strong' list of a level."""
    k = {"weak": 0, "strong": 1}[kind]
    ptr = np.zeros((1 << level) + 1, np.int64)
    lib = load()
    _check(lib.fmm_plan_list(plan.handle, level, k, ptr.ctypes.data, None), "fmm_plan_list")
    src = np.zeros(max(int(ptr[-1]), 1), np.int32)
    _check(lib.fmm_plan_list(plan.handle, level, k, ptr.ctypes.data, src.ctypes.data),
           "fmm_plan_list")
    return ptr, src[: int(ptr[-1])]


def fmm_eval_check(plan: Plan) -> None:
    """Synchronise and raise if a device-side wait of an evaluation ran out."""
    _check(load().fmm_eval_check(plan.handle), "fmm_eval_check")


def fmm_eval_expansions(plan: Plan, which: str) -> np.ndarray:
    """'M' or 'L' coefficients of every box after the last fmm_eval."""
    nb = (2 << plan.levels) - 1
    nc = (plan.p + 1) * (plan.p + 2) // 2
    out = np.zeros(nb * nc * 2)
    _check(load().fmm_eval_expansions(plan.handle, {"M": 0, "L": 1}[which], out.ctypes.data),
           "fmm_eval_expansions")
    return out.view(np.complex128).reshape(nb, nc)


def fmm_strerror(status: int) -> str:
    return load().fmm_strerror(status).decode()


def fmm_stage_times(plan: Plan) -> dict:
    """Device ms per stage of the plan build and its last evaluation
    (the plan must have been made with profile=True)."""
    ms = np.zeros(len(STAGES))
    _check(load().fmm_stage_times(plan.handle, ms.ctypes.data), "fmm_stage_times")
    return dict(zip(STAGES, ms.tolist()))


def fmm_pool_trim(device: int = 0) -> None:
    """Return the memory cached by the library's own pool on `device` (plans
    made with allocator=None) to the system."""
    _check(load().fmm_pool_trim(int(device)), "fmm_pool_trim")


PEAK_KINDS = {"ffma": 0, "ffma2": 1, "dfma": 2, "rsqrt": 3}


def fmm_measure_peak(kind: str, iters: int = 1 << 16, stream=None):
    """(ops per second, ms) of one arithmetic pipe: 'ffma', 'ffma2', 'dfma'
    (flop/s) or 'rsqrt' (XU operations/s)."""
    v, ms = C.c_double(), C.c_double()
    _check(load().fmm_measure_peak(PEAK_KINDS[kind], int(iters), _stream(stream), C.byref(v), C.byref(ms)),
           "fmm_measure_peak")
    return v.value, ms.value


def fmm_set_wait_limit(sleeps: int, withhold: int = -1) -> int:
    """Bound of the downward pass's device waits (sleeps of ~0.1 us; <= 0:
    default) and, for tests, a box whose completion is never signalled."""
    return int(load().fmm_set_wait_limit(int(sleeps), int(withhold)))


def fmm_set_list_capacity(entries: int) -> int:
    """Largest candidate-pair count per connectivity level (tests lower it to
    reach FMM_ECAPACITY); returns the previous value. 0 restores the default."""
    return int(load().fmm_set_list_capacity(int(entries)))


def fmm_kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().fmm_kernel_launches())


def fmm_orb_order_noalloc(points, levels: int, perm=None, stream=None):
    """Leaf order of the balanced tree for <= 4096 points without any device
    allocation inside the library (for callers whose host application owns
    all device memory, or whose loop cannot wait on an allocator). `points`
    is a contiguous (n, 3) float64/float32 CUDA tensor; `perm` an int32 CUDA
    tensor of at least n entries on the same device (created here if not
    given). Raises FmmError(FMM_EINVAL) for anything else."""
    import torch
    if (not _is_torch(points) or not points.is_cuda or points.dim() != 2 or points.shape[1] != 3
            or not points.is_contiguous()):
        raise FmmError(-1, "fmm_orb_order_noalloc: points must be a contiguous (n, 3) CUDA tensor")
    n = int(points.shape[0])
    if perm is None:
        perm = torch.empty(n, dtype=torch.int32, device=points.device)
    elif (not _is_torch(perm) or perm.dtype != torch.int32 or perm.device != points.device
          or perm.numel() < n or not perm.is_contiguous()):
        raise FmmError(-1, "fmm_orb_order_noalloc: perm must be a contiguous int32 tensor of "
                           "at least n entries on the points' device")
    _check(load().fmm_orb_order_noalloc(points.data_ptr(), n, _dtype_code(points), int(levels),
                                        perm.data_ptr(), _stream(stream)),
           "fmm_orb_order_noalloc")
    return perm


class Batch:
    """Owning handle of an fmm_batch_t (graph of many evaluations)."""

    def __init__(self, handle, keep):
        self.handle, self._keep = handle, keep

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.fmm_batch_destroy(self.handle)
            self.handle = None


def fmm_batch_create(plans, charges, potentials, fields=None, nstreams: int = 16, stream=None):
    """Record the evaluations of many plans (device buffers) into one graph."""
    lib = load()
    n = len(plans)
    arr = lambda xs: (C.c_void_p * n)(*[(x.data_ptr() if x is not None else None) for x in xs])
    hp, hq, hpot = (C.c_void_p * n)(*[p.handle for p in plans]), arr(charges), arr(potentials)
    hf = arr(fields) if fields is not None else None
    h = C.c_void_p()
    _check(lib.fmm_batch_create(hp, n, hq, hpot, hf, int(nstreams), _stream(stream), C.byref(h)),
           "fmm_batch_create")
    return Batch(h.value, (plans, charges, potentials, fields))


def fmm_batch_launch(batch: Batch, stream=None) -> None:
    _check(load().fmm_batch_launch(batch.handle, _stream(stream)), "fmm_batch_launch")


def fmm_batch_info(batch: Batch) -> dict:
    """{'kernels': kernel launches per fmm_batch_launch, 'fused': batched stages (True) or per-plan branches}"""
    k, f = C.c_int64(), C.c_int32()
    _check(load().fmm_batch_info(batch.handle, C.byref(k), C.byref(f)), "fmm_batch_info")
    return {"kernels": int(k.value), "fused": bool(f.value)}


def fmm_batch_destroy(batch: Batch) -> None:
    if batch.handle:
        load().fmm_batch_destroy(batch.handle)
        batch.handle = None
