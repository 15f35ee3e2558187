"""FP64 CPU oracle for the balanced-tree FMM (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It wraps ``fmm_oracle.c`` (plain C,
double precision, no code shared with the CUDA implementation) through
ctypes. The shared object is compiled with gcc into ``oracle/_build`` on
first use, or ahead of time by :func:`build`.

Every function follows a passage of Bull & Engblom, arXiv:2002.04894:
Eq. 2.1 (the pairwise sum), Eq. 2.2 (the theta-criterion), Sec. 2.1.2 (median
splits of a balanced tree) and Algorithms 1-4 (the stage order).
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = None

_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_c128p = np.ctypeslib.ndpointer(np.complex128, flags="C_CONTIGUOUS")


def _lib_path() -> str:
    return os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP if present)."""
    out = _lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", _SRC, "-o", out + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(out + ".tmp", out)
    return out


def _lib():
    global _LIB
    if _LIB is not None:
        return _LIB
    lib = C.CDLL(build())
    lib.orc_ncoef.argtypes = [C.c_int]
    lib.orc_ncoef.restype = C.c_int
    lib.orc_regular.argtypes = [_f64p, C.c_int, _c128p]
    lib.orc_irregular.argtypes = [_f64p, C.c_int, _c128p]
    lib.orc_p2m.argtypes = [C.c_int64, _f64p, _f64p, _f64p, C.c_int, _c128p]
    lib.orc_m2m.argtypes = [_c128p, _f64p, _f64p, C.c_int, _c128p]
    lib.orc_m2l.argtypes = [_c128p, _f64p, _f64p, C.c_int, _c128p]
    lib.orc_l2l.argtypes = [_c128p, _f64p, _f64p, C.c_int, _c128p]
    lib.orc_l2p.argtypes = [_c128p, _f64p, C.c_int, _f64p, _f64p, _f64p]
    lib.orc_direct.argtypes = [C.c_int64, _f64p, _f64p, C.c_int64, _i64p, _f64p, C.c_void_p]
    lib.orc_theta_weak.argtypes = [C.c_double, _f64p, C.c_double, _f64p, C.c_double]
    lib.orc_theta_weak.restype = C.c_int
    lib.orc_build.argtypes = [C.c_int64, _f64p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                              C.c_int, C.c_void_p, C.c_void_p]
    lib.orc_build.restype = C.c_void_p
    lib.orc_free.argtypes = [C.c_void_p]
    lib.orc_nbox.argtypes = [C.c_void_p]
    lib.orc_nbox.restype = C.c_int64
    lib.orc_get_tree.argtypes = [C.c_void_p, _i64p, _i64p, _i64p, _f64p, _f64p, _f64p,
                                 _f64p, _i32p, _f64p]
    lib.orc_list_size.argtypes = [C.c_void_p, C.c_int, C.c_int]
    lib.orc_list_size.restype = C.c_int64
    lib.orc_get_list.argtypes = [C.c_void_p, C.c_int, C.c_int, _i64p, _i32p]
    lib.orc_eval.argtypes = [C.c_void_p, _f64p, _f64p, C.c_void_p]
    lib.orc_get_expansions.argtypes = [C.c_void_p, C.c_int, _f64p]
    lib.orc_num_threads.restype = C.c_int
    lib.orc_bisect_box.argtypes = [C.c_int64, _f64p, _f64p, _f64p,
                                   np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS"), _f64p]
    lib.orc_bisect_box.restype = C.c_int
    _LIB = lib
    return lib


def ncoef(p: int) -> int:
    """Number of stored coefficients (n, m), 0 <= m <= n <= p."""
    return (p + 1) * (p + 2) // 2


def num_threads() -> int:
    return int(_lib().orc_num_threads())


def _vec3(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(3))


def regular(x, p: int) -> np.ndarray:
    """R_n^m(x), packed triangle (n(n+1)/2 + m), no Condon-Shortley phase."""
    out = np.zeros(ncoef(p), np.complex128)
    _lib().orc_regular(_vec3(x), p, out)
    return out


def irregular(x, p: int) -> np.ndarray:
    """I_n^m(x) = (n-m)! P_n^m(cos t) e^{i m phi} / r^{n+1}, packed triangle."""
    out = np.zeros(ncoef(p), np.complex128)
    _lib().orc_irregular(_vec3(x), p, out)
    return out


def p2m(x, q, c, p: int, M=None) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, np.float64)
    M = np.zeros(ncoef(p), np.complex128) if M is None else M
    _lib().orc_p2m(len(q), x, q, _vec3(c), p, M)
    return M


def m2m(Mc, cc, cp, p: int, Mp=None) -> np.ndarray:
    Mp = np.zeros(ncoef(p), np.complex128) if Mp is None else Mp
    _lib().orc_m2m(np.ascontiguousarray(Mc), _vec3(cc), _vec3(cp), p, Mp)
    return Mp


def m2l(Ms, cs, ct, p: int, Lt=None) -> np.ndarray:
    Lt = np.zeros(ncoef(p), np.complex128) if Lt is None else Lt
    _lib().orc_m2l(np.ascontiguousarray(Ms), _vec3(cs), _vec3(ct), p, Lt)
    return Lt


def l2l(Lp, cp, cc, p: int, Lc=None) -> np.ndarray:
    Lc = np.zeros(ncoef(p), np.complex128) if Lc is None else Lc
    _lib().orc_l2l(np.ascontiguousarray(Lp), _vec3(cp), _vec3(cc), p, Lc)
    return Lc


def l2p(L, c, p: int, x):
    """Potential and field E = -grad phi of a local expansion at x."""
    phi = np.zeros(1)
    E = np.zeros(3)
    _lib().orc_l2p(np.ascontiguousarray(L), _vec3(c), p, _vec3(x), phi, E)
    return float(phi[0]), E


def direct(x, q, targets=None, field: bool = True):
    """Exact sum of Eq. 2.1 at the given target indices (default: all)."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, np.float64)
    n = len(q)
    t = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
    phi = np.zeros(len(t))
    E = np.zeros((len(t), 3)) if field else None
    _lib().orc_direct(n, x, q, len(t), t, phi,
                      E.ctypes.data_as(C.c_void_p) if field else None)
    return (phi, E) if field else phi


def theta_weak(theta: float, ca, ra: float, cb, rb: float) -> bool:
    return bool(_lib().orc_theta_weak(theta, _vec3(ca), ra, _vec3(cb), rb))


def bisect_box(x, lo, hi):
    """One median bisection of a box given its points (ascending original
    index) and cell: returns (axis, left mask, plane)."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    left = np.zeros(len(x), np.int8)
    plane = np.zeros(1)
    ax = _lib().orc_bisect_box(len(x), x, _vec3(lo), _vec3(hi), left, plane)
    return int(ax), left.astype(bool), float(plane[0])


class Tree:
    """Balanced tree, connectivity and expansions of one point set."""

    def __init__(self, x, levels: int, p: int, theta: float, eta: float = 1.0, step: int = 1,
                 tight: bool = False, root_cell=None):
        """`levels` bisections; `step` bisections per FMM level (3: octree
        levels of 8 children), `levels` a multiple of it; `tight`: box centres
        and radii from each box's own points instead of its cell; `root_cell`
        = (lo[3], hi[3]) replaces the points' bounding box as the root cell."""
        x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
        if step < 1 or levels % step:
            raise ValueError("levels must be a multiple of step >= 1")
        self.n, self.levels, self.p, self.theta, self.eta, self.step = len(x), levels, p, theta, eta, step
        self.tight = bool(tight)
        rl = rh = None
        if root_cell is not None:
            self._root = (np.ascontiguousarray(root_cell[0], np.float64).reshape(3),
                          np.ascontiguousarray(root_cell[1], np.float64).reshape(3))
            rl, rh = self._root[0].ctypes.data, self._root[1].ctypes.data
        self._h = _lib().orc_build(self.n, x, levels, p, theta, eta, step, int(self.tight), rl, rh)
        if not self._h:
            raise MemoryError("oracle build failed")

    def __del__(self):
        if getattr(self, "_h", None):
            _lib().orc_free(self._h)
            self._h = None

    @property
    def nbox(self) -> int:
        return (2 << self.levels) - 1

    def tree(self) -> dict:
        nb = self.nbox
        out = dict(perm=np.zeros(self.n, np.int64), begin=np.zeros(nb, np.int64),
                   count=np.zeros(nb, np.int64), lo=np.zeros((nb, 3)), hi=np.zeros((nb, 3)),
                   centre=np.zeros((nb, 3)), radius=np.zeros(nb),
                   axis=np.zeros(nb, np.int32), plane=np.zeros(nb))
        _lib().orc_get_tree(self._h, out["perm"], out["begin"], out["count"], out["lo"],
                            out["hi"], out["centre"], out["radius"], out["axis"], out["plane"])
        return out

    def lists(self, level: int, kind: str):
        """CSR (ptr, src) of the weak ('weak') or strong ('strong') list."""
        k = {"weak": 0, "strong": 1}[kind]
        size = int(_lib().orc_list_size(self._h, level, k))
        ptr = np.zeros((1 << level) + 1, np.int64)
        src = np.zeros(max(size, 1), np.int32)
        _lib().orc_get_list(self._h, level, k, ptr, src)
        return ptr, src[:size]

    def eval(self, q, field: bool = True):
        q = np.ascontiguousarray(q, np.float64)
        phi = np.zeros(self.n)
        E = np.zeros((self.n, 3)) if field else None
        _lib().orc_eval(self._h, q, phi, E.ctypes.data_as(C.c_void_p) if field else None)
        return (phi, E) if field else phi

    def expansions(self, which: str) -> np.ndarray:
        """Per-box coefficients after eval: 'M' (multipole) or 'L' (local)."""
        out = np.zeros(self.nbox * ncoef(self.p) * 2)
        _lib().orc_get_expansions(self._h, {"M": 0, "L": 1}[which], out)
        return out.view(np.complex128).reshape(self.nbox, ncoef(self.p))
