"""Plain FP64 CPU oracle of the Magritte radiation-field hot path.

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
CPU-baseline leg of ``bench.py`` may import this package; the library under
``paper_2011_14998_gb300`` never does.  The arithmetic lives in ``oracle.c``
(plain C, double precision, no fused multiply-add) and in ``mlp.py`` (NumPy);
this module only compiles and marshals.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FP contraction, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


class Model(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("pos", C.c_void_p), ("vel", C.c_void_p),
        ("nbr_off", C.c_void_p), ("nbr_idx", C.c_void_p),
        ("n_lines", C.c_int32), ("nu0", C.c_void_p), ("chi0", C.c_void_p),
        ("eta0", C.c_void_p), ("dvw", C.c_void_p), ("chi_c", C.c_void_p),
        ("eta_c", C.c_void_p), ("n_freq", C.c_int32), ("x_span", C.c_double),
        ("l_min", C.c_int32), ("l_max", C.c_int32), ("rays", C.c_void_p),
    ]


class Params(C.Structure):
    _fields_ = [("dtau_max", C.c_double), ("dv_max", C.c_double), ("I_bdy", C.c_double),
                ("order", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            i64, i32, u64, dbl, vp = C.c_int64, C.c_int32, C.c_uint64, C.c_double, C.c_void_p
            sig = {
                "orc_npix": (i64, [C.c_int]),
                "orc_pix2vec_nest": (None, [C.c_int, i64, vp]),
                "orc_vec2pix_nest": (i64, [C.c_int, vp]),
                "orc_antipode": (i64, [C.c_int, i64]),
                "orc_rayset_npairs": (i64, [C.c_int, C.c_int]),
                "orc_rayset_one": (C.c_int, [i64, vp, i64, i64, vp, C.c_int, C.c_int, vp]),
                "orc_rayset": (C.c_int, [i64, vp, i64, vp, C.c_int, C.c_int, vp, C.c_int]),
                "orc_trace_half": (i64, [vp, i64, vp, i64, vp, vp]),
                "orc_profile_arg": (dbl, [dbl, dbl, dbl, dbl, dbl, dbl]),
                "orc_bin_x": (dbl, [i32, dbl, i32]),
                "orc_subdivide": (i64, [i64, vp, vp, vp, i64, dbl, i64, vp, vp, vp]),
                "orc_feautrier": (dbl, [i64, vp, vp, i64, dbl, vp]),
                "orc_feautrier4": (dbl, [i64, vp, vp, i64, dbl, vp]),
                "orc_analytic_mesh": (i64, [i32, i32, i32, vp, dbl, dbl, dbl, C.c_uint64, vp, vp, vp]),
                "orc_pair_line": (i64, [vp, vp, i64, C.c_uint32, i32, i32, i64, vp, vp, vp]),
                "orc_vline_size": (i64, [vp, vp, i64, C.c_uint32, vp]),
                "orc_solve_J": (C.c_int, [vp, vp, i64, vp, i64, vp, C.c_int]),
                "orc_solve_u": (C.c_int, [vp, vp, i64, vp, i64, vp, C.c_int]),
                "orc_uniform01": (dbl, [u64, i64]),
                "orc_reduce": (None, [i64, vp, vp, vp, vp, dbl, dbl, dbl, u64, vp, vp, vp, vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- HEALPix
def npix(l: int) -> int:
    return int(lib().orc_npix(l))


def pix2vec(l: int, p) -> np.ndarray:
    ps = np.atleast_1d(np.asarray(p, dtype=np.int64))
    out = np.empty((ps.size, 3))
    v = np.empty(3)
    for i, q in enumerate(ps):
        lib().orc_pix2vec_nest(l, int(q), _p(v))
        out[i] = v
    return out if np.ndim(p) else out[0]


def vec2pix(l: int, d) -> np.ndarray:
    d = np.ascontiguousarray(np.atleast_2d(np.asarray(d, dtype=np.float64)))
    out = np.empty(len(d), dtype=np.int64)
    for i in range(len(d)):
        out[i] = lib().orc_vec2pix_nest(l, _p(np.ascontiguousarray(d[i])))
    return out


def antipode(l: int, p: int) -> int:
    return int(lib().orc_antipode(l, int(p)))


# ---------------------------------------------------------------- ray sets
def rayset_npairs(l_min: int, l_max: int) -> int:
    return int(lib().orc_rayset_npairs(l_min, l_max))


def rayset(pos, l_min, l_max, sample=None, threads=None) -> np.ndarray:
    """[n][npairs] uint32 ray sets, (level << 28) | pixel, one global sample."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = len(pos)
    sample = np.zeros(0, np.int32) if sample is None else np.ascontiguousarray(sample, np.int32)
    npairs = rayset_npairs(l_min, l_max)
    out = np.zeros((n, npairs), dtype=np.uint32)
    rc = lib().orc_rayset(n, _p(pos), len(sample), _p(sample), l_min, l_max, _p(out),
                          threads or os.cpu_count() or 1)
    if rc != 0:
        raise ValueError("oracle ray set failed")
    return out


def rayset_at(pos, origins, l_min, l_max, sample=None) -> np.ndarray:
    """Ray sets of the given origins only: [len(origins)][npairs]."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    sample = np.zeros(0, np.int32) if sample is None else np.ascontiguousarray(sample, np.int32)
    npairs = rayset_npairs(l_min, l_max)
    out = np.zeros((len(origins), npairs), dtype=np.uint32)
    for q, o in enumerate(origins):
        row = np.zeros(npairs, np.uint32)
        if lib().orc_rayset_one(len(pos), _p(pos), int(o), len(sample), _p(sample), l_min, l_max, _p(row)) != 0:
            raise ValueError("oracle ray set failed")
        out[q] = row
    return out


# ---------------------------------------------------------------- model
class OracleModel:
    """Holds contiguous FP64 copies of a model and the oracle's own ray set."""

    def __init__(self, m, l_min=None, l_max=None, sample=None, rays=None, threads=None):
        self.pos = np.ascontiguousarray(m["pos"], np.float64)
        self.vel = np.ascontiguousarray(m["vel"], np.float64)
        self.nbr_off = np.ascontiguousarray(m["nbr_off"], np.int64)
        self.nbr_idx = np.ascontiguousarray(m["nbr_idx"], np.int32)
        self.nu0 = np.ascontiguousarray(m["nu0"], np.float64)
        self.chi0 = np.ascontiguousarray(m["chi0"], np.float64)
        self.eta0 = np.ascontiguousarray(m["eta0"], np.float64)
        self.dvw = np.ascontiguousarray(m["dvw"], np.float64)
        self.chi_c = np.ascontiguousarray(m["chi_c"], np.float64)
        self.eta_c = np.ascontiguousarray(m["eta_c"], np.float64)
        self.n_freq = int(m["n_freq"])
        self.x_span = float(m["x_span"])
        self.l_min = int(m["l_min"] if l_min is None else l_min)
        self.l_max = int(m["l_max"] if l_max is None else l_max)
        if rays is None:
            smp = m.get("sample") if sample is None else sample
            rays = rayset(self.pos, self.l_min, self.l_max, smp, threads)
        self.rays = np.ascontiguousarray(rays, np.uint32)
        n = len(self.pos)
        if self.rays.shape != (n, rayset_npairs(self.l_min, self.l_max)):
            raise ValueError(f"rays {self.rays.shape} do not match {n} points at levels {self.l_min}..{self.l_max}")
        self.s = Model(n, self.pos.ctypes.data, self.vel.ctypes.data, self.nbr_off.ctypes.data,
                       self.nbr_idx.ctypes.data, len(self.nu0), self.nu0.ctypes.data,
                       self.chi0.ctypes.data, self.eta0.ctypes.data, self.dvw.ctypes.data,
                       self.chi_c.ctypes.data, self.eta_c.ctypes.data, self.n_freq, self.x_span,
                       self.l_min, self.l_max, self.rays.ctypes.data)

    @property
    def n(self):
        return len(self.pos)

    def trace_half(self, o: int, d) -> tuple[np.ndarray, np.ndarray]:
        d = np.ascontiguousarray(d, np.float64)
        cap = self.n + 1
        idx = np.empty(cap, np.int32)
        Z = np.empty(cap, np.float64)
        k = lib().orc_trace_half(C.byref(self.s), int(o), _p(d), cap, _p(idx), _p(Z))
        return idx[:k].copy(), Z[:k].copy()

    def pair_line(self, o, ray, l, k, params, max_pts=1 << 22):
        dtau = np.empty(max_pts)
        S = np.empty(max_pts + 1)
        io = C.c_int64(0)
        M = lib().orc_pair_line(C.byref(self.s), C.byref(params), int(o), int(ray), int(l), int(k),
                                max_pts, _p(dtau), _p(S), C.byref(io))
        if M < 0:
            raise ValueError("line too long")
        return dtau[:M].copy(), S[:M + 1].copy(), int(io.value)

    def vline_size(self, o, ray, params):
        io = C.c_int64(0)
        mv = lib().orc_vline_size(C.byref(self.s), C.byref(params), int(o), int(ray), C.byref(io))
        return int(mv), int(io.value)

    def solve_J(self, params, origins=None, threads=None, max_pts=1 << 22) -> np.ndarray:
        origins = np.arange(self.n, dtype=np.int64) if origins is None else \
            np.ascontiguousarray(origins, np.int64)
        nb = len(self.nu0) * self.n_freq
        J = np.zeros((len(origins), nb))
        rc = lib().orc_solve_J(C.byref(self.s), C.byref(params), len(origins), _p(origins), max_pts,
                               _p(J), threads or os.cpu_count() or 1)
        if rc != 0:
            raise ValueError("oracle solve failed (line longer than max_pts or bad sizes)")
        return J

    def solve_u(self, params, origins, threads=None, max_pts=1 << 22) -> np.ndarray:
        """u at the origin of every pair line: [len(origins), pairs, L*F]."""
        origins = np.ascontiguousarray(origins, np.int64)
        nb = len(self.nu0) * self.n_freq
        u = np.zeros((len(origins), self.rays.shape[1], nb))
        rc = lib().orc_solve_u(C.byref(self.s), C.byref(params), len(origins), _p(origins), max_pts, _p(u),
                               threads or os.cpu_count() or 1)
        if rc != 0:
            raise ValueError("oracle solve failed (line longer than max_pts or bad sizes)")
        return u


def params(dtau_max=0.5, dv_max=1.0 / 3.0, I_bdy=0.0, order=2) -> Params:
    """order: 2 (second-order scheme) or 4 (Hermitian scheme, Section 2.1)."""
    if order not in (2, 4):
        raise ValueError("order must be 2 or 4")
    return Params(dtau_max, dv_max, I_bdy, int(order))


def feautrier(dtau, S, io, I_bdy=0.0, all_rows=False, order=2):
    dtau = np.ascontiguousarray(dtau, np.float64)
    S = np.ascontiguousarray(S, np.float64)
    M = len(dtau)
    u = np.empty(M + 1)
    fn = lib().orc_feautrier4 if order == 4 else lib().orc_feautrier
    uo = fn(M, _p(dtau), _p(S), int(io), float(I_bdy), _p(u))
    return u if all_rows else uo


def subdivide(s, chi, eta, io, dtau_max, max_pts=1 << 20):
    s = np.ascontiguousarray(s, np.float64)
    chi = np.ascontiguousarray(chi, np.float64)
    eta = np.ascontiguousarray(eta, np.float64)
    dtau = np.empty(max_pts)
    S = np.empty(max_pts + 1)
    ioo = C.c_int64(0)
    M = lib().orc_subdivide(len(s), _p(s), _p(chi), _p(eta), int(io), float(dtau_max), max_pts, _p(dtau),
                            _p(S), C.byref(ioo))
    if M < 0:
        raise ValueError("too many sub-points")
    return dtau[:M].copy(), S[:M + 1].copy(), int(ioo.value)


def profile_arg(nu_l, nu_lp, x, dv_o, delta, dv):
    return float(lib().orc_profile_arg(nu_l, nu_lp, x, dv_o, delta, dv))


def bin_x(n_freq, x_span, k):
    return float(lib().orc_bin_x(n_freq, x_span, k))


# ---------------------------------------------------------------- reduction
def uniform01(seed: int, i: int) -> float:
    return float(lib().orc_uniform01(C.c_uint64(seed & (2**64 - 1)), int(i)))


def reduce(pos, nbr_off, nbr_idx, f, f_small, f_large, G_thres, seed):
    pos = np.ascontiguousarray(pos, np.float64)
    nbr_off = np.ascontiguousarray(nbr_off, np.int64)
    nbr_idx = np.ascontiguousarray(nbr_idx, np.int32)
    f = np.ascontiguousarray(f, np.float64)
    n = len(pos)
    Gf, L, ell = np.empty(n), np.empty(n), np.empty(n)
    keep = np.empty(n, np.uint8)
    lib().orc_reduce(n, _p(pos), _p(nbr_off), _p(nbr_idx), _p(f), f_small, f_large, G_thres,
                     C.c_uint64(seed & (2**64 - 1)), _p(Gf), _p(L), _p(ell), _p(keep))
    return Gf, L, ell, keep


def analytic_mesh(f, h, ell_min, ell_max, seed):
    """Element-size field of a tracer f [nx, ny, nz] on a Cartesian background
    mesh of spacing h (Section 2.2.1, Eq. 5) and its thinning to the density
    ell^-3 (keep probability (h / ell)^3): (Gf, ell, keep)."""
    f = np.ascontiguousarray(f, np.float64)
    nx, ny, nz = f.shape
    Gf = np.empty(f.size)
    ell = np.empty(f.size)
    keep = np.empty(f.size, np.uint8)
    lib().orc_analytic_mesh(nx, ny, nz, _p(f), float(h), float(ell_min), float(ell_max), int(seed), _p(Gf),
                            _p(ell), _p(keep))
    return Gf.reshape(f.shape), ell.reshape(f.shape), keep.reshape(f.shape)
