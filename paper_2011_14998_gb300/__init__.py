"""GB300 radiation-field library (Magritte II hot path) -- Python binding.

Thin ctypes marshalling over the C ABI in ``include/mgx.h``; every step of
the method runs in the CUDA kernels of ``libmgx.so``.  PyTorch supplies the
CUDA stream (and device tensors for device-side outputs).  There is no CPU
fallback: if the shared library is missing or fails to load, every call raises.

The functions keep the C names (``mgx_create``, ``mgx_load_mesh`` ...); the
``Context`` class is a convenience wrapper that owns one context.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmgx.so")

MGX_OK, MGX_EINVAL, MGX_ENOMEM, MGX_ECUDA, MGX_ESTATE, MGX_ERANGE = 0, -1, -2, -3, -4, -6
MGX_FP64, MGX_FP32, MGX_FP32_DT64 = 0, 1, 2
MGX_MAX_LINES = 8

# every symbol the header declares
ABI_SYMBOLS = ("mgx_create", "mgx_destroy", "mgx_last_error", "mgx_rayset_npairs", "mgx_load_mesh",
               "mgx_free_model", "mgx_set_lines", "mgx_set_rays", "mgx_get_rays", "mgx_trace",
               "mgx_solve_J", "mgx_reduce_mesh", "mgx_profile_enable", "mgx_profile_read",
               "mgx_solve_J_noalloc", "mgx_solve_J_batch", "mgx_mlp_set_params", "mgx_mlp_get_params",
               "mgx_mlp_forward", "mgx_mlp_grad", "mgx_mlp_train", "mgx_mlp_features", "mgx_reduce_mesh_learned",
               "mgx_set_tuning", "mgx_get_tuning", "mgx_autotune", "mgx_analytic_mesh", "mgx_solve_u",
               "mgx_pix2vec", "mgx_antipode", "mgx_reduce_mesh_learned_weighted", "mgx_eval_approx", "mgx_alu_peaks")
MGX_MLP_NPARAM = 4801
MGX_BATCH_GRAPH, MGX_BATCH_RAYS = 1, 2
KERNEL_CLASSES = ("rays", "trace_count", "scan", "trace_emit", "solve", "other")


class MgxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mgx status {status}: {msg}")
        self.status = status


class SolveParams(C.Structure):
    _fields_ = [("dtau_max", C.c_double), ("dv_max", C.c_double), ("I_bdy", C.c_double),
                ("precision", C.c_int32), ("out_on_device", C.c_int32), ("order", C.c_int32),
                ("reserved", C.c_int32)]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 6), ("launches", C.c_int64 * 6), ("trace_points", C.c_int64),
                ("solves", C.c_int64), ("updates", C.c_int64), ("samples", C.c_int64),
                ("trace_steps", C.c_int64), ("trace_exact_steps", C.c_int64), ("decisions_redone", C.c_int64)]


class Tuning(C.Structure):
    _fields_ = [("bins_per_lane", C.c_int32), ("trace_ctas_per_sm", C.c_int32), ("tail_permille", C.c_int32),
                ("schedule", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class TuneTrial(C.Structure):
    _fields_ = [("tuning", Tuning), ("step_ms", C.c_double)]


_lib = None


def build(force: bool = False) -> str:
    from . import _build

    return _build.build(force=force)


def load_library(path: str = LIB_PATH):
    """Load libmgx.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmgx.so not built ({path}); run paper_2011_14998_gb300.build()")
    L = C.CDLL(path)
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    sig = {
        "mgx_create": (i32, [C.c_int, vp, C.POINTER(vp)]),
        "mgx_destroy": (None, [vp]),
        "mgx_last_error": (C.c_char_p, [vp]),
        "mgx_rayset_npairs": (i64, [i32, i32]),
        "mgx_load_mesh": (i32, [vp, i64, vp, vp, vp, vp, C.POINTER(i32)]),
        "mgx_free_model": (i32, [vp, i32]),
        "mgx_set_lines": (i32, [vp, i32, i32, vp, vp, vp, vp, vp, vp, i32, dbl]),
        "mgx_set_rays": (i32, [vp, i32, i32, i32, i64, vp]),
        "mgx_get_rays": (i32, [vp, i32, vp]),
        "mgx_trace": (i32, [vp, i32, i64, i64, vp, vp, vp, vp, i64]),
        "mgx_solve_J": (i32, [vp, i32, C.POINTER(SolveParams), vp]),
        "mgx_reduce_mesh": (i32, [vp, i32, vp, dbl, dbl, dbl, u64, vp, vp, vp, vp, C.POINTER(i64)]),
        "mgx_solve_J_noalloc": (i32, [vp, i32, C.POINTER(SolveParams), vp]),
        "mgx_solve_J_batch": (i32, [vp, vp, i32, C.POINTER(SolveParams), vp, i32]),
        "mgx_mlp_set_params": (i32, [vp, vp]),
        "mgx_mlp_get_params": (i32, [vp, vp]),
        "mgx_mlp_forward": (i32, [vp, vp, i64, vp]),
        "mgx_mlp_grad": (i32, [vp, vp, vp, i64, vp, vp]),
        "mgx_mlp_train": (i32, [vp, vp, vp, i64, i32, i32, C.c_float, u64, vp]),
        "mgx_mlp_features": (i32, [vp, i32, vp, vp, vp]),
        "mgx_reduce_mesh_learned": (i32, [vp, i32, vp, dbl, vp, C.POINTER(i64)]),
        "mgx_profile_enable": (i32, [vp, i32]),
        "mgx_profile_read": (i32, [vp, C.POINTER(Profile)]),
        "mgx_eval_approx": (i32, [vp, i32, vp, i64, vp, C.POINTER(C.c_float)]),
        "mgx_alu_peaks": (i32, [vp, i32, vp]),
        "mgx_set_tuning": (i32, [vp, C.POINTER(Tuning)]),
        "mgx_pix2vec": (i32, [i32, i64, vp]),
        "mgx_reduce_mesh_learned_weighted": (i32, [vp, i32, vp, dbl, dbl, u64, vp, C.POINTER(i64),
                                                   C.POINTER(dbl)]),
        "mgx_antipode": (i64, [i32, i64]),
        "mgx_solve_u": (i32, [vp, i32, C.POINTER(SolveParams), i64, i64, vp]),
        "mgx_analytic_mesh": (i32, [vp, i32, i32, i32, vp, dbl, dbl, dbl, u64, vp, vp, vp, C.POINTER(i64)]),
        "mgx_get_tuning": (i32, [vp, C.POINTER(Tuning)]),
        "mgx_autotune": (i32, [vp, vp, i32, C.POINTER(SolveParams), vp, i32, i32, C.POINTER(TuneTrial), i32,
                               C.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(a) -> C.c_void_p | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    return C.c_void_p(a.data_ptr())  # torch tensor (host or device)


def _arr(a, dtype):
    """C-contiguous numpy view/copy, or a torch tensor passed through (pinned host buffers)."""
    if hasattr(a, "data_ptr") and not isinstance(a, np.ndarray):
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=dtype)


def _check(ctx, status: int):
    if status != MGX_OK:
        msg = load_library().mgx_last_error(ctx)
        raise MgxError(status, msg.decode() if msg else "")


# ------------------------------------------------------------ C-named wrappers
def mgx_create(device: int = 0, stream: int | None = None) -> C.c_void_p:
    out = C.c_void_p()
    st = load_library().mgx_create(int(device), C.c_void_p(stream) if stream else None, C.byref(out))
    if st != MGX_OK:
        raise MgxError(st, "mgx_create failed (no CUDA device?)")
    return out


def mgx_destroy(ctx) -> None:
    load_library().mgx_destroy(ctx)


def mgx_last_error(ctx) -> str:
    return load_library().mgx_last_error(ctx).decode()


def mgx_rayset_npairs(l_min: int, l_max: int) -> int:
    return int(load_library().mgx_rayset_npairs(int(l_min), int(l_max)))


def mgx_load_mesh(ctx, pos, vel, nbr_off, nbr_idx) -> int:
    pos, vel = _arr(pos, np.float64), _arr(vel, np.float64)
    nbr_off, nbr_idx = _arr(nbr_off, np.int64), _arr(nbr_idx, np.int32)
    mid = C.c_int32(-1)
    n = len(pos)
    _check(ctx, load_library().mgx_load_mesh(ctx, n, _ptr(pos), _ptr(vel), _ptr(nbr_off), _ptr(nbr_idx),
                                             C.byref(mid)))
    return mid.value


def mgx_free_model(ctx, model: int) -> None:
    _check(ctx, load_library().mgx_free_model(ctx, int(model)))


def mgx_set_lines(ctx, model, nu0, chi0, eta0, dvw, chi_c, eta_c, n_freq, x_span) -> None:
    nu0 = _arr(nu0, np.float64)
    arrs = [_arr(a, np.float64) for a in (chi0, eta0, dvw, chi_c, eta_c)]
    _check(ctx, load_library().mgx_set_lines(ctx, int(model), len(nu0), _ptr(nu0), *[_ptr(a) for a in arrs],
                                             int(n_freq), float(x_span)))


def mgx_set_rays(ctx, model, l_min, l_max, sample=None) -> None:
    smp = None if sample is None else _arr(sample, np.int32)
    ns = 0 if smp is None else len(smp)
    _check(ctx, load_library().mgx_set_rays(ctx, int(model), int(l_min), int(l_max), ns, _ptr(smp)))


def mgx_get_rays(ctx, model, n, npairs) -> np.ndarray:
    out = np.empty((n, npairs), np.uint32)
    _check(ctx, load_library().mgx_get_rays(ctx, int(model), _ptr(out)))
    return out


def mgx_trace(ctx, model, o_begin, o_end, npairs, with_delta=False, ids=True):
    """Returns (off [n_half+1], idx, Z, delta-or-None); with ids=False only the
    offsets are traced and (off, None, None, None) is returned."""
    n_half = (o_end - o_begin) * npairs * 2
    off = np.empty(n_half + 1, np.int64)
    L = load_library()
    _check(ctx, L.mgx_trace(ctx, int(model), int(o_begin), int(o_end), _ptr(off), None, None, None, 0))
    if not ids:
        return off, None, None, None
    tot = int(off[-1])
    idx = np.empty(max(tot, 1), np.int32)
    Z = np.empty(max(tot, 1), np.float64)
    de = np.empty(max(tot, 1), np.float64) if with_delta else None
    _check(ctx, L.mgx_trace(ctx, int(model), int(o_begin), int(o_end), _ptr(off), _ptr(idx), _ptr(Z),
                            _ptr(de), tot))
    return off, idx[:tot], Z[:tot], (de[:tot] if with_delta else None)


def mgx_solve_J(ctx, model, params: SolveParams, J_out) -> None:
    _check(ctx, load_library().mgx_solve_J(ctx, int(model), C.byref(params), _ptr(J_out)))


def mgx_solve_J_noalloc(ctx, model, params: SolveParams, J_out) -> None:
    """Allocation-free solve into a caller-owned CUDA tensor (see include/mgx.h)."""
    _check(ctx, load_library().mgx_solve_J_noalloc(ctx, int(model), C.byref(params), _ptr(J_out)))


def mgx_solve_J_batch(ctx, models, params: SolveParams, J_outs, flags: int = 0) -> None:
    """Batched solve of several models into contiguous float64 tensors J_outs[k], on the context's
    device or in host memory (see include/mgx.h)."""
    ids = np.ascontiguousarray(models, np.int32)
    ptrs = (C.c_void_p * len(J_outs))(*[t.data_ptr() for t in J_outs])
    _check(ctx, load_library().mgx_solve_J_batch(ctx, _ptr(ids), len(ids), C.byref(params), ptrs, int(flags)))


def mgx_reduce_mesh_learned_weighted(ctx, model, X, keep_fraction, alpha=1.0, seed=0):
    """Weighted learned thinning (see include/mgx.h); returns (keep, n_kept, scale)."""
    X = np.ascontiguousarray(X, np.float32)
    n = X.shape[0]
    keep = np.empty(n, np.uint8)
    nk = C.c_int64(0)
    sc = C.c_double(0.0)
    _check(ctx, load_library().mgx_reduce_mesh_learned_weighted(ctx, int(model), _ptr(X), float(keep_fraction),
                                                                float(alpha), int(seed) & (2**64 - 1), _ptr(keep),
                                                                C.byref(nk), C.byref(sc)))
    return keep, int(nk.value), float(sc.value)


def mgx_pix2vec(l: int, p: int) -> np.ndarray:
    v = np.empty(3)
    if load_library().mgx_pix2vec(int(l), int(p), _ptr(v)) != 0:
        raise ValueError("bad HEALPix level or pixel")
    return v


def mgx_antipode(l: int, p: int) -> int:
    a = load_library().mgx_antipode(int(l), int(p))
    if a < 0:
        raise ValueError("bad HEALPix level or pixel")
    return int(a)


def mgx_analytic_mesh(ctx, f, h, ell_min, ell_max, seed=0):
    """Element-size field of a tracer f [nx, ny, nz] on a Cartesian background
    mesh (Section 2.2.1, Eq. 5) and its thinning; returns (Gf, ell, keep, n_kept)."""
    f = np.ascontiguousarray(f, np.float64)
    nx, ny, nz = f.shape
    Gf = np.empty(f.shape)
    ell = np.empty(f.shape)
    keep = np.empty(f.shape, np.uint8)
    nk = C.c_int64(0)
    _check(ctx, load_library().mgx_analytic_mesh(ctx, nx, ny, nz, _ptr(f), float(h), float(ell_min), float(ell_max),
                                                 int(seed) & (2**64 - 1), _ptr(Gf), _ptr(ell), _ptr(keep),
                                                 C.byref(nk)))
    return Gf, ell, keep, int(nk.value)


def mgx_set_tuning(ctx, tuning: dict | None) -> None:
    """Set the batched solve's launch parameters (None: automatic; see include/mgx.h)."""
    t = None if tuning is None else C.byref(Tuning(**{k: int(v) for k, v in tuning.items()}))
    _check(ctx, load_library().mgx_set_tuning(ctx, t))


def mgx_get_tuning(ctx) -> dict:
    t = Tuning()
    _check(ctx, load_library().mgx_get_tuning(ctx, C.byref(t)))
    return t.as_dict()


def mgx_autotune(ctx, models, params: SolveParams, J_outs, flags: int = 0, reps: int = 3) -> list[dict]:
    """Time candidate tunings of the batched solve and keep the fastest; returns the trials."""
    ids = np.ascontiguousarray(models, np.int32)
    ptrs = (C.c_void_p * len(J_outs))(*[t.data_ptr() for t in J_outs])
    trials = (TuneTrial * 16)()
    n = C.c_int32(0)
    _check(ctx, load_library().mgx_autotune(ctx, _ptr(ids), len(ids), C.byref(params), ptrs, int(flags), int(reps),
                                            trials, 16, C.byref(n)))
    return [dict(trials[i].tuning.as_dict(), step_ms=float(trials[i].step_ms)) for i in range(min(n.value, 16))]


def mgx_mlp_set_params(ctx, theta) -> None:
    theta = np.ascontiguousarray(theta, np.float32)
    assert theta.size == MGX_MLP_NPARAM
    _check(ctx, load_library().mgx_mlp_set_params(ctx, _ptr(theta)))


def mgx_mlp_get_params(ctx) -> np.ndarray:
    out = np.empty(MGX_MLP_NPARAM, np.float32)
    _check(ctx, load_library().mgx_mlp_get_params(ctx, _ptr(out)))
    return out


def mgx_mlp_forward(ctx, X) -> np.ndarray:
    X = np.ascontiguousarray(X, np.float32)
    y = np.empty(len(X), np.float32)
    _check(ctx, load_library().mgx_mlp_forward(ctx, _ptr(X), len(X), _ptr(y)))
    return y


def mgx_mlp_grad(ctx, X, t):
    X = np.ascontiguousarray(X, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    g = np.empty(MGX_MLP_NPARAM, np.float32)
    loss = C.c_float(0.0)
    _check(ctx, load_library().mgx_mlp_grad(ctx, _ptr(X), _ptr(t), len(X), _ptr(g), C.byref(loss)))
    return g, float(loss.value)


def mgx_mlp_train(ctx, X, t, epochs, batch, lr, seed) -> np.ndarray:
    X = np.ascontiguousarray(X, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    losses = np.empty(epochs, np.float32)
    _check(ctx, load_library().mgx_mlp_train(ctx, _ptr(X), _ptr(t), len(X), int(epochs), int(batch), float(lr),
                                             C.c_uint64(int(seed) & (2**64 - 1)), _ptr(losses)))
    return losses


def mgx_mlp_features(ctx, model, rho, T) -> np.ndarray:
    rho = np.ascontiguousarray(rho, np.float64)
    T = np.ascontiguousarray(T, np.float64)
    X = np.empty((len(rho), 8), np.float32)
    _check(ctx, load_library().mgx_mlp_features(ctx, int(model), _ptr(rho), _ptr(T), _ptr(X)))
    return X


def mgx_reduce_mesh_learned(ctx, model, X, keep_fraction):
    X = np.ascontiguousarray(X, np.float32)
    keep = np.empty(len(X), np.uint8)
    nk = C.c_int64(0)
    _check(ctx, load_library().mgx_reduce_mesh_learned(ctx, int(model), _ptr(X), float(keep_fraction), _ptr(keep),
                                                       C.byref(nk)))
    return keep, int(nk.value)


def mgx_reduce_mesh(ctx, model, f, f_small, f_large, G_thres, seed):
    f = _arr(f, np.float64)
    n = len(f)
    Gf, L_, ell = np.empty(n), np.empty(n), np.empty(n)
    keep = np.empty(n, np.uint8)
    nk = C.c_int64(0)
    _check(ctx, load_library().mgx_reduce_mesh(ctx, int(model), _ptr(f), float(f_small), float(f_large),
                                               float(G_thres), C.c_uint64(int(seed) & (2**64 - 1)),
                                               _ptr(Gf), _ptr(L_), _ptr(ell), _ptr(keep), C.byref(nk)))
    return Gf, L_, ell, keep, int(nk.value)


def mgx_eval_approx(ctx, kind: int, x, y) -> float:
    """y = 2^x (kind 0), 1/x (kind 1) or atan2f(x[n:], x[:n]) (kind 2) by the
    approximate single-precision functions the certified decisions rest on;
    x, y float32 device tensors (x of y's size, twice it for kind 2).  Returns
    the error bound assumed for that function (relative; absolute for kind 2)."""
    b = C.c_float(0.0)
    _check(ctx, load_library().mgx_eval_approx(ctx, int(kind), _ptr(x), int(y.numel()), _ptr(y), C.byref(b)))
    return float(b.value)


def mgx_alu_peaks(ctx, reps: int = 3) -> dict:
    """Measured pipe throughputs: FP32 and FP64 FMA TFLOP/s, exp2 and rcp Gop/s."""
    out = np.zeros(4)
    _check(ctx, load_library().mgx_alu_peaks(ctx, int(reps), _ptr(out)))
    return {"fp32_fma_tflops": float(out[0]), "fp64_fma_tflops": float(out[1]), "ex2_gops": float(out[2]),
            "rcp_gops": float(out[3])}


def mgx_profile_enable(ctx, enable: bool = True) -> None:
    _check(ctx, load_library().mgx_profile_enable(ctx, int(bool(enable))))


def mgx_profile_read(ctx) -> dict:
    p = Profile()
    _check(ctx, load_library().mgx_profile_read(ctx, C.byref(p)))
    return dict(ms={k: p.ms[i] for i, k in enumerate(KERNEL_CLASSES)},
                launches={k: int(p.launches[i]) for i, k in enumerate(KERNEL_CLASSES)},
                trace_points=int(p.trace_points), solves=int(p.solves), updates=int(p.updates),
                samples=int(p.samples), trace_steps=int(p.trace_steps),
                trace_exact_steps=int(p.trace_exact_steps), decisions_redone=int(p.decisions_redone))


def solve_params(dtau_max=0.5, dv_max=1.0 / 3.0, I_bdy=0.0, precision=MGX_FP64, out_on_device=False, order=2):
    """order: 2 (second-order scheme) or 4 (Hermitian scheme, Section 2.1)."""
    return SolveParams(float(dtau_max), float(dv_max), float(I_bdy), int(precision), int(bool(out_on_device)),
                       int(order), 0)


# ------------------------------------------------------------ convenience class
class Context:
    """One library context bound to a CUDA device and a torch stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self.ptr = mgx_create(self.device, stream.cuda_stream)
        self.models: dict[int, dict] = {}

    def close(self):
        if self.ptr:
            mgx_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, m: dict, rays: bool = True, sample=None, l_min=None, l_max=None) -> int:
        """Load a model dict (see synth) and set its lines and ray set."""
        mid = mgx_load_mesh(self.ptr, m["pos"], m["vel"], m["nbr_off"], m["nbr_idx"])
        mgx_set_lines(self.ptr, mid, m["nu0"], m["chi0"], m["eta0"], m["dvw"], m["chi_c"], m["eta_c"],
                      m["n_freq"], m["x_span"])
        info = dict(n=len(m["pos"]), L=len(m["nu0"]), F=int(m["n_freq"]))
        self.models[mid] = info
        if rays:
            self.set_rays(mid, m["l_min"] if l_min is None else l_min, m["l_max"] if l_max is None else l_max,
                          m.get("sample") if sample is None else sample)
        return mid

    def set_rays(self, mid, l_min, l_max, sample=None):
        mgx_set_rays(self.ptr, mid, l_min, l_max, sample if l_min < l_max else None)
        self.models[mid]["npairs"] = mgx_rayset_npairs(l_min, l_max)

    def rays(self, mid) -> np.ndarray:
        i = self.models[mid]
        return mgx_get_rays(self.ptr, mid, i["n"], i["npairs"])

    def trace(self, mid, o_begin=0, o_end=None, with_delta=False, ids=True):
        i = self.models[mid]
        return mgx_trace(self.ptr, mid, o_begin, i["n"] if o_end is None else o_end, i["npairs"], with_delta, ids)

    def solve_J(self, mid, precision=MGX_FP64, dtau_max=0.5, dv_max=1.0 / 3.0, I_bdy=0.0, out=None, order=2):
        """J [n, L*F] float64; `out` may be a CUDA float64 tensor (device output)."""
        i = self.models[mid]
        if out is not None:
            p = solve_params(dtau_max, dv_max, I_bdy, precision, out_on_device=True, order=order)
            mgx_solve_J(self.ptr, mid, p, out)
            return out
        J = np.empty((i["n"], i["L"] * i["F"]), np.float64)
        mgx_solve_J(self.ptr, mid, solve_params(dtau_max, dv_max, I_bdy, precision, False, order), J)
        return J

    def solve_u(self, mid, o_begin, o_end, precision=MGX_FP64, dtau_max=0.5, dv_max=1.0 / 3.0, I_bdy=0.0,
                order=2):
        """u at the origin of every pair line of origins [o_begin, o_end): [n_o, pairs, L*F]."""
        i = self.models[mid]
        u = np.empty((o_end - o_begin, i["npairs"], i["L"] * i["F"]), np.float64)
        _check(self.ptr, load_library().mgx_solve_u(self.ptr, mid, C.byref(solve_params(
            dtau_max, dv_max, I_bdy, precision, False, order)), int(o_begin), int(o_end), _ptr(u)))
        return u

    def solve_J_batch(self, mids, precision=MGX_FP32, dtau_max=0.5, dv_max=1.0 / 3.0, I_bdy=0.0, outs=None,
                      flags=0, order=2):
        """J of several models in one persistent launch; returns CUDA float64 tensors."""
        import torch

        if outs is None:
            outs = [torch.empty((self.models[m]["n"], self.models[m]["L"] * self.models[m]["F"]),
                                dtype=torch.float64, device=f"cuda:{self.device}") for m in mids]
        mgx_solve_J_batch(self.ptr, list(mids), solve_params(dtau_max, dv_max, I_bdy, precision, True, order), outs,
                          flags)
        return outs

    def set_tuning(self, tuning: dict | None):
        mgx_set_tuning(self.ptr, tuning)

    def tuning(self) -> dict:
        return mgx_get_tuning(self.ptr)

    def autotune(self, mids, precision=MGX_FP32, dtau_max=0.5, dv_max=1.0 / 3.0, I_bdy=0.0, outs=None, flags=0,
                 reps=3, order=2):
        """Pick the batched solve's launch parameters for these models by timing; returns (trials, outs)."""
        import torch

        if outs is None:
            outs = [torch.empty((self.models[m]["n"], self.models[m]["L"] * self.models[m]["F"]),
                                dtype=torch.float64, device=f"cuda:{self.device}") for m in mids]
        trials = mgx_autotune(self.ptr, list(mids), solve_params(dtau_max, dv_max, I_bdy, precision, True, order), outs,
                              flags, reps)
        return trials, outs

    def reduce_mesh(self, mid, f, f_small, f_large, G_thres, seed):
        return mgx_reduce_mesh(self.ptr, mid, f, f_small, f_large, G_thres, seed)

    def profile(self, enable: bool = True):
        mgx_profile_enable(self.ptr, enable)

    def profile_read(self) -> dict:
        return mgx_profile_read(self.ptr)

    def free(self, mid):
        mgx_free_model(self.ptr, mid)
        self.models.pop(mid, None)
