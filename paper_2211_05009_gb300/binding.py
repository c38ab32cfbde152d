"""Thin ctypes binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every function below has the name of the C entry point it calls and does no arithmetic of the
method: all of it runs in the sm_103a kernels of ``liblbm.so``.  Buffers may be torch CUDA tensors
(passed by device pointer), torch CPU tensors or numpy arrays (passed by host pointer).  Errors
come back as :class:`LBMError` with the library's message.  There is no CPU fallback: if
``liblbm.so`` has not been built, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EDIVERGED, LBM_ETIMEOUT, LBM_ENOTREADY, LBM_EIO, LBM_ETOOBIG = range(9)
ERROR_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_EDIVERGED",
               5: "LBM_ETIMEOUT", 6: "LBM_ENOTREADY", 7: "LBM_EIO", 8: "LBM_ETOOBIG"}
LBM_STATIC_SCRATCH_DOUBLES = 1 << 19
DTYPES = {"f64": 0, "f32": 1, "f32s": 2, "f16s": 3, "bf16s": 4, "q16s": 5}
LBM_FLAG_LID_CORNERS_MOVING = 1
LBM_MAX_PROBES = 4
LBM_BATCH_SHAPES = 10
LBM_INIT_NEQ = 1
LBM_BATCH_MAX = 512
RESIDUAL_INTERVAL = 100


class LBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class lbm_info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("pitch", ctypes.c_long),
                ("tau", ctypes.c_double), ("nu", ctypes.c_double), ("U", ctypes.c_double),
                ("Re", ctypes.c_double), ("dtype", ctypes.c_int), ("flags", ctypes.c_uint),
                ("step", ctypes.c_long), ("device_bytes", ctypes.c_size_t), ("launch_config", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None

# (name, restype, argtypes)
_D, _I, _L, _P, _DP = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
_SIGS = [
    ("lbm_create", _I, [_I, _I, _D, _D, _I, ctypes.POINTER(_P)]),
    ("lbm_create_flags", _I, [_I, _I, _D, _D, _I, ctypes.c_uint, ctypes.POINTER(_P)]),
    ("lbm_create_ex", _I, [_I, _I, _D, _D, _I, ctypes.c_uint, ctypes.POINTER(_P)]),
    ("lbm_destroy", None, [_P]),
    ("lbm_last_error", ctypes.c_char_p, [_P]),
    ("lbm_set_stream", _I, [_P, _P]),
    ("lbm_set_allocator", _I, [ALLOC_FN, RELEASE_FN, _P]),
    ("lbm_get_info", _I, [_P, ctypes.POINTER(lbm_info)]),
    ("lbm_launch_config_count", _I, []),
    ("lbm_set_launch_config", _I, [_P, _I]),
    ("lbm_autotune", _I, [_P, _I, ctypes.POINTER(_I), _DP]),
    ("lbm_step", _I, [_P, _L]),
    ("lbm_run_to_residual", _I, [_P, _D, _L, ctypes.POINTER(_L)]),
    ("lbm_moments", _I, [_P, _P, _P, _P]),
    ("lbm_set_moments", _I, [_P, _P, _P, _P]),
    ("lbm_set_moments_ex", _I, [_P, _P, _P, _P, _I]),
    ("lbm_get_populations", _I, [_P, _P]),
    ("lbm_set_populations", _I, [_P, _P]),
    ("lbm_residual", _I, [_P, _DP]),
    ("lbm_mass", _I, [_P, _DP]),
    ("lbm_stream_function", _I, [_P, _P, _DP, _DP, _DP]),
    ("lbm_stream_function_window", _I, [_P, _I, _I, _I, _I, _DP, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                         _DP, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("lbm_probe", _I, [_P, _D, _D, _I, _P, _L]),
    ("lbm_probe_count", _I, [_P, _I, ctypes.POINTER(_L)]),
    ("lbm_probe_clear", _I, [_P]),
    ("lbm_stream_function_static", _I, [_P, _I, _I, _P, _P, _P]),
    ("lbm_batch_create", _I, [_I, _P, _P, _P, _P, _I, ctypes.POINTER(_P)]),
    ("lbm_batch_destroy", None, [_P]),
    ("lbm_batch_last_error", ctypes.c_char_p, [_P]),
    ("lbm_batch_set_stream", _I, [_P, _P]),
    ("lbm_batch_step", _I, [_P, _L]),
    ("lbm_batch_run_to_residual", _I, [_P, _D, _L, _P]),
    ("lbm_batch_residual", _I, [_P, _P, _P]),
    ("lbm_batch_cavity_steps", _I, [_P, _P]),
    ("lbm_batch_moments", _I, [_P, _I, _P, _P, _P]),
    ("lbm_batch_get_populations", _I, [_P, _I, _P]),
    ("lbm_batch_stream_function", _I, [_P, _I, _P, _DP, _DP, _DP]),
    ("lbm_batch_probe", _I, [_P, _P, _P, _I, _P, _L]),
    ("lbm_batch_set_moments", _I, [_P, _I, _P, _P, _P]),
    ("lbm_batch_set_moments_ex", _I, [_P, _I, _P, _P, _P, _I]),
    ("lbm_batch_info", _I, [_P, _I, ctypes.POINTER(lbm_info)]),
    ("lbm_batch_set_barrier_limit", _I, [_P, _D, _I]),
    ("lbm_batch_set_shape", _I, [_P, _I]),
    ("lbm_batch_autotune", _I, [_P, _I, _P, _P]),
    ("lbm_batch_launch_info", _I, [_P, _P, _P, _P, _P]),
    ("lbm_net_create", _I, [_I, ctypes.c_ulonglong, ctypes.POINTER(_P)]),
    ("lbm_net_destroy", None, [_P]),
    ("lbm_net_last_error", ctypes.c_char_p, [_P]),
    ("lbm_net_set_stream", _I, [_P, _P]),
    ("lbm_net_param_count", _L, [_P]),
    ("lbm_net_get_params", _I, [_P, _P]),
    ("lbm_net_set_params", _I, [_P, _P]),
    ("lbm_net_get_grads", _I, [_P, _P]),
    ("lbm_net_zero_grads", _I, [_P]),
    ("lbm_net_forward", _I, [_P, _P, _I, _I, _P]),
    ("lbm_net_backward", _I, [_P, _P, _P, _P, _P, _I, _I, _DP]),
    ("lbm_net_set_backend", _I, [_P, _I]),
    ("lbm_net_adam_step", _I, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    ("lbm_net_save", _I, [_P, ctypes.c_char_p]),
    ("lbm_net_load", _I, [_P, ctypes.c_char_p]),
    ("lbm_warm_input", _I, [_P, _P, _P, _I, _I, _D, _D, _D, _I, _I, _I, _P, _P]),
    ("lbm_warm_output", _I, [_P, _P, _I, _I, _I, _D, _P, _P, _P, _P]),
    ("lbm_warm_target", _I, [_P, _P, _P, _I, _I, _I, _D, _P, _P]),
    ("lbm_warm_smooth", _I, [_P, _I, _I, _I, _I, _P, _P]),
    ("lbm_nn_gemm_bf16", _I, [_I, _I, _I, _P, _I, _P, _I, _P, _I, _I, _I, _P]),
    ("lbm_nn_gemm_bf16_tc05", _I, [_I, _I, _I, _P, _I, _P, _I, _P, _I, _I, _I, _I, _P, _P]),
    ("lbm_fma_peak", _I, [_I, _I, _DP, _DP]),
    ("lbm_nn_conv3x3_bf16_tc05", _I, [_P, _I, _P, _I, _I, _I, _I, _P, _I, _P, _I, _I, _I, _P, _P]),
    ("lbm_nn_weights_tap_major", _I, [_P, _I, _I, _I, _P, _P]),
    ("lbm_nn_conv3x3_bf16_tma", _I, [_P, _I, _P, _I, _I, _I, _P, _I, _P, _I, _I, _I, _P, _P, _P]),
    ("lbm_save", _I, [_P, ctypes.c_char_p]),
    ("lbm_load", _I, [_P, ctypes.c_char_p]),
]
EXPORTED = [s[0] for s in _SIGS]


def library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblbm.so (built by ``paper_2211_05009_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first "
                               "(python -m paper_2211_05009_gb300.build); there is no CPU fallback")
        lib = ctypes.CDLL(path)
        for name, res, args in _SIGS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(buf) -> int | None:
    """Device or host address of a torch tensor / numpy array (contiguous), or None."""
    if buf is None:
        return None
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous or buf.dtype != np.float64:
            raise ValueError("numpy buffers must be C-contiguous float64")
        return buf.ctypes.data
    import torch
    if isinstance(buf, torch.Tensor):
        if not buf.is_contiguous() or buf.dtype != torch.float64:
            raise ValueError("torch buffers must be contiguous float64")
        return buf.data_ptr()
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _check(ctx, rc: int):
    if rc != LBM_OK:
        msg = library().lbm_last_error(ctx).decode(errors="replace")
        raise LBMError(rc, msg)


# ------------------------------------------------------------------ one wrapper per entry point
def lbm_create(nx: int, ny: int, Re: float, U_lid: float, dtype: str | int = "f32s"):
    out = ctypes.c_void_p()
    rc = library().lbm_create(nx, ny, Re, U_lid, DTYPES.get(dtype, dtype), ctypes.byref(out))
    _check(None, rc)
    return out.value


def lbm_create_flags(nx: int, ny: int, Re: float, U_lid: float, dtype: str | int = "f32s", flags: int = 0):
    out = ctypes.c_void_p()
    rc = library().lbm_create_flags(nx, ny, Re, U_lid, DTYPES.get(dtype, dtype), flags, ctypes.byref(out))
    _check(None, rc)
    return out.value


def lbm_create_ex(nx: int, ny: int, tau: float, U_lid: float, dtype: str | int = "f32s", flags: int = 0):
    out = ctypes.c_void_p()
    rc = library().lbm_create_ex(nx, ny, tau, U_lid, DTYPES.get(dtype, dtype), flags, ctypes.byref(out))
    _check(None, rc)
    return out.value


def lbm_destroy(ctx) -> None:
    library().lbm_destroy(ctx)


def lbm_last_error(ctx) -> str:
    return library().lbm_last_error(ctx).decode(errors="replace")


def lbm_set_stream(ctx, stream_handle: int | None) -> None:
    _check(ctx, library().lbm_set_stream(ctx, stream_handle))


def lbm_set_allocator(alloc, release, user=None) -> None:
    """alloc/release are ALLOC_FN/RELEASE_FN instances (keep them alive) or None for cudaMalloc."""
    a = alloc if alloc is not None else ctypes.cast(None, ALLOC_FN)
    r = release if release is not None else ctypes.cast(None, RELEASE_FN)
    _check(None, library().lbm_set_allocator(a, r, user))


def lbm_get_info(ctx) -> lbm_info:
    info = lbm_info()
    _check(ctx, library().lbm_get_info(ctx, ctypes.byref(info)))
    return info


def lbm_launch_config_count() -> int:
    return library().lbm_launch_config_count()


def lbm_set_launch_config(ctx, cfg: int) -> None:
    _check(ctx, library().lbm_set_launch_config(ctx, int(cfg)))


def lbm_autotune(ctx, steps_per_trial: int = 20) -> tuple[int, float]:
    best, glups = ctypes.c_int(), ctypes.c_double()
    _check(ctx, library().lbm_autotune(ctx, int(steps_per_trial), ctypes.byref(best), ctypes.byref(glups)))
    return best.value, glups.value


def lbm_step(ctx, n: int) -> None:
    _check(ctx, library().lbm_step(ctx, int(n)))


def lbm_run_to_residual(ctx, tol: float, max_steps: int) -> tuple[int, int]:
    """Returns (return code, steps taken): LBM_OK when converged, LBM_ENOTREADY when the step
    budget ran out; other codes raise."""
    done = ctypes.c_long(0)
    rc = library().lbm_run_to_residual(ctx, float(tol), int(max_steps), ctypes.byref(done))
    if rc not in (LBM_OK, LBM_ENOTREADY):
        _check(ctx, rc)
    return rc, done.value


def lbm_moments(ctx, rho=None, ux=None, uy=None) -> None:
    _check(ctx, library().lbm_moments(ctx, _ptr(rho), _ptr(ux), _ptr(uy)))


def lbm_set_moments(ctx, rho, ux, uy, flags: int = 0) -> None:
    _check(ctx, library().lbm_set_moments_ex(ctx, _ptr(rho), _ptr(ux), _ptr(uy), int(flags)))


def lbm_get_populations(ctx, f) -> None:
    _check(ctx, library().lbm_get_populations(ctx, _ptr(f)))


def lbm_set_populations(ctx, f) -> None:
    _check(ctx, library().lbm_set_populations(ctx, _ptr(f)))


def lbm_residual(ctx) -> float:
    r = ctypes.c_double()
    _check(ctx, library().lbm_residual(ctx, ctypes.byref(r)))
    return r.value


def lbm_mass(ctx) -> float:
    m = ctypes.c_double()
    _check(ctx, library().lbm_mass(ctx, ctypes.byref(m)))
    return m.value


def lbm_stream_function(ctx, psi=None) -> tuple[float, float, float]:
    vmin, xc, yc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, library().lbm_stream_function(ctx, _ptr(psi), ctypes.byref(vmin), ctypes.byref(xc), ctypes.byref(yc)))
    return vmin.value, xc.value, yc.value


def lbm_stream_function_window(ctx, i0: int, i1: int, j0: int, j1: int):
    vmin, vmax = ctypes.c_double(), ctypes.c_double()
    imin, jmin, imax, jmax = (ctypes.c_int() for _ in range(4))
    _check(ctx, library().lbm_stream_function_window(ctx, i0, i1, j0, j1, ctypes.byref(vmin), ctypes.byref(imin),
                                                     ctypes.byref(jmin), ctypes.byref(vmax), ctypes.byref(imax),
                                                     ctypes.byref(jmax)))
    return (vmin.value, imin.value, jmin.value), (vmax.value, imax.value, jmax.value)


def lbm_probe(ctx, x: float, y: float, every: int, dev_series, cap: int) -> int:
    q = library().lbm_probe(ctx, float(x), float(y), int(every), _ptr(dev_series), int(cap))
    if q < 0:
        _check(ctx, -q)
    return q


def lbm_probe_count(ctx, p: int) -> int:
    n = ctypes.c_long()
    _check(ctx, library().lbm_probe_count(ctx, p, ctypes.byref(n)))
    return n.value


def lbm_probe_clear(ctx) -> None:
    _check(ctx, library().lbm_probe_clear(ctx))


def lbm_stream_function_static(ux, nx: int, ny: int, psi, result, stream_handle=None) -> int:
    """Allocation-free stream function of a device u_x field (no context).  ux, psi and result are
    device buffers; returns the library's code (LBM_OK, LBM_EINVAL, LBM_ETOOBIG, LBM_ECUDA)."""
    return library().lbm_stream_function_static(_ptr(ux), int(nx), int(ny), _ptr(psi), _ptr(result),
                                                 stream_handle)


def lbm_save(ctx, path: str) -> None:
    _check(ctx, library().lbm_save(ctx, path.encode()))


def lbm_load(ctx, path: str) -> None:
    _check(ctx, library().lbm_load(ctx, path.encode()))


# ------------------------------------------------------------------ batched sweep
def _bcheck(b, rc: int):
    if rc != LBM_OK:
        raise LBMError(rc, library().lbm_batch_last_error(b).decode(errors="replace"))


def lbm_batch_create(nx, ny, Re, U, dtype: str | int = "f32s"):
    n = len(nx)
    a_nx = np.ascontiguousarray(nx, dtype=np.int32)
    a_ny = np.ascontiguousarray(ny, dtype=np.int32)
    a_re = np.ascontiguousarray(Re, dtype=np.float64)
    a_u = np.ascontiguousarray(U, dtype=np.float64)
    out = ctypes.c_void_p()
    rc = library().lbm_batch_create(n, a_nx.ctypes.data, a_ny.ctypes.data, a_re.ctypes.data, a_u.ctypes.data,
                                    DTYPES.get(dtype, dtype), ctypes.byref(out))
    _bcheck(None, rc)
    return out.value


def lbm_batch_destroy(b) -> None:
    library().lbm_batch_destroy(b)


def lbm_batch_last_error(b) -> str:
    return library().lbm_batch_last_error(b).decode(errors="replace")


def lbm_batch_set_stream(b, stream_handle) -> None:
    _bcheck(b, library().lbm_batch_set_stream(b, stream_handle))


def lbm_batch_step(b, n: int) -> None:
    _bcheck(b, library().lbm_batch_step(b, int(n)))


def lbm_batch_run_to_residual(b, n_cav: int, tol: float, max_steps: int):
    """(return code, steps per cavity); LBM_OK / LBM_ENOTREADY are returned, others raise."""
    done = np.zeros(n_cav, dtype=np.int64)
    rc = library().lbm_batch_run_to_residual(b, float(tol), int(max_steps), done.ctypes.data)
    if rc not in (LBM_OK, LBM_ENOTREADY):
        _bcheck(b, rc)
    return rc, done


def lbm_batch_residual(b, n_cav: int):
    r = np.zeros(n_cav)
    st = np.zeros(n_cav, dtype=np.int32)
    _bcheck(b, library().lbm_batch_residual(b, r.ctypes.data, st.ctypes.data))
    return r, st


def lbm_batch_cavity_steps(b, n_cav: int):
    s = np.zeros(n_cav, dtype=np.int64)
    _bcheck(b, library().lbm_batch_cavity_steps(b, s.ctypes.data))
    return s


def lbm_batch_moments(b, i: int, rho=None, ux=None, uy=None) -> None:
    _bcheck(b, library().lbm_batch_moments(b, i, _ptr(rho), _ptr(ux), _ptr(uy)))


def lbm_batch_get_populations(b, i: int, f) -> None:
    _bcheck(b, library().lbm_batch_get_populations(b, i, _ptr(f)))


def lbm_batch_stream_function(b, i: int, psi=None):
    vmin, xc, yc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _bcheck(b, library().lbm_batch_stream_function(b, i, _ptr(psi), ctypes.byref(vmin), ctypes.byref(xc), ctypes.byref(yc)))
    return vmin.value, xc.value, yc.value


def lbm_batch_set_moments(b, i: int, rho, ux, uy, flags: int = 0) -> None:
    _bcheck(b, library().lbm_batch_set_moments_ex(b, i, _ptr(rho), _ptr(ux), _ptr(uy), int(flags)))


def lbm_batch_probe(b, x, y, every: int, dev_series, cap: int) -> None:
    ax = np.ascontiguousarray(x, dtype=np.float64)
    ay = np.ascontiguousarray(y, dtype=np.float64)
    _bcheck(b, library().lbm_batch_probe(b, ax.ctypes.data, ay.ctypes.data, int(every), _ptr(dev_series), int(cap)))


def lbm_batch_info(b, i: int) -> lbm_info:
    info = lbm_info()
    _bcheck(b, library().lbm_batch_info(b, i, ctypes.byref(info)))
    return info


def lbm_batch_set_barrier_limit(b, seconds: float, absent_block: int = -1) -> None:
    _bcheck(b, library().lbm_batch_set_barrier_limit(b, float(seconds), int(absent_block)))


def lbm_batch_set_shape(b, shape: int) -> None:
    _bcheck(b, library().lbm_batch_set_shape(b, int(shape)))


def lbm_batch_autotune(b, steps: int = 50):
    """Returns (chosen shape, trial times in ms per shape)."""
    chosen = ctypes.c_int()
    ms = np.zeros(LBM_BATCH_SHAPES, dtype=np.float32)
    _bcheck(b, library().lbm_batch_autotune(b, int(steps), ctypes.byref(chosen), ms.ctypes.data))
    return chosen.value, ms


def lbm_batch_launch_info(b):
    """Returns (shape, rows per item, blocks, graph replays)."""
    sh, rows, blocks, gl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_long()
    _bcheck(b, library().lbm_batch_launch_info(b, ctypes.byref(sh), ctypes.byref(rows), ctypes.byref(blocks),
                                               ctypes.byref(gl)))
    return sh.value, rows.value, blocks.value, gl.value


# ------------------------------------------------------------------ learned warm start
LBM_WARM_RHO_SCALE = 100.0


def _tptr(t):
    """Device address of a torch tensor of any dtype (contiguous), or None."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return t.data_ptr()


def _ncheck(n, rc: int):
    if rc != LBM_OK:
        raise LBMError(rc, library().lbm_net_last_error(n).decode(errors="replace"))


def lbm_net_create(width: int, seed: int = 0):
    out = ctypes.c_void_p()
    _ncheck(None, library().lbm_net_create(int(width), int(seed), ctypes.byref(out)))
    return out.value


def lbm_net_destroy(n) -> None:
    library().lbm_net_destroy(n)


def lbm_net_set_stream(n, stream_handle) -> None:
    _ncheck(n, library().lbm_net_set_stream(n, stream_handle))


def lbm_net_param_count(n) -> int:
    return library().lbm_net_param_count(n)


def lbm_net_get_params(n, p) -> None:
    _ncheck(n, library().lbm_net_get_params(n, _tptr(p) if not isinstance(p, np.ndarray) else p.ctypes.data))


def lbm_net_set_params(n, p) -> None:
    _ncheck(n, library().lbm_net_set_params(n, _tptr(p) if not isinstance(p, np.ndarray) else p.ctypes.data))


def lbm_net_get_grads(n, g) -> None:
    _ncheck(n, library().lbm_net_get_grads(n, _tptr(g) if not isinstance(g, np.ndarray) else g.ctypes.data))


def lbm_net_zero_grads(n) -> None:
    _ncheck(n, library().lbm_net_zero_grads(n))


def lbm_net_forward(n, inp, H: int, W: int, out) -> None:
    _ncheck(n, library().lbm_net_forward(n, _tptr(inp), int(H), int(W), _tptr(out)))


def lbm_net_backward(n, inp, base, target, mask, H: int, W: int) -> float:
    loss = ctypes.c_double()
    _ncheck(n, library().lbm_net_backward(n, _tptr(inp), _tptr(base), _tptr(target), _tptr(mask), int(H), int(W),
                                          ctypes.byref(loss)))
    return loss.value


def lbm_net_set_backend(n, backend: int) -> None:
    _ncheck(n, library().lbm_net_set_backend(n, int(backend)))


def lbm_net_adam_step(n, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0) -> None:
    _ncheck(n, library().lbm_net_adam_step(n, lr, beta1, beta2, eps, grad_scale))


def lbm_net_save(n, path: str) -> None:
    _ncheck(n, library().lbm_net_save(n, path.encode()))


def lbm_net_load(n, path: str) -> None:
    _ncheck(n, library().lbm_net_load(n, path.encode()))


def lbm_warm_input(rho_c, ux_c, uy_c, nxc, nyc, Re, Ar, U, nx, ny, H, inp, stream_handle=None) -> None:
    rc = library().lbm_warm_input(_tptr(rho_c), _tptr(ux_c), _tptr(uy_c), nxc, nyc, float(Re), float(Ar), float(U),
                                  nx, ny, H, _tptr(inp), stream_handle)
    if rc != LBM_OK:
        raise LBMError(rc, "lbm_warm_input")


def lbm_warm_output(inp, out, nx, ny, H, U, rho, ux, uy, stream_handle=None) -> None:
    rc = library().lbm_warm_output(_tptr(inp), _tptr(out), nx, ny, H, float(U), _tptr(rho), _tptr(ux), _tptr(uy),
                                   stream_handle)
    if rc != LBM_OK:
        raise LBMError(rc, "lbm_warm_output")


def lbm_warm_smooth(out, ny, H, W, passes, scratch, stream_handle=None) -> None:
    rc = library().lbm_warm_smooth(_tptr(out), ny, H, W, int(passes), _tptr(scratch), stream_handle)
    if rc != LBM_OK:
        raise LBMError(rc, "lbm_warm_smooth")


def lbm_warm_target(rho, ux, uy, nx, ny, H, U, target, stream_handle=None) -> None:
    rc = library().lbm_warm_target(_tptr(rho), _tptr(ux), _tptr(uy), nx, ny, H, float(U), _tptr(target), stream_handle)
    if rc != LBM_OK:
        raise LBMError(rc, "lbm_warm_target")


def lbm_nn_gemm_bf16(M, N, K, A, lda, B, ldb, C, ldc, op=0, split_k=1, stream_handle=None) -> int:
    return library().lbm_nn_gemm_bf16(M, N, K, _tptr(A), lda, _tptr(B), ldb, _tptr(C), ldc, op, split_k, stream_handle)


def lbm_nn_conv3x3_bf16_tc05(x1, c1, x2, c2, H, W, K, Wt, N, C, ldc, op, err, trans_c=0, stream_handle=None) -> int:
    return library().lbm_nn_conv3x3_bf16_tc05(_tptr(x1), c1, _tptr(x2) if x2 is not None else None, c2, H, W, K,
                                              _tptr(Wt), N, _tptr(C), ldc, op, trans_c, _tptr(err), stream_handle)


def lbm_nn_weights_tap_major(Wt, ldk, C, N, Wtap, stream_handle=None) -> int:
    return library().lbm_nn_weights_tap_major(_tptr(Wt), ldk, C, N, _tptr(Wtap), stream_handle)


def lbm_nn_conv3x3_bf16_tma(x1, c1, x2, c2, H, W, Wtap, N, C, ldc, op, xs, err, trans_c=0, stream_handle=None) -> int:
    return library().lbm_nn_conv3x3_bf16_tma(_tptr(x1), c1, _tptr(x2) if x2 is not None else None, c2, H, W, _tptr(Wtap),
                                             N, _tptr(C), ldc, op, trans_c, _tptr(xs), _tptr(err), stream_handle)


def lbm_nn_gemm_bf16_tc05(M, N, K, A, lda, B, ldb, C, ldc, op, err, trans_c=0, split_k=1, stream_handle=None) -> int:
    return library().lbm_nn_gemm_bf16_tc05(M, N, K, _tptr(A), lda, _tptr(B), ldb, _tptr(C), ldc, op, trans_c, split_k,
                                           _tptr(err), stream_handle)


def lbm_fma_peak(fp64: bool = True, trips: int = 2000):
    """(FLOP/s, milliseconds of the timed launch) of the device's FMA pipe, FP64 or FP32."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    _check(None, library().lbm_fma_peak(1 if fp64 else 0, trips, ctypes.byref(rate), ctypes.byref(ms)))
    return rate.value, ms.value
