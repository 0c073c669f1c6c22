"""Thin ctypes binding of the C ABI in include/lbm.h.

Every ``lbm_*`` function here marshals its arguments and calls the function of
the same name in ``_lib/liblbm.so``; all computation happens in that library's
CUDA kernels.  A non-zero status raises :class:`LBMError`.  Importing this
module raises ImportError when the library has not been built: there is no
CPU fallback.

Array arguments may be NumPy arrays (host memory), torch tensors (host or
CUDA) or raw integer addresses.  :class:`Simulation` is a convenience wrapper
that lets PyTorch own the device memory (``lbm_bind_memory``) and supplies
torch's current CUDA stream (``lbm_set_stream``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_L = ctypes.CDLL(LIB_PATH)

# ---- constants (mirror include/lbm.h) -------------------------------------
from .abi import *  # noqa: E402,F401,F403
from .abi import MLP_NPARAM  # noqa: E402,F401

STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ESTATE", 3: "LBM_ENOMEM",
                4: "LBM_ECUDA", 5: "LBM_ENAN", 6: "LBM_ETIMEOUT", 7: "LBM_ENOCONV"}


class LBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_ll = ctypes.c_longlong
_sz = ctypes.c_size_t
_PROTOS = {
    "lbm_create": (_i, [_i, _i, _i, _i, _i, _d, _i, ctypes.POINTER(_vp)]),
    "lbm_multi_create": (_i, [_i, _i, _i, _i, _i, _d, _i, _i, ctypes.POINTER(_vp)]),
    "lbm_multi_destroy": (_i, [_vp]),
    "lbm_multi_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_multi_set_stream": (_i, [_vp, _vp]),
    "lbm_multi_set_overlap": (_i, [_vp, _i]),
    "lbm_multi_set_graph": (_i, [_vp, _i]),
    "lbm_multi_set_transfer": (_i, [_vp, _i]),
    "lbm_multi_set_force": (_i, [_vp, _d, _d, _d]),
    "lbm_multi_set_rounding": (_i, [_vp, _i]),
    "lbm_multi_set_smagorinsky": (_i, [_vp, _d]),
    "lbm_multi_set_elbm": (_i, [_vp, _i, _d, _i, _d]),
    "lbm_multi_set_boundary": (_i, [_vp, _i, _i, _i, _i, _vp]),
    "lbm_multi_set_geometry": (_i, [_vp, _vp]),
    "lbm_multi_init_equilibrium": (_i, [_vp, _vp, _vp, _i]),
    "lbm_multi_step": (_i, [_vp, _i]),
    "lbm_multi_get_macro": (_i, [_vp, _vp, _vp, _i]),
    "lbm_multi_halo_bytes": (_i, [_vp, ctypes.POINTER(_ll)]),
    "lbm_multi_create_rank": (_i, [_i, _i, _i, _i, _i, _d, _i, _i, _i, ctypes.POINTER(_vp)]),
    "lbm_multi_face_buffers": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                    ctypes.POINTER(_sz)]),
    "lbm_multi_step_begin": (_i, [_vp, _i]),
    "lbm_multi_step_end": (_i, [_vp]),
    "lbm_multi_exchange_stream": (_i, [_vp, ctypes.POINTER(_vp)]),
    "lbm_multi_rows": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "lbm_multi_launch_count": (_ll, [_vp]),
    "lbm_multi_sync": (_i, [_vp]),
    "lbm_destroy": (_i, [_vp]),
    "lbm_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_debug_fail_allocations": (_i, [_i]),
    "lbm_required_bytes": (_sz, [_vp]),
    "lbm_bind_memory": (_i, [_vp, _vp, _sz]),
    "lbm_set_stream": (_i, [_vp, _vp]),
    "lbm_set_access_pattern": (_i, [_vp, _i]),
    "lbm_set_geometry": (_i, [_vp, _vp]),
    "lbm_set_masked_kernel": (_i, [_vp, _i]),
    "lbm_get_nearwall_fraction": (_i, [_vp, ctypes.POINTER(_d)]),
    "lbm_set_force": (_i, [_vp, _d, _d, _d]),
    "lbm_set_mrt_rates": (_i, [_vp, _vp, _i]),
    "lbm_set_smagorinsky": (_i, [_vp, _d]),
    "lbm_set_boundary": (_i, [_vp, _i, _i, _i, _i, _vp]),
    "lbm_set_elbm": (_i, [_vp, _i, _d, _i, _d]),
    "lbm_set_elbm_guard": (_i, [_vp, _i, _d]),
    "lbm_set_elbm_feq": (_i, [_vp, _i]),
    "lbm_load_alpha_mlp": (_i, [_vp, _vp, _i]),
    "lbm_set_alpha_output": (_i, [_vp, _i]),
    "lbm_set_graph": (_i, [_vp, _i]),
    "lbm_set_rounding": (_i, [_vp, _i]),
    "lbm_init_equilibrium": (_i, [_vp, _vp, _vp, _i]),
    "lbm_step": (_i, [_vp, _i]),
    "lbm_get_time": (_i, [_vp, ctypes.POINTER(_ll)]),
    "lbm_get_macro": (_i, [_vp, _vp, _vp, _i]),
    "lbm_get_alpha": (_i, [_vp, _vp]),
    "lbm_reduce": (_i, [_vp, _vp]),
    "lbm_kinetic_energy_enstrophy": (_i, [_vp, _vp]),
    "lbm_get_elbm_stats": (_i, [_vp, _vp]),
    "lbm_set_elbm_diagnostics": (_i, [_vp, _i]),
    "lbm_get_elbm_entropy_error": (_i, [_vp, _vp]),
    "lbm_state_bytes": (_sz, [_vp]),
    "lbm_get_state": (_i, [_vp, _vp, ctypes.POINTER(_ll)]),
    "lbm_set_state": (_i, [_vp, _vp, _ll]),
    "lbm_sync": (_i, [_vp]),
    "lbm_launch_count": (_ll, [_vp]),
    "lbm_batch_create": (_i, [_i, _vp, _vp, _vp, _i, _i, ctypes.POINTER(_vp)]),
    "lbm_batch_destroy": (_i, [_vp]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_batch_set_stream": (_i, [_vp, _vp]),
    "lbm_batch_set_geometry": (_i, [_vp, _i, _vp]),
    "lbm_batch_set_force": (_i, [_vp, _i, _d, _d]),
    "lbm_batch_init_equilibrium": (_i, [_vp, _i, _vp, _vp, _i]),
    "lbm_batch_autotune": (_i, [_vp]),
    "lbm_batch_get_config": (_i, [_vp, _vp]),
    "lbm_batch_set_config": (_i, [_vp, _vp]),
    "lbm_batch_step": (_i, [_vp, _i]),
    "lbm_batch_get_macro": (_i, [_vp, _i, _vp, _vp, _i]),
    "lbm_batch_sync": (_i, [_vp]),
    "lbm_batch_set_wait_limit": (_i, [_vp, _ll]),
    "lbm_batch_set_rounding": (_i, [_vp, _i]),
    "lbm_batch_inject_missing_arrival": (_i, [_vp, _i]),
    "lbm_batch_launch_count": (_ll, [_vp]),
    "lbm_batch_nodes": (_sz, [_vp]),
    "lbm_elbm_collect_pairs": (_i, [_vp, _i, _vp, _vp, _i, ctypes.POINTER(_i)]),
    "lbm_mlp_train": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "lbm_mlp_grad": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "lbm_mlp_forward": (_i, [_vp, _i, _vp, _vp, _vp]),
    "lbm_mlp_last_error": (ctypes.c_char_p, []),
    "lbm_mlp_grad_static": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "lbm_mlp_grad_tc": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "lbm_mlp_train_cfg": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp, _vp]),
    "lbm_probe_fp64_rate": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(_d)]),
}
for _name, (_res, _args) in _PROTOS.items():
    _f = getattr(_L, _name)
    _f.restype = _res
    _f.argtypes = _args


def exported_symbols():
    """Names of the ABI functions this binding declares (all must resolve)."""
    return sorted(_PROTOS)


# ---- argument marshalling --------------------------------------------------
def _ptr(x):
    """Address of a NumPy array / torch tensor / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _check(code, handle=None, batch=False, mlp=False, multi=False):
    if code != LBM_OK:
        if mlp:
            msg = _L.lbm_mlp_last_error()
        elif multi:
            msg = _L.lbm_multi_last_error(handle)
        elif batch:
            msg = _L.lbm_batch_last_error(handle)
        else:
            msg = _L.lbm_last_error(handle)
        raise LBMError(code, (msg or b"").decode())


def _field_dtype(a):
    dt = getattr(a, "dtype", None)
    name = str(dt)
    if "float64" in name:
        return LBM_FIELD_F64
    if "float32" in name:
        return LBM_FIELD_F32
    raise TypeError(f"fields must be float32 or float64, got {dt}")


def _pair_dtype(rho, u):
    """The one element type of a (rho, u) pair (either may be None): the ABI
    takes a single field type for both arrays, so arrays of different types
    would have one of them written with the other's element size."""
    if rho is not None and u is not None:
        fd = _field_dtype(rho)
        if _field_dtype(u) != fd:
            raise TypeError("rho and u must share a dtype")
        return fd
    return _field_dtype(rho if rho is not None else u)


# ---- the ABI, name for name ------------------------------------------------
def lbm_create(nx, ny, nz, lattice, model, tau, dtype):
    h = _vp()
    _check(_L.lbm_create(nx, ny, nz, lattice, model, float(tau), dtype, ctypes.byref(h)), None)
    return h.value


def lbm_destroy(h):
    _check(_L.lbm_destroy(h), h)


def lbm_last_error(h):
    return (_L.lbm_last_error(h) or b"").decode()


def lbm_debug_fail_allocations(n):
    """Make the library's next n device allocations fail (testing)."""
    _check(_L.lbm_debug_fail_allocations(int(n)))


def lbm_required_bytes(h):
    return int(_L.lbm_required_bytes(h))


def lbm_bind_memory(h, dev, nbytes):
    _check(_L.lbm_bind_memory(h, _ptr(dev), nbytes), h)


def lbm_set_access_pattern(h, pattern):
    _check(_L.lbm_set_access_pattern(h, int(pattern)), h)


def lbm_set_stream(h, stream):
    _check(_L.lbm_set_stream(h, stream), h)


def lbm_set_geometry(h, mask):
    _check(_L.lbm_set_geometry(h, _ptr(mask)), h)


def lbm_set_masked_kernel(h, mode):
    _check(_L.lbm_set_masked_kernel(h, int(mode)), h)


def lbm_get_nearwall_fraction(h):
    out = _d(0.0)
    _check(_L.lbm_get_nearwall_fraction(h, ctypes.byref(out)), h)
    return float(out.value)


def lbm_set_force(h, fx, fy, fz=0.0):
    _check(_L.lbm_set_force(h, float(fx), float(fy), float(fz)), h)


def lbm_set_mrt_rates(h, s):
    s = np.ascontiguousarray(s, dtype=np.float64)
    _check(_L.lbm_set_mrt_rates(h, _ptr(s), int(s.size)), h)


def _bc_value(value):
    v = np.zeros(3)
    vals = np.atleast_1d(np.asarray(value, dtype=np.float64))
    v[:len(vals)] = vals
    return v


def lbm_set_boundary(h, cid, kind, method, normal, value):
    """Condition cid (mask code 2 + cid): value = velocity or [rho]."""
    v = _bc_value(value)
    _check(_L.lbm_set_boundary(h, int(cid), int(kind), int(method), int(normal), _ptr(v)), h)


def lbm_set_smagorinsky(h, cs):
    _check(_L.lbm_set_smagorinsky(h, float(cs)), h)


def lbm_set_elbm(h, alpha_mode, tol=1e-12, max_iter=20, skip_eps=1e-3):
    _check(_L.lbm_set_elbm(h, alpha_mode, float(tol), int(max_iter), float(skip_eps)), h)


def lbm_set_elbm_guard(h, guard_steps=2, guard_tol=1e-6):
    _check(_L.lbm_set_elbm_guard(h, int(guard_steps), float(guard_tol)), h)


def lbm_set_elbm_feq(h, variant):
    _check(_L.lbm_set_elbm_feq(h, int(variant)), h)


def lbm_load_alpha_mlp(h, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(_L.lbm_load_alpha_mlp(h, _ptr(p), int(p.size)), h)


def lbm_set_alpha_output(h, on):
    _check(_L.lbm_set_alpha_output(h, int(bool(on))), h)


def lbm_set_rounding(h, mode):
    _check(_L.lbm_set_rounding(h, int(mode)), h)


def lbm_set_graph(h, on):
    _check(_L.lbm_set_graph(h, int(bool(on))), h)


def lbm_init_equilibrium(h, rho, u):
    fd = _field_dtype(rho)
    if _field_dtype(u) != fd:
        raise TypeError("rho and u must share a dtype")
    _check(_L.lbm_init_equilibrium(h, _ptr(rho), _ptr(u), fd), h)


def lbm_step(h, n=1):
    _check(_L.lbm_step(h, int(n)), h)


def lbm_get_time(h):
    t = _ll()
    _check(_L.lbm_get_time(h, ctypes.byref(t)), h)
    return t.value


def lbm_get_macro(h, rho, u):
    """Fill rho / u (either may be None) with the last step's fields."""
    _check(_L.lbm_get_macro(h, _ptr(rho), _ptr(u), _pair_dtype(rho, u)), h)


def lbm_get_alpha(h, alpha):
    _check(_L.lbm_get_alpha(h, _ptr(alpha)), h)


def lbm_reduce(h, D):
    out = np.zeros(D + 2)
    _check(_L.lbm_reduce(h, _ptr(out)), h)
    return out


def lbm_kinetic_energy_enstrophy(h):
    """(E, Omega) of the last output step, FP64, computed on the GPU."""
    out = np.zeros(2)
    _check(_L.lbm_kinetic_energy_enstrophy(h, _ptr(out)), h)
    return float(out[0]), float(out[1])


def lbm_set_elbm_diagnostics(h, on):
    _check(_L.lbm_set_elbm_diagnostics(h, int(bool(on))), h)


def lbm_get_elbm_entropy_error(h):
    """(mean, max, samples) of |g(alpha)| / a_2 since diagnostics were set."""
    out = np.zeros(3)
    _check(_L.lbm_get_elbm_entropy_error(h, _ptr(out)), h)
    return float(out[0]), float(out[1]), int(out[2])


def lbm_get_elbm_stats(h):
    out = np.zeros(6)
    _check(_L.lbm_get_elbm_stats(h, _ptr(out)), h)
    return out


def lbm_state_bytes(h):
    return int(_L.lbm_state_bytes(h))


def lbm_get_state(h, dst):
    t = _ll()
    _check(_L.lbm_get_state(h, _ptr(dst), ctypes.byref(t)), h)
    return t.value


def lbm_set_state(h, src, t):
    _check(_L.lbm_set_state(h, _ptr(src), int(t)), h)


def lbm_sync(h):
    _check(_L.lbm_sync(h), h)


def lbm_launch_count(h):
    return int(_L.lbm_launch_count(h))


def lbm_elbm_collect_pairs(h, stride, X_dev, y_dev):
    cnt = _i()
    cap = int(y_dev.numel())
    _check(_L.lbm_elbm_collect_pairs(h, int(stride), _ptr(X_dev), _ptr(y_dev), cap,
                                     ctypes.byref(cnt)), h)
    return cnt.value


def lbm_mlp_train(X_dev, alpha_dev, n, cfg, params, loss_out, stream=None):
    c = np.ascontiguousarray(cfg, dtype=np.float64)
    _check(_L.lbm_mlp_train(_ptr(X_dev), _ptr(alpha_dev), int(n), _ptr(c), _ptr(params),
                            _ptr(loss_out), stream), mlp=True)


class MlpCfg(ctypes.Structure):
    """struct lbm_mlp_cfg."""
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("kernel", ctypes.c_int), ("reserved", ctypes.c_int)]


class TrainStats(ctypes.Structure):
    """struct lbm_train_stats."""
    _fields_ = [("steps", ctypes.c_int), ("reserved", ctypes.c_int), ("gpu_ms", ctypes.c_double),
                ("samples_per_s", ctypes.c_double), ("final_loss", ctypes.c_double)]


def lbm_mlp_train_cfg(X_dev, alpha_dev, n, epochs, batch, lr, seed, kernel, params, loss_out,
                      stream=None):
    """Training with the kernel choice (LBM_MLP_FP32 / LBM_MLP_BF16_TC);
    returns the stats as a dict."""
    cfg = MlpCfg(int(epochs), int(batch), float(lr), int(seed), int(kernel), 0)
    st = TrainStats()
    _check(_L.lbm_mlp_train_cfg(_ptr(X_dev), _ptr(alpha_dev), int(n), ctypes.byref(cfg),
                                _ptr(params), _ptr(loss_out), ctypes.byref(st), stream), mlp=True)
    return {"steps": st.steps, "gpu_ms": st.gpu_ms, "samples_per_s": st.samples_per_s,
            "final_loss": st.final_loss}


def lbm_mlp_grad(X_dev, t_dev, n, params, stream=None):
    p = np.ascontiguousarray(params, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    grad = np.zeros(MLP_NPARAM, dtype=np.float32)
    _check(_L.lbm_mlp_grad(_ptr(X_dev), _ptr(t_dev), int(n), _ptr(p), _ptr(loss), _ptr(grad),
                           stream), mlp=True)
    return float(loss[0]), grad


def lbm_mlp_grad_tc(X_dev, t_dev, n, params, stream=None):
    """lbm_mlp_grad on the BF16 tensor-core kernel (weights rounded to BF16)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    grad = np.zeros(MLP_NPARAM, dtype=np.float32)
    _check(_L.lbm_mlp_grad_tc(_ptr(X_dev), _ptr(t_dev), int(n), _ptr(p), _ptr(loss), _ptr(grad),
                              stream), mlp=True)
    return float(loss[0]), grad


def lbm_mlp_grad_static(X_dev, t_dev, n, params, stream=None):
    """lbm_mlp_grad without allocation (static device scratch, n <= 4096)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    grad = np.zeros(MLP_NPARAM, dtype=np.float32)
    _check(_L.lbm_mlp_grad_static(_ptr(X_dev), _ptr(t_dev), int(n), _ptr(p), _ptr(loss),
                                  _ptr(grad), stream), mlp=True)
    return float(loss[0]), grad


def lbm_probe_fp64_rate(stream=None):
    """(FP64 warp instructions per second, FP64 FLOP/s) of the current GPU."""
    w, f = _d(0.0), _d(0.0)
    code = _L.lbm_probe_fp64_rate(stream, ctypes.byref(w), ctypes.byref(f))
    if code:
        raise LBMError(code, "FP64 rate probe failed")
    return float(w.value), float(f.value)


def lbm_mlp_last_error():
    return (_L.lbm_mlp_last_error() or b"").decode()


def lbm_mlp_forward(X_dev, n, params, alpha_dev, stream=None):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(_L.lbm_mlp_forward(_ptr(X_dev), int(n), _ptr(p), _ptr(alpha_dev), stream), mlp=True)


# ---- batch ABI --------------------------------------------------------------
def lbm_batch_create(nx, ny, tau, dtype, lattice=LBM_D2Q9):
    nx = np.ascontiguousarray(nx, dtype=np.int32)
    ny = np.ascontiguousarray(ny, dtype=np.int32)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    b = _vp()
    code = _L.lbm_batch_create(int(nx.size), _ptr(nx), _ptr(ny), _ptr(tau), int(lattice), dtype,
                               ctypes.byref(b))
    _check(code, None, batch=True)
    return b.value


def lbm_batch_destroy(b):
    _check(_L.lbm_batch_destroy(b), b, batch=True)


def lbm_batch_set_stream(b, stream):
    _check(_L.lbm_batch_set_stream(b, stream), b, batch=True)


def lbm_batch_set_geometry(b, d, mask):
    _check(_L.lbm_batch_set_geometry(b, int(d), _ptr(mask)), b, batch=True)


def lbm_batch_set_force(b, d, fx, fy):
    _check(_L.lbm_batch_set_force(b, int(d), float(fx), float(fy)), b, batch=True)


def lbm_batch_init_equilibrium(b, d, rho, u):
    _check(_L.lbm_batch_init_equilibrium(b, int(d), _ptr(rho), _ptr(u), _pair_dtype(rho, u)), b,
           batch=True)


def lbm_batch_autotune(b):
    _check(_L.lbm_batch_autotune(b), b, batch=True)


def lbm_batch_get_config(b):
    out = np.zeros(5, dtype=np.int32)
    _check(_L.lbm_batch_get_config(b, _ptr(out)), b, batch=True)
    return out


def lbm_batch_set_config(b, cfg):
    """cfg: (threads, ctas, tile width, tile rows, rows per thread and pass)."""
    arr = np.ascontiguousarray(np.asarray(cfg, dtype=np.int32).reshape(5))
    _check(_L.lbm_batch_set_config(b, _ptr(arr)), b, batch=True)


def lbm_batch_step(b, n=1):
    _check(_L.lbm_batch_step(b, int(n)), b, batch=True)


def lbm_batch_get_macro(b, d, rho, u):
    _check(_L.lbm_batch_get_macro(b, int(d), _ptr(rho), _ptr(u), _pair_dtype(rho, u)), b,
           batch=True)


def lbm_batch_set_rounding(b, mode):
    _check(_L.lbm_batch_set_rounding(b, int(mode)), b, batch=True)


def lbm_batch_set_wait_limit(b, spins):
    _check(_L.lbm_batch_set_wait_limit(b, int(spins)), b, batch=True)


def lbm_batch_inject_missing_arrival(b, on):
    _check(_L.lbm_batch_inject_missing_arrival(b, int(on)), b, batch=True)


def lbm_batch_sync(b):
    _check(_L.lbm_batch_sync(b), b, batch=True)


def lbm_batch_launch_count(b):
    return int(_L.lbm_batch_launch_count(b))


def lbm_batch_nodes(b):
    return int(_L.lbm_batch_nodes(b))


# ---- subdomain decomposition (ghost layers, one GPU) ----------------------------
def _mcheck(code, m):
    _check(code, m, multi=True)


def lbm_multi_create(nx, ny, nz, lattice, model, tau, dtype, nsub):
    m = _vp()
    _mcheck(_L.lbm_multi_create(int(nx), int(ny), int(nz), int(lattice), int(model), float(tau),
                                int(dtype), int(nsub), ctypes.byref(m)), None)
    return m.value


def lbm_multi_destroy(m):
    _mcheck(_L.lbm_multi_destroy(m), m)


def lbm_multi_set_stream(m, stream):
    _mcheck(_L.lbm_multi_set_stream(m, _ptr(stream)), m)


def lbm_multi_set_overlap(m, on):
    _mcheck(_L.lbm_multi_set_overlap(m, int(bool(on))), m)


def lbm_multi_set_transfer(m, mode):
    _mcheck(_L.lbm_multi_set_transfer(m, int(mode)), m)


def lbm_multi_set_graph(m, on):
    _mcheck(_L.lbm_multi_set_graph(m, int(bool(on))), m)


def lbm_multi_set_force(m, fx, fy, fz=0.0):
    _mcheck(_L.lbm_multi_set_force(m, float(fx), float(fy), float(fz)), m)


def lbm_multi_set_rounding(m, mode):
    _mcheck(_L.lbm_multi_set_rounding(m, int(mode)), m)


def lbm_multi_set_smagorinsky(m, cs):
    _mcheck(_L.lbm_multi_set_smagorinsky(m, float(cs)), m)


def lbm_multi_set_boundary(m, cid, kind, method, normal, value):
    v = _bc_value(value)
    _mcheck(_L.lbm_multi_set_boundary(m, int(cid), int(kind), int(method), int(normal),
                                      _ptr(v)), m)


def lbm_multi_set_elbm(m, alpha_mode, tol=1e-12, max_iter=20, skip_eps=1e-3):
    _mcheck(_L.lbm_multi_set_elbm(m, int(alpha_mode), float(tol), int(max_iter),
                                  float(skip_eps)), m)


def lbm_multi_set_geometry(m, mask):
    if isinstance(mask, np.ndarray):
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
    _mcheck(_L.lbm_multi_set_geometry(m, _ptr(mask)), m)


def lbm_multi_init_equilibrium(m, rho, u):
    fd = _field_dtype(rho)
    if _field_dtype(u) != fd:
        raise TypeError("rho and u must share a dtype")
    _mcheck(_L.lbm_multi_init_equilibrium(m, _ptr(rho), _ptr(u), fd), m)


def lbm_multi_step(m, n=1):
    _mcheck(_L.lbm_multi_step(m, int(n)), m)


def lbm_multi_get_macro(m, rho, u):
    _mcheck(_L.lbm_multi_get_macro(m, _ptr(rho), _ptr(u), _pair_dtype(rho, u)), m)


def lbm_multi_halo_bytes(m):
    v = _ll(0)
    _mcheck(_L.lbm_multi_halo_bytes(m, ctypes.byref(v)), m)
    return int(v.value)


def lbm_multi_create_rank(nx, ny, nz, lattice, model, tau, dtype, nsub, rank):
    m = _vp()
    _mcheck(_L.lbm_multi_create_rank(int(nx), int(ny), int(nz), int(lattice), int(model),
                                     float(tau), int(dtype), int(nsub), int(rank),
                                     ctypes.byref(m)), None)
    return m.value


def lbm_multi_face_buffers(m):
    """(send address, recv address, bytes per face) of a rank handle."""
    s, r, nb = _vp(), _vp(), _sz(0)
    _mcheck(_L.lbm_multi_face_buffers(m, ctypes.byref(s), ctypes.byref(r), ctypes.byref(nb)), m)
    return int(s.value), int(r.value), int(nb.value)


def lbm_multi_step_begin(m, output=False):
    _mcheck(_L.lbm_multi_step_begin(m, 1 if output else 0), m)


def lbm_multi_step_end(m):
    _mcheck(_L.lbm_multi_step_end(m), m)


def lbm_multi_exchange_stream(m):
    s = _vp()
    _mcheck(_L.lbm_multi_exchange_stream(m, ctypes.byref(s)), m)
    return int(s.value or 0)


def lbm_multi_rows(m):
    lo, hi = _i(0), _i(0)
    _mcheck(_L.lbm_multi_rows(m, ctypes.byref(lo), ctypes.byref(hi)), m)
    return int(lo.value), int(hi.value)


def lbm_multi_launch_count(m):
    return int(_L.lbm_multi_launch_count(m))


def lbm_multi_sync(m):
    _mcheck(_L.lbm_multi_sync(m), m)


# ---- convenience wrapper ------------------------------------------------------
class Simulation:
    """One lattice on the current CUDA device, memory owned by a torch tensor.

    >>> sim = Simulation(256, 256, 256, LBM_D3Q19, LBM_BGK, 0.6, LBM_F32S)
    >>> sim.init(rho, u); sim.step(100); rho, u = sim.macro()
    """

    def __init__(self, nx, ny, nz, lattice, model, tau, dtype, stream=None, torch_memory=True,
                 pattern=LBM_PATTERN_AB):
        import torch
        self.nx, self.ny, self.nz = nx, ny, nz
        self.lattice, self.model, self.dtype = lattice, model, dtype
        self.D = 2 if lattice == LBM_D2Q9 else 3
        self.h = lbm_create(nx, ny, nz, lattice, model, tau, dtype)
        if pattern != LBM_PATTERN_AB:
            lbm_set_access_pattern(self.h, pattern)
        self._mem = None
        if torch_memory:
            nb = lbm_required_bytes(self.h)
            self._mem = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
            addr = self._mem.data_ptr()
            lbm_bind_memory(self.h, (addr + 255) // 256 * 256, nb)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        lbm_set_stream(self.h, s)

    def close(self):
        if self.h:
            lbm_destroy(self.h)
            self.h = None
            self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, mask):
        lbm_set_geometry(self.h, np.ascontiguousarray(mask, dtype=np.uint8)
                         if isinstance(mask, np.ndarray) else mask)

    def set_force(self, fx, fy, fz=0.0):
        lbm_set_force(self.h, fx, fy, fz)

    def init(self, rho, u):
        if isinstance(rho, np.ndarray):
            rho = np.ascontiguousarray(rho)
            u = np.ascontiguousarray(u, dtype=rho.dtype)
        lbm_init_equilibrium(self.h, rho, u)

    def step(self, n=1):
        lbm_step(self.h, n)

    def macro(self, dtype=np.float64):
        rho = np.empty((self.nz, self.ny, self.nx), dtype=dtype)
        u = np.empty((self.D, self.nz, self.ny, self.nx), dtype=dtype)
        lbm_get_macro(self.h, rho, u)
        return rho, u

    def reduce(self):
        return lbm_reduce(self.h, self.D)

    def state(self):
        buf = np.empty(lbm_state_bytes(self.h), dtype=np.uint8)
        t = lbm_get_state(self.h, buf)
        return buf, t

    def set_state(self, buf, t):
        lbm_set_state(self.h, buf, t)
