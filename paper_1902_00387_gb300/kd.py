"""Thin ctypes binding of libkd.so (include/kd.h).

Argument marshalling only: every step of the fine propagator, the coarse
propagator, the Parareal update and the norms runs in the library's CUDA kernels.
Functions keep the C names.  Device buffers are torch CUDA tensors; the host
buffers that kd_parareal_run / kd_fine_serial accept may be numpy arrays or CPU
tensors.  A missing library raises immediately: there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkd.so")

KD_OK, KD_EINVAL, KD_ENOMEM, KD_ECUDA, KD_ENOTCONV, KD_ETIMEOUT, KD_ENONFINITE, KD_EUNSUPPORTED = range(8)
STATUS_NAMES = ["KD_OK", "KD_EINVAL", "KD_ENOMEM", "KD_ECUDA", "KD_ENOTCONV", "KD_ETIMEOUT",
                "KD_ENONFINITE", "KD_EUNSUPPORTED"]
KD_FLOW_ROBERTS, KD_FLOW_GALLOWAY_PROCTOR, KD_FLOW_NONE = 0, 1, 2
KD_C64, KD_C128 = 0, 1
KD_COARSE_CLASSICAL, KD_COARSE_LEARNED = 0, 1
KD_FINE_DIRECT, KD_FINE_INCREMENT = 0, 1
KD_FINE_FFT, KD_FINE_CONV = 0, 1
KD_RK443, KD_RK222, KD_RK111 = 0, 1, 2
KD_SYNC_CLUSTER, KD_SYNC_P2P, KD_SYNC_PULL = 0, 1, 2
KD_GEMM_TCGEN05, KD_GEMM_MMA_SYNC = 0, 1
KD_TRAIN_ADAM, KD_TRAIN_MOMENTUM, KD_TRAIN_MINNORM = 0, 1, 2
KD_GRID_FINE, KD_GRID_COARSE = 0, 1
KD_MAX_SLICES = 1024
KD_MAX_ITERS = 256


class KdError(RuntimeError):
    def __init__(self, status, message):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s" % (name, message))
        self.status = status


class kd_params(ctypes.Structure):
    _fields_ = [("flow", ctypes.c_int), ("n", ctypes.c_int), ("kz", ctypes.c_double),
                ("Rm", ctypes.c_double), ("dt_fine", ctypes.c_double), ("prec_fine", ctypes.c_int),
                ("n_coarse", ctypes.c_int), ("dt_coarse", ctypes.c_double), ("prec_coarse", ctypes.c_int),
                ("coarse_kind", ctypes.c_int), ("learned_modes", ctypes.c_int), ("fine_form", ctypes.c_int),
                ("fine_operator", ctypes.c_int), ("fine_scheme", ctypes.c_int)]


class kd_parareal_stats(ctypes.Structure):
    _fields_ = [("k_con", ctypes.c_int), ("converged", ctypes.c_int), ("n_fine_steps", ctypes.c_int),
                ("n_coarse_steps", ctypes.c_int), ("dt_fine_used", ctypes.c_double),
                ("dt_coarse_used", ctypes.c_double), ("sigma", ctypes.c_double * KD_MAX_ITERS),
                ("energy", ctypes.c_double * (KD_MAX_SLICES + 1)), ("growth_rate", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_fine", ctypes.c_double), ("ms_coarse", ctypes.c_double),
                ("fallback_used", ctypes.c_int), ("n_launches", ctypes.c_longlong),
                ("true_err", ctypes.c_double * KD_MAX_ITERS)]


class kd_instance(ctypes.Structure):
    _fields_ = [("flow", ctypes.c_int), ("n", ctypes.c_int), ("kz", ctypes.c_double), ("Rm", ctypes.c_double),
                ("dt_fine", ctypes.c_double), ("n_coarse", ctypes.c_int), ("dt_coarse", ctypes.c_double)]


class kd_instance_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("k_con", ctypes.c_int), ("n_fine_steps", ctypes.c_int),
                ("n_coarse_steps", ctypes.c_int), ("dt_fine_used", ctypes.c_double),
                ("dt_coarse_used", ctypes.c_double), ("sigma", ctypes.c_double * KD_MAX_ITERS),
                ("growth_rate", ctypes.c_double)]


class kd_sweep_stats(ctypes.Structure):
    _fields_ = [("n_groups", ctypes.c_int), ("ms_total", ctypes.c_double), ("ms_fine", ctypes.c_double),
                ("ms_coarse", ctypes.c_double), ("n_launches", ctypes.c_longlong),
                ("fine_dof_steps", ctypes.c_double)]


_lib = None
EXPORTS = ["kd_create", "kd_destroy", "kd_fine_batched", "kd_fine_batched_host", "kd_fine_batched_kept",
           "kd_fine_batched_host_kept", "kd_coarse", "kd_parareal_run", "kd_fine_serial",
           "kd_energy", "kd_growth_rate", "kd_launch_count", "kd_profile", "kd_profile_read", "kd_last_error",
           "kd_version", "kd_fine_batched_static", "kd_learned_init", "kd_learned_pairs", "kd_learned_train",
           "kd_learned_eval", "kd_learned_loss_grad", "kd_learned_apply", "kd_plan_variants", "kd_set_plan",
           "kd_get_plan", "kd_autotune", "kd_sweep_run", "kd_set_dependent_launch", "kd_block_init",
           "kd_block_boundary_bytes", "kd_block_set_initial", "kd_block_set_boundary", "kd_block_get_boundary",
           "kd_block_fine", "kd_block_sweep", "kd_block_get_state", "kd_growth_power", "kd_growth_arnoldi", "kd_hessenberg_eig", "kd_gemm_bf16_tn",
           "kd_set_learned_gemm", "kd_learned_get", "kd_learned_set", "kd_selftest_wait", "kd_parareal_resume", "kd_set_graphs",
           "kd_set_reference", "kd_set_overlap", "kd_set_coarse_cluster",
           "kd_set_coarse_sync", "kd_sweep_create", "kd_sweep_exec", "kd_sweep_set_graphs", "kd_sweep_destroy",
           "kd_set_alloc_limit", "kd_get_alloc_bytes"]
KD_STATIC_SCRATCH_BYTES = 33554432


def load():
    """Load libkd.so once and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libkd.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "kd_create": (I, [ctypes.POINTER(kd_params), P, ctypes.POINTER(P)]),
        "kd_destroy": (I, [P]),
        "kd_fine_batched": (I, [P, P, P, P, I, I]),
        "kd_fine_batched_host": (I, [P, P, P, P, I, I, I]),
        "kd_fine_batched_kept": (I, [P, P, P, P, I, I]),
        "kd_fine_batched_host_kept": (I, [P, P, P, P, I, I, I]),
        "kd_coarse": (I, [P, P, P, P, I, I]),
        "kd_parareal_run": (I, [P, P, D, I, I, D, P, ctypes.POINTER(kd_parareal_stats)]),
        "kd_fine_serial": (I, [P, P, D, I, P]),
        "kd_energy": (I, [P, P, I, P]),
        "kd_growth_rate": (I, [P, P, I, D, D, ctypes.POINTER(D)]),
        "kd_fine_batched_static": (I, [ctypes.POINTER(kd_params), P, P, P, I, I, P]),
        "kd_learned_init": (I, [P, I, D]),
        "kd_learned_pairs": (I, [P, P, I, P, P]),
        "kd_learned_train": (I, [P, P, P, P, I, I, ctypes.c_float, ctypes.c_float, I, P]),
        "kd_learned_eval": (I, [P, P, P, P, I, P, P]),
        "kd_learned_loss_grad": (I, [P, P, P, ctypes.c_float, P, P, I, ctypes.POINTER(D), P]),
        "kd_learned_apply": (I, [P, P, P, I, I]),
        "kd_plan_variants": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "kd_set_plan": (I, [P, I, I, I]),
        "kd_set_dependent_launch": (I, [P, I]),
        "kd_set_overlap": (I, [P, I]),
        "kd_set_coarse_cluster": (I, [P, I]),
        "kd_set_coarse_sync": (I, [P, I]),
        "kd_get_plan": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "kd_autotune": (I, [P, I, I, I, ctypes.c_char_p, ctypes.POINTER(D)]),
        "kd_sweep_run": (I, [ctypes.POINTER(kd_instance), I, ctypes.POINTER(P), D, I, I, D, ctypes.c_char_p,
                             ctypes.POINTER(P), ctypes.POINTER(kd_instance_result), ctypes.POINTER(kd_sweep_stats),
                             P, ctypes.c_char_p]),
        "kd_sweep_create": (I, [ctypes.POINTER(kd_instance), I, D, I, P, ctypes.POINTER(P), ctypes.c_char_p]),
        "kd_sweep_exec": (I, [P, ctypes.POINTER(P), I, D, ctypes.c_char_p, ctypes.POINTER(P),
                              ctypes.POINTER(kd_instance_result), ctypes.POINTER(kd_sweep_stats), ctypes.c_char_p]),
        "kd_sweep_set_graphs": (I, [P, I]),
        "kd_sweep_destroy": (I, [P]),
        "kd_growth_power": (I, [P, P, D, D, I, D, ctypes.POINTER(D), ctypes.POINTER(I), P]),
        "kd_growth_arnoldi": (I, [P, P, D, D, I, I, I, D, P, P, ctypes.POINTER(I), P]),
        "kd_hessenberg_eig": (I, [I, P, P, P]),
        "kd_gemm_bf16_tn": (I, [P, P, P, I, I, I, I, I, P]),
        "kd_set_learned_gemm": (I, [P, I]),
        "kd_learned_get": (I, [P, I, P, ctypes.POINTER(I)]),
        "kd_learned_set": (I, [P, I, P, I]),
        "kd_selftest_wait": (I, [I, D, P]),
        "kd_set_graphs": (I, [P, I]),
        "kd_set_reference": (I, [P, P]),
        "kd_parareal_resume": (I, [P, P, I, D, I, I, D, P, ctypes.POINTER(kd_parareal_stats)]),
        "kd_block_init": (I, [P, I, I, D, I]),
        "kd_block_boundary_bytes": (ctypes.c_size_t, [P]),
        "kd_block_set_initial": (I, [P, P]),
        "kd_block_set_boundary": (I, [P, P]),
        "kd_block_get_boundary": (I, [P, P]),
        "kd_block_fine": (I, [P, I]),
        "kd_block_sweep": (I, [P, I, ctypes.POINTER(D)]),
        "kd_block_get_state": (I, [P, I, P]),
        "kd_launch_count": (ctypes.c_longlong, [P]),
        "kd_set_alloc_limit": (I, [P, ctypes.c_size_t]),
        "kd_get_alloc_bytes": (I, [P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
        "kd_profile": (I, [P, I]),
        "kd_profile_read": (I, [P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong)]),
        "kd_last_error": (ctypes.c_char_p, [P]),
        "kd_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def make_params(flow, n, kz, Rm, dt_fine, prec_fine=KD_C64, n_coarse=None, dt_coarse=None,
                prec_coarse=None, coarse_kind=KD_COARSE_CLASSICAL, fine_form=KD_FINE_DIRECT, learned_modes=0,
                fine_operator=KD_FINE_FFT, fine_scheme=KD_RK443):
    return kd_params(int(flow), int(n), float(kz), float(Rm), float(dt_fine), int(prec_fine),
                     int(n_coarse if n_coarse else max(16, n // 4 * 2)),   # even, about n / 2
                     float(dt_coarse if dt_coarse else dt_fine), int(prec_fine if prec_coarse is None else prec_coarse),
                     int(coarse_kind), int(learned_modes), int(fine_form), int(fine_operator), int(fine_scheme))


def _ptr(x, dtype=None, device=True):
    """Address of a contiguous buffer (torch tensor or numpy array)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if device:
            raise TypeError("a device (CUDA) buffer is required here")
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("buffer must be C-contiguous")
        if dtype is not None and x.dtype != np.dtype(dtype):
            raise TypeError("expected %s, got %s" % (dtype, x.dtype))
        return x.ctypes.data
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError("expected a torch tensor or numpy array")
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if device and not x.is_cuda:
        raise TypeError("a CUDA tensor is required here")
    if dtype is not None:
        want = {"complex64": torch.complex64, "complex128": torch.complex128, "float64": torch.float64}[dtype]
        if x.dtype != want:
            raise TypeError("expected %s, got %s" % (want, x.dtype))
    return x.data_ptr()


def _current_stream():
    import torch
    if torch.cuda.is_available() and torch.cuda.is_initialized():
        return torch.cuda.current_stream().cuda_stream
    return None


def _check(ctx, status, allow=()):
    if status != KD_OK and status not in allow:
        msg = load().kd_last_error(ctx) if ctx else b""
        raise KdError(status, (msg or b"").decode())
    return status


def kd_version():
    return load().kd_version().decode()


def kd_last_error(ctx):
    return load().kd_last_error(ctx).decode()


# Grid side of every live context (by address), for the buffer-size checks below: the
# library takes plain pointers and cannot tell how large a caller's buffer is.
_CTX_N = {}


def _addr(ctx):
    return ctx.value if isinstance(ctx, ctypes.c_void_p) else ctx


def _numel(x):
    return x.size if isinstance(x, np.ndarray) else x.numel()


def _need(ctx, x, fields, what, n=None):
    """Raise ValueError unless buffer x holds at least `fields` fields [3][n][n] of the
    context's grid (x may be None where the ABI allows NULL)."""
    if x is None:
        return
    n = n if n is not None else _CTX_N.get(_addr(ctx))
    if n is None:
        return
    want = int(fields) * 3 * n * n
    if _numel(x) < want:
        raise ValueError("%s holds %d elements; %d fields of 3 x %d x %d need %d" % (what, _numel(x), fields, n, n,
                                                                                  want))


def _need_count(x, count, what):
    if x is not None and _numel(x) < int(count):
        raise ValueError("%s holds %d elements, needs %d" % (what, _numel(x), int(count)))


def kd_create(params, stream=None):
    """Create a context; `stream` is a cudaStream_t address (default: torch's current stream)."""
    lib = load()
    out = ctypes.c_void_p()
    st = _current_stream() if stream is None else stream
    s = lib.kd_create(ctypes.byref(params), st, ctypes.byref(out))
    if s != KD_OK:
        raise KdError(s, "kd_create failed")
    _CTX_N[out.value] = int(params.n)
    return out


def kd_destroy(ctx):
    _CTX_N.pop(_addr(ctx), None)
    return _check(None, load().kd_destroy(ctx))


def _cdt(params_prec):
    return "complex128" if params_prec == KD_C128 else "complex64"


def kd_fine_batched(ctx, b_in, b_out, t0, nsteps, batch, prec=KD_C64):
    """F: advance `batch` fields [batch][3][n][n] by `nsteps` fine steps (device tensors)."""
    dt = _cdt(prec)
    _need(ctx, b_in, batch, "b_in")
    _need(ctx, b_out, batch, "b_out")
    _need_count(t0, batch, "t0")
    return _check(ctx, load().kd_fine_batched(ctx, _ptr(b_in, dt), _ptr(b_out, dt), _ptr(t0, "float64"),
                                              int(nsteps), int(batch)))


def _host_ptr(x, dtype):
    """Address of a contiguous HOST buffer (numpy array or CPU torch tensor)."""
    try:
        import torch
        if isinstance(x, torch.Tensor) and x.is_cuda:
            raise TypeError("a host (CPU) buffer is required here")
    except ImportError:
        pass
    return _ptr(x, dtype, device=False)


def kd_fine_batched_host(ctx, h_in, h_out, t0, nsteps, batch, chunk=0, prec=KD_C64):
    """F on fields in host memory (numpy arrays or CPU tensors, page-locked for overlap):
    the batch streams through the GPU in chunks of `chunk` fields (0: a graded plan from
    batch / 32 up to batch / 4 and back); t0 is a host float64 array.  Returns when h_out
    holds the result."""
    dt = _cdt(prec)
    _need(ctx, h_in, batch, "h_in")
    _need(ctx, h_out, batch, "h_out")
    _need_count(t0, batch, "t0")
    return _check(ctx, load().kd_fine_batched_host(ctx, _host_ptr(h_in, dt), _host_ptr(h_out, dt),
                                                   _host_ptr(t0, "float64"), int(nsteps), int(batch), int(chunk)))


def kept_side(n):
    """P = 2 floor(n / 3) + 1: the side of a field's kept-mode square (|kx|, |ky| <= n / 3)."""
    return 2 * (int(n) // 3) + 1


def _need_kept(ctx, x, fields, what):
    """Raise ValueError unless buffer x holds `fields` kept-mode fields [3][P][P]."""
    n = _CTX_N.get(_addr(ctx))
    if n is None:
        return
    P = kept_side(n)
    want = int(fields) * 3 * P * P
    if _numel(x) < want:
        raise ValueError("%s holds %d elements; %d kept-mode fields of 3 x %d x %d need %d" % (
            what, _numel(x), fields, P, P, want))


def kd_fine_batched_kept(ctx, c_in, c_out, t0, nsteps, batch, prec=KD_C64):
    """F on device fields in the kept-mode layout [batch][3][P][P] (P = kept_side(n); entry
    [c][iy][ix] is the coefficient of kx = ix - n // 3, ky = iy - n // 3); steps in place on
    c_out."""
    dt = _cdt(prec)
    _need_kept(ctx, c_in, batch, "c_in")
    _need_kept(ctx, c_out, batch, "c_out")
    _need_count(t0, batch, "t0")
    return _check(ctx, load().kd_fine_batched_kept(ctx, _ptr(c_in, dt), _ptr(c_out, dt), _ptr(t0, "float64"),
                                                   int(nsteps), int(batch)))


def kd_fine_batched_host_kept(ctx, h_in, h_out, t0, nsteps, batch, chunk=0, prec=KD_C64):
    """kd_fine_batched_host on host fields in the kept-mode layout [batch][3][P][P]."""
    dt = _cdt(prec)
    _need_kept(ctx, h_in, batch, "h_in")
    _need_kept(ctx, h_out, batch, "h_out")
    _need_count(t0, batch, "t0")
    return _check(ctx, load().kd_fine_batched_host_kept(ctx, _host_ptr(h_in, dt), _host_ptr(h_out, dt),
                                                        _host_ptr(t0, "float64"), int(nsteps), int(batch),
                                                        int(chunk)))


def kd_fine_batched_static(params, b_in, b_out, t0, nsteps, batch, stream=None):
    """Allocation-free fine propagator (workspace in the library's static device array)."""
    dt = _cdt(params.prec_fine)
    _need(None, b_in, batch, "b_in", n=params.n)
    _need(None, b_out, batch, "b_out", n=params.n)
    _need_count(t0, batch, "t0")
    st = _current_stream() if stream is None else stream
    s = load().kd_fine_batched_static(ctypes.byref(params), _ptr(b_in, dt), _ptr(b_out, dt), _ptr(t0, "float64"),
                                      int(nsteps), int(batch), st)
    if s != KD_OK:
        raise KdError(s, "kd_fine_batched_static failed (see stderr)")
    return s


def kd_coarse(ctx, b_in, b_out, t0, nsteps, batch):
    """G: restrict, coarse steps, prolong; complex128 device tensors [batch][3][n][n]."""
    _need(ctx, b_in, batch, "b_in")
    _need(ctx, b_out, batch, "b_out")
    _need_count(t0, batch, "t0")
    return _check(ctx, load().kd_coarse(ctx, _ptr(b_in, "complex128"), _ptr(b_out, "complex128"),
                                        _ptr(t0, "float64"), int(nsteps), int(batch)))


def _any_ptr(x, dtype):
    if isinstance(x, np.ndarray):
        return _ptr(x, dtype, device=False)
    return _ptr(x, dtype, device=False) if x is not None else None


def kd_parareal_run(ctx, b0, T, n_slices, k_max, tol, u_slices=None):
    """Parareal over [0, T]; b0 complex128 [3][n][n] and u_slices complex128
    [n_slices+1][3][n][n] may live on the host or the device.  Returns (status, stats)."""
    _need(ctx, b0, 1, "b0")
    _need(ctx, u_slices, n_slices + 1, "u_slices")
    st = kd_parareal_stats()
    s = load().kd_parareal_run(ctx, _any_ptr(b0, "complex128"), float(T), int(n_slices), int(k_max), float(tol),
                               _any_ptr(u_slices, "complex128"), ctypes.byref(st))
    _check(ctx, s, allow=(KD_ENOTCONV,))
    return s, st


def kd_parareal_resume(ctx, u_init, k_done, T, n_slices, k_max, tol, u_slices=None):
    """Continue Parareal from the iterate u_init (complex128 [n_slices+1][3][n][n]) of an
    earlier run after k_done iterations.  Returns (status, stats)."""
    _need(ctx, u_init, n_slices + 1, "u_init")
    _need(ctx, u_slices, n_slices + 1, "u_slices")
    st = kd_parareal_stats()
    s = load().kd_parareal_resume(ctx, _any_ptr(u_init, "complex128"), int(k_done), float(T), int(n_slices),
                                  int(k_max), float(tol), _any_ptr(u_slices, "complex128"), ctypes.byref(st))
    _check(ctx, s, allow=(KD_ENOTCONV,))
    return s, st


def kd_fine_serial(ctx, b0, T, n_slices, u_slices):
    """Serial fine solution at the slice boundaries (same step rule as kd_parareal_run)."""
    _need(ctx, b0, 1, "b0")
    _need(ctx, u_slices, n_slices + 1, "u_slices")
    return _check(ctx, load().kd_fine_serial(ctx, _any_ptr(b0, "complex128"), float(T), int(n_slices),
                                             _any_ptr(u_slices, "complex128")))


def kd_energy(ctx, fields, count, energy_out):
    _need(ctx, fields, count, "fields")
    _need_count(energy_out, count, "energy_out")
    return _check(ctx, load().kd_energy(ctx, _ptr(fields, "complex128"), int(count), _ptr(energy_out, "float64")))


def kd_growth_rate(ctx, u_slices, n_samples, T, fit_from):
    _need(ctx, u_slices, n_samples, "u_slices")
    rate = ctypes.c_double()
    _check(ctx, load().kd_growth_rate(ctx, _ptr(u_slices, "complex128"), int(n_samples), float(T),
                                      float(fit_from), ctypes.byref(rate)))
    return rate.value


def _phase_arr(phase):
    a = np.ascontiguousarray(np.asarray(phase, dtype=np.int32))
    return a, a.ctypes.data


def kd_learned_init(ctx, n_phase, slice_T):
    return _check(ctx, load().kd_learned_init(ctx, int(n_phase), float(slice_T)))


def kd_learned_pairs(ctx, x, n, phase, y):
    """y_i = R F(P x_i); x, y: complex64 CUDA tensors [n][3][m][m]; phase: ints."""
    ph, pp = _phase_arr(phase)
    return _check(ctx, load().kd_learned_pairs(ctx, _ptr(x, "complex64"), int(n), pp, _ptr(y, "complex64")))


def kd_learned_train(ctx, x, y, phase, n, epochs, lr, weight_decay, n_phase, method=KD_TRAIN_ADAM):
    """Train every phase operator; returns the data loss [n_phase][epochs]."""
    ph, pp = _phase_arr(phase)
    loss = np.zeros((n_phase, max(1, epochs)), np.float64)
    _check(ctx, load().kd_learned_train(ctx, _ptr(x, "complex64"), _ptr(y, "complex64"), pp, int(n), int(epochs),
                                        float(lr), float(weight_decay), int(method), loss.ctypes.data))
    return loss[:, :epochs]


def kd_learned_eval(ctx, x, y, phase, n, n_phase):
    """Per-phase relative errors (learned, classical) against the pairs."""
    ph, pp = _phase_arr(phase)
    el = np.zeros(n_phase, np.float64)
    ec = np.zeros(n_phase, np.float64)
    _check(ctx, load().kd_learned_eval(ctx, _ptr(x, "complex64"), _ptr(y, "complex64"), pp, int(n), el.ctypes.data,
                                       ec.ctypes.data))
    return el, ec


def kd_learned_loss_grad(ctx, W, W0, weight_decay, x, y, n, grad):
    loss = ctypes.c_double()
    _check(ctx, load().kd_learned_loss_grad(ctx, _ptr(W, None), _ptr(W0, None) if W0 is not None else None,
                                            float(weight_decay), _ptr(x, "complex64"), _ptr(y, "complex64"), int(n),
                                            ctypes.byref(loss), _ptr(grad, None)))
    return loss.value


def kd_learned_apply(ctx, x, y, phase, n):
    return _check(ctx, load().kd_learned_apply(ctx, _ptr(x, "complex64"), _ptr(y, "complex64"), int(phase), int(n)))


def kd_plan_variants(ctx, grid=KD_GRID_FINE):
    """(number of column variants, number of row variants) of a grid."""
    c, r = ctypes.c_int(), ctypes.c_int()
    _check(ctx, load().kd_plan_variants(ctx, int(grid), ctypes.byref(c), ctypes.byref(r)))
    return c.value, r.value


def kd_set_plan(ctx, grid, col, row):
    return _check(ctx, load().kd_set_plan(ctx, int(grid), int(col), int(row)))


def kd_set_coarse_cluster(ctx, blocks):
    return _check(ctx, load().kd_set_coarse_cluster(ctx, int(blocks)))


def kd_set_coarse_sync(ctx, mode):
    """KD_SYNC_CLUSTER (default), KD_SYNC_P2P or KD_SYNC_PULL halo exchange of the coarse solver."""
    return _check(ctx, load().kd_set_coarse_sync(ctx, int(mode)))


def kd_set_overlap(ctx, chunks):
    return _check(ctx, load().kd_set_overlap(ctx, int(chunks)))


def kd_set_dependent_launch(ctx, enable):
    return _check(ctx, load().kd_set_dependent_launch(ctx, int(bool(enable))))


def kd_get_plan(ctx, grid=KD_GRID_FINE):
    c, r = ctypes.c_int(), ctypes.c_int()
    _check(ctx, load().kd_get_plan(ctx, int(grid), ctypes.byref(c), ctypes.byref(r)))
    return c.value, r.value


def kd_autotune(ctx, grid, batch, nsteps=2, cache_path=None):
    """Autotune a grid's plan; returns the chosen plan's ms per step (-1 if read from the cache)."""
    ms = ctypes.c_double()
    path = cache_path.encode() if cache_path else None
    _check(ctx, load().kd_autotune(ctx, int(grid), int(batch), int(nsteps), path, ctypes.byref(ms)))
    return ms.value


def make_instance(flow, n, kz, Rm, dt_fine, n_coarse, dt_coarse):
    return kd_instance(int(flow), int(n), float(kz), float(Rm), float(dt_fine), int(n_coarse), float(dt_coarse))


def kd_sweep_run(instances, b0, T, n_slices, k_max, tol, u_final=None, tune_cache=None, stream=None):
    """Batched Parareal over independent instances.  b0 / u_final: lists of complex128
    [3][n_i][n_i] buffers (numpy arrays or tensors, host or device; u_final entries may be
    None).  Returns (status, results list, stats)."""
    lib = load()
    m = len(instances)
    arr = (kd_instance * m)(*instances)
    keep = list(b0) + [u for u in (u_final or []) if u is not None]
    b_ptrs = (ctypes.c_void_p * m)(*[_any_ptr(b, "complex128") for b in b0])
    u_ptrs = None
    if u_final is not None:
        u_ptrs = (ctypes.c_void_p * m)(*[_any_ptr(u, "complex128") if u is not None else None for u in u_final])
    res = (kd_instance_result * m)()
    st = kd_sweep_stats()
    err = ctypes.create_string_buffer(256)
    strm = _current_stream() if stream is None else stream
    s = lib.kd_sweep_run(arr, m, b_ptrs, float(T), int(n_slices), int(k_max), float(tol),
                         tune_cache.encode() if tune_cache else None, u_ptrs, res, ctypes.byref(st), strm, err)
    del keep
    if s not in (KD_OK, KD_ENOTCONV):
        raise KdError(s, err.value.decode())
    return s, list(res), st


class Sweep:
    """A prepared batched sweep (kd_sweep_create): groups, contexts and device buffers made
    once; exec() runs the Parareal iterations of every instance and may be repeated (the
    fine steps of recurring (iteration, active set) shapes replay captured CUDA graphs)."""

    def __init__(self, instances, T, n_slices, stream=None):
        lib = load()
        self.m = len(instances)
        self.instances = list(instances)
        arr = (kd_instance * self.m)(*instances)
        err = ctypes.create_string_buffer(256)
        h = ctypes.c_void_p()
        strm = _current_stream() if stream is None else stream
        s = lib.kd_sweep_create(arr, self.m, float(T), int(n_slices), strm, ctypes.byref(h), err)
        if s != KD_OK:
            raise KdError(s, err.value.decode())
        self.h = h

    def set_graphs(self, enable):
        load().kd_sweep_set_graphs(self.h, int(bool(enable)))

    def exec(self, b0, k_max, tol, u_final=None, tune_cache=None):
        """Returns (status, results list, stats), as kd_sweep_run."""
        lib = load()
        m = self.m
        if len(b0) != m or (u_final is not None and len(u_final) != m):
            raise ValueError("one initial field (and one output, if given) per instance")
        for i, (q, b) in enumerate(zip(self.instances, b0)):
            _need(None, b, 1, "b0[%d]" % i, n=q.n)
        keep = list(b0) + [u for u in (u_final or []) if u is not None]
        b_ptrs = (ctypes.c_void_p * m)(*[_any_ptr(b, "complex128") for b in b0])
        u_ptrs = None
        if u_final is not None:
            u_ptrs = (ctypes.c_void_p * m)(*[_any_ptr(u, "complex128") if u is not None else None for u in u_final])
        res = (kd_instance_result * m)()
        st = kd_sweep_stats()
        err = ctypes.create_string_buffer(256)
        s = lib.kd_sweep_exec(self.h, b_ptrs, int(k_max), float(tol), tune_cache.encode() if tune_cache else None,
                              u_ptrs, res, ctypes.byref(st), err)
        del keep
        if s not in (KD_OK, KD_ENOTCONV):
            raise KdError(s, err.value.decode())
        return s, list(res), st

    def close(self):
        if self.h:
            load().kd_sweep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kd_sweep_create(instances, T, n_slices, stream=None):
    """kd_sweep_create: a prepared sweep (a Sweep object)."""
    return Sweep(instances, T, n_slices, stream)


def kd_sweep_exec(sw, b0, k_max, tol, u_final=None, tune_cache=None):
    """kd_sweep_exec: returns (status, results list, stats)."""
    return sw.exec(b0, k_max, tol, u_final=u_final, tune_cache=tune_cache)


def kd_sweep_set_graphs(sw, enable):
    sw.set_graphs(enable)


def kd_sweep_destroy(sw):
    sw.close()


def kd_growth_power(ctx, b0, t0, tau, max_iter, tol, b_out=None):
    """Power-iteration growth rate; returns (status, rate, iterations)."""
    _need(ctx, b0, 1, "b0")
    _need(ctx, b_out, 1, "b_out")
    rate, its = ctypes.c_double(), ctypes.c_int()
    s = load().kd_growth_power(ctx, _any_ptr(b0, "complex128"), float(t0), float(tau), int(max_iter), float(tol),
                               ctypes.byref(rate), ctypes.byref(its), _any_ptr(b_out, "complex128"))
    _check(ctx, s, allow=(KD_ENOTCONV,))
    return s, rate.value, its.value


def kd_growth_arnoldi(ctx, b0, t0, tau, m, nev, restarts, tol, b_out=None):
    """Restarted Arnoldi on the fine propagator over [t0, t0 + tau]; returns (status,
    multipliers (complex numpy array [nev], by decreasing modulus), rates ln|mu| / tau,
    restarts used)."""
    _need(ctx, b0, 1, "b0")
    _need(ctx, b_out, 1, "b_out")
    mu = np.zeros(2 * int(nev), np.float64)
    rate = np.zeros(int(nev), np.float64)
    its = ctypes.c_int()
    s = load().kd_growth_arnoldi(ctx, _any_ptr(b0, "complex128"), float(t0), float(tau), int(m), int(nev),
                                 int(restarts), float(tol), mu.ctypes.data, rate.ctypes.data, ctypes.byref(its),
                                 _any_ptr(b_out, "complex128"))
    _check(ctx, s, allow=(KD_ENOTCONV,))
    return s, mu[0::2] + 1j * mu[1::2], rate, its.value


def kd_gemm_bf16_tn(A, Bt, C, engine=KD_GEMM_TCGEN05, stream=None):
    """C = A Bt^T for BF16 device tensors A [M][K], Bt [N][K] (K % 8 == 0) into the FP32
    device tensor C [M][>= N]; synchronous."""
    import torch
    if A.dtype != torch.bfloat16 or Bt.dtype != torch.bfloat16 or C.dtype != torch.float32:
        raise TypeError("A, Bt must be bfloat16 and C float32")
    M, K = A.shape
    N = Bt.shape[0]
    if Bt.shape[1] != K or C.shape[0] != M or C.shape[1] < N:
        raise ValueError("shape mismatch")
    st = _current_stream() if stream is None else stream
    s = load().kd_gemm_bf16_tn(_ptr(A), _ptr(Bt), _ptr(C), int(M), int(N), int(K), int(C.stride(0)), int(engine), st)
    if s != KD_OK:
        raise KdError(s, "kd_gemm_bf16_tn failed")


def kd_learned_get(ctx, phase, W):
    """Copy W_phase into W (bfloat16 [2 nc][nc], host numpy uint16 / torch tensor or
    device tensor); returns its usability flag."""
    valid = ctypes.c_int()
    _check(ctx, load().kd_learned_get(ctx, int(phase), _any_ptr_raw(W), ctypes.byref(valid)))
    return bool(valid.value)


def kd_learned_set(ctx, phase, W, valid):
    return _check(ctx, load().kd_learned_set(ctx, int(phase), _any_ptr_raw(W), int(bool(valid))))


def _any_ptr_raw(x):
    """Address of a contiguous host numpy array or torch tensor (host or device), any dtype."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("buffer must be C-contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr()


def kd_selftest_wait(arrive, max_ms=1.0):
    """Bounded-wait self-test; returns the status (KD_OK or KD_ETIMEOUT)."""
    return load().kd_selftest_wait(int(bool(arrive)), float(max_ms), _current_stream())


def kd_set_reference(ctx, b_ref):
    """Reference field at t = T (complex128 [3][n][n], host or device; None removes it)
    for stats.true_err of kd_parareal_run."""
    _need(ctx, b_ref, 1, "b_ref")
    return _check(ctx, load().kd_set_reference(ctx, _any_ptr(b_ref, "complex128") if b_ref is not None else None))


def kd_set_graphs(ctx, enable):
    return _check(ctx, load().kd_set_graphs(ctx, int(bool(enable))))


def kd_set_learned_gemm(ctx, engine):
    return _check(ctx, load().kd_set_learned_gemm(ctx, int(engine)))


def kd_hessenberg_eig(h, vectors=False):
    """Eigenvalues (and unit eigenvectors as columns) of a complex upper Hessenberg matrix
    by the library's host QR routine (no GPU)."""
    h = np.ascontiguousarray(h, dtype=np.complex128)
    m = h.shape[0]
    eig = np.zeros(m, np.complex128)
    vec = np.zeros((m, m), np.complex128) if vectors else None
    s = load().kd_hessenberg_eig(m, h.ctypes.data, eig.ctypes.data, vec.ctypes.data if vectors else None)
    if s != KD_OK:
        raise KdError(s, "kd_hessenberg_eig failed")
    return (eig, vec) if vectors else eig


def kd_block_init(ctx, lo, n_local, T, n_slices):
    return _check(ctx, load().kd_block_init(ctx, int(lo), int(n_local), float(T), int(n_slices)))


def kd_block_boundary_bytes(ctx):
    return int(load().kd_block_boundary_bytes(ctx))


def kd_block_set_initial(ctx, b0):
    return _check(ctx, load().kd_block_set_initial(ctx, _any_ptr(b0, "complex128")))


def _f64_ptr(x):
    if isinstance(x, np.ndarray):
        return _ptr(x, "float64", device=False)
    return _ptr(x, "float64", device=False)


def kd_block_set_boundary(ctx, u_lo):
    """u_lo: float64 buffer of kd_block_boundary_bytes(ctx) bytes (host or device)."""
    return _check(ctx, load().kd_block_set_boundary(ctx, _f64_ptr(u_lo)))


def kd_block_get_boundary(ctx, u_hi):
    return _check(ctx, load().kd_block_get_boundary(ctx, _f64_ptr(u_hi)))


def kd_block_fine(ctx, k):
    return _check(ctx, load().kd_block_fine(ctx, int(k)))


def kd_block_sweep(ctx, k):
    """Serial sweep of iteration k over the block; returns the defect (0 unless this
    block holds the last slice and k >= 1)."""
    sig = ctypes.c_double()
    _check(ctx, load().kd_block_sweep(ctx, int(k), ctypes.byref(sig)))
    return sig.value


def kd_block_get_state(ctx, i, u):
    return _check(ctx, load().kd_block_get_state(ctx, int(i), _any_ptr(u, "complex128")))


def kd_launch_count(ctx):
    return int(load().kd_launch_count(ctx))


def kd_set_alloc_limit(ctx, max_bytes):
    """Cap the device bytes the context may hold in its own buffers (0: no cap); a call
    that needs more raises KdError with status KD_ENOMEM."""
    if int(max_bytes) < 0:
        raise ValueError("max_bytes must be >= 0")
    return _check(ctx, load().kd_set_alloc_limit(ctx, int(max_bytes)))


def kd_get_alloc_bytes(ctx):
    """(bytes held, limit) of the context's own device buffers (limit 0: none)."""
    held, limit = ctypes.c_size_t(), ctypes.c_size_t()
    _check(ctx, load().kd_get_alloc_bytes(ctx, ctypes.byref(held), ctypes.byref(limit)))
    return int(held.value), int(limit.value)


def kd_profile(ctx, enable):
    return _check(ctx, load().kd_profile(ctx, int(bool(enable))))


def kd_profile_read(ctx):
    """(ms[2], launches[2]) of the fine column (0) and row (1) kernels since kd_profile(ctx, 1)."""
    ms = (ctypes.c_double * 2)()
    n = (ctypes.c_longlong * 2)()
    _check(ctx, load().kd_profile_read(ctx, ms, n))
    return [ms[0], ms[1]], [n[0], n[1]]


def stats_dict(st):
    k = st.k_con
    return {"k_con": k, "converged": bool(st.converged), "n_fine_steps": st.n_fine_steps,
            "n_coarse_steps": st.n_coarse_steps, "dt_fine_used": st.dt_fine_used,
            "dt_coarse_used": st.dt_coarse_used, "sigma": list(st.sigma[:k]), "growth_rate": st.growth_rate,
            "ms_total": st.ms_total, "ms_fine": st.ms_fine, "ms_coarse": st.ms_coarse,
            "n_launches": st.n_launches, "fallback_used": bool(st.fallback_used)}
