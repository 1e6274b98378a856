"""Thin ctypes binding of libhelm (include/helm.h): argument marshalling only.

Every array argument may be a torch tensor (CUDA or CPU) or a numpy array;
the binding passes its data pointer and sizes, and libhelm does all the
work on the GPU.  The shared library is built in-tree by
``paper_2405_17696_gb300.build``; importing this module fails loudly if it
is missing - there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhelm.so")

HELM_OK, HELM_EINVAL, HELM_ENOMEM, HELM_ECUDA, HELM_ENOCONV, HELM_EBREAKDOWN, HELM_ETIMEOUT, \
    HELM_EUNSUPPORTED = range(8)
HELM_PC_NONE, HELM_PC_MG, HELM_PC_CNN = 0, 1, 2
HELM_COARSE_GMRES, HELM_COARSE_JACOBI = 0, 1
HELM_OP_H, HELM_OP_SL = 0, 1
HELM_SOLVE_ADJOINT, HELM_SOLVE_ZERO_X0 = 1, 2

STATUS_NAMES = {0: "HELM_OK", 1: "HELM_EINVAL", 2: "HELM_ENOMEM", 3: "HELM_ECUDA", 4: "HELM_ENOCONV",
                5: "HELM_EBREAKDOWN", 6: "HELM_ETIMEOUT", 7: "HELM_EUNSUPPORTED"}


class HelmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class helm_opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_iter", ctypes.c_int), ("mg_levels", ctypes.c_int),
                ("pre", ctypes.c_int), ("post", ctypes.c_int), ("jacobi_w", ctypes.c_float),
                ("sl_beta", ctypes.c_float), ("sl_include_gamma", ctypes.c_int), ("coarse_kind", ctypes.c_int),
                ("coarse_iters", ctypes.c_int), ("precond", ctypes.c_int), ("max_rhs", ctypes.c_int),
                ("cnn_vcycle", ctypes.c_int), ("autotune", ctypes.c_int), ("stream", ctypes.c_void_p)]


class fwi_survey_t(ctypes.Structure):
    _fields_ = [("src_idx", ctypes.c_void_p), ("nsrc", ctypes.c_int), ("src_w", ctypes.c_void_p),
                ("nsim", ctypes.c_int), ("rcv_idx", ctypes.c_void_p), ("nrcv", ctypes.c_int)]


class fwi_gn_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("tol_sens", ctypes.c_double), ("cg_iters", ctypes.c_int),
                ("reg", ctypes.c_float), ("m_min", ctypes.c_float), ("m_max", ctypes.c_float),
                ("max_backtracks", ctypes.c_int), ("reg_kind", ctypes.c_int), ("alpha", ctypes.c_float),
                ("m_ref", ctypes.c_void_p)]


class fwi_gn_info(ctypes.Structure):
    _fields_ = [("misfit_before", ctypes.c_double), ("misfit_after", ctypes.c_double), ("step", ctypes.c_double),
                ("cg_iters", ctypes.c_int), ("iters_forward", ctypes.c_longlong),
                ("iters_adjoint", ctypes.c_longlong), ("iters_sensitivity", ctypes.c_longlong),
                ("iters_line_search", ctypes.c_longlong), ("objective_before", ctypes.c_double),
                ("objective_after", ctypes.c_double)]


class cnn_retrain_opts(ctypes.Structure):
    _fields_ = [("initial_size", ctypes.c_int), ("data_epochs", ctypes.c_int), ("epochs", ctypes.c_int),
                ("max_gmres_steps", ctypes.c_int), ("literal", ctypes.c_int), ("seed", ctypes.c_ulonglong)]


class helm_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.POINTER(ctypes.c_int)), ("rel_res", ctypes.POINTER(ctypes.c_double)),
                ("status", ctypes.POINTER(ctypes.c_int))]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhelm.so is not built ({LIB_PATH}); run paper_2405_17696_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip, fp = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    lib.helm_default_opts.argtypes = [ctypes.POINTER(helm_opts)]
    lib.helm_default_opts.restype = None
    lib.helm_setup.argtypes = [ctypes.POINTER(vp), vp, vp, ip, ip, fp, fp, vp, ip, vp, ctypes.POINTER(helm_opts)]
    lib.helm_setup.restype = ip
    lib.helm_set_medium.argtypes = [vp, vp, vp, vp, ip]
    lib.helm_set_medium.restype = ip
    lib.helm_solve.argtypes = [vp, vp, vp, ip, vp, ctypes.c_double, ip, ctypes.POINTER(helm_stats)]
    lib.helm_solve.restype = ip
    lib.helm_residual.argtypes = [vp, vp, vp, vp, ip, vp, ctypes.POINTER(ctypes.c_double)]
    lib.helm_residual.restype = ip
    lib.helm_residual_noalloc.argtypes = [vp, vp, ip, ip, fp, fp, vp, vp, vp, vp, vp, ip, vp]
    lib.helm_residual_noalloc.restype = ip
    lib.helm_apply.argtypes = [vp, vp, vp, ip, vp, ip]
    lib.helm_apply.restype = ip
    lib.helm_vcycle.argtypes = [vp, vp, vp, vp, ip, vp]
    lib.helm_vcycle.restype = ip
    lib.fwi_misfit_grad.argtypes = [vp, vp, ip, vp, ip, vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double), vp]
    lib.fwi_misfit_grad.restype = ip
    lib.cnn_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(ctypes.c_int), ctypes.c_ulonglong]
    lib.cnn_create.restype = ip
    lib.cnn_destroy.argtypes = [vp]
    lib.cnn_destroy.restype = None
    lib.cnn_num_params.argtypes = [vp]
    lib.cnn_num_params.restype = ctypes.c_longlong
    lib.cnn_set_params.argtypes = [vp, vp, ctypes.c_longlong]
    lib.cnn_set_params.restype = ip
    lib.cnn_get_params.argtypes = [vp, vp, ctypes.c_longlong]
    lib.cnn_get_params.restype = ip
    lib.cnn_forward.argtypes = [vp, vp, ip, vp, ip, ip, ip, vp]
    lib.cnn_forward.restype = ip
    lib.cnn_make_samples.argtypes = [vp, vp, vp, vp, ip, vp, vp]
    lib.cnn_make_samples.restype = ip
    lib.cnn_refine_samples.argtypes = [vp, vp, vp, vp, ip, ip, vp, vp]
    lib.cnn_refine_samples.restype = ip
    lib.cnn_loss_grad.argtypes = [vp, vp, vp, vp, vp, ip, ctypes.POINTER(ctypes.c_double), vp]
    lib.cnn_loss_grad.restype = ip
    lib.cnn_train_step.argtypes = [vp, vp, vp, vp, vp, ip, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
    lib.cnn_train_step.restype = ip
    lib.cnn_adam_reset.argtypes = [vp]
    lib.cnn_adam_reset.restype = ip
    lib.cnn_precond_apply.argtypes = [vp, vp, vp, ip, vp, ip]
    lib.cnn_precond_apply.restype = ip
    lib.cnn_conv3x3.argtypes = [vp, ip, vp, ip, ip, ip, ip, ip, vp, vp, ip, vp, ip, ip, vp]
    lib.cnn_conv3x3.restype = ip
    lib.cnn_set_loss.argtypes = [vp, ip]
    lib.cnn_set_loss.restype = ip
    lib.cnn_init_params.argtypes = [vp, ctypes.c_ulonglong, fp]
    lib.cnn_init_params.restype = ip
    lib.cnn_set_conv_path.argtypes = [ip]
    lib.cnn_set_conv_path.restype = ip
    lib.cnn_set_conv_tiling.argtypes = [ip]
    lib.cnn_set_conv_tiling.restype = ip
    lib.cnn_set_conv_buffers.argtypes = [ip]
    lib.cnn_set_conv_buffers.restype = ip
    lib.cnn_set_conv_upsplit.argtypes = [ip]
    lib.cnn_set_conv_upsplit.restype = ip
    lib.cnn_conv_plan.argtypes = [ip] * 11 + [ctypes.POINTER(ctypes.c_int)]
    lib.cnn_conv_plan.restype = ip
    lib.cnn_autotune.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int)]
    lib.cnn_autotune.restype = ip
    lib.cnn_autotune_reset.argtypes = []
    lib.cnn_autotune_reset.restype = None
    lib.helm_set_graphs.argtypes = [vp, ip]
    lib.helm_set_graphs.restype = ip
    lib.cnn_set_conv_ring.argtypes = [ip, ip]
    lib.cnn_set_conv_ring.restype = ip
    lib.cnn_conv_narrow_launches.argtypes = []
    lib.cnn_conv_narrow_launches.restype = ctypes.c_longlong
    lib.cnn_conv_rowtaps_launches.argtypes = []
    lib.cnn_conv_rowtaps_launches.restype = ctypes.c_longlong
    lib.cnn_conv_last_launch.argtypes = [ctypes.POINTER(ctypes.c_int)]
    lib.cnn_conv_last_launch.restype = None
    lib.cnn_conv_launch_counts.argtypes = [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.cnn_conv_launch_counts.restype = None
    lib.cnn_retrain_default_opts.argtypes = [ctypes.POINTER(cnn_retrain_opts)]
    lib.cnn_retrain_default_opts.restype = None
    lib.cnn_retrain_begin.argtypes = [vp, ctypes.POINTER(cnn_retrain_opts)]
    lib.cnn_retrain_begin.restype = ip
    lib.cnn_retrain_step.argtypes = [vp, vp, ip, fp, ctypes.POINTER(ctypes.c_float)]
    lib.cnn_retrain_step.restype = ip
    lib.cnn_retrain_state.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    lib.cnn_retrain_state.restype = ip
    lib.cnn_retrain_pairs.argtypes = [vp, ip, ip, vp, vp, ctypes.POINTER(ctypes.c_int)]
    lib.cnn_retrain_pairs.restype = ip
    sp = ctypes.POINTER(fwi_survey_t)
    lib.fwi_forward_data.argtypes = [vp, sp, ctypes.c_double, vp, ctypes.POINTER(ctypes.c_longlong)]
    lib.fwi_forward_data.restype = ip
    lib.fwi_jacobian.argtypes = [vp, sp, vp, ctypes.c_double, vp]
    lib.fwi_jacobian.restype = ip
    lib.fwi_jacobian_adjoint.argtypes = [vp, sp, vp, ctypes.c_double, vp]
    lib.fwi_jacobian_adjoint.restype = ip
    lib.helm_autotune.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int)]
    lib.helm_autotune.restype = ip
    lib.helm_autotune_reset.argtypes = []
    lib.helm_autotune_reset.restype = None
    lib.helm_resample.argtypes = [vp, ip, ip, vp, ip, ip, fp, fp, vp]
    lib.helm_resample.restype = ip
    lib.helm_solve_multi.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp), ctypes.c_double, ip,
                                     ctypes.POINTER(helm_stats)]
    lib.helm_solve_multi.restype = ip
    lib.fwi_model_to_kappa.argtypes = [vp, vp, ctypes.c_longlong]
    lib.fwi_model_to_kappa.restype = ip
    lib.fwi_default_gn_opts.argtypes = [ctypes.POINTER(fwi_gn_opts)]
    lib.fwi_default_gn_opts.restype = None
    lib.fwi_gn_iteration.argtypes = [vp, sp, vp, ctypes.POINTER(fwi_gn_opts), vp, ctypes.POINTER(fwi_gn_info)]
    lib.fwi_gn_iteration.restype = ip
    lib.cnn_wgrad_plan.argtypes = [ip] * 8 + [ctypes.POINTER(ctypes.c_longlong)]
    lib.cnn_wgrad_plan.restype = ip
    lib.cnn_set_wgrad_path.argtypes = [ip]
    lib.cnn_set_wgrad_path.restype = ip
    lib.cnn_conv3x3_backward.argtypes = [vp, ip, vp, ip, ip, ip, ip, ip, vp, ip, ip, vp, vp, vp, vp, vp]
    lib.cnn_conv3x3_backward.restype = ip
    lib.cnn_save.argtypes = [vp, ctypes.c_char_p]
    lib.cnn_save.restype = ip
    lib.cnn_load.argtypes = [ctypes.POINTER(vp), ctypes.c_char_p]
    lib.cnn_load.restype = ip
    lib.helm_destroy.argtypes = [vp]
    lib.helm_destroy.restype = None
    lib.helm_last_error.argtypes = []
    lib.helm_last_error.restype = ctypes.c_char_p
    lib.helm_profile_enable.argtypes = [vp, ip]
    lib.helm_profile_enable.restype = ip
    lib.helm_profile_read.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int)]
    lib.helm_profile_read.restype = ip
    lib.helm_profile_flops.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    lib.helm_profile_flops.restype = ip
    lib.helm_launch_count.argtypes = []
    lib.helm_launch_count.restype = ctypes.c_longlong
    return lib


lib = _load()


def last_error() -> str:
    return lib.helm_last_error().decode()


def _check(status: int, where: str, ok=(HELM_OK,)):
    if status not in ok:
        raise HelmError(status, where, last_error())
    return status


def _ptr(a, dtype_name: str):
    """Data pointer of a contiguous torch tensor or numpy array of the expected dtype."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        if a.dtype.name != dtype_name:
            raise TypeError(f"expected {dtype_name}, got {a.dtype.name}")
        return a.ctypes.data
    # torch tensor
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    tname = str(a.dtype).replace("torch.", "")
    if tname != dtype_name:
        raise TypeError(f"expected {dtype_name}, got {tname}")
    return a.data_ptr()


def _int_array(freq_idx, n):
    if freq_idx is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(freq_idx, dtype=np.int32))
    if arr.shape != (n,):
        raise ValueError("freq_idx must have one entry per right-hand side")
    return arr, arr.ctypes.data


def helm_default_opts(**overrides) -> helm_opts:
    o = helm_opts()
    lib.helm_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def helm_setup(kappa, gamma, nx: int, nz: int, hx: float, hz: float, omegas, net=None, opts=None):
    """Returns an opaque context handle (ctypes.c_void_p)."""
    om = omegas
    if not hasattr(om, "data_ptr") and not isinstance(om, np.ndarray):
        om = np.ascontiguousarray(np.asarray(om, dtype=np.float32))
    nfreq = int(om.shape[0]) if hasattr(om, "shape") else len(om)
    ctx = ctypes.c_void_p()
    o = opts if opts is not None else helm_default_opts()
    st = lib.helm_setup(ctypes.byref(ctx), _ptr(kappa, "float32"), _ptr(gamma, "float32"), nx, nz, hx, hz,
                        _ptr(om, "float32"), nfreq, net, ctypes.byref(o))
    _check(st, "helm_setup")
    return ctx


def helm_set_medium(ctx, kappa, gamma, omegas):
    om = omegas
    if not hasattr(om, "data_ptr") and not isinstance(om, np.ndarray):
        om = np.ascontiguousarray(np.asarray(om, dtype=np.float32))
    nfreq = int(om.shape[0])
    _check(lib.helm_set_medium(ctx, _ptr(kappa, "float32"), _ptr(gamma, "float32"), _ptr(om, "float32"), nfreq),
           "helm_set_medium")


def helm_solve(ctx, rhs, x, nrhs: int, freq_idx=None, tol: float = 1e-6, flags: int = 0, check=True):
    """flags: HELM_SOLVE_ADJOINT | HELM_SOLVE_ZERO_X0.
    Returns (status, iters[nrhs], rel_res[nrhs], per_rhs_status[nrhs]) as numpy arrays."""
    iters = np.zeros(nrhs, dtype=np.int32)
    rel = np.zeros(nrhs, dtype=np.float64)
    stat = np.zeros(nrhs, dtype=np.int32)
    stats = helm_stats(iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                       rel.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       stat.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    _keep, fptr = _int_array(freq_idx, nrhs)
    st = lib.helm_solve(ctx, _ptr(rhs, "complex64"), _ptr(x, "complex128"), nrhs, fptr, tol, flags,
                        ctypes.byref(stats))
    if check:
        _check(st, "helm_solve", ok=(HELM_OK, HELM_ENOCONV, HELM_EBREAKDOWN))
    return st, iters, rel, stat


def helm_residual(ctx, rhs, x, r, nrhs: int, freq_idx=None):
    """r = rhs - H x (FP64 evaluation, stored complex64); returns the relative residuals."""
    rel = np.zeros(nrhs, dtype=np.float64)
    _keep, fptr = _int_array(freq_idx, nrhs)
    _check(lib.helm_residual(ctx, _ptr(rhs, "complex64"), _ptr(x, "complex128"), _ptr(r, "complex64"), nrhs, fptr,
                             rel.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "helm_residual")
    return rel


def helm_residual_noalloc(kappa, gamma, nx: int, nz: int, hx: float, hz: float, omega_rhs, rhs, x, r, rel_res,
                          nrhs: int, stream=None):
    """Allocation-free FP64 residual: every array a device tensor; returns without waiting."""
    _check(lib.helm_residual_noalloc(_ptr(kappa, "float32"), _ptr(gamma, "float32"), nx, nz, hx, hz,
                                     _ptr(omega_rhs, "float32"), _ptr(rhs, "complex64"), _ptr(x, "complex128"),
                                     _ptr(r, "complex64"), _ptr(rel_res, "float64"), nrhs, stream),
           "helm_residual_noalloc")


def helm_apply(ctx, x, y, nrhs: int, freq_idx=None, op: int = HELM_OP_H):
    _keep, fptr = _int_array(freq_idx, nrhs)
    _check(lib.helm_apply(ctx, _ptr(x, "complex64"), _ptr(y, "complex64"), nrhs, fptr, op), "helm_apply")


def helm_vcycle(ctx, f, u0, u, nrhs: int, freq_idx=None):
    _keep, fptr = _int_array(freq_idx, nrhs)
    _check(lib.helm_vcycle(ctx, _ptr(f, "complex64"), _ptr(u0, "complex64"), _ptr(u, "complex64"), nrhs, fptr),
           "helm_vcycle")


def fwi_misfit_grad(ctx, src_idx, rcv_idx, d_obs, grad_m, tol: float = 1e-8) -> float:
    """Returns the misfit; writes dPhi/dm into ``grad_m`` (float32 [nz][nx])."""
    src = np.ascontiguousarray(np.asarray(src_idx, dtype=np.int32))
    rcv = np.ascontiguousarray(np.asarray(rcv_idx, dtype=np.int32))
    phi = ctypes.c_double(0.0)
    _check(lib.fwi_misfit_grad(ctx, src.ctypes.data, src.size, rcv.ctypes.data, rcv.size, _ptr(d_obs, "complex64"),
                               tol, ctypes.byref(phi), _ptr(grad_m, "float32")), "fwi_misfit_grad")
    return phi.value


class Survey:
    """An FWI survey (include/helm.h fwi_survey): point-source and receiver node indices
    (flat iz * nx + ix) and, for simultaneous sources, the weights [nsim][nsrc]."""

    def __init__(self, src_idx, rcv_idx, src_w=None):
        self.src = np.ascontiguousarray(np.asarray(src_idx, dtype=np.int32))
        self.rcv = np.ascontiguousarray(np.asarray(rcv_idx, dtype=np.int32))
        self.w = None if src_w is None else np.ascontiguousarray(np.asarray(src_w, dtype=np.float32))
        self.nsim = self.src.size if self.w is None else int(self.w.shape[0])
        self.c = fwi_survey_t(self.src.ctypes.data, self.src.size, None if self.w is None else self.w.ctypes.data,
                              0 if self.w is None else self.nsim, self.rcv.ctypes.data, self.rcv.size)


def fwi_forward_data(ctx, survey: Survey, d_out, tol: float = 1e-6) -> int:
    """Synthetic data [nfreq][nsources][nrcv] into d_out; returns the Helmholtz iterations used."""
    it = ctypes.c_longlong(0)
    _check(lib.fwi_forward_data(ctx, ctypes.byref(survey.c), tol, _ptr(d_out, "complex64"), ctypes.byref(it)),
           "fwi_forward_data")
    return int(it.value)


def fwi_jacobian(ctx, survey: Survey, dm, dd_out, tol: float = 1e-4):
    _check(lib.fwi_jacobian(ctx, ctypes.byref(survey.c), _ptr(dm, "float32"), tol, _ptr(dd_out, "complex64")),
           "fwi_jacobian")


def fwi_jacobian_adjoint(ctx, survey: Survey, dd, dm_out, tol: float = 1e-4):
    _check(lib.fwi_jacobian_adjoint(ctx, ctypes.byref(survey.c), _ptr(dd, "complex64"), tol,
                                    _ptr(dm_out, "float32")), "fwi_jacobian_adjoint")


def fwi_model_to_kappa(m, kappa):
    """kappa = sqrt(m) (device tensors)."""
    _check(lib.fwi_model_to_kappa(_ptr(m, "float32"), _ptr(kappa, "float32"), int(m.numel())),
           "fwi_model_to_kappa")


def fwi_default_gn_opts(**overrides) -> fwi_gn_opts:
    o = fwi_gn_opts()
    lib.fwi_default_gn_opts(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def fwi_gn_iteration(ctx, survey: Survey, d_obs, m, opts=None, m_ref=None) -> dict:
    """One Gauss-Newton iteration; m (float32 [nz][nx]) updated in place.  m_ref (float32
    [nz][nx], host or device) is the regulariser's reference model, kept alive by the caller
    for the call.  Returns the info fields."""
    o = opts if opts is not None else fwi_default_gn_opts()
    if m_ref is not None:
        o = fwi_gn_opts.from_buffer_copy(o)
        o.m_ref = _ptr(m_ref, "float32")
    info = fwi_gn_info()
    _check(lib.fwi_gn_iteration(ctx, ctypes.byref(survey.c), _ptr(d_obs, "complex64"), ctypes.byref(o),
                                _ptr(m, "float32"), ctypes.byref(info)), "fwi_gn_iteration")
    return {k: getattr(info, k) for k, _ in fwi_gn_info._fields_}


def helm_autotune(ctx, nrhs: int) -> int:
    """Time the multigrid sweeps' block shapes (and the convolutions with a network); returns the
    number of tuned sweep entries."""
    n = ctypes.c_int(0)
    _check(lib.helm_autotune(ctx, nrhs, ctypes.byref(n)), "helm_autotune")
    return int(n.value)


def helm_autotune_reset():
    lib.helm_autotune_reset()


def helm_resample(src, nx0: int, nz0: int, dst, nx1: int, nz1: int, alpha: float = 1.0, beta: float = 0.0,
                  stream=None):
    """dst = alpha * bilinear(src) + beta * dst between node grids of one rectangle (device tensors)."""
    _check(lib.helm_resample(_ptr(src, "float32"), nx0, nz0, _ptr(dst, "float32"), nx1, nz1, alpha, beta, stream),
           "helm_resample")


def helm_solve_multi(ctxs, rhs_list, x_list, nrhs_list, freq_list=None, tol: float = 1e-6, flags: int = 0):
    """helm_solve of several contexts in one call.  Returns (status, [(iters, rel_res, status) per context])."""
    n = len(ctxs)
    carr = (ctypes.c_void_p * n)(*[c.value if hasattr(c, "value") else c for c in ctxs])
    rarr = (ctypes.c_void_p * n)(*[_ptr(r, "complex64") for r in rhs_list])
    xarr = (ctypes.c_void_p * n)(*[_ptr(x, "complex128") for x in x_list])
    nb = (ctypes.c_int * n)(*[int(v) for v in nrhs_list])
    keep, fptrs = [], []
    for i in range(n):
        f = None if freq_list is None else freq_list[i]
        k, p = _int_array(f, int(nrhs_list[i]))
        keep.append(k)
        fptrs.append(p)
    farr = (ctypes.c_void_p * n)(*fptrs)
    outs, stats = [], (helm_stats * n)()
    for i in range(n):
        it = np.zeros(nrhs_list[i], np.int32)
        rel = np.zeros(nrhs_list[i], np.float64)
        st = np.zeros(nrhs_list[i], np.int32)
        outs.append((it, rel, st))
        stats[i] = helm_stats(it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                              rel.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    status = lib.helm_solve_multi(carr, n, rarr, xarr, nb, farr, tol, flags, stats)
    _check(status, "helm_solve_multi", ok=(HELM_OK, HELM_ENOCONV, HELM_EBREAKDOWN))
    return status, outs


def helm_destroy(ctx):
    if ctx:
        lib.helm_destroy(ctx)


def helm_profile_enable(ctx, on: bool = True):
    _check(lib.helm_profile_enable(ctx, 1 if on else 0), "helm_profile_enable")


def helm_profile_read(ctx) -> dict:
    """{kernel class: (total ms, launches, algorithmic bytes)}"""
    n = 64
    names = (ctypes.c_char_p * n)()
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    nbytes = (ctypes.c_double * n)()
    k = ctypes.c_int(0)
    _check(lib.helm_profile_read(ctx, n, names, ms, cnt, nbytes, ctypes.byref(k)), "helm_profile_read")
    return {names[i].decode(): (ms[i], cnt[i], nbytes[i]) for i in range(k.value)}


def helm_profile_flops(ctx) -> dict:
    """{kernel class: algorithmic flops} since profiling was enabled"""
    n = 64
    names = (ctypes.c_char_p * n)()
    k = ctypes.c_int(0)
    _check(lib.helm_profile_read(ctx, n, names, None, None, None, ctypes.byref(k)), "helm_profile_read")
    fl = (ctypes.c_double * n)()
    _check(lib.helm_profile_flops(ctx, n, fl, ctypes.byref(k)), "helm_profile_flops")
    return {names[i].decode(): fl[i] for i in range(k.value)}


def helm_launch_count() -> int:
    return int(lib.helm_launch_count())


def helm_set_graphs(ctx, on: bool):
    """Capture and replay the restart cycles of MG / plain FGMRES as a CUDA graph (default on)."""
    _check(lib.helm_set_graphs(ctx, 1 if on else 0), "helm_set_graphs")


# --------------------------------------------------------------------------
# encoder-solver network
# --------------------------------------------------------------------------

def cnn_create(levels: int, widths, seed: int = 2):
    """The network with seeded half-scale He-normal weights (seed 2 is the library's CNN stream)."""
    w = (ctypes.c_int * levels)(*widths)
    net = ctypes.c_void_p()
    _check(lib.cnn_create(ctypes.byref(net), levels, w, seed), "cnn_create")
    return net


def cnn_save(net, path: str):
    _check(lib.cnn_save(net, os.fsencode(path)), "cnn_save")


def cnn_load(path: str):
    net = ctypes.c_void_p()
    _check(lib.cnn_load(ctypes.byref(net), os.fsencode(path)), "cnn_load")
    return net


def cnn_retrain_default_opts(**overrides) -> cnn_retrain_opts:
    o = cnn_retrain_opts()
    lib.cnn_retrain_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def cnn_retrain_begin(ctx, **opts):
    o = cnn_retrain_default_opts(**opts)
    _check(lib.cnn_retrain_begin(ctx, ctypes.byref(o)), "cnn_retrain_begin")


def cnn_retrain_step(net, ctx, batch: int, lr: float) -> float:
    loss = ctypes.c_float(0.0)
    _check(lib.cnn_retrain_step(net, ctx, batch, lr, ctypes.byref(loss)), "cnn_retrain_step")
    return float(loss.value)


def cnn_retrain_state(ctx) -> dict:
    v = (ctypes.c_longlong * 6)()
    _check(lib.cnn_retrain_state(ctx, v), "cnn_retrain_state")
    return dict(zip(("epoch", "pos", "size", "steps", "done", "capacity"), (int(x) for x in v)))


def cnn_retrain_pairs(ctx, first: int, n: int, r_out, e_out):
    """Copies pairs first .. first + n - 1 of the dataset; returns their frequency indices."""
    f = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib.cnn_retrain_pairs(ctx, first, n, _ptr(r_out, "complex64"), _ptr(e_out, "complex64"),
                                 f.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), "cnn_retrain_pairs")
    return f[:n]


def cnn_destroy(net):
    if net:
        lib.cnn_destroy(net)


def cnn_num_params(net) -> int:
    return int(lib.cnn_num_params(net))


def cnn_set_params(net, params):
    _check(lib.cnn_set_params(net, _ptr(params, "float32"), int(np.prod(params.shape))), "cnn_set_params")


def cnn_get_params(net, params):
    _check(lib.cnn_get_params(net, _ptr(params, "float32"), int(np.prod(params.shape))), "cnn_get_params")


def cnn_forward(net, enc_in, nenc: int, sol_in, nsol: int, ny: int, nx: int, out):
    _check(lib.cnn_forward(net, _ptr(enc_in, "float32"), nenc, _ptr(sol_in, "float32"), nsol, ny, nx,
                           _ptr(out, "float32")), "cnn_forward")


def cnn_conv3x3(x0, c0: int, x1, c1: int, x1_bcast: int, nb: int, hin: int, win: int, w, bias, cout: int, res,
                mode: int, relu: int, y):
    _check(lib.cnn_conv3x3(_ptr(x0, "float32"), c0, _ptr(x1, "float32"), c1, x1_bcast, nb, hin, win,
                           _ptr(w, "float32"), _ptr(bias, "float32"), cout, _ptr(res, "float32"), mode, relu,
                           _ptr(y, "float32")), "cnn_conv3x3")


def cnn_init_params(net, seed: int, gain: float = 1.0):
    """Seeded He-normal weights (scaled by gain), zero biases."""
    _check(lib.cnn_init_params(net, int(seed), float(gain)), "cnn_init_params")


def cnn_set_loss(net, kind: int):
    """0: Eq. 4.2 mean squared error (default); 1: per-sample error relative to ||e||^2."""
    _check(lib.cnn_set_loss(net, int(kind)), "cnn_set_loss")


def cnn_set_conv_path(path: int):
    """0: TMA halo-tile kernel (default); 1: gather kernel for all layers;
    2: TMA kernel with the column-taps-in-N variant of the 16-channel layers;
    3: TMA kernel with the three tap rows in N for the 16- and 32-channel same-grid
    layers."""
    _check(lib.cnn_set_conv_path(int(path)), "cnn_set_conv_path")


def cnn_set_conv_buffers(nbuf: int):
    """TMEM accumulator buffers of the TMA conv kernel: 1 single buffer, 0/2 default."""
    _check(lib.cnn_set_conv_buffers(int(nbuf)), "cnn_set_conv_buffers")


def cnn_set_conv_upsplit(on: int):
    """Up layers of the TMA conv kernel: 1 a tile per output row parity, 0 default."""
    _check(lib.cnn_set_conv_upsplit(int(on)), "cnn_set_conv_upsplit")


def cnn_set_conv_tiling(max_rows: int):
    """Tile-height limit of the TMA conv kernel (0 = automatic)."""
    _check(lib.cnn_set_conv_tiling(int(max_rows)), "cnn_set_conv_tiling")


CONV_PLAN_FIELDS = ("tiles", "tw", "rows", "pw", "mb", "nph", "nplanes", "plane", "pstride", "wbytes", "stage",
                    "ns", "tmem_cols", "nslot", "slot_cols", "mode", "nwg", "chunk", "nbuf")


def cnn_conv_plan(mode: int, c0: int, c1: int, npad: int, hin: int, win: int, nb: int = 1, stage_kb: int = 0,
                  ring_kb: int = 0, rows_cap: int = 0, narrow: int = 0):
    """Host-side tile plan of the TMA convolution (dict of CONV_PLAN_FIELDS), or None when
    the kernel does not take the layer.  narrow: 0 plain, 1 (or True) the column-taps-in-N
    variant, 2 the row-taps-in-N variant, 3 the single-accumulator-buffer tiling, 4 up layers
    with a tile per output row parity, 5 both of the last two."""
    out = (ctypes.c_int * 19)()
    st = lib.cnn_conv_plan(mode, c0, c1, npad, hin, win, nb, stage_kb, ring_kb, rows_cap, int(narrow), out)
    if st != HELM_OK:
        return None
    return dict(zip(CONV_PLAN_FIELDS, list(out)))


WGRAD_PLAN_FIELDS = ("ktiles", "tw", "rows", "P", "tiles_x", "tiles_y", "phases", "cx", "cx0", "gchunks", "tpg",
                     "ngroups", "max_chunks", "plane", "stage", "ns", "slack", "tmem_cols", "splits", "smem")


def cnn_wgrad_plan(mode: int, c0: int, c1: int, npad: int, hin: int, win: int, nb: int = 1, sms: int = 0):
    """Host-side tile plan of the tensor-core weight gradient (dict of WGRAD_PLAN_FIELDS), or
    None when the kernel does not take the layer."""
    out = (ctypes.c_longlong * 20)()
    if lib.cnn_wgrad_plan(mode, c0, c1, npad, hin, win, nb, sms, out) != HELM_OK:
        return None
    return dict(zip(WGRAD_PLAN_FIELDS, list(out)))


def cnn_set_wgrad_path(path: int):
    """Weight gradients on the tensor cores (0, default) or the FP32 CUDA cores (1)."""
    _check(lib.cnn_set_wgrad_path(path), "cnn_set_wgrad_path")


def cnn_conv3x3_backward(x0, c0: int, x1, c1: int, x1_bcast: int, nb: int, hin: int, win: int, w, cout: int,
                         mode: int, gy, gx0=None, gx1=None, dw=None, db=None):
    _check(lib.cnn_conv3x3_backward(_ptr(x0, "float32"), c0, _ptr(x1, "float32"), c1, x1_bcast, nb, hin, win,
                                    _ptr(w, "float32"), cout, mode, _ptr(gy, "float32"), _ptr(gx0, "float32"),
                                    _ptr(gx1, "float32"), _ptr(dw, "float32"), _ptr(db, "float32")),
           "cnn_conv3x3_backward")


def cnn_autotune(ctx, nrhs: int) -> int:
    """Time the candidate tilings of every layer shape of the solver pass; returns the tuned shapes."""
    n = ctypes.c_int(0)
    _check(lib.cnn_autotune(ctx, int(nrhs), ctypes.byref(n)), "cnn_autotune")
    return int(n.value)


def cnn_autotune_reset():
    """Forget every tuned convolution tiling."""
    lib.cnn_autotune_reset()


def cnn_conv_narrow_launches() -> int:
    """Launches of the column-taps-in-N convolution since the library was loaded."""
    return int(lib.cnn_conv_narrow_launches())


def cnn_conv_rowtaps_launches() -> int:
    """Launches of the row-taps-in-N convolution since the library was loaded."""
    return int(lib.cnn_conv_rowtaps_launches())


def cnn_set_conv_ring(stage_kb: int, ring_kb: int):
    """Stage and ring shared-memory budgets of the TMA conv kernel in KB (0 = default)."""
    _check(lib.cnn_set_conv_ring(int(stage_kb), int(ring_kb)), "cnn_set_conv_ring")


def cnn_conv_last_launch():
    """(grid, CTAs per SM, CTAs per SM allowed by registers and smem, shared memory bytes, registers, static smem)
    of the last TMA conv."""
    out = (ctypes.c_int * 6)()
    lib.cnn_conv_last_launch(out)
    return tuple(out)


def cnn_conv_launch_counts():
    """(TMA-kernel launches, gather-kernel launches) since the library was loaded."""
    t, g = ctypes.c_longlong(0), ctypes.c_longlong(0)
    lib.cnn_conv_launch_counts(ctypes.byref(t), ctypes.byref(g))
    return t.value, g.value


def cnn_precond_apply(ctx, r, e, nrhs: int, freq_idx=None, with_vcycle: int = 1):
    _keep, fptr = _int_array(freq_idx, nrhs)
    _check(lib.cnn_precond_apply(ctx, _ptr(r, "complex64"), _ptr(e, "complex64"), nrhs, fptr, with_vcycle),
           "cnn_precond_apply")


def cnn_make_samples(ctx, x, iters, r_out, e_out, nb: int, freq_idx=None):
    _keep, fptr = _int_array(freq_idx, nb)
    it = np.ascontiguousarray(np.asarray(iters, dtype=np.int32))
    _check(lib.cnn_make_samples(ctx, _ptr(x, "complex64"), fptr, it.ctypes.data, nb, _ptr(r_out, "complex64"),
                                _ptr(e_out, "complex64")), "cnn_make_samples")


def cnn_refine_samples(ctx, r, e, r_out, e_out, nb: int, freq_idx=None, literal: int = 0):
    _keep, fptr = _int_array(freq_idx, nb)
    _check(lib.cnn_refine_samples(ctx, _ptr(r, "complex64"), _ptr(e, "complex64"), fptr, nb, literal,
                                  _ptr(r_out, "complex64"), _ptr(e_out, "complex64")), "cnn_refine_samples")


def cnn_loss_grad(net, ctx, r, e, nb: int, freq_idx=None, grad_out=None) -> float:
    _keep, fptr = _int_array(freq_idx, nb)
    loss = ctypes.c_double(0.0)
    _check(lib.cnn_loss_grad(net, ctx, _ptr(r, "complex64"), _ptr(e, "complex64"), fptr, nb, ctypes.byref(loss),
                             _ptr(grad_out, "float32")), "cnn_loss_grad")
    return loss.value


def cnn_train_step(net, ctx, r, e, nb: int, lr: float, freq_idx=None) -> float:
    _keep, fptr = _int_array(freq_idx, nb)
    loss = ctypes.c_double(0.0)
    _check(lib.cnn_train_step(net, ctx, _ptr(r, "complex64"), _ptr(e, "complex64"), fptr, nb, lr,
                              ctypes.byref(loss)), "cnn_train_step")
    return loss.value


def cnn_adam_reset(net):
    _check(lib.cnn_adam_reset(net), "cnn_adam_reset")
