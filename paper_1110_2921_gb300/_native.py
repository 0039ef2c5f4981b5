"""ctypes binding of libvfmm (include/vfmm.h): argument marshalling only.

The library must exist (built by ``paper_1110_2921_gb300.build``); there is no fallback
implementation, and importing fails loudly if it is missing.
"""
import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libvfmm.so")

VFMM_OK = 0
VFMM_ERR_ARG = -1
VFMM_ERR_CUDA = -2
VFMM_ERR_OOM = -3
VFMM_ERR_NOT_BUILT = -4
VFMM_ERR_BOUNDS = -5
VFMM_ERR_TIMEOUT = -6
VFMM_ERR_UNSUPPORTED = -7
VFMM_F32 = 0
VFMM_F64 = 1
VFMM_M2L_FP32 = 0
VFMM_M2L_FP64 = 1
VFMM_M2L_TF32X3 = 2
VFMM_M2L_BF16X3 = 3
VFMM_METHOD_FMM = 0
VFMM_METHOD_DIRECT = 1
VFMM_PROBE_FFMA = 0
VFMM_PROBE_EX2 = 1
VFMM_PROBE_RSQRT = 2
VFMM_PROBE_DFMA = 3
VFMM_PROBE_MMA_TF32 = 4
VFMM_PROBE_MMA_BF16 = 5


class vfmm_config(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("depth", ctypes.c_int), ("ncrit", ctypes.c_int),
                ("near_rings", ctypes.c_int), ("rho_cut", ctypes.c_double),
                ("periodic_levels", ctypes.c_int), ("box", ctypes.c_double),
                ("dtype", ctypes.c_int), ("m2l_prec", ctypes.c_int), ("method", ctypes.c_int),
                ("direct_images", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("concurrent_far", ctypes.c_int)]


class VfmmError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__("%s failed: %s (%d)%s" % (where, strerror(status), status,
                                                   (": " + detail) if detail else ""))


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libvfmm.so is not built (run paper_1110_2921_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        H = ctypes.c_void_p
        V = ctypes.c_void_p
        sig = {
            "vfmm_config_default": ([ctypes.POINTER(vfmm_config)], ctypes.c_int),
            "vfmm_create": ([ctypes.POINTER(vfmm_config), ctypes.POINTER(H)], ctypes.c_int),
            "vfmm_destroy": ([H], ctypes.c_int),
            "vfmm_set_stream": ([H, V], ctypes.c_int),
            "vfmm_set_wait_limit": ([H, ctypes.c_int64], ctypes.c_int),
            "vfmm_build_tree": ([H, ctypes.c_int64, V], ctypes.c_int),
            "vfmm_eval_velocity_stretching": ([H, V, ctypes.c_double, V, V], ctypes.c_int),
            "vfmm_eval_host": ([H, ctypes.c_int64, V, V, ctypes.c_double, V, V], ctypes.c_int),
            "vfmm_eval_velocity_gradient": ([H, V, ctypes.c_double, V, V], ctypes.c_int),
            "vfmm_eval_adjoint": ([H, V, ctypes.c_double, V, V, V, V], ctypes.c_int),
            "vfmm_rk_step": ([H, ctypes.c_int64, V, V, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                              ctypes.c_double], ctypes.c_int),
            "vfmm_diagnostics": ([H, ctypes.c_int64, V, V, V, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "vfmm_energy_spectrum": ([H, ctypes.c_int, V, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "vfmm_derivative_moments": ([H, ctypes.c_int64, V, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "vfmm_reinit": ([H, ctypes.c_int64, V, V, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                             V, V, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "vfmm_sync": ([H], ctypes.c_int),
            "vfmm_get_timings": ([H, ctypes.POINTER(ctypes.c_double), ctypes.c_int], ctypes.c_int),
            "vfmm_get_tree_info": ([H, ctypes.POINTER(ctypes.c_int64), ctypes.c_int], ctypes.c_int),
            "vfmm_probe_peak": ([ctypes.c_int, ctypes.c_int64, V, V, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "vfmm_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "vfmm_last_error": ([H], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def strerror(status):
    return lib().vfmm_strerror(int(status)).decode()


def check(status, where, handle=None):
    if status != VFMM_OK:
        detail = ""
        if handle:
            detail = lib().vfmm_last_error(handle).decode()
        raise VfmmError(status, where, detail)


def config_default():
    c = vfmm_config()
    check(lib().vfmm_config_default(ctypes.byref(c)), "vfmm_config_default")
    return c


def vfmm_create(cfg):
    h = ctypes.c_void_p()
    check(lib().vfmm_create(ctypes.byref(cfg), ctypes.byref(h)), "vfmm_create")
    return h


def vfmm_destroy(h):
    check(lib().vfmm_destroy(h), "vfmm_destroy")


def vfmm_set_stream(h, stream_ptr):
    check(lib().vfmm_set_stream(h, ctypes.c_void_p(stream_ptr)), "vfmm_set_stream", h)


def vfmm_set_wait_limit(h, tries):
    check(lib().vfmm_set_wait_limit(h, int(tries)), "vfmm_set_wait_limit", h)


def vfmm_build_tree(h, n, x_ptr):
    check(lib().vfmm_build_tree(h, int(n), ctypes.c_void_p(x_ptr)), "vfmm_build_tree", h)


def vfmm_eval_velocity_stretching(h, gamma_ptr, sigma, u_ptr, s_ptr):
    check(lib().vfmm_eval_velocity_stretching(h, ctypes.c_void_p(gamma_ptr), float(sigma),
                                              ctypes.c_void_p(u_ptr),
                                              ctypes.c_void_p(s_ptr) if s_ptr else None),
          "vfmm_eval_velocity_stretching", h)


def vfmm_eval_velocity_gradient(h, gamma_ptr, sigma, u_ptr, g_ptr):
    check(lib().vfmm_eval_velocity_gradient(h, ctypes.c_void_p(gamma_ptr), float(sigma), ctypes.c_void_p(u_ptr),
                                            ctypes.c_void_p(g_ptr)), "vfmm_eval_velocity_gradient", h)


def vfmm_eval_adjoint(h, gamma_ptr, sigma, w_ptr, v_ptr, dgamma_ptr, dx_ptr):
    check(lib().vfmm_eval_adjoint(h, ctypes.c_void_p(gamma_ptr), float(sigma), ctypes.c_void_p(w_ptr),
                                  ctypes.c_void_p(v_ptr) if v_ptr else None, ctypes.c_void_p(dgamma_ptr),
                                  ctypes.c_void_p(dx_ptr)), "vfmm_eval_adjoint", h)


def vfmm_rk_step(h, n, x_ptr, gamma_ptr, sigma, dt, nu):
    s = ctypes.c_double(sigma)
    check(lib().vfmm_rk_step(h, int(n), ctypes.c_void_p(x_ptr), ctypes.c_void_p(gamma_ptr), ctypes.byref(s),
                             float(dt), float(nu)), "vfmm_rk_step", h)
    return s.value


def vfmm_reinit(h, n, x_ptr, gamma_ptr, sigma, m, sigma_new, iters, x_new_ptr, gamma_new_ptr):
    res = ctypes.c_double(0.0)
    check(lib().vfmm_reinit(h, int(n), ctypes.c_void_p(x_ptr), ctypes.c_void_p(gamma_ptr), float(sigma), int(m),
                            float(sigma_new), int(iters), ctypes.c_void_p(x_new_ptr), ctypes.c_void_p(gamma_new_ptr),
                            ctypes.byref(res)), "vfmm_reinit", h)
    return res.value


def vfmm_diagnostics(h, n, x_ptr, gamma_ptr, u_ptr):
    out = (ctypes.c_double * 8)()
    check(lib().vfmm_diagnostics(h, int(n), ctypes.c_void_p(x_ptr), ctypes.c_void_p(gamma_ptr),
                                 ctypes.c_void_p(u_ptr) if u_ptr else None, out), "vfmm_diagnostics", h)
    return list(out)


def vfmm_energy_spectrum(h, n, u_ptr, kmax):
    out = (ctypes.c_double * (kmax + 1))()
    check(lib().vfmm_energy_spectrum(h, int(n), ctypes.c_void_p(u_ptr), int(kmax), out), "vfmm_energy_spectrum", h)
    return list(out)


def vfmm_derivative_moments(h, n, g_ptr):
    out = (ctypes.c_double * 5)()
    check(lib().vfmm_derivative_moments(h, int(n), ctypes.c_void_p(g_ptr), out), "vfmm_derivative_moments", h)
    return list(out)


def vfmm_eval_host(h, n, x_ptr, gamma_ptr, sigma, u_ptr, s_ptr):
    check(lib().vfmm_eval_host(h, int(n), ctypes.c_void_p(x_ptr), ctypes.c_void_p(gamma_ptr),
                               float(sigma), ctypes.c_void_p(u_ptr),
                               ctypes.c_void_p(s_ptr) if s_ptr else None), "vfmm_eval_host", h)


def vfmm_sync(h):
    check(lib().vfmm_sync(h), "vfmm_sync", h)


def vfmm_get_timings(h):
    buf = (ctypes.c_double * 8)()
    check(lib().vfmm_get_timings(h, buf, 8), "vfmm_get_timings", h)
    return list(buf)


def vfmm_get_tree_info(h):
    buf = (ctypes.c_int64 * 8)()
    check(lib().vfmm_get_tree_info(h, buf, 8), "vfmm_get_tree_info", h)
    return {"depth": buf[0], "near_rings": buf[1], "leaves_per_side": buf[2],
            "max_leaf": buf[3], "n": buf[4], "launches": buf[5], "correction_rings": buf[6],
            "p2p_pairs_checked": buf[7]}


def vfmm_probe_peak(kind, reps, stream_ptr, err_ptr=None):
    """Launch one peak-rate probe on the stream; returns the operations it performs."""
    ops = ctypes.c_double(0.0)
    check(lib().vfmm_probe_peak(int(kind), int(reps), ctypes.c_void_p(stream_ptr),
                                ctypes.c_void_p(err_ptr) if err_ptr else None, ctypes.byref(ops)),
          "vfmm_probe_peak")
    return ops.value
