"""Thin ctypes binding of the C ABI in include/pywolf_gb.h (argument marshalling only).

Every function has the C name and takes plain integers / device addresses; every step of
the propagation runs in the library's CUDA kernels.  A non-PW_OK status raises PwError with
the library's message.  There is no fallback: if libpywolf_gb.so is missing or fails to
load, importing this module raises.
"""
import ctypes
import os

from . import build as _build

PW_OK, PW_EINVAL, PW_ESIZE, PW_ECUDA, PW_ETIMEOUT, PW_ESTATE, PW_EUNSUPPORTED = range(7)

if not os.path.exists(_build.LIB):
    raise ImportError("libpywolf_gb.so is not built: run `python -c \"import __graft_entry__ as g; g.build()\"` "
                      "or `python -m paper_2203_02734_gb300.build`")
LIB = ctypes.CDLL(_build.LIB)

_vp = ctypes.c_void_p
_d = ctypes.c_double
_i = ctypes.c_int

# name: (restype, argtypes)
SIGNATURES = {
    "pw_last_error": (ctypes.c_char_p, []),
    "pw_status_string": (ctypes.c_char_p, [_i]),
    "pw_supported_n": (_i, [_i]),
    "pw_csda_bytes": (ctypes.c_size_t, [_i]),
    "pw_csd_create": (_i, [ctypes.POINTER(_vp), _i, _d, _d, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t, _vp]),
    "pw_csd_destroy": (_i, [_vp]),
    "pw_csd_set_stream": (_i, [_vp, _vp]),
    "pw_csd_reset": (_i, [_vp, _d]),
    "pw_csd_check": (_i, [_vp]),
    "pw_csd_enable_timing": (_i, [_vp, _i]),
    "pw_csd_set_dft_mode": (_i, [_vp, _i]),
    "pw_csd_set_padding": (_i, [_vp, _i]),
    "pw_csd_inject_stall": (_i, [_vp, _i]),
    "pw_csd_get_padding": (_i, [_vp, ctypes.POINTER(_i)]),
    "pw_csd_get_dft_mode": (_i, [_vp, ctypes.POINTER(_i)]),
    "pw_csd_pass_times": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_i)]),
    "pw_csd_pass_times3": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_i)]),
    "pw_source_gsm": (_i, [_vp, _d, _d, _d]),
    "pw_source_aperture": (_i, [_vp, _d]),
    "pw_source_lens": (_i, [_vp, _d]),
    "pw_source_mask": (_i, [_vp, _vp]),
    "pw_source_array": (_i, [_vp, _vp, _i]),
    "pw_source_diagonal": (_i, [_vp, _vp, _d]),
    "pw_gsm_gradient": (_i, [_vp, _d, _d, _d, _vp, _d, _d, _i, _vp, _vp]),
    "pw_propagate_fresnel": (_i, [_vp, _d]),
    "pw_propagate_farfield": (_i, [_vp, _d]),
    "pw_get_sampling": (_i, [_vp, ctypes.POINTER(_d)]),
    "pw_spectral_density": (_i, [_vp, _vp]),
    "pw_degree_of_coherence": (_i, [_vp, _i, _i, _vp]),
    "pw_propagate_gsm_fresnel_noalloc": (_i, [_i, _d, _d, _d, _d, _d, _d, _d, _d, _vp, _vp, ctypes.c_size_t,
                                             _vp, _vp]),
}
for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(LIB, _name)
    _f.restype = _res
    _f.argtypes = _args


class pw_instance(ctypes.Structure):
    """Mirror of the C struct pw_instance (include/pywolf_gb.h)."""
    _fields_ = [("N", _i), ("dxi_m", _d), ("lambda_m", _d), ("z_m", _d), ("farfield", _i),
                ("sigma_S_m", _d), ("sigma_mu_m", _d), ("amplitude", _d), ("aperture_m", _d),
                ("lens_f_m", _d), ("dev_mask", _vp), ("iP", _i), ("jP", _i), ("dev_W", _vp),
                ("dev_S", _vp), ("dev_mu", _vp)]


_IP = ctypes.POINTER(pw_instance)
for _name, (_res, _args) in {
    "pw_batch_workspace_bytes": (ctypes.c_size_t, [_IP, _i, _i]),
    "pw_batch_create": (_i, [ctypes.POINTER(_vp), _IP, _i, _i, _vp, ctypes.c_size_t, _vp]),
    "pw_batch_run": (_i, [_vp]),
    "pw_batch_check": (_i, [_vp]),
    "pw_batch_set_chunk": (_i, [_vp, _i]),
    "pw_batch_get_chunk": (_i, [_vp, ctypes.POINTER(_i)]),
    "pw_batch_set_mode": (_i, [_vp, _i]),
    "pw_batch_spectral_sum": (_i, [_vp, ctypes.POINTER(_d), _vp]),
    "pw_batch_get_mode": (_i, [_vp, ctypes.POINTER(_i)]),
    "pw_batch_autotune": (_i, [_vp, ctypes.POINTER(_i)]),
    "pw_batch_inject_stall": (_i, [_vp, _i, _d]),
    "pw_batch_destroy": (_i, [_vp]),
}.items():
    SIGNATURES[_name] = (_res, _args)
    _f = getattr(LIB, _name)
    _f.restype = _res
    _f.argtypes = _args


class pw_adjoint(ctypes.Structure):
    """Mirror of the C struct pw_adjoint (include/pywolf_gb.h)."""
    _fields_ = [("dev_dS", _vp), ("dev_dmu", _vp), ("iP", _i), ("jP", _i), ("dev_S", _vp), ("dev_mu", _vp),
                ("sigma_S_m", _d), ("sigma_mu_m", _d), ("amplitude", _d), ("dev_amask", _vp),
                ("dev_grad3", _vp), ("dev_grad_amask", _vp), ("grad_W0", _i)]


_AP = ctypes.POINTER(pw_adjoint)
for _name, (_res, _args) in {
    "pw_propagate_fresnel_adjoint": (_i, [_vp, _d, _AP]),
    "pw_propagate_farfield_adjoint": (_i, [_vp, _d, _AP]),
}.items():
    SIGNATURES[_name] = (_res, _args)
    _f = getattr(LIB, _name)
    _f.restype = _res
    _f.argtypes = _args


class PwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (LIB.pw_status_string(status).decode(), msg))
        self.status = status


def _check(status):
    if status != PW_OK:
        raise PwError(status, LIB.pw_last_error().decode())
    return status


def pw_last_error():
    return LIB.pw_last_error().decode()


def pw_supported_n(N):
    return bool(LIB.pw_supported_n(N))


def pw_csda_bytes(N):
    return int(LIB.pw_csda_bytes(N))


def pw_csd_create(N, dxi_m, lambda_m, dev_W, W_bytes, dev_work, work_bytes, stream=0):
    h = _vp()
    _check(LIB.pw_csd_create(ctypes.byref(h), N, dxi_m, lambda_m, dev_W, W_bytes, dev_work, work_bytes, stream))
    return h.value


def pw_csd_destroy(h):
    _check(LIB.pw_csd_destroy(h))


def pw_csd_set_stream(h, stream):
    _check(LIB.pw_csd_set_stream(h, stream))


def pw_csd_check(h):
    _check(LIB.pw_csd_check(h))


def pw_csd_reset(h, dxi_m):
    _check(LIB.pw_csd_reset(h, dxi_m))


PW_DFT_AUTO, PW_DFT_FP32, PW_DFT_TC_BF16X3 = 0, 1, 2
PW_MAX_N = 512


def pw_csd_inject_stall(h, chunk):
    _check(LIB.pw_csd_inject_stall(h, chunk))


def pw_csd_set_padding(h, Nz):
    _check(LIB.pw_csd_set_padding(h, Nz))


def pw_csd_get_padding(h):
    n = _i()
    _check(LIB.pw_csd_get_padding(h, ctypes.byref(n)))
    return n.value


def pw_csd_set_dft_mode(h, mode):
    _check(LIB.pw_csd_set_dft_mode(h, mode))


def pw_csd_get_dft_mode(h):
    m = _i()
    _check(LIB.pw_csd_get_dft_mode(h, ctypes.byref(m)))
    return m.value


def pw_csd_enable_timing(h, max_props):
    _check(LIB.pw_csd_enable_timing(h, max_props))


def pw_csd_pass_times(h):
    """Returns (ms_first_pass_total, ms_second_pass_total, count)."""
    a, b, n = _d(), _d(), _i()
    _check(LIB.pw_csd_pass_times(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
    return a.value, b.value, n.value


def pw_csd_pass_times3(h):
    """(ms of the first pass, of the second, of the third (0 for two-pass engines), count)."""
    a, b, c, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(LIB.pw_csd_pass_times3(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(n)))
    return a.value, b.value, c.value, n.value


def pw_source_gsm(h, sigma_S_m, sigma_mu_m, amplitude=1.0):
    _check(LIB.pw_source_gsm(h, sigma_S_m, sigma_mu_m, amplitude))


def pw_source_aperture(h, radius_m):
    _check(LIB.pw_source_aperture(h, radius_m))


def pw_source_lens(h, focal_m):
    _check(LIB.pw_source_lens(h, focal_m))


def pw_source_mask(h, dev_mask):
    _check(LIB.pw_source_mask(h, dev_mask))


def pw_source_array(h, dev_W0, hermitian=True):
    _check(LIB.pw_source_array(h, dev_W0, 1 if hermitian else 0))


def pw_source_diagonal(h, dev_d, weight=1.0):
    _check(LIB.pw_source_diagonal(h, dev_d, weight))


def pw_gsm_gradient(h, sigma_S_m, sigma_mu_m, amplitude, dev_amask, lambda_m, z_m, farfield, dev_grad3,
                    dev_grad_mask):
    _check(LIB.pw_gsm_gradient(h, sigma_S_m, sigma_mu_m, amplitude, dev_amask, lambda_m, z_m, 1 if farfield else 0,
                               dev_grad3, dev_grad_mask))


def pw_propagate_fresnel(h, z_m):
    _check(LIB.pw_propagate_fresnel(h, z_m))


def pw_propagate_farfield(h, z_m):
    _check(LIB.pw_propagate_farfield(h, z_m))


def pw_get_sampling(h):
    d = _d()
    _check(LIB.pw_get_sampling(h, ctypes.byref(d)))
    return d.value


def pw_spectral_density(h, dev_S):
    _check(LIB.pw_spectral_density(h, dev_S))


def pw_degree_of_coherence(h, iP, jP, dev_mu):
    _check(LIB.pw_degree_of_coherence(h, iP, jP, dev_mu))


def pw_propagate_gsm_fresnel_noalloc(N, dxi_m, lambda_m, z_m, sigma_S_m, sigma_mu_m, amplitude, aperture_m,
                                     lens_f_m, dev_mask, dev_W_out, W_bytes, dev_S_out, stream=0):
    """Allocation-free propagation (N <= 32) into caller buffers; see include/pywolf_gb.h."""
    _check(LIB.pw_propagate_gsm_fresnel_noalloc(N, dxi_m, lambda_m, z_m, sigma_S_m, sigma_mu_m, amplitude,
                                                 aperture_m, lens_f_m, dev_mask, dev_W_out, W_bytes, dev_S_out,
                                                 stream))


def _instances(insts):
    arr = (pw_instance * len(insts))(*insts)
    return arr


def pw_batch_workspace_bytes(insts, pool):
    arr = _instances(insts)
    return int(LIB.pw_batch_workspace_bytes(arr, len(insts), pool))


def pw_batch_create(insts, pool, dev_ws, ws_bytes, stream=0):
    arr = _instances(insts)
    b = _vp()
    _check(LIB.pw_batch_create(ctypes.byref(b), arr, len(insts), pool, dev_ws, ws_bytes, stream))
    return b.value


def pw_batch_run(b):
    _check(LIB.pw_batch_run(b))


def pw_batch_check(b):
    _check(LIB.pw_batch_check(b))


def pw_batch_set_chunk(b, chunk):
    _check(LIB.pw_batch_set_chunk(b, chunk))


def pw_batch_get_chunk(b):
    c = _i()
    _check(LIB.pw_batch_get_chunk(b, ctypes.byref(c)))
    return c.value


PW_BATCH_PERSISTENT, PW_BATCH_SEQUENCED = 0, 1


def pw_batch_spectral_sum(b, weights, dev_I):
    w = (_d * len(weights))(*[float(x) for x in weights])
    _check(LIB.pw_batch_spectral_sum(b, w, dev_I))


def pw_batch_set_mode(b, mode):
    _check(LIB.pw_batch_set_mode(b, mode))


def pw_batch_get_mode(b):
    m = ctypes.c_int()
    _check(LIB.pw_batch_get_mode(b, ctypes.byref(m)))
    return m.value


def pw_batch_autotune(b):
    c = _i()
    _check(LIB.pw_batch_autotune(b, ctypes.byref(c)))
    return c.value


def pw_batch_inject_stall(b, instance, wait_s):
    _check(LIB.pw_batch_inject_stall(b, instance, wait_s))


def pw_batch_destroy(b):
    _check(LIB.pw_batch_destroy(b))


def pw_propagate_fresnel_adjoint(h, z_m, adj):
    """adj: a pw_adjoint (device addresses as integers, 0 for NULL)."""
    _check(LIB.pw_propagate_fresnel_adjoint(h, z_m, ctypes.byref(adj)))


def pw_propagate_farfield_adjoint(h, z_m, adj):
    _check(LIB.pw_propagate_farfield_adjoint(h, z_m, ctypes.byref(adj)))
