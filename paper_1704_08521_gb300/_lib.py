"""ctypes loader of libfvns.so: signatures of every exported entry point."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfvns.so")

STATUS_NAMES = {0: "FV_OK", 1: "FV_EINVAL", 2: "FV_ENOMEM", 3: "FV_ECUDA", 4: "FV_ENOCONV",
                5: "FV_ENAN", 6: "FV_ETIMEOUT"}


class FvError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
    return ctypes.CDLL(LIB_PATH)


lib = _load()

_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_SIGS = {
    "fv_grid_create": (_I, [_I, _I, _I, _I, _D, _D, _P, ctypes.POINTER(_P)]),
    "fv_grid_set_re": (_I, [_P, _D]),
    "fv_grid_set_stream": (_I, [_P, _P]),
    "fv_grid_get_info": (_I, [_P, _P]),
    "fv_grid_set_base": (_I, [_P, _P]),
    "fv_grid_destroy": (None, [_P]),
    "fv_last_error": (ctypes.c_char_p, []),
    "ns_residual": (_I, [_P, _P, _P, _P, _P]),
    "ns_jacvec": (_I, [_P, _P, _P, _P, _I]),
    "simple_krylov_solve": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "newton_steady": (_I, [_P, _P, _P, _P, _P]),
    "arnoldi_leading": (_I, [_P, _P, _P, _I, _I, _P, _P, _P, _P, _P]),
    "fv_dot_w": (_I, [_P, _P, _P, _P]),
    "fv_plane_projection": (_I, [_P, _P, _I, _P, _P]),
    "ns_divergence": (_I, [_P, _P, _P]),
    "fv_unet_create": (_I, [ctypes.c_uint64, _P, ctypes.POINTER(_P)]),
    "fv_unet_destroy": (None, [_P]),
    "fv_unet_param_count": (_I, [_P]),
    "fv_unet_set_stream": (_I, [_P, _P]),
    "fv_unet_set_params": (_I, [_P, _P]),
    "fv_unet_get_params": (_I, [_P, _P, _P]),
    "fv_unet_forward": (_I, [_P, _I, _I, _I, _P, _P]),
    "fv_unet_backward": (_I, [_P, _P, ctypes.POINTER(_D)]),
    "fv_unet_adam": (_I, [_P, ctypes.c_float]),
    "fv_unet_guess": (_I, [_P, _P, _P, _P]),
    "fv_unet_train_step": (_I, [_P, _P, _P, _P, ctypes.c_float, ctypes.POINTER(_D)]),
    "simple_krylov_solve_guess": (_I, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "fv_batch_create": (_I, [_I, _P, _P, ctypes.POINTER(_P)]),
    "fv_batch_destroy": (None, [_P]),
    "fv_batch_krylov": (_I, [_P, _P, _P, _P, _D, _D, _P]),
    "fv_batch_autotune": (_I, [_P, _P, _P]),
    "fv_batch_set_tile": (_I, [_P, _I]),
    "fv_critical_re": (_I, [_P, _P, _P, _P, _D, _D, _P, _P, _P, _P]),
    "fv_pressure_solve": (_I, [_P, _P, _P, _I]),
    "fv_pressure_solve_noalloc": (_I, [_I, _I, _I, _I, _P, _P, _P]),
    "fv_pressure_solve_mg": (_I, [_P, _P, _P, _P, _P, _P]),
    "fv_host_mg_axis": (_I, [_I, _I, _I, _P, _P, _P, _P]),
    "fv_host_mg_levels": (_I, [_I, _I, _I]),
    "fv_profile_enable": (_I, [_P, _I]),
    "fv_profile_read": (_I, [_P, _P, _P]),
    "fv_launch_count": (ctypes.c_int64, []),
    "fv_debug_inject_status": (_I, [_P, _I]),
    "fv_bench_kernel": (_I, [_P, _I, _I, _P]),
    "fv_host_hess_eigenvalues": (_I, [_I, _P, _P, _P]),
    "fv_host_shift_steps": (_I, [_I, _P, _P, _I, _P, _P]),
    "fv_host_ff_convert": (_I, [ctypes.c_int64, _P, _P, _P, _P, _P]),
    "fv_host_ff_arith": (_I, [ctypes.c_int64, _P, _P, _P, _P]),
    "fv_host_ff_dot": (_I, [ctypes.c_int64, _P, _P, _P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def check(status, where):
    if status != 0:
        msg = lib.fv_last_error()
        raise FvError(status, where, msg.decode() if msg else "")
