"""ctypes declarations of include/mrip.h (argument marshalling only)."""
import contextlib
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmrip.so")

MRIP_MM1, MRIP_TANDEM3, MRIP_FOREST_FIRE, MRIP_WALK_L1_EXIT = 1, 2, 3, 4
(MRIP_MAP_AUTO, MRIP_MAP_THREAD, MRIP_MAP_WARP_1LANE, MRIP_MAP_WARP_COOP, MRIP_MAP_CTA,
 MRIP_MAP_PERSISTENT) = range(6)
STATUS_NAMES = {0: "MRIP_OK", 1: "MRIP_EINVAL", 2: "MRIP_ENOMEM", 3: "MRIP_ECUDA",
                4: "MRIP_ESTEPCAP", 5: "MRIP_ESTATE", 6: "MRIP_EUNSUPPORTED"}


class MripError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, code), msg))
        self.code = code


class MripLibraryMissing(ImportError):
    pass


class mrip_stat(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("mean", ctypes.c_double), ("var", ctypes.c_double),
                ("half_width", ctypes.c_double), ("t_crit", ctypes.c_double)]


class mrip_cv_stat(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("beta", ctypes.c_double),
                ("mean", ctypes.c_double), ("var", ctypes.c_double),
                ("half_width", ctypes.c_double), ("t_crit", ctypes.c_double)]


class mrip_mm1_params(ctypes.Structure):
    _fields_ = [("n_clients", ctypes.c_int64)]


class mrip_tandem3_params(ctypes.Structure):
    _fields_ = [("n_clients", ctypes.c_int64), ("window", ctypes.c_int64)]


class mrip_forest_fire_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("n_steps", ctypes.c_int32), ("density", ctypes.c_double),
                ("window", ctypes.c_int32)]


class mrip_walk_params(ctypes.Structure):
    _fields_ = [("max_steps", ctypes.c_int64)]


class mrip_train_params(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int64), ("epochs", ctypes.c_int32), ("patience", ctypes.c_int32),
                ("max_steps", ctypes.c_int64), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("order_seed", ctypes.c_uint64),
                ("epoch0", ctypes.c_int32), ("pad", ctypes.c_int32)]


class mrip_cv_params(ctypes.Structure):
    _fields_ = [("train_frac", ctypes.c_double), ("val_frac", ctypes.c_double),
                ("epochs", ctypes.c_int32), ("patience", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("gate", ctypes.c_int32), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("m_ctrl", ctypes.c_int64),
                ("conf", ctypes.c_double), ("net_seed", ctypes.c_uint64)]


class mrip_cv_report(ctypes.Structure):
    _fields_ = [("declined", ctypes.c_int32), ("epochs_run", ctypes.c_int32),
                ("best_epoch", ctypes.c_int32), ("n_val", ctypes.c_int32),
                ("m_ctrl", ctypes.c_int64), ("train_loss", ctypes.c_float),
                ("val_loss", ctypes.c_float), ("val_rho2", ctypes.c_double),
                ("var_ratio", ctypes.c_double), ("ms_simulate", ctypes.c_double),
                ("ms_train", ctypes.c_double), ("ms_control", ctypes.c_double),
                ("ms_infer", ctypes.c_double), ("ms_estimate", ctypes.c_double)]


_P = ctypes.c_void_p
_I32, _I64, _U32, _U64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
_D, _F, _SZ, _INT = ctypes.c_double, ctypes.c_float, ctypes.c_size_t, ctypes.c_int

SIGNATURES = {
    "mrip_create_model": (_INT, [_INT, _P, _SZ, _P]),
    "mrip_set_stream": (_INT, [_P, _P]),
    "mrip_run": (_INT, [_P, _P, _I32, _I64, _U64]),
    "mrip_run_range": (_INT, [_P, _P, _I32, _I64, _I64, _U64]),
    "mrip_moments": (_INT, [_P, _P]),
    "mrip_run_device": (_INT, [_P, _P, _I32, _I64, _U64]),
    "mrip_stats": (_INT, [_P, _D, _P]),
    "mrip_outputs": (_INT, [_P, _INT, _P, _SZ, _INT]),
    "mrip_output_bytes": (_INT, [_P, _INT, _P]),
    "mrip_set_plan": (_INT, [_P, ctypes.c_char_p]),
    "mrip_get_plan": (_INT, [_P, ctypes.c_char_p, _SZ]),
    "mrip_autotune": (_INT, [_P, _P, _I32, _I64, _U64, _INT, ctypes.c_char_p]),
    "mrip_run_cv": (_INT, [_P, _P, _I32, _I64, _U64, _P, _P, _P, _P]),
    "mrip_cv_network": (_INT, [_P, _P, _P]),
    "mrip_destroy": (None, [_P]),
    "mrip_last_error": (ctypes.c_char_p, []),
    "mrip_philox": (_INT, [_P, _P, _I64, _P, _P]),
    "mrip_expo": (_INT, [_P, _P, _P, _I64, _P, _P, _P]),
    "mrip_mm1_simulate": (_INT, [_P, _I32, _I64, _I64, _I64, _U64, _INT, _P, _P, _P, _P]),
    "mrip_tandem3_simulate": (_INT, [_P, _I32, _I64, _I64, _I64, _I64, _U64, _U32, _INT, _P, _P,
                                     _P]),
    "mrip_forest_fire_simulate": (_INT, [_P, _I32, _I64, _I64, _I32, _I32, _D, _U64, _P, _P, _P,
                                         _P, _P]),
    "mrip_forest_fire_skip_simulate": (_INT, [_P, _I32, _I64, _I64, _I32, _I32, _D, _U64, _P, _P,
                                              _P, _P, _P]),
    "mrip_walk_simulate": (_INT, [_P, _I32, _I64, _I64, _U64, _I64, _INT, _I32, _I32, _I32, _P,
                                  _P]),
    "mrip_walk_simulate_noalloc": (_INT, [_P, _I32, _I64, _I64, _U64, _I64, _INT, _I32, _I32, _I32,
                                          _P, _P]),
    "mrip_area_walk_simulate": (_INT, [_I64, _I64, _I32, _U64, _INT, _P, _P, _P]),
    "mrip_pi_simulate": (_INT, [_I64, _I64, _I64, _U64, _P, _P]),
    "mrip_check_device_flags": (_INT, []),
    "mrip_debug_checks": (_INT, [_P, _P]),
    "mrip_debug_selftest": (_INT, []),
    "mrip_probe_mul_wide": (_INT, [_P, _P]),
    "mrip_stats_reduce": (_INT, [_P, _I32, _I64, _P, _P]),
    "mrip_stats_reduce_i64": (_INT, [_P, _I32, _I64, _P, _P]),
    "mrip_stats_finalize": (_INT, [_P, _I32, _D, _P]),
    "mrip_t_crit": (_INT, [_D, _I64, _P]),
    "mrip_stats_merge": (_INT, [_P, _I32, _I32, _P]),
    "mrip_mlp_param_count": (_I64, [_I32]),
    "mrip_mlp_init": (_INT, [_I32, _U64, _P, _P]),
    "mrip_mlp_forward": (_INT, [_P, _I32, _P, _I64, _P, _P]),
    "mrip_mlp_loss_grad": (_INT, [_P, _I32, _P, _P, _I64, _P, _I64, _P, _P, _P]),
    "mrip_adam_step": (_INT, [_P, _P, _P, _P, _I64, _I64, _F, _F, _F, _F, _P]),
    "mrip_mlp_train": (_INT, [_I32, _P, _P, _I64, _P, _P, _I64, _P, _P, _P, _P, _P, _P, _P, _P,
                              _P, _P, _P]),
    "mrip_cv_reduce": (_INT, [_P, _P, _I64, _P, _I64, _I32, _P, _P]),
}

_lib = None


def library_path():
    return LIB_PATH


def load_library(path):
    """Load an engine library (e.g. the debug variant) with the ABI's
    signatures, without making it the binding's library."""
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


def lib():
    """The loaded engine library; raises MripLibraryMissing if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise MripLibraryMissing(
            "libmrip.so not found at %s: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    _lib = load_library(LIB_PATH)
    return _lib


@contextlib.contextmanager
def using_library(L):
    """Route the binding's calls to the library L for the duration."""
    global _lib
    saved = lib()
    _lib = L
    try:
        yield L
    finally:
        _lib = saved


def check(code):
    if code != 0:
        raise MripError(code, lib().mrip_last_error().decode())
