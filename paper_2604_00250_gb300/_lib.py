"""ctypes declarations of the C-ABI in include/prism.h (argument marshalling only)."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libprism_gb300.so")

PRISM_OK = 0
STATUS_NAMES = {1: "E_INVALID_ARG", 2: "E_SHAPE", 3: "E_CUDA", 4: "E_OOM", 5: "E_NONFINITE",
                6: "E_TIMEOUT", 7: "E_STATE"}
MEM_HOST, MEM_DEVICE = 0, 1
LOSS_MSE, LOSS_NLL = 0, 1
OPT_ADAM, OPT_RPROP = 0, 1

EXPORTS = [
    "prism_default_options", "prism_fit_init", "prism_step", "prism_sync", "prism_info",
    "prism_get_params", "prism_set_params", "prism_group_layout", "prism_get_groups",
    "prism_set_groups", "prism_get_loss", "prism_forward", "prism_backward", "prism_state_size",
    "prism_get_state", "prism_set_state", "prism_fit", "prism_fit_destroy", "prism_last_error",
    "prism_profile", "prism_grad_noalloc", "prism_microbench", "prism_get_fibers",
    "prism_fit_init_slabs", "prism_stitch_slabs", "prism_get_shape", "prism_wait_probe",
]


class PrismError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Volume(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("n_meas", ctypes.c_int32), ("mem", ctypes.c_int32), ("norm_count", ctypes.c_int32),
        ("mask", ctypes.c_void_p), ("signal", ctypes.c_void_p), ("bvals", ctypes.c_void_p),
        ("bvecs", ctypes.c_void_p), ("init", ctypes.c_void_p),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32), ("loss", ctypes.c_int32), ("calibration", ctypes.c_int32),
        ("patch_dim", ctypes.c_int32),
        ("lam_rep", ctypes.c_float), ("lam_sparse", ctypes.c_float), ("tau", ctypes.c_float),
        ("lam_sp", ctypes.c_float), ("huber_delta", ctypes.c_float), ("lam_dir", ctypes.c_float),
        ("lam_orphan", ctypes.c_float), ("s_orphan", ctypes.c_float), ("lam_order", ctypes.c_float),
        ("connectivity", ctypes.c_int32),
        ("w_alpha", ctypes.c_float), ("w_beta", ctypes.c_float), ("w_blr", ctypes.c_float),
        ("w_tv", ctypes.c_float), ("tv_eps", ctypes.c_float), ("sigma_init", ctypes.c_float),
        ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
        ("eps", ctypes.c_float),
        ("optimizer", ctypes.c_int32), ("rprop_eta_minus", ctypes.c_float), ("rprop_eta_plus", ctypes.c_float),
        ("rprop_step_min", ctypes.c_float), ("rprop_step_max", ctypes.c_float),
        ("fused", ctypes.c_int32), ("use_graph", ctypes.c_int32),
        ("threads_per_voxel", ctypes.c_int32), ("cta_threads", ctypes.c_int32),
        ("autotune", ctypes.c_int32), ("seed", ctypes.c_int32), ("shells", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 3),
    ]


_lib = None


def load():
    """Loads the library; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2604_00250_gb300.build` "
                          "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    sig = {
        "prism_default_options": (None, [P(Options)]),
        "prism_fit_init": (ctypes.c_int, [P(Volume), i32, P(Options), vp, P(vp)]),
        "prism_step": (ctypes.c_int, [vp, i32, vp]),
        "prism_sync": (ctypes.c_int, [vp, vp]),
        "prism_wait_probe": (ctypes.c_int, [vp, i32, vp]),
        "prism_info": (ctypes.c_int, [vp, P(i64), P(i32), P(i32), P(i64), P(i64)]),
        "prism_get_shape": (ctypes.c_int, [vp, P(i32), P(i32), P(i32), P(i32)]),
        "prism_get_params": (ctypes.c_int, [vp, vp, i32, vp]),
        "prism_set_params": (ctypes.c_int, [vp, vp, i32, vp]),
        "prism_group_layout": (ctypes.c_int, [vp, vp]),
        "prism_get_groups": (ctypes.c_int, [vp, vp, i32, vp]),
        "prism_set_groups": (ctypes.c_int, [vp, vp, i32, vp]),
        "prism_get_loss": (ctypes.c_int, [vp, vp, vp, i32, P(i32)]),
        "prism_forward": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
        "prism_backward": (ctypes.c_int, [vp, vp, vp, vp]),
        "prism_state_size": (ctypes.c_int, [vp, P(i64)]),
        "prism_get_state": (ctypes.c_int, [vp, vp, i64, vp]),
        "prism_set_state": (ctypes.c_int, [vp, vp, i64, vp]),
        "prism_fit": (ctypes.c_int, [P(Volume), i32, P(Options), i32, vp, vp, i32, vp]),
        "prism_fit_destroy": (None, [vp]),
        "prism_last_error": (ctypes.c_char_p, []),
        "prism_profile": (ctypes.c_int, [vp, i32, vp, vp]),
        "prism_microbench": (ctypes.c_int, [i32, vp, vp]),
        "prism_get_fibers": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_float, i32, vp]),
        "prism_fit_init_slabs": (ctypes.c_int, [vp, i32, i32, vp, vp, vp]),
        "prism_stitch_slabs": (ctypes.c_int, [vp, vp, vp, vp, vp, i32, vp]),
        "prism_grad_noalloc": (ctypes.c_int, [vp, vp, vp, vp, i64, i32, i32, ctypes.c_float, ctypes.c_float,
                                              ctypes.c_float, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc):
    if rc != PRISM_OK:
        msg = load().prism_last_error().decode(errors="replace")
        raise PrismError(rc, msg)
