"""ctypes declarations of the C ABI in include/adg.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

ADG_OK, ADG_EINVAL, ADG_ENOMEM, ADG_ECUDA, ADG_ENONFINITE, ADG_ETIMEOUT, ADG_ESTATE = \
    0, -1, -2, -3, -4, -5, -6
ADG_ADVECTION, ADG_BURGERS, ADG_EULER = 0, 1, 2
ADG_UPWIND, ADG_LLF = 0, 1
ADG_RK1, ADG_RK2, ADG_SSPRK3, ADG_LSRK3, ADG_LSRK4 = 1, 2, 3, 4, 5
ADG_SYNC, ADG_ASYNC, ADG_ASYNC_AT = 0, 1, 2
ADG_VARIANT_AUTO, ADG_VARIANT_STAGED, ADG_VARIANT_COMPOSED, ADG_VARIANT_COMPOSED_FIXED = 0, 1, 2, 3

STATUS_NAMES = {0: "ADG_OK", -1: "ADG_EINVAL", -2: "ADG_ENOMEM", -3: "ADG_ECUDA",
                -4: "ADG_ENONFINITE", -5: "ADG_ETIMEOUT", -6: "ADG_ESTATE"}

# Every entry point declared in include/adg.h.
EXPORTS = [
    "adg_config_default", "adg_init", "adg_batch_init", "adg_step", "adg_run",
    "adg_get_state", "adg_get_dt", "adg_get_variant", "adg_grad", "adg_integral", "adg_check_finite",
    "adg_delay_table", "adg_eval_modes", "adg_lgl_nodes", "adg_last_error", "adg_destroy",
    "adg_integral_noalloc", "adg_misfit", "adg_comm_stats", "adg_get_fixed_basis",
    "adg_init_host", "adg_get_state_host",
]


class AdgConfig(C.Structure):
    _fields_ = [
        ("pde", C.c_int32), ("flux", C.c_int32), ("rk", C.c_int32),
        ("K", C.c_int32), ("p", C.c_int32), ("P", C.c_int32),
        ("x0", C.c_double), ("x1", C.c_double), ("a", C.c_double),
        ("cfl", C.c_double), ("dt", C.c_double),
        ("mode", C.c_int32), ("L", C.c_int32), ("at_order", C.c_int32),
        ("seed", C.c_uint64), ("probs", C.POINTER(C.c_double)),
        ("delay_table", C.POINTER(C.c_uint8)), ("table_steps", C.c_int64),
        ("variant", C.c_int32), ("caa_sync", C.c_int32), ("nu", C.c_double),
        ("limiter", C.c_int32), ("tvb_m", C.c_double), ("ept", C.c_int32),
    ]


class AdgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(require: bool = True):
    """Load libadg.so (built in-tree by __graft_entry__.build()). Fails loudly if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(path)
    vp, dp, i32, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_int64
    cfgp = C.POINTER(AdgConfig)
    sig = {
        "adg_config_default": (None, [cfgp]),
        "adg_init": (C.c_int, [cfgp, vp, vp, C.POINTER(vp)]),
        "adg_init_host": (C.c_int, [cfgp, vp, vp, C.POINTER(vp)]),
        "adg_batch_init": (C.c_int, [cfgp, C.POINTER(vp), i32, vp, C.POINTER(vp)]),
        "adg_step": (C.c_int, [vp, i64]),
        "adg_run": (C.c_int, [vp, C.c_double]),
        "adg_get_state": (C.c_int, [vp, i32, vp, C.POINTER(i64)]),
        "adg_get_state_host": (C.c_int, [vp, i32, vp, C.POINTER(i64)]),
        "adg_get_dt": (C.c_int, [vp, i32, dp]),
        "adg_get_variant": (C.c_int, [vp, i32, C.POINTER(i32), C.POINTER(i32)]),
        "adg_get_fixed_basis": (C.c_int, [vp, i32, C.POINTER(i32)]),
        "adg_grad": (C.c_int, [vp, vp, i64, i32, vp, dp]),
        "adg_integral": (C.c_int, [vp, i32, dp]),
        "adg_check_finite": (C.c_int, [vp]),
        "adg_delay_table": (C.c_int, [cfgp, i64, i64, C.POINTER(C.c_uint8)]),
        "adg_eval_modes": (C.c_int, [cfgp, i32, dp, dp, dp, C.c_double, vp, vp]),
        "adg_lgl_nodes": (C.c_int, [i32, dp, dp]),
        "adg_last_error": (C.c_char_p, [vp]),
        "adg_destroy": (None, [vp]),
        "adg_integral_noalloc": (C.c_int, [i32, i32, C.c_double, vp, vp, vp]),
        "adg_misfit": (C.c_int, [vp, i32, vp, dp]),
        "adg_comm_stats": (C.c_int, [vp, i32, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(code: int, ctx=None):
    if code != ADG_OK:
        msg = load().adg_last_error(ctx)
        raise AdgError(code, msg.decode() if msg else "")
    return code
