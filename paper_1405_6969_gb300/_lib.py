"""ctypes view of the C ABI declared in ``include/erpp.h``.

Argument marshalling only: every computation happens in ``liberpp.so``.
Loading fails loudly when the library has not been built; there is no
fallback implementation.
"""

from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liberpp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "erpp.h")

FP32 = 1 << 0
FP64 = 1 << 1
NORMALIZE = 1 << 2
SELF_REMOVAL = 1 << 3
KAHAN = 1 << 4
PIC = 1 << 5
POINT_GATHER = 1 << 6
LAG = 1 << 7
FULL_FORCE = 1 << 8

SCATTER_MODES = {"merge": 0, "cluster": 1, "xclip": 2}

STATUS = {0: "ERPP_OK", 1: "ERPP_EINVAL", 2: "ERPP_ENOMEM", 3: "ERPP_ECUDA",
          4: "ERPP_ERANGE", 5: "ERPP_EBOUNDS", 6: "ERPP_ETIMEOUT", 7: "ERPP_ESTATE"}


class ErppError(RuntimeError):
    def __init__(self, status, where):
        self.status = int(status)
        super().__init__(f"{where}: {STATUS.get(self.status, self.status)} "
                         f"({_describe(self.status)})")


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
        ("nu", ctypes.c_double), ("rho_f", ctypes.c_double),
        ("eps_R", ctypes.c_double), ("cutoff", ctypes.c_double),
        ("dt", ctypes.c_double), ("gravity", ctypes.c_double * 3),
        ("shear_rate", ctypes.c_double),
    ]


_dp = ctypes.POINTER(ctypes.c_double)
_dp3 = _dp * 3


class Particles(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("x", _dp3), ("v", _dp3), ("x_prev", _dp3), ("D", _dp3),
        ("radius", _dp), ("rho_p", _dp),
    ]


class BoxDesc(ctypes.Structure):
    _fields_ = [("params", Params), ("u", ctypes.c_void_p), ("particles", Particles),
                ("S", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_st = ctypes.c_int
_SIGS = {
    "erpp_init": (_st, [ctypes.POINTER(Params), ctypes.POINTER(_vp)]),
    "erpp_destroy": (_st, [_vp]),
    "erpp_status_string": (ctypes.c_char_p, [_st]),
    "erpp_interpolate": (_st, [_vp, _vp, _i64, _dp3, _dp3, _vp]),
    "erpp_particle_advance": (_st, [_vp, _dp3, ctypes.POINTER(Particles), ctypes.c_int, _vp]),
    "erpp_scatter_source": (_st, [_vp, _i64, _dp3, _dp3, _vp, _vp]),
    "erpp_step": (_st, [_vp, _vp, ctypes.POINTER(Particles), _vp, ctypes.c_int, _vp]),
    "erpp_step_host": (_st, [_vp, _vp, ctypes.POINTER(Particles), _vp, ctypes.c_int, _vp]),
    "erpp_step_host_wait": (_st, [_vp, _vp]),
    "erpp_momentum": (_st, [_vp, _vp, _i64, _dp3, _dp3, _dp, _vp]),
    "erpp_check": (_st, [_vp, _vp]),
    "erpp_debug_windows": (_st, [_vp, _i64, _dp3, _vp, _vp, _vp]),
    "erpp_debug_set_wait": (_st, [_vp, _i64, ctypes.c_int32]),
    "erpp_interpolate_noalloc": (_st, [ctypes.POINTER(Params), _vp, _i64, _dp3, _dp3, _vp]),
    "erpp_profile_enable": (_st, [_vp, ctypes.c_int]),
    "erpp_profile_read": (_st, [_vp, _dp, ctypes.POINTER(ctypes.c_int64)]),
    "erpp_shared_add_rate": (_st, [ctypes.c_int32, _dp]),
    "erpp_batch_init": (_st, [ctypes.c_int32, ctypes.POINTER(BoxDesc), ctypes.POINTER(_vp)]),
    "erpp_step_batched": (_st, [_vp, ctypes.c_int, ctypes.c_int, _vp]),
    "erpp_batch_check": (_st, [_vp, _vp]),
    "erpp_batch_set_tiling": (_st, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32]),
    "erpp_batch_destroy": (_st, [_vp]),
    "erpp_batch_set_form": (_st, [_vp, ctypes.c_int32]),
    "erpp_set_tiling": (_st, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "erpp_get_tiling": (_st, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "erpp_set_scatter_mode": (_st, [_vp, ctypes.c_int32]),
    "erpp_last_step_launches": (_st, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "erpp_batch_last_step_launches": (_st, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "erpp_batch_get_tiling": (_st, [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "erpp_fluid_init": (_st, [ctypes.POINTER(Params), ctypes.POINTER(_vp)]),
    "erpp_fluid_stokes_step": (_st, [_vp, _vp, _vp, _vp]),
    "erpp_fluid_destroy": (_st, [_vp]),
    "erpp_scatter_backward": (_st, [_vp, _i64, _dp3, _dp3, _vp, ctypes.POINTER(_dp3),
                                    ctypes.POINTER(_dp3), _vp]),
    "erpp_gather_backward": (_st, [_vp, _i64, _dp3, _vp, _dp3, _vp, ctypes.POINTER(_dp3),
                                   _vp]),
}


def header_symbols(path=HEADER):
    """Names of the functions declared in include/erpp.h."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(erpp_\w+)\s*\(",
                                 text, flags=re.M)))


def load():
    """Load liberpp.so (raises if it is missing: build it first)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} not found: build the CUDA library with "
                    "`python -m paper_1405_6969_gb300.build`")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _describe(status):
    try:
        return load().erpp_status_string(int(status)).decode()
    except Exception:  # pragma: no cover
        return "?"


def check(status, where):
    if status != 0:
        raise ErppError(status, where)
