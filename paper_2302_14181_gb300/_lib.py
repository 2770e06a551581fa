"""ctypes declarations of libtevo.so (C ABI in include/tevo.h)."""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtevo.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "tevo.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2302_14181_gb300/_build.py` or __graft_entry__.build() "
                      "(there is no fallback implementation)")

lib = ctypes.CDLL(LIB_PATH)

FP64, TF32, TF32X3, BF16X3 = 0, 1, 2, 3
TC_ONLY = 0x100
OZAKI = 0x200
TWO_SITE = 0x400


def OZAKI_SLICES(g):
    """TEVO_OZAKI_SLICES(g): the Ozaki-scheme fp64 contractions with g digit slices."""
    return OZAKI | (int(g) << 12)


MPO_PLAIN, MPO_EXACT, MPO_EXTENDED, MPO_FULL = 0, 1, 2, 3
PROF_GEMM64, PROF_GEMMTC, PROF_QR, PROF_FORMQ, PROF_GEMMOZ, PROF_OZSPLIT = 0, 1, 2, 3, 4, 5


class tevo_ctx(ctypes.c_void_p):
    pass


class tevo_mpo(ctypes.c_void_p):
    pass


class tevo_mps(ctypes.c_void_p):
    pass


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_i, _d, _p, _pd = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
_pi = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "tevo_ctx_create": [_p, ctypes.POINTER(tevo_ctx)],
    "tevo_ctx_destroy": [tevo_ctx],
    "tevo_ctx_set_allocator": [tevo_ctx, ALLOC_FN, FREE_FN, _p],
    "tevo_ctx_set_stream": [tevo_ctx, _p],
    "tevo_launch_count": [tevo_ctx, ctypes.POINTER(ctypes.c_longlong), _i],
    "mpo_build": [tevo_ctx, _i, _i, _i, _pd, _pd, _pd, _pd, _i, _d, _d, _i, ctypes.POINTER(tevo_mpo)],
    "mpo_build_host": [_i, _i, _i, _pd, _pd, _pd, _pd, _i, _d, _d, _i, _pi, _pd,
                       ctypes.POINTER(ctypes.c_size_t)],
    "mpo_bond_dims": [tevo_mpo, _pi],
    "mpo_get_site": [tevo_mpo, _i, _pd],
    "mpo_destroy": [tevo_mpo],
    "mps_init": [tevo_ctx, _i, _i, _i, _pd, ctypes.POINTER(tevo_mps)],
    "mps_bond_dims": [tevo_mps, _pi],
    "mps_get_site": [tevo_mps, _i, _pd],
    "mps_set_site": [tevo_mps, _i, _pd],
    "mps_log_norm": [tevo_mps, _pd],
    "mps_destroy": [tevo_mps],
    "evolve_step": [tevo_mps, tevo_mpo, _d, _d, _i, _i, _i],
    "evolve_step_batched": [ctypes.POINTER(tevo_mps), ctypes.POINTER(tevo_mpo), _i, _i, _i],
    "measure_local": [tevo_mps, _i, _pd, _pd],
    "mps_overlap": [tevo_mps, tevo_mps, _pd, _pd],
    "tevo_gemm": [tevo_ctx, _i, _i, _i, _i, _p, _p, _p],
    "tevo_gemm_noalloc": [tevo_ctx, _i, _i, _i, _i, _p, _p, _p],
    "tevo_wait_selftest": [tevo_ctx, _d, _pi],
    "tevo_prof_enable": [tevo_ctx, _i],
    "tevo_prof_read": [tevo_ctx, _i, _pd, ctypes.POINTER(ctypes.c_longlong), _pd, _pd],
}

for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
lib.tevo_strerror.argtypes = [ctypes.c_int]
lib.tevo_strerror.restype = ctypes.c_char_p


class TevoError(RuntimeError):
    def __init__(self, code):
        self.code = code
        super().__init__(f"libtevo error {code}: {lib.tevo_strerror(code).decode()}")


def check(code):
    if code != 0:
        raise TevoError(code)


def declared_symbols():
    """Function names declared in include/tevo.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", txt, flags=re.M)))
