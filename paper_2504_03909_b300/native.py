"""ctypes binding of the C ABI in ``include/paillier.h`` (argument marshalling only).

The shared library is built in-tree by ``python -m paper_2504_03909_b300.build``.
Loading fails loudly when it is missing: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
# PAILLIER_B300_LIB=checked loads the bounds-checked build (build.py --checked)
LIB_PATH = os.path.join(HERE, "libpaillier_b300_checked.so" if os.environ.get("PAILLIER_B300_LIB") == "checked"
                        else "libpaillier_b300.so")
HEADER_DIR = os.path.join(os.path.dirname(HERE), "include")

PL_OK, PL_EINVAL, PL_ENOMEM, PL_ECUDA, PL_ERANGE, PL_ETIMEDOUT, PL_EBUSY, PL_EDEVICE = range(8)
STATUS_NAMES = {0: "PL_OK", 1: "PL_EINVAL", 2: "PL_ENOMEM", 3: "PL_ECUDA", 4: "PL_ERANGE",
                5: "PL_ETIMEDOUT", 6: "PL_EBUSY", 7: "PL_EDEVICE"}

_u32p = C.c_void_p
_vp = C.c_void_p
_sz = C.c_size_t
_i = C.c_int

# name -> (restype, argtypes)
SIGNATURES = {
    "paillier_keygen": (_i, [_i, C.c_uint64, C.POINTER(C.c_void_p)]),
    "paillier_key_import": (_i, [_i, _vp, _vp, C.POINTER(C.c_void_p)]),
    "paillier_key_import_public": (_i, [_i, _vp, C.POINTER(C.c_void_p)]),
    "paillier_key_export": (_i, [_vp, _vp, _vp, _vp]),
    "paillier_key_bits": (_i, [_vp]),
    "paillier_key_is_private": (_i, [_vp]),
    "paillier_key_free": (None, [_vp]),
    "paillier_encode": (_i, [_vp, _sz, _vp, _vp]),
    "paillier_decode": (_i, [_vp, _vp, _sz, _vp, _vp]),
    "paillier_encrypt": (_i, [_vp, _vp, _vp, _sz, _vp, _vp]),
    "paillier_ct_prepare": (_i, [_vp, _vp, _sz, _vp, _vp]),
    "paillier_hist_aggregate": (_i, [_vp, _vp, _sz, _vp, _i, _i, _vp, _i, _vp, _vp, _vp]),
    "paillier_hist_aggregate_per_node": (_i, [_vp, _vp, _sz, _vp, _i, _i, _vp, _i, _vp, _vp, _vp]),
    "paillier_decrypt": (_i, [_vp, _vp, _sz, _vp, _vp]),
    "paillier_decrypt_u64": (_i, [_vp, _vp, _sz, _vp, _vp]),
    "paillier_decrypt_u64_noalloc": (_i, [_vp, _vp, _sz, _vp, _vp]),
    "paillier_sync": (_i, [_vp, C.POINTER(_i)]),
    "paillier_last_error": (C.c_char_p, []),
    "paillier_test_mont_mul": (_i, [_i, _i, _vp, _vp, _vp, _sz, _vp, _vp]),
    "paillier_test_mont_sos": (_i, [_i, _i, _vp, _vp, _vp, _sz, _vp, _vp]),
    "paillier_test_bounds_report": (_i, [_i, _vp]),
    "paillier_test_schedule_ops": (_i, [_vp, _i, _i, _vp, _vp]),
    "paillier_imad_peak": (_i, [_i, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double), _vp]),
    "paillier_fp64_peak": (_i, [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double), _vp]),
    "paillier_launch_count": (C.c_ulonglong, []),
    "paillier_profile": (_i, [_i]),
    "paillier_profile_read": (_i, [C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "paillier_level_plan_create": (_i, [_vp, _sz, _i, _i, _i, C.POINTER(C.c_void_p)]),
    "paillier_level_plan_create_gh": (_i, [_vp, _sz, _i, _i, _i, C.POINTER(C.c_void_p)]),
    "paillier_level_run": (_i, [_vp, _vp, _vp, _vp, _i, _vp, _vp, _vp]),
    "paillier_level_plan_stats": (_i, [_vp, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)]),
    "paillier_level_plan_free": (None, [_vp]),
    "paillier_get_config": (_i, [_vp, _i, C.POINTER(_i), C.POINTER(_i)]),
    "paillier_set_config": (_i, [_vp, _i, _i, _i]),
    "paillier_autotune": (_i, [_vp, _i, C.c_char_p, _vp, C.POINTER(_i), C.POINTER(_i)]),
}

OP_ENCRYPT, OP_DECRYPT, OP_HIST = 0, 1, 2

class Request(C.Structure):
    """pl_request of include/paillier_serve.h."""
    _fields_ = [("key", C.c_void_p), ("d_ctm", C.c_void_p), ("gh_stride", C.c_size_t), ("M", C.c_size_t),
                ("F", C.c_int), ("K", C.c_int), ("d_bins", C.c_void_p), ("bins_stride", C.c_size_t),
                ("d_node", C.c_void_p), ("num_nodes", C.c_int), ("h_sums", C.c_void_p), ("h_counts", C.c_void_p),
                ("pack_bits", C.c_int), ("gh_bits", C.c_int), ("pack_slots", C.c_int)]


SIGNATURES.update({
    "paillier_pack_slots": (_i, [_vp, _i]),
    "paillier_pack": (_i, [_vp, _vp, _sz, _i, _vp, _vp]),
    "paillier_decrypt_packed_u64": (_i, [_vp, _vp, _sz, _i, _vp, _vp]),
    "paillier_encode_gh": (_i, [_vp, _vp, _sz, _i, _vp, _vp]),
    "paillier_encrypt_gh": (_i, [_vp, _vp, _vp, _sz, _vp, _vp]),
    "paillier_hist_aggregate_gh": (_i, [_vp, _vp, _sz, _vp, _i, _i, _vp, _i, _vp, _vp, _vp]),
    "paillier_decrypt_gh": (_i, [_vp, _vp, _sz, _i, _vp, _vp]),
    "paillier_decrypt_packed_gh": (_i, [_vp, _vp, _sz, _i, _vp, _vp]),
    "paillier_pack_n": (_i, [_vp, _vp, _sz, _i, _i, _vp, _vp]),
    "paillier_decrypt_packed_u64_n": (_i, [_vp, _vp, _sz, _i, _i, _vp, _vp]),
    "paillier_decrypt_packed_gh_n": (_i, [_vp, _vp, _sz, _i, _i, _vp, _vp]),
    "paillier_split_find": (_i, [_vp, _vp, _i, _i, _i, C.c_double, C.c_double, C.c_double, _vp, _vp, _vp, _vp]),
    "paillier_split_apply": (_i, [_vp, _sz, _i, _vp, _i, _vp, _vp, _vp, _vp]),
    "paillier_tree_decide": (_i, [_vp, _i, _i, _sz, _vp, _vp, _i, _vp, _vp]),
    "paillier_tree_route": (_i, [_vp, _sz, _vp, _i, _vp, _vp]),
    "paillier_leaf_weights": (_i, [_vp, _vp, _i, _i, _i, C.c_double, _vp, _vp]),
    "paillier_child_select": (_i, [_vp, _sz, _vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp]),
    "paillier_child_subtract": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _vp, _vp, _vp]),
    "pl_server_create": (_i, [_i, _sz, C.POINTER(C.c_void_p)]),
    "pl_server_submit": (_i, [_vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "pl_server_poll": (_i, [_vp, C.c_uint64, C.POINTER(_i), C.POINTER(C.c_double), C.POINTER(_i)]),
    "pl_server_wait": (_i, [_vp, C.c_uint64, _i, C.POINTER(_i), C.POINTER(C.c_double)]),
    "pl_server_cancel": (_i, [_vp, C.c_uint64]),
    "pl_server_request_bytes": (_i, [C.POINTER(Request), C.POINTER(_sz)]),
    "pl_server_request_plan": (_i, [C.POINTER(Request), C.POINTER(_i), C.POINTER(C.c_double)]),
    "pl_server_set_policy": (_i, [_vp, C.c_double, C.c_double, C.c_double, _i]),
    "pl_server_set_aging": (_i, [_vp, C.c_double]),
    "pl_server_policy_stats": (_i, [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(_i),
                                    C.POINTER(C.c_longlong)]),
    "pl_server_stats": (_i, [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                             C.POINTER(C.c_longlong), C.POINTER(_i), C.POINTER(_sz)]),
    "pl_server_destroy": (None, [_vp]),
    "ckks_create": (_i, [_i, C.c_uint64, C.c_double, C.POINTER(C.c_void_p)]),
    "ckks_free": (None, [_vp]),
    "ckks_slots": (_i, [_vp]),
    "ckks_set_cluster_limit": (_i, [_vp, _sz]),
    "ckks_encode": (_i, [_vp, _vp, _vp, _sz, _vp, _vp]),
    "ckks_decode": (_i, [_vp, _vp, _sz, _vp, _vp, _vp]),
    "ckks_keygen": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "ckks_encrypt": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "ckks_sum": (_i, [_vp, C.POINTER(C.c_void_p), _i, _sz, _vp, _vp]),
    "ckks_decrypt": (_i, [_vp, _vp, _vp, _sz, _vp, _vp]),
    "ckks_prepare_public_key": (_i, [_vp, _vp, _vp, _vp]),
    "ckks_prepare_secret_key": (_i, [_vp, _vp, _vp]),
    "ckks_encrypt_prepared": (_i, [_vp, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "ckks_decrypt_prepared": (_i, [_vp, _vp, _sz, _vp, _vp]),
})
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = range(5)

_lib = None


class PaillierError(RuntimeError):
    def __init__(self, code: int, fn: str, msg: str):
        super().__init__(f"{fn} failed with {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def header_functions() -> list:
    """Function names declared in include/*.h (for the export check)."""
    names = []
    for fn in sorted(os.listdir(HEADER_DIR)):
        if fn.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:[A-Za-z_][\w ]*?[\s\*]+)(\w+)\s*\(", text, flags=re.M)
    return [n for n in names if not n.startswith("PL_") and n not in ("if", "while", "defined")]


def lib():
    """Load the library once (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"native library missing: {LIB_PATH}; run python -m paper_2504_03909_b300.build")
        l = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(l, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = l
    return _lib


def last_error() -> str:
    m = lib().paillier_last_error()
    return m.decode() if m else ""


def check(code: int, fn: str):
    if code != PL_OK:
        raise PaillierError(code, fn, last_error())


def call(fn: str, *args):
    """Call a status-returning entry point; raise PaillierError on failure."""
    rc = getattr(lib(), fn)(*args)
    check(rc, fn)
    return rc
