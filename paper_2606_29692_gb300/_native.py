"""ctypes declarations of the C ABI in ``include/tq.h`` (marshalling only).

The library is loaded from ``lib/libtq.so`` inside this package.  There is no
fallback: if the library has not been built, ``lib()`` raises, so a missing
extension can never silently turn into some other code path.
"""

from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libtq.so")

TQ_JW, TQ_BK = 0, 1
TQ_C128, TQ_C64 = 0, 1
STATUS = {0: "TQ_OK", -1: "TQ_EINVAL", -2: "TQ_ENOMEM", -3: "TQ_ECUDA", -4: "TQ_ETIMEOUT",
          -5: "TQ_EBUSY", -6: "TQ_ENUMERIC"}


class TQError(RuntimeError):
    def __init__(self, code, func, msg):
        super().__init__(f"{func}: {STATUS.get(code, code)}: {msg}")
        self.code = code


class Request(C.Structure):
    _fields_ = [("kind", C.c_int), ("session", C.c_int), ("op", C.c_int), ("pad", C.c_int),
                ("theta", C.c_double), ("tag", C.c_ulonglong)]


class Completion(C.Structure):
    _fields_ = [("tag", C.c_ulonglong), ("kind", C.c_int), ("session", C.c_int), ("status", C.c_int),
                ("argmax", C.c_int), ("energy", C.c_double), ("max_grad", C.c_double),
                ("norm2", C.c_double), ("t_submit", C.c_double), ("t_done", C.c_double)]


class AdaptResult(C.Structure):
    _fields_ = [("energy", C.c_double), ("max_grad", C.c_double), ("theta", C.c_double),
                ("selected", C.c_int), ("converged", C.c_int)]


vp = C.c_void_p
i32 = C.c_int
i64 = C.c_longlong
f64 = C.c_double
P = C.POINTER

# name -> argument types (every function returns int unless listed in _RET)
SIGNATURES = {
    "tq_last_error": [],
    "tq_version": [],
    "tq_ctx_create": [i32, P(vp)],
    "tq_ctx_destroy": [vp],
    "tq_ctx_launch_count": [vp, P(i64)],
    "tq_ctx_trace": [vp, i32],
    "tq_ctx_set_pair_schedule": [vp, i32, i32],
    "tq_ctx_get_pair_schedule": [vp, i32, P(i32)],
    "tq_autotune_pair": [vp, vp, i32, i32, P(i32), P(f64)],
    "tq_ctx_set_spmv_schedule": [vp, i32],
    "tq_ctx_set_test_flags": [vp, i32],
    "tq_autotune_spmv": [vp, vp, vp, P(i32), P(f64)],
    "tq_ctx_trace_report": [vp, vp, C.c_size_t],
    "tq_pauli_hamiltonian": [i32, vp, vp, f64, i32, P(i64), vp, vp, vp, i64],
    "tq_pool_excitations": [i32, i32, P(i32), vp, i32],
    "tq_pauli_pool": [i32, i32, i32, i32, vp, vp, vp, vp],
    "tq_pool_support_forms": [i32, i32, i32, i32, vp, vp, vp, vp, vp, vp],
    "tq_hf_index": [i32, i32, i32, P(i64)],
    "tq_build_hamiltonian": [vp, i32, vp, vp, f64, i32, i32, P(vp)],
    "tq_ham_info": [vp, P(i32), P(i32), P(i64), P(i64), P(i64), P(i64), P(C.c_size_t)],
    "tq_ham_csr": [vp, P(vp), P(vp), P(vp), P(vp)],
    "tq_ham_xell": [vp, P(i64), P(i64), P(vp), P(vp), P(vp)],
    "tq_ham_free": [vp],
    "tq_build_pool": [vp, i32, i32, i32, P(vp)],
    "tq_pool_info": [vp, P(i32), P(i32), vp],
    "tq_pool_csr": [vp, vp, i32, i32, P(vp), P(vp), P(vp), P(i64)],
    "tq_pool_free": [vp],
    "tq_state_create": [vp, i32, i32, P(vp)],
    "tq_state_wrap": [vp, i32, i32, vp, P(vp)],
    "tq_state_data": [vp, P(vp), P(i32), P(i32)],
    "tq_state_set_hf": [vp, i32, i32, vp],
    "tq_state_free": [vp],
    "tq_read_fcidump": [C.c_char_p, P(i32), P(i32), P(i32), P(f64), vp, vp, i32],
    "tq_write_fcidump": [C.c_char_p, i32, i32, i32, vp, vp, f64, f64],
    "tq_state_save": [vp, C.c_char_p],
    "tq_state_load": [vp, C.c_char_p],
    "tq_ansatz_energy_grad": [vp, vp, vp, vp, i32, vp, vp, P(f64), vp, vp, vp],
    "tq_adapt_vqe": [vp, vp, vp, vp, f64, i32, f64, i32, P(i32), vp, vp, vp, vp],
    "tq_pool_families": [vp, i32, vp, vp, P(i32)],
    "tq_pool_families_host": [i32, i32, i32, i32, i32, vp, vp, P(i32)],
    "tq_sector_dim": [i32, i32, i32, P(i64)],
    "tq_sector_basis": [i32, i32, i32, i32, i64, vp],
    "tq_build_hamiltonian_sector": [vp, i32, vp, vp, f64, i32, i32, i32, i32, P(vp)],
    "tq_build_pool_sector": [vp, i32, i32, i32, i32, i32, P(vp)],
    "tq_pool_sector_table": [vp, P(i64), P(vp), P(vp)],
    "tq_state_create_sector": [vp, i32, i32, i32, i32, P(vp)],
    "tq_state_wrap_sector": [vp, i32, i32, i32, i32, vp, P(vp)],
    "tq_evolve_taylor5": [vp, vp, i32, f64, vp, i32, vp],
    "tq_evolve_taylor5_csr": [vp, i32, vp, vp, vp, f64, vp, i32, vp],
    "tq_energy": [vp, vp, vp, P(f64), vp],
    "tq_energy_matrix_free": [vp, vp, vp, P(f64), vp],
    "tq_energy_noalloc": [i32, i32, vp, vp, vp, vp, vp, vp, vp],
    "tq_pool_gradients": [vp, vp, vp, vp, vp, i32, vp],
    "tq_adapt_step": [vp, vp, vp, vp, f64, f64, P(AdaptResult), vp],
    "tq_adapt_run": [vp, vp, vp, vp, f64, vp, i32, vp, P(i32), vp],
    "tq_evolve_taylor5_batch": [vp, vp, i32, i32, vp, vp, vp, vp, vp],
    "tq_evolve_taylor5_batch_support": [vp, vp, i32, i32, vp, vp, vp, vp, vp],
    "tq_evolve_taylor5_batch_support_host": [vp, vp, i32, i32, vp, vp, vp, vp],
    "tq_ctx_set_support_schedule": [vp, i32, i32],
    "tq_autotune_support": [vp, vp, i32, i32, P(i32), P(f64)],
    "tq_fp64_fma_rate": [vp, i32, P(f64)],
    "tq_evolve_taylor5_batch_grouped": [vp, vp, i32, i32, vp, vp, vp, vp, vp],
    "tq_ctx_set_grouped_schedule": [vp, i32, i32, i32],
    "tq_ctx_set_support_occupancy": [vp, i32, i32],
    "tq_mapping_relabelled": [i32, i32, vp, P(i32)],
    "tq_pool_sector_order": [i32, i32, i32, i32, vp],
    "tq_mapping_linear": [i32, i32, vp, P(i32)],
    "tq_evolve_taylor5_batch_support_touch": [vp, vp, i32, i32, vp, vp, vp, vp],
    "tq_pool_sector_basis": [i32, i32, i32, i32, vp],
    "tq_l2_read_rate": [vp, i64, i32, P(f64)],
    "tq_ctx_set_l2_fetch": [vp, i32],
    "tq_ctx_get_l2_fetch": [vp, P(i32)],
    "tq_evolve_taylor5_batch_host": [vp, vp, i32, i32, vp, vp, vp, vp],
    "tq_batch_create": [vp, i32, vp, vp, vp, vp, vp, vp, f64, P(vp)],
    "tq_batch_set_schedule": [vp, i32],
    "tq_batch_autotune": [vp, P(i32), P(f64)],
    "tq_batch_run": [vp, i32, vp],
    "tq_batch_results": [vp, vp, vp, vp, vp, vp, vp],
    "tq_batch_state": [vp, i32, P(vp), P(i32)],
    "tq_batch_free": [vp],
    "tq_server_create": [vp, i32, C.c_size_t, i32, P(vp)],
    "tq_server_add_hamiltonian": [vp, vp, vp, P(i32)],
    "tq_server_add_session": [vp, i32, i32, i32, P(i32)],
    "tq_server_start": [vp],
    "tq_server_submit": [vp, P(Request)],
    "tq_server_poll": [vp, vp, i32, P(i32), i32],
    "tq_server_stats": [vp, P(i64), P(i64), P(i64)],
    "tq_server_session_state": [vp, i32, P(vp), P(i32)],
    "tq_server_stop": [vp],
    "tq_server_free": [vp],
}
_RET = {"tq_last_error": C.c_char_p}

_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"native library {LIB_PATH} is missing: build it with "
                "`python -m paper_2606_29692_gb300.build` (needs nvcc); there is no fallback")
        l = C.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(l, name)
            f.argtypes = args
            f.restype = _RET.get(name, C.c_int)
        _lib = l
    return _lib


def call(name, *args):
    """Call ``name``; raise TQError with the library's reason on failure."""
    rc = getattr(lib(), name)(*args)
    if rc != 0:
        msg = lib().tq_last_error()
        raise TQError(rc, name, msg.decode() if msg else "")
    return rc
