"""ctypes declarations of the qcmps C ABI (include/qcmps.h).  Loading fails loudly when the
library has not been built: there is no other implementation to fall back to."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqcmps.so")

QC_OK, QC_PENDING, QC_EINVAL, QC_ENOMEM, QC_EDEVICE, QC_ENOCONV, QC_ETIMEOUT, QC_ECANCELLED, QC_ECAPACITY = \
    0, 1, -1, -2, -3, -4, -5, -6, -7
QC_C64, QC_C128 = 0, 1

STATUS_NAMES = {0: "QC_OK", 1: "QC_PENDING", -1: "QC_EINVAL", -2: "QC_ENOMEM", -3: "QC_EDEVICE",
                -4: "QC_ENOCONV", -5: "QC_ETIMEOUT", -6: "QC_ECANCELLED", -7: "QC_ECAPACITY"}


class QcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class CircuitInfo(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_ops", C.c_int64), ("n_channels", C.c_int64),
                ("n_measurements", C.c_int64), ("n_decided", C.c_int64), ("n_resets", C.c_int64),
                ("n_t", C.c_int64), ("n_mps_updates", C.c_int64),
                ("n_product_swaps", C.c_int64)]


class Noise(C.Structure):
    _fields_ = [("p", C.c_double), ("seed", C.c_uint64), ("fault_weight", C.c_int32)]


class Survivors(C.Structure):
    _fields_ = [("shots_dev", C.c_void_p), ("capacity", C.c_uint64), ("count", C.c_uint64)]


class MpsParams(C.Structure):
    _fields_ = [("chi_max", C.c_int32), ("cutoff", C.c_double), ("precision", C.c_int32), ("tau", C.c_double)]


class Counts(C.Structure):
    _fields_ = [("n", C.c_uint64), ("n_acc", C.c_uint64), ("n_err", C.c_uint64)]


class ShotResult(C.Structure):
    _fields_ = [("shot", C.c_uint64), ("status", C.c_int32), ("weight", C.c_int32),
                ("logical_error", C.c_int32), ("chi_peak", C.c_int32), ("abort_op", C.c_int64),
                ("fidelity", C.c_double), ("discarded", C.c_double), ("degenerate_cuts", C.c_int32),
                ("n_updates", C.c_int32), ("sweeps", C.c_int32), ("alg_flops", C.c_double),
                ("gmem_updates", C.c_int32), ("fp64_resplits", C.c_int32)]


class MpsTrace(C.Structure):
    _fields_ = [("readout_p1_dev", C.c_void_p), ("readout_k", C.c_int32), ("sweep_cap", C.c_int32),
                ("phase_cycles_dev", C.c_void_p), ("launch_threads_out", C.c_int32), ("launch_kb_out", C.c_int32)]


class AluPeaks(C.Structure):
    _fields_ = [("sm_count", C.c_int32), ("sm_clock_mhz", C.c_double), ("ffma_tflops", C.c_double),
                ("ffma2_tflops", C.c_double), ("dfma_tflops", C.c_double), ("lop3_tops", C.c_double),
                ("imad_tops", C.c_double)]


class ServeCfg(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("max_slots", C.c_int32), ("n_streams", C.c_int32)]


class JobResult(C.Structure):
    _fields_ = [("state", C.c_int32), ("shots", C.c_uint64), ("survivors", C.c_uint64),
                ("counts", Counts * 16), ("submit_ms", C.c_double), ("start_ms", C.c_double),
                ("end_ms", C.c_double), ("error", C.c_char * 224)]


_lib = None


def lib():
    """The library: the in-tree build, or the file named by QCMPS_LIB (for comparing builds)."""
    global _lib
    if _lib is None:
        path = os.environ.get("QCMPS_LIB") or LIB_PATH
        if not os.path.exists(path):
            raise ImportError(f"qcmps CUDA library not built ({path}); run "
                              "`python -m paper_2609_19116_b300.build`")
        L = C.CDLL(path)
        vp, u64, i32, sz = C.c_void_p, C.c_uint64, C.c_int32, C.c_size_t
        sig = {
            "qc_last_error": (C.c_char_p, []),
            "qc_circuit_parse": (C.c_int, [C.c_char_p, sz, C.POINTER(vp)]),
            "qc_circuit_free": (None, [vp]),
            "qc_circuit_get_info": (C.c_int, [vp, C.POINTER(CircuitInfo)]),
            "qc_circuit_decided": (C.c_int, [vp, vp]),
            "qc_sample_faults": (C.c_int, [vp, Noise, vp, u64, C.c_uint32, vp, vp, vp, vp]),
            "pauli_prescreen": (C.c_int, [vp, Noise, u64, u64, vp, C.POINTER(Survivors), vp, vp, i32, vp]),
            "pauli_prescreen_noalloc": (C.c_int, [vp, Noise, u64, u64, vp, vp, u64, C.POINTER(u64), vp, vp, i32,
                                                  vp]),
            "mps_sample_batch": (C.c_int, [vp, Noise, vp, u64, MpsParams, vp, i32, vp, vp]),
            "mps_sample_batch_traced": (C.c_int, [vp, Noise, vp, u64, MpsParams, vp, i32, vp,
                                                  C.POINTER(MpsTrace), vp]),
            "mps_shot_footprint": (C.c_int, [vp, MpsParams, C.POINTER(u64)]),
            "qc_measure_alu_peaks": (C.c_int, [C.POINTER(AluPeaks), vp]),
            "mps_serve_create": (C.c_int, [C.POINTER(ServeCfg), C.POINTER(vp)]),
            "mps_serve_submit": (C.c_int, [vp, vp, Noise, MpsParams, u64, u64, C.POINTER(u64)]),
            "mps_serve_poll": (C.c_int, [vp, u64, C.POINTER(JobResult)]),
            "mps_serve_cancel": (C.c_int, [vp, u64]),
            "mps_serve_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int):
    if status < 0:
        raise QcError(status, lib().qc_last_error().decode(errors="replace"))
    return status


EXPORTED = ("qc_last_error", "qc_circuit_parse", "qc_circuit_free", "qc_circuit_get_info", "qc_circuit_decided",
            "qc_sample_faults", "pauli_prescreen", "pauli_prescreen_noalloc", "mps_sample_batch", "mps_sample_batch_traced", "mps_shot_footprint", "qc_measure_alu_peaks", "mps_serve_create",
            "mps_serve_submit", "mps_serve_poll", "mps_serve_cancel", "mps_serve_destroy")
