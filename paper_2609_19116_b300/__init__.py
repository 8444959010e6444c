"""qcmps: B300-native noisy-shot MPS sampling of cultivation-shaped Clifford+T circuits.

The sampling path runs in the CUDA library libqcmps.so (include/qcmps.h); this package only
binds it.  Importing it does not touch the GPU.
"""
from ._native import QC_C64, QC_C128, QcError  # noqa: F401
from .api import (Circuit, Server, mps_sample_batch, mps_sample_batch_traced, pauli_prescreen,  # noqa: F401
                  qc_sample_faults, measure_alu_peaks, SHOT_DTYPE)
