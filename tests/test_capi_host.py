"""C-ABI library on the host (no GPU calls): it loads, exports every entry point the header
declares, and its host-side circuit analysis agrees with the oracle's."""
import ctypes
import os
import re

import pytest

from oracle import prescreen
from oracle.circuit import parse as oracle_parse
from synth import random_circuit, workload_circuit

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qcmps.h")


@pytest.fixture(scope="module")
def native():
    from paper_2609_19116_b300 import build
    if build.needs_build():
        build.build()
    from paper_2609_19116_b300 import _native
    return _native


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qc_\w+|pauli_\w+|mps_\w+)\s*\(", text)))


def test_header_symbols_exported(native):
    lib = ctypes.CDLL(native.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(native.EXPORTED) == declared


@pytest.mark.parametrize("text", [workload_circuit("d3_17q_12l"), workload_circuit("d5_49q_60l", layers=6),
                                  random_circuit(9, 300, seed=2, p_meas=0.1, p_reset=0.05)])
def test_host_analysis_matches_oracle(native, text):
    from paper_2609_19116_b300.api import Circuit
    c = Circuit(text)
    oc = oracle_parse(text)
    info = c.info()
    assert info["n_qubits"] == oc.n
    assert info["n_channels"] == oc.n_channels
    assert info["n_measurements"] == sum(1 for n, _ in oc.ops if n == "M")
    dec = prescreen.decided_measurements(oc)
    expect = [dec[i] for i, (n, _) in enumerate(oc.ops) if n == "M"]
    assert list(c.decided()) == expect
    assert info["n_mps_updates"] > 0


@pytest.mark.parametrize("bad", ["", "H 0\n", "QUBITS 2\nCX 0 0\n", "QUBITS 2\nFOO 1\n", "QUBITS 2\nH 5\n",
                                 "QUBITS 2\nQUBITS 3\n", "QUBITS 2\nH 0 1\n"])
def test_malformed_text_is_rejected(native, bad):
    from paper_2609_19116_b300.api import Circuit
    with pytest.raises(native.QcError) as ei:
        Circuit(bad)
    assert ei.value.status == native.QC_EINVAL


def test_footprint_formula(native):
    from paper_2609_19116_b300.api import Circuit
    c = Circuit(workload_circuit("d5_49q_60l", layers=2))
    small, big = c.footprint(16), c.footprint(64)
    assert 0 < small < big
    # complex128 doubles the site tensors; a complex64 slot also holds room for an FP64 re-split
    assert big < c.footprint(64, native.QC_C128) <= 2 * big


@pytest.mark.parametrize("chi,cutoff,prec", [(0, 1e-10, 0), (1025, 1e-10, 0), (2048, 0.0, 1), (32, -1.0, 0),
                                             (32, 1e-10, 7)])
def test_sampling_arguments_are_checked_before_device_work(native, chi, cutoff, prec):
    """chi_max in [1, 1024] (the engine's index arithmetic and slot layout assume it), cutoff >= 0, a known
    precision: rejected with QC_EINVAL by the host before any device call, so this runs without a GPU."""
    import ctypes as C
    from paper_2609_19116_b300.api import Circuit
    c = Circuit(workload_circuit("d3_17q_12l", layers=2))
    lib = native.lib()
    st = lib.mps_sample_batch(c._h, native.Noise(1e-3, 1, -1), None, 0, native.MpsParams(chi, cutoff, prec, 0.0),
                              None, 0, None, None)
    assert st == native.QC_EINVAL
