"""pauli_prescreen_noalloc, the pre-screen for callers that cannot allocate device memory.

Such callers (code inside an allocation-free region, or a process whose device memory belongs to
someone else's fixed pool) get the same pre-screen with its scratch held in a device array that
is part of the library image.  Here it is called through the C ABI and must give exactly what
pauli_prescreen gives, on two calls in a row (the array keeps the first call's contents, so the
second call checks that everything that must start at zero is cleared).
"""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import workload_circuit

pytestmark = pytest.mark.gpu


def _noalloc(q, N, circ, shot0, nshots, p, seed, w_max=15):
    nwords = (nshots + 63) // 64
    mask = torch.zeros(max(nwords, 1), dtype=torch.int64, device="cuda")
    surv = torch.zeros(max(nshots, 1), dtype=torch.int64, device="cuda")
    n_kept = C.c_uint64()
    hd = np.zeros(w_max + 1, dtype=np.uint64)
    hk = np.zeros(w_max + 1, dtype=np.uint64)
    st = N.lib().pauli_prescreen_noalloc(
        circ.handle, N.Noise(p, seed, -1), shot0, nshots, C.c_void_p(mask.data_ptr()),
        C.c_void_p(surv.data_ptr()), nshots, C.byref(n_kept), hd.ctypes.data_as(C.c_void_p),
        hk.ctypes.data_as(C.c_void_p), w_max, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    N.check(st)
    return mask[:nwords], surv[:n_kept.value], n_kept.value, hd, hk


def test_noalloc_prescreen_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_common import lib_ready
    q = lib_ready()
    from paper_2609_19116_b300 import _native as N
    circ = q.Circuit(workload_circuit("d3_17q_12l"))
    circ2 = q.Circuit(workload_circuit("d5_49q_60l", layers=10))
    calls = [(circ, 0, 20000 + 37, 3e-3, 9), (circ2, 64 * 777, 100000, 1e-3, 4)]
    for c, shot0, n, p, seed in calls:
        ref = q.pauli_prescreen(c, shot0, n, p=p, seed=seed)
        mask, surv, n_kept, hd, hk = _noalloc(q, N, c, shot0, n, p, seed)
        assert n_kept == ref["n_kept"]
        assert torch.equal(mask, ref["kept_mask"])
        assert torch.equal(surv, ref["survivors"])
        assert np.array_equal(hd, ref["hist_drawn"]) and np.array_equal(hk, ref["hist_kept"])
        assert hd.sum() == n


def test_noalloc_rejects_oversized_requests():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_common import lib_ready
    q = lib_ready()
    from paper_2609_19116_b300 import _native as N
    circ = q.Circuit(workload_circuit("d3_17q_12l", layers=2))
    too_many = 8192 * 1024 * 64 + 64
    mask = torch.zeros(16, dtype=torch.int64, device="cuda")  # never touched: the size check comes first
    st = N.lib().pauli_prescreen_noalloc(circ.handle, N.Noise(1e-3, 0, -1), 0, too_many, C.c_void_p(mask.data_ptr()),
                                         None, 0, C.byref(C.c_uint64()), None, None, 15, None)
    assert st == N.QC_ECAPACITY
