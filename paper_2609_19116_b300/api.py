"""Python binding of the qcmps C ABI: argument marshalling only.

Device buffers are torch CUDA tensors and streams are torch CUDA streams; every computation runs
in the library's kernels.  Names follow the C entry points.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N

SHOT_DTYPE = np.dtype([("shot", "<u8"), ("status", "<i4"), ("weight", "<i4"), ("logical_error", "<i4"),
                       ("chi_peak", "<i4"), ("abort_op", "<i8"), ("fidelity", "<f8"), ("discarded", "<f8"),
                       ("degenerate_cuts", "<i4"), ("n_updates", "<i4"), ("sweeps", "<i4"), ("alg_flops", "<f8"),
                       ("gmem_updates", "<i4"), ("fp64_resplits", "<i4")], align=True)
assert SHOT_DTYPE.itemsize == C.sizeof(N.ShotResult)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dev_u64(t):
    if not (t.is_cuda and t.dtype in (torch.int64, torch.uint64) and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA int64/uint64 tensor")
    return t


class Circuit:
    """A parsed circuit (qc_circuit_parse), with its offline stabiliser analysis."""

    def __init__(self, text: str):
        L = N.lib()
        h = C.c_void_p()
        b = text.encode()
        N.check(L.qc_circuit_parse(b, len(b), C.byref(h)))
        self._h = h
        self.text = text

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = N.CircuitInfo()
        N.check(N.lib().qc_circuit_get_info(self._h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in N.CircuitInfo._fields_}

    def decided(self) -> np.ndarray:
        n = self.info()["n_measurements"]
        out = np.zeros(max(n, 1), dtype=np.uint8)
        N.check(N.lib().qc_circuit_decided(self._h, out.ctypes.data_as(C.c_void_p)))
        return out[:n].astype(bool)

    def footprint(self, chi_max: int, precision: int = N.QC_C64) -> int:
        v = C.c_uint64()
        N.check(N.lib().mps_shot_footprint(self._h, N.MpsParams(chi_max, 0.0, precision, 0.0), C.byref(v)))
        return v.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            N.lib().qc_circuit_free(h)
            self._h = None


def qc_sample_faults(circ: Circuit, shots: torch.Tensor, *, p: float, seed: int, fault_weight: int = -1,
                     max_faults: int = 64, stream=None):
    shots = _dev_u64(shots)
    n = shots.numel()
    dev = shots.device
    count = torch.zeros(n, dtype=torch.int32, device=dev)
    chan = torch.zeros(n * max_faults, dtype=torch.int32, device=dev)
    code = torch.zeros(n * max_faults, dtype=torch.uint8, device=dev)
    N.check(N.lib().qc_sample_faults(circ.handle, N.Noise(p, seed, fault_weight), _ptr(shots), n, max_faults,
                                     _ptr(count), _ptr(chan), _ptr(code), _stream(stream)))
    return count, chan.view(n, max_faults), code.view(n, max_faults)


def pauli_prescreen(circ: Circuit, shot0: int, nshots: int, *, p: float, seed: int, w_max: int = 15,
                    survivors_capacity: int | None = None, kept_mask: torch.Tensor | None = None,
                    survivors: torch.Tensor | None = None, fault_weight: int = -1, device=None, stream=None):
    """Returns dict(kept_mask (int64 words), survivors (int64, first n), n_kept, hist_drawn, hist_kept)."""
    device = device or torch.device("cuda")
    nwords = (nshots + 63) // 64
    if kept_mask is None:
        kept_mask = torch.empty(max(nwords, 1), dtype=torch.int64, device=device)
    if survivors_capacity is None:
        survivors_capacity = nshots
    if survivors is None and survivors_capacity > 0:
        survivors = torch.empty(survivors_capacity, dtype=torch.int64, device=device)
    surv = N.Survivors(survivors.data_ptr() if survivors is not None else None,
                       survivors.numel() if survivors is not None else 0, 0)
    hd = np.zeros(w_max + 1, dtype=np.uint64)
    hk = np.zeros(w_max + 1, dtype=np.uint64)
    N.check(N.lib().pauli_prescreen(circ.handle, N.Noise(p, seed, fault_weight), shot0, nshots, _ptr(kept_mask),
                                    C.byref(surv), hd.ctypes.data_as(C.c_void_p), hk.ctypes.data_as(C.c_void_p),
                                    w_max, _stream(stream)))
    n = surv.count
    return {"kept_mask": kept_mask[:nwords], "survivors": survivors[:min(n, surv.capacity)] if survivors is not None else None,
            "n_kept": n, "hist_drawn": hd, "hist_kept": hk}


def mps_sample_batch(circ: Circuit, shots: torch.Tensor, *, p: float, seed: int, chi_max: int, cutoff: float,
                     precision: int = N.QC_C64, tau: float = 0.0, w_max: int = 15, fault_weight: int = -1,
                     per_shot: bool = True, per_shot_buf: torch.Tensor | None = None, copy_back: bool = True,
                     launch: dict | None = None, stream=None):
    """Returns (counts[w_max+1, 3] numpy uint64 (n, n_acc, n_err), per-shot structured array or None).

    With copy_back=False the per-shot results stay in per_shot_buf on the device.  launch: optional dict
    that receives the launch configuration of the first pass (threads per shot, KB of work area)."""
    shots = _dev_u64(shots)
    n = shots.numel()
    counts = (N.Counts * (w_max + 1))()
    buf = None
    if per_shot:
        buf = per_shot_buf if per_shot_buf is not None else torch.zeros(
            max(n, 1) * SHOT_DTYPE.itemsize, dtype=torch.uint8, device=shots.device)
    prm = N.MpsParams(chi_max, cutoff, precision, tau)
    if launch is None:
        N.check(N.lib().mps_sample_batch(circ.handle, N.Noise(p, seed, fault_weight), _ptr(shots), n, prm,
                                         C.cast(counts, C.c_void_p), w_max, _ptr(buf), _stream(stream)))
    else:
        tr = N.MpsTrace(None, 0, 0, None)
        N.check(N.lib().mps_sample_batch_traced(circ.handle, N.Noise(p, seed, fault_weight), _ptr(shots), n, prm,
                                                C.cast(counts, C.c_void_p), w_max, _ptr(buf), C.byref(tr),
                                                _stream(stream)))
        launch.update(threads=tr.launch_threads_out, kb=tr.launch_kb_out)
    arr = np.array([[c.n, c.n_acc, c.n_err] for c in counts], dtype=np.uint64)
    res = None
    if per_shot and copy_back:
        res = np.frombuffer(buf[: n * SHOT_DTYPE.itemsize].cpu().numpy().tobytes(), dtype=SHOT_DTYPE)
    return arr, res


def mps_sample_batch_traced(circ: Circuit, shots: torch.Tensor, *, p: float, seed: int, chi_max: int, cutoff: float,
                            precision: int = N.QC_C64, tau: float = 0.0, w_max: int = 15, fault_weight: int = -1,
                            readout_k: int = 0, sweep_cap: int = 0, phase_cycles: torch.Tensor | None = None,
                            launch: dict | None = None, stream=None):
    """mps_sample_batch with the verification hooks: returns (counts, per-shot results, readout
    probabilities [nshots, readout_k] as a float64 numpy array, NaN after a shot's end).  phase_cycles:
    optional CUDA int64 tensor of 8 counters that the call adds the engines' cycles per phase to; launch:
    optional dict that receives the launch configuration of the first pass (threads per shot, KB)."""
    shots = _dev_u64(shots)
    n = shots.numel()
    counts = (N.Counts * (w_max + 1))()
    buf = torch.zeros(max(n, 1) * SHOT_DTYPE.itemsize, dtype=torch.uint8, device=shots.device)
    p1 = torch.empty(max(n * readout_k, 1), dtype=torch.float64, device=shots.device)
    tr = N.MpsTrace(p1.data_ptr() if readout_k > 0 else None, readout_k, sweep_cap,
                    _dev_u64(phase_cycles).data_ptr() if phase_cycles is not None else None)
    prm = N.MpsParams(chi_max, cutoff, precision, tau)
    N.check(N.lib().mps_sample_batch_traced(circ.handle, N.Noise(p, seed, fault_weight), _ptr(shots), n, prm,
                                            C.cast(counts, C.c_void_p), w_max, _ptr(buf), C.byref(tr),
                                            _stream(stream)))
    arr = np.array([[c.n, c.n_acc, c.n_err] for c in counts], dtype=np.uint64)
    res = np.frombuffer(buf[: n * SHOT_DTYPE.itemsize].cpu().numpy().tobytes(), dtype=SHOT_DTYPE)
    rec = p1[: n * readout_k].cpu().numpy().reshape(n, readout_k) if readout_k > 0 else None
    if launch is not None:
        launch.update(threads=tr.launch_threads_out, kb=tr.launch_kb_out)
    return arr, res, rec


def measure_alu_peaks(stream=None) -> dict:
    """qc_measure_alu_peaks: measured FP32 / paired-FP32 / FP64 FMA and INT32 LOP3 / IMAD rates."""
    r = N.AluPeaks()
    N.check(N.lib().qc_measure_alu_peaks(C.byref(r), _stream(stream)))
    return {k: getattr(r, k) for k, _ in N.AluPeaks._fields_}


class Server:
    """The serving loop (mps_serve_create / submit / poll / cancel / destroy)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 0, n_streams: int = 0):
        h = C.c_void_p()
        cfg = N.ServeCfg(hbm_budget_bytes, max_slots, n_streams)
        N.check(N.lib().mps_serve_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._circuits = {}

    def submit(self, circ: Circuit, shot0: int, nshots: int, *, p: float, seed: int, chi_max: int,
               cutoff: float, precision: int = N.QC_C64, tau: float = 0.0) -> int:
        jid = C.c_uint64()
        N.check(N.lib().mps_serve_submit(self._h, circ.handle, N.Noise(p, seed, -1),
                                         N.MpsParams(chi_max, cutoff, precision, tau), shot0, nshots, C.byref(jid)))
        self._circuits[jid.value] = circ  # keep alive
        return jid.value

    def poll(self, job_id: int):
        r = N.JobResult()
        st = N.check(N.lib().mps_serve_poll(self._h, job_id, C.byref(r)))
        if st == N.QC_PENDING:
            return None
        counts = np.array([[c.n, c.n_acc, c.n_err] for c in r.counts], dtype=np.uint64)
        return {"state": r.state, "shots": r.shots, "survivors": r.survivors, "counts": counts,
                "submit_ms": r.submit_ms, "start_ms": r.start_ms, "end_ms": r.end_ms,
                "error": r.error.decode(errors="replace")}

    def cancel(self, job_id: int):
        N.check(N.lib().mps_serve_cancel(self._h, job_id))

    def close(self):
        if getattr(self, "_h", None):
            N.lib().mps_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def shot_results(buf: torch.Tensor, n: int) -> np.ndarray:
    """Per-shot results left on the device by mps_sample_batch(copy_back=False)."""
    return np.frombuffer(buf[: n * SHOT_DTYPE.itemsize].cpu().numpy().tobytes(), dtype=SHOT_DTYPE)
