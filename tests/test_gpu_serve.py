"""The serving loop on the GPU: jobs of different circuits and rates overlap on the device, and a
job's result is the same alone and in the mix."""
import time

import numpy as np
import pytest
import torch

from synth import workload_circuit

from gpu_common import lib_ready

pytestmark = pytest.mark.gpu


def _wait(srv, ids, timeout=300.0):
    out = {}
    t0 = time.time()
    while len(out) < len(ids):
        for j in ids:
            if j not in out:
                r = srv.poll(j)
                if r is not None:
                    out[j] = r
        if time.time() - t0 > timeout:
            raise TimeoutError("jobs did not finish")
        time.sleep(0.005)
    return out


def _job(q, c, shot0, n, p, seed, chi):
    """The same job through the direct entry points: pre-screen, then the MPS batch."""
    pre = q.pauli_prescreen(c, shot0, n, p=p, seed=seed, w_max=15)
    counts, _ = q.mps_sample_batch(c, pre["survivors"], p=p, seed=seed, chi_max=chi, cutoff=1e-10, w_max=15,
                                   per_shot=False)
    counts[:, 0] = pre["hist_drawn"]
    return counts, pre["n_kept"]


def test_job_alone_equals_job_in_mix():
    q = lib_ready()
    c17 = q.Circuit(workload_circuit("d3_17q_12l"))
    c49 = q.Circuit(workload_circuit("d5_49q_60l", layers=8))
    job_a = (c17, 64 * 10, 64 * 30, 1e-3, 5, 32)
    others = [(c49, 0, 64 * 200, 2e-3, 1, 128), (c17, 64 * 7, 64 * 50, 5e-4, 9, 32),
              (c49, 64 * 3, 64 * 100, 1e-3, 2, 64), (c17, 0, 64 * 20, 2e-3, 3, 128)]
    srv = q.Server(hbm_budget_bytes=8 << 30)
    try:
        ja = srv.submit(job_a[0], *job_a[1:3], p=job_a[3], seed=job_a[4], chi_max=job_a[5], cutoff=1e-10)
        alone = _wait(srv, [ja])[ja]
    finally:
        srv.close()
    srv = q.Server(hbm_budget_bytes=8 << 30)
    try:
        ids = [srv.submit(c, s0, n, p=p, seed=sd, chi_max=ch, cutoff=1e-10) for c, s0, n, p, sd, ch in others[:2]]
        jb = srv.submit(job_a[0], *job_a[1:3], p=job_a[3], seed=job_a[4], chi_max=job_a[5], cutoff=1e-10)
        ids += [srv.submit(c, s0, n, p=p, seed=sd, chi_max=ch, cutoff=1e-10) for c, s0, n, p, sd, ch in others[2:]]
        res = _wait(srv, ids + [jb])
    finally:
        srv.close()
    mixed = res[jb]
    assert alone["state"] == 0 and mixed["state"] == 0
    assert np.array_equal(alone["counts"], mixed["counts"])
    assert alone["survivors"] == mixed["survivors"]
    # and the served result equals the direct entry points
    direct, kept = _job(q, *job_a)
    assert np.array_equal(direct, alone["counts"]) and kept == alone["survivors"]
    for (c, s0, n, p, sd, ch), j in zip(others, ids):
        d, k = _job(q, c, s0, n, p, sd, ch)
        assert np.array_equal(d, res[j]["counts"]) and k == res[j]["survivors"]
        assert res[j]["end_ms"] >= res[j]["start_ms"] >= res[j]["submit_ms"]


def test_admission_budget_and_cancel():
    """A budget that admits one in-flight shot at a time still completes jobs with the right counts;
    a cancelled job ends cancelled (or done, if it finished first)."""
    q = lib_ready()
    c17 = q.Circuit(workload_circuit("d3_17q_12l", layers=4))
    tiny = c17.footprint(32) + 1
    srv = q.Server(hbm_budget_bytes=tiny, n_streams=2)
    try:
        j1 = srv.submit(c17, 0, 64 * 4, p=2e-3, seed=4, chi_max=32, cutoff=1e-10)
        r = _wait(srv, [j1])
        assert r[j1]["state"] == 0
        d, k = _job(q, c17, 0, 64 * 4, 2e-3, 4, 32)
        assert np.array_equal(d, r[j1]["counts"])
        j2 = srv.submit(c17, 64 * 80, 64 * 40, p=2e-3, seed=4, chi_max=32, cutoff=1e-10)
        srv.cancel(j2)
        r2 = _wait(srv, [j2])
        assert r2[j2]["state"] in (0, -6)
    finally:
        srv.close()


def test_interleaved_mixed_jobs_all_complete():
    """Many 17-qubit and 49-qubit jobs submitted back to back over 16 worker streams: their pre-screen
    and engine launches need different shared-memory sizes and run concurrently; every job must end
    with state 0 and the counts of the direct entry points."""
    q = lib_ready()
    c17 = q.Circuit(workload_circuit("d3_17q_12l", layers=6))
    c49 = q.Circuit(workload_circuit("d5_49q_60l", layers=6))
    jobs = []
    for i in range(24):
        c, chi = (c17, 32) if i % 2 == 0 else (c49, 128)
        jobs.append((c, 64 * 100 * i, 64 * (4 + 3 * (i % 5)), (5e-4, 1e-3, 2e-3)[i % 3], 7 + i, chi))
    srv = q.Server(hbm_budget_bytes=4 << 30, n_streams=16)
    try:
        ids = [srv.submit(c, s0, n, p=p, seed=sd, chi_max=ch, cutoff=1e-10) for c, s0, n, p, sd, ch in jobs]
        res = _wait(srv, ids)
    finally:
        srv.close()
    for (c, s0, n, p, sd, ch), j in zip(jobs, ids):
        r = res[j]
        assert r["state"] == 0, (r["state"], r["error"])
        d, k = _job(q, c, s0, n, p, sd, ch)
        assert np.array_equal(d, r["counts"]) and k == r["survivors"]


def test_large_job_is_not_starved_by_a_stream_of_small_jobs():
    """Shortest-remaining-work first, aged: a large job that shares two worker streams with a steady
    stream of small jobs still finishes while the small jobs keep arriving."""
    q = lib_ready()
    c17 = q.Circuit(workload_circuit("d3_17q_12l", layers=3))
    c_big = q.Circuit(workload_circuit("d3_17q_12l"))
    big = (c_big, 0, 64 * 60, 2e-3, 1, 32)
    srv = q.Server(hbm_budget_bytes=8 << 30, n_streams=2)
    try:
        t0 = time.time()
        jb = srv.submit(big[0], *big[1:3], p=big[3], seed=big[4], chi_max=big[5], cutoff=1e-10)
        alone_s = None
        while srv.poll(jb) is None:
            time.sleep(0.002)
        alone_s = time.time() - t0
    finally:
        srv.close()
    window = max(4.0, 4 * alone_s + 3.0)
    srv = q.Server(hbm_budget_bytes=8 << 30, n_streams=2)
    try:
        small, k = [], 0
        t0 = time.time()
        jb = srv.submit(big[0], 64 * 5000, big[2], p=big[3], seed=big[4], chi_max=big[5], cutoff=1e-10)
        big_done = None
        while time.time() - t0 < window:
            small.append(srv.submit(c17, 64 * 10 * k, 64 * 2, p=1e-3, seed=k, chi_max=32, cutoff=1e-10))
            k += 1
            if big_done is None and srv.poll(jb) is not None:
                big_done = time.time() - t0
            time.sleep(0.01)
        _wait(srv, small + [jb])
        r = srv.poll(jb)
    finally:
        srv.close()
    assert r["state"] == 0, r["error"]
    assert big_done is not None and big_done < window, (big_done, window, alone_s)
