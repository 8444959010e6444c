"""The plain FP64 comparator (CPU runs of its PyTorch code): its routing plan keeps gates on
neighbouring sites and ends in a known layout, its product SWAP is exact, and its shots agree with
the oracle's state vector."""
import numpy as np
import pytest
import torch

from oracle import statevector as osv
from oracle.circuit import parse as oparse
from oracle.sampler import draw_faults
from paper_2609_19116_b300 import plain_fp64 as pf
from synth.circuits import workload_circuit
from synth.random_circuits import random_circuit


def _dense(m):
    v = m.A[0]
    for k in range(1, m.n):
        v = torch.tensordot(v, m.A[k], dims=([-1], [0]))
    return v.reshape(-1).cpu().numpy()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plan_gates_are_adjacent_and_state_matches(seed):
    text = random_circuit(8, 120, seed=seed, max_dist=5, noise=False, one_q=("H", "T", "S"))
    n, ops = pf.parse(text)
    steps, pos = pf.plan(n, ops, return_layout=True)
    assert sorted(pos) == list(range(n))
    one, two, _ = pf._gates("cpu")
    m = pf.PlainMPS(n, 1 << 20, 0.0, "cpu")
    sw = two["SWAP"]
    for st in steps:
        if st[0] == "1q":
            m.one(one[st[1]], st[2])
        elif st[0] == "g2":
            m.two_site(two[st[1]] if st[3] else sw @ two[st[1]] @ sw, st[2])
        elif st[0] == "swap":
            m.two_site(sw, st[1])
        elif st[0] == "pswap":
            m.product_swap(st[1], st[2])
    v = _dense(m).reshape((2,) * n)
    # site k holds logical qubit at[k]; bring logical order back
    at = [0] * n
    for q, k in enumerate(pos):
        at[k] = q
    v = np.transpose(v, np.argsort(at)).reshape(-1)
    sv = osv.run_shot(oparse(text), reference=True)[1]
    ref = sv.psi.reshape(-1) if hasattr(sv, "psi") else np.asarray(sv).reshape(-1)
    assert abs(abs(np.vdot(ref, v)) - 1.0) < 1e-10


def test_product_swap_equals_svd_swap():
    rng = np.random.default_rng(5)
    n = 5
    m1 = pf.PlainMPS(n, 1 << 20, 0.0, "cpu")
    one, two, _ = pf._gates("cpu")
    # entangle qubits 0..4 except 2, then put qubit 2 in a random single-qubit state
    for (a, b) in [(0, 1), (3, 4), (1, 0), (4, 3)]:
        m1.one(one["H"], min(a, b))
        m1.two_site(two["CX"], min(a, b))
        m1.one(one["T"], max(a, b))
    m1.one(one["H"], 2)
    m1.one(one["T"], 2)
    m2 = pf.PlainMPS(n, 1 << 20, 0.0, "cpu")
    m2.A = [a.clone() for a in m1.A]
    m2.center = m1.center
    m1.product_swap(2, True)
    m2.two_site(two["SWAP"], 2)
    v1, v2 = _dense(m1), _dense(m2)
    assert abs(abs(np.vdot(v1, v2)) - 1.0) < 1e-12
    m1.product_swap(2, False)  # the product qubit, now on site 3, back to site 2
    m2.two_site(two["SWAP"], 2)
    assert abs(abs(np.vdot(_dense(m1), _dense(m2))) - 1.0) < 1e-12


def test_shot_statuses_match_state_vector():
    text = workload_circuit("d3_17q_12l", layers=3)
    oc = oparse(text)
    n, ops = pf.parse(text)
    steps = pf.plan(n, ops)
    shots = list(range(0, 24))
    faults = draw_faults(oc, p=4e-3, seed=9, shots=shots)
    for s in shots:
        fl = faults[s]
        st_o = osv.run_shot(oc, fl, seed=9, shot=s)[0]
        st_p, _ = pf.run_shot(n, ops, dict(fl), seed=9, shot=s, chi_max=1 << 20, cutoff=0.0, dev="cpu", steps=steps)
        assert st_o == st_p, s
