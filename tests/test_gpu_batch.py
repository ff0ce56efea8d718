"""Batches of independent circuits of different sizes (sv_batch_*): every
member, run together with the others (direct launches first, then the
replayed CUDA graph), must match the oracle on its own."""

import numpy as np
import pytest

from paper_1912_03243_gb300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03243_gb300 import build, sv

    build.build()
    sv.lib()
    return sv


def members(seed=0):
    rng = np.random.default_rng(seed)
    ns = [12, 13, 14, 15, 16, 17, 18, 20, 22, 24] + [int(x) for x in rng.integers(12, 19, size=6)]
    return [(n, C.random_circuit(n, int(rng.integers(2, 9)), 100 + i)) for i, (n) in enumerate(ns)]


def test_every_member_matches_the_oracle(S, orc):
    import torch

    mem = members()
    states = [S.StateVector(n, "c64") for n, _ in mem]
    refs = [orc.run(c) for _, c in mem]
    b = S.Batch(states, [c for _, c in mem])
    assert b.gates == sum(len(c) for _, c in mem)
    for rep in range(3):  # direct launches, then the captured graph, then its replay
        for st in states:
            st.set_basis(0)
        b.execute()
        torch.cuda.synchronize()
        for (n, c), st, ref in zip(mem, states, refs):
            got = st.to_numpy().astype(np.complex128)
            assert np.max(np.abs(got - ref)) <= 1e-6, (rep, n)
    assert b.info().uses_graph
    b.free()


def test_complex128_and_run_once(S, orc):
    mem = [(13, C.random_circuit(13, 5, 7)), (15, C.qft_circuit(15, 0x1234)), (12, C.ghz_circuit(12))]
    states = [S.StateVector(n, "c128") for n, _ in mem]
    S.sv_run_batch(states, [c for _, c in mem])
    for (n, c), st in zip(mem, states):
        assert np.max(np.abs(st.to_numpy() - orc.run(c))) <= 1e-12, n


def test_batch_rejects_shared_states_and_codes(S):
    a, b = S.StateVector(13, "c64"), S.StateVector(14, "c64")
    c = C.random_circuit(13, 2, 1)
    with pytest.raises(S.SVError):
        S.Batch([a, a], [c, c])
    e = S.StateVector(13, "enc2b")
    with pytest.raises(S.SVError):
        S.Batch([a, e], [c, c])
    with pytest.raises(S.SVError):  # a qubit outside member 0's state
        S.Batch([a, b], [C.random_circuit(14, 2, 1), C.random_circuit(14, 2, 1)])
