"""Plan replay through CUDA graphs: the first execution of a plan launches its
kernels directly, the second captures them on the plan's own stream and every
later one replays the graph.  Every execution gives the oracle's state (the
two-byte code: the CPU codec mirror's codes, bit for bit), on torch's default
stream and on a stream of the caller's, and SV_GRAPH=0 gives the same bits."""

import math

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


def check(dtype, got, ref):
    got = np.asarray(got, dtype=np.complex128)
    if dtype == "c128":
        assert np.max(np.abs(got - ref)) <= 1e-12
    else:
        nrm = math.sqrt(np.vdot(ref, ref).real)
        assert np.max(np.abs(got - ref)) <= 1e-6 * nrm
        f = abs(np.vdot(ref, got)) ** 2 / (np.vdot(ref, ref).real * np.vdot(got, got).real)
        assert 1 - f <= 1e-5


@pytest.mark.parametrize("mode,dtype,n", [("pergate", "c64", 12), ("pergate", "c128", 10), ("tiled", "c64", 16),
                                          ("tiled", "c128", 15), ("fused", "c64", 14)])
def test_repeated_execution_matches_oracle(S, orc, mode, dtype, n):
    c = C.random_circuit(n, 6, 5)
    ref = orc.run(c)
    s = S.StateVector(n, dtype)
    p = s.plan(c, mode)
    graph = []
    for _ in range(4):
        s.set_basis(0)
        p.execute()
        check(dtype, s.to_numpy(), ref)
        graph.append(p.uses_graph())
    assert graph == [False, True, True, True], graph
    p.free()


def test_two_byte_code_replay_bit_exact(S, orc):
    n = 12
    c = C.random_circuit(n, 4, 6)
    rc, rs = orc.enc_run(c)
    e = S.StateVector(n, "enc2b")
    p = e.plan(c, "pergate")
    for _ in range(3):
        e.set_basis(0)
        p.execute()
        gc, gs = e.codes()
        assert np.array_equal(gc, rc)
        assert np.array_equal(gs.view(np.uint32), rs.view(np.uint32))
    assert p.uses_graph()
    p.free()


def test_caller_stream_order(S, orc):
    """On a stream of the caller's: the graph waits for the reset queued
    before it, and the read-back queued after it waits for the graph."""
    import torch

    n = 16
    c = C.random_circuit(n, 8, 7)
    ref = orc.run(c)
    st = torch.cuda.Stream()
    s = S.StateVector(n, "c64", stream=st)
    p = s.plan(c, "tiled")
    for _ in range(3):
        s.set_basis(0)
        p.execute()
        check("c64", s.to_numpy(), ref)
    assert p.uses_graph()
    p.free()


def test_graph_off_same_bits(S, monkeypatch):
    n = 16
    c = C.random_circuit(n, 10, 8)
    s = S.StateVector(n, "c64")
    p = s.plan(c, "tiled")
    for _ in range(3):
        s.set_basis(0)
        p.execute()
    a = s.to_numpy()
    assert p.uses_graph()
    p.free()
    monkeypatch.setenv("SV_GRAPH", "0")
    q = s.plan(c, "tiled")
    for _ in range(3):
        s.set_basis(0)
        q.execute()
    assert not q.uses_graph()
    assert np.array_equal(a, s.to_numpy())
    q.free()
