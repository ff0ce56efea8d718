"""SV_MODE_FUSED: gates fused into k-qubit blocks (k = 3..6 picked by the
planner's autotuner), one HBM pass per block (tensor cores for complex64,
FP64 CUDA cores for complex128), against the oracle."""

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
        return
    nrm = math.sqrt(np.vdot(ref, ref).real)
    assert np.max(np.abs(got - ref)) <= 1e-6 * nrm
    f = abs(np.vdot(ref, got)) ** 2 / (np.vdot(ref, ref).real * np.vdot(got, got).real)
    assert 1 - f <= 1e-5


@pytest.mark.parametrize("n,depth,seed", [(13, 10, 1), (16, 16, 2), (20, 20, 3)])
def test_random_circuit_c64(S, orc, n, depth, seed):
    c = C.random_circuit(n, depth, seed)
    s = S.StateVector(n, "c64")
    p = s.plan(c, "fused")
    names = {k for k, _ in p.launch_info()}
    assert all(k.startswith(("k_fused_tc<k=", "k_fused_tc_groups<k=")) for k in names)  # tensor-core blocks
    assert p.passes < len(c) / 3
    p.execute()
    check("c64", s.to_numpy(), orc.run(c))


@pytest.mark.parametrize("dtype,n", [("c64", 15), ("c128", 12), ("c64", 9)])
def test_every_gate_kind(S, orc, dtype, n):
    c = C.random_unitary_gates(n, 300, 31 + n)
    s = S.StateVector(n, dtype)
    s.run(c, "fused")
    check(dtype, s.to_numpy(), orc.run(c))


def test_qft_and_ghz(S, orc):
    n = 18
    for c in (C.qft_circuit(n, 0x1F2E3), C.ghz_circuit(n)):
        s = S.StateVector(n, "c64")
        s.run(c, "fused")
        check("c64", s.to_numpy(), orc.run(c))


def test_32q_roundtrip(S):
    """The 32-qubit depth-24 benchmark circuit and its inverse in fused mode
    return to |0...0> within the complex64 bar."""
    import torch

    n = 32
    if torch.cuda.mem_get_info()[0] < (8 << n) + (4 << 30):
        pytest.skip("not enough device memory")
    s = S.StateVector(n, "c64")
    c = C.random_circuit(n, 24, 1)
    s.run(c, "fused")
    s.run(C.inverse_circuit(c), "fused")
    a = s.amplitudes([0, 7, (1 << n) - 1])
    nrm = s.norm()
    assert 1 - abs(a[0]) ** 2 / nrm <= 1e-5
    assert np.max(np.abs(a[1:])) <= 1e-6
    del s
    torch.cuda.empty_cache()
