"""GPU parity of the per-gate path, fused blocks and read-out against the CPU
oracle, through the C ABI.  Tolerances (from the stated accuracy bar):
complex128 max |d amp| <= 1e-12; complex64 1 - F <= 1e-5 and
max |d amp| <= 1e-6 * ||psi||."""

import math

import numpy as np
import pytest

from paper_1912_03243_gb300 import circuits as C

pytestmark = pytest.mark.gpu

TOL_C128 = 1e-12
TOL_C64_F = 1e-5
TOL_C64_AMP = 1e-6


@pytest.fixture(scope="module")
def S():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03243_gb300 import build, sv

    build.build()
    sv.lib()
    return sv


def fidelity(a, b):
    return abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def check(dtype, got, ref):
    got = np.asarray(got, dtype=np.complex128)
    if dtype == "c128":
        assert np.max(np.abs(got - ref)) <= TOL_C128
    else:
        nrm = math.sqrt(np.vdot(ref, ref).real)
        assert np.max(np.abs(got - ref)) <= TOL_C64_AMP * nrm
        assert 1 - fidelity(ref, got) <= TOL_C64_F


def random_u(rng, d=2):
    z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 2, 3, 7])
def test_every_target_and_control(S, orc, dtype, n):
    """Every (target, control) pair with a dense, a diagonal (u00 = 1) and a
    general diagonal matrix against the oracle's Eq. 1 loops."""
    rng = np.random.default_rng(100 + n)
    psi0 = C.random_state(n, n)
    mats = [random_u(rng), np.diag([1, np.exp(0.3j)]), np.diag([np.exp(-0.2j), np.exp(0.7j)]),
            orc.gate_matrix("X")]
    sv_ = S.StateVector(n, dtype)
    for u in mats:
        for t in range(n):
            for c in [-1] + [q for q in range(n) if q != t]:
                sv_.from_numpy(psi0)
                sv_.apply_gate(t, u, control=c)
                if c < 0:
                    ref = orc.apply_1q(psi0, t, u)
                else:
                    cu = np.eye(4, dtype=complex)
                    cu[np.ix_([1, 3], [1, 3])] = u
                    ref = orc.apply_kq(psi0, [c, t], cu)
                check(dtype, sv_.to_numpy(), ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_circuit_20q(S, orc, dtype, seed):
    """20 qubits, depth 20 random circuit, full 16 MB vector against the oracle."""
    c = C.random_circuit(20, 20, seed)
    ref = orc.run(c)
    sv_ = S.StateVector(20, dtype)
    sv_.run(c, "pergate")
    check(dtype, sv_.to_numpy(), ref)
    assert abs(sv_.norm() - 1) < (1e-12 if dtype == "c128" else 1e-5)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_all_gate_kinds(S, orc, dtype):
    n = 9
    c = C.random_unitary_gates(n, 300, 17)
    ref = orc.run(c)
    sv_ = S.StateVector(n, dtype)
    sv_.run(c, "pergate")
    check(dtype, sv_.to_numpy(), ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_fused_block(S, orc, dtype, k):
    n = 10
    rng = np.random.default_rng(k)
    psi0 = C.random_state(n, 50 + k)
    sv_ = S.StateVector(n, dtype)
    for trial in range(3):
        qs = [int(q) for q in rng.choice(n, size=k, replace=False)]
        u = random_u(rng, 1 << k)
        sv_.from_numpy(psi0)
        sv_.apply_fused(qs, u)
        check(dtype, sv_.to_numpy(), orc.apply_kq(psi0, qs, u))


def test_closed_forms_large(S):
    """GHZ (Sec. 3) and the uniform state at 26 qubits, read out by sampled
    amplitudes and the norm (closed forms, no oracle vector needed)."""
    n = 26
    g = S.StateVector(n, "c64")
    g.run(C.ghz_circuit(n))
    a = g.amplitudes([0, (1 << n) - 1, 1, 12345, 1 << (n - 1)])
    assert np.allclose(a[:2], 1 / math.sqrt(2), atol=1e-7) and np.all(a[2:] == 0)
    assert abs(g.norm() - 1) < 1e-6
    u = S.StateVector(n, "c128")
    u.run(C.uniform_circuit(n))
    idx = np.random.default_rng(0).integers(0, 1 << n, size=1000, dtype=np.uint64)
    assert np.allclose(u.amplitudes(idx), 2.0 ** (-n / 2), rtol=1e-13, atol=0)
    assert abs(u.norm() - 1) < 1e-12


def test_qft_sampled_32q(S):
    """QFT of a basis state at 32 qubits (32 GB, complex64), sampled against
    the closed form 2^{-n/2} exp(2 pi i x y / 2^n)."""
    import torch

    n = 32
    if torch.cuda.mem_get_info()[0] < (8 << n) + (4 << 30):
        pytest.skip("not enough device memory")
    x = 0x9E3779B9
    s = S.StateVector(n, "c64")
    s.set_basis(x)
    s.run(C.qft_circuit(n), "pergate")
    y = np.random.default_rng(1).integers(0, 1 << n, size=4096, dtype=np.uint64)
    got = s.amplitudes(y)
    ph = ((x * y.astype(object)) % (1 << n)).astype(np.float64) / (1 << n)
    expect = np.exp(2j * np.pi * ph) / math.sqrt(1 << n)
    assert np.max(np.abs(got - expect)) <= TOL_C64_AMP
    assert abs(s.norm() - 1) < 1e-4
    del s
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_30q_inverse_and_24q_oracle(S, orc, dtype):
    """30 qubits, depth 16: the circuit followed by its inverse returns to
    |0...0>; the same rule at 24 qubits is compared with the oracle."""
    import torch

    c24 = C.random_circuit(24, 16, 1)
    ref = orc.run(c24)
    s24 = S.StateVector(24, dtype)
    s24.run(c24, "pergate")
    check(dtype, s24.to_numpy(), ref)
    del s24
    n = 30
    s = S.StateVector(n, dtype)
    c = C.random_circuit(n, 16, 1)
    s.run(c, "pergate")
    nrm = s.norm()
    s.run(C.inverse_circuit(c), "pergate")
    a = s.amplitudes([0, 1, 2, (1 << n) - 1, 987654321])
    tol = 1e-11 if dtype == "c128" else 2e-5
    assert abs(a[0] - 1) < tol and np.max(np.abs(a[1:])) < tol
    assert abs(nrm - 1) < (1e-12 if dtype == "c128" else 1e-5)
    del s
    torch.cuda.empty_cache()


def test_argument_errors(S):
    s = S.StateVector(5, "c64")
    with pytest.raises(S.SVError) as e:
        s.apply_gate(5, np.eye(2))
    assert e.value.status == 1
    with pytest.raises(S.SVError):
        s.apply_gate(2, np.eye(2), control=2)
    with pytest.raises(S.SVError):
        s.apply_fused([1, 1], np.eye(4))
    with pytest.raises(S.SVError):
        s.amplitudes([32])
    with pytest.raises(S.SVError) as e:
        s.run("qubits 5\nFOO 1\n")
    assert e.value.status == 7
    with pytest.raises(S.SVError):
        s.run("qubits 4\nH 1\n")
    # the state is unchanged by rejected calls
    a = s.amplitudes([0])
    assert a[0] == 1


def test_basis_and_norm(S):
    for dtype in ("c64", "c128", "enc2b"):
        s = S.StateVector(12, dtype)
        s.set_basis(1234)
        a = s.amplitudes([1234, 0])
        assert a[0] == 1 and a[1] == 0
        assert s.norm() == 1.0
