"""<sigma^alpha_i> for every qubit in one call (Sec. 3: the validation
observable <Q_alpha(i)> = (1 - <sigma^alpha_i>)/2) against the oracle, which
applies the Pauli matrix to a copy and takes the inner product; the paper's
values for the uniform superposition at 32 qubits; GHZ."""

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


def oracle_expect(orc, psi):
    n = int(math.log2(psi.size))
    return np.array([[orc.expect_pauli(psi, q, a) for a in "xyz"] for q in range(n)])


@pytest.mark.parametrize("dtype,tol", [("c64", 2e-6), ("c128", 1e-12)])
@pytest.mark.parametrize("n", [1, 3, 12, 13, 17, 22])
def test_random_states(S, orc, dtype, tol, n):
    """n = 1..12 fit one tile; 13 is one tile of 2^13 (complex64) or two
    (complex128); 17 and 22 need several passes (complex64 tiles keep the low
    3 qubits and take up to 10 uncovered ones)."""
    psi = C.random_state(n, 40 + n)
    s = S.StateVector(n, dtype)
    s.from_numpy(psi)
    got = s.expect_pauli()
    ref = oracle_expect(orc, s.to_numpy().astype(np.complex128))
    assert got.shape == (n, 3)
    assert np.max(np.abs(got - ref)) <= tol


@pytest.mark.parametrize("n", [14, 15, 24])
def test_persistent_tiles(S, orc, n):
    """Complex64 passes over 2^13-amplitude tiles run persistent CTAs (two
    per SM): n = 14 and 15 give some CTAs one tile and leave the rest idle,
    n = 24 gives each CTA six or seven tiles (the next tile's copies issued
    under the current one's arithmetic, FP32 chunks of 8 tiles summed in
    FP64)."""
    psi = C.random_state(n, 90 + n)
    s = S.StateVector(n, "c64")
    s.from_numpy(psi)
    got = s.expect_pauli()
    ref = oracle_expect(orc, s.to_numpy().astype(np.complex128))
    assert np.max(np.abs(got - ref)) <= 4e-6


@pytest.mark.parametrize("low", ["4", "5", "8"])
def test_low_qubit_variants(S, orc, monkeypatch, low):
    """Later passes that keep 4, 5 or 8 low qubits (SV_EXPECT_LOW) instead of
    3: more passes, uncovered qubits in other tile bits, covered ones as
    fillers; the same values."""
    monkeypatch.setenv("SV_EXPECT_LOW", low)
    n = 21
    psi = C.random_state(n, 77)
    s = S.StateVector(n, "c64")
    s.from_numpy(psi)
    got = s.expect_pauli()
    ref = oracle_expect(orc, s.to_numpy().astype(np.complex128))
    assert np.max(np.abs(got - ref)) <= 2e-6


@pytest.mark.parametrize("n", [5, 8, 12, 16, 21])
def test_two_byte_code(S, orc, n):
    """The encoded state is decoded on the fly; the values equal those of the
    decoded complex64 state (n = 5 is a single short block, 8-12 one tile,
    16 and 21 several passes over whole blocks)."""
    c = C.random_circuit(n, 3, 5)
    s = S.StateVector(n, "c64")
    s.run(c, "pergate")
    e = S.StateVector(n, "enc2b")
    e.encode_from(s)
    d = S.StateVector(n, "c64")
    e.decode_to(d)
    got = e.expect_pauli()
    ref = oracle_expect(orc, d.to_numpy().astype(np.complex128))
    assert np.max(np.abs(got - ref)) <= 2e-6


def test_uniform_32q_paper_values(S, orc):
    """Sec. 3: for the uniform superposition <Q_x(i)> = 0 and <Q_y(i)> =
    <Q_z(i)> = 1/2 for every qubit (tests/golden/uniform_expectations.txt),
    here at 32 qubits (32 GiB, complex64)."""
    import torch

    n = 32
    if torch.cuda.mem_get_info()[0] < (40 << 30):
        pytest.skip("not enough device memory")
    s = S.StateVector(n, "c64")
    s.run(C.uniform_circuit(n), "tiled")
    sig = s.expect_pauli() / s.norm()
    q = (1 - sig) / 2
    assert np.max(np.abs(q[:, 0] - 0.0)) < 1e-5
    assert np.max(np.abs(q[:, 1:] - 0.5)) < 1e-5


@pytest.mark.parametrize("dtype", ["c64", "c128", "enc2b"])
def test_ghz(S, dtype):
    """GHZ (Secs. 3-4): <sigma^x_i> = <sigma^y_i> = <sigma^z_i> = 0 for every
    qubit of an n >= 2 chain."""
    n = 20
    s = S.StateVector(n, "c64" if dtype == "enc2b" else dtype)
    s.run(C.ghz_circuit(n), "pergate")
    if dtype == "enc2b":
        e = S.StateVector(n, "enc2b")
        e.encode_from(s)
        s = e
    assert np.max(np.abs(s.expect_pauli())) < 1e-6
