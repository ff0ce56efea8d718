"""GPU two-byte code against the CPU codec mirror: codes and scales must be
bit-exact (integer/byte work); fidelity against the exact oracle is
measured and reported."""

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


def raw_of(codes, scales):
    return np.concatenate([codes.view(np.uint8), scales.view(np.uint8)])


def split_raw(raw, n):
    codes = raw[: 2 << n].view(np.int8)
    scales = raw[2 << n:].view(np.float32)
    return codes, scales


def rand_c64(n, seed, zero_block=True):
    rng = np.random.default_rng(seed)
    psi = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    if zero_block and n >= 9:
        psi[256:512] = 0
    return psi


@pytest.mark.parametrize("n", [1, 3, 7, 8, 9, 12])
def test_encode_decode_bit_exact(S, orc, n):
    psi = rand_c64(n, n)
    src = S.StateVector(n, "c64")
    src.from_numpy(psi)
    enc = S.StateVector(n, "enc2b")
    enc.encode_from(src)
    codes, scales = enc.codes()
    rc, rs = orc.enc_encode(psi)
    assert np.array_equal(codes, rc)
    assert np.array_equal(scales.view(np.uint32), rs.view(np.uint32))
    dst = S.StateVector(n, "c64")
    enc.decode_to(dst)
    got = dst.to_numpy()
    ref = orc.enc_decode(rc, rs)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("n", [4, 10])
def test_gate_every_target_control_bit_exact(S, orc, n):
    psi = rand_c64(n, 77 + n)
    codes, scales = orc.enc_encode(psi)
    enc = S.StateVector(n, "enc2b")
    mats = [orc.gate_matrix(k) for k in ("H", "SX", "SY", "T", "X", "Z")]
    rng = np.random.default_rng(n)
    z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    mats.append(np.linalg.qr(z)[0])
    mats.append(np.diag([1.0, np.exp(0.3j)]))  # a phase (u00 = 1) other than T
    for u in mats:
        for t in range(n):
            for c in [-1] + [q for q in range(n) if q != t]:
                enc.from_numpy(raw_of(codes, scales))
                enc.apply_gate(t, u, control=c)
                gc, gs = enc.codes()
                rc, rs = orc.enc_apply_gate(codes, scales, t, c, u)
                assert np.array_equal(gc, rc), (t, c)
                assert np.array_equal(gs.view(np.uint32), rs.view(np.uint32)), (t, c)


@pytest.mark.parametrize("n,depth,seed", [(6, 6, 1), (16, 8, 2), (18, 12, 3)])
def test_random_circuit_bit_exact(S, orc, n, depth, seed):
    c = C.random_circuit(n, depth, seed)
    rc, rs = orc.enc_run(c)
    enc = S.StateVector(n, "enc2b")
    enc.run(c, "pergate")
    gc, gs = enc.codes()
    assert np.array_equal(gc, rc)
    assert np.array_equal(gs.view(np.uint32), rs.view(np.uint32))


def test_qft_and_ghz_bit_exact(S, orc):
    n = 12
    for c in (C.qft_circuit(n, 0x5A5), C.ghz_circuit(n)):
        rc, rs = orc.enc_run(c)
        enc = S.StateVector(n, "enc2b")
        enc.run(c)
        gc, gs = enc.codes()
        assert np.array_equal(gc, rc) and np.array_equal(gs, rs)


def test_uniform_exact_large(S):
    """Sec. 3: the code represents the uniform superposition exactly (all
    codes 127), here at 28 qubits."""
    n = 28
    enc = S.StateVector(n, "enc2b")
    enc.run(C.uniform_circuit(n))
    codes, scales = enc.codes()
    assert np.all(codes[0::2] == 127) and np.all(codes[1::2] == 0)
    assert np.all(scales == scales[0])
    nrm = enc.norm()
    assert abs(nrm / ((1 << n) * float(scales[0]) ** 2) - 1) < 1e-12


def test_fidelity_24q(S, orc, record_property):
    """Fidelity of the encoded simulation against the FP64 oracle on a
    24-qubit instance of the depth-12 random circuit (measured, reported)."""
    n = 24
    c = C.random_circuit(n, 12, 1)
    exact = orc.run(c)
    enc = S.StateVector(n, "enc2b")
    enc.run(c)
    dec = S.StateVector(n, "c64")
    enc.decode_to(dec)
    got = dec.to_numpy().astype(np.complex128)
    f = abs(np.vdot(exact, got)) ** 2 / (np.vdot(exact, exact).real * np.vdot(got, got).real)
    record_property("fidelity_enc2b_24q_d12", f)
    print(f"enc2b fidelity 24q d12: {f:.6f}")
    assert f > 0.95


@pytest.mark.parametrize("n,seed", [(9, 1), (12, 2), (14, 3)])
def test_in_block_runs_bit_exact(S, orc, n, seed):
    """Runs of consecutive in-block gates and sign flips applied in one pass
    each (the default per-gate plan of the two-byte code) give the CPU codec
    mirror's codes: every gate kind of the format on random qubits, so runs
    hold controls inside and outside the blocks, X, P, U and CZ/CP flips, and
    runs are broken by gates across blocks."""
    c = C.random_unitary_gates(n, 400, 50 + seed)
    layer_like = C.random_circuit(n, 8, seed)  # long runs: in-block layers and CZ rows
    for circ in (c, layer_like):
        rc, rs = orc.enc_run(circ)
        enc = S.StateVector(n, "enc2b")
        plan = enc.plan(circ, "pergate")
        kinds = {name for name, _ in plan.launch_info()}
        plan.execute()
        gc, gs = enc.codes()
        assert np.array_equal(gc, rc), n
        assert np.array_equal(gs.view(np.uint32), rs.view(np.uint32)), n
        plan.free()
    assert "k_enc_run_in" in kinds


def test_in_block_runs_equal_one_pass_per_gate(S, monkeypatch):
    """At 22 qubits (beyond the mirror's quick range) the fused runs and one
    pass per gate (SV_ENC_RUNS=0) write the same codes and scales."""
    n = 22
    c = C.random_circuit(n, 6, 8)
    out = []
    for runs in ("1", "0"):
        monkeypatch.setenv("SV_ENC_RUNS", runs)
        enc = S.StateVector(n, "enc2b")
        enc.run(c, "pergate")
        out.append(enc.codes())
        enc.free()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1].view(np.uint32), out[1][1].view(np.uint32))
