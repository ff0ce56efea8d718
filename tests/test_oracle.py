"""Pins for the CPU oracle: closed forms, the paper's printed values,
brute force and invariants.  No GPU; each check is chosen so that a dropped
term, a wrong sign, a wrong index or a transposed operand in the oracle fails
at least one of them."""

import cmath
import math
import os

import numpy as np
import pytest

from paper_1912_03243_gb300 import circuits as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- gate table

PAULI = {
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


def test_gate_table_algebra(orc):
    g = {k: orc.gate_matrix(k) for k in C.ONE_QUBIT}
    eye = np.eye(2)
    for k, m in g.items():
        assert np.allclose(m.conj().T @ m, eye, atol=1e-15), k
        assert np.allclose(g[C.ADJOINT[k]] @ m, eye, atol=1e-15), k
    for k in "XYZ":
        assert np.allclose(g[k], PAULI[k], atol=0)
    # principal square roots and the Clifford+T relations
    assert np.allclose(g["SX"] @ g["SX"], PAULI["X"], atol=1e-15)
    assert np.allclose(g["SY"] @ g["SY"], PAULI["Y"], atol=1e-15)
    assert np.allclose(g["T"] @ g["T"], g["S"], atol=1e-15)
    assert np.allclose(g["S"] @ g["S"], PAULI["Z"], atol=1e-15)
    assert np.allclose(g["H"] @ PAULI["X"] @ g["H"], PAULI["Z"], atol=1e-15)
    # eigenvalues of the principal roots are {1, i}
    for k in ("SX", "SY"):
        ev = sorted(np.linalg.eigvals(g[k]), key=lambda z: z.imag)
        assert np.allclose(ev, [1, 1j], atol=1e-15), k
    assert np.allclose(orc.gate_matrix("P", [0.3]), np.diag([1, cmath.exp(0.3j)]), atol=1e-16)


def test_two_qubit_gate_table(orc):
    # local index = bit(first qubit) + 2 * bit(second qubit)
    cz = orc.gate_matrix("CZ")
    assert np.allclose(cz, np.diag([1, 1, 1, -1]))
    cx = orc.gate_matrix("CX")
    # control = first qubit (LSB), target = second: |c=1,t=0> (1) <-> |c=1,t=1> (3)
    e = np.eye(4)
    assert np.allclose(cx, e[[0, 3, 2, 1]])
    sw = orc.gate_matrix("SWAP")
    assert np.allclose(sw, e[[0, 2, 1, 3]])
    assert np.allclose(orc.gate_matrix("CP", [0.7]), np.diag([1, 1, 1, cmath.exp(0.7j)]))


# ------------------------------------------------------- paper's closed forms

@pytest.mark.parametrize("n", [1, 2, 5, 10, 14])
def test_uniform_superposition(orc, n):
    """Sec. 3: H on every qubit gives 2^{-n/2} on every basis state and the
    validation observable <Q_alpha(i)> = (1 - <sigma^alpha_i>)/2 takes the
    values printed in the paper."""
    psi = orc.run(C.uniform_circuit(n))
    assert np.allclose(psi, 2.0 ** (-n / 2), rtol=1e-14, atol=0)
    golden = {a: float(v) for a, v in _golden("uniform_expectations.txt")}
    for i in sorted({0, n // 2, n - 1}):
        for a in "xyz":
            q = (1.0 - orc.expect_pauli(psi, i, a)) / 2.0
            assert abs(q - golden[a]) < 1e-13, (i, a, q)


@pytest.mark.parametrize("n,seed", [(1, 3), (4, 5), (7, 11)])
def test_expect_pauli_product_states(orc, n, seed):
    """For a product state psi = phi_{n-1} (x) ... (x) phi_0 (qubit j = index
    bit j) the expectation values of qubit j are its Bloch vector, from its
    own two amplitudes (a, b): <sigma^x> = 2 Re(conj(a) b), <sigma^y> =
    2 Im(conj(a) b), <sigma^z> = |a|^2 - |b|^2 (sigma^y = [[0, -i], [i, 0]]).
    Random phases make every sign matter."""
    rng = np.random.default_rng(seed)
    phis = []
    for _ in range(n):
        v = rng.normal(size=2) + 1j * rng.normal(size=2)
        phis.append(v / np.linalg.norm(v))
    psi = np.array([1.0 + 0j])
    for j in range(n):
        psi = np.kron(phis[j], psi)  # qubit j becomes the more significant factor
    for j, (a, b) in enumerate(phis):
        want = {"x": 2 * (np.conj(a) * b).real, "y": 2 * (np.conj(a) * b).imag, "z": abs(a) ** 2 - abs(b) ** 2}
        for alpha in "xyz":
            assert abs(orc.expect_pauli(psi, j, alpha) - want[alpha]) < 1e-13, (j, alpha)


def test_expect_pauli_basis_and_eigenstates(orc):
    """Basis state |b>: <sigma^z_i> = 1 - 2 b_i, <sigma^x_i> = <sigma^y_i> = 0;
    single-qubit eigenstates |+>, |->, |+i>, |-i> give +-1 on their axis."""
    n, b = 6, 0b101100
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[b] = 1.0
    for i in range(n):
        assert orc.expect_pauli(psi, i, "z") == 1 - 2 * ((b >> i) & 1)
        assert orc.expect_pauli(psi, i, "x") == 0 and orc.expect_pauli(psi, i, "y") == 0
    r = 1 / math.sqrt(2)
    for state, axis, val in (([r, r], "x", 1), ([r, -r], "x", -1), ([r, 1j * r], "y", 1), ([r, -1j * r], "y", -1)):
        assert abs(orc.expect_pauli(np.array(state, dtype=np.complex128), 0, axis) - val) < 1e-15


@pytest.mark.parametrize("n", [2, 3, 8, 16])
def test_ghz(orc, n):
    """Sec. 3: H(0) + CNOT chain gives (|0..0> + |1..1>)/sqrt(2)."""
    psi = orc.run(C.ghz_circuit(n))
    rows = {r[0]: complex(float(r[1]), float(r[2])) for r in _golden("ghz_amplitudes.txt")}
    assert abs(psi[0] - rows["zeros"]) < 1e-15
    assert abs(psi[-1] - rows["ones"]) < 1e-15
    rest = psi[1:-1]
    assert np.all(rest == 0)


@pytest.mark.parametrize("n,x", [(1, 1), (3, 5), (5, 0), (6, 41), (8, 0x9E)])
def test_qft_closed_form(orc, n, x):
    """QFT|x> = 2^{-n/2} sum_y exp(2 pi i x y / 2^n) |y> (textbook closed form)."""
    psi = orc.run(C.qft_circuit(n, x))
    y = np.arange(1 << n)
    expect = np.exp(2j * np.pi * ((x * y) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
    assert np.max(np.abs(psi - expect)) < 1e-13


def test_memory_formula():
    """Sec. 1: an N-qubit complex128 state needs 2^{N+4} bytes; 45 qubits need
    slightly more than 0.5 PB."""
    assert (1 << 45) * 16 == 2 ** (45 + 4)
    assert 2 ** 49 > 0.5e15


# ------------------------------------------------------------ brute force

@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3), (4, 4), (5, 5), (6, 6)])
def test_sparse_matches_dense(orc, n, seed):
    """Eq. 1 loops against the full 2^n x 2^n product, column by column."""
    c = C.random_unitary_gates(n, 40, seed)
    U = orc.dense(c)
    assert np.allclose(U.conj().T @ U, np.eye(1 << n), atol=1e-12)
    for j in range(1 << n):
        col = orc.run(c, psi=orc.basis_state(n, j))
        assert np.max(np.abs(col - U[:, j])) < 1e-13


def _kron_full(n, q, u):
    """Full matrix of a 1-qubit gate by numpy.kron (qubit n-1 leftmost)."""
    m = np.eye(1)
    for k in range(n - 1, -1, -1):
        m = np.kron(m, u if k == q else np.eye(2))
    return m


def test_dense_matches_numpy_kron(orc):
    """Single-qubit and neighbouring two-qubit gates: the oracle's dense
    builder equals the Kronecker product written with numpy."""
    n = 4
    rng = np.random.default_rng(0)
    for name in C.ONE_QUBIT:
        for q in range(n):
            c = C.Circuit(n)
            c.add(name, q)
            assert np.allclose(orc.dense(c), _kron_full(n, q, orc.gate_matrix(name)), atol=1e-15)
    # CX(q, q+1): the 4x4 in the (target, control) = (hi, lo) kron basis
    for q in range(n - 1):
        c = C.Circuit(n)
        c.add("CX", q, q + 1)
        m = np.eye(1)
        cx = np.array([[1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0], [0, 1, 0, 0]])  # rows: t*2+c
        for k in range(n - 1, -1, -1):
            if k == q + 1:
                m = np.kron(m, cx)
            elif k == q:
                continue
            else:
                m = np.kron(m, np.eye(2))
        assert np.allclose(orc.dense(c), m)
    # a random unitary gate on qubit 2
    z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    u, _ = np.linalg.qr(z)
    c = C.Circuit(n)
    c.add("U", 2, params=tuple(v for x in u.reshape(-1) for v in (x.real, x.imag)))
    assert np.allclose(orc.dense(c), _kron_full(n, 2, u), atol=1e-15)


def test_apply_kq_against_single_gates(orc):
    n = 6
    psi = C.random_state(n, 11)
    rng = np.random.default_rng(3)
    z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    u0, _ = np.linalg.qr(z)
    z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    u1, _ = np.linalg.qr(z)
    # k = 1 equals the 1-qubit update
    assert np.allclose(orc.apply_kq(psi, [4], u0), orc.apply_1q(psi, 4, u0), atol=1e-15)
    # k = 2 with kron(u1, u0) (qubits[0] is the low local bit) equals u0 on q0 then u1 on q1
    ref = orc.apply_1q(orc.apply_1q(psi, 1, u0), 5, u1)
    assert np.allclose(orc.apply_kq(psi, [1, 5], np.kron(u1, u0)), ref, atol=1e-14)
    # swapping the qubit order transposes the local index
    assert np.allclose(orc.apply_kq(psi, [5, 1], np.kron(u0, u1)), ref, atol=1e-14)
    # k = 3: against the dense definition
    z = rng.normal(size=(8, 8)) + 1j * rng.normal(size=(8, 8))
    u3, _ = np.linalg.qr(z)
    qs = [3, 0, 4]
    out = orc.apply_kq(psi, qs, u3)
    expect = np.zeros_like(psi)
    for i in range(1 << n):
        li = sum(((i >> q) & 1) << j for j, q in enumerate(qs))
        base = i & ~sum(1 << q for q in qs)
        for lj in range(8):
            jdx = base | sum(((lj >> j) & 1) << q for j, q in enumerate(qs))
            expect[i] += u3[li, lj] * psi[jdx]
    assert np.allclose(out, expect, atol=1e-14)


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("n,depth,seed", [(8, 6, 1), (12, 10, 2), (20, 20, 1)])
def test_norm_and_inverse(orc, n, depth, seed):
    c = C.random_circuit(n, depth, seed)
    psi = orc.run(c)
    assert abs(orc.norm(psi) - 1.0) < 1e-13
    back = orc.run(C.inverse_circuit(c), psi=psi)
    assert abs(back[0] - 1.0) < 1e-12
    assert np.max(np.abs(back[1:])) < 1e-12


def test_circuit_gate_counts():
    """Gate counts of the benchmark circuit family."""
    for (n, d), g in {(20, 20): 590, (30, 16): 712, (24, 16): 568, (32, 24): 1140, (35, 12): 624}.items():
        assert len(C.random_circuit(n, d, 1)) == g
    q = C.qft_circuit(32)
    assert len(q) == 32 + 496 + 16


def test_parse_errors(orc):
    with pytest.raises(orc.OracleError):
        orc.run("qubits 2\nFOO 0\n", 2)
    with pytest.raises(orc.OracleError):
        orc.run("qubits 2\nCZ 0 0\n", 2)
    with pytest.raises(orc.OracleError):
        orc.run("qubits 2\nH 2\n", 2)


# -------------------------------------------------------- decomposition (Sec. 4)

def test_eq2_root_and_identity(orc):
    x, dplus, dminus = orc.eq2_terms()
    (re, im), = [(float(a), float(b)) for a, b in _golden("eq2_root.txt")]
    assert abs(x - complex(re, im)) < 1e-15
    assert abs(cmath.cos(2 * x) - 1j) < 1e-15
    # 1/2 sum_s D_s (x) D_s = CZ (Eq. 2), as a 4x4 matrix
    m = 0.5 * (np.kron(np.diag(dplus), np.diag(dplus)) + np.kron(np.diag(dminus), np.diag(dminus)))
    assert np.allclose(m, np.diag([1, 1, 1, -1]), atol=1e-15)
    # the closed forms: D_+ = diag(r, 1/r), D_- = diag(-i/r, i r), r = sqrt(1+sqrt 2)
    r = math.sqrt(1 + math.sqrt(2))
    assert np.allclose(dplus, [r, 1 / r], atol=1e-15)
    assert np.allclose(dminus, [-1j / r, 1j * r], atol=1e-15)
    # CZ is diag(e^{i pi (1 + z_i z_j - z_i - z_j)/4}) (Sec. 4)
    for zi in (1, -1):
        for zj in (1, -1):
            assert abs(cmath.exp(1j * math.pi * (1 + zi * zj - zi - zj) / 4) - (-1 if zi == zj == -1 else 1)) < 1e-15


def _all_z(n):
    return np.arange(1 << n, dtype=np.uint64)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("rows,cols,rows_a,depth,seed", [(2, 3, 1, 6, 1), (3, 4, 1, 8, 2), (4, 3, 2, 12, 3)])
def test_cut_matches_full_state(orc, form, rows, cols, rows_a, depth, seed):
    """Eq. 3 branch sum over all 2^n bit strings equals the full state."""
    c = C.grid_circuit(rows, cols, depth, seed)
    mask = C.grid_partition_mask(rows, cols, rows_a)
    full = orc.run(c)
    amps, s = orc.cut_amplitudes(c, mask, _all_z(c.n), form=form)
    assert s > 0
    assert np.max(np.abs(amps - full)) < 1e-12


@pytest.mark.parametrize("form", [0, 1])
def test_cut_with_cx_and_cp(orc, form):
    """A CNOT across the cut is rewritten as H CZ H; CP works in the projector form."""
    n = 6
    c = C.random_unitary_gates(n, 30, 9)
    # keep only gates the decomposition supports across the cut {0,1,2} | {3,4,5}
    keep = C.Circuit(n)
    for name, qs, ps in c.gates:
        if name == "SWAP":
            continue
        if form == 1 and name == "CP" and ((qs[0] < 3) != (qs[1] < 3)):
            continue
        keep.add(name, *qs, params=ps)
    full = orc.run(keep)
    amps, s = orc.cut_amplitudes(keep, 0b000111, _all_z(n), form=form)
    assert s > 0
    assert np.max(np.abs(amps - full)) < 1e-12


@pytest.mark.parametrize("n", [16, 40])
def test_cut_ghz_paper_values(orc, n):
    """Sec. 4 (Fig. 3 discussion): with the GHZ chain cut between the halves,
    the coefficients of |0..0> and |1..1> are 1/sqrt(2)."""
    c = C.ghz_circuit(n)
    mask = (1 << (n // 2)) - 1
    z = np.array([0, (1 << n) - 1, 1, 1 << (n - 1)], dtype=np.uint64)
    rows = {r[0]: complex(float(r[1]), float(r[2])) for r in _golden("ghz_amplitudes.txt")}
    for form in (0, 1):
        amps, s = orc.cut_amplitudes(c, mask, z, form=form)
        assert s == 1
        assert abs(amps[0] - rows["zeros"]) < 1e-14
        assert abs(amps[1] - rows["ones"]) < 1e-14
        assert np.max(np.abs(amps[2:])) < 1e-14


def test_cut_rejects_swap_across(orc):
    c = C.Circuit(4)
    c.add("SWAP", 0, 3)
    with pytest.raises(orc.OracleError):
        orc.cut_amplitudes(c, 0b0011, np.array([0], dtype=np.uint64))


# --------------------------------------------------- two-byte codec mirror

def test_codec_uniform_state_exact(orc):
    """Sec. 3: the encoding represents the uniform superposition exactly: all
    codes are +127 (real) and 0 (imag), and every block has the same scale."""
    for n in (4, 8, 11):
        codes, scales = orc.enc_run(C.uniform_circuit(n))
        cr = codes.reshape(-1, 2)
        assert np.all(cr[:, 0] == 127) and np.all(cr[:, 1] == 0)
        assert np.all(scales == scales[0])
        psi = orc.enc_decode(codes, scales).astype(np.complex128)
        psi /= math.sqrt(orc.norm(psi))
        for a, v in (("x", 0.0), ("y", 0.5), ("z", 0.5)):
            q = (1 - orc.expect_pauli(psi, 0, a)) / 2
            assert abs(q - v) < 1e-12


def test_codec_ghz_and_basis_exact(orc):
    for n in (3, 9, 12):
        codes, scales = orc.enc_run(C.ghz_circuit(n))
        psi = orc.enc_decode(codes, scales)
        nz = np.flatnonzero(psi)
        assert list(nz) == [0, (1 << n) - 1]
        assert psi[0] == psi[-1]
    codes, scales = orc.enc_zero_state(10)
    assert codes[0] == 127 and np.all(codes[1:] == 0) and scales[0] == 1.0 and np.all(scales[1:] == 0)


def test_codec_roundtrip_bounds(orc):
    rng = np.random.default_rng(5)
    n = 12
    psi = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    psi[256:512] = 0  # one all-zero block
    codes, scales = orc.enc_encode(psi)
    assert scales[1] == 0 and np.all(codes[512:1024] == 0)
    dec = orc.enc_decode(codes, scales)
    blk = np.repeat(scales, 256)
    err = np.maximum(np.abs(dec.real - psi.real), np.abs(dec.imag - psi.imag))
    # half a quantisation step plus FP32 rounding
    assert np.all(err <= blk / 254 * (1 + 1e-5) + 1e-30)
    # the largest component of each nonzero block codes to +-127 and decodes exactly
    cr = codes.reshape(-1, 512)
    for b in range(len(scales)):
        if scales[b] > 0:
            assert np.max(np.abs(cr[b].astype(int))) == 127
    # decode -> encode is the identity on codes and scales
    codes2, scales2 = orc.enc_encode(dec)
    assert np.array_equal(codes2, codes) and np.array_equal(scales2, scales)
    assert np.all(np.abs(codes.astype(int)) <= 127)


def test_codec_permutation_gates_exact(orc):
    """X permutes codes; Z negates the codes of the flipped half (no rounding)."""
    rng = np.random.default_rng(6)
    n = 10
    psi = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    codes, scales = orc.enc_encode(psi)
    for t in (0, 3, 8, 9):
        cx, sx = orc.enc_apply_gate(codes, scales, t, -1, orc.gate_matrix("X"))
        idx = np.arange(1 << n) ^ (1 << t)
        dec = orc.enc_decode(codes, scales)
        assert np.array_equal(orc.enc_decode(cx, sx), dec[idx])
        cz, sz = orc.enc_apply_gate(codes, scales, t, -1, orc.gate_matrix("Z"))
        sign = np.where((np.arange(1 << n) >> t) & 1, -1, 1)
        assert np.array_equal(cz.reshape(-1, 2), codes.reshape(-1, 2) * sign[:, None])
        assert np.array_equal(sz, scales)


def test_codec_gate_close_to_exact(orc):
    """One encoded gate equals the complex128 gate on the decoded input to
    within one quantisation step of the output block."""
    rng = np.random.default_rng(7)
    n = 10
    psi = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    codes, scales = orc.enc_encode(psi)
    dec = orc.enc_decode(codes, scales).astype(np.complex128)
    for name in ("H", "SX", "SY", "T"):
        u = orc.gate_matrix(name)
        for t, ctl in ((0, -1), (5, 2), (9, -1), (8, 9)):
            c2, s2 = orc.enc_apply_gate(codes, scales, t, ctl, u)
            ref = dec.copy()
            if ctl < 0:
                ref = orc.apply_1q(ref, t, u)
            else:
                cu = np.eye(4, dtype=complex)
                cu[np.ix_([1, 3], [1, 3])] = u  # local index ctl + 2 t, acts where ctl = 1
                ref = orc.apply_kq(ref, [ctl, t], cu)
            got = orc.enc_decode(c2, s2)
            blk = np.repeat(s2, 256)
            err = np.maximum(np.abs(got.real - ref.real), np.abs(got.imag - ref.imag))
            assert np.all(err <= blk / 254 + 2e-6 * blk), (name, t, ctl)


def test_codec_fidelity_random_circuit(orc):
    """Fidelity of the encoded simulation of a random circuit against the
    exact one.  The paper reports roughly three digits of precision for
    standard circuits (Sec. 1) but gives no format, so this is only a sanity
    floor for the int8/block-scale reading (measured: 1 - F = 1.2e-3 after
    140 gates at n = 12, one decode-gate-encode per gate)."""
    n = 12
    c = C.random_circuit(n, 8, 4)
    exact = orc.run(c)
    codes, scales = orc.enc_run(c)
    got = orc.enc_decode(codes, scales).astype(np.complex128)
    f = abs(np.vdot(exact, got)) ** 2 / (orc.norm(exact) * orc.norm(got))
    assert f > 0.995, f


# --------------------------------------------- P-partition decomposition

@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("rows,cols,depth,P", [(4, 3, 8, 4), (3, 4, 9, 3), (4, 3, 10, 2)])
def test_cut_multi_equals_full_state(orc, form, rows, cols, depth, P):
    """Sec. 4 over P partitions (row bands of a grid): every amplitude equals
    the full-state simulation, the plain definition of <z|C|0>."""
    c = C.grid_circuit(rows, cols, depth, 3)
    n = c.n
    band = -(-rows // P)
    part_of = [min((q // cols) // band, P - 1) for q in range(n)]
    amps, s = orc.cut_amplitudes_multi(c, part_of, list(range(1 << n)), form=form)
    assert s > 0
    assert np.max(np.abs(amps - orc.run(c))) < 1e-12


def test_cut_multi_parts_add_up(orc):
    c = C.grid_circuit(4, 3, 8, 5)
    part_of = [q // 3 for q in range(12)]
    z = list(range(1 << 12))
    full, s = orc.cut_amplitudes_multi(c, part_of, z)
    acc = sum(orc.cut_amplitudes_multi(c, part_of, z, part=p, nparts_log2=2)[0] for p in range(4))
    assert np.max(np.abs(acc - full)) < 1e-12


def test_cut_multi_ghz_128(orc):
    """Sec. 4: the 128-qubit GHZ chain in 8 partitions of 16 qubits (7 cut
    CNOTs, bit strings of two 64-bit words): <0...0|C|0> = <1...1|C|0> =
    1/sqrt(2), other coefficients 0."""
    n = 128
    c = C.ghz_circuit(n)
    idx = [0, (1 << n) - 1, 1, 1 << 64, (1 << 127) | 5, (1 << 64) - 1]
    for form in (0, 1):
        amps, s = orc.cut_amplitudes_multi(c, [q // 16 for q in range(n)], idx, form=form)
        assert s == 7
        assert np.allclose(amps[:2], 1 / math.sqrt(2), atol=1e-14)
        assert np.max(np.abs(amps[2:])) < 1e-14


# ------------------------------------------------------- input generators

def test_grid_circuit_structure():
    """The grid workload (reading R8): on a 6x8 grid at depth 8 the CZ
    patterns A B C D E F A B give 124 CZs; rows 0-2 | 3-5 are crossed only by
    the vertical edges (2, c)-(3, c) of C and D, S = 8, and each half keeps
    58 CZs; the 6x4 check grid has S = 4 at depth 8 and S = 8 at depth 12.
    Every layer's CZs act on disjoint qubits between grid neighbours, and the
    six patterns together hold every neighbour edge exactly once."""

    def counts(rows, cols, depth):
        c = C.grid_circuit(rows, cols, depth, 1)
        mask = C.grid_partition_mask(rows, cols, 3)
        cz = [qs for name, qs, _ in c.gates if name == "CZ"]
        cut = [e for e in cz if ((mask >> e[0]) & 1) != ((mask >> e[1]) & 1)]
        in_a = [e for e in cz if (mask >> e[0]) & 1 and (mask >> e[1]) & 1]
        return len(cz), len(cut), len(in_a), len(cz) - len(cut) - len(in_a)

    assert counts(6, 8, 8) == (124, 8, 58, 58)
    assert counts(6, 4, 8)[1] == 4 and counts(6, 4, 12)[1] == 8
    for rows, cols in ((6, 8), (5, 4), (3, 3)):
        seen = []
        for pat in "ABCDEF":
            edges = C.grid_edges(rows, cols, pat)
            qubits = [q for e in edges for q in e]
            assert len(qubits) == len(set(qubits)), pat  # one CZ per qubit per layer
            for a, b in edges:
                (ra, ca), (rb, cb) = divmod(a, cols), divmod(b, cols)
                assert abs(ra - rb) + abs(ca - cb) == 1  # grid neighbours
            seen += [tuple(sorted(e)) for e in edges]
        every = {(r * cols + c, r * cols + c + 1) for r in range(rows) for c in range(cols - 1)}
        every |= {(r * cols + c, (r + 1) * cols + c) for r in range(rows - 1) for c in range(cols)}
        assert sorted(seen) == sorted(every)


def test_random_circuit_structure():
    """The random family (reading R3): each layer is one gate from
    {H, T, SX, SY} on every qubit in ascending order, then CZ on (2i, 2i+1)
    in even layers and (2i+1, 2i+2) in odd layers; a seed fixes the circuit,
    and the draws use all four gates."""
    n, depth = 9, 6
    c = C.random_circuit(n, depth, 4)
    assert c.gates == C.random_circuit(n, depth, 4).gates
    assert c.gates != C.random_circuit(n, depth, 5).gates
    i, names = 0, set()
    for layer in range(depth):
        for q in range(n):
            name, qs, _ = c.gates[i]
            assert qs == (q,) and name in ("H", "T", "SX", "SY")
            names.add(name)
            i += 1
        start = 0 if layer % 2 == 0 else 1
        for a in range(start, n - 1, 2):
            assert c.gates[i][0] == "CZ" and c.gates[i][1] == (a, a + 1)
            i += 1
    assert i == len(c.gates) and names == {"H", "T", "SX", "SY"}
