"""GPU parity of the tiled multi-gate passes against the CPU oracle (same
tolerances as the per-gate path), from one tile (13 qubits) upwards, with
every gate kind of the circuit format, and at the benchmark sizes through
closed forms and the inverse-circuit round trip."""

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


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,depth,seed", [(13, 12, 1), (14, 20, 2), (16, 20, 3), (20, 20, 1), (22, 16, 4)])
def test_random_circuit(S, orc, dtype, n, depth, seed):
    c = C.random_circuit(n, depth, seed)
    ref = orc.run(c)
    s = S.StateVector(n, dtype)
    p = s.plan(c, "tiled")
    assert p.passes < len(c)
    p.execute()
    check(dtype, s.to_numpy(), ref)
    p.free()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,seed", [(13, 5), (15, 6), (18, 7)])
def test_every_gate_kind(S, orc, dtype, n, seed):
    """U, P, S, T, X, Y, Z, SX/SY and adjoints, CZ, CX, CP, SWAP on random
    qubits: exercises general, structured, controlled and diagonal ops with
    conditions on register, thread and CTA index bits."""
    c = C.random_unitary_gates(n, 400, seed)
    ref = orc.run(c)
    s = S.StateVector(n, dtype)
    s.run(c, "tiled")
    check(dtype, s.to_numpy(), ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_ghz_qft_uniform(S, orc, dtype):
    n = 18
    for c in (C.ghz_circuit(n), C.qft_circuit(n, 0x2B6D1), C.uniform_circuit(n)):
        s = S.StateVector(n, dtype)
        s.run(c, "tiled")
        check(dtype, s.to_numpy(), orc.run(c))


def test_small_state_uses_per_gate_path(S, orc):
    c = C.random_circuit(8, 6, 2)
    s = S.StateVector(8, "c64")
    p = s.plan(c, "tiled")
    assert p.passes == p.gates  # below one tile every launch is a per-gate update
    p.execute()
    check("c64", s.to_numpy(), orc.run(c))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_24q_against_oracle(S, orc, dtype):
    c = C.random_circuit(24, 16, 1)
    s = S.StateVector(24, dtype)
    s.run(c, "tiled")
    check(dtype, s.to_numpy(), orc.run(c))


def test_tiled_equals_pergate_c64(S):
    c = C.random_circuit(22, 16, 9)
    a = S.StateVector(22, "c64")
    a.run(c, "tiled")
    b = S.StateVector(22, "c64")
    b.run(c, "pergate")
    x, y = a.to_numpy().astype(np.complex128), b.to_numpy().astype(np.complex128)
    assert np.max(np.abs(x - y)) < 1e-6
    assert 1 - fidelity(x, y) < 1e-6


def test_benchmark_size_32q(S):
    """The 32-qubit benchmark workload: the depth-24 random circuit followed
    by its inverse returns to |0...0> (1 - F <= 1e-5), and the 32-qubit QFT of
    a basis state matches its closed form at sampled outputs."""
    import torch

    n = 32
    if torch.cuda.mem_get_info()[0] < (8 << n) + (4 << 30):
        pytest.skip("not enough device memory")
    s = S.StateVector(n, "c64")
    c = C.random_circuit(n, 24, 1)
    s.run(c, "tiled")
    assert abs(s.norm() - 1) < 1e-4
    s.run(C.inverse_circuit(c), "tiled")
    a = s.amplitudes([0, 1, 12345, (1 << n) - 1])
    assert 1 - abs(a[0]) ** 2 <= TOL_C64_F
    assert np.max(np.abs(a[1:])) <= TOL_C64_AMP
    x = 0x9E3779B9
    s.set_basis(x)
    s.run(C.qft_circuit(n), "tiled")
    y = np.random.default_rng(2).integers(0, 1 << n, size=4096, dtype=np.uint64)
    got = s.amplitudes(y)
    ph = ((x * y.astype(object)) % (1 << n)).astype(np.float64) / (1 << n)
    expect = np.exp(2j * np.pi * ph) / math.sqrt(1 << n)
    assert np.max(np.abs(got - expect)) <= TOL_C64_AMP
    del s
    torch.cuda.empty_cache()


@pytest.mark.parametrize("mode", ["tiled", "fused"])
def test_32q_random_amplitudes_vs_oracle(S, orc, mode):
    """Random-circuit amplitudes at the benchmark size: the 32-qubit circuit
    of the benchmark family (depth 12, seed 5) in complex64, 64 sampled
    amplitudes against the oracle's exact Eq. 3 evaluation of the same
    amplitudes (qubits 0-15 | 16-31: the 6 CZs on the edge (15, 16) are
    decomposed, 64 branches of 16-qubit states), which the CPU tests pin to
    the full state.  A wrong qubit in a tile slot or a lost phase shows here
    even where a circuit and its inverse would cancel it."""
    import torch

    n = 32
    if torch.cuda.mem_get_info()[0] < (36 << 30):
        pytest.skip("needs 36 GiB of device memory")
    c = C.random_circuit(n, 12, 5)
    z = C.random_bitstrings(64, n, 3)
    ref, cuts = orc.cut_amplitudes(c, (1 << 16) - 1, z)
    assert cuts == 6
    s = S.StateVector(n, "c64")
    s.run(c, mode)
    got = s.amplitudes(z)
    rms = float(np.sqrt(np.mean(np.abs(ref) ** 2)))
    err = float(np.max(np.abs(got - ref)))
    assert err <= TOL_C64_AMP  # the complex64 bound (norm 1)
    # and a relative one at this amplitude size: FP32 butterflies (tiled), or
    # split-BF16 products of about 2^-16 relative error each, over some 30
    # dense blocks (fused)
    assert err <= (2e-5 if mode == "tiled" else 2e-4) * rms, (err, rms)
    s.free()
    del s
    torch.cuda.empty_cache()


def test_30q_c128_roundtrip(S):
    n = 30
    s = S.StateVector(n, "c128")
    c = C.random_circuit(n, 16, 1)
    s.run(c, "tiled")
    s.run(C.inverse_circuit(c), "tiled")
    a = s.amplitudes([0, 5, (1 << n) - 1])
    assert abs(a[0] - 1) < 1e-11 and np.max(np.abs(a[1:])) < 1e-11


@pytest.mark.parametrize("ctas", ["1", "3"])
def test_register_budget_variants(S, orc, monkeypatch, ctas):
    """The pass kernels compiled for 1 or 3 resident CTAs per SM
    (SV_TILE_CTAS: 255 or 85 registers per thread, the latter with spills)
    give the same states as the default of 2."""
    monkeypatch.setenv("SV_TILE_CTAS", ctas)
    c = C.random_circuit(21, 10, 11)
    s = S.StateVector(21, "c64")
    s.run(c, "tiled")
    check("c64", s.to_numpy(), orc.run(c))


@pytest.mark.parametrize("n", [12, 13, 21])
def test_twelve_bit_tiles(S, orc, monkeypatch, n):
    """Passes on 2^12-amplitude tiles (SV_TILE_M=12: 128-thread CTAs, four
    per SM) give the same states as the default 2^13 tiles, from one tile
    upwards."""
    monkeypatch.setenv("SV_TILE_M", "12")
    monkeypatch.setenv("SV_TILE_CTAS", "4")
    c = C.random_circuit(n, 10, 17)
    s = S.StateVector(n, "c64")
    s.run(c, "tiled")
    check("c64", s.to_numpy(), orc.run(c))


@pytest.mark.parametrize("rb", ["4", "6"])
def test_register_qubit_variants(S, orc, monkeypatch, rb):
    """Passes generated for 4 or 6 register qubits per thread (SV_TILE_RB:
    512- or 128-thread CTAs, other register sets and segment boundaries) give
    the same states as the default of 5."""
    monkeypatch.setenv("SV_TILE_RB", rb)
    c = C.random_circuit(21, 10, 13)
    s = S.StateVector(21, "c64")
    s.run(c, "tiled")
    check("c64", s.to_numpy(), orc.run(c))


@pytest.mark.parametrize("direct", ["0", "1"])
@pytest.mark.parametrize("n,depth,seed", [(13, 8, 21), (20, 12, 22), (24, 16, 23)])
def test_hbm_io_forms(S, orc, monkeypatch, direct, n, depth, seed):
    """The forms of a pass's HBM access give the same states: whole tiles
    staged through shared memory (SV_TILE_DIRECT=0), and persistent CTAs that
    copy the next tile into shared memory while the last segment computes
    (SV_TILE_PREFETCH=1; with 2^(n-13) tiles over the resident CTAs, from one
    tile to many per CTA)."""
    monkeypatch.setenv("SV_TILE_DIRECT", direct)
    monkeypatch.setenv("SV_TILE_PREFETCH", "1")
    c = C.random_circuit(n, depth, seed)
    s = S.StateVector(n, "c64")
    s.run(c, "tiled")
    check("c64", s.to_numpy(), orc.run(c))
    p = s.plan(c, "tiled")
    for _ in range(3):  # direct launches, then the captured graph, then its replay
        s.set_basis(0)
        p.execute()
        check("c64", s.to_numpy(), orc.run(c))
    p.free()


def test_plan_cache_reuse(S, orc):
    """Tiled plans are cached by circuit text (with the device, dtype, qubit
    count and planner settings in the key): running the same text again on a
    second state, in complex128, and the same gates on a larger state gives
    the oracle's state every time; a text for another qubit count is still
    refused."""
    c = C.random_circuit(15, 12, 21)
    text = c.text()
    ref = orc.run(c)
    for _ in range(2):
        s = S.StateVector(15, "c64")
        s.run(text, "tiled")
        check("c64", s.to_numpy(), ref)
    s = S.StateVector(15, "c128")
    s.run(text, "tiled")
    check("c128", s.to_numpy(), ref)
    # the same gates declared for 17 qubits: another text, another plan
    big = C.Circuit(17)
    big.gates = list(c.gates)
    s = S.StateVector(17, "c64")
    s.run(big.text(), "tiled")
    check("c64", s.to_numpy(), orc.run(big))
    # a text declaring 15 qubits is refused on a 17-qubit state, cached or not
    with pytest.raises(S.SVError):
        s.run(text, "tiled")
