"""Dense k-qubit blocks on the tensor cores (complex64, 3 x BF16 split
products, FP32 accumulation) against the oracle's k-qubit update, with the
complex64 tolerances (1 - F <= 1e-5, max |d amp| <= 1e-6 ||psi||); and the
bounded-wait failure path."""

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


def random_u(rng, d):
    z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def check_c64(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    nrm = math.sqrt(np.vdot(ref, ref).real)
    assert np.max(np.abs(got - ref)) <= 1e-6 * nrm
    f = abs(np.vdot(ref, got)) ** 2 / (np.vdot(ref, ref).real * np.vdot(got, got).real)
    assert 1 - f <= 1e-5


# The sets reach both tensor-core kernels and every epilogue form: blocks
# holding qubits 0..3 (pipeline, rows along the low qubits), blocks without
# qubit 0 at k = 6 (pipeline, columns along the low qubits), and the rest
# (two-group kernel: k < 6 with far-apart qubits, qubit 0 among far-apart ones).
QUBIT_SETS = {
    1: [[0], [7], [13]],
    2: [[0, 1], [12, 3], [9, 5]],
    3: [[0, 1, 2], [13, 11, 12], [4, 0, 9]],
    4: [[0, 1, 2, 3], [10, 11, 12, 13], [8, 1, 12, 5]],
    5: [[0, 1, 2, 3, 4], [9, 10, 11, 12, 13], [13, 0, 6, 2, 11]],
    6: [[0, 1, 2, 3, 4, 5], [8, 9, 10, 11, 12, 13], [1, 12, 4, 9, 0, 7]],
}


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_blocks_14q(S, orc, k):
    n = 14
    rng = np.random.default_rng(100 + k)
    psi0 = C.random_state(n, k)
    s = S.StateVector(n, "c64")
    for qs in QUBIT_SETS[k]:
        u = random_u(rng, 1 << k)
        s.from_numpy(psi0)
        s.apply_fused(qs, u)
        check_c64(s.to_numpy(), orc.apply_kq(psi0, qs, u))


@pytest.mark.parametrize("n", [12, 13, 14, 20, 22])
def test_blocks_one_and_many_tiles(S, orc, n):
    """Tiles hold 2^12 amplitudes: n = 12 is one tile (one CTA, most roles
    idle after one pass), n = 13 two, n = 14 four, n = 20 gives 256 tiles,
    n = 22 1024 (several per CTA: the staging ring and the accumulators wrap,
    mbarrier phases alternate)."""
    rng = np.random.default_rng(n)
    psi0 = C.random_state(n, 7 + n)
    s = S.StateVector(n, "c64")
    for k in (2, 4, 6):
        qs = [int(q) for q in rng.choice(n, size=k, replace=False)]
        u = random_u(rng, 1 << k)
        s.from_numpy(psi0)
        s.apply_fused(qs, u)
        check_c64(s.to_numpy(), orc.apply_kq(psi0, qs, u))


# (n, qubits) reaching each kernel and load form (the host picks them from the
# layout): the pipeline with loader warps and rows along the low qubits, the
# pipeline with loader warps and columns along them (too many qubit runs for
# the tensor map's five dimensions), the pipeline with tensor-map loads (one
# box per tile; four boxes when two runs are iterated; columns along qubits
# 0..1 only), and the two-group
# kernel (qubit 0 among far-apart qubits, k < 6 with far-apart qubits).
FORMS = [
    (22, [0, 1, 2, 3, 4, 5]),
    (14, [0, 1]),
    (22, [8, 10, 12, 14, 16, 18]),
    (14, [8, 9, 10, 11, 12, 13]),
    (20, [14, 15, 16, 17, 18, 19]),
    (13, [7, 8, 9, 10, 11, 12]),
    (22, [3, 9, 12, 15, 18, 21]),
    (22, [2, 3, 11, 12, 17, 18]),
    (14, [0, 9]),
    (22, [0, 7, 12, 13, 20, 21]),
    (22, [19, 20, 21]),
    (22, [0, 9, 14, 20]),
]


@pytest.mark.parametrize("n,qs", FORMS)
def test_every_kernel_form(S, orc, n, qs):
    rng = np.random.default_rng(n + len(qs))
    psi0 = C.random_state(n, 31 + n)
    u = random_u(rng, 1 << len(qs))
    s = S.StateVector(n, "c64")
    s.from_numpy(psi0)
    s.apply_fused(qs, u)
    check_c64(s.to_numpy(), orc.apply_kq(psi0, qs, u))


def test_block_sequence(S, orc):
    """A sequence of dense 5-qubit blocks (each the oracle's dense matrix of
    one window's gates) applied on the tensor cores equals the oracle
    applying the same blocks, at 16 qubits."""
    n = 16
    c = C.random_circuit(n, 4, 3)
    windows = [list(range(lo, min(lo + 5, n))) for lo in range(0, n, 5)]
    s = S.StateVector(n, "c64")
    ref = orc.basis_state(n)
    for _ in range(2):
        for qs in windows:
            sub = C.Circuit(len(qs))
            for name, gq, ps in c.gates:
                if all(q in qs for q in gq):
                    sub.add(name, *[qs.index(q) for q in gq], params=ps)
            u = orc.dense(sub)
            s.apply_fused(qs, u)
            ref = orc.apply_kq(ref, qs, u)
        for a in (4, 9, 14):
            one = C.Circuit(n)
            one.add("CZ", a, a + 1)
            one.add("H", a + 1)
            s.run(one, "pergate")
            ref = orc.run(one, psi=ref)
    check_c64(s.to_numpy(), ref)


@pytest.mark.parametrize("qs", [[0, 1], [8, 9, 10, 11, 12, 13], [0, 9]])
def test_timeout_path_reports_and_recovers(S, monkeypatch, qs):
    """Every wait of the tensor-core kernels is bounded by the global timer.
    With the host-side hook the MMAs are never issued: the waits for them
    (and, in the pipeline, every role's wait behind them) run out after 1 ms,
    the kernel waits for its copies in flight, releases its tensor memory and
    sets the error word; the next synchronising call reports SV_ERR_TIMEOUT
    and the context stays usable.  The three qubit sets reach the pipeline
    with loader warps, the pipeline with tensor-map loads and the two-group
    kernel."""
    n = 14
    s = S.StateVector(n, "c64")
    monkeypatch.setenv("SV_FAULT_INJECT", "tc_wait")
    s.apply_fused(qs, np.eye(1 << len(qs)))
    with pytest.raises(S.SVError) as e:
        s.sync()
    assert e.value.status == 5
    monkeypatch.delenv("SV_FAULT_INJECT")
    s.set_basis(3)
    s.apply_fused([0, 1], np.eye(4)[[1, 0, 3, 2]])  # X on qubit 0
    a = s.amplitudes([2, 3])
    assert abs(a[0] - 1) < 1e-6 and abs(a[1]) < 1e-6
