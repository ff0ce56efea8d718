"""Eq. 3 over P partitions (Sec. 4) on the GPU: small grids in 3 and 4
partitions against the full-state oracle (every amplitude, both
decompositions), agreement with the two-partition entry point, and the
paper's GHZ values at N = 128 qubits in 8 partitions (Sec. 4: the
coefficients of |0...0> and |1...1> are 1/sqrt(2))."""

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


def words(idx, n):
    """Integer bit strings -> (m, ceil(n/64)) little-endian uint64 words."""
    nw = (n + 63) // 64
    out = np.zeros((len(idx), nw), dtype=np.uint64)
    for j, v in enumerate(idx):
        v = int(v)
        for w in range(nw):
            out[j, w] = (v >> (64 * w)) & ((1 << 64) - 1)
    return out


def close(got, ref, rel=1e-5):
    assert np.max(np.abs(got - ref)) <= rel * np.max(np.abs(ref))


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("rows,cols,depth,P", [(4, 4, 8, 4), (4, 4, 10, 2), (6, 3, 8, 3), (3, 5, 9, 3)])
def test_row_partitions_all_outputs(S, orc, form, rows, cols, depth, P):
    """Partition p = a band of grid rows; every amplitude against the full
    state."""
    c = C.grid_circuit(rows, cols, depth, 2)
    n = c.n
    band = -(-rows // P)
    part_of = [min((q // cols) // band, P - 1) for q in range(n)]
    z = np.arange(1 << n)
    got, s = S.sv_cut_amplitudes_multi(c, n, part_of, words(z, n), form=form)
    assert s > 0
    close(got, orc.run(c))


def test_matches_two_partition_entry(S):
    c = C.grid_circuit(6, 4, 12, 1)
    mask = C.grid_partition_mask(6, 4, 3)
    z = C.random_bitstrings(512, 24, 3)
    ref, s0 = S.sv_cut_amplitudes(c, 24, mask, z)
    part_of = [0 if (mask >> q) & 1 else 1 for q in range(24)]
    got, s1 = S.sv_cut_amplitudes_multi(c, 24, part_of, words(z, 24))
    assert s0 == s1
    close(got, ref)


def test_parts_add_up(S):
    c = C.grid_circuit(4, 4, 8, 4)
    part_of = [q // 4 for q in range(16)]
    z = words(np.arange(1 << 16), 16)
    full, s = S.sv_cut_amplitudes_multi(c, 16, part_of, z)
    acc = sum(S.sv_cut_amplitudes_multi(c, 16, part_of, z, part=p, nparts_log2=2)[0] for p in range(4))
    close(acc, full)


def test_ghz_128_paper_values(S):
    """Sec. 4: H on qubit 0 and CNOT(i, i+1) on 128 qubits, cut into 8
    partitions of 16 (7 decomposed CNOTs); <0...0|C|0> = <1...1|C|0> =
    1/sqrt(2) and every other sampled coefficient is 0."""
    n = 128
    c = C.ghz_circuit(n)
    part_of = [q // 16 for q in range(n)]
    rng = np.random.default_rng(11)
    others = [int.from_bytes(rng.bytes(16), "little") for _ in range(1000)]
    idx = [0, (1 << n) - 1] + [v for v in others if v not in (0, (1 << n) - 1)] + list(range(1, 1 << 12))
    for form in (0, 1):
        amps, s = S.sv_cut_amplitudes_multi(c, n, part_of, words(idx, n), form=form)
        assert s == 7
        assert np.allclose(amps[:2], 1 / math.sqrt(2), atol=1e-7)
        assert np.max(np.abs(amps[2:])) < 1e-7


def test_errors(S):
    c = C.ghz_circuit(8)
    z = words([0], 8)
    with pytest.raises(S.SVError):  # partition 1 empty (P taken as max + 1 = 3)
        S.sv_cut_amplitudes_multi(c, 8, [0, 0, 0, 0, 2, 2, 2, 2], z)
    with pytest.raises(S.SVError):  # bits above qubit 7
        S.sv_cut_amplitudes_multi(c, 8, [q // 4 for q in range(8)], words([1 << 9], 8))
    with pytest.raises(S.SVError):  # SWAP across partitions
        sw = C.Circuit(8)
        sw.add("SWAP", 0, 7)
        S.sv_cut_amplitudes_multi(sw, 8, [q // 4 for q in range(8)], z)


@pytest.mark.parametrize("form", [0, 1])
def test_30q_three_partitions_vs_oracle(S, orc, form):
    """Beyond the full state's reach in the oracle: a 6x5 grid (30 qubits),
    depth 8, in three partitions of two rows (10 decomposed CZs), 256 seeded
    amplitudes against the oracle's own P-partition sum."""
    c = C.grid_circuit(6, 5, 8, 4)
    part_of = [(q // 5) // 2 for q in range(30)]
    idx = [int(v) for v in C.random_bitstrings(256, 30, 9)]
    got, s = S.sv_cut_amplitudes_multi(c, 30, part_of, words(idx, 30), form=form)
    ref, s_ref = orc.cut_amplitudes_multi(c, part_of, idx, form=form)
    assert s == s_ref == 10
    close(got, ref)
