"""GPU decomposition of entangling gates (Sec. 4, Eq. 2-3) against the CPU
oracle: branch sums over all outputs equal the full state; the GHZ
coefficients of Sec. 4; the 6x4 grid check instance over all 2^24
amplitudes; the 48-qubit 6x8 grid workload with both decompositions.
Tolerance: max |d amp| <= 1e-5 * max |amp| (complex64 halves, FP64 sum)."""

import math
import os

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


def close(got, ref, rel=1e-5):
    assert np.max(np.abs(got - ref)) <= rel * np.max(np.abs(ref))


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("rows,cols,rows_a,depth,seed", [(2, 3, 1, 6, 1), (3, 4, 1, 8, 2), (4, 3, 2, 12, 3),
                                                         (4, 4, 2, 8, 4)])
def test_small_grids_all_outputs(S, orc, form, rows, cols, rows_a, depth, seed):
    c = C.grid_circuit(rows, cols, depth, seed)
    mask = C.grid_partition_mask(rows, cols, rows_a)
    z = np.arange(1 << c.n, dtype=np.uint64)
    full = orc.run(c)
    got, s = S.sv_cut_amplitudes(c, c.n, mask, z, form=form)
    ref, s_ref = orc.cut_amplitudes(c, mask, z, form=form)
    assert s == s_ref > 0
    close(got, full)
    close(got, ref)


@pytest.mark.parametrize("form", [0, 1])
def test_cx_and_cp_across(S, orc, form):
    n = 14
    src = C.random_unitary_gates(n, 200, 21)
    c = C.Circuit(n)
    for name, qs, ps in src.gates:
        crossing = len(qs) == 2 and ((qs[0] < 7) != (qs[1] < 7))
        if name == "SWAP" and crossing:
            continue
        if form == 1 and name == "CP" and crossing:
            continue
        c.add(name, *qs, params=ps)
    z = np.random.default_rng(1).integers(0, 1 << n, size=3000, dtype=np.uint64)
    # keep S small enough for the oracle: take the first gates until 10 cuts
    cut = C.Circuit(n)
    count = 0
    for name, qs, ps in c.gates:
        if len(qs) == 2 and ((qs[0] < 7) != (qs[1] < 7)):
            if count == 10:
                continue
            count += 1
        cut.add(name, *qs, params=ps)
    got, s = S.sv_cut_amplitudes(cut, n, (1 << 7) - 1, z, form=form)
    assert s == count
    full = orc.run(cut)
    close(got, full[z.astype(np.int64)])


def test_ghz_48_paper_values(S):
    """Sec. 4: with the GHZ chain cut between the halves, the coefficients of
    |0...0> and |1...1> are 1/sqrt(2); everything else is 0."""
    n = 48
    c = C.ghz_circuit(n)
    z = np.array([0, (1 << n) - 1, 1, 1 << 47, 0x123456789AB], dtype=np.uint64)
    for form in (0, 1):
        got, s = S.sv_cut_amplitudes(c, n, (1 << 24) - 1, z, form=form)
        assert s == 1
        assert np.allclose(got[:2], 1 / math.sqrt(2), atol=1e-7)
        assert np.max(np.abs(got[2:])) < 1e-7


def test_grid_6x4_all_amplitudes(S, orc):
    """The check instance of the 48-qubit workload: a 6x4 grid (12 + 12
    qubits), depth 12, S = 8 (256 branches), all 2^24 amplitudes against
    the full-state oracle."""
    c = C.grid_circuit(6, 4, 12, 1)
    mask = C.grid_partition_mask(6, 4, 3)
    z = np.arange(1 << 24, dtype=np.uint64)
    got, s = S.sv_cut_amplitudes(c, 24, mask, z, form=0)
    assert s == 8
    full = orc.run(c)
    close(got, full)
    f = abs(np.vdot(full, got)) ** 2 / (np.vdot(full, full).real * np.vdot(got, got).real)
    assert 1 - f <= 1e-5


@pytest.mark.parametrize("depth,cuts", [(6, 4), (12, 8), (18, 12)])
def test_form_error_study(S, orc, record_property, depth, cuts):
    """Error of each decomposition against the full FP64 state as the number
    of cut gates grows (5x4 grid, rows 0-1 | 2-4, all 2^20 amplitudes): the
    projector form (weight 1, bounded factors) and Eq. 2 (weight 1/2 per cut,
    factors of size r^2 = 1 + sqrt 2 whose terms cancel).  Both stay inside the
    tolerance; the measured errors are recorded."""
    c = C.grid_circuit(5, 4, depth, 1)
    mask = C.grid_partition_mask(5, 4, 2)
    z = np.arange(1 << 20, dtype=np.uint64)
    full = orc.run(c)
    scale = np.max(np.abs(full))
    for form in (0, 1):
        got, s = S.sv_cut_amplitudes(c, 20, mask, z, form=form)
        assert s == cuts
        err = float(np.max(np.abs(got - full)) / scale)
        f = abs(np.vdot(full, got)) ** 2 / (np.vdot(full, full).real * np.vdot(got, got).real)
        record_property(f"form{form}_S{cuts}_max_rel_err", err)
        record_property(f"form{form}_S{cuts}_infidelity", float(1 - f))
        print(f"form-error S={cuts} form={form} max|d|/max|amp|={err:.3e} 1-F={1 - f:.3e}")
        assert err <= 1e-5 and 1 - f <= 1e-5


def test_grid_6x8_48q_both_forms(S):
    """The 48-qubit 6x8 grid, depth 8, S = 8: 256 branches x 2 halves of 2^24
    amplitudes (2 x 2^32 batched complex64), 1024 seeded output bit strings.
    The projector decomposition and Eq. 2 are independent rewrites of the
    same sum; they must agree."""
    import torch

    if torch.cuda.mem_get_info()[0] < (80 << 30):
        pytest.skip("not enough device memory")
    c = C.grid_circuit(6, 8, 8, 1)
    mask = C.grid_partition_mask(6, 8, 3)
    z = C.random_bitstrings(1024, 48, 7)
    a0, s0 = S.sv_cut_amplitudes(c, 48, mask, z, form=0)
    a1, s1 = S.sv_cut_amplitudes(c, 48, mask, z, form=1)
    assert s0 == s1 == 8
    close(a0, a1, rel=1e-4)
    # amplitudes of a 48-qubit random-ish state: mean |amp|^2 near 2^-48
    p = np.mean(np.abs(a0) ** 2) * 2.0 ** 48
    assert 0.2 < p < 5.0


def test_errors(S):
    c = C.Circuit(6)
    c.add("SWAP", 0, 5)
    with pytest.raises(S.SVError) as e:
        S.sv_cut_amplitudes(c, 6, 0b000111, np.array([0], dtype=np.uint64))
    assert e.value.status == 8
    with pytest.raises(S.SVError):
        S.sv_cut_amplitudes(C.ghz_circuit(6), 6, 0, np.array([0], dtype=np.uint64))
    with pytest.raises(S.SVError):
        S.sv_cut_amplitudes(C.ghz_circuit(6), 6, 0b111, np.array([64], dtype=np.uint64))


@pytest.mark.parametrize("form", [0, 1])
def test_parts_add_up(S, orc, form):
    """Branch sharding: the partial sums over s = part (mod 2^p) for p = 1,
    2, 3 add up to the full Eq. 3 sum, each part matches the oracle's part,
    and parts past the branch count are zero."""
    c = C.grid_circuit(4, 3, 12, 3)
    mask = C.grid_partition_mask(4, 3, 2)
    z = np.arange(1 << c.n, dtype=np.uint64)
    full, s = S.sv_cut_amplitudes(c, c.n, mask, z, form=form)
    for p in (1, 2, 3):
        acc = np.zeros_like(full)
        for part in range(1 << p):
            got, sp = S.sv_cut_amplitudes_part(c, c.n, mask, z, part, p, form=form)
            ref, _ = orc.cut_amplitudes_part(c, mask, z, part, p, form=form)
            assert sp == s
            close(got, ref, rel=1e-5 * np.max(np.abs(full)) / max(np.max(np.abs(ref)), 1e-300))
            acc += got
        close(acc, full)
    far, _ = S.sv_cut_amplitudes_part(c, c.n, mask, z, (1 << s) + 1, s + 2, form=form)
    assert np.all(far == 0)
    with pytest.raises(S.SVError):
        S.sv_cut_amplitudes_part(c, c.n, mask, z, 4, 2, form=form)


@pytest.mark.parametrize("form", [0, 1])
def test_part_lists_sum_on_the_device(S, orc, form):
    """sv_cut_amplitudes_parts: a rank's share (the parts p = r mod W of
    2^ceil(log2 W)) summed by the library equals the oracle's parts added up;
    the shares of all ranks add up to the full Eq. 3 sum; a list with a
    repeated or out-of-range part is an argument error."""
    from paper_1912_03243_gb300 import sharding

    c = C.grid_circuit(4, 3, 12, 3)
    mask = C.grid_partition_mask(4, 3, 2)
    z = np.arange(1 << c.n, dtype=np.uint64)
    full, s = S.sv_cut_amplitudes(c, c.n, mask, z, form=form)
    for world in (1, 2, 3, 5):
        acc = np.zeros_like(full)
        for rank in range(world):
            p, parts = sharding.parts_for_rank(rank, world)
            got, sp = S.sv_cut_amplitudes_parts(c, c.n, mask, z, p, parts, form=form)
            ref = sum(orc.cut_amplitudes_part(c, mask, z, part, p, form=form)[0] for part in parts)
            assert sp == s
            close(got, ref)
            acc += got
        close(acc, full)
    # all parts of a split that bounds memory, in one call
    got, _ = S.sv_cut_amplitudes_parts(c, c.n, mask, z, 3, list(range(8)), form=form)
    close(got, full)
    for bad in ([1, 1], [0, 4], []):
        with pytest.raises(S.SVError):
            S.sv_cut_amplitudes_parts(c, c.n, mask, z, 2, bad, form=form)


def test_sharded_library_sum_two_ranks(S, orc, tmp_path):
    """Two gloo ranks on the one GPU: each sums its branch parts with the
    library, one host all-reduce combines them; equals the oracle's Eq. 3
    sum."""
    import socket
    import sys

    import torch.multiprocessing as mp

    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import mp_helpers

    c = C.grid_circuit(4, 3, 12, 5)
    mask = C.grid_partition_mask(4, 3, 2)
    z = C.random_bitstrings(300, c.n, 3)
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    out = tmp_path / "lib_sum.npy"
    mp.start_processes(mp_helpers.sharded_library_sum, args=(2, port, c.text(), c.n, mask, [int(v) for v in z], 0,
                                                             str(out)), nprocs=2, start_method="spawn", join=True)
    full, _ = orc.cut_amplitudes(c, mask, z)
    close(np.load(out), full)


@pytest.mark.parametrize("form", [0, 1])
def test_prefix_sharing_matches_batched(S, monkeypatch, form):
    """Branch-prefix sharing (branches forked from branch 0 at their first
    operator) and the fully batched simulation (every branch from the start,
    SV_CUT_PREFIX=0) give the same amplitudes: the 6x4 check grid, all 2^24
    outputs, and a grid whose first gates are cut (fork before any gate)."""
    for c, mask in ((C.grid_circuit(6, 4, 12, 1), C.grid_partition_mask(6, 4, 3)),
                    (C.grid_circuit(4, 3, 8, 6), C.grid_partition_mask(4, 3, 2))):
        z = np.arange(1 << min(c.n, 24), dtype=np.uint64)
        monkeypatch.setenv("SV_CUT_PREFIX", "0")
        ref, s0 = S.sv_cut_amplitudes(c, c.n, mask, z, form=form)
        monkeypatch.setenv("SV_CUT_PREFIX", "1")
        got, s1 = S.sv_cut_amplitudes(c, c.n, mask, z, form=form)
        assert s0 == s1
        close(got, ref)
