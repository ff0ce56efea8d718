"""Multi-process paths on CPU with the gloo backend: branch sharding of the
decomposition (Sec. 4), the bench's cross-rank timing, and the bench's
reference arm launched as two ranks."""

import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_1912_03243_gb300 import circuits as C
from paper_1912_03243_gb300 import sharding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def spawn(fn, world, *args):
    import torch.multiprocessing as mp

    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    mp.start_processes(fn, args=(world, free_port()) + args, nprocs=world, start_method="spawn", join=True)


def test_parts_for_rank():
    assert sharding.parts_for_rank(0, 1) == (0, [0])
    assert sharding.parts_for_rank(1, 2) == (1, [1])
    assert sharding.parts_for_rank(0, 3) == (2, [0, 3])
    assert sharding.parts_for_rank(2, 3) == (2, [2])
    allp = sorted(p for r in range(5) for p in sharding.parts_for_rank(r, 5)[1])
    assert allp == list(range(8))
    with pytest.raises(ValueError):
        sharding.parts_for_rank(2, 2)


@pytest.mark.parametrize("form", [0, 1])
def test_oracle_parts_add_up(orc, form):
    c = C.grid_circuit(3, 4, 8, 2)
    mask = C.grid_partition_mask(3, 4, 1)
    z = np.arange(1 << c.n, dtype=np.uint64)
    full, s = orc.cut_amplitudes(c, mask, z, form=form)
    for p in (1, 2, 3):
        acc = sum(orc.cut_amplitudes_part(c, mask, z, part, p, form=form)[0] for part in range(1 << p))
        assert np.max(np.abs(acc - full)) < 1e-12
    # parts beyond the branch count are empty
    far, _ = orc.cut_amplitudes_part(c, mask, z, (1 << s) + 1, s + 2, form=form)
    assert np.all(far == 0)


def _run_sharded(orc, tmp_path, world):
    import mp_helpers

    c = C.grid_circuit(4, 3, 12, 5)
    mask = C.grid_partition_mask(4, 3, 2)
    z = C.random_bitstrings(200, c.n, 3)
    out = tmp_path / f"sum{world}.npy"
    spawn(mp_helpers.sharded_oracle_sum, world, c.text(), c.n, mask, [int(v) for v in z], 0, str(out))
    got = np.load(out)
    full, _ = orc.cut_amplitudes(c, mask, z)
    assert np.max(np.abs(got - full)) < 1e-12


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_branch_sum_gloo(orc, tmp_path, world):
    """Each rank sums its branch parts (CPU oracle), one FP64 all-reduce
    combines them; the result equals the unsharded Eq. 3 sum."""
    _run_sharded(orc, tmp_path, world)


def test_bench_max_over_ranks_gloo(tmp_path):
    import mp_helpers

    out = tmp_path / "max.json"
    spawn(mp_helpers.bench_max, 2, str(out))
    assert json.load(open(out))["max"] == 11.0


def test_bench_reference_arm_two_ranks():
    """The benchmark's launch form for N > 1 (torch.distributed.run, two
    ranks): rank 0 prints one JSON line, the other rank exits 0 without
    work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={free_port()}", "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--qubits", "16"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "gates/s" and d["value"] > 0


def test_sharded_multi_partition_sum_gloo(orc, tmp_path):
    """Branch parts of the P-partition sum (4 partitions) over 2 gloo ranks
    equal the unsharded oracle sum."""
    import mp_helpers

    c = C.grid_circuit(4, 3, 8, 7)
    part_of = [q // 3 for q in range(12)]
    z = list(range(0, 1 << 12, 3))
    out = tmp_path / "multi.npy"
    spawn(mp_helpers.sharded_oracle_multi_sum, 2, c.text(), c.n, part_of, z, str(out))
    full, _ = orc.cut_amplitudes_multi(c, part_of, z)
    assert np.max(np.abs(np.load(out) - full)) < 1e-12
