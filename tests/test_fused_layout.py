"""Tensor-map copies of the tensor-core pipeline, checked without a GPU.

For dense blocks on many qubit layouts (Sec. 2: a k-qubit gate acts on the
amplitudes that differ only in its qubits), the library reports which
kernel a block runs and, for tensor-map loads, the map it would encode
(sv_fused_tc_layout: dimensions as ranges of qubits, box, iterated boxes).
The copies are emulated element by element as the tensor-map definition
gives them (a box is copied in dimension order, dimension 0 innermost, into
consecutive shared memory; the 128-byte swizzle then permutes 16-byte
chunks inside each 1024-byte block, which the kernel's reads undo), and
every element of sample tiles must carry the amplitude the split reads at
that tile index: the tile's base plus the index bits placed at the tile's
qubits."""

import numpy as np
import pytest

from paper_1912_03243_gb300 import build as B
from paper_1912_03243_gb300 import sv


@pytest.fixture(scope="module")
def L():
    B.build()
    return sv.lib()


def layouts():
    rng = np.random.default_rng(2024)
    out = [(26, [20, 21, 22, 23, 24, 25]), (26, [3, 9, 14, 17, 21, 24]), (22, [3, 9, 12, 15, 18, 21]),
           (22, [2, 3, 11, 12, 17, 18]), (12, [6, 7, 8, 9, 10, 11]), (34, [5, 9, 13, 20, 27, 31])]
    for n in (13, 16, 20, 26, 32, 34):
        for k in (1, 2, 3, 4, 5, 6):
            for _ in range(4):
                out.append((n, sorted(int(q) for q in rng.choice(n, size=k, replace=False))))
    return out


def place(j, tile_pos):
    """Global offset of tile index j (bit t of j is state qubit tile_pos[t])."""
    g = np.zeros_like(j, dtype=np.uint64)
    for t, q in enumerate(tile_pos):
        g |= ((j >> np.uint64(t)) & np.uint64(1)) << np.uint64(q)
    return g


def emulate_tile(lay, n, tile):
    """Global element of every shared position of one tile's boxes."""
    tp = lay["tile_pos"]
    outer = [q for q in range(n) if q not in tp]
    base = 0
    for o, q in enumerate(outer):
        if tile >> o & 1:
            base |= 1 << q
    rank, start, dim, box = lay["rank"], lay["start"], lay["dim"], lay["box"]
    elem_stride = [1] + [s // 8 for s in lay["stride"]]
    boxel = int(np.prod(box))
    got = np.zeros(boxel * lay["nbox"], dtype=np.uint64)
    idx = np.indices(box[::-1]).reshape(5, -1)[::-1]  # idx[d][e]: coordinate d of element e, dim 0 fastest
    for b in range(lay["nbox"]):
        g = base | lay["boff"][b]
        c = [((g >> start[d]) & (dim[d] - 1)) if d < rank else 0 for d in range(5)]
        assert c[0] == 0  # innermost coordinate: whole 128-byte rows (the 16-byte alignment rule)
        flat = np.zeros(boxel, dtype=np.uint64)
        for d in range(5):
            cd = np.uint64(c[d]) + idx[d].astype(np.uint64)
            assert np.all(cd < np.uint64(dim[d]))  # inside the tensor
            flat += cd * np.uint64(elem_stride[d])
        got[b * boxel:(b + 1) * boxel] = flat
    return base, got


@pytest.mark.parametrize("n,qs", layouts())
def test_tensor_map_copies_land_where_the_split_reads(L, n, qs):
    lay = sv.sv_fused_tc_layout(n, qs)
    k = len(qs)
    assert lay["kernel"] in (f"k_fused_tc<k={k}>", f"k_fused_tc<k={k},tma>", f"k_fused_tc_groups<k={k}>")
    tp = lay["tile_pos"]
    assert sorted(tp) == tp and set(qs) <= set(tp) and tp[:6] == [0, 1, 2, 3, 4, 5]
    if not lay["kernel"].endswith(",tma>"):
        assert lay["rank"] == 0 and lay["nbox"] == 0
        return
    assert 2 <= lay["rank"] <= 5 and lay["nbox"] in (1, 2, 4)
    assert lay["box"][0] == 16  # 128 bytes: the swizzle's row
    assert all(1 <= b <= 256 for b in lay["box"])
    assert int(np.prod(lay["box"])) * lay["nbox"] == 4096
    total = 1
    for d in range(5):  # the plain layout: each stride the product of the sizes below
        if d > 0:
            assert lay["stride"][d - 1] == 8 * total
        total *= lay["dim"][d]
    assert total == 1 << n
    j = np.arange(4096, dtype=np.uint64)
    ntiles = 1 << (n - 12)
    for tile in sorted({0, 1 % ntiles, (ntiles * 5) // 7, ntiles - 1}):
        base, got = emulate_tile(lay, n, tile)
        want = np.uint64(base) | place(j, tp)
        assert np.array_equal(got, want), (n, qs, tile)


def test_forms_cover_the_kernels(L):
    """The layouts above reach all three kernel forms."""
    kinds = {sv.sv_fused_tc_layout(n, qs)["kernel"].split("<")[0] + ("+tma" if ",tma" in
             sv.sv_fused_tc_layout(n, qs)["kernel"] else "") for n, qs in layouts()}
    assert {"k_fused_tc", "k_fused_tc+tma", "k_fused_tc_groups"} <= kinds


@pytest.mark.parametrize("n,qs", [(11, [0]), (41, [0]), (20, []), (20, [0, 0]), (20, [20]),
                                  (20, [0, 1, 2, 3, 4, 5, 6])])
def test_layout_rejects_bad_arguments(L, n, qs):
    with pytest.raises(sv.SVError):
        sv.sv_fused_tc_layout(n, qs)
