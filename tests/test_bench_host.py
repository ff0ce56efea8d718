"""Host logic of bench.py (no GPU): which roof heads the roofline object, and
the FP32 lane operations a circuit needs at least."""

import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_1912_03243_gb300 import circuits as C  # noqa: E402

HBM = {"bound": "hbm", "achieved": 3490.0, "peak": 6690.8, "unit": "GB/s", "frac": 3490.0 / 6690.8,
       "traffic": 6.8e10, "kernel": "svp<f32,13,5>", "launches": 55, "avg_launch_ms": 19.7,
       "bytes_per_launch": 6.87e10, "peak_kind": "measured", "frac_of_nominal_8tbs": 3490.0 / 8000.0,
       "share_of_step": 1.0}
FP32 = {"bound": "alu", "achieved": 26.4, "peak": 40.27, "unit": "T FP32 lane-ops/s", "frac": 26.4 / 40.27}


def test_fp32_roof_heads_when_its_floor_is_longer():
    r = bench.binding_roofline(HBM, FP32, fp32_floor_s=0.710, hbm_floor_s=0.565, steps=5)
    assert r["bound"] == "alu" and r["frac"] == FP32["frac"] and r["unit"] == FP32["unit"]
    # the launch facts and the DRAM traffic of the dominant kernel stay at the top
    for k in ("kernel", "launches", "avg_launch_ms", "share_of_step", "traffic"):
        assert r[k] == HBM[k]
    assert r["hbm"]["bound"] == "hbm" and r["hbm"]["frac"] == HBM["frac"]
    assert r["floors_ms"] == pytest.approx({"fp32": 142.0, "hbm": 113.0})
    assert "fp32" not in r


def test_hbm_roof_heads_otherwise():
    r = bench.binding_roofline(HBM, FP32, fp32_floor_s=0.2, hbm_floor_s=0.565, steps=5)
    assert r["bound"] == "hbm" and r["frac"] == HBM["frac"] and r["fp32"] == FP32
    assert r["floors_ms"] == pytest.approx({"fp32": 40.0, "hbm": 113.0})


def test_fp32_ops_per_amplitude():
    """2 per H / SX / SY (one addition per real component), 1 per T (two
    additions on half the amplitudes), 0 for sign flips and permutations, 8
    for a dense 2x2."""
    c = C.Circuit(4)
    for name, qs in (("H", (0,)), ("T", (1,)), ("CZ", (0, 1)), ("SX", (2,)), ("SY", (3,)), ("X", (0,)),
                     ("SWAP", (1, 2))):
        c.add(name, *qs)
    c.add("U", 0, params=(1, 0, 0, 0, 0, 0, 1, 0))
    assert bench.fp32_ops_per_amplitude(c) == 2 + 1 + 0 + 2 + 2 + 0 + 0 + 8


def test_benchmark_circuit_ops():
    c = C.random_circuit(32, 24, 1)
    names = [g[0] for g in c.gates]
    assert bench.fp32_ops_per_amplitude(c) == 2 * sum(n in ("H", "SX", "SY") for n in names) + names.count("T")
    assert bench.fp32_ops_per_amplitude(c) == 1331


@pytest.mark.parametrize("kernel", ["svp", "k_gate_across", "k_fused_tc", "k_enc_gate_across"])
def test_profiles_match_the_sources(kernel):
    """Every kernel the bench reports a roofline for has a committed ncu summary
    whose source hash matches the current source (a stale one reads as no
    traffic); its DRAM bytes per amplitude are near the algorithmic 16 (4 for
    the two-byte code)."""
    traffic, path = bench.traffic_from_profiles(kernel, 28)
    assert traffic is not None and path is not None
    per_amp = traffic / 2 ** 28
    assert (3.0 < per_amp < 4.5) if kernel == "k_enc_gate_across" else (14.0 < per_amp < 17.0)


def test_kernel_text_ignores_comments_and_host_code(tmp_path):
    """The validity hash of a profile covers the kernel and what it uses, not
    comments, host functions or other kernels of the same file."""
    hdr = tmp_path / "k.h"
    hdr.write_text("#pragma once\nstruct Args { int n; };\nconstexpr int kUnused = 3;\n")
    base = '''#include "k.h"
namespace sv {
namespace {
constexpr int kW = 4;  // width
__device__ __forceinline__ int twice(int x) { return 2 * x; }
__global__ void __launch_bounds__(128) k_a(int *p, Args a) { p[threadIdx.x] = twice(a.n) + kW; }
__global__ void k_b(int *p) { p[0] = 1; }
}  // namespace
int host_fn(int x) { return x + 1; }
}  // namespace sv
'''
    src = tmp_path / "k.cu"

    def h(text, header=None):
        src.write_text(text)
        if header is not None:
            hdr.write_text(header)
        return bench.kernel_text(str(src), "k_a")

    ref = h(base)
    assert "twice" in ref and "kW = 4" in ref and "struct Args" in ref and "k_b" not in ref and "host_fn" not in ref
    assert h(base.replace("// width", "// a new comment\n/* block */")) == ref
    assert h(base.replace("return x + 1;", "return x + 2;")) == ref          # host code
    assert h(base.replace("p[0] = 1;", "p[0] = 2;")) == ref                  # another kernel
    assert h(base.replace("2 * x", "3 * x")) != ref                          # a helper it calls
    assert h(base.replace("kW = 4", "kW = 5")) != ref                        # a constant it uses
    assert h(base, "#pragma once\nstruct Args { long n; };\nconstexpr int kUnused = 3;\n") != ref  # header struct


def test_cut_count_of_the_42_qubit_grid():
    """S(depth) of the 6x7 grid cut between rows 2 and 3, as the bench
    states it (+7 per six layers), equals the library's count of decomposed
    gates (a host-only call: no bit strings, no device work)."""
    import ctypes

    import numpy as np

    from paper_1912_03243_gb300 import sv

    L = sv.lib()
    mask = C.grid_partition_mask(6, 7, 3)
    z = np.zeros(1, dtype=np.uint64)
    out = np.zeros(2)
    for depth in range(1, 26):
        c = C.grid_circuit(6, 7, depth, 1)
        s = ctypes.c_int(-1)
        r = L.sv_cut_amplitudes_part(c.text().encode(), 42, ctypes.c_uint64(mask), 0, ctypes.c_uint64(0), 16, 0,
                                     z.ctypes.data_as(sv._u64p), out.ctypes.data_as(sv._dp), ctypes.byref(s), None)
        assert r == 0 and s.value == bench.cut_gates_42q(depth), depth
