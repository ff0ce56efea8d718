"""The C-ABI library without a GPU: it builds, loads, exports every symbol
include/sv.h declares, and answers host-only calls and argument errors."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_1912_03243_gb300 import build as B
from paper_1912_03243_gb300 import circuits as C
from paper_1912_03243_gb300 import sv

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sv.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    return sv.lib()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sv_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    # and the binding knows the same set
    assert set(names) == set(sv.SIGNATURES), set(names) ^ set(sv.SIGNATURES)


def test_bytes_required(L):
    assert sv.sv_bytes_required(20, "c64") == 8 << 20
    assert sv.sv_bytes_required(30, "c128") == 2 ** (30 + 4)  # Sec. 1: 2^(N+4) bytes
    assert sv.sv_bytes_required(35, "enc2b") == 2 * 2 ** 35 + 4 * 2 ** 27  # 64 GB + 512 MB
    assert sv.sv_bytes_required(5, "enc2b") == 64 + 4
    assert sv.sv_bytes_required(0, "c64") == 0
    assert sv.sv_bytes_required(41, "c64") == 0


def test_gate_tables_agree(L, orc):
    """Both sides hard-code the gate table independently; they must agree."""
    for name in C.ONE_QUBIT:
        assert np.array_equal(sv.sv_gate_matrix(name), orc.gate_matrix(name)), name
    for name, ps in (("P", [0.37]), ("CP", [-1.1]), ("CZ", []), ("CX", []), ("SWAP", [])):
        assert np.allclose(sv.sv_gate_matrix(name, ps), orc.gate_matrix(name, ps), atol=0, rtol=0), name
    u = [0.6, 0.0, 0.0, 0.8, 0.0, 0.8, 0.6, 0.0]
    assert np.array_equal(sv.sv_gate_matrix("U", u), orc.gate_matrix("U", u))
    with pytest.raises(ValueError):
        sv.sv_gate_matrix("NOPE")


def test_argument_errors_without_gpu(L):
    h = ctypes.c_void_p()
    assert L.sv_alloc(0, 0, None, ctypes.byref(h)) == 1          # SV_ERR_ARG
    assert L.sv_alloc(20, 7, None, ctypes.byref(h)) == 1
    assert L.sv_alloc(20, 0, None, None) == 1
    u = (ctypes.c_double * 8)()
    assert L.sv_apply_gate(None, 0, -1, u) == 1
    assert L.sv_norm(None, None) == 1
    assert L.sv_free(None) == 0
    assert L.sv_attach(10, 0, None, 0, None, ctypes.byref(h)) == 1
    assert b"NULL" in L.sv_last_error()
    assert L.sv_version().startswith(b"libsv")


def test_fault_injection_alloc(L, monkeypatch):
    """SV_FAULT_INJECT=alloc reports SV_ERR_OOM before touching the GPU."""
    monkeypatch.setenv("SV_FAULT_INJECT", "alloc")
    h = ctypes.c_void_p()
    assert L.sv_alloc(10, 0, None, ctypes.byref(h)) == 2
    assert b"injected" in L.sv_last_error()
    assert not h.value


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    """No CPU fallback: a missing libsv.so is an error, not a silent path."""
    monkeypatch.setattr(sv, "_lib", None)
    monkeypatch.setattr(sv, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        sv.lib()


def test_tiled_plans_compile_for_sm103a(L):
    """The tiled mode emits one straight-line kernel per pass; planning and
    NVRTC compilation need no GPU.  Pass counts of the benchmark circuits."""
    g, p, s = sv.sv_plan_stats(C.random_circuit(14, 6, 1), 14, "c64", compile=True)
    assert g == 14 * 6 + 3 * 7 + 3 * 6 and 1 <= p < g and s >= p
    g, p, s = sv.sv_plan_stats(C.random_unitary_gates(13, 120, 4), 13, "c128", compile=True)
    assert p >= 1
    g, p, s = sv.sv_plan_stats(C.random_circuit(32, 24, 1), 32, "c64")
    assert g == 1140 and p <= 30
    with pytest.raises(sv.SVError):
        sv.sv_plan_stats(C.random_circuit(8, 2, 1), 8, "c64")


@pytest.mark.parametrize("env", [{}, {"SV_JIT_PROCS": "0"}, {"SV_JIT_WORKER": "/nonexistent/sv_nvrtc_worker"}])
def test_pass_compiles_in_workers_or_in_process(L, monkeypatch, env):
    """Tiled passes compile in worker processes (NVRTC serialises work within
    one process), in-process with SV_JIT_PROCS=0, and in-process when no
    worker can be started."""
    assert os.access(os.path.join(os.path.dirname(sv.__file__), "sv_nvrtc_worker"), os.X_OK)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    g, p, s = sv.sv_plan_stats(C.random_circuit(14, 4, 9), 14, "c64", compile=True)
    assert g == 14 * 4 + 2 * 7 + 2 * 6 and p >= 1


def test_plain_c_client(L, tmp_path):
    """The boundary is a C ABI: a C99 program (tests/c_abi_probe.c) compiles
    against include/sv.h with warnings as errors, links libsv.so and runs its
    host-only calls, with the same answers as the Python binding."""
    import subprocess

    here = os.path.dirname(os.path.abspath(__file__))
    libdir = os.path.dirname(os.path.abspath(sv.__file__))
    exe = str(tmp_path / "c_abi_probe")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(os.path.dirname(here), "include"),
           os.path.join(here, "c_abi_probe.c"), "-L", libdir, "-lsv", f"-Wl,-rpath,{libdir}", "-lm", "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = {line.split()[0]: line.split()[1:] for line in out if line}
    assert int(rows["bytes_c64_20"][0]) == sv.sv_bytes_required(20, "c64") == 8 << 20
    assert int(rows["bytes_enc_20"][0]) == sv.sv_bytes_required(20, "enc2b")
    assert rows["gate_H"][0] == "1"
    assert float(rows["gate_H"][1]) == pytest.approx(2 ** -0.5) and float(rows["gate_H"][2]) == pytest.approx(-(2 ** -0.5))
    assert rows["plan"][0] == "0" and rows["plan"][1] == "4" and int(rows["plan"][2]) >= 1
    assert rows["bad"][0] != "0" and rows["bad"][1] == "message"


def test_compiled_pass_disk_cache(L, monkeypatch, tmp_path):
    """Compiled passes are kept on disk, one file per pass source (the source
    and the cubin); a damaged file is a miss and is written again; with
    SV_JIT_CACHE=0 nothing is written."""
    c = C.random_circuit(16, 6, 12)
    monkeypatch.setenv("SV_JIT_CACHE", str(tmp_path))
    g, p, s = sv.sv_plan_stats(c, 16, "c64", compile=True)
    files = sorted(tmp_path.iterdir())
    assert len(files) == p and all(f.read_bytes().startswith(b"SVJIT1\n") for f in files)
    good = files[0].read_bytes()
    files[0].write_bytes(good[: len(good) // 2])
    assert sv.sv_plan_stats(c, 16, "c64", compile=True) == (g, p, s)
    assert files[0].read_bytes() == good  # recompiled: the same source gives the same cubin
    off = tmp_path / "off"
    off.mkdir()
    monkeypatch.setenv("SV_JIT_CACHE", "0")
    monkeypatch.setenv("TMPDIR", str(off))  # the workers' scratch without a cache: created and removed
    sv.sv_plan_stats(C.random_circuit(15, 5, 13), 15, "c64", compile=True)
    assert not any(off.iterdir()) and sorted(tmp_path.iterdir()) == sorted(files + [off])


@pytest.mark.parametrize("name,n,gates,passes,segments", [("random", 32, 1140, 11, 32), ("random", 28, 996, 9, 30),
                                                         ("random", 30, 712, 8, 23), ("qft", 32, 564, 6, 17)])
def test_planner_does_not_regress(L, name, n, gates, passes, segments):
    """Upper bounds on HBM passes and shared-memory transpositions of the
    benchmark circuits (each pass moves the whole state twice; each segment
    transposes a tile through shared memory): the planner's lookahead plans
    (complex64, 2^13-amplitude tiles, 5 register qubits per thread)."""
    c = C.random_circuit(n, {32: 24, 28: 24, 30: 16}[n], 1) if name == "random" else C.qft_circuit(n, 0x9E3779B9)
    g, p, s = sv.sv_plan_stats(c, n, "c64")
    assert g == gates
    assert p <= passes and s <= segments, (p, s)


def test_direct_hbm_segments_cover_whole_sectors(L):
    """Host only: in the generated passes of the 28-qubit depth-24 benchmark
    family, every register segment that loads from or stores to HBM directly
    has lanes on global qubits 0, 1 and 2 (8 lanes x 8 contiguous bytes: whole
    32-byte sectors per warp access), and every pass starts with such a load
    or with the staged copy."""
    import re

    c = C.random_circuit(28, 24, 1)
    _, passes, _ = sv.sv_plan_stats(c, 28, "c64")
    direct = 0
    for i in range(passes):
        src = sv.sv_plan_pass_source(c, 28, "c64", i)
        assert ("psi[gq + " in src) or ("cpa16(smem" in src), i
        for block in src.split("u64 gq = 0;")[1:]:
            lanes = set()
            for m in re.finditer(r"gq \|= \(\(u64\)\(\(t >> (\d+)\) & (\d+)ull\)\) << (\d+);", block[:1200]):
                k, mask, p = int(m.group(1)), int(m.group(2)), int(m.group(3))
                for b in range(mask.bit_length()):
                    if k + b < 5:
                        lanes.add(p + b)
            assert {0, 1, 2} <= lanes, (i, sorted(lanes))
            direct += 1
    assert direct >= passes  # most passes load and store directly
