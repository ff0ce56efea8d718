#!/usr/bin/env python
"""Benchmark: gates/s and HBM GB/s at 32 qubits, fused vs per-gate.

Workload: the random circuit family at 32 qubits, depth 24, seed 1 (1140
gates: {H,T,SX,SY} on every qubit per layer, then CZ on alternating
neighbour pairs), complex64 state of 2^32 amplitudes (32 GiB) starting from
|0...0>.  One step = reset to |0...0> plus the whole circuit.  The state is
larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead (the reference arm of this project), on a bounded sample of the same
workload.  Multi-GPU runs are independent replicas (the state-vector path
does not shard without an exchange step); value = all ranks' gates / max time.
"""

from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gates/s & HBM GB/s at 32 qubits: fused vs per-gate, err <=1e-5 vs FP64"
HBM_FALLBACK = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="auto", choices=["auto", "pergate", "tiled", "fused"])
    ap.add_argument("--qubits", "--n", dest="n", type=int, default=32,
                    help="state size; --qubits under torch.distributed.run, whose own parser takes --n as an abbreviation")
    ap.add_argument("--depth", type=int, default=24)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--compare-steps", type=int, default=1,
                    help="steps of each other mode (per-gate, fused) timed for comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the two-byte-code (35 qubits) and decomposition (48 qubits) measurements")
    ap.add_argument("--cut42-budget", type=float, default=60.0,
                    help="seconds the 42-qubit depth sweep may spend on depths 15-16 (S = 18, 21); a depth whose "
                         "projected time exceeds what is left is reported as skipped")
    ap.add_argument("--profile-case", default=None, choices=sorted(PROFILE_CASES),
                    help="run one small fixed invocation of a kernel family for a profiler capture, then exit")
    return ap.parse_args()


# Small fixed invocations of each kernel family for profiler captures (the
# commands in profiles/*.md): a few GB of device memory at most, states larger
# than L2 (129 MB).
PROFILE_CASES = {
    "tiled": "28 qubits, random circuit depth 4, tiled passes (compiled kernels)",
    "tiled24": "28 qubits, random circuit depth 24 (passes as full as at 32 qubits)",
    "pergate": "28 qubits, random circuit depth 1, one launch per gate",
    "enc": "28 qubits, two-byte code, random circuit depth 1",
    "fused": "26 qubits, three dense 6-qubit blocks on the tensor cores (low, high and mixed qubits)",
    "cut": "6x4 grid (24 qubits), depth 12, 8 cut CZs: 256 branches x 2 batched halves of 2^12 amplitudes each",
    "expect": "28 qubits, uniform superposition, <sigma^alpha_i> of every qubit (complex64, then the two-byte code)",
}


def run_profile_case(case: str) -> None:
    import numpy as np

    from paper_1912_03243_gb300 import build
    from paper_1912_03243_gb300 import circuits as C
    from paper_1912_03243_gb300 import sv

    build.build()
    if case in ("tiled", "tiled24", "pergate"):
        s = sv.StateVector(28, "c64")
        depth = {"tiled": 4, "tiled24": 24, "pergate": 1}[case]
        s.run(C.random_circuit(28, depth, 1), "pergate" if case == "pergate" else "tiled")
    elif case == "enc":
        s = sv.StateVector(28, "enc2b")
        s.run(C.random_circuit(28, 1, 1), "pergate")
    elif case == "fused":
        s = sv.StateVector(26, "c64")
        rng = np.random.default_rng(0)
        z = rng.normal(size=(64, 64)) + 1j * rng.normal(size=(64, 64))
        u, _ = np.linalg.qr(z)
        for qs in ([0, 1, 2, 3, 4, 5], [20, 21, 22, 23, 24, 25], [3, 9, 14, 17, 21, 24]):
            s.apply_fused(qs, u)
    elif case == "expect":
        s = sv.StateVector(28, "c64")
        s.run(C.uniform_circuit(28), "tiled")
        s.expect_pauli()
        e = sv.StateVector(28, "enc2b")
        e.encode_from(s)
        e.expect_pauli()
    else:  # cut
        c = C.grid_circuit(6, 4, 12, 1)
        sv.sv_cut_amplitudes(c, 24, C.grid_partition_mask(6, 4, 3), C.random_bitstrings(1024, 24, 7))
        print("ok")
        return
    s.sync()
    print("ok")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "ours":
        torch.cuda.set_device(local)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(args):
    from paper_1912_03243_gb300 import circuits as C

    circ = C.random_circuit(args.n, args.depth, args.seed)
    desc = (f"random circuit, {args.n} qubits, depth {args.depth}, seed {args.seed} "
            f"({len(circ)} gates: {{H,T,SX,SY}} per qubit per layer + alternating CZ), complex64 from |0...0>")
    return circ, desc


# ----------------------------------------------------------------- CPU oracle

def oracle_layers(n, depth, seed, chunk: int = 8):
    """Pieces of `chunk` gates of the benchmark family's circuit at n qubits,
    each a spread sample of it: piece k holds gates k, k + s, k + 2s, ... (s
    = gates / chunk), so that every piece mixes targets across all qubits and
    every gate kind in proportion (the oracle's time per gate depends on the
    target's stride).  The pieces together hold every gate; the timing stops
    between pieces (what is timed is the cost per gate, not the state)."""
    from paper_1912_03243_gb300 import circuits as C

    gates = C.random_circuit(n, depth, seed).gates
    stride = max(1, len(gates) // chunk)
    pieces = []
    for k in range(stride):
        c = C.Circuit(n)
        c.gates = gates[k::stride]
        pieces.append(c)
    return pieces


def oracle_point(n, depth, seed, budget_s: float, min_s: float):
    """Gates/s of the CPU oracle (single thread, complex128) on the family at n
    qubits, a few gates at a time, until min_s of work."""
    import oracle

    psi = oracle.basis_state(n)
    done, t_used = 0, 0.0
    for c in oracle_layers(n, depth, seed):
        t0 = time.perf_counter()
        psi = oracle.run(c, psi=psi)
        t_used += time.perf_counter() - t0
        done += len(c)
        if t_used >= min_s or t_used >= budget_s:
            break
    return done / t_used, done, t_used


def oracle_sample(args, budget_s: float, min_s: float = 10.0, ns=None, weights=None):
    """Time the CPU oracle at one or more qubit counts below args.n and scale
    each to args.n by 2^(n_sample - n) (its cost per gate is proportional to
    the amplitude count; the spread of the scaled values checks that).  The
    value is the point at the largest n.  Returns (gates/s at args.n,
    description, seconds, points)."""
    ns = ns or [min(args.n, 26)]
    weights = weights or [1.0] * len(ns)
    wsum = sum(weights)
    points = []
    for n, w in zip(ns, weights):
        gps, done, t = oracle_point(n, args.depth, args.seed, budget_s * w / wsum, min_s * w / wsum)
        points.append({"n": n, "gates": done, "s": round(t, 3), "gates_per_s": gps,
                       "scaled_to_n": gps * 2.0 ** (n - args.n)})
    top = points[-1]
    desc = (f"oracle (plain C, complex128, 1 thread of {os.cpu_count()} host cores) on spread samples of the gates of the same "
            f"circuit family at n = {', '.join(str(p['n']) for p in points)} qubits, each scaled by 2^(n-{args.n}) "
            f"to {args.n} qubits: " + ", ".join(f"{p['gates_per_s']:.3g} gates/s at {p['n']} -> "
                                                f"{p['scaled_to_n']:.3g}" for p in points)
            + f"; value from n = {top['n']}")
    return top["scaled_to_n"], desc, sum(p["s"] for p in points), points


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle as it stands, on host cores."""
    if rank != 0:
        return
    per_step = []
    desc = None
    for k in range(args.warmup + args.steps):
        v, desc, t, _ = oracle_sample(args, budget_s=8.0, min_s=2.0)
        if k >= args.warmup:
            per_step.append((v, t))
    value = statistics.median([v for v, _ in per_step])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median([t for _, t in per_step]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(args)[1], "n": args.n, "depth": args.depth},
        "cpu_baseline": {"value": value, "unit": "gates/s", "cores": 1, "host_cores": os.cpu_count(),
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- ncu traffic
#
# A committed ncu summary stays valid while the code it measured is unchanged.
# For a kernel of a .cu file that code is the kernel's own text: its
# definition plus every namespace-level definition it uses (device helpers,
# constants, structs, also from the local headers the file includes), with
# comments and whitespace dropped, so that host-only edits and comments do not
# invalidate a capture.  For the compiled tile passes it is the generated
# source of the passes of the profiled case.

def _strip_comments(src: str) -> str:
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c == '"':
            j = i + 1
            while j < n and src[j] != '"':
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "".join(out)


def _top_level_chunks(src: str) -> list:
    """Namespace-level constructs of comment-free C++ source: function
    definitions, structs and declarations ending in ';' (preprocessor lines
    dropped, namespace and extern "C" braces transparent)."""
    import re

    src = "\n".join(ln for ln in src.split("\n") if not ln.lstrip().startswith("#"))
    chunks, stack, start, i, n = [], [], 0, 0, len(src)
    while i < n:
        c = src[i]
        if c == '"':
            j = i + 1
            while j < n and src[j] != '"':
                j += 2 if src[j] == "\\" else 1
            i = j + 1
            continue
        if c == "{":
            if "blk" not in stack and re.search(r'(namespace\s*\w*|extern\s*"C")\s*$', src[start:i]):
                stack.append("ns")
                start = i + 1
            else:
                stack.append("blk")
        elif c == "}":
            kind = stack.pop() if stack else "ns"
            if kind == "ns":
                start = i + 1
            elif "blk" not in stack:
                j = i + 1
                m = re.match(r"\s*;", src[j:])
                if m:
                    j += m.end()
                chunks.append(src[start:j])
                start = i = j
                continue
        elif c == ";" and "blk" not in stack:
            chunks.append(src[start:i + 1])
            start = i + 1
        i += 1
    return [c.strip() for c in chunks if c.strip()]


_NOT_NAMES = {"__launch_bounds__", "__align__", "alignas", "decltype", "sizeof", "static_assert", "if", "for",
              "while", "switch", "return", "template", "asm", "defined"}


def _chunk_names(ch: str) -> set:
    import re

    head = ch.split("{", 1)[0]
    head = re.sub(r"template\s*<[^{]*?>\s*", "", head, count=1)
    m = re.match(r"\s*(?:struct|class|union|enum)\s+(?:class\s+)?(\w+)", head)
    if m:
        return {m.group(1)}
    for m in re.finditer(r"(\w+)\s*\(", head):
        if m.group(1) not in _NOT_NAMES:
            if "=" in head[:m.start()]:
                break
            return {m.group(1)}
    m = re.search(r"(\w+)\s*(?:\[[^\]]*\]\s*)*(?:=|;|\{)", head + ";")
    return {m.group(1)} if m else set()


def kernel_text(path: str, kernel: str, read=None) -> str:
    """The text of __global__ function `kernel` of the .cu file at path and
    of every namespace-level definition it uses, transitively (from the file
    and the local headers it includes), comments and whitespace normalised."""
    import re

    def _read(p):
        try:
            with open(p) as f:
                return f.read()
        except OSError:
            return None

    read = read or _read
    texts, seen = [], set()

    def add(p):
        if p in seen:
            return
        seen.add(p)
        s = read(p)
        if s is None:
            return
        texts.append(s)
        for inc in re.findall(r'#include\s+"([^"]+)"', s):
            add(os.path.normpath(os.path.join(os.path.dirname(p), inc)))

    add(path)
    named = [(_chunk_names(c), c) for s in texts for c in _top_level_chunks(_strip_comments(s))]
    want, done, out = {kernel}, set(), []
    while want:
        name = want.pop()
        done.add(name)
        for names, c in named:
            if name in names and c not in out:
                out.append(c)
                want |= set(re.findall(r"[A-Za-z_]\w*", c)) - done
    order = {c: k for k, (_, c) in enumerate(named)}
    out.sort(key=order.get)
    return "\n".join(" ".join(c.split()) for c in out)


def kernel_text_sha1(kv: dict):
    """Current hash of the code a summary measured (None if it cannot be
    computed here)."""
    if kv.get("kernel_case"):
        try:
            from paper_1912_03243_gb300 import sv

            return hashlib.sha1(sv.tiled_pass_sources(kv["kernel_case"]).encode()).hexdigest()
        except Exception:
            return None
    src = os.path.join(ROOT, "paper_1912_03243_gb300", "csrc", kv.get("source", ""))
    if not os.path.exists(src):
        return None
    return hashlib.sha1(kernel_text(src, kv.get("function", kv["kernel"])).encode()).hexdigest()


def traffic_from_profiles(kernel: str, n: int):
    """DRAM bytes per launch from a committed ncu summary: a summary file under
    profiles/ carries lines 'kernel: <name>', 'dram_bytes_per_amplitude: <x>'
    and 'kernel_text_sha1: <hash of the measured code at capture>'; a summary
    whose code has changed since gives None."""
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip().strip("-* `")] = v.strip().strip("`")
        if kv.get("kernel") != kernel or "dram_bytes_per_amplitude" not in kv:
            continue
        if "kernel_text_sha1" in kv:
            if kernel_text_sha1(kv) != kv["kernel_text_sha1"]:
                return None, path
        else:
            src = os.path.join(ROOT, "paper_1912_03243_gb300", "csrc", kv.get("source", ""))
            if not os.path.exists(src):
                continue
            with open(src, "rb") as f:
                if hashlib.sha1(f.read()).hexdigest() != kv.get("source_sha1"):
                    return None, path
        return float(kv["dram_bytes_per_amplitude"]) * (1 << n), path
    return None, None


# ----------------------------------------------------------------- GPU arm

def time_plan(S, state, plan, steps, warmup, world, with_events=True):
    """Returns (max-over-ranks seconds for `steps` steps, per-launch durations in ms)."""
    import torch

    stream = state.stream
    for _ in range(warmup):
        state.set_basis(0)
        plan.execute()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(plan.passes + 1)] for _ in range(steps)]
    if with_events:
        # torch creates the CUDA event on its first record(); do that before
        # handing the handles to the library
        for row in ev:
            for e in row:
                e.record(stream)
        torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        start.record(stream)
        for k in range(steps):
            state.set_basis(0)
            if with_events:
                plan.execute_timed(ev[k])
            else:
                plan.execute()
        end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    t = start.elapsed_time(end) / 1e3
    per_launch = []
    if with_events:
        for k in range(steps):
            per_launch.append([ev[k][i].elapsed_time(ev[k][i + 1]) for i in range(plan.passes)])
    return max_over_ranks(world, t), per_launch


# FP32 lane operations per amplitude a gate needs at least: a structured
# 2x2 (entries 0, +-1, +-i up to one scalar) is one real addition per
# component and amplitude; T / Tdg multiply half the amplitudes by
# (1 +- i) / sqrt(2), two additions each; P and CP a complex product (4) on
# half / a quarter of them; X, Y, Z, S, CX, CZ and SWAP are signs and swaps;
# anything else (U) is a dense 2x2, 8.
FP32_OPS = {"H": 2, "SX": 2, "SXDG": 2, "SY": 2, "SYDG": 2, "T": 1, "TDG": 1, "P": 2, "CP": 1,
            "X": 0, "Y": 0, "Z": 0, "S": 0, "SDG": 0, "CX": 0, "CNOT": 0, "CZ": 0, "SWAP": 0}


def fp32_ops_per_amplitude(circ) -> int:
    return sum(FP32_OPS.get(name.upper(), 8) for name, _, _ in circ.gates)


def binding_roofline(hbm, fp32, fp32_floor_s, hbm_floor_s, steps):
    """The roofline object headed by the binding roof: the FP32 lanes when the
    step's minimum FP32 time exceeds its minimum HBM time, else HBM; the other
    roof is kept beside it, and both minimum times (ms per step) with it."""
    if fp32_floor_s > hbm_floor_s:
        out = dict(fp32, **{k: hbm[k] for k in ("kernel", "launches", "avg_launch_ms", "share_of_step", "traffic")})
        out["hbm"] = {k: hbm[k] for k in ("bound", "achieved", "peak", "unit", "frac", "peak_kind",
                                           "frac_of_nominal_8tbs", "bytes_per_launch")}
    else:
        out = dict(hbm, fp32=fp32)
    out["floors_ms"] = {"fp32": 1e3 * fp32_floor_s / steps, "hbm": 1e3 * hbm_floor_s / steps}
    return out


def dominant_roofline(info, per_launch, steps, peak, peak_kind, n=None):
    tot, cnt, byt = {}, {}, {}
    for k in range(steps):
        for i, (name, b) in enumerate(info):
            tot[name] = tot.get(name, 0.0) + per_launch[k][i]
            cnt[name] = cnt.get(name, 0) + 1
            byt[name] = byt.get(name, 0.0) + b
    dom = max(tot, key=tot.get)
    achieved = byt[dom] / (tot[dom] / 1e3) / 1e9
    traffic, tsrc = traffic_from_profiles(dom.split("<")[0], n) if n is not None else (None, None)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_source": os.path.basename(tsrc) if tsrc else None,
            "kernel": dom, "launches": cnt[dom], "avg_launch_ms": tot[dom] / cnt[dom],
            "bytes_per_launch": byt[dom] / cnt[dom], "peak_kind": peak_kind,
            "share_of_step": tot[dom] / sum(tot.values())}


def enc2b_fidelity_24q(S, C, seed):
    """1 - F of the two-byte code against FP64 on the 24-qubit instance of the
    depth-12 random circuit: the encoded run (decoded to complex64) against
    the library's complex128 run of the same circuit (the FP64 reference on
    the GPU; the tests hold it to the oracle within 1e-12)."""
    import torch

    n = 24
    circ = C.random_circuit(n, 12, seed)
    enc = S.StateVector(n, "enc2b")
    enc.run(circ, "pergate")
    dec = S.StateVector(n, "c64")
    enc.decode_to(dec)
    ref = S.StateVector(n, "c128")
    ref.run(circ, "tiled")
    torch.cuda.synchronize()
    a = ref.buffer.view(torch.complex128)
    b = dec.buffer.view(torch.complex64).to(torch.complex128)
    f = float(abs(torch.vdot(a, b)) ** 2 / (torch.vdot(a, a).real * torch.vdot(b, b).real))
    for st in (enc, dec, ref):
        st.free()
    del enc, dec, ref, a, b
    torch.cuda.empty_cache()
    return {"workload": f"random circuit, {n} qubits, depth 12, seed {seed} ({len(circ)} gates)",
            "one_minus_fidelity": 1.0 - f, "fidelity": f,
            "reference": "complex128 run of the same circuit on the GPU (held to the FP64 oracle within 1e-12 by the tests)"}


def bench_enc2b(S, C, args, world, peak, peak_kind):
    """Two-byte code at 35 qubits (2^35 x 2 B + 2^27 x 4 B = 64.5 GB): the
    whole depth-12 random circuit (624 gates), one decode-gate-encode pass per
    gate (code-level fast paths for signs and X), timed once after a warm-up
    of its first layer; plus the 24-qubit fidelity against FP64."""
    import torch

    n, depth = 35, 12
    need = S.sv_bytes_required(n, "enc2b")
    if torch.cuda.mem_get_info()[0] < need + (8 << 30):
        return {"skipped": "not enough device memory"}
    circ = C.random_circuit(n, depth, args.seed)
    layer = C.Circuit(n)
    layer.gates = circ.gates[: n + n // 2]
    st = S.StateVector(n, "enc2b")
    warm = st.plan(layer, "pergate")
    warm.execute()
    warm.free()
    plan = st.plan(circ, "pergate")
    info = plan.launch_info()
    t, per_launch = time_plan(S, st, plan, 1, 0, world)
    out = {"workload": f"the {n}-qubit depth-{depth} random circuit ({plan.gates} gates), two-byte code "
                       f"({need / 2**30:.1f} GiB), from |0...0>",
           "s_per_circuit": t, "gates_per_s": plan.gates / t, "ms_per_gate": 1e3 * t / plan.gates,
           "layers_per_s": depth / t, "gbs": plan.bytes / t / 1e9, "launches": plan.passes,
           "roofline": dominant_roofline(info, per_launch, 1, peak, peak_kind, n)}
    plan.free()
    st.free()
    del st
    torch.cuda.empty_cache()
    out["fidelity_24q"] = enc2b_fidelity_24q(S, C, args.seed)
    return out


def bench_cut(S, C):
    """Decomposition of the 48-qubit 6x8 grid (depth 8, S = 8): 256 branches
    x 2 halves of 2^24 amplitudes (two batched 2^32 complex64 vectors),
    1024 output amplitudes; the second of two calls is timed (the first
    compiles the passes)."""
    import torch

    if torch.cuda.mem_get_info()[0] < (72 << 30):
        return {"skipped": "not enough device memory"}
    c = C.grid_circuit(6, 8, 8, 1)
    mask = C.grid_partition_mask(6, 8, 3)
    z = C.random_bitstrings(1024, 48, 7)
    times = {}
    for label, flag in (("batched", "0"), ("prefix", "1")):
        os.environ["SV_CUT_PREFIX"] = flag
        S.sv_cut_amplitudes(c, 48, mask, z)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        amps, s = S.sv_cut_amplitudes(c, 48, mask, z)
        torch.cuda.synchronize()
        times[label] = time.perf_counter() - t0
    os.environ.pop("SV_CUT_PREFIX", None)
    return {"workload": "6x8 grid, 48 qubits, depth 8, rows 0-2 | 3-5, projector decomposition", "cut_gates": s,
            "branches": 1 << s, "amplitudes": int(z.size), "ms_per_call": 1e3 * times["prefix"],
            "ms_per_call_batched": 1e3 * times["batched"],
            "note": "end to end: planning, allocation, both halves (branch-prefix sharing; batched: every branch "
                    "from the first gate), FP64 branch sum, copy back",
            "mean_abs2_times_2^48": float((abs(amps) ** 2).mean() * 2.0 ** 48)}


def bench_qft(S, C, hbm_peak):
    """QFT-32 of the basis state x = 0x9E3779B9 (32 H + 496 CP + 16 SWAP, 544
    gates), complex64, tiled and fused modes; sampled amplitudes against the
    closed form 2^(-16) exp(2 pi i x y / 2^32)."""
    import numpy as np
    import torch

    n, x = 32, 0x9E3779B9
    circ = C.qft_circuit(n, x)
    st = S.StateVector(n, "c64")
    out = {"workload": f"QFT-32 of |{x:#x}>, {len(circ)} gates, complex64"}
    ys = np.array([0, 1, 12345, x, (1 << 32) - 1, 0xDEADBEEF], dtype=np.uint64)
    for mode in ("tiled", "fused"):
        plan = st.plan(circ, mode)
        t, _ = time_plan(S, st, plan, 2, 1, 1)
        st.set_basis(0)
        plan.execute()
        got = st.amplitudes(ys)
        ref = 2.0 ** -16 * np.exp(2j * np.pi * ((x * ys.astype(object)) % (1 << 32)).astype(np.float64) / 2.0 ** 32)
        out[mode] = {"gates_per_s": plan.gates * 2 / t, "ms_per_circuit": 1e3 * t / 2, "launches": plan.passes,
                     "gbs": plan.bytes * 2 / t / 1e9,
                     "max_abs_err_sampled": float(np.max(np.abs(got - ref))) / 2.0 ** -16}
        plan.free()
    st.free()
    del st
    torch.cuda.empty_cache()
    return out


def bench_h_sweep(S, C, hbm_peak, peak_kind):
    """Dense H on every target t = 0..31 of a 32-qubit complex64 state, one
    per-gate launch each (68.7 GB algorithmic), against the measured HBM copy
    rate."""
    import torch

    n = 32
    st = S.StateVector(n, "c64")
    rates = []
    for t in range(n):
        c = C.Circuit(n)
        c.add("H", t)
        plan = st.plan(c, "pergate")
        _, per_launch = time_plan(S, st, plan, 2, 1, 1)
        ms = sum(per_launch[k][0] for k in range(2)) / 2
        rates.append(plan.bytes / (ms / 1e3) / 1e9)
        plan.free()
    st.free()
    del st
    torch.cuda.empty_cache()
    srt = sorted(rates)
    return {"workload": "H on target t = 0..31, 32 qubits complex64, one launch each",
            "gbs_per_target": [round(r, 1) for r in rates], "min_gbs": srt[0], "median_gbs": srt[len(srt) // 2],
            "min_frac": srt[0] / hbm_peak, "peak": hbm_peak, "peak_kind": peak_kind}


def bench_30q(S, C, hbm_peak):
    """The 30-qubit depth-16 random circuit (712 gates) in tiled mode, complex64
    (8 GiB) and complex128 (16 GiB; its passes are bound by GB300's FP64 rate)."""
    import torch

    n, depth = 30, 16
    circ = C.random_circuit(n, depth, 1)
    out = {"workload": f"random circuit, {n} qubits, depth {depth}, seed 1 ({len(circ)} gates), tiled"}
    for dt, steps in (("c64", 3), ("c128", 1)):
        st = S.StateVector(n, dt)
        plan = st.plan(circ, "tiled")
        t, _ = time_plan(S, st, plan, steps, 1, 1)
        gbs = plan.bytes * steps / t / 1e9
        out[dt] = {"gates_per_s": plan.gates * steps / t, "ms_per_circuit": 1e3 * t / steps, "launches": plan.passes,
                   "gbs": gbs, "frac_of_measured_hbm": gbs / hbm_peak}
        plan.free()
        st.free()
        del st
        torch.cuda.empty_cache()
    return out


def bench_expect(S, C, hbm_peak):
    """<sigma^alpha_i> for all 32 qubits and alpha = x, y, z of the 32-qubit
    uniform superposition (Sec. 3 validation observable): read-only passes
    over the 32 GiB state, 2^13-amplitude tiles of which the later passes
    share SV_EXPECT_LOW (default 3) low qubits with the first:
    1 + ceil((32 - 13) / (13 - 3)) = 3."""
    import numpy as np
    import torch

    n = 32
    st = S.StateVector(n, "c64")
    st.run(C.uniform_circuit(n), "tiled")
    st.expect_pauli()
    torch.cuda.synchronize()
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        sig = st.expect_pauli()
    t = (time.perf_counter() - t0) / reps
    low = max(3, min(8, int(os.environ.get("SV_EXPECT_LOW", "3"))))
    passes = 1 + -(-(n - 13) // (13 - low))
    q = (1 - sig / st.norm()) / 2
    st.free()
    del st
    torch.cuda.empty_cache()
    gbs = passes * (8 << n) / t / 1e9
    return {"workload": "uniform superposition, 32 qubits, <Q_alpha(i)> for all i and alpha (96 values)",
            "ms_per_call": 1e3 * t, "passes": passes, "read_gbs": gbs, "frac_of_measured_hbm": gbs / hbm_peak,
            "max_dev_from_paper_values": float(max(np.max(np.abs(q[:, 0])), np.max(np.abs(q[:, 1:] - 0.5)))),
            "note": "host wall time of the synchronous call (passes, partial-sum copies and host sums)"}


def bench_ghz_sweep(S, C):
    """The circuit of the paper's weak-scaling figures (Sec. 3, Figs. 1-2): H on
    qubit 0, CNOT(i, i+1) for i = 0..n-2, then <sigma^alpha_i> of every qubit;
    elapsed time per gate operation against n on one GPU, normalised like the
    figures by the value at n = 32 (complex64) and n = 35 (two-byte code).
    The timed execution replays the plan's CUDA graph (captured in warm-up)."""
    import torch

    out = {"workload": "H(0) + CNOT chain + all expectation values, per-gate mode, one GPU"}
    for dt, ns, nref in (("c64", range(20, 35, 2), 32), ("enc2b", list(range(21, 36, 2)) + [36], 35)):
        rows = {}
        for n in ns:
            if torch.cuda.mem_get_info()[0] < S.sv_bytes_required(n, dt) + (8 << 30):
                continue
            st = S.StateVector(n, dt)
            circ = C.ghz_circuit(n)
            plan = st.plan(circ, "pergate")
            for _ in range(2):  # direct launches, then the CUDA-graph capture
                st.set_basis(0)
                plan.execute()
            st.expect_pauli()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st.set_basis(0)
            plan.execute()
            sig = st.expect_pauli()
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            rows[n] = {"s_per_gate": t / plan.gates, "gates": plan.gates,
                       "z0": float(sig[0, 2] / max(st.norm(), 1e-300))}
            plan.free()
            st.free()
            del st
            torch.cuda.empty_cache()
        ref = rows.get(nref, {}).get("s_per_gate")
        for n, r in rows.items():
            # the figures' form (time per gate / time at the reference n), and
            # the one-GPU analogue of weak scaling: per amplitude
            r["normalised"] = r["s_per_gate"] / ref if ref else None
            r["normalised_per_amplitude"] = r["s_per_gate"] * 2.0 ** (nref - n) / ref if ref else None
        out[dt] = {"reference_n": nref, "by_n": rows}
    out["paper_reference"] = ("elapsed s per gate at the normalisation point: JUQCS-E N=32 0.9 (JUWELS) ... 5.1 "
                              "(Sunway); JUQCS-A N=35 2.2 (JUWELS) ... 19.9 (Sunway); other hardware, context only")
    return out


def cut_gates_42q(depth: int) -> int:
    """Cut gates of the 6x7 grid (rows 0-2 | 3-5) after `depth` layers: the
    vertical edges between rows 2 and 3 appear in patterns C (4 of them, even
    columns) and D (3, odd columns), layers 2 and 3 of every six, so S grows
    by 7 per six layers: 14 at depth 14, 18 at 15, 21 at 16-20, 25 at 21, 28
    at 22-25."""
    full, rem = divmod(depth, 6)
    return 7 * full + (4 if rem > 2 else 0) + (3 if rem > 3 else 0)


def bench_cut42_depth(S, C, budget_s: float = 60.0):
    """Decomposition at the paper's scale (Sec. 4, Fig. 4 workload shape): a
    42-qubit 6x7 grid circuit cut between rows 0-2 and 3-5 (21 + 21 qubits),
    1024 seeded amplitudes.  The branches are split into 2^p parts (p chosen
    so a partition's batched vector holds at most 2^31 amplitudes) that run
    one after another on this GPU with the same compiled passes and are summed
    in FP64 on the device (one sv_cut_amplitudes_parts call); a first call on
    one part compiles.  Depths 4-14 also run the Eq. 2 form (the two forms
    must agree); 15 and 16 (S = 18, 21) the projector form, while the
    projected time stays inside the budget.  Depths 17-20 have the same S as
    16; 21-25 need 2^4 to 2^7 times the work of depth 16 (S = 25, 28) and are
    out of reach of a bench run."""
    import numpy as np
    import torch

    n, mask = 42, C.grid_partition_mask(6, 7, 3)
    z = C.random_bitstrings(1024, n, 7)
    rows, spent = {}, 0.0
    for depth in (4, 6, 8, 10, 12, 14, 15, 16):
        c = C.grid_circuit(6, 7, depth, 1)
        _, s = S.sv_cut_amplitudes_part(c, n, mask, z[:0], 0, 16)  # m = 0: counts the cut gates only
        assert s == cut_gates_42q(depth)
        plog = max(0, 21 + s - 31)
        parts = list(range(1 << plog))
        res = {}
        for form in ((0, 1) if depth <= 14 else (0,)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            S.sv_cut_amplitudes_parts(c, n, mask, z, plog, [0], form=form)  # compiles, runs one part
            torch.cuda.synchronize()
            tpart = time.perf_counter()
            if len(parts) > 1:  # one compiled part, for the projection
                S.sv_cut_amplitudes_parts(c, n, mask, z, plog, [1], form=form)
                torch.cuda.synchronize()
            t1 = time.perf_counter()
            est = (t1 - tpart) * len(parts)
            if depth > 14 and spent + est > budget_s:
                rows[depth] = {"gates": len(c), "cut_gates": s, "parts": len(parts),
                               "skipped": f"projected {est:.0f} s (one compiled part x {len(parts)}) exceeds the "
                                          f"remaining budget of {budget_s - spent:.0f} s"}
                break
            a, _ = S.sv_cut_amplitudes_parts(c, n, mask, z, plog, parts, form=form)
            torch.cuda.synchronize()
            t = time.perf_counter() - t1
            spent += time.perf_counter() - t0
            res[form] = (a, t, tpart - t0)
        if 0 not in res:
            continue
        a0, t, tc = res[0]
        row = {"gates": len(c), "cut_gates": s, "parts": len(parts), "s_per_call": t,
               "ms_per_gate": 1e3 * t / len(c), "s_first_part_with_compile": tc,
               "mean_abs2_times_2^42": float(np.mean(np.abs(a0) ** 2) * 2.0 ** n)}
        if 1 in res:
            a1, t1_, _ = res[1]
            row["s_per_call_eq2"] = t1_
            row["forms_max_rel_diff"] = float(np.max(np.abs(a0 - a1)) / np.max(np.abs(a0)))
        rows[depth] = row
    return {"workload": "6x7 grid (42 qubits), rows 0-2 | 3-5, 1024 amplitudes, branch parts summed on the device",
            "budget_s": budget_s, "by_depth": rows}


def bench_batch(S, C):
    """Many independent circuits of uneven size (64 random circuits, n drawn
    from 13..22, depth 10, complex64) run as one batch (each member its own
    chain of compiled passes in one CUDA graph) against the same members run
    one after another on one stream (each plan replaying its own graph):
    aggregate gates/s.  The states total 2^13..2^22 amplitudes each."""
    import numpy as np
    import torch

    rng = np.random.default_rng(64)
    ns = [int(x) for x in rng.integers(13, 23, size=64)]
    circs = [C.random_circuit(n, 10, 500 + i) for i, n in enumerate(ns)]
    states = [S.StateVector(n, "c64") for n in ns]
    batch = S.Batch(states, circs)
    plans = [st.plan(c, "tiled") for st, c in zip(states, circs)]
    reps = 20

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    def one_by_one():
        for p in plans:
            p.execute()

    t_batch = timed(batch.execute)
    t_seq = timed(one_by_one)
    gates = batch.gates
    out = {"workload": f"64 random circuits, n in 13..22 (sum 2^n = {sum(1 << n for n in ns)} amplitudes), depth 10, "
                       f"complex64, {gates} gates, {batch.launches} pass launches",
           "batched": {"ms": 1e3 * t_batch, "gates_per_s": gates / t_batch, "gbs": batch.bytes / t_batch / 1e9},
           "one_by_one": {"ms": 1e3 * t_seq, "gates_per_s": gates / t_seq, "gbs": batch.bytes / t_seq / 1e9},
           "speedup": t_seq / t_batch, "uses_graph": batch.info().uses_graph,
           "note": "host wall time per execution of all members (asynchronous launches, synchronised every 20)"}
    for p in plans:
        p.free()
    batch.free()
    for st in states:
        st.free()
    torch.cuda.empty_cache()
    return out


def bench_ghz128(S, C):
    """The paper's largest decomposition run (Sec. 4): the 128-qubit GHZ chain
    (H(0), CNOT(i, i+1)) in 8 partitions of 16 qubits (7 decomposed CNOTs),
    M = 2^27 coefficients: the first 2^27 - 1 basis states and |1...1>.
    <0...0|C|0> and <1...1|C|0> must be 1/sqrt(2), every other one 0."""
    import math

    import numpy as np
    import torch

    n, m = 128, 1 << 27
    z = np.zeros((m, 2), dtype=np.uint64)
    z[: m - 1, 0] = np.arange(m - 1, dtype=np.uint64)
    z[m - 1] = np.uint64(0xFFFFFFFFFFFFFFFF)
    part_of = [q // 16 for q in range(n)]
    c = C.ghz_circuit(n)
    S.sv_cut_amplitudes_multi(c, n, part_of, z[:1024])  # compiles the passes
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    amps, s = S.sv_cut_amplitudes_multi(c, n, part_of, z)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    h = 1 / math.sqrt(2)
    return {"workload": "GHZ chain, 128 qubits, 8 partitions x 16, M = 2^27 coefficients", "cut_gates": s,
            "s_per_call": t, "coefficients_per_s": m / t,
            "amp_0": [float(amps[0].real), float(amps[0].imag)], "amp_1s": [float(amps[-1].real), float(amps[-1].imag)],
            "max_err_vs_paper": float(max(abs(amps[0] - h), abs(amps[-1] - h), np.max(np.abs(amps[1:-1])))),
            "note": "end to end: host bit strings (2 GiB) in, 2^27 complex128 out"}


def summarize(line: dict) -> dict:
    """Headline figures of the comparisons and extras, a few hundred bytes."""
    def g(d, *path):
        for k in path:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return round(d, 4) if isinstance(d, float) else d

    out = {"tiled_gates_per_s": g(line, "value"), "ms_per_step": g(line, "ms_per_step"),
           "fp32_frac": g(line, "roofline", "frac"), "hbm_frac": g(line, "roofline", "hbm", "frac"),
           "per_pass_floor_ms": g(line, "roofline", "floors_ms", "per_pass_max_sum"),
           "autotune_chosen": g(line, "config", "autotune", "chosen"),
           "fused_gates_per_s": g(line, "compare", "fused", "gates_per_s"),
           "pergate_gates_per_s": g(line, "compare", "pergate", "gates_per_s"),
           "pergate_hbm_frac": g(line, "compare", "pergate", "roofline", "frac")}
    ex = line.get("extras") or {}
    out["enc2b_35q"] = {"s_per_circuit": g(ex, "enc2b_35q", "s_per_circuit"),
                        "gates_per_s": g(ex, "enc2b_35q", "gates_per_s"),
                        "one_minus_fidelity_24q": g(ex, "enc2b_35q", "fidelity_24q", "one_minus_fidelity")}
    out["cut_48q_ms"] = g(ex, "cut_48q", "ms_per_call")
    out["qft_32q_gates_per_s"] = g(ex, "qft_32q", "tiled", "gates_per_s")
    out["h_sweep_min_frac"] = g(ex, "h_sweep_32q", "min_frac")
    out["random_30q_gates_per_s"] = {"c64": g(ex, "random_30q", "c64", "gates_per_s"),
                                     "c128": g(ex, "random_30q", "c128", "gates_per_s")}
    out["expect_32q_ms"] = g(ex, "expect_32q", "ms_per_call")
    out["batch_64_speedup"] = g(ex, "batch_64", "speedup")
    depths = (g(ex, "cut_42q_depth", "by_depth") or {})
    out["cut_42q_s_by_depth"] = {str(k): (round(v["s_per_call"], 3) if "s_per_call" in v else "skipped")
                                 for k, v in depths.items()}
    out["ghz128_s"] = g(ex, "ghz128_m2e27", "s_per_call")
    return out


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_1912_03243_gb300 import build as B
    from paper_1912_03243_gb300 import circuits as C
    from paper_1912_03243_gb300 import sv as S

    if not os.path.exists(S.LIB_PATH):
        B.build()
    S.lib()
    circ, desc = workload(args)
    state = S.StateVector(args.n, "c64")
    tuning = None
    if args.mode == "auto":
        # the library's autotuner times every candidate (tiled configurations,
        # fused k = 3..6) on a scratch state and keeps the fastest
        plan = state.plan(circ, "auto")
        tuning = plan.tuning()
        mode = tuning["chosen"].split()[0]
    else:
        mode, plan = args.mode, state.plan(circ, args.mode)
    info = plan.launch_info()
    hbm_peak, peak_kind = peaks()

    with ClockSampler(local) as clk:
        t, per_launch = time_plan(S, state, plan, args.steps, args.warmup, world)
    clocks = clk.summary()
    gates = plan.gates
    value = gates * args.steps * world / t
    ms_per_step = 1e3 * t / args.steps
    gbs = plan.bytes * args.steps * world / t / 1e9

    # dominant kernel: largest total device time over the timed steps
    tot, cnt, byt = {}, {}, {}
    for k in range(args.steps):
        for i, (name, b) in enumerate(info):
            tot[name] = tot.get(name, 0.0) + per_launch[k][i]
            cnt[name] = cnt.get(name, 0) + 1
            byt[name] = byt.get(name, 0.0) + b
    dom = max(tot, key=tot.get)
    achieved = byt[dom] / (tot[dom] / 1e3) / 1e9
    traffic, tsrc = traffic_from_profiles(dom.split("<")[0], args.n)
    launches_per_step = len(info)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": traffic,
                "kernel": dom, "launches": cnt[dom], "avg_launch_ms": tot[dom] / cnt[dom],
                "bytes_per_launch": byt[dom] / cnt[dom], "peak_kind": peak_kind,
                "frac_of_nominal_8tbs": achieved / 8000.0,
                "share_of_step": tot[dom] / sum(tot.values())}

    # The tiled passes can be bound by FP32 arithmetic more than by HBM: the
    # same launches against the FP32 lanes (152 SMs x 128 lanes x SM clock)
    # with the algorithmic operations the gates need.  Whichever roof gives
    # the longer minimum time for the step is the binding one and heads the
    # roofline object; the other is kept beside it.
    if mode == "tiled":
        ops = fp32_ops_per_amplitude(circ) * (1 << args.n) * args.steps
        secs = sum(tot.values()) / 1e3
        mhz = clocks.get("sm_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        peak_ops = sms * 128 * mhz * 1e6
        roofline_fp32 = {"bound": "alu", "achieved": ops / secs / 1e12, "peak": peak_ops / 1e12,
                         "unit": "T FP32 lane-ops/s", "frac": ops / secs / peak_ops,
                         "ops_per_amplitude": fp32_ops_per_amplitude(circ),
                         "peak_kind": f"derived: {sms} SMs (cudaDevAttrMultiProcessorCount) x 128 FP32 lanes x "
                                      f"the sampled SM clock ({mhz:.0f} MHz)",
                         "note": "2 per amplitude for each H/SX/SY (one addition per real component), 1 for T "
                                 "(two additions on half the amplitudes), 0 for CZ"}
        fp32_floor = ops / peak_ops
        hbm_floor = sum(byt.values()) / (hbm_peak * 1e9)
        roofline = binding_roofline(roofline, roofline_fp32, fp32_floor, hbm_floor, args.steps)
        # per pass: measured time against its own two floors (the pass's FP32
        # work at the lane peak, its read + write of the state at the copy rate)
        stats = plan.launch_stats()
        per_pass = []
        for i, (nm, b) in enumerate(info):
            ms = sum(per_launch[k][i] for k in range(args.steps)) / args.steps
            f32 = 1e3 * stats[i][0] * (1 << args.n) / peak_ops
            hb = 1e3 * b / (hbm_peak * 1e9)
            per_pass.append({"ms": round(ms, 3), "fp32_floor_ms": round(f32, 3), "hbm_floor_ms": round(hb, 3),
                             "lane_ops_per_amp": stats[i][0], "segments": stats[i][1],
                             "frac_of_binding_floor": round(max(f32, hb) / ms, 3)})
        roofline["per_pass"] = per_pass
        roofline["floors_ms"]["per_pass_max_sum"] = sum(max(r["fp32_floor_ms"], r["hbm_floor_ms"]) for r in per_pass)

    # accuracy: the circuit followed by its inverse returns |0...0>
    inv = state.plan(C.inverse_circuit(circ), mode)
    state.set_basis(0)
    plan.execute()
    inv.execute()
    a0 = state.amplitudes([0])[0]
    nrm = state.norm()
    roundtrip_infidelity = 1.0 - abs(a0) ** 2 / nrm
    norm_drift = nrm - 1.0
    inv.free()

    # comparison: the other modes on the same workload (fused k-qubit blocks on
    # the tensor cores; the plain per-gate path)
    compare = {}
    for other in ("fused", "pergate"):
        if other == mode or args.compare_steps <= 0:
            continue
        pg = state.plan(circ, other)
        pinfo = pg.launch_info()
        tp, plaunch = time_plan(S, state, pg, args.compare_steps, 1, world)
        kernels = sorted({k for k, _ in pinfo})
        compare[other] = {"gates_per_s": pg.gates * args.compare_steps * world / tp,
                          "gbs": pg.bytes * args.compare_steps * world / tp / 1e9, "launches_per_step": pg.passes,
                          "ms_per_step": 1e3 * tp / args.compare_steps,
                          "layers_per_s": args.depth * args.compare_steps * world / tp,
                          "kernels": kernels[:4],
                          "roofline": dominant_roofline(pinfo, plaunch, args.compare_steps, hbm_peak, peak_kind, args.n)}
        if other == "fused":
            state.set_basis(0)
            pg.execute()
            inv = state.plan(C.inverse_circuit(circ), other)
            inv.execute()
            a0 = state.amplitudes([0])[0]
            compare[other]["roundtrip_1_minus_fidelity"] = 1.0 - abs(a0) ** 2 / state.norm()
            inv.free()
        pg.free()

    # end to end through the C ABI with host buffers: circuit text in, 1024
    # amplitudes out, parse + plan + upload + run + read-back every step
    e2e = None
    if not args.no_e2e:
        idx = C.random_bitstrings(1024, args.n, 7)
        text = circ.text()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            state.set_basis(0)
            state.run(text, args.mode)
            amps = state.amplitudes(idx)
        torch.cuda.synchronize()
        te = max_over_ranks(world, time.perf_counter() - t0)
        e2e = {"value": gates * args.steps * world / te, "unit": "gates/s",
               "h2d_bytes_per_step": len(text.encode()) + idx.nbytes, "d2h_bytes_per_step": amps.nbytes,
               "ms_per_step": 1e3 * te / args.steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # most of the time on the largest point (26 qubits, a 1 GiB state, well
        # beyond the host caches), the smaller ones to check the 2^n scaling
        pick = [(m, w) for m, w in ((20, 1.0), (22, 1.0), (24, 2.0), (26, 8.0)) if m <= args.n]
        v, sdesc, tcpu, pts = oracle_sample(args, budget_s=36.0, min_s=24.0, ns=[m for m, _ in pick],
                                            weights=[w for _, w in pick])
        cpu = {"value": v, "unit": "gates/s", "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
               "sample": sdesc, "points": pts}

    plan.free()
    extras = None
    if rank == 0 and world == 1 and not args.no_extras and args.n == 32:
        state.free()
        del state
        torch.cuda.empty_cache()
        extras = {"enc2b_35q": bench_enc2b(S, C, args, world, hbm_peak, peak_kind), "cut_48q": bench_cut(S, C),
                  "qft_32q": bench_qft(S, C, hbm_peak), "h_sweep_32q": bench_h_sweep(S, C, hbm_peak, peak_kind),
                  "random_30q": bench_30q(S, C, hbm_peak), "expect_32q": bench_expect(S, C, hbm_peak),
                  "ghz_sweep": bench_ghz_sweep(S, C), "batch_64": bench_batch(S, C),
                  "cut_42q_depth": bench_cut42_depth(S, C, args.cut42_budget),
                  "ghz128_m2e27": bench_ghz128(S, C)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "n": args.n, "depth": args.depth, "seed": args.seed, "state": "complex64",
                       "mode": mode, "autotune": tuning, "launches_per_step": launches_per_step,
                       "parallelism": f"replicas x{world}",
                       "l2": "state (32 GiB) larger than L2, no flush"},
            "hbm_gbs": gbs, "layers_per_s": args.depth * args.steps * world / t,
            "accuracy": {"roundtrip_1_minus_fidelity": roundtrip_infidelity, "roundtrip_norm_minus_1": norm_drift,
                         "note": "circuit then its inverse from |0...0>; fidelity = |<0|psi>|^2 / ||psi||^2"},
            "compare": compare, "extras": extras, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": args.steps * (launches_per_step + 1),
        }
        # a compact digest of the comparisons and extras last, so that a reader
        # of only the line's end still sees them
        line["summary"] = summarize(line)
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
