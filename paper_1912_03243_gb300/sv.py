"""Thin ctypes binding of libsv (include/sv.h).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  The module-level functions carry the C names; ``StateVector`` wraps
a handle whose storage is a torch CUDA tensor attached with ``sv_attach`` and
whose stream is torch's current stream.  There is no CPU fallback: if
``libsv.so`` is missing or fails to load, every call raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsv.so")

SV_C64, SV_C128, SV_ENC2B = 0, 1, 2
DTYPES = {"c64": SV_C64, "c128": SV_C128, "enc2b": SV_ENC2B}
SV_MODE_PERGATE, SV_MODE_TILED, SV_MODE_FUSED, SV_MODE_AUTO = 0, 1, 2, 3
MODES = {"pergate": SV_MODE_PERGATE, "tiled": SV_MODE_TILED, "fused": SV_MODE_FUSED, "auto": SV_MODE_AUTO}

STATUS = {0: "SV_OK", 1: "SV_ERR_ARG", 2: "SV_ERR_OOM", 3: "SV_ERR_DTYPE", 4: "SV_ERR_CUDA",
          5: "SV_ERR_TIMEOUT", 6: "SV_ERR_STATE", 7: "SV_ERR_PARSE", 8: "SV_ERR_UNSUPPORTED"}

# every symbol include/sv.h declares, with (restype, argtypes)
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_st = ctypes.c_int
SIGNATURES = {
    "sv_bytes_required": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int]),
    "sv_alloc": (_st, [ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "sv_attach": (_st, [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
    "sv_free": (_st, [_vp]),
    "sv_set_basis": (_st, [_vp, ctypes.c_uint64]),
    "sv_sync": (_st, [_vp]),
    "sv_last_error": (ctypes.c_char_p, []),
    "sv_num_qubits": (ctypes.c_int, [_vp]),
    "sv_dtype_of": (ctypes.c_int, [_vp]),
    "sv_apply_gate": (_st, [_vp, ctypes.c_int, ctypes.c_int, _dp]),
    "sv_apply_fused": (_st, [_vp, ctypes.c_int, _ip, _dp]),
    "sv_run_circuit": (_st, [_vp, ctypes.c_char_p, ctypes.c_int]),
    "sv_plan_create": (_st, [_vp, ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(_vp)]),
    "sv_plan_execute": (_st, [_vp]),
    "sv_plan_info": (_st, [_vp, _i64p, _i64p, _dp]),
    "sv_plan_uses_graph": (_st, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "sv_plan_execute_timed": (_st, [_vp, ctypes.POINTER(_vp), ctypes.c_int64]),
    "sv_plan_free": (_st, [_vp]),
    "sv_plan_stats": (_st, [ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64p, _i64p, _i64p]),
    "sv_plan_launch_info": (_st, [_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_char_p), _dp]),
    "sv_plan_launch_stats": (_st, [_vp, ctypes.c_int64, _dp, _i64p]),
    "sv_plan_tuning": (_st, [_vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "sv_plan_pass_source": (_st, [ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_char_p,
                                  ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "sv_fused_tc_layout": (_st, [ctypes.c_int, ctypes.c_int, _ip, ctypes.c_char_p, ctypes.c_size_t, _ip, _ip, _ip,
                                 _ip, _u64p, _u64p, _u64p, ctypes.POINTER(ctypes.c_uint32)]),
    "sv_encode2b": (_st, [_vp, _vp]),
    "sv_decode2b": (_st, [_vp, _vp]),
    "sv_get_codes": (_st, [_vp, ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_float)]),
    "sv_amplitudes": (_st, [_vp, ctypes.c_size_t, _u64p, _dp]),
    "sv_norm": (_st, [_vp, _dp]),
    "sv_expect_pauli": (_st, [_vp, _dp]),
    "sv_amplitudes_noalloc": (_st, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_size_t, _u64p, _dp, _vp]),
    "sv_copy_to_host": (_st, [_vp, _vp, ctypes.c_size_t]),
    "sv_copy_from_host": (_st, [_vp, _vp, ctypes.c_size_t]),
    "sv_cut_amplitudes": (_st, [ctypes.c_char_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t,
                                _u64p, _dp, _ip, _vp]),
    "sv_cut_amplitudes_part": (_st, [ctypes.c_char_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.c_int, ctypes.c_size_t, _u64p, _dp, _ip, _vp]),
    "sv_cut_amplitudes_multi": (_st, [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int,
                                      ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t, _u64p, _dp,
                                      ctypes.POINTER(ctypes.c_int), _vp]),
    "sv_cut_amplitudes_parts": (_st, [ctypes.c_char_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_size_t, _u64p, ctypes.c_size_t, _u64p, _dp, _ip, _vp]),
    "sv_cut_amplitudes_multi_parts": (_st, [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8),
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_size_t, _u64p,
                                            ctypes.c_size_t, _u64p, _dp, _ip, _vp]),
    "sv_batch_create": (_st, [ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_char_p), ctypes.c_int,
                              ctypes.POINTER(_vp)]),
    "sv_batch_execute": (_st, [_vp]),
    "sv_batch_info": (_st, [_vp, _i64p, _i64p, _dp, ctypes.POINTER(ctypes.c_int)]),
    "sv_batch_free": (_st, [_vp]),
    "sv_run_batch": (_st, [ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_char_p), ctypes.c_int]),
    "sv_gate_matrix": (ctypes.c_int, [ctypes.c_char_p, _dp, ctypes.c_int, _dp]),
    "sv_version": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


class SVError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load libsv.so (built by paper_1912_03243_gb300.build); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libsv.so not built ({LIB_PATH}); run paper_1912_03243_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, where: str) -> None:
    if status != 0:
        raise SVError(status, where, lib().sv_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _text(circuit) -> bytes:
    return (circuit if isinstance(circuit, str) else circuit.text()).encode()


# ---- module-level functions with the C names --------------------------------

def sv_bytes_required(n: int, dtype: str | int = "c64") -> int:
    return int(lib().sv_bytes_required(n, DTYPES.get(dtype, dtype)))


def sv_gate_matrix(name: str, params=()) -> np.ndarray:
    p = np.ascontiguousarray(params, dtype=np.float64)
    out = np.zeros(32, dtype=np.float64)
    k = lib().sv_gate_matrix(name.encode(), _dptr(p) if p.size else None, int(p.size), _dptr(out))
    if k < 0:
        raise ValueError(f"unknown gate {name}")
    d = 2 if k == 1 else 4
    return out[: 2 * d * d].view(np.complex128).reshape(d, d).copy()


def sv_cut_amplitudes(circuit, n: int, mask_a: int, z, form: int = 0, stream=None):
    """Eq. 3 branch sum on the GPU; returns (amplitudes complex128[m], S)."""
    import torch

    zz = np.ascontiguousarray(z, dtype=np.uint64)
    out = np.zeros(2 * zz.size, dtype=np.float64)
    s = ctypes.c_int(0)
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    _check(lib().sv_cut_amplitudes(_text(circuit), n, ctypes.c_uint64(mask_a), form, zz.size,
                                   zz.ctypes.data_as(_u64p), _dptr(out), ctypes.byref(s), _vp(st)),
           "sv_cut_amplitudes")
    return out.view(np.complex128).copy(), s.value


def sv_plan_pass_source(circuit, n: int, dtype: str | int, pass_index: int) -> str:
    """Host-only: the generated CUDA source of one pass of the tiled plan."""
    ln = ctypes.c_size_t(0)
    t, dt = _text(circuit), DTYPES.get(dtype, dtype)
    _check(lib().sv_plan_pass_source(t, n, dt, pass_index, None, 0, ctypes.byref(ln)), "sv_plan_pass_source")
    buf = ctypes.create_string_buffer(ln.value + 1)
    _check(lib().sv_plan_pass_source(t, n, dt, pass_index, buf, ln.value + 1, ctypes.byref(ln)),
           "sv_plan_pass_source")
    return buf.value.decode()


def sv_fused_tc_layout(n: int, qubits) -> dict:
    """Host-only: the tensor-core kernel a dense block on these qubits runs
    and its tensor-map layout (see include/sv.h)."""
    qs = np.asarray(list(qubits), dtype=np.int32)
    name = ctypes.create_string_buffer(64)
    tpos = np.zeros(12, np.int32)
    rank, nbox = ctypes.c_int(), ctypes.c_int()
    start = np.zeros(5, np.int32)
    boff, dim, stride = np.zeros(4, np.uint64), np.zeros(5, np.uint64), np.zeros(4, np.uint64)
    box = np.zeros(5, np.uint32)
    _check(lib().sv_fused_tc_layout(n, len(qs), qs.ctypes.data_as(_ip), name, 64, tpos.ctypes.data_as(_ip),
                                    ctypes.byref(rank), ctypes.byref(nbox), start.ctypes.data_as(_ip),
                                    boff.ctypes.data_as(_u64p), dim.ctypes.data_as(_u64p),
                                    stride.ctypes.data_as(_u64p), box.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))),
           "sv_fused_tc_layout")
    return {"kernel": name.value.decode(), "tile_pos": tpos.tolist(), "rank": rank.value, "nbox": nbox.value,
            "start": start.tolist(), "boff": [int(x) for x in boff], "dim": [int(x) for x in dim],
            "stride": [int(x) for x in stride], "box": [int(x) for x in box]}


def tiled_pass_sources(case: str) -> str:
    """Generated sources of every pass of a named tiled case, concatenated:
    "random <n> <depth> <seed> <dtype>" (the random circuit family)."""
    from paper_1912_03243_gb300 import circuits as C

    kind, n, depth, seed, dtype = case.split()
    if kind != "random":
        raise ValueError(f"unknown case {case!r}")
    n, depth, seed = int(n), int(depth), int(seed)
    circ = C.random_circuit(n, depth, seed)
    _, passes, _ = sv_plan_stats(circ, n, dtype)
    return "".join(sv_plan_pass_source(circ, n, dtype, i) for i in range(passes))


def sv_plan_stats(circuit, n: int, dtype: str | int = "c64", compile: bool = False):
    """Host-only tiled planning statistics: (gates, passes, segments)."""
    g, p, s = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().sv_plan_stats(_text(circuit), n, DTYPES.get(dtype, dtype), int(compile), ctypes.byref(g),
                               ctypes.byref(p), ctypes.byref(s)), "sv_plan_stats")
    return g.value, p.value, s.value


def sv_amplitudes_noalloc(state_ptr: int, n: int, dtype: str | int, idx, stream=None) -> np.ndarray:
    """Gather amplitudes from a raw device pointer without any device
    allocation (scratch lives in a fixed device array inside the library)."""
    ii = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.zeros(2 * ii.size, dtype=np.float64)
    if stream is None:
        import torch

        stream = torch.cuda.current_stream().cuda_stream
    _check(lib().sv_amplitudes_noalloc(_vp(state_ptr), n, DTYPES.get(dtype, dtype), ii.size,
                                       ii.ctypes.data_as(_u64p), _dptr(out), _vp(stream)),
           "sv_amplitudes_noalloc")
    return out.view(np.complex128).copy()


def sv_cut_amplitudes_part(circuit, n: int, mask_a: int, z, part: int, nparts_log2: int, form: int = 0,
                           stream=None):
    """Partial Eq. 3 sum over branches s with s mod 2^nparts_log2 == part."""
    import torch

    zz = np.ascontiguousarray(z, dtype=np.uint64)
    out = np.zeros(2 * zz.size, dtype=np.float64)
    s = ctypes.c_int(0)
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    _check(lib().sv_cut_amplitudes_part(_text(circuit), n, ctypes.c_uint64(mask_a), form, ctypes.c_uint64(part),
                                        nparts_log2, zz.size, zz.ctypes.data_as(_u64p), _dptr(out), ctypes.byref(s),
                                        _vp(st)), "sv_cut_amplitudes_part")
    return out.view(np.complex128).copy(), s.value


def sv_cut_amplitudes_parts(circuit, n: int, mask_a: int, z, nparts_log2: int, parts, form: int = 0,
                            stream=None):
    """Eq. 3 summed over the listed branch parts (each < 2^nparts_log2), in
    FP64 on the device: (amplitudes, S)."""
    import torch

    zz = np.ascontiguousarray(z, dtype=np.uint64)
    pl = np.ascontiguousarray(parts, dtype=np.uint64)
    out = np.zeros(2 * zz.size, dtype=np.float64)
    s = ctypes.c_int(0)
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    _check(lib().sv_cut_amplitudes_parts(_text(circuit), n, ctypes.c_uint64(mask_a), form, nparts_log2, pl.size,
                                         pl.ctypes.data_as(_u64p), zz.size, zz.ctypes.data_as(_u64p), _dptr(out),
                                         ctypes.byref(s), _vp(st)), "sv_cut_amplitudes_parts")
    return out.view(np.complex128).copy(), s.value


def sv_cut_amplitudes_multi_parts(circuit, n: int, part_of, z_words, nparts_log2: int, parts, form: int = 0,
                                  stream=None):
    """The same over P partitions (z_words: (m, ceil(n/64)) uint64)."""
    import torch

    po = np.ascontiguousarray(part_of, dtype=np.uint8)
    zz = np.ascontiguousarray(z_words, dtype=np.uint64).reshape(-1, (n + 63) // 64)
    pl = np.ascontiguousarray(parts, dtype=np.uint64)
    out = np.zeros(2 * zz.shape[0], dtype=np.float64)
    s = ctypes.c_int(0)
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    _check(lib().sv_cut_amplitudes_multi_parts(_text(circuit), n, po.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                               int(po.max()) + 1, form, nparts_log2, pl.size,
                                               pl.ctypes.data_as(_u64p), zz.shape[0], zz.ctypes.data_as(_u64p),
                                               _dptr(out), ctypes.byref(s), _vp(st)), "sv_cut_amplitudes_multi_parts")
    return out.view(np.complex128).copy(), s.value


def sv_cut_amplitudes_multi(circuit, n: int, part_of, z_words, form: int = 0, part: int = 0, nparts_log2: int = 0,
                            stream=None):
    """Eq. 3 over P partitions (part_of[q] = partition of qubit q); z_words:
    (m, ceil(n/64)) uint64 bit strings, qubit q = bit q % 64 of word q // 64.
    Returns (amplitudes complex128[m], S)."""
    import torch

    po = np.ascontiguousarray(part_of, dtype=np.uint8)
    zz = np.ascontiguousarray(z_words, dtype=np.uint64).reshape(-1, (n + 63) // 64)
    m = zz.shape[0]
    out = np.zeros(2 * m, dtype=np.float64)
    s = ctypes.c_int(0)
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    _check(lib().sv_cut_amplitudes_multi(_text(circuit), n, po.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                         int(po.max()) + 1, form, ctypes.c_uint64(part), nparts_log2, m,
                                         zz.ctypes.data_as(_u64p), _dptr(out), ctypes.byref(s), _vp(st)),
           "sv_cut_amplitudes_multi")
    return out.view(np.complex128).copy(), s.value


class Plan:
    """A planned circuit (sv_plan_create); execute() replays it."""

    def __init__(self, state: "StateVector", circuit, mode: str | int = "pergate"):
        self.state = state
        self.handle = _vp()
        _check(lib().sv_plan_create(state.handle, _text(circuit), MODES.get(mode, mode), ctypes.byref(self.handle)),
               "sv_plan_create")
        g, p, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().sv_plan_info(self.handle, ctypes.byref(g), ctypes.byref(p), ctypes.byref(b)), "sv_plan_info")
        self.gates, self.passes, self.bytes = g.value, p.value, b.value

    def execute(self) -> None:
        _check(lib().sv_plan_execute(self.handle), "sv_plan_execute")

    def uses_graph(self) -> bool:
        """True once executions replay a CUDA graph (from the second one on)."""
        v = ctypes.c_int()
        _check(lib().sv_plan_uses_graph(self.handle, ctypes.byref(v)), "sv_plan_uses_graph")
        return bool(v.value)

    def execute_timed(self, events) -> None:
        """events: list of torch.cuda.Event (passes + 1), recorded around each launch."""
        arr = (_vp * len(events))(*[_vp(e.cuda_event) for e in events])
        _check(lib().sv_plan_execute_timed(self.handle, arr, len(events)), "sv_plan_execute_timed")

    def tuning(self) -> dict:
        """SV_MODE_AUTO: the measured candidates and the choice ({} otherwise)."""
        import json

        ln = ctypes.c_size_t(0)
        _check(lib().sv_plan_tuning(self.handle, None, 0, ctypes.byref(ln)), "sv_plan_tuning")
        buf = ctypes.create_string_buffer(ln.value + 1)
        _check(lib().sv_plan_tuning(self.handle, buf, ln.value + 1, ctypes.byref(ln)), "sv_plan_tuning")
        return json.loads(buf.value.decode()) if ln.value else {}

    def launch_stats(self):
        """[(FP32 lane operations per amplitude, register segments)] for every
        launch (compiled tile passes; (0, 0) for other launches)."""
        out = []
        ops, seg = ctypes.c_double(), ctypes.c_int64()
        for i in range(self.passes):
            _check(lib().sv_plan_launch_stats(self.handle, i, ctypes.byref(ops), ctypes.byref(seg)),
                   "sv_plan_launch_stats")
            out.append((ops.value, seg.value))
        return out

    def launch_info(self):
        """[(kernel name, algorithmic bytes)] for every launch of one execution."""
        out = []
        name, b = ctypes.c_char_p(), ctypes.c_double()
        for i in range(self.passes):
            _check(lib().sv_plan_launch_info(self.handle, i, ctypes.byref(name), ctypes.byref(b)),
                   "sv_plan_launch_info")
            out.append((name.value.decode(), b.value))
        return out

    def free(self) -> None:
        if self.handle:
            _check(lib().sv_plan_free(self.handle), "sv_plan_free")
            self.handle = _vp()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Batch:
    """Independent circuits on their own states run together (sv_batch_*):
    each member is its own chain of launches in one CUDA graph."""

    def __init__(self, states, circuits):
        if len(states) != len(circuits):
            raise ValueError("one circuit per state")
        self.states = list(states)
        self._texts = [_text(c) for c in circuits]
        hs = (_vp * len(states))(*[s.handle for s in states])
        ts = (ctypes.c_char_p * len(states))(*self._texts)
        self.handle = _vp()
        _check(lib().sv_batch_create(hs, ts, len(states), ctypes.byref(self.handle)), "sv_batch_create")
        self.info()

    def info(self):
        g, n, b, u = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int()
        _check(lib().sv_batch_info(self.handle, ctypes.byref(g), ctypes.byref(n), ctypes.byref(b), ctypes.byref(u)),
               "sv_batch_info")
        self.gates, self.launches, self.bytes, self.uses_graph = g.value, n.value, b.value, bool(u.value)
        return self

    def execute(self) -> None:
        _check(lib().sv_batch_execute(self.handle), "sv_batch_execute")

    def free(self) -> None:
        if self.handle:
            _check(lib().sv_batch_free(self.handle), "sv_batch_free")
            self.handle = _vp()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sv_run_batch(states, circuits) -> None:
    """Run each circuit on its state, all members together, once."""
    texts = [_text(c) for c in circuits]
    hs = (_vp * len(states))(*[s.handle for s in states])
    ts = (ctypes.c_char_p * len(states))(*texts)
    _check(lib().sv_run_batch(hs, ts, len(states)), "sv_run_batch")


class StateVector:
    """An n-qubit state in device memory owned by a torch tensor."""

    def __init__(self, n: int, dtype: str = "c64", device=None, stream=None):
        import torch

        self.n = n
        self.dtype = dtype
        self.dt = DTYPES[dtype]
        nbytes = sv_bytes_required(n, self.dt)
        if nbytes == 0:
            raise ValueError(f"bad qubit count {n}")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.handle = _vp()
        _check(lib().sv_attach(n, self.dt, _vp(self.buffer.data_ptr()), nbytes, _vp(self.stream.cuda_stream),
                               ctypes.byref(self.handle)), "sv_attach")
        self.set_basis(0)

    # lifecycle
    def free(self) -> None:
        if self.handle:
            _check(lib().sv_free(self.handle), "sv_free")
            self.handle = _vp()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def set_basis(self, idx: int = 0) -> None:
        _check(lib().sv_set_basis(self.handle, idx), "sv_set_basis")

    def sync(self) -> None:
        _check(lib().sv_sync(self.handle), "sv_sync")

    # gates
    def apply_gate(self, target: int, u, control: int = -1) -> None:
        m = np.ascontiguousarray(u, dtype=np.complex128).reshape(4)
        _check(lib().sv_apply_gate(self.handle, target, control, _dptr(m.view(np.float64))), "sv_apply_gate")

    def apply_fused(self, qubits, u) -> None:
        qs = np.ascontiguousarray(qubits, dtype=np.int32)
        m = np.ascontiguousarray(u, dtype=np.complex128).reshape(-1)
        _check(lib().sv_apply_fused(self.handle, len(qs), qs.ctypes.data_as(_ip), _dptr(m.view(np.float64))),
               "sv_apply_fused")

    def run(self, circuit, mode: str | int = "pergate") -> None:
        _check(lib().sv_run_circuit(self.handle, _text(circuit), MODES.get(mode, mode)), "sv_run_circuit")

    def plan(self, circuit, mode: str | int = "pergate") -> Plan:
        return Plan(self, circuit, mode)

    # codec
    def encode_from(self, src: "StateVector") -> None:
        _check(lib().sv_encode2b(src.handle, self.handle), "sv_encode2b")

    def decode_to(self, dst: "StateVector") -> None:
        _check(lib().sv_decode2b(self.handle, dst.handle), "sv_decode2b")

    def codes(self):
        nb = max(1, (1 << self.n) >> 8)
        codes = np.zeros(2 << self.n, dtype=np.int8)
        scales = np.zeros(nb, dtype=np.float32)
        _check(lib().sv_get_codes(self.handle, codes.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                  scales.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "sv_get_codes")
        return codes, scales

    # read-out
    def amplitudes(self, idx) -> np.ndarray:
        ii = np.ascontiguousarray(idx, dtype=np.uint64)
        out = np.zeros(2 * ii.size, dtype=np.float64)
        _check(lib().sv_amplitudes(self.handle, ii.size, ii.ctypes.data_as(_u64p), _dptr(out)), "sv_amplitudes")
        return out.view(np.complex128).copy()

    def norm(self) -> float:
        out = ctypes.c_double()
        _check(lib().sv_norm(self.handle, ctypes.byref(out)), "sv_norm")
        return out.value

    def expect_pauli(self) -> np.ndarray:
        """<sigma^alpha_i> for every qubit: an (n, 3) array, columns x, y, z
        (not divided by the norm)."""
        out = np.zeros(3 * self.n, dtype=np.float64)
        _check(lib().sv_expect_pauli(self.handle, _dptr(out)), "sv_expect_pauli")
        return out.reshape(self.n, 3)

    def to_numpy(self) -> np.ndarray:
        """Whole state to host (complex64/complex128; raw bytes for enc2b)."""
        nbytes = sv_bytes_required(self.n, self.dt)
        raw = np.empty(nbytes, dtype=np.uint8)
        _check(lib().sv_copy_to_host(self.handle, raw.ctypes.data_as(_vp), nbytes), "sv_copy_to_host")
        if self.dt == SV_C64:
            return raw.view(np.complex64)
        if self.dt == SV_C128:
            return raw.view(np.complex128)
        return raw

    def from_numpy(self, psi: np.ndarray) -> None:
        want = {SV_C64: np.complex64, SV_C128: np.complex128}.get(self.dt)
        arr = np.ascontiguousarray(psi, dtype=want) if want else np.ascontiguousarray(psi, dtype=np.uint8)
        nbytes = sv_bytes_required(self.n, self.dt)
        if arr.nbytes != nbytes:
            raise ValueError(f"need {nbytes} bytes, got {arr.nbytes}")
        _check(lib().sv_copy_from_host(self.handle, arr.ctypes.data_as(_vp), nbytes), "sv_copy_from_host")
