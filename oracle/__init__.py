"""CPU oracle for the state-vector simulator -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never does, and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, complex128; the two-byte codec
mirror in FP32 with explicit fmaf).  This module only builds it with gcc and
marshals numpy arrays through ctypes.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fcx-limited-range",
          "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no GPU)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            i8p = ctypes.POINTER(ctypes.c_int8)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            ip = ctypes.POINTER(ctypes.c_int)
            L.orc_last_error.restype = ctypes.c_char_p
            L.orc_gate_matrix.argtypes = [ctypes.c_char_p, dp, ctypes.c_int, dp]
            L.orc_apply_1q.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
            L.orc_apply_1q.restype = None
            L.orc_apply_kq.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, dp]
            L.orc_run.argtypes = [ctypes.c_char_p, ctypes.c_int, dp]
            L.orc_count_gates.argtypes = [ctypes.c_char_p]
            L.orc_dense.argtypes = [ctypes.c_char_p, ctypes.c_int, dp]
            L.orc_norm.argtypes = [dp, ctypes.c_int]
            L.orc_norm.restype = ctypes.c_double
            L.orc_expect_pauli.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
            L.orc_enc_encode.argtypes = [fp, ctypes.c_int, i8p, fp]
            L.orc_enc_decode.argtypes = [i8p, fp, ctypes.c_int, fp]
            L.orc_enc_apply_gate.argtypes = [i8p, fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
            L.orc_enc_run.argtypes = [ctypes.c_char_p, ctypes.c_int, i8p, fp]
            L.orc_eq2_terms.argtypes = [dp, dp, dp]
            L.orc_eq2_terms.restype = None
            L.orc_cut_amplitudes.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                             ctypes.c_int64, u64p, dp, ip]
            L.orc_cut_amplitudes_part.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                                  ctypes.c_uint64, ctypes.c_int, ctypes.c_int64, u64p, dp, ip]
            L.orc_cut_amplitudes_multi.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_ubyte),
                                                   ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                                   ctypes.c_int64, u64p, ctypes.c_int, dp, ip]
            _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc: int) -> None:
    if rc != 0:
        raise OracleError(f"oracle error {rc}: {lib().orc_last_error().decode()}")


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _text(circuit) -> bytes:
    return (circuit if isinstance(circuit, str) else circuit.text()).encode()


def gate_matrix(name: str, params=()) -> np.ndarray:
    p = np.asarray(params, dtype=np.float64)
    out = np.zeros(32, dtype=np.float64)
    k = lib().orc_gate_matrix(name.encode(), _dp(p) if p.size else None, int(p.size), _dp(out))
    if k < 0:
        raise OracleError(f"unknown gate {name}")
    d = 2 if k == 1 else 4
    return out[: 2 * d * d].view(np.complex128).reshape(d, d).copy()


def basis_state(n: int, idx: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[idx] = 1.0
    return psi


def run(circuit, n: int | None = None, psi: np.ndarray | None = None) -> np.ndarray:
    """Apply the circuit (text or Circuit) to psi (default |0...0>)."""
    if n is None:
        n = circuit.n
    if psi is None:
        psi = basis_state(n)
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    _check(lib().orc_run(_text(circuit), n, _dp(psi.view(np.float64))))
    return psi


def apply_1q(psi: np.ndarray, t: int, u: np.ndarray) -> np.ndarray:
    n = int(psi.size).bit_length() - 1
    out = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    um = np.ascontiguousarray(u, dtype=np.complex128).reshape(4)
    lib().orc_apply_1q(_dp(out.view(np.float64)), n, t, _dp(um.view(np.float64)))
    return out


def apply_kq(psi: np.ndarray, qubits, u: np.ndarray) -> np.ndarray:
    n = int(psi.size).bit_length() - 1
    out = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    qs = np.asarray(qubits, dtype=np.int32)
    um = np.ascontiguousarray(u, dtype=np.complex128).reshape(-1)
    _check(lib().orc_apply_kq(_dp(out.view(np.float64)), n, len(qs),
                              qs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(um.view(np.float64))))
    return out


def count_gates(circuit) -> int:
    k = lib().orc_count_gates(_text(circuit))
    if k < 0:
        raise OracleError(lib().orc_last_error().decode())
    return k


def dense(circuit, n: int | None = None) -> np.ndarray:
    if n is None:
        n = circuit.n
    out = np.zeros(2 * (1 << (2 * n)), dtype=np.float64)
    _check(lib().orc_dense(_text(circuit), n, _dp(out)))
    return out.view(np.complex128).reshape(1 << n, 1 << n)


def norm(psi: np.ndarray) -> float:
    n = int(psi.size).bit_length() - 1
    p = np.ascontiguousarray(psi, dtype=np.complex128)
    return float(lib().orc_norm(_dp(p.view(np.float64)), n))


def expect_pauli(psi: np.ndarray, q: int, alpha: str) -> float:
    n = int(psi.size).bit_length() - 1
    p = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros(1, dtype=np.float64)
    _check(lib().orc_expect_pauli(_dp(p.view(np.float64)), n, q, "xyz".index(alpha), _dp(out)))
    return float(out[0])


# --- two-byte codec mirror -------------------------------------------------

ENC_BLOCK = 256


def n_blocks(n: int) -> int:
    return max(1, (1 << n) // ENC_BLOCK)


def enc_encode(psi32: np.ndarray):
    """FP32 complex amplitudes -> (int8 codes [2^n, 2], float32 scales)."""
    n = int(psi32.size).bit_length() - 1
    p = np.ascontiguousarray(psi32, dtype=np.complex64)
    codes = np.zeros(2 << n, dtype=np.int8)
    scales = np.zeros(n_blocks(n), dtype=np.float32)
    _check(lib().orc_enc_encode(p.view(np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n,
                                codes.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                scales.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return codes, scales


def enc_decode(codes: np.ndarray, scales: np.ndarray) -> np.ndarray:
    n = int(codes.size // 2).bit_length() - 1
    c = np.ascontiguousarray(codes, dtype=np.int8)
    s = np.ascontiguousarray(scales, dtype=np.float32)
    out = np.zeros(1 << n, dtype=np.complex64)
    _check(lib().orc_enc_decode(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                s.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n,
                                out.view(np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def enc_zero_state(n: int):
    psi = np.zeros(1 << n, dtype=np.complex64)
    psi[0] = 1.0
    return enc_encode(psi)


def enc_apply_gate(codes, scales, t: int, control: int, u: np.ndarray):
    n = int(codes.size // 2).bit_length() - 1
    c = np.ascontiguousarray(codes, dtype=np.int8).copy()
    s = np.ascontiguousarray(scales, dtype=np.float32).copy()
    um = np.ascontiguousarray(u, dtype=np.complex128).reshape(4)
    _check(lib().orc_enc_apply_gate(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                    s.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n, t, control,
                                    _dp(um.view(np.float64))))
    return c, s


def enc_run(circuit, n: int | None = None, codes=None, scales=None):
    if n is None:
        n = circuit.n
    if codes is None:
        codes, scales = enc_zero_state(n)
    c = np.ascontiguousarray(codes, dtype=np.int8).copy()
    s = np.ascontiguousarray(scales, dtype=np.float32).copy()
    _check(lib().orc_enc_run(_text(circuit), n, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                             s.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return c, s


# --- decomposition (Sec. 4) --------------------------------------------------

def eq2_terms():
    x = np.zeros(2)
    dp_ = np.zeros(4)
    dm = np.zeros(4)
    lib().orc_eq2_terms(_dp(x), _dp(dp_), _dp(dm))
    return complex(x[0], x[1]), dp_.view(np.complex128).copy(), dm.view(np.complex128).copy()


def cut_amplitudes_part(circuit, mask_a: int, z, part: int, nparts_log2: int, form: int = 0,
                        n: int | None = None):
    """Partial Eq. 3 sum over the terms s with s mod 2^nparts_log2 == part."""
    if n is None:
        n = circuit.n
    zz = np.ascontiguousarray(z, dtype=np.uint64)
    out = np.zeros(2 * zz.size, dtype=np.float64)
    s = ctypes.c_int(0)
    _check(lib().orc_cut_amplitudes_part(_text(circuit), n, ctypes.c_uint64(mask_a), form, ctypes.c_uint64(part),
                                         nparts_log2, zz.size, zz.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                         _dp(out), ctypes.byref(s)))
    return out.view(np.complex128).copy(), s.value


def bit_words(idx, n: int) -> np.ndarray:
    """Python-int bit strings -> (m, ceil(n/64)) little-endian uint64 words."""
    nw = (n + 63) // 64
    out = np.zeros((len(idx), nw), dtype=np.uint64)
    for j, v in enumerate(idx):
        v = int(v)
        for w in range(nw):
            out[j, w] = (v >> (64 * w)) & ((1 << 64) - 1)
    return out


def cut_amplitudes_multi(circuit, part_of, z, form: int = 0, part: int = 0, nparts_log2: int = 0,
                         n: int | None = None):
    """Eq. 3 over P partitions (part_of[q] = partition of qubit q); z: Python
    ints or (m, ceil(n/64)) uint64 words.  Returns (amplitudes, S)."""
    if n is None:
        n = circuit.n
    po = np.ascontiguousarray(part_of, dtype=np.uint8)
    z = np.asarray(z)
    zz = np.ascontiguousarray(z if z.dtype == np.uint64 and z.ndim == 2 else bit_words(list(z), n), dtype=np.uint64)
    m = zz.shape[0]
    out = np.zeros(2 * m, dtype=np.float64)
    s = ctypes.c_int(0)
    _check(lib().orc_cut_amplitudes_multi(_text(circuit), n, po.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                          int(po.max()) + 1, form, ctypes.c_uint64(part), nparts_log2, m,
                                          zz.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), zz.shape[1], _dp(out),
                                          ctypes.byref(s)))
    return out.view(np.complex128).copy(), s.value


def cut_amplitudes(circuit, mask_a: int, z, form: int = 0, n: int | None = None):
    """<z|C|0> via the branch sum of Eq. 3; returns (amplitudes, S)."""
    if n is None:
        n = circuit.n
    zz = np.ascontiguousarray(z, dtype=np.uint64)
    out = np.zeros(2 * zz.size, dtype=np.float64)
    s = ctypes.c_int(0)
    _check(lib().orc_cut_amplitudes(_text(circuit), n, ctypes.c_uint64(mask_a), form, zz.size,
                                    zz.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _dp(out),
                                    ctypes.byref(s)))
    return out.view(np.complex128).copy(), s.value
