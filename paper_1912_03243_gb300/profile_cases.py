"""Small, fixed invocations of each kernel family, for profiler captures.

    python -m paper_1912_03243_gb300.profile_cases <case>

Cases (each a few GB of device memory at most, states larger than L2):
  tiled    28 qubits, random circuit depth 4, tiled passes (compiled kernels)
  tiled24  28 qubits, random circuit depth 24 (passes as full as at 32 qubits)
  pergate  28 qubits, random circuit depth 1, one launch per gate
  enc      28 qubits, two-byte code, random circuit depth 1
  fused    26 qubits, three dense 6-qubit blocks on the tensor cores
           (low, high and mixed qubits)
  cut      6x4 grid (24 qubits), depth 12, 8 cut CZs: 256 branches x 2
           batched halves of 2^12 amplitudes each
  expect   28 qubits, uniform superposition, <sigma^alpha_i> of every qubit
           (complex64; then the same from the two-byte code)
"""

from __future__ import annotations

import sys

import numpy as np


def main(case: str) -> None:
    from paper_1912_03243_gb300 import build
    from paper_1912_03243_gb300 import circuits as C
    from paper_1912_03243_gb300 import sv

    build.build()
    if case == "tiled":
        s = sv.StateVector(28, "c64")
        s.run(C.random_circuit(28, 4, 1), "tiled")
    elif case == "tiled24":
        s = sv.StateVector(28, "c64")
        s.run(C.random_circuit(28, 24, 1), "tiled")
    elif case == "pergate":
        s = sv.StateVector(28, "c64")
        s.run(C.random_circuit(28, 1, 1), "pergate")
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
    elif case == "cut":
        c = C.grid_circuit(6, 4, 12, 1)
        sv.sv_cut_amplitudes(c, 24, C.grid_partition_mask(6, 4, 3), C.random_bitstrings(1024, 24, 7))
        print("ok")
        return
    else:
        raise SystemExit(f"unknown case {case!r}")
    s.sync()
    print("ok")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "tiled")
