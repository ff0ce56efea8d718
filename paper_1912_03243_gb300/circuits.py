"""Seeded synthetic circuit generators and the circuit text format.

This module only *names* gates and qubits; it holds none of the simulation
arithmetic (no gate matrices, no amplitudes).  Both the CPU oracle and the GPU
library parse the text it writes, each with its own parser and its own gate
table, so the two sides share inputs but no code.

Text format, one instruction per line (``#`` starts a comment)::

    qubits N
    H q | X q | Y q | Z q | S q | SDG q | T q | TDG q
    SX q | SXDG q | SY q | SYDG q
    P q theta            single-qubit phase diag(1, e^{i theta})
    CZ a b               sign flip where bits a and b are both 1
    CX c t               controlled NOT (control c, target t)
    CP c t theta         controlled phase diag(1,1,1,e^{i theta})
    SWAP a b
    U q u00r u00i u01r u01i u10r u10i u11r u11i     arbitrary 2x2 (row-major)

Qubit j is bit j of the amplitude index (qubit 0 is the least significant
bit).  The paper leaves the ordering open (Sec. 2, after Eq. 1); this is the
reading used throughout.

Generators:

* ``random_circuit`` -- the random circuit family of the benchmarks: every
  layer applies one gate drawn uniformly from {H, T, SX, SY} to every qubit,
  then CZ on alternating neighbour pairs ((0,1),(2,3),... on even layers,
  (1,2),(3,4),... on odd layers).  The paper generates its random circuits
  with the procedure of Boixo et al. (Sec. 4); that procedure is not
  reproduced here, this family stands in for it.
* ``ghz_circuit`` -- H on qubit 0 followed by CNOT(i, i+1) for i = 0..N-2,
  the validation and weak-scaling circuit of Sec. 3 (Figs. 1-3).
* ``uniform_circuit`` -- H on every qubit, the first validation circuit of
  Sec. 3.
* ``qft_circuit`` -- the quantum Fourier transform (not in the paper; a
  circuit with a closed-form output used as a correctness pin).
* ``grid_circuit`` -- a low-depth rows x cols grid circuit: random gates from
  {SX, SY, T} on every qubit, then CZ on one of six edge patterns per layer
  (a stand-in for the paper's Sec. 4 random circuits that are split into two
  partitions).
* ``inverse_circuit`` -- the circuit run backwards with every gate replaced by
  its adjoint, by name.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ONE_QUBIT = ("H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "SX", "SXDG", "SY", "SYDG")
ADJOINT = {
    "H": "H", "X": "X", "Y": "Y", "Z": "Z",
    "S": "SDG", "SDG": "S", "T": "TDG", "TDG": "T",
    "SX": "SXDG", "SXDG": "SX", "SY": "SYDG", "SYDG": "SY",
    "CZ": "CZ", "CX": "CX", "SWAP": "SWAP",
}

RANDOM_1Q = ("H", "T", "SX", "SY")
GRID_1Q = ("SX", "SY", "T")


@dataclass
class Circuit:
    """A circuit as a list of (name, qubits, params) plus its text form."""

    n: int
    gates: list = field(default_factory=list)

    def add(self, name: str, *qubits: int, params: tuple = ()) -> None:
        for q in qubits:
            if not 0 <= q < self.n:
                raise ValueError(f"qubit {q} out of range for n={self.n}")
        self.gates.append((name, tuple(qubits), tuple(params)))

    def text(self) -> str:
        lines = [f"qubits {self.n}"]
        for name, qs, ps in self.gates:
            fields = [name] + [str(q) for q in qs] + [repr(float(p)) for p in ps]
            lines.append(" ".join(fields))
        return "\n".join(lines) + "\n"

    def __len__(self) -> int:
        return len(self.gates)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_circuit(n: int, depth: int, seed: int) -> Circuit:
    """Random layered circuit: {H,T,SX,SY} on every qubit, then CZ pairs.

    Draws are layer-major, qubit-ascending, from numpy's PCG64 seeded with
    ``seed``.  Layer l applies CZ to (2i, 2i+1) if l is even and to
    (2i+1, 2i+2) if l is odd.
    """
    c = Circuit(n)
    draws = _rng(seed).integers(0, len(RANDOM_1Q), size=(depth, n))
    for layer in range(depth):
        for q in range(n):
            c.add(RANDOM_1Q[int(draws[layer, q])], q)
        start = 0 if layer % 2 == 0 else 1
        for a in range(start, n - 1, 2):
            c.add("CZ", a, a + 1)
    return c


def ghz_circuit(n: int) -> Circuit:
    """H(0) then CNOT(i, i+1) for i = 0..n-2 (Sec. 3, Figs. 1-2)."""
    c = Circuit(n)
    c.add("H", 0)
    for i in range(n - 1):
        c.add("CX", i, i + 1)
    return c


def uniform_circuit(n: int) -> Circuit:
    """A Hadamard on every qubit (Sec. 3, first validation circuit)."""
    c = Circuit(n)
    for q in range(n):
        c.add("H", q)
    return c


def basis_prep(c: Circuit, x: int) -> None:
    """Append X gates that turn |0...0> into the basis state |x>."""
    for q in range(c.n):
        if (x >> q) & 1:
            c.add("X", q)


def qft_circuit(n: int, x: int | None = None) -> Circuit:
    """QFT on n qubits (optionally preceded by X gates preparing |x>).

    For j = n-1 down to 0: H on j, then CP(k, j, pi / 2^(j-k)) for k = j-1 down
    to 0; finally SWAP(j, n-1-j).  With qubit 0 the least significant bit this
    maps |x> to 2^{-n/2} sum_y exp(2 pi i x y / 2^n) |y>.
    """
    c = Circuit(n)
    if x is not None:
        basis_prep(c, x)
    for j in range(n - 1, -1, -1):
        c.add("H", j)
        for k in range(j - 1, -1, -1):
            c.add("CP", k, j, params=(math.pi / (1 << (j - k)),))
    for j in range(n // 2):
        c.add("SWAP", j, n - 1 - j)
    return c


# Six CZ edge patterns of a rows x cols grid, qubit index q = cols*r + c.
GRID_PATTERNS = "ABCDEF"


def grid_edges(rows: int, cols: int, pattern: str) -> list[tuple[int, int]]:
    """Edges of one CZ pattern: A/B horizontal (c even/odd), C..F vertical
    (C: r even c even, D: r even c odd, E: r odd c even, F: r odd c odd)."""
    edges = []
    if pattern in "AB":
        par = 0 if pattern == "A" else 1
        for r in range(rows):
            for col in range(par, cols - 1, 2):
                edges.append((cols * r + col, cols * r + col + 1))
    else:
        rpar, cpar = {"C": (0, 0), "D": (0, 1), "E": (1, 0), "F": (1, 1)}[pattern]
        for r in range(rpar, rows - 1, 2):
            for col in range(cpar, cols, 2):
                edges.append((cols * r + col, cols * (r + 1) + col))
    return edges


def grid_circuit(rows: int, cols: int, depth: int, seed: int) -> Circuit:
    """Grid circuit: {SX,SY,T} on every qubit, then the CZ pattern
    GRID_PATTERNS[layer % 6] (sequence A B C D E F A B ...)."""
    n = rows * cols
    c = Circuit(n)
    draws = _rng(seed).integers(0, len(GRID_1Q), size=(depth, n))
    for layer in range(depth):
        for q in range(n):
            c.add(GRID_1Q[int(draws[layer, q])], q)
        for a, b in grid_edges(rows, cols, GRID_PATTERNS[layer % 6]):
            c.add("CZ", a, b)
    return c


def grid_partition_mask(rows: int, cols: int, rows_a: int) -> int:
    """Bit mask of the qubits in rows 0..rows_a-1 (partition A)."""
    return (1 << (rows_a * cols)) - 1


def inverse_circuit(c: Circuit) -> Circuit:
    """Adjoint circuit: gates in reverse order, each replaced by its inverse."""
    inv = Circuit(c.n)
    for name, qs, ps in reversed(c.gates):
        if name in ("CP", "P"):
            inv.add(name, *qs, params=(-ps[0],))
        elif name == "U":
            u = ps  # (u00r,u00i,u01r,u01i,u10r,u10i,u11r,u11i); adjoint = conj transpose
            inv.add("U", *qs, params=(u[0], -u[1], u[4], -u[5], u[2], -u[3], u[6], -u[7]))
        else:
            inv.add(ADJOINT[name], *qs)
    return inv


def concat(a: Circuit, b: Circuit) -> Circuit:
    if a.n != b.n:
        raise ValueError("qubit counts differ")
    c = Circuit(a.n)
    c.gates = list(a.gates) + list(b.gates)
    return c


def random_unitary_gates(n: int, count: int, seed: int) -> Circuit:
    """A circuit of every gate kind in the format, on random qubits, with
    random parameters (used for brute-force checks).  The 'U' gates carry
    random complex 2x2 matrices made unitary by a QR step in numpy."""
    rng = _rng(seed)
    c = Circuit(n)
    kinds = list(ONE_QUBIT) + ["P", "U", "CZ", "CX", "CP", "SWAP"]
    for _ in range(count):
        k = kinds[int(rng.integers(0, len(kinds)))]
        if k in ONE_QUBIT:
            c.add(k, int(rng.integers(0, n)))
        elif k == "P":
            c.add("P", int(rng.integers(0, n)), params=(float(rng.uniform(-math.pi, math.pi)),))
        elif k == "U":
            z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
            qm, rm = np.linalg.qr(z)
            qm = qm * (np.diag(rm) / np.abs(np.diag(rm)))
            ps = []
            for i in range(2):
                for j in range(2):
                    ps += [float(qm[i, j].real), float(qm[i, j].imag)]
            c.add("U", int(rng.integers(0, n)), params=tuple(ps))
        else:
            if n < 2:
                continue
            a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
            if k == "CP":
                c.add("CP", a, b, params=(float(rng.uniform(-math.pi, math.pi)),))
            else:
                c.add(k, a, b)
    return c


def random_bitstrings(m: int, nbits: int, seed: int) -> np.ndarray:
    """m uniform nbits-bit integers (uint64) from PCG64(seed)."""
    rng = _rng(seed)
    hi = rng.integers(0, 1 << 32, size=m, dtype=np.uint64)
    lo = rng.integers(0, 1 << 32, size=m, dtype=np.uint64)
    v = (hi << np.uint64(32)) | lo
    if nbits < 64:
        v &= np.uint64((1 << nbits) - 1)
    return v


def random_state(n: int, seed: int) -> np.ndarray:
    """A normalised random complex128 state of 2^n amplitudes."""
    rng = _rng(seed)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)
