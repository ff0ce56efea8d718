"""Guard words around every state (the stand-in for a memory checker, which
is not available here): a state is attached inside a larger buffer whose
bytes before and after it hold a known pattern; after gates, circuits in
every mode, the two-byte code, expectation values and read-outs, the pattern
must be intact, i.e. no kernel wrote outside the state it was given."""

import ctypes

import numpy as np
import pytest

from paper_1912_03243_gb300 import circuits as C

pytestmark = pytest.mark.gpu

GUARD = 1 << 16  # bytes on each side (a multiple of 256: the state stays aligned)


@pytest.fixture(scope="module")
def S():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03243_gb300 import build, sv

    build.build()
    sv.lib()
    return sv


class Guarded:
    """A handle attached to the middle of a buffer with guard bytes around it."""

    def __init__(self, S, n, dtype):
        import torch

        self.S, self.n, self.dtype = S, n, dtype
        self.nbytes = S.sv_bytes_required(n, dtype)
        self.buf = torch.empty(self.nbytes + 2 * GUARD, dtype=torch.uint8, device="cuda")
        g = torch.Generator(device="cuda")
        g.manual_seed(n)
        self.buf.random_(0, 256, generator=g)
        self.before = self.buf[:GUARD].clone()
        self.after = self.buf[GUARD + self.nbytes:].clone()
        self.stream = torch.cuda.current_stream()
        self.handle = S._vp()
        S._check(S.lib().sv_attach(n, S.DTYPES[dtype], S._vp(self.buf.data_ptr() + GUARD), self.nbytes,
                                   S._vp(self.stream.cuda_stream), ctypes.byref(self.handle)), "sv_attach")
        S._check(S.lib().sv_set_basis(self.handle, 0), "sv_set_basis")

    def intact(self):
        import torch

        torch.cuda.synchronize()
        return bool(torch.equal(self.buf[:GUARD], self.before)) and bool(
            torch.equal(self.buf[GUARD + self.nbytes:], self.after))

    def free(self):
        self.S._check(self.S.lib().sv_free(self.handle), "sv_free")


@pytest.mark.parametrize("dtype,n", [("c64", 13), ("c64", 17), ("c128", 12), ("c128", 15), ("c64", 9)])
def test_modes_stay_inside_the_state(S, dtype, n):
    g = Guarded(S, n, dtype)
    c = C.random_circuit(n, 6, n)
    for mode in ("pergate", "tiled", "fused", "auto"):
        S._check(S.lib().sv_run_circuit(g.handle, c.text().encode(), S.MODES[mode]), mode)
        assert g.intact(), mode
    u = np.linalg.qr(np.random.default_rng(n).normal(size=(8, 8)) + 0j)[0]
    qs = np.array([0, n // 2, n - 1], dtype=np.int32)
    S._check(S.lib().sv_apply_fused(g.handle, 3, qs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                    u.astype(np.complex128).view(np.float64).ctypes.data_as(S._dp)), "fused")
    out = np.zeros(3 * n)
    S._check(S.lib().sv_expect_pauli(g.handle, out.ctypes.data_as(S._dp)), "expect")
    nrm = ctypes.c_double()
    S._check(S.lib().sv_norm(g.handle, ctypes.byref(nrm)), "norm")
    idx = np.array([0, (1 << n) - 1], dtype=np.uint64)
    amps = np.zeros(4)
    S._check(S.lib().sv_amplitudes(g.handle, 2, idx.ctypes.data_as(S._u64p), amps.ctypes.data_as(S._dp)), "amps")
    assert g.intact()
    g.free()


@pytest.mark.parametrize("n", [6, 9, 14])
def test_two_byte_code_stays_inside_the_state(S, n):
    g = Guarded(S, n, "enc2b")
    c = C.random_circuit(n, 6, 30 + n)
    S._check(S.lib().sv_run_circuit(g.handle, c.text().encode(), S.MODES["pergate"]), "enc2b")
    out = np.zeros(3 * n)
    S._check(S.lib().sv_expect_pauli(g.handle, out.ctypes.data_as(S._dp)), "expect")
    assert g.intact()
    g.free()


def test_batch_members_stay_inside_their_states(S):
    gs = [Guarded(S, n, "c64") for n in (12, 13, 16)]
    texts = [C.random_circuit(g.n, 5, g.n).text().encode() for g in gs]
    hs = (S._vp * 3)(*[g.handle for g in gs])
    ts = (ctypes.c_char_p * 3)(*texts)
    S._check(S.lib().sv_run_batch(hs, ts, 3), "batch")
    assert all(g.intact() for g in gs)
    for g in gs:
        g.free()
