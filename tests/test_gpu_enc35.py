"""Two-byte code at its configured size, 35 qubits (64 GiB of codes, whose
16-byte chunk index reaches 2^32): one gate of each matrix shape on low,
block-boundary and top targets, checked bit-exact against the CPU codec
mirror on sampled blocks.

A gate on target t changes block b only together with block b ^ 2^(t-8)
(t >= 8) or alone (t < 8): each sample is that pair (or block) laid out as
a 9- (8-) qubit state, run through the mirror's gate, and compared code for
code and scale for scale with what the GPU wrote.  The input is a seeded
random encoded state written directly as codes and scales (every nonzero
block holds a code +-127, as an encoded state does; some blocks are zero).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N = 35
NB = 1 << (N - 8)     # 256-amplitude blocks
SAMPLES = 192


@pytest.fixture(scope="module")
def S():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03243_gb300 import build, sv

    build.build()
    sv.lib()
    need = sv.sv_bytes_required(N, "enc2b")
    if torch.cuda.mem_get_info()[0] < need + (4 << 30):
        pytest.skip("not enough device memory for a 35-qubit two-byte state")
    return sv


@pytest.fixture(scope="module")
def state(S):
    """A seeded random 35-qubit encoded state, written on the device."""
    import torch

    st = S.StateVector(N, "enc2b")
    g = torch.Generator(device=st.buffer.device)
    g.manual_seed(35)
    codes = st.buffer[: 2 << N].view(torch.int8)
    codes.random_(-127, 128, generator=g)
    blocks = codes.view(NB, 512)
    blocks[:, 0] = 127                     # block maximum: decode-encode is the identity
    scales = st.buffer[2 << N:].view(torch.float32)
    scales.uniform_(1.0, 4.0, generator=g)
    scales.mul_(2.0 ** -17)
    zero = torch.randint(0, NB, (NB // 64,), device=st.buffer.device, generator=g)
    blocks.index_fill_(0, zero, 0)
    scales.index_fill_(0, zero, 0.0)
    torch.cuda.synchronize()
    yield st
    st.free()
    del st
    torch.cuda.empty_cache()


def read_blocks(st, idx):
    """Codes (k, 512) and scales (k,) of blocks idx, copied to the host."""
    import torch

    t = torch.as_tensor(idx, dtype=torch.int64, device=st.buffer.device)
    codes = st.buffer[: 2 << N].view(torch.int8).view(NB, 512).index_select(0, t)
    scales = st.buffer[2 << N:].view(torch.float32).index_select(0, t)
    return codes.cpu().numpy(), scales.cpu().numpy()


def gate_cases():
    rng = np.random.default_rng(8)
    z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    u = np.linalg.qr(z)[0]
    z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    cu = np.linalg.qr(z)[0]
    cases = []
    for t in (0, 7, 8, 31, 32, 34):
        cases += [("H", t, -1, None), ("SX", t, -1, None), ("T", t, -1, None), ("U", t, -1, u)]
        # controlled general gate: an in-block control for block-level targets,
        # a block-level control for in-block targets
        cases.append(("CU", t, 3 if t >= 8 else 20 + t, cu))
    cases.append(("CU", 8, 33, cu))
    return cases


def sample_low_blocks(rng, t):
    """Blocks b with bit t-8 clear (t >= 8), or any blocks (t < 8); always the
    first and last ones among them."""
    b = rng.integers(0, NB, size=SAMPLES, dtype=np.int64)
    extra = np.array([0, NB - 1, NB // 2, NB // 2 - 1], dtype=np.int64)
    b = np.concatenate([b, extra])
    if t >= 8:
        b &= ~np.int64(1 << (t - 8))
    return np.unique(b)


def test_one_gate_of_each_shape_bit_exact(S, orc, state):
    rng = np.random.default_rng(35)
    for name, t, c, u in gate_cases():
        m = u if u is not None else orc.gate_matrix(name)
        lo = sample_low_blocks(rng, t)
        hi = lo | (1 << (t - 8)) if t >= 8 else None
        idx = np.concatenate([lo, hi]) if hi is not None else lo
        c0, s0 = read_blocks(state, idx)
        state.apply_gate(t, m, control=c)
        c1, s1 = read_blocks(state, idx)
        k = lo.size
        for j in range(k):
            b = int(lo[j])
            if t >= 8:
                sub_c = np.concatenate([c0[j], c0[k + j]])
                sub_s = np.array([s0[j], s0[k + j]], dtype=np.float32)
                got_c = np.concatenate([c1[j], c1[k + j]])
                got_s = np.array([s1[j], s1[k + j]], dtype=np.float32)
                sub_t = 8
            else:
                sub_c, sub_s, got_c, got_s, sub_t = c0[j], s0[j:j + 1], c1[j], s1[j:j + 1], t
            if c >= 8:  # a block-level control: the gate acts on the whole sample or not at all
                active = (b >> (c - 8)) & 1
                sub_ctl = -1
            else:
                active, sub_ctl = 1, c
            if active:
                want_c, want_s = orc.enc_apply_gate(sub_c, sub_s, sub_t, sub_ctl, m)
            else:
                want_c, want_s = sub_c, sub_s
            assert np.array_equal(got_c, want_c), (name, t, c, b)
            assert np.array_equal(got_s.view(np.uint32), want_s.view(np.uint32)), (name, t, c, b)
