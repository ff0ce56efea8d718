"""sv_amplitudes_noalloc: the amplitude gather for callers that cannot call
cudaMalloc (and so cannot create a handle, whose scratch is cudaMalloc'ed).
Its scratch is a fixed device array inside the library; it must return what
the handle-based sv_amplitudes returns, call after call.  This file is
collected last so that a stop-at-first-failure run has run everything else."""

import numpy as np
import pytest

from paper_1912_03243_gb300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03243_gb300 import build, sv

    build.build()
    sv.lib()
    return sv


@pytest.mark.parametrize("dtype,n", [("c64", 20), ("c128", 18), ("enc2b", 16), ("c64", 5), ("enc2b", 6)])
def test_matches_handle_gather_twice(S, dtype, n):
    st = S.StateVector(n, dtype)
    st.run(C.random_circuit(n, 6, 3), "pergate")
    st.sync()
    rng = np.random.default_rng(n)
    for call in range(2):  # two calls in a row share the same scratch array
        m = 4096 if call == 0 else 777
        idx = rng.integers(0, 1 << n, size=m, dtype=np.uint64)
        got = S.sv_amplitudes_noalloc(st.buffer.data_ptr(), n, dtype, idx, stream=st.stream.cuda_stream)
        ref = st.amplitudes(idx)
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref)) <= 1e-12


def test_rejects_more_than_the_maximum(S):
    st = S.StateVector(17, "c64")
    idx = np.zeros(65537, dtype=np.uint64)
    with pytest.raises(S.SVError) as e:
        S.sv_amplitudes_noalloc(st.buffer.data_ptr(), 17, "c64", idx)
    assert e.value.status == 1 and "at most 65536" in str(e.value)
    ok = S.sv_amplitudes_noalloc(st.buffer.data_ptr(), 17, "c64", idx[:65536])
    assert ok[0] == 1 and np.all(ok[1:] == 1)  # |0...0>: every index is 0
    with pytest.raises(S.SVError):
        S.sv_amplitudes_noalloc(st.buffer.data_ptr(), 17, "c64", np.array([1 << 17], dtype=np.uint64))


def _segment_end(torch, ptr: int) -> int:
    """End address of the cudaMalloc'ed segment of torch's allocator that
    holds ptr (the driver reports the extent of that segment, not of the
    tensor carved out of it)."""
    for seg in torch.cuda.memory_snapshot():
        if seg["address"] <= ptr < seg["address"] + seg["total_size"]:
            return seg["address"] + seg["total_size"]
    raise AssertionError("pointer not found in torch's segments")


@pytest.mark.parametrize("case", ["misaligned_c128", "misaligned_c64", "past_the_allocation", "host_memory"])
def test_rejects_bad_state_pointers_on_the_host(S, case):
    """A misaligned, host, or too-short state pointer is an argument error
    reported before any copy or launch, never a fault on the GPU."""
    import torch

    st = S.StateVector(12, "c128")
    idx = np.array([0, 5], dtype=np.uint64)
    base = st.buffer.data_ptr()
    host = np.zeros(1 << 13, dtype=np.complex128)
    ptr, n, dt, msg = {
        "misaligned_c128": (base + 8, 12, "c128", "aligned"),  # c128 reads 16-byte values
        "misaligned_c64": (base + 4, 12, "c64", "aligned"),  # c64 and codes: 8 bytes
        # a 12-qubit complex128 state (64 KiB) starting 1 KiB before the end of the allocation
        "past_the_allocation": (_segment_end(torch, base) - 1024, 12, "c128", "needs"),
        "host_memory": (host.ctypes.data, 12, "c128", "not device memory"),
    }[case]
    with pytest.raises(S.SVError) as e:
        S.sv_amplitudes_noalloc(ptr, n, dt, idx, stream=st.stream.cuda_stream)
    assert e.value.status == 1 and msg in str(e.value), str(e.value)
    # the context is intact: a valid call right after the rejected one
    got = S.sv_amplitudes_noalloc(base, 12, "c128", idx, stream=st.stream.cuda_stream)
    assert got[0] == 1 and got[1] == 0
    torch.cuda.synchronize()
