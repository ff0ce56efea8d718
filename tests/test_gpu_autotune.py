"""The measurement-driven autotuner (SV_MODE_AUTO): every candidate strategy
is timed on a scratch state, the fastest is kept and remembered; the tuned
plan computes what the oracle computes, and the tuning leaves the handle's
own state untouched."""

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


@pytest.fixture
def fresh_tuning(monkeypatch, tmp_path):
    """Remembered choices go to a file of their own (nothing from earlier runs)."""
    monkeypatch.setenv("SV_JIT_CACHE", str(tmp_path / "cache"))


@pytest.mark.parametrize("n,dtype,tol", [(16, "c64", 1e-6), (14, "c128", 1e-12), (10, "c64", 1e-6)])
def test_tuned_plan_matches_the_oracle(S, orc, fresh_tuning, n, dtype, tol):
    c = C.random_circuit(n, 8, 40 + n)
    st = S.StateVector(n, dtype)
    st.set_basis(5)  # the tuning runs on a scratch state: this one must stay |5>
    plan = st.plan(c, "auto")
    rep = plan.tuning()
    assert rep["timed"] is True
    names = [x["strategy"] for x in rep["candidates"]]
    assert rep["chosen"] in names
    assert all(x["ms"] > 0 for x in rep["candidates"] if not x.get("failed"))
    best = min((x for x in rep["candidates"] if x["ms"] > 0), key=lambda x: x["ms"])
    chosen_ms = next(x["ms"] for x in rep["candidates"] if x["strategy"] == rep["chosen"])
    assert chosen_ms <= best["ms"] + 2e-6  # the fastest (ties within the report's rounding aside)
    if n >= 13:
        assert any(nm.startswith("tiled") for nm in names)
    assert any(nm.startswith("fused k=6") for nm in names)
    psi = st.to_numpy()
    assert psi[5] == 1 and np.count_nonzero(psi) == 1
    st.set_basis(0)
    plan.execute()
    got = st.to_numpy().astype(np.complex128)
    ref = orc.run(c)
    assert np.max(np.abs(got - ref)) <= tol
    plan.free()
    # a second plan of the same circuit takes the remembered choice without timing
    again = st.plan(c, "auto")
    rep2 = again.tuning()
    assert rep2["timed"] is False and rep2["remembered"] is True and rep2["chosen"] == rep["chosen"]
    again.free()


def test_tuned_two_byte_code_is_bit_exact(S, orc, fresh_tuning):
    n = 12
    c = C.random_circuit(n, 6, 9)
    enc = S.StateVector(n, "enc2b")
    plan = enc.plan(c, "auto")
    assert plan.tuning()["chosen"] == "pergate"
    enc.set_basis(0)
    plan.execute()
    gc, gs = enc.codes()
    rc, rs = orc.enc_run(c)
    assert np.array_equal(gc, rc) and np.array_equal(gs, rs)
    plan.free()
