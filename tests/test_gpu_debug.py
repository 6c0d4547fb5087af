"""Debug checks on the GPU (they take compute-sanitizer's place for the
inputs, which is closed here): with a context's checks on, a clean evaluation
equals the unchecked one bit for bit, and an input residue that is not below
its prime -- in a ciphertext, a feature plaintext, an op's input -- makes the
call return BCN_E_INVAL before anything launches, leaving the output and the
status word untouched; nothing traps.  Without the checks the same input is
just evaluated."""
import numpy as np
import pytest
import torch

import workloads
from paper_2402_01296_gb300 import bcn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    cfg = workloads.with_batch(workloads.get_config("cnn3_small"), 64)
    ctx = bcn.Context.from_config(cfg)
    wq = [bcn.quantize(w) for w in workloads.cipher_weights(cfg)]
    model = bcn.Model(ctx, cfg["cipher"], [a for a, _ in wq], [s for _, s in wq])
    evk = ctx.evk_prepare(bcn.to_device(ctx.keygen(7)[1]))
    cts = workloads.random_residues(ctx.q, (model.n_in, 2), ctx.N, 11)
    pts = [workloads.random_residues(ctx.q[:s[1]], (s[0],), ctx.N, 12 + k) for k, s in enumerate(model.pt_shapes())]
    return ctx, model, evk, cts, pts


def _eval(model, evk, cts, pts):
    out = torch.zeros(model.out_shape(), dtype=torch.int32, device="cuda")
    model.eval(evk, bcn.to_device(cts), [bcn.to_device(p) for p in pts], out, model.alloc_workspace())
    return out


def test_clean_inputs_pass_and_match(setup):
    ctx, model, evk, cts, pts = setup
    ctx.set_debug(False)
    want = bcn.to_host_u32(_eval(model, evk, cts, pts))
    ctx.set_debug(True)
    try:
        assert ctx.debug()
        got = bcn.to_host_u32(_eval(model, evk, cts, pts))
    finally:
        ctx.set_debug(False)
    assert np.array_equal(got, want)
    assert ctx.device_status() == 0


def test_bad_residue_is_refused(setup):
    ctx, model, evk, cts, pts = setup
    bad = cts.copy()
    bad[3, 1, 1, 17] = ctx.q[1]  # equal to its prime
    badp = [p.copy() for p in pts]
    badp[0][2, 0, 5] = 0xFFFFFFFF
    ctx.set_debug(True)
    try:
        for c_, p_ in ((bad, pts), (cts, badp)):
            out = torch.zeros(model.out_shape(), dtype=torch.int32, device="cuda")
            with pytest.raises(bcn.BcnError, match="not below its prime"):
                model.eval(evk, bcn.to_device(c_), [bcn.to_device(p) for p in p_], out, model.alloc_workspace())
            torch.cuda.synchronize()
            assert int(out.abs().sum()) == 0  # nothing launched
            assert ctx.device_status() == 0  # the check's bit was cleared
        # a single operation too
        level = ctx.L
        x = workloads.random_residues(ctx.q, (2, 2), ctx.N, 3)
        x[1, 0, 0, 0] = ctx.q[0] + 5
        out = torch.zeros((2, 2, level - 1, ctx.N), dtype=torch.int32, device="cuda")
        with pytest.raises(bcn.BcnError, match="not below its prime"):
            ctx.op_square_relin_rescale(level, evk, bcn.to_device(x), 2, out)
    finally:
        ctx.set_debug(False)
    # without the checks the same input is simply evaluated (no fault either way)
    _eval(model, evk, bad, pts)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
