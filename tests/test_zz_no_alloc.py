"""The allocation-free square activation (bcn_op_square_relin_rescale_noalloc)
against the workspace-based entry point (bcn_op_square_relin_rescale).

The allocation-free call serves callers that may not allocate device memory
themselves (budgeted serving processes, code under a framework allocator): its
key-switching intermediates sit in the library's fixed 32 MiB device array.
Both calls go through the C ABI; results must be identical residue by residue
(the tolerance of every ciphertext test here), on two calls in a row with
different inputs, one of them larger than a single chunk of the fixed array.
This file is collected last so a stop-at-first-failure run has already run
every other test.
"""
import numpy as np
import pytest
import torch

import workloads
from paper_2402_01296_gb300 import bcn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("params,n_cts", [((13, 7, 1, 1), (30, 5)), ((14, 11, 2, 2), (3, 9))])
def test_noalloc_square_matches_workspace_entry_point(params, n_cts):
    ctx = bcn.Context(*params, device=0)
    _, evk = ctx.keygen(workloads.SEED_KEYS)
    evk_eval = ctx.evk_prepare(bcn.to_device(evk))
    level = ctx.L
    xs, wants, gots = [], [], []
    for call, n_ct in enumerate(n_cts):  # every buffer of both calls, allocated up front
        xs.append(bcn.to_device(workloads.random_residues(ctx.q, (n_ct, 2), ctx.N, 100 + call)))
        wants.append(torch.empty((n_ct, 2, level - 1, ctx.N), dtype=torch.int32, device="cuda"))
        gots.append(torch.full_like(wants[-1], -1))
        ctx.op_square_relin_rescale(level, evk_eval, xs[-1], n_ct, wants[-1])
    torch.cuda.synchronize()
    # warm-up call: the one-time lookup of the array's device address happens here
    warm = torch.empty_like(gots[0])
    ctx.op_square_relin_rescale_noalloc(level, evk_eval, xs[0], n_cts[0], warm)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for call, n_ct in enumerate(n_cts):  # two calls in a row share the fixed array
        ctx.op_square_relin_rescale_noalloc(level, evk_eval, xs[call], n_ct, gots[call])
        torch.cuda.synchronize()
        # the call allocated no device memory (the device's free bytes did not move)
        assert torch.cuda.mem_get_info()[0] == free_before
        assert np.array_equal(bcn.to_host_u32(gots[call]), bcn.to_host_u32(wants[call]))
    assert ctx.device_status() == 0
