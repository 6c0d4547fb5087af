"""Autotuner for the batched evaluation: measures candidates on the device and
keeps the fastest.

Knobs:
  * lanes      -- streams the batch's evaluations are spread over (bcn_batch);
  * chunk      -- ciphertexts per key-switching chunk of a model
                  (bcn_model_set_chunk; the workspace follows);
  * alpha      -- primes per key-switching digit (a parameter of the context and
                  of its evaluation key), where K > 1 allows a choice;
  * NTT shape  -- residues per thread of the NTT-based kernels of a context
                  (bcn_ctx_set_ntt_shape: the default or the alternative block
                  shape, N >= 4096).
Every candidate computes the same residues; only the time differs.  Timing is
CUDA events on the launching stream, after a warm-up launch.
"""
from __future__ import annotations

import torch

from . import bcn


def _time(fn, reps: int = 2) -> float:
    fn()  # warm-up (and first-touch of the workspace)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def tune_lanes(items, candidates=(1, 2, 4, 8), budget_bytes: int | None = None, reps: int = 2):
    """Fastest lane count whose workspace fits `budget_bytes`.  Returns
    (lanes, ms, {lanes: ms})."""
    results = {}
    for lanes in candidates:
        if lanes > len(items):
            continue
        need = bcn.Batch.plan_items(items, lanes)
        if budget_bytes is not None and need > budget_bytes:
            continue
        b = bcn.Batch(items, lanes)
        results[lanes] = _time(b.launch, reps)
        b.close()
        del b
        torch.cuda.empty_cache()
    best = min(results, key=results.get)
    return best, results[best], results


def tune_chunk(model, evk_eval, cts, pts, out, candidates=(0, 256, 128, 64)):
    """Fastest key-switching chunk for one model (0 = the library's default).
    Leaves the model set to the winner.  Returns (chunk, ms, {chunk: ms})."""
    results = {}
    for ch in candidates:
        model.set_chunk(ch)
        ws = model.alloc_workspace()
        results[ch] = _time(lambda: model.eval(evk_eval, cts, pts, out, ws))
        del ws
    best = min(results, key=results.get)
    model.set_chunk(best)
    return best, results[best], results


def tune_alpha(make_eval, alphas):
    """Fastest digit size: make_eval(alpha) returns a zero-argument callable
    evaluating one representative model with a context and key of that alpha.
    Returns (alpha, ms, {alpha: ms})."""
    results = {a: _time(make_eval(a)) for a in alphas}
    best = min(results, key=results.get)
    return best, results[best], results


def tune_ntt_shape(ctx, run, shapes=(0, 1)):
    """Fastest block shape of the context's NTT-based kernels: run() is a
    zero-argument callable evaluating a representative model on the context.
    Leaves the context set to the winner.  Returns (shape, ms, {shape: ms})."""
    if ctx.N < 4096:
        return 0, _time(run), {0: _time(run)}
    results = {}
    for sh in shapes:
        ctx.set_ntt_shape(sh)
        results[sh] = _time(run)
    best = min(results, key=results.get)
    ctx.set_ntt_shape(best)
    return best, results[best], results
