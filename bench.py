"""Benchmark: encrypted inferences/s of the bi-CryptoNets ciphertext branch.

A step is one ciphertext-branch evaluation (every layer: integer-weight MAC,
unidirectional feature add, square = tensor square + relinearisation +
rescale) over one slot batch of the CryptoNets-scale workload: 4096 MNIST-
shaped images, a 16x16 sensitive segment (256 ciphertexts), N = 8192, 7 data
primes + 1 special prime, conv 5x5/2 -> add -> square -> dense 100 -> add ->
square -> dense 10.  Inputs are seeded synthetic data made by the library's own
client calls.  Replicas only across GPUs: every rank evaluates its own batch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead (a bounded number of whole evaluations).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import pathlib
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = pathlib.Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

import workloads  # noqa: E402

METRIC = "encrypted inferences/s + p50/p99 latency; NTT/keyswitch HBM GB/s vs peak"
UNIT = "encrypted inferences/s"
WORKLOAD = "cryptonets"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=list(workloads.CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget-s", type=float, default=150.0, help="wall budget of the reference arm")
    return ap.parse_args()


def config_desc(cfg):
    return {
        "workload": f"{cfg['name']}: {cfg['batch']} images/slot batch, segment {cfg['segment'][2]}x{cfg['segment'][3]}"
                    f"x{cfg['image'][2]} ({workloads.n_input_cts(cfg)} ciphertexts), N={1 << cfg['log_n']}, "
                    f"{cfg['n_data']}+{cfg['n_special']} primes, alpha={cfg['alpha']}",
        "layers": " -> ".join(
            (f"conv{l['k']}x{l['k']}/{l['stride']}x{l['cout']}" if l["type"] == "conv" else f"dense{l['n_out']}")
            + ("+add" if l["add"] else "") + ("+square" if l["square"] else "") for l in cfg["cipher"]),
        "images_per_step": cfg["batch"],
    }


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def csrc_hash():
    h = hashlib.sha256()
    for f in sorted((ROOT / "paper_2402_01296_gb300" / "csrc").glob("*")):
        h.update(f.name.encode())
        h.update(f.read_bytes())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from a committed ncu summary, if it was
    taken on the current sources; else None."""
    p = ROOT / "profiles" / "ncu_traffic.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text())
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("csrc_hash") != csrc_hash():
        return None
    return e.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# the oracle (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_problem(cfg):
    from oracle import oracle as O

    return O, O.Problem(cfg)


def oracle_time(cfg, max_evals: int, budget_s: float):
    O, prob = oracle_problem(cfg)
    times = []
    t_start = time.perf_counter()
    for _ in range(max_evals):
        t0 = time.perf_counter()
        prob.evaluate()
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s:
            break
    return times, O.max_threads()


def run_reference(args, cfg, rank, world):
    if rank != 0:
        return
    W = min(args.warmup, 1)
    K = max(1, args.steps)
    O, prob = oracle_problem(cfg)
    for _ in range(W):
        prob.evaluate()
    times = []
    t_start = time.perf_counter()
    for _ in range(K):
        t0 = time.perf_counter()
        prob.evaluate()
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > args.ref_budget_s:
            break
    mean = statistics.mean(times)
    value = cfg["batch"] / mean
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": len(times),
        "warmup": W, "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic", "config": config_desc(cfg),
        "p50_ms": statistics.median(times) * 1e3, "p99_ms": float(np.percentile(times, 99)) * 1e3,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                         "sample": f"{len(times)} whole evaluations of the workload (of {K} requested; wall budget "
                                   f"{args.ref_budget_s:.0f} s), inputs prepared outside the timed region"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def build_inputs(bcn, torch, cfg, device):
    """Client side with the library: keys, encrypted segment, plaintext-branch
    features (GPU, fp32) and their encodings; then the evaluator's model."""
    B = cfg["batch"]
    ctx = bcn.Context.from_config(cfg, device=device)
    w_q = [bcn.quantize(w) for w in workloads.cipher_weights(cfg)]
    model = bcn.Model(ctx, cfg["cipher"], [a for a, _ in w_q], [s for _, s in w_q])
    scale0 = 2.0 ** cfg["log_scale"]
    adds, out_scale = model.scales(scale0)
    imgs, noise = workloads.images(cfg), workloads.laplace_noise(cfg)
    pm = bcn.PlainModel(ctx, cfg["plain"], workloads.plain_weights(cfg), cfg["image"], cfg["segment"])
    feats = torch.empty((pm.n_feat, B), dtype=torch.float32, device=device)
    ws_p = torch.empty(pm.workspace_bytes(B) // 4 + 1, dtype=torch.int32, device=device)
    pm.forward(torch.from_numpy(imgs).to(device), torch.from_numpy(noise).to(device), feats, ws_p)
    f = feats.cpu().numpy().astype(np.float64)
    sizes = [model.n_outs[i] for i in model.add_layers]
    f_split = np.split(f, np.cumsum(sizes)[:-1]) if sizes else []
    pts = [ctx.encode(fv, model.levels[i], sc) for fv, i, sc in zip(f_split, model.add_layers, adds)]
    sk, evk = ctx.keygen(workloads.SEED_KEYS)
    cts = ctx.encrypt_segment(sk, imgs, cfg["segment"], scale0, workloads.SEED_ENC)
    return ctx, model, sk, evk, cts, pts, out_scale


def run_ours(args, cfg, rank, world, local_rank):
    import torch

    from paper_2402_01296_gb300 import bcn

    device = local_rank
    torch.cuda.set_device(device)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl", device_id=torch.device("cuda", device))

    ctx, model, sk, evk, cts, pts, out_scale = build_inputs(bcn, torch, cfg, device)
    dev = f"cuda:{device}"
    evk_eval = ctx.evk_prepare(bcn.to_device(evk, dev))
    cts_d = bcn.to_device(cts, dev)
    pts_d = [bcn.to_device(p, dev) for p in pts]
    out = torch.empty(model.out_shape(), dtype=torch.int32, device=dev)
    ws = model.alloc_workspace()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2: evicts it between steps
    stream = torch.cuda.current_stream()

    # correctness gate on this very run: decrypted logits are finite and sensible
    model.eval(evk_eval, cts_d, pts_d, out, ws)
    torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        model.eval(evk_eval, cts_d, pts_d, out, ws)
    torch.cuda.synchronize()

    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(device)
    model.profile_enable(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(K):
        flush.zero_()
        starts[i].record(stream)
        model.eval(evk_eval, cts_d, pts_d, out, ws)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    prof = model.profile_read()
    model.profile_enable(False)
    mean_ms = statistics.mean(step_ms)
    if dist:
        t = torch.tensor([mean_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        mean_ms = float(t.item())

    # decrypt once to make sure the timed result is the real one
    res = bcn.to_host_u32(out)
    dec = ctx.decrypt_decode(sk, res, model.out_level, out_scale, cfg["batch"])
    sane = bool(np.all(np.isfinite(dec)) and np.abs(dec).max() < 1e3)

    # end to end through the C ABI with host buffers (pinned), copies included
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory()  # noqa: E731
    cts_h = pin(cts)
    pts_h = [pin(p) for p in pts]
    out_h = torch.empty(model.out_shape(), dtype=torch.int32).pin_memory()
    as_u32 = lambda t: t.numpy().view(np.uint32)  # noqa: E731
    ws_h = model.alloc_workspace(host=True)
    model.eval_host(evk_eval, as_u32(cts_h), [as_u32(p) for p in pts_h], as_u32(out_h), ws_h)
    e2e_s = []
    for i in range(K):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        model.eval_host(evk_eval, as_u32(cts_h), [as_u32(p) for p in pts_h], as_u32(out_h), ws_h)
        e2e_s.append(time.perf_counter() - t0)
    e2e_mean = statistics.mean(e2e_s)
    if dist:
        t = torch.tensor([e2e_mean], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_mean = float(t.item())
    assert np.array_equal(as_u32(out_h), res), "host-buffer evaluation differs from the device evaluation"
    h2d = cts.nbytes + sum(p.nbytes for p in pts)
    d2h = out_h.numel() * 4

    B = cfg["batch"]
    value = world * B / (mean_ms / 1e3)
    launches = sum(v[1] for v in prof.values())
    # roofline of the dominant kernel (largest device time)
    dom = max(prof, key=lambda k: prof[k][0])
    dms, dn, dbytes = prof[dom]
    achieved = (dbytes / dn) / (dms / dn / 1e3) / 1e9 if dn else 0.0
    peak, peak_src = measured_peaks()
    traffic = ncu_traffic(dom, cfg["name"])
    kernels = {k: {"launches": n, "ms_total": ms, "ms_per_step": ms / K, "share": ms / max(1e-9, sum(
        v[0] for v in prof.values())), "algorithmic_GBps": (b / (ms / 1e3) / 1e9) if ms else None}
               for k, (ms, n, b) in prof.items()}
    ks_ms = sum(prof[k][0] for k in ("keyswitch", "moddown_rescale"))
    ks_b = sum(prof[k][2] for k in ("keyswitch", "moddown_rescale"))
    ntt_ms = prof["square"][0]
    ntt_b = prof["square"][2]

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        times, cores = oracle_time(cfg, max_evals=3, budget_s=30.0)
        cpu = {"value": B / statistics.mean(times), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{len(times)} whole evaluation(s) of the same workload ({B} images each) by the C oracle "
                         f"with OpenMP over ciphertexts; inputs prepared outside the timing"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": max(3, args.warmup),
        "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": {**config_desc(cfg), "parallelism": f"replicas x{world}",
                                        "l2": "flushed (512 MiB write) between timed steps, outside the events"},
        "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
        "e2e": {"value": world * B / e2e_mean, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_mean * 1e3},
        "gpu_launches": int(launches),
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src},
        "ntt_GBps": ntt_b / (ntt_ms / 1e3) / 1e9 if ntt_ms else None,
        "keyswitch_GBps": ks_b / (ks_ms / 1e3) / 1e9 if ks_ms else None,
        "kernels": kernels,
        "cpu_baseline": cpu,
        "clocks": clk,
        "decrypt_sane": sane,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    cfg = workloads.get_config(args.workload)
    if args.impl == "reference":
        run_reference(args, cfg, rank, world)
    else:
        run_ours(args, cfg, rank, world, local_rank)


if __name__ == "__main__":
    main()
