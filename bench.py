"""Benchmark: encrypted inferences/s of the bi-CryptoNets ciphertext branch.

A step is one ciphertext-branch evaluation (every layer: integer-weight MAC,
unidirectional feature add, square = tensor square + relinearisation +
rescale) over one slot batch of the CIFAR-shaped workload: 8192 CIFAR-shaped
images, a 16x16x3 sensitive segment (768 ciphertexts), N = 16384, 11 data
primes + 2 special primes (alpha 2), conv 3x3 x16 -> add -> square -> conv
3x3/2 x32 -> add -> square -> dense 10.  Inputs are seeded synthetic data made
by the library's own client calls.  Replicas only across GPUs: every rank
evaluates its own batch.  --workload selects the smaller configurations and the
batched, serving and rotation workloads.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead (bounded samples of one evaluation, projected to the whole).
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
WORKLOAD = "cifar_cnn"


E2E_LANES = 2  # workspaces used in turn by the end-to-end measurement


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=list(workloads.CONFIGS) + ["cifar_profile", "uneven64", "serve", "rotate", "op_square",
                                                       "op_mac", "bhw"])
    ap.add_argument("--cts", type=int, default=384, help="op_square: ciphertexts")
    ap.add_argument("--map", type=int, default=8, help="op_mac: input map height and width")
    ap.add_argument("--groups", type=int, default=16, help="bhw: ciphertext groups of 16 images per step")
    ap.add_argument("--rates", default="50,100,200,500,1000,2000", help="serve: request rates (req/s)")
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="serve: seconds of arrivals per rate")
    ap.add_argument("--lanes", type=int, default=32, help="serve: batches in flight")
    ap.add_argument("--stacks", default="",
                    help="serve: stack sizes per model, e.g. 'cnn3_small:2,4,8;cryptonets:2' (requests of one "
                         "model sharing launches; measured no faster than captured per-request graphs here, so "
                         "off by default)")
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
        """Starts sampling and returns once the first sample is in: the
        sampler's start-up (NVML initialisation) stays out of the timed region,
        where it has been seen to stall the launching thread for tens of ms."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)

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


def replica_summary(mean_ms: float, images_per_rank: int, dist=None, device="cpu"):
    """Replicas only: every rank evaluated its own batch.  The job takes as long
    as the slowest rank, so the whole-job throughput is world * images / max ms.
    Returns (images/s, max ms)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch

        world = dist.get_world_size()
        t = torch.tensor([mean_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        mean_ms = float(t.item())
    return world * images_per_rank / (mean_ms / 1e3), mean_ms


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# Integer issue peak: every SM issues one warp instruction (32 lanes) per clock
# on each of its 4 schedulers, and its 128 lanes all run 32-bit integer
# multiply-adds, so 152 SMs x 128 lane-ops x the maximum SM clock.
GB300_SMS, INT_LANES_PER_SM = 152, 128
# Algorithmic 32-bit integer operations per unit of the NTT-based kernels: a
# butterfly (modular product by a precomputed twiddle with its quotient
# estimate, one addition and one subtraction, each with its conditional
# correction) counts 10, a modular multiply-add (product, reduction, addition)
# counts 5.
OPS_BUTTERFLY, OPS_MULADD = 10, 5


def int_peak_ops():
    p = ROOT / "MEASURED_PEAKS.json"
    mhz = json.loads(p.read_text()).get("sm_max_mhz", 2070.0) if p.exists() else 2070.0
    return GB300_SMS * INT_LANES_PER_SM * mhz * 1e6, mhz


def alu_work(cfg):
    """Integer work per evaluation of the NTT-based kernel classes:
    {"square" | "keyswitch" | "moddown_rescale": {"fwd": forward NTTs, "inv":
    inverse NTTs, "mont": N-element passes of products of two variables,
    "shoup": N-element passes of products by constants}} (every product a
    multiply-add).

    From the first square layer on, ciphertexts stay in the NTT domain.  Tensor
    square of a ciphertext at n limbs: per limb 2 forward NTTs (only on
    coefficient-form input, the first square layer) and 1 inverse NTT (d2 for
    ModUp); per coefficient the 3 products c0^2, c0 c1, c1^2 and the N^{-1}
    scaling of the inverse transform's input, and with digits of more than one
    prime the ModUp's constant product of d2 (done there once for the key
    switch's every target prime).  The square class also holds the
    domain changes: a forward NTT of every feature-plaintext limb that meets
    NTT-domain ciphertexts and the inverse NTT of the outputs.  Key switch of d2
    (hybrid, digits of at most alpha primes, n + K target primes): ModUp (one
    constant product per digit residue -- in the square kernel when alpha > 1 --
    then alpha per coefficient and prime outside the digit), a forward NTT of every digit in every target prime
    outside it (inside it, the tensor square's NTT form is reused), two products
    per digit and target prime with the key, then two inverse NTTs on each
    special prime and on the top data prime (with its 4 constant products
    folding in the rescale's first step) and a constant product by N on the
    other data primes.  ModDown and rescale: per poly, K + 1 constant products
    per coefficient for the top limb's correction (shared by every limb), then
    per data limb below the top K + 3 and one forward NTT (the conversion's
    first factor Phat_m^-1 rides in the prepared key)."""
    import math

    import workloads
    K, a = cfg["n_special"], cfg["alpha"]
    levels, _ = workloads.level_schedule(cfg)
    w = {k: {"fwd": 0, "inv": 0, "mont": 0, "shoup": 0} for k in ("square", "keyswitch", "moddown_rescale")}
    in_ntt = False
    for layer, n in zip(cfg["cipher"], levels):
        n_out = workloads.cipher_layer_io(layer)[1]
        if layer["add"] and in_ntt:
            w["square"]["fwd"] += n_out * n
        if not layer["square"]:
            continue
        C = n_out
        w["square"]["fwd"] += C * n * (0 if in_ntt else 2)
        w["square"]["inv"] += C * n
        w["square"]["mont"] += C * 3 * n
        # with multi-prime digits the square kernel also multiplies d2 by each
        # limb's ModUp factor Dhat^-1 (once, for every target prime of the key switch)
        pre = a >= 2
        w["square"]["shoup"] += C * n * (2 if pre else 1)
        digits = [min(a, n - j * a) for j in range(math.ceil(n / a))]
        nb = n + K
        w["keyswitch"]["fwd"] += C * sum(nb - d for d in digits)
        w["keyswitch"]["inv"] += C * 2 * (K + 1)
        w["keyswitch"]["mont"] += C * 2 * nb * len(digits)
        w["keyswitch"]["shoup"] += C * ((0 if pre else sum(digits)) + sum(d * (nb - d) for d in digits) + 2 * (n - 1) + 4)
        w["moddown_rescale"]["fwd"] += C * 2 * (n - 1)
        w["moddown_rescale"]["shoup"] += C * 2 * ((n - 1) * (K + 3) + K + 1)
        in_ntt = True
    last = cfg["cipher"][-1]
    if in_ntt:
        lout = levels[-1] - (1 if last["square"] else 0)
        w["square"]["inv"] += workloads.cipher_layer_io(last)[1] * 2 * lout
    return w


def alu_ops(cfg):
    """Algorithmic integer operations per evaluation of the NTT-based kernel
    classes (alu_work: 10 per butterfly, (N/2) log N butterflies per NTT, 5 per
    multiply-add, N per pass)."""
    N, logN = 1 << cfg["log_n"], cfg["log_n"]
    bf = (N // 2) * logN
    return {k: (v["fwd"] + v["inv"]) * bf * OPS_BUTTERFLY + (v["mont"] + v["shoup"]) * N * OPS_MULADD
            for k, v in alu_work(cfg).items()}


def alu_units(cfg):
    """The same work in the microbenchmark's units: {class: (forward
    butterflies, inverse butterflies, Montgomery multiply-adds, Shoup
    multiply-adds)} per evaluation."""
    N, logN = 1 << cfg["log_n"], cfg["log_n"]
    bf = (N // 2) * logN
    return {k: (v["fwd"] * bf, v["inv"] * bf, v["mont"] * N, v["shoup"] * N) for k, v in alu_work(cfg).items()}


def csrc_hash():
    h = hashlib.sha256()
    for f in sorted((ROOT / "paper_2402_01296_gb300" / "csrc").glob("*")):
        h.update(f.name.encode())
        h.update(f.read_bytes())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str, units_per_launch: float):
    """DRAM bytes per launch of `kernel` from a committed ncu capture taken on
    the current sources (else None): its bytes per unit of work (one block of
    the kernel) times the units of this run's average launch."""
    p = ROOT / "profiles" / "ncu_traffic.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text())
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("csrc_hash") != csrc_hash() or "dram_bytes_per_unit" not in e:
        return None
    return e["dram_bytes_per_unit"] * units_per_launch


def ks_units(cfg):
    """(target prime, ciphertext) blocks of the key-switching kernel per evaluation."""
    import workloads
    levels, _ = workloads.level_schedule(cfg)
    return sum(workloads.cipher_layer_io(l)[1] * (n + cfg["n_special"])
               for l, n in zip(cfg["cipher"], levels) if l["square"])


# ---------------------------------------------------------------------------
# the oracle (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_problem(cfg):
    from oracle import oracle as O

    return O, O.Problem(cfg)


class OracleSample:
    """A bounded sample of one evaluation by the oracle, projected to the whole
    evaluation: per cipher layer the MAC of a subset of its outputs (with only
    the input ciphertexts they read) and the square activation of a subset of
    its ciphertexts, each timed and scaled by the layer's output count.  The
    oracle's time does not depend on the residues' values, so the inputs are
    uniform residues of the right shapes.  `scale` shrinks every subset (the
    single-thread run)."""

    MAC_OUTPUTS, SQUARE_CTS, DENSE_OUTPUTS = 64, 64, 2

    def __init__(self, cfg, scale: float = 1.0, seed: int = 77):
        from oracle import oracle as O

        self.O, self.cfg = O, cfg
        self.P = O.Params.from_config(cfg)
        _, self.evk = self.P.keygen(workloads.SEED_KEYS)
        w_int = [O.quantize(w)[0] for w in workloads.cipher_weights(cfg)]
        self.levels, _ = workloads.level_schedule(cfg)
        self.parts = []  # (kind, level, n_total, args)
        rng_seed = seed
        for layer, wi, n in zip(cfg["cipher"], w_int, self.levels):
            idx, wt = O.layer_table(layer, wi)
            n_out = idx.shape[0]
            cap = self.MAC_OUTPUTS if layer["type"] == "conv" else self.DENSE_OUTPUTS
            s_mac = max(1, min(n_out, int(round(cap * scale))))
            # whole groups of outputs that read the same taps (a conv position's
            # channels, a dense layer), so that the sample reads few inputs
            _, first, inv = np.unique(idx, axis=0, return_index=True, return_inverse=True)
            inv = np.asarray(inv).reshape(-1)
            chosen = []
            for gr in np.argsort(first):
                chosen.extend(np.nonzero(inv == gr)[0].tolist())
                if len(chosen) >= s_mac:
                    break
            chosen = np.array(chosen[:s_mac])
            sel = idx[chosen]
            used = np.unique(sel[sel >= 0])
            remap = np.full(int(idx.max()) + 1 if idx.size else 1, -1, dtype=np.int32)
            remap[used] = np.arange(used.size, dtype=np.int32)
            sidx = np.where(sel >= 0, remap[np.maximum(sel, 0)], -1).astype(np.int32)
            x = workloads.random_residues(self.P.q[:n], (max(1, used.size), 2), self.P.N, rng_seed)
            rng_seed += 1
            pt = workloads.random_residues(self.P.q[:n], (s_mac,), self.P.N, rng_seed) if layer["add"] else None
            rng_seed += 1
            self.parts.append(("mac", n, n_out, (sidx, wt[chosen], x, pt)))
            if layer["square"]:
                s_sq = max(1, min(n_out, int(round(self.SQUARE_CTS * scale))))
                y = workloads.random_residues(self.P.q[:n], (s_sq, 2), self.P.N, rng_seed)
                rng_seed += 1
                self.parts.append(("square", n, n_out, (y,)))

    def describe(self):
        return "; ".join(
            f"{k} at {n} limbs: {a[0].shape[0]} of {tot}" for k, n, tot, a in self.parts)

    def run(self) -> float:
        """Seconds one whole evaluation would take (sum of the scaled parts)."""
        total = 0.0
        for kind, n, n_total, a in self.parts:
            t0 = time.perf_counter()
            if kind == "mac":
                self.P.mac(n, a[0], a[1], a[2], a[3])
            else:
                self.P.square_relin_rescale(n, self.evk, a[0])
            total += (time.perf_counter() - t0) * n_total / a[0].shape[0]
        return total


def oracle_time(cfg, max_samples: int, budget_s: float, single_thread: bool = False):
    """Projected seconds per whole evaluation by the oracle with OpenMP on every
    core (OracleSample, up to max_samples samples within budget_s); with
    single_thread, one more sample, 16x smaller, on one thread.  Returns
    (projected times, cores, single-thread projection or None, sample text)."""
    from oracle import oracle as O

    samp = OracleSample(cfg)
    times = []
    t_start = time.perf_counter()
    for _ in range(max_samples):
        times.append(samp.run())
        if time.perf_counter() - t_start > budget_s:
            break
    cores = O.max_threads()
    t1 = None
    if single_thread:
        small = OracleSample(cfg, scale=1.0 / 16)
        O.set_threads(1)
        try:
            t1 = small.run()
        finally:
            O.set_threads(cores)
    return times, cores, t1, samp.describe()


def run_reference(args, cfg, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O

    W = min(args.warmup, 1)
    K = max(1, args.steps)
    samp = OracleSample(cfg)
    for _ in range(W):
        samp.run()
    times = []
    t_start = time.perf_counter()
    for _ in range(K):
        times.append(samp.run())
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
                         "sample": f"{len(times)} steps (of {K} requested; wall budget {args.ref_budget_s:.0f} s), "
                                   f"each a timed sample of one evaluation projected to the whole by the layers' "
                                   f"output counts: {samp.describe()}; inputs prepared outside the timing"},
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
    # the same features as integer coefficients, for the compact upload (None
    # where a coefficient reaches 2^63)
    try:
        feats_i64 = [ctx.encode_i64(fv, sc) for fv, sc in zip(f_split, adds)]
    except bcn.BcnError:
        feats_i64 = None
    return ctx, model, sk, evk, cts, pts, out_scale, feats_i64


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

    ctx, model, sk, evk, cts, pts, out_scale, feats_i64 = build_inputs(bcn, torch, cfg, device)
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

    # integer-issue rates of this GPU (register-resident butterflies and
    # multiply-adds): the roofline of the NTT-based kernels, measured here
    from paper_2402_01296_gb300 import peak as peak_mod
    pclk = ClockSampler(device)
    pclk.start()
    rates = peak_mod.measure(device)
    peak_clocks = pclk.stop()

    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(device)
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
    value, mean_ms = replica_summary(statistics.mean(step_ms), cfg["batch"], dist, dev)
    # per-kernel split: the same steps again with the library's kernel timing on
    # (events around every launch; the square layers' chunk halves then run in
    # sequence on one stream, so this pass is a little slower than the timed one)
    model.profile_enable(True)
    for i in range(K):
        flush.zero_()
        model.eval(evk_eval, cts_d, pts_d, out, ws)
    torch.cuda.synchronize()
    prof = model.profile_read()
    model.profile_enable(False)

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
    assert np.array_equal(as_u32(out_h), res), "host-buffer evaluation differs from the device evaluation"
    # E2E_LANES workspaces and output buffers in turn on one stream: the
    # library copies a step's inputs as soon as its workspace's previous
    # evaluation is done, i.e. while the step before it computes.  Every step's
    # copies and its result read are inside the timed region.  Two forms of the
    # client's upload: seeded ciphertexts (c0 and the encryption seed; the
    # device draws c1 -- the headline e2e) and full ciphertexts.
    ws_h2 = [ws_h] + [model.alloc_workspace(host=True) for _ in range(E2E_LANES - 1)]
    outs_h = [out_h] + [torch.empty(model.out_shape(), dtype=torch.int32).pin_memory() for _ in range(E2E_LANES - 1)]
    # c0 of the same ciphertexts: bcn_encrypt_segment_seeded writes these words
    c0_h = pin(np.ascontiguousarray(cts[:, 0]))
    pts_u = [as_u32(p) for p in pts_h]

    def e2e_run(step):
        for i in range(E2E_LANES):  # warm every workspace
            step(i)
        torch.cuda.synchronize()
        flush.zero_()
        torch.cuda.synchronize()
        # an event after every step on the stream: the first interval holds the
        # pipeline fill (the first step's copies overlap nothing)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        t0 = time.perf_counter()
        ev[0].record()
        for i in range(K):
            step(i)
            ev[i + 1].record()
        torch.cuda.synchronize()
        total = time.perf_counter() - t0
        for o in outs_h:
            assert np.array_equal(as_u32(o), res), "host-buffer evaluation differs from the device evaluation"
        return total, [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]

    full_total, full_steps = e2e_run(lambda i: model.eval_host_async(
        evk_eval, as_u32(cts_h), pts_u, as_u32(outs_h[i % E2E_LANES]), ws_h2[i % E2E_LANES]))
    full_value, full_ms = replica_summary(full_total / K * 1e3, cfg["batch"], dist, dev)
    seed_total, seed_steps = e2e_run(lambda i: model.eval_host_seeded_async(
        evk_eval, as_u32(c0_h), workloads.SEED_ENC, pts_u, as_u32(outs_h[i % E2E_LANES]), ws_h2[i % E2E_LANES]))
    seed_value, seed_ms = replica_summary(seed_total / K * 1e3, cfg["batch"], dist, dev)
    h2d_seed = c0_h.numel() * 4 + sum(p.nbytes for p in pts)
    h2d_full = cts.nbytes + sum(p.nbytes for p in pts)
    if feats_i64 is not None:  # the headline upload: c0, the seed and the features' integer coefficients
        f64_h = [torch.from_numpy(np.ascontiguousarray(f)).pin_memory().numpy() for f in feats_i64]
        e2e_total, e2e_steps = e2e_run(lambda i: model.eval_host_compact_async(
            evk_eval, as_u32(c0_h), workloads.SEED_ENC, f64_h, as_u32(outs_h[i % E2E_LANES]), ws_h2[i % E2E_LANES]))
        e2e_value, e2e_ms = replica_summary(e2e_total / K * 1e3, cfg["batch"], dist, dev)
        h2d = c0_h.numel() * 4 + sum(f.nbytes for f in feats_i64)
        upload = ("seeded ciphertexts (c0 and the encryption seed, c1 drawn on the device) and the features' "
                  "integer coefficients (reduced mod each prime on the device)")
        e2e_path = "bcn_eval_host_compact_async"
    else:
        e2e_total, e2e_steps, e2e_value, e2e_ms, h2d = seed_total, seed_steps, seed_value, seed_ms, h2d_seed
        upload = "seeded ciphertexts (c0 and the encryption seed, c1 drawn on the device) and the encoded features"
        e2e_path = "bcn_eval_host_seeded_async"
    d2h = out_h.numel() * 4

    B = cfg["batch"]
    launches = sum(v[1] for v in prof.values())
    # roofline of the dominant kernel (largest device time).  The NTT-based
    # kernels are bound by integer issue, not HBM: they are reported against
    # the integer peak, the others against measured HBM bandwidth.
    dom = max(prof, key=lambda k: prof[k][0])
    dms, dn, dbytes = prof[dom]
    ops = alu_ops(cfg)
    units = alu_units(cfg)
    mix = {k: peak_mod.mix_peak(rates, *units[k]) for k in ops}
    traffic = ncu_traffic(dom, cfg["name"], ks_units(cfg) * K / dn) if dom == "keyswitch" and dn else None
    dpeak, mhz = int_peak_ops()
    if dom in ops:
        achieved = ops[dom] * K / (dms / 1e3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": mix[dom] / 1e12, "unit": "Tintop/s",
                "frac": achieved * 1e12 / mix[dom], "traffic": traffic,
                "traffic_source": "ncu dram bytes per block of this kernel (profiles/ncu_traffic.json) x blocks per "
                                  "launch of this run" if traffic else None,
                "peak_source": "measured in this run: register-resident rates of the evaluator's own lazy forward "
                               "and inverse butterflies, Montgomery and Shoup multiply-adds (bcn_int_peak_launch, "
                               "full occupancy), weighted by this kernel's mix of the four",
                "derived_peak": dpeak / 1e12,
                "derived_peak_source": f"{GB300_SMS} SMs x {INT_LANES_PER_SM} int32 lanes x {mhz:.0f} MHz",
                "ops_per_launch": ops[dom] * K / dn,
                "hbm_achieved_GBps": (dbytes / (dms / 1e3)) / 1e9, "hbm_peak_GBps": measured_peaks()[0]}
    else:
        peak, peak_src = measured_peaks()
        achieved = (dbytes / dn) / (dms / dn / 1e3) / 1e9 if dn else 0.0
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src}
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
        times, cores, t1, desc = oracle_time(cfg, max_samples=3, budget_s=30.0, single_thread=True)
        cpu = {"value": B / statistics.mean(times), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{len(times)} timed sample(s) of one evaluation of the same workload ({B} images) by the "
                         f"C oracle with OpenMP over outputs, each projected to the whole evaluation by the layers' "
                         f"output counts ({desc}); inputs prepared outside the timing",
               "single_thread": {"value": B / t1, "unit": UNIT, "cores": 1,
                                 "sample": "the same projection from a 16x smaller sample on one thread"}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": max(3, args.warmup),
        "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": {**config_desc(cfg), "parallelism": f"replicas x{world}",
                                        "l2": "flushed (512 MiB write) between timed steps, outside the events"},
        "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms,
                "first_step_ms": e2e_steps[0],
                "later_steps_ms": statistics.mean(e2e_steps[1:]) if K > 1 else None,
                "upload": upload,
                "pipelining": f"{e2e_path} with {E2E_LANES} workspaces in turn on one stream: a step's inputs "
                              "copy while the step before it computes",
                "seeded_ciphertexts": {"value": seed_value, "ms_per_step": seed_ms,
                                       "h2d_bytes_per_step": int(h2d_seed), "first_step_ms": seed_steps[0],
                                       "later_steps_ms": statistics.mean(seed_steps[1:]) if K > 1 else None,
                                       "path": "bcn_eval_host_seeded_async (features as residues)"},
                "full_ciphertexts": {"value": full_value, "ms_per_step": full_ms, "h2d_bytes_per_step": int(h2d_full),
                                     "first_step_ms": full_steps[0],
                                     "later_steps_ms": statistics.mean(full_steps[1:]) if K > 1 else None,
                                     "path": "bcn_eval_host_async on (c0, c1)"}},
        "gpu_launches": int(launches),
        "roofline": roof,
        "alu_frac": {k: ops[k] * K / (prof[k][0] / 1e3) / mix[k] for k in ops if prof[k][0]},
        "alu_frac_of_derived_peak": {k: ops[k] * K / (prof[k][0] / 1e3) / dpeak for k in ops if prof[k][0]},
        "int_peak": {"rates_per_s": {k: v["units_per_s"] for k, v in rates.items()},
                     "per_sm_per_clk": {k: v["units_per_s"] / GB300_SMS / (peak_clocks["sm_mhz"] * 1e6)
                                        for k, v in rates.items()} if peak_clocks.get("sm_mhz") else None,
                     "mix_peak_Tops": {k: v / 1e12 for k, v in mix.items()},
                     "clocks": peak_clocks,
                     "units": "instructions (imad_lo, imad_hi, imad_wide, dp4a), modular additions (modadd), butterflies "
                              "(butterfly_fwd, butterfly_inv), multiply-adds (mont_muladd, shoup_muladd)"},
        "ntt_GBps": ntt_b / (ntt_ms / 1e3) / 1e9 if ntt_ms else None,
        "keyswitch_GBps": ks_b / (ks_ms / 1e3) / 1e9 if ks_ms else None,
        "kernels": kernels,
        "kernel_timing": "CUDA events around every launch, on the launching stream, in a second pass of the same "
                         "steps (kernel timing makes the square layers' chunk halves run in sequence)",
        "cpu_baseline": cpu,
        "clocks": clk,
        "decrypt_sane": sane,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the batched uneven workload (64 evaluations, one graph)
# ---------------------------------------------------------------------------
def _dev_residues(torch, primes, lead, N, gen, device):
    """uniform residues [*lead][len(primes)][N] generated on the device"""
    t = torch.empty(tuple(lead) + (len(primes), N), dtype=torch.int32, device=device)
    for i, q in enumerate(primes):
        t[..., i, :] = torch.randint(0, int(q), tuple(lead) + (N,), generator=gen, device=device, dtype=torch.int32)
    return t


def run_uneven(args, rank, world, local_rank):
    import torch

    from paper_2402_01296_gb300 import bcn, tuner

    device = local_rank
    torch.cuda.set_device(device)
    dev = f"cuda:{device}"
    cfgs = workloads.uneven_batch(64)
    gen = torch.Generator(device=dev)
    gen.manual_seed(workloads.SEED_ENC + 1000 * rank)
    # contexts and keys per ring degree; alpha tuned where the chain allows a choice
    ctxs, evks, alpha_note = {}, {}, {}
    for cfg in cfgs:
        if cfg["log_n"] in ctxs:
            continue
        alphas = list(range(1, cfg["n_special"] + 1))
        best_alpha = cfg["alpha"]
        if len(alphas) > 1:
            probe = [c for c in cfgs if c["log_n"] == cfg["log_n"]][0]

            def make_eval(a, probe=probe):
                cx = bcn.Context(probe["log_n"], probe["n_data"], probe["n_special"], a, device)
                _, ek = cx.keygen(workloads.SEED_KEYS)
                ev = cx.evk_prepare(bcn.to_device(ek, dev))
                wq = [bcn.quantize(w) for w in workloads.cipher_weights(probe)]
                m = bcn.Model(cx, probe["cipher"], [x for x, _ in wq], [y for _, y in wq])
                c_ = _dev_residues(torch, cx.q, (m.n_in, 2), cx.N, gen, dev)
                p_ = [_dev_residues(torch, cx.q[:sh[1]], (sh[0],), cx.N, gen, dev) for sh in m.pt_shapes()]
                o_ = torch.empty(m.out_shape(), dtype=torch.int32, device=dev)
                ws_ = m.alloc_workspace()
                keep = (cx, ev, m, c_, p_, o_, ws_)
                return lambda: keep[2].eval(keep[1], keep[3], keep[4], keep[5], keep[6])

            best_alpha, _, res = tuner.tune_alpha(make_eval, alphas)
            alpha_note[cfg["log_n"]] = {str(a): round(v, 3) for a, v in res.items()}
            torch.cuda.empty_cache()
        cx = bcn.Context(cfg["log_n"], cfg["n_data"], cfg["n_special"], best_alpha, device)
        _, ek = cx.keygen(workloads.SEED_KEYS)
        ctxs[cfg["log_n"]] = cx
        evks[cfg["log_n"]] = cx.evk_prepare(bcn.to_device(ek, dev))
    items, images = [], 0
    for cfg in cfgs:
        cx = ctxs[cfg["log_n"]]
        wq = [bcn.quantize(w) for w in workloads.cipher_weights(cfg)]
        m = bcn.Model(cx, cfg["cipher"], [x for x, _ in wq], [y for _, y in wq])
        cts = _dev_residues(torch, cx.q, (m.n_in, 2), cx.N, gen, dev)
        pts = [_dev_residues(torch, cx.q[:sh[1]], (sh[0],), cx.N, gen, dev) for sh in m.pt_shapes()]
        out = torch.empty(m.out_shape(), dtype=torch.int32, device=dev)
        items.append((m, evks[cfg["log_n"]], cts, pts, out))
        images += cfg["batch"]
    torch.cuda.synchronize()
    # the NTT-based kernels' block shape per ring degree, timed on each
    # context's first evaluation (the context keeps the faster)
    shape_note, chunk_note = {}, {}
    for log_n, cx in ctxs.items():
        m0, ev0, c0, p0, o0 = next(it for it, cf in zip(items, cfgs) if cf["log_n"] == log_n)
        ws0 = m0.alloc_workspace()
        best, _, res = tuner.tune_ntt_shape(cx, lambda: m0.eval(ev0, c0, p0, o0, ws0))
        shape_note[str(log_n)] = {"chosen": best, "residues_per_thread": cx.ntt_shape()[1],
                                  "ms": {str(k): round(v, 3) for k, v in res.items()}}
        del ws0
        # the key-switching chunk, on the same representative, for every model of the ring degree
        ch, _, res = tuner.tune_chunk(m0, ev0, c0, p0, o0)
        chunk_note[str(log_n)] = {"chosen": ch, "ms": {str(k): round(v, 3) for k, v in res.items()}}
        for it, cf in zip(items, cfgs):
            if cf["log_n"] == log_n:
                it[0].set_chunk(ch)
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info()
    budget = max(0, free - (8 << 30))
    lanes, _, lane_res = tuner.tune_lanes(items, candidates=(1, 2, 4, 8), budget_bytes=budget)
    batch = bcn.Batch(items, lanes)
    for _ in range(max(1, args.warmup)):
        batch.launch()
    torch.cuda.synchronize()
    K = args.steps
    st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(device)
    clocks.start()
    for i in range(K):
        st[i].record()
        batch.launch()
        en[i].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in zip(st, en)]
    batch.close()
    del batch
    torch.cuda.empty_cache()
    # the same tuned models one after another, no graph (what the graph and lanes add)
    big = max((it[0] for it in items), key=lambda m: m.workspace_bytes())
    ws = big.alloc_workspace()

    def time_seq(seq_items, reps=2):
        best = None
        for _ in range(reps):
            s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            s0.record()
            for (m, evk, cts, pts, out) in seq_items:
                m.eval(evk, cts, pts, out, ws)
            e0.record()
            torch.cuda.synchronize()
            t = s0.elapsed_time(e0)
            best = t if best is None else min(best, t)
        return best

    seq_tuned_ms = time_seq(items)
    # the plain per-request path: each evaluation alone, every kernel in order
    # on one stream (no chunk halves side by side, no feature transforms ahead),
    # the configuration's own digit size and the default chunk, no graph
    plain_ctx, plain_evk = {}, {}
    plain_items = []
    for cfg, (m_t, _, cts, pts, out) in zip(cfgs, items):
        if cfg["log_n"] not in plain_ctx:
            cx = bcn.Context.from_config(cfg, device)
            _, ek = cx.keygen(workloads.SEED_KEYS)
            plain_ctx[cfg["log_n"]], plain_evk[cfg["log_n"]] = cx, cx.evk_prepare(bcn.to_device(ek, dev))
        wq = [bcn.quantize(w) for w in workloads.cipher_weights(cfg)]
        m = bcn.Model(plain_ctx[cfg["log_n"]], cfg["cipher"], [x for x, _ in wq], [y for _, y in wq])
        m.set_overlap(False)
        plain_items.append((m, plain_evk[cfg["log_n"]], cts, pts, out))
    del ws
    torch.cuda.empty_cache()
    big = max((it[0] for it in plain_items), key=lambda m: m.workspace_bytes())
    ws = big.alloc_workspace()
    plain_ms = [time_seq(plain_items)]
    value, mean_ms = replica_summary(statistics.mean(ms), images, None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": max(1, args.warmup),
        "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (uniform residues as ciphertexts and encoded features)",
        "config": {"workload": "uneven64: 64 evaluations, N in {4096, 8192, 16384}, sensitive fraction 10-60%, "
                               "slot occupancy 25-100%, one CUDA graph",
                   "images_per_step": images, "lanes": lanes,
                   "counts": {str(k): sum(1 for c in cfgs if c["log_n"] == k) for k in (12, 13, 14)}},
        "p50_ms": statistics.median(ms), "p99_ms": float(np.percentile(ms, 99)),
        "tuning": {"lanes_ms": {str(k): round(v, 3) for k, v in lane_res.items()}, "alpha_ms": alpha_note,
                   "ntt_shape": shape_note, "chunk": chunk_note},
        "plain_sequential": {"value": images / (min(plain_ms) / 1e3), "ms_per_step": min(plain_ms),
                             "path": "each evaluation alone, every kernel in order on one stream, the "
                                     "configuration's digit size and the default chunk, no graph"},
        "speedup_vs_plain": min(plain_ms) / statistics.mean(ms),
        "sequential_tuned_models": {"value": images / (seq_tuned_ms / 1e3), "ms_per_step": seq_tuned_ms,
                                    "path": "the batch's own (tuned) models one after another, no graph"},
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# serving: Poisson arrivals, continuous batching over lanes, 16 clients
# ---------------------------------------------------------------------------
def run_serve(args, rank, world, local_rank):
    import torch

    from paper_2402_01296_gb300 import bcn, serve

    device = local_rank
    torch.cuda.set_device(device)
    dev = f"cuda:{device}"
    n_clients, budget = 16, 120 << 30
    models, images = {}, {}
    for name in ("cnn3_small", "cryptonets"):
        cfg = workloads.get_config(name)
        ctx = bcn.Context.from_config(cfg, device)
        wq = [bcn.quantize(w) for w in workloads.cipher_weights(cfg)]
        model = bcn.Model(ctx, cfg["cipher"], [a for a, _ in wq], [s_ for _, s_ in wq])
        evks = [ctx.evk_prepare(bcn.to_device(ctx.keygen(1000 + c)[1], dev)) for c in range(n_clients)]
        models[name] = (model, evks)
        images[name] = cfg["batch"]
    # one seeded payload per (model, client), page-locked on the host
    g = np.random.default_rng(workloads.SEED_ENC)
    payload = {}
    for name, (model, _) in models.items():
        ctx = model.ctx
        for c in range(n_clients):
            def res(primes, lead):
                a = np.empty(tuple(lead) + (len(primes), ctx.N), dtype=np.uint32)
                for i, q in enumerate(primes):
                    a[..., i, :] = g.integers(0, q, size=tuple(lead) + (ctx.N,), dtype=np.uint32)
                t = torch.from_numpy(a.view(np.int32)).pin_memory()
                return t.numpy().view(np.uint32)
            payload[(name, c)] = (res(ctx.q, (model.n_in, 2)),
                                  [res(ctx.q[:sh[1]], (sh[0],)) for sh in model.pt_shapes()])
    stacks = {}
    for part in filter(None, args.stacks.split(";")):
        name, sizes = part.split(":")
        stacks[name] = [int(v) for v in sizes.split(",")]
    srv = serve.Server(models, lanes=args.lanes, budget_bytes=budget, device=device, stacks=stacks)
    srv.warm(args.lanes)  # idle slots with their evaluations captured for every client key
    rates = [float(r) for r in args.rates.split(",")]
    results = []
    for rate in rates:
        arr = serve.poisson_arrivals(rate, args.serve_seconds, seed=int(rate))
        gg = np.random.default_rng(int(rate) + 1)
        def make():
            out = []
            for i, t in enumerate(arr):
                name = "cnn3_small" if gg.random() < 0.7 else "cryptonets"
                c = int(gg.integers(0, n_clients))
                cts, pts = payload[(name, c)]
                out.append(serve.Request(rid=i, client=c, model=name, arrival=float(t), cts=cts, pts=pts))
            return out
        reqs = make()
        srv.run(reqs[: min(20, len(reqs))])  # warm-up
        torch.cuda.synchronize()
        clocks = ClockSampler(device)
        clocks.start()
        done = srv.run(reqs)
        clk = clocks.stop()
        st = serve.latency_stats(done, images)
        gg = np.random.default_rng(int(rate) + 1)
        plain = serve.latency_stats(serve.run_plain(models, make(), device), images)
        results.append({"rate_req_per_s": rate, "served": st, "plain": plain, "clocks": clk,
                        "host": dict(srv.scheduler.stats)})
    best = max(r["served"]["throughput_inferences_per_s"] for r in results)
    line = {
        "metric": METRIC, "value": best, "unit": UNIT, "n_gpus": world, "steps": len(rates), "warmup": 1,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (uniform residues as request ciphertexts and encoded features)",
        "config": {"workload": "serve: Poisson arrivals, 70% cnn3_small (N=4096, 2048 images) / 30% cryptonets "
                               "(N=8192, 4096 images), 16 clients with resident keys, 120 GiB budget",
                   "lanes": len(srv.lanes), "seconds_per_rate": args.serve_seconds,
                   "admission": "per request working set (inputs, features, output, workspace) from the arena "
                                "left after the keys; idle working sets kept as slots with captured graphs, "
                                "reclaimed for other models on demand",
                   "stacks": stacks,
                   "slots_created": srv.scheduler.n_slots, "slot_evictions": srv.scheduler.evictions,
                   "arena_peak_bytes": srv.scheduler.peak_used},
        "rates": results,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# slot rotations (automorphism + key switch with a Galois key)
# ---------------------------------------------------------------------------
def run_rotate(args, rank, world, local_rank):
    """Rotations of the CryptoNets-scale ciphertexts (N = 8192, 7 + 1 primes,
    the 256 ciphertexts of a slot batch at the top level) and of the CIFAR-shaped
    ones (N = 16384, 11 + 2 primes, alpha 2, 768 ciphertexts): rotations/s, L2
    flushed between timed steps."""
    import torch

    from paper_2402_01296_gb300 import bcn

    device = local_rank
    torch.cuda.set_device(device)
    dev = f"cuda:{device}"
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(workloads.SEED_ENC)
    res = {}
    for name, n_ct in (("cryptonets", 256), ("cifar_cnn", 768)):
        cfg = workloads.get_config(name)
        ctx = bcn.Context.from_config(cfg, device)
        sk, _ = ctx.keygen(workloads.SEED_KEYS)
        gk = ctx.evk_prepare(bcn.to_device(ctx.galois_keygen(sk, 1, workloads.SEED_KEYS), dev))
        x = _dev_residues(torch, ctx.q, (n_ct, 2), ctx.N, gen, dev)
        out = torch.empty_like(x)
        ws, nb = ctx._ws(ctx.L, n_ct)
        run = lambda: bcn.lib().bcn_op_rotate(ctx.handle, ctx.L, gk.data_ptr(), 1, x.data_ptr(), n_ct,  # noqa: E731
                                              out.data_ptr(), ws.data_ptr(), nb,
                                              torch.cuda.current_stream().cuda_stream)
        for _ in range(max(3, args.warmup)):
            assert run() == 0
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record()
            assert run() == 0
            e_.record()
            torch.cuda.synchronize()
            ms.append(s_.elapsed_time(e_))
        t = statistics.mean(ms)
        res[name] = {"ciphertexts": n_ct, "level": ctx.L, "ms_per_step": t, "rotations_per_s": n_ct / (t / 1e3)}
        # the nine offsets of a 3x3 packed convolution over rows of 16 slots:
        # one at a time (nine bcn_op_rotate calls) against one hoisted call
        steps = [i * 16 + j for i in range(3) for j in range(3) if i * 16 + j]
        gks = {r: ctx.evk_prepare(bcn.to_device(ctx.galois_keygen(sk, r, workloads.SEED_KEYS + r), dev))
               for r in steps}
        n_h = min(n_ct, 64)
        xh = x[:n_h].contiguous()
        many = torch.empty((n_h, len(steps), 2, ctx.L, ctx.N), dtype=torch.int32, device=dev)
        one = torch.empty((n_h, 2, ctx.L, ctx.N), dtype=torch.int32, device=dev)
        ws_h, nb_h = ctx._ws(ctx.L, n_h)

        def seq():
            for r in steps:
                assert bcn.lib().bcn_op_rotate(ctx.handle, ctx.L, gks[r].data_ptr(), r, xh.data_ptr(), n_h,
                                               one.data_ptr(), ws_h.data_ptr(), nb_h,
                                               torch.cuda.current_stream().cuda_stream) == 0

        def hoisted():
            ctx.op_rotate_many(ctx.L, gks, steps, xh, n_h, many)

        tm = {}
        for label, fn in (("one_at_a_time", seq), ("hoisted", hoisted)):
            for _ in range(2):
                fn()
            torch.cuda.synchronize()
            mm = []
            for _ in range(max(1, args.steps // 2)):
                flush.zero_()
                s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s_.record()
                fn()
                e_.record()
                torch.cuda.synchronize()
                mm.append(s_.elapsed_time(e_))
            tm[label] = statistics.mean(mm)
        res[name]["conv3x3_rotations"] = {
            "ciphertexts": n_h, "rotations_each": len(steps),
            "ms_one_at_a_time": tm["one_at_a_time"], "ms_hoisted": tm["hoisted"],
            "rotations_per_s_hoisted": n_h * len(steps) / (tm["hoisted"] / 1e3),
            "speedup": tm["one_at_a_time"] / tm["hoisted"]}
        del ctx
    if rank == 0:
        print(json.dumps({"metric": "rotations/s", "value": res["cryptonets"]["rotations_per_s"],
                          "unit": "rotations/s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
                          "higher_is_better": True, "dtype": "u32", "data": "synthetic (uniform residues)",
                          "config": {"workload": "rotate: one-slot rotations of a slot batch's ciphertexts",
                                     "l2": "flushed (512 MiB write) between timed steps, outside the events"},
                          "rotations": res}), flush=True)


def run_bhw(args, rank, world, local_rank):
    """The CryptoNets-scale ciphertext branch in BHW packing (App. D): 16
    images' 16 x 16 segments per ciphertext (N = 8192, 7 + 1 primes), 5 x 5
    stride-2 conv to 5 maps by hoisted rotations and the MAC, square, 180 -> 100
    and 100 -> 10 by the diagonal method over the strided outputs, the feature
    adds and the second square.  --groups ciphertext groups per step, and one
    group alone (the latency of 16 images); L2 flushed between timed steps."""
    import torch

    from paper_2402_01296_gb300 import bcn, bhw

    device = local_rank
    torch.cuda.set_device(device)
    dev = f"cuda:{device}"
    cfg = workloads.get_config("cryptonets")
    ctx = bcn.Context.from_config(cfg, device)
    n_img, G = 16, args.groups
    layers = [dict(cfg["cipher"][0])] + [dict(l) for l in cfg["cipher"][1:]]
    rng = np.random.default_rng(workloads.SEED_WEIGHTS)
    ho = (16 - 5) // 2 + 1
    wts = [rng.integers(-3, 4, (5, 1, 5, 5)).astype(np.int8), rng.integers(-3, 4, (100, 5 * ho * ho)),
           rng.integers(-3, 4, (10, 100))]
    sk, ek = ctx.keygen(workloads.SEED_KEYS)
    steps = bhw.BranchBHW.steps_for(layers, n_img, ctx.N)
    gks = {r: ctx.evk_prepare(bcn.to_device(ctx.galois_keygen(sk, r, workloads.SEED_KEYS + r), dev)) for r in steps}
    br = bhw.BranchBHW(ctx, layers, wts, n_img, gks, ctx.evk_prepare(bcn.to_device(ek, dev)))
    gen = torch.Generator(device=dev)
    gen.manual_seed(workloads.SEED_ENC)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    n_rot = len(br.conv_steps) - 1 + sum(d["n_in"] * len(d["steps"]) for d in br.dense)

    def timed(g, steps_):
        x = _dev_residues(torch, ctx.q, (g, 1, 2), ctx.N, gen, dev)
        feats = []
        for shp in br.feature_shapes(g):
            feats.append(_dev_residues(torch, ctx.q[:shp[-2]], shp[:-2], ctx.N, gen, dev))
        out = torch.empty((g, 2, br.out_level, ctx.N), dtype=torch.int32, device=dev)
        for _ in range(max(3, args.warmup)):
            br(x, g, feats, out)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps_):
            flush.zero_()
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record()
            br(x, g, feats, out)
            e_.record()
            torch.cuda.synchronize()
            ms.append(s_.elapsed_time(e_))
        assert ctx.device_status() == 0
        return statistics.mean(ms)

    clocks = ClockSampler(device)
    clocks.start()
    t = timed(G, args.steps)
    clk = clocks.stop()
    t1 = timed(1, args.steps)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": G * n_img * world / (t / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (uniform residues as ciphertexts and features; integer weights in [-3, 3])",
            "config": {"workload": f"bhw: CryptoNets-scale branch in BHW packing, {G} groups of {n_img} images "
                                   "(N=8192, 7+1 primes)",
                       "l2": "flushed (512 MiB write) between timed steps, outside the events"},
            "rotations_per_group": n_rot, "rotations_per_s": G * n_rot * world / (t / 1e3),
            "latency_ms_one_group": t1, "clocks": clk}), flush=True)


# ---------------------------------------------------------------------------
# op-level workloads (small cases for kernel profiles)
# ---------------------------------------------------------------------------
def run_op(args, rank, world, local_rank):
    """One operation of the CIFAR-shaped network on a bounded number of
    ciphertexts, L2 flushed between timed steps: `op_square` is the square
    activation (tensor square, key switch, ModDown, rescale) of --cts
    ciphertexts at the top level (N = 16384, 11 + 2 primes, alpha 2); `op_mac`
    is one layer shaped like the network's second convolution (16 -> 32 maps,
    3x3, stride 2, padding 1) on a --map x --map input at 11 limbs, on the
    tensor cores."""
    import torch

    from paper_2402_01296_gb300 import bcn

    device = local_rank
    torch.cuda.set_device(device)
    dev = f"cuda:{device}"
    cfg = workloads.get_config("cifar_cnn")
    ctx = bcn.Context.from_config(cfg, device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(workloads.SEED_ENC)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    if args.workload == "op_square":
        n = args.cts
        _, ek = ctx.keygen(workloads.SEED_KEYS)
        evk = ctx.evk_prepare(bcn.to_device(ek, dev))
        x = _dev_residues(torch, ctx.q, (n, 2), ctx.N, gen, dev)
        out = torch.empty((n, 2, ctx.L - 1, ctx.N), dtype=torch.int32, device=dev)
        run = lambda: ctx.op_square_relin_rescale(ctx.L, evk, x, n, out)  # noqa: E731
        what, unit = f"op_square: {n} ciphertexts at 11 limbs, N=16384, 11+2 primes, alpha 2", "squares/s"
    else:
        hw = args.map
        layer = dict(type="conv", cin=16, h=hw, w=hw, cout=32, k=3, stride=2, pad=1, add=True, square=False)
        n_in, n = workloads.cipher_layer_io(layer)
        w = np.random.default_rng(workloads.SEED_WEIGHTS).integers(-127, 128, (32, 16, 3, 3)).astype(np.int8)
        m = bcn.Model(ctx, [layer], [w], [1.0])
        x = _dev_residues(torch, ctx.q, (n_in, 2), ctx.N, gen, dev)
        pt = [_dev_residues(torch, ctx.q, (n,), ctx.N, gen, dev)]
        out = torch.empty(m.out_shape(), dtype=torch.int32, device=dev)
        ws = m.alloc_workspace()
        key = torch.zeros(ctx.evk_words(), dtype=torch.int32, device=dev)  # no square: the key is not read
        run = lambda: m.eval(key, x, pt, out, ws)  # noqa: E731
        what, unit = f"op_mac: conv 16->32 3x3/2 pad 1 on {hw}x{hw} ({n_in} -> {n} ciphertexts, 11 limbs)", "outputs/s"
    for _ in range(max(3, args.warmup)):
        run()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_.record(stream)
        run()
        e_.record(stream)
        torch.cuda.synchronize()
        ms.append(s_.elapsed_time(e_))
    t = statistics.mean(ms)
    if rank == 0:
        print(json.dumps({"metric": unit, "value": n / (t / 1e3), "unit": unit, "n_gpus": world,
                          "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": t,
                          "higher_is_better": True, "dtype": "u32", "data": "synthetic (uniform residues)",
                          "config": {"workload": what,
                                     "l2": "flushed (512 MiB write) between timed steps, outside the events"}}),
              flush=True)


def main():
    # no garbage-collector pause inside a timed step (the steps are timed on the
    # device, and a host pause while a step is being enqueued idles the GPU)
    import gc
    gc.disable()
    try:
        _main()
    finally:
        gc.enable()


def _main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.workload == "uneven64":
        return run_uneven(args, rank, world, local_rank)
    if args.workload == "serve":
        return run_serve(args, rank, world, local_rank)
    if args.workload == "rotate":
        return run_rotate(args, rank, world, local_rank)
    if args.workload == "bhw":
        return run_bhw(args, rank, world, local_rank)
    if args.workload in ("op_square", "op_mac"):
        return run_op(args, rank, world, local_rank)
    if args.workload == "cifar_profile":
        # the CIFAR-shaped network on the full ring and chain (N = 16384, 11 + 2
        # primes, 16x16x3 segment) with 4 and 8 maps: the same kernels and launch
        # sizes as the full network with a few GB on the device (profiling captures)
        cfg = workloads.reduced_cifar(cout1=4, cout2=8, seg=16, batch=8192)
    else:
        cfg = workloads.get_config(args.workload)
    if args.impl == "reference":
        run_reference(args, cfg, rank, world)
    else:
        run_ours(args, cfg, rank, world, local_rank)


if __name__ == "__main__":
    main()
