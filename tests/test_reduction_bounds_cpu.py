"""The range arguments behind the device's shortcut reductions, checked on the
host for every prime chain of the benchmark networks (host-only contexts):

* the MAC epilogues reduce a sum below 2^59 with a 32-bit quotient estimate
  from floor(2^61 / q) = floor(floor(2^64 / q) / 8): the estimate is at most 2
  below the true quotient and never above it, which needs every data prime in
  (2^29, 2^30) -- the context refuses a chain that is not;
* the MAC sums start at the limb's offset (a multiple of q >= 2^58), so with the
  2^20-tap limit and int8 weights they stay in (0, 2^59);
* the key switch's lazy two-prime ModUp residue and ModDown's lazy conversion
  stay below 4q and are congruent to the canonical values.

Each step is simulated with 32-bit wrap-around as the kernels compute it."""
import numpy as np
import pytest

import workloads
from paper_2402_01296_gb300 import bcn

M32 = (1 << 32) - 1
CONFIGS = ["cnn3_small", "cryptonets", "cifar_cnn"]


def shoup_lazy(a, w, q):
    """a w - floor(a floor(w 2^32 / q) / 2^32) q, the device's lazy Shoup product."""
    wp = (w << 32) // q
    return (a * w - ((a * wp) >> 32) * q) & M32


def reduce59(x, q):
    mu = (1 << 64) // q
    qe = (((x >> 29) & M32) * ((mu >> 3) & M32)) >> 32
    r = (x - qe * q) & M32
    r = min(r, (r - 2 * q) & M32)
    r = min(r, (r - q) & M32)
    return qe, r


def chain(name):
    cfg = workloads.get_config(name)
    return bcn.Context(cfg["log_n"], cfg["n_data"], cfg["n_special"], cfg["alpha"], device=-1)


@pytest.mark.parametrize("name", CONFIGS)
def test_mac_reduction_quotient_estimate(name):
    ctx = chain(name)
    rng = np.random.default_rng(5)
    for q in ctx.q:
        assert (1 << 29) < q < (1 << 30)
        off = ((1 << 58) // q + 1) * q
        span = (1 << 20) * 128 * (q - 1)  # the largest |sum of products| (int8 weights, 2^20 taps)
        assert 0 < off - span and off + span < (1 << 59)
        xs = [0, 1, q - 1, q, off - span, off + span, (1 << 59) - 1, off]
        xs += [int(v) for v in rng.integers(0, 1 << 59, size=200, dtype=np.uint64)]
        xs += [k * q + d for k in (1, 2 ** 20, (1 << 59) // q - 1) for d in (0, 1, q - 1)]
        for x in xs:
            qe, r = reduce59(x, q)
            assert x // q - 2 <= qe <= x // q
            assert r == x % q


@pytest.mark.parametrize("name", CONFIGS)
def test_lazy_conversions_stay_below_4q(name):
    ctx = chain(name)
    rng = np.random.default_rng(6)
    qs, ps = ctx.q, ctx.p
    for t in qs:
        # two-prime ModUp digit (q_a, q_b) into data prime t: products, one fold,
        # t - (D mod t) per centred correction
        qa, qb = qs[0], qs[1]
        if t in (qa, qb):
            qa, qb = qs[-1], qs[-2]
        D = qa * qb
        tmq = t - D % t
        dha, dhb = (D // qa) % t, (D // qb) % t
        for _ in range(200):
            ra, rb = int(rng.integers(0, qa)), int(rng.integers(0, qb))
            y = shoup_lazy(ra, dha, t) + shoup_lazy(rb, dhb, t)
            assert y < 4 * t
            y = min(y, (y - 2 * t) & M32)
            y += (tmq if ra > (qa - 1) // 2 else 0) + (tmq if rb > (qb - 1) // 2 else 0)
            assert y < 4 * t
            canon = (ra * dha + rb * dhb - ((ra > (qa - 1) // 2) + (rb > (qb - 1) // 2)) * D) % t
            assert y % t == canon
        # ModDown's conversion of up to two special-prime limbs into t
        if len(ps) > 2:
            continue
        P = int(np.prod([int(p) for p in ps], dtype=object))
        pmod = P % t
        phat = [(P // p) % t for p in ps]
        pinv = pow(P, -1, t)
        for _ in range(200):
            rs = [int(rng.integers(0, p)) for p in ps]
            conv, corr = 0, 0
            for m, (r, p) in enumerate(zip(rs, ps)):
                conv += shoup_lazy(r, phat[m], t)
                if m > 0:
                    conv = min(conv, (conv - 2 * t) & M32)
                corr += (t - pmod) if r > (p - 1) // 2 else 0
            assert conv + corr < 4 * t
            lift = int(rng.integers(0, t))
            x = shoup_lazy(conv + corr, pinv, t) + lift
            assert x < 3 * t
            cnt = sum(r > (p - 1) // 2 for r, p in zip(rs, ps))
            canon = ((sum(r * h for r, h in zip(rs, phat)) - cnt * P) * pinv + lift) % t
            assert x % t == canon
