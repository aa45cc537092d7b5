"""GPU parity of the float64 classification at the limits of its fast path.

The float64 kernels decide each bin id and each error-bound check (§III.C) from a float32
estimate of the change ratio (Eq. 1) and fall back to the exact float64 sequence where the
estimate's error bound cannot decide. The estimate is only used when prev's biased exponent lies
in [200, 1940] (bin and check) and cur's in [100, 1940] (check), and it rescales the difference
cur - prev by prev's power of two into float32's exponent range. These inputs sit on both sides of
each of those limits, so both branches run next to each other:

  * prev with biased exponent 199, 200, 201, 1939, 1940, 1941 and ratios from a mixture (small
    changes, bin edges a few ulps either side, wide ratios, unchanged points, ratios near -1);
  * cur with biased exponent 99, 100, 101, 1940, 1941 and prev = cur / (1 + ratio);
  * cur 2^100 and more below prev (ratio -1: the bin near -1/(2E), and a check that fails);
  * cur 2^k above prev (ratios 2^k - 1, bins inside and far outside the 16-bit code window);
  * differences whose rescaled exponent is at the top of float32's range (|cur/prev| of 2^125 to
    2^129: the estimate overflows, or the ratio is far beyond the cap);
  * unchanged points at every limit: the only way the rescaled difference falls below float32's
    normal range, since for normal prev a non-zero cur - prev is at least half an ulp of prev;
  * prev and cur drawn log-uniformly over the whole float64 range, subnormals included.

Each case is compared byte for byte with the oracle on both grids, and on the zero-centred grid
also through the chained step, whose fused kernel classifies the same way.
"""
import numpy as np
import pytest
import torch

from oracle import numarck_oracle as O
from paper_1703_02438_gb300 import numarck as N
from tests.test_gpu_parity import check_pair
from tests.test_gpu_step import run_chain

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1703_02438_gb300 import build
    build.build()
    N.lib()


def _ratios(rng, k, E):
    """A ratio mixture: small changes, bin edges +- a few ulps, wide ratios, zeros, near -1."""
    w = 2 * E
    kind = rng.integers(0, 6, k)
    r = rng.normal(0.0, 1e-3, k)
    edge = (-E + rng.integers(-400, 400, k) * w) * (1.0 + rng.integers(-3, 4, k) * 2.0 ** -52)
    r = np.where(kind == 1, edge, r)
    r = np.where(kind == 2, rng.uniform(-0.9, 3.0, k), r)
    r = np.where(kind == 3, 0.0, r)
    r = np.where(kind == 4, rng.uniform(-1.0, -0.99, k), r)
    r = np.where(kind == 5, rng.normal(8e-3, 2e-3, k), r)
    return r


def _scaled(rng, k, e):
    """sign * [1, 2) * 2^(e - 1023): biased exponent e (subnormal for e = 0)."""
    return rng.choice([-1.0, 1.0], k) * np.ldexp(1.0 + rng.random(k), np.asarray(e) - 1023)


def guard_pair(E=1e-3, per=2000, seed=71):
    rng = np.random.default_rng(seed)
    ps, xs = [], []
    with np.errstate(all="ignore"):
        for ep in (199, 200, 201, 1939, 1940, 1941):
            p = _scaled(rng, per, ep)
            ps.append(p)
            xs.append(p * (1.0 + _ratios(rng, per, E)))
        for ex in (99, 100, 101, 1940, 1941):
            x = _scaled(rng, per, ex)
            xs.append(x)
            ps.append(x / (1.0 + _ratios(rng, per, E)))
        for ex in (99, 100, 101):
            xs.append(_scaled(rng, per, ex))
            ps.append(_scaled(rng, per, rng.integers(200, 261, per)))
        for ex in (1940, 1941):
            k = rng.integers(0, 13, per)
            x = _scaled(rng, per, ex)
            xs.append(x)
            ps.append(np.abs(x) * rng.choice([-1.0, 1.0], per) * np.ldexp(1.0, -k)
                      * (1.0 + rng.uniform(-1e-3, 1e-3, per)))
        for ep in (200, 201, 1000, 1700, 1811):
            k = rng.integers(125, 130, per)
            p = _scaled(rng, per, ep)
            ps.append(p)
            xs.append(_scaled(rng, per, np.minimum(ep + k, 2046)))
        for e in (99, 100, 101, 199, 200, 201, 1939, 1940, 1941):
            p = _scaled(rng, per // 4, e)
            ps.append(p)
            xs.append(p.copy())
        # non-finite x against p whose biased exponent is 1920..1940, where x - p = +-inf or NaN
        # still passes the estimate's exponent test: its size (>= 2^106) must keep it out
        nanbits = np.array([0x7FF8000000000000, 0x7FF0000000000001, 0xFFF4000000000ABC],
                           dtype=np.uint64).view(np.float64)
        specials = np.concatenate([[np.inf, -np.inf], nanbits])
        p = _scaled(rng, per, rng.integers(1920, 1941, per))
        ps.append(p)
        xs.append(specials[rng.integers(0, specials.size, per)])
        bits = (rng.integers(0, 2047, 4 * per).astype(np.uint64) << np.uint64(52)) | \
            rng.integers(0, 1 << 52, 4 * per, dtype=np.uint64)
        p = bits.view(np.float64) * rng.choice([-1.0, 1.0], 4 * per)
        half = 2 * per
        x = np.concatenate([p[:half] * (1.0 + _ratios(rng, half, E)),
                            _scaled(rng, half, rng.integers(0, 2047, half))])
        ps.append(p)
        xs.append(x)
    p = np.concatenate(ps)
    x = np.concatenate(xs)
    order = rng.permutation(p.size)
    return p[order].copy(), x[order].copy()


def test_guard_inputs_reach_both_sides():
    """The generator's own check: the inputs cover the exponents named above."""
    p, x = guard_pair()
    ep = (p.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)
    ex = (x.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)
    for e in (199, 200, 201, 1939, 1940, 1941):
        assert (ep == e).sum() >= 500, e
    for e in (99, 100, 101, 1940, 1941):
        assert (ex == e).sum() >= 500, e
    assert ((ep == 0) & (p != 0)).any() and ((ex == 0) & (x != 0)).any()   # subnormals
    high = (ep >= 1920) & (ep <= 1940)
    assert (high & np.isinf(x)).sum() >= 500 and (high & np.isnan(x)).sum() >= 500
    with np.errstate(all="ignore"):
        q = np.abs(x / p)
    assert ((q > 2.0 ** 125) & (q < 2.0 ** 130)).sum() >= 1000


@pytest.mark.parametrize("B", [10, 14])
@pytest.mark.parametrize("E", [1e-3, 3.3e-5])
@pytest.mark.parametrize("anchor", [N.ANCHOR_ZERO, N.ANCHOR_MIN])
def test_f64_guard_limits_match_oracle(E, B, anchor):
    p, x = guard_pair(E)
    h, _ = check_pair(p, x, E, B, anchor=anchor, ranges=[(0, p.size), (12_345, 6_789)])
    assert 0 < h["n_inc"] < h["n"]


@pytest.mark.parametrize("B", [10, 14])
@pytest.mark.parametrize("E", [1e-3, 3.3e-5])
def test_f64_guard_limits_chained_step(E, B):
    """prev -> prev (unchanged: the reconstruction is prev bit for bit) -> cur, so the fused
    step classifies (prev, cur) against the reconstruction."""
    p, x = guard_pair(E, seed=72)
    s = [torch.from_numpy(v).to(DEV) for v in (p, p.copy(), x)]
    run_chain(s, E, B)
