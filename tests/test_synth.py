"""The seeded generators: deterministic, and shaped as their recipes state (CPU only)."""
import math

import torch

from paper_1703_02438_gb300 import synth


def test_plain_pair_recipe():
    p, x = synth.plain_pair(1 << 16)
    p2, x2 = synth.plain_pair(1 << 16)
    assert torch.equal(p, p2) and torch.equal(x, x2)
    assert p.dtype == torch.float64 and p.shape == (1 << 16,)
    assert int((p == 0).sum()) == round(0.01 * (1 << 16))
    nz = p != 0
    r = x[nz] / p[nz] - 1
    assert abs(float(torch.log(p[nz]).mean())) < 0.03          # LogNormal(0, 1)
    assert 0.09 < float((r.abs() > 0.02).double().mean()) < 0.11 # ~10% uniform tail (|r| > 2%)
    assert float(r.min()) >= -0.5 and float(r.max()) <= 0.5


def test_flash_series_small():
    s = synth.flash_series(side=32, steps=3)
    assert len(s) == 3 and all(t.shape == (32 ** 3,) and t.dtype == torch.float64 for t in s)
    assert all(bool((t > 0).all()) for t in s)
    ratio = s[1] / s[0] - 1
    shocks = ratio.abs() > 0.05
    assert 0.03 < float(shocks.double().mean()) < 0.07          # ~5% shock cells
    # smooth drift: 2e-3 sinusoid + 1e-3 smooth field (a few shock draws land below 5%)
    assert float((ratio[~shocks].abs() < 0.01).double().mean()) > 0.99


def test_climate_series_small():
    steps = list(synth.climate_series(nlat=90, nlon=180, steps=3))
    assert [t for t, _ in steps] == [0, 1, 2]
    v0, v1 = steps[0][1], steps[1][1]
    assert v0.dtype == torch.float32 and v0.shape == (90 * 180,)
    mask0, mask1 = v0 == 0, v1 == 0
    assert torch.equal(mask0, mask1)
    assert 0.02 < float(mask0.double().mean()) < 0.04
    alone = dict(synth.climate_series(nlat=90, nlon=180, steps=3, start=1))
    assert torch.equal(alone[1], v1)
    assert math.isclose(float(v0[~mask0].mean()), 288 - 40 * 0.5, rel_tol=0.05)
