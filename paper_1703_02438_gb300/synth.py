"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws data. It contains none of the compression arithmetic, and it is the one
module that both the CUDA path's tests/bench and the CPU oracle's tests take inputs from.

The paper evaluates on FLASH (Sedov, Stir), ASR and CMIP outputs (§V, Table 1), which are not
available here; these generators stand in for them:

* ``plain_pair``   one 1-D float64 variable pair: prev ~ LogNormal(0, 1) with 1% exact zeros;
                   cur = prev * (1 + r), r from the mixture 60% N(0, 1e-3), 30% N(8e-3, 2e-3),
                   10% U(-0.5, 0.5). (Stands in for a generic temporal variable; the heavy
                   uniform tail makes many near-equal bin counts.)
* ``flash_series`` a 3-D float64 density-like field series (stands in for FLASH Stir/Sedov):
                   rho_0 = exp(g), g a unit-variance Gaussian random field with power
                   spectrum |k|^(-5/3); rho_{t+1} = rho_t * (1 + delta_t), delta_t a smooth
                   advection-like drift 2e-3 * sin(2*pi*(i+j+k)/side + 0.7 t) plus 1e-3 times a
                   fresh smooth random field, and on a seeded 5% of cells large jumps
                   ("shocks") delta ~ U(-0.5, 2).
* ``climate_series`` a 2-D float32 lat x lon field series (stands in for CMIP / ASR): smooth
                   latitude profile 288 - 40 sin^2(lat) plus a seasonal term
                   10 sin(lat) sin(2 pi t / 12), times (1 + 0.5% correlated noise) (Gaussian-
                   smoothed N(0,1), sigma = 4 cells, renormalised, fresh per month); a fixed
                   seeded 3% of cells ("ocean mask") is exactly 0 in every step.

Seeds follow 170302438 + 1000 * workload + variant. All generation is done with torch so the
same code runs on the host (small sizes, oracle tests) and on the GPU (full sizes).
"""
from __future__ import annotations

import math

import torch

SEED_BASE = 170302438


def seed_for(workload: int, variant: int = 0) -> int:
    return SEED_BASE + 1000 * workload + variant


def _gen(device, seed: int) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


# ----------------------------------------------------------------------------------------
# Plain 1-D pair
# ----------------------------------------------------------------------------------------
def plain_pair(n: int = 1 << 20, seed: int = seed_for(0), dtype=torch.float64,
               zero_frac: float = 0.01, scale: float = 1.0, device="cpu"):
    """(prev, cur) as tensors of `dtype` on `device` (generated in float64, then cast)."""
    g = _gen(device, seed)
    kw = dict(generator=g, dtype=torch.float64, device=device)
    prev = torch.empty(n, dtype=torch.float64, device=device).log_normal_(0.0, 1.0, generator=g)
    nz = int(round(zero_frac * n))
    if nz:
        prev[torch.randperm(n, generator=g, device=device)[:nz]] = 0.0
    pick = torch.rand(n, **kw)
    r1 = torch.randn(n, **kw) * 1e-3
    r2 = 8e-3 + torch.randn(n, **kw) * 2e-3
    r3 = torch.rand(n, **kw) - 0.5
    r = torch.where(pick < 0.6, r1, torch.where(pick < 0.9, r2, r3)) * scale
    cur = prev * (1.0 + r)
    return prev.to(dtype), cur.to(dtype)


def batch_specs(count: int = 256, seed: int = seed_for(3), n_lo: float = 1e4, n_hi: float = 2e8):
    """Per-variable recipe of a batch: (n, dtype, E, B, scale) with n log-uniform in
    [n_lo, n_hi], dtype float32/float64 with equal odds, E in {1e-2, 1e-3, 1e-4}, B in
    {6, 8, 10}, and the ratio mixture of plain_pair scaled by U(0.5, 4)."""
    g = _gen("cpu", seed)
    out = []
    for _ in range(count):
        u = torch.rand(5, generator=g, dtype=torch.float64).tolist()
        n = int(round(math.exp(math.log(n_lo) + u[0] * (math.log(n_hi) - math.log(n_lo)))))
        dtype = torch.float64 if u[1] < 0.5 else torch.float32
        E = (1e-2, 1e-3, 1e-4)[min(2, int(u[2] * 3))]
        B = (6, 8, 10)[min(2, int(u[3] * 3))]
        out.append((n, dtype, E, B, 0.5 + 3.5 * u[4]))
    return out


# ----------------------------------------------------------------------------------------
# 3-D FLASH-like series
# ----------------------------------------------------------------------------------------
def _spectral_field(side: int, slope: float, g: torch.Generator, device) -> torch.Tensor:
    """Unit-variance Gaussian random field on side^3 with power spectrum |k|^slope (k != 0)."""
    white = torch.randn((side, side, side), generator=g, dtype=torch.float64, device=device)
    spec = torch.fft.rfftn(white)
    del white
    k1 = torch.fft.fftfreq(side, d=1.0 / side, device=device, dtype=torch.float64)
    kz = torch.fft.rfftfreq(side, d=1.0 / side, device=device, dtype=torch.float64)
    k2 = (k1[:, None, None] ** 2 + k1[None, :, None] ** 2) + kz[None, None, :] ** 2
    k2[0, 0, 0] = 1.0
    amp = k2.pow(slope / 4.0)        # |k|^(slope/2) in amplitude = |k|^slope in power
    amp[0, 0, 0] = 0.0
    del k2
    spec.mul_(amp)
    del amp
    f = torch.fft.irfftn(spec, s=(side, side, side))
    del spec
    f.sub_(f.mean())
    f.div_(f.std())
    return f


def flash_series(side: int = 1024, steps: int = 4, seed: int = seed_for(1), device="cpu",
                 shock_frac: float = 0.05):
    """List of `steps` float64 tensors of side^3 elements (flattened, contiguous)."""
    g = _gen(device, seed)
    rho = torch.exp(_spectral_field(side, -5.0 / 3.0, g, device)).reshape(-1)
    out = [rho.clone()]
    n = side ** 3
    ar = torch.arange(side, device=device, dtype=torch.float64)
    phase_base = (ar[:, None, None] + ar[None, :, None] + ar[None, None, :]).reshape(-1)
    phase_base.mul_(2.0 * math.pi / side)
    shock = torch.rand(n, generator=g, device=device, dtype=torch.float64) < shock_frac
    for t in range(steps - 1):
        delta = torch.sin(phase_base + 0.7 * t).mul_(2e-3)
        delta.add_(_spectral_field(side, -11.0 / 3.0, g, device).reshape(-1), alpha=1e-3)
        jump = torch.rand(n, generator=g, device=device, dtype=torch.float64).mul_(2.5).sub_(0.5)
        delta = torch.where(shock, jump, delta)
        del jump
        rho = rho * (1.0 + delta)
        del delta
        out.append(rho.clone())
    return out


# ----------------------------------------------------------------------------------------
# 2-D climate-like series
# ----------------------------------------------------------------------------------------
def _smooth_noise_2d(nlat: int, nlon: int, sigma: float, g: torch.Generator, device):
    white = torch.randn((nlat, nlon), generator=g, dtype=torch.float64, device=device)
    spec = torch.fft.rfft2(white)
    fy = torch.fft.fftfreq(nlat, device=device, dtype=torch.float64)
    fx = torch.fft.rfftfreq(nlon, device=device, dtype=torch.float64)
    gauss = torch.exp(-2.0 * (math.pi * sigma) ** 2 * (fy[:, None] ** 2 + fx[None, :] ** 2))
    f = torch.fft.irfft2(spec * gauss, s=(nlat, nlon))
    f = f - f.mean()
    return f / f.std()


def climate_series(nlat: int = 1800, nlon: int = 3600, steps: int = 120,
                   seed: int = seed_for(2), device="cpu", mask_frac: float = 0.03,
                   start: int = 0):
    """Generator of (t, float32 tensor of nlat*nlon) for months start..steps-1.

    Each month's noise comes from its own seed, so any month can be produced alone."""
    lat = torch.linspace(-math.pi / 2, math.pi / 2, nlat, device=device, dtype=torch.float64)
    s = torch.sin(lat)[:, None]
    base = (288.0 - 40.0 * s * s).expand(nlat, nlon)
    gm = _gen(device, seed)
    mask = (torch.rand((nlat, nlon), generator=gm, device=device, dtype=torch.float64)
            < mask_frac)
    for t in range(start, steps):
        gt = _gen(device, seed + 1 + t)
        noise = _smooth_noise_2d(nlat, nlon, 4.0, gt, device)
        v = (base + 10.0 * s * math.sin(2.0 * math.pi * t / 12.0)) * (1.0 + 0.005 * noise)
        v = torch.where(mask, torch.zeros_like(v), v)
        yield t, v.to(torch.float32).reshape(-1).contiguous()
