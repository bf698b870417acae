"""Seeded synthetic inputs shaped like the paper's workloads.

This module only makes input fields and threshold arrays; it holds none of
the EC arithmetic.  Tests, the benchmark and the smoke check all take their
inputs from here, and the CUDA path and the CPU oracle then read the same
bytes.  The paper's own synthetic fields (Sec. 3.1) are iid uniform / normal
noise quantised to 0..255; its real datasets are not available, so smoothed
Gaussian random fields and Gaussian-blob densities stand in for them.

Recipes (all seeded):
  grf_2d          N(0,1) pixels (torch CPU generator, float64) -> Gaussian blur
                  (separable, kernel truncated at 4 sigma, reflect border, or
                  periodic FFT for large fields) -> optional uint8 quantisation
                  q = clamp(round(255 (f - min) / (max - min)), 0, 255).
  blobs_3d        sum of isotropic Gaussian blobs a exp(-|x - c|^2 / (2 r^2)),
                  c ~ U[0, n)^3, r ~ U[3, 12], a ~ U[0.5, 1.5], each added
                  within 4r of its centre and clipped at the domain, plus
                  N(0, 0.05^2) iid noise; float32.
  uniform_thresholds  t_k = float32(min + (max - min) k / (L - 1)) computed in
                  float64, t_0 = min and t_{L-1} = max exactly.
  request_stream  the served workload: Poisson arrivals, 70 % 2D uint8 fields
                  (side log-uniform 64..4096, 256 levels), 30 % 3D float32
                  fields (side log-uniform 32..512, L ~ U{64..1024}), each a
                  smoothed Gaussian random field with sigma ~ U[2, 10].
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _gen(seed: int) -> torch.Generator:
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


def gaussian_kernel_1d(sigma: float) -> torch.Tensor:
    r = int(math.ceil(4 * sigma))
    x = torch.arange(-r, r + 1, dtype=torch.float64)
    k = torch.exp(-x * x / (2 * sigma * sigma))
    return k / k.sum()


def _blur_separable(f: torch.Tensor, sigma: float) -> torch.Tensor:
    """Separable Gaussian blur with reflect padding, along every axis of f."""
    k = gaussian_kernel_1d(sigma).to(f.device)
    r = (k.numel() - 1) // 2
    out = f
    for axis in range(f.dim()):
        x = out.movedim(axis, -1)
        shp = x.shape
        x = x.reshape(-1, 1, shp[-1])
        pad = min(r, shp[-1] - 1)
        if pad > 0:
            x = torch.nn.functional.pad(x, (pad, pad), mode="reflect")
        kk = k if pad == r else k[r - pad:r + pad + 1] / k[r - pad:r + pad + 1].sum()
        x = torch.nn.functional.conv1d(x, kk.view(1, 1, -1))
        out = x.reshape(shp).movedim(-1, axis)
    return out


def _blur_fft(f: torch.Tensor, sigma: float) -> torch.Tensor:
    """Periodic Gaussian blur by FFT (float64)."""
    freqs = [torch.fft.fftfreq(n, device=f.device, dtype=torch.float64) for n in f.shape]
    grids = torch.meshgrid(*freqs, indexing="ij")
    w2 = sum(g * g for g in grids)
    H = torch.exp(-2 * (math.pi ** 2) * (sigma ** 2) * w2)
    return torch.fft.ifftn(torch.fft.fftn(f) * H).real


def quantize_u8(f: torch.Tensor) -> torch.Tensor:
    lo, hi = f.min(), f.max()
    q = torch.round(255.0 * (f - lo) / (hi - lo)).clamp(0, 255)
    return q.to(torch.uint8)


def grf_2d(seed: int, h: int, w: int, sigma: float, device="cpu", fft: bool = False) -> torch.Tensor:
    """Smoothed Gaussian random field, float64, shape (h, w)."""
    noise = torch.randn((h, w), generator=_gen(seed), dtype=torch.float64).to(device)
    return _blur_fft(noise, sigma) if fft else _blur_separable(noise, sigma)


def grf_nd(seed: int, shape, sigma: float, device="cpu") -> torch.Tensor:
    noise = torch.randn(tuple(shape), generator=_gen(seed), dtype=torch.float64).to(device)
    if max(shape) >= 512:
        return _blur_fft(noise, sigma)
    return _blur_separable(noise, sigma)


def uniform_thresholds(lo: float, hi: float, L: int, device="cpu") -> torch.Tensor:
    lo, hi = float(lo), float(hi)
    if L == 1:
        t = np.array([hi], dtype=np.float64)
    else:
        t = lo + (hi - lo) * np.arange(L, dtype=np.float64) / (L - 1)
    t32 = t.astype(np.float32)
    t32[0] = np.float32(lo)
    t32[-1] = np.float32(hi)
    return torch.from_numpy(t32).to(device)


def blobs_3d(seed: int, n: int = 512, nblobs: int = 2000, noise_sigma: float = 0.05, device="cpu",
             r_range=(3.0, 12.0), a_range=(0.5, 1.5)) -> torch.Tensor:
    """Gaussian-blob density plus iid noise, float32, shape (n, n, n)."""
    g = _gen(seed)
    centres = torch.rand((nblobs, 3), generator=g, dtype=torch.float64) * n
    radii = r_range[0] + (r_range[1] - r_range[0]) * torch.rand(nblobs, generator=g, dtype=torch.float64)
    amps = a_range[0] + (a_range[1] - a_range[0]) * torch.rand(nblobs, generator=g, dtype=torch.float64)
    field = torch.zeros((n, n, n), dtype=torch.float32, device=device)
    for i in range(nblobs):
        c = centres[i].tolist()
        r = float(radii[i])
        a = float(amps[i])
        lo = [max(0, int(math.floor(ci - 4 * r))) for ci in c]
        hi = [min(n, int(math.ceil(ci + 4 * r)) + 1) for ci in c]
        if any(h <= l for l, h in zip(lo, hi)):
            continue
        zz = torch.arange(lo[0], hi[0], device=device, dtype=torch.float32) - c[0]
        yy = torch.arange(lo[1], hi[1], device=device, dtype=torch.float32) - c[1]
        xx = torch.arange(lo[2], hi[2], device=device, dtype=torch.float32) - c[2]
        d2 = zz.view(-1, 1, 1) ** 2 + yy.view(1, -1, 1) ** 2 + xx.view(1, 1, -1) ** 2
        field[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] += a * torch.exp(-d2 / (2 * r * r))
    noise = torch.randn((n, n, n), generator=g, dtype=torch.float32).to(device)
    field += noise_sigma * noise
    return field


# ----------------------------------------------------------- named workloads

def config1(device="cpu"):
    """256 x 256 uint8 smoothed GRF (sigma 4), 256 identity levels."""
    f = quantize_u8(grf_2d(1, 256, 256, 4.0))
    return f.to(device)


def config2(device="cpu", n: int = 16384):
    """n x n smoothed GRF (sigma 16, periodic FFT): the uint8 quantisation and
    the float32 copy of the same field with 1024 uniform thresholds."""
    f = grf_2d(2, n, n, 16.0, device=device, fft=True)
    u8 = quantize_u8(f)
    f32 = f.to(torch.float32)
    thr = uniform_thresholds(f32.min().item(), f32.max().item(), 1024, device=device)
    return u8, f32, thr


def config3(device="cpu", n: int = 512, nblobs: int = 2000, L: int = 1024):
    """n^3 float32 Gaussian-blob density + noise with L uniform thresholds."""
    f = blobs_3d(3, n=n, nblobs=nblobs, device=device)
    thr = uniform_thresholds(f.min().item(), f.max().item(), L, device=device)
    return f, thr


def request_stream(seed: int = 5, n: int = 4096, rho_rate: float = 1000.0, max_2d: int = 4096,
                   max_3d: int = 512):
    """Request descriptors of the served workload (no field data): list of
    dicts {ndim, side, dtype, L, sigma, seed, arrival_s}."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(n):
        t += rng.exponential(1.0 / rho_rate)
        if rng.random() < 0.7:
            side = int(math.floor(math.exp(rng.uniform(math.log(64), math.log(max_2d)))))
            reqs.append(dict(ndim=2, side=side, dtype="u8", L=256, sigma=float(rng.uniform(2, 10)),
                             seed=int(rng.integers(1 << 31)), arrival_s=t))
        else:
            side = int(math.floor(math.exp(rng.uniform(math.log(32), math.log(max_3d)))))
            reqs.append(dict(ndim=3, side=side, dtype="f32", L=int(rng.integers(64, 1025)),
                             sigma=float(rng.uniform(2, 10)), seed=int(rng.integers(1 << 31)), arrival_s=t))
    return reqs


def _blur_fft32(f: torch.Tensor, sigma: float) -> torch.Tensor:
    """Periodic Gaussian blur by a real FFT in float32 (device fields)."""
    dims = tuple(range(f.dim()))
    freqs = [torch.fft.fftfreq(n, device=f.device) for n in f.shape[:-1]]
    freqs.append(torch.fft.rfftfreq(f.shape[-1], device=f.device))
    c = -2 * (math.pi ** 2) * (sigma ** 2)
    H = None
    for a, w in enumerate(freqs):   # separable: product of 1D factors
        shp = [1] * f.dim()
        shp[a] = -1
        h = torch.exp(c * w * w).view(shp)
        H = h if H is None else H * h
    return torch.fft.irfftn(torch.fft.rfftn(f, dim=dims) * H, s=f.shape, dim=dims)


def request_field_device(req: dict, device="cuda"):
    """One request's field generated on the device: float32 N(0,1) noise from
    a device generator seeded with the request's seed on the power-of-two
    box that holds the field, smoothed by a periodic Gaussian (sigma) through
    a float32 FFT and cropped to the field (so a stream of uneven sizes needs
    only a few FFT plans); 2D fields are quantised to uint8, 3D fields get L
    uniform float32 thresholds over [min, max].  Same recipe as
    request_field, other random numbers (the device generator)."""
    g = torch.Generator(device=device)
    g.manual_seed(int(req["seed"]))
    side = req["side"]
    box = 1 << max(0, (side - 1).bit_length())
    f = _blur_fft32(torch.randn((box,) * req["ndim"], generator=g, dtype=torch.float32, device=device), req["sigma"])
    f = f[(slice(0, side),) * req["ndim"]].contiguous()
    if req["ndim"] == 2:
        return quantize_u8(f), None
    thr = uniform_thresholds(f.min().item(), f.max().item(), req["L"], device=device)
    return f.contiguous(), thr


def request_field(req: dict, device="cpu"):
    """Materialise one request's field (and thresholds for float32 fields)."""
    if req["ndim"] == 2:
        f = grf_2d(req["seed"], req["side"], req["side"], req["sigma"], device=device,
                   fft=req["side"] >= 1024)
        return quantize_u8(f), None
    f = grf_nd(req["seed"], (req["side"],) * 3, req["sigma"], device=device).to(torch.float32)
    thr = uniform_thresholds(f.min().item(), f.max().item(), req["L"], device=device)
    return f, thr
