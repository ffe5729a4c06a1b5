"""Seeded synthetic FP32 fields shaped like the paper's workloads.

This module holds input generators only (no compression arithmetic); both the
CUDA path and the CPU oracle read the arrays it returns. The paper's datasets
(SDRBench / Open-SciVis, Sec. 5.1) are not available, so these stand in:

* ``sinusoids``   - 1-D sum of 5 sinusoids plus Gaussian noise (smooth signal).
* ``grf``         - Gaussian random field with isotropic power spectrum k^-3
                    (smooth simulation-like field, Miranda/NYX stand-in).
* ``zero_slabs``  - a GRF + 280.0 with 30% of the z-planes set to exactly 0.0 in
                    contiguous slabs (large constant offset: exercises centring).
* ``particles``   - clustered particle x-coordinates in cell-sorted order, then
                    velocities ~ N(0, 300) (low smoothness, HACC stand-in).
* ``field_mix``   - many fields of log-uniform size and mixed class (batched path).

Generation is float64 then cast to float32. Large fields can be made on a CUDA
device through torch (``device="cuda"``); small ones use numpy on the host.
"""
from __future__ import annotations

import math

import numpy as np


def sinusoids(n: int = 1 << 20, seed: int = 0) -> np.ndarray:
    """x_i = sum_k a_k sin(2 pi i / P_k + phi_k) + N(0, (1e-3 R)^2), R = noiseless range."""
    rng = np.random.default_rng(seed)
    periods = np.exp(rng.uniform(math.log(64.0), math.log(65536.0), size=5))
    amps = rng.uniform(0.1, 1.0, size=5)
    phases = rng.uniform(0.0, 2.0 * math.pi, size=5)
    i = np.arange(n, dtype=np.float64)
    x = np.zeros(n, np.float64)
    for a, p, f in zip(amps, periods, phases):
        x += a * np.sin(2.0 * math.pi * i / p + f)
    R = float(x.max() - x.min()) if n else 0.0
    x += rng.normal(0.0, 1e-3 * R, size=n)
    return x.astype(np.float32)


def _grf_numpy(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(shape)
    axes = list(range(len(shape)))
    spec = np.fft.rfftn(white, axes=axes)
    ks = [np.fft.fftfreq(s) * s for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1]) * shape[-1]]
    grids = np.meshgrid(*ks, indexing="ij")
    k = np.sqrt(sum(g * g for g in grids))
    with np.errstate(divide="ignore"):
        amp = np.where(k > 0, k ** -1.5, 0.0)
    field = np.fft.irfftn(spec * amp, s=shape, axes=axes)
    sd = field.std()
    return (field / (sd if sd > 0 else 1.0)).astype(np.float32)


def _grf_torch(shape, seed: int, device: str):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    white = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
    spec = torch.fft.rfftn(white)
    del white
    amp = None
    for ax, s in enumerate(shape):
        if ax == len(shape) - 1:
            f = torch.fft.rfftfreq(s, device=device) * s
        else:
            f = torch.fft.fftfreq(s, device=device) * s
        view = [1] * len(shape)
        view[ax] = -1
        term = (f * f).reshape(view)
        amp = term if amp is None else amp + term
    amp = amp.sqrt_()
    amp = torch.where(amp > 0, amp.pow(-1.5), torch.zeros_like(amp))
    spec.mul_(amp)
    del amp
    field = torch.fft.irfftn(spec, s=shape)
    del spec
    field.div_(field.std())
    return field.contiguous()


def grf(shape=(512, 512, 512), seed: int = 1, device: str = "cpu"):
    """Gaussian random field, P(k) ~ k^-3: white N(0,1) -> rFFT -> x k^-3/2 (k=0 -> 0)
    -> irFFT -> unit standard deviation. numpy (float64) on the host, torch float32
    on a CUDA device."""
    shape = tuple(int(s) for s in shape)
    if device == "cpu":
        return _grf_numpy(shape, seed)
    return _grf_torch(shape, seed, device)


def _slab_offsets(nz: int, seed: int, nslabs: int = 3, frac: float = 0.3):
    rng = np.random.default_rng(seed + 1000)
    width = max(1, int(round(frac * nz / nslabs)))
    width = min(width, max(1, nz // nslabs))
    free = nz - nslabs * width
    cuts = np.sort(rng.integers(0, free + 1, size=nslabs))
    return [int(c) + j * width for j, c in enumerate(cuts)], width


def zero_slabs(shape=(512, 512, 512), seed: int = 1, device: str = "cpu", base=None):
    """The GRF + 280.0, with 3 contiguous slabs of z-planes (about 30% of voxels) set to
    exactly 0.0 at seeded non-overlapping offsets."""
    f = grf(shape, seed, device) if base is None else base
    starts, width = _slab_offsets(shape[0], seed)
    if device == "cpu":
        out = f.astype(np.float32) + np.float32(280.0)
        for z0 in starts:
            out[z0:z0 + width] = 0.0
        return out
    out = f + 280.0
    for z0 in starts:
        out[z0:z0 + width] = 0.0
    return out


def particles(n: int = 1 << 28, seed: int = 2, device: str = "cpu", ncenters: int = 10_000):
    """First n/2 values: x-coordinates of points drawn around ``ncenters`` uniform centres
    in [0,256)^3 with N(0, 0.5^2) per axis, wrapped mod 256 and stably sorted by cell key
    (floor z * 256 + floor y) * 256 + floor x. Last n - n/2 values: velocities N(0, 300^2)."""
    npos = n // 2
    nvel = n - npos
    if device == "cpu":
        rng = np.random.default_rng(seed)
        centres = rng.uniform(0.0, 256.0, size=(ncenters, 3))
        which = rng.integers(0, ncenters, size=npos)
        pts = np.mod(centres[which] + rng.normal(0.0, 0.5, size=(npos, 3)), 256.0)
        cell = np.floor(pts).astype(np.int64)
        key = (cell[:, 2] * 256 + cell[:, 1]) * 256 + cell[:, 0]
        order = np.argsort(key, kind="stable")
        xs = pts[order, 0]
        vel = rng.normal(0.0, 300.0, size=nvel)
        return np.concatenate([xs, vel]).astype(np.float32)
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    centres = torch.rand((ncenters, 3), generator=g, device=device, dtype=torch.float64) * 256.0
    which = torch.randint(0, ncenters, (npos,), generator=g, device=device)
    out = torch.empty(n, device=device, dtype=torch.float32)
    xs_all = None
    key = torch.zeros(npos, device=device, dtype=torch.int64)
    for ax in (2, 1, 0):  # z, y, x: build the cell key, keep x
        c = centres[:, ax][which] + torch.randn(npos, generator=g, device=device,
                                                dtype=torch.float64) * 0.5
        c = torch.remainder(c, 256.0)
        key = key * 256 + torch.floor(c).to(torch.int64)
        if ax == 0:
            xs_all = c
    _, order = torch.sort(key, stable=True)
    out[:npos] = xs_all[order].to(torch.float32)
    del key, order, xs_all
    out[npos:] = (torch.randn(nvel, generator=g, device=device, dtype=torch.float64) * 300.0
                  ).to(torch.float32)
    return out


def near_cubic_dims(n: int, ndim: int):
    """Near-cubic integer dims whose product is close to n (row-major, last fastest)."""
    if ndim == 1:
        return (max(1, n),)
    side = max(1, int(round(n ** (1.0 / ndim))))
    dims = [side] * (ndim - 1)
    last = max(1, int(round(n / side ** (ndim - 1))))
    return tuple(dims + [last])


def field_mix_specs(nfields: int = 512, seed: int = 3, min_bytes: int = 64 << 10,
                    max_bytes: int = 64 << 20):
    """Descriptors of the batched workload: log-uniform sizes, ndim in {1,2,3}, class
    smooth (40%) / particle-like (40%) / zero-heavy offset (20%), REL in {1e-2,1e-3,1e-4}."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(nfields):
        nbytes = math.exp(rng.uniform(math.log(min_bytes), math.log(max_bytes)))
        n = max(1, int(nbytes // 4))
        ndim = int(rng.integers(1, 4))
        dims = near_cubic_dims(n, ndim)
        u = rng.uniform()
        cls = "smooth" if u < 0.4 else ("particle" if u < 0.8 else "zero_heavy")
        rel = float(rng.choice([1e-2, 1e-3, 1e-4]))
        specs.append(dict(index=i, dims=dims, n=int(np.prod(dims)), cls=cls, rel=rel,
                          seed=seed * 100_000 + i))
    return specs


def make_field(spec, device: str = "cpu"):
    """One field of the batched mix, as a flat float32 array (numpy) or tensor (torch)."""
    dims, n, cls, sd = spec["dims"], spec["n"], spec["cls"], spec["seed"]
    if cls == "smooth":
        f = grf(dims, sd, device)
    elif cls == "particle":
        f = particles(n, sd, device, ncenters=max(16, n // 2048))
    else:
        f = zero_slabs(dims, sd, device)
    return f.reshape(-1)


# ----------------------------------------------------------------------------- serving mix

SERVING_POOL_SHAPE = (256, 512, 512)


def serving_pool(seed: int = 4, device: str = "cuda"):
    """The serving workload's source fields (flat float32 tensors on the device): a k^-3
    GRF, a particle-like array and the GRF's zero-slab/+280 variant, 2^26 elements each."""
    g = grf(SERVING_POOL_SHAPE, seed=seed, device=device)
    pool = [g.reshape(-1).contiguous(),
            particles(g.numel(), seed=seed, device=device),
            zero_slabs(SERVING_POOL_SHAPE, seed=seed, device=device, base=g).reshape(-1).contiguous()]
    return pool


def serving_windows(rng, pool_numels, count: int, min_elems: int = 4096,
                    max_elems: int = 64 << 20):
    """Request windows: (pool index, element offset, n, REL) with n log-uniform in
    [min_elems, max_elems] (16 KiB - 256 MiB of float32), rounded down to a multiple of 4 and
    to the field's size, at a uniformly drawn 16-byte-aligned offset; `rng` is a
    random.Random."""
    out = []
    for _ in range(count):
        k = rng.randrange(len(pool_numels))
        size = int(pool_numels[k])
        n = int(math.exp(rng.uniform(math.log(min_elems), math.log(max_elems))))
        n = max(4, min(n, size) // 4 * 4)
        off = rng.randrange(0, (size - n) // 4 + 1) * 4
        out.append((k, off, n, rng.choice([1e-2, 1e-3, 1e-4])))
    return out


def serving_trace(rng, pool_numels, count: int, nsources: int, dec_share: float = 0.4):
    """A request trace: each entry is ("compress", pool index, offset, n, REL) or
    ("decompress", source index), the latter with probability `dec_share` when there are
    `nsources` earlier streams to draw from."""
    rows = []
    for k, off, n, rel in serving_windows(rng, pool_numels, count):
        if nsources and rng.random() < dec_share:
            rows.append(("decompress", rng.randrange(nsources)))
        else:
            rows.append(("compress", k, off, n, rel))
    return rows
