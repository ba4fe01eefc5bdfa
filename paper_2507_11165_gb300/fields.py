"""Seeded synthetic float32 fields and request streams.

These stand in for the paper's datasets (Sec. 6.1.3, Table 3: CESM-ATM
1800x3600, JHTDB / Nyx 512^3, Miranda, QMCPack, RTM), which are not available
here.  Every generator is a pure function of its seed; it holds none of the
compressor's arithmetic and is the only module shared by the CUDA path's tests
and the CPU oracle.  Fields are synthesised in float64 and rounded to float32.

Recipes (sizes are those of the workloads they stand in for):

* :func:`bumps_field` -- 16 Gaussian bumps (amplitude U[-1,1], width U[2,12]
  cells, centres uniform in the box) + 3 sinusoid modes (integer wave-vector
  components U{1..4} per axis, amplitude U[0.1,0.5], phase U[0,2pi)) +
  N(0, 1e-3) noise.  Default 64^3.
* :func:`lognormal_grf` -- Gaussian random field with power spectrum
  P(k) ~ k^-3 (P(0) = 0), FFT-synthesised from white noise, scaled to unit
  variance and exponentiated (a log-normal "density").  Default 512^3.
* :func:`fronts_2d` -- 6 low-wave-number sinusoid modes (|k| <= 6) + 5 tanh
  fronts (random orientation and offset, width U[2,10] cells, amplitude
  U[0.5,2]) + N(0, 1e-4) noise.  Default 1800 x 3600.
* :func:`stratified_3d` -- exp(-z/25) x (1 + 0.2 T), T a unit-variance 2D
  horizontal field with a k^-5/3 spectrum drawn independently per level z.
  Default 100 x 500 x 500.
* :func:`batch_fields` -- 256 fields, each side log-uniform in [32,256],
  alternating the bump and log-normal recipes, rel eb from {1e-2,1e-3,1e-4}.
* :func:`request_stream` -- Poisson arrivals (mean 200/s), half compress and
  half decompress of an earlier result, cubic sides log-uniform in
  [64,512], rel eb from {1e-2,1e-3,1e-4,1e-5}.
"""
from __future__ import annotations

import math
import os

import numpy as np

try:  # multithreaded FFT when scipy is present
    import scipy.fft as _sfft

    def _rfftn(a, axes=None):
        return _sfft.rfftn(a, axes=axes, workers=os.cpu_count())

    def _irfftn(a, s, axes=None):
        return _sfft.irfftn(a, s=s, axes=axes, workers=os.cpu_count())
except ImportError:  # pragma: no cover
    def _rfftn(a, axes=None):
        return np.fft.rfftn(a, axes=axes)

    def _irfftn(a, s, axes=None):
        return np.fft.irfftn(a, s=s, axes=axes)


def _grid_axes(shape):
    return [np.arange(n, dtype=np.float64) for n in shape]


def bumps_field(shape=(64, 64, 64), seed=0, n_bumps=16, n_modes=3, noise=1e-3):
    """Gaussian bumps + sinusoid modes + white noise (float32, C order)."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    axes = _grid_axes(shape)
    f = np.zeros(shape, dtype=np.float64)
    for _ in range(n_bumps):
        amp = rng.uniform(-1.0, 1.0)
        sigma = rng.uniform(2.0, 12.0)
        centre = [rng.uniform(0.0, n) for n in shape]
        g = amp
        for d in range(nd):  # separable: product of 1D Gaussians
            prof = np.exp(-0.5 * ((axes[d] - centre[d]) / sigma) ** 2)
            g = np.multiply.outer(g, prof) if d else amp * prof
        f += g
    for _ in range(n_modes):
        kv = rng.integers(1, 5, size=nd)
        amp = rng.uniform(0.1, 0.5)
        phase = rng.uniform(0.0, 2.0 * math.pi)
        z = np.exp(1j * phase)
        for d in range(nd):
            e = np.exp(1j * 2.0 * math.pi * kv[d] * axes[d] / shape[d])
            z = np.multiply.outer(z, e) if d else z * e
        f += amp * np.imag(z)
    f += rng.normal(0.0, noise, size=shape)
    return np.ascontiguousarray(f, dtype=np.float32)


def _spectral_field(shape, rng, slope, axes=None):
    """Real Gaussian field with P(k) ~ k^slope over ``axes`` (all by default), unit variance."""
    shape = tuple(int(s) for s in shape)
    axes = tuple(range(len(shape))) if axes is None else tuple(axes)
    w = rng.standard_normal(size=shape)
    W = _rfftn(w, axes=axes)
    del w
    k2 = None
    for j, ax in enumerate(axes):
        n = shape[ax]
        kk = (np.fft.rfftfreq(n) if j == len(axes) - 1 else np.fft.fftfreq(n)) * n
        bshape = [1] * len(shape)
        bshape[ax] = kk.size
        term = (kk ** 2).reshape(bshape)
        k2 = term if k2 is None else k2 + term
    with np.errstate(divide="ignore"):
        amp = np.where(k2 > 0, k2 ** (slope / 4.0), 0.0)  # sqrt(P) = k^(slope/2)
    W *= amp
    del amp, k2
    g = _irfftn(W, s=[shape[a] for a in axes], axes=axes)
    del W
    # unit variance over the transformed axes
    red = tuple(axes)
    g -= g.mean(axis=red, keepdims=True)
    sd = g.std(axis=red, keepdims=True)
    g /= np.where(sd > 0, sd, 1.0)
    return g


def lognormal_grf(shape=(512, 512, 512), seed=1, slope=-3.0):
    """exp(g), g a unit-variance Gaussian random field with P(k) ~ k^slope."""
    rng = np.random.default_rng(seed)
    g = _spectral_field(shape, rng, slope)
    np.exp(g, out=g)
    return np.ascontiguousarray(g, dtype=np.float32)


def fronts_2d(shape=(1800, 3600), seed=2, n_modes=6, n_fronts=5, noise=1e-4):
    """Smooth large-scale modes + sharp tanh fronts + white noise (2D)."""
    rng = np.random.default_rng(seed)
    ny, nx = (int(s) for s in shape)
    y = np.arange(ny, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    f = np.zeros((ny, nx), dtype=np.float64)
    for _ in range(n_modes):
        ky = rng.integers(0, 7)
        kx = rng.integers(0, 7)
        if kx == 0 and ky == 0:
            kx = 1
        amp = rng.uniform(0.2, 1.0)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        f += amp * np.sin(2.0 * math.pi * (ky * y / ny + kx * x / nx) + ph)
    for _ in range(n_fronts):
        th = rng.uniform(0.0, math.pi)
        off = rng.uniform(0.2, 0.8)
        width = rng.uniform(2.0, 10.0)
        amp = rng.uniform(0.5, 2.0)
        dist = (x - off * nx) * math.cos(th) + (y - off * ny) * math.sin(th)
        f += amp * np.tanh(dist / width)
    f += rng.normal(0.0, noise, size=(ny, nx))
    return np.ascontiguousarray(f, dtype=np.float32)


def stratified_3d(shape=(100, 500, 500), seed=3, scale_height=25.0, turb=0.2):
    """Vertical exponential profile x (1 + 0.2 T), T with a k^-5/3 horizontal spectrum."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = (int(s) for s in shape)
    T = _spectral_field((nz, ny, nx), rng, -5.0 / 3.0, axes=(1, 2))
    prof = np.exp(-np.arange(nz, dtype=np.float64) / scale_height)[:, None, None]
    f = prof * (1.0 + turb * T)
    return np.ascontiguousarray(f, dtype=np.float32)


def batch_specs(n_fields=256, seed=4, lo=32, hi=256):
    """Shapes, recipes and rel error bounds of the batched workload."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n_fields):
        shape = tuple(int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(3))
        eb = float(rng.choice([1e-2, 1e-3, 1e-4]))
        specs.append(dict(shape=shape, eb=eb, kind="bumps" if i % 2 == 0 else "grf",
                          seed=int(rng.integers(0, 2 ** 31 - 1))))
    return specs


def make_field(spec):
    if spec["kind"] == "bumps":
        return bumps_field(spec["shape"], seed=spec["seed"])
    return lognormal_grf(spec["shape"], seed=spec["seed"])


def batch_fields(n_fields=256, seed=4, lo=32, hi=256):
    specs = batch_specs(n_fields, seed, lo, hi)
    return specs, [make_field(s) for s in specs]


def request_stream(n_requests=2000, rate=200.0, seed=5, lo=64, hi=512, n_sides=None):
    """Poisson request stream: list of dicts (t_arrival, op, side, eb, field)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        side = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        eb = float(rng.choice([1e-2, 1e-3, 1e-4, 1e-5]))
        op = "compress" if (i == 0 or rng.uniform() < 0.5) else "decompress"
        reqs.append(dict(id=i, t=t, op=op, side=side, eb=eb, seed=int(rng.integers(0, 2 ** 31 - 1))))
    return reqs
