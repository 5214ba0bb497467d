"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the sampling method itself.  It only
produces *inputs*: model-stack descriptions (plain data), random-init
network weights, query workloads and the fBm low-band fixture.  Both the
CPU oracle and the CUDA path receive what it makes; neither side's
computation lives here.

Weights follow the initialisation rule of the synthetic stacks: every
tensor is drawn N(0, 1) * 0.5 / sqrt(fan_in), tensor after tensor in the
declaration order the caller passes in, from one NumPy PCG64 stream per
(weight_seed, level) pair.  The paper ships no weights (its networks are
trained, Table "Hyperparameters", App. F), so random-init stacks of the
paper's shapes stand in for them.
"""
from __future__ import annotations

import copy
import math
from typing import Iterable, Sequence

import numpy as np

# ---------------------------------------------------------------------------
# Model-stack descriptions (data only).  Field names mirror idf_level_desc /
# idf_model_stack in include/idf.h.
# ---------------------------------------------------------------------------

_LEVEL_DEFAULTS = dict(
    levels=2, channels=(16, 16), in_ch=1, out_ch=1, gn_groups=4,
    attn_at_bottom=0, attn_heads=0,
    window=32, stride=16, offset=0, steps=4,
    sigma_max=80.0, sigma_min=0.02, rho=7.0, sigma_data=0.5,
    scale_to_parent=0, test_denoiser=0,
)

_STACK_DEFAULTS = dict(
    laplacian=0, lap_factor=8, lap_blur_sigma=5.0, lap_radius=15,
    low_mu=0.0, low_scale=50.0, res_scale=1.5, blend_eps=1e-3,
)


def level(**kw) -> dict:
    d = dict(_LEVEL_DEFAULTS)
    d.update(kw)
    d["channels"] = tuple(int(c) for c in d["channels"])
    return d


def stack(levels: Sequence[dict], **kw) -> dict:
    d = dict(_STACK_DEFAULTS)
    d.update(kw)
    d["level"] = [dict(l) for l in levels]
    return d


def config1_stack(test_denoiser: int = 0) -> dict:
    """Single level, 2-level UNet of 16 channels, 32x32 windows at stride 16, 4 steps."""
    return stack([level(levels=2, channels=(16, 16), in_ch=1, out_ch=1,
                        window=32, stride=16, steps=4,
                        test_denoiser=test_denoiser)])


def config2_stack(steps: int = 20, test_denoiser: int = 0) -> dict:
    """Two-level hierarchy: coarse UNet (64/128/128) at 1/8 resolution conditions
    a fine UNet (64/128/256/256, self-attention at the bottom); 128x128 windows
    at stride 64; Laplacian elevation decode (low band at 1/8, residual at 1)."""
    coarse = level(levels=3, channels=(64, 128, 128), in_ch=1, out_ch=1,
                   window=128, stride=64, steps=steps, test_denoiser=test_denoiser)
    fine = level(levels=4, channels=(64, 128, 256, 256), in_ch=2, out_ch=1,
                 attn_at_bottom=1, attn_heads=4,
                 window=128, stride=64, steps=steps, scale_to_parent=8,
                 test_denoiser=test_denoiser)
    return stack([coarse, fine], laplacian=1)


def small_hier_stack(steps: int = 3, window: int = 32, stride: int = 16,
                     coarse_channels=(16, 16), fine_channels=(16, 32),
                     attn: bool = True, test_denoiser: int = 0) -> dict:
    """A reduced two-level stack with the same structure as the 2-level
    hierarchy (attention at the fine bottom, Laplacian decode) but small
    enough for the FP64 oracle to sample whole cones in seconds."""
    coarse = level(levels=len(coarse_channels), channels=coarse_channels, in_ch=1,
                   out_ch=1, window=window, stride=stride, steps=steps,
                   test_denoiser=test_denoiser)
    fine = level(levels=len(fine_channels), channels=fine_channels, in_ch=2, out_ch=1,
                 attn_at_bottom=1 if attn else 0, attn_heads=2 if attn else 0,
                 window=window, stride=stride, steps=steps, scale_to_parent=8,
                 test_denoiser=test_denoiser)
    return stack([coarse, fine], laplacian=1)


def config4_stack(fixture: np.ndarray, steps: int = 4, test_denoiser: int = 0) -> dict:
    """Earth-scale single-level stack: the 16-channel config-1 UNet generates
    the residual band H (32x32 windows at stride 16) and the low band is the
    given periodic fixture of signed-sqrt values (low_mu 0, low_scale 1), so
    that the decoded metres span the fixture's range; Laplacian factor 8,
    blur sigma 5, radius 15, residual scale 1.5."""
    fine = level(levels=2, channels=(16, 16), in_ch=1, out_ch=1, window=32, stride=16, steps=steps,
                 test_denoiser=test_denoiser)
    st = stack([fine], laplacian=1, low_mu=0.0, low_scale=1.0, res_scale=1.5)
    st["low_band_fixture"] = np.ascontiguousarray(fixture, dtype=np.float32)
    return st


def student_level(window: int = 128, stride: int = 64) -> dict:
    """The half-width 2-step student: 4 levels of 32/64/128/128 channels,
    128x128 windows at stride 64, sigma 80 then 0.35."""
    return level(levels=4, channels=(32, 64, 128, 128), in_ch=1, out_ch=1, window=window,
                 stride=stride, steps=2, sigma_max=80.0, sigma_min=0.35)


def with_steps(st: dict, steps: int) -> dict:
    st = copy.deepcopy(st)
    for l in st["level"]:
        l["steps"] = int(steps)
    return st


# ---------------------------------------------------------------------------
# Weights
# ---------------------------------------------------------------------------

def weights(shapes: Iterable[Sequence[int]], weight_seed: int = 0,
            level_index: int = 0) -> np.ndarray:
    """Flat float32 weight vector for the tensor shapes given, in order.

    Each shape is (C_out, C_in, kh, kw); fan_in = C_in*kh*kw.
    """
    rng = np.random.Generator(np.random.PCG64([int(weight_seed), int(level_index)]))
    parts = []
    for shp in shapes:
        shp = tuple(int(s) for s in shp)
        fan_in = int(np.prod(shp[1:]))
        w = rng.standard_normal(shp) * (0.5 / math.sqrt(fan_in))
        parts.append(w.astype(np.float32).ravel())
    if not parts:
        return np.zeros(0, np.float32)
    return np.concatenate(parts)


def guide_weights(main: np.ndarray, shapes: Iterable[Sequence[int]], level_index: int = 0,
                  mix: float = 0.3) -> np.ndarray:
    """Weights of an AutoGuidance guide network for a synthetic main network:
    a degraded copy, (1 - mix) main + mix (an independent draw of the same
    shapes, weight seed 1).  The paper's guides are smaller or less trained
    versions of the main model (Table "Hyperparameters"); none exist here."""
    other = weights(shapes, 1, level_index)
    return ((1.0 - mix) * np.asarray(main, dtype=np.float64) + mix * other).astype(np.float32)


def conditioned(st: dict, dim: int = 4, z=(0.5, -1.0, 0.25, 2.0), amp: float = 0.3,
                guidance: float = 0.0, levels=None) -> dict:
    """A copy of a stack whose levels (all, or the indices given) take a
    per-window conditioning vector of `dim` values around z (and, with
    guidance != 0, an AutoGuidance guide network)."""
    st = copy.deepcopy(st)
    for i, lv in enumerate(st["level"]):
        if levels is None or i in levels:
            lv["cond_dim"] = int(dim)
            lv["cond_z"] = tuple(float(v) for v in z[:dim])
            lv["cond_amp"] = float(amp)
            lv["guidance"] = float(guidance)
    return st


# ---------------------------------------------------------------------------
# Window inputs for per-window network tests
# ---------------------------------------------------------------------------

def window_batch(batch: int, channels: int, size: int, seed: int = 0,
                 scale: float = 1.0) -> np.ndarray:
    """(B, C, H, W) float32 standard-normal window inputs."""
    rng = np.random.Generator(np.random.PCG64([int(seed), 7]))
    return (rng.standard_normal((batch, channels, size, size)) * scale).astype(np.float32)


# ---------------------------------------------------------------------------
# Random-access query workload (batched serving)
# ---------------------------------------------------------------------------

def random_queries(n: int = 1024, seed: int = 0, lo: int = 64, hi: int = 2048,
                   extent: float = 1e6, p_overlap: float = 0.3):
    """Queries (x0, y0, w, h): sides log-uniform in [lo, hi], centres uniform in
    +-extent, with probability p_overlap (after the first) centred on an
    earlier query's centre shifted by up to half of its size."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    out = []
    centres = []
    for q in range(n):
        w = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        h = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        if q > 0 and rng.uniform() < p_overlap:
            j = int(rng.integers(0, q))
            cx, cy, pw, ph = centres[j]
            cx = cx + rng.uniform(-0.5, 0.5) * pw
            cy = cy + rng.uniform(-0.5, 0.5) * ph
        else:
            cx = rng.uniform(-extent, extent)
            cy = rng.uniform(-extent, extent)
        x0 = int(math.floor(cx - w / 2))
        y0 = int(math.floor(cy - h / 2))
        centres.append((cx, cy, w, h))
        out.append((x0, y0, w, h))
    return out


# ---------------------------------------------------------------------------
# fBm low-band fixture
# ---------------------------------------------------------------------------

def fbm_lowband(n: int = 2048, beta: float = 2.2, seed: int = 0,
                lo_m: float = -11000.0, hi_m: float = 9000.0) -> np.ndarray:
    """Periodic n x n spectral fBm (amplitude ~ f^(-beta/2), random phases),
    affinely mapped so that its signed-sqrt image spans the signed square roots
    of [lo_m, hi_m].  Returned as float32 signed-sqrt values (low-res grid)."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    fy = np.fft.fftfreq(n)[:, None]
    fx = np.fft.rfftfreq(n)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    f[0, 0] = 1.0
    amp = f ** (-beta / 2.0)
    amp[0, 0] = 0.0
    phase = rng.uniform(0.0, 2.0 * np.pi, size=amp.shape)
    spec = amp * np.exp(1j * phase)
    field = np.fft.irfft2(spec, s=(n, n))
    lo_s = -math.sqrt(-lo_m) if lo_m < 0 else math.sqrt(lo_m)
    hi_s = math.sqrt(hi_m) if hi_m > 0 else -math.sqrt(-hi_m)
    fmin, fmax = field.min(), field.max()
    field = lo_s + (field - fmin) * (hi_s - lo_s) / (fmax - fmin)
    return field.astype(np.float32)


# ---------------------------------------------------------------------------
# Voxel volumes (sampling on Z^3)
# ---------------------------------------------------------------------------

def volume_desc(test_denoiser: int = 0, channels: int = 8, window: int = 16, stride: int = 8,
                steps: int = 3) -> dict:
    """A volume level: 16^3 windows at stride 8, 3 steps from 80 to 0.02, and
    (test_denoiser 0) the small 3-D network of 8 hidden channels, GroupNorm(4)."""
    return dict(window=window, stride=stride, steps=steps, sigma_max=80.0, sigma_min=0.02, rho=7.0,
                sigma_data=0.5, blend_eps=1e-3, channels=channels, groups=4, test_denoiser=test_denoiser)


def volume_weights(desc: dict, weight_seed: int = 0) -> np.ndarray:
    """Weights of the 3-D network (conv1 (C, 1, 3, 3, 3), conv2 (1, C, 3, 3, 3))."""
    C = int(desc["channels"])
    return weights([(C, 1, 3, 3, 3), (1, C, 3, 3, 3)], weight_seed, 100)
