"""Sigma schedule, EDM preconditioning and the blend weight window (oracle).

Test infrastructure (see the package header).

* Schedule.  The paper fixes no schedule for the blended steps; the synthetic
  stacks use "a fixed sigma schedule from 80 to 0.02", read here as the EDM
  rho-schedule (the paper's backbone is EDM2, Sec. 5.3):
      sigma_k = (smax^(1/rho) + k/(K-1) (smin^(1/rho) - smax^(1/rho)))^rho,
  k = 0..K-1 (K = 1 gives sigma_0 = smax).
* Preconditioning (EDM): D(x; sigma) = c_skip x + c_out F(c_in x) with
  c_skip = sd^2/(sigma^2+sd^2), c_out = sigma sd / sqrt(sigma^2+sd^2),
  c_in = 1/sqrt(sigma^2+sd^2), sd = sigma_data.
* Weight window (Sec. 6): separable, linear, 1 at the centre and eps at the
  boundary: w1(u) = 1 - (1-eps)|u - c|/c with c = (H-1)/2, W = w1 (x) w1.

Pins: the schedule's end points and monotonicity; c_skip + c_out^2/sd^2 = 1
(EDM identity) ; the weight window's end and centre values and the closed form
of the per-axis weight sum for H = 2s, B1 = 2 - (1-eps) s/(s-1/2)
(tests/test_oracle_sampler.py).
"""
from __future__ import annotations

import math

import numpy as np


def sigmas(steps: int, sigma_max: float, sigma_min: float, rho: float) -> np.ndarray:
    if steps < 1:
        raise ValueError("steps >= 1")
    if steps == 1:
        return np.array([float(sigma_max)])
    a = sigma_max ** (1.0 / rho)
    b = sigma_min ** (1.0 / rho)
    k = np.arange(steps, dtype=np.float64)
    return (a + k / (steps - 1) * (b - a)) ** rho


def edm_coeffs(sigma: float, sigma_data: float):
    s2 = sigma * sigma + sigma_data * sigma_data
    c_skip = sigma_data * sigma_data / s2
    c_out = sigma * sigma_data / math.sqrt(s2)
    c_in = 1.0 / math.sqrt(s2)
    return c_skip, c_out, c_in


def weight_1d(size: int, eps: float) -> np.ndarray:
    c = (size - 1) / 2.0
    u = np.arange(size, dtype=np.float64)
    return 1.0 - (1.0 - eps) * np.abs(u - c) / c


def weight_2d(size: int, eps: float) -> np.ndarray:
    w = weight_1d(size, eps)
    return np.outer(w, w)
