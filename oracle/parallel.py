"""Worker-process evaluation of the window denoiser F (oracle), FP64.

Test infrastructure (see the package header).

Every window of a step is evaluated from J_k alone (Thm 3: the windows of a
step are one round, independent of each other), so F of a step's windows may
be computed in any order or in parallel without changing a value.  This
module only distributes calls of ``oracle.unet.forward`` over worker
processes (one BLAS thread each) for long one-off oracle runs; it adds no
arithmetic.  Workers are started with the ``spawn`` method, so a pool may be
created in a process that already uses a GPU.

Pins: a pooled evaluation equals the serial loop up to BLAS summation order
(1e-15 relative; tests/test_oracle_sampler.py).
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from . import unet as U_

_NETS: dict = {}


def _init(nets):
    for key, (lv, flat) in nets.items():
        _NETS[key] = (lv, U_.unpack(lv, flat))


def _run(args):
    key, x = args
    lv, p = _NETS[key]
    return U_.forward(lv, p, x)


class PoolForward:
    """F of the levels of a stack in ``processes`` worker processes.

    ``fmap(level_index)`` returns a callable xin (B, in_ch, H, H) -> F (B, H, H)
    for ``oracle.sampler`` levels (their ``fmap`` attribute)."""

    def __init__(self, stack: dict, weights: list, processes: int, chunk: int = 2):
        nets = {li: (dict(lv), np.asarray(weights[li], dtype=np.float32))
                for li, lv in enumerate(stack["level"]) if int(lv.get("test_denoiser", 0)) == 0}
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                                  "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(processes, initializer=_init, initargs=(nets,))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.chunk = int(chunk)

    def fmap(self, level_index: int):
        def f(xin):
            parts = self.pool.map(_run, [(level_index, xin[a:a + self.chunk])
                                         for a in range(0, len(xin), self.chunk)])
            return np.concatenate(parts)[:, 0]
        return f

    def close(self):
        self.pool.close()
        self.pool.join()
