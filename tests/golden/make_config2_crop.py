"""Writes config2_crop_k20.npz: the FP64 oracle's result of the 2-level
stack (coarse UNet 64/128/128 at 1/8 resolution, fine UNet 64/128/256/256
with attention; 128-pixel windows at stride 64; 20 blended steps; world seed
0, weight seed 0) over the 256 x 256 crop at (x, y) = (1920, 1920), in model
units (the fine level's J_K), the coarse level's J_K over the low-band rect
the decode reads, and in metres (Laplacian decode, Sec. 5.2, App. H).

It calls only the oracle (Eq. 1 brute force on a canvas that holds the whole
dependency cone of the crop and of the decode's halo: about 18.3k fine and
16.2k coarse window evaluations, ~0.64 PFLOP in FP64) and the seeded input
generators.  Values are stored as float32 next to the FP64 sigma_out of
each; the tests compare at 2e-2 sigma_out, far above float32 storage
rounding.

    python tests/golden/make_config2_crop.py [processes]
    python tests/golden/make_config2_crop.py 7 -128 -128 256 256 config2_crop_k20_origin.npz
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import laplacian as OL  # noqa: E402
from oracle import parallel as OP  # noqa: E402
from oracle import sampler as OS  # noqa: E402
from oracle import unet as OU  # noqa: E402

CROP = (1920, 1920, 256, 256)   # x0, y0, w, h
STEPS = 20
SEED = 0


def main(processes: int, steps: int = STEPS, crop=CROP, out_name="config2_crop_k20.npz"):
    st = synth.config2_stack(steps=steps)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    x0, y0, w, h = crop
    pool = OP.PoolForward(st, wts, processes)
    t = time.time()
    try:
        ew = OS.EagerWorld(SEED, st, wts, y0, x0, h, w, metres=True, fmap=pool.fmap)
    finally:
        pool.close()
    model = ew.model(y0, x0, h, w)
    metres = ew.metres(y0, x0, h, w)
    (ly0, lx0, lh, lw), _ = OL.decode_rects(y0, x0, h, w, factor=st["lap_factor"], radius=st["lap_radius"])
    low = ew.coarse.final(ly0, lx0, lh, lw)
    calls = (ew.coarse.phi_calls, ew.fine.phi_calls)
    secs = time.time() - t
    np.savez_compressed(os.path.join(HERE, out_name), model=model.astype(np.float32),
                        metres=metres.astype(np.float32), sigma_model=float(model.std()),
                        sigma_metres=float(metres.std()), crop=np.array(crop, np.int64),
                        low=low.astype(np.float32), sigma_low=float(low.std()),
                        low_rect=np.array([lx0, ly0, lw, lh], np.int64),
                        steps=steps, seed=SEED, windows=np.array(calls, np.int64),
                        seconds=secs, processes=processes)
    print(f"windows coarse {calls[0]} fine {calls[1]}; {secs:.0f} s on {processes} processes; "
          f"sigma_out {model.std():.6f}, metres std {metres.std():.3f}")


if __name__ == "__main__":
    # make_config2_crop.py [processes] [x0 y0 w h out_name]
    a = sys.argv[1:]
    procs = int(a[0]) if a else os.cpu_count()
    if len(a) >= 6:
        main(procs, crop=(int(a[1]), int(a[2]), int(a[3]), int(a[4])), out_name=a[5])
    else:
        main(procs)
