"""Multi-GPU option (ii), prototyped on CPU with the oracle: the tiles of a
region are split between two ranks (gloo) at a stride-aligned column, at
every step and on the whole dependency cone.  Before each step a rank
receives from its neighbour the (window - stride)-wide strip of J_k beyond
the split, which the windows covering its own tiles read; it evaluates those
windows (the column of windows straddling the split is evaluated by both
ranks) and blends its tiles (Eq. 2).  One point-to-point exchange per step,
no all-reduce.  The stitched result must equal the single-process dense
computation (Eq. 1 on a canvas holding the cone), on the 16-channel UNet."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _level():
    # the 16-channel UNet: its 3x3 convolutions mix neighbouring pixels, so a
    # window's output near the split depends on the received strip (a
    # pointwise test denoiser would hide a wrong exchange)
    import synth
    from oracle import unet as OU
    lv = synth.level(levels=2, channels=(16, 16), window=32, stride=16, steps=4)
    return lv, synth.weights([sh for _, sh in OU.param_shapes(lv)], 0, 0)


def _halo_rank(rank, world, port, q, rect, xs):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import kappa as K_
        from oracle import sampler as OS
        lv, wts = _level()
        lvl = OS.EagerLevel(0, lv, 0, weights=wts)
        H, s = lvl.H, lvl.s
        halo = H - s
        cone = OS.cone_rects(lvl, *rect)          # cone[k] = (y, x, h, w) of J_k

        def owned(k):
            cy, cx, ch, cw = cone[k]
            return (cy, cx, ch, xs - cx) if rank == 0 else (cy, xs, ch, cx + cw - xs)

        oy, ox, oh, ow = owned(0)
        J = lvl.sig[0] * lvl.noise(0, oy, ox, oh, ow)
        for k in range(lvl.K):
            oy, ox, oh, ow = owned(k)
            # the one exchange of the step: the strip next to the split
            send = torch.from_numpy(np.ascontiguousarray(J[:, ow - halo:] if rank == 0 else J[:, :halo]))
            recv = torch.empty((oh, halo), dtype=torch.float64)
            req = dist.isend(send, 1 - rank)
            dist.recv(recv, 1 - rank)
            req.wait()
            if rank == 0:
                Jx, ex0 = np.concatenate([J, recv.numpy()], axis=1), ox
            else:
                Jx, ex0 = np.concatenate([recv.numpy(), J], axis=1), ox - halo
            ny, nx, nh, nw = owned(k + 1)
            ri = K_.kappa_1d(ny, ny + nh, H, s)
            rj = K_.kappa_1d(nx, nx + nw, H, s)
            rr = [K_.window_rect(i, j, H, s) for i in range(ri[0], ri[1] + 1) for j in range(rj[0], rj[1] + 1)]
            xin = [Jx[r[0] - oy:r[0] - oy + H, r[1] - ex0:r[1] - ex0 + H] for r in rr]
            for x in xin:
                assert x.shape == (H, H)          # every window input lies in owned + halo
            phis = lvl.phi(k, xin, rr)
            A = np.zeros((nh, nw))
            B = np.zeros((nh, nw))
            for r, p in zip(rr, phis):
                y0, y1 = max(r[0], ny), min(r[0] + H, ny + nh)
                x0, x1 = max(r[1], nx), min(r[1] + H, nx + nw)
                wsub = lvl.W[y0 - r[0]:y1 - r[0], x0 - r[1]:x1 - r[1]]
                A[y0 - ny:y1 - ny, x0 - nx:x1 - nx] += wsub * p[y0 - r[0]:y1 - r[0], x0 - r[1]:x1 - r[1]]
                B[y0 - ny:y1 - ny, x0 - nx:x1 - nx] += wsub
            J = np.zeros((nh, nw))
            nz = B != 0
            J[nz] = A[nz] / B[nz]
        q.put((rank, owned(lvl.K), J))
    finally:
        dist.destroy_process_group()


def test_two_ranks_halo_exchange_equals_dense():
    from oracle import sampler as OS
    rect = (0, -32, 48, 96)       # y0, x0, h, w
    xs = 16                       # split column, a multiple of the stride
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_halo_rank, args=(r, 2, port, q, rect, xs)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(2)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, o0, J0), (_, o1, J1) = res
    assert o0[1] == rect[1] and o0[1] + o0[3] == xs and o1[1] == xs and o1[1] + o1[3] == rect[1] + rect[3]
    got = np.concatenate([J0, J1], axis=1)
    lv, wts = _level()
    ref = OS.EagerLevel(0, lv, 0, weights=wts).run(*rect)
    assert got.shape == ref.shape
    assert np.allclose(got, ref, rtol=0, atol=1e-12)
