"""InfiniteDiffusion sampling (oracle): lazy Alg. 1 and eager Eq. 1, FP64.

Test infrastructure (see the package header).

Indexing.  The paper counts steps down (J_T noise, J_0 result, query J_t from
J_{t+1}); this module counts up: J_0 = sigma_0 N(seed, level, 0, .) is the
paper's J_T, step k maps J_k to J_{k+1}, and J_K is the result (paper J_0).

One blended step (Sec. 3.1-3.3).  Each window i of step k applies Phi, one
sampler step of the window: with x = J_k[R_i],
    Phi_i = D(x; sigma_k) + sigma_{k+1} N(seed, level, k+1, R_i)   (k+1 < K)
    Phi_i = D(x; sigma_k)                                          (k+1 = K)
D the EDM-preconditioned denoiser (oracle.schedule).  The update is Eq. 2:
J_{k+1}[R] = (sum_{i in kappa(R)} U_i(W (x) Phi_i)) / (sum_{j in kappa(R)} U_j(W))
restricted to R, division by zero taken as zero (App. B).  Because the noise
is keyed on absolute coordinates, this equals blending D alone and adding the
noise once per pixel; the CUDA path uses that fused form.

* ``Level`` is Alg. 1 literally: per step, A and B are kept as per-window
  contributions (i, W (x) Phi_i) with the processed set P given by the keys
  present, an LRU per step of bounded capacity, and eviction that removes i
  from P (Sec. 3.3 "To keep storage bounded ...").  Contributions are summed
  in the canonical order of kappa (row index i, then column index j).
* ``eager_level`` is Eq. 1 (bounded MultiDiffusion): every window lying
  inside a canvas that holds the whole dependency cone, all steps dense.
* ``World`` chains levels as a DAG (App. C.3): the fine level's conditioning
  channel is the nearest x scale upsampling of the coarse level's result
  (Sec. 5.3, decoder conditioning), fetched lazily.

Blending only at selected noise levels (the T variants, Sec. 4 "Latency",
App. G): a level may group its K sampler steps into T rounds of m_1 + ... +
m_T = K steps (``round_steps``).  Within a round every window runs its m_r
steps on its own, x <- D(x; sigma_j) + sigma_{j+1} N(seed, level, j+1, .)
(noise keyed on absolute coordinates, the last step of the sampler without
noise), and Eq. 2 blends the windows' results only at the round's end.  The
lazy recursion, the cache and the cone then advance by rounds: J_r is the
blended state after round r.  One step per round (the default) is the
blend-every-step sampler above.

Conditioning and guidance (App. B "Seeds and initial noise", Sec. 5.3,
Table "Hyperparameters"): a level with cond_dim = D > 0 gives window i =
(row, column) the vector y_i = Lambda(z, i) = z + cond_amp G_d(i), where z
(cond_z) is the world's conditioning vector and G_d(i) the seed function's
standard normal N(seed, level, COND_STEP + d, column, row) at a step counter
no sampler step reaches; the network adds E y_i after its in-conv.  With
guidance w != 0 a guide network (the same architecture, its own weights)
runs beside the main one and Phi uses the AutoGuidance combination
F = F_guide + w (F_main - F_guide) (w = 1: the main network alone).

Pins: the two routes agree (Lemma 3); query-order and cache-size
independence (Thm 1); closed forms with the test denoisers; window counts of
Lemma 4 / Thm 2 (tests/test_oracle_sampler.py).
"""
from __future__ import annotations

from collections import OrderedDict

import numpy as np

from . import kappa as K_
from . import noise as N_
from . import schedule as S_
from . import unet as U_

COND_STEP = 0x7FFF0000  # step counter of the conditioning draws G_d(i) (+ d)


class _LevelCommon:
    def __init__(self, seed: int, lv: dict, level_index: int, weights=None,
                 blend_eps: float = 1e-3, parent=None, guide_weights=None):
        self.seed = int(seed)
        self.lv = dict(lv)
        self.level_index = int(level_index)
        self.H = int(lv["window"])
        self.s = int(lv["stride"])
        self.o = int(lv.get("offset", 0))
        self.K = int(lv["steps"])
        self.sig = S_.sigmas(self.K, lv["sigma_max"], lv["sigma_min"], lv["rho"])
        rs = lv.get("round_steps")
        self.round_steps = [1] * self.K if not rs else [int(v) for v in rs]
        if sum(self.round_steps) != self.K or min(self.round_steps) < 1:
            raise ValueError("round_steps must be positive and sum to steps")
        self.R = len(self.round_steps)
        self.round_start = [sum(self.round_steps[:r]) for r in range(self.R)]
        self.sd = float(lv["sigma_data"])
        self.W = S_.weight_2d(self.H, blend_eps)
        self.params = None
        self.guide = None
        if int(lv.get("test_denoiser", 0)) == 0:
            self.params = U_.unpack(lv, weights)
        self.w_guide = float(lv.get("guidance", 0.0))
        if self.w_guide != 0.0:
            self.guide = U_.unpack(lv, guide_weights)
        self.cond_dim = int(lv.get("cond_dim", 0))
        if self.cond_dim:
            self.cond_z = np.asarray(lv["cond_z"], dtype=np.float64)
            self.cond_amp = float(lv.get("cond_amp", 1.0))
        self.parent = parent
        self.scale = int(lv.get("scale_to_parent", 0))
        self.phi_calls = 0
        self.fmap = None      # optional xin -> F over a batch (oracle.parallel); same values

    def cond_vector(self, i: int, j: int) -> np.ndarray:
        """y_i = Lambda(z, i) for window (i, j)."""
        g = [float(N_.normal_region(self.seed, self.level_index, COND_STEP + d, j, i, 1, 1)[0, 0])
             for d in range(self.cond_dim)]
        return self.cond_z + self.cond_amp * np.array(g)

    def net(self, xin: np.ndarray, ys) -> np.ndarray:
        """F of a batch of window inputs, with conditioning and guidance."""
        def run(p):
            F = np.empty((len(xin), self.H, self.H))
            if self.fmap is not None and ys is None and p is self.params:
                F[:] = self.fmap(xin)
                return F
            bs = 64 if self.H <= 32 else 1
            for b0 in range(0, len(xin), bs):
                y = None if ys is None else ys[b0:b0 + bs]
                F[b0:b0 + bs] = U_.forward(self.lv, p, xin[b0:b0 + bs], y)[:, 0]
            return F
        F = run(self.params)
        if self.guide is not None:
            Fg = run(self.guide)
            F = Fg + self.w_guide * (F - Fg)
        return F

    def noise(self, step, y0, x0, h, w):
        return N_.normal_region(self.seed, self.level_index, step, x0, y0, w, h).astype(np.float64)

    def cond(self, y0, x0, h, w):
        """Nearest-neighbour upsampled parent result over the fine rect."""
        f = self.scale
        cy0, cx0 = y0 // f, x0 // f
        cy1, cx1 = (y0 + h - 1) // f, (x0 + w - 1) // f
        P = self.parent.final(cy0, cx0, cy1 - cy0 + 1, cx1 - cx0 + 1)
        ys = (np.arange(y0, y0 + h) // f) - cy0
        xs = (np.arange(x0, x0 + w) // f) - cx0
        return P[np.ix_(ys, xs)]

    def phi(self, k: int, xs: list, rects: list) -> list:
        """Phi of round k for windows with inputs xs (H x H each) at rects:
        the round's sampler steps, each D(x; sigma_j) + sigma_{j+1} N."""
        cond = None
        if int(self.lv["in_ch"]) == 2:
            cond = np.stack([self.cond(*r) for r in rects])[:, None]
        out = [np.asarray(x, dtype=np.float64) for x in xs]
        ys = None
        if self.cond_dim and self.params is not None:
            ys = np.stack([self.cond_vector((r[0] - self.o) // self.s, (r[1] - self.o) // self.s) for r in rects])
        j0 = self.round_start[k]
        for j in range(j0, j0 + self.round_steps[k]):
            c_skip, c_out, c_in = S_.edm_coeffs(self.sig[j], self.sd)
            chans = [np.stack(out)[:, None] * c_in]
            if cond is not None:
                chans.append(cond)
            xin = np.concatenate(chans, axis=1)
            if self.params is None:
                F = U_.forward(self.lv, None, xin)[:, 0]
            else:
                F = self.net(xin, ys)
            self.phi_calls += len(xs)
            nxt = []
            for x, r, f in zip(out, rects, F):
                d = c_skip * x + c_out * f
                if j + 1 < self.K:
                    d = d + self.sig[j + 1] * self.noise(j + 1, *r)
                nxt.append(d)
            out = nxt
        return out


class Level(_LevelCommon):
    """Lazy InfiniteDiffusion (Alg. 1) for one level of the stack."""

    def __init__(self, *a, capacity=None, **kw):
        super().__init__(*a, **kw)
        self.capacity = capacity          # per-round contribution LRU capacity (None = unbounded)
        self.contrib = [OrderedDict() for _ in range(self.R + 1)]  # round -> {(i,j): W (x) Phi}

    def clear(self):
        for c in self.contrib:
            c.clear()

    def J(self, k: int, y0: int, x0: int, h: int, w: int) -> np.ndarray:
        if k == 0:
            return self.sig[0] * self.noise(0, y0, x0, h, w)
        win = K_.kappa(y0, x0, h, w, self.H, self.s, self.o)
        store = self.contrib[k]
        todo = [i for i in win if i not in store]
        if todo:
            rects = [K_.window_rect(i, j, self.H, self.s, self.o) for (i, j) in todo]
            xs = [self.J(k - 1, *r) for r in rects]
            phis = self.phi(k - 1, xs, rects)
            for key, p in zip(todo, phis):
                store[key] = self.W * p
        A = np.zeros((h, w))
        B = np.zeros((h, w))
        for (i, j) in win:
            store.move_to_end((i, j))
            wy, wx, _, _ = K_.window_rect(i, j, self.H, self.s, self.o)
            ya, yb = max(y0, wy), min(y0 + h, wy + self.H)
            xa, xb = max(x0, wx), min(x0 + w, wx + self.H)
            A[ya - y0:yb - y0, xa - x0:xb - x0] += store[(i, j)][ya - wy:yb - wy, xa - wx:xb - wx]
            B[ya - y0:yb - y0, xa - x0:xb - x0] += self.W[ya - wy:yb - wy, xa - wx:xb - wx]
        if self.capacity is not None:
            while len(store) > self.capacity:
                store.popitem(last=False)     # evict (i, x_i): i leaves P_k
        out = np.zeros((h, w))
        nz = B != 0
        out[nz] = A[nz] / B[nz]
        return out

    def final(self, y0, x0, h, w):
        return self.J(self.R, y0, x0, h, w)


def cone_rects(lvl: _LevelCommon, y0, x0, h, w):
    """rects[k] = region of J_k (the state after round k) a cold query of the
    result touches."""
    rects = [None] * (lvl.R + 1)
    rects[lvl.R] = (y0, x0, h, w)
    for k in range(lvl.R, 0, -1):
        ry0, rx0, rh, rw = rects[k]
        ri = K_.kappa_1d(ry0, ry0 + rh, lvl.H, lvl.s, lvl.o)
        rj = K_.kappa_1d(rx0, rx0 + rw, lvl.H, lvl.s, lvl.o)
        rects[k - 1] = (ri[0] * lvl.s + lvl.o, rj[0] * lvl.s + lvl.o,
                        (ri[1] - ri[0]) * lvl.s + lvl.H, (rj[1] - rj[0]) * lvl.s + lvl.H)
    return rects


class EagerLevel(_LevelCommon):
    """Eq. 1 on a bounded canvas holding the cone of one region.

    Round k evaluates every window that covers a pixel of rects[k + 1] (the
    region of J_{k+1} the result depends on) and forms J_{k+1} there: each
    such pixel gets the sum over all windows that contain it, in the order
    (i, j) ascending, so it equals the dense form (``dense=True``: every
    window of rects[0] in every round) term for term; the dense form also
    computes pixels nothing reads."""

    def run(self, y0, x0, h, w, dense=False):
        rects = cone_rects(self, y0, x0, h, w)
        if not dense:
            return self._run_cone(rects, y0, x0, h, w)
        cy, cx, ch, cw = rects[0]
        J = self.sig[0] * self.noise(0, cy, cx, ch, cw)
        ni = (ch - self.H) // self.s + 1
        nj = (cw - self.H) // self.s + 1
        i0 = (cy - self.o) // self.s
        j0 = (cx - self.o) // self.s
        wins = [(i0 + a, j0 + b) for a in range(ni) for b in range(nj)]
        rr = [K_.window_rect(i, j, self.H, self.s, self.o) for (i, j) in wins]
        for k in range(self.R):
            xs = [J[r[0] - cy:r[0] - cy + self.H, r[1] - cx:r[1] - cx + self.H] for r in rr]
            phis = self.phi(k, xs, rr)
            A = np.zeros((ch, cw))
            B = np.zeros((ch, cw))
            for r, p in zip(rr, phis):
                A[r[0] - cy:r[0] - cy + self.H, r[1] - cx:r[1] - cx + self.H] += self.W * p
                B[r[0] - cy:r[0] - cy + self.H, r[1] - cx:r[1] - cx + self.H] += self.W
            J = np.zeros((ch, cw))
            nz = B != 0
            J[nz] = A[nz] / B[nz]
        self._canvas = (cy, cx, J)
        return J[y0 - cy:y0 - cy + h, x0 - cx:x0 - cx + w]

    def _run_cone(self, rects, y0, x0, h, w):
        H = self.H
        cy, cx, ch, cw = rects[0]
        J = self.sig[0] * self.noise(0, cy, cx, ch, cw)
        for k in range(self.R):
            ny, nx, nh, nw = rects[k + 1]
            wins = K_.kappa(ny, nx, nh, nw, H, self.s, self.o)
            rr = [K_.window_rect(i, j, H, self.s, self.o) for (i, j) in wins]
            xs = [J[r[0] - cy:r[0] - cy + H, r[1] - cx:r[1] - cx + H] for r in rr]
            phis = self.phi(k, xs, rr)
            A = np.zeros((nh, nw))
            B = np.zeros((nh, nw))
            for r, p in zip(rr, phis):
                # the part of window r inside rects[k + 1]
                ya, yb = max(r[0], ny), min(r[0] + H, ny + nh)
                xa, xb = max(r[1], nx), min(r[1] + H, nx + nw)
                wp = (self.W * p)[ya - r[0]:yb - r[0], xa - r[1]:xb - r[1]]
                A[ya - ny:yb - ny, xa - nx:xb - nx] += wp
                B[ya - ny:yb - ny, xa - nx:xb - nx] += self.W[ya - r[0]:yb - r[0], xa - r[1]:xb - r[1]]
            J = np.zeros((nh, nw))
            nz = B != 0
            J[nz] = A[nz] / B[nz]
            cy, cx, ch, cw = ny, nx, nh, nw
        self._canvas = (cy, cx, J)
        return J[y0 - cy:y0 - cy + h, x0 - cx:x0 - cx + w]

    def final(self, y0, x0, h, w):
        cy, cx, J = self._canvas
        assert y0 >= cy and x0 >= cx and y0 + h <= cy + J.shape[0] and x0 + w <= cx + J.shape[1]
        return J[y0 - cy:y0 - cy + h, x0 - cx:x0 - cx + w]


class World:
    """A model stack (coarse level first) with lazy levels and the Laplacian decode."""

    def __init__(self, seed: int, stack: dict, weights: list, capacity=None, guide_weights=None):
        self.stack = stack
        self.levels = []
        parent = None
        for li, lv in enumerate(stack["level"]):
            lvl = Level(seed, lv, li, weights=weights[li] if weights else None,
                        blend_eps=stack.get("blend_eps", 1e-3), parent=parent,
                        capacity=capacity,
                        guide_weights=guide_weights[li] if guide_weights else None)
            self.levels.append(lvl)
            parent = lvl

    def model(self, y0, x0, h, w):
        """Result J_K of the last level over the region (model units)."""
        return self.levels[-1].final(y0, x0, h, w)

    def metres(self, y0, x0, h, w):
        """Laplacian decode (Sec. 5.2, App. H) of the last level's residual
        band with the first level's low band, or, for a single level with a
        given low band (stack["low_band_fixture"], a periodic low-resolution
        array), with that array read periodically."""
        from . import laplacian as L_
        st = self.stack
        fine = self.levels[-1]
        fx = st.get("low_band_fixture")
        lfun = L_.periodic_lowband(fx) if fx is not None else self.levels[0].final
        return L_.decode_metres(lfun, fine.final, y0, x0, h, w,
                                factor=st["lap_factor"], blur_sigma=st["lap_blur_sigma"],
                                radius=st["lap_radius"], low_mu=st["low_mu"],
                                low_scale=st["low_scale"], res_scale=st["res_scale"])


def eager_world_model(seed: int, stack: dict, weights: list, y0, x0, h, w, dense=False):
    """Eq. 1 brute force for the last level's result over a region; for a
    two-level stack the coarse level runs eagerly over the canvas the fine
    cone's conditioning needs.  dense: every window of the canvas in every
    round (EagerLevel)."""
    lvls = stack["level"]
    eps = stack.get("blend_eps", 1e-3)
    if len(lvls) == 1:
        e = EagerLevel(seed, lvls[0], 0, weights=weights[0] if weights else None, blend_eps=eps)
        return e.run(y0, x0, h, w, dense=dense)
    fine_lv = lvls[1]
    fine = EagerLevel(seed, fine_lv, 1, weights=weights[1] if weights else None, blend_eps=eps)
    rects = cone_rects(fine, y0, x0, h, w)
    cy, cx, ch, cw = rects[0]
    f = int(fine_lv["scale_to_parent"])
    coarse = EagerLevel(seed, lvls[0], 0, weights=weights[0] if weights else None, blend_eps=eps)
    qy0, qx0 = cy // f, cx // f
    qy1, qx1 = (cy + ch - 1) // f, (cx + cw - 1) // f
    coarse.run(qy0, qx0, qy1 - qy0 + 1, qx1 - qx0 + 1, dense=dense)
    fine.parent = coarse
    return fine.run(y0, x0, h, w, dense=dense)


class EagerWorld:
    """Eq. 1 brute force for a model stack over one region, grown by the
    Laplacian decode's halo when metres are wanted (App. C.3 chaining: the
    coarse level runs eagerly over every coarse pixel that the fine cone's
    conditioning or the decode's low band reads).  ``fmap`` optionally
    supplies a batch evaluator of F per level (oracle.parallel)."""

    def __init__(self, seed: int, stack: dict, weights: list, y0, x0, h, w, *,
                 metres: bool = False, fmap=None):
        from . import laplacian as L_
        lvls = stack["level"]
        eps = stack.get("blend_eps", 1e-3)
        self.stack = stack
        mk = lambda li, parent=None: EagerLevel(seed, lvls[li], li,
                                                weights=weights[li] if weights else None,
                                                blend_eps=eps, parent=parent)
        rect = (y0, x0, h, w)
        lrect = None
        if metres:
            (ly0, lx0, lh, lw), rect = L_.decode_rects(y0, x0, h, w, factor=stack["lap_factor"],
                                                        radius=stack["lap_radius"])
            lrect = (ly0, lx0, lh, lw)
        self.fine = mk(len(lvls) - 1)
        self.coarse = None
        if len(lvls) == 2:
            f = int(lvls[1]["scale_to_parent"])
            cy, cx, ch, cw = cone_rects(self.fine, *rect)[0]
            qy0, qx0 = cy // f, cx // f
            qy1, qx1 = (cy + ch - 1) // f, (cx + cw - 1) // f
            if lrect is not None:
                qy0, qx0 = min(qy0, lrect[0]), min(qx0, lrect[1])
                qy1, qx1 = max(qy1, lrect[0] + lrect[2] - 1), max(qx1, lrect[1] + lrect[3] - 1)
            self.coarse = mk(0)
            if fmap is not None:
                self.coarse.fmap = fmap(0)
            self.coarse.run(qy0, qx0, qy1 - qy0 + 1, qx1 - qx0 + 1)
            self.fine.parent = self.coarse
        if fmap is not None:
            self.fine.fmap = fmap(len(lvls) - 1)
        self.fine.run(*rect)

    def model(self, y0, x0, h, w):
        return self.fine.final(y0, x0, h, w)

    def metres(self, y0, x0, h, w):
        from . import laplacian as L_
        st = self.stack
        fx = st.get("low_band_fixture")
        lfun = L_.periodic_lowband(fx) if fx is not None else self.coarse.final
        return L_.decode_metres(lfun, self.fine.final, y0, x0, h, w,
                                factor=st["lap_factor"], blur_sigma=st["lap_blur_sigma"],
                                radius=st["lap_radius"], low_mu=st["low_mu"],
                                low_scale=st["low_scale"], res_scale=st["res_scale"])
