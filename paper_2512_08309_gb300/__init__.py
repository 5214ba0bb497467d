"""GB300 implementation of InfiniteDiffusion sampling (arXiv 2512.08309).

A thin ctypes binding over libidf (include/idf.h): argument marshalling only,
every step of the sampling path runs in the library's CUDA kernels.  The
library is built in-tree by ``paper_2512_08309_gb300.build.build()``; if it
is missing, every call raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import json
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libidf.so")

IDF_OK, IDF_EINVAL, IDF_ENOMEM, IDF_ECUDA, IDF_ETIMEOUT, IDF_EMODEL, IDF_EDEVICE_CHECK, \
    IDF_EINTERNAL, IDF_EUNSUPPORTED = range(9)
STATUS_NAMES = ["IDF_OK", "IDF_EINVAL", "IDF_ENOMEM", "IDF_ECUDA", "IDF_ETIMEOUT", "IDF_EMODEL",
                "IDF_EDEVICE_CHECK", "IDF_EINTERNAL", "IDF_EUNSUPPORTED"]
IDF_FP32, IDF_BF16, IDF_FP8_E4M3, IDF_BF16X3, IDF_TF32 = 0, 1, 2, 3, 4
IDF_OUT_MODEL, IDF_OUT_METRES = 0, 1

PRECISIONS = {"fp32": IDF_FP32, "bf16": IDF_BF16, "fp8": IDF_FP8_E4M3, "bf16x3": IDF_BF16X3, "tf32": IDF_TF32}

# Every symbol include/idf.h declares.
EXPORTS = [
    "idf_world_create", "idf_world_query", "idf_world_query_device", "idf_world_query_batch",
    "idf_world_cache_clear", "idf_world_stats", "idf_world_last_error", "idf_world_destroy",
    "idf_world_store_open", "idf_world_store_close",
    "idf_debug_cone", "idf_debug_cache_keys", "idf_debug_set_status", "idf_noise_fill",
    "idf_model_param_count", "idf_model_param_shape",
    "idf_unet_forward", "idf_laplacian_decode", "idf_laplacian_halo", "idf_laplacian_decode_noalloc",
    "idf_student_create", "idf_student_loss_grad", "idf_student_adamw", "idf_student_zero_grad",
    "idf_student_read", "idf_student_write", "idf_student_last_error", "idf_student_destroy",
    "idf_volume_create", "idf_volume_query", "idf_volume_stats", "idf_volume_last_error", "idf_volume_destroy",
]


class IdfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


class idf_level_desc(C.Structure):
    _fields_ = [
        ("levels", C.c_int32), ("channels", C.POINTER(C.c_int32)),
        ("in_ch", C.c_int32), ("out_ch", C.c_int32), ("gn_groups", C.c_int32),
        ("attn_at_bottom", C.c_int32), ("attn_heads", C.c_int32),
        ("weights", C.POINTER(C.c_float)), ("n_weights", C.c_size_t),
        ("window", C.c_int32), ("stride", C.c_int32), ("offset", C.c_int32), ("steps", C.c_int32),
        ("sigma_max", C.c_double), ("sigma_min", C.c_double), ("rho", C.c_double),
        ("sigma_data", C.c_double),
        ("scale_to_parent", C.c_int32), ("test_denoiser", C.c_int32),
        ("round_steps", C.POINTER(C.c_int32)), ("n_rounds", C.c_int32),
        ("cond_dim", C.c_int32), ("cond_z", C.POINTER(C.c_float)), ("cond_amp", C.c_double),
        ("guidance", C.c_double), ("guide_weights", C.POINTER(C.c_float)), ("n_guide_weights", C.c_size_t),
    ]


class idf_model_stack(C.Structure):
    _fields_ = [
        ("n_levels", C.c_int32), ("level", C.POINTER(idf_level_desc)),
        ("laplacian", C.c_int32), ("lap_factor", C.c_int32), ("lap_blur_sigma", C.c_double),
        ("lap_radius", C.c_int32), ("low_mu", C.c_double), ("low_scale", C.c_double),
        ("res_scale", C.c_double), ("blend_eps", C.c_double),
        ("low_band_fixture", C.POINTER(C.c_float)), ("fixture_period", C.c_int64),
    ]


class idf_world_opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int32), ("cache_bytes", C.c_size_t), ("device", C.c_int32),
        ("workspace_bytes", C.c_size_t), ("max_batch", C.c_int32), ("profile", C.c_int32),
        ("device_wait_budget_cycles", C.c_uint64), ("autotune", C.c_int32), ("groupnorm_in_conv", C.c_int32),
        ("cuda_graphs", C.c_int32), ("cta_pairs", C.c_int32),
    ]


class idf_volume_desc(C.Structure):
    _fields_ = [
        ("window", C.c_int32), ("stride", C.c_int32), ("steps", C.c_int32),
        ("sigma_max", C.c_double), ("sigma_min", C.c_double), ("rho", C.c_double), ("sigma_data", C.c_double),
        ("blend_eps", C.c_double), ("channels", C.c_int32), ("groups", C.c_int32), ("test_denoiser", C.c_int32),
        ("weights", C.POINTER(C.c_float)), ("n_weights", C.c_size_t),
    ]


class idf_region(C.Structure):
    _fields_ = [("x0", C.c_int64), ("y0", C.c_int64), ("w", C.c_int32), ("h", C.c_int32),
                ("out_dev", C.c_void_p), ("pitch_elems", C.c_int64)]


_lib = None


def lib():
    """Load libidf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libidf is not built ({LIB_PATH} missing); run "
                           "paper_2512_08309_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_uint32
    fp = C.POINTER(C.c_float)
    sig = {
        "idf_world_create": ([u64, C.POINTER(idf_model_stack), C.POINTER(idf_world_opts), C.POINTER(vp)], i32),
        "idf_world_query": ([vp, i64, i64, i32, i32, i32, vp], i32),
        "idf_world_query_device": ([vp, i64, i64, i32, i32, i32, vp, i64, vp], i32),
        "idf_world_query_batch": ([vp, C.POINTER(idf_region), i32, i32, vp], i32),
        "idf_world_cache_clear": ([vp], i32),
        "idf_world_store_open": ([vp, C.c_char_p, i32], i32),
        "idf_world_store_close": ([vp], i32),
        "idf_world_stats": ([vp, C.c_char_p, C.c_size_t], i32),
        "idf_world_last_error": ([vp], C.c_char_p),
        "idf_world_destroy": ([vp], None),
        "idf_debug_cone": ([vp, i64, i64, i32, i32, i32, i32, C.POINTER(i64), i32, C.POINTER(i32)], i32),
        "idf_debug_cache_keys": ([vp, i32, i32, C.POINTER(i32), i32, C.POINTER(i32)], i32),
        "idf_debug_set_status": ([vp, i32, i32], i32),
        "idf_noise_fill": ([u64, u32, u32, i64, i64, i32, i32, vp, i64, vp], i32),
        "idf_model_param_count": ([C.POINTER(idf_level_desc), C.POINTER(i32), C.POINTER(C.c_size_t)], i32),
        "idf_model_param_shape": ([C.POINTER(idf_level_desc), i32, C.POINTER(i32)], i32),
        "idf_unet_forward": ([vp, i32, vp, i32, vp, vp], i32),
        "idf_laplacian_decode": ([C.POINTER(idf_model_stack), vp, i64, i64, i32, i32, i64, vp, i64, i64,
                                  i32, i32, i64, i64, i64, i32, i32, vp, i64, vp], i32),
        "idf_laplacian_halo": ([C.POINTER(idf_model_stack), i64, i64, i32, i32, C.POINTER(i64),
                                C.POINTER(i64)], i32),
        "idf_laplacian_decode_noalloc": ([C.POINTER(idf_model_stack), vp, i64, i64, i32, i32, i64, vp, i64,
                                          i64, i32, i32, i64, i64, i64, i32, i32, vp, i64, vp], i32),
        "idf_student_create": ([C.POINTER(idf_level_desc), i32, i32, C.POINTER(vp)], i32),
        "idf_student_loss_grad": ([vp, vp, vp, i32, C.c_double, C.POINTER(C.c_double), vp], i32),
        "idf_student_adamw": ([vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double], i32),
        "idf_student_zero_grad": ([vp], i32),
        "idf_student_read": ([vp, i32, C.POINTER(C.c_float), C.c_size_t], i32),
        "idf_student_write": ([vp, C.POINTER(C.c_float), C.c_size_t], i32),
        "idf_student_last_error": ([vp], C.c_char_p),
        "idf_student_destroy": ([vp], None),
        "idf_volume_create": ([u64, C.POINTER(idf_volume_desc), i32, C.c_size_t, C.POINTER(vp)], i32),
        "idf_volume_query": ([vp, i64, i64, i64, i32, i32, i32, vp], i32),
        "idf_volume_stats": ([vp, C.POINTER(i64)], i32),
        "idf_volume_last_error": ([vp], C.c_char_p),
        "idf_volume_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


# --------------------------------------------------------------- descriptors

class _Keep:
    """Holds the ctypes arrays a descriptor points into."""

    def __init__(self):
        self.refs = []


def level_desc(lv: dict, weights=None, keep: Optional[_Keep] = None, guide=None) -> idf_level_desc:
    import numpy as np
    keep = keep or _Keep()
    ch = (C.c_int32 * len(lv["channels"]))(*lv["channels"])
    keep.refs.append(ch)
    d = idf_level_desc()
    d.levels = lv["levels"]
    d.channels = ch
    d.in_ch, d.out_ch, d.gn_groups = lv["in_ch"], lv["out_ch"], lv["gn_groups"]
    d.attn_at_bottom, d.attn_heads = lv["attn_at_bottom"], lv["attn_heads"]
    if weights is not None:
        w = np.ascontiguousarray(weights, dtype=np.float32)
        keep.refs.append(w)
        d.weights = w.ctypes.data_as(C.POINTER(C.c_float))
        d.n_weights = w.size
    d.window, d.stride, d.offset, d.steps = lv["window"], lv["stride"], lv["offset"], lv["steps"]
    d.sigma_max, d.sigma_min, d.rho, d.sigma_data = lv["sigma_max"], lv["sigma_min"], lv["rho"], lv["sigma_data"]
    d.scale_to_parent, d.test_denoiser = lv["scale_to_parent"], lv["test_denoiser"]
    rs = lv.get("round_steps")
    if rs:
        arr = (C.c_int32 * len(rs))(*[int(v) for v in rs])
        keep.refs.append(arr)
        d.round_steps = arr
        d.n_rounds = len(rs)
    if int(lv.get("cond_dim", 0)) > 0:
        z = np.ascontiguousarray(lv["cond_z"], dtype=np.float32)
        keep.refs.append(z)
        d.cond_dim = int(lv["cond_dim"])
        d.cond_z = z.ctypes.data_as(C.POINTER(C.c_float))
        d.cond_amp = float(lv.get("cond_amp", 1.0))
    d.guidance = float(lv.get("guidance", 0.0))
    if guide is not None:
        g = np.ascontiguousarray(guide, dtype=np.float32)
        keep.refs.append(g)
        d.guide_weights = g.ctypes.data_as(C.POINTER(C.c_float))
        d.n_guide_weights = g.size
    return d


def model_stack(st: dict, weights: Optional[Sequence] = None, keep: Optional[_Keep] = None,
                guide_weights: Optional[Sequence] = None) -> idf_model_stack:
    keep = keep or _Keep()
    n = len(st["level"])
    arr = (idf_level_desc * n)()
    for i, lv in enumerate(st["level"]):
        arr[i] = level_desc(lv, None if weights is None else weights[i], keep,
                            None if guide_weights is None else guide_weights[i])
    keep.refs.append(arr)
    s = idf_model_stack()
    s.n_levels = n
    s.level = arr
    s.laplacian, s.lap_factor, s.lap_blur_sigma, s.lap_radius = (
        st["laplacian"], st["lap_factor"], st["lap_blur_sigma"], st["lap_radius"])
    s.low_mu, s.low_scale, s.res_scale, s.blend_eps = st["low_mu"], st["low_scale"], st["res_scale"], st["blend_eps"]
    fx = st.get("low_band_fixture")
    if fx is not None:
        import numpy as np
        fx = np.ascontiguousarray(fx, dtype=np.float32)
        if fx.ndim != 2 or fx.shape[0] != fx.shape[1]:
            raise ValueError("low_band_fixture must be a square 2-D array")
        keep.refs.append(fx)
        s.low_band_fixture = fx.ctypes.data_as(C.POINTER(C.c_float))
        s.fixture_period = fx.shape[0]
    keep.refs.append(s)
    return s


def param_shapes(lv: dict):
    """[(C_out, C_in, kh, kw)] of a level's UNet, in the library's declaration order."""
    L = lib()
    keep = _Keep()
    d = level_desc(lv, None, keep)
    nt, nw = C.c_int32(), C.c_size_t()
    _check(L.idf_model_param_count(C.byref(d), C.byref(nt), C.byref(nw)), "param count")
    out = []
    for i in range(nt.value):
        s = (C.c_int32 * 4)()
        _check(L.idf_model_param_shape(C.byref(d), i, s), "param shape")
        out.append(tuple(s))
    return out


def _check(status: int, what: str, world=None):
    if status != IDF_OK:
        msg = what
        if world is not None:
            m = lib().idf_world_last_error(world)
            msg = f"{what}: {m.decode() if m else ''}"
        raise IdfError(status, msg)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class World:
    """idf_world: a seeded infinite canvas of one model stack."""

    def __init__(self, seed: int, stack: dict, weights: Optional[Sequence] = None,
                 precision: str = "fp32", cache_bytes: int = 0, device: int = 0,
                 workspace_bytes: int = 0, max_batch: int = 0, profile: bool = False,
                 wait_budget_cycles: int = 0, groupnorm_in_conv: bool = False,
                 guide_weights: Optional[Sequence] = None, autotune: bool = False,
                 cuda_graphs: bool = True, cta_pairs: bool = False):
        L = lib()
        self._keep = _Keep()
        self.stack = stack
        st = model_stack(stack, weights, self._keep, guide_weights)
        o = idf_world_opts()
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.cache_bytes, o.device, o.workspace_bytes, o.max_batch = cache_bytes, device, workspace_bytes, max_batch
        o.profile = 1 if profile else 0
        o.device_wait_budget_cycles = int(wait_budget_cycles)
        o.groupnorm_in_conv = 1 if groupnorm_in_conv else 0
        o.autotune = 1 if autotune else 0
        o.cuda_graphs = 1 if cuda_graphs else 0
        o.cta_pairs = 1 if cta_pairs else 0
        h = C.c_void_p()
        _check(L.idf_world_create(C.c_uint64(seed), C.byref(st), C.byref(o), C.byref(h)), "idf_world_create")
        self._h = h
        self._stack_c = st

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().idf_world_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, x0: int, y0: int, w: int, h: int, kind: int = IDF_OUT_MODEL, out=None):
        """idf_world_query into a host float32 array (h, w)."""
        import numpy as np
        if out is None:
            out = np.empty((h, w), dtype=np.float32)
        assert out.dtype == np.float32 and out.flags.c_contiguous and out.size >= w * h
        _check(lib().idf_world_query(self._h, x0, y0, w, h, kind, out.ctypes.data_as(C.c_void_p)),
               "idf_world_query", self._h)
        return out

    def query_device(self, x0: int, y0: int, w: int, h: int, out_ptr: int, pitch: int,
                     kind: int = IDF_OUT_MODEL, stream=None):
        """idf_world_query_device into device memory (e.g. a torch tensor's data_ptr())."""
        _check(lib().idf_world_query_device(self._h, x0, y0, w, h, kind, C.c_void_p(out_ptr), pitch,
                                            _stream_ptr(stream)), "idf_world_query_device", self._h)

    def query_batch(self, regions, kind: int = IDF_OUT_MODEL, stream=None):
        """regions: [(x0, y0, w, h, out_ptr, pitch)]"""
        arr = (idf_region * len(regions))()
        for i, (x0, y0, w, h, p, pitch) in enumerate(regions):
            arr[i] = idf_region(x0, y0, w, h, p, pitch)
        _check(lib().idf_world_query_batch(self._h, arr, len(regions), kind, _stream_ptr(stream)),
               "idf_world_query_batch", self._h)

    def store_open(self, path: str, writable: bool = True):
        """idf_world_store_open: persistent tile store in directory `path`."""
        _check(lib().idf_world_store_open(self._h, path.encode(), 1 if writable else 0), "idf_world_store_open",
               self._h)

    def store_close(self):
        _check(lib().idf_world_store_close(self._h), "idf_world_store_close", self._h)

    def cache_clear(self):
        _check(lib().idf_world_cache_clear(self._h), "idf_world_cache_clear", self._h)

    def stats(self) -> dict:
        n = 1 << 16
        while True:
            buf = C.create_string_buffer(n)
            r = lib().idf_world_stats(self._h, buf, len(buf))
            if r == IDF_EINVAL and n < (1 << 26):
                n *= 4   # the summary did not fit
                continue
            _check(r, "idf_world_stats", self._h)
            return json.loads(buf.value.decode())

    def last_error(self) -> str:
        m = lib().idf_world_last_error(self._h)
        return m.decode() if m else ""

    def debug_cone(self, x0: int, y0: int, w: int, h: int, level: int, step: int):
        n = C.c_int32()
        _check(lib().idf_debug_cone(self._h, x0, y0, w, h, level, step, None, 0, C.byref(n)),
               "idf_debug_cone", self._h)
        buf = (C.c_int64 * (2 * max(1, n.value)))()
        _check(lib().idf_debug_cone(self._h, x0, y0, w, h, level, step, buf, n.value, C.byref(n)),
               "idf_debug_cone", self._h)
        return [(buf[2 * i], buf[2 * i + 1]) for i in range(n.value)]

    def debug_cache_keys(self, level: int, step: int):
        """Sorted (tile row, tile column) keys of J_step cached for a level."""
        n = C.c_int32()
        _check(lib().idf_debug_cache_keys(self._h, level, step, None, 0, C.byref(n)),
               "idf_debug_cache_keys", self._h)
        buf = (C.c_int32 * (2 * max(1, n.value)))()
        _check(lib().idf_debug_cache_keys(self._h, level, step, buf, n.value, C.byref(n)),
               "idf_debug_cache_keys", self._h)
        return [(buf[2 * i], buf[2 * i + 1]) for i in range(n.value)]

    def debug_set_status(self, which: int, value: int):
        """Host-side failure injection into a device status word (test only)."""
        _check(lib().idf_debug_set_status(self._h, which, value), "idf_debug_set_status", self._h)

    def unet_forward(self, level: int, x_ptr: int, n: int, y_ptr: int, stream=None):
        _check(lib().idf_unet_forward(self._h, level, C.c_void_p(x_ptr), n, C.c_void_p(y_ptr),
                                      _stream_ptr(stream)), "idf_unet_forward", self._h)


def noise_fill(seed: int, level: int, step: int, x0: int, y0: int, w: int, h: int, out_ptr: int,
               pitch: int, stream=None):
    _check(lib().idf_noise_fill(C.c_uint64(seed), level, step, x0, y0, w, h, C.c_void_p(out_ptr), pitch,
                                _stream_ptr(stream)), "idf_noise_fill")


def laplacian_halo(stack: dict, x0: int, y0: int, w: int, h: int):
    keep = _Keep()
    st = model_stack(stack, None, keep)
    Lr, Hr = (C.c_int64 * 4)(), (C.c_int64 * 4)()
    _check(lib().idf_laplacian_halo(C.byref(st), x0, y0, w, h, Lr, Hr), "idf_laplacian_halo")
    return tuple(Lr), tuple(Hr)


def laplacian_decode(stack: dict, L_ptr: int, lrect, lpitch: int, H_ptr: int, hrect, hpitch: int,
                     x0: int, y0: int, w: int, h: int, out_ptr: int, pitch: int, stream=None):
    """lrect / hrect = (x0, y0, w, h) of the bands on their own grids."""
    keep = _Keep()
    st = model_stack(stack, None, keep)
    _check(lib().idf_laplacian_decode(C.byref(st), C.c_void_p(L_ptr), lrect[0], lrect[1], lrect[2], lrect[3],
                                      lpitch, C.c_void_p(H_ptr), hrect[0], hrect[1], hrect[2], hrect[3], hpitch,
                                      x0, y0, w, h, C.c_void_p(out_ptr), pitch, _stream_ptr(stream)),
           "idf_laplacian_decode")


def laplacian_decode_noalloc(stack: dict, L_ptr: int, lrect, lpitch: int, H_ptr: int, hrect, hpitch: int,
                             x0: int, y0: int, w: int, h: int, out_ptr: int, pitch: int, stream=None):
    """idf_laplacian_decode_noalloc: the decode without device allocation
    (fixed 4 MiB scratch in the library; see include/idf.h)."""
    keep = _Keep()
    st = model_stack(stack, None, keep)
    _check(lib().idf_laplacian_decode_noalloc(C.byref(st), C.c_void_p(L_ptr), lrect[0], lrect[1], lrect[2],
                                              lrect[3], lpitch, C.c_void_p(H_ptr), hrect[0], hrect[1], hrect[2],
                                              hrect[3], hpitch, x0, y0, w, h, C.c_void_p(out_ptr), pitch,
                                              _stream_ptr(stream)),
           "idf_laplacian_decode_noalloc")


class Student:
    """idf_student: a student denoiser trained with the library's kernels."""

    def __init__(self, lv: dict, weights, max_batch: int, device: int = 0):
        import numpy as np
        self._keep = _Keep()
        self.lv = lv
        self.n_params = int(np.asarray(weights).size)
        d = level_desc(lv, weights, self._keep)
        h = C.c_void_p()
        st = lib().idf_student_create(C.byref(d), max_batch, device, C.byref(h))
        if st != IDF_OK:
            raise IdfError(st, "idf_student_create")
        self._h = h

    def _chk(self, st, what):
        if st != IDF_OK:
            m = lib().idf_student_last_error(self._h)
            raise IdfError(st, f"{what}: {m.decode() if m else ''}")

    def loss_grad(self, x_ptr: int, t_ptr: int, n: int, sigma: float, stream=None) -> float:
        out = C.c_double()
        self._chk(lib().idf_student_loss_grad(self._h, C.c_void_p(x_ptr), C.c_void_p(t_ptr), n, sigma,
                                              C.byref(out), _stream_ptr(stream)), "idf_student_loss_grad")
        return out.value

    def adamw(self, lr=2e-4, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01):
        self._chk(lib().idf_student_adamw(self._h, lr, beta1, beta2, eps, weight_decay), "idf_student_adamw")

    def zero_grad(self):
        self._chk(lib().idf_student_zero_grad(self._h), "idf_student_zero_grad")

    def read(self, what: int):
        import numpy as np
        out = np.empty(self.n_params, dtype=np.float32)
        self._chk(lib().idf_student_read(self._h, what, out.ctypes.data_as(C.POINTER(C.c_float)), out.size),
                  "idf_student_read")
        return out

    def write(self, weights):
        """Replace the weights (declaration order) by a host float32 array."""
        import numpy as np
        w = np.ascontiguousarray(weights, dtype=np.float32)
        self._chk(lib().idf_student_write(self._h, w.ctypes.data_as(C.POINTER(C.c_float)), w.size),
                  "idf_student_write")

    def weights(self):
        return self.read(0)

    def grads(self):
        return self.read(1)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().idf_student_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Volume:
    """idf_volume: a seeded infinite voxel volume (sampling on Z^3)."""

    def __init__(self, seed: int, desc: dict, weights=None, device: int = 0, cache_bytes: int = 0):
        import numpy as np
        self._keep = _Keep()
        d = idf_volume_desc()
        for k in ("window", "stride", "steps", "channels", "groups", "test_denoiser"):
            setattr(d, k, int(desc.get(k, 0)))
        for k in ("sigma_max", "sigma_min", "rho", "sigma_data", "blend_eps"):
            setattr(d, k, float(desc[k]))
        if weights is not None:
            w = np.ascontiguousarray(weights, dtype=np.float32)
            self._keep.refs.append(w)
            d.weights = w.ctypes.data_as(C.POINTER(C.c_float))
            d.n_weights = w.size
        h = C.c_void_p()
        st = lib().idf_volume_create(C.c_uint64(seed), C.byref(d), device, cache_bytes, C.byref(h))
        if st != IDF_OK:
            raise IdfError(st, "idf_volume_create")
        self._h = h

    def query(self, x0: int, y0: int, z0: int, w: int, h: int, d: int):
        import numpy as np
        out = np.empty((d, h, w), dtype=np.float32)
        st = lib().idf_volume_query(self._h, x0, y0, z0, w, h, d, out.ctypes.data_as(C.c_void_p))
        if st != IDF_OK:
            m = lib().idf_volume_last_error(self._h)
            raise IdfError(st, f"idf_volume_query: {m.decode() if m else ''}")
        return out

    def stats(self) -> dict:
        a = (C.c_int64 * 4)()
        _check(lib().idf_volume_stats(self._h, a), "idf_volume_stats")
        return {"windows_evaluated": a[0], "tiles_computed": a[1], "cache_hits": a[2], "cache_misses": a[3]}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().idf_volume_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
