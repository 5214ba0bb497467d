// Sampler kernels of libidf: noise, window gather, the fused blend / update /
// re-noise of one InfiniteDiffusion step, tile assembly and the Laplacian
// decode.  All of them are bandwidth-bound; each thread owns whole pixels so
// that every pixel's arithmetic runs in a fixed order (bitwise determinism).
#include "internal.h"
#include "noise.cuh"

namespace idf {

// ------------------------------------------------------------------ noise
__global__ void noise_fill_kernel(uint64_t seed, uint32_t level, uint32_t step, int64_t x0,
                                  int64_t y0, int w, int h, float* out, int64_t pitch) {
  const int64_t n = (int64_t)w * h;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / w), c = (int)(i % w);
    out[r * pitch + c] = normal_at(seed, level, step, x0 + c, y0 + r);
  }
}

static int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g > 152 * 64) g = 152 * 64;
  if (g < 1) g = 1;
  return (int)g;
}

void launch_noise_fill(uint64_t seed, uint32_t level, uint32_t step, int64_t x0, int64_t y0,
                       int w, int h, float* out, int64_t pitch, cudaStream_t st) {
  noise_fill_kernel<<<grid_for((int64_t)w * h, 256), 256, 0, st>>>(seed, level, step, x0, y0, w,
                                                                   h, out, pitch);
}

// ------------------------------------------------------------------ gather
// x_in[b][u][v][0] = c_in * J_k(Y, X); channel 1 (conditioned levels) is the
// parent's result at (floor(Y/f), floor(X/f)), unscaled.
__global__ void gather_kernel(GatherArgs a) {
  const int H = a.H, s = a.s, r = a.r;
  const int64_t per = (int64_t)H * H;
  const int64_t n = per * a.n_win;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx / per);
    const int p = (int)(idx % per);
    const int u = p / H, v = p % H;
    const int64_t wi = a.win_ij[2 * b], wj = a.win_ij[2 * b + 1];
    const int64_t Y = wi * s + u, X = wj * s + v;
    float J;
    if (a.noise_step0) {
      J = __fmul_rn(a.sigma0, normal_at(a.seed, a.level, 0u, X, Y));
    } else {
      const int m = u / s, q = v / s;
      const int slot = a.win_slots[(int64_t)b * r * r + m * r + q];
      J = a.pool[(int64_t)slot * s * s + (u - m * s) * s + (v - q * s)];
    }
    float* o = a.x_in + idx * a.in_ch;
    o[0] = __fmul_rn(a.c_in, J);
    if (a.xs) a.xs[idx] = J;
    if (a.in_ch == 2) {
      const int64_t cy = fdiv(Y, a.cond_f) - a.cond_y0, cx = fdiv(X, a.cond_f) - a.cond_x0;
      float c = 0.0f;
      if (cy >= 0 && cy < a.cond_h && cx >= 0 && cx < a.cond_w) {
        c = a.cond[cy * a.cond_pitch + cx];
      } else {
        atomicOr(a.err_flag, 1);
      }
      o[1] = c;
    }
  }
}

void launch_gather(const GatherArgs& a, cudaStream_t st) {
  const int64_t n = (int64_t)a.H * a.H * a.n_win;
  gather_kernel<<<grid_for(n, 256), 256, 0, st>>>(a);
}

// ------------------------------------------------------------ window step
__global__ void window_step_kernel(WindowStepArgs a) {
  const int H = a.H;
  const int64_t per = (int64_t)H * H;
  const int64_t n = per * a.n_win;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const float d = __fadd_rn(__fmul_rn(a.c_skip, a.xs[idx]), __fmul_rn(a.c_out, a.F[idx]));
    if (a.last) {
      a.F[idx] = d;
      continue;
    }
    float xn = d;
    if (a.noise) {
      const int b = (int)(idx / per);
      const int p = (int)(idx % per);
      const int64_t Y = (int64_t)a.win_ij[2 * b] * a.s + p / H, X = (int64_t)a.win_ij[2 * b + 1] * a.s + p % H;
      xn = __fadd_rn(d, __fmul_rn(a.sigma_next, normal_at(a.seed, a.level, a.step_next, X, Y)));
    }
    a.xs[idx] = xn;
    a.x_in[idx * a.in_ch] = __fmul_rn(a.c_in_next, xn);
  }
}

void launch_window_step(const WindowStepArgs& a, cudaStream_t st) {
  const int64_t n = (int64_t)a.H * a.H * a.n_win;
  window_step_kernel<<<grid_for(n, 256), 256, 0, st>>>(a);
}

// ------------------------------------------------------------ conditioning
__global__ void cond_bias_kernel(const int32_t* win_ij, int n, uint64_t seed, uint32_t level, const float* z,
                                 float amp, const float* E, int D, int C, float* bias) {
  const int64_t total = (int64_t)n * C;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / C), c = (int)(t % C);
    const int64_t i = win_ij[2 * b], j = win_ij[2 * b + 1];
    float acc = 0.0f;
    for (int d = 0; d < D; ++d) {
      const float y = __fadd_rn(z[d], __fmul_rn(amp, normal_at(seed, level, COND_STEP + (uint32_t)d, j, i)));
      acc = __fadd_rn(acc, __fmul_rn(E[c * D + d], y));
    }
    bias[t] = acc;
  }
}

void launch_cond_bias(const int32_t* win_ij, int n, uint64_t seed, uint32_t level, const float* z, float amp,
                      const float* E, int D, int C, float* bias, cudaStream_t st) {
  cond_bias_kernel<<<grid_for((int64_t)n * C, 256), 256, 0, st>>>(win_ij, n, seed, level, z, amp, E, D, C, bias);
}

__global__ void guidance_kernel(float* F, const float* Fg, int64_t n, float w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = Fg[i];
    F[i] = __fadd_rn(g, __fmul_rn(w, __fsub_rn(F[i], g)));
  }
}

void launch_guidance(float* F, const float* Fg, int64_t n, float w, cudaStream_t st) {
  guidance_kernel<<<grid_for(n, 256), 256, 0, st>>>(F, Fg, n, w);
}

// ------------------------------------------------------------------ blend
// One step of Eq. 2 for the missing tiles of J_{k+1}, in the fused form
//   J_{k+1} = c_skip J_k + c_out (sum_i W_i F_i) / B + sigma_{k+1} N(k+1)
// (the noise and J_k terms are the same for every window covering a pixel,
// so blending D_i and adding them once equals blending full window updates).
// The r*r window terms of a pixel are summed in a fixed order: window row
// index ascending, then column index ascending.
__global__ void blend_kernel(BlendArgs a) {
  const int t = blockIdx.x;
  const int s = a.s, r = a.r, H = a.H;
  const int32_t* tl = a.tiles + 4 * t;
  const int64_t ty = tl[0], tx = tl[1];
  const int slot_in = tl[2], slot_out = tl[3];
  const int32_t* tw = a.tile_wins + (int64_t)t * r * r;
  const int64_t HH = (int64_t)H * H;
  for (int p = threadIdx.x; p < s * s; p += blockDim.x) {
    const int pa = p / s, pb = p % s;
    float acc = 0.0f;
    for (int mi = r - 1; mi >= 0; --mi) {
      const int u = mi * s + pa;
      const float wu = a.w1[u];
      for (int ni = r - 1; ni >= 0; --ni) {
        const int v = ni * s + pb;
        const int wb = tw[mi * r + ni];
        const float f = a.F[(int64_t)wb * HH + (int64_t)u * H + v];
        acc = __fadd_rn(acc, __fmul_rn(__fmul_rn(wu, a.w1[v]), f));
      }
    }
    const int64_t Y = ty * s + pa, X = tx * s + pb;
    float Jk;
    if (a.noise_in) {
      Jk = __fmul_rn(a.sigma0, normal_at(a.seed, a.level, 0u, X, Y));
    } else {
      Jk = a.pool[(int64_t)slot_in * s * s + p];
    }
    const float avg = __fmul_rn(__fmul_rn(acc, a.invB1[pa]), a.invB1[pb]);
    float J = __fadd_rn(__fmul_rn(a.c_skip, Jk), __fmul_rn(a.c_out, avg));
    if (a.noise_next) {
      J = __fadd_rn(J, __fmul_rn(a.sigma_next, normal_at(a.seed, a.level, a.step_next, X, Y)));
    }
    a.pool_out[(int64_t)slot_out * s * s + p] = J;
  }
}

void launch_blend(const BlendArgs& a, cudaStream_t st) {
  if (a.n_tiles <= 0) return;
  const int block = a.s * a.s >= 1024 ? 512 : 256;
  blend_kernel<<<a.n_tiles, block, 0, st>>>(a);
}

// ------------------------------------------------------------ test denoisers
__global__ void test_denoiser_kernel(int kind, const float* x, int n, int H, int in_ch, float* F) {
  const int64_t per = (int64_t)H * H;
  const int64_t total = per * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v;
    if (kind == 1) {
      v = 0.5f;
    } else {
      v = x[i * in_ch];
      for (int c = 1; c < in_ch; ++c) v = __fadd_rn(v, x[i * in_ch + c]);
      if (kind == 3) {
        const int p = (int)(i % per);
        const float uu = __fdiv_rn((float)(p / H), (float)H);
        const float vv = __fdiv_rn((float)(p % H), (float)H);
        v = __fadd_rn(v, __fsub_rn(uu, __fmul_rn(2.0f, vv)));
      }
    }
    F[i] = v;
  }
}

void launch_test_denoiser(int kind, const float* x_in, int n, int H, int in_ch, float* F,
                          cudaStream_t st) {
  const int64_t total = (int64_t)H * H * n;
  test_denoiser_kernel<<<grid_for(total, 256), 256, 0, st>>>(kind, x_in, n, H, in_ch, F);
}

// ------------------------------------------------------------------ assemble
__global__ void assemble_kernel(const float* pool, const int32_t* slots, int64_t ty0, int64_t tx0,
                                int ntx, int s, int64_t y0, int64_t x0, int h, int w, float* out,
                                int64_t pitch) {
  const int64_t n = (int64_t)w * h;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int rr = (int)(i / w), cc = (int)(i % w);
    const int64_t Y = y0 + rr, X = x0 + cc;
    const int64_t ty = fdiv(Y, s), tx = fdiv(X, s);
    const int slot = slots[(ty - ty0) * ntx + (tx - tx0)];
    out[rr * pitch + cc] =
        pool[(int64_t)slot * s * s + (Y - ty * s) * s + (X - tx * s)];
  }
}

void launch_assemble(const float* pool, const int32_t* tile_slots, int64_t ty0, int64_t tx0,
                     int nty, int ntx, int s, int64_t y0, int64_t x0, int h, int w, float* out,
                     int64_t pitch, cudaStream_t st) {
  (void)nty;
  assemble_kernel<<<grid_for((int64_t)w * h, 256), 256, 0, st>>>(pool, tile_slots, ty0, tx0, ntx,
                                                                 s, y0, x0, h, w, out, pitch);
}

// ------------------------------------------------------------------ layouts
__global__ void nchw_to_nhwc_kernel(const float* x, int n, int c, int hw, float* y) {
  const int64_t total = (int64_t)n * c * hw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / ((int64_t)c * hw);
    const int64_t rem = i % ((int64_t)c * hw);
    const int ch = (int)(rem / hw), p = (int)(rem % hw);
    y[(b * hw + p) * c + ch] = x[i];
  }
}
__global__ void nhwc_to_nchw_kernel(const float* x, int n, int c, int hw, float* y) {
  const int64_t total = (int64_t)n * c * hw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / ((int64_t)c * hw);
    const int64_t rem = i % ((int64_t)c * hw);
    const int ch = (int)(rem / hw), p = (int)(rem % hw);
    y[i] = x[(b * hw + p) * c + ch];
  }
}
void launch_nchw_to_nhwc(const float* x, int n, int c, int hw, float* y, cudaStream_t st) {
  nchw_to_nhwc_kernel<<<grid_for((int64_t)n * c * hw, 256), 256, 0, st>>>(x, n, c, hw, y);
}
void launch_nhwc_to_nchw(const float* x, int n, int c, int hw, float* y, cudaStream_t st) {
  nhwc_to_nchw_kernel<<<grid_for((int64_t)n * c * hw, 256), 256, 0, st>>>(x, n, c, hw, y);
}

// ------------------------------------------------------------------ decode
// Laplacian denoising decode (Sec. 5.2).  With l = low_mu + low_scale L and
// h = res_scale H:  P = up(l) + h;  D = down(P);  l^ = blur(D);
// v = up(l^) + h;  metres = sign(v) v^2.
// down(up(l)) for an even factor with half-pixel bilinear weights is the
// separable 3-tap filter [1/8, 3/4, 1/8] on the coarse grid (the block mean
// of the upsampled image), which D uses instead of materialising P.
__global__ void decode_down_kernel(DecodeArgs a) {
  const int R = a.R, f = a.f;
  const int dw = a.qw + 2 * R, dh = a.qh + 2 * R;
  const int64_t n = (int64_t)dw * dh;
  const float k3[3] = {0.125f, 0.75f, 0.125f};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int dy = (int)(i / dw), dx = (int)(i % dw);
    const int64_t Y = a.qy0 - R + dy, X = a.qx0 - R + dx;
    float lo = 0.0f;
    for (int p = 0; p < 3; ++p) {
      const float* row = a.L + (Y - 1 + p - a.ly0) * a.lpitch + (X - 1 - a.lx0);
      float rs = 0.0f;
      for (int q = 0; q < 3; ++q) rs = __fadd_rn(rs, __fmul_rn(k3[q], row[q]));
      lo = __fadd_rn(lo, __fmul_rn(k3[p], rs));
    }
    const float l = __fadd_rn(a.low_mu, __fmul_rn(a.low_scale, lo));
    const float* hb = a.H + (Y * f - a.hy0) * a.hpitch + (X * f - a.hx0);
    float hs = 0.0f;
    for (int yy = 0; yy < f; ++yy)
      for (int xx = 0; xx < f; ++xx) hs = __fadd_rn(hs, hb[yy * a.hpitch + xx]);
    const float hm = __fmul_rn(a.res_scale, __fdiv_rn(hs, (float)(f * f)));
    a.D[i] = __fadd_rn(l, hm);
  }
}

__global__ void decode_blur_h_kernel(DecodeArgs a) {
  const int R = a.R;
  const int dw = a.qw + 2 * R, dh = a.qh + 2 * R;
  const int64_t n = (int64_t)a.qw * dh;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / a.qw), x = (int)(i % a.qw);
    const float* d = a.D + (int64_t)y * dw + x;
    float acc = 0.0f;
    for (int k = 0; k <= 2 * R; ++k) acc = __fadd_rn(acc, __fmul_rn(a.taps[k], d[k]));
    a.T[i] = acc;
  }
}

__global__ void decode_blur_v_kernel(DecodeArgs a) {
  const int R = a.R;
  const int64_t n = (int64_t)a.qw * a.qh;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / a.qw), x = (int)(i % a.qw);
    float acc = 0.0f;
    for (int k = 0; k <= 2 * R; ++k)
      acc = __fadd_rn(acc, __fmul_rn(a.taps[k], a.T[(int64_t)(y + k) * a.qw + x]));
    a.Lhat[i] = acc;
  }
}

__global__ void decode_final_kernel(DecodeArgs a) {
  const int f = a.f;
  const int64_t n = (int64_t)a.w * a.h;
  const float inv2f = 1.0f / (2.0f * f);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / a.w), c = (int)(i % a.w);
    const int64_t y = a.y0 + r, x = a.x0 + c;
    // half-pixel bilinear: lower coarse index and weight of the upper one
    const int64_t ny = 2 * y + 1 - f, nx = 2 * x + 1 - f;
    const int64_t Y0 = fdiv(ny, 2 * f), X0 = fdiv(nx, 2 * f);
    const float ay = (float)(ny - Y0 * 2 * f) * inv2f;   // exact: multiples of 1/(2f)
    const float ax = (float)(nx - X0 * 2 * f) * inv2f;
    const float* q0 = a.Lhat + (Y0 - a.qy0) * a.qw + (X0 - a.qx0);
    const float* q1 = q0 + a.qw;
    const float top = __fadd_rn(__fmul_rn(1.0f - ax, q0[0]), __fmul_rn(ax, q0[1]));
    const float bot = __fadd_rn(__fmul_rn(1.0f - ax, q1[0]), __fmul_rn(ax, q1[1]));
    const float up = __fadd_rn(__fmul_rn(1.0f - ay, top), __fmul_rn(ay, bot));
    const float hv = __fmul_rn(a.res_scale, a.H[(y - a.hy0) * a.hpitch + (x - a.hx0)]);
    const float v = __fadd_rn(up, hv);
    a.out[r * a.pitch + c] = copysignf(__fmul_rn(v, v), v);
  }
}

void launch_decode(const DecodeArgs& a, cudaStream_t st) {
  const int64_t nd = (int64_t)(a.qw + 2 * a.R) * (a.qh + 2 * a.R);
  decode_down_kernel<<<grid_for(nd, 256), 256, 0, st>>>(a);
  decode_blur_h_kernel<<<grid_for((int64_t)a.qw * (a.qh + 2 * a.R), 256), 256, 0, st>>>(a);
  decode_blur_v_kernel<<<grid_for((int64_t)a.qw * a.qh, 256), 256, 0, st>>>(a);
  decode_final_kernel<<<grid_for((int64_t)a.w * a.h, 256), 256, 0, st>>>(a);
}

// ---------------------------------------------------------------- fixture
__global__ void fixture_gather_kernel(const float* __restrict__ fx, int64_t P, int64_t x0, int64_t y0, int w,
                                      int h, float* __restrict__ dst) {
  const int64_t n = (int64_t)w * h;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / w, x = i % w;
    int64_t gy = (y0 + y) % P, gx = (x0 + x) % P;
    if (gy < 0) gy += P;
    if (gx < 0) gx += P;
    dst[i] = fx[gy * P + gx];
  }
}

void launch_fixture_gather(const float* fixture, int64_t P, int64_t x0, int64_t y0, int w, int h, float* dst,
                           cudaStream_t st) {
  const int64_t n = (int64_t)w * h;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  if (n > 0) fixture_gather_kernel<<<blocks, 256, 0, st>>>(fixture, P, x0, y0, w, h, dst);
}

}  // namespace idf
