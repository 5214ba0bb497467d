// Learned student denoiser: training on the GPU with the library's own
// forward and backward kernels (the library's counterpart of the paper's few-step
// distilled models, Sec. 5.4 / App. F "Consistency Distillation").
//
// The network is the ResBlock UNet of unet.cu (same layer reading and weight
// order, no attention block).  A training step evaluates
//   D(x; sigma) = c_skip x + c_out S(c_in x),  loss = mean((D - t)^2)
// and accumulates dloss/dw; AdamW applies the accumulated gradient.  With
// in_ch > 1 the input x (NCHW) carries the noisy state in channel 0 and side
// inputs in the others: D = c_skip x_0 + c_out S([c_in x_0, x_1, ...]).
//
// Engine: the forward runs as a tape of ops (conv, GroupNorm+SiLU, pool,
// upsample-concat) that keeps every activation; the backward walks the tape in
// reverse, adding each op's input gradients into zero-initialised gradient
// buffers (one kernel per accumulation, so the sums have a fixed order):
//   conv      dX += conv(dY, W^T) (taps flipped, C_in/C_out swapped),
//             dW += sum over pixels of X_shifted dY^T (split-K partials
//             summed in chunk order), dRes += dY;
//   GN+SiLU   z = (x - mu) r, dz = dy s (1 + z (1 - s)) with s = sigmoid(z),
//             dx = r (dz - mean_g(dz) - z mean_g(dz z)) per (window, group);
//   pool      dX[2y+a][2x+b] += dY[y][x] / 4;
//   upcat     dA[y][x] += sum of dY over its 2x2 block (first C_a channels),
//             dSkip += dY (remaining channels).
// Everything is float32 with float64 reductions.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/idf.h"
#include "internal.h"

using namespace idf;

namespace {

int grid_n(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

// ---------------------------------------------------------------- kernels

// W^T for the input gradient: wk [tap*Cin + ci][Cout] -> wt [tap'*Cout + co][Cin]
// with tap' = taps - 1 - tap (a 180-degree flip of the kernel).
__global__ void conv_w_transpose_kernel(const float* __restrict__ wk, float* __restrict__ wt, int taps,
                                        int Cin, int Cout) {
  const int64_t n = (int64_t)taps * Cin * Cout;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int co = (int)(i % Cout);
    const int64_t r = i / Cout;
    const int ci = (int)(r % Cin);
    const int tap = (int)(r / Cin);
    wt[((int64_t)(taps - 1 - tap) * Cout + co) * Cin + ci] = wk[i];
  }
}

// Weight gradient partials: part[chunk][k][co] = sum over the chunk's pixels m
// of X[m shifted by tap][ci] * G[m][co], k = tap*Cin + ci.  CTA tile 64 k x 64
// co, 16 pixels per smem step, thread = 4 x 4 outputs.
template <int KS>
__global__ void __launch_bounds__(256) wgrad_partial_kernel(const float* __restrict__ x,
                                                            const float* __restrict__ g,
                                                            float* __restrict__ part, int n, int H, int W,
                                                            int Cin, int Cout, int64_t chunk_px) {
  __shared__ float Xs[16][64 + 1];
  __shared__ float Gs[16][64 + 1];
  const int K = KS * KS * Cin;
  const int k0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
  const int64_t M = (int64_t)n * H * W;
  const int64_t m_begin = (int64_t)blockIdx.z * chunk_px;
  const int64_t m_end = min(M, m_begin + chunk_px);
  const int tid = threadIdx.x;
  const int tr = tid / 16, tc = tid % 16;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  for (int64_t mb = m_begin; mb < m_end; mb += 16) {
    // 16 x 64 of each operand, 4 elements per thread each
#pragma unroll
    for (int e4 = 0; e4 < 4; ++e4) {
      const int e = tid + e4 * 256;
      const int mm = e / 64, kk = e % 64;
      const int64_t m = mb + mm;
      float xv = 0.0f, gv = 0.0f;
      if (m < m_end) {
        const int k = k0 + kk;
        const int64_t b = m / ((int64_t)H * W);
        const int p = (int)(m - b * H * W);
        const int py = p / W, px = p % W;
        if (k < K) {
          const int tap = k / Cin, ci = k % Cin;
          const int sy = py + tap / KS - KS / 2, sx = px + tap % KS - KS / 2;
          if (sy >= 0 && sy < H && sx >= 0 && sx < W) xv = x[((b * H + sy) * W + sx) * Cin + ci];
        }
        const int co = c0 + kk;
        if (co < Cout) gv = g[m * Cout + co];
      }
      Xs[mm][kk] = xv;
      Gs[mm][kk] = gv;
    }
    __syncthreads();
#pragma unroll
    for (int mm = 0; mm < 16; ++mm) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Xs[mm][tr * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Gs[mm][tc * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* pp = part + (int64_t)blockIdx.z * K * Cout;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = k0 + tr * 4 + i;
    if (k >= K) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int co = c0 + tc * 4 + j;
      if (co < Cout) pp[(int64_t)k * Cout + co] = acc[i][j];
    }
  }
}

// dW[e] += sum over chunks (in order) of part[chunk][e]
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int chunks, int64_t n_el,
                                    float* __restrict__ dw) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += (double)part[(int64_t)c * n_el + e];
    dw[e] += (float)s;
  }
}

__device__ __forceinline__ float gn_dz(float x, float dy, float2 ms, bool silu, float* zout) {
  const float z = (x - ms.x) * ms.y;
  *zout = z;
  if (!silu) return dy;
  const float s = 1.0f / (1.0f + expf(-z));
  return dy * s * (1.0f + z * (1.0f - s));
}

// per (window, group, chunk): sums of dz and dz*z
__global__ void __launch_bounds__(256) gnb_partial_kernel(const float* __restrict__ x,
                                                          const float* __restrict__ dy,
                                                          const float2* __restrict__ stats, int HW,
                                                          int C, int G, int chunk_px, bool silu,
                                                          double2* __restrict__ part) {
  __shared__ double r1[256], r2[256];
  const int Cg = C / G;
  const int chunk = blockIdx.x, g = blockIdx.y, b = blockIdx.z;
  const float2 ms = stats[b * G + g];
  const int p0 = chunk * chunk_px, p1 = min(HW, p0 + chunk_px);
  const int64_t base = (int64_t)b * HW * C + g * Cg;
  double s1 = 0.0, s2 = 0.0;
  float a1 = 0.0f, a2 = 0.0f;
  const int nel = (p1 - p0) * Cg;
  for (int e = threadIdx.x; e < nel; e += blockDim.x) {
    const int p = p0 + e / Cg, c = e % Cg;
    const int64_t off = base + (int64_t)p * C + c;
    float z;
    const float dz = gn_dz(x[off], dy[off], ms, silu, &z);
    a1 += dz;
    a2 += dz * z;
  }
  s1 = a1;
  s2 = a2;
  r1[threadIdx.x] = s1;
  r2[threadIdx.x] = s2;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      r1[threadIdx.x] += r1[threadIdx.x + o];
      r2[threadIdx.x] += r2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[((int64_t)b * G + g) * gridDim.x + chunk] = make_double2(r1[0], r2[0]);
}

__global__ void gnb_finalize_kernel(const double2* __restrict__ part, int n_win, int chunks, int HW, int Cg,
                                    int G, float2* __restrict__ means) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_win * G) return;
  double s1 = 0.0, s2 = 0.0;
  for (int c = 0; c < chunks; ++c) {
    const double2 pp = part[(int64_t)i * chunks + c];
    s1 += pp.x;
    s2 += pp.y;
  }
  const double n = (double)HW * Cg;
  means[i] = make_float2((float)(s1 / n), (float)(s2 / n));
}

__global__ void gnb_apply_kernel(const float* __restrict__ x, const float* __restrict__ dy,
                                 const float2* __restrict__ stats, const float2* __restrict__ means,
                                 int64_t n_el, int HW, int C, int G, bool silu, float* __restrict__ dx) {
  const int Cg = C / G;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_el; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t b = i / ((int64_t)HW * C);
    const int bg = (int)(b * G + c / Cg);
    const float2 ms = stats[bg];
    const float2 mm = means[bg];
    float z;
    const float dz = gn_dz(x[i], dy[i], ms, silu, &z);
    dx[i] += ms.y * (dz - mm.x - z * mm.y);
  }
}

__global__ void pool_bwd_kernel(const float* __restrict__ dy, int n, int H, int C, float* __restrict__ dx) {
  // dx at full resolution H; dy at H/2
  const int64_t n_el = (int64_t)n * H * H * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_el; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t pix = i / C;
    const int xx = (int)(pix % H);
    const int64_t r = pix / H;
    const int yy = (int)(r % H);
    const int64_t b = r / H;
    dx[i] += 0.25f * dy[((b * (H / 2) + yy / 2) * (H / 2) + xx / 2) * C + c];
  }
}

// split the concat gradient: dA (H/2 resolution) gets the 2x2 block sums of
// the first Ca channels, dSkip the remaining Cb channels
__global__ void upcat_bwd_a_kernel(const float* __restrict__ dy, int Ca, int Cb, int n, int H,
                                   float* __restrict__ da) {
  const int Hh = H / 2, C = Ca + Cb;
  const int64_t n_el = (int64_t)n * Hh * Hh * Ca;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_el; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % Ca);
    const int64_t pix = i / Ca;
    const int xx = (int)(pix % Hh);
    const int64_t r = pix / Hh;
    const int yy = (int)(r % Hh);
    const int64_t b = r / Hh;
    const float* p = dy + ((b * H + 2 * yy) * H + 2 * xx) * C + c;
    da[i] += (p[0] + p[C]) + (p[(int64_t)H * C] + p[(int64_t)H * C + C]);
  }
}

__global__ void upcat_bwd_skip_kernel(const float* __restrict__ dy, int Ca, int Cb, int64_t n_pix,
                                      float* __restrict__ ds) {
  const int C = Ca + Cb;
  const int64_t n_el = n_pix * Cb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_el; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pix = i / Cb;
    const int c = (int)(i % Cb);
    ds[i] += dy[pix * C + Ca + c];
  }
}

__global__ void add_kernel(const float* __restrict__ a, int64_t n_el, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_el; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a[i];
}

// NCHW x -> NHWC network input: channel 0 scaled by c_in, side channels as they are
__global__ void precond_in_kernel(const float* __restrict__ x, float c_in, int64_t npx, int HW, int C,
                                  float* __restrict__ y) {
  const int64_t n_el = npx * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_el; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t m = i / C, b = m / HW, px = m % HW;
    const float v = x[(b * C + c) * HW + px];
    y[i] = c == 0 ? c_in * v : v;
  }
}

// D = c_skip x + c_out F; per-block sums of (D - t)^2 in double; gF = 2 c_out (D - t) / N
// (x: channel 0 of the NCHW input, C channels of HW pixels per window)
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ x, const float* __restrict__ F,
                                                  const float* __restrict__ t, int64_t N, float c_skip,
                                                  float c_out, float* __restrict__ gF,
                                                  double* __restrict__ block_sums, int HW, int C) {
  __shared__ double red[256];
  double s = 0.0;
  const float k = 2.0f * c_out / (float)N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = c_skip * x[(i / HW) * C * HW + i % HW] + c_out * F[i] - t[i];
    s += (double)d * d;
    gF[i] = k * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = red[0];
}

__global__ void adamw_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                             float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float wd,
                             float bc1, float bc2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / bc1, vh = vi / bc2;
    w[i] = w[i] - lr * (mh / (sqrtf(vh) + eps) + wd * w[i]);
  }
}

// ---------------------------------------------------------------- tape

struct SBuf {
  size_t off;  // floats into the activation / gradient arenas (per window x max_batch)
  int C, H;
};

enum OpKind { OP_CONV, OP_GN, OP_POOL, OP_UPCAT };

struct SOp {
  OpKind kind;
  int in = -1, in2 = -1, out = -1, res = -1;
  int conv = -1;
  bool silu = true;
  size_t stats_off = 0;  // float2 index into the stats arena (per window x G)
};

struct SConv {
  int cin, cout, ks;
  size_t w_off;  // packed [K][Cout] offset in the parameter vector
  size_t n;
};

}  // namespace

struct idf_student {
  UNetDesc d;
  int max_batch = 0;
  std::vector<SConv> convs;
  std::vector<SBuf> bufs;
  std::vector<SOp> ops;
  size_t n_params = 0, per_window = 0, stats_per_window = 0;
  int buf_x = -1, buf_F = -1;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *wt = nullptr;
  float *act = nullptr, *grad = nullptr, *wpart = nullptr;
  float2* stats = nullptr;
  float2* gmeans = nullptr;
  double2* part = nullptr;
  double* loss_parts = nullptr;
  size_t wt_cap = 0, wpart_cap = 0;
  int step = 0;
  cudaStream_t st = nullptr;
  std::string err;
};

namespace {

int add_buf(idf_student* s, int C, int H) {
  SBuf b{s->per_window, C, H};
  s->per_window += (size_t)C * H * H;
  s->bufs.push_back(b);
  return (int)s->bufs.size() - 1;
}

int add_conv_op(idf_student* s, size_t& ci, int in, int res) {
  const SConv& c = s->convs[ci];
  SOp op;
  op.kind = OP_CONV;
  op.in = in;
  op.res = res;
  op.conv = (int)ci++;
  op.out = add_buf(s, c.cout, s->bufs[in].H);
  s->ops.push_back(op);
  return op.out;
}

int add_gn_op(idf_student* s, int in, bool silu) {
  SOp op;
  op.kind = OP_GN;
  op.in = in;
  op.silu = silu;
  op.stats_off = s->stats_per_window;
  s->stats_per_window += s->d.groups;
  op.out = add_buf(s, s->bufs[in].C, s->bufs[in].H);
  s->ops.push_back(op);
  return op.out;
}

int add_resblock(idf_student* s, size_t& ci, int X, int cin, int cout) {
  const size_t c1 = ci;
  (void)c1;
  const int A1 = add_gn_op(s, X, true);
  const int T = add_conv_op(s, ci, A1, -1);
  const int A2 = add_gn_op(s, T, true);
  // declaration order is conv1, conv2, skip: take conv2 after the shortcut
  const size_t conv2 = ci++;
  int S = X;
  if (cin != cout) S = add_conv_op(s, ci, X, -1);
  SOp op;
  op.kind = OP_CONV;
  op.in = A2;
  op.res = S;
  op.conv = (int)conv2;
  op.out = add_buf(s, cout, s->bufs[X].H);
  s->ops.push_back(op);
  return op.out;
}

void build_tape(idf_student* s) {
  const UNetDesc& d = s->d;
  const int L = d.levels;
  size_t ci = 0;
  s->buf_x = add_buf(s, d.in_ch, d.window);
  int h = add_conv_op(s, ci, s->buf_x, -1);
  int prev = d.ch[0];
  std::vector<int> skips;
  for (int l = 0; l < L; ++l) {
    h = add_resblock(s, ci, h, prev, d.ch[l]);
    prev = d.ch[l];
    skips.push_back(h);
    if (l < L - 1) {
      SOp op;
      op.kind = OP_POOL;
      op.in = h;
      op.out = add_buf(s, prev, s->bufs[h].H / 2);
      s->ops.push_back(op);
      h = op.out;
    }
  }
  h = add_resblock(s, ci, h, prev, prev);
  for (int l = L - 2; l >= 0; --l) {
    SOp op;
    op.kind = OP_UPCAT;
    op.in = h;
    op.in2 = skips[l];
    op.out = add_buf(s, prev + d.ch[l], s->bufs[skips[l]].H);
    s->ops.push_back(op);
    h = add_resblock(s, ci, op.out, prev + d.ch[l], d.ch[l]);
    prev = d.ch[l];
  }
  const int A = add_gn_op(s, h, true);
  s->buf_F = add_conv_op(s, ci, A, -1);
}

bool ck(idf_student* s, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  s->err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return false;
}

template <typename T>
bool grow(idf_student* s, T** p, size_t* cap, size_t n) {
  if (n <= *cap) return true;
  cudaFree(*p);
  *p = nullptr;
  if (!ck(s, cudaMalloc((void**)p, n * sizeof(T)), "cudaMalloc")) {
    *cap = 0;
    return false;
  }
  *cap = n;
  return true;
}

float* A(idf_student* s, int b) { return s->act + s->bufs[b].off * s->max_batch; }
float* Gd(idf_student* s, int b) { return s->grad + s->bufs[b].off * s->max_batch; }

}  // namespace

// ==================================================================== C ABI
extern "C" {

void idf_student_destroy(idf_student* s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  cudaFree(s->w); cudaFree(s->g); cudaFree(s->m); cudaFree(s->v); cudaFree(s->wt);
  cudaFree(s->act); cudaFree(s->grad); cudaFree(s->wpart); cudaFree(s->stats); cudaFree(s->gmeans);
  cudaFree(s->part); cudaFree(s->loss_parts);
  if (s->st) cudaStreamDestroy(s->st);
  delete s;
}

idf_status idf_student_create(const idf_level_desc* net, int32_t max_batch, int32_t device, idf_student** out) {
  if (!out) return IDF_EINVAL;
  *out = nullptr;
  if (!net || max_batch < 1 || net->levels < 1 || net->levels > 6 || !net->channels || net->attn_at_bottom ||
      net->in_ch < 1 || net->in_ch > 8 || net->out_ch != 1 || net->gn_groups < 1 || net->window < 2 ||
      net->window % (1 << (net->levels - 1)) || !(net->sigma_data > 0))
    return IDF_EINVAL;
  for (int l = 0; l < net->levels; ++l)
    if (net->channels[l] < 1 || net->channels[l] % net->gn_groups) return IDF_EINVAL;
  int32_t nt;
  size_t nw;
  if (idf_model_param_count(net, &nt, &nw) != IDF_OK) return IDF_EINVAL;
  if (!net->weights || net->n_weights != nw) return IDF_EMODEL;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return IDF_ECUDA;
  }
  idf_student* s = new idf_student();
  s->d.levels = net->levels;
  s->d.ch.assign(net->channels, net->channels + net->levels);
  s->d.in_ch = net->in_ch;
  s->d.out_ch = 1;
  s->d.groups = net->gn_groups;
  s->d.attn = 0;
  s->d.heads = 0;
  s->d.window = net->window;
  s->max_batch = max_batch;
  // packed parameters: per conv [tap*Cin + ci][Cout]
  auto shapes = unet_param_shapes(s->d);
  std::vector<float> packed;
  size_t off = 0;
  for (auto& sh : shapes) {
    SConv c{sh[1], sh[0], sh[2], packed.size(), (size_t)sh[0] * sh[1] * sh[2] * sh[3]};
    const int taps = c.ks * c.ks;
    const size_t base = packed.size();
    packed.resize(base + c.n);
    for (int o = 0; o < c.cout; ++o)
      for (int ci = 0; ci < c.cin; ++ci)
        for (int t = 0; t < taps; ++t)
          packed[base + ((size_t)t * c.cin + ci) * c.cout + o] = net->weights[off + ((size_t)o * c.cin + ci) * taps + t];
    off += c.n;
    s->convs.push_back(c);
  }
  s->n_params = packed.size();
  build_tape(s);
  const size_t B = (size_t)max_batch;
  bool ok = ck(s, cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking), "stream") &&
            ck(s, cudaMalloc(&s->w, s->n_params * 4), "cudaMalloc") &&
            ck(s, cudaMalloc(&s->g, s->n_params * 4), "cudaMalloc") &&
            ck(s, cudaMalloc(&s->m, s->n_params * 4), "cudaMalloc") &&
            ck(s, cudaMalloc(&s->v, s->n_params * 4), "cudaMalloc") &&
            ck(s, cudaMalloc(&s->act, s->per_window * B * 4), "cudaMalloc activations") &&
            ck(s, cudaMalloc(&s->grad, s->per_window * B * 4), "cudaMalloc gradients") &&
            ck(s, cudaMalloc(&s->stats, s->stats_per_window * B * sizeof(float2)), "cudaMalloc") &&
            ck(s, cudaMalloc(&s->gmeans, (size_t)s->d.groups * B * sizeof(float2)), "cudaMalloc") &&
            ck(s, cudaMalloc(&s->part, gn_part_elems((int)B, s->d.groups) * sizeof(double2)), "cudaMalloc") &&
            ck(s, cudaMalloc(&s->loss_parts, 1024 * sizeof(double)), "cudaMalloc");
  if (ok)
    ok = ck(s, cudaMemcpy(s->w, packed.data(), s->n_params * 4, cudaMemcpyHostToDevice), "copy") &&
         ck(s, cudaMemset(s->g, 0, s->n_params * 4), "memset") && ck(s, cudaMemset(s->m, 0, s->n_params * 4), "memset") &&
         ck(s, cudaMemset(s->v, 0, s->n_params * 4), "memset");
  if (!ok) {
    const bool oom = s->err.find("memory") != std::string::npos;
    idf_student_destroy(s);
    return oom ? IDF_ENOMEM : IDF_ECUDA;
  }
  *out = s;
  return IDF_OK;
}

const char* idf_student_last_error(const idf_student* s) { return s ? s->err.c_str() : "null student"; }

idf_status idf_student_loss_grad(idf_student* s, const float* x_dev, const float* t_dev, int32_t n, double sigma,
                                 double* loss_out, void* stream) {
  if (!s || !x_dev || !t_dev || n < 1 || n > s->max_batch || !(sigma > 0)) return IDF_EINVAL;
  cudaStream_t st = s->st;
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, (cudaStream_t)stream);
  cudaStreamWaitEvent(st, ev, 0);
  const double sd = 0.5;
  const double s2 = sigma * sigma + sd * sd;
  const float c_skip = (float)(sd * sd / s2), c_out = (float)(sigma * sd / sqrt(s2)), c_in = (float)(1.0 / sqrt(s2));
  const int H = s->d.window;
  const int64_t npx = (int64_t)n * H * H;
  // ---- forward
  precond_in_kernel<<<grid_n(npx * s->d.in_ch, 256), 256, 0, st>>>(x_dev, c_in, npx, H * H, s->d.in_ch,
                                                                   A(s, s->buf_x));
  for (const SOp& op : s->ops) {
    const SBuf& bi = s->bufs[op.in];
    switch (op.kind) {
      case OP_CONV: {
        const SConv& c = s->convs[op.conv];
        launch_conv_f32(A(s, op.in), s->w + c.w_off, op.res >= 0 ? A(s, op.res) : nullptr, A(s, op.out), n, bi.H,
                        bi.H, c.cin, c.cout, c.ks, st);
        break;
      }
      case OP_GN:
        launch_gn_f32(A(s, op.in), n, bi.H, bi.C, s->d.groups, op.silu, s->part,
                      s->stats + op.stats_off * s->max_batch, A(s, op.out), st);
        break;
      case OP_POOL:
        launch_avgpool2_f32(A(s, op.in), n, bi.H, bi.C, A(s, op.out), st);
        break;
      case OP_UPCAT: {
        const SBuf& sk = s->bufs[op.in2];
        launch_upcat_f32(A(s, op.in), bi.C, A(s, op.in2), sk.C, n, sk.H, A(s, op.out), st);
        break;
      }
    }
  }
  // ---- loss and dF
  if (!ck(s, cudaMemsetAsync(s->grad, 0, s->per_window * s->max_batch * 4, st), "memset grad")) return IDF_ECUDA;
  const int nb = std::min<int64_t>(1024, (npx + 255) / 256);
  mse_kernel<<<nb, 256, 0, st>>>(x_dev, A(s, s->buf_F), t_dev, npx, c_skip, c_out, Gd(s, s->buf_F), s->loss_parts,
                                 H * H, s->d.in_ch);
  // ---- backward
  for (int oi = (int)s->ops.size() - 1; oi >= 0; --oi) {
    const SOp& op = s->ops[oi];
    const SBuf& bi = s->bufs[op.in];
    const SBuf& bo = s->bufs[op.out];
    switch (op.kind) {
      case OP_CONV: {
        const SConv& c = s->convs[op.conv];
        const int taps = c.ks * c.ks;
        // dRes
        if (op.res >= 0)
          add_kernel<<<grid_n((int64_t)n * bo.H * bo.H * bo.C, 256), 256, 0, st>>>(
              Gd(s, op.out), (int64_t)n * bo.H * bo.H * bo.C, Gd(s, op.res));
        // dW (split-K over pixels)
        const int K = taps * c.cin;
        const int64_t M = (int64_t)n * bi.H * bi.H;
        int chunks = (int)std::min<int64_t>(256, std::max<int64_t>(1, M / 2048));
        while (chunks > 1 && (size_t)chunks * K * c.cout > ((size_t)48 << 20)) chunks /= 2;
        const int64_t chunk_px = (M + chunks - 1) / chunks;
        if (!grow(s, &s->wpart, &s->wpart_cap, (size_t)chunks * K * c.cout)) return IDF_ENOMEM;
        dim3 gw((K + 63) / 64, (c.cout + 63) / 64, chunks);
        if (c.ks == 3)
          wgrad_partial_kernel<3><<<gw, 256, 0, st>>>(A(s, op.in), Gd(s, op.out), s->wpart, n, bi.H, bi.H, c.cin, c.cout, chunk_px);
        else
          wgrad_partial_kernel<1><<<gw, 256, 0, st>>>(A(s, op.in), Gd(s, op.out), s->wpart, n, bi.H, bi.H, c.cin, c.cout, chunk_px);
        wgrad_reduce_kernel<<<grid_n((int64_t)K * c.cout, 256), 256, 0, st>>>(s->wpart, chunks, (int64_t)K * c.cout,
                                                                          s->g + c.w_off);
        // dX = conv(dY, W^T), accumulated in place (the input of the network needs none)
        if (op.in != s->buf_x) {
          if (!grow(s, &s->wt, &s->wt_cap, c.n)) return IDF_ENOMEM;
          conv_w_transpose_kernel<<<grid_n((int64_t)c.n, 256), 256, 0, st>>>(s->w + c.w_off, s->wt, taps, c.cin, c.cout);
          launch_conv_f32(Gd(s, op.out), s->wt, Gd(s, op.in), Gd(s, op.in), n, bi.H, bi.H, c.cout, c.cin, c.ks, st);
        }
        break;
      }
      case OP_GN: {
        const int G = s->d.groups, Cg = bi.C / G, HW = bi.H * bi.H;
        int chunk_px = std::max(1, 4096 / Cg);
        int chunks = (HW + chunk_px - 1) / chunk_px;
        if (chunks > 1024) {
          chunk_px = (HW + 1023) / 1024;
          chunks = (HW + chunk_px - 1) / chunk_px;
        }
        const float2* stv = s->stats + op.stats_off * s->max_batch;
        gnb_partial_kernel<<<dim3(chunks, G, n), 256, 0, st>>>(A(s, op.in), Gd(s, op.out), stv, HW, bi.C, G, chunk_px,
                                                              op.silu, s->part);
        gnb_finalize_kernel<<<(n * G + 127) / 128, 128, 0, st>>>(s->part, n, chunks, HW, Cg, G, s->gmeans);
        const int64_t nel = (int64_t)n * HW * bi.C;
        gnb_apply_kernel<<<grid_n(nel, 256), 256, 0, st>>>(A(s, op.in), Gd(s, op.out), stv, s->gmeans, nel, HW, bi.C,
                                                          G, op.silu, Gd(s, op.in));
        break;
      }
      case OP_POOL:
        pool_bwd_kernel<<<grid_n((int64_t)n * bi.H * bi.H * bi.C, 256), 256, 0, st>>>(Gd(s, op.out), n, bi.H, bi.C,
                                                                                    Gd(s, op.in));
        break;
      case OP_UPCAT: {
        const SBuf& sk = s->bufs[op.in2];
        upcat_bwd_a_kernel<<<grid_n((int64_t)n * bi.H * bi.H * bi.C, 256), 256, 0, st>>>(Gd(s, op.out), bi.C, sk.C, n,
                                                                                       sk.H, Gd(s, op.in));
        upcat_bwd_skip_kernel<<<grid_n((int64_t)n * sk.H * sk.H * sk.C, 256), 256, 0, st>>>(
            Gd(s, op.out), bi.C, sk.C, (int64_t)n * sk.H * sk.H, Gd(s, op.in2));
        break;
      }
    }
  }
  std::vector<double> parts(nb);
  if (!ck(s, cudaMemcpyAsync(parts.data(), s->loss_parts, nb * sizeof(double), cudaMemcpyDeviceToHost, st), "copy loss") ||
      !ck(s, cudaStreamSynchronize(st), "student step"))
    return IDF_ECUDA;
  double tot = 0.0;
  for (double p : parts) tot += p;
  if (loss_out) *loss_out = tot / (double)npx;
  cudaEventRecord(ev, st);
  cudaStreamWaitEvent((cudaStream_t)stream, ev, 0);
  cudaEventDestroy(ev);
  return IDF_OK;
}

idf_status idf_student_adamw(idf_student* s, double lr, double beta1, double beta2, double eps, double weight_decay) {
  if (!s || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0)) return IDF_EINVAL;
  s->step++;
  const float bc1 = (float)(1.0 - pow(beta1, s->step)), bc2 = (float)(1.0 - pow(beta2, s->step));
  adamw_kernel<<<grid_n((int64_t)s->n_params, 256), 256, 0, s->st>>>(s->w, s->g, s->m, s->v, (int64_t)s->n_params,
                                                                    (float)lr, (float)beta1, (float)beta2, (float)eps,
                                                                    (float)weight_decay, bc1, bc2);
  if (!ck(s, cudaMemsetAsync(s->g, 0, s->n_params * 4, s->st), "memset") || !ck(s, cudaStreamSynchronize(s->st), "adamw"))
    return IDF_ECUDA;
  return IDF_OK;
}

idf_status idf_student_zero_grad(idf_student* s) {
  if (!s) return IDF_EINVAL;
  if (!ck(s, cudaMemsetAsync(s->g, 0, s->n_params * 4, s->st), "memset") || !ck(s, cudaStreamSynchronize(s->st), "sync"))
    return IDF_ECUDA;
  return IDF_OK;
}

idf_status idf_student_write(idf_student* s, const float* host_in, size_t n) {
  if (!s || !host_in || n != s->n_params) return IDF_EINVAL;
  std::vector<float> packed(s->n_params);
  size_t off = 0;
  for (const SConv& c : s->convs) {
    const int taps = c.ks * c.ks;
    for (int o = 0; o < c.cout; ++o)
      for (int ci = 0; ci < c.cin; ++ci)
        for (int t = 0; t < taps; ++t)
          packed[c.w_off + ((size_t)t * c.cin + ci) * c.cout + o] = host_in[off + ((size_t)o * c.cin + ci) * taps + t];
    off += c.n;
  }
  if (!ck(s, cudaStreamSynchronize(s->st), "sync") ||
      !ck(s, cudaMemcpy(s->w, packed.data(), s->n_params * 4, cudaMemcpyHostToDevice), "copy"))
    return IDF_ECUDA;
  return IDF_OK;
}

idf_status idf_student_read(const idf_student* sc, int32_t what, float* host_out, size_t n) {
  idf_student* s = const_cast<idf_student*>(sc);
  if (!s || !host_out || (what != 0 && what != 1) || n != s->n_params) return IDF_EINVAL;
  std::vector<float> packed(s->n_params);
  if (!ck(s, cudaStreamSynchronize(s->st), "sync") ||
      !ck(s, cudaMemcpy(packed.data(), what == 0 ? s->w : s->g, s->n_params * 4, cudaMemcpyDeviceToHost), "copy"))
    return IDF_ECUDA;
  size_t off = 0;
  for (const SConv& c : s->convs) {
    const int taps = c.ks * c.ks;
    for (int o = 0; o < c.cout; ++o)
      for (int ci = 0; ci < c.cin; ++ci)
        for (int t = 0; t < taps; ++t)
          host_out[off + ((size_t)o * c.cin + ci) * taps + t] = packed[c.w_off + ((size_t)t * c.cin + ci) * c.cout + o];
    off += c.n;
  }
  return IDF_OK;
}

}  // extern "C"
