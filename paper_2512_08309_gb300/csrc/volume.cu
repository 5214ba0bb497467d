// InfiniteDiffusion on Z^3: lazy, seed-consistent windowed sampling of an
// unbounded voxel volume (the method is defined on S = Z^d, Sec. 3.2; Alg. 3
// computes kappa per dimension; the conclusion names voxel volumes).
//
// The same scheme as the 2-D world, one dimension up: s^3 tiles aligned at
// multiples of the stride, window (i, j, l) covering tiles i..i+r-1 x
// j..j+r-1 x l..l+r-1; a query's cone walked back one blended step at a
// time over the tiles not cached; per step one batch of windows gathered,
// denoised and blended (Eq. 2 with the separable linear weight cubed) with
// the update and re-noise fused; finalized tiles of every step cached with
// LRU eviction of tiles the running query does not use.
//
// Noise N3(seed, level, step, x, y, z): Philox4x32-10 with counter (x, y, z,
// 2^31 + level 2^16 + step) -- the top bit keeps volumes apart from the 2-D
// counter (x, y, step, level) -- and the library's Box-Muller (noise.cuh).
//
// Denoiser: F(x) = conv3(silu(gn(conv3(x)))) (3x3x3, zero padding per
// window, C <= 8 hidden channels, GroupNorm), one CTA per window with the
// window and its hidden channels in shared memory (16^3 x 8 floats), or a
// closed-form test denoiser.  FP32.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <new>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/idf.h"
#include "internal.h"
#include "noise.cuh"

namespace idf {
namespace {

constexpr int64_t VLIM = (int64_t)1 << 20;  // |tile index| bound (21-bit keys)

__device__ __forceinline__ float normal3_at(uint64_t seed, uint32_t level, uint32_t step, int64_t x, int64_t y,
                                            int64_t z) {
  uint32_t c0 = (uint32_t)(uint64_t)x, c1 = (uint32_t)(uint64_t)y, c2 = (uint32_t)(uint64_t)z;
  uint32_t c3 = 0x80000000u + ((level & 0x7FFFu) << 16) + (step & 0xFFFFu);
  philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
  const float u1 = __fmul_rn((float)((c0 >> 8) + 1u), 0x1p-24f);
  const float l = series_ln(u1);
  const float s = __fsqrt_rn(__fmul_rn(-2.0f, l));
  return __fmul_rn(s, series_cos2pi((int32_t)(c1 >> 8)));
}

inline uint64_t vkey(int64_t a, int64_t b, int64_t c) {
  return ((uint64_t)(a + VLIM) << 42) | ((uint64_t)(b + VLIM) << 21) | (uint64_t)(c + VLIM);
}
inline int64_t kz(uint64_t k) { return (int64_t)(k >> 42) - VLIM; }
inline int64_t ky(uint64_t k) { return (int64_t)((k >> 21) & 0x1FFFFF) - VLIM; }
inline int64_t kx(uint64_t k) { return (int64_t)(k & 0x1FFFFF) - VLIM; }

// ---------------------------------------------------------------- kernels
struct VGather {
  const float* pool;
  const int32_t* win;     // [n][3] (i, j, l)
  const int32_t* slots;   // [n][r^3] slots of the J_k tiles (k >= 1)
  int n, H, s, r, step0;
  float c_in, sigma0;
  uint64_t seed;
  float* x;               // [n][H^3]
};

__global__ void vgather_kernel(VGather a) {
  const int64_t per = (int64_t)a.H * a.H * a.H, tot = per * a.n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx / per), p = (int)(idx % per);
    const int u = p / (a.H * a.H), v = (p / a.H) % a.H, w = p % a.H;
    float J;
    if (a.step0) {
      const int64_t Z = (int64_t)a.win[3 * b] * a.s + u, Y = (int64_t)a.win[3 * b + 1] * a.s + v,
                    X = (int64_t)a.win[3 * b + 2] * a.s + w;
      J = __fmul_rn(a.sigma0, normal3_at(a.seed, 0u, 0u, X, Y, Z));
    } else {
      const int m = u / a.s, q = v / a.s, o = w / a.s;
      const int sl = a.slots[(int64_t)b * a.r * a.r * a.r + (m * a.r + q) * a.r + o];
      J = a.pool[(int64_t)sl * a.s * a.s * a.s + ((u - m * a.s) * a.s + (v - q * a.s)) * a.s + (w - o * a.s)];
    }
    a.x[idx] = __fmul_rn(a.c_in, J);
  }
}

// F = conv2(silu(gn(conv1(x)))) for one window per CTA (H^3 <= 4096, C <= 8)
__global__ void __launch_bounds__(256) vnet_kernel(const float* __restrict__ x, const float* __restrict__ w1,
                                                   const float* __restrict__ w2, int H, int C, int G,
                                                   float* __restrict__ F) {
  extern __shared__ float sm[];
  const int N = H * H * H;
  float* xs = sm;            // [N]
  float* hid = sm + N;       // [C][N]
  __shared__ float red[2][8][32];
  __shared__ float st[2][8];
  const float* xw = x + (size_t)blockIdx.x * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) xs[i] = xw[i];
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int u = i / (H * H), v = (i / H) % H, t = i % H;
    for (int c = 0; c < C; ++c) {
      float acc = 0.0f;
      for (int dz = 0; dz < 3; ++dz)
        for (int dy = 0; dy < 3; ++dy)
          for (int dx = 0; dx < 3; ++dx) {
            const int zz = u + dz - 1, yy = v + dy - 1, xx = t + dx - 1;
            if (zz < 0 || zz >= H || yy < 0 || yy >= H || xx < 0 || xx >= H) continue;
            acc = fmaf(w1[c * 27 + (dz * 3 + dy) * 3 + dx], xs[(zz * H + yy) * H + xx], acc);
          }
      hid[c * N + i] = acc;
    }
  }
  __syncthreads();
  // GroupNorm statistics: two passes (mean, then squared deviations)
  const int cpg = C / G, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int pass = 0; pass < 2; ++pass) {
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int g = 0; g < G; ++g)
      for (int c = g * cpg; c < (g + 1) * cpg; ++c)
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
          const float v = hid[c * N + i];
          acc[g] += pass == 0 ? v : (v - st[0][g]) * (v - st[0][g]);
        }
    for (int g = 0; g < G; ++g) {
      float v = acc[g];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[pass][g][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < G) {
      float s = 0.0f;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[pass][threadIdx.x][w];
      const float n = (float)(cpg * N);
      st[pass][threadIdx.x] = pass == 0 ? s / n : rsqrtf(s / n + 1e-5f);
    }
    __syncthreads();
  }
  for (int c = 0; c < C; ++c) {
    const int g = c / cpg;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const float z = (hid[c * N + i] - st[0][g]) * st[1][g];
      hid[c * N + i] = z / (1.0f + expf(-z));
    }
  }
  __syncthreads();
  float* Fw = F + (size_t)blockIdx.x * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int u = i / (H * H), v = (i / H) % H, t = i % H;
    float acc = 0.0f;
    for (int c = 0; c < C; ++c)
      for (int dz = 0; dz < 3; ++dz)
        for (int dy = 0; dy < 3; ++dy)
          for (int dx = 0; dx < 3; ++dx) {
            const int zz = u + dz - 1, yy = v + dy - 1, xx = t + dx - 1;
            if (zz < 0 || zz >= H || yy < 0 || yy >= H || xx < 0 || xx >= H) continue;
            acc = fmaf(w2[c * 27 + (dz * 3 + dy) * 3 + dx], hid[c * N + (zz * H + yy) * H + xx], acc);
          }
    Fw[i] = acc;
  }
}

__global__ void vtest_kernel(int kind, const float* x, int n, int H, float* F) {
  const int64_t per = (int64_t)H * H * H, tot = per * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    float v = kind == 1 ? 0.5f : x[i];
    if (kind == 3) {
      const int p = (int)(i % per);
      const float fh = (float)H;
      v = __fadd_rn(v, __fadd_rn(__fsub_rn(__fdiv_rn((float)(p / (H * H)), fh), __fmul_rn(2.0f, __fdiv_rn((float)((p / H) % H), fh))),
                                 __fmul_rn(3.0f, __fdiv_rn((float)(p % H), fh))));
    }
    F[i] = v;
  }
}

struct VBlend {
  const float* pool;
  float* pool_out;
  const int32_t* tiles;     // [n][5] tz, ty, tx, slot_in (-1: noise), slot_out
  const int32_t* tile_wins; // [n][r^3] batch index of window (tz-m, ty-q, tx-o)
  const float* F;
  const float* w1;
  const float* invB1;
  int n, H, s, r, noise_in, noise_next;
  float c_skip, c_out, sigma0, sigma_next;
  uint32_t step_next;
  uint64_t seed;
};

__global__ void vblend_kernel(VBlend a) {
  const int t = blockIdx.x, s = a.s, r = a.r, H = a.H;
  const int32_t* tl = a.tiles + 5 * t;
  const int64_t HHH = (int64_t)H * H * H;
  for (int p = threadIdx.x; p < s * s * s; p += blockDim.x) {
    const int pa = p / (s * s), pb = (p / s) % s, pc = p % s;
    float acc = 0.0f;
    for (int m = r - 1; m >= 0; --m)
      for (int q = r - 1; q >= 0; --q)
        for (int o = r - 1; o >= 0; --o) {
          const int u = m * s + pa, v = q * s + pb, w = o * s + pc;
          const int wb = a.tile_wins[(int64_t)t * r * r * r + (m * r + q) * r + o];
          const float f = a.F[(int64_t)wb * HHH + ((int64_t)u * H + v) * H + w];
          acc = __fadd_rn(acc, __fmul_rn(__fmul_rn(__fmul_rn(a.w1[u], a.w1[v]), a.w1[w]), f));
        }
    const int64_t Z = (int64_t)tl[0] * s + pa, Y = (int64_t)tl[1] * s + pb, X = (int64_t)tl[2] * s + pc;
    const float Jk = a.noise_in ? __fmul_rn(a.sigma0, normal3_at(a.seed, 0u, 0u, X, Y, Z))
                                : a.pool[(int64_t)tl[3] * s * s * s + p];
    const float avg = __fmul_rn(__fmul_rn(__fmul_rn(acc, a.invB1[pa]), a.invB1[pb]), a.invB1[pc]);
    float J = __fadd_rn(__fmul_rn(a.c_skip, Jk), __fmul_rn(a.c_out, avg));
    if (a.noise_next) J = __fadd_rn(J, __fmul_rn(a.sigma_next, normal3_at(a.seed, 0u, a.step_next, X, Y, Z)));
    a.pool_out[(int64_t)tl[4] * s * s * s + p] = J;
  }
}

__global__ void vassemble_kernel(const float* pool, const int32_t* slots, int64_t tz0, int64_t ty0, int64_t tx0,
                                 int ntz, int nty, int ntx, int s, int64_t z0, int64_t y0, int64_t x0, int d, int h,
                                 int w, float* out) {
  const int64_t tot = (int64_t)d * h * w;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t Z = z0 + i / ((int64_t)h * w), Y = y0 + (i / w) % h, X = x0 + i % w;
    const int64_t a = fdiv(Z, s) - tz0, b = fdiv(Y, s) - ty0, c = fdiv(X, s) - tx0;
    const int sl = slots[(a * nty + b) * ntx + c];
    out[i] = pool[(int64_t)sl * s * s * s + ((Z - fdiv(Z, s) * s) * s + (Y - fdiv(Y, s) * s)) * s + (X - fdiv(X, s) * s)];
  }
}

int vgrid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32)); }

struct VRound {
  std::vector<int32_t> win, slots, tiles, tile_wins;
};

}  // namespace
}  // namespace idf

using namespace idf;

struct idf_volume {
  uint64_t seed = 0;
  idf_volume_desc d{};
  int H = 0, s = 0, r = 0, K = 0;
  std::vector<double> sig, cs, co, ci;
  float *w1 = nullptr, *invB1 = nullptr, *wn1 = nullptr, *wn2 = nullptr;
  // cache
  int64_t n_slots = 0;
  float* pool = nullptr;
  std::vector<std::unordered_map<uint64_t, int32_t>> map;  // [step] key -> slot
  std::vector<int32_t> slot_step;
  std::vector<uint64_t> slot_key, lru_t, pin;
  std::vector<int32_t> free_list;
  uint64_t tick = 0, epoch = 1;
  // buffers
  float *x = nullptr, *F = nullptr, *out = nullptr;
  size_t x_cap = 0, F_cap = 0, out_cap = 0;
  int32_t* tab = nullptr;
  size_t tab_cap = 0;
  cudaStream_t st = nullptr;
  int64_t windows = 0, tiles = 0, hits = 0, misses = 0;
  std::string err;
};

namespace {

bool vgrow(idf_volume* V, void** p, size_t* cap, size_t bytes) {
  if (bytes <= *cap) return true;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    V->err = "cudaMalloc failed";
    return false;
  }
  *cap = bytes;
  return true;
}

int32_t valloc(idf_volume* V) {
  if (!V->free_list.empty()) {
    const int32_t sl = V->free_list.back();
    V->free_list.pop_back();
    return sl;
  }
  // least recently used slot not used by the running query
  int32_t best = -1;
  for (int64_t sl = 0; sl < V->n_slots; ++sl)
    if (V->pin[sl] != V->epoch && (best < 0 || V->lru_t[sl] < V->lru_t[best])) best = (int32_t)sl;
  if (best >= 0) V->map[V->slot_step[best]].erase(V->slot_key[best]);
  return best;
}

idf_status vquery(idf_volume* V, int64_t x0, int64_t y0, int64_t z0, int w, int h, int d, float* out_dev) {
  const int K = V->K, r = V->r, s = V->s, H = V->H;
  bool lost = false;
  auto slot_at = [&](int k, uint64_t key) -> int32_t {
    auto it = V->map[k].find(key);
    if (it == V->map[k].end()) {
      lost = true;
      return 0;
    }
    return it->second;
  };
  V->epoch++;
  const int64_t tz0 = fdiv(z0, s), ty0 = fdiv(y0, s), tx0 = fdiv(x0, s);
  const int64_t tz1 = fdiv(z0 + d - 1, s), ty1 = fdiv(y0 + h - 1, s), tx1 = fdiv(x0 + w - 1, s);
  const int64_t lim = VLIM - (int64_t)(K + 2) * r;
  for (int64_t v : {tz0, ty0, tx0, tz1, ty1, tx1})
    if (v <= -lim || v >= lim) {
      V->err = "region too far from the origin";
      return IDF_EINVAL;
    }
  // cone, last step first
  std::vector<std::vector<uint64_t>> missing(K + 1);
  std::vector<std::vector<uint64_t>> wins(K);
  std::vector<uint64_t> need;
  for (int64_t a = tz0; a <= tz1; ++a)
    for (int64_t b = ty0; b <= ty1; ++b)
      for (int64_t c = tx0; c <= tx1; ++c) need.push_back(vkey(a, b, c));
  for (int k = K; k >= 1; --k) {
    std::sort(need.begin(), need.end());
    for (uint64_t t : need) {
      auto it = V->map[k].find(t);
      if (it != V->map[k].end()) {
        V->lru_t[it->second] = ++V->tick;
        V->pin[it->second] = V->epoch;
        V->hits++;
      } else {
        missing[k].push_back(t);
      }
    }
    V->misses += (int64_t)missing[k].size();
    std::unordered_set<uint64_t> ws;
    for (uint64_t t : missing[k])
      for (int m = 0; m < r; ++m)
        for (int q = 0; q < r; ++q)
          for (int o = 0; o < r; ++o) ws.insert(vkey(kz(t) - m, ky(t) - q, kx(t) - o));
    wins[k - 1].assign(ws.begin(), ws.end());
    std::sort(wins[k - 1].begin(), wins[k - 1].end());
    std::unordered_set<uint64_t> ns;
    if (k > 1)
      for (uint64_t wv : wins[k - 1])
        for (int m = 0; m < r; ++m)
          for (int q = 0; q < r; ++q)
            for (int o = 0; o < r; ++o) ns.insert(vkey(kz(wv) + m, ky(wv) + q, kx(wv) + o));
    need.assign(ns.begin(), ns.end());
  }
  // slots for the missing tiles (undone on exhaustion)
  std::vector<std::pair<int, uint64_t>> ins;
  for (int k = 1; k <= K; ++k)
    for (uint64_t t : missing[k]) {
      const int32_t sl = valloc(V);
      if (sl < 0) {
        for (auto& e : ins) {
          const int32_t os = V->map[e.first][e.second];
          V->map[e.first].erase(e.second);
          V->free_list.push_back(os);
        }
        V->err = "tile cache too small for this query's working set";
        return IDF_ENOMEM;
      }
      V->map[k][t] = sl;
      V->slot_step[sl] = k;
      V->slot_key[sl] = t;
      V->lru_t[sl] = ++V->tick;
      V->pin[sl] = V->epoch;
      ins.emplace_back(k, t);
    }
  // run the steps
  for (int k = 0; k < K; ++k) {
    const auto& wk = wins[k];
    const int nw = (int)wk.size();
    if (nw == 0) continue;
    const int r3 = r * r * r;
    VRound R;
    std::unordered_map<uint64_t, int32_t> widx;
    for (int i = 0; i < nw; ++i) {
      widx[wk[i]] = i;
      R.win.push_back((int32_t)kz(wk[i]));
      R.win.push_back((int32_t)ky(wk[i]));
      R.win.push_back((int32_t)kx(wk[i]));
      if (k >= 1)
        for (int m = 0; m < r; ++m)
          for (int q = 0; q < r; ++q)
            for (int o = 0; o < r; ++o) R.slots.push_back(slot_at(k, vkey(kz(wk[i]) + m, ky(wk[i]) + q, kx(wk[i]) + o)));
    }
    for (uint64_t t : missing[k + 1]) {
      R.tiles.push_back((int32_t)kz(t));
      R.tiles.push_back((int32_t)ky(t));
      R.tiles.push_back((int32_t)kx(t));
      R.tiles.push_back(k >= 1 ? slot_at(k, t) : -1);
      R.tiles.push_back(slot_at(k + 1, t));
      for (int m = 0; m < r; ++m)
        for (int q = 0; q < r; ++q)
          for (int o = 0; o < r; ++o) {
            auto it = widx.find(vkey(kz(t) - m, ky(t) - q, kx(t) - o));
            if (it == widx.end()) lost = true;
            R.tile_wins.push_back(it == widx.end() ? 0 : it->second);
          }
    }
    if (lost) {
      V->err = "internal: tile or window missing from the plan";
      return IDF_EINTERNAL;
    }
    const size_t n1 = R.win.size(), n2 = R.slots.size(), n3 = R.tiles.size(), n4 = R.tile_wins.size();
    if (!vgrow(V, (void**)&V->tab, &V->tab_cap, (n1 + n2 + n3 + n4) * 4) ||
        !vgrow(V, (void**)&V->x, &V->x_cap, (size_t)nw * H * H * H * 4) ||
        !vgrow(V, (void**)&V->F, &V->F_cap, (size_t)nw * H * H * H * 4))
      return IDF_ENOMEM;
    std::vector<int32_t> all;
    all.reserve(n1 + n2 + n3 + n4);
    all.insert(all.end(), R.win.begin(), R.win.end());
    all.insert(all.end(), R.slots.begin(), R.slots.end());
    all.insert(all.end(), R.tiles.begin(), R.tiles.end());
    all.insert(all.end(), R.tile_wins.begin(), R.tile_wins.end());
    if (cudaMemcpy(V->tab, all.data(), all.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) return IDF_ECUDA;
    VGather g{};
    g.pool = V->pool;
    g.win = V->tab;
    g.slots = V->tab + n1;
    g.n = nw; g.H = H; g.s = s; g.r = r; g.step0 = k == 0;
    g.c_in = (float)V->ci[k];
    g.sigma0 = (float)V->sig[0];
    g.seed = V->seed;
    g.x = V->x;
    vgather_kernel<<<vgrid((int64_t)nw * H * H * H), 256, 0, V->st>>>(g);
    if (V->d.test_denoiser) {
      vtest_kernel<<<vgrid((int64_t)nw * H * H * H), 256, 0, V->st>>>(V->d.test_denoiser, V->x, nw, H, V->F);
    } else {
      const size_t smem = (size_t)(1 + V->d.channels) * H * H * H * 4;
      cudaFuncSetAttribute(vnet_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      vnet_kernel<<<nw, 256, smem, V->st>>>(V->x, V->wn1, V->wn2, H, V->d.channels, V->d.groups, V->F);
    }
    V->windows += nw;
    VBlend b{};
    b.pool = V->pool;
    b.pool_out = V->pool;
    b.tiles = V->tab + n1 + n2;
    b.tile_wins = V->tab + n1 + n2 + n3;
    b.F = V->F;
    b.w1 = V->w1;
    b.invB1 = V->invB1;
    b.n = (int)(n3 / 5); b.H = H; b.s = s; b.r = r;
    b.noise_in = k == 0;
    b.noise_next = k + 1 < K;
    b.c_skip = (float)V->cs[k];
    b.c_out = (float)V->co[k];
    b.sigma0 = (float)V->sig[0];
    b.sigma_next = k + 1 < K ? (float)V->sig[k + 1] : 0.0f;
    b.step_next = (uint32_t)(k + 1);
    b.seed = V->seed;
    if (b.n > 0) vblend_kernel<<<b.n, 256, 0, V->st>>>(b);
    V->tiles += b.n;
    if (cudaStreamSynchronize(V->st) != cudaSuccess) {
      V->err = cudaGetErrorString(cudaGetLastError());
      return IDF_ECUDA;
    }
  }
  // assemble the final tiles over the box
  const int ntz = (int)(tz1 - tz0 + 1), nty = (int)(ty1 - ty0 + 1), ntx = (int)(tx1 - tx0 + 1);
  std::vector<int32_t> sl((size_t)ntz * nty * ntx);
  for (int a = 0; a < ntz; ++a)
    for (int b = 0; b < nty; ++b)
      for (int c = 0; c < ntx; ++c) sl[((size_t)a * nty + b) * ntx + c] = slot_at(K, vkey(tz0 + a, ty0 + b, tx0 + c));
  if (lost) {
    V->err = "internal: final tile missing";
    return IDF_EINTERNAL;
  }
  if (!vgrow(V, (void**)&V->tab, &V->tab_cap, sl.size() * 4)) return IDF_ENOMEM;
  if (cudaMemcpy(V->tab, sl.data(), sl.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) return IDF_ECUDA;
  vassemble_kernel<<<vgrid((int64_t)d * h * w), 256, 0, V->st>>>(V->pool, V->tab, tz0, ty0, tx0, ntz, nty, ntx, s, z0,
                                                                 y0, x0, d, h, w, out_dev);
  if (cudaStreamSynchronize(V->st) != cudaSuccess) {
    V->err = cudaGetErrorString(cudaGetLastError());
    return IDF_ECUDA;
  }
  return IDF_OK;
}

}  // namespace

extern "C" {

void idf_volume_destroy(idf_volume* V) {
  if (!V) return;
  if (V->st) cudaStreamSynchronize(V->st);
  cudaFree(V->w1); cudaFree(V->invB1); cudaFree(V->wn1); cudaFree(V->wn2); cudaFree(V->pool);
  cudaFree(V->x); cudaFree(V->F); cudaFree(V->out); cudaFree(V->tab);
  if (V->st) cudaStreamDestroy(V->st);
  delete V;
}

idf_status idf_volume_create(uint64_t seed, const idf_volume_desc* d, int32_t device, size_t cache_bytes,
                             idf_volume** out) {
  if (!out) return IDF_EINVAL;
  *out = nullptr;
  if (!d || d->window < 2 || d->stride < 1 || d->window % d->stride || d->steps < 1 || d->steps > 64 ||
      !(d->sigma_max > 0) || !(d->sigma_min > 0) || !(d->rho > 0) || !(d->sigma_data > 0) ||
      !(d->blend_eps > 0) || d->test_denoiser < 0 || d->test_denoiser > 3)
    return IDF_EINVAL;
  if (d->test_denoiser == 0) {
    const int H = d->window;
    if (d->channels < 1 || d->channels > 8 || d->groups < 1 || d->channels % d->groups || H * H * H > 4096 ||
        (size_t)(1 + d->channels) * H * H * H * 4 > 200 * 1024)
      return IDF_EINVAL;
    if (!d->weights || d->n_weights != (size_t)d->channels * 27 * 2) return IDF_EMODEL;
  }
  std::unique_ptr<idf_volume> V(new (std::nothrow) idf_volume());
  if (!V) return IDF_ENOMEM;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return IDF_ECUDA;
  }
  V->seed = seed;
  V->d = *d;
  V->d.weights = nullptr;
  V->H = d->window;
  V->s = d->stride;
  V->r = d->window / d->stride;
  V->K = d->steps;
  const int K = V->K;
  const double a = pow(d->sigma_max, 1.0 / d->rho), b = pow(d->sigma_min, 1.0 / d->rho);
  for (int k = 0; k < K; ++k) {
    const double sg = K == 1 ? d->sigma_max : pow(a + (double)k / (K - 1) * (b - a), d->rho);
    const double s2 = sg * sg + d->sigma_data * d->sigma_data;
    V->sig.push_back(sg);
    V->cs.push_back(d->sigma_data * d->sigma_data / s2);
    V->co.push_back(sg * d->sigma_data / sqrt(s2));
    V->ci.push_back(1.0 / sqrt(s2));
  }
  std::vector<double> w1d(V->H);
  std::vector<float> w1(V->H), ib(V->s);
  const double c = (V->H - 1) / 2.0;
  for (int u = 0; u < V->H; ++u) {
    w1d[u] = 1.0 - (1.0 - d->blend_eps) * fabs(u - c) / c;
    w1[u] = (float)w1d[u];
  }
  for (int q = 0; q < V->s; ++q) {
    double sum = 0;
    for (int m = 0; m < V->r; ++m) sum += w1d[q + m * V->s];
    ib[q] = (float)(1.0 / sum);
  }
  const size_t tile = (size_t)V->s * V->s * V->s;
  V->n_slots = (int64_t)((cache_bytes ? cache_bytes : ((size_t)1 << 30)) / (tile * 4));
  if (V->n_slots < 1 || V->n_slots > INT32_MAX) return IDF_EINVAL;
  if (cudaStreamCreateWithFlags(&V->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&V->w1, V->H * 4) != cudaSuccess || cudaMalloc(&V->invB1, V->s * 4) != cudaSuccess ||
      cudaMalloc(&V->pool, (size_t)V->n_slots * tile * 4) != cudaSuccess) {
    cudaGetLastError();
    idf_volume_destroy(V.release());
    return IDF_ENOMEM;
  }
  cudaMemcpy(V->w1, w1.data(), V->H * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(V->invB1, ib.data(), V->s * 4, cudaMemcpyHostToDevice);
  if (d->test_denoiser == 0) {
    const size_t n = (size_t)d->channels * 27;
    if (cudaMalloc(&V->wn1, n * 4) != cudaSuccess || cudaMalloc(&V->wn2, n * 4) != cudaSuccess) {
      cudaGetLastError();
      idf_volume_destroy(V.release());
      return IDF_ENOMEM;
    }
    cudaMemcpy(V->wn1, d->weights, n * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(V->wn2, d->weights + n, n * 4, cudaMemcpyHostToDevice);
  }
  V->map.resize(K + 1);
  V->slot_step.assign(V->n_slots, 0);
  V->slot_key.assign(V->n_slots, 0);
  V->lru_t.assign(V->n_slots, 0);
  V->pin.assign(V->n_slots, 0);
  for (int64_t i = V->n_slots - 1; i >= 0; --i) V->free_list.push_back((int32_t)i);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    idf_volume_destroy(V.release());
    return IDF_ECUDA;
  }
  *out = V.release();
  return IDF_OK;
}

idf_status idf_volume_query(idf_volume* V, int64_t x0, int64_t y0, int64_t z0, int32_t w, int32_t h, int32_t d,
                            float* out_host) {
  if (!V || !out_host || w < 1 || h < 1 || d < 1 || (double)w * h * d > 1073741824.0) return IDF_EINVAL;
  const size_t n = (size_t)w * h * d;
  if (!vgrow(V, (void**)&V->out, &V->out_cap, n * 4)) return IDF_ENOMEM;
  const idf_status s = vquery(V, x0, y0, z0, w, h, d, V->out);
  if (s != IDF_OK) return s;
  if (cudaMemcpy(out_host, V->out, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return IDF_ECUDA;
  return IDF_OK;
}

idf_status idf_volume_stats(const idf_volume* V, int64_t out[4]) {
  if (!V || !out) return IDF_EINVAL;
  out[0] = V->windows;
  out[1] = V->tiles;
  out[2] = V->hits;
  out[3] = V->misses;
  return IDF_OK;
}

const char* idf_volume_last_error(const idf_volume* V) { return V ? V->err.c_str() : "null volume"; }

}  // extern "C"
