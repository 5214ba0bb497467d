// Internal declarations shared by the translation units of libidf.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <map>
#include <vector>

namespace idf {

typedef __nv_bfloat16 bf16;

// Floor division and modulo for possibly negative numerators, positive d.
__host__ __device__ __forceinline__ int64_t fdiv(int64_t a, int64_t d) {
  int64_t q = a / d;
  return (a % d != 0 && a < 0) ? q - 1 : q;
}
__host__ __device__ __forceinline__ int64_t fmod_pos(int64_t a, int64_t d) {
  return a - fdiv(a, d) * d;
}

// ------------------------------------------------------------------ status
struct Err {
  int code = 0;  // idf_status
  std::string msg;
};

// ---------------------------------------------------------------- sampler
// A tile is stride x stride float32 values stored contiguously in one slot of
// the tile pool.  slot < 0 means "not stored": the J_0 noise tile, computed on
// the fly.
struct GatherArgs {
  const float* pool;         // tile pool base
  const int32_t* win_slots;  // [n_win][r][r] slots of the tiles a window covers (row-major)
  const int32_t* win_ij;     // [n_win][2] window indices (i row, j column)
  int n_win, H, s, r, in_ch;
  float c_in, sigma0;        // step-0 inputs are sigma0 * N(seed, level, 0, .)
  int noise_step0;           // 1: inputs are the J_0 noise
  uint64_t seed;
  uint32_t level;
  const float* cond;         // dense conditioning image (parent result) or null
  int64_t cond_x0, cond_y0;  // its origin on the parent grid
  int64_t cond_pitch;
  int cond_w, cond_h, cond_f;
  float* x_in;               // [n_win][H][H][in_ch] float32 (NHWC)
  int* err_flag;             // device flag set on out-of-range reads
  float* xs = nullptr;       // optional [n_win][H][H]: the window state J_k[R_i] (multi-step rounds)
};
void launch_gather(const GatherArgs& a, cudaStream_t st);

// One window-local sampler step inside a multi-step round (blending only at
// selected noise levels): D = c_skip xs + c_out F per window pixel; with
// last, F = D (the round's result, blended next); otherwise xs = D +
// sigma_next N(seed, level, step_next, .) (absolute coordinates) and the
// network input channel 0 becomes c_in_next xs.
struct WindowStepArgs {
  float* x_in;               // [n_win][H][H][in_ch]
  float* xs;                 // [n_win][H][H]
  float* F;                  // [n_win][H][H]
  const int32_t* win_ij;     // [n_win][2]
  int n_win, H, s, in_ch;
  float c_skip, c_out, c_in_next, sigma_next;
  int noise, last;
  uint32_t step_next;
  uint64_t seed;
  uint32_t level;
};
void launch_window_step(const WindowStepArgs& a, cudaStream_t st);

// Per-window conditioning bias: window b = (i, j) gets y_d = z_d + amp
// N(seed, level, COND_STEP + d, j, i) and bias[b][c] = sum_d E[c][d] y_d.
constexpr uint32_t COND_STEP = 0x7FFF0000u;
void launch_cond_bias(const int32_t* win_ij, int n, uint64_t seed, uint32_t level, const float* z, float amp,
                      const float* E, int D, int C, float* bias, cudaStream_t st);
// AutoGuidance: F = Fg + w (F - Fg), n values
void launch_guidance(float* F, const float* Fg, int64_t n, float w, cudaStream_t st);

struct BlendArgs {
  const float* pool;
  float* pool_out;
  const int32_t* tiles;      // [n_tiles][4]: ty, tx, slot_in (J_k, -1 for noise), slot_out
  const int32_t* tile_wins;  // [n_tiles][r][r] batch index of window (ty-m, tx-n), m,n = 0..r-1
  const float* F;            // [n_win][H][H] float32 network outputs
  const float* w1;           // [H] blend weights per axis
  const float* invB1;        // [s] 1 / per-axis weight sum
  int n_tiles, H, s, r;
  float c_skip, c_out, c_in, sigma_next, sigma0;
  int noise_next;            // 1: add sigma_next N(seed, level, k+1, .)
  int noise_in;              // 1: J_k is the J_0 noise (slot_in < 0)
  uint32_t step_next;
  uint64_t seed;
  uint32_t level;
};
void launch_blend(const BlendArgs& a, cudaStream_t st);

// Closed-form test denoisers on x_in (NHWC, in_ch channels) -> F [n][H][H].
void launch_test_denoiser(int kind, const float* x_in, int n, int H, int in_ch, float* F,
                          cudaStream_t st);

// Copy finalized tiles into a dense row-major rect.
void launch_assemble(const float* pool, const int32_t* tile_slots, int64_t ty0, int64_t tx0,
                     int nty, int ntx, int s, int64_t y0, int64_t x0, int h, int w, float* out,
                     int64_t pitch, cudaStream_t st);

void launch_noise_fill(uint64_t seed, uint32_t level, uint32_t step, int64_t x0, int64_t y0,
                       int w, int h, float* out, int64_t pitch, cudaStream_t st);

// NCHW <-> NHWC helpers for the single-channel window images.
void launch_nchw_to_nhwc(const float* x, int n, int c, int hw, float* y, cudaStream_t st);
void launch_nhwc_to_nchw(const float* x, int n, int c, int hw, float* y, cudaStream_t st);

// --------------------------------------------------------------- decode
struct DecodeArgs {
  const float* L;  int64_t lx0, ly0, lpitch; int lw, lh;
  const float* H;  int64_t hx0, hy0, hpitch; int hw, hh;
  int64_t x0, y0; int w, h;
  float* out; int64_t pitch;
  int f, R;
  float low_mu, low_scale, res_scale;
  const float* taps;      // device, 2R+1
  float* D;               // scratch coarse (qh + 2R) x (qw + 2R)
  float* T;               // scratch coarse (qh + 2R) x qw
  float* Lhat;            // scratch coarse qh x qw
  int64_t qx0, qy0; int qw, qh;   // coarse rect of L^ that the output reads
};
void launch_decode(const DecodeArgs& a, cudaStream_t st);
// dst[y * w + x] = fixture[((y0 + y) mod P) * P + ((x0 + x) mod P)] (a
// periodic low-band fixture read over a rect of the low-resolution grid)
void launch_fixture_gather(const float* fixture, int64_t P, int64_t x0, int64_t y0, int w, int h, float* dst,
                           cudaStream_t st);

// --------------------------------------------------------------- profiling
// Optional per-launch CUDA-event timing on the launching stream, grouped by
// kernel class, with the algorithmic FLOPs / bytes of each launch.
enum ProfKind { PK_CONV_TC = 0, PK_CONV_SIMT, PK_GROUPNORM, PK_ATTENTION, PK_RESAMPLE,
                PK_GATHER, PK_DENOISE_TEST, PK_BLEND, PK_ASSEMBLE, PK_DECODE, PK_COUNT };
// One timed launch: flops = the class's work (FLOPs of the convolutions
// and attention; for the blend, the normal samples it draws), bytes = its
// algorithmic memory traffic.
struct ProfRec {
  int kind;
  cudaEvent_t a, b;
  double flops, bytes;
};
struct Prof {
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  double ms[PK_COUNT] = {0}, flops[PK_COUNT] = {0}, bytes[PK_COUNT] = {0};
  int64_t launches[PK_COUNT] = {0};
  cudaEvent_t ev() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  // start a record; returns its index or -1
  int begin(int kind, cudaStream_t st, double fl, double by) {
    if (!on) return -1;
    ProfRec r{kind, ev(), ev(), fl, by};
    cudaEventRecord(r.a, st);
    recs.push_back(r);
    return (int)recs.size() - 1;
  }
  void end(int idx, cudaStream_t st) {
    if (idx >= 0) cudaEventRecord(recs[idx].b, st);
  }
  // fold completed records into the totals (call after a synchronize)
  void resolve() {
    for (auto& r : recs) {
      float t = 0;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        ms[r.kind] += t;
        flops[r.kind] += r.flops;
        bytes[r.kind] += r.bytes;
        launches[r.kind]++;
        if (r.kind == 0) {
          // tensor-core convolutions by launch shape (FLOPs, algorithmic
          // bytes): a per-launch roofline needs both
          auto& e = conv_shapes[{r.flops, r.bytes}];
          e.first++;
          e.second += t;
        }
      }
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
    cudaGetLastError();
  }
  void reset() {
    for (int k = 0; k < PK_COUNT; ++k) ms[k] = flops[k] = bytes[k] = 0, launches[k] = 0;
    conv_shapes.clear();
  }
  std::map<std::pair<double, double>, std::pair<int64_t, double>> conv_shapes;  // -> (launches, ms)
  ~Prof() {
    for (auto e : pool) cudaEventDestroy(e);
    for (auto& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  }
};

// --------------------------------------------------------------- UNet
struct UNet;  // opaque, unet.cu
struct UNetDesc {
  int levels;
  std::vector<int> ch;
  int in_ch, out_ch, groups, attn, heads, window;
  int cond_dim = 0;  // > 0: a conditioning embedding (ch[0], cond_dim, 1, 1) declared last
};
// Shapes (Cout, Cin, kh, kw) in declaration order.
std::vector<std::vector<int>> unet_param_shapes(const UNetDesc& d);
// Create / destroy; weights are host float32 in declaration order.
// With an arena, the activation buffers are carved from it (levels of a
// world run one after another and share one arena); otherwise allocated.
UNet* unet_create(const UNetDesc& d, const float* w_host, int precision, int max_batch,
                  Err* err, void* arena = nullptr, size_t arena_bytes = 0);
size_t unet_arena_bytes(const UNetDesc& d, int precision, int max_batch);
void unet_destroy(UNet* u);
int unet_max_batch(const UNet* u);
size_t unet_bytes_per_window(const UNetDesc& d, int precision);
// x_in NHWC float32 [n][H][H][in_ch] -> F [n][H][H] float32 (out_ch = 1);
// bias: optional [n][ch[0]] per-window conditioning bias added after the in-conv.
bool unet_forward(UNet* u, const float* x_in, int n, float* F, cudaStream_t st, Err* err,
                  const float* bias = nullptr);
int64_t unet_launches(const UNet* u);
// device status word set by bounded device-side waits that ran out
int* unet_status(const UNet* u);
// fuse_groupnorm (IDF_TF32 only): GroupNorm and SiLU inside the tensor-core
// convolutions' operand path;
// wait_limit: clock64 cycles a bounded device wait may take (0: about
// 0.5 s); graphs: replay repeated forwards (same x_in, n, F, bias) as one
// CUDA graph launch (bitwise the same kernels and arguments)
// pairs: tensor-core convolutions on clusters of two CTAs (cta_group::2)
// wherever the operands and shape allow them
void unet_set_options(UNet* u, bool fuse_groupnorm, long long wait_limit, bool autotune = false,
                      bool graphs = false, bool pairs = false);
// CUDA-graph summary: forwards captured, forwards replayed, kernels those
// replays ran
void unet_graph_stats(const UNet* u, int64_t* captures, int64_t* replays, int64_t* kernels);
// autotuner summary: layer classes tuned, and those whose fastest tile shape
// differs from the built-in choice
void unet_autotune_stats(const UNet* u, int* tuned, int* changed);
void unet_set_prof(UNet* u, Prof* p);

// tcgen05 conv (conv_tc.cu)
bool conv_tc_supported(int cin, int cout, int ks);
// co-resident clusters of two CTAs the pair kernels launch with (0 before the first)
int conv_tc_pair_clusters();
// Self-attention on the tensor cores (bfloat16 products, float32 softmax and
// accumulation): qkv float32 [n][Tn][3C] (Q, K, V; head h at channels
// 64h .. 64h + 63 of each), out [n][Tn][C] as bfloat16, or as tf32-rounded
// float32 (out_tf32).  Tn = 256 and head width 64 only.
bool attention_tc_supported(int Tn, int dh);
bool attention_tc_forward(const float* qkv, int n, int C, int heads, void* out, bool out_tf32, int* status,
                          long long wait_limit, cudaStream_t st, std::string* err);
bool conv_tc_shape_ok(int H, int W);

// Geometry options of a tensor-core convolution: the input offset of tap
// (0, 0) (the default -ks/2 centres the kernel), a phase-scattered output
// (pixel (y, x) of the H x W grid is stored at (2y + py, 2x + px) of a
// 2H x 2W output: one phase of a convolution over a nearest-upsampled
// input), and a half-resolution residual (pixel (y, x) adds element
// (y/2, x/2) of an H/2 x W/2 tensor: a nearest-upsampled residual).
struct TcGeom {
  int oy = 0, ox = 0;
  int out_up = 0, py = 0, px = 0;
  int res_up = 0;
};

// Operand transform of a TF32 tensor-core convolution: x is a raw float32
// tensor; on its way to the tensor cores each real pixel's value becomes
// tf32(silu((v - mean) * rstd)) (or without SiLU) with the (mean, rstd) =
// stats[window * G + (coff + channel) / cpg] of its GroupNorm group, or,
// with stats null, just tf32(v).  Zero padding stays zero.  A folded x2 is
// read as it is.
struct TcXf {
  const float2* stats = nullptr;
  int G = 1, cpg = 1, coff = 0, silu = 0;
};

// Tile shape of a tensor-core convolution: BN output channels per tile, MT
// 128-pixel M tiles per work unit, dxr = 1 to stage one 130-pixel box per
// kernel row (3x3 on 128-pixel rows, BN = 64) or 0 for a box per tap.  Zero
// / negative fields take the built-in choice; every valid shape gives the
// same result bit for bit (the K order of each output element is fixed).
struct TcTile {
  int bn = 0, mt = 0, dxr = -1;
  int pair = -1;  // 1: clusters of two CTAs issuing cta_group::2 products; 0 / -1: one CTA
};
// The valid tile shapes of a convolution (for autotuning).
std::vector<TcTile> conv_tc_tiles(int H, int W, int Cin, int Cout, int ks, bool split, bool xf,
                                  const TcGeom* geom);

// y (float32 NHWC, Cout) = conv(x) over (tap, Cin) [+ the 1x1 conv of x2
// over Cin2, folded into the same accumulator] [+ res], x / x2 in bfloat16
// (with low parts for the compensated split) or tf32-rounded float32.  With
// bstats the epilogue also writes GroupNorm block partials of y.  Returns
// false with err set when the shape or combination is not supported or a
// launch fails.
bool conv_tc_forward(const void* x, const void* w, const void* x_lo, const void* w_lo, const float* res,
                     float* y, float2* bstats, int n, int H, int W, int Cin, int Cout, int ks, int* status,
                     cudaStream_t st, std::string* err, const void* x2 = nullptr, const void* w2 = nullptr,
                     const void* x2_lo = nullptr, const void* w2_lo = nullptr, int Cin2 = 0, bool tf32 = false,
                     const TcGeom* geom = nullptr, const TcXf* xf = nullptr, long long wait_limit = 0,
                     const TcTile* tile = nullptr);

// Fused per-window UNet of the 16-channel networks (unet_small.cu): 2
// levels of 16 channels, 32 x 32 windows, GroupNorm(4), no attention, on
// the tensor cores in BF16 or FP8 E4M3 (per-output-channel weight scales).
struct SmallNet;
bool small_net_eligible(const UNetDesc& d);
SmallNet* small_net_create(const UNetDesc& d, const float* w_host, bool fp8, Err* err);
void small_net_destroy(SmallNet* s);
// F (n, 32, 32) float32 of x (n, 32, 32, in_ch) NHWC float32
bool small_net_forward(const SmallNet* s, const float* x, int n, float* F, int* status, long long wait_limit,
                       cudaStream_t st, std::string* err, const float* bias = nullptr);

// Persistent tile store (store.cpp): chunk files of finalized tiles in a
// directory, tied to a world identity by a manifest.
struct TileStore;
TileStore* store_open(const std::string& dir, uint64_t identity, const std::vector<int>& tile_side, bool writable,
                      std::string* err);
void store_close(TileStore* s);
bool store_has(TileStore* s, int level, int32_t ty, int32_t tx);
bool store_read(TileStore* s, int level, int32_t ty, int32_t tx, float* dst);
bool store_write(TileStore* s, int level, int32_t ty, int32_t tx, const float* src);

// float32 building blocks (unet.cu), NHWC, square images
void launch_conv_f32(const float* x, const float* wk, const float* res, float* y, int n, int H, int W,
                     int Cin, int Cout, int ks, cudaStream_t st);
void launch_gn_f32(const float* x, int n, int H, int C, int G, bool silu, double2* part, float2* stats,
                   float* y, cudaStream_t st);
size_t gn_part_elems(int n, int G);
void launch_avgpool2_f32(const float* x, int n, int H, int C, float* y, cudaStream_t st);
void launch_upcat_f32(const float* a, int Ca, const float* sk, int Cb, int n, int H, float* y,
                      cudaStream_t st);

}  // namespace idf
