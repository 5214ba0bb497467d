/*
 * idf.h -- C ABI of libidf, a GB300 (sm_103a) implementation of
 * InfiniteDiffusion sampling (arXiv 2512.08309) over an unbounded 2-D canvas.
 *
 * The library answers region queries J_0[R] of the paper's lazily evaluated
 * infinite image (Sec. 3.2-3.3, Eq. 2, Alg. 1): a seed fixes the whole world
 * (Sec. 3.5 "Seed consistency", App. B "Seeds and initial noise"), any
 * rectangle can be queried in any order at constant cost (Sec. 3.5
 * "Constant-time random access", Thm 2), and a model stack may chain a coarse
 * level into a fine one (App. C.3 "Dependency chaining", Sec. 5.3) whose pair
 * of outputs is decoded from the Laplacian encoding into metres (Sec. 5.2,
 * App. H).
 *
 * Conventions shared by every call
 *   - Coordinates are absolute pixel indices on Z^2; x is the column axis
 *     (the paper's second window index j), y the row axis.  Outputs are
 *     row-major: out[r * pitch + c] holds pixel (x0 + c, y0 + r).
 *   - The caller owns every buffer it passes; the library copies what it
 *     keeps (weights, descriptors) and owns the world, its tile cache, its
 *     device workspace and its CUDA stream.
 *   - Every call returns an idf_status; nothing aborts and no C++ exception
 *     crosses the ABI.  idf_world_last_error() gives a message.
 *   - After IDF_ECUDA or IDF_ETIMEOUT a world refuses further queries with
 *     IDF_EINTERNAL; destroy it and create a new one.
 *   - A world is not thread-safe: one host thread per world.
 *   - Identical (seed, stack, opts) give bitwise identical results whatever
 *     the query order, the batching of queries or the cache size.
 */
#ifndef IDF_H_
#define IDF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct idf_world idf_world;

typedef enum {
  IDF_OK = 0,
  IDF_EINVAL = 1,        /* bad argument or descriptor */
  IDF_ENOMEM = 2,        /* device or host allocation failed, or cache too small */
  IDF_ECUDA = 3,         /* a CUDA call failed; the world is unusable afterwards */
  IDF_ETIMEOUT = 4,      /* a bounded device-side wait ran out */
  IDF_EMODEL = 5,        /* weights do not match the described network */
  IDF_EDEVICE_CHECK = 6, /* a device-side bounds check fired */
  IDF_EINTERNAL = 7,     /* world poisoned by an earlier failure, or a bug */
  IDF_EUNSUPPORTED = 8   /* valid request that this library does not implement */
} idf_status;

/* Arithmetic of the UNet convolutions.  IDF_FP32: float32 SIMT (the plain
 * sampler).  IDF_BF16: bfloat16 operands on the tensor cores, float32
 * accumulation, float32 residual stream (for the 16-channel networks -- 2
 * levels of 16 channels, 32 x 32 windows, no attention -- the whole UNet of
 * a window runs as one fused tensor-core kernel).  IDF_FP8_E4M3: that fused
 * kernel with E4M3 operands, per-output-channel float32 weight scales and
 * power-of-two activation scales, float32 accumulation and statistics; built
 * for the 16-channel networks only (other networks: IDF_EUNSUPPORTED).  IDF_BF16X3: the same tensor-core
 * path with each operand split as hi + lo (both bfloat16) and the products
 * hi*hi + lo*hi + hi*lo accumulated, which compensates the rounding of both
 * operands at three times the tensor work.  IDF_TF32: operands rounded to
 * tf32 (10 explicit mantissa bits, round to nearest, ties away) and one tensor-core
 * product per multiply-add (kind::tf32, half the bf16 rate), float32
 * accumulation and residual stream. */
typedef enum { IDF_FP32 = 0, IDF_BF16 = 1, IDF_FP8_E4M3 = 2, IDF_BF16X3 = 3, IDF_TF32 = 4 } idf_precision;

typedef enum {
  IDF_OUT_MODEL = 0,  /* the last level's final sample J_K in model units */
  IDF_OUT_METRES = 1  /* Laplacian decode of (coarse, fine) to metres (stacks with laplacian=1) */
} idf_output_kind;

/*
 * One level of the model stack: a window denoiser Phi and its sliding-window
 * layout (Sec. 3.2: window (i,j) covers rows [i*stride, i*stride+window) and
 * columns [j*stride, j*stride+window)).  window must be a multiple of stride
 * (r = window/stride windows cover each stride x stride tile per axis) and
 * offset must be 0.
 *
 * The denoiser (test_denoiser = 0) is the ResBlock UNet described in
 * idf_model_param_shape(); it is EDM-preconditioned:
 *   D(x; sigma) = c_skip x + c_out F(c_in x [, conditioning]).
 * steps = K blended sampler steps on the rho-schedule from sigma_max to
 * sigma_min.  scale_to_parent = f > 0 makes the level conditioned on the
 * previous level of the stack: input channel 1 is that level's result
 * upsampled (nearest) by f (Sec. 5.3).  test_denoiser 1/2/3 replace F by a
 * closed-form function (constant 0.5 / sum of input channels / sum of input
 * channels + u/H - 2v/H in window-local row u and column v) for tests.
 */
typedef struct {
  int32_t levels;            /* UNet resolution levels L >= 1 */
  const int32_t* channels;   /* L channel counts (host, copied) */
  int32_t in_ch, out_ch;     /* in_ch = 1, or 2 with scale_to_parent > 0; out_ch = 1 */
  int32_t gn_groups;         /* GroupNorm groups (divides every channel count) */
  int32_t attn_at_bottom;    /* 1: self-attention block before the bottom ResBlock */
  int32_t attn_heads;        /* heads of that block (divides channels[L-1]) */
  const float* weights;      /* host, n_weights floats in declaration order (copied) */
  size_t n_weights;
  int32_t window, stride, offset, steps;
  double sigma_max, sigma_min, rho, sigma_data;
  int32_t scale_to_parent;   /* 0 for the first level; 8 for fine-under-coarse */
  int32_t test_denoiser;     /* 0 = UNet */
  /* Blending at selected noise levels only (the T variants, Sec. 4
   * "Latency", App. G): n_rounds > 0 groups the `steps` sampler steps into
   * n_rounds rounds of round_steps[r] >= 1 steps (summing to steps).  Inside
   * a round each window runs its steps on its own, x <- D(x; sigma_j) +
   * sigma_{j+1} N(.) with the noise of absolute coordinates, and Eq. 2
   * blends the windows only at the round's end; the dependency cone and the
   * tile cache advance by rounds.  n_rounds = 0 (round_steps NULL): every
   * step is blended.  round_steps is host memory, copied. */
  const int32_t* round_steps;
  int32_t n_rounds;
  /* Per-window conditioning (App. B "Seeds and initial noise": y_i =
   * Lambda(z, i); Sec. 5.3 feeds such a vector, the climate scalars, to the
   * network): cond_dim = D > 0 gives window i = (row, column) the vector
   * y_i = cond_z + cond_amp G_d(i), G_d(i) = N(seed, level, 0x7FFF0000 + d,
   * column, row) (the seed function at counters no sampler step uses), and
   * the UNet adds E y_i to its in-conv output, E = the (channels[0], D, 1, 1)
   * tensor declared last among its weights.  cond_z: host, D floats. */
  int32_t cond_dim;
  const float* cond_z;
  double cond_amp;
  /* AutoGuidance (Table "Hyperparameters"): guidance = w != 0 runs a guide
   * network of the same architecture (guide_weights, n_weights floats, host,
   * copied; with cond_dim > 0 it embeds y_i with its own E) beside the main
   * one on every window and uses F = F_guide + w (F_main - F_guide); 0 =
   * main network only. */
  double guidance;
  const float* guide_weights;
  size_t n_guide_weights;
} idf_level_desc;

/*
 * A chain of levels, coarse first (at most 2).  laplacian = 1 (two levels)
 * reads level 0 as the normalised low band L and level 1 as the normalised
 * residual H of the Laplacian encoding (Sec. 5.2; with one level and a
 * low_band_fixture, L comes from the fixture) and enables
 * IDF_OUT_METRES: l = low_mu + low_scale L, h = res_scale H,
 * P = up(l) + h, l^ = blur(down(P)), v = up(l^) + h, metres = sign(v) v^2
 * (App. H), with down = mean over lap_factor^2 blocks, blur = Gaussian of
 * lap_blur_sigma low-res pixels truncated at lap_radius, up = bilinear with
 * half-pixel centres.  blend_eps is the weight at a window's border
 * (Sec. 6: separable linear window, 1 at the centre).
 */
typedef struct {
  int32_t n_levels;
  const idf_level_desc* level;
  int32_t laplacian;
  int32_t lap_factor;
  double lap_blur_sigma;
  int32_t lap_radius;
  double low_mu, low_scale, res_scale;
  double blend_eps;
  /* Optional given low band (a single-level stack with laplacian = 1): a
   * host array of fixture_period^2 float32 normalised low-band values L on
   * the low-resolution grid, row-major, read periodically
   * (L(x, y) = fixture[(y mod P) * P + (x mod P)]), copied at create time.
   * The single level is then the residual band H.  NULL / 0 otherwise. */
  const float* low_band_fixture;
  int64_t fixture_period;
} idf_model_stack;

typedef struct {
  idf_precision precision;          /* arithmetic of the UNet convolutions */
  size_t cache_bytes;               /* device tile cache; 0 = default (8 GiB) */
  int32_t device;                   /* CUDA device ordinal */
  size_t workspace_bytes;           /* UNet activation arena shared by the levels; 0 = 128 GiB or
                                       45% of the device's free memory, whichever is less */
  int32_t max_batch;                /* windows per UNet launch; 0 = from workspace */
  int32_t profile;                  /* 1: time every kernel launch with CUDA events on the
                                       world's stream; per-class totals in idf_world_stats */
  uint64_t device_wait_budget_cycles; /* clock64 cycles a bounded device-side wait of the
                                       tensor-core kernels may take before it gives up and
                                       the query returns IDF_ETIMEOUT; 0 = 1e9 (about 0.5 s) */
  int32_t autotune;                 /* 1: the first launch of every tensor-core convolution (per
                                       layer, geometry and batch class) times each valid tile
                                       shape (BN, MT, staging) and keeps the fastest; results are
                                       the same bit for bit; 0 = built-in shapes */
  int32_t groupnorm_in_conv;        /* IDF_TF32: 1 applies GroupNorm and SiLU inside the
                                       tensor-core convolutions' operand path (no normalised
                                       operand in memory); 0 (default) runs them as separate
                                       passes, which is faster here.  Same results bit for bit */
  int32_t cuda_graphs;              /* 1: a UNet forward repeated with the same batch buffers and
                                       size (every full batch of a round, every round) is
                                       captured once as a CUDA graph and then replayed with one
                                       launch call; same kernels and arguments, same results bit
                                       for bit.  Off while profile is on.  0 = eager launches */
  int32_t cta_pairs;                /* 1: the tensor-core convolutions of plain BF16 / TF32 run on
                                       clusters of two CTAs (cta_group::2: M = 256 products,
                                       each CTA staging its own pixels and half of the weight
                                       tile) wherever the shape allows; same products per
                                       output element.  0 = one CTA per tile */
} idf_world_opts;

typedef struct {
  int64_t x0, y0;
  int32_t w, h;
  float* out_dev;                   /* device, caller-owned, h rows of pitch_elems */
  int64_t pitch_elems;
} idf_region;

/* ---------------------------------------------------------------- worlds */

/* Create a world: validates the stack, copies weights to the device (and
 * packs the tensor-core layouts for IDF_BF16 / IDF_BF16X3 / IDF_TF32: bf16
 * with low parts or tf32-rounded float32, plus the derived weights of the
 * half-resolution decoder blocks), copies a low-band fixture if given,
 * computes the sigma schedule, preconditioning coefficients, blend table and
 * blur taps in FP64 on the host, and allocates the tile cache and the UNet
 * arena.  Returns IDF_EINVAL for an invalid stack or options (among them a
 * low-band fixture with two levels, without laplacian = 1 or with a level of
 * in_ch != 1, and laplacian = 1 with one level and no fixture) before any
 * device call, IDF_EUNSUPPORTED for IDF_FP8_E4M3 with a level that is not a
 * 16-channel network, IDF_ENOMEM / IDF_ECUDA on
 * device allocation or CUDA failures.  *out is NULL on failure.  A level
 * whose in_ch is not 1 (2 under a parent), up to 8, is a side-input network
 * (a student fed its teacher's noise fields): the world is then
 * network-only, idf_unet_forward runs its levels and queries return
 * IDF_EMODEL. */
idf_status idf_world_create(uint64_t seed, const idf_model_stack* stack,
                            const idf_world_opts* opts, idf_world** out);

/* Query J_K (or metres) over [x0, x0+w) x [y0, y0+h) into a host buffer of
 * w*h floats (row-major, caller-owned).  w, h >= 1, w*h <= 2^31, and every
 * tile index must fit in int32.  Blocks until the result is on the host. */
idf_status idf_world_query(idf_world* world, int64_t x0, int64_t y0, int32_t w, int32_t h,
                           idf_output_kind kind, float* out_host);

/* Same, writing into device memory (h rows of pitch_elems >= w floats) on
 * the caller's CUDA stream (NULL = legacy default stream).  The world's own
 * stream is joined to it before and after; returns once the work is queued. */
idf_status idf_world_query_device(idf_world* world, int64_t x0, int64_t y0, int32_t w,
                                  int32_t h, idf_output_kind kind, float* out_dev,
                                  int64_t pitch_elems, void* cuda_stream);

/* Serve n regions as one batch: the window evaluations of all regions at
 * each step share launches (Thm 3: T - t rounds for any finite query set).
 * Results are bitwise identical to serving the regions one by one. */
idf_status idf_world_query_batch(idf_world* world, const idf_region* regions, int32_t n,
                                 idf_output_kind kind, void* cuda_stream);

/* Persistent tile store ("Caching and Persistence", infinite-tensor
 * appendix): open a directory of chunk files holding finalized tiles of the
 * last round of every level.  Planning then reads such tiles from the store
 * instead of computing their dependency cones (Lemma 3: a tile depends only
 * on the seed and its position), and, with writable != 0, every query writes
 * the final tiles it computed (a synchronous device-to-host copy and file
 * writes at the end of the query).  The directory's manifest ties it to one
 * world (seed, stack, weights, precision); opening it from another world
 * returns IDF_EINVAL, as does a missing directory without writable, or a
 * second open.  Files are plain chunk files of 16 x 16 tiles. */
idf_status idf_world_store_open(idf_world* world, const char* dir, int32_t writable);

/* Close the store (pending writes are complete when queries return). */
idf_status idf_world_store_close(idf_world* world);

/* Drop every cached tile (Sec. 3.3: eviction makes windows unprocessed). *//* Drop every cached tile (Sec. 3.3: eviction makes windows unprocessed). */
idf_status idf_world_cache_clear(idf_world* world);

/* JSON object with counters: windows evaluated per level, tiles computed,
 * cache hits / misses / evictions, kernel launches, bytes of the cache, and
 * (with opts.profile) per kernel class the launches, device milliseconds and
 * algorithmic FLOPs / bytes.  Synchronizes the world's stream. */
idf_status idf_world_stats(const idf_world* world, char* json_buf, size_t buf_len);

/* Message of the last failure on this world; valid until the next call. */
const char* idf_world_last_error(const idf_world* world);

/* Release everything the world owns; NULL-safe. */
void idf_world_destroy(idf_world* world);

/* Window indices (i = row, j = column) that a query of the region with the
 * current cache evaluates at step `step` (0 = first denoising step) of a
 * level: kappa of the missing tiles (Alg. 3) applied recursively as in
 * Alg. 1.  Writes up to cap pairs (i, j) into win_ij and the total count
 * into *n_out.  Does not evaluate anything. */
idf_status idf_debug_cone(idf_world* world, int64_t x0, int64_t y0, int32_t w, int32_t h,
                          int32_t level, int32_t step, int64_t* win_ij, int32_t cap,
                          int32_t* n_out);

/* Test-only: the tile keys (tile row, tile column) of J_step held in a
 * level's cache (step 1..K; J_0 is the noise and is never cached), sorted
 * by row then column.  Writes up to cap pairs into ty_tx and the total count
 * into *n_out.  Reads host bookkeeping only (Sec. 3.3: the processed set P
 * of the lazy algorithm, kept here as finalized tiles). */
idf_status idf_debug_cache_keys(idf_world* world, int32_t level, int32_t step, int32_t* ty_tx,
                                int32_t cap, int32_t* n_out);

/* Test-only failure injection from the host: after synchronizing the
 * world's stream, writes `value` into a device status word -- which = 0:
 * the word the tensor-core convolutions set when a bounded wait runs out
 * (read back as IDF_ETIMEOUT by the next synchronizing query, which also
 * makes every later tensor-core launch return at once); which = 1: the
 * conditioning gather's bounds-check flag (read back as IDF_EDEVICE_CHECK
 * and cleared).  No kernel faults or waits; the failure paths that follow
 * are the same as for a real expiry or bounds violation.  IDF_EINVAL for
 * another `which`. */
idf_status idf_debug_set_status(idf_world* world, int32_t which, int32_t value);

/* --------------------------------------------------------- building blocks */

/* The seed function G (App. B): N(seed, level, step, x, y), standard normal
 * in binary32, defined bit for bit by Philox4x32-10 (key = seed, counter =
 * (x mod 2^32, y mod 2^32, step, level)) and Box-Muller with the library's
 * own binary32 polynomials for ln and cos.  Writes h rows of w values at
 * out_dev (pitch_elems floats per row) on the given stream. */
idf_status idf_noise_fill(uint64_t seed, uint32_t level, uint32_t step, int64_t x0, int64_t y0,
                          int32_t w, int32_t h, float* out_dev, int64_t pitch_elems,
                          void* cuda_stream);

/* Number of weight tensors of a level's UNet and the shape (C_out, C_in,
 * kh, kw) of tensor `index` in declaration order: in_conv; per encoder level
 * conv1, conv2, [1x1 skip when channels change]; [attention qkv (3C, C, 1, 1),
 * proj (C, C, 1, 1)]; bottom ResBlock; per decoder level (deepest first)
 * conv1, conv2, skip; out_conv. */
idf_status idf_model_param_count(const idf_level_desc* level, int32_t* n_tensors,
                                 size_t* n_weights);
idf_status idf_model_param_shape(const idf_level_desc* level, int32_t index, int32_t shape[4]);

/* Phi's network F (Sec. 5.3, the UNet of a level) on a batch of windows:
 * x_dev (n, in_ch, window, window) float32 NCHW, y_dev (n, out_ch, window,
 * window) float32, both device.  Runs in the world's precision, ordered on
 * cuda_stream and asynchronous: a bounded device-side wait that ran out
 * during it is not returned here but shows in idf_world_stats
 * ("device_status") and makes the world's next query fail with
 * IDF_ETIMEOUT. */
idf_status idf_unet_forward(idf_world* world, int32_t level, const float* x_dev, int32_t n,
                            float* y_dev, void* cuda_stream);

/* Laplacian denoising decode (Sec. 5.2, App. H) of explicit bands: L_dev is
 * the normalised low band on the coarse grid, origin (lx0, ly0), lw x lh,
 * pitch lpitch; H_dev the normalised residual on the fine grid, origin (hx0,
 * hy0), hw x hh, pitch hpitch.  Writes metres for [x0, x0+w) x [y0, y0+h)
 * into out_dev.  The bands must cover the rects idf_laplacian_halo()
 * returns for the query (IDF_EINVAL otherwise); about (lap_radius + 1) *
 * lap_factor fine pixels of H and lap_radius + 2 coarse pixels of L on each
 * side. */
idf_status idf_laplacian_decode(const idf_model_stack* stack, const float* L_dev, int64_t lx0,
                                int64_t ly0, int32_t lw, int32_t lh, int64_t lpitch,
                                const float* H_dev, int64_t hx0, int64_t hy0, int32_t hw,
                                int32_t hh, int64_t hpitch, int64_t x0, int64_t y0, int32_t w,
                                int32_t h, float* out_dev, int64_t pitch_elems,
                                void* cuda_stream);

/* The same decode as idf_laplacian_decode, for callers that cannot allocate
 * device memory at call time (a plugin whose host engine owns all device
 * memory through its own pool, a frame loop that cannot take an allocation's
 * latency or implicit synchronization).  The paper has no counterpart; this
 * is a deployment variant.  It calls no cudaMalloc, cudaFree or allocating
 * library routine: its scratch (2^20 floats, 4 MiB) is a fixed array in the
 * library's device image, held by every GPU that loads the library until the
 * process exits.  Queries whose scratch would exceed it (anything larger
 * than about 4096 x 4096 pixels at lap_factor 8, lap_radius 15) return
 * IDF_EINVAL.  Runs on the current device; the first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) and should come
 * before any stream capture.  All calls on a device share the array: calls
 * whose kernels overlap on the GPU race and must be ordered by the caller.
 * Arguments and results are those of idf_laplacian_decode. */
idf_status idf_laplacian_decode_noalloc(const idf_model_stack* stack, const float* L_dev, int64_t lx0,
                                        int64_t ly0, int32_t lw, int32_t lh, int64_t lpitch,
                                        const float* H_dev, int64_t hx0, int64_t hy0, int32_t hw,
                                        int32_t hh, int64_t hpitch, int64_t x0, int64_t y0, int32_t w,
                                        int32_t h, float* out_dev, int64_t pitch_elems,
                                        void* cuda_stream);

/* Halo the decode of [x0, x0+w) x [y0, y0+h) reads: the coarse rect of L and
 * the fine rect of H, each as (x0, y0, w, h). */
idf_status idf_laplacian_halo(const idf_model_stack* stack, int64_t x0, int64_t y0, int32_t w,
                              int32_t h, int64_t L_rect[4], int64_t H_rect[4]);

/* ------------------------------------------------------- voxel volumes */

/* InfiniteDiffusion on Z^3 (the method is defined on S = Z^d, Sec. 3.2;
 * Alg. 3 computes kappa per dimension): a seeded, lazily evaluated, infinite
 * voxel volume queried by boxes in any order.  Windows (i, j, l) cover
 * [i s, i s + window) x [j s, ...) x [l s, ...) in (z, y, x); tiles are
 * stride^3, cached per blended step with LRU eviction; blending is Eq. 2
 * with the separable linear weight window cubed; the noise is N3(seed, 0,
 * step, x, y, z) = Philox4x32-10 with counter (x, y, z, 2^31 + level 2^16 +
 * step) and this library's Box-Muller (see idf_noise_fill); EDM
 * preconditioning and the rho-schedule as for a 2-D level.  The denoiser is
 * F(x) = conv2(silu(gn(conv1(x)))) (3x3x3, zero padding per window, `channels`
 * <= 8 hidden channels in `groups` GroupNorm groups, window^3 <= 4096,
 * weights conv1 (channels, 1, 3, 3, 3) then conv2 (1, channels, 3, 3, 3)),
 * or with test_denoiser 1 / 2 / 3 the constant 0.5 / identity / identity +
 * u/H - 2 v/H + 3 w/H (window-local z, y, x).  Float32 throughout. */
typedef struct {
  int32_t window, stride, steps;
  double sigma_max, sigma_min, rho, sigma_data, blend_eps;
  int32_t channels, groups;
  int32_t test_denoiser;
  const float* weights;  /* host, copied; NULL for test denoisers */
  size_t n_weights;
} idf_volume_desc;

typedef struct idf_volume idf_volume;

/* Create a volume on a device with a tile cache of cache_bytes (0 = 1 GiB).
 * IDF_EINVAL for an invalid descriptor, IDF_EMODEL for weights that do not
 * match, IDF_ENOMEM / IDF_ECUDA on device failures. */
idf_status idf_volume_create(uint64_t seed, const idf_volume_desc* desc, int32_t device, size_t cache_bytes,
                             idf_volume** out);

/* The result over [x0, x0+w) x [y0, y0+h) x [z0, z0+d) into out_host
 * (caller-owned, w*h*d floats, out[(z * h + y) * w + x]); blocks until done.
 * Tile indices must stay within +-2^20; w*h*d <= 2^30. */
idf_status idf_volume_query(idf_volume* v, int64_t x0, int64_t y0, int64_t z0, int32_t w, int32_t h,
                            int32_t d, float* out_host);

/* Counters: out[0] windows evaluated, out[1] tiles computed, out[2] cache
 * hits, out[3] cache misses. */
idf_status idf_volume_stats(const idf_volume* v, int64_t out[4]);

const char* idf_volume_last_error(const idf_volume* v);

/* NULL-safe. */
void idf_volume_destroy(idf_volume* v);

/* ------------------------------------------------------ learned student */

/* A student denoiser trained on the GPU by this library's own forward and
 * backward kernels (the library's few-step counterpart of the paper's
 * consistency-distilled networks, Sec. 5.4 and App. F "Consistency
 * Distillation").  The network is the UNet of idf_level_desc (same layers and
 * weight order; no attention block; out_ch = 1, 1 <= in_ch <= 8; `window` is
 * the training window size); parameters are float32 master weights.  One
 * training step evaluates D(x; sigma) = c_skip x_0 + c_out S([c_in x_0, x_1,
 * ..., x_{in_ch - 1}]) with the EDM coefficients (sigma_data of the
 * descriptor): channel 0 is the noisy state, the others side inputs given
 * to the network as they are (the teacher's re-noise fields); the loss is
 * mean((D - t)^2), and d loss / d weights is added to the student's
 * gradient accumulator.  Everything the student holds is owned by the
 * library. */
typedef struct idf_student idf_student;

/* net->weights (n_weights floats, declaration order) are copied as the
 * initial weights.  max_batch windows per step; device = CUDA ordinal. */
idf_status idf_student_create(const idf_level_desc* net, int32_t max_batch, int32_t device,
                              idf_student** out);

/* x_dev: device float32 (n, in_ch, window, window); target_dev: (n, window,
 * window); 1 <= n <= max_batch.
 * Writes the batch loss to *loss_out (host) and accumulates its gradient.
 * Ordered after the caller's stream; synchronizes before returning. */
idf_status idf_student_loss_grad(idf_student* s, const float* x_dev, const float* target_dev,
                                 int32_t n, double sigma, double* loss_out, void* cuda_stream);

/* One AdamW step (decoupled weight decay) with the accumulated gradient,
 * which is then cleared. */
idf_status idf_student_adamw(idf_student* s, double lr, double beta1, double beta2, double eps,
                             double weight_decay);

/* Clear the gradient accumulator. */
idf_status idf_student_zero_grad(idf_student* s);

/* Copy the weights (what = 0) or the accumulated gradient (what = 1) to host
 * memory in declaration order; n must equal the parameter count. */
idf_status idf_student_read(const idf_student* s, int32_t what, float* host_out, size_t n);

/* Replace the student's weights by host_in (n floats, declaration order;
 * n must equal the parameter count); the AdamW moments are kept. */
idf_status idf_student_write(idf_student* s, const float* host_in, size_t n);

/* Message of the last failure on this student. */
const char* idf_student_last_error(const idf_student* s);

/* NULL-safe. */
void idf_student_destroy(idf_student* s);

#ifdef __cplusplus
}
#endif

#endif /* IDF_H_ */
