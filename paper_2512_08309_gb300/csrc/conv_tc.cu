// Implicit-GEMM convolution on the sm_103a tensor cores (tcgen05 + TMEM),
// fed by TMA.  This is the dense contraction of the window denoiser F
// (Sec. 5.3): a 3x3 (or 1x1) zero-padded convolution of bfloat16 NHWC
// activations with bfloat16 weights, accumulated in float32 in tensor memory.
//
//   GEMM view: M = pixels of a window batch, N = C_out, K = taps * C_in.
//   CTA tile:  128 pixels (whole rows of one window) x BN output channels.
//   K stage:   one tap (dy, dx) and 64 input channels: a 4-D TMA box of the
//              activation tensor (64 channels x W x 128/W rows x 1 window)
//              at the tap's offset -- out-of-range rows and columns are
//              zero-filled by TMA, which is exactly the window's zero padding
//              -- and a 2-D TMA box of the weights (64 channels x BN rows).
//              Both land in shared memory in the 128-byte swizzled K-major
//              layout that the UMMA descriptors describe.
//   Warps:     persistent CTAs, one per SM.  Warp 0 lane 0 issues TMA into a
//              ring of stages; warp 1 allocates 2 x BN TMEM columns and lane
//              0 issues tcgen05.mma (M=128, N=BN, K=16, four per stage) into
//              one of two accumulators and tcgen05.commit; warps 2-5 read the
//              other accumulator with tcgen05.ld (warp w reads TMEM lanes
//              32*(w%4)..+31) and write float32 NHWC output, adding the
//              residual if given, while the next tile accumulates.
//   TF32:      with float32 operands (IDF_TF32, values already rounded to
//              tf32 by their producers) the same pipeline issues
//              tcgen05.mma kind::tf32 (K = 8 per instruction); a stage then
//              carries 32 channels, so its bytes and layout are those of a
//              64-channel bfloat16 stage.
//   Split:     with low parts given (IDF_BF16X3) a stage holds A_hi, A_lo,
//              B_hi and B_lo and issues A_hi B_hi + A_lo B_hi + A_hi B_lo per
//              K step, where x = hi + lo with hi = bf16(x), lo = bf16(x - hi):
//              bfloat16 products with the rounding of both operands
//              compensated.
//   Fold:      optionally the tile's K loop continues over a second operand,
//              a 1x1 convolution of another tensor (the ResBlock shortcut)
//              accumulated into the same TMEM tile: one 128-pixel box and
//              one weight box per 64 input channels, from its own tensor
//              maps.  The shortcut's output never goes through memory.
//   Stats:     optionally the epilogue also emits GroupNorm partials of the
//              values it writes: per 32-pixel block (one warp's TMEM lanes)
//              and 16-channel slice, the mean and the sum of squared
//              deviations M2 of those 512 values (per pixel over 16 channels,
//              then merged across the warp's lanes by the pairwise update of
//              Chan et al. 1979).  The GroupNorm then needs no statistics
//              pass over its input.
//   Transform: optionally (TF32, XF kernels) the activation is the raw
//              float32 tensor and GroupNorm (+ SiLU) is applied on its way
//              to the tensor cores: four more warps wait for each landed
//              stage, replace every staged value x of a real pixel by
//              tf32(silu((x - mean) * rstd)) with its window's and group's
//              statistics (leaving the zero padding zero), fence the
//              generic-proxy writes for the async proxy and release the
//              stage to the MMA thread; folded 1x1 stages pass unchanged
//              (raw float32, read as tf32).  The arithmetic is that of the
//              separate GroupNorm apply pass, so the result is the same bit
//              for bit while the normalised operand never goes through
//              memory.  Measured on the 2-level stack it is slower than the
//              separate pass (each staged box is transformed once per tap
//              and N tile, up to 9x the elements, and the exponential and
//              reciprocal of SiLU bind the transform warps), so it is an
//              option, off by default.
//   Waits:     every mbarrier wait is bounded (clock64 budget); on expiry
//              the CTA sets the status word, drains what it issued and
//              frees its TMEM before returning.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <string>

#include "internal.h"

namespace idf {
namespace {

constexpr int BM = 128;
constexpr int XF_THREADS = 128;  // the transform warpgroup of the XF kernels

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// The same with acquire at cluster scope: for barriers that the other CTA of
// a pair arrives on (remote arrivals, multicast commits).
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait.  honour_abort: give up as soon as another role aborted.
// CL: acquire at cluster scope.
template <bool CL = false>
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                         int* status, bool honour_abort, long long limit) {
  const long long t0 = clock64();
  while (!(CL ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity))) {
    if (honour_abort && *abort_flag) return false;
    if (clock64() - t0 > limit) {
      atomicExch(status, 1);
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

// CTA-pair forms: the copy lands in this CTA's shared memory and completes
// its bytes on the barrier at cluster address bar_cl, which may be the even
// CTA's (one barrier per stage counts both CTAs' copies).
__device__ __forceinline__ void tma_load_4d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cl, int c0,
                                                 int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cta.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(bar_cl), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cl, int c0,
                                                 int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(bar_cl), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// Shared-memory matrix descriptor (tcgen05): K-major operand, 128-byte
// swizzle, 8-row core-matrix groups 1024 bytes apart.
// The 128-byte swizzle phase follows the shared-memory address bits, so an
// operand may start 32-byte steps into a row (K steps) or whole 128-byte rows
// into a staged tile (the horizontal taps of row reuse) with the base-offset
// field left at zero (measured: setting it to (address >> 7) & 7 applies the
// phase twice).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
  d |= (uint64_t)1 << 46;               // descriptor version
  d |= (uint64_t)2 << 61;               // 128-byte swizzle
  return d;
}

// Instruction descriptor: f32 accumulator (bits 4-5 = 1), A and B formats
// (bits 7-9, 10-12: 1 = bf16 under kind::f16, 2 = tf32 under kind::tf32),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_mma(int M, int N, bool tf32) {
  return (1u << 4) | ((tf32 ? 2u : 1u) << 7) | ((tf32 ? 2u : 1u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// One K step of 32 bytes per operand row: 16 bf16 or 8 tf32 values.
template <bool TF32>
__device__ __forceinline__ void mma_step(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  if (TF32) mma_tf32(tmem_d, adesc, bdesc, idesc, accumulate);
  else mma_bf16(tmem_d, adesc, bdesc, idesc, accumulate);
}

// CTA-pair (cta_group::2) forms: one thread of the even CTA of a cluster
// pair issues M = 256 products whose rows 0-127 come from its own shared
// memory and rows 128-255 from its peer's (the same offsets), whose B columns
// are split between the two (the first BN / 2 rows of the weight tile in the
// even CTA, the rest in the odd one), and whose accumulator tile lives at
// the same tensor-memory address in both CTAs, each holding its own 128 rows.
__device__ __forceinline__ void mma_bf16_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_tf32_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrives once on the barrier at this offset in both CTAs of the pair when
// every product this thread issued before it has completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((unsigned short)3)
      : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Address of the same shared-memory object in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Named-barrier reduction among the n threads of barrier id: true iff every
// participant passed true.  Lets the transform warps leave their loop
// together when any of them gave up on a wait.
__device__ __forceinline__ bool bar_and(bool v, int id, int n) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// The operand arithmetic of the GroupNorm apply pass (unet.cu): round to
// tf32 (nearest at mantissa bit 13, ties away), SiLU with the fast
// exponential and division.
__device__ __forceinline__ float xf_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}
__device__ __forceinline__ float xf_silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

struct TcParams {
  const float* res;
  float* y;
  float2* bstats;  // null, or (mean, M2) per (32-pixel block, 16-channel slice)
  int* status;
  int H, W, Cout, ks, n_kc, n_iter;
  int oy, ox;            // input offset of tap (0, 0): tap t reads (y + t / ks + oy, x + t % ks + ox)
  int out_up, py, px;    // out_up: pixel (y, x) is stored at (2y + py, 2x + px) of a 2H x 2W output
  int res_up;            // res_up: the residual of pixel (y, x) is element (y / 2, x / 2) of an H/2 x W/2 tensor
  int kch;               // input channels per K stage (64 bf16 or 32 tf32: 128 bytes)
  int n_iter1;           // K iterations of the main operand; the rest are the folded 1x1 operand
  int m_tiles, n_tiles;  // output tiles: 128-pixel rows x BN channels
  long long wait_limit;  // clock64 cycles a bounded wait may take
  // XF kernels: (mean, rstd) per (window, group) of the main operand's
  // GroupNorm (null: round only), groups G of cpg channels, the operand's
  // channel offset in the normalised tensor, SiLU after the normalisation
  const float2* xf_stats;
  int xf_G, xf_cpg, xf_coff, xf_silu;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent kernel: CTA c handles work units c, c + gridDim.x, ...  A unit
// is MT consecutive 128-pixel M tiles of one window (MT = 1 or 2) times one
// BN-channel N tile; with MT = 2 the two M tiles share every staged weight
// tile (twice the MMA work per staged byte) and accumulate into two TMEM
// tiles.  Channel tiles of the same pixels are adjacent units, so they share
// the activations in L2.  The shared-memory ring of STAGES stages runs
// across unit boundaries; two TMEM accumulator sets (2 x MT x BN columns)
// let the epilogue of one unit overlap the main loop of the next.
//
// PAIR (clusters of two CTAs on one TPC, cta_group::2): a unit is 2 MT M
// tiles, MT of them in each CTA, times one BN-channel N tile.  Each CTA
// stages its own pixels and half of the weight tile (BN / 2 rows), so a
// stage carries a third fewer bytes per product; the even CTA's MMA thread
// issues M = 256 products over both CTAs' stages once a stage's copies have
// landed in both (they complete their bytes on one barrier of the even CTA,
// which expects those of both), and its commits arrive on both CTAs'
// barriers.  Both
// epilogues read their own accumulator rows and release the accumulator with
// arrivals on the even CTA's barrier.  The arithmetic per output element is
// that of the single-CTA kernel.
template <int BN, int STAGES, bool SPLIT, bool DXR, bool TF32, int MT, bool XF, bool PAIR = false>
__global__ void __launch_bounds__(XF ? 192 + XF_THREADS : 192, 1) conv_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB,
                                                         const __grid_constant__ CUtensorMap tmA_lo,
                                                         const __grid_constant__ CUtensorMap tmB_lo,
                                                         const __grid_constant__ CUtensorMap tmA2,
                                                         const __grid_constant__ CUtensorMap tmB2,
                                                         const __grid_constant__ CUtensorMap tmA2_lo,
                                                         const __grid_constant__ CUtensorMap tmB2_lo,
                                                         TcParams p) {
  // DXR (3x3 convs on 128-pixel rows): a stage holds one kernel row dy: a
  // 130-pixel activation box per image row (halo columns zero-filled; MT
  // rows in one box) read by the three horizontal taps at row offsets 0, 1,
  // 2, and the three taps' weights.
  static_assert(!PAIR || (!SPLIT && !XF), "the CTA-pair kernels take plain bf16 / tf32 operands");
  constexpr int A_ROW = DXR ? (BM + 2) * 128 : BM * 128;    // bytes of one M tile's rows
  constexpr int A_BOX = A_ROW * MT;                         // bytes TMA writes
  constexpr int A_BYTES = (A_BOX + 1023) / 1024 * 1024;     // region, 1024-aligned
  constexpr int BNL = PAIR ? BN / 2 : BN;                   // weight rows staged by this CTA
  constexpr int B_BYTES = BNL * 128;
  constexpr int NB = DXR ? 3 : 1;                           // weight tiles per stage
  constexpr int NP = SPLIT ? 2 : 1;                         // hi (and lo) parts per operand
  constexpr int STAGE_BYTES = NP * (A_BYTES + NB * B_BYTES);
  constexpr int TX_BYTES = NP * (A_BOX + NB * B_BYTES);
  constexpr int TX2_BYTES = NP * (BM * 128 * MT + B_BYTES); // a folded 1x1 stage
  constexpr uint32_t ACC_COLS = MT * BN;                    // TMEM columns of one accumulator set
  extern __shared__ uint8_t dsmem[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ __align__(8) uint64_t ready_bar[XF ? STAGES : 1];  // XF: stage transformed
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  __shared__ int skip_sh;
  uint8_t* smem = dsmem + ((1024 - (smem_u32(dsmem) & 1023)) & 1023);
  volatile int* abort_flag = &abort_sh;
  const uint32_t rank = PAIR ? cluster_rank() : 0u;  // PAIR: 0 = the MMA-issuing CTA
  // once any CTA of any launch has given up on a wait, later CTAs return at
  // once (one thread reads the status so that the whole CTA decides alike;
  // for a pair, the even CTA decides for both, after the cluster sync below)
  if (!PAIR) {
    if (threadIdx.x == 0) skip_sh = *(volatile int*)p.status;
    __syncthreads();
    if (skip_sh) return;
  }

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t HW = (int64_t)p.H * p.W;
  constexpr int MU = PAIR ? 2 * MT : MT;  // M tiles per unit
  int n_units = p.m_tiles / MU * p.n_tiles;
  const int cta0 = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;  // this CTA's (pair's) first unit
  const int ncta = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;   // unit stride
  // first pixel of unit u's rows in this CTA
  auto unit_m0 = [&](int u) -> int64_t {
    return (int64_t)(u / p.n_tiles) * (BM * MU) + (int64_t)rank * (BM * MT);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
      if (XF) mbar_init(&ready_bar[s], XF_THREADS);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], PAIR ? 256 : 128);  // PAIR: both CTAs' epilogue threads
    }
    mbar_init(&drain_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0 && lane == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
    if (SPLIT) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA_lo) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB_lo) : "memory");
    }
    if (p.n_iter > p.n_iter1) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA2) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB2) : "memory");
      if (SPLIT) {
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA2_lo) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB2_lo) : "memory");
      }
    }
  }
  if (warp == 1) {
    if (PAIR) {
      // allocated by one warp of each CTA of the pair together
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(&tmem_base_sh)),
                   "r"(2 * ACC_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(&tmem_base_sh)),
                   "r"(2 * ACC_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  if (PAIR) {
    // both CTAs have started and their barriers exist before either touches
    // the other's shared memory; then the even CTA's view of the status word
    // decides for both
    fence_before();
    cluster_sync();
    fence_after();
    if (rank == 0 && threadIdx.x == 0) {
      const int v = *(volatile int*)p.status;
      skip_sh = v;
      asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(peer_addr(&skip_sh, 1)), "r"(v) : "memory");
    }
    cluster_sync();
    if (skip_sh) n_units = 0;
  } else {
    fence_before();
    __syncthreads();
    fence_after();
  }
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) {
      int last_issue[STAGES];
      for (int s = 0; s < STAGES; ++s) last_issue[s] = -1;
      // PAIR: both CTAs' copies of a stage complete on the even CTA's
      // barrier, which expects the bytes of both
      const uint32_t fb0 = PAIR ? peer_addr(&full_bar[0], 0) : 0u;
      auto expect = [&](int s, uint32_t bytes) {
        if (!PAIR) mbar_expect_tx(&full_bar[s], bytes);
        else if (rank == 0) mbar_expect_tx(&full_bar[s], 2u * bytes);
      };
      auto ld4 = [&](void* dst, const CUtensorMap* map, int s, int c0, int c1, int c2, int c3) {
        if (PAIR) tma_load_4d_pair(dst, map, fb0 + 8u * (uint32_t)s, c0, c1, c2, c3);
        else tma_load_4d(dst, map, &full_bar[s], c0, c1, c2, c3);
      };
      auto ld2 = [&](void* dst, const CUtensorMap* map, int s, int c0, int c1) {
        if (PAIR) tma_load_2d_pair(dst, map, fb0 + 8u * (uint32_t)s, c0, c1);
        else tma_load_2d(dst, map, &full_bar[s], c0, c1);
      };
      uint32_t it = 0;
      bool ok = true;
      for (int u = cta0; u < n_units && ok; u += ncta) {
        const int64_t m0 = unit_m0(u);
        // this CTA's weight rows: all BN, or its half of them (PAIR)
        const int n0 = (u % p.n_tiles) * BN + (int)rank * BNL;
        const int win = (int)(m0 / HW);
        const int y0 = (int)((m0 % HW) / p.W);
        for (int kk = 0; kk < p.n_iter; ++kk, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1u;
          if (!wait_bar<PAIR>(&empty_bar[s], ph ^ 1u, abort_flag, p.status, true, p.wait_limit)) {
            ok = false;
            break;
          }
          uint8_t* a = smem + (size_t)s * STAGE_BYTES;
          uint8_t* b = a + NP * A_BYTES;
          if (kk >= p.n_iter1) {
            // folded 1x1 operand: the unit's own pixels, kch channels
            const int kc = kk - p.n_iter1;
            expect(s, TX2_BYTES);
            ld4(a, &tmA2, s, kc * p.kch, 0, y0, win);
            ld2(b, &tmB2, s, kc * p.kch, n0);
            if (SPLIT) {
              ld4(a + A_BYTES, &tmA2_lo, s, kc * p.kch, 0, y0, win);
              ld2(b + NB * B_BYTES, &tmB2_lo, s, kc * p.kch, n0);
            }
          } else if (DXR) {
            expect(s, TX_BYTES);
            const int dyi = kk / p.n_kc, kc = kk % p.n_kc;
            ld4(a, &tmA, s, kc * p.kch, p.ox, y0 + dyi + p.oy, win);
            if (SPLIT) ld4(a + A_BYTES, &tmA_lo, s, kc * p.kch, p.ox, y0 + dyi + p.oy, win);
            for (int t = 0; t < 3; ++t) {
              ld2(b + t * B_BYTES, &tmB, s, kc * p.kch, (dyi * 3 + t) * p.Cout + n0);
              if (SPLIT) ld2(b + (3 + t) * B_BYTES, &tmB_lo, s, kc * p.kch, (dyi * 3 + t) * p.Cout + n0);
            }
          } else {
            expect(s, TX_BYTES);
            const int tap = kk / p.n_kc, kc = kk % p.n_kc;
            const int dy = tap / p.ks + p.oy, dx = tap % p.ks + p.ox;
            ld4(a, &tmA, s, kc * p.kch, dx, y0 + dy, win);
            ld2(b, &tmB, s, kc * p.kch, tap * p.Cout + n0);
            if (SPLIT) {
              ld4(a + A_BYTES, &tmA_lo, s, kc * p.kch, dx, y0 + dy, win);
              ld2(b + B_BYTES, &tmB_lo, s, kc * p.kch, tap * p.Cout + n0);
            }
          }
          last_issue[s] = (int)it;
        }
      }
      if (*abort_flag) {
        if (PAIR && rank == 1) {
          // this CTA's copies complete on the even CTA's barriers: give the
          // ones in flight a fixed 100k cycles (tens of microseconds) to land
          const long long t0 = clock64();
          while (clock64() - t0 < 100000) {
          }
        } else {
          // drain the copies this thread issued before leaving
          for (int s = 0; s < STAGES; ++s)
            if (last_issue[s] >= 0)
              wait_bar<PAIR>(&full_bar[s], (uint32_t)(last_issue[s] / STAGES) & 1u, abort_flag, p.status, false,
                             p.wait_limit);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && PAIR && rank == 1) {
      // odd CTA of a pair: the even CTA's last commit means that every
      // product reading this CTA's stages or writing its accumulators is done
      wait_bar<true>(&drain_bar, 0, abort_flag, p.status, false, p.wait_limit);
    } else if (lane == 0) {
      constexpr uint32_t idesc = idesc_mma(PAIR ? 2 * BM : BM, BN, TF32);
      uint32_t it = 0, acc = 0;
      bool ok = true;
      for (int u = cta0; u < n_units && ok; u += ncta, ++acc) {
        const uint32_t buf = acc & 1u, aph = (acc >> 1) & 1u;
        if (!wait_bar<PAIR>(&acce_bar[buf], aph ^ 1u, abort_flag, p.status, true, p.wait_limit)) break;
        fence_after();
        const uint32_t d = tmem + buf * ACC_COLS;
        for (int kk = 0; kk < p.n_iter; ++kk, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1u;
          if (!wait_bar<PAIR>(XF ? &ready_bar[s] : &full_bar[s], ph, abort_flag, p.status, true, p.wait_limit)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t a = smem_u32(smem + (size_t)s * STAGE_BYTES);
          const uint32_t b = a + NP * A_BYTES;
          auto step = [&](uint32_t dd, uint32_t aa, uint32_t bb, uint32_t accum) {
            if (PAIR) {
              if (TF32) mma_tf32_pair(dd, umma_desc(aa), umma_desc(bb), idesc, accum);
              else mma_bf16_pair(dd, umma_desc(aa), umma_desc(bb), idesc, accum);
            } else {
              mma_step<TF32>(dd, umma_desc(aa), umma_desc(bb), idesc, accum);
            }
          };
          if (kk >= p.n_iter1) {
            // folded 1x1 operand (never the first K step of a unit); its M
            // tiles are whole 128-pixel blocks of the box
#pragma unroll
            for (int i = 0; i < MT; ++i) {
              const uint32_t ai = a + i * BM * 128, di = d + i * BN;
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                step(di, ai + 32 * k, b + 32 * k, 1u);
                if (SPLIT) {
                  step(di, ai + A_BYTES + 32 * k, b + 32 * k, 1u);
                  step(di, ai + 32 * k, b + NB * B_BYTES + 32 * k, 1u);
                }
              }
            }
            if (PAIR) mma_commit_pair(&empty_bar[s]);
            else mma_commit(&empty_bar[s]);
            continue;
          }
#pragma unroll
          for (int t = 0; t < NB; ++t) {
            const uint32_t bt = b + B_BYTES * t;
#pragma unroll
            for (int i = 0; i < MT; ++i) {
              // M tile i reads its own rows of the box; DXR: horizontal tap t
              // starts t rows further
              const uint32_t at = a + i * A_ROW + (DXR ? 128 * t : 0), di = d + i * BN;
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                step(di, at + 32 * k, bt + 32 * k, (kk > 0 || t > 0 || k > 0) ? 1u : 0u);
                if (SPLIT) {
                  step(di, at + A_BYTES + 32 * k, bt + 32 * k, 1u);
                  step(di, at + 32 * k, bt + NB * B_BYTES + 32 * k, 1u);
                }
              }
            }
          }
          if (PAIR) mma_commit_pair(&empty_bar[s]);
          else mma_commit(&empty_bar[s]);
        }
        if (!ok) break;
        if (PAIR) mma_commit_pair(&accf_bar[buf]);
        else mma_commit(&accf_bar[buf]);
      }
      // every MMA this thread issued has completed once this commit arrives
      if (PAIR) mma_commit_pair(&drain_bar);
      else mma_commit(&drain_bar);
      wait_bar<PAIR>(&drain_bar, 0, abort_flag, p.status, false, p.wait_limit);
    }
  } else if (!XF || warp < 6) {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    uint32_t acc = 0;
    // Global memory is touched in whole 128-byte pixel chunks: lane l moves
    // 16-byte piece l % 8 of pixels l / 8, l / 8 + 4, ... of the warp's 32
    // pixels, and a per-warp shared buffer (32 rows of 36 floats) turns
    // that into one row per thread (the thread owns its TMEM lane's pixel)
    // and back.  The residual is read one 32-column chunk ahead (the next
    // unit's first chunk after a unit's last), so its memory latency
    // overlaps the work on the current chunk; every residual element is
    // read before the same output element is written.
    float* T = reinterpret_cast<float*>(smem + (size_t)STAGES * STAGE_BYTES) + (size_t)q * (32 * 36);
    const int pc = lane & 7, pr = lane >> 3;  // piece, first pixel of this lane
    float4 nx[8];
    // a warp's 32 pixels lie in one window (M tiles are 128-pixel blocks of
    // windows of 128 k pixels) whose width W is a power of two: their rows
    // and columns follow from the first pixel's offset with shifts.  The
    // residual of pixel (y, x) is the same grid's, or (res_up) element
    // (y / 2, x / 2) of the half-resolution grid.
    const int wsh = 31 - __clz(p.W);
    auto load_res = [&](int uu, int i, int c) {
      const int64_t mw = unit_m0(uu) + i * BM + q * 32;  // the warp's first pixel
      const float* src = p.res + (uu % p.n_tiles) * BN + c + 4 * pc;
      if (!p.res_up) {
#pragma unroll
        for (int k = 0; k < 8; ++k) nx[k] = *reinterpret_cast<const float4*>(src + (mw + pr + 4 * k) * p.Cout);
      } else {
        const int64_t w0 = mw / HW;
        const int r0 = (int)(mw - w0 * HW);
        const int64_t b0 = w0 * (HW / 4);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int rr = r0 + pr + 4 * k, yy = rr >> wsh, xx = rr & (p.W - 1);
          nx[k] = *reinterpret_cast<const float4*>(src + (b0 + (yy >> 1) * (p.W >> 1) + (xx >> 1)) * p.Cout);
        }
      }
    };
    if (p.res && cta0 < n_units) load_res(cta0, 0, 0);
    // PAIR: the accumulator is released on the even CTA's barrier
    const uint32_t acce_remote = PAIR && rank == 1 ? peer_addr(&acce_bar[0], 0) : 0u;
    for (int u = cta0; u < n_units; u += ncta, ++acc) {
      const uint32_t buf = acc & 1u, aph = (acc >> 1) & 1u;
      if (!wait_bar<PAIR>(&accf_bar[buf], aph, abort_flag, p.status, true, p.wait_limit)) break;
      fence_after();
      const int n0 = (u % p.n_tiles) * BN;
#pragma unroll 1
      for (int i = 0; i < MT; ++i) {
        const int64_t m = unit_m0(u) + i * BM + row;
        const int64_t mw = unit_m0(u) + i * BM + q * 32;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
          float4 rv[8];
          if (p.res) {
#pragma unroll
            for (int k = 0; k < 8; ++k) *reinterpret_cast<float4*>(T + (pr + 4 * k) * 36 + 4 * pc) = nx[k];
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 8; ++j) rv[j] = *reinterpret_cast<const float4*>(T + lane * 36 + 4 * j);
            if (c0 + 32 < BN) load_res(u, i, c0 + 32);
            else if (i + 1 < MT) load_res(u, i + 1, 0);
            else if (u + ncta < n_units) load_res(u + ncta, 0, 0);
          }
          uint32_t r[32];
          tmem_ld32(tmem + buf * ACC_COLS + i * BN + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float4 v = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                   __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
            if (p.res) {
              v.x += rv[j].x; v.y += rv[j].y; v.z += rv[j].z; v.w += rv[j].w;
            }
            *reinterpret_cast<float4*>(T + lane * 36 + 4 * j) = v;
            r[4 * j] = __float_as_uint(v.x);
            r[4 * j + 1] = __float_as_uint(v.y);
            r[4 * j + 2] = __float_as_uint(v.z);
            r[4 * j + 3] = __float_as_uint(v.w);
          }
          __syncwarp();
          // the warp's 32 pixels x 32 channels leave in whole 128-byte chunks
          if (!p.out_up) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
              *reinterpret_cast<float4*>(p.y + (mw + pr + 4 * k) * p.Cout + n0 + c0 + 4 * pc) =
                  *reinterpret_cast<const float4*>(T + (pr + 4 * k) * 36 + 4 * pc);
          } else {
            const int64_t w0 = mw / HW;
            const int r0 = (int)(mw - w0 * HW);
            const int64_t b0 = w0 * (4 * HW);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int rr = r0 + pr + 4 * k, yy = rr >> wsh, xx = rr & (p.W - 1);
              const int64_t mo = b0 + (int64_t)(2 * yy + p.py) * (2 * p.W) + (2 * xx + p.px);
              *reinterpret_cast<float4*>(p.y + mo * p.Cout + n0 + c0 + 4 * pc) =
                  *reinterpret_cast<const float4*>(T + (pr + 4 * k) * 36 + 4 * pc);
            }
          }
          __syncwarp();  // T is free for the next chunk
          if (p.bstats) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float sum = 0.0f;
#pragma unroll
              for (int k = 0; k < 16; ++k) sum += __uint_as_float(r[16 * h + k]);
              float mu = sum * 0.0625f, m2 = 0.0f;
#pragma unroll
              for (int k = 0; k < 16; ++k) {
                const float dv = __uint_as_float(r[16 * h + k]) - mu;
                m2 = fmaf(dv, dv, m2);
              }
              // merge equal-count partials of lanes l and l ^ o (n values each)
              float half_n = 16.0f * 0.5f;
#pragma unroll
              for (int o = 1; o < 32; o <<= 1) {
                const float mo = __shfl_xor_sync(0xffffffffu, mu, o);
                const float m2o = __shfl_xor_sync(0xffffffffu, m2, o);
                const float dm = mo - mu;
                m2 = (m2 + m2o) + dm * dm * half_n;
                mu = (mu + mo) * 0.5f;
                half_n *= 2.0f;
              }
              if (lane == 0)
                p.bstats[(m >> 5) * (p.Cout >> 4) + ((n0 + c0) >> 4) + h] = make_float2(mu, m2);
            }
          }
        }
      }
      fence_before();
      if (PAIR && rank == 1) mbar_arrive_remote(acce_remote + 8u * buf);
      else mbar_arrive(&acce_bar[buf]);
    }
  } else if constexpr (XF) {
    // Transform warpgroup (XF).  Thread t owns the 16-byte chunk t % 8 of
    // pixels t / 8, t / 8 + 16, ... of every stage; with pixel rows 128
    // bytes apart from a 1024-aligned base, the 128-byte swizzle puts
    // logical chunk jl (channels 4 jl .. 4 jl + 3 of the stage's slice) at
    // physical chunk jl ^ (pixel % 8), the same for all of them.
    const int t = (int)threadIdx.x - 192;
    const int jp = t & 7;
    const int jl = jp ^ ((t >> 3) & 7);
    uint32_t it = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const int64_t m0 = (int64_t)(u / p.n_tiles) * (BM * MT);
      const int win = (int)(m0 / HW);
      const int y0 = (int)((m0 % HW) / p.W);
      for (int kk = 0; kk < p.n_iter; ++kk, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (it / STAGES) & 1u;
        const bool got = wait_bar(&full_bar[s], ph, abort_flag, p.status, true, p.wait_limit);
        if (!bar_and(got, 1, XF_THREADS)) {
          ok = false;
          break;
        }
        // the staged box: origin (bx0, by0) in the window, bw pixels per row
        int bx0, by0, bw, npx, kc;
        bool norm;
        if (kk >= p.n_iter1) {
          // folded 1x1 operand: raw float32, used as tf32 as it is
          kc = kk - p.n_iter1;
          bx0 = 0; by0 = y0; bw = p.W; npx = 0; norm = false;
        } else if (DXR) {
          kc = kk % p.n_kc;
          bx0 = p.ox; by0 = y0 + kk / p.n_kc + p.oy; bw = BM + 2; npx = (BM + 2) * MT;
          norm = p.xf_stats != nullptr;
        } else {
          const int tap = kk / p.n_kc;
          kc = kk % p.n_kc;
          bx0 = tap % p.ks + p.ox; by0 = y0 + tap / p.ks + p.oy; bw = p.W; npx = BM * MT;
          norm = p.xf_stats != nullptr;
        }
        float mu = 0.0f, rs = 1.0f;
        if (norm) {
          const float2 ms = p.xf_stats[(int64_t)win * p.xf_G + (p.xf_coff + kc * p.kch + 4 * jl) / p.xf_cpg];
          mu = ms.x;
          rs = ms.y;
        }
        const bool act = norm && p.xf_silu;
        float* a = reinterpret_cast<float*>(smem + (size_t)s * STAGE_BYTES);
        int px = t >> 3;
        int r = px / bw, xc = px - r * bw;
        for (; px < npx; px += 16) {
          const int xx = bx0 + xc, yy = by0 + r;
          if ((unsigned)xx < (unsigned)p.W && (unsigned)yy < (unsigned)p.H) {
            float4* qp = reinterpret_cast<float4*>(a + px * 32 + jp * 4);
            float4 v = *qp;
            if (norm) {
              v.x = (v.x - mu) * rs;
              v.y = (v.y - mu) * rs;
              v.z = (v.z - mu) * rs;
              v.w = (v.w - mu) * rs;
            }
            if (act) {
              v.x = xf_silu(v.x);
              v.y = xf_silu(v.y);
              v.z = xf_silu(v.z);
              v.w = xf_silu(v.w);
            }
            v.x = xf_tf32(v.x);
            v.y = xf_tf32(v.y);
            v.z = xf_tf32(v.z);
            v.w = xf_tf32(v.w);
            *qp = v;
          }
          xc += 16;
          while (xc >= bw) {
            xc -= bw;
            ++r;
          }
        }
        // make the generic-proxy writes visible to the tensor cores' reads
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&ready_bar[s]);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (PAIR) {
    // neither CTA leaves (or frees its tensor memory) while the other may
    // still signal its barriers
    cluster_sync();
    if (warp == 1) {
      __syncwarp();
      fence_after();
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ACC_COLS)
                   : "memory");
    }
  } else if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ACC_COLS)
                 : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  }
  return n;
}

int g_pair_clusters = 0;  // co-resident CTA pairs of the last pair kernel set up

struct Maps {
  CUtensorMap a, b, alo, blo;      // main operand (and low parts)
  CUtensorMap a2, b2, a2lo, b2lo;  // folded 1x1 operand (copies of the above when absent)
};

// Shared memory of one stage, as the kernel lays it out (PAIR: half the
// weight rows).
constexpr int stage_bytes(int BN, bool SPLIT, bool DXR, int MT, bool PAIR = false) {
  return (SPLIT ? 2 : 1) * ((((DXR ? (BM + 2) * 128 : BM * 128) * MT + 1023) / 1024 * 1024) +
                            (DXR ? 3 : 1) * (PAIR ? BN / 2 : BN) * 128);
}

template <int BN, int STAGES, bool SPLIT, bool DXR, bool TF32, int MT, bool XF = false, bool PAIR = false>
bool launch(const Maps& m, const TcParams& p, cudaStream_t st, std::string* err) {
  // stages, then the epilogue's four 32 x 36-float transpose buffers
  constexpr size_t smem = (size_t)STAGES * stage_bytes(BN, SPLIT, DXR, MT, PAIR) + 1024 + 4 * 32 * 36 * 4;
  static_assert(smem <= 227 * 1024, "stages exceed the shared memory of a CTA");
  static_assert(2 * MT * BN <= 512, "accumulators exceed tensor memory");
  static bool attr = false;
  static int max_pairs = 0;
  auto kern = conv_tc_kernel<BN, STAGES, SPLIT, DXR, TF32, MT, XF, PAIR>;
  if (!attr) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      *err = "cudaFuncSetAttribute failed";
      return false;
    }
    if (PAIR) {
      // co-resident clusters of two (one pair per TPC at most)
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 2;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(2 * (unsigned)(sm_count() / 2));
      cfg.blockDim = dim3(192);
      cfg.dynamicSmemBytes = smem;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n < 1) {
        cudaGetLastError();
        *err = "no co-resident CTA pairs for the tensor-core convolution";
        return false;
      }
      max_pairs = n;
      g_pair_clusters = n;
    }
    attr = true;
  }
  const int units = p.m_tiles / (PAIR ? 2 * MT : MT) * p.n_tiles;
  if (PAIR) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    const int pairs = units < max_pairs ? units : max_pairs;
    cfg.gridDim = dim3(2 * (unsigned)pairs);
    cfg.blockDim = dim3(192);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t le = cudaLaunchKernelEx(&cfg, kern, m.a, m.b, m.alo, m.blo, m.a2, m.b2, m.a2lo, m.b2lo, p);
    if (le != cudaSuccess) {
      cudaGetLastError();
      *err = cudaGetErrorString(le);
      return false;
    }
  } else {
    const int grid = units < sm_count() ? units : sm_count();
    kern<<<grid, XF ? 192 + XF_THREADS : 192, smem, st>>>(m.a, m.b, m.alo, m.blo, m.a2, m.b2, m.a2lo, m.b2lo, p);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return false;
  }
  return true;
}


// ------------------------------------------------------------ attention
// Self-attention of one window and one head on the tensor cores (the
// attention block at the bottom of the fine UNet, Sec. 5.3): 256 tokens
// (16 x 16 pixels), head width 64.  Q, K and V (float32, from the qkv
// projection) are staged in shared memory in the 128-byte swizzled K-major
// layout: Q and K with the tokens as rows, each as a bfloat16 high part and
// the bfloat16 rounding of its remainder (x = hi + lo), V rounded to bfloat16
// and transposed (head channels as rows, tokens along K).  For each of the
// two 128-query M tiles: S = Q K^T (M = 128, N = 256, K = 64) into tensor
// memory as Qhi Khi + Qlo Khi + Qhi Klo (the scores go through exp, so their
// rounding is compensated; bfloat16 alone moved the fine network's output by
// several 1e-3 sigma);
// every thread owns one query row, takes its maximum, p = exp((s - max) / 8)
// and the row sum in float32, and writes p as bfloat16 in the same swizzled
// layout (four 64-key K chunks); then O = P V (M = 128, N = 64, K = 256) into
// tensor memory, and O / sum leaves as the operand of the output projection.
// The products are bfloat16 with float32 accumulation; the softmax is
// float32.  Every wait is bounded (status word, as the convolutions).
template <bool OUT_TF32>
__global__ void __launch_bounds__(128, 1) attention_tc_kernel(const float* __restrict__ qkv, int C, int heads,
                                                              void* __restrict__ out, int* status,
                                                              long long wait_limit) {
  constexpr int TN = 256, D = 64;
  constexpr int Q_OFF = 0, QL_OFF = 32768, K_OFF = 65536, KL_OFF = 98304, V_OFF = 131072, P_OFF = 163840;
  extern __shared__ uint8_t dsmem[];
  uint8_t* sm = dsmem + ((1024 - (smem_u32(dsmem) & 1023)) & 1023);
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_sh;
  __shared__ int skip_sh;
  __shared__ int abort_sh;
  const int b = blockIdx.x / heads, h = blockIdx.x % heads;
  const int tid = threadIdx.x, warp = tid / 32;
  if (tid == 0) {
    skip_sh = *(volatile int*)status;
    abort_sh = 0;
  }
  __syncthreads();
  if (skip_sh) return;
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // 8 bfloat16 values as one 16-byte chunk
  auto pack8 = [](const float* v) {
    uint4 r;
    uint32_t* w = reinterpret_cast<uint32_t*>(&r);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_bfloat162 t = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      w[i] = *reinterpret_cast<const uint32_t*>(&t);
    }
    return r;
  };
  // the same for the bfloat16 remainders x - bf16(x)
  auto pack8_lo = [&](const float* v) {
    float l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) l[i] = v[i] - __bfloat162float(__float2bfloat16_rn(v[i]));
    return pack8(l);
  };
  const float* base = qkv + (int64_t)b * TN * 3 * C + h * D;
  // Q and K: chunk j (channels 8j .. 8j + 7) of token t at row t, physical
  // chunk j ^ (t % 8)
  // (unrolled so that several global loads of each thread are in flight)
#pragma unroll 4
  for (int e = tid; e < TN * 8; e += 128) {
    const int t = e >> 3, j = e & 7;
    float v[8];
    const float4* q = reinterpret_cast<const float4*>(base + (int64_t)t * 3 * C + 8 * j);
    const int o = t * 128 + ((j ^ (t & 7)) << 4);
    *reinterpret_cast<float4*>(v) = q[0];
    *reinterpret_cast<float4*>(v + 4) = q[1];
    *reinterpret_cast<uint4*>(sm + Q_OFF + o) = pack8(v);
    *reinterpret_cast<uint4*>(sm + QL_OFF + o) = pack8_lo(v);
    const float4* k = reinterpret_cast<const float4*>(base + (int64_t)t * 3 * C + C + 8 * j);
    *reinterpret_cast<float4*>(v) = k[0];
    *reinterpret_cast<float4*>(v + 4) = k[1];
    *reinterpret_cast<uint4*>(sm + K_OFF + o) = pack8(v);
    *reinterpret_cast<uint4*>(sm + KL_OFF + o) = pack8_lo(v);
  }
  // V^T: row d of K chunk c holds tokens 64c .. 64c + 63; tokens 8g .. 8g + 7
  // of a chunk form logical chunk g
#pragma unroll 4
  for (int e = tid; e < D * (TN / 8); e += 128) {
    const int d = e % D, tg = e / D, t0 = 8 * tg;
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = base[(int64_t)(t0 + i) * 3 * C + 2 * C + d];
    const int c = t0 / 64, g = (t0 % 64) / 8;
    *reinterpret_cast<uint4*>(sm + V_OFF + c * 8192 + d * 128 + ((g ^ (d & 7)) << 4)) = pack8(v);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_sh;
  const uint32_t S_COL = 0, O_COL = 256;
  const int r = tid;  // query row of the M tile = TMEM lane
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
  volatile int* abort_flag = &abort_sh;
  uint32_t uses = 0;  // completed phases of bar
  bool ok = true;
  for (int m = 0; m < 2 && ok; ++m) {
    if (tid == 0) {
      constexpr uint32_t idS = idesc_mma(128, 256, false);
      const uint32_t a = smem_u32(sm + Q_OFF + m * 16384), al = smem_u32(sm + QL_OFF + m * 16384);
      const uint32_t bk = smem_u32(sm + K_OFF), bl = smem_u32(sm + KL_OFF);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        mma_bf16(tmem + S_COL, umma_desc(a + 32 * k), umma_desc(bk + 32 * k), idS, k > 0);
        mma_bf16(tmem + S_COL, umma_desc(al + 32 * k), umma_desc(bk + 32 * k), idS, 1u);
        mma_bf16(tmem + S_COL, umma_desc(a + 32 * k), umma_desc(bl + 32 * k), idS, 1u);
      }
      mma_commit(&bar);
    }
    // every thread takes the same decision (a lone timeout must not split
    // the block at the barriers below)
    if (!__syncthreads_and(wait_bar(&bar, uses & 1u, abort_flag, status, true, wait_limit))) {
      ok = false;
      break;
    }
    ++uses;
    fence_after();
    float mx = -INFINITY;
    for (int c0 = 0; c0 < TN; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + lane_off + S_COL + c0, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) mx = fmaxf(mx, __uint_as_float(v[i]));
    }
    float sum = 0.0f;
    for (int c0 = 0; c0 < TN; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + lane_off + S_COL + c0, v);
      float pv[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        pv[i] = __expf((__uint_as_float(v[i]) - mx) * 0.125f);
        sum += pv[i];
      }
      const int c = c0 / 64;
#pragma unroll
      for (int g4 = 0; g4 < 4; ++g4) {
        const int g = (c0 % 64) / 8 + g4;
        *reinterpret_cast<uint4*>(sm + P_OFF + c * 16384 + r * 128 + ((g ^ (r & 7)) << 4)) = pack8(pv + 8 * g4);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
      constexpr uint32_t idO = idesc_mma(128, 64, false);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint32_t a = smem_u32(sm + P_OFF + c * 16384), bv = smem_u32(sm + V_OFF + c * 8192);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          mma_bf16(tmem + O_COL, umma_desc(a + 32 * k), umma_desc(bv + 32 * k), idO, (c | k) > 0);
      }
      mma_commit(&bar);
    }
    if (!__syncthreads_and(wait_bar(&bar, uses & 1u, abort_flag, status, true, wait_limit))) {
      ok = false;
      break;
    }
    ++uses;
    fence_after();
    const float inv = 1.0f / sum;
    const int64_t row = (int64_t)b * TN + m * 128 + r;
#pragma unroll
    for (int c0 = 0; c0 < D; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + lane_off + O_COL + c0, v);
      float o[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) o[i] = __uint_as_float(v[i]) * inv;
      if (OUT_TF32) {
        float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + row * C + h * D + c0);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          dst[i] = make_float4(xf_tf32(o[4 * i]), xf_tf32(o[4 * i + 1]), xf_tf32(o[4 * i + 2]), xf_tf32(o[4 * i + 3]));
      } else {
        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(out) + row * C + h * D + c0);
#pragma unroll
        for (int i = 0; i < 4; ++i) dst[i] = pack8(o + 8 * i);
      }
    }
    fence_before();
    __syncthreads();  // S and O are free for the next M tile
    fence_after();
  }
  if (!ok) {
    // let the products already issued finish before freeing their memory
    wait_bar(&bar, uses & 1u, abort_flag, status, false, wait_limit);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

}  // namespace

int conv_tc_pair_clusters() { return g_pair_clusters; }

bool conv_tc_supported(int cin, int cout, int ks) {
  return (ks == 1 || ks == 2 || ks == 3) && cin >= 64 && cin % 64 == 0 && cout >= 64 && cout % 64 == 0 &&
         (cout <= 256 || cout % 256 == 0);
}

std::vector<TcTile> conv_tc_tiles(int H, int W, int Cin, int Cout, int ks, bool split, bool /*xf*/,
                                  const TcGeom* geom) {
  std::vector<TcTile> out;
  if (!conv_tc_supported(Cin, Cout, ks) || !conv_tc_shape_ok(H, W)) return out;
  for (int bn : {64, 128, 256}) {
    if (bn > Cout || Cout % bn) continue;
    const bool dxr_ok = ks == 3 && W == 128 && bn == 64 && (!geom || (geom->oy == -1 && geom->ox == -1));
    const bool mt2_ok = ((int64_t)H * W / BM) % 2 == 0 && !(split && bn == 64) && bn <= 128;
    for (int mt = 1; mt <= (mt2_ok ? 2 : 1); ++mt)
      for (int dx = 0; dx <= (dxr_ok ? 1 : 0); ++dx) {
        // split kernels exist for BN = 64 (MT 1), 128 (MT 1, 2), 256 (MT 1)
        if (split && bn == 64 && mt == 2) continue;
        TcTile t;
        t.bn = bn;
        t.mt = mt;
        t.dxr = dx;
        out.push_back(t);
      }
  }
  return out;
}

bool conv_tc_shape_ok(int H, int W) {
  return W >= 1 && W <= 128 && 128 % W == 0 && ((int64_t)H * W) % 128 == 0 && 128 / W <= H;
}

bool conv_tc_forward(const void* x, const void* w, const void* x_lo, const void* w_lo, const float* res,
                     float* y, float2* bstats, int n, int H, int W, int Cin, int Cout, int ks, int* status,
                     cudaStream_t st, std::string* err, const void* x2, const void* w2, const void* x2_lo,
                     const void* w2_lo, int Cin2, bool tf32, const TcGeom* geom, const TcXf* xf,
                     long long wait_limit, const TcTile* tile) {
  if (!conv_tc_supported(Cin, Cout, ks) || !conv_tc_shape_ok(H, W)) {
    *err = "shape not supported by the tensor-core convolution";
    return false;
  }
  const bool fold = x2 != nullptr;
  if (fold && (!w2 || !conv_tc_supported(Cin2, Cout, 1))) {
    *err = "folded 1x1 operand not supported by the tensor-core convolution";
    return false;
  }
  auto enc = encode_fn();
  if (!enc) {
    *err = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  int BN = Cout <= 256 ? Cout : 256;
  if (tile && tile->bn > 0) {
    if (!(tile->bn == 64 || tile->bn == 128 || tile->bn == 256) || Cout % tile->bn) {
      *err = "invalid tile shape (BN)";
      return false;
    }
    BN = tile->bn;
  }
  const bool split = x_lo && w_lo;
  if (tf32 && split) {
    *err = "tf32 operands have no low parts";
    return false;
  }
  if (xf && (!tf32 || (xf->stats && (xf->G < 1 || xf->cpg < 1 || xf->cpg % 4)))) {
    *err = "the operand transform needs raw float32 (tf32) operands and 4-channel-aligned groups";
    return false;
  }
  // one K stage reads 128 bytes of channels per pixel / weight row
  const int es = tf32 ? 4 : 2, kch = 128 / es;
  const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (fold && split != (x2_lo && w2_lo)) {
    *err = "folded operand low parts must be given exactly when the main operand's are";
    return false;
  }
  Maps m;
  // 3x3 convs on 128-pixel rows stage one 130-pixel box per kernel row
  const bool dxr_ok = ks == 3 && W == 128 && BN == 64 && (!geom || (geom->oy == -1 && geom->ox == -1));
  const bool dxr = dxr_ok && !(tile && tile->dxr == 0);
  // activations (n, H, W, C); box of kch channels x bw pixels x bh rows
  auto encA = [&](CUtensorMap* mp, const void* ptr, int C, int bw, int bh) {
    cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)n};
    cuuint64_t strides[3] = {(cuuint64_t)C * es, (cuuint64_t)W * C * es, (cuuint64_t)H * W * C * es};
    cuuint32_t box[4] = {(cuuint32_t)kch, (cuuint32_t)bw, (cuuint32_t)bh, 1};
    cuuint32_t ones[4] = {1, 1, 1, 1};
    return enc(mp, dt, 4, (void*)ptr, dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  // CTA pairs (cta_group::2): plain operands, and every CTA's MT M tiles
  // paired with the next MT (an even number of unit halves).  pair == 1
  // requires them, pair == 2 takes them where the shape allows.
  const int64_t m_tiles = (int64_t)n * H * W / BM;
  const bool pair_shape = !split && !xf;
  bool pair = tile && (tile->pair == 1 || (tile->pair == 2 && pair_shape));
  // weights [tap][Cout][C]; box of kch channels x BN rows (a pair's CTA
  // stages BN / 2 of them)
  auto encB = [&](CUtensorMap* mp, const void* ptr, int C, int taps) {
    cuuint64_t dims[2] = {(cuuint64_t)C, (cuuint64_t)taps * Cout};
    cuuint64_t strides[1] = {(cuuint64_t)C * es};
    cuuint32_t box[2] = {(cuuint32_t)kch, (cuuint32_t)(pair ? BN / 2 : BN)};
    cuuint32_t ones[2] = {1, 1};
    return enc(mp, dt, 2, (void*)ptr, dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  // two M tiles per work unit when every window holds an even number of
  // them, except for split 64-channel stages (too large twice over)
  const bool mt2_ok = ((int64_t)H * W / BM) % 2 == 0 && !(split && BN == 64) && BN <= 128;
  int mt = mt2_ok ? 2 : 1;
  if (tile && tile->mt > 0) {
    if (tile->mt > 2 || (tile->mt == 2 && !mt2_ok)) {
      *err = "invalid tile shape (MT)";
      return false;
    }
    mt = tile->mt;
  }
  // preferred pairs: where measured faster (N tiles of 128 or 256 weight
  // rows; the 64-channel row-reuse layers stay on one CTA)
  if (pair && tile->pair == 2 && (m_tiles % (2 * mt) != 0 || BN < 128 || dxr)) pair = false;
  if (pair && (!pair_shape || m_tiles % (2 * mt) != 0)) {
    *err = "invalid tile shape (CTA pair): needs plain operands and an even number of unit halves";
    return false;
  }
  const int abw = dxr ? W + 2 : W, abh = dxr ? mt : mt * 128 / W;
  if (!encA(&m.a, x, Cin, abw, abh) || !encB(&m.b, w, Cin, ks * ks)) {
    *err = "tensor map (activations or weights) encode failed";
    return false;
  }
  if (split && (!encA(&m.alo, x_lo, Cin, abw, abh) || !encB(&m.blo, w_lo, Cin, ks * ks))) {
    *err = "tensor map (low parts) encode failed";
    return false;
  }
  if (!split) {
    m.alo = m.a;
    m.blo = m.b;
  }
  if (fold) {
    if (!encA(&m.a2, x2, Cin2, W, mt * 128 / W) || !encB(&m.b2, w2, Cin2, 1)) {
      *err = "tensor map (folded operand) encode failed";
      return false;
    }
    if (split && (!encA(&m.a2lo, x2_lo, Cin2, W, mt * 128 / W) || !encB(&m.b2lo, w2_lo, Cin2, 1))) {
      *err = "tensor map (folded operand low parts) encode failed";
      return false;
    }
    if (!split) {
      m.a2lo = m.a2;
      m.b2lo = m.b2;
    }
  } else {
    m.a2 = m.a;
    m.b2 = m.b;
    m.a2lo = m.alo;
    m.b2lo = m.blo;
  }
  TcParams p;
  p.res = res;
  p.y = y;
  p.bstats = bstats;
  p.status = status;
  p.H = H;
  p.W = W;
  p.Cout = Cout;
  p.ks = ks;
  const TcGeom g = geom ? *geom : TcGeom{};
  p.oy = geom ? g.oy : -(ks / 2);
  p.ox = geom ? g.ox : -(ks / 2);
  p.out_up = g.out_up;
  p.py = g.py;
  p.px = g.px;
  p.res_up = g.res_up;
  if ((p.out_up && (bstats || res)) || (p.res_up && ((H | W) & 1))) {
    *err = "unsupported combination of phase output, residual and statistics";
    return false;
  }
  p.kch = kch;
  p.n_kc = Cin / kch;
  p.n_iter1 = (dxr ? ks : ks * ks) * p.n_kc;
  p.n_iter = p.n_iter1 + (fold ? Cin2 / kch : 0);
  p.m_tiles = (int)((int64_t)n * H * W / BM);
  p.n_tiles = Cout / BN;
  p.wait_limit = wait_limit > 0 ? wait_limit : 1000000000LL;
  p.xf_stats = xf ? xf->stats : nullptr;
  p.xf_G = xf ? xf->G : 1;
  p.xf_cpg = xf ? xf->cpg : 1;
  p.xf_coff = xf ? xf->coff : 0;
  p.xf_silu = xf ? xf->silu : 0;
  if (xf) {
    // raw float32 operands normalised (or rounded) in shared memory
    if (mt == 2) {
      switch (BN) {
        case 64: return dxr ? launch<64, 3, false, true, true, 2, true>(m, p, st, err)
                            : launch<64, 5, false, false, true, 2, true>(m, p, st, err);
        case 128: return launch<128, 4, false, false, true, 2, true>(m, p, st, err);
      }
    } else {
      switch (BN) {
        case 64: return dxr ? launch<64, 5, false, true, true, 1, true>(m, p, st, err)
                            : launch<64, 8, false, false, true, 1, true>(m, p, st, err);
        case 128: return launch<128, 6, false, false, true, 1, true>(m, p, st, err);
        case 256: return launch<256, 4, false, false, true, 1, true>(m, p, st, err);
      }
    }
    *err = "unsupported N tile";
    return false;
  }
  if (pair) {
    // stages: about 180-205 KB per CTA (a third fewer bytes per stage)
#define IDF_TC_PAIR(TF)                                                                       \
    if (mt == 2) {                                                                            \
      switch (BN) {                                                                           \
        case 64: return dxr ? launch<64, 4, false, true, TF, 2, false, true>(m, p, st, err)   \
                            : launch<64, 5, false, false, TF, 2, false, true>(m, p, st, err); \
        case 128: return launch<128, 5, false, false, TF, 2, false, true>(m, p, st, err);     \
      }                                                                                       \
    } else {                                                                                  \
      switch (BN) {                                                                           \
        case 64: return dxr ? launch<64, 6, false, true, TF, 1, false, true>(m, p, st, err)   \
                            : launch<64, 8, false, false, TF, 1, false, true>(m, p, st, err); \
        case 128: return launch<128, 8, false, false, TF, 1, false, true>(m, p, st, err);     \
        case 256: return launch<256, 6, false, false, TF, 1, false, true>(m, p, st, err);     \
      }                                                                                       \
    }
    if (tf32) {
      IDF_TC_PAIR(true)
    } else {
      IDF_TC_PAIR(false)
    }
#undef IDF_TC_PAIR
    *err = "unsupported N tile";
    return false;
  }
  // stages: about 170-200 KB of shared memory per CTA, one CTA per SM
  if (!split) {
    // bfloat16 or tf32 operands: the same stage bytes
#define IDF_TC_PLAIN(TF)                                                                      \
    if (mt == 2) {                                                                            \
      switch (BN) {                                                                           \
        case 64: return dxr ? launch<64, 3, false, true, TF, 2>(m, p, st, err)                \
                            : launch<64, 5, false, false, TF, 2>(m, p, st, err);              \
        case 128: return launch<128, 4, false, false, TF, 2>(m, p, st, err);                  \
      }                                                                                       \
    } else {                                                                                  \
      switch (BN) {                                                                           \
        case 64: return dxr ? launch<64, 5, false, true, TF, 1>(m, p, st, err)                \
                            : launch<64, 8, false, false, TF, 1>(m, p, st, err);              \
        case 128: return launch<128, 6, false, false, TF, 1>(m, p, st, err);                  \
        case 256: return launch<256, 4, false, false, TF, 1>(m, p, st, err);                  \
      }                                                                                       \
    }
    if (tf32) {
      IDF_TC_PLAIN(true)
    } else {
      IDF_TC_PLAIN(false)
    }
#undef IDF_TC_PLAIN
  } else {
    switch (BN) {
      case 64: return dxr ? launch<64, 2, true, true, false, 1>(m, p, st, err)
                          : launch<64, 4, true, false, false, 1>(m, p, st, err);
      case 128: return mt == 2 ? launch<128, 2, true, false, false, 2>(m, p, st, err)
                               : launch<128, 3, true, false, false, 1>(m, p, st, err);
      case 256: return launch<256, 2, true, false, false, 1>(m, p, st, err);
    }
  }
  *err = "unsupported N tile";
  return false;
}


bool attention_tc_supported(int Tn, int dh) { return Tn == 256 && dh == 64; }

bool attention_tc_forward(const float* qkv, int n, int C, int heads, void* out, bool out_tf32, int* status,
                          long long wait_limit, cudaStream_t st, std::string* err) {
  if (C != heads * 64) {
    *err = "attention: head width must be 64";
    return false;
  }
  constexpr size_t smem = 229376 + 1024;
  static bool attr[2] = {false, false};
  auto kern = out_tf32 ? attention_tc_kernel<true> : attention_tc_kernel<false>;
  if (!attr[out_tf32]) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      *err = "cudaFuncSetAttribute failed";
      return false;
    }
    attr[out_tf32] = true;
  }
  kern<<<n * heads, 128, smem, st>>>(qkv, C, heads, out, status, wait_limit > 0 ? wait_limit : 1000000000LL);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return false;
  }
  return true;
}

}  // namespace idf
