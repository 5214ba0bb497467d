// idf_laplacian_decode_noalloc: the Laplacian decode without any device
// allocation, for callers that cannot allocate device memory when they call
// us.  Examples: a plugin inside a host engine that hands out all device
// memory from its own pool and forbids cudaMalloc, or a frame loop that
// cannot afford the latency and implicit synchronization of an allocation.
//
// The decode needs coarse-grid scratch (the down-sampled provisional image,
// its horizontal blur, the re-extracted low band and the blur taps).  Here
// it lives in one file-scope device array of fixed size that every GPU
// loading the library holds until the process exits.  Host code cannot use
// the array's name as a device address (on the host it names a stand-in
// object), so the first call on each device, with that device current, asks
// the runtime for the array's device address with cudaGetSymbolAddress and
// keeps it; later calls on that device reuse it.  That first call should
// come before any stream capture.
//
// All calls on a device share the array and it keeps the last call's
// contents.  Each call writes every scratch element before reading it, so
// nothing needs clearing, but calls whose kernels overlap on the GPU (e.g.
// on two streams without ordering between them) race on the array.
#include <mutex>
#include <string>
#include <vector>

#include "../../include/idf.h"
#include "internal.h"

namespace {

// 2^20 floats (4 MiB): enough for every query up to 4096 x 4096 pixels with
// an 8x factor and blur radius 15 (about 0.85 Mi floats).
constexpr size_t kScratchFloats = (size_t)1 << 20;

static __device__ __align__(256) float g_decode_scratch[kScratchFloats];

std::mutex g_mu;
float* g_scratch_ptr[256] = {};

// Device address of the scratch array on the current device (set up once).
float* scratch_on_current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_decode_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return nullptr;
    }
    g_scratch_ptr[dev] = (float*)p;
  }
  return g_scratch_ptr[dev];
}

// Gaussian taps exp(-k^2 / (2 sigma^2)), |k| <= R, normalised, in double.
__global__ void taps_kernel(float* taps, double sigma, int R) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int k = -R; k <= R; ++k) s += exp(-(double)k * k / (2.0 * sigma * sigma));
  for (int k = -R; k <= R; ++k) taps[k + R] = (float)(exp(-(double)k * k / (2.0 * sigma * sigma)) / s);
}

}  // namespace

extern "C" idf_status idf_laplacian_decode_noalloc(
    const idf_model_stack* stack, const float* L_dev, int64_t lx0, int64_t ly0, int32_t lw, int32_t lh,
    int64_t lpitch, const float* H_dev, int64_t hx0, int64_t hy0, int32_t hw, int32_t hh, int64_t hpitch,
    int64_t x0, int64_t y0, int32_t w, int32_t h, float* out_dev, int64_t pitch, void* stream) {
  using idf::fdiv;
  if (!stack || !L_dev || !H_dev || !out_dev || w < 1 || h < 1 || pitch < w || lpitch < lw || hpitch < hw)
    return IDF_EINVAL;
  const int f = stack->lap_factor, R = stack->lap_radius;
  if (f < 2 || f % 2 || R < 0 || R > 64 || !(stack->lap_blur_sigma > 0)) return IDF_EINVAL;
  const int64_t lim = (int64_t)1 << 40;
  if (x0 < -lim || y0 < -lim || x0 + w > lim || y0 + h > lim) return IDF_EINVAL;
  // coarse rect of the re-extracted low band the output reads, and the band rects
  auto lo = [&](int64_t c) { return fdiv(2 * c + 1 - f, 2 * f); };
  const int64_t qx0 = lo(x0), qy0 = lo(y0);
  const int64_t qw = lo(x0 + w - 1) + 1 - qx0 + 1, qh = lo(y0 + h - 1) + 1 - qy0 + 1;
  const int64_t Lx0 = qx0 - R - 1, Ly0 = qy0 - R - 1, Lw = qw + 2 * R + 2, Lh = qh + 2 * R + 2;
  const int64_t Hx0 = (int64_t)f * (qx0 - R), Hy0 = (int64_t)f * (qy0 - R);
  const int64_t Hw = (int64_t)f * (qw + 2 * R), Hh = (int64_t)f * (qh + 2 * R);
  if (Lx0 < lx0 || Ly0 < ly0 || Lx0 + Lw > lx0 + lw || Ly0 + Lh > ly0 + lh) return IDF_EINVAL;
  if (Hx0 < hx0 || Hy0 < hy0 || Hx0 + Hw > hx0 + hw || Hy0 + Hh > hy0 + hh) return IDF_EINVAL;
  const size_t nD = (size_t)(qw + 2 * R) * (qh + 2 * R);
  const size_t nT = (size_t)qw * (qh + 2 * R);
  const size_t nQ = (size_t)qw * qh;
  const size_t need = nD + nT + nQ + (size_t)(2 * R + 1);
  if (need > kScratchFloats) return IDF_EINVAL;  // query too large for the fixed scratch
  float* scratch = scratch_on_current_device();
  if (!scratch) return IDF_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  idf::DecodeArgs a{};
  a.L = L_dev; a.lx0 = lx0; a.ly0 = ly0; a.lpitch = lpitch; a.lw = lw; a.lh = lh;
  a.H = H_dev; a.hx0 = hx0; a.hy0 = hy0; a.hpitch = hpitch; a.hw = hw; a.hh = hh;
  a.x0 = x0; a.y0 = y0; a.w = w; a.h = h; a.out = out_dev; a.pitch = pitch;
  a.f = f; a.R = R;
  a.low_mu = (float)stack->low_mu; a.low_scale = (float)stack->low_scale; a.res_scale = (float)stack->res_scale;
  a.D = scratch;
  a.T = a.D + nD;
  a.Lhat = a.T + nT;
  float* taps = a.Lhat + nQ;
  a.taps = taps;
  a.qx0 = qx0; a.qy0 = qy0; a.qw = (int)qw; a.qh = (int)qh;
  taps_kernel<<<1, 32, 0, st>>>(taps, stack->lap_blur_sigma, R);
  idf::launch_decode(a, st);
  return cudaGetLastError() == cudaSuccess ? IDF_OK : IDF_ECUDA;
}
