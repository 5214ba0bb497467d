// libidf host side: worlds, the tile-dependency scheduler, the device tile
// cache and the C ABI of include/idf.h.
//
// Scheduling (Alg. 1 made step-synchronous, Thm 3).  A level's canvas is
// cut into stride x stride tiles aligned at multiples of the stride; window
// (i, j) covers tiles i..i+r-1 x j..j+r-1 (r = window / stride).  A query
// needs the tiles of J_K that cover it.  Walking the steps backwards, the
// tiles of J_k that are not cached are "missing"; the windows evaluated at
// step k-1 are kappa of the missing tiles (Alg. 3: for a tile t, windows
// t-r+1..t per axis), and their inputs are the tiles of J_{k-1} they cover.
// Execution then runs forward, one round per step: gather every window of
// the step into one batch, evaluate the network, and blend the missing
// tiles of J_k (fused update and re-noise).
//
// Caching.  The cache holds finalized tiles of every step (all r^2 windows
// of a tile applied, normalised, updated), keyed by (step, tile row, tile
// column) per level, with LRU eviction of tiles the running query does not
// use.  A tile's value depends only on the seed and its position (Lemma 3),
// so any cache state gives the same results; evicting a tile only makes the
// windows that produce it count as unprocessed again (Sec. 3.3).
#include <math.h>
#include <stdio.h>
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

using namespace idf;

namespace {

inline uint64_t tkey(int32_t a, int32_t b) { return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b; }
inline int32_t khi(uint64_t k) { return (int32_t)(uint32_t)(k >> 32); }
inline int32_t klo(uint64_t k) { return (int32_t)(uint32_t)k; }

struct TileCache {
  int s = 0;
  int64_t n_slots = 0;
  float* pool = nullptr;
  std::vector<std::unordered_map<uint64_t, int32_t>> map;  // [step] -> slot
  std::vector<int32_t> slot_step;
  std::vector<uint64_t> slot_key;
  std::vector<int32_t> prv, nxt;
  int32_t head = -1, tail = -1;  // head = least recently used
  std::vector<uint32_t> pin;
  uint32_t epoch = 1;
  std::vector<int32_t> free_list;
  int64_t hits = 0, misses = 0, evictions = 0;

  void unlink(int32_t sl) {
    if (prv[sl] >= 0) nxt[prv[sl]] = nxt[sl]; else head = nxt[sl];
    if (nxt[sl] >= 0) prv[nxt[sl]] = prv[sl]; else tail = prv[sl];
    prv[sl] = nxt[sl] = -1;
  }
  void push_back(int32_t sl) {
    prv[sl] = tail;
    nxt[sl] = -1;
    if (tail >= 0) nxt[tail] = sl; else head = sl;
    tail = sl;
  }
  void touch(int32_t sl) {
    unlink(sl);
    push_back(sl);
    pin[sl] = epoch;
  }
  int32_t alloc() {
    if (!free_list.empty()) {
      int32_t sl = free_list.back();
      free_list.pop_back();
      return sl;
    }
    for (int32_t sl = head; sl >= 0; sl = nxt[sl]) {
      if (pin[sl] == epoch) continue;
      map[slot_step[sl]].erase(slot_key[sl]);
      unlink(sl);
      evictions++;
      return sl;
    }
    return -1;
  }
  void insert(int step, uint64_t key, int32_t sl) {
    map[step][key] = sl;
    slot_step[sl] = step;
    slot_key[sl] = key;
    push_back(sl);
    pin[sl] = epoch;
  }
  void clear() {
    for (auto& m : map) m.clear();
    free_list.clear();
    for (int64_t i = n_slots - 1; i >= 0; --i) free_list.push_back((int32_t)i);
    std::fill(prv.begin(), prv.end(), -1);
    std::fill(nxt.begin(), nxt.end(), -1);
    head = tail = -1;
  }
};

struct StepPlan {
  std::vector<int32_t> win_ij;     // 2 per window, sorted (i, then j)
  std::vector<int32_t> win_slots;  // r*r per window: slots of the J_k tiles (k >= 1)
  std::vector<int32_t> tiles;      // 4 per tile of J_{k+1} to compute
  std::vector<int32_t> tile_wins;  // r*r per tile
  size_t off_win_ij = 0, off_win_slots = 0, off_tiles = 0, off_tile_wins = 0;
};

struct Level {
  idf_level_desc d{};
  std::vector<int32_t> ch;
  // K sampler steps grouped into R blended rounds of rsteps[k] steps from
  // rstart[k] (one step per round unless the level asks otherwise); the
  // cone, the cache and the tables are indexed by round
  int H = 0, s = 0, r = 0, K = 0, R = 0, index = 0;
  std::vector<int> rsteps, rstart;
  std::vector<int32_t> rsteps_copy;
  std::vector<double> sig, c_skip, c_out, c_in;
  float* d_w1 = nullptr;
  float* d_invB1 = nullptr;
  UNet* unet = nullptr;
  TileCache cache;
  int64_t windows_evaluated = 0, tiles_computed = 0;
  int64_t store_reads = 0, store_writes = 0;
  // conditioning vector and embedding (cond_dim > 0), AutoGuidance guide
  std::vector<float> condz;
  float* d_condE = nullptr;   // the main network's embedding E
  float* d_condEg = nullptr;  // the guide network's own E
  float* d_condz = nullptr;
  UNet* guide = nullptr;
  float w_guide = 0.0f;
};

}  // namespace

struct idf_world {
  uint64_t seed = 0;
  idf_model_stack stack{};
  idf_world_opts opts{};
  std::vector<Level> lv;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_join = nullptr;
  std::string last_error;
  bool poisoned = false;
  // growable device buffers
  float* F = nullptr; size_t F_cap = 0;
  float* x_in = nullptr; size_t x_cap = 0;
  float* xs = nullptr; size_t xs_cap = 0;          // window states of multi-step rounds
  float* bias = nullptr; size_t bias_cap = 0;      // per-window conditioning biases (main, then guide)
  float* Fg = nullptr; size_t Fg_cap = 0;          // guide network outputs
  int32_t* tab = nullptr; size_t tab_cap = 0;
  float* dense = nullptr; size_t dense_cap = 0;    // assembled level results
  float* dec = nullptr; size_t dec_cap = 0;        // decode scratch
  float* outbuf = nullptr; size_t out_cap = 0;     // for host-output queries
  float* d_taps = nullptr;
  float* d_fixture = nullptr;                      // given low band (single-level Laplacian stack)
  int* d_err = nullptr;
  int32_t* h_tab = nullptr; size_t h_tab_cap = 0; // pinned staging
  void* arena = nullptr; size_t arena_bytes = 0;  // UNet activations, shared by the levels
  int64_t launches = 0, queries = 0;
  Prof prof;
  // persistent tile store (idf_world_store_open) and its pinned staging
  uint64_t identity = 0;
  TileStore* store = nullptr;
  bool store_writable = false;
  float* h_store = nullptr; size_t h_store_cap = 0;
};

namespace {

idf_status fail(idf_world* w, idf_status code, const std::string& msg) {
  if (w) {
    w->last_error = msg;
    if (code == IDF_ECUDA || code == IDF_ETIMEOUT) w->poisoned = true;
  }
  return code;
}

bool cuda_ok(idf_world* w, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  w->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  w->poisoned = true;
  return false;
}

template <typename T>
bool grow(idf_world* w, T** p, size_t* cap, size_t n, const char* what) {
  if (n <= *cap) return true;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  size_t want = std::max(n, (size_t)(*cap * 3 / 2));
  if (cudaMalloc((void**)p, want * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    w->last_error = std::string("cudaMalloc ") + what + " failed";
    return false;
  }
  *cap = want;
  return true;
}

// sigma schedule (EDM rho form) and preconditioning, FP64 on the host
void schedule(Level& L) {
  const int K = L.K;
  const double a = pow(L.d.sigma_max, 1.0 / L.d.rho), b = pow(L.d.sigma_min, 1.0 / L.d.rho);
  L.sig.resize(K);
  for (int k = 0; k < K; ++k)
    L.sig[k] = K == 1 ? L.d.sigma_max : pow(a + (double)k / (K - 1) * (b - a), L.d.rho);
  const double sd = L.d.sigma_data;
  L.c_skip.resize(K);
  L.c_out.resize(K);
  L.c_in.resize(K);
  for (int k = 0; k < K; ++k) {
    const double s2 = L.sig[k] * L.sig[k] + sd * sd;
    L.c_skip[k] = sd * sd / s2;
    L.c_out[k] = L.sig[k] * sd / sqrt(s2);
    L.c_in[k] = 1.0 / sqrt(s2);
  }
}

UNetDesc unet_desc(const idf_level_desc& d) {
  UNetDesc u;
  u.levels = d.levels;
  u.ch.assign(d.channels, d.channels + d.levels);
  u.in_ch = d.in_ch;
  u.out_ch = d.out_ch;
  u.groups = d.gn_groups;
  u.attn = d.attn_at_bottom;
  u.heads = d.attn_heads;
  u.window = d.window;
  u.cond_dim = d.cond_dim;
  return u;
}

std::string check_level(const idf_level_desc& d, int index) {
  char buf[256];
  auto bad = [&](const char* m) {
    snprintf(buf, sizeof buf, "level %d: %s", index, m);
    return std::string(buf);
  };
  if (d.window < 2 || d.stride < 1 || d.window % d.stride) return bad("window must be a positive multiple of stride");
  if (d.offset != 0) return bad("offset must be 0");
  if (d.steps < 1 || d.steps > 64) return bad("steps must be in [1, 64]");
  if (!(d.sigma_max > 0) || !(d.sigma_min > 0) || !(d.sigma_data > 0) || !(d.rho > 0)) return bad("sigmas must be positive");
  if (d.out_ch != 1) return bad("out_ch must be 1");
  // in_ch 1 (2 with a parent) for a level the sampler runs; other widths
  // (side-input networks, e.g. a student fed the teacher's noise fields)
  // make a network-only world: idf_unet_forward runs, queries do not
  if (d.in_ch < 1 || d.in_ch > 8) return bad("in_ch must be in [1, 8]");
  if (d.scale_to_parent > 0 && index == 0) return bad("the first level has no parent");
  if (d.test_denoiser < 0 || d.test_denoiser > 3) return bad("test_denoiser must be 0..3");
  if (d.n_rounds < 0 || (d.n_rounds > 0 && !d.round_steps)) return bad("round_steps missing");
  if (d.cond_dim < 0 || d.cond_dim > 64 || (d.cond_dim > 0 && !d.cond_z)) return bad("cond_dim in [0, 64] with cond_z");
  if (!(d.guidance == d.guidance)) return bad("guidance must be a number");
  if (d.n_rounds > 0) {
    int64_t sum = 0;
    for (int r = 0; r < d.n_rounds; ++r) {
      if (d.round_steps[r] < 1) return bad("round_steps must be >= 1");
      sum += d.round_steps[r];
    }
    if (sum != d.steps) return bad("round_steps must sum to steps");
  }
  if (d.test_denoiser == 0) {
    if (d.levels < 1 || d.levels > 6 || !d.channels) return bad("levels must be in [1, 6] with channels");
    if (d.window % (1 << (d.levels - 1))) return bad("window must be divisible by 2^(levels-1)");
    if (d.gn_groups < 1) return bad("gn_groups must be >= 1");
    for (int l = 0; l < d.levels; ++l)
      if (d.channels[l] < 1 || d.channels[l] % d.gn_groups) return bad("channels must be positive multiples of gn_groups");
    if (d.attn_at_bottom) {
      const int C = d.channels[d.levels - 1];
      if (d.attn_heads < 1 || C % d.attn_heads || C / d.attn_heads > 64) return bad("attention head width must divide channels and be <= 64");
      const int Hb = d.window >> (d.levels - 1);
      if (Hb * Hb > 1024 || (size_t)2 * Hb * Hb * (C / d.attn_heads) * 4 > 200 * 1024) return bad("attention block too large");
    }
  }
  return "";
}

// ------------------------------------------------------------------ planning
struct LevelPlan {
  std::vector<StepPlan> steps;  // steps[k]: windows on J_k, tiles of J_{k+1}
  int64_t wi_min = 0, wi_max = -1, wj_min = 0, wj_max = -1;
  bool any_windows = false;
  size_t n_win_max = 0;
  // final-round tiles read from the persistent store instead of computed:
  // (slot, key) once slots are allocated
  std::vector<uint64_t> from_store;
  std::vector<std::pair<int32_t, uint64_t>> loads;
};

struct RectT {
  int64_t ty0, tx0, ty1, tx1;  // inclusive tile range
};

// Dense form of plan_level for compact requests: the needed tiles of every
// round, the missing ones and the windows over them are bitmaps over
// bounding boxes instead of hash sets (a cold 8192^2 query touches about a
// million windows), visited row by row, i.e. in the sorted order the hash
// form sorts into, so that the windows, the cache walk (hits touched,
// misses, LRU order), the allocation and the tables are the same.
struct DBox {
  int64_t y0 = 0, x0 = 0, y1 = -1, x1 = -1;
  int64_t h() const { return y1 - y0 + 1; }
  int64_t w() const { return x1 - x0 + 1; }
  int64_t area() const { return h() > 0 && w() > 0 ? h() * w() : 0; }
  int64_t at(int64_t y, int64_t x) const { return (y - y0) * w() + (x - x0); }
};

bool plan_level_dense(Level& L, const std::vector<RectT>& rects, bool dry, LevelPlan& P, std::string* err,
                      TileStore* store) {
  const int K = L.R, r = L.r;
  TileCache& C = L.cache;
  P.steps.assign(K, StepPlan());
  std::vector<DBox> nb(K + 1);                 // need box of J_k
  std::vector<std::vector<int32_t>> slot(K + 1);  // per need cell: -2 not needed, -1 missing, else slot
  std::vector<std::vector<uint64_t>> missing(K + 1);
  std::vector<DBox> wb(K);                      // window box of round k (windows on J_k)
  std::vector<std::vector<int32_t>> widx(K);    // per window cell: batch index or -1
  DBox& b = nb[K];
  b.y0 = rects[0].ty0; b.x0 = rects[0].tx0; b.y1 = rects[0].ty1; b.x1 = rects[0].tx1;
  for (auto& R : rects) {
    b.y0 = std::min(b.y0, R.ty0); b.x0 = std::min(b.x0, R.tx0);
    b.y1 = std::max(b.y1, R.ty1); b.x1 = std::max(b.x1, R.tx1);
  }
  slot[K].assign(b.area(), -2);
  for (auto& R : rects)
    for (int64_t ty = R.ty0; ty <= R.ty1; ++ty)
      for (int64_t tx = R.tx0; tx <= R.tx1; ++tx) slot[K][b.at(ty, tx)] = -1;
  for (int k = K; k >= 1; --k) {
    const DBox& B = nb[k];
    auto& S = slot[k];
    auto& mk = missing[k];
    const bool empty = C.map[k].empty();
    for (int64_t ty = B.y0; ty <= B.y1; ++ty)
      for (int64_t tx = B.x0; tx <= B.x1; ++tx) {
        int32_t& c = S[B.at(ty, tx)];
        if (c == -2) continue;
        const uint64_t t = tkey((int32_t)ty, (int32_t)tx);
        if (!empty) {
          auto it = C.map[k].find(t);
          if (it != C.map[k].end()) {
            if (!dry) {
              C.touch(it->second);
              C.hits++;
            }
            c = it->second;
            continue;
          }
        }
        if (k == K && store && store_has(store, L.index, (int32_t)ty, (int32_t)tx)) {
          P.from_store.push_back(t);
          c = -3;  // filled by the allocation below
        } else {
          mk.push_back(t);
        }
      }
    if (!dry) C.misses += (int64_t)mk.size();
    // windows over the missing tiles: (ty - m, tx - n), m, n < r
    DBox& W = wb[k - 1];
    W.y0 = B.y0 - (r - 1); W.x0 = B.x0 - (r - 1); W.y1 = B.y1; W.x1 = B.x1;
    std::vector<uint8_t> wm(W.area(), 0);
    for (uint64_t t : mk)
      for (int m = 0; m < r; ++m)
        for (int n = 0; n < r; ++n) wm[W.at(khi(t) - m, klo(t) - n)] = 1;
    StepPlan& sp = P.steps[k - 1];
    auto& wi = widx[k - 1];
    wi.assign(W.area(), -1);
    int32_t nw = 0;
    for (int64_t i = W.y0; i <= W.y1; ++i)
      for (int64_t j = W.x0; j <= W.x1; ++j) {
        if (!wm[W.at(i, j)]) continue;
        wi[W.at(i, j)] = nw++;
        sp.win_ij.push_back((int32_t)i);
        sp.win_ij.push_back((int32_t)j);
        if (!P.any_windows) {
          P.wi_min = P.wi_max = i;
          P.wj_min = P.wj_max = j;
        }
        P.any_windows = true;
        P.wi_min = std::min(P.wi_min, i);
        P.wi_max = std::max(P.wi_max, i);
        P.wj_min = std::min(P.wj_min, j);
        P.wj_max = std::max(P.wj_max, j);
      }
    P.n_win_max = std::max(P.n_win_max, (size_t)nw);
    if (k - 1 >= 1) {
      DBox& N = nb[k - 1];
      N.y0 = W.y0; N.x0 = W.x0; N.y1 = W.y1 + (r - 1); N.x1 = W.x1 + (r - 1);
      auto& Sn = slot[k - 1];
      Sn.assign(N.area(), -2);
      for (int64_t i = W.y0; i <= W.y1; ++i)
        for (int64_t j = W.x0; j <= W.x1; ++j) {
          if (!wm[W.at(i, j)]) continue;
          for (int m = 0; m < r; ++m)
            for (int n = 0; n < r; ++n) Sn[N.at(i + m, j + n)] = -1;
        }
    }
  }
  if (dry) return true;
  std::vector<std::pair<int, uint64_t>> inserted;
  auto rollback = [&]() {
    for (auto& kt : inserted) {
      auto it = C.map[kt.first].find(kt.second);
      const int32_t os = it->second;
      C.map[kt.first].erase(it);
      C.unlink(os);
      C.free_list.push_back(os);
    }
    *err = "tile cache too small for this query's working set; raise cache_bytes";
    P.loads.clear();
    return false;
  };
  for (uint64_t t : P.from_store) {
    const int32_t sl = C.alloc();
    if (sl < 0) return rollback();
    C.insert(K, t, sl);
    inserted.emplace_back(K, t);
    P.loads.emplace_back(sl, t);
    slot[K][nb[K].at(khi(t), klo(t))] = sl;
  }
  for (int k = 1; k <= K; ++k)
    for (uint64_t t : missing[k]) {
      const int32_t sl = C.alloc();
      if (sl < 0) return rollback();
      C.insert(k, t, sl);
      inserted.emplace_back(k, t);
      slot[k][nb[k].at(khi(t), klo(t))] = sl;
    }
  // tables
  for (int k = 0; k < K; ++k) {
    StepPlan& sp = P.steps[k];
    const size_t nw = sp.win_ij.size() / 2;
    if (k >= 1) {
      sp.win_slots.resize(nw * r * r);
      const DBox& B = nb[k];
      for (size_t i = 0; i < nw; ++i)
        for (int m = 0; m < r; ++m)
          for (int n = 0; n < r; ++n) {
            const int32_t sl = slot[k][B.at(sp.win_ij[2 * i] + m, sp.win_ij[2 * i + 1] + n)];
            if (sl < 0) {
              *err = "internal: input tile missing from the plan";
              return false;
            }
            sp.win_slots[(i * r + m) * r + n] = sl;
          }
    }
    const auto& mt = missing[k + 1];
    sp.tiles.resize(4 * mt.size());
    sp.tile_wins.resize(mt.size() * r * r);
    const DBox& W = wb[k];
    for (size_t t = 0; t < mt.size(); ++t) {
      const int32_t ty = khi(mt[t]), tx = klo(mt[t]);
      sp.tiles[4 * t] = ty;
      sp.tiles[4 * t + 1] = tx;
      sp.tiles[4 * t + 2] = k >= 1 ? slot[k][nb[k].at(ty, tx)] : -1;
      sp.tiles[4 * t + 3] = slot[k + 1][nb[k + 1].at(ty, tx)];
      for (int m = 0; m < r; ++m)
        for (int n = 0; n < r; ++n) sp.tile_wins[(t * r + m) * r + n] = widx[k][W.at(ty - m, tx - n)];
    }
  }
  return true;
}

// Plan (and, unless dry, allocate cache slots for) the query of J_K over the
// tile rects.  With a persistent store, final-round tiles it holds count as
// available (read into cache slots instead of computed).  Returns false with
// a message on cache exhaustion.
bool plan_level(Level& L, const std::vector<RectT>& rects, bool dry, LevelPlan& P,
                std::string* err, TileStore* store = nullptr) {
  const int K = L.R, r = L.r;
  // compact requests (their bounding box at most 4x their area, grown by
  // the cone, a few million cells at most) take the dense form
  if (!rects.empty()) {
    int64_t y0 = rects[0].ty0, x0 = rects[0].tx0, y1 = rects[0].ty1, x1 = rects[0].tx1, area = 0;
    for (auto& R : rects) {
      y0 = std::min(y0, R.ty0); x0 = std::min(x0, R.tx0); y1 = std::max(y1, R.ty1); x1 = std::max(x1, R.tx1);
      area += (R.ty1 - R.ty0 + 1) * (R.tx1 - R.tx0 + 1);
    }
    const int64_t g = (int64_t)K * (r - 1);
    const double box = (double)(y1 - y0 + 1 + 2 * g) * (double)(x1 - x0 + 1 + 2 * g);
    if ((double)(y1 - y0 + 1) * (x1 - x0 + 1) <= 4.0 * area && box <= 6.4e7)
      return plan_level_dense(L, rects, dry, P, err, store);
  }
  TileCache& C = L.cache;
  P.steps.assign(K, StepPlan());
  std::vector<uint64_t> need;
  {
    std::unordered_set<uint64_t> s;
    for (auto& R : rects)
      for (int64_t ty = R.ty0; ty <= R.ty1; ++ty)
        for (int64_t tx = R.tx0; tx <= R.tx1; ++tx) s.insert(tkey((int32_t)ty, (int32_t)tx));
    need.assign(s.begin(), s.end());
  }
  std::vector<std::vector<uint64_t>> missing(K + 1);
  for (int k = K; k >= 1; --k) {
    std::sort(need.begin(), need.end(), [](uint64_t a, uint64_t b) {
      return khi(a) != khi(b) ? khi(a) < khi(b) : klo(a) < klo(b);
    });
    auto& mk = missing[k];
    for (uint64_t t : need) {
      auto it = C.map[k].find(t);
      if (it != C.map[k].end()) {
        if (!dry) {
          C.touch(it->second);
          C.hits++;
        }
      } else if (k == K && store && store_has(store, L.index, khi(t), klo(t))) {
        P.from_store.push_back(t);
      } else {
        mk.push_back(t);
      }
    }
    if (!dry) C.misses += (int64_t)mk.size();
    std::unordered_set<uint64_t> ws;
    for (uint64_t t : mk)
      for (int m = 0; m < r; ++m)
        for (int n = 0; n < r; ++n) ws.insert(tkey(khi(t) - m, klo(t) - n));
    std::vector<uint64_t> wins(ws.begin(), ws.end());
    std::sort(wins.begin(), wins.end(), [](uint64_t a, uint64_t b) {
      return khi(a) != khi(b) ? khi(a) < khi(b) : klo(a) < klo(b);
    });
    StepPlan& sp = P.steps[k - 1];
    sp.win_ij.resize(2 * wins.size());
    for (size_t i = 0; i < wins.size(); ++i) {
      sp.win_ij[2 * i] = khi(wins[i]);
      sp.win_ij[2 * i + 1] = klo(wins[i]);
      if (!P.any_windows) {
        P.wi_min = P.wi_max = khi(wins[i]);
        P.wj_min = P.wj_max = klo(wins[i]);
      }
      P.any_windows = true;
      P.wi_min = std::min<int64_t>(P.wi_min, khi(wins[i]));
      P.wi_max = std::max<int64_t>(P.wi_max, khi(wins[i]));
      P.wj_min = std::min<int64_t>(P.wj_min, klo(wins[i]));
      P.wj_max = std::max<int64_t>(P.wj_max, klo(wins[i]));
    }
    P.n_win_max = std::max(P.n_win_max, wins.size());
    if (k - 1 >= 1) {
      std::unordered_set<uint64_t> ns;
      for (uint64_t w : wins)
        for (int m = 0; m < r; ++m)
          for (int n = 0; n < r; ++n) ns.insert(tkey(khi(w) + m, klo(w) + n));
      need.assign(ns.begin(), ns.end());
    } else {
      need.clear();
    }
  }
  if (dry) return true;
  // allocate slots for the missing tiles, step by step; on exhaustion undo
  // every insertion of this plan so that no uncomputed tile stays visible
  std::vector<std::pair<int, uint64_t>> inserted;
  for (uint64_t t : P.from_store) missing[0].push_back(t);  // (slots first; J_0 is never cached)
  for (int k = 0; k <= K; ++k) {
    for (uint64_t t : missing[k]) {
      const int kk = k == 0 ? K : k;
      const int32_t sl = C.alloc();
      if (sl < 0) {
        for (auto& kt : inserted) {
          auto it = C.map[kt.first].find(kt.second);
          const int32_t os = it->second;
          C.map[kt.first].erase(it);
          C.unlink(os);
          C.free_list.push_back(os);
        }
        *err = "tile cache too small for this query's working set; raise cache_bytes";
        P.loads.clear();
        return false;
      }
      C.insert(kk, t, sl);
      inserted.emplace_back(kk, t);
      if (k == 0) P.loads.emplace_back(sl, t);
    }
  }
  missing[0].clear();
  // tables
  for (int k = 0; k < K; ++k) {
    StepPlan& sp = P.steps[k];
    const size_t nw = sp.win_ij.size() / 2;
    std::unordered_map<uint64_t, int32_t> widx;
    widx.reserve(nw * 2);
    for (size_t i = 0; i < nw; ++i) widx[tkey(sp.win_ij[2 * i], sp.win_ij[2 * i + 1])] = (int32_t)i;
    if (k >= 1) {
      sp.win_slots.resize(nw * r * r);
      for (size_t i = 0; i < nw; ++i)
        for (int m = 0; m < r; ++m)
          for (int n = 0; n < r; ++n) {
            auto it = C.map[k].find(tkey(sp.win_ij[2 * i] + m, sp.win_ij[2 * i + 1] + n));
            if (it == C.map[k].end()) {
              *err = "internal: input tile missing from the plan";
              return false;
            }
            sp.win_slots[(i * r + m) * r + n] = it->second;
          }
    }
    const auto& mt = missing[k + 1];
    sp.tiles.resize(4 * mt.size());
    sp.tile_wins.resize(mt.size() * r * r);
    for (size_t t = 0; t < mt.size(); ++t) {
      const int32_t ty = khi(mt[t]), tx = klo(mt[t]);
      int32_t sin = -1;
      if (k >= 1) {
        auto it = C.map[k].find(mt[t]);
        if (it == C.map[k].end()) {
          *err = "internal: J_k tile missing";
          return false;
        }
        sin = it->second;
      }
      sp.tiles[4 * t] = ty;
      sp.tiles[4 * t + 1] = tx;
      sp.tiles[4 * t + 2] = sin;
      sp.tiles[4 * t + 3] = C.map[k + 1][mt[t]];
      for (int m = 0; m < r; ++m)
        for (int n = 0; n < r; ++n) sp.tile_wins[(t * r + m) * r + n] = widx[tkey(ty - m, tx - n)];
    }
  }
  return true;
}

RectT tile_rect(const Level& L, int64_t x0, int64_t y0, int64_t w, int64_t h) {
  return RectT{fdiv(y0, L.s), fdiv(x0, L.s), fdiv(y0 + h - 1, L.s), fdiv(x0 + w - 1, L.s)};
}

// dense result of a level: the assembled J_K over a pixel rect
struct Dense {
  float* p = nullptr;
  int64_t x0 = 0, y0 = 0, pitch = 0;
  int w = 0, h = 0;
};

bool run_level(idf_world* W, Level& L, LevelPlan& P, const Dense* cond) {
  const int K = L.R, r = L.r, H = L.H, s = L.s;
  cudaStream_t st = W->st;
  // upload every table in one copy
  size_t total = 0;
  for (auto& sp : P.steps) {
    sp.off_win_ij = total; total += sp.win_ij.size();
    sp.off_win_slots = total; total += sp.win_slots.size();
    sp.off_tiles = total; total += sp.tiles.size();
    sp.off_tile_wins = total; total += sp.tile_wins.size();
  }
  if (total == 0) return true;
  if (!grow(W, &W->tab, &W->tab_cap, total, "scheduler tables")) return false;
  if (total > W->h_tab_cap) {
    // the previous copy from the staging buffer must be done before it is reused
    if (!cuda_ok(W, cudaStreamSynchronize(st), "sync")) return false;
    if (W->h_tab) cudaFreeHost(W->h_tab);
    W->h_tab = nullptr;
    W->h_tab_cap = 0;
    if (cudaMallocHost((void**)&W->h_tab, total * 4 * 3 / 2) != cudaSuccess) {
      cudaGetLastError();
      W->last_error = "cudaMallocHost staging failed";
      return false;
    }
    W->h_tab_cap = total * 3 / 2;
  } else {
    if (!cuda_ok(W, cudaStreamSynchronize(st), "sync")) return false;
  }
  for (auto& sp : P.steps) {
    memcpy(W->h_tab + sp.off_win_ij, sp.win_ij.data(), sp.win_ij.size() * 4);
    memcpy(W->h_tab + sp.off_win_slots, sp.win_slots.data(), sp.win_slots.size() * 4);
    memcpy(W->h_tab + sp.off_tiles, sp.tiles.data(), sp.tiles.size() * 4);
    memcpy(W->h_tab + sp.off_tile_wins, sp.tile_wins.data(), sp.tile_wins.size() * 4);
  }
  if (!cuda_ok(W, cudaMemcpyAsync(W->tab, W->h_tab, total * 4, cudaMemcpyHostToDevice, st), "upload tables"))
    return false;
  const int B = L.unet ? unet_max_batch(L.unet) : 4096;
  if (!grow(W, &W->F, &W->F_cap, P.n_win_max * (size_t)H * H, "window outputs")) return false;
  if (!grow(W, &W->x_in, &W->x_cap, (size_t)std::min<size_t>(B, P.n_win_max) * H * H * L.d.in_ch, "window inputs")) return false;
  bool multi = false;
  for (int m : L.rsteps) multi = multi || m > 1;
  if (multi && !grow(W, &W->xs, &W->xs_cap, (size_t)std::min<size_t>(B, P.n_win_max) * H * H, "window states"))
    return false;
  for (int k = 0; k < K; ++k) {
    StepPlan& sp = P.steps[k];
    const int nw = (int)(sp.win_ij.size() / 2);
    if (nw == 0) continue;
    // round k: sampler steps j0 .. jl, window-local between its blends
    const int j0 = L.rstart[k], m = L.rsteps[k], jl = j0 + m - 1;
    for (int b0 = 0; b0 < nw; b0 += B) {
      const int nb = std::min(B, nw - b0);
      GatherArgs g{};
      g.pool = L.cache.pool;
      g.win_slots = k >= 1 ? W->tab + sp.off_win_slots + (size_t)b0 * r * r : nullptr;
      g.win_ij = W->tab + sp.off_win_ij + 2 * (size_t)b0;
      g.n_win = nb;
      g.H = H; g.s = s; g.r = r; g.in_ch = L.d.in_ch;
      g.c_in = (float)L.c_in[j0];
      g.sigma0 = (float)L.sig[0];
      g.xs = m > 1 ? W->xs : nullptr;
      g.noise_step0 = k == 0;
      g.seed = W->seed;
      g.level = (uint32_t)L.index;
      if (cond) {
        g.cond = cond->p; g.cond_x0 = cond->x0; g.cond_y0 = cond->y0; g.cond_pitch = cond->pitch;
        g.cond_w = cond->w; g.cond_h = cond->h; g.cond_f = L.d.scale_to_parent;
      }
      g.x_in = W->x_in;
      g.err_flag = W->d_err;
      int pr = W->prof.begin(PK_GATHER, st, 0.0, (double)nb * H * H * 4 * (L.d.in_ch + (k ? 1 : 0)));
      launch_gather(g, st);
      W->prof.end(pr, st);
      W->launches++;
      float* Fb = W->F + (size_t)b0 * H * H;
      const float* bias = nullptr;
      const float* bias_g = nullptr;
      if (L.d.cond_dim > 0 && L.unet) {
        // each network embeds y_i with its own E
        const int c0 = L.d.channels[0];
        if (!grow(W, &W->bias, &W->bias_cap, (size_t)2 * nb * c0, "conditioning biases")) return false;
        launch_cond_bias(g.win_ij, nb, W->seed, (uint32_t)L.index, L.d_condz, (float)L.d.cond_amp, L.d_condE,
                         L.d.cond_dim, c0, W->bias, st);
        W->launches++;
        bias = W->bias;
        if (L.guide) {
          launch_cond_bias(g.win_ij, nb, W->seed, (uint32_t)L.index, L.d_condz, (float)L.d.cond_amp, L.d_condEg,
                           L.d.cond_dim, c0, W->bias + (size_t)nb * c0, st);
          W->launches++;
          bias_g = W->bias + (size_t)nb * c0;
        }
      }
      for (int i = 0; i < m; ++i) {
        const int j = j0 + i;
        if (L.d.test_denoiser) {
          pr = W->prof.begin(PK_DENOISE_TEST, st, 0.0, (double)nb * H * H * 4 * (L.d.in_ch + 1));
          launch_test_denoiser(L.d.test_denoiser, W->x_in, nb, H, L.d.in_ch, Fb, st);
          W->prof.end(pr, st);
          W->launches++;
        } else {
          Err e;
          const int64_t l0 = unet_launches(L.unet);
          if (!unet_forward(L.unet, W->x_in, nb, Fb, st, &e, bias)) {
            W->last_error = e.msg;
            W->poisoned = e.code == 3;
            return false;
          }
          W->launches += unet_launches(L.unet) - l0;
          if (L.guide) {
            // AutoGuidance: the guide network on the same inputs, then
            // F = F_guide + w (F_main - F_guide)
            if (!grow(W, &W->Fg, &W->Fg_cap, (size_t)nb * H * H, "guide outputs")) return false;
            const int64_t g0 = unet_launches(L.guide);
            if (!unet_forward(L.guide, W->x_in, nb, W->Fg, st, &e, bias_g)) {
              W->last_error = e.msg;
              W->poisoned = e.code == 3;
              return false;
            }
            W->launches += unet_launches(L.guide) - g0;
            launch_guidance(Fb, W->Fg, (int64_t)nb * H * H, L.w_guide, st);
            W->launches++;
          }
        }
        if (m > 1) {
          // window-local update; the round's last step leaves D in F
          WindowStepArgs ws{};
          ws.x_in = W->x_in;
          ws.xs = W->xs;
          ws.F = Fb;
          ws.win_ij = g.win_ij;
          ws.n_win = nb;
          ws.H = H; ws.s = s; ws.in_ch = L.d.in_ch;
          ws.c_skip = (float)L.c_skip[j];
          ws.c_out = (float)L.c_out[j];
          ws.last = i == m - 1;
          ws.c_in_next = ws.last ? 0.0f : (float)L.c_in[j + 1];
          ws.noise = !ws.last && j + 1 < L.K;
          ws.sigma_next = j + 1 < L.K ? (float)L.sig[j + 1] : 0.0f;
          ws.step_next = (uint32_t)(j + 1);
          ws.seed = W->seed;
          ws.level = (uint32_t)L.index;
          pr = W->prof.begin(PK_GATHER, st, 0.0, (double)nb * H * H * 4 * (ws.last ? 3 : 4 + L.d.in_ch));
          launch_window_step(ws, st);
          W->prof.end(pr, st);
          W->launches++;
        }
      }
    }
    L.windows_evaluated += (int64_t)nw * m;
    BlendArgs bl{};
    bl.pool = L.cache.pool;
    bl.pool_out = L.cache.pool;
    bl.tiles = W->tab + sp.off_tiles;
    bl.tile_wins = W->tab + sp.off_tile_wins;
    bl.F = W->F;
    bl.w1 = L.d_w1;
    bl.invB1 = L.d_invB1;
    bl.n_tiles = (int)(sp.tiles.size() / 4);
    bl.H = H; bl.s = s; bl.r = r;
    // one step: J = c_skip J_k + c_out (blended F) + noise; several steps:
    // F already holds each window's D, J = (blended D) + noise
    bl.c_skip = m == 1 ? (float)L.c_skip[j0] : 0.0f;
    bl.c_out = m == 1 ? (float)L.c_out[j0] : 1.0f;
    bl.c_in = (float)L.c_in[j0];
    bl.sigma0 = (float)L.sig[0];
    bl.noise_in = k == 0;
    bl.noise_next = jl + 1 < L.K;
    bl.sigma_next = jl + 1 < L.K ? (float)L.sig[jl + 1] : 0.0f;
    bl.step_next = (uint32_t)(jl + 1);
    bl.seed = W->seed;
    bl.level = (uint32_t)L.index;
    // algorithmic bytes per tile pixel: r^2 window outputs, J_k (unless it is
    // the noise) and J_{k+1}; the work field counts the normal samples drawn
    // (J_0 at the first step, the re-noise before every later one), whose
    // Philox + Box-Muller arithmetic, not memory, bounds this kernel
    const double normals = (double)bl.n_tiles * s * s * ((k == 0 ? 1 : 0) + (jl + 1 < L.K ? 1 : 0));
    const int pr = W->prof.begin(PK_BLEND, st, normals, (double)bl.n_tiles * s * s * 4.0 * (r * r + (k ? 2 : 1)));
    launch_blend(bl, st);
    W->prof.end(pr, st);
    W->launches++;
    L.tiles_computed += bl.n_tiles;
  }
  return cuda_ok(W, cudaGetLastError(), "sampler launch");
}

// Assemble J_K of level L over a pixel rect into out (pitch floats).
bool assemble(idf_world* W, Level& L, int64_t x0, int64_t y0, int w, int h, float* out,
              int64_t pitch) {
  const RectT R = tile_rect(L, x0, y0, w, h);
  const int nty = (int)(R.ty1 - R.ty0 + 1), ntx = (int)(R.tx1 - R.tx0 + 1);
  std::vector<int32_t> slots((size_t)nty * ntx);
  for (int a = 0; a < nty; ++a)
    for (int b = 0; b < ntx; ++b) {
      auto it = L.cache.map[L.R].find(tkey((int32_t)(R.ty0 + a), (int32_t)(R.tx0 + b)));
      if (it == L.cache.map[L.R].end()) {
        W->last_error = "internal: final tile missing";
        return false;
      }
      slots[(size_t)a * ntx + b] = it->second;
    }
  // tables live after the scheduler tables; use a dedicated small buffer
  int32_t* d_slots = nullptr;
  if (cudaMallocAsync((void**)&d_slots, slots.size() * 4, W->st) != cudaSuccess) {
    cudaGetLastError();
    W->last_error = "cudaMallocAsync assemble table failed";
    return false;
  }
  if (!cuda_ok(W, cudaMemcpyAsync(d_slots, slots.data(), slots.size() * 4, cudaMemcpyHostToDevice, W->st), "assemble upload"))
    return false;
  const int pr = W->prof.begin(PK_ASSEMBLE, W->st, 0.0, 8.0 * w * h);
  launch_assemble(L.cache.pool, d_slots, R.ty0, R.tx0, nty, ntx, L.s, y0, x0, h, w, out, pitch, W->st);
  W->prof.end(pr, W->st);
  W->launches++;
  // a pageable source is staged before cudaMemcpyAsync returns, so `slots`
  // may go out of scope now
  cudaFreeAsync(d_slots, W->st);
  return cuda_ok(W, cudaGetLastError(), "assemble");
}

// pinned staging of n floats for store transfers (waits for earlier copies)
bool store_staging(idf_world* W, size_t n) {
  if (!cuda_ok(W, cudaStreamSynchronize(W->st), "sync")) return false;
  if (n <= W->h_store_cap) return true;
  if (W->h_store) cudaFreeHost(W->h_store);
  W->h_store = nullptr;
  W->h_store_cap = 0;
  if (cudaMallocHost((void**)&W->h_store, n * 4) != cudaSuccess) {
    cudaGetLastError();
    W->last_error = "cudaMallocHost store staging failed";
    return false;
  }
  W->h_store_cap = n;
  return true;
}

// read the plan's stored final tiles into their cache slots
bool store_load(idf_world* W, Level& L, const LevelPlan& P) {
  if (P.loads.empty()) return true;
  const size_t ts = (size_t)L.s * L.s;
  if (!store_staging(W, P.loads.size() * ts)) return false;
  for (size_t i = 0; i < P.loads.size(); ++i) {
    const uint64_t t = P.loads[i].second;
    if (!store_read(W->store, L.index, khi(t), klo(t), W->h_store + i * ts)) {
      W->last_error = "tile store read failed";
      return false;
    }
    if (!cuda_ok(W, cudaMemcpyAsync(L.cache.pool + (size_t)P.loads[i].first * ts, W->h_store + i * ts, ts * 4,
                                    cudaMemcpyHostToDevice, W->st),
                 "store upload"))
      return false;
  }
  L.store_reads += (int64_t)P.loads.size();
  return true;
}

// write the final-round tiles this plan computed into the store
bool store_save(idf_world* W, Level& L, const LevelPlan& P) {
  if (P.steps.empty()) return true;
  const StepPlan& sp = P.steps[L.R - 1];
  const size_t nt = sp.tiles.size() / 4, ts = (size_t)L.s * L.s;
  if (nt == 0) return true;
  if (!store_staging(W, nt * ts)) return false;
  for (size_t t = 0; t < nt; ++t)
    if (!cuda_ok(W, cudaMemcpyAsync(W->h_store + t * ts, L.cache.pool + (size_t)sp.tiles[4 * t + 3] * ts, ts * 4,
                                    cudaMemcpyDeviceToHost, W->st),
                 "store download"))
      return false;
  if (!cuda_ok(W, cudaStreamSynchronize(W->st), "sync")) return false;
  for (size_t t = 0; t < nt; ++t)
    if (!store_write(W->store, L.index, sp.tiles[4 * t], sp.tiles[4 * t + 1], W->h_store + t * ts)) {
      W->last_error = "tile store write failed";
      return false;
    }
  L.store_writes += (int64_t)nt;
  return true;
}

// Decode halo: coarse rect of l^ read by the final upsampling, and the
// L / H rects the decode reads (see the decode kernels).
struct Halo {
  int64_t qx0, qy0, qw, qh;   // l^ rect
  int64_t Lx0, Ly0, Lw, Lh;   // L rect (coarse)
  int64_t Hx0, Hy0, Hw, Hh;   // H rect (fine)
};

Halo decode_halo(int f, int R, int64_t x0, int64_t y0, int64_t w, int64_t h) {
  Halo o;
  auto lo = [&](int64_t c) { return fdiv(2 * c + 1 - f, 2 * f); };
  o.qx0 = lo(x0);
  o.qy0 = lo(y0);
  o.qw = lo(x0 + w - 1) + 1 - o.qx0 + 1;
  o.qh = lo(y0 + h - 1) + 1 - o.qy0 + 1;
  o.Lx0 = o.qx0 - R - 1;
  o.Ly0 = o.qy0 - R - 1;
  o.Lw = o.qw + 2 * R + 2;
  o.Lh = o.qh + 2 * R + 2;
  o.Hx0 = (int64_t)f * (o.qx0 - R);
  o.Hy0 = (int64_t)f * (o.qy0 - R);
  o.Hw = (int64_t)f * (o.qw + 2 * R);
  o.Hh = (int64_t)f * (o.qh + 2 * R);
  return o;
}

std::vector<float> blur_taps(double sigma, int R) {
  std::vector<double> g(2 * R + 1);
  double s = 0;
  for (int k = -R; k <= R; ++k) {
    g[k + R] = exp(-(double)k * k / (2 * sigma * sigma));
    s += g[k + R];
  }
  std::vector<float> o(2 * R + 1);
  for (int i = 0; i < 2 * R + 1; ++i) o[i] = (float)(g[i] / s);
  return o;
}

bool valid_region(int64_t x0, int64_t y0, int64_t w, int64_t h) {
  if (w < 1 || h < 1) return false;
  if ((double)w * (double)h > 2147483648.0) return false;
  const int64_t lim = (int64_t)1 << 40;
  if (x0 < -lim || y0 < -lim || x0 + w > lim || y0 + h > lim) return false;
  return true;
}

bool tiles_fit(const Level& L, int64_t x0, int64_t y0, int64_t w, int64_t h) {
  const int64_t margin = (int64_t)(L.R + 2) * L.r + 2;
  auto fits = [&](int64_t v) { return v > INT32_MIN + margin && v < INT32_MAX - margin; };
  return fits(fdiv(x0, L.s)) && fits(fdiv(y0, L.s)) && fits(fdiv(x0 + w - 1, L.s)) &&
         fits(fdiv(y0 + h - 1, L.s));
}

struct Req {
  int64_t x0, y0;
  int w, h;
  float* out;
  int64_t pitch;
};

// Serve requests (all of one output kind) on the world's stream.
idf_status serve(idf_world* W, const std::vector<Req>& reqs, idf_output_kind kind) {
  if (W->poisoned) return fail(W, IDF_EINTERNAL, "world unusable after an earlier CUDA failure: " + W->last_error);
  for (const Level& L : W->lv)
    if (L.d.in_ch != (L.d.scale_to_parent > 0 ? 2 : 1))
      return fail(W, IDF_EMODEL, "a level with side-input channels runs only through idf_unet_forward");
  const int nl = (int)W->lv.size();
  if (kind == IDF_OUT_METRES && !W->stack.laplacian)
    return fail(W, IDF_EINVAL, "IDF_OUT_METRES needs a stack with laplacian = 1");
  for (auto& q : reqs) {
    if (!valid_region(q.x0, q.y0, q.w, q.h) || !q.out || q.pitch < q.w)
      return fail(W, IDF_EINVAL, "invalid region, output pointer or pitch");
  }
  for (auto& L : W->lv) { L.cache.epoch++; if (L.cache.epoch == 0) L.cache.epoch = 1; }
  Level& F = W->lv[nl - 1];
  const int f = W->stack.lap_factor, R = W->stack.lap_radius;
  // rect of the last level each request needs
  std::vector<Halo> halos(reqs.size());
  std::vector<RectT> frects;
  for (size_t i = 0; i < reqs.size(); ++i) {
    const Req& q = reqs[i];
    int64_t fx = q.x0, fy = q.y0, fw = q.w, fh = q.h;
    if (kind == IDF_OUT_METRES) {
      halos[i] = decode_halo(f, R, q.x0, q.y0, q.w, q.h);
      fx = halos[i].Hx0; fy = halos[i].Hy0; fw = halos[i].Hw; fh = halos[i].Hh;
    }
    if (!tiles_fit(F, fx, fy, fw, fh)) return fail(W, IDF_EINVAL, "region too far from the origin");
    frects.push_back(tile_rect(F, fx, fy, fw, fh));
  }
  std::string err;
  LevelPlan fp;
  if (!plan_level(F, frects, false, fp, &err, W->store)) return fail(W, IDF_ENOMEM, err);
  if (!store_load(W, F, fp)) return fail(W, W->poisoned ? IDF_ECUDA : IDF_EINTERNAL, W->last_error);
  LevelPlan cp;
  Dense cond;
  std::vector<Dense> lows(reqs.size());
  if (nl == 2) {
    Level& C = W->lv[0];
    const int fs = F.d.scale_to_parent;
    std::vector<RectT> crects;
    // conditioning: every window the fine plan evaluates
    int64_t cx0 = 0, cy0 = 0, cx1 = -1, cy1 = -1;
    if (fp.any_windows) {
      cy0 = fdiv(fp.wi_min * F.s, fs);
      cx0 = fdiv(fp.wj_min * F.s, fs);
      cy1 = fdiv(fp.wi_max * F.s + F.H - 1, fs);
      cx1 = fdiv(fp.wj_max * F.s + F.H - 1, fs);
      if (!tiles_fit(C, cx0, cy0, cx1 - cx0 + 1, cy1 - cy0 + 1))
        return fail(W, IDF_EINVAL, "region too far from the origin");
      crects.push_back(tile_rect(C, cx0, cy0, cx1 - cx0 + 1, cy1 - cy0 + 1));
    }
    if (kind == IDF_OUT_METRES)
      for (auto& hl : halos) crects.push_back(tile_rect(C, hl.Lx0, hl.Ly0, hl.Lw, hl.Lh));
    if (!crects.empty()) {
      if (!plan_level(C, crects, false, cp, &err, W->store)) return fail(W, IDF_ENOMEM, err);
      if (!store_load(W, C, cp)) return fail(W, W->poisoned ? IDF_ECUDA : IDF_EINTERNAL, W->last_error);
      if (!run_level(W, C, cp, nullptr)) return fail(W, W->poisoned ? IDF_ECUDA : IDF_ENOMEM, W->last_error);
    }
    // dense coarse results: one for the conditioning, one per decode
    size_t need = 0;
    if (fp.any_windows) need += (size_t)(cx1 - cx0 + 1) * (cy1 - cy0 + 1);
    if (kind == IDF_OUT_METRES)
      for (auto& hl : halos) need += (size_t)hl.Lw * hl.Lh;
    if (!grow(W, &W->dense, &W->dense_cap, need + 1, "dense coarse")) return fail(W, IDF_ENOMEM, W->last_error);
    size_t off = 0;
    if (fp.any_windows) {
      cond = Dense{W->dense, cx0, cy0, cx1 - cx0 + 1, (int)(cx1 - cx0 + 1), (int)(cy1 - cy0 + 1)};
      if (!assemble(W, C, cx0, cy0, cond.w, cond.h, cond.p, cond.pitch))
        return fail(W, W->poisoned ? IDF_ECUDA : IDF_EINTERNAL, W->last_error);
      off += (size_t)cond.w * cond.h;
    }
    if (kind == IDF_OUT_METRES)
      for (size_t i = 0; i < reqs.size(); ++i) {
        const Halo& hl = halos[i];
        lows[i] = Dense{W->dense + off, hl.Lx0, hl.Ly0, hl.Lw, (int)hl.Lw, (int)hl.Lh};
        if (!assemble(W, C, hl.Lx0, hl.Ly0, (int)hl.Lw, (int)hl.Lh, lows[i].p, lows[i].pitch))
          return fail(W, W->poisoned ? IDF_ECUDA : IDF_EINTERNAL, W->last_error);
        off += (size_t)hl.Lw * hl.Lh;
      }
  }
  if (nl == 1 && kind == IDF_OUT_METRES) {
    // given low band: read the periodic fixture over each decode's L rect
    size_t need = 0;
    for (auto& hl : halos) need += (size_t)hl.Lw * hl.Lh;
    if (!grow(W, &W->dense, &W->dense_cap, need + 1, "low band")) return fail(W, IDF_ENOMEM, W->last_error);
    size_t off = 0;
    for (size_t i = 0; i < reqs.size(); ++i) {
      const Halo& hl = halos[i];
      lows[i] = Dense{W->dense + off, hl.Lx0, hl.Ly0, hl.Lw, (int)hl.Lw, (int)hl.Lh};
      launch_fixture_gather(W->d_fixture, W->stack.fixture_period, hl.Lx0, hl.Ly0, (int)hl.Lw, (int)hl.Lh,
                            lows[i].p, W->st);
      W->launches++;
      off += (size_t)hl.Lw * hl.Lh;
    }
  }
  if (!run_level(W, F, fp, nl == 2 && fp.any_windows ? &cond : nullptr))
    return fail(W, W->poisoned ? IDF_ECUDA : IDF_ENOMEM, W->last_error);
  for (size_t i = 0; i < reqs.size(); ++i) {
    const Req& q = reqs[i];
    if (kind == IDF_OUT_MODEL) {
      if (!assemble(W, F, q.x0, q.y0, q.w, q.h, q.out, q.pitch))
        return fail(W, W->poisoned ? IDF_ECUDA : IDF_EINTERNAL, W->last_error);
      continue;
    }
    const Halo& hl = halos[i];
    const size_t nH = (size_t)hl.Hw * hl.Hh;
    const size_t nD = (size_t)(hl.qw + 2 * R) * (hl.qh + 2 * R);
    const size_t nT = (size_t)hl.qw * (hl.qh + 2 * R);
    const size_t nQ = (size_t)hl.qw * hl.qh;
    if (!grow(W, &W->dec, &W->dec_cap, nH + nD + nT + nQ, "decode scratch")) return fail(W, IDF_ENOMEM, W->last_error);
    float* Hd = W->dec;
    if (!assemble(W, F, hl.Hx0, hl.Hy0, (int)hl.Hw, (int)hl.Hh, Hd, hl.Hw))
      return fail(W, W->poisoned ? IDF_ECUDA : IDF_EINTERNAL, W->last_error);
    DecodeArgs a{};
    a.L = lows[i].p; a.lx0 = lows[i].x0; a.ly0 = lows[i].y0; a.lpitch = lows[i].pitch; a.lw = lows[i].w; a.lh = lows[i].h;
    a.H = Hd; a.hx0 = hl.Hx0; a.hy0 = hl.Hy0; a.hpitch = hl.Hw; a.hw = (int)hl.Hw; a.hh = (int)hl.Hh;
    a.x0 = q.x0; a.y0 = q.y0; a.w = q.w; a.h = q.h; a.out = q.out; a.pitch = q.pitch;
    a.f = f; a.R = R;
    a.low_mu = (float)W->stack.low_mu; a.low_scale = (float)W->stack.low_scale; a.res_scale = (float)W->stack.res_scale;
    a.taps = W->d_taps;
    a.D = Hd + nH; a.T = a.D + nD; a.Lhat = a.T + nT;
    a.qx0 = hl.qx0; a.qy0 = hl.qy0; a.qw = (int)hl.qw; a.qh = (int)hl.qh;
    // algorithmic bytes: H read over the halo rect and the query, the low band,
    // the metres written, the coarse scratch (D, its blur passes) read and written
    const double dby = 4.0 * ((double)nH + (double)q.w * q.h * 2 + (double)hl.Lw * hl.Lh + 2.0 * (nD + nT + nQ));
    const int pr = W->prof.begin(PK_DECODE, W->st, 0.0, dby);
    launch_decode(a, W->st);
    W->prof.end(pr, W->st);
    W->launches += 4;
  }
  if (!cuda_ok(W, cudaGetLastError(), "decode launch")) return fail(W, IDF_ECUDA, W->last_error);
  if (W->store && W->store_writable) {
    if (nl == 2 && !store_save(W, W->lv[0], cp)) return fail(W, W->poisoned ? IDF_ECUDA : IDF_EINTERNAL, W->last_error);
    if (!store_save(W, F, fp)) return fail(W, W->poisoned ? IDF_ECUDA : IDF_EINTERNAL, W->last_error);
  }
  W->queries += (int64_t)reqs.size();
  return IDF_OK;
}

// Read the device status words after a synchronize: bounds checks of the
// gather, and bounded waits of the tensor-core kernels that ran out.
idf_status check_err_flag(idf_world* W) {
  for (auto& L : W->lv) {
    if (!L.unet) continue;
    int t = 0;
    if (!cuda_ok(W, cudaMemcpy(&t, unet_status(L.unet), sizeof(int), cudaMemcpyDeviceToHost), "read status"))
      return IDF_ECUDA;
    if (t) return fail(W, IDF_ETIMEOUT, "a bounded device-side wait in the tensor-core convolution ran out");
  }
  int h = 0;
  if (!cuda_ok(W, cudaMemcpy(&h, W->d_err, sizeof(int), cudaMemcpyDeviceToHost), "read status"))
    return IDF_ECUDA;
  if (h) {
    cudaMemset(W->d_err, 0, sizeof(int));
    return fail(W, IDF_EDEVICE_CHECK, "a device-side bounds check fired (conditioning read)");
  }
  return IDF_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void idf_world_destroy(idf_world* W);

idf_status idf_model_param_count(const idf_level_desc* level, int32_t* n_tensors, size_t* n_weights) {
  if (!level || !n_tensors || !n_weights) return IDF_EINVAL;
  if (level->test_denoiser) {
    *n_tensors = 0;
    *n_weights = 0;
    return IDF_OK;
  }
  if (level->levels < 1 || level->levels > 6 || !level->channels) return IDF_EINVAL;
  auto sh = unet_param_shapes(unet_desc(*level));
  size_t n = 0;
  for (auto& s : sh) n += (size_t)s[0] * s[1] * s[2] * s[3];
  *n_tensors = (int32_t)sh.size();
  *n_weights = n;
  return IDF_OK;
}

idf_status idf_model_param_shape(const idf_level_desc* level, int32_t index, int32_t shape[4]) {
  if (!level || !shape || level->levels < 1 || level->levels > 6 || !level->channels) return IDF_EINVAL;
  auto sh = unet_param_shapes(unet_desc(*level));
  if (index < 0 || index >= (int32_t)sh.size()) return IDF_EINVAL;
  for (int i = 0; i < 4; ++i) shape[i] = sh[index][i];
  return IDF_OK;
}

idf_status idf_world_create(uint64_t seed, const idf_model_stack* stack, const idf_world_opts* opts,
                            idf_world** out) {
  if (!out) return IDF_EINVAL;
  *out = nullptr;
  if (!stack || !opts || stack->n_levels < 1 || stack->n_levels > 2 || !stack->level) return IDF_EINVAL;
  if (opts->precision != IDF_FP8_E4M3 && opts->precision != IDF_FP32 && opts->precision != IDF_BF16 && opts->precision != IDF_BF16X3 &&
      opts->precision != IDF_TF32)
    return IDF_EINVAL;
  if (!(stack->blend_eps > 0) || !(stack->blend_eps <= 1)) return IDF_EINVAL;
  if (stack->laplacian) {
    // two levels (L then H), or one level (H) with a given low band
    const bool fixture = stack->n_levels == 1 && stack->low_band_fixture && stack->fixture_period >= 1 &&
                         stack->fixture_period <= (1 << 15) && stack->level[0].in_ch == 1;
    if ((stack->n_levels != 2 && !fixture) || (stack->n_levels == 2 && stack->low_band_fixture) ||
        stack->lap_factor < 2 || stack->lap_factor % 2 || stack->lap_radius < 0 || stack->lap_radius > 64 ||
        !(stack->lap_blur_sigma > 0))
      return IDF_EINVAL;
  } else if (stack->low_band_fixture) {
    return IDF_EINVAL;
  }
  std::unique_ptr<idf_world> W(new (std::nothrow) idf_world());
  if (!W) return IDF_ENOMEM;
  W->seed = seed;
  W->stack = *stack;
  W->stack.level = nullptr;
  W->stack.low_band_fixture = nullptr;  // copied to W->d_fixture below
  W->opts = *opts;
  for (int i = 0; i < stack->n_levels; ++i) {
    const idf_level_desc& d = stack->level[i];
    std::string m = check_level(d, i);
    if (!m.empty()) return IDF_EINVAL;
    if (i == 1 && stack->n_levels == 2 && d.scale_to_parent <= 0 && stack->laplacian) return IDF_EINVAL;
    // FP8 E4M3 contractions exist for the 16-channel networks only
    if (opts->precision == IDF_FP8_E4M3 && d.test_denoiser == 0 && !small_net_eligible(unet_desc(d)))
      return IDF_EUNSUPPORTED;
  }
  if (cudaSetDevice(opts->device) != cudaSuccess) {
    cudaGetLastError();
    return IDF_ECUDA;
  }
  auto bail = [&](idf_status code) {
    cudaGetLastError();
    idf_world_destroy(W.release());
    return code;
  };
  if (cudaStreamCreateWithFlags(&W->st, cudaStreamNonBlocking) != cudaSuccess) return bail(IDF_ECUDA);
  if (cudaEventCreateWithFlags(&W->ev_join, cudaEventDisableTiming) != cudaSuccess) return bail(IDF_ECUDA);
  if (cudaMalloc(&W->d_err, sizeof(int)) != cudaSuccess || cudaMemset(W->d_err, 0, sizeof(int)) != cudaSuccess)
    return bail(IDF_ECUDA);
  const size_t cache_bytes = opts->cache_bytes ? opts->cache_bytes : ((size_t)8 << 30);
  // default arena: 128 GiB, or 45% of the device's free memory if that is
  // less (larger window batches amortise the per-launch ramp of the
  // persistent convolutions; results do not depend on the batch)
  size_t ws_bytes = opts->workspace_bytes;
  if (!ws_bytes) {
    size_t fr = 0, tot = 0;
    ws_bytes = (size_t)64 << 30;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) ws_bytes = std::min((size_t)128 << 30, fr / 100 * 45);
  }
  // one activation arena shared by the levels' UNets (they never run at the
  // same time): each level batches as many windows as the arena holds
  size_t arena_need = 0;
  std::vector<int> batches(stack->n_levels, 0);
  for (int i = 0; i < stack->n_levels; ++i) {
    const idf_level_desc& d = stack->level[i];
    if (d.test_denoiser) continue;
    UNetDesc ud = unet_desc(d);
    const size_t per = unet_arena_bytes(ud, opts->precision, 1) + 256 * 11 * d.levels;
    int mb = opts->max_batch > 0 ? opts->max_batch : (int)std::max<size_t>(1, ws_bytes / per);
    mb = std::min(mb, 4096);
    batches[i] = mb;
    arena_need = std::max(arena_need, unet_arena_bytes(ud, opts->precision, mb));
  }
  // world identity for the persistent tile store: FNV-1a over the seed, the
  // precision, the stack and level descriptions and the weights
  {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
      const uint8_t* b = (const uint8_t*)p;
      for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    };
    mix(&seed, sizeof seed);
    mix(&opts->precision, sizeof opts->precision);
    const double sd[7] = {stack->lap_blur_sigma, stack->low_mu, stack->low_scale, stack->res_scale, stack->blend_eps,
                          (double)stack->lap_factor, (double)stack->lap_radius};
    mix(sd, sizeof sd);
    mix(&stack->laplacian, sizeof stack->laplacian);
    if (stack->low_band_fixture)
      mix(stack->low_band_fixture, (size_t)stack->fixture_period * stack->fixture_period * sizeof(float));
    for (int i = 0; i < stack->n_levels; ++i) {
      const idf_level_desc& d = stack->level[i];
      const int32_t iv[13] = {d.levels, d.in_ch, d.out_ch, d.gn_groups, d.attn_at_bottom, d.attn_heads,
                              d.window, d.stride, d.offset, d.steps, d.scale_to_parent, d.test_denoiser,
                              d.n_rounds};
      mix(iv, sizeof iv);
      if (d.channels && d.test_denoiser == 0) mix(d.channels, (size_t)d.levels * sizeof(int32_t));
      if (d.round_steps && d.n_rounds > 0) mix(d.round_steps, (size_t)d.n_rounds * sizeof(int32_t));
      const double dv[4] = {d.sigma_max, d.sigma_min, d.rho, d.sigma_data};
      mix(dv, sizeof dv);
      if (d.weights && d.test_denoiser == 0) mix(d.weights, d.n_weights * sizeof(float));
      mix(&d.cond_dim, sizeof d.cond_dim);
      if (d.cond_dim > 0 && d.cond_z) mix(d.cond_z, (size_t)d.cond_dim * sizeof(float));
      const double cv[2] = {d.cond_amp, d.guidance};
      mix(cv, sizeof cv);
      if (d.guidance != 0.0 && d.guide_weights) mix(d.guide_weights, d.n_guide_weights * sizeof(float));
    }
    W->identity = h;
  }
  W->prof.on = opts->profile != 0;
  W->lv.resize(stack->n_levels);
  for (int i = 0; i < stack->n_levels; ++i) {
    Level& L = W->lv[i];
    L.d = stack->level[i];
    if (L.d.test_denoiser == 0) {
      L.ch.assign(L.d.channels, L.d.channels + L.d.levels);
      L.d.channels = L.ch.data();
    }
    L.d.weights = nullptr;
    L.d.cond_z = nullptr;
    L.d.guide_weights = nullptr;
    L.index = i;
    L.H = L.d.window;
    L.s = L.d.stride;
    L.r = L.d.window / L.d.stride;
    L.K = L.d.steps;
    if (L.d.n_rounds > 0) {
      L.rsteps.assign(L.d.round_steps, L.d.round_steps + L.d.n_rounds);
    } else {
      L.rsteps.assign(L.K, 1);
    }
    L.R = (int)L.rsteps.size();
    L.rstart.resize(L.R);
    for (int k = 0, j = 0; k < L.R; j += L.rsteps[k], ++k) L.rstart[k] = j;
    L.rsteps_copy.assign(L.rsteps.begin(), L.rsteps.end());
    L.d.round_steps = L.rsteps_copy.data();
    schedule(L);
    // blend tables: w1(u) = 1 - (1-eps) |u - c| / c, c = (H-1)/2; B1(a) = sum_m w1(a + m s)
    std::vector<float> w1(L.H), ib(L.s);
    std::vector<double> w1d(L.H);
    const double c = (L.H - 1) / 2.0;
    for (int u = 0; u < L.H; ++u) {
      w1d[u] = 1.0 - (1.0 - stack->blend_eps) * fabs(u - c) / c;
      w1[u] = (float)w1d[u];
    }
    for (int a = 0; a < L.s; ++a) {
      double b = 0;
      for (int m = 0; m < L.r; ++m) b += w1d[a + m * L.s];
      ib[a] = (float)(1.0 / b);
    }
    if (cudaMalloc(&L.d_w1, L.H * 4) != cudaSuccess || cudaMalloc(&L.d_invB1, L.s * 4) != cudaSuccess)
      return bail(IDF_ENOMEM);
    cudaMemcpy(L.d_w1, w1.data(), L.H * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(L.d_invB1, ib.data(), L.s * 4, cudaMemcpyHostToDevice);
    // cache
    TileCache& C = L.cache;
    C.s = L.s;
    C.n_slots = (int64_t)(cache_bytes / stack->n_levels / ((size_t)L.s * L.s * 4));
    if (C.n_slots < 1 || C.n_slots > INT32_MAX) return bail(IDF_EINVAL);
    if (cudaMalloc(&C.pool, (size_t)C.n_slots * L.s * L.s * 4) != cudaSuccess) {
      return bail(IDF_ENOMEM);
    }
    C.map.resize(L.R + 1);
    C.slot_step.assign(C.n_slots, 0);
    C.slot_key.assign(C.n_slots, 0);
    C.prv.assign(C.n_slots, -1);
    C.nxt.assign(C.n_slots, -1);
    C.pin.assign(C.n_slots, 0);
    C.clear();
    if (L.d.test_denoiser == 0) {
      int32_t nt;
      size_t nw;
      idf_model_param_count(&stack->level[i], &nt, &nw);
      if (!stack->level[i].weights || stack->level[i].n_weights != nw) {
        return bail(IDF_EMODEL);
      }
      UNetDesc ud = unet_desc(L.d);
      if (!W->arena && arena_need) {
        if (cudaMalloc(&W->arena, arena_need) != cudaSuccess) return bail(IDF_ENOMEM);
        W->arena_bytes = arena_need;
      }
      Err e;
      L.unet = unet_create(ud, stack->level[i].weights, opts->precision, batches[i], &e, W->arena, W->arena_bytes);
      if (!L.unet) {
        return bail(e.code == 2 ? IDF_ENOMEM : IDF_ECUDA);
      }
      unet_set_prof(L.unet, &W->prof);
      unet_set_options(L.unet, opts->groupnorm_in_conv != 0, (long long)opts->device_wait_budget_cycles,
                       opts->autotune != 0, opts->cuda_graphs != 0,
                       opts->cta_pairs != 0);
      const idf_level_desc& dsrc = stack->level[i];
      if (dsrc.cond_dim > 0) {
        // the embedding E is the last (channels[0], cond_dim, 1, 1) tensor
        const size_t ne = (size_t)L.d.channels[0] * dsrc.cond_dim;
        L.condz.assign(dsrc.cond_z, dsrc.cond_z + dsrc.cond_dim);
        if (cudaMalloc(&L.d_condE, ne * 4) != cudaSuccess || cudaMalloc(&L.d_condz, dsrc.cond_dim * 4) != cudaSuccess ||
            cudaMemcpy(L.d_condE, dsrc.weights + nw - ne, ne * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(L.d_condz, L.condz.data(), dsrc.cond_dim * 4, cudaMemcpyHostToDevice) != cudaSuccess)
          return bail(IDF_ENOMEM);
      }
      if (dsrc.guidance != 0.0) {
        if (!dsrc.guide_weights || dsrc.n_guide_weights != nw) return bail(IDF_EMODEL);
        if (dsrc.cond_dim > 0) {
          const size_t ne = (size_t)L.d.channels[0] * dsrc.cond_dim;
          if (cudaMalloc(&L.d_condEg, ne * 4) != cudaSuccess ||
              cudaMemcpy(L.d_condEg, dsrc.guide_weights + nw - ne, ne * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(IDF_ENOMEM);
        }
        L.guide = unet_create(ud, dsrc.guide_weights, opts->precision, batches[i], &e, W->arena, W->arena_bytes);
        if (!L.guide) return bail(e.code == 2 ? IDF_ENOMEM : IDF_ECUDA);
        unet_set_prof(L.guide, &W->prof);
        unet_set_options(L.guide, opts->groupnorm_in_conv != 0, (long long)opts->device_wait_budget_cycles,
                         opts->autotune != 0, opts->cuda_graphs != 0,
                       opts->cta_pairs != 0);
        L.w_guide = (float)dsrc.guidance;
      }
    }
  }
  if (stack->laplacian) {
    auto taps = blur_taps(stack->lap_blur_sigma, stack->lap_radius);
    if (cudaMalloc(&W->d_taps, taps.size() * 4) != cudaSuccess) return bail(IDF_ENOMEM);
    cudaMemcpy(W->d_taps, taps.data(), taps.size() * 4, cudaMemcpyHostToDevice);
    if (stack->low_band_fixture) {
      const size_t nf = (size_t)stack->fixture_period * stack->fixture_period;
      if (cudaMalloc(&W->d_fixture, nf * 4) != cudaSuccess) return bail(IDF_ENOMEM);
      if (cudaMemcpy(W->d_fixture, stack->low_band_fixture, nf * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(IDF_ECUDA);
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(IDF_ECUDA);
  *out = W.release();
  return IDF_OK;
}

void idf_world_destroy(idf_world* W) {
  if (!W) return;
  if (W->st) cudaStreamSynchronize(W->st);
  for (auto& L : W->lv) {
    unet_destroy(L.unet);
    unet_destroy(L.guide);
    cudaFree(L.d_condE);
    cudaFree(L.d_condEg);
    cudaFree(L.d_condz);
    cudaFree(L.d_w1);
    cudaFree(L.d_invB1);
    cudaFree(L.cache.pool);
  }
  cudaFree(W->F); cudaFree(W->x_in); cudaFree(W->xs); cudaFree(W->bias); cudaFree(W->Fg); cudaFree(W->tab); cudaFree(W->dense); cudaFree(W->dec);
  cudaFree(W->outbuf); cudaFree(W->d_taps); cudaFree(W->d_fixture); cudaFree(W->d_err); cudaFree(W->arena);
  if (W->h_tab) cudaFreeHost(W->h_tab);
  if (W->h_store) cudaFreeHost(W->h_store);
  store_close(W->store);
  if (W->ev_join) cudaEventDestroy(W->ev_join);
  if (W->st) cudaStreamDestroy(W->st);
  delete W;
}

const char* idf_world_last_error(const idf_world* W) { return W ? W->last_error.c_str() : "null world"; }

static idf_status join_in(idf_world* W, cudaStream_t user) {
  if (!cuda_ok(W, cudaEventRecord(W->ev_join, user), "event record") ||
      !cuda_ok(W, cudaStreamWaitEvent(W->st, W->ev_join, 0), "stream wait"))
    return IDF_ECUDA;
  return IDF_OK;
}
static idf_status join_out(idf_world* W, cudaStream_t user) {
  if (!cuda_ok(W, cudaEventRecord(W->ev_join, W->st), "event record") ||
      !cuda_ok(W, cudaStreamWaitEvent(user, W->ev_join, 0), "stream wait"))
    return IDF_ECUDA;
  return IDF_OK;
}

idf_status idf_world_query_device(idf_world* W, int64_t x0, int64_t y0, int32_t w, int32_t h,
                                  idf_output_kind kind, float* out_dev, int64_t pitch, void* stream) {
  if (!W) return IDF_EINVAL;
  if (kind != IDF_OUT_MODEL && kind != IDF_OUT_METRES) return fail(W, IDF_EINVAL, "unknown output kind");
  cudaStream_t user = (cudaStream_t)stream;
  if (join_in(W, user) != IDF_OK) return IDF_ECUDA;
  std::vector<Req> r{Req{x0, y0, w, h, out_dev, pitch}};
  idf_status s = serve(W, r, kind);
  if (s != IDF_OK) return s;
  return join_out(W, user);
}

idf_status idf_world_query(idf_world* W, int64_t x0, int64_t y0, int32_t w, int32_t h,
                           idf_output_kind kind, float* out_host) {
  if (!W) return IDF_EINVAL;
  if (!out_host) return fail(W, IDF_EINVAL, "null output");
  if (kind != IDF_OUT_MODEL && kind != IDF_OUT_METRES) return fail(W, IDF_EINVAL, "unknown output kind");
  if (!valid_region(x0, y0, w, h)) return fail(W, IDF_EINVAL, "invalid region");
  if (!grow(W, &W->outbuf, &W->out_cap, (size_t)w * h, "output")) return fail(W, IDF_ENOMEM, W->last_error);
  std::vector<Req> r{Req{x0, y0, w, h, W->outbuf, (int64_t)w}};
  idf_status s = serve(W, r, kind);
  if (s != IDF_OK) return s;
  if (!cuda_ok(W, cudaMemcpyAsync(out_host, W->outbuf, (size_t)w * h * 4, cudaMemcpyDeviceToHost, W->st), "copy out") ||
      !cuda_ok(W, cudaStreamSynchronize(W->st), "query"))
    return fail(W, IDF_ECUDA, W->last_error);
  return check_err_flag(W);
}

idf_status idf_world_query_batch(idf_world* W, const idf_region* regions, int32_t n,
                                 idf_output_kind kind, void* stream) {
  if (!W) return IDF_EINVAL;
  if (n < 0 || (n > 0 && !regions)) return fail(W, IDF_EINVAL, "bad region list");
  if (kind != IDF_OUT_MODEL && kind != IDF_OUT_METRES) return fail(W, IDF_EINVAL, "unknown output kind");
  if (n == 0) return IDF_OK;
  cudaStream_t user = (cudaStream_t)stream;
  if (join_in(W, user) != IDF_OK) return IDF_ECUDA;
  std::vector<Req> r;
  for (int i = 0; i < n; ++i)
    r.push_back(Req{regions[i].x0, regions[i].y0, regions[i].w, regions[i].h, regions[i].out_dev,
                    regions[i].pitch_elems});
  idf_status s = serve(W, r, kind);
  if (s != IDF_OK) return s;
  return join_out(W, user);
}

idf_status idf_world_cache_clear(idf_world* W) {
  if (!W) return IDF_EINVAL;
  if (!cuda_ok(W, cudaStreamSynchronize(W->st), "sync")) return IDF_ECUDA;
  for (auto& L : W->lv) L.cache.clear();
  return IDF_OK;
}

idf_status idf_world_stats(const idf_world* Wc, char* buf, size_t len) {
  if (!Wc || !buf || len == 0) return IDF_EINVAL;
  idf_world* W = const_cast<idf_world*>(Wc);
  if (cudaStreamSynchronize(W->st) != cudaSuccess) return fail(W, IDF_ECUDA, "sync in stats");
  W->prof.resolve();
  std::string s = "{\"levels\": [";
  for (size_t i = 0; i < W->lv.size(); ++i) {
    const Level& L = W->lv[i];
    char b[512];
    size_t used = 0;
    for (auto& m : L.cache.map) used += m.size();
    snprintf(b, sizeof b,
             "%s{\"windows_evaluated\": %lld, \"tiles_computed\": %lld, \"cache_hits\": %lld, "
             "\"cache_misses\": %lld, \"evictions\": %lld, \"tiles_cached\": %zu, \"slots\": %lld, "
             "\"unet_batch\": %d, \"store_reads\": %lld, \"store_writes\": %lld}",
             i ? ", " : "", (long long)L.windows_evaluated, (long long)L.tiles_computed,
             (long long)L.cache.hits, (long long)L.cache.misses, (long long)L.cache.evictions, used,
             (long long)L.cache.n_slots, L.unet ? unet_max_batch(L.unet) : 0, (long long)L.store_reads,
             (long long)L.store_writes);
    s += b;
  }
  int tuned = 0, changed = 0;
  for (const Level& L : W->lv) {
    int t = 0, c = 0;
    unet_autotune_stats(L.unet, &t, &c);
    tuned += t;
    changed += c;
  }
  int64_t gcap = 0, grep = 0, gker = 0;
  for (const Level& L : W->lv)
    for (const UNet* u : {L.unet, L.guide}) {
      int64_t a = 0, r = 0, k = 0;
      unet_graph_stats(u, &a, &r, &k);
      gcap += a;
      grep += r;
      gker += k;
    }
  char b[512];
  // host launch calls: every kernel launched eagerly, plus one per graph replay
  snprintf(b, sizeof b,
           "], \"kernel_launches\": %lld, \"queries\": %lld, \"autotune\": {\"tuned\": %d, \"changed\": %d}, "
           "\"graphs\": {\"captured\": %lld, \"replays\": %lld, \"replayed_kernels\": %lld, "
           "\"host_launch_calls\": %lld}",
           (long long)W->launches, (long long)W->queries, tuned, changed, (long long)gcap, (long long)grep,
           (long long)gker, (long long)(W->launches - gker + grep));
  s += b;
  // the device status words as they stand (read, not cleared): a bounded
  // wait of a level's tensor-core kernels that ran out, a bounds check that
  // fired.  Calls that synchronize (queries) fail on them; an asynchronous
  // idf_unet_forward leaves them here.
  {
    int waits = 0, checks = 0;
    for (const Level& L : W->lv)
      for (const UNet* u : {L.unet, L.guide}) {
        int t = 0;
        if (u && cudaMemcpy(&t, unet_status(u), sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && t) ++waits;
      }
    if (W->d_err) cudaMemcpy(&checks, W->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    char d[128];
    snprintf(d, sizeof d, ", \"device_status\": {\"waits_expired\": %d, \"bounds_check\": %d}, "
             "\"cta_pair_clusters\": %d", waits, checks ? 1 : 0, conv_tc_pair_clusters());
    s += d;
  }
  static const char* names[PK_COUNT] = {"conv_tc", "conv_simt", "groupnorm", "attention", "resample",
                                        "gather", "test_denoiser", "blend", "assemble", "decode"};
  s += ", \"profile\": {";
  for (int k = 0; k < PK_COUNT; ++k) {
    char e[256];
    snprintf(e, sizeof e, "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"flops\": %.6e, \"bytes\": %.6e}",
             k ? ", " : "", names[k], (long long)W->prof.launches[k], W->prof.ms[k], W->prof.flops[k],
             W->prof.bytes[k]);
    s += e;
  }
  s += "}, \"conv_tc_shapes\": [";
  {
    bool first = true;
    for (const auto& kv : W->prof.conv_shapes) {
      char e[160];
      snprintf(e, sizeof e, "%s[%.6e, %.6e, %lld, %.6f]", first ? "" : ", ", kv.first.first, kv.first.second,
               (long long)kv.second.first, kv.second.second);
      s += e;
      first = false;
    }
  }
  s += "]}";
  if (s.size() + 1 > len) return IDF_EINVAL;
  memcpy(buf, s.c_str(), s.size() + 1);
  return IDF_OK;
}

idf_status idf_debug_cone(idf_world* W, int64_t x0, int64_t y0, int32_t w, int32_t h, int32_t level,
                          int32_t step, int64_t* win_ij, int32_t cap, int32_t* n_out) {
  if (!W || !n_out) return IDF_EINVAL;
  if (level < 0 || level >= (int)W->lv.size()) return fail(W, IDF_EINVAL, "bad level");
  Level& L = W->lv[level];
  if (step < 0 || step >= L.R) return fail(W, IDF_EINVAL, "bad step");
  if (!valid_region(x0, y0, w, h) || !tiles_fit(L, x0, y0, w, h)) return fail(W, IDF_EINVAL, "invalid region");
  LevelPlan P;
  std::string err;
  std::vector<RectT> rs{tile_rect(L, x0, y0, w, h)};
  plan_level(L, rs, true, P, &err, W->store);
  const auto& wi = P.steps[step].win_ij;
  const int32_t n = (int32_t)(wi.size() / 2);
  *n_out = n;
  if (win_ij)
    for (int32_t i = 0; i < std::min(n, cap); ++i) {
      win_ij[2 * i] = wi[2 * i];
      win_ij[2 * i + 1] = wi[2 * i + 1];
    }
  return IDF_OK;
}

idf_status idf_world_store_open(idf_world* W, const char* dir, int32_t writable) {
  if (!W || !dir || !dir[0]) return IDF_EINVAL;
  if (W->store) return fail(W, IDF_EINVAL, "a tile store is already open on this world");
  std::vector<int> side;
  for (auto& L : W->lv) side.push_back(L.s);
  std::string err;
  TileStore* s = store_open(dir, W->identity, side, writable != 0, &err);
  if (!s) return fail(W, IDF_EINVAL, err);
  W->store = s;
  W->store_writable = writable != 0;
  return IDF_OK;
}

idf_status idf_world_store_close(idf_world* W) {
  if (!W) return IDF_EINVAL;
  if (!cuda_ok(W, cudaStreamSynchronize(W->st), "sync")) return IDF_ECUDA;
  store_close(W->store);
  W->store = nullptr;
  W->store_writable = false;
  return IDF_OK;
}

idf_status idf_debug_cache_keys(idf_world* W, int32_t level, int32_t step, int32_t* ty_tx, int32_t cap,
                                int32_t* n_out) {
  if (!W || !n_out) return IDF_EINVAL;
  if (level < 0 || level >= (int)W->lv.size()) return fail(W, IDF_EINVAL, "bad level");
  Level& L = W->lv[level];
  if (step < 1 || step > L.R) return fail(W, IDF_EINVAL, "bad step");
  std::vector<uint64_t> keys;
  keys.reserve(L.cache.map[step].size());
  for (auto& kv : L.cache.map[step]) keys.push_back(kv.first);
  std::sort(keys.begin(), keys.end(), [](uint64_t a, uint64_t b) {
    return khi(a) != khi(b) ? khi(a) < khi(b) : klo(a) < klo(b);
  });
  *n_out = (int32_t)keys.size();
  if (ty_tx)
    for (int32_t i = 0; i < std::min(*n_out, cap); ++i) {
      ty_tx[2 * i] = khi(keys[i]);
      ty_tx[2 * i + 1] = klo(keys[i]);
    }
  return IDF_OK;
}

idf_status idf_debug_set_status(idf_world* W, int32_t which, int32_t value) {
  if (!W || which < 0 || which > 1) return IDF_EINVAL;
  if (!cuda_ok(W, cudaStreamSynchronize(W->st), "sync")) return fail(W, IDF_ECUDA, W->last_error);
  if (which == 0) {
    for (auto& L : W->lv)
      if (L.unet && !cuda_ok(W, cudaMemcpy(unet_status(L.unet), &value, sizeof(int), cudaMemcpyHostToDevice),
                             "write status"))
        return fail(W, IDF_ECUDA, W->last_error);
  } else if (!cuda_ok(W, cudaMemcpy(W->d_err, &value, sizeof(int), cudaMemcpyHostToDevice), "write status")) {
    return fail(W, IDF_ECUDA, W->last_error);
  }
  return IDF_OK;
}

idf_status idf_noise_fill(uint64_t seed, uint32_t level, uint32_t step, int64_t x0, int64_t y0,
                          int32_t w, int32_t h, float* out_dev, int64_t pitch, void* stream) {
  if (!out_dev || w < 1 || h < 1 || pitch < w) return IDF_EINVAL;
  launch_noise_fill(seed, level, step, x0, y0, w, h, out_dev, pitch, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? IDF_OK : IDF_ECUDA;
}

idf_status idf_unet_forward(idf_world* W, int32_t level, const float* x_dev, int32_t n, float* y_dev,
                            void* stream) {
  if (!W || !x_dev || !y_dev || n < 0) return IDF_EINVAL;
  if (level < 0 || level >= (int)W->lv.size()) return fail(W, IDF_EINVAL, "bad level");
  if (W->poisoned) return fail(W, IDF_EINTERNAL, "world unusable after an earlier CUDA failure");
  Level& L = W->lv[level];
  if (n == 0) return IDF_OK;
  cudaStream_t user = (cudaStream_t)stream;
  if (join_in(W, user) != IDF_OK) return IDF_ECUDA;
  const int H = L.H, cin = L.d.in_ch;
  const int B = L.unet ? unet_max_batch(L.unet) : n;
  if (!grow(W, &W->x_in, &W->x_cap, (size_t)std::min(B, n) * H * H * cin, "window inputs"))
    return fail(W, IDF_ENOMEM, W->last_error);
  for (int b0 = 0; b0 < n; b0 += B) {
    const int nb = std::min(B, n - b0);
    launch_nchw_to_nhwc(x_dev + (size_t)b0 * cin * H * H, nb, cin, H * H, W->x_in, W->st);
    float* y = y_dev + (size_t)b0 * H * H;
    if (L.d.test_denoiser) {
      launch_test_denoiser(L.d.test_denoiser, W->x_in, nb, H, cin, y, W->st);
    } else {
      Err e;
      if (!unet_forward(L.unet, W->x_in, nb, y, W->st, &e)) {
        W->last_error = e.msg;
        W->poisoned = e.code == 3;
        return e.code == 3 ? IDF_ECUDA : IDF_EINTERNAL;
      }
    }
  }
  if (!cuda_ok(W, cudaGetLastError(), "unet launch")) return IDF_ECUDA;
  return join_out(W, user);
}

idf_status idf_laplacian_halo(const idf_model_stack* stack, int64_t x0, int64_t y0, int32_t w, int32_t h,
                              int64_t L_rect[4], int64_t H_rect[4]) {
  if (!stack || !L_rect || !H_rect || stack->lap_factor < 2 || stack->lap_factor % 2 ||
      stack->lap_radius < 0 || !valid_region(x0, y0, w, h))
    return IDF_EINVAL;
  Halo hl = decode_halo(stack->lap_factor, stack->lap_radius, x0, y0, w, h);
  L_rect[0] = hl.Lx0; L_rect[1] = hl.Ly0; L_rect[2] = hl.Lw; L_rect[3] = hl.Lh;
  H_rect[0] = hl.Hx0; H_rect[1] = hl.Hy0; H_rect[2] = hl.Hw; H_rect[3] = hl.Hh;
  return IDF_OK;
}

idf_status idf_laplacian_decode(const idf_model_stack* stack, const float* L_dev, int64_t lx0, int64_t ly0,
                                int32_t lw, int32_t lh, int64_t lpitch, const float* H_dev, int64_t hx0,
                                int64_t hy0, int32_t hw, int32_t hh, int64_t hpitch, int64_t x0, int64_t y0,
                                int32_t w, int32_t h, float* out_dev, int64_t pitch, void* stream) {
  if (!stack || !L_dev || !H_dev || !out_dev || pitch < w || lpitch < lw || hpitch < hw) return IDF_EINVAL;
  if (stack->lap_factor < 2 || stack->lap_factor % 2 || stack->lap_radius < 0 || stack->lap_radius > 64 ||
      !(stack->lap_blur_sigma > 0) || !valid_region(x0, y0, w, h))
    return IDF_EINVAL;
  const int f = stack->lap_factor, R = stack->lap_radius;
  Halo hl = decode_halo(f, R, x0, y0, w, h);
  if (hl.Lx0 < lx0 || hl.Ly0 < ly0 || hl.Lx0 + hl.Lw > lx0 + lw || hl.Ly0 + hl.Lh > ly0 + lh) return IDF_EINVAL;
  if (hl.Hx0 < hx0 || hl.Hy0 < hy0 || hl.Hx0 + hl.Hw > hx0 + hw || hl.Hy0 + hl.Hh > hy0 + hh) return IDF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nD = (size_t)(hl.qw + 2 * R) * (hl.qh + 2 * R);
  const size_t nT = (size_t)hl.qw * (hl.qh + 2 * R);
  const size_t nQ = (size_t)hl.qw * hl.qh;
  auto taps = blur_taps(stack->lap_blur_sigma, R);
  float* scratch = nullptr;
  const size_t n = nD + nT + nQ + taps.size();
  if (cudaMallocAsync((void**)&scratch, n * 4, st) != cudaSuccess) {
    cudaGetLastError();
    return IDF_ENOMEM;
  }
  if (cudaMemcpyAsync(scratch + nD + nT + nQ, taps.data(), taps.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return IDF_ECUDA;
  DecodeArgs a{};
  a.L = L_dev; a.lx0 = lx0; a.ly0 = ly0; a.lpitch = lpitch; a.lw = lw; a.lh = lh;
  a.H = H_dev; a.hx0 = hx0; a.hy0 = hy0; a.hpitch = hpitch; a.hw = hw; a.hh = hh;
  a.x0 = x0; a.y0 = y0; a.w = w; a.h = h; a.out = out_dev; a.pitch = pitch;
  a.f = f; a.R = R;
  a.low_mu = (float)stack->low_mu; a.low_scale = (float)stack->low_scale; a.res_scale = (float)stack->res_scale;
  a.D = scratch; a.T = scratch + nD; a.Lhat = a.T + nT; a.taps = a.Lhat + nQ;
  a.qx0 = hl.qx0; a.qy0 = hl.qy0; a.qw = (int)hl.qw; a.qh = (int)hl.qh;
  launch_decode(a, st);
  // the pageable taps vector is staged before cudaMemcpyAsync returns
  cudaFreeAsync(scratch, st);
  return cudaGetLastError() == cudaSuccess ? IDF_OK : IDF_ECUDA;
}

}  // extern "C"
