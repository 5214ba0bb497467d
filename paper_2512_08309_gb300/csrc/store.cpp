// Persistent tile store of libidf: finalized tiles of a world kept in a
// directory of chunk files, so that a later session of the same world (same
// seed, model stack and precision) reads them instead of recomputing their
// dependency cones ("Caching and Persistence" in the infinite-tensor
// appendix).  A tile's value depends only on the seed and its position
// (Lemma 3), so a stored tile is valid for every later query of that world.
//
// Layout: a manifest file names the world's identity (a 64-bit FNV-1a hash
// of the seed, the stack description, the weights and the precision) and the
// tile side of every level; tiles live in chunk files of 16 x 16 tiles,
// L<level>_<chunk row>_<chunk column>.tiles, each a 64-byte header, a
// 256-byte presence map and 256 fixed slots of side^2 float32 values, read
// and written with pread / pwrite at fixed offsets.  A process keeps at most
// 64 chunk files open (least recently used closed first).
#include <errno.h>
#include <fcntl.h>
#include <stdio.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <list>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace idf {
namespace {

constexpr int CT = 16;             // tiles per chunk side
constexpr int HDR = 64;            // header bytes
constexpr int MAP = CT * CT;       // presence bytes
constexpr size_t MAX_OPEN = 64;
const char MAGIC[8] = {'I', 'D', 'F', 'T', 'I', 'L', 'E', '1'};

inline int32_t cdiv(int32_t a) { return (int32_t)fdiv(a, CT); }

struct Chunk {
  int fd = -1;
  uint8_t present[MAP];
  std::list<uint64_t>::iterator lru;
};

}  // namespace

struct TileStore {
  std::string dir;
  bool writable = false;
  std::vector<int> side;                       // tile side per level
  std::unordered_map<uint64_t, Chunk> chunks;  // (level, cy, cx) -> chunk
  std::list<uint64_t> lru;                     // open chunks, most recent first
  std::vector<float> zero;
};

namespace {

// chunk indices of int32 tile indices fit in 28 bits (|c| < 2^27)
uint64_t ckey(int level, int32_t cy, int32_t cx) {
  const uint64_t a = (uint64_t)((int64_t)cy + (1 << 27)) & 0xFFFFFFFull;
  const uint64_t b = (uint64_t)((int64_t)cx + (1 << 27)) & 0xFFFFFFFull;
  return ((uint64_t)(uint32_t)level << 56) | (a << 28) | b;
}

std::string chunk_path(const TileStore* s, int level, int32_t cy, int32_t cx) {
  char b[96];
  snprintf(b, sizeof b, "/L%d_%d_%d.tiles", level, (int)cy, (int)cx);
  return s->dir + b;
}

// the chunk holding (level, ty, tx), opened (and, when writable, created) on
// first use; null when it does not exist and cannot be created
Chunk* get_chunk(TileStore* s, int level, int32_t ty, int32_t tx, bool create) {
  const int32_t cy = cdiv(ty), cx = cdiv(tx);
  const uint64_t k = ckey(level, cy, cx);
  auto it = s->chunks.find(k);
  if (it != s->chunks.end()) {
    if (it->second.fd < 0) return &it->second;  // known absent
    s->lru.erase(it->second.lru);
    s->lru.push_front(k);
    it->second.lru = s->lru.begin();
    return &it->second;
  }
  const std::string path = chunk_path(s, level, cy, cx);
  const size_t tile_bytes = (size_t)s->side[level] * s->side[level] * 4;
  int fd = open(path.c_str(), s->writable ? O_RDWR : O_RDONLY);
  Chunk c;
  memset(c.present, 0, MAP);
  if (fd < 0) {
    if (!(create && s->writable)) {
      // remember that the chunk is absent (until this process writes it)
      c.fd = -1;
      auto& e = s->chunks[k];
      e = c;
      return &e;
    }
    fd = open(path.c_str(), O_RDWR | O_CREAT, 0644);
    if (fd < 0) return nullptr;
    uint8_t h[HDR + MAP];
    memset(h, 0, sizeof h);
    memcpy(h, MAGIC, 8);
    const int32_t meta[4] = {level, s->side[level], cy, cx};
    memcpy(h + 8, meta, sizeof meta);
    if (pwrite(fd, h, sizeof h, 0) != (ssize_t)sizeof h ||
        ftruncate(fd, (off_t)(HDR + MAP) + (off_t)MAP * (off_t)tile_bytes) != 0) {
      close(fd);
      return nullptr;
    }
  } else {
    uint8_t h[HDR];
    int32_t meta[4];
    if (pread(fd, h, HDR, 0) != HDR || memcmp(h, MAGIC, 8) != 0 || pread(fd, c.present, MAP, HDR) != MAP) {
      close(fd);
      return nullptr;
    }
    memcpy(meta, h + 8, sizeof meta);
    if (meta[0] != level || meta[1] != s->side[level] || meta[2] != cy || meta[3] != cx) {
      close(fd);
      return nullptr;
    }
  }
  c.fd = fd;
  s->lru.push_front(k);
  c.lru = s->lru.begin();
  s->chunks[k] = c;
  // keep at most MAX_OPEN files open; closed chunks are forgotten and
  // re-read from disk when needed again
  while (s->lru.size() > MAX_OPEN) {
    const uint64_t old = s->lru.back();
    s->lru.pop_back();
    auto o = s->chunks.find(old);
    if (o != s->chunks.end()) {
      close(o->second.fd);
      s->chunks.erase(o);
    }
  }
  return &s->chunks[k];
}

int slot_of(int32_t ty, int32_t tx) { return (int)(fmod_pos(ty, CT) * CT + fmod_pos(tx, CT)); }

}  // namespace

TileStore* store_open(const std::string& dir, uint64_t identity, const std::vector<int>& side, bool writable,
                      std::string* err) {
  if (writable) mkdir(dir.c_str(), 0755);
  struct stat st;
  if (stat(dir.c_str(), &st) != 0 || !S_ISDIR(st.st_mode)) {
    *err = "tile store directory missing: " + dir;
    return nullptr;
  }
  const std::string mf = dir + "/idf_store.manifest";
  char want[256];
  int n = snprintf(want, sizeof want, "idf-tile-store 1\nidentity %016llx\nlevels %d", (unsigned long long)identity,
                   (int)side.size());
  for (int v : side) n += snprintf(want + n, sizeof want - n, " %d", v);
  snprintf(want + n, sizeof want - n, "\n");
  FILE* f = fopen(mf.c_str(), "rb");
  if (f) {
    char got[256] = {0};
    const size_t r = fread(got, 1, sizeof got - 1, f);
    fclose(f);
    got[r] = 0;
    if (strcmp(got, want) != 0) {
      *err = "tile store belongs to another world (seed, stack, weights or precision differ)";
      return nullptr;
    }
  } else {
    if (!writable) {
      *err = "tile store has no manifest: " + mf;
      return nullptr;
    }
    f = fopen(mf.c_str(), "wb");
    if (!f || fwrite(want, 1, strlen(want), f) != strlen(want)) {
      if (f) fclose(f);
      *err = "cannot write the tile store manifest";
      return nullptr;
    }
    fclose(f);
  }
  TileStore* s = new TileStore();
  s->dir = dir;
  s->writable = writable;
  s->side = side;
  return s;
}

void store_close(TileStore* s) {
  if (!s) return;
  for (auto& kv : s->chunks)
    if (kv.second.fd >= 0) close(kv.second.fd);
  delete s;
}

bool store_has(TileStore* s, int level, int32_t ty, int32_t tx) {
  Chunk* c = get_chunk(s, level, ty, tx, false);
  return c && c->fd >= 0 && c->present[slot_of(ty, tx)];
}

bool store_read(TileStore* s, int level, int32_t ty, int32_t tx, float* dst) {
  Chunk* c = get_chunk(s, level, ty, tx, false);
  const int sl = slot_of(ty, tx);
  if (!c || c->fd < 0 || !c->present[sl]) return false;
  const size_t tb = (size_t)s->side[level] * s->side[level] * 4;
  return pread(c->fd, dst, tb, (off_t)(HDR + MAP) + (off_t)sl * (off_t)tb) == (ssize_t)tb;
}

bool store_write(TileStore* s, int level, int32_t ty, int32_t tx, const float* src) {
  if (!s->writable) return false;
  Chunk* c = get_chunk(s, level, ty, tx, true);
  if (c && c->fd < 0) {
    // known absent so far: forget that and create it
    const uint64_t k = ckey(level, cdiv(ty), cdiv(tx));
    s->chunks.erase(k);
    c = get_chunk(s, level, ty, tx, true);
  }
  if (!c || c->fd < 0) return false;
  const int sl = slot_of(ty, tx);
  const size_t tb = (size_t)s->side[level] * s->side[level] * 4;
  if (pwrite(c->fd, src, tb, (off_t)(HDR + MAP) + (off_t)sl * (off_t)tb) != (ssize_t)tb) return false;
  if (!c->present[sl]) {
    c->present[sl] = 1;
    const uint8_t one = 1;
    if (pwrite(c->fd, &one, 1, HDR + sl) != 1) return false;
  }
  return true;
}

}  // namespace idf
