// Grouped apply: C ABI, launch plans and the autotuner.
//
// A group is a list of (operator, input, output, quantisation tables)
// items run by one persistent launch of apply_group_kernel; a pixel group's
// items are (operator, coefficients, uint8 image) for the fused pixel
// output.  Creating a
// group encodes every item's TMA tensor maps once and uploads the
// descriptors; launching it is then a single kernel launch with no host work,
// so it can be captured in a CUDA graph and replayed.
//
// Autotuner.  Three launch parameters matter for uneven batches: the number
// of persistent CTAs, the tile height (128-row tiles, or 64-row tiles that
// balance small items better) and the shared-memory layout (input stages x
// operator slots: more stages keep more loads in flight, two slots let
// operator switches overlap the previous item's tiles).  dctf_group_tune
// times every candidate on the group itself (CUDA events around four
// back-to-back launches, median of `reps` rounds) and keeps the fastest; the
// choice is also cached per (device, I/O type, size class) and used as the
// default for later groups of that class.  With
// DCTF_TUNE_CACHE naming a file, the cache is read from it at the first
// group and written back after every tuning, so later processes start from
// the tuned choice.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "apply_group.cuh"

struct dctf_group {
  int device;
  int nitems;
  bool i16;
  bool pixels;     // items write uint8 images (fused pixel output)
  int64_t total_halves;
  dctf::GroupItem *d_items;
  uint32_t *d_err;
  int grid;        // CTAs (0: one per SM)
  int max_take;    // 2: 128-row tiles, 1: 64-row tiles
  int variant;     // shared-memory layout (stages x slots), 0..kGroupVariants-1
  bool in_place;   // some item filters in place (tuning would re-filter it)
  uint32_t flags;  // DCTF_APPLY_INPUTS_READY: launch with programmatic serialisation
};

namespace dctf {
namespace {

struct TuneKey {
  int sms;          // the device, by its SM count (one process may see several kinds)
  int kind;         // 0: FP32 coefficients, 1: int16, 2: pixels
  int size_class;   // floor(log2(total halves))
  bool operator<(const TuneKey &o) const {
    if (sms != o.sms) return sms < o.sms;
    return kind != o.kind ? kind < o.kind : size_class < o.size_class;
  }
};
int kind_of(const dctf_group *g) { return g->pixels ? 2 : g->i16 ? 1 : 0; }
struct TuneVal { int grid_num, grid_den, max_take, variant; };

std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;
bool g_tune_loaded = false;

// The persistent cache file (DCTF_TUNE_CACHE), one line per entry:
// "sms kind size_class grid_num grid_den max_take variant".  Unreadable or
// malformed lines are ignored; callers hold g_tune_mu.
void tune_cache_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *path = getenv("DCTF_TUNE_CACHE");
  if (path == nullptr || *path == 0) return;
  FILE *f = fopen(path, "r");
  if (f == nullptr) return;
  TuneKey k;
  TuneVal v;
  while (fscanf(f, "%d %d %d %d %d %d %d", &k.sms, &k.kind, &k.size_class, &v.grid_num,
                &v.grid_den, &v.max_take, &v.variant) == 7) {
    if (k.kind >= 0 && k.kind <= 2 && v.grid_num > 0 && v.grid_den > 0 && v.grid_num <= v.grid_den &&
        (v.max_take == 1 || v.max_take == 2) && v.variant >= 0 && v.variant < kGroupVariants)
      g_tune_cache[k] = v;
  }
  fclose(f);
}
void tune_cache_save() {
  const char *path = getenv("DCTF_TUNE_CACHE");
  if (path == nullptr || *path == 0) return;
  FILE *f = fopen(path, "w");
  if (f == nullptr) return;
  for (const auto &kv : g_tune_cache)
    fprintf(f, "%d %d %d %d %d %d %d\n", kv.first.sms, kv.first.kind, kv.first.size_class,
            kv.second.grid_num, kv.second.grid_den, kv.second.max_take, kv.second.variant);
  fclose(f);
}

int size_class(int64_t halves) {
  int c = 0;
  while ((halves >> (c + 1)) > 0) ++c;
  return c;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

dctf_status check_items(const dctf_group_item *items, int nitems, dctf_io io) {
  if (nitems < 0 || (nitems > 0 && items == nullptr))
    return set_error(DCTF_EINVAL, "bad item list");
  if (io != DCTF_IO_F32 && io != DCTF_IO_I16) return set_error(DCTF_EINVAL, "bad io type %d", io);
  for (int i = 0; i < nitems; ++i) {
    const dctf_group_item &it = items[i];
    if (it.op == nullptr) return set_error(DCTF_EINVAL, "item %d: operator is NULL", i);
    if (it.op->n != 8 || it.op->d_f16 == nullptr)
      return set_error(DCTF_EUNSUPPORTED, "item %d: grouped apply needs an 8x8 operator", i);
    if (it.nblocks < 0) return set_error(DCTF_EINVAL, "item %d: nblocks < 0", i);
    if (it.nblocks == 0) continue;
    if (it.in == nullptr || it.out == nullptr || !aligned16(it.in) || !aligned16(it.out))
      return set_error(DCTF_EINVAL, "item %d: buffers must be non-NULL and 16-byte aligned", i);
    if (it.nblocks > ((int64_t)1 << 31) - 128)
      return set_error(DCTF_EINVAL, "item %d: nblocks too large", i);
    const size_t bytes = (size_t)it.nblocks * 64 * (io == DCTF_IO_I16 ? 2 : 4);
    const char *a = static_cast<const char *>(it.in);
    const char *b = static_cast<const char *>(it.out);
    if (a != b && a < b + bytes && b < a + bytes)
      return set_error(DCTF_EINVAL, "item %d: input and output overlap without being equal", i);
    if (io == DCTF_IO_I16) {
      if (it.q_in == nullptr || it.q_out == nullptr || !aligned16(it.q_in) || !aligned16(it.q_out))
        return set_error(DCTF_EINVAL, "item %d: int16 items need 16-byte aligned q tables", i);
    }
  }
  return DCTF_OK;
}

dctf_status fill_items(const dctf_group_item *items, int nitems, dctf_io io,
                       std::vector<GroupItem> *out, int64_t *total) {
  out->resize(nitems > 0 ? nitems : 1);
  int64_t h = 0;
  for (int i = 0; i < nitems; ++i) {
    const dctf_group_item &it = items[i];
    GroupItem &gi = (*out)[i];
    if (it.nblocks > 0) {
      cudaError_t e = fill_group_item(&gi, it.op, it.in, it.out, it.nblocks, io == DCTF_IO_I16,
                                      it.q_in, it.q_out);
      if (e != cudaSuccess) return cuda_error(e, "tensor map encode");
    } else {
      memset(&gi, 0, sizeof gi);
    }
    gi.half_begin = h;
    h += (it.nblocks + 63) / 64;
  }
  *total = h;
  return DCTF_OK;
}

dctf_status check_pixel_items(const dctf_pixel_item *items, int nitems) {
  if (nitems < 0 || (nitems > 0 && items == nullptr))
    return set_error(DCTF_EINVAL, "bad item list");
  for (int i = 0; i < nitems; ++i) {
    const dctf_pixel_item &it = items[i];
    if (it.op == nullptr) return set_error(DCTF_EINVAL, "item %d: operator is NULL", i);
    if (it.op->n != 8 || it.op->d_f16_pix == nullptr)
      return set_error(DCTF_EUNSUPPORTED, "item %d: the fused pixel apply needs an 8x8 operator", i);
    if (it.coeffs == nullptr || it.image == nullptr)
      return set_error(DCTF_EINVAL, "item %d: NULL buffer", i);
    if (it.height <= 0 || it.width <= 0 || it.height % 8 || it.width % 8)
      return set_error(DCTF_EINVAL, "item %d: image %dx%d: sides must be positive multiples of 8",
                       i, it.height, it.width);
    if (it.pitch < it.width || it.pitch % 8)
      return set_error(DCTF_EINVAL, "item %d: pitch must be >= width and a multiple of 8", i);
    if (!aligned16(it.coeffs) || (reinterpret_cast<uintptr_t>(it.image) & 7))
      return set_error(DCTF_EINVAL, "item %d: coeffs must be 16-byte, image 8-byte aligned", i);
    const int64_t nb = (int64_t)(it.height / 8) * (it.width / 8);
    if (nb > ((int64_t)1 << 31) - 128) return set_error(DCTF_EINVAL, "item %d: image too large", i);
    const char *a = reinterpret_cast<const char *>(it.coeffs);
    const char *b = reinterpret_cast<const char *>(it.image);
    const size_t la = (size_t)nb * 64 * sizeof(float);
    const size_t lb = (size_t)(it.height - 1) * it.pitch + it.width;
    if (a < b + lb && b < a + la)
      return set_error(DCTF_EINVAL, "item %d: coefficients and image overlap", i);
  }
  return DCTF_OK;
}

dctf_status fill_pixel_items(const dctf_pixel_item *items, int nitems,
                             std::vector<GroupItem> *out, int64_t *total) {
  out->resize(nitems > 0 ? nitems : 1);
  int64_t h = 0;
  for (int i = 0; i < nitems; ++i) {
    const dctf_pixel_item &it = items[i];
    GroupItem &gi = (*out)[i];
    const int64_t nb = (int64_t)(it.height / 8) * (it.width / 8);
    // (the coefficient output map is not used: pointed at the input)
    cudaError_t e = fill_group_item(&gi, it.op, it.coeffs, const_cast<float *>(it.coeffs), nb,
                                    false, nullptr, nullptr);
    if (e != cudaSuccess) return cuda_error(e, "tensor map encode");
    gi.pieces = it.op->d_f16_pix;
    gi.mdc = it.op->d_Gdc;
    gi.img = it.image;
    gi.pitch = it.pitch;
    gi.bw = it.width / 8;
    gi.half_begin = h;
    h += (nb + 63) / 64;
  }
  *total = h;
  return DCTF_OK;
}

cudaError_t launch(const dctf_group *g, int grid, int max_take, int variant, cudaStream_t s) {
  const bool pdl = (g->flags & DCTF_APPLY_INPUTS_READY) != 0;
  if (g->pixels)
    return launch_apply_group_pixels(g->d_items, g->nitems, g->total_halves, grid, max_take,
                                     g->d_err, s, variant, pdl);
  return launch_apply_group(g->d_items, nullptr, g->nitems, g->total_halves, g->i16, grid,
                            max_take, g->d_err, s, pdl, variant);
}

// Uploads the descriptors and picks the launch parameters (the autotuner's
// cached choice for this kind and size class, else one CTA per SM and
// 128-row tiles).
dctf_status make_group(const std::vector<GroupItem> &host, int nitems, int64_t total, bool i16,
                       bool pixels, bool in_place, dctf_group **out) {
  dctf_group *g = new (std::nothrow) dctf_group();
  if (g == nullptr) return set_error(DCTF_ENOMEM, "host allocation failed");
  g->nitems = nitems;
  g->i16 = i16;
  g->pixels = pixels;
  g->total_halves = total;
  g->in_place = in_place;
  cudaError_t e = cudaGetDevice(&g->device);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_items, host.size() * sizeof(GroupItem) + 256);
  if (e == cudaSuccess) {
    g->d_err = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(g->d_items) +
                                            host.size() * sizeof(GroupItem));
    e = cudaMemcpy(g->d_items, host.data(), host.size() * sizeof(GroupItem),
                   cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemset(g->d_err, 0, 256);
  if (e != cudaSuccess) {
    if (g->d_items) cudaFree(g->d_items);
    delete g;
    return cuda_error(e, "group descriptors");
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache_load();
    const int sms = sm_count(g->device);
    auto it = g_tune_cache.find(TuneKey{sms, kind_of(g), size_class(total)});
    if (it != g_tune_cache.end()) {
      g->grid = std::max(1, sms * it->second.grid_num / it->second.grid_den);
      g->max_take = it->second.max_take;
      g->variant = it->second.variant;
    } else {
      g->grid = 0;
      g->max_take = 2;
      g->variant = 0;
    }
  }
  *out = g;
  return DCTF_OK;
}

}  // namespace
}  // namespace dctf

using namespace dctf;

extern "C" {

dctf_status dctf_group_create(const dctf_group_item *items, int nitems, dctf_io io,
                              dctf_group **out) {
  if (out == nullptr) return set_error(DCTF_EINVAL, "out is NULL");
  *out = nullptr;
  dctf_status st = check_items(items, nitems, io);
  if (st != DCTF_OK) return st;
  std::vector<GroupItem> host;
  int64_t total = 0;
  st = fill_items(items, nitems, io, &host, &total);
  if (st != DCTF_OK) return st;
  bool in_place = false;
  for (int i = 0; i < nitems; ++i)
    if (items[i].nblocks > 0 && items[i].in == items[i].out) in_place = true;
  return make_group(host, nitems, total, io == DCTF_IO_I16, false, in_place, out);
}

dctf_status dctf_group_create_pixels(const dctf_pixel_item *items, int nitems, dctf_group **out) {
  if (out == nullptr) return set_error(DCTF_EINVAL, "out is NULL");
  *out = nullptr;
  dctf_status st = check_pixel_items(items, nitems);
  if (st != DCTF_OK) return st;
  std::vector<GroupItem> host;
  int64_t total = 0;
  st = fill_pixel_items(items, nitems, &host, &total);
  if (st != DCTF_OK) return st;
  return make_group(host, nitems, total, false, true, false, out);
}

dctf_status dctf_group_launch(const dctf_group *g, dctf_stream_t stream) {
  if (g == nullptr) return set_error(DCTF_EINVAL, "group is NULL");
  if (g->total_halves == 0) return DCTF_OK;
  int grid = g->grid > 0 ? g->grid : sm_count(g->device);
  cudaError_t e = launch(g, grid, g->max_take, g->variant, stream);
  if (e != cudaSuccess) return cuda_error(e, "grouped apply launch");
  return DCTF_OK;
}

dctf_status dctf_group_tune(dctf_group *g, dctf_stream_t stream, int reps) {
  if (g == nullptr) return set_error(DCTF_EINVAL, "group is NULL");
  if (g->total_halves == 0) return DCTF_OK;
  if (g->in_place)
    return set_error(DCTF_EINVAL, "tuning runs the group repeatedly: items must not be in place");
  if (reps < 1) reps = 5;
  const int sms = sm_count(g->device);
  static const int kFrac[][2] = {{1, 1}, {3, 4}, {1, 2}};
  constexpr int kBackToBack = 4;
  cudaEvent_t e0, e1;
  DCTF_CUDA(cudaEventCreate(&e0));
  DCTF_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  TuneVal best_v{1, 1, 2, 0};
  for (int v = 0; v < kGroupVariants; ++v)
  for (const auto &f : kFrac) {
    for (int take = 2; take >= 1; --take) {
      const int grid = std::max(1, sms * f[0] / f[1]);
      std::vector<float> ts;
      for (int r = 0; r < reps + 1; ++r) {
        // kBackToBack launches between the events, as a graph replays them:
        // one launch alone would add its launch latency and its fill and
        // drain to every candidate alike
        cudaEventRecord(e0, stream);
        cudaError_t e = cudaSuccess;
        for (int q = 0; q < kBackToBack && e == cudaSuccess; ++q) e = launch(g, grid, take, v, stream);
        cudaEventRecord(e1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return cuda_error(e, "autotune launch");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) ts.push_back(ms / kBackToBack);   // first round warms the caches
      }
      std::sort(ts.begin(), ts.end());
      const float med = ts[ts.size() / 2];
      if (med < best) { best = med; best_v = TuneVal{f[0], f[1], take, v}; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g->grid = std::max(1, sms * best_v.grid_num / best_v.grid_den);
  g->max_take = best_v.max_take;
  g->variant = best_v.variant;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_cache_load();
  g_tune_cache[TuneKey{sms, kind_of(g), size_class(g->total_halves)}] = best_v;
  tune_cache_save();
  return DCTF_OK;
}

dctf_status dctf_group_config(const dctf_group *g, int *grid, int *tile_rows, int *stages,
                              int *slots) {
  if (g == nullptr) return set_error(DCTF_EINVAL, "group is NULL");
  if (grid) *grid = g->grid > 0 ? g->grid : sm_count(g->device);
  if (tile_rows) *tile_rows = 64 * g->max_take;
  if (stages) *stages = group_variant_stages(kind_of(g), g->variant);
  if (slots) *slots = group_variant_slots(kind_of(g), g->variant);
  return DCTF_OK;
}

dctf_status dctf_group_set_config(dctf_group *g, int grid, int tile_rows, int stages, int slots) {
  if (g == nullptr) return set_error(DCTF_EINVAL, "group is NULL");
  if (grid < 0 || (tile_rows != 64 && tile_rows != 128))
    return set_error(DCTF_EINVAL, "grid must be >= 0 and tile_rows 64 or 128");
  int v = -1;
  for (int k = 0; k < kGroupVariants; ++k)
    if (group_variant_stages(kind_of(g), k) == stages && group_variant_slots(kind_of(g), k) == slots)
      v = k;
  if (v < 0) return set_error(DCTF_EUNSUPPORTED, "no layout with %d stages and %d slots", stages, slots);
  g->grid = grid;
  g->max_take = tile_rows / 64;
  g->variant = v;
  return DCTF_OK;
}

dctf_status dctf_group_set_flags(dctf_group *g, uint32_t flags) {
  if (g == nullptr) return set_error(DCTF_EINVAL, "group is NULL");
  if (flags & ~(uint32_t)DCTF_APPLY_INPUTS_READY) return set_error(DCTF_EINVAL, "unknown flags");
  g->flags = flags;
  return DCTF_OK;
}

dctf_status dctf_group_status(dctf_group *g, uint32_t *code, int clear) {
  if (g == nullptr || code == nullptr) return set_error(DCTF_EINVAL, "NULL argument");
  DCTF_CUDA(cudaDeviceSynchronize());
  DCTF_CUDA(cudaMemcpy(code, g->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (clear) DCTF_CUDA(cudaMemset(g->d_err, 0, sizeof(uint32_t)));
  return DCTF_OK;
}

void dctf_group_destroy(dctf_group *g) {
  if (g == nullptr) return;
  if (g->d_items) cudaFree(g->d_items);
  delete g;
}

dctf_status dctf_apply_grouped(const dctf_group_item *items, int nitems, dctf_io io,
                               dctf_stream_t stream) {
  dctf_group *g = nullptr;
  dctf_status st = dctf_group_create(items, nitems, io, &g);
  if (st != DCTF_OK) return st;
  st = dctf_group_launch(g, stream);
  // the descriptors must outlive the launch
  cudaError_t e = cudaStreamSynchronize(stream);
  dctf_group_destroy(g);
  if (st != DCTF_OK) return st;
  if (e != cudaSuccess) return cuda_error(e, "grouped apply");
  return DCTF_OK;
}

}  // extern "C"
