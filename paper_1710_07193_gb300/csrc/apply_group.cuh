// Descriptor of one work item of the persistent grouped apply kernel.
#pragma once

#include "sm100_ptx.cuh"

namespace dctf {

// Per-item operator slot in shared memory: B pieces (F16X3, 8x8 blocks),
// M[:,0], and the two quantisation tables of the int16 path.
constexpr int kSlotPieces = 2 * 64 * 128;   // 128 rows x 128 B
constexpr int kSlotMdc = 64 * 4;
constexpr int kSlotQ = 64 * 2;
constexpr int kSlotBytes = 17408;            // rounded up to 1024 (swizzle atom)
static_assert(kSlotPieces + kSlotMdc + 2 * kSlotQ <= kSlotBytes, "slot size");

struct GroupItem {              // CUtensorMap members keep it 128-byte aligned
  CUtensorMap tm_in;        // 128-row boxes
  CUtensorMap tm_in_half;   // 64-row boxes (tiles at range / item ends)
  CUtensorMap tm_out;       // 32-row boxes (one per epilogue warp)
  const void *pieces;       // FP16 hi/lo B image (16 KB, SWIZZLE_128B layout)
  const float *mdc;         // M[:, 0], FP32
  const uint16_t *qin;      // quantisation table of the input (int16 path)
  const uint16_t *qout;     // quantisation table of the output (int16 path)
  float out_scale;          // 2^-s of the pieces
  int pad0;
  int64_t nblocks;
  int64_t half_begin;       // first 64-block half tile of the item in the group
  uint8_t *img;             // pixel output (apply_pixels): uint8 image,
  int64_t pitch;            //   its row pitch in bytes (image-plane layout:
                            //   the plane's width in blocks),
  int64_t bw;               //   and its width in blocks (image-plane layout:
                            //   padded to a multiple of 128)
  const void *hin;          // host-direct apply: mapped page-locked host input
  void *hout;               //   and output, [nblocks][64] FP32 or int16, 16-byte aligned
};

cudaError_t fill_group_item(GroupItem *gi, const dctf_operator *op, const void *in, void *out,
                            int64_t nblocks, bool i16, const uint16_t *qin,
                            const uint16_t *qout);
// Descriptor of a host-direct item: hin / hout are device addresses of
// mapped page-locked host memory (16-byte aligned); no tensor maps.
cudaError_t fill_group_item_host(GroupItem *gi, const dctf_operator *op, const void *hin,
                                 void *hout, int64_t nblocks, const uint16_t *qin,
                                 const uint16_t *qout);

// d_items: device array (group mode, single == nullptr) or single: one item
// passed by value.  grid <= 0 means one CTA per SM.  max_take: 2 for 128-row
// tiles, 1 for 64-row tiles.  pdl: launch with programmatic stream
// serialisation (the inputs must not be written by the preceding kernel).
// Fused pixel output, one item: the item's pieces and mdc are those of the
// pixel operator G = H K^T (and G[:, 0]); the epilogue writes uint8 pixels
// into item.img instead of coefficients.
cudaError_t launch_apply_pixels(const GroupItem &single, int64_t total_halves, int grid,
                                uint32_t *err, cudaStream_t s, bool pdl);

// Image-plane coefficient layout (8x8 blocks, F16X3): in/out are FP32
// arrays of `height` rows of `pitch` floats, block (by, bx)'s coefficient
// (u, v) at row 8 by + u, column 8 bx + v.
cudaError_t launch_apply_planar(const dctf_operator *op, const float *in, int height, int width,
                                int64_t in_pitch, float *out, int64_t out_pitch, uint32_t *err,
                                cudaStream_t s, bool pdl);

// Host-direct apply, one item (8x8 blocks, F16X3, FP32 coefficients): the
// producer warp copies each input tile from item.hin (page-locked host
// memory, mapped) with 16-byte cp.async and the epilogue writes item.hout
// with plain stores, so the coefficients cross the host link once each way
// with no device staging.  Same arithmetic and per-block order as
// launch_apply_group.  `grid` CTAs (the host link bounds this launch, not
// the SMs), 64-block tiles.  Never uses programmatic dependent launch.
cudaError_t launch_apply_host_direct(const GroupItem &single, int64_t total_halves, int grid,
                                     uint32_t *err, cudaStream_t s);

// Grouped launches come in kGroupVariants shared-memory layouts (input
// stages x operator slots), the autotuner's third axis; kind 0 = FP32
// coefficients, 1 = int16, 2 = pixels.  Every variant gives the same bits.
constexpr int kGroupVariants = 3;
int group_variant_stages(int kind, int variant);
int group_variant_slots(int kind, int variant);

// Fused pixel output for many items (descriptors in global memory, each
// filled as for launch_apply_pixels): one persistent launch, contiguous
// schedule.
cudaError_t launch_apply_group_pixels(const GroupItem *d_items, int nitems, int64_t total_halves,
                                      int grid, int max_take, uint32_t *err, cudaStream_t s,
                                      int variant = 0, bool pdl = false);

// Host-direct grouped apply of int16 items (serving): each item's hin/hout
// are mapped page-locked host buffers, its quantisation tables and operator
// pieces are in device memory; 128-block tiles, contiguous schedule.
cudaError_t launch_apply_group_host(const GroupItem *d_items, int nitems, int64_t total_halves,
                                    int grid, uint32_t *err, cudaStream_t s);

cudaError_t launch_apply_group(const GroupItem *d_items, const GroupItem *single, int nitems,
                               int64_t total_halves, bool i16, int grid, int max_take,
                               uint32_t *err, cudaStream_t s, bool pdl = false, int variant = 0);

}  // namespace dctf
