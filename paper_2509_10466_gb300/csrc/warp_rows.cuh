// Warp-cooperative row I/O for the tensor-memory epilogues.
//
// A tcgen05.ld of shape 32x32b hands lane i the consecutive columns of accumulator row
// i, so an epilogue thread owns one row.  Storing (or loading) that row directly makes
// every warp instruction touch 32 different rows, 16 bytes each: 32 L1 wavefronts and
// half-used sectors per instruction.  These helpers instead pass each 32-row x 32-column
// block through a 2 KB per-warp shared-memory tile (rows of 64 bytes, 16-byte chunk j of
// row r at slot j ^ ((r >> 1) & 3), which keeps both the row-wise and the column-wise
// phases free of bank conflicts), so that each global instruction covers 8 whole rows
// x 64 bytes.
//
// `base` points at element (0, 0) of the block, `ld` is the row pitch in elements and
// rows >= `nvalid` are neither read (zeros are returned) nor written.  `tile` is the
// warp's 2 KB, 128-byte-aligned staging area.  All 32 lanes must call.
#pragma once
#include "common.cuh"
#include "tc_primitives.cuh"

namespace inpaint {
namespace rows {

constexpr int TILE_BYTES = 32 * 64;

__device__ __forceinline__ int slot(int r, int j) { return r * 64 + ((j ^ ((r >> 1) & 3)) << 4); }

// Two halves of load32_f32, so that the next block's loads can be in flight while the
// current one is processed: issue the coalesced global loads into g ...
__device__ __forceinline__ void load32_issue(const float* base, size_t ld, int nvalid, int lane, float4 (&g)[8]) {
  const int rr = lane >> 2, ch = lane & 3;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int h = i >> 2, r = 8 * (i & 3) + rr;
    g[i] = r < nvalid ? *reinterpret_cast<const float4*>(base + (size_t)r * ld + 16 * h + 4 * ch)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// ... then transpose them through the tile into row `lane`.
__device__ __forceinline__ void load32_finish(uint8_t* tile, int lane, const float4 (&g)[8], float (&v)[32]) {
  const int rr = lane >> 2, ch = lane & 3;
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // columns 16h .. 16h+15
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 4; ++i) *reinterpret_cast<float4*>(tile + slot(8 * i + rr, ch)) = g[4 * h + i];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 t = *reinterpret_cast<const float4*>(tile + slot(lane, j));
      v[16 * h + 4 * j] = t.x; v[16 * h + 4 * j + 1] = t.y; v[16 * h + 4 * j + 2] = t.z; v[16 * h + 4 * j + 3] = t.w;
    }
  }
  __syncwarp();
}

// v = row `lane` of a 32 x 32 FP32 block.
__device__ __forceinline__ void load32_f32(const float* base, size_t ld, int nvalid, uint8_t* tile, int lane,
                                           float (&v)[32]) {
  float4 g[8];
  load32_issue(base, ld, nvalid, lane, g);
  load32_finish(tile, lane, g, v);
}

// Row `lane` of a 32 x 32 FP32 block = v.
__device__ __forceinline__ void store32_f32(float* base, size_t ld, int nvalid, uint8_t* tile, int lane,
                                            const float (&v)[32]) {
  const int rr = lane >> 2, ch = lane & 3;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; ++j)
      *reinterpret_cast<float4*>(tile + slot(lane, j)) =
          make_float4(v[16 * h + 4 * j], v[16 * h + 4 * j + 1], v[16 * h + 4 * j + 2], v[16 * h + 4 * j + 3]);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = 8 * i + rr;
      const float4 t = *reinterpret_cast<const float4*>(tile + slot(r, ch));
      if (r < nvalid) *reinterpret_cast<float4*>(base + (size_t)r * ld + 16 * h + 4 * ch) = t;
    }
  }
  __syncwarp();
}

// Row `lane` of a 32 x 32 block of 16-bit type T = v (rounded to nearest even).
template <typename T>
__device__ __forceinline__ void store32_h16(T* base, size_t ld, int nvalid, uint8_t* tile, int lane,
                                            const float (&v)[32]) {
  const int rr = lane >> 2, ch = lane & 3;
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) w[e] = H16<T>::pack2(v[8 * j + 2 * e], v[8 * j + 2 * e + 1]);
    *reinterpret_cast<uint4*>(tile + slot(lane, j)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = 8 * i + rr;
    const uint4 t = *reinterpret_cast<const uint4*>(tile + slot(r, ch));
    if (r < nvalid) *reinterpret_cast<uint4*>(base + (size_t)r * ld + 8 * ch) = t;
  }
  __syncwarp();
}

// Asynchronous form for the tensor-memory epilogues: the warp stages a 32-row x 64-byte
// box in one of its two tiles (the same swizzle, which is the TMA 64-byte swizzle when
// the tile is 512-byte aligned) and lane 0 hands it to a TMA store; the warp does not
// wait for global memory.  A tile is reused only once the store issued from it two boxes
// earlier has read it.  Rows past the tensor map's extent are not written, and a box with
// no row inside it (nvalid <= 0) is not issued at all; it still commits a (then empty)
// bulk group, so that the group count behind each tile stays the box count.
struct AsyncRows {
  uint8_t* tiles;  // 2 x TILE_BYTES, 512-byte aligned (1024-byte aligned for the wide boxes)
  int k;
  int wide = 0;    // the last store was a wide box over both tiles
};

__device__ __forceinline__ uint8_t* async_acquire(AsyncRows& a, int lane) {
  uint8_t* t = a.tiles + (a.k & 1) * TILE_BYTES;
  ++a.k;
  if (lane == 0) {
    if (a.wide) tc::bulk_wait_read<0>();  // a wide box covers both tiles
    else tc::bulk_wait_read<1>();
  }
  a.wide = 0;
  __syncwarp();
  return t;
}

__device__ __forceinline__ void async_issue(const CUtensorMap* map, const uint8_t* t, int c0, int r0, int nvalid,
                                            int lane) {
  tc::fence_proxy_async_smem();
  __syncwarp();
  if (lane == 0) {
    if (nvalid > 0) tc::tma_store_2d(map, t, c0, r0);
    tc::bulk_commit();  // an empty group when nothing is stored: the tile rotation counts every box
  }
}

// Row `lane` of a 32 x 32 box of 16-bit type T at (column c0, row r0) = v.
template <typename T>
__device__ __forceinline__ void store32_h16_async(const CUtensorMap* map, AsyncRows& a, int c0, int r0, int nvalid,
                                                  int lane, const float (&v)[32]) {
  uint8_t* t = async_acquire(a, lane);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) w[e] = H16<T>::pack2(v[8 * j + 2 * e], v[8 * j + 2 * e + 1]);
    *reinterpret_cast<uint4*>(t + slot(lane, j)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  async_issue(map, t, c0, r0, nvalid, lane);
}

// Row `lane` of a 32 x 32 FP32 block at (column c0, row r0) = v, as two 16-column boxes.
__device__ __forceinline__ void store32_f32_async(const CUtensorMap* map, AsyncRows& a, int c0, int r0, int nvalid,
                                                  int lane, const float (&v)[32]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint8_t* t = async_acquire(a, lane);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      *reinterpret_cast<float4*>(t + slot(lane, j)) =
          make_float4(v[16 * h + 4 * j], v[16 * h + 4 * j + 1], v[16 * h + 4 * j + 2], v[16 * h + 4 * j + 3]);
    async_issue(map, t, c0 + 16 * h, r0, nvalid, lane);
  }
}

// Row `lane` of a 32 x 32 FP32 block at (column c0, row r0) = v, as one box of 32 rows x
// 128 bytes staged over both tiles (128-byte swizzle: 16-byte chunk c of row r at
// c ^ (r % 8); the tiles must be 1024-byte aligned): half the TMA row requests of two
// 64-byte boxes.  Waits until every earlier store of the warp has read its tile.
__device__ __forceinline__ void store32_f32_async_wide(const CUtensorMap* map, AsyncRows& a, int c0, int r0,
                                                       int nvalid, int lane, const float (&v)[32]) {
  if (lane == 0) tc::bulk_wait_read<0>();
  __syncwarp();
  uint8_t* t = a.tiles;
#pragma unroll
  for (int c = 0; c < 8; ++c)
    *reinterpret_cast<float4*>(t + lane * 128 + ((c ^ (lane & 7)) << 4)) =
        make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
  a.wide = 1;
  async_issue(map, t, c0, r0, nvalid, lane);
}

// All of this warp's stores complete (before the CTA exits).
__device__ __forceinline__ void async_drain(int lane) {
  if (lane == 0) tc::bulk_wait<0>();
  __syncwarp();
}

}  // namespace rows
}  // namespace inpaint
