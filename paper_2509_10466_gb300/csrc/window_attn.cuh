// Mask-aware window attention of one warp's 16 query rows, shared by the attention kernels
// of the 16-bit forms (tensor cores: mma.sync m16n8k16 with FP32 accumulation).
//
// A window is 8 x 8 token slots; its Q, K and V head slices (64 slots x 32 channels) sit in
// shared memory in 64-byte rows with the 64-byte swizzle (16-byte chunk c of slot row r at
// c ^ ((r >> 1) & 3)), the layout of a TMA box.  Keys are the slots whose bit is set in
// `keymask`; the scores are scaled by 1 / sqrt(32), plus the relative-position bias when
// RP, masked, and normalized with a base-2 softmax in FP32 (row maxima by quad shuffles);
// O = P V with P rounded to the operand type, its row sums taken by one more MMA against
// ones.  Every query row must have a usable key (keymask != 0).
#pragma once
#include "common.cuh"

namespace inpaint {

constexpr int WA_SLOTS = 64;  // slots of an 8 x 8 window
constexpr int WA_DH = 32;     // head dim
constexpr float LOG2E = 1.4426950408889634f;

template <bool B>
struct BoolTag {
  static constexpr bool value = B;
};

__device__ __forceinline__ uint32_t swz64(int row, int chunk) {
  return (uint32_t)(row * 64 + ((chunk ^ ((row >> 1) & 3)) << 4));
}

// Relative-position bias of query slot s and key slot k: table[(ky - sy + 7) * 15 + (kx - sx + 7)].
__device__ __forceinline__ int relpos_index(int s, int k) { return ((k >> 3) - (s >> 3) + 7) * 15 + ((k & 7) - (s & 7) + 7); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// Query rows r0 .. r0 + 15 of a window (one warp, `lane` = lane id): the output rows pass
// through the warp's own Q rows and leave as 16-byte chunks to o + stok[slot] * ld_o + col0
// for the slots with stok >= 0.  rp: the head's [225] bias table (RP only).
template <bool RP, typename T>
__device__ __forceinline__ void window_attention_rows(uint8_t* Qt, const uint8_t* Kt, const uint8_t* Vt,
                                                      unsigned long long keymask, const float* rp, const int* stok,
                                                      T* __restrict__ o, size_t ld_o, int col0, int r0, int lane) {
  const int g = lane >> 2, tq = lane & 3;
  // ---- S = Q K^T
  uint32_t qa[2][4];
  {
    const int row = r0 + (lane & 15);
    ldsm_x4(qa[0], Qt + swz64(row, lane >> 4));
    ldsm_x4(qa[1], Qt + swz64(row, 2 + (lane >> 4)));
  }
  float sc[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    sc[j][0] = sc[j][1] = sc[j][2] = sc[j][3] = 0.f;
    uint32_t kb[4];  // (k 0-7, 8-15) of k-step 0 and (16-23, 24-31) of k-step 1, keys 8j .. 8j+7
    ldsm_x4(kb, Kt + swz64(8 * j + (lane & 7), lane >> 3));
    mma16816<T>(sc[j], qa[0], kb[0], kb[1]);
    mma16816<T>(sc[j], qa[1], kb[2], kb[3]);
  }
  // ---- masked softmax (rows g and g+8 of this warp's 16), FP32, base 2.  Without the
  // relative-position bias the maxima are taken on the raw scores (the scale is positive)
  // and the scale enters with the maximum in one FMA in the exponent.
  const float sl2 = 1.4426950408889634f / sqrtf((float)WA_DH);  // scale * log2(e)
  const unsigned long long km = keymask >> (2 * tq);  // bit 8j + c: key 8j + 2tq + c
  float mx0 = -INFINITY, mx1 = -INFINITY;
  auto mask_and_max = [&](auto masked) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const bool okk = (km >> (8 * j + c)) & 1ull;
        if constexpr (RP) {
          const int key = 8 * j + 2 * tq + c;
          const float bb0 = rp[relpos_index(r0 + g, key)] * LOG2E;
          const float bb1 = rp[relpos_index(r0 + g + 8, key)] * LOG2E;
          sc[j][c] = okk ? fmaf(sc[j][c], sl2, bb0) : -INFINITY;
          sc[j][2 + c] = okk ? fmaf(sc[j][2 + c], sl2, bb1) : -INFINITY;
        } else if constexpr (decltype(masked)::value) {
          sc[j][c] = okk ? sc[j][c] : -INFINITY;
          sc[j][2 + c] = okk ? sc[j][2 + c] : -INFINITY;
        }
        mx0 = fmaxf(mx0, sc[j][c]);
        mx1 = fmaxf(mx1, sc[j][2 + c]);
      }
    }
  };
  // a window whose 64 keys are all usable (most of a frame) skips the selects
  if (RP || keymask != ~0ull) mask_and_max(BoolTag<true>{});
  else mask_and_max(BoolTag<false>{});
  mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, 1));
  mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, 2));
  mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, 1));
  mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, 2));
  // every row has a usable key (keymask != 0), so the maxima are finite
  const float sx = RP ? 1.f : sl2;
  const float o0 = -mx0 * sx, o1 = -mx1 * sx;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      sc[j][c] = ex2_approx(fmaf(sc[j][c], sx, o0));
      sc[j][2 + c] = ex2_approx(fmaf(sc[j][2 + c], sx, o1));
    }
  }
  // ---- O = P V, and the row sums of the 16-bit P as one more MMA against ones (FP32
  // accumulation; every column of `ls` holds its row's sum, so no shuffles)
  float oc[4][4], ls[4] = {0.f, 0.f, 0.f, 0.f};
  const uint32_t ones = H16<T>::pack2(1.f, 1.f);
#pragma unroll
  for (int j = 0; j < 4; ++j) oc[j][0] = oc[j][1] = oc[j][2] = oc[j][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {  // keys 16kk .. 16kk+15
    uint32_t pa[4];
    pa[0] = H16<T>::pack2(sc[2 * kk][0], sc[2 * kk][1]);
    pa[1] = H16<T>::pack2(sc[2 * kk][2], sc[2 * kk][3]);
    pa[2] = H16<T>::pack2(sc[2 * kk + 1][0], sc[2 * kk + 1][1]);
    pa[3] = H16<T>::pack2(sc[2 * kk + 1][2], sc[2 * kk + 1][3]);
#pragma unroll
    for (int nn = 0; nn < 2; ++nn) {  // head dims 16nn .. 16nn+15
      uint32_t vb[4];
      ldsm_x4_t(vb, Vt + swz64(16 * kk + (lane & 7) + ((lane >> 3) & 1) * 8, 2 * nn + (lane >> 4)));
      mma16816<T>(oc[2 * nn], pa, vb[0], vb[1]);
      mma16816<T>(oc[2 * nn + 1], pa, vb[2], vb[3]);
    }
    mma16816<T>(ls, pa, ones, ones);
  }
  const float inv0 = 1.f / ls[0], inv1 = 1.f / ls[2];
  __syncwarp();
  // stage this warp's 16 output rows in its own Q rows, then store 16-byte chunks
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    *reinterpret_cast<uint32_t*>(Qt + swz64(r0 + g, j) + 4 * tq) = H16<T>::pack2(oc[j][0] * inv0, oc[j][1] * inv0);
    *reinterpret_cast<uint32_t*>(Qt + swz64(r0 + g + 8, j) + 4 * tq) = H16<T>::pack2(oc[j][2] * inv1, oc[j][3] * inv1);
  }
  __syncwarp();
#pragma unroll
  for (int e = lane; e < 16 * 4; e += 32) {
    const int sl = r0 + (e >> 2), ch = e & 3;
    const int t = stok[sl];
    if (t >= 0)
      *reinterpret_cast<uint4*>(o + (size_t)t * ld_o + col0 + ch * 8) =
          *reinterpret_cast<const uint4*>(Qt + swz64(sl, ch));
  }
}

}  // namespace inpaint

