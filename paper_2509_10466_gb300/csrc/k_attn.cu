// Mask-aware window attention with the token-mask update.
//
// Attention is plain scaled dot-product attention ("Inpainting Model", item
// "Distinct Transformer Blocks"), computed inside 8x8-token windows.  Keys are the
// tokens whose mask bit is set; a window with no such key is skipped (its outputs are
// 0) and a window with at least one becomes valid as a whole:
//   v_out[t] = OR over t's window of v_in.
// The integer part is exact.  Windows of odd blocks are offset by half a window; their
// slots outside the token grid are void.
//
// SIMT form: one CTA per (window, head, frame), one thread per window slot.  K and V
// of the window's usable keys are staged in shared memory; each query thread runs a
// two-pass softmax (max, then exp-sum and weighted V) in FP32.
#include "common.cuh"

namespace inpaint {

namespace {

constexpr int WS = 8;      // window side
constexpr int SLOTS = 64;  // WS * WS
constexpr int DH = 32;     // head dim

template <typename T>
__global__ void __launch_bounds__(SLOTS) attn_simt_kernel(const T* __restrict__ qkv, const uint8_t* __restrict__ v_in,
                                                          T* __restrict__ o, uint8_t* __restrict__ v_out, int Ht,
                                                          int Wt, int d, int offset, int nwx) {
  __shared__ float Ks[SLOTS][DH + 1];
  __shared__ float Vs[SLOTS][DH + 1];
  __shared__ int okS[SLOTS];
  const int w = blockIdx.x, h = blockIdx.y, b = blockIdx.z;
  const int wy = w / nwx, wx = w - (w / nwx) * nwx;
  const int s = threadIdx.x;
  const int ty = wy * WS - offset + (s >> 3), tx = wx * WS - offset + (s & 7);
  const bool real = ty >= 0 && ty < Ht && tx >= 0 && tx < Wt;
  const size_t Nt = (size_t)Ht * Wt;
  const size_t t = real ? (size_t)b * Nt + (size_t)ty * Wt + tx : 0;
  const bool ok = real && v_in[t] != 0;
  okS[s] = ok;
  const T* row = qkv + t * 3 * d;
#pragma unroll 8
  for (int i = 0; i < DH; ++i) {
    Ks[s][i] = ok ? to_f32(row[d + h * DH + i]) : 0.f;
    Vs[s][i] = ok ? to_f32(row[2 * d + h * DH + i]) : 0.f;
  }
  const int any = __syncthreads_or(ok);
  if (!real) return;
  T* orow = o + t * d + h * DH;
  if (!any) {
#pragma unroll 8
    for (int i = 0; i < DH; ++i) orow[i] = from_f32<T>(0.f);
    if (h == 0) v_out[t] = 0;
    return;
  }
  if (h == 0) v_out[t] = 1;
  float q[DH];
#pragma unroll
  for (int i = 0; i < DH; ++i) q[i] = to_f32(row[h * DH + i]);
  const float scale = 1.0f / sqrtf((float)DH);
  float mx = -INFINITY;
  for (int k = 0; k < SLOTS; ++k) {
    if (!okS[k]) continue;
    float sc = 0.f;
#pragma unroll
    for (int i = 0; i < DH; ++i) sc = fmaf(q[i], Ks[k][i], sc);
    mx = fmaxf(mx, sc * scale);
  }
  float l = 0.f, acc[DH];
#pragma unroll
  for (int i = 0; i < DH; ++i) acc[i] = 0.f;
  for (int k = 0; k < SLOTS; ++k) {
    if (!okS[k]) continue;
    float sc = 0.f;
#pragma unroll
    for (int i = 0; i < DH; ++i) sc = fmaf(q[i], Ks[k][i], sc);
    const float p = expf(sc * scale - mx);
    l += p;
#pragma unroll
    for (int i = 0; i < DH; ++i) acc[i] = fmaf(p, Vs[k][i], acc[i]);
  }
  const float inv = 1.f / l;
#pragma unroll
  for (int i = 0; i < DH; ++i) orow[i] = from_f32<T>(acc[i] * inv);
}

}  // namespace

template <typename T>
cudaError_t launch_attention(const T* qkv, const uint8_t* v_in, T* o, uint8_t* v_out, int B, int Ht, int Wt, int d,
                             int heads, int offset, cudaStream_t st) {
  const int nwy = (Ht + offset + WS - 1) / WS, nwx = (Wt + offset + WS - 1) / WS;
  dim3 grid(nwy * nwx, heads, B);
  attn_simt_kernel<T><<<grid, SLOTS, 0, st>>>(qkv, v_in, o, v_out, Ht, Wt, d, offset, nwx);
  return cudaGetLastError();
}

template cudaError_t launch_attention<float>(const float*, const uint8_t*, float*, uint8_t*, int, int, int, int, int,
                                             int, cudaStream_t);
template cudaError_t launch_attention<bf16>(const bf16*, const uint8_t*, bf16*, uint8_t*, int, int, int, int, int,
                                            int, cudaStream_t);

}  // namespace inpaint
