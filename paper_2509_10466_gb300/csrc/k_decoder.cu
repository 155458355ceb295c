// Convolutional decoder and composite.
//
// The paper replaces DSTT's fold-based Vec2Patch with a convolutional reduction and a
// final crop ("Inpainting Model", item "Modified Vec2Patch Algorithm").  Here: two
// stages of nearest x2 upsampling + 3x3 conv (zero padding) + GELU, a 3x3 conv to RGB,
// then the composite out = hole ? pred : x (a select, so known pixels are copied
// bit-exactly) and the crop of the padding back to H x W.
//
// SIMT form: implicit GEMM over (tap, input channel), tiles of 8x8 output pixels by
// 64 output channels; the upsampling is folded into the gather (source row = (y+ky-1)/2).
// All activations are NHWC.
#include "common.cuh"

namespace inpaint {

namespace {

constexpr int TPIX = 64;  // 8x8 output pixels per CTA
constexpr int TCO = 64;   // output channels per CTA
constexpr int KC = 16;    // input channels per step

// out = act(conv3x3(UP ? upsample2(in) : in) + bias); bias may be NULL; act: 0 none,
// 1 GELU; if `preact` is given it also receives the value before the activation.
template <typename T, bool UP>
__global__ void __launch_bounds__(256) upconv_simt_kernel(const T* __restrict__ in, int Hi, int Wi, int Cin,
                                                          const float* __restrict__ wt, const float* __restrict__ bias,
                                                          T* __restrict__ out, int Cout, int act,
                                                          float* __restrict__ preact) {
  __shared__ __align__(16) float As[KC][TPIX];
  __shared__ __align__(16) float Bs[KC][TCO];
  const int Ho = UP ? 2 * Hi : Hi, Wo = UP ? 2 * Wi : Wi;
  const int tilesX = (Wo + 7) / 8;
  const int oy0 = (blockIdx.x / tilesX) * 8, ox0 = (blockIdx.x % tilesX) * 8;
  const int co0 = blockIdx.y * TCO;
  const int b = blockIdx.z;
  const int tid = threadIdx.x;
  const int pg = tid >> 4;  // 4 output pixels: pg*4 .. pg*4+3
  const int cg = tid & 15;  // 4 output channels: cg*4 .. cg*4+3
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  // loader roles: A: pixel lp, channels lc..lc+3; B: channel row lk, output cols lo..lo+3
  const int lp = tid >> 2, lc = (tid & 3) * 4;
  const int lk = tid >> 4, lo = (tid & 15) * 4;
  const int loy = oy0 + (lp >> 3), lox = ox0 + (lp & 7);
  for (int tap = 0; tap < 9; ++tap) {
    const int ky = tap / 3, kx = tap - (tap / 3) * 3;
    const int uy = loy + ky - 1, ux = lox + kx - 1;
    const bool inb = uy >= 0 && uy < Ho && ux >= 0 && ux < Wo;
    const int iy = UP ? (uy >> 1) : uy, ix = UP ? (ux >> 1) : ux;
    const T* src = in + (((size_t)b * Hi + (inb ? iy : 0)) * Wi + (inb ? ix : 0)) * Cin;
    for (int ci0 = 0; ci0 < Cin; ci0 += KC) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int ci = ci0 + lc + c;
        As[lc + c][lp] = (inb && ci < Cin) ? to_f32(src[ci]) : 0.f;
      }
      {
        const int ci = ci0 + lk;
        const float* wr = wt + ((size_t)tap * Cin + ci) * Cout;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int co = co0 + lo + c;
          Bs[lk][lo + c] = (ci < Cin && co < Cout) ? wr[co] : 0.f;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const float4 a = *reinterpret_cast<const float4*>(&As[k][pg * 4]);
        const float4 w = *reinterpret_cast<const float4*>(&Bs[k][cg * 4]);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], wv[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int p = pg * 4 + i;
    const int oy = oy0 + (p >> 3), ox = ox0 + (p & 7);
    if (oy >= Ho || ox >= Wo) continue;
    const size_t pix = ((size_t)b * Ho + oy) * Wo + ox;
    T* dst = out + pix * Cout;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int co = co0 + cg * 4 + j;
      if (co >= Cout) continue;
      const float z = acc[i][j] + (bias ? bias[co] : 0.f);
      if (preact) preact[pix * Cout + co] = z;
      dst[co] = from_f32<T>(act ? gelu_erf(z) : z);
    }
  }
}

// One thread per output pixel of the cropped frame.  wh: [3][C][3][3].
template <typename T>
__global__ void __launch_bounds__(256) head_composite_kernel(const T* __restrict__ in, int Hp, int Wp, int C,
                                                             const float* __restrict__ wh,
                                                             const float* __restrict__ bh,
                                                             const float* __restrict__ x,
                                                             const uint8_t* __restrict__ hole, int H, int W,
                                                             float* __restrict__ out, float* __restrict__ pred) {
  extern __shared__ float wsm[];  // [9][C][3]
  for (int e = threadIdx.x; e < 27 * C; e += blockDim.x) {
    const int o = e % 3, rest = e / 3, c = rest % C, tap = rest / C;
    wsm[e] = wh[((size_t)o * C + c) * 9 + tap];
  }
  __syncthreads();
  const int b = blockIdx.z;
  const int y = blockIdx.y * 16 + (threadIdx.x >> 4);
  const int xx = blockIdx.x * 16 + (threadIdx.x & 15);
  if (y >= H || xx >= W) return;
  float p0 = bh[0], p1 = bh[1], p2 = bh[2];
  for (int tap = 0; tap < 9; ++tap) {
    const int sy = y + tap / 3 - 1, sx = xx + tap % 3 - 1;
    if (sy < 0 || sy >= Hp || sx < 0 || sx >= Wp) continue;
    const T* src = in + (((size_t)b * Hp + sy) * Wp + sx) * C;
    const float* wr = wsm + tap * C * 3;
    for (int c = 0; c < C; ++c) {
      const float v = to_f32(src[c]);
      p0 = fmaf(wr[3 * c + 0], v, p0);
      p1 = fmaf(wr[3 * c + 1], v, p1);
      p2 = fmaf(wr[3 * c + 2], v, p2);
    }
  }
  const size_t HW = (size_t)H * W;
  const size_t q = (size_t)y * W + xx;
  const size_t o = (size_t)b * 3 * HW + q;
  const bool h = hole[(size_t)b * HW + q] != 0;
  out[o] = h ? p0 : x[o];
  out[o + HW] = h ? p1 : x[o + HW];
  out[o + 2 * HW] = h ? p2 : x[o + 2 * HW];
  if (pred) {
    pred[o] = p0;
    pred[o + HW] = p1;
    pred[o + 2 * HW] = p2;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_upconv(const T* in, int B, int Hi, int Wi, int Cin, const float* wt, const float* bias, T* out,
                          int Cout, cudaStream_t st) {
  const int Ho = 2 * Hi, Wo = 2 * Wi;
  dim3 grid(cdiv(Ho, 8) * cdiv(Wo, 8), cdiv(Cout, TCO), B);
  upconv_simt_kernel<T, true><<<grid, 256, 0, st>>>(in, Hi, Wi, Cin, wt, bias, out, Cout, 1, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_conv3x3_f32(const float* in, int B, int Hi, int Wi, int Cin, bool upsample, const float* wt,
                               const float* bias, int act, float* out, float* preact, int Cout, cudaStream_t st) {
  const int Ho = upsample ? 2 * Hi : Hi, Wo = upsample ? 2 * Wi : Wi;
  dim3 grid(cdiv(Ho, 8) * cdiv(Wo, 8), cdiv(Cout, TCO), B);
  if (upsample)
    upconv_simt_kernel<float, true><<<grid, 256, 0, st>>>(in, Hi, Wi, Cin, wt, bias, out, Cout, act, preact);
  else
    upconv_simt_kernel<float, false><<<grid, 256, 0, st>>>(in, Hi, Wi, Cin, wt, bias, out, Cout, act, preact);
  return cudaGetLastError();
}
template cudaError_t launch_upconv<float>(const float*, int, int, int, int, const float*, const float*, float*, int,
                                          cudaStream_t);
template cudaError_t launch_upconv<bf16>(const bf16*, int, int, int, int, const float*, const float*, bf16*, int,
                                         cudaStream_t);

template <typename T>
cudaError_t launch_head_composite(const T* in, int B, int Hp, int Wp, int C, const float* wh, const float* bh,
                                  const float* x, const uint8_t* hole, int H, int W, float* out, float* pred,
                                  cudaStream_t st) {
  dim3 grid(cdiv(W, 16), cdiv(H, 16), B);
  head_composite_kernel<T><<<grid, 256, 27 * C * sizeof(float), st>>>(in, Hp, Wp, C, wh, bh, x, hole, H, W, out,
                                                                      pred);
  return cudaGetLastError();
}
template cudaError_t launch_head_composite<float>(const float*, int, int, int, int, const float*, const float*,
                                                  const float*, const uint8_t*, int, int, float*, float*,
                                                  cudaStream_t);
template cudaError_t launch_head_composite<bf16>(const bf16*, int, int, int, int, const float*, const float*,
                                                 const float*, const uint8_t*, int, int, float*, float*,
                                                 cudaStream_t);

}  // namespace inpaint
