// GPU pre/post-processing around the half-resolution inpainting pass.
//
// The paper runs segmentation and inpainting at half resolution (640x360) and scales
// the outputs by 2 to 1280x720 ("Upscaling"); the processing server builds the hole
// from the masks of the objects the user selected ("Object Control"), and the paper
// names the CPU pre/post processing as the bottleneck it would move to the GPU
// (Future Work).  Readings used here:
//   hole_half[b,i,j] = OR over selected objects k of (mask[b,k,i,j] != 0)    (integer)
//   x_half[b,c,i,j]  = mean of the 2x2 full-resolution pixels (fixed summation order)
//   out[b,c,y,x]     = hole_half[b,y/2,x/2] ? pred_half[b,c,y/2,x/2] : x[b,c,y,x]
// i.e. nearest x2 upscaling of both the prediction and the hole (the "slight
// pixelation" and "jagged outlines" the paper reports), and known full-resolution
// pixels copied exactly.
#include "common.cuh"

namespace inpaint {

namespace {

__global__ void mask_union_kernel(const uint8_t* __restrict__ masks, const uint8_t* __restrict__ selected, int B,
                                  int K, int h, int w, uint8_t* __restrict__ hole) {
  const size_t hw = (size_t)h * w, n = (size_t)B * hw;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / hw, p = i - b * hw;
    uint8_t v = 0;
    for (int k = 0; k < K; ++k)
      if (selected[b * K + k] && masks[(b * K + k) * hw + p]) v = 1;
    hole[i] = v;
  }
}

__global__ void downscale2_kernel(const float* __restrict__ x, int B, int H, int W, float* __restrict__ xh) {
  const int h = H / 2, w = W / 2;
  const size_t n = (size_t)B * 3 * h * w;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % w);
    const int r = (int)((i / w) % h);
    const size_t bc = i / ((size_t)w * h);
    const float* s = x + bc * H * W + (size_t)(2 * r) * W + 2 * j;
    xh[i] = 0.25f * ((s[0] + s[1]) + (s[W] + s[W + 1]));
  }
}

__global__ void upscale_composite_kernel(const float* __restrict__ pred_h, const uint8_t* __restrict__ hole_h,
                                         const float* __restrict__ x, int B, int H, int W, float* __restrict__ out) {
  const int h = H / 2, w = W / 2;
  const size_t HW = (size_t)H * W, n = (size_t)B * HW;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int xx = (int)(i % W);
    const int y = (int)((i / W) % H);
    const size_t b = i / HW;
    const size_t q = (size_t)(y >> 1) * w + (xx >> 1);
    const bool hl = hole_h[b * h * w + q] != 0;
    const size_t o = b * 3 * HW + (size_t)y * W + xx;
    const size_t oh = b * 3 * (size_t)h * w + q;
#pragma unroll
    for (int c = 0; c < 3; ++c) out[o + c * HW] = hl ? pred_h[oh + c * (size_t)h * w] : x[o + c * HW];
  }
}

unsigned grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  return (unsigned)(g > 65535 ? 65535 : (g ? g : 1));
}

}  // namespace

cudaError_t launch_mask_union(const uint8_t* masks, const uint8_t* selected, int B, int K, int h, int w, uint8_t* hole,
                              cudaStream_t st) {
  mask_union_kernel<<<grid_for((size_t)B * h * w), 256, 0, st>>>(masks, selected, B, K, h, w, hole);
  return cudaGetLastError();
}

cudaError_t launch_downscale2(const float* x, int B, int H, int W, float* xh, cudaStream_t st) {
  downscale2_kernel<<<grid_for((size_t)B * 3 * (H / 2) * (W / 2)), 256, 0, st>>>(x, B, H, W, xh);
  return cudaGetLastError();
}

cudaError_t launch_upscale_composite(const float* pred_h, const uint8_t* hole_h, const float* x, int B, int H, int W,
                                     float* out, cudaStream_t st) {
  upscale_composite_kernel<<<grid_for((size_t)B * H * W), 256, 0, st>>>(pred_h, hole_h, x, B, H, W, out);
  return cudaGetLastError();
}

}  // namespace inpaint
