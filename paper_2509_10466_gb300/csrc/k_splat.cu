// Coloured point cloud from the inpainted frame and its depth map, and a z-buffered
// point splat of that cloud into an image at another viewpoint.
//
// The paper transplants the inpainted RGB onto the depth measurements ("Point Cloud
// Visualisation"), maps camera points into the viewer's world with a rigid transform
// p' = R p + t ("Perspective Alignment") and draws the cloud with OpenGL; here the draw
// is a headless splat into a device image buffer.  Camera model: pinhole (fx, fy, cx,
// cy), pixel centres at +0.5; a pixel is a point when its depth is finite and > 0.
//
// The projection decides integers (which pixel a point covers and which point wins), so
// every product, sum and quotient is rounded separately in a fixed order (no FMA
// contraction): the result is reproducible bit for bit.  The z-buffer is one 64-bit key
// per output pixel, (depth bits << 32) | point index, lowered with atomicMin: positive
// floats order like their bit patterns, so the nearest point wins and equal depths go to
// the lower index, independent of thread order.
#include "common.cuh"

namespace inpaint {

namespace {

struct Rigid {
  float r[9], t[3];
};

__device__ __forceinline__ void rigid(const Rigid& m, float x, float y, float z, float& ox, float& oy, float& oz) {
  float o[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float a = __fmul_rn(m.r[3 * k], x), b = __fmul_rn(m.r[3 * k + 1], y), c = __fmul_rn(m.r[3 * k + 2], z);
    o[k] = __fadd_rn(__fadd_rn(__fadd_rn(a, b), c), m.t[k]);
  }
  ox = o[0];
  oy = o[1];
  oz = o[2];
}

// points [H*W][6] = world x, y, z (NaN when the depth is not usable), r, g, b
__global__ void point_cloud_kernel(const float* __restrict__ depth, const float* __restrict__ rgb, int H, int W,
                                   float fx, float fy, float cx, float cy, const Rigid m, float* __restrict__ pts) {
  const size_t n = (size_t)H * W;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int v = (int)(i / W), u = (int)(i - (size_t)v * W);
    const float d = depth[i];
    float wx = __int_as_float(0x7fc00000), wy = wx, wz = wx;
    if (d > 0.f && isfinite(d)) {
      const float su = __fsub_rn(__fadd_rn((float)u, 0.5f), cx);
      const float sv = __fsub_rn(__fadd_rn((float)v, 0.5f), cy);
      const float x = __fdiv_rn(__fmul_rn(d, su), fx);
      const float y = __fdiv_rn(__fmul_rn(d, sv), fy);
      rigid(m, x, y, d, wx, wy, wz);
    }
    float* p = pts + i * 6;
    p[0] = wx; p[1] = wy; p[2] = wz;
    p[3] = rgb[i]; p[4] = rgb[n + i]; p[5] = rgb[2 * n + i];
  }
}

__global__ void splat_key_kernel(const float* __restrict__ pts, int64_t N, float fx, float fy, float cx, float cy,
                                 const Rigid m, int Ho, int Wo, unsigned long long* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float* p = pts + i * 6;
    const float x = p[0], y = p[1], z = p[2];
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) continue;
    float qx, qy, qz;
    rigid(m, x, y, z, qx, qy, qz);
    if (!(qz > 1e-3f)) continue;
    const float up = __fadd_rn(__fmul_rn(fx, __fdiv_rn(qx, qz)), cx);
    const float vp = __fadd_rn(__fmul_rn(fy, __fdiv_rn(qy, qz)), cy);
    if (!(up >= 0.f && up < (float)Wo && vp >= 0.f && vp < (float)Ho)) continue;  // also rejects NaN
    const int col = (int)floorf(up), row = (int)floorf(vp);
    const unsigned long long key = ((unsigned long long)__float_as_uint(qz) << 32) | (unsigned long long)(uint32_t)i;
    atomicMin(keys + (size_t)row * Wo + col, key);
  }
}

__global__ void splat_resolve_kernel(const unsigned long long* __restrict__ keys, const float* __restrict__ pts,
                                     int Ho, int Wo, float* __restrict__ img, float* __restrict__ dep,
                                     int32_t* __restrict__ ind) {
  const size_t n = (size_t)Ho * Wo;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[i];
    float r = 0.f, g = 0.f, b = 0.f, z = __int_as_float(0x7f800000);
    int32_t idx = -1;
    if (k != ~0ull) {
      idx = (int32_t)(uint32_t)(k & 0xffffffffull);
      const float* p = pts + (size_t)idx * 6;
      r = p[3]; g = p[4]; b = p[5];
      z = __uint_as_float((uint32_t)(k >> 32));
    }
    img[i] = r;
    img[n + i] = g;
    img[2 * n + i] = b;
    if (dep) dep[i] = z;
    if (ind) ind[i] = idx;
  }
}

unsigned grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  return (unsigned)(g > 65535 ? 65535 : (g ? g : 1));
}

Rigid make_rigid(const float* rt) {
  Rigid m;
  for (int k = 0; k < 9; ++k) m.r[k] = rt[k];
  for (int k = 0; k < 3; ++k) m.t[k] = rt[9 + k];
  return m;
}

}  // namespace

cudaError_t launch_point_cloud(const float* depth, const float* rgb, int H, int W, const float* cam, const float* rt,
                               float* pts, cudaStream_t st) {
  point_cloud_kernel<<<grid_for((size_t)H * W), 256, 0, st>>>(depth, rgb, H, W, cam[0], cam[1], cam[2], cam[3],
                                                               make_rigid(rt), pts);
  return cudaGetLastError();
}

cudaError_t launch_splat(const float* pts, int64_t N, const float* view, const float* rt, int Ho, int Wo,
                         unsigned long long* keys, float* img, float* dep, int32_t* ind, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(keys, 0xff, (size_t)Ho * Wo * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (N > 0)
    splat_key_kernel<<<grid_for((size_t)N), 256, 0, st>>>(pts, N, view[0], view[1], view[2], view[3], make_rigid(rt),
                                                          Ho, Wo, keys);
  splat_resolve_kernel<<<grid_for((size_t)Ho * Wo), 256, 0, st>>>(keys, pts, Ho, Wo, img, dep, ind);
  return cudaGetLastError();
}

}  // namespace inpaint
