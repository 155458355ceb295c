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

// Tiled form for 16-bit activations (T = bf16 or f16): a CTA computes 16 x 32 output pixels of one frame
// from an 18 x 34 x C halo tile staged in shared memory with 16-byte loads (chunk
// index XOR-swizzled by pixel so that neighbouring threads hit different banks).
// Requires C % 8 == 0.
template <typename T>
__global__ void __launch_bounds__(256) head_tile_kernel(const T* __restrict__ in, int Hp, int Wp, int C,
                                                        const float* __restrict__ wh, const float* __restrict__ bh,
                                                        const float* __restrict__ x, const uint8_t* __restrict__ hole,
                                                        int H, int W, float* __restrict__ out,
                                                        float* __restrict__ pred) {
  extern __shared__ __align__(16) uint8_t hsm[];
  constexpr int TY = 16, TX = 32, HY = TY + 2, HX = TX + 2;
  const int nch = C >> 3;
  const int swz = (nch & (nch - 1)) == 0 ? nch - 1 : 0;
  T* tile = reinterpret_cast<T*>(hsm);                                         // [HY*HX][C]
  float* wsm = reinterpret_cast<float*>(hsm + (size_t)HY * HX * C * 2);        // [9][C][3]
  const int b = blockIdx.z, y0 = blockIdx.y * TY, x0 = blockIdx.x * TX;
  for (int e = threadIdx.x; e < 27 * C; e += blockDim.x) {
    const int o = e % 3, rest = e / 3, c = rest % C, tap = rest / C;
    wsm[e] = wh[((size_t)o * C + c) * 9 + tap];
  }
  for (int e = threadIdx.x; e < HY * HX * nch; e += blockDim.x) {
    const int k = e % nch, pix = e / nch;
    const int hy = pix / HX, hx = pix - (pix / HX) * HX;
    const int sy = y0 - 1 + hy, sx = x0 - 1 + hx;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (sy >= 0 && sy < Hp && sx >= 0 && sx < Wp)
      v = *reinterpret_cast<const uint4*>(in + (((size_t)b * Hp + sy) * Wp + sx) * C + 8 * k);
    *reinterpret_cast<uint4*>(tile + (size_t)pix * C + 8 * (k ^ (pix & swz))) = v;
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, ty0 = threadIdx.x >> 5;
  const size_t HW = (size_t)H * W;
#pragma unroll 1
  for (int rr = 0; rr < 2; ++rr) {
    const int ty = ty0 + 8 * rr;
    const int y = y0 + ty, xx = x0 + tx;
    if (y >= H || xx >= W) continue;
    float p0 = bh[0], p1 = bh[1], p2 = bh[2];
    for (int tap = 0; tap < 9; ++tap) {
      const int pix = (ty + tap / 3) * HX + tx + tap % 3;
      const T* src = tile + (size_t)pix * C;
      const float* wr = wsm + tap * C * 3;
      for (int k = 0; k < nch; ++k) {
        const uint4 raw = *reinterpret_cast<const uint4*>(src + 8 * (k ^ (pix & swz)));
        const uint32_t h2[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 f = H16<T>::unpack2(h2[q]);
          const float* w0 = wr + 3 * (8 * k + 2 * q);
          p0 = fmaf(w0[0], f.x, p0); p1 = fmaf(w0[1], f.x, p1); p2 = fmaf(w0[2], f.x, p2);
          p0 = fmaf(w0[3], f.y, p0); p1 = fmaf(w0[4], f.y, p1); p2 = fmaf(w0[5], f.y, p2);
        }
      }
    }
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
}

// Tensor-core form of the head for 16-bit activations with C % 16 == 0 (C <= 64):
// out(16 x 32 pixel tile) = conv3x3 as an implicit GEMM with M = 16 pixels of a row,
// K = 9 taps x C channels, N = 8 (3 used) on mma.sync m16n8k16.  The 18 x 34 x C halo
// tile is staged in shared memory with 16-byte chunks XOR-swizzled by pixel; A fragments
// come from ldmatrix.  The CTA turns the weights into the 16-bit B fragments once, in shared
// memory, from which every warp reads its lane's.  Each warp owns two output rows (4
// m-tiles); the three predicted channels then go through shared memory (over the halo
// tile) so that bias, composite and crop run over whole rows with 16-byte accesses.
__device__ __forceinline__ void ldsm_x4_h(uint32_t (&r)[4], const void* p) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
template <int C, typename T>
__global__ void __launch_bounds__(256) head_mma_kernel(const T* __restrict__ in, int Hp, int Wp,
                                                       const float* __restrict__ wh, const float* __restrict__ bh,
                                                       const float* __restrict__ x, const uint8_t* __restrict__ hole,
                                                       int H, int W, float* __restrict__ out,
                                                       float* __restrict__ pred, int vec) {
  constexpr int TY = 16, TX = 32, HY = TY + 2, HX = TX + 2, NCH = C / 8, KC = C / 16;
  constexpr int NFRAG = 9 * KC * 2;  // B fragments per lane: (tap, kc, half)
  extern __shared__ __align__(16) uint8_t hsm[];
  T* tile = reinterpret_cast<T*>(hsm);  // [HY*HX][C], chunk k of pixel p at 8*(k ^ (p & (NCH-1)))
  __shared__ uint32_t sfrag[NFRAG][32];  // 16-bit pairs, per lane
  // predictions of the tile with the bias added, over the halo tile once the MMAs are done
  float(*spred)[TY][TX] = reinterpret_cast<float(*)[TY][TX]>(hsm);
  static_assert(3 * TY * TX * 4 <= HY * HX * C * 2, "prediction tile exceeds the halo tile");
  const int b = blockIdx.z, y0 = blockIdx.y * TY, x0 = blockIdx.x * TX;
  pdl_trigger();
  pdl_wait();
  // halo tile by cp.async, all copies in flight at once (zero fill outside the image)
  for (int e = threadIdx.x; e < HY * HX * NCH; e += blockDim.x) {
    const int k = e % NCH, pix = e / NCH;
    const int hy = pix / HX, hx = pix - (pix / HX) * HX;
    const int sy = y0 - 1 + hy, sx = x0 - 1 + hx;
    const bool inside = sy >= 0 && sy < Hp && sx >= 0 && sx < Wp;
    const T* src = in + (((size_t)b * Hp + (inside ? sy : 0)) * Wp + (inside ? sx : 0)) * C + 8 * k;
    const uint32_t dst = static_cast<uint32_t>(
        __cvta_generic_to_shared(tile + (size_t)pix * C + 8 * (k ^ (pix & (NCH - 1)))));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(inside ? 16 : 0)
                 : "memory");
  }
  // B fragment (tap, kc, half) of lane (g, tq): rows k = channels kc*16 + half*8 + 2tq, +1 of
  // that tap, column n = output channel g (zero for g >= 3)
  for (int e = threadIdx.x; e < NFRAG * 32; e += blockDim.x) {
    const int f = e >> 5, ln = e & 31, fg = ln >> 2, ftq = ln & 3;
    const int tap = f / (KC * 2), kc = (f / 2) % KC, hlf = f & 1;
    const int c0 = kc * 16 + hlf * 8 + 2 * ftq;
    const float w0 = fg < 3 ? __ldg(wh + (fg * C + c0) * 9 + tap) : 0.f;
    const float w1 = fg < 3 ? __ldg(wh + (fg * C + c0 + 1) * 9 + tap) : 0.f;
    sfrag[f][ln] = H16<T>::pack2(w0, w1);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
  uint32_t bw[9][KC][2];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap)
#pragma unroll
    for (int kc = 0; kc < KC; ++kc)
#pragma unroll
      for (int hlf = 0; hlf < 2; ++hlf) bw[tap][kc][hlf] = sfrag[(tap * KC + kc) * 2 + hlf][lane];
  const float bias0 = bh[0], bias1 = bh[1], bias2 = bh[2];
  float acc[4][4];
#pragma unroll
  for (int mt = 0; mt < 4; ++mt) {
    const int ty = 2 * warp + (mt >> 1), xs = (mt & 1) * 16;  // output row / first column of this m-tile
    acc[mt][0] = acc[mt][1] = acc[mt][2] = acc[mt][3] = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int pix = (ty + tap / 3) * HX + xs + tap % 3 + (lane & 15);
#pragma unroll
      for (int kc = 0; kc < KC; ++kc) {
        const int chunk = 2 * kc + (lane >> 4);
        uint32_t a[4];
        ldsm_x4_h(a, tile + (size_t)pix * C + 8 * (chunk ^ (pix & (NCH - 1))));
        mma16816<T>(acc[mt], a, bw[tap][kc][0], bw[tap][kc][1]);
      }
    }
  }
  __syncthreads();  // every warp is done with the halo tile
#pragma unroll
  for (int mt = 0; mt < 4; ++mt) {
    const int ty = 2 * warp + (mt >> 1), xs = (mt & 1) * 16;
    // accumulator rows g, g + 8 = pixels xs + g, xs + g + 8; columns 2tq, 2tq + 1 = channels
    if (tq == 0) {
      spred[0][ty][xs + g] = acc[mt][0] + bias0;
      spred[1][ty][xs + g] = acc[mt][1] + bias1;
      spred[0][ty][xs + g + 8] = acc[mt][2] + bias0;
      spred[1][ty][xs + g + 8] = acc[mt][3] + bias1;
    } else if (tq == 1) {
      spred[2][ty][xs + g] = acc[mt][0] + bias2;
      spred[2][ty][xs + g + 8] = acc[mt][2] + bias2;
    }
  }
  __syncthreads();
  // composite and crop: out = hole ? pred : x, rows of the tile, four pixels per thread step
  const size_t HW = (size_t)H * W;
  for (int e = threadIdx.x; e < 3 * TY * (TX / 4); e += blockDim.x) {
    const int ch = e / (TY * (TX / 4)), r = (e / (TX / 4)) % TY, x4 = 4 * (e % (TX / 4));
    const int y = y0 + r, xx = x0 + x4;
    if (y >= H || xx >= W) continue;
    const size_t q = (size_t)y * W + xx;
    const size_t o = (size_t)b * 3 * HW + (size_t)ch * HW + q;
    const float* pv = &spred[ch][r][x4];
    if (vec && xx + 4 <= W) {  // 16-byte aligned: W % 4 == 0 and aligned bases
      const uchar4 hm = *reinterpret_cast<const uchar4*>(hole + (size_t)b * HW + q);
      const float4 xv = *reinterpret_cast<const float4*>(x + o);
      const float4 p4 = *reinterpret_cast<const float4*>(pv);
      *reinterpret_cast<float4*>(out + o) =
          make_float4(hm.x ? p4.x : xv.x, hm.y ? p4.y : xv.y, hm.z ? p4.z : xv.z, hm.w ? p4.w : xv.w);
      if (pred) *reinterpret_cast<float4*>(pred + o) = p4;
    } else {
      for (int k = 0; k < 4 && xx + k < W; ++k) {
        const bool h = hole[(size_t)b * HW + q + k] != 0;
        out[o + k] = h ? pv[k] : x[o + k];
        if (pred) pred[o + k] = pv[k];
      }
    }
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
template cudaError_t launch_upconv<f16>(const f16*, int, int, int, int, const float*, const float*, f16*, int,
                                        cudaStream_t);

template <typename T>
cudaError_t launch_head_composite(const T* in, int B, int Hp, int Wp, int C, const float* wh, const float* bh,
                                  const float* x, const uint8_t* hole, int H, int W, float* out, float* pred,
                                  cudaStream_t st) {
  if constexpr (sizeof(T) == 2) {
    if (C == 16 || C == 32 || C == 64) {
      const size_t smem = (size_t)18 * 34 * C * 2;
      static size_t attr = 0;
      if (C == 64 && smem > attr) {
        cudaError_t e =
            cudaFuncSetAttribute(head_mma_kernel<64, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
      }
      dim3 grid(cdiv(W, 32), cdiv(H, 16), B);
      // whole-row 16-byte accesses of x, out, pred (and 4-byte of the hole mask) when aligned
      const int vec = W % 4 == 0 && ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(out) |
                                      reinterpret_cast<uintptr_t>(pred) | reinterpret_cast<uintptr_t>(hole)) &
                                     15) == 0;
      if (C == 16)
        return launch_pdl(head_mma_kernel<16, T>, grid, dim3(256), smem, st, in, Hp, Wp, wh, bh, x, hole, H, W, out,
                          pred, vec);
      if (C == 32)
        return launch_pdl(head_mma_kernel<32, T>, grid, dim3(256), smem, st, in, Hp, Wp, wh, bh, x, hole, H, W, out,
                          pred, vec);
      return launch_pdl(head_mma_kernel<64, T>, grid, dim3(256), smem, st, in, Hp, Wp, wh, bh, x, hole, H, W, out,
                        pred, vec);
    }
    if (C % 8 == 0) {
      const size_t smem = (size_t)18 * 34 * C * 2 + (size_t)27 * C * 4;
      static size_t attr = 0;
      if (smem > attr) {
        cudaError_t e =
            cudaFuncSetAttribute(head_tile_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
      }
      dim3 grid(cdiv(W, 32), cdiv(H, 16), B);
      head_tile_kernel<T><<<grid, 256, smem, st>>>(in, Hp, Wp, C, wh, bh, x, hole, H, W, out, pred);
      return cudaGetLastError();
    }
  }
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
template cudaError_t launch_head_composite<f16>(const f16*, int, int, int, int, const float*, const float*,
                                                const float*, const uint8_t*, int, int, float*, float*,
                                                cudaStream_t);

}  // namespace inpaint
