// Patch embedding with token-mask init, LayerNorm, and the hole-L1 loss.
//
// Patch embedding: the model input is the frame with its masked regions set to 0 plus
// the known-pixel mask ("Inpainting Manager": the model accepts a frame with masked
// regions set to 0); a 4x4 stride-4 convolution turns it into tokens.  Because the
// patches do not overlap this is a GEMM over 64-value patches; with K = 64 it is
// HBM-bound (13 B/pixel in, 4d B/token out), so it runs on the SIMT pipes.
#include "common.cuh"

namespace inpaint {

namespace {

constexpr int EMB_TOK = 32;  // tokens per CTA: warp w owns tokens w, w+8, w+16, w+24

__device__ __forceinline__ float warp_sum(float v);

// we_t: embedding weights transposed to [64][d] (k = c*16 + i*4 + j), read as float4 from
// L1.  Lane l owns channels 8l .. 8l+7 (looping in steps of 256 channels), so a token's
// row is spread over one warp and its LayerNorm is a warp reduction.  With ln_out set,
// also writes LayerNorm(tok) (FP32 statistics) in the 16-bit type T.
template <typename T>
__global__ void __launch_bounds__(256) embed_kernel(const float* __restrict__ x, const uint8_t* __restrict__ hole,
                                                    int H, int W, int Ht, int Wt,
                                                    const float* __restrict__ we_t, const float* __restrict__ be,
                                                    int d, float* __restrict__ tok, uint8_t* __restrict__ v0,
                                                    const float* __restrict__ ln_g, const float* __restrict__ ln_b,
                                                    T* __restrict__ ln_out) {
  __shared__ float P[64][EMB_TOK + 1];
  __shared__ int known_any[EMB_TOK];
  const int b = blockIdx.y;
  const int t0 = blockIdx.x * EMB_TOK;
  const int Nt = Ht * Wt;
  const size_t HW = (size_t)H * W;
  if (threadIdx.x < EMB_TOK) known_any[threadIdx.x] = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < EMB_TOK * 16; e += blockDim.x) {
    const int tl = e >> 4, pix = e & 15;
    const int t = t0 + tl;
    float r = 0.f, g = 0.f, bl = 0.f, m = 0.f;
    if (t < Nt) {
      const int ty = t / Wt, tx = t - (t / Wt) * Wt;
      const int y = ty * 4 + (pix >> 2), xx = tx * 4 + (pix & 3);
      if (y < H && xx < W) {
        const size_t q = (size_t)y * W + xx;
        if (hole[(size_t)b * HW + q] == 0) {   // known pixel: keep it; hole pixels enter as 0
          const float* xb = x + (size_t)b * 3 * HW + q;
          r = xb[0]; g = xb[HW]; bl = xb[2 * HW];
          m = 1.f;
        }
      }
    }
    P[pix][tl] = r;
    P[16 + pix][tl] = g;
    P[32 + pix][tl] = bl;
    P[48 + pix][tl] = m;
    if (m != 0.f) known_any[tl] = 1;  // every writer stores the same value
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c0 = 8 * lane; c0 < d; c0 += 256) {
    float acc[4][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float bj = be[c0 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i][j] = bj;
    }
#pragma unroll 8
    for (int k = 0; k < 64; ++k) {
      const float4 wa = __ldg(reinterpret_cast<const float4*>(we_t + (size_t)k * d + c0));
      const float4 wb = __ldg(reinterpret_cast<const float4*>(we_t + (size_t)k * d + c0 + 4));
      const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float pv = P[k][warp + 8 * i];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(wv[j], pv, acc[i][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int t = t0 + warp + 8 * i;
      if (t >= Nt) continue;
      float4* dst = reinterpret_cast<float4*>(tok + ((size_t)b * Nt + t) * d + c0);
      dst[0] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      dst[1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
  }
  if (threadIdx.x < EMB_TOK && t0 + (int)threadIdx.x < Nt)
    v0[(size_t)b * Nt + t0 + threadIdx.x] = (uint8_t)known_any[threadIdx.x];
  if (!ln_out) return;
  // LayerNorm of the 4 tokens of this warp (rows just written by this warp)
  __syncwarp();
  for (int i = 0; i < 4; ++i) {
    const int t = t0 + warp + 8 * i;
    if (t >= Nt) continue;  // uniform across the warp
    const float* row = tok + ((size_t)b * Nt + t) * d;
    float s = 0.f;
    for (int c = lane; c < d; c += 32) s += row[c];
    const float mean = warp_sum(s) / (float)d;
    float q = 0.f;
    for (int c = lane; c < d; c += 32) {
      const float v = row[c] - mean;
      q = fmaf(v, v, q);
    }
    const float rstd = rsqrtf(warp_sum(q) / (float)d + 1e-5f);
    T* orow = ln_out + ((size_t)b * Nt + t) * d;
    for (int c = lane; c < d; c += 32) orow[c] = from_f32<T>((row[c] - mean) * rstd * ln_g[c] + ln_b[c]);
  }
}

// Tensor-core form (16-bit forms), persistent: a CTA stages the embedding weights [d][64]
// in shared memory once and takes tiles of 32 tokens (one token row segment; 76 KB of
// shared memory at d = 256, so three CTAs per SM), loading the next tile's pixels into
// registers while the current tile is computed and stored.  The patch matrix P [32 tok]
// [64] and the weights are held in T (rows padded to 144 bytes for conflict-free
// ldmatrix); warp w computes tokens 16(w%2).. x channels (w/2)*d/4 .. with mma.sync
// m16n8k16 (K = 64 in 4 steps, FP32 accumulate).  The tile goes through shared memory so
// the FP32 token rows, the token mask and the fused LayerNorm are written coalesced.  The
// LayerNorm statistics (FP32, two passes: mean, then squared deviations) come from the
// accumulator registers: quad shuffles, then the four column parts of a row through
// shared memory in a fixed order, so that the store loop has no reductions left.
template <int D>
struct EmbTc {
  static constexpr int TOK = 32, KP = 72;          // tokens per tile; padded row length (16-bit) of P and W
  static constexpr int MT = TOK / 16, NQ = 8 / MT;  // warps: MT token tiles x NQ column parts
  static constexpr int P_BYTES = TOK * KP * 2;
  static constexpr int W_BYTES = D * KP * 2;
  static constexpr int OUT_STRIDE = D + 4;         // floats per staged output row
  static constexpr int SMEM = P_BYTES + W_BYTES + TOK * OUT_STRIDE * 4 + TOK * 4 * 4 /*known, per pixel row*/ +
                              2 * NQ * TOK * 4 /*row statistics*/;
};

__device__ __forceinline__ void ldsm_x4_e(uint32_t (&r)[4], const void* p) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_e(uint32_t (&r)[2], const void* p) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

// One pixel row (4 pixels) of one token: RGB and the known-pixel bits (bit j: pixel j known).
struct PatchRow {
  float r[4], g[4], b[4];
  uint32_t known;
};

// Pixel row pr of token t of frame b (zeros and no known pixel outside the frame or the grid).
__device__ __forceinline__ PatchRow load_patch_row(const float* __restrict__ x, const uint8_t* __restrict__ hole,
                                                   int b, int t, int pr, int H, int W, int Wt, int Nt, bool vec) {
  PatchRow v;
#pragma unroll
  for (int j = 0; j < 4; ++j) v.r[j] = v.g[j] = v.b[j] = 0.f;
  v.known = 0;
  if (t >= Nt) return v;
  const int ty = t / Wt, tx = t - (t / Wt) * Wt;
  const int y = ty * 4 + pr, xx0 = tx * 4;
  if (y >= H) return v;
  const size_t HW = (size_t)H * W, q = (size_t)y * W + xx0;
  const float* xb = x + (size_t)b * 3 * HW + q;
  const uint8_t* hb = hole + (size_t)b * HW + q;
  if (vec && xx0 + 3 < W) {  // 16-byte aligned rows: vector loads
    const float4 r4 = *reinterpret_cast<const float4*>(xb);
    const float4 g4 = *reinterpret_cast<const float4*>(xb + HW);
    const float4 b4 = *reinterpret_cast<const float4*>(xb + 2 * HW);
    const uchar4 h4 = *reinterpret_cast<const uchar4*>(hb);
    v.r[0] = r4.x; v.r[1] = r4.y; v.r[2] = r4.z; v.r[3] = r4.w;
    v.g[0] = g4.x; v.g[1] = g4.y; v.g[2] = g4.z; v.g[3] = g4.w;
    v.b[0] = b4.x; v.b[1] = b4.y; v.b[2] = b4.z; v.b[3] = b4.w;
    v.known = (h4.x == 0) | ((h4.y == 0) << 1) | ((h4.z == 0) << 2) | ((h4.w == 0) << 3);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (xx0 + j < W) {
        v.r[j] = xb[j]; v.g[j] = xb[HW + j]; v.b[j] = xb[2 * HW + j];
        v.known |= (uint32_t)(hb[j] == 0) << j;
      }
  }
  return v;
}

template <int D, typename T>
__global__ void __launch_bounds__(256) embed_tc_kernel(const float* __restrict__ x, const uint8_t* __restrict__ hole,
                                                       int B, int H, int W, int Ht, int Wt, const T* __restrict__ we16,
                                                       const float* __restrict__ be, float* __restrict__ tok,
                                                       uint8_t* __restrict__ v0, const float* __restrict__ ln_g,
                                                       const float* __restrict__ ln_b, T* __restrict__ ln_out) {
  using C = EmbTc<D>;
  extern __shared__ __align__(16) uint8_t esm[];
  T* P = reinterpret_cast<T*>(esm);                                         // [TOK][KP]
  T* Ws = reinterpret_cast<T*>(esm + C::P_BYTES);                           // [D][KP]
  float* O = reinterpret_cast<float*>(esm + C::P_BYTES + C::W_BYTES);      // [TOK][OUT_STRIDE]
  uint32_t* known = reinterpret_cast<uint32_t*>(esm + C::P_BYTES + C::W_BYTES + C::TOK * C::OUT_STRIDE * 4);  // [TOK][4]
  float* red = reinterpret_cast<float*>(known + 4 * C::TOK);  // [TOK][NQ column parts] row sums
  float* red2 = red + C::NQ * C::TOK;                          // [TOK][NQ] squared deviations
  const int Nt = Ht * Wt, tpf = (Nt + C::TOK - 1) / C::TOK, tiles = B * tpf;
  const int tid = threadIdx.x;
  // weights: [D][64] 16-bit rows of 128 B -> padded rows, once per CTA
  for (int e = tid; e < D * 8; e += 256) {
    const int n = e >> 3, ch = e & 7;
    *reinterpret_cast<uint4*>(Ws + n * C::KP + ch * 8) = *reinterpret_cast<const uint4*>(we16 + (size_t)n * 64 + ch * 8);
  }
  pdl_trigger();
  pdl_wait();
  static_assert(C::TOK * 4 <= 256, "one thread per (token, pixel row)");
  // thread -> pixel row pr of token tl; a warp covers 32 neighbouring tokens of one pixel
  // row, so its loads are contiguous 16-byte runs; all loads are independent
  const bool loader = tid < C::TOK * 4;
  const int tl_ld = tid & (C::TOK - 1), pr = tid / C::TOK;
  const bool vec = (W & 3) == 0 && ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(hole)) & 15) == 0;
  PatchRow cur{};
  if (loader && (int)blockIdx.x < tiles)
    cur = load_patch_row(x, hole, blockIdx.x / tpf, (blockIdx.x % tpf) * C::TOK + tl_ld, pr, H, W, Wt, Nt, vec);
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;
  const int m0 = (warp % C::MT) * 16;
  constexpr int NT = D / 8 / C::NQ;  // n-tiles of 8 per warp (D / NQ columns)
  const int n0 = (warp / C::MT) * (D / C::NQ);
  const int half = warp / C::MT;     // this warp's column part
  auto part_sum = [&](const float* r, int row) {  // the column parts of a row, in a fixed order
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < C::NQ; ++k) v += r[row * C::NQ + k];
    return v;
  };
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int b = tile / tpf, t0 = (tile - b * tpf) * C::TOK;
    __syncthreads();  // the previous tile's P, O, known and statistics are no longer read
    if (loader) {
      T* prow = P + tl_ld * C::KP + 4 * pr;
#pragma unroll
      for (int j = 0; j < 4; ++j) {  // hole pixels enter as 0 (the mask channel carries them)
        const bool kn = (cur.known >> j) & 1u;
        prow[j] = from_f32<T>(kn ? cur.r[j] : 0.f);
        prow[16 + j] = from_f32<T>(kn ? cur.g[j] : 0.f);
        prow[32 + j] = from_f32<T>(kn ? cur.b[j] : 0.f);
        prow[48 + j] = from_f32<T>(kn ? 1.f : 0.f);
      }
      known[tl_ld * 4 + pr] = cur.known;
      // the next tile's pixels, in flight while this tile is computed and stored
      const int nt = tile + gridDim.x;
      if (nt < tiles) cur = load_patch_row(x, hole, nt / tpf, (nt % tpf) * C::TOK + tl_ld, pr, H, W, Wt, Nt, vec);
    }
    __syncthreads();
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      uint32_t a[4];
      ldsm_x4_e(a, P + (m0 + (lane & 15)) * C::KP + ks * 16 + (lane >> 4) * 8);
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        uint32_t bb[2];
        ldsm_x2_e(bb, Ws + (n0 + 8 * j + (lane & 7)) * C::KP + ks * 16 + ((lane >> 3) & 1) * 8);
        mma16816<T>(acc[j], a, bb[0], bb[1]);
      }
    }
    // bias; this thread's parts of rows m0 + g and m0 + g + 8 (columns n0 + 8j + 2tq, +1)
    float sa = 0.f, sb = 0.f;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int c = n0 + 8 * j + 2 * tq;
      const float b0 = be[c], b1 = be[c + 1];
      acc[j][0] += b0;
      acc[j][1] += b1;
      acc[j][2] += b0;
      acc[j][3] += b1;
      sa += acc[j][0] + acc[j][1];
      sb += acc[j][2] + acc[j][3];
    }
    sa += __shfl_xor_sync(0xffffffffu, sa, 1);
    sa += __shfl_xor_sync(0xffffffffu, sa, 2);
    sb += __shfl_xor_sync(0xffffffffu, sb, 1);
    sb += __shfl_xor_sync(0xffffffffu, sb, 2);
    if (tq == 0) {
      red[(m0 + g) * C::NQ + half] = sa;
      red[(m0 + g + 8) * C::NQ + half] = sb;
    }
    __syncthreads();
    const float ma = part_sum(red, m0 + g) * (1.f / D);
    const float mb = part_sum(red, m0 + g + 8) * (1.f / D);
    float qa = 0.f, qb = 0.f;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int c = n0 + 8 * j + 2 * tq;
      qa = fmaf(acc[j][0] - ma, acc[j][0] - ma, qa);
      qa = fmaf(acc[j][1] - ma, acc[j][1] - ma, qa);
      qb = fmaf(acc[j][2] - mb, acc[j][2] - mb, qb);
      qb = fmaf(acc[j][3] - mb, acc[j][3] - mb, qb);
      O[(m0 + g) * C::OUT_STRIDE + c] = acc[j][0];
      O[(m0 + g) * C::OUT_STRIDE + c + 1] = acc[j][1];
      O[(m0 + g + 8) * C::OUT_STRIDE + c] = acc[j][2];
      O[(m0 + g + 8) * C::OUT_STRIDE + c + 1] = acc[j][3];
    }
    qa += __shfl_xor_sync(0xffffffffu, qa, 1);
    qa += __shfl_xor_sync(0xffffffffu, qa, 2);
    qb += __shfl_xor_sync(0xffffffffu, qb, 1);
    qb += __shfl_xor_sync(0xffffffffu, qb, 2);
    if (tq == 0) {
      red2[(m0 + g) * C::NQ + half] = qa;
      red2[(m0 + g + 8) * C::NQ + half] = qb;
    }
    __syncthreads();
    if (tid < C::TOK && t0 + tid < Nt) {
      const uint32_t* kw = known + tid * 4;
      v0[(size_t)b * Nt + t0 + tid] = (uint8_t)((kw[0] | kw[1] | kw[2] | kw[3]) != 0u);
    }
    // each warp writes TOK / 8 token rows and their LayerNorm
#pragma unroll 2
    for (int i = 0; i < C::TOK / 8; ++i) {
      const int tl = warp * (C::TOK / 8) + i, t = t0 + tl;
      if (t >= Nt) break;
      const float* orow = O + tl * C::OUT_STRIDE;
      float* trow = tok + ((size_t)b * Nt + t) * D;
      const float mean = part_sum(red, tl) * (1.f / D);
      const float rstd = rsqrtf(part_sum(red2, tl) * (1.f / D) + 1e-5f);
      T* lrow = ln_out + ((size_t)b * Nt + t) * D;
      for (int c = 2 * lane; c < D; c += 64) {  // two channels per lane: 256-byte warp stores
        const float2 v = *reinterpret_cast<const float2*>(orow + c);
        *reinterpret_cast<float2*>(trow + c) = v;
        float y0 = (v.x - mean) * rstd, y1 = (v.y - mean) * rstd;
        if (ln_g) {  // else the affine part is folded into the next GEMM
          y0 = y0 * ln_g[c] + ln_b[c];
          y1 = y1 * ln_g[c + 1] + ln_b[c + 1];
        }
        *reinterpret_cast<uint32_t*>(lrow + c) = H16<T>::pack2(y0, y1);
      }
    }
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per row; NPER = values per lane (d <= 32 * NPER).
template <typename OutT, int NPER>
__global__ void __launch_bounds__(256) layernorm_kernel(const float* __restrict__ x, const float* __restrict__ g,
                                                        const float* __restrict__ bta, OutT* __restrict__ y,
                                                        int M, int d) {
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  const float* xr = x + (size_t)row * d;
  const int n = d >> 5;
  float v[NPER];
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NPER; ++i) {
    v[i] = (i < n) ? xr[lane + 32 * i] : 0.f;
    s += v[i];
  }
  const float mean = warp_sum(s) / (float)d;
  float q = 0.f;
#pragma unroll
  for (int i = 0; i < NPER; ++i) {
    const float t = (i < n) ? v[i] - mean : 0.f;
    q = fmaf(t, t, q);
  }
  const float rstd = rsqrtf(warp_sum(q) / (float)d + 1e-5f);
  OutT* yr = y + (size_t)row * d;
#pragma unroll
  for (int i = 0; i < NPER; ++i) {
    if (i < n) {
      const int c = lane + 32 * i;
      yr[c] = from_f32<OutT>((v[i] - mean) * rstd * g[c] + bta[c]);
    }
  }
}

constexpr int LOSS_THREADS = 256;
constexpr int LOSS_PIX_PER_CTA = 4096;

// Pass 1: per-CTA sum of |out - target| over hole pixels and count of hole pixels.
__global__ void __launch_bounds__(LOSS_THREADS) l1_partial_kernel(const float* __restrict__ out,
                                                                  const float* __restrict__ tgt,
                                                                  const uint8_t* __restrict__ hole, int HW,
                                                                  size_t npix, float* partials,
                                                                  unsigned* counts) {
  __shared__ float ss[LOSS_THREADS];
  __shared__ unsigned sc[LOSS_THREADS];
  float s = 0.f;
  unsigned c = 0;
  const size_t base = (size_t)blockIdx.x * LOSS_PIX_PER_CTA;
  for (int i = threadIdx.x; i < LOSS_PIX_PER_CTA; i += LOSS_THREADS) {
    const size_t p = base + i;
    if (p >= npix) break;
    if (hole[p] != 0) {
      const size_t b = p / HW, q = p - b * HW;
      const size_t o = b * 3 * HW + q;
      s += fabsf(out[o] - tgt[o]) + fabsf(out[o + HW] - tgt[o + HW]) + fabsf(out[o + 2 * HW] - tgt[o + 2 * HW]);
      ++c;
    }
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int w = LOSS_THREADS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      ss[threadIdx.x] += ss[threadIdx.x + w];
      sc[threadIdx.x] += sc[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = ss[0];
    counts[blockIdx.x] = sc[0];
  }
}

// Pass 2: one CTA reduces the partials in a fixed order (FP64) and writes the loss;
// counts[0] is overwritten with the total hole count for pass 3.
__global__ void __launch_bounds__(LOSS_THREADS) l1_final_kernel(const float* partials, unsigned* counts, int n,
                                                                float* loss) {
  __shared__ double ss[LOSS_THREADS];
  __shared__ unsigned long long sc[LOSS_THREADS];
  double s = 0.0;
  unsigned long long c = 0;
  for (int i = threadIdx.x; i < n; i += LOSS_THREADS) {
    s += (double)partials[i];
    c += counts[i];
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int w = LOSS_THREADS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      ss[threadIdx.x] += ss[threadIdx.x + w];
      sc[threadIdx.x] += sc[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    loss[0] = sc[0] ? (float)(ss[0] / (3.0 * (double)sc[0])) : 0.f;
    counts[0] = (unsigned)sc[0];
  }
}

// Pass 3: grad = sign(out - target) / (3 n_hole) on hole pixels, 0 elsewhere.
__global__ void l1_grad_kernel(const float* __restrict__ out, const float* __restrict__ tgt,
                               const uint8_t* __restrict__ hole, int HW, size_t npix,
                               const unsigned* __restrict__ total, float* __restrict__ grad) {
  const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (p >= npix) return;
  const unsigned n = total[0];
  const float scale = n ? 1.0f / (3.0f * (float)n) : 0.f;
  const size_t b = p / HW, q = p - b * HW;
  const size_t o = b * 3 * HW + q;
  const bool h = hole[p] != 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float df = out[o + c * HW] - tgt[o + c * HW];
    const float sg = df > 0.f ? 1.f : (df < 0.f ? -1.f : 0.f);
    grad[o + c * HW] = h ? sg * scale : 0.f;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_embed(const float* x, const uint8_t* hole, int B, int H, int W, int Ht, int Wt,
                         const float* we_t, const float* be, int d, float* tok, uint8_t* v0, cudaStream_t st,
                         const float* ln_g, const float* ln_b, T* ln_out) {
  if (d % 8) return cudaErrorInvalidValue;
  dim3 grid(cdiv(Ht * Wt, EMB_TOK), B);
  embed_kernel<T><<<grid, 256, 0, st>>>(x, hole, H, W, Ht, Wt, we_t, be, d, tok, v0, ln_g, ln_b, ln_out);
  return cudaGetLastError();
}
template cudaError_t launch_embed<bf16>(const float*, const uint8_t*, int, int, int, int, int, const float*,
                                        const float*, int, float*, uint8_t*, cudaStream_t, const float*,
                                        const float*, bf16*);
template cudaError_t launch_embed<f16>(const float*, const uint8_t*, int, int, int, int, int, const float*,
                                       const float*, int, float*, uint8_t*, cudaStream_t, const float*, const float*,
                                       f16*);

bool embed_tc_supported(int d) { return d == 64 || d == 128 || d == 256; }

template <int D, typename T>
cudaError_t launch_embed_tc_d(const float* x, const uint8_t* hole, int B, int H, int W, int Ht, int Wt, const T* we16,
                              const float* be, float* tok, uint8_t* v0, const float* ln_g, const float* ln_b,
                              T* ln_out, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(embed_tc_kernel<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, EmbTc<D>::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // persistent: three CTAs per SM (the shared memory of a tile allows three)
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
  }
  const int tiles = B * cdiv(Ht * Wt, EmbTc<D>::TOK);
  dim3 grid(tiles < 3 * sms ? tiles : 3 * sms);
  return launch_pdl(embed_tc_kernel<D, T>, grid, dim3(256), EmbTc<D>::SMEM, st, x, hole, B, H, W, Ht, Wt, we16, be, tok,
                    v0, ln_g, ln_b, ln_out);
}

template <typename T>
cudaError_t launch_embed_tc(const float* x, const uint8_t* hole, int B, int H, int W, int Ht, int Wt, const T* we16,
                            const float* be, int d, float* tok, uint8_t* v0, const float* ln_g, const float* ln_b,
                            T* ln_out, cudaStream_t st) {
  if (d == 256) return launch_embed_tc_d<256, T>(x, hole, B, H, W, Ht, Wt, we16, be, tok, v0, ln_g, ln_b, ln_out, st);
  if (d == 128) return launch_embed_tc_d<128, T>(x, hole, B, H, W, Ht, Wt, we16, be, tok, v0, ln_g, ln_b, ln_out, st);
  if (d == 64) return launch_embed_tc_d<64, T>(x, hole, B, H, W, Ht, Wt, we16, be, tok, v0, ln_g, ln_b, ln_out, st);
  return cudaErrorInvalidValue;
}
template cudaError_t launch_embed_tc<bf16>(const float*, const uint8_t*, int, int, int, int, int, const bf16*,
                                           const float*, int, float*, uint8_t*, const float*, const float*, bf16*,
                                           cudaStream_t);
template cudaError_t launch_embed_tc<f16>(const float*, const uint8_t*, int, int, int, int, int, const f16*,
                                          const float*, int, float*, uint8_t*, const float*, const float*, f16*,
                                          cudaStream_t);

template <typename OutT>
cudaError_t launch_layernorm(const float* x, const float* g, const float* b, OutT* y, int M, int d,
                             cudaStream_t st) {
  const int blocks = cdiv(M, 8);
  if (d <= 256)
    layernorm_kernel<OutT, 8><<<blocks, 256, 0, st>>>(x, g, b, y, M, d);
  else
    layernorm_kernel<OutT, 32><<<blocks, 256, 0, st>>>(x, g, b, y, M, d);
  return cudaGetLastError();
}
template cudaError_t launch_layernorm<float>(const float*, const float*, const float*, float*, int, int, cudaStream_t);
template cudaError_t launch_layernorm<bf16>(const float*, const float*, const float*, bf16*, int, int, cudaStream_t);
template cudaError_t launch_layernorm<f16>(const float*, const float*, const float*, f16*, int, int, cudaStream_t);

int loss_partials(int B, int H, int W) {
  return (int)(((size_t)B * H * W + LOSS_PIX_PER_CTA - 1) / LOSS_PIX_PER_CTA);
}

cudaError_t launch_l1_hole_loss(const float* out, const float* target, const uint8_t* hole, int B, int H,
                                int W, float* partials, unsigned* counts, float* loss, float* grad,
                                cudaStream_t st) {
  const size_t npix = (size_t)B * H * W;
  const int nb = loss_partials(B, H, W);
  l1_partial_kernel<<<nb, LOSS_THREADS, 0, st>>>(out, target, hole, H * W, npix, partials, counts);
  l1_final_kernel<<<1, LOSS_THREADS, 0, st>>>(partials, counts, nb, loss);
  if (grad)
    l1_grad_kernel<<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(out, target, hole, H * W, npix, counts, grad);
  return cudaGetLastError();
}

}  // namespace inpaint
