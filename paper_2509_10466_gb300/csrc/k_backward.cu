// Backward pass of the inpainting forward: the gradient of sum(out * grad_out) with
// respect to every weight, for fine-tuning with the hole-L1 loss (the paper trains with
// a per-pixel L1 loss weighted towards the masked region, "Training structure").
//
// FP32 throughout.  The forward is run once keeping only each block's input; the
// reverse sweep recomputes one block at a time from its saved input (per-block
// activation recomputation) and then applies the adjoint of each step:
//   composite -> head conv -> GELU -> conv (+ x2 upsample adjoint) -> ... -> final LN
//   block l: fc2 -> GELU -> fc1 -> LN2 (+ residual) -> proj -> masked window attention
//            -> QKV -> LN1 (+ residual)
//   patch embedding.
// The token masks are integers and carry no gradient.  Every reduction (bias, LN scale
// and shift, split-K weight gradients) sums fixed partitions in a fixed order, so the
// result is bit-reproducible.
#include "common.cuh"
#include "context.cuh"

#include <algorithm>

namespace inpaint {

int gemm_split_count(int K, int splits);

namespace {

constexpr int WS = 8, SLOTS = 64, DH = 32;

__device__ __forceinline__ float gelu_grad(float z) {
  const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752440f));
  const float pdf = 0.39894228040143267794f * expf(-0.5f * z * z);
  return cdf + z * pdf;
}

__global__ void gelu_fwd_kernel(const float* __restrict__ z, float* __restrict__ h, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    h[i] = gelu_erf(z[i]);
}

__global__ void gelu_bwd_kernel(const float* __restrict__ z, float* __restrict__ g, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    g[i] *= gelu_grad(z[i]);
}

// FP32 products on the tensor cores, accurate to about 1e-5: a value x is split into hi =
// bf16(x) and lo = bf16(x - hi) (x = hi + lo within 2^-17 |x|), and A . B^T is taken as
// Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T (the dropped Alo Blo^T is below 2^-16 of a product)
// in ONE bf16 GEMM with FP32 accumulation over a tripled K: A' = [Ahi | Ahi | Alo],
// B' = [Bhi | Blo | Bhi].
// split3_kernel writes such a K-major operand from FP32 X [R][C] (row pitch ld):
// TRANS = false: out [Ro][3 Kp], row r = row r of X, K along C (Ro >= R, Kp >= C);
// TRANS = true:  out [Ro][3 Kp], row r = column r of X, K along R (Ro >= C, Kp >= R);
// part p of a row at columns p Kp .. p Kp + Kp - 1 (b_side: hi, lo, hi; else hi, hi, lo);
// padding rows and columns are zero.  32 x 64 tiles through shared memory, two K positions
// per 32-bit store.
template <bool TRANS>
__global__ void __launch_bounds__(256) split3_kernel(const float* __restrict__ X, int R, int C, int ld, int Ro,
                                                     int Kp, int b_side, bf16* __restrict__ out) {
  // tile: 32 output rows x 64 K positions, t[o][k] (row pitch 66 floats: 8-byte aligned pairs)
  __shared__ float t[32][66];
  const int o0 = blockIdx.y * 32, k0 = blockIdx.x * 64;  // output rows, K positions
  if (TRANS) {  // rows of X = K positions, columns of X = output rows: coalesced reads along o
    for (int i = threadIdx.y; i < 64; i += 8) {
      const int r = k0 + i, cc = o0 + threadIdx.x;
      t[threadIdx.x][i] = r < R && cc < C ? X[(size_t)r * ld + cc] : 0.f;
    }
  } else {  // rows of X = output rows, columns = K positions: coalesced reads along k
    for (int i = threadIdx.y; i < 32; i += 8) {
      const int r = o0 + i;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int cc = k0 + 32 * h + threadIdx.x;
        t[i][32 * h + threadIdx.x] = r < R && cc < C ? X[(size_t)r * ld + cc] : 0.f;
      }
    }
  }
  __syncthreads();
  // K positions k, k + 1 of output row orow per thread: one 32-bit store per part
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int orow = o0 + i, k = k0 + 2 * threadIdx.x;
    if (orow >= Ro || k >= Kp) continue;
    const float2 v = *reinterpret_cast<const float2*>(&t[i][2 * threadIdx.x]);
    const __nv_bfloat162 hi = __floats2bfloat162_rn(v.x, v.y);
    const float2 hf = __bfloat1622float2(hi);
    const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
    bf16* row = out + (size_t)orow * 3 * Kp;
    *reinterpret_cast<__nv_bfloat162*>(row + k) = hi;
    *reinterpret_cast<__nv_bfloat162*>(row + Kp + k) = b_side ? lo : hi;
    *reinterpret_cast<__nv_bfloat162*>(row + 2 * (size_t)Kp + k) = b_side ? hi : lo;
  }
}

// dst[i][j] = sum_s part[s][i][j], s ascending, for i < m, j < n (slices of m_pad x n_pad).
__global__ void reduce_part_kernel(const float* __restrict__ part, int splits, int m, int n, int m_pad, int n_pad,
                                   float* __restrict__ dst) {
  const size_t total = (size_t)m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    float acc = 0.f;
    for (int sp = 0; sp < splits; ++sp) acc += part[((size_t)sp * m_pad + i) * n_pad + j];
    dst[e] = acc;
  }
}

// out[i] = sum_s parts[s*n + i], s ascending.
__global__ void reduce_splits_kernel(const float* __restrict__ parts, int splits, size_t n, float* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += parts[(size_t)k * n + i];
    out[i] = s;
  }
}

// part[c][n] = sum over rows [c*rows, (c+1)*rows) of A[m][n], rows in order.
__global__ void colsum_partial_kernel(const float* __restrict__ A, int M, int N, int rows, float* __restrict__ part) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (n >= N) return;
  const int m0 = c * rows, m1 = min(M, m0 + rows);
  float s = 0.f;
  for (int m = m0; m < m1; ++m) s += A[(size_t)m * N + n];
  part[(size_t)c * N + n] = s;
}

// gp[b][y][x][c] over the padded frame: grad_out on hole pixels of the H x W crop, else 0.
__global__ void pred_grad_kernel(const float* __restrict__ gout, const uint8_t* __restrict__ hole, int B, int H, int W,
                                 int Hp, int Wp, float* __restrict__ gp) {
  const size_t n = (size_t)B * Hp * Wp;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int xx = (int)(i % Wp);
    const int y = (int)((i / Wp) % Hp);
    const int b = (int)(i / ((size_t)Wp * Hp));
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (y < H && xx < W) {
      const size_t HW = (size_t)H * W, q = (size_t)y * W + xx;
      if (hole[(size_t)b * HW + q] != 0) {
        const float* g = gout + (size_t)b * 3 * HW + q;
        g0 = g[0]; g1 = g[HW]; g2 = g[2 * HW];
      }
    }
    gp[i * 3 + 0] = g0;
    gp[i * 3 + 1] = g1;
    gp[i * 3 + 2] = g2;
  }
}

// out[p][c] = (UP ? upsample2(in) : in)[p + offset(tap)][c], zero outside.  in NHWC.
template <bool UP>
__global__ void im2col_tap_kernel(const float* __restrict__ in, int B, int Hi, int Wi, int C, int tap,
                                  float* __restrict__ out) {
  const int Ho = UP ? 2 * Hi : Hi, Wo = UP ? 2 * Wi : Wi;
  const int ky = tap / 3 - 1, kx = tap % 3 - 1;
  const size_t n = (size_t)B * Ho * Wo * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const size_t p = i / C;
    const int ox = (int)(p % Wo), oy = (int)((p / Wo) % Ho), b = (int)(p / ((size_t)Wo * Ho));
    const int uy = oy + ky, ux = ox + kx;
    float v = 0.f;
    if (uy >= 0 && uy < Ho && ux >= 0 && ux < Wo) {
      const int iy = UP ? uy >> 1 : uy, ix = UP ? ux >> 1 : ux;
      v = in[(((size_t)b * Hi + iy) * Wi + ix) * C + c];
    }
    out[i] = v;
  }
}

// gf[b][i][j][c] = sum of the 2x2 children of (i, j) in gu (adjoint of nearest x2 upsampling).
__global__ void upsample_adjoint_kernel(const float* __restrict__ gu, int B, int Hi, int Wi, int C,
                                        float* __restrict__ gf) {
  const size_t n = (size_t)B * Hi * Wi * C;
  const int Wo = 2 * Wi;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const size_t p = i / C;
    const int x = (int)(p % Wi), y = (int)((p / Wi) % Hi), b = (int)(p / ((size_t)Wi * Hi));
    const size_t r0 = ((size_t)b * 2 * Hi + 2 * y) * Wo + 2 * x;
    const size_t r1 = r0 + Wo;
    gf[i] = gu[r0 * C + c] + gu[(r0 + 1) * C + c] + gu[r1 * C + c] + gu[(r1 + 1) * C + c];
  }
}

// Data-gradient weights of a 3x3 conv: wf[tap][co][ci] = w[co][ci][8 - tap] (input = grad, Cin' = Cout).
__global__ void flip_conv_w_kernel(const float* __restrict__ w, int Cout, int Cin, float* __restrict__ wf) {
  const size_t n = (size_t)9 * Cout * Cin;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int ci = (int)(i % Cin);
    const int co = (int)((i / Cin) % Cout);
    const int tap = (int)(i / ((size_t)Cin * Cout));
    wf[i] = w[((size_t)co * Cin + ci) * 9 + (8 - tap)];
  }
}

// blob[co][ci][tap] = tmp[tap][co][ci]
__global__ void tap_grad_scatter_kernel(const float* __restrict__ tmp, int Cout, int Cin, float* __restrict__ blob) {
  const size_t n = (size_t)9 * Cout * Cin;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int tap = (int)(i % 9);
    const size_t r = i / 9;
    const int ci = (int)(r % Cin), co = (int)(r / Cin);
    blob[i] = tmp[((size_t)tap * Cout + co) * Cin + ci];
  }
}

// P[b*Nt + t][k], k = ch*16 + i*4 + j: the model input of token t's patch.
__global__ void patch_matrix_kernel(const float* __restrict__ x, const uint8_t* __restrict__ hole, int B, int H,
                                    int W, int Ht, int Wt, float* __restrict__ P) {
  const size_t n = (size_t)B * Ht * Wt * 64;
  const size_t HW = (size_t)H * W;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i & 63);
    const size_t tok = i >> 6;
    const int t = (int)(tok % ((size_t)Ht * Wt)), b = (int)(tok / ((size_t)Ht * Wt));
    const int ch = k >> 4, pi = (k >> 2) & 3, pj = k & 3;
    const int y = (t / Wt) * 4 + pi, xx = (t % Wt) * 4 + pj;
    float v = 0.f;
    if (y < H && xx < W && hole[(size_t)b * HW + (size_t)y * W + xx] == 0)
      v = (ch < 3) ? x[((size_t)b * 3 + ch) * HW + (size_t)y * W + xx] : 1.f;
    P[i] = v;
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// LayerNorm adjoint, one warp per row: gx = rstd*(gy*g - mean(gy*g) - xhat*mean(gy*g*xhat))
// (+ gres when given); gyxhat = gy * xhat for the scale gradient.
template <int NPER>
__global__ void __launch_bounds__(256) ln_bwd_kernel(const float* __restrict__ x, const float* __restrict__ gamma,
                                                     const float* __restrict__ gy, const float* __restrict__ gres,
                                                     float* __restrict__ gx, float* __restrict__ gyxhat, int M,
                                                     int d) {
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  const size_t base = (size_t)row * d;
  const int n = d >> 5;
  float xv[NPER], gv[NPER];
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NPER; ++i) {
    xv[i] = (i < n) ? x[base + lane + 32 * i] : 0.f;
    gv[i] = (i < n) ? gy[base + lane + 32 * i] : 0.f;
    s += xv[i];
  }
  const float mean = warp_sum(s) / (float)d;
  float q = 0.f;
#pragma unroll
  for (int i = 0; i < NPER; ++i) {
    const float t = (i < n) ? xv[i] - mean : 0.f;
    q = fmaf(t, t, q);
  }
  const float rstd = rsqrtf(warp_sum(q) / (float)d + 1e-5f);
  float s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int i = 0; i < NPER; ++i) {
    if (i < n) {
      const float xh = (xv[i] - mean) * rstd;
      const float gxh = gv[i] * gamma[lane + 32 * i];
      s1 += gxh;
      s2 = fmaf(gxh, xh, s2);
    }
  }
  s1 = warp_sum(s1) / (float)d;
  s2 = warp_sum(s2) / (float)d;
#pragma unroll
  for (int i = 0; i < NPER; ++i) {
    if (i < n) {
      const int c = lane + 32 * i;
      const float xh = (xv[i] - mean) * rstd;
      const float gxh = gv[i] * gamma[c];
      float g = rstd * (gxh - s1 - xh * s2);
      if (gres) g += gres[base + c];
      gx[base + c] = g;
      gyxhat[base + c] = gv[i] * xh;
    }
  }
}

// Adjoint of the masked window attention for one (window, head, frame); 64 threads.
struct AttnBwdSmem {
  float Q[SLOTS][DH + 1], K[SLOTS][DH + 1], V[SLOTS][DH + 1], GO[SLOTS][DH + 1];
  float P[SLOTS][SLOTS + 1], GS[SLOTS][SLOTS + 1];
  float rp[225];
  int ok[SLOTS], tok[SLOTS];
};

__device__ __forceinline__ int relpos_idx(int s, int k) { return ((k >> 3) - (s >> 3) + 7) * 15 + ((k & 7) - (s & 7) + 7); }

// One CTA per (window, head), thread s = slot s: the query-side gradients of row s, then the
// key-side gradients of key s.  Rows move between global and shared memory a whole 32-value
// head slice per warp instruction (lane = channel); the scores are computed once and kept in
// P; dot products run four keys at a time (independent FMA chains, each in ascending channel
// order, so every value equals the one-key-at-a-time evaluation).
__global__ void __launch_bounds__(SLOTS) attn_bwd_kernel(const float* __restrict__ qkv, const uint8_t* __restrict__ v_in,
                                                         const float* __restrict__ go, float* __restrict__ gqkv, int Ht,
                                                         int Wt, int d, int offset, int nwx,
                                                         const float* __restrict__ relpos, float* __restrict__ gbias) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  AttnBwdSmem& sm = *reinterpret_cast<AttnBwdSmem*>(smem_raw);
  const int w = blockIdx.x, h = blockIdx.y, b = blockIdx.z;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = SLOTS / 32;  // warps
  // this CTA's partial gradient of the relative-position table: [frame][window][head][225]
  float* gb = gbias ? gbias + (((size_t)b * gridDim.x + w) * gridDim.y + h) * 225 : nullptr;
  for (int e = threadIdx.x; e < 225; e += SLOTS) sm.rp[e] = relpos ? relpos[h * 225 + e] : 0.f;
  const int wy = w / nwx, wx = w - (w / nwx) * nwx;
  const int s = threadIdx.x;
  const int ty = wy * WS - offset + (s >> 3), tx = wx * WS - offset + (s & 7);
  const bool real = ty >= 0 && ty < Ht && tx >= 0 && tx < Wt;
  const size_t t = real ? (size_t)b * Ht * Wt + (size_t)ty * Wt + tx : 0;
  const bool ok = real && v_in[t] != 0;
  sm.ok[s] = ok;
  sm.tok[s] = real ? (int)t : -1;
  __syncthreads();
  for (int sl = warp; sl < SLOTS; sl += NW) {  // the window's head slices, one row per warp step
    const int ts = sm.tok[sl];
    const bool oks = sm.ok[sl];
    const float* row = qkv + (size_t)(ts < 0 ? 0 : ts) * 3 * d + h * DH + lane;
    sm.Q[sl][lane] = ts >= 0 ? row[0] : 0.f;
    sm.K[sl][lane] = oks ? row[d] : 0.f;
    sm.V[sl][lane] = oks ? row[2 * d] : 0.f;
    sm.GO[sl][lane] = ts >= 0 ? go[(size_t)ts * d + h * DH + lane] : 0.f;
  }
  const int any = __syncthreads_or(ok);
  if (!any) {
    float* gq = gqkv + t * 3 * d + h * DH;
    if (real)
      for (int i = 0; i < DH; ++i) { gq[i] = 0.f; gq[d + i] = 0.f; gq[2 * d + i] = 0.f; }
    if (gb)
      for (int e = s; e < 225; e += SLOTS) gb[e] = 0.f;
    return;
  }
  const float scale = 1.0f / sqrtf((float)DH);
  // query side: probabilities, score gradients, dQ
  float acc[DH];
  if (real) {
    float mx = -INFINITY;
    for (int k0 = 0; k0 < SLOTS; k0 += 4) {  // scores (with bias) into P, -inf for excluded keys
      float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < DH; ++i) {
        const float qi = sm.Q[s][i];
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j] = fmaf(qi, sm.K[k0 + j][i], a[j]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = k0 + j;
        const float z = sm.ok[k] ? a[j] * scale + sm.rp[relpos_idx(s, k)] : -INFINITY;
        sm.P[s][k] = z;
        mx = fmaxf(mx, z);
      }
    }
    float l = 0.f;
    for (int k = 0; k < SLOTS; ++k) {
      const float p = sm.ok[k] ? expf(sm.P[s][k] - mx) : 0.f;
      sm.P[s][k] = p;
      l += p;
    }
    const float inv = 1.f / l;
    float D = 0.f;
    for (int k0 = 0; k0 < SLOTS; k0 += 4) {  // dO . V for four keys at a time
      float g[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < DH; ++i) {
        const float gi = sm.GO[s][i];
#pragma unroll
        for (int j = 0; j < 4; ++j) g[j] = fmaf(gi, sm.V[k0 + j][i], g[j]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = k0 + j;
        const float p = sm.P[s][k] * inv;
        sm.P[s][k] = p;
        const float gp = sm.ok[k] ? g[j] : 0.f;
        sm.GS[s][k] = gp;
        D = fmaf(p, gp, D);
      }
    }
    for (int i = 0; i < DH; ++i) acc[i] = 0.f;
    for (int k = 0; k < SLOTS; ++k) {
      const float gs = sm.P[s][k] * (sm.GS[s][k] - D);
      sm.GS[s][k] = gs;
      if (sm.ok[k])
        for (int i = 0; i < DH; ++i) acc[i] = fmaf(gs, sm.K[k][i], acc[i]);
    }
  } else {
    for (int k = 0; k < SLOTS; ++k) { sm.P[s][k] = 0.f; sm.GS[s][k] = 0.f; }
  }
  __syncthreads();
  // V is no longer read: it takes dQ
  if (real)
    for (int i = 0; i < DH; ++i) sm.V[s][i] = acc[i] * scale;
  // relative-position table: d score / d table entry = 1, so its gradient is the sum of the
  // score gradients over the (query, key) slot pairs at that offset (fixed order)
  if (gb)
    for (int e = s; e < 225; e += SLOTS) {
      const int dy = e / 15 - 7, dx = e % 15 - 7;
      float a = 0.f;
      for (int q = 0; q < SLOTS; ++q) {
        const int ky = (q >> 3) + dy, kx = (q & 7) + dx;
        if (ky >= 0 && ky < 8 && kx >= 0 && kx < 8) a += sm.GS[q][ky * 8 + kx];
      }
      gb[e] = a;
    }
  // key side: dK = scale * GS^T Q, dV = P^T dO
  float gk[DH], gv[DH];
  for (int i = 0; i < DH; ++i) { gk[i] = 0.f; gv[i] = 0.f; }
  if (ok) {
    for (int q = 0; q < SLOTS; ++q) {
      const float gs = sm.GS[q][s], p = sm.P[q][s];
      for (int i = 0; i < DH; ++i) {
        gk[i] = fmaf(gs, sm.Q[q][i], gk[i]);
        gv[i] = fmaf(p, sm.GO[q][i], gv[i]);
      }
    }
  }
  __syncthreads();  // K and dO are no longer read: they take dK and dV
  for (int i = 0; i < DH; ++i) {
    sm.K[s][i] = gk[i] * scale;
    sm.GO[s][i] = gv[i];
  }
  __syncthreads();
  for (int sl = warp; sl < SLOTS; sl += NW) {  // the gradient rows of the window's real slots
    const int ts = sm.tok[sl];
    if (ts < 0) continue;
    float* gq = gqkv + (size_t)ts * 3 * d + h * DH + lane;
    gq[0] = sm.V[sl][lane];
    gq[d] = sm.K[sl][lane];
    gq[2 * d] = sm.GO[sl][lane];
  }
}

// out[h][r] = sum over the n windows (fixed order) of part[(i * heads + h) * 225 + r]
__global__ void relpos_grad_reduce_kernel(const float* __restrict__ part, int n, int heads, float* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= heads * 225) return;
  const int h = e / 225, r = e - h * 225;
  float acc = 0.f;
  for (int i = 0; i < n; ++i) acc += part[((size_t)i * heads + h) * 225 + r];
  out[e] = acc;
}

inline unsigned grid1d(size_t n) {
  size_t g = (n + 255) / 256;
  return (unsigned)(g > 65535 ? 65535 : (g ? g : 1));
}

}  // namespace

// gout: dL/dout from the caller; or, with gout null, the loss is taken here: the forward
// also runs the head and composite (into out, or scratch when out is null), then the
// hole-L1 loss against target into *loss and its gradient, which the sweep then uses.
int backward_impl(inpaint_ctx* c, const float* x, const uint8_t* hole, const float* gout, int B, int H, int W,
                  float* gw, cudaStream_t st, const float* target, float* loss, float* out) {
  const Offsets& o = c->off;
  const int Hp = (H + 31) / 32 * 32, Wp = (W + 31) / 32 * 32;
  const int Ht = Hp / 4, Wt = Wp / 4, Nt = Ht * Wt, M = B * Nt;
  const int d = c->d, hid = c->hid, L = c->L, c1 = c->c1, c2 = c->c2;
  const size_t P1 = (size_t)B * 4 * Nt, P2 = (size_t)B * 16 * Nt;   // decoder stage-1 / stage-2 pixels
  const size_t wmax = std::max({(size_t)d * 3 * d, (size_t)d * hid, (size_t)c1 * d, (size_t)c2 * c1, (size_t)d * 64,
                                (size_t)3 * c2});
  const size_t im2 = std::max({P2 * c2, P2 * c1, P1 * d, (size_t)M * 64});
  const int CH = 128;  // column-sum chunks
  const size_t nmax = std::max({(size_t)3 * d, (size_t)hid, (size_t)c1, (size_t)c2, (size_t)3});

  // ---- workspace
  size_t q = 0;
  auto take = [&](size_t bytes) { size_t at = q; q = align_up(q + bytes, 256); return at; };
  const size_t oX = take((size_t)(L + 1) * M * d * 4), oMask = take((size_t)(L + 1) * M);
  const size_t oY1 = take((size_t)M * d * 4), oQKV = take((size_t)M * 3 * d * 4), oO = take((size_t)M * d * 4);
  const size_t oXM = take((size_t)M * d * 4), oY2 = take((size_t)M * d * 4), oA = take((size_t)M * hid * 4);
  const size_t oH = take((size_t)M * hid * 4), oGX = take((size_t)M * d * 4), oGXM = take((size_t)M * d * 4);
  const size_t oGH = take((size_t)M * hid * 4), oGY = take((size_t)M * d * 4), oGQKV = take((size_t)M * 3 * d * 4);
  const size_t oGO = take((size_t)M * d * 4), oGYX = take((size_t)M * d * 4);
  const size_t oZ1 = take(P1 * c1 * 4), oF1 = take(P1 * c1 * 4), oZ2 = take(P2 * c2 * 4), oF2 = take(P2 * c2 * 4);
  const size_t oGP = take(P2 * 3 * 4), oGF2 = take(P2 * c2 * 4), oGU1 = take(P2 * c1 * 4), oGF1 = take(P1 * c1 * 4);
  const size_t oGU0 = take(P1 * d * 4), oIM = take(im2 * 4);
  const size_t oCS = take((size_t)CH * nmax * 4), oWF = take((size_t)9 * wmax * 4), oTAP = take((size_t)9 * wmax * 4);
  const int nw_max = ((Ht + 4 + WS - 1) / WS) * ((Wt + 4 + WS - 1) / WS);  // windows of the offset grid (the larger)
  const size_t oRP = take(c->cfg.pos_bias ? (size_t)B * nw_max * c->heads * 225 * 4 : 256);
  // split operands of the tensor-core products (bf16, three parts along K) and their
  // split-K partial sums
  auto r64 = [](size_t v) { return (v + 63) / 64 * 64; };
  auto r128 = [](size_t v) { return (v + 127) / 128 * 128; };
  const size_t splitA = 3 * std::max({(size_t)hid * r64(M), (size_t)d * r64(M), (size_t)3 * d * r64(M),
                                      (size_t)c2 * r64(P2), (size_t)c1 * r64(P1), (size_t)3 * r64(P2),
                                      (size_t)M * r64(3 * d), (size_t)M * r64(hid)});
  const size_t splitB = 3 * std::max({r64(hid) * r64(M), r64(3 * d) * r64(M), r64(c1) * r64(P2),
                                      r64(d) * r64(P1), r64(c2) * r64(P2), (size_t)64 * r64(M),
                                      r64(d) * r64(hid), r64(hid) * r64(d), r64(d) * r64(3 * d)});
  constexpr int TC_SPLIT_MAX = 32;
  const size_t pmax = std::max({r128(d) * r64(3 * d), r128(d) * r64(hid), r128(hid) * r64(d), r128(c1) * r64(d),
                                r128(c2) * r64(c1), r128(3) * r64(c2), r128(d) * 64});
  const size_t oSA = take(splitA * 2), oSB = take(splitB * 2), oTP = take((size_t)TC_SPLIT_MAX * pmax * 4);
  // the loss taken here: the output frame (unless the caller's), dL/dout, the partial sums
  const bool own_loss = gout == nullptr;
  const size_t frame = (size_t)B * 3 * H * W;
  const int nbl = own_loss ? loss_partials(B, H, W) : 0;
  const size_t oOUT = take(own_loss && !out ? frame * 4 : 0), oGOUT = take(own_loss ? frame * 4 : 0);
  const size_t oLP = take((size_t)nbl * 4), oLC = take((size_t)nbl * 4);
  int rc = grow(&c->bws, &c->bws_bytes, q, c, c->arena_bytes + c->stage_bytes);
  if (rc != INPAINT_OK) return rc;
  uint8_t* ws = c->bws;
  auto F = [&](size_t off) { return reinterpret_cast<float*>(ws + off); };
  float* X = F(oX);
  uint8_t* masks = ws + oMask;
  float *y1 = F(oY1), *qkv = F(oQKV), *ao = F(oO), *xm = F(oXM), *y2 = F(oY2), *a = F(oA), *hh = F(oH);
  float *gx = F(oGX), *gxm = F(oGXM), *gh = F(oGH), *gy = F(oGY), *gqkv = F(oGQKV), *go = F(oGO), *gyx = F(oGYX);
  float *z1 = F(oZ1), *f1 = F(oF1), *z2 = F(oZ2), *f2 = F(oF2), *gp = F(oGP), *gf2 = F(oGF2), *gu1 = F(oGU1);
  float *gf1 = F(oGF1), *gu0 = F(oGU0), *im = F(oIM), *cs = F(oCS), *wf = F(oWF), *tap = F(oTAP);
  float* rpart = F(oRP);
  const float* w = c->w32;
  auto Xl = [&](int l) { return X + (size_t)l * M * d; };

  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) { if (r != cudaSuccess && e == cudaSuccess) e = r; };
  auto K = [&](int cls) { return LaunchScope(c, st, cls); };

  // column sums of A [rows][n] into dst[n]
  auto colsum = [&](const float* A, int rows, int n, float* dst) {
    const int rpc = (rows + CH - 1) / CH;
    const int chunks = (rows + rpc - 1) / rpc;
    { auto ls = K(K_OTHER); colsum_partial_kernel<<<dim3(cdiv(n, 256), chunks), 256, 0, st>>>(A, rows, n, rpc, cs); }
    { auto ls = K(K_OTHER); reduce_splits_kernel<<<grid1d(n), 256, 0, st>>>(cs, chunks, (size_t)n, dst); }
    ok(cudaGetLastError());
  };
  bf16* sA = reinterpret_cast<bf16*>(ws + oSA);
  bf16* sB = reinterpret_cast<bf16*>(ws + oSB);
  float* tpart = F(oTP);
  auto split3 = [&](bool trans, const float* X, int R, int C, int ld, int Ro, int Kp, bool b_side, bf16* out) {
    auto ls = K(K_OTHER);
    const dim3 grid(cdiv(Kp, 64), cdiv(Ro, 32));  // Kp: a multiple of 64
    if (trans) split3_kernel<true><<<grid, dim3(32, 8), 0, st>>>(X, R, C, ld, Ro, Kp, b_side ? 1 : 0, out);
    else split3_kernel<false><<<grid, dim3(32, 8), 0, st>>>(X, R, C, ld, Ro, Kp, b_side ? 1 : 0, out);
    ok(cudaGetLastError());
  };
  // dst[m][n] = sum_r A[r][m] * G[r][n]  (weight gradient X^T G) on the tensor cores, split-K
  // over the rows with a fixed-order reduction
  auto wgrad = [&](const float* A, int lda, int m, const float* G, int ldg, int n, int rows, float* dst) {
    const int Kp = (int)r64(rows), n_pad = (int)r64(n), m_pad = (int)r128(m);
    split3(true, A, rows, m, lda, m, Kp, false, sA);
    split3(true, G, rows, n, ldg, n_pad, Kp, true, sB);
    // the GEMM's tile width for this n (its launcher's rule)
    const int bn = n_pad % 256 == 0 ? 256 : (n_pad % 128 == 0 ? 128 : (n_pad % 192 == 0 ? 192 : 64));
    const int tiles = (m_pad / 128) * (n_pad / bn);
    const int splits = std::max(1, std::min({TC_SPLIT_MAX, 3 * Kp / 64, (2 * 152 + tiles - 1) / tiles}));
    { auto ls = K(K_OTHER); ok(launch_gemm_tc_splitk(sA, sB, tpart, m, n_pad, 3 * Kp, splits, c->dev_err, st)); }
    { auto ls = K(K_OTHER); reduce_part_kernel<<<grid1d((size_t)m * n), 256, 0, st>>>(tpart, splits, m, n, m_pad, n_pad, dst); }
    ok(cudaGetLastError());
  };
  // out[M][n] = G[M][k] . Wt^T where Wt is [n][k] row-major (a linear weight [in=n][out=k]):
  // on the tensor cores when n is a multiple of 64 (the GEMM's tile width), else FP32 SIMT
  auto dgrad = [&](const float* G, int k, const float* Wm, int n, float* out) {
    if (n % 64 == 0) {
      const int Kp = (int)r64(k);
      split3(false, G, M, k, k, M, Kp, false, sA);
      split3(false, Wm, n, k, k, n, Kp, true, sB);
      auto ls = K(K_OTHER);
      ok(launch_gemm_tc<bf16>(sA, sB, out, n, M, n, 3 * Kp, EPI_NONE, nullptr, nullptr, c->dev_err, st));
      return;
    }
    auto ls = K(K_OTHER);
    ok(launch_gemm_f32_ex(false, true, G, k, Wm, k, out, n, M, n, k, 1, EPI_NONE, nullptr, nullptr, st));
  };
  // weight + bias gradient of a 3x3 conv whose output gradient is gz [P][cout] (NHWC)
  // and whose input is `in` (NHWC [B, hi, wi, cin], upsampled first when up).
  auto conv_wgrad = [&](const float* gz, int cout, const float* in, int hi, int wi, int cin, bool up, size_t P,
                        size_t wofs, size_t bofs) {
    colsum(gz, (int)P, cout, gw + bofs);
    for (int t = 0; t < 9; ++t) {
      {
        auto ls = K(K_OTHER);
        if (up) im2col_tap_kernel<true><<<grid1d(P * cin), 256, 0, st>>>(in, B, hi, wi, cin, t, im);
        else im2col_tap_kernel<false><<<grid1d(P * cin), 256, 0, st>>>(in, B, hi, wi, cin, t, im);
      }
      wgrad(gz, cout, cout, im, cin, cin, (int)P, tap + (size_t)t * cout * cin);
    }
    { auto ls = K(K_OTHER); tap_grad_scatter_kernel<<<grid1d((size_t)9 * cout * cin), 256, 0, st>>>(tap, cout, cin, gw + wofs); }
    ok(cudaGetLastError());
  };
  auto ln_bwd = [&](const float* xin, const float* g, const float* gyv, const float* gres, float* gxo, size_t gofs,
                    size_t bofs) {
    {
      auto ls = K(K_OTHER);
      if (d <= 256) ln_bwd_kernel<8><<<cdiv(M, 8), 256, 0, st>>>(xin, g, gyv, gres, gxo, gyx, M, d);
      else ln_bwd_kernel<32><<<cdiv(M, 8), 256, 0, st>>>(xin, g, gyv, gres, gxo, gyx, M, d);
    }
    ok(cudaGetLastError());
    colsum(gyx, M, d, gw + gofs);
    colsum(gyv, M, d, gw + bofs);
  };
  // C[M][N] = epi(X[M][K] . Wl + bias) for a linear weight Wl [K][N] (in, out): on the tensor
  // cores (split products, FP32 epilogue) when N is a multiple of 64, else FP32 SIMT
  auto linear = [&](int cls, const float* Xa, int Kd, const float* Wl, int N, float* C, int epi, const float* bias,
                    const float* resid) {
    if (N % 64 == 0) {
      const int Kp = (int)r64(Kd);
      split3(false, Xa, M, Kd, Kd, M, Kp, false, sA);
      split3(true, Wl, Kd, N, N, N, Kp, true, sB);  // Wl^T: row n = column n of Wl, K along the inputs
      auto ls = K(cls);
      ok(launch_gemm_tc<bf16>(sA, sB, C, N, M, N, 3 * Kp, epi == EPI_BIAS ? EPI_BIAS_F32 : epi, bias, resid,
                              c->dev_err, st));
      return;
    }
    auto ls = K(cls);
    ok(launch_gemm_f32(Xa, Kd, Wl, N, C, N, M, N, Kd, epi, bias, resid, st));
  };
  // block l forward from X[l]; keeps y1, qkv, o, xm, y2, a, h; writes X[l+1] when `out`
  auto block_fwd = [&](int l, bool out) {
    const BlockOff& bo = o.blk[l];
    const int offset = (c->cfg.shift && (l & 1)) ? 4 : 0;
    { auto ls = K(K_LN); ok(launch_layernorm<float>(Xl(l), w + bo.ln1g, w + bo.ln1b, y1, M, d, st)); }
    linear(K_QKV, y1, d, w + bo.qkvw, 3 * d, qkv, EPI_BIAS, w + bo.qkvb, nullptr);
    const float* rp = c->cfg.pos_bias ? w + bo.relpos : nullptr;
    { auto ls = K(K_ATTN); ok(launch_attention<float>(qkv, masks + (size_t)l * M, ao, masks + (size_t)(l + 1) * M, B, Ht, Wt, d, c->heads, offset, st, rp)); }
    linear(K_PROJ, ao, d, w + bo.projw, d, xm, EPI_BIAS_RESID, w + bo.projb, Xl(l));
    { auto ls = K(K_LN); ok(launch_layernorm<float>(xm, w + bo.ln2g, w + bo.ln2b, y2, M, d, st)); }
    linear(K_FC1, y2, d, w + bo.fc1w, hid, a, EPI_BIAS, w + bo.fc1b, nullptr);
    { auto ls = K(K_OTHER); gelu_fwd_kernel<<<grid1d((size_t)M * hid), 256, 0, st>>>(a, hh, (size_t)M * hid); }
    if (out) linear(K_FC2, hh, hid, w + bo.fc2w, d, Xl(l + 1), EPI_BIAS_RESID, w + bo.fc2b, xm);
    ok(cudaGetLastError());
  };

  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(attn_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(AttnBwdSmem)) !=
        cudaSuccess)
      return INPAINT_E_CUDA;
    attr = true;
  }

  ok(cudaMemsetAsync(gw, 0, c->nparams * 4, st));
  // ---- forward, keeping the block inputs
  { auto ls = K(K_EMBED); ok(launch_embed(x, hole, B, H, W, Ht, Wt, c->embed_wt, w + o.embb, d, X, masks, st)); }
  for (int l = 0; l < L; ++l) block_fwd(l, true);
  float* yf = y1;
  { auto ls = K(K_LN); ok(launch_layernorm<float>(Xl(L), w + o.lnfg, w + o.lnfb, yf, M, d, st)); }
  { auto ls = K(K_DEC1); ok(launch_conv3x3_f32(yf, B, Ht, Wt, d, true, c->dec1_wt, w + o.d1b, 1, f1, z1, c1, st)); }
  { auto ls = K(K_DEC2); ok(launch_conv3x3_f32(f1, B, 2 * Ht, 2 * Wt, c1, true, c->dec2_wt, w + o.d2b, 1, f2, z2, c2, st)); }

  if (own_loss) {  // the head and composite of the forward, then the hole-L1 loss and dL/dout
    float* of = out ? out : F(oOUT);
    float* g = F(oGOUT);
    { auto ls = K(K_HEAD); ok(launch_head_composite<float>(f2, B, Hp, Wp, c2, w + o.hw, w + o.hb, x, hole, H, W, of, nullptr, st)); }
    {
      auto ls = K(K_OTHER);
      ok(launch_l1_hole_loss(of, target, hole, B, H, W, F(oLP), reinterpret_cast<unsigned*>(ws + oLC), loss, g, st));
    }
    gout = g;
  }
  // ---- head conv and composite
  { auto ls = K(K_OTHER); pred_grad_kernel<<<grid1d(P2), 256, 0, st>>>(gout, hole, B, H, W, Hp, Wp, gp); }
  conv_wgrad(gp, 3, f2, Hp, Wp, c2, false, P2, o.hw, o.hb);
  { auto ls = K(K_OTHER); flip_conv_w_kernel<<<grid1d((size_t)27 * c2), 256, 0, st>>>(w + o.hw, 3, c2, wf); }
  { auto ls = K(K_OTHER); ok(launch_conv3x3_f32(gp, B, Hp, Wp, 3, false, wf, nullptr, 0, gf2, nullptr, c2, st)); }
  // ---- decoder stage 2
  { auto ls = K(K_OTHER); gelu_bwd_kernel<<<grid1d(P2 * c2), 256, 0, st>>>(z2, gf2, P2 * c2); }
  conv_wgrad(gf2, c2, f1, 2 * Ht, 2 * Wt, c1, true, P2, o.d2w, o.d2b);
  { auto ls = K(K_OTHER); flip_conv_w_kernel<<<grid1d((size_t)9 * c2 * c1), 256, 0, st>>>(w + o.d2w, c2, c1, wf); }
  { auto ls = K(K_OTHER); ok(launch_conv3x3_f32(gf2, B, Hp, Wp, c2, false, wf, nullptr, 0, gu1, nullptr, c1, st)); }
  { auto ls = K(K_OTHER); upsample_adjoint_kernel<<<grid1d(P1 * c1), 256, 0, st>>>(gu1, B, 2 * Ht, 2 * Wt, c1, gf1); }
  // ---- decoder stage 1
  { auto ls = K(K_OTHER); gelu_bwd_kernel<<<grid1d(P1 * c1), 256, 0, st>>>(z1, gf1, P1 * c1); }
  conv_wgrad(gf1, c1, yf, Ht, Wt, d, true, P1, o.d1w, o.d1b);
  { auto ls = K(K_OTHER); flip_conv_w_kernel<<<grid1d((size_t)9 * c1 * d), 256, 0, st>>>(w + o.d1w, c1, d, wf); }
  { auto ls = K(K_OTHER); ok(launch_conv3x3_f32(gf1, B, 2 * Ht, 2 * Wt, c1, false, wf, nullptr, 0, gu0, nullptr, d, st)); }
  { auto ls = K(K_OTHER); upsample_adjoint_kernel<<<grid1d((size_t)M * d), 256, 0, st>>>(gu0, B, Ht, Wt, d, gy); }
  // ---- final LayerNorm
  ln_bwd(Xl(L), w + o.lnfg, gy, nullptr, gx, o.lnfg, o.lnfb);

  // ---- blocks, last to first, each recomputed from its saved input
  for (int l = L - 1; l >= 0; --l) {
    const BlockOff& bo = o.blk[l];
    const int offset = (c->cfg.shift && (l & 1)) ? 4 : 0;
    block_fwd(l, false);
    // MLP: x_{l+1} = xm + gelu(y2 W1 + b1) W2 + b2
    colsum(gx, M, d, gw + bo.fc2b);
    wgrad(hh, hid, hid, gx, d, d, M, gw + bo.fc2w);
    dgrad(gx, d, w + bo.fc2w, hid, gh);
    { auto ls = K(K_OTHER); gelu_bwd_kernel<<<grid1d((size_t)M * hid), 256, 0, st>>>(a, gh, (size_t)M * hid); }
    colsum(gh, M, hid, gw + bo.fc1b);
    wgrad(y2, d, d, gh, hid, hid, M, gw + bo.fc1w);
    dgrad(gh, hid, w + bo.fc1w, d, gy);
    ln_bwd(xm, w + bo.ln2g, gy, gx, gxm, bo.ln2g, bo.ln2b);
    // attention: xm = x_l + attn(LN1(x_l)) Wo + bo
    colsum(gxm, M, d, gw + bo.projb);
    wgrad(ao, d, d, gxm, d, d, M, gw + bo.projw);
    dgrad(gxm, d, w + bo.projw, d, go);
    {
      auto ls = K(K_OTHER);
      const int nwy = (Ht + offset + WS - 1) / WS, nwx = (Wt + offset + WS - 1) / WS;
      const bool rpb = c->cfg.pos_bias != 0;
      attn_bwd_kernel<<<dim3(nwy * nwx, c->heads, B), SLOTS, sizeof(AttnBwdSmem), st>>>(
          qkv, masks + (size_t)l * M, go, gqkv, Ht, Wt, d, offset, nwx, rpb ? w + bo.relpos : nullptr,
          rpb ? rpart : nullptr);
      ok(cudaGetLastError());
      if (rpb) {
        relpos_grad_reduce_kernel<<<cdiv(c->heads * 225, 256), 256, 0, st>>>(rpart, B * nwy * nwx, c->heads,
                                                                               gw + bo.relpos);
        ok(cudaGetLastError());
      }
    }
    colsum(gqkv, M, 3 * d, gw + bo.qkvb);
    wgrad(y1, d, d, gqkv, 3 * d, 3 * d, M, gw + bo.qkvw);
    dgrad(gqkv, 3 * d, w + bo.qkvw, d, gy);
    ln_bwd(Xl(l), w + bo.ln1g, gy, gxm, gx, bo.ln1g, bo.ln1b);
  }
  // ---- patch embedding
  colsum(gx, M, d, gw + o.embb);
  { auto ls = K(K_OTHER); patch_matrix_kernel<<<grid1d((size_t)M * 64), 256, 0, st>>>(x, hole, B, H, W, Ht, Wt, im); }
  wgrad(gx, d, d, im, 64, 64, M, gw + o.embw);
  ok(cudaGetLastError());
  return e == cudaSuccess ? INPAINT_OK : INPAINT_E_CUDA;
}

}  // namespace inpaint
