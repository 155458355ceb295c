// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include "inpaint.h"

namespace inpaint {

typedef __nv_bfloat16 bf16;
typedef __half f16;

// Kernel-class ids for event timing (match INPAINT_PROFILE_CLASSES in inpaint.h).
enum KClass {
  K_EMBED = 0, K_LN = 1, K_QKV = 2, K_ATTN = 3, K_PROJ = 4, K_FC1 = 5, K_FC2 = 6,
  K_DEC1 = 7, K_DEC2 = 8, K_HEAD = 9, K_OTHER = 10, K_MLP = 11, K_CLOUD = 12, K_SPLAT = 13, K_QKV_ATTN = 14
};

// Device-side error codes written into the context's error word.
enum DevErr { DEV_OK = 0, DEV_MBAR_TIMEOUT = 1, DEV_BAD_SHAPE = 2 };

// GEMM epilogues.
enum Epi {
  EPI_BIAS = 0,        // C = acc + bias                     (output type T)
  EPI_BIAS_GELU = 1,   // C = gelu(acc + bias)               (output type T)
  EPI_BIAS_RESID = 2,  // C(f32) = resid(f32) + acc + bias   (C may alias resid)
  EPI_NONE = 3,        // C(f32) = acc
  EPI_RESID_LN = 4,    // C(f32) = resid + acc + bias, and LayerNorm(C row) -> bf16 (N == tile width)
  EPI_BIAS_F32 = 5     // C(f32) = acc + bias
};

// INPAINT_OK for cudaSuccess; otherwise records `e` as the calling host thread's last CUDA
// error (inpaint_last_cuda_error) and returns INPAINT_E_CUDA.
int record_cuda_error(cudaError_t e);

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Programmatic dependent launch.  The forward's kernels are launched with programmatic
// stream serialization: a kernel may be scheduled while the previous kernel on the stream
// finishes (its CTAs take SMs as they free up and run their prologue: barriers, TMEM,
// weights), and every thread calls pdl_wait() before it touches any activation, which
// returns once the previous kernel has completed and its memory is visible.  Each kernel
// lets its successor be scheduled as soon as all its own CTAs are running.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = grid;
  lc.blockDim = block;
  lc.dynamicSmemBytes = smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, kern, args...);
}
__host__ __device__ inline int cdiv(int a, int b) { return (a + b - 1) / b; }

__device__ __forceinline__ float gelu_erf(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752440f));
}
// GELU for the BF16 form, whose GELU outputs are rounded to bf16 right away:
//   gelu(x) ~ x * sigmoid(2u) = 0.5 x (1 + tanh(u)),  u = x P(x^2),  P of degree 4,
// the logistic form of the normal CDF with an odd polynomial argument whose coefficients
// were fitted (iteratively reweighted least squares, minimax-like) to
// 0.5 x (1 + erf(x / sqrt 2)) on [-12, 12]: |error| <= 5e-6 absolute there with an exact
// tanh; u is increasing in x and the form saturates to x and to 0 beyond.  The tanh is the
// PTX approximate hyperbolic tangent (one MUFU operation, relative error about 2^-11),
// which adds at most about 2.5e-4 |x| absolute: 2.5e-4 relative to the output for x > 0,
// an eighth of the bf16 rounding step 2^-9 of the output; for x < 0 (output near 0) the
// added error is absolute.  8 FP32 operations and 1 MUFU per value.
// 2^x by the PTX approximate base-2 exponential (one MUFU operation; subnormal results
// flush to 0, 2^-inf = 0).
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float tanh_approx(float x) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float gelu_as(float x) {
  const float x2 = x * x;
  float p = fmaf(9.163219942820433e-07f, x2, -2.670336834853515e-05f);
  p = fmaf(p, x2, -1.468761620344594e-04f);
  p = fmaf(p, x2, 3.6510955542325974e-02f);
  p = fmaf(p, x2, 7.97806978225708e-01f);
  const float hx = 0.5f * x;
  return fmaf(hx, tanh_approx(x * p), hx);
}

// The same GELU on a pair of values in FP16 arithmetic (packed: one instruction per pair
// for each step, one MUFU tanh per pair), for the 16-bit forms' hidden activations, whose
// result is rounded to a 16-bit type anyway.  Large |x| saturate through tanh(+-inf).
__device__ __forceinline__ __half2 gelu_h2(__half2 x) {
  const __half2 x2 = __hmul2(x, x);
  __half2 p = __hfma2(__float2half2_rn(9.163219942820433e-07f), x2, __float2half2_rn(-2.670336834853515e-05f));
  p = __hfma2(p, x2, __float2half2_rn(-1.468761620344594e-04f));
  p = __hfma2(p, x2, __float2half2_rn(3.6510955542325974e-02f));
  p = __hfma2(p, x2, __float2half2_rn(7.97806978225708e-01f));
  const __half2 hx = __hmul2(__float2half2_rn(0.5f), x);
  const __half2 z = __hmul2(x, p);
  uint32_t zi = *reinterpret_cast<const uint32_t*>(&z), ti;
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(ti) : "r"(zi));
  return __hfma2(hx, *reinterpret_cast<const __half2*>(&ti), hx);
}

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(bf16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(f16 v) { return __half2float(v); }
template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ bf16 from_f32<bf16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ f16 from_f32<f16>(float v) { return __float2half_rn(v); }

// The two 16-bit operand types of the tensor-core forms, BF16 (8-bit exponent, 8-bit
// significand) and FP16 (5-bit exponent, 11-bit significand): a pair of FP32 values packed
// into one 32-bit word (low half first, round to nearest even) and back, and the operand
// format code of the kind::f16 tcgen05 instruction descriptor (0 = F16, 1 = BF16).
template <typename T> struct H16;
template <> struct H16<bf16> {
  static constexpr uint32_t kMmaFmt = 1;
  static __device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ float2 unpack2(uint32_t v) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v));
  }
};
template <> struct H16<f16> {
  static constexpr uint32_t kMmaFmt = 0;
  static __device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ float2 unpack2(uint32_t v) {
    return __half22float2(*reinterpret_cast<const __half2*>(&v));
  }
};

// A pair of FP32 values rounded to FP16 (a in the low half), saturating at +-65504.
__device__ __forceinline__ __half2 f32x2_to_h2_satfinite(float a, float b) {
  uint32_t r;
  asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return *reinterpret_cast<const __half2*>(&r);
}

// GELU of a pair of FP32 values (evaluated by gelu_h2), packed in the 16-bit type T.
template <typename T>
__device__ __forceinline__ uint32_t gelu2_pack(float a, float b) {
  const __half2 r = gelu_h2(f32x2_to_h2_satfinite(a, b));
  if constexpr (sizeof(T) == 2 && H16<T>::kMmaFmt == 0) {
    return *reinterpret_cast<const uint32_t*>(&r);
  } else {
    const float2 f = __half22float2(r);
    return H16<T>::pack2(f.x, f.y);
  }
}

// D(16x8, f32) += A(16x16) . B(16x8) on the warp-level tensor-core instruction, with A and
// B in 16-bit type T (register fragments of mma.m16n8k16, row.col).
template <typename T>
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1);
template <>
__device__ __forceinline__ void mma16816<bf16>(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
template <>
__device__ __forceinline__ void mma16816<f16>(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------- launchers
// Every launcher enqueues on `st` and returns the cudaGetLastError() of its launch.

// Patch embedding + token-mask init.  x [B,3,H,W] f32, hole [B,H,W] u8 -> tok f32
// [B*Ht*Wt, d] (rows in raster token order), v0 u8 [B*Ht*Wt].
// With ln_out set, also writes LayerNorm(tok; ln_g, ln_b) in T (block 0's LN1).  T is the
// 16-bit type of the tensor-core forms (bf16 or f16); the FP32 form passes no ln_out.
template <typename T = bf16>
cudaError_t launch_embed(const float* x, const uint8_t* hole, int B, int H, int W, int Ht, int Wt,
                         const float* we, const float* be, int d, float* tok, uint8_t* v0, cudaStream_t st,
                         const float* ln_g = nullptr, const float* ln_b = nullptr, T* ln_out = nullptr);

// Tensor-core form of the patch embedding (16-bit forms): patches and weights in T
// (we16 = embed.w as T [d][64]), FP32 accumulation; writes tok, v0 and LN(tok)
// (without the affine part when ln_g is null: it is then folded into the next GEMM).
bool embed_tc_supported(int d);
template <typename T>
cudaError_t launch_embed_tc(const float* x, const uint8_t* hole, int B, int H, int W, int Ht, int Wt, const T* we16,
                            const float* be, int d, float* tok, uint8_t* v0, const float* ln_g, const float* ln_b,
                            T* ln_out, cudaStream_t st);

// LayerNorm over the last dim (eps 1e-5, biased variance, FP32 statistics).
template <typename OutT>
cudaError_t launch_layernorm(const float* x, const float* g, const float* b, OutT* y, int M, int d,
                             cudaStream_t st);

// FP32 SIMT GEMM C[M,N] = epi(A[M,K] . B[K,N]) with row-major A (lda) and B (ldb).
cudaError_t launch_gemm_f32(const float* A, int lda, const float* Bm, int ldb, float* C, int ldc,
                            int M, int N, int K, int epi, const float* bias, const float* resid,
                            cudaStream_t st);

// 16-bit tcgen05 GEMM C[M,N] = epi(A[M,K] . Bt[N,K]^T); A, Bt in T (bf16 or f16),
// K-contiguous.  Output: T for EPI_BIAS / EPI_BIAS_GELU, f32 for EPI_BIAS_RESID / EPI_NONE.
template <typename T>
cudaError_t launch_gemm_tc(const T* A, const T* Bt, void* C, int ldc, int M, int N, int K,
                           int epi, const float* bias, const float* resid, int* err, cudaStream_t st);

// Split-K form (FP32 partial products): C holds `splits` slices of round_up(M, 128) rows x N
// (row pitch N); slice s = A[:, ks .. ke) . Bt[:, ks .. ke)^T over its share of the K
// blocks of 64, to be summed in a fixed order.  1 <= splits <= K / 64.
cudaError_t launch_gemm_tc_splitk(const bf16* A, const bf16* Bt, float* C, int M, int N, int K, int splits, int* err,
                                  cudaStream_t st);

// Residual epilogue that also writes LayerNorm(x) (in T) of each finished row: X is
// updated in place (X = X + A.Bt^T + bias) and ln_out = LN(X; ln_g, ln_b).  N must be
// 64, 128 or 256 (one tile spans the row).
bool gemm_tc_ln_supported(int N);
template <typename T>
cudaError_t launch_gemm_tc_resid_ln(const T* A, const T* Bt, float* X, int M, int N, int K, const float* bias,
                                    const float* ln_g, const float* ln_b, T* ln_out, int* err, cudaStream_t st);

// Fused attention projection + MLP on tcgen05: x1 = X + A Wp + bp, Y = normalized x1
// (LN2 without its affine part, which is folded into W1t / b1), X = x1 + gelu(Y W1 + b1)
// W2 + b2 and ln_out = normalized X (times ln_g plus ln_b when they are given), without
// writing x1, Y or the hidden activations; Wpt [d][d], W1t [hid][d] and W2t [d][hid] in T
// (K-major), A [M][d] in T (bf16 or f16).  Supported for d in {64, 128, 256} and hid a
// multiple of 128 up to 1024.
bool mlp_tc_supported(int d, int hid);
template <typename T>
cudaError_t launch_proj_mlp_tc(const T* A, const T* Wpt, const float* bp, const T* W1t, const T* W2t,
                               const float* b1, const float* b2, float* X, const float* ln_g, const float* ln_b,
                               T* ln_out, int M, int d, int hid, int* err, cudaStream_t st);

// Mask-aware window attention of all frames; qkv [B*Nt, 3d] (T), v_in/v_out u8 [B*Nt].
// relpos (optional, device f32 [heads][15][15]): relative-position bias added to the
// score of query slot (qy, qx) and key slot (ky, kx) at [(ky - qy + 7) * 15 + kx - qx + 7].
template <typename T>
cudaError_t launch_attention(const T* qkv, const uint8_t* v_in, T* o, uint8_t* v_out, int B, int Ht,
                             int Wt, int d, int heads, int offset, cudaStream_t st, const float* relpos = nullptr);

// Tensor-core form for 16-bit activations T (bf16 or f16; mma.sync, FP32 softmax
// statistics); err (optional) receives DEV_MBAR_TIMEOUT if a window's TMA staging does not
// complete.
template <typename T>
cudaError_t launch_attention_tc(const T* qkv, const uint8_t* v_in, T* o, uint8_t* v_out, int B, int Ht,
                                int Wt, int d, int heads, int offset, cudaStream_t st,
                                const float* relpos = nullptr, int* err = nullptr);

// Spatial blocks of the 16-bit forms in one kernel: y (the block's normalized rows, T
// [B*Nt][d]) -> Q, K, V on tcgen05 (wqkv_t: W_qkv^T [3d][d] in T, bias [3d]) -> the same
// mask-aware window attention as launch_attention_tc, writing o and v_out; Q, K, V stay
// on chip.  Supported when d % 64 == 0, heads is even and at most 16 (d = 32 heads).
bool qkv_attn_supported(int d, int heads);
template <typename T>
cudaError_t launch_qkv_attn(const T* y, const T* wqkv_t, const float* bias, const uint8_t* v_in, T* o, uint8_t* v_out,
                            int B, int Ht, int Wt, int d, int heads, int offset, const float* relpos, int* err,
                            cudaStream_t st);

// Temporal blocks: as above, plus the keys of m memory slots.  tab->p[b*m + j] is a device
// pointer to a previous frame's memory buffer (null = empty slot; tab null = no memory);
// a buffer holds, at off_kv, k | v rows [Nt][2d] (T) and, at off_mask, the usable-key
// mask [Nt] of this block.  The table travels by value in the kernel parameters.
constexpr int MEM_TAB_MAX = 512;
struct MemTab {
  const uint8_t* p[MEM_TAB_MAX];
};
template <typename T>
cudaError_t launch_attention_mem(const T* qkv, const uint8_t* v_in, T* o, uint8_t* v_out, int B, int Ht, int Wt, int d,
                                 int heads, int offset, const MemTab* tab, int m, size_t off_kv, size_t off_mask,
                                 cudaStream_t st, const float* relpos = nullptr);
// The tensor-core form also records each frame's own memory tensor of this block: with
// out (host array [B], null entries skipped) it writes the k | v rows of the frame's tokens
// and the block's input key mask (v_in) at the same offsets off_kv / off_mask of out[b].
template <typename T>
cudaError_t launch_attention_tc_mem(const T* qkv, const uint8_t* v_in, T* o, uint8_t* v_out, int B, int Ht,
                                    int Wt, int d, int heads, int offset, const MemTab* tab, int m, size_t off_kv,
                                    size_t off_mask, uint8_t* const* out, cudaStream_t st,
                                    const float* relpos = nullptr, int* err = nullptr);

// Coloured point cloud (world x, y, z, r, g, b per pixel; NaN coordinates where the depth
// is not usable) and z-buffered splat into an Ho x Wo image.  cam / view: fx, fy, cx, cy;
// rt: R row-major (9) then t (3), host arrays.  keys: Ho*Wo scratch.
cudaError_t launch_point_cloud(const float* depth, const float* rgb, int H, int W, const float* cam, const float* rt,
                               float* pts, cudaStream_t st);
cudaError_t launch_splat(const float* pts, int64_t N, const float* view, const float* rt, int Ho, int Wo,
                         unsigned long long* keys, float* img, float* dep, int32_t* ind, cudaStream_t st);

// Decoder stage: out = gelu(conv3x3(upsample2(in)) + bias), NHWC.  wt: [9][Cin][Cout] f32.
template <typename T>
cudaError_t launch_upconv(const T* in, int B, int Hi, int Wi, int Cin, const float* wt,
                          const float* bias, T* out, int Cout, cudaStream_t st);

// Decoder stage on tcgen05 (sub-pixel implicit GEMM); wp = merged weights from
// launch_subpixel_weights ([4][Cout][4*Cin] in T, bf16 or f16).  Supported when Cin % 64
// == 0 and Cout is 32, 64, 96 or 128.
bool upconv_tc_supported(int Cin, int Cout);
template <typename T>
cudaError_t launch_subpixel_weights(const float* w, int Cout, int Cin, T* wp, cudaStream_t st);
template <typename T>
cudaError_t launch_upconv_tc(const T* in, int B, int Hi, int Wi, int Cin, const T* wp, const float* bias,
                             T* out, int Cout, int* err, cudaStream_t st);
// The same stage with the parities stacked on the MMA's M side (128 x 256 x 16 MMAs): ws =
// launch_stacked_weights's [groups][shifts][128][Cin] in T, upconv_t_weight_elems(Cin,
// Cout) elements (0 = unsupported).  Supported when Cin % 64 == 0, Cout is 32 or 64 and
// the input is at least 16 x 16 pixels.
bool upconv_t_supported(int Cin, int Cout, int Hi, int Wi);
size_t upconv_t_weight_elems(int Cin, int Cout);
template <typename T>
cudaError_t launch_stacked_weights(const float* w, int Cout, int Cin, T* ws, cudaStream_t st);
template <typename T>
cudaError_t launch_upconv_t(const T* in, int B, int Hi, int Wi, int Cin, const T* ws, const float* bias,
                            T* out, int Cout, int* err, cudaStream_t st);

// Generic FP32 3x3 conv (NHWC), optional x2 upsampling of the input, optional bias
// (NULL = none), act 0 = identity / 1 = GELU, optional pre-activation output.
cudaError_t launch_conv3x3_f32(const float* in, int B, int Hi, int Wi, int Cin, bool upsample, const float* wt,
                               const float* bias, int act, float* out, float* preact, int Cout, cudaStream_t st);

// FP32 SIMT GEMM with optional transposed operands and deterministic split-K: with
// splits > 1 the raw partial products go to C + s*M*ldc (s = split) for a later
// fixed-order reduction.
cudaError_t launch_gemm_f32_ex(bool ta, bool tb, const float* A, int lda, const float* Bm, int ldb, float* C, int ldc,
                               int M, int N, int K, int splits, int epi, const float* bias, const float* resid,
                               cudaStream_t st);

// Final 3x3 conv to RGB + composite + crop.  in NHWC [B,Hp,Wp,C]; wh [3][C][3][3] f32.
template <typename T>
cudaError_t launch_head_composite(const T* in, int B, int Hp, int Wp, int C, const float* wh,
                                  const float* bh, const float* x, const uint8_t* hole, int H, int W,
                                  float* out, float* pred, cudaStream_t st);

// Pre/post-processing around the half-resolution pass (see k_prepost.cu).
cudaError_t launch_mask_union(const uint8_t* masks, const uint8_t* selected, int B, int K, int h, int w, uint8_t* hole,
                              cudaStream_t st);
cudaError_t launch_downscale2(const float* x, int B, int H, int W, float* xh, cudaStream_t st);
cudaError_t launch_upscale_composite(const float* pred_h, const uint8_t* hole_h, const float* x, int B, int H, int W,
                                     float* out, cudaStream_t st);

// Hole-L1 loss: per-block partial sums into `partials` (>= loss_partials(n) floats),
// then a fixed-order final reduction into *loss.
int loss_partials(int B, int H, int W);
cudaError_t launch_l1_hole_loss(const float* out, const float* target, const uint8_t* hole, int B,
                                int H, int W, float* partials, unsigned* counts, float* loss,
                                float* grad, cudaStream_t st);

}  // namespace inpaint
