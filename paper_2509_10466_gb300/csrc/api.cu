// C ABI and runtime of the inpainting library: context, weight layouts, workspace
// planning, the forward sequence and event-based per-kernel timing.
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "context.cuh"
#include "tc_primitives.cuh"

namespace inpaint {
int backward_impl(inpaint_ctx* c, const float* x, const uint8_t* hole, const float* grad_out, int B, int H, int W,
                  float* grad_w, cudaStream_t st, const float* target = nullptr, float* loss = nullptr,
                  float* out = nullptr);
}  // namespace inpaint

using namespace inpaint;

// ------------------------------------------------------------------------- layout

namespace {

bool check_cfg(const inpaint_config* c) {
  if (!c) return false;
  if (c->window != 8 || c->patch != 4) return false;
  if (c->dim <= 0 || c->dim % 32 || c->heads <= 0 || c->dim != c->heads * 32) return false;
  if ((c->precision == INPAINT_BF16 || c->precision == INPAINT_FP16) && c->dim % 64)
    return false;  // tensor-core tiles are 64 wide
  if (c->blocks < 0 || c->blocks > 64 || c->mlp_ratio <= 0 || c->mlp_ratio > 16) return false;
  if (c->precision != INPAINT_FP32 && c->precision != INPAINT_BF16 && c->precision != INPAINT_FP16) return false;
  const int c1 = c->dec_c1 ? c->dec_c1 : c->dim / 4;
  const int c2 = c->dec_c2 ? c->dec_c2 : c->dim / 8;
  if (c1 <= 0 || c2 <= 0 || c1 % 4 || c2 % 4 || c1 > 4096 || c2 > 1024) return false;
  if (c->mem_slots < 0 || c->mem_slots > 4) return false;
  if (c->pos_bias != 0 && c->pos_bias != 1) return false;
  return true;
}

Offsets make_offsets(const inpaint_config& c) {
  const size_t d = c.dim, r = c.mlp_ratio;
  const size_t c1 = c.dec_c1 ? c.dec_c1 : d / 4, c2 = c.dec_c2 ? c.dec_c2 : d / 8;
  Offsets o;
  size_t p = 0;
  auto take = [&](size_t n) { size_t at = p; p += n; return at; };
  o.embw = take(d * 64);
  o.embb = take(d);
  for (int l = 0; l < c.blocks; ++l) {
    BlockOff b;
    b.ln1g = take(d); b.ln1b = take(d);
    b.qkvw = take(d * 3 * d); b.qkvb = take(3 * d);
    b.projw = take(d * d); b.projb = take(d);
    b.ln2g = take(d); b.ln2b = take(d);
    b.fc1w = take(d * r * d); b.fc1b = take(r * d);
    b.fc2w = take(r * d * d); b.fc2b = take(d);
    if (c.pos_bias) b.relpos = take((size_t)c.heads * 225);
    o.blk.push_back(b);
  }
  o.lnfg = take(d); o.lnfb = take(d);
  o.d1w = take(c1 * d * 9); o.d1b = take(c1);
  o.d2w = take(c2 * c1 * 9); o.d2b = take(c2);
  o.hw = take(3 * c2 * 9); o.hb = take(3);
  o.total = p;
  return o;
}

// Default weights from a seed (inpaint_init with NULL weights, inpaint_default_weights).
// Counter-based, so value i of the blob depends on (seed, i) only:
//   r  = mix(mix(seed) + i)   mix = the SplitMix64 output function (Steele, Lea and
//                             Flood 2014): z += 0x9E3779B97F4A7C15;
//                             z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
//                             z = (z ^ z>>27) * 0x94D049BB133111EB; z ^ z>>31
//   u1 = (r>>32 + 0.5) / 2^32,  u2 = (r & 0xFFFFFFFF + 0.5) / 2^32
//   z  = sqrt(-2 ln u1) cos(2 pi u2)                        (Box and Muller 1958, FP64)
// Matrices, conv kernels and relative-position tables: float(0.02 z); LayerNorm scales 1;
// biases and LayerNorm shifts 0.
uint64_t splitmix_out(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void default_weights(const inpaint_config& c, const Offsets& o, uint64_t seed, float* w) {
  const uint64_t key = splitmix_out(seed);
  auto normal = [&](size_t at, size_t n) {
    for (size_t i = at; i < at + n; ++i) {
      const uint64_t r = splitmix_out(key + (uint64_t)i);
      const double u1 = ((double)(r >> 32) + 0.5) * (1.0 / 4294967296.0);
      const double u2 = ((double)(r & 0xFFFFFFFFull) + 0.5) * (1.0 / 4294967296.0);
      const double z = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
      w[i] = (float)(0.02 * z);
    }
  };
  auto fill = [&](size_t at, size_t n, float v) {
    for (size_t i = at; i < at + n; ++i) w[i] = v;
  };
  const size_t d = c.dim, r = c.mlp_ratio;
  const size_t c1 = c.dec_c1 ? c.dec_c1 : d / 4, c2 = c.dec_c2 ? c.dec_c2 : d / 8;
  normal(o.embw, d * 64);
  fill(o.embb, d, 0.f);
  for (int l = 0; l < c.blocks; ++l) {
    const BlockOff& b = o.blk[l];
    fill(b.ln1g, d, 1.f); fill(b.ln1b, d, 0.f);
    normal(b.qkvw, d * 3 * d); fill(b.qkvb, 3 * d, 0.f);
    normal(b.projw, d * d); fill(b.projb, d, 0.f);
    fill(b.ln2g, d, 1.f); fill(b.ln2b, d, 0.f);
    normal(b.fc1w, d * r * d); fill(b.fc1b, r * d, 0.f);
    normal(b.fc2w, r * d * d); fill(b.fc2b, d, 0.f);
    if (c.pos_bias) normal(b.relpos, (size_t)c.heads * 225);
  }
  fill(o.lnfg, d, 1.f); fill(o.lnfb, d, 0.f);
  normal(o.d1w, c1 * d * 9); fill(o.d1b, c1, 0.f);
  normal(o.d2w, c2 * c1 * 9); fill(o.d2b, c2, 0.f);
  normal(o.hw, 3 * c2 * 9); fill(o.hb, 3, 0.f);
}

// out[n*K + k] = T(in[k*N + n])  (linear weight [in=K, out=N] -> K-major B operand)
// in [K][N] -> out [N][K] in the 16-bit type T, row k of `in` scaled by kscale[k] if given
template <typename T>
__global__ void transpose_to_h16(const float* __restrict__ in, T* __restrict__ out, int K, int N,
                                 const float* __restrict__ kscale) {
  __shared__ float t[32][33];
  const int k0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int k = k0 + i, n = n0 + threadIdx.x;
    t[i][threadIdx.x] = (k < K && n < N) ? in[(size_t)k * N + n] * (kscale ? kscale[k] : 1.f) : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int n = n0 + i, k = k0 + threadIdx.x;
    if (n < N && k < K) out[(size_t)n * K + k] = from_f32<T>(t[threadIdx.x][i]);
  }
}

// A LayerNorm's shift beta [K] folded into the bias of the linear layer W [K][N] that
// follows it: out[n] = b[n] + sum_k beta[k] W[k][n] (its scale goes into W itself).
__global__ void fold_bias_kernel(const float* __restrict__ W, const float* __restrict__ beta,
                                 const float* __restrict__ b, float* __restrict__ out, int K, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double acc = b[n];
  for (int k = 0; k < K; ++k) acc += (double)beta[k] * W[(size_t)k * N + n];
  out[n] = (float)acc;
}

// conv weight [Cout][Cin][9] -> [9][Cin][Cout]
__global__ void conv_w_to_tap_major(const float* __restrict__ in, float* __restrict__ out, int Cout, int Cin) {
  const size_t n = (size_t)Cout * Cin * 9;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int tap = (int)(e % 9);
    const size_t rest = e / 9;
    const int ci = (int)(rest % Cin), co = (int)(rest / Cin);
    out[((size_t)tap * Cin + ci) * Cout + co] = in[e];
  }
}

// [d][64] -> [64][d]
__global__ void transpose_f32(const float* __restrict__ in, float* __restrict__ out, int R, int C) {
  const size_t n = (size_t)R * C;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / C), c = (int)(e % C);
    out[(size_t)c * R + r] = in[e];
  }
}

}  // namespace

namespace inpaint {

static thread_local cudaError_t g_last_cuda_error = cudaSuccess;

int record_cuda_error(cudaError_t e) {
  if (e == cudaSuccess) return INPAINT_OK;
  g_last_cuda_error = e;
  return INPAINT_E_CUDA;
}

}  // namespace inpaint

namespace {

Plan make_plan(const inpaint_ctx* c, int B, int H, int W) {
  Plan p;
  p.B = B; p.H = H; p.W = W;
  p.Hp = (H + 31) / 32 * 32;
  p.Wp = (W + 31) / 32 * 32;
  p.Ht = p.Hp / 4;
  p.Wt = p.Wp / 4;
  p.Nt = p.Ht * p.Wt;
  p.M = B * p.Nt;
  const size_t es = c->use_tc ? 2 : 4;
  const size_t M = p.M, d = c->d;
  size_t q = 0;
  auto take = [&](size_t bytes) { size_t at = q; q = align_up(q + bytes, 256); return at; };
  p.tok = take(M * d * 4);
  p.ln = take(M * d * es);
  p.qkv = take(M * 3 * d * es);
  p.o = take(M * d * es);
  p.hid = take(M * (size_t)c->hid * es);
  p.masks = take((size_t)(c->L + 1) * M);
  p.f1 = take((size_t)B * (2 * p.Ht) * (2 * p.Wt) * c->c1 * es);
  p.f2 = take((size_t)B * p.Hp * p.Wp * c->c2 * es);
  p.err = take(256);
  p.end = q;
  return p;
}

MemLayout mem_layout(const inpaint_ctx* c, int Nt) {
  const size_t es = c->use_tc ? 2 : 4;
  MemLayout m;
  m.kv_bytes = (size_t)Nt * 2 * c->d * es;
  m.stride = align_up(m.kv_bytes + Nt, 256);
  m.total = (size_t)(c->L / 2) * m.stride;
  return m;
}

int cuda_err(cudaError_t e) { return record_cuda_error(e); }

#define TRY(call)                          \
  do {                                     \
    int rc_ = (call);                      \
    if (rc_ != INPAINT_OK) return rc_;     \
  } while (0)

// Derived weight copies of a 16-bit form (operand type T).
template <typename T>
int prepare_layouts_h16(inpaint_ctx* c, cudaStream_t st) {
  const Offsets& o = c->off;
  if (c->embed_w16) {
    // embed.w [d][64] in T = the transpose of the [64][d] FP32 copy
    transpose_to_h16<T><<<dim3(cdiv(c->d, 32), cdiv(64, 32)), dim3(32, 8), 0, st>>>(
        c->embed_wt, reinterpret_cast<T*>(c->embed_w16), 64, c->d, nullptr);
  }
  if (c->dec1_wp &&
      launch_subpixel_weights<T>(c->w32 + o.d1w, c->c1, c->d, reinterpret_cast<T*>(c->dec1_wp), st) != cudaSuccess)
    return INPAINT_E_CUDA;
  if (c->dec2_wp &&
      launch_subpixel_weights<T>(c->w32 + o.d2w, c->c2, c->c1, reinterpret_cast<T*>(c->dec2_wp), st) != cudaSuccess)
    return INPAINT_E_CUDA;
  if (c->dec1_ws &&
      launch_stacked_weights<T>(c->w32 + o.d1w, c->c1, c->d, reinterpret_cast<T*>(c->dec1_ws), st) != cudaSuccess)
    return INPAINT_E_CUDA;
  if (c->dec2_ws &&
      launch_stacked_weights<T>(c->w32 + o.d2w, c->c2, c->c1, reinterpret_cast<T*>(c->dec2_ws), st) != cudaSuccess)
    return INPAINT_E_CUDA;
  const int d = c->d, h = c->hid;
  for (int l = 0; l < c->L; ++l) {
    T* base = reinterpret_cast<T*>(c->lin16) + (size_t)l * c->lin_block_elems;
    const BlockOff& b = o.blk[l];
    const float* g1 = c->fold_ln ? c->w32 + b.ln1g : nullptr;
    const float* g2 = c->fold_ln ? c->w32 + b.ln2g : nullptr;
    struct { size_t src; int K, N; size_t dst; const float* kscale; } mats[4] = {
        {b.qkvw, d, 3 * d, 0, g1},
        {b.projw, d, d, (size_t)3 * d * d, nullptr},
        {b.fc1w, d, h, (size_t)4 * d * d, g2},
        {b.fc2w, h, d, (size_t)4 * d * d + (size_t)h * d, nullptr}};
    for (auto& m : mats) {
      dim3 grid(cdiv(m.N, 32), cdiv(m.K, 32));
      transpose_to_h16<T><<<grid, dim3(32, 8), 0, st>>>(c->w32 + m.src, base + m.dst, m.K, m.N, m.kscale);
    }
    if (c->fold_ln) {
      float* fb = c->fold_b + (size_t)l * (3 * d + h);
      fold_bias_kernel<<<cdiv(3 * d, 128), 128, 0, st>>>(c->w32 + b.qkvw, c->w32 + b.ln1b, c->w32 + b.qkvb, fb, d,
                                                         3 * d);
      fold_bias_kernel<<<cdiv(h, 128), 128, 0, st>>>(c->w32 + b.fc1w, c->w32 + b.ln2b, c->w32 + b.fc1b, fb + 3 * d, d,
                                                     h);
    }
  }
  return INPAINT_OK;
}

int prepare_layouts(inpaint_ctx* c, cudaStream_t st) {
  const Offsets& o = c->off;
  transpose_f32<<<64, 256, 0, st>>>(c->w32 + o.embw, c->embed_wt, c->d, 64);
  conv_w_to_tap_major<<<256, 256, 0, st>>>(c->w32 + o.d1w, c->dec1_wt, c->c1, c->d);
  conv_w_to_tap_major<<<256, 256, 0, st>>>(c->w32 + o.d2w, c->dec2_wt, c->c2, c->c1);
  if (c->use_tc) TRY(c->fp16 ? prepare_layouts_h16<f16>(c, st) : prepare_layouts_h16<bf16>(c, st));
  return cuda_err(cudaGetLastError());
}

// The whole forward pass into workspace `ws` laid out by plan `p`, with activations of
// type A: float for the FP32 SIMT form, bf16 or f16 for the 16-bit tensor-core forms.
template <typename A>
int run_forward_t(inpaint_ctx* c, uint8_t* ws, const Plan& p, const float* x, const uint8_t* hole, float* out,
                  float* pred, cudaStream_t st, const MemArgs* mem, const FramePipe* pipe) {
  constexpr bool TC = sizeof(A) == 2;
  const Offsets& o = c->off;
  const int d = c->d, M = p.M;
  float* tok = reinterpret_cast<float*>(ws + p.tok);
  uint8_t* masks = ws + p.masks;
  int* err = c->dev_err;
  // 16-bit forms: the embedding also writes the first LayerNorm (block 0's LN1, or the
  // final LN when there are no blocks) straight into the 16-bit GEMM operand
  bool ln_ready = TC;
  // frames f0 .. f0 + nb - 1 (the whole batch, or frame by frame behind the input copies)
  auto embed = [&](int f0, int nb) -> int {
    const size_t HW = (size_t)p.H * p.W, nt = (size_t)p.Ht * p.Wt;
    const float* xf = x + f0 * 3 * HW;
    const uint8_t* hf = hole + f0 * HW;
    float* tf = tok + f0 * nt * d;
    uint8_t* mf = masks + f0 * nt;
    LaunchScope ls(c, st, K_EMBED);
    if constexpr (TC) {
      // with folding, block 0's LN1 affine lives in its QKV weights: normalized rows only
      const float* g0 = c->fold_ln ? nullptr : c->w32 + (c->L ? o.blk[0].ln1g : o.lnfg);
      const float* b0 = c->fold_ln ? nullptr : c->w32 + (c->L ? o.blk[0].ln1b : o.lnfb);
      A* lf = reinterpret_cast<A*>(ws + p.ln) + f0 * nt * d;
      if (c->embed_w16)
        return cuda_err(launch_embed_tc<A>(xf, hf, nb, p.H, p.W, p.Ht, p.Wt, reinterpret_cast<const A*>(c->embed_w16),
                                           c->w32 + o.embb, d, tf, mf, g0, b0, lf, st));
      return cuda_err(launch_embed<A>(xf, hf, nb, p.H, p.W, p.Ht, p.Wt, c->embed_wt, c->w32 + o.embb, d, tf, mf, st, g0,
                                      b0, lf));
    } else {
      return cuda_err(launch_embed(xf, hf, nb, p.H, p.W, p.Ht, p.Wt, c->embed_wt, c->w32 + o.embb, d, tf, mf, st));
    }
  };
  if (pipe) {
    for (int f = 0; f < p.B; ++f) {
      TRY(cuda_err(cudaStreamWaitEvent(st, pipe->in_ready[f], 0)));
      TRY(embed(f, 1));
    }
  } else {
    TRY(embed(0, p.B));
  }
  // the 3x3 head + composite + crop, for the whole batch or frame by frame (each frame's
  // output then announced to the copy stream)
  auto head = [&](const auto* f2) -> int {
    using F = std::remove_cv_t<std::remove_pointer_t<decltype(f2)>>;
    const size_t HW = (size_t)p.H * p.W, fin = (size_t)p.Hp * p.Wp * c->c2;
    const int nf = pipe ? p.B : 1, nb = pipe ? 1 : p.B;
    for (int f = 0; f < nf; ++f) {
      {
        LaunchScope ls(c, st, K_HEAD);
        TRY(cuda_err(launch_head_composite<F>(f2 + f * fin, nb, p.Hp, p.Wp, c->c2, c->w32 + o.hw, c->w32 + o.hb,
                                              x + f * 3 * HW, hole + f * HW, p.H, p.W, out + f * 3 * HW,
                                              pred ? pred + f * 3 * HW : nullptr, st)));
      }
      if (pipe) TRY(cuda_err(cudaEventRecord(pipe->out_ready[f], st)));
    }
    return INPAINT_OK;
  };
  // 16-bit forms: the LayerNorm that follows each residual update is fused into the GEMM
  // epilogue that produces it (proj -> LN2, fc2 -> next LN1 or the final LN) when a
  // tile spans the whole row; `ln_ready` tracks whether `ln` already holds the input
  // LayerNorm of the next GEMM.
  const bool fuse_ln = TC && gemm_tc_ln_supported(d);
  for (int l = 0; l < c->L; ++l) {
    const BlockOff& b = o.blk[l];
    const int offset = (c->cfg.shift && (l & 1)) ? 4 : 0;
    uint8_t* v_in = masks + (size_t)l * M;
    uint8_t* v_out = masks + (size_t)(l + 1) * M;
    // temporal block: the queries also see the memory slots' keys of this block, and each
    // frame's own k | v and key mask here become part of its memory tensor
    const bool temporal = c->cfg.mem_slots > 0 && (l & 1);
    const float* rp = c->cfg.pos_bias ? c->w32 + b.relpos : nullptr;
    const MemTab* mtab = mem ? mem->tab : nullptr;
    const size_t moff = mem ? (size_t)(l / 2) * mem->lay.stride : 0, mkv = mem ? mem->lay.kv_bytes : 0;
    auto record_memory = [&](const void* qkv_any) -> int {
      if (!mem || !mem->out) return INPAINT_OK;
      const size_t es = sizeof(A);
      const uint8_t* q8 = static_cast<const uint8_t*>(qkv_any);
      for (int b = 0; b < p.B; ++b) {
        uint8_t* dst = mem->out[b];
        if (!dst) continue;
        const uint8_t* src = q8 + ((size_t)b * p.Nt * 3 * d + d) * es;
        if (cudaMemcpy2DAsync(dst + moff, 2 * d * es, src, 3 * d * es, 2 * d * es, p.Nt, cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(dst + moff + mkv, v_in + (size_t)b * p.Nt, p.Nt, cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess)
          return INPAINT_E_CUDA;
      }
      return INPAINT_OK;
    };
    if constexpr (TC) {
      A* ln = reinterpret_cast<A*>(ws + p.ln);
      A* qkv = reinterpret_cast<A*>(ws + p.qkv);
      A* ao = reinterpret_cast<A*>(ws + p.o);
      A* hid = reinterpret_cast<A*>(ws + p.hid);
      const A* wl = reinterpret_cast<const A*>(c->lin16) + (size_t)l * c->lin_block_elems;
      const A* wqkv = wl;
      const A* wproj = wl + (size_t)3 * d * d;
      const A* wfc1 = wl + (size_t)4 * d * d;
      const A* wfc2 = wfc1 + (size_t)c->hid * d;
      if (!ln_ready) { LaunchScope ls(c, st, K_LN); TRY(cuda_err(launch_layernorm<A>(tok, c->w32 + b.ln1g, c->w32 + b.ln1b, ln, M, d, st))); }
      const float* fold = c->fold_ln ? c->fold_b + (size_t)l * (3 * d + c->hid) : nullptr;
      const float* qkv_bias = fold ? fold : c->w32 + b.qkvb;
      if (!temporal && qkv_attn_supported(d, c->heads)) {
        // spatial block: Q, K, V computed and consumed on chip, per pair of windows
        LaunchScope ls(c, st, K_QKV_ATTN);
        TRY(cuda_err(launch_qkv_attn<A>(ln, wqkv, qkv_bias, v_in, ao, v_out, p.B, p.Ht, p.Wt, d, c->heads, offset, rp, err, st)));
      } else {
      { LaunchScope ls(c, st, K_QKV); TRY(cuda_err(launch_gemm_tc(ln, wqkv, qkv, 3 * d, M, 3 * d, d, EPI_BIAS, qkv_bias, nullptr, err, st))); }
      if (temporal) {
        LaunchScope ls(c, st, K_ATTN);
        // the kernel also records this block's part of each frame's memory tensor
        TRY(cuda_err(launch_attention_tc_mem<A>(qkv, v_in, ao, v_out, p.B, p.Ht, p.Wt, d, c->heads, offset, mtab, c->cfg.mem_slots, moff, moff + mkv, mem ? mem->out : nullptr, st, rp, err)));
      } else {
        LaunchScope ls(c, st, K_ATTN);
        TRY(cuda_err(launch_attention_tc(qkv, v_in, ao, v_out, p.B, p.Ht, p.Wt, d, c->heads, offset, st, rp, err)));
      }
      }
      if (c->fold_ln) {
        // projection, residual, LN2 and the whole MLP in one kernel: only the attention
        // output and the residual row come in, only the new residual row and its LN leave
        // (normalized only: the next block's LN1 affine is folded too; the final LN keeps it)
        const bool last = l + 1 == c->L;
        const float* ng = last ? c->w32 + o.lnfg : nullptr;
        const float* nb = last ? c->w32 + o.lnfb : nullptr;
        LaunchScope ls(c, st, K_MLP);
        TRY(cuda_err(launch_proj_mlp_tc(ao, wproj, c->w32 + b.projb, wfc1, wfc2, fold + 3 * d, c->w32 + b.fc2b, tok,
                                        ng, nb, ln, M, d, c->hid, err, st)));
        ln_ready = true;
        continue;
      }
      if (fuse_ln) {
        LaunchScope ls(c, st, K_PROJ);
        TRY(cuda_err(launch_gemm_tc_resid_ln(ao, wproj, tok, M, d, d, c->w32 + b.projb, c->w32 + b.ln2g, c->w32 + b.ln2b, ln, err, st)));
      } else {
        { LaunchScope ls(c, st, K_PROJ); TRY(cuda_err(launch_gemm_tc(ao, wproj, tok, d, M, d, d, EPI_BIAS_RESID, c->w32 + b.projb, tok, err, st))); }
        { LaunchScope ls(c, st, K_LN); TRY(cuda_err(launch_layernorm<A>(tok, c->w32 + b.ln2g, c->w32 + b.ln2b, ln, M, d, st))); }
      }
      { LaunchScope ls(c, st, K_FC1); TRY(cuda_err(launch_gemm_tc(ln, wfc1, hid, c->hid, M, c->hid, d, EPI_BIAS_GELU, c->w32 + b.fc1b, nullptr, err, st))); }
      if (fuse_ln) {
        const bool last = l + 1 == c->L;
        const float* ng = c->w32 + (last ? o.lnfg : o.blk[l + 1].ln1g);
        const float* nb = c->w32 + (last ? o.lnfb : o.blk[l + 1].ln1b);
        LaunchScope ls(c, st, K_FC2);
        TRY(cuda_err(launch_gemm_tc_resid_ln(hid, wfc2, tok, M, d, c->hid, c->w32 + b.fc2b, ng, nb, ln, err, st)));
        ln_ready = true;
      } else {
        LaunchScope ls(c, st, K_FC2);
        TRY(cuda_err(launch_gemm_tc(hid, wfc2, tok, d, M, d, c->hid, EPI_BIAS_RESID, c->w32 + b.fc2b, tok, err, st)));
        ln_ready = false;
      }
    } else {
      float* ln = reinterpret_cast<float*>(ws + p.ln);
      float* qkv = reinterpret_cast<float*>(ws + p.qkv);
      float* ao = reinterpret_cast<float*>(ws + p.o);
      float* hid = reinterpret_cast<float*>(ws + p.hid);
      { LaunchScope ls(c, st, K_LN); TRY(cuda_err(launch_layernorm<float>(tok, c->w32 + b.ln1g, c->w32 + b.ln1b, ln, M, d, st))); }
      { LaunchScope ls(c, st, K_QKV); TRY(cuda_err(launch_gemm_f32(ln, d, c->w32 + b.qkvw, 3 * d, qkv, 3 * d, M, 3 * d, d, EPI_BIAS, c->w32 + b.qkvb, nullptr, st))); }
      if (temporal) {
        LaunchScope ls(c, st, K_ATTN);
        TRY(cuda_err(launch_attention_mem<float>(qkv, v_in, ao, v_out, p.B, p.Ht, p.Wt, d, c->heads, offset, mtab, c->cfg.mem_slots, moff, moff + mkv, st, rp)));
      } else {
        LaunchScope ls(c, st, K_ATTN);
        TRY(cuda_err(launch_attention<float>(qkv, v_in, ao, v_out, p.B, p.Ht, p.Wt, d, c->heads, offset, st, rp)));
      }
      if (temporal) TRY(record_memory(qkv));
      { LaunchScope ls(c, st, K_PROJ); TRY(cuda_err(launch_gemm_f32(ao, d, c->w32 + b.projw, d, tok, d, M, d, d, EPI_BIAS_RESID, c->w32 + b.projb, tok, st))); }
      { LaunchScope ls(c, st, K_LN); TRY(cuda_err(launch_layernorm<float>(tok, c->w32 + b.ln2g, c->w32 + b.ln2b, ln, M, d, st))); }
      { LaunchScope ls(c, st, K_FC1); TRY(cuda_err(launch_gemm_f32(ln, d, c->w32 + b.fc1w, c->hid, hid, c->hid, M, c->hid, d, EPI_BIAS_GELU, c->w32 + b.fc1b, nullptr, st))); }
      { LaunchScope ls(c, st, K_FC2); TRY(cuda_err(launch_gemm_f32(hid, c->hid, c->w32 + b.fc2w, d, tok, d, M, d, c->hid, EPI_BIAS_RESID, c->w32 + b.fc2b, tok, st))); }
    }
  }
  if constexpr (TC) {
    A* ln = reinterpret_cast<A*>(ws + p.ln);
    A* f1 = reinterpret_cast<A*>(ws + p.f1);
    A* f2 = reinterpret_cast<A*>(ws + p.f2);
    const A* dec1_ws = reinterpret_cast<const A*>(c->dec1_ws);
    const A* dec2_ws = reinterpret_cast<const A*>(c->dec2_ws);
    const A* dec1_wp = reinterpret_cast<const A*>(c->dec1_wp);
    const A* dec2_wp = reinterpret_cast<const A*>(c->dec2_wp);
    if (!ln_ready) { LaunchScope ls(c, st, K_LN); TRY(cuda_err(launch_layernorm<A>(tok, c->w32 + o.lnfg, c->w32 + o.lnfb, ln, M, d, st))); }
    if (c->dec1_ws && upconv_t_supported(d, c->c1, p.Ht, p.Wt)) {
      LaunchScope ls(c, st, K_DEC1);
      TRY(cuda_err(launch_upconv_t<A>(ln, p.B, p.Ht, p.Wt, d, dec1_ws, c->w32 + o.d1b, f1, c->c1, c->dev_err, st)));
    } else if (c->dec1_wp && p.Wt >= 16 && p.Ht >= 8) {  // TMA box is 16 x 8 input pixels
      LaunchScope ls(c, st, K_DEC1);
      TRY(cuda_err(launch_upconv_tc<A>(ln, p.B, p.Ht, p.Wt, d, dec1_wp, c->w32 + o.d1b, f1, c->c1, c->dev_err, st)));
    } else {
      LaunchScope ls(c, st, K_DEC1);
      TRY(cuda_err(launch_upconv<A>(ln, p.B, p.Ht, p.Wt, d, c->dec1_wt, c->w32 + o.d1b, f1, c->c1, st)));
    }
    if (c->dec2_ws && upconv_t_supported(c->c1, c->c2, 2 * p.Ht, 2 * p.Wt)) {
      LaunchScope ls(c, st, K_DEC2);
      TRY(cuda_err(launch_upconv_t<A>(f1, p.B, 2 * p.Ht, 2 * p.Wt, c->c1, dec2_ws, c->w32 + o.d2b, f2, c->c2, c->dev_err, st)));
    } else if (c->dec2_wp) {
      LaunchScope ls(c, st, K_DEC2);
      TRY(cuda_err(launch_upconv_tc<A>(f1, p.B, 2 * p.Ht, 2 * p.Wt, c->c1, dec2_wp, c->w32 + o.d2b, f2, c->c2, c->dev_err, st)));
    } else {
      LaunchScope ls(c, st, K_DEC2);
      TRY(cuda_err(launch_upconv<A>(f1, p.B, 2 * p.Ht, 2 * p.Wt, c->c1, c->dec2_wt, c->w32 + o.d2b, f2, c->c2, st)));
    }
    TRY(head(f2));
  } else {
    float* ln = reinterpret_cast<float*>(ws + p.ln);
    float* f1 = reinterpret_cast<float*>(ws + p.f1);
    float* f2 = reinterpret_cast<float*>(ws + p.f2);
    { LaunchScope ls(c, st, K_LN); TRY(cuda_err(launch_layernorm<float>(tok, c->w32 + o.lnfg, c->w32 + o.lnfb, ln, M, d, st))); }
    { LaunchScope ls(c, st, K_DEC1); TRY(cuda_err(launch_upconv<float>(ln, p.B, p.Ht, p.Wt, d, c->dec1_wt, c->w32 + o.d1b, f1, c->c1, st))); }
    { LaunchScope ls(c, st, K_DEC2); TRY(cuda_err(launch_upconv<float>(f1, p.B, 2 * p.Ht, 2 * p.Wt, c->c1, c->dec2_wt, c->w32 + o.d2b, f2, c->c2, st))); }
    TRY(head(f2));
  }
  return INPAINT_OK;
}

int run_forward(inpaint_ctx* c, uint8_t* ws, const Plan& p, const float* x, const uint8_t* hole, float* out,
                float* pred, cudaStream_t st, const MemArgs* mem = nullptr, const FramePipe* pipe = nullptr) {
  if (!c->use_tc) return run_forward_t<float>(c, ws, p, x, hole, out, pred, st, mem, pipe);
  if (c->fp16) return run_forward_t<f16>(c, ws, p, x, hole, out, pred, st, mem, pipe);
  return run_forward_t<bf16>(c, ws, p, x, hole, out, pred, st, mem, pipe);
}

bool bad_shape(int B, int H, int W) {
  return B < 1 || H < 1 || W < 1 || H > 16384 || W > 16384 || (size_t)B * H * W > ((size_t)1 << 34);
}

}  // namespace

// ------------------------------------------------------------------------- C ABI

extern "C" {

int inpaint_last_cuda_error(void) { return (int)g_last_cuda_error; }

const char* inpaint_cuda_error_name(int cuda_error) { return cudaGetErrorName((cudaError_t)cuda_error); }

const char* inpaint_strerror(int code) {
  switch (code) {
    case INPAINT_OK: return "ok";
    case INPAINT_E_INVAL: return "invalid argument or unsupported configuration";
    case INPAINT_E_NOMEM: return "device memory allocation failed or exceeds the context's HBM budget";
    case INPAINT_E_CUDA: return "CUDA runtime error";
    case INPAINT_E_TIMEOUT: return "deadline passed before the stream finished";
    case INPAINT_E_STATE: return "call not valid in the current state";
    case INPAINT_E_DEVICE: return "a kernel reported a device-side error (bounded wait expired)";
    default: return "unknown error code";
  }
}

int inpaint_num_params(const inpaint_config* cfg, size_t* n) {
  if (!check_cfg(cfg) || !n) return INPAINT_E_INVAL;
  *n = make_offsets(*cfg).total;
  return INPAINT_OK;
}

int inpaint_default_weights(const inpaint_config* cfg, uint64_t seed, float* host_out, size_t n) {
  if (!check_cfg(cfg) || !host_out) return INPAINT_E_INVAL;
  const Offsets o = make_offsets(*cfg);
  if (n < o.total) return INPAINT_E_INVAL;
  default_weights(*cfg, o, seed, host_out);
  return INPAINT_OK;
}

void inpaint_destroy(inpaint_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  cudaFree(c->w32);
  cudaFree(c->embed_wt);
  cudaFree(c->dec1_wt);
  cudaFree(c->dec2_wt);
  cudaFree(c->lin16);
  cudaFree(c->fold_b);
  cudaFree(c->dec1_wp);
  cudaFree(c->embed_w16);
  cudaFree(c->dec2_wp);
  cudaFree(c->dec1_ws);
  cudaFree(c->dec2_ws);
  cudaFree(c->dev_err);
  cudaFree(c->arena);
  cudaFree(c->stage);
  cudaFree(c->bws);
  cudaFree(c->pp);
  cudaFree(c->zbuf);
  for (auto& e : c->events) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (cudaEvent_t e : c->in_ev) cudaEventDestroy(e);
  for (cudaEvent_t e : c->out_ev) cudaEventDestroy(e);
  if (c->start_ev) cudaEventDestroy(c->start_ev);
  if (c->done_ev) cudaEventDestroy(c->done_ev);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  delete c;
}

int inpaint_init(const inpaint_config* cfg, const float* weights, size_t n_weights, inpaint_ctx** out) {
  if (!out) return INPAINT_E_INVAL;
  *out = nullptr;
  if (!check_cfg(cfg)) return INPAINT_E_INVAL;
  inpaint_ctx* c = new (std::nothrow) inpaint_ctx();
  if (!c) return INPAINT_E_NOMEM;
  c->cfg = *cfg;
  c->d = cfg->dim;
  c->heads = cfg->heads;
  c->L = cfg->blocks;
  c->r = cfg->mlp_ratio;
  c->hid = cfg->dim * cfg->mlp_ratio;
  c->c1 = cfg->dec_c1 ? cfg->dec_c1 : cfg->dim / 4;
  c->c2 = cfg->dec_c2 ? cfg->dec_c2 : cfg->dim / 8;
  c->use_tc = cfg->precision == INPAINT_BF16 || cfg->precision == INPAINT_FP16;
  c->fp16 = cfg->precision == INPAINT_FP16;
  c->off = make_offsets(*cfg);
  c->nparams = c->off.total;
  std::vector<float> generated;
  if (!weights) {  // the documented default blob of cfg->seed
    if (n_weights != 0 && n_weights != c->nparams) {
      delete c;
      return INPAINT_E_INVAL;
    }
    try {
      generated.resize(c->nparams);
    } catch (...) {
      delete c;
      return INPAINT_E_NOMEM;
    }
    default_weights(*cfg, c->off, cfg->seed, generated.data());
    weights = generated.data();
  } else if (n_weights != c->nparams) {
    delete c;
    return INPAINT_E_INVAL;
  }
  const size_t d = c->d, h = c->hid;
  c->lin_block_elems = 4 * d * d + 2 * h * d;
  c->fold_ln = c->use_tc && c->L > 0 && gemm_tc_ln_supported(c->d) && mlp_tc_supported(c->d, c->hid) &&
               embed_tc_supported(c->d);
  c->weight_bytes = c->nparams * 4 + 64 * d * 4 + 9 * d * c->c1 * 4 + 9 * (size_t)c->c1 * c->c2 * 4 +
                    (c->use_tc ? (size_t)c->L * c->lin_block_elems * 2 + (size_t)32 * (c->c1 * d + c->c2 * c->c1) + 128 * d : 0) +
                    (c->fold_ln ? (size_t)c->L * (3 * d + h) * 4 : 0) +
                    (c->use_tc ? 2 * (upconv_t_weight_elems(d, c->c1) + upconv_t_weight_elems(c->c1, c->c2)) : 0) +
                    256;
  if (cfg->hbm_budget_bytes && c->weight_bytes > cfg->hbm_budget_bytes) {
    delete c;
    return INPAINT_E_NOMEM;
  }
  bool ok = cudaMalloc(&c->w32, c->nparams * 4) == cudaSuccess &&
            cudaMalloc(&c->embed_wt, 64 * d * 4) == cudaSuccess &&
            cudaMalloc(&c->dec1_wt, 9 * d * c->c1 * 4) == cudaSuccess &&
            cudaMalloc(&c->dec2_wt, 9 * (size_t)c->c1 * c->c2 * 4) == cudaSuccess &&
            cudaMalloc(&c->dev_err, 256) == cudaSuccess &&
            (!c->use_tc || cudaMalloc(&c->lin16, (size_t)c->L * c->lin_block_elems * 2) == cudaSuccess) &&
            (!c->fold_ln || cudaMalloc(&c->fold_b, (size_t)c->L * (3 * d + h) * 4) == cudaSuccess) &&
            (!c->use_tc || !embed_tc_supported(c->d) || cudaMalloc(&c->embed_w16, 64 * d * 2) == cudaSuccess) &&
            (!c->use_tc || !upconv_tc_supported(c->d, c->c1) ||
             cudaMalloc(&c->dec1_wp, (size_t)16 * c->c1 * c->d * 2) == cudaSuccess) &&
            (!c->use_tc || !upconv_tc_supported(c->c1, c->c2) ||
             cudaMalloc(&c->dec2_wp, (size_t)16 * c->c2 * c->c1 * 2) == cudaSuccess) &&
            (!c->use_tc || !upconv_t_weight_elems(c->d, c->c1) ||
             cudaMalloc(&c->dec1_ws, upconv_t_weight_elems(c->d, c->c1) * 2) == cudaSuccess) &&
            (!c->use_tc || !upconv_t_weight_elems(c->c1, c->c2) ||
             cudaMalloc(&c->dec2_ws, upconv_t_weight_elems(c->c1, c->c2) * 2) == cudaSuccess);
  if (!ok) {
    cudaGetLastError();
    inpaint_destroy(c);
    return INPAINT_E_NOMEM;
  }
  if (cudaMemcpy(c->w32, weights, c->nparams * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->dev_err, 0, 256) != cudaSuccess || prepare_layouts(c, 0) != INPAINT_OK ||
      cudaDeviceSynchronize() != cudaSuccess) {
    inpaint_destroy(c);
    return INPAINT_E_CUDA;
  }
  *out = c;
  return INPAINT_OK;
}

int inpaint_set_weights(inpaint_ctx* c, const float* w, int on_device, void* stream) {
  if (!c || !w) return INPAINT_E_INVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (on_device) {
    if (cudaMemcpyAsync(c->w32, w, c->nparams * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return INPAINT_E_CUDA;
    return prepare_layouts(c, st);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return INPAINT_E_CUDA;
  if (cudaMemcpy(c->w32, w, c->nparams * 4, cudaMemcpyHostToDevice) != cudaSuccess) return INPAINT_E_CUDA;
  TRY(prepare_layouts(c, st));
  return cuda_err(cudaStreamSynchronize(st));
}

int inpaint_get_weights(inpaint_ctx* c, float* host) {
  if (!c || !host) return INPAINT_E_INVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return INPAINT_E_CUDA;
  return cuda_err(cudaMemcpy(host, c->w32, c->nparams * 4, cudaMemcpyDeviceToHost));
}

int inpaint_workspace_bytes(inpaint_ctx* c, int B, int H, int W, size_t* bytes) {
  if (!c || !bytes || bad_shape(B, H, W)) return INPAINT_E_INVAL;
  *bytes = make_plan(c, B, H, W).end;
  return INPAINT_OK;
}

int inpaint_batch(inpaint_ctx* c, const float* x, const uint8_t* hole, int B, int H, int W, float* out, float* pred,
                  void* stream) {
  if (!c || !x || !hole || !out || bad_shape(B, H, W)) return INPAINT_E_INVAL;
  const Plan p = make_plan(c, B, H, W);
  TRY(grow(&c->arena, &c->arena_bytes, p.end, c, c->stage_bytes + c->bws_bytes));
  c->have_masks = false;
  TRY(run_forward(c, c->arena, p, x, hole, out, pred, (cudaStream_t)stream));
  c->last = p;
  c->have_masks = true;
  return INPAINT_OK;
}

int inpaint_memory_bytes(inpaint_ctx* c, int H, int W, size_t* bytes) {
  if (!c || !bytes || bad_shape(1, H, W)) return INPAINT_E_INVAL;
  *bytes = c->cfg.mem_slots > 0 ? mem_layout(c, make_plan(c, 1, H, W).Nt).total : 0;
  return INPAINT_OK;
}

int inpaint_batch_mem(inpaint_ctx* c, void* workspace, size_t ws_bytes, const float* x, const uint8_t* hole, int B,
                      int H, int W, float* out, float* pred, const void* const* mem_in, void* const* mem_out,
                      void* stream) {
  if (!c || !x || !hole || !out || bad_shape(B, H, W)) return INPAINT_E_INVAL;
  if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255)) return INPAINT_E_INVAL;
  const int m = c->cfg.mem_slots;
  if (m == 0 && (mem_in || mem_out)) return INPAINT_E_INVAL;
  auto misaligned = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 255) != 0; };
  if (mem_in && (size_t)B * m > (size_t)MEM_TAB_MAX) return INPAINT_E_INVAL;
  MemTab tab{};
  if (mem_in)
    for (int i = 0; i < B * m; ++i) {
      tab.p[i] = static_cast<const uint8_t*>(mem_in[i]);
      if (tab.p[i] && misaligned(tab.p[i])) return INPAINT_E_INVAL;
    }
  if (mem_out)
    for (int b = 0; b < B; ++b)
      if (mem_out[b] && misaligned(mem_out[b])) return INPAINT_E_INVAL;
  const Plan p = make_plan(c, B, H, W);
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  if (ws) {
    if (ws_bytes < p.end) return INPAINT_E_INVAL;
  } else {
    TRY(grow(&c->arena, &c->arena_bytes, p.end, c, c->stage_bytes + c->bws_bytes));
    ws = c->arena;
  }
  cudaStream_t st = (cudaStream_t)stream;
  MemArgs ma;
  ma.lay = mem_layout(c, p.Nt);
  ma.out = reinterpret_cast<uint8_t* const*>(mem_out);
  if (mem_in) ma.tab = &tab;  // passed by value in each attention launch
  if (ws != c->arena) return run_forward(c, ws, p, x, hole, out, pred, st, &ma);
  c->have_masks = false;
  TRY(run_forward(c, ws, p, x, hole, out, pred, st, &ma));
  c->last = p;
  c->have_masks = true;
  return INPAINT_OK;
}

int inpaint_point_cloud(inpaint_ctx* c, const float* depth, const float* rgb, int H, int W, const float* cam,
                        const float* rt, float* points, void* stream) {
  if (!c || !depth || !rgb || !cam || !rt || !points || H < 1 || W < 1 || (size_t)H * W > ((size_t)1 << 30))
    return INPAINT_E_INVAL;
  if (!(cam[0] != 0.f && cam[1] != 0.f)) return INPAINT_E_INVAL;
  LaunchScope ls(c, (cudaStream_t)stream, K_CLOUD);
  return cuda_err(launch_point_cloud(depth, rgb, H, W, cam, rt, points, (cudaStream_t)stream));
}

int inpaint_point_splat(inpaint_ctx* c, const float* points, int64_t n_points, const float* view, const float* rt,
                        int Ho, int Wo, float* img, float* depth_out, int32_t* index_out, void* stream) {
  if (!c || (!points && n_points > 0) || n_points < 0 || n_points > ((int64_t)1 << 32) - 1 || !view || !rt || !img ||
      Ho < 1 || Wo < 1 || (size_t)Ho * Wo > ((size_t)1 << 30))
    return INPAINT_E_INVAL;
  const size_t need = (size_t)Ho * Wo * sizeof(unsigned long long);
  TRY(grow(&c->zbuf, &c->zbuf_bytes, need, c, c->arena_bytes + c->stage_bytes + c->bws_bytes + c->pp_bytes));
  LaunchScope ls(c, (cudaStream_t)stream, K_SPLAT);
  return cuda_err(launch_splat(points, n_points, view, rt, Ho, Wo, reinterpret_cast<unsigned long long*>(c->zbuf), img,
                               depth_out, index_out, (cudaStream_t)stream));
}

int inpaint_frame(inpaint_ctx* c, const float* x, const uint8_t* hole, int H, int W, float* out, void* stream) {
  return inpaint_batch(c, x, hole, 1, H, W, out, nullptr, stream);
}

int inpaint_batch_ws(inpaint_ctx* c, void* workspace, size_t ws_bytes, const float* x, const uint8_t* hole, int B,
                     int H, int W, float* out, float* pred, void* stream) {
  if (!c || !workspace || !x || !hole || !out || bad_shape(B, H, W)) return INPAINT_E_INVAL;
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return INPAINT_E_INVAL;
  const Plan p = make_plan(c, B, H, W);
  if (ws_bytes < p.end) return INPAINT_E_INVAL;
  return run_forward(c, static_cast<uint8_t*>(workspace), p, x, hole, out, pred, (cudaStream_t)stream);
}

int inpaint_batch_host(inpaint_ctx* c, const float* xh, const uint8_t* hh, int B, int H, int W, float* oh,
                       void* stream) {
  if (!c || !xh || !hh || !oh || bad_shape(B, H, W)) return INPAINT_E_INVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nx = (size_t)B * 3 * H * W, nh = (size_t)B * H * W;
  const size_t bx = align_up(nx * 4, 256), bh = align_up(nh, 256);
  TRY(grow(&c->stage, &c->stage_bytes, 2 * bx + bh, c, c->arena_bytes + c->bws_bytes));
  float* xd = reinterpret_cast<float*>(c->stage);
  float* od = reinterpret_cast<float*>(c->stage + bx);
  uint8_t* hd = c->stage + 2 * bx;
  // The copies run on the context's copy stream frame by frame: frame f is embedded as
  // soon as its inputs have landed, and its output is copied back as soon as its head
  // kernel has written it, while the later frames' copies and kernels proceed.
  if (!c->copy_stream) TRY(cuda_err(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking)));
  auto events = [&](std::vector<cudaEvent_t>& v) -> int {
    while ((int)v.size() < B) {
      cudaEvent_t e;
      TRY(cuda_err(cudaEventCreateWithFlags(&e, cudaEventDisableTiming)));
      v.push_back(e);
    }
    return INPAINT_OK;
  };
  TRY(events(c->in_ev));
  TRY(events(c->out_ev));
  if (!c->start_ev) TRY(cuda_err(cudaEventCreateWithFlags(&c->start_ev, cudaEventDisableTiming)));
  if (!c->done_ev) TRY(cuda_err(cudaEventCreateWithFlags(&c->done_ev, cudaEventDisableTiming)));
  const Plan p = make_plan(c, B, H, W);
  TRY(grow(&c->arena, &c->arena_bytes, p.end, c, c->stage_bytes + c->bws_bytes));
  cudaStream_t cs = c->copy_stream;
  // the staging buffers are free once the work already queued on `st` is done
  TRY(cuda_err(cudaEventRecord(c->start_ev, st)));
  TRY(cuda_err(cudaStreamWaitEvent(cs, c->start_ev, 0)));
  const size_t HW = (size_t)H * W;
  c->have_masks = false;
  auto run = [&]() -> int {
    for (int f = 0; f < B; ++f) {
      TRY(cuda_err(cudaMemcpyAsync(xd + f * 3 * HW, xh + f * 3 * HW, 3 * HW * 4, cudaMemcpyHostToDevice, cs)));
      TRY(cuda_err(cudaMemcpyAsync(hd + f * HW, hh + f * HW, HW, cudaMemcpyHostToDevice, cs)));
      TRY(cuda_err(cudaEventRecord(c->in_ev[f], cs)));
    }
    const FramePipe pipe{c->in_ev.data(), c->out_ev.data()};
    TRY(run_forward(c, c->arena, p, xd, hd, od, nullptr, st, nullptr, &pipe));
    for (int f = 0; f < B; ++f) {
      TRY(cuda_err(cudaStreamWaitEvent(cs, c->out_ev[f], 0)));
      TRY(cuda_err(cudaMemcpyAsync(oh + f * 3 * HW, od + f * 3 * HW, 3 * HW * 4, cudaMemcpyDeviceToHost, cs)));
    }
    TRY(cuda_err(cudaEventRecord(c->done_ev, cs)));
    TRY(cuda_err(cudaStreamWaitEvent(st, c->done_ev, 0)));  // the caller's stream sees the results
    return cuda_err(cudaStreamSynchronize(cs));
  };
  const int rc = run();
  if (rc != INPAINT_OK) {  // no copy of the caller's host buffers may still be in flight
    cudaStreamSynchronize(cs);
    cudaStreamSynchronize(st);
    return rc;
  }
  c->last = p;
  c->have_masks = true;
  return INPAINT_OK;
}

int inpaint_token_masks(inpaint_ctx* c, uint8_t* host, size_t n) {
  if (!c || !host) return INPAINT_E_INVAL;
  if (!c->have_masks) return INPAINT_E_STATE;
  const size_t need = (size_t)(c->L + 1) * c->last.M;
  if (n < need) return INPAINT_E_INVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return INPAINT_E_CUDA;
  return cuda_err(cudaMemcpy(host, c->arena + c->last.masks, need, cudaMemcpyDeviceToHost));
}

int inpaint_fullres(inpaint_ctx* c, const float* x, const uint8_t* obj_masks, const uint8_t* selected, int B, int K,
                    int H, int W, float* out, uint8_t* hole_half_out, void* stream) {
  if (!c || !x || !obj_masks || !selected || !out || K < 1 || (H & 1) || (W & 1) || bad_shape(B, H, W))
    return INPAINT_E_INVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int h = H / 2, w = W / 2;
  const size_t nx = (size_t)B * 3 * h * w, nh = (size_t)B * h * w;
  const size_t bx = align_up(nx * 4, 256), bh = align_up(nh, 256);
  TRY(grow(&c->pp, &c->pp_bytes, 3 * bx + bh, c, c->arena_bytes + c->stage_bytes + c->bws_bytes));
  float* xh = reinterpret_cast<float*>(c->pp);
  float* pred = reinterpret_cast<float*>(c->pp + bx);
  float* outh = reinterpret_cast<float*>(c->pp + 2 * bx);
  uint8_t* hole = hole_half_out ? hole_half_out : c->pp + 3 * bx;
  { LaunchScope ls(c, st, K_OTHER); TRY(cuda_err(launch_mask_union(obj_masks, selected, B, K, h, w, hole, st))); }
  { LaunchScope ls(c, st, K_OTHER); TRY(cuda_err(launch_downscale2(x, B, H, W, xh, st))); }
  TRY(inpaint_batch(c, xh, hole, B, h, w, outh, pred, stream));
  LaunchScope ls(c, st, K_OTHER);
  return cuda_err(launch_upscale_composite(pred, hole, x, B, H, W, out, st));
}

int inpaint_l1_hole_loss(inpaint_ctx* c, const float* out, const float* target, const uint8_t* hole, int B, int H,
                         int W, float* loss, float* grad, void* stream) {
  if (!c || !out || !target || !hole || !loss || bad_shape(B, H, W)) return INPAINT_E_INVAL;
  const int nb = loss_partials(B, H, W);
  // partial sums live in the backward scratch area (separate from the forward arena)
  const size_t need = align_up((size_t)nb * 4, 256) * 2;
  TRY(grow(&c->bws, &c->bws_bytes, need, c, c->arena_bytes + c->stage_bytes));
  float* partials = reinterpret_cast<float*>(c->bws);
  unsigned* counts = reinterpret_cast<unsigned*>(c->bws + align_up((size_t)nb * 4, 256));
  LaunchScope ls(c, (cudaStream_t)stream, K_OTHER);
  return cuda_err(launch_l1_hole_loss(out, target, hole, B, H, W, partials, counts, loss, grad, (cudaStream_t)stream));
}

int inpaint_backward(inpaint_ctx* c, const float* x, const uint8_t* hole, const float* grad_out, int B, int H, int W,
                     float* grad_w, void* stream) {
  if (!c || !x || !hole || !grad_out || !grad_w || bad_shape(B, H, W)) return INPAINT_E_INVAL;
  return backward_impl(c, x, hole, grad_out, B, H, W, grad_w, (cudaStream_t)stream);
}

int inpaint_train_step(inpaint_ctx* c, const float* x, const uint8_t* hole, const float* target, int B, int H, int W,
                       float* loss, float* grad_w, float* out, void* stream) {
  if (!c || !x || !hole || !target || !loss || !grad_w || bad_shape(B, H, W)) return INPAINT_E_INVAL;
  return backward_impl(c, x, hole, nullptr, B, H, W, grad_w, (cudaStream_t)stream, target, loss, out);
}

int inpaint_sync(inpaint_ctx* c, void* stream, int timeout_ms) {
  if (!c) return INPAINT_E_INVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t q = cudaStreamQuery(st);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return INPAINT_E_CUDA;
    if (timeout_ms >= 0 && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
      return INPAINT_E_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  int flag = 0;
  if (cudaMemcpy(&flag, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return INPAINT_E_CUDA;
  if (flag) {
    cudaMemset(c->dev_err, 0, sizeof(int));
    return INPAINT_E_DEVICE;
  }
  return INPAINT_OK;
}

int inpaint_profile_enable(inpaint_ctx* c, int on) {
  if (!c) return INPAINT_E_INVAL;
  c->prof = on != 0;
  return INPAINT_OK;
}

int inpaint_profile_read(inpaint_ctx* c, float* ms, int64_t* launches) {
  if (!c || !ms || !launches) return INPAINT_E_INVAL;
  for (int k = 0; k < INPAINT_PROFILE_CLASSES; ++k) {
    ms[k] = 0.f;
    launches[k] = 0;
  }
  for (size_t i = 0; i < c->ev_used; ++i) {
    EventPair& e = c->events[i];
    if (cudaEventSynchronize(e.b) != cudaSuccess) return INPAINT_E_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e.a, e.b) != cudaSuccess) return INPAINT_E_CUDA;
    ms[e.cls] += t;
    launches[e.cls] += 1;
  }
  c->ev_used = 0;
  return INPAINT_OK;
}

int inpaint_launch_count(inpaint_ctx* c, int64_t* n) {
  if (!c || !n) return INPAINT_E_INVAL;
  *n = c->launches;
  return INPAINT_OK;
}

}  // extern "C"

namespace {
// One thread waits on an mbarrier that expects one arrival which never comes (bounded by
// limit_ns), then reports the expired wait as the tensor-core kernels do.
__global__ void wait_expiry_kernel(int* err, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  abort_flag = 0;
  tc::mbar_init(&bar, 1);
  tc::fence_mbar_init();
  if (!tc::mbar_wait(&bar, 0, &abort_flag, limit_ns)) atomicExch(err, DEV_MBAR_TIMEOUT);
}

__global__ void gelu_pair_kernel(const float* __restrict__ x, float* __restrict__ y_bf16_form,
                                 float* __restrict__ y_fp32_form, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    y_bf16_form[i] = gelu_as(x[i]);
    y_fp32_form[i] = gelu_erf(x[i]);
  }
}
__global__ void gelu_h16_kernel(const float* __restrict__ x, float* __restrict__ y, int n) {
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i < n) {
    const float a = x[i], b = i + 1 < n ? x[i + 1] : 0.f;
    const float2 r = __half22float2(gelu_h2(f32x2_to_h2_satfinite(a, b)));
    y[i] = r.x;
    if (i + 1 < n) y[i + 1] = r.y;
  }
}
}  // namespace

extern "C" {

int inpaint_test_wait_expiry(inpaint_ctx* c, int limit_us, void* stream) {
  if (!c || limit_us < 1 || limit_us > 1000000) return INPAINT_E_INVAL;
  LaunchScope ls(c, (cudaStream_t)stream, K_OTHER);
  wait_expiry_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(c->dev_err, (uint64_t)limit_us * 1000ull);
  return cuda_err(cudaGetLastError());
}

int inpaint_test_gelu(const float* x, float* y_bf16_form, float* y_fp32_form, int n, void* stream) {
  if (!x || !y_bf16_form || !y_fp32_form || n < 0) return INPAINT_E_INVAL;
  if (n == 0) return INPAINT_OK;
  gelu_pair_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, y_bf16_form, y_fp32_form, n);
  return cuda_err(cudaGetLastError());
}

int inpaint_test_gelu_h16(const float* x, float* y, int n, void* stream) {
  if (!x || !y || n < 0) return INPAINT_E_INVAL;
  if (n == 0) return INPAINT_OK;
  gelu_h16_kernel<<<((n + 1) / 2 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, y, n);
  return cuda_err(cudaGetLastError());
}

int inpaint_test_gemm_bf16(const void* A, const void* Bt, float* C, int M, int N, int K, void* stream) {
  if (!A || !Bt || !C || M <= 0 || N <= 0 || K <= 0 || N % 64 || K % 64) return INPAINT_E_INVAL;
  static int* err = nullptr;
  if (!err) {
    if (cudaMalloc(&err, 256) != cudaSuccess) return INPAINT_E_NOMEM;
    cudaMemset(err, 0, 256);
  }
  return cuda_err(launch_gemm_tc(static_cast<const bf16*>(A), static_cast<const bf16*>(Bt), C, N, M, N, K, EPI_NONE,
                                 nullptr, nullptr, err, (cudaStream_t)stream));
}

}  // extern "C"
