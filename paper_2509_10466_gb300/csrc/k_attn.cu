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
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc_primitives.cuh"
#include "window_attn.cuh"

namespace inpaint {

namespace {

constexpr int WS = 8;      // window side
constexpr int SLOTS = 64;  // WS * WS
constexpr int DH = 32;     // head dim


// One CTA per (window, head), thread s = slot s.  Rows move a whole 32-value head slice per
// warp instruction (lane = channel) between global and shared memory; the scores are dot
// products four keys at a time (independent FMA chains, each in ascending channel order, so
// every value equals the one-key-at-a-time evaluation); excluded keys add exact zeros.
template <typename T>
__global__ void __launch_bounds__(SLOTS) attn_simt_kernel(const T* __restrict__ qkv, const uint8_t* __restrict__ v_in,
                                                          T* __restrict__ o, uint8_t* __restrict__ v_out, int Ht,
                                                          int Wt, int d, int offset, int nwx,
                                                          const float* __restrict__ relpos) {
  __shared__ float Qs[SLOTS][DH + 1];
  __shared__ float Ks[SLOTS][DH + 1];
  __shared__ float Vs[SLOTS][DH + 1];
  __shared__ int okS[SLOTS], tokS[SLOTS];
  __shared__ float rp[225];
  const int w = blockIdx.x, h = blockIdx.y, b = blockIdx.z;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < 225; e += SLOTS) rp[e] = relpos ? relpos[h * 225 + e] : 0.f;
  const int wy = w / nwx, wx = w - (w / nwx) * nwx;
  const int s = threadIdx.x;
  const int ty = wy * WS - offset + (s >> 3), tx = wx * WS - offset + (s & 7);
  const bool real = ty >= 0 && ty < Ht && tx >= 0 && tx < Wt;
  const size_t Nt = (size_t)Ht * Wt;
  const size_t t = real ? (size_t)b * Nt + (size_t)ty * Wt + tx : 0;
  const bool ok = real && v_in[t] != 0;
  okS[s] = ok;
  tokS[s] = real ? (int)t : -1;
  __syncthreads();
  for (int sl = warp; sl < SLOTS; sl += SLOTS / 32) {  // the window's head slices
    const int ts = tokS[sl];
    const bool oks = okS[sl];
    const T* row = qkv + (size_t)(ts < 0 ? 0 : ts) * 3 * d + h * DH + lane;
    Qs[sl][lane] = ts >= 0 ? to_f32(row[0]) : 0.f;
    Ks[sl][lane] = oks ? to_f32(row[d]) : 0.f;
    Vs[sl][lane] = oks ? to_f32(row[2 * d]) : 0.f;
  }
  const int any = __syncthreads_or(ok);
  if (!any) {  // the same for every thread of the CTA
    if (real) {
      T* orow = o + t * d + h * DH;
#pragma unroll 8
      for (int i = 0; i < DH; ++i) orow[i] = from_f32<T>(0.f);
      if (h == 0) v_out[t] = 0;
    }
    return;
  }
  if (real && h == 0) v_out[t] = 1;
  float acc[DH], inv = 0.f;
  if (real) {
    float q[DH];
#pragma unroll
    for (int i = 0; i < DH; ++i) q[i] = Qs[s][i];
    const float scale = 1.0f / sqrtf((float)DH);
    float mx = -INFINITY;
    for (int k0 = 0; k0 < SLOTS; k0 += 4) {
      float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < DH; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j] = fmaf(q[i], Ks[k0 + j][i], a[j]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (okS[k0 + j]) mx = fmaxf(mx, a[j] * scale + rp[relpos_index(s, k0 + j)]);
    }
    float l = 0.f;
#pragma unroll
    for (int i = 0; i < DH; ++i) acc[i] = 0.f;
    for (int k0 = 0; k0 < SLOTS; k0 += 4) {
      float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < DH; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j] = fmaf(q[i], Ks[k0 + j][i], a[j]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = k0 + j;
        if (!okS[k]) continue;
        const float p = expf(a[j] * scale + rp[relpos_index(s, k)] - mx);
        l += p;
#pragma unroll
        for (int i = 0; i < DH; ++i) acc[i] = fmaf(p, Vs[k][i], acc[i]);
      }
    }
    inv = 1.f / l;
  }
  __syncthreads();  // K is no longer read: it takes the output rows
  if (real)
#pragma unroll
    for (int i = 0; i < DH; ++i) Ks[s][i] = acc[i] * inv;
  __syncthreads();
  for (int sl = warp; sl < SLOTS; sl += SLOTS / 32) {
    const int ts = tokS[sl];
    if (ts >= 0) o[(size_t)ts * d + h * DH + lane] = from_f32<T>(Ks[sl][lane]);
  }
}

// Temporal form: the window's keys are its usable current tokens and, for each of the m
// memory slots (a previous frame's k | v and usable-key mask at this block, or none),
// the usable tokens at the window's positions.  Key blocks of 64 are staged one after
// the other; each query keeps a running maximum, sum and weighted V (the max is raised
// once per block and the partial results rescaled).
template <typename T>
__global__ void __launch_bounds__(SLOTS) attn_simt_mem_kernel(const T* __restrict__ qkv,
                                                              const uint8_t* __restrict__ v_in, T* __restrict__ o,
                                                              uint8_t* __restrict__ v_out, int Ht, int Wt, int d,
                                                              int offset, int nwx,
                                                              const __grid_constant__ MemTab mem_tab, int m,
                                                              size_t off_kv, size_t off_mask,
                                                              const float* __restrict__ relpos) {
  __shared__ float Ks[SLOTS][DH + 1];
  __shared__ float Vs[SLOTS][DH + 1];
  __shared__ int okS[SLOTS];
  __shared__ float rp[225];
  const int w = blockIdx.x, h = blockIdx.y, b = blockIdx.z;
  for (int e = threadIdx.x; e < 225; e += SLOTS) rp[e] = relpos ? relpos[h * 225 + e] : 0.f;
  const int wy = w / nwx, wx = w - (w / nwx) * nwx;
  const int s = threadIdx.x;
  const int ty = wy * WS - offset + (s >> 3), tx = wx * WS - offset + (s & 7);
  const bool real = ty >= 0 && ty < Ht && tx >= 0 && tx < Wt;
  const size_t Nt = (size_t)Ht * Wt;
  const size_t i = real ? (size_t)ty * Wt + tx : 0;  // token within the frame
  const size_t t = (size_t)b * Nt + i;
  // key of slot s in key block kb (0 = current frame, 1 + j = memory slot j), or null
  auto key_row = [&](int kb) -> const T* {
    if (!real) return nullptr;
    if (kb == 0) return v_in[t] ? qkv + t * 3 * d + d : nullptr;
    const uint8_t* base = mem_tab.p[b * m + kb - 1];
    if (!base || !base[off_mask + i]) return nullptr;
    return reinterpret_cast<const T*>(base + off_kv) + i * 2 * d;
  };
  bool anyk = false;
  for (int kb = 0; kb <= m; ++kb) anyk = anyk || key_row(kb) != nullptr;
  const int any = __syncthreads_or(anyk);
  T* orow = o + t * d + h * DH;
  if (!any) {
    if (real) {
#pragma unroll 8
      for (int e = 0; e < DH; ++e) orow[e] = from_f32<T>(0.f);
      if (h == 0) v_out[t] = 0;
    }
    return;
  }
  if (real && h == 0) v_out[t] = 1;
  float q[DH];
  const T* qrow = qkv + t * 3 * d + h * DH;
#pragma unroll
  for (int e = 0; e < DH; ++e) q[e] = real ? to_f32(qrow[e]) : 0.f;
  const float scale = 1.0f / sqrtf((float)DH);
  float mx = -INFINITY, l = 0.f, acc[DH];
#pragma unroll
  for (int e = 0; e < DH; ++e) acc[e] = 0.f;
  for (int kb = 0; kb <= m; ++kb) {
    const T* kr = key_row(kb);
    __syncthreads();  // the previous block's keys are no longer read
    okS[s] = kr != nullptr;
#pragma unroll 8
    for (int e = 0; e < DH; ++e) {
      Ks[s][e] = kr ? to_f32(kr[h * DH + e]) : 0.f;
      Vs[s][e] = kr ? to_f32(kr[d + h * DH + e]) : 0.f;
    }
    if (!__syncthreads_or(kr != nullptr)) continue;
    if (!real) continue;
    float bm = -INFINITY;
    for (int k = 0; k < SLOTS; ++k) {
      if (!okS[k]) continue;
      float sc = 0.f;
#pragma unroll
      for (int e = 0; e < DH; ++e) sc = fmaf(q[e], Ks[k][e], sc);
      bm = fmaxf(bm, sc * scale + rp[relpos_index(s, k)]);
    }
    if (bm > mx) {
      const float a = expf(mx - bm);
      l *= a;
#pragma unroll
      for (int e = 0; e < DH; ++e) acc[e] *= a;
      mx = bm;
    }
    for (int k = 0; k < SLOTS; ++k) {
      if (!okS[k]) continue;
      float sc = 0.f;
#pragma unroll
      for (int e = 0; e < DH; ++e) sc = fmaf(q[e], Ks[k][e], sc);
      const float p = expf(sc * scale + rp[relpos_index(s, k)] - mx);
      l += p;
#pragma unroll
      for (int e = 0; e < DH; ++e) acc[e] = fmaf(p, Vs[k][e], acc[e]);
    }
  }
  if (!real) return;
  const float inv = 1.f / l;
#pragma unroll
  for (int e = 0; e < DH; ++e) orow[e] = from_f32<T>(acc[e] * inv);
}

}  // namespace

template <typename T>
cudaError_t launch_attention(const T* qkv, const uint8_t* v_in, T* o, uint8_t* v_out, int B, int Ht, int Wt, int d,
                             int heads, int offset, cudaStream_t st, const float* relpos) {
  const int nwy = (Ht + offset + WS - 1) / WS, nwx = (Wt + offset + WS - 1) / WS;
  dim3 grid(nwy * nwx, heads, B);
  attn_simt_kernel<T><<<grid, SLOTS, 0, st>>>(qkv, v_in, o, v_out, Ht, Wt, d, offset, nwx, relpos);
  return cudaGetLastError();
}

template cudaError_t launch_attention<float>(const float*, const uint8_t*, float*, uint8_t*, int, int, int, int, int,
                                             int, cudaStream_t, const float*);
template cudaError_t launch_attention<bf16>(const bf16*, const uint8_t*, bf16*, uint8_t*, int, int, int, int, int,
                                            int, cudaStream_t, const float*);
template cudaError_t launch_attention<f16>(const f16*, const uint8_t*, f16*, uint8_t*, int, int, int, int, int, int,
                                           cudaStream_t, const float*);

template <typename T>
cudaError_t launch_attention_mem(const T* qkv, const uint8_t* v_in, T* o, uint8_t* v_out, int B, int Ht, int Wt, int d,
                                 int heads, int offset, const MemTab* tab, int m, size_t off_kv, size_t off_mask,
                                 cudaStream_t st, const float* relpos) {
  const int nwy = (Ht + offset + WS - 1) / WS, nwx = (Wt + offset + WS - 1) / WS;
  if (tab && (size_t)B * m > (size_t)MEM_TAB_MAX) return cudaErrorInvalidValue;
  static const MemTab none{};
  dim3 grid(nwy * nwx, heads, B);
  attn_simt_mem_kernel<T><<<grid, SLOTS, 0, st>>>(qkv, v_in, o, v_out, Ht, Wt, d, offset, nwx, tab ? *tab : none,
                                                  tab ? m : 0, off_kv, off_mask, relpos);
  return cudaGetLastError();
}

template cudaError_t launch_attention_mem<float>(const float*, const uint8_t*, float*, uint8_t*, int, int, int, int,
                                                 int, int, const MemTab*, int, size_t, size_t, cudaStream_t,
                                                 const float*);
template cudaError_t launch_attention_mem<bf16>(const bf16*, const uint8_t*, bf16*, uint8_t*, int, int, int, int, int,
                                                int, const MemTab*, int, size_t, size_t, cudaStream_t, const float*);
template cudaError_t launch_attention_mem<f16>(const f16*, const uint8_t*, f16*, uint8_t*, int, int, int, int, int,
                                               int, const MemTab*, int, size_t, size_t, cudaStream_t, const float*);

}  // namespace inpaint

// ---------------------------------------------------------------------------------
// Tensor-core form (16-bit operands T = bf16 or f16, FP32 scores / softmax statistics /
// accumulation).
//
// One CTA per (window, head, frame), 4 warps; warp w owns query slots 16w .. +15.  The
// slot -> token map and the usable-key bitmask of the window are computed once per CTA.
// Q, K, V of the window (64 x 32 values each) are staged in shared memory by TMA while the
// key mask is read, then per warp:
//   S = Q K^T      16 x 64, 2 k-steps x 8 n-tiles of mma.m16n8k16 (fragments by ldmatrix)
//   masked softmax over the 64 keys in registers (quad shuffles for row max / sum)
//   O = P V        16 x 32, P re-packed to T straight from the S accumulators,
//                  V fragments by ldmatrix.trans; O scaled by 1/rowsum in FP32.
// The window is small (64x64x32), so the kernel is bound by reading Q, K, V and
// writing O; many small CTAs per SM keep enough loads in flight.
namespace inpaint {
namespace {



// Q, K and V are staged by TMA: a 4D tensor map views qkv as [B][Ht][Wt][3d], so one box
// {32 channels, 8 x 8 tokens} is the window's 64 rows of one part (Q, K or V) of one
// head; void slots of shifted border windows lie outside the map and arrive as zeros.
// The boxes land in 64-byte rows with the 64-byte TMA swizzle (16-byte chunk c of slot row r
// at c ^ ((r >> 1) & 3)), which the ldmatrix addresses below follow (conflict-free).

// One head per CTA: 128 threads and 12 KB of boxes, so that many CTAs per SM keep TMA
// loads in flight (two or more heads per CTA measured slower).
constexpr int HPT = 1;
constexpr int TMA_THREADS = 128 * HPT;
static_assert(3 * HPT * SLOTS * DH * 2 + 512 <= 48 * 1024, "boxes exceed the default dynamic shared memory");

template <bool RP, typename T>
__global__ void __launch_bounds__(TMA_THREADS, 8) attn_tma_kernel(const __grid_constant__ CUtensorMap tmQKV,
                                                              const uint8_t* __restrict__ v_in,
                                                              T* __restrict__ o, uint8_t* __restrict__ v_out,
                                                              int Ht, int Wt, int d, int offset, int nwx,
                                                              const float* __restrict__ relpos, int* err) {
  extern __shared__ uint8_t asm_raw[];
  // [part Q, K, V][head of the CTA] tiles of 64 slot rows x 64 bytes, 512-byte aligned
  uint8_t* tiles = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(asm_raw) + 511) & ~uintptr_t(511));
  __shared__ float rps[RP ? HPT : 1][RP ? 225 : 1];
  __shared__ int stok[SLOTS];
  __shared__ unsigned okw[2];
  __shared__ __align__(8) uint64_t bar;
  const int w = blockIdx.x, b = blockIdx.z;
  const int wy = w / nwx, wx = w - (w / nwx) * nwx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Nt = Ht * Wt;
  const int h0 = HPT * blockIdx.y;
  constexpr int TILE = SLOTS * DH * 2;
  auto tile = [&](int part, int hh) { return tiles + (part * HPT + hh) * TILE; };

  if (RP)
    for (int e = tid; e < HPT * 225; e += TMA_THREADS) rps[e / 225][e % 225] = relpos[(h0 + e / 225) * 225 + e % 225];
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmQKV);
  }
  __syncthreads();
  pdl_trigger();
  pdl_wait();
  if (tid == 0) {
    tc::mbar_expect_tx(&bar, 3 * HPT * TILE);
    for (int part = 0; part < 3; ++part)
      for (int hh = 0; hh < HPT; ++hh)
        tc::tma_load_4d(tile(part, hh), &tmQKV, &bar, part * d + (h0 + hh) * DH, wx * WS - offset, wy * WS - offset,
                        b);
  }
  // the window's key mask while the boxes land
  if (tid < SLOTS) {
    const int ty = wy * WS - offset + (tid >> 3), tx = wx * WS - offset + (tid & 7);
    const bool real = ty >= 0 && ty < Ht && tx >= 0 && tx < Wt;
    const int t = real ? b * Nt + ty * Wt + tx : -1;
    stok[tid] = t;
    const bool ok = real && v_in[t] != 0;
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) okw[warp] = bal;
  }
  const bool landed = tc::mbar_wait_timed(&bar, 0);
  __syncthreads();
  if (!landed) {
    if (tid == 0 && err) atomicExch(err, DEV_MBAR_TIMEOUT);
    return;
  }
  const unsigned long long keymask = (unsigned long long)okw[0] | ((unsigned long long)okw[1] << 32);

  if (keymask == 0ull) {  // no usable key: the window outputs 0 and stays invalid
    for (int e = tid; e < SLOTS * 4 * HPT; e += TMA_THREADS) {
      const int sl = e / (4 * HPT), hh = (e >> 2) % HPT, ch = e & 3;
      const int t = stok[sl];
      if (t >= 0) {
        *reinterpret_cast<uint4*>(o + (size_t)t * d + (h0 + hh) * DH + ch * 8) = make_uint4(0, 0, 0, 0);
        if (h0 == 0 && hh == 0 && ch == 0) v_out[t] = 0;
      }
    }
    return;
  }
  if (h0 == 0 && tid < SLOTS && stok[tid] >= 0) v_out[stok[tid]] = 1;

  const int hh = warp >> 2, wq = warp & 3;
  window_attention_rows<RP, T>(tile(0, hh), tile(1, hh), tile(2, hh), keymask, RP ? rps[hh] : nullptr, stok, o, d,
                               (h0 + hh) * DH, wq * 16, lane);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// qkv [B][Ht][Wt][3d] (16-bit T) as a 4D map with {32 channels, 8, 8, 1} boxes, 64-byte swizzle
template <typename T>
bool qkv_map(CUtensorMap* m, const T* qkv, int B, int Ht, int Wt, int d) {
  auto fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(qkv) & 15)) return false;
  const uint64_t row = (uint64_t)3 * d * 2;
  cuuint64_t dims[4] = {(cuuint64_t)3 * d, (cuuint64_t)Wt, (cuuint64_t)Ht, (cuuint64_t)B};
  cuuint64_t strides[3] = {row, row * Wt, row * Wt * Ht};
  cuuint32_t box[4] = {DH, WS, WS, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, tc::tma_dtype<T>(), 4, const_cast<T*>(qkv), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Temporal form on tensor cores, one head per CTA.  Key blocks of 64: the window's
// current tokens, then each memory slot's tokens at the window's positions.  All staging is
// issued at once: the current Q, K, V boxes by TMA (as in the spatial kernel) and, for each
// memory slot, the head slices (64 bytes) of its key rows by 16-byte cp.async copies of all
// threads into 80-byte rows (conflict-free ldmatrix), one commit group per slot, so that
// the current block is computed while the slots land.  Rows of keys that are not usable
// are filled with zeros by the copies themselves (their probability is 0).
// Per block the running row maximum is raised, the running sum and O rescaled by
// 2^(old max - new max), and O += P V; blocks without a usable key are skipped.
constexpr int MROW = 80;                // bytes per staged memory key row: 64 + 16 pad
constexpr int MTILE = SLOTS * MROW;     // one part (K or V) of one memory slot
constexpr int MEM_SLOTS_MAX = 4;

// 16 bytes global -> shared, or 16 zero bytes when !valid (the source is then not read)
__device__ __forceinline__ void cp_async16z(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(dst)), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// at most n (0 .. MEM_SLOTS_MAX - 1) of this thread's committed groups still pending
__device__ __forceinline__ void cp_async_wait_pending(int n) {
  switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
  }
}

template <bool RP, typename T>
__global__ void __launch_bounds__(TMA_THREADS, 5) attn_mem_tma_kernel(
    const __grid_constant__ CUtensorMap tmQKV, const uint8_t* __restrict__ v_in, T* __restrict__ o,
    uint8_t* __restrict__ v_out, int Ht, int Wt, int d, int offset, int nwx, const __grid_constant__ MemTab mem_tab,
    int m, size_t off_kv, size_t off_mask, const __grid_constant__ MemTab out_tab, int record,
    const float* __restrict__ relpos, int* err) {
  extern __shared__ uint8_t msm_raw[];
  constexpr int TILE = SLOTS * DH * 2;
  // Q, K, V boxes [3][TILE] (512-byte aligned for the 64-byte swizzle), then the memory
  // slots' [m][K, V][MTILE]
  uint8_t* tiles = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(msm_raw) + 511) & ~uintptr_t(511));
  uint8_t* mtiles = tiles + 3 * TILE;
  __shared__ float rps[RP ? 225 : 1];
  __shared__ int stok[SLOTS], sidx[SLOTS];
  __shared__ unsigned okw[1 + MEM_SLOTS_MAX][2];  // usable-key bits of each key block
  __shared__ __align__(8) uint64_t bar;
  const int w = blockIdx.x, h = blockIdx.y, b = blockIdx.z;
  const int wy = w / nwx, wx = w - (w / nwx) * nwx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Nt = Ht * Wt;
  auto mK = [&](int j) { return mtiles + (size_t)(2 * j) * MTILE; };
  auto mV = [&](int j) { return mtiles + (size_t)(2 * j + 1) * MTILE; };
  auto keymask = [&](int kb) { return (unsigned long long)okw[kb][0] | ((unsigned long long)okw[kb][1] << 32); };

  if (RP)
    for (int e = tid; e < 225; e += TMA_THREADS) rps[e] = relpos[h * 225 + e];
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmQKV);
  }
  __syncthreads();
  pdl_trigger();
  pdl_wait();
  if (tid == 0) {
    tc::mbar_expect_tx(&bar, 3 * TILE);
    for (int part = 0; part < 3; ++part)
      tc::tma_load_4d(tiles + part * TILE, &tmQKV, &bar, part * d + h * DH, wx * WS - offset, wy * WS - offset, b);
  }
  // the window's slots while the boxes land
  if (tid < SLOTS) {
    const int ty = wy * WS - offset + (tid >> 3), tx = wx * WS - offset + (tid & 7);
    const bool real = ty >= 0 && ty < Ht && tx >= 0 && tx < Wt;
    sidx[tid] = real ? ty * Wt + tx : -1;
    stok[tid] = real ? b * Nt + ty * Wt + tx : -1;
  }
  __syncthreads();
  // memory rows of every present slot, all threads, one commit group per slot (committed
  // for every slot, empty ones too, so that slot j is group j): every real token's row
  // (recorded k | v values, finite), zeros for void slots; the usable-key masks, read
  // meanwhile, select the keys in the softmax
  // (row, part, 16-byte chunk) e = tid + 128 q of every slot: the rows' byte offsets and
  // validity, the same for every slot
  constexpr int CP_PER_THREAD = SLOTS * 8 / TMA_THREADS;
  static_assert(SLOTS * 8 % TMA_THREADS == 0, "memory row copies per thread");
  const int cpart = (tid >> 2) & 1, cc = tid & 3;
  size_t src_off[CP_PER_THREAD];
  bool src_ok[CP_PER_THREAD];
#pragma unroll
  for (int q = 0; q < CP_PER_THREAD; ++q) {
    const int i = sidx[(tid + q * TMA_THREADS) >> 3];
    src_ok[q] = i >= 0;
    src_off[q] = i >= 0 ? (((size_t)i * 2 + cpart) * d + (size_t)h * DH) * sizeof(T) + cc * 16 : 0;
  }
  for (int j = 0; j < m; ++j) {
    const uint8_t* base = mem_tab.p[b * m + j];
    if (base) {
      const uint8_t* kv = base + off_kv;
      uint8_t* dst = (cpart ? mV(j) : mK(j)) + cc * 16;
#pragma unroll
      for (int q = 0; q < CP_PER_THREAD; ++q)
        cp_async16z(dst + ((tid + q * TMA_THREADS) >> 3) * MROW, kv + src_off[q], src_ok[q]);
    }
    cp_async_commit();
  }
  if (tid < SLOTS) {  // every mask byte is loaded before the first ballot
    const int i = sidx[tid];
    bool use[1 + MEM_SLOTS_MAX];
    use[0] = i >= 0 && v_in[b * Nt + i] != 0;
#pragma unroll
    for (int j = 0; j < MEM_SLOTS_MAX; ++j) {
      const uint8_t* base = j < m ? mem_tab.p[b * m + j] : nullptr;
      use[1 + j] = i >= 0 && base && base[off_mask + i] != 0;
    }
#pragma unroll
    for (int j = 0; j <= MEM_SLOTS_MAX; ++j) {
      const unsigned bal = __ballot_sync(0xffffffffu, use[j]);
      if (lane == 0 && j <= m) okw[j][warp] = bal;
    }
  }
  __syncthreads();
  unsigned long long any = 0ull;
  for (int kb = 0; kb <= m; ++kb) any |= keymask(kb);
  const bool landed = tc::mbar_wait_timed(&bar, 0);
  __syncthreads();
  if (!landed) {
    if (tid == 0 && err) atomicExch(err, DEV_MBAR_TIMEOUT);
    cp_async_wait_pending(0);
    return;
  }
  // this frame's memory tensor of this block: k | v of the window's tokens (this head's
  // 64-byte slices, from the staged boxes) and the block's input key mask
  uint8_t* rec = record ? const_cast<uint8_t*>(out_tab.p[b]) : nullptr;
  if (rec) {
    for (int e = tid; e < SLOTS * 8; e += TMA_THREADS) {  // (row, part K / V, 16-byte chunk)
      const int r = e >> 3, part = (e >> 2) & 1, c = e & 3;
      const int i = sidx[r];
      if (i >= 0)
        *reinterpret_cast<uint4*>(rec + off_kv + (((size_t)i * 2 + part) * d + (size_t)h * DH) * sizeof(T) + c * 16) =
            *reinterpret_cast<const uint4*>(tiles + (1 + part) * TILE + swz64(r, c));
    }
    if (h == 0 && tid < SLOTS && sidx[tid] >= 0) rec[off_mask + sidx[tid]] = v_in[b * Nt + sidx[tid]];
  }
  if (!any) {  // no usable key anywhere: the window outputs 0 and stays invalid
    for (int e = tid; e < SLOTS * 4; e += TMA_THREADS) {
      const int sl = e >> 2, ch = e & 3;
      const int t = stok[sl];
      if (t >= 0) {
        *reinterpret_cast<uint4*>(o + (size_t)t * d + h * DH + ch * 8) = make_uint4(0, 0, 0, 0);
        if (h == 0 && ch == 0) v_out[t] = 0;
      }
    }
    cp_async_wait_pending(0);  // the memory rows land before the CTA's shared memory is released
    return;
  }
  if (h == 0 && tid < SLOTS && stok[tid] >= 0) v_out[stok[tid]] = 1;

  const int g = lane >> 2, tq = lane & 3;
  const int r0 = warp * 16;
  uint8_t* Qt = tiles;
  const uint8_t* Kt = tiles + TILE;
  const uint8_t* Vt = tiles + 2 * TILE;
  uint32_t qa[2][4];
  {
    const int row = r0 + (lane & 15);
    ldsm_x4(qa[0], Qt + swz64(row, lane >> 4));
    ldsm_x4(qa[1], Qt + swz64(row, 2 + (lane >> 4)));
  }
  const float sl2 = 1.4426950408889634f / sqrtf((float)DH);  // scale * log2(e)
  // Without the relative-position bias the running maxima are taken on the raw scores (the
  // scale is positive) and the scale enters with the maximum in one FMA in the exponent;
  // with it the scores are scaled and biased first (sx = 1).  The running row sums are
  // those of the 16-bit probabilities, by one more MMA against ones per block (every
  // column of `ls` holds its row's sum).
  const float sx = RP ? 1.f : sl2;
  const uint32_t ones = H16<T>::pack2(1.f, 1.f);
  float mx0 = -INFINITY, mx1 = -INFINITY;
  float oc[4][4], ls[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int j = 0; j < 4; ++j) oc[j][0] = oc[j][1] = oc[j][2] = oc[j][3] = 0.f;
  for (int kb = 0; kb <= m; ++kb) {
    const unsigned long long km = keymask(kb);
    if (!km) continue;  // uniform across the CTA
    if (kb > 0) {  // slot kb - 1's copies (group kb - 1) of every thread have landed
      cp_async_wait_pending(m - kb);
      __syncthreads();
    }
    // K / V fragment addresses: the swizzled TMA boxes (current block) or the padded rows
    auto kaddr = [&](int row, int chunk) -> const uint8_t* {
      return kb == 0 ? Kt + swz64(row, chunk) : mK(kb - 1) + row * MROW + chunk * 16;
    };
    auto vaddr = [&](int row, int chunk) -> const uint8_t* {
      return kb == 0 ? Vt + swz64(row, chunk) : mV(kb - 1) + row * MROW + chunk * 16;
    };
    float sc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      sc[j][0] = sc[j][1] = sc[j][2] = sc[j][3] = 0.f;
      uint32_t kbf[4];
      ldsm_x4(kbf, kaddr(8 * j + (lane & 7), lane >> 3));
      mma16816<T>(sc[j], qa[0], kbf[0], kbf[1]);
      mma16816<T>(sc[j], qa[1], kbf[2], kbf[3]);
    }
    float bm0 = -INFINITY, bm1 = -INFINITY;
    const unsigned long long kq = km >> (2 * tq);  // bit 8j + c: key 8j + 2tq + c
    auto mask_and_max = [&](auto masked) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const bool okk = (kq >> (8 * j + c)) & 1ull;
          if constexpr (RP) {
            const int key = 8 * j + 2 * tq + c;
            const float bb0 = rps[relpos_index(r0 + g, key)] * LOG2E;
            const float bb1 = rps[relpos_index(r0 + g + 8, key)] * LOG2E;
            sc[j][c] = okk ? fmaf(sc[j][c], sl2, bb0) : -INFINITY;
            sc[j][2 + c] = okk ? fmaf(sc[j][2 + c], sl2, bb1) : -INFINITY;
          } else if constexpr (decltype(masked)::value) {
            sc[j][c] = okk ? sc[j][c] : -INFINITY;
            sc[j][2 + c] = okk ? sc[j][2 + c] : -INFINITY;
          }
          bm0 = fmaxf(bm0, sc[j][c]);
          bm1 = fmaxf(bm1, sc[j][2 + c]);
        }
      }
    };
    // a block whose 64 keys are all usable skips the selects
    if (RP || km != ~0ull) mask_and_max(BoolTag<true>{});
    else mask_and_max(BoolTag<false>{});
    bm0 = fmaxf(bm0, __shfl_xor_sync(0xffffffffu, bm0, 1));
    bm0 = fmaxf(bm0, __shfl_xor_sync(0xffffffffu, bm0, 2));
    bm1 = fmaxf(bm1, __shfl_xor_sync(0xffffffffu, bm1, 1));
    bm1 = fmaxf(bm1, __shfl_xor_sync(0xffffffffu, bm1, 2));
    // every row sees a usable key of this block (km != 0), so the new maxima are finite
    const float n0 = fmaxf(mx0, bm0), n1 = fmaxf(mx1, bm1);
    const float a0 = ex2_approx((mx0 - n0) * sx), a1 = ex2_approx((mx1 - n1) * sx);  // 0 on the first usable block
    mx0 = n0;
    mx1 = n1;
    ls[0] *= a0; ls[1] *= a0;
    ls[2] *= a1; ls[3] *= a1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      oc[j][0] *= a0; oc[j][1] *= a0;
      oc[j][2] *= a1; oc[j][3] *= a1;
    }
    const float o0 = -n0 * sx, o1 = -n1 * sx;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        sc[j][c] = ex2_approx(fmaf(sc[j][c], sx, o0));
        sc[j][2 + c] = ex2_approx(fmaf(sc[j][2 + c], sx, o1));
      }
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      uint32_t pa[4];
      pa[0] = H16<T>::pack2(sc[2 * kk][0], sc[2 * kk][1]);
      pa[1] = H16<T>::pack2(sc[2 * kk][2], sc[2 * kk][3]);
      pa[2] = H16<T>::pack2(sc[2 * kk + 1][0], sc[2 * kk + 1][1]);
      pa[3] = H16<T>::pack2(sc[2 * kk + 1][2], sc[2 * kk + 1][3]);
#pragma unroll
      for (int nn = 0; nn < 2; ++nn) {
        uint32_t vb[4];
        ldsm_x4_t(vb, vaddr(16 * kk + (lane & 7) + ((lane >> 3) & 1) * 8, 2 * nn + (lane >> 4)));
        mma16816<T>(oc[2 * nn], pa, vb[0], vb[1]);
        mma16816<T>(oc[2 * nn + 1], pa, vb[2], vb[3]);
      }
      mma16816<T>(ls, pa, ones, ones);
    }
  }
  const float l0 = ls[0], l1 = ls[2];
  const float inv0 = 1.f / l0, inv1 = 1.f / l1;
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
      *reinterpret_cast<uint4*>(o + (size_t)t * d + h * DH + ch * 8) = *reinterpret_cast<const uint4*>(Qt + swz64(sl, ch));
  }
}

}  // namespace

template <typename T>
cudaError_t launch_attention_tc(const T* qkv, const uint8_t* v_in, T* o, uint8_t* v_out, int B, int Ht, int Wt,
                                int d, int heads, int offset, cudaStream_t st, const float* relpos, int* err) {
  const int nwy = (Ht + offset + WS - 1) / WS, nwx = (Wt + offset + WS - 1) / WS;
  // one kernel only: a tensor map that cannot be built (no driver entry point, a
  // misaligned qkv) is an error, not a reason to run another kernel
  CUtensorMap m;
  if (heads % HPT || !qkv_map<T>(&m, qkv, B, Ht, Wt, d)) return cudaErrorInvalidValue;
  constexpr int smem = 3 * HPT * SLOTS * DH * 2 + 512;
  const dim3 tgrid(nwy * nwx, heads / HPT, B);
  if (relpos)
    return launch_pdl(attn_tma_kernel<true, T>, tgrid, dim3(TMA_THREADS), smem, st, m, v_in, o, v_out, Ht, Wt, d,
                      offset, nwx, relpos, err);
  return launch_pdl(attn_tma_kernel<false, T>, tgrid, dim3(TMA_THREADS), smem, st, m, v_in, o, v_out, Ht, Wt, d,
                    offset, nwx, (const float*)nullptr, err);
}

template <typename T>
cudaError_t launch_attention_tc_mem(const T* qkv, const uint8_t* v_in, T* o, uint8_t* v_out, int B, int Ht, int Wt,
                                    int d, int heads, int offset, const MemTab* tab, int m, size_t off_kv,
                                    size_t off_mask, uint8_t* const* out, cudaStream_t st, const float* relpos,
                                    int* err) {
  const int nwy = (Ht + offset + WS - 1) / WS, nwx = (Wt + offset + WS - 1) / WS;
  if (m < 0 || m > MEM_SLOTS_MAX) return cudaErrorInvalidValue;
  if (out && B > MEM_TAB_MAX) return cudaErrorInvalidValue;
  MemTab otab{};
  if (out)
    for (int b = 0; b < B; ++b) otab.p[b] = out[b];
  if (tab && (size_t)B * m > (size_t)MEM_TAB_MAX) return cudaErrorInvalidValue;
  // bulk copies read 16-byte aligned memory rows: buffers are 256-byte aligned, offsets and
  // row pitches multiples of 16 bytes
  if ((off_kv | ((size_t)d * sizeof(T))) & 15) return cudaErrorInvalidValue;
  CUtensorMap map;
  if (!qkv_map<T>(&map, qkv, B, Ht, Wt, d)) return cudaErrorInvalidValue;
  static const MemTab none{};
  const int mm = tab ? m : 0;
  const int smem = 511 + 3 * SLOTS * DH * 2 + mm * 2 * MTILE;
  auto kern = relpos ? attn_mem_tma_kernel<true, T> : attn_mem_tma_kernel<false, T>;
  static bool attr[2] = {false, false};
  if (!attr[relpos ? 1 : 0]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         511 + 3 * SLOTS * DH * 2 + MEM_SLOTS_MAX * 2 * MTILE);
    if (e != cudaSuccess) return e;
    attr[relpos ? 1 : 0] = true;
  }
  const dim3 grid(nwy * nwx, heads, B);
  return launch_pdl(kern, grid, dim3(TMA_THREADS), (size_t)smem, st, map, v_in, o, v_out, Ht, Wt, d, offset, nwx,
                    tab ? *tab : none, mm, off_kv, off_mask, otab, out ? 1 : 0, relpos, err);
}

#define INSTANTIATE(T)                                                                                              \
  template cudaError_t launch_attention_tc<T>(const T*, const uint8_t*, T*, uint8_t*, int, int, int, int, int, int,  \
                                              cudaStream_t, const float*, int*);                                    \
  template cudaError_t launch_attention_tc_mem<T>(const T*, const uint8_t*, T*, uint8_t*, int, int, int, int, int,   \
                                                  int, const MemTab*, int, size_t, size_t, uint8_t* const*,         \
                                                  cudaStream_t, const float*, int*);
INSTANTIATE(bf16)
INSTANTIATE(f16)
#undef INSTANTIATE

}  // namespace inpaint
