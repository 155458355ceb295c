// LN1-normalized tokens -> Q, K, V -> mask-aware window attention, in one kernel (the
// 16-bit forms, spatial blocks).
//
// A CTA takes two neighbouring windows of a frame (128 token slots).  Their normalized rows
// Y (64 x d per window) arrive by TMA as 4D boxes {64 channels, 8 x 8 tokens}, which land
// in the 128-byte-swizzled K-major layout of a tcgen05 operand; slots outside the token
// grid (offset windows) arrive as zeros.  The projection runs in passes of two heads:
// pass p computes [q | k | v] of heads 2p, 2p + 1 (192 columns) for all 128 slots on
// tcgen05 (M = 128, N = 192, FP32 accumulation in tensor memory, two accumulators so that
// pass p + 1 runs while pass p is consumed).  Sixteen warps take the accumulator of a pass
// (eight per head: two per TMEM lane quarter, one taking the q columns and half of the k
// columns, the other the rest of k and the v columns), add the bias, round to T and write
// the heads' Q, K, V tiles of both windows into shared memory in the 64-byte-swizzled
// layout of the TMA boxes of the separate attention kernel, and run the same masked window
// softmax on them (one window and 16 query rows per warp, mma.sync), writing the attention
// output rows.  The tiles are double-buffered by pass parity, so a warp drains pass p + 1
// while the other warps of its head still attend pass p.  Q, K and V never reach global
// memory; the weights stream through a two-stage ring of 24 KB stages (three 64-row boxes:
// the q, k and v rows of the pass's heads).
//
// Warps: 0 TMA producer, 1 TMEM owner + MMA issuer, 2..17 drain + attention.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc_primitives.cuh"
#include "window_attn.cuh"

namespace inpaint {

namespace {

constexpr int QA_BM = 128, QA_BK = 64, QA_N = 192, QA_RING = 2;
constexpr int QA_ATT_WARPS = 16;                    // drain + attention warps (8 per head of a pass)
constexpr int QA_THREADS = 64 + 32 * QA_ATT_WARPS;
constexpr int QA_STAGE = QA_N * QA_BK * 2;            // 24 KB: q, k, v rows of two heads, one k-block
constexpr int QA_TILE = WA_SLOTS * WA_DH * 2;         // 4 KB: one part of one head of one window
constexpr int QA_MAX_HEADS = 16;

__host__ __device__ constexpr int qa_smem_bytes(int d, int heads) {
  return 1024 /*alignment*/ + (d / QA_BK) * QA_BM * QA_BK * 2 /*Y*/ + QA_RING * QA_STAGE +
         2 * 2 * 2 * 3 * QA_TILE /*Q, K, V tiles of two passes x two heads x two windows*/ + heads * 225 * 4 /*bias tables*/ +
         3 * d * 4 /*QKV bias*/;
}

__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

struct QaArgs {
  const uint8_t* v_in;  // [B*Nt] usable keys of this block
  uint8_t* v_out;       // [B*Nt] the next block's token mask
  void* o;              // [B*Nt][d] attention output (T)
  const float* bias;    // [3d] QKV bias (q | k | v)
  const float* relpos;  // [heads][225] or null
  int Ht, Wt, d, heads, offset, nwx, nwin, units;  // units = B * ceil(nwin / 2) window pairs
  int* err;
};

// Token index of slot s of window wi of frame b (-1 outside the grid or past the last window).
__device__ __forceinline__ int qa_slot_token(const QaArgs& a, int b, int wi, int s) {
  if (wi >= a.nwin) return -1;
  const int wy = wi / a.nwx, wx = wi - wy * a.nwx;
  const int ty = wy * 8 - a.offset + (s >> 3), tx = wx * 8 - a.offset + (s & 7);
  return ty >= 0 && ty < a.Ht && tx >= 0 && tx < a.Wt ? (b * a.Ht + ty) * a.Wt + tx : -1;
}

// Persistent: CTA c takes window pairs c, c + gridDim.x, ...; the producer loads the next
// pair's Y as soon as the current pair's MMAs have read it, and the MMAs of the next pair's
// first passes run while the current pair's last passes are drained and attended.
template <bool RP, typename T>
__global__ void __launch_bounds__(QA_THREADS, 1) qkv_attn_kernel(const __grid_constant__ CUtensorMap tmY,
                                                                 const __grid_constant__ CUtensorMap tmW,
                                                                 const QaArgs args) {
  extern __shared__ uint8_t qsm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(qsm_raw) + 1023) & ~uintptr_t(1023));
  const int d = args.d, KA = d / QA_BK, P = args.heads / 2;
  const int pairs = (args.nwin + 1) / 2;
  uint8_t* sY = smem;                                   // [KA][128 rows x 128 B]: window 0 rows, then window 1
  uint8_t* sW = sY + KA * QA_BM * QA_BK * 2;            // [RING][192 rows x 128 B]
  uint8_t* sT = sW + QA_RING * QA_STAGE;  // [pass parity][head 0, 1][window 0, 1][Q, K, V][64 x 64 B]
  float* s_bias = reinterpret_cast<float*>(sT + 24 * QA_TILE);  // [3d], 16-byte aligned
  float* s_rp = s_bias + 3 * d;                                 // [heads][225]
  __shared__ __align__(8) uint64_t full[QA_RING], empty[QA_RING], a_full, y_empty, acc_full[2], acc_empty[2],
      teardown;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int stok[2][WA_SLOTS];
  __shared__ unsigned okw[2][2];
  auto tile = [&](uint32_t buf, int hh, int win, int part) {
    return sT + (((buf * 2 + hh) * 2 + win) * 3 + part) * QA_TILE;
  };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* err = args.err;

  if (threadIdx.x == 0) {
    for (int s = 0; s < QA_RING; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
    tc::mbar_init(&a_full, 1);
    tc::mbar_init(&y_empty, 1);
    for (int i = 0; i < 2; ++i) { tc::mbar_init(&acc_full[i], 1); tc::mbar_init(&acc_empty[i], QA_ATT_WARPS); }
    tc::mbar_init(&teardown, 1);
    abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmY);
    tc::prefetch_tmap(&tmW);
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_slot, 512);
    tc::tmem_relinquish();
  }
  if (RP)
    for (int e = threadIdx.x; e < args.heads * 225; e += QA_THREADS) s_rp[e] = args.relpos[e];
  for (int e = threadIdx.x; e < 3 * d; e += QA_THREADS) s_bias[e] = args.bias[e];
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem_base = tmem_slot;
  // this CTA's contiguous share of the (window pair, head pass) items, pair-major: pairs
  // u_lo .. u_hi, from pass p_lo(u_lo) of the first to pass p_hi(u_hi) - 1 of the last
  const long long items = (long long)args.units * P;
  const int lo = (int)(items * blockIdx.x / gridDim.x), hi = (int)(items * (blockIdx.x + 1) / gridDim.x);
  const int u_lo = lo / P, u_hi = (hi - 1) / P;
  auto p_lo = [&](int u) { return u == u_lo ? lo - u * P : 0; };
  auto p_hi = [&](int u) { return u == u_hi ? hi - u * P : P; };
  pdl_trigger();
  pdl_wait();

  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      uint32_t g = 0, i = 0;
      for (int u = u_lo; u <= u_hi && ok; ++u, ++i) {
        const int b = u / pairs, w0 = 2 * (u - b * pairs), nh = w0 + 1 < args.nwin ? 2 : 1;
        // Y boxes of the pair: k-block kb of window k at rows 64k of tile kb, once the
        // previous pair's MMAs have read sY
        if (i >= 1 && !tc::mbar_wait(&y_empty, (i - 1) & 1, &abort_flag)) { ok = false; break; }
        tc::mbar_expect_tx(&a_full, (uint32_t)(KA * nh * WA_SLOTS * QA_BK * 2));
        for (int k = 0; k < nh; ++k) {
          const int wi = w0 + k, wy = wi / args.nwx, wx = wi - wy * args.nwx;
          for (int kb = 0; kb < KA; ++kb)
            tc::tma_load_4d(sY + kb * QA_BM * QA_BK * 2 + k * WA_SLOTS * QA_BK * 2, &tmY, &a_full, kb * QA_BK,
                            wx * 8 - args.offset, wy * 8 - args.offset, b);
        }
        for (int p = p_lo(u); p < p_hi(u) && ok; ++p)
          for (int kb = 0; kb < KA; ++kb, ++g) {
            const int s = g % QA_RING;
            if (g >= (uint32_t)QA_RING && !tc::mbar_wait(&empty[s], ((g / QA_RING) & 1) ^ 1, &abort_flag)) {
              ok = false;
              break;
            }
            tc::mbar_expect_tx(&full[s], QA_STAGE);
            for (int part = 0; part < 3; ++part)  // the q, k, v rows of heads 2p, 2p + 1
              tc::tma_load_2d(sW + s * QA_STAGE + part * (QA_N / 3) * QA_BK * 2, &tmW, &full[s], kb * QA_BK,
                              part * d + p * 2 * WA_DH);
          }
      }
      // the loads land before the CTA may exit
      for (uint32_t h = (g > (uint32_t)QA_RING ? g - QA_RING : 0); h < g; ++h)
        if (!tc::mbar_wait_timed(&full[h % QA_RING], (h / QA_RING) & 1)) break;
      if (i >= 1) tc::mbar_wait_timed(&a_full, (i - 1) & 1);
      if (!ok) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        abort_flag = 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_f32acc(H16<T>::kMmaFmt, QA_BM, QA_N);
      bool ok = true;
      uint32_t g = 0, gp = 0, i = 0;
      for (int u = u_lo; u <= u_hi && ok; ++u, ++i) {
        if (!tc::mbar_wait(&a_full, i & 1, &abort_flag)) { ok = false; break; }
        tc::fence_after_sync();
        for (int p = p_lo(u); p < p_hi(u) && ok; ++p, ++gp) {
          const uint32_t buf = gp & 1, use = gp >> 1;
          if (use >= 1 && !tc::mbar_wait(&acc_empty[buf], (use & 1) ^ 1, &abort_flag)) { ok = false; break; }
          tc::fence_after_sync();
          for (int kb = 0; kb < KA; ++kb, ++g) {
            const int s = g % QA_RING;
            if (!tc::mbar_wait(&full[s], (g / QA_RING) & 1, &abort_flag)) { ok = false; break; }
            tc::fence_after_sync();
            const uint64_t ad = tc::desc_kmajor_sw128(tc::smem_u32(sY + kb * QA_BM * QA_BK * 2));
            const uint64_t bd = tc::desc_kmajor_sw128(tc::smem_u32(sW + s * QA_STAGE));
#pragma unroll
            for (int kk = 0; kk < QA_BK / 16; ++kk)
              tc::mma_f16(tmem_base + buf * 256, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0);
            tc::mma_commit(&empty[s]);
          }
          if (ok) tc::mma_commit(&acc_full[buf]);
        }
        if (ok) tc::mma_commit(&y_empty);  // sY is free once the pair's MMAs have completed
      }
      if (!ok) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        abort_flag = 1;
      }
      tc::mma_commit(&teardown);  // every issued MMA has finished before TMEM is released
      tc::mbar_wait_timed(&teardown, 0);
    }
    __syncwarp();
  } else {
    // ---- drain + attention: head hh of every pass for the eight warps of group hh; warp j
    // of a group drains TMEM lane quarter (warp & 3), the q columns and k channels 0..15
    // (j < 4) or k channels 16..31 and the v columns, then runs query rows 16 (j & 3) ..
    // + 15 of window j >> 2
    const int quarter = warp & 3, hh = (warp - 2) >> 3, j = (warp - 2) & 7;
    const int win = quarter >> 1, slot = 32 * (quarter & 1) + lane;  // this thread's accumulator row
    const int awin = j >> 2, wq = j & 3;
    const int e = threadIdx.x - 64;  // slot e & 63 of window e >> 6 of a pair, for e < 128
    T* o = static_cast<T*>(args.o);
    // the usable-key flag of this thread's slot of the next pair, loaded a pair ahead
    int t_next = -1;
    bool ok_next = false;
    auto fetch = [&](int u) {
      t_next = -1;
      ok_next = false;
      if (e < 2 * WA_SLOTS && u < args.units) {
        const int b = u / pairs;
        t_next = qa_slot_token(args, b, 2 * (u - b * pairs) + (e >> 6), e & 63);
        if (t_next >= 0) ok_next = args.v_in[t_next] != 0;
      }
    };
    fetch(u_lo);
    // every attention warp passes every named barrier of every pair, also after a failed
    // wait (then skipping the work), so that no warp waits for a peer that has left
    bool ok = true;
    uint32_t gp = 0;
    for (int u = u_lo; u <= u_hi; ++u) {
      const int b = u / pairs, nh = 2 * (u - b * pairs) + 1 < args.nwin ? 2 : 1;
      named_sync(3, 32 * QA_ATT_WARPS);  // the previous pair's windows are no longer read
      if (e < 2 * WA_SLOTS) {
        stok[e >> 6][e & 63] = t_next;
        const unsigned bal = __ballot_sync(0xffffffffu, ok_next);
        if (lane == 0) okw[e >> 6][(e >> 5) & 1] = bal;
      }
      named_sync(3, 32 * QA_ATT_WARPS);
      // the next block's token mask of the pair: written by the CTA that runs its first pass
      if (p_lo(u) == 0 && e < 2 * WA_SLOTS && t_next >= 0)
        args.v_out[t_next] = (okw[e >> 6][0] | okw[e >> 6][1]) != 0u;
      fetch(u < u_hi ? u + 1 : args.units);
      for (int p = p_lo(u); p < p_hi(u); ++p, ++gp) {
        const uint32_t buf = gp & 1, use = gp >> 1;
        const int hg = 2 * p + hh;
        if (ok && !tc::mbar_wait(&acc_full[buf], use & 1, &abort_flag)) ok = false;
        if (ok) {
          __syncwarp();
          tc::fence_after_sync();
          const uint32_t tb = tmem_base + ((uint32_t)(quarter * 32) << 16) + buf * 256 + hh * 32;
          // 8 FP32 accumulator values + bias -> T, as 16-byte chunk c of the row of `part`
          auto put = [&](int part, int c, const uint32_t* v) {
            const float* bb = s_bias + part * d + hg * WA_DH + 8 * c;
            const float4 b0 = *reinterpret_cast<const float4*>(bb);
            const float4 b1 = *reinterpret_cast<const float4*>(bb + 4);
            *reinterpret_cast<uint4*>(tile(buf, hh, win, part) + swz64(slot, c)) =
                make_uint4(H16<T>::pack2(__uint_as_float(v[0]) + b0.x, __uint_as_float(v[1]) + b0.y),
                           H16<T>::pack2(__uint_as_float(v[2]) + b0.z, __uint_as_float(v[3]) + b0.w),
                           H16<T>::pack2(__uint_as_float(v[4]) + b1.x, __uint_as_float(v[5]) + b1.y),
                           H16<T>::pack2(__uint_as_float(v[6]) + b1.z, __uint_as_float(v[7]) + b1.w));
          };
          // 48 of the head's 96 columns each: q and the first half of k, or the second half
          // of k and v
          uint32_t v32[32], v16[16];
          if (j < 4) {
            tc::tmem_ld_32x32b_x32(tb, v32);       // q
            tc::tmem_ld_32x32b_x16(tb + 64, v16);  // k channels 0..15
          } else {
            tc::tmem_ld_32x32b_x32(tb + 128, v32);     // v
            tc::tmem_ld_32x32b_x16(tb + 64 + 16, v16);  // k channels 16..31
          }
          tc::tmem_ld_wait();
          const int p32 = j < 4 ? 0 : 2, c16 = j < 4 ? 0 : 2;
#pragma unroll
          for (int c = 0; c < 4; ++c) put(p32, c, v32 + 8 * c);
#pragma unroll
          for (int c = 0; c < 2; ++c) put(1, c16 + c, v16 + 8 * c);
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&acc_empty[buf]);  // the accumulator is free for pass gp + 2
        }
        // the head's Q, K, V tiles of both windows are complete; the group's warps have also
        // left pass gp - 1's attention, so pass gp + 1 may drain into that pass's tiles
        named_sync(1 + hh, 256);
        if (ok && awin < nh) {
          const unsigned long long keymask =
              (unsigned long long)okw[awin][0] | ((unsigned long long)okw[awin][1] << 32);
          if (keymask == 0ull) {  // no usable key: the window outputs 0
            for (int x = lane; x < 16 * 4; x += 32) {
              const int t = stok[awin][16 * wq + (x >> 2)];
              if (t >= 0)
                *reinterpret_cast<uint4*>(o + (size_t)t * d + hg * WA_DH + (x & 3) * 8) = make_uint4(0, 0, 0, 0);
            }
          } else {
            window_attention_rows<RP, T>(tile(buf, hh, awin, 0), tile(buf, hh, awin, 1), tile(buf, hh, awin, 2), keymask,
                                         RP ? s_rp + hg * 225 : nullptr, stok[awin], o, d, hg * WA_DH, 16 * wq,
                                         lane);
          }
        }
      }
    }
    if (!ok) {
      if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
      abort_flag = 1;
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, 512);
  }
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

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n < 1) n = 1;
  }
  return n;
}

template <bool RP, typename T>
cudaError_t launch_t(const CUtensorMap& my, const CUtensorMap& mw, const QaArgs& a, cudaStream_t st) {
  static int attr = 0;
  const int smem = qa_smem_bytes(a.d, a.heads);
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(qkv_attn_kernel<RP, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  const int items = a.units * (a.heads / 2);  // (window pair, head pass) items
  const dim3 grid(items < num_sms() ? items : num_sms());
  return launch_pdl(qkv_attn_kernel<RP, T>, grid, dim3(QA_THREADS), (size_t)smem, st, my, mw, a);
}

}  // namespace

bool qkv_attn_supported(int d, int heads) {
  return d % QA_BK == 0 && d == heads * WA_DH && heads % 2 == 0 && heads <= QA_MAX_HEADS &&
         qa_smem_bytes(d, heads) <= 232448;
}

template <typename T>
cudaError_t launch_qkv_attn(const T* y, const T* wqkv_t, const float* bias, const uint8_t* v_in, T* o, uint8_t* v_out,
                            int B, int Ht, int Wt, int d, int heads, int offset, const float* relpos, int* err,
                            cudaStream_t st) {
  if (!qkv_attn_supported(d, heads) || B < 1 || Ht < 1 || Wt < 1) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(wqkv_t) | reinterpret_cast<uintptr_t>(o)) & 15)
    return cudaErrorInvalidValue;
  auto fn = encode_fn();
  if (!fn) return cudaErrorInvalidValue;
  CUtensorMap my, mw;
  {  // Y [B][Ht][Wt][d]: boxes {64 channels, 8 x 8 tokens}, 128-byte swizzle (the K-major operand layout)
    const uint64_t row = (uint64_t)d * 2;
    cuuint64_t dims[4] = {(cuuint64_t)d, (cuuint64_t)Wt, (cuuint64_t)Ht, (cuuint64_t)B};
    cuuint64_t strides[3] = {row, row * Wt, row * Wt * Ht};
    cuuint32_t box[4] = {QA_BK, 8, 8, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    if (fn(&my, tc::tma_dtype<T>(), 4, const_cast<T*>(y), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {  // W^T [3d][d]: boxes of 64 output rows x 64 inputs
    cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)3 * d};
    cuuint64_t strides[1] = {(cuuint64_t)d * 2};
    cuuint32_t box[2] = {QA_BK, (cuuint32_t)(QA_N / 3)};
    cuuint32_t es[2] = {1, 1};
    if (fn(&mw, tc::tma_dtype<T>(), 2, const_cast<T*>(wqkv_t), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  const int nwy = (Ht + offset + 7) / 8, nwx = (Wt + offset + 7) / 8;
  const int nwin = nwy * nwx;
  QaArgs a{v_in, v_out, o, bias, relpos, Ht, Wt, d, heads, offset, nwx, nwin, B * ((nwin + 1) / 2), err};
  return relpos ? launch_t<true, T>(my, mw, a, st) : launch_t<false, T>(my, mw, a, st);
}

template cudaError_t launch_qkv_attn<bf16>(const bf16*, const bf16*, const float*, const uint8_t*, bf16*, uint8_t*, int,
                                           int, int, int, int, int, const float*, int*, cudaStream_t);
template cudaError_t launch_qkv_attn<f16>(const f16*, const f16*, const float*, const uint8_t*, f16*, uint8_t*, int,
                                          int, int, int, int, int, const float*, int*, cudaStream_t);

}  // namespace inpaint
