// Fused MLP of a transformer block on tcgen05 (BF16 form):
//   for a tile of 128 token rows and hidden chunks j of 128 columns
//     H_j  = gelu(Y . W1[:, j] + b1[j])            (MMA1 into TMEM, epilogue to SMEM)
//     OUT += H_j . W2[j, :]                         (MMA2 from SMEM into TMEM)
//   x = x + OUT + b2, ln_out = LayerNorm(x) (the next block's LN1, or the final LN).
// The hidden activations never leave the SM: this removes the write and re-read of the
// [M, r*d] hidden tensor and keeps the MLP bound by the tensor pipe, not HBM.
//
// Y (LN2 output, bf16 [M, D]) is loaded once per tile by TMA and stays in SMEM; W1^T
// ([hid][D]) k-blocks and W2^T ([D][hid]) k-blocks (as <=128-row halves, one MMA2 per
// half of OUT's columns) stream through a 5-stage ring of 16 KB in the order the MMA
// warp consumes them (MMA1 of chunk j+1 is issued before MMA2 of chunk j, so the tensor
// core works while the epilogue warps turn H_j into bf16).  TMEM: OUT (D cols)
// + two H buffers (128 cols each).  The bf16 H_j is written in the 128-byte-swizzled
// K-major layout that the MMA descriptor expects (16-byte chunk c of row r at c ^ (r%8)).
//
// Warps: 0 TMA producer, 1 TMEM owner + MMA issuer (2, 3 idle: warpgroup 0 hands its
// registers to the final warps), 4..11 hidden-chunk epilogue (two per
// TMEM lane quarter, splitting the chunk's columns), then 4*OW final-epilogue warps (OW per
// lane quarter, D/OW columns of a row each: residual, store, LayerNorm; the parts'
// statistics are merged through shared memory).  OW = 1 measured fastest.  The final epilogue of a tile overlaps the next tile's
// hidden chunks; it drains the output accumulator before the next tile's MMA2 can start,
// so each chunk's residual loads overlap its TMEM load, and rows move between global and
// shared memory in whole 64-byte segments (warp_rows.cuh).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc_primitives.cuh"
#include "warp_rows.cuh"

namespace inpaint {

namespace {

constexpr int BM = 128, BK = 64, HC = 128;   // rows per tile, k-block, hidden chunk
constexpr int ROLE_WARPS = 4;                 // warpgroup 0: TMA producer, MMA issuer, two idle
constexpr int EW = 2, EPI_WARPS = 4 * EW;     // GELU warps: two per TMEM lane quarter
constexpr int OW = 1, OUT_WARPS = 4 * OW;     // final-epilogue warps per lane quarter
constexpr int THREADS = 32 * (ROLE_WARPS + EPI_WARPS + OUT_WARPS);
// Registers per thread: launched with 65536 / THREADS; warpgroup 0 gives most of its share
// to the final-epilogue warpgroup, which keeps two chunks of residual loads in flight.
constexpr int REG_LAUNCH = 65536 / THREADS, REG_ROLE = 64, REG_FINAL = 184;
static_assert(OUT_WARPS == 4 && ROLE_WARPS == 4, "register reallocation is per warpgroup");
static_assert(ROLE_WARPS * REG_ROLE + EPI_WARPS * REG_LAUNCH + OUT_WARPS * REG_FINAL <=
                  (ROLE_WARPS + EPI_WARPS + OUT_WARPS) * REG_LAUNCH,
              "register reallocation exceeds the launch allotment");
constexpr int RING = 5;                      // 16 KB weight stages

template <int D>
struct MlpCfg {
  static constexpr int A_BYTES = BM * D * 2;                  // Y tile, D/64 atoms of 16 KB
  static constexpr int HS_BYTES = BM * HC * 2;                // one bf16 H chunk, 2 atoms
  static constexpr int W1_BYTES = HC * BK * 2;                // one W1 k-block (HC rows)
  static constexpr int HR = D < 128 ? D : 128;                // W2 rows per load (N of MMA2)
  static constexpr int NHALF = D / HR;                        // W2 k-block = NHALF loads
  static constexpr int W2_BYTES = HR * BK * 2;
  static constexpr int STAGE_BYTES = 16384;
  static constexpr int PARAM_FLOATS = 1024 + 3 * D;          // b1 (hid <= 1024), b2, LayerNorm scale/shift
  static constexpr int SMEM_BYTES = A_BYTES + 2 * HS_BYTES + RING * STAGE_BYTES + 1024 /*align slack*/ +
                                    512 /*barriers*/ + OUT_WARPS * 32 * 2 * 4 /*LayerNorm partials*/ +
                                    PARAM_FLOATS * 4 + OUT_WARPS * rows::TILE_BYTES /*row staging tiles*/;
  static constexpr int H_COL0 = 256;                          // H buffers at TMEM columns 256 and 384
  static_assert(SMEM_BYTES <= 232448, "exceeds the 227 KB dynamic shared memory of an sm_100-family CTA");
};

struct MlpArgs {
  float* X;              // residual stream [M, D] f32, updated in place
  bf16* ln_out;          // [M, D]
  const float* b1;       // [hid]
  const float* b2;       // [D]
  const float* ln_g;
  const float* ln_b;
  int M, hid;
  int* err;
};

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void load32s(const float* p, float (&v)[32]) {  // shared memory
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 t = *reinterpret_cast<const float4*>(p + 4 * i);
    v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
  }
}
template <int D, int CS>
__global__ void __launch_bounds__(THREADS, 1) mlp_tc_kernel(const __grid_constant__ CUtensorMap tmY,
                                                            const __grid_constant__ CUtensorMap tmW1,
                                                            const __grid_constant__ CUtensorMap tmW2,
                                                            const MlpArgs args) {
  using Cfg = MlpCfg<D>;
  constexpr int KA = D / BK;   // k-blocks of MMA1 (and atoms of the Y tile)
  constexpr int KH = HC / BK;  // k-blocks of MMA2 per hidden chunk
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sH = sA + Cfg::A_BYTES;                      // 2 buffers
  uint8_t* sR = sH + 2 * Cfg::HS_BYTES;                 // ring
  uint64_t* bar = reinterpret_cast<uint64_t*>(sR + RING * Cfg::STAGE_BYTES);
  static_assert(Cfg::W1_BYTES <= Cfg::STAGE_BYTES && Cfg::W2_BYTES <= Cfg::STAGE_BYTES, "stage too small");
  uint64_t* full = bar;                 // [RING]
  uint64_t* empty = full + RING;        // [RING]
  uint64_t* a_full = empty + RING;
  uint64_t* a_empty = a_full + 1;
  uint64_t* h_full = a_empty + 1;       // [2]
  uint64_t* h_empty = h_full + 2;       // [2]
  uint64_t* hs_full = h_empty + 2;      // [2]
  uint64_t* hs_empty = hs_full + 2;     // [2]
  uint64_t* o_full = hs_empty + 2;
  uint64_t* o_empty = o_full + 1;
  uint64_t* teardown = o_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(teardown + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* ln_stats = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bar) + 512);  // [OUT_WARPS][32][2]
  float* s_b1 = ln_stats + OUT_WARPS * 32 * 2;   // [hid]
  float* s_b2 = s_b1 + 1024;                     // [D]
  float* s_lng = s_b2 + D;
  float* s_lnb = s_lng + D;
  uint8_t* s_tile = reinterpret_cast<uint8_t*>(s_lnb + D);  // [OUT_WARPS][2 KB]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = args.M, NJ = args.hid / HC;
  const int tiles = (M + BM - 1) / BM;
  int* err = args.err;
  // A cluster of CS CTAs walks groups of CS consecutive tiles in lockstep (every tile
  // consumes the same weight sequence); CTA `rank` takes tile grp*CS + rank, which may lie
  // past the last tile: it then computes on zero rows and stores nothing.
  const int rank = CS > 1 ? (int)tc::cluster_ctarank() : 0;
  const int cid = blockIdx.x / CS, ncl = gridDim.x / CS;
  const int groups = (tiles + CS - 1) / CS;
  constexpr uint16_t MASK = (uint16_t)((1u << CS) - 1);

  if (threadIdx.x == 0) {
    // a ring slot is refilled (in every CTA of the cluster) once all CS consumers released it
    for (int s = 0; s < RING; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], CS); }
    tc::mbar_init(a_full, 1);
    tc::mbar_init(a_empty, 1);
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&h_full[b], 1);
      tc::mbar_init(&h_empty[b], EPI_WARPS);
      tc::mbar_init(&hs_full[b], EPI_WARPS);
      tc::mbar_init(&hs_empty[b], 1);
    }
    tc::mbar_init(o_full, 1);
    tc::mbar_init(o_empty, OUT_WARPS);
    tc::mbar_init(teardown, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmY);
    tc::prefetch_tmap(&tmW1);
    tc::prefetch_tmap(&tmW2);
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, 512);
    tc::tmem_relinquish();
  }
  for (int c = threadIdx.x; c < args.hid; c += blockDim.x) s_b1[c] = args.b1[c];
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    s_b2[c] = args.b2[c];
    s_lng[c] = args.ln_g[c];
    s_lnb[c] = args.ln_b[c];
  }
  tc::fence_before_sync();
  __syncthreads();
  if (CS > 1) tc::cluster_sync();  // every CTA's barriers exist before any multicast reaches them
  tc::fence_after_sync();
  const uint32_t tmem_base = *tmem_slot;

  if (warp < ROLE_WARPS) {
  tc::setmaxnreg_dec<REG_ROLE>();
  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;  // ring slot counter
      bool ok = true;
      // each CTA loads 1/CS of every weight stage (rows rank*slice ..) and multicasts it
      // to the whole cluster; the stage's barrier expects the full stage
      auto push = [&](const CUtensorMap* map, int c0, int c1, uint32_t bytes, int slice_rows) {
        const int s = g % RING;
        if (g >= (uint32_t)RING && !tc::mbar_wait(&empty[s], ((g / RING) & 1) ^ 1, abort_flag)) return false;
        tc::mbar_expect_tx(&full[s], bytes);
        uint8_t* dst = sR + s * Cfg::STAGE_BYTES + rank * slice_rows * 128;
        if (CS > 1)
          tc::tma_load_2d_mc(dst, map, &full[s], c0, c1 + rank * slice_rows, MASK);
        else
          tc::tma_load_2d(dst, map, &full[s], c0, c1);
        ++g;
        return true;
      };
      int t = 0;
      for (int grp = cid; grp < groups && ok; grp += ncl, ++t) {
        const int m0 = (grp * CS + rank) * BM;
        if (t >= 1 && !tc::mbar_wait(a_empty, (t - 1) & 1, abort_flag)) { ok = false; break; }
        if (m0 < M) {
          tc::mbar_expect_tx(a_full, Cfg::A_BYTES);
          for (int kb = 0; kb < KA; ++kb) tc::tma_load_2d(sA + kb * (BM * BK * 2), &tmY, a_full, kb * BK, m0);
        } else {
          tc::mbar_arrive(a_full);  // a tile past the end: its results are never stored
        }
        for (int j = 0; j <= NJ && ok; ++j) {
          if (j < NJ)
            for (int kb = 0; kb < KA && ok; ++kb) ok = push(&tmW1, kb * BK, j * HC, Cfg::W1_BYTES, HC / CS);
          if (j >= 1)
            for (int kb = 0; kb < KH && ok; ++kb)
              for (int hf = 0; hf < Cfg::NHALF && ok; ++hf)
                ok = push(&tmW2, (j - 1) * HC + kb * BK, hf * Cfg::HR, Cfg::W2_BYTES, Cfg::HR / CS);
        }
      }
      for (uint32_t h = (g > (uint32_t)RING ? g - RING : 0); h < g; ++h)
        if (!tc::mbar_wait_timed(&full[h % RING], (h / RING) & 1)) break;
      // and the other CTAs' releases of the last stages, which arrive on this CTA's barriers
      if (CS > 1)
        for (uint32_t h = (g > (uint32_t)RING ? g - RING : 0); h < g; ++h)
          if (!tc::mbar_wait_timed(&empty[h % RING], (h / RING) & 1)) break;
      if (!ok) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        *abort_flag = 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t id1 = tc::idesc_bf16_f32(BM, HC);
      constexpr uint32_t id2 = tc::idesc_bf16_f32(BM, Cfg::HR);
      uint32_t g = 0, q = 0;  // ring slot counter, hidden-chunk counter (across tiles)
      bool ok = true;
      auto release = [&](int s) {  // the stage's MMAs are done: free it in every CTA of the cluster
        if (CS > 1)
          tc::mma_commit_mc(&empty[s], MASK);
        else
          tc::mma_commit(&empty[s]);
      };
      auto pop = [&](int& s) {
        s = g % RING;
        if (!tc::mbar_wait(&full[s], (g / RING) & 1, abort_flag)) return false;
        tc::fence_after_sync();
        ++g;
        return true;
      };
      auto mma1 = [&](uint32_t qq) {  // H[qq & 1] = Y . W1_chunk^T
        const uint32_t hb = qq & 1, use = qq >> 1;
        if (use >= 1 && !tc::mbar_wait(&h_empty[hb], (use & 1) ^ 1, abort_flag)) return false;
        tc::fence_after_sync();
        const uint32_t dt = tmem_base + Cfg::H_COL0 + hb * HC;
        for (int kb = 0; kb < KA; ++kb) {
          int s;
          if (!pop(s)) return false;
          const uint64_t ad = tc::desc_kmajor_sw128(tc::smem_u32(sA + kb * (BM * BK * 2)));
          const uint64_t bd = tc::desc_kmajor_sw128(tc::smem_u32(sR + s * Cfg::STAGE_BYTES));
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) tc::mma_f16(dt, ad + 2 * kk, bd + 2 * kk, id1, (kb | kk) != 0);
          release(s);
        }
        tc::mma_commit(&h_full[hb]);
        return true;
      };
      auto mma2 = [&](uint32_t qq, bool first, bool last, int t) {  // OUT (+)= Hs[qq & 1] . W2_chunk^T
        const uint32_t hb = qq & 1, use = qq >> 1;
        if (first && t >= 1 && !tc::mbar_wait(o_empty, (t - 1) & 1, abort_flag)) return false;
        if (!tc::mbar_wait(&hs_full[hb], use & 1, abort_flag)) return false;
        tc::fence_after_sync();
        for (int kb = 0; kb < KH; ++kb) {
          const uint64_t ad = tc::desc_kmajor_sw128(tc::smem_u32(sH + hb * Cfg::HS_BYTES + kb * (BM * BK * 2)));
          for (int hf = 0; hf < Cfg::NHALF; ++hf) {  // OUT columns hf*HR .. +HR
            int s;
            if (!pop(s)) return false;
            const uint64_t bd = tc::desc_kmajor_sw128(tc::smem_u32(sR + s * Cfg::STAGE_BYTES));
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              tc::mma_f16(tmem_base + hf * Cfg::HR, ad + 2 * kk, bd + 2 * kk, id2, (!first || kb || kk) ? 1u : 0u);
            release(s);
          }
        }
        tc::mma_commit(&hs_empty[hb]);
        if (last) tc::mma_commit(o_full);
        return true;
      };
      int t = 0;
      for (int grp = cid; grp < groups && ok; grp += ncl, ++t) {
        if (!tc::mbar_wait(a_full, t & 1, abort_flag)) { ok = false; break; }
        tc::fence_after_sync();
        const uint32_t q0 = q;
        for (int j = 0; j <= NJ && ok; ++j) {
          if (j < NJ) {
            ok = mma1(q0 + j);
            if (ok && j == NJ - 1) tc::mma_commit(a_empty);  // Y tile no longer read after the last MMA1
          }
          if (ok && j >= 1) ok = mma2(q0 + j - 1, j == 1, j == NJ, t);
        }
        q = q0 + NJ;
      }
      if (!ok) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        *abort_flag = 1;
      }
      tc::mma_commit(teardown);
      tc::mbar_wait_timed(teardown, 0);
    }
    __syncwarp();
  }
  } else if (warp < ROLE_WARPS + EPI_WARPS) {
    // ---- hidden chunks: TMEM H -> bias + GELU -> bf16 swizzled SMEM operand of MMA2
    const int quarter = warp & 3, cg = (warp - ROLE_WARPS) >> 2;
    const int r = quarter * 32 + lane;  // row within the tile (= TMEM lane)
    const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
    uint32_t q = 0;
    bool ok = true;
    for (int grp = cid; grp < groups && ok; grp += ncl) {
      for (int j = 0; j < NJ; ++j, ++q) {
        const uint32_t hb = q & 1, use = q >> 1;
        if (!tc::mbar_wait(&h_full[hb], use & 1, abort_flag)) { ok = false; break; }
        if (use >= 1 && !tc::mbar_wait(&hs_empty[hb], (use & 1) ^ 1, abort_flag)) { ok = false; break; }
        __syncwarp();
        tc::fence_after_sync();
        uint8_t* hs = sH + hb * Cfg::HS_BYTES;
#pragma unroll 1
        for (int c0 = cg * (HC / EW); c0 < (cg + 1) * (HC / EW); c0 += 32) {
          uint32_t v[32];
          tc::tmem_ld_32x32b_x32(lane_base + Cfg::H_COL0 + hb * HC + c0, v);
          tc::tmem_ld_wait();
          float bv[32];
          load32s(s_b1 + j * HC + c0, bv);
          uint32_t pk[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float a0 = gelu_as(__uint_as_float(v[2 * k]) + bv[2 * k]);
            const float a1 = gelu_as(__uint_as_float(v[2 * k + 1]) + bv[2 * k + 1]);
            __nv_bfloat162 h2 = __floats2bfloat162_rn(a0, a1);
            pk[k] = *reinterpret_cast<uint32_t*>(&h2);
          }
          // columns c0 .. c0+31 of row r: atom c0/64, 16-byte chunks (c0%64)/8 .. +3, swizzled by r%8
          uint8_t* rowp = hs + (c0 >> 6) * (BM * BK * 2) + r * 128;
          const int ch0 = (c0 & 63) >> 3;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            *reinterpret_cast<uint4*>(rowp + (((ch0 + k) ^ (r & 7)) << 4)) =
                make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
        }
        tc::fence_before_sync();
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          tc::mbar_arrive(&h_empty[hb]);
          tc::mbar_arrive(&hs_full[hb]);
        }
      }
    }
    if (!ok) {
      if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
      *abort_flag = 1;
    }
  } else {
    // ---- final: x = x + OUT + b2, LayerNorm(x) -> bf16; D/OW columns of a row per thread
    tc::setmaxnreg_inc<REG_FINAL>();
    const int fw = warp - ROLE_WARPS - EPI_WARPS;  // 0 .. OUT_WARPS-1
    const int quarter = warp & 3, half = fw >> 2;
    const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
    const int c_lo = half * (D / OW);
    uint8_t* tl = s_tile + (size_t)fw * rows::TILE_BYTES;
    bool ok = true;
    int t = 0;
    for (int grp = cid; grp < groups && ok; grp += ncl, ++t) {
      const int row0 = (grp * CS + rank) * BM + quarter * 32;  // this warp's 32 rows; the thread owns row0 + lane
      const int nvalid = M - row0;
      float* xb = args.X + (size_t)row0 * D;
      if (lane < nvalid)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(xb + (size_t)lane * D + c_lo), "r"(D / OW * 4)
                     : "memory");
      if (!tc::mbar_wait(o_full, t & 1, abort_flag)) { ok = false; break; }
      __syncwarp();
      tc::fence_after_sync();
      float run_n = 0.f, run_mean = 0.f, run_m2 = 0.f;
      constexpr int c_hi = D / OW;  // (c_lo = 0 when OW = 1)
      float4 gn[8];                 // the next chunk's residual, loaded one chunk ahead
      rows::load32_issue(xb + c_lo, D, nvalid, lane, gn);
#pragma unroll 1
      for (int c0 = c_lo; c0 < c_lo + c_hi; c0 += 32) {
        uint32_t v[32];
        tc::tmem_ld_32x32b_x32(lane_base + c0, v);
        float f[32];
        rows::load32_finish(tl, lane, gn, f);
        if (c0 + 32 < c_lo + c_hi) rows::load32_issue(xb + c0 + 32, D, nvalid, lane, gn);
        tc::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 32; k += 4) {
          const float4 b = *reinterpret_cast<const float4*>(s_b2 + c0 + k);
          f[k] += __uint_as_float(v[k]) + b.x;
          f[k + 1] += __uint_as_float(v[k + 1]) + b.y;
          f[k + 2] += __uint_as_float(v[k + 2]) + b.z;
          f[k + 3] += __uint_as_float(v[k + 3]) + b.w;
        }
        rows::store32_f32(xb + c0, D, nvalid, tl, lane, f);
        float cm = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) cm += f[k];
        cm *= (1.f / 32.f);
        float cq = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) cq = fmaf(f[k] - cm, f[k] - cm, cq);
        const float nn = run_n + 32.f;
        const float dl = cm - run_mean;
        run_mean += dl * (32.f / nn);
        run_m2 += cq + dl * dl * (run_n * 32.f / nn);
        run_n = nn;
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(o_empty);  // OUT drained: the next tile's MMA2 may start
      float mean = run_mean, m2 = run_m2, n = run_n;
      if (OW > 1) {
        // merge the parts of each row in a fixed order
        float* st = ln_stats + ((size_t)fw * 32 + lane) * 2;
        st[0] = run_mean;
        st[1] = run_m2;
        named_sync(1 + quarter, 32 * OW);
        mean = 0.f; m2 = 0.f; n = 0.f;
#pragma unroll
        for (int g2 = 0; g2 < OW; ++g2) {
          // final warp of part g2 in this quarter: fw = 4*g2 + ((quarter - 2) & 3)
          const float* o = ln_stats + ((size_t)(4 * g2 + ((quarter - 2) & 3)) * 32 + lane) * 2;
          const float om = o[0], oq = o[1], on = (float)(D / OW);
          const float nn = n + on;
          const float dl = om - mean;
          mean += dl * (on / nn);
          m2 += oq + dl * dl * (n * on / nn);
          n = nn;
        }
        named_sync(1 + quarter, 32 * OW);  // the partial slots are reused by the next tile
      }
      const float rstd = rsqrtf(m2 / n + 1e-5f);
      rows::load32_issue(xb + c_lo, D, nvalid, lane, gn);
#pragma unroll 1
      for (int c0 = c_lo; c0 < c_lo + c_hi; c0 += 32) {
        float xv[32];
        rows::load32_finish(tl, lane, gn, xv);  // the rows this warp stored above
        if (c0 + 32 < c_lo + c_hi) rows::load32_issue(xb + c0 + 32, D, nvalid, lane, gn);
#pragma unroll
        for (int k = 0; k < 32; k += 4) {
          const float4 g4 = *reinterpret_cast<const float4*>(s_lng + c0 + k);
          const float4 b4 = *reinterpret_cast<const float4*>(s_lnb + c0 + k);
          xv[k] = (xv[k] - mean) * rstd * g4.x + b4.x;
          xv[k + 1] = (xv[k + 1] - mean) * rstd * g4.y + b4.y;
          xv[k + 2] = (xv[k + 2] - mean) * rstd * g4.z + b4.z;
          xv[k + 3] = (xv[k + 3] - mean) * rstd * g4.w + b4.w;
        }
        rows::store32_bf16(args.ln_out + (size_t)row0 * D + c0, D, nvalid, tl, lane, xv);
      }
    }
    if (!ok) {
      if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
      *abort_flag = 1;
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (CS > 1) tc::cluster_sync();  // no CTA leaves while another may still signal it
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

bool map2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint32_t box_inner, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <int D, int CS>
cudaError_t launch_dc(const bf16* Y, const bf16* W1t, const bf16* W2t, const MlpArgs& a, cudaStream_t st) {
  using Cfg = MlpCfg<D>;
  auto kern = mlp_tc_kernel<D, CS>;
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.blockDim = dim3(THREADS);
  lc.dynamicSmemBytes = Cfg::SMEM_BYTES;
  lc.stream = st;
  lc.attrs = at;
  lc.numAttrs = 1;
  static int max_clusters = 0;  // co-resident clusters of CS CTAs at one CTA per SM
  if (!max_clusters) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    lc.gridDim = dim3(num_sms() / CS * CS);
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &lc);
    if (e != cudaSuccess) return e;
    max_clusters = n > 0 ? n : 1;
  }
  CUtensorMap my, m1, m2;
  if (!map2d(&my, Y, D, (uint64_t)a.M, BK, BM)) return cudaErrorInvalidValue;
  if (!map2d(&m1, W1t, D, (uint64_t)a.hid, BK, HC / CS)) return cudaErrorInvalidValue;
  if (!map2d(&m2, W2t, (uint64_t)a.hid, D, BK, Cfg::HR / CS)) return cudaErrorInvalidValue;
  const int groups = ((a.M + BM - 1) / BM + CS - 1) / CS;
  lc.gridDim = dim3((groups < max_clusters ? groups : max_clusters) * CS);
  cudaError_t e = cudaLaunchKernelEx(&lc, kern, my, m1, m2, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Weight stages are shared by clusters of two CTAs: half the L2 reads of the weights per
// tile, which all CTAs otherwise stream from the same lines at the same time.
constexpr int MLP_CLUSTER = 2;

template <int D>
cudaError_t launch_d(const bf16* Y, const bf16* W1t, const bf16* W2t, const MlpArgs& a, cudaStream_t st) {
  return launch_dc<D, MLP_CLUSTER>(Y, W1t, W2t, a, st);
}

}  // namespace

bool mlp_tc_supported(int d, int hid) {
  return (d == 64 || d == 128 || d == 256) && hid % HC == 0 && hid >= HC && hid <= 1024;
}

cudaError_t launch_mlp_tc(const bf16* Y, const bf16* W1t, const bf16* W2t, const float* b1, const float* b2, float* X,
                          const float* ln_g, const float* ln_b, bf16* ln_out, int M, int d, int hid, int* err,
                          cudaStream_t st) {
  if (!mlp_tc_supported(d, hid) || M <= 0) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(Y) | reinterpret_cast<uintptr_t>(W1t) | reinterpret_cast<uintptr_t>(W2t)) & 15)
    return cudaErrorInvalidValue;
  MlpArgs a{X, ln_out, b1, b2, ln_g, ln_b, M, hid, err};
  if (d == 256) return launch_d<256>(Y, W1t, W2t, a, st);
  if (d == 128) return launch_d<128>(Y, W1t, W2t, a, st);
  return launch_d<64>(Y, W1t, W2t, a, st);
}

}  // namespace inpaint
