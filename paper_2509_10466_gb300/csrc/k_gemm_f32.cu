// FP32 SIMT GEMM: the plain FP32 form of the token GEMMs (QKV, proj, MLP) and the
// GEMMs of the backward pass.  FFMA only (no TF32), 128x128x8 CTA tiles, 8x8 outputs
// per thread, register-prefetched double-buffered shared memory.  Split-K writes
// partial tiles that a fixed-order reduction sums, so results are deterministic.
#include "common.cuh"

namespace inpaint {

namespace {

constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8, NT = 256;

template <bool TA, bool TB>
__device__ __forceinline__ void load_tiles(const float* __restrict__ A, int lda, const float* __restrict__ Bm,
                                           int ldb, int M, int N, int K, int m0, int n0, int k0, float ra[4],
                                           float rb[4]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = tid + i * NT;
    int m, k;
    if (TA) { m = e % BM; k = e / BM; } else { k = e % BK; m = e / BK; }
    const int gm = m0 + m, gk = k0 + k;
    ra[i] = (gm < M && gk < K) ? (TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = tid + i * NT;
    int n, k;
    if (TB) { k = e % BK; n = e / BK; } else { n = e % BN; k = e / BN; }
    const int gn = n0 + n, gk = k0 + k;
    rb[i] = (gn < N && gk < K) ? (TB ? Bm[(size_t)gn * ldb + gk] : Bm[(size_t)gk * ldb + gn]) : 0.f;
  }
}

template <bool TA, bool TB>
__device__ __forceinline__ void store_tiles(float (*As)[BM], float (*Bs)[BN], const float ra[4], const float rb[4]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = tid + i * NT;
    int m, k;
    if (TA) { m = e % BM; k = e / BM; } else { k = e % BK; m = e / BK; }
    As[k][m] = ra[i];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = tid + i * NT;
    int n, k;
    if (TB) { k = e % BK; n = e / BK; } else { n = e % BN; k = e / BN; }
    Bs[k][n] = rb[i];
  }
}

// blockIdx.z = split index; split s covers K range [s*kchunk, (s+1)*kchunk).
// With gridDim.z > 1 the raw partial tile goes to C + s*M*ldc (EPI_NONE semantics).
template <bool TA, bool TB>
__global__ void __launch_bounds__(NT) gemm_f32_kernel(const float* __restrict__ A, int lda,
                                                      const float* __restrict__ Bm, int ldb, float* C, int ldc,
                                                      int M, int N, int K, int kchunk, int epi,
                                                      const float* __restrict__ bias, const float* resid) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int tr = threadIdx.x / (BN / TN), tc = threadIdx.x % (BN / TN);
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  float ra[4], rb[4];
  load_tiles<TA, TB>(A, lda, Bm, ldb, M, N, kend, m0, n0, kbeg, ra, rb);
  store_tiles<TA, TB>(As[0], Bs[0], ra, rb);
  __syncthreads();
  int buf = 0;
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) load_tiles<TA, TB>(A, lda, Bm, ldb, M, N, kend, m0, n0, k0 + BK, ra, rb);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[TM], b[TN];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tr * TM]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][tr * TM + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tc * TN]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tc * TN + 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w; a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w; b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store_tiles<TA, TB>(As[buf ^ 1], Bs[buf ^ 1], ra, rb);
      __syncthreads();
      buf ^= 1;
    }
  }

  float* Cz = C + (size_t)blockIdx.z * M * ldc;
  const bool split = gridDim.z > 1;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + tr * TM + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tc * TN + j;
      if (gn >= N) continue;
      float v = acc[i][j];
      const size_t o = (size_t)gm * ldc + gn;
      if (split || epi == EPI_NONE) {
        Cz[o] = v;
      } else if (epi == EPI_BIAS) {
        C[o] = v + bias[gn];
      } else if (epi == EPI_BIAS_GELU) {
        C[o] = gelu_erf(v + bias[gn]);
      } else {  // EPI_BIAS_RESID
        C[o] = resid[o] + (v + bias[gn]);
      }
    }
  }
}

}  // namespace

cudaError_t launch_gemm_f32_ex(bool ta, bool tb, const float* A, int lda, const float* Bm, int ldb, float* C,
                               int ldc, int M, int N, int K, int splits, int epi, const float* bias,
                               const float* resid, cudaStream_t st) {
  if (splits < 1) splits = 1;
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  splits = (K + kchunk - 1) / kchunk;
  if (splits < 1) splits = 1;
  dim3 grid(cdiv(N, BN), cdiv(M, BM), splits);
  if (!ta && !tb)
    gemm_f32_kernel<false, false><<<grid, NT, 0, st>>>(A, lda, Bm, ldb, C, ldc, M, N, K, kchunk, epi, bias, resid);
  else if (!ta && tb)
    gemm_f32_kernel<false, true><<<grid, NT, 0, st>>>(A, lda, Bm, ldb, C, ldc, M, N, K, kchunk, epi, bias, resid);
  else if (ta && !tb)
    gemm_f32_kernel<true, false><<<grid, NT, 0, st>>>(A, lda, Bm, ldb, C, ldc, M, N, K, kchunk, epi, bias, resid);
  else
    gemm_f32_kernel<true, true><<<grid, NT, 0, st>>>(A, lda, Bm, ldb, C, ldc, M, N, K, kchunk, epi, bias, resid);
  return cudaGetLastError();
}

cudaError_t launch_gemm_f32(const float* A, int lda, const float* Bm, int ldb, float* C, int ldc, int M, int N,
                            int K, int epi, const float* bias, const float* resid, cudaStream_t st) {
  return launch_gemm_f32_ex(false, false, A, lda, Bm, ldb, C, ldc, M, N, K, 1, epi, bias, resid, st);
}

}  // namespace inpaint

namespace inpaint {
// Number of K splits launch_gemm_f32_ex actually uses for a requested count.
int gemm_split_count(int K, int splits) {
  if (splits < 1) splits = 1;
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  const int s = (K + kchunk - 1) / kchunk;
  return s < 1 ? 1 : s;
}
}  // namespace inpaint
