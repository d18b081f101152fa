// Dense products on the SIMT tile engine: tall-skinny rotations
// (N x K times K x n), Gram matrices A^T B with a long reduction (split over
// row chunks, summed in a fixed order in FP64), and the small FP64 products of
// the data-space algebra.
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "common.h"
#include "dense.h"
#include "tile.cuh"

namespace {

// The FP64 tile kernels ask for the largest shared-memory carveout: an SM
// that runs a persistent tensor-core kernel with a large shared-memory
// footprint (phase 2 of the H-apply) then also takes one of their CTAs beside
// it, instead of draining first to switch configurations.  Set once per
// kernel and device (a hint: a refusal is ignored).
template <typename Kern>
void prefer_max_shared(Kern kernel, std::atomic<uint32_t>& done, int device) {
  const uint32_t bit = 1u << (device & 31);
  if (done.load(std::memory_order_relaxed) & bit) return;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
      cudaSuccess)
    cudaGetLastError();
  done.fetch_or(bit);
}
#define FKF_MAXSHARED(kern)                          \
  do {                                               \
    static std::atomic<uint32_t> done_{0};           \
    prefer_max_shared(kern, done_, ctx->device);     \
  } while (0)

// C = alpha op(A) op(B) + beta C, all row-major.
template <typename T, bool A_KC, bool B_KC>
__global__ void __launch_bounds__(kTileThreads) k_gemm(int M, int N, int K, T alpha, const T* __restrict__ A,
                                                       int64_t lda, const T* __restrict__ B, int64_t ldb, T beta,
                                                       T* __restrict__ C, int64_t ldc) {
  __shared__ TileSmem<T> sm;
  constexpr int BM = TileCfg<T>::BM, BN = TileCfg<T>::BN;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int mv = min(BM, M - m0), nv = min(BN, N - n0);
  T acc[TileCfg<T>::TM][TileCfg<T>::TN];
  tile_zero<T>(acc);
  const T* Ap = A_KC ? A + (int64_t)m0 * lda : A + m0;
  const T* Bp = B_KC ? B + (int64_t)n0 * ldb : B + n0;
  tile_mma<T, A_KC, B_KC>(acc, Ap, lda, mv, Bp, ldb, nv, K, sm);
#pragma unroll
  for (int i = 0; i < TileCfg<T>::TM; i++) {
    const int r = tile_row<T>(i);
    if (r >= mv) continue;
    T* dst = C + (int64_t)(m0 + r) * ldc + n0;
#pragma unroll
    for (int j = 0; j < TileCfg<T>::TN; j++) {
      const int c = tile_col<T>(j);
      if (c < nv) dst[c] = beta == T(0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * dst[c];
    }
  }
}

// Symmetric result C = alpha op(A) op(B) + beta C (N x N) when op(A) op(B) is
// symmetric: only the tiles on and below the diagonal are computed (tile t of
// the lower triangle, row-major order), and each computed entry (i >= j) is
// written to (i, j) and, with MIRROR, to (j, i) as well (without it the upper
// triangle is left as it was).  With MIRROR, C must be symmetric on entry
// when beta is not zero.  Entries with i, j >= skip are left untouched (tiles
// entirely among them are not computed).
template <typename T, bool A_KC, bool B_KC, bool MIRROR>
__global__ void __launch_bounds__(kTileThreads) k_gemm_sym(int N, int K, T alpha, const T* __restrict__ A,
                                                           int64_t lda, const T* __restrict__ B, int64_t ldb,
                                                           T beta, T* __restrict__ C, int64_t ldc, int skip) {
  static_assert(TileCfg<T>::BM == TileCfg<T>::BN, "square tiles");
  __shared__ TileSmem<T> sm;
  constexpr int BM = TileCfg<T>::BM;
  const int t = blockIdx.x;
  int bi = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((bi + 1) * (bi + 2) / 2 <= t) bi++;
  while (bi * (bi + 1) / 2 > t) bi--;
  const int bj = t - bi * (bi + 1) / 2;
  const int m0 = bi * BM, n0 = bj * BM;
  if (n0 >= skip) return;  // every entry has i >= j >= skip (uniform over the CTA)
  const int mv = min(BM, N - m0), nv = min(BM, N - n0);
  T acc[TileCfg<T>::TM][TileCfg<T>::TN];
  tile_zero<T>(acc);
  const T* Ap = A_KC ? A + (int64_t)m0 * lda : A + m0;
  const T* Bp = B_KC ? B + (int64_t)n0 * ldb : B + n0;
  tile_mma<T, A_KC, B_KC>(acc, Ap, lda, mv, Bp, ldb, nv, K, sm);
#pragma unroll
  for (int i = 0; i < TileCfg<T>::TM; i++) {
    const int r = tile_row<T>(i);
    if (r >= mv) continue;
#pragma unroll
    for (int j = 0; j < TileCfg<T>::TN; j++) {
      const int c = tile_col<T>(j);
      const int gi = m0 + r, gj = n0 + c;
      if (c >= nv || gi < gj || gj >= skip) continue;
      T* dst = C + (int64_t)gi * ldc + gj;
      const T v = beta == T(0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *dst;
      *dst = v;
      if (MIRROR && gi != gj) C[(int64_t)gj * ldc + gi] = v;
    }
  }
}

// Matrix-vector form of the FP64 GEMM (N = 1): y_i = sum_k op(A)(i, k) x_k,
// C[i] = alpha y_i + beta C[i].  Rows of A (not transposed): one warp per
// output, lanes over k, shuffle reduction; columns (transposed): a CTA per 32
// outputs, lanes over outputs (coalesced), its warps splitting k.
constexpr int kGemvTThreads = 1024;  // CTA of the transposed GEMV
__global__ void k_gemv_f64(int M, int K, bool ta, double alpha, const double* __restrict__ A, int64_t lda,
                           const double* __restrict__ x, int64_t incx, double beta, double* __restrict__ C,
                           int64_t ldc) {
  if (!ta) {
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= M) return;
    const double* a = A + (int64_t)i * lda;
    double s = 0.0;
    for (int k = lane; k < K; k += 32) s += a[k] * x[(int64_t)k * incx];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) C[(int64_t)i * ldc] = beta == 0.0 ? alpha * s : alpha * s + beta * C[(int64_t)i * ldc];
  } else {
    // 32 outputs per CTA of kGemvTThreads (lanes over outputs: coalesced
    // rows of A); warp w sums k = w, w + nw, ...; the warps' partial sums of an
    // output are added in warp order (deterministic)
    __shared__ double part[kGemvTThreads / 32][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (i < M)
      for (int k = w; k < K; k += nw) s += A[(int64_t)k * lda + i] * x[(int64_t)k * incx];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && i < M) {
      double t = 0.0;
      for (int q = 0; q < nw; q++) t += part[q][lane];
      C[(int64_t)i * ldc] = beta == 0.0 ? alpha * t : alpha * t + beta * C[(int64_t)i * ldc];
    }
  }
}

// Partial Gram: part[z] = A[rows z]^T B[rows z] (A: K x M, B: K x N row-major).
template <typename T>
__global__ void __launch_bounds__(kTileThreads) k_gram_part(int M, int N, int64_t K, int64_t chunk,
                                                            const T* __restrict__ A, int64_t lda,
                                                            const T* __restrict__ B, int64_t ldb,
                                                            T* __restrict__ part) {
  __shared__ TileSmem<T> sm;
  constexpr int BM = TileCfg<T>::BM, BN = TileCfg<T>::BN;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int mv = min(BM, M - m0), nv = min(BN, N - n0);
  const int64_t k0 = (int64_t)blockIdx.z * chunk;
  const int kv = (int)min(chunk, K - k0);
  T acc[TileCfg<T>::TM][TileCfg<T>::TN];
  tile_zero<T>(acc);
  tile_mma<T, false, false>(acc, A + k0 * lda + m0, lda, mv, B + k0 * ldb + n0, ldb, nv, kv, sm);
  T* P = part + (int64_t)blockIdx.z * M * N;
#pragma unroll
  for (int i = 0; i < TileCfg<T>::TM; i++) {
    const int r = tile_row<T>(i);
    if (r >= mv) continue;
#pragma unroll
    for (int j = 0; j < TileCfg<T>::TN; j++) {
      const int c = tile_col<T>(j);
      if (c < nv) P[(int64_t)(m0 + r) * N + n0 + c] = acc[i][j];
    }
  }
}

template <typename T>
__global__ void k_gram_reduce(int M, int N, int nz, const T* __restrict__ part, double* __restrict__ C,
                              int64_t ldc) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int z = 0; z < nz; z++) s += (double)part[(int64_t)z * total + e];
    C[(e / N) * ldc + e % N] = s;
  }
}

template <typename T>
fkf_status gemm_impl(fkf_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, T alpha, const T* A,
                     int64_t lda, const T* B, int64_t ldb, T beta, T* C, int64_t ldc) {
  if (M <= 0 || N <= 0) return FKF_OK;
  constexpr int BM = TileCfg<T>::BM, BN = TileCfg<T>::BN;
  if (cdiv(M, BM) > 65535 * 1024LL)
    return set_err(ctx, FKF_EINVAL, "gemm: M too large");
  dim3 grid((unsigned)cdiv(N, BN), (unsigned)cdiv(M, BM));
  // op(A)(m,k): ta=false -> A[m*lda+k] (k-contiguous); ta=true -> A[k*lda+m]
  // op(B)(k,n): tb=false -> B[k*ldb+n]; tb=true -> B[n*ldb+k] (k-contiguous)
  constexpr bool f64 = std::is_same<T, double>::value;
  if (!ta && !tb) {
    if (f64) FKF_MAXSHARED((k_gemm<T, true, false>));
    k_gemm<T, true, false><<<grid, kTileThreads, 0, ctx->stream>>>((int)M, (int)N, (int)K, alpha, A, lda, B, ldb, beta, C, ldc);
  } else if (!ta && tb) {
    if (f64) FKF_MAXSHARED((k_gemm<T, true, true>));
    k_gemm<T, true, true><<<grid, kTileThreads, 0, ctx->stream>>>((int)M, (int)N, (int)K, alpha, A, lda, B, ldb, beta, C, ldc);
  } else if (ta && !tb) {
    if (f64) FKF_MAXSHARED((k_gemm<T, false, false>));
    k_gemm<T, false, false><<<grid, kTileThreads, 0, ctx->stream>>>((int)M, (int)N, (int)K, alpha, A, lda, B, ldb, beta, C, ldc);
  } else {
    if (f64) FKF_MAXSHARED((k_gemm<T, false, true>));
    k_gemm<T, false, true><<<grid, kTileThreads, 0, ctx->stream>>>((int)M, (int)N, (int)K, alpha, A, lda, B, ldb, beta, C, ldc);
  }
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}

}  // namespace

fkf_status gemm_f64(fkf_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                    int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
  if (K <= 0) {
    // C = beta C
    return scale_f64(ctx, M, N, beta, C, ldc);
  }
  if (N == 1) {
    // op(B)(k, 0) = B[k * ldb] (tb = false) or B[k] (tb = true)
    const int64_t incx = tb ? 1 : ldb;
    const unsigned grid = ta ? (unsigned)cdiv(M, 32) : (unsigned)cdiv(M * 32, 256);
    k_gemv_f64<<<grid, ta ? kGemvTThreads : 256, 0, ctx->stream>>>((int)M, (int)K, ta, alpha, A, lda, B, incx,
                                                                  beta, C, ldc);
    FKF_LAUNCHED(ctx);
    return FKF_OK;
  }
  return gemm_impl<double>(ctx, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

fkf_status gemm_sym_f64(fkf_ctx* ctx, bool ta, bool tb, int64_t N, int64_t K, double alpha, const double* A,
                        int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                        bool lower_only, int64_t skip) {
  if (N <= 0) return FKF_OK;
  if (K <= 0) return scale_f64(ctx, N, N, beta, C, ldc);
  if (skip >= 0 && skip < N && !lower_only) return set_err(ctx, FKF_EINVAL, "gemm_sym_f64: skip needs lower_only");
  const int sk = (skip < 0 || skip >= N) ? (int)N : (int)skip;
  constexpr int BM = TileCfg<double>::BM;
  const int64_t nb = cdiv(N, BM);
  const unsigned grid = (unsigned)(nb * (nb + 1) / 2);
#define FKF_SYM_LAUNCH(AK, BK)                                                                                    \
  if (lower_only) {                                                                                                \
    FKF_MAXSHARED((k_gemm_sym<double, AK, BK, false>));                                                            \
    k_gemm_sym<double, AK, BK, false><<<grid, kTileThreads, 0, ctx->stream>>>((int)N, (int)K, alpha, A, lda, B, \
                                                                              ldb, beta, C, ldc, sk);           \
  } else {                                                                                                         \
    FKF_MAXSHARED((k_gemm_sym<double, AK, BK, true>));                                                             \
    k_gemm_sym<double, AK, BK, true><<<grid, kTileThreads, 0, ctx->stream>>>((int)N, (int)K, alpha, A, lda, B,  \
                                                                             ldb, beta, C, ldc, sk);            \
  }
  if (!ta && !tb) {
    FKF_SYM_LAUNCH(true, false)
  } else if (!ta && tb) {
    FKF_SYM_LAUNCH(true, true)
  } else if (ta && !tb) {
    FKF_SYM_LAUNCH(false, false)
  } else {
    FKF_SYM_LAUNCH(false, true)
  }
#undef FKF_SYM_LAUNCH
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}

fkf_status gemm_f32(fkf_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                    int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc) {
  if (K <= 0) return scale_f32(ctx, M, N, beta, C, ldc);
  return gemm_impl<float>(ctx, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

template <typename T>
fkf_status gram_impl(fkf_ctx* ctx, int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, const T* B,
                     int64_t ldb, double* C, int64_t ldc, DevBuf& ws) {
  if (M <= 0 || N <= 0) return FKF_OK;
  if (K <= 0) return scale_f64(ctx, M, N, 0.0, C, ldc);
  constexpr int BM = TileCfg<T>::BM, BN = TileCfg<T>::BN;
  const int64_t tiles = cdiv(M, BM) * cdiv(N, BN);
  // enough chunks to fill the GPU, each at least 512 rows
  int64_t nz = std::max<int64_t>(1, std::min<int64_t>(cdiv(4 * 152, tiles), cdiv(K, 512)));
  nz = std::min<int64_t>(nz, 1024);
  const int64_t chunk = cdiv(K, nz);
  nz = cdiv(K, chunk);
  const size_t need = (size_t)nz * M * N * sizeof(T);
  if (ws.bytes < need) FKF_TRY(dev_alloc(ctx, ws, need));
  dim3 grid((unsigned)cdiv(N, BN), (unsigned)cdiv(M, BM), (unsigned)nz);
  k_gram_part<T><<<grid, kTileThreads, 0, ctx->stream>>>((int)M, (int)N, K, chunk, A, lda, B, ldb, ws.as<T>());
  FKF_LAUNCHED(ctx);
  const int blocks = (int)std::min<int64_t>(cdiv(M * N, 256), 4096);
  k_gram_reduce<T><<<blocks, 256, 0, ctx->stream>>>((int)M, (int)N, (int)nz, ws.as<T>(), C, ldc);
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}

fkf_status gram_f64(fkf_ctx* ctx, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
                    int64_t ldb, double* C, int64_t ldc, DevBuf& ws) {
  return gram_impl<double>(ctx, M, N, K, A, lda, B, ldb, C, ldc, ws);
}
fkf_status gram_f32(fkf_ctx* ctx, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                    int64_t ldb, double* C, int64_t ldc, DevBuf& ws) {
  return gram_impl<float>(ctx, M, N, K, A, lda, B, ldb, C, ldc, ws);
}

namespace {
template <typename T>
__global__ void k_scale(int64_t M, int64_t N, T beta, T* C, int64_t ldc) {
  const int64_t total = M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    T* p = C + (e / N) * ldc + e % N;
    *p = beta == T(0) ? T(0) : beta * *p;
  }
}
}  // namespace

fkf_status scale_f64(fkf_ctx* ctx, int64_t M, int64_t N, double beta, double* C, int64_t ldc) {
  if (M <= 0 || N <= 0) return FKF_OK;
  k_scale<double><<<(int)std::min<int64_t>(cdiv(M * N, 256), 4096), 256, 0, ctx->stream>>>(M, N, beta, C, ldc);
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}
fkf_status scale_f32(fkf_ctx* ctx, int64_t M, int64_t N, float beta, float* C, int64_t ldc) {
  if (M <= 0 || N <= 0) return FKF_OK;
  k_scale<float><<<(int)std::min<int64_t>(cdiv(M * N, 256), 4096), 256, 0, ctx->stream>>>(M, N, beta, C, ldc);
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}
