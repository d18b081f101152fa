// SIMT register-tiled matrix-multiply engine shared by the H-apply and the
// dense kernels.  One CTA of 256 threads accumulates a BM x BN tile of
// op(A) op(B) in registers (TM x TN per thread), staging BK-deep slabs of A and
// B through shared memory with a register prefetch of the next slab.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

template <typename T>
struct TileCfg;
template <>
struct TileCfg<float> {
  static constexpr int BM = 64, BN = 128, BK = 16, TM = 4, TN = 8;
};
template <>
struct TileCfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};

constexpr int kTileThreads = 256;

template <typename T>
struct TileSmem {
  static constexpr int BM = TileCfg<T>::BM, BN = TileCfg<T>::BN, BK = TileCfg<T>::BK;
  static constexpr int LDA = BM + 4, LDB = BN + 4;
  alignas(16) T a[BK * LDA];
  alignas(16) T b[BK * LDB];
};

// Accumulate acc += op(A)[0:M, 0:K] * op(B)[0:K, 0:N] for one CTA tile.
//   A_KC (A "k-contiguous"): element (m, k) at A[m*lda + k]; else at A[k*lda + m].
//   B_KC (B "k-contiguous"): element (k, n) at B[n*ldb + k]; else at B[k*ldb + n].
// M <= BM and N <= BN are the valid extents of this tile; out-of-range
// elements are read as zero.  All 256 threads must call this.
template <typename T, bool A_KC, bool B_KC>
__device__ __forceinline__ void tile_mma(T (&acc)[TileCfg<T>::TM][TileCfg<T>::TN], const T* __restrict__ A,
                                         int64_t lda, int M, const T* __restrict__ B, int64_t ldb, int N, int K,
                                         TileSmem<T>& sm) {
  constexpr int BM = TileCfg<T>::BM, BN = TileCfg<T>::BN, BK = TileCfg<T>::BK;
  constexpr int TM = TileCfg<T>::TM, TN = TileCfg<T>::TN;
  constexpr int LDA = TileSmem<T>::LDA, LDB = TileSmem<T>::LDB;
  constexpr int NA = BM * BK / kTileThreads;  // A elements per thread per slab
  constexpr int NB = BN * BK / kTileThreads;
  const int tid = threadIdx.x;
  const int ty = tid / (BN / TN), tx = tid % (BN / TN);
  T ra[NA], rb[NB];

  auto load = [&](int k0) {
#pragma unroll
    for (int i = 0; i < NA; i++) {
      const int e = tid + i * kTileThreads;
      int mm, kk;
      if (A_KC) {
        mm = e / BK;
        kk = e % BK;
      } else {
        kk = e / BM;
        mm = e % BM;
      }
      const int k = k0 + kk;
      ra[i] = (mm < M && k < K) ? (A_KC ? A[(int64_t)mm * lda + k] : A[(int64_t)k * lda + mm]) : T(0);
    }
#pragma unroll
    for (int i = 0; i < NB; i++) {
      const int e = tid + i * kTileThreads;
      int nn, kk;
      if (B_KC) {
        nn = e / BK;
        kk = e % BK;
      } else {
        kk = e / BN;
        nn = e % BN;
      }
      const int k = k0 + kk;
      rb[i] = (nn < N && k < K) ? (B_KC ? B[(int64_t)nn * ldb + k] : B[(int64_t)k * ldb + nn]) : T(0);
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int i = 0; i < NA; i++) {
      const int e = tid + i * kTileThreads;
      const int mm = A_KC ? e / BK : e % BM;
      const int kk = A_KC ? e % BK : e / BM;
      sm.a[kk * LDA + mm] = ra[i];
    }
#pragma unroll
    for (int i = 0; i < NB; i++) {
      const int e = tid + i * kTileThreads;
      const int nn = B_KC ? e / BK : e % BN;
      const int kk = B_KC ? e % BK : e / BN;
      sm.b[kk * LDB + nn] = rb[i];
    }
  };

  if (K <= 0) return;
  load(0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    __syncthreads();  // previous slab fully consumed
    store();
    __syncthreads();
    if (k0 + BK < K) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
      // 16-byte shared loads; the thread's TN columns are two strips of TN/2
      // at tx*TN/2 and BN/2 + tx*TN/2 so that each quarter-warp reads one
      // contiguous 128-byte line (no bank conflicts)
      T a[TM], b[TN];
      constexpr int V = 16 / sizeof(T);  // elements per 16-byte vector
      using vec_t = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
#pragma unroll
      for (int i = 0; i < TM; i += V) {
        const vec_t v = *reinterpret_cast<const vec_t*>(&sm.a[kk * LDA + ty * TM + i]);
        const T* pv = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int u = 0; u < V; u++) a[i + u] = pv[u];
      }
#pragma unroll
      for (int h = 0; h < 2; h++)
#pragma unroll
        for (int j = 0; j < TN / 2; j += V) {
          const vec_t v = *reinterpret_cast<const vec_t*>(&sm.b[kk * LDB + h * (BN / 2) + tx * (TN / 2) + j]);
          const T* pv = reinterpret_cast<const T*>(&v);
#pragma unroll
          for (int u = 0; u < V; u++) b[h * (TN / 2) + j + u] = pv[u];
        }
#pragma unroll
      for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
}

template <typename T>
__device__ __forceinline__ void tile_zero(T (&acc)[TileCfg<T>::TM][TileCfg<T>::TN]) {
#pragma unroll
  for (int i = 0; i < TileCfg<T>::TM; i++)
#pragma unroll
    for (int j = 0; j < TileCfg<T>::TN; j++) acc[i][j] = T(0);
}

// Row/column of accumulator element (i, j) of this thread inside the tile.
template <typename T>
__device__ __forceinline__ int tile_row(int i) {
  return (threadIdx.x / (TileCfg<T>::BN / TileCfg<T>::TN)) * TileCfg<T>::TM + i;
}
template <typename T>
__device__ __forceinline__ int tile_col(int j) {
  constexpr int TN = TileCfg<T>::TN, BN = TileCfg<T>::BN;
  const int tx = threadIdx.x % (BN / TN);
  return (j < TN / 2 ? 0 : BN / 2) + tx * (TN / 2) + (j % (TN / 2));
}
