// The fast random-walk Kalman filter step and the Sec. 3 uncertainty measures.
//
// State (cluster order): s_hat (N, FP64), alpha, D (r, FP64), W (N x r) and
// X = Gamma^-1 W (N x r), precision T.  W is stored right-aligned in a wide
// buffer so that [W G] (G = Gamma H_k^T) is one contiguous N x (r + m) block:
//     WG row i = [ ... | W(i, 0:r) | G(i, 0:m) ]   columns r_max - r ... r_max + m.
//
// One step (Sec. 2.4, Alg. extkalman with a linear H_k; Alg. lowrankaddition):
//   alpha' = alpha + 1                                    (predict, F = I)
//   G = Gamma_H H^T,  A = H G,  HW = H W                  (one H-apply, gathers)
//   S = alpha' A - HW D HW^T + R,  z = S^-1 (y - H s)     (Alg. kalmanconstantH)
//   s += alpha' G z - W (D (HW^T z))
//   GEP in data space: R^-1/2 A R^-1/2 = Q diag(lam) Q^T, C = R^-1/2 Q lam^-1/2,
//     U = G C satisfies U^T Gamma^-1 U = I and Gamma^-1 U Lam U^T Gamma^-1 =
//     H^T R^-1 H (Eq. geneigendecomposition restricted to its range).
//   Gamma^-1-orthonormalisation against W (Alg. lowrankaddition steps 1-2),
//     with W^T Gamma^-1 U = HW^T C =: P and the Gram of U - W P equal to
//     T = I - P^T P (no N-scale Gram needed); a rank-revealing pivoted
//     Cholesky T ~= Lp Lp^T gives the new directions (U - W P) Y,
//     Y = Lp (Lp^T Lp)^-1 (written Q_T Theta^-1/2 below, Lp^T as Theta^1/2 Q_T^T:
//     what an eigendecomposition T = Q_T Theta Q_T^T would give).
//   Merge (step 3-4): M = diag(Dbar, 0) + [P; Theta^1/2 Q_T^T] Lam [...]^T,
//     Dbar = D / (alpha' (alpha' - D))  (the sign-consistent form of the SMW
//     expansion of Sigma_pred^-1, as in Alg. extkalman); M = S Dhat S^T,
//     truncated at trunc_tol * max.
//   D' = alpha'^2 Dhat / (1 + alpha' Dhat)  (= alpha'(I + alpha'^-1 Dhat^-1)^-1
//     written without Dhat^-1), and the basis rotation
//     W' = [W G] [E_W; E_G],  X' = X E_W + H^T E_G           (one tall GEMM each)
//   with E_G = C Q_T Theta^-1/2 S_2 and E_W = S_1 - P Q_T Theta^-1/2 S_2.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "common.h"
#include "dense.h"

namespace {

template <typename T>
__global__ void k_densify(int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          const double* __restrict__ val, const int64_t* __restrict__ iperm, int64_t n,
                          T* __restrict__ Bt, int64_t ldb, int* __restrict__ flag) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  for (int64_t p = rowptr[j]; p < rowptr[j + 1]; p++) {
    const int64_t c = col[p];
    if (c < 0 || c >= n) {
      atomicOr(flag, 1);
      continue;
    }
    Bt[iperm[c] * ldb + j] += (T)val[p];
  }
}

// Column counts of H in cluster order (warp per row); flags column indices
// outside [0, n).
__global__ void k_csc_count(int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const int64_t* __restrict__ iperm, int64_t n, int* __restrict__ cnt,
                            int* __restrict__ flag) {
  const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (j >= m) return;
  for (int64_t p = rowptr[j] + lane; p < rowptr[j + 1]; p += 32) {
    const int64_t c = col[p];
    if (c >= 0 && c < n)
      atomicAdd(&cnt[iperm[c]], 1);
    else
      atomicOr(flag, 1);
  }
}

// Exclusive scan of n ints into n + 1 int64 (out[n] = total) in three
// passes over blocks of 1024: block sums, a scan of the block sums, and the
// block-local scans plus their offsets.
constexpr int kScanBlock = 1024;

// exclusive scan of v across the CTA (kScanBlock threads); *total = CTA sum
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = sh[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int64_t before = warp > 0 ? sh[warp - 1] : 0;
  *total = sh[31];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_sums(int64_t n, const int* __restrict__ cnt,
                                                          int64_t* __restrict__ bsum) {
  __shared__ int64_t sh[32];
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  int64_t tot;
  block_excl_scan(i < n ? cnt[i] : 0, sh, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// exclusive scan of the nb block sums in place; bsum[nb] = total (one CTA)
__global__ void __launch_bounds__(kScanBlock) k_scan_bsums(int64_t nb, int64_t* __restrict__ bsum) {
  __shared__ int64_t sh[32];
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += kScanBlock) {
    const int64_t i = b0 + threadIdx.x;
    const int64_t v = i < nb ? bsum[i] : 0;
    int64_t tot;
    const int64_t e = block_excl_scan(v, sh, &tot);
    if (i < nb) bsum[i] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_out(int64_t n, const int* __restrict__ cnt,
                                                         const int64_t* __restrict__ bsum, int64_t nb,
                                                         int64_t* __restrict__ out) {
  __shared__ int64_t sh[32];
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  int64_t tot;
  const int64_t e = block_excl_scan(i < n ? cnt[i] : 0, sh, &tot);
  if (i < n) out[i] = bsum[blockIdx.x] + e;
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = bsum[nb];
}

static fkf_status scan_counts(fkf_ctx* ctx, int64_t n, const int* cnt, int64_t* out, DevBuf& ws) {
  const int64_t nb = std::max<int64_t>(1, cdiv(n, kScanBlock));
  if (ws.bytes < (size_t)(nb + 1) * 8) FKF_TRY(dev_alloc(ctx, ws, (size_t)(nb + 1) * 8));
  k_scan_sums<<<(unsigned)nb, kScanBlock, 0, ctx->stream>>>(n, cnt, ws.as<int64_t>());
  FKF_LAUNCHED(ctx);
  k_scan_bsums<<<1, kScanBlock, 0, ctx->stream>>>(nb, ws.as<int64_t>());
  FKF_LAUNCHED(ctx);
  k_scan_out<<<(unsigned)nb, kScanBlock, 0, ctx->stream>>>(n, cnt, ws.as<int64_t>(), nb, out);
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}

// Scatter the entries into their columns (warp per row; the order inside a
// column is fixed afterwards by k_csc_sort).
__global__ void k_csc_fill(int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const int64_t* __restrict__ iperm, int64_t n,
                           const int64_t* __restrict__ colptr, int* __restrict__ cursor, int* __restrict__ crow,
                           double* __restrict__ cval) {
  const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (j >= m) return;
  for (int64_t p = rowptr[j] + lane; p < rowptr[j + 1]; p += 32) {
    const int64_t c = col[p];
    if (c < 0 || c >= n) continue;
    const int64_t ci = iperm[c];
    const int64_t pos = colptr[ci] + atomicAdd(&cursor[ci], 1);
    crow[pos] = j;
    cval[pos] = val[p];
  }
}

// sort each column's entries by row (deterministic summation order); merge
// duplicates is not needed: sums over duplicates are order-fixed after sorting
__global__ void k_csc_sort(int64_t n, const int64_t* __restrict__ colptr, int* __restrict__ crow,
                           double* __restrict__ cval) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t a = colptr[i], b = colptr[i + 1];
  for (int64_t p = a + 1; p < b; p++) {
    const int r = crow[p];
    const double v = cval[p];
    int64_t q = p - 1;
    while (q >= a && (crow[q] > r || (crow[q] == r && cval[q] > v))) {
      crow[q + 1] = crow[q];
      cval[q + 1] = cval[q];
      q--;
    }
    crow[q + 1] = r;
    cval[q + 1] = v;
  }
}

// *diff |= (a[i] != b[i]) over n 32-bit words (byte comparison of two arrays)
__global__ void k_words_differ(int64_t n, const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                               int* __restrict__ diff) {
  bool d = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d |= a[i] != b[i];
  if (__any_sync(0xffffffffu, d) && (threadIdx.x & 31) == 0) atomicOr(diff, 1);
}

// Bt (n x m, cluster order) += H^T from the sorted CSC form: thread per
// column of H = row of Bt; duplicates are summed in the sorted order.
template <typename T>
__global__ void k_densify_csc(int64_t n, const int64_t* __restrict__ colptr, const int* __restrict__ crow,
                              const double* __restrict__ cval, T* __restrict__ Bt, int64_t ldb,
                              unsigned* __restrict__ cmax) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  T* row = Bt + i * ldb;
  for (int64_t p = colptr[i]; p < colptr[i + 1]; p++) row[crow[p]] += (T)cval[p];
  // column maxima of |Bt| (ordered bits of non-negative floats), from the
  // final values (repeated entries summed); zero columns keep 0
  if (cmax)
    for (int64_t p = colptr[i]; p < colptr[i + 1]; p++)
      atomicMax(&cmax[crow[p]], __float_as_uint(fabsf((float)row[crow[p]])));
}

// The column maxima k_densify_csc<float> would record, without writing H^T:
// per row of H^T, each column's entries summed in FP32 in their order.
__global__ void k_csc_colmax(int64_t n, const int64_t* __restrict__ colptr, const int* __restrict__ crow,
                             const double* __restrict__ cval, unsigned* __restrict__ cmax) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t p1 = colptr[i + 1];
  for (int64_t p = colptr[i]; p < p1;) {
    const int c = crow[p];
    float v = 0.f;
    for (; p < p1 && crow[p] == c; p++) v += (float)cval[p];
    atomicMax(&cmax[c], __float_as_uint(fabsf(v)));
  }
}

// out (m x ncols, FP64) = H * src[:, 0:ncols]  (src rows in cluster order)
// out[j, c] = sum_p val[p] * src[iperm[col[p]], c] for the rows j of a CSR
// matrix (c < ncols).  One CTA per (row, column block); the row's (index,
// value) pairs are staged in shared memory in chunks, and each thread keeps V
// consecutive columns (one 16-byte load per nonzero when V > 1).  The loads of
// four nonzeros are issued before their products, which are summed in p order.
constexpr int kGatherThreads = 256;
constexpr int kGatherChunk = 1024;

template <typename T, int V>
__device__ __forceinline__ void load_cols(const T* p, T (&o)[V]) {
  if constexpr (V == 1) {
    o[0] = *p;
  } else if constexpr (sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    o[0] = x.x, o[1] = x.y, o[2] = x.z, o[3] = x.w;
  } else {
    const double2 x = *reinterpret_cast<const double2*>(p);
    o[0] = x.x, o[1] = x.y;
  }
}

template <typename T, int V>
__global__ void __launch_bounds__(kGatherThreads, 4)
    k_csr_gather(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                 const double* __restrict__ val, const int64_t* __restrict__ iperm, int64_t n,
                 const T* __restrict__ src, int64_t lds, int ncols, double* __restrict__ out, int64_t ldo) {
  __shared__ int s_idx[kGatherChunk];
  __shared__ T s_val[kGatherChunk];
  const int j = blockIdx.x;
  const int c0 = (blockIdx.y * kGatherThreads + threadIdx.x) * V;
  const int64_t a = rowptr[j], b = rowptr[j + 1];
  T acc[V];
#pragma unroll
  for (int u = 0; u < V; u++) acc[u] = 0;
  const bool full = c0 + V <= ncols;
  for (int64_t base = a; base < b; base += kGatherChunk) {
    const int cnt = (int)(b - base < kGatherChunk ? b - base : kGatherChunk);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += kGatherThreads) {
      const int64_t cc = col[base + i];
      const bool ok = cc >= 0 && cc < n;
      s_idx[i] = ok ? (int)iperm[cc] : 0;
      s_val[i] = ok ? (T)val[base + i] : (T)0;
    }
    __syncthreads();
    if (full) {
      const T* s0 = src + c0;
      int i = 0;
      for (; i + 4 <= cnt; i += 4) {
        T x[4][V];
#pragma unroll
        for (int q = 0; q < 4; q++) load_cols<T, V>(s0 + (int64_t)s_idx[i + q] * lds, x[q]);
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const T v = s_val[i + q];
#pragma unroll
          for (int u = 0; u < V; u++) acc[u] += v * x[q][u];
        }
      }
      for (; i < cnt; i++) {
        T x[V];
        load_cols<T, V>(s0 + (int64_t)s_idx[i] * lds, x);
        const T v = s_val[i];
#pragma unroll
        for (int u = 0; u < V; u++) acc[u] += v * x[u];
      }
    } else if (c0 < ncols) {
      for (int i = 0; i < cnt; i++) {
        const T* xr = src + (int64_t)s_idx[i] * lds;
        const T v = s_val[i];
#pragma unroll
        for (int u = 0; u < V; u++)
          if (c0 + u < ncols) acc[u] += v * xr[c0 + u];
      }
    }
  }
#pragma unroll
  for (int u = 0; u < V; u++)
    if (c0 + u < ncols) out[(int64_t)j * ldo + c0 + u] = (double)acc[u];
}

// Launch of k_csr_gather: 16-byte column vectors when src and lds allow them.
template <typename T>
static void csr_gather(int m, const int64_t* rowptr, const int32_t* col, const double* val, const int64_t* iperm,
                       int64_t n, const T* src, int64_t lds, int ncols, double* out, int64_t ldo, cudaStream_t st) {
  constexpr int V = 16 / sizeof(T);
  if (m <= 0 || ncols <= 0) return;
  const bool vec = (reinterpret_cast<uintptr_t>(src) % 16 == 0) && (lds % V == 0);
  if (vec) {
    const dim3 grid((unsigned)m, (unsigned)cdiv(ncols, kGatherThreads * V));
    k_csr_gather<T, V><<<grid, kGatherThreads, 0, st>>>(rowptr, col, val, iperm, n, src, lds, ncols, out, ldo);
  } else {
    const dim3 grid((unsigned)m, (unsigned)cdiv(ncols, kGatherThreads));
    k_csr_gather<T, 1><<<grid, kGatherThreads, 0, st>>>(rowptr, col, val, iperm, n, src, lds, ncols, out, ldo);
  }
}

// nu = y - H s (warp per row)
__global__ void k_innovation(int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const int64_t* __restrict__ iperm, int64_t n,
                             const double* __restrict__ s, const double* __restrict__ y, double* __restrict__ nu) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= m) return;
  double acc = 0;
  for (int64_t p = rowptr[w] + lane; p < rowptr[w + 1]; p += 32) {
    const int64_t c = col[p];
    if (c >= 0 && c < n) acc += val[p] * s[iperm[c]];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) nu[w] = y[w] - acc;
}

// Extended filter with the Box-Cox map (Sec. 4.2, Eq. nonlinear, Alg.
// extkalman): the state x is the transformed field, the measurement map is
// h(x) = H s(x) with s(x) = ((x + a)/a)^a.  At the predicted mean (= the
// previous posterior mean, F = I) this kernel forms the innovation
// nu = y - H s(x) and replaces H's values in place by those of the Jacobian
// H_k = H diag(s'(x)), s'(x) = ((x + a)/a)^(a - 1).  Warp per row; each
// warp reads its row's values before it rewrites them.
__global__ void k_boxcox_linearize(int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                   double* __restrict__ val, const int64_t* __restrict__ iperm, int64_t n,
                                   const double* __restrict__ x, double a, const double* __restrict__ y,
                                   double* __restrict__ nu) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= m) return;
  double acc = 0;
  for (int64_t p = rowptr[w] + lane; p < rowptr[w + 1]; p += 32) {
    const int64_t c = col[p];
    if (c >= 0 && c < n) {
      const double b = (x[iperm[c]] + a) / a;
      const double sp = pow(b, a - 1.0);  // s'(x)
      acc += val[p] * (sp * b);            // s(x) = b^a = b^(a-1) b
      val[p] *= sp;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) nu[w] = y[w] - acc;
}

// As = (A + A^T)/2, At = diag(rs) As diag(rs); S = alpha' As + diag(R)
__global__ void k_sym(int m, const double* __restrict__ A, int64_t lda, const double* __restrict__ rs,
                      const double* __restrict__ rdiag, double alpha1, double* __restrict__ As,
                      double* __restrict__ At, double* __restrict__ S, int64_t lds) {
  const int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    const double v = 0.5 * (A[(int64_t)i * lda + j] + A[(int64_t)j * lda + i]);
    As[e] = v;
    At[e] = v * rs[i] * rs[j];
    S[(int64_t)i * lds + j] = alpha1 * v + (i == j ? rdiag[i] : 0.0);
  }
}

// HWD = HW * diag(D)
__global__ void k_scale_cols(int m, int r, const double* __restrict__ HW, int64_t ld, const double* __restrict__ D,
                             double* __restrict__ out) {
  const int64_t total = (int64_t)m * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / r), j = (int)(e % r);
    out[e] = HW[(int64_t)i * ld + j] * D[j];
  }
}

// NLL = 1/2 (nu^T z + log det S + m log 2 pi) with S's Cholesky factor on the diagonal
__global__ void k_nll(int m, const double* __restrict__ nu, const double* __restrict__ z,
                      const double* __restrict__ L, int64_t ldl, double* __restrict__ out) {
  __shared__ double sh[2][32];
  double a = 0, b = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    a += nu[i] * z[i];
    b += log(L[(int64_t)i * ldl + i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = a;
    sh[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0, sb = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      sa += sh[0][w];
      sb += sh[1][w];
    }
    out[0] = 0.5 * (sa + 2.0 * sb + m * log(2.0 * 3.14159265358979323846));
  }
}

// v = [-D .* uz ; alpha' z] cast to T (uz = HW^T z, r entries)
template <typename T>
__global__ void k_mean_coef(int r, int m, const double* __restrict__ D, const double* __restrict__ uz,
                            const double* __restrict__ z, double alpha1, T* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < r) v[i] = (T)(D ? -D[i] * uz[i] : -uz[i]);  // D == nullptr: uz already weighted
  else if (i < r + m) v[i] = (T)(alpha1 * z[i - r]);
}

// s_out = s_in + WG[:, 0:K] v   (warp per row)
template <typename T>
__global__ void k_gemv_add(int64_t n, int K, const T* __restrict__ A, int64_t lda, const T* __restrict__ v,
                           const double* __restrict__ s_in, double* __restrict__ s_out) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const T* row = A + w * lda;
  T acc = 0;
  for (int k = lane; k < K; k += 32) acc += row[k] * v[k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) s_out[w] = s_in[w] + (double)acc;
}

// C[i, q] = rs[i] * Vt[(m-1-q), i] / sqrt(a[m-1-q]);  lam[q] = a[m-1-q]
__global__ void k_build_C(int m, int mlam, const double* __restrict__ Vt, const double* __restrict__ a,
                          const double* __restrict__ rs, double* __restrict__ C, double* __restrict__ lam) {
  const int64_t total = (int64_t)m * mlam;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / mlam), q = (int)(e % mlam);
    const int src = m - 1 - q;
    C[e] = rs[i] * Vt[(int64_t)src * m + i] / sqrt(a[src]);
    if (i == 0) lam[q] = a[src];
  }
}

// out[p, :] = Vt[n-1-p, :] * f(w[n-1-p]) for p < cnt; mode 0: sqrt(w), 1: 1/sqrt(w), 2: 1
__global__ void k_top_rows(int n, int cnt, const double* __restrict__ Vt, const double* __restrict__ w, int mode,
                           double* __restrict__ out, int64_t ldo, int nv = -1) {
  // nv: eigenpairs held (rows of Vt, entries of w), the largest last; all n by default
  const int top = (nv < 0 ? n : nv) - 1;
  const int64_t total = (int64_t)cnt * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / n), j = (int)(e % n);
    const int src = top - p;
    const double f = mode == 0 ? sqrt(w[src]) : (mode == 1 ? 1.0 / sqrt(w[src]) : 1.0);
    out[(int64_t)p * ldo + j] = Vt[(int64_t)src * n + j] * f;
  }
}

// A[i, :] *= d[i] * d[i] (sq) or d[i]
__global__ void k_scale_rows(int rows, int cols, double* __restrict__ A, int64_t lda, const double* __restrict__ d,
                             int sq) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols);
    A[(int64_t)i * lda + e % cols] *= sq ? d[i] * d[i] : d[i];
  }
}

__global__ void k_identity(int n, double* __restrict__ out, int64_t ldo) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    out[(e / n) * ldo + e % n] = (e / n == e % n) ? 1.0 : 0.0;
}

__global__ void k_add_identity(int n, double* __restrict__ A, int64_t lda, double s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[(int64_t)i * lda + i] += s;
}

// ZL[i, q] = Z[i, q] * sqrt(lam[q]) (rows of Z from P (first r) then Po)
__global__ void k_stack_scale(int r, int mp, int mlam, const double* __restrict__ P, const double* __restrict__ Po,
                              const double* __restrict__ lam, double* __restrict__ ZL) {
  const int64_t total = (int64_t)(r + mp) * mlam;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / mlam), q = (int)(e % mlam);
    const double z = i < r ? P[(int64_t)i * mlam + q] : Po[(int64_t)(i - r) * mlam + q];
    ZL[e] = z * sqrt(lam[q]);
  }
}

// M[j, j] += D[j] / (alpha' (alpha' - D[j])) for j < r
__global__ void k_add_dbar(int r, const double* __restrict__ D, double alpha1, double* __restrict__ M, int64_t ldm) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < r) M[(int64_t)j * ldm + j] += D[j] / (alpha1 * (alpha1 - D[j]));
}

// D'[q] = alpha'^2 th / (1 + alpha' th), th = w[n-1-q]
__global__ void k_new_D(int n, int rnew, const double* __restrict__ w, double alpha1, double* __restrict__ Dn) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < rnew) {
    const double th = w[n - 1 - q];
    Dn[q] = alpha1 * alpha1 * th / (1.0 + alpha1 * th);
  }
}

// E_W[i, q] = Sk[q, i] for i < r (transpose copy)
__global__ void k_transpose(int rows, int cols, const double* __restrict__ src, int64_t lds, double* __restrict__ dst,
                            int64_t ldd) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols), q = (int)(e % cols);
    dst[(int64_t)i * ldd + q] = src[(int64_t)q * lds + i];
  }
}

// C = a*A + b*B (+ d on the diagonal), n x n; C may alias A or B (elementwise)
__global__ void k_lincomb(int n, double a, const double* A, double b, const double* B, double d, double* C) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    C[e] = a * A[e] + (B ? b * B[e] : 0.0) + ((e / n == e % n) ? d : 0.0);
}

// Rows m .. m+r-1 of the augmented matrix [[S, K], [K^T, E]] (ld lda):
// [K^T | E] with K^T = (alpha' HW - HW D)^T (HW: m x r, ld ldh; HWD: m x r,
// ld r) and E = alpha' I - D (D = diag(d) if d, else the full weight Df).
__global__ void k_aug_rows(int m, int r, const double* __restrict__ HW, int64_t ldh, const double* __restrict__ HWD,
                           const double* __restrict__ d, const double* __restrict__ Df, double alpha1,
                           double* __restrict__ out, int64_t lda) {
  const int64_t total = lda * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / lda), j = (int)(e % lda);
    double v;
    if (j < m) {
      v = alpha1 * HW[(int64_t)j * ldh + i] - HWD[(int64_t)j * r + i];
    } else {
      const int q = j - m;
      v = d ? (i == q ? alpha1 - d[i] : 0.0) : (i == q ? alpha1 : 0.0) - Df[(int64_t)i * r + q];
    }
    out[(int64_t)i * lda + j] = v;
  }
}

// C (n x n) = a A + d I for a symmetric A given by its lower triangle
// (leading dimension lda); C comes out exactly symmetric
__global__ void k_lincomb_ld(int n, double a, const double* __restrict__ A, int64_t lda, double d,
                             double* __restrict__ C) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    C[e] = a * A[(int64_t)max(i, j) * lda + min(i, j)] + (i == j ? d : 0.0);
  }
}


// M[i, j] += B[i, j] + (i == j ? c : 0) for the leading r x r block of M (ld ldm)
__global__ void k_add_block(int r, const double* __restrict__ B, double c, double* __restrict__ M, int64_t ldm) {
  const int64_t total = (int64_t)r * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / r), j = (int)(e % r);
    M[(int64_t)i * ldm + j] += B[e] + (i == j ? c : 0.0);
  }
}

// out = d .* x (n)
__global__ void k_vmul(int n, const double* __restrict__ d, const double* __restrict__ x, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = d[i] * x[i];
}


// out = ||A||_F over n entries (single CTA)
// Frobenius norms in two passes with a fixed summation order: block b sums
// the squares of its contiguous range of A (optionally scaled as
// rs[i] A[i, j] rs[j] for an m x m matrix) into part[b]; one block adds the
// kFrobBlocks partials.
constexpr int kFrobBlocks = 304;

__global__ void k_frob_part(int64_t n, const double* __restrict__ A, const double* __restrict__ rs, int m,
                            double* __restrict__ part) {
  __shared__ double sh[32];
  const int64_t per = (n + kFrobBlocks - 1) / kFrobBlocks;
  const int64_t a = blockIdx.x * per, b = a + per < n ? a + per : n;
  double s = 0;
  for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) {
    const double v = rs ? A[e] * rs[e / m] * rs[e % m] : A[e];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_frob_final(const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double t = 0;
    for (int b = 0; b < kFrobBlocks; b++) t += part[b];
    out[0] = sqrt(t);
  }
}


// Partial sums of ((A - C)_ij rs_i rs_j)^2 over m x m arrays, A in FP64 and C in FP32.
__global__ void k_frob_diff_part(int64_t n, const double* __restrict__ A, const float* __restrict__ C,
                                 const double* __restrict__ rs, int m, double* __restrict__ part) {
  __shared__ double sh[32];
  const int64_t per = (n + kFrobBlocks - 1) / kFrobBlocks;
  const int64_t a = blockIdx.x * per, b = a + per < n ? a + per : n;
  double s = 0;
  for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) {
    const double v = (A[e] - (double)C[e]) * rs[e / m] * rs[e % m];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// HW (m x r, ld ldh, FP64) in FP32, row-major (ld r) and transposed (r x m).
__global__ void k_hw_f32(int m, int r, const double* __restrict__ HW, int64_t ldh, float* __restrict__ hw,
                         float* __restrict__ hwt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * r) return;
  const int i = (int)(e / r), j = (int)(e % r);
  const float v = (float)HW[(int64_t)i * ldh + j];
  hw[e] = v;
  hwt[(int64_t)j * m + i] = v;
}

// out[0] = ||A||_F (n entries; scaled by rs[i] rs[j] as an m x m matrix when rs is given)
static fkf_status frob(fkf_ctx* ctx, int64_t n, const double* A, const double* rs, int m, double* part,
                       double* out) {
  k_frob_part<<<kFrobBlocks, 256, 0, ctx->stream>>>(n, A, rs, m, part);
  FKF_LAUNCHED(ctx);
  k_frob_final<<<1, 32, 0, ctx->stream>>>(part, out);
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}



// A = (A + A^T) / 2 in place (n x n)
__global__ void k_symmetrize(int n, double* __restrict__ A) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i < j) {
      const double v = 0.5 * (A[e] + A[(int64_t)j * n + i]);
      A[e] = v;
      A[(int64_t)j * n + i] = v;
    }
  }
}

template <typename T>
__global__ void k_cast(int64_t n, const double* __restrict__ src, T* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (T)src[e];
}

// X[ci, q] += sum_p cval[p] E[crow[p], q]   (warp per cluster-order cell)
template <typename T>
__global__ void k_csc_spmm(int64_t n, const int64_t* __restrict__ colptr, const int* __restrict__ crow,
                           const double* __restrict__ cval, const double* __restrict__ E, int ncols,
                           T* __restrict__ X, int64_t ldx) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const int64_t a = colptr[w], b = colptr[w + 1];
  if (a == b) return;
  for (int q = lane; q < ncols; q += 32) {
    double acc = 0;
    for (int64_t p = a; p < b; p++) acc += cval[p] * E[(int64_t)crow[p] * ncols + q];
    X[w * ldx + q] += (T)acc;
  }
}

// var[perm[i]] = alpha sigma2 - sum_j D[j] W[i, j]^2   (warp per row)
template <typename T>
__global__ void k_variance(int64_t n, int r, const T* __restrict__ W, int64_t ldw, const double* __restrict__ D,
                           double alpha_sigma2, const int64_t* __restrict__ perm, double* __restrict__ var) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const T* row = W + w * ldw;
  double acc = 0;
  for (int j = lane; j < r; j += 32) {
    const double x = (double)row[j];
    acc += D[j] * x * x;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) var[perm[w]] = alpha_sigma2 - acc;
}

// column sums of squares, per row chunk (partials), then ordered reduction
template <typename T>
__global__ void k_colsq_part(int64_t n, int r, const T* __restrict__ W, int64_t ldw, int64_t chunk,
                             double* __restrict__ part) {
  const int64_t a = blockIdx.y * chunk, b = a + chunk < n ? a + chunk : n;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < r; j += gridDim.x * blockDim.x) {
    double s = 0;
    for (int64_t i = a; i < b; i++) {
      const double x = (double)W[i * ldw + j];
      s += x * x;
    }
    part[(int64_t)blockIdx.y * r + j] = s;
  }
}

// a (FP64, original order, ld ns) -> ac (T, cluster order, ld ns)
template <typename T>
__global__ void k_gather_cast(int64_t n, int ns, const double* __restrict__ a, const int64_t* __restrict__ perm,
                              T* __restrict__ ac) {
  const int64_t total = n * ns;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ns;
    ac[e] = (T)a[perm[i] * ns + e % ns];
  }
}

// out[perm[i], j] = s[i] + sqrt(alpha) (a[i, j] - t[i, j])
template <typename T>
__global__ void k_realize(int64_t n, int ns, const double* __restrict__ s, const T* __restrict__ ac,
                          const T* __restrict__ t, double sqa, const int64_t* __restrict__ perm,
                          double* __restrict__ out) {
  const int64_t total = n * ns;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ns;
    const int j = (int)(e % ns);
    out[perm[i] * ns + j] = s[i] + sqa * ((double)ac[e] - (double)t[e]);
  }
}

// Ys[j, q] = sig_j * Y[j, q], sig_j = 1 - sqrt(1 - D_j / alpha)
__global__ void k_sig_rows(int r, int ns, const double* __restrict__ Y, const double* __restrict__ D, double alpha,
                           double* __restrict__ Ys) {
  const int64_t total = (int64_t)r * ns;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / ns);
    Ys[e] = (1.0 - sqrt(1.0 - D[j] / alpha)) * Y[e];
  }
}

inline int nblk(int64_t total, int threads = 256, int cap = 152 * 32) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, threads), cap));
}

}  // namespace

struct fkf_filter {
  fkf_hmat* h = nullptr;
  fkf_ctx* ctx = nullptr;
  int64_t n = 0;
  int m_max = 0, r_max = 0;
  int64_t ldwg = 0;
  double trunc_tol = 0, gep_tol = 0, orth_tol = 0;
  int64_t k = 0;
  int64_t chol_exact_retries = 0;  // innovation factorisations redone with exact FP64 products
  double alpha = 0;
  int r = 0;
  int cur = 0;
  size_t w = 8;
  DevBuf WG[2], Xb[2], Bt, s_hat, s_new, D, Dn;
  // When diag is false the low-rank weight is the full symmetric r x r matrix
  // Df (Sigma = alpha Gamma - W Df W^T, W^T Gamma^-1 W = I); observers first
  // diagonalise it (canonicalize) so that the state has the paper's form.
  bool diag = true;
  DevBuf Df, Dfn, Ep, Qm;
  double new_tol = 0;  // relative information outside span(W) below which the basis is kept
  int last_path = 0;   // 0: general merge, 1: basis kept (no new directions), 3: fixed-H reuse
  int gep_rank = 0, new_dirs = 0, t_eig = 0;  // last merge step
  double t_lmax = 0;
  // The last step kept the basis, and G, [HW | A], the dense H^T and its CSC
  // index still hold that step's products for the current W (prev_*: its H and R).
  bool products_valid = false;
  int prev_m = -1;
  int64_t prev_nnz = -1;
  std::vector<int64_t> prev_rp;
  std::vector<double> prev_rdiag;
  std::vector<int32_t> prev_col;  // host copies, kept for host-side inputs only
  std::vector<double> prev_val;
  // step inputs
  DevBuf rowptr, col, val, y, rdiag, rs, flag;
  DevBuf cnt, cursor, colptr, crow, cval;
  // small FP64 buffers
  DevBuf HWA, As, At, S, a, C, lam, P, Tm, th, Po, F1t, ZL, M, thM, Sk, J, E, Ecast;
  DevBuf nu, z, uz, vcoef, HWD, nll, dbar, red, scanws;
  DevBuf Lpv, Gm, F1c, pcws;  // pivoted Cholesky of T: factor, its Gram, the solved factor, workspace
  DevBuf eigws, cholws, gramws, tmp1, tmp2, tmp3;
  DevBuf sbak;  // copy of the innovation system while its factorisation uses slice products
  TcGemmWs rot;       // tensor-core products (FP32 state): the rotation and the basis test
  DevBuf hw32, c32;   // basis test of the FP32 state: HW and HW^T in FP32, HW HW^T
  cudaEvent_t ev[7] = {};
  // HW gathered (main stream) -> HWD and the product HWD HW^T on the
  // low-priority stream, beside the H-apply -> consumed on the main stream
  cudaEvent_t ev_hw = nullptr, ev_p = nullptr;
  cudaEvent_t ev_schur = nullptr;  // the kept-basis weight E' (Schur complement) is formed
  DevBuf Pw;  // HWD HW^T (m x m, lower triangle)
  DevBuf xcmax;  // column maxima of the dense H^T (FP32 state), for the H-apply's split
  int refresh_every = 0;  // scheduled refresh (W <- Gamma_H X) after every refresh_every-th step; 0: never
  // randomized GHEP (App. B): k modes from a sketch of l = k + p Gaussian columns
  // (Omega, N x l, cluster order, FP64); rk = 0: the exact data-space GEP
  int rk = 0, rl = 0;
  DevBuf omega, rZ, rAZ, rGram, rLp, rGm, rY, rB, rV, rT, rSk;
  std::vector<double> rlam_h;
  DevBuf refw;            // Gamma_H X when r exceeds the spare buffer's m_max columns
  double phase_ms[6] = {};
};

static fkf_status alloc_small(fkf_filter* f) {
  fkf_ctx* ctx = f->ctx;
  const int64_t m = f->m_max, r = f->r_max, nm = r + m;
  auto A = [&](DevBuf& b, int64_t elems) { return dev_alloc(ctx, b, (size_t)std::max<int64_t>(elems, 1) * 8); };
  FKF_TRY(A(f->HWA, m * nm));
  FKF_TRY(A(f->As, m * m));
  FKF_TRY(A(f->At, m * m));
  FKF_TRY(A(f->S, (m + r) * (m + r)));  // the augmented matrix [[S, K], [K^T, E]]
  FKF_TRY(A(f->a, m));
  FKF_TRY(A(f->C, m * m));
  FKF_TRY(A(f->lam, m));
  FKF_TRY(A(f->P, r * m));
  FKF_TRY(A(f->Tm, m * m));
  FKF_TRY(A(f->th, m));
  FKF_TRY(A(f->Po, m * m));
  FKF_TRY(A(f->F1t, m * m));
  FKF_TRY(A(f->ZL, nm * m));
  FKF_TRY(A(f->M, nm * nm));
  FKF_TRY(A(f->thM, nm));
  FKF_TRY(A(f->Sk, r * nm));
  FKF_TRY(A(f->J, m * r));
  FKF_TRY(A(f->E, nm * r));
  FKF_TRY(dev_alloc(ctx, f->Ecast, (size_t)std::max<int64_t>(nm * r, 1) * f->w));
  FKF_TRY(A(f->nu, m));
  FKF_TRY(A(f->z, m));
  FKF_TRY(A(f->uz, r));
  FKF_TRY(dev_alloc(ctx, f->vcoef, (size_t)std::max<int64_t>(nm, 1) * f->w));
  FKF_TRY(A(f->HWD, m * r));
  FKF_TRY(A(f->Pw, m * m));
  FKF_TRY(A(f->nll, 4));
  FKF_TRY(A(f->Lpv, m * m));
  FKF_TRY(A(f->Gm, m * m));
  FKF_TRY(A(f->F1c, m * m));
  FKF_TRY(A(f->red, kFrobBlocks));
  FKF_TRY(A(f->dbar, r));
  FKF_TRY(A(f->y, m));
  FKF_TRY(A(f->rdiag, m));
  FKF_TRY(A(f->rs, m));
  FKF_TRY(A(f->rowptr, m + 1));
  FKF_TRY(dev_alloc(ctx, f->flag, 64));
  FKF_TRY(A(f->Df, r * r));
  FKF_TRY(A(f->Dfn, r * r));
  FKF_TRY(A(f->Ep, r * r));
  FKF_TRY(A(f->Qm, r * r));
  if (f->w == 4) {
    FKF_TRY(dev_alloc(ctx, f->xcmax, (size_t)std::max<int64_t>(m, 1) * sizeof(unsigned)));
    FKF_TRY(A(f->hw32, m * r));        // 2 m r floats
    FKF_TRY(A(f->c32, m * m / 2 + 1));  // m^2 floats
  }
  return FKF_OK;
}

fkf_status filter_create(fkf_hmat* h, const double* s0, double alpha0, double trunc_tol, int m_max, int r_max,
                         fkf_filter** out) {
  fkf_ctx* ctx = h->ctx;
  if (alpha0 < 0 || !(trunc_tol >= 0) || m_max < 1 || r_max < 1)
    return set_err(ctx, FKF_EINVAL, "filter_create: alpha0 >= 0, trunc_tol >= 0, m_max >= 1, r_max >= 1 required");
  fkf_filter* f = new fkf_filter();
  f->h = h;
  f->ctx = ctx;
  f->n = h->n;
  f->m_max = m_max;
  f->r_max = r_max;
  f->ldwg = (int64_t)r_max + m_max;
  f->trunc_tol = trunc_tol;
  f->w = h->prec == FKF_FP64 ? 8 : 4;
  f->gep_tol = h->prec == FKF_FP64 ? 1e-13 : 1e-7;
  // FP32 storage of W, X and G leaves a noise floor of ~1e-5 in the data-space
  // Gram T; new directions are only accepted clearly above it.
  f->orth_tol = h->prec == FKF_FP64 ? 1e-10 : 1e-3;
  // ||R^-1/2 (A - HW HW^T) R^-1/2||_F / ||R^-1/2 A R^-1/2||_F below new_tol:
  // the step's information lies in span(W) and the basis is kept
  f->new_tol = h->prec == FKF_FP64 ? 1e-10 : 1e-4;
  f->alpha = alpha0;
  auto fail = [&](fkf_status st) {
    delete f;
    return st;
  };
  const int64_t n = f->n;
  fkf_status st;
  for (int b = 0; b < 2; b++) {
    if ((st = dev_alloc(ctx, f->WG[b], (size_t)n * f->ldwg * f->w)) != FKF_OK) return fail(st);
    if ((st = dev_alloc(ctx, f->Xb[b], (size_t)n * r_max * f->w)) != FKF_OK) return fail(st);
  }
  if ((st = dev_alloc(ctx, f->Bt, (size_t)n * m_max * f->w)) != FKF_OK) return fail(st);
  if ((st = dev_alloc(ctx, f->s_hat, (size_t)n * 8)) != FKF_OK) return fail(st);
  if ((st = dev_alloc(ctx, f->s_new, (size_t)n * 8)) != FKF_OK) return fail(st);
  if ((st = dev_alloc(ctx, f->D, (size_t)r_max * 8)) != FKF_OK) return fail(st);
  if ((st = dev_alloc(ctx, f->Dn, (size_t)r_max * 8)) != FKF_OK) return fail(st);
  if ((st = dev_alloc(ctx, f->cnt, (size_t)n * 4 + 64)) != FKF_OK) return fail(st);
  if ((st = dev_alloc(ctx, f->cursor, (size_t)n * 4 + 64)) != FKF_OK) return fail(st);
  if ((st = dev_alloc(ctx, f->colptr, (size_t)(n + 1) * 8)) != FKF_OK) return fail(st);
  if ((st = alloc_small(f)) != FKF_OK) return fail(st);
  if (s0) {
    std::vector<double> sc(n);
    for (int64_t i = 0; i < n; i++) sc[i] = s0[h->perm[i]];
    if (cudaMemcpyAsync(f->s_hat.p, sc.data(), n * 8, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
      return fail(set_err(ctx, FKF_ECUDA, "upload s0"));
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return fail(set_err(ctx, FKF_ECUDA, "sync"));
  } else if (cudaMemsetAsync(f->s_hat.p, 0, n * 8, ctx->stream) != cudaSuccess) {
    return fail(set_err(ctx, FKF_ECUDA, "memset s0"));
  }
  for (int i = 0; i < 7; i++) cudaEventCreate(&f->ev[i]);
  cudaEventCreateWithFlags(&f->ev_hw, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&f->ev_p, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&f->ev_schur, cudaEventDisableTiming);
  *out = f;
  return FKF_OK;
}

void filter_destroy(fkf_filter* f) {
  if (!f) return;
  for (int i = 0; i < 7; i++)
    if (f->ev[i]) cudaEventDestroy(f->ev[i]);
  if (f->ev_hw) cudaEventDestroy(f->ev_hw);
  if (f->ev_p) cudaEventDestroy(f->ev_p);
  if (f->ev_schur) cudaEventDestroy(f->ev_schur);
  delete f;
}

template <typename T>
static fkf_status gemm_T(fkf_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const T* A,
                         int64_t lda, const T* B, int64_t ldb, double beta, T* C, int64_t ldc);
template <>
fkf_status gemm_T<double>(fkf_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                          const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                          int64_t ldc) {
  return gemm_f64(ctx, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}
template <>
fkf_status gemm_T<float>(fkf_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                         const float* A, int64_t lda, const float* B, int64_t ldb, double beta, float* C,
                         int64_t ldc) {
  return gemm_f32(ctx, ta, tb, M, N, K, (float)alpha, A, lda, B, ldb, (float)beta, C, ldc);
}

// The data-space products of the general (merge) step: the large ones as FP64
// GEMMs on the tensor cores (integer slices, 49 bits of every value relative to
// its row or column scale), the small ones on the FP64 tile GEMM.  Nothing of
// the step's own runs beside them (unlike the kept-basis weight products, which
// share the SMs with the H-apply's phase 2 and stay on the FP64 pipe).
static fkf_status gemm_merge(fkf_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                             const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                             int64_t ldc) {
  if (ctx->fp64_tc && (double)M * N * K >= 1e8 && cdiv(M, 128) * cdiv(N, 64) >= 16)
    return gemm_f64_tc(ctx, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  return gemm_f64(ctx, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

// For the scope of a filter operation: the tensor-core FP64 products only for
// an FP32 state (an FP64 state keeps exact FP64 arithmetic in its m x m and
// r x r algebra, where products with cancellation decide ranks).
struct Fp64TcScope {
  fkf_ctx* ctx;
  bool saved;
  Fp64TcScope(fkf_ctx* c, bool allow) : ctx(c), saved(c->fp64_tc) { ctx->fp64_tc = saved && allow; }
  ~Fp64TcScope() { ctx->fp64_tc = saved; }
};

// The innovation system's blocked Cholesky factorisation (n x n, lda, the
// first nf pivots; schur_done as chol_blocked_f64).  Its large trailing
// updates run on the tensor cores with 49-bit slice products when
// ctx->fp64_tc is set; the Schur complements cancel, and on a system whose
// conditioning nears the limit of FP64 the slices' rounding can leave a
// pivot that is not positive where exact FP64 products would not.  The
// factorisation then starts again from a copy of the system with exact FP64
// products throughout.
static fkf_status chol_innovation(fkf_filter* f, int n, int nf, double* A, int64_t lda, cudaEvent_t schur_done) {
  fkf_ctx* ctx = f->ctx;
  if (!ctx->fp64_tc) return chol_blocked_f64(ctx, n, nf, A, lda, f->cholws, schur_done);
  const size_t bytes = (size_t)n * lda * sizeof(double);
  if (f->sbak.bytes < bytes) FKF_TRY(dev_alloc(ctx, f->sbak, bytes));
  FKF_CUDA(ctx, cudaMemcpyAsync(f->sbak.p, A, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  const fkf_status st = chol_blocked_f64(ctx, n, nf, A, lda, f->cholws, schur_done);
  if (st != FKF_ENOTSPD) return st;
  // (a failed attempt returns with none of its work in flight)
  FKF_CUDA(ctx, cudaMemcpyAsync(A, f->sbak.p, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  f->chol_exact_retries++;
  Fp64TcScope exact(ctx, false);
  return chol_blocked_f64(ctx, n, nf, A, lda, f->cholws, schur_done);
}

static fkf_status gram_T(fkf_ctx* ctx, size_t w, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                         const void* B, int64_t ldb, double* C, int64_t ldc, DevBuf& ws) {
  if (w == 8) return gram_f64(ctx, M, N, K, (const double*)A, lda, (const double*)B, ldb, C, ldc, ws);
  return gram_f32(ctx, M, N, K, (const float*)A, lda, (const float*)B, ldb, C, ldc, ws);
}

// C[i][j] -= P[i][j] for j <= i < m (lower triangles).
__global__ void k_sub_lower(int m, const double* __restrict__ P, int64_t ldp, double* __restrict__ C, int64_t ldc) {
  const int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / m, j = e % m;
    if (j <= i) C[i * ldc + j] -= P[i * ldp + j];
  }
}

namespace {
// Runs the library's stream-ordered helpers on another stream for its scope.
struct OnStream {
  fkf_ctx* ctx;
  cudaStream_t saved;
  OnStream(fkf_ctx* c, cudaStream_t s) : ctx(c), saved(c->stream) { ctx->stream = s; }
  ~OnStream() { ctx->stream = saved; }
};
}  // namespace

// The products of the step that involve the low-rank weight and HW only,
// HWD = HW D (D diagonal, or the full weight Df) and Pw = HWD HW^T (lower
// triangle), once HW = H W is in HWA (m x r, ld ldh) and ev_hw has been
// recorded after it on the context stream.  They go to the context's
// low-priority stream, so that on an FP32 state they run on the SMs' FP64
// units beside the tensor-core H-apply's phase 2 (which leaves room for one
// FP64 tile CTA per SM) instead of after it; the step's main stream waits for
// ev_p before it uses HWD or Pw.  Nothing to do when r = 0.
static fkf_status weight_products(fkf_filter* f, int m, const double* HW, int64_t ldh) {
  fkf_ctx* ctx = f->ctx;
  const int r = f->r;
  if (r <= 0) return FKF_OK;
  FKF_TRY(ctx_side_lo(ctx));
  cudaStream_t lo = ctx->side_lo;
  FKF_CUDA(ctx, cudaStreamWaitEvent(lo, f->ev_hw, 0));
  {
    OnStream on(ctx, lo);
    if (f->diag) {
      k_scale_cols<<<nblk((int64_t)m * r), 256, 0, lo>>>(m, r, HW, ldh, f->D.as<double>(), f->HWD.as<double>());
      FKF_LAUNCHED(ctx);
    } else {
      FKF_TRY(gemm_f64(ctx, false, false, m, r, r, 1.0, HW, ldh, f->Df.as<double>(), r, 0.0, f->HWD.as<double>(), r));
    }
    FKF_TRY(gemm_sym_f64(ctx, false, true, m, r, 1.0, f->HWD.as<double>(), r, HW, ldh, 0.0, f->Pw.as<double>(), m,
                         true));
  }
  FKF_CUDA(ctx, cudaEventRecord(f->ev_p, lo));
  return FKF_OK;
}

// Randomized GHEP (App. B, Alg. randomizedghepuncert) for A = H^T R^-1 H and
// B = Gamma^-1, written in data space: with the Gaussian sketch Omega (N x l)
// and Z = R^-1 H Omega (m x l),
//   step 1  Ybar = A Omega = H^T Z;
//   step 2  the Gamma-orthonormal basis of Ybar: its Gram Ybar^T Gamma Ybar =
//           Z^T (H Gamma H^T) Z = Z^T As Z (l x l, data space) is factored by
//           the rank-revealing pivoted Cholesky Gram ~= Lp Lp^T, and
//           Qhat = Ybar Y with Y = Lp (Lp^T Lp)^-1 (Y^T Gram Y = I);
//   step 3  Q = Gamma Qhat = G B with B = Z Y (G = Gamma H^T), Q^T Gamma^-1 Q = I;
//   step 4  T = Q^T A Q = V^T R^-1 V with V = H Q = As B = (As Z) Y;
//   step 5  T = S Lambda S^T, the k largest modes kept: U = Q S_k = G C with
//           C = B S_k (m x k), Lambda_k in lam.
// C and lam take the place of the exact GEP's (U = G C, U^T Gamma^-1 U =
// C^T As C = I), so the orthonormalisation and merge that follow are
// unchanged.  Cost O(m^2 l) instead of the O(m^3) eigensolve.
static fkf_status randomized_gep(fkf_filter* f, int m, int* mlam_out) {
  fkf_ctx* ctx = f->ctx;
  cudaStream_t st = ctx->stream;
  const int l = f->rl, k = f->rk;
  const int64_t n = f->n;
  *mlam_out = 0;
  double* Z = f->rZ.as<double>();
  double* AZ = f->rAZ.as<double>();
  double* Gram = f->rGram.as<double>();
  // step 1: H Omega (gather of Omega's rows at H's columns), then Z = R^-1 H Omega
  csr_gather<double>(m, f->rowptr.as<int64_t>(), f->col.as<int32_t>(), f->val.as<double>(),
                     f->h->iperm_d.as<int64_t>(), n, f->omega.as<double>(), l, l, Z, l, st);
  FKF_LAUNCHED(ctx);
  k_scale_rows<<<nblk((int64_t)m * l), 256, 0, st>>>(m, l, Z, l, f->rs.as<double>(), 1);
  FKF_LAUNCHED(ctx);
  // step 2: Gram = Z^T As Z, pivoted Cholesky relative to its largest diagonal entry
  FKF_TRY(gemm_f64(ctx, false, false, m, l, m, 1.0, f->As.as<double>(), m, Z, l, 0.0, AZ, l));
  FKF_TRY(gemm_sym_f64(ctx, true, false, l, m, 1.0, Z, l, AZ, l, 0.0, Gram, l));
  std::vector<double> gdiag(l);
  FKF_CUDA(ctx, cudaMemcpy2DAsync(gdiag.data(), 8, Gram, (size_t)(l + 1) * 8, 8, l, cudaMemcpyDeviceToHost, st));
  FKF_CUDA(ctx, cudaStreamSynchronize(st));
  double gmax = 0;
  for (double v : gdiag) gmax = std::max(gmax, v);
  if (!(gmax > 0)) return FKF_OK;  // H Omega = 0: no information
  int rank = 0;
  double* Lp = f->rLp.as<double>();
  FKF_TRY(pchol_f64(ctx, l, Gram, l, f->gep_tol * gmax, l, Lp, l, f->pcws, &rank));
  if (rank == 0) return FKF_OK;
  double* Gm = f->rGm.as<double>();
  double* Y = f->rY.as<double>();  // l x rank
  FKF_TRY(gemm_f64(ctx, true, false, rank, rank, l, 1.0, Lp, l, Lp, l, 0.0, Gm, rank));
  FKF_CUDA(ctx, cudaMemcpy2DAsync(Y, (size_t)rank * 8, Lp, (size_t)l * 8, (size_t)rank * 8, l,
                                  cudaMemcpyDeviceToDevice, st));
  FKF_TRY(chol_f64(ctx, rank, Gm, f->cholws));
  FKF_TRY(chol_solve_f64(ctx, rank, Gm, Y, l));  // rows of Y: Lp (Lp^T Lp)^-1
  // step 3: B = Z Y;  step 4: V = (As Z) Y, T = V^T R^-1 V
  double* B = f->rB.as<double>();
  double* V = f->rV.as<double>();
  double* T = f->rT.as<double>();
  FKF_TRY(gemm_f64(ctx, false, false, m, rank, l, 1.0, Z, l, Y, rank, 0.0, B, rank));
  FKF_TRY(gemm_f64(ctx, false, false, m, rank, l, 1.0, AZ, l, Y, rank, 0.0, V, rank));
  k_scale_rows<<<nblk((int64_t)m * rank), 256, 0, st>>>(m, rank, V, rank, f->rs.as<double>(), 0);
  FKF_LAUNCHED(ctx);
  FKF_TRY(gemm_sym_f64(ctx, true, false, rank, m, 1.0, V, rank, V, rank, 0.0, T, rank));
  // step 5: eigenpairs of T, the k largest above the GEP threshold
  std::vector<double> w_h;
  FKF_TRY(eigh_f64(ctx, rank, T, f->a.as<double>(), w_h, f->eigws));
  const double wmax = w_h.empty() ? 0.0 : w_h.back();
  int kk = 0;
  for (int i = rank - 1; i >= 0 && kk < k; i--)
    if (wmax > 0 && w_h[i] > f->gep_tol * wmax) kk++;
    else break;
  if (kk == 0) return FKF_OK;
  double* Sk = f->rSk.as<double>();  // kk x rank, rows = eigenvectors, largest first
  k_top_rows<<<nblk((int64_t)kk * rank), 256, 0, st>>>(rank, kk, T, f->a.as<double>(), 2, Sk, rank);
  FKF_LAUNCHED(ctx);
  FKF_TRY(gemm_f64(ctx, false, true, m, kk, rank, 1.0, B, rank, Sk, rank, 0.0, f->C.as<double>(), kk));
  f->rlam_h.assign(kk, 0.0);
  for (int q = 0; q < kk; q++) f->rlam_h[q] = w_h[rank - 1 - q];
  FKF_CUDA(ctx, cudaMemcpyAsync(f->lam.p, f->rlam_h.data(), kk * 8, cudaMemcpyHostToDevice, st));
  *mlam_out = kk;
  return FKF_OK;
}

fkf_status filter_set_randomized_ghep(fkf_filter* f, int k, int p, const double* omega_dev) {
  fkf_ctx* ctx = f->ctx;
  if (k == 0) {
    f->rk = f->rl = 0;
    return FKF_OK;
  }
  const int l = k + p;
  if (k < 0 || p < 0 || l > f->m_max || !omega_dev)
    return set_err(ctx, FKF_EINVAL, "set_randomized_ghep: k >= 1, p >= 0, k + p <= m_max and a sketch required");
  const int64_t n = f->n, m = f->m_max;
  auto A = [&](DevBuf& b, int64_t elems) { return dev_alloc(ctx, b, (size_t)std::max<int64_t>(elems, 1) * 8); };
  FKF_TRY(A(f->omega, n * l));
  FKF_TRY(A(f->rZ, m * l));
  FKF_TRY(A(f->rAZ, m * l));
  FKF_TRY(A(f->rGram, (int64_t)l * l));
  FKF_TRY(A(f->rLp, (int64_t)l * l));
  FKF_TRY(A(f->rGm, (int64_t)l * l));
  FKF_TRY(A(f->rY, (int64_t)l * l));
  FKF_TRY(A(f->rB, m * l));
  FKF_TRY(A(f->rV, m * l));
  FKF_TRY(A(f->rT, (int64_t)l * l));
  FKF_TRY(A(f->rSk, (int64_t)l * l));
  // cluster order: row i of the stored sketch is the caller's row perm[i]
  FKF_TRY(hmat_permute_rows_f64(ctx, omega_dev, l, f->h->perm_d.as<int64_t>(), f->omega.as<double>(), l, n, l));
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  f->rk = k;
  f->rl = l;
  return FKF_OK;
}

template <typename T>
static fkf_status step_impl(fkf_filter* f, const double* y_in, int m, const int64_t* rowptr_in,
                            const int32_t* col_in, const double* val_in, const double* R_in, double r_scalar,
                            int flags, double* nll_out, double bc) {
  fkf_ctx* ctx = f->ctx;
  fkf_hmat* h = f->h;
  cudaStream_t st = ctx->stream;
  const int64_t n = f->n;
  const bool on_dev = (flags & FKF_STEP_INPUTS_ON_DEVICE) != 0;
  if (m < 1 || m > f->m_max) return set_err(ctx, FKF_EINVAL, "filter_step: m=%d outside [1, %d]", m, f->m_max);
  if (!R_in && !(r_scalar > 0)) return set_err(ctx, FKF_EINVAL, "filter_step: r_scalar must be > 0 when R is NULL");
  // ---- inputs: validate rowptr on the host, stage everything on the device
  std::vector<int64_t> rp(m + 1);
  if (on_dev)
    FKF_CUDA(ctx, cudaMemcpyAsync(rp.data(), rowptr_in, (m + 1) * 8, cudaMemcpyDeviceToHost, st));
  FKF_CUDA(ctx, cudaStreamSynchronize(st));
  if (!on_dev) std::memcpy(rp.data(), rowptr_in, (m + 1) * 8);
  if (rp[0] != 0) return set_err(ctx, FKF_EINVAL, "filter_step: rowptr[0] must be 0");
  for (int j = 0; j < m; j++)
    if (rp[j + 1] < rp[j]) return set_err(ctx, FKF_EINVAL, "filter_step: rowptr not nondecreasing at %d", j);
  const int64_t nnz = rp[m];
  std::vector<double> rdiag(m), rs(m);
  if (R_in) {
    if (on_dev)
      FKF_CUDA(ctx, cudaMemcpyAsync(rdiag.data(), R_in, m * 8, cudaMemcpyDeviceToHost, st));
    FKF_CUDA(ctx, cudaStreamSynchronize(st));
    if (!on_dev) std::memcpy(rdiag.data(), R_in, m * 8);
  } else {
    std::fill(rdiag.begin(), rdiag.end(), r_scalar);
  }
  for (int j = 0; j < m; j++) {
    if (!(rdiag[j] > 0) || !std::isfinite(rdiag[j]))
      return set_err(ctx, FKF_EINVAL, "filter_step: R[%d] must be finite and > 0", j);
    rs[j] = 1.0 / std::sqrt(rdiag[j]);
  }
  // ---- fixed-H fast path (opt-in): H and R byte-identical to the previous
  // step's, which kept the basis, so G = Gamma_H H^T, [HW | A] and the basis
  // decision are unchanged (Alg. kalmanconstantH: the products with Gamma are
  // formed once for a constant H)
  // the extended filter re-linearises every step: its Jacobian changes with the mean
  const bool allow_fixed = (flags & FKF_STEP_ALLOW_FIXED_H) && !(flags & FKF_STEP_FULL_UPDATE) && bc == 0.0;
  bool reuse = false;
  if (allow_fixed && f->products_valid && m == f->prev_m && nnz == f->prev_nnz && rp == f->prev_rp &&
      rdiag == f->prev_rdiag) {
    if (on_dev) {
      int* diff = f->flag.as<int>() + 8;
      FKF_CUDA(ctx, cudaMemsetAsync(diff, 0, sizeof(int), st));
      if (nnz > 0) {
        k_words_differ<<<nblk(nnz), 256, 0, st>>>(nnz, reinterpret_cast<const uint32_t*>(col_in),
                                                 f->col.as<uint32_t>(), diff);
        FKF_LAUNCHED(ctx);
        k_words_differ<<<nblk(2 * nnz), 256, 0, st>>>(2 * nnz, reinterpret_cast<const uint32_t*>(val_in),
                                                     f->val.as<uint32_t>(), diff);
        FKF_LAUNCHED(ctx);
      }
      int hd = 1;
      FKF_CUDA(ctx, cudaMemcpyAsync(&hd, diff, sizeof(int), cudaMemcpyDeviceToHost, st));
      FKF_CUDA(ctx, cudaStreamSynchronize(st));
      reuse = hd == 0;
    } else {
      reuse = (size_t)nnz == f->prev_col.size() && std::memcmp(col_in, f->prev_col.data(), nnz * 4) == 0 &&
              std::memcmp(val_in, f->prev_val.data(), nnz * 8) == 0;
    }
  }
  f->products_valid = false;  // set again when this step keeps the basis
  if (f->col.bytes < (size_t)std::max<int64_t>(nnz, 1) * 4) FKF_TRY(dev_alloc(ctx, f->col, std::max<int64_t>(nnz, 1) * 4));
  if (f->val.bytes < (size_t)std::max<int64_t>(nnz, 1) * 8) FKF_TRY(dev_alloc(ctx, f->val, std::max<int64_t>(nnz, 1) * 8));
  if (f->crow.bytes < (size_t)std::max<int64_t>(nnz, 1) * 4) FKF_TRY(dev_alloc(ctx, f->crow, std::max<int64_t>(nnz, 1) * 4));
  if (f->cval.bytes < (size_t)std::max<int64_t>(nnz, 1) * 8) FKF_TRY(dev_alloc(ctx, f->cval, std::max<int64_t>(nnz, 1) * 8));
  const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (!reuse) {
    FKF_CUDA(ctx, cudaMemcpyAsync(f->rowptr.p, rowptr_in, (m + 1) * 8, kind, st));
    if (nnz > 0) {
      FKF_CUDA(ctx, cudaMemcpyAsync(f->col.p, col_in, nnz * 4, kind, st));
      FKF_CUDA(ctx, cudaMemcpyAsync(f->val.p, val_in, nnz * 8, kind, st));
    }
  }
  FKF_CUDA(ctx, cudaMemcpyAsync(f->y.p, y_in, m * 8, kind, st));
  FKF_CUDA(ctx, cudaMemcpyAsync(f->rdiag.p, rdiag.data(), m * 8, cudaMemcpyHostToDevice, st));
  FKF_CUDA(ctx, cudaMemcpyAsync(f->rs.p, rs.data(), m * 8, cudaMemcpyHostToDevice, st));
  FKF_CUDA(ctx, cudaMemsetAsync(f->flag.p, 0, 64, st));
  if (bc > 0.0) {
    // EKF: nu = y - H s(x_pred) and H <- H_k = H diag(s'(x_pred)) before anything reads H
    k_boxcox_linearize<<<(int)cdiv((int64_t)m * 32, 256), 256, 0, st>>>(
        m, f->rowptr.as<int64_t>(), f->col.as<int32_t>(), f->val.as<double>(), h->iperm_d.as<int64_t>(), n,
        f->s_hat.as<double>(), bc, f->y.as<double>(), f->nu.as<double>());
    FKF_LAUNCHED(ctx);
  }

  const int r = f->r, rmax = f->r_max;
  const double alpha1 = f->alpha + 1.0;  // predict
  const int64_t ld = f->ldwg;
  T* WGc = f->WG[f->cur].as<T>();
  T* WGn = f->WG[1 - f->cur].as<T>();
  T* Xc = f->Xb[f->cur].as<T>();
  T* Xn = f->Xb[1 - f->cur].as<T>();
  T* Wc = WGc + (rmax - r);       // N x r, ld
  T* G = WGc + rmax;              // N x m, ld
  const int64_t* iperm = h->iperm_d.as<int64_t>();
  const int64_t* rowptr = f->rowptr.as<int64_t>();
  const int32_t* col = f->col.as<int32_t>();
  const double* val = f->val.as<double>();

  // work a previous step left on the low-priority stream (if it failed part-way)
  // is finished before this step touches the buffers it reads or writes
  FKF_CUDA(ctx, cudaStreamWaitEvent(st, f->ev_p, 0));
  FKF_CUDA(ctx, cudaStreamWaitEvent(st, f->ev_schur, 0));
  FKF_CUDA(ctx, cudaEventRecord(f->ev[0], st));
  const int nm = r + m;
  double* HWA = f->HWA.as<double>();
  if (!reuse) {
    // ---- S1: column index of H (CSC, cluster order) and the dense H^T
    FKF_CUDA(ctx, cudaMemsetAsync(f->cnt.p, 0, (size_t)n * 4, st));
    FKF_CUDA(ctx, cudaMemsetAsync(f->cursor.p, 0, (size_t)n * 4, st));
    k_csc_count<<<(int)cdiv((int64_t)m * 32, 256), 256, 0, st>>>(m, rowptr, col, iperm, n, f->cnt.as<int>(),
                                                                  f->flag.as<int>());
    FKF_LAUNCHED(ctx);
    FKF_TRY(scan_counts(ctx, n, f->cnt.as<int>(), f->colptr.as<int64_t>(), f->scanws));
    k_csc_fill<<<(int)cdiv((int64_t)m * 32, 256), 256, 0, st>>>(m, rowptr, col, val, iperm, n, f->colptr.as<int64_t>(),
                                                                 f->cursor.as<int>(), f->crow.as<int>(),
                                                                 f->cval.as<double>());
    FKF_LAUNCHED(ctx);
    k_csc_sort<<<(int)cdiv(n, 256), 256, 0, st>>>(n, f->colptr.as<int64_t>(), f->crow.as<int>(), f->cval.as<double>());
    FKF_LAUNCHED(ctx);
    unsigned* xcmax = sizeof(T) == 4 ? f->xcmax.as<unsigned>() : nullptr;  // the FP32 split's column scales
    if (xcmax) FKF_CUDA(ctx, cudaMemsetAsync(xcmax, 0, (size_t)m * sizeof(unsigned), st));
    // the FP16 split engine takes H^T straight from the CSC index (no dense H^T)
    const bool sparse_x = sizeof(T) == 4 && !(flags & FKF_STEP_DENSE_HT) && hmat_sparse_x_ok(h, m);
    if (sparse_x) {
      k_csc_colmax<<<(int)cdiv(n, 256), 256, 0, st>>>(n, f->colptr.as<int64_t>(), f->crow.as<int>(),
                                                     f->cval.as<double>(), xcmax);
    } else {
      FKF_CUDA(ctx, cudaMemsetAsync(f->Bt.p, 0, (size_t)n * m * sizeof(T), st));
      k_densify_csc<T><<<(int)cdiv(n, 256), 256, 0, st>>>(n, f->colptr.as<int64_t>(), f->crow.as<int>(),
                                                          f->cval.as<double>(), f->Bt.as<T>(), m, xcmax);
    }
    FKF_LAUNCHED(ctx);
    // ---- gather HW = H W (needs no product with Gamma)
    csr_gather<T>(m, rowptr, col, val, iperm, n, Wc, ld, r, HWA, nm, st);
    FKF_LAUNCHED(ctx);
    FKF_CUDA(ctx, cudaEventRecord(f->ev[1], st));
    // ---- S2: G = Gamma_H H^T; the weight products start with its phase 2
    // (or after it, when the apply sets no mark)
    ctx->ph2_mark = r > 0 ? f->ev_hw : nullptr;
    ctx->ph2_marked = false;
    ctx->x_colmax = xcmax;
    const TcSparseX sx{n, nnz, f->colptr.as<int64_t>(), f->crow.as<int>(), f->cval.as<double>()};
    ctx->x_sparse = sparse_x ? &sx : nullptr;
    const fkf_status ast = hmat_apply_step(h, f->Bt.p, m, G, ld, m);
    const bool marked = ctx->ph2_marked;
    ctx->ph2_mark = nullptr;
    ctx->ph2_marked = false;
    ctx->x_colmax = nullptr;
    ctx->x_sparse = nullptr;
    FKF_TRY(ast);
    if (r > 0 && !marked) FKF_CUDA(ctx, cudaEventRecord(f->ev_hw, st));
    FKF_TRY(weight_products(f, m, HWA, nm));
    FKF_CUDA(ctx, cudaEventRecord(f->ev[2], st));
    // ---- gather A = H G; innovation
    csr_gather<T>(m, rowptr, col, val, iperm, n, G, ld, m, HWA + r, nm, st);
    FKF_LAUNCHED(ctx);
  } else {
    if (r > 0) FKF_CUDA(ctx, cudaEventRecord(f->ev_hw, st));
    FKF_TRY(weight_products(f, m, HWA, nm));
    for (int e = 1; e < 3; e++) FKF_CUDA(ctx, cudaEventRecord(f->ev[e], st));
  }
  if (bc == 0.0) {
    k_innovation<<<(int)cdiv((int64_t)m * 32, 256), 256, 0, st>>>(m, rowptr, col, val, iperm, n,
                                                                 f->s_hat.as<double>(), f->y.as<double>(),
                                                                 f->nu.as<double>());
    FKF_LAUNCHED(ctx);
  }
  const double* HW = HWA;       // m x r, ld nm
  const double* Araw = HWA + r;  // m x m, ld nm
  // S lives in the top-left m x m block of the augmented matrix (ld m + r)
  const int64_t lda_aug = (int64_t)m + r;
  double* S = f->S.as<double>();
  k_sym<<<nblk((int64_t)m * m), 256, 0, st>>>(m, Araw, nm, f->rs.as<double>(), f->rdiag.as<double>(), alpha1,
                                              f->As.as<double>(), f->At.as<double>(), S, lda_aug);
  FKF_LAUNCHED(ctx);
  // ---- does the step bring information outside span(W)?  The Gamma^-1-Gram
  // of G's component outside span(W) is A - HW HW^T (X^T G = (HW)^T, X^T W = I);
  // compared with A in the noise-whitened metric.
  double ratio = reuse ? 0.0 : 1.0;  // unchanged H, W and G: the previous step's decision stands
  if (!reuse) {
    double* nrm = f->nll.as<double>() + 1;
    int tc_fail = 0;
    if (r > 0) {
      if (sizeof(T) == 4) {
        // FP32 state: the test threshold (1e-4) is three orders above FP32 rounding of HW, so
        // HW HW^T runs on the tensor cores (3xTF32) and A - HW HW^T is formed in FP64
        float* hw = f->hw32.as<float>();
        float* hwt = hw + (int64_t)m * r;
        k_hw_f32<<<nblk((int64_t)m * r), 256, 0, st>>>(m, r, HW, nm, hw, hwt);
        FKF_LAUNCHED(ctx);
        const TcGemmProblem pr{hw, r, m, r, f->c32.as<float>(), m};
        FKF_TRY(tc_gemm_f32(ctx, &pr, 1, hwt, m, r, m, f->rot));
        k_frob_diff_part<<<kFrobBlocks, 256, 0, st>>>((int64_t)m * m, f->As.as<double>(), f->c32.as<float>(),
                                                     f->rs.as<double>(), m, f->red.as<double>());
        FKF_LAUNCHED(ctx);
        k_frob_final<<<1, 32, 0, st>>>(f->red.as<double>(), nrm);
        FKF_LAUNCHED(ctx);
        FKF_CUDA(ctx, cudaMemcpyAsync(&tc_fail, f->rot.ctl.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      } else {
        double* T0 = f->Tm.as<double>();
        FKF_CUDA(ctx, cudaMemcpyAsync(T0, f->As.p, (size_t)m * m * 8, cudaMemcpyDeviceToDevice, st));
        FKF_TRY(gemm_sym_f64(ctx, false, true, m, r, -1.0, HW, nm, HW, nm, 1.0, T0, m));
        FKF_TRY(frob(ctx, (int64_t)m * m, T0, f->rs.as<double>(), m, f->red.as<double>(), nrm));
      }
      FKF_TRY(frob(ctx, (int64_t)m * m, f->At.as<double>(), nullptr, m, f->red.as<double>(), nrm + 1));
    }
    double hv[2] = {1.0, 1.0};
    int hflag = 0, apply_fail = 0;
    if (r > 0) FKF_CUDA(ctx, cudaMemcpyAsync(hv, nrm, 16, cudaMemcpyDeviceToHost, st));
    FKF_CUDA(ctx, cudaMemcpyAsync(&hflag, f->flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    // a tensor-core wait of the H-apply that gave up: stop before G is used
    if (h->tc_err.p) FKF_CUDA(ctx, cudaMemcpyAsync(&apply_fail, h->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    FKF_CUDA(ctx, cudaStreamSynchronize(st));
    if (apply_fail) FKF_TRY(hmat_tc_check(h));
    if (tc_fail) FKF_TRY(tc_gemm_check(ctx, f->rot));
    if (hflag) return set_err(ctx, FKF_EINVAL, "filter_step: H column index outside [0, N)");
    if (r > 0) ratio = hv[1] > 0 ? hv[0] / hv[1] : 0.0;
  }
  const bool kept = r > 0 && ratio <= f->new_tol && !(flags & FKF_STEP_FULL_UPDATE);
  // S = alpha' A + R - HW D HW^T   (D diagonal, or the full r x r weight Df)
  const bool diag = f->diag;
  double* Dfc = f->Df.as<double>();
  if (r > 0) {
    // S -= HWD HW^T (formed beside the H-apply; S is read only through its
    // lower triangle by the blocked Cholesky)
    FKF_CUDA(ctx, cudaStreamWaitEvent(st, f->ev_p, 0));
    k_sub_lower<<<nblk((int64_t)m * m), 256, 0, st>>>(m, f->Pw.as<double>(), m, S, lda_aug);
    FKF_LAUNCHED(ctx);
  }
  if (kept) {
    // ---- basis kept: Sigma+ = alpha' Gamma - W D' W^T with the weight updated
    // in information form, E' = (E^-1 + Q)^-1, E = alpha' I - D (predicted),
    // Q = HW^T R^-1 HW  (Alg. kalmanconstantH with a non-diagonal weight),
    // evaluated in the Woodbury form E' = E - K^T S^-1 K, K = HW E, with the
    // innovation covariance S = alpha' A - HW D HW^T + R (= HW E HW^T + R up to
    // the new_tol residual A - HW HW^T).  Both come out of one Cholesky
    // factorisation of the augmented matrix [[S, K], [K^T, E]] stopped after
    // its first m pivots: the leading block is S's factor L (for the mean and
    // the NLL) and the trailing block the Schur complement E - K^T S^-1 K = E'.
    double* Eaug = S + (int64_t)m * lda_aug;  // rows m.. : [K^T | E]
    k_aug_rows<<<nblk(lda_aug * r), 256, 0, st>>>(m, r, HW, nm, f->HWD.as<double>(), diag ? f->D.as<double>() : nullptr,
                                                 diag ? nullptr : Dfc, alpha1, Eaug, lda_aug);
    FKF_LAUNCHED(ctx);
    FKF_TRY(chol_innovation(f, m + r, m, S, lda_aug, f->ev_schur));
  } else {
    FKF_TRY(chol_innovation(f, m, m, S, lda_aug, nullptr));
  }
  FKF_CUDA(ctx, cudaMemcpyAsync(f->z.p, f->nu.p, m * 8, cudaMemcpyDeviceToDevice, st));
  FKF_TRY(chol_solve_rowlower_f64(ctx, m, S, lda_aug, f->z.as<double>(), 1));
  k_nll<<<1, 256, 0, st>>>(m, f->nu.as<double>(), f->z.as<double>(), S, lda_aug, f->nll.as<double>());
  FKF_LAUNCHED(ctx);
  // mean: s' = s + [W G] [-D (HW^T z); alpha' z]
  if (r > 0) {
    FKF_TRY(gemm_f64(ctx, true, false, r, 1, m, 1.0, HW, nm, f->z.as<double>(), 1, 0.0, f->uz.as<double>(), 1));
    if (diag) {
      k_vmul<<<(int)cdiv(r, 256), 256, 0, st>>>(r, f->D.as<double>(), f->uz.as<double>(), f->dbar.as<double>());
      FKF_LAUNCHED(ctx);
    } else {
      FKF_TRY(gemm_f64(ctx, false, false, r, 1, r, 1.0, Dfc, r, f->uz.as<double>(), 1, 0.0, f->dbar.as<double>(), 1));
    }
  }
  k_mean_coef<T><<<(int)cdiv(nm, 256), 256, 0, st>>>(r, m, nullptr, f->dbar.as<double>(), f->z.as<double>(), alpha1,
                                                     f->vcoef.as<T>());
  FKF_LAUNCHED(ctx);
  k_gemv_add<T><<<(int)cdiv(n * 32, 256), 256, 0, st>>>(n, nm, Wc, ld, f->vcoef.as<T>(), f->s_hat.as<double>(),
                                                       f->s_new.as<double>());
  FKF_LAUNCHED(ctx);
  FKF_CUDA(ctx, cudaEventRecord(f->ev[3], st));
  if (kept) {
    double* Dn2 = f->Dfn.as<double>();
    // D' = alpha' I - E' (E' = trailing r x r block of the augmented factorisation,
    // formed beside the solve for z and the mean update)
    FKF_CUDA(ctx, cudaStreamWaitEvent(st, f->ev_schur, 0));
    k_lincomb_ld<<<nblk((int64_t)r * r), 256, 0, st>>>(r, -1.0, S + (int64_t)m * lda_aug + m, lda_aug, alpha1, Dn2);
    FKF_LAUNCHED(ctx);
    for (int e = 4; e < 7; e++) FKF_CUDA(ctx, cudaEventRecord(f->ev[e], st));
    double nll = 0;
    FKF_CUDA(ctx, cudaMemcpyAsync(&nll, f->nll.p, 8, cudaMemcpyDeviceToHost, st));
    FKF_CUDA(ctx, cudaStreamSynchronize(st));
    FKF_CUDA(ctx, cudaGetLastError());
    FKF_TRY(hmat_tc_check(h));
    std::swap(f->s_hat.p, f->s_new.p);
    std::swap(f->Df.p, f->Dfn.p);
    f->diag = false;
    f->alpha = alpha1;
    f->k++;
    f->last_path = reuse ? 3 : 1;
    // this step's products stay valid for the next step with the same H and R
    f->products_valid = bc == 0.0;
    if (!reuse) {
      f->prev_m = m;
      f->prev_nnz = nnz;
      f->prev_rp = rp;
      f->prev_rdiag = rdiag;
      if (allow_fixed && !on_dev) {
        f->prev_col.assign(col_in, col_in + nnz);
        f->prev_val.assign(val_in, val_in + nnz);
      } else {
        f->prev_col.clear();
        f->prev_val.clear();
      }
    }
    if (nll_out && !(flags & FKF_STEP_SKIP_MEAN_SYNC)) *nll_out = nll;
    for (int i = 0; i < 6; i++) {
      float ms = 0;
      cudaEventElapsedTime(&ms, f->ev[i], f->ev[i + 1]);
      f->phase_ms[i] = ms;
    }
    return FKF_OK;
  }
  // ---- S3: data-space GEP  R^-1/2 A R^-1/2 = Q diag(a) Q^T
  std::vector<double> a_h, thM_h;
  int mlam = 0;
  double* C = f->C.as<double>();
  if (f->rk > 0) {
    FKF_TRY(randomized_gep(f, m, &mlam));
  } else {
    FKF_TRY(eigh_f64(ctx, m, f->At.as<double>(), f->a.as<double>(), a_h, f->eigws));
    const double amax = a_h.empty() ? 0.0 : a_h.back();
    for (int i = m - 1; i >= 0; i--)
      if (amax > 0 && a_h[i] > f->gep_tol * amax) mlam++;
      else break;
    if (mlam > 0) {
      k_build_C<<<nblk((int64_t)m * mlam), 256, 0, st>>>(m, mlam, f->At.as<double>(), f->a.as<double>(),
                                                         f->rs.as<double>(), C, f->lam.as<double>());
      FKF_LAUNCHED(ctx);
    }
  }
  FKF_CUDA(ctx, cudaEventRecord(f->ev[4], st));
  // ---- S4: Gamma^-1-orthonormalisation of U = G C against W (data space)
  double* P = f->P.as<double>();
  int mp = mlam, t_eig = 0;
  double t_lmax = r > 0 ? 0.0 : 1.0;  // without W, T = I
  if (r > 0 && mlam > 0) {
    FKF_TRY(gemm_merge(ctx, true, false, r, mlam, m, 1.0, HW, nm, C, mlam, 0.0, P, mlam));
    double* Tm = f->Tm.as<double>();
    FKF_TRY(gemm_merge(ctx, true, false, mlam, mlam, r, -1.0, P, mlam, P, mlam, 0.0, Tm, mlam));
    k_add_identity<<<(int)cdiv(mlam, 256), 256, 0, st>>>(mlam, Tm, mlam, 1.0);
    FKF_LAUNCHED(ctx);
    // every eigenvalue of T is bounded by ||T||_F: below the threshold there
    // is nothing new to factor
    FKF_TRY(frob(ctx, (int64_t)mlam * mlam, Tm, nullptr, mlam, f->red.as<double>(), f->nll.as<double>() + 1));
    double tfrob = 0;
    FKF_CUDA(ctx, cudaMemcpyAsync(&tfrob, f->nll.as<double>() + 1, 8, cudaMemcpyDeviceToHost, st));
    FKF_CUDA(ctx, cudaStreamSynchronize(st));
    mp = 0;
    t_lmax = tfrob;
    const bool factor_t = tfrob > f->orth_tol;
    if (factor_t) {
      // rank-revealing pivoted Cholesky T ~= Lp Lp^T (Lp = Pi L, mlam x mp), pivots above
      // orth_tol.  With Y = Lp (Lp^T Lp)^-1 the new directions V = (U - W P) Y are
      // Gamma^-1-orthonormal (Y^T T Y = I) and U - W P = V Lp^T up to the dropped
      // pivots, so Po = Lp^T and F1 = Y take the places of Theta^1/2 Q_T^T and
      // Q_T Theta^-1/2 of an eigendecomposition.
      double* Lp = f->Lpv.as<double>();
      FKF_TRY(pchol_f64(ctx, mlam, Tm, mlam, f->orth_tol, mlam, Lp, mlam, f->pcws, &mp));
      if (mp > 0) {
        k_transpose<<<nblk((int64_t)mp * mlam), 256, 0, st>>>(mp, mlam, Lp, mlam, f->Po.as<double>(), mlam);
        FKF_LAUNCHED(ctx);
        double* Gm = f->Gm.as<double>();
        double* F1 = f->F1c.as<double>();  // mlam x mp
        FKF_TRY(gemm_f64(ctx, true, false, mp, mp, mlam, 1.0, Lp, mlam, Lp, mlam, 0.0, Gm, mp));
        FKF_CUDA(ctx, cudaMemcpy2DAsync(F1, (size_t)mp * 8, Lp, (size_t)mlam * 8, (size_t)mp * 8, mlam,
                                        cudaMemcpyDeviceToDevice, st));
        FKF_TRY(chol_f64(ctx, mp, Gm, f->cholws));
        // column-major, F1 is the mp x mlam right-hand side Lp^T: F1 <- Lp (Lp^T Lp)^-1
        FKF_TRY(chol_solve_f64(ctx, mp, Gm, F1, mlam));
        k_transpose<<<nblk((int64_t)mp * mlam), 256, 0, st>>>(mp, mlam, F1, mp, f->F1t.as<double>(), mlam);
        FKF_LAUNCHED(ctx);
      }
    }
    t_eig = factor_t ? 1 : 0;
  } else if (mlam > 0) {
    k_identity<<<nblk((int64_t)mlam * mlam), 256, 0, st>>>(mlam, f->Po.as<double>(), mlam);
    FKF_LAUNCHED(ctx);
    k_identity<<<nblk((int64_t)mlam * mlam), 256, 0, st>>>(mlam, f->F1t.as<double>(), mlam);
    FKF_LAUNCHED(ctx);
  }
  // ---- S5: merge  M = diag(Dbar, 0) + Z Lam Z^T, Z = [P; Po]
  const int nM = r + mp;
  double* M = f->M.as<double>();
  int rnew = 0, meig = 0;
  if (nM > 0) {
    if (mlam > 0) {
      k_stack_scale<<<nblk((int64_t)nM * mlam), 256, 0, st>>>(r, mp, mlam, P, f->Po.as<double>(), f->lam.as<double>(),
                                                            f->ZL.as<double>());
      FKF_LAUNCHED(ctx);
    }
    // (the eigensolver symmetrises M: the tensor-core product's rounding asymmetry is harmless)
    if (ctx->fp64_tc && (double)nM * nM * mlam >= 1e8)
      FKF_TRY(gemm_f64_tc(ctx, false, true, nM, nM, mlam, 1.0, f->ZL.as<double>(), mlam, f->ZL.as<double>(), mlam,
                          0.0, M, nM));
    else
      FKF_TRY(gemm_sym_f64(ctx, false, true, nM, mlam, 1.0, f->ZL.as<double>(), mlam, f->ZL.as<double>(), mlam, 0.0,
                           M, nM));
    if (r > 0 && diag) {
      k_add_dbar<<<(int)cdiv(r, 256), 256, 0, st>>>(r, f->D.as<double>(), alpha1, M, nM);
      FKF_LAUNCHED(ctx);
    } else if (r > 0) {
      // full weight: Dbar = D (alpha' I - D)^-1 / alpha' = (alpha' I - D)^-1 - I / alpha'
      const int64_t rr = (int64_t)r * r;
      double* Ep = f->Ep.as<double>();
      k_lincomb<<<nblk(rr), 256, 0, st>>>(r, -1.0, Dfc, 0.0, nullptr, alpha1, Ep);
      FKF_LAUNCHED(ctx);
      FKF_TRY(chol_f64(ctx, r, Ep, f->cholws));
      k_identity<<<nblk(rr), 256, 0, st>>>(r, f->Qm.as<double>(), r);
      FKF_LAUNCHED(ctx);
      FKF_TRY(chol_solve_f64(ctx, r, Ep, f->Qm.as<double>(), r));
      k_add_block<<<nblk(rr), 256, 0, st>>>(r, f->Qm.as<double>(), -1.0 / alpha1, M, nM);
      FKF_LAUNCHED(ctx);
    }
    // only the r_max largest eigenpairs can be kept
    FKF_TRY(eigh_top_f64(ctx, nM, rmax, M, f->thM.as<double>(), thM_h, f->eigws, &meig));
    const double tmax = thM_h.empty() ? 0.0 : thM_h.back();
    for (int i = meig - 1; i >= 0 && rnew < rmax; i--)
      if (tmax > 0 && thM_h[i] > f->trunc_tol * tmax && thM_h[i] > 0) rnew++;
      else break;
  }
  double* Dn = f->Dn.as<double>();
  double* E = f->E.as<double>();
  if (rnew > 0) {
    k_new_D<<<(int)cdiv(rnew, 256), 256, 0, st>>>(meig, rnew, f->thM.as<double>(), alpha1, Dn);
    FKF_LAUNCHED(ctx);
    // Sk (rnew x nM): rows = kept eigenvectors of M (descending)
    k_top_rows<<<nblk((int64_t)rnew * nM), 256, 0, st>>>(nM, rnew, M, f->thM.as<double>(), 2, f->Sk.as<double>(), nM,
                                                        meig);
    FKF_LAUNCHED(ctx);
    double* EW = E;                       // r x rnew
    double* EG = E + (int64_t)r * rnew;   // m x rnew
    double* J = f->J.as<double>();        // mlam x rnew
    if (mp > 0) {
      // J = F1 S2 with F1^T (mp x mlam) and S2^T = Sk[:, r:r+mp]
      FKF_TRY(gemm_merge(ctx, true, true, mlam, rnew, mp, 1.0, f->F1t.as<double>(), mlam, f->Sk.as<double>() + r,
                         nM, 0.0, J, rnew));
      FKF_TRY(gemm_merge(ctx, false, false, m, rnew, mlam, 1.0, C, mlam, J, rnew, 0.0, EG, rnew));
    } else {
      FKF_CUDA(ctx, cudaMemsetAsync(EG, 0, (size_t)m * rnew * 8, st));
    }
    if (r > 0) {
      k_transpose<<<nblk((int64_t)r * rnew), 256, 0, st>>>(r, rnew, f->Sk.as<double>(), nM, EW, rnew);
      FKF_LAUNCHED(ctx);
      if (mp > 0) FKF_TRY(gemm_merge(ctx, false, false, r, rnew, mlam, -1.0, P, mlam, J, rnew, 1.0, EW, rnew));
    }
  }
  FKF_CUDA(ctx, cudaEventRecord(f->ev[5], st));
  // ---- S6: rotation  W' = [W G] E,  X' = X E_W + H^T E_G
  T* Wn = WGn + (rmax - rnew);
  if (rnew > 0) {
    const T* Et;
    if (sizeof(T) == 8) {
      Et = reinterpret_cast<const T*>(E);
    } else {
      k_cast<T><<<nblk((int64_t)nm * rnew), 256, 0, st>>>((int64_t)nm * rnew, E, f->Ecast.as<T>());
      FKF_LAUNCHED(ctx);
      Et = f->Ecast.as<T>();
    }
    if (sizeof(T) == 4) {
      // both products on the tensor cores in one launch (they share E's split)
      const TcGemmProblem pr[2] = {
          {reinterpret_cast<const float*>(Wc), ld, n, (int)nm, reinterpret_cast<float*>(Wn), ld},
          {reinterpret_cast<const float*>(Xc), rmax, n, r, reinterpret_cast<float*>(Xn), rmax}};
      FKF_TRY(tc_gemm_f32(ctx, pr, 2, reinterpret_cast<const float*>(Et), rnew, nm, rnew, f->rot));
    } else {
      FKF_TRY(gemm_T<T>(ctx, false, false, n, rnew, nm, 1.0, Wc, ld, Et, rnew, 0.0, Wn, ld));
      FKF_TRY(gemm_T<T>(ctx, false, false, n, rnew, r, 1.0, Xc, rmax, Et, rnew, 0.0, Xn, rmax));
    }
    k_csc_spmm<T><<<(int)cdiv(n * 32, 256), 256, 0, st>>>(n, f->colptr.as<int64_t>(), f->crow.as<int>(),
                                                          f->cval.as<double>(), E + (int64_t)r * rnew, rnew, Xn, rmax);
    FKF_LAUNCHED(ctx);
  }
  FKF_CUDA(ctx, cudaEventRecord(f->ev[6], st));
  double nll = 0;
  FKF_CUDA(ctx, cudaMemcpyAsync(&nll, f->nll.p, 8, cudaMemcpyDeviceToHost, st));
  FKF_CUDA(ctx, cudaStreamSynchronize(st));
  FKF_CUDA(ctx, cudaGetLastError());
  FKF_TRY(hmat_tc_check(h));
  FKF_TRY(tc_gemm_check(ctx, f->rot));
  FKF_TRY(gemm_f64_tc_check(ctx));
  // ---- commit
  std::swap(f->s_hat.p, f->s_new.p);
  std::swap(f->D.p, f->Dn.p);
  f->cur = 1 - f->cur;
  f->r = rnew;
  f->alpha = alpha1;
  f->k++;
  f->diag = true;
  f->last_path = 0;
  f->gep_rank = mlam;
  f->new_dirs = mp;
  f->t_eig = t_eig;
  f->t_lmax = t_lmax;
  if (nll_out && !(flags & FKF_STEP_SKIP_MEAN_SYNC)) *nll_out = nll;
  for (int i = 0; i < 6; i++) {
    float ms = 0;
    cudaEventElapsedTime(&ms, f->ev[i], f->ev[i + 1]);
    f->phase_ms[i] = ms;
  }
  return FKF_OK;
}

fkf_status filter_refresh(fkf_filter* f);

fkf_status filter_step(fkf_filter* f, const double* y, int m, const int64_t* rowptr, const int32_t* col,
                       const double* val, const double* R, double r_scalar, int flags, double* nll_out,
                       double boxcox_a) {
  if (!(boxcox_a >= 0.0) || !std::isfinite(boxcox_a))
    return set_err(f->ctx, FKF_EINVAL, "filter_step: Box-Cox parameter must be finite and >= 0 (0: linear)");
  Fp64TcScope tc(f->ctx, f->w == 4);
  const fkf_status st =
      f->w == 8 ? step_impl<double>(f, y, m, rowptr, col, val, R, r_scalar, flags, nll_out, boxcox_a)
                : step_impl<float>(f, y, m, rowptr, col, val, R, r_scalar, flags, nll_out, boxcox_a);
  if (st != FKF_OK) return st;
  // S10: the scheduled refresh W <- Gamma_H X (after the step has committed;
  // the refresh is transactional on its own and keeps the covariance)
  if (f->refresh_every > 0 && f->k % f->refresh_every == 0 && f->r > 0) return filter_refresh(f);
  return FKF_OK;
}

fkf_status filter_set_refresh(fkf_filter* f, int every) {
  if (every < 0) return set_err(f->ctx, FKF_EINVAL, "set_refresh: every >= 0 required");
  f->refresh_every = every;
  return FKF_OK;
}

// Bring the state to the paper's form (Eq. sigmakk with D diagonal): with the
// full weight Df = V diag(d) V^T (V orthogonal), W <- W V and X <- X V keep
// X^T W = I and Sigma unchanged.
template <typename T>
static fkf_status canonicalize_impl(fkf_filter* f) {
  fkf_ctx* ctx = f->ctx;
  cudaStream_t st = ctx->stream;
  const int r = f->r, rmax = f->r_max;
  const int64_t n = f->n, ld = f->ldwg, rr = (int64_t)r * r;
  double* Vt = f->Qm.as<double>();
  FKF_CUDA(ctx, cudaMemcpyAsync(Vt, f->Df.p, rr * 8, cudaMemcpyDeviceToDevice, st));
  std::vector<double> w_h;
  FKF_TRY(eigh_f64(ctx, r, Vt, f->thM.as<double>(), w_h, f->eigws));
  double* E = f->E.as<double>();
  k_transpose<<<nblk(rr), 256, 0, st>>>(r, r, Vt, r, E, r);  // E = V (columns = eigenvectors)
  FKF_LAUNCHED(ctx);
  const T* Et;
  if (sizeof(T) == 8) {
    Et = reinterpret_cast<const T*>(E);
  } else {
    k_cast<T><<<nblk(rr), 256, 0, st>>>(rr, E, f->Ecast.as<T>());
    FKF_LAUNCHED(ctx);
    Et = f->Ecast.as<T>();
  }
  const T* Wc = f->WG[f->cur].as<T>() + (rmax - r);
  T* Wn = f->WG[1 - f->cur].as<T>() + (rmax - r);
  FKF_TRY(gemm_T<T>(ctx, false, false, n, r, r, 1.0, Wc, ld, Et, r, 0.0, Wn, ld));
  FKF_TRY(gemm_T<T>(ctx, false, false, n, r, r, 1.0, f->Xb[f->cur].as<T>(), rmax, Et, r, 0.0,
                    f->Xb[1 - f->cur].as<T>(), rmax));
  FKF_CUDA(ctx, cudaMemcpyAsync(f->D.p, f->thM.p, r * 8, cudaMemcpyDeviceToDevice, st));
  FKF_CUDA(ctx, cudaStreamSynchronize(st));
  FKF_CUDA(ctx, cudaGetLastError());
  f->cur = 1 - f->cur;
  f->diag = true;
  f->products_valid = false;
  return FKF_OK;
}

static fkf_status canonicalize(fkf_filter* f) {
  if (f->diag) return FKF_OK;
  if (f->r == 0) {
    f->diag = true;
    return FKF_OK;
  }
  Fp64TcScope tc(f->ctx, f->w == 4);
  if (f->w == 8) return canonicalize_impl<double>(f);
  return canonicalize_impl<float>(f);
}

fkf_status filter_get(fkf_filter* f, double* s_hat, double* alpha, int* r, double* D, void* W_dev, int64_t ldw) {
  fkf_ctx* ctx = f->ctx;
  if (D || W_dev) FKF_TRY(canonicalize(f));
  if (alpha) *alpha = f->alpha;
  if (r) *r = f->r;
  if (s_hat) {
    std::vector<double> sc(f->n);
    FKF_CUDA(ctx, cudaMemcpyAsync(sc.data(), f->s_hat.p, f->n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int64_t i = 0; i < f->n; i++) s_hat[f->h->perm[i]] = sc[i];
  }
  if (D && f->r > 0) {
    FKF_CUDA(ctx, cudaMemcpyAsync(D, f->D.p, f->r * 8, cudaMemcpyDeviceToHost, ctx->stream));
    FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (W_dev && f->r > 0) {
    if (ldw < f->r) return set_err(ctx, FKF_EINVAL, "filter_get: ldw < r");
    const char* Wc = f->WG[f->cur].as<char>() + (f->r_max - f->r) * f->w;
    FKF_TRY(hmat_permute_rows(f->h, Wc, f->ldwg, f->h->iperm_d.as<int64_t>(), W_dev, ldw, f->n, f->r));
    FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return FKF_OK;
}

fkf_status filter_variance(fkf_filter* f, double* var_dev) {
  fkf_ctx* ctx = f->ctx;
  FKF_TRY(canonicalize(f));
  const int64_t n = f->n;
  const double as2 = f->alpha * f->h->kernel.sigma2;
  const char* Wc = f->WG[f->cur].as<char>() + (f->r_max - f->r) * f->w;
  if (f->w == 8)
    k_variance<double><<<(int)cdiv(n * 32, 256), 256, 0, ctx->stream>>>(n, f->r, (const double*)Wc, f->ldwg,
                                                                         f->D.as<double>(), as2, f->h->perm_d.as<int64_t>(), var_dev);
  else
    k_variance<float><<<(int)cdiv(n * 32, 256), 256, 0, ctx->stream>>>(n, f->r, (const float*)Wc, f->ldwg,
                                                                        f->D.as<double>(), as2, f->h->perm_d.as<int64_t>(), var_dev);
  FKF_LAUNCHED(ctx);
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return FKF_OK;
}

template <typename T>
static fkf_status realization_impl(fkf_filter* f, const double* a_dev, int ns, double* out_dev) {
  fkf_ctx* ctx = f->ctx;
  cudaStream_t st = ctx->stream;
  const int64_t n = f->n;
  const int r = f->r;
  FKF_TRY(dev_alloc(ctx, f->tmp1, (size_t)n * ns * sizeof(T)));
  FKF_TRY(dev_alloc(ctx, f->tmp2, (size_t)n * ns * sizeof(T)));
  FKF_TRY(dev_alloc(ctx, f->tmp3, (size_t)std::max(r, 1) * ns * 8 * 2));
  T* ac = f->tmp1.as<T>();
  T* t = f->tmp2.as<T>();
  k_gather_cast<T><<<nblk(n * ns), 256, 0, st>>>(n, ns, a_dev, f->h->perm_d.as<int64_t>(), ac);
  FKF_LAUNCHED(ctx);
  const T* Wc = f->WG[f->cur].as<T>() + (f->r_max - r);
  const T* Xc = f->Xb[f->cur].as<T>();
  if (r > 0) {
    double* Y = f->tmp3.as<double>();
    double* Ys = Y + (int64_t)r * ns;
    FKF_TRY(gram_T(ctx, f->w, r, ns, n, Xc, f->r_max, ac, ns, Y, ns, f->gramws));  // X^T a
    k_sig_rows<<<nblk((int64_t)r * ns), 256, 0, st>>>(r, ns, Y, f->D.as<double>(), f->alpha, Ys);
    FKF_LAUNCHED(ctx);
    T* Yt = reinterpret_cast<T*>(Y);  // reuse: cast Ys into the first half
    k_cast<T><<<nblk((int64_t)r * ns), 256, 0, st>>>((int64_t)r * ns, Ys, Yt);
    FKF_LAUNCHED(ctx);
    FKF_TRY(gemm_T<T>(ctx, false, false, n, ns, r, 1.0, Wc, f->ldwg, Yt, ns, 0.0, t, ns));
  } else {
    FKF_CUDA(ctx, cudaMemsetAsync(t, 0, (size_t)n * ns * sizeof(T), st));
  }
  k_realize<T><<<nblk(n * ns), 256, 0, st>>>(n, ns, f->s_hat.as<double>(), ac, t, std::sqrt(f->alpha),
                                              f->h->perm_d.as<int64_t>(), out_dev);
  FKF_LAUNCHED(ctx);
  FKF_CUDA(ctx, cudaStreamSynchronize(st));
  return FKF_OK;
}

fkf_status filter_realization(fkf_filter* f, const double* a_dev, int ns, double* out_dev) {
  if (ns < 1) return set_err(f->ctx, FKF_EINVAL, "conditional_realization: ns >= 1 required");
  if (f->alpha <= 0) return set_err(f->ctx, FKF_ESTATE, "conditional_realization: alpha must be > 0 (run a step)");
  FKF_TRY(canonicalize(f));
  if (f->w == 8) return realization_impl<double>(f, a_dev, ns, out_dev);
  return realization_impl<float>(f, a_dev, ns, out_dev);
}

fkf_status filter_uncertainty(fkf_filter* f, double* ent, double* tr) {
  fkf_ctx* ctx = f->ctx;
  FKF_TRY(canonicalize(f));
  const int r = f->r;
  std::vector<double> d(r);
  if (r > 0) {
    FKF_CUDA(ctx, cudaMemcpyAsync(d.data(), f->D.p, r * 8, cudaMemcpyDeviceToHost, ctx->stream));
    FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (ent) {
    if (f->alpha <= 0) return set_err(ctx, FKF_ESTATE, "relative entropy needs alpha > 0");
    double s = (double)f->n * std::log(f->alpha);
    for (int j = 0; j < r; j++) s += std::log1p(-d[j] / f->alpha);
    *ent = 0.5 * s;
  }
  if (tr) {
    double t = f->alpha * (double)f->n * f->h->kernel.sigma2;
    if (r > 0) {
      const int64_t n = f->n, chunk = 4096, nz = cdiv(n, chunk);
      FKF_TRY(dev_alloc(ctx, f->tmp3, (size_t)nz * r * 8));
      const char* Wc = f->WG[f->cur].as<char>() + (f->r_max - r) * f->w;
      dim3 grid((unsigned)cdiv(r, 256), (unsigned)nz);
      if (f->w == 8)
        k_colsq_part<double><<<grid, 256, 0, ctx->stream>>>(n, r, (const double*)Wc, f->ldwg, chunk, f->tmp3.as<double>());
      else
        k_colsq_part<float><<<grid, 256, 0, ctx->stream>>>(n, r, (const float*)Wc, f->ldwg, chunk, f->tmp3.as<double>());
      FKF_LAUNCHED(ctx);
      std::vector<double> part((size_t)nz * r);
      FKF_CUDA(ctx, cudaMemcpyAsync(part.data(), f->tmp3.p, part.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
      FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      for (int j = 0; j < r; j++) {
        double s = 0;
        for (int64_t z = 0; z < nz; z++) s += part[z * r + j];
        t -= d[j] * s;
      }
    }
    *tr = t;
  }
  return FKF_OK;
}

fkf_status filter_orthonormality(fkf_filter* f, double* err) {
  fkf_ctx* ctx = f->ctx;
  const int r = f->r;
  if (r == 0) {
    *err = 0;
    return FKF_OK;
  }
  FKF_TRY(dev_alloc(ctx, f->tmp3, (size_t)r * r * 8));
  const char* Wc = f->WG[f->cur].as<char>() + (f->r_max - r) * f->w;
  FKF_TRY(gram_T(ctx, f->w, r, r, f->n, f->Xb[f->cur].p, f->r_max, Wc, f->ldwg, f->tmp3.as<double>(), r, f->gramws));
  std::vector<double> g((size_t)r * r);
  FKF_CUDA(ctx, cudaMemcpyAsync(g.data(), f->tmp3.p, g.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double e = 0;
  for (int i = 0; i < r; i++)
    for (int j = 0; j < r; j++) e = std::max(e, std::fabs(g[(size_t)i * r + j] - (i == j ? 1.0 : 0.0)));
  *err = e;
  return FKF_OK;
}

// W <- Gamma_H X, then re-orthonormalise: with Q = X^T W = V th V^T,
// W~ = W Q^-1/2, and the low-rank term W D W^T = W~ (Q^1/2 D Q^1/2) W~^T is
// re-diagonalised: Q^1/2 D Q^1/2 = S D' S^T;  E = Q^-1/2 S.
template <typename T>
static fkf_status refresh_impl(fkf_filter* f) {
  fkf_ctx* ctx = f->ctx;
  cudaStream_t st = ctx->stream;
  const int r = f->r, rmax = f->r_max;
  if (r == 0) return FKF_OK;
  const int64_t n = f->n, ld = f->ldwg, rr = (int64_t)r * r;
  T* Xc = f->Xb[f->cur].as<T>();
  // Gamma_H X goes to the G columns of the spare buffer when r fits in them,
  // else to a scratch of its own (N x r, kept for later refreshes)
  T* Wtmp = f->WG[1 - f->cur].as<T>() + rmax;
  int64_t ldt = ld;
  if (r > f->m_max) {
    FKF_TRY(dev_alloc(ctx, f->refw, (size_t)n * r * sizeof(T)));
    Wtmp = f->refw.as<T>();
    ldt = r;
  }
  FKF_TRY(hmat_apply_clustered(f->h, Xc, rmax, Wtmp, ldt, r));
  FKF_TRY(dev_alloc(ctx, f->tmp3, (size_t)rr * 8 * 6));
  double* Q = f->tmp3.as<double>();
  double* B1 = Q + rr;
  double* Bm1 = B1 + rr;
  double* Qh = Bm1 + rr;
  double* Qmh = Qh + rr;
  double* E = Qmh + rr;
  FKF_TRY(gram_T(ctx, f->w, r, r, n, Xc, rmax, Wtmp, ldt, Q, r, f->gramws));
  k_symmetrize<<<nblk(rr), 256, 0, st>>>(r, Q);
  FKF_LAUNCHED(ctx);
  std::vector<double> w_h;
  double* thr = f->thM.as<double>();  // r eigenvalues (r <= r_max)
  FKF_TRY(eigh_f64(ctx, r, Q, thr, w_h, f->eigws));  // Q -> Vt
  if (!(w_h[0] > 0)) return set_err(ctx, FKF_ENOTSPD, "refresh: X^T Gamma X not positive definite");
  k_top_rows<<<nblk(rr), 256, 0, st>>>(r, r, Q, thr, 0, B1, r);   // diag(sqrt th) Vt
  FKF_LAUNCHED(ctx);
  k_top_rows<<<nblk(rr), 256, 0, st>>>(r, r, Q, thr, 1, Bm1, r);  // diag(1/sqrt th) Vt
  FKF_LAUNCHED(ctx);
  k_top_rows<<<nblk(rr), 256, 0, st>>>(r, r, Q, thr, 2, E, r);    // Vt (same order)
  FKF_LAUNCHED(ctx);
  FKF_TRY(gemm_f64(ctx, true, false, r, r, r, 1.0, E, r, B1, r, 0.0, Qh, r));    // Q^1/2
  FKF_TRY(gemm_f64(ctx, true, false, r, r, r, 1.0, E, r, Bm1, r, 0.0, Qmh, r));  // Q^-1/2
  // Mx = Q^1/2 D Q^1/2
  k_scale_cols<<<nblk(rr), 256, 0, st>>>(r, r, Qh, r, f->D.as<double>(), B1);
  FKF_LAUNCHED(ctx);
  FKF_TRY(gemm_f64(ctx, false, false, r, r, r, 1.0, B1, r, Qh, r, 0.0, Q, r));
  k_symmetrize<<<nblk(rr), 256, 0, st>>>(r, Q);
  FKF_LAUNCHED(ctx);
  FKF_TRY(eigh_f64(ctx, r, Q, thr, w_h, f->eigws));
  k_top_rows<<<nblk(rr), 256, 0, st>>>(r, r, Q, thr, 2, f->Sk.as<double>(), r);  // S^T (desc)
  FKF_LAUNCHED(ctx);
  FKF_TRY(gemm_f64(ctx, false, true, r, r, r, 1.0, Qmh, r, f->Sk.as<double>(), r, 0.0, E, r));  // E = Q^-1/2 S
  std::vector<double> dn(r);
  for (int q = 0; q < r; q++) dn[q] = std::max(0.0, w_h[r - 1 - q]);
  FKF_CUDA(ctx, cudaMemcpyAsync(f->Dn.p, dn.data(), r * 8, cudaMemcpyHostToDevice, st));
  const T* Et;
  if (sizeof(T) == 8) {
    Et = reinterpret_cast<const T*>(E);
  } else {
    k_cast<T><<<nblk(rr), 256, 0, st>>>(rr, E, f->Ecast.as<T>());
    FKF_LAUNCHED(ctx);
    Et = f->Ecast.as<T>();
  }
  T* Wn = f->WG[1 - f->cur].as<T>() + (rmax - r);  // columns [rmax - r, rmax): disjoint from Wtmp
  FKF_TRY(gemm_T<T>(ctx, false, false, n, r, r, 1.0, Wtmp, ldt, Et, r, 0.0, Wn, ld));
  FKF_TRY(gemm_T<T>(ctx, false, false, n, r, r, 1.0, Xc, rmax, Et, r, 0.0, f->Xb[1 - f->cur].as<T>(), rmax));
  FKF_CUDA(ctx, cudaStreamSynchronize(st));
  FKF_CUDA(ctx, cudaGetLastError());
  std::swap(f->D.p, f->Dn.p);
  f->cur = 1 - f->cur;
  f->products_valid = false;
  return FKF_OK;
}

fkf_status filter_refresh(fkf_filter* f) {
  Fp64TcScope tc(f->ctx, f->w == 4);
  FKF_TRY(canonicalize(f));
  if (f->w == 8) return refresh_impl<double>(f);
  return refresh_impl<float>(f);
}

struct CkptHeader {
  char magic[8];
  int64_t n, k;
  double alpha;
  int32_t r, w;
};

fkf_status filter_checkpoint(fkf_filter* f, const char* path) {
  fkf_ctx* ctx = f->ctx;
  FKF_TRY(canonicalize(f));
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return set_err(ctx, FKF_EINVAL, "checkpoint: cannot open %s", path);
  CkptHeader hd{};
  std::memcpy(hd.magic, "FKFCKPT1", 8);
  hd.n = f->n;
  hd.k = f->k;
  hd.alpha = f->alpha;
  hd.r = f->r;
  hd.w = (int32_t)f->w;
  const int64_t n = f->n, r = f->r;
  std::vector<char> buf((size_t)std::max<int64_t>(n * 8, n * r * (int64_t)f->w));
  bool ok = std::fwrite(&hd, sizeof(hd), 1, fp) == 1;
  auto put_dev = [&](const void* src, size_t bytes, int64_t rows, int64_t rowbytes, int64_t ldbytes) -> fkf_status {
    // rows of rowbytes with stride ldbytes
    if (cudaMemcpy2D(buf.data(), rowbytes, src, ldbytes, rowbytes, rows, cudaMemcpyDeviceToHost) != cudaSuccess)
      return set_err(ctx, FKF_ECUDA, "checkpoint copy");
    ok = ok && std::fwrite(buf.data(), 1, bytes, fp) == bytes;
    return FKF_OK;
  };
  fkf_status s = put_dev(f->s_hat.p, n * 8, 1, n * 8, n * 8);
  if (s == FKF_OK && r > 0) s = put_dev(f->D.p, r * 8, 1, r * 8, r * 8);
  if (s == FKF_OK && r > 0)
    s = put_dev(f->WG[f->cur].as<char>() + (f->r_max - r) * f->w, n * r * f->w, n, r * f->w, f->ldwg * f->w);
  if (s == FKF_OK && r > 0) s = put_dev(f->Xb[f->cur].p, n * r * f->w, n, r * f->w, f->r_max * f->w);
  std::fclose(fp);
  if (s != FKF_OK) return s;
  if (!ok) return set_err(ctx, FKF_EINVAL, "checkpoint: write failed");
  return FKF_OK;
}

fkf_status filter_restore(fkf_filter* f, const char* path) {
  fkf_ctx* ctx = f->ctx;
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return set_err(ctx, FKF_EINVAL, "restore: cannot open %s", path);
  CkptHeader hd{};
  bool ok = std::fread(&hd, sizeof(hd), 1, fp) == 1 && std::memcmp(hd.magic, "FKFCKPT1", 8) == 0;
  if (!ok || hd.n != f->n || hd.w != (int32_t)f->w || hd.r < 0 || hd.r > f->r_max) {
    std::fclose(fp);
    return set_err(ctx, FKF_EINVAL, "restore: incompatible checkpoint %s", path);
  }
  const int64_t n = f->n, r = hd.r;
  std::vector<char> buf((size_t)std::max<int64_t>(n * 8, n * r * (int64_t)f->w));
  auto get_dev = [&](void* dst, size_t bytes, int64_t rows, int64_t rowbytes, int64_t ldbytes) -> fkf_status {
    if (std::fread(buf.data(), 1, bytes, fp) != bytes) return set_err(ctx, FKF_EINVAL, "restore: truncated file");
    if (cudaMemcpy2D(dst, ldbytes, buf.data(), rowbytes, rowbytes, rows, cudaMemcpyHostToDevice) != cudaSuccess)
      return set_err(ctx, FKF_ECUDA, "restore copy");
    return FKF_OK;
  };
  const int nb = 1 - f->cur;  // write into the spare buffers, then swap (transactional)
  fkf_status s = get_dev(f->s_new.p, n * 8, 1, n * 8, n * 8);
  if (s == FKF_OK && r > 0) s = get_dev(f->Dn.p, r * 8, 1, r * 8, r * 8);
  if (s == FKF_OK && r > 0)
    s = get_dev(f->WG[nb].as<char>() + (f->r_max - r) * f->w, n * r * f->w, n, r * f->w, f->ldwg * f->w);
  if (s == FKF_OK && r > 0) s = get_dev(f->Xb[nb].p, n * r * f->w, n, r * f->w, f->r_max * f->w);
  std::fclose(fp);
  if (s != FKF_OK) return s;
  std::swap(f->s_hat.p, f->s_new.p);
  std::swap(f->D.p, f->Dn.p);
  f->cur = nb;
  f->r = (int)r;
  f->k = hd.k;
  f->alpha = hd.alpha;
  f->diag = true;
  f->products_valid = false;
  return FKF_OK;
}

fkf_status filter_set_tolerances(fkf_filter* f, double gep_tol, double orth_tol, double trunc_tol) {
  if (!(gep_tol >= 0 && gep_tol < 1) || !(orth_tol >= 0 && orth_tol < 1) || !(trunc_tol >= 0 && trunc_tol < 1))
    return set_err(f->ctx, FKF_EINVAL, "set_tolerances: each tolerance must be in [0, 1)");
  f->gep_tol = gep_tol;
  f->orth_tol = orth_tol;
  f->trunc_tol = trunc_tol;
  return FKF_OK;
}

fkf_status filter_phase_times(fkf_filter* f, double* ms6) {
  for (int i = 0; i < 6; i++) ms6[i] = f->phase_ms[i];
  return FKF_OK;
}

fkf_ctx* filter_ctx(fkf_filter* f) { return f->ctx; }

void filter_stats(const fkf_filter* f, fkf_filter_stats* s) {
  s->k = f->k;
  s->alpha = f->alpha;
  s->r = f->r;
  s->last_path = f->last_path;
  s->diagonal = f->diag ? 1 : 0;
  s->gep_rank = f->gep_rank;
  s->new_dirs = f->new_dirs;
  s->t_eig = f->t_eig;
  s->t_lmax = f->t_lmax;
  s->chol_exact_retries = f->chol_exact_retries;
}

// ---------------------------------------------------------------------------
// Reverse-mode gradient of the summed innovation NLL for a fixed H.
//
// For a fixed H (the setting of Alg. kalmanconstantH) the NLL depends on the
// state only through h_k = H s_k|k and T_k = H Sigma_k|k H^T, whose recursion
// closes in data space (predict Sigma += Gamma, Sec. 2.3):
//   P_k = T_{k-1} + A,  S_k = P_k + rho I,  nu_k = y_k - h_{k-1},
//   z_k = S_k^-1 nu_k,  h_k = h_{k-1} + P_k z_k,  T_k = rho P_k S_k^-1,
//   NLL = sum_k 1/2 (nu_k^T z_k + log det S_k + m log 2 pi),
// with A = H Gamma_H H^T from one H-apply, h_0 = H s_0, T_0 = alpha_0 A.
// The adjoint runs k = K..1 with hbar, Tbar (m x m):
//   zbar = P hbar,  X1 = P S^-1,  w = S^-1 zbar,
//   Sbar = 1/2 S^-1 - 1/2 z z^T + X1^T Tbar X1 - 1/2 (w z^T + z w^T)
//   Pbar = Tbar - (Tbar X1 + X1^T Tbar) + 1/2 (hbar z^T + z hbar^T) + Sbar
//   ybar_k = z + w,  hbar <- hbar - ybar_k,  Tbar <- Pbar,
//   dNLL/drho += tr(Sbar),  dNLL/dsigma2 += tr(Pbar A) / sigma2,
// and finally dNLL/ds0 = H^T hbar_0, dNLL/dsigma2 += alpha_0 tr(Tbar_0 A)/sigma2
// (Gamma_H = sigma2 Gamma_1: the H-matrix scales linearly with sigma2).
// The Cholesky factors of S_k are recomputed in the backward pass from the
// stored T_{k-1}; nothing of size N is stored per step.
// ---------------------------------------------------------------------------
namespace {

__global__ void k_spmv_orig(int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const double* __restrict__ val, int64_t n, const double* __restrict__ s,
                            double* __restrict__ out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= m) return;
  double acc = 0;
  for (int64_t p = rowptr[w] + lane; p < rowptr[w + 1]; p += 32) {
    const int64_t c = col[p];
    if (c >= 0 && c < n) acc += val[p] * s[c];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[w] = acc;
}


// v_out = a*x + b*y (n)
__global__ void k_axpby(int n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}

// Sbar = sym(Q) + 1/2 Sinv - 1/2 z z^T - 1/2 (w z^T + z w^T), Q = X1^T Tbar X1
// Pbar = Tbar - (TX + TX^T) + 1/2 (hb z^T + z hb^T) + Sbar
__global__ void k_adjoint_mats(int m, const double* __restrict__ Q, const double* __restrict__ Sinv,
                               const double* __restrict__ z, const double* __restrict__ w,
                               const double* __restrict__ Tbar, const double* __restrict__ TX,
                               const double* __restrict__ hb, double* __restrict__ Sbar, double* __restrict__ Pbar) {
  const int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    const int64_t t = (int64_t)j * m + i;
    const double sb = 0.5 * (Q[e] + Q[t]) + 0.5 * Sinv[e] - 0.5 * z[i] * z[j] - 0.5 * (w[i] * z[j] + z[i] * w[j]);
    Sbar[e] = sb;
    Pbar[e] = Tbar[e] - (TX[e] + TX[t]) + 0.5 * (hb[i] * z[j] + z[i] * hb[j]) + sb;
  }
}

// acc[0] += tr(Sbar), acc[1] += sum(Pbar .* A)  (single CTA)
__global__ void k_adjoint_scalars(int m, const double* __restrict__ Sbar, const double* __restrict__ Pbar,
                                  const double* __restrict__ A, double* __restrict__ acc) {
  __shared__ double sh[2][32];
  double a = 0, b = 0;
  const int64_t total = (int64_t)m * m;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    if (e / m == e % m) a += Sbar[e];
    b += Pbar[e] * A[e];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = a;
    sh[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0, sb = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
      sa += sh[0][i];
      sb += sh[1][i];
    }
    acc[0] += sa;
    acc[1] += sb;
  }
}

}  // namespace

template <typename T>
static fkf_status nll_gradient_impl(fkf_hmat* h, int K, int m, const double* y, const int64_t* rowptr_h,
                                    const int32_t* col_h, const double* val_h, double rho, const double* s0,
                                    double alpha0, double* nll_out, double* gy, double* gs0, double* gsig,
                                    double* grho) {
  fkf_ctx* ctx = h->ctx;
  cudaStream_t st = ctx->stream;
  const int64_t n = h->n, mm = (int64_t)m * m;
  const int64_t nnz = rowptr_h[m];
  // --- inputs
  DevBuf rowptr, col, val, yd, s0d, Bt, G, HG, flag;
  FKF_TRY(dev_upload(ctx, rowptr, rowptr_h, (m + 1) * 8));
  FKF_TRY(dev_upload(ctx, col, col_h, std::max<int64_t>(nnz, 1) * 4));
  FKF_TRY(dev_upload(ctx, val, val_h, std::max<int64_t>(nnz, 1) * 8));
  FKF_TRY(dev_upload(ctx, yd, y, (size_t)K * m * 8));
  FKF_TRY(dev_alloc(ctx, s0d, n * 8));
  if (s0) {
    FKF_CUDA(ctx, cudaMemcpyAsync(s0d.p, s0, n * 8, cudaMemcpyHostToDevice, st));
  } else {
    FKF_CUDA(ctx, cudaMemsetAsync(s0d.p, 0, n * 8, st));
  }
  FKF_TRY(dev_alloc(ctx, flag, 64));
  FKF_CUDA(ctx, cudaMemsetAsync(flag.p, 0, 64, st));
  const int64_t* iperm = h->iperm_d.as<int64_t>();
  // --- A = H Gamma_H H^T (one H-apply of m columns)
  FKF_TRY(dev_alloc(ctx, Bt, (size_t)n * m * sizeof(T)));
  FKF_TRY(dev_alloc(ctx, G, (size_t)n * m * sizeof(T)));
  FKF_CUDA(ctx, cudaMemsetAsync(Bt.p, 0, (size_t)n * m * sizeof(T), st));
  k_densify<T><<<(int)cdiv(m, 128), 128, 0, st>>>(m, rowptr.as<int64_t>(), col.as<int32_t>(), val.as<double>(), iperm,
                                                  n, Bt.as<T>(), m, flag.as<int>());
  FKF_LAUNCHED(ctx);
  FKF_TRY(hmat_apply_clustered(h, Bt.p, m, G.p, m, m));
  DevBuf A, Araw;
  FKF_TRY(dev_alloc(ctx, Araw, mm * 8));
  FKF_TRY(dev_alloc(ctx, A, mm * 8));
  csr_gather<T>(m, rowptr.as<int64_t>(), col.as<int32_t>(), val.as<double>(), iperm, n, G.as<T>(), m, m,
                Araw.as<double>(), m, st);
  FKF_LAUNCHED(ctx);
  FKF_CUDA(ctx, cudaMemcpyAsync(A.p, Araw.p, mm * 8, cudaMemcpyDeviceToDevice, st));
  k_symmetrize<<<nblk(mm), 256, 0, st>>>(m, A.as<double>());
  FKF_LAUNCHED(ctx);
  G.release();
  Bt.release();
  int hflag = 0;
  FKF_CUDA(ctx, cudaMemcpyAsync(&hflag, flag.p, 4, cudaMemcpyDeviceToHost, st));
  FKF_CUDA(ctx, cudaStreamSynchronize(st));
  if (hflag) return set_err(ctx, FKF_EINVAL, "nll_gradient: H column index outside [0, N)");
  // --- forward data-space recursion, storing T_{k-1} and h_{k-1}
  DevBuf Ts, hs, T0, P, S, X1, nu, z, nll_acc, chws;
  FKF_TRY(dev_alloc(ctx, Ts, (size_t)K * mm * 8));
  FKF_TRY(dev_alloc(ctx, hs, (size_t)(K + 1) * m * 8));
  FKF_TRY(dev_alloc(ctx, P, mm * 8));
  FKF_TRY(dev_alloc(ctx, S, mm * 8));
  FKF_TRY(dev_alloc(ctx, X1, mm * 8));
  FKF_TRY(dev_alloc(ctx, nu, m * 8));
  FKF_TRY(dev_alloc(ctx, z, m * 8));
  FKF_TRY(dev_alloc(ctx, nll_acc, 64));
  double* Ad = A.as<double>();
  double* Td = Ts.as<double>();
  double* hd = hs.as<double>();
  k_lincomb<<<nblk(mm), 256, 0, st>>>(m, alpha0, Ad, 0.0, nullptr, 0.0, Td);  // T_0 = alpha0 A
  FKF_LAUNCHED(ctx);
  k_spmv_orig<<<(int)cdiv((int64_t)m * 32, 256), 256, 0, st>>>(m, rowptr.as<int64_t>(), col.as<int32_t>(),
                                                              val.as<double>(), n, s0d.as<double>(), hd);
  FKF_LAUNCHED(ctx);
  double nll = 0;
  for (int k = 0; k < K; k++) {
    double* Tk = Td + (int64_t)k * mm;  // T_{k-1} (the state before step k)
    double* hk = hd + (int64_t)k * m;   // h_{k-1}
    k_lincomb<<<nblk(mm), 256, 0, st>>>(m, 1.0, Tk, 1.0, Ad, 0.0, P.as<double>());
    FKF_LAUNCHED(ctx);
    k_lincomb<<<nblk(mm), 256, 0, st>>>(m, 1.0, P.as<double>(), 0.0, nullptr, rho, S.as<double>());
    FKF_LAUNCHED(ctx);
    FKF_TRY(chol_f64(ctx, m, S.as<double>(), chws));
    k_axpby<<<(int)cdiv(m, 256), 256, 0, st>>>(m, 1.0, yd.as<double>() + (int64_t)k * m, -1.0, hk, nu.as<double>());
    FKF_LAUNCHED(ctx);
    FKF_CUDA(ctx, cudaMemcpyAsync(z.p, nu.p, m * 8, cudaMemcpyDeviceToDevice, st));
    FKF_TRY(chol_solve_f64(ctx, m, S.as<double>(), z.as<double>(), 1));
    k_nll<<<1, 256, 0, st>>>(m, nu.as<double>(), z.as<double>(), S.as<double>(), m, nll_acc.as<double>());
    FKF_LAUNCHED(ctx);
    double nk = 0;
    FKF_CUDA(ctx, cudaMemcpyAsync(&nk, nll_acc.p, 8, cudaMemcpyDeviceToHost, st));
    // h_k = h_{k-1} + P z
    FKF_CUDA(ctx, cudaMemcpyAsync(hk + m, hk, m * 8, cudaMemcpyDeviceToDevice, st));
    FKF_TRY(gemm_f64(ctx, false, false, m, 1, m, 1.0, P.as<double>(), m, z.as<double>(), 1, 1.0, hk + m, 1));
    if (k + 1 < K) {
      // T_k = rho P S^-1 (row-major P S^-1 from a column-major solve of the symmetric P)
      FKF_CUDA(ctx, cudaMemcpyAsync(X1.p, P.p, mm * 8, cudaMemcpyDeviceToDevice, st));
      FKF_TRY(chol_solve_f64(ctx, m, S.as<double>(), X1.as<double>(), m));
      k_lincomb<<<nblk(mm), 256, 0, st>>>(m, rho, X1.as<double>(), 0.0, nullptr, 0.0, Tk + mm);
      FKF_LAUNCHED(ctx);
      k_symmetrize<<<nblk(mm), 256, 0, st>>>(m, Tk + mm);
      FKF_LAUNCHED(ctx);
    }
    FKF_CUDA(ctx, cudaStreamSynchronize(st));
    nll += nk;
  }
  if (nll_out) *nll_out = nll;
  if (!gy && !gs0 && !gsig && !grho) return FKF_OK;
  // --- backward
  DevBuf Tbar, Pbar, Sbar, Sinv, TX, Q, hbar, zbar, w, gyd, acc;
  FKF_TRY(dev_alloc(ctx, Tbar, mm * 8));
  FKF_TRY(dev_alloc(ctx, Pbar, mm * 8));
  FKF_TRY(dev_alloc(ctx, Sbar, mm * 8));
  FKF_TRY(dev_alloc(ctx, Sinv, mm * 8));
  FKF_TRY(dev_alloc(ctx, TX, mm * 8));
  FKF_TRY(dev_alloc(ctx, Q, mm * 8));
  FKF_TRY(dev_alloc(ctx, hbar, m * 8));
  FKF_TRY(dev_alloc(ctx, zbar, m * 8));
  FKF_TRY(dev_alloc(ctx, w, m * 8));
  FKF_TRY(dev_alloc(ctx, gyd, (size_t)K * m * 8));
  FKF_TRY(dev_alloc(ctx, acc, 64));
  FKF_CUDA(ctx, cudaMemsetAsync(Tbar.p, 0, mm * 8, st));
  FKF_CUDA(ctx, cudaMemsetAsync(hbar.p, 0, m * 8, st));
  FKF_CUDA(ctx, cudaMemsetAsync(acc.p, 0, 64, st));
  for (int k = K - 1; k >= 0; k--) {
    double* Tk = Td + (int64_t)k * mm;
    double* hk = hd + (int64_t)k * m;
    // recompute P, S = chol(P + rho I), z
    k_lincomb<<<nblk(mm), 256, 0, st>>>(m, 1.0, Tk, 1.0, Ad, 0.0, P.as<double>());
    FKF_LAUNCHED(ctx);
    k_lincomb<<<nblk(mm), 256, 0, st>>>(m, 1.0, P.as<double>(), 0.0, nullptr, rho, S.as<double>());
    FKF_LAUNCHED(ctx);
    FKF_TRY(chol_f64(ctx, m, S.as<double>(), chws));
    k_axpby<<<(int)cdiv(m, 256), 256, 0, st>>>(m, 1.0, yd.as<double>() + (int64_t)k * m, -1.0, hk, z.as<double>());
    FKF_LAUNCHED(ctx);
    FKF_TRY(chol_solve_f64(ctx, m, S.as<double>(), z.as<double>(), 1));
    // zbar = P hbar ; w = S^-1 zbar ; X1 = P S^-1 ; Sinv
    FKF_TRY(gemm_f64(ctx, false, false, m, 1, m, 1.0, P.as<double>(), m, hbar.as<double>(), 1, 0.0, zbar.as<double>(), 1));
    FKF_CUDA(ctx, cudaMemcpyAsync(w.p, zbar.p, m * 8, cudaMemcpyDeviceToDevice, st));
    FKF_TRY(chol_solve_f64(ctx, m, S.as<double>(), w.as<double>(), 1));
    FKF_CUDA(ctx, cudaMemcpyAsync(X1.p, P.p, mm * 8, cudaMemcpyDeviceToDevice, st));
    FKF_TRY(chol_solve_f64(ctx, m, S.as<double>(), X1.as<double>(), m));
    k_identity<<<nblk(mm), 256, 0, st>>>(m, Sinv.as<double>(), m);
    FKF_LAUNCHED(ctx);
    FKF_TRY(chol_solve_f64(ctx, m, S.as<double>(), Sinv.as<double>(), m));
    // TX = Tbar X1 ; Q = X1^T TX
    FKF_TRY(gemm_f64(ctx, false, false, m, m, m, 1.0, Tbar.as<double>(), m, X1.as<double>(), m, 0.0, TX.as<double>(), m));
    FKF_TRY(gemm_f64(ctx, true, false, m, m, m, 1.0, X1.as<double>(), m, TX.as<double>(), m, 0.0, Q.as<double>(), m));
    k_adjoint_mats<<<nblk(mm), 256, 0, st>>>(m, Q.as<double>(), Sinv.as<double>(), z.as<double>(), w.as<double>(),
                                             Tbar.as<double>(), TX.as<double>(), hbar.as<double>(), Sbar.as<double>(),
                                             Pbar.as<double>());
    FKF_LAUNCHED(ctx);
    k_adjoint_scalars<<<1, 1024, 0, st>>>(m, Sbar.as<double>(), Pbar.as<double>(), Ad, acc.as<double>());
    FKF_LAUNCHED(ctx);
    // ybar_k = z + w ; hbar <- hbar - ybar_k ; Tbar <- Pbar
    double* gk = gyd.as<double>() + (int64_t)k * m;
    k_axpby<<<(int)cdiv(m, 256), 256, 0, st>>>(m, 1.0, z.as<double>(), 1.0, w.as<double>(), gk);
    FKF_LAUNCHED(ctx);
    k_axpby<<<(int)cdiv(m, 256), 256, 0, st>>>(m, 1.0, hbar.as<double>(), -1.0, gk, hbar.as<double>());
    FKF_LAUNCHED(ctx);
    std::swap(Tbar.p, Pbar.p);
  }
  // alpha0 term of the sigma2 gradient: acc[1] += alpha0 tr(Tbar_0 A)
  if (alpha0 != 0.0) {
    FKF_CUDA(ctx, cudaMemsetAsync(Sbar.p, 0, mm * 8, st));
    k_lincomb<<<nblk(mm), 256, 0, st>>>(m, alpha0, Tbar.as<double>(), 0.0, nullptr, 0.0, Pbar.as<double>());
    FKF_LAUNCHED(ctx);
    k_adjoint_scalars<<<1, 1024, 0, st>>>(m, Sbar.as<double>(), Pbar.as<double>(), Ad, acc.as<double>());
    FKF_LAUNCHED(ctx);
  }
  double acc_h[2] = {0, 0};
  FKF_CUDA(ctx, cudaMemcpyAsync(acc_h, acc.p, 16, cudaMemcpyDeviceToHost, st));
  if (gy) FKF_CUDA(ctx, cudaMemcpyAsync(gy, gyd.p, (size_t)K * m * 8, cudaMemcpyDeviceToHost, st));
  if (gs0) {
    // dNLL/ds0 = H^T hbar_0 through a column index of H (deterministic order)
    DevBuf cnt, cursor, colptr, crow, cval, gc, go, scanws;
    FKF_TRY(dev_alloc(ctx, cnt, n * 4 + 64));
    FKF_TRY(dev_alloc(ctx, cursor, n * 4 + 64));
    FKF_TRY(dev_alloc(ctx, colptr, (n + 1) * 8));
    FKF_TRY(dev_alloc(ctx, crow, std::max<int64_t>(nnz, 1) * 4));
    FKF_TRY(dev_alloc(ctx, cval, std::max<int64_t>(nnz, 1) * 8));
    FKF_TRY(dev_alloc(ctx, gc, n * 8));
    FKF_TRY(dev_alloc(ctx, go, n * 8));
    FKF_CUDA(ctx, cudaMemsetAsync(cnt.p, 0, n * 4, st));
    FKF_CUDA(ctx, cudaMemsetAsync(cursor.p, 0, n * 4, st));
    FKF_CUDA(ctx, cudaMemsetAsync(gc.p, 0, n * 8, st));
    k_csc_count<<<(int)cdiv((int64_t)m * 32, 256), 256, 0, st>>>(m, rowptr.as<int64_t>(), col.as<int32_t>(), iperm, n,
                                                                  cnt.as<int>(), flag.as<int>());
    FKF_LAUNCHED(ctx);
    FKF_TRY(scan_counts(ctx, n, cnt.as<int>(), colptr.as<int64_t>(), scanws));
    k_csc_fill<<<(int)cdiv((int64_t)m * 32, 256), 256, 0, st>>>(m, rowptr.as<int64_t>(), col.as<int32_t>(), val.as<double>(), iperm,
                                                   n, colptr.as<int64_t>(), cursor.as<int>(), crow.as<int>(),
                                                   cval.as<double>());
    FKF_LAUNCHED(ctx);
    k_csc_sort<<<(int)cdiv(n, 256), 256, 0, st>>>(n, colptr.as<int64_t>(), crow.as<int>(), cval.as<double>());
    FKF_LAUNCHED(ctx);
    k_csc_spmm<double><<<(int)cdiv(n * 32, 256), 256, 0, st>>>(n, colptr.as<int64_t>(), crow.as<int>(),
                                                               cval.as<double>(), hbar.as<double>(), 1, gc.as<double>(), 1);
    FKF_LAUNCHED(ctx);
    FKF_TRY(hmat_permute_rows_f64(ctx, gc.as<double>(), 1, iperm, go.as<double>(), 1, n, 1));
    FKF_CUDA(ctx, cudaMemcpyAsync(gs0, go.p, n * 8, cudaMemcpyDeviceToHost, st));
    FKF_CUDA(ctx, cudaStreamSynchronize(st));
  }
  FKF_CUDA(ctx, cudaStreamSynchronize(st));
  FKF_CUDA(ctx, cudaGetLastError());
  if (grho) *grho = acc_h[0];
  if (gsig) *gsig = acc_h[1] / h->kernel.sigma2;
  return FKF_OK;
}

fkf_status filter_nll_gradient(fkf_hmat* h, int K, int m, const double* y, const int64_t* rowptr, const int32_t* col,
                               const double* val, double rho, const double* s0, double alpha0, double* nll,
                               double* gy, double* gs0, double* gsig, double* grho) {
  fkf_ctx* ctx = h->ctx;
  Fp64TcScope tc(ctx, false);  // the adjoint's data-space recursion keeps exact FP64 products
  if (K < 1 || m < 1) return set_err(ctx, FKF_EINVAL, "nll_gradient: K >= 1 and m >= 1 required");
  if (!(rho > 0) || !(alpha0 >= 0)) return set_err(ctx, FKF_EINVAL, "nll_gradient: rho > 0 and alpha0 >= 0 required");
  if (rowptr[0] != 0) return set_err(ctx, FKF_EINVAL, "nll_gradient: rowptr[0] must be 0");
  for (int j = 0; j < m; j++)
    if (rowptr[j + 1] < rowptr[j]) return set_err(ctx, FKF_EINVAL, "nll_gradient: rowptr not nondecreasing");
  if (h->prec == FKF_FP64)
    return nll_gradient_impl<double>(h, K, m, y, rowptr, col, val, rho, s0, alpha0, nll, gy, gs0, gsig, grho);
  return nll_gradient_impl<float>(h, K, m, y, rowptr, col, val, rho, s0, alpha0, nll, gy, gs0, gsig, grho);
}
