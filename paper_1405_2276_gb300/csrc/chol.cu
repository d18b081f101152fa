// Blocked FP64 Cholesky factorisation and forward substitution for the m x m
// innovation covariance S of the filter step (row-major, S = L L^T with L in
// the lower triangle).
//
// FP64 throughput on this part is a small fraction of FP32's and a warp-wide
// FP64 instruction holds its sub-partition for many clocks, so the design
// keeps the sequential part short and spreads everything else over the SMs:
// blocks of kB; a diagonal block is factored by one CTA (kB rank-1 steps in
// shared memory); the panel below it is solved row by row (one warp per row,
// kB / 32 columns per lane, the factor block in shared memory, 8 rows per CTA);
// the trailing matrix is updated by the symmetric FP64 tile GEMM (lower tiles
// only).  Stopping after the first nf pivots of a bordered matrix
// [[S, K], [K^T, E]] leaves the Schur complement E - K^T S^-1 K in the
// trailing block.  Column-major BLAS reads this row-major lower factor as the
// upper factor U = L^T of S = U^T U.
#include <algorithm>
#include <cmath>

#include "common.h"
#include "dense.h"

#ifndef FKF_CHOL_BLOCK
#define FKF_CHOL_BLOCK 64
#endif

namespace {

constexpr int kB = FKF_CHOL_BLOCK;  // block size (a multiple of 32, at most 64)
constexpr int kV = kB / 32;         // columns per lane in the row kernels
constexpr int kPB = 32;             // pivots per panel of the pivoted Cholesky

// 1 / sqrt(d) for d > 0 by Newton's iteration for f(r) = r^-2 - d,
// r <- r + r (1 - d r^2) / 2 (quadratic convergence), seeded with the
// single-precision hardware estimate rsqrtf (relative error about 2^-22):
// two steps bring the error below FP64 rounding.  A pivot's square root and
// reciprocal then cost a handful of FP64 operations instead of a square root
// and a division (long FP64 sequences on this part).  d outside the
// single-precision range takes 1 / sqrt(d).
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-36 && d < 1e36)) return 1.0 / sqrt(d);
  double r = (double)rsqrtf((float)d);
#pragma unroll
  for (int it = 0; it < 2; it++) {
    const double e = fma(-(d * r), r, 1.0);  // 1 - d r^2
    r = fma(0.5 * r, e, r);
  }
  return r;
}

// Factor the b x b diagonal block A (ld lda, lower triangle) in place; the
// reciprocals of the factor's diagonal go to dinv[0:b].  A pivot that is not
// positive sets *flag and is replaced by 1 so that the factorisation
// completes without NaNs (the caller reports the failure).
__global__ void __launch_bounds__(256) k_potrf_diag(double* __restrict__ A, int64_t lda, int b,
                                                    int* __restrict__ flag, double* __restrict__ dinv) {
  __shared__ double a[kB][kB + 1];
  // the lower triangle's entries ordered by column, last column first:
  // entry t = (row, column) packed as row << 8 | column, so that the entries
  // right of column j are the first (b-j-1)(b-j)/2 (the update of step j
  // issues no FP64 instruction for entries it leaves alone)
  __shared__ unsigned short tri[kB * (kB + 1) / 2];
  const int t = threadIdx.x;
  for (int e = t; e < b * (b + 1) / 2; e += blockDim.x) {
    int u = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)e)) * 0.5f);  // columns b-u.. hold the first u(u+1)/2
    while (u * (u - 1) / 2 > e) u--;
    while (u * (u + 1) / 2 <= e) u++;
    const int c = b - u, i = c + (e - u * (u - 1) / 2);
    tri[e] = (unsigned short)(i << 8 | c);
  }
  // launched early behind the previous kernel of the stream (programmatic
  // dependent launch): its results are visible after this wait
  cudaGridDependencySynchronize();
  for (int e = t; e < kB * kB; e += blockDim.x) {
    const int i = e / kB, j = e % kB;
    a[i][j] = (i < b && j <= i) ? A[(int64_t)i * lda + j] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < b; j++) {
    // the pivot's reciprocal square root by one warp (the other warps do not
    // repeat it): L_jj = d r, column j below it times r = 1 / L_jj
    if (t < 32) {
      double d = a[j][j];
      __syncwarp();  // every lane has read the pivot before lane 0 overwrites it
      if (!(d > 0.0)) {
        if (t == 0) atomicOr(flag, 1);
        d = 1.0;
      }
      const double r = rsqrt_newton(d);
      for (int i = j + 1 + t; i < b; i += 32) a[i][j] *= r;  // (blocks wider than a warp: two rows per lane)
      if (t == 0) {
        a[j][j] = d * r;
        dinv[j] = r;
      }
    }
    __syncthreads();
    // a[i][l] -= a[i][j] a[l][j] for j < l <= i < b
    const int cnt = (b - j - 1) * (b - j) / 2;
    for (int e = t; e < cnt; e += blockDim.x) {
      const int i = tri[e] >> 8, l = tri[e] & 255;
      a[i][l] -= a[i][j] * a[l][j];
    }
    __syncthreads();
  }
  for (int e = t; e < kB * kB; e += blockDim.x) {
    const int i = e / kB, j = e % kB;
    if (i < b && j <= i) A[(int64_t)i * lda + j] = a[i][j];
  }
}

// X[r, 0:b] <- X[r, 0:b] Lkk^-T for rows r < rows (forward substitution per
// row: x_j = (x_j - sum_{l<j} x_l Lkk[j][l]) / Lkk[j][j]); Lkk is the b x b
// lower factor block at L (ld lda).  One warp per row, lane j holding x_j,
// x_{j+32}, ...: after x_q is final it is broadcast and every later column
// subtracts its term, so a row costs b dependent steps (FP64 instructions are
// slow per warp here; many short rows in flight use all the SMs).
// dinv_g[0:b]: the reciprocals of Lkk's diagonal (from k_potrf_diag).
constexpr int kRowWarps = 8;
__global__ void __launch_bounds__(32 * kRowWarps) k_trsm_rows(double* __restrict__ X, int64_t ldx, int64_t rows,
                                                              int b, const double* __restrict__ L, int64_t lda,
                                                              const double* __restrict__ dinv_g) {
  __shared__ double l[kB][kB + 1];
  __shared__ double dinv[kB];
  const int t = threadIdx.x;
  cudaGridDependencySynchronize();  // launched early behind the diagonal block's kernel
  for (int e = t; e < kB * kB; e += blockDim.x) {
    const int i = e / kB, j = e % kB;
    l[i][j] = (i < b && j <= i) ? L[(int64_t)i * lda + j] : 0.0;
  }
  if (t < b) dinv[t] = dinv_g[t];
  __syncthreads();
  const int lane = t & 31;
  const int64_t r = (int64_t)blockIdx.x * kRowWarps + (t >> 5);
  if (r >= rows) return;
  double* xr = X + r * ldx;
  double s[kV];
#pragma unroll
  for (int v = 0; v < kV; v++) s[v] = 32 * v + lane < b ? xr[32 * v + lane] : 0.0;
#pragma unroll
  for (int q = 0; q < kB; q++) {
    if (q >= b) break;
    const int qv = q >> 5, ql = q & 31;
    const double xq = __shfl_sync(0xffffffffu, s[qv] * dinv[q], ql);
#pragma unroll
    for (int v = 0; v < kV; v++) {
      const int c = 32 * v + lane;
      if (c == q) s[v] = xq;
      if (c > q) s[v] -= xq * l[c][q];
    }
  }
#pragma unroll
  for (int v = 0; v < kV; v++)
    if (32 * v + lane < b) xr[32 * v + lane] = s[v];
}

// C[r, 0:nc] -= P[r, 0:b] Q^T for rows r < rows, with Q = P[0:nc, 0:b] (the
// rows of the next diagonal block): the update of the next block column by
// the current panel.  One warp per row, lane j accumulating columns j,
// j + 32, ...; Q in shared memory, P's row broadcast by shuffles.
__global__ void __launch_bounds__(32 * kRowWarps) k_next_column(double* __restrict__ C, int64_t ldc, int64_t rows,
                                                                int nc, const double* __restrict__ P, int64_t ldp,
                                                                int b) {
  __shared__ double q[kB][kB + 1];
  const int t = threadIdx.x;
  for (int e = t; e < kB * kB; e += blockDim.x) {
    const int i = e / kB, l = e % kB;
    q[i][l] = (i < nc && l < b) ? P[(int64_t)i * ldp + l] : 0.0;
  }
  __syncthreads();
  const int lane = t & 31;
  const int64_t r = (int64_t)blockIdx.x * kRowWarps + (t >> 5);
  if (r >= rows) return;
  double pl[kV], acc[kV];
#pragma unroll
  for (int v = 0; v < kV; v++) {
    pl[v] = 32 * v + lane < b ? P[r * ldp + 32 * v + lane] : 0.0;
    acc[v] = 0.0;
  }
#pragma unroll
  for (int l = 0; l < kB; l++) {
    const double p = __shfl_sync(0xffffffffu, pl[l >> 5], l & 31);
#pragma unroll
    for (int v = 0; v < kV; v++) acc[v] += p * q[32 * v + lane][l];
  }
#pragma unroll
  for (int v = 0; v < kV; v++)
    if (32 * v + lane < nc) C[r * ldc + 32 * v + lane] -= acc[v];
}

// One panel of a pivoted (rank-revealing) Cholesky factorisation, one CTA:
// up to maxc pivots, each the index with the largest remaining diagonal
// among those not yet pivoted; stops when that diagonal is <= tol.  A
// (symmetric, lower triangle valid) already carries the updates of the
// previous panels; column k0 + j of Lp (n x ., ld ldl) becomes
// (A(:, p) - sum_{jj < j} Lp(:, k0 + jj) Lp(p, k0 + jj)) / sqrt(d_p), zero on
// rows pivoted earlier; diag and pivoted are updated; *count = columns made.
constexpr int kPcholThreads = 1024;
__global__ void __launch_bounds__(kPcholThreads) k_pchol_panel(int n, const double* __restrict__ A, int64_t lda,
                                                               double* __restrict__ diag, int* __restrict__ pivoted,
                                                               double* __restrict__ Lp, int64_t ldl, int k0, int maxc,
                                                               double tol, int* __restrict__ count) {
  __shared__ double bv[32];
  __shared__ int bi[32];
  __shared__ double prow[kPB];  // Lp(p, k0 .. k0 + j - 1) of the current pivot
  __shared__ int sp;
  __shared__ double sd;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int j = 0;
  for (; j < maxc; j++) {
    // argmax of the remaining diagonal (ties: smallest index)
    double v = -1.0;
    int vi = n;
    for (int i = t; i < n; i += kPcholThreads)
      if (!pivoted[i] && diag[i] > v) v = diag[i], vi = i;
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, vi, o);
      if (ov > v || (ov == v && oi < vi)) v = ov, vi = oi;
    }
    if (lane == 0) bv[warp] = v, bi[warp] = vi;
    __syncthreads();
    if (t == 0) {
      double b = -1.0;
      int p = n;
      for (int w = 0; w < kPcholThreads / 32; w++)
        if (bv[w] > b || (bv[w] == b && bi[w] < p)) b = bv[w], p = bi[w];
      sp = p;
      sd = b;
    }
    __syncthreads();
    const int p = sp;
    const double dp = sd;
    if (!(dp > tol) || p >= n) break;
    if (t < j) prow[t] = Lp[(int64_t)p * ldl + k0 + t];
    __syncthreads();
    const double rp = sqrt(dp);
    for (int i = t; i < n; i += kPcholThreads) {
      double l = 0.0;
      if (i == p) {
        l = rp;
      } else if (!pivoted[i]) {
        double c = A[(int64_t)max(i, p) * lda + min(i, p)];
        for (int jj = 0; jj < j; jj++) c -= Lp[(int64_t)i * ldl + k0 + jj] * prow[jj];
        l = c / rp;
        diag[i] -= l * l;
      }
      Lp[(int64_t)i * ldl + k0 + j] = l;
    }
    __syncthreads();
    if (t == 0) {
      pivoted[p] = 1;
      diag[p] = 0.0;
    }
    __syncthreads();
  }
  if (t == 0) *count = j;
}

__global__ void k_diag_of(int n, const double* __restrict__ A, int64_t lda, double* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = A[(int64_t)i * lda + i];
}

// Launch with programmatic stream serialisation: the kernel may start while
// the previous kernel of the stream finishes and waits for it on the device
// (cudaGridDependencySynchronize), which hides the launch gap of the chain.
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kern)(P...), unsigned grid, unsigned block, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<P>(args)...);
}

}  // namespace

fkf_status pchol_f64(fkf_ctx* ctx, int n, double* A, int64_t lda, double tol, int max_rank, double* Lp, int64_t ldl,
                     DevBuf& ws, int* rank_out) {
  *rank_out = 0;
  if (n <= 0 || max_rank <= 0) return FKF_OK;
  const size_t need = (size_t)n * (sizeof(double) + sizeof(int)) + 256;
  if (ws.bytes < need) FKF_TRY(dev_alloc(ctx, ws, need));
  double* diag = ws.as<double>();
  int* pivoted = reinterpret_cast<int*>(diag + n);
  int* count = reinterpret_cast<int*>(ws.as<char>() + need - 64);
  cudaStream_t st = ctx->stream;
  k_diag_of<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, A, lda, diag);
  FKF_LAUNCHED(ctx);
  FKF_CUDA(ctx, cudaMemsetAsync(pivoted, 0, (size_t)n * sizeof(int), st));
  int rank = 0;
  while (rank < max_rank) {
    const int maxc = std::min(kPB, max_rank - rank);
    k_pchol_panel<<<1, kPcholThreads, 0, st>>>(n, A, lda, diag, pivoted, Lp, ldl, rank, maxc, tol, count);
    FKF_LAUNCHED(ctx);
    int c = 0;
    FKF_CUDA(ctx, cudaMemcpyAsync(&c, count, sizeof(int), cudaMemcpyDeviceToHost, st));
    FKF_CUDA(ctx, cudaStreamSynchronize(st));
    if (c > 0)  // the rest of the matrix loses this panel's contribution
      FKF_TRY(gemm_sym_f64(ctx, false, true, n, c, -1.0, Lp + rank, ldl, Lp + rank, ldl, 1.0, A, lda, true));
    rank += c;
    if (c < maxc) break;
  }
  *rank_out = rank;
  return FKF_OK;
}

// With look-ahead (several blocks): the critical chain -- diagonal block k,
// its panel, and the update of the next block column k+1 by panel k -- runs
// on the context's high-priority second stream, while the rest of panel k's
// trailing update (rows and columns from block k+2 on, the bulk of the flops)
// runs on the context stream; the block scheduler serves the chain first.
// Ordering: the trailing update of panel k waits for panel k; the update of
// block column k+1 by panel k waits for the trailing update of panel k-1
// (which also wrote block column k+1).  Every other pair of concurrent
// launches touches disjoint blocks.
// A bordered matrix (nf < n): the panels' trailing updates leave the block
// A22 = A[nf:, nf:] alone, and it becomes the Schur complement in one
// rank-nf product A22 -= L21 L21^T at the end (a long reduction that runs
// near the FP64 tile GEMM's rate, instead of nf / kB rank-kB updates).
fkf_status chol_blocked_f64(fkf_ctx* ctx, int n, int nf, double* A, int64_t lda, DevBuf& ws, cudaEvent_t schur_done) {
  if (n <= 0 || nf <= 0) return FKF_OK;
  nf = std::min(nf, n);
  // flag, then the reciprocals of the factor's diagonal (one slot per pivot)
  if (ws.bytes < 64 + (size_t)nf * sizeof(double)) FKF_TRY(dev_alloc(ctx, ws, 64 + (size_t)nf * sizeof(double)));
  int* flag = ws.as<int>();
  double* dinv = reinterpret_cast<double*>(ws.as<char>() + 64);
  FKF_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  const int nb = (int)cdiv(nf, kB);
  const bool la = nb >= 2 && n - kB > 2 * kB;
  cudaStream_t bs = ctx->stream, cs = ctx->stream;  // bulk, chain
  cudaEvent_t* evT = nullptr;
  cudaEvent_t* evS = nullptr;
  if (la || nf < n) FKF_TRY(ctx_side(ctx, 2 * (size_t)nb + 2));
  if (la) {
    cs = ctx->side;
    evT = ctx->side_ev.data();
    evS = evT + nb;
    // the chain starts after everything queued so far
    FKF_CUDA(ctx, cudaEventRecord(evS[nb], bs));
    FKF_CUDA(ctx, cudaStreamWaitEvent(cs, evS[nb], 0));
  }
  auto factor = [&]() -> fkf_status {
    for (int k = 0; k < nb; k++) {
      const int k0 = k * kB;
      const int b = std::min(kB, nf - k0);
      double* Akk = A + (int64_t)k0 * lda + k0;
      FKF_CUDA(ctx, launch_pdl(k_potrf_diag, 1, 256, cs, Akk, lda, b, flag, dinv + k0));
      FKF_LAUNCHED(ctx);
      const int rem = n - k0 - b;
      if (rem <= 0) continue;
      double* P = A + (int64_t)(k0 + b) * lda + k0;  // rem x b panel
      FKF_CUDA(ctx, launch_pdl(k_trsm_rows, (unsigned)cdiv(rem, kRowWarps), 32 * kRowWarps, cs, P, lda,
                               (int64_t)rem, b, (const double*)Akk, lda, (const double*)(dinv + k0)));
      FKF_LAUNCHED(ctx);
      double* C = P + b;  // trailing block at (k0 + b, k0 + b)
      // entries of the trailing block in A22 (relative index >= skip) wait for the final product
      const int64_t skip = nf < n ? nf - (k0 + b) : -1;
      if (!la) {
        if (skip != 0) FKF_TRY(gemm_sym_f64(ctx, false, true, rem, b, -1.0, P, lda, P, lda, 1.0, C, lda, true, skip));
        continue;
      }
      FKF_CUDA(ctx, cudaEventRecord(evT[k], cs));
      const int b1 = k + 1 < nb ? std::min(kB, nf - (k0 + b)) : 0;  // next block column (critical chain)
      if (b1 > 0) {
        if (k >= 1) FKF_CUDA(ctx, cudaStreamWaitEvent(cs, evS[k - 1], 0));
        k_next_column<<<(unsigned)cdiv(rem, kRowWarps), 32 * kRowWarps, 0, cs>>>(C, lda, rem, b1, P, lda, b);
        FKF_LAUNCHED(ctx);
      }
      const int rem2 = rem - b1;
      FKF_CUDA(ctx, cudaStreamWaitEvent(bs, evT[k], 0));
      const int64_t skip2 = nf < n ? nf - (k0 + b + b1) : -1;
      if (rem2 > 0 && skip2 != 0) {
        // the columns left of A22 (all of them without a border): large updates as one FP64
        // GEMM on the tensor cores over the whole rectangle (the upper triangle of the part
        // still to be factored is scratch), the others on the lower triangle alone
        const int64_t ncol = skip2 > 0 ? std::min<int64_t>(skip2, rem2) : rem2;
        double* P2 = P + (int64_t)b1 * lda;
        if (ctx->fp64_tc && (double)rem2 * ncol * b >= 1.6e7 && cdiv(rem2, 128) * cdiv(ncol, 64) >= 16)
          FKF_TRY(gemm_f64_tc(ctx, false, true, rem2, ncol, b, -1.0, P2, lda, P2, lda, 1.0, C + (int64_t)b1 * lda + b1,
                              lda));
        else
          FKF_TRY(gemm_sym_f64(ctx, false, true, rem2, b, -1.0, P2, lda, P2, lda, 1.0, C + (int64_t)b1 * lda + b1, lda,
                               true, skip2));
      }
      FKF_CUDA(ctx, cudaEventRecord(evS[k], bs));
    }
    return FKF_OK;
  };
  const fkf_status st = factor();
  if (la) {
    // join: the context stream continues after all of the chain's work (also when a launch
    // failed part-way)
    FKF_CUDA(ctx, cudaEventRecord(evS[nb], cs));
    FKF_CUDA(ctx, cudaStreamWaitEvent(bs, evS[nb], 0));
  }
  FKF_TRY(st);
  if (nf < n) {  // A22 -= L21 L21^T
    const double* L21 = A + (int64_t)nf * lda;
    double* A22 = A + (int64_t)nf * lda + nf;
    if (schur_done) {
      FKF_TRY(ctx_side_lo(ctx));
      cudaEvent_t fac = ctx->side_ev[2 * (size_t)nb + 1];
      FKF_CUDA(ctx, cudaEventRecord(fac, bs));
      FKF_CUDA(ctx, cudaStreamWaitEvent(ctx->side_lo, fac, 0));
      const cudaStream_t saved = ctx->stream;
      ctx->stream = ctx->side_lo;
      // (large: one FP64 GEMM on the tensor cores with the low-priority stream's
      // workspace, both triangles; else the lower triangle on the FP64 tile GEMM)
      const fkf_status ss =
          ctx->fp64_tc && (double)(n - nf) * (n - nf) * nf >= 1e8
              ? gemm_f64_tc(ctx, false, true, n - nf, n - nf, nf, -1.0, L21, lda, L21, lda, 1.0, A22, lda,
                            &ctx->ozgemm_ws_lo)
              : gemm_sym_f64(ctx, false, true, n - nf, nf, -1.0, L21, lda, L21, lda, 1.0, A22, lda, true);
      ctx->stream = saved;
      FKF_TRY(ss);
      FKF_CUDA(ctx, cudaEventRecord(schur_done, ctx->side_lo));
    } else {
      FKF_TRY(gemm_sym_f64(ctx, false, true, n - nf, nf, -1.0, L21, lda, L21, lda, 1.0, A22, lda, true));
    }
  }
  int hflag = 0;
  FKF_CUDA(ctx, cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, bs));
  FKF_CUDA(ctx, cudaStreamSynchronize(bs));
  if (hflag) {
    if (nf < n && schur_done) FKF_CUDA(ctx, cudaStreamWaitEvent(bs, schur_done, 0));  // nothing left in flight
    return set_err(ctx, FKF_ENOTSPD, "matrix not positive definite (n=%d, %d pivots)", n, nf);
  }
  return FKF_OK;
}

namespace {
// Triangular solves of one diagonal block for every right-hand side (thread
// per RHS row q of B): forward L_kk y = b (in place), or backward L_kk^T x = y.
__global__ void k_trsv_block_fwd(int nrhs, int b, const double* __restrict__ Lkk, int64_t ldl, double* B,
                                 int64_t ldb) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nrhs) return;
  double* Bq = B + (int64_t)q * ldb;
  for (int i = 0; i < b; i++) {
    double y0 = Bq[i], y1 = 0;
    int j = 0;
    for (; j + 1 < i; j += 2) {
      y0 -= Lkk[(int64_t)i * ldl + j] * Bq[j];
      y1 -= Lkk[(int64_t)i * ldl + j + 1] * Bq[j + 1];
    }
    for (; j < i; j++) y0 -= Lkk[(int64_t)i * ldl + j] * Bq[j];
    Bq[i] = (y0 + y1) / Lkk[(int64_t)i * ldl + i];
  }
}

__global__ void k_trsv_block_bwd(int nrhs, int b, const double* __restrict__ Lkk, int64_t ldl, double* B,
                                 int64_t ldb) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nrhs) return;
  double* Bq = B + (int64_t)q * ldb;
  for (int i = b - 1; i >= 0; i--) {
    double x0 = Bq[i], x1 = 0;
    int j = i + 1;
    for (; j + 1 < b; j += 2) {
      x0 -= Lkk[(int64_t)j * ldl + i] * Bq[j];
      x1 -= Lkk[(int64_t)(j + 1) * ldl + i] * Bq[j + 1];
    }
    for (; j < b; j++) x0 -= Lkk[(int64_t)j * ldl + i] * Bq[j];
    Bq[i] = (x0 + x1) / Lkk[(int64_t)i * ldl + i];
  }
}
}  // namespace

// Solve L L^T x = b for nrhs right-hand sides, the rows of B (nrhs x n,
// leading dimension ldb), with the lower factor L of chol_blocked_f64 (n x n
// row-major, ld ldl; only its lower triangle is read).  Row form: the
// forward substitution is Y = B L^-T, the backward one X = Y L^-1, both by
// blocks of kB columns: a triangular solve of the diagonal block per
// right-hand side, then one GEMM update of the remaining columns.
fkf_status chol_solve_rows_f64(fkf_ctx* ctx, int n, const double* L, int64_t ldl, double* B, int nrhs, int64_t ldb) {
  if (n <= 0 || nrhs <= 0) return FKF_OK;
  cudaStream_t st = ctx->stream;
  const unsigned g = (unsigned)cdiv(nrhs, 128);
  for (int k0 = 0; k0 < n; k0 += kB) {
    const int b = std::min(kB, n - k0);
    k_trsv_block_fwd<<<g, 128, 0, st>>>(nrhs, b, L + (int64_t)k0 * ldl + k0, ldl, B + k0, ldb);
    FKF_LAUNCHED(ctx);
    const int rest = n - k0 - b;
    if (rest > 0)
      FKF_TRY(gemm_f64(ctx, false, true, nrhs, rest, b, -1.0, B + k0, ldb, L + (int64_t)(k0 + b) * ldl + k0, ldl, 1.0,
                       B + k0 + b, ldb));
  }
  for (int k0 = ((n - 1) / kB) * kB; k0 >= 0; k0 -= kB) {
    const int b = std::min(kB, n - k0);
    k_trsv_block_bwd<<<g, 128, 0, st>>>(nrhs, b, L + (int64_t)k0 * ldl + k0, ldl, B + k0, ldb);
    FKF_LAUNCHED(ctx);
    if (k0 > 0)
      FKF_TRY(gemm_f64(ctx, false, false, nrhs, k0, b, -1.0, B + k0, ldb, L + (int64_t)k0 * ldl, ldl, 1.0, B, ldb));
  }
  return FKF_OK;
}
