// Small dense FP64 factorisations for the m x m and r x r data-space algebra:
// symmetric eigendecomposition and Cholesky.  These run on the GPU through
// cuSOLVER's dense routines (syevd, potrf, potrs) on the context stream.
#include <cusolverDn.h>

#include <cstring>

#include "dense.h"

static fkf_status solver(fkf_ctx* ctx, cusolverDnHandle_t* out) {
  if (!ctx->solver) {
    cusolverDnHandle_t h = nullptr;
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return set_err(ctx, FKF_ECUDA, "cusolverDnCreate failed");
    ctx->solver = reinterpret_cast<cusolverDnContext*>(h);
  }
  cusolverDnHandle_t h = reinterpret_cast<cusolverDnHandle_t>(ctx->solver);
  if (cusolverDnSetStream(h, ctx->stream) != CUSOLVER_STATUS_SUCCESS)
    return set_err(ctx, FKF_ECUDA, "cusolverDnSetStream failed");
  *out = h;
  return FKF_OK;
}

fkf_status eigh_f64(fkf_ctx* ctx, int n, double* A, double* w_dev, std::vector<double>& w_host, DevBuf& ws) {
  w_host.assign(n, 0.0);
  if (n == 0) return FKF_OK;
  cusolverDnHandle_t h;
  FKF_TRY(solver(ctx, &h));
  int lwork = 0;
  if (cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A, n, w_dev, &lwork) !=
      CUSOLVER_STATUS_SUCCESS)
    return set_err(ctx, FKF_ECUDA, "syevd_bufferSize failed (n=%d)", n);
  const size_t need = (size_t)lwork * sizeof(double) + 256;
  if (ws.bytes < need) FKF_TRY(dev_alloc(ctx, ws, need));
  int* info = reinterpret_cast<int*>(ws.as<char>() + (size_t)lwork * sizeof(double));
  // Row-major symmetric A is the same matrix in column-major order; on exit
  // column j (column-major) = row j (row-major) holds eigenvector j.
  if (cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A, n, w_dev, ws.as<double>(), lwork,
                       info) != CUSOLVER_STATUS_SUCCESS)
    return set_err(ctx, FKF_ECUDA, "syevd failed (n=%d)", n);
  ctx->lib_calls++;
  int hinfo = 0;
  FKF_CUDA(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FKF_CUDA(ctx, cudaMemcpyAsync(w_host.data(), w_dev, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hinfo != 0) return set_err(ctx, FKF_ENOCONV, "symmetric eigensolver did not converge (n=%d, info=%d)", n, hinfo);
  return FKF_OK;
}

fkf_status eigh_top_f64(fkf_ctx* ctx, int n, int k, double* A, double* w_dev, std::vector<double>& w_host, DevBuf& ws,
                        int* meig_out) {
  *meig_out = 0;
  w_host.clear();
  if (n == 0 || k <= 0) return FKF_OK;
  if (k >= n) {
    FKF_TRY(eigh_f64(ctx, n, A, w_dev, w_host, ws));
    *meig_out = n;
    return FKF_OK;
  }
  cusolverDnHandle_t h;
  FKF_TRY(solver(ctx, &h));
  int lwork = 0, meig = 0;
  const int il = n - k + 1, iu = n;
  if (cusolverDnDsyevdx_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, n, A, n,
                                   0.0, 0.0, il, iu, &meig, w_dev, &lwork) != CUSOLVER_STATUS_SUCCESS)
    return set_err(ctx, FKF_ECUDA, "syevdx_bufferSize failed (n=%d)", n);
  const size_t need = (size_t)lwork * sizeof(double) + 256;
  if (ws.bytes < need) FKF_TRY(dev_alloc(ctx, ws, need));
  int* info = reinterpret_cast<int*>(ws.as<char>() + (size_t)lwork * sizeof(double));
  if (cusolverDnDsyevdx(h, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, n, A, n, 0.0, 0.0,
                        il, iu, &meig, w_dev, ws.as<double>(), lwork, info) != CUSOLVER_STATUS_SUCCESS)
    return set_err(ctx, FKF_ECUDA, "syevdx failed (n=%d)", n);
  ctx->lib_calls++;
  int hinfo = 0;
  w_host.assign(std::max(meig, 0), 0.0);
  FKF_CUDA(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (meig > 0)
    FKF_CUDA(ctx, cudaMemcpyAsync(w_host.data(), w_dev, meig * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hinfo != 0) return set_err(ctx, FKF_ENOCONV, "symmetric eigensolver did not converge (n=%d, info=%d)", n, hinfo);
  *meig_out = meig;
  return FKF_OK;
}

fkf_status chol_f64(fkf_ctx* ctx, int n, double* A, DevBuf& ws) {
  if (n == 0) return FKF_OK;
  cusolverDnHandle_t h;
  FKF_TRY(solver(ctx, &h));
  int lwork = 0;
  if (cusolverDnDpotrf_bufferSize(h, CUBLAS_FILL_MODE_LOWER, n, A, n, &lwork) != CUSOLVER_STATUS_SUCCESS)
    return set_err(ctx, FKF_ECUDA, "potrf_bufferSize failed");
  const size_t need = (size_t)lwork * sizeof(double) + 256;
  if (ws.bytes < need) FKF_TRY(dev_alloc(ctx, ws, need));
  int* info = reinterpret_cast<int*>(ws.as<char>() + (size_t)lwork * sizeof(double));
  if (cusolverDnDpotrf(h, CUBLAS_FILL_MODE_LOWER, n, A, n, ws.as<double>(), lwork, info) != CUSOLVER_STATUS_SUCCESS)
    return set_err(ctx, FKF_ECUDA, "potrf failed");
  ctx->lib_calls++;
  int hinfo = 0;
  FKF_CUDA(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hinfo > 0) return set_err(ctx, FKF_ENOTSPD, "matrix not positive definite (leading minor %d of %d)", hinfo, n);
  if (hinfo < 0) return set_err(ctx, FKF_ECUDA, "potrf argument %d invalid", -hinfo);
  return FKF_OK;
}

fkf_status chol_solve_f64(fkf_ctx* ctx, int n, const double* Afact, double* b, int nrhs) {
  if (n == 0 || nrhs == 0) return FKF_OK;
  cusolverDnHandle_t h;
  FKF_TRY(solver(ctx, &h));
  if (ctx->solver_info.bytes < 256) FKF_TRY(dev_alloc(ctx, ctx->solver_info, 256));
  if (cusolverDnDpotrs(h, CUBLAS_FILL_MODE_LOWER, n, nrhs, Afact, n, b, n, ctx->solver_info.as<int>()) !=
      CUSOLVER_STATUS_SUCCESS)
    return set_err(ctx, FKF_ECUDA, "potrs failed");
  ctx->lib_calls++;
  return FKF_OK;
}

fkf_status chol_solve_rowlower_f64(fkf_ctx* ctx, int n, const double* L, int64_t ldl, double* b, int nrhs) {
  if (n == 0 || nrhs == 0) return FKF_OK;
  cusolverDnHandle_t h;
  FKF_TRY(solver(ctx, &h));
  if (ctx->solver_info.bytes < 256) FKF_TRY(dev_alloc(ctx, ctx->solver_info, 256));
  // the row-major lower factor is the column-major upper factor U = L^T, S = U^T U
  if (cusolverDnDpotrs(h, CUBLAS_FILL_MODE_UPPER, n, nrhs, L, (int)ldl, b, n, ctx->solver_info.as<int>()) !=
      CUSOLVER_STATUS_SUCCESS)
    return set_err(ctx, FKF_ECUDA, "potrs failed");
  ctx->lib_calls++;
  return FKF_OK;
}
