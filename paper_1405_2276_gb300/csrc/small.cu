// Small dense FP64 factorisations for the m x m and r x r data-space algebra:
// the symmetric eigendecompositions (the library's own solver, eigh.cu), the
// Cholesky factorisation and solves of small SPD systems (the library's own,
// chol.cu), and the one-right-hand-side solve of the step's innovation system
// (cuSOLVER's potrs on the context stream).
#include <cusolverDn.h>

#include <algorithm>
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

// The symmetric eigenproblems (data-space GEP, merge, re-diagonalisations)
// run on the library's own eigensolver (eigh.cu).
fkf_status eigh_f64(fkf_ctx* ctx, int n, double* A, double* w_dev, std::vector<double>& w_host, DevBuf& ws) {
  return eigh_own(ctx, n, A, w_dev, w_host, ws, n);
}

fkf_status eigh_top_f64(fkf_ctx* ctx, int n, int k, double* A, double* w_dev, std::vector<double>& w_host, DevBuf& ws,
                        int* meig_out) {
  *meig_out = 0;
  w_host.clear();
  if (n == 0 || k <= 0) return FKF_OK;
  k = std::min(k, n);
  std::vector<double> all;
  FKF_TRY(eigh_own(ctx, n, A, w_dev, all, ws, k));
  // the k largest, ascending, at the front of w
  if (k < n) {
    FKF_CUDA(ctx, cudaMemcpyAsync(w_dev, all.data() + (n - k), (size_t)k * 8, cudaMemcpyHostToDevice, ctx->stream));
    FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  w_host.assign(all.end() - k, all.end());
  *meig_out = k;
  return FKF_OK;
}

// Cholesky factorisation and solves of small SPD systems: the library's own
// blocked factorisation (chol.cu) and blocked triangular solves.
fkf_status chol_f64(fkf_ctx* ctx, int n, double* A, DevBuf& ws) { return chol_blocked_f64(ctx, n, n, A, n, ws); }

fkf_status chol_solve_f64(fkf_ctx* ctx, int n, const double* Afact, double* b, int nrhs) {
  return chol_solve_rows_f64(ctx, n, Afact, n, b, nrhs, n);
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
