// C-ABI entry points (include/fkf.h): argument checks, object lifetime,
// error reporting, and dispatch to the device implementations.
#include <cusolverDn.h>

#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>
#include <thread>
#include <algorithm>
#include <condition_variable>
#include <mutex>
#include <utility>

#include "common.h"
#include "hmat_host.h"

// filter.cu
struct fkf_filter;
fkf_status filter_create(fkf_hmat* h, const double* s0, double alpha0, double trunc_tol, int m_max, int r_max,
                         fkf_filter** out);
void filter_destroy(fkf_filter* f);
fkf_status filter_step(fkf_filter* f, const double* y, int m, const int64_t* rowptr, const int32_t* col,
                       const double* val, const double* R, double r_scalar, int flags, double* nll_out,
                       double boxcox_a);
fkf_status filter_set_refresh(fkf_filter* f, int every);
fkf_status filter_set_randomized_ghep(fkf_filter* f, int k, int p, const double* omega_dev);
fkf_status filter_get(fkf_filter* f, double* s_hat, double* alpha, int* r, double* D, void* W_dev, int64_t ldw);
fkf_status filter_variance(fkf_filter* f, double* var_dev);
fkf_status filter_realization(fkf_filter* f, const double* a_dev, int ns, double* out_dev);
fkf_status filter_uncertainty(fkf_filter* f, double* ent, double* tr);
fkf_status filter_orthonormality(fkf_filter* f, double* err);
fkf_status filter_refresh(fkf_filter* f);
fkf_status filter_checkpoint(fkf_filter* f, const char* path);
fkf_status filter_restore(fkf_filter* f, const char* path);
fkf_status filter_phase_times(fkf_filter* f, double* ms6);
fkf_status filter_set_tolerances(fkf_filter* f, double gep_tol, double orth_tol, double trunc_tol);
fkf_ctx* filter_ctx(fkf_filter* f);

fkf_status set_err(fkf_ctx* ctx, fkf_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

fkf_status dev_alloc(fkf_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return FKF_OK;
  b.release();
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, FKF_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  b.p = p;
  b.bytes = bytes;
  return FKF_OK;
}

fkf_status dev_upload(fkf_ctx* ctx, DevBuf& b, const void* host, size_t bytes) {
  FKF_TRY(dev_alloc(ctx, b, bytes));
  FKF_CUDA(ctx, cudaMemcpyAsync(b.p, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return FKF_OK;
}

#define FKF_API extern "C" __attribute__((visibility("default")))

FKF_API fkf_status fkf_create(fkf_ctx** out, int32_t device, void* cuda_stream) {
  if (!out) return FKF_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return FKF_ECUDA;
  }
  if (device < 0 || device >= ndev) return FKF_EINVAL;
  fkf_ctx* ctx = new (std::nothrow) fkf_ctx();
  if (!ctx) return FKF_ENOMEM;
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return FKF_ECUDA;
  }
  if (cuda_stream) {
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return FKF_ECUDA;
    }
    ctx->own_stream = true;
  }
  *out = ctx;
  return FKF_OK;
}

fkf_status ctx_side(fkf_ctx* ctx, size_t n_events) {
  if (!ctx->side) {
    int least = 0, greatest = 0;
    FKF_CUDA(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    FKF_CUDA(ctx, cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, greatest));
  }
  while (ctx->side_ev.size() < n_events) {
    cudaEvent_t e;
    FKF_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->side_ev.push_back(e);
  }
  return FKF_OK;
}

fkf_status ctx_side_lo(fkf_ctx* ctx) {
  if (!ctx->side_lo) {
    int least = 0, greatest = 0;
    FKF_CUDA(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    FKF_CUDA(ctx, cudaStreamCreateWithPriority(&ctx->side_lo, cudaStreamNonBlocking, least));
  }
  return FKF_OK;
}

FKF_API void fkf_destroy(fkf_ctx* ctx) {
  if (!ctx) return;
  if (ctx->side_lo) cudaStreamDestroy(ctx->side_lo);
  for (cudaEvent_t e : ctx->side_ev) cudaEventDestroy(e);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->solver) cusolverDnDestroy(reinterpret_cast<cusolverDnHandle_t>(ctx->solver));
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

FKF_API const char* fkf_last_error(const fkf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

FKF_API int64_t fkf_launch_count(const fkf_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

FKF_API int64_t fkf_library_call_count(const fkf_ctx* ctx) { return ctx ? ctx->lib_calls.load() : 0; }

FKF_API fkf_status fkf_hmatrix_build(fkf_ctx* ctx, const double* points, int64_t n, int32_t dim, fkf_matern kernel,
                                     fkf_hparams hp, fkf_precision prec, fkf_hmat** out) {
  if (!ctx || !out) return FKF_EINVAL;
  *out = nullptr;
  if (!points || n < 1) return set_err(ctx, FKF_EINVAL, "hmatrix_build: points and n >= 1 required");
  if (dim != 2 && dim != 3) return set_err(ctx, FKF_EINVAL, "hmatrix_build: dim must be 2 or 3");
  if (!(kernel.nu == 0.5 || kernel.nu == 1.5 || kernel.nu == 2.5))
    return set_err(ctx, FKF_EINVAL, "hmatrix_build: nu must be 0.5, 1.5 or 2.5");
  if (!(kernel.ell > 0) || !(kernel.sigma2 > 0))
    return set_err(ctx, FKF_EINVAL, "hmatrix_build: ell and sigma2 must be > 0");
  if (hp.leaf < 1 || !(hp.eta >= 0) || !(hp.aca_tol > 0) || hp.k_cap < 1)
    return set_err(ctx, FKF_EINVAL, "hmatrix_build: leaf >= 1, eta >= 0, aca_tol > 0, k_cap >= 1 required");
  if (prec != FKF_FP64 && prec != FKF_FP32) return set_err(ctx, FKF_EINVAL, "hmatrix_build: bad precision");
  for (int64_t i = 0; i < n * dim; i++)
    if (!std::isfinite(points[i])) return set_err(ctx, FKF_EINVAL, "hmatrix_build: non-finite coordinate");
  FKF_CUDA(ctx, cudaSetDevice(ctx->device));
  fkf_hmat* h = new (std::nothrow) fkf_hmat();
  if (!h) return set_err(ctx, FKF_ENOMEM, "host allocation");
  h->ctx = ctx;
  h->n = n;
  h->dim = dim;
  h->prec = prec;
  h->kernel = kernel;
  h->hp = hp;
  HostHmat* hh = nullptr;
  fkf_status st = hmat_build_host(ctx, points, n, dim, kernel, hp, &hh, h->perm);
  if (st == FKF_OK) st = hmat_upload(h, *hh);
  if (st == FKF_OK) {
    std::vector<int64_t> iperm(n);
    for (int64_t i = 0; i < n; i++) iperm[h->perm[i]] = i;
    st = dev_upload(ctx, h->perm_d, h->perm.data(), n * 8);
    if (st == FKF_OK) st = dev_upload(ctx, h->iperm_d, iperm.data(), n * 8);
    h->points_clustered = hh->pts;
  }
  hmat_free_host(hh);
  if (st != FKF_OK) {
    delete h;
    return st;
  }
  // panel width: keep the slot workspace under ~8 GB
  const size_t w = prec == FKF_FP64 ? 8 : 4;
  int64_t panel = 1024;
  while (panel > 128 && (double)h->ktot * panel * w > 8e9) panel /= 2;
  h->panel = panel;
  *out = h;
  return FKF_OK;
}

FKF_API fkf_status fkf_hmatrix_info(const fkf_hmat* h, fkf_hmat_info* info) {
  if (!h || !info) return FKF_EINVAL;
  *info = h->info;
  info->device_bytes = hmat_device_bytes(h);
  return FKF_OK;
}

static fkf_status check_apply_args(fkf_hmat* h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t ncols) {
  if (!X || !Y || ncols < 0 || ldx < ncols || ldy < ncols)
    return set_err(h->ctx, FKF_EINVAL, "hmatrix_apply: need X, Y, ncols >= 0, ldx >= ncols, ldy >= ncols");
  const size_t w = h->prec == FKF_FP64 ? 8 : 4;
  const char* x0 = (const char*)X;
  const char* x1 = x0 + ((h->n - 1) * ldx + ncols) * w;
  const char* y0 = (const char*)Y;
  const char* y1 = y0 + ((h->n - 1) * ldy + ncols) * w;
  if (ncols > 0 && x0 < y1 && y0 < x1) return set_err(h->ctx, FKF_EINVAL, "hmatrix_apply: X and Y overlap");
  return FKF_OK;
}

FKF_API fkf_status fkf_hmatrix_apply_clustered(fkf_hmat* h, const void* X_dev, int64_t ldx, void* Y_dev,
                                               int64_t ldy, int64_t ncols) {
  if (!h) return FKF_EINVAL;
  FKF_TRY(check_apply_args(h, X_dev, ldx, Y_dev, ldy, ncols));
  FKF_TRY(hmat_apply_clustered(h, X_dev, ldx, Y_dev, ldy, ncols));
  FKF_CUDA(h->ctx, cudaStreamSynchronize(h->ctx->stream));
  return hmat_tc_check(h);
}

FKF_API fkf_status fkf_hmatrix_get_engine(const fkf_hmat* h, int32_t* engine) {
  if (!h || !engine) return FKF_EINVAL;
  *engine = h->engine;
  return FKF_OK;
}

FKF_API fkf_status fkf_hmatrix_autotune(fkf_hmat* h, int64_t ncols, int32_t* variant, double* ms) {
  if (!h) return FKF_EINVAL;
  if (ncols < 1) return set_err(h->ctx, FKF_EINVAL, "autotune: ncols >= 1 required");
  int v = 0;
  double t = 0.0;
  FKF_TRY(hmat_autotune(h, ncols, &v, &t));
  if (variant) *variant = v;
  if (ms) *ms = t;
  return FKF_OK;
}

FKF_API fkf_status fkf_hmatrix_release_values(fkf_hmat* h) {
  if (!h) return FKF_EINVAL;
  if (h->prec != FKF_FP32 || (h->engine != 1 && h->engine != 2))
    return set_err(h->ctx, FKF_ESTATE, "release_values: an FP32 operator on a tensor-core engine (1, 2) is required");
  if (h->tca_fmt != h->engine) FKF_TRY(hmat_set_engine(h, h->engine));  // the stream the engine reads
  FKF_CUDA(h->ctx, cudaStreamSynchronize(h->ctx->stream));
  h->fac.release();
  h->nearv.release();
  h->values_released = true;
  return FKF_OK;
}

FKF_API fkf_status fkf_hmatrix_set_engine(fkf_hmat* h, int32_t engine) {
  if (!h) return FKF_EINVAL;
  if (h->values_released && engine != h->engine)
    return set_err(h->ctx, FKF_ESTATE, "set_engine: the operator's values were released");
  if (engine < 0 || engine > 3) return set_err(h->ctx, FKF_EINVAL, "set_engine: engine must be 0, 1, 2 or 3");
  if ((engine == 1 || engine == 2) && h->prec != FKF_FP32)
    return set_err(h->ctx, FKF_EINVAL, "set_engine: engines 1 and 2 need an FP32 operator");
  if (engine == 3 && h->prec != FKF_FP64)
    return set_err(h->ctx, FKF_EINVAL, "set_engine: engine 3 needs an FP64 operator");
  return hmat_set_engine(h, engine);
}

// Variant that never allocates device memory (static scratch; see fkf.h).
FKF_API fkf_status fkf_hmatrix_apply_clustered_noalloc(fkf_hmat* h, const void* X_dev, int64_t ldx, void* Y_dev,
                                                       int64_t ldy, int64_t ncols) {
  if (!h) return FKF_EINVAL;
  FKF_TRY(check_apply_args(h, X_dev, ldx, Y_dev, ldy, ncols));
  if (h->values_released)
    return set_err(h->ctx, FKF_ESTATE, "apply_noalloc: the operator's values were released");
  FKF_TRY(hmat_apply_clustered_noalloc(h, X_dev, ldx, Y_dev, ldy, ncols));
  FKF_CUDA(h->ctx, cudaStreamSynchronize(h->ctx->stream));
  return FKF_OK;
}

FKF_API fkf_status fkf_rotate_f32(fkf_ctx* ctx, const float* A_dev, int64_t lda, int64_t rows, int32_t K,
                                  const float* E_dev, int64_t lde, int64_t ke, int32_t ncols, float* C_dev,
                                  int64_t ldc) {
  if (!ctx) return FKF_EINVAL;
  if (rows < 0 || K < 0 || ke < K || ncols < 0 || lda < K || lde < ncols || ldc < ncols)
    return set_err(ctx, FKF_EINVAL, "fkf_rotate_f32: bad sizes");
  if (rows == 0 || ncols == 0) return FKF_OK;
  if (!A_dev || !E_dev || !C_dev) return set_err(ctx, FKF_EINVAL, "fkf_rotate_f32: null pointer");
  auto span = [](const float* p, int64_t nr, int64_t ld, int64_t nc) {
    const char* b = reinterpret_cast<const char*>(p);
    return std::make_pair(b, b + ((nr - 1) * ld + nc) * (int64_t)sizeof(float));
  };
  auto overlap = [](std::pair<const char*, const char*> a, std::pair<const char*, const char*> b) {
    return a.first < b.second && b.first < a.second;
  };
  const auto c = span(C_dev, rows, ldc, ncols);
  if ((K > 0 && overlap(c, span(A_dev, rows, lda, K))) || (K > 0 && overlap(c, span(E_dev, K, lde, ncols))))
    return set_err(ctx, FKF_EINVAL, "fkf_rotate_f32: C overlaps A or E");
  const TcGemmProblem p{A_dev, lda, rows, K, C_dev, ldc};
  FKF_TRY(tc_gemm_f32(ctx, &p, 1, E_dev, lde, ke, ncols, ctx->gemm_ws));
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  FKF_CUDA(ctx, cudaGetLastError());
  return tc_gemm_check(ctx, ctx->gemm_ws);
}

FKF_API fkf_status fkf_gemm_f64(fkf_ctx* ctx, int32_t trans_a, int32_t trans_b, int64_t M, int64_t N, int64_t K,
                                double alpha, const double* A_dev, int64_t lda, const double* B_dev, int64_t ldb,
                                double beta, double* C_dev, int64_t ldc) {
  if (!ctx) return FKF_EINVAL;
  if (M < 0 || N < 0 || K < 0 || ldc < N || lda < (trans_a ? M : K) || ldb < (trans_b ? K : N))
    return set_err(ctx, FKF_EINVAL, "fkf_gemm_f64: bad sizes");
  if (M == 0 || N == 0) return FKF_OK;
  if (!C_dev || (K > 0 && (!A_dev || !B_dev))) return set_err(ctx, FKF_EINVAL, "fkf_gemm_f64: null pointer");
  auto span = [](const double* p, int64_t nr, int64_t ld, int64_t nc) {
    const char* b = reinterpret_cast<const char*>(p);
    return std::make_pair(b, b + ((nr - 1) * ld + nc) * (int64_t)sizeof(double));
  };
  auto overlap = [](std::pair<const char*, const char*> a, std::pair<const char*, const char*> b) {
    return a.first < b.second && b.first < a.second;
  };
  const auto c = span(C_dev, M, ldc, N);
  if (K > 0 && (overlap(c, trans_a ? span(A_dev, K, lda, M) : span(A_dev, M, lda, K)) ||
                overlap(c, trans_b ? span(B_dev, N, ldb, K) : span(B_dev, K, ldb, N))))
    return set_err(ctx, FKF_EINVAL, "fkf_gemm_f64: C overlaps A or B");
  FKF_TRY(gemm_f64_tc(ctx, trans_a != 0, trans_b != 0, M, N, K, alpha, A_dev, lda, B_dev, ldb, beta, C_dev, ldc));
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  FKF_CUDA(ctx, cudaGetLastError());
  return gemm_f64_tc_check(ctx);
}

FKF_API fkf_status fkf_hmatrix_apply(fkf_hmat* h, const void* X_dev, int64_t ldx, void* Y_dev, int64_t ldy,
                                     int64_t ncols) {
  if (!h) return FKF_EINVAL;
  FKF_TRY(check_apply_args(h, X_dev, ldx, Y_dev, ldy, ncols));
  if (ncols == 0) return FKF_OK;
  fkf_ctx* ctx = h->ctx;
  const size_t w = h->prec == FKF_FP64 ? 8 : 4;
  const size_t need = (size_t)h->n * ncols * w;
  FKF_TRY(dev_alloc(ctx, h->xperm, need));
  FKF_TRY(dev_alloc(ctx, h->yperm, need));
  FKF_TRY(hmat_permute_rows(h, X_dev, ldx, h->perm_d.as<int64_t>(), h->xperm.p, ncols, h->n, ncols));
  FKF_TRY(hmat_apply_clustered(h, h->xperm.p, ncols, h->yperm.p, ncols, ncols));
  FKF_TRY(hmat_permute_rows(h, h->yperm.p, ncols, h->iperm_d.as<int64_t>(), Y_dev, ldy, h->n, ncols));
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return hmat_tc_check(h);
}

FKF_API fkf_status fkf_hmatrix_apply_adjoint(fkf_hmat* h, const void* gY_dev, int64_t ldg, const void* Y_dev,
                                             int64_t ldy, void* gX_dev, int64_t ldgx, int64_t ncols,
                                             double* grad_sigma2) {
  if (!h) return FKF_EINVAL;
  FKF_TRY(fkf_hmatrix_apply(h, gY_dev, ldg, gX_dev, ldgx, ncols));
  if (grad_sigma2) {
    if (!Y_dev || ldy < ncols) return set_err(h->ctx, FKF_EINVAL, "hmatrix_apply_adjoint: Y_dev, ldy >= ncols required");
    double dot = 0;
    if (ncols > 0) FKF_TRY(hmat_dot(h, gY_dev, ldg, Y_dev, ldy, h->n, ncols, &dot));
    *grad_sigma2 = dot / h->kernel.sigma2;
  }
  return FKF_OK;
}

fkf_status eigh_own(fkf_ctx* ctx, int n, double* A, double* w_dev, std::vector<double>& w_host, DevBuf& ws,
                    int want);

FKF_API fkf_status fkf_eigh(fkf_ctx* ctx, int32_t n, double* A_dev, double* w_dev, int32_t want) {
  if (!ctx) return FKF_EINVAL;
  if (n < 0 || !A_dev || !w_dev || want < 0 || want > n)
    return set_err(ctx, FKF_EINVAL, "eigh: n >= 0, 0 <= want <= n and device pointers required");
  FKF_CUDA(ctx, cudaSetDevice(ctx->device));
  std::vector<double> w;
  DevBuf ws;
  return eigh_own(ctx, n, A_dev, w_dev, w, ws, want);
}

FKF_API fkf_status fkf_hmatrix_set_wait_limit(fkf_hmat* h, int64_t polls) {
  if (!h) return FKF_EINVAL;
  if (polls > 0xffffffffLL) return set_err(h->ctx, FKF_EINVAL, "set_wait_limit: polls <= 2^32 - 1 required");
  h->tc_polls = polls < 0 ? (1u << 22) : (uint32_t)polls;
  return FKF_OK;
}

FKF_API fkf_status fkf_hmatrix_permutation(const fkf_hmat* h, int64_t* perm_host) {
  if (!h || !perm_host) return FKF_EINVAL;
  std::memcpy(perm_host, h->perm.data(), h->n * sizeof(int64_t));
  return FKF_OK;
}

FKF_API fkf_status fkf_hmatrix_densify(fkf_hmat* h, double* out_host) {
  if (!h || !out_host) return FKF_EINVAL;
  fkf_ctx* ctx = h->ctx;
  const int64_t n = h->n;
  if (n > 8192) return set_err(ctx, FKF_EINVAL, "hmatrix_densify: N <= 8192 required");
  const size_t w = h->prec == FKF_FP64 ? 8 : 4;
  const int64_t cb = std::min<int64_t>(n, 1024);
  DevBuf X, Y;
  FKF_TRY(dev_alloc(ctx, X, (size_t)n * cb * w));
  FKF_TRY(dev_alloc(ctx, Y, (size_t)n * cb * w));
  std::vector<char> hx((size_t)n * cb * w), hy((size_t)n * cb * w);
  for (int64_t c0 = 0; c0 < n; c0 += cb) {
    const int64_t nc = std::min<int64_t>(cb, n - c0);
    std::memset(hx.data(), 0, hx.size());
    for (int64_t j = 0; j < nc; j++) {
      if (w == 8)
        reinterpret_cast<double*>(hx.data())[(c0 + j) * nc + j] = 1.0;
      else
        reinterpret_cast<float*>(hx.data())[(c0 + j) * nc + j] = 1.0f;
    }
    FKF_CUDA(ctx, cudaMemcpyAsync(X.p, hx.data(), (size_t)n * nc * w, cudaMemcpyHostToDevice, ctx->stream));
    FKF_TRY(fkf_hmatrix_apply(h, X.p, nc, Y.p, nc, nc));
    FKF_CUDA(ctx, cudaMemcpyAsync(hy.data(), Y.p, (size_t)n * nc * w, cudaMemcpyDeviceToHost, ctx->stream));
    FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int64_t i = 0; i < n; i++)
      for (int64_t j = 0; j < nc; j++)
        out_host[i * n + c0 + j] = w == 8 ? reinterpret_cast<double*>(hy.data())[i * nc + j]
                                          : (double)reinterpret_cast<float*>(hy.data())[i * nc + j];
  }
  return FKF_OK;
}

FKF_API void fkf_hmatrix_destroy(fkf_hmat* h) { delete h; }

FKF_API fkf_status fkf_filter_create(fkf_hmat* h, const double* s0, double alpha0, double trunc_tol, int32_t m_max,
                                     int32_t r_max, fkf_filter** out) {
  if (!h || !out) return FKF_EINVAL;
  *out = nullptr;
  FKF_CUDA(h->ctx, cudaSetDevice(h->ctx->device));
  return filter_create(h, s0, alpha0, trunc_tol, m_max, r_max, out);
}

FKF_API void fkf_filter_destroy(fkf_filter* f) { filter_destroy(f); }

FKF_API fkf_status fkf_filter_step(fkf_filter* f, const double* y, int32_t m, const int64_t* H_rowptr,
                                   const int32_t* H_col, const double* H_val, const double* R, double r_scalar,
                                   int32_t flags, double* nll_out) {
  if (!f) return FKF_EINVAL;
  if (!y || !H_rowptr || (!H_col && m > 0) || (!H_val && m > 0))
    return set_err(filter_ctx(f), FKF_EINVAL, "filter_step: null input pointer");
  return filter_step(f, y, m, H_rowptr, H_col, H_val, R, r_scalar, flags, nll_out, 0.0);
}

FKF_API fkf_status fkf_filter_step_ekf(fkf_filter* f, const double* y, int32_t m, const int64_t* H_rowptr,
                                       const int32_t* H_col, const double* H_val, const double* R, double r_scalar,
                                       double boxcox_a, int32_t flags, double* nll_out) {
  if (!f) return FKF_EINVAL;
  if (!y || !H_rowptr || (!H_col && m > 0) || (!H_val && m > 0))
    return set_err(filter_ctx(f), FKF_EINVAL, "filter_step_ekf: null input pointer");
  if (!(boxcox_a > 0.0)) return set_err(filter_ctx(f), FKF_EINVAL, "filter_step_ekf: Box-Cox parameter a > 0 required");
  return filter_step(f, y, m, H_rowptr, H_col, H_val, R, r_scalar, flags, nll_out, boxcox_a);
}

FKF_API fkf_status fkf_filter_set_randomized_ghep(fkf_filter* f, int32_t k, int32_t p, const double* omega_dev) {
  if (!f) return FKF_EINVAL;
  return filter_set_randomized_ghep(f, k, p, omega_dev);
}

FKF_API fkf_status fkf_filter_set_refresh(fkf_filter* f, int32_t every) {
  if (!f) return FKF_EINVAL;
  return filter_set_refresh(f, every);
}

// ---- merged H-applies of a batch of steps ------------------------------------
// Every step of fkf_filter_step_batched runs on its own host thread.  A step
// that reaches its H-apply (S2) registers the request here and waits; a step
// that ends without one (an error, or the products reused) withdraws.  When
// every step has registered or withdrawn, the last thread issues one merged
// launch per phase for all registered applies on the first requester's
// stream (after each requester's stream reached its apply), and every
// requester's stream then waits for it.  Operators that cannot be merged are
// applied one by one on their own streams.
namespace {
struct ApplyBatch {
  struct Req {
    fkf_hmat* h;
    const float* X;
    int64_t ldx;
    float* Y;
    int64_t ldy;
    int64_t ncols;
    cudaEvent_t ready;
  };
  std::mutex mu;
  std::condition_variable cv;
  int expected = 0, arrived = 0, left = 0;
  bool finished = false;
  fkf_status status = FKF_OK;
  std::vector<Req> reqs;
  std::vector<cudaEvent_t> evs;  // one per step (ready) + done
  cudaEvent_t done = nullptr;
  std::vector<bool> merged_req;  // per request: its apply ran in the merged launch

  // with mu held, once every step has registered or withdrawn
  void run() {
    if (reqs.empty()) {
      finished = true;
      return;
    }
    std::vector<fkf_hmat*> hs;
    std::vector<const float*> X;
    std::vector<float*> Y;
    std::vector<int64_t> ldx, ldy, nc;
    for (const Req& r : reqs) {
      hs.push_back(r.h);
      X.push_back(r.X);
      Y.push_back(r.Y);
      ldx.push_back(r.ldx);
      ldy.push_back(r.ldy);
      nc.push_back(r.ncols);
    }
    // the requests that fit one merged launch with the first one (same tensor-core format,
    // pipeline shape and device, one column pass each); the others are applied one by one
    // (the largest such group, whatever order the requests arrived in)
    merged_req.assign(reqs.size(), false);
    std::vector<size_t> idx;
    for (size_t k = 0; k < reqs.size(); k++) {
      if (!hmat_tc_multi_ok(&hs[k], 1, &nc[k])) continue;
      std::vector<size_t> g{k};
      for (size_t i = 0; i < reqs.size(); i++) {
        if (i == k) continue;
        fkf_hmat* pair[2] = {hs[k], hs[i]};
        const int64_t pnc[2] = {nc[k], nc[i]};
        if (hmat_tc_multi_ok(pair, 2, pnc)) g.push_back(i);
      }
      if (g.size() > idx.size()) idx.swap(g);
    }
    std::sort(idx.begin(), idx.end());
    fkf_status st = FKF_OK;
    if (idx.size() > 1) {
      std::vector<fkf_hmat*> mh;
      std::vector<const float*> mX;
      std::vector<float*> mY;
      std::vector<int64_t> mldx, mldy, mnc;
      for (size_t i : idx) {
        mh.push_back(hs[i]);
        mX.push_back(X[i]);
        mY.push_back(Y[i]);
        mldx.push_back(ldx[i]);
        mldy.push_back(ldy[i]);
        mnc.push_back(nc[i]);
      }
      fkf_ctx* lctx = reqs[idx[0]].h->ctx;
      if (cudaSetDevice(lctx->device) != cudaSuccess) st = set_err(lctx, FKF_ECUDA, "cudaSetDevice failed");
      for (size_t i : idx)
        if (st == FKF_OK && cudaStreamWaitEvent(lctx->stream, reqs[i].ready, 0) != cudaSuccess)
          st = set_err(lctx, FKF_ECUDA, "batched apply: stream wait failed");
      if (st == FKF_OK)
        st = hmat_apply_tc_multi(lctx, mh.data(), (int)mh.size(), mX.data(), mldx.data(), mY.data(), mldy.data(),
                                 mnc.data());
      if (st == FKF_OK && cudaEventRecord(done, lctx->stream) != cudaSuccess)
        st = set_err(lctx, FKF_ECUDA, "batched apply: event record failed");
      for (size_t i : idx) merged_req[i] = true;
    }
    for (size_t i = 0; i < reqs.size(); i++)
      if (st == FKF_OK && !merged_req[i])
        st = hmat_apply_clustered(reqs[i].h, reqs[i].X, reqs[i].ldx, reqs[i].Y, reqs[i].ldy, reqs[i].ncols);
    status = st;
    finished = true;
  }

  bool merged_of(fkf_hmat* h) const {
    for (size_t i = 0; i < reqs.size(); i++)
      if (reqs[i].h == h) return merged_req[i];
    return false;
  }

  fkf_status apply(const Req& req) {
    std::unique_lock<std::mutex> lk(mu);
    reqs.push_back(req);
    arrived++;
    if (arrived + left == expected)
      run();
    else
      cv.wait(lk, [&] { return finished; });
    lk.unlock();
    cv.notify_all();
    return status;
  }

  void withdraw() {
    std::unique_lock<std::mutex> lk(mu);
    left++;
    if (arrived + left == expected && !finished) run();
    lk.unlock();
    cv.notify_all();
  }
};

thread_local ApplyBatch* tls_batch = nullptr;
thread_local int tls_batch_index = -1;
thread_local bool tls_batch_arrived = false;
thread_local fkf_hmat* tls_batch_h = nullptr;  // the operator of this thread's batched apply
}  // namespace

fkf_status hmat_apply_step(fkf_hmat* h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t ncols) {
  ApplyBatch* b = tls_batch;
  if (!b || tls_batch_arrived || h->prec != FKF_FP32 || h->engine == 0)
    return hmat_apply_clustered(h, X, ldx, Y, ldy, ncols);
  tls_batch_arrived = true;
  tls_batch_h = h;
  fkf_ctx* ctx = h->ctx;
  const cudaEvent_t ready = b->evs[tls_batch_index];
  FKF_CUDA(ctx, cudaEventRecord(ready, ctx->stream));
  const fkf_status st =
      b->apply({h, static_cast<const float*>(X), ldx, static_cast<float*>(Y), ldy, ncols, ready});
  if (st != FKF_OK) return set_err(ctx, st, "batched H-apply failed");
  if (b->merged_of(h)) FKF_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, b->done, 0));
  return FKF_OK;
}

FKF_API fkf_status fkf_filter_step_batched(fkf_step_desc* descs, int32_t nb, int32_t flags) {
  if (!descs || nb < 1) return FKF_EINVAL;
  std::vector<fkf_ctx*> ctxs(nb);
  for (int i = 0; i < nb; i++) {
    if (!descs[i].filter) return FKF_EINVAL;
    ctxs[i] = filter_ctx(descs[i].filter);
    for (int j = 0; j < i; j++)
      if (ctxs[j] == ctxs[i]) return set_err(ctxs[i], FKF_EINVAL, "step_batched: filters %d and %d share a context", j, i);
  }
  ApplyBatch batch;
  batch.expected = nb;
  batch.evs.resize(nb + 1, nullptr);
  for (int i = 0; i <= nb; i++)
    if (cudaSetDevice(ctxs[std::min(i, nb - 1)]->device) != cudaSuccess ||
        cudaEventCreateWithFlags(&batch.evs[i], cudaEventDisableTiming) != cudaSuccess) {
      for (int j = 0; j < i; j++) cudaEventDestroy(batch.evs[j]);
      return set_err(ctxs[0], FKF_ECUDA, "step_batched: event creation failed");
    }
  batch.done = batch.evs[nb];
  // one host thread per step: a step waits in its H-apply for the others
  auto worker = [&](int i) {
    fkf_step_desc& d = descs[i];
    fkf_ctx* ctx = ctxs[i];
    tls_batch = &batch;
    tls_batch_index = i;
    tls_batch_arrived = false;
    tls_batch_h = nullptr;
    fkf_status st = FKF_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) st = set_err(ctx, FKF_ECUDA, "cudaSetDevice failed");
    if (st == FKF_OK)
      st = fkf_filter_step(d.filter, d.y, d.m, d.H_rowptr, d.H_col, d.H_val, d.R, d.r_scalar, flags, &d.nll);
    if (!tls_batch_arrived) batch.withdraw();
    d.merged = tls_batch_arrived && batch.merged_of(tls_batch_h) ? 1 : 0;
    tls_batch = nullptr;
    d.status = st;
  };
  std::vector<std::thread> pool;
  for (int i = 0; i < nb; i++) pool.emplace_back(worker, i);
  for (auto& t : pool) t.join();
  for (cudaEvent_t e : batch.evs) cudaEventDestroy(e);
  for (int i = 0; i < nb; i++)
    if (descs[i].status != FKF_OK) return (fkf_status)descs[i].status;
  return FKF_OK;
}

FKF_API fkf_status fkf_filter_get(fkf_filter* f, double* s_hat, double* alpha, int32_t* r, double* D, void* W_dev,
                                  int64_t ldw) {
  if (!f) return FKF_EINVAL;
  return filter_get(f, s_hat, alpha, r, D, W_dev, ldw);
}

FKF_API fkf_status fkf_variance(fkf_filter* f, double* var_dev) {
  if (!f || !var_dev) return FKF_EINVAL;
  return filter_variance(f, var_dev);
}

FKF_API fkf_status fkf_conditional_realization(fkf_filter* f, const double* a_dev, int32_t ns, double* out_dev) {
  if (!f || !a_dev || !out_dev) return FKF_EINVAL;
  return filter_realization(f, a_dev, ns, out_dev);
}

FKF_API fkf_status fkf_uncertainty_scalars(fkf_filter* f, double* rel_entropy, double* trace_sigma) {
  if (!f) return FKF_EINVAL;
  return filter_uncertainty(f, rel_entropy, trace_sigma);
}

FKF_API fkf_status fkf_filter_orthonormality(fkf_filter* f, double* max_abs_err) {
  if (!f || !max_abs_err) return FKF_EINVAL;
  return filter_orthonormality(f, max_abs_err);
}

FKF_API fkf_status fkf_filter_refresh(fkf_filter* f) {
  if (!f) return FKF_EINVAL;
  return filter_refresh(f);
}

FKF_API fkf_status fkf_filter_checkpoint(fkf_filter* f, const char* path) {
  if (!f || !path) return FKF_EINVAL;
  return filter_checkpoint(f, path);
}

FKF_API fkf_status fkf_filter_restore(fkf_filter* f, const char* path) {
  if (!f || !path) return FKF_EINVAL;
  return filter_restore(f, path);
}

fkf_status filter_nll_gradient(fkf_hmat* h, int K, int m, const double* y, const int64_t* rowptr, const int32_t* col,
                               const double* val, double rho, const double* s0, double alpha0, double* nll,
                               double* gy, double* gs0, double* gsig, double* grho);

FKF_API fkf_status fkf_nll_gradient(fkf_hmat* h, int32_t K, int32_t m, const double* y, const int64_t* H_rowptr,
                                    const int32_t* H_col, const double* H_val, double rho, const double* s0,
                                    double alpha0, double* nll_out, double* grad_y, double* grad_s0,
                                    double* grad_sigma2, double* grad_rho) {
  if (!h) return FKF_EINVAL;
  if (!y || !H_rowptr || !H_col || !H_val) return set_err(h->ctx, FKF_EINVAL, "nll_gradient: null input pointer");
  return filter_nll_gradient(h, K, m, y, H_rowptr, H_col, H_val, rho, s0, alpha0, nll_out, grad_y, grad_s0,
                             grad_sigma2, grad_rho);
}

void filter_stats(const fkf_filter* f, fkf_filter_stats* s);

FKF_API fkf_status fkf_filter_get_stats(const fkf_filter* f, fkf_filter_stats* out) {
  if (!f || !out) return FKF_EINVAL;
  filter_stats(f, out);
  return FKF_OK;
}

FKF_API fkf_status fkf_filter_set_tolerances(fkf_filter* f, double gep_tol, double orth_tol, double trunc_tol) {
  if (!f) return FKF_EINVAL;
  return filter_set_tolerances(f, gep_tol, orth_tol, trunc_tol);
}

FKF_API fkf_status fkf_filter_phase_times(fkf_filter* f, double* ms6) {
  if (!f || !ms6) return FKF_EINVAL;
  return filter_phase_times(f, ms6);
}
