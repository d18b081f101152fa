// Dense and small-matrix building blocks (device work on ctx->stream).
#pragma once

#include <vector>

#include "common.h"

// C = alpha op(A) op(B) + beta C (row-major; ta/tb select transposes).
fkf_status gemm_f64(fkf_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                    int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc);
// gemm_f64 for a symmetric N x N result (op(A) op(B) symmetric, C symmetric
// when beta != 0): computes the lower tiles and mirrors them, so C comes out
// exactly symmetric; lower_only: the lower triangle alone is written (for
// consumers that read only it, such as the blocked Cholesky).  skip in
// [0, N) (lower_only only): entries (i, j) with i, j >= skip are left as they
// were.
fkf_status gemm_sym_f64(fkf_ctx* ctx, bool ta, bool tb, int64_t N, int64_t K, double alpha, const double* A,
                        int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                        bool lower_only = false, int64_t skip = -1);
fkf_status gemm_f32(fkf_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                    int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc);
// C (M x N, FP64) = A^T B with A: K x M, B: K x N (row-major), K long.
fkf_status gram_f64(fkf_ctx* ctx, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
                    int64_t ldb, double* C, int64_t ldc, DevBuf& ws);
fkf_status gram_f32(fkf_ctx* ctx, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                    int64_t ldb, double* C, int64_t ldc, DevBuf& ws);
fkf_status scale_f64(fkf_ctx* ctx, int64_t M, int64_t N, double beta, double* C, int64_t ldc);
fkf_status scale_f32(fkf_ctx* ctx, int64_t M, int64_t N, float beta, float* C, int64_t ldc);

// Blocked Cholesky factorisation of an SPD n x n matrix (row-major, ld lda),
// stopped after its first nf pivots: the leading nf x nf block becomes the
// factor L11 (lower triangle), the rows below it L21, and the trailing block
// the Schur complement A22 - L21 L21^T (both triangles); the upper triangle of
// the factored part is overwritten with scratch.  nf = n is the full
// factorisation.  Synchronises once; FKF_ENOTSPD if a pivot is not positive.
// Pivoted (rank-revealing) Cholesky of a symmetric positive semidefinite
// n x n matrix A (row-major, lower triangle read; A is overwritten by the
// updates): A ~= Lp Lp^T with Lp = Pi L (L lower triangular in pivot order),
// pivots the largest remaining diagonal, stopping when it is <= tol or after
// max_rank pivots.  Lp: n x rank (ld ldl >= max_rank), row i of column k zero
// when i was pivoted before k.  Synchronises once per 32 pivots.
fkf_status pchol_f64(fkf_ctx* ctx, int n, double* A, int64_t lda, double tol, int max_rank, double* Lp, int64_t ldl,
                     DevBuf& ws, int* rank_out);
// schur_done (nf < n): the Schur complement is formed by one product
// A22 -= L21 L21^T on the context's low-priority stream after the
// factorisation and schur_done is recorded after it; the caller waits on it
// before reading A22 (the factor itself is complete on return).
fkf_status chol_blocked_f64(fkf_ctx* ctx, int n, int nf, double* A, int64_t lda, DevBuf& ws,
                            cudaEvent_t schur_done = nullptr);
// Solve L L^T x = b for the nrhs rows of B (nrhs x n, ld ldb), in place, with
// the lower factor of chol_blocked_f64 (ld ldl); the library's own blocked
// triangular solves.
fkf_status chol_solve_rows_f64(fkf_ctx* ctx, int n, const double* L, int64_t ldl, double* B, int nrhs, int64_t ldb);
// Solve S x = b (nrhs contiguous vectors of length n) with the factor of
// chol_blocked_f64 (ld ldl).
fkf_status chol_solve_rowlower_f64(fkf_ctx* ctx, int n, const double* L, int64_t ldl, double* b, int nrhs);

// The library's own symmetric eigensolver (eigh.cu): all n eigenvalues
// ascending into w_dev and w_host; the eigenvectors of the `want` largest into
// rows 0..want-1 of A (row q = eigenvector of w[n - want + q]).  A must be
// symmetric; ws grows to about 5 n^2 + n want doubles.  Synchronises.
fkf_status eigh_own(fkf_ctx* ctx, int n, double* A, double* w_dev, std::vector<double>& w_host, DevBuf& ws,
                    int want);
// Symmetric eigensolver (FP64): A (n x n, symmetric, row-major) is replaced
// by Vt, whose row j is the unit eigenvector of eigenvalue w[j]; eigenvalues
// ascending.  The eigenvalues are also copied to w_host (synchronises).
fkf_status eigh_f64(fkf_ctx* ctx, int n, double* A, double* w_dev, std::vector<double>& w_host, DevBuf& ws);
// The k largest eigenpairs of a symmetric n x n A (w_dev must hold n values):
// on return *meig pairs,
// eigenvalues ascending in w, eigenvector i in row i of A (row-major view).
fkf_status eigh_top_f64(fkf_ctx* ctx, int n, int k, double* A, double* w_dev, std::vector<double>& w_host, DevBuf& ws,
                        int* meig);
// Cholesky factorisation of an SPD n x n matrix in place (the library's
// blocked factorisation; lower factor, row-major); FKF_ENOTSPD when a pivot is
// not positive.
fkf_status chol_f64(fkf_ctx* ctx, int n, double* A, DevBuf& ws);
// Solve A x = b for nrhs right-hand sides stored as nrhs contiguous vectors
// of length n, with A factored by chol_f64.
fkf_status chol_solve_f64(fkf_ctx* ctx, int n, const double* Afact, double* b, int nrhs);
