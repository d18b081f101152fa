// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/fkf.h"

struct cusolverDnContext;

// A device buffer owned by the library.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};


// Workspace of the tensor-core dense GEMM (split operands, error flag and
// tile counter).
struct TcGemmWs {
  DevBuf asplit, bsplit, ctl, scales;
};

// Workspace of the merged multi-operator H-apply (job lists and their host
// staging, tile counters and error flag).
struct TcMultiWs {
  DevBuf jobs, ctl;
  void* staging = nullptr;  // pinned host copy of the job lists
  size_t staging_bytes = 0;
  cudaEvent_t staged = nullptr;  // the last upload from the staging buffer completed
  ~TcMultiWs() {
    if (staging) cudaFreeHost(staging);
    if (staged) cudaEventDestroy(staged);
  }
};

// Workspace of the FP64 GEMM on the tensor cores (sliced operands, scales,
// error flag and tile counter).
struct OzGemmWs {
  DevBuf as, bs, sc, ctl;
};

struct TcSparseX;  // a sparse X for the tensor-core H-apply (below)

struct fkf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  cusolverDnContext* solver = nullptr;
  std::atomic<int64_t> launches{0};   // kernels of this library
  std::atomic<int64_t> lib_calls{0};  // cuSOLVER routine calls
  DevBuf solver_info;  // status word for cuSOLVER calls
  TcGemmWs gemm_ws;    // fkf_rotate_f32
  OzGemmWs ozgemm_ws;  // FP64 GEMMs on the tensor cores (gemm_f64_tc) on the context stream
  OzGemmWs ozgemm_ws_lo;  // the same on the low-priority stream (concurrent with the context stream)
  // Whether the dense FP64 algebra may run its large products on the tensor
  // cores (49-bit slices; gemm_f64_tc).  Filters with an FP64 state clear it for
  // the duration of their operations: there the products with cancellation
  // (Schur complements, I - P^T P, basis tests) keep exact FP64 arithmetic.
  bool fp64_tc = true;
  cudaStream_t side = nullptr;        // high-priority second stream for critical-path work (created on first use)
  cudaStream_t side_lo = nullptr;     // low-priority stream for work that fills SMs beside a persistent kernel
  // When set, the tensor-core H-apply on this context records ph2_mark on the
  // context stream just before its last phase-2 launch and sets ph2_marked.
  cudaEvent_t ph2_mark = nullptr;
  bool ph2_marked = false;
  // When set, the column maxima of |X| for the tensor-core H-apply's split of
  // X (ncols unsigned, ordered float bits), already computed on the context
  // stream by the caller: the apply uses them instead of scanning X.
  const unsigned* x_colmax = nullptr;
  // When set (with x_colmax), X of the next tensor-core H-apply on this
  // context is this sparse matrix and the X argument is not read: the FP16
  // split engine scatters its entries straight into the split format.
  const TcSparseX* x_sparse = nullptr;
  std::vector<cudaEvent_t> side_ev;   // events ordering the two streams
  TcMultiWs multi_ws;                 // merged H-applies of batched steps launched on this context
};

// Second stream of the context and at least n events (created on first use).
fkf_status ctx_side(fkf_ctx* ctx, size_t n_events);
// The context's low-priority stream (created on first use).
fkf_status ctx_side_lo(fkf_ctx* ctx);

// Error plumbing: every internal function returns fkf_status and records a
// message on the context.
fkf_status set_err(fkf_ctx* ctx, fkf_status st, const char* fmt, ...);

#define FKF_CUDA(ctx, expr)                                                                             \
  do {                                                                                                  \
    cudaError_t e_ = (expr);                                                                            \
    if (e_ != cudaSuccess) {                                                                            \
      cudaGetLastError(); /* a failed call's error must not surface again at a later launch check */    \
      return set_err((ctx), e_ == cudaErrorMemoryAllocation ? FKF_ENOMEM : FKF_ECUDA, "%s: %s (%s:%d)", \
                     #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                                \
    }                                                                                                   \
  } while (0)

#define FKF_TRY(expr)               \
  do {                              \
    fkf_status s_ = (expr);         \
    if (s_ != FKF_OK) return s_;    \
  } while (0)

// Check the most recent launch.
#define FKF_LAUNCHED(ctx)                                                                    \
  do {                                                                                       \
    (ctx)->launches++;                                                                       \
    cudaError_t e_ = cudaGetLastError();                                                     \
    if (e_ != cudaSuccess)                                                                   \
      return set_err((ctx), FKF_ECUDA, "launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, \
                     __LINE__);                                                              \
  } while (0)

fkf_status dev_alloc(fkf_ctx* ctx, DevBuf& b, size_t bytes);  // grows, keeps nothing
fkf_status dev_upload(fkf_ctx* ctx, DevBuf& b, const void* host, size_t bytes);

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ----------------------------------------------------------------------------
// H-matrix, device side
// ----------------------------------------------------------------------------
// Phase-1 work item: rows [r0, r0+nr) of cluster c, slot tile [q0, q0+nq).
struct P1Item {
  int64_t fac_off;   // element offset of Fac_c (|c| x K_c, row-major)
  int64_t x_row;     // first row of X (cluster order) = c.begin + r0
  int64_t out_row;   // first output row: partial buffer row, or -1 => scatter via map
  int64_t map_off;   // global slot index of slot q0 (for the scatter map)
  int32_t K;         // K_c (row stride of Fac_c)
  int32_t r0, nr;    // row range inside the cluster
  int32_t q0, nq;    // slot range
  int32_t nchunk;    // tensor-core engine: K-chunks of 16 rows
  int64_t a_chunk0;  // tensor-core engine: first chunk of the item's split operator stream
};

// Phase-1b reduction item: sum `nch` partials of nq slots x panel, scatter.
struct P1Reduce {
  int64_t part_row;  // first partial row (chunk-major: chunk j at part_row + j*nq)
  int64_t map_off;   // global slot index of the first slot
  int32_t nq, nch;
};

// Phase-2 segment: Y_tau += A (|tau| x K, row-major, lda) * B (K rows, ldb = panel)
struct P2Seg {
  int64_t a_off;     // element offset into Fac (far) or Near (near)
  int64_t b_row;     // first row of the B operand (Zmix row for far, X row for near)
  int32_t lda;
  int32_t K;
  int32_t near;      // 0: A in Fac, B in Zmix; 1: A in Near, B in X
  int32_t pad;
};

struct P2Leaf {
  int64_t row0;      // first row of the leaf (cluster order)
  int32_t rows;      // |tau|
  int32_t seg0, nseg;
  int32_t pad;
};

// Tensor-core phase-2 tile: 128 consecutive rows (whole leaves packed) and
// its merged segment list.
// Tensor-core phase-2 segment: rows [row_lo, row_hi) of the tile times the
// segment's A block (a_off addresses the A row of tile row row_lo, row
// stride lda) and its B operand: K rows starting at the split-vector chunk
// b_row (of X if near, else of the slot workspace).  A near segment may hold
// a second row range [row_lo2, row_hi2) with its own A block (a_off2, lda2):
// two leaves of a tile that share a near partner read its X chunks once, and
// the rows of a leaf without that partner stay zero.
struct TcSeg {
  int64_t a_off;
  int64_t b_row;
  int32_t lda;
  int32_t K;
  int32_t near;
  int32_t row_lo, row_hi;
  int32_t lda2;
  int64_t a_off2;
  int32_t row_lo2, row_hi2;  // empty when equal
};

struct TcTile {
  int64_t row0;
  int64_t a_chunk0;  // first chunk of the tile's split operator stream
  int32_t rows;
  int32_t seg0, nseg;
  int32_t nchunk;    // K-chunks of 16 over all segments
};

// One 128 x 16 chunk of a split operator stream: element (i, k) is
// src[src_off + (i - row_lo) * si + k * sk] for row_lo <= i < row_hi,
// src[src_off2 + (i - row_lo2) * si2 + k * sk] for row_lo2 <= i < row_hi2,
// and k < kv, zero elsewhere (src = the far factors, or the near blocks if
// near).
// For the scaled FP16 format, row i is scaled by the scale of natural slot
// s_off + i (phase 1) or of point s_off + i (phase 2), and column k of a far
// phase-2 chunk by the inverse scale of slot-workspace position k_off + k.
struct TcAChunk {
  int64_t src_off;
  int64_t s_off;
  int64_t k_off;   // -1: no column scale
  int32_t si, sk;
  int32_t row_lo, row_hi;
  int32_t kv, near;
  int32_t phase, si2;
  int64_t src_off2;
  int32_t row_lo2, row_hi2;  // second row range (empty when equal)
};

// One 16-row chunk of the split X operand: rows row0 .. row0 + rows - 1 of X
// (cluster order), zero rows after them.
struct TcXChunk {
  int64_t row0;
  int32_t rows, pad;
};

// Host-side tensor-core schedule handed from the upload to happly_tc.cu.
// Phase-1 items: x_row = first X chunk, nchunk = its chunk count; their
// operator chunks in item_chunks.  slotmap[g] = position (chunk * 16 + row)
// of the partner of natural slot g in the split slot workspace.
struct TcUpload {
  std::vector<P1Item> items;
  std::vector<std::vector<TcAChunk>> item_chunks;
  std::vector<P1Reduce> reduces;
  std::vector<TcTile> tiles;
  std::vector<TcSeg> segs;
  std::vector<TcXChunk> xmap;
  std::vector<int64_t> slotmap;
  int64_t nz = 0, part_rows = 0;
};

// ---- FP64 operators on the tensor cores (engine 3, happly_oz.cu) ----------
// Products of FP64 values from exact products of 7-bit integer slices (FP16
// MMAs, FP32 accumulation that stays exact per K-block).  The vector
// operand (X, or the slot workspace) is the MMA's A: 128 vector columns x 16
// K per chunk; the operator is B: 64 rows (slots in phase 1, points in phase
// 2) x 16 K per chunk.  Vector chunks are indexed chunk * nct + column tile.
struct OzItem {      // phase 1: slots [q0, q0 + nq) of a cluster times the X rows of a leaf group
  int64_t x_chunk0;  // first X chunk of the group
  int64_t b_chunk0;  // first operator chunk of the item
  int64_t map_off;   // natural slot of slot q0
  int64_t out_row;   // -1: the slot workspace; else first row of the FP64 partials
  int32_t nchunk;    // K-chunks
  int32_t nq;        // slots (<= 64)
};
struct OzTile {      // phase 2: up to 64 consecutive points of one leaf
  int64_t row0;
  int64_t b_chunk0;
  int32_t rows, seg0, nseg, nchunk;
};
struct OzSeg {       // phase-2 segment: nch vector chunks from chunk a0 (of X if near, else of the workspace)
  int64_t a0;
  int32_t nch, near;
};
// One operator chunk: element (n, k) = src[src_off + n * si + k * sk] for
// n < rows, k < kv (src = the far factors, or the near blocks if near), times
// the workspace-position bound of column k (k_off + k) for far phase-2
// chunks, over the power-of-two scale of row n (natural slot s_off + n in
// phase 1, point s_off + n in phase 2); zero elsewhere.
struct OzBChunk {
  int64_t src_off;
  int64_t s_off;
  int64_t k_off;  // -1: no column factor
  int32_t si, sk;
  int32_t rows, kv;
  int32_t near, phase;
};
// Host-side schedule and scales of engine 3, handed from the upload.
struct OzUpload {
  std::vector<OzItem> items;
  std::vector<P1Reduce> reduces;
  std::vector<OzTile> tiles;
  std::vector<OzSeg> segs;
  std::vector<OzBChunk> bchunks;
  std::vector<TcXChunk> xmap;
  std::vector<int64_t> slotpos;      // natural slot -> workspace position of its partner
  std::vector<double> sig_slot;      // per natural slot: power of two >= max |V| of its column
  std::vector<double> q_slot;        // per natural slot: power of two >= the column's L1 norm
  std::vector<int32_t> q_shift;      // per natural slot: log2(q_slot / sig_slot) >= 0
  std::vector<double> q_pos;         // per workspace position: q_slot of the slot whose product lands there
  std::vector<double> sig_pt;        // per point: power of two >= max |phase-2 operator row element|
  int64_t nz = 0, part_rows = 0;
};

struct HostHmat;  // host-side build result (hbuild.cpp)

struct fkf_hmat {
  fkf_ctx* ctx = nullptr;
  int64_t n = 0;
  int dim = 0;
  fkf_precision prec = FKF_FP64;
  fkf_matern kernel{};
  fkf_hparams hp{};
  fkf_hmat_info info{};
  std::vector<int64_t> perm;  // perm[i] = original index of cluster-order point i
  std::vector<double> points_clustered;  // N x dim in cluster order
  // device operator
  DevBuf fac, nearv;          // factor stacks, near stacks (element type = precision)
  DevBuf p1items, p1red, p2seg, p2leaf, slotmap;  // schedules
  DevBuf perm_d, iperm_d;     // int64
  int64_t n_p1 = 0, n_p1red = 0, n_leaf = 0, ktot = 0, part_rows = 0;
  int32_t max_leaf = 0;
  // tensor-core schedules (FP32 operators)
  DevBuf tcp1, tcred, tctile, tcseg, tc_err;
  DevBuf tca;  // split operator streams: one chunk per 128 x 16 block (hi | lo, tensor-core smem layout)
  DevBuf tcadesc;  // TcAChunk per chunk of tca
  DevBuf tcxmap, tcslot;  // TcXChunk per X chunk; split-workspace position per natural slot
  DevBuf xsplit, zsplit;  // split X and slot workspace, per (chunk, 256-column tile)
  // scaled FP16 format: power-of-two scales per natural slot (phase-1 rows),
  // per slot-workspace position, per point (phase-2 rows); column scales of X
  DevBuf tc_qslot, tc_qpos, tc_rpt, tc_col;
  int64_t n_tcp1 = 0, n_tcred = 0, n_tctile = 0, tc_part_rows = 0, n_tca = 0, n_tcx = 0, n_tcz = 0;
  int64_t tc_panel = 0;  // columns per tensor-core pass
  uint32_t tc_polls = 1u << 22;  // poll limit of the tensor-core kernels' pipeline waits
  int tca_fmt = 0;       // format the split operator stream holds (1, 2)
  int tc_variant = 0;    // pipeline shape of the FP16 engine (0: 4 chunks x 2 stages, 1: 2 x 4; hmat_autotune)
  int zsplit_fmt = 0;    // format last written to the split slot workspace
  // sparse splits of X (FP16 engine): chunk of each cluster-order row, and the
  // byte offsets the last sparse split wrote (xs_count of them, in a split of
  // xs_nct column tiles; xs_count < 0: the split X holds other data)
  DevBuf tc_rowchunk, xs_pos;
  int64_t xs_count = -1;
  int xs_nct = 0;
  int engine = 0;  // 0: SIMT tile engine; tensor cores: 1 = 3xTF32, 2 = scaled 2xFP16 (FP32 operators),
                   // 3 = integer slices (FP64 operators)
  // engine 3 (FP64 operators): schedule, scales, sliced operator stream,
  // sliced X and slot workspace per column pass, FP64 partials
  DevBuf ozitem, ozred, oztile, ozseg, ozbdesc, ozxmap, ozslot, oz_sigslot, oz_qslot, oz_qshift, oz_qpos, oz_sigpt;
  DevBuf ozb, ozx, ozz, ozpart, oz_col, oz_err;
  int64_t n_ozitem = 0, n_ozred = 0, n_oztile = 0, n_ozb = 0, n_ozx = 0, n_ozz = 0, oz_part_rows = 0;
  int64_t oz_panel = 0;
  bool ozb_built = false;
  bool values_released = false;  // FP32 factor/near values freed (fkf_hmatrix_release_values)
  // workspace
  DevBuf zmix, part, xperm, yperm;
  int64_t panel = 256;
};

// happly.cu
fkf_status hmat_upload(fkf_hmat* h, const HostHmat& hh);
int64_t hmat_device_bytes(const fkf_hmat* h);
fkf_status hmat_apply_clustered(fkf_hmat* h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t ncols);
// <A, B> = sum_ij A_ij B_ij over nrows x ncols blocks of the operator's
// element type (FP64 accumulation, fixed order; synchronises).
fkf_status hmat_dot(fkf_hmat* h, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t nrows, int64_t ncols,
                    double* out);
fkf_status hmat_apply_clustered_noalloc(fkf_hmat* h, const void* X, int64_t ldx, void* Y, int64_t ldy,
                                        int64_t ncols);
// dst[i, :] = src[idx[i], :] for i < nrows (element type = precision / FP64)
fkf_status hmat_permute_rows(fkf_hmat* h, const void* src, int64_t lds, const int64_t* idx_dev, void* dst,
                             int64_t ldd, int64_t nrows, int64_t ncols);
fkf_status hmat_permute_rows_f64(fkf_ctx* ctx, const double* src, int64_t lds, const int64_t* idx_dev, double* dst,
                                 int64_t ldd, int64_t nrows, int64_t ncols);

// happly_oz.cu
fkf_status hmat_upload_oz(fkf_hmat* h, OzUpload& ou);
fkf_status hmat_apply_clustered_oz(fkf_hmat* h, const double* X, int64_t ldx, double* Y, int64_t ldy,
                                   int64_t ncols);
fkf_status hmat_oz_check(fkf_hmat* h);
// Writes the sliced operator stream of engine 3 if it is not there yet.
fkf_status hmat_oz_prepare(fkf_hmat* h);
// C = alpha op(A) op(B) + beta C for FP64 row-major device matrices on the
// tensor cores, by the integer slices of engine 3 (op(A) sliced per row,
// op(B) per column); C must not overlap A or B.  On ctx->stream; reports an
// expired pipeline wait through the context's GEMM error flag (checked by
// gemm_f64_tc_check).
fkf_status gemm_f64_tc(fkf_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                       int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                       OzGemmWs* ws = nullptr);
fkf_status gemm_f64_tc_check(fkf_ctx* ctx);

// A sparse X (N x ncols, cluster order) given by its rows: row i holds the
// entries (crow[p], cval[p]) for colptr[i] <= p < colptr[i + 1], sorted by
// column, repeated columns summed in FP32 in that order (the CSC index of H,
// whose columns are the rows of X = H^T).
struct TcSparseX {
  int64_t n, nnz;
  const int64_t* colptr;
  const int* crow;
  const double* cval;
};

// happly_tc.cu
// True when an apply of ncols columns on this operator can take a sparse X
// (ctx->x_sparse): FP32 operator on the FP16 split engine, one column pass.
bool hmat_sparse_x_ok(const fkf_hmat* h, int64_t ncols);
fkf_status hmat_apply_clustered_tc(fkf_hmat* h, const float* X, int64_t ldx, float* Y, int64_t ldy, int64_t ncols);
fkf_status hmat_tc_check(fkf_hmat* h);
void hmat_build_tc_schedule(const std::vector<P2Leaf>& leaves, const std::vector<P2Seg>& segs,
                            std::vector<TcTile>& tiles, std::vector<TcSeg>& tsegs);
// Uploads the tensor-core schedule and writes the split operator streams
// (after fac/nearv are on the device).
fkf_status hmat_upload_tc(fkf_hmat* h, TcUpload& tu);
// Selects the engine (0, 1, 2); rewrites the split operator stream when the
// tensor-core format changes.
fkf_status hmat_set_engine(fkf_hmat* h, int engine);
// Y_f = Gamma_f X_f (cluster order) for nb FP32 operators on the same
// tensor-core format, each in one column pass (ncols_f <= its panel), with
// one persistent launch per phase for all of them, on ctx's stream; the
// caller orders that stream after the producers of every X_f.  A failed wait
// is reported through every operator's tensor-core error flag.
fkf_status hmat_apply_tc_multi(fkf_ctx* ctx, fkf_hmat* const* hs, int nb, const float* const* X, const int64_t* ldx,
                               float* const* Y, const int64_t* ldy, const int64_t* ncols);
// Times the FP16 engine's pipeline shapes on an apply of ncols columns and
// keeps the faster one for this operator (no-op for other engines).
fkf_status hmat_autotune(fkf_hmat* h, int64_t ncols, int* variant, double* ms_best);
// True when hmat_apply_tc_multi can run these operators together.
bool hmat_tc_multi_ok(fkf_hmat* const* hs, int nb, const int64_t* ncols);
// The step's H-apply (S2): through the batch of the calling host thread when
// it takes part in one (fkf_filter_step_batched), else a plain apply.
fkf_status hmat_apply_step(fkf_hmat* h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t ncols);
// Dense C_p = A_p B[0:K_p, 0:ncols] for p < np <= 2 (row-major FP32 in and
// out) on the tensor cores with two-term split products; B has kb >= K_p rows.  The
// launch is asynchronous: tc_gemm_check reads the error flag after a sync.
struct TcGemmProblem {
  const float* A;
  int64_t lda, rows;
  int K;
  float* C;
  int64_t ldc;
};
// fmt: 2 = scaled two-term FP16 split (kind::f16, default), 1 = 3xTF32.
fkf_status tc_gemm_f32(fkf_ctx* ctx, const TcGemmProblem* p, int np, const float* B, int64_t ldb, int64_t kb,
                       int ncols, TcGemmWs& ws, int fmt = 2);
fkf_status tc_gemm_check(fkf_ctx* ctx, TcGemmWs& ws);

// hbuild.cpp
fkf_status hmat_build_host(fkf_ctx* ctx, const double* pts, int64_t n, int dim, fkf_matern k, fkf_hparams hp,
                           HostHmat** out, std::vector<int64_t>& perm);
void hmat_free_host(HostHmat* hh);
double kernel_eval(const fkf_matern& k, double r);
