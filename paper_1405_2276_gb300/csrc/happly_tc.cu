// H-apply on the 5th-generation tensor cores (FP32 operators): both phases of
// the two-phase apply run as 128 x 128 tiles of tcgen05.mma kind::tf32 with
// the accumulator in TMEM.  Each FP32 operand value x is split into
// hi = tf32(x) and lo = tf32(x - hi) while it is staged, and every product is
// accumulated as hi*hi + hi*lo + lo*hi (3xTF32, FP32 accumulation), which
// keeps FP32-level accuracy.
//
// Pipeline per CTA (256 threads, two CTAs per SM):
//   raw stages (3): cp.async copies FP32 chunks (K = 16) of A and B from
//                   global memory, two chunks ahead of the one being split;
//   split stages (2): every thread splits its part of the landed raw chunk
//                   into hi/lo TF32 halves in the canonical K-major no-swizzle
//                   core-matrix layout (umma.cuh);
//   one thread issues the chunk's 6 MMAs (2 K-steps x 3 products) and commits
//   them to the split stage's mbarrier, which guards that stage's reuse.
// The epilogue reads TMEM with tcgen05.ld (warp w: lanes 32*(w%4).., columns
// 64*(w/4)..).  Every mbarrier wait is bounded; an expired wait sets an error
// flag, the tile drains what it issued, frees its TMEM and returns.
//
// Phase 2 tiles are 128 consecutive rows (whole leaves packed together); the
// segments of the packed leaves are merged where they read the same slot rows
// with contiguous factor rows (every common ancestor), so those B operands
// are loaded once per tile instead of once per leaf.
#include <algorithm>
#include <cstring>

#include "common.h"
#include "umma.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kConv = 2;                                 // split (hi/lo) stages
constexpr int kRaw = 3;                                  // raw FP32 stages
constexpr int kConvBytes = 4 * umma::kChunkBytes;        // A_hi, A_lo, B_hi, B_lo (32 KB)
constexpr int kRawBytes = 2 * umma::kChunkBytes;         // A, B fp32 (16 KB)
constexpr int kSmemBytes = kConv * kConvBytes + kRaw * kRawBytes + 256;  // 112.25 KB: two CTAs per SM
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kMaxPolls = 1u << 22;  // bounded mbarrier waits (error flag on expiry)
constexpr uint32_t kIdesc = umma::idesc_tf32(128, 128);

// Stage addresses are computed, not stored in arrays (a dynamically indexed
// pointer array would live in local memory).
struct Smem {
  uint8_t* base;
  uint64_t* mbar;  // [kConv]
  uint32_t* tmem_slot;
  int* fail;
  __device__ __forceinline__ uint8_t* conv(int i) const { return base + i * kConvBytes; }
  __device__ __forceinline__ uint8_t* raw(int i) const { return base + kConv * kConvBytes + i * kRawBytes; }
};

__device__ __forceinline__ Smem smem_layout(uint8_t* base) {
  Smem s;
  s.base = base;
  uint8_t* tail = base + kConv * kConvBytes + kRaw * kRawBytes;
  s.mbar = reinterpret_cast<uint64_t*>(tail);
  s.tmem_slot = reinterpret_cast<uint32_t*>(tail + 64);
  s.fail = reinterpret_cast<int*>(tail + 128);
  return s;
}

// ---- asynchronous global -> shared copies ---------------------------------
// 16-byte copy of `bytes` (0..16) valid bytes; the rest of the 16 is zero-filled.
__device__ __forceinline__ void cp16(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(umma::smem_u32(dst)), "l"(src), "r"(bytes)
               : "memory");
}
// 4-byte copy, for sources not 16-byte aligned
__device__ __forceinline__ void cp4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(umma::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// A quad (4 floats) of `valid` leading elements from src into dst (16 bytes);
// src is read only where valid, the missing elements are stored as zeros.
__device__ __forceinline__ void copy_quad(void* dst, const float* src, int valid, bool vec) {
  if (valid <= 0) {
    *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
  } else if (vec) {
    cp16(dst, src, 4 * min(valid, 4));
  } else {
#pragma unroll
    for (int u = 0; u < 4; u++) {
      float* d = reinterpret_cast<float*>(dst) + u;
      if (u < valid)
        cp4(d, src + u);
      else
        *d = 0.f;
    }
  }
}

// Raw A in "rows" form: 128 rows x 16 floats, quad q of row r at byte
// r * 64 + ((q ^ ((r >> 1) & 3)) * 16) (conflict-free 16-byte reads by row).
__device__ __forceinline__ uint32_t raw_row_off(int r, int q) { return (uint32_t)(r * 64 + ((q ^ ((r >> 1) & 3)) * 16)); }

// Raw operand in "k-rows" form: 16 rows (k) x 128 floats, quad q of row k at k * 512 + q * 16.
__device__ __forceinline__ uint32_t raw_krow_off(int k, int q) { return (uint32_t)(k * 512 + q * 16); }

// Issue the copies of A rows: A(m, k) = A[(m - lo) * lda + k0 + k], m in [lo, hi), k < kv.
__device__ __forceinline__ void issue_a_rows(uint8_t* raw, const float* A, int64_t lda, int lo, int hi, int k0,
                                             int kv, bool vec) {
#pragma unroll
  for (int j = 0; j < 2; j++) {
    const int i = threadIdx.x + j * kThreads;
    const int r = i >> 2, q = i & 3;
    const bool rv = r >= lo && r < hi;
    const int valid = rv ? kv - (k0 + 4 * q) : 0;
    copy_quad(raw + raw_row_off(r, q), A + (int64_t)(rv ? r - lo : 0) * lda + k0 + 4 * q, valid, vec);
  }
}

// Issue the copies of a k-rows operand: P(k, c) = P[(k0 + k) * ld + c], k < kv, c < cv.
__device__ __forceinline__ void issue_krows(uint8_t* raw, const float* P, int64_t ld, int cv, int k0, int kv,
                                            bool vec) {
#pragma unroll
  for (int j = 0; j < 2; j++) {
    const int i = threadIdx.x + j * kThreads;
    const int k = i >> 5, q = i & 31;
    const bool kvld = k0 + k < kv;
    const int valid = kvld ? cv - 4 * q : 0;
    copy_quad(raw + raw_krow_off(k, q), P + (int64_t)(kvld ? k0 + k : 0) * ld + 4 * q, valid, vec);
  }
}

// ---- split into the tensor-core layout ---------------------------------------
__device__ __forceinline__ void put4(uint8_t* hi_base, uint8_t* lo_base, int row, int k, float v0, float v1, float v2,
                                     float v3) {
  uint4 h, l;
  umma::split_tf32(v0, h.x, l.x);
  umma::split_tf32(v1, h.y, l.y);
  umma::split_tf32(v2, h.z, l.z);
  umma::split_tf32(v3, h.w, l.w);
  const uint32_t off = umma::chunk_offset(row, k);
  *reinterpret_cast<uint4*>(hi_base + off) = h;
  *reinterpret_cast<uint4*>(lo_base + off) = l;
}

// row r (= tl) of a raw rows-form operand -> (row, k = 0..15)
__device__ __forceinline__ void split_row(const uint8_t* raw, uint8_t* hi, uint8_t* lo, int r) {
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const float4 v = *reinterpret_cast<const float4*>(raw + raw_row_off(r, q));
    put4(hi, lo, r, 4 * q, v.x, v.y, v.z, v.w);
  }
}

// column c (= tl) of a raw k-rows operand -> (row = c, k = 0..15); a warp reads
// 32 consecutive floats per k and writes 8 distinct rows per quarter-warp
// (both free of bank conflicts)
__device__ __forceinline__ void split_col(const uint8_t* raw, uint8_t* hi, uint8_t* lo, int c) {
  const float* r = reinterpret_cast<const float*>(raw) + c;
#pragma unroll
  for (int q = 0; q < 4; q++)
    put4(hi, lo, c, 4 * q, r[(4 * q + 0) * 128], r[(4 * q + 1) * 128], r[(4 * q + 2) * 128], r[(4 * q + 3) * 128]);
}

// Issue the 3xTF32 MMAs of one split chunk (one thread).
__device__ __forceinline__ void issue_mma(uint8_t* st, uint32_t tmem, bool first) {
  const uint32_t a_hi = umma::smem_u32(st), a_lo = a_hi + umma::kChunkBytes;
  const uint32_t b_hi = a_hi + 2 * umma::kChunkBytes, b_lo = a_hi + 3 * umma::kChunkBytes;
#pragma unroll
  for (int kk = 0; kk < umma::kChunk / 8; kk++) {
    const uint32_t koff = kk * 2 * umma::kLBO;  // two core matrices along K per MMA
    umma::mma_tf32(tmem, umma::smem_desc(a_hi + koff), umma::smem_desc(b_hi + koff), kIdesc, (first && kk == 0) ? 0u : 1u);
    umma::mma_tf32(tmem, umma::smem_desc(a_hi + koff), umma::smem_desc(b_lo + koff), kIdesc, 1u);
    umma::mma_tf32(tmem, umma::smem_desc(a_lo + koff), umma::smem_desc(b_hi + koff), kIdesc, 1u);
  }
}

// Main loop.  src.issue(raw) issues the copies of the next chunk (uniform
// across the CTA; false when there is none); src.split(raw, conv) splits a
// landed chunk.  Returns the number of chunks handed to the tensor core.
template <typename Src>
__device__ __forceinline__ int run_chunks(const Smem& s, uint32_t tmem, Src& src) {
  int issued = 0;
#pragma unroll
  for (int i = 0; i < kRaw - 1; i++) {
    if (src.issue(s.raw(i))) issued++;
    cp_commit();
  }
  int c = 0;
  while (c < issued) {
    const int cs = c % kConv;
    if (c >= kConv) {
      if (!umma::mbar_wait(&s.mbar[cs], ((c - kConv) / kConv) & 1, kMaxPolls)) atomicExch(s.fail, 1);
    }
    cp_wait1();  // this thread's copies of chunk c have landed
    __syncthreads();
    if (*s.fail) break;
    // the raw stage of chunk c-1 is free (split in the previous iteration)
    if (src.issue(s.raw((c + kRaw - 1) % kRaw))) issued++;
    cp_commit();
    src.split(s.raw(c % kRaw), s.conv(cs));
    umma::fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      umma::fence_after_sync();
      issue_mma(s.conv(cs), tmem, c == 0);
      umma::commit(&s.mbar[cs]);
    }
    c++;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  return c;
}

__device__ __forceinline__ void tile_begin(const Smem& s) {
  if (threadIdx.x < 32) umma::tmem_alloc(s.tmem_slot, kTmemCols);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kConv; i++) umma::mbar_init(&s.mbar[i], 1);
    *s.fail = 0;
    umma::fence_mbar_init();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
}

// Wait for the last chunk's MMAs (bounded); returns false on expiry.
__device__ __forceinline__ bool tile_drain(const Smem& s, int nchunks) {
  bool ok = true;
  if (nchunks > 0) {
    const int c = nchunks - 1;
    ok = umma::mbar_wait(&s.mbar[c % kConv], (c / kConv) & 1, kMaxPolls);
    if (!ok) atomicExch(s.fail, 1);
  }
  __syncthreads();
  umma::fence_after_sync();
  return ok && !*s.fail;
}

__device__ __forceinline__ void tile_end(const Smem& s, uint32_t tmem) {
  umma::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) umma::tmem_dealloc(tmem, kTmemCols);
}

// Epilogue: thread owns row (32 * (warp % 4) + lane) and 64 columns starting at
// 64 * (warp / 4); calls out(row, col, value) for valid entries.
template <typename OutFn>
__device__ __forceinline__ void tile_store(uint32_t tmem, int rows, int nv, bool zero, OutFn&& out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (warp & 3) + lane;
  const int c0 = 64 * (warp >> 2);
  for (int h = 0; h < 2; h++) {
    float v[32];
    if (zero) {
#pragma unroll
      for (int i = 0; i < 32; i++) v[i] = 0.f;
    } else {
      umma::tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + 32 * h), v);
    }
    if (row < rows) {
#pragma unroll
      for (int i = 0; i < 32; i++) {
        const int col = c0 + 32 * h + i;
        if (col < nv) out(row, col, v[i]);
      }
    }
  }
}

// Chunk source for phase 2: the tile's segments, K-chunks of kChunk each.
// A = factor / near-field rows (k-contiguous, rows form); B = slot rows of
// Zmix or rows of X (k-rows form).
struct P2Src {
  const TcSeg* segs;
  int seg0, nseg;
  const float *fac, *nearv, *zmix, *X;
  int64_t ldz, ldx;
  int n0, nv;
  bool bvec_z, bvec_x;
  int si = 0, k0 = 0;
  bool started = false;
  __device__ bool issue(uint8_t* raw) {
    if (!started) {
      started = true;
      si = 0;
      k0 = 0;
    } else {
      k0 += umma::kChunk;
      if (si < nseg && k0 >= segs[seg0 + si].K) {
        k0 = 0;
        si++;
      }
    }
    while (si < nseg && segs[seg0 + si].K <= 0) si++;
    if (si >= nseg) return false;
    const TcSeg sg = segs[seg0 + si];
    const float* A = (sg.near ? nearv : fac) + sg.a_off;
    const bool avec = ((sg.a_off & 3) == 0) && ((sg.lda & 3) == 0);
    issue_a_rows(raw, A, sg.lda, sg.row_lo, sg.row_hi, k0, sg.K, avec);
    const float* B = sg.near ? X + sg.b_row * ldx + n0 : zmix + sg.b_row * ldz + n0;
    issue_krows(raw + umma::kChunkBytes, B, sg.near ? ldx : ldz, nv, k0, sg.K, sg.near ? bvec_x : bvec_z);
    return true;
  }
  __device__ void split(const uint8_t* raw, uint8_t* conv) const {
    const int t = threadIdx.x;
    if (t < 128)
      split_row(raw, conv, conv + umma::kChunkBytes, t);
    else
      split_col(raw + umma::kChunkBytes, conv + 2 * umma::kChunkBytes, conv + 3 * umma::kChunkBytes, t - 128);
  }
};

// Chunk source for phase 1: rows of one cluster chunk, K-chunks of kChunk.
// A(m = slot, k = row) and B(k = row, n) are both in k-rows form.
struct P1Src {
  const float *A, *B;
  int64_t lda, ldb;
  int mv, kv, nv;
  bool avec, bvec;
  int k0 = -umma::kChunk;
  __device__ bool issue(uint8_t* raw) {
    k0 += umma::kChunk;
    if (k0 >= kv) return false;
    issue_krows(raw, A, lda, mv, k0, kv, avec);
    issue_krows(raw + umma::kChunkBytes, B, ldb, nv, k0, kv, bvec);
    return true;
  }
  __device__ void split(const uint8_t* raw, uint8_t* conv) const {
    const int t = threadIdx.x;
    if (t < 128)
      split_col(raw, conv, conv + umma::kChunkBytes, t);
    else
      split_col(raw + umma::kChunkBytes, conv + 2 * umma::kChunkBytes, conv + 3 * umma::kChunkBytes, t - 128);
  }
};

__global__ void __launch_bounds__(kThreads, 2)
    k_phase2_tc(const TcTile* __restrict__ tiles, const TcSeg* __restrict__ segs, const float* __restrict__ fac,
                const float* __restrict__ nearv, const float* __restrict__ zmix, int64_t ldz,
                const float* __restrict__ X, int64_t ldx, float* __restrict__ Y, int64_t ldy, int ncols,
                int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const Smem s = smem_layout(smem_raw);
  // x = column tile (fastest): the column tiles of one row tile run together
  // and share the tile's operator rows through L2
  const TcTile tl = tiles[blockIdx.y];
  const int n0 = blockIdx.x * 128;
  const int nv = min(128, ncols - n0);
  if (nv <= 0) return;
  tile_begin(s);
  const uint32_t tmem = *s.tmem_slot;
  const bool bz = ((ldz & 3) == 0) && ((reinterpret_cast<uintptr_t>(zmix + n0) & 15) == 0);
  const bool bx = ((ldx & 3) == 0) && ((reinterpret_cast<uintptr_t>(X + n0) & 15) == 0);
  P2Src src{segs, tl.seg0, tl.nseg, fac, nearv, zmix, X, ldz, ldx, n0, nv, bz, bx};
  const int c = run_chunks(s, tmem, src);
  const bool ok = tile_drain(s, c);
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    float* Yt = Y + tl.row0 * ldy + n0;
    tile_store(tmem, tl.rows, nv, c == 0, [&](int row, int col, float v) { Yt[(int64_t)row * ldy + col] = v; });
  }
  tile_end(s, tmem);
}

__global__ void __launch_bounds__(kThreads, 2)
    k_phase1_tc(const P1Item* __restrict__ items, const float* __restrict__ fac, const float* __restrict__ X,
                int64_t ldx, int ncols, const int64_t* __restrict__ slotmap, float* __restrict__ zmix,
                float* __restrict__ part, int64_t ldz, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const Smem s = smem_layout(smem_raw);
  const P1Item it = items[blockIdx.x];
  const int n0 = blockIdx.y * 128;
  const int nv = min(128, ncols - n0);
  if (nv <= 0) return;
  tile_begin(s);
  const uint32_t tmem = *s.tmem_slot;
  // A(m = slot, k = row) = Fac_c[(r0 + row) * K + q0 + slot]; B(k = row, n) = X[(x_row + row) * ldx + n0 + n]
  const float* A = fac + it.fac_off + (int64_t)it.r0 * it.K + it.q0;
  const float* B = X + it.x_row * ldx + n0;
  const bool av = ((it.K & 3) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  const bool bv = ((ldx & 3) == 0) && ((reinterpret_cast<uintptr_t>(B) & 15) == 0);
  P1Src src{A, B, it.K, ldx, it.nq, it.nr, nv, av, bv};
  const int c = run_chunks(s, tmem, src);
  const bool ok = tile_drain(s, c);
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    tile_store(tmem, it.nq, nv, c == 0, [&](int q, int col, float v) {
      float* dst = it.out_row < 0 ? zmix + slotmap[it.map_off + q] * ldz : part + (it.out_row + q) * ldz;
      dst[n0 + col] = v;
    });
  }
  tile_end(s, tmem);
}

__global__ void k_phase1_reduce_tc(const P1Reduce* __restrict__ items, const float* __restrict__ part,
                                   const int64_t* __restrict__ slotmap, float* __restrict__ zmix, int64_t ldz,
                                   int ncols) {
  const P1Reduce it = items[blockIdx.x];
  const int64_t total = (int64_t)it.nq * ncols;
  for (int64_t e = threadIdx.x + (int64_t)blockIdx.y * blockDim.x; e < total; e += (int64_t)blockDim.x * gridDim.y) {
    const int q = (int)(e / ncols), n = (int)(e % ncols);
    float acc = 0.f;
    for (int c = 0; c < it.nch; c++) acc += part[(it.part_row + (int64_t)c * it.nq + q) * ldz + n];
    zmix[slotmap[it.map_off + q] * ldz + n] = acc;
  }
}

}  // namespace

// Tensor-core apply for an FP32 operator (cluster order).
fkf_status hmat_apply_clustered_tc(fkf_hmat* h, const float* X, int64_t ldx, float* Y, int64_t ldy, int64_t ncols) {
  fkf_ctx* ctx = h->ctx;
  const int64_t P = h->panel;
  const size_t zbytes = (size_t)std::max<int64_t>(h->ktot, 1) * P * sizeof(float);
  if (h->zmix.bytes < zbytes) FKF_TRY(dev_alloc(ctx, h->zmix, zbytes));
  const size_t pbytes = (size_t)std::max<int64_t>(h->tc_part_rows, 1) * P * sizeof(float);
  if (h->part.bytes < pbytes) FKF_TRY(dev_alloc(ctx, h->part, pbytes));
  if (h->tc_err.bytes < 64) {
    FKF_TRY(dev_alloc(ctx, h->tc_err, 64));
    FKF_CUDA(ctx, cudaMemsetAsync(h->tc_err.p, 0, 64, ctx->stream));
  }
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_phase2_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_phase1_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
  for (int64_t c0 = 0; c0 < ncols; c0 += P) {
    const int nc = (int)std::min<int64_t>(P, ncols - c0);
    const int ntile = (int)cdiv(nc, 128);
    if (h->n_tcp1 > 0) {
      k_phase1_tc<<<dim3((unsigned)h->n_tcp1, ntile), kThreads, kSmemBytes, ctx->stream>>>(
          h->tcp1.as<P1Item>(), h->fac.as<float>(), X + c0, ldx, nc, h->slotmap.as<int64_t>(), h->zmix.as<float>(),
          h->part.as<float>(), P, h->tc_err.as<int>());
      FKF_LAUNCHED(ctx);
    }
    if (h->n_tcred > 0) {
      k_phase1_reduce_tc<<<dim3((unsigned)h->n_tcred, 4), 256, 0, ctx->stream>>>(
          h->tcred.as<P1Reduce>(), h->part.as<float>(), h->slotmap.as<int64_t>(), h->zmix.as<float>(), P, nc);
      FKF_LAUNCHED(ctx);
    }
    k_phase2_tc<<<dim3(ntile, (unsigned)h->n_tctile), kThreads, kSmemBytes, ctx->stream>>>(
        h->tctile.as<TcTile>(), h->tcseg.as<TcSeg>(), h->fac.as<float>(), h->nearv.as<float>(), h->zmix.as<float>(),
        P, X + c0, ldx, Y + c0, ldy, nc, h->tc_err.as<int>());
    FKF_LAUNCHED(ctx);
  }
  return FKF_OK;
}

// Reads (and clears) the tensor-core wait-expiry flag; synchronises.
fkf_status hmat_tc_check(fkf_hmat* h) {
  if (!h->tc_err.p) return FKF_OK;
  int e = 0;
  FKF_CUDA(h->ctx, cudaMemcpyAsync(&e, h->tc_err.p, 4, cudaMemcpyDeviceToHost, h->ctx->stream));
  FKF_CUDA(h->ctx, cudaStreamSynchronize(h->ctx->stream));
  if (e) {
    FKF_CUDA(h->ctx, cudaMemsetAsync(h->tc_err.p, 0, 64, h->ctx->stream));
    return set_err(h->ctx, FKF_ETIMEOUT, "tensor-core H-apply: an mbarrier wait expired");
  }
  return FKF_OK;
}

// Build the tensor-core work lists from the per-leaf segment lists and the
// cluster factor layout (host).
void hmat_build_tc_schedule(const std::vector<P2Leaf>& leaves, const std::vector<P2Seg>& segs,
                            std::vector<TcTile>& tiles, std::vector<TcSeg>& tsegs) {
  size_t i = 0;
  while (i < leaves.size()) {
    TcTile t{};
    t.row0 = leaves[i].row0;
    t.seg0 = (int)tsegs.size();
    int rows = 0;
    while (i < leaves.size() && rows + leaves[i].rows <= 128 && leaves[i].row0 == t.row0 + rows) {
      const P2Leaf& lf = leaves[i];
      const int ro = rows;
      for (int k = 0; k < lf.nseg; k++) {
        const P2Seg& sg = segs[lf.seg0 + k];
        const int64_t a_off = sg.a_off + (int64_t)lf.pad * sg.lda;
        bool merged = false;
        for (size_t q = t.seg0; q < tsegs.size(); q++) {
          TcSeg& e = tsegs[q];
          if (e.near == sg.near && e.b_row == sg.b_row && e.K == sg.K && e.lda == sg.lda && e.row_hi == ro &&
              e.a_off + (int64_t)(e.row_hi - e.row_lo) * e.lda == a_off) {
            e.row_hi = ro + lf.rows;
            merged = true;
            break;
          }
        }
        if (!merged) {
          TcSeg e{};
          e.a_off = a_off;
          e.b_row = sg.b_row;
          e.lda = sg.lda;
          e.K = sg.K;
          e.near = sg.near;
          e.row_lo = ro;
          e.row_hi = ro + lf.rows;
          tsegs.push_back(e);
        }
      }
      rows += lf.rows;
      i++;
    }
    t.rows = rows;
    t.nseg = (int)tsegs.size() - t.seg0;
    tiles.push_back(t);
  }
}
