// Symmetric eigensolver (FP64) of the library's own, for the data-space
// generalized eigenproblem (Eq. ghep written in data space, Sec. 2.2.2) and the
// merge eigenproblem of Alg. lowrankaddition (step 4, Sec. 2.4):
//
//  1. Householder reduction to tridiagonal form T = Q_H^T A Q_H, blocked by
//     panels of kNB columns: the column steps of a panel run in one cooperative
//     kernel (grid-wide barriers between the column's phases: the column's
//     update with the panel's earlier reflectors, the reflector, the
//     symmetric product A v, the correction w), the trailing update
//     A -= V W^T + W V^T after the panel in one symmetric FP64 tile GEMM;
//  2. divide and conquer on T (Cuppen's splitting T = diag(T1, T2) + |b| u u^T):
//     leaves of at most kLeaf rows by implicit QL (one warp per leaf); each
//     merge sorts the children's eigenvalues, deflates (small components of
//     z, and pairs of close eigenvalues rotated until one component vanishes),
//     solves the secular equation 1/rho + sum z_i^2 / (d_i - lambda) = 0 for
//     every remaining root (one thread per root: a fit of the two nearest
//     poles by rational functions, safeguarded by bisection, with lambda kept
//     as an offset from its nearest pole), recomputes z from the roots
//     (Loewner's formula, which makes the eigenvectors orthogonal to working
//     precision), forms the eigenvectors of the rank-one update and applies
//     them to the children's eigenvectors with one FP64 GEMM;
//  3. back-transformation X = Q_H Z of the wanted eigenvectors, one block
//     reflector (I - V T V^T, compact WY form) per panel, by GEMMs.
//
// Every spin (the grid barrier) is bounded and sets an error flag; iteration
// counts are bounded.  Results: eigenvalues ascending; eigenvector j in row j.
#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>

#include "dense.h"

namespace {

constexpr int kNB = 32;                  // panel width of the reduction and the back-transformation
constexpr int kLeaf = 32;                // largest leaf of the divide and conquer (one warp)
constexpr int kTrdThreads = 256;
constexpr uint32_t kBarPolls = 1u << 24;  // bounded grid-barrier spin
constexpr double kEps = DBL_EPSILON;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double x = lane < nw ? sh[lane] : 0.0;
    x = warp_sum(x);
    if (lane == 0) sh[32] = x;
  }
  __syncthreads();
  const double r = sh[32];
  __syncthreads();
  return r;
}

// Grid-wide barrier of a cooperative launch (all CTAs co-resident): a
// monotonic arrival counter; the wait is bounded and records a failure.
__device__ void grid_barrier(unsigned* bar, unsigned& gen, int* err) {
  __syncthreads();
  gen += gridDim.x;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    uint32_t polls = 0;
    while (*reinterpret_cast<volatile unsigned*>(bar) < gen) {
      if (++polls > kBarPolls) {
        atomicExch(err, 1);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
}

struct TrdArgs {
  double* A;     // n x n, row-major, symmetric (both triangles current in the trailing block)
  int64_t n;
  int64_t j0;    // first column of the panel
  int nbp;       // columns in the panel
  double* VW;    // n x 2kNB: [V | W] of the panel
  double* WV;    // n x 2kNB: [W | V]
  double* d;     // diagonal of T
  double* e;     // off-diagonal of T
  double* tau;   // reflector scalars
  double* col;   // n: current column
  double* vg;    // n: reflector
  double* pg;    // n: A v
  double* part;  // gridDim.x * (1 + 2 kNB) partial sums
  unsigned* bar;
  int* err;
};

// One panel of the Householder reduction (lower form).  Column j of the panel
// (c = j - j0):
//   a = A[j:, j] - V[j:, :c] W[j, :c]^T - W[j:, :c] V[j, :c]^T   (current column)
//   d_j = a_0; reflector H = I - tau v v^T with H a[1:] = beta e_1, v_0 = 1
//   p = A[j+1:, j+1:] v - V (W^T v) - W (V^T v)                    (current matrix times v)
//   w = tau p - tau^2/2 (p^T v) v;  V[:, c] = v, W[:, c] = w
// The reflector (below its leading 1) is stored in A[j+2:, j].
__global__ void __launch_bounds__(kTrdThreads) k_trd_panel(TrdArgs a) {
  __shared__ double sh[33];
  __shared__ double red[4][2 * kNB];
  __shared__ double wv[2 * kNB];
  __shared__ double bc[4];
  const int64_t n = a.n;
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  constexpr int L = 2 * kNB;
  unsigned gen = 0;
  double* part2 = a.part + G;
  for (int c = 0; c < a.nbp; c++) {
    const int64_t j = a.j0 + c;
    if (j >= n) break;
    // ---- phase A: current column on rows [j, n), this CTA's chunk
    {
      const int64_t rows = n - j, R = (rows + G - 1) / G;
      const int64_t r0 = j + b * R, r1 = min(n, r0 + R);
      const double* Vj = a.VW + j * L;
      double ss = 0;
      for (int64_t i = r0 + t; i < r1; i += blockDim.x) {
        double v = a.A[j * n + i];  // A[i][j] = A[j][i]
        const double* Vi = a.VW + i * L;
        for (int q = 0; q < c; q++) v -= Vi[q] * Vj[kNB + q] + Vi[kNB + q] * Vj[q];
        a.col[i] = v;
        if (i >= j + 2) ss += v * v;
      }
      ss = block_sum(ss, sh);
      if (t == 0) a.part[b] = ss;
    }
    grid_barrier(a.bar, gen, a.err);
    // ---- phase B: the reflector (every CTA computes it from the same partials)
    if (t == 0) {
      double s2 = 0;
      for (int q = 0; q < G; q++) s2 += a.part[q];
      double beta = 0, tau = 0, scale = 0;
      if (j + 1 < n) {
        const double alpha = a.col[j + 1];
        if (s2 == 0.0) {
          beta = alpha;
        } else {
          beta = -copysign(sqrt(alpha * alpha + s2), alpha);
          tau = (beta - alpha) / beta;
          scale = 1.0 / (alpha - beta);
        }
      }
      bc[0] = tau;
      bc[1] = scale;
      if (b == 0) {
        a.d[j] = a.col[j];
        if (j + 1 < n) {
          a.e[j] = beta;
          a.tau[j] = tau;
        }
      }
    }
    __syncthreads();
    if (j + 1 >= n) break;  // the last diagonal entry has no reflector (uniform over the grid)
    const double tau = bc[0], scale = bc[1];
    const int64_t rows1 = n - j - 1, R1 = (rows1 + G - 1) / G;
    const int64_t s0 = j + 1 + b * R1, s1 = min(n, s0 + R1);
    for (int64_t i = s0 + t; i < s1; i += blockDim.x) {
      const double v = (i == j + 1) ? 1.0 : a.col[i] * scale;
      a.vg[i] = v;
      a.VW[i * L + c] = v;
      a.WV[i * L + kNB + c] = v;
      if (i >= j + 2) a.A[i * n + j] = v;
    }
    __syncthreads();
    if (c > 0) {
      // partial W^T v (entries 0..c-1) and V^T v (c..2c-1) over this CTA's rows
      const int ql = t % L, rl = t / L;  // 4 row lanes x 64 entry lanes
      double acc = 0;
      if (ql < 2 * c) {
        const int colofs = ql < c ? kNB + ql : ql - c;
        for (int64_t i = s0 + rl; i < s1; i += 4) acc += a.VW[i * L + colofs] * a.vg[i];
      }
      red[rl][ql] = acc;
      __syncthreads();
      if (t < 2 * c) part2[(int64_t)b * L + t] = red[0][t] + red[1][t] + red[2][t] + red[3][t];
    }
    grid_barrier(a.bar, gen, a.err);
    // ---- phase C: p = A v - V (W^T v) - W (V^T v), a warp per row of this CTA's chunk
    if (t < 2 * c) {
      double s = 0;
      for (int q = 0; q < G; q++) s += part2[(int64_t)q * L + t];
      wv[t] = s;
    }
    __syncthreads();
    double pv = 0;
    for (int64_t i = s0 + warp; i < s1; i += nw) {
      const double* Ai = a.A + i * n;
      double acc = 0;
      for (int64_t k = j + 1 + lane; k < n; k += 32) acc += Ai[k] * a.vg[k];
      acc = warp_sum(acc);
      if (lane == 0) {
        const double* Vi = a.VW + i * L;
        for (int q = 0; q < c; q++) acc -= Vi[q] * wv[q] + Vi[kNB + q] * wv[c + q];
        a.pg[i] = acc;
        pv += acc * a.vg[i];
      }
    }
    pv = block_sum(pv, sh);
    if (t == 0) a.part[b] = pv;
    grid_barrier(a.bar, gen, a.err);
    // ---- phase D: w = tau p - tau^2/2 (p^T v) v
    if (t == 0) {
      double s = 0;
      for (int q = 0; q < G; q++) s += a.part[q];
      bc[2] = s;
    }
    __syncthreads();
    const double k2 = 0.5 * tau * tau * bc[2];
    for (int64_t i = s0 + t; i < s1; i += blockDim.x) {
      const double w = tau * a.pg[i] - k2 * a.vg[i];
      a.VW[i * L + kNB + c] = w;
      a.WV[i * L + c] = w;
    }
    grid_barrier(a.bar, gen, a.err);
  }
}

// d[p - 1] -= |e[p - 1]| and d[p] -= |e[p - 1]| at every split point p of the
// divide and conquer tree (Cuppen's splitting), in order.
__global__ void k_dc_split_d(int ns, const int* __restrict__ splits, double* __restrict__ d,
                             const double* __restrict__ e) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int q = 0; q < ns; q++) {
    const int p = splits[q];
    const double bb = fabs(e[p - 1]);
    d[p - 1] -= bb;
    d[p] -= bb;
  }
}

// Leaves: implicit QL with a Wilkinson-type shift on a tridiagonal of s <=
// kLeaf rows, one warp per leaf.  Lane 0 runs the scalar recurrence of a sweep
// and records its rotations; every lane applies them to its row of Z.  The
// eigenvalues (ascending) go to D[off..], the eigenvectors to the diagonal
// block of Q (column q = eigenvector q).
__global__ void __launch_bounds__(32) k_dc_leaf(const int* __restrict__ loff, const int* __restrict__ lsize,
                                                 const double* __restrict__ d, const double* __restrict__ e,
                                                 double* __restrict__ D, double* __restrict__ Q, int64_t ldq,
                                                 int* __restrict__ err) {
  __shared__ double Z[kLeaf][kLeaf + 1];
  __shared__ double dd[kLeaf], ee[kLeaf], cs[2][kLeaf];
  __shared__ int lo_sh, perm[kLeaf];
  const int off = loff[blockIdx.x], s = lsize[blockIdx.x], lane = threadIdx.x;
  for (int q = 0; q < s; q++) Z[lane][q] = (lane == q) ? 1.0 : 0.0;
  if (lane < s) {
    dd[lane] = d[off + lane];
    ee[lane] = lane < s - 1 ? e[off + lane] : 0.0;
  }
  __syncwarp();
  for (int l = 0; l < s; l++) {
    for (int iter = 0;; iter++) {
      int m = l;
      for (; m < s - 1; m++) {
        const double dm = fabs(dd[m]) + fabs(dd[m + 1]);
        if (fabs(ee[m]) <= kEps * dm) break;
      }
      if (m == l) break;
      if (iter >= 60) {
        if (lane == 0) atomicExch(err, 2);
        break;
      }
      if (lane == 0) {
        double g = (dd[l + 1] - dd[l]) / (2.0 * ee[l]);
        double r = hypot(g, 1.0);
        g = dd[m] - dd[l] + ee[l] / (g + copysign(r, g));
        double sn = 1.0, c = 1.0, p = 0.0;
        int i = m - 1;
        bool early = false;
        for (; i >= l; i--) {
          const double f = sn * ee[i], bb = c * ee[i];
          r = hypot(f, g);
          ee[i + 1] = r;
          if (r == 0.0) {
            dd[i + 1] -= p;
            ee[m] = 0.0;
            early = true;
            break;
          }
          sn = f / r;
          c = g / r;
          g = dd[i + 1] - p;
          r = (dd[i] - g) * sn + 2.0 * c * bb;
          p = sn * r;
          dd[i + 1] = g + p;
          g = c * r - bb;
          cs[0][i] = c;
          cs[1][i] = sn;
        }
        lo_sh = early ? i + 1 : l;
        if (!early) {
          dd[l] -= p;
          ee[l] = g;
          ee[m] = 0.0;
        }
      }
      __syncwarp();
      const int lo = lo_sh;
      if (lane < s) {
        for (int i = m - 1; i >= lo; i--) {
          const double c = cs[0][i], sn = cs[1][i];
          const double zi = Z[lane][i], zi1 = Z[lane][i + 1];
          Z[lane][i + 1] = sn * zi + c * zi1;
          Z[lane][i] = c * zi - sn * zi1;
        }
      }
      __syncwarp();
    }
  }
  if (lane == 0) {
    for (int q = 0; q < s; q++) perm[q] = q;
    for (int q = 1; q < s; q++) {  // insertion sort by eigenvalue
      const int x = perm[q];
      int p = q - 1;
      while (p >= 0 && dd[perm[p]] > dd[x]) {
        perm[p + 1] = perm[p];
        p--;
      }
      perm[p + 1] = x;
    }
  }
  __syncwarp();
  if (lane < s) {
    D[off + lane] = dd[perm[lane]];
    for (int q = 0; q < s; q++) Q[(int64_t)(off + lane) * ldq + off + q] = Z[lane][perm[q]];
  }
}

// Scratch of one merge (every array sized for the largest node, n).
struct DcMerge {
  int* perm;    // sorted position -> column of the node's block
  double* Dp;   // eigenvalues in sorted order (rotated ones updated)
  double* zp;   // z in sorted order
  int* gi;      // Givens rotations (sorted positions gi < gj)
  int* gj;
  double* gc;
  double* gs;
  int* nd;      // non-deflated positions, by ascending Dp
  int* df;      // deflated positions, by ascending Dp
  double* dk;   // Dp[nd]
  double* zk;   // zp[nd]
  int* orig;    // secular roots: lambda_j = dk[orig_j] + taus_j
  double* taus;
  double* lam;
  double* zh;   // Loewner z
  double* cnrm; // eigenvector column norms
  int* ctl;     // [0] K, [1] number of rotations, [2] deflated count, [3] error
  int* src;     // final position -> source (>= 0: non-deflated root, < 0: -1 - deflated index)
  double* rho;  // [0]
};

// Merge preparation (one CTA; the sequential scans on thread 0): z from the
// children's eigenvectors, the children's sorted eigenvalue lists merged,
// deflation, the remaining poles and z compacted.
__global__ void k_dc_prep(int64_t off, int s, int m, int64_t bidx, const double* __restrict__ e,
                          const double* __restrict__ D, const double* __restrict__ Q, int64_t ldq, DcMerge mg,
                          double* __restrict__ zc) {
  const double beta = e[bidx];
  const double sgn = beta < 0 ? -1.0 : 1.0;
  const double inv2 = 0.70710678118654752440;
  for (int p = threadIdx.x; p < s; p += blockDim.x)
    zc[p] = (p < m ? Q[(off + m - 1) * ldq + off + p] : sgn * Q[(off + m) * ldq + off + p]) * inv2;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double rho = 2.0 * fabs(beta);
  mg.rho[0] = rho;
  // merge the two ascending lists
  int a = 0, b2 = m, q = 0;
  while (a < m || b2 < s) {
    int pick;
    if (b2 >= s || (a < m && D[off + a] <= D[off + b2])) pick = a++;
    else pick = b2++;
    mg.perm[q] = pick;
    mg.Dp[q] = D[off + pick];
    mg.zp[q] = zc[pick];
    q++;
  }
  double dmax = 0, zmax = 0;
  for (int p = 0; p < s; p++) {
    dmax = fmax(dmax, fabs(mg.Dp[p]));
    zmax = fmax(zmax, fabs(mg.zp[p]));
  }
  const double tol = 8.0 * kEps * fmax(dmax, rho * zmax);
  // deflation scan: flag 1 = deflated; mg.src doubles as the flag array here
  int* defl = mg.src;
  int ng = 0, pend = -1;
  for (int j = 0; j < s; j++) {
    defl[j] = 0;
    if (rho * fabs(mg.zp[j]) <= tol) {
      defl[j] = 1;
      continue;
    }
    if (pend < 0) {
      pend = j;
      continue;
    }
    const int i = pend;
    const double r = hypot(mg.zp[i], mg.zp[j]);
    const double c = mg.zp[j] / r, sn = -mg.zp[i] / r;
    const double tdiff = mg.Dp[j] - mg.Dp[i];
    if (fabs(tdiff * c * sn) <= tol) {
      mg.zp[j] = r;
      mg.zp[i] = 0.0;
      mg.gi[ng] = i;
      mg.gj[ng] = j;
      mg.gc[ng] = c;
      mg.gs[ng] = sn;
      ng++;
      const double di = mg.Dp[i], dj = mg.Dp[j];
      mg.Dp[i] = di * c * c + dj * sn * sn;
      mg.Dp[j] = di * sn * sn + dj * c * c;
      defl[i] = 1;
    }
    pend = j;
  }
  int K = 0, nf = 0;
  for (int p = 0; p < s; p++) {
    if (defl[p]) mg.df[nf++] = p;
    else mg.nd[K++] = p;
  }
  // both lists by ascending Dp (the rotations may have moved a value slightly)
  for (int u = 1; u < K; u++) {
    const int x = mg.nd[u];
    int v = u - 1;
    while (v >= 0 && mg.Dp[mg.nd[v]] > mg.Dp[x]) {
      mg.nd[v + 1] = mg.nd[v];
      v--;
    }
    mg.nd[v + 1] = x;
  }
  for (int u = 1; u < nf; u++) {
    const int x = mg.df[u];
    int v = u - 1;
    while (v >= 0 && mg.Dp[mg.df[v]] > mg.Dp[x]) {
      mg.df[v + 1] = mg.df[v];
      v--;
    }
    mg.df[v + 1] = x;
  }
  for (int u = 0; u < K; u++) {
    mg.dk[u] = mg.Dp[mg.nd[u]];
    mg.zk[u] = mg.zp[mg.nd[u]];
  }
  mg.ctl[0] = K;
  mg.ctl[1] = ng;
  mg.ctl[2] = nf;
}

// QsT[q][r] = column perm[q] of the node's block (row r), then the deflation
// rotations applied in order (thread per row r).
__global__ void k_dc_gather_rotate(int64_t off, int s, const double* __restrict__ Q, int64_t ldq, DcMerge mg,
                                   double* __restrict__ QsT) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  const double* Qr = Q + (off + r) * ldq + off;
  for (int q = 0; q < s; q++) QsT[(int64_t)q * s + r] = Qr[mg.perm[q]];
  const int ng = mg.ctl[1];
  for (int g = 0; g < ng; g++) {
    const int i = mg.gi[g], j = mg.gj[g];
    const double c = mg.gc[g], sn = mg.gs[g];
    const double qi = QsT[(int64_t)i * s + r], qj = QsT[(int64_t)j * s + r];
    QsT[(int64_t)i * s + r] = c * qi + sn * qj;
    QsT[(int64_t)j * s + r] = -sn * qi + c * qj;
  }
}

// Root j of the secular equation F(l) = 1/rho + sum_i z_i^2 / (d_i - l) = 0
// (d ascending, rho > 0): in (d_j, d_j+1) for j < K-1, in (d_K-1, d_K-1 + rho
// |z|^2] for the last.  The root is carried as an offset tau from the nearer
// pole (origin), so that every difference d_i - lambda = (d_i - d_o) - tau is
// accurate.  Each iteration fits the poles left of the interval by
// c1 + s1/(d_j - l) and those right of it by c2 + s2/(d_j+1 - l) (value and
// derivative matched at the current point) and takes the root of the fit in
// the interval, falling back to bisection of the bracket.
__global__ void k_dc_secular(DcMerge mg, int* __restrict__ err) {
  const int K = mg.ctl[0];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= K) return;
  const double rho = mg.rho[0];
  const double* dk = mg.dk;
  const double* zk = mg.zk;
  int o;
  double lo, hi;
  if (j < K - 1) {
    const double mid = 0.5 * (dk[j + 1] - dk[j]);
    double f = 1.0 / rho;
    for (int i = 0; i < K; i++) f += zk[i] * zk[i] / ((dk[i] - dk[j]) - mid);
    if (f >= 0) {
      o = j;
      lo = 0.0;
      hi = mid;
    } else {
      o = j + 1;
      lo = -mid;
      hi = 0.0;
    }
  } else {
    o = j;
    double z2 = 0;
    for (int i = 0; i < K; i++) z2 += zk[i] * zk[i];
    lo = 0.0;
    hi = rho * z2;
  }
  const double dor = dk[o];
  double tau = 0.5 * (lo + hi);
  bool conv = false;
  for (int it = 0; it < 200; it++) {
    double F = 1.0 / rho, aF = 1.0 / rho, p1 = 0, dp1 = 0, p2 = 0, dp2 = 0;
    for (int i = 0; i < K; i++) {
      const double del = (dk[i] - dor) - tau;
      const double tm = zk[i] * zk[i] / del;
      F += tm;
      aF += fabs(tm);
      if (i <= j) {
        p1 += tm;
        dp1 += tm / del;
      } else {
        p2 += tm;
        dp2 += tm / del;
      }
    }
    if (fabs(F) <= 8.0 * kEps * aF) {
      conv = true;
      break;
    }
    if (F < 0) lo = tau;
    else hi = tau;
    double eta;
    const double a1 = (dk[j] - dor) - tau;
    if (j < K - 1) {
      const double a2 = (dk[j + 1] - dor) - tau;
      const double s1 = dp1 * a1 * a1, s2 = dp2 * a2 * a2;
      const double c = 1.0 / rho + (p1 - s1 / a1) + (p2 - s2 / a2);
      // c (a1 - x)(a2 - x) + s1 (a2 - x) + s2 (a1 - x) = 0, root x in (a1, a2)
      const double qa = c, qb = -(c * (a1 + a2) + s1 + s2), qc = c * a1 * a2 + s1 * a2 + s2 * a1;
      eta = NAN;
      if (qa == 0.0) {
        if (qb != 0.0) eta = -qc / qb;
      } else {
        const double disc = fmax(qb * qb - 4.0 * qa * qc, 0.0);
        const double qq = -0.5 * (qb + copysign(sqrt(disc), qb));
        const double x1 = qq / qa, x2 = qq != 0.0 ? qc / qq : NAN;
        const double lo_x = fmin(a1, a2), hi_x = fmax(a1, a2);
        if (x1 > lo_x && x1 < hi_x) eta = x1;
        else if (x2 > lo_x && x2 < hi_x) eta = x2;
      }
    } else {
      const double s1 = dp1 * a1 * a1;
      const double c = 1.0 / rho + (p1 - s1 / a1);
      eta = c != 0.0 ? a1 + s1 / c : NAN;
    }
    double nt = tau + eta;
    if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
    if (nt == tau) {
      conv = true;
      break;
    }
    tau = nt;
  }
  if (!conv) atomicExch(err, 3);
  mg.orig[j] = o;
  mg.taus[j] = tau;
  mg.lam[j] = dor + tau;
}

// Loewner: zh_i^2 = prod_j (lambda_j - d_i) / (rho prod_{j != i} (d_j - d_i)),
// as a product of ratios of order one; sign of z_i.
__global__ void k_dc_lowner(DcMerge mg) {
  const int K = mg.ctl[0];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K) return;
  const double* dk = mg.dk;
  const double di = dk[i];
  auto lmd = [&](int j) { return (dk[mg.orig[j]] - di) + mg.taus[j]; };
  double prod = lmd(K - 1) / mg.rho[0];
  for (int j = 0; j < K - 1; j++) prod *= lmd(j) / ((j < i ? dk[j] : dk[j + 1]) - di);
  mg.zh[i] = copysign(sqrt(fmax(prod, 0.0)), mg.zk[i]);
}

// Column norms of u_j = zh / (d - lambda_j) (thread per column).
__global__ void k_dc_colnorm(DcMerge mg) {
  const int K = mg.ctl[0];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= K) return;
  const double dor = mg.dk[mg.orig[j]], tj = mg.taus[j];
  double s = 0;
  for (int i = 0; i < K; i++) {
    const double u = mg.zh[i] / ((mg.dk[i] - dor) - tj);
    s += u * u;
  }
  mg.cnrm[j] = sqrt(s);
}

// U[i][j] = zh_i / (d_i - lambda_j) / |u_j| (K x K, row-major), and the
// non-deflated columns of QsT gathered: QselT[q][r] = QsT[nd[q]][r].
__global__ void k_dc_vectors(int s, DcMerge mg, double* __restrict__ U, const double* __restrict__ QsT,
                             double* __restrict__ QselT) {
  const int K = mg.ctl[0];
  const int64_t tot = (int64_t)K * K, tot2 = (int64_t)K * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot + tot2;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < tot) {
      const int i = (int)(e / K), j = (int)(e % K);
      U[e] = mg.zh[i] / ((mg.dk[i] - mg.dk[mg.orig[j]]) - mg.taus[j]) / mg.cnrm[j];
    } else {
      const int64_t f = e - tot;
      const int q = (int)(f / s), r = (int)(f % s);
      QselT[f] = QsT[(int64_t)mg.nd[q] * s + r];
    }
  }
}

// The node's eigenvalues in ascending order (roots and deflated values
// merged) and, per final position, the source column.
__global__ void k_dc_order(int64_t off, DcMerge mg, double* __restrict__ D) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int K = mg.ctl[0], nf = mg.ctl[2];
  int a = 0, b = 0, t = 0;
  while (a < K || b < nf) {
    const bool root = b >= nf || (a < K && mg.lam[a] <= mg.Dp[mg.df[b]]);
    if (root) {
      D[off + t] = mg.lam[a];
      mg.src[t] = a++;
    } else {
      D[off + t] = mg.Dp[mg.df[b]];
      mg.src[t] = -1 - b++;
    }
    t++;
  }
}

// Q block column t <- its source: row r of Qn (s x K) or of column df[.] of QsT.
__global__ void k_dc_assemble(int64_t off, int s, DcMerge mg, const double* __restrict__ Qn,
                              const double* __restrict__ QsT, double* __restrict__ Q, int64_t ldq) {
  const int K = mg.ctl[0];
  const int64_t tot = (int64_t)s * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / s), t = (int)(e % s);
    const int sc = mg.src[t];
    Q[(off + r) * ldq + off + t] =
        sc >= 0 ? Qn[(int64_t)r * K + sc] : QsT[(int64_t)mg.df[-1 - sc] * s + r];
  }
}

// Block reflector of the back-transformation: Vp (rows x nbp, rows [j0+1, n))
// with the unit leading entries and the stored reflectors of columns
// j0 .. j0+nbp-1 of A.
__global__ void k_bt_vp(int64_t n, int64_t j0, int nbp, const double* __restrict__ A, double* __restrict__ Vp) {
  const int64_t rows = n - j0 - 1, tot = rows * nbp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = j0 + 1 + e / nbp;
    const int c = (int)(e % nbp);
    const int64_t jc = j0 + c;
    Vp[e] = i == jc + 1 ? 1.0 : (i > jc + 1 ? A[i * n + jc] : 0.0);
  }
}

// Triangular factor of the compact WY form H_j0 ... H_j0+nbp-1 = I - V T V^T:
// T[c][c] = tau_c, T[0:c, c] = -tau_c T[0:c, 0:c] (V^T V)[0:c, c].
__global__ void k_bt_tfactor(int nbp, const double* __restrict__ VtV, const double* __restrict__ tau,
                             double* __restrict__ T) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int e = 0; e < nbp * nbp; e++) T[e] = 0.0;
  for (int c = 0; c < nbp; c++) {
    const double tc = tau[c];
    T[c * nbp + c] = tc;
    for (int r = 0; r < c; r++) {
      double s = 0;
      for (int q = r; q < c; q++) s += T[r * nbp + q] * VtV[q * nbp + c];
      T[r * nbp + c] = -tc * s;
    }
  }
}

__global__ void k_copy_cols(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                            double* __restrict__ dst, int64_t ldd) {
  const int64_t tot = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
    dst[(e / cols) * ldd + e % cols] = src[(e / cols) * lds + e % cols];
}

__global__ void k_transpose_into(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                                 double* __restrict__ dst, int64_t ldd) {
  const int64_t tot = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    dst[c * ldd + r] = src[r * lds + c];
  }
}

__global__ void k_symmetrize_full(int64_t n, double* __restrict__ A) {
  const int64_t tot = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    if (j > i) {
      const double v = 0.5 * (A[i * n + j] + A[j * n + i]);
      A[i * n + j] = v;
      A[j * n + i] = v;
    }
  }
}

inline unsigned grid_for(int64_t tot, int threads = 256) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(tot, threads), 152 * 16));
}

struct Node {
  int off, s, m;
};

void build_tree(int off, int s, std::vector<Node>& merges, std::vector<int>& loff, std::vector<int>& lsize) {
  if (s <= kLeaf) {
    loff.push_back(off);
    lsize.push_back(s);
    return;
  }
  const int m = s / 2;
  build_tree(off, m, merges, loff, lsize);
  build_tree(off + m, s - m, merges, loff, lsize);
  merges.push_back({off, s, m});  // post-order: children first
}

}  // namespace

// Eigen-decomposition of a symmetric n x n A (row-major; both triangles read
// and symmetrised): all eigenvalues ascending into w_dev (and w_host); the
// eigenvectors of the `want` largest (want <= n) into rows 0..want-1 of A,
// ascending, row q = eigenvector of w[n - want + q].
fkf_status eigh_own(fkf_ctx* ctx, int n, double* A, double* w_dev, std::vector<double>& w_host, DevBuf& ws,
                    int want) {
  cudaStream_t st = ctx->stream;
  w_host.assign(n, 0.0);
  if (n <= 0) return FKF_OK;
  want = std::max(0, std::min(want, n));
  const int64_t N = n, nn = N * N;
  const int64_t L = 2 * kNB;
  // workspace layout (doubles)
  int sms = 0;
  FKF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  const int gmax = std::max(1, sms);
  const int64_t w_Q = nn, w_QsT = nn, w_QselT = nn, w_U = nn, w_Qn = nn;
  const int64_t w_X = N * std::max(want, 1);
  const int64_t w_VW = N * L, w_WV = N * L;
  const int64_t w_vec = 20 * N + 64;                       // d, e, tau, col, vg, pg, zc, the merge arrays
  const int64_t w_part = (int64_t)gmax * (1 + L) + 64;
  const int64_t w_small = 4 * kNB * kNB + 2 * N * kNB + 64;  // back-transformation
  const int64_t total = w_Q + w_QsT + w_QselT + w_U + w_Qn + w_X + w_VW + w_WV + w_vec + w_part + w_small;
  const size_t ints = (size_t)12 * N + 64;
  const size_t need = (size_t)total * 8 + ints * 4 + 256;
  if (ws.bytes < need) FKF_TRY(dev_alloc(ctx, ws, need));
  double* p = ws.as<double>();
  auto take = [&](int64_t k) {
    double* r = p;
    p += k;
    return r;
  };
  double* Q = take(w_Q);
  double* QsT = take(w_QsT);
  double* QselT = take(w_QselT);
  double* U = take(w_U);
  double* Qn = take(w_Qn);
  double* X = take(w_X);
  double* VW = take(w_VW);
  double* WV = take(w_WV);
  double* d = take(N);
  double* e = take(N);
  double* tau = take(N);
  double* col = take(N);
  double* vg = take(N);
  double* pg = take(N);
  DcMerge mg{};
  mg.Dp = take(N);
  mg.zp = take(N);
  mg.gc = take(N);
  mg.gs = take(N);
  mg.dk = take(N);
  mg.zk = take(N);
  mg.taus = take(N);
  mg.lam = take(N);
  mg.zh = take(N);
  mg.cnrm = take(N);
  mg.rho = take(8);
  double* zc = take(N);
  double* part = take(w_part);
  double* Vp = take(N * kNB);
  double* Y1 = take(N * kNB);
  double* VtV = take(kNB * kNB);
  double* Tf = take(kNB * kNB);
  int* ip = reinterpret_cast<int*>(p + 8);
  mg.perm = ip;
  mg.gi = ip + N;
  mg.gj = ip + 2 * N;
  mg.nd = ip + 3 * N;
  mg.df = ip + 4 * N;
  mg.orig = ip + 5 * N;
  mg.src = ip + 6 * N;
  int* loff_d = ip + 7 * N;
  int* lsize_d = ip + 8 * N;
  int* splits_d = ip + 9 * N;
  mg.ctl = ip + 10 * N;   // 8 ints
  unsigned* bar = reinterpret_cast<unsigned*>(ip + 10 * N + 8);
  int* err = ip + 10 * N + 16;
  FKF_CUDA(ctx, cudaMemsetAsync(err, 0, 4 * sizeof(int), st));
  FKF_CUDA(ctx, cudaMemsetAsync(e, 0, N * 8, st));
  FKF_CUDA(ctx, cudaMemsetAsync(tau, 0, N * 8, st));
  k_symmetrize_full<<<grid_for(nn), 256, 0, st>>>(N, A);
  FKF_LAUNCHED(ctx);

  // ---- 1. tridiagonal reduction
  for (int64_t j0 = 0; j0 < N; j0 += kNB) {
    const int nbp = (int)std::min<int64_t>(kNB, N - j0);
    FKF_CUDA(ctx, cudaMemsetAsync(VW, 0, w_VW * 8, st));
    FKF_CUDA(ctx, cudaMemsetAsync(WV, 0, w_WV * 8, st));
    FKF_CUDA(ctx, cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(gmax, (N - j0) / 16));
    TrdArgs ta{A, N, j0, nbp, VW, WV, d, e, tau, col, vg, pg, part, bar, err};
    void* args[] = {&ta};
    FKF_CUDA(ctx, cudaLaunchCooperativeKernel((const void*)k_trd_panel, dim3(G), dim3(kTrdThreads), args, 0, st));
    ctx->launches++;
    const int64_t j1 = j0 + nbp;
    if (j1 < N) {
      // A[j1:, j1:] -= [V W] [W V]^T = V W^T + W V^T
      FKF_TRY(gemm_sym_f64(ctx, false, true, N - j1, L, -1.0, VW + j1 * L, L, WV + j1 * L, L, 1.0, A + j1 * N + j1, N));
    }
  }

  // ---- 2. divide and conquer on the tridiagonal (d, e)
  std::vector<Node> merges;
  std::vector<int> loff, lsize, splits;
  build_tree(0, n, merges, loff, lsize);
  for (const Node& nd : merges) splits.push_back(nd.off + nd.m);
  FKF_CUDA(ctx, cudaMemsetAsync(Q, 0, nn * 8, st));
  FKF_CUDA(ctx, cudaMemcpyAsync(loff_d, loff.data(), loff.size() * 4, cudaMemcpyHostToDevice, st));
  FKF_CUDA(ctx, cudaMemcpyAsync(lsize_d, lsize.data(), lsize.size() * 4, cudaMemcpyHostToDevice, st));
  if (!splits.empty()) {
    FKF_CUDA(ctx, cudaMemcpyAsync(splits_d, splits.data(), splits.size() * 4, cudaMemcpyHostToDevice, st));
    k_dc_split_d<<<1, 32, 0, st>>>((int)splits.size(), splits_d, d, e);
    FKF_LAUNCHED(ctx);
  }
  double* Dv = w_dev;  // eigenvalues of the nodes, in place
  k_dc_leaf<<<(unsigned)loff.size(), 32, 0, st>>>(loff_d, lsize_d, d, e, Dv, Q, N, err);
  FKF_LAUNCHED(ctx);
  for (const Node& nd : merges) {
    const int s = nd.s;
    k_dc_prep<<<1, 256, 0, st>>>(nd.off, s, nd.m, nd.off + nd.m - 1, e, Dv, Q, N, mg, zc);
    FKF_LAUNCHED(ctx);
    int hc[3] = {0, 0, 0};
    FKF_CUDA(ctx, cudaMemcpyAsync(hc, mg.ctl, sizeof(hc), cudaMemcpyDeviceToHost, st));
    k_dc_gather_rotate<<<(unsigned)cdiv(s, 128), 128, 0, st>>>(nd.off, s, Q, N, mg, QsT);
    FKF_LAUNCHED(ctx);
    FKF_CUDA(ctx, cudaStreamSynchronize(st));
    const int K = hc[0];
    if (K > 0) {
      k_dc_secular<<<(unsigned)cdiv(K, 64), 64, 0, st>>>(mg, err);
      FKF_LAUNCHED(ctx);
      k_dc_lowner<<<(unsigned)cdiv(K, 64), 64, 0, st>>>(mg);
      FKF_LAUNCHED(ctx);
      k_dc_colnorm<<<(unsigned)cdiv(K, 64), 64, 0, st>>>(mg);
      FKF_LAUNCHED(ctx);
      k_dc_vectors<<<grid_for((int64_t)K * K + (int64_t)K * s), 256, 0, st>>>(s, mg, U, QsT, QselT);
      FKF_LAUNCHED(ctx);
      // Qn (s x K) = QselT^T U
      FKF_TRY(gemm_f64(ctx, true, false, s, K, K, 1.0, QselT, s, U, K, 0.0, Qn, K));
    }
    k_dc_order<<<1, 32, 0, st>>>(nd.off, mg, Dv);
    FKF_LAUNCHED(ctx);
    k_dc_assemble<<<grid_for((int64_t)s * s), 256, 0, st>>>(nd.off, s, mg, Qn, QsT, Q, N);
    FKF_LAUNCHED(ctx);
  }

  // ---- 3. back-transformation of the wanted eigenvectors (the last `want` columns of Q)
  if (want > 0) {
    const int64_t k = want;
    k_copy_cols<<<grid_for(N * k), 256, 0, st>>>(N, k, Q + (N - k), N, X, k);
    FKF_LAUNCHED(ctx);
    const int64_t nref = N - 1;  // reflectors 0 .. n-2 (the last has tau = 0 when n - 2 < 0)
    for (int64_t j0 = ((nref - 1) / kNB) * kNB; nref > 0 && j0 >= 0; j0 -= kNB) {
      const int nbp = (int)std::min<int64_t>(kNB, nref - j0);
      const int64_t rows = N - j0 - 1;
      if (rows <= 0 || nbp <= 0) continue;
      k_bt_vp<<<grid_for(rows * nbp), 256, 0, st>>>(N, j0, nbp, A, Vp);
      FKF_LAUNCHED(ctx);
      FKF_TRY(gemm_f64(ctx, true, false, nbp, nbp, rows, 1.0, Vp, nbp, Vp, nbp, 0.0, VtV, nbp));
      k_bt_tfactor<<<1, 32, 0, st>>>(nbp, VtV, tau + j0, Tf);
      FKF_LAUNCHED(ctx);
      double* Xs = X + (j0 + 1) * k;
      FKF_TRY(gemm_f64(ctx, true, false, nbp, k, rows, 1.0, Vp, nbp, Xs, k, 0.0, Y1, k));
      FKF_TRY(gemm_f64(ctx, false, false, nbp, k, nbp, 1.0, Tf, nbp, Y1, k, 0.0, QselT, k));
      FKF_TRY(gemm_f64(ctx, false, false, rows, k, nbp, -1.0, Vp, nbp, QselT, k, 1.0, Xs, k));
    }
    // eigenvector q (column q of X) -> row q of A
    k_transpose_into<<<grid_for(N * k), 256, 0, st>>>(N, k, X, k, A, N);
    FKF_LAUNCHED(ctx);
  }
  int herr = 0;
  FKF_CUDA(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  FKF_CUDA(ctx, cudaMemcpyAsync(w_host.data(), w_dev, N * 8, cudaMemcpyDeviceToHost, st));
  FKF_CUDA(ctx, cudaStreamSynchronize(st));
  if (herr) return set_err(ctx, FKF_ENOCONV, "symmetric eigensolver: %s (n=%d)",
                           herr == 1 ? "a grid barrier timed out" : (herr == 2 ? "QL did not converge" :
                                                                                  "secular equation did not converge"),
                           n);
  return FKF_OK;
}
