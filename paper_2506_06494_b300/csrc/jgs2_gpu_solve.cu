// Multi-RHS substitutions with the rest Hessian's supernodal factor on the GPU, for the
// offline stage (Sec. 6: H_bar is factorised once and every later solve reuses the factor;
// Sec. 5: the training poses come from block inverse iteration, Eq. u from the rows of
// H_bar^{-1} at the pool vertices).
//
// Device layout:
//   L32    every supernode's L block (column-major, leading dimension m = 3nJ + 3nR),
//          rounded to FP32, one after another (offset Loff[s]).
//   rdof   per supernode, the global DOF of each of its 3nR below-rows.
//   items  each supernode's 3nJ columns are cut into panels of at most kPW columns, and the
//          rows below a panel into ranges of at most kRS rows; one work item is a (panel,
//          row range). Panel q of supernode s runs after panel q-1 of s and after every
//          panel of s's descendants in the elimination tree: level(s, 0) = max over the
//          children c of level(c, last) + 1. Items are sorted by level.
//   H      H_bar in block CSR (both triangles, row-major 3x3 blocks), FP64.
//   X, B, R row-major [n][k] FP64 (iterate, right-hand sides, residual); W [n][k] FP32.
//
// Forward (L y = r), level by level: one block per panel solves the panel's diagonal
// block in shared memory and stores y_panel; then every item subtracts L_rows y_panel
// from its row range: rows of the panel's own supernode by plain stores (no other item of
// the level touches them), ancestor rows by atomicAdd (several supernodes of one level can
// share an ancestor row). The atomics make the order of the FP32 sums vary from run to
// run; the FP64 refinement below absorbs it.
// Backward (L^T x = y), levels in reverse: an item gathers L_rows^T x_rows over its row
// range (reads of rows that are already final); a panel with several items sums their
// partials from scratch in a fixed order, then solves with the diagonal block transposed.
// Refinement: X += solve32(R), R = B - H_bar X in FP64, until every column has
// |R| <= tol |B|. With kappa(H_bar) eps_32 < 1 each round contracts the error by about
// kappa eps_32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "jgs2_precompute.h"

namespace jgs2 {
namespace pre {

namespace {

constexpr int kPW = 32;    // panel width (columns of L)
constexpr int kCW = 32;    // right-hand-side columns per block
constexpr int kRT = 64;    // rows per shared-memory tile
constexpr int kRS = 256;   // rows per work item at most
constexpr int kThreads = 256;
static_assert(kPW == 32, "panel solves keep one panel row per lane");

struct SolveDev {
  const float* L;
  const long long* Loff;    // [ns]
  const int* sn_f3;         // [ns] first DOF
  const int* sn_nJ;         // [ns] 3 nJ
  const int* sn_m;          // [ns] 3 nJ + 3 nR
  const int* rdof_off;      // [ns]
  const int* rdof;          // below-row DOFs
  const int* it_sn;         // [items] supernode
  const int* it_c0;         // panel's first column (local)
  const int* it_c1;         // one past the panel's last column
  const int* it_r0;         // row range [r0, r1) (local rows, >= c1)
  const int* it_r1;
  const int* pn_item0;      // per panel (level order): its first item and item count
  const int* pn_nitem;
  const int* it_slot;       // backward scratch slot of an item of a multi-item panel, else -1
};

__device__ __forceinline__ int dof_of(const SolveDev& d, int s, int f3, int nJ, int r) {
  return r < nJ ? f3 + r : d.rdof[d.rdof_off[s] + r - nJ];
}

// Loads the panel's diagonal block (rows and columns [c0, c1)) into Ld (zero padded).
__device__ __forceinline__ void load_diag(const float* __restrict__ L, int m, int c0, int pw,
                                          float (&Ld)[kPW][kPW + 1]) {
  for (int q = threadIdx.x; q < kPW * kPW; q += kThreads) {
    const int j = q / kPW, i = q % kPW;
    Ld[i][j] = (i < pw && j < pw) ? L[(size_t)(c0 + j) * m + c0 + i] : 0.f;
  }
}

// Loads rows [r0, r0 + nr) of the panel's columns into Lt (zero padded).
__device__ __forceinline__ void load_rows(const float* __restrict__ L, int m, int c0, int pw, int r0, int nr,
                                          float (&Lt)[kRT][kPW + 1]) {
  for (int q = threadIdx.x; q < kRT * kPW; q += kThreads) {
    const int j = q / kRT, i = q % kRT;
    Lt[i][j] = (i < nr && j < pw) ? L[(size_t)(c0 + j) * m + r0 + i] : 0.f;
  }
}

// xs <- L_d^{-1} xs (L_d lower triangular, pw x pw, zero padded), every column of xs: warp w
// takes columns w, w + 8, ...; lane i holds row i, and step j broadcasts x_j by a shuffle.
__device__ __forceinline__ void panel_solve_lower(const float (&Ld)[kPW][kPW + 1], float (&xs)[kPW][kCW + 1],
                                                  int pw) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float dinv = lane < pw ? 1.f / Ld[lane][lane] : 0.f;
  for (int c = wid; c < kCW; c += kThreads / 32) {
    float x = xs[lane][c];
    for (int j = 0; j < pw; ++j) {
      const float xj = __shfl_sync(0xffffffffu, x * dinv, j);
      if (lane == j) x = xj;
      else if (lane > j) x -= Ld[lane][j] * xj;
    }
    xs[lane][c] = x;
  }
}

// xs <- L_d^{-T} xs (the transposed panel solve of the backward pass), same layout.
__device__ __forceinline__ void panel_solve_upper(const float (&Ld)[kPW][kPW + 1], float (&xs)[kPW][kCW + 1],
                                                  int pw) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float dinv = lane < pw ? 1.f / Ld[lane][lane] : 0.f;
  for (int c = wid; c < kCW; c += kThreads / 32) {
    float x = xs[lane][c];
    for (int j = pw - 1; j >= 0; --j) {
      const float xj = __shfl_sync(0xffffffffu, x * dinv, j);
      if (lane == j) x = xj;
      else if (lane < j) x -= Ld[j][lane] * xj;
    }
    xs[lane][c] = x;
  }
}

// Forward, step 1 of a level: y_panel = L_panel^{-1} r_panel for the level's panels.
__global__ void __launch_bounds__(kThreads) k_fwd_panel(SolveDev d, int pn0, float* __restrict__ W, int k) {
  __shared__ float Ld[kPW][kPW + 1];
  __shared__ float xs[kPW][kCW + 1];
  const int it = d.pn_item0[pn0 + blockIdx.x];
  const int s = d.it_sn[it], c0 = d.it_c0[it], pw = d.it_c1[it] - c0;
  const int m = d.sn_m[s], f3 = d.sn_f3[s];
  const float* L = d.L + d.Loff[s];
  const int col0 = blockIdx.y * kCW, cw = min(kCW, k - col0);
  const int tid = threadIdx.x;
  load_diag(L, m, c0, pw, Ld);
  for (int q = tid; q < kPW * kCW; q += kThreads) {
    const int i = q / kCW, c = q % kCW;
    xs[i][c] = (i < pw && c < cw) ? W[(size_t)(f3 + c0 + i) * k + col0 + c] : 0.f;
  }
  __syncthreads();
  panel_solve_lower(Ld, xs, pw);
  __syncthreads();
  for (int q = tid; q < pw * kCW; q += kThreads) {
    const int i = q / kCW, c = q % kCW;
    if (c < cw) W[(size_t)(f3 + c0 + i) * k + col0 + c] = xs[i][c];
  }
}

// Forward, step 2 of a level: every item subtracts L_rows y_panel from its row range.
__global__ void __launch_bounds__(kThreads) k_fwd_update(SolveDev d, int i0, float* __restrict__ W, int k) {
  __shared__ float xs[kPW][kCW + 1];
  __shared__ float Lt[kRT][kPW + 1];
  const int it = i0 + blockIdx.x;
  const int s = d.it_sn[it], c0 = d.it_c0[it], c1 = d.it_c1[it], pw = c1 - c0;
  const int r0 = d.it_r0[it], r1 = d.it_r1[it];
  if (r0 >= r1) return;
  const int m = d.sn_m[s], nJ = d.sn_nJ[s], f3 = d.sn_f3[s];
  const float* L = d.L + d.Loff[s];
  const int col0 = blockIdx.y * kCW, cw = min(kCW, k - col0);
  const int tid = threadIdx.x;
  for (int q = tid; q < kPW * kCW; q += kThreads) {
    const int i = q / kCW, c = q % kCW;
    xs[i][c] = (i < pw && c < cw) ? W[(size_t)(f3 + c0 + i) * k + col0 + c] : 0.f;
  }
  const int c = tid % 32, rg = tid / 32;
  __syncthreads();
  float xv[kPW];  // this thread's column of y_panel, in registers
#pragma unroll
  for (int j = 0; j < kPW; ++j) xv[j] = xs[j][c];
  for (int t0 = r0; t0 < r1; t0 += kRT) {
    const int nr = min(kRT, r1 - t0);
    __syncthreads();
    load_rows(L, m, c0, pw, t0, nr, Lt);
    __syncthreads();
    for (int i = rg; i < nr; i += kThreads / 32) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < kPW; ++j) acc += Lt[i][j] * xv[j];
      if (c < cw) {
        const int r = t0 + i;
        if (r < nJ)
          W[(size_t)(f3 + r) * k + col0 + c] -= acc;
        else
          atomicAdd(&W[(size_t)d.rdof[d.rdof_off[s] + r - nJ] * k + col0 + c], -acc);
      }
    }
  }
}

// Gathers acc[q] = sum over the item's rows r of L[r][c0 + ig + 8q] x[r] for this thread's
// column c (ig = warp index).
__device__ __forceinline__ void bwd_gather(const SolveDev& d, int it, const float* __restrict__ W, int k, int col0,
                                           int cw, float (&Lt)[kRT][kPW + 1], float (&Wt)[kRT][kCW + 1],
                                           float (&acc)[kPW / 8]) {
  const int s = d.it_sn[it], c0 = d.it_c0[it], pw = d.it_c1[it] - c0;
  const int r0 = d.it_r0[it], r1 = d.it_r1[it];
  const int m = d.sn_m[s], nJ = d.sn_nJ[s], f3 = d.sn_f3[s];
  const float* L = d.L + d.Loff[s];
  const int tid = threadIdx.x, c = tid % 32, ig = tid / 32;
  for (int t0 = r0; t0 < r1; t0 += kRT) {
    const int nr = min(kRT, r1 - t0);
    __syncthreads();
    load_rows(L, m, c0, pw, t0, nr, Lt);
    for (int q = tid; q < kRT * kCW; q += kThreads) {
      const int i = q / kCW, cc = q % kCW;
      Wt[i][cc] = (i < nr && cc < cw) ? W[(size_t)dof_of(d, s, f3, nJ, t0 + i) * k + col0 + cc] : 0.f;
    }
    __syncthreads();
    for (int i = 0; i < nr; ++i) {
      const float w = Wt[i][c];
#pragma unroll
      for (int q = 0; q < kPW / 8; ++q) acc[q] += Lt[i][ig + 8 * q] * w;
    }
  }
}

// Backward partial sums of the items of multi-item panels: scratch[slot][chunk][kPW][kCW].
__global__ void __launch_bounds__(kThreads) k_bwd_partial(SolveDev d, int i0, const float* __restrict__ W, int k,
                                                          float* __restrict__ scratch, int nchunk) {
  __shared__ float Lt[kRT][kPW + 1];
  __shared__ float Wt[kRT][kCW + 1];
  const int it = i0 + blockIdx.x;
  const int slot = d.it_slot[it];
  if (slot < 0) return;
  const int col0 = blockIdx.y * kCW, cw = min(kCW, k - col0);
  float acc[kPW / 8] = {0.f, 0.f, 0.f, 0.f};
  bwd_gather(d, it, W, k, col0, cw, Lt, Wt, acc);
  const int c = threadIdx.x % 32, ig = threadIdx.x / 32;
  float* o = scratch + ((size_t)slot * nchunk + blockIdx.y) * kPW * kCW;
#pragma unroll
  for (int q = 0; q < kPW / 8; ++q) o[(ig + 8 * q) * kCW + c] = acc[q];
}

// Backward solve of the panels of one level (pn0 .. pn0 + gridDim.x).
__global__ void __launch_bounds__(kThreads) k_bwd_panel(SolveDev d, int pn0, float* __restrict__ W, int k,
                                                        const float* __restrict__ scratch, int nchunk) {
  __shared__ float Ld[kPW][kPW + 1];
  __shared__ float xs[kPW][kCW + 1];
  __shared__ float Lt[kRT][kPW + 1];
  __shared__ float Wt[kRT][kCW + 1];
  const int pn = pn0 + blockIdx.x;
  const int it0 = d.pn_item0[pn], nit = d.pn_nitem[pn];
  const int s = d.it_sn[it0], c0 = d.it_c0[it0], pw = d.it_c1[it0] - c0;
  const int m = d.sn_m[s], f3 = d.sn_f3[s];
  const float* L = d.L + d.Loff[s];
  const int col0 = blockIdx.y * kCW, cw = min(kCW, k - col0);
  const int tid = threadIdx.x, c = tid % 32, ig = tid / 32;
  float acc[kPW / 8] = {0.f, 0.f, 0.f, 0.f};
  if (nit == 1) {
    bwd_gather(d, it0, W, k, col0, cw, Lt, Wt, acc);
  } else {
    for (int q = 0; q < nit; ++q) {  // fixed order
      const float* o = scratch + ((size_t)d.it_slot[it0 + q] * nchunk + blockIdx.y) * kPW * kCW;
#pragma unroll
      for (int u = 0; u < kPW / 8; ++u) acc[u] += o[(ig + 8 * u) * kCW + c];
    }
  }
  __syncthreads();
  load_diag(L, m, c0, pw, Ld);
#pragma unroll
  for (int q = 0; q < kPW / 8; ++q) {
    const int i = ig + 8 * q;
    xs[i][c] = (i < pw && c < cw) ? W[(size_t)(f3 + c0 + i) * k + col0 + c] - acc[q] : 0.f;
  }
  __syncthreads();
  panel_solve_upper(Ld, xs, pw);
  __syncthreads();
  for (int q = tid; q < pw * kCW; q += kThreads) {
    const int i = q / kCW, cc = q % kCW;
    if (cc < cw) W[(size_t)(f3 + c0 + i) * k + col0 + cc] = xs[i][cc];
  }
}

// R = B - H X (FP64), thread per (vertex row, column).
__global__ void k_residual(const int* __restrict__ hp, const int* __restrict__ hc, const double* __restrict__ hv,
                           const double* __restrict__ B, const double* __restrict__ X, double* __restrict__ R,
                           int nv, int k) {
  const long long total = (long long)nv * k;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(q / k), c = (int)(q % k);
    double a0 = B[(size_t)(3 * v) * k + c], a1 = B[(size_t)(3 * v + 1) * k + c], a2 = B[(size_t)(3 * v + 2) * k + c];
    for (int e = hp[v]; e < hp[v + 1]; ++e) {
      const int u = hc[e];
      const double* h = hv + (size_t)9 * e;
      const double x0 = X[(size_t)(3 * u) * k + c], x1 = X[(size_t)(3 * u + 1) * k + c],
                   x2 = X[(size_t)(3 * u + 2) * k + c];
      a0 -= h[0] * x0 + h[1] * x1 + h[2] * x2;
      a1 -= h[3] * x0 + h[4] * x1 + h[5] * x2;
      a2 -= h[6] * x0 + h[7] * x1 + h[8] * x2;
    }
    R[(size_t)(3 * v) * k + c] = a0;
    R[(size_t)(3 * v + 1) * k + c] = a1;
    R[(size_t)(3 * v + 2) * k + c] = a2;
  }
}

// Column sums of squares of A ([n][k]) added into out[k] (rows split over blockIdx.y).
__global__ void k_colnorm2(const double* __restrict__ A, int n, int k, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const int rows = (n + gridDim.y - 1) / gridDim.y;
  const int a = blockIdx.y * rows, b = min(n, a + rows);
  double s = 0.0;
  for (int i = a; i < b; ++i) {
    const double v = A[(size_t)i * k + c];
    s += v * v;
  }
  atomicAdd(&out[c], s);
}

__global__ void k_to_f32(const double* __restrict__ R, float* __restrict__ W, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    W[q] = (float)R[q];
}

__global__ void k_add_f32(double* __restrict__ X, const float* __restrict__ W, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    X[q] += (double)W[q];
}

// --- block inverse iteration on the device (Sec. 5's training poses): the block Q stays in
// device memory; the p x p pieces (Gram matrices, Cholesky, Ritz eigenproblem) go through
// the host.

constexpr int kEigP = 64;     // block width at most
constexpr int kEigRows = 32;  // rows per shared-memory tile of k_gram

// Per-block partial sums of A^T B (both [n][p] row-major) into partial[blk][p*p].
__global__ void __launch_bounds__(256) k_gram(const double* __restrict__ A, const double* __restrict__ Bm, int n,
                                              int p, double* __restrict__ partial) {
  __shared__ double As[kEigRows][kEigP], Bs[kEigRows][kEigP];
  double acc[kEigP * kEigP / 256];
  const int ne = p * p;
#pragma unroll
  for (int q = 0; q < kEigP * kEigP / 256; ++q) acc[q] = 0.0;
  const int rows = (n + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rows, r1 = min(n, r0 + rows);
  for (int t0 = r0; t0 < r1; t0 += kEigRows) {
    const int nr = min(kEigRows, r1 - t0);
    __syncthreads();
    for (int q = threadIdx.x; q < kEigRows * p; q += blockDim.x) {
      const int i = q / p, j = q % p;
      As[i][j] = i < nr ? A[(size_t)(t0 + i) * p + j] : 0.0;
      Bs[i][j] = i < nr ? Bm[(size_t)(t0 + i) * p + j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kEigP * kEigP / 256; ++q) {
      const int e = threadIdx.x + 256 * q;
      if (e < ne) {
        const int a = e / p, b = e % p;
        double s = 0.0;
        for (int i = 0; i < nr; ++i) s += As[i][a] * Bs[i][b];
        acc[q] += s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kEigP * kEigP / 256; ++q) {
    const int e = threadIdx.x + 256 * q;
    if (e < ne) partial[(size_t)blockIdx.x * ne + e] = acc[q];
  }
}

// out[e] = sum over blocks of partial[blk][e], in block order.
__global__ void k_sum_blocks(const double* __restrict__ partial, int nblk, int ne, double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * ne + e];
  out[e] = s;
}

// Row-wise forward substitution x <- x L^-T with L the lower Cholesky factor of the Gram
// matrix (column-major, element (j, q) at L[j + q p]): X R^-1 with R = L^T.
__global__ void k_rowsolve(double* __restrict__ X, const double* __restrict__ L, int n, int p) {
  __shared__ double Ls[kEigP * kEigP];
  for (int q = threadIdx.x; q < p * p; q += blockDim.x) Ls[q] = L[q];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[kEigP];
  for (int j = 0; j < p; ++j) x[j] = X[(size_t)i * p + j];
  for (int j = 0; j < p; ++j) {
    double v = x[j];
    for (int q = 0; q < j; ++q) v -= x[q] * Ls[j + q * p];
    x[j] = v / Ls[j + j * p];
  }
  for (int j = 0; j < p; ++j) X[(size_t)i * p + j] = x[j];
}

// out = A M, A [n][p] row-major, M [p][p] row-major.
__global__ void k_rowmul(const double* __restrict__ A, const double* __restrict__ M, int n, int p,
                         double* __restrict__ out) {
  __shared__ double Ms[kEigP * kEigP];
  for (int q = threadIdx.x; q < p * p; q += blockDim.x) Ms[q] = M[q];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a[kEigP];
  for (int j = 0; j < p; ++j) a[j] = A[(size_t)i * p + j];
  for (int j = 0; j < p; ++j) {
    double s = 0.0;
    for (int q = 0; q < p; ++q) s += a[q] * Ms[q * p + j];
    out[(size_t)i * p + j] = s;
  }
}

// Y = H_bar X (block CSR, both triangles), thread per (vertex row, column).
__global__ void k_hmul(const int* __restrict__ hp, const int* __restrict__ hc, const double* __restrict__ hv,
                       const double* __restrict__ X, double* __restrict__ Y, int nv, int k) {
  const long long total = (long long)nv * k;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(q / k), c = (int)(q % k);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int e = hp[v]; e < hp[v + 1]; ++e) {
      const int u = hc[e];
      const double* h = hv + (size_t)9 * e;
      const double x0 = X[(size_t)(3 * u) * k + c], x1 = X[(size_t)(3 * u + 1) * k + c],
                   x2 = X[(size_t)(3 * u + 2) * k + c];
      a0 += h[0] * x0 + h[1] * x1 + h[2] * x2;
      a1 += h[3] * x0 + h[4] * x1 + h[5] * x2;
      a2 += h[6] * x0 + h[7] * x1 + h[8] * x2;
    }
    Y[(size_t)(3 * v) * k + c] = a0;
    Y[(size_t)(3 * v + 1) * k + c] = a1;
    Y[(size_t)(3 * v + 2) * k + c] = a2;
  }
}

// out[j] += sum over rows of (HQ[i][j] - lam[j] Q[i][j])^2 for j < nt (rows split over blockIdx.y).
__global__ void k_ritz_residual(const double* __restrict__ HQ, const double* __restrict__ Q,
                                const double* __restrict__ lam, int n, int p, int nt, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nt) return;
  const int rows = (n + gridDim.y - 1) / gridDim.y;
  const int a = blockIdx.y * rows, b = min(n, a + rows);
  double s = 0.0;
  for (int i = a; i < b; ++i) {
    const double d = HQ[(size_t)i * p + j] - lam[j] * Q[(size_t)i * p + j];
    s += d * d;
  }
  atomicAdd(&out[j], s);
}

template <typename T>
bool dalloc(T** p, size_t n, std::string& err) {
  *p = nullptr;
  if (n == 0) n = 1;
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
  if (e != cudaSuccess) {
    err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    *p = nullptr;
    return false;
  }
  return true;
}

template <typename T>
bool upload(T** p, const std::vector<T>& v, std::string& err) {
  if (!dalloc(p, v.size(), err)) return false;
  if (v.empty()) return true;
  const cudaError_t e = cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    err = std::string("cudaMemcpy: ") + cudaGetErrorString(e);
    return false;
  }
  return true;
}

}  // namespace

class GpuSolver {
 public:
  int nv = 0, n = 0, ns = 0;
  // level schedule
  std::vector<int> lev_item;   // [nlev + 1] item offsets
  std::vector<int> lev_panel;  // [nlev + 1] panel offsets
  std::vector<int> lev_slots;  // [nlev] scratch slots used by the level
  int max_slots = 0;
  // device
  float* L = nullptr;
  long long* Loff = nullptr;
  int *sn_f3 = nullptr, *sn_nJ = nullptr, *sn_m = nullptr, *rdof_off = nullptr, *rdof = nullptr;
  int *it_sn = nullptr, *it_c0 = nullptr, *it_c1 = nullptr, *it_r0 = nullptr, *it_r1 = nullptr,
      *it_slot = nullptr, *pn_item0 = nullptr, *pn_nitem = nullptr;
  int *hp = nullptr, *hc = nullptr;
  double* hv = nullptr;
  cudaStream_t stream = nullptr;
  // work buffers of gpu_solve_many, kept between calls (grown on demand)
  size_t cap_nk = 0, cap_k = 0, cap_scr = 0;
  double *B = nullptr, *X = nullptr, *R = nullptr, *nb = nullptr, *nr = nullptr;
  float *W = nullptr, *scr = nullptr;
  // block inverse iteration: the block Q, H_bar Q, a rotation target, Gram partials, p x p
  int en = 0, ep = 0, enblk = 0;
  double *eQ = nullptr, *eHQ = nullptr, *eT = nullptr, *ePart = nullptr, *eSmall = nullptr, *eLam = nullptr,
         *eRes = nullptr;

  SolveDev view() const {
    return SolveDev{L, Loff, sn_f3, sn_nJ, sn_m, rdof_off, rdof, it_sn, it_c0, it_c1, it_r0, it_r1,
                    pn_item0, pn_nitem, it_slot};
  }

  ~GpuSolver() {
    void* ptrs[] = {L, Loff, sn_f3, sn_nJ, sn_m, rdof_off, rdof, it_sn, it_c0, it_c1, it_r0, it_r1,
                    it_slot, pn_item0, pn_nitem, hp, hc, hv, B, X, R, nb, nr, W, scr,
                    eQ, eHQ, eT, ePart, eSmall, eLam, eRes};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    if (stream) cudaStreamDestroy(stream);
  }
};

GpuSolver* gpu_solver_create(const Factor& F, const std::vector<BlockCol>& H, std::string& err) {
  GpuSolver* S = new GpuSolver();
  S->nv = F.nv;
  S->n = 3 * F.nv;
  const int ns = F.nsn();
  S->ns = ns;
  // supernode data, parents and panel counts
  std::vector<int> f3(ns), nJ(ns), m(ns), roff(ns), par(ns, -1), npan(ns);
  std::vector<long long> Loff(ns);
  std::vector<int> rd;
  long long tot = 0;
  for (int s = 0; s < ns; ++s) {
    const int f = F.sn_first[s];
    f3[s] = 3 * f;
    nJ[s] = 3 * (F.sn_first[s + 1] - f);
    const std::vector<int>& R = F.sn_rows[s];
    m[s] = nJ[s] + 3 * (int)R.size();
    Loff[s] = tot;
    tot += (long long)m[s] * nJ[s];
    roff[s] = (int)rd.size();
    for (int v : R)
      for (int a = 0; a < 3; ++a) rd.push_back(3 * v + a);
    if (!R.empty()) par[s] = F.sn_of[R[0]];
    npan[s] = (nJ[s] + kPW - 1) / kPW;
  }
  // level of each supernode's first panel (children come before parents in supernode order)
  std::vector<int> lvl0(ns, 0);
  int nlev = 0;
  for (int s = 0; s < ns; ++s) {
    const int end = lvl0[s] + npan[s];
    nlev = std::max(nlev, end);
    if (par[s] >= 0) {
      if (par[s] <= s) {
        err = "supernode order is not topological";
        delete S;
        return nullptr;
      }
      lvl0[par[s]] = std::max(lvl0[par[s]], end);
    }
  }
  // panels per level, then items (row ranges) per panel
  std::vector<int> pcount(nlev + 1, 0);
  for (int s = 0; s < ns; ++s)
    for (int q = 0; q < npan[s]; ++q) pcount[lvl0[s] + q + 1]++;
  for (int l = 0; l < nlev; ++l) pcount[l + 1] += pcount[l];
  const int npanels = pcount[nlev];
  std::vector<int> p_sn(npanels), p_c0(npanels), p_c1(npanels);
  {
    std::vector<int> fill(pcount.begin(), pcount.end() - 1);
    for (int s = 0; s < ns; ++s)
      for (int q = 0; q < npan[s]; ++q) {
        const int at = fill[lvl0[s] + q]++;
        p_sn[at] = s;
        p_c0[at] = q * kPW;
        p_c1[at] = std::min(nJ[s], (q + 1) * kPW);
      }
  }
  std::vector<int> i_sn, i_c0, i_c1, i_r0, i_r1, i_slot, pn_item0(npanels), pn_nitem(npanels);
  S->lev_item.assign(nlev + 1, 0);
  S->lev_panel = pcount;
  S->lev_slots.assign(nlev, 0);
  for (int l = 0; l < nlev; ++l) {
    int slots = 0;
    for (int pn = pcount[l]; pn < pcount[l + 1]; ++pn) {
      const int s = p_sn[pn], c1 = p_c1[pn];
      const int rows = m[s] - c1;
      const int nit = std::max(1, (rows + kRS - 1) / kRS);
      pn_item0[pn] = (int)i_sn.size();
      pn_nitem[pn] = nit;
      for (int q = 0; q < nit; ++q) {
        i_sn.push_back(s);
        i_c0.push_back(p_c0[pn]);
        i_c1.push_back(c1);
        i_r0.push_back(c1 + q * kRS);
        i_r1.push_back(std::min(m[s], c1 + (q + 1) * kRS));
        i_slot.push_back(nit > 1 ? slots++ : -1);
      }
    }
    S->lev_item[l + 1] = (int)i_sn.size();
    S->lev_slots[l] = slots;
    S->max_slots = std::max(S->max_slots, slots);
  }
  if (std::getenv("JGS2_VERBOSE")) {
    int maxp = 0;
    for (int l = 0; l < nlev; ++l) maxp = std::max(maxp, pcount[l + 1] - pcount[l]);
    std::fprintf(stderr,
                 "[jgs2_precompute] gpu schedule: %d supernodes, %d panels, %d items, %d levels "
                 "(widest %d panels), %d scratch slots, %.3e factor entries\n",
                 ns, npanels, (int)i_sn.size(), nlev, maxp, S->max_slots, (double)tot);
  }
  // H_bar in block CSR, both triangles
  const int nvv = F.nv;
  std::vector<int> cnt(nvv + 1, 0);
  for (int c = 0; c < nvv; ++c)
    for (int u : H[c].row) {
      cnt[u + 1]++;
      if (u != c) cnt[c + 1]++;
    }
  for (int v = 0; v < nvv; ++v) cnt[v + 1] += cnt[v];
  std::vector<int> hc(cnt[nvv]);
  std::vector<double> hv((size_t)9 * cnt[nvv]);
  {
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int c = 0; c < nvv; ++c)
      for (size_t q = 0; q < H[c].row.size(); ++q) {
        const int u = H[c].row[q];
        const double* b = &H[c].val[9 * q];  // block (u, c)
        int at = fill[u]++;
        hc[at] = c;
        for (int e = 0; e < 9; ++e) hv[(size_t)9 * at + e] = b[e];
        if (u != c) {
          at = fill[c]++;
          hc[at] = u;
          for (int a = 0; a < 3; ++a)
            for (int b2 = 0; b2 < 3; ++b2) hv[(size_t)9 * at + 3 * a + b2] = b[3 * b2 + a];
        }
      }
  }
  // factor in FP32
  bool ok = dalloc(&S->L, (size_t)tot, err);
  if (ok) {
    std::vector<float> buf;
    for (int s = 0; s < ns && ok; ++s) {
      const RawVec& Ls = F.L[s];
      buf.resize(Ls.size());
      for (size_t q = 0; q < Ls.size(); ++q) buf[q] = (float)Ls[q];
      const cudaError_t e =
          cudaMemcpy(S->L + Loff[s], buf.data(), buf.size() * sizeof(float), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        err = std::string("cudaMemcpy: ") + cudaGetErrorString(e);
        ok = false;
      }
    }
  }
  ok = ok && upload(&S->Loff, Loff, err) && upload(&S->sn_f3, f3, err) && upload(&S->sn_nJ, nJ, err) &&
       upload(&S->sn_m, m, err) && upload(&S->rdof_off, roff, err) && upload(&S->rdof, rd, err) &&
       upload(&S->it_sn, i_sn, err) && upload(&S->it_c0, i_c0, err) && upload(&S->it_c1, i_c1, err) &&
       upload(&S->it_r0, i_r0, err) && upload(&S->it_r1, i_r1, err) &&
       upload(&S->it_slot, i_slot, err) && upload(&S->pn_item0, pn_item0, err) &&
       upload(&S->pn_nitem, pn_nitem, err) && upload(&S->hp, cnt, err) && upload(&S->hc, hc, err) &&
       upload(&S->hv, hv, err);
  if (ok) {
    const cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
      ok = false;
    }
  }
  if (!ok) {
    delete S;
    return nullptr;
  }
  return S;
}

// Work buffers for k right-hand sides (grown on demand).
static bool ensure_bufs(GpuSolver* S, int n, int k, std::string& err) {
  const size_t nk = (size_t)n * k;
  const int nchunk = (k + kCW - 1) / kCW;
  const size_t nscr = (size_t)std::max(1, S->max_slots) * nchunk * kPW * kCW;
  if (nk > S->cap_nk || (size_t)k > S->cap_k || nscr > S->cap_scr) {
    void* old[] = {S->B, S->X, S->R, S->nb, S->nr, S->W, S->scr};
    for (void* p : old)
      if (p) cudaFree(p);
    S->B = S->X = S->R = S->nb = S->nr = nullptr;
    S->W = S->scr = nullptr;
    S->cap_nk = S->cap_k = S->cap_scr = 0;
    if (!dalloc(&S->B, nk, err) || !dalloc(&S->X, nk, err) || !dalloc(&S->R, nk, err) ||
        !dalloc(&S->W, nk, err) || !dalloc(&S->nb, k, err) || !dalloc(&S->nr, k, err) ||
        !dalloc(&S->scr, nscr, err))
      return false;
    S->cap_nk = nk;
    S->cap_k = k;
    S->cap_scr = nscr;
  }
  return true;
}

// H_bar X = B for the k columns in S->B (device), solution in S->X: FP32 substitutions,
// FP64 refinement (see gpu_solve_many). Returns the rounds taken, or -1 with err set.
static int solve_core(GpuSolver* S, int n, int k, double tol, double accept, int max_refine, std::string& err) {
  const size_t nk = (size_t)n * k;
  const int nchunk = (k + kCW - 1) / kCW;
  double *B = S->B, *X = S->X, *R = S->R, *nb = S->nb, *nr = S->nr;
  float *W = S->W, *scr = S->scr;
  const bool verbose = std::getenv("JGS2_VERBOSE") != nullptr;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  float t_fwd = 0.f, t_bwd = 0.f;
  if (verbose)
    for (auto& e : ev) cudaEventCreate(&e);
  cudaStream_t st = S->stream;
  const SolveDev d = S->view();
  const int nlev = (int)S->lev_slots.size();
  const int ew_grid = 148 * 8;
  std::vector<double> hb(k), hr(k);
  int rounds = -1;
  double prev = INFINITY, worst = INFINITY;
  cudaError_t e = cudaMemsetAsync(X, 0, nk * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(R, B, nk * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(nb, 0, k * sizeof(double), st);
  if (e == cudaSuccess) {
    const int gy = std::max(1, std::min(256, n / 256));
    k_colnorm2<<<dim3((k + 127) / 128, gy), 128, 0, st>>>(B, n, k, nb);
    e = cudaMemcpyAsync(hb.data(), nb, k * sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (int round = 0; e == cudaSuccess && round < max_refine; ++round) {
    k_to_f32<<<ew_grid, 256, 0, st>>>(R, W, (long long)nk);
    if (verbose) cudaEventRecord(ev[0], st);
    for (int l = 0; l < nlev; ++l) {
      const int np = S->lev_panel[l + 1] - S->lev_panel[l];
      if (np > 0) k_fwd_panel<<<dim3(np, nchunk), kThreads, 0, st>>>(d, S->lev_panel[l], W, k);
      const int ni = S->lev_item[l + 1] - S->lev_item[l];
      if (ni > 0) k_fwd_update<<<dim3(ni, nchunk), kThreads, 0, st>>>(d, S->lev_item[l], W, k);
    }
    if (verbose) cudaEventRecord(ev[1], st);
    for (int l = nlev - 1; l >= 0; --l) {
      const int ni = S->lev_item[l + 1] - S->lev_item[l];
      if (S->lev_slots[l] > 0) k_bwd_partial<<<dim3(ni, nchunk), kThreads, 0, st>>>(d, S->lev_item[l], W, k, scr, nchunk);
      const int np = S->lev_panel[l + 1] - S->lev_panel[l];
      if (np > 0) k_bwd_panel<<<dim3(np, nchunk), kThreads, 0, st>>>(d, S->lev_panel[l], W, k, scr, nchunk);
    }
    if (verbose) cudaEventRecord(ev[2], st);
    k_add_f32<<<ew_grid, 256, 0, st>>>(X, W, (long long)nk);
    k_residual<<<ew_grid, 256, 0, st>>>(S->hp, S->hc, S->hv, B, X, R, S->nv, k);
    cudaMemsetAsync(nr, 0, k * sizeof(double), st);
    const int gy = std::max(1, std::min(256, n / 256));
    k_colnorm2<<<dim3((k + 127) / 128, gy), 128, 0, st>>>(R, n, k, nr);
    e = cudaMemcpyAsync(hr.data(), nr, k * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) break;
    if (verbose) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, ev[0], ev[1]);
      cudaEventElapsedTime(&b, ev[1], ev[2]);
      t_fwd += a;
      t_bwd += b;
    }
    worst = 0.0;
    for (int c = 0; c < k; ++c) {
      const double rel = hb[c] > 0.0 ? std::sqrt(hr[c] / hb[c]) : std::sqrt(hr[c]);
      worst = std::max(worst, std::isfinite(rel) ? rel : INFINITY);
    }
    rounds = round + 1;
    // done at tol, or when a round no longer halves the worst residual (the FP64 residual's
    // own rounding floor, or kappa eps_32 too large to contract)
    if (worst <= tol || !(worst < 0.5 * prev)) break;
    prev = worst;
  }
  if (!(worst <= accept)) {
    if (err.empty())
      err = "gpu_solve_many: refinement ended at relative residual " + std::to_string(worst * 1e10) + "e-10" + " after " +
            std::to_string(rounds) + " rounds";
    rounds = -1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    err = std::string("gpu_solve_many: ") + cudaGetErrorString(e);
    rounds = -1;
  }
  if (verbose) {
    std::fprintf(stderr, "[jgs2_precompute] gpu solve: %d columns, substitutions %.2f ms forward, %.2f ms backward\n",
                 k, t_fwd, t_bwd);
    for (auto& ev1 : ev) cudaEventDestroy(ev1);
  }
  return rounds;
}

int gpu_solve_many(GpuSolver* S, double* Bh, int n, int k, double tol, double accept, int max_refine,
                   std::string& err) {
  if (!S || n != S->n || k <= 0) {
    err = "gpu_solve_many: bad arguments";
    return -1;
  }
  if (!ensure_bufs(S, n, k, err)) return -1;
  const size_t nk = (size_t)n * k;
  cudaError_t e = cudaMemcpyAsync(S->B, Bh, nk * sizeof(double), cudaMemcpyHostToDevice, S->stream);
  if (e != cudaSuccess) {
    err = std::string("gpu_solve_many: ") + cudaGetErrorString(e);
    return -1;
  }
  const int rounds = solve_core(S, n, k, tol, accept, max_refine, err);
  e = cudaMemcpyAsync(Bh, S->X, nk * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
  if (e != cudaSuccess) {
    err = std::string("gpu_solve_many: ") + cudaGetErrorString(e);
    return -1;
  }
  return rounds;
}

// ------------------------------------------------------------------ block inverse iteration

static bool cuda_ok(cudaError_t e, const char* what, std::string& err) {
  if (e == cudaSuccess) return true;
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

bool gpu_eig_begin(GpuSolver* S, const double* Qh, int n, int p, std::string& err) {
  if (!S || n != S->n || p <= 0 || p > kEigP) {
    err = "gpu_eig_begin: block wider than the device kernels take";
    return false;
  }
  const size_t np = (size_t)n * p;
  S->en = n;
  S->ep = p;
  S->enblk = std::max(1, std::min(148 * 4, (n + kEigRows - 1) / kEigRows));
  if (!ensure_bufs(S, n, p, err) || !dalloc(&S->eQ, np, err) || !dalloc(&S->eHQ, np, err) ||
      !dalloc(&S->eT, np, err) || !dalloc(&S->ePart, (size_t)S->enblk * p * p, err) ||
      !dalloc(&S->eSmall, (size_t)p * p, err) || !dalloc(&S->eLam, p, err) || !dalloc(&S->eRes, p, err))
    return false;
  return cuda_ok(cudaMemcpyAsync(S->eQ, Qh, np * sizeof(double), cudaMemcpyHostToDevice, S->stream), "gpu_eig_begin",
                 err);
}

int gpu_eig_solve(GpuSolver* S, double tol, double accept, int max_refine, std::string& err) {
  const size_t np = (size_t)S->en * S->ep;
  if (!cuda_ok(cudaMemcpyAsync(S->B, S->eQ, np * sizeof(double), cudaMemcpyDeviceToDevice, S->stream), "gpu_eig_solve",
               err))
    return -1;
  const int rounds = solve_core(S, S->en, S->ep, tol, accept, max_refine, err);
  if (rounds < 0) return -1;
  if (!cuda_ok(cudaMemcpyAsync(S->eQ, S->X, np * sizeof(double), cudaMemcpyDeviceToDevice, S->stream), "gpu_eig_solve",
               err))
    return -1;
  return rounds;
}

bool gpu_eig_gram(GpuSolver* S, bool with_hq, double* out, std::string& err) {
  const int p = S->ep;
  k_gram<<<S->enblk, 256, 0, S->stream>>>(S->eQ, with_hq ? S->eHQ : S->eQ, S->en, p, S->ePart);
  k_sum_blocks<<<(p * p + 255) / 256, 256, 0, S->stream>>>(S->ePart, S->enblk, p * p, S->eSmall);
  return cuda_ok(cudaMemcpyAsync(out, S->eSmall, sizeof(double) * p * p, cudaMemcpyDeviceToHost, S->stream),
                 "gpu_eig_gram", err) &&
         cuda_ok(cudaStreamSynchronize(S->stream), "gpu_eig_gram", err);
}

bool gpu_eig_rowsolve(GpuSolver* S, const double* L, std::string& err) {
  const int p = S->ep;
  if (!cuda_ok(cudaMemcpyAsync(S->eSmall, L, sizeof(double) * p * p, cudaMemcpyHostToDevice, S->stream),
               "gpu_eig_rowsolve", err))
    return false;
  k_rowsolve<<<(S->en + 127) / 128, 128, 0, S->stream>>>(S->eQ, S->eSmall, S->en, p);
  return cuda_ok(cudaGetLastError(), "gpu_eig_rowsolve", err);
}

bool gpu_eig_hmul(GpuSolver* S, std::string& err) {
  k_hmul<<<148 * 8, 256, 0, S->stream>>>(S->hp, S->hc, S->hv, S->eQ, S->eHQ, S->nv, S->ep);
  return cuda_ok(cudaGetLastError(), "gpu_eig_hmul", err);
}

bool gpu_eig_rotate(GpuSolver* S, const double* Vs, std::string& err) {
  const int p = S->ep, nb = (S->en + 127) / 128;
  if (!cuda_ok(cudaMemcpyAsync(S->eSmall, Vs, sizeof(double) * p * p, cudaMemcpyHostToDevice, S->stream),
               "gpu_eig_rotate", err))
    return false;
  k_rowmul<<<nb, 128, 0, S->stream>>>(S->eQ, S->eSmall, S->en, p, S->eT);
  std::swap(S->eQ, S->eT);
  k_rowmul<<<nb, 128, 0, S->stream>>>(S->eHQ, S->eSmall, S->en, p, S->eT);
  std::swap(S->eHQ, S->eT);
  return cuda_ok(cudaGetLastError(), "gpu_eig_rotate", err);
}

bool gpu_eig_residuals(GpuSolver* S, const double* lam, int nt, double* out, std::string& err) {
  const int p = S->ep;
  if (!cuda_ok(cudaMemcpyAsync(S->eLam, lam, sizeof(double) * p, cudaMemcpyHostToDevice, S->stream),
               "gpu_eig_residuals", err) ||
      !cuda_ok(cudaMemsetAsync(S->eRes, 0, sizeof(double) * p, S->stream), "gpu_eig_residuals", err))
    return false;
  const int gy = std::max(1, std::min(256, S->en / 256));
  k_ritz_residual<<<dim3((nt + 63) / 64, gy), 64, 0, S->stream>>>(S->eHQ, S->eQ, S->eLam, S->en, p, nt, S->eRes);
  return cuda_ok(cudaMemcpyAsync(out, S->eRes, sizeof(double) * nt, cudaMemcpyDeviceToHost, S->stream),
                 "gpu_eig_residuals", err) &&
         cuda_ok(cudaStreamSynchronize(S->stream), "gpu_eig_residuals", err);
}

bool gpu_eig_end(GpuSolver* S, double* Qh, std::string& err) {
  const size_t np = (size_t)S->en * S->ep;
  const bool ok = cuda_ok(cudaMemcpyAsync(Qh, S->eQ, np * sizeof(double), cudaMemcpyDeviceToHost, S->stream),
                          "gpu_eig_end", err) &&
                  cuda_ok(cudaStreamSynchronize(S->stream), "gpu_eig_end", err);
  double** bufs[] = {&S->eQ, &S->eHQ, &S->eT, &S->ePart, &S->eSmall, &S->eLam, &S->eRes};
  for (double** b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  return ok;
}

void gpu_solver_destroy(GpuSolver* S) { delete S; }

}  // namespace pre
}  // namespace jgs2
