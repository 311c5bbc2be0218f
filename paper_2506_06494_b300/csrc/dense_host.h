// Blocked dense FP64 kernels for the host precompute (column-major throughout).
// GEMM follows the packed-panel scheme of Goto & van de Geijn (ACM TOMS 2008): panels of
// op(A) and op(B) are packed into contiguous slivers and a 16x6 register-blocked
// micro-kernel (GCC vector extensions, AVX-512 width) accumulates tiles of C.
#pragma once
#include <omp.h>

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <vector>

namespace jgs2 {
namespace dense {

typedef double v8d __attribute__((vector_size(64)));

constexpr int MR = 16, NR = 6, KC = 256, MC = 128, NCT = 96;

// element (i, p) of op(A): A is m x k after op; trans -> A stored k x m
static inline double at(const double* A, int lda, bool trans, int i, int p) {
  return trans ? A[p + (size_t)i * lda] : A[i + (size_t)p * lda];
}

static inline void pack_a(const double* A, int lda, bool tA, int i0, int mb, int p0, int kb, double* out) {
  for (int ir = 0; ir < mb; ir += MR) {
    const int mr = std::min(MR, mb - ir);
    for (int p = 0; p < kb; ++p) {
      double* o = out + (size_t)(ir / MR) * MR * kb + (size_t)p * MR;
      int i = 0;
      for (; i < mr; ++i) o[i] = at(A, lda, tA, i0 + ir + i, p0 + p);
      for (; i < MR; ++i) o[i] = 0.0;
    }
  }
}

// element (p, j) of op(B): B is k x n after op; "NT" callers pass trans=true with B n x k
static inline double bt(const double* B, int ldb, bool trans, int p, int j) {
  return trans ? B[j + (size_t)p * ldb] : B[p + (size_t)j * ldb];
}

static inline void pack_b(const double* B, int ldb, bool tB, int p0, int kb, int j0, int nb, double* out) {
  for (int jr = 0; jr < nb; jr += NR) {
    const int nr = std::min(NR, nb - jr);
    for (int p = 0; p < kb; ++p) {
      double* o = out + (size_t)(jr / NR) * NR * kb + (size_t)p * NR;
      int j = 0;
      for (; j < nr; ++j) o[j] = bt(B, ldb, tB, p0 + p, j0 + jr + j);
      for (; j < NR; ++j) o[j] = 0.0;
    }
  }
}

static inline void micro(int kb, const double* a, const double* b, double alpha, double* C, int ldc, int mr,
                         int nr) {
  v8d c[NR][2];
  for (int j = 0; j < NR; ++j) c[j][0] = c[j][1] = (v8d){0, 0, 0, 0, 0, 0, 0, 0};
  for (int p = 0; p < kb; ++p) {
    v8d a0, a1;
    std::memcpy(&a0, a + (size_t)p * MR, 64);
    std::memcpy(&a1, a + (size_t)p * MR + 8, 64);
    const double* bp = b + (size_t)p * NR;
#pragma GCC unroll 6
    for (int j = 0; j < NR; ++j) {
      const double s = bp[j];
      c[j][0] += a0 * s;
      c[j][1] += a1 * s;
    }
  }
  for (int j = 0; j < nr; ++j) {
    double* cj = C + (size_t)j * ldc;
    double tmp[16];
    std::memcpy(tmp, &c[j][0], 64);
    std::memcpy(tmp + 8, &c[j][1], 64);
    for (int i = 0; i < mr; ++i) cj[i] += alpha * tmp[i];
  }
}

// C (m x n) += alpha op(A) op(B); op(A) m x k, op(B) k x n. lower: only tiles touching
// the lower triangle (j <= i) of C are formed (diagonal tiles are written whole).
static void gemm(bool tA, bool tB, int m, int n, int k, double alpha, const double* A, int lda, const double* B,
                 int ldb, double* C, int ldc, bool lower = false) {
  if (m <= 0 || n <= 0 || k <= 0) return;
  if ((double)m * n * k < 65536.0) {
    // small: direct loops (inner loop over rows of C is contiguous)
    for (int j = 0; j < n; ++j) {
      double* cj = C + (size_t)j * ldc;
      const int i0 = lower ? std::min(j, m) : 0;
      for (int p = 0; p < k; ++p) {
        const double b = alpha * bt(B, ldb, tB, p, j);
        if (b == 0.0) continue;
        if (!tA) {
          const double* ap = A + (size_t)p * lda;
          for (int i = i0; i < m; ++i) cj[i] += ap[i] * b;
        } else {
          for (int i = i0; i < m; ++i) cj[i] += A[p + (size_t)i * lda] * b;
        }
      }
    }
    return;
  }
  const int nti = (m + MC - 1) / MC, ntj = (n + NCT - 1) / NCT;
  const bool par = !omp_in_parallel() && (double)m * n * k > 4e6;
  std::vector<double> pb((size_t)((n + NR - 1) / NR) * NR * KC);
  for (int p0 = 0; p0 < k; p0 += KC) {
    const int kb = std::min(KC, k - p0);
    // pack all of op(B)[p0:p0+kb, :]
    const int nsl = (n + NR - 1) / NR;
#pragma omp parallel for schedule(static) if (par)
    for (int s = 0; s < nsl; ++s) {
      const int j0 = s * NR;
      pack_b(B, ldb, tB, p0, kb, j0, std::min(NR, n - j0), pb.data() + (size_t)s * NR * kb);
    }
#pragma omp parallel if (par)
    {
      std::vector<double> pa((size_t)MC * KC + MR * KC);
#pragma omp for schedule(dynamic, 1) collapse(2)
      for (int ti = 0; ti < nti; ++ti)
        for (int tj = 0; tj < ntj; ++tj) {
          const int i0 = ti * MC, j0 = tj * NCT;
          const int mb = std::min(MC, m - i0), nb = std::min(NCT, n - j0);
          if (lower && j0 >= i0 + mb) continue;
          pack_a(A, lda, tA, i0, mb, p0, kb, pa.data());
          for (int jr = 0; jr < nb; jr += NR) {
            const int nr = std::min(NR, nb - jr);
            const double* bsl = pb.data() + (size_t)((j0 + jr) / NR) * NR * kb;
            for (int ir = 0; ir < mb; ir += MR) {
              const int mr = std::min(MR, mb - ir);
              if (lower && j0 + jr >= i0 + ir + mr) continue;
              micro(kb, pa.data() + (size_t)(ir / MR) * MR * kb, bsl, alpha, C + (i0 + ir) + (size_t)(j0 + jr) * ldc,
                    ldc, mr, nr);
            }
          }
        }
    }
  }
}

// B (m x n) <- B L^{-T}, L lower n x n.
static void trsm_rlt(double* B, int m, int n, int ldb, const double* L, int ldl) {
  const int nb = 96;
  for (int j0 = 0; j0 < n; j0 += nb) {
    const int jb = std::min(nb, n - j0);
    // B[:, j0:j0+jb] -= B[:, 0:j0] L[j0:j0+jb, 0:j0]^T
    gemm(false, true, m, jb, j0, -1.0, B, ldb, L + j0, ldl, B + (size_t)j0 * ldb, ldb);
#pragma omp parallel for schedule(static) if (!omp_in_parallel() && (size_t)m * jb * jb > 2000000)
    for (int ib = 0; ib < m; ib += 256) {
      const int ie = std::min(m, ib + 256);
      for (int j = j0; j < j0 + jb; ++j) {
        double* cj = B + (size_t)j * ldb;
        for (int p = j0; p < j; ++p) {
          const double l = L[j + (size_t)p * ldl];
          const double* cp = B + (size_t)p * ldb;
          for (int i = ib; i < ie; ++i) cj[i] -= cp[i] * l;
        }
        const double inv = 1.0 / L[j + (size_t)j * ldl];
        for (int i = ib; i < ie; ++i) cj[i] *= inv;
      }
    }
  }
}

// B (m x n) <- B L^{-1}, L lower n x n (right side, no transpose).
static void trsm_rln(double* B, int m, int n, int ldb, const double* L, int ldl) {
  const int nb = 96;
  const int nblk = (n + nb - 1) / nb;
  for (int bk = nblk - 1; bk >= 0; --bk) {
    const int j0 = bk * nb, jb = std::min(nb, n - j0), j1 = j0 + jb;
    // B[:, j0:j1] -= B[:, j1:n] L[j1:n, j0:j1]
    gemm(false, false, m, jb, n - j1, -1.0, B + (size_t)j1 * ldb, ldb, L + j1 + (size_t)j0 * ldl, ldl,
         B + (size_t)j0 * ldb, ldb);
#pragma omp parallel for schedule(static) if (!omp_in_parallel() && (size_t)m * jb * jb > 2000000)
    for (int ib = 0; ib < m; ib += 256) {
      const int ie = std::min(m, ib + 256);
      for (int j = j1 - 1; j >= j0; --j) {
        double* cj = B + (size_t)j * ldb;
        for (int p = j + 1; p < j1; ++p) {
          const double l = L[p + (size_t)j * ldl];
          const double* cp = B + (size_t)p * ldb;
          for (int i = ib; i < ie; ++i) cj[i] -= cp[i] * l;
        }
        const double inv = 1.0 / L[j + (size_t)j * ldl];
        for (int i = ib; i < ie; ++i) cj[i] *= inv;
      }
    }
  }
}

// Right-looking forms of the two solves above, for a B with few rows (a block of
// right-hand sides): after each diagonal block the rest of B is updated by one GEMM whose
// output spans the remaining columns, so the work splits over threads by columns.
// B (m x n) <- B L^{-T}.
static void trsm_rlt_wide(double* B, int m, int n, int ldb, const double* L, int ldl) {
  const int nb = 96;
  for (int j0 = 0; j0 < n; j0 += nb) {
    const int jb = std::min(nb, n - j0), j1 = j0 + jb;
    for (int j = j0; j < j1; ++j) {
      double* cj = B + (size_t)j * ldb;
      for (int p = j0; p < j; ++p) {
        const double l = L[j + (size_t)p * ldl];
        const double* cp = B + (size_t)p * ldb;
        for (int i = 0; i < m; ++i) cj[i] -= cp[i] * l;
      }
      const double inv = 1.0 / L[j + (size_t)j * ldl];
      for (int i = 0; i < m; ++i) cj[i] *= inv;
    }
    // B[:, j1:n] -= B[:, j0:j1] L[j1:n, j0:j1]^T
    if (j1 < n) gemm(false, true, m, n - j1, jb, -1.0, B + (size_t)j0 * ldb, ldb, L + j1 + (size_t)j0 * ldl, ldl,
                     B + (size_t)j1 * ldb, ldb);
  }
}

// B (m x n) <- B L^{-1}.
static void trsm_rln_wide(double* B, int m, int n, int ldb, const double* L, int ldl) {
  const int nb = 96;
  const int nblk = (n + nb - 1) / nb;
  for (int bk = nblk - 1; bk >= 0; --bk) {
    const int j0 = bk * nb, jb = std::min(nb, n - j0), j1 = j0 + jb;
    for (int j = j1 - 1; j >= j0; --j) {
      double* cj = B + (size_t)j * ldb;
      for (int p = j + 1; p < j1; ++p) {
        const double l = L[p + (size_t)j * ldl];
        const double* cp = B + (size_t)p * ldb;
        for (int i = 0; i < m; ++i) cj[i] -= cp[i] * l;
      }
      const double inv = 1.0 / L[j + (size_t)j * ldl];
      for (int i = 0; i < m; ++i) cj[i] *= inv;
    }
    // B[:, 0:j0] -= B[:, j0:j1] L[j0:j1, 0:j0]
    if (j0 > 0) gemm(false, false, m, j0, jb, -1.0, B + (size_t)j0 * ldb, ldb, L + j0, ldl, B, ldb);
  }
}

// Lower Cholesky in place; false if a pivot is not positive.
static bool potrf(double* A, int n, int lda) {
  const int nb = 96;
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int kb = std::min(nb, n - k0);
    for (int j = k0; j < k0 + kb; ++j) {
      double d = A[j + (size_t)j * lda];
      for (int p = k0; p < j; ++p) d -= A[j + (size_t)p * lda] * A[j + (size_t)p * lda];
      if (!(d > 0.0)) return false;
      d = __builtin_sqrt(d);
      A[j + (size_t)j * lda] = d;
      for (int i = j + 1; i < k0 + kb; ++i) {
        double s = A[i + (size_t)j * lda];
        for (int p = k0; p < j; ++p) s -= A[i + (size_t)p * lda] * A[j + (size_t)p * lda];
        A[i + (size_t)j * lda] = s / d;
      }
    }
    const int r0 = k0 + kb, m = n - r0;
    if (m <= 0) continue;
    // panel below the diagonal block (its left part was updated by earlier trailing updates)
#pragma omp parallel for schedule(static) if (!omp_in_parallel() && (size_t)m * kb * kb > 2000000)
    for (int ib = 0; ib < m; ib += 256) {
      const int ie = std::min(m, ib + 256);
      for (int j = k0; j < k0 + kb; ++j) {
        double* cj = A + (size_t)j * lda + r0;
        for (int p = k0; p < j; ++p) {
          const double l = A[j + (size_t)p * lda];
          const double* cp = A + (size_t)p * lda + r0;
          for (int i = ib; i < ie; ++i) cj[i] -= cp[i] * l;
        }
        const double inv = 1.0 / A[j + (size_t)j * lda];
        for (int i = ib; i < ie; ++i) cj[i] *= inv;
      }
    }
    // trailing lower update A[r0:, r0:] -= P P^T
    const double* P = A + r0 + (size_t)k0 * lda;
    gemm(false, true, m, m, kb, -1.0, P, lda, P, lda, A + r0 + (size_t)r0 * lda, lda, true);
  }
  return true;
}

// X (n x n) = L^{-1}, L lower; X lower, zero above the diagonal.
static void trtri_lower(const double* L, int n, int ldl, double* X) {
  std::fill(X, X + (size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) X[i + (size_t)i * n] = 1.0;
  // solve L X = I by block rows: X[b,:] = L_bb^{-1} (I_b - L[b, 0:b] X[0:b, :])
  const int nb = 96;
  for (int b0 = 0; b0 < n; b0 += nb) {
    const int bb = std::min(nb, n - b0);
    // X[b0:b0+bb, 0:b0] -= L[b0:b0+bb, 0:b0] X[0:b0, 0:b0]   (columns >= b0 of rows b are I)
    gemm(false, false, bb, b0, b0, -1.0, L + b0, ldl, X, n, X + b0, n);
    // triangular solve with L_bb on columns 0:b0+bb
#pragma omp parallel for schedule(static) if (!omp_in_parallel() && (size_t)bb * bb * (b0 + bb) > 2000000)
    for (int c = 0; c < b0 + bb; ++c) {
      double* xc = X + (size_t)c * n;
      for (int i = b0; i < b0 + bb; ++i) {
        double s = xc[i];
        for (int p = b0; p < i; ++p) s -= L[i + (size_t)p * ldl] * xc[p];
        xc[i] = s / L[i + (size_t)i * ldl];
      }
    }
  }
}

}  // namespace dense
}  // namespace jgs2
