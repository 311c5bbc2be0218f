// Offline stage of JGS2 on the host, FP64 (Secs. 5-6 of Lan et al.).
//
// Per distinct body (bodies equal up to translation share one precompute):
//   1. H_bar = M/h^2 + K_bar over the body's free DOFs (rest Hessian, reading R2; the
//      element blocks are V_e (mu (b_a.b_c) I + mu b_c b_a^T + lam b_a b_c^T)).
//   2. Nested-dissection order (recursive coordinate bisection with one-sided vertex
//      separators), elimination tree, fundamental supernodes, multifrontal Cholesky
//      H_bar = L L^T with dense fronts (Sec. 6: one factorisation serves every solve).
//   3. Training poses: the n_train lowest eigenpairs of H_bar by block inverse iteration
//      with Rayleigh-Ritz (Sec. 5, last paragraph).
//   4. Rows of H_bar^{-1} at the vertices of the body's cubature pool, by multi-RHS
//      forward/backward substitution (Sec. 6: substitutions with the one factor).
//   5. Diagonal blocks A_i = (H_bar^{-1})_ii for every free vertex by selected inversion
//      (Takahashi recurrences on the supernodal pattern), so that
//      U_bar_{i,a} = (H_bar^{-1})_{a,i} A_i^{-1}  (Eq. u: U_bar_i = H^-1 S_i^T (S_i H^-1 S_i^T)^-1).
//   6. Greedy NNLS cubature per vertex (Eq. cubature_weight) with the same seeded draws,
//      training rows and stopping rule as described in the header.
#include <omp.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/jgs2.h"
#include "dense_host.h"
#include "jgs2_host.h"
#include "jgs2_precompute.h"

namespace jgs2 {
namespace pre {

using std::vector;

static bool verbose() {
  static const bool v = std::getenv("JGS2_VERBOSE") != nullptr;
  return v;
}
static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
#define PHASE(name)                                                                  \
  do {                                                                               \
    if (verbose()) std::fprintf(stderr, "[jgs2_precompute] %-18s %8.3f s\n", name, now_s() - t_phase); \
    t_phase = now_s();                                                               \
  } while (0)

// ------------------------------------------------------------------ SplitMix64
// Steele, Lea & Flood (OOPSLA 2014): state += 0x9E3779B97F4A7C15, then the output mix.
struct SplitMix {
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
};

// Stream derived from a seed and two keys by feeding each key through one output.
static SplitMix keyed(uint64_t seed, uint64_t a, uint64_t b) {
  SplitMix g{seed};
  g.s = g.next() ^ a;
  g.s = g.next() ^ b;
  return g;
}

// Partial Fisher-Yates: the first k picks of `items` (in the given order).
static vector<int> draw(SplitMix g, vector<int> items, int k) {
  const int n = (int)items.size();
  k = std::min(k, n);
  for (int j = 0; j < k; ++j) {
    const int r = j + (int)(g.next() % (uint64_t)(n - j));
    std::swap(items[j], items[r]);
  }
  items.resize(k);
  return items;
}

// Small symmetric eigen-decomposition by cyclic Jacobi (n x n row-major, vectors in V columns).
static void sym_eig(vector<double>& A, int n, vector<double>& w, vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = 0; i < n; ++i) {
      dia += A[(size_t)i * n + i] * A[(size_t)i * n + i];
      for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    }
    if (off <= 1e-30 * dia || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double tau = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// ------------------------------------------------------------------ NNLS (Lawson & Hanson 1974)
// min |A w - b|, w >= 0; A is m x n column-major (n small). Returns the residual norm.
static double lstsq_cols(const vector<double>& A, int m, const vector<int>& cols, const vector<double>& b,
                         vector<double>& s) {
  // modified Gram-Schmidt QR of the selected columns
  const int k = (int)cols.size();
  vector<double> Q((size_t)m * k), R((size_t)k * k, 0.0);
  for (int j = 0; j < k; ++j) std::memcpy(&Q[(size_t)j * m], &A[(size_t)cols[j] * m], sizeof(double) * m);
  for (int j = 0; j < k; ++j) {
    double* qj = &Q[(size_t)j * m];
    for (int p = 0; p < j; ++p) {
      const double* qp = &Q[(size_t)p * m];
      double d = 0.0;
      for (int i = 0; i < m; ++i) d += qp[i] * qj[i];
      R[(size_t)p * k + j] = d;
      for (int i = 0; i < m; ++i) qj[i] -= d * qp[i];
    }
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += qj[i] * qj[i];
    nrm = std::sqrt(nrm);
    R[(size_t)j * k + j] = nrm;
    if (nrm > 0)
      for (int i = 0; i < m; ++i) qj[i] /= nrm;
  }
  vector<double> y(k, 0.0);
  for (int j = 0; j < k; ++j) {
    double d = 0.0;
    for (int i = 0; i < m; ++i) d += Q[(size_t)j * m + i] * b[i];
    y[j] = d;
  }
  s.assign(k, 0.0);
  for (int j = k - 1; j >= 0; --j) {
    double v = y[j];
    for (int p = j + 1; p < k; ++p) v -= R[(size_t)j * k + p] * s[p];
    s[j] = R[(size_t)j * k + j] > 0 ? v / R[(size_t)j * k + j] : 0.0;
  }
  double r2 = 0.0;
  for (int i = 0; i < m; ++i) {
    double v = b[i];
    for (int j = 0; j < k; ++j) v -= A[(size_t)cols[j] * m + i] * s[j];
    r2 += v * v;
  }
  return std::sqrt(r2);
}

static double nnls(const vector<double>& A, int m, int n, const vector<double>& b, vector<double>& w) {
  w.assign(n, 0.0);
  vector<char> inP(n, 0);
  double scale = 0.0;  // stopping threshold relative to the largest |A_j^T b|
  for (int j = 0; j < n; ++j) {
    double gj = 0.0;
    for (int i = 0; i < m; ++i) gj += A[(size_t)j * m + i] * b[i];
    scale = std::max(scale, std::fabs(gj));
  }
  const double tol = 1e-13 * std::max(scale, 1e-300);
  for (int outer = 0; outer < 3 * n + 10; ++outer) {
    vector<double> r(b);
    for (int j = 0; j < n; ++j)
      if (w[j] != 0.0)
        for (int i = 0; i < m; ++i) r[i] -= A[(size_t)j * m + i] * w[j];
    int jmax = -1;
    double gmax = tol;
    for (int j = 0; j < n; ++j) {
      if (inP[j]) continue;
      double gj = 0.0;
      for (int i = 0; i < m; ++i) gj += A[(size_t)j * m + i] * r[i];
      if (gj > gmax) {
        gmax = gj;
        jmax = j;
      }
    }
    if (jmax < 0) break;
    inP[jmax] = 1;
    for (int inner = 0; inner < 3 * n + 10; ++inner) {
      vector<int> P;
      for (int j = 0; j < n; ++j)
        if (inP[j]) P.push_back(j);
      vector<double> sv;
      lstsq_cols(A, m, P, b, sv);
      bool feasible = true;
      for (double v : sv)
        if (v <= 0.0) feasible = false;
      if (feasible) {
        std::fill(w.begin(), w.end(), 0.0);
        for (size_t q = 0; q < P.size(); ++q) w[P[q]] = sv[q];
        break;
      }
      double alpha = 2.0;
      for (size_t q = 0; q < P.size(); ++q)
        if (sv[q] <= 0.0) alpha = std::min(alpha, w[P[q]] / (w[P[q]] - sv[q]));
      for (size_t q = 0; q < P.size(); ++q) w[P[q]] += alpha * (sv[q] - w[P[q]]);
      for (size_t q = 0; q < P.size(); ++q)
        if (w[P[q]] <= 1e-15) {
          w[P[q]] = 0.0;
          inP[P[q]] = 0;
        }
    }
  }
  double r2 = 0.0;
  for (int i = 0; i < m; ++i) {
    double v = b[i];
    for (int j = 0; j < n; ++j) v -= A[(size_t)j * m + i] * w[j];
    r2 += v * v;
  }
  return std::sqrt(r2);
}

// ------------------------------------------------------------------ sparse Cholesky

static void nd_order(const vector<double>& P, const vector<vector<int>>& adj, vector<int>& idx,
                     vector<char>& side, vector<int>& out) {
  if (idx.size() <= 64) {
    for (int v : idx) out.push_back(v);
    return;
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v : idx)
    for (int q = 0; q < 3; ++q) {
      lo[q] = std::min(lo[q], P[3 * v + q]);
      hi[q] = std::max(hi[q], P[3 * v + q]);
    }
  int ax = 0;
  for (int q = 1; q < 3; ++q)
    if (hi[q] - lo[q] > hi[ax] - lo[ax]) ax = q;
  const size_t mid = idx.size() / 2;
  std::nth_element(idx.begin(), idx.begin() + mid, idx.end(), [&](int a, int b) {
    if (P[3 * a + ax] != P[3 * b + ax]) return P[3 * a + ax] < P[3 * b + ax];
    return a < b;
  });
  vector<int> left(idx.begin(), idx.begin() + mid), right(idx.begin() + mid, idx.end());
  for (int v : left) side[v] = 1;
  for (int v : right) side[v] = 2;
  vector<int> sep, l2;
  for (int v : left) {
    bool s = false;
    for (int u : adj[v])
      if (side[u] == 2) {
        s = true;
        break;
      }
    (s ? sep : l2).push_back(v);
  }
  for (int v : idx) side[v] = 0;
  std::sort(l2.begin(), l2.end());
  std::sort(right.begin(), right.end());
  std::sort(sep.begin(), sep.end());
  idx.clear();
  idx.shrink_to_fit();
  nd_order(P, adj, l2, side, out);
  nd_order(P, adj, right, side, out);
  for (int v : sep) out.push_back(v);
}


// Multifrontal supernodal Cholesky of the block matrix given by its lower block columns.
static bool factorize(int nv, const vector<BlockCol>& H, Factor& F) {
  F.nv = nv;
  // elimination tree (Liu) on the vertex graph
  vector<int> parent(nv, -1), anc(nv, -1);
  for (int j = 0; j < nv; ++j) {
    // rows u > j of column j are the entries (j, u) of row u < ... : use symmetric pattern
    (void)j;
  }
  // build upper adjacency: for each column v, rows u > v; the etree needs for each j the
  // neighbours i < j
  vector<vector<int>> lowN(nv);
  for (int v = 0; v < nv; ++v)
    for (int u : H[v].row)
      if (u > v) lowN[u].push_back(v);
  for (int j = 0; j < nv; ++j)
    for (int i : lowN[j]) {
      int r = i;
      while (anc[r] != -1 && anc[r] != j) {
        const int t = anc[r];
        anc[r] = j;
        r = t;
      }
      if (anc[r] == -1) {
        anc[r] = j;
        parent[r] = j;
      }
    }
  // column structures (vertices > j), children first (ascending order is topological)
  vector<int> nchild(nv, 0);
  for (int j = 0; j < nv; ++j)
    if (parent[j] >= 0) nchild[parent[j]]++;
  vector<vector<int>> kids(nv);
  for (int j = 0; j < nv; ++j)
    if (parent[j] >= 0) kids[parent[j]].push_back(j);
  vector<vector<int>> st(nv);
  vector<int> mark(nv, -1);
  for (int j = 0; j < nv; ++j) {
    vector<int>& s = st[j];
    for (int u : H[j].row)
      if (u > j && mark[u] != j) {
        mark[u] = j;
        s.push_back(u);
      }
    for (int c : kids[j]) {
      for (int u : st[c])
        if (u > j && mark[u] != j) {
          mark[u] = j;
          s.push_back(u);
        }
    }
    std::sort(s.begin(), s.end());
  }
  // fundamental supernodes
  F.sn_first.clear();
  F.sn_of.assign(nv, 0);
  for (int j = 0; j < nv; ++j) {
    const bool merge = j > 0 && parent[j - 1] == j && nchild[j] == 1 && st[j - 1].size() == st[j].size() + 1;
    if (!merge) F.sn_first.push_back(j);
    F.sn_of[j] = (int)F.sn_first.size() - 1;
  }
  F.sn_first.push_back(nv);
  const int ns = F.nsn();
  F.sn_rows.assign(ns, {});
  for (int s = 0; s < ns; ++s) F.sn_rows[s] = st[F.sn_first[s + 1] - 1];
  st.clear();
  st.shrink_to_fit();
  // supernode tree
  vector<vector<int>> skids(ns);
  for (int s = 0; s < ns; ++s) {
    const int last = F.sn_first[s + 1] - 1;
    if (parent[last] >= 0) skids[F.sn_of[parent[last]]].push_back(s);
  }
  F.L.assign(ns, {});
  vector<RawVec> upd(ns);  // update matrices, (3 nR)^2 column-major, lower triangle used
  // Large update matrices are recycled from front to front, one pool per thread: a fresh
  // allocation of that size costs a page fault per page on first touch, which dominated
  // the fronts near the root and contends between threads deeper down.
  const int nthr = std::max(1, omp_get_max_threads());
  vector<vector<RawVec>> spares(nthr);
  auto take = [&](size_t n) {
    RawVec v;
    vector<RawVec>& spare = spares[omp_get_thread_num() % nthr];
    if (n >= (size_t)1 << 14) {
      int best = -1;
      for (int q = 0; q < (int)spare.size(); ++q)
        if (spare[q].capacity() >= n && (best < 0 || spare[q].capacity() < spare[best].capacity())) best = q;
      if (best >= 0) {
        v.swap(spare[best]);
        spare.erase(spare.begin() + best);
      }
    }
    v.resize(n);  // not initialised: the caller zeroes what it reads
    return v;
  };
  auto release = [&](RawVec& v) {
    vector<RawVec>& spare = spares[omp_get_thread_num() % nthr];
    if (v.capacity() >= (size_t)1 << 14) {
      spare.push_back(std::move(v));
      if (spare.size() > 3) {  // keep the largest few
        auto small = std::min_element(spare.begin(), spare.end(),
                                      [](const RawVec& a, const RawVec& b) { return a.capacity() < b.capacity(); });
        spare.erase(small);
      }
    }
    v = RawVec();
  };
  // One front: assemble supernode s's columns and its children's updates, factor them,
  // leave its own update matrix. loc is a scratch map vertex -> front row (-1 elsewhere).
  auto front = [&](int s, vector<int>& loc) -> bool {
    const int f = F.sn_first[s], l = F.sn_first[s + 1];
    const int nJ = 3 * (l - f);
    const vector<int>& R = F.sn_rows[s];
    const int nR = 3 * (int)R.size();
    const int m = nJ + nR;
    RawVec& Fm = F.L[s];
    Fm = RawVec((size_t)m * nJ);
    // zeroed by columns, in parallel for a large front (its first touch)
#pragma omp parallel for schedule(static) if (!omp_in_parallel() && (size_t)m * nJ >= ((size_t)1 << 20))
    for (int j = 0; j < nJ; ++j) std::memset(&Fm[(size_t)j * m], 0, sizeof(double) * m);
    RawVec U = take((size_t)nR * nR);
    // only the lower triangle of an update matrix is formed and read
#pragma omp parallel for schedule(dynamic, 64) if (!omp_in_parallel() && nR >= 768)
    for (int j = 0; j < nR; ++j) std::memset(&U[(size_t)j * nR + j], 0, sizeof(double) * (nR - j));
    for (int v = f; v < l; ++v) loc[v] = 3 * (v - f);
    for (size_t q = 0; q < R.size(); ++q) loc[R[q]] = nJ + 3 * (int)q;
    // original entries of the columns of J
    for (int v = f; v < l; ++v) {
      const int c0 = 3 * (v - f);
      for (size_t q = 0; q < H[v].row.size(); ++q) {
        const int u = H[v].row[q];
        const int r0 = loc[u];
        const double* b = &H[v].val[9 * q];
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) {
            const int rr = r0 + a, cc = c0 + c;
            if (rr >= cc) Fm[rr + (size_t)cc * m] += b[3 * a + c];
          }
      }
    }
    // extend-add of the children's update matrices
    for (int c : skids[s]) {
      const vector<int>& Rc = F.sn_rows[c];
      const int nc = 3 * (int)Rc.size();
      const RawVec& Uc = upd[c];
      vector<int> map(nc);
      for (size_t q = 0; q < Rc.size(); ++q)
        for (int a = 0; a < 3; ++a) map[3 * q + a] = loc[Rc[q]] + a;
      // map is increasing (front rows follow vertex order), so column cc of the child's
      // lower triangle lands in column map[cc] alone: columns are independent
#pragma omp parallel for schedule(dynamic, 16) if (!omp_in_parallel() && nc >= 384)
      for (int cc = 0; cc < nc; ++cc) {
        const int gc = map[cc];
        const double* uc = &Uc[(size_t)cc * nc];
        if (gc < nJ) {
          double* fc = &Fm[(size_t)gc * m];
          for (int rr = cc; rr < nc; ++rr) fc[map[rr]] += uc[rr];
        } else {
          double* uo = &U[(size_t)(gc - nJ) * nR];
          for (int rr = cc; rr < nc; ++rr) uo[map[rr] - nJ] += uc[rr];
        }
      }
      release(upd[c]);
    }
    for (int v = f; v < l; ++v) loc[v] = -1;
    for (int u : R) loc[u] = -1;
    // partial factorisation
    if (!dense::potrf(Fm.data(), nJ, m)) return false;
    if (nR > 0) {
      dense::trsm_rlt(Fm.data() + nJ, nR, nJ, m, Fm.data(), m);
      const double* LR = Fm.data() + nJ;
      dense::gemm(false, true, nR, nR, nJ, -1.0, LR, m, LR, m, U.data(), nR, true);
      upd[s].swap(U);
    }
    return true;
  };
  // Fronts by height in the supernode tree (leaves 0, a parent above all its children):
  // the fronts of one height are independent. Within a height, a front costing more than
  // a thread's share of the height runs alone on parallel dense kernels; the others run one
  // per thread (their kernels single-threaded), largest first. Each front's arithmetic
  // does not depend on the schedule.
  vector<int> height(ns, 0);
  int nh = 0;
  for (int s = 0; s < ns; ++s) {  // children precede parents
    for (int c : skids[s]) height[s] = std::max(height[s], height[c] + 1);
    nh = std::max(nh, height[s] + 1);
  }
  vector<vector<int>> by_h(nh);
  for (int s = 0; s < ns; ++s) by_h[height[s]].push_back(s);
  vector<vector<int>> locs(nthr, vector<int>(nv, -1));
  auto cost = [&](int s) {
    const double nJ = 3.0 * (F.sn_first[s + 1] - F.sn_first[s]), nR = 3.0 * F.sn_rows[s].size();
    return nJ * nJ * nJ / 3.0 + nJ * nJ * nR + nJ * nR * nR + 4.0 * nR * nR;
  };
  for (int h = 0; h < nh; ++h) {
    vector<int> lv = by_h[h];
    std::stable_sort(lv.begin(), lv.end(), [&](int a, int b2) { return cost(a) > cost(b2); });
    double total = 0.0;
    for (int q : lv) total += cost(q);
    int nbig = 0;  // the leading fronts above a thread's share
    while (nbig < (int)lv.size() && cost(lv[nbig]) > total / nthr) ++nbig;
    for (int q = 0; q < nbig; ++q)
      if (!front(lv[q], locs[0])) return false;
    const int rest = (int)lv.size() - nbig;
    if (rest >= 2 && nthr > 1 && !omp_in_parallel()) {
      int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthr) reduction(| : bad)
      for (int q = nbig; q < (int)lv.size(); ++q)
        if (!front(lv[q], locs[omp_get_thread_num()])) bad |= 1;
      if (bad) return false;
    } else {
      for (int q = nbig; q < (int)lv.size(); ++q)
        if (!front(lv[q], locs[0])) return false;
    }
  }
  return true;
}

// X (n_scalar x nrhs, row-major) <- H^{-1} X with the supernodal factor. In column-major
// terms X is the nrhs x n matrix X^T, so each supernode's steps are right-side solves and
// GEMMs on X^T: forward X_J <- X_J L_JJ^{-T}, X_R -= X_J L_RJ^T; backward
// X_J -= X_R L_RJ, X_J <- X_J L_JJ^{-1}.
static void solve_inplace(const Factor& F, double* X, int nrhs) {
  const int ns = F.nsn();
  vector<double> XR;
  for (int s = 0; s < ns; ++s) {
    const int f = F.sn_first[s], nJ = 3 * (F.sn_first[s + 1] - f);
    const vector<int>& R = F.sn_rows[s];
    const int nR = 3 * (int)R.size(), m = nJ + nR;
    const double* L = F.L[s].data();
    double* XJ = X + (size_t)3 * f * nrhs;
    dense::trsm_rlt(XJ, nrhs, nJ, nrhs, L, m);
    if (nR == 0) continue;
    XR.assign((size_t)nR * nrhs, 0.0);
    dense::gemm(false, true, nrhs, nR, nJ, -1.0, XJ, nrhs, L + nJ, m, XR.data(), nrhs);
    for (size_t q = 0; q < R.size(); ++q)
      for (int a = 0; a < 3; ++a) {
        double* xr = X + (size_t)(3 * R[q] + a) * nrhs;
        const double* d = XR.data() + (size_t)(3 * q + a) * nrhs;
        for (int c = 0; c < nrhs; ++c) xr[c] += d[c];
      }
  }
  for (int s = ns - 1; s >= 0; --s) {
    const int f = F.sn_first[s], nJ = 3 * (F.sn_first[s + 1] - f);
    const vector<int>& R = F.sn_rows[s];
    const int nR = 3 * (int)R.size(), m = nJ + nR;
    const double* L = F.L[s].data();
    double* XJ = X + (size_t)3 * f * nrhs;
    if (nR > 0) {
      XR.resize((size_t)nR * nrhs);
      for (size_t q = 0; q < R.size(); ++q)
        for (int a = 0; a < 3; ++a)
          std::memcpy(XR.data() + (size_t)(3 * q + a) * nrhs, X + (size_t)(3 * R[q] + a) * nrhs,
                      sizeof(double) * nrhs);
      dense::gemm(false, false, nrhs, nJ, nR, -1.0, XR.data(), nrhs, L + nJ, m, XJ, nrhs);
    }
    dense::trsm_rln(XJ, nrhs, nJ, nrhs, L, m);
  }
}

// Multi-RHS solve for many right-hand sides: one contiguous chunk of columns per thread,
// each a whole sequential solve (compute-bound once a chunk is a few dozen columns wide).
static void solve_chunked(const Factor& F, vector<double>& B /* n x nrhs row-major */, int n, int nrhs) {
  const int nt = std::max(1, std::min(omp_get_max_threads(), (nrhs + 3) / 4));
  if (nt == 1) {
    solve_inplace(F, B.data(), nrhs);
    return;
  }
#pragma omp parallel for schedule(static, 1) num_threads(nt)
  for (int c = 0; c < nt; ++c) {
    const int c0 = (int)((long)nrhs * c / nt), c1 = (int)((long)nrhs * (c + 1) / nt), cw = c1 - c0;
    vector<double> X((size_t)n * cw);
    for (int i = 0; i < n; ++i) std::memcpy(&X[(size_t)i * cw], &B[(size_t)i * nrhs + c0], sizeof(double) * cw);
    solve_inplace(F, X.data(), cw);
    for (int i = 0; i < n; ++i) std::memcpy(&B[(size_t)i * nrhs + c0], &X[(size_t)i * cw], sizeof(double) * cw);
  }
}

// Multi-RHS solve H X = B for a narrow block of right-hand sides (B row-major n x nrhs,
// overwritten), all of them at once, so that the factor is streamed once per solve. In column-major terms a run of rows
// of B is an nrhs x (rows) block, and each supernode's steps are right-side solves and GEMMs
// on it. The supernode tree is walked level by level, a supernode costing more than a
// thread's share of its level alone on parallel kernels, the others one per thread:
//  - forward (L Y = B), by height from the leaves: a supernode subtracts its children's
//    update rows that fall in its own columns and carries the others, solves
//    Y_J <- Y_J L_JJ^{-T}, and hands W = (carried rows) + Y_J L_RJ^T to its parent;
//  - backward (L^T X = Y), by depth from the roots: X_J <- (X_J - X_R L_RJ) L_JJ^{-1}, its
//    rows X_R belonging to ancestors that are already final.
// Each supernode's arithmetic is independent of the schedule.
static void solve_tree(const Factor& F, vector<double>& B /* n x nrhs row-major */, int n, int nrhs) {
  const int ns = F.nsn();
  if (ns == 0 || nrhs <= 0 || n <= 0) return;
  double* X = B.data();
  vector<int> par(ns, -1);
  vector<vector<int>> kids(ns);
  for (int s = 0; s < ns; ++s)
    if (!F.sn_rows[s].empty()) {
      par[s] = F.sn_of[F.sn_rows[s][0]];
      kids[par[s]].push_back(s);
    }
  vector<int> height(ns, 0), depth(ns, 0);
  int nh = 0, nd = 0;
  for (int s = 0; s < ns; ++s) {  // children come before parents
    for (int c : kids[s]) height[s] = std::max(height[s], height[c] + 1);
    nh = std::max(nh, height[s] + 1);
  }
  for (int s = ns - 1; s >= 0; --s) {
    depth[s] = par[s] < 0 ? 0 : depth[par[s]] + 1;
    nd = std::max(nd, depth[s] + 1);
  }
  vector<vector<int>> by_h(nh), by_d(nd);
  for (int s = 0; s < ns; ++s) by_h[height[s]].push_back(s);
  for (int s = ns - 1; s >= 0; --s) by_d[depth[s]].push_back(s);
  const int nthr = std::max(1, omp_get_max_threads());
  auto cost = [&](int s) {
    const double nJ = 3.0 * (F.sn_first[s + 1] - F.sn_first[s]), nR = 3.0 * F.sn_rows[s].size();
    return nJ * (nJ + 2.0 * nR) + nR;
  };
  // runs fn over the supernodes of one level: the costly ones alone, the rest in parallel
  auto run_level = [&](vector<int> lv, auto&& fn) {
    std::stable_sort(lv.begin(), lv.end(), [&](int a, int b2) { return cost(a) > cost(b2); });
    double total = 0.0;
    for (int q : lv) total += cost(q);
    int nbig = 0;
    while (nbig < (int)lv.size() && cost(lv[nbig]) > total / nthr) ++nbig;
    for (int q = 0; q < nbig; ++q) fn(lv[q], 0);
    if ((int)lv.size() - nbig >= 2 && nthr > 1 && !omp_in_parallel()) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthr)
      for (int q = nbig; q < (int)lv.size(); ++q) fn(lv[q], omp_get_thread_num());
    } else {
      for (int q = nbig; q < (int)lv.size(); ++q) fn(lv[q], 0);
    }
  };
  // forward
  vector<RawVec> W(ns);  // update rows handed to the parent: [nR][nrhs]
  vector<vector<int>> locs(nthr, vector<int>(F.nv, -1));
  auto fwd = [&](int s, int t) {
    vector<int>& loc = locs[t];
    const int f = F.sn_first[s], l = F.sn_first[s + 1], nJ = 3 * (l - f);
    const vector<int>& R = F.sn_rows[s];
    const int nR = 3 * (int)R.size(), m = nJ + nR;
    const double* L = F.L[s].data();
    double* XJ = X + (size_t)3 * f * nrhs;
    RawVec Ws((size_t)nR * nrhs);
    std::memset(Ws.data(), 0, sizeof(double) * Ws.size());
    for (size_t q = 0; q < R.size(); ++q) loc[R[q]] = (int)q;
    for (int c : kids[s]) {
      const vector<int>& Rc = F.sn_rows[c];
      const double* Wc = W[c].data();
      for (size_t qc = 0; qc < Rc.size(); ++qc) {
        const int v = Rc[qc];
        const double* src = Wc + (size_t)3 * qc * nrhs;
        if (v < l) {
          double* dst = X + (size_t)3 * v * nrhs;
          for (int i = 0; i < 3 * nrhs; ++i) dst[i] -= src[i];
        } else {
          double* dst = Ws.data() + (size_t)3 * loc[v] * nrhs;
          for (int i = 0; i < 3 * nrhs; ++i) dst[i] += src[i];
        }
      }
      W[c] = RawVec();
    }
    for (int u : R) loc[u] = -1;
    dense::trsm_rlt_wide(XJ, nrhs, nJ, nrhs, L, m);
    if (nR > 0) {
      dense::gemm(false, true, nrhs, nR, nJ, 1.0, XJ, nrhs, L + nJ, m, Ws.data(), nrhs);
      W[s].swap(Ws);
    }
  };
  for (int h = 0; h < nh; ++h) run_level(by_h[h], fwd);
  // backward
  vector<RawVec> XRs(nthr);
  auto bwd = [&](int s, int t) {
    const int f = F.sn_first[s], nJ = 3 * (F.sn_first[s + 1] - f);
    const vector<int>& R = F.sn_rows[s];
    const int nR = 3 * (int)R.size(), m = nJ + nR;
    const double* L = F.L[s].data();
    double* XJ = X + (size_t)3 * f * nrhs;
    if (nR > 0) {
      RawVec& XR = XRs[t];
      XR.resize((size_t)nR * nrhs);
      for (size_t q = 0; q < R.size(); ++q)
        std::memcpy(XR.data() + (size_t)3 * q * nrhs, X + (size_t)3 * R[q] * nrhs, sizeof(double) * 3 * nrhs);
      dense::gemm(false, false, nrhs, nJ, nR, -1.0, XR.data(), nrhs, L + nJ, m, XJ, nrhs);
    }
    dense::trsm_rln_wide(XJ, nrhs, nJ, nrhs, L, m);
  };
  for (int d = 0; d < nd; ++d) run_level(by_d[d], bwd);
}

// H X = B: narrow blocks (the inverse iteration's) by the tree pass, which streams the
// factor once; wide ones (the pool rows) by per-thread column chunks.
static void solve_many(const Factor& F, vector<double>& B /* n x nrhs row-major */, int n, int nrhs) {
  if (nrhs >= 32 * std::max(1, omp_get_max_threads()))
    solve_chunked(F, B, n, nrhs);
  else
    solve_tree(F, B, n, nrhs);
}

// Diagonal 3x3 blocks of H^{-1} by the Takahashi recurrences on the supernodal pattern
// (consumes the factor: L is overwritten with the selected inverse Z).
static void selected_inverse_diag(Factor& F, vector<double>& Adiag /* nv x 9 */) {
  const int ns = F.nsn();
  Adiag.assign((size_t)F.nv * 9, 0.0);
  // Work buffers, one set per thread, reused from supernode to supernode (fresh large
  // allocations cost a page fault per page, which dominated the deep supernodes)
  struct Bufs {
    RawVec Li, Y, ZRR, ZRJ, ZJJ;
  };
  auto sized = [](RawVec& v, size_t n, bool zero) {
    if (v.capacity() < n)
      v = RawVec(n);
    else
      v.resize(n);
    if (zero) std::memset(v.data(), 0, sizeof(double) * n);
    return v.data();
  };
  const int nthr = std::max(1, omp_get_max_threads());
  vector<Bufs> bufs(nthr);
  // Z of supernode s from the Z of its ancestors (the supernodes of its rows)
  auto sel = [&](int s, Bufs& b) {
    const int f = F.sn_first[s], nJ = 3 * (F.sn_first[s + 1] - f);
    const vector<int>& R = F.sn_rows[s];
    const int nR = 3 * (int)R.size();
    const int m = nJ + nR;
    RawVec& L = F.L[s];
    // Li = L_JJ^{-1} (lower), Y = L_RJ Li  (nR x nJ)
    double* Li = sized(b.Li, (size_t)nJ * nJ, false);  // trtri writes all of it
    dense::trtri_lower(L.data(), nJ, m, Li);
    double* Y = sized(b.Y, (size_t)nR * nJ, true);
    dense::gemm(false, false, nR, nJ, nJ, 1.0, L.data() + nJ, m, Li, nJ, Y, nR);
    // Z_RR gathered from the ancestors (already holding Z); the gather writes every entry
    double* ZRR = sized(b.ZRR, (size_t)nR * nR, false);
#pragma omp parallel for schedule(dynamic, 4) if (!omp_in_parallel() && R.size() > 64)
    for (int cb = 0; cb < (int)R.size(); ++cb) {
      const int v2 = R[cb];
      const int K = F.sn_of[v2];
      const int fK = F.sn_first[K], nJK = 3 * (F.sn_first[K + 1] - fK);
      const vector<int>& RK = F.sn_rows[K];
      const int mK = nJK + 3 * (int)RK.size();
      const double* Z = F.L[K].data();
      // rows v1 = R[rb] ascend, so their places in K's row structure (which holds every
      // row of s beyond K's own columns) are found by one forward walk
      size_t pos = 0;
      for (int rb = cb; rb < (int)R.size(); ++rb) {
        const int v1 = R[rb];
        int lr;
        if (v1 < F.sn_first[K + 1]) {
          lr = 3 * (v1 - fK);
        } else {
          while (RK[pos] < v1) ++pos;
          lr = nJK + 3 * (int)pos;
        }
        const int lc = 3 * (v2 - fK);
        // columns of the block's lower triangle (the whole block on the diagonal)
        for (int c = 0; c < 3; ++c) {
          double* zc = ZRR + (size_t)(3 * cb + c) * nR + 3 * rb;
          for (int a = 0; a < 3; ++a) {
            const int rr = lr + a, cc = lc + c;
            zc[a] = rr >= cc ? Z[rr + (size_t)cc * mK] : Z[cc + (size_t)rr * mK];  // K's diagonal block is symmetric
          }
        }
      }
    }
    // upper triangle from the lower one, by tiles
    {
      constexpr int TB = 48;
      const int nt = (nR + TB - 1) / TB;
#pragma omp parallel for schedule(dynamic, 1) if (!omp_in_parallel() && nR >= 768)
      for (int tj = 0; tj < nt; ++tj)
        for (int ti = tj; ti < nt; ++ti) {
          const int i0 = ti * TB, i1 = std::min(nR, i0 + TB), j0 = tj * TB, j1 = std::min(nR, j0 + TB);
          for (int j = j0; j < j1; ++j)
            for (int i = std::max(i0, j + 1); i < i1; ++i) ZRR[j + (size_t)i * nR] = ZRR[i + (size_t)j * nR];
        }
    }
    // Z_RJ = -Z_RR Y ; Z_JJ = Li^T Li - Y^T Z_RJ
    double* ZRJ = sized(b.ZRJ, (size_t)nR * nJ, true);
    dense::gemm(false, false, nR, nJ, nR, -1.0, ZRR, nR, Y, nR, ZRJ, nR);
    double* ZJJ = sized(b.ZJJ, (size_t)nJ * nJ, true);
    dense::gemm(true, false, nJ, nJ, nJ, 1.0, Li, nJ, Li, nJ, ZJJ, nJ);
    dense::gemm(true, false, nJ, nJ, nR, -1.0, Y, nR, ZRJ, nR, ZJJ, nJ);
    // store Z in place of L
    for (int j = 0; j < nJ; ++j) {
      for (int i = 0; i < nJ; ++i) L[i + (size_t)j * m] = ZJJ[i + (size_t)j * nJ];
      for (int r = 0; r < nR; ++r) L[nJ + r + (size_t)j * m] = ZRJ[r + (size_t)j * nR];
    }
    for (int v = f; v < F.sn_first[s + 1]; ++v)
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c)
          Adiag[(size_t)v * 9 + 3 * a + c] = ZJJ[(3 * (v - f) + a) + (size_t)(3 * (v - f) + c) * nJ];
  };
  // Supernodes by depth below their root (a parent's depth is less than its children's):
  // those of one depth read only their ancestors' Z, so they are independent. Within a
  // depth, a supernode costing more than a thread's share of the depth runs alone on
  // parallel kernels; the others run one per thread, largest first. The schedule changes
  // no arithmetic.
  vector<int> depth(ns, 0);
  int nd = 0;
  for (int s = ns - 1; s >= 0; --s) {  // parents come after their children
    const vector<int>& R = F.sn_rows[s];
    depth[s] = R.empty() ? 0 : depth[F.sn_of[R[0]]] + 1;
    nd = std::max(nd, depth[s] + 1);
  }
  vector<vector<int>> by_d(nd);
  for (int s = ns - 1; s >= 0; --s) by_d[depth[s]].push_back(s);
  auto cost = [&](int s) {
    const double nJ = 3.0 * (F.sn_first[s + 1] - F.sn_first[s]), nR = 3.0 * F.sn_rows[s].size();
    return nR * nR * (nJ + 4.0) + nJ * nJ * (nJ + nR);
  };
  for (int d = 0; d < nd; ++d) {
    vector<int> lv = by_d[d];
    std::stable_sort(lv.begin(), lv.end(), [&](int a, int b2) { return cost(a) > cost(b2); });
    double total = 0.0;
    for (int q : lv) total += cost(q);
    int nbig = 0;  // the leading supernodes above a thread's share
    while (nbig < (int)lv.size() && cost(lv[nbig]) > total / nthr) ++nbig;
    for (int q = 0; q < nbig; ++q) sel(lv[q], bufs[0]);
    const int rest = (int)lv.size() - nbig;
    if (rest >= 2 && nthr > 1 && !omp_in_parallel()) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthr)
      for (int q = nbig; q < (int)lv.size(); ++q) sel(lv[q], bufs[omp_get_thread_num()]);
    } else {
      for (int q = nbig; q < (int)lv.size(); ++q) sel(lv[q], bufs[0]);
    }
  }
}

// ------------------------------------------------------------------ per-body precompute

struct BodyResult {
  // per body-local free vertex: n_cub slots
  vector<int> elem_local;  // body-local element index or -1
  vector<double> w, u, resid;
};

static void inv3(const double* A, double* Ai) {
  const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
  const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  Ai[0] = c00 / det;
  Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  Ai[3] = c01 / det;
  Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  Ai[6] = c02 / det;
  Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

static jgs2_status body_precompute(const Mesh& M, const vector<int>& bverts, const vector<int>& belems,
                                   const jgs2_precompute_opts& o, BodyResult& out, std::string& err) {
  const int nvb = (int)bverts.size();
  // body-local vertex ids, free numbering
  std::map<int, int> lidx;
  for (int q = 0; q < nvb; ++q) lidx[bverts[q]] = q;
  vector<int> fid(nvb, -1), fverts;
  for (int q = 0; q < nvb; ++q)
    if (!M.pinned[bverts[q]]) {
      fid[q] = (int)fverts.size();
      fverts.push_back(q);
    }
  const int nf = (int)fverts.size();
  const int nc = o.n_cub;
  double t_phase = now_s();
  out.elem_local.assign((size_t)nvb * nc, -1);
  out.w.assign((size_t)nvb * nc, 0.0);
  out.u.assign((size_t)nvb * nc * 36, 0.0);
  out.resid.assign(nvb, std::nan(""));
  if (nf == 0) return JGS2_OK;
  const double ih2 = 1.0 / (M.h * M.h);
  // adjacency among free vertices and coordinates
  vector<vector<int>> adj(nf);
  vector<double> P((size_t)3 * nf);
  for (int a = 0; a < nf; ++a)
    for (int q = 0; q < 3; ++q) P[3 * a + q] = M.X[3 * bverts[fverts[a]] + q];
  vector<int> tl((size_t)4 * belems.size());
  for (size_t e = 0; e < belems.size(); ++e)
    for (int a = 0; a < 4; ++a) tl[4 * e + a] = lidx[M.tets_c[4 * (size_t)belems[e] + a]];
  for (size_t e = 0; e < belems.size(); ++e)
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c) {
        const int fa = fid[tl[4 * e + a]], fc = fid[tl[4 * e + c]];
        if (a != c && fa >= 0 && fc >= 0) adj[fa].push_back(fc);
      }
  for (auto& a : adj) {
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  // nested dissection order: ord[k] = free index of the k-th vertex in factor order
  vector<int> ord, idx(nf);
  std::iota(idx.begin(), idx.end(), 0);
  vector<char> side(nf, 0);
  nd_order(P, adj, idx, side, ord);
  vector<int> pos(nf);
  for (int k = 0; k < nf; ++k) pos[ord[k]] = k;
  // rest Hessian, lower block columns in factor order
  vector<BlockCol> H(nf);
  {
    vector<std::map<int, std::array<double, 9>>> cols(nf);
    for (size_t e = 0; e < belems.size(); ++e) {
      const int t = belems[e];
      const double* B = &M.B[9 * (size_t)t];
      double b[4][3];
      for (int j = 0; j < 3; ++j) {
        b[0][j] = -(B[j] + B[3 + j] + B[6 + j]);
        for (int k = 1; k < 4; ++k) b[k][j] = B[3 * (k - 1) + j];
      }
      const double V = M.vol[t], mu = M.mu[t], lam = M.lp[t] - M.mu[t];
      const double mq = M.rho[t] * V / 4.0 * ih2;
      for (int a = 0; a < 4; ++a) {
        const int fa = fid[tl[4 * e + a]];
        if (fa < 0) continue;
        for (int c = 0; c < 4; ++c) {
          const int fc = fid[tl[4 * e + c]];
          if (fc < 0) continue;
          const int ra = pos[fa], cc = pos[fc];
          if (ra < cc) continue;  // lower: row >= column
          const double bb = b[a][0] * b[c][0] + b[a][1] * b[c][1] + b[a][2] * b[c][2];
          auto& blk = cols[cc][ra];
          for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k)
              blk[3 * i + k] += V * ((i == k ? mu * bb : 0.0) + mu * b[c][i] * b[a][k] + lam * b[a][i] * b[c][k]) +
                                (a == c && i == k ? mq : 0.0);
        }
      }
    }
    for (int c = 0; c < nf; ++c) {
      for (auto& kv : cols[c]) {
        H[c].row.push_back(kv.first);
        H[c].val.insert(H[c].val.end(), kv.second.begin(), kv.second.end());
      }
    }
  }
  PHASE("order+assemble");
  Factor F;
  if (!factorize(nf, H, F)) {
    err = "rest Hessian is not positive definite";
    return JGS2_EINVAL;
  }
  const int n = 3 * nf;
  if (verbose()) {
    size_t nnz = 0;
    for (const auto& l : F.L) nnz += l.size();
    std::fprintf(stderr, "[jgs2_precompute] nf %d supernodes %d L entries %.3e\n", nf, F.nsn(), (double)nnz);
  }
  PHASE("factorize");
  // multi-RHS solves H_bar X = B: on the GPU (FP32 substitutions, FP64 refinement) when
  // asked, else the host's FP64 substitutions
  struct SolverGuard {
    GpuSolver* s = nullptr;
    ~SolverGuard() { gpu_solver_destroy(s); }
  } gsv;
  if (o.gpu) {
    gsv.s = gpu_solver_create(F, H, err);
    if (!gsv.s) return JGS2_ECUDA;
    PHASE("gpu upload");
  }
  // A body whose FP32-substitution refinement stalls above 1e-10 (kappa(H_bar) too large for
  // FP32) takes the host's FP64 substitutions from then on.
  bool use_gpu = gsv.s != nullptr;
  auto to_host = [&](const std::string& why) {
    if (verbose()) std::fprintf(stderr, "[jgs2_precompute] gpu solves stopped (%s); host solves\n", why.c_str());
    use_gpu = false;
  };
  auto solve = [&](vector<double>& B, int k) {
    if (!use_gpu) {
      solve_many(F, B, n, k);
      return;
    }
    vector<double> B0(B);  // the right-hand sides, for a host solve if the refinement stalls
    std::string e2;
    const int rounds = gpu_solve_many(gsv.s, B.data(), n, k, 1e-14, 1e-10, 40, e2);
    if (verbose()) std::fprintf(stderr, "[jgs2_precompute] gpu solve: %d columns, %d refinement rounds\n", k, rounds);
    if (rounds < 0) {
      to_host(e2);
      B.swap(B0);
      solve_many(F, B, n, k);
    }
  };
  // ---- training poses: lowest eigenpairs by block inverse iteration
  const int nt = std::min(o.n_train, n);
  const int p = std::min(n, nt + std::max(10, nt));
  vector<double> Q((size_t)n * p);  // row-major n x p (factor order)
  {
    SplitMix g = keyed(o.seed, 0xE16E0000ULL, 0);
    for (auto& q : Q) q = (double)(g.next() >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
  // full (both triangles) block rows of H_bar for the products H Q
  vector<vector<std::pair<int, const double*>>> Hrow(nf);
  for (int c = 0; c < nf; ++c)
    for (size_t q = 0; q < H[c].row.size(); ++q) {
      const int r = H[c].row[q];
      Hrow[r].push_back({c, &H[c].val[9 * q]});
      if (r != c) Hrow[c].push_back({-1 - r, &H[c].val[9 * q]});  // transposed block
    }
  auto Hmul = [&](const vector<double>& Xin, vector<double>& Yout, int k) {
    Yout.assign((size_t)n * k, 0.0);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < nf; ++r)
      for (const auto& e : Hrow[r]) {
        const bool tr = e.first < 0;
        const int c = tr ? -1 - e.first : e.first;
        for (int a = 0; a < 3; ++a) {
          double* yr = &Yout[(size_t)(3 * r + a) * k];
          for (int cc = 0; cc < 3; ++cc) {
            const double hv = tr ? e.second[3 * cc + a] : e.second[3 * a + cc];
            const double* xc = &Xin[(size_t)(3 * c + cc) * k];
            for (int j = 0; j < k; ++j) yr[j] += hv * xc[j];
          }
        }
      }
  };
  // column-major views: X (n x k, row-major) = X^T (k x n, column-major, ld k)
  auto orthonormalise = [&](vector<double>& X, int k) {
    // Cholesky QR twice: G = X^T X, X <- X R^{-1}
    for (int pass = 0; pass < 2; ++pass) {
      vector<double> G((size_t)k * k, 0.0);
      dense::gemm(false, true, k, k, n, 1.0, X.data(), k, X.data(), k, G.data(), k);
      for (int a = 0; a < k; ++a)
        for (int b2 = a + 1; b2 < k; ++b2) G[a + (size_t)b2 * k] = G[b2 + (size_t)a * k];
      if (!dense::potrf(G.data(), k, k)) {
        // fall back to modified Gram-Schmidt (rank-deficient block)
        for (int j = 0; j < k; ++j) {
          for (int q = 0; q < j; ++q) {
            double d = 0.0;
            for (int i = 0; i < n; ++i) d += X[(size_t)i * k + q] * X[(size_t)i * k + j];
            for (int i = 0; i < n; ++i) X[(size_t)i * k + j] -= d * X[(size_t)i * k + q];
          }
          double nr = 0.0;
          for (int i = 0; i < n; ++i) nr += X[(size_t)i * k + j] * X[(size_t)i * k + j];
          nr = std::sqrt(std::max(nr, 1e-300));
          for (int i = 0; i < n; ++i) X[(size_t)i * k + j] /= nr;
        }
        continue;
      }
      // X^T (k x n col-major) <- R^{-T} X^T with R = G^T: rows of X times R^{-1}
      // X (n x k row-major) = X_cm^T; X R^{-1} == (R^{-T} X^T)^T: solve per row
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) {
        double* xi = &X[(size_t)i * k];
        for (int j = 0; j < k; ++j) {
          double v = xi[j];
          for (int q = 0; q < j; ++q) v -= xi[q] * G[j + (size_t)q * k];
          xi[j] = v / G[j + (size_t)j * k];
        }
      }
    }
  };
  vector<double> lam(p, 0.0);
  // the same iteration with the block resident on the device (the p x p Gram, Cholesky and
  // Ritz problems on the host); falls back to the host loop if a Gram matrix is singular
  bool eig_done = false;
  if (use_gpu && p <= 64) {
    std::string e2;
    if (!gpu_eig_begin(gsv.s, Q.data(), n, p, e2)) {
      err = e2;
      return JGS2_ECUDA;
    }
    vector<double> G((size_t)p * p), T((size_t)p * p), w, Vv, Vs((size_t)p * p), rr(nt);
    bool ok = true;
    for (int it = 0; it < 80 && ok; ++it) {
      const int rounds = gpu_eig_solve(gsv.s, 1e-14, 1e-10, 40, e2);
      if (rounds < 0) {  // the block is still the one before this solve
        to_host(e2);
        ok = false;
        break;
      }
      for (int pass = 0; pass < 2 && ok; ++pass) {  // Cholesky QR twice
        if (!gpu_eig_gram(gsv.s, false, G.data(), e2)) {
          err = e2;
          return JGS2_ECUDA;
        }
        if (!dense::potrf(G.data(), p, p)) ok = false;
        else if (!gpu_eig_rowsolve(gsv.s, G.data(), e2)) {
          err = e2;
          return JGS2_ECUDA;
        }
      }
      if (!ok) break;
      if (!gpu_eig_hmul(gsv.s, e2) || !gpu_eig_gram(gsv.s, true, T.data(), e2)) {
        err = e2;
        return JGS2_ECUDA;
      }
      for (int a = 0; a < p; ++a)
        for (int b2 = a + 1; b2 < p; ++b2) T[(size_t)a * p + b2] = T[(size_t)b2 * p + a] = 0.5 * (T[(size_t)a * p + b2] + T[(size_t)b2 * p + a]);
      sym_eig(T, p, w, Vv);
      vector<int> o2(p);
      std::iota(o2.begin(), o2.end(), 0);
      std::sort(o2.begin(), o2.end(), [&](int a, int b2) { return w[a] < w[b2]; });
      for (int a = 0; a < p; ++a)
        for (int j = 0; j < p; ++j) Vs[(size_t)a * p + j] = Vv[(size_t)a * p + o2[j]];
      for (int j = 0; j < p; ++j) lam[j] = w[o2[j]];
      if (!gpu_eig_rotate(gsv.s, Vs.data(), e2) || !gpu_eig_residuals(gsv.s, lam.data(), nt, rr.data(), e2)) {
        err = e2;
        return JGS2_ECUDA;
      }
      double worst = 0.0;
      for (int j = 0; j < nt; ++j) worst = std::max(worst, std::sqrt(rr[j]) / std::fabs(lam[j]));
      if (verbose() && (it % 10 == 0)) std::fprintf(stderr, "[jgs2_precompute] eig it %d resid %.2e (gpu)\n", it, worst);
      if (worst < 1e-8) {
        eig_done = true;
        break;
      }
    }
    if (!gpu_eig_end(gsv.s, Q.data(), e2)) {
      err = e2;
      return JGS2_ECUDA;
    }
    if (ok) eig_done = true;  // the 80-iteration cap, as on the host
  }
  if (!eig_done) {
    vector<double> HQ;
    for (int it = 0; it < 80; ++it) {
      solve(Q, p);
      orthonormalise(Q, p);
      Hmul(Q, HQ, p);
      vector<double> T((size_t)p * p, 0.0), w, Vv;
      dense::gemm(false, true, p, p, n, 1.0, Q.data(), p, HQ.data(), p, T.data(), p);
      for (int a = 0; a < p; ++a)
        for (int b2 = a + 1; b2 < p; ++b2) T[(size_t)a * p + b2] = T[(size_t)b2 * p + a] = 0.5 * (T[(size_t)a * p + b2] + T[(size_t)b2 * p + a]);
      sym_eig(T, p, w, Vv);
      vector<int> o2(p);
      std::iota(o2.begin(), o2.end(), 0);
      std::sort(o2.begin(), o2.end(), [&](int a, int b2) { return w[a] < w[b2]; });
      vector<double> Vs((size_t)p * p);
      for (int a = 0; a < p; ++a)
        for (int j = 0; j < p; ++j) Vs[(size_t)a * p + j] = Vv[(size_t)a * p + o2[j]];
      for (int j = 0; j < p; ++j) lam[j] = w[o2[j]];
      // rotate Q and HQ by the Ritz vectors: row-major (n x p) times (p x p)
      vector<double> Qn((size_t)n * p, 0.0), HQn((size_t)n * p, 0.0);
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i)
        for (int a = 0; a < p; ++a) {
          const double qa = Q[(size_t)i * p + a], ha = HQ[(size_t)i * p + a];
          const double* va = &Vs[(size_t)a * p];
          double* qo = &Qn[(size_t)i * p];
          double* ho = &HQn[(size_t)i * p];
          for (int j = 0; j < p; ++j) {
            qo[j] += qa * va[j];
            ho[j] += ha * va[j];
          }
        }
      Q.swap(Qn);
      HQ.swap(HQn);
      double worst = 0.0;
      for (int j = 0; j < nt; ++j) {
        double rr = 0.0;
        for (int i = 0; i < n; ++i) {
          const double d = HQ[(size_t)i * p + j] - lam[j] * Q[(size_t)i * p + j];
          rr += d * d;
        }
        worst = std::max(worst, std::sqrt(rr) / std::fabs(lam[j]));
      }
      if (verbose() && (it % 10 == 0)) std::fprintf(stderr, "[jgs2_precompute] eig it %d resid %.2e\n", it, worst);
      if (worst < 1e-8) break;
    }
  }
  PHASE("eigen");
  // ---- cubature pool (body-local element indices) and its free vertices
  const int ne = (int)belems.size();
  vector<int> all(ne);
  std::iota(all.begin(), all.end(), 0);
  vector<int> pool = draw(keyed(o.seed, 0xFFFFFFFFULL, 0), all, o.n_pool);
  std::sort(pool.begin(), pool.end());
  vector<int> pv;  // free index of pool vertices
  for (int e : pool)
    for (int a = 0; a < 4; ++a) {
      const int fa = fid[tl[4 * e + a]];
      if (fa >= 0) pv.push_back(fa);
    }
  std::sort(pv.begin(), pv.end());
  pv.erase(std::unique(pv.begin(), pv.end()), pv.end());
  vector<int> pv_slot(nf, -1);
  for (size_t q = 0; q < pv.size(); ++q) pv_slot[pv[q]] = (int)q;
  const int np = (int)pv.size();
  if (o.gs) {
    // ---- Gauss-Seidel groups (Sec. 8.1): greedy colouring of the free vertices in caller
    // order; each colour is one generalised sub-problem whose U_bar_i^G keeps the group's
    // other DOFs at zero: on C = the free vertices of the other colours,
    // U_bar_{i,a}^G = -sum_c (H_CC^{-1})_{a,c} H_{c,i} over the neighbours c of i in C.
    vector<int> colour(nf, -1);
    int ncol = 0;
    for (int f = 0; f < nf; ++f) {  // free index order = body-local (caller) order
      vector<char> used(nf + 1, 0);
      for (int c : adj[f])
        if (c < f && colour[c] >= 0) used[colour[c]] = 1;
      int k = 0;
      while (used[k]) ++k;
      colour[f] = k;
      ncol = std::max(ncol, k + 1);
    }
    // full 3x3 blocks H_{r,c} of the rest Hessian by free index (both triangles)
    auto Hblock = [&](int r, int c, double* out9) {
      const bool lower = pos[r] >= pos[c];
      const BlockCol& col = H[lower ? pos[c] : pos[r]];
      const int row = lower ? pos[r] : pos[c];
      const auto it = std::lower_bound(col.row.begin(), col.row.end(), row);
      if (it == col.row.end() || *it != row) {
        std::fill(out9, out9 + 9, 0.0);
        return;
      }
      const double* b = &col.val[9 * (size_t)(it - col.row.begin())];
      for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) out9[3 * a + k] = lower ? b[3 * a + k] : b[3 * k + a];
    };
    // training poses in free-index order
    vector<double> qf((size_t)nt * n);
    for (int j = 0; j < nt; ++j)
      for (int f = 0; f < nf; ++f)
        for (int a = 0; a < 3; ++a) qf[(size_t)j * n + 3 * f + a] = Q[(size_t)(3 * pos[f] + a) * p + j];
    vector<vector<int>> inc(nvb);
    for (int e = 0; e < ne; ++e)
      for (int a = 0; a < 4; ++a) inc[tl[4 * e + a]].push_back(e);
    for (int g = 0; g < ncol; ++g) {
      // H_CC in the body's factor order restricted to C
      vector<int> cidx(nf, -1), corder;
      for (int k = 0; k < nf; ++k)
        if (colour[ord[k]] != g) {
          cidx[ord[k]] = (int)corder.size();
          corder.push_back(ord[k]);
        }
      const int nC = (int)corder.size(), n3 = 3 * nC;
      vector<int> G;
      for (int f = 0; f < nf; ++f)
        if (colour[f] == g) G.push_back(f);
      vector<double> Z, GC;  // Z: H_CC^{-1} q_C (n3 x nt); GC: H_CC^{-1} at pool columns
      vector<int> cslot(np, -1);
      int npc = 0;
      if (nC > 0) {
        vector<BlockCol> Hc(nC);
        for (int kc = 0; kc < nC; ++kc) {
          const BlockCol& col = H[pos[corder[kc]]];
          for (size_t q = 0; q < col.row.size(); ++q) {
            const int rf = ord[col.row[q]];
            if (cidx[rf] < 0) continue;
            Hc[kc].row.push_back(cidx[rf]);
            Hc[kc].val.insert(Hc[kc].val.end(), col.val.begin() + 9 * q, col.val.begin() + 9 * q + 9);
          }
        }
        Factor Fc;
        if (!factorize(nC, Hc, Fc)) {
          err = "rest Hessian restricted to a colour's complement is not positive definite";
          return JGS2_EINVAL;
        }
        Z.assign((size_t)n3 * nt, 0.0);
        for (int kc = 0; kc < nC; ++kc)
          for (int a = 0; a < 3; ++a)
            for (int t = 0; t < nt; ++t) Z[(size_t)(3 * kc + a) * nt + t] = qf[(size_t)t * n + 3 * corder[kc] + a];
        solve_many(Fc, Z, n3, nt);
        for (int q = 0; q < np; ++q)
          if (cidx[pv[q]] >= 0) cslot[q] = npc++;
        GC.assign((size_t)nC * npc * 9, 0.0);  // [kc][slot] 3x3: (H_CC^{-1})_{c, pool vertex}
        const int batch = 384;
        vector<int> pcols;
        for (int q = 0; q < np; ++q)
          if (cslot[q] >= 0) pcols.push_back(q);
        for (int q0 = 0; q0 < 3 * npc; q0 += batch) {
          const int k = std::min(batch, 3 * npc - q0);
          vector<double> Bm((size_t)n3 * k, 0.0);
          for (int j = 0; j < k; ++j) {
            const int col = q0 + j;
            Bm[(size_t)(3 * cidx[pv[pcols[col / 3]]] + col % 3) * k + j] = 1.0;
          }
          solve_many(Fc, Bm, n3, k);
          for (int kc = 0; kc < nC; ++kc)
            for (int j = 0; j < k; ++j) {
              const int col = q0 + j, sl = col / 3, c = col % 3;
              for (int a = 0; a < 3; ++a) GC[((size_t)kc * npc + sl) * 9 + 3 * a + c] = Bm[(size_t)(3 * kc + a) * k + j];
            }
        }
      }
#pragma omp parallel for schedule(dynamic, 8)
      for (int gi = 0; gi < (int)G.size(); ++gi) {
        const int f = G[gi], lv = fverts[f];
        // neighbours of i in C with H_{c,i}
        vector<int> nb_c;
        vector<double> Hci;
        for (int c : adj[f])
          if (cidx[c] >= 0) {
            double b9[9];
            Hblock(c, f, b9);
            nb_c.push_back(c);
            Hci.insert(Hci.end(), b9, b9 + 9);
          }
        // target b_t = lam_t (U_bar_i^T q_t - q_ti) = -lam_t sum_c H_{i,c} (H_CC^{-1} q_t)_c
        vector<double> bt((size_t)3 * nt, 0.0), nbv(nt);
        double nbmax = 0.0;
        for (int t = 0; t < nt; ++t) {
          for (size_t m2 = 0; m2 < nb_c.size(); ++m2) {
            const double* hb = &Hci[9 * m2];  // H_{c,i}: rows c, cols i; H_{i,c} = hb^T
            const double* z = &Z[(size_t)(3 * cidx[nb_c[m2]]) * nt + t];
            for (int a = 0; a < 3; ++a)
              bt[3 * t + a] -= lam[t] * (hb[a] * z[0] + hb[3 + a] * z[(size_t)nt] + hb[6 + a] * z[(size_t)2 * nt]);
          }
          nbv[t] = std::sqrt(bt[3 * t] * bt[3 * t] + bt[3 * t + 1] * bt[3 * t + 1] + bt[3 * t + 2] * bt[3 * t + 2]);
          nbmax = std::max(nbmax, nbv[t]);
        }
        // U_bar_{i,a}^G for a free vertex a (zero inside the group)
        auto ubar_block = [&](int fa, double* U) {
          std::fill(U, U + 9, 0.0);
          if (cidx[fa] < 0) return;
          const int sl = cslot[pv_slot[fa]];
          for (size_t m2 = 0; m2 < nb_c.size(); ++m2) {
            const double* gq = &GC[((size_t)cidx[nb_c[m2]] * npc + sl) * 9];  // (H_CC^{-1})_{c,a}
            const double* hb = &Hci[9 * m2];
            // U_{a,i} -= (H_CC^{-1})_{a,c} H_{c,i} = gq^T hb
            for (int r = 0; r < 3; ++r)
              for (int c = 0; c < 3; ++c)
                U[3 * r + c] -= gq[r] * hb[c] + gq[3 + r] * hb[3 + c] + gq[6 + r] * hb[6 + c];
          }
        };
        vector<int> keep;
        for (int t = 0; t < nt; ++t)
          if (nbv[t] > 1e-12 * std::max(nbmax, 1e-300)) keep.push_back(t);
        const int mrows = 3 * (int)keep.size();
        vector<double> y(mrows);
        for (size_t r = 0; r < keep.size(); ++r)
          for (int a = 0; a < 3; ++a) y[3 * r + a] = bt[3 * keep[r] + a] / nbv[keep[r]];
        double ynorm = 0.0;
        for (double v : y) ynorm += v * v;
        ynorm = std::sqrt(ynorm);
        auto column = [&](int e, double* col) {
          for (int r = 0; r < mrows; ++r) col[r] = 0.0;
          for (int a = 0; a < 4; ++a) {
            const int fa = fid[tl[4 * e + a]];
            if (fa < 0) continue;
            double U[9];
            ubar_block(fa, U);
            for (size_t r = 0; r < keep.size(); ++r) {
              const int t = keep[r];
              const double* qa = &qf[(size_t)t * n + 3 * fa];
              for (int c = 0; c < 3; ++c)
                col[3 * r + c] += lam[t] * (U[c] * qa[0] + U[3 + c] * qa[1] + U[6 + c] * qa[2]) / nbv[t];
            }
          }
        };
        vector<int> sel;
        vector<double> w_sel, Acols;
        double res = 1.0;
        for (int r = 0; r < nc && mrows > 0; ++r) {
          if (res < o.nnls_tol) break;
          vector<int> elig;
          for (int e : pool) {
            if (std::find(sel.begin(), sel.end(), e) != sel.end()) continue;
            if (std::find(inc[lv].begin(), inc[lv].end(), e) != inc[lv].end()) continue;
            elig.push_back(e);
          }
          vector<int> cands = draw(keyed(o.seed, (uint64_t)lv, (uint64_t)r), elig, o.n_cand);
          double best = 0.0;
          int best_e = -1;
          vector<double> best_w;
          const int k = (int)sel.size() + 1;
          vector<double> Am((size_t)mrows * k);
          std::copy(Acols.begin(), Acols.end(), Am.begin());
          for (int c : cands) {
            column(c, &Am[(size_t)(k - 1) * mrows]);
            vector<double> wc;
            const double rn = nnls(Am, mrows, k, y, wc) / ynorm;
            if (best_e < 0 || rn < best || (rn == best && c < best_e)) {
              best = rn;
              best_e = c;
              best_w = wc;
            }
          }
          if (best_e < 0) break;
          sel.push_back(best_e);
          w_sel = best_w;
          res = best;
          Acols.resize((size_t)mrows * k);
          column(best_e, &Acols[(size_t)(k - 1) * mrows]);
        }
        out.resid[lv] = res;
        for (size_t s2 = 0; s2 < sel.size(); ++s2) {
          const int e = sel[s2];
          out.elem_local[(size_t)lv * nc + s2] = e;
          out.w[(size_t)lv * nc + s2] = w_sel[s2];
          for (int a = 0; a < 4; ++a) {
            const int fa = fid[tl[4 * e + a]];
            if (fa < 0) continue;
            double U[9];
            ubar_block(fa, U);
            for (int q = 0; q < 9; ++q) out.u[((size_t)lv * nc + s2) * 36 + 9 * a + q] = U[q];
          }
        }
      }
    }
    PHASE("gs groups");
    return JGS2_OK;
  }
  // rows of H^{-1} at the pool vertices: G[f][q] = (H^{-1})_{f, pv[q]} (3x3), f free index
  // FP64 when it fits in 2 GB, else FP32 (rows of H^-1 only shape the cubature)
  const bool g64 = (size_t)nf * np * 9 <= ((size_t)1 << 28);
  vector<double> G64(g64 ? (size_t)nf * np * 9 : 0);
  vector<float> G32(g64 ? 0 : (size_t)nf * np * 9);
  auto Gat = [&](size_t q) -> double { return g64 ? G64[q] : (double)G32[q]; };
  {
    const int batch = use_gpu ? 768 : 384;  // RHS per batch (multiple of 3)
    for (int q0 = 0; q0 < 3 * np; q0 += batch) {
      const int k = std::min(batch, 3 * np - q0);
      vector<double> Bm((size_t)n * k, 0.0);
      for (int j = 0; j < k; ++j) {
        const int col = q0 + j;
        const int v = pv[col / 3];
        Bm[(size_t)(3 * pos[v] + col % 3) * k + j] = 1.0;
      }
      solve(Bm, k);
      for (int f = 0; f < nf; ++f)
        for (int j = 0; j < k; ++j) {
          const int col = q0 + j, q = col / 3, c = col % 3;
          for (int a = 0; a < 3; ++a)
          {
            const double val = Bm[(size_t)(3 * pos[f] + a) * k + j];
            const size_t gi = ((size_t)f * np + q) * 9 + 3 * a + c;
            if (g64)
              G64[gi] = val;
            else
              G32[gi] = (float)val;
          }
        }
    }
  }
  PHASE("pool solves");
  // eigenvectors in free-index order (nt columns)
  vector<double> q_free((size_t)nt * n);
  for (int j = 0; j < nt; ++j)
    for (int f = 0; f < nf; ++f)
      for (int a = 0; a < 3; ++a) q_free[(size_t)j * n + 3 * f + a] = Q[(size_t)(3 * pos[f] + a) * p + j];
  Q.clear();
  Q.shrink_to_fit();
  // ---- diagonal blocks of H^{-1} (consumes the factor)
  vector<double> Adiag;
  selected_inverse_diag(F, Adiag);
  F.L.clear();
  PHASE("selected inverse");
  // incident elements per body-local vertex (for eligibility)
  vector<vector<int>> inc(nvb);
  for (int e = 0; e < ne; ++e)
    for (int a = 0; a < 4; ++a) inc[tl[4 * e + a]].push_back(e);
  // ---- greedy NNLS per free vertex
#pragma omp parallel for schedule(dynamic, 16)
  for (int f = 0; f < nf; ++f) {
    const int lv = fverts[f];  // body-local vertex index
    double A[9], Ai[9];
    for (int q = 0; q < 9; ++q) A[q] = Adiag[(size_t)pos[f] * 9 + q];
    inv3(A, Ai);
    // target rows b^(t) = A^{-1} q_ti - lam_t q_ti, kept if |b| > 1e-12 max|b|
    vector<double> bt((size_t)3 * nt), nb(nt);
    double nbmax = 0.0;
    for (int t = 0; t < nt; ++t) {
      const double* qi = &q_free[(size_t)t * n + 3 * f];
      for (int a = 0; a < 3; ++a) bt[3 * t + a] = Ai[3 * a] * qi[0] + Ai[3 * a + 1] * qi[1] + Ai[3 * a + 2] * qi[2] - lam[t] * qi[a];
      nb[t] = std::sqrt(bt[3 * t] * bt[3 * t] + bt[3 * t + 1] * bt[3 * t + 1] + bt[3 * t + 2] * bt[3 * t + 2]);
      nbmax = std::max(nbmax, nb[t]);
    }
    vector<int> keep;
    for (int t = 0; t < nt; ++t)
      if (nb[t] > 1e-12 * std::max(nbmax, 1e-300)) keep.push_back(t);
    const int mrows = 3 * (int)keep.size();
    vector<double> y(mrows);
    for (size_t r = 0; r < keep.size(); ++r)
      for (int a = 0; a < 3; ++a) y[3 * r + a] = bt[3 * keep[r] + a] / nb[keep[r]];
    double ynorm = 0.0;
    for (double v : y) ynorm += v * v;
    ynorm = std::sqrt(ynorm);
    // U_bar_{i,a} = (H^-1)_{a,i} A_i^{-1} = G[f][a]^T A_i^{-1}
    auto ubar_block = [&](int fa, double* U) {
      const size_t g0 = ((size_t)f * np + pv_slot[fa]) * 9;
      double g[9];
      for (int q = 0; q < 9; ++q) g[q] = Gat(g0 + q);
      // g = (H^-1)_{i,a}; U = g^T A_i^{-1}
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) U[3 * r + c] = g[0 * 3 + r] * Ai[c] + g[1 * 3 + r] * Ai[3 + c] + g[2 * 3 + r] * Ai[6 + c];
    };
    auto column = [&](int e, double* col) {
      for (int r = 0; r < mrows; ++r) col[r] = 0.0;
      for (int a = 0; a < 4; ++a) {
        const int fa = fid[tl[4 * e + a]];
        if (fa < 0) continue;
        double U[9];
        ubar_block(fa, U);
        for (size_t r = 0; r < keep.size(); ++r) {
          const int t = keep[r];
          const double* qa = &q_free[(size_t)t * n + 3 * fa];
          for (int c = 0; c < 3; ++c)
            col[3 * r + c] += lam[t] * (U[c] * qa[0] + U[3 + c] * qa[1] + U[6 + c] * qa[2]) / nb[t];
        }
      }
    };
    vector<int> sel;
    vector<double> w_sel;
    double res = 1.0;
    vector<double> Acols;
    for (int r = 0; r < nc; ++r) {
      if (res < o.nnls_tol) break;
      vector<int> elig;
      for (int e : pool) {
        if (std::find(sel.begin(), sel.end(), e) != sel.end()) continue;
        if (std::find(inc[lv].begin(), inc[lv].end(), e) != inc[lv].end()) continue;
        elig.push_back(e);
      }
      vector<int> cands = draw(keyed(o.seed, (uint64_t)lv, (uint64_t)r), elig, o.n_cand);
      double best = 0.0;
      int best_e = -1;
      vector<double> best_w;
      const int k = (int)sel.size() + 1;
      vector<double> Am((size_t)mrows * k);
      std::copy(Acols.begin(), Acols.end(), Am.begin());
      for (int c : cands) {
        column(c, &Am[(size_t)(k - 1) * mrows]);
        vector<double> wc;
        const double rn = nnls(Am, mrows, k, y, wc) / ynorm;
        if (best_e < 0 || rn < best || (rn == best && c < best_e)) {
          best = rn;
          best_e = c;
          best_w = wc;
        }
      }
      if (best_e < 0) break;
      sel.push_back(best_e);
      w_sel = best_w;
      res = best;
      Acols.resize((size_t)mrows * k);
      column(best_e, &Acols[(size_t)(k - 1) * mrows]);
    }
    out.resid[lv] = res;
    for (size_t s = 0; s < sel.size(); ++s) {
      const int e = sel[s];
      out.elem_local[(size_t)lv * nc + s] = e;
      out.w[(size_t)lv * nc + s] = w_sel[s];
      for (int a = 0; a < 4; ++a) {
        const int fa = fid[tl[4 * e + a]];
        if (fa < 0) continue;
        double U[9];
        ubar_block(fa, U);
        for (int q = 0; q < 9; ++q) out.u[((size_t)lv * nc + s) * 36 + 9 * a + q] = U[q];
      }
    }
  }
  PHASE("greedy nnls");
  return JGS2_OK;
}

// Bodies equal up to translation (same local connectivity, material and pins).
static bool same_body(const Mesh& M, const vector<int>& va, const vector<int>& ea, const vector<int>& vb,
                      const vector<int>& eb) {
  if (va.size() != vb.size() || ea.size() != eb.size()) return false;
  double ext = 0.0;
  for (size_t q = 0; q < va.size(); ++q)
    for (int c = 0; c < 3; ++c) ext = std::max(ext, std::fabs(M.X[3 * va[q] + c] - M.X[3 * va[0] + c]));
  for (size_t q = 0; q < va.size(); ++q) {
    if (M.pinned[va[q]] != M.pinned[vb[q]]) return false;
    for (int c = 0; c < 3; ++c) {
      const double da = M.X[3 * va[q] + c] - M.X[3 * va[0] + c];
      const double db = M.X[3 * vb[q] + c] - M.X[3 * vb[0] + c];
      if (std::fabs(da - db) > 1e-9 * std::max(ext, 1e-300)) return false;
    }
  }
  for (size_t e = 0; e < ea.size(); ++e) {
    const int ta = ea[e], tb = eb[e];
    if (M.E[ta] != M.E[tb] || M.nu[ta] != M.nu[tb] || M.rho[ta] != M.rho[tb]) return false;
    for (int a = 0; a < 4; ++a)
      if (M.tets_c[4 * (size_t)ta + a] - va[0] != M.tets_c[4 * (size_t)tb + a] - vb[0]) return false;
  }
  return true;
}

}  // namespace pre

jgs2_status precompute(Mesh* m, const jgs2_precompute_opts* o) {
  using namespace pre;
  if (!m || !o) return fail(JGS2_EINVAL, "null argument");
  if (o->n_cub < 1 || o->n_cub > kMaxCub || o->n_train < 1 || o->n_cand < 1 || o->n_pool < 1 ||
      !(o->nnls_tol >= 0.0) || (o->gpu != 0 && o->gpu != 1))
    return fail(JGS2_EINVAL, "precompute options out of range");
  const int saved = omp_get_max_threads();
  if (o->n_threads > 0) omp_set_num_threads(o->n_threads);
  const int nb = m->n_bodies;
  vector<vector<int>> bv(nb), be(nb);
  for (int v = 0; v < m->V; ++v) bv[m->body[v]].push_back(v);
  for (int t = 0; t < m->T; ++t) be[m->body[m->tets_c[4 * (size_t)t]]].push_back(t);
  vector<int> rep(nb, -1);
  vector<BodyResult> res(nb);
  vector<int> todo;  // one body of each distinct shape
  for (int b = 0; b < nb; ++b) {
    for (int c = 0; c < b; ++c)
      if (rep[c] == c && same_body(*m, bv[c], be[c], bv[b], be[b])) {
        rep[b] = c;
        break;
      }
    if (rep[b] < 0) {
      rep[b] = b;
      todo.push_back(b);
    }
  }
  vector<jgs2_status> bst(nb, JGS2_OK);
  vector<std::string> berr(nb);
  // Bodies below kSmallBody vertices, when there are several, run side by side on the host,
  // one thread each, largest first: their own tree passes are too small to keep the threads
  // busy, and their GPU solves too short to hide the level schedule's launch latency. Larger
  // bodies (and a lone small one) then run one at a time on all threads, with GPU solves if
  // asked for.
  constexpr size_t kSmallBody = 20000;
  vector<int> small, large;
  for (int b : todo) (bv[b].size() < kSmallBody && omp_get_max_threads() > 1 ? small : large).push_back(b);
  if (small.size() < 2) {  // a lone small body runs on all threads
    large.insert(large.begin(), small.begin(), small.end());
    small.clear();
  }
  std::stable_sort(small.begin(), small.end(), [&](int a, int b2) { return bv[a].size() > bv[b2].size(); });
  if (!small.empty()) {
    jgs2_precompute_opts oh = *o;
    oh.gpu = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < (int)small.size(); ++q) {
      omp_set_num_threads(1);  // nested regions of this body run on its own thread
      const int b = small[q];
      bst[b] = body_precompute(*m, bv[b], be[b], oh, res[b], berr[b]);
    }
  }
  for (int b : large) {
    bst[b] = body_precompute(*m, bv[b], be[b], *o, res[b], berr[b]);
    if (bst[b] != JGS2_OK) break;
  }
  omp_set_num_threads(saved);
  for (int b : todo)  // the first failure in body order
    if (bst[b] != JGS2_OK) return fail(bst[b], "jgs2_precompute: " + berr[b]);
  const int nc = o->n_cub;
  const size_t Vf = m->Vf;
  vector<int> e_int(Vf * nc, -1);
  vector<double> w(Vf * nc, 0.0), u(Vf * nc * 36, 0.0);
  m->cub_resid.assign(m->V, std::nan(""));
  for (int b = 0; b < nb; ++b) {
    const BodyResult& r = res[rep[b]];
    for (size_t q = 0; q < bv[b].size(); ++q) {
      const int c = bv[b][q];
      m->cub_resid[c] = r.resid[q];
      const int i = m->iperm[c];
      if (i >= m->Vf) continue;
      for (int s = 0; s < nc; ++s) {
        const int el = r.elem_local[q * nc + s];
        if (el < 0) continue;
        e_int[(size_t)i * nc + s] = m->tiperm[be[b][el]];
        w[(size_t)i * nc + s] = r.w[q * nc + s];
        for (int k = 0; k < 36; ++k) u[((size_t)i * nc + s) * 36 + k] = r.u[(q * nc + s) * 36 + k];
      }
    }
  }
  return set_cubature(m, nc, e_int, w, u);
}

}  // namespace jgs2

extern "C" jgs2_status jgs2_precompute(jgs2_mesh* mesh, const jgs2_precompute_opts* opts) {
  return jgs2::precompute(reinterpret_cast<jgs2::Mesh*>(mesh), opts);
}
