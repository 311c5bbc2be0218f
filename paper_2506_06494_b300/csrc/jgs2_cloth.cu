// Cloth: StVK membrane triangles and quadratic bending on interior edges, stepped by the
// per-vertex Jacobi sweep with the global line search (the cloth material of the paper's
// Table 1 caption; readings R17 and R26; no cubature correction, whose Ubar records are
// built on tets only).
//
// Per step (FP64 setup): F(x_t) (3x2), its Green strain E(x_t) and each hinge's
// w(x_t) = sum K_j x_t,j are formed in FP64 and stored in the sweep precision, so FP32
// sweeps work on the displacement u = x - x_t without cancellation:
//   F = F_t + G, G = sum_a u_a b_a^T;  E = E_t + sym(F_t^T G) + G^T G / 2;  w = w_t + sum K_j u_j.
// Per sweep:
//   k_cloth_gather  thread per free vertex: g_v and H_vv over its incident triangles
//                   (membrane blocks summed, then their positive semidefinite part) and
//                   hinges, plus inertia; D_v = -H_vv^-1 g_v; block sums of |g|^2, g.D.
//   k_cloth_poly    E(x + a D) - E(x) as a quartic in a: tiles of triangles, hinges and
//                   vertices, float-float (FP64-class) per-thread sums, per-block partials.
//   k_cloth_decide  one block: fixed-order FP64 sums, residual test, Armijo choice over
//                   a = 2^-j, j < 8 (the first trial with dE <= 1e-4 a g.D).
//   k_cloth_update  u += a D.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <array>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/jgs2.h"
#include "jgs2_host.h"
#include "jgs2_kernels.cuh"

namespace jgs2 {

namespace {

constexpr int kClothTrials = 8;

template <typename T>
struct alignas(16) TriRec {
  int32_t v[3];
  int32_t pad;
  T b[6];    // b_0, b_1, b_2 (2 each): F = sum_a x_a b_a^T
  T Ft[6];   // F(x_t), row-major 3x2 (per step)
  T Et[3];   // E(x_t): e00, e01, e11 (per step)
  T area, mu, lam;
};

template <typename T>
struct alignas(16) HingeRec {
  int32_t v[4];
  T K[4];
  T wt[3];   // sum K_j x_t,j (per step)
  T kb;
};

template <typename T>
struct ClothDev {
  int V, F, H;
  const TriRec<T>* tris;
  TriRec<T>* tris_mut;
  const HingeRec<T>* hinges;
  HingeRec<T>* hinges_mut;
  const int32_t* tri_off;    // [V + 1] incident (triangle, corner) entries, value 4 t + a
  const int32_t* tri_inc;
  const int32_t* hin_off;    // [V + 1] incident (hinge, slot) entries, value 4 e + i
  const int32_t* hin_inc;
  const uint8_t* pinned;     // [V]
  const T* mh2;              // [V] m / h^2 (0 pinned)
  Vec4<T>* u;                // [V] x - x_t
  Vec4<T>* dz;               // [V] h v_t + h^2 g
  Vec4<T>* D;                // [V]
  double* xt;                // [V][3]
  double h;
  double grav[3];
  // walls n.x >= c: IPC barrier kappa B(d) below dhat, step limit 0.45 min(rc - dhat, d_min)
  int n_planes;
  const double* planes;      // [n_planes][4]
  double dhat, kappa, rc;
};

struct ClothState {
  int32_t done, converged, k, sweeps, max_sweeps, ls_rejects;
  double rel_tol, g0, r, alpha;
};

// --- per-step setup (FP64)

template <typename T>
__global__ void k_cloth_setup_vertices(ClothDev<T> m, const double* __restrict__ x, const double* __restrict__ v,
                                       const double* __restrict__ xk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.V) return;
  const bool pin = m.pinned[i] != 0;
  Vec4<T> u{T(0), T(0), T(0), T(0)}, d{T(0), T(0), T(0), T(0)};
  for (int q = 0; q < 3; ++q) m.xt[3 * i + q] = x[3 * i + q];
  if (!pin) {
    if (xk) {
      u.x = T(xk[3 * i] - x[3 * i]);
      u.y = T(xk[3 * i + 1] - x[3 * i + 1]);
      u.z = T(xk[3 * i + 2] - x[3 * i + 2]);
    }
    d.x = T(m.h * v[3 * i] + m.h * m.h * m.grav[0]);
    d.y = T(m.h * v[3 * i + 1] + m.h * m.h * m.grav[1]);
    d.z = T(m.h * v[3 * i + 2] + m.h * m.h * m.grav[2]);
  }
  m.u[i] = u;
  m.dz[i] = d;
  m.D[i] = Vec4<T>{T(0), T(0), T(0), T(0)};
}

template <typename T>
__global__ void k_cloth_setup_elements(ClothDev<T> m) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < m.F) {
    TriRec<T>& r = m.tris_mut[q];
    double F[6] = {0, 0, 0, 0, 0, 0};
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 2; ++j) F[2 * i + j] += m.xt[3 * r.v[a] + i] * double(r.b[2 * a + j]);
    const double c00 = F[0] * F[0] + F[2] * F[2] + F[4] * F[4];
    const double c01 = F[0] * F[1] + F[2] * F[3] + F[4] * F[5];
    const double c11 = F[1] * F[1] + F[3] * F[3] + F[5] * F[5];
    for (int k = 0; k < 6; ++k) r.Ft[k] = T(F[k]);
    r.Et[0] = T(0.5 * (c00 - 1.0));
    r.Et[1] = T(0.5 * c01);
    r.Et[2] = T(0.5 * (c11 - 1.0));
  }
  if (q < m.H) {
    HingeRec<T>& e = m.hinges_mut[q];
    for (int i = 0; i < 3; ++i) {
      double w = 0.0;
      for (int j = 0; j < 4; ++j) w += double(e.K[j]) * m.xt[3 * e.v[j] + i];
      e.wt[i] = T(w);
    }
  }
}

// --- element kinematics in the sweep precision

// G = sum_a u_a b_a^T, F = F_t + G, E = E_t + sym(F_t^T G) + G^T G / 2 (2x2 symmetric).
template <typename T>
__device__ __forceinline__ void tri_state(const TriRec<T>& r, const Vec4<T>* u, T (&F)[6], T (&E)[3]) {
  T G[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const Vec4<T> ua = u[r.v[a]];
    const T uu[3] = {ua.x, ua.y, ua.z};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      G[2 * i] += uu[i] * r.b[2 * a];
      G[2 * i + 1] += uu[i] * r.b[2 * a + 1];
    }
  }
  // F_t^T G (2x2) and G^T G
  T A00 = T(0), A01 = T(0), A10 = T(0), A11 = T(0), B00 = T(0), B01 = T(0), B11 = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    A00 += r.Ft[2 * i] * G[2 * i];
    A01 += r.Ft[2 * i] * G[2 * i + 1];
    A10 += r.Ft[2 * i + 1] * G[2 * i];
    A11 += r.Ft[2 * i + 1] * G[2 * i + 1];
    B00 += G[2 * i] * G[2 * i];
    B01 += G[2 * i] * G[2 * i + 1];
    B11 += G[2 * i + 1] * G[2 * i + 1];
  }
  E[0] = r.Et[0] + (A00 + T(0.5) * B00);
  E[1] = r.Et[1] + (T(0.5) * (A01 + A10) + T(0.5) * B01);
  E[2] = r.Et[2] + (A11 + T(0.5) * B11);
#pragma unroll
  for (int k = 0; k < 6; ++k) F[k] = r.Ft[k] + G[k];
}

// --- sweep kernels

template <typename T>
__global__ void __launch_bounds__(128) k_cloth_gather(ClothDev<T> m, const ClothState* __restrict__ st,
                                                      double* __restrict__ partial) {
  __shared__ Acc<T> sred[64];
  if (st->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  Acc<T> acc[2];
  if (i < m.V && !m.pinned[i]) {
    T g[3] = {T(0), T(0), T(0)}, Hm[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    for (int q = m.tri_off[i]; q < m.tri_off[i + 1]; ++q) {
      const int ent = m.tri_inc[q], t = ent >> 2, a = ent & 3;
      const TriRec<T>& r = m.tris[t];
      T F[6], E[3];
      tri_state(r, m.u, F, E);
      const T tr = E[0] + E[2];
      const T S00 = T(2) * r.mu * E[0] + r.lam * tr, S01 = T(2) * r.mu * E[1], S11 = T(2) * r.mu * E[2] + r.lam * tr;
      const T b0 = r.b[2 * a], b1 = r.b[2 * a + 1];
      const T Sb0 = S00 * b0 + S01 * b1, Sb1 = S01 * b0 + S11 * b1;
      const T bSb = b0 * Sb0 + b1 * Sb1, bb = b0 * b0 + b1 * b1;
      T Fb[3], FFt[6];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        g[k] += r.area * (F[2 * k] * Sb0 + F[2 * k + 1] * Sb1);
        Fb[k] = F[2 * k] * b0 + F[2 * k + 1] * b1;
      }
      FFt[0] = F[0] * F[0] + F[1] * F[1];
      FFt[1] = F[0] * F[2] + F[1] * F[3];
      FFt[2] = F[0] * F[4] + F[1] * F[5];
      FFt[3] = F[2] * F[2] + F[3] * F[3];
      FFt[4] = F[2] * F[4] + F[3] * F[5];
      FFt[5] = F[4] * F[4] + F[5] * F[5];
      const T ml = r.mu + r.lam, mb = r.mu * bb;
      const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int k = 0; k < 6; ++k)
        Hm[k] += r.area * ((ia[k] == ib[k] ? bSb : T(0)) + ml * Fb[ia[k]] * Fb[ib[k]] + mb * FFt[k]);
    }
    // positive semidefinite part of the summed membrane block (StVK's can be indefinite)
    {
      T A[6] = {Hm[0], Hm[1], Hm[2], Hm[3], Hm[4], Hm[5]}, Q[9];
      sym3_eig(A, Q);
      const T l[3] = {A[0] > T(0) ? A[0] : T(0), A[3] > T(0) ? A[3] : T(0), A[5] > T(0) ? A[5] : T(0)};
      const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int k = 0; k < 6; ++k)
        Hm[k] = Q[3 * ia[k]] * l[0] * Q[3 * ib[k]] + Q[3 * ia[k] + 1] * l[1] * Q[3 * ib[k] + 1] +
                Q[3 * ia[k] + 2] * l[2] * Q[3 * ib[k] + 2];
    }
    T hb = T(0);
    for (int q = m.hin_off[i]; q < m.hin_off[i + 1]; ++q) {
      const int ent = m.hin_inc[q], e = ent >> 2, s = ent & 3;
      const HingeRec<T>& h = m.hinges[e];
      T w[3] = {h.wt[0], h.wt[1], h.wt[2]};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const Vec4<T> uj = m.u[h.v[j]];
        w[0] += h.K[j] * uj.x;
        w[1] += h.K[j] * uj.y;
        w[2] += h.K[j] * uj.z;
      }
      const T ks = h.kb * h.K[s];
      g[0] += ks * w[0];
      g[1] += ks * w[1];
      g[2] += ks * w[2];
      hb += ks * h.K[s];
    }
    const Vec4<T> ui = m.u[i], dzi = m.dz[i];
    const T mh = m.mh2[i];
    g[0] += mh * (ui.x - dzi.x);
    g[1] += mh * (ui.y - dzi.y);
    g[2] += mh * (ui.z - dzi.z);
    T H[6] = {Hm[0] + hb + mh, Hm[1], Hm[2], Hm[3] + hb + mh, Hm[4], Hm[5] + hb + mh};
    T lim = T(INFINITY);
    if (m.n_planes > 0) {
      // walls: barrier gradient and Gauss-Newton block, and the step limit (FP64 distances)
      const double x[3] = {m.xt[3 * i] + double(ui.x), m.xt[3 * i + 1] + double(ui.y),
                           m.xt[3 * i + 2] + double(ui.z)};
      double dmin = INFINITY;
      for (int p = 0; p < m.n_planes; ++p) {
        const double* pl = m.planes + 4 * p;
        const double dd = pl[0] * x[0] + pl[1] * x[1] + pl[2] * x[2] - pl[3];
        if (dd < m.rc) dmin = fmin(dmin, dd);
        if (dd > 0.0 && dd < m.dhat) {
          const double b1 = m.kappa * barrier_b1(dd, m.dhat), b2 = m.kappa * barrier_b2(dd, m.dhat);
          const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
          for (int k = 0; k < 3; ++k) g[k] += T(b1 * pl[k]);
          for (int k = 0; k < 6; ++k) H[k] += T(b2 * pl[ia[k]] * pl[ib[k]]);
        }
      }
      lim = T(0.45 * fmin(m.rc - m.dhat, dmin));
    }
    T rhs[3] = {-g[0], -g[1], -g[2]}, d[3];
    if (!chol3_solve(H, rhs, d)) d[0] = d[1] = d[2] = T(0);
    truncate3(d, lim);
    m.D[i] = Vec4<T>{d[0], d[1], d[2], T(0)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc[0].add_prod(g[k], g[k]);
      acc[1].add_prod(g[k], d[k]);
    }
  }
  double bs[2];
  block_sum_acc<T, 2>(acc, bs, sred);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = bs[0];
    partial[gridDim.x + blockIdx.x] = bs[1];
  }
}

// E(x + a D) - E(x) = c1 a + c2 a^2 + c3 a^3 + c4 a^4: blocks [0, nbT) take triangles,
// [nbT, nbT + nbH) hinges, the rest vertices.
template <typename T>
__global__ void __launch_bounds__(128) k_cloth_poly(ClothDev<T> m, const ClothState* __restrict__ st, int nbT,
                                                    int nbH, double* __restrict__ partial) {
  __shared__ Acc<T> sred[128];
  if (st->done) return;
  Acc<T> acc[4];
  const int b = blockIdx.x;
  if (b < nbT) {
    const int t = b * 128 + threadIdx.x;
    if (t < m.F) {
      const TriRec<T>& r = m.tris[t];
      T F[6], E[3];
      tri_state(r, m.u, F, E);
      // G_D = sum_a D_a b_a^T; E(a) = E + a E1 + a^2 E2, E1 = sym(F^T G_D), E2 = G_D^T G_D / 2
      T GD[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const Vec4<T> da = m.D[r.v[a]];
        const T dd[3] = {da.x, da.y, da.z};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          GD[2 * i] += dd[i] * r.b[2 * a];
          GD[2 * i + 1] += dd[i] * r.b[2 * a + 1];
        }
      }
      T A00 = T(0), A01 = T(0), A10 = T(0), A11 = T(0), B00 = T(0), B01 = T(0), B11 = T(0);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        A00 += F[2 * i] * GD[2 * i];
        A01 += F[2 * i] * GD[2 * i + 1];
        A10 += F[2 * i + 1] * GD[2 * i];
        A11 += F[2 * i + 1] * GD[2 * i + 1];
        B00 += GD[2 * i] * GD[2 * i];
        B01 += GD[2 * i] * GD[2 * i + 1];
        B11 += GD[2 * i + 1] * GD[2 * i + 1];
      }
      const T E1[3] = {A00, T(0.5) * (A01 + A10), A11};
      const T E2[3] = {T(0.5) * B00, T(0.5) * B01, T(0.5) * B11};
      // tr(X Y) of 2x2 symmetric (x00 x01 x11)
      auto tr2 = [](const T (&X)[3], const T (&Y)[3]) { return X[0] * Y[0] + T(2) * X[1] * Y[1] + X[2] * Y[2]; };
      const T e0 = E[0] + E[2], e1 = E1[0] + E1[2], e2 = E2[0] + E2[2];
      const T mu = r.mu, hl = T(0.5) * r.lam, A = r.area;
      acc[0].add(A * (mu * T(2) * tr2(E, E1) + hl * T(2) * e0 * e1));
      acc[1].add(A * (mu * (tr2(E1, E1) + T(2) * tr2(E, E2)) + hl * (e1 * e1 + T(2) * e0 * e2)));
      acc[2].add(A * (mu * T(2) * tr2(E1, E2) + hl * T(2) * e1 * e2));
      acc[3].add(A * (mu * tr2(E2, E2) + hl * e2 * e2));
    }
  } else if (b < nbT + nbH) {
    const int e = (b - nbT) * 128 + threadIdx.x;
    if (e < m.H) {
      const HingeRec<T>& h = m.hinges[e];
      T w[3] = {h.wt[0], h.wt[1], h.wt[2]}, wd[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const Vec4<T> uj = m.u[h.v[j]], dj = m.D[h.v[j]];
        w[0] += h.K[j] * uj.x;
        w[1] += h.K[j] * uj.y;
        w[2] += h.K[j] * uj.z;
        wd[0] += h.K[j] * dj.x;
        wd[1] += h.K[j] * dj.y;
        wd[2] += h.K[j] * dj.z;
      }
      acc[0].add(h.kb * (w[0] * wd[0] + w[1] * wd[1] + w[2] * wd[2]));
      acc[1].add(T(0.5) * h.kb * (wd[0] * wd[0] + wd[1] * wd[1] + wd[2] * wd[2]));
    }
  } else {
    const int v = (b - nbT - nbH) * 128 + threadIdx.x;
    if (v < m.V && !m.pinned[v]) {
      const Vec4<T> uv = m.u[v], dz = m.dz[v], d = m.D[v];
      const T mh = m.mh2[v];
      acc[0].add(mh * (d.x * (uv.x - dz.x) + d.y * (uv.y - dz.y) + d.z * (uv.z - dz.z)));
      acc[1].add(T(0.5) * mh * (d.x * d.x + d.y * d.y + d.z * d.z));
    }
  }
  double bs[4];
  block_sum_acc<T, 4>(acc, bs, sred);
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) partial[(size_t)j * gridDim.x + blockIdx.x] = bs[j];
}

// Walls: kappa (B(d + a n.D) - B(d)) per trial a = 2^-j over every free vertex and wall,
// exact (the barrier is not a polynomial); per-block partials [kClothTrials][grid].
template <typename T>
__global__ void __launch_bounds__(128) k_cloth_wall_trials(ClothDev<T> m, const ClothState* __restrict__ st,
                                                           double* __restrict__ partial) {
  __shared__ double red[32 * kClothTrials];
  if (st->done) return;
  double acc[kClothTrials];
#pragma unroll
  for (int j = 0; j < kClothTrials; ++j) acc[j] = 0.0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m.V && !m.pinned[i]) {
    const Vec4<T> ui = m.u[i], di = m.D[i];
    const double x[3] = {m.xt[3 * i] + double(ui.x), m.xt[3 * i + 1] + double(ui.y), m.xt[3 * i + 2] + double(ui.z)};
    for (int p = 0; p < m.n_planes; ++p) {
      const double* pl = m.planes + 4 * p;
      const double d0 = pl[0] * x[0] + pl[1] * x[1] + pl[2] * x[2] - pl[3];
      const double dn = pl[0] * double(di.x) + pl[1] * double(di.y) + pl[2] * double(di.z);
      // the step limit keeps every trial of a vertex beyond r_c outside dhat
      if (!(d0 < m.rc)) continue;
      const double b0 = barrier_b(d0, m.dhat);
#pragma unroll
      for (int j = 0; j < kClothTrials; ++j) {
        const double a = 1.0 / double(1 << j);
        acc[j] += m.kappa * (barrier_b(d0 + a * dn, m.dhat) - b0);
      }
    }
  }
  block_sum<kClothTrials>(acc, red);
  if (threadIdx.x == 0)
    for (int j = 0; j < kClothTrials; ++j) partial[(size_t)j * gridDim.x + blockIdx.x] = acc[j];
}

// One block: fixed-order sums (thread-strided, then a shared-memory tree), residual test,
// Armijo choice; writes alpha (0 when the step stops or no trial passes).
__global__ void __launch_bounds__(256) k_cloth_decide(ClothState* st, const double* __restrict__ pg, int nbg,
                                                      const double* __restrict__ pp, int nbp,
                                                      const double* __restrict__ pw, int nbw, int ls) {
  constexpr int NS = 6 + kClothTrials;
  __shared__ double red[NS][256];
  if (st->done) return;
  double s[NS];
  for (int j = 0; j < NS; ++j) s[j] = 0.0;
  for (int q = threadIdx.x; q < nbg; q += blockDim.x) {
    s[0] += pg[q];
    s[1] += pg[nbg + q];
  }
  for (int q = threadIdx.x; q < nbp; q += blockDim.x)
    for (int j = 0; j < 4; ++j) s[2 + j] += pp[(size_t)j * nbp + q];
  if (pw)
    for (int q = threadIdx.x; q < nbw; q += blockDim.x)
      for (int j = 0; j < kClothTrials; ++j) s[6 + j] += pw[(size_t)j * nbw + q];
  for (int j = 0; j < NS; ++j) red[j][threadIdx.x] = s[j];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int j = 0; j < NS; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double gn = sqrt(red[0][0]), gd = red[1][0];
  const int k = st->k;
  if (k == 0) st->g0 = gn;
  const double r = st->g0 > 0.0 ? gn / st->g0 : 0.0;
  st->r = r;
  st->alpha = 0.0;
  if (!isfinite(r)) {
    st->done = 1;
    st->sweeps = k;
    return;
  }
  if (r <= st->rel_tol || st->g0 == 0.0) {
    st->converged = 1;
    st->done = 1;
    st->sweeps = k;
    return;
  }
  if (k >= st->max_sweeps) {
    st->done = 1;
    st->sweeps = k;
    return;
  }
  double alpha = 1.0;
  if (ls) {
    alpha = 0.0;
    for (int j = 0; j < kClothTrials; ++j) {
      const double a = 1.0 / double(1 << j);
      const double de = a * (red[2][0] + a * (red[3][0] + a * (red[4][0] + a * red[5][0]))) + red[6 + j][0];
      if (de <= 1e-4 * a * gd) {
        alpha = a;
        break;
      }
    }
    if (alpha == 0.0) st->ls_rejects += 1;
  }
  st->alpha = alpha;
  st->k = k + 1;
}

template <typename T>
__global__ void k_cloth_update(ClothDev<T> m, const ClothState* __restrict__ st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.V || m.pinned[i]) return;
  // after the decision: a step that stopped in this sweep has alpha 0
  const T a = T(st->alpha);
  if (a == T(0)) return;
  Vec4<T> u = m.u[i];
  const Vec4<T> d = m.D[i];
  u.x += a * d.x;
  u.y += a * d.y;
  u.z += a * d.z;
  m.u[i] = u;
}

template <typename T>
__global__ void k_cloth_finish(ClothDev<T> m, double* __restrict__ x, double* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.V) return;
  const Vec4<T> u = m.u[i];
  const double uu[3] = {double(u.x), double(u.y), double(u.z)};
  for (int q = 0; q < 3; ++q) {
    const double xn = m.xt[3 * i + q] + uu[q];
    if (v) v[3 * i + q] = m.pinned[i] ? 0.0 : uu[q] / m.h;
    x[3 * i + q] = xn;
  }
}

// Energy at x (FP64 records): membrane + bending + inertia, block partials.
__global__ void __launch_bounds__(128) k_cloth_energy(ClothDev<double> m, int nbT, int nbH, double* partial) {
  __shared__ double red[32];
  double e[1] = {0.0};
  const int b = blockIdx.x;
  if (b < nbT) {
    const int t = b * 128 + threadIdx.x;
    if (t < m.F) {
      const TriRec<double>& r = m.tris[t];
      double F[6], E[3];
      tri_state(r, m.u, F, E);
      const double tr = E[0] + E[2];
      e[0] = r.area * (r.mu * (E[0] * E[0] + 2.0 * E[1] * E[1] + E[2] * E[2]) + 0.5 * r.lam * tr * tr);
    }
  } else if (b < nbT + nbH) {
    const int q = (b - nbT) * 128 + threadIdx.x;
    if (q < m.H) {
      const HingeRec<double>& h = m.hinges[q];
      double w[3] = {h.wt[0], h.wt[1], h.wt[2]};
      for (int j = 0; j < 4; ++j) {
        const Vec4<double> uj = m.u[h.v[j]];
        w[0] += h.K[j] * uj.x;
        w[1] += h.K[j] * uj.y;
        w[2] += h.K[j] * uj.z;
      }
      e[0] = 0.5 * h.kb * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    }
  } else {
    const int v = (b - nbT - nbH) * 128 + threadIdx.x;
    if (v < m.V && !m.pinned[v]) {
      const Vec4<double> u = m.u[v], dz = m.dz[v];
      const double a = u.x - dz.x, bb = u.y - dz.y, c = u.z - dz.z;
      e[0] = 0.5 * m.mh2[v] * (a * a + bb * bb + c * c);
      for (int p = 0; p < m.n_planes; ++p) {
        const double* pl = m.planes + 4 * p;
        const double d = pl[0] * (m.xt[3 * v] + u.x) + pl[1] * (m.xt[3 * v + 1] + u.y) + pl[2] * (m.xt[3 * v + 2] + u.z) -
                         pl[3];
        if (d < m.dhat) e[0] += m.kappa * barrier_b(d, m.dhat);
      }
    }
  }
  block_sum<1>(e, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = e[0];
}

// Gradient at x (FP64): the gather's g, written in caller layout (zero for pinned).
__global__ void __launch_bounds__(128) k_cloth_grad(ClothDev<double> m, double* __restrict__ g_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.V) return;
  double g[3] = {0, 0, 0};
  if (!m.pinned[i]) {
    for (int q = m.tri_off[i]; q < m.tri_off[i + 1]; ++q) {
      const int ent = m.tri_inc[q], t = ent >> 2, a = ent & 3;
      const TriRec<double>& r = m.tris[t];
      double F[6], E[3];
      tri_state(r, m.u, F, E);
      const double tr = E[0] + E[2];
      const double S00 = 2 * r.mu * E[0] + r.lam * tr, S01 = 2 * r.mu * E[1], S11 = 2 * r.mu * E[2] + r.lam * tr;
      const double b0 = r.b[2 * a], b1 = r.b[2 * a + 1];
      const double Sb0 = S00 * b0 + S01 * b1, Sb1 = S01 * b0 + S11 * b1;
      for (int k = 0; k < 3; ++k) g[k] += r.area * (F[2 * k] * Sb0 + F[2 * k + 1] * Sb1);
    }
    for (int q = m.hin_off[i]; q < m.hin_off[i + 1]; ++q) {
      const int ent = m.hin_inc[q], e = ent >> 2, s = ent & 3;
      const HingeRec<double>& h = m.hinges[e];
      double w[3] = {h.wt[0], h.wt[1], h.wt[2]};
      for (int j = 0; j < 4; ++j) {
        const Vec4<double> uj = m.u[h.v[j]];
        w[0] += h.K[j] * uj.x;
        w[1] += h.K[j] * uj.y;
        w[2] += h.K[j] * uj.z;
      }
      for (int k = 0; k < 3; ++k) g[k] += h.kb * h.K[s] * w[k];
    }
    const Vec4<double> u = m.u[i], dz = m.dz[i];
    g[0] += m.mh2[i] * (u.x - dz.x);
    g[1] += m.mh2[i] * (u.y - dz.y);
    g[2] += m.mh2[i] * (u.z - dz.z);
    for (int p = 0; p < m.n_planes; ++p) {
      const double* pl = m.planes + 4 * p;
      const double d = pl[0] * (m.xt[3 * i] + u.x) + pl[1] * (m.xt[3 * i + 1] + u.y) + pl[2] * (m.xt[3 * i + 2] + u.z) -
                       pl[3];
      if (d > 0.0 && d < m.dhat) {
        const double b1 = m.kappa * barrier_b1(d, m.dhat);
        for (int k = 0; k < 3; ++k) g[k] += b1 * pl[k];
      }
    }
  }
  for (int k = 0; k < 3; ++k) g_out[3 * i + k] = g[k];
}

template <typename X>
cudaError_t cdalloc(X** p, size_t n) {
  *p = nullptr;
  return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(X));
}

}  // namespace

// ------------------------------------------------------------------------- host side

template <typename T>
struct ClothBufs {
  TriRec<T>* tris = nullptr;
  HingeRec<T>* hinges = nullptr;
  T* mh2 = nullptr;
  Vec4<T>*u = nullptr, *dz = nullptr, *D = nullptr;
  bool ready = false;
  void release() {
    cudaFree(tris);
    cudaFree(hinges);
    cudaFree(mh2);
    cudaFree(u);
    cudaFree(dz);
    cudaFree(D);
    *this = ClothBufs();
  }
};

struct Cloth {
  int V = 0, F = 0, H = 0;
  int device = -1;
  double h = 0.0, grav[3] = {0, 0, 0};
  // host rest data (FP64)
  std::vector<int32_t> tv, hv;      // [F][3], [H][4]
  std::vector<double> b, area, mu, lam, K, kb, mass;
  std::vector<uint8_t> pinned;
  std::vector<int32_t> tri_off, tri_inc, hin_off, hin_inc;
  std::vector<double> planes;       // [n][4] walls
  double dhat = 0.0, kappa = 0.0;
  // device
  bool device_ready = false;
  int32_t *d_tri_off = nullptr, *d_tri_inc = nullptr, *d_hin_off = nullptr, *d_hin_inc = nullptr;
  uint8_t* d_pinned = nullptr;
  double *d_xt = nullptr, *d_partial = nullptr, *d_planes = nullptr;
  ClothState* d_state = nullptr;
  ClothBufs<float> f32;
  ClothBufs<double> f64;
  int nb_partial = 0;
  ~Cloth() {
    f32.release();
    f64.release();
    void* p[] = {d_tri_off, d_tri_inc, d_hin_off, d_hin_inc, d_pinned, d_xt, d_partial, d_state, d_planes};
    for (void* q : p)
      if (q) cudaFree(q);
  }
};

namespace {

#define CKC(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? JGS2_ENOMEM : JGS2_ECUDA,       \
                  std::string(#call) + ": " + cudaGetErrorString(e_));              \
  } while (0)

jgs2_status cloth_device(Cloth* c) {
  if (c->device_ready) {
    int dev = -1;
    CKC(cudaGetDevice(&dev));
    if (dev != c->device) return fail(JGS2_EINVAL, "cloth used on another device than its first call's");
    return JGS2_OK;
  }
  CKC(cudaGetDevice(&c->device));
  // a failed earlier call may have left some of these allocated
  void* prior[] = {c->d_tri_off, c->d_tri_inc, c->d_hin_off, c->d_hin_inc, c->d_pinned,
                   c->d_xt,      c->d_partial, c->d_state,   c->d_planes};
  for (void* q : prior)
    if (q) cudaFree(q);
  c->d_tri_off = c->d_tri_inc = c->d_hin_off = c->d_hin_inc = nullptr;
  c->d_pinned = nullptr;
  c->d_xt = c->d_partial = c->d_planes = nullptr;
  c->d_state = nullptr;
  const int V = c->V;
  CKC(cdalloc(&c->d_tri_off, V + 1));
  CKC(cdalloc(&c->d_tri_inc, c->tri_inc.size()));
  CKC(cdalloc(&c->d_hin_off, V + 1));
  CKC(cdalloc(&c->d_hin_inc, c->hin_inc.size()));
  CKC(cdalloc(&c->d_pinned, V));
  CKC(cdalloc(&c->d_xt, 3 * (size_t)V));
  CKC(cudaMemcpy(c->d_tri_off, c->tri_off.data(), sizeof(int32_t) * (V + 1), cudaMemcpyHostToDevice));
  if (!c->tri_inc.empty())
    CKC(cudaMemcpy(c->d_tri_inc, c->tri_inc.data(), sizeof(int32_t) * c->tri_inc.size(), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(c->d_hin_off, c->hin_off.data(), sizeof(int32_t) * (V + 1), cudaMemcpyHostToDevice));
  if (!c->hin_inc.empty())
    CKC(cudaMemcpy(c->d_hin_inc, c->hin_inc.data(), sizeof(int32_t) * c->hin_inc.size(), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(c->d_pinned, c->pinned.data(), V, cudaMemcpyHostToDevice));
  const int nbT = (c->F + 127) / 128, nbH = (c->H + 127) / 128, nbV = (V + 127) / 128;
  c->nb_partial = nbT + nbH + nbV;
  CKC(cdalloc(&c->d_partial, (size_t)6 * c->nb_partial + (size_t)kClothTrials * nbV + 16));
  if (!c->planes.empty()) {
    CKC(cdalloc(&c->d_planes, c->planes.size()));
    CKC(cudaMemcpy(c->d_planes, c->planes.data(), sizeof(double) * c->planes.size(), cudaMemcpyHostToDevice));
  }
  CKC(cdalloc(&c->d_state, 1));
  c->device_ready = true;
  return JGS2_OK;
}

template <typename T>
ClothBufs<T>& cbufs(Cloth* c);
template <>
ClothBufs<float>& cbufs<float>(Cloth* c) { return c->f32; }
template <>
ClothBufs<double>& cbufs<double>(Cloth* c) { return c->f64; }

template <typename T>
jgs2_status cloth_prec(Cloth* c) {
  jgs2_status st = cloth_device(c);
  if (st != JGS2_OK) return st;
  ClothBufs<T>& b = cbufs<T>(c);
  if (b.ready) return JGS2_OK;
  b.release();  // what a failed earlier call left allocated
  const int V = c->V, F = c->F, H = c->H;
  std::vector<TriRec<T>> tr(F);
  for (int t = 0; t < F; ++t) {
    TriRec<T> r;
    std::memset(&r, 0, sizeof(r));
    for (int a = 0; a < 3; ++a) r.v[a] = c->tv[3 * t + a];
    for (int k = 0; k < 6; ++k) r.b[k] = T(c->b[6 * (size_t)t + k]);
    r.area = T(c->area[t]);
    r.mu = T(c->mu[t]);
    r.lam = T(c->lam[t]);
    tr[t] = r;
  }
  std::vector<HingeRec<T>> hr(H);
  for (int e = 0; e < H; ++e) {
    HingeRec<T> r;
    std::memset(&r, 0, sizeof(r));
    for (int j = 0; j < 4; ++j) {
      r.v[j] = c->hv[4 * e + j];
      r.K[j] = T(c->K[4 * (size_t)e + j]);
    }
    r.kb = T(c->kb[e]);
    hr[e] = r;
  }
  std::vector<T> mh2(V);
  for (int v = 0; v < V; ++v) mh2[v] = c->pinned[v] ? T(0) : T(c->mass[v] / (c->h * c->h));
  CKC(cdalloc(&b.tris, F));
  CKC(cdalloc(&b.hinges, H));
  CKC(cdalloc(&b.mh2, V));
  CKC(cdalloc(&b.u, V));
  CKC(cdalloc(&b.dz, V));
  CKC(cdalloc(&b.D, V));
  CKC(cudaMemcpy(b.tris, tr.data(), sizeof(TriRec<T>) * F, cudaMemcpyHostToDevice));
  if (H) CKC(cudaMemcpy(b.hinges, hr.data(), sizeof(HingeRec<T>) * H, cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(b.mh2, mh2.data(), sizeof(T) * V, cudaMemcpyHostToDevice));
  b.ready = true;
  return JGS2_OK;
}

template <typename T>
ClothDev<T> cloth_view(Cloth* c) {
  ClothBufs<T>& b = cbufs<T>(c);
  ClothDev<T> d;
  d.V = c->V;
  d.F = c->F;
  d.H = c->H;
  d.tris = b.tris;
  d.tris_mut = b.tris;
  d.hinges = b.hinges;
  d.hinges_mut = b.hinges;
  d.tri_off = c->d_tri_off;
  d.tri_inc = c->d_tri_inc;
  d.hin_off = c->d_hin_off;
  d.hin_inc = c->d_hin_inc;
  d.pinned = c->d_pinned;
  d.mh2 = b.mh2;
  d.u = b.u;
  d.dz = b.dz;
  d.D = b.D;
  d.xt = c->d_xt;
  d.n_planes = (int)c->planes.size() / 4;
  d.planes = c->d_planes;
  d.dhat = c->dhat;
  d.kappa = c->kappa;
  d.rc = 2.0 * c->dhat;
  d.h = c->h;
  for (int q = 0; q < 3; ++q) d.grav[q] = c->grav[q];
  return d;
}

// n sweeps (max_sweeps = n, rel_tol < 0) or a step (the options' cap and tolerance).
template <typename T>
jgs2_status cloth_run(Cloth* c, const double* x, const double* v, const double* xk, int max_sweeps, double rel_tol,
                      int ls, int check_every, cudaStream_t s, ClothState* out) {
  jgs2_status st = cloth_prec<T>(c);
  if (st != JGS2_OK) return st;
  ClothDev<T> d = cloth_view<T>(c);
  const int V = c->V;
  const int nbV = (V + 127) / 128, nbT = (c->F + 127) / 128, nbH = (c->H + 127) / 128;
  k_cloth_setup_vertices<T><<<nbV, 128, 0, s>>>(d, x, v, xk);
  k_cloth_setup_elements<T><<<std::max(1, (std::max(c->F, c->H) + 127) / 128), 128, 0, s>>>(d);
  ClothState init;
  std::memset(&init, 0, sizeof(init));
  init.max_sweeps = max_sweeps;
  init.rel_tol = rel_tol;
  CKC(cudaMemcpyAsync(c->d_state, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  double* pg = c->d_partial;
  double* pp = c->d_partial + 2 * (size_t)nbV;
  const int nbp = nbT + nbH + nbV;
  double* pw = pp + 4 * (size_t)nbp;
  const bool walls = !c->planes.empty();
  ClothState h_st;
  const int chunk = std::max(1, check_every);
  for (int k0 = 0;; k0 += chunk) {
    for (int q = 0; q < chunk; ++q) {
      k_cloth_gather<T><<<nbV, 128, 0, s>>>(d, c->d_state, pg);
      if (ls) k_cloth_poly<T><<<nbp, 128, 0, s>>>(d, c->d_state, nbT, nbH, pp);
      if (ls && walls) k_cloth_wall_trials<T><<<nbV, 128, 0, s>>>(d, c->d_state, pw);
      k_cloth_decide<<<1, 256, 0, s>>>(c->d_state, pg, nbV, pp, nbp, walls ? pw : nullptr, nbV, ls);
      k_cloth_update<T><<<nbV, 128, 0, s>>>(d, c->d_state);
    }
    CKC(cudaGetLastError());
    CKC(cudaMemcpyAsync(&h_st, c->d_state, sizeof(h_st), cudaMemcpyDeviceToHost, s));
    CKC(cudaStreamSynchronize(s));
    if (h_st.done || k0 + chunk > max_sweeps + 1) break;
  }
  *out = h_st;
  return JGS2_OK;
}

jgs2_status cloth_check_opts(const jgs2_step_opts* o) {
  if (!o) return fail(JGS2_EINVAL, "null options");
  if (o->precision != JGS2_FP32 && o->precision != JGS2_FP64) return fail(JGS2_EINVAL, "bad precision");
  if (o->max_sweeps < 0) return fail(JGS2_EINVAL, "max_sweeps must be >= 0");
  return JGS2_OK;
}

}  // namespace

jgs2_status cloth_create(const jgs2_cloth_desc* d, Cloth** out) {
  if (!d || !out) return fail(JGS2_EINVAL, "null argument");
  *out = nullptr;
  const int V = d->n_vertices, F = d->n_tris;
  if (V <= 0 || F <= 0 || !d->rest_pos || !d->tris) return fail(JGS2_EINVAL, "empty cloth");
  if (!(d->dt > 0.0) || !(d->youngs > 0.0) || !(d->poisson > -1.0 && d->poisson < 0.5) ||
      !(d->thickness > 0.0) || !(d->density > 0.0) || !(d->bend >= 0.0))
    return fail(JGS2_EINVAL, "cloth material or time step out of range");
  std::unique_ptr<Cloth> c(new Cloth());
  c->V = V;
  c->F = F;
  c->h = d->dt;
  for (int q = 0; q < 3; ++q) c->grav[q] = d->gravity[q];
  c->tv.assign(d->tris, d->tris + 3 * (size_t)F);
  if (d->n_planes < 0 || (d->n_planes > 0 && (!d->planes || !(d->dhat > 0.0) || !(d->kappa > 0.0))))
    return fail(JGS2_EINVAL, "cloth walls need planes, dhat > 0 and kappa > 0");
  if (d->n_planes > 0) {
    c->planes.assign(d->planes, d->planes + 4 * (size_t)d->n_planes);
    c->dhat = d->dhat;
    c->kappa = d->kappa;
  }
  c->pinned.assign(V, 0);
  if (d->pinned)
    for (int v = 0; v < V; ++v) c->pinned[v] = d->pinned[v] ? 1 : 0;
  const double* X = d->rest_pos;
  // walls: unit normals, and every free vertex of the rest state strictly on the open side
  // (the barrier is undefined at and behind a wall)
  for (int p = 0; p < d->n_planes; ++p) {
    const double* pl = d->planes + 4 * (size_t)p;
    const double nn = std::sqrt(pl[0] * pl[0] + pl[1] * pl[1] + pl[2] * pl[2]);
    if (!std::isfinite(pl[3]) || !(std::fabs(nn - 1.0) <= 1e-9))
      return fail(JGS2_EINVAL, "cloth wall " + std::to_string(p) + ": the normal must be a unit vector, the offset finite");
    for (int v = 0; v < V; ++v)
      if (!c->pinned[v] && !(pl[0] * X[3 * (size_t)v] + pl[1] * X[3 * (size_t)v + 1] + pl[2] * X[3 * (size_t)v + 2] -
                                 pl[3] > 0.0))
        return fail(JGS2_EINTERSECT, "free rest vertex " + std::to_string(v) + " is on or behind cloth wall " +
                                         std::to_string(p));
  }
  c->b.resize(6 * (size_t)F);
  c->area.resize(F);
  c->mu.assign(F, d->youngs * d->thickness / (2.0 * (1.0 + d->poisson)));
  c->lam.assign(F, d->youngs * d->thickness * d->poisson / (1.0 - d->poisson * d->poisson));
  c->mass.assign(V, 0.0);
  for (int t = 0; t < F; ++t) {
    const int* tv = &c->tv[3 * (size_t)t];
    for (int a = 0; a < 3; ++a)
      if (tv[a] < 0 || tv[a] >= V) return fail(JGS2_EINVAL, "triangle vertex index out of range");
    if (tv[0] == tv[1] || tv[1] == tv[2] || tv[0] == tv[2]) return fail(JGS2_EINVAL, "degenerate triangle");
    double e1[3], e2[3];
    for (int q = 0; q < 3; ++q) {
      e1[q] = X[3 * tv[1] + q] - X[3 * tv[0] + q];
      e2[q] = X[3 * tv[2] + q] - X[3 * tv[0] + q];
    }
    const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    const double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    if (!(nn > 1e-300) || !(l1 > 0.0)) return fail(JGS2_EINVAL, "triangle with zero area");
    // orthonormal frame of the triangle's plane: t1 along e1, t2 = n x t1
    double t1[3], t2[3];
    for (int q = 0; q < 3; ++q) t1[q] = e1[q] / l1;
    const double nu[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
    t2[0] = nu[1] * t1[2] - nu[2] * t1[1];
    t2[1] = nu[2] * t1[0] - nu[0] * t1[2];
    t2[2] = nu[0] * t1[1] - nu[1] * t1[0];
    auto dot = [](const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
    const double D00 = dot(e1, t1), D01 = dot(e2, t1), D10 = dot(e1, t2), D11 = dot(e2, t2);
    const double det = D00 * D11 - D01 * D10;
    // rows of Dm^-1: r0 = ( D11, -D01)/det, r1 = (-D10, D00)/det; b_1 = r0, b_2 = r1, b_0 = -(b_1 + b_2)
    const double r0[2] = {D11 / det, -D01 / det}, r1[2] = {-D10 / det, D00 / det};
    double* bt = &c->b[6 * (size_t)t];
    bt[0] = -(r0[0] + r1[0]);
    bt[1] = -(r0[1] + r1[1]);
    bt[2] = r0[0];
    bt[3] = r0[1];
    bt[4] = r1[0];
    bt[5] = r1[1];
    c->area[t] = 0.5 * nn;
    const double mv = d->density * d->thickness * c->area[t] / 3.0;
    for (int a = 0; a < 3; ++a) c->mass[tv[a]] += mv;
  }
  for (int v = 0; v < V; ++v)
    if (!c->pinned[v] && !(c->mass[v] > 0.0)) return fail(JGS2_EINVAL, "a free vertex is in no triangle");
  // hinges: interior edges with their two opposite vertices, in (min, max) edge order
  {
    std::vector<std::array<int, 4>> ed;  // (lo, hi, opposite, tri)
    ed.reserve(3 * (size_t)F);
    for (int t = 0; t < F; ++t)
      for (int k = 0; k < 3; ++k) {
        const int a = c->tv[3 * t + k], b2 = c->tv[3 * t + (k + 1) % 3], o = c->tv[3 * t + (k + 2) % 3];
        ed.push_back({std::min(a, b2), std::max(a, b2), o, t});
      }
    std::sort(ed.begin(), ed.end());
    auto cot = [&](int p, int q, int r) {
      double u[3], w[3];
      for (int k = 0; k < 3; ++k) {
        u[k] = X[3 * q + k] - X[3 * p + k];
        w[k] = X[3 * r + k] - X[3 * p + k];
      }
      const double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2], cz = u[0] * w[1] - u[1] * w[0];
      return (u[0] * w[0] + u[1] * w[1] + u[2] * w[2]) / std::sqrt(cx * cx + cy * cy + cz * cz);
    };
    for (size_t q = 0; q < ed.size();) {
      size_t r = q;
      while (r < ed.size() && ed[r][0] == ed[q][0] && ed[r][1] == ed[q][1]) ++r;
      if (r - q == 2) {
        // the first triangle (in triangle order) gives x_2, the second x_3
        const auto& A = ed[q][3] < ed[q + 1][3] ? ed[q] : ed[q + 1];
        const auto& B = ed[q][3] < ed[q + 1][3] ? ed[q + 1] : ed[q];
        const int x0 = A[0], x1 = A[1], x2 = A[2], x3 = B[2];
        const double ca0 = cot(x0, x1, x2), ca1 = cot(x1, x0, x2), cc0 = cot(x0, x1, x3), cc1 = cot(x1, x0, x3);
        c->hv.insert(c->hv.end(), {x0, x1, x2, x3});
        c->K.insert(c->K.end(), {ca1 + cc1, ca0 + cc0, -(ca0 + ca1), -(cc0 + cc1)});
        c->kb.push_back(3.0 * d->bend / (c->area[A[3]] + c->area[B[3]]));
      }
      q = r;
    }
    c->H = (int)c->kb.size();
  }
  // incidence (CSR, ascending element order per vertex)
  c->tri_off.assign(V + 1, 0);
  for (int t = 0; t < F; ++t)
    for (int a = 0; a < 3; ++a) c->tri_off[c->tv[3 * t + a] + 1]++;
  for (int v = 0; v < V; ++v) c->tri_off[v + 1] += c->tri_off[v];
  c->tri_inc.assign(c->tri_off[V], 0);
  {
    std::vector<int> fill(c->tri_off.begin(), c->tri_off.end() - 1);
    for (int t = 0; t < F; ++t)
      for (int a = 0; a < 3; ++a) c->tri_inc[fill[c->tv[3 * t + a]]++] = 4 * t + a;
  }
  c->hin_off.assign(V + 1, 0);
  for (int e = 0; e < c->H; ++e)
    for (int j = 0; j < 4; ++j) c->hin_off[c->hv[4 * e + j] + 1]++;
  for (int v = 0; v < V; ++v) c->hin_off[v + 1] += c->hin_off[v];
  c->hin_inc.assign(c->hin_off[V], 0);
  {
    std::vector<int> fill(c->hin_off.begin(), c->hin_off.end() - 1);
    for (int e = 0; e < c->H; ++e)
      for (int j = 0; j < 4; ++j) c->hin_inc[fill[c->hv[4 * e + j]]++] = 4 * e + j;
  }
  *out = c.release();
  return JGS2_OK;
}

}  // namespace jgs2

using jgs2::Cloth;

extern "C" {

jgs2_status jgs2_cloth_create(const jgs2_cloth_desc* desc, jgs2_cloth** out) {
  Cloth* c = nullptr;
  const jgs2_status s = jgs2::cloth_create(desc, &c);
  if (out) *out = reinterpret_cast<jgs2_cloth*>(c);
  return s;
}

jgs2_status jgs2_cloth_step(jgs2_cloth* cloth, double* x, double* v, const jgs2_step_opts* opts, void* stream,
                            jgs2_cloth_report* report) {
  Cloth* c = reinterpret_cast<Cloth*>(cloth);
  if (!c || !x || !v) return jgs2::fail(JGS2_EINVAL, "null argument");
  jgs2_status st = jgs2::cloth_check_opts(opts);
  if (st != JGS2_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  jgs2::ClothState out;
  st = opts->precision == JGS2_FP64
           ? jgs2::cloth_run<double>(c, x, v, nullptr, opts->max_sweeps, opts->rel_tol, opts->line_search,
                                     opts->check_every, s, &out)
           : jgs2::cloth_run<float>(c, x, v, nullptr, opts->max_sweeps, opts->rel_tol, opts->line_search,
                                    opts->check_every, s, &out);
  if (st != JGS2_OK) return st;
  if (report) {
    report->sweeps = out.sweeps;
    report->converged = out.converged;
    report->ls_rejects = out.ls_rejects;
    report->rel_residual = out.r;
    report->g0 = out.g0;
  }
  if (!std::isfinite(out.r)) return jgs2::fail(JGS2_EDIVERGED, "cloth residual is not finite");
  const int nb = (c->V + 127) / 128;
  if (opts->precision == JGS2_FP64)
    jgs2::k_cloth_finish<double><<<nb, 128, 0, s>>>(jgs2::cloth_view<double>(c), x, v);
  else
    jgs2::k_cloth_finish<float><<<nb, 128, 0, s>>>(jgs2::cloth_view<float>(c), x, v);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return jgs2::fail(JGS2_ECUDA, cudaGetErrorString(e));
  return out.converged ? JGS2_OK : JGS2_ENOTCONVERGED;
}

jgs2_status jgs2_cloth_sweeps(jgs2_cloth* cloth, const double* x_t, const double* v_t, double* x, int32_t n,
                              const jgs2_step_opts* opts, void* stream) {
  Cloth* c = reinterpret_cast<Cloth*>(cloth);
  if (!c || !x_t || !v_t || !x || n < 0) return jgs2::fail(JGS2_EINVAL, "bad argument");
  jgs2_status st = jgs2::cloth_check_opts(opts);
  if (st != JGS2_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  jgs2::ClothState out;
  st = opts->precision == JGS2_FP64
           ? jgs2::cloth_run<double>(c, x_t, v_t, x, n, -1.0, opts->line_search, std::max(1, n), s, &out)
           : jgs2::cloth_run<float>(c, x_t, v_t, x, n, -1.0, opts->line_search, std::max(1, n), s, &out);
  if (st != JGS2_OK) return st;
  const int nb = (c->V + 127) / 128;
  if (opts->precision == JGS2_FP64)
    jgs2::k_cloth_finish<double><<<nb, 128, 0, s>>>(jgs2::cloth_view<double>(c), x, nullptr);
  else
    jgs2::k_cloth_finish<float><<<nb, 128, 0, s>>>(jgs2::cloth_view<float>(c), x, nullptr);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return jgs2::fail(JGS2_ECUDA, cudaGetErrorString(e));
  return JGS2_OK;
}

jgs2_status jgs2_cloth_energy_gradient(jgs2_cloth* cloth, const double* x_t, const double* v_t, const double* x,
                                       double* energy, double* g, void* stream) {
  Cloth* c = reinterpret_cast<Cloth*>(cloth);
  if (!c || !x_t || !v_t || !x || (!energy && !g)) return jgs2::fail(JGS2_EINVAL, "bad argument");
  jgs2_status st = jgs2::cloth_prec<double>(c);
  if (st != JGS2_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  jgs2::ClothDev<double> d = jgs2::cloth_view<double>(c);
  const int nbV = (c->V + 127) / 128, nbT = (c->F + 127) / 128, nbH = (c->H + 127) / 128;
  jgs2::k_cloth_setup_vertices<double><<<nbV, 128, 0, s>>>(d, x_t, v_t, x);
  jgs2::k_cloth_setup_elements<double><<<std::max(1, (std::max(c->F, c->H) + 127) / 128), 128, 0, s>>>(d);
  if (g) jgs2::k_cloth_grad<<<nbV, 128, 0, s>>>(d, g);
  if (energy) {
    const int nb = nbT + nbH + nbV;
    jgs2::k_cloth_energy<<<nb, 128, 0, s>>>(d, nbT, nbH, c->d_partial);
    std::vector<double> p(nb);
    cudaError_t e = cudaMemcpyAsync(p.data(), c->d_partial, sizeof(double) * nb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return jgs2::fail(JGS2_ECUDA, cudaGetErrorString(e));
    double acc = 0.0;
    for (double q : p) acc += q;
    *energy = acc;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return jgs2::fail(JGS2_ECUDA, cudaGetErrorString(e));
  return JGS2_OK;
}

int32_t jgs2_cloth_n_hinges(const jgs2_cloth* cloth) {
  const Cloth* c = reinterpret_cast<const Cloth*>(cloth);
  return c ? c->H : -1;
}

void jgs2_cloth_destroy(jgs2_cloth* cloth) { delete reinterpret_cast<Cloth*>(cloth); }

}  // extern "C"
