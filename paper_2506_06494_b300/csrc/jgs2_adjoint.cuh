// Adjoint of a converged step (implicit-function theorem on Eq. 1's optimality condition):
//     H(x*) lam = gbar = dL/dx_{t+1} + dL/dv_{t+1} / h        (free DOFs)
// solved by flexible conjugate gradients whose preconditioner is the corrected sweep's local
// solve in linear mode: z_i = (H_ii + H~_i)^{-1} r_i, with H_ii, R_i and the rotated cubature
// element Hessians (Eq. cubature) taken at x*. The sweep's cubature estimate of the
// residual's reduced part (k_lin_pool, k_lin_precond<CORR = true>) is kept in the source but
// not used: it makes the preconditioned operator indefinite (eigenvalues of negative real
// part), and conjugate gradients stall with it. Without the correction the preconditioner
// is block Jacobi H_ii^{-1}. Then dL/dx_t, dL/dv_t and dL/dE_e follow from lam (see
// jgs2_step_adjoint in jgs2.h).
#pragma once
#include "jgs2_kernels.cuh"

namespace jgs2 {

struct AdjScalars {
  double pq, rp, zq, rr, rr0, alpha, beta;
  int32_t done, iters;
  uint32_t ticket;
  int32_t pad;
};

// directional derivative of cof F along dF (cof is quadratic: column j of cof is the
// cross product of the other two columns)
template <typename T>
__device__ __forceinline__ void cof_dir(const T (&F)[9], const T (&dF)[9], T (&dC)[9]) {
  T f[3][3], d[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      f[k][i] = F[3 * i + k];
      d[k][i] = dF[3 * i + k];
    }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int a = (j + 1) % 3, b = (j + 2) % 3;
    const T c0 = d[a][1] * f[b][2] - d[a][2] * f[b][1] + f[a][1] * d[b][2] - f[a][2] * d[b][1];
    const T c1 = d[a][2] * f[b][0] - d[a][0] * f[b][2] + f[a][2] * d[b][0] - f[a][0] * d[b][2];
    const T c2 = d[a][0] * f[b][1] - d[a][1] * f[b][0] + f[a][0] * d[b][1] - f[a][1] * d[b][0];
    dC[j] = c0;
    dC[3 + j] = c1;
    dC[6 + j] = c2;
  }
}

// dP = dP/dF : dF = mu dF + lam' (cof F : dF) cof F + s dcof   (s = lam'(J-1) - mu)
template <typename T>
__device__ __forceinline__ void tet_dP(const TetRec<T>& r, const T (&F)[9], const T (&C)[9], T J, const T (&dF)[9],
                                       T (&dP)[9]) {
  T dC[9];
  cof_dir(F, dF, dC);
  T cd = T(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) cd += C[q] * dF[q];
  const T s = r.lp * (J - T(1)) - r.mu;
#pragma unroll
  for (int q = 0; q < 9; ++q) dP[q] = r.mu * dF[q] + r.lp * cd * C[q] + s * dC[q];
}

// y = H(x*) v over free vertices (exact elastic Hessian plus inertia), thread per vertex
template <typename T>
__global__ void __launch_bounds__(128) k_hv(DevMesh<T> m, const Vec4<T>* __restrict__ v, Vec4<T>* __restrict__ y,
                                            const AdjScalars* sc) {
  if (sc && sc->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.Vf) return;
  const int slice = i / kSlice, lane = i % kSlice;
  const int base = m.inc_off[slice] + lane;
  const int n = m.inc_len[i];
  T acc[3] = {T(0), T(0), T(0)};
  for (int j = 0; j < n; ++j) {
    const int ent = __ldg(m.inc + base + j * kSlice);
    const int t = ent >> 2, c = ent & 3;
    const TetRec<T> r = m.tets[t];
    T F[9], C[9], dF[9], dP[9], b[3];
    tet_F(r, m.u, F);
    cofactor(F, C);
    const T J = F[0] * C[0] + F[1] * C[1] + F[2] * C[2];
    tet_dF(r, v, m.Vf, dF);
    tet_dP(r, F, C, J, dF, dP);
    corner_b(r, c, b);
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[a] += r.vol * (dP[3 * a] * b[0] + dP[3 * a + 1] * b[1] + dP[3 * a + 2] * b[2]);
  }
  const Vec4<T> vi = v[i];
  const T mh = m.mh2[i];
  y[i] = Vec4<T>{acc[0] + mh * vi.x, acc[1] + mh * vi.y, acc[2] + mh * vi.z, T(0)};
}

// once per adjoint: Cholesky factors of H_ii + H~_i (and of H_ii) per vertex, from the
// gather (g, H, R in ghr) and the rotated cubature element Hessians at x*
template <typename T, bool CORR>
__global__ void __launch_bounds__(128) k_lin_setup(DevMesh<T> m, T* __restrict__ lin /* [24][Vf] */) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.Vf) return;
  const size_t S = m.Vf;
  const T* o = m.ghr + i;
  T H[6], R[9];
#pragma unroll
  for (int q = 0; q < 6; ++q) H[q] = o[(3 + q) * S];
#pragma unroll
  for (int q = 0; q < 9; ++q) R[q] = o[(9 + q) * S];
  T A[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) A[q] = H[q];
  if (CORR) {
    T Ht[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    for (int s = 0; s < m.n_cub; ++s) {
      const int p = m.cub_p[(size_t)s * m.cs + i];
      if (p < 0) continue;
      const T w = m.cub_w[(size_t)s * m.cs + i];
      T U[36];
      const T* up = m.cub_u + (size_t)s * 36 * m.cs + i;
#pragma unroll
      for (int q = 0; q < 36; ++q) U[q] = up[(size_t)q * m.cs];
      T gdummy[3] = {T(0), T(0), T(0)};
      slot_sums(m.pool_H + (size_t)p * kPoolStride, w, U, Ht, gdummy);
    }
    T Hf[9] = {Ht[0], Ht[1], Ht[2], Ht[1], Ht[3], Ht[4], Ht[2], Ht[4], Ht[5]}, RH[9], Hw[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        RH[3 * a + b] = R[3 * a] * Hf[b] + R[3 * a + 1] * Hf[3 + b] + R[3 * a + 2] * Hf[6 + b];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        Hw[3 * a + b] = RH[3 * a] * R[3 * b] + RH[3 * a + 1] * R[3 * b + 1] + RH[3 * a + 2] * R[3 * b + 2];
    A[0] += Hw[0];
    A[1] += T(0.5) * (Hw[1] + Hw[3]);
    A[2] += T(0.5) * (Hw[2] + Hw[6]);
    A[3] += Hw[4];
    A[4] += T(0.5) * (Hw[5] + Hw[7]);
    A[5] += Hw[8];
  }
  // use A if it is positive definite, else H (reading R7)
  T e1[3] = {T(1), T(0), T(0)}, tmp[3];
  const bool ok = chol3_solve(A, e1, tmp);
#pragma unroll
  for (int q = 0; q < 6; ++q) lin[q * S + i] = ok ? A[q] : H[q];
#pragma unroll
  for (int q = 0; q < 9; ++q) lin[(6 + q) * S + i] = R[q];
}

// rotated residual at the cubature elements' corners: G'[p][3a+j] = (R_a^T r_a)_j
template <typename T>
__global__ void k_lin_pool(DevMesh<T> m, const Vec4<T>* __restrict__ r, const AdjScalars* sc) {
  if (sc->done) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.nP * 12) return;
  const int p = e / 12, k = e % 12, a = k / 3, j = k % 3;
  const int v = m.tets[m.pool_tet[p]].v[a];
  T val = T(0);
  if (v < m.Vf) {
    const Vec4<T> rv = r[v];
    const T* R = m.pool_R + (size_t)p * 36 + 9 * a;
    val = R[j] * rv.x + R[3 + j] * rv.y + R[6 + j] * rv.z;
  }
  m.pool_G[(size_t)p * 12 + k] = val;
}

// z = (H_ii + H~_i)^{-1} (r_i + R_i sum_s w_s U_s^T G'_s)
template <typename T, bool CORR>
__global__ void __launch_bounds__(128) k_lin_precond(DevMesh<T> m, const T* __restrict__ lin,
                                                     const Vec4<T>* __restrict__ r, Vec4<T>* __restrict__ z,
                                                     const AdjScalars* sc) {
  if (sc->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.Vf) return;
  const size_t S = m.Vf;
  T A[6], R[9];
#pragma unroll
  for (int q = 0; q < 6; ++q) A[q] = lin[q * S + i];
  const Vec4<T> ri = r[i];
  T rhs[3] = {ri.x, ri.y, ri.z};
  if (CORR) {
#pragma unroll
    for (int q = 0; q < 9; ++q) R[q] = lin[(6 + q) * S + i];
    T gt[3] = {T(0), T(0), T(0)};
    for (int s = 0; s < m.n_cub; ++s) {
      const int p = m.cub_p[(size_t)s * m.cs + i];
      if (p < 0) continue;
      const T w = m.cub_w[(size_t)s * m.cs + i];
      const T* up = m.cub_u + (size_t)s * 36 * m.cs + i;
      const T* Gp = m.pool_G + (size_t)p * 12;
#pragma unroll
      for (int rr = 0; rr < 12; ++rr) {
        const T gr = w * __ldg(Gp + rr);
        gt[0] += up[(size_t)(3 * rr) * m.cs] * gr;
        gt[1] += up[(size_t)(3 * rr + 1) * m.cs] * gr;
        gt[2] += up[(size_t)(3 * rr + 2) * m.cs] * gr;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) rhs[a] += R[3 * a] * gt[0] + R[3 * a + 1] * gt[1] + R[3 * a + 2] * gt[2];
  }
  T d[3];
  if (!chol3_solve(A, rhs, d)) d[0] = d[1] = d[2] = T(0);
  z[i] = Vec4<T>{d[0], d[1], d[2], T(0)};
}

// FP64 dot products a.b and c.d over free vertices; the last block runs the FCG scalar step
// (mode 0: alpha = r.p / p.q; mode 1: beta = -z.q / p.q and the stopping test)
template <typename T>
__global__ void __launch_bounds__(128) k_dots(DevMesh<T> m, const Vec4<T>* a, const Vec4<T>* b, const Vec4<T>* c,
                                              const Vec4<T>* d, double* partial, AdjScalars* sc, int mode,
                                              double tol2, int max_iters) {
  if (sc->done) return;
  __shared__ double red[64];
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.Vf; i += gridDim.x * blockDim.x) {
    const Vec4<T> x = a[i], y = b[i], u = c[i], w = d[i];
    acc[0] += double(x.x) * double(y.x) + double(x.y) * double(y.y) + double(x.z) * double(y.z);
    acc[1] += double(u.x) * double(w.x) + double(u.y) * double(w.y) + double(u.z) * double(w.z);
  }
  block_sum<2>(acc, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = acc[0];
    partial[gridDim.x + blockIdx.x] = acc[1];
  }
  if (!last_block(&sc->ticket)) return;
  const double s0 = block_sum_array(partial, gridDim.x, 1, red);
  const double s1 = block_sum_array(partial + gridDim.x, gridDim.x, 1, red);
  if (threadIdx.x == 0) {
    sc->ticket = 0;
    if (mode == 2) {
      sc->rr0 = s0;
      sc->rr = s0;
      if (!(s0 > 0.0)) sc->done = 1;
    } else if (mode == 0) {
      sc->pq = s0;
      sc->rp = s1;
      sc->alpha = s0 > 0.0 ? s1 / s0 : 0.0;
      if (!(s0 > 0.0)) sc->done = 2;  // H not positive definite along p
    } else {
      sc->zq = s0;
      sc->rr = s1;
      sc->beta = sc->pq > 0.0 ? -s0 / sc->pq : 0.0;
      sc->iters += 1;
      if (s1 <= tol2 * sc->rr0 || sc->iters >= max_iters) sc->done = 1;
    }
  }
}

template <typename T>
__global__ void k_axpy2(DevMesh<T> m, Vec4<T>* lam, Vec4<T>* r, const Vec4<T>* p, const Vec4<T>* q,
                        const AdjScalars* sc) {
  if (sc->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.Vf) return;
  const T a = T(sc->alpha);
  Vec4<T> l = lam[i], rr = r[i];
  const Vec4<T> pp = p[i], qq = q[i];
  l.x += a * pp.x;
  l.y += a * pp.y;
  l.z += a * pp.z;
  rr.x -= a * qq.x;
  rr.y -= a * qq.y;
  rr.z -= a * qq.z;
  lam[i] = l;
  r[i] = rr;
}

template <typename T>
__global__ void k_pupdate(DevMesh<T> m, Vec4<T>* p, const Vec4<T>* z, const AdjScalars* sc) {
  if (sc->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.Vf) return;
  const T b = T(sc->beta);
  Vec4<T> pp = p[i];
  const Vec4<T> zz = z[i];
  p[i] = Vec4<T>{zz.x + b * pp.x, zz.y + b * pp.y, zz.z + b * pp.z, T(0)};
}

// gbar = dL/dx1 + dL/dv1 / h in internal order (free vertices)
template <typename T>
__global__ void k_adj_rhs(DevMesh<T> m, const double* __restrict__ gx1, const double* __restrict__ gv1,
                          Vec4<T>* r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.Vf) return;
  const int c = m.perm[i];
  r[i] = Vec4<T>{T(gx1[3 * c] + gv1[3 * c] / m.h), T(gx1[3 * c + 1] + gv1[3 * c + 1] / m.h),
                 T(gx1[3 * c + 2] + gv1[3 * c + 2] / m.h), T(0)};
}

// per tet: elastic coupling of pinned corners -(H_pf lam)_p (into coup, FP64 atomics) and
// dL/dE_e = -sum_a lam_a . (V P b_a) / E_e (accumulated into gE in caller tet order)
template <typename T>
__global__ void k_adj_tets(DevMesh<T> m, const Vec4<T>* __restrict__ lam, const int32_t* __restrict__ tperm,
                           const double* __restrict__ youngs, double* __restrict__ coup, double* __restrict__ gE) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.T_) return;
  const TetRec<T> r = m.tets[t];
  T F[9], C[9];
  tet_F(r, m.u, F);
  cofactor(F, C);
  const T J = F[0] * C[0] + F[1] * C[1] + F[2] * C[2];
  const T s = r.lp * (J - T(1)) - r.mu;
  double dl = 0.0;
  bool any_pinned = false;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int v = r.v[c];
    if (v >= m.Vf) {
      any_pinned = true;
      continue;
    }
    T b[3];
    corner_b(r, c, b);
    const Vec4<T> l = lam[v];
    T g[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T Pb = (r.mu * F[3 * a] + s * C[3 * a]) * b[0] + (r.mu * F[3 * a + 1] + s * C[3 * a + 1]) * b[1] +
                   (r.mu * F[3 * a + 2] + s * C[3 * a + 2]) * b[2];
      g[a] = r.vol * Pb;
    }
    dl += double(l.x) * double(g[0]) + double(l.y) * double(g[1]) + double(l.z) * double(g[2]);
  }
  const int tc = tperm[t];
  gE[tc] += -dl / youngs[tc];
  if (!any_pinned) return;
  T dF[9], dP[9];
  tet_dF(r, lam, m.Vf, dF);
  tet_dP(r, F, C, J, dF, dP);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int v = r.v[c];
    if (v < m.Vf) continue;
    T b[3];
    corner_b(r, c, b);
#pragma unroll
    for (int a = 0; a < 3; ++a)
      atomicAdd(coup + 3 * (size_t)v + a, double(r.vol * (dP[3 * a] * b[0] + dP[3 * a + 1] * b[1] + dP[3 * a + 2] * b[2])));
  }
}

// outputs in caller order
template <typename T>
__global__ void k_adj_out(DevMesh<T> m, const Vec4<T>* __restrict__ lam, const double* __restrict__ coup,
                          const double* __restrict__ gx1, const double* __restrict__ gv1, double* __restrict__ gx,
                          double* __restrict__ gv) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= m.V) return;
  const int c = m.perm[v];
  if (v < m.Vf) {
    const Vec4<T> l = lam[v];
    const double mh = double(m.mh2[v]);
    const double lv[3] = {double(l.x), double(l.y), double(l.z)};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      gx[3 * c + q] = mh * lv[q] - gv1[3 * c + q] / m.h;
      gv[3 * c + q] = mh * m.h * lv[q];
    }
  } else {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      gx[3 * c + q] = gx1[3 * c + q] - coup[3 * (size_t)v + q];
      gv[3 * c + q] = 0.0;
    }
  }
}

}  // namespace jgs2
