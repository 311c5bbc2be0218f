// Device code of the JGS2 sweep (sm_103a). One sweep k from x^k = x_t + u:
//   k_elem       per tet: F_e(x^k) into the element records (tiles staged in shared memory).
//   k_gather     per free vertex: g_i, H_ii and the volume-weighted deformation gradient
//                from the incident element records, R_i = polar(F_i), the uncorrected
//                direction D_J, FP64-class partial sums |g|^2 and g.D_J.
//   k_pool       per cubature pool element: the element Hessian at x^k rotated into the
//                rest frames of its corners (the R_a factors of Eq. tilde_phi) and the
//                rotated corner gradients, from the gather's g and R.
//   k_correct    per free vertex: the cubature sums H~_i, g~_i (Eq. cubature), the 3x3
//                solve of Eq. reduced_local, the direction D_i and g.D; its last block
//                closes the sweep's reduction (residual, stopping test).
//   k_pair_trials, k_energy, k_ls_decide  (line search, reading R17): the barrier and the
//                exact elastic/inertial energy change E(x + alpha_j d) - E(x) for
//                alpha_j = 2^-j along the pass's direction(s); one block picks the step.
//   k_update     u += alpha d.
// A Gauss-Seidel colour pass runs the same kernels with a vertex mask (DevMesh::vmask):
// vertices off the colour get D = D_J = 0.
#pragma once
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <utility>

#include "jgs2_internal.h"

namespace jgs2 {
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem);
}
#include "jgs2_contact.cuh"

namespace jgs2 {

// ------------------------------------------------------------------ small helpers

template <typename T>
__device__ __forceinline__ T dsqrt(T x) { return sqrt(x); }
template <>
__device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum of NV doubles per thread; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem /* [32*NV] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) smem[j * 32 + wid] = v[j];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double x = lane < nw ? smem[j * 32 + lane] : 0.0;
      v[j] = warp_sum(x);
    }
  }
  __syncthreads();
}

// Per-thread accumulator of a reduction. FP64 path: a double. FP32 path: a float-float
// pair h + l (|l| <= ulp(h)/2, about 48 significant bits) formed with Knuth's two-sum and
// exact FMA products on the FP32 units, so the sums keep FP64-class precision without
// the FP64 pipe (a small fraction of FP32 throughput on this part).
template <typename T>
struct Acc;

template <>
struct Acc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ double value() const { return v; }
  __device__ __forceinline__ void add_lane(int o) { v += __shfl_down_sync(0xffffffffu, v, o); }
};

template <>
struct Acc<float> {
  float h = 0.f, l = 0.f;
  // (h, l) += (bh, bl): two-sum of the leading parts, then the trailing parts
  __device__ __forceinline__ void add2(float bh, float bl) {
    const float s = h + bh;
    const float bb = s - h;
    float e = (h - (s - bb)) + (bh - bb);
    e += l + bl;
    h = s + e;
    l = e - (h - s);
  }
  __device__ __forceinline__ void add(float x) { add2(x, 0.f); }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    add2(p, fmaf(a, b, -p));  // a*b = p + fma(a, b, -p) exactly
  }
  __device__ __forceinline__ double value() const { return double(h) + double(l); }
  __device__ __forceinline__ void add_lane(int o) {
    const float bh = __shfl_down_sync(0xffffffffu, h, o);
    const float bl = __shfl_down_sync(0xffffffffu, l, o);
    add2(bh, bl);
  }
};

// Fixed-order block sum of NV accumulators per thread; out valid in thread 0.
// smem holds 32 * NV entries of Acc<T>.
template <typename T, int NV>
__device__ __forceinline__ void block_sum_acc(Acc<T> (&a)[NV], double (&out)[NV], Acc<T>* smem) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[j].add_lane(o);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) smem[j * 32 + wid] = a[j];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      Acc<T> x;
      if (lane < nw) x = smem[j * 32 + lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x.add_lane(o);
      out[j] = x.value();
    }
  }
  __syncthreads();
}

// Batch meshes: adds NV per-thread accumulators into the per-scene FP64 sums of scene sc
// (-1: none). Called by every thread of the block. A block whose threads all belong to one
// scene (or none) reduces with Acc<T> and adds once per value (scenes are contiguous, so
// that is almost every block); otherwise a warp whose lanes share one scene adds once, and
// a mixed warp adds per lane.
template <typename T, int NV>
__device__ __forceinline__ void scene_reduce_acc(Acc<T> (&a)[NV], int sc, double* sacc, int off) {
  __shared__ int s_min, s_max;
  __shared__ Acc<T> s_red[32 * NV];
  if (threadIdx.x == 0) {
    s_min = INT_MAX;
    s_max = -1;
  }
  __syncthreads();
  {
    const int lo = __reduce_min_sync(0xffffffffu, sc >= 0 ? sc : INT_MAX);
    const int hi = __reduce_max_sync(0xffffffffu, sc);
    if ((threadIdx.x & 31) == 0) {
      if (lo != INT_MAX) atomicMin(&s_min, lo);
      if (hi >= 0) atomicMax(&s_max, hi);
    }
  }
  __syncthreads();
  const int bmin = s_min, bmax = s_max;
  if (bmax < 0) return;  // nothing to add (block-uniform)
  if (bmin == bmax) {
    double out[NV];
    block_sum_acc<T, NV>(a, out, s_red);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int j = 0; j < NV; ++j) atomicAdd(sacc + (size_t)bmin * kSceneAcc + off + j, out[j]);
    }
    return;
  }
  const int s0 = __shfl_sync(0xffffffffu, sc, 0);
  if (__all_sync(0xffffffffu, sc == s0)) {
    if (s0 < 0) return;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a[j].add_lane(o);
      if ((threadIdx.x & 31) == 0) atomicAdd(sacc + (size_t)s0 * kSceneAcc + off + j, a[j].value());
    }
  } else if (sc >= 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) atomicAdd(sacc + (size_t)sc * kSceneAcc + off + j, a[j].value());
  }
}

// Sum of n partials (fixed order) by one block; result valid in thread 0.
__device__ __forceinline__ double block_sum_array(const double* p, int n, int stride,
                                                  double* smem) {
  double acc[1] = {0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc[0] += p[(size_t)i * stride];
  block_sum<1>(acc, smem);
  return acc[0];
}

// Last-block-done ticket: returns true in every thread of the block that finishes last.
__device__ __forceinline__ bool last_block(uint32_t* ticket) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

template <typename T>
__device__ __forceinline__ void load3(const Vec4<T>* a, int i, T (&o)[3]) {
  Vec4<T> q = a[i];
  o[0] = q.x;
  o[1] = q.y;
  o[2] = q.z;
}

// ------------------------------------------------------------------ bulk copies
// Asynchronous global -> shared copies of contiguous byte ranges (cp.async.bulk, the
// Blackwell copy engine's 1-D form) completed on an mbarrier: one thread posts the
// expected byte count and the copy; every thread waits on the barrier's phase. Waits are
// bounded (kWaitPolls polls of mbarrier.try_wait); a caller that gives up reports
// JGS2_ETIMEOUT. Addresses and sizes are multiples of 16 bytes.
constexpr int kWaitPolls = 1 << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// true once the barrier's phase with this parity has completed; false after kWaitPolls polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < kWaitPolls; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Copies the records of tets [t0, t0 + n) into shared memory with coalesced 16-byte loads
// (a record is a whole number of 16-byte words), so that the per-tet reads that follow
// come from shared memory instead of strided global loads.
template <typename T, int NT>
__device__ __forceinline__ void stage_tets(const TetRec<T>* __restrict__ src, int t0, int n, TetRec<T>* dst) {
  constexpr int W = int(sizeof(TetRec<T>) / 16);
  static_assert(sizeof(TetRec<T>) % 16 == 0, "tet record must be a whole number of 16-byte words");
  const float4* s = reinterpret_cast<const float4*>(src + t0);
  float4* d = reinterpret_cast<float4*>(dst);
  for (int q = threadIdx.x; q < n * W; q += NT) d[q] = __ldg(s + q);
}

// Deformation gradient of a tet at x = x_t + u: F = F(x_t) + [u1-u0, u2-u0, u3-u0] B.
template <typename T>
__device__ __forceinline__ void tet_F(const TetRec<T>& r, const Vec4<T>* u, T (&F)[9]) {
  T u0[3], uk[3];
  load3(u, r.v[0], u0);
#pragma unroll
  for (int q = 0; q < 9; ++q) F[q] = r.Ft[q];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    load3(u, r.v[k + 1], uk);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T d = uk[i] - u0[i];
#pragma unroll
      for (int j = 0; j < 3; ++j) F[3 * i + j] += d * r.B[3 * k + j];
    }
  }
}

template <typename T>
__device__ __forceinline__ void cofactor(const T (&F)[9], T (&C)[9]);

// F_e(x) = F(x_t) + G with G = [u_1 - u_0, u_2 - u_0, u_3 - u_0] B, and J - 1 without the
// cancellation of det F - 1 near rest (which costs FP32 most of its digits where the
// volumetric stiffness lam' is large): for 3x3 matrices
//   det(F_t + G) - 1 = (det F_t - 1) + cof(F_t):G + F_t:cof(G) + det G,
// with det F_t - 1 formed in FP64 at step setup and every other term small.
template <typename T>
__device__ __forceinline__ void tet_F_jm1(const TetRec<T>& r, const Vec4<T>* u, T (&F)[9], T& jm1) {
  T u0[3], uk[3], G[9];
  load3(u, r.v[0], u0);
#pragma unroll
  for (int q = 0; q < 9; ++q) G[q] = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    load3(u, r.v[k + 1], uk);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T d = uk[i] - u0[i];
#pragma unroll
      for (int j = 0; j < 3; ++j) G[3 * i + j] += d * r.B[3 * k + j];
    }
  }
  T Ct[9], Cg[9];
  cofactor(r.Ft, Ct);
  cofactor(G, Cg);
  T a = T(0), b = T(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    a += Ct[q] * G[q];
    b += r.Ft[q] * Cg[q];
  }
  const T dg = G[0] * Cg[0] + G[1] * Cg[1] + G[2] * Cg[2];
  jm1 = r.jt1 + (a + (b + dg));
#pragma unroll
  for (int q = 0; q < 9; ++q) F[q] = r.Ft[q] + G[q];
}

// cof F = dJ/dF: column j of cof is the cross product of the other two columns of F.
template <typename T>
__device__ __forceinline__ void cofactor(const T (&F)[9], T (&C)[9]) {
  C[0] = F[4] * F[8] - F[5] * F[7];
  C[3] = F[2] * F[7] - F[1] * F[8];
  C[6] = F[1] * F[5] - F[2] * F[4];
  C[1] = F[5] * F[6] - F[3] * F[8];
  C[4] = F[0] * F[8] - F[2] * F[6];
  C[7] = F[2] * F[3] - F[0] * F[5];
  C[2] = F[3] * F[7] - F[4] * F[6];
  C[5] = F[1] * F[6] - F[0] * F[7];
  C[8] = F[0] * F[4] - F[1] * F[3];
}

template <typename T>
__device__ __forceinline__ void corner_b(const TetRec<T>& r, int c, T (&b)[3]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const T r0 = r.B[j], r1 = r.B[3 + j], r2 = r.B[6 + j];
    b[j] = c == 0 ? -(r0 + r1 + r2) : (c == 1 ? r0 : (c == 2 ? r1 : r2));
  }
}

// Gather of vertex v over its incident tets, each F_e formed from the tet record and the
// displacements of its corners (used outside the sweep, where no element pass ran):
//   g  += V_e P(F_e) b_c                      (elastic gradient, P = mu F + s cof F)
//   H  += V_e (mu |b_c|^2 I + lam' G G^T)     (diagonal 3x3 block; G = cof(F) b_c. The
//         det-Hessian term of dP/dF contributes nothing to a diagonal block because
//         eps_jln b_j b_l = 0, so this block is exact and positive definite.)
//   Fs += V_e F_e,  W += V_e
template <typename T>
__device__ __forceinline__ void gather_vertex_rec(const DevMesh<T>& m, int v, T (&g)[3], T (&H)[6],
                                              T (&Fs)[9], T& W) {
  const int slice = v / kSlice, lane = v % kSlice;
  const int base = m.inc_off[slice] + lane;
  const int n = m.inc_len[v];
#pragma unroll
  for (int q = 0; q < 3; ++q) g[q] = T(0);
#pragma unroll
  for (int q = 0; q < 6; ++q) H[q] = T(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) Fs[q] = T(0);
  W = T(0);
  for (int j = 0; j < n; ++j) {
    const int ent = __ldg(m.inc + base + j * kSlice);
    const int t = ent >> 2, c = ent & 3;
    const TetRec<T> r = m.tets[t];
    T F[9], C[9], b[3];
    tet_F(r, m.u, F);
    cofactor(F, C);
    const T J = F[0] * C[0] + F[1] * C[1] + F[2] * C[2];
    const T s = r.lp * (J - T(1)) - r.mu;
    corner_b(r, c, b);
    T Fb[3], G[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Fb[i] = F[3 * i] * b[0] + F[3 * i + 1] * b[1] + F[3 * i + 2] * b[2];
      G[i] = C[3 * i] * b[0] + C[3 * i + 1] * b[1] + C[3 * i + 2] * b[2];
    }
    const T vm = r.vol * r.mu, vl = r.vol * r.lp, vs = r.vol * s;
    const T bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) g[i] += vm * Fb[i] + vs * G[i];
    H[0] += vm * bb + vl * G[0] * G[0];
    H[1] += vl * G[0] * G[1];
    H[2] += vl * G[0] * G[2];
    H[3] += vm * bb + vl * G[1] * G[1];
    H[4] += vl * G[1] * G[2];
    H[5] += vm * bb + vl * G[2] * G[2];
#pragma unroll
    for (int q = 0; q < 9; ++q) Fs[q] += r.vol * F[q];
    W += r.vol;
  }
}

// Gather of vertex v over its incident tets (Sec. 3 energy; Sec. 4.3 vertex rotation),
// from the element pass's F_e (FRec, three 16-byte loads) and the corner vector b_c (one);
// incv points at the vertex's first incidence entry (entry j at incv[32 j], in the block's
// shared-memory copy of its slices):
//   g  += V_e P(F_e) b_c                      (elastic gradient, P = mu F + s cof F)
//   H  += V_e (mu |b_c|^2 I + lam' G G^T)     (diagonal 3x3 block; G = cof(F) b_c. The
//         det-Hessian term of dP/dF contributes nothing to a diagonal block because
//         eps_jln b_j b_l = 0, so this block is exact and positive definite.)
//   Fs += V_e F_e,  W += V_e
// With TPV > 1 lanes per vertex, lane q of the vertex's group takes incidences q, q + TPV,
// ... and the group's partial sums are added by the caller.
template <typename T, int TPV = 1>
__device__ __forceinline__ void gather_vertex(const DevMesh<T>& m, int v, const int* __restrict__ incv, T (&g)[3],
                                              T (&H)[6], T (&Fs)[9], T& W, int q0 = 0) {
  const int n = m.inc_len[v];
#pragma unroll
  for (int q = 0; q < 3; ++q) g[q] = T(0);
#pragma unroll
  for (int q = 0; q < 6; ++q) H[q] = T(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) Fs[q] = T(0);
  W = T(0);
  // four incidences per trip (two with lanes sharing the vertex): their record loads are
  // in flight together
#pragma unroll(TPV == 1 ? 4 : 2)
  for (int j = q0; j < n; j += TPV) {
    const int ent = incv[j * kSlice];
    const int t = ent >> 2, c = ent & 3;
    const FRec<T> r = m.frec[t];
    const Vec4<T> bq = m.bc[4 * (size_t)t + c];
    const T b[3] = {bq.x, bq.y, bq.z};
    const T vol = bq.w;
    T C[9];
    cofactor(r.F, C);
    const T s = r.lp * r.jm1 - r.mu;
    T Fb[3], G[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Fb[i] = r.F[3 * i] * b[0] + r.F[3 * i + 1] * b[1] + r.F[3 * i + 2] * b[2];
      G[i] = C[3 * i] * b[0] + C[3 * i + 1] * b[1] + C[3 * i + 2] * b[2];
    }
    const T vm = vol * r.mu, vl = vol * r.lp, vs = vol * s;
    const T bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) g[i] += vm * Fb[i] + vs * G[i];
    H[0] += vm * bb + vl * G[0] * G[0];
    H[1] += vl * G[0] * G[1];
    H[2] += vl * G[0] * G[2];
    H[3] += vm * bb + vl * G[1] * G[1];
    H[4] += vl * G[1] * G[2];
    H[5] += vm * bb + vl * G[2] * G[2];
#pragma unroll
    for (int q = 0; q < 9; ++q) Fs[q] += vol * r.F[q];
    W += vol;
  }
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (Golub & Van Loan 8.5);
// A packed (a00 a01 a02 a11 a12 a22), eigenvectors are the columns of V (row-major).
template <typename T>
__device__ void sym3_eig(T (&A)[6], T (&V)[9]) {
  T a[3][3] = {{A[0], A[1], A[2]}, {A[1], A[3], A[4]}, {A[2], A[4], A[5]}};
#pragma unroll
  for (int q = 0; q < 9; ++q) V[q] = (q % 4 == 0) ? T(1) : T(0);
  const T eps = sizeof(T) == 4 ? T(1e-7) : T(1e-16);
  for (int sweep = 0; sweep < 30; ++sweep) {
    T off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    T dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off <= eps * eps * dia || off == T(0)) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const T apq = a[p][q];
      if (apq == T(0)) continue;
      const T tau = (a[q][q] - a[p][p]) / (T(2) * apq);
      const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + dsqrt(T(1) + tau * tau));
      const T c = T(1) / dsqrt(T(1) + t * t), s = t * c;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T akp = a[k][p], akq = a[k][q];
        a[k][p] = c * akp - s * akq;
        a[k][q] = s * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T apk = a[p][k], aqk = a[q][k];
        a[p][k] = c * apk - s * aqk;
        a[q][k] = s * apk + c * aqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T vkp = V[3 * k + p], vkq = V[3 * k + q];
        V[3 * k + p] = c * vkp - s * vkq;
        V[3 * k + q] = s * vkp + c * vkq;
      }
    }
  }
  A[0] = a[0][0];
  A[3] = a[1][1];
  A[5] = a[2][2];
}

// Rotation closest to F with det +1 (reading R5): F^T F = V S^2 V^T; u_k = F v_k / s_k
// for the two largest s_k, u_3 = u_1 x u_2, det V forced to +1, R = U V^T. When det F < 0
// this flips the smallest singular value, as the SVD-based polar with a sign fix does.
template <typename T>
__device__ void polar_rotation(const T (&F)[9], T (&R)[9]) {
  T S[6];
  S[0] = F[0] * F[0] + F[3] * F[3] + F[6] * F[6];
  S[1] = F[0] * F[1] + F[3] * F[4] + F[6] * F[7];
  S[2] = F[0] * F[2] + F[3] * F[5] + F[6] * F[8];
  S[3] = F[1] * F[1] + F[4] * F[4] + F[7] * F[7];
  S[4] = F[1] * F[2] + F[4] * F[5] + F[7] * F[8];
  S[5] = F[2] * F[2] + F[5] * F[5] + F[8] * F[8];
  T V[9];
  sym3_eig(S, V);
  T ev[3] = {S[0], S[3], S[5]};
  int o[3] = {0, 1, 2};
  // sort eigenvalues descending
  if (ev[o[0]] < ev[o[1]]) { int t = o[0]; o[0] = o[1]; o[1] = t; }
  if (ev[o[1]] < ev[o[2]]) { int t = o[1]; o[1] = o[2]; o[2] = t; }
  if (ev[o[0]] < ev[o[1]]) { int t = o[0]; o[0] = o[1]; o[1] = t; }
  T v1[3], v2[3], v3[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    v1[k] = V[3 * k + o[0]];
    v2[k] = V[3 * k + o[1]];
    v3[k] = V[3 * k + o[2]];
  }
  // det V = +1
  const T dv = v1[0] * (v2[1] * v3[2] - v2[2] * v3[1]) - v1[1] * (v2[0] * v3[2] - v2[2] * v3[0]) +
               v1[2] * (v2[0] * v3[1] - v2[1] * v3[0]);
  if (dv < T(0)) {
#pragma unroll
    for (int k = 0; k < 3; ++k) v3[k] = -v3[k];
  }
  T u1[3], u2[3], u3[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    u1[i] = F[3 * i] * v1[0] + F[3 * i + 1] * v1[1] + F[3 * i + 2] * v1[2];
    u2[i] = F[3 * i] * v2[0] + F[3 * i + 1] * v2[1] + F[3 * i + 2] * v2[2];
  }
  T n1 = dsqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
  if (!(n1 > T(0))) {
#pragma unroll
    for (int q = 0; q < 9; ++q) R[q] = (q % 4 == 0) ? T(1) : T(0);
    return;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) u1[i] /= n1;
  const T d12 = u1[0] * u2[0] + u1[1] * u2[1] + u1[2] * u2[2];
#pragma unroll
  for (int i = 0; i < 3; ++i) u2[i] -= d12 * u1[i];
  T n2 = dsqrt(u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
  if (!(n2 > T(1e-30) * n1)) {
    // rank-1 F: any unit vector orthogonal to u1
    T a[3] = {T(1), T(0), T(0)};
    if (fabs(u1[0]) > T(0.9)) { a[0] = T(0); a[1] = T(1); }
    const T d = a[0] * u1[0] + a[1] * u1[1] + a[2] * u1[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) u2[i] = a[i] - d * u1[i];
    n2 = dsqrt(u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) u2[i] /= n2;
  u3[0] = u1[1] * u2[2] - u1[2] * u2[1];
  u3[1] = u1[2] * u2[0] - u1[0] * u2[2];
  u3[2] = u1[0] * u2[1] - u1[1] * u2[0];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) R[3 * i + j] = u1[i] * v1[j] + u2[i] * v2[j] + u3[i] * v3[j];
}

// Pool row layout of a symmetric 12x12 (corner blocks): the 3x3 blocks (a, c), a <= c, of
// corners a and c, in row order (0,0) (0,1) (0,2) (0,3) (1,1) (1,2) (1,3) (2,2) (2,3) (3,3),
// each row-major. Block b of corner pair (a, c): 4a - a(a-1)/2 + (c - a).
__host__ __device__ constexpr int pool_block(int a, int c) { return 4 * a - (a * (a - 1)) / 2 + (c - a); }
__host__ __device__ constexpr int pool_block_row(int b) { return b < 4 ? 0 : (b < 7 ? 1 : (b < 9 ? 2 : 3)); }
__host__ __device__ constexpr int pool_block_col(int b) {
  return pool_block_row(b) + (b - pool_block(pool_block_row(b), pool_block_row(b)));
}
// Index of entry (r, c) of the symmetric 12x12 in the pool row.
__host__ __device__ constexpr int pool_idx(int r, int c) {
  return (r / 3) <= (c / 3) ? 9 * pool_block(r / 3, c / 3) + 3 * (r % 3) + (c % 3)
                            : 9 * pool_block(c / 3, r / 3) + 3 * (c % 3) + (r % 3);
}

// One entry q of a streamed pool row (indices fixed at compile time). Block (a, c) entries
// accumulate P = H'_ac U_c (3x3); its last entry closes the block: Q = U_a^T P and
// H~' += w (Q + Q^T) (w Q for a diagonal block, which is symmetric). Gradient entries:
// g~' += w U^T G.
template <int Q, typename T>
__device__ __forceinline__ void pool_entry(T h, T w, const T (&U)[36], T (&P)[9], T (&Ht)[6], T (&gt)[3]) {
  if constexpr (Q < kPoolH) {
    constexpr int b = Q / 9, e = Q % 9, i = e / 3, j = e % 3;
    constexpr int a = pool_block_row(b), c = pool_block_col(b);
    if constexpr (e == 0) {
#pragma unroll
      for (int q = 0; q < 9; ++q) P[q] = T(0);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) P[3 * i + k] += h * U[3 * (3 * c + j) + k];
    if constexpr (e == 8) {
      T Qm[9];
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          Qm[3 * l + k] = U[3 * (3 * a) + l] * P[k] + U[3 * (3 * a + 1) + l] * P[3 + k] +
                          U[3 * (3 * a + 2) + l] * P[6 + k];
      if constexpr (a == c) {
        Ht[0] += w * Qm[0];
        Ht[1] += w * Qm[1];
        Ht[2] += w * Qm[2];
        Ht[3] += w * Qm[4];
        Ht[4] += w * Qm[5];
        Ht[5] += w * Qm[8];
      } else {
        Ht[0] += w * (Qm[0] + Qm[0]);
        Ht[1] += w * (Qm[1] + Qm[3]);
        Ht[2] += w * (Qm[2] + Qm[6]);
        Ht[3] += w * (Qm[4] + Qm[4]);
        Ht[4] += w * (Qm[5] + Qm[7]);
        Ht[5] += w * (Qm[8] + Qm[8]);
      }
    }
  } else if constexpr (Q < kPoolH + 12) {
    constexpr int r = Q - kPoolH;
    const T wg = w * h;
#pragma unroll
    for (int k = 0; k < 3; ++k) gt[k] += wg * U[3 * r + k];
  }
}

template <typename T>
__device__ __forceinline__ void load4(const T* __restrict__ p, T (&o)[4]);
template <typename T>
__device__ __forceinline__ void load4_coherent(const T* p, T (&o)[4]);

// NC = false: the pool rows were written earlier in the same (persistent) launch, so they
// are read with plain coherent loads instead of the read-only path.
template <int Q4, bool NC, typename T>
__device__ __forceinline__ void pool_chunk(const T* Hp, T w, const T (&U)[36], T (&P)[9], T (&Ht)[6],
                                           T (&gt)[3]) {
  T hv[4];
  if constexpr (NC)
    load4(Hp + 4 * Q4, hv);
  else
    load4_coherent(Hp + 4 * Q4, hv);
  pool_entry<4 * Q4 + 0>(hv[0], w, U, P, Ht, gt);
  pool_entry<4 * Q4 + 1>(hv[1], w, U, P, Ht, gt);
  pool_entry<4 * Q4 + 2>(hv[2], w, U, P, Ht, gt);
  pool_entry<4 * Q4 + 3>(hv[3], w, U, P, Ht, gt);
}

template <bool NC, typename T, int... Q4>
__device__ __forceinline__ void pool_row(const T* Hp, T w, const T (&U)[36], T (&P)[9], T (&Ht)[6], T (&gt)[3],
                                         std::integer_sequence<int, Q4...>) {
  (pool_chunk<Q4, NC>(Hp, w, U, P, Ht, gt), ...);
}

// FP32 pool rows in 32-byte pieces: one 256-bit load per lane and instruction (sm_100 and
// later), so a warp's request uses every byte of the 32-byte sectors it touches (a 16-byte
// load per lane uses half of each). Rows are 416 bytes, and the pool array comes from
// cudaMalloc, so every row starts on a 32-byte boundary. NC as in pool_chunk.
static_assert(kPoolStride * sizeof(float) % 32 == 0, "FP32 pool rows must keep 32-byte alignment");
template <bool NC>
__device__ __forceinline__ void load8f(const float* p, float (&o)[8]) {
  if constexpr (NC)
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]), "=f"(o[7])
        : "l"(p));
  else
    asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]), "=f"(o[7])
                 : "l"(p));
}
template <int Q8, bool NC>
__device__ __forceinline__ void pool_chunk8(const float* Hp, float w, const float (&U)[36], float (&P)[9],
                                            float (&Ht)[6], float (&gt)[3]) {
  float hv[8];
  load8f<NC>(Hp + 8 * Q8, hv);
  pool_entry<8 * Q8 + 0>(hv[0], w, U, P, Ht, gt);
  pool_entry<8 * Q8 + 1>(hv[1], w, U, P, Ht, gt);
  pool_entry<8 * Q8 + 2>(hv[2], w, U, P, Ht, gt);
  pool_entry<8 * Q8 + 3>(hv[3], w, U, P, Ht, gt);
  pool_entry<8 * Q8 + 4>(hv[4], w, U, P, Ht, gt);
  pool_entry<8 * Q8 + 5>(hv[5], w, U, P, Ht, gt);
  pool_entry<8 * Q8 + 6>(hv[6], w, U, P, Ht, gt);
  pool_entry<8 * Q8 + 7>(hv[7], w, U, P, Ht, gt);
}
template <bool NC, int... Q8>
__device__ __forceinline__ void pool_row8(const float* Hp, float w, const float (&U)[36], float (&P)[9],
                                          float (&Ht)[6], float (&gt)[3], std::integer_sequence<int, Q8...>) {
  (pool_chunk8<Q8, NC>(Hp, w, U, P, Ht, gt), ...);
}

// One cubature slot of Eq. cubature: the pool row Hp (rotated element Hessian blocks, then
// the rotated corner gradients) against the slot's weight w and U_bar rows U (12x3):
// H~' += w U^T H' U = w sum_{a <= c} (U_a^T H'_ac U_c + its transpose if a != c),
// g~' += w U^T G'. Blocks are closed one at a time, so only a 3x3 partial product is
// live besides U.
template <typename T, bool NC = true>
__device__ __forceinline__ void slot_sums(const T* Hp, T w, const T (&U)[36], T (&Ht)[6], T (&gt)[3]) {
  T P[9];
  if constexpr (sizeof(T) == 4)
    pool_row8<NC>(Hp, w, U, P, Ht, gt, std::make_integer_sequence<int, (kPoolH + 12 + 7) / 8>{});
  else
    pool_row<NC>(Hp, w, U, P, Ht, gt, std::make_integer_sequence<int, (kPoolH + 12 + 3) / 4>{});
}

// Cubature sums for vertex i over its n_cub slots, records read directly from global memory.
// Fixed slot count: every slot's pool index and weight are loaded first, so the pool rows'
// addresses are known before the first slot's work starts.
template <typename T, bool NC, int NCUB>
__device__ __forceinline__ void cubature_sums_n(const DevMesh<T>& m, int i, T (&Ht)[6], T (&gt)[3]) {
  int ps[NCUB];
  T ws[NCUB];
#pragma unroll
  for (int s = 0; s < NCUB; ++s) {
    ps[s] = m.cub_p[(size_t)s * m.cs + i];
    ws[s] = m.cub_w[(size_t)s * m.cs + i];
  }
#pragma unroll
  for (int s = 0; s < NCUB; ++s) {
    if (ps[s] < 0) continue;
    T U[36];
    const T* up = m.cub_u + (size_t)s * 36 * m.cs + i;
#pragma unroll
    for (int q = 0; q < 36; ++q) U[q] = up[(size_t)q * m.cs];
    slot_sums<T, NC>(m.pool_H + (size_t)ps[s] * kPoolStride, ws[s], U, Ht, gt);
  }
}

// PF: with four slots, take the prefetching form above (the autotuner picks per mesh).
template <typename T, bool NC = true, bool PF = false>
__device__ __forceinline__ void cubature_sums(const DevMesh<T>& m, int i, T (&Ht)[6], T (&gt)[3]) {
  if (PF && m.n_cub == 4) {
    cubature_sums_n<T, NC, 4>(m, i, Ht, gt);
    return;
  }
  for (int s = 0; s < m.n_cub; ++s) {
    const int p = m.cub_p[(size_t)s * m.cs + i];
    if (p < 0) continue;
    const T w = m.cub_w[(size_t)s * m.cs + i];
    T U[36];
    const T* up = m.cub_u + (size_t)s * 36 * m.cs + i;
#pragma unroll
    for (int q = 0; q < 36; ++q) U[q] = up[(size_t)q * m.cs];
    slot_sums<T, NC>(m.pool_H + (size_t)p * kPoolStride, w, U, Ht, gt);
  }
}

// Four consecutive values from a 16-byte aligned address through the read-only path (one
// 16-byte load in FP32, two in FP64).
template <>
__device__ __forceinline__ void load4<float>(const float* __restrict__ p, float (&o)[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
template <>
__device__ __forceinline__ void load4<double>(const double* __restrict__ p, double (&o)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  o[0] = a.x;
  o[1] = a.y;
  o[2] = b.x;
  o[3] = b.y;
}
// The same four values through plain (coherent, L1-cached) global loads.
template <>
__device__ __forceinline__ void load4_coherent<float>(const float* p, float (&o)[4]) {
  asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3])
               : "l"(p));
}
template <>
__device__ __forceinline__ void load4_coherent<double>(const double* p, double (&o)[4]) {
  asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(o[0]), "=d"(o[1]) : "l"(p));
  asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(o[2]), "=d"(o[3]) : "l"(p + 2));
}

// Step truncation: scale d so that |d| <= lim (reading R11).
template <typename T>
__device__ __forceinline__ void truncate3(T (&d)[3], T lim) {
  const T n = dsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (n > lim) {
    const T s = lim / n;
    d[0] *= s;
    d[1] *= s;
    d[2] *= s;
  }
}

// 3x3 SPD solve by Cholesky; returns false if a pivot is not positive.
template <typename T>
__device__ __forceinline__ bool chol3_solve(const T (&A)[6], const T (&b)[3], T (&x)[3]) {
  const T l00s = A[0];
  if (!(l00s > T(0))) return false;
  const T l00 = dsqrt(l00s);
  const T l10 = A[1] / l00, l20 = A[2] / l00;
  const T l11s = A[3] - l10 * l10;
  if (!(l11s > T(0))) return false;
  const T l11 = dsqrt(l11s);
  const T l21 = (A[4] - l20 * l10) / l11;
  const T l22s = A[5] - l20 * l20 - l21 * l21;
  if (!(l22s > T(0))) return false;
  const T l22 = dsqrt(l22s);
  const T y0 = b[0] / l00;
  const T y1 = (b[1] - l10 * y0) / l11;
  const T y2 = (b[2] - l20 * y0 - l21 * y1) / l22;
  x[2] = y2 / l22;
  x[1] = (y1 - l21 * x[2]) / l11;
  x[0] = (y0 - l10 * x[1] - l20 * x[2]) / l00;
  return true;
}

// ------------------------------------------------------------------ kernels

// Step setup: caller-order FP64 state -> internal order; u = x^0 - x_t = 0 (reading R8:
// x^0 = x_t), dz = h v_t + h^2 g for free vertices.
template <typename T>
__global__ void k_setup_vertices(DevMesh<T> m, const double* __restrict__ x_caller,
                                 const double* __restrict__ v_caller,
                                 const double* __restrict__ xk_caller) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= m.V) return;
  const int c = m.perm[v];
  double x[3], vel[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    x[q] = x_caller[3 * c + q];
    vel[q] = v < m.Vf ? v_caller[3 * c + q] : 0.0;
    m.xt[3 * v + q] = x[q];
    m.vt[3 * v + q] = vel[q];
  }
  Vec4<T> u0{T(0), T(0), T(0), T(0)};
  if (xk_caller != nullptr && v < m.Vf) {
    u0.x = T(xk_caller[3 * c] - x[0]);
    u0.y = T(xk_caller[3 * c + 1] - x[1]);
    u0.z = T(xk_caller[3 * c + 2] - x[2]);
  }
  m.u[v] = u0;
  if (v < m.Vf) {
    Vec4<T> d;
    d.x = T(m.h * vel[0] + m.h * m.h * m.grav[0]);
    d.y = T(m.h * vel[1] + m.h * m.h * m.grav[1]);
    d.z = T(m.h * vel[2] + m.h * m.h * m.grav[2]);
    d.w = T(0);
    m.dz[v] = d;
  }
  if (m.c.fr_lam) {
    // friction lagged at the step start: the normal force of each wall within dhat of a free
    // surface vertex, -kappa E'(d(x_t)) (zero elsewhere)
    for (int p = 0; p < m.c.n_planes; ++p) {
      double lam = 0.0;
      if (v < m.Vf && m.c.is_surf[v]) {
        const double* pl = m.c.planes + 4 * p;
        const double d = pl[0] * x[0] + pl[1] * x[1] + pl[2] * x[2] - pl[3];
        if (d > 0.0 && d < m.c.dhat) lam = -m.c.kappa * barrier_b1(d, m.c.dhat, m.c.pen);
      }
      m.c.fr_lam[(size_t)p * m.V + v] = lam;
    }
  }
}

// F(x_t) per tet in FP64 from the FP64 step-start positions (no cancellation in FP32).
template <typename T>
__global__ void k_setup_tets(DevMesh<T> m) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.T_) return;
  TetRec<T>& r = m.tets_mut[t];
  double x0[3], D[9], Fd[9];
#pragma unroll
  for (int q = 0; q < 3; ++q) x0[q] = m.xt[3 * r.v[0] + q];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) D[3 * i + k] = m.xt[3 * r.v[k + 1] + i] - x0[i];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double f = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) f += D[3 * i + k] * double(r.B[3 * k + j]);
      Fd[3 * i + j] = f;
      r.Ft[3 * i + j] = T(f);
    }
  {
    double Cd[9];
    cofactor(Fd, Cd);
    r.jt1 = T((Fd[0] * Cd[0] + Fd[1] * Cd[1] + Fd[2] * Cd[2]) - 1.0);
  }
  // corner vectors of the gather (the same values corner_b forms from the record), with
  // the element volume in the fourth entry
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    T b[3];
    corner_b(r, c, b);
    m.bc[4 * (size_t)t + c] = Vec4<T>{b[0], b[1], b[2], r.vol};
  }
}

// Element pass of a sweep (Sec. 3 energy terms, computed once per tet): F_e(x^k) =
// F(x_t) + [u_1 - u_0, u_2 - u_0, u_3 - u_0] B with the tet's constants, for the vertex
// gather. Tiles of 128 records are staged in shared memory with coalesced loads; each
// thread writes one 16-byte aligned FRec. Batch meshes skip the tets of finished scenes.
// One tile of 128 tets: block bid of nb (srec: the block's 128-record staging buffer).
template <typename T, bool BATCH>
__device__ __forceinline__ void elem_body(const DevMesh<T>& m, int bid, int nb, TetRec<T>* srec) {
  // tiles in descending order: the lowest tets, which the gather (ascending vertices)
  // reads first, are written last and are still in L2 when it starts
  const int t0 = (nb - 1 - bid) * 128, n = min(128, m.T_ - t0);
  stage_tets<T, 128>(m.tets, t0, n, srec);
  __syncthreads();
  if ((int)threadIdx.x >= n) return;
  const int t = t0 + threadIdx.x;
  if (BATCH && m.scenes[m.t_scene[t]].done) return;
  const TetRec<T>& r = srec[threadIdx.x];
  FRec<T> o;
  tet_F_jm1(r, m.u, o.F, o.jm1);
  o.mu = r.mu;
  o.lp = r.lp;
  m.frec[t] = o;
}

template <typename T, bool BATCH>
__global__ void __launch_bounds__(128) k_elem(DevMesh<T> m, const StepState* __restrict__ st) {
  if (!BATCH && st->done) return;
  __shared__ __align__(16) TetRec<T> srec[128];
  elem_body<T, BATCH>(m, blockIdx.x, gridDim.x, srec);
}

// Per cubature element, one warp (kPoolWarps elements per block), after the sweep's gather:
// lanes 0-3 take corner a's assembled gradient g_a and rotation R_a from the gather's
// hand-off (identity and zero at pinned corners), then the lanes form dP/dF (81 entries)
// and the 90 outputs: the element Hessian of E_hat_e = V_e Psi(F_e) + sum_a
// m_e/(2h^2)|x_a - z_a|^2 at x^k rotated into the rest frames of its corners (packed, 78)
// and the rotated corner gradients (12).
// ASM = true: corner gradients are the assembled g_a (reading R3 "asm");
// ASM = false: the element's own gradient of E_hat_e (literal Eq. cubature, "elem").
constexpr int kPoolWarps = 4;

template <typename T>
struct PoolShared {
  T R[4][9], g[4][3], b[4][3], A[81];
};

template <typename T, bool ASM>
__device__ __forceinline__ void pool_body(const DevMesh<T>& m, int bid) {
  __shared__ PoolShared<T> sh_all[kPoolWarps];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = bid * kPoolWarps + wid;
  if (p >= m.nP) return;  // whole warps only; no block-wide barrier below
  PoolShared<T>& sh = sh_all[wid];
  const int t = m.pool_tet[p];
  const TetRec<T>& rec = m.tets[t];  // read in place (global, cached)
  if (lane < 4) {
    const int v = rec.v[lane];
    T R[9], g[3];
    if (v < m.Vf) {
      const T* o = m.ghr + v;
      const size_t S = m.Vf;
#pragma unroll
      for (int i = 0; i < 3; ++i) g[i] = o[i * S];
#pragma unroll
      for (int q = 0; q < 9; ++q) R[q] = o[(9 + q) * S];
    } else {
#pragma unroll
      for (int q = 0; q < 9; ++q) R[q] = (q % 4 == 0) ? T(1) : T(0);
#pragma unroll
      for (int i = 0; i < 3; ++i) g[i] = T(0);
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) sh.R[lane][q] = R[q];
#pragma unroll
    for (int i = 0; i < 3; ++i) sh.g[lane][i] = g[i];
    const Vec4<T> bq = m.bc[4 * (size_t)t + lane];
    sh.b[lane][0] = bq.x;
    sh.b[lane][1] = bq.y;
    sh.b[lane][2] = bq.z;
    if (m.pool_R != nullptr) {
#pragma unroll
      for (int q = 0; q < 9; ++q) m.pool_R[(size_t)p * 36 + 9 * lane + q] = R[q];
    }
  }
  // element quantities at x^k (every lane), dP/dF = mu I + lam' c c^T + s d2J/dF2 (9x9,
  // index 3i+j), c = vec(cof F); d2J/dF_ij dF_kl = eps_ikm eps_jln F_mn (i != k, j != l)
  T F[9], C[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) F[q] = m.frec[t].F[q];
  cofactor(F, C);
  const T mu = rec.mu, lp = rec.lp, vol = rec.vol;
  const T ss = lp * m.frec[t].jm1 - mu;
  for (int e = lane; e < 81; e += 32) {
    const int row = e / 9, col = e % 9;
    const int i = row / 3, j = row % 3, k = col / 3, l = col % 3;
    T v = lp * C[row] * C[col] + (row == col ? mu : T(0));
    if (i != k && j != l) {
      const int mm = 3 - i - k, n = 3 - j - l;
      const T sik = ((k - i + 3) % 3 == 1) ? T(1) : T(-1);
      const T sjl = ((l - j + 3) % 3 == 1) ? T(1) : T(-1);
      v += ss * sik * sjl * F[3 * mm + n];
    }
    sh.A[e] = v;
  }
  __syncwarp();
  const T mi = rec.mq * T(m.inv_h2);
  T* Hrow = m.pool_H + (size_t)p * kPoolStride;
  for (int e = lane; e < kPoolH + 12; e += 32) {
    if (e < kPoolH) {
      // entry (jj, ll) of block (a, cc), a <= cc, of H' = blockdiag(R)^T H_e blockdiag(R),
      // with H_e[(a,i),(c,k)] = V sum_{j,l} b_a[j] A[(i,j),(k,l)] b_c[l] + m_e/h^2 delta
      const int blk = e / 9, q = e % 9;
      const int a = pool_block_row(blk), cc = pool_block_col(blk), jj = q / 3, ll = q % 3;
      T Hac[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          T acc = T(0);
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            T row = T(0);
#pragma unroll
            for (int l = 0; l < 3; ++l) row += sh.A[9 * (3 * i + j) + 3 * k + l] * sh.b[cc][l];
            acc += sh.b[a][j] * row;
          }
          Hac[3 * i + k] = vol * acc + ((a == cc && i == k) ? mi : T(0));
        }
      T v = T(0);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) v += sh.R[a][3 * i + jj] * Hac[3 * i + k] * sh.R[cc][3 * k + ll];
      Hrow[e] = v;
    } else {
      // rotated corner gradient entry (a, j)
      const int q = e - kPoolH, a = q / 3, j = q % 3;
      T ga[3];
      if (ASM) {
#pragma unroll
        for (int i = 0; i < 3; ++i) ga[i] = sh.g[a][i];
      } else {
        const int v = rec.v[a];
        if (v < m.Vf) {
          T uv[3], dz[3];
          load3(m.u, v, uv);
          load3(m.dz, v, dz);
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const T Pb = (mu * F[3 * i] + ss * C[3 * i]) * sh.b[a][0] + (mu * F[3 * i + 1] + ss * C[3 * i + 1]) * sh.b[a][1] +
                         (mu * F[3 * i + 2] + ss * C[3 * i + 2]) * sh.b[a][2];
            ga[i] = vol * Pb + mi * (uv[i] - dz[i]);
          }
        } else {
          ga[0] = ga[1] = ga[2] = T(0);
        }
      }
      Hrow[e] = sh.R[a][j] * ga[0] + sh.R[a][3 + j] * ga[1] + sh.R[a][6 + j] * ga[2];
    }
  }
}

template <typename T, bool ASM>
__global__ void __launch_bounds__(32 * kPoolWarps) k_pool(DevMesh<T> m, const StepState* __restrict__ st) {
  if (st->done) return;
  pool_body<T, ASM>(m, blockIdx.x);
}

// Residual bookkeeping of sweep k (reading R9), run by one thread of the last block.
// dd2, ddj2: |D|^2 and |D_J|^2 of the sweep's directions. Besides r_k <= rel_tol, a step
// with the position-change test on (dx2_tol > 0) stops at the first k >= 1 whose last
// update moved the free vertices by |x^k - x^{k-1}|^2 <= dx2_tol (Sec. 8).
__device__ __forceinline__ void finalize_sweep(StepState* st, double r2, double gd, double gdj, double dd2,
                                               double ddj2, double* trace, int record) {
  st->ticket_main = 0;
  if (st->gs_ncol > 0) {
    // Gauss-Seidel step: a GS sweep is gs_ncol colour passes; the stopping test (on the
    // full gradient, which the gather forms for every vertex) is taken at the first
    const int pass = st->pass;
    st->pass = pass + 1;
    if (pass % st->gs_ncol != 0) {
      st->slope = gd;
      st->slope_j = gdj;
      st->alpha = 1.0;
      st->dir = 0;
      st->need_j = 0;
      st->ls_mode = st->prev_dir;
      st->dd2 = dd2;
      st->ddj2 = ddj2;
      st->dx2 = dd2;
      if (!isfinite(gd) || !isfinite(gdj) || !isfinite(r2)) {
        st->status = 6;  // JGS2_EDIVERGED
        st->done = 1;
        st->sweeps = st->k;
      }
      return;
    }
  }
  const int k = st->k;
  const double gn = sqrt(r2);
  if (k == 0) st->g0 = gn;
  const double g0 = st->g0;
  const double r = g0 > 0.0 ? gn / g0 : 0.0;
  st->r = r;
  st->slope = gd;
  st->slope_j = gdj;
  st->alpha = 1.0;
  st->dir = 0;
  st->need_j = 0;
  st->ls_mode = st->prev_dir;
  const double dx2_last = st->dx2;
  st->dx2_applied = k >= 1 ? dx2_last : 0.0;
  st->dd2 = dd2;
  st->ddj2 = ddj2;
  st->dx2 = dd2;  // the update without line search (alpha 1 along D); k_ls_decide overrides
  if (record && k < 4096) trace[k] = r;
  if (!isfinite(r) || !isfinite(gd) || !isfinite(gdj)) {
    st->status = 6;  // JGS2_EDIVERGED
    st->done = 1;
    st->sweeps = k;
  } else if (r <= st->rel_tol || g0 == 0.0) {
    st->converged = 1;
    st->done = 1;
    st->sweeps = k;
  } else if (k >= 1 && st->dx2_tol > 0.0 && dx2_last <= st->dx2_tol) {
    st->stopped_dx = 1;
    st->done = 1;
    st->sweeps = k;
  } else if (k >= st->max_sweeps) {
    st->done = 1;
    st->sweeps = k;
  } else {
    st->k = k + 1;
  }
}

// Sweep phase 1, thread per free vertex (dynamic shared memory: the block's incidence
// entries, inc_block_bytes of the launch's block size): gather g_i and H_ii (+ inertia)
// over the incident tets (Eq. reduced_local terms), the uncorrected direction D_J = -H_ii^{-1} g_i, and, with
// the correction on, R_i = polar(F_i) (Eq. tilde_phi). Writes g, H, R as [18][Vf] for
// phase 2 and the FP64 partial sums |g|^2 and g.D_J. Without the correction D = D_J and
// this kernel closes the sweep's reduction.
// TPV threads per vertex (1 or 4; BS / TPV vertices per block, a whole number of 32-vertex
// slices): with 4, the lanes of a vertex's group split its incidences and add their sums
// with warp shuffles, so more record loads are in flight per vertex; every lane of the group
// then holds the vertex's sums and lane 0 writes its results.
template <typename T, bool CORR, bool BATCH, int BS, int TPV>
__device__ __forceinline__ void gather_body(const DevMesh<T>& m, StepState* st, double* __restrict__ partial,
                                            double* __restrict__ trace, int record, int bid, int nb) {
  static_assert(TPV == 1 || TPV == 4, "1 or 4 threads per vertex");
  static_assert((BS / TPV) % kSlice == 0, "whole slices per block");
  constexpr int VPB = BS / TPV;
  __shared__ double red[96];
  __shared__ Acc<T> sred[96];
  // the block's incidence slices form one contiguous, 128-byte aligned range of entries;
  // copy it into shared memory first (coalesced 16-byte loads), so that each incidence's
  // record loads do not wait on a global load of its entry
  extern __shared__ __align__(16) int s_inc[];
  const int s0 = bid * (VPB / kSlice), s1 = min(s0 + VPB / kSlice, m.n_slices);
  const int e0 = m.inc_off[s0];
  {
    const int4* src = reinterpret_cast<const int4*>(m.inc + e0);
    int4* dst = reinterpret_cast<int4*>(s_inc);
    const int n4 = (m.inc_off[s1] - e0) / 4;
    for (int q = threadIdx.x; q < n4; q += BS) dst[q] = __ldg(src + q);
  }
  __syncthreads();
  const int i = bid * VPB + (int)threadIdx.x / TPV;
  const int lane_v = (int)threadIdx.x % TPV;
  Acc<T> acc[3];  // |g|^2, g.D_J, |D_J|^2
  const int sc = (BATCH && i < m.Vf) ? m.v_scene[i] : -1;
  const bool active = i < m.Vf && (!BATCH || !m.scenes[sc].done);
  T g[3], H[6], Fs[9], W;
  if (active) gather_vertex<T, TPV>(m, i, s_inc + (m.inc_off[i / kSlice] - e0) + i % kSlice, g, H, Fs, W, lane_v);
  if (TPV > 1) {
    // groups are aligned runs of TPV lanes of one warp; every lane takes part (inactive
    // lanes add zeros)
    if (!active) {
#pragma unroll
      for (int q = 0; q < 3; ++q) g[q] = T(0);
#pragma unroll
      for (int q = 0; q < 6; ++q) H[q] = T(0);
#pragma unroll
      for (int q = 0; q < 9; ++q) Fs[q] = T(0);
      W = T(0);
    }
#pragma unroll
    for (int o = 1; o < TPV; o <<= 1) {
#pragma unroll
      for (int q = 0; q < 3; ++q) g[q] += __shfl_xor_sync(0xffffffffu, g[q], o);
#pragma unroll
      for (int q = 0; q < 6; ++q) H[q] += __shfl_xor_sync(0xffffffffu, H[q], o);
#pragma unroll
      for (int q = 0; q < 9; ++q) Fs[q] += __shfl_xor_sync(0xffffffffu, Fs[q], o);
      W += __shfl_xor_sync(0xffffffffu, W, o);
    }
  }
  const bool writer = active && lane_v == 0;
  if (active) {
    T ui[3], dz[3];
    load3(m.u, i, ui);
    load3(m.dz, i, dz);
    const T mh = m.mh2[i];
#pragma unroll
    for (int q = 0; q < 3; ++q) g[q] += mh * (ui[q] - dz[q]);
    H[0] += mh;
    H[3] += mh;
    H[5] += mh;
    T lim = T(INFINITY);
    if (m.c.on) {
      // IPC barrier (Sec. 7): exact gradient and Gauss-Newton diagonal block of the pairs
      // around a surface vertex i, and its step limit 0.45 min(r_c - dhat, d_min)
      if (m.c.is_surf[i]) {
        const size_t V = m.V;
#pragma unroll
        for (int q = 0; q < 3; ++q) g[q] += T(m.c.bg[q * V + i]);
#pragma unroll
        for (int q = 0; q < 6; ++q) H[q] += T(m.c.bH[q * V + i]);
        lim = T(0.45 * fmin(m.c.rc - m.c.dhat, m.c.dmin[i]));
      }
      if (writer) m.c.lim[i] = double(lim);
    }
    T dj[3];
    {
      T rg[3] = {-g[0], -g[1], -g[2]};
      if (!chol3_solve(H, rg, dj)) dj[0] = dj[1] = dj[2] = T(0);
      truncate3(dj, lim);
      if (m.vmask && !m.vmask[i]) dj[0] = dj[1] = dj[2] = T(0);  // not this colour
    }
    Vec4<T> djv{dj[0], dj[1], dj[2], T(0)};
    if (writer) m.DJ[i] = djv;
    if (CORR) {
      T R[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) Fs[q] /= W;
      polar_rotation(Fs, R);
      if (writer) {
        T* o = m.ghr + i;
        const size_t S = m.Vf;
#pragma unroll
        for (int q = 0; q < 3; ++q) o[q * S] = g[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) o[(3 + q) * S] = H[q];
#pragma unroll
        for (int q = 0; q < 9; ++q) o[(9 + q) * S] = R[q];
      }
    } else if (writer) {
      m.D[i] = djv;
    }
    if (writer) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        acc[0].add_prod(g[q], g[q]);
        acc[1].add_prod(g[q], dj[q]);
        if (!BATCH) acc[2].add_prod(dj[q], dj[q]);
      }
    }
  }
  if (BATCH) {
    Acc<T> sacc2[2] = {acc[0], acc[1]};
    scene_reduce_acc<T, 2>(sacc2, writer ? sc : -1, m.sacc, 0);
    return;
  }
  double bs[3];
  block_sum_acc<T, 3>(acc, bs, sred);
  if (threadIdx.x == 0) {
    partial[bid] = bs[0];
    partial[nb + bid] = bs[1];
    partial[3 * nb + bid] = bs[2];
  }
  if (CORR) return;
  if (!last_block(&st->ticket_main)) return;
  const double r2 = block_sum_array(partial, nb, 1, red);
  const double gdj = block_sum_array(partial + nb, nb, 1, red);
  const double djj = block_sum_array(partial + 3 * nb, nb, 1, red);
  if (threadIdx.x == 0) finalize_sweep(st, r2, gdj, gdj, djj, djj, trace, record);
}

template <typename T, bool CORR, bool BATCH, int BS, int TPV = 1>
__global__ void __launch_bounds__(BS, (sizeof(T) == 4 ? 768 : 512) / BS)
    k_gather(DevMesh<T> m, StepState* st, double* __restrict__ partial /* [3][grid] */,
             double* __restrict__ trace, int record) {
  if (!BATCH && st->done) return;
  gather_body<T, CORR, BATCH, BS, TPV>(m, st, partial, trace, record, blockIdx.x, gridDim.x);
}

// Sweep phase 2, thread per free vertex: the cubature sums H~_i, g~_i (Eq. cubature) from
// the rotated pool element data (L2-resident rows), the 3x3 solve of Eq. reduced_local, D_i, and g.D. The
// last block closes the sweep's reduction with phase 1's partial sums.
template <typename T, bool BATCH, int BS, bool NC = true, bool PF = false>
__device__ __forceinline__ void correct_body(const DevMesh<T>& m, StepState* st, double* __restrict__ partial,
                                             double* __restrict__ trace, int record, int bid, int nb) {
  __shared__ double red[96];
  __shared__ Acc<T> sred[64];
  const int i = bid * BS + threadIdx.x;
  Acc<T> acc[2];  // g.D, |D|^2
  int fb = 0;
  const int sc = (BATCH && i < m.Vf) ? m.v_scene[i] : -1;
  const bool active = i < m.Vf && (!BATCH || !m.scenes[sc].done);
  if (active) {
    T Ht[6] = {T(0), T(0), T(0), T(0), T(0), T(0)}, gt[3] = {T(0), T(0), T(0)};
    cubature_sums<T, NC, PF>(m, i, Ht, gt);
    // the vertex's own g, H_ii, R_i from the gather (loaded after the cubature loop, so
    // they hold no registers during it)
    const T* o = m.ghr + i;
    const size_t S = m.Vf;
    T g[3], H[6], R[9];
#pragma unroll
    for (int q = 0; q < 3; ++q) g[q] = o[q * S];
#pragma unroll
    for (int q = 0; q < 6; ++q) H[q] = o[(3 + q) * S];
#pragma unroll
    for (int q = 0; q < 9; ++q) R[q] = o[(9 + q) * S];
    // contact-aware local terms (Sec. 7) replace g_i, H_ii in the local system; the slope
    // g.D below keeps the true gradient
    T gl[3] = {g[0], g[1], g[2]};
    if (m.cpl_on && m.cpl_on[i]) {
#pragma unroll
      for (int q = 0; q < 3; ++q) gl[q] = m.cpl[q * S + i];
#pragma unroll
      for (int q = 0; q < 6; ++q) H[q] = m.cpl[(3 + q) * S + i];
    }
    // back to world: H~ = R H~' R^T, g~ = R g~'
    T Hf[9] = {Ht[0], Ht[1], Ht[2], Ht[1], Ht[3], Ht[4], Ht[2], Ht[4], Ht[5]};
    T RH[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        RH[3 * a + b] = R[3 * a] * Hf[b] + R[3 * a + 1] * Hf[3 + b] + R[3 * a + 2] * Hf[6 + b];
    T Hw[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        Hw[3 * a + b] = RH[3 * a] * R[3 * b] + RH[3 * a + 1] * R[3 * b + 1] + RH[3 * a + 2] * R[3 * b + 2];
    T A[6] = {H[0] + Hw[0], H[1] + T(0.5) * (Hw[1] + Hw[3]), H[2] + T(0.5) * (Hw[2] + Hw[6]),
              H[3] + Hw[4], H[4] + T(0.5) * (Hw[5] + Hw[7]), H[5] + Hw[8]};
    T rhs[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) rhs[a] = -gl[a] - (R[3 * a] * gt[0] + R[3 * a + 1] * gt[1] + R[3 * a + 2] * gt[2]);
    T d[3];
    if (!chol3_solve(A, rhs, d)) {
      // reading R7: the vertex takes the uncorrected step (already truncated)
      load3(m.DJ, i, d);
      fb = 1;
    } else if (m.c.on) {
      truncate3(d, T(m.c.lim[i]));
    }
    if (m.vmask && !m.vmask[i]) d[0] = d[1] = d[2] = T(0);  // not this colour
    Vec4<T> dv{d[0], d[1], d[2], T(0)};
    m.D[i] = dv;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      acc[0].add_prod(g[q], d[q]);
      if (!BATCH) acc[1].add_prod(d[q], d[q]);
    }
  }
  if (BATCH) {
    if (fb) atomicAdd(&m.scenes[sc].fallback, 1);
    Acc<T> sacc1[1] = {acc[0]};
    scene_reduce_acc<T, 1>(sacc1, active ? sc : -1, m.sacc, 2);
    return;
  }
  if (__syncthreads_or(fb)) {
    const int nfb = __syncthreads_count(fb);
    if (threadIdx.x == 0) atomicAdd(&st->fallback, nfb);
  }
  double bs[2];
  block_sum_acc<T, 2>(acc, bs, sred);
  if (threadIdx.x == 0) {
    partial[2 * nb + bid] = bs[0];
    partial[4 * nb + bid] = bs[1];
  }
  if (!last_block(&st->ticket_main)) return;
  const double r2 = block_sum_array(partial, nb, 1, red);
  const double gdj = block_sum_array(partial + nb, nb, 1, red);
  const double gd = block_sum_array(partial + 2 * nb, nb, 1, red);
  const double djj = block_sum_array(partial + 3 * nb, nb, 1, red);
  const double dd = block_sum_array(partial + 4 * nb, nb, 1, red);
  if (threadIdx.x == 0) finalize_sweep(st, r2, gd, gdj, dd, djj, trace, record);
}

template <typename T, bool BATCH, int BS, bool PF = false>
__global__ void __launch_bounds__(BS, (sizeof(T) == 4 ? 768 : 256) / BS) k_correct(DevMesh<T> m, StepState* st,
                                                double* __restrict__ partial /* [3][grid] */,
                                                double* __restrict__ trace, int record) {
  if (!BATCH && st->done) return;
  correct_body<T, BATCH, BS, true, PF>(m, st, partial, trace, record, blockIdx.x, gridDim.x);
}

// Exact energy change of a tet for the displacement increment alpha*d (no cancellation):
// with G = alpha dF, det(F+G) - det F = cof(F):G + F:cof(G) + det G, and
// Psi(F+G) - Psi(F) = mu/2 (2F:G + G:G) - mu dJ + lam'/2 dJ (dJ + 2(J - 1)).
template <typename T>
__device__ __forceinline__ void tet_dF(const TetRec<T>& r, const Vec4<T>* D, int Vf, T (&dF)[9]) {
  T d0[3] = {T(0), T(0), T(0)}, dk[3];
  if (r.v[0] < Vf) load3(D, r.v[0], d0);
#pragma unroll
  for (int q = 0; q < 9; ++q) dF[q] = T(0);
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    dk[0] = dk[1] = dk[2] = T(0);
    if (r.v[kk + 1] < Vf) load3(D, r.v[kk + 1], dk);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) dF[3 * i + j] += (dk[i] - d0[i]) * r.B[3 * kk + j];
  }
}

// Coefficients c_1..c_6 of Psi(F + a dF) - Psi(F) = sum_p c_p a^p (exact polynomial in a):
// with A = cof(F):dF, B = F:cof(dF), C = det dF, dJ(a) = A a + B a^2 + C a^3, and
// dPsi = mu (F:dF) a + mu/2 (dF:dF) a^2 - mu dJ + lam'/2 dJ (dJ + 2 (J - 1)).
template <typename T>
__device__ __forceinline__ void tet_dpsi_poly(const TetRec<T>& r, const T (&F)[9], const T (&C)[9], T jm1,
                                              const T (&dF)[9], T (&c)[6]) {
  T cdF[9];
  cofactor(dF, cdF);
  T f = T(0), q = T(0), A = T(0), B = T(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    f += F[k] * dF[k];
    q += dF[k] * dF[k];
    A += C[k] * dF[k];
    B += F[k] * cdF[k];
  }
  const T Cc = dF[0] * cdF[0] + dF[1] * cdF[1] + dF[2] * cdF[2];
  const T mu = r.mu, lp = r.lp, j1 = jm1, s = lp * j1 - mu;
  c[0] = r.vol * (mu * f + s * A);
  c[1] = r.vol * (T(0.5) * mu * q + s * B + T(0.5) * lp * A * A);
  c[2] = r.vol * (s * Cc + lp * A * B);
  c[3] = r.vol * (T(0.5) * lp * (B * B + T(2) * A * Cc));
  c[4] = r.vol * (lp * B * Cc);
  c[5] = r.vol * (T(0.5) * lp * Cc * Cc);
}

// Which line-search pass runs in a sweep (reading R17), by the mode latched when the sweep
// began: DIR 0 along D, when the last accepted step was along D; DIR 1 along D_J, after
// every trial of a DIR 0 pass failed; DIR 2 both directions in one pass, when the last
// accepted step was along D_J (its D trials are then tried first, the same order as DIR 0
// followed by DIR 1). One of the paths does the work; the others' launches return at once.
template <int DIR>
__device__ __forceinline__ bool ls_pass_runs(const StepState* st) {
  if (st->done) return false;
  if (DIR == 0) return st->ls_mode == 0;
  if (DIR == 1) return st->need_j != 0;
  return st->ls_mode != 0;
}

// Line search, IPC barrier part: the barrier change of the candidate pairs for each trial
// step a = 2^-j along the pass's direction(s) (not polynomial in a), FP64 sums per block into
// pp[(d * kLsTrials + j)][blockIdx], d the direction's place in the pass. k_energy adds them.
// A warp takes 32 candidates at a time; the few within r_c are handed to the whole warp in
// turn, lane l evaluating trial l % kLsTrials of direction l / kLsTrials, so a pair's trials
// run side by side instead of one after another in a single lane.
template <typename T, int DIR>
__global__ void __launch_bounds__(128) k_pair_trials(DevMesh<T> m, const StepState* __restrict__ st,
                                                     double* __restrict__ pp /* [ND * kLsTrials][grid] */) {
  if (!ls_pass_runs<DIR>(st)) return;
  constexpr int ND = DIR == 2 ? 2 : 1;
  constexpr int NB = ND * kLsTrials;
  static_assert(NB <= 32, "one lane per (direction, trial)");
  __shared__ double red[4][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int my_d = lane / kLsTrials, my_j = lane % kLsTrials;
  const bool has_slot = lane < NB;
  const Vec4<T>* my_dir = (DIR == 1 || my_d == 1) ? m.DJ : m.D;
  const double my_a = 1.0 / double(1 << my_j);
  double acc = 0.0;  // this lane's (direction, trial) sum
  const int np = min(*m.c.n_pairs, m.c.cap);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int base = (blockIdx.x * (blockDim.x >> 5) + wid) * 32; base < np; base += nwarps * 32) {
    const int q = base + lane;
    // a pair beyond r_c stays beyond dhat for every trial (each vertex moves at most
    // 0.45 (r_c - dhat)): its barrier is zero throughout
    const double dq_own = q < np ? m.c.d0[q] : INFINITY;
    unsigned near = __ballot_sync(0xffffffffu, dq_own < m.c.rc);
    while (near) {
      const int src = __ffs(near) - 1;
      near &= near - 1;
      const int qq = base + src;
      const double dq = __shfl_sync(0xffffffffu, dq_own, src);
      if (has_slot) {
        const uint64_t key = m.c.pairs[qq];
        // no trial brings the pair within dhat (and it starts outside): zero change
        if (dq - pair_motion(m, m.c, key, my_dir) < m.c.dhat * (1.0 + 1e-9)) {
          int vs[4], nv;
          P3 Jg[4];
          const double d = pair_geom(m, m.c, key, my_a, my_dir, vs, Jg, nv);
          acc += m.c.kappa * (barrier_b(d, m.c.dhat, m.c.pen) - barrier_b(dq, m.c.dhat, m.c.pen));
        }
      }
    }
  }
  if (m.c.fr_lam) {
    // friction change along the trial: mu lam (f0(|P(u + a d)|) - f0(|P u|)) per wall of
    // every surface vertex with a lagged normal force
    const size_t V = m.c.n_vertices;
    for (int base = (blockIdx.x * (blockDim.x >> 5) + wid) * 32; base < m.c.n_sverts; base += nwarps * 32) {
      const int q = base + lane;
      const int v_own = q < m.c.n_sverts ? m.c.sverts[q] : -1;
      bool has = false;
      if (v_own >= 0 && v_own < m.Vf)
        for (int p = 0; p < m.c.n_planes; ++p) has |= m.c.fr_lam[(size_t)p * V + v_own] > 0.0;
      unsigned todo = __ballot_sync(0xffffffffu, has);
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int v = __shfl_sync(0xffffffffu, v_own, src);
        if (has_slot) {
          const Vec4<T> uv = m.u[v], dv = my_dir[v];
          const double u0[3] = {double(uv.x), double(uv.y), double(uv.z)};
          const double u1[3] = {u0[0] + my_a * double(dv.x), u0[1] + my_a * double(dv.y),
                                u0[2] + my_a * double(dv.z)};
          acc += fric_energy_at(m.c, v, u1) - fric_energy_at(m.c, v, u0);
        }
      }
    }
  }
  // fixed-order sums: per (direction, trial) slot over the block's warps
  red[wid][lane] = acc;
  __syncthreads();
  if (threadIdx.x < NB) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w][threadIdx.x];
    pp[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = sum;
  }
}

// Line search (reading R17), passes as in ls_pass_runs: DIR 0 along the sweep direction D,
// DIR 1 along the uncorrected direction D_J (only when every trial along D failed), DIR 2
// along both in one pass (the tile loads, F and the displacement gathers are shared). The
// energy change along a direction is a polynomial in the step a; its coefficients are
// summed over tets (tiles of 128 records brought into shared memory by bulk copies,
// double-buffered in FP32) and free vertices, per thread and per block with Acc<T>
// (FP64-class), into per-block partials; k_ls_decide adds them up and decides.
template <typename T, int DIR>
__global__ void __launch_bounds__(128) k_energy(DevMesh<T> m, StepState* st,
                                                double* __restrict__ partial /* [6 ND][grid] */) {
  if (!ls_pass_runs<DIR>(st)) return;
  constexpr int ND = DIR == 2 ? 2 : 1;
  constexpr int NC = 6 * ND;
  // tiles of 128 records arrive by bulk copy; FP32 double-buffers them (the next tile is in
  // flight while this one is evaluated), FP64 (records twice as large) uses one buffer
  constexpr int NBUF = sizeof(T) == 4 ? 2 : 1;
  __shared__ __align__(128) TetRec<T> srec[NBUF][128];
  __shared__ __align__(8) uint64_t bar[NBUF];
  __shared__ Acc<T> sacc[32 * NC];
  const Vec4<T>* dirs[2] = {DIR == 1 ? m.DJ : m.D, m.DJ};
  Acc<T> acc[NC];
  const int ntile = (m.T_ + 127) / 128;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int b = 0; b < NBUF; ++b) mbar_init(&bar[b], 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int tl, int b) {
    if (threadIdx.x == 0 && tl < ntile) {
      const uint32_t bytes = uint32_t(min(128, m.T_ - tl * 128)) * uint32_t(sizeof(TetRec<T>));
      mbar_expect_tx(&bar[b], bytes);
      bulk_copy_g2s(&srec[b][0], m.tets + (size_t)tl * 128, bytes, &bar[b]);
    }
  };
  issue(blockIdx.x, 0);
  int k = 0;
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x, ++k) {
    const int t0 = tile * 128, n = min(128, m.T_ - t0);
    const int b = NBUF == 2 ? (k & 1) : 0;
    if (NBUF == 2) issue(tile + gridDim.x, b ^ 1);
    const bool got = mbar_wait(&bar[b], uint32_t((k / NBUF) & 1));
    if (__syncthreads_or(!got)) {
      // the copy never completed: report, wait (bounded) for the copies in flight, leave
      if (threadIdx.x == 0) {
        st->status = 8;  // JGS2_ETIMEOUT
        st->done = 1;
      }
      mbar_wait(&bar[b], uint32_t((k / NBUF) & 1));
      if (NBUF == 2 && tile + (int)gridDim.x < ntile) mbar_wait(&bar[b ^ 1], uint32_t(((k + 1) / NBUF) & 1));
      return;
    }
    const TetRec<T>* srec_b = srec[b];
    if ((int)threadIdx.x < n) {
      // F_e(x^k) is recomputed from the staged record and the corners' displacements
      // (L2-resident) rather than read back from the element pass, whose records have
      // left L2 by now
      const TetRec<T>& r = srec_b[threadIdx.x];
      T F[9], C[9], J1;
      tet_F_jm1(r, m.u, F, J1);
      cofactor(F, C);
#pragma unroll
      for (int dd = 0; dd < ND; ++dd) {
        T dF[9], c[6];
        tet_dF(r, dirs[dd], m.Vf, dF);
        tet_dpsi_poly(r, F, C, J1, dF, c);
#pragma unroll
        for (int j = 0; j < 6; ++j) acc[6 * dd + j].add(c[j]);
      }
    }
    __syncthreads();  // buffer b is read; it may be refilled
    if (NBUF == 1) issue(tile + gridDim.x, 0);
  }
  // inertia: m/(2h^2) (2 a d.(u - dz) + a^2 |d|^2)
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < m.Vf; v += stride) {
    T uv[3], dz[3];
    load3(m.u, v, uv);
    load3(m.dz, v, dz);
    const T mh = m.mh2[v];
#pragma unroll
    for (int di = 0; di < ND; ++di) {
      T d[3];
      load3(dirs[di], v, d);
      T dd = T(0), de = T(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        dd += d[q] * d[q];
        de += d[q] * (uv[q] - dz[q]);
      }
      acc[6 * di].add(mh * de);
      acc[6 * di + 1].add(T(0.5) * mh * dd);
    }
  }
  double bs[NC];
  block_sum_acc<T, NC>(acc, bs, sacc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NC; ++j) partial[(size_t)j * gridDim.x + blockIdx.x] = bs[j];
  }
}

// Line search decision (one block, after the pass's k_pair_trials and k_energy): sums every
// partial array (FP64, one warp per coefficient, fixed order: strided lane sums, then a
// fixed shuffle tree), evaluates E(x + a d) - E(x) at a = 2^-j along the pass's direction(s)
// in order and takes the first Armijo-satisfying trial. has_j = 0 (no correction, D = D_J):
// a failed D is a rejection.
template <int DIR>
__global__ void __launch_bounds__(1024) k_ls_decide(StepState* st, int has_j, const double* __restrict__ partial,
                                                    int n_part, const double* __restrict__ pp, int n_pp) {
  if (!ls_pass_runs<DIR>(st)) return;
  constexpr int ND = DIR == 2 ? 2 : 1;
  constexpr int NC = 6 * ND;
  constexpr int NB = ND * kLsTrials;
  static_assert(NC + NB <= 32, "one warp per coefficient");
  __shared__ double cf[NC + NB];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w < NC + NB) {
    const double* src = w < NC ? partial + (size_t)w * n_part : pp + (size_t)(w - NC) * n_pp;
    const int n = w < NC ? n_part : n_pp;
    double v = 0.0;
    for (int q = lane; q < n; q += 32) v += src[q];
    v = warp_sum(v);
    if (lane == 0) cf[w] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double alpha = 0.0;
  int chosen = -1;
  for (int dd = 0; dd < ND && chosen < 0; ++dd) {
    const int dir_id = (DIR == 1 || dd == 1) ? 1 : 0;
    const double slope = dir_id == 0 ? st->slope : st->slope_j;
    const double* c = cf + 6 * dd;
    for (int j = 0; j < kLsTrials; ++j) {
      const double a = 1.0 / double(1 << j);
      const double dE = a * (c[0] + a * (c[1] + a * (c[2] + a * (c[3] + a * (c[4] + a * c[5]))))) +
                        cf[NC + dd * kLsTrials + j];
      if (dE <= 1e-4 * a * slope) {
        alpha = a;
        chosen = dir_id;
        break;
      }
    }
  }
  const bool ok = chosen >= 0;
  st->alpha = alpha;
  st->dir = ok ? chosen : (DIR == 1 ? 1 : 0);
  if (DIR == 0) st->need_j = (!ok && has_j) ? 1 : 0;
  // |x^{k+1} - x^k|^2 of this sweep's update (zero when no trial passed)
  st->dx2 = alpha * alpha * (st->dir ? st->ddj2 : st->dd2);
  st->ls_passes[DIR] += 1;
  if (ok) {
    st->prev_dir = chosen;
    if (chosen == 1) st->dj_steps += 1;
  }
  if (!ok && (DIR != 0 || !has_j)) st->ls_rejects += 1;
}

// Batch meshes: the energy-change coefficients of k_energy, per scene, for the pass each
// scene takes (as ls_pass_runs, per scene: DIR 0 along D after a D sweep, DIR 1 along D_J
// after a failed DIR 0, DIR 2 along both after a D_J sweep); thread per tet in blocks
// [0, tet_blocks) (tiles staged in shared memory), thread per free vertex after; no
// contact. Blocks whose scenes have nothing to do return before loading.
template <typename T, int DIR>
__device__ __forceinline__ void energy_batch_body(const DevMesh<T>& m, int tet_blocks, int bid, TetRec<T>* srec) {
  constexpr int ND = DIR == 2 ? 2 : 1;
  constexpr int NC = 6 * ND;
  __shared__ int busy;
  const bool tets = bid < tet_blocks;
  const int i0 = tets ? bid * 128 : (bid - tet_blocks) * 128;
  const int n = min(128, (tets ? m.T_ : m.Vf) - i0);
  const int32_t* scene_of = tets ? m.t_scene : m.v_scene;
  auto wants = [&](int sc) {
    const SceneState& S = m.scenes[sc];
    return !S.done && (DIR == 0 ? S.ls_mode == 0 : (DIR == 1 ? S.need_j != 0 : S.ls_mode != 0));
  };
  if (threadIdx.x == 0) {
    // scenes are contiguous: the block covers scenes scene_of[i0] .. scene_of[i0 + n - 1]
    int any = 0;
    for (int sc = scene_of[i0]; sc <= scene_of[i0 + n - 1] && !any; ++sc) any = wants(sc) ? 1 : 0;
    busy = any;
  }
  __syncthreads();
  if (!busy) return;
  const Vec4<T>* dirs[2] = {DIR == 1 ? m.DJ : m.D, m.DJ};
  Acc<T> acc[NC];
  int sc = -1;
  if (tets) {
    stage_tets<T, 128>(m.tets, i0, n, srec);
    __syncthreads();
    if ((int)threadIdx.x < n) {
      const int t = i0 + threadIdx.x;
      sc = m.t_scene[t];
      if (wants(sc)) {
        const TetRec<T>& r = srec[threadIdx.x];
        T F[9], C[9], J1;
        tet_F_jm1(r, m.u, F, J1);
        cofactor(F, C);
#pragma unroll
        for (int dd = 0; dd < ND; ++dd) {
          T dF[9], c[6];
          tet_dF(r, dirs[dd], m.Vf, dF);
          tet_dpsi_poly(r, F, C, J1, dF, c);
#pragma unroll
          for (int j = 0; j < 6; ++j) acc[6 * dd + j].add(c[j]);
        }
      } else {
        sc = -1;
      }
    }
  } else if ((int)threadIdx.x < n) {
    const int v = i0 + threadIdx.x;
    sc = m.v_scene[v];
    if (wants(sc)) {
      T uv[3], dz[3];
      load3(m.u, v, uv);
      load3(m.dz, v, dz);
      const T mh = m.mh2[v];
#pragma unroll
      for (int di = 0; di < ND; ++di) {
        T d[3];
        load3(dirs[di], v, d);
        T dd = T(0), de = T(0);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          dd += d[q] * d[q];
          de += d[q] * (uv[q] - dz[q]);
        }
        acc[6 * di].add(mh * de);
        acc[6 * di + 1].add(T(0.5) * mh * dd);
      }
    } else {
      sc = -1;
    }
  }
  scene_reduce_acc<T, NC>(acc, sc, m.sacc, 3);
}

template <typename T, int DIR>
__global__ void __launch_bounds__(128) k_energy_batch(DevMesh<T> m, int tet_blocks) {
  __shared__ __align__(16) TetRec<T> srec[128];
  energy_batch_body<T, DIR>(m, tet_blocks, blockIdx.x, srec);
}

// Batch meshes, thread per scene: residual bookkeeping of the sweep (reading R9) from the
// per-scene sums, then clear them.
__device__ __forceinline__ void scene_finalize_main_body(SceneState* scenes, double* sacc, int n, double rel_tol,
                                                         int max_sweeps, int corr, int32_t* n_done, int s) {
  if (s >= n) return;
  SceneState& S = scenes[s];
  double* a = sacc + (size_t)s * kSceneAcc;
  if (!S.done) {
    const int k = S.k;
    const double gn = sqrt(a[0]);
    if (k == 0) S.g0 = gn;
    const double r = S.g0 > 0.0 ? gn / S.g0 : 0.0;
    S.r = r;
    S.slope_j = a[1];
    S.slope = corr ? a[2] : a[1];
    S.alpha = 1.0;
    S.dir = 0;
    S.need_j = 0;
    S.ls_mode = S.prev_dir;
    bool fin = false;
    if (!isfinite(r) || !isfinite(S.slope)) {
      S.status = 6;
      fin = true;
    } else if (r <= rel_tol || S.g0 == 0.0) {
      S.converged = 1;
      fin = true;
    } else if (k >= max_sweeps) {
      fin = true;
    }
    if (fin) {
      S.done = 1;
      S.sweeps = k;
      atomicAdd(n_done, 1);
    } else {
      S.k = k + 1;
    }
  }
  a[0] = a[1] = a[2] = 0.0;
}

static __global__ void k_scene_finalize_main(SceneState* scenes, double* sacc, int n, double rel_tol, int max_sweeps,
                                             int corr, int32_t* n_done) {
  scene_finalize_main_body(scenes, sacc, n, rel_tol, max_sweeps, corr, n_done, blockIdx.x * blockDim.x + threadIdx.x);
}

// Batch meshes, thread per scene: Armijo choice from the per-scene polynomial sums of the
// scene's pass (DIR as in k_energy_batch; DIR 0 records need_j when every trial failed and
// D_J differs), then the sums are cleared for the next pass.
template <int DIR>
__device__ __forceinline__ void scene_finalize_energy_body(SceneState* scenes, double* sacc, int n, int has_j, int s) {
  constexpr int ND = DIR == 2 ? 2 : 1;
  if (s >= n) return;
  SceneState& S = scenes[s];
  double* cf = sacc + (size_t)s * kSceneAcc + 3;
  const bool runs = !S.done && (DIR == 0 ? S.ls_mode == 0 : (DIR == 1 ? S.need_j != 0 : S.ls_mode != 0));
  if (runs) {
    double alpha = 0.0;
    int chosen = -1;
    for (int dd = 0; dd < ND && chosen < 0; ++dd) {
      const int dir_id = (DIR == 1 || dd == 1) ? 1 : 0;
      const double slope = dir_id == 0 ? S.slope : S.slope_j;
      const double* c = cf + 6 * dd;
      for (int j = 0; j < kLsTrials; ++j) {
        const double a = 1.0 / double(1 << j);
        const double dE = a * (c[0] + a * (c[1] + a * (c[2] + a * (c[3] + a * (c[4] + a * c[5])))));
        if (dE <= 1e-4 * a * slope) {
          alpha = a;
          chosen = dir_id;
          break;
        }
      }
    }
    const bool ok = chosen >= 0;
    S.alpha = alpha;
    S.dir = ok ? chosen : (DIR == 1 ? 1 : 0);
    if (DIR == 0) S.need_j = (!ok && has_j) ? 1 : 0;
    if (ok) S.prev_dir = chosen;
    if (!ok && (DIR != 0 || !has_j)) S.ls_rejects += 1;
  }
  for (int j = 0; j < 6 * ND; ++j) cf[j] = 0.0;
}

template <int DIR>
static __global__ void k_scene_finalize_energy(SceneState* scenes, double* sacc, int n, int has_j) {
  scene_finalize_energy_body<DIR>(scenes, sacc, n, has_j, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__device__ __forceinline__ void update_batch_body(const DevMesh<T>& m, int i) {
  if (i >= m.Vf) return;
  const SceneState& S = m.scenes[m.v_scene[i]];
  if (S.done) return;
  const T a = T(S.alpha);
  Vec4<T> u = m.u[i];
  const Vec4<T> d = S.dir ? m.DJ[i] : m.D[i];
  u.x += a * d.x;
  u.y += a * d.y;
  u.z += a * d.z;
  m.u[i] = u;
}

template <typename T>
__global__ void k_update_batch(DevMesh<T> m) {
  update_batch_body<T>(m, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(128) k_update(DevMesh<T> m, const StepState* __restrict__ st) {
  if (st->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float step = 0.f;
  if (i < m.Vf) {
    const T a = T(st->alpha);
    Vec4<T> u = m.u[i];
    const Vec4<T> d = st->dir ? m.DJ[i] : m.D[i];
    u.x += a * d.x;
    u.y += a * d.y;
    u.z += a * d.z;
    m.u[i] = u;
    if (m.c.on) {
      // an upper bound of the vertex's motion for the contact skip test's path bound, in
      // FP32: |a d| with a 1e-5 relative allowance for its own rounding, plus the rounding
      // of u + a d (a few FP32 ulps of the new u)
      const float dx = float(d.x), dy = float(d.y), dz = float(d.z);
      const float ux = float(u.x), uy = float(u.y), uz = float(u.z);
      step = fabsf(float(a)) * sqrtf(dx * dx + dy * dy + dz * dz) * (1.f + 1e-5f) +
             3e-7f * sqrtf(ux * ux + uy * uy + uz * uz);
    }
  }
  if (m.c.on) {
    // the sweep's largest step: warp and block maxima, one atomic per block (non-negative
    // floats order like their bit patterns)
    __shared__ uint32_t wmax[4];
    const uint32_t w = __reduce_max_sync(0xffffffffu, __float_as_uint(step));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t b = max(max(wmax[0], wmax[1]), max(wmax[2], wmax[3]));
      if (b != 0u) atomicMax(&m.c.ctl[kCtlStep], b);
    }
  }
}

// x_{t+1} = x_t + u, v_{t+1} = u / h, written back in caller order.
template <typename T>
__global__ void k_finish(DevMesh<T> m, double* __restrict__ x_caller, double* __restrict__ v_caller) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= m.V) return;
  const int c = m.perm[v];
  T u[3];
  load3(m.u, v, u);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    x_caller[3 * c + q] = m.xt[3 * v + q] + double(u[q]);
    if (v_caller) v_caller[3 * c + q] = double(u[q]) / m.h;
  }
}

// FP64 energy and gradient of the current state (parity helper).
template <typename T>
__global__ void k_grad(DevMesh<T> m, double* __restrict__ g_caller) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.V) return;
  const int c = m.perm[i];
  if (i >= m.Vf) {
    g_caller[3 * c] = g_caller[3 * c + 1] = g_caller[3 * c + 2] = 0.0;
    return;
  }
  T g[3], H[6], Fs[9], W;
  gather_vertex_rec(m, i, g, H, Fs, W);
  T ui[3], dz[3];
  load3(m.u, i, ui);
  load3(m.dz, i, dz);
#pragma unroll
  for (int q = 0; q < 3; ++q)
    g_caller[3 * c + q] = double(g[q] + m.mh2[i] * (ui[q] - dz[q])) + (m.c.on ? m.c.bg[(size_t)q * m.V + i] : 0.0);
}

template <typename T>
__global__ void __launch_bounds__(128) k_energy_abs(DevMesh<T> m, double* __restrict__ partial,
                                                    int tet_blocks) {
  __shared__ double red[32];
  double acc[1] = {0.0};
  if ((int)blockIdx.x < tet_blocks) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m.T_) {
      const TetRec<T> r = m.tets[t];
      T F[9], C[9], J1;
      tet_F_jm1(r, m.u, F, J1);
      cofactor(F, C);
      T FF = T(0);
#pragma unroll
      for (int q = 0; q < 9; ++q) FF += F[q] * F[q];
      acc[0] = double(r.vol) * (0.5 * double(r.mu) * (double(FF) - 3.0) - double(r.mu) * double(J1) +
                                0.5 * double(r.lp) * double(J1) * double(J1));
    }
  } else {
    const int v = (blockIdx.x - tet_blocks) * blockDim.x + threadIdx.x;
    if (v < m.Vf) {
      T uv[3], dz[3];
      load3(m.u, v, uv);
      load3(m.dz, v, dz);
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < 3; ++q) s += (double(uv[q]) - double(dz[q])) * (double(uv[q]) - double(dz[q]));
      acc[0] = 0.5 * double(m.mh2[v]) * s;
    }
  }
  block_sum<1>(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc[0];
}

}  // namespace jgs2
