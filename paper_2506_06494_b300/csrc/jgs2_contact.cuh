// IPC contact on the device (Sec. 7, Eq. barrier): candidate pairs within r_c by a hashed
// uniform grid, closest points in FP64, the barrier's per-vertex gradient and Gauss-Newton
// diagonal blocks (FP64 accumulators), the per-vertex step limit and the barrier part of
// the line-search energy.
//
// Pair kinds: 0 vertex-wall (vertex, plane), 1 vertex-face (vertex, face), 2 edge-edge
// (edge i < edge j, no shared vertex). Walls are planes n.x >= c.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "jgs2_internal.h"

namespace jgs2 {

__device__ __forceinline__ double barrier_b(double d, double dh) {
  if (d <= 0.0) return INFINITY;
  if (d >= dh) return 0.0;
  const double e = d - dh;
  return -e * e * log(d / dh);
}
__device__ __forceinline__ double barrier_b1(double d, double dh) {
  if (d <= 0.0 || d >= dh) return 0.0;
  const double e = d - dh;
  return -2.0 * e * log(d / dh) - e * e / d;
}
__device__ __forceinline__ double barrier_b2(double d, double dh) {
  if (d <= 0.0 || d >= dh) return 0.0;
  const double e = d - dh;
  return -2.0 * log(d / dh) - 4.0 * e / d + e * e / (d * d);
}

struct P3 {
  double x, y, z;
};
__device__ __forceinline__ P3 sub(P3 a, P3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ P3 add(P3 a, P3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ P3 mul(P3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ double dot(P3 a, P3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ P3 cross(P3 a, P3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double norm(P3 a) { return sqrt(dot(a, a)); }

// position x = x_t + u (+ a d) of internal vertex v, FP64
template <typename T>
__device__ __forceinline__ P3 vpos(const DevMesh<T>& m, int v, double a = 0.0, const Vec4<T>* D = nullptr) {
  const Vec4<T> u = m.u[v];
  P3 p{m.xt[3 * v] + double(u.x), m.xt[3 * v + 1] + double(u.y), m.xt[3 * v + 2] + double(u.z)};
  if (D != nullptr && v < m.Vf) {
    const Vec4<T> d = D[v];
    p.x += a * double(d.x);
    p.y += a * double(d.y);
    p.z += a * double(d.z);
  }
  return p;
}

// closest point of segment ab to p: distance and parameter t
__device__ __forceinline__ double point_segment(P3 p, P3 a, P3 b, double& t) {
  const P3 ab = sub(b, a);
  const double L2 = dot(ab, ab);
  t = L2 == 0.0 ? 0.0 : fmin(fmax(dot(sub(p, a), ab) / L2, 0.0), 1.0);
  return norm(sub(p, add(a, mul(ab, t))));
}

// Closest point of triangle abc to p: the projection onto the plane when its barycentric
// coordinates are non-negative, else the nearest edge (ab, bc, ca in that order, strict <).
__device__ __forceinline__ double point_triangle(P3 p, P3 a, P3 b, P3 c, double (&w)[3]) {
  const P3 n = cross(sub(b, a), sub(c, a));
  const double nn = dot(n, n);
  if (nn > 0.0) {
    const P3 q = sub(p, mul(n, dot(sub(p, a), n) / nn));
    const P3 v0 = sub(b, a), v1 = sub(c, a), v2 = sub(q, a);
    const double d00 = dot(v0, v0), d01 = dot(v0, v1), d11 = dot(v1, v1), d20 = dot(v2, v0), d21 = dot(v2, v1);
    const double den = d00 * d11 - d01 * d01;
    const double wb = (d11 * d20 - d01 * d21) / den, wc = (d00 * d21 - d01 * d20) / den, wa = 1.0 - wb - wc;
    if (wa >= 0.0 && wb >= 0.0 && wc >= 0.0) {
      w[0] = wa;
      w[1] = wb;
      w[2] = wc;
      return norm(sub(p, q));
    }
  }
  double t, best;
  double d = point_segment(p, a, b, t);
  best = d;
  w[0] = 1.0 - t;
  w[1] = t;
  w[2] = 0.0;
  d = point_segment(p, b, c, t);
  if (d < best) {
    best = d;
    w[0] = 0.0;
    w[1] = 1.0 - t;
    w[2] = t;
  }
  d = point_segment(p, c, a, t);
  if (d < best) {
    best = d;
    w[0] = t;
    w[1] = 0.0;
    w[2] = 1.0 - t;
  }
  return best;
}

// Closest points of segments p0p1, q0q1: the interior critical point of |p(s) - q(t)|^2 when
// the segments are not parallel and it lies in [0,1]^2, else the nearest of the endpoint
// cases (p0 to q, p1 to q, q0 to p, q1 to p, in that order, strict <).
__device__ __forceinline__ double segment_segment(P3 p0, P3 p1, P3 q0, P3 q1, double& s, double& t) {
  const P3 d1 = sub(p1, p0), d2 = sub(q1, q0), r = sub(p0, q0);
  const double a = dot(d1, d1), e = dot(d2, d2), b = dot(d1, d2), c = dot(d1, r), f = dot(d2, r);
  const double den = a * e - b * b;
  if (den > 1e-14 * a * e && a > 0.0 && e > 0.0) {
    const double ss = (b * f - c * e) / den, tt = (a * f - b * c) / den;
    if (ss >= 0.0 && ss <= 1.0 && tt >= 0.0 && tt <= 1.0) {
      s = ss;
      t = tt;
      return norm(sub(add(p0, mul(d1, ss)), add(q0, mul(d2, tt))));
    }
  }
  double tq, best = point_segment(p0, q0, q1, tq);
  s = 0.0;
  t = tq;
  double dd = point_segment(p1, q0, q1, tq);
  if (dd < best) {
    best = dd;
    s = 1.0;
    t = tq;
  }
  double sp;
  dd = point_segment(q0, p0, p1, sp);
  if (dd < best) {
    best = dd;
    s = sp;
    t = 0.0;
  }
  dd = point_segment(q1, p0, p1, sp);
  if (dd < best) {
    best = dd;
    s = sp;
    t = 1.0;
  }
  return best;
}

__device__ __forceinline__ uint64_t cell_key(P3 p, double h) {
  const long long ix = (long long)floor(p.x / h) + (1 << 20), iy = (long long)floor(p.y / h) + (1 << 20),
                  iz = (long long)floor(p.z / h) + (1 << 20);
  return ((uint64_t)(ix & 0x1fffff) << 42) | ((uint64_t)(iy & 0x1fffff) << 21) | (uint64_t)(iz & 0x1fffff);
}

__device__ __forceinline__ void emit_pair(const ContactView& c, uint64_t kind, uint64_t a, uint64_t b) {
  const int idx = atomicAdd(c.n_pairs, 1);
  if (idx < c.cap)
    c.pairs[idx] = (kind << 60) | (a << 30) | b;
  else
    c.flags[0] = 1;
}

// cell keys of face centroids (kind 0) and edge midpoints (kind 1)
template <typename T>
__global__ void k_prim_keys(DevMesh<T> m, ContactView c, uint64_t* fkeys, int32_t* fids, uint64_t* ekeys,
                            int32_t* eids) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < c.n_faces) {
    const P3 a = vpos(m, c.faces[3 * i]), b = vpos(m, c.faces[3 * i + 1]), d = vpos(m, c.faces[3 * i + 2]);
    fkeys[i] = cell_key(mul(add(add(a, b), d), 1.0 / 3.0), c.cell);
    fids[i] = i;
  }
  if (i < c.n_edges) {
    const P3 a = vpos(m, c.edges[2 * i]), b = vpos(m, c.edges[2 * i + 1]);
    ekeys[i] = cell_key(mul(add(a, b), 0.5), c.cell);
    eids[i] = i;
  }
}

__device__ __forceinline__ int lower_bound_key(const uint64_t* k, int n, uint64_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (k[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// surface vertex queries: walls and faces within rc
template <typename T>
__global__ void k_query_vertices(DevMesh<T> m, ContactView c) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= c.n_sverts) return;
  const int v = c.sverts[q];
  const P3 p = vpos(m, v);
  for (int k = 0; k < c.n_planes; ++k) {
    const double d = c.planes[4 * k] * p.x + c.planes[4 * k + 1] * p.y + c.planes[4 * k + 2] * p.z - c.planes[4 * k + 3];
    if (d < c.rc) emit_pair(c, 0, v, k);
  }
  const long long cx = (long long)floor(p.x / c.cell), cy = (long long)floor(p.y / c.cell),
                  cz = (long long)floor(p.z / c.cell);
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz) {
        const uint64_t key = ((uint64_t)((cx + dx + (1 << 20)) & 0x1fffff) << 42) |
                             ((uint64_t)((cy + dy + (1 << 20)) & 0x1fffff) << 21) |
                             (uint64_t)((cz + dz + (1 << 20)) & 0x1fffff);
        for (int j = lower_bound_key(c.fkeys, c.n_faces, key); j < c.n_faces && c.fkeys[j] == key; ++j) {
          const int f = c.fids[j];
          const int a = c.faces[3 * f], b = c.faces[3 * f + 1], cc = c.faces[3 * f + 2];
          if (a == v || b == v || cc == v) continue;
          const P3 pa = vpos(m, a), pb = vpos(m, b), pc = vpos(m, cc);
          // box distance is a lower bound of the distance
          const double gx = fmax(fmax(fmin(fmin(pa.x, pb.x), pc.x) - p.x, p.x - fmax(fmax(pa.x, pb.x), pc.x)), 0.0);
          const double gy = fmax(fmax(fmin(fmin(pa.y, pb.y), pc.y) - p.y, p.y - fmax(fmax(pa.y, pb.y), pc.y)), 0.0);
          const double gz = fmax(fmax(fmin(fmin(pa.z, pb.z), pc.z) - p.z, p.z - fmax(fmax(pa.z, pb.z), pc.z)), 0.0);
          if (gx * gx + gy * gy + gz * gz >= c.rc * c.rc) continue;
          double w[3];
          if (point_triangle(p, pa, pb, pc, w) < c.rc) emit_pair(c, 1, v, f);
        }
      }
}

// edge queries: edges j > i sharing no vertex within rc
template <typename T>
__global__ void k_query_edges(DevMesh<T> m, ContactView c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.n_edges) return;
  const int a0 = c.edges[2 * i], a1 = c.edges[2 * i + 1];
  const P3 p0 = vpos(m, a0), p1 = vpos(m, a1);
  const P3 mid = mul(add(p0, p1), 0.5);
  const long long cx = (long long)floor(mid.x / c.cell), cy = (long long)floor(mid.y / c.cell),
                  cz = (long long)floor(mid.z / c.cell);
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz) {
        const uint64_t key = ((uint64_t)((cx + dx + (1 << 20)) & 0x1fffff) << 42) |
                             ((uint64_t)((cy + dy + (1 << 20)) & 0x1fffff) << 21) |
                             (uint64_t)((cz + dz + (1 << 20)) & 0x1fffff);
        for (int j = lower_bound_key(c.ekeys, c.n_edges, key); j < c.n_edges && c.ekeys[j] == key; ++j) {
          const int e = c.eids[j];
          if (e <= i) continue;
          const int b0 = c.edges[2 * e], b1 = c.edges[2 * e + 1];
          if (b0 == a0 || b0 == a1 || b1 == a0 || b1 == a1) continue;
          const P3 q0 = vpos(m, b0), q1 = vpos(m, b1);
          const double gx = fmax(fmax(fmin(q0.x, q1.x) - fmax(p0.x, p1.x), fmin(p0.x, p1.x) - fmax(q0.x, q1.x)), 0.0);
          const double gy = fmax(fmax(fmin(q0.y, q1.y) - fmax(p0.y, p1.y), fmin(p0.y, p1.y) - fmax(q0.y, q1.y)), 0.0);
          const double gz = fmax(fmax(fmin(q0.z, q1.z) - fmax(p0.z, p1.z), fmin(p0.z, p1.z) - fmax(q0.z, q1.z)), 0.0);
          if (gx * gx + gy * gy + gz * gz >= c.rc * c.rc) continue;
          double s, t;
          if (segment_segment(p0, p1, q0, q1, s, t) < c.rc) emit_pair(c, 2, i, e);
        }
      }
}

// Geometry of a pair at x (+ a d): distance, involved vertices and dd/dx per vertex.
template <typename T>
__device__ __forceinline__ double pair_geom(const DevMesh<T>& m, const ContactView& c, uint64_t key, double a,
                                            const Vec4<T>* D, int (&vs)[4], P3 (&J)[4], int& nv) {
  const int kind = (int)(key >> 60), ia = (int)((key >> 30) & 0x3fffffff), ib = (int)(key & 0x3fffffff);
  if (kind == 0) {
    const P3 p = vpos(m, ia, a, D);
    const double* pl = c.planes + 4 * ib;
    nv = 1;
    vs[0] = ia;
    J[0] = {pl[0], pl[1], pl[2]};
    return pl[0] * p.x + pl[1] * p.y + pl[2] * p.z - pl[3];
  }
  if (kind == 1) {
    const int f0 = c.faces[3 * ib], f1 = c.faces[3 * ib + 1], f2 = c.faces[3 * ib + 2];
    const P3 p = vpos(m, ia, a, D), pa = vpos(m, f0, a, D), pb = vpos(m, f1, a, D), pc = vpos(m, f2, a, D);
    double w[3];
    const double d = point_triangle(p, pa, pb, pc, w);
    const P3 q = add(add(mul(pa, w[0]), mul(pb, w[1])), mul(pc, w[2]));
    const P3 n = d > 0.0 ? mul(sub(p, q), 1.0 / d) : P3{0, 0, 0};
    nv = 4;
    vs[0] = ia;
    vs[1] = f0;
    vs[2] = f1;
    vs[3] = f2;
    J[0] = n;
    J[1] = mul(n, -w[0]);
    J[2] = mul(n, -w[1]);
    J[3] = mul(n, -w[2]);
    return d;
  }
  const int e0 = c.edges[2 * ia], e1 = c.edges[2 * ia + 1], g0 = c.edges[2 * ib], g1 = c.edges[2 * ib + 1];
  const P3 p0 = vpos(m, e0, a, D), p1 = vpos(m, e1, a, D), q0 = vpos(m, g0, a, D), q1 = vpos(m, g1, a, D);
  double s, t;
  const double d = segment_segment(p0, p1, q0, q1, s, t);
  const P3 pp = add(p0, mul(sub(p1, p0), s)), qq = add(q0, mul(sub(q1, q0), t));
  const P3 n = d > 0.0 ? mul(sub(pp, qq), 1.0 / d) : P3{0, 0, 0};
  nv = 4;
  vs[0] = e0;
  vs[1] = e1;
  vs[2] = g0;
  vs[3] = g1;
  J[0] = mul(n, 1.0 - s);
  J[1] = mul(n, s);
  J[2] = mul(n, -(1.0 - t));
  J[3] = mul(n, -t);
  return d;
}

static __global__ void k_contact_reset(ContactView c, int V) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
#pragma unroll
  for (int q = 0; q < 3; ++q) c.bg[(size_t)q * V + v] = 0.0;
#pragma unroll
  for (int q = 0; q < 6; ++q) c.bH[(size_t)q * V + v] = 0.0;
  c.dmin[v] = INFINITY;
}

// per pair: distance at x^k, smallest candidate distance per vertex, and for active pairs
// (d < dhat) kappa B'(d) dd/dx and kappa B''(d) (dd/dx)(dd/dx)^T into the FP64 accumulators
template <typename T>
__global__ void k_pair_terms(DevMesh<T> m, ContactView c, StepState* st) {
  const int n = min(*c.n_pairs, c.cap);
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int vs[4], nv;
  P3 J[4];
  const double d = pair_geom(m, c, c.pairs[q], 0.0, (const Vec4<T>*)nullptr, vs, J, nv);
  c.d0[q] = d;
  if (!(d > 0.0)) {
    c.flags[1] = 1;
    st->status = 9;  // JGS2_EINTERSECT
    st->done = 1;
    return;
  }
  // positive doubles order like their bit patterns
  for (int k = 0; k < nv; ++k)
    atomicMin(reinterpret_cast<unsigned long long*>(c.dmin + vs[k]), (unsigned long long)__double_as_longlong(d));
  if (d >= c.dhat) return;
  const double b1 = c.kappa * barrier_b1(d, c.dhat), b2 = c.kappa * barrier_b2(d, c.dhat);
  const size_t V = m.V;
  for (int k = 0; k < nv; ++k) {
    const int v = vs[k];
    if (v >= m.Vf) continue;
    const P3 j = J[k];
    atomicAdd(c.bg + v, b1 * j.x);
    atomicAdd(c.bg + V + v, b1 * j.y);
    atomicAdd(c.bg + 2 * V + v, b1 * j.z);
    atomicAdd(c.bH + v, b2 * j.x * j.x);
    atomicAdd(c.bH + V + v, b2 * j.x * j.y);
    atomicAdd(c.bH + 2 * V + v, b2 * j.x * j.z);
    atomicAdd(c.bH + 3 * V + v, b2 * j.y * j.y);
    atomicAdd(c.bH + 4 * V + v, b2 * j.y * j.z);
    atomicAdd(c.bH + 5 * V + v, b2 * j.z * j.z);
  }
}

// barrier energy of the pairs at x^k (for jgs2_energy_gradient)
template <typename T>
__global__ void k_pair_energy(DevMesh<T> m, ContactView c, double* out) {
  __shared__ double red[32];
  const int n = min(*c.n_pairs, c.cap);
  double acc[1] = {0.0};
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
    acc[0] += c.kappa * barrier_b(c.d0[q], c.dhat);
  block_sum<1>(acc, red);
  if (threadIdx.x == 0) atomicAdd(out, acc[0]);
}

}  // namespace jgs2
