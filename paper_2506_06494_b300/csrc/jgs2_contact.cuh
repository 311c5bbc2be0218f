// IPC contact on the device (Sec. 7, Eq. barrier): candidate pairs by hashed uniform grids
// (rebuilt on demand), closest points in FP64, the barrier's per-vertex gradient and Gauss-Newton
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

// Contact energy per pair and its derivatives in d: the IPC log barrier of Eq. barrier
// (pen = 0), or the implicit quadratic penalty (pen = 1): (dh - d)^2 / 2 for d < dh, the
// other form Sec. 7 admits (any contact written as an unconstrained energy).
__device__ __forceinline__ double barrier_b(double d, double dh, int pen = 0) {
  if (pen) return d >= dh ? 0.0 : 0.5 * (dh - d) * (dh - d);
  if (d <= 0.0) return INFINITY;
  if (d >= dh) return 0.0;
  const double e = d - dh;
  return -e * e * log(d / dh);
}
__device__ __forceinline__ double barrier_b1(double d, double dh, int pen = 0) {
  if (pen) return d >= dh ? 0.0 : d - dh;
  if (d <= 0.0 || d >= dh) return 0.0;
  const double e = d - dh;
  return -2.0 * e * log(d / dh) - e * e / d;
}
__device__ __forceinline__ double barrier_b2(double d, double dh, int pen = 0) {
  if (pen) return d >= dh ? 0.0 : 1.0;
  if (d <= 0.0 || d >= dh) return 0.0;
  const double e = d - dh;
  return -2.0 * log(d / dh) - 4.0 * e / d + e * e / (d * d);
}

// Friction on the walls (IPC's lagged friction potential): a surface vertex v within dhat of
// wall p at the step start carries the lagged normal force lam = -kappa E'(d(x_t)), and the
// step adds mu lam f0(|P_p (x_v - x_t,v)|), P_p = I - n n^T; f0 smooths |u| below the slip
// eps: -y^3/(3 eps^2) + y^2/eps + eps/3 for y < eps, y beyond (C^1 at eps).
__device__ __forceinline__ double fric_f0(double y, double e) {
  return y < e ? -y * y * y / (3.0 * e * e) + y * y / e + e / 3.0 : y;
}
__device__ __forceinline__ double fric_f1_over_y(double y, double e) {
  return y < e ? -y / (e * e) + 2.0 / e : 1.0 / y;
}
// tangential part P_p u of a displacement u at wall p (unit normal n)
__device__ __forceinline__ void fric_tangential(const double* n, const double (&u)[3], double (&ut)[3]) {
  const double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  ut[0] = u[0] - un * n[0];
  ut[1] = u[1] - un * n[1];
  ut[2] = u[2] - un * n[2];
}
__device__ __forceinline__ double fric_norm(const double (&a)[3]) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

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

// ---------------------------------------------------------------------------------------
// Broadphase. The candidate list holds every pair closer than R = r_c + 2M at the positions
// of its last rebuild. Before every sweep k_bp_check measures the largest displacement of a
// surface vertex since then and rebuilds the list when it exceeds M. A pair within r_c at the
// sweep's positions was then closer than r_c + 2M at the rebuild, so it is in the list, and
// the sweep's pair set (the pairs within r_c, evaluated exactly in FP64) is the one a fresh
// search would give. Pairs beyond r_c at x^k stay beyond dhat through the sweep's line search
// (a surface vertex moves at most 0.45 (r_c - dhat) per sweep). The grids are hashed (counting sort by bucket, no host round trip): a
// sweep that needs no rebuild runs the rebuild kernels as empty launches.
// ---------------------------------------------------------------------------------------
enum { kCtlMove = 0, kCtlRebuild = 1, kCtlForce = 2, kCtlTicket = 3, kCtlExtF = 4, kCtlExtE = 5, kCtlAcc = 6,
       kCtlCoord = 7, kCtlNear = 8, kCtlStep = 9, kCtlPath = 10, kCtlWords = 11 };

__device__ __forceinline__ uint64_t cell_key(P3 p, double h) {
  const long long ix = (long long)floor(p.x / h) + (1 << 20), iy = (long long)floor(p.y / h) + (1 << 20),
                  iz = (long long)floor(p.z / h) + (1 << 20);
  return ((uint64_t)(ix & 0x1fffff) << 42) | ((uint64_t)(iy & 0x1fffff) << 21) | (uint64_t)(iz & 0x1fffff);
}
__device__ __forceinline__ uint64_t cell_key_of(long long cx, long long cy, long long cz) {
  return ((uint64_t)((cx + (1 << 20)) & 0x1fffff) << 42) | ((uint64_t)((cy + (1 << 20)) & 0x1fffff) << 21) |
         (uint64_t)((cz + (1 << 20)) & 0x1fffff);
}
__device__ __forceinline__ uint32_t bucket_of(uint64_t key, int hbits) {
  return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - hbits));
}
// grid cells: a face within R of a point has its centroid within R + (largest centroid-corner
// distance); two edges within R have midpoints within R + 2 (largest half length)
__device__ __forceinline__ void grid_cells(const ContactView& c, double& hf, double& he) {
  const double ef = double(__uint_as_float(c.ctl[kCtlExtF])), ee = double(__uint_as_float(c.ctl[kCtlExtE]));
  hf = (c.R + ef) * (1.0 + 1e-6) + 1e-12;
  he = (c.R + 2.0 * ee) * (1.0 + 1e-6) + 1e-12;
}
// FP32 rounding slack of the position snapshot (a few ulps of the largest coordinate)
__device__ __forceinline__ double snap_slack(const ContactView& c) {
  return 8.0 * 5.9604644775390625e-8 * double(__uint_as_float(c.ctl[kCtlCoord])) + 1e-30;
}

__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ void warp_atomic_max(uint32_t* w, float v) {
  v = warp_maxf(v);
  if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(w, __float_as_uint(v));
}

__device__ __forceinline__ void emit_pair(const ContactView& c, uint64_t kind, uint64_t a, uint64_t b, double d) {
  const int idx = atomicAdd(c.n_pairs, 1);
  if (idx < c.cap) {
    c.pairs[idx] = (kind << 60) | (a << 30) | b;
    c.dbp[idx] = __double2float_rd(d);
    c.pmarg[idx] = -1.f;  // no motion check yet
  } else {
    c.flags[0] = 1;
  }
}

// Largest surface-vertex displacement since the last rebuild; the last block decides the
// rebuild (forced at the start of a step) and clears the counters of the next one.
template <typename T>
__global__ void __launch_bounds__(256) k_bp_check(DevMesh<T> m, ContactView c, StepState* st) {
  if (st->done) {
    if (blockIdx.x == 0 && threadIdx.x == 0) c.ctl[kCtlRebuild] = 0u;
    return;
  }
  __shared__ float red[8];
  __shared__ bool last;
  float mx = 0.f;
  const size_t V = c.n_vertices;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < c.n_sverts; q += gridDim.x * blockDim.x) {
    const int v = c.sverts[q];
    // clear this sweep's barrier accumulators (only surface vertices are ever written)
#pragma unroll
    for (int k = 0; k < 3; ++k) c.bg[(size_t)k * V + v] = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) c.bH[(size_t)k * V + v] = 0.0;
    c.dmin[v] = INFINITY;
    if (c.vp_cnt) c.vp_cnt[v] = 0;
    const P3 p = vpos(m, v);
    const float4 b = c.pbp[v];
    const double dx = p.x - double(b.x), dy = p.y - double(b.y), dz = p.z - double(b.z);
    const double d = sqrt(dx * dx + dy * dy + dz * dz);
    mx = fmaxf(mx, d == d ? __double2float_ru(d) : INFINITY);
  }
  mx = warp_maxf(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
    if (mx > 0.f) atomicMax(&c.ctl[kCtlMove], __float_as_uint(mx));
    __threadfence();
    last = atomicAdd(&c.ctl[kCtlTicket], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  volatile uint32_t* ctl = c.ctl;
  const float moved = __uint_as_float(ctl[kCtlMove]);
  const bool rebuild = ctl[kCtlForce] != 0u || !(double(moved) + snap_slack(c) <= c.trig);
  ctl[kCtlRebuild] = rebuild ? 1u : 0u;
  ctl[kCtlAcc] = rebuild ? 0u : __float_as_uint(moved);
  // path bound: the sum of the sweeps' largest vertex steps since the rebuild (k_update
  // leaves the last one in kCtlStep), rounded up; no vertex has moved farther since then
  const float path = rebuild ? 0.f : __fadd_ru(__uint_as_float(ctl[kCtlPath]), __uint_as_float(ctl[kCtlStep]));
  ctl[kCtlPath] = __float_as_uint(path);
  ctl[kCtlStep] = 0u;
  ctl[kCtlMove] = 0u;
  ctl[kCtlForce] = 0u;
  ctl[kCtlTicket] = 0u;
  ctl[kCtlNear] = 0u;
  if (rebuild) {
    st->rebuilds += 1;
    *c.n_pairs = 0;
    ctl[kCtlExtF] = 0u;
    ctl[kCtlExtE] = 0u;
    ctl[kCtlCoord] = 0u;
  }
}

// Rebuild 1: FP32 snapshot of the surface positions, primitive extents, cleared buckets.
template <typename T>
__global__ void __launch_bounds__(256) k_bp_snapshot(DevMesh<T> m, ContactView c) {
  if (c.ctl[kCtlRebuild] == 0u) return;
  const int H2 = 2 << c.hbits;
  const int n = max(max(c.n_sverts, c.n_faces), max(c.n_edges, H2 + 1));
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const int q = base + threadIdx.x;
    float co = 0.f, ef = 0.f, ee = 0.f;
    if (q < c.n_sverts) {
      const int v = c.sverts[q];
      const P3 p = vpos(m, v);
      c.pbp[v] = make_float4(float(p.x), float(p.y), float(p.z), 0.f);
      co = __double2float_ru(fmax(fmax(fabs(p.x), fabs(p.y)), fabs(p.z)));
    }
    if (q < c.n_faces) {
      const P3 a = vpos(m, c.faces[3 * q]), b = vpos(m, c.faces[3 * q + 1]), d = vpos(m, c.faces[3 * q + 2]);
      const P3 g = mul(add(add(a, b), d), 1.0 / 3.0);
      ef = __double2float_ru(fmax(fmax(norm(sub(a, g)), norm(sub(b, g))), norm(sub(d, g))));
    }
    if (q < c.n_edges) {
      const P3 a = vpos(m, c.edges[2 * q]), b = vpos(m, c.edges[2 * q + 1]);
      ee = __double2float_ru(0.5 * norm(sub(a, b)) * (1.0 + 1e-12));
    }
    if (q <= H2) c.hcnt[q] = 0;
    warp_atomic_max(&c.ctl[kCtlCoord], co);
    warp_atomic_max(&c.ctl[kCtlExtF], ef);
    warp_atomic_max(&c.ctl[kCtlExtE], ee);
  }
}

// Rebuild 2: cell key and rank within its bucket of every face (centroid) and edge (midpoint).
template <typename T>
__global__ void __launch_bounds__(256) k_bp_keys(DevMesh<T> m, ContactView c) {
  if (c.ctl[kCtlRebuild] == 0u) return;
  double hf, he;
  grid_cells(c, hf, he);
  const int H = 1 << c.hbits;
  const int n = max(c.n_faces, c.n_edges);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    if (q < c.n_faces) {
      const P3 a = vpos(m, c.faces[3 * q]), b = vpos(m, c.faces[3 * q + 1]), d = vpos(m, c.faces[3 * q + 2]);
      const uint64_t key = cell_key(mul(add(add(a, b), d), 1.0 / 3.0), hf);
      c.fkeys[q] = key;
      c.frank[q] = atomicAdd(&c.hcnt[bucket_of(key, c.hbits)], 1);
    }
    if (q < c.n_edges) {
      const P3 a = vpos(m, c.edges[2 * q]), b = vpos(m, c.edges[2 * q + 1]);
      const uint64_t key = cell_key(mul(add(a, b), 0.5), he);
      c.ekeys[q] = key;
      c.erank[q] = atomicAdd(&c.hcnt[H + bucket_of(key, c.hbits)], 1);
    }
  }
}

// Exclusive scan of the bucket counts (2H + 1 entries, 4096 per block of 1024 threads).
__device__ __forceinline__ int block_excl_scan(int v, int* sh, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  total = sh[(blockDim.x >> 5) - 1];
  const int r = x - v + (w > 0 ? sh[w - 1] : 0);
  __syncthreads();
  return r;
}
static __global__ void __launch_bounds__(1024) k_bp_scan_blocks(ContactView c) {
  if (c.ctl[kCtlRebuild] == 0u) return;
  __shared__ int sh[32];
  const int n = (2 << c.hbits) + 1;
  const int base = blockIdx.x * 4096 + threadIdx.x * 4;
  int s = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) s += base + j < n ? c.hcnt[base + j] : 0;
  int total;
  block_excl_scan(s, sh, total);
  if (threadIdx.x == 0) c.hblk[blockIdx.x] = total;
}
static __global__ void __launch_bounds__(1024) k_bp_scan_top(ContactView c, int nblk) {
  if (c.ctl[kCtlRebuild] == 0u) return;
  __shared__ int sh[32];
  const int v = (int)threadIdx.x < nblk ? c.hblk[threadIdx.x] : 0;
  int total;
  const int e = block_excl_scan(v, sh, total);
  if ((int)threadIdx.x < nblk) c.hblk[threadIdx.x] = e;
}
static __global__ void __launch_bounds__(1024) k_bp_scan_apply(ContactView c) {
  if (c.ctl[kCtlRebuild] == 0u) return;
  __shared__ int sh[32];
  const int n = (2 << c.hbits) + 1;
  const int base = blockIdx.x * 4096 + threadIdx.x * 4;
  int v[4], s = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = base + j < n ? c.hcnt[base + j] : 0;
    s += v[j];
  }
  int total;
  int e = block_excl_scan(s, sh, total) + c.hblk[blockIdx.x];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (base + j < n) c.hcnt[base + j] = e;
    e += v[j];
  }
}

// Rebuild 3: in bucket order (faces, then edges), each primitive's id, its FP32 centre on the
// snapshot (face centroid, edge midpoint) and its cell key: the queries scan these three
// contiguous arrays and reject most candidates on the centre alone.
static __global__ void __launch_bounds__(256) k_bp_fill(ContactView c) {
  if (c.ctl[kCtlRebuild] == 0u) return;
  const int H = 1 << c.hbits;
  const int n = max(c.n_faces, c.n_edges);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    if (q < c.n_faces) {
      const int pos = c.hcnt[bucket_of(c.fkeys[q], c.hbits)] + c.frank[q];
      const float4 a = c.pbp[c.faces[3 * q]], b = c.pbp[c.faces[3 * q + 1]], d = c.pbp[c.faces[3 * q + 2]];
      c.hids[pos] = q;
      c.hrec[pos] = make_float4((a.x + b.x + d.x) / 3.f, (a.y + b.y + d.y) / 3.f, (a.z + b.z + d.z) / 3.f, 0.f);
      c.hkey[pos] = c.fkeys[q];
    }
    if (q < c.n_edges) {
      const int pos = c.hcnt[H + bucket_of(c.ekeys[q], c.hbits)] + c.erank[q];
      const float4 a = c.pbp[c.edges[2 * q]], b = c.pbp[c.edges[2 * q + 1]];
      c.hids[pos] = q;
      c.hrec[pos] = make_float4(0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z), 0.f);
      c.hkey[pos] = c.ekeys[q];
    }
  }
}

// Centre prefilter on the FP32 snapshot: false only when the centres are provably farther
// apart than r (r already holds the primitives' extents and the snapshot's rounding slack).
__device__ __forceinline__ bool centres_near(float4 a, float4 b, float r) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return dx * dx + dy * dy + dz * dz <= r * r;
}

// AABB gap test on the FP32 snapshot: false only when the boxes are provably farther than R
__device__ __forceinline__ bool boxes_near(float4 lo, float4 hi, float4 plo, float4 phi, float r) {
  const float gx = fmaxf(fmaxf(lo.x - phi.x, plo.x - hi.x), 0.f);
  const float gy = fmaxf(fmaxf(lo.y - phi.y, plo.y - hi.y), 0.f);
  const float gz = fmaxf(fmaxf(lo.z - phi.z, plo.z - hi.z), 0.f);
  return gx * gx + gy * gy + gz * gz < r * r;
}
__device__ __forceinline__ float4 fmin4(float4 a, float4 b) {
  return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), 0.f);
}
__device__ __forceinline__ float4 fmax4(float4 a, float4 b) {
  return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), 0.f);
}

// Rebuild 4: surface vertices against walls and faces (27 neighbouring cells), exact FP64
// distance below R.
template <typename T>
__global__ void __launch_bounds__(128) k_query_vertices(DevMesh<T> m, ContactView c) {
  if (c.ctl[kCtlRebuild] == 0u) return;
  double hf, he;
  grid_cells(c, hf, he);
  const float rf = float((c.R + 2.0 * snap_slack(c)) * (1.0 + 1e-6));
  // a face within R of a point has its centroid within R + (largest centroid-corner distance)
  const float rs = float((c.R + double(__uint_as_float(c.ctl[kCtlExtF])) + 8.0 * snap_slack(c)) * (1.0 + 1e-5));
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < c.n_sverts; q += gridDim.x * blockDim.x) {
    const int v = c.sverts[q];
    const P3 p = vpos(m, v);
    const float4 pf = c.pbp[v];
    for (int k = 0; k < c.n_planes; ++k) {
      const double d =
          c.planes[4 * k] * p.x + c.planes[4 * k + 1] * p.y + c.planes[4 * k + 2] * p.z - c.planes[4 * k + 3];
      if (d < c.R) emit_pair(c, 0, v, k, d);
    }
    const long long cx = (long long)floor(p.x / hf), cy = (long long)floor(p.y / hf), cz = (long long)floor(p.z / hf);
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          const uint64_t key = cell_key_of(cx + dx, cy + dy, cz + dz);
          const uint32_t b = bucket_of(key, c.hbits);
          const int j1 = c.hcnt[b + 1];
          for (int j = c.hcnt[b]; j < j1; ++j) {
            if (!centres_near(c.hrec[j], pf, rs) || c.hkey[j] != key) continue;
            const int f = c.hids[j];
            const int a = c.faces[3 * f], bb = c.faces[3 * f + 1], cc = c.faces[3 * f + 2];
            if (a == v || bb == v || cc == v) continue;
            const float4 fa = c.pbp[a], fb = c.pbp[bb], fc = c.pbp[cc];
            if (!boxes_near(fmin4(fmin4(fa, fb), fc), fmax4(fmax4(fa, fb), fc), pf, pf, rf)) continue;
            double w[3];
            const double d = point_triangle(p, vpos(m, a), vpos(m, bb), vpos(m, cc), w);
            if (d < c.R) emit_pair(c, 1, v, f, d);
          }
        }
  }
}

// Rebuild 5: edge pairs sharing no vertex (each unordered pair once), exact FP64 distance
// below R.
template <typename T>
__global__ void __launch_bounds__(128) k_query_edges(DevMesh<T> m, ContactView c) {
  if (c.ctl[kCtlRebuild] == 0u) return;
  double hf, he;
  grid_cells(c, hf, he);
  const float rf = float((c.R + 2.0 * snap_slack(c)) * (1.0 + 1e-6));
  // two edges within R have midpoints within R + 2 (largest half length)
  const float rs =
      float((c.R + 2.0 * double(__uint_as_float(c.ctl[kCtlExtE])) + 8.0 * snap_slack(c)) * (1.0 + 1e-5));
  const int H = 1 << c.hbits;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.n_edges; i += gridDim.x * blockDim.x) {
    const int a0 = c.edges[2 * i], a1 = c.edges[2 * i + 1];
    const P3 p0 = vpos(m, a0), p1 = vpos(m, a1);
    const float4 f0 = c.pbp[a0], f1 = c.pbp[a1];
    const float4 lo = fmin4(f0, f1), hi = fmax4(f0, f1);
    const float4 mf = make_float4(0.5f * (f0.x + f1.x), 0.5f * (f0.y + f1.y), 0.5f * (f0.z + f1.z), 0.f);
    const P3 mid = mul(add(p0, p1), 0.5);
    const long long cx = (long long)floor(mid.x / he), cy = (long long)floor(mid.y / he),
                    cz = (long long)floor(mid.z / he);
    // half stencil: the own cell (partners e > i) and the 13 cells after it in (dx, dy, dz)
    // order (every partner); each unordered pair of cells is visited from one side only
    for (int cell = 13; cell < 27; ++cell) {
      const int dx = cell / 9 - 1, dy = (cell / 3) % 3 - 1, dz = cell % 3 - 1;
      const bool own = cell == 13;
      const uint64_t key = cell_key_of(cx + dx, cy + dy, cz + dz);
      const uint32_t b = H + bucket_of(key, c.hbits);
      const int j1 = c.hcnt[b + 1];
      for (int j = c.hcnt[b]; j < j1; ++j) {
        if (!centres_near(c.hrec[j], mf, rs) || c.hkey[j] != key) continue;
        const int e = c.hids[j];
        if (own && e <= i) continue;
        const int b0 = c.edges[2 * e], b1 = c.edges[2 * e + 1];
        if (b0 == a0 || b0 == a1 || b1 == a0 || b1 == a1) continue;
        const float4 g0 = c.pbp[b0], g1 = c.pbp[b1];
        if (!boxes_near(lo, hi, fmin4(g0, g1), fmax4(g0, g1), rf)) continue;
        double s, t;
        const double d = segment_segment(p0, p1, vpos(m, b0), vpos(m, b1), s, t);
        if (d < c.R) emit_pair(c, 2, i, e, d);
      }
    }
  }
}

// Length of the step d of vertex v (0 for pinned vertices, which never move).
template <typename T>
__device__ __forceinline__ double step_len(const DevMesh<T>& m, int v, const Vec4<T>* D) {
  if (v >= m.Vf) return 0.0;
  const Vec4<T> d = D[v];
  return sqrt(double(d.x) * double(d.x) + double(d.y) * double(d.y) + double(d.z) * double(d.z));
}

// Bound on how much a pair's distance can shrink along a d (0 < a <= 1): the distance of a
// point to a plane, of a point to a triangle and of two segments is 1-Lipschitz in each
// side's motion, and a closest point on a triangle or segment is a convex combination of
// its corners, so d(x + a d) >= d(x) - (max step on one side + max step on the other).
template <typename T>
__device__ __forceinline__ double pair_motion(const DevMesh<T>& m, const ContactView& c, uint64_t key,
                                              const Vec4<T>* D) {
  const int kind = (int)(key >> 60), ia = (int)((key >> 30) & 0x3fffffff), ib = (int)(key & 0x3fffffff);
  if (kind == 0) return step_len(m, ia, D);
  if (kind == 1) {
    const int f0 = c.faces[3 * ib], f1 = c.faces[3 * ib + 1], f2 = c.faces[3 * ib + 2];
    return step_len(m, ia, D) + fmax(step_len(m, f0, D), fmax(step_len(m, f1, D), step_len(m, f2, D)));
  }
  const int e0 = c.edges[2 * ia], e1 = c.edges[2 * ia + 1], g0 = c.edges[2 * ib], g1 = c.edges[2 * ib + 1];
  return fmax(step_len(m, e0, D), step_len(m, e1, D)) + fmax(step_len(m, g0, D), step_len(m, g1, D));
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

// Displacement of surface vertex v since the last rebuild (current position minus the FP32
// snapshot; the snapshot's rounding is covered by snap_slack).
template <typename T>
__device__ __forceinline__ float3 snap_disp(const DevMesh<T>& m, const ContactView& c, int v) {
  const P3 p = vpos(m, v);
  const float4 s = c.pbp[v];
  return make_float3(float(p.x - double(s.x)), float(p.y - double(s.y)), float(p.z - double(s.z)));
}
__device__ __forceinline__ float dist3(float3 a, float3 b) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return sqrtf(dx * dx + dy * dy + dz * dz);
}

// Bound on how much a pair's distance changed since the last rebuild, from its vertices'
// motion relative to one of them: a common translation leaves every distance unchanged,
// and the point-plane, point-triangle and segment-segment distances are 1-Lipschitz in the
// relative motion (closest points on a triangle or segment are convex combinations of its
// corners). Walls do not move, so a vertex-wall pair takes the vertex's own motion.
template <typename T>
__device__ __forceinline__ float pair_rel_motion(const DevMesh<T>& m, const ContactView& c, uint64_t key) {
  const int kind = (int)(key >> 60), ia = (int)((key >> 30) & 0x3fffffff), ib = (int)(key & 0x3fffffff);
  if (kind == 0) {
    const float3 d = snap_disp(m, c, ia);
    return sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
  }
  if (kind == 1) {
    const float3 r = snap_disp(m, c, ia);
    return fmaxf(dist3(snap_disp(m, c, c.faces[3 * ib]), r),
                 fmaxf(dist3(snap_disp(m, c, c.faces[3 * ib + 1]), r), dist3(snap_disp(m, c, c.faces[3 * ib + 2]), r)));
  }
  const float3 r = snap_disp(m, c, c.edges[2 * ia]);
  return dist3(snap_disp(m, c, c.edges[2 * ia + 1]), r) +
         fmaxf(dist3(snap_disp(m, c, c.edges[2 * ib]), r), dist3(snap_disp(m, c, c.edges[2 * ib + 1]), r));
}

// Per candidate pair: its distance at x^k. Pairs within r_c count: smallest distance per
// vertex, and for active pairs (d < dhat) kappa B'(d) dd/dx and kappa B''(d) (dd/dx)(dd/dx)^T
// into the FP64 accumulators. A pair whose rebuild distance exceeds r_c by more than its
// distance can have changed since the rebuild (twice the largest displacement, or its own
// vertices' relative motion) cannot be within r_c and is skipped (d0 = inf).
template <typename T>
__global__ void __launch_bounds__(256) k_pair_terms(DevMesh<T> m, ContactView c, StepState* st) {
  if (st->done) return;
  const int n = min(*c.n_pairs, c.cap);
  const double far = c.rc + 2.0 * (double(__uint_as_float(c.ctl[kCtlAcc])) + snap_slack(c));
  const float path = __uint_as_float(c.ctl[kCtlPath]);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const double dbp = double(c.dbp[q]);
    // beyond r_c by more than any motion since the rebuild could close: global bound
    // first (one load)
    if (dbp >= far) {
      c.d0[q] = INFINITY;
      continue;
    }
    // then the margin found at the pair's last motion check, less what the motion since
    // then can have taken from it: every vertex has moved at most (path - ppath) since,
    // and the pair's relative-motion bound grows by at most 4 times that (edge-edge: two
    // relative displacements, each by at most twice the motion)
    const float mq = c.pmarg[q];
    if (mq >= 0.f && double(mq) - 4.0 * (double(path) - double(c.ppath[q])) * (1.0 + 1e-5) >= 0.0) {
      c.d0[q] = INFINITY;
      continue;
    }
    // then the pair's own motion relative to one of its vertices since the rebuild
    const double marg =
        dbp - double(pair_rel_motion(m, c, c.pairs[q])) * (1.0 + 1e-5) - 4.0 * snap_slack(c) - c.rc;
    if (marg >= 0.0) {
      c.pmarg[q] = __double2float_rd(marg);
      c.ppath[q] = path;
      c.d0[q] = INFINITY;
      continue;
    }
    c.pmarg[q] = -1.f;
    int vs[4], nv;
    P3 J[4];
    const double d = pair_geom(m, c, c.pairs[q], 0.0, (const Vec4<T>*)nullptr, vs, J, nv);
    c.d0[q] = d;
    if (!(d > 0.0)) {
      c.flags[1] = 1;
      st->status = 9;  // JGS2_EINTERSECT
      st->done = 1;
      continue;
    }
    if (d >= c.rc) continue;
    atomicAdd(&c.ctl[kCtlNear], 1u);  // pairs within r_c at this sweep (diagnostic)
    // positive doubles order like their bit patterns
    for (int k = 0; k < nv; ++k)
      atomicMin(reinterpret_cast<unsigned long long*>(c.dmin + vs[k]), (unsigned long long)__double_as_longlong(d));
    if (d >= c.dhat) continue;
    if (c.vp_cnt) {
      // an active pair that reaches another body: listed at each of its vertices
      bool cross = false;
      for (int k = 1; k < nv; ++k) cross |= c.body[vs[k]] != c.body[vs[0]];
      if (cross)
        for (int k = 0; k < nv; ++k) {
          const int slot = atomicAdd(c.vp_cnt + vs[k], 1);
          if (slot < kMaxVertexPairs)
            c.vp[(size_t)vs[k] * kMaxVertexPairs + slot] = q;
          else
            c.flags[2] = 1;
        }
    }
    const double b1 = c.kappa * barrier_b1(d, c.dhat, c.pen), b2 = c.kappa * barrier_b2(d, c.dhat, c.pen);
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
}

// Contact-aware local terms (Sec. 7, reading R24), thread per free vertex after the gather:
// a vertex with active pairs reaching other bodies moves, in its sub-problem, together with
// those bodies' free colliding vertices P(i). With S_i = {i} + P(i):
//   g' = g_i - sum_l kappa B'(d_l) J_i,l + sum_l kappa B'(d_l) J_S,l + sum_{b in P} (g_b - bg_b)
//   H' = H_ii - sum_l kappa B'' J_i J_i^T + sum_l kappa B'' J_S J_S^T + sum_{b in P} (H_bb - bH_b)
// over the vertex's listed pairs l (J_S,l: the pair's distance gradients summed over its
// vertices in S_i), written to cpl for k_correct's local system. Pairs are taken in
// ascending order, so the sums do not depend on the order the lists were filled.
template <typename T>
__global__ void __launch_bounds__(128) k_couple(DevMesh<T> m, ContactView c, const StepState* __restrict__ st) {
  if (st->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.Vf) return;
  const int n = c.vp_cnt[i] < kMaxVertexPairs ? c.vp_cnt[i] : kMaxVertexPairs;
  m.cpl_on[i] = n > 0 ? 1 : 0;
  if (n == 0) return;
  int lst[kMaxVertexPairs];
  for (int k = 0; k < n; ++k) lst[k] = c.vp[(size_t)i * kMaxVertexPairs + k];
  for (int a = 1; a < n; ++a) {  // insertion sort (at most kMaxVertexPairs entries)
    const int v = lst[a];
    int b = a - 1;
    while (b >= 0 && lst[b] > v) {
      lst[b + 1] = lst[b];
      --b;
    }
    lst[b + 1] = v;
  }
  const int bi = c.body[i];
  const size_t S = m.Vf, V = m.V;
  double g[3], H[6];
  for (int q = 0; q < 3; ++q) g[q] = double(m.ghr[q * S + i]);
  for (int q = 0; q < 6; ++q) H[q] = double(m.ghr[(3 + q) * S + i]);
  int part[4 * kMaxVertexPairs];
  int np = 0;
  for (int k = 0; k < n; ++k) {
    int vs[4], nv;
    P3 J[4];
    const double d = pair_geom(m, c, c.pairs[lst[k]], 0.0, (const Vec4<T>*)nullptr, vs, J, nv);
    const double b1 = c.kappa * barrier_b1(d, c.dhat, c.pen), b2 = c.kappa * barrier_b2(d, c.dhat, c.pen);
    P3 Ji{0, 0, 0}, JS{0, 0, 0};
    for (int q = 0; q < nv; ++q) {
      const int v = vs[q];
      if (v == i) {
        Ji = add(Ji, J[q]);
        JS = add(JS, J[q]);
      } else if (c.body[v] != bi && v < m.Vf) {
        JS = add(JS, J[q]);
        bool seen = false;
        for (int r = 0; r < np; ++r) seen |= part[r] == v;
        if (!seen) part[np++] = v;
      }
    }
    g[0] += b1 * (JS.x - Ji.x);
    g[1] += b1 * (JS.y - Ji.y);
    g[2] += b1 * (JS.z - Ji.z);
    H[0] += b2 * (JS.x * JS.x - Ji.x * Ji.x);
    H[1] += b2 * (JS.x * JS.y - Ji.x * Ji.y);
    H[2] += b2 * (JS.x * JS.z - Ji.x * Ji.z);
    H[3] += b2 * (JS.y * JS.y - Ji.y * Ji.y);
    H[4] += b2 * (JS.y * JS.z - Ji.y * Ji.z);
    H[5] += b2 * (JS.z * JS.z - Ji.z * Ji.z);
  }
  // partners in ascending order: a fixed summation order
  for (int a = 1; a < np; ++a) {
    const int v = part[a];
    int b = a - 1;
    while (b >= 0 && part[b] > v) {
      part[b + 1] = part[b];
      --b;
    }
    part[b + 1] = v;
  }
  for (int r = 0; r < np; ++r) {
    const int b = part[r];
    for (int q = 0; q < 3; ++q) g[q] += double(m.ghr[q * S + b]) - c.bg[q * V + b];
    for (int q = 0; q < 6; ++q) H[q] += double(m.ghr[(3 + q) * S + b]) - c.bH[q * V + b];
  }
  for (int q = 0; q < 3; ++q) m.cpl[q * S + i] = T(g[q]);
  for (int q = 0; q < 6; ++q) m.cpl[(3 + q) * S + i] = T(H[q]);
}

// Friction terms at x^k, after k_pair_terms (thread per surface vertex): the gradient
// mu lam f1(y)/y u_t and the diagonal block mu lam [(f1/y) P + ((f1' y - f1)/y^3) u_t u_t^T]
// (positive semidefinite on both branches of f0), added to the vertex's contact sums.
template <typename T>
__global__ void __launch_bounds__(256) k_friction_terms(DevMesh<T> m, ContactView c, const StepState* st) {
  if (st->done) return;
  const size_t V = c.n_vertices;
  const double e = c.feps;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < c.n_sverts; q += gridDim.x * blockDim.x) {
    const int v = c.sverts[q];
    if (v >= m.Vf) continue;
    const Vec4<T> uv = m.u[v];
    const double u[3] = {double(uv.x), double(uv.y), double(uv.z)};
    for (int p = 0; p < c.n_planes; ++p) {
      const double lam = c.fr_lam[(size_t)p * V + v];
      if (!(lam > 0.0)) continue;
      const double* n = c.planes + 4 * p;
      double ut[3];
      fric_tangential(n, u, ut);
      const double y = fric_norm(ut);
      const double k = c.fmu * lam, fy = fric_f1_over_y(y, e);
      const double c2 = y == 0.0 ? 0.0 : (y < e ? -1.0 / (e * e * y) : -1.0 / (y * y * y));
#pragma unroll
      for (int a = 0; a < 3; ++a) c.bg[(size_t)a * V + v] += k * fy * ut[a];
      // packed xx xy xz yy yz zz of k (fy (I - n n^T) + c2 ut ut^T)
      const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        const int a = ia[r], b = ib[r];
        c.bH[(size_t)r * V + v] += k * (fy * ((a == b ? 1.0 : 0.0) - n[a] * n[b]) + c2 * ut[a] * ut[b]);
      }
    }
  }
}

// Friction energy of surface vertex v at displacement u (sum over its walls).
__device__ __forceinline__ double fric_energy_at(const ContactView& c, int v, const double (&u)[3]) {
  const size_t V = c.n_vertices;
  double e = 0.0;
  for (int p = 0; p < c.n_planes; ++p) {
    const double lam = c.fr_lam[(size_t)p * V + v];
    if (!(lam > 0.0)) continue;
    double ut[3];
    fric_tangential(c.planes + 4 * p, u, ut);
    e += c.fmu * lam * fric_f0(fric_norm(ut), c.feps);
  }
  return e;
}

// barrier energy of the pairs at x^k, plus the friction energy (for jgs2_energy_gradient)
template <typename T>
__global__ void k_pair_energy(DevMesh<T> m, ContactView c, double* out) {
  __shared__ double red[32];
  const int n = min(*c.n_pairs, c.cap);
  double acc[1] = {0.0};
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
    acc[0] += c.kappa * barrier_b(c.d0[q], c.dhat, c.pen);
  if (c.fr_lam) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < c.n_sverts; q += gridDim.x * blockDim.x) {
      const int v = c.sverts[q];
      if (v >= m.Vf) continue;
      const Vec4<T> uv = m.u[v];
      const double u[3] = {double(uv.x), double(uv.y), double(uv.z)};
      acc[0] += fric_energy_at(c, v, u);
    }
  }
  block_sum<1>(acc, red);
  if (threadIdx.x == 0) atomicAdd(out, acc[0]);
}

}  // namespace jgs2
