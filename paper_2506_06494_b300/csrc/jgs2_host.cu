// Host side of the JGS2 library: C ABI, mesh ingest and reordering, the step driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <memory>
#include <numeric>
#include <set>
#include <string>
#include <vector>

#include <map>

#include "../../include/jgs2.h"
#include "jgs2_adjoint.cuh"
#include "jgs2_host.h"
#include "jgs2_kernels.cuh"
#include "jgs2_persistent.cuh"

namespace jgs2 {

thread_local std::string g_last_error;

jgs2_status fail(jgs2_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? JGS2_ENOMEM : JGS2_ECUDA,         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

template <typename X>
static cudaError_t dalloc(X** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc((void**)p, n * sizeof(X));
}

template <typename T>
void PrecBufs<T>::release() {
  cudaFree(tets); cudaFree(frec); cudaFree(bc); cudaFree(u); cudaFree(dz); cudaFree(D); cudaFree(DJ); cudaFree(ghr); cudaFree(mh2);
  cudaFree(cub_p); cudaFree(cub_w); cudaFree(cub_u); cudaFree(pool_H); cudaFree(pool_G); cudaFree(pool_R);
  cudaFree(cpl);
  cudaFree(a_lam); cudaFree(a_r); cudaFree(a_z); cudaFree(a_p); cudaFree(a_q); cudaFree(a_lin);
  *this = PrecBufs<T>();
}
template struct PrecBufs<float>;
template struct PrecBufs<double>;

Mesh::~Mesh() {
  f32.release();
  f64.release();
  cudaFree(d_inc_off); cudaFree(d_inc_len); cudaFree(d_inc); cudaFree(d_pool_tet);
  cudaFree(d_xt); cudaFree(d_vt); cudaFree(d_perm); cudaFree(d_state); cudaFree(d_partial);
  cudaFree(d_trace); cudaFree(d_xbuf); cudaFree(d_vbuf); cudaFree(d_tperm); cudaFree(d_youngs); cudaFree(d_coup);
  cudaFree(d_adjsc);
  if (h_state) cudaFreeHost(h_state);
  for (cudaEvent_t e : events) cudaEventDestroy(e);
  for (cudaEvent_t e : gevents) cudaEventDestroy(e);
  if (graph) cudaGraphExecDestroy(graph);
  if (gstream) cudaStreamDestroy(gstream);
  if (gstream2) cudaStreamDestroy(gstream2);
  for (cudaEvent_t e : gfork)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : gev)
    if (e) cudaEventDestroy(e);
  cudaFree(d_vscene); cudaFree(d_tscene); cudaFree(d_ndone); cudaFree(d_scenes); cudaFree(d_sacc);
  cudaFree(d_gbar);
  cudaFree(d_planes); cudaFree(d_d0); cudaFree(d_bg); cudaFree(d_bH); cudaFree(d_faces); cudaFree(d_edges);
  cudaFree(d_sverts); cudaFree(d_npairs); cudaFree(d_cflags); cudaFree(d_is_surf); cudaFree(d_pairs);
  cudaFree(d_fr_lam);
  cudaFree(d_dmin); cudaFree(d_lim); cudaFree(d_body); cudaFree(d_vp_cnt); cudaFree(d_vp); cudaFree(d_cpl_on); cudaFree(d_frank); cudaFree(d_erank); cudaFree(d_hcnt); cudaFree(d_hblk);
  cudaFree(d_hids); cudaFree(d_hrec); cudaFree(d_hkey); cudaFree(d_fkeys); cudaFree(d_ekeys); cudaFree(d_pbp); cudaFree(d_dbp); cudaFree(d_ctl);
  cudaFree(d_pmarg); cudaFree(d_ppath);
  cudaFree(d_gsmask); cudaFree(d_vmask); cudaFree(d_gs_xt); cudaFree(d_gs_xk); cudaFree(d_gs_g);
}

static uint64_t spread3(uint64_t x) {
  x &= 0x1fffff;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}

// ------------------------------------------------------------------ mesh create

jgs2_status mesh_create(const jgs2_mesh_desc* d, Mesh** out, const std::vector<int>* scene_of_vertex = nullptr) {
  if (!d || !out) return fail(JGS2_EINVAL, "null argument");
  *out = nullptr;
  const int V = d->n_vertices, T = d->n_tets;
  if (V <= 0 || T <= 0) return fail(JGS2_EINVAL, "n_vertices and n_tets must be positive");
  if (!d->rest_pos || !d->tets || !d->youngs || !d->poisson || !d->density)
    return fail(JGS2_EINVAL, "null mesh array");
  if (!(d->dt > 0.0) || !std::isfinite(d->dt)) return fail(JGS2_EINVAL, "dt must be positive");
  std::unique_ptr<Mesh> m(new Mesh());
  m->V = V;
  m->T = T;
  m->h = d->dt;
  for (int q = 0; q < 3; ++q) m->grav[q] = d->gravity[q];
  m->X.assign(d->rest_pos, d->rest_pos + 3 * (size_t)V);
  m->tets_c.assign(d->tets, d->tets + 4 * (size_t)T);
  m->E.assign(d->youngs, d->youngs + T);
  m->nu.assign(d->poisson, d->poisson + T);
  m->rho.assign(d->density, d->density + T);
  m->pinned.assign(V, 0);
  if (d->pinned)
    for (int v = 0; v < V; ++v) m->pinned[v] = d->pinned[v] ? 1 : 0;
  for (int v = 0; v < 3 * V; ++v)
    if (!std::isfinite(m->X[v])) return fail(JGS2_EINVAL, "non-finite rest position");
  for (int q = 0; q < 3; ++q) {
    double lo = m->X[q], hi = m->X[q];
    for (int v = 1; v < V; ++v) {
      lo = std::min(lo, m->X[3 * (size_t)v + q]);
      hi = std::max(hi, m->X[3 * (size_t)v + q]);
    }
    m->extent = std::max(m->extent, hi - lo);
  }
  // rest data (FP64): B = D_m^{-1}, V_e, Lame, mass shares
  m->B.resize(9 * (size_t)T);
  m->vol.resize(T);
  m->mu.resize(T);
  m->lp.resize(T);
  m->mass.assign(V, 0.0);
  for (int t = 0; t < T; ++t) {
    const int* tv = &m->tets_c[4 * (size_t)t];
    for (int a = 0; a < 4; ++a)
      if (tv[a] < 0 || tv[a] >= V) return fail(JGS2_EINVAL, "tet index out of range at tet " + std::to_string(t));
    if (!(m->E[t] > 0) || !(m->nu[t] > -1.0 && m->nu[t] < 0.5) || !(m->rho[t] > 0))
      return fail(JGS2_EINVAL, "material out of range at tet " + std::to_string(t));
    double Dm[9];
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 3; ++i) Dm[3 * i + k] = m->X[3 * tv[k + 1] + i] - m->X[3 * tv[0] + i];
    const double c00 = Dm[4] * Dm[8] - Dm[5] * Dm[7], c01 = Dm[5] * Dm[6] - Dm[3] * Dm[8],
                 c02 = Dm[3] * Dm[7] - Dm[4] * Dm[6];
    const double det = Dm[0] * c00 + Dm[1] * c01 + Dm[2] * c02;
    if (!(det > 0.0)) return fail(JGS2_EINVAL, "non-positive tet volume at tet " + std::to_string(t));
    double* B = &m->B[9 * (size_t)t];
    B[0] = c00 / det;
    B[1] = (Dm[2] * Dm[7] - Dm[1] * Dm[8]) / det;
    B[2] = (Dm[1] * Dm[5] - Dm[2] * Dm[4]) / det;
    B[3] = c01 / det;
    B[4] = (Dm[0] * Dm[8] - Dm[2] * Dm[6]) / det;
    B[5] = (Dm[2] * Dm[3] - Dm[0] * Dm[5]) / det;
    B[6] = c02 / det;
    B[7] = (Dm[1] * Dm[6] - Dm[0] * Dm[7]) / det;
    B[8] = (Dm[0] * Dm[4] - Dm[1] * Dm[3]) / det;
    m->vol[t] = det / 6.0;
    const double E = m->E[t], nu = m->nu[t];
    m->mu[t] = E / (2.0 * (1.0 + nu));
    m->lp[t] = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)) + m->mu[t];
    for (int a = 0; a < 4; ++a) m->mass[tv[a]] += m->rho[t] * m->vol[t] / 4.0;
  }
  // a free vertex outside every tet would have no mass and no elastic term (a singular
  // 3x3 system): an input error
  for (int v = 0; v < V; ++v)
    if (!m->pinned[v] && !(m->mass[v] > 0.0))
      return fail(JGS2_EINVAL, "free vertex " + std::to_string(v) + " belongs to no tet");
  // internal order: free vertices along a Morton curve, then pinned vertices
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v = 0; v < V; ++v)
    for (int q = 0; q < 3; ++q) {
      lo[q] = std::min(lo[q], m->X[3 * v + q]);
      hi[q] = std::max(hi[q], m->X[3 * v + q]);
    }
  double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
  std::vector<uint64_t> key(V);
  for (int v = 0; v < V; ++v) {
    uint64_t c[3];
    for (int q = 0; q < 3; ++q) c[q] = (uint64_t)std::min(2097151.0, std::floor((m->X[3 * v + q] - lo[q]) / ext * 2097151.0));
    key[v] = spread3(c[0]) | spread3(c[1]) << 1 | spread3(c[2]) << 2;
  }
  m->perm.resize(V);
  std::iota(m->perm.begin(), m->perm.end(), 0);
  std::stable_sort(m->perm.begin(), m->perm.end(), [&](int a, int b) {
    if (m->pinned[a] != m->pinned[b]) return m->pinned[a] < m->pinned[b];
    if (scene_of_vertex && (*scene_of_vertex)[a] != (*scene_of_vertex)[b])
      return (*scene_of_vertex)[a] < (*scene_of_vertex)[b];
    return key[a] < key[b];
  });
  m->iperm.resize(V);
  for (int i = 0; i < V; ++i) m->iperm[m->perm[i]] = i;
  m->Vf = 0;
  while (m->Vf < V && !m->pinned[m->perm[m->Vf]]) ++m->Vf;
  // tets in internal ids, sorted by smallest corner
  m->tperm.resize(T);
  std::iota(m->tperm.begin(), m->tperm.end(), 0);
  std::vector<int> tmin(T);
  for (int t = 0; t < T; ++t) {
    int mn = V;
    for (int a = 0; a < 4; ++a) mn = std::min(mn, m->iperm[m->tets_c[4 * (size_t)t + a]]);
    tmin[t] = mn;
  }
  std::stable_sort(m->tperm.begin(), m->tperm.end(), [&](int a, int b) { return tmin[a] < tmin[b]; });
  m->tiperm.resize(T);
  for (int i = 0; i < T; ++i) m->tiperm[m->tperm[i]] = i;
  // incidence of free vertices, in internal tet order
  std::vector<int> cnt(m->Vf, 0);
  for (int ti = 0; ti < T; ++ti) {
    const int t = m->tperm[ti];
    for (int a = 0; a < 4; ++a) {
      const int v = m->iperm[m->tets_c[4 * (size_t)t + a]];
      if (v < m->Vf) cnt[v]++;
    }
  }
  const int ns = (m->Vf + kSlice - 1) / kSlice;
  m->n_slices = ns;
  m->inc_off.assign(ns + 1, 0);
  for (int s = 0; s < ns; ++s) {
    int mx = 0;
    for (int l = 0; l < kSlice && s * kSlice + l < m->Vf; ++l) mx = std::max(mx, cnt[s * kSlice + l]);
    m->inc_off[s + 1] = m->inc_off[s] + mx * kSlice;
  }
  for (int q = 0; q < 4; ++q) {
    const int spb = (q < 3 ? (64 << q) : 32) / kSlice;  // slices per block of 64, 128, 256, 32 vertices
    for (int s0 = 0; s0 < ns; s0 += spb)
      m->inc_blk[q] = std::max(m->inc_blk[q], m->inc_off[std::min(s0 + spb, ns)] - m->inc_off[s0]);
  }
  m->inc.assign(m->inc_off[ns], 0);
  m->inc_len.assign(m->Vf, 0);
  for (int ti = 0; ti < T; ++ti) {
    const int t = m->tperm[ti];
    for (int a = 0; a < 4; ++a) {
      const int v = m->iperm[m->tets_c[4 * (size_t)t + a]];
      if (v >= m->Vf) continue;
      const int s = v / kSlice, l = v % kSlice;
      m->inc[m->inc_off[s] + m->inc_len[v] * kSlice + l] = ti * 4 + a;
      m->inc_len[v]++;
    }
  }
  // bodies: connected components, numbered by smallest caller vertex index
  {
    std::vector<int> par(V);
    std::iota(par.begin(), par.end(), 0);
    auto find = [&](int a) {
      while (par[a] != a) a = par[a] = par[par[a]];
      return a;
    };
    for (int t = 0; t < T; ++t) {
      const int r0 = find(m->tets_c[4 * (size_t)t]);
      for (int a = 1; a < 4; ++a) {
        const int r = find(m->tets_c[4 * (size_t)t + a]);
        if (r != r0) par[r] = r0;
      }
    }
    std::vector<int> id(V, -1);
    m->body.assign(V, 0);
    int nb = 0;
    for (int v = 0; v < V; ++v) {
      const int r = find(v);
      if (id[r] < 0) id[r] = nb++;
      m->body[v] = id[r];
    }
    m->n_bodies = nb;
  }
  // contact surface (Sec. 7): boundary faces (used by one tet) oriented outward, their
  // edges and vertices, in internal vertex ids
  if (d->contact < 0 || d->contact > 2) return fail(JGS2_EINVAL, "contact must be 0, 1 (IPC) or 2 (penalty)");
  if (!(d->friction_mu >= 0.0) || !std::isfinite(d->friction_mu))
    return fail(JGS2_EINVAL, "friction_mu must be finite and >= 0");
  if (d->friction_mu > 0.0) {
    if (!d->contact) return fail(JGS2_EINVAL, "friction needs contact (the walls' normal forces)");
    if (!(d->friction_eps_v > 0.0) || !std::isfinite(d->friction_eps_v))
      return fail(JGS2_EINVAL, "friction_eps_v must be finite and > 0");
    m->fmu = d->friction_mu;
    m->feps_v = d->friction_eps_v;
  }
  if (d->contact) {
    if (!(d->dhat > 0.0) || !(d->kappa > 0.0) || d->n_planes < 0 || (d->n_planes > 0 && !d->planes))
      return fail(JGS2_EINVAL, "contact needs dhat > 0, kappa > 0 and n_planes planes");
    m->contact = 1;
    m->penalty = d->contact == 2 ? 1 : 0;
    m->dhat = d->dhat;
    m->kappa = d->kappa;
    m->rc = 2.0 * d->dhat;
    m->planes.assign(d->planes, d->planes + 4 * (size_t)d->n_planes);
    for (int p = 0; p < d->n_planes; ++p) {
      const double* pl = &m->planes[4 * (size_t)p];
      const double nn = std::sqrt(pl[0] * pl[0] + pl[1] * pl[1] + pl[2] * pl[2]);
      if (!std::isfinite(pl[3]) || !(std::fabs(nn - 1.0) <= 1e-9))
        return fail(JGS2_EINVAL, "wall " + std::to_string(p) + ": the normal must be a unit vector, the offset finite");
    }
    std::map<std::array<int, 3>, std::pair<std::array<int, 3>, int>> fc;
    std::map<std::array<int, 3>, int> count;
    for (int t = 0; t < T; ++t) {
      const int* tv = &m->tets_c[4 * (size_t)t];
      for (int k = 0; k < 4; ++k) {
        std::array<int, 3> f;
        int q = 0;
        for (int a = 0; a < 4; ++a)
          if (a != k) f[q++] = tv[a];
        std::array<int, 3> key = f;
        std::sort(key.begin(), key.end());
        if (++count[key] == 1) fc[key] = {f, tv[k]};
      }
    }
    std::set<std::pair<int, int>> es;
    std::vector<uint8_t> surf(V, 0);
    double rmax = 0.0;
    for (auto& kv : count) {
      if (kv.second != 1) continue;
      auto f = fc[kv.first].first;
      const int opp = fc[kv.first].second;
      const double* a = &m->X[3 * f[0]];
      const double* b = &m->X[3 * f[1]];
      const double* c = &m->X[3 * f[2]];
      const double* o = &m->X[3 * opp];
      const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      const double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
      if (n[0] * (o[0] - a[0]) + n[1] * (o[1] - a[1]) + n[2] * (o[2] - a[2]) > 0) std::swap(f[1], f[2]);
      double cen[3];
      for (int q = 0; q < 3; ++q) cen[q] = (a[q] + b[q] + c[q]) / 3.0;
      for (int r = 0; r < 3; ++r) {
        const double* pr = &m->X[3 * f[r]];
        rmax = std::max(rmax, std::sqrt((pr[0] - cen[0]) * (pr[0] - cen[0]) + (pr[1] - cen[1]) * (pr[1] - cen[1]) +
                                        (pr[2] - cen[2]) * (pr[2] - cen[2])));
        const int x0 = f[r], x1 = f[(r + 1) % 3];
        es.insert({std::min(x0, x1), std::max(x0, x1)});
        surf[f[r]] = 1;
      }
      for (int r = 0; r < 3; ++r) m->sfaces.push_back(m->iperm[f[r]]);
    }
    for (auto& e : es) {
      m->sedges.push_back(m->iperm[e.first]);
      m->sedges.push_back(m->iperm[e.second]);
      const double* a = &m->X[3 * e.first];
      const double* b = &m->X[3 * e.second];
      rmax = std::max(rmax, std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) +
                                      (a[2] - b[2]) * (a[2] - b[2])));
    }
    m->is_surf.assign(V, 0);
    for (int v = 0; v < V; ++v)
      if (surf[v]) {
        m->sverts.push_back(m->iperm[v]);
        m->is_surf[m->iperm[v]] = 1;
      }
    // candidate list radius R = r_c + 2M, rebuilt once a surface vertex has moved more than M
    // since the last rebuild; M = 2 delta, delta = 0.45 (r_c - dhat) the per-sweep step limit
    // (a list then lasts at least two sweeps of the largest possible motion)
    const double delta = 0.45 * (m->rc - m->dhat);
    m->bp_R = m->rc + 4.0 * delta;
    m->bp_trig = 2.0 * delta * (1.0 - 1e-6);
    (void)rmax;
    const int nprim = std::max<int>(std::max<int>((int)m->sfaces.size() / 3, (int)m->sedges.size() / 2), 1);
    m->hbits = 10;
    while (m->hbits < 20 && (1 << m->hbits) < 2 * nprim) ++m->hbits;
    m->pair_cap = std::max<int>(1 << 16, 32 * (int)m->sverts.size() + 16 * d->n_planes);
  }
  *out = m.release();
  return JGS2_OK;
}

// ------------------------------------------------------------------ per-precision buffers

template <typename T>
static PrecBufs<T>& bufs(Mesh* m);
template <>
PrecBufs<float>& bufs<float>(Mesh* m) { return m->f32; }
template <>
PrecBufs<double>& bufs<double>(Mesh* m) { return m->f64; }

// Device-side shared arrays, allocated on first use (mesh creation and the precompute
// touch no device, so they also run on a host without a GPU).
static jgs2_status ensure_device(Mesh* m) {
  if (!m->device_ready) {
    const int V = m->V, T = m->T, ns = m->n_slices;
    CK(cudaGetDevice(&m->device));
    CK(dalloc(&m->d_inc_off, ns + 1));
    CK(dalloc(&m->d_inc_len, m->Vf));
    CK(dalloc(&m->d_inc, m->inc.size()));
    CK(dalloc(&m->d_xt, 3 * (size_t)V));
    CK(dalloc(&m->d_vt, 3 * (size_t)V));
    CK(dalloc(&m->d_perm, V));
    CK(dalloc(&m->d_state, 1));
    CK(dalloc(&m->d_trace, JGS2_TRACE_MAX));
    // sweep partials: [3][vertex blocks] (gather/correct), [12][energy blocks] plus
    // [2 kLsTrials][kPairTrialBlocks] (line search); batch and adjoint passes use fewer
    const size_t np = std::max<size_t>(4 * kLsTrials * ((size_t)(T + 127) / 128 + (m->Vf + 127) / 128 + 1),
                                       (size_t)12 * kEnergyBlocksMax + (size_t)2 * kLsTrials * kPairTrialBlocks + 16);
    CK(dalloc(&m->d_partial, np));
    CK(cudaMallocHost((void**)&m->h_state, sizeof(StepState)));
    CK(cudaMemcpy(m->d_inc_off, m->inc_off.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice));
    if (m->Vf) CK(cudaMemcpy(m->d_inc_len, m->inc_len.data(), sizeof(int) * m->Vf, cudaMemcpyHostToDevice));
    if (!m->inc.empty()) CK(cudaMemcpy(m->d_inc, m->inc.data(), sizeof(int) * m->inc.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d_perm, m->perm.data(), sizeof(int) * V, cudaMemcpyHostToDevice));
    CK(cudaMemset(m->d_state, 0, sizeof(StepState)));
    CK(dalloc(&m->d_tperm, T));
    CK(cudaMemcpy(m->d_tperm, m->tperm.data(), sizeof(int) * T, cudaMemcpyHostToDevice));
    CK(dalloc(&m->d_youngs, T));
    CK(cudaMemcpy(m->d_youngs, m->E.data(), sizeof(double) * T, cudaMemcpyHostToDevice));
    if (m->contact) {
      const int nF = (int)m->sfaces.size() / 3, nE = (int)m->sedges.size() / 2, nS = (int)m->sverts.size();
      const int np = (int)m->planes.size() / 4;
      CK(dalloc(&m->d_planes, std::max(1, 4 * np)));
      CK(dalloc(&m->d_faces, std::max(1, 3 * nF)));
      CK(dalloc(&m->d_edges, std::max(1, 2 * nE)));
      CK(dalloc(&m->d_sverts, std::max(1, nS)));
      CK(dalloc(&m->d_is_surf, V));
      const int H2 = 2 << m->hbits;
      CK(dalloc(&m->d_fkeys, std::max(1, nF)));
      CK(dalloc(&m->d_frank, std::max(1, nF)));
      CK(dalloc(&m->d_ekeys, std::max(1, nE)));
      CK(dalloc(&m->d_erank, std::max(1, nE)));
      CK(dalloc(&m->d_hcnt, H2 + 1));
      CK(dalloc(&m->d_hblk, (H2 + 1 + 4095) / 4096));
      CK(dalloc(&m->d_hids, std::max(1, nF + nE)));
      CK(dalloc(&m->d_hrec, std::max(1, nF + nE)));
      CK(dalloc(&m->d_hkey, std::max(1, nF + nE)));
      CK(dalloc(&m->d_pbp, V));
      CK(dalloc(&m->d_ctl, kCtlWords));
      CK(dalloc(&m->d_dbp, m->pair_cap));
      CK(dalloc(&m->d_pmarg, m->pair_cap));
      CK(dalloc(&m->d_ppath, m->pair_cap));
      CK(cudaMemset(m->d_ctl, 0, sizeof(uint32_t) * kCtlWords));
      CK(cudaMemset(m->d_pbp, 0, sizeof(float4) * V));
      CK(dalloc(&m->d_pairs, m->pair_cap));
      CK(dalloc(&m->d_d0, m->pair_cap));
      CK(dalloc(&m->d_npairs, 1));
      CK(dalloc(&m->d_cflags, 3));
      CK(dalloc(&m->d_bg, 3 * (size_t)V));
      CK(dalloc(&m->d_bH, 6 * (size_t)V));
      CK(dalloc(&m->d_dmin, V));
      CK(dalloc(&m->d_lim, std::max(1, m->Vf)));
      if (np) CK(cudaMemcpy(m->d_planes, m->planes.data(), sizeof(double) * 4 * np, cudaMemcpyHostToDevice));
      if (nF) CK(cudaMemcpy(m->d_faces, m->sfaces.data(), sizeof(int) * 3 * nF, cudaMemcpyHostToDevice));
      if (nE) CK(cudaMemcpy(m->d_edges, m->sedges.data(), sizeof(int) * 2 * nE, cudaMemcpyHostToDevice));
      if (nS) CK(cudaMemcpy(m->d_sverts, m->sverts.data(), sizeof(int) * nS, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(m->d_is_surf, m->is_surf.data(), V, cudaMemcpyHostToDevice));
      CK(cudaMemset(m->d_cflags, 0, 3 * sizeof(int32_t)));
      {
        // contact-aware coupling: body id per vertex (internal order), per-vertex pair lists
        std::vector<int> bod(V);
        for (int v = 0; v < V; ++v) bod[v] = m->body[m->perm[v]];
        CK(dalloc(&m->d_body, V));
        CK(cudaMemcpy(m->d_body, bod.data(), sizeof(int) * V, cudaMemcpyHostToDevice));
        CK(dalloc(&m->d_vp_cnt, V));
        CK(cudaMemset(m->d_vp_cnt, 0, sizeof(int32_t) * V));
        CK(dalloc(&m->d_vp, (size_t)V * kMaxVertexPairs));
        CK(dalloc(&m->d_cpl_on, std::max(1, m->Vf)));
      }
      // accumulators of non-surface vertices are never written: zero them once
      CK(cudaMemset(m->d_bg, 0, sizeof(double) * 3 * (size_t)V));
      CK(cudaMemset(m->d_bH, 0, sizeof(double) * 6 * (size_t)V));
      if (m->fmu > 0.0 && !m->planes.empty()) {
        const size_t nl = m->planes.size() / 4 * (size_t)V;
        CK(dalloc(&m->d_fr_lam, nl));
        CK(cudaMemset(m->d_fr_lam, 0, sizeof(double) * nl));
      }
    }
    if (m->n_scenes > 0) {
      std::vector<int> vs(std::max(1, m->Vf)), ts(T);
      for (int i = 0; i < m->Vf; ++i) vs[i] = m->vscene[m->perm[i]];
      for (int ti = 0; ti < T; ++ti) ts[ti] = m->vscene[m->tets_c[4 * (size_t)m->tperm[ti]]];
      CK(dalloc(&m->d_vscene, std::max(1, m->Vf)));
      CK(dalloc(&m->d_tscene, T));
      CK(dalloc(&m->d_scenes, m->n_scenes));
      CK(dalloc(&m->d_sacc, (size_t)m->n_scenes * kSceneAcc));
      CK(dalloc(&m->d_ndone, 1));
      {
        GridBarrier* gb = nullptr;
        CK(dalloc(&gb, 1));
        m->d_gbar = gb;
      }
      CK(cudaMemcpy(m->d_vscene, vs.data(), sizeof(int) * std::max(1, m->Vf), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(m->d_tscene, ts.data(), sizeof(int) * T, cudaMemcpyHostToDevice));
    }
    m->device_ready = true;
  }
  if (m->pool_version != m->cub_version) {
    cudaFree(m->d_pool_tet);
    m->d_pool_tet = nullptr;
    CK(dalloc(&m->d_pool_tet, std::max(1, m->nP)));
    if (m->nP) CK(cudaMemcpy(m->d_pool_tet, m->pool.data(), sizeof(int) * m->nP, cudaMemcpyHostToDevice));
    m->pool_version = m->cub_version;
  }
  return JGS2_OK;
}

// Host copy of the tet records in internal order (F(x_t) is filled per step on the device).
template <typename T>
static void tet_records(const Mesh* m, std::vector<TetRec<T>>& rec) {
  rec.resize(m->T);
  for (int ti = 0; ti < m->T; ++ti) {
    const int t = m->tperm[ti];
    TetRec<T>& r = rec[ti];
    for (int a = 0; a < 4; ++a) r.v[a] = m->iperm[m->tets_c[4 * (size_t)t + a]];
    for (int q = 0; q < 9; ++q) {
      r.B[q] = T(m->B[9 * (size_t)t + q]);
      r.Ft[q] = T(q % 4 == 0 ? 1.0 : 0.0);
    }
    r.vol = T(m->vol[t]);
    r.mu = T(m->mu[t]);
    r.lp = T(m->lp[t]);
    r.mq = T(m->rho[t] * m->vol[t] / 4.0);
  }
}

static cudaError_t prepare_gather(const Mesh* m);

template <typename T>
static jgs2_status ensure_prec(Mesh* m) {
  jgs2_status ds = ensure_device(m);
  if (ds != JGS2_OK) return ds;
  CK(prepare_gather(m));
  PrecBufs<T>& b = bufs<T>(m);
  if (!b.ready) {
    const int V = m->V, T_ = m->T;
    std::vector<TetRec<T>> rec;
    tet_records<T>(m, rec);
    std::vector<T> mh2(V, T(0));
    for (int i = 0; i < m->Vf; ++i) mh2[i] = T(m->mass[m->perm[i]] / (m->h * m->h));
    CK(dalloc(&b.tets, T_));
    CK(dalloc(&b.frec, T_));
    CK(dalloc(&b.bc, 4 * (size_t)T_));
    CK(dalloc(&b.u, V));
    CK(dalloc(&b.dz, m->Vf));
    CK(dalloc(&b.D, m->Vf));
    CK(dalloc(&b.DJ, m->Vf));
    CK(dalloc(&b.ghr, 18 * (size_t)m->Vf));
    CK(dalloc(&b.mh2, V));
    CK(cudaMemcpy(b.tets, rec.data(), sizeof(TetRec<T>) * T_, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b.mh2, mh2.data(), sizeof(T) * V, cudaMemcpyHostToDevice));
    CK(cudaMemset(b.D, 0, sizeof(Vec4<T>) * std::max(1, m->Vf)));
    CK(cudaMemset(b.DJ, 0, sizeof(Vec4<T>) * std::max(1, m->Vf)));
    b.ready = true;
  }
  if (m->cub_version != b.cub_version && m->n_cub > 0) {
    cudaFree(b.cub_p); cudaFree(b.cub_w); cudaFree(b.cub_u); cudaFree(b.pool_H); cudaFree(b.pool_G);
    // rows of cs = Vf rounded up to 4 entries: every row starts 16-byte aligned (bulk copies);
    // padding entries are unused slots (p = -1, w = 0, U_bar = 0)
    const size_t Vf = m->Vf, nc = m->n_cub, cs = cub_stride(m->Vf);
    std::vector<T> w(nc * cs, T(0)), u(nc * 36 * cs, T(0));
    for (size_t s = 0; s < nc; ++s)
      for (size_t i = 0; i < Vf; ++i) {
        w[s * cs + i] = T(m->cub_w[i * nc + s]);
        for (int q = 0; q < 36; ++q) u[(s * 36 + q) * cs + i] = T(m->cub_u[(i * nc + s) * 36 + q]);
      }
    std::vector<int32_t> p(nc * cs, -1);
    for (size_t s = 0; s < nc; ++s)
      for (size_t i = 0; i < Vf; ++i) p[s * cs + i] = m->cub_p[i * nc + s];
    CK(dalloc(&b.cub_p, nc * cs));
    CK(dalloc(&b.cub_w, nc * cs));
    CK(dalloc(&b.cub_u, nc * 36 * cs));
    CK(dalloc(&b.pool_H, (size_t)m->nP * kPoolStride));
    CK(dalloc(&b.pool_G, (size_t)m->nP * 12));
    cudaFree(b.pool_R);
    CK(dalloc(&b.pool_R, (size_t)m->nP * 36));
    CK(cudaMemcpy(b.cub_p, p.data(), sizeof(int32_t) * p.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b.cub_w, w.data(), sizeof(T) * w.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b.cub_u, u.data(), sizeof(T) * u.size(), cudaMemcpyHostToDevice));
    b.cub_version = m->cub_version;
  }
  return JGS2_OK;
}

template <typename T>
static DevMesh<T> dev_view(Mesh* m) {
  PrecBufs<T>& b = bufs<T>(m);
  DevMesh<T> d;
  // zero every byte (padding included): a captured sweep graph is re-used only while the
  // view compares equal byte for byte (all defaults of the view are zero)
  static_assert(std::is_trivially_copyable<DevMesh<T>>::value, "device view must be trivially copyable");
  std::memset(static_cast<void*>(&d), 0, sizeof(d));
  d.V = m->V;
  d.Vf = m->Vf;
  d.T_ = m->T;
  d.vmask = m->vmask_on ? m->d_vmask : nullptr;
  d.n_slices = m->n_slices;
  d.nP = m->nP;
  d.n_cub = m->n_cub;
  d.tets = b.tets;
  d.tets_mut = b.tets;
  d.frec = b.frec;
  d.bc = b.bc;
  d.inc_off = m->d_inc_off;
  d.inc_len = m->d_inc_len;
  d.inc = m->d_inc;
  d.u = b.u;
  d.dz = b.dz;
  d.D = b.D;
  d.DJ = b.DJ;
  d.ghr = b.ghr;
  d.mh2 = b.mh2;
  d.cub_p = b.cub_p;
  d.cub_w = b.cub_w;
  d.cub_u = b.cub_u;
  d.cs = cub_stride(m->Vf);
  d.pool_tet = m->d_pool_tet;
  d.pool_H = b.pool_H;
  d.pool_G = b.pool_G;
  d.pool_R = b.pool_R;
  d.xt = m->d_xt;
  d.vt = m->d_vt;
  d.perm = m->d_perm;
  d.c = ContactView();
  if (m->contact) {
    ContactView& c = d.c;
    c.on = 1;
    c.pen = m->penalty;
    c.n_planes = (int)m->planes.size() / 4;
    c.n_faces = (int)m->sfaces.size() / 3;
    c.n_edges = (int)m->sedges.size() / 2;
    c.n_sverts = (int)m->sverts.size();
    c.planes = m->d_planes;
    c.faces = m->d_faces;
    c.edges = m->d_edges;
    c.sverts = m->d_sverts;
    c.is_surf = m->d_is_surf;
    c.dhat = m->dhat;
    c.kappa = m->kappa;
    c.rc = m->rc;
    c.n_vertices = m->V;
    c.R = m->bp_R;
    c.trig = m->bp_trig;
    c.hbits = m->hbits;
    c.fkeys = m->d_fkeys;
    c.ekeys = m->d_ekeys;
    c.frank = m->d_frank;
    c.erank = m->d_erank;
    c.hcnt = m->d_hcnt;
    c.hblk = m->d_hblk;
    c.hids = m->d_hids;
    c.hrec = m->d_hrec;
    c.hkey = m->d_hkey;
    c.pbp = m->d_pbp;
    c.ctl = m->d_ctl;
    c.dbp = m->d_dbp;
    c.pmarg = m->d_pmarg;
    c.ppath = m->d_ppath;
    c.pairs = m->d_pairs;
    c.n_pairs = m->d_npairs;
    c.cap = m->pair_cap;
    c.d0 = m->d_d0;
    c.bg = m->d_bg;
    c.bH = m->d_bH;
    c.dmin = m->d_dmin;
    c.lim = m->d_lim;
    c.flags = m->d_cflags;
    c.body = m->d_body;
    c.vp_cnt = m->d_vp_cnt;
    c.vp = m->d_vp;
    c.fmu = m->fmu;
    c.feps = m->feps_v * m->h;
    c.fr_lam = m->d_fr_lam;
  }
  d.n_scenes = m->n_scenes;
  d.v_scene = m->d_vscene;
  d.t_scene = m->d_tscene;
  d.scenes = m->d_scenes;
  d.sacc = m->d_sacc;
  d.n_done = m->d_ndone;
  d.inv_h2 = 1.0 / (m->h * m->h);
  d.h = m->h;
  for (int q = 0; q < 3; ++q) d.grav[q] = m->grav[q];
  return d;
}

bool dev_view_f64_if_ready(Mesh* m, DevMesh<double>* out) {
  if (!m || !m->device_ready || !m->f64.ready) return false;
  *out = dev_view<double>(m);
  return true;
}

// ------------------------------------------------------------------ cubature records

jgs2_status set_cubature(Mesh* m, int n_cub, const std::vector<int>& elem_int /* [Vf][nc] internal tet, -1 */,
                         const std::vector<double>& w, const std::vector<double>& u) {
  if (n_cub <= 0 || n_cub > kMaxCub) return fail(JGS2_EINVAL, "n_cub must be in [1, 8]");
  // pool = distinct referenced elements, ordered by (body, internal id): the slots a block
  // of nearby vertices references then form a short contiguous range (k_correct stages it)
  std::vector<int> pool;
  for (int e : elem_int)
    if (e >= 0) pool.push_back(e);
  auto body_of = [&](int t) { return m->body[m->tets_c[4 * (size_t)m->tperm[t]]]; };
  auto by_body = [&](int a, int b) {
    const int ba = body_of(a), bb = body_of(b);
    return ba != bb ? ba < bb : a < b;
  };
  std::sort(pool.begin(), pool.end(), by_body);
  pool.erase(std::unique(pool.begin(), pool.end()), pool.end());
  m->n_cub = n_cub;
  m->nP = (int)pool.size();
  m->pool = pool;
  m->cub_p.assign(elem_int.size(), -1);
  for (size_t q = 0; q < elem_int.size(); ++q)
    if (elem_int[q] >= 0)
      m->cub_p[q] = (int)(std::lower_bound(pool.begin(), pool.end(), elem_int[q], by_body) - pool.begin());
  m->cub_elem = elem_int;
  m->cub_w = w;
  m->cub_u = u;
  m->cub_version++;
  return JGS2_OK;
}

jgs2_status import_cubature(Mesh* m, const jgs2_cubature_blob* b) {
  if (!m || !b || !b->elem || !b->weight || !b->ubar) return fail(JGS2_EINVAL, "null argument");
  const int nc = b->n_cub;
  if (nc <= 0 || nc > kMaxCub) return fail(JGS2_EINVAL, "n_cub must be in [1, 8]");
  const size_t Vf = m->Vf;
  std::vector<int> e(Vf * nc, -1);
  std::vector<double> w(Vf * nc, 0.0), u(Vf * nc * 36, 0.0);
  for (size_t i = 0; i < Vf; ++i) {
    const int c = m->perm[i];
    for (int s = 0; s < nc; ++s) {
      const int et = b->elem[(size_t)c * nc + s];
      if (et < -1 || et >= m->T) return fail(JGS2_EINVAL, "cubature element out of range");
      const double ww = b->weight[(size_t)c * nc + s];
      if (et >= 0 && !(ww >= 0.0 && std::isfinite(ww))) return fail(JGS2_EINVAL, "cubature weight must be finite and >= 0");
      if (et < 0) continue;
      // the slot's 4 corners follow the caller tet's corner order, which the internal
      // record keeps (corner a of internal tet = corner a of caller tet)
      e[i * nc + s] = m->tiperm[et];
      w[i * nc + s] = ww;
      for (int q = 0; q < 36; ++q) u[(i * nc + s) * 36 + q] = b->ubar[((size_t)c * nc + s) * 36 + q];
    }
  }
  m->cub_resid.assign(m->V, std::nan(""));
  return set_cubature(m, nc, e, w, u);
}

// ------------------------------------------------------------------ step driver

// Candidate pairs within r_c at x^k, the barrier accumulators and the per-vertex minimum
// distances (Sec. 7). Pair order is not canonical here (the sums use atomics).
constexpr int kContactKernels = 10;  // launches of one contact_pass (one more with wall friction)

template <typename T>
static jgs2_status contact_pass(Mesh* m, DevMesh<T>& d, cudaStream_t s, StepState* st) {
  const ContactView& c = d.c;
  const int nS = c.n_sverts, nF = c.n_faces, nE = c.n_edges;
  const int H2 = 2 << c.hbits;
  const int cap_blocks = 148 * 4;
  auto grid = [&](int n, int bs) { return std::max(1, std::min((n + bs - 1) / bs, cap_blocks)); };
  k_bp_check<T><<<grid(nS, 256), 256, 0, s>>>(d, c, st);
  // rebuild kernels: empty launches unless k_bp_check asked for a rebuild
  k_bp_snapshot<T><<<grid(std::max(std::max(nS, nF), std::max(nE, H2 + 1)), 256), 256, 0, s>>>(d, c);
  k_bp_keys<T><<<grid(std::max(nF, nE), 256), 256, 0, s>>>(d, c);
  const int nblk = (H2 + 1 + 4095) / 4096;
  k_bp_scan_blocks<<<nblk, 1024, 0, s>>>(c);
  k_bp_scan_top<<<1, 1024, 0, s>>>(c, nblk);
  k_bp_scan_apply<<<nblk, 1024, 0, s>>>(c);
  k_bp_fill<<<grid(std::max(nF, nE), 256), 256, 0, s>>>(c);
  k_query_vertices<T><<<grid(nS, 128), 128, 0, s>>>(d, c);
  k_query_edges<T><<<grid(nE, 128), 128, 0, s>>>(d, c);
  // per sweep: barrier terms of the listed pairs at x^k (k_bp_check cleared the sums)
  k_pair_terms<T><<<grid(c.cap, 256), 256, 0, s>>>(d, c, st);
  // wall friction (lagged at the step start) into the same per-vertex sums
  if (c.fr_lam) k_friction_terms<T><<<grid(nS, 256), 256, 0, s>>>(d, c, st);
  CK(cudaGetLastError());
  return JGS2_OK;
}

// Forces a candidate-list rebuild at the next contact pass (start of a step).
static jgs2_status contact_force_rebuild(Mesh* m, cudaStream_t s) {
  CK(cudaMemsetAsync(m->d_ctl + kCtlForce, 1, sizeof(uint32_t), s));  // any non-zero word
  return JGS2_OK;
}

// Dynamic shared memory of k_gather for blocks of vpb vertices: the block's incidence
// entries.
static size_t gather_smem(const Mesh* m, int vpb) {
  const int q = vpb == 64 ? 0 : (vpb == 256 ? 2 : (vpb == 32 ? 3 : 1));
  return (size_t)std::max(m->inc_blk[q], 4) * sizeof(int);
}

// k_gather launch shapes (threads per block, threads per vertex) the library builds.
static const int kGatherShapes[5][2] = {{64, 1}, {128, 1}, {256, 1}, {128, 4}, {256, 4}};

// Raises the dynamic shared memory limit of every k_gather variant to what this mesh needs
// (once per new maximum; before any launch or graph capture of the mesh).
static cudaError_t prepare_gather(const Mesh* m) {
  static size_t have = 48 * 1024;
  size_t need = 0;
  for (int vpb : {32, 64, 128, 256}) need = std::max(need, gather_smem(m, vpb));
  if (need <= have) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  auto set = [&](auto kern) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
  };
#define JGS2_SET(T)                                            \
  set(k_gather<T, true, false, 64, 1>);                        \
  set(k_gather<T, true, false, 128, 1>);                       \
  set(k_gather<T, true, false, 256, 1>);                       \
  set(k_gather<T, true, false, 128, 4>);                       \
  set(k_gather<T, true, false, 256, 4>);                       \
  set(k_gather<T, false, false, 64, 1>);                       \
  set(k_gather<T, false, false, 128, 1>);                      \
  set(k_gather<T, false, false, 256, 1>);                      \
  set(k_gather<T, false, false, 128, 4>);                      \
  set(k_gather<T, false, false, 256, 4>);                      \
  set(k_gather<T, true, true, 64, 1>);                         \
  set(k_gather<T, true, true, 128, 1>);                        \
  set(k_gather<T, true, true, 256, 1>);                        \
  set(k_gather<T, true, true, 128, 4>);                        \
  set(k_gather<T, true, true, 256, 4>);                        \
  set(k_gather<T, false, true, 64, 1>);                        \
  set(k_gather<T, false, true, 128, 1>);                       \
  set(k_gather<T, false, true, 256, 1>);                       \
  set(k_gather<T, false, true, 128, 4>);                       \
  set(k_gather<T, false, true, 256, 4>);
  JGS2_SET(float)
  JGS2_SET(double)
#undef JGS2_SET
  if (e == cudaSuccess) have = need;
  return e;
}

// k_gather with a runtime shape: bs threads per block (64, 128 or 256), tpv threads per
// vertex (1; or 4 with 128 or 256 threads)
template <typename T, bool BATCH>
static void launch_gather(DevMesh<T>& d, const Mesh* m, bool corr, int bs, int tpv, cudaStream_t s, StepState* st,
                          double* partial, double* trace, int rec) {
  const int Vf = d.Vf;
#define JGS2_G(B, P)                                                                                      \
  {                                                                                                       \
    const size_t sm = gather_smem(m, B / P);                                                              \
    const int nb = (Vf + B / P - 1) / (B / P);                                                            \
    if (corr)                                                                                             \
      k_gather<T, true, BATCH, B, P><<<nb, B, sm, s>>>(d, st, partial, trace, rec);                       \
    else                                                                                                  \
      k_gather<T, false, BATCH, B, P><<<nb, B, sm, s>>>(d, st, partial, trace, rec);                      \
  }
  if (tpv == 4 && bs == 256) {
    JGS2_G(256, 4)
  } else if (tpv == 4) {
    JGS2_G(128, 4)
  } else if (bs == 64) {
    JGS2_G(64, 1)
  } else if (bs == 256) {
    JGS2_G(256, 1)
  } else {
    JGS2_G(128, 1)
  }
#undef JGS2_G
}

// k_correct with a runtime shape: bs threads per block (64, 128 or 256); pf = 1 loads
// every slot's pool index and weight first (four slots)
template <typename T, bool BATCH>
static void launch_correct(DevMesh<T>& d, int bs, cudaStream_t s, StepState* st, double* partial,
                           double* trace, int rec, int pf = 0) {
  const int Vf = d.Vf;
#define JGS2_C(B, P) k_correct<T, BATCH, B, P><<<(Vf + B - 1) / B, B, 0, s>>>(d, st, partial, trace, rec)
  if (bs == 64)
    pf ? JGS2_C(64, true) : JGS2_C(64, false);
  else if (bs == 256)
    pf ? JGS2_C(256, true) : JGS2_C(256, false);
  else
    pf ? JGS2_C(128, true) : JGS2_C(128, false);
#undef JGS2_C
}

// Launch bookkeeping of one step: counts per kernel kind and, when profiling, a CUDA
// event pair around every launch (events are pooled per mesh).
struct Launches {
  Mesh* m;
  cudaStream_t s;
  bool prof;
  int count[JGS2_NKERNELS] = {};
  double gms[JGS2_NKERNELS] = {};  // event times of graph replays (the profiled sweeps)
  int psweeps = 0;                 // profiled sweeps: one per replay begun before the stop
  std::vector<std::pair<int, int>> rec;  // (kind, event index)
  int used = 0;
  cudaError_t err = cudaSuccess;
  // a group of n kernels of one kind launched directly on the stream
  int begin(int kind, int n = 1) {
    count[kind] += n;
    if (!prof) return -1;
    if ((int)m->events.size() < used + 2) {
      for (int q = 0; q < 64; ++q) {
        cudaEvent_t e;
        if ((err = cudaEventCreate(&e)) != cudaSuccess) return -1;
        m->events.push_back(e);
      }
    }
    const int id = used;
    used += 2;
    cudaEventRecord(m->events[id], s);
    rec.push_back({kind, id});
    return id;
  }
  void end(int id) {
    if (id >= 0) cudaEventRecord(m->events[id + 1], s);
  }
  void report(jgs2_step_report* r) {
    int tot = 0;
    for (int q = 0; q < JGS2_NKERNELS; ++q) {
      tot += count[q];
      if (r) {
        r->kernel_launches[q] = count[q];
        r->kernel_ms[q] = 0.0;
      }
    }
    if (r) {
      r->launches = tot;
      r->profiled_sweeps = prof ? psweeps : 0;
    }
    if (!r || !prof) return;
    for (int q = 0; q < JGS2_NKERNELS; ++q) r->kernel_ms[q] += gms[q];
    for (auto& kv : rec) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, m->events[kv.second], m->events[kv.second + 1]) == cudaSuccess)
        r->kernel_ms[kv.first] += ms;
    }
  }
};

// Blocks of k_energy<T, DIR> that are resident at once on the device (capped at
// kEnergyBlocksMax, which sizes the partial-sum buffer).
template <typename T, int DIR>
static int energy_blocks() {
  static int nb = 0;
  if (nb == 0) {
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_energy<T, DIR>, 128, 0) !=
        cudaSuccess)
      per_sm = 1;
    nb = std::max(1, std::min(sms * std::max(1, per_sm), kEnergyBlocksMax));
  }
  return nb;
}

// Private non-blocking stream (and ordering events) the sweep graphs are captured and
// replayed on: the caller's stream may be the legacy default stream, which cannot be
// captured. Work on it is ordered after and before the caller's stream by events.
static jgs2_status ensure_gstream(Mesh* m) {
  if (!m->gstream) {
    CK(cudaStreamCreateWithFlags(&m->gstream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&m->gstream2, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&m->gev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&m->gev[1], cudaEventDisableTiming));
    for (cudaEvent_t& e : m->gfork) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  return JGS2_OK;
}

// The sweeps of one step (single scene). Sweep k reads its index from the device step
// state, so every sweep is the same sequence of launches: a chunk of check_every sweeps is
// captured once per launch configuration into a CUDA graph and replayed until the device
// flags the step done (converged, diverged or max_k sweeps). Sweeps after that flag are
// empty launches. With check = false the host does not wait between replays and runs
// ceil((max_k + 1) / chunk) of them. Profiling puts external event nodes around every
// kernel group of the chunk's last sweep; their times are read after each replay.
template <typename T>
static jgs2_status run_sweeps(Mesh* m, const jgs2_step_opts& o, cudaStream_t cs, int max_k, double rel_tol,
                              bool check, StepState* hs, Launches& L, int gs_ncol = 0) {
  DevMesh<T> d = dev_view<T>(m);
  const bool corr = o.correction != JGS2_CORR_OFF;
  // contact-aware local terms (Sec. 7): only with contact and the correction on
  const bool coupling = o.contact_coupling && m->contact && corr;
  if (coupling) {
    PrecBufs<T>& b = bufs<T>(m);
    if (!b.cpl) CK(dalloc(&b.cpl, 9 * (size_t)std::max(1, m->Vf)));
    d.cpl = b.cpl;
    d.cpl_on = m->d_cpl_on;
  }
  const int nbV = (m->Vf + 127) / 128;
  const int nbT = (m->T + 127) / 128;
  // line-search passes: one full wave of resident blocks each (SM count x blocks per SM at
  // the pass's registers and shared memory), grid-stride over tet tiles and vertices
  const int nbE0 = std::max(1, std::min(std::max(nbT, nbV), energy_blocks<T, 0>()));
  const int nbE1 = std::max(1, std::min(std::max(nbT, nbV), energy_blocks<T, 1>()));
  const int nbE2 = std::max(1, std::min(std::max(nbT, nbV), energy_blocks<T, 2>()));
  const int pi = sizeof(T) == 4 ? 1 : 0;
  const int bs = m->bs[pi], gbs = m->gbs[pi], gtpv = m->gtpv[pi];
  const int chunk = std::max(1, o.check_every);
  const bool prof = L.prof;
  jgs2_status gs = ensure_gstream(m);
  if (gs != JGS2_OK) return gs;
  cudaStream_t s = m->gstream;
  CK(cudaEventRecord(m->gev[0], cs));
  CK(cudaStreamWaitEvent(s, m->gev[0], 0));
  StepState init;
  std::memset(&init, 0, sizeof(init));
  init.max_sweeps = max_k;
  init.rel_tol = rel_tol;
  init.alpha = 1.0;
  init.gs_ncol = gs_ncol;
  if (rel_tol >= 0.0 && o.dx_tol > 0.0 && gs_ncol == 0) {
    // Sec. 8: |x^k - x^{k-1}| on the scene normalised to a unit cube
    const double L = o.length_scale > 0.0 ? o.length_scale : m->extent;
    init.dx2_tol = (o.dx_tol * L) * (o.dx_tol * L);
  }
  CK(cudaMemcpyAsync(m->d_state, &init, sizeof(StepState), cudaMemcpyHostToDevice, s));
  if (m->contact) {
    jgs2_status cst = contact_force_rebuild(m, s);
    if (cst != JGS2_OK) return cst;
  }
  long key = (long)(sizeof(T) == 4);
  key = key * 3 + o.correction;
  key = key * 2 + (o.line_search != 0);
  key = key * 2 + m->contact;
  key = key * 2 + (prof ? 1 : 0);
  key = key * 2 + (o.record_trace != 0);
  key = key * 512 + bs;
  key = key * 512 + gbs;
  key = key * 8 + gtpv;
  key = key * 2 + m->cpf[pi];
  key = key * 8192 + chunk;
  key = key * 64 + gs_ncol + (1L << 60);
  const bool same_view = m->gdev.size() == sizeof(d) && std::memcmp(m->gdev.data(), &d, sizeof(d)) == 0;
  if (m->graph_key != key || !same_view) {
    if (m->graph) cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
    m->graph_key = -1;
    m->ggroups.clear();
    // profiling: event nodes around the kernel groups of the chunk's last sweep only (not
    // the first: a step's sweep 0 always rebuilds the contact list)
    const size_t nev = prof ? (size_t)32 : 0;
    while (m->gevents.size() < nev) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      m->gevents.push_back(e);
    }
    size_t evi = 0;
    cudaError_t cerr = cudaSuccess;
    bool timed = false;  // set per sweep of the chunk
    auto group = [&](int kind, int n, cudaStream_t gs, auto&& launch) {
      Mesh::GraphGroup g{kind, n, nullptr, nullptr};
      if (timed) {
        g.e0 = m->gevents[evi++];
        g.e1 = m->gevents[evi++];
        if (cerr == cudaSuccess) cerr = cudaEventRecordWithFlags(g.e0, gs, cudaEventRecordExternal);
      }
      launch();
      if (timed && cerr == cudaSuccess) cerr = cudaEventRecordWithFlags(g.e1, gs, cudaEventRecordExternal);
      m->ggroups.push_back(g);
    };
    // a second branch of the graph: work on s2 starts after the fork point on s and
    // joins s before the kernel that needs it
    cudaStream_t s2 = m->gstream2;
    auto fork = [&](cudaEvent_t e) {
      if (cerr == cudaSuccess) cerr = cudaEventRecord(e, s);
      if (cerr == cudaSuccess) cerr = cudaStreamWaitEvent(s2, e, 0);
    };
    auto join = [&](cudaEvent_t e) {
      if (cerr == cudaSuccess) cerr = cudaEventRecord(e, s2);
      if (cerr == cudaSuccess) cerr = cudaStreamWaitEvent(s, e, 0);
    };
    const bool pool = corr && m->nP > 0;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    // a Gauss-Seidel sweep is one pass per colour, each with the colour's vertex mask
    const int passes = gs_ncol > 0 ? chunk * gs_ncol : chunk;
    const DevMesh<T> d_base = d;
    for (int q = 0; q < passes; ++q) {
      timed = prof && q == passes - 1;
      if (gs_ncol > 0) d.vmask = m->d_gsmask + (size_t)(q % gs_ncol) * m->Vf;
      // contact pass (positions only) alongside the element pass; both feed the gather
      if (m->contact) {
        fork(m->gfork[0]);
        group(JGS2_K_CONTACT, kContactKernels + (m->d_fr_lam ? 1 : 0), s2,
              [&] { contact_pass<T>(m, d, s2, m->d_state); });
      }
      if (nbV > 0) group(JGS2_K_ELEM, 1, s, [&] { k_elem<T, false><<<nbT, 128, 0, s>>>(d, m->d_state); });
      if (m->contact) join(m->gfork[1]);
      if (nbV > 0)
        group(JGS2_K_GATHER, 1, s,
              [&] {
                launch_gather<T, false>(d, m, corr, gbs, gtpv, s, m->d_state, m->d_partial, m->d_trace, o.record_trace);
              });
      if (coupling)
        group(JGS2_K_CONTACT, 1, s, [&] { k_couple<T><<<nbV, 128, 0, s>>>(d, d.c, m->d_state); });
      // cubature pool after the gather, whose g and R at the pool elements' corners it reads
      if (pool)
        group(JGS2_K_POOL, 1, s, [&] {
          if (o.correction == JGS2_CORR_ASM)
            k_pool<T, true><<<(m->nP + kPoolWarps - 1) / kPoolWarps, 32 * kPoolWarps, 0, s>>>(d, m->d_state);
          else
            k_pool<T, false><<<(m->nP + kPoolWarps - 1) / kPoolWarps, 32 * kPoolWarps, 0, s>>>(d, m->d_state);
        });
      if (nbV > 0) {
        if (corr)
          group(JGS2_K_CORRECT, 1, s,
                [&] {
                  launch_correct<T, false>(d, bs, s, m->d_state, m->d_partial, m->d_trace, o.record_trace, m->cpf[pi]);
                });
      }
      if (o.line_search) {
        // along D; along D_J only when every trial along D failed (those launches return
        // at once otherwise)
        const int npp = m->contact ? kPairTrialBlocks : 0;
        double* pp = m->d_partial + (size_t)12 * kEnergyBlocksMax;
        // one timing group per launch, so that each kernel of the pass is timed alone
        if (m->contact)
          group(JGS2_K_LS_PAIRS, 1, s, [&] { k_pair_trials<T, 0><<<npp, 128, 0, s>>>(d, m->d_state, pp); });
        group(JGS2_K_ENERGY, 1, s, [&] { k_energy<T, 0><<<nbE0, 128, 0, s>>>(d, m->d_state, m->d_partial); });
        group(JGS2_K_LS_DECIDE, 1, s, [&] {
          k_ls_decide<0><<<1, 1024, 0, s>>>(m->d_state, corr ? 1 : 0, m->d_partial, nbE0, pp, npp);
        });
        if (corr) {
          if (m->contact)
            group(JGS2_K_LS_PAIRS, 1, s, [&] { k_pair_trials<T, 1><<<npp, 128, 0, s>>>(d, m->d_state, pp); });
          group(JGS2_K_ENERGY, 1, s, [&] { k_energy<T, 1><<<nbE1, 128, 0, s>>>(d, m->d_state, m->d_partial); });
          group(JGS2_K_LS_DECIDE, 1, s,
                [&] { k_ls_decide<1><<<1, 1024, 0, s>>>(m->d_state, 1, m->d_partial, nbE1, pp, npp); });
          if (m->contact)
            group(JGS2_K_LS_PAIRS, 1, s, [&] { k_pair_trials<T, 2><<<npp, 128, 0, s>>>(d, m->d_state, pp); });
          group(JGS2_K_ENERGY, 1, s, [&] { k_energy<T, 2><<<nbE2, 128, 0, s>>>(d, m->d_state, m->d_partial); });
          group(JGS2_K_LS_DECIDE, 1, s,
                [&] { k_ls_decide<2><<<1, 1024, 0, s>>>(m->d_state, 1, m->d_partial, nbE2, pp, npp); });
        }
      }
      if (nbV > 0) group(JGS2_K_UPDATE, 1, s, [&] { k_update<T><<<nbV, 128, 0, s>>>(d, m->d_state); });
    }
    d = d_base;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) return fail(JGS2_ECUDA, std::string("sweep capture: ") + cudaGetErrorString(e));
    if (cerr != cudaSuccess) {
      cudaGraphDestroy(g);
      return fail(JGS2_ECUDA, std::string("sweep capture (timing events): ") + cudaGetErrorString(cerr));
    }
    e = cudaGraphInstantiate(&m->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(JGS2_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    m->graph_key = key;
    m->gdev.assign(reinterpret_cast<const char*>(&d), reinterpret_cast<const char*>(&d) + sizeof(d));
  }
  const int replays = (max_k + chunk) / chunk;  // ceil((max_k + 1) / chunk)
  for (int rp = 0; rp < replays; ++rp) {
    CK(cudaGraphLaunch(m->graph, s));
    for (const auto& g : m->ggroups) L.count[g.kind] += g.n;
    if (check || prof) {
      CK(cudaMemcpyAsync(hs, m->d_state, sizeof(StepState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      // the timed (last) sweep of this replay did work unless the step stopped before it
      if (prof && (!hs->done || rp * chunk + chunk - 1 <= hs->sweeps)) {
        L.psweeps += 1;
        for (const auto& g : m->ggroups) {
          float ms = 0.f;
          if (g.e0 && cudaEventElapsedTime(&ms, g.e0, g.e1) == cudaSuccess) L.gms[g.kind] += ms;
        }
      }
      if (check && hs->done) break;
    }
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(hs, m->d_state, sizeof(StepState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaEventRecord(m->gev[1], s));
  CK(cudaStreamWaitEvent(cs, m->gev[1], 0));
  if (m->contact) {
    int32_t fl[3];
    CK(cudaMemcpy(fl, m->d_cflags, sizeof(fl), cudaMemcpyDeviceToHost));
    if (fl[0]) {
      CK(cudaMemset(m->d_cflags, 0, sizeof(fl)));
      return fail(JGS2_ENOMEM, "contact pair buffer overflow (" + std::to_string(m->pair_cap) + " pairs)");
    }
    if (fl[2] && coupling) {
      CK(cudaMemset(m->d_cflags, 0, sizeof(fl)));
      return fail(JGS2_ENOMEM, "a vertex has more than " + std::to_string(kMaxVertexPairs) +
                                   " active pairs reaching other bodies (contact-aware coupling)");
    }
    if (fl[1] || fl[2]) CK(cudaMemset(m->d_cflags, 0, sizeof(fl)));
  }
  return JGS2_OK;
}

// The persistent batch kernel for the sweep's flags (correction, line search, threads per
// vertex of the gather).
template <typename T>
static void (*persistent_kernel(bool corr, bool ls, int tpv))(DevMesh<T>, PersistArgs) {
  if (tpv == 4) {
    if (corr) return ls ? k_batch_persistent<T, true, true, 4> : k_batch_persistent<T, true, false, 4>;
    return ls ? k_batch_persistent<T, false, true, 4> : k_batch_persistent<T, false, false, 4>;
  }
  if (corr) return ls ? k_batch_persistent<T, true, true, 1> : k_batch_persistent<T, true, false, 1>;
  return ls ? k_batch_persistent<T, false, true, 1> : k_batch_persistent<T, false, false, 1>;
}

// Batch meshes, persistent form: each chunk of check_every sweeps is one cooperative launch
// (grid: every block resident, the occupancy limit times the SM count) whose phases are
// separated by the bounded grid barrier, captured with the barrier reset in a CUDA graph
// and replayed until every scene has stopped or a wait gave up.
template <typename T>
static jgs2_status run_batch_persistent(Mesh* m, const jgs2_step_opts& o, cudaStream_t s, Launches& L,
                                        DevMesh<T>& d, bool corr) {
  const int pi = sizeof(T) == 4 ? 1 : 0;
  const int tpv = m->gtpv[pi] == 4 ? 4 : 1;
  const int S = m->n_scenes;
  const int chunk = std::max(1, o.check_every);
  PersistArgs a{};
  a.chunk = chunk;
  a.nbT = (m->T + 127) / 128;
  a.nbG = (m->Vf + 128 / tpv - 1) / (128 / tpv);
  a.nbP = (m->nP + kPoolWarps - 1) / kPoolWarps;
  a.nbC = (m->Vf + 127) / 128;
  a.nbV = (m->Vf + 127) / 128;
  a.nbS = (S + 127) / 128;
  a.corr = corr ? 1 : 0;
  a.ls = o.line_search ? 1 : 0;
  a.max_sweeps = o.max_sweeps;
  a.rel_tol = o.rel_tol;
  a.wait_polls = o.wait_polls > 0 ? o.wait_polls : (1 << 20);
  a.bar = static_cast<GridBarrier*>(m->d_gbar);
  a.st = m->d_state;
  a.partial = m->d_partial;
  auto kern = persistent_kernel<T>(corr, o.line_search != 0, tpv);
  const size_t smem = gather_smem(m, 128 / tpv);
  CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int nbps = 0, dev = 0, sms = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbps, kern, 128, smem));
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (nbps < 1) return fail(JGS2_ECUDA, "persistent batch kernel cannot be resident on an SM");
  const int grid = nbps * sms;
  long key = (long)(sizeof(T) == 4);
  key = key * 2 + (corr ? 1 : 0);
  key = key * 2 + (o.line_search != 0);
  key = key * 8 + tpv;
  key = key * 2 + (o.test_unreachable_barrier != 0);
  key = key * 4096 + chunk;
  key = key * 1000003L + o.max_sweeps;
  key = key * 4194304L + (long)a.wait_polls;
  key = (key ^ (long)(o.rel_tol * 1e12)) | (1L << 61);
  const bool same_view = m->gdev.size() == sizeof(d) && std::memcmp(m->gdev.data(), &d, sizeof(d)) == 0;
  if (m->graph_key != key || !same_view) {
    if (m->graph) cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
    m->graph_key = -1;
    m->ggroups.clear();
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(m->d_gbar, 0, sizeof(GridBarrier), s);
    if (e == cudaSuccess && o.test_unreachable_barrier)
      e = cudaMemsetAsync(static_cast<char*>(m->d_gbar) + offsetof(GridBarrier, extra), 1, 1, s);
    if (e == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(grid);
      cfg.blockDim = dim3(128);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, kern, d, a);
    }
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) {
      if (e2 == cudaSuccess) cudaGraphDestroy(g);
      return fail(JGS2_ECUDA, std::string("persistent batch launch capture: ") + cudaGetErrorString(e));
    }
    if (e2 != cudaSuccess) return fail(JGS2_ECUDA, std::string("persistent batch capture: ") + cudaGetErrorString(e2));
    e = cudaGraphInstantiate(&m->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(JGS2_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    m->graph_key = key;
    m->gdev.assign(reinterpret_cast<const char*>(&d), reinterpret_cast<const char*>(&d) + sizeof(d));
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (L.prof) {
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
  }
  int32_t done = 0;
  StepState hs;
  for (int sw = 0; sw <= o.max_sweeps; sw += chunk) {
    if (L.prof) CK(cudaEventRecord(e0, s));
    CK(cudaGraphLaunch(m->graph, s));
    if (L.prof) CK(cudaEventRecord(e1, s));
    L.count[JGS2_K_PERSISTENT] += 1;
    CK(cudaMemcpyAsync(&done, m->d_ndone, sizeof(done), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hs, m->d_state, sizeof(StepState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (L.prof) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) L.gms[JGS2_K_PERSISTENT] += ms;
    }
    if (hs.status != 0 || done >= S) break;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  CK(cudaGetLastError());
  return JGS2_OK;
}

// Batch meshes: every scene runs its own sweeps and stopping test; a chunk of check_every
// sweeps (all kernels of all scenes, one launch per kernel) is captured once in a CUDA
// graph and replayed until every scene has stopped.
template <typename T>
static jgs2_status run_sweeps_batch(Mesh* m, const jgs2_step_opts& o, cudaStream_t cs, Launches& L) {
  DevMesh<T> d = dev_view<T>(m);
  // the caller's stream may be the legacy default stream, which cannot be captured: the
  // sweeps run on a private stream ordered after (and before) the caller's work
  jgs2_status gs = ensure_gstream(m);
  if (gs != JGS2_OK) return gs;
  cudaStream_t s = m->gstream;
  CK(cudaEventRecord(m->gev[0], cs));
  CK(cudaStreamWaitEvent(s, m->gev[0], 0));
  const bool corr = o.correction != JGS2_CORR_OFF && m->nP > 0;
  const int S = m->n_scenes;
  const int nbV = (m->Vf + 127) / 128, nbT = (m->T + 127) / 128;
  const int pi = sizeof(T) == 4 ? 1 : 0;
  const int bs = m->bs[pi], gbs = m->gbs[pi], gtpv = m->gtpv[pi];
  const int chunk = std::max(1, o.check_every);
  StepState init;
  std::memset(&init, 0, sizeof(init));
  init.max_sweeps = 1 << 30;
  init.rel_tol = -1.0;
  CK(cudaMemcpyAsync(m->d_state, &init, sizeof(StepState), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(m->d_scenes, 0, sizeof(SceneState) * S, s));
  CK(cudaMemsetAsync(m->d_sacc, 0, sizeof(double) * kSceneAcc * S, s));
  CK(cudaMemsetAsync(m->d_ndone, 0, sizeof(int32_t), s));
  if (o.persistent) {
    jgs2_status pst = run_batch_persistent<T>(m, o, s, L, d, corr);
    if (pst != JGS2_OK) return pst;
    StepState hs;
    CK(cudaMemcpyAsync(&hs, m->d_state, sizeof(StepState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs.status == JGS2_ETIMEOUT) return fail(JGS2_ETIMEOUT, "a bounded device wait timed out; state not written");
    CK(cudaEventRecord(m->gev[1], s));
    CK(cudaStreamWaitEvent(cs, m->gev[1], 0));
    return JGS2_OK;
  }
  const bool prof = L.prof;
  const long key = ((((((long)(sizeof(T) == 4) * 3 + o.correction) * 2 + (o.line_search != 0)) * 2 + (prof ? 1 : 0)) *
                          512 + bs) * 4096 + gbs * 8 + gtpv) * 4096 + chunk * 2 + m->cpf[pi] +
                        (long)(o.max_sweeps) * 1000003L +
                        (long)(o.rel_tol * 1e12);
  const bool same_view = m->gdev.size() == sizeof(d) && std::memcmp(m->gdev.data(), &d, sizeof(d)) == 0;
  if (m->graph_key != key || !same_view) {
    if (m->graph) cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
    m->graph_key = -1;
    m->ggroups.clear();
    const size_t nev = prof ? (size_t)32 : 0;
    while (m->gevents.size() < nev) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      m->gevents.push_back(e);
    }
    size_t evi = 0;
    cudaError_t cerr = cudaSuccess;
    bool timed = false;
    // kernel groups as in run_sweeps: kind, kernels, timing events on the chunk's last sweep
    auto group = [&](int kind, int n, cudaStream_t gs, auto&& launch) {
      Mesh::GraphGroup g{kind, n, nullptr, nullptr};
      if (timed) {
        g.e0 = m->gevents[evi++];
        g.e1 = m->gevents[evi++];
        if (cerr == cudaSuccess) cerr = cudaEventRecordWithFlags(g.e0, gs, cudaEventRecordExternal);
      }
      launch();
      if (timed && cerr == cudaSuccess) cerr = cudaEventRecordWithFlags(g.e1, gs, cudaEventRecordExternal);
      m->ggroups.push_back(g);
    };
    const int nbS = (S + 127) / 128;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int q = 0; q < chunk; ++q) {
      timed = prof && q == chunk - 1;
      group(JGS2_K_ELEM, 1, s, [&] { k_elem<T, true><<<nbT, 128, 0, s>>>(d, m->d_state); });
      group(JGS2_K_GATHER, 1, s,
            [&] { launch_gather<T, true>(d, m, corr, gbs, gtpv, s, m->d_state, m->d_partial, m->d_trace, 0); });
      // the cubature pool after the gather, whose g and R at the corners it reads
      if (corr) {
        group(JGS2_K_POOL, 1, s, [&] { k_pool<T, true><<<(m->nP + kPoolWarps - 1) / kPoolWarps, 32 * kPoolWarps, 0, s>>>(d, m->d_state); });
        group(JGS2_K_CORRECT, 1, s,
              [&] { launch_correct<T, true>(d, bs, s, m->d_state, m->d_partial, m->d_trace, 0, m->cpf[pi]); });
      }
      // per-scene stopping test (counted with the update)
      group(JGS2_K_UPDATE, 1, s, [&] {
        k_scene_finalize_main<<<nbS, 128, 0, s>>>(m->d_scenes, m->d_sacc, S, o.rel_tol, o.max_sweeps, corr ? 1 : 0,
                                                  m->d_ndone);
      });
      if (o.line_search) {
        // along D; along D_J only for the scenes whose trials along D all failed
        group(JGS2_K_ENERGY, corr ? 6 : 2, s, [&] {
          k_energy_batch<T, 0><<<nbT + nbV, 128, 0, s>>>(d, nbT);
          k_scene_finalize_energy<0><<<nbS, 128, 0, s>>>(m->d_scenes, m->d_sacc, S, corr ? 1 : 0);
          if (corr) {
            k_energy_batch<T, 1><<<nbT + nbV, 128, 0, s>>>(d, nbT);
            k_scene_finalize_energy<1><<<nbS, 128, 0, s>>>(m->d_scenes, m->d_sacc, S, 1);
            k_energy_batch<T, 2><<<nbT + nbV, 128, 0, s>>>(d, nbT);
            k_scene_finalize_energy<2><<<nbS, 128, 0, s>>>(m->d_scenes, m->d_sacc, S, 1);
          }
        });
      }
      group(JGS2_K_UPDATE, 1, s, [&] { k_update_batch<T><<<nbV, 128, 0, s>>>(d); });
    }
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) return fail(JGS2_ECUDA, std::string("batch sweep capture: ") + cudaGetErrorString(e));
    if (cerr != cudaSuccess) {
      cudaGraphDestroy(g);
      return fail(JGS2_ECUDA, std::string("batch sweep capture (events): ") + cudaGetErrorString(cerr));
    }
    e = cudaGraphInstantiate(&m->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(JGS2_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    m->graph_key = key;
    m->gdev.assign(reinterpret_cast<const char*>(&d), reinterpret_cast<const char*>(&d) + sizeof(d));
  }
  int32_t done = 0;
  for (int sw = 0; sw <= o.max_sweeps; sw += chunk) {
    CK(cudaGraphLaunch(m->graph, s));
    for (const auto& g : m->ggroups) L.count[g.kind] += g.n;
    CK(cudaMemcpyAsync(&done, m->d_ndone, sizeof(done), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (prof) {
      // the timed (last) sweep of this replay did work unless every scene stopped before it
      bool did = done < S;
      if (!did) {
        std::vector<SceneState> sc(S);
        CK(cudaMemcpy(sc.data(), m->d_scenes, sizeof(SceneState) * S, cudaMemcpyDeviceToHost));
        int kmax = 0;
        for (const auto& q : sc) kmax = std::max(kmax, (int)q.sweeps);
        did = sw + chunk - 1 <= kmax;
      }
      if (did) {
        L.psweeps += 1;
        for (const auto& g : m->ggroups) {
          float ms = 0.f;
          if (g.e0 && cudaEventElapsedTime(&ms, g.e0, g.e1) == cudaSuccess) L.gms[g.kind] += ms;
        }
      }
    }
    if (done >= S) break;
  }
  {
    // a bounded device wait that gave up stops the batch step (status in the step state)
    StepState hs;
    CK(cudaMemcpyAsync(&hs, m->d_state, sizeof(StepState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs.status == JGS2_ETIMEOUT) return fail(JGS2_ETIMEOUT, "a bounded device wait timed out; state not written");
  }
  CK(cudaGetLastError());
  CK(cudaEventRecord(m->gev[1], s));
  CK(cudaStreamWaitEvent(cs, m->gev[1], 0));
  return JGS2_OK;
}

static jgs2_status check_opts(const Mesh* m, const jgs2_step_opts* o) {
  if (!o) return fail(JGS2_EINVAL, "null options");
  if (o->max_sweeps < 0 || o->max_sweeps > 1000000) return fail(JGS2_EINVAL, "max_sweeps out of range");
  if (o->precision != JGS2_FP64 && o->precision != JGS2_FP32) return fail(JGS2_EINVAL, "bad precision");
  if (o->correction < 0 || o->correction > 2) return fail(JGS2_EINVAL, "bad correction");
  if (o->correction != JGS2_CORR_OFF && m->n_cub == 0)
    return fail(JGS2_ENOTPRECOMPUTED, "correction requested before jgs2_precompute / jgs2_precompute_import");
  if (!(o->dx_tol >= 0.0)) return fail(JGS2_EINVAL, "dx_tol must be >= 0");
  if (o->wait_polls < 0) return fail(JGS2_EINVAL, "wait_polls must be >= 0");
  if (o->dx_tol > 0.0 && m->n_scenes > 0)
    return fail(JGS2_EINVAL, "the position-change test (dx_tol) is for single scenes, not batch meshes");
  return JGS2_OK;
}

template <typename T>
static jgs2_status step_impl(Mesh* m, double* x, double* v, const jgs2_step_opts* o, cudaStream_t s,
                             jgs2_step_report* rep, int gs_ncol = 0) {
  jgs2_status st = ensure_prec<T>(m);
  if (st != JGS2_OK) return st;
  DevMesh<T> d = dev_view<T>(m);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  const int nb = (m->V + 127) / 128;
  Launches L{m, s, o->profile != 0};
  int id = L.begin(JGS2_K_SETUP);
  k_setup_vertices<T><<<nb, 128, 0, s>>>(d, x, v, nullptr);
  L.end(id);
  id = L.begin(JGS2_K_SETUP);
  k_setup_tets<T><<<(m->T + 127) / 128, 128, 0, s>>>(d);
  L.end(id);
  CK(cudaGetLastError());
  StepState* hs = m->h_state;
  if (m->Vf == 0) {
    // no free vertex: every position is prescribed, x_{t+1} = x_t with no sweep (r = 0)
    std::memset(hs, 0, sizeof(StepState));
    hs->converged = 1;
  } else if (m->n_scenes > 0) {
    st = run_sweeps_batch<T>(m, *o, s, L);
    if (st != JGS2_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return st;
    }
    std::vector<SceneState> sc(m->n_scenes);
    CK(cudaMemcpy(sc.data(), m->d_scenes, sizeof(SceneState) * m->n_scenes, cudaMemcpyDeviceToHost));
    std::memset(hs, 0, sizeof(StepState));
    hs->converged = 1;
    for (auto& q : sc) {
      hs->sweeps = std::max(hs->sweeps, q.sweeps);
      hs->converged &= q.converged;
      hs->fallback += q.fallback;
      hs->ls_rejects += q.ls_rejects;
      hs->r = std::max(hs->r, q.r);
      if (q.status) hs->status = q.status;
    }
  } else {
    st = run_sweeps<T>(m, *o, s, o->max_sweeps, o->rel_tol, true, hs, L, gs_ncol);
  }
  if (st != JGS2_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
  }
  if (hs->status == 0) {
    id = L.begin(JGS2_K_SETUP);
    k_finish<T><<<nb, 128, 0, s>>>(d, x, v);
    L.end(id);
  }
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rep) {
    rep->sweeps = hs->sweeps;
    rep->converged = hs->converged;
    rep->fallback = hs->fallback;
    rep->ls_rejects = hs->ls_rejects;
    rep->dj_steps = hs->dj_steps;
    rep->contact_rebuilds = hs->rebuilds;
    rep->contact_candidates = 0;
    rep->contact_near = 0;
    if (m->contact) {
      uint32_t near = 0;
      int32_t cand = 0;
      CK(cudaMemcpy(&cand, m->d_npairs, sizeof(cand), cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(&near, m->d_ctl + kCtlNear, sizeof(near), cudaMemcpyDeviceToHost));
      rep->contact_candidates = cand;
      rep->contact_near = (int32_t)near;
    }
    rep->rel_residual = hs->r;
    rep->g0 = hs->g0;
    rep->ms = ms;
    rep->trace_len = 0;
    rep->stopped_dx = hs->stopped_dx;
    for (int q = 0; q < 3; ++q) rep->ls_passes[q] = hs->ls_passes[q];
    {
      const double L = o->length_scale > 0.0 ? o->length_scale : m->extent;
      rep->last_dx = (hs->sweeps > 0 && L > 0.0) ? std::sqrt(hs->dx2_applied) / L : 0.0;
    }
    L.report(rep);
    if (o->record_trace) {
      const int n = std::min(hs->sweeps + 1, JGS2_TRACE_MAX);
      CK(cudaMemcpy(rep->trace, m->d_trace, sizeof(double) * n, cudaMemcpyDeviceToHost));
      rep->trace_len = n;
    }
  }
  if (hs->status != 0) {
    const char* why = hs->status == JGS2_ETIMEOUT     ? "a bounded device wait timed out; state not written"
                      : hs->status == JGS2_EINTERSECT ? "contact pair at zero distance; state not written"
                                                      : "residual became non-finite; state not written";
    return fail((jgs2_status)hs->status, why);
  }
  if (!hs->converged && !hs->stopped_dx) return fail(JGS2_ENOTCONVERGED, "max_sweeps reached before rel_tol");
  return JGS2_OK;
}

jgs2_status step(Mesh* m, double* x, double* v, const jgs2_step_opts* o, void* stream, jgs2_step_report* rep) {
  if (!m || !x || !v) return fail(JGS2_EINVAL, "null argument");
  jgs2_status st = check_opts(m, o);
  if (st != JGS2_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  return o->precision == JGS2_FP64 ? step_impl<double>(m, x, v, o, s, rep) : step_impl<float>(m, x, v, o, s, rep);
}

template <typename T>
static jgs2_status sweeps_impl(Mesh* m, const double* xt, const double* vt, double* xk, int n,
                               const jgs2_step_opts* o, cudaStream_t s) {
  jgs2_status st = ensure_prec<T>(m);
  if (st != JGS2_OK) return st;
  DevMesh<T> d = dev_view<T>(m);
  const int nb = (m->V + 127) / 128;
  k_setup_vertices<T><<<nb, 128, 0, s>>>(d, xt, vt, xk);
  k_setup_tets<T><<<(m->T + 127) / 128, 128, 0, s>>>(d);
  CK(cudaGetLastError());
  // exactly n sweeps: no convergence test (rel_tol < 0), stop after the n-th update
  Launches L{m, s, false};
  if (m->Vf > 0) st = run_sweeps<T>(m, *o, s, n, -1.0, false, m->h_state, L);
  if (st != JGS2_OK) return st;
  k_finish<T><<<nb, 128, 0, s>>>(d, xk, nullptr);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return JGS2_OK;
}

jgs2_status sweeps(Mesh* m, const double* xt, const double* vt, double* xk, int n, const jgs2_step_opts* o,
                   void* stream) {
  if (!m || !xt || !vt || !xk || n < 0) return fail(JGS2_EINVAL, "bad argument");
  jgs2_status st = check_opts(m, o);
  if (st != JGS2_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  return o->precision == JGS2_FP64 ? sweeps_impl<double>(m, xt, vt, xk, n, o, s)
                                   : sweeps_impl<float>(m, xt, vt, xk, n, o, s);
}

jgs2_status energy_gradient(Mesh* m, const double* xt, const double* vt, const double* x, double* E, double* g,
                            void* stream) {
  if (!m || !xt || !vt || !x) return fail(JGS2_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  jgs2_status st = ensure_prec<double>(m);
  if (st != JGS2_OK) return st;
  DevMesh<double> d = dev_view<double>(m);
  const int nb = (m->V + 127) / 128;
  k_setup_vertices<double><<<nb, 128, 0, s>>>(d, xt, vt, x);
  k_setup_tets<double><<<(m->T + 127) / 128, 128, 0, s>>>(d);
  // pinned vertices keep x_t; a caller x that moves them is a different problem
  if (m->contact) {
    CK(cudaMemsetAsync(m->d_state, 0, sizeof(StepState), s));
    st = contact_force_rebuild(m, s);
    if (st != JGS2_OK) return st;
    st = contact_pass<double>(m, d, s, m->d_state);
    if (st != JGS2_OK) return st;
  }
  if (g) k_grad<double><<<nb, 128, 0, s>>>(d, g);
  if (E) {
    const int nbT = (m->T + 127) / 128, nbV = (m->Vf + 127) / 128;
    k_energy_abs<double><<<nbT + nbV, 128, 0, s>>>(d, m->d_partial, nbT);
    std::vector<double> p(nbT + nbV);
    CK(cudaMemcpyAsync(p.data(), m->d_partial, sizeof(double) * p.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double acc = 0.0;
    for (double q : p) acc += q;
    if (m->contact) {
      CK(cudaMemsetAsync(m->d_partial, 0, sizeof(double), s));
      k_pair_energy<double><<<148, 128, 0, s>>>(d, d.c, m->d_partial);
      double eb = 0.0;
      CK(cudaMemcpyAsync(&eb, m->d_partial, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      acc += eb;
    }
    *E = acc;
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return JGS2_OK;
}

jgs2_status contact_pairs(Mesh* m, const double* xt, const double* x, double radius, int32_t* out, int cap,
                          int32_t* n_out, void* stream) {
  if (!m || !xt || !x || !n_out || (cap > 0 && !out)) return fail(JGS2_EINVAL, "null argument");
  if (!m->contact) return fail(JGS2_EINVAL, "mesh was created without contact");
  if (!(radius > 0.0)) return fail(JGS2_EINVAL, "radius must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  jgs2_status st = ensure_prec<double>(m);
  if (st != JGS2_OK) return st;
  DevMesh<double> d = dev_view<double>(m);
  d.c.R = radius;
  d.c.rc = radius;
  const int nb = (m->V + 127) / 128;
  k_setup_vertices<double><<<nb, 128, 0, s>>>(d, xt, xt, x);
  CK(cudaMemsetAsync(m->d_state, 0, sizeof(StepState), s));
  st = contact_force_rebuild(m, s);
  if (st != JGS2_OK) return st;
  st = contact_pass<double>(m, d, s, m->d_state);
  if (st != JGS2_OK) return st;
  int32_t n = 0, fl[2] = {0, 0};
  CK(cudaMemcpyAsync(&n, m->d_npairs, sizeof(n), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(fl, m->d_cflags, sizeof(fl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaMemset(m->d_cflags, 0, sizeof(fl)));
  if (fl[0] || n > m->pair_cap) return fail(JGS2_ENOMEM, "contact pair buffer overflow");
  std::vector<uint64_t> keys(n);
  if (n) CK(cudaMemcpy(keys.data(), m->d_pairs, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost));
  std::vector<std::array<int, 5>> rows(n);
  for (int q = 0; q < n; ++q) {
    const int kind = (int)(keys[q] >> 60), a = (int)((keys[q] >> 30) & 0x3fffffff), b = (int)(keys[q] & 0x3fffffff);
    std::array<int, 5> r{kind, -1, -1, -1, -1};
    if (kind == 0) {
      r[1] = m->perm[a];
      r[2] = b;
    } else if (kind == 1) {
      r[1] = m->perm[a];
      int f[3] = {m->perm[m->sfaces[3 * b]], m->perm[m->sfaces[3 * b + 1]], m->perm[m->sfaces[3 * b + 2]]};
      std::sort(f, f + 3);
      r[2] = f[0];
      r[3] = f[1];
      r[4] = f[2];
    } else {
      int e1[2] = {m->perm[m->sedges[2 * a]], m->perm[m->sedges[2 * a + 1]]};
      int e2[2] = {m->perm[m->sedges[2 * b]], m->perm[m->sedges[2 * b + 1]]};
      std::sort(e1, e1 + 2);
      std::sort(e2, e2 + 2);
      if (std::make_pair(e2[0], e2[1]) < std::make_pair(e1[0], e1[1])) {
        std::swap(e1[0], e2[0]);
        std::swap(e1[1], e2[1]);
      }
      r[1] = e1[0];
      r[2] = e1[1];
      r[3] = e2[0];
      r[4] = e2[1];
    }
    rows[q] = r;
  }
  std::sort(rows.begin(), rows.end());
  *n_out = n;
  for (int q = 0; q < std::min(n, cap); ++q)
    for (int k = 0; k < 5; ++k) out[5 * q + k] = rows[q][k];
  if (n > cap) return fail(JGS2_ENOMEM, "more pairs than cap");
  return JGS2_OK;
}

// Several scenes in one mesh (scene-major vertex order), each with its own convergence.
jgs2_status mesh_create_batch(const jgs2_mesh_desc* ds, int n, Mesh** out) {
  if (!ds || n <= 0 || !out) return fail(JGS2_EINVAL, "bad batch arguments");
  jgs2_mesh_desc all = ds[0];
  std::vector<double> X, E, nu, rho;
  std::vector<int> tets, scene;
  std::vector<uint8_t> pin;
  int V = 0;
  for (int k = 0; k < n; ++k) {
    const jgs2_mesh_desc& d = ds[k];
    if (d.contact || d.friction_mu != 0.0) return fail(JGS2_EINVAL, "batch meshes do not support contact");
    if (d.dt != all.dt || d.gravity[0] != all.gravity[0] || d.gravity[1] != all.gravity[1] ||
        d.gravity[2] != all.gravity[2])
      return fail(JGS2_EINVAL, "all scenes of a batch must share dt and gravity");
    if (d.n_vertices <= 0 || d.n_tets <= 0 || !d.rest_pos || !d.tets || !d.youngs || !d.poisson || !d.density)
      return fail(JGS2_EINVAL, "bad scene " + std::to_string(k));
    X.insert(X.end(), d.rest_pos, d.rest_pos + 3 * (size_t)d.n_vertices);
    for (int q = 0; q < 4 * d.n_tets; ++q) {
      if (d.tets[q] < 0 || d.tets[q] >= d.n_vertices) return fail(JGS2_EINVAL, "tet index out of range");
      tets.push_back(d.tets[q] + V);
    }
    E.insert(E.end(), d.youngs, d.youngs + d.n_tets);
    nu.insert(nu.end(), d.poisson, d.poisson + d.n_tets);
    rho.insert(rho.end(), d.density, d.density + d.n_tets);
    for (int v = 0; v < d.n_vertices; ++v) {
      pin.push_back(d.pinned ? (d.pinned[v] ? 1 : 0) : 0);
      scene.push_back(k);
    }
    V += d.n_vertices;
  }
  all.n_vertices = V;
  all.n_tets = (int)E.size();
  all.rest_pos = X.data();
  all.tets = tets.data();
  all.youngs = E.data();
  all.poisson = nu.data();
  all.density = rho.data();
  all.pinned = pin.data();
  all.contact = 0;
  Mesh* m = nullptr;
  jgs2_status st = mesh_create(&all, &m, &scene);
  if (st != JGS2_OK) return st;
  m->n_scenes = n;
  m->vscene = scene;
  *out = m;
  return JGS2_OK;
}

jgs2_status batch_report(const Mesh* m, int32_t* sweeps, int32_t* converged, double* rel) {
  if (!m || m->n_scenes <= 0) return fail(JGS2_EINVAL, "not a batch mesh");
  if (!m->d_scenes) return fail(JGS2_EINVAL, "no step has run on this mesh");
  std::vector<SceneState> sc(m->n_scenes);
  CK(cudaMemcpy(sc.data(), m->d_scenes, sizeof(SceneState) * m->n_scenes, cudaMemcpyDeviceToHost));
  for (int k = 0; k < m->n_scenes; ++k) {
    if (sweeps) sweeps[k] = sc[k].sweeps;
    if (converged) converged[k] = sc[k].converged;
    if (rel) rel[k] = sc[k].r;
  }
  return JGS2_OK;
}

// Autotuner: on the state (x, v), times k_gather in each launch shape (threads per block x
// threads per vertex: 64/128/256 x 1, 128/256 x 4) and k_correct at 64, 128 and 256 threads
// per block, and keeps the fastest of each for this precision.
template <typename T>
static jgs2_status autotune_impl(Mesh* m, double* x, double* v, const jgs2_step_opts* o, cudaStream_t s,
                                 int32_t* chosen) {
  jgs2_status st = ensure_prec<T>(m);
  if (st != JGS2_OK) return st;
  const int pi = sizeof(T) == 4 ? 1 : 0;
  if (m->Vf == 0) {
    // nothing to time: the step of a mesh without free vertices launches no sweep kernel
    if (chosen) *chosen = m->bs[pi];
    return JGS2_OK;
  }
  DevMesh<T> d = dev_view<T>(m);
  const int nb = (m->V + 127) / 128;
  const bool corr = o->correction != JGS2_CORR_OFF && m->nP > 0;
  k_setup_vertices<T><<<nb, 128, 0, s>>>(d, x, v, nullptr);
  k_setup_tets<T><<<(m->T + 127) / 128, 128, 0, s>>>(d);
  StepState init;
  std::memset(&init, 0, sizeof(init));
  init.max_sweeps = 1 << 30;
  init.rel_tol = -1.0;
  CK(cudaMemcpyAsync(m->d_state, &init, sizeof(StepState), cudaMemcpyHostToDevice, s));
  k_elem<T, false><<<(m->T + 127) / 128, 128, 0, s>>>(d, m->d_state);
  launch_gather<T, false>(d, m, corr, 128, 1, s, m->d_state, m->d_partial, m->d_trace, 0);
  if (corr) k_pool<T, true><<<(m->nP + kPoolWarps - 1) / kPoolWarps, 32 * kPoolWarps, 0, s>>>(d, m->d_state);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // times `launch` (2 untimed, 5 timed launches); every launch is sweep 0 of a fresh state:
  // it sets |g(x^0)| and never stops the step (rel_tol < 0, no sweep cap), so each launch
  // does the full work
  auto time_it = [&](auto&& launch) -> float {
    for (int rep = 0; rep < 2; ++rep) launch();
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 5; ++rep) launch();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  float best = 1e30f;
  int gpick = 0;
  for (int c = 0; c < 5; ++c) {
    const int b = kGatherShapes[c][0], p = kGatherShapes[c][1];
    const float ms =
        time_it([&] { launch_gather<T, false>(d, m, corr, b, p, s, m->d_state, m->d_partial, m->d_trace, 0); });
    if (ms < best) {
      best = ms;
      gpick = c;
    }
  }
  int cpick = 128, ppick = 0;
  if (corr) {
    best = 1e30f;
    for (int pf = 0; pf < 2; ++pf)
      for (int c : {64, 128, 256}) {
        const float ms =
            time_it([&] { launch_correct<T, false>(d, c, s, m->d_state, m->d_partial, m->d_trace, 0, pf); });
        if (ms < best) {
          best = ms;
          cpick = c;
          ppick = pf;
        }
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  m->bs[pi] = cpick;
  m->cpf[pi] = ppick;
  m->gbs[pi] = kGatherShapes[gpick][0];
  m->gtpv[pi] = kGatherShapes[gpick][1];
  m->graph_key = -1;
  if (chosen) *chosen = cpick;
  return JGS2_OK;
}

jgs2_status autotune(Mesh* m, double* x, double* v, const jgs2_step_opts* o, void* stream, int32_t* chosen) {
  if (!m || !x || !v) return fail(JGS2_EINVAL, "null argument");
  jgs2_status st = check_opts(m, o);
  if (st != JGS2_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  return o->precision == JGS2_FP64 ? autotune_impl<double>(m, x, v, o, s, chosen)
                                   : autotune_impl<float>(m, x, v, o, s, chosen);
}

// New Young's moduli (caller tet order): mu, lam' and the device records are updated. The
// cubature records keep the rest subspace of the old moduli (it only shapes the rate).
jgs2_status set_youngs(Mesh* m, const double* E) {
  if (!m || !E) return fail(JGS2_EINVAL, "null argument");
  for (int t = 0; t < m->T; ++t)
    if (!(E[t] > 0.0) || !std::isfinite(E[t])) return fail(JGS2_EINVAL, "Young's modulus must be positive");
  for (int t = 0; t < m->T; ++t) {
    m->E[t] = E[t];
    const double nu = m->nu[t];
    m->mu[t] = E[t] / (2.0 * (1.0 + nu));
    m->lp[t] = E[t] * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)) + m->mu[t];
  }
  if (m->device_ready) CK(cudaMemcpy(m->d_youngs, m->E.data(), sizeof(double) * m->T, cudaMemcpyHostToDevice));
  if (m->f32.ready) {
    std::vector<TetRec<float>> rec;
    tet_records<float>(m, rec);
    CK(cudaMemcpy(m->f32.tets, rec.data(), sizeof(TetRec<float>) * m->T, cudaMemcpyHostToDevice));
  }
  if (m->f64.ready) {
    std::vector<TetRec<double>> rec;
    tet_records<double>(m, rec);
    CK(cudaMemcpy(m->f64.tets, rec.data(), sizeof(TetRec<double>) * m->T, cudaMemcpyHostToDevice));
  }
  return JGS2_OK;
}

template <typename T>
static jgs2_status adjoint_impl(Mesh* m, const double* xt, const double* vt, const double* x1, const double* gx1,
                                const double* gv1, double* gx, double* gv, double* gE, const jgs2_adjoint_opts* o,
                                cudaStream_t s, jgs2_adjoint_report* rep) {
  jgs2_status st = ensure_prec<T>(m);
  if (st != JGS2_OK) return st;
  PrecBufs<T>& b = bufs<T>(m);
  const int Vf = m->Vf;
  if (!b.a_lam) {
    CK(dalloc(&b.a_lam, Vf));
    CK(dalloc(&b.a_r, Vf));
    CK(dalloc(&b.a_z, Vf));
    CK(dalloc(&b.a_p, Vf));
    CK(dalloc(&b.a_q, Vf));
    CK(dalloc(&b.a_lin, 15 * (size_t)Vf));
  }
  if (!m->d_coup) {
    CK(dalloc(&m->d_coup, 3 * (size_t)m->V));
    CK(cudaMalloc(&m->d_adjsc, sizeof(AdjScalars)));
  }
  DevMesh<T> d = dev_view<T>(m);
  const bool corr = o->correction != JGS2_CORR_OFF && m->nP > 0;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  const int nb = (m->V + 127) / 128, nbV = (Vf + 127) / 128, nbT = (m->T + 127) / 128;
  k_setup_vertices<T><<<nb, 128, 0, s>>>(d, xt, vt, x1);
  k_setup_tets<T><<<nbT, 128, 0, s>>>(d);
  StepState init;
  std::memset(&init, 0, sizeof(init));
  init.max_sweeps = 1 << 30;
  init.rel_tol = -1.0;
  CK(cudaMemcpyAsync(m->d_state, &init, sizeof(StepState), cudaMemcpyHostToDevice, s));
  // H_ii, R_i at x* (and the rotated cubature element Hessians)
  k_elem<T, false><<<nbT, 128, 0, s>>>(d, m->d_state);
  launch_gather<T, false>(d, m, true, 128, 1, s, m->d_state, m->d_partial, m->d_trace, 0);
  if (corr) k_pool<T, true><<<(m->nP + kPoolWarps - 1) / kPoolWarps, 32 * kPoolWarps, 0, s>>>(d, m->d_state);
  if (corr)
    k_lin_setup<T, true><<<nbV, 128, 0, s>>>(d, b.a_lin);
  else
    k_lin_setup<T, false><<<nbV, 128, 0, s>>>(d, b.a_lin);
  AdjScalars* sc = static_cast<AdjScalars*>(m->d_adjsc);
  AdjScalars sc0;
  std::memset(&sc0, 0, sizeof(sc0));
  CK(cudaMemcpyAsync(sc, &sc0, sizeof(sc0), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(b.a_lam, 0, sizeof(Vec4<T>) * Vf, s));
  k_adj_rhs<T><<<nbV, 128, 0, s>>>(d, gx1, gv1, b.a_r);
  const int nbD = std::max(1, std::min(nbV, 148 * 8));
  const double tol2 = o->rel_tol * o->rel_tol;
  k_dots<T><<<nbD, 128, 0, s>>>(d, b.a_r, b.a_r, b.a_r, b.a_r, m->d_partial, sc, 2, tol2, o->max_iters);
  // preconditioner: the local matrices of the sweep at x* (H_ii, plus the rotated cubature
  // Hessian H~_i with the correction on; both symmetric positive definite). The cubature
  // estimate of the residual's reduced part is left out: with it the preconditioned operator
  // has eigenvalues of negative real part, and conjugate gradients stall
  auto precond = [&]() { k_lin_precond<T, false><<<nbV, 128, 0, s>>>(d, b.a_lin, b.a_r, b.a_z, sc); };
  precond();
  CK(cudaMemcpyAsync(b.a_p, b.a_z, sizeof(Vec4<T>) * Vf, cudaMemcpyDeviceToDevice, s));
  AdjScalars hs;
  const int every = std::max(1, o->check_every);
  for (int it = 0; it < o->max_iters; ++it) {
    k_hv<T><<<nbV, 128, 0, s>>>(d, b.a_p, b.a_q, sc);
    k_dots<T><<<nbD, 128, 0, s>>>(d, b.a_p, b.a_q, b.a_r, b.a_p, m->d_partial, sc, 0, tol2, o->max_iters);
    k_axpy2<T><<<nbV, 128, 0, s>>>(d, b.a_lam, b.a_r, b.a_p, b.a_q, sc);
    precond();
    k_dots<T><<<nbD, 128, 0, s>>>(d, b.a_z, b.a_q, b.a_r, b.a_r, m->d_partial, sc, 1, tol2, o->max_iters);
    k_pupdate<T><<<nbV, 128, 0, s>>>(d, b.a_p, b.a_z, sc);
    CK(cudaGetLastError());
    if ((it + 1) % every == 0) {
      CK(cudaMemcpyAsync(&hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (hs.done) break;
    }
  }
  CK(cudaMemsetAsync(m->d_coup, 0, sizeof(double) * 3 * m->V, s));
  k_adj_tets<T><<<nbT, 128, 0, s>>>(d, b.a_lam, m->d_tperm, m->d_youngs, m->d_coup, gE);
  k_adj_out<T><<<nb, 128, 0, s>>>(d, b.a_lam, m->d_coup, gx1, gv1, gx, gv);
  CK(cudaEventRecord(e1, s));
  CK(cudaMemcpyAsync(&hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const bool conv = hs.rr0 == 0.0 || hs.rr <= tol2 * hs.rr0;
  if (rep) {
    rep->iters = hs.iters;
    rep->converged = conv ? 1 : 0;
    rep->rel_residual = hs.rr0 > 0.0 ? std::sqrt(hs.rr / hs.rr0) : 0.0;
    rep->ms = ms;
  }
  if (hs.done == 2) return fail(JGS2_ENONSPD, "Hessian not positive definite along a search direction");
  if (!conv) return fail(JGS2_ENOTCONVERGED, "adjoint solve reached max_iters before rel_tol");
  return JGS2_OK;
}

jgs2_status step_adjoint(Mesh* m, const double* xt, const double* vt, const double* x1, const double* gx1,
                         const double* gv1, double* gx, double* gv, double* gE, const jgs2_adjoint_opts* o,
                         void* stream, jgs2_adjoint_report* rep) {
  if (!m || !xt || !vt || !x1 || !gx1 || !gv1 || !gx || !gv || !gE || !o) return fail(JGS2_EINVAL, "null argument");
  if (m->contact) return fail(JGS2_EINVAL, "the adjoint does not include contact terms");
  if (o->max_iters < 1 || !(o->rel_tol > 0.0)) return fail(JGS2_EINVAL, "bad adjoint options");
  if (m->Vf == 0) return fail(JGS2_EINVAL, "the mesh has no free vertex");
  if (o->correction != JGS2_CORR_OFF && m->n_cub == 0)
    return fail(JGS2_ENOTPRECOMPUTED, "corrected preconditioner requested before a precompute");
  cudaStream_t s = (cudaStream_t)stream;
  return o->precision == JGS2_FP64 ? adjoint_impl<double>(m, xt, vt, x1, gx1, gv1, gx, gv, gE, o, s, rep)
                                   : adjoint_impl<float>(m, xt, vt, x1, gx1, gv1, gx, gv, gE, o, s, rep);
}


// Gauss-Seidel step (Sec. 8.1; readings R19-R21): the free vertices are coloured greedily in
// caller order; a GS sweep runs the colours in turn, each as one sweep of the Jacobi
// machinery whose directions are masked to the colour (the line search then moves only that
// colour). The relative residual is taken in FP64 at the start of each GS sweep.
jgs2_status step_gs(Mesh* m, double* x, double* v, const jgs2_step_opts* o, void* stream,
                    jgs2_step_report* rep) {
  if (!m || !x || !v) return fail(JGS2_EINVAL, "null argument");
  jgs2_status st = check_opts(m, o);
  if (st != JGS2_OK) return st;
  if (m->contact || m->n_scenes > 0)
    return fail(JGS2_EINVAL, "the Gauss-Seidel step takes single scenes without contact");
  cudaStream_t s = (cudaStream_t)stream;
  const int V = m->V, Vf = m->Vf;
  if (!m->d_gsmask && Vf > 0) {
    // greedy colouring in caller order over the free vertices that share a tet
    std::vector<std::vector<int>> nbr(V);
    for (int t = 0; t < m->T; ++t)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          if (a != b) nbr[m->tets_c[4 * (size_t)t + a]].push_back(m->tets_c[4 * (size_t)t + b]);
    std::vector<int> col(V, -1);
    int ncol = 0;
    for (int c = 0; c < V; ++c) {
      if (m->pinned[c]) continue;
      std::vector<char> used(nbr[c].size() + 1, 0);
      for (int u : nbr[c])
        if (col[u] >= 0 && col[u] < (int)used.size()) used[col[u]] = 1;
      int k = 0;
      while (used[k]) ++k;
      col[c] = k;
      ncol = std::max(ncol, k + 1);
    }
    std::vector<uint8_t> masks((size_t)ncol * Vf, 0);
    for (int i = 0; i < Vf; ++i) masks[(size_t)col[m->perm[i]] * Vf + i] = 1;
    CK(dalloc(&m->d_gsmask, masks.size()));
    CK(cudaMemcpy(m->d_gsmask, masks.data(), masks.size(), cudaMemcpyHostToDevice));
    m->gs_ncol = ncol;
  }
  // the GS sweeps run as graph-captured colour passes of the Jacobi machinery (one pass per
  // colour with the colour's vertex mask; the stopping test at each GS sweep's first pass)
  return o->precision == JGS2_FP64 ? step_impl<double>(m, x, v, o, s, rep, m->gs_ncol)
                                   : step_impl<float>(m, x, v, o, s, rep, m->gs_ncol);
}

}  // namespace jgs2

// ------------------------------------------------------------------ C ABI

using namespace jgs2;

extern "C" {

void jgs2_precompute_opts_default(jgs2_precompute_opts* o) {
  if (!o) return;
  o->n_cub = 4;
  o->n_train = 20;
  o->n_cand = 32;
  o->n_pool = 256;
  o->nnls_tol = 0.01;
  o->seed = 0;
  o->n_threads = 0;
  o->gs = 0;
  o->gpu = 0;
}

void jgs2_step_opts_default(jgs2_step_opts* o) {
  if (!o) return;
  o->max_sweeps = 500;
  o->rel_tol = 1e-4;
  o->precision = JGS2_FP32;
  o->correction = JGS2_CORR_ASM;
  o->line_search = 1;
  o->check_every = 16;
  o->record_trace = 0;
  o->profile = 0;
  o->dx_tol = 0.0;
  o->length_scale = 0.0;
  o->persistent = 0;
  o->wait_polls = 0;
  o->test_unreachable_barrier = 0;
  o->contact_coupling = 0;
}

jgs2_status jgs2_mesh_create(const jgs2_mesh_desc* desc, jgs2_mesh** out) {
  Mesh* m = nullptr;
  jgs2_status s = mesh_create(desc, &m);
  if (out) *out = reinterpret_cast<jgs2_mesh*>(m);
  return s;
}

jgs2_status jgs2_precompute_import(jgs2_mesh* mesh, const jgs2_cubature_blob* blob) {
  return import_cubature(reinterpret_cast<Mesh*>(mesh), blob);
}

int32_t jgs2_mesh_n_cub(const jgs2_mesh* mesh) {
  return mesh ? reinterpret_cast<const Mesh*>(mesh)->n_cub : 0;
}

jgs2_status jgs2_precompute_export(const jgs2_mesh* mesh, int32_t* elem, double* weight, double* ubar,
                                   double* residual) {
  const Mesh* m = reinterpret_cast<const Mesh*>(mesh);
  if (!m || !elem || !weight || !ubar) return fail(JGS2_EINVAL, "null argument");
  const int nc = m->n_cub;
  if (nc == 0) return fail(JGS2_ENOTPRECOMPUTED, "no cubature records");
  for (int c = 0; c < m->V; ++c) {
    const int i = m->iperm[c];
    for (int s = 0; s < nc; ++s) {
      const size_t o = (size_t)c * nc + s;
      elem[o] = -1;
      weight[o] = 0.0;
      for (int q = 0; q < 36; ++q) ubar[o * 36 + q] = 0.0;
      if (i >= m->Vf) continue;
      const int e = m->cub_elem[(size_t)i * nc + s];
      if (e < 0) continue;
      elem[o] = m->tperm[e];
      weight[o] = m->cub_w[(size_t)i * nc + s];
      for (int q = 0; q < 36; ++q) ubar[o * 36 + q] = m->cub_u[((size_t)i * nc + s) * 36 + q];
    }
    if (residual) residual[c] = (size_t)c < m->cub_resid.size() ? m->cub_resid[c] : std::nan("");
  }
  return JGS2_OK;
}

jgs2_status jgs2_step(jgs2_mesh* mesh, double* x, double* v, const jgs2_step_opts* opts, void* stream,
                      jgs2_step_report* report) {
  return step(reinterpret_cast<Mesh*>(mesh), x, v, opts, stream, report);
}

jgs2_status jgs2_step_gs(jgs2_mesh* mesh, double* x, double* v, const jgs2_step_opts* opts, void* stream,
                         jgs2_step_report* report) {
  return step_gs(reinterpret_cast<Mesh*>(mesh), x, v, opts, stream, report);
}

jgs2_status jgs2_step_host(jgs2_mesh* mesh, double* x, double* v, const jgs2_step_opts* opts, void* stream,
                           jgs2_step_report* report) {
  Mesh* m = reinterpret_cast<Mesh*>(mesh);
  if (!m || !x || !v) return fail(JGS2_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = 3 * (size_t)m->V;
  if (!m->d_xbuf) {
    CK(dalloc(&m->d_xbuf, n));
    CK(dalloc(&m->d_vbuf, n));
  }
  CK(cudaMemcpyAsync(m->d_xbuf, x, n * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(m->d_vbuf, v, n * sizeof(double), cudaMemcpyHostToDevice, s));
  jgs2_status st = step(m, m->d_xbuf, m->d_vbuf, opts, stream, report);
  if (st != JGS2_OK && st != JGS2_ENOTCONVERGED) return st;
  CK(cudaMemcpyAsync(x, m->d_xbuf, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(v, m->d_vbuf, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return st;
}

jgs2_status jgs2_sweeps(jgs2_mesh* mesh, const double* x_t, const double* v_t, double* x_k, int32_t n_sweeps,
                        const jgs2_step_opts* opts, void* stream) {
  return sweeps(reinterpret_cast<Mesh*>(mesh), x_t, v_t, x_k, n_sweeps, opts, stream);
}

jgs2_status jgs2_energy_gradient(jgs2_mesh* mesh, const double* x_t, const double* v_t, const double* x,
                                 double* energy, double* g, void* stream) {
  return energy_gradient(reinterpret_cast<Mesh*>(mesh), x_t, v_t, x, energy, g, stream);
}

jgs2_status jgs2_contact_pairs(jgs2_mesh* mesh, const double* x_t, const double* x, double radius, int32_t* out,
                               int32_t cap, int32_t* n_out, void* stream) {
  return contact_pairs(reinterpret_cast<Mesh*>(mesh), x_t, x, radius, out, cap, n_out, stream);
}

void jgs2_adjoint_opts_default(jgs2_adjoint_opts* o) {
  if (!o) return;
  o->max_iters = 5000;
  o->rel_tol = 1e-6;
  o->precision = JGS2_FP64;
  o->correction = JGS2_CORR_OFF;
  o->check_every = 32;
}

jgs2_status jgs2_step_adjoint(jgs2_mesh* mesh, const double* x_t, const double* v_t, const double* x_t1,
                              const double* gx_t1, const double* gv_t1, double* gx_t, double* gv_t, double* gE,
                              const jgs2_adjoint_opts* opts, void* stream, jgs2_adjoint_report* report) {
  return step_adjoint(reinterpret_cast<Mesh*>(mesh), x_t, v_t, x_t1, gx_t1, gv_t1, gx_t, gv_t, gE, opts, stream,
                      report);
}

jgs2_status jgs2_mesh_set_youngs(jgs2_mesh* mesh, const double* youngs) {
  return set_youngs(reinterpret_cast<Mesh*>(mesh), youngs);
}

jgs2_status jgs2_mesh_create_batch(const jgs2_mesh_desc* descs, int32_t n_scenes, jgs2_mesh** out) {
  Mesh* m = nullptr;
  jgs2_status s = mesh_create_batch(descs, n_scenes, &m);
  if (out) *out = reinterpret_cast<jgs2_mesh*>(m);
  return s;
}

jgs2_status jgs2_batch_report(const jgs2_mesh* mesh, int32_t* sweeps, int32_t* converged, double* rel_residual) {
  return batch_report(reinterpret_cast<const Mesh*>(mesh), sweeps, converged, rel_residual);
}

jgs2_status jgs2_autotune(jgs2_mesh* mesh, double* x, double* v, const jgs2_step_opts* opts, void* stream,
                          int32_t* block_size) {
  return autotune(reinterpret_cast<Mesh*>(mesh), x, v, opts, stream, block_size);
}

jgs2_status jgs2_mesh_launch_config(const jgs2_mesh* mesh, int32_t precision, int32_t* config) {
  const Mesh* m = reinterpret_cast<const Mesh*>(mesh);
  if (!m || !config) return fail(JGS2_EINVAL, "null argument");
  if (precision != JGS2_FP64 && precision != JGS2_FP32) return fail(JGS2_EINVAL, "bad precision");
  const int pi = precision == JGS2_FP32 ? 1 : 0;
  config[0] = m->gbs[pi];
  config[1] = m->gtpv[pi];
  config[2] = m->bs[pi];
  config[3] = m->cpf[pi];
  return JGS2_OK;
}

void jgs2_mesh_destroy(jgs2_mesh* mesh) { delete reinterpret_cast<Mesh*>(mesh); }

const char* jgs2_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
