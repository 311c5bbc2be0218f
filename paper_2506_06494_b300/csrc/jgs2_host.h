// Host-side mesh object of the JGS2 library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/jgs2.h"
#include "jgs2_internal.h"

namespace jgs2 {

template <typename T>
struct PrecBufs {
  bool ready = false;
  int cub_version = -1;
  TetRec<T>* tets = nullptr;
  FRec<T>* frec = nullptr;
  Vec4<T>* bc = nullptr;
  Vec4<T>* u = nullptr;
  Vec4<T>* dz = nullptr;
  Vec4<T>* D = nullptr;
  Vec4<T>* DJ = nullptr;
  T* ghr = nullptr;
  T* mh2 = nullptr;
  int32_t* cub_p = nullptr;
  T* cub_w = nullptr;
  T* cub_u = nullptr;
  T* pool_H = nullptr;
  T* pool_G = nullptr;
  T* pool_R = nullptr;
  T* cpl = nullptr;  // [9][Vf] contact-aware local terms (allocated when first used)
  // adjoint workspace
  Vec4<T>*a_lam = nullptr, *a_r = nullptr, *a_z = nullptr, *a_p = nullptr, *a_q = nullptr;
  T* a_lin = nullptr;
  void release();
};

struct Mesh {
  int V = 0, T = 0, Vf = 0, n_slices = 0, n_bodies = 0;
  double h = 0.0;
  double grav[3] = {0, 0, 0};
  double extent = 0.0;             // largest extent of the rest positions' bounding box
  // caller-order inputs and FP64 rest data
  std::vector<double> X, E, nu, rho;
  std::vector<int> tets_c;
  std::vector<uint8_t> pinned;
  std::vector<double> B, vol, mu, lp, mass;
  std::vector<int> body;  // caller vertex -> body id (by smallest caller vertex index)
  // orderings
  std::vector<int> perm, iperm;    // internal <-> caller vertex
  std::vector<int> tperm, tiperm;  // internal <-> caller tet
  std::vector<int> inc_off, inc_len, inc;
  int inc_blk[4] = {0, 0, 0, 0};  // largest incidence range of a 64/128/256/32-vertex block (entries)
  // cubature records, internal order: [Vf][n_cub]
  int n_cub = 0, nP = 0, cub_version = 0, pool_version = -1;
  bool device_ready = false;
  int device = -1;                // CUDA device of the mesh's buffers (set at first allocation)
  std::vector<int> pool;          // internal tet ids of the pool, ascending
  std::vector<int> cub_p, cub_elem;
  std::vector<double> cub_w, cub_u, cub_resid;
  // device
  int32_t *d_inc_off = nullptr, *d_inc_len = nullptr, *d_inc = nullptr, *d_pool_tet = nullptr, *d_perm = nullptr;
  double *d_xt = nullptr, *d_vt = nullptr, *d_partial = nullptr, *d_trace = nullptr;
  double *d_xbuf = nullptr, *d_vbuf = nullptr;
  int32_t* d_tperm = nullptr;    // internal -> caller tet
  double* d_youngs = nullptr;    // caller tet order
  double* d_coup = nullptr;      // [3V] adjoint coupling of pinned vertices
  void* d_adjsc = nullptr;       // AdjScalars
  StepState* d_state = nullptr;
  StepState* h_state = nullptr;
  std::vector<cudaEvent_t> events;  // pooled profiling events
  // batch meshes (several independent scenes in one mesh, each with its own convergence)
  int n_scenes = 0;                   // 0: not a batch mesh
  std::vector<int> vscene;            // caller vertex -> scene
  int32_t *d_vscene = nullptr, *d_tscene = nullptr, *d_ndone = nullptr;
  void* d_gbar = nullptr;             // grid barrier of the persistent batch launch
  SceneState* d_scenes = nullptr;
  double* d_sacc = nullptr;
  // launch shapes per precision (autotuned): k_correct block size, k_gather block size and
  // threads per vertex
  int bs[2] = {128, 128};
  int gbs[2] = {128, 128};
  int gtpv[2] = {1, 1};
  int cpf[2] = {0, 0};     // k_correct: load every slot's pool index and weight first
  // captured sweep chunk of a batch step: key = (precision, correction, line search, bs, chunk)
  cudaGraphExec_t graph = nullptr;
  long graph_key = -1;
  cudaStream_t gstream = nullptr;   // private stream the graph is captured on and replayed on
  cudaStream_t gstream2 = nullptr;  // second branch of a captured sweep (contact, pool)
  cudaEvent_t gev[2] = {nullptr, nullptr};
  cudaEvent_t gfork[4] = {nullptr, nullptr, nullptr, nullptr};
  // single-scene steps: the device view the chunk was captured with (re-captured when a
  // device buffer moves) and its kernel groups in launch order, each with the number of
  // kernels and, when profiling, the pair of external timing events recorded around it
  struct GraphGroup {
    int kind, n;
    cudaEvent_t e0, e1;
  };
  std::vector<char> gdev;
  std::vector<GraphGroup> ggroups;
  std::vector<cudaEvent_t> gevents;
  // contact (Sec. 7): surface in internal vertex ids
  int contact = 0;
  int penalty = 0;                            // 1: quadratic penalty instead of the IPC barrier
  double dhat = 0.0, kappa = 0.0, rc = 0.0;
  double fmu = 0.0, feps_v = 0.0;             // wall friction coefficient and smoothing slip speed
  double* d_fr_lam = nullptr;                 // [n_planes][V] lagged normal forces (friction on)
  double bp_R = 0.0, bp_trig = 0.0;           // candidate-list radius and rebuild trigger
  int hbits = 0;                              // log2 buckets per hashed grid
  std::vector<double> planes;                 // [n][4]
  std::vector<int> sfaces, sedges, sverts;    // [nF][3], [nE][2], [nS]
  std::vector<uint8_t> is_surf;               // [V] internal order
  int pair_cap = 0;
  double *d_planes = nullptr, *d_d0 = nullptr, *d_bg = nullptr, *d_bH = nullptr;
  int32_t *d_faces = nullptr, *d_edges = nullptr, *d_sverts = nullptr, *d_npairs = nullptr, *d_cflags = nullptr;
  int32_t *d_frank = nullptr, *d_erank = nullptr, *d_hcnt = nullptr, *d_hblk = nullptr, *d_hids = nullptr;
  float4* d_hrec = nullptr;
  uint64_t* d_hkey = nullptr;
  uint8_t* d_is_surf = nullptr;
  uint64_t *d_fkeys = nullptr, *d_ekeys = nullptr, *d_pairs = nullptr;
  float4* d_pbp = nullptr;
  float* d_dbp = nullptr;
  float *d_pmarg = nullptr, *d_ppath = nullptr;
  // Gauss-Seidel step: per-colour masks [ncol][Vf], the active mask, scratch states
  uint8_t *d_gsmask = nullptr, *d_vmask = nullptr;
  int gs_ncol = 0;
  bool vmask_on = false;
  double *d_gs_xt = nullptr, *d_gs_xk = nullptr, *d_gs_g = nullptr;
  uint32_t* d_ctl = nullptr;
  double *d_dmin = nullptr, *d_lim = nullptr;
  int32_t *d_body = nullptr, *d_vp_cnt = nullptr, *d_vp = nullptr;  // contact-aware coupling
  uint8_t* d_cpl_on = nullptr;
  PrecBufs<float> f32;
  PrecBufs<double> f64;
  ~Mesh();
};

jgs2_status fail(jgs2_status s, const std::string& msg);
jgs2_status precompute(Mesh* m, const jgs2_precompute_opts* o);
jgs2_status set_youngs(Mesh* m, const double* youngs);
// FP64 device view if the mesh's device buffers already exist (never allocates).
bool dev_view_f64_if_ready(Mesh* m, DevMesh<double>* out);
jgs2_status set_cubature(Mesh* m, int n_cub, const std::vector<int>& elem_int, const std::vector<double>& w,
                         const std::vector<double>& u);

}  // namespace jgs2
