// Internal data layout of the JGS2 library (device side and host bookkeeping).
//
// HBM layout (all arrays in the library's internal vertex order: free vertices first,
// sorted along a Morton curve of the rest positions, then pinned vertices):
//   TetRec<T>   one 16-byte aligned record per tet, tets sorted by smallest corner:
//               corner ids, D_m^{-1} (B), F(x_t) (per step), V_e, mu, lam' = lam + mu,
//               rho V_e / 4 (the element's share of each corner's lumped mass).
//   FRec<T>     per tet, rewritten every sweep by the element pass: F_e(x^k), J - 1, mu, lam'.
//   bc          per tet and corner, the corner vector b_a and V_e (Vec4, one 16-byte load).
//   Vec4<T>     per-vertex displacement u = x - x_t (the sweep works in displacement so
//               that FP32 keeps the precision of small per-step motions), the inertia
//               offset dz = z - x_t = h v_t + h^2 g, and the sweep direction D.
//   incidence   sliced-ELL list per 32-vertex slice: entry j of lane l sits at
//               off[slice] + 32 j + l, value = 4*tet + corner (coalesced warp reads).
//   cubature    per free vertex and slot s: pool slot index, weight, and U_bar rows
//               (12x3) as [slot][36][cs] (cs = Vf rounded up to 4) so a warp's loads are
//               coalesced and a block's rows can be bulk-copied.
//   pool        per sweep, one 16-byte aligned row per cubature element: the rotated
//               12x12 element Hessian as its ten 3x3 corner blocks (a, c), a <= c, in row
//               order (90 values), then the 12 rotated gradient entries, 2 pad.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace jgs2 {

constexpr int kSlice = 32;       // vertices per incidence slice (one warp)
constexpr int kMaxCub = 8;       // cubature slots per vertex at most
constexpr int kLsTrials = 8;     // line-search steps alpha = 2^-j, j < kLsTrials
constexpr int kPairTrialBlocks = 148 * 4;  // blocks of the line-search barrier-trial pass (2 x kLsTrials sums each)
constexpr int kEnergyBlocksMax = 148 * 8;  // blocks of the line-search energy pass, at most
constexpr int kMaxVertexPairs = 64;  // active cross-body pairs listed per vertex at most
constexpr int kPoolH = 90;       // 12x12 symmetric as ten 3x3 corner blocks (a <= c)
// Row stride of the per-slot cubature record arrays: Vf rounded up to 4 entries, so that
// every row starts on a 16-byte boundary.
__host__ __device__ constexpr int cub_stride(int Vf) { return ((Vf + 3) / 4) * 4; }
constexpr int kPoolStride = 104;  // pool row: 90 Hessian block entries, 12 gradient entries, 2 pad

template <typename T>
struct alignas(16) TetRec {
  int32_t v[4];
  T B[9];      // B = D_m^{-1}, row-major; corner k>0 uses row k-1, corner 0 minus the sum
  T Ft[9];     // F(x_t), row-major (i, j) -> 3i + j
  T vol, mu, lp, mq;
  T jt1;       // det F(x_t) - 1, formed in FP64 per step (J - 1 without cancellation)
};

template <typename T>
struct alignas(16) Vec4 {
  T x, y, z, w;
};

// Per-sweep element record written by the element pass: F_e(x^k), J - 1 (formed without
// cancellation) and the element's Lame constants, read by the vertex gather (48 bytes in
// FP32: three 16-byte loads). The element volume rides in the corner vectors' fourth entry.
template <typename T>
struct alignas(16) FRec {
  T F[9];
  T jm1, mu, lp;
};

// Device-resident step state (one per mesh), read and written by the sweep kernels.
struct StepState {
  int32_t done;        // set once the step stops (converged / max sweeps / diverged)
  int32_t converged;
  int32_t status;      // 0 ok, else a jgs2_status
  int32_t sweeps;      // sweeps applied when done
  int32_t fallback;    // vertex solves that fell back to the uncorrected step
  int32_t ls_rejects;
  int32_t max_sweeps;
  int32_t k;           // index of the next sweep (read and advanced by finalize_sweep)
  double rel_tol;
  double g0;           // |g(x^0)|
  double r;            // last relative residual
  double slope;        // g^T D of the current sweep
  double slope_j;      // g^T D_J (uncorrected direction)
  double alpha;        // accepted step of the current sweep
  int32_t dir;         // 0: step along D, 1: along D_J
  int32_t need_j;      // every line-search trial along D failed: try D_J
  int32_t dj_steps;    // sweeps that stepped along D_J
  int32_t rebuilds;    // contact candidate-list rebuilds
  int32_t prev_dir;    // direction the last accepted line-search step took (0: D, 1: D_J)
  int32_t ls_mode;     // this sweep's line-search pass: prev_dir as the sweep began
  uint32_t ticket_main;
  uint32_t ticket_energy;
  // position-change stopping test (Sec. 8's |dx| check): |x^k - x^{k-1}|^2 of the last
  // update, the squared tolerance (0: off), and |D|^2, |D_J|^2 of the current sweep
  double dx2;
  double dx2_tol;
  double dd2;
  double ddj2;
  int32_t stopped_dx;  // the step stopped on the position-change test
  int32_t pad_dx;
  double dx2_applied;  // |x^k - x^{k-1}|^2 of the last update applied (for the report)
  int32_t ls_passes[3];  // line-search passes that did work, by pass (D, D_J, both)
  int32_t gs_ncol;       // Gauss-Seidel step: colour passes per GS sweep (0: Jacobi sweeps)
  int32_t pass;          // Gauss-Seidel step: colour passes begun
  int32_t pad_gs;
};

// Contact data of a mesh (Sec. 7); pairs: 0 vertex-wall, 1 vertex-face, 2 edge-edge.
struct ContactView {
  int on = 0;
  int pen = 0;                       // 0: IPC log barrier (Eq. barrier), 1: quadratic penalty
  int n_planes = 0, n_faces = 0, n_edges = 0, n_sverts = 0, n_vertices = 0;
  const double* planes = nullptr;    // [n_planes][4]
  const int32_t* faces = nullptr;    // [n_faces][3] internal vertex ids (outward)
  const int32_t* edges = nullptr;    // [n_edges][2]
  const int32_t* sverts = nullptr;   // [n_sverts]
  const uint8_t* is_surf = nullptr;  // [V]
  double dhat = 0, kappa = 0, rc = 0;
  // broadphase: candidate list of the pairs within R at the last rebuild; rebuild when a
  // surface vertex has moved more than trig since then
  double R = 0, trig = 0;
  int hbits = 0;                 // log2 of the buckets per hashed grid (faces grid, edges grid)
  uint64_t* fkeys = nullptr;     // [n_faces] cell key of the centroid
  uint64_t* ekeys = nullptr;     // [n_edges] cell key of the midpoint
  int32_t* frank = nullptr;      // [n_faces] rank within its bucket
  int32_t* erank = nullptr;      // [n_edges]
  int32_t* hcnt = nullptr;       // [2H + 1] bucket counts, then exclusive starts
  int32_t* hblk = nullptr;       // [scan blocks] block sums
  int32_t* hids = nullptr;       // [n_faces + n_edges] primitive ids in bucket order
  float4* hrec = nullptr;        // [n_faces + n_edges] bucket order: FP32 centre (centroid / midpoint), pad
  uint64_t* hkey = nullptr;      // [n_faces + n_edges] bucket order: cell key
  float4* pbp = nullptr;         // [V] surface vertex positions at the last rebuild (FP32)
  uint32_t* ctl = nullptr;       // control words (displacement, rebuild flags, extents)
  // pairs
  uint64_t* pairs = nullptr;     // packed (kind << 60 | a << 30 | b)
  int32_t* n_pairs = nullptr;    // device counter
  int cap = 0;
  float* dbp = nullptr;          // [cap] distance at the last rebuild (rounded down)
  double* d0 = nullptr;          // [cap] distance at x^k (inf when provably beyond r_c)
  float* pmarg = nullptr;        // [cap] margin beyond r_c at the pair's last motion check
                                 // (rounded down; < 0: check again at every sweep)
  float* ppath = nullptr;        // [cap] path bound (kCtlPath) when that margin was taken
  // per-vertex accumulators
  double* bg = nullptr;          // [3][V]
  double* bH = nullptr;          // [6][V]
  double* dmin = nullptr;        // [V] smallest distance of a pair within r_c (atomicMin on the bits)
  double* lim = nullptr;         // [Vf] step limit 0.45 min(rc - dhat, dmin)
  int32_t* flags = nullptr;      // [0] overflow, [1] intersection, [2] pair-list overflow
  // contact-aware coupling (Sec. 7): per vertex, its active (d < dhat) pairs that reach
  // another body (vp_cnt, vp [V][kMaxVertexPairs]); body id per vertex
  const int32_t* body = nullptr;  // [V]
  int32_t* vp_cnt = nullptr;      // [V]
  int32_t* vp = nullptr;          // [V][kMaxVertexPairs]
  // friction on the walls (lagged at the step start): coefficient, smoothing slip
  // eps_v h, and the lagged normal force of each (wall, vertex) [n_planes][V] (null: off)
  double fmu = 0, feps = 0;
  double* fr_lam = nullptr;
};

// Per-scene state of a batch mesh (one slot per scene; a single mesh is not batched).
struct SceneState {
  int32_t done, converged, status, sweeps, k, fallback, ls_rejects, dir;
  int32_t need_j;    // every line-search trial along D failed: try D_J
  int32_t prev_dir;  // direction the scene's last accepted line-search step took (0: D, 1: D_J)
  int32_t ls_mode;   // this sweep's line-search pass: prev_dir as the sweep began
  int32_t pad;
  double g0, r, slope, slope_j, alpha;
};
constexpr int kSceneAcc = 16;  // per-scene FP64 sums: |g|^2, g.D_J, g.D, 6 line-search coefficients

template <typename T>
struct DevMesh {
  int V, Vf, T_, n_slices, nP, n_cub;
  const TetRec<T>* tets;
  TetRec<T>* tets_mut;
  FRec<T>* frec;            // [T] F_e(x^k) of the current sweep (element pass)
  Vec4<T>* bc;              // [T][4] corner vectors b_a = rows of D_m^{-1}, b_0 = -(b_1+b_2+b_3); w = V_e
  const int32_t* inc_off;   // [n_slices + 1]
  const int32_t* inc_len;   // [Vf]
  const int32_t* inc;       // entries
  Vec4<T>* u;               // [V]
  Vec4<T>* dz;              // [Vf]
  Vec4<T>* D;               // [Vf] JGS2 direction
  Vec4<T>* DJ;              // [Vf] uncorrected direction -H_ii^{-1} g_i
  const uint8_t* vmask;     // [Vf] or null: vertices that move in this sweep (a Gauss-Seidel
                            // colour); the others get D = D_J = 0
  T* cpl;                   // [9][Vf] or null: contact-aware local terms g' (3), H' (6) that
                            // replace g_i, H_ii in the corrected local system where cpl_on
  uint8_t* cpl_on;          // [Vf]
  T* ghr;                   // [18][Vf] g_i, H_ii (6), R_i (9) between the two sweep phases
  const T* mh2;             // [V] m_v / h^2 (0 for pinned)
  int cs;                   // row stride of the cubature records: Vf rounded up to 4
  const int32_t* cub_p;     // [n_cub][cs] pool slot, -1 unused
  const T* cub_w;           // [n_cub][cs]
  const T* cub_u;           // [n_cub][36][cs]
  const int32_t* pool_tet;  // [nP]
  T* pool_H;                // [nP][104] rotated Hessian blocks (90), rotated gradient (12), pad
  T* pool_G;                // [nP][12]
  T* pool_R;                // [nP][4][9] corner rotations of the last pool pass
  double* xt;               // [V][3]
  double* vt;               // [V][3]
  const int32_t* perm;      // internal -> caller
  ContactView c;            // IPC barrier data (c.on = 0: no contact)
  int n_scenes;             // batch meshes: scenes, vertex/tet scene ids, per-scene state
  const int32_t* v_scene;   // [Vf]
  const int32_t* t_scene;   // [T]
  SceneState* scenes;       // [n_scenes]
  double* sacc;             // [n_scenes][kSceneAcc]
  int32_t* n_done;          // scenes finished in this step
  double inv_h2;            // 1/h^2
  double h;
  double grav[3];
};

}  // namespace jgs2
