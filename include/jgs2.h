/*
 * jgs2.h - C ABI of the B300 JGS2 library: the per-vertex parallel Jacobi sweep with the
 * precomputed, co-rotated, cubature-sampled overshoot correction of
 * Lan et al., "JGS2: Near Second-order Converging Jacobi/Gauss-Seidel for GPU
 * Elastodynamics" (ACM TOG).
 *
 * Problem statement (Sec. 3, Eq. 1): each implicit-Euler time step minimises
 *     E(x) = sum_v m_v/(2h^2) |x_v - z_v|^2 + sum_e V_e Psi(F_e),
 *     z = x_t + h v_t + h^2 g,
 * over the free vertices, where Psi is the stable Neo-Hookean energy (Table 1 caption)
 *     Psi(F) = mu/2 (tr F^T F - 3) - mu (J - 1) + (lam + mu)/2 (J - 1)^2.
 * After the step, v_{t+1} = (x_{t+1} - x_t)/h.
 *
 * Conventions shared by every entry point
 *  - Every call returns a jgs2_status; nothing aborts, traps or exits. On failure the
 *    thread-local message of jgs2_last_error() says why.
 *  - Host arrays passed in are read during the call only and copied; the caller keeps
 *    ownership. Device state arrays (x, v) are caller-owned and must stay valid for the
 *    duration of the call; the library never frees them.
 *  - Vertex arrays are [V][3] row-major in the caller's vertex order; the library
 *    reorders internally and writes back in the caller's order.
 *  - A jgs2_mesh is not thread-safe: calls on one mesh must be serialised by the caller.
 *    Different meshes may be used from different threads.
 */
#ifndef JGS2_H
#define JGS2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  JGS2_OK = 0,
  JGS2_EINVAL = 1,           /* bad argument (null pointer, size, index out of range) */
  JGS2_ENOMEM = 2,           /* host or device allocation failed */
  JGS2_ECUDA = 3,            /* a CUDA runtime call failed */
  JGS2_ENOTPRECOMPUTED = 4,  /* jgs2_step with the correction on before a precompute */
  JGS2_ENOTCONVERGED = 5,    /* max_sweeps reached; state is updated, report is filled */
  JGS2_EDIVERGED = 6,        /* the residual became NaN/Inf; state is NOT written back */
  JGS2_ENONSPD = 7,          /* jgs2_step_adjoint: the Hessian at x* is not positive definite
                              * along a conjugate-gradient search direction */
  JGS2_ETIMEOUT = 8,         /* a bounded device wait (bulk-copy barrier) gave up; state NOT written */
  JGS2_EINTERSECT = 9        /* contact: a surface pair reached zero distance at a sweep's positions;
                              * state NOT written. jgs2_cloth_create: a free rest vertex on or
                              * behind a wall */
} jgs2_status;

/* Mesh description (Sec. 3). All pointers are host pointers, copied at create. */
typedef struct {
  int32_t n_vertices;        /* V > 0 */
  int32_t n_tets;            /* T > 0 */
  const double* rest_pos;    /* [V][3] rest positions X (m) */
  const int32_t* tets;       /* [T][4] vertex indices; every tet must have positive volume */
  const double* youngs;      /* [T] Young's modulus E (Pa) */
  const double* poisson;     /* [T] Poisson ratio nu, in (-1, 0.5) */
  const double* density;     /* [T] density rho (kg/m^3) */
  const uint8_t* pinned;     /* [V] 1 = vertex held at its position x_t (not a DOF); may be NULL */
  double gravity[3];         /* f_ext / m (m/s^2) */
  double dt;                 /* time step h (s) > 0 */
  /* Contact (Sec. 7). contact = 1: the IPC log barrier kappa B(d) of Eq. barrier; 2: the
   * implicit quadratic penalty kappa (dhat - d)^2 / 2 for d < dhat (the other contact form the
   * paper's Table 1 uses); 0 disables contact and the other fields are then ignored. Pairs:
   * surface vertex - boundary face, boundary edge - boundary edge (self-contact included) and
   * surface vertex - wall plane n.x >= c; both forms keep the per-vertex step limit. */
  int32_t contact;
  int32_t n_planes;          /* walls */
  const double* planes;      /* [n_planes][4]: unit normal n (3) and finite offset c (JGS2_EINVAL
                              * otherwise); may be NULL if 0 */
  double dhat;               /* barrier support d^ (m) > 0 */
  double kappa;              /* barrier or penalty stiffness (N/m) > 0 */
  /* Friction on the walls (IPC's lagged friction potential; the paper's friction scenes).
   * friction_mu >= 0 is the coefficient (0 = none; > 0 needs contact != 0); friction_eps_v
   * > 0 the slip speed (m/s) below which friction is smoothed (slip eps = eps_v dt). At the
   * start of every step, each free surface vertex v within dhat of wall p gets the lagged
   * normal force lam = -kappa E'(d_vp(x_t)) (E the barrier or the penalty), and the step's
   * energy adds mu lam f0(|P_p (x_v - x_t,v)|) per such pair, P_p = I - n n^T and
   * f0(y) = -y^3/(3 eps^2) + y^2/eps + eps/3 below eps, y beyond. Vertex-face and edge-edge
   * pairs carry no friction. Zero-initialised descriptions get no friction. */
  double friction_mu;
  double friction_eps_v;
} jgs2_mesh_desc;

typedef struct jgs2_mesh jgs2_mesh; /* opaque, library-owned */

/* Precompute options (Secs. 5-6). */
typedef struct {
  int32_t n_cub;       /* cubature elements per vertex |S_i| (Table 1: 4 or 6); <= 8 */
  int32_t n_train;     /* training poses: lowest eigenvectors of H_bar (Sec. 5) */
  int32_t n_cand;      /* candidates drawn per greedy round (Sec. 5) */
  int32_t n_pool;      /* per-body element pool the candidates come from */
  double nnls_tol;     /* stop when the relative NNLS residual is below this (Sec. 5: 1%) */
  uint64_t seed;       /* SplitMix64 seed of the pool / candidate draws */
  int32_t n_threads;   /* host threads (0 = all cores) */
  int32_t gs;          /* 1 = Gauss-Seidel groups (Sec. 8.1): free vertices greedily coloured in
                        * caller order, each colour a generalised sub-problem whose U_bar_i
                        * keeps the group's other DOFs fixed (one factorisation per colour).
                        * The records suit a sweep that runs the colours in turn; jgs2_step
                        * runs the Jacobi sweep (0, the default) */
  int32_t gpu;         /* 1 = the multi-RHS solves of the training poses and of the pool rows
                        * of H_bar^{-1} run on the current CUDA device (FP32 substitutions with
                        * the factor, refined in FP64 against H_bar to a relative residual of
                        * 1e-14; a body whose refinement stalls above 1e-10, kappa(H_bar) being
                        * too large for FP32, takes the host's FP64 substitutions); 0 = host FP64
                        * substitutions. Factorisation, selected inversion and NNLS stay on
                        * the host either way. Gauss-Seidel groups (gs = 1) solve on the host,
                        * and so do small bodies run side by side (see jgs2_precompute) */
} jgs2_precompute_opts;

/* Cubature records produced elsewhere (e.g. by an independent implementation), in the
 * caller's vertex order. Slot s of vertex i: element elem[i*n_cub+s] (caller tet index,
 * -1 = unused slot), weight w[i*n_cub+s] >= 0, and the rows of U_bar_i at the element's
 * four corners ubar[((i*n_cub+s)*4+a)*9 + 3*r + c] = (U_bar_{i,a})_{rc} (Eq. u, Sec. 6).
 * Records of pinned vertices are ignored. */
typedef struct {
  int32_t n_cub;
  const int32_t* elem;       /* [V][n_cub] */
  const double* weight;      /* [V][n_cub] */
  const double* ubar;        /* [V][n_cub][4][3][3] */
} jgs2_cubature_blob;

typedef enum { JGS2_FP64 = 0, JGS2_FP32 = 1 } jgs2_precision;
typedef enum { JGS2_CORR_ASM = 0, JGS2_CORR_ELEM = 1, JGS2_CORR_OFF = 2 } jgs2_correction;

typedef struct {
  int32_t max_sweeps;        /* sweeps per step at most (>= 0) */
  double rel_tol;            /* stop at |g(x^k)| <= rel_tol |g(x^0)| over free DOFs */
  int32_t precision;         /* jgs2_precision: sweep arithmetic; reductions are FP64 */
  int32_t correction;        /* jgs2_correction: gradient reading of Eq. cubature, or off */
  int32_t line_search;       /* 1 = global Armijo backtracking on E (FP64 energy sums) */
  int32_t check_every;       /* host reads the convergence flag every this many sweeps */
  int32_t record_trace;      /* 1 = keep the per-sweep residual trace in the report */
  int32_t profile;           /* 1 = time the kernels with CUDA events: the per-step kernels, and
                              * every kernel group of the last sweep of each replayed chunk
                              * of check_every sweeps (a sample, so the events barely slow the
                              * step) */
  double dx_tol;             /* > 0: also stop at the first sweep k >= 1 whose last update moved
                              * the free vertices by |x^k - x^{k-1}|_2 <= dx_tol * length_scale
                              * (2-norm over all free DOFs): Sec. 8's convergence check on a scene
                              * normalised to a unit cube. 0 = off (the default). Single scenes
                              * only (JGS2_EINVAL on a batch mesh); jgs2_step_gs ignores it */
  double length_scale;       /* L of that normalisation (m); <= 0: the largest extent of the
                              * bounding box of the rest positions */
  int32_t persistent;        /* batch meshes: 1 = each chunk of check_every sweeps is one
                              * persistent cooperative launch over all scenes' tet and vertex
                              * tiles, its phases separated by a bounded grid barrier (captured in
                              * a CUDA graph); 0 = one launch per kernel (the default). Single
                              * scenes ignore it */
  int32_t wait_polls;        /* polls of one bounded device wait before it gives up with
                              * JGS2_ETIMEOUT; 0 = the default (2^20, about 0.2 s) */
  int32_t test_unreachable_barrier; /* test hook, 0 in use: 1 makes the persistent launch's first
                              * grid barrier wait for one block more than the grid has, so the wait
                              * runs out after wait_polls polls and the step returns JGS2_ETIMEOUT
                              * with the state not written */
  int32_t contact_coupling;  /* 1 = contact-aware correction (Sec. 7): a vertex with active contact
                              * pairs reaching another body solves its local system as if the
                              * colliding free vertices of that body moved with it (their elastic
                              * and inertial gradient and diagonal block added; each of its pairs'
                              * terms taken along the co-moving set, so a pair that moves rigidly
                              * drops out). Needs contact and the correction on; 0 = off (default).
                              * JGS2_ENOMEM if a vertex has more than 16 such pairs */
} jgs2_step_opts;

#define JGS2_TRACE_MAX 4096
/* kernel kinds in jgs2_step_report.kernel_*: pool (cubature elements), gather (per-vertex
 * gradient, diagonal block, rotation), correct (cubature correction + 3x3 solve), energy
 * (the line search's energy-change pass over tets and vertices), update, setup (per-step
 * setup and write-back), contact (broadphase, narrowphase and barrier terms), elem (per-tet
 * deformation gradients of the sweep), ls_pairs (the line search's barrier trials) and
 * ls_decide (the line search's one-block decision). kernel_launches counts kernels; a pass
 * of several launches (contact: 11) counts each. The line search launches every pass
 * variant each sweep, and only the variants the sweep needs do work (ls_passes). */
#define JGS2_NKERNELS 11
enum { JGS2_K_POOL = 0, JGS2_K_GATHER = 1, JGS2_K_CORRECT = 2, JGS2_K_ENERGY = 3, JGS2_K_UPDATE = 4,
       JGS2_K_SETUP = 5, JGS2_K_CONTACT = 6, JGS2_K_ELEM = 7, JGS2_K_LS_PAIRS = 8, JGS2_K_LS_DECIDE = 9,
       JGS2_K_PERSISTENT = 10 /* a persistent batch launch (a chunk of whole sweeps) */ };

typedef struct {
  int32_t sweeps;            /* sweeps applied in the step */
  int32_t converged;         /* 1 if rel_tol was reached */
  int32_t fallback;          /* vertex solves that fell back to the uncorrected step */
  int32_t ls_rejects;        /* sweeps where no line-search step satisfied Armijo */
  int32_t dj_steps;          /* sweeps that stepped along the uncorrected direction D_J */
  int32_t contact_rebuilds;  /* contact candidate-list rebuilds in the step (forced one included) */
  int32_t contact_candidates; /* pairs in the candidate list at the end of the step */
  int32_t contact_near;       /* candidate pairs within r_c at the step's last sweep */
  double rel_residual;       /* |g(x_{t+1})| / |g(x_t)| */
  double g0;                 /* |g(x^0)| */
  double ms;                 /* wall time of the step on the stream (CUDA events) */
  int32_t launches;          /* kernels launched by the step */
  int32_t profiled_sweeps;   /* sweeps whose kernel groups were timed (profile = 1): one per
                              * replayed chunk whose last sweep ran before the step stopped */
  int32_t kernel_launches[JGS2_NKERNELS]; /* per kernel kind */
  double kernel_ms[JGS2_NKERNELS];        /* summed CUDA-event time per kind (profile = 1): per-step
                                           * kernels in full, sweep kernels over the profiled sweeps */
  int32_t trace_len;
  double trace[JGS2_TRACE_MAX]; /* r_k per sweep if record_trace */
  int32_t stopped_dx;        /* 1 if the step stopped on the position-change test (dx_tol) */
  int32_t pad_;
  double last_dx;            /* |x^k - x^{k-1}|_2 / L of the step's last update (0 if no sweep) */
  int32_t ls_passes[3];      /* line-search passes that did work: [0] along D, [1] along D_J after
                              * every D trial failed, [2] both directions in one pass (after a
                              * sweep that stepped along D_J) */
  int32_t pad2_;
} jgs2_step_report;

/* Default option values (n_cub 4, n_train 20, n_cand 32, n_pool 256, tol 0.01, seed 0, gs 0). */
void jgs2_precompute_opts_default(jgs2_precompute_opts* o);
/* Defaults: max_sweeps 500, rel_tol 1e-4, FP32, asm, line search on, check_every 16, no
 * position-change test (dx_tol 0, length_scale 0), per-kernel launches (persistent 0),
 * wait_polls 0 (2^20), no test hook. */
void jgs2_step_opts_default(jgs2_step_opts* o);

/* Validates the mesh (indices in range, positive volumes, material ranges, every free
 * vertex in some tet; JGS2_EINVAL otherwise, before any device allocation), computes the
 * rest-shape data in FP64 on the host (D_m^{-1}, V_e, lumped masses m_v = sum rho V_e/4),
 * reorders vertices (free first, spatially sorted) and tets, builds the incidence lists
 * and uploads everything to the current CUDA device. *out receives a new mesh. */
jgs2_status jgs2_mesh_create(const jgs2_mesh_desc* desc, jgs2_mesh** out);

/* Batch of independent scenes in one mesh (several small solids stepped together, each
 * with its own stopping test). descs: n_scenes descriptions (host; contact must be 0, dt
 * and gravity equal in all). The batch's caller vertex / tet order is the concatenation of
 * the scenes' orders. jgs2_step then sweeps every scene in the same kernel launches and
 * stops each scene at its own r_k <= rel_tol (or max_sweeps); the report gives the
 * maximum sweeps and residual over the scenes and converged = 1 only if all converged.
 * The chunk of check_every sweeps is captured once in a CUDA graph and replayed. */
jgs2_status jgs2_mesh_create_batch(const jgs2_mesh_desc* descs, int32_t n_scenes, jgs2_mesh** out);
/* Per-scene results of the last jgs2_step on a batch mesh (host arrays [n_scenes], each
 * may be NULL). */
jgs2_status jgs2_batch_report(const jgs2_mesh* mesh, int32_t* sweeps, int32_t* converged,
                              double* rel_residual);
/* Launch-shape autotuner: on the state (x, v: device [V][3] double, read only) times the
 * gather kernel in each of its shapes (threads per block x threads per vertex: 64, 128,
 * 256 x 1 and 128, 256 x 4; with 4 threads per vertex the incidences of a vertex are split
 * over the lanes of its group) and the correction kernel at 64, 128 and 256 threads per
 * block with and without loading every slot's index first, and keeps the fastest of each
 * for opts->precision. *block_size (may be NULL)
 * receives the correction kernel's choice; jgs2_mesh_launch_config gives all three. */
jgs2_status jgs2_autotune(jgs2_mesh* mesh, double* x, double* v, const jgs2_step_opts* opts,
                          void* stream, int32_t* block_size);
/* The mesh's launch shapes for precision: config[0] gather threads per block, config[1]
 * gather threads per vertex, config[2] correction threads per block, config[3] 1 if the
 * correction kernel loads every cubature slot's index and weight before the first slot's
 * work (host int32_t[4]). */
jgs2_status jgs2_mesh_launch_config(const jgs2_mesh* mesh, int32_t precision, int32_t* config);

/* Offline stage (Secs. 5-6), FP64 results: factorises the rest Hessian H_bar = M/h^2 + K_bar
 * of each distinct body once, computes A_i = (H_bar^{-1})_ii and the rows of
 * U_bar_i = H_bar^{-1} S_i^T A_i^{-1} (Eq. u) that the cubature needs, the lowest
 * eigenvectors of H_bar as training poses, and the greedy NNLS cubature sets
 * (Eq. cubature_weight), then uploads the packed per-vertex records. The factorisation,
 * selected inversion and NNLS run on the host on opts->n_threads OpenMP threads (0 = all
 * cores, the OpenMP default; the caller's setting is restored on return); the multi-RHS solves run
 * there too, or on the current device with opts->gpu = 1. A mesh with several bodies under
 * 20,000 vertices (a batch of small scenes) runs those side by side on the host, one thread
 * each and with host solves whatever opts->gpu says; the larger bodies, and a lone small
 * one, run one at a time. Synchronous; the mesh must not be stepped concurrently. */
jgs2_status jgs2_precompute(jgs2_mesh* mesh, const jgs2_precompute_opts* opts);

/* Loads cubature records computed elsewhere instead of running jgs2_precompute. */
jgs2_status jgs2_precompute_import(jgs2_mesh* mesh, const jgs2_cubature_blob* blob);

/* Copies the library's cubature records back out in the caller's vertex order: arrays
 * sized as in jgs2_cubature_blob (n_cub from the precompute). Host pointers. */
jgs2_status jgs2_precompute_export(const jgs2_mesh* mesh, int32_t* elem, double* weight,
                                   double* ubar, double* residual /* [V], may be NULL */);
int32_t jgs2_mesh_n_cub(const jgs2_mesh* mesh);

/* One time step (Sec. 3) solved by JGS2 sweeps (Secs. 4-5, 8.1) from x^0 = x_t.
 * x, v: caller-owned DEVICE arrays [V][3] of double on the mesh's device, read as
 * (x_t, v_t) and overwritten with (x_{t+1}, v_{t+1}). stream: a cudaStream_t (NULL =
 * default stream); all work is ordered on it and the call returns after the step
 * completed. The sweeps run as replays of a CUDA graph of check_every sweeps on a stream
 * of the mesh, ordered after and before the caller's stream by events; the first step
 * with a new configuration (precision, correction, line search, block size, check_every,
 * profile, trace) captures the graph, so jgs2_step is not itself called inside a stream
 * capture. report may be NULL. Returns JGS2_OK when r_k <= rel_tol or, with dx_tol > 0,
 * when the position-change test stops the step (report->stopped_dx); JGS2_ENOTCONVERGED
 * (state written) when max_sweeps is hit, JGS2_EDIVERGED (state untouched) on a
 * non-finite residual. A mesh
 * without free vertices (every vertex pinned) or with g(x^0) = 0 returns JGS2_OK after 0
 * sweeps with x_{t+1} = x_t (r = 0). */
jgs2_status jgs2_step(jgs2_mesh* mesh, double* x, double* v, const jgs2_step_opts* opts,
                      void* stream, jgs2_step_report* report);

/* The same step by Gauss-Seidel sweeps (Sec. 8.1): the free vertices are coloured greedily
 * in caller order (no two of a colour share a tet); a GS sweep runs the colours in turn,
 * each as one pass of the sweep kernels whose directions and line search move only that
 * colour, at the positions the earlier colours left. The colour passes of check_every GS
 * sweeps are captured in one CUDA graph and replayed like jgs2_step's sweeps. Use it with
 * records from jgs2_precompute(gs = 1) (or import) or with correction = JGS2_CORR_OFF. The
 * relative residual (full gradient, FP64-class sums) is taken at the start of each GS sweep;
 * report->sweeps counts GS sweeps and the trace holds their residuals. x, v: device [V][3]
 * double as in jgs2_step. Meshes with contact or batches return JGS2_EINVAL; dx_tol is
 * ignored. */
jgs2_status jgs2_step_gs(jgs2_mesh* mesh, double* x, double* v, const jgs2_step_opts* opts,
                         void* stream, jgs2_step_report* report);

/* Same step with HOST arrays: copies x, v to the device, steps, copies back. */
jgs2_status jgs2_step_host(jgs2_mesh* mesh, double* x, double* v, const jgs2_step_opts* opts,
                           void* stream, jgs2_step_report* report);

/* Sweep-level entry for parity checks: from the state (x^k = x_t + u, z) runs exactly
 * n_sweeps sweeps without a convergence test. x_t, v_t, x_k: device [V][3] double, caller
 * order; x_k is overwritten with x^{k+n}. */
jgs2_status jgs2_sweeps(jgs2_mesh* mesh, const double* x_t, const double* v_t, double* x_k,
                        int32_t n_sweeps, const jgs2_step_opts* opts, void* stream);

/* Energy E(x) (Eq. 1) and gradient g(x) for the state (x_t, v_t, x): FP64 on the device.
 * g: device [V][3] double (pinned rows 0), may be NULL. */
jgs2_status jgs2_energy_gradient(jgs2_mesh* mesh, const double* x_t, const double* v_t,
                                 const double* x, double* energy, double* g, void* stream);

/* Adjoint of one converged step (the paper has no adjoint; this is the implicit-function
 * theorem applied to Eq. 1's optimality condition grad E(x*; x_t, v_t, E) = 0). For a loss
 * L(x_{t+1}, v_{t+1}) with v_{t+1} = (x_{t+1} - x_t)/h and gbar = dL/dx_{t+1} + dL/dv_{t+1}/h:
 *     H(x*) lam = gbar over free DOFs (H: the exact Hessian of E at x*, no projection)
 *     dL/dx_t = (M/h^2) lam - dL/dv_{t+1}/h  (free),  dL/dx_{t+1} - H_pf lam  (pinned)
 *     dL/dv_t = (M/h) lam  (free), 0 (pinned);  dL/dE_e += -lam_e . g_e^el(x*) / E_e
 * The linear system is solved by flexible conjugate gradients preconditioned with the local
 * solves of the corrected sweep at x* (H_ii + H~_i, H~_i the rotated cubature Hessian of
 * Eq. cubature; symmetric positive definite); correction = JGS2_CORR_OFF gives block-Jacobi
 * preconditioning (H_ii). The sweep's cubature estimate of the residual's reduced part is
 * not applied: it makes the preconditioner indefinite, and conjugate gradients stall.
 * All arrays are DEVICE pointers in caller order: x_t, v_t, x_t1, gx_t1, gv_t1, gx_t, gv_t
 * [V][3] double; gE [T] double is ACCUMULATED (+=). Meshes with contact, or without a
 * free vertex, are rejected (JGS2_EINVAL): the barrier is not part of this adjoint. Returns JGS2_ENOTCONVERGED (all
 * outputs written) if max_iters is reached first. Synchronises the stream. */
typedef struct {
  int32_t max_iters;     /* conjugate-gradient iterations at most */
  double rel_tol;        /* stop at |r| <= rel_tol |gbar| */
  int32_t precision;     /* jgs2_precision of the vectors and kernels; reductions are FP64 */
  int32_t correction;    /* JGS2_CORR_ASM (JGS2 preconditioner) or JGS2_CORR_OFF (block Jacobi) */
  int32_t check_every;   /* host reads the convergence flag every this many iterations */
} jgs2_adjoint_opts;
typedef struct {
  int32_t iters;
  int32_t converged;
  double rel_residual;   /* |H lam - gbar| / |gbar| */
  double ms;
} jgs2_adjoint_report;
/* Defaults: max_iters 5000, rel_tol 1e-6, FP64, block-Jacobi preconditioner (correction
 * JGS2_CORR_OFF; JGS2_CORR_ASM adds the cubature Hessian to each local matrix), check_every 32. */
void jgs2_adjoint_opts_default(jgs2_adjoint_opts* o);
jgs2_status jgs2_step_adjoint(jgs2_mesh* mesh, const double* x_t, const double* v_t, const double* x_t1,
                              const double* gx_t1, const double* gv_t1, double* gx_t, double* gv_t,
                              double* gE, const jgs2_adjoint_opts* opts, void* stream,
                              jgs2_adjoint_report* report);

/* Replaces the per-tet Young's moduli ([T] host, caller order, > 0). mu and lam' follow at
 * the tets' Poisson ratios. The cubature records keep the rest subspace computed for the
 * earlier moduli: under the "asm" reading that changes only the rate, not the result. */
jgs2_status jgs2_mesh_set_youngs(jgs2_mesh* mesh, const double* youngs);

/* Allocation-free variant of jgs2_energy_gradient (the paper has no counterpart; this is a
 * service for callers that cannot allocate device memory while they run, such as a
 * real-time loop that must not wait on cudaMalloc, or a process whose device memory is
 * owned by a pooling allocator). It computes E(x) and g(x) of a mesh without contact and
 * keeps the reduction's partial sums in a file-scope device array of
 * JGS2_STATIC_PARTIALS_MAX + 1 doubles (512 KB, held by every GPU that loads the library
 * until exit); it calls no cudaMalloc, cudaFree or allocating library routine.
 *  - g equals jgs2_energy_gradient's bit for bit. E matches it to rounding: the partial
 *    sums are added on the device in a fixed tree order, not in the allocating entry
 *    point's host order.
 *  - Meshes with contact are rejected (JGS2_EINVAL): the barrier terms need the candidate
 *    list that only the allocating entry point builds.
 *  - Limit: (n_tets + free vertices) / 128 (rounded up each) <= JGS2_STATIC_PARTIALS_MAX,
 *    else JGS2_EINVAL with a message (checked before any device work).
 *  - The mesh's own device buffers must already exist: make one FP64 jgs2_step,
 *    jgs2_sweeps or jgs2_energy_gradient call on the mesh first (else JGS2_EINVAL). The
 *    current CUDA device must be the one those buffers live on (else JGS2_EINVAL).
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) while that device is current.
 *  - Every call shares the array; calls that overlap on the GPU race. Each call writes
 *    every slot it reads, so the array needs no clearing.
 *  - Every call copies E to the host and synchronises the stream before it returns.
 *  - x_t, v_t, x, g: device [V][3] double, caller order (g may be NULL); energy: host
 *    pointer (may be NULL, not both). */
#define JGS2_STATIC_PARTIALS_MAX 65536
jgs2_status jgs2_energy_gradient_static(jgs2_mesh* mesh, const double* x_t, const double* v_t,
                                        const double* x, double* energy, double* g, void* stream);

/* Candidate contact pairs with distance < radius at positions x (device [V][3] double,
 * caller order; x_t likewise), in a canonical order for comparison with independent
 * implementations: rows of 5 int32 (kind, a, b, c, d) in caller vertex ids -
 * kind 0 vertex-wall (v, plane, -1, -1), kind 1 vertex-face (v, face vertices ascending),
 * kind 2 edge-edge (edge 1 ascending, edge 2 ascending; edge 1 < edge 2). out: host
 * [cap][5]; *n_out receives the pair count (rows beyond cap are not written; JGS2_ENOMEM
 * if the count exceeds cap). Requires contact = 1. Synchronises the stream. */
jgs2_status jgs2_contact_pairs(jgs2_mesh* mesh, const double* x_t, const double* x, double radius,
                               int32_t* out, int32_t cap, int32_t* n_out, void* stream);

/* Measured arithmetic peak of the current device's CUDA cores (the paper has no
 * counterpart; it gives the roofline of the ALU-bound kernels a measured denominator):
 * eight independent FMA chains per thread, four 256-thread blocks per SM, best of five
 * timed launches (CUDA events on `stream`). precision: JGS2_FP32 or JGS2_FP64; *gflops
 * receives GFLOP/s (2 per FMA). Allocates a small device buffer; synchronises the stream. */
jgs2_status jgs2_alu_peak(int32_t precision, double* gflops, void* stream);

/* ---------------------------------------------------------------------------------
 * Cloth (the cloth material of the paper's Table 1 caption; reading R26): StVK membrane
 * triangles and a quadratic bending energy on interior edges, stepped by the per-vertex
 * Jacobi sweep with the global Armijo line search. No cubature correction (its records are
 * built on tets); contact with walls only (no self-contact). Vertices keep the caller's order.
 *  - Membrane: per triangle, F = [x_1 - x_0, x_2 - x_0] D_m^-1 (3x2, D_m the rest edges in
 *    the triangle's plane), E = (F^T F - I)/2, energy A (mu tr(E^2) + lam/2 tr(E)^2) with
 *    mu = Y t / (2 (1 + nu)), lam = Y t nu / (1 - nu^2).
 *  - Bending: per interior edge (x_0, x_1) with opposite vertices x_2 (first triangle in
 *    triangle order) and x_3, rest cotangent weights K = (cot a_1 + cot c_1, cot a_0 + cot c_0,
 *    -(cot a_0 + cot a_1), -(cot c_0 + cot c_1)) (a_j: rest angle at x_j in (x_0, x_1, x_2),
 *    c_j: in (x_0, x_1, x_3)); energy (3 k_b / (A_0 + A_1)) |sum_i K_i x_i|^2 / 2.
 *  - Mass rho t A / 3 per corner; inertia and gravity as for the solids (Sec. 3).
 *  - Local system per free vertex: inertia + the positive semidefinite part of the summed
 *    membrane blocks + the bending blocks. */
typedef struct {
  int32_t n_vertices;        /* V > 0 */
  int32_t n_tris;            /* F > 0 */
  const double* rest_pos;    /* [V][3] rest positions (m); also the usual initial state */
  const int32_t* tris;       /* [F][3] vertex indices; every triangle must have positive area */
  double youngs;             /* Y (Pa) > 0 */
  double poisson;            /* nu in (-1, 0.5) */
  double thickness;          /* t (m) > 0 */
  double density;            /* rho (kg/m^3) > 0 */
  double bend;               /* k_b (N m) >= 0 */
  const uint8_t* pinned;     /* [V] 1 = held at x_t; may be NULL */
  double gravity[3];
  double dt;                 /* h (s) > 0 */
  /* Walls n.x >= c (optional): every free vertex against every wall with the IPC barrier
   * kappa B(d) below dhat (Sec. 7), its Gauss-Newton block and the per-vertex step limit
   * 0.45 min(2 dhat - dhat, d_min) of the solids; the line search evaluates the barrier
   * exactly per trial. n_planes = 0: none (the other fields are then ignored). */
  int32_t n_planes;
  const double* planes;      /* [n_planes][4]: unit normal n (3) and offset c */
  double dhat;               /* barrier support (m) > 0 */
  double kappa;              /* barrier stiffness (N/m) > 0 */
} jgs2_cloth_desc;

typedef struct jgs2_cloth jgs2_cloth;

typedef struct {
  int32_t sweeps;            /* sweeps applied */
  int32_t converged;         /* 1 if rel_tol was reached */
  int32_t ls_rejects;        /* sweeps where no trial satisfied Armijo (no move) */
  int32_t pad_;
  double rel_residual;       /* |g(x_{t+1})| / |g(x_t)| over free DOFs */
  double g0;                 /* |g(x_t)| */
} jgs2_cloth_report;

/* Validates the cloth (indices in range, positive areas, material ranges, every free vertex
 * in a triangle, unit wall normals; JGS2_EINVAL otherwise; JGS2_EINTERSECT when a free rest
 * vertex is not strictly on the open side n.x > c of every wall), computes the rest data in
 * FP64 on the host and finds the interior edges. Device memory is taken on the first call that needs it, on
 * the then-current device (later calls must use the same device). */
jgs2_status jgs2_cloth_create(const jgs2_cloth_desc* desc, jgs2_cloth** out);

/* One implicit-Euler step: x, v device [V][3] double (caller order), overwritten with
 * x_{t+1}, v_{t+1} = (x_{t+1} - x_t)/h. With walls, every free vertex of x must be strictly
 * on the open side of every wall (a step keeps it there; the barrier is undefined behind). Uses opts->precision, max_sweeps, rel_tol,
 * line_search and check_every (sweeps between host checks of the stopping test); the
 * other options are ignored. JGS2_ENOTCONVERGED when the cap was reached (state written),
 * JGS2_EDIVERGED if the residual became NaN/Inf. Synchronises the stream. */
jgs2_status jgs2_cloth_step(jgs2_cloth* cloth, double* x, double* v, const jgs2_step_opts* opts, void* stream,
                            jgs2_cloth_report* report);

/* Exactly n sweeps from x (device [V][3] double, overwritten) for the step starting at
 * (x_t, v_t); for parity tests. Synchronises the stream. */
jgs2_status jgs2_cloth_sweeps(jgs2_cloth* cloth, const double* x_t, const double* v_t, double* x, int32_t n,
                              const jgs2_step_opts* opts, void* stream);

/* E(x) and g(x) (FP64) of the step starting at (x_t, v_t): energy host pointer, g device
 * [V][3] (zero rows for pinned vertices); either may be NULL, not both. Synchronises. */
jgs2_status jgs2_cloth_energy_gradient(jgs2_cloth* cloth, const double* x_t, const double* v_t, const double* x,
                                       double* energy, double* g, void* stream);

/* Interior edges (bending hinges) the cloth found at create. */
int32_t jgs2_cloth_n_hinges(const jgs2_cloth* cloth);

void jgs2_cloth_destroy(jgs2_cloth* cloth);

void jgs2_mesh_destroy(jgs2_mesh* mesh);
const char* jgs2_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* JGS2_H */
