// Shared data of the offline stage (Secs. 5-6): the rest Hessian's block columns, its
// supernodal Cholesky factor, and the device solver that runs the factor's multi-RHS
// substitutions on the GPU.
#pragma once
#include <memory>
#include <string>
#include <utility>
#include <vector>

namespace jgs2 {
namespace pre {

// An allocator that leaves new doubles uninitialised, so that the first touch of a large
// buffer happens where its owner writes it (in parallel), not in a serial zero fill.
template <class T>
struct NoInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U>&) {}
  template <class U>
  void construct(U* p) {
    ::new ((void*)p) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new ((void*)p) U(std::forward<A>(a)...);
  }
};
typedef std::vector<double, NoInitAlloc<double>> RawVec;

// Supernodal Cholesky factor H_bar = L L^T of one body (vertex blocks of 3 DOFs).
struct Factor {
  int nv = 0;                                // free vertices of the body (factor order)
  std::vector<int> sn_first;                 // supernode -> first vertex (factor order)
  std::vector<int> sn_of;                    // vertex -> supernode
  std::vector<std::vector<int>> sn_rows;     // supernode -> row structure below (vertices, ascending)
  std::vector<RawVec> L;                     // supernode -> (3nJ + 3nR) x 3nJ column-major
  int nsn() const { return (int)sn_first.size() - 1; }
};

// Lower block of the rest Hessian in factor order: for column vertex v, rows u >= v.
struct BlockCol {
  std::vector<int> row;
  std::vector<double> val;  // 9 per row, row-major 3x3 (row dof of u, col dof of v)
};

// Multi-RHS solves H_bar X = B on the GPU (Sec. 6: every solve reuses the one factor).
// The substitutions run in FP32 over a level schedule of the factor's column panels;
// FP64 iterative refinement against H_bar itself (residual B - H_bar X in FP64 on the
// device) brings each column to the FP64 solve's accuracy.
class GpuSolver;

// Uploads the factor (rounded to FP32) and H_bar (FP64, both triangles) to the current
// device. Returns nullptr with err set when the device cannot take them.
GpuSolver* gpu_solver_create(const Factor& F, const std::vector<BlockCol>& H, std::string& err);

// Solves H_bar X = B in place for B row-major [n][nrhs] (host, factor order, n = 3 nv).
// Refines until every column's residual |B - H_bar X| <= tol |B|, or until a round no
// longer halves the worst column's (at most max_refine rounds). Returns the rounds taken
// if every column ended at or below accept, else -1 with err set (B then holds the last
// iterate).
int gpu_solve_many(GpuSolver* S, double* B, int n, int nrhs, double tol, double accept, int max_refine,
                   std::string& err);

// Block inverse iteration with the block on the device (Sec. 5's training poses): begin
// uploads the start block Q ([n][p] row-major host, p <= 64); solve sets Q <- H_bar^-1 Q
// (as gpu_solve_many); gram copies Q^T Q (with_hq: Q^T H_bar Q) to the host (p x p); rowsolve
// applies Q <- Q L^-T for the host's lower Cholesky factor L (column-major); hmul forms
// H_bar Q; rotate applies Q <- Q V, H_bar Q <- H_bar Q V (V row-major p x p); residuals copies
// |H_bar q_j - lam_j q_j|^2 for j < nt; end downloads Q and frees the block's buffers.
bool gpu_eig_begin(GpuSolver* S, const double* Q, int n, int p, std::string& err);
int gpu_eig_solve(GpuSolver* S, double tol, double accept, int max_refine, std::string& err);
bool gpu_eig_gram(GpuSolver* S, bool with_hq, double* out, std::string& err);
bool gpu_eig_rowsolve(GpuSolver* S, const double* L, std::string& err);
bool gpu_eig_hmul(GpuSolver* S, std::string& err);
bool gpu_eig_rotate(GpuSolver* S, const double* V, std::string& err);
bool gpu_eig_residuals(GpuSolver* S, const double* lam, int nt, double* out, std::string& err);
bool gpu_eig_end(GpuSolver* S, double* Q, std::string& err);

void gpu_solver_destroy(GpuSolver* S);

}  // namespace pre
}  // namespace jgs2
