// Persistent batch sweep: one cooperative launch runs a chunk of sweeps of every scene of a
// batch mesh (several independent solids in one mesh, each with its own stopping test).
//
// The phases of a sweep are the batch kernels' bodies, each over its own tiles in a
// grid-stride loop, separated by a grid barrier:
//   elem (tet tiles) | gather (vertex tiles) | pool, correct (with the correction) |
//   per-scene residual test | per pass of the line search: energy tiles, per-scene choice |
//   update.
// Scenes that have stopped are skipped inside every body (their tiles return at once).
// The launch is cooperative, so every block is resident and the barrier cannot wait on a
// block that never runs. Every barrier wait is bounded: after wait_polls polls without a
// release, the block records JGS2_ETIMEOUT in the step state and returns; every other
// block then gives up at its own next wait, so the launch always ends.
#pragma once
#include "jgs2_kernels.cuh"

namespace jgs2 {

// Grid barrier state in device memory (zeroed before every launch).
struct GridBarrier {
  uint32_t count;  // arrivals at the current barrier
  uint32_t gen;    // barriers completed
  uint32_t extra;  // arrivals that never come: 0 in use; a test sets 1 to make a wait run out
  uint32_t pad;
};

struct PersistArgs {
  int chunk;                 // sweeps per launch
  int nbT, nbG, nbP, nbC;    // tiles: tets (128), gather blocks, pool blocks, correct blocks
  int nbV, nbS;              // vertex tiles (128), scene tiles (128)
  int corr, ls;
  int max_sweeps;
  double rel_tol;
  long long wait_polls;      // polls of one barrier wait at most
  GridBarrier* bar;
  StepState* st;             // status (JGS2_ETIMEOUT) of a wait that gave up
  double* partial;
};

// Bounded grid barrier (all threads of every block call it). Thread 0 of each block arrives;
// the last arrival resets the count and releases the others by advancing the generation.
// Returns false (in every thread of the block) when the wait gave up or another block had.
__device__ __forceinline__ bool grid_barrier(const PersistArgs& a) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    GridBarrier* b = a.bar;
    volatile uint32_t* vgen = &b->gen;
    const uint32_t g = *vgen;
    __threadfence();
    const uint32_t expected = gridDim.x + b->extra;
    const uint32_t arrived = atomicAdd(&b->count, 1u) + 1u;
    int ok = 1;
    if (arrived == expected) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      long long polls = 0;
      while (*vgen == g) {
        if (++polls > a.wait_polls) {
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    if (!ok) {
      a.st->status = 8;  // JGS2_ETIMEOUT
      a.st->done = 1;
    }
    if (*(volatile int32_t*)&a.st->status == 8) ok = 0;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <typename T, bool CORR, bool LS, int TPV>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 2) k_batch_persistent(DevMesh<T> m, PersistArgs a) {
  __shared__ __align__(16) TetRec<T> srec[128];
  const int stride = gridDim.x;
  for (int q = 0; q < a.chunk; ++q) {
    for (int b = blockIdx.x; b < a.nbT; b += stride) {
      elem_body<T, true>(m, b, a.nbT, srec);
      __syncthreads();
    }
    if (!grid_barrier(a)) return;
    for (int b = blockIdx.x; b < a.nbG; b += stride) {
      gather_body<T, CORR, true, 128, TPV>(m, a.st, a.partial, nullptr, 0, b, a.nbG);
      __syncthreads();
    }
    if (!grid_barrier(a)) return;
    if (CORR) {
      for (int b = blockIdx.x; b < a.nbP; b += stride) {
        pool_body<T, true>(m, b);
        __syncthreads();
      }
      if (!grid_barrier(a)) return;
      for (int b = blockIdx.x; b < a.nbC; b += stride) {
        correct_body<T, true, 128, false>(m, a.st, a.partial, nullptr, 0, b, a.nbC);
        __syncthreads();
      }
      if (!grid_barrier(a)) return;
    }
    for (int b = blockIdx.x; b < a.nbS; b += stride)
      scene_finalize_main_body(m.scenes, m.sacc, m.n_scenes, a.rel_tol, a.max_sweeps, CORR ? 1 : 0, m.n_done,
                               b * 128 + threadIdx.x);
    if (!grid_barrier(a)) return;
    if (LS) {
      // along D; along D_J for the scenes whose trials along D all failed; both after a
      // sweep that stepped along D_J (as the separate launches do)
      for (int b = blockIdx.x; b < a.nbT + a.nbV; b += stride) {
        energy_batch_body<T, 0>(m, a.nbT, b, srec);
        __syncthreads();
      }
      if (!grid_barrier(a)) return;
      for (int b = blockIdx.x; b < a.nbS; b += stride)
        scene_finalize_energy_body<0>(m.scenes, m.sacc, m.n_scenes, CORR ? 1 : 0, b * 128 + threadIdx.x);
      if (!grid_barrier(a)) return;
      if (CORR) {
        for (int b = blockIdx.x; b < a.nbT + a.nbV; b += stride) {
          energy_batch_body<T, 1>(m, a.nbT, b, srec);
          __syncthreads();
        }
        if (!grid_barrier(a)) return;
        for (int b = blockIdx.x; b < a.nbS; b += stride)
          scene_finalize_energy_body<1>(m.scenes, m.sacc, m.n_scenes, 1, b * 128 + threadIdx.x);
        if (!grid_barrier(a)) return;
        for (int b = blockIdx.x; b < a.nbT + a.nbV; b += stride) {
          energy_batch_body<T, 2>(m, a.nbT, b, srec);
          __syncthreads();
        }
        if (!grid_barrier(a)) return;
        for (int b = blockIdx.x; b < a.nbS; b += stride)
          scene_finalize_energy_body<2>(m.scenes, m.sacc, m.n_scenes, 1, b * 128 + threadIdx.x);
        if (!grid_barrier(a)) return;
      }
    }
    for (int b = blockIdx.x; b < a.nbV; b += stride) update_batch_body<T>(m, b * 128 + threadIdx.x);
    if (!grid_barrier(a)) return;
  }
}

}  // namespace jgs2
