// Allocation-free variant of jgs2_energy_gradient.
//
// Some callers cannot call cudaMalloc while they run: a real-time loop that must never
// wait on the driver's allocator (cudaMalloc may synchronise the device and its latency is
// unbounded), or a host process whose device memory was handed to a pooling allocator up
// front so that a direct cudaMalloc can fail. jgs2_energy_gradient keeps its per-block
// partial sums in a buffer the mesh allocates on first use; this variant keeps them in the
// file-scope device array below instead and allocates nothing.
//
// The array is a file-scope __device__ symbol: every GPU that loads the library holds it
// until the process exits, and every call shares it. Its host-side name is only a stand-in
// for the device symbol, so the kernels get the device address obtained once per device
// with cudaGetSymbolAddress (the first call on a device does that set-up while the device
// is current). Each call overwrites every slot it reads, so no clearing is needed; calls
// that overlap on the GPU (on different streams, or from different threads) race on the
// array. Every call copies E to the host and synchronises its stream. Meshes with contact
// are rejected: their barrier terms need the candidate list that only the allocating entry
// point builds.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/jgs2.h"
#include "jgs2_host.h"
#include "jgs2_kernels.cuh"

namespace jgs2 {

// partial sums of the energy reduction: one slot per 128-thread block, plus the result
constexpr int kStaticPartials = JGS2_STATIC_PARTIALS_MAX;
static __device__ __align__(256) double g_static_partials[kStaticPartials + 1];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double* g_static_addr[kMaxDevices] = {nullptr};

// Device address of the static array on the current device (set up once per device).
jgs2_status static_partials(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(JGS2_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(JGS2_EINVAL, "device index out of range for the static scratch table");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_partials);
    if (e != cudaSuccess)
      return fail(JGS2_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_static_addr[dev] = static_cast<double*>(p);
  }
  *out = g_static_addr[dev];
  return JGS2_OK;
}

// Fixed-order sum of n partials into slot n (one block).
__global__ void k_sum_partials(double* p, int n) {
  __shared__ double red[32];
  const double s = block_sum_array(p, n, 1, red);
  if (threadIdx.x == 0) p[n] = s;
}
}  // namespace

jgs2_status energy_gradient_static(Mesh* m, const double* xt, const double* vt, const double* x, double* E,
                                   double* g, void* stream) {
  if (!m || !xt || !vt || !x || (!E && !g)) return fail(JGS2_EINVAL, "null argument");
  // the barrier terms need the contact candidate list, which only the allocating entry
  // point builds: a contact mesh would get a stale barrier gradient and no barrier energy
  if (m->contact) return fail(JGS2_EINVAL, "meshes with contact are not supported by the allocation-free entry");
  const int nbT = (m->T + 127) / 128, nbV = (m->Vf + 127) / 128;
  if (nbT + nbV > kStaticPartials)
    return fail(JGS2_EINVAL, "mesh too large for the static scratch: (n_tets + free vertices) / 128 must be <= " +
                                 std::to_string(kStaticPartials));
  DevMesh<double> d;
  if (!dev_view_f64_if_ready(m, &d))
    return fail(JGS2_EINVAL,
                "mesh device buffers not created yet: make one jgs2_step, jgs2_sweeps or jgs2_energy_gradient "
                "call (FP64) on this mesh first");
  int dev = -1;
  cudaError_t de = cudaGetDevice(&dev);
  if (de != cudaSuccess) return fail(JGS2_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(de));
  if (dev != m->device)
    return fail(JGS2_EINVAL, "the current CUDA device is not the device of the mesh's buffers (device " +
                                 std::to_string(m->device) + ")");
  double* scratch = nullptr;
  jgs2_status st = static_partials(&scratch);
  if (st != JGS2_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (m->V + 127) / 128;
  k_setup_vertices<double><<<nb, 128, 0, s>>>(d, xt, vt, x);
  k_setup_tets<double><<<(m->T + 127) / 128, 128, 0, s>>>(d);
  if (g) k_grad<double><<<nb, 128, 0, s>>>(d, g);
  if (E) {
    k_energy_abs<double><<<nbT + nbV, 128, 0, s>>>(d, scratch, nbT);
    k_sum_partials<<<1, 256, 0, s>>>(scratch, nbT + nbV);
    cudaError_t e = cudaMemcpyAsync(E, scratch + (nbT + nbV), sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return fail(JGS2_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(JGS2_ECUDA, std::string("energy_gradient_static: ") + cudaGetErrorString(e));
  return JGS2_OK;
}

}  // namespace jgs2

extern "C" jgs2_status jgs2_energy_gradient_static(jgs2_mesh* mesh, const double* x_t, const double* v_t,
                                                   const double* x, double* energy, double* g, void* stream) {
  return jgs2::energy_gradient_static(reinterpret_cast<jgs2::Mesh*>(mesh), x_t, v_t, x, energy, g, stream);
}
