// lbm_step_gnn_noalloc: the GNN-LBM step for callers that cannot allocate
// device memory.
//
// lbm_step_gnn needs 512 bytes of scratch per node, which its caller passes
// in.  Some callers cannot provide that: a host application whose own
// allocator owns all device memory and forbids other allocations after
// start-up, a real-time loop that may not allocate once running, or a
// language binding that has no way to hand out a device buffer.  This entry
// point takes its scratch from a fixed array in the library's own device
// memory instead, so the caller passes only inputs and outputs.
//
// The array is a file-scope __device__ variable of NOALLOC_BYTES (16 MiB),
// enough for NOALLOC_MAX_NODES = 32,768 nodes per call.  Every GPU on which
// the library's device code is loaded holds it until the process exits.  In
// host code the array's name is only a host-side stand-in, so its device
// address is looked up with cudaGetSymbolAddress, once per device, with that
// device current; the first call on each device does this set-up (so make
// that first call before any stream capture).  Nothing is allocated: no
// cudaMalloc, cudaFree or allocating library routine is called.
//
// All calls share the one array and it keeps the previous call's contents.
// Nothing in it needs to start at zero (every value the kernels read from it
// was written earlier in the same call), but calls that overlap on the GPU
// (on different streams, or from several host threads) race on it.
#include <atomic>
#include <cmath>

#include "common.cuh"
#include "trace.h"

namespace {

constexpr int64_t NOALLOC_MAX_NODES = LBM_STEP_GNN_NOALLOC_MAX_NODES;
constexpr size_t NOALLOC_BYTES = (size_t)NOALLOC_MAX_NODES * 512;

static __device__ __align__(256) unsigned char g_gnn_step_scratch[NOALLOC_BYTES];

// Device address of the scratch array on the current device (set-up on the
// first use per device); nullptr if the lookup failed.  The per-device cache
// is atomic: host threads whose first calls race each look the address up
// and store the same value.
void* scratch_address() {
  static std::atomic<void*> addr[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  void* a = addr[dev].load(std::memory_order_acquire);
  if (!a) {
    if (cudaGetSymbolAddress(&a, g_gnn_step_scratch) != cudaSuccess) return nullptr;
    addr[dev].store(a, std::memory_order_release);
  }
  return a;
}

}  // namespace

extern "C" {

int lbm_step_gnn_noalloc(const float* f_in, float* f_out, lbm_shape s, float tau,
                         const float* taus, const void* packed, double* totals, void* stream) {
  LBM_TRACE("lbm_step_gnn_noalloc");
  if (s.nx < 1 || s.ny < 1 || s.nb < 1) return LBM_ERR_SIZE;
  const int64_t n = (int64_t)s.nx * s.ny * s.nb;
  if (n > NOALLOC_MAX_NODES) return LBM_ERR_SIZE;
  void* scratch = scratch_address();
  if (!scratch) return LBM_ERR_CUDA;
  return lbm_step_gnn(f_in, f_out, s, tau, taus, packed, totals, scratch, NOALLOC_BYTES, stream);
}

}  // extern "C"
