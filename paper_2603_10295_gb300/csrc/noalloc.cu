// eph_bands_noalloc: band energies and eigenvectors of H(k) without any device
// allocation by the library.
//
// Who needs it: callers whose device memory belongs to someone else -- a
// framework's caching allocator that has reserved the HBM up front, or an
// embedding application with a fixed memory budget -- and callers that must
// not trigger the device-wide synchronisation cudaMalloc/cudaFree can cause
// (latency-sensitive loops sharing the GPU with other streams).  They pass
// device pointers for every input and output; the intermediate phases
// e^{i k.Re} and the H(k) matrices live in one fixed file-scope device array.
//
// The same three kernels as eph_set_k run here (phases, the H(k) Fourier sum,
// the batched Jacobi eigensolve); only where their scratch lives differs.
#include <cuda_runtime.h>

#include <mutex>

#include "eph.h"
#include "eph_kernels.cuh"

namespace {

// Shared scratch: EPH_NOALLOC_SCRATCH_BYTES of phases and H(k), plus the
// eigensolver's convergence flag.  Every device that loads the library holds
// it until the process exits.  All calls share it: calls that overlap on the
// GPU (different streams, or different host threads on one device) race.
__device__ __align__(256) unsigned char g_noalloc_scratch[EPH_NOALLOC_SCRATCH_BYTES];
__device__ __align__(256) int g_noalloc_status;

constexpr int kMaxDevices = 256;
struct Addr {
  void* ctx = nullptr;  // the CUDA context the addresses belong to
  void* scratch = nullptr;
  int* status = nullptr;
};
Addr g_addr[kMaxDevices];
std::mutex g_setup_mutex;

// cuCtxGetCurrent through the runtime's driver entry point (the library links only the runtime)
typedef int (*CtxGetCurrentFn)(void**);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  return fn;
}

// Host code cannot use the array's name as a device address: it is a
// host-side stand-in.  Look the device address up once per device, with that
// device current.  The cached address is tied to the CUDA context that was
// current at the lookup: after cudaDeviceReset, or under another context on
// the same device, the next call looks it up again.
int device_addresses(void** scratch, int** status) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return EPH_ECUDA;
  }
  void* cur = nullptr;
  CtxGetCurrentFn get = ctx_get_current();
  if (!get || get(&cur) != 0) return EPH_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  Addr& a = g_addr[dev];
  if (!cur || a.ctx != cur || !a.scratch) {
    void* s = nullptr;
    void* f = nullptr;
    // (the lookup also makes the device's primary context current if no context was)
    if (cudaGetSymbolAddress(&s, g_noalloc_scratch) != cudaSuccess ||
        cudaGetSymbolAddress(&f, g_noalloc_status) != cudaSuccess || !s || !f) {
      cudaGetLastError();
      return EPH_ECUDA;
    }
    if (!cur && (get(&cur) != 0 || !cur)) return EPH_ECUDA;
    a.ctx = cur;
    a.scratch = s;
    a.status = static_cast<int*>(f);
  }
  *scratch = a.scratch;
  *status = a.status;
  return EPH_OK;
}

// bytes of scratch one call needs: phases [nk][ne] (rounded up to 256 B) + H(k) [nk][nb][nb]
size_t scratch_bytes(int nk, int nb, int ne) {
  const size_t pk = (size_t)nk * ne * sizeof(double2);
  return ((pk + 255) & ~(size_t)255) + (size_t)nk * nb * nb * sizeof(double2);
}
}  // namespace

extern "C" int eph_bands_noalloc(int nk, const double* kpts, int nb, int ne, const int* Re, const double* we,
                                 const double* H_Re, double* eps, double* U, int max_sweeps, void* cuda_stream) {
  if (nk < 1 || nb < 1 || nb > 16 || ne < 1 || !kpts || !Re || !H_Re || !eps || !U) return EPH_EINVAL;
  const size_t need = scratch_bytes(nk, nb, ne);
  if (need > (size_t)EPH_NOALLOC_SCRATCH_BYTES) return EPH_EINVAL;  // beyond the fixed scratch
  void* scratch = nullptr;
  int* status = nullptr;
  int rc = device_addresses(&scratch, &status);
  if (rc != EPH_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nb2 = nb * nb;
  double2* Pk = static_cast<double2*>(scratch);
  const size_t pk = ((size_t)nk * ne * sizeof(double2) + 255) & ~(size_t)255;
  double2* Hk = reinterpret_cast<double2*>(static_cast<unsigned char*>(scratch) + pk);
  // the convergence flag must start at zero; the scratch arrays are fully overwritten
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return EPH_ECUDA;
  if (eph::launch_phase(kpts, nk, Re, we, ne, Pk, ne, st) != cudaSuccess) return EPH_ECUDA;
  if (eph::launch_zgemm(nk, nb2, ne, Pk, ne, 0, reinterpret_cast<const double2*>(H_Re), nb2, 0, Hk, nb2, 0, 1, st) !=
      cudaSuccess)
    return EPH_ECUDA;
  if (eph::launch_jacobi(Hk, nb2, nb, nb, nk, eps, nb, reinterpret_cast<double2*>(U), nb2,
                         max_sweeps > 0 ? max_sweeps : 20, status, st) != cudaSuccess)
    return EPH_ECUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return EPH_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return EPH_ECUDA;
  return h ? EPH_ENOTCONV : EPH_OK;
}
