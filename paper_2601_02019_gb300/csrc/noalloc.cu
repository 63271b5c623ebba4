// as_symeig_noalloc: the FP64 symmetric eigensolver with no allocation.
//
// Some callers cannot allocate device memory: allocators' own callbacks, and
// real-time serving paths that forbid allocation after start-up.  This
// entry point takes device pointers for its input and outputs and keeps its
// scratch space (a copy of A, since the solver overwrites its input, and the
// solver's work vectors) in one file-scope device array.
//
// The array is reserved on every GPU that loads this library until the
// process exits.  All calls share it and it keeps the last call's contents
// (nothing in it has to start at zero: every value the solver reads is
// written earlier in the same call).  Calls whose work overlaps on the GPU
// race with each other.  The first call on a device (and the first call after
// that device's context was destroyed and made again, for example after
// cudaDeviceReset, which loads the module and its array anew) does a one-time
// set-up: it looks up the array's device address with cudaGetSymbolAddress,
// which allocates nothing.  Make that first call on each device before any
// stream capture begins.
#include <mutex>

#include "eig.cuh"
#include "kernels.cuh"

namespace {

// Largest supported order and the resulting scratch size (doubles):
// n*n for the copy of A plus the solver's work vectors for nev <= n.
constexpr int kNoAllocMaxN = 128;
constexpr size_t kNoAllocDoubles = (size_t)kNoAllocMaxN * kNoAllocMaxN + 2 * (size_t)kNoAllocMaxN +
                                   5 * (size_t)kNoAllocMaxN * kNoAllocMaxN + 64;   // 98,624 doubles = 788,992 bytes

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
// Per device: the context in which the array's address was looked up, and
// that address.  A new context (after a device reset) holds a new copy of the
// module, so the address is looked up again when the current context differs.
struct ScratchAddr {
  CUcontext ctx = nullptr;
  double* ptr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// cuCtxGetCurrent through the runtime's driver entry point (the library links
// the CUDA runtime only).
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(p);
  }();
  return fn;
}

}  // namespace

extern "C" as_status as_symeig_noalloc(int32_t n, const double* A, int32_t nev, double* evals, double* vecs,
                                       void* cuda_stream) {
  if (n < 1 || n > kNoAllocMaxN || nev < 1 || nev > n || !A || !evals || !vecs) return AS_EINVAL;
  int dev = 0;
  AS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return AS_EINVAL;
  CtxGetCurrentFn get_ctx = ctx_get_current();
  if (!get_ctx) return AS_ENOTSUP;
  CUcontext ctx = nullptr;
  if (get_ctx(&ctx) != CUDA_SUCCESS) return AS_EDEVICE;
  if (!ctx) {   // no context current on this thread yet: cudaSetDevice makes the primary one current
    AS_CUDA_TRY(cudaSetDevice(dev));
    if (get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return AS_EDEVICE;
  }
  double* Acopy = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    ScratchAddr& sa = g_scratch[dev];
    if (sa.ctx != ctx || !sa.ptr) {
      // once per device and context, with that device current: the host-side
      // name of the array is only a stand-in, the kernels need its device address
      void* p = nullptr;
      AS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      sa.ctx = ctx;
      sa.ptr = (double*)p;
    }
    Acopy = sa.ptr;
  }
  double* work = Acopy + (size_t)kNoAllocMaxN * kNoAllocMaxN;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  AS_CUDA_TRY(cudaMemcpyAsync(Acopy, A, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return as::launch_eig(s, n, Acopy, n, nev, evals, vecs, nev, work);
}
