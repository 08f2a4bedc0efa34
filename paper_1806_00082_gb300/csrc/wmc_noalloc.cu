// wmc_kernel_eval_noalloc: the Wigner-kernel evaluation of wmc_kernel_eval for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or hand the library a workspace): code
// embedded in an application whose device memory is owned by a pool allocator
// (a framework's caching allocator, an inference server, an engine with a
// fixed memory budget), where an outside cudaMalloc may fail, stall, implicitly
// synchronise the device, or go untracked; and applications that allocate
// everything at start-up and forbid allocation afterwards.  For them the only
// scratch this evaluation needs -- the sine matrix S[m][r] of the contraction
// -- lives in a fixed array in the library's own device memory instead of in a
// caller workspace.  The caller still passes the potential, the cell list and
// the output.
//
// The array holds the matrix for Q <= 1024 (512 x 512 floats, 1 MiB).  Every
// GPU that loads the library holds it until the process exits.  All calls share
// it and it keeps the contents of the last call: each call refills the part it
// uses (zero padding included) before reading it, so nothing depends on what an
// earlier call left there, but calls that overlap on the GPU (on different
// streams, or from several threads) race on it and must be serialised by the
// caller.
#include "wmc_device.cuh"

namespace wmc {
namespace {

constexpr int kNoallocMaxQ = 1024;
constexpr int kNoallocMaxKp = 512;  // (Q/2 - 1) rounded up to 32
constexpr int kNoallocMaxNp = 512;  // Q/2 rounded up to 64

static __device__ __align__(256) float g_sine_scratch[kNoallocMaxKp * kNoallocMaxNp];

// B[kk][r] = sin(2 pi ((kk+1) r mod Q) / Q) for kk < h-1, r < h, zero elsewhere.
__global__ void k_fill_sine_scratch(float* __restrict__ B, int Q, int Kp, int Np) {
  const long long n = (long long)Kp * Np;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    B[q] = sine_entry_n1(Q, (int)(q / Np), (int)(q % Np));
}

// Device address of the scratch array in the current context.  In host code
// the name g_sine_scratch is only a host-side stand-in for the symbol, so the
// address is looked up on every call: a cached address would outlive the
// context it belongs to (after cudaDeviceReset the next context may place the
// array elsewhere).
wmc_status scratch_on_current_device(float** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_sine_scratch);
  if (e != cudaSuccess || ptr == nullptr) return WMC_ERR_CUDA;
  *out = static_cast<float*>(ptr);
  return WMC_OK;
}

}  // namespace
}  // namespace wmc

extern "C" wmc_status wmc_kernel_eval_noalloc(const wmc_params* p, const float* V, const int32_t* occ,
                                              int32_t n_occ, float* VWh, wmc_stream_t stream) {
  using namespace wmc;
  if (!params_ok(p) || !V || n_occ < 0 || (n_occ > 0 && (!occ || !VWh))) return WMC_ERR_ARG;
  if (p->Q > kNoallocMaxQ) return WMC_ERR_CAPACITY;
  float* B = nullptr;
  const wmc_status st = scratch_on_current_device(&B);
  if (st != WMC_OK) return st;
  if (n_occ == 0) return WMC_OK;
  const Layout L = layout(*p);
  cudaStream_t s = (cudaStream_t)stream;
  k_fill_sine_scratch<<<128, 256, 0, s>>>(B, p->Q, L.Kp, L.Np);
  if (cudaGetLastError() != cudaSuccess) return WMC_ERR_CUDA;
  return launch_kernel_eval(*p, V, occ, nullptr, n_occ, n_occ, B, VWh, s) == cudaSuccess ? WMC_OK : WMC_ERR_CUDA;
}
