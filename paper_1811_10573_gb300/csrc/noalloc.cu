// The tensor-core first-level contraction without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// this contraction: a host framework that owns every byte of device memory
// through its own pool and forbids raw allocations after start-up, a
// latency-critical loop that cannot afford the implicit synchronisation of
// cudaMalloc/cudaFree, or a process whose device-memory budget is already
// committed.  For them this entry point runs the split-K contraction with its
// partial sums in a file-scope device array instead of a context workspace;
// the caller passes only its inputs and its output.
#include <atomic>
#include <cstdio>
#include <mutex>

#include "../../include/cpals.h"
#include "internal.h"

namespace {

// Scratch for the split-K partial sums: every GPU that loads the library
// holds these 16 MiB (plus the error word) until the process exits.
constexpr size_t kNoallocScratchFloats = CPALS_NOALLOC_SCRATCH_FLOATS;
__device__ __align__(256) float g_noalloc_scratch[kNoallocScratchFloats];
__device__ __align__(256) int g_noalloc_err[4];

constexpr int kMaxDevices = 64;
constexpr int64_t kBK = 64;          // K granularity of the tensor-core kernel's splits
// Device addresses of the two arrays, per device.  The scratch pointer is
// published last with release ordering, so a thread that sees it also sees
// the error pointer; the set-up itself runs under a mutex, so host threads
// making their first call on a device at the same time do it once.
std::atomic<float*> g_scratch_ptr[kMaxDevices];
int* g_err_ptr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

// Host code sees the arrays' names only as host-side stand-ins; the device
// addresses come from cudaGetSymbolAddress, taken once per device with that
// device current (together with the kernels' shared-memory limits).
cudaError_t setup_device(int dev) {
  if (g_scratch_ptr[dev].load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[dev].load(std::memory_order_relaxed)) return cudaSuccess;
  void* sp = nullptr;
  void* ep = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&sp, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  e = cudaGetSymbolAddress(&ep, g_noalloc_err);
  if (e != cudaSuccess) return e;
  e = cpals::setup_umma_kernels();
  if (e != cudaSuccess) return e;
  g_err_ptr[dev] = static_cast<int*>(ep);
  g_scratch_ptr[dev].store(static_cast<float*>(sp), std::memory_order_release);
  return cudaSuccess;
}

}  // namespace

extern "C" cpals_status cpals_contract_bf16_noalloc(const void* Xb, const void* Bt, float* out,
                                                    int64_t batch, int64_t K, int64_t M, int R,
                                                    int64_t Kstride, int kmajor, int splits,
                                                    void* stream) {
  if (!Xb || !Bt || !out || batch < 1 || K < 1 || M < 1 || R < 1 || R > 128 || splits < 1 ||
      Kstride < K || Kstride % 8 != 0 || (kmajor && batch != 1))
    return CPALS_E_INVALID;
  if (!cpals::umma_supported(K, M, kmajor != 0, R)) return CPALS_E_UNSUPPORTED;
  // the partial sums of all splits must fit in the fixed scratch array; the
  // kernel rounds each K chunk up to its K granularity, which may leave fewer
  // splits than requested, and the bound applies to the splits it will use
  const int64_t kchunk = ((K + splits - 1) / splits + kBK - 1) / kBK * kBK;
  const int64_t used = (K + kchunk - 1) / kchunk;
  if (used > 1 && (double)used * (double)batch * (double)M * (double)R >
                      (double)kNoallocScratchFloats)
    return CPALS_E_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return CPALS_E_CUDA;
  }
  if (setup_device(dev) != cudaSuccess) {
    cudaGetLastError();
    return CPALS_E_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* scratch = g_scratch_ptr[dev].load(std::memory_order_acquire);
  int* err = g_err_ptr[dev];
  // the error word keeps the previous call's value: clear it first
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return CPALS_E_CUDA;
  int64_t launches = 0;
  const int Rpad = (R + 15) / 16 * 16;
  cudaError_t e = cpals::umma_gemm_bf16(static_cast<const __nv_bfloat16*>(Xb),
                                        static_cast<const __nv_bfloat16*>(Bt), out,
                                        scratch, batch, K, M, R, Rpad, Kstride,
                                        kmajor != 0, splits, err, nullptr,
                                        cpals::Launch{s, &launches});
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorInvalidValue ? CPALS_E_UNSUPPORTED : CPALS_E_CUDA;
  }
  int herr = 0;
  if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CPALS_E_CUDA;
  }
  return herr ? CPALS_E_TIMEOUT : CPALS_OK;
}
