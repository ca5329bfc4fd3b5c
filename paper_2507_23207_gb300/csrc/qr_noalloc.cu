// krp_qr_noalloc: the FP64 thin QR of one FP32 sketch without any device
// allocation.
//
// Who needs this: callers that are not allowed to call cudaMalloc once they
// are running -- code that lives inside a framework whose caching allocator
// owns all device memory (a raw cudaMalloc would bypass its accounting and can
// fail or fragment the pool), latency-critical loops in which the implicit
// device synchronisation of cudaMalloc/cudaFree is unacceptable, and programs
// that reserve their whole device memory budget up front.  krp_qr grows the
// context's workspace with cudaMalloc when it is too small; this entry point
// instead uses one fixed scratch array that lives in the library image.
//
// The scratch is a file-scope __device__ array (KRP_QR_NOALLOC_MAX_DOUBLES
// doubles, 4 MiB), present on every GPU that loads the library until the
// process exits.  Its host-side name is only a stand-in, so the device address
// is looked up once per device with cudaGetSymbolAddress and cached.
#include <mutex>

#include "common.cuh"

namespace krp {
cudaError_t cholqr3_single_on_stream(const float* Y, int64_t m, int l, double* Q, double* R,
                                     double* scratch, cudaStream_t st);
}

namespace {

__device__ __align__(256) double g_qr_noalloc_scratch[KRP_QR_NOALLOC_MAX_DOUBLES];

constexpr int kMaxDevices = 256;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
cudaError_t scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_qr_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" krp_status krp_qr_noalloc(const float* Y, int64_t m, int l, double* Q, double* R,
                                     void* cuda_stream) {
  if (!Y || !Q) return KRP_EINVAL;
  if (l < 1 || l > 64 || m < l) return KRP_EINVAL;
  // working matrix + Gram + three pass factors + refill mask + status word
  const int64_t need = m * l + 4 * (int64_t)l * l + 2;
  if (m > (int64_t(1) << 40) || need > KRP_QR_NOALLOC_MAX_DOUBLES) return KRP_EINVAL;
  double* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return KRP_ECUDA;
  }
  const cudaError_t e = krp::cholqr3_single_on_stream(Y, m, l, Q, R, scratch,
                                                      static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return KRP_ECUDA;
  }
  return KRP_OK;
}
