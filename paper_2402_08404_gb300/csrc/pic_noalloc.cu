// Allocation-free form of pic_emission_eval.
//
// pic_emission_eval stages its inputs and outputs in device memory it takes with cudaMalloc and
// gives back with cudaFree.  Some callers cannot do that: a process whose device memory is
// entirely reserved by another framework's pool, or a latency-bound loop that cannot afford the
// device-wide synchronisation cudaFree implies.  pic_emission_eval_noalloc stages through a
// fixed array compiled into the library instead, and allocates nothing.
//
// The staging array below is a file-scope __device__ variable: every GPU that loads the
// library holds it (1.5 MiB) until the process exits.  Host code must not pass the symbol
// itself to a kernel (on the host it is only a stand-in); its device address is looked up once
// per device with cudaGetSymbolAddress, with that device current, on the first call made on
// that device.  Make that first call before any stream capture starts on the device.  A call
// made while another device is current is refused with PIC_E_INVALID (the staging address and
// the handle's stream would belong to different GPUs).
//
// All calls share the one array: two calls whose work overlaps on the GPU (different streams,
// different threads) race on it and must be serialised by the caller.  Nothing in it has to
// start at zero: every call writes all of the inputs it reads and all of the outputs it returns.
#include <mutex>
#include <string>

#include "pic_internal.cuh"

namespace pic {

constexpr int64_t kNoAllocMax = PIC_NOALLOC_MAX_TUPLES;

// F, T, phi_w, R (inputs) and J, PN (outputs), kNoAllocMax doubles each
static __device__ __align__(256) double g_emission_staging[6 * kNoAllocMax];

constexpr int kMaxDevices = 128;
static std::mutex g_staging_mutex;
static double *g_staging_ptr[kMaxDevices] = {};

// Device address of the staging array on the handle's device, which the caller has checked is
// current (looked up once per device).
static int staging_address(pic_t *h, double **out) {
  const int dev = h->device;
  cudaError_t e = cudaSuccess;
  if (dev < 0 || dev >= kMaxDevices) return pic_fail(h, PIC_E_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lock(g_staging_mutex);
  if (!g_staging_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_emission_staging);
    if (e != cudaSuccess || !p)
      return pic_fail(h, PIC_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_staging_ptr[dev] = (double *)p;
  }
  *out = g_staging_ptr[dev];
  return PIC_OK;
}

}  // namespace pic

using namespace pic;

extern "C" int pic_emission_eval_noalloc(pic_t *h, const double *F, const double *T, const double *phi_w,
                                         const double *R, double *J, double *PN, int64_t n) {
  if (!h || n < 0 || (n > 0 && (!F || !T || !phi_w || !R || !J || !PN))) return PIC_E_INVALID;
  if (n > kNoAllocMax)
    return pic_fail(h, PIC_E_INVALID, "pic_emission_eval_noalloc: n = " + std::to_string(n) +
                                          " exceeds the fixed staging size of " + std::to_string(kNoAllocMax) +
                                          " tuples; split the call");
  PIC_TRY(check_device(h));
  if (n == 0) return PIC_OK;
  double *buf = nullptr;
  PIC_TRY(staging_address(h, &buf));
  double *dF = buf, *dT = buf + kNoAllocMax, *dW = buf + 2 * kNoAllocMax, *dR = buf + 3 * kNoAllocMax;
  double *dJ = buf + 4 * kNoAllocMax, *dP = buf + 5 * kNoAllocMax;
  cudaStream_t st = h->stream;
  PIC_CUDA(h, cudaMemcpyAsync(dF, F, n * 8, cudaMemcpyHostToDevice, st));
  PIC_CUDA(h, cudaMemcpyAsync(dT, T, n * 8, cudaMemcpyHostToDevice, st));
  PIC_CUDA(h, cudaMemcpyAsync(dW, phi_w, n * 8, cudaMemcpyHostToDevice, st));
  PIC_CUDA(h, cudaMemcpyAsync(dR, R, n * 8, cudaMemcpyHostToDevice, st));
  PIC_TRY(emission_eval_dev(h, dF, dT, dW, dR, dJ, dP, n, (h->prm.flags & PIC_F_FAST_INTEGRAL) != 0));
  PIC_CUDA(h, cudaMemcpyAsync(J, dJ, n * 8, cudaMemcpyDeviceToHost, st));
  PIC_CUDA(h, cudaMemcpyAsync(PN, dP, n * 8, cudaMemcpyDeviceToHost, st));
  PIC_CUDA(h, cudaStreamSynchronize(st));
  return PIC_OK;
}
