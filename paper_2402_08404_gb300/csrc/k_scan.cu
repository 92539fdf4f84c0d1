// Deterministic exclusive scans over device arrays whose length may live in device memory
// (so the step never reads a count back to the host).  Three phases with a fixed number of
// blocks: per-block chunk sums, one-block scan of the sums, per-block chunk scan.
#include "pic_internal.cuh"

namespace pic {

constexpr int kScanThreads = 512;

template <typename T>
__device__ T block_sum(T v, T *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T s = 0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    sh[32] = s;
  }
  __syncthreads();
  s = sh[32];
  __syncthreads();
  return s;
}

// inclusive scan of one value per thread across the block; returns inclusive prefix, *tot = sum
template <typename T>
__device__ T block_incl_scan(T v, T *sh, T *tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T w = (lane < nw) ? sh[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < nw) sh[lane] = w;
  }
  __syncthreads();
  if (wid > 0) v += sh[wid - 1];
  *tot = sh[nw - 1];
  __syncthreads();
  return v;
}

template <typename T>
__global__ void k_scan_partial(const T *__restrict__ in, int64_t n_host, const int64_t *n_dev, T *partial) {
  __shared__ T sh[33];
  const int64_t n = n_dev ? *n_dev : n_host;
  const int nb = gridDim.x;
  const int64_t chunk = (n + nb - 1) / nb;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  T s = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += in[i];
  s = block_sum<T>(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename T>
__global__ void k_scan_top(T *partial, int nb, T *total) {
  __shared__ T sh[33];
  T carry = 0;
  for (int base = 0; base < nb; base += blockDim.x) {
    const int i = base + threadIdx.x;
    T v = i < nb ? partial[i] : T(0);
    T tot;
    T inc = block_incl_scan<T>(v, sh, &tot);
    if (i < nb) partial[i] = carry + inc - v;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T>
__global__ void k_scan_apply(const T *__restrict__ in, T *__restrict__ out, int64_t n_host, const int64_t *n_dev,
                             const T *__restrict__ partial) {
  __shared__ T sh[33];
  const int64_t n = n_dev ? *n_dev : n_host;
  const int nb = gridDim.x;
  const int64_t chunk = (n + nb - 1) / nb;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  T carry = partial[blockIdx.x];
  for (int64_t base = lo; base < hi; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    T v = i < hi ? in[i] : T(0);
    T tot;
    T inc = block_incl_scan<T>(v, sh, &tot);
    if (i < hi) out[i] = carry + inc - v;
    carry += tot;
  }
}

template <typename T>
static int scan_impl(pic_t *h, const T *in, T *out, int64_t n, const int64_t *n_dev, T *total) {
  const int nb = 2 * h->nsm;
  T *partial = (T *)h->scan_tmp;
  ++h->nlaunch;
  k_scan_partial<T><<<nb, kScanThreads, 0, h->stream>>>(in, n, n_dev, partial);
  ++h->nlaunch;
  k_scan_top<T><<<1, 1024, 0, h->stream>>>(partial, nb, total);
  ++h->nlaunch;
  k_scan_apply<T><<<nb, kScanThreads, 0, h->stream>>>(in, out, n, n_dev, partial);
  return launch_check(h, "scan");
}

int scan_u32(pic_t *h, const uint32_t *in, uint32_t *out, int64_t n, const int64_t *n_dev, uint32_t *total) {
  return scan_impl<uint32_t>(h, in, out, n, n_dev, total);
}
int scan_u64(pic_t *h, const uint64_t *in, uint64_t *out, int64_t n, const int64_t *n_dev, uint64_t *total) {
  return scan_impl<uint64_t>(h, in, out, n, n_dev, total);
}

}  // namespace pic
