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

// elements per thread in the chunk scan; block chunks start on multiples of it (aligned vectors)
constexpr int kItems = 16;
__device__ __forceinline__ int64_t scan_chunk(int64_t n, int nb) {
  return ((n + nb - 1) / nb + kItems - 1) / kItems * kItems;
}

// per-block chunk sums: whole 16-byte vectors while they last (chunks start on multiples of
// kItems elements, so the vectors are aligned), the ragged end element by element
template <typename T>
__global__ void k_scan_partial(const T *__restrict__ in, int64_t n_host, const int64_t *n_dev, T *partial) {
  __shared__ T sh[33];
  constexpr int kPer = 16 / (int)sizeof(T);
  const int64_t n = n_dev ? *n_dev : n_host;
  const int nb = gridDim.x;
  const int64_t chunk = scan_chunk(n, nb);
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  T s = 0;
  const int64_t nvec = hi > lo ? (hi - lo) / kPer : 0;
  const uint4 *v = reinterpret_cast<const uint4 *>(in + lo);
  // four independent vector loads in flight per thread before any sum
  constexpr int kU = 4;
  for (int64_t q0 = threadIdx.x; q0 < nvec; q0 += (int64_t)kU * blockDim.x) {
    union { uint4 u; T e[kPer]; } x[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t q = q0 + (int64_t)u * blockDim.x;
      x[u].u = q < nvec ? v[q] : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u)
#pragma unroll
      for (int e = 0; e < kPer; ++e) s += x[u].e[e];
  }
  for (int64_t i = lo + nvec * kPer + threadIdx.x; i < hi; i += blockDim.x) s += in[i];
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

// per-block chunk scan: each thread scans kItems consecutive elements in registers (16-byte
// vector loads and stores when the run is whole), the block scans the thread totals
template <typename T>
__global__ void k_scan_apply(const T *__restrict__ in, T *__restrict__ out, int64_t n_host, const int64_t *n_dev,
                             const T *__restrict__ partial) {
  static_assert((kItems * sizeof(T)) % 16 == 0, "whole vectors per thread");
  constexpr int kVec = kItems * (int)sizeof(T) / 16;
  __shared__ T sh[33];
  const int64_t n = n_dev ? *n_dev : n_host;
  const int nb = gridDim.x;
  const int64_t chunk = scan_chunk(n, nb);
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  T carry = partial[blockIdx.x];
  using Run = union { uint4 q[kVec]; T e[kItems]; };
  // the run of kItems elements a thread takes at base (zeros past hi)
  auto load_run = [&](int64_t base, Run &v) {
    const int64_t i0 = base + (int64_t)threadIdx.x * kItems;
    if (i0 + kItems <= hi) {
      const uint4 *src = reinterpret_cast<const uint4 *>(in + i0);
#pragma unroll
      for (int q = 0; q < kVec; ++q) v.q[q] = src[q];
    } else {
#pragma unroll
      for (int q = 0; q < kItems; ++q) v.e[q] = i0 + q < hi ? in[i0 + q] : T(0);
    }
  };
  const int64_t span = (int64_t)blockDim.x * kItems;
  Run nxt;
  if (lo < hi) load_run(lo, nxt);
  for (int64_t base = lo; base < hi; base += span) {
    const int64_t i0 = base + (int64_t)threadIdx.x * kItems;
    const bool whole = i0 + kItems <= hi;
    Run v = nxt;
    if (base + span < hi) load_run(base + span, nxt);   // the next run's loads overlap this run's scan
    T s = 0;
#pragma unroll
    for (int q = 0; q < kItems; ++q) s += v.e[q];
    T tot;
    const T inc = block_incl_scan<T>(s, sh, &tot);
    T run = carry + inc - s;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      const T x = v.e[q];
      v.e[q] = run;
      run += x;
    }
    if (whole) {
      uint4 *dst = reinterpret_cast<uint4 *>(out + i0);
#pragma unroll
      for (int q = 0; q < kVec; ++q) dst[q] = v.q[q];
    } else {
#pragma unroll
      for (int q = 0; q < kItems; ++q)
        if (i0 + q < hi) out[i0 + q] = v.e[q];
    }
    carry += tot;
  }
}

template <typename T>
static int scan_impl(pic_t *h, const T *in, T *out, int64_t n, const int64_t *n_dev, T *total) {
  const int nb = 2 * h->nsm;
  T *partial = (T *)h->scan_tmp;
  ++h->nlaunch;
  { KtScope kt_(h, kidScanPartial, (double)n); k_scan_partial<T><<<nb, kScanThreads, 0, h->stream>>>(in, n, n_dev, partial); }
  ++h->nlaunch;
  k_scan_top<T><<<1, 1024, 0, h->stream>>>(partial, nb, total);
  ++h->nlaunch;
  { KtScope kt_(h, kidScanApply, (double)n); k_scan_apply<T><<<nb, kScanThreads, 0, h->stream>>>(in, out, n, n_dev, partial); }
  return launch_check(h, "scan");
}

int scan_u32(pic_t *h, const uint32_t *in, uint32_t *out, int64_t n, const int64_t *n_dev, uint32_t *total) {
  return scan_impl<uint32_t>(h, in, out, n, n_dev, total);
}
int scan_u64(pic_t *h, const uint64_t *in, uint64_t *out, int64_t n, const int64_t *n_dev, uint64_t *total) {
  return scan_impl<uint64_t>(h, in, out, n, n_dev, total);
}

}  // namespace pic
