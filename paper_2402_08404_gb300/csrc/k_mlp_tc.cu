// Emission surrogate inference on the fifth-generation tensor cores (tcgen05, TMEM accumulator):
// the whole forward pass of the 7 -> 128 -> 128 -> 128 -> 2 MLP in one persistent kernel.
//
// A CTA of 256 threads owns a tile of 128 rows at a time, two threads per row (each takes half of
// the 128 columns; warps w and w + 4 share TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31):
//   layer 1 (7 -> 128, FP32 on the CUDA cores) -> GELU -> BF16 activations in shared memory;
//   layer 2: 8 tcgen05.mma (M = N = 128, K = 16 each) from shared memory into a 128-column FP32
//            accumulator in tensor memory; tcgen05.ld brings each row back to its thread for
//            bias + GELU -> BF16 activations (the same shared tile);
//   layer 3: the same with W3; layer 4 (128 -> 2, FP32) straight from the registers.
// The hidden weights stay in shared memory for all the CTA's tiles.  The arithmetic is that of
// the reference path of k_mlp.cu (BF16 operands, FP32 accumulation, exact-erf GELU, FP32 input
// and output layers); only the order of the FP32 accumulation inside a 128-term dot product
// differs.
//
// Operand layout (no swizzle, K-major): a 128 x 128 BF16 matrix is stored as 16 x 16 "core
// matrices" of 8 rows x 16 bytes; core matrix (g, q) -- rows 8g..8g+7, columns 8q..8q+7 -- sits
// at byte (16 g + q) 128 and row r of it at +16 r.  Core matrices adjacent in K are 128 bytes
// apart (leading byte offset), adjacent in M/N 2048 bytes (stride byte offset).
//
// Every wait on the MMA completion barrier is bounded; a wait that runs out sets the device
// error word, releases the tensor memory and ends the kernel.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr int kH = 128, kIn = 7, kXld = 8, kOut = 2;
constexpr int kTile = 128;                     // rows per tile = MMA M
constexpr int kThreadsTc = 256;                // two threads per row
constexpr int kMatBytes = kH * kH * 2;         // one 128 x 128 BF16 operand
constexpr uint32_t kLBO = 128, kSBO = 2048;    // core-matrix offsets along K and along M/N
constexpr uint32_t kTmemCols = 128;            // FP32 accumulator columns (N)
constexpr long kWaitLimit = 1L << 24;          // polls of the completion barrier before giving up

// shared memory: [A | W2 | W3] operands, then FP32 small layers, barrier, TMEM address
struct Smem {
  alignas(1024) unsigned char A[kMatBytes];
  alignas(1024) unsigned char W2[kMatBytes];
  alignas(1024) unsigned char W3[kMatBytes];
  float w1[kH * kIn], b1[kH], b2[kH], b3[kH], w4[kOut * kH], b4[kOut];
  float ypart[2][kTile];                       // second half's output-layer partial sums
  alignas(8) unsigned long long bar;
  uint32_t tmem;
  int fail;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) of a core-matrix tile
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)(((row >> 3) * 16 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading and stride byte offsets (all >> 4),
// descriptor version 1 (bits 46-47), no swizzle (layout type 0, bits 61-63)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kLBO >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((kSBO >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kH >> 3) << 17) |
                            ((uint32_t)(kTile >> 4) << 24);

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}

// bounded wait for the completion of phase `parity` of the barrier; false when it runs out
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (long it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 32 consecutive FP32 accumulator columns of this thread's row (its TMEM lane)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// eight BF16 activations of this thread's row into columns 8q..8q+7 of the A tile
__device__ __forceinline__ void store8(unsigned char *A, int row, int q, const float a[8]) {
  uint4 v;
  __nv_bfloat162 p0 = __floats2bfloat162_rn(a[0], a[1]), p1 = __floats2bfloat162_rn(a[2], a[3]);
  __nv_bfloat162 p2 = __floats2bfloat162_rn(a[4], a[5]), p3 = __floats2bfloat162_rn(a[6], a[7]);
  v.x = *reinterpret_cast<uint32_t *>(&p0);
  v.y = *reinterpret_cast<uint32_t *>(&p1);
  v.z = *reinterpret_cast<uint32_t *>(&p2);
  v.w = *reinterpret_cast<uint32_t *>(&p3);
  *reinterpret_cast<uint4 *>(A + core_off(row, 8 * q)) = v;
}

}  // namespace

// Y (rows x 2) of the feature rows X (rows x 8, 7 used); master: FP32 parameters in the public
// layout (W1 b1 W2 b2 W3 b3 W4 b4, row-major [out][in]); w2, w3: their BF16 copies.
__global__ void __launch_bounds__(kThreadsTc, 1) k_mlp_forward_tc(const float *__restrict__ X, int64_t rows,
                                                            const float *__restrict__ master,
                                                            const __nv_bfloat16 *__restrict__ w2,
                                                            const __nv_bfloat16 *__restrict__ w3, float *Y, int *err) {
  extern __shared__ unsigned char smem_raw[];
  Smem &S = *reinterpret_cast<Smem *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kTile - 1), half = tid >> 7;   // this thread's row and column half
  constexpr int oW1 = 0, oB1 = kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH * kH,
                oW4 = oB3 + kH, oB4 = oW4 + kOut * kH;
  for (int e = tid; e < kH * kH; e += kThreadsTc) {
    const int n = e / kH, k = e - n * kH;
    *reinterpret_cast<__nv_bfloat16 *>(S.W2 + core_off(n, k)) = w2[e];
    *reinterpret_cast<__nv_bfloat16 *>(S.W3 + core_off(n, k)) = w3[e];
  }
  for (int e = tid; e < kH * kIn; e += kThreadsTc) S.w1[e] = master[oW1 + e];
  for (int e = tid; e < kOut * kH; e += kThreadsTc) S.w4[e] = master[oW4 + e];
  if (tid < kH) {
    S.b1[tid] = master[oB1 + tid];
    S.b2[tid] = master[oB2 + tid];
    S.b3[tid] = master[oB3 + tid];
  }
  if (tid < kOut) S.b4[tid] = master[oB4 + tid];
  const uint32_t bar = smem_u32(&S.bar);
  if (tid == 0) {
    S.fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&S.tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = S.tmem;
  const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16);   // this warp's 32 lanes (rows)
  const uint32_t a_addr = smem_u32(S.A), w_addr[2] = {smem_u32(S.W2), smem_u32(S.W3)};
  uint32_t phase = 0;
  for (int64_t t0 = (int64_t)blockIdx.x * kTile; t0 < rows; t0 += (int64_t)gridDim.x * kTile) {
    const int64_t r = t0 + row;
    float x[kIn];
#pragma unroll
    for (int c = 0; c < kIn; ++c) x[c] = r < rows ? X[r * kXld + c] : 0.f;
    // layer 1 (FP32), GELU, BF16 activations of this row's column half
    for (int q = half * (kH / 16); q < (half + 1) * (kH / 16); ++q) {
      float a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int o = 8 * q + u;
        float z = S.b1[o];
#pragma unroll
        for (int c = 0; c < kIn; ++c) z += S.w1[o * kIn + c] * x[c];
        a[u] = gelu_f(z);
      }
      store8(S.A, row, q, a);
    }
    float y0 = 0.f, y1 = 0.f;
    for (int layer = 0; layer < 2; ++layer) {
      // the activations written by every thread are visible to the tensor core's async proxy
      fence_proxy_async();
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
      if (tid == 0) {
#pragma unroll
        for (int kk = 0; kk < kH / 16; ++kk)   // K = 16 per instruction: two core matrices along K
          mma_bf16(tmem, smem_desc(a_addr + kk * 2 * kLBO), smem_desc(w_addr[layer] + kk * 2 * kLBO), kk > 0 ? 1u : 0u);
        mma_commit(bar);
      }
      const bool ok = bar_wait(bar, phase);
      phase ^= 1u;
      if (!ok) atomicExch(&S.fail, 1);
      fence_after_sync();
      __syncthreads();
      if (S.fail) break;
      const float *bias = layer == 0 ? S.b2 : S.b3;
      for (int cc = half * 2; cc < half * 2 + 2; ++cc) {   // this thread's 64 columns
        float v[32];
        tmem_ld32(taddr + 32 * cc, v);
        if (layer == 0) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = gelu_f(v[8 * q + u] + bias[32 * cc + 8 * q + u]);
            store8(S.A, row, 4 * cc + q, a);
          }
        } else {
#pragma unroll
          for (int u = 0; u < 32; ++u) {
            const int k = 32 * cc + u;
            const float a = gelu_f(v[u] + bias[k]);
            y0 += S.w4[k] * a;
            y1 += S.w4[kH + k] * a;
          }
        }
      }
      // every thread's accumulator reads are done before the next MMA overwrites the columns
      fence_before_sync();
    }
    if (S.fail) break;
    if (half) {
      S.ypart[0][row] = y0;
      S.ypart[1][row] = y1;
    }
    __syncthreads();
    if (!half && r < rows) {
      Y[r * kOut] = (y0 + S.ypart[0][row]) + S.b4[0];
      Y[r * kOut + 1] = (y1 + S.ypart[1][row]) + S.b4[1];
    }
    fence_before_sync();
    __syncthreads();   // A and the accumulator are free for the next tile
    fence_after_sync();
  }
  if (S.fail && tid == 0) atomicOr(err, kErrTimeout);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// Launch the fused forward pass for `rows` feature rows (two CTAs per SM at most).
int mlp_forward_tc(pic_t *h, const float *X, int64_t rows, const float *master, const __nv_bfloat16 *w2,
                   const __nv_bfloat16 *w3, float *Y) {
  if (rows <= 0) return PIC_OK;
  const int smem = (int)sizeof(Smem) + 1024;
  static int configured_dev = -1;
  int dev = 0;
  PIC_CUDA(h, cudaGetDevice(&dev));
  if (configured_dev != dev) {
    PIC_CUDA(h, cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    configured_dev = dev;
  }
  const int64_t tiles = (rows + kTile - 1) / kTile;
  const int grid = (int)std::min<int64_t>(tiles, 2 * (int64_t)h->nsm);   // two CTAs fit an SM
  ++h->nlaunch;
  k_mlp_forward_tc<<<grid, kThreadsTc, smem, h->stream>>>(X, rows, master, w2, w3, Y, &h->clock->err);
  return launch_check(h, "mlp forward (tcgen05)");
}


// ---- training GEMMs on the tensor cores -------------------------------------------------------
// C(M x 128) = A(M x K) B(K x 128) with BF16 operands and FP32 accumulation in tensor memory, for
// the surrogate's training: the hidden layers' forward products (K = 128), the gradients of their
// inputs (K = 128) and their weight gradients (M = 128, K = the batch, split over CTAs).  The
// operands are addressed with element strides, A(m, k) = A[m sam + k sak] and B(k, n) =
// B[k sbk + n sbn], so the transposed products read the stored matrices directly.  CTA (x, y, z)
// owns rows 128 x, columns 64 y and the z-th range of K: it stages 128 x 128 blocks of A and
// 64 x 128 blocks of B into shared memory in the K-major core-matrix layout with 16-byte
// transfers (an operand stored with unit stride along M or N is transposed in registers, 8 x 8
// elements at a time), zero outside the matrices, and one thread issues the eight K = 16 MMAs of
// a block.  With several K ranges each CTA writes its own partial (row-major M x 128 at
// C + z M 128), which a fixed-order sum then adds, so the result does not depend on scheduling.
namespace {
constexpr int kGemmThreads = 128;   // one thread per row of the tile (its TMEM lane)
constexpr int kGemmN = 64;          // columns per CTA (MMA N)
constexpr uint32_t kIdesc64 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kGemmN >> 3) << 17) |
                              ((uint32_t)(kTile >> 4) << 24);
struct GemmSmem {
  alignas(1024) unsigned char A[kTile * kH * 2];
  alignas(1024) unsigned char B[kGemmN * kH * 2];
  alignas(8) unsigned long long bar;
  uint32_t tmem;
  int fail;
};

__device__ __forceinline__ void mma_bf16_n64(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc64), "r"(accumulate));
}

// One 128-row-wide (rows = the tile's M or N index) by 128-K block of a strided BF16 operand into
// the core-matrix layout: X(r, k) = src[(r0 + r) sr + (k0 + k) sk] for r < nr, valid where
// r0 + r < rmax and k0 + k < kmax (zero elsewhere).  Unit stride along K: each thread moves 16-byte
// rows of 8 K-elements.  Unit stride along r: each thread loads 8 rows of K (8 r-elements each),
// transposes the 8 x 8 block in registers and stores 8 16-byte rows.
__device__ __forceinline__ void stage_block(unsigned char *dst, const __nv_bfloat16 *src, int64_t sr, int64_t sk, int r0,
                                            int nr, int rmax, int k0, int kmax, int tid) {
  if (sk == 1) {
    for (int e = tid; e < nr * (kH / 8); e += kGemmThreads) {
      const int r = e >> 4, k8 = (e & 15) * 8;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (r0 + r < rmax && k0 + k8 < kmax)
        v = *reinterpret_cast<const uint4 *>(src + (int64_t)(r0 + r) * sr + (k0 + k8));
      *reinterpret_cast<uint4 *>(dst + core_off(r, k8)) = v;
    }
  } else {
    for (int e = tid; e < (nr / 8) * (kH / 8); e += kGemmThreads) {
      const int rb = (e % (nr / 8)) * 8, kb = (e / (nr / 8)) * 8;
      uint32_t in[8][4];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (k0 + kb + kk < kmax && r0 + rb < rmax)
          v = *reinterpret_cast<const uint4 *>(src + (int64_t)(k0 + kb + kk) * sk + (r0 + rb));
        in[kk][0] = v.x; in[kk][1] = v.y; in[kk][2] = v.z; in[kk][3] = v.w;
      }
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        const uint32_t sel = (rr & 1) ? 0x7632u : 0x5410u;
        uint4 o;
        o.x = __byte_perm(in[0][rr >> 1], in[1][rr >> 1], sel);
        o.y = __byte_perm(in[2][rr >> 1], in[3][rr >> 1], sel);
        o.z = __byte_perm(in[4][rr >> 1], in[5][rr >> 1], sel);
        o.w = __byte_perm(in[6][rr >> 1], in[7][rr >> 1], sel);
        *reinterpret_cast<uint4 *>(dst + core_off(rb + rr, kb)) = o;
      }
    }
  }
}
}  // namespace

__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm_tc(GemmTcArgs g, int *err) {
  extern __shared__ unsigned char smem_raw[];
  GemmSmem &S = *reinterpret_cast<GemmSmem *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * kTile, n0 = blockIdx.y * kGemmN;
  const int kb = blockIdx.z * g.kper, ke = min(g.K, kb + g.kper);
  const uint32_t bar = smem_u32(&S.bar);
  if (tid == 0) {
    S.fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&S.tmem)),
                 "r"((uint32_t)kGemmN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = S.tmem;
  const uint32_t a_addr = smem_u32(S.A), b_addr = smem_u32(S.B);
  const __nv_bfloat16 *Ag = static_cast<const __nv_bfloat16 *>(g.A), *Bg = static_cast<const __nv_bfloat16 *>(g.B);
  uint32_t phase = 0;
  bool any = false;
  for (int k0 = kb; k0 < ke; k0 += kH) {
    stage_block(S.A, Ag, g.sam, g.sak, m0, kTile, g.M, k0, ke, tid);
    stage_block(S.B, Bg, g.sbn, g.sbk, n0, kGemmN, kH, k0, ke, tid);
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (tid == 0) {
#pragma unroll
      for (int q = 0; q < kH / 16; ++q)
        mma_bf16_n64(tmem, smem_desc(a_addr + q * 2 * kLBO), smem_desc(b_addr + q * 2 * kLBO), (any || q > 0) ? 1u : 0u);
      mma_commit(bar);
    }
    any = true;
    const bool ok = bar_wait(bar, phase);
    phase ^= 1u;
    if (!ok) atomicExch(&S.fail, 1);
    fence_after_sync();
    __syncthreads();   // the MMAs have read the staged blocks: they may be overwritten
    if (S.fail) break;
  }
  if (!S.fail) {
    float *C = g.C;
    int64_t scm = g.scm, scn = g.scn;
    if (g.splits > 1) {
      C = g.C + (int64_t)blockIdx.z * g.M * kH;
      scm = kH;
      scn = 1;
    }
    const int r = m0 + tid;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int cc = 0; cc < kGemmN / 32; ++cc) {
      float v[32];
      if (any) tmem_ld32(taddr + 32 * cc, v);
      else
        for (int u = 0; u < 32; ++u) v[u] = 0.f;
      if (r < g.M) {
        float *row = C + (int64_t)r * scm + (int64_t)(n0 + 32 * cc) * scn;
        if (scn == 1 && (((uintptr_t)row & 15) == 0)) {
#pragma unroll
          for (int u = 0; u < 32; u += 4) *reinterpret_cast<float4 *>(row + u) = make_float4(v[u], v[u + 1], v[u + 2], v[u + 3]);
        } else {
          for (int u = 0; u < 32; ++u) row[(int64_t)u * scn] = v[u];
        }
      }
    }
  }
  if (S.fail && tid == 0) atomicOr(err, kErrTimeout);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)kGemmN) : "memory");
}

int gemm_tc(pic_t *h, const GemmTcArgs &g0) {
  GemmTcArgs g = g0;
  // the 16-byte staging needs the unit-stride operand 16-byte aligned along that dimension
  if (!(g.sak == 1 || g.sam == 1) || !(g.sbk == 1 || g.sbn == 1) || ((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15) ||
      (g.sak != 1 && g.sak % 8) || (g.sak == 1 && g.sam % 8) || (g.sbk != 1 && g.sbk % 8) || (g.sbk == 1 && g.sbn % 8) ||
      (g.sam == 1 && g.M % 8) || ((g.sak == 1 || g.sbk == 1) && g.K % 8))
    return pic_fail(h, PIC_E_INVALID, "gemm_tc: operand layout not supported");
  g.kper = (g.K + g.splits - 1) / g.splits;
  g.kper = (g.kper + kH - 1) / kH * kH;
  const int smem = (int)sizeof(GemmSmem) + 1024;
  static int configured_dev = -1;
  int dev = 0;
  PIC_CUDA(h, cudaGetDevice(&dev));
  if (configured_dev != dev) {
    PIC_CUDA(h, cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    configured_dev = dev;
  }
  const dim3 grid((g.M + kTile - 1) / kTile, kH / kGemmN, g.splits);
  ++h->nlaunch;
  k_gemm_tc<<<grid, kGemmThreads, smem, h->stream>>>(g, &h->clock->err);
  return launch_check(h, "gemm (tcgen05)");
}

}  // namespace pic
