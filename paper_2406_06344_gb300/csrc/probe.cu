// Peak probes: one-kernel loops that measure what the arithmetic pipes of this GPU deliver, as
// denominators for the rooflines of kernels that are not bound by HBM or by cuBLAS-class GEMMs
// (the FP64 grid and TT-SVD kernels, the FP32 and FP64 SIMT factor chains, the adjoint). The
// paper has no counterpart; these are measurement helpers.
//
//   DFMA   FP64 fused multiply-add, eight independent chains per thread, 32 per loop trip;
//   FFMA   FP32 fused multiply-add, the same;
//   DMMA   FP64 warp-level MMA (mma.sync m8n8k4), four independent accumulators per warp;
//   TF32   tcgen05.mma kind::tf32, M = 128, N = 256, K = 8 per instruction, one CTA per SM;
//   F16    tcgen05.mma kind::f16 (FP16 operands), M = 128, N = 256, K = 16 per instruction;
//   F16S*  the same with N = 64, 128 or 256 and operands that walk through four A and four B
//          slots of shared memory (every MMA reads new operand bytes, as in a pipelined GEMM).
// Operand values are seeded, nonzero and bounded, so the pipes switch real bits (power, and
// hence clocks, depend on the data). Each loop runs for tens of milliseconds.
#include <cuda_fp16.h>
#include <stdint.h>

#include "pttk_internal.cuh"

namespace pttk {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_loop_kernel(int64_t iters, T seed, T* __restrict__ sink) {
  T a[8], b = seed * T(0.999), c = T(1.0) - seed * T(1e-3);
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = seed + T(threadIdx.x + i) * T(1e-7);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == T(-12345.678)) sink[0] = s;  // keeps the loop alive; never true for these inputs
}

__global__ void __launch_bounds__(256) dmma_loop_kernel(int64_t iters, double seed, double* __restrict__ sink) {
  double a = seed + 1e-9 * threadIdx.x, b = 1.0 - 1e-9 * threadIdx.x;
  double c[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) c[i][0] = c[i][1] = 0.25 * i;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[i][0]), "+d"(c[i][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += c[i][0] + c[i][1];
  if (s == -12345.678) sink[0] = s;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// UMMA shared-memory descriptor: no swizzle, K-major, core matrices 128 B apart along K and
// 8-row groups `sbo` bytes apart.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// One CTA per SM; one thread issues `iters` MMAs of M = 128, N = 256 into one TMEM
// accumulator, then commits them to an mbarrier and waits for it (bounded: gives up after
// ~2 s and reports PTTK_ETIMEOUT). Operands: 128 rows (A) and 256 rows (B) of 32 bytes of K
// each in the K-major no-swizzle layout, seeded values.
template <bool TF32>
__global__ void __launch_bounds__(128, 1) umma_loop_kernel(int64_t iters, int* __restrict__ status) {
  __shared__ __align__(1024) uint8_t ops[(128 + 256) * 32];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x;
  for (int i = tid; i < (128 + 256) * 32 / 4; i += blockDim.x) {
    const float v = 0.25f + 0.5f * (float)((i * 2654435761u) >> 24) / 256.f;
    if (TF32) {
      reinterpret_cast<float*>(ops)[i] = v;
    } else {
      reinterpret_cast<__half2*>(ops)[i] = __floats2half2_rn(v, 1.f - v);
    }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    // A: 128 rows x 32 B at ops; B: 256 rows x 32 B after it. Rows of one 8-row group are 16 B
    // apart inside a 128-B core matrix; the two 16-B halves of a row's 32 B are two core
    // matrices 128 B apart; 8-row groups 256 B apart.
    const uint64_t a = umma_desc(smem_u32(ops), 256), b = umma_desc(smem_u32(ops + 128 * 32), 256);
    // instruction descriptor: FP32 accumulator, A/B format (TF32 = 2, FP16 = 0), K-major, N, M
    const uint32_t fmt = TF32 ? 2u : 0u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    for (int64_t it = 0; it < iters; ++it) {
      const uint32_t acc = it > 0 ? 1u : 0u;
      if (TF32)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                     "l"(a), "l"(b), "r"(idesc), "r"(acc)
                     : "memory");
      else
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                     "l"(a), "l"(b), "r"(idesc), "r"(acc)
                     : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bar))
                 : "memory");
    const long long t0 = clock64();
    bool done = false;
    while (!done) {
      uint32_t ok;
      asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                   "selp.u32 %0, 1, 0, p;\n\t}\n"
                   : "=r"(ok)
                   : "r"(smem_u32(&bar))
                   : "memory");
      done = ok != 0;
      if (!done && clock64() - t0 > (4ll << 30)) {
        atomicExch(status, (int)PTTK_ETIMEOUT);
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

constexpr int kUmmaPadSmem = 120 * 1024;

// Streaming-operand MMA loop: M = 128, K = 16 FP16 MMAs of width N whose operands walk through
// 4 A slots (128 rows x 128 B) and 4 B slots (256 rows x 128 B) in the K-major no-swizzle layout
// (core matrices 128 B apart along K, 8-row groups 1024 B apart); MMA it reads slot it % 4 at K
// step (it / 4) % 4. One CTA per SM, one thread issues; bounded final wait as in umma_loop_kernel.
constexpr int kStreamASlot = 128 * 128, kStreamBSlot = 256 * 128;
constexpr int kStreamOps = 4 * (kStreamASlot + kStreamBSlot);  // 196,608 bytes
constexpr int kStreamSmem = kStreamOps + 16;                    // + mbarrier and TMEM address

__device__ __forceinline__ uint64_t stream_desc(uint32_t saddr) {
  return umma_desc(saddr, 1024);
}

template <int N>
__global__ void __launch_bounds__(128, 1) umma_stream_kernel(int64_t iters, int* __restrict__ status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kStreamOps);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kStreamOps + 8);
  const int tid = threadIdx.x;
  for (int i = tid; i < kStreamOps / 4; i += blockDim.x) {
    const float v = 0.25f + 0.5f * (float)((i * 2654435761u) >> 24) / 256.f;
    reinterpret_cast<__half2*>(smem)[i] = __floats2half2_rn(v, 1.f - v);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    const uint32_t a0 = smem_u32(smem), b0 = a0 + 4 * kStreamASlot;
    const uint32_t idesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    for (int64_t it = 0; it < iters; ++it) {
      const uint32_t slot = (uint32_t)(it & 3), koff = (uint32_t)((it >> 2) & 3) * 256u;  // 2 core matrices
      const uint64_t a = stream_desc(a0 + slot * kStreamASlot + koff), b = stream_desc(b0 + slot * kStreamBSlot + koff);
      const uint32_t acc = it > 0 ? 1u : 0u;
      asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                   "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                   "l"(a), "l"(b), "r"(idesc), "r"(acc)
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
    const long long t0 = clock64();
    bool done = false;
    while (!done) {
      uint32_t ok;
      asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                   "selp.u32 %0, 1, 0, p;\n\t}\n"
                   : "=r"(ok)
                   : "r"(smem_u32(bar))
                   : "memory");
      done = ok != 0;
      if (!done && clock64() - t0 > (4ll << 30)) {
        atomicExch(status, (int)PTTK_ETIMEOUT);
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

}  // namespace
}  // namespace pttk

extern "C" pttk_status pttk_peak_probe(int kind, int64_t iters, void* stream, double* tflops, double* ms) {
  using namespace pttk;
  clear_error();
  if (!tflops || iters < 1 || iters > (int64_t)1 << 32) return set_error(PTTK_EINVAL, "bad probe argument");
  if (kind < PTTK_PROBE_DFMA || kind > PTTK_PROBE_F16S256) return set_error(PTTK_EINVAL, "unknown probe");
  cudaStream_t s = as_stream(stream);
  const int sms = sm_count();
  int* d_status = nullptr;
  PTTK_CUDA(cudaMallocAsync(&d_status, 16, s));
  PTTK_CUDA(cudaMemsetAsync(d_status, 0, 16, s));
  cudaEvent_t e0, e1;
  PTTK_CUDA(cudaEventCreate(&e0));
  PTTK_CUDA(cudaEventCreate(&e1));
  // the MMA loops take more than half an SM's shared memory (unused), so that no two of
  // their CTAs share an SM
  PTTK_CUDA(cudaFuncSetAttribute(umma_loop_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUmmaPadSmem));
  PTTK_CUDA(cudaFuncSetAttribute(umma_loop_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUmmaPadSmem));
  PTTK_CUDA(cudaFuncSetAttribute(umma_stream_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStreamSmem));
  PTTK_CUDA(cudaFuncSetAttribute(umma_stream_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStreamSmem));
  PTTK_CUDA(cudaFuncSetAttribute(umma_stream_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStreamSmem));
  double flops = 0.0;
  PTTK_CUDA(cudaEventRecord(e0, s));
  switch (kind) {
    case PTTK_PROBE_DFMA: {
      const unsigned blocks = (unsigned)sms * 8;
      fma_loop_kernel<double><<<blocks, 256, 0, s>>>(iters, 0.5, reinterpret_cast<double*>(d_status));
      flops = 2.0 * 32 * 256.0 * blocks * (double)iters;
      break;
    }
    case PTTK_PROBE_FFMA: {
      const unsigned blocks = (unsigned)sms * 8;
      fma_loop_kernel<float><<<blocks, 256, 0, s>>>(iters, 0.5f, reinterpret_cast<float*>(d_status));
      flops = 2.0 * 32 * 256.0 * blocks * (double)iters;
      break;
    }
    case PTTK_PROBE_DMMA: {
      const unsigned blocks = (unsigned)sms * 8;
      dmma_loop_kernel<<<blocks, 256, 0, s>>>(iters, 0.5, reinterpret_cast<double*>(d_status));
      flops = 2.0 * 8 * 8 * 4 * 4.0 * (256.0 / 32.0) * blocks * (double)iters;
      break;
    }
    case PTTK_PROBE_TF32:
      umma_loop_kernel<true><<<(unsigned)sms, 128, kUmmaPadSmem, s>>>(iters, d_status);
      flops = 2.0 * 128 * 256 * 8 * (double)sms * (double)iters;
      break;
    case PTTK_PROBE_F16S64:
      umma_stream_kernel<64><<<(unsigned)sms, 128, kStreamSmem, s>>>(iters, d_status);
      flops = 2.0 * 128 * 64 * 16 * (double)sms * (double)iters;
      break;
    case PTTK_PROBE_F16S128:
      umma_stream_kernel<128><<<(unsigned)sms, 128, kStreamSmem, s>>>(iters, d_status);
      flops = 2.0 * 128 * 128 * 16 * (double)sms * (double)iters;
      break;
    case PTTK_PROBE_F16S256:
      umma_stream_kernel<256><<<(unsigned)sms, 128, kStreamSmem, s>>>(iters, d_status);
      flops = 2.0 * 128 * 256 * 16 * (double)sms * (double)iters;
      break;
    default:
      umma_loop_kernel<false><<<(unsigned)sms, 128, kUmmaPadSmem, s>>>(iters, d_status);
      flops = 2.0 * 128 * 256 * 16 * (double)sms * (double)iters;
      break;
  }
  pttk::count_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(d_status, s);
  if (e != cudaSuccess) return cuda_error(e, "peak probe");
  if (kind >= PTTK_PROBE_TF32 && h == (int)PTTK_ETIMEOUT) return set_error(PTTK_ETIMEOUT, "peak probe: MMA wait ran out");
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return PTTK_OK;
}
