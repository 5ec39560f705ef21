// Factor chain of Algorithm 2, Phase 3 on the 5th-generation tensor cores (tcgen05).
//
// One CTA (4 warps) owns 128 points at a time (persistent over point tiles). Chain step i
// computes S_out (128 x R_out) = A (128 x K) * Gs (K x R_out), K = n R_in, with
//   A[p, a + R_in j] = T_j(xhat_{p,i}) * S_in[p, a]
// generated by the threads (thread t = point t) straight into shared memory in the UMMA
// K-major layout, and Gs the oriented core, pre-laid out once per handle as per-chunk images
// in the same layout and fetched chunk by chunk with one cp.async.bulk (TMA) copy. The
// accumulator lives in tensor memory (TMEM, 128 lanes = points, N_pad columns); one elected
// thread issues tcgen05.mma and commits to an mbarrier; after the last chunk the threads read
// the accumulator back with tcgen05.ld: into S_in (FP32, shared memory) for the next step, or,
// after the last step, into a shared-memory output tile that is copied to U/V with coalesced
// 16-byte stores (a tile's 128 rows are contiguous in the row-major output).
//
// Precision forms (FP32 accumulation throughout):
//   TF32   kind::tf32, operands rounded to TF32 (10-bit mantissa);
//   TF32X3 a = a_hi + a_lo, b = b_hi + b_lo (each TF32), D += a_hi b_hi + a_hi b_lo + a_lo b_hi;
//   BF16   kind::f16 with BF16 operands (7-bit mantissa);
//   BF16X3 the same split with BF16 parts.
// Core images are split from the FP64 cores; A is split after its FP32 product.
//
// Shared-memory operand layout (UMMA "no swizzle" K-major): 16-byte units, a core matrix is
// 8 rows x 16 bytes stored contiguously (128 B). Chunk of KC_BYTES = 128 bytes of K per row:
// unit (row r, k-unit u) at byte (r / 8) * 1024 + u * 128 + (r % 8) * 16. Descriptor: leading
// (K-direction) byte offset 128, stride (M/N-direction) byte offset 1024; one MMA consumes 32
// bytes of K (8 TF32 or 16 BF16), so k-step s starts at +256 s.
//
// Waits: every mbarrier wait is bounded; on timeout the CTA records PTTK_ETIMEOUT in a device
// status word, stops issuing work, waits (bounded) for its outstanding copies and MMAs, frees
// its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "pttk_internal.cuh"

namespace pttk {

int oriented_core_dims(const pttk_tt* tt, bool source, int step, int* R_in, int* R_out, int* coord);
const void* oriented_core_ptr(const pttk_tt* tt, bool source, int k, bool fp64);

namespace {

constexpr int TILE_M = 128;
constexpr int NTHREADS = 128;
constexpr int KC_BYTES = 128;            // bytes of K per row per chunk
constexpr int CHUNK_ROW_GROUP = 1024;    // bytes per 8-row group in a chunk
constexpr int BV_LD = PTTK_MAX_N + 1;    // basis row stride (odd: conflict-free)

// ---------------- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the completion of the phase with the given parity.
__device__ __noinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < (1u << 24); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i >= 32) __nanosleep(128);
  }
  return false;
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void umma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// 32 consecutive TMEM columns of this warp's 32 lanes (one row per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// UMMA shared-memory descriptor: no swizzle, K-major, LBO = 128 B, SBO = 1024 B.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((KC_BYTES >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((CHUNK_ROW_GROUP >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of tcgen05
  return d;                // base offset 0, absolute LBO mode, layout type 0 (no swizzle)
}

// Instruction descriptor: FP32 accumulator, A/B format (TF32 = 2, BF16 = 1), K-major A and B.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t ab_format, int M, int N) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

struct TcStep {
  const uint8_t* img_hi;  // nchunks x (Npad x 128 B)
  const uint8_t* img_lo;  // same, or null for single-product forms
  int K, nchunks, R_in, R_out, Npad, coord;
  float lo, hi;           // box of the coordinate
};
struct TcArgs {
  TcStep st[3];
  int nsteps, n, d;
  int64_t N;
  const float* pts;
  float* out;
  int* status;
  int ld_s;        // row stride of S_in (floats, odd)
  int tmem_cols;
  uint32_t b_slot_bytes;  // bytes reserved per B part per slot
  int out_aligned;        // output base is 16-byte aligned
};

// One unit (16 bytes) of the generated A operand: 4 TF32 or 8 BF16 elements of row p.
template <bool BF16, bool SPLIT>
__device__ __forceinline__ void gen_unit(const float* bv, const float* srow, int R_in, int K, int k,
                                         uint8_t* dst_hi, uint8_t* dst_lo) {
  constexpr int E = BF16 ? 8 : 4;
  float v[E];
  int j = k / R_in;
  int a = k - j * R_in;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    v[e] = (k + e < K) ? bv[j] * srow[a] : 0.f;
    if (++a == R_in) {
      a = 0;
      ++j;
    }
  }
  if constexpr (!BF16) {
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      h[e] = to_tf32(v[e]);
      l[e] = SPLIT ? to_tf32(v[e] - h[e]) : 0.f;
    }
    *reinterpret_cast<float4*>(dst_hi) = make_float4(h[0], h[1], h[2], h[3]);
    if (SPLIT) *reinterpret_cast<float4*>(dst_lo) = make_float4(l[0], l[1], l[2], l[3]);
  } else {
    __nv_bfloat162 h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * e]), h1 = __float2bfloat16_rn(v[2 * e + 1]);
      h[e] = __halves2bfloat162(h0, h1);
      if (SPLIT)
        l[e] = __halves2bfloat162(__float2bfloat16_rn(v[2 * e] - __bfloat162float(h0)),
                                  __float2bfloat16_rn(v[2 * e + 1] - __bfloat162float(h1)));
    }
    *reinterpret_cast<uint4*>(dst_hi) = *reinterpret_cast<uint4*>(h);
    if (SPLIT) *reinterpret_cast<uint4*>(dst_lo) = *reinterpret_cast<uint4*>(l);
  }
}

template <bool BF16, bool SPLIT>
__global__ void __launch_bounds__(NTHREADS, 1) chain_tc_kernel(TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  // layout: [A slots: 2 x (hi, lo) x 16 KB][B slots: 2 x (hi, lo) x b_slot_bytes]
  //         [S_in: 128 x ld_s floats][Bv: 128 x BV_LD floats][mbarriers][tmem addr][flags]
  constexpr uint32_t A_PART = TILE_M * KC_BYTES;  // 16 KB
  uint8_t* a_base = smem;
  uint8_t* b_base = a_base + 2 * 2 * A_PART;
  float* S = reinterpret_cast<float*>(b_base + 2 * 2 * (size_t)a.b_slot_bytes);
  float* Bv = S + (size_t)TILE_M * a.ld_s;
  uint64_t* bars = reinterpret_cast<uint64_t*>(Bv + (size_t)TILE_M * BV_LD + 1);  // 8-byte aligned below
  bars = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(bars) + 7) & ~uintptr_t(7));
  uint64_t* bar_b = bars;        // [2] B chunk arrived
  uint64_t* bar_mma = bars + 2;  // [2] MMAs of the chunk done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bar_b[0], 1);
    mbar_init(&bar_b[1], 1);
    mbar_init(&bar_mma[0], 1);
    mbar_init(&bar_mma[1], 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, (uint32_t)a.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t ntiles = (a.N + TILE_M - 1) / TILE_M;
  uint32_t g = 0;          // chunks issued so far by this CTA (slot = g & 1)
  uint32_t b_issued[2] = {0, 0}, b_waited[2] = {0, 0};  // TMA uses per slot (thread 0)
  bool failed = false;

  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t row0 = tile * TILE_M;
    const int rows = (int)std::min<int64_t>(TILE_M, a.N - row0);
    S[tid * a.ld_s] = 1.f;  // S_0 = 1 (r_0 = 1)
    for (int si = 0; si < a.nsteps && !failed; ++si) {
      const TcStep st = a.st[si];
      // Chebyshev basis T_0..T_{n-1} of this point's coordinate (three-term recurrence)
      {
        const int64_t gp = row0 + tid;
        const float x = tid < rows ? a.pts[gp * a.d + st.coord] : st.lo;
        const float xh = (2.f * x - st.lo - st.hi) / (st.lo - st.hi);
        float t0 = 1.f, t1 = xh;
        Bv[tid * BV_LD] = t0;
        if (a.n > 1) Bv[tid * BV_LD + 1] = t1;
        for (int k = 2; k < a.n; ++k) {
          const float t2 = 2.f * xh * t1 - t0;
          Bv[tid * BV_LD + k] = t2;
          t0 = t1;
          t1 = t2;
        }
      }
      __syncthreads();
      const uint32_t idesc = instr_desc(BF16 ? 1u : 2u, TILE_M, st.Npad);
      const uint32_t b_bytes = (uint32_t)st.Npad * KC_BYTES;
      constexpr int E = BF16 ? 8 : 4;  // elements per 16-byte unit
      const float* bv = Bv + tid * BV_LD;
      const float* srow = S + (size_t)tid * a.ld_s;
      for (int c = 0; c < st.nchunks; ++c, ++g) {
        const int slot = g & 1;
        if (g >= 2 && !mbar_wait(&bar_mma[slot], ((g >> 1) - 1) & 1)) *abort_flag = 1;
        uint8_t* a_hi = a_base + (size_t)slot * 2 * A_PART;
        uint8_t* a_lo = a_hi + A_PART;
        uint8_t* b_hi = b_base + (size_t)slot * 2 * a.b_slot_bytes;
        uint8_t* b_lo = b_hi + a.b_slot_bytes;
        if (tid == 0 && !*abort_flag) {
          fence_proxy_async();  // earlier generic accesses of this slot precede the TMA write
          mbar_arrive_expect_tx(&bar_b[slot], SPLIT ? 2 * b_bytes : b_bytes);
          tma_load_1d(b_hi, st.img_hi + (size_t)c * b_bytes, b_bytes, &bar_b[slot]);
          if (SPLIT) tma_load_1d(b_lo, st.img_lo + (size_t)c * b_bytes, b_bytes, &bar_b[slot]);
          ++b_issued[slot];
        }
        // generate this chunk of A for row tid: 8 units of 16 bytes
        const int kbase = c * (KC_BYTES / (BF16 ? 2 : 4));
        const uint32_t row_off = (uint32_t)(tid >> 3) * CHUNK_ROW_GROUP + (uint32_t)(tid & 7) * 16;
#pragma unroll 2
        for (int u = 0; u < 8; ++u)
          gen_unit<BF16, SPLIT>(bv, srow, st.R_in, st.K, kbase + u * E, a_hi + row_off + u * 128,
                                a_lo + row_off + u * 128);
        fence_proxy_async();
        __syncthreads();
        if (*abort_flag) {
          failed = true;
          break;
        }
        if (tid == 0) {
          if (!mbar_wait(&bar_b[slot], (b_waited[slot]++) & 1)) {
            *abort_flag = 1;
          } else {
            tc_fence_after();
            const uint32_t sa_hi = smem_u32(a_hi), sa_lo = smem_u32(a_lo);
            const uint32_t sb_hi = smem_u32(b_hi), sb_lo = smem_u32(b_lo);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
              const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
              const uint64_t ah = smem_desc(sa_hi + s * 256), bh = smem_desc(sb_hi + s * 256);
              if constexpr (BF16) {
                umma_f16(tmem, ah, bh, idesc, acc);
                if (SPLIT) {
                  umma_f16(tmem, ah, smem_desc(sb_lo + s * 256), idesc, 1u);
                  umma_f16(tmem, smem_desc(sa_lo + s * 256), bh, idesc, 1u);
                }
              } else {
                umma_tf32(tmem, ah, bh, idesc, acc);
                if (SPLIT) {
                  umma_tf32(tmem, ah, smem_desc(sb_lo + s * 256), idesc, 1u);
                  umma_tf32(tmem, smem_desc(sa_lo + s * 256), bh, idesc, 1u);
                }
              }
            }
            umma_commit(&bar_mma[slot]);
          }
        }
      }
      if (failed) break;
      // all MMAs of this step are complete once the last chunk's commit has landed
      const uint32_t glast = g - 1;
      if (!mbar_wait(&bar_mma[glast & 1], (glast >> 1) & 1)) *abort_flag = 1;
      __syncthreads();
      if (*abort_flag) {
        failed = true;
        break;
      }
      tc_fence_after();
      const bool last = si == a.nsteps - 1;
      float* otile = reinterpret_cast<float*>(a_base);  // output tile (reuses operand space)
      const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
      for (int cb = 0; cb < st.Npad; cb += 32) {
        float v[32];
        tmem_ld32(lane_addr + (uint32_t)cb, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int col = cb + i;
          if (col < st.R_out) {
            if (last) otile[(size_t)tid * st.R_out + col] = v[i];
            else S[(size_t)tid * a.ld_s + col] = v[i];
          }
        }
      }
      tc_fence_before();
      __syncthreads();
      if (last) {
        // rows row0 .. row0 + rows - 1 of the row-major output are one contiguous block
        float* dst = a.out + row0 * st.R_out;
        const int64_t nflt = (int64_t)rows * st.R_out;
        if (rows == TILE_M && a.out_aligned) {  // 128 * R_out * 4 bytes: a multiple of 16
          const float4* s4 = reinterpret_cast<const float4*>(otile);
          float4* d4 = reinterpret_cast<float4*>(dst);
          for (int64_t e = tid; e < nflt / 4; e += NTHREADS) d4[e] = s4[e];
        } else {
          for (int64_t e = tid; e < nflt; e += NTHREADS) dst[e] = otile[e];
        }
        __syncthreads();
      }
    }
  }

  // drain: outstanding TMA copies and MMA commits (bounded), then release TMEM
  if (tid == 0) {
    for (int s = 0; s < 2; ++s)
      while (b_waited[s] < b_issued[s]) {
        if (!mbar_wait(&bar_b[s], (b_waited[s]++) & 1)) break;
      }
  }
  if (failed && tid == 0) atomicExch(a.status, (int)PTTK_ETIMEOUT);
  if (g > 0) {
    const uint32_t glast = g - 1;
    mbar_wait(&bar_mma[glast & 1], (glast >> 1) & 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

// ---------------- core images -------------------------------------------------------------
// Image of the oriented core (K x R_out, column-major, FP64) for one chain step: chunk c holds
// rows o < Npad and K-elements [c*KC, (c+1)*KC) in the K-major no-swizzle layout above.
template <bool BF16>
__global__ void core_image_kernel(const double* __restrict__ G, int K, int R_out, int Npad, int nchunks,
                                  bool split, uint8_t* __restrict__ hi, uint8_t* __restrict__ lo) {
  constexpr int KC = BF16 ? 64 : 32;
  constexpr int E = BF16 ? 8 : 4;
  const int64_t total = (int64_t)nchunks * Npad * KC;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(e % KC);
    const int o = (int)((e / KC) % Npad);
    const int c = (int)(e / ((int64_t)KC * Npad));
    const int k = c * KC + kk;
    const double v = (k < K && o < R_out) ? G[k + (int64_t)K * o] : 0.0;
    const size_t off = (size_t)c * Npad * KC_BYTES + (size_t)(o >> 3) * CHUNK_ROW_GROUP +
                       (size_t)(kk / E) * 128 + (size_t)(o & 7) * 16;
    if constexpr (BF16) {
      const __nv_bfloat16 h = __double2bfloat16(v);
      reinterpret_cast<__nv_bfloat16*>(hi + off)[kk % E] = h;
      if (split) reinterpret_cast<__nv_bfloat16*>(lo + off)[kk % E] = __double2bfloat16(v - (double)__bfloat162float(h));
    } else {
      const float h = to_tf32((float)v);
      reinterpret_cast<float*>(hi + off)[kk % E] = h;
      if (split) reinterpret_cast<float*>(lo + off)[kk % E] = to_tf32((float)(v - (double)h));
    }
  }
}

struct Images {
  uint8_t* buf = nullptr;
  size_t hi_off[2][3] = {}, lo_off[2][3] = {};
  int Npad[2][3] = {}, nchunks[2][3] = {};
};

std::mutex g_img_mu;

}  // namespace

// Per-handle image cache (indexed by form), allocated on first use and freed with the handle.
struct TcImageCache {
  Images img[4];
};

static int form_index(pttk_prec p) {
  switch (p) {
    case PTTK_TF32: return 0;
    case PTTK_TF32X3: return 1;
    case PTTK_BF16: return 2;
    case PTTK_BF16X3: return 3;
    default: return -1;
  }
}

TcImageCache* tc_cache_new() { return new TcImageCache(); }
void tc_cache_free(TcImageCache* c) {
  if (!c) return;
  for (auto& im : c->img)
    if (im.buf) cudaFree(im.buf);
  delete c;
}

static pttk_status build_images(const pttk_tt* tt, pttk_prec prec, Images& im, cudaStream_t s) {
  const bool bf16 = prec == PTTK_BF16 || prec == PTTK_BF16X3;
  const bool split = prec == PTTK_TF32X3 || prec == PTTK_BF16X3;
  const int KC = bf16 ? 64 : 32;
  size_t total = 0;
  for (int side = 0; side < 2; ++side)
    for (int i = 0; i < tt->d; ++i) {
      int rin, rout, coord;
      oriented_core_dims(tt, side == 0, i, &rin, &rout, &coord);
      const int K = tt->n * rin;
      im.Npad[side][i] = ((rout + 15) / 16) * 16;
      im.nchunks[side][i] = (K + KC - 1) / KC;
      const size_t bytes = (size_t)im.nchunks[side][i] * im.Npad[side][i] * KC_BYTES;
      im.hi_off[side][i] = total;
      total += bytes;
      im.lo_off[side][i] = total;
      if (split) total += bytes;
    }
  PTTK_CUDA(cudaMalloc(&im.buf, std::max<size_t>(total, 16)));
  PTTK_CUDA(cudaMemsetAsync(im.buf, 0, std::max<size_t>(total, 16), s));
  for (int side = 0; side < 2; ++side)
    for (int i = 0; i < tt->d; ++i) {
      int rin, rout, coord;
      const int k = oriented_core_dims(tt, side == 0, i, &rin, &rout, &coord);
      const double* G = static_cast<const double*>(oriented_core_ptr(tt, side == 0, k, true));
      const int K = tt->n * rin;
      const int64_t work = (int64_t)im.nchunks[side][i] * im.Npad[side][i] * KC;
      const unsigned blocks = (unsigned)std::min<int64_t>((work + 255) / 256, (int64_t)sm_count() * 8);
      if (bf16)
        core_image_kernel<true><<<blocks, 256, 0, s>>>(G, K, rout, im.Npad[side][i], im.nchunks[side][i], split,
                                                       im.buf + im.hi_off[side][i], im.buf + im.lo_off[side][i]);
      else
        core_image_kernel<false><<<blocks, 256, 0, s>>>(G, K, rout, im.Npad[side][i], im.nchunks[side][i], split,
                                                        im.buf + im.hi_off[side][i], im.buf + im.lo_off[side][i]);
    }
  PTTK_CUDA(cudaGetLastError());
  PTTK_CUDA(cudaStreamSynchronize(s));
  return PTTK_OK;
}

// Shared memory needed by chain_tc_kernel for this handle and form.
static size_t tc_smem_bytes(int ld_s, uint32_t b_slot_bytes) {
  return 2 * 2 * (size_t)TILE_M * KC_BYTES + 2 * 2 * (size_t)b_slot_bytes +
         sizeof(float) * ((size_t)TILE_M * ld_s + (size_t)TILE_M * BV_LD + 1) + 8 + 6 * 8 + 16;
}

pttk_status factor_build_tc(const pttk_tt* tt, TcImageCache* cache, bool source, const float* P, int64_t N,
                            pttk_prec prec, float* out, int* d_status, cudaStream_t s) {
  if (N == 0) return PTTK_OK;
  const int fi = form_index(prec);
  if (fi < 0) return set_error(PTTK_EINVAL, "not a tensor-core form");
  Images& im = cache->img[fi];
  {
    std::lock_guard<std::mutex> lk(g_img_mu);
    if (!im.buf) PTTK_TRY(build_images(tt, prec, im, s));
  }
  const int side = source ? 0 : 1;
  const bool bf16 = prec == PTTK_BF16 || prec == PTTK_BF16X3;
  const bool split = prec == PTTK_TF32X3 || prec == PTTK_BF16X3;
  TcArgs a{};
  a.nsteps = tt->d;
  a.n = tt->n;
  a.d = tt->d;
  a.N = N;
  a.pts = P;
  a.out = out;
  a.status = d_status;
  int rin_max = 1, npad_max = 16;
  for (int i = 0; i < tt->d; ++i) {
    int rin, rout, coord;
    oriented_core_dims(tt, source, i, &rin, &rout, &coord);
    TcStep& st = a.st[i];
    st.img_hi = im.buf + im.hi_off[side][i];
    st.img_lo = split ? im.buf + im.lo_off[side][i] : nullptr;
    st.K = tt->n * rin;
    st.nchunks = im.nchunks[side][i];
    st.R_in = rin;
    st.R_out = rout;
    st.Npad = im.Npad[side][i];
    st.coord = coord;
    const int bj = source ? coord : tt->d + tt->dtheta + coord;
    st.lo = (float)tt->box[bj][0];
    st.hi = (float)tt->box[bj][1];
    rin_max = std::max(rin_max, rin);
    npad_max = std::max(npad_max, st.Npad);
  }
  if (npad_max > 256) return set_error(PTTK_ENOTSUP, "tensor-core chain: a rank above 256");
  a.ld_s = (rin_max | 1);
  if (a.ld_s < rin_max) a.ld_s += 2;
  int cols = 32;
  while (cols < npad_max) cols <<= 1;
  a.tmem_cols = cols;
  a.b_slot_bytes = (uint32_t)npad_max * KC_BYTES;
  // the final output tile (128 x R_out floats) reuses the operand slots
  const int rout_last = a.st[tt->d - 1].R_out;
  const size_t operand_bytes = 2 * 2 * (size_t)TILE_M * KC_BYTES + 2 * 2 * (size_t)a.b_slot_bytes;
  if ((size_t)TILE_M * rout_last * 4 > operand_bytes) return set_error(PTTK_ENOTSUP, "tensor-core chain: output tile");
  a.out_aligned = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  // at least 116 KB so that one CTA (and one TMEM allocation) fits per SM
  const size_t smem = std::max<size_t>(tc_smem_bytes(a.ld_s, a.b_slot_bytes), 116 * 1024);
  if (smem > 227 * 1024) return set_error(PTTK_ENOTSUP, "tensor-core chain: ranks too large for shared memory");
  const int64_t ntiles = (N + TILE_M - 1) / TILE_M;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, sm_count());
  PTTK_PROF("chain_tc", s);
  auto launch = [&](auto kfn) -> pttk_status {
    PTTK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kfn<<<grid, NTHREADS, smem, s>>>(a);
    PTTK_CUDA(cudaGetLastError());
    return PTTK_OK;
  };
  if (bf16) return split ? launch(chain_tc_kernel<true, true>) : launch(chain_tc_kernel<true, false>);
  return split ? launch(chain_tc_kernel<false, true>) : launch(chain_tc_kernel<false, false>);
}

}  // namespace pttk
