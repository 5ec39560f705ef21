// Factor chain of Algorithm 2, Phase 3 on the 5th-generation tensor cores (tcgen05).
//
// One persistent launch builds both factors: a CTA (10 warps, one per SM) takes 128-point
// tiles of the source points, then of the target points. Chain step i computes
// S_out (128 x R_out) = A (128 x K) * Gs (K x R_out), K = n R_in, with
//   A[p, a + R_in j] = T_j(xhat_{p,i}) * S_in[p, a]
// generated by the generator warps (two threads per point row) straight into shared memory
// in the UMMA K-major layout, and Gs the oriented core, pre-laid out once per handle as
// per-chunk images in the same layout and fetched chunk by chunk by one cp.async.bulk (TMA)
// copy into a ring of NSLOT operand slots. The accumulator lives in tensor memory (TMEM,
// 128 lanes = points, N_pad columns); one lane of the MMA warp issues tcgen05.mma and commits
// to mbarriers; after the last chunk of a step the generator warps read the accumulator back
// with tcgen05.ld: into S_in (FP32, shared memory) for the next step, or, after the last step,
// into a shared-memory output tile that is copied to U/V with coalesced 16-byte stores (a
// tile's 128 rows are contiguous in the row-major output).
//
// Precision forms (FP32 accumulation throughout):
//   TF32   kind::tf32, operands rounded to TF32 (10-bit mantissa);
//   TF32X3 a = a_hi + a_lo, b = b_hi + b_lo (each TF32), D += a_hi b_hi + a_hi b_lo + a_lo b_hi;
//   BF16   kind::f16 with BF16 operands (7-bit mantissa);
//   BF16X3 the same split with BF16 parts;
//   FP16   kind::f16 with FP16 operands (10-bit mantissa, like TF32, at half the bytes);
//   FP16X3 the same split with FP16 parts.
// Core images are split from the FP64 cores; A is split after its FP32 product. FP16 has a
// narrow exponent range, so the FP16 forms scale by exact powers of two: each core image so
// that its largest entry is <= 2^14, and each step's A operand (folded into the basis values)
// by an a-priori bound on |S_in| (|S_out| <= max|S_in| times the largest column 1-norm of
// the core, since |T_j| <= 1); the FP32 accumulator is unscaled when read back. Small
// entries then lose only what lies below 2^-24 of 2^14, far under the form's rounding.
//
// Shared-memory operand layout (UMMA "no swizzle" K-major): 16-byte units, a core matrix is
// 8 rows x 16 bytes stored contiguously (128 B). Chunk of KCB bytes of K per row (64 or 128,
// a launch configuration): unit (row r, k-unit u) at byte (r / 8) * 8 KCB + u * 128 + (r % 8) * 16.
// Descriptor: leading (K-direction) byte offset 128, stride (M/N-direction) byte offset 8 KCB;
// one MMA consumes 32 bytes of K (8 TF32 or 16 BF16), so k-step s starts at +256 s.
//
// Waits: every mbarrier wait is bounded; on timeout the CTA records PTTK_ETIMEOUT in a device
// status word, stops issuing work, waits (bounded) for its outstanding copies and MMAs, frees
// its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "pttk_internal.cuh"

namespace pttk {

int oriented_core_dims(const pttk_tt* tt, bool source, int step, int* R_in, int* R_out, int* coord);
const void* oriented_core_ptr(const pttk_tt* tt, bool source, int k, bool fp64);

namespace {

constexpr int TILE_M = 128;

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
// try_wait with a suspend-time hint: the thread sleeps in hardware until the phase completes
// or about `ns` nanoseconds have passed, whichever comes first (the completion wakes it at
// once, so the hint costs no latency; it only spares the issue slots of repeated polls).
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
// Bounded wait for the completion of the phase with the given parity: gives up after ~2 s
// (2^32 SM clocks, or 2^24 polls of up to 0.1 ms each) or as soon as another thread of the CTA
// has raised the abort flag. Each poll suspends the thread in hardware until the phase
// completes (or the hint runs out), so no software sleep adds a wake-up delay to a hand-off.
__device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity, const volatile int* abort_flag) {
  const long long t0 = clock64();
  for (uint32_t i = 0; i < (1u << 24); ++i) {
    if (mbar_try_wait_hint(bar, parity, 100000u)) return true;
    if (*abort_flag || clock64() - t0 > (4ll << 30)) return false;
  }
  return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const volatile int* abort_flag) {
  return mbar_try_wait(bar, parity) || mbar_wait_slow(bar, parity, abort_flag);
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
// 16 consecutive TMEM columns of this warp's 32 lanes (one row per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// UMMA shared-memory descriptor: no swizzle, K-major; K-adjacent core matrices 128 B apart
// (leading byte offset), 8-row groups `sbo` bytes apart (stride byte offset).
__device__ __forceinline__ uint64_t smem_desc2(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;  // K-adjacent core matrices: 128 B apart
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;   // 8-row groups: sbo bytes apart
  d |= (uint64_t)1 << 46;
  return d;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Instruction descriptor: FP32 accumulator, A/B format (kind::tf32: TF32 = 2; kind::f16: FP16 = 0,
// BF16 = 1), K-major A and B.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t ab_format, int M, int N) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

struct TcStep {
  const uint8_t* img_hi;  // nchunks x (Npad x KCB)
  const uint8_t* img_lo;  // same, or null for single-product forms
  int nchunks, R_in, R_in_pad, R_out, Npad, coord;
  float lo, hi;           // box of the coordinate
  float a_scale;          // power of two applied to the A operand (folded into the basis)
  float out_scale;        // power of two that unscales the accumulator
};
// One launch builds both factors: work item i < T0 is tile i of the source points (side 0),
// item i >= T0 is tile i - T0 of the target points (side 1). Factor rows depend only on their
// own point, so a tile may span several instances of a batch.
struct TcArgs {
  TcStep st[2][3];
  int nsteps, n, d;
  // S of the first step: 1 (s0_coord < 0) or the basis vector T(xhat) of coordinate s0_coord
  // on [s0_lo, s0_hi] (the first two chain steps merged into one)
  int s0_coord[2];
  float s0_lo[2], s0_hi[2];
  int64_t N[2];
  int64_t T0, ntiles;
  const float* pts[2];
  float* out[2];
  int* status;
  int ld_s;               // row stride of S (floats, multiple of 4)
  int ld_seed;            // row stride of the first step's input (floats, multiple of 4)
  int acc1_col;           // TMEM column of the first step's accumulator when it has its own
  int tmem_cols;
  uint32_t b_slot_bytes;  // bytes reserved per B part per slot
  int region_col;         // chain_tce_kernel: TMEM column of accumulator region 1 (region 0 at 0)
};

constexpr int NGEN_WARPS = 16;             // A generators: NPART threads per point row
constexpr int NPART = NGEN_WARPS / 4;      // generator warps per TMEM lane quarter
constexpr int TC_THREADS = 64 + 32 * NGEN_WARPS;  // warp 0: TMA, warp 1: MMA, warps 2..17: A
constexpr int STAGE_COLS = 16;             // epilogue staging: 32 rows x 16 columns per warp
constexpr int STAGE_LD = STAGE_COLS + 1;   // its row stride (floats; odd: no bank conflicts)

// Launch configurations: bytes of K per row per chunk (KCB) and operand ring depth (NS).
// Operand formats of the tensor-core forms.
constexpr int FMT_TF32 = 0, FMT_BF16 = 1, FMT_FP16 = 2;
__host__ __device__ constexpr uint32_t fmt_code(int fmt) { return fmt == FMT_TF32 ? 2u : fmt == FMT_BF16 ? 1u : 0u; }

template <int FMT, bool SPLIT, int KCB_, int NS>
struct Cfg {
  static constexpr int KCB = KCB_;
  static constexpr int NSLOT = NS;
  static constexpr int PARTS = SPLIT ? 2 : 1;             // hi (and lo) operand parts
  static constexpr int E = FMT == FMT_TF32 ? 4 : 8;       // elements per 16-byte unit
  static constexpr int UNITS = KCB / 16;                  // units per row per chunk
  static constexpr int KC = KCB / (FMT == FMT_TF32 ? 4 : 2);  // K elements per chunk
  static constexpr uint32_t SBO = 8 * KCB;                // 8-row group stride
  static constexpr uint32_t A_PART = TILE_M * KCB;
  static constexpr int KSTEPS = KCB / 32;                 // MMAs (per product) per chunk
};

// 16-byte unit of the generated A operand from E consecutive S values times one basis value.
template <int FMT, bool SPLIT>
__device__ __forceinline__ void write_unit(float b, const float* sv, uint8_t* hi, uint8_t* lo) {
  if constexpr (FMT == FMT_TF32) {
    const float4 x = *reinterpret_cast<const float4*>(sv);
    const float v[4] = {b * x.x, b * x.y, b * x.z, b * x.w};
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      h[e] = to_tf32(v[e]);
      if (SPLIT) l[e] = to_tf32(v[e] - h[e]);
    }
    *reinterpret_cast<float4*>(hi) = make_float4(h[0], h[1], h[2], h[3]);
    if (SPLIT) *reinterpret_cast<float4*>(lo) = make_float4(l[0], l[1], l[2], l[3]);
  } else if constexpr (FMT == FMT_BF16) {
    const float4 x0 = *reinterpret_cast<const float4*>(sv);
    const float4 x1 = *reinterpret_cast<const float4*>(sv + 4);
    const float v[8] = {b * x0.x, b * x0.y, b * x0.z, b * x0.w, b * x1.x, b * x1.y, b * x1.z, b * x1.w};
    __nv_bfloat162 h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * e]), h1 = __float2bfloat16_rn(v[2 * e + 1]);
      h[e] = __halves2bfloat162(h0, h1);
      if (SPLIT)
        l[e] = __halves2bfloat162(__float2bfloat16_rn(v[2 * e] - __bfloat162float(h0)),
                                  __float2bfloat16_rn(v[2 * e + 1] - __bfloat162float(h1)));
    }
    *reinterpret_cast<uint4*>(hi) = *reinterpret_cast<uint4*>(h);
    if (SPLIT) *reinterpret_cast<uint4*>(lo) = *reinterpret_cast<uint4*>(l);
  } else {
    const float4 x0 = *reinterpret_cast<const float4*>(sv);
    const float4 x1 = *reinterpret_cast<const float4*>(sv + 4);
    const float v[8] = {b * x0.x, b * x0.y, b * x0.z, b * x0.w, b * x1.x, b * x1.y, b * x1.z, b * x1.w};
    __half2 h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      h[e] = __floats2half2_rn(v[2 * e], v[2 * e + 1]);
      if (SPLIT) {
        const float2 hf = __half22float2(h[e]);
        l[e] = __floats2half2_rn(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
      }
    }
    *reinterpret_cast<uint4*>(hi) = *reinterpret_cast<uint4*>(h);
    if (SPLIT) *reinterpret_cast<uint4*>(lo) = *reinterpret_cast<uint4*>(l);
  }
}

__device__ __forceinline__ void gen_barrier() {  // the generator threads only
  asm volatile("bar.sync 1, %0;" ::"n"(32 * NGEN_WARPS) : "memory");
}

// Per-step constants, staged once in shared memory.
struct StepS {
  const uint8_t* hi;
  const uint8_t* lo;
  uint32_t bytes;   // bytes of one chunk part (Npad x KCB)
  uint32_t idesc;
  int nchunks, R_in_pad, R_out, Npad, coord;
  float lo_box, hi_box, a_scale, out_scale;
};

// Warp-specialised factor chain over both sides. Warp 0 (one lane) loads the core chunks with
// TMA into an NSLOT-deep ring; warp 1 (one lane) issues the MMAs; warps 2..17 generate the A
// chunks (NPART = 4 threads per point row, each writing a quarter of the row's units: enough
// warps per scheduler to hide the shared-memory latency of the generation) and run the
// epilogues. Barriers per slot: full_a (8 generator warps arrive), full_b (TMA transaction
// bytes), empty (tcgen05.commit of the slot's MMAs); acc_ready is committed after each step's
// last chunk.
template <int FMT, bool SPLIT, int KCB_, int NS>
__global__ void __launch_bounds__(TC_THREADS, 1) chain_tc_kernel(TcArgs a) {
  using C = Cfg<FMT, SPLIT, KCB_, NS>;
  constexpr int NSLOT = C::NSLOT;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int bv_ld = (a.n + 1) | 1;                                   // odd row stride > n
  uint8_t* a_base = smem;                                            // NSLOT x PARTS x A_PART
  uint8_t* b_base = a_base + (size_t)NSLOT * C::PARTS * C::A_PART;    // NSLOT x PARTS x b_slot_bytes
  float* S = reinterpret_cast<float*>(b_base + (size_t)NSLOT * C::PARTS * a.b_slot_bytes);  // 128 x ld_s
  float* Bv = S + (size_t)TILE_M * a.ld_s;                           // 2 x 128 x bv_ld
  float* Sseed = Bv + (size_t)2 * TILE_M * bv_ld;                     // 128 x ld_seed: step 0's input
  StepS* steps = reinterpret_cast<StepS*>(
      (reinterpret_cast<uintptr_t>(Sseed + (size_t)TILE_M * a.ld_seed) + 15) & ~uintptr_t(15));  // [2][3]
  uint64_t* bars = reinterpret_cast<uint64_t*>(steps + 6);
  uint64_t* full_a = bars;
  uint64_t* full_b = bars + NSLOT;
  uint64_t* empty = bars + 2 * NSLOT;
  uint64_t* acc_ready = bars + 3 * NSLOT;  // [0]: accumulator 0, [1]: the first step's own
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * NSLOT + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* stage = S;  // epilogue staging of the last step aliases S (8 x 32 x STAGE_LD floats)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < NSLOT; ++i) {
      mbar_init(&full_a[i], NGEN_WARPS);
      mbar_init(&full_b[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&acc_ready[0], 1);
    mbar_init(&acc_ready[1], 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (tid < 2 * a.nsteps) {
    const int sd = tid / a.nsteps, si = tid % a.nsteps;
    const TcStep& st = a.st[sd][si];
    StepS v;
    v.hi = st.img_hi;
    v.lo = st.img_lo;
    v.bytes = (uint32_t)st.Npad * C::KCB;
    v.idesc = instr_desc(fmt_code(FMT), TILE_M, st.Npad);
    v.nchunks = st.nchunks;
    v.R_in_pad = st.R_in_pad;
    v.R_out = st.R_out;
    v.Npad = st.Npad;
    v.coord = st.coord;
    v.lo_box = st.lo;
    v.hi_box = st.hi;
    v.a_scale = st.a_scale;
    v.out_scale = st.out_scale;
    steps[sd * 3 + si] = v;
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, (uint32_t)a.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t ntiles = a.ntiles;
  const int nsteps = a.nsteps;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t h = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < ntiles && ok; it += gridDim.x) {
        const int sd = it >= a.T0 ? 1 : 0;
        for (int si = 0; si < nsteps && ok; ++si) {
          const StepS st = steps[sd * 3 + si];
          for (int c = 0; c < st.nchunks; ++c, ++h) {
            const uint32_t slot = h % NSLOT;
            if (h >= NSLOT && !mbar_wait(&empty[slot], ((h / NSLOT) - 1) & 1, abort_flag)) { ok = false; break; }
            uint8_t* bh = b_base + (size_t)slot * C::PARTS * a.b_slot_bytes;
            fence_proxy_async();
            mbar_arrive_expect_tx(&full_b[slot], SPLIT ? 2 * st.bytes : st.bytes);
            tma_load_1d(bh, st.hi + (size_t)c * st.bytes, st.bytes, &full_b[slot]);
            if (SPLIT) tma_load_1d(bh + a.b_slot_bytes, st.lo + (size_t)c * st.bytes, st.bytes, &full_b[slot]);
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(a.status, (int)PTTK_ETIMEOUT);
      }
      // drain: every issued load has landed before the CTA may exit
      const int zero = 0;
      for (uint32_t k = (h > (uint32_t)NSLOT ? h - NSLOT : 0); k < h; ++k)
        mbar_wait(&full_b[k % NSLOT], (k / NSLOT) & 1, &zero);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < ntiles && ok; it += gridDim.x) {
        const int sd = it >= a.T0 ? 1 : 0;
        for (int si = 0; si < nsteps && ok; ++si) {
          const StepS st = steps[sd * 3 + si];
          // the first step has its own accumulator when there are later steps
          const int ab = (si == 0 && nsteps > 1) ? 1 : 0;
          const uint32_t dacc = tmem + (ab ? (uint32_t)a.acc1_col : 0u);
          for (int c = 0; c < st.nchunks; ++c, ++g) {
            const uint32_t slot = g % NSLOT, par = (g / NSLOT) & 1;
            if (!mbar_wait(&full_a[slot], par, abort_flag) || !mbar_wait(&full_b[slot], par, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(a_base + (size_t)slot * C::PARTS * C::A_PART);
            const uint32_t sb = smem_u32(b_base + (size_t)slot * C::PARTS * a.b_slot_bytes);
#pragma unroll
            for (int k = 0; k < C::KSTEPS; ++k) {
              const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
              const uint64_t ah = smem_desc2(sa + k * 256, C::SBO), bh = smem_desc2(sb + k * 256, C::SBO);
              if constexpr (FMT != FMT_TF32) {
                umma_f16(dacc, ah, bh, st.idesc, acc);
                if (SPLIT) {
                  umma_f16(dacc, ah, smem_desc2(sb + a.b_slot_bytes + k * 256, C::SBO), st.idesc, 1u);
                  umma_f16(dacc, smem_desc2(sa + C::A_PART + k * 256, C::SBO), bh, st.idesc, 1u);
                }
              } else {
                umma_tf32(dacc, ah, bh, st.idesc, acc);
                if (SPLIT) {
                  umma_tf32(dacc, ah, smem_desc2(sb + a.b_slot_bytes + k * 256, C::SBO), st.idesc, 1u);
                  umma_tf32(dacc, smem_desc2(sa + C::A_PART + k * 256, C::SBO), bh, st.idesc, 1u);
                }
              }
            }
            umma_commit(&empty[slot]);
            if (c == st.nchunks - 1) umma_commit(&acc_ready[ab]);
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(a.status, (int)PTTK_ETIMEOUT);
      }
      const int zero = 0;
      if (g > 0) mbar_wait(&empty[(g - 1) % NSLOT], ((g - 1) / NSLOT) & 1, &zero);
    }
    __syncwarp();
  } else {
    // ---------------- generator warps: A chunks and epilogues ----------------
    // Every generator thread runs the same sequence of named barriers whatever happens: a wait
    // that gives up only marks the warp dead (warp-uniform), after which its work is skipped.
    const int gw = warp - 2;                   // 0..NGEN_WARPS-1
    const int row = 32 * (warp & 3) + lane;    // TMEM lane quarter of this warp
    const int part = gw >> 2;                  // which part of the row's units
    uint32_t g = 0;
    bool dead = false;
    // basis of step si of side sd into Bv buffer `buf` (threads of part 0; zero from index n on)
    auto basis = [&](int sd, int si, int buf, float x) {
      const StepS& st = steps[sd * 3 + si];
      const float xh = (2.f * x - st.lo_box - st.hi_box) / (st.lo_box - st.hi_box);
      float* bv = Bv + ((size_t)buf * TILE_M + row) * bv_ld;
      const float sc = st.a_scale;
      float t0 = 1.f, t1 = xh;
      bv[0] = sc;
      for (int k = 1; k < a.n; ++k) {
        bv[k] = t1 * sc;
        const float t2 = 2.f * xh * t1 - t0;
        t0 = t1;
        t1 = t2;
      }
      for (int k = a.n; k < bv_ld; ++k) bv[k] = 0.f;
    };
    auto coord_of = [&](int64_t it, int si) -> float {
      const int sd = it >= a.T0 ? 1 : 0;
      const int64_t gp = (sd ? it - a.T0 : it) * TILE_M + row;
      const StepS& st = steps[sd * 3 + si];
      return gp < a.N[sd] ? a.pts[sd][gp * a.d + st.coord] : st.lo_box;
    };
    // coordinate of the seed basis (merged first steps) of this row in item `it`
    auto seed_coord_of = [&](int64_t it) -> float {
      const int sd = it >= a.T0 ? 1 : 0;
      const int64_t gp = (sd ? it - a.T0 : it) * TILE_M + row;
      return (a.s0_coord[sd] >= 0 && gp < a.N[sd]) ? a.pts[sd][gp * a.d + a.s0_coord[sd]] : a.s0_lo[sd];
    };
    // input of the first step for item `it` into Sseed (threads of part 0): the seed basis
    // T_0..T_{n-1}(xhat) of the merged first steps, or S_0 = 1; zero padding
    auto write_seed = [&](int64_t it, float x) {
      const int sd = it >= a.T0 ? 1 : 0;
      float* w = Sseed + (size_t)row * a.ld_seed;
      const int pad = steps[sd * 3].R_in_pad;
      if (a.s0_coord[sd] >= 0) {
        const float lo = a.s0_lo[sd], hi = a.s0_hi[sd];
        const float xh = (2.f * x - lo - hi) / (lo - hi);
        float t0 = 1.f, t1 = xh;
        w[0] = 1.f;
        for (int k = 1; k < pad; ++k) {
          w[k] = k < a.n ? t1 : 0.f;
          const float t2 = 2.f * xh * t1 - t0;
          t0 = t1;
          t1 = t2;
        }
      } else {
        w[0] = 1.f;
        for (int k = 1; k < pad; ++k) w[k] = 0.f;
      }
    };
    // output rows of the last step of item (osd, orow0, orows) from accumulator 0: each warp
    // stages 32 rows x 16 columns, then writes two row segments of 16 columns per store
    auto write_output = [&](int osd, int64_t orow0, int orows, uint32_t lane_addr) {
      const StepS& st = steps[osd * 3 + nsteps - 1];
      float* stg = stage + (size_t)gw * 32 * STAGE_LD;
      const int R = st.R_out;
      float* outbase = a.out[osd] + (orow0 + 32 * (warp & 3)) * R;
      const int wrows = std::max(0, std::min(32, orows - 32 * (warp & 3)));
      const int sub = lane >> 4, lc = lane & 15;
      for (int cb = STAGE_COLS * part; cb < st.Npad; cb += STAGE_COLS * NPART) {
        float v[STAGE_COLS];
        tmem_ld16(lane_addr + (uint32_t)cb, v);
#pragma unroll
        for (int i = 0; i < STAGE_COLS; ++i) stg[lane * STAGE_LD + i] = v[i] * st.out_scale;
        __syncwarp();
        const int col = cb + lc;
        if (col < R)
          for (int rr = sub; rr < wrows; rr += 2) outbase[(int64_t)rr * R + col] = stg[rr * STAGE_LD + lc];
        __syncwarp();
      }
    };
    // Each accumulator barrier completes one phase per step that uses it; a waiter is never
    // more than one phase behind, because the next step on that accumulator needs chunks that
    // are generated only after the wait.
    uint32_t done_acc[2] = {0u, 0u};
    auto wait_acc = [&](int ab) {
      if (!dead && !*abort_flag) dead = !mbar_wait(&acc_ready[ab], done_acc[ab] & 1, abort_flag);
      ++done_acc[ab];
      dead = __any_sync(0xffffffffu, dead || *abort_flag);
      if (dead && lane == 0) *abort_flag = 1;
      tc_fence_after();
    };
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    // With two or more steps the last step's output is written after the next item's first
    // step has been generated: the tensor cores run that step (into its own accumulator)
    // while the output leaves.
    const bool defer = nsteps > 1;
    // coordinates of this row for the next tile to build; xn[3]: the seed coordinate
    float xn[4] = {0.f, 0.f, 0.f, 0.f};
    if (part == 0 && blockIdx.x < ntiles) {
      #pragma unroll
      for (int si = 0; si < 3; ++si)
        if (si < nsteps) xn[si] = coord_of(blockIdx.x, si);
      xn[3] = seed_coord_of(blockIdx.x);
      basis(blockIdx.x >= a.T0 ? 1 : 0, 0, 0, xn[0]);
      write_seed(blockIdx.x, xn[3]);
    }
    gen_barrier();
    uint32_t bufsel = 0;
    bool out_pending = false;
    int out_sd = 0, out_rows = 0;
    int64_t out_row0 = 0;
    for (int64_t it = blockIdx.x; it < ntiles; it += gridDim.x) {
      const int sd = it >= a.T0 ? 1 : 0;
      const int64_t row0 = (sd ? it - a.T0 : it) * TILE_M;
      const int rows = (int)std::min<int64_t>(TILE_M, a.N[sd] - row0);
      const float xcur1 = xn[1], xcur2 = xn[2];
      const int64_t itn = it + gridDim.x;  // next item: prefetch its coordinates
      if (part == 0 && itn < ntiles) {
        #pragma unroll
        for (int si = 0; si < 3; ++si)
          if (si < nsteps) xn[si] = coord_of(itn, si);
        xn[3] = seed_coord_of(itn);
      }
      for (int si = 0; si < nsteps; ++si) {
        const StepS st = steps[sd * 3 + si];
        const float* bvrow = Bv + ((size_t)bufsel * TILE_M + row) * bv_ld;
        const float* srow = si == 0 ? Sseed + (size_t)row * a.ld_seed : S + (size_t)row * a.ld_s;
        for (int c = 0; c < st.nchunks; ++c, ++g) {
          const uint32_t slot = g % NSLOT, use = g / NSLOT;
          dead = dead || *abort_flag;
          if (!dead && g >= (uint32_t)NSLOT) dead = !mbar_wait(&empty[slot], (use - 1) & 1, abort_flag);
          dead = __any_sync(0xffffffffu, dead);
          if (dead && lane == 0) *abort_flag = 1;
          if (!dead) {
            uint8_t* ah = a_base + (size_t)slot * C::PARTS * C::A_PART;
            const uint32_t row_off = (uint32_t)(row >> 3) * C::SBO + (uint32_t)(row & 7) * 16;
            constexpr int UH = C::UNITS / NPART;  // units of this thread
            static_assert(C::UNITS % NPART == 0, "units per chunk row must split evenly");
            const int k = c * C::KC + part * UH * C::E;
            int j = k / st.R_in_pad;
            int ai = k - j * st.R_in_pad;
#pragma unroll
            for (int u = 0; u < UH; ++u) {
              const uint32_t off = row_off + (uint32_t)(part * UH + u) * 128;
              write_unit<FMT, SPLIT>(bvrow[j < a.n ? j : a.n], srow + ai, ah + off, ah + C::A_PART + off);
              ai += C::E;
              if (ai == st.R_in_pad) {
                ai = 0;
                ++j;
              }
            }
            fence_proxy_async();
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&full_a[slot]);
        }
        // the next basis (next step, or step 0 of the next item) goes to the other buffer
        // while this step's MMAs drain
        const bool last = si == nsteps - 1;
        if (part == 0) {
          if (!last) basis(sd, si + 1, bufsel ^ 1, si == 0 ? xcur1 : xcur2);
          else if (itn < ntiles) basis(itn >= a.T0 ? 1 : 0, 0, bufsel ^ 1, xn[0]);
        }
        if (si == 0 && out_pending) {
          // the previous item's output, while this item's first step runs; its staging aliases
          // S, which the epilogue below writes, hence the barrier
          wait_acc(0);
          if (!dead) write_output(out_sd, out_row0, out_rows, tmem + lanes);
          out_pending = false;
          gen_barrier();
        }
        if (last && defer && itn < ntiles) {
          // this item's output is written during the next item's first step; the first
          // step's input of the next item goes to Sseed (its last reader was step 0 of this
          // item, finished before the barrier that ended step 0)
          out_pending = true;
          out_sd = sd;
          out_row0 = row0;
          out_rows = rows;
          if (part == 0) write_seed(itn, xn[3]);
          bufsel ^= 1;
          tc_fence_before();
          gen_barrier();
          continue;
        }
        // accumulator of this step is complete (all A chunks of the step, hence all reads of
        // its input, are done once it is)
        const int ab = (si == 0 && defer) ? 1 : 0;
        wait_acc(ab);
        const uint32_t lane_addr = tmem + lanes + (ab ? (uint32_t)a.acc1_col : 0u);
        if (!last) {
          // S for the next step: columns [0, Npad) (zero beyond R_out); this thread's share of
          // the 32-column blocks
          if (!dead)
            for (int cb = 32 * part; cb < st.Npad; cb += 32 * NPART) {
              float v[32];
              tmem_ld32(lane_addr + (uint32_t)cb, v);
              float* dst = S + (size_t)row * a.ld_s + cb;
              const float osc = st.out_scale;
#pragma unroll
              for (int i = 0; i < 32; i += 4)
                if (cb + i < a.ld_s)
                  *reinterpret_cast<float4*>(dst + i) =
                      make_float4(v[i] * osc, v[i + 1] * osc, v[i + 2] * osc, v[i + 3] * osc);
            }
        } else if (!dead) {
          write_output(sd, row0, rows, lane_addr);
        }
        bufsel ^= 1;
        tc_fence_before();
        gen_barrier();
        if (last && !defer && itn < ntiles) {
          // a single step: its input is read until the barrier above
          if (part == 0) write_seed(itn, xn[3]);
          gen_barrier();
        }
      }
    }
    if (dead && lane == 0) {
      *abort_flag = 1;
      atomicExch(a.status, (int)PTTK_ETIMEOUT);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

// ---------------- dedicated epilogue warps, double-buffered accumulators ------------------
// The same chain with the output written by four epilogue warps of their own (one per TMEM lane
// quarter) from one of two accumulator regions, while the MMAs of the next tile fill the other:
// a tile's steps all accumulate into region (tile parity), the first step's result being read
// back as the second step's input before the second step's first MMA overwrites it. The
// generators then never wait for a tile's last step and never write output; the output of a
// tile leaves while the next tile is computed.
// Barriers: full_a / full_b / empty per ring slot as in chain_tc_kernel; mid[r] (committed after
// the last chunk of every step but the last into region r; the generators wait for each in
// turn), last[r] (committed after a tile's last step; the epilogue waits for it), free[r] (the
// four epilogue warps arrive once they have read region r; the MMA lane waits for it before the
// first MMA of the next tile in region r). Each barrier has one kind of waiter that can fall at
// most one phase behind, which is what a parity wait needs.
constexpr int NEPI_WARPS = 4;
constexpr int TCE_THREADS = 64 + 32 * NGEN_WARPS + 32 * NEPI_WARPS;

template <int FMT, bool SPLIT, int KCB_, int NS>
__global__ void __launch_bounds__(TCE_THREADS, 1) chain_tce_kernel(TcArgs a) {
  using C = Cfg<FMT, SPLIT, KCB_, NS>;
  constexpr int NSLOT = C::NSLOT;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int bv_ld = (a.n + 1) | 1;
  uint8_t* a_base = smem;                                            // NSLOT x PARTS x A_PART
  uint8_t* b_base = a_base + (size_t)NSLOT * C::PARTS * C::A_PART;    // NSLOT x PARTS x b_slot_bytes
  float* S = reinterpret_cast<float*>(b_base + (size_t)NSLOT * C::PARTS * a.b_slot_bytes);  // 128 x ld_s
  float* Bv = S + (size_t)TILE_M * a.ld_s;                           // 2 x 128 x bv_ld
  float* Sseed = Bv + (size_t)2 * TILE_M * bv_ld;                     // 128 x ld_seed
  float* stage = Sseed + (size_t)TILE_M * a.ld_seed;                  // NEPI_WARPS x 32 x STAGE_LD
  StepS* steps = reinterpret_cast<StepS*>(
      (reinterpret_cast<uintptr_t>(stage + (size_t)NEPI_WARPS * 32 * STAGE_LD) + 15) & ~uintptr_t(15));  // [2][3]
  uint64_t* bars = reinterpret_cast<uint64_t*>(steps + 6);
  uint64_t* full_a = bars;
  uint64_t* full_b = bars + NSLOT;
  uint64_t* empty = bars + 2 * NSLOT;
  uint64_t* mid = bars + 3 * NSLOT;        // [2]
  uint64_t* last_done = bars + 3 * NSLOT + 2;  // [2]
  uint64_t* rfree = bars + 3 * NSLOT + 4;  // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * NSLOT + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < NSLOT; ++i) {
      mbar_init(&full_a[i], NGEN_WARPS);
      mbar_init(&full_b[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int r = 0; r < 2; ++r) {
      mbar_init(&mid[r], 1);
      mbar_init(&last_done[r], 1);
      mbar_init(&rfree[r], NEPI_WARPS);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (tid < 2 * a.nsteps) {
    const int sd = tid / a.nsteps, si = tid % a.nsteps;
    const TcStep& st = a.st[sd][si];
    StepS v;
    v.hi = st.img_hi;
    v.lo = st.img_lo;
    v.bytes = (uint32_t)st.Npad * C::KCB;
    v.idesc = instr_desc(fmt_code(FMT), TILE_M, st.Npad);
    v.nchunks = st.nchunks;
    v.R_in_pad = st.R_in_pad;
    v.R_out = st.R_out;
    v.Npad = st.Npad;
    v.coord = st.coord;
    v.lo_box = st.lo;
    v.hi_box = st.hi;
    v.a_scale = st.a_scale;
    v.out_scale = st.out_scale;
    steps[sd * 3 + si] = v;
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, (uint32_t)a.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t ntiles = a.ntiles;
  const int nsteps = a.nsteps;
  auto region_addr = [&](uint32_t r) { return tmem + (r ? (uint32_t)a.region_col : 0u); };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t h = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < ntiles && ok; it += gridDim.x) {
        const int sd = it >= a.T0 ? 1 : 0;
        for (int si = 0; si < nsteps && ok; ++si) {
          const StepS& st = steps[sd * 3 + si];
          for (int c = 0; c < st.nchunks; ++c, ++h) {
            const uint32_t slot = h % NSLOT;
            if (h >= NSLOT && !mbar_wait(&empty[slot], ((h / NSLOT) - 1) & 1, abort_flag)) { ok = false; break; }
            uint8_t* bh = b_base + (size_t)slot * C::PARTS * a.b_slot_bytes;
            fence_proxy_async();
            mbar_arrive_expect_tx(&full_b[slot], SPLIT ? 2 * st.bytes : st.bytes);
            tma_load_1d(bh, st.hi + (size_t)c * st.bytes, st.bytes, &full_b[slot]);
            if (SPLIT) tma_load_1d(bh + a.b_slot_bytes, st.lo + (size_t)c * st.bytes, st.bytes, &full_b[slot]);
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(a.status, (int)PTTK_ETIMEOUT);
      }
      const int zero = 0;
      for (uint32_t k = (h > (uint32_t)NSLOT ? h - NSLOT : 0); k < h; ++k)
        mbar_wait(&full_b[k % NSLOT], (k / NSLOT) & 1, &zero);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t g = 0, tile = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < ntiles && ok; it += gridDim.x, ++tile) {
        const int sd = it >= a.T0 ? 1 : 0;
        const uint32_t r = tile & 1, use = tile >> 1;
        // the region's previous tile must have left it
        if (use >= 1 && !mbar_wait(&rfree[r], (use - 1) & 1, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t dacc = region_addr(r);
        for (int si = 0; si < nsteps && ok; ++si) {
          const StepS& st = steps[sd * 3 + si];
          for (int c = 0; c < st.nchunks; ++c, ++g) {
            const uint32_t slot = g % NSLOT, par = (g / NSLOT) & 1;
            if (!mbar_wait(&full_a[slot], par, abort_flag) || !mbar_wait(&full_b[slot], par, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(a_base + (size_t)slot * C::PARTS * C::A_PART);
            const uint32_t sb = smem_u32(b_base + (size_t)slot * C::PARTS * a.b_slot_bytes);
            const uint64_t ah0 = smem_desc2(sa, C::SBO), al0 = smem_desc2(sa + C::A_PART, C::SBO);
            const uint64_t bh0 = smem_desc2(sb, C::SBO), bl0 = smem_desc2(sb + a.b_slot_bytes, C::SBO);
#pragma unroll
            for (int k = 0; k < C::KSTEPS; ++k) {
              const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
              // +256 bytes of K per MMA: +16 in the descriptors' address fields
              const uint64_t ah = ah0 + (uint64_t)(16 * k), bh = bh0 + (uint64_t)(16 * k);
              if constexpr (FMT != FMT_TF32) {
                umma_f16(dacc, ah, bh, st.idesc, acc);
                if (SPLIT) {
                  umma_f16(dacc, ah, bl0 + (uint64_t)(16 * k), st.idesc, 1u);
                  umma_f16(dacc, al0 + (uint64_t)(16 * k), bh, st.idesc, 1u);
                }
              } else {
                umma_tf32(dacc, ah, bh, st.idesc, acc);
                if (SPLIT) {
                  umma_tf32(dacc, ah, bl0 + (uint64_t)(16 * k), st.idesc, 1u);
                  umma_tf32(dacc, al0 + (uint64_t)(16 * k), bh, st.idesc, 1u);
                }
              }
            }
            umma_commit(&empty[slot]);
            if (c == st.nchunks - 1) umma_commit(si == nsteps - 1 ? &last_done[r] : &mid[r]);
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(a.status, (int)PTTK_ETIMEOUT);
      }
      const int zero = 0;
      if (g > 0) mbar_wait(&empty[(g - 1) % NSLOT], ((g - 1) / NSLOT) & 1, &zero);
    }
    __syncwarp();
  } else if (warp < 2 + NGEN_WARPS) {
    // ---------------- generator warps: A chunks ----------------
    const int gw = warp - 2;
    const int row = 32 * (warp & 3) + lane;
    const int part = gw >> 2;
    uint32_t g = 0, tile = 0;
    bool dead = false;
    auto basis = [&](int sd, int si, int buf, float x) {
      const StepS& st = steps[sd * 3 + si];
      const float xh = (2.f * x - st.lo_box - st.hi_box) / (st.lo_box - st.hi_box);
      float* bv = Bv + ((size_t)buf * TILE_M + row) * bv_ld;
      const float sc = st.a_scale;
      float t0 = 1.f, t1 = xh;
      bv[0] = sc;
      for (int k = 1; k < a.n; ++k) {
        bv[k] = t1 * sc;
        const float t2 = 2.f * xh * t1 - t0;
        t0 = t1;
        t1 = t2;
      }
      for (int k = a.n; k < bv_ld; ++k) bv[k] = 0.f;
    };
    auto coord_of = [&](int64_t it, int si) -> float {
      const int sd = it >= a.T0 ? 1 : 0;
      const int64_t gp = (sd ? it - a.T0 : it) * TILE_M + row;
      const StepS& st = steps[sd * 3 + si];
      return gp < a.N[sd] ? a.pts[sd][gp * a.d + st.coord] : st.lo_box;
    };
    auto seed_coord_of = [&](int64_t it) -> float {
      const int sd = it >= a.T0 ? 1 : 0;
      const int64_t gp = (sd ? it - a.T0 : it) * TILE_M + row;
      return (a.s0_coord[sd] >= 0 && gp < a.N[sd]) ? a.pts[sd][gp * a.d + a.s0_coord[sd]] : a.s0_lo[sd];
    };
    auto write_seed = [&](int64_t it, float x) {
      const int sd = it >= a.T0 ? 1 : 0;
      float* w = Sseed + (size_t)row * a.ld_seed;
      const int pad = steps[sd * 3].R_in_pad;
      if (a.s0_coord[sd] >= 0) {
        const float lo = a.s0_lo[sd], hi = a.s0_hi[sd];
        const float xh = (2.f * x - lo - hi) / (lo - hi);
        float t0 = 1.f, t1 = xh;
        w[0] = 1.f;
        for (int k = 1; k < pad; ++k) {
          w[k] = k < a.n ? t1 : 0.f;
          const float t2 = 2.f * xh * t1 - t0;
          t0 = t1;
          t1 = t2;
        }
      } else {
        w[0] = 1.f;
        for (int k = 1; k < pad; ++k) w[k] = 0.f;
      }
    };
    // the coordinates of the next tile are loaded one tile ahead into registers (constant
    // indices only: a runtime-indexed array would sit in local memory, and the store into it
    // would wait for the global load at once)
    float xn[4] = {0.f, 0.f, 0.f, 0.f};
    if (part == 0 && blockIdx.x < ntiles) {
#pragma unroll
      for (int si = 0; si < 3; ++si)
        if (si < nsteps) xn[si] = coord_of(blockIdx.x, si);
      xn[3] = seed_coord_of(blockIdx.x);
      basis(blockIdx.x >= a.T0 ? 1 : 0, 0, 0, xn[0]);
      write_seed(blockIdx.x, xn[3]);
    }
    gen_barrier();
    uint32_t bufsel = 0;
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    for (int64_t it = blockIdx.x; it < ntiles; it += gridDim.x, ++tile) {
      const int sd = it >= a.T0 ? 1 : 0;
      const uint32_t r = tile & 1, use = tile >> 1;
      const float xcur1 = xn[1], xcur2 = xn[2];
      const int64_t itn = it + gridDim.x;
      if (part == 0 && itn < ntiles) {
#pragma unroll
        for (int si = 0; si < 3; ++si)
          if (si < nsteps) xn[si] = coord_of(itn, si);
        xn[3] = seed_coord_of(itn);
      }
      for (int si = 0; si < nsteps; ++si) {
        const StepS st = steps[sd * 3 + si];
        const float* bvrow = Bv + ((size_t)bufsel * TILE_M + row) * bv_ld;
        const float* srow = si == 0 ? Sseed + (size_t)row * a.ld_seed : S + (size_t)row * a.ld_s;
        for (int c = 0; c < st.nchunks; ++c, ++g) {
          const uint32_t slot = g % NSLOT, use_s = g / NSLOT;
          dead = dead || *abort_flag;
          if (!dead && g >= (uint32_t)NSLOT) dead = !mbar_wait(&empty[slot], (use_s - 1) & 1, abort_flag);
          dead = __any_sync(0xffffffffu, dead);
          if (dead && lane == 0) *abort_flag = 1;
          if (!dead) {
            uint8_t* ah = a_base + (size_t)slot * C::PARTS * C::A_PART;
            const uint32_t row_off = (uint32_t)(row >> 3) * C::SBO + (uint32_t)(row & 7) * 16;
            constexpr int UH = C::UNITS / NPART;
            static_assert(C::UNITS % NPART == 0, "units per chunk row must split evenly");
            const int k = c * C::KC + part * UH * C::E;
            int j = k / st.R_in_pad;
            int ai = k - j * st.R_in_pad;
#pragma unroll
            for (int u = 0; u < UH; ++u) {
              const uint32_t off = row_off + (uint32_t)(part * UH + u) * 128;
              write_unit<FMT, SPLIT>(bvrow[j < a.n ? j : a.n], srow + ai, ah + off, ah + C::A_PART + off);
              ai += C::E;
              if (ai == st.R_in_pad) {
                ai = 0;
                ++j;
              }
            }
            fence_proxy_async();
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&full_a[slot]);
        }
        const bool last = si == nsteps - 1;
        if (part == 0) {
          if (!last) basis(sd, si + 1, bufsel ^ 1, si == 0 ? xcur1 : xcur2);
          else if (itn < ntiles) basis(itn >= a.T0 ? 1 : 0, 0, bufsel ^ 1, xn[0]);
        }
        if (!last) {
          // this step's result is the next step's input: wait for it and copy it to S
          const uint32_t phase = use * (uint32_t)(nsteps - 1) + (uint32_t)si;
          if (!dead && !*abort_flag) dead = !mbar_wait(&mid[r], phase & 1, abort_flag);
          dead = __any_sync(0xffffffffu, dead || *abort_flag);
          if (dead && lane == 0) *abort_flag = 1;
          tc_fence_after();
          if (!dead)
            for (int cb = 32 * part; cb < st.Npad; cb += 32 * NPART) {
              float v[32];
              tmem_ld32(region_addr(r) + lanes + (uint32_t)cb, v);
              float* dst = S + (size_t)row * a.ld_s + cb;
              const float osc = st.out_scale;
#pragma unroll
              for (int i = 0; i < 32; i += 4)
                if (cb + i < a.ld_s)
                  *reinterpret_cast<float4*>(dst + i) =
                      make_float4(v[i] * osc, v[i + 1] * osc, v[i + 2] * osc, v[i + 3] * osc);
            }
          tc_fence_before();
        } else if (itn < ntiles && part == 0 && nsteps > 1) {
          // the seed of the next tile (this tile's seed was last read by its first step, which
          // every thread finished before the barrier after that step)
          write_seed(itn, xn[3]);
        }
        bufsel ^= 1;
        gen_barrier();
        if (last && nsteps == 1 && itn < ntiles) {
          // a single step reads its seed until the barrier above
          if (part == 0) write_seed(itn, xn[3]);
          gen_barrier();
        }
      }
    }
    if (dead && lane == 0) {
      *abort_flag = 1;
      atomicExch(a.status, (int)PTTK_ETIMEOUT);
    }
  } else {
    // ---------------- epilogue warps: one TMEM lane quarter each ----------------
    const int ew = warp - 2 - NGEN_WARPS;      // 0..3
    const int quarter = warp & 3;
    const uint32_t lanes = (uint32_t)(32 * quarter) << 16;
    float* stg = stage + (size_t)ew * 32 * STAGE_LD;
    const int sub = lane >> 4, lc = lane & 15;
    uint32_t tile = 0;
    bool dead = false;
    for (int64_t it = blockIdx.x; it < ntiles; it += gridDim.x, ++tile) {
      const int sd = it >= a.T0 ? 1 : 0;
      const uint32_t r = tile & 1, use = tile >> 1;
      const StepS& st = steps[sd * 3 + nsteps - 1];
      if (!dead && !*abort_flag) dead = !mbar_wait(&last_done[r], use & 1, abort_flag);
      dead = __any_sync(0xffffffffu, dead || *abort_flag);
      if (dead && lane == 0) *abort_flag = 1;
      tc_fence_after();
      if (!dead) {
        const int64_t row0 = (sd ? it - a.T0 : it) * TILE_M;
        const int rows = (int)std::min<int64_t>(TILE_M, a.N[sd] - row0);
        const int R = st.R_out;
        float* outbase = a.out[sd] + (row0 + 32 * quarter) * R;
        const int wrows = std::max(0, std::min(32, rows - 32 * quarter));
        for (int cb = 0; cb < st.Npad; cb += STAGE_COLS) {
          float v[STAGE_COLS];
          tmem_ld16(region_addr(r) + lanes + (uint32_t)cb, v);
#pragma unroll
          for (int i = 0; i < STAGE_COLS; ++i) stg[lane * STAGE_LD + i] = v[i] * st.out_scale;
          __syncwarp();
          const int col = cb + lc;
          if (col < R)
            for (int rr = sub; rr < wrows; rr += 2) outbase[(int64_t)rr * R + col] = stg[rr * STAGE_LD + lc];
          __syncwarp();
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&rfree[r]);
    }
    if (dead && lane == 0) {
      *abort_flag = 1;
      atomicExch(a.status, (int)PTTK_ETIMEOUT);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

// ---------------- A operand in tensor memory ---------------------------------------------
// The second form of the chain kernel ("TS": A from tensor memory, B from shared memory), for
// the kind::f16 forms (FP16, BF16 and their split forms). Shared memory then carries only the
// core chunks: the generated A operand is written by the generator threads straight into
// TMEM with tcgen05.st, and the step input S_in stays in registers, read back from the
// previous step's accumulator with tcgen05.ld. In the shared-memory form every A chunk is
// written once and read by up to three MMAs, and every step reads S_in from shared memory,
// which together exceed what shared memory delivers per MMA clock.
//
// K order of a step: k = a + R_in_pad j (a < R_in_pad, R_in_pad a multiple of 16). Chunk c
// holds j in [c jpc, (c + 1) jpc), i.e. jpc R_in_pad values of K (about 64). TMEM layout of one
// A chunk part (kind::f16, M = 128): lane = point row, column = K pair (two 16-bit values per
// 32-bit column), so one MMA of K = 16 reads 8 columns. The four generator warps of a lane
// quarter split the a range: part p owns a in [p spt, (p + 1) spt), spt = R_in_pad / 4, and
// keeps S_in[row, p spt + i] for i < spt in registers.
__device__ __forceinline__ void umma_f16_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tmem_st1(uint32_t taddr, uint32_t v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(v) : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 16 single columns c0 .. c0 + 15 of this warp's 32 lanes, one load each, and the wait for
// them, in one block (so that no use of the values can be scheduled before the wait).
__device__ __forceinline__ void tmem_ld1x16(uint32_t c0, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%16];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%1}, [%17];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%2}, [%18];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%3}, [%19];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%4}, [%20];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%5}, [%21];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%6}, [%22];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%7}, [%23];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%8}, [%24];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%9}, [%25];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%10}, [%26];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%11}, [%27];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%12}, [%28];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%13}, [%29];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%14}, [%30];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%15}, [%31];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(c0), "r"(c0 + 1), "r"(c0 + 2), "r"(c0 + 3), "r"(c0 + 4), "r"(c0 + 5), "r"(c0 + 6), "r"(c0 + 7),
        "r"(c0 + 8), "r"(c0 + 9), "r"(c0 + 10), "r"(c0 + 11), "r"(c0 + 12), "r"(c0 + 13), "r"(c0 + 14),
        "r"(c0 + 15)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int TS_SPT = 16;  // largest a range per generator thread (R_in_pad <= 64)

// Per-step constants of the TS kernel, staged once in shared memory.
struct TsStepS {
  const uint8_t* hi;
  const uint8_t* lo;
  uint32_t bytes;   // bytes of one chunk part (Npad x kcb)
  uint32_t idesc;
  uint32_t sbo;     // 8-row group stride of a B chunk (8 kcb)
  int nchunks, jpc, R_in_pad, spt, R_out, Npad, coord, ksteps;
  float lo_box, hi_box, a_scale, out_scale;
};
struct TsArgs {
  TsStepS st[2][3];
  int nsteps, n, d;
  int s0_coord[2];
  float s0_lo[2], s0_hi[2];
  int64_t N[2];
  int64_t T0p;       // source tiles, padded to a multiple of the cluster size
  int64_t nitems;    // cluster items: CL consecutive tiles of one side each
  const float* pts[2];
  float* out[2];
  int* status;
  int ld_seed;       // row stride of the first step's input (odd)
  int bv_ld;         // row stride of the basis buffers (odd, > every step's nchunks jpc)
  int acc1_col;      // TMEM column of the first step's own accumulator (two or more steps)
  int a_col;         // TMEM column of A slot 0
  int a_part_cols;   // TMEM columns of one A part of a slot
  int region_col;    // columns of one accumulator region (tensor-memory-A kernel with epilogue warps)
  int tmem_cols;
  uint32_t b_slot_bytes;  // bytes reserved per B part per slot
};

// 16-bit pair of a generated A value pair: FP16 or BF16, and the residual's pair for the split
template <int FMT, bool SPLIT>
__device__ __forceinline__ void pack_pair(float v0, float v1, uint32_t& h, uint32_t& l) {
  if constexpr (FMT == FMT_BF16) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(v0, v1);
    h = *reinterpret_cast<const uint32_t*>(&hb);
    if (SPLIT) {
      const float2 hf = __bfloat1622float2(hb);
      const __nv_bfloat162 lb = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
      l = *reinterpret_cast<const uint32_t*>(&lb);
    }
  } else {
    const __half2 hh = __floats2half2_rn(v0, v1);
    h = *reinterpret_cast<const uint32_t*>(&hh);
    if (SPLIT) {
      const float2 hf = __half22float2(hh);
      const __half2 lh = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
      l = *reinterpret_cast<const uint32_t*>(&lh);
    }
  }
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// bulk copy of `bytes` from global memory to the same shared-memory offset in every CTA of the
// cluster named by `mask`, each destination's mbarrier (same offset) receiving the bytes
__device__ __forceinline__ void tma_load_1d_mc(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}
// arrive on the mbarrier at this offset in every CTA of `mask` once this thread's MMAs complete
__device__ __forceinline__ void umma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                   smem_u32(bar)),
               "h"(mask)
               : "memory");
}

// Warp roles as in chain_tc_kernel: warp 0 (one lane) streams core chunks into the NS-deep
// shared-memory ring with TMA, warp 1 (one lane) issues the MMAs, warps 2..17 generate A into
// the NS-deep TMEM ring and run the epilogues.
//
// Every 128-point tile streams the whole oriented core through shared memory, so at these
// ranks the core traffic from L2 rivals the MMA time. The CL CTAs of a thread-block cluster
// therefore work in lockstep on CL consecutive tiles of one side (a cluster item; each side's
// tile count is padded to a multiple of CL with empty tiles), and each CTA loads 1/CL of every
// core chunk with a multicast copy into all CL CTAs: the L2 traffic of the cores falls by CL.
// Barriers per slot: full_a (16 generator warps arrive after their tcgen05.st completed),
// full_b (the chunk's bytes from all CL copies), empty_a (the local MMAs of the slot completed:
// the TMEM slot may be rewritten), empty_b (the MMAs of the slot completed in every CTA of the
// cluster: the shared-memory slot, written by every CTA's copies, may be reloaded).
template <int FMT, bool SPLIT, int NS, int CL>
__global__ void __launch_bounds__(TC_THREADS, 1) chain_ts_kernel(TsArgs a) {
  constexpr int PARTS = SPLIT ? 2 : 1;
  constexpr uint16_t MASK = (uint16_t)((1u << CL) - 1u);
  extern __shared__ __align__(1024) uint8_t smem[];
  const int bv_ld = a.bv_ld;
  uint8_t* b_base = smem;                                                // NS x PARTS x b_slot_bytes
  float* Bv = reinterpret_cast<float*>(b_base + (size_t)NS * PARTS * a.b_slot_bytes);  // 2 x 128 x bv_ld
  float* Sseed = Bv + (size_t)2 * TILE_M * bv_ld;                        // 128 x ld_seed
  float* stage = Sseed + (size_t)TILE_M * a.ld_seed;                     // NGEN_WARPS x 32 x STAGE_LD
  TsStepS* steps = reinterpret_cast<TsStepS*>(
      (reinterpret_cast<uintptr_t>(stage + (size_t)NGEN_WARPS * 32 * STAGE_LD) + 15) & ~uintptr_t(15));  // [2][3]
  uint64_t* bars = reinterpret_cast<uint64_t*>(steps + 6);
  uint64_t* full_a = bars;
  uint64_t* full_b = bars + NS;
  uint64_t* empty_a = bars + 2 * NS;
  uint64_t* empty_b = bars + 3 * NS;
  uint64_t* acc_ready = bars + 4 * NS;  // [0]: accumulator 0, [1]: the first step's own
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4 * NS + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int crank = CL > 1 ? (int)cluster_rank() : 0;
  const int64_t cid = blockIdx.x / CL, ncl = gridDim.x / CL;
  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full_a[i], NGEN_WARPS);
      mbar_init(&full_b[i], 1);
      mbar_init(&empty_a[i], 1);
      mbar_init(&empty_b[i], CL);
    }
    mbar_init(&acc_ready[0], 1);
    mbar_init(&acc_ready[1], 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (tid < 2 * a.nsteps) steps[(tid / a.nsteps) * 3 + tid % a.nsteps] = a.st[tid / a.nsteps][tid % a.nsteps];
  if (warp == 1) {
    tmem_alloc(tmem_slot, (uint32_t)a.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (CL > 1) cluster_sync_all();  // every CTA's barriers exist before any copy or commit reaches them
  const uint32_t tmem = *tmem_slot;
  const int64_t nitems = a.nitems;
  const int nsteps = a.nsteps;
  // side, first row and row count of this CTA's tile in cluster item k
  auto item_side = [&](int64_t k) -> int { return k * CL < a.T0p ? 0 : 1; };
  auto item_row0 = [&](int64_t k) -> int64_t {
    const int sd = item_side(k);
    return (k * CL + crank - (sd ? a.T0p : 0)) * TILE_M;
  };

  if (warp == 0) {
    // ---------------- TMA producer: this CTA's share of every chunk, to every CTA ----------------
    if (lane == 0) {
      uint32_t h = 0;
      bool ok = true;
      for (int64_t it = cid; it < nitems && ok; it += ncl) {
        const int sd = item_side(it);
        for (int si = 0; si < nsteps && ok; ++si) {
          const TsStepS& st = steps[sd * 3 + si];
          const uint32_t bytes = st.bytes;
          // the chunk's 8-row groups are split over the CL CTAs (the last ones may get none)
          const uint32_t groups = bytes / st.sbo, gper = (groups + CL - 1) / CL;
          const uint32_t off = min((uint32_t)crank * gper, groups) * st.sbo;
          const uint32_t len = min(gper * st.sbo, bytes - off);
          for (int c = 0; c < st.nchunks; ++c, ++h) {
            const uint32_t slot = h % NS;
            if (h >= NS && !mbar_wait(&empty_b[slot], ((h / NS) - 1) & 1, abort_flag)) { ok = false; break; }
            uint8_t* bh = b_base + (size_t)slot * PARTS * a.b_slot_bytes;
            mbar_arrive_expect_tx(&full_b[slot], SPLIT ? 2 * bytes : bytes);
            if (len > 0) {
              if (CL > 1) {
                tma_load_1d_mc(bh + off, st.hi + (size_t)c * bytes + off, len, &full_b[slot], MASK);
                if (SPLIT) tma_load_1d_mc(bh + a.b_slot_bytes + off, st.lo + (size_t)c * bytes + off, len, &full_b[slot], MASK);
              } else {
                tma_load_1d(bh, st.hi + (size_t)c * bytes, bytes, &full_b[slot]);
                if (SPLIT) tma_load_1d(bh + a.b_slot_bytes, st.lo + (size_t)c * bytes, bytes, &full_b[slot]);
              }
            }
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(a.status, (int)PTTK_ETIMEOUT);
      }
      const int zero = 0;
      for (uint32_t k = (h > (uint32_t)NS ? h - NS : 0); k < h; ++k) mbar_wait(&full_b[k % NS], (k / NS) & 1, &zero);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (int64_t it = cid; it < nitems && ok; it += ncl) {
        const int sd = item_side(it);
        for (int si = 0; si < nsteps && ok; ++si) {
          const TsStepS& st = steps[sd * 3 + si];
          const uint32_t idesc = st.idesc, sbo = st.sbo;
          const int ksteps = st.ksteps, nch = st.nchunks;
          const int ab = (si == 0 && nsteps > 1) ? 1 : 0;
          const uint32_t dacc = tmem + (ab ? (uint32_t)a.acc1_col : 0u);
          for (int c = 0; c < nch; ++c, ++g) {
            const uint32_t slot = g % NS, par = (g / NS) & 1;
            if (!mbar_wait(&full_a[slot], par, abort_flag) || !mbar_wait(&full_b[slot], par, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t ta = tmem + (uint32_t)(a.a_col + (int)slot * PARTS * a.a_part_cols);
            const uint32_t sb = smem_u32(b_base + (size_t)slot * PARTS * a.b_slot_bytes);
            const uint64_t bh0 = smem_desc2(sb, sbo);
            const uint64_t bl0 = smem_desc2(sb + a.b_slot_bytes, sbo);
            for (int k = 0; k < ksteps; ++k) {
              const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
              // +256 bytes of K per MMA: +16 in the descriptor's address field (no carry: the
              // chunk lies inside the 256 KB the 14-bit field addresses)
              const uint64_t bh = bh0 + (uint64_t)(16 * k);
              umma_f16_ts(dacc, ta + 8 * k, bh, idesc, acc);
              if (SPLIT) {
                umma_f16_ts(dacc, ta + 8 * k, bl0 + (uint64_t)(16 * k), idesc, 1u);
                umma_f16_ts(dacc, ta + (uint32_t)a.a_part_cols + 8 * k, bh, idesc, 1u);
              }
            }
            umma_commit(&empty_a[slot]);
            if (CL > 1) umma_commit_mc(&empty_b[slot], MASK);
            else umma_commit(&empty_b[slot]);
            if (c == nch - 1) umma_commit(&acc_ready[ab]);
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(a.status, (int)PTTK_ETIMEOUT);
      }
      const int zero = 0;
      if (g > 0) mbar_wait(&empty_a[(g - 1) % NS], ((g - 1) / NS) & 1, &zero);
    }
    __syncwarp();
  } else {
    // ---------------- generator warps: A chunks into TMEM, S in registers, epilogues ----------
    const int gw = warp - 2;                   // 0..NGEN_WARPS-1
    const int quarter = warp & 3;              // TMEM lane quarter this warp may access
    const int row = 32 * quarter + lane;
    const int part = gw >> 2;                  // which quarter of the a range
    const uint32_t lanes = (uint32_t)(32 * quarter) << 16;
    uint32_t g = 0;
    bool dead = false;
    float S[TS_SPT];                           // S_in[row, part spt + i]
    auto basis = [&](int sd, int si, int buf, float x) {
      const TsStepS& st = steps[sd * 3 + si];
      const float xh = (2.f * x - st.lo_box - st.hi_box) / (st.lo_box - st.hi_box);
      float* bv = Bv + ((size_t)buf * TILE_M + row) * bv_ld;
      const float sc = st.a_scale;
      float t0 = 1.f, t1 = xh;
      bv[0] = sc;
      for (int k = 1; k < a.n; ++k) {
        bv[k] = t1 * sc;
        const float t2 = 2.f * xh * t1 - t0;
        t0 = t1;
        t1 = t2;
      }
      for (int k = a.n; k < bv_ld; ++k) bv[k] = 0.f;
    };
    auto coord_of = [&](int64_t it, int si) -> float {
      const int sd = item_side(it);
      const int64_t gp = item_row0(it) + row;
      const TsStepS& st = steps[sd * 3 + si];
      return gp < a.N[sd] ? a.pts[sd][gp * a.d + st.coord] : st.lo_box;
    };
    auto seed_coord_of = [&](int64_t it) -> float {
      const int sd = item_side(it);
      const int64_t gp = item_row0(it) + row;
      return (a.s0_coord[sd] >= 0 && gp < a.N[sd]) ? a.pts[sd][gp * a.d + a.s0_coord[sd]] : a.s0_lo[sd];
    };
    // input of the first step of item `it` (threads of part 0): T_0..T_{n-1}(xhat) of the seed
    // coordinate (merged first steps), or S_0 = 1; zero up to the step's R_in_pad
    auto write_seed = [&](int64_t it, float x) {
      const int sd = item_side(it);
      float* w = Sseed + (size_t)row * a.ld_seed;
      const int pad = steps[sd * 3].R_in_pad;
      if (a.s0_coord[sd] >= 0) {
        const float lo = a.s0_lo[sd], hi = a.s0_hi[sd];
        const float xh = (2.f * x - lo - hi) / (lo - hi);
        float t0 = 1.f, t1 = xh;
        w[0] = 1.f;
        for (int k = 1; k < pad; ++k) {
          w[k] = k < a.n ? t1 : 0.f;
          const float t2 = 2.f * xh * t1 - t0;
          t0 = t1;
          t1 = t2;
        }
      } else {
        w[0] = 1.f;
        for (int k = 1; k < pad; ++k) w[k] = 0.f;
      }
    };
    auto load_seed = [&](int sd) {
      const int spt = steps[sd * 3].spt;
      const float* w = Sseed + (size_t)row * a.ld_seed + part * spt;
#pragma unroll
      for (int i = 0; i < TS_SPT; ++i) S[i] = i < spt ? w[i] : 0.f;
    };
    auto write_output = [&](int osd, int64_t orow0, int orows, uint32_t lane_addr) {
      const TsStepS& st = steps[osd * 3 + nsteps - 1];
      float* stg = stage + (size_t)gw * 32 * STAGE_LD;
      const int R = st.R_out;
      float* outbase = a.out[osd] + (orow0 + 32 * quarter) * R;
      const int wrows = std::max(0, std::min(32, orows - 32 * quarter));
      if (wrows == 0) return;
      const int sub = lane >> 4, lc = lane & 15;
      for (int cb = STAGE_COLS * part; cb < st.Npad; cb += STAGE_COLS * NPART) {
        float v[STAGE_COLS];
        tmem_ld16(lane_addr + (uint32_t)cb, v);
#pragma unroll
        for (int i = 0; i < STAGE_COLS; ++i) stg[lane * STAGE_LD + i] = v[i] * st.out_scale;
        __syncwarp();
        const int col = cb + lc;
        if (col < R)
          for (int rr = sub; rr < wrows; rr += 2) outbase[(int64_t)rr * R + col] = stg[rr * STAGE_LD + lc];
        __syncwarp();
      }
    };
    uint32_t done_acc[2] = {0u, 0u};
    auto wait_acc = [&](int ab) {
      if (!dead && !*abort_flag) dead = !mbar_wait(&acc_ready[ab], done_acc[ab] & 1, abort_flag);
      ++done_acc[ab];
      dead = __any_sync(0xffffffffu, dead || *abort_flag);
      if (dead && lane == 0) *abort_flag = 1;
      tc_fence_after();
    };
    const bool defer = nsteps > 1;
    float xn[4] = {0.f, 0.f, 0.f, 0.f};
    if (part == 0 && cid < nitems) {
      #pragma unroll
      for (int si = 0; si < 3; ++si)
        if (si < nsteps) xn[si] = coord_of(cid, si);
      xn[3] = seed_coord_of(cid);
      basis(item_side(cid), 0, 0, xn[0]);
      write_seed(cid, xn[3]);
    }
    gen_barrier();
    uint32_t bufsel = 0;
    bool out_pending = false;
    int out_sd = 0, out_rows = 0;
    int64_t out_row0 = 0;
    for (int64_t it = cid; it < nitems; it += ncl) {
      const int sd = item_side(it);
      const int64_t row0 = item_row0(it);
      const int rows = (int)std::max<int64_t>(0, std::min<int64_t>(TILE_M, a.N[sd] - row0));
      const float xcur1 = xn[1], xcur2 = xn[2];
      const int64_t itn = it + ncl;
      if (part == 0 && itn < nitems) {
        #pragma unroll
        for (int si = 0; si < 3; ++si)
          if (si < nsteps) xn[si] = coord_of(itn, si);
        xn[3] = seed_coord_of(itn);
      }
      load_seed(sd);
      for (int si = 0; si < nsteps; ++si) {
        const TsStepS& st = steps[sd * 3 + si];
        const int nch = st.nchunks, jpc = st.jpc, rpad = st.R_in_pad, spt = st.spt;
        const float* bvrow = Bv + ((size_t)bufsel * TILE_M + row) * bv_ld;
        for (int c = 0; c < nch; ++c, ++g) {
          const uint32_t slot = g % NS, use = g / NS;
          dead = dead || *abort_flag;
          if (!dead && g >= (uint32_t)NS) dead = !mbar_wait(&empty_a[slot], (use - 1) & 1, abort_flag);
          dead = __any_sync(0xffffffffu, dead);
          if (dead && lane == 0) *abort_flag = 1;
          if (!dead) {
            tc_fence_after();
            const uint32_t cbase = tmem + lanes + (uint32_t)(a.a_col + (int)slot * PARTS * a.a_part_cols);
            for (int jj = 0; jj < jpc; ++jj) {
              const float b = bvrow[c * jpc + jj];
              const uint32_t col = cbase + (uint32_t)((jj * rpad + part * spt) >> 1);
#pragma unroll
              for (int i = 0; i < TS_SPT; i += 2) {
                if (i < spt) {
                  uint32_t h, l;
                  pack_pair<FMT, SPLIT>(b * S[i], b * S[i + 1], h, l);
                  tmem_st1(col + (uint32_t)(i >> 1), h);
                  if (SPLIT) tmem_st1(col + (uint32_t)a.a_part_cols + (uint32_t)(i >> 1), l);
                }
              }
            }
            tmem_wait_st();
            tc_fence_before();
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&full_a[slot]);
        }
        const bool last = si == nsteps - 1;
        if (part == 0) {
          if (!last) basis(sd, si + 1, bufsel ^ 1, si == 0 ? xcur1 : xcur2);
          else if (itn < nitems) basis(item_side(itn), 0, bufsel ^ 1, xn[0]);
        }
        if (si == 0 && out_pending) {
          wait_acc(0);
          if (!dead) write_output(out_sd, out_row0, out_rows, tmem + lanes);
          out_pending = false;
        }
        if (last && defer && itn < nitems) {
          out_pending = true;
          out_sd = sd;
          out_row0 = row0;
          out_rows = rows;
          // the seed of the next item: this item's seed was read into registers before its
          // first step, and every thread passed the barrier below since
          if (part == 0) write_seed(itn, xn[3]);
          bufsel ^= 1;
          tc_fence_before();
          gen_barrier();
          continue;
        }
        const int ab = (si == 0 && defer) ? 1 : 0;
        wait_acc(ab);
        const uint32_t lane_addr = tmem + lanes + (ab ? (uint32_t)a.acc1_col : 0u);
        if (!last) {
          // S_in of the next step: this thread's spt columns of the accumulator (columns at or
          // beyond R_out hold zeros: the core images are zero there)
          const TsStepS& nx = steps[sd * 3 + si + 1];
          if (!dead) {
            float v[16];
            tmem_ld1x16(lane_addr + (uint32_t)(part * nx.spt), v);
            const float osc = st.out_scale;
#pragma unroll
            for (int i = 0; i < TS_SPT; ++i) S[i] = i < nx.spt ? v[i] * osc : 0.f;
          }
        } else if (!dead) {
          write_output(sd, row0, rows, lane_addr);
        }
        bufsel ^= 1;
        tc_fence_before();
        gen_barrier();
        if (last && !defer && itn < nitems) {
          if (part == 0) write_seed(itn, xn[3]);
          gen_barrier();
        }
      }
    }
    if (dead && lane == 0) {
      *abort_flag = 1;
      atomicExch(a.status, (int)PTTK_ETIMEOUT);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // no CTA leaves while a peer may still copy into its shared memory or commit to its barriers
  if (CL > 1) cluster_sync_all();
  if (warp == 1) tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

// ---------------- A in tensor memory, dedicated epilogue warps -------------------------------
// The tensor-memory-A chain (A generated into TMEM, S_in in registers, B alone in shared
// memory) with the output written by four epilogue warps of their own from one of two
// accumulator regions, as in chain_tce_kernel. With A out of shared memory, shared memory holds
// a deeper B ring (NSB slots): a B chunk of a split form is 36-48 KB, whose copy from L2 takes
// about 2,000 SM clocks, so a ring of two slots (what fits beside a shared-memory A ring)
// leaves every chunk waiting for its copy, while NSB >= 3 keeps the copies ahead of the MMAs.
// A and B have rings of their own (NSA = 2 TMEM slots, NSB shared-memory slots), each with
// full and empty barriers.
// TMEM: region r (r = tile parity) at column r * RC holds a tile's accumulators (the first
// step's result is read back as the second step's input before the second step's first MMA
// overwrites it); the NSA A slots follow at column 2 RC.
// Barriers: full_a[NSA] (the 16 generator warps, after their tcgen05.st completed),
// empty_a[NSA] (commit of the slot's MMAs), full_b[NSB] (TMA bytes), empty_b[NSB] (commit),
// mid[r], last_done[r], rfree[r] as in chain_tce_kernel.
constexpr int NSA_TSE = 2;
constexpr int EPI_LD = 33;  // epilogue staging: 32 rows x 32 columns, row stride 33 floats

// 32 consecutive TMEM columns of this warp's 32 lanes and the wait for them, in one block (no
// use of the values can be scheduled before the wait)
__device__ __forceinline__ void tmem_ld32_wait(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int FMT, bool SPLIT, int NSB>
__global__ void __launch_bounds__(TCE_THREADS, 1) chain_tse_kernel(TsArgs a) {
  constexpr int PARTS = SPLIT ? 2 : 1;
  constexpr int NSA = NSA_TSE;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int bv_ld = a.bv_ld;
  const int RC = a.region_col;
  uint8_t* b_base = smem;                                                // NSB x PARTS x b_slot_bytes
  float* Bv = reinterpret_cast<float*>(b_base + (size_t)NSB * PARTS * a.b_slot_bytes);  // 2 x 128 x bv_ld
  float* Sseed = Bv + (size_t)2 * TILE_M * bv_ld;                        // 128 x ld_seed
  float* stage = Sseed + (size_t)TILE_M * a.ld_seed;                     // NEPI_WARPS x 32 x EPI_LD
  TsStepS* steps = reinterpret_cast<TsStepS*>(
      (reinterpret_cast<uintptr_t>(stage + (size_t)NEPI_WARPS * 32 * EPI_LD) + 15) & ~uintptr_t(15));  // [2][3]
  uint64_t* bars = reinterpret_cast<uint64_t*>(steps + 6);
  uint64_t* full_a = bars;
  uint64_t* empty_a = bars + NSA;
  uint64_t* full_b = bars + 2 * NSA;
  uint64_t* empty_b = bars + 2 * NSA + NSB;
  uint64_t* mid = bars + 2 * NSA + 2 * NSB;        // [2]
  uint64_t* last_done = mid + 2;                    // [2]
  uint64_t* rfree = mid + 4;                        // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mid + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < NSA; ++i) {
      mbar_init(&full_a[i], NGEN_WARPS);
      mbar_init(&empty_a[i], 1);
    }
    for (int i = 0; i < NSB; ++i) {
      mbar_init(&full_b[i], 1);
      mbar_init(&empty_b[i], 1);
    }
    for (int r = 0; r < 2; ++r) {
      mbar_init(&mid[r], 1);
      mbar_init(&last_done[r], 1);
      mbar_init(&rfree[r], NEPI_WARPS);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (tid < 2 * a.nsteps) steps[(tid / a.nsteps) * 3 + tid % a.nsteps] = a.st[tid / a.nsteps][tid % a.nsteps];
  if (warp == 1) {
    tmem_alloc(tmem_slot, (uint32_t)a.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t nitems = a.nitems;
  const int nsteps = a.nsteps;
  auto item_side = [&](int64_t k) -> int { return k < a.T0p ? 0 : 1; };
  auto item_row0 = [&](int64_t k) -> int64_t { return (k - (item_side(k) ? a.T0p : 0)) * TILE_M; };

  if (warp == 0) {
    // ---------------- TMA producer: B chunks into the NSB-deep ring ----------------
    if (lane == 0) {
      uint32_t h = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        const int sd = item_side(it);
        for (int si = 0; si < nsteps && ok; ++si) {
          const TsStepS& st = steps[sd * 3 + si];
          for (int c = 0; c < st.nchunks; ++c, ++h) {
            const uint32_t slot = h % NSB;
            if (h >= (uint32_t)NSB && !mbar_wait(&empty_b[slot], ((h / NSB) - 1) & 1, abort_flag)) {
              ok = false;
              break;
            }
            uint8_t* bh = b_base + (size_t)slot * PARTS * a.b_slot_bytes;
            mbar_arrive_expect_tx(&full_b[slot], SPLIT ? 2 * st.bytes : st.bytes);
            tma_load_1d(bh, st.hi + (size_t)c * st.bytes, st.bytes, &full_b[slot]);
            if (SPLIT) tma_load_1d(bh + a.b_slot_bytes, st.lo + (size_t)c * st.bytes, st.bytes, &full_b[slot]);
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(a.status, (int)PTTK_ETIMEOUT);
      }
      const int zero = 0;
      for (uint32_t k = (h > (uint32_t)NSB ? h - NSB : 0); k < h; ++k) mbar_wait(&full_b[k % NSB], (k / NSB) & 1, &zero);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t g = 0, tile = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++tile) {
        const int sd = item_side(it);
        const uint32_t r = tile & 1, use = tile >> 1;
        // the region's previous tile must have left it
        if (use >= 1 && !mbar_wait(&rfree[r], (use - 1) & 1, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dacc = tmem + r * (uint32_t)RC;
        for (int si = 0; si < nsteps && ok; ++si) {
          const TsStepS& st = steps[sd * 3 + si];
          const uint32_t idesc = st.idesc, sbo = st.sbo;
          const int ksteps = st.ksteps, nch = st.nchunks;
          for (int c = 0; c < nch; ++c, ++g) {
            const uint32_t sa = g % NSA, sb = g % NSB;
            if (!mbar_wait(&full_a[sa], (g / NSA) & 1, abort_flag) ||
                !mbar_wait(&full_b[sb], (g / NSB) & 1, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t ta = tmem + (uint32_t)(a.a_col + (int)sa * PARTS * a.a_part_cols);
            const uint32_t bsm = smem_u32(b_base + (size_t)sb * PARTS * a.b_slot_bytes);
            const uint64_t bh0 = smem_desc2(bsm, sbo);
            const uint64_t bl0 = smem_desc2(bsm + a.b_slot_bytes, sbo);
            for (int k = 0; k < ksteps; ++k) {
              const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
              const uint64_t bh = bh0 + (uint64_t)(16 * k);
              umma_f16_ts(dacc, ta + 8 * k, bh, idesc, acc);
              if (SPLIT) {
                umma_f16_ts(dacc, ta + 8 * k, bl0 + (uint64_t)(16 * k), idesc, 1u);
                umma_f16_ts(dacc, ta + (uint32_t)a.a_part_cols + 8 * k, bh, idesc, 1u);
              }
            }
            umma_commit(&empty_a[sa]);
            umma_commit(&empty_b[sb]);
            if (c == nch - 1) umma_commit(si == nsteps - 1 ? &last_done[r] : &mid[r]);
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(a.status, (int)PTTK_ETIMEOUT);
      }
      const int zero = 0;
      if (g > 0) mbar_wait(&empty_a[(g - 1) % NSA], ((g - 1) / NSA) & 1, &zero);
    }
    __syncwarp();
  } else if (warp < 2 + NGEN_WARPS) {
    // ---------------- generator warps: A chunks into TMEM, S_in in registers ----------------
    const int gw = warp - 2;
    const int quarter = warp & 3;
    const int row = 32 * quarter + lane;
    const int part = gw >> 2;
    const uint32_t lanes = (uint32_t)(32 * quarter) << 16;
    uint32_t g = 0, tile = 0;
    bool dead = false;
    float S[TS_SPT];
    auto basis = [&](int sd, int si, int buf, float x) {
      const TsStepS& st = steps[sd * 3 + si];
      const float xh = (2.f * x - st.lo_box - st.hi_box) / (st.lo_box - st.hi_box);
      float* bv = Bv + ((size_t)buf * TILE_M + row) * bv_ld;
      const float sc = st.a_scale;
      float t0 = 1.f, t1 = xh;
      bv[0] = sc;
      for (int k = 1; k < a.n; ++k) {
        bv[k] = t1 * sc;
        const float t2 = 2.f * xh * t1 - t0;
        t0 = t1;
        t1 = t2;
      }
      for (int k = a.n; k < bv_ld; ++k) bv[k] = 0.f;
    };
    auto coord_of = [&](int64_t it, int si) -> float {
      const int sd = item_side(it);
      const int64_t gp = item_row0(it) + row;
      const TsStepS& st = steps[sd * 3 + si];
      return gp < a.N[sd] ? a.pts[sd][gp * a.d + st.coord] : st.lo_box;
    };
    auto seed_coord_of = [&](int64_t it) -> float {
      const int sd = item_side(it);
      const int64_t gp = item_row0(it) + row;
      return (a.s0_coord[sd] >= 0 && gp < a.N[sd]) ? a.pts[sd][gp * a.d + a.s0_coord[sd]] : a.s0_lo[sd];
    };
    auto write_seed = [&](int64_t it, float x) {
      const int sd = item_side(it);
      float* w = Sseed + (size_t)row * a.ld_seed;
      const int pad = steps[sd * 3].R_in_pad;
      if (a.s0_coord[sd] >= 0) {
        const float lo = a.s0_lo[sd], hi = a.s0_hi[sd];
        const float xh = (2.f * x - lo - hi) / (lo - hi);
        float t0 = 1.f, t1 = xh;
        w[0] = 1.f;
        for (int k = 1; k < pad; ++k) {
          w[k] = k < a.n ? t1 : 0.f;
          const float t2 = 2.f * xh * t1 - t0;
          t0 = t1;
          t1 = t2;
        }
      } else {
        w[0] = 1.f;
        for (int k = 1; k < pad; ++k) w[k] = 0.f;
      }
    };
    float xn[4] = {0.f, 0.f, 0.f, 0.f};
    if (part == 0 && blockIdx.x < nitems) {
      #pragma unroll
      for (int si = 0; si < 3; ++si)
        if (si < nsteps) xn[si] = coord_of(blockIdx.x, si);
      xn[3] = seed_coord_of(blockIdx.x);
      basis(item_side(blockIdx.x), 0, 0, xn[0]);
      write_seed(blockIdx.x, xn[3]);
    }
    gen_barrier();
    uint32_t bufsel = 0;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x, ++tile) {
      const int sd = item_side(it);
      const uint32_t r = tile & 1, use = tile >> 1;
      const float xcur1 = xn[1], xcur2 = xn[2];
      const int64_t itn = it + gridDim.x;
      if (part == 0 && itn < nitems) {
        #pragma unroll
        for (int si = 0; si < 3; ++si)
          if (si < nsteps) xn[si] = coord_of(itn, si);
        xn[3] = seed_coord_of(itn);
      }
      {
        const int spt = steps[sd * 3].spt;
        const float* w = Sseed + (size_t)row * a.ld_seed + part * spt;
#pragma unroll
        for (int i = 0; i < TS_SPT; ++i) S[i] = i < spt ? w[i] : 0.f;
      }
      for (int si = 0; si < nsteps; ++si) {
        const TsStepS& st = steps[sd * 3 + si];
        const int nch = st.nchunks, jpc = st.jpc, rpad = st.R_in_pad, spt = st.spt;
        const float* bvrow = Bv + ((size_t)bufsel * TILE_M + row) * bv_ld;
        for (int c = 0; c < nch; ++c, ++g) {
          const uint32_t sa = g % NSA, use_a = g / NSA;
          dead = dead || *abort_flag;
          if (!dead && g >= (uint32_t)NSA) dead = !mbar_wait(&empty_a[sa], (use_a - 1) & 1, abort_flag);
          dead = __any_sync(0xffffffffu, dead);
          if (dead && lane == 0) *abort_flag = 1;
          if (!dead) {
            tc_fence_after();
            const uint32_t cbase = tmem + lanes + (uint32_t)(a.a_col + (int)sa * PARTS * a.a_part_cols);
            for (int jj = 0; jj < jpc; ++jj) {
              const float b = bvrow[c * jpc + jj];
              const uint32_t col = cbase + (uint32_t)((jj * rpad + part * spt) >> 1);
#pragma unroll
              for (int i = 0; i < TS_SPT; i += 2) {
                if (i < spt) {
                  uint32_t h, l;
                  pack_pair<FMT, SPLIT>(b * S[i], b * S[i + 1], h, l);
                  tmem_st1(col + (uint32_t)(i >> 1), h);
                  if (SPLIT) tmem_st1(col + (uint32_t)a.a_part_cols + (uint32_t)(i >> 1), l);
                }
              }
            }
            tmem_wait_st();
            tc_fence_before();
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&full_a[sa]);
        }
        const bool last = si == nsteps - 1;
        if (part == 0) {
          if (!last) basis(sd, si + 1, bufsel ^ 1, si == 0 ? xcur1 : xcur2);
          else if (itn < nitems) basis(item_side(itn), 0, bufsel ^ 1, xn[0]);
        }
        if (!last) {
          // this step's result is the next step's input: wait for it and keep this thread's
          // spt columns of it in registers (columns at or past R_out hold zeros)
          const uint32_t phase = use * (uint32_t)(nsteps - 1) + (uint32_t)si;
          if (!dead && !*abort_flag) dead = !mbar_wait(&mid[r], phase & 1, abort_flag);
          dead = __any_sync(0xffffffffu, dead || *abort_flag);
          if (dead && lane == 0) *abort_flag = 1;
          tc_fence_after();
          const TsStepS& nx = steps[sd * 3 + si + 1];
          if (!dead) {
            float v[16];
            tmem_ld1x16(tmem + lanes + r * (uint32_t)RC + (uint32_t)(part * nx.spt), v);
            const float osc = st.out_scale;
#pragma unroll
            for (int i = 0; i < TS_SPT; ++i) S[i] = i < nx.spt ? v[i] * osc : 0.f;
          }
        }
        bufsel ^= 1;
        tc_fence_before();
        gen_barrier();
        if (last && itn < nitems) {
          // the next tile's seed: every thread read this tile's seed into registers before
          // the barrier above
          if (part == 0) write_seed(itn, xn[3]);
          gen_barrier();
        }
      }
    }
    if (dead && lane == 0) {
      *abort_flag = 1;
      atomicExch(a.status, (int)PTTK_ETIMEOUT);
    }
  } else {
    // ---------------- epilogue warps: one TMEM lane quarter each ----------------
    const int ew = warp - 2 - NGEN_WARPS;  // 0..3
    const int quarter = warp & 3;
    const uint32_t lanes = (uint32_t)(32 * quarter) << 16;
    float* stg = stage + (size_t)ew * 32 * EPI_LD;
    uint32_t tile = 0;
    bool dead = false;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x, ++tile) {
      const int sd = item_side(it);
      const uint32_t r = tile & 1, use = tile >> 1;
      const TsStepS& st = steps[sd * 3 + nsteps - 1];
      if (!dead && !*abort_flag) dead = !mbar_wait(&last_done[r], use & 1, abort_flag);
      dead = __any_sync(0xffffffffu, dead || *abort_flag);
      if (dead && lane == 0) *abort_flag = 1;
      tc_fence_after();
      if (!dead) {
        const int64_t row0 = item_row0(it);
        const int rows = (int)std::max<int64_t>(0, std::min<int64_t>(TILE_M, a.N[sd] - row0));
        const int R = st.R_out;
        float* outbase = a.out[sd] + (row0 + 32 * quarter) * R;
        const int wrows = std::max(0, std::min(32, rows - 32 * quarter));
        const float osc = st.out_scale;
        // 32 columns at a time: each row's 32 values through the staging tile, then each store
        // instruction writes 32 consecutive columns (128 bytes) of one row
        for (int cb = 0; cb < st.Npad; cb += 32) {
          float v[32];
          tmem_ld32_wait(tmem + lanes + r * (uint32_t)RC + (uint32_t)cb, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) stg[lane * EPI_LD + i] = v[i] * osc;
          __syncwarp();
          const int col = cb + lane;
          if (col < R)
            for (int rr = 0; rr < wrows; ++rr) outbase[(int64_t)rr * R + col] = stg[rr * EPI_LD + lane];
          __syncwarp();
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&rfree[r]);
    }
    if (dead && lane == 0) {
      *abort_flag = 1;
      atomicExch(a.status, (int)PTTK_ETIMEOUT);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

// ---------------- core images -------------------------------------------------------------
// Image of the oriented core (K x R_out, column-major, FP64; K = n R_in) for one chain step in
// the padded K order k' = a + R_in_pad j (zero rows for a >= R_in): chunk c holds rows o < Npad
// and K'-elements [c KC, (c+1) KC) in the K-major no-swizzle layout (row group stride 8 KCB).
template <int FMT>
__global__ void core_image_kernel(const double* __restrict__ G, int n, int R_in, int R_in_pad, int R_out,
                                  int Npad, int nchunks, int KCB, bool split, double scale,
                                  uint8_t* __restrict__ hi, uint8_t* __restrict__ lo) {
  constexpr int E = FMT == FMT_TF32 ? 4 : 8;
  const int KC = KCB / (FMT == FMT_TF32 ? 4 : 2);
  const int K = n * R_in;
  const int64_t total = (int64_t)nchunks * Npad * KC;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(e % KC);
    const int o = (int)((e / KC) % Npad);
    const int c = (int)(e / ((int64_t)KC * Npad));
    const int kp = c * KC + kk;
    const int j = kp / R_in_pad, ai = kp - j * R_in_pad;
    const double v = (ai < R_in && j < n && o < R_out) ? scale * G[(ai + R_in * j) + (int64_t)K * o] : 0.0;
    const size_t off = (size_t)c * Npad * KCB + (size_t)(o >> 3) * (8 * KCB) + (size_t)(kk / E) * 128 +
                       (size_t)(o & 7) * 16;
    if constexpr (FMT == FMT_BF16) {
      const __nv_bfloat16 h = __double2bfloat16(v);
      reinterpret_cast<__nv_bfloat16*>(hi + off)[kk % E] = h;
      if (split) reinterpret_cast<__nv_bfloat16*>(lo + off)[kk % E] = __double2bfloat16(v - (double)__bfloat162float(h));
    } else if constexpr (FMT == FMT_FP16) {
      const __half h = __double2half(v);
      reinterpret_cast<__half*>(hi + off)[kk % E] = h;
      if (split) reinterpret_cast<__half*>(lo + off)[kk % E] = __double2half(v - (double)__half2float(h));
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
  int Npad[2][3] = {}, nchunks[2][3] = {}, R_in_pad[2][3] = {};
  int jpc[2][3] = {}, kcb[2][3] = {};  // TS images: basis values per chunk, bytes of K per row
  float a_scale[2][3] = {}, out_scale[2][3] = {};
};

std::mutex g_img_mu;

}  // namespace

// Per-handle image cache, indexed by form and chunk width (64 or 128 bytes of K per row).
struct TcImageCache {
  Images img[6][2];
  Images ts[6];                       // images of the TS kernel (kind::f16 forms)
  double* L[2] = {nullptr, nullptr};  // merged first two cores per side (see tc_chain_steps)
};

static int form_index(pttk_prec p) {
  switch (p) {
    case PTTK_TF32: return 0;
    case PTTK_TF32X3: return 1;
    case PTTK_BF16: return 2;
    case PTTK_BF16X3: return 3;
    case PTTK_FP16: return 4;
    case PTTK_FP16X3: return 5;
    default: return -1;
  }
}

TcImageCache* tc_cache_new() { return new TcImageCache(); }
void tc_cache_free(TcImageCache* c) {
  if (!c) return;
  for (auto& f : c->img)
    for (auto& im : f)
      if (im.buf) cudaFree(im.buf);
  for (auto& im : c->ts)
    if (im.buf) cudaFree(im.buf);
  for (double* L : c->L)
    if (L) cudaFree(L);
  delete c;
}

// Steps of the tensor-core chain on one side (0: source, 1: target). With d >= 2 the first two
// steps of Algorithm 2, Phase 3 are merged: S_2 = (B_2 face-split B_1) L with
// L[i + n (j + n b)] = sum_a G_1[i, a] G_2[a, j, b] (G_1, G_2 the first two oriented cores), one
// chain step whose input S is the basis vector of the first coordinate (R_in = n). It has the
// K and N of the second step, so it adds no MMA work, and each tile runs one step (one pipeline
// drain and epilogue) fewer. Returns the step count; *s0_coord is the seed coordinate, or -1
// when S starts as 1.
struct TcChainStep {
  int R_in, R_out, coord;
  const double* G;  // FP64 oriented core (R_in x n x R_out, column-major) on the device
};
static int tc_chain_steps(const pttk_tt* tt, const TcImageCache* cache, int side, TcChainStep* st,
                          int* s0_coord) {
  const bool src = side == 0;
  const bool merged = tt->d >= 2 && cache->L[side] != nullptr;
  int nst = 0;
  for (int i = merged ? 1 : 0; i < tt->d; ++i) {
    int rin, rout, coord;
    const int k = oriented_core_dims(tt, src, i, &rin, &rout, &coord);
    TcChainStep c{rin, rout, coord, static_cast<const double*>(oriented_core_ptr(tt, src, k, true))};
    if (merged && i == 1) {
      c.R_in = tt->n;
      c.G = cache->L[side];
    }
    st[nst++] = c;
  }
  *s0_coord = -1;
  if (merged) {
    int rin, rout, coord;
    oriented_core_dims(tt, src, 0, &rin, &rout, &coord);
    *s0_coord = coord;
  }
  return nst;
}

// The merged cores L of both sides, formed once per handle in FP64 on the host.
static pttk_status ensure_merged(const pttk_tt* tt, TcImageCache* cache) {
  if (tt->d < 2) return PTTK_OK;
  const int n = tt->n;
  for (int side = 0; side < 2; ++side) {
    if (cache->L[side]) continue;
    int r0in, r0, c0, r1in, r1, c1;
    const int k0 = oriented_core_dims(tt, side == 0, 0, &r0in, &r0, &c0);
    const int k1 = oriented_core_dims(tt, side == 0, 1, &r1in, &r1, &c1);
    if (r0in != 1 || r1in != r0) return set_error(PTTK_ECUDA, "unexpected TT ranks at the chain ends");
    std::vector<double> G0((size_t)n * r0), G1((size_t)r0 * n * r1), L((size_t)n * n * r1, 0.0);
    PTTK_CUDA(cudaMemcpy(G0.data(), oriented_core_ptr(tt, side == 0, k0, true), sizeof(double) * G0.size(),
                         cudaMemcpyDeviceToHost));
    PTTK_CUDA(cudaMemcpy(G1.data(), oriented_core_ptr(tt, side == 0, k1, true), sizeof(double) * G1.size(),
                         cudaMemcpyDeviceToHost));
    for (int b = 0; b < r1; ++b)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          double acc = 0.0;
          for (int a = 0; a < r0; ++a) acc += G0[(size_t)i + (size_t)n * a] * G1[(size_t)a + (size_t)r0 * (j + (size_t)n * b)];
          L[(size_t)i + (size_t)n * (j + (size_t)n * b)] = acc;
        }
    double* dL = nullptr;
    PTTK_CUDA(cudaMalloc(&dL, sizeof(double) * L.size()));
    const cudaError_t e = cudaMemcpy(dL, L.data(), sizeof(double) * L.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(dL);
      return cuda_error(e, "merged chain core");
    }
    cache->L[side] = dL;
  }
  return PTTK_OK;
}

static int form_fmt(pttk_prec p) {
  return (p == PTTK_BF16 || p == PTTK_BF16X3) ? FMT_BF16 : (p == PTTK_FP16 || p == PTTK_FP16X3) ? FMT_FP16 : FMT_TF32;
}
static bool form_split(pttk_prec p) { return p == PTTK_TF32X3 || p == PTTK_BF16X3 || p == PTTK_FP16X3; }

// Power-of-two scales of the FP16 forms (1 for the others): per chain step, the image scale
// 2^sB with max|G| 2^sB <= 2^14 and the A scale 2^sA with bound(|S_in|) 2^sA <= 2^14, where
// bound(S_in of step 0) = 1 and bound(S_out) = bound(S_in) * max over columns of sum |G|.
static pttk_status step_scales(const pttk_tt* tt, const TcImageCache* cache, pttk_prec prec, Images& im,
                               double img_scale[2][3]) {
  for (int side = 0; side < 2; ++side) {
    double bound = 1.0;  // |S| of the first step: 1, or |T_j| <= 1 for a seed basis
    TcChainStep cs[3];
    int s0;
    const int nst = tc_chain_steps(tt, cache, side, cs, &s0);
    for (int i = 0; i < nst; ++i) {
      img_scale[side][i] = 1.0;
      im.a_scale[side][i] = 1.f;
      im.out_scale[side][i] = 1.f;
      if (form_fmt(prec) != FMT_FP16) continue;
      const int rin = cs[i].R_in, rout = cs[i].R_out;
      const int64_t K = (int64_t)tt->n * rin;
      std::vector<double> G((size_t)(K * rout));
      PTTK_CUDA(cudaMemcpy(G.data(), cs[i].G, sizeof(double) * G.size(), cudaMemcpyDeviceToHost));
      double gmax = 0.0, colmax = 0.0;
      for (int o = 0; o < rout; ++o) {
        double cs = 0.0;
        for (int64_t q = 0; q < K; ++q) {
          const double g = fabs(G[(size_t)(q + K * o)]);
          gmax = std::max(gmax, g);
          cs += g;
        }
        colmax = std::max(colmax, cs);
      }
      const int sB = gmax > 0.0 ? 14 - (int)ceil(log2(gmax)) : 0;
      const int sA = bound > 0.0 ? 14 - (int)ceil(log2(bound)) : 0;
      img_scale[side][i] = ldexp(1.0, sB);
      im.a_scale[side][i] = (float)ldexp(1.0, sA);
      im.out_scale[side][i] = (float)ldexp(1.0, -(sA + sB));
      bound *= std::max(colmax, 1e-300);
    }
  }
  return PTTK_OK;
}

static pttk_status build_images(const pttk_tt* tt, const TcImageCache* cache, pttk_prec prec, int KCB,
                                Images& im, cudaStream_t s) {
  const int fmt = form_fmt(prec);
  const bool split = form_split(prec);
  const int KC = KCB / (fmt == FMT_TF32 ? 4 : 2);
  const int E = fmt == FMT_TF32 ? 4 : 8;
  double img_scale[2][3];
  PTTK_TRY(step_scales(tt, cache, prec, im, img_scale));
  TcChainStep cs[2][3];
  int s0[2], nst = 0;
  for (int side = 0; side < 2; ++side) nst = tc_chain_steps(tt, cache, side, cs[side], &s0[side]);
  size_t total = 0;
  for (int side = 0; side < 2; ++side)
    for (int i = 0; i < nst; ++i) {
      const int rin = cs[side][i].R_in, rout = cs[side][i].R_out;
      im.R_in_pad[side][i] = ((rin + E - 1) / E) * E;
      im.Npad[side][i] = ((rout + 15) / 16) * 16;
      im.nchunks[side][i] = (tt->n * im.R_in_pad[side][i] + KC - 1) / KC;
      const size_t bytes = (size_t)im.nchunks[side][i] * im.Npad[side][i] * KCB;
      im.hi_off[side][i] = total;
      total += bytes;
      im.lo_off[side][i] = total;
      if (split) total += bytes;
    }
  PTTK_CUDA(cudaMalloc(&im.buf, std::max<size_t>(total, 16)));
  PTTK_CUDA(cudaMemsetAsync(im.buf, 0, std::max<size_t>(total, 16), s));
  for (int side = 0; side < 2; ++side)
    for (int i = 0; i < nst; ++i) {
      const int rin = cs[side][i].R_in, rout = cs[side][i].R_out;
      const double* G = cs[side][i].G;
      const int64_t work = (int64_t)im.nchunks[side][i] * im.Npad[side][i] * KC;
      const unsigned blocks = (unsigned)std::min<int64_t>((work + 255) / 256, (int64_t)sm_count() * 8);
      auto* kfn = fmt == FMT_BF16 ? core_image_kernel<FMT_BF16>
                                  : fmt == FMT_FP16 ? core_image_kernel<FMT_FP16> : core_image_kernel<FMT_TF32>;
      kfn<<<blocks, 256, 0, s>>>(G, tt->n, rin, im.R_in_pad[side][i], rout, im.Npad[side][i], im.nchunks[side][i],
                                 KCB, split, img_scale[side][i], im.buf + im.hi_off[side][i],
                                 im.buf + im.lo_off[side][i]); pttk::count_launch();
    }
  PTTK_CUDA(cudaGetLastError());
  PTTK_CUDA(cudaStreamSynchronize(s));
  return PTTK_OK;
}

// Launch configurations. 0: the shared-memory kernel with dedicated epilogue warps and
// double-buffered accumulators (chain_tce_kernel; the default), 128 bytes of K per chunk row;
// 1 and 2: the shared-memory kernel without them, with {KCB, NSLOT} below; 3..5: the TS kernel
// (A in tensor memory, a ring of 3 slots) in thread-block clusters of 1, 2 or 4 CTAs, for the
// kind::f16 forms whose ranks fit it. A configuration whose kernel cannot hold the ranks falls
// back to configuration 1. 6: A in tensor memory with the epilogue warps (falls back to 0).
// 7: configuration 0 with 64 bytes of K per chunk row and a ring of 4 slots: the same shared
// memory as 0's 128-byte ring of 2 at large ranks, so each core chunk's copy has three chunks
// of products to land behind.
static const int kTcConfigs[2][2] = {{128, 4}, {64, 4}};
static const int kTcConfigsSplit[2][2] = {{128, 2}, {64, 4}};
constexpr int kTceConfigs = 1, kTcSubConfigs = 2, kTsConfigs = 3, kTseConfigs = 1, kTce64Configs = 1;
constexpr int kTceFirst = 0, kSubFirst = kTceFirst + kTceConfigs, kTsFirst = kSubFirst + kTcSubConfigs,
              kTseFirst = kTsFirst + kTsConfigs, kTce64First = kTseFirst + kTseConfigs;
static const int kTsCluster[kTsConfigs] = {1, 2, 4};

int tc_config_count() { return kTseConfigs + kTceConfigs + kTcSubConfigs + kTsConfigs + kTce64Configs; }
static bool ts_form(pttk_prec p) { return p == PTTK_FP16 || p == PTTK_FP16X3 || p == PTTK_BF16 || p == PTTK_BF16X3; }
static bool ts_config(int cfg) { return cfg >= kTsFirst && cfg < kTsFirst + kTsConfigs; }
static int ts_cluster(int cfg) { return kTsCluster[cfg - kTsFirst]; }
static bool tse_config(int cfg) { return cfg >= kTseFirst && cfg < kTseFirst + kTseConfigs; }
static bool tce_config(int cfg) {
  return (cfg >= kTceFirst && cfg < kTceFirst + kTceConfigs) || (cfg >= kTce64First && cfg < kTce64First + kTce64Configs);
}
static int tc_sub_config(int cfg) {
  if (cfg >= kTce64First && cfg < kTce64First + kTce64Configs) return 1;  // {64, 4}
  return cfg >= kSubFirst && cfg < kSubFirst + kTcSubConfigs ? cfg - kSubFirst : 0;
}

static void tc_config(pttk_prec prec, int cfg, int* KCB, int* NS) {
  const bool split = form_split(prec);
  const int (*t)[2] = split ? kTcConfigsSplit : kTcConfigs;
  cfg = tc_sub_config(cfg);
  *KCB = t[cfg][0];
  *NS = t[cfg][1];
}

// TS images: per step, R_in padded to 16, jpc basis values per chunk (K of a chunk about 64),
// each chunk of a part Npad x kcb bytes in the K-major no-swizzle layout.
static pttk_status build_images_ts(const pttk_tt* tt, const TcImageCache* cache, pttk_prec prec, Images& im,
                                   cudaStream_t s) {
  const int fmt = form_fmt(prec);
  const bool split = form_split(prec);
  double img_scale[2][3];
  PTTK_TRY(step_scales(tt, cache, prec, im, img_scale));
  TcChainStep cs[2][3];
  int s0[2], nst = 0;
  for (int side = 0; side < 2; ++side) nst = tc_chain_steps(tt, cache, side, cs[side], &s0[side]);
  size_t total = 0;
  for (int side = 0; side < 2; ++side)
    for (int i = 0; i < nst; ++i) {
      const int rin = cs[side][i].R_in, rout = cs[side][i].R_out;
      const int rpad = ((rin + 15) / 16) * 16;
      const int jpc = std::max(1, std::min(tt->n, 64 / rpad));
      im.R_in_pad[side][i] = rpad;
      im.jpc[side][i] = jpc;
      im.kcb[side][i] = 2 * jpc * rpad;
      im.Npad[side][i] = ((rout + 15) / 16) * 16;
      im.nchunks[side][i] = (tt->n + jpc - 1) / jpc;
      const size_t bytes = (size_t)im.nchunks[side][i] * im.Npad[side][i] * im.kcb[side][i];
      im.hi_off[side][i] = total;
      total += bytes;
      im.lo_off[side][i] = total;
      if (split) total += bytes;
    }
  PTTK_CUDA(cudaMalloc(&im.buf, std::max<size_t>(total, 16)));
  PTTK_CUDA(cudaMemsetAsync(im.buf, 0, std::max<size_t>(total, 16), s));
  for (int side = 0; side < 2; ++side)
    for (int i = 0; i < nst; ++i) {
      const int KC = im.kcb[side][i] / 2;
      const int64_t work = (int64_t)im.nchunks[side][i] * im.Npad[side][i] * KC;
      const unsigned blocks = (unsigned)std::min<int64_t>((work + 255) / 256, (int64_t)sm_count() * 8);
      auto* kfn = fmt == FMT_BF16 ? core_image_kernel<FMT_BF16> : core_image_kernel<FMT_FP16>;
      kfn<<<blocks, 256, 0, s>>>(cs[side][i].G, tt->n, cs[side][i].R_in, im.R_in_pad[side][i], cs[side][i].R_out,
                                 im.Npad[side][i], im.nchunks[side][i], im.kcb[side][i], split, img_scale[side][i],
                                 im.buf + im.hi_off[side][i], im.buf + im.lo_off[side][i]); pttk::count_launch();
    }
  PTTK_CUDA(cudaGetLastError());
  PTTK_CUDA(cudaStreamSynchronize(s));
  return PTTK_OK;
}

// Launch arguments of the TS kernel for these inputs; false (and no error) when the ranks do
// not fit it (an a range above 16 per thread, a rank above 256, tensor or shared memory).
static bool ts_plan(const pttk_tt* tt, const TcImageCache* cache, const Images& im, pttk_prec prec, int NS,
                    TsArgs& a, size_t* smem_out) {
  const bool split = form_split(prec);
  const int parts = split ? 2 : 1;
  const int fmt = form_fmt(prec);
  a = TsArgs{};
  a.n = tt->n;
  a.d = tt->d;
  int nst = 0, acc0w = 16, acc1w = 0, a_part = 8, bvl = 1;
  uint32_t bslot = 0;
  for (int side = 0; side < 2; ++side) {
    TcChainStep cs[3];
    int s0;
    nst = tc_chain_steps(tt, cache, side, cs, &s0);
    a.s0_coord[side] = s0;
    const int b0 = s0 < 0 ? 0 : (side == 0 ? s0 : tt->d + tt->dtheta + s0);
    a.s0_lo[side] = (float)tt->box[b0][0];
    a.s0_hi[side] = (float)tt->box[b0][1];
    for (int i = 0; i < nst; ++i) {
      TsStepS& st = a.st[side][i];
      const int rpad = im.R_in_pad[side][i], jpc = im.jpc[side][i], kcb = im.kcb[side][i];
      if (rpad > 4 * TS_SPT || im.Npad[side][i] > 256) return false;
      st.hi = im.buf + im.hi_off[side][i];
      st.lo = split ? im.buf + im.lo_off[side][i] : nullptr;
      st.Npad = im.Npad[side][i];
      st.bytes = (uint32_t)st.Npad * kcb;
      st.idesc = instr_desc(fmt_code(fmt), TILE_M, st.Npad);
      st.sbo = 8u * (uint32_t)kcb;
      st.nchunks = im.nchunks[side][i];
      st.jpc = jpc;
      st.R_in_pad = rpad;
      st.spt = rpad / 4;
      st.R_out = cs[i].R_out;
      st.coord = cs[i].coord;
      st.ksteps = jpc * rpad / 16;
      const int bj = side == 0 ? cs[i].coord : tt->d + tt->dtheta + cs[i].coord;
      st.lo_box = (float)tt->box[bj][0];
      st.hi_box = (float)tt->box[bj][1];
      st.a_scale = im.a_scale[side][i];
      st.out_scale = im.out_scale[side][i];
      if (nst > 1 && i == 0) acc1w = std::max(acc1w, st.Npad);
      else acc0w = std::max(acc0w, st.Npad);
      a_part = std::max(a_part, jpc * rpad / 2);
      bslot = std::max(bslot, st.bytes);
      bvl = std::max(bvl, st.nchunks * jpc);
    }
  }
  a.nsteps = nst;
  a.bv_ld = (bvl + 1) | 1;
  const int pad0 = std::max(a.st[0][0].R_in_pad, a.st[1][0].R_in_pad);
  a.ld_seed = pad0 | 1;
  auto r32 = [](int x) { return ((x + 31) / 32) * 32; };
  a.acc1_col = nst > 1 ? r32(acc0w) : 0;
  a.a_col = nst > 1 ? a.acc1_col + r32(acc1w) : r32(acc0w);
  a.a_part_cols = a_part;
  // columns in use; the readback of S may read up to 4 TS_SPT columns past an accumulator's start
  const int need = std::max(a.a_col + NS * parts * a_part, (nst > 1 ? a.acc1_col : 0) + 4 * TS_SPT);
  int cols = 32;
  while (cols < need) cols <<= 1;
  if (cols > 512) return false;
  a.tmem_cols = cols;
  a.b_slot_bytes = bslot;
  const size_t smem = (size_t)NS * parts * bslot +
                      sizeof(float) * ((size_t)2 * TILE_M * a.bv_ld + (size_t)TILE_M * a.ld_seed +
                                       (size_t)NGEN_WARPS * 32 * STAGE_LD) +
                      16 + sizeof(TsStepS) * 6 + 8 * (4 * NS + 2) + 16;
  if (smem > 227 * 1024) return false;
  *smem_out = std::max<size_t>(smem, 116 * 1024);  // one CTA (one TMEM allocation) per SM
  return true;
}

// Grid of the TS kernel: one CTA per SM in clusters of CL, as many clusters as can be
// resident at once (clusters are placed within a GPC, so with CL > 1 a few SMs may stay idle),
// and no more than there are cluster items.
template <int FMT, bool SPLIT, int NS, int CL>
static pttk_status launch_ts(TsArgs a, int64_t T0, int64_t T1, size_t smem, cudaStream_t s) {
  auto kfn = chain_ts_kernel<FMT, SPLIT, NS, CL>;
  PTTK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (CL > 1) PTTK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 0));
  a.T0p = (T0 + CL - 1) / CL * CL;
  a.nitems = (a.T0p + (T1 + CL - 1) / CL * CL) / CL;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  int64_t nclusters = sm_count() / CL;
  if (CL > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)(nclusters * CL));
    int active = 0;
    PTTK_CUDA(cudaOccupancyMaxActiveClusters(&active, kfn, &cfg));
    if (active < 1) return set_error(PTTK_ENOTSUP, "tensor-core chain: no cluster of this size fits");
    nclusters = std::min<int64_t>(nclusters, active);
  }
  nclusters = std::max<int64_t>(1, std::min<int64_t>(nclusters, a.nitems));
  cfg.gridDim = dim3((unsigned)(nclusters * CL));
  PTTK_CUDA(cudaLaunchKernelEx(&cfg, kfn, a));
  pttk::count_launch();
  return PTTK_OK;
}

// Launch arguments of the tensor-memory-A kernel with epilogue warps; false (and no error) when
// the ranks do not fit it: two accumulator regions of the widest step and NSA_TSE A slots in
// 512 TMEM columns, and at least three B slots in shared memory. *nsb_out: the B ring depth
// (3 or 4).
static bool tse_plan(const pttk_tt* tt, const TcImageCache* cache, const Images& im, pttk_prec prec, TsArgs& a,
                     size_t* smem_out, int* nsb_out) {
  if (!ts_plan(tt, cache, im, prec, 1, a, smem_out)) return false;
  const int parts = form_split(prec) ? 2 : 1;
  int npad = 16;
  for (int side = 0; side < 2; ++side)
    for (int i = 0; i < a.nsteps; ++i) npad = std::max(npad, a.st[side][i].Npad);
  a.region_col = ((npad + 31) / 32) * 32;
  a.a_col = 2 * a.region_col;
  if (a.a_col + NSA_TSE * parts * a.a_part_cols > 512) return false;
  a.tmem_cols = 512;
  const size_t fixed = sizeof(float) * ((size_t)2 * TILE_M * a.bv_ld + (size_t)TILE_M * a.ld_seed +
                                        (size_t)NEPI_WARPS * 32 * EPI_LD) +
                       16 + sizeof(TsStepS) * 6 + 8 * (2 * NSA_TSE + 2 * 4 + 6) + 16;
  int nsb = 0;
  for (int k = 4; k >= 3 && !nsb; --k)
    if ((size_t)k * parts * a.b_slot_bytes + fixed <= 227 * 1024) nsb = k;
  if (!nsb) return false;
  *nsb_out = nsb;
  *smem_out = std::max<size_t>((size_t)nsb * parts * a.b_slot_bytes + fixed, 116 * 1024);
  return true;
}

template <int FMT, bool SPLIT, int NSB>
static pttk_status launch_tse(TsArgs a, int64_t T0, int64_t T1, size_t smem, cudaStream_t s) {
  auto kfn = chain_tse_kernel<FMT, SPLIT, NSB>;
  PTTK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  a.T0p = T0;
  a.nitems = T0 + T1;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(a.nitems, sm_count()));
  kfn<<<grid, TCE_THREADS, smem, s>>>(a);
  pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

// Images for (prec, config) exist after this returns (first use lays them out; synchronises).
pttk_status tc_prepare(const pttk_tt* tt, TcImageCache* cache, pttk_prec prec, int cfg, cudaStream_t s) {
  const int fi = form_index(prec);
  if (fi < 0) return set_error(PTTK_EINVAL, "not a tensor-core form");
  int KCB, NS;
  tc_config(prec, cfg, &KCB, &NS);
  Images& im = cache->img[fi][KCB == 64 ? 0 : 1];
  std::lock_guard<std::mutex> lk(g_img_mu);
  PTTK_TRY(ensure_merged(tt, cache));
  if ((ts_config(cfg) || tse_config(cfg)) && ts_form(prec)) {
    Images& ti = cache->ts[fi];
    if (!ti.buf) PTTK_TRY(build_images_ts(tt, cache, prec, ti, s));
    TsArgs probe;
    size_t smem;
    int nsb;
    if (tse_config(cfg) ? tse_plan(tt, cache, ti, prec, probe, &smem, &nsb) : ts_plan(tt, cache, ti, prec, 3, probe, &smem))
      return PTTK_OK;
  }
  if (!im.buf) PTTK_TRY(build_images(tt, cache, prec, KCB, im, s));
  return PTTK_OK;
}

template <int FMT, bool SPLIT, int KCB, int NS>
static pttk_status launch_tc(const TcArgs& a, size_t smem, cudaStream_t s) {
  auto kfn = chain_tc_kernel<FMT, SPLIT, KCB, NS>;
  PTTK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)std::min<int64_t>(a.ntiles, sm_count());
  kfn<<<grid, TC_THREADS, smem, s>>>(a); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

template <int FMT, bool SPLIT, int KCB, int NS>
static pttk_status launch_tce(const TcArgs& a, size_t smem, cudaStream_t s) {
  auto kfn = chain_tce_kernel<FMT, SPLIT, KCB, NS>;
  PTTK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)std::min<int64_t>(a.ntiles, sm_count());
  kfn<<<grid, TCE_THREADS, smem, s>>>(a); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

// Both factors in one persistent launch: U (N_s rows from X) and V (N_t rows from Y).
pttk_status factor_build_tc(const pttk_tt* tt, TcImageCache* cache, const float* X, int64_t N_s,
                            const float* Y, int64_t N_t, pttk_prec prec, float* U, float* V, int* d_status,
                            int cfg, cudaStream_t s) {
  if (N_s == 0 && N_t == 0) return PTTK_OK;
  PTTK_TRY(tc_prepare(tt, cache, prec, cfg, s));
  const int fi = form_index(prec);
  if (tse_config(cfg) && ts_form(prec)) {
    TsArgs a;
    size_t smem = 0;
    int nsb = 0;
    if (tse_plan(tt, cache, cache->ts[fi], prec, a, &smem, &nsb)) {
      a.N[0] = N_s;
      a.N[1] = N_t;
      a.pts[0] = X;
      a.pts[1] = Y;
      a.out[0] = U;
      a.out[1] = V;
      a.status = d_status;
      const int64_t T0 = (N_s + TILE_M - 1) / TILE_M, T1 = (N_t + TILE_M - 1) / TILE_M;
      PTTK_PROF("chain_tc", s);
      const int fmt = form_fmt(prec);
      const bool split = form_split(prec);
#define PTTK_TSE_LAUNCH(F, SP) \
  return nsb == 4 ? launch_tse<F, SP, 4>(a, T0, T1, smem, s) : launch_tse<F, SP, 3>(a, T0, T1, smem, s);
      if (fmt == FMT_BF16) {
        if (split) { PTTK_TSE_LAUNCH(FMT_BF16, true) }
        PTTK_TSE_LAUNCH(FMT_BF16, false)
      }
      if (split) { PTTK_TSE_LAUNCH(FMT_FP16, true) }
      PTTK_TSE_LAUNCH(FMT_FP16, false)
#undef PTTK_TSE_LAUNCH
    }
  }
  if (ts_config(cfg) && ts_form(prec)) {
    const int NS = 3, CL = ts_cluster(cfg);
    TsArgs a;
    size_t smem = 0;
    if (ts_plan(tt, cache, cache->ts[fi], prec, NS, a, &smem)) {
      a.N[0] = N_s;
      a.N[1] = N_t;
      a.pts[0] = X;
      a.pts[1] = Y;
      a.out[0] = U;
      a.out[1] = V;
      a.status = d_status;
      const int64_t T0 = (N_s + TILE_M - 1) / TILE_M, T1 = (N_t + TILE_M - 1) / TILE_M;
      PTTK_PROF("chain_tc", s);
      const int fmt = form_fmt(prec);
      const bool split = form_split(prec);
#define PTTK_TS_LAUNCH(F, SP)                                                            \
  return CL == 4 ? launch_ts<F, SP, 3, 4>(a, T0, T1, smem, s)                            \
                 : CL == 2 ? launch_ts<F, SP, 3, 2>(a, T0, T1, smem, s) : launch_ts<F, SP, 3, 1>(a, T0, T1, smem, s);
      if (fmt == FMT_BF16) {
        if (split) { PTTK_TS_LAUNCH(FMT_BF16, true) }
        PTTK_TS_LAUNCH(FMT_BF16, false)
      }
      if (split) { PTTK_TS_LAUNCH(FMT_FP16, true) }
      PTTK_TS_LAUNCH(FMT_FP16, false)
#undef PTTK_TS_LAUNCH
    }
  }
  int KCB, NS;
  tc_config(prec, cfg, &KCB, &NS);
  const Images& im = cache->img[fi][KCB == 64 ? 0 : 1];
  const int fmt = form_fmt(prec);
  const bool split = form_split(prec);
  TcArgs a{};
  a.nsteps = tt->d;
  a.n = tt->n;
  a.d = tt->d;
  a.N[0] = N_s;
  a.N[1] = N_t;
  a.T0 = (N_s + TILE_M - 1) / TILE_M;
  a.ntiles = a.T0 + (N_t + TILE_M - 1) / TILE_M;
  a.pts[0] = X;
  a.pts[1] = Y;
  a.out[0] = U;
  a.out[1] = V;
  a.status = d_status;
  int npad_max = 16, spad_max = 8;
  for (int side = 0; side < 2; ++side) {
    TcChainStep cs[3];
    int s0;
    a.nsteps = tc_chain_steps(tt, cache, side, cs, &s0);
    a.s0_coord[side] = s0;
    const int b0 = s0 < 0 ? 0 : (side == 0 ? s0 : tt->d + tt->dtheta + s0);
    a.s0_lo[side] = (float)tt->box[b0][0];
    a.s0_hi[side] = (float)tt->box[b0][1];
    for (int i = 0; i < a.nsteps; ++i) {
      const int rin = cs[i].R_in, rout = cs[i].R_out, coord = cs[i].coord;
      TcStep& st = a.st[side][i];
      st.img_hi = im.buf + im.hi_off[side][i];
      st.img_lo = split ? im.buf + im.lo_off[side][i] : nullptr;
      st.nchunks = im.nchunks[side][i];
      st.R_in = rin;
      st.R_in_pad = im.R_in_pad[side][i];
      st.R_out = rout;
      st.Npad = im.Npad[side][i];
      st.coord = coord;
      const int bj = side == 0 ? coord : tt->d + tt->dtheta + coord;
      st.lo = (float)tt->box[bj][0];
      st.hi = (float)tt->box[bj][1];
      st.a_scale = im.a_scale[side][i];
      st.out_scale = im.out_scale[side][i];
      npad_max = std::max(npad_max, st.Npad);
      // S must hold every R_in_pad (read) and, for non-last steps, Npad columns (written)
      spad_max = std::max(spad_max, st.R_in_pad);
      if (i < a.nsteps - 1) spad_max = std::max(spad_max, st.Npad);
    }
  }
  if (npad_max > 256) return set_error(PTTK_ENOTSUP, "tensor-core chain: a rank above 256");
  // row stride of S: a multiple of 4 floats, = 4 (mod 32) so float4 rows fall in distinct banks;
  // it also holds the last step's NGEN_WARPS x 32 x STAGE_LD staging floats
  int ld_s = ((spad_max + 31) / 32) * 32 + 4;
  while ((size_t)TILE_M * ld_s < (size_t)NGEN_WARPS * 32 * STAGE_LD) ld_s += 32;
  a.ld_s = ld_s;
  // the first step's input (Sseed) row stride: its padded width rounded to 8, plus 4, so the
  // 16-byte reads of consecutive rows fall in distinct banks
  int pad0 = 4, npad0 = 16, npad_rest = 16;
  for (int side = 0; side < 2; ++side) {
    pad0 = std::max(pad0, a.st[side][0].R_in_pad);
    npad0 = std::max(npad0, a.st[side][0].Npad);
    for (int i = 1; i < a.nsteps; ++i) npad_rest = std::max(npad_rest, a.st[side][i].Npad);
  }
  a.ld_seed = ((pad0 + 7) / 8) * 8 + 4;
  const int bv_ld = (tt->n + 1) | 1;
  const size_t parts = split ? 2 : 1;
  if (tce_config(cfg) || tse_config(cfg)) {
    // two accumulator regions of the widest step, an epilogue staging tile per epilogue warp
    TcArgs b = a;
    b.ld_s = ((spad_max + 31) / 32) * 32 + 4;
    b.region_col = ((npad_max + 31) / 32) * 32;
    int tcols = 32;
    while (tcols < 2 * b.region_col) tcols <<= 1;
    b.tmem_cols = tcols;
    b.b_slot_bytes = (uint32_t)npad_max * KCB;
    auto smem_tce = [&](int ns) {
      return (size_t)ns * parts * TILE_M * KCB + (size_t)ns * parts * b.b_slot_bytes +
             sizeof(float) * ((size_t)TILE_M * b.ld_s + (size_t)2 * TILE_M * bv_ld + (size_t)TILE_M * b.ld_seed +
                              (size_t)NEPI_WARPS * 32 * STAGE_LD) +
             16 + sizeof(StepS) * 6 + 8 * (3 * ns + 6) + 16;
    };
    // the split forms' {128, 2} ring takes a third slot where shared memory has room for it
    // (ranks up to ~100): each core chunk's TMA then has two chunks of MMAs to land behind
    const bool ring3 = split && KCB == 128 && NS == 2 && smem_tce(3) <= 227 * 1024;
    const size_t smem_e = smem_tce(ring3 ? 3 : NS);
    if (tcols <= 512 && smem_e <= 227 * 1024) {
      const size_t req = std::max<size_t>(smem_e, 116 * 1024);
      PTTK_PROF("chain_tc", s);
#define PTTK_TCE_LAUNCH(F)                                                                                     \
  if (split)                                                                                                   \
    return KCB == 64 ? launch_tce<F, true, 64, 4>(b, req, s)                                                   \
                     : ring3 ? launch_tce<F, true, 128, 3>(b, req, s) : launch_tce<F, true, 128, 2>(b, req, s); \
  return KCB == 128 ? launch_tce<F, false, 128, 4>(b, req, s) : launch_tce<F, false, 64, 4>(b, req, s);
      if (fmt == FMT_BF16) { PTTK_TCE_LAUNCH(FMT_BF16) }
      if (fmt == FMT_FP16) { PTTK_TCE_LAUNCH(FMT_FP16) }
      PTTK_TCE_LAUNCH(FMT_TF32)
#undef PTTK_TCE_LAUNCH
    }
  }
  // TMEM: accumulator 0 at column 0; with two or more steps the first step has its own
  // accumulator after it, so that the next item's first step can run while the last step's
  // accumulator is read out
  a.acc1_col = a.nsteps > 1 ? ((npad_rest + 31) / 32) * 32 : 0;
  const int tmem_need = a.nsteps > 1 ? a.acc1_col + npad0 : npad_max;
  int cols = 32;
  while (cols < tmem_need) cols <<= 1;
  if (cols > 512) return set_error(PTTK_ENOTSUP, "tensor-core chain: accumulators exceed tensor memory");
  a.tmem_cols = cols;
  a.b_slot_bytes = (uint32_t)npad_max * KCB;
  const size_t smem = (size_t)NS * parts * TILE_M * KCB + (size_t)NS * parts * a.b_slot_bytes +
                      sizeof(float) * ((size_t)TILE_M * a.ld_s + (size_t)2 * TILE_M * bv_ld +
                                       (size_t)TILE_M * a.ld_seed) + 16 +
                      sizeof(StepS) * 6 + 8 * (3 * NS + 2) + 16;
  if (smem > 227 * 1024) return set_error(PTTK_ENOTSUP, "tensor-core chain: ranks too large for shared memory");
  const size_t smem_req = std::max<size_t>(smem, 116 * 1024);  // one CTA (one TMEM allocation) per SM
  PTTK_PROF("chain_tc", s);
  // configurations: split forms {128, 2} and {64, 4}; single forms {128, 4} and {64, 4}
#define PTTK_TC_LAUNCH(F)                                                                        \
  if (split) return KCB == 64 ? launch_tc<F, true, 64, 4>(a, smem_req, s) : launch_tc<F, true, 128, 2>(a, smem_req, s); \
  return KCB == 128 ? launch_tc<F, false, 128, 4>(a, smem_req, s) : launch_tc<F, false, 64, 4>(a, smem_req, s);
  if (fmt == FMT_BF16) { PTTK_TC_LAUNCH(FMT_BF16) }
  if (fmt == FMT_FP16) { PTTK_TC_LAUNCH(FMT_FP16) }
  PTTK_TC_LAUNCH(FMT_TF32)
#undef PTTK_TC_LAUNCH
}

}  // namespace pttk

namespace pttk {
namespace {
// One thread waits, with the kernels' bounded wait, on an mbarrier that nothing arrives on:
// the wait must give up (after ~2 s) and the kernel must report PTTK_ETIMEOUT and return.
__global__ void selftest_wait_kernel(int* __restrict__ status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    fence_mbar_init();
    const bool ok = mbar_wait(&bar, 0, &abort_flag);
    *status = ok ? (int)PTTK_OK : (int)PTTK_ETIMEOUT;
  }
}
}  // namespace
}  // namespace pttk

extern "C" pttk_status pttk_selftest_wait_timeout(void* stream) {
  using namespace pttk;
  clear_error();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* d_status = nullptr;
  PTTK_CUDA(cudaMalloc(&d_status, sizeof(int)));
  PTTK_CUDA(cudaMemsetAsync(d_status, 0xff, sizeof(int), s));
  selftest_wait_kernel<<<1, 32, 0, s>>>(d_status); pttk::count_launch();
  int h = -1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_status);
  if (e != cudaSuccess) return cuda_error(e, "self-test of the bounded wait");
  if (h == (int)PTTK_ETIMEOUT) return set_error(PTTK_ETIMEOUT, "self-test: the bounded wait gave up as it should");
  return set_error(PTTK_ECUDA, "self-test: the bounded wait did not give up");
}
