// Batched online stage: B instances (theta_b, X_b, Y_b) of one TT in one call.
//
// The factor rows of Algorithm 2, Phase 3 depend only on the point and the TT, never on
// theta, so the factors of all instances are one chain over the concatenated source points
// and one over the concatenated target points; the tensor-core form builds both in a single
// persistent launch whose 128-point tiles may straddle instances (every tile costs the same,
// so instance sizes that vary 100x need no scheduling). Only H(theta_b) (Eq. hmat,
// Algorithm 3) is per instance: one launch contracts every instance's theta cores.
//
// A plan (pttk_batch) owns everything that needs allocating or synchronising (core images,
// the scratch of two-parameter H products), so pttk_instantiate_batched only enqueues kernels
// and can be captured in a CUDA graph.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "pttk_internal.cuh"

struct pttk_tt_ext;  // defined in api.cu

namespace pttk {
TcImageCache* tt_tc_cache(const pttk_tt* tt);

namespace {

// out[b][a + ra c] = sum_k G[a + ra (k + n c)] T_k(thetahat_b), thetahat_b from thetas[b * dth + j]
// on the box [lo, hi] with the printed interval map; theta outside the box (beyond a 1e-12
// relative slack) records PTTK_EDOMAIN in *status.
__global__ void theta_contract_batched(const double* __restrict__ G, int ra, int n, int rb,
                                       const double* __restrict__ thetas, int B, int dth, int j,
                                       double lo, double hi, double* __restrict__ out,
                                       int* __restrict__ status) {
  const int64_t per = (int64_t)ra * rb;
  const int64_t total = per * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / per);
    const int64_t q = e % per;
    const int64_t a = q % ra, c = q / ra;
    const double th = thetas[(int64_t)b * dth + j];
    const double slack = 1e-12 * (hi - lo);
    if ((th < lo - slack || th > hi + slack) && q == 0) atomicExch(status, (int)PTTK_EDOMAIN);
    const double x = (2.0 * th - lo - hi) / (lo - hi);
    const double* g = G + a + (int64_t)ra * n * c;
    double t0 = 1.0, t1 = x, acc = g[0];
    if (n > 1) acc = fma(g[(int64_t)ra], t1, acc);
    for (int k = 2; k < n; ++k) {
      const double t2 = 2.0 * x * t1 - t0;
      acc = fma(g[(int64_t)ra * k], t2, acc);
      t0 = t1;
      t1 = t2;
    }
    out[e] = acc;
  }
}

// H[b] = H1[b] (ra x rm) * H2[b] (rm x rb), all column-major per instance
__global__ void batched_product(const double* __restrict__ H1, const double* __restrict__ H2, int ra, int rm,
                                int rb, int B, double* __restrict__ H) {
  const int64_t per = (int64_t)ra * rb;
  const int64_t total = per * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / per);
    const int64_t q = e % per;
    const int64_t a = q % ra, c = q / ra;
    const double* x = H1 + (int64_t)b * ra * rm + a;
    const double* y = H2 + (int64_t)b * rm * rb + c * rm;
    double acc = 0.0;
    for (int m = 0; m < rm; ++m) acc = fma(x[(int64_t)m * ra], y[m], acc);
    H[e] = acc;
  }
}

// H[b] = identity (r x r): kernels without a parameter (d_theta = 0) have H(theta) = I
__global__ void identity_batched(int r, int B, double* __restrict__ H) {
  const int64_t total = (int64_t)B * r * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e % ((int64_t)r * r);
    H[e] = (q % r == q / r) ? 1.0 : 0.0;
  }
}

// M[b] row-major (rs x rt) from H[b] column-major
template <typename T>
__global__ void store_batched_rowmajor(const double* __restrict__ H, int rs, int rt, int B, T* __restrict__ M) {
  const int64_t per = (int64_t)rs * rt;
  const int64_t total = per * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / per, q = e % per;
    const int64_t a = q / rt, c = q % rt;
    M[e] = (T)H[b * per + a + (int64_t)rs * c];
  }
}

unsigned blocks_for(int64_t work) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)sm_count() * 8));
}

}  // namespace
}  // namespace pttk

struct pttk_batch {
  const pttk_tt* tt = nullptr;
  int B = 0;
  int64_t Ns = 0, Nt = 0;
  pttk_prec prec = PTTK_FP32;
  int cfg = 0;
  double* scratch = nullptr;  // H products (FP64)
  size_t scratch_elems = 0;
};

using namespace pttk;

static bool tc_form(pttk_prec p) {
  return p >= PTTK_TF32 && p <= PTTK_FP16X3;
}

extern "C" {

pttk_status pttk_batch_create(const pttk_tt* tt, int B, const int64_t* xoff, const int64_t* yoff,
                              pttk_prec prec, void* stream, pttk_batch** out) {
  clear_error();
  if (!out) return set_error(PTTK_EINVAL, "NULL out");
  *out = nullptr;
  if (!tt || !xoff || !yoff) return set_error(PTTK_EINVAL, "NULL argument");
  if (B < 1) return set_error(PTTK_EINVAL, "B must be >= 1");
  if (prec < PTTK_FP64 || prec > PTTK_FP16X3) return set_error(PTTK_EINVAL, "unknown precision");
  if (xoff[0] != 0 || yoff[0] != 0) return set_error(PTTK_EINVAL, "offsets must start at 0");
  for (int b = 0; b < B; ++b)
    if (xoff[b + 1] < xoff[b] || yoff[b + 1] < yoff[b]) return set_error(PTTK_EINVAL, "offsets must not decrease");
  pttk_batch* p = new pttk_batch();
  p->tt = tt;
  p->B = B;
  p->Ns = xoff[B];
  p->Nt = yoff[B];
  p->prec = prec;
  const int d = tt->d, dth = tt->dtheta;
  size_t elems = (size_t)B * tt->ranks[d] * tt->ranks[d + dth];
  if (dth == 2)
    elems += (size_t)B * ((size_t)tt->ranks[d] * tt->ranks[d + 1] + (size_t)tt->ranks[d + 1] * tt->ranks[d + 2]);
  p->scratch_elems = elems;
  cudaError_t e = cudaMalloc(&p->scratch, sizeof(double) * std::max<size_t>(elems, 1));
  if (e != cudaSuccess) {
    delete p;
    return cuda_error(e, "cudaMalloc(batch scratch)");
  }
  if (tc_form(prec)) {
    const pttk_status st = tc_prepare(tt, tt_tc_cache(tt), prec, 0, as_stream(stream));
    if (st != PTTK_OK) {
      cudaFree(p->scratch);
      delete p;
      return st;
    }
  }
  *out = p;
  return PTTK_OK;
}

pttk_status pttk_batch_set_config(pttk_batch* b, int cfg) {
  clear_error();
  if (!b) return set_error(PTTK_EINVAL, "NULL batch");
  if (cfg < 0 || cfg >= tc_config_count()) return set_error(PTTK_EINVAL, "no such launch configuration");
  if (tc_form(b->prec)) PTTK_TRY(tc_prepare(b->tt, tt_tc_cache(b->tt), b->prec, cfg, nullptr));
  b->cfg = cfg;
  return PTTK_OK;
}

pttk_status pttk_batch_get_config(const pttk_batch* b, int* cfg, int* n_configs) {
  clear_error();
  if (!b) return set_error(PTTK_EINVAL, "NULL batch");
  if (cfg) *cfg = b->cfg;
  if (n_configs) *n_configs = tc_form(b->prec) ? tc_config_count() : 1;
  return PTTK_OK;
}

pttk_status pttk_batch_autotune(pttk_batch* b, const void* X, const void* Y, void* U, void* V, float* ms_out,
                                void* stream) {
  clear_error();
  if (!b) return set_error(PTTK_EINVAL, "NULL batch");
  const int nc = tc_form(b->prec) ? tc_config_count() : 1;
  if (nc == 1) {
    if (ms_out) ms_out[0] = 0.f;
    b->cfg = 0;
    return PTTK_OK;
  }
  cudaStream_t s = as_stream(stream);
  const int* st = tt_status_word(b->tt);
  (void)st;
  cudaEvent_t e0, e1;
  PTTK_CUDA(cudaEventCreate(&e0));
  PTTK_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_cfg = 0;
  pttk_status rs = PTTK_OK;
  for (int c = 0; c < nc && rs == PTTK_OK; ++c) {
    rs = tc_prepare(b->tt, tt_tc_cache(b->tt), b->prec, c, s);
    if (rs != PTTK_OK) break;
    float total = 0.f;
    for (int rep = 0; rep < 4 && rs == PTTK_OK; ++rep) {
      cudaEventRecord(e0, s);
      rs = factor_build_tc(b->tt, tt_tc_cache(b->tt), static_cast<const float*>(X), b->Ns,
                           static_cast<const float*>(Y), b->Nt, b->prec, static_cast<float*>(U),
                           static_cast<float*>(V), tt_status_word(b->tt), c, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) total += ms;  // first run is a warm-up
    }
    const float avg = total / 3.f;
    if (ms_out) ms_out[c] = avg;
    if (avg < best) {
      best = avg;
      best_cfg = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rs != PTTK_OK) return rs;
  b->cfg = best_cfg;
  return PTTK_OK;
}

pttk_status pttk_instantiate_batched(const pttk_batch* b, const double* thetas, const void* X, const void* Y,
                                     void* U, void* M, void* V, void* stream) {
  clear_error();
  if (!b || !M || (b->tt->dtheta > 0 && !thetas)) return set_error(PTTK_EINVAL, "NULL argument");
  if ((b->Ns > 0 && (!X || !U)) || (b->Nt > 0 && (!Y || !V))) return set_error(PTTK_EINVAL, "NULL point or factor buffer");
  const pttk_tt* tt = b->tt;
  cudaStream_t s = as_stream(stream);
  const int d = tt->d, dth = tt->dtheta, n = tt->n, B = b->B;
  const int rs = tt->ranks[d], rt = tt->ranks[d + dth];
  int* status = tt_status_word(tt);
  const double* H = nullptr;
  double* Hout = b->scratch;
  if (dth == 0) {
    identity_batched<<<blocks_for((int64_t)B * rs * rt), 256, 0, s>>>(rs, B, Hout); pttk::count_launch();
    H = Hout;
  } else if (dth == 1) {
    theta_contract_batched<<<blocks_for((int64_t)B * rs * rt), 256, 0, s>>>(
        tt->cores64 + tt->core_off[d], rs, n, rt, thetas, B, 1, 0, tt->box[d][0], tt->box[d][1], Hout, status); pttk::count_launch();
    H = Hout;
  } else {
    const int rm = tt->ranks[d + 1];
    double* H1 = Hout + (size_t)B * rs * rt;
    double* H2 = H1 + (size_t)B * rs * rm;
    theta_contract_batched<<<blocks_for((int64_t)B * rs * rm), 256, 0, s>>>(
        tt->cores64 + tt->core_off[d], rs, n, rm, thetas, B, 2, 0, tt->box[d][0], tt->box[d][1], H1, status); pttk::count_launch();
    theta_contract_batched<<<blocks_for((int64_t)B * rm * rt), 256, 0, s>>>(
        tt->cores64 + tt->core_off[d + 1], rm, n, rt, thetas, B, 2, 1, tt->box[d + 1][0], tt->box[d + 1][1], H2,
        status); pttk::count_launch();
    batched_product<<<blocks_for((int64_t)B * rs * rt), 256, 0, s>>>(H1, H2, rs, rm, rt, B, Hout); pttk::count_launch();
    H = Hout;
  }
  if (b->prec == PTTK_FP64)
    { store_batched_rowmajor<double><<<blocks_for((int64_t)B * rs * rt), 256, 0, s>>>(H, rs, rt, B, static_cast<double*>(M)); pttk::count_launch(); }
  else
    { store_batched_rowmajor<float><<<blocks_for((int64_t)B * rs * rt), 256, 0, s>>>(H, rs, rt, B, static_cast<float*>(M)); pttk::count_launch(); }
  PTTK_CUDA(cudaGetLastError());
  PTTK_TRY(point_domain_check(tt, X, b->Ns, Y, b->Nt, b->prec == PTTK_FP64, status, s));
  if (tc_form(b->prec))
    return factor_build_tc(tt, tt_tc_cache(tt), static_cast<const float*>(X), b->Ns, static_cast<const float*>(Y),
                           b->Nt, b->prec, static_cast<float*>(U), static_cast<float*>(V), status, b->cfg, s);
  PTTK_TRY(factor_build_run(tt, true, X, b->Ns, b->prec, U, s));
  PTTK_TRY(factor_build_run(tt, false, Y, b->Nt, b->prec, V, s));
  return PTTK_OK;
}

void pttk_batch_free(pttk_batch* b) {
  if (!b) return;
  if (b->scratch) cudaFree(b->scratch);
  delete b;
}

}  // extern "C"
