// C-ABI entry points of libpttk (declared and documented in include/pttk.h).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "pttk_internal.cuh"

namespace pttk {

static thread_local std::string g_error;

pttk_status set_error(pttk_status s, const std::string& msg) {
  g_error = msg;
  return s;
}

pttk_status cuda_error(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a non-sticky error so the context stays usable
  const pttk_status s = (e == cudaErrorMemoryAllocation) ? PTTK_ENOMEM : PTTK_ECUDA;
  return set_error(s, std::string(what) + ": " + cudaGetErrorString(e));
}

void clear_error() { g_error.clear(); }

int sm_count() {
  static int count[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!count[dev]) {
    int c = 0;
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    count[dev] = c > 0 ? c : 1;
  }
  return count[dev];
}

// Target-side cores transposed to (right rank, j, left rank) so both factor chains read
// their cores as (input rank, j, output rank).
__global__ void orient_kernel(const double* __restrict__ G, int ra, int n, int rb,
                              double* __restrict__ out64, float* __restrict__ out32) {
  const int64_t total = (int64_t)ra * n * rb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e % ra, j = (e / ra) % n, b = e / ((int64_t)ra * n);
    const int64_t o = b + rb * (j + (int64_t)n * a);
    out64[o] = G[e];
    out32[o] = (float)G[e];
  }
}

}  // namespace pttk

// Handles keep their target-side oriented cores next to the cores (allocated together).
struct pttk_tt_ext : pttk_tt {
  double* tgt64 = nullptr;
  float* tgt32 = nullptr;
  pttk::TcImageCache* tc = nullptr;  // tensor-core core images, built on first use per form
  int* dstatus = nullptr;            // device status word (bounded waits that ran out)
};

namespace pttk {

int* tt_status_word(const pttk_tt* tt) { return static_cast<const pttk_tt_ext*>(tt)->dstatus; }
TcImageCache* tt_tc_cache(const pttk_tt* tt) { return static_cast<const pttk_tt_ext*>(tt)->tc; }

const void* oriented_core_ptr(const pttk_tt* tt, bool source, int k, bool fp64) {
  const pttk_tt_ext* t = static_cast<const pttk_tt_ext*>(tt);
  if (source) return fp64 ? (const void*)(t->cores64 + t->core_off[k]) : (const void*)(t->cores32 + t->core_off[k]);
  return fp64 ? (const void*)(t->tgt64 + t->core_off[k]) : (const void*)(t->tgt32 + t->core_off[k]);
}

static pttk_status prepare_oriented(pttk_tt_ext* t, cudaStream_t s) {
  t->tc = tc_cache_new();
  PTTK_CUDA(cudaMalloc(&t->dstatus, sizeof(int)));
  PTTK_CUDA(cudaMemsetAsync(t->dstatus, 0, sizeof(int), s));
  PTTK_CUDA(cudaMalloc(&t->tgt64, sizeof(double) * std::max<size_t>(t->core_total, 1)));
  PTTK_CUDA(cudaMalloc(&t->tgt32, sizeof(float) * std::max<size_t>(t->core_total, 1)));
  for (int k = t->d + t->dtheta; k < t->D; ++k) {
    const int64_t total = (int64_t)t->core_elems(k);
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, sm_count() * 8);
    orient_kernel<<<blocks, 256, 0, s>>>(t->cores64 + t->core_off[k], t->ranks[k], t->n,
                                         t->ranks[k + 1], t->tgt64 + t->core_off[k],
                                         t->tgt32 + t->core_off[k]); pttk::count_launch();
  }
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

static void free_handle(pttk_tt_ext* t) {
  if (!t) return;
  if (t->cores64) cudaFree(t->cores64);
  if (t->cores32) cudaFree(t->cores32);
  if (t->tgt64) cudaFree(t->tgt64);
  if (t->tgt32) cudaFree(t->tgt32);
  if (t->dstatus) cudaFree(t->dstatus);
  tc_cache_free(t->tc);
  delete t;
}

static pttk_status check_problem(int kernel, int d, const double* src_box, const double* tgt_box,
                                 int d_theta, const double* theta_box, int n, bool whole_grid = true) {
  if (kernel < PTTK_GAUSS || kernel > PTTK_THIN_PLATE) return set_error(PTTK_EINVAL, "unknown kernel");
  if (d < 1 || d > 3) return set_error(PTTK_EINVAL, "d must be 1, 2 or 3");
  const int need_dth = kernel_dtheta(kernel);
  if (d_theta != need_dth)
    return set_error(PTTK_EINVAL, need_dth == 2   ? "the general-nu Matern kernel takes theta = (l, nu): d_theta = 2"
                                  : need_dth == 1 ? "this kernel takes theta = (l): d_theta = 1"
                                                  : "this kernel has no parameter: d_theta = 0");
  if (n < 2 || n > PTTK_MAX_N) return set_error(PTTK_EINVAL, "n must be in [2, 32]");
  if (!src_box || !tgt_box || (d_theta > 0 && !theta_box)) return set_error(PTTK_EINVAL, "NULL box");
  double gap2 = 0.0;  // squared distance between the source and target boxes
  for (int j = 0; j < d; ++j) {
    if (!(src_box[2 * j] < src_box[2 * j + 1]) || !(tgt_box[2 * j] < tgt_box[2 * j + 1]))
      return set_error(PTTK_EINVAL, "box with lo >= hi");
    if (!std::isfinite(src_box[2 * j]) || !std::isfinite(src_box[2 * j + 1]) || !std::isfinite(tgt_box[2 * j]) ||
        !std::isfinite(tgt_box[2 * j + 1]))
      return set_error(PTTK_EINVAL, "box ends must be finite");
    const double g = std::max({0.0, tgt_box[2 * j] - src_box[2 * j + 1], src_box[2 * j] - tgt_box[2 * j + 1]});
    gap2 += g * g;
  }
  if (d_theta == 0 && !(gap2 > 0.0))
    return set_error(PTTK_EINVAL, "this kernel is singular at r = 0: the boxes must be apart (dist > 0)");
  for (int j = 0; j < d_theta; ++j) {
    if (!(theta_box[2 * j] < theta_box[2 * j + 1])) return set_error(PTTK_EINVAL, "theta box with lo >= hi");
    if (!std::isfinite(theta_box[2 * j]) || !std::isfinite(theta_box[2 * j + 1]))
      return set_error(PTTK_EINVAL, "box ends must be finite");
  }
  if (d_theta > 0 && !(theta_box[0] > 0.0)) return set_error(PTTK_EINVAL, "length scale box must be positive");
  if (kernel == PTTK_MATERN_NU && !(theta_box[2] > 0.0))
    return set_error(PTTK_EINVAL, "nu box must be positive");
  double prod = 1.0;
  for (int j = 0; j < 2 * d + d_theta; ++j) prod *= n;
  if (whole_grid && prod > 4e9) return set_error(PTTK_EINVAL, "n^D above 4e9 entries");
  return PTTK_OK;
}

static void fill_meta(pttk_tt* t, int kernel, int d, const double* src_box, const double* tgt_box,
                      int d_theta, const double* theta_box, int n) {
  t->kernel = kernel;
  t->d = d;
  t->dtheta = d_theta;
  t->D = 2 * d + d_theta;
  t->n = n;
  for (int j = 0; j < d; ++j) {
    t->box[j][0] = src_box[2 * j];
    t->box[j][1] = src_box[2 * j + 1];
    t->box[d + d_theta + j][0] = tgt_box[2 * j];
    t->box[d + d_theta + j][1] = tgt_box[2 * j + 1];
  }
  for (int j = 0; j < d_theta; ++j) {
    t->box[d + j][0] = theta_box[2 * j];
    t->box[d + j][1] = theta_box[2 * j + 1];
  }
  cudaGetDevice(&t->device);
}

static int64_t grid_elems(int n, int D) {
  int64_t t = 1;
  for (int j = 0; j < D; ++j) t *= n;
  return t;
}

// TT-SVD from an owned FP64 work buffer
static pttk_status from_work(pttk_tt_ext* t, double* X, double tol, cudaStream_t s) {
  PTTK_TRY(tt_svd_run(t, X, tol, s));
  PTTK_TRY(prepare_oriented(t, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  return PTTK_OK;
}

pttk_status theta_hat(const pttk_tt* tt, const double* theta, double* th) {
  if (!theta && tt->dtheta > 0) return set_error(PTTK_EINVAL, "NULL theta");
  for (int j = 0; j < tt->dtheta; ++j) {
    const double lo = tt->box[tt->d + j][0], hi = tt->box[tt->d + j][1];
    const double slack = 1e-12 * (hi - lo);
    if (!(theta[j] >= lo - slack && theta[j] <= hi + slack)) {
      char buf[160];
      snprintf(buf, sizeof buf, "theta[%d] = %.17g outside its box [%.17g, %.17g]", j, theta[j], lo, hi);
      return set_error(PTTK_EDOMAIN, buf);
    }
    th[j] = (2.0 * theta[j] - lo - hi) / (lo - hi);  // phi^{-1} for the printed map
  }
  return PTTK_OK;
}

}  // namespace pttk

using namespace pttk;

extern "C" {

const char* pttk_last_error(void) { return g_error.c_str(); }

int pttk_version(void) { return 100; }

pttk_status pttk_grid_coeffs(pttk_kernel kernel, int d, const double* src_box,
                             const double* tgt_box, int d_theta, const double* theta_box, int n,
                             pttk_prec grid_prec, void* C, void* stream) {
  clear_error();
  PTTK_TRY(check_problem(kernel, d, src_box, tgt_box, d_theta, theta_box, n));
  if (grid_prec != PTTK_FP64 && grid_prec != PTTK_FP32)
    return set_error(PTTK_EINVAL, "grid precision must be FP64 or FP32");
  if (!C) return set_error(PTTK_EINVAL, "NULL output");
  pttk_tt meta;
  fill_meta(&meta, kernel, d, src_box, tgt_box, d_theta, theta_box, n);
  return grid_coeffs_launch(kernel, d, d_theta, n, meta.box, grid_prec == PTTK_FP64, C,
                            as_stream(stream));
}

pttk_status pttk_grid_entries(pttk_kernel kernel, int d, const double* src_box,
                              const double* tgt_box, int d_theta, const double* theta_box, int n,
                              const int32_t* idx, int64_t M, pttk_prec prec, void* out, void* stream) {
  clear_error();
  PTTK_TRY(check_problem(kernel, d, src_box, tgt_box, d_theta, theta_box, n, false));
  if (prec != PTTK_FP64 && prec != PTTK_FP32) return set_error(PTTK_EINVAL, "entry precision must be FP64 or FP32");
  if (M < 0) return set_error(PTTK_EINVAL, "negative entry count");
  if (M > 0 && (!idx || !out)) return set_error(PTTK_EINVAL, "NULL index or output buffer");
  if (M == 0) return PTTK_OK;
  pttk_tt meta;
  fill_meta(&meta, kernel, d, src_box, tgt_box, d_theta, theta_box, n);
  cudaStream_t s = as_stream(stream);
  int* dstat = nullptr;
  PTTK_CUDA(cudaMallocAsync(&dstat, sizeof(int), s));
  pttk_status st = PTTK_OK;
  int h = 0;
  if (cudaMemsetAsync(dstat, 0, sizeof(int), s) != cudaSuccess) st = cuda_error(cudaGetLastError(), "memset");
  if (st == PTTK_OK)
    st = grid_entries_launch(kernel, d, d_theta, n, meta.box, idx, M, prec == PTTK_FP64, out, dstat, s);
  if (st == PTTK_OK) {
    const cudaError_t e = cudaMemcpyAsync(&h, dstat, sizeof(int), cudaMemcpyDeviceToHost, s);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    if (e != cudaSuccess || e2 != cudaSuccess) st = cuda_error(e != cudaSuccess ? e : e2, "grid entries");
  }
  cudaFreeAsync(dstat, s);
  if (st != PTTK_OK) return st;
  if (h != 0) return set_error(PTTK_EINVAL, "a multi-index lies outside [0, n)");
  return PTTK_OK;
}

pttk_status pttk_tt_from_coeffs(pttk_kernel kernel, int d, const double* src_box,
                                const double* tgt_box, int d_theta, const double* theta_box,
                                int n, double tol, const void* C, pttk_prec c_prec,
                                void* stream, pttk_tt** out) {
  clear_error();
  if (!out) return set_error(PTTK_EINVAL, "NULL out");
  *out = nullptr;
  PTTK_TRY(check_problem(kernel, d, src_box, tgt_box, d_theta, theta_box, n));
  if (!(tol > 0.0)) return set_error(PTTK_EINVAL, "tol must be positive");
  if (!C) return set_error(PTTK_EINVAL, "NULL coefficient tensor");
  if (c_prec != PTTK_FP64 && c_prec != PTTK_FP32)
    return set_error(PTTK_EINVAL, "coefficient precision must be FP64 or FP32");
  cudaStream_t s = as_stream(stream);
  pttk_tt_ext* t = new pttk_tt_ext();
  fill_meta(t, kernel, d, src_box, tgt_box, d_theta, theta_box, n);
  const int64_t total = grid_elems(n, t->D);
  double* X = nullptr;
  cudaError_t e = cudaMalloc(&X, sizeof(double) * total);
  if (e != cudaSuccess) {
    free_handle(t);
    return cuda_error(e, "cudaMalloc(work)");
  }
  pttk_status st;
  if (c_prec == PTTK_FP64) {
    e = cudaMemcpyAsync(X, C, sizeof(double) * total, cudaMemcpyDeviceToDevice, s);
    st = e == cudaSuccess ? PTTK_OK : cuda_error(e, "cudaMemcpyAsync");
  } else {
    st = widen_to_f64(static_cast<const float*>(C), total, X, s);
  }
  if (st == PTTK_OK) st = from_work(t, X, tol, s);
  cudaFree(X);
  if (st != PTTK_OK) {
    free_handle(t);
    return st;
  }
  *out = t;
  return PTTK_OK;
}

pttk_status pttk_build_offline(pttk_kernel kernel, int d, const double* src_box,
                               const double* tgt_box, int d_theta, const double* theta_box,
                               int n, double tol, pttk_prec grid_prec, void* stream,
                               pttk_tt** out) {
  clear_error();
  if (!out) return set_error(PTTK_EINVAL, "NULL out");
  *out = nullptr;
  PTTK_TRY(check_problem(kernel, d, src_box, tgt_box, d_theta, theta_box, n));
  if (!(tol > 0.0)) return set_error(PTTK_EINVAL, "tol must be positive");
  if (grid_prec != PTTK_FP64 && grid_prec != PTTK_FP32)
    return set_error(PTTK_EINVAL, "grid precision must be FP64 or FP32");
  cudaStream_t s = as_stream(stream);
  pttk_tt_ext* t = new pttk_tt_ext();
  fill_meta(t, kernel, d, src_box, tgt_box, d_theta, theta_box, n);
  const int64_t total = grid_elems(n, t->D);
  double* X = nullptr;
  float* Cf = nullptr;
  cudaError_t e = cudaMalloc(&X, sizeof(double) * total);
  if (e == cudaSuccess && grid_prec == PTTK_FP32) e = cudaMalloc(&Cf, sizeof(float) * total);
  pttk_status st = e == cudaSuccess ? PTTK_OK : cuda_error(e, "cudaMalloc(grid)");
  if (st == PTTK_OK) {
    if (grid_prec == PTTK_FP64) {
      st = grid_coeffs_launch(kernel, d, d_theta, n, t->box, true, X, s);
    } else {
      st = grid_coeffs_launch(kernel, d, d_theta, n, t->box, false, Cf, s);
      if (st == PTTK_OK) st = widen_to_f64(Cf, total, X, s);
    }
  }
  if (st == PTTK_OK) st = from_work(t, X, tol, s);
  if (X) cudaFree(X);
  if (Cf) cudaFree(Cf);
  if (st != PTTK_OK) {
    free_handle(t);
    return st;
  }
  *out = t;
  return PTTK_OK;
}

pttk_status pttk_tt_dims(const pttk_tt* tt, int* d, int* d_theta, int* n, int* kernel) {
  clear_error();
  if (!tt) return set_error(PTTK_EINVAL, "NULL handle");
  if (d) *d = tt->d;
  if (d_theta) *d_theta = tt->dtheta;
  if (n) *n = tt->n;
  if (kernel) *kernel = tt->kernel;
  return PTTK_OK;
}

pttk_status pttk_tt_ranks(const pttk_tt* tt, int* ranks) {
  clear_error();
  if (!tt || !ranks) return set_error(PTTK_EINVAL, "NULL argument");
  for (int k = 0; k <= tt->D; ++k) ranks[k] = tt->ranks[k];
  return PTTK_OK;
}

pttk_status pttk_tt_get_core(const pttk_tt* tt, int k, double* host_out) {
  clear_error();
  if (!tt || !host_out) return set_error(PTTK_EINVAL, "NULL argument");
  if (k < 0 || k >= tt->D) return set_error(PTTK_EINVAL, "core index out of range");
  PTTK_CUDA(cudaMemcpy(host_out, tt->cores64 + tt->core_off[k], sizeof(double) * tt->core_elems(k),
                       cudaMemcpyDeviceToHost));
  return PTTK_OK;
}

static const char kMagic[8] = {'P', 'T', 'T', 'K', 'T', 'T', '0', '1'};

pttk_status pttk_tt_save(const pttk_tt* tt, const char* path) {
  clear_error();
  if (!tt || !path) return set_error(PTTK_EINVAL, "NULL argument");
  std::vector<double> host(tt->core_total);
  PTTK_CUDA(cudaMemcpy(host.data(), tt->cores64, sizeof(double) * tt->core_total, cudaMemcpyDeviceToHost));
  FILE* f = fopen(path, "wb");
  if (!f) return set_error(PTTK_EINVAL, std::string("cannot open ") + path);
  int32_t hdr[5] = {tt->kernel, tt->d, tt->dtheta, tt->n, tt->D};
  bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof hdr, 1, f) == 1;
  for (int j = 0; ok && j < tt->D; ++j) ok = fwrite(tt->box[j], sizeof(double), 2, f) == 2;
  for (int k = 0; ok && k <= tt->D; ++k) {
    const int32_t r = tt->ranks[k];
    ok = fwrite(&r, sizeof r, 1, f) == 1;
  }
  if (ok && tt->core_total) ok = fwrite(host.data(), sizeof(double), host.size(), f) == host.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? PTTK_OK : set_error(PTTK_EINVAL, std::string("write failed: ") + path);
}

// Copies host FP64 cores (packed in core order, each column-major) into a handle whose
// metadata and ranks are set, and prepares its FP32 and oriented copies. Frees the handle
// on failure.
static pttk_status upload_cores(pttk_tt_ext* t, const double* host, pttk_tt** out) {
  size_t off = 0;
  for (int k = 0; k < t->D; ++k) {
    t->core_off[k] = off;
    off += t->core_elems(k);
  }
  t->core_total = off;
  cudaGetDevice(&t->device);
  cudaError_t e = cudaMalloc(&t->cores64, sizeof(double) * t->core_total);
  if (e == cudaSuccess) e = cudaMalloc(&t->cores32, sizeof(float) * t->core_total);
  if (e == cudaSuccess)
    e = cudaMemcpy(t->cores64, host, sizeof(double) * t->core_total, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    std::vector<float> h32(host, host + t->core_total);
    e = cudaMemcpy(t->cores32, h32.data(), sizeof(float) * t->core_total, cudaMemcpyHostToDevice);
  }
  pttk_status st = e == cudaSuccess ? prepare_oriented(t, 0) : cuda_error(e, "uploading cores");
  if (st == PTTK_OK) {
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_error(e, "uploading cores");
  }
  if (st != PTTK_OK) {
    free_handle(t);
    return st;
  }
  *out = t;
  return PTTK_OK;
}

pttk_status pttk_tt_load(const char* path, pttk_tt** out) {
  clear_error();
  if (!path || !out) return set_error(PTTK_EINVAL, "NULL argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(PTTK_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  int32_t hdr[5];
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 && fread(hdr, sizeof hdr, 1, f) == 1;
  pttk_tt_ext* t = new pttk_tt_ext();
  if (ok) {
    t->kernel = hdr[0];
    t->d = hdr[1];
    t->dtheta = hdr[2];
    t->n = hdr[3];
    t->D = hdr[4];
    ok = t->d >= 1 && t->d <= 3 && t->dtheta >= 0 && t->dtheta <= 2 && t->D == 2 * t->d + t->dtheta &&
         t->n >= 2 && t->n <= PTTK_MAX_N && t->kernel >= 0 && t->kernel <= PTTK_THIN_PLATE &&
         t->dtheta == kernel_dtheta(t->kernel);
  }
  for (int j = 0; ok && j < t->D; ++j) ok = fread(t->box[j], sizeof(double), 2, f) == 2;
  for (int k = 0; ok && k <= t->D; ++k) {
    int32_t r;
    ok = fread(&r, sizeof r, 1, f) == 1 && r >= 1 && r <= (1 << 20);
    t->ranks[k] = r;
  }
  ok = ok && t->ranks[0] == 1 && t->ranks[t->D] == 1;
  std::vector<double> host;
  if (ok) {
    size_t total = 0;
    for (int k = 0; k < t->D; ++k) total += t->core_elems(k);
    host.resize(total);
    ok = fread(host.data(), sizeof(double), total, f) == total;
  }
  fclose(f);
  if (!ok) {
    delete t;
    return set_error(PTTK_EINVAL, std::string("not a valid TT file: ") + path);
  }
  return upload_cores(t, host.data(), out);
}

pttk_status pttk_tt_from_cores(pttk_kernel kernel, int d, const double* src_box, const double* tgt_box,
                               int d_theta, const double* theta_box, int n, const int* ranks,
                               const double* cores, pttk_tt** out) {
  clear_error();
  if (!out || !ranks || !cores) return set_error(PTTK_EINVAL, "NULL argument");
  *out = nullptr;
  PTTK_TRY(check_problem(kernel, d, src_box, tgt_box, d_theta, theta_box, n, false));
  const int D = 2 * d + d_theta;
  if (ranks[0] != 1 || ranks[D] != 1) return set_error(PTTK_EINVAL, "ranks[0] and ranks[D] must be 1");
  for (int k = 1; k < D; ++k)
    if (ranks[k] < 1 || ranks[k] > (1 << 20)) return set_error(PTTK_EINVAL, "TT rank out of range");
  pttk_tt_ext* t = new pttk_tt_ext();
  fill_meta(t, kernel, d, src_box, tgt_box, d_theta, theta_box, n);
  for (int k = 0; k <= D; ++k) t->ranks[k] = ranks[k];
  return upload_cores(t, cores, out);
}

pttk_status pttk_tt_round(const pttk_tt* in, double tol, void* stream, pttk_tt** out) {
  clear_error();
  if (!in || !out) return set_error(PTTK_EINVAL, "NULL argument");
  *out = nullptr;
  if (!(tol > 0.0) || !(tol < 1.0)) return set_error(PTTK_EINVAL, "tol must be in (0, 1)");
  cudaStream_t s = as_stream(stream);
  pttk_tt_ext* t = new pttk_tt_ext();
  t->kernel = in->kernel;
  t->d = in->d;
  t->dtheta = in->dtheta;
  t->D = in->D;
  t->n = in->n;
  for (int j = 0; j < in->D; ++j) {
    t->box[j][0] = in->box[j][0];
    t->box[j][1] = in->box[j][1];
  }
  cudaGetDevice(&t->device);
  pttk_status st = tt_round_run(in, tol, t, s);
  if (st == PTTK_OK) st = prepare_oriented(t, s);
  if (st == PTTK_OK) {
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_error(e, "TT-Round");
  }
  if (st != PTTK_OK) {
    free_handle(t);
    return st;
  }
  *out = t;
  return PTTK_OK;
}

void pttk_tt_free(pttk_tt* tt) { free_handle(static_cast<pttk_tt_ext*>(tt)); }

pttk_status pttk_theta_core(const pttk_tt* tt, const double* theta, pttk_prec prec, void* M,
                            void* stream) {
  clear_error();
  if (!tt || !M) return set_error(PTTK_EINVAL, "NULL argument");
  if (prec < PTTK_FP64 || prec > PTTK_FP16X3) return set_error(PTTK_EINVAL, "unknown precision");
  double th[PTTK_MAX_D];
  PTTK_TRY(theta_hat(tt, theta, th));
  return theta_core_run(tt, th, prec == PTTK_FP64, M, as_stream(stream));
}

pttk_status pttk_instantiate(const pttk_tt* tt, const double* theta, const void* X, int64_t N_s,
                             const void* Y, int64_t N_t, pttk_prec prec, void* U, void* M,
                             void* V, void* stream) {
  clear_error();
  if (!tt || !M) return set_error(PTTK_EINVAL, "NULL argument");
  if (N_s < 0 || N_t < 0) return set_error(PTTK_EINVAL, "negative point count");
  if ((N_s > 0 && (!X || !U)) || (N_t > 0 && (!Y || !V))) return set_error(PTTK_EINVAL, "NULL point or factor buffer");
  if (prec < PTTK_FP64 || prec > PTTK_FP16X3) return set_error(PTTK_EINVAL, "unknown precision");
  double th[PTTK_MAX_D];
  PTTK_TRY(theta_hat(tt, theta, th));
  cudaStream_t s = as_stream(stream);
  PTTK_TRY(theta_core_run(tt, th, prec == PTTK_FP64, M, s));
  PTTK_TRY(point_domain_check(tt, X, N_s, Y, N_t, prec == PTTK_FP64, tt_status_word(tt), s));
  if (prec == PTTK_FP64 || prec == PTTK_FP32) {
    PTTK_TRY(factor_build_run(tt, true, X, N_s, prec, U, s));
    PTTK_TRY(factor_build_run(tt, false, Y, N_t, prec, V, s));
    return PTTK_OK;
  }
  const pttk_tt_ext* t = static_cast<const pttk_tt_ext*>(tt);
  return factor_build_tc(tt, t->tc, static_cast<const float*>(X), N_s, static_cast<const float*>(Y), N_t, prec,
                         static_cast<float*>(U), static_cast<float*>(V), t->dstatus, 0, s);
}

uint64_t pttk_splitmix64(uint64_t key, uint64_t counter) { return splitmix64(key, counter); }

pttk_status pttk_tt_check(const pttk_tt* tt, void* stream) {
  clear_error();
  if (!tt) return set_error(PTTK_EINVAL, "NULL handle");
  const pttk_tt_ext* t = static_cast<const pttk_tt_ext*>(tt);
  cudaStream_t s = as_stream(stream);
  PTTK_CUDA(cudaStreamSynchronize(s));
  int h = 0;
  PTTK_CUDA(cudaMemcpy(&h, t->dstatus, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    PTTK_CUDA(cudaMemset(t->dstatus, 0, sizeof(int)));
    if (h == (int)PTTK_EDOMAIN)
      return set_error(PTTK_EDOMAIN, "a kernel using this handle met a point or a theta outside its box");
    return set_error((pttk_status)h, "a bounded device-side wait ran out in a kernel using this handle");
  }
  return PTTK_OK;
}

pttk_status pttk_apply(const void* U, const void* M, const void* V, int64_t N_s, int64_t N_t,
                       int rs, int rt, pttk_prec prec, const void* w, void* out, void* stream) {
  clear_error();
  if (!M || (N_s > 0 && (!U || !out)) || (N_t > 0 && (!V || !w))) return set_error(PTTK_EINVAL, "NULL argument");
  if (N_s < 0 || N_t < 0 || rs < 1 || rt < 1) return set_error(PTTK_EINVAL, "bad size");
  if (prec != PTTK_FP64 && prec != PTTK_FP32) return set_error(PTTK_EINVAL, "apply precision must be FP64 or FP32");
  cudaStream_t s = as_stream(stream);
  const bool fp64 = prec == PTTK_FP64;
  void* scratch = nullptr;
  PTTK_CUDA(cudaMallocAsync(&scratch, apply_scratch_bytes(N_t, rs, rt, fp64), s));
  const pttk_status st = apply_run(U, M, V, N_s, N_t, rs, rt, fp64, w, out, scratch, s);
  cudaFreeAsync(scratch, s);
  return st;
}

}  // extern "C"
