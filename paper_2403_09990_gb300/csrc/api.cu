// C ABI of libpurse (declared in include/purse.h): argument validation,
// handle lifetime, handle-owned scratch, the device status word.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "dev.cuh"
#include "internal.h"

namespace purse {

static thread_local std::string g_error = "";
static thread_local const char* g_injected = nullptr;  // site of the last injected allocation refusal

void set_error(const std::string& msg) { g_error = msg; }

bool fault_at(const char* site) {
  const char* f = std::getenv("PURSE_FAULT");
  if (!f || !*f) return false;
  const size_t n = std::strlen(site);
  for (const char* p = f; *p;) {
    const char* e = std::strchr(p, ',');
    const size_t len = e ? (size_t)(e - p) : std::strlen(p);
    if (len == n && std::strncmp(p, site, n) == 0) return true;
    if (!e) break;
    p = e + 1;
  }
  return false;
}

purse_status injected_fault(const char* site, const char* where) {
  set_error(std::string(where) + ": injected fault (PURSE_FAULT=" + site + ")");
  if (std::strcmp(site, "alloc") == 0) return PURSE_ERR_NOMEM;
  if (std::strcmp(site, "empty_seed") == 0) return PURSE_ERR_EMPTY;
  return PURSE_ERR_CUDA;
}

cudaError_t dev_alloc(void** ptr, size_t bytes) {
  if (fault_at("alloc")) {
    *ptr = nullptr;
    g_injected = "alloc";
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(ptr, bytes);
}

purse_status cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation && g_injected) {
    g_injected = nullptr;
    return injected_fault("alloc", where);
  }
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PURSE_ERR_NOMEM : PURSE_ERR_CUDA;
}

static purse_status arg_error(const std::string& msg) {
  set_error(msg);
  return PURSE_ERR_ARG;
}

purse_status ensure_scratch(purse_t h, size_t bytes) {
  if (bytes <= h->scratch_bytes) return PURSE_OK;
  if (h->d_scratch) {
    cudaError_t e = cudaFree(h->d_scratch);  // synchronises the device
    h->d_scratch = nullptr;
    h->scratch_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFree(scratch)");
  }
  const size_t sz = bytes < (1 << 16) ? (1 << 16) : bytes + bytes / 4;
  cudaError_t e = dev_alloc(&h->d_scratch, sz);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(scratch)");
  h->scratch_bytes = sz;
  return PURSE_OK;
}

static bool finite_all(const double* v, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(v[k])) return false;
  return true;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace purse

using namespace purse;

extern "C" {

const char* purse_last_error(void) { return g_error.c_str(); }

const char* purse_version(void) { return "libpurse 0.1 (CUDA sm_103a)"; }

purse_status purse_create(int kind, int n, const double* model, const double* obs, const double* radii,
                          const purse_intrinsics* K, purse_t* out) {
  if (!out) return arg_error("purse_create: out is NULL");
  *out = nullptr;
  if (kind != PURSE_3D3D && kind != PURSE_2D3D) return arg_error("purse_create: kind must be 0 (3D-3D) or 1 (2D-3D)");
  if (n < 3 || n > 256) return arg_error("purse_create: n must be in [3, 256]");
  if (!model || !obs || !radii) return arg_error("purse_create: NULL input array");
  const int od = kind == PURSE_3D3D ? 3 : 2;
  std::vector<double> obs_fault;
  if (fault_at("nan_input")) {  // the caller's array is left as it is
    obs_fault.assign(obs, obs + (size_t)od * n);
    obs_fault[0] = std::nan("");
    obs = obs_fault.data();
  }
  if (!finite_all(model, 3 * (size_t)n) || !finite_all(obs, (size_t)od * n) || !finite_all(radii, n))
    return arg_error("purse_create: non-finite input");
  for (int i = 0; i < n; ++i)
    if (!(radii[i] > 0)) return arg_error("purse_create: radii must be > 0");
  purse_intrinsics Kc{0, 0, 0, 0};
  if (kind == PURSE_2D3D) {
    if (!K) return arg_error("purse_create: 2D-3D needs intrinsics");
    Kc = *K;
    if (!(std::isfinite(Kc.fx) && std::isfinite(Kc.fy) && std::isfinite(Kc.cx) && std::isfinite(Kc.cy)) ||
        !(Kc.fx > 0 && Kc.fy > 0))
      return arg_error("purse_create: intrinsics must be finite with fx, fy > 0");
  }
  std::vector<double> t64(8 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    double* a = &t64[4 * i];
    double* b = &t64[4 * (n + i)];
    a[0] = model[3 * i], a[1] = model[3 * i + 1], a[2] = model[3 * i + 2], a[3] = radii[i];
    b[0] = obs[od * i], b[1] = obs[od * i + 1], b[2] = od == 3 ? obs[od * i + 2] : 0.0, b[3] = radii[i] * radii[i];
  }
  double rho_max = 0.0;
  for (int i = 0; i < n; ++i)
    rho_max = std::max(rho_max, std::sqrt(model[3 * i] * model[3 * i] + model[3 * i + 1] * model[3 * i + 1] +
                                          model[3 * i + 2] * model[3 * i + 2]));
  return make_handle(kind, n, t64, Kc, rho_max, out);
}

}  // extern "C"

namespace purse {

// A handle owning device copies (FP64 and FP32) of the constraint table t64.
purse_status make_handle(int kind, int n, const std::vector<double>& t64, const purse_intrinsics& Kc, double rho_max,
                         purse_t* out) {
  if (fault_at("alloc")) return injected_fault("alloc", "purse_create");
  std::vector<float> t32(t64.size());
  for (size_t k = 0; k < t64.size(); ++k) t32[k] = (float)t64[k];
  purse_s* h = new purse_s();
  h->kind = kind;
  h->n = n;
  h->rho_max = rho_max;
  h->K = Kc;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = dev_alloc((void**)&h->tables.f64, t64.size() * sizeof(double));
  if (e == cudaSuccess) e = dev_alloc((void**)&h->tables.f32, t32.size() * sizeof(float));
  if (e == cudaSuccess) e = dev_alloc((void**)&h->d_status, 256);
  if (e == cudaSuccess) e = cudaMemcpy(h->tables.f64, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->tables.f32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, 256);
  if (e != cudaSuccess) {
    purse_status s = cuda_fail(e, "purse_create");
    purse_destroy(h);
    return s;
  }
  h->d_evals = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(h->d_status) + 64);
  *out = h;
  return PURSE_OK;
}

}  // namespace purse

extern "C" {

purse_status purse_create_regression(int n, const double* hyp, const double* beta_rot, const double* beta_t,
                                     purse_t* out) {
  if (!out) return arg_error("purse_create_regression: out is NULL");
  *out = nullptr;
  if (n < 1 || n > 256) return arg_error("purse_create_regression: n must be in [1, 256]");
  if (!hyp || !beta_rot || !beta_t) return arg_error("purse_create_regression: NULL input array");
  std::vector<double> hyp_fault;
  if (fault_at("nan_input")) {
    hyp_fault.assign(hyp, hyp + 12 * (size_t)n);
    hyp_fault[9] = std::nan("");
    hyp = hyp_fault.data();
  }
  if (!finite_all(hyp, 12 * (size_t)n) || !finite_all(beta_rot, n) || !finite_all(beta_t, n))
    return arg_error("purse_create_regression: non-finite input");
  for (int i = 0; i < n; ++i) {
    if (!(beta_rot[i] > 0) || !(beta_t[i] > 0)) return arg_error("purse_create_regression: radii must be > 0");
    const double* R = hyp + 12 * (size_t)i;
    double err = 0.0;  // |R R^T - I| and det R - 1
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        const double d = R[3 * r] * R[3 * c] + R[3 * r + 1] * R[3 * c + 1] + R[3 * r + 2] * R[3 * c + 2];
        err = std::max(err, std::fabs(d - (r == c ? 1.0 : 0.0)));
      }
    const double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                       R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (err > 1e-6 || std::fabs(det - 1.0) > 1e-6)
      return arg_error("purse_create_regression: a hypothesis rotation is not a rotation matrix");
  }
  // rows [0, n): (t_i, beta_i^t); rows [n, 4n): the rows of R_i, beta_i^R in the first, 0 in the others
  std::vector<double> t64(16 * (size_t)n, 0.0);
  for (int i = 0; i < n; ++i) {
    const double* H = hyp + 12 * (size_t)i;
    double* a = &t64[4 * (size_t)i];
    a[0] = H[9], a[1] = H[10], a[2] = H[11], a[3] = beta_t[i];
    for (int r = 0; r < 3; ++r) {
      double* row = &t64[4 * ((size_t)(1 + r) * n + i)];
      row[0] = H[3 * r], row[1] = H[3 * r + 1], row[2] = H[3 * r + 2], row[3] = r == 0 ? beta_rot[i] : 0.0;
    }
  }
  return make_handle(PURSE_REG, n, t64, purse_intrinsics{0, 0, 0, 0}, 0.0, out);
}

}  // extern "C"

namespace purse {
// Noise factor of one constraint (eq. 4): the Cholesky factor Lambda = U^T U, U upper triangular, of
// the d x d matrix L (row-major), written as 8 values (3D: u00 u01 u02 u11 u12 u22; 2D: u00 u01 u11;
// the rest 0).  Returns NULL, or why L is not a symmetric positive definite matrix.
const char* noise_factor(const double* L, int d, double* o) {
  double scale = 0.0;  // symmetry is judged against the size of the matrix, not of the entry (an entry
                      // near 0 formed as a sum of products differs from its transpose by their rounding)
  for (int k = 0; k < d * d; ++k) scale = std::max(scale, std::fabs(L[k]));
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < r; ++c)
      if (std::fabs(L[r * d + c] - L[c * d + r]) > 1e-12 * scale + 1e-300) return "a noise matrix is not symmetric";
  double U[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int r = 0; r < d; ++r) {
    double s2 = L[r * d + r];
    for (int k = 0; k < r; ++k) s2 -= U[k][r] * U[k][r];
    if (!(s2 > 0)) return "a noise matrix is not positive definite";
    U[r][r] = std::sqrt(s2);
    for (int c = r + 1; c < d; ++c) {
      double v = L[r * d + c];
      for (int k = 0; k < r; ++k) v -= U[k][r] * U[k][c];
      U[r][c] = v / U[r][r];
    }
  }
  for (int k = 0; k < 8; ++k) o[k] = 0.0;
  if (d == 3) {
    o[0] = U[0][0], o[1] = U[0][1], o[2] = U[0][2], o[3] = U[1][1], o[4] = U[1][2], o[5] = U[2][2];
  } else {
    o[0] = U[0][0], o[1] = U[0][1], o[2] = U[1][1];
  }
  return nullptr;
}
}  // namespace purse

extern "C" {

purse_status purse_set_noise(purse_t h, const double* lam) {
  if (!h) return arg_error("purse_set_noise: NULL handle");
  if (h->kind == PURSE_REG) return arg_error("purse_set_noise: regression PURSEs take no noise matrices");
  if (!lam) {  // back to the identity
    if (h->ell64) cudaFree(h->ell64);
    if (h->ell32) cudaFree(h->ell32);
    h->ell64 = nullptr, h->ell32 = nullptr;
    return PURSE_OK;
  }
  const int d = h->kind == PURSE_3D3D ? 3 : 2, n = h->n;
  if (!finite_all(lam, (size_t)n * d * d)) return arg_error("purse_set_noise: non-finite input");
  std::vector<double> u64(8 * (size_t)n, 0.0);
  for (int i = 0; i < n; ++i) {
    const char* why = noise_factor(lam + (size_t)i * d * d, d, &u64[8 * (size_t)i]);
    if (why) return arg_error(std::string("purse_set_noise: ") + why);
  }
  std::vector<float> u32(u64.size());
  for (size_t k = 0; k < u64.size(); ++k) u32[k] = (float)u64[k];
  cudaError_t e = cudaSuccess;
  if (!h->ell64) e = dev_alloc((void**)&h->ell64, u64.size() * sizeof(double));
  if (e == cudaSuccess && !h->ell32) e = dev_alloc((void**)&h->ell32, u32.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(h->ell64, u64.data(), u64.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->ell32, u32.data(), u32.size() * sizeof(float), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_set_noise");
}

purse_status purse_destroy(purse_t h) {
  if (!h) return PURSE_OK;
  if (h->tables.f64) cudaFree(h->tables.f64);
  if (h->tables.f32) cudaFree(h->tables.f32);
  if (h->d_status) cudaFree(h->d_status);
  if (h->ell64) cudaFree(h->ell64);
  if (h->ell32) cudaFree(h->ell32);
  if (h->d_scratch) cudaFree(h->d_scratch);
  delete h;
  return PURSE_OK;
}

purse_status purse_eval(purse_t h, int precision, const void* d_poses, int n_poses, void* d_margin, int32_t* d_active,
                        void* d_grad, purse_stream_t stream) {
  if (!h) return arg_error("purse_eval: NULL handle");
  if (precision != 0 && precision != 1) return arg_error("purse_eval: precision must be 0 or 1");
  if (n_poses < 0) return arg_error("purse_eval: n_poses < 0");
  if (n_poses > 0 && !d_poses) return arg_error("purse_eval: NULL poses");
  if (h->kind == PURSE_REG || h->ell64)
    return arg_error("purse_eval: not available for regression PURSEs or noise matrices (use purse_dist)");
  if (fault_at("launch")) return injected_fault("launch", "purse_eval");
  cudaError_t e = launch_eval(h, precision, d_poses, n_poses, d_margin, d_active, d_grad, (cudaStream_t)stream);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_eval");
}

purse_status purse_dist(purse_t h, int mode, const float* d_poses, long long n_poses, float* d_dist,
                        purse_stream_t stream) {
  if (!h) return arg_error("purse_dist: NULL handle");
  if (mode < 0 || mode > 2) return arg_error("purse_dist: mode must be 0 (FP32), 1 (split TF32) or 2 (TF32)");
  if (n_poses < 0) return arg_error("purse_dist: n_poses < 0");
  if (n_poses > 0 && (!d_poses || !d_dist)) return arg_error("purse_dist: NULL buffer");
  if ((reinterpret_cast<uintptr_t>(d_poses) & 15) != 0) return arg_error("purse_dist: d_poses must be 16-byte aligned");
  if (mode != 0 && (h->kind == PURSE_REG || h->ell64))
    return arg_error("purse_dist: regression PURSEs and noise matrices take mode 0");
  if (fault_at("launch")) return injected_fault("launch", "purse_dist");
  cudaError_t e = mode == 0 ? launch_plain_dist(h, d_poses, (long)n_poses, d_dist, (cudaStream_t)stream)
                            : launch_tc_dist(h, mode == 1 ? 3 : 1, d_poses, (long)n_poses, d_dist, (cudaStream_t)stream);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_dist");
}

purse_status purse_ransag(purse_t h, uint64_t seed, int n_trials, int max_seeds, double* d_seeds, int* n_seeds,
                          purse_stream_t stream) {
  if (!h) return arg_error("purse_ransag: NULL handle");
  if (n_trials < 1 || max_seeds < 1) return arg_error("purse_ransag: n_trials and max_seeds must be >= 1");
  if (!d_seeds || !n_seeds) return arg_error("purse_ransag: NULL output");
  if (fault_at("empty_seed")) {
    *n_seeds = 0;
    return injected_fault("empty_seed", "purse_ransag");
  }
  if (fault_at("launch")) return injected_fault("launch", "purse_ransag");
  cudaStream_t st = (cudaStream_t)stream;
  const int chunk = 1 << 16;
  const int slots = h->kind == PURSE_2D3D ? 4 : 1;  // candidate poses per trial (P3P: up to four)
  const size_t pose_bytes = align256((size_t)chunk * slots * 12 * sizeof(double));
  const size_t acc_bytes = align256((size_t)chunk * slots);
  purse_status s = ensure_scratch(h, pose_bytes + acc_bytes + 256);
  if (s != PURSE_OK) return s;
  double* d_pose = reinterpret_cast<double*>(h->d_scratch);
  uint8_t* d_acc = reinterpret_cast<uint8_t*>(h->d_scratch) + pose_bytes;
  int* d_count = reinterpret_cast<int*>(reinterpret_cast<char*>(h->d_scratch) + pose_bytes + acc_bytes);
  cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(int), st);
  int count = 0;
  for (int t0 = 0; t0 < n_trials && e == cudaSuccess; t0 += chunk) {
    const int nt = n_trials - t0 < chunk ? n_trials - t0 : chunk;
    e = h->kind == PURSE_3D3D   ? launch_ransag(h, seed, t0, nt, d_pose, d_acc, st)
        : h->kind == PURSE_2D3D ? launch_ransag_p3p(h, seed, t0, nt, d_pose, d_acc, st)
                                : launch_convex_seeds(h, seed, t0, nt, d_pose, d_acc, st);
    if (e == cudaSuccess) e = launch_compact(d_pose, d_acc, nt * slots, d_seeds, d_count, max_seeds, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&count, d_count, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (count >= max_seeds) break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "purse_ransag");
  *n_seeds = count;
  if (count == 0) {
    set_error("purse_ransag: no trial pose inside the PURSE");
    return PURSE_ERR_EMPTY;
  }
  return PURSE_OK;
}

purse_status purse_sample(purse_t h, const purse_params* p, uint64_t seed, const double* d_seeds, int s0,
                          int n_samples, void* d_q, void* d_t, int16_t* d_trace, void* d_snap,
                          purse_stream_t stream) {
  if (!h || !p) return arg_error("purse_sample: NULL handle or params");
  if (h->kind == PURSE_REG && d_snap) return arg_error("purse_sample: no boundary snap for regression PURSEs");
  if (p->n_iter < 0) return arg_error("purse_sample: n_iter < 0");
  if (p->n_perturb < 1 || p->n_perturb > 256) return arg_error("purse_sample: n_perturb must be in [1, 256]");
  if (p->n_keep < 1 || p->n_keep > 32 || p->n_keep > p->n_perturb)
    return arg_error("purse_sample: n_keep must be in [1, min(32, n_perturb)]");
  if (p->n_steps < 1 || p->n_steps > 32) return arg_error("purse_sample: n_steps must be in [1, 32]");
  if (!(p->gamma > 0 && p->gamma <= 1)) return arg_error("purse_sample: gamma must be in (0, 1]");
  if (!std::isfinite(p->omega0) || !std::isfinite(p->v0) || !std::isfinite(p->rot_perturb) ||
      !std::isfinite(p->trans_perturb) || p->rot_perturb < 0 || p->trans_perturb < 0)
    return arg_error("purse_sample: speeds and perturbation scales must be finite (scales >= 0)");
  if (p->sampler != 0 && p->sampler != 1) return arg_error("purse_sample: sampler must be 0 or 1");
  if (p->precision != 0 && p->precision != 1) return arg_error("purse_sample: precision must be 0 or 1");
  if (p->perturb_units != 0 && p->perturb_units != 1) return arg_error("purse_sample: perturb_units must be 0 or 1");
  if (s0 < 1 || !d_seeds) return arg_error("purse_sample: need at least one seed pose");
  if (n_samples < 0) return arg_error("purse_sample: n_samples < 0");
  if (n_samples > 0 && (!d_q || !d_t)) return arg_error("purse_sample: NULL output");
  if ((long long)p->n_iter * (p->n_keep + 2) * (long long)n_samples > (1LL << 40))
    return arg_error("purse_sample: trace too large");
  if (fault_at("empty_seed")) return injected_fault("empty_seed", "purse_sample");
  if (fault_at("launch")) return injected_fault("launch", "purse_sample");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t stats_bytes = align256(sizeof(WalkStats));
  const size_t seed_bytes = align256((size_t)s0 * kSeedStride * sizeof(double));
  purse_status s = ensure_scratch(h, stats_bytes + seed_bytes);
  if (s != PURSE_OK) return s;
  WalkStats* d_stats = reinterpret_cast<WalkStats*>(h->d_scratch);
  double* d_seed_data = reinterpret_cast<double*>(reinterpret_cast<char*>(h->d_scratch) + stats_bytes);
  cudaError_t e = cudaMemsetAsync(h->d_evals, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = launch_stats(h, d_seeds, s0, p, d_stats, d_seed_data, st);
  if (e != cudaSuccess) return cuda_fail(e, "purse_sample (stats)");
  if (n_samples == 0) return PURSE_OK;
  WalkArgs a;
  a.table = p->precision == 0 ? (const void*)h->tables.f32 : (const void*)h->tables.f64;
  a.table64 = h->tables.f64;
  a.ell = !h->ell64 ? nullptr : p->precision == 0 ? (const void*)h->ell32 : (const void*)h->ell64;
  a.ell64 = h->ell64;
  a.n = h->n;
  a.fx = h->K.fx, a.fy = h->K.fy, a.cx = h->K.cx, a.cy = h->K.cy;
  a.rho_max = h->rho_max;
  a.seed_data = d_seed_data;
  a.s0 = s0;
  a.stats = d_stats;
  a.n_samples = n_samples;
  a.n_iter = p->n_iter, a.n_perturb = p->n_perturb, a.n_keep = p->n_keep, a.n_steps = p->n_steps;
  a.omega0 = p->omega0, a.v0 = p->v0, a.gamma = p->gamma;
  a.key0 = (uint32_t)seed, a.key1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    a.rk[2 * r] = a.key0 + (uint32_t)r * 0x9E3779B9u;
    a.rk[2 * r + 1] = a.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  a.out_q = d_q, a.out_t = d_t;
  a.trace = d_trace;
  a.out_snap = d_snap;
  a.status = h->d_status;
  a.evals = h->d_evals;
  a.stall_probe = fault_at("stall") ? 1 : 0;
  e = launch_walk(h, p, a, st);
  if (e == cudaErrorInvalidConfiguration || e == cudaErrorInvalidValue) {
    set_error("purse_sample: walk configuration does not fit in shared memory");
    return PURSE_ERR_ARG;
  }
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_sample (walk)");
}

purse_status purse_sample_plain(purse_t h, const purse_params* p, uint64_t seed, const double* d_seeds, int s0,
                                int n_samples, void* d_q, void* d_t, int16_t* d_trace, purse_stream_t stream) {
  if (!h || !p) return arg_error("purse_sample_plain: NULL handle or params");
  if (p->n_iter < 0) return arg_error("purse_sample_plain: n_iter < 0");
  if (p->n_perturb < 1 || p->n_perturb > 256) return arg_error("purse_sample_plain: n_perturb must be in [1, 256]");
  if (p->n_keep < 1 || p->n_keep > 32 || p->n_keep > p->n_perturb)
    return arg_error("purse_sample_plain: n_keep must be in [1, min(32, n_perturb)]");
  if (p->n_steps < 1 || p->n_steps > 32) return arg_error("purse_sample_plain: n_steps must be in [1, 32]");
  if (!(p->gamma > 0 && p->gamma <= 1)) return arg_error("purse_sample_plain: gamma must be in (0, 1]");
  if (!std::isfinite(p->omega0) || !std::isfinite(p->v0) || !std::isfinite(p->rot_perturb) ||
      !std::isfinite(p->trans_perturb) || p->rot_perturb < 0 || p->trans_perturb < 0)
    return arg_error("purse_sample_plain: speeds and perturbation scales must be finite (scales >= 0)");
  if (p->sampler != 0 && p->sampler != 1) return arg_error("purse_sample_plain: sampler must be 0 or 1");
  if (p->precision != 0 && p->precision != 1) return arg_error("purse_sample_plain: precision must be 0 or 1");
  if (p->perturb_units != 0 && p->perturb_units != 1)
    return arg_error("purse_sample_plain: perturb_units must be 0 or 1");
  if (s0 < 1 || !d_seeds) return arg_error("purse_sample_plain: need at least one seed pose");
  if (n_samples < 0) return arg_error("purse_sample_plain: n_samples < 0");
  if (n_samples > 0 && (!d_q || !d_t)) return arg_error("purse_sample_plain: NULL output");
  if (fault_at("empty_seed")) return injected_fault("empty_seed", "purse_sample_plain");
  if (fault_at("launch")) return injected_fault("launch", "purse_sample_plain");
  cudaStream_t st = (cudaStream_t)stream;
  int chunk = 1;
  const size_t stats_bytes = align256(sizeof(WalkStats));
  const size_t seed_bytes = align256((size_t)s0 * kSeedStride * sizeof(double));
  const size_t work_bytes = plain_scratch_bytes(p, n_samples, &chunk);
  purse_status s = ensure_scratch(h, stats_bytes + seed_bytes + work_bytes);
  if (s != PURSE_OK) return s;
  WalkStats* d_stats = reinterpret_cast<WalkStats*>(h->d_scratch);
  double* d_seed_data = reinterpret_cast<double*>(reinterpret_cast<char*>(h->d_scratch) + stats_bytes);
  void* work = reinterpret_cast<char*>(h->d_scratch) + stats_bytes + seed_bytes;
  cudaError_t e = cudaMemsetAsync(h->d_evals, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = launch_stats(h, d_seeds, s0, p, d_stats, d_seed_data, st);
  if (e != cudaSuccess) return cuda_fail(e, "purse_sample_plain (stats)");
  if (n_samples == 0) return PURSE_OK;
  e = launch_plain(h, p, d_stats, d_seed_data, s0, seed, n_samples, d_q, d_t, d_trace, work, work_bytes, chunk, st);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_sample_plain");
}

purse_status purse_last_evals(purse_t h, unsigned long long* evals, purse_stream_t stream) {
  if (!h || !evals) return arg_error("purse_last_evals: NULL argument");
  cudaError_t e = cudaMemcpyAsync(evals, h->d_evals, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                  (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_last_evals");
}

static purse_status megb_solve_impl(const char* fn, purse_t h, int precision, int n_iters, int n_last, const void* d_q,
                                    int n_rot, const void* d_t, int n_tr, double* d_result, int32_t* d_farthest,
                                    purse_stream_t stream) {
  const std::string f(fn);
  if (!h) return arg_error(f + ": NULL handle");
  if (precision != 0 && precision != 1) return arg_error(f + ": precision must be 0 or 1");
  if (n_iters < 1 || n_iters > (1 << 20)) return arg_error(f + ": n_iters must be in [1, 2^20]");
  if (n_last < 1) return arg_error(f + ": n_last must be >= 1");
  if (n_rot < 0 || n_tr < 0) return arg_error(f + ": negative sample count");
  if (n_rot > kMaxBallSamples || n_tr > kMaxBallSamples)
    return arg_error(f + ": more than 2^31 - 2^21 samples (32-bit sample indices)");
  if ((n_rot > 0 && !d_q) || (n_tr > 0 && !d_t) || !d_result) return arg_error(f + ": NULL buffer");
  if (fault_at("launch")) return injected_fault("launch", fn);
  const size_t need = megb_scratch_bytes(n_iters, h->sm_count);
  // the walk scratch (stats, seeds) is not needed any more once sampling is enqueued,
  // but megb keeps its own region after it so both can coexist on one stream
  purse_status s = ensure_scratch(h, need);
  if (s != PURSE_OK) return s;
  cudaError_t e = launch_megb(h, precision, n_iters, d_q, n_rot, d_t, n_tr, d_result, d_farthest, h->d_scratch,
                              (cudaStream_t)stream, n_last);
  if (e != cudaSuccess) return cuda_fail(e, fn);
  h->megb_iters = n_iters;
  h->megb_precision = precision;
  h->megb_q = d_q, h->megb_t = d_t;
  h->megb_nrot = n_rot, h->megb_ntr = n_tr;
  h->megb_navg = n_last;
  return PURSE_OK;
}

purse_status megb_solve(purse_t h, int precision, int n_iters, const void* d_q, int n_rot, const void* d_t, int n_tr,
                        double* d_result, int32_t* d_farthest, purse_stream_t stream) {
  return megb_solve_impl("megb_solve", h, precision, n_iters, 1, d_q, n_rot, d_t, n_tr, d_result, d_farthest, stream);
}

purse_status megb_solve_mean(purse_t h, int precision, int n_iters, int n_last, const void* d_q, int n_rot,
                             const void* d_t, int n_tr, double* d_result, int32_t* d_farthest, purse_stream_t stream) {
  return megb_solve_impl("megb_solve_mean", h, precision, n_iters, n_last, d_q, n_rot, d_t, n_tr, d_result, d_farthest,
                         stream);
}

purse_status megb_solve_exact(purse_t h, int precision, const void* d_q, int n_rot, const void* d_t, int n_tr,
                              const double* d_ref, double* d_result, purse_stream_t stream) {
  if (!h) return arg_error("megb_solve_exact: NULL handle");
  if (precision != 0 && precision != 1) return arg_error("megb_solve_exact: precision must be 0 or 1");
  if (n_rot < 0 || n_tr < 0) return arg_error("megb_solve_exact: negative sample count");
  if (n_rot > kMaxBallSamples || n_tr > kMaxBallSamples)
    return arg_error("megb_solve_exact: more than 2^31 - 2^21 samples (32-bit sample indices)");
  if ((n_rot > 0 && !d_q) || (n_tr > 0 && !d_t) || !d_result) return arg_error("megb_solve_exact: NULL buffer");
  if (fault_at("launch")) return injected_fault("launch", "megb_solve_exact");
  purse_status s = ensure_scratch(h, exact_scratch_bytes(h->sm_count));
  if (s != PURSE_OK) return s;
  cudaError_t e = launch_megb_exact(h, precision, d_q, n_rot, d_t, n_tr, d_ref, d_result, h->d_scratch,
                                    (cudaStream_t)stream);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "megb_solve_exact");
}

purse_status megb_backward(purse_t h, int precision, int n_iters, const void* d_q, const void* d_snap_rot, int n_rot,
                           const void* d_t, const void* d_snap_tr, int n_tr, const int32_t* d_farthest,
                           const double* d_result, const double* d_grad_result, double* d_grad_obs,
                           double* d_grad_radii, purse_stream_t stream) {
  if (!h) return arg_error("megb_backward: NULL handle");
  if (h->megb_navg != 1)
    return arg_error("megb_backward: the last ball solve on this handle was megb_solve_mean (not differentiated)");
  if (precision != 0 && precision != 1) return arg_error("megb_backward: precision must be 0 or 1");
  if (n_iters < 1 || n_iters > (1 << 20)) return arg_error("megb_backward: n_iters must be in [1, 2^20]");
  if (n_rot < 0 || n_tr < 0) return arg_error("megb_backward: negative sample count");
  if (n_rot > kMaxBallSamples || n_tr > kMaxBallSamples)
    return arg_error("megb_backward: more than 2^31 - 2^21 samples (32-bit sample indices)");
  if ((n_rot > 0 && (!d_q || !d_snap_rot)) || (n_tr > 0 && (!d_t || !d_snap_tr)))
    return arg_error("megb_backward: NULL samples or snap records");
  if (!d_farthest || !d_result || !d_grad_result || !d_grad_obs || !d_grad_radii)
    return arg_error("megb_backward: NULL buffer");
  if (fault_at("launch")) return injected_fault("launch", "megb_backward");
  purse_status s = ensure_scratch(h, megb_backward_scratch_bytes(n_iters, h->sm_count, h->n));
  if (s != PURSE_OK) return s;
  cudaError_t e = launch_megb_backward(h, precision, n_iters, d_q, d_snap_rot, n_rot, d_t, d_snap_tr, n_tr, d_farthest,
                                       d_result, d_grad_result, d_grad_obs, d_grad_radii, h->d_scratch,
                                       (cudaStream_t)stream);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "megb_backward");
}

purse_status purse_rng_words(uint64_t seed, uint32_t phase, uint32_t j, uint32_t i, uint32_t w0, int n_streams,
                             int n_words, uint32_t* d_words, int32_t* d_lattice, int unit, purse_stream_t stream) {
  if (n_streams < 0 || n_words < 0 || (n_streams > 0 && n_words > 0 && !d_words))
    return arg_error("purse_rng_words: bad sizes or NULL output");
  if (j >= (1u << 24) || phase > 255u) return arg_error("purse_rng_words: j must be < 2^24 and phase < 256");
  if (fault_at("launch")) return injected_fault("launch", "purse_rng_words");
  cudaError_t e = launch_rng_words(seed, phase, j, i, w0, n_streams, n_words, d_words, d_lattice, unit,
                                   (cudaStream_t)stream);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_rng_words");
}

purse_status purse_sync(purse_t h, purse_stream_t stream) {
  if (!h) return arg_error("purse_sync: NULL handle");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "purse_sync");
  int st = 0;
  e = cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "purse_sync (status)");
  if (st & kDevErrTimeout) {
    set_error("a bounded device wait ran out");
    return PURSE_ERR_TIMEOUT;
  }
  if (st & kDevErrNumeric) {
    set_error("non-finite value on the device");
    return PURSE_ERR_NUMERIC;
  }
  return PURSE_OK;
}

}  // extern "C"
