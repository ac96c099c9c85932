// Batched CLOSURE (Alg. 1 over many PURSEs): centre statistics, one persistent walk launch over
// all (PURSE, sampler, walk) items, and one block per ball -- three kernels captured once into a
// CUDA graph and replayed.  The walk launch shape (work-queue chunk, warps per block) is chosen
// by purse_batch_tune, which times the candidates on the caller's batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dev.cuh"
#include "internal.h"

struct purse_batch_s {
  int n_purses = 0, nmax = 0, total_rows = 0, sm_count = 0;
  purse::BatchPurseInfo* d_info = nullptr;
  float* d_tab32 = nullptr;
  double* d_tab64 = nullptr;
  // noise matrices of eq. 4 (purse_batch_set_noise): factors U_i, 8 values per keypoint, or NULL
  float* d_ell32 = nullptr;
  double* d_ell64 = nullptr;
  std::vector<int> kinds, offsets;  // host copies (kind per PURSE, CSR keypoint offsets)
  int reg = 0;  // pose-regression batch (purse_batch_create_regression)
  purse::WalkStats* d_stats = nullptr;
  double* d_seed_data = nullptr;
  unsigned int* d_counter = nullptr;
  unsigned long long* d_seed = nullptr;
  unsigned long long* d_evals = nullptr;
  int* d_status = nullptr;
  float* d_samples = nullptr;  // q_rot, t_rot, q_tr, t_tr
  size_t samples_cap = 0;      // samples per PURSE the buffer holds
  int last_samples = 0;        // samples per PURSE of the last solve (layout of the sample buffers)
  int last_iters = 0;          // GGD iterations of the last solve
  int32_t* d_far = nullptr;
  size_t far_cap = 0;
  // differentiation: snap records of both samplers, farthest samples of the final centres,
  // scratch for the recomputed rotation iterates
  int grad = 0;
  float* d_snap = nullptr;
  size_t snap_cap = 0;
  int32_t* d_fstar = nullptr;
  void* d_cs = nullptr;
  size_t cs_cap = 0;
  int last_grad = 0;  // the last solve wrote snap records
  int last_tr3d = 0;
  // launch shape of the walk kernel (autotuned)
  int chunk = 8, warps = 8;
  // captured graph and what it was captured for
  cudaGraphExec_t exec = nullptr;
  std::vector<char> graph_key;
  unsigned long long host_seed = 0;
};

namespace purse {

static purse_status barg(const std::string& m) {
  set_error(m);
  return PURSE_ERR_ARG;
}

static bool params_ok(const purse_params* p, std::string& why) {
  if (!p) return why = "NULL params", false;
  if (p->n_iter < 0 || p->n_perturb < 1 || p->n_perturb > 256 || p->n_keep < 1 || p->n_keep > 32 ||
      p->n_keep > p->n_perturb || p->n_steps < 1 || p->n_steps > 32 || !(p->gamma > 0 && p->gamma <= 1) ||
      !std::isfinite(p->omega0) || !std::isfinite(p->v0) || !(p->rot_perturb >= 0) || !(p->trans_perturb >= 0) ||
      (p->perturb_units != 0 && p->perturb_units != 1))
    return why = "parameters out of range (see purse_params)", false;
  if (p->precision != 0) return why = "batched walks run in FP32 (precision 0)", false;
  return true;
}

static BatchArgs make_args(purse_batch_t b, const purse_params* p3, const purse_params* p2, int n_samples) {
  BatchArgs a;
  a.info = b->d_info;
  a.table = b->d_tab32;
  a.table64 = b->d_tab64;
  a.ell = b->d_ell32;
  a.ell64 = b->d_ell64;
  a.stats = b->d_stats;
  a.seed_data = b->d_seed_data;
  a.n_purses = b->n_purses;
  a.n_samples = n_samples;
  a.nmax = b->nmax;
  const purse_params* pp[2] = {p3, p2};
  for (int k = 0; k < 2; ++k) {
    a.n_iter[k] = pp[k]->n_iter, a.n_perturb[k] = pp[k]->n_perturb, a.n_keep[k] = pp[k]->n_keep;
    a.n_steps[k] = pp[k]->n_steps, a.omega0[k] = pp[k]->omega0, a.v0[k] = pp[k]->v0, a.gamma[k] = pp[k]->gamma;
  }
  a.seed = b->d_seed;
  a.counter = b->d_counter;
  a.total_items = 2u * (unsigned)b->n_purses * (unsigned)n_samples;
  const size_t S = (size_t)b->n_purses * n_samples;
  a.q_rot = b->d_samples;
  a.t_rot = a.q_rot + 4 * S;
  a.q_tr = a.t_rot + 3 * S;
  a.t_tr = a.q_tr + 4 * S;
  a.snap_rot = b->grad ? b->d_snap : nullptr;
  a.snap_tr = b->grad ? b->d_snap + (size_t)kSnapStride * S : nullptr;
  a.fstar = b->grad ? b->d_fstar : nullptr;
  a.tr3d = p3->v0 > 0.0 ? 1 : 0;
  a.reg = b->reg;
  a.status = b->d_status;
  a.evals = b->d_evals;
  return a;
}

static purse_status ensure_batch_buffers(purse_batch_t b, int n_samples, int n_iters) {
  if ((size_t)n_samples > b->samples_cap) {
    if (b->d_samples) cudaFree(b->d_samples);
    b->d_samples = nullptr;
    b->samples_cap = 0;
    const size_t bytes = (size_t)b->n_purses * n_samples * 14 * sizeof(float);
    cudaError_t e = dev_alloc((void**)&b->d_samples, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "purse_batch_solve (sample buffers)");
    b->samples_cap = n_samples;
  }
  if ((size_t)n_iters > b->far_cap) {
    if (b->d_far) cudaFree(b->d_far);
    b->d_far = nullptr;
    b->far_cap = 0;
    cudaError_t e = dev_alloc((void**)&b->d_far, (size_t)b->n_purses * 2 * n_iters * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "purse_batch_solve (traces)");
    b->far_cap = n_iters;
  }
  if (b->grad && (size_t)n_samples > b->snap_cap) {
    if (b->d_snap) cudaFree(b->d_snap);
    b->d_snap = nullptr;
    b->snap_cap = 0;
    cudaError_t e = dev_alloc((void**)&b->d_snap, 2 * (size_t)b->n_purses * n_samples * kSnapStride * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "purse_batch_solve (snap records)");
    b->snap_cap = n_samples;
  }
  if (b->grad && !b->d_fstar) {
    cudaError_t e = dev_alloc((void**)&b->d_fstar, 2 * (size_t)b->n_purses * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "purse_batch_solve (farthest samples)");
  }
  return PURSE_OK;
}

static cudaError_t enqueue_batch(purse_batch_t b, const purse_params* p3, const purse_params* p2,
                                 const double* d_seeds, int n_samples, int n_iters, double* d_results, int chunk,
                                 int warps, bool walks_only, cudaStream_t st) {
  BatchStatParams sp;
  const purse_params* pp[2] = {p3, p2};
  for (int k = 0; k < 2; ++k) sp.t_p[k] = pp[k]->trans_perturb, sp.th_p[k] = pp[k]->rot_perturb, sp.raw[k] = pp[k]->perturb_units;
  const BatchArgs a = make_args(b, p3, p2, n_samples);
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_evals, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess)
    e = launch_stats_batch(b->n_purses, b->d_info, b->d_tab64, b->d_ell64, d_seeds, sp, b->d_stats, b->d_seed_data,
                           st);
  if (e == cudaSuccess) e = launch_batch_walk(a, chunk, warps, b->sm_count, st);
  if (e == cudaSuccess && !walks_only) e = launch_megb_batch(a, n_iters, d_results, b->d_far, st);
  return e;
}

}  // namespace purse

namespace purse {
// Device copies of a batch's per-PURSE records and concatenated tables (FP64 and FP32), statistics
// and seed-data slots and the status/counter words; the batch handle owns them.
static purse_status upload_batch(const char* fn, int n_purses, int nmax, int reg, const int* kinds, const int* offsets,
                                 const std::vector<BatchPurseInfo>& info, const std::vector<double>& t64,
                                 purse_batch_t* out) {
  std::vector<float> t32(t64.begin(), t64.end());
  if (fault_at("alloc")) return injected_fault("alloc", fn);
  purse_batch_s* b = new purse_batch_s();
  b->n_purses = n_purses, b->nmax = nmax, b->total_rows = (int)(t64.size() / 4), b->reg = reg;
  b->kinds.assign(kinds, kinds + n_purses);
  b->offsets.assign(offsets, offsets + n_purses + 1);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = dev_alloc((void**)&b->d_info, info.size() * sizeof(BatchPurseInfo));
  if (e == cudaSuccess) e = dev_alloc((void**)&b->d_tab64, t64.size() * sizeof(double));
  if (e == cudaSuccess) e = dev_alloc((void**)&b->d_tab32, t32.size() * sizeof(float));
  if (e == cudaSuccess) e = dev_alloc((void**)&b->d_stats, n_purses * sizeof(WalkStats));
  if (e == cudaSuccess) e = dev_alloc((void**)&b->d_seed_data, (size_t)n_purses * kSeedStride * sizeof(double));
  if (e == cudaSuccess) e = dev_alloc((void**)&b->d_counter, 256);
  if (e == cudaSuccess) {
    b->d_seed = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(b->d_counter) + 64);
    b->d_evals = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(b->d_counter) + 128);
    b->d_status = reinterpret_cast<int*>(reinterpret_cast<char*>(b->d_counter) + 192);
    e = cudaMemset(b->d_counter, 0, 256);
  }
  if (e == cudaSuccess) e = cudaMemcpy(b->d_info, info.data(), info.size() * sizeof(BatchPurseInfo), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tab64, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tab32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    purse_status s = cuda_fail(e, fn);
    purse_batch_destroy(b);
    return s;
  }
  *out = b;
  return PURSE_OK;
}
}  // namespace purse

using namespace purse;

extern "C" {

purse_status purse_batch_create(int n_purses, const int* kinds, const int* offsets, const double* model,
                                const double* obs, const double* radii, const purse_intrinsics* K,
                                purse_batch_t* out) {
  if (!out) return barg("purse_batch_create: out is NULL");
  *out = nullptr;
  if (n_purses < 1) return barg("purse_batch_create: n_purses must be >= 1");
  if (!kinds || !offsets || !model || !obs || !radii) return barg("purse_batch_create: NULL input");
  std::vector<double> obs_fault;
  if (fault_at("nan_input") && offsets[n_purses] > 0) {  // the caller's array is left as it is
    obs_fault.assign(obs, obs + 3 * (size_t)offsets[n_purses]);
    obs_fault[0] = std::nan("");
    obs = obs_fault.data();
  }
  if (offsets[0] != 0) return barg("purse_batch_create: offsets[0] must be 0");
  int nmax = 0;
  for (int p = 0; p < n_purses; ++p) {
    const int n = offsets[p + 1] - offsets[p];
    if (kinds[p] != 0 && kinds[p] != 1) return barg("purse_batch_create: kinds must be 0 or 1");
    if (n < 3 || n > 256) return barg("purse_batch_create: every PURSE needs 3..256 constraints");
    if (kinds[p] == 1 && (!K || !(K[p].fx > 0) || !(K[p].fy > 0) || !std::isfinite(K[p].cx) || !std::isfinite(K[p].cy)))
      return barg("purse_batch_create: 2D-3D PURSEs need finite intrinsics with fx, fy > 0");
    nmax = n > nmax ? n : nmax;
  }
  const int total = offsets[n_purses];
  for (int i = 0; i < total; ++i) {
    if (!(radii[i] > 0) || !std::isfinite(radii[i])) return barg("purse_batch_create: radii must be finite and > 0");
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(model[3 * i + c]) || !std::isfinite(obs[3 * i + c]))
        return barg("purse_batch_create: non-finite keypoint");
  }
  // tables: PURSE p occupies rows [2 offsets[p], 2 offsets[p+1]): model rows then observation rows
  std::vector<double> t64(8 * (size_t)total);
  std::vector<BatchPurseInfo> info(n_purses);
  for (int p = 0; p < n_purses; ++p) {
    const int n = offsets[p + 1] - offsets[p], o = offsets[p];
    info[p].kind = kinds[p], info[p].n = n, info[p].table_off = 2 * o, info[p].pad = 0;
    info[p].fx = kinds[p] ? K[p].fx : 0.0, info[p].fy = kinds[p] ? K[p].fy : 0.0;
    info[p].cx = kinds[p] ? K[p].cx : 0.0, info[p].cy = kinds[p] ? K[p].cy : 0.0;
    info[p].rho_max = 0.0;
    for (int i = 0; i < n; ++i) {
      const double* m = model + 3 * (size_t)(o + i);
      info[p].rho_max = std::max(info[p].rho_max, std::sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]));
    }
    for (int i = 0; i < n; ++i) {
      double* a = &t64[4 * (2 * (size_t)o + i)];
      double* bb = &t64[4 * (2 * (size_t)o + n + i)];
      const int g = o + i;
      a[0] = model[3 * g], a[1] = model[3 * g + 1], a[2] = model[3 * g + 2], a[3] = radii[g];
      bb[0] = obs[3 * g], bb[1] = obs[3 * g + 1], bb[2] = kinds[p] ? 0.0 : obs[3 * g + 2];
      bb[3] = radii[g] * radii[g];
    }
  }
  return upload_batch("purse_batch_create", n_purses, nmax, 0, kinds, offsets, info, t64, out);
}

purse_status purse_batch_create_regression(int n_purses, const int* offsets, const double* hyp, const double* beta_rot,
                                           const double* beta_t, purse_batch_t* out) {
  if (!out) return barg("purse_batch_create_regression: out is NULL");
  *out = nullptr;
  if (n_purses < 1) return barg("purse_batch_create_regression: n_purses must be >= 1");
  if (!offsets || !hyp || !beta_rot || !beta_t) return barg("purse_batch_create_regression: NULL input");
  if (offsets[0] != 0) return barg("purse_batch_create_regression: offsets[0] must be 0");
  int nmax = 0;
  for (int p = 0; p < n_purses; ++p) {
    const int n = offsets[p + 1] - offsets[p];
    if (n < 1 || n > 256) return barg("purse_batch_create_regression: every PURSE needs 1..256 hypotheses");
    nmax = n > nmax ? n : nmax;
  }
  const int total = offsets[n_purses];
  for (int i = 0; i < total; ++i) {
    if (!(beta_rot[i] > 0) || !(beta_t[i] > 0) || !std::isfinite(beta_rot[i]) || !std::isfinite(beta_t[i]))
      return barg("purse_batch_create_regression: radii must be finite and > 0");
    const double* R = hyp + 12 * (size_t)i;
    double err = 0.0;  // |R R^T - I| and det R - 1
    for (int k = 0; k < 12; ++k)
      if (!std::isfinite(R[k])) return barg("purse_batch_create_regression: non-finite hypothesis");
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        const double d = R[3 * r] * R[3 * c] + R[3 * r + 1] * R[3 * c + 1] + R[3 * r + 2] * R[3 * c + 2];
        err = std::max(err, std::fabs(d - (r == c ? 1.0 : 0.0)));
      }
    const double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                       R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (err > 1e-6 || std::fabs(det - 1.0) > 1e-6)
      return barg("purse_batch_create_regression: a hypothesis rotation is not a rotation matrix");
  }
  // PURSE p: rows [4 offsets[p], 4 offsets[p+1]) in the layout of purse_create_regression -- (t_i, beta_i^t),
  // then the rows of R_i with beta_i^R in the first
  std::vector<double> t64(16 * (size_t)total, 0.0);
  std::vector<BatchPurseInfo> info(n_purses);
  std::vector<int> kinds(n_purses, PURSE_REG);
  for (int p = 0; p < n_purses; ++p) {
    const int n = offsets[p + 1] - offsets[p], o = offsets[p];
    info[p].kind = PURSE_REG, info[p].n = n, info[p].table_off = 4 * o, info[p].pad = 0;
    info[p].fx = info[p].fy = info[p].cx = info[p].cy = 0.0;
    info[p].rho_max = 0.0;
    double* tp = &t64[16 * (size_t)o];
    for (int i = 0; i < n; ++i) {
      const double* H = hyp + 12 * (size_t)(o + i);
      double* a = tp + 4 * (size_t)i;
      a[0] = H[9], a[1] = H[10], a[2] = H[11], a[3] = beta_t[o + i];
      for (int r = 0; r < 3; ++r) {
        double* row = tp + 4 * ((size_t)(1 + r) * n + i);
        row[0] = H[3 * r], row[1] = H[3 * r + 1], row[2] = H[3 * r + 2], row[3] = r == 0 ? beta_rot[o + i] : 0.0;
      }
    }
  }
  return upload_batch("purse_batch_create_regression", n_purses, nmax, 1, kinds.data(), offsets, info, t64, out);
}

purse_status purse_batch_destroy(purse_batch_t b) {
  if (!b) return PURSE_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  cudaFree(b->d_info);
  cudaFree(b->d_tab32);
  cudaFree(b->d_tab64);
  cudaFree(b->d_ell32);
  cudaFree(b->d_ell64);
  cudaFree(b->d_stats);
  cudaFree(b->d_seed_data);
  cudaFree(b->d_counter);
  cudaFree(b->d_samples);
  cudaFree(b->d_far);
  cudaFree(b->d_snap);
  cudaFree(b->d_fstar);
  cudaFree(b->d_cs);
  delete b;
  return PURSE_OK;
}

purse_status purse_batch_set_noise(purse_batch_t b, const double* lam) {
  if (!b) return barg("purse_batch_set_noise: NULL batch");
  if (b->reg) return barg("purse_batch_set_noise: regression PURSEs take no noise matrices");
  if (b->exec) cudaGraphExecDestroy(b->exec);  // the next solve captures a graph with the new tables
  b->exec = nullptr;
  b->graph_key.clear();
  if (!lam) {  // back to the identity norm
    cudaFree(b->d_ell32);
    cudaFree(b->d_ell64);
    b->d_ell32 = nullptr, b->d_ell64 = nullptr;
    return PURSE_OK;
  }
  const int total = b->offsets[b->n_purses];
  for (size_t k = 0; k < 9 * (size_t)total; ++k)
    if (!std::isfinite(lam[k])) return barg("purse_batch_set_noise: non-finite input");
  std::vector<double> u64(8 * (size_t)total, 0.0);
  for (int p = 0; p < b->n_purses; ++p) {
    const int d = b->kinds[p] == 0 ? 3 : 2;
    for (int g = b->offsets[p]; g < b->offsets[p + 1]; ++g) {
      const double* L9 = lam + 9 * (size_t)g;
      const double L2[4] = {L9[0], L9[1], L9[3], L9[4]};  // 2D-3D: the top-left 2 x 2 block, row-major
      const char* why = noise_factor(d == 3 ? L9 : L2, d, &u64[8 * (size_t)g]);
      if (why) return barg(std::string("purse_batch_set_noise: ") + why);
    }
  }
  std::vector<float> u32(u64.begin(), u64.end());
  if (fault_at("alloc")) return injected_fault("alloc", "purse_batch_set_noise");
  cudaError_t e = cudaSuccess;
  if (!b->d_ell64) e = dev_alloc((void**)&b->d_ell64, u64.size() * sizeof(double));
  if (e == cudaSuccess && !b->d_ell32) e = dev_alloc((void**)&b->d_ell32, u32.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_ell64, u64.data(), u64.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_ell32, u32.data(), u32.size() * sizeof(float), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_batch_set_noise");
}

purse_status purse_batch_solve(purse_batch_t b, const purse_params* p3d, const purse_params* p2d, uint64_t seed,
                               const double* d_seeds, int n_samples, int n_iters, double* d_results,
                               purse_stream_t stream) {
  if (!b) return barg("purse_batch_solve: NULL batch");
  std::string why;
  if (!params_ok(p3d, why) || !params_ok(p2d, why)) return barg("purse_batch_solve: " + why);
  if (p3d->sampler != 0 || p2d->sampler != 0)
    return barg("purse_batch_solve: sampler is chosen per kind (set sampler = 0 in both parameter sets)");
  if (n_samples < 1 || n_samples > 12288) return barg("purse_batch_solve: n_samples must be in [1, 12288]");
  if (n_iters < 1 || n_iters > 100000) return barg("purse_batch_solve: n_iters must be in [1, 100000]");
  if ((unsigned long long)2 * b->n_purses * n_samples >= (1ull << 32))
    return barg("purse_batch_solve: too many work items (2 x n_purses x n_samples >= 2^32)");
  if (!d_seeds || !d_results) return barg("purse_batch_solve: NULL buffer");
  if (batch_walk_smem(b->nmax, p3d->n_perturb > p2d->n_perturb ? p3d->n_perturb : p2d->n_perturb,
                      p3d->n_steps > p2d->n_steps ? p3d->n_steps : p2d->n_steps, b->warps, b->d_ell32 != nullptr,
                      b->reg != 0) > 227 * 1024)
    return barg("purse_batch_solve: the largest PURSE does not fit the walk kernel's shared memory");
  if (fault_at("launch")) return injected_fault("launch", "purse_batch_solve");
  purse_status s = ensure_batch_buffers(b, n_samples, n_iters);
  if (s != PURSE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  b->host_seed = seed;
  b->last_samples = n_samples;
  b->last_iters = n_iters;
  b->last_grad = b->grad;
  b->last_tr3d = p3d->v0 > 0.0 ? 1 : 0;
  cudaError_t e = cudaMemcpyAsync(b->d_seed, &b->host_seed, sizeof(unsigned long long), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "purse_batch_solve (seed)");
  // the graph is captured once per (parameters, sizes, buffers, launch shape) and replayed
  std::vector<char> key(sizeof(purse_params) * 2 + 64);
  memcpy(key.data(), p3d, sizeof(purse_params));
  memcpy(key.data() + sizeof(purse_params), p2d, sizeof(purse_params));
  char* kp = key.data() + 2 * sizeof(purse_params);
  const void* ptrs[2] = {d_seeds, d_results};
  const int ints[5] = {n_samples, n_iters, b->chunk, b->warps, b->grad};
  memcpy(kp, ptrs, sizeof(ptrs));
  memcpy(kp + sizeof(ptrs), ints, sizeof(ints));
  if (!b->exec || key != b->graph_key) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "purse_batch_solve (capture stream)");
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue_batch(b, p3d, p2d, d_seeds, n_samples, n_iters, d_results, b->chunk, b->warps, false, cap);
      e = cudaStreamEndCapture(cap, &g);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return cuda_fail(e, "purse_batch_solve (graph capture)");
    }
    b->graph_key = key;
  }
  e = cudaGraphLaunch(b->exec, st);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_batch_solve (graph launch)");
}

purse_status purse_batch_tune(purse_batch_t b, const purse_params* p3d, const purse_params* p2d, uint64_t seed,
                              const double* d_seeds, int n_samples, int* best_chunk, int* best_warps,
                              float* best_ms, purse_stream_t stream) {
  if (!b) return barg("purse_batch_tune: NULL batch");
  std::string why;
  if (!params_ok(p3d, why) || !params_ok(p2d, why)) return barg("purse_batch_tune: " + why);
  if (n_samples < 1 || n_samples > 12288 || !d_seeds) return barg("purse_batch_tune: bad sample count or seeds");
  if (fault_at("launch")) return injected_fault("launch", "purse_batch_tune");
  purse_status s = ensure_batch_buffers(b, n_samples, 1);
  if (s != PURSE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  b->host_seed = seed;
  b->last_samples = n_samples;
  cudaError_t e = cudaMemcpyAsync(b->d_seed, &b->host_seed, sizeof(unsigned long long), cudaMemcpyHostToDevice, st);
  const int chunks[] = {1, 4, 16, 64};
  const int warps[] = {4, 8};
  const int np = p3d->n_perturb > p2d->n_perturb ? p3d->n_perturb : p2d->n_perturb;
  const int nt = p3d->n_steps > p2d->n_steps ? p3d->n_steps : p2d->n_steps;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bc = b->chunk, bw = b->warps;
  for (int wi = 0; wi < 2 && e == cudaSuccess; ++wi) {
    if (batch_walk_smem(b->nmax, np, nt, warps[wi], b->d_ell32 != nullptr, b->reg != 0) > 227 * 1024) continue;
    for (int ci = 0; ci < 4 && e == cudaSuccess; ++ci) {
      float ms = 0.f;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // first run warms up
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess)
          e = enqueue_batch(b, p3d, p2d, d_seeds, n_samples, 1, nullptr, chunks[ci], warps[wi], true, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      }
      if (e == cudaSuccess && ms < best) best = ms, bc = chunks[ci], bw = warps[wi];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "purse_batch_tune");
  if (bc != b->chunk || bw != b->warps) {
    b->chunk = bc, b->warps = bw;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (best_chunk) *best_chunk = bc;
  if (best_warps) *best_warps = bw;
  if (best_ms) *best_ms = best;
  return PURSE_OK;
}

purse_status purse_batch_copy_farthest(purse_batch_t b, int32_t* d_out, purse_stream_t stream) {
  if (!b || !d_out) return barg("purse_batch_copy_farthest: NULL argument");
  if (!b->d_far || b->last_iters == 0) return (set_error("purse_batch_copy_farthest: no solve yet"), PURSE_ERR_STATE);
  const int K = b->last_iters;
  cudaError_t e = cudaMemcpyAsync(d_out, b->d_far, (size_t)b->n_purses * 2 * K * sizeof(int32_t),
                                  cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_batch_copy_farthest");
}

purse_status purse_batch_copy_samples(purse_batch_t b, int p, float* d_q_rot, float* d_t_rot, float* d_q_tr,
                                      float* d_t_tr, purse_stream_t stream) {
  if (!b) return barg("purse_batch_copy_samples: NULL batch");
  if (p < 0 || p >= b->n_purses) return barg("purse_batch_copy_samples: PURSE index out of range");
  if (!b->d_samples || b->last_samples == 0) return (set_error("purse_batch_copy_samples: no solve yet"), PURSE_ERR_STATE);
  const size_t S = (size_t)b->n_purses * b->last_samples, n = (size_t)b->last_samples, o = (size_t)p * n;
  const float* src[4] = {b->d_samples + 4 * o, b->d_samples + 4 * S + 3 * o, b->d_samples + 7 * S + 4 * o,
                         b->d_samples + 11 * S + 3 * o};
  float* dst[4] = {d_q_rot, d_t_rot, d_q_tr, d_t_tr};
  const size_t width[4] = {4, 3, 4, 3};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    if (dst[k])
      e = cudaMemcpyAsync(dst[k], src[k], width[k] * n * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_batch_copy_samples");
}

purse_status purse_batch_set_grad(purse_batch_t b, int enable) {
  if (!b) return barg("purse_batch_set_grad: NULL batch");
  if (enable != 0 && enable != 1) return barg("purse_batch_set_grad: enable must be 0 or 1");
  if (enable && b->reg) return barg("purse_batch_set_grad: no boundary snap (and no adjoint) for regression PURSEs");
  if (b->grad != enable) {
    b->grad = enable;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return PURSE_OK;
}

purse_status purse_batch_copy_snap(purse_batch_t b, int p, float* d_snap_rot, float* d_snap_tr, purse_stream_t stream) {
  if (!b) return barg("purse_batch_copy_snap: NULL batch");
  if (p < 0 || p >= b->n_purses) return barg("purse_batch_copy_snap: PURSE index out of range");
  if (!b->last_grad) return (set_error("purse_batch_copy_snap: no solve with gradients enabled yet"), PURSE_ERR_STATE);
  const size_t S = (size_t)b->n_purses * b->last_samples, n = (size_t)b->last_samples, o = (size_t)p * n;
  const float* src[2] = {b->d_snap + kSnapStride * o, b->d_snap + kSnapStride * (S + o)};
  float* dst[2] = {d_snap_rot, d_snap_tr};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    if (dst[k])
      e = cudaMemcpyAsync(dst[k], src[k], kSnapStride * n * sizeof(float), cudaMemcpyDeviceToDevice,
                          (cudaStream_t)stream);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_batch_copy_snap");
}

purse_status purse_batch_backward(purse_batch_t b, const double* d_results, const double* d_grad_results,
                                  double* d_grad_obs, double* d_grad_radii, purse_stream_t stream) {
  if (!b) return barg("purse_batch_backward: NULL batch");
  if (!d_results || !d_grad_results || !d_grad_obs || !d_grad_radii) return barg("purse_batch_backward: NULL buffer");
  if (!b->last_grad || b->last_iters == 0)
    return (set_error("purse_batch_backward: no solve with gradients enabled yet"), PURSE_ERR_STATE);
  if (fault_at("launch")) return injected_fault("launch", "purse_batch_backward");
  const int K = b->last_iters;
  const size_t need = (size_t)b->n_purses * (K + 1) * 4 * sizeof(double);
  if (need > b->cs_cap) {
    if (b->d_cs) cudaFree(b->d_cs);
    b->d_cs = nullptr;
    b->cs_cap = 0;
    cudaError_t e = dev_alloc((void**)&b->d_cs, need);
    if (e != cudaSuccess) return cuda_fail(e, "purse_batch_backward (scratch)");
    b->cs_cap = need;
  }
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.info = b->d_info;
  a.n_purses = b->n_purses;
  a.n_samples = b->last_samples;
  a.nmax = b->nmax;
  const size_t S = (size_t)b->n_purses * b->last_samples;
  a.q_rot = b->d_samples;
  a.t_rot = a.q_rot + 4 * S;
  a.q_tr = a.t_rot + 3 * S;
  a.t_tr = a.q_tr + 4 * S;
  a.snap_rot = b->d_snap;
  a.snap_tr = b->d_snap + (size_t)kSnapStride * S;
  a.fstar = b->d_fstar;
  a.tr3d = b->last_tr3d;
  a.status = b->d_status;
  cudaError_t e = launch_batch_backward(a, K, b->d_far, d_results, d_grad_results, b->d_cs, d_grad_obs, d_grad_radii,
                                        (cudaStream_t)stream);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "purse_batch_backward");
}

purse_status purse_batch_sync(purse_batch_t b, unsigned long long* evals, purse_stream_t stream) {
  if (!b) return barg("purse_batch_sync: NULL batch");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && evals) e = cudaMemcpy(evals, b->d_evals, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "purse_batch_sync");
  if (status & kDevErrNumeric) {
    set_error("non-finite value on the device");
    return PURSE_ERR_NUMERIC;
  }
  return PURSE_OK;
}

}  // extern "C"
