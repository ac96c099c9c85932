// Host-side internals shared by the translation units of libpurse.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/purse.h"

namespace purse {

// Constraint table in the layout the kernels stage into shared memory:
// rows 0..n-1: (model x, y, z, r), rows n..2n-1: (obs x, y, z or 0, r^2).
// One copy per arithmetic type; 8 n values, a multiple of 16 bytes.
struct purse_tables {
  float* f32 = nullptr;
  double* f64 = nullptr;
};

// Output of the centre-statistics kernel (Alg. 2, R-bar / t-bar lines; PCA of
// Section IV for 2D-3D; perturbation radii).
struct WalkStats {
  double Rbar[9];
  double tbar[3];
  double S[9];
  double sigma_t, rho_a, r_trans, r_rot;
  float Sf[9];  // S rounded, for the FP32 walks
};

// Per-seed data (kSeedStride doubles): doubles 0-3 unit quaternion (w >= 0) and 4-6
// translation of the seed, 7-9 the axis u of R_0 R-bar^T (0 below 1e-9 rad), 10-12 the unit
// direction of t_0 - t-bar (0 when degenerate); from double 16 on, floats for the FP32 walks:
// 0-3 quaternion hi, 4-7 quaternion lo, 8-10 translation hi, 11-13 translation lo (hi + lo the
// double-float split of the FP64 values), 14-16 u, 17-19 direction.
constexpr int kSeedStride = 32;
constexpr int kSeedFloats = 16;  // double offset of the float part

// Values per walk in the boundary-snap record (see purse_sample).
constexpr int kSnapStride = 12;

// Largest sample count of a ball call: sample indices are 32-bit and the grid-stride loops of
// the ball kernels step by up to 2^20 past the last index.
constexpr int kMaxBallSamples = 2147483647 - (1 << 21);

// Per-PURSE description inside a batch (device array).
struct BatchPurseInfo {
  int kind, n, table_off, pad;  // table rows [table_off, table_off + 2 n) of the concatenated tables
  double fx, fy, cx, cy;
  double rho_max;  // largest model-point radius max_i |a_i| (or |Z_i|)
};

// Perturbation parameters of the two kinds (index = kind) for the batched statistics.
struct BatchStatParams {
  double t_p[2], th_p[2];
  int raw[2];
};

// Everything the batched walk kernel reads (kernel parameter).
struct BatchArgs {
  const BatchPurseInfo* info;
  const float* table;  // FP32 tables, rows of 4 floats
  const double* table64;  // the same tables in FP64 (read by the boundary snap)
  const float* ell;       // NULL, or noise factors U_i of eq. 4: 8 floats per keypoint in CSR order
  const double* ell64;    // the same in FP64 (statistics, boundary snap)
  const WalkStats* stats;
  const double* seed_data;
  int n_purses, n_samples, nmax;
  int n_iter[2], n_perturb[2], n_keep[2], n_steps[2];
  double omega0[2], v0[2], gamma[2];
  const unsigned long long* seed;  // device scalar: PURSE p uses key seed + p
  unsigned int* counter;           // work queue head
  unsigned int total_items;        // 2 x n_purses x n_samples items (p, sampler, walk)
  float* q_rot;                    // n_purses x n_samples x 4 (dS_R sampler)
  float* t_rot;                    // n_purses x n_samples x 3
  float* q_tr;                     // dS_t sampler
  float* t_tr;
  float* snap_rot;  // NULL or n_purses x n_samples x kSnapStride snap records (dS_R walks)
  float* snap_tr;   // same for the dS_t walks
  int32_t* fstar;   // NULL or n_purses x 2: farthest sample from each final centre
  int tr3d;         // 3D-3D: run the dS_t walks and take the translation ball from them (v0 > 0)
  int reg;          // every PURSE is a pose-regression PURSE (Example 3), parameters in slot 0
  int* status;
  unsigned long long* evals;
};

struct WalkArgs {
  const void* table;
  const double* table64;  // the FP64 table (read by the boundary snap at either walk precision)
  const void* ell;  // noise factors U_i of eq. 4 (8 values per constraint, the table's precision) or NULL
  const double* ell64;  // the same in FP64 (read by the boundary snap) or NULL
  int n;
  double fx, fy, cx, cy;
  double rho_max;  // largest model-point radius max_i |Z_i|
  const double* seed_data;  // s0 x kSeedStride
  int s0;
  const WalkStats* stats;
  int n_samples, n_iter, n_perturb, n_keep, n_steps;
  double omega0, v0, gamma;
  uint32_t key0, key1;
  uint32_t rk[20];  // Philox round keys: (key0 + r W0, key1 + r W1), r = 0..9
  void* out_q;
  void* out_t;
  int16_t* trace;
  void* out_snap;
  int* status;
  unsigned long long* evals;  // executed (pose, constraint) evaluations
  int stall_probe;            // PURSE_FAULT=stall: a bounded wait that runs out after the staging
};

}  // namespace purse

struct purse_s {
  int kind = 0;
  int n = 0;
  double rho_max = 0;  // largest model-point radius
  purse_intrinsics K{0, 0, 0, 0};
  purse::purse_tables tables;
  // noise factors of eq. 4 (Lambda_i = U_i^T U_i, 8 values per constraint) or NULL (identity)
  double* ell64 = nullptr;
  float* ell32 = nullptr;
  int* d_status = nullptr;
  unsigned long long* d_evals = nullptr;  // evaluation counter of the last purse_sample
  // scratch owned by the handle, grown on demand
  void* d_scratch = nullptr;
  size_t scratch_bytes = 0;
  // state kept by megb_solve
  int megb_iters = 0;
  int megb_precision = 0;
  const void* megb_q = nullptr;
  const void* megb_t = nullptr;
  int megb_nrot = 0, megb_ntr = 0;
  int megb_navg = 1;  // 1: the last solve returned C_K, c_K (megb_backward differentiates only that)
  int sm_count = 0;
};

namespace purse {

void set_error(const std::string& msg);

// Host-side fault injection for the failure-detection tests.  The environment variable
// PURSE_FAULT (read at every call) lists sites, comma-separated:
//   alloc       every device allocation of the library is refused (PURSE_ERR_NOMEM) before
//               cudaMalloc is called;
//   launch      every call that would queue GPU work is refused (PURSE_ERR_CUDA) before it does;
//   nan_input   the PURSE constructors see a NaN in their first observation (PURSE_ERR_ARG);
//   empty_seed  Step I accepts no pose and purse_sample sees no seed (PURSE_ERR_EMPTY);
//   stall       the walk kernels, after staging their table, wait on a barrier that nothing
//               arrives at, give up after a short poll limit and flag a timeout
//               (PURSE_ERR_TIMEOUT at the next purse_sync).
// No site faults, traps or hangs the GPU: every refusal happens on the host, and the stall is a
// bounded wait with no copy in flight.
bool fault_at(const char* site);
purse_status injected_fault(const char* site, const char* where);  // sets the message
cudaError_t dev_alloc(void** ptr, size_t bytes);  // cudaMalloc, refused under PURSE_FAULT=alloc
purse_status make_handle(int kind, int n, const std::vector<double>& t64, const purse_intrinsics& Kc, double rho_max,
                         purse_t* out);
purse_status cuda_fail(cudaError_t e, const char* where);
purse_status ensure_scratch(purse_t h, size_t bytes);

// Autotuner cache (tune.cu).  Operations: walk (warps per block), megb (samples per thread of the
// persistent ball kernel), dist (resident tensor-core CTAs per SM), batch (reserved).
enum TuneOp { kTuneWalk = 0, kTuneMegb = 1, kTuneDist = 2, kTuneBatch = 3 };
struct TuneEntry {
  int cfg;
  float ms, default_ms;
};
// The shape a launcher uses: a tuning call's forced candidate, else the cached choice for
// (op, kind, n, samples, variant, this GPU), else fallback.
int tuned_config(int op, int kind, int n, long long samples, int variant, int fallback);
bool tune_lookup(int op, int kind, int n, long long samples, int variant, const char* gpu, TuneEntry* out);
void tune_store(int op, int kind, int n, long long samples, int variant, const char* gpu, const TuneEntry& e);

// Launchers (one translation unit each).
cudaError_t launch_stats(purse_t h, const double* d_seeds, int s0, const purse_params* p, WalkStats* d_stats,
                         double* d_seed_data, cudaStream_t st);  // takes h->ell64 into the translation scale
cudaError_t launch_walk(purse_t h, const purse_params* p, const WalkArgs& a, cudaStream_t st);
cudaError_t launch_stats_batch(int n_purses, const BatchPurseInfo* info, const double* tab64, const double* ell64,
                               const double* seeds, const BatchStatParams& sp, WalkStats* out, double* seed_data,
                               cudaStream_t st);
// lam: the batch carries noise matrices (the tables and slabs of the walks with U_i)
size_t batch_walk_smem(int nmax, int n_perturb, int n_steps, int warps, bool lam = false, bool reg = false);
cudaError_t launch_batch_walk(const BatchArgs& b, int chunk, int warps, int sm_count, cudaStream_t st);
cudaError_t launch_megb_batch(const BatchArgs& b, int n_iters, double* d_results, int32_t* d_farthest,
                              cudaStream_t st);
cudaError_t launch_ransag(purse_t h, uint64_t seed, int trial0, int n_trials, double* d_pose, uint8_t* d_acc,
                          cudaStream_t st);
cudaError_t launch_ransag_p3p(purse_t h, uint64_t seed, int trial0, int n_trials, double* d_pose, uint8_t* d_acc,
                              cudaStream_t st);
cudaError_t launch_convex_seeds(purse_t h, uint64_t seed, int trial0, int n_trials, double* d_pose, uint8_t* d_acc,
                                cudaStream_t st);
cudaError_t launch_compact(const double* d_pose, const uint8_t* d_acc, int n_trials, double* d_seeds,
                           int* d_count, int max_seeds, cudaStream_t st);
size_t plain_scratch_bytes(const purse_params* p, int n_samples, int* chunk);
cudaError_t launch_plain(purse_t h, const purse_params* p, const WalkStats* d_stats, const double* d_seed_data, int s0,
                         uint64_t seed, int n_samples, void* d_q, void* d_t, int16_t* d_trace, void* scratch,
                         size_t scratch_bytes, int chunk, cudaStream_t st);
cudaError_t launch_plain_dist(purse_t h, const float* d_poses, long n_poses, float* d_dist, cudaStream_t st);
cudaError_t launch_tc_dist(purse_t h, int passes, const float* d_poses, long n_poses, float* d_dist, cudaStream_t st);
cudaError_t launch_eval(purse_t h, int precision, const void* d_poses, int n_poses, void* d_margin,
                        int32_t* d_active, void* d_grad, cudaStream_t st);
cudaError_t launch_rng_words(uint64_t seed, uint32_t phase, uint32_t j, uint32_t i, uint32_t w0, int n_streams,
                             int n_words, uint32_t* d_words, int32_t* d_lattice, int unit, cudaStream_t st);
size_t megb_scratch_bytes(int n_iters, int sm_count);
const char* noise_factor(const double* L, int d, double* o);
// navg > 1: the output rule of Alg. 6 (centre from the last navg iterates; megb_solve_mean)
cudaError_t launch_megb(purse_t h, int precision, int n_iters, const void* d_q, int n_rot, const void* d_t,
                        int n_tr, double* d_result, int32_t* d_farthest, void* scratch, cudaStream_t st,
                        int navg = 1);
size_t exact_scratch_bytes(int sm_count);
cudaError_t launch_megb_exact(purse_t h, int precision, const void* d_q, long n_rot, const void* d_t, long n_tr,
                              const double* d_ref, double* d_result, void* scratch, cudaStream_t st);
size_t megb_backward_scratch_bytes(int n_iters, int sm_count, int n);
cudaError_t launch_batch_backward(const BatchArgs& b, int n_iters, const int32_t* d_far, const double* d_results,
                                  const double* d_grad_results, void* d_cs, double* d_grad_obs, double* d_grad_radii,
                                  cudaStream_t st);
cudaError_t launch_megb_backward(purse_t h, int precision, int n_iters, const void* d_q, const void* d_snap_rot,
                                 int n_rot, const void* d_t, const void* d_snap_tr, int n_tr,
                                 const int32_t* d_farthest, const double* d_result, const double* d_grad_result,
                                 double* d_grad_obs, double* d_grad_radii, void* scratch, cudaStream_t st);

}  // namespace purse
