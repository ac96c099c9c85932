// Step I (RANSAG for 3D-3D, Section IV) and the centre statistics of Step II
// (Alg. 2: R-bar = proj_SO3(sum R_j), t-bar = mean t_j; PCA velocity scaling
// for 2D-3D; perturbation radii), all in FP64.
#include "dev.cuh"
#include "internal.h"

namespace purse {

constexpr int kStatsThreads = 256;

// Block-wide sum of NV doubles per thread (result valid in thread 0).
template <int NV>
__device__ void block_sum(double (&v)[NV], double* red) {
  const int tid = threadIdx.x;
  for (int k = 0; k < NV; ++k) red[k * kStatsThreads + tid] = v[k];
  __syncthreads();
  for (int s = kStatsThreads / 2; s > 0; s >>= 1) {
    if (tid < s)
      for (int k = 0; k < NV; ++k) red[k * kStatsThreads + tid] += red[k * kStatsThreads + tid + s];
    __syncthreads();
  }
  for (int k = 0; k < NV; ++k) v[k] = red[k * kStatsThreads];
  __syncthreads();
}

// Centre statistics of one PURSE by one block of kStatsThreads threads.
// tab: FP64 constraint table (rows (a_i, r_i), then (b_i or z_i, r_i^2)).
__device__ void stats_block(const double* seeds, int s0, const double* tab, int n, int kind, double fx, double fy,
                            double t_p, double th_p, int raw_units, WalkStats* out, double* seed_data, double* red,
                            WalkStats& sh) {
  const int tid = threadIdx.x;
  // sums of seed rotations and translations
  double acc[12];
  for (int k = 0; k < 12; ++k) acc[k] = 0.0;
  for (int s = tid; s < s0; s += kStatsThreads)
    for (int k = 0; k < 12; ++k) acc[k] += seeds[12 * (size_t)s + k];
  block_sum<12>(acc, red);
  if (tid == 0) {
    const Q4<double> qb = rotation_maximising_trace(acc);  // proj_SO3(sum R_j)
    const M3<double> Rb = qmat(qb);
    for (int k = 0; k < 9; ++k) sh.Rbar[k] = Rb.m[k];
    for (int c = 0; c < 3; ++c) sh.tbar[c] = acc[9 + c] / s0;
  }
  __syncthreads();
  // covariance of the seed translations
  double cov[6] = {0, 0, 0, 0, 0, 0};
  for (int s = tid; s < s0; s += kStatsThreads) {
    const double d0 = seeds[12 * (size_t)s + 9] - sh.tbar[0];
    const double d1 = seeds[12 * (size_t)s + 10] - sh.tbar[1];
    const double d2 = seeds[12 * (size_t)s + 11] - sh.tbar[2];
    cov[0] += d0 * d0, cov[1] += d0 * d1, cov[2] += d0 * d2;
    cov[3] += d1 * d1, cov[4] += d1 * d2, cov[5] += d2 * d2;
  }
  block_sum<6>(cov, red);
  if (tid == 0) {
    // RMS spread of the model points
    double mean[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) mean[c] += tab[4 * i + c];
    for (int c = 0; c < 3; ++c) mean[c] /= n;
    double ss = 0.0, rsum = 0.0;
    for (int i = 0; i < n; ++i) {
      for (int c = 0; c < 3; ++c) ss += (tab[4 * i + c] - mean[c]) * (tab[4 * i + c] - mean[c]);
      rsum += tab[4 * i + 3];
    }
    sh.rho_a = sqrt(ss / n);
    for (int k = 0; k < 9; ++k) sh.S[k] = (k % 4 == 0) ? 1.0 : 0.0;
    if (kind == 0) {
      sh.sigma_t = rsum / n;
    } else {
      sh.sigma_t = rsum / n * sh.tbar[2] / (0.5 * (fx + fy));
      // PCA scaling of the centre velocity (Section IV, Step II; appendix dS_t sampler)
      double A[3][3] = {{cov[0] / s0, cov[1] / s0, cov[2] / s0},
                        {cov[1] / s0, cov[3] / s0, cov[4] / s0},
                        {cov[2] / s0, cov[4] / s0, cov[5] / s0}};
      double V[3][3];
      jacobi_eigen<3>(A, V);
      double sig[3], smax = 0.0;
      for (int k = 0; k < 3; ++k) {
        sig[k] = sqrt(fmax(A[k][k], 0.0));
        smax = fmax(smax, sig[k]);
      }
      if (s0 >= 4 && smax > 0.0) {
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) v += V[r][k] * (sig[k] / smax) * V[c][k];
            sh.S[3 * r + c] = v;
          }
      } else {
        const double tn = sqrt(sh.tbar[0] * sh.tbar[0] + sh.tbar[1] * sh.tbar[1] + sh.tbar[2] * sh.tbar[2]);
        const double u[3] = {sh.tbar[0] / tn, sh.tbar[1] / tn, sh.tbar[2] / tn};
        const double ratio = fmin(1.0, sh.rho_a / tn);
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) sh.S[3 * r + c] = u[r] * u[c] + ratio * ((r == c ? 1.0 : 0.0) - u[r] * u[c]);
      }
    }
    sh.r_trans = raw_units ? t_p : t_p * sh.sigma_t;
    sh.r_rot = raw_units ? th_p : th_p * sh.sigma_t / sh.rho_a;
    *out = sh;
  }
  __syncthreads();
  // per-seed start data: quaternion, translation, rotation axis away from R-bar, direction away from t-bar
  const double tn = sqrt(sh.tbar[0] * sh.tbar[0] + sh.tbar[1] * sh.tbar[1] + sh.tbar[2] * sh.tbar[2]);
  const double thr = 1e-9 * (1.0 + tn);
  for (int s = tid; s < s0; s += kStatsThreads) {
    const double* R0 = seeds + 12 * (size_t)s;
    double* o = seed_data + (size_t)s * kSeedStride;
    const Q4<double> q0 = quat_from_mat(R0);
    o[0] = q0.w, o[1] = q0.x, o[2] = q0.y, o[3] = q0.z;
    for (int c = 0; c < 3; ++c) o[4 + c] = R0[9 + c];
    double rel[9];  // R_0 R-bar^T
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        rel[3 * r + c] = R0[3 * r] * sh.Rbar[3 * c] + R0[3 * r + 1] * sh.Rbar[3 * c + 1] + R0[3 * r + 2] * sh.Rbar[3 * c + 2];
    const Q4<double> qr = quat_from_mat(rel);
    const double sn = sqrt(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z);
    const double ang = 2.0 * atan2(sn, qr.w);
    const bool has_u = ang > 1e-9;
    o[7] = has_u ? qr.x / sn : 0.0, o[8] = has_u ? qr.y / sn : 0.0, o[9] = has_u ? qr.z / sn : 0.0;
    const double d[3] = {R0[9] - sh.tbar[0], R0[10] - sh.tbar[1], R0[11] - sh.tbar[2]};
    const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const bool has_d = dn > thr;
    for (int c = 0; c < 3; ++c) o[10 + c] = has_d ? d[c] / dn : 0.0;
    for (int c = 13; c < kSeedStride; ++c) o[c] = 0.0;
  }
}

__global__ void __launch_bounds__(kStatsThreads)
    stats_kernel(const double* seeds, int s0, const double* tab, int n, int kind, double fx, double fy, double t_p,
                 double th_p, int raw_units, WalkStats* out, double* seed_data) {
  __shared__ double red[12 * kStatsThreads];
  __shared__ WalkStats sh;
  stats_block(seeds, s0, tab, n, kind, fx, fy, t_p, th_p, raw_units, out, seed_data, red, sh);
}

// One block per PURSE of a batch; one seed pose per PURSE.
__global__ void __launch_bounds__(kStatsThreads) stats_batch_kernel(const BatchPurseInfo* info, const double* tab64,
                                                                    const double* seeds, BatchStatParams sp,
                                                                    WalkStats* out, double* seed_data) {
  __shared__ double red[12 * kStatsThreads];
  __shared__ WalkStats sh;
  const int p = blockIdx.x;
  const BatchPurseInfo in = info[p];
  stats_block(seeds + 12 * (size_t)p, 1, tab64 + 4 * (size_t)in.table_off, in.n, in.kind, in.fx, in.fy,
              sp.t_p[in.kind], sp.th_p[in.kind], sp.raw[in.kind], out + p, seed_data + (size_t)p * kSeedStride, red,
              sh);
}

cudaError_t launch_stats_batch(int n_purses, const BatchPurseInfo* info, const double* tab64, const double* seeds,
                               const BatchStatParams& sp, WalkStats* out, double* seed_data, cudaStream_t st) {
  stats_batch_kernel<<<n_purses, kStatsThreads, 0, st>>>(info, tab64, seeds, sp, out, seed_data);
  return cudaGetLastError();
}

cudaError_t launch_stats(purse_t h, const double* d_seeds, int s0, const purse_params* p, WalkStats* d_stats,
                         double* d_seed_data, cudaStream_t st) {
  stats_kernel<<<1, kStatsThreads, 0, st>>>(d_seeds, s0, h->tables.f64, h->n, h->kind, h->K.fx, h->K.fy,
                                            p->trans_perturb, p->rot_perturb, p->perturb_units, d_stats, d_seed_data);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- RANSAG (3D-3D)
__device__ __forceinline__ uint32_t uniform_index(uint32_t word, uint32_t n) {
  return (uint32_t)(((uint64_t)word * n) >> 32);
}

__global__ void __launch_bounds__(128)
    ransag_kernel(const double* tab, int n, uint32_t k0, uint32_t k1, int trial0, int n_trials, double* pose,
                  uint8_t* acc) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n_trials) return;
  const uint32_t tau = (uint32_t)(trial0 + tid);
  Stream s(k0, k1, kPhaseRansag, 0u, 0u, tau);
  const uint32_t w0 = s.next(), w1 = s.next(), w2 = s.next();
  uint32_t i1 = uniform_index(w0, n);
  uint32_t i2 = uniform_index(w1, n - 1);
  i2 += (i2 >= i1);
  uint32_t i3 = uniform_index(w2, n - 2);
  const uint32_t lo = min(i1, i2), hi = max(i1, i2);
  i3 += (i3 >= lo);
  i3 += (i3 >= hi);
  const uint32_t idx[3] = {i1, i2, i3};
  double A[3][3], B[3][3];
  for (int c = 0; c < 3; ++c) {
    Stream sc(k0, k1, kPhaseRansag, (uint32_t)(c + 1), 0u, tau);
    int X, Y, Z;
    lattice_draw<false>(sc, X, Y, Z);
    const double* ai = tab + 4 * idx[c];
    const double* bi = tab + 4 * (n + idx[c]);
    const double r = ai[3];
    A[c][0] = ai[0], A[c][1] = ai[1], A[c][2] = ai[2];
    B[c][0] = bi[0] + r * (X / 1024.0);
    B[c][1] = bi[1] + r * (Y / 1024.0);
    B[c][2] = bi[2] + r * (Z / 1024.0);
  }
  double abar[3], bbar[3];
  for (int d = 0; d < 3; ++d) {
    abar[d] = (A[0][d] + A[1][d] + A[2][d]) / 3.0;
    bbar[d] = (B[0][d] + B[1][d] + B[2][d]) / 3.0;
  }
  double M[9];  // sum (b - bbar)(a - abar)^T
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double v = 0.0;
      for (int k = 0; k < 3; ++k) v += (B[k][r] - bbar[r]) * (A[k][c] - abar[c]);
      M[3 * r + c] = v;
    }
  const M3<double> R = qmat(rotation_maximising_trace(M));
  double t[3];
  for (int r = 0; r < 3; ++r) t[r] = bbar[r] - (R.m[3 * r] * abar[0] + R.m[3 * r + 1] * abar[1] + R.m[3 * r + 2] * abar[2]);
  bool ok = true;
  for (int i = 0; i < n && ok; ++i) {
    const double* ai = tab + 4 * i;
    const double* bi = tab + 4 * (n + i);
    double e2 = 0.0;
    for (int r = 0; r < 3; ++r) {
      const double e = R.m[3 * r] * ai[0] + R.m[3 * r + 1] * ai[1] + R.m[3 * r + 2] * ai[2] + t[r] - bi[r];
      e2 += e * e;
    }
    ok = e2 <= bi[3];
  }
  double* o = pose + 12 * (size_t)tid;
  for (int k = 0; k < 9; ++k) o[k] = R.m[k];
  for (int r = 0; r < 3; ++r) o[9 + r] = t[r];
  acc[tid] = ok ? 1 : 0;
}

cudaError_t launch_ransag(purse_t h, uint64_t seed, int trial0, int n_trials, double* d_pose, uint8_t* d_acc,
                          cudaStream_t st) {
  const int threads = 128;
  ransag_kernel<<<(n_trials + threads - 1) / threads, threads, 0, st>>>(
      h->tables.f64, h->n, (uint32_t)seed, (uint32_t)(seed >> 32), trial0, n_trials, d_pose, d_acc);
  return cudaGetLastError();
}

// In-order compaction of accepted trials: appends to d_seeds after *d_count entries.
__global__ void __launch_bounds__(1024)
    compact_kernel(const double* pose, const uint8_t* acc, int n_trials, double* seeds, int* count, int max_seeds) {
  __shared__ int warp_tot[32];
  __shared__ int base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) base = *count;
  __syncthreads();
  for (int tile = 0; tile < n_trials; tile += 1024) {
    if (base >= max_seeds) break;
    const int i = tile + tid;
    const bool f = i < n_trials && acc[i];
    const unsigned bal = __ballot_sync(kFullMask, f);
    const int before = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int k = 0; k < 32; ++k) {
      if (k < warp) off += warp_tot[k];
      tot += warp_tot[k];
    }
    const int pos = base + off + before;
    if (f && pos < max_seeds)
      for (int k = 0; k < 12; ++k) seeds[12 * (size_t)pos + k] = pose[12 * (size_t)i + k];
    __syncthreads();
    if (tid == 0) base += tot;
    __syncthreads();
  }
  if (tid == 0) *count = min(base, max_seeds);
}

cudaError_t launch_compact(const double* d_pose, const uint8_t* d_acc, int n_trials, double* d_seeds,
                           int* d_count, int max_seeds, cudaStream_t st) {
  compact_kernel<<<1, 1024, 0, st>>>(d_pose, d_acc, n_trials, d_seeds, d_count, max_seeds);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- stream inspection
__global__ void rng_words_kernel(uint32_t k0, uint32_t k1, uint32_t phase, uint32_t j, uint32_t i, uint32_t w0,
                                 int n_streams, int n_words, uint32_t* words, int32_t* lattice, int unit) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_streams) return;
  Stream st(k0, k1, phase, j, i, w0 + (uint32_t)s);
  for (int k = 0; k < n_words; ++k) words[(size_t)s * n_words + k] = st.next();
  if (!lattice) return;
  Stream sl(k0, k1, phase, j, i, w0 + (uint32_t)s);
  int X, Y, Z, used = 0;
  bool ok = false;
  // same acceptance as lattice_draw, also reporting the attempts used
  for (int a = 0; a < kMaxAttempts && !ok; ++a) {
    const uint32_t wd = sl.next();
    X = 2 * (int)(wd & 1023u) - 1023;
    Y = 2 * (int)((wd >> 10) & 1023u) - 1023;
    Z = 2 * (int)((wd >> 20) & 1023u) - 1023;
    const int r2 = X * X + Y * Y + Z * Z;
    ok = unit ? (r2 <= (1 << 20) && r2 >= (1 << 14)) : (r2 <= (1 << 20));
    used = a + 1;
  }
  Stream sv(k0, k1, phase, j, i, w0 + (uint32_t)s);
  int x2, y2, z2;
  const bool ok2 = unit ? lattice_draw<true>(sv, x2, y2, z2) : lattice_draw<false>(sv, x2, y2, z2);
  int32_t* o = lattice + 4 * (size_t)s;
  o[0] = x2, o[1] = y2, o[2] = z2, o[3] = (ok && ok2) ? used : kMaxAttempts;
}

cudaError_t launch_rng_words(uint64_t seed, uint32_t phase, uint32_t j, uint32_t i, uint32_t w0, int n_streams,
                             int n_words, uint32_t* d_words, int32_t* d_lattice, int unit, cudaStream_t st) {
  if (n_streams == 0) return cudaSuccess;
  rng_words_kernel<<<(n_streams + 127) / 128, 128, 0, st>>>((uint32_t)seed, (uint32_t)(seed >> 32), phase, j, i, w0,
                                                            n_streams, n_words, d_words, d_lattice, unit);
  return cudaGetLastError();
}

}  // namespace purse
