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
                            WalkStats& sh, const double* ell = nullptr) {
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
      // noise radius; with a noise matrix (eq. 4) the geometric-mean semi-axis r_i det(Lambda_i)^(-1/(2d)),
      // det(Lambda_i) = (prod of the diagonal of its Cholesky factor)^2
      double scale = 1.0;
      if (ell && kind == 0) scale = 1.0 / cbrt(ell[8 * i] * ell[8 * i + 3] * ell[8 * i + 5]);
      if (ell && kind == 1) scale = 1.0 / sqrt(ell[8 * i] * ell[8 * i + 2]);
      rsum += tab[4 * i + 3] * scale;
    }
    sh.rho_a = sqrt(ss / n);
    for (int k = 0; k < 9; ++k) sh.S[k] = (k % 4 == 0) ? 1.0 : 0.0;
    if (kind == 0) {
      sh.sigma_t = rsum / n;
    } else if (kind == 2) {
      // pose regression: translation scale mean beta^t (rows 0..n-1 hold (t_i, beta_i^t)); rotation scale
      // mean beta^R / sqrt(2), the angle of a Frobenius distance, written through rho_a
      double rb = 0.0;
      for (int i = 0; i < n; ++i) rb += tab[4 * (n + i) + 3];
      sh.sigma_t = rsum / n;
      sh.rho_a = sh.sigma_t * sqrt(2.0) / (rb / n);
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
    for (int k = 0; k < 9; ++k) sh.Sf[k] = (float)sh.S[k];
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
    for (int c = 13; c < kSeedFloats; ++c) o[c] = 0.0;
    float* f = reinterpret_cast<float*>(o + kSeedFloats);
    for (int c = 0; c < 7; ++c) {
      const float hi = (float)o[c];
      f[(c < 4 ? c : c + 4)] = hi;
      f[(c < 4 ? c + 4 : c + 7)] = (float)(o[c] - (double)hi);
    }
    for (int c = 0; c < 6; ++c) f[14 + c] = (float)o[7 + c];
    for (int c = 20; c < 2 * (kSeedStride - kSeedFloats); ++c) f[c] = 0.0f;
  }
}

__global__ void __launch_bounds__(kStatsThreads)
    stats_kernel(const double* seeds, int s0, const double* tab, const double* ell, int n, int kind, double fx,
                 double fy, double t_p,
                 double th_p, int raw_units, WalkStats* out, double* seed_data) {
  __shared__ double red[12 * kStatsThreads];
  __shared__ WalkStats sh;
  stats_block(seeds, s0, tab, n, kind, fx, fy, t_p, th_p, raw_units, out, seed_data, red, sh, ell);
}

// One block per PURSE of a batch; one seed pose per PURSE.
__global__ void __launch_bounds__(kStatsThreads) stats_batch_kernel(const BatchPurseInfo* info, const double* tab64,
                                                                    const double* ell64, const double* seeds,
                                                                    BatchStatParams sp, WalkStats* out,
                                                                    double* seed_data) {
  __shared__ double red[12 * kStatsThreads];
  __shared__ WalkStats sh;
  const int p = blockIdx.x;
  const BatchPurseInfo in = info[p];
  const int pk = in.kind == 1 ? 1 : 0;  // parameter slot: 2D-3D, else 3D-3D or pose regression
  stats_block(seeds + 12 * (size_t)p, 1, tab64 + 4 * (size_t)in.table_off, in.n, in.kind, in.fx, in.fy,
              sp.t_p[pk], sp.th_p[pk], sp.raw[pk], out + p, seed_data + (size_t)p * kSeedStride, red,
              sh, ell64 ? ell64 + 8 * (size_t)(in.table_off / 2) : nullptr);
}

cudaError_t launch_stats_batch(int n_purses, const BatchPurseInfo* info, const double* tab64, const double* ell64,
                               const double* seeds, const BatchStatParams& sp, WalkStats* out, double* seed_data,
                               cudaStream_t st) {
  stats_batch_kernel<<<n_purses, kStatsThreads, 0, st>>>(info, tab64, ell64, seeds, sp, out, seed_data);
  return cudaGetLastError();
}

cudaError_t launch_stats(purse_t h, const double* d_seeds, int s0, const purse_params* p, WalkStats* d_stats,
                         double* d_seed_data, cudaStream_t st) {
  stats_kernel<<<1, kStatsThreads, 0, st>>>(d_seeds, s0, h->tables.f64, h->ell64, h->n, h->kind, h->K.fx, h->K.fy,
                                            p->trans_perturb, p->rot_perturb, p->perturb_units, d_stats, d_seed_data);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- RANSAG (3D-3D)
__device__ __forceinline__ uint32_t uniform_index(uint32_t word, uint32_t n) {
  return (uint32_t)(((uint64_t)word * n) >> 32);
}

// Least-squares rotation of point pairs (the maximiser of tr(R^T M), M = sum (b - bbar)(a - abar)^T) by
// Theobald's quaternion characteristic polynomial method (QCP, Acta Cryst. A 61, 2005): the largest
// eigenvalue of Horn's 4 x 4 matrix N is the largest root of det(N - l I) = l^4 + c2 l^2 + c1 l + c0 with
// c2 = -2 |M|_F^2, c1 = -8 det M, c0 = det N, reached by Newton's method from the bound
// l0 = (E_a + E_b) / 2 >= l_max (E the centred sums of squares); its eigenvector is a column of the
// adjugate of N - l I (the one of largest norm, as in Liu, Agrafiotis and Theobald, 2010), then one
// step of inverse iteration on N - l I takes it to rounding.  The same optimum as Horn's Jacobi
// solution (rotation_maximising_trace) in a few hundred FP64 operations instead of some fifteen hundred;
// any non-finite step falls back to that solution.
__device__ __forceinline__ void adj4(const double (&a)[4][4], double (&b)[4][4], double& det) {
  const double s0 = a[0][0] * a[1][1] - a[1][0] * a[0][1], s1 = a[0][0] * a[1][2] - a[1][0] * a[0][2];
  const double s2 = a[0][0] * a[1][3] - a[1][0] * a[0][3], s3 = a[0][1] * a[1][2] - a[1][1] * a[0][2];
  const double s4 = a[0][1] * a[1][3] - a[1][1] * a[0][3], s5 = a[0][2] * a[1][3] - a[1][2] * a[0][3];
  const double c5 = a[2][2] * a[3][3] - a[3][2] * a[2][3], c4 = a[2][1] * a[3][3] - a[3][1] * a[2][3];
  const double c3 = a[2][1] * a[3][2] - a[3][1] * a[2][2], c2 = a[2][0] * a[3][3] - a[3][0] * a[2][3];
  const double c1 = a[2][0] * a[3][2] - a[3][0] * a[2][2], c0 = a[2][0] * a[3][1] - a[3][0] * a[2][1];
  b[0][0] = a[1][1] * c5 - a[1][2] * c4 + a[1][3] * c3, b[0][1] = -a[0][1] * c5 + a[0][2] * c4 - a[0][3] * c3;
  b[0][2] = a[3][1] * s5 - a[3][2] * s4 + a[3][3] * s3, b[0][3] = -a[2][1] * s5 + a[2][2] * s4 - a[2][3] * s3;
  b[1][0] = -a[1][0] * c5 + a[1][2] * c2 - a[1][3] * c1, b[1][1] = a[0][0] * c5 - a[0][2] * c2 + a[0][3] * c1;
  b[1][2] = -a[3][0] * s5 + a[3][2] * s2 - a[3][3] * s1, b[1][3] = a[2][0] * s5 - a[2][2] * s2 + a[2][3] * s1;
  b[2][0] = a[1][0] * c4 - a[1][1] * c2 + a[1][3] * c0, b[2][1] = -a[0][0] * c4 + a[0][1] * c2 - a[0][3] * c0;
  b[2][2] = a[3][0] * s4 - a[3][1] * s2 + a[3][3] * s0, b[2][3] = -a[2][0] * s4 + a[2][1] * s2 - a[2][3] * s0;
  b[3][0] = -a[1][0] * c3 + a[1][1] * c1 - a[1][2] * c0, b[3][1] = a[0][0] * c3 - a[0][1] * c1 + a[0][2] * c0;
  b[3][2] = -a[3][0] * s3 + a[3][1] * s1 - a[3][2] * s0, b[3][3] = a[2][0] * s3 - a[2][1] * s1 + a[2][2] * s0;
  det = s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
}

__device__ Q4<double> rotation_qcp(const double* M, double l0) {
  double N[4][4];
  N[0][0] = M[0] + M[4] + M[8], N[1][1] = M[0] - M[4] - M[8];
  N[2][2] = -M[0] + M[4] - M[8], N[3][3] = -M[0] - M[4] + M[8];
  N[0][1] = N[1][0] = M[7] - M[5], N[0][2] = N[2][0] = M[2] - M[6], N[0][3] = N[3][0] = M[3] - M[1];
  N[1][2] = N[2][1] = M[1] + M[3], N[1][3] = N[3][1] = M[2] + M[6], N[2][3] = N[3][2] = M[5] + M[7];
  double f2 = 0.0;
  for (int k = 0; k < 9; ++k) f2 += M[k] * M[k];
  const double c2 = -2.0 * f2;
  const double c1 = -8.0 * (M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                            M[2] * (M[3] * M[7] - M[4] * M[6]));
  double B[4][4], c0;
  adj4(N, B, c0);
  double l = l0;
  for (int it = 0; it < 40; ++it) {  // from above, decreasing to the largest root
    const double P = ((l * l + c2) * l + c1) * l + c0, dP = (4.0 * l * l + 2.0 * c2) * l + c1;
    if (!(dP != 0.0)) break;
    const double dl = P / dP;
    l -= dl;
    if (!(dl > 1e-14 * fabs(l))) break;
  }
  double A[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) A[i][j] = N[i][j] - (i == j ? l : 0.0);
  double det;
  adj4(A, B, det);
  int best = 0;
  double bn = -1.0;
  for (int j = 0; j < 4; ++j) {
    const double nj = B[0][j] * B[0][j] + B[1][j] * B[1][j] + B[2][j] * B[2][j] + B[3][j] * B[3][j];
    if (nj > bn) bn = nj, best = j;
  }
  // one step of inverse iteration: solve A y = v (Gaussian elimination with partial pivoting)
  double G[4][5];
  const double inv = rsqrt(bn);
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) G[i][j] = A[i][j];
    G[i][4] = B[i][best] * inv;
  }
  Q4<double> q{G[0][4], G[1][4], G[2][4], G[3][4]};
  bool solved = bn > 0.0;
  for (int c = 0; c < 4 && solved; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(G[r][c]) > fabs(G[piv][c])) piv = r;
    if (G[piv][c] == 0.0) {
      solved = false;  // A singular to rounding: v is already the eigenvector
      break;
    }
    if (piv != c)
      for (int j = 0; j < 5; ++j) {
        const double tmp = G[c][j];
        G[c][j] = G[piv][j], G[piv][j] = tmp;
      }
    for (int r = c + 1; r < 4; ++r) {
      const double f = G[r][c] / G[c][c];
      for (int j = c; j < 5; ++j) G[r][j] -= f * G[c][j];
    }
  }
  if (solved) {
    double y[4];
    for (int r = 3; r >= 0; --r) {
      double acc = G[r][4];
      for (int j = r + 1; j < 4; ++j) acc -= G[r][j] * y[j];
      y[r] = acc / G[r][r];
    }
    q = Q4<double>{y[0], y[1], y[2], y[3]};
  }
  q = qnormalize(q);
  if (!(isfinite(q.w) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z)) || !(bn > 0.0))
    return rotation_maximising_trace(M);
  if (q.w < 0.0) q = Q4<double>{-q.w, -q.x, -q.y, -q.z};
  return q;
}

__global__ void __launch_bounds__(128)
    ransag_kernel(const double* tab, const double* ell, int n, uint32_t k0, uint32_t k1, int trial0, int n_trials,
                  double* pose, uint8_t* acc) {
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
    double e0 = X / 1024.0, e1 = Y / 1024.0, e2 = Z / 1024.0;
    if (ell) {  // a point of the noise ellipsoid: e = U^-1 u (back substitution)
      const double* U = ell + 8 * idx[c];
      e2 = e2 / U[5];
      e1 = (e1 - U[4] * e2) / U[3];
      e0 = (e0 - U[1] * e1 - U[2] * e2) / U[0];
    }
    A[c][0] = ai[0], A[c][1] = ai[1], A[c][2] = ai[2];
    B[c][0] = bi[0] + r * e0;
    B[c][1] = bi[1] + r * e1;
    B[c][2] = bi[2] + r * e2;
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
  double ea = 0.0, eb = 0.0;  // centred sums of squares: (ea + eb) / 2 bounds the largest eigenvalue
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d)
      ea += (A[k][d] - abar[d]) * (A[k][d] - abar[d]), eb += (B[k][d] - bbar[d]) * (B[k][d] - bbar[d]);
  const M3<double> R = qmat(rotation_qcp(M, 0.5 * (ea + eb)));
  double t[3];
  for (int r = 0; r < 3; ++r) t[r] = bbar[r] - (R.m[3 * r] * abar[0] + R.m[3 * r + 1] * abar[1] + R.m[3 * r + 2] * abar[2]);
  bool ok = true;
  for (int i = 0; i < n && ok; ++i) {
    const double* ai = tab + 4 * i;
    const double* bi = tab + 4 * (n + i);
    double e[3];
    for (int r = 0; r < 3; ++r)
      e[r] = R.m[3 * r] * ai[0] + R.m[3 * r + 1] * ai[1] + R.m[3 * r + 2] * ai[2] + t[r] - bi[r];
    double e2;
    if (ell) {
      const double* U = ell + 8 * i;
      const double a = U[0] * e[0] + U[1] * e[1] + U[2] * e[2], b = U[3] * e[1] + U[4] * e[2], c = U[5] * e[2];
      e2 = a * a + b * b + c * c;
    } else {
      e2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
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
      h->tables.f64, h->ell64, h->n, (uint32_t)seed, (uint32_t)(seed >> 32), trial0, n_trials, d_pose, d_acc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- RANSAG (2D-3D, P3P)
// First accepted 2-D lattice point of the stream: X = 2 (word & 1023) - 1023,
// Y = 2 ((word >> 10) & 1023) - 1023, accepted when X^2 + Y^2 <= 2^20 (zero after kMaxAttempts).
__device__ __forceinline__ void disk_draw(Stream& s, int& x, int& y) {
  for (int a = 0; a < kMaxAttempts; ++a) {
    const uint32_t wd = s.next();
    const int X = 2 * (int)(wd & 1023u) - 1023;
    const int Y = 2 * (int)((wd >> 10) & 1023u) - 1023;
    if (X * X + Y * Y <= (1 << 20)) {
      x = X, y = Y;
      return;
    }
  }
  x = y = 0;
}

__device__ __forceinline__ double horner(const double* c, int deg, double x) {
  double v = c[deg];
  for (int k = deg - 1; k >= 0; --k) v = fma(v, x, c[k]);
  return v;
}

// Real roots of c3 x^3 + c2 x^2 + c1 x + c0 (c3 != 0), Cardano's formula for one real root and
// the trigonometric form for three, each polished by two Newton steps; ascending.
__device__ int cubic_real_roots(double c3, double c2, double c1, double c0, double (&r)[3]) {
  const double a = c2 / c3, b = c1 / c3, c = c0 / c3;
  const double p = b - a * a / 3.0, q = 2.0 * a * a * a / 27.0 - a * b / 3.0 + c;
  const double disc = q * q / 4.0 + p * p * p / 27.0;
  int m;
  if (disc > 0.0 || p == 0.0) {
    const double sd = sqrt(fmax(disc, 0.0));
    r[0] = cbrt(-q / 2.0 + sd) + cbrt(-q / 2.0 - sd) - a / 3.0;
    m = 1;
  } else {
    const double s = 2.0 * sqrt(-p / 3.0);
    const double arg = fmin(1.0, fmax(-1.0, (3.0 * q) / (p * s)));
    const double phi = acos(arg) / 3.0;
    for (int k = 0; k < 3; ++k) r[k] = s * cos(phi - 2.0943951023931957 * k) - a / 3.0;
    m = 3;
  }
  const double cc[4] = {c0, c1, c2, c3}, dc[3] = {c1, 2.0 * c2, 3.0 * c3};
  for (int k = 0; k < m; ++k)
    for (int it = 0; it < 2; ++it) {
      const double d = horner(dc, 2, r[k]);
      if (d != 0.0) r[k] -= horner(cc, 3, r[k]) / d;
    }
  for (int i = 1; i < m; ++i)
    for (int j = i; j > 0 && r[j] < r[j - 1]; --j) {
      const double t = r[j];
      r[j] = r[j - 1], r[j - 1] = t;
    }
  return m;
}

// Real roots of the quartic A (increasing powers, A[4] != 0), ascending: the critical points (roots
// of the derivative) split [-B, B] (B = 1 + max |A_k / A_4|, Cauchy's bound) into intervals where A is
// monotone; each interval with a sign change holds one root, found by Newton steps safeguarded by
// bisection to full precision.  A double root without a sign change is not reported.
__device__ int quartic_real_roots(const double (&A)[5], double (&out)[4]) {
  double B = 0.0;
  for (int k = 0; k < 4; ++k) B = fmax(B, fabs(A[k] / A[4]));
  B += 1.0;
  double cr[3];
  const int m = cubic_real_roots(4.0 * A[4], 3.0 * A[3], 2.0 * A[2], A[1], cr);
  double x[5];
  int nx = 0;
  x[nx++] = -B;
  for (int k = 0; k < m; ++k)
    if (cr[k] > -B && cr[k] < B) x[nx++] = cr[k];
  x[nx++] = B;
  const double dA[4] = {A[1], 2.0 * A[2], 3.0 * A[3], 4.0 * A[4]};
  int nr = 0;
  for (int k = 0; k + 1 < nx; ++k) {
    double lo = x[k], hi = x[k + 1];
    double flo = horner(A, 4, lo), fhi = horner(A, 4, hi);
    if (flo == 0.0) {
      if (nr == 0 || out[nr - 1] != lo) out[nr++] = lo;
      continue;
    }
    if (fhi == 0.0 || (flo < 0.0) == (fhi < 0.0)) continue;  // the right end is the next interval's left end
    if (flo > 0.0) {  // orient: A(lo) < 0 < A(hi)
      const double t = lo;
      lo = hi, hi = t;
    }
    double v = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
      const double fv = horner(A, 4, v);
      if (fv == 0.0) break;
      if (fv < 0.0) lo = v; else hi = v;
      const double d = horner(dA, 3, v);
      double vn = d != 0.0 ? v - fv / d : 0.5 * (lo + hi);
      const double a0 = fmin(lo, hi), a1 = fmax(lo, hi);
      if (!(vn > a0 && vn < a1)) vn = 0.5 * (lo + hi);
      const bool done = fabs(vn - v) <= 1e-16 * fmax(1.0, fabs(v));
      v = vn;
      if (done) break;
    }
    out[nr++] = v;
  }
  return nr;
}

// Orthonormal frame (columns F[.][0..2]) of the triangle X_0 X_1 X_2: e_1 along X_1 - X_0, e_2 the
// unit part of X_2 - X_0 orthogonal to it, e_3 = e_1 x e_2.  For two congruent triangles the rotation
// F_X F_P^T maps one onto the other.
__device__ __forceinline__ void triangle_frame(const double (&X)[3][3], double (&F)[3][3]) {
  double u[3], v[3];
  for (int d = 0; d < 3; ++d) u[d] = X[1][d] - X[0][d], v[d] = X[2][d] - X[0][d];
  const double iu = rsqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  for (int d = 0; d < 3; ++d) u[d] *= iu;
  const double uv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
  for (int d = 0; d < 3; ++d) v[d] -= uv * u[d];
  const double iv = rsqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int d = 0; d < 3; ++d) v[d] *= iv;
  const double w[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
  for (int d = 0; d < 3; ++d) F[d][0] = u[d], F[d][1] = v[d], F[d][2] = w[d];
}

// One RANSAG trial of Step I for 2D-3D: three distinct constraints (index words as for 3D-3D), one
// pixel uniform in each noise disk, bearings f_i = K^-1 (z_i, 1) / |.|, and P3P by Grunert's
// elimination: the law of cosines on the triangle sides a = |P_2 - P_3|, b = |P_1 - P_3|,
// c = |P_1 - P_2| with s_2 = u s_1, s_3 = v s_1 gives the quartic
//   N(v)^2 - 2 cos(g) N(v) D(v) + (1 - (c^2 / b^2) Q(v)) D(v)^2 = 0,
//   Q = 1 + v^2 - 2 v cos(b'), N = k Q + v^2 - 1, k = (c^2 - a^2) / b^2, D = 2 (v cos(a') - cos(g))
// (a', b', g: the angles between bearings 2-3, 1-3, 1-2).  Per real root v (ascending):
// s_1 = b / sqrt(Q(v)); u from u^2 - 2 cos(g) u + 1 - (c^2 / b^2) Q(v) = 0, each root kept when
// u^2 + v^2 - 2 u v cos(a') = (a^2 / b^2) Q(v) holds to 1e-8 relative and every depth is positive;
// the pose maps P_i onto s_i f_i.  Those depths make the camera-frame triangle X_i = s_i f_i congruent
// to the model triangle (up to the root's rounding), so the rotation taking the orthonormal frame of
// (P_2 - P_1, P_3 - P_1) onto that of (X_2 - X_1, X_3 - X_1) is the least-squares (Horn / Arun) fit of
// the three pairs to rounding, formed without an eigen-decomposition (each FP64 instruction is
// expensive on this part); t = mean X - R mean P.
// Acceptance is division-free: P_z > 0 and |(y_i - c) X_z - f X_xy|_(Lambda) <= r_i X_z per constraint.
// Candidate slot k of the trial holds the k-th pose
// and acc = 1 when it lies in the PURSE (eq. 2/5, FP64).  Up to four slots per trial.
__global__ void __launch_bounds__(128)
    ransag_p3p_kernel(const double* tab, const double* ell, int n, double fx, double fy, double cx, double cy,
                      uint32_t k0, uint32_t k1, int trial0, int n_trials, double* pose, uint8_t* acc) {
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
  double P[3][3], f[3][3];
  for (int c = 0; c < 3; ++c) {
    Stream sc(k0, k1, kPhaseRansag, (uint32_t)(c + 1), 0u, tau);
    int X, Y;
    disk_draw(sc, X, Y);
    const double* ai = tab + 4 * idx[c];
    const double* bi = tab + 4 * (n + idx[c]);
    const double r = ai[3];
    P[c][0] = ai[0], P[c][1] = ai[1], P[c][2] = ai[2];
    double e0 = X / 1024.0, e1 = Y / 1024.0;
    if (ell) {  // a point of the noise ellipse: e = U^-1 u
      const double* U = ell + 8 * idx[c];
      e1 = e1 / U[2];
      e0 = (e0 - U[1] * e1) / U[0];
    }
    const double zx = bi[0] + r * e0, zy = bi[1] + r * e1;
    const double rx = (zx - cx) / fx, ry = (zy - cy) / fy;
    const double nr = sqrt(rx * rx + ry * ry + 1.0);
    f[c][0] = rx / nr, f[c][1] = ry / nr, f[c][2] = 1.0 / nr;
  }
  auto d2 = [&](int i, int j) {
    double v = 0.0;
    for (int k = 0; k < 3; ++k) v += (P[i][k] - P[j][k]) * (P[i][k] - P[j][k]);
    return v;
  };
  auto dotf = [&](int i, int j) { return f[i][0] * f[j][0] + f[i][1] * f[j][1] + f[i][2] * f[j][2]; };
  const double a2 = d2(1, 2), b2 = d2(0, 2), c2 = d2(0, 1), b = sqrt(b2);
  const double ca = dotf(1, 2), cb = dotf(0, 2), cg = dotf(0, 1);
  const double k = (c2 - a2) / b2;
  const double Q[3] = {1.0, -2.0 * cb, 1.0};
  const double N[3] = {k - 1.0, -2.0 * k * cb, k + 1.0};
  const double D[2] = {-2.0 * cg, 2.0 * ca};
  const double Rq[3] = {1.0 - (c2 / b2) * Q[0], -(c2 / b2) * Q[1], -(c2 / b2) * Q[2]};
  double A[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[i + j] += N[i] * N[j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 2; ++j) A[i + j] -= 2.0 * cg * N[i] * D[j];
  double DD[3] = {D[0] * D[0], 2.0 * D[0] * D[1], D[1] * D[1]};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[i + j] += Rq[i] * DD[j];
  double roots[4];
  const int nroots = A[4] != 0.0 ? quartic_real_roots(A, roots) : 0;
  int slot = 0;
  double* o = pose + 48 * (size_t)tid;
  uint8_t* ac = acc + 4 * (size_t)tid;
  for (int q = 0; q < nroots && slot < 4; ++q) {
    const double v = roots[q];
    const double Qv = horner(Q, 2, v);
    if (!(Qv > 0.0)) continue;
    const double disc = cg * cg - 1.0 + (c2 / b2) * Qv;
    if (disc < -1e-12) continue;
    const double r = sqrt(fmax(disc, 0.0));
    for (int h = 0; h < (r > 0.0 ? 2 : 1) && slot < 4; ++h) {
      const double u = h == 0 ? cg - r : cg + r;
      if (fabs(u * u + v * v - 2.0 * u * v * ca - (a2 / b2) * Qv) > 1e-8 * (1.0 + u * u + v * v)) continue;
      const double s1 = b / sqrt(Qv);
      const double sd[3] = {s1, u * s1, v * s1};
      if (!(sd[0] > 0.0 && sd[1] > 0.0 && sd[2] > 0.0)) continue;
      double B3[3][3], pbar[3], xbar[3];
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) B3[c][d] = sd[c] * f[c][d];
      for (int d = 0; d < 3; ++d) {
        pbar[d] = (P[0][d] + P[1][d] + P[2][d]) / 3.0;
        xbar[d] = (B3[0][d] + B3[1][d] + B3[2][d]) / 3.0;
      }
      double E[3][3], F[3][3];  // orthonormal frames (columns) of the model and camera triangles
      triangle_frame(P, E);
      triangle_frame(B3, F);
      M3<double> R;
      for (int rr = 0; rr < 3; ++rr)
        for (int cc = 0; cc < 3; ++cc) R.m[3 * rr + cc] = F[rr][0] * E[cc][0] + F[rr][1] * E[cc][1] + F[rr][2] * E[cc][2];
      double t[3];
      for (int rr = 0; rr < 3; ++rr)
        t[rr] = xbar[rr] - (R.m[3 * rr] * pbar[0] + R.m[3 * rr + 1] * pbar[1] + R.m[3 * rr + 2] * pbar[2]);
      bool ok = true;
      for (int i = 0; i < n && ok; ++i) {
        const double* ai = tab + 4 * i;
        const double* bi = tab + 4 * (n + i);
        const double X0 = R.m[0] * ai[0] + R.m[1] * ai[1] + R.m[2] * ai[2] + t[0];
        const double X1 = R.m[3] * ai[0] + R.m[4] * ai[1] + R.m[5] * ai[2] + t[1];
        const double X2 = R.m[6] * ai[0] + R.m[7] * ai[1] + R.m[8] * ai[2] + t[2];
        if (!(X2 > 0.0)) {
          ok = false;
        } else {
          // the pixel residual times X_z > 0
          const double gu = (bi[0] - cx) * X2 - fx * X0, gv = (bi[1] - cy) * X2 - fy * X1;
          double g2 = gu * gu + gv * gv;
          if (ell) {
            const double* U = ell + 8 * i;
            const double a = U[0] * gu + U[1] * gv, b = U[2] * gv;
            g2 = a * a + b * b;
          }
          const double rz = ai[3] * X2;
          ok = g2 <= rz * rz;
        }
      }
      double* os = o + 12 * slot;
      for (int kk = 0; kk < 9; ++kk) os[kk] = R.m[kk];
      for (int rr = 0; rr < 3; ++rr) os[9 + rr] = t[rr];
      ac[slot] = ok ? 1 : 0;
      ++slot;
    }
  }
  for (; slot < 4; ++slot) ac[slot] = 0;
}

cudaError_t launch_ransag_p3p(purse_t h, uint64_t seed, int trial0, int n_trials, double* d_pose, uint8_t* d_acc,
                              cudaStream_t st) {
  const int threads = 128;
  ransag_p3p_kernel<<<(n_trials + threads - 1) / threads, threads, 0, st>>>(
      h->tables.f64, h->ell64, h->n, h->K.fx, h->K.fy, h->K.cx, h->K.cy, (uint32_t)seed, (uint32_t)(seed >> 32),
      trial0, n_trials, d_pose, d_acc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Step I for pose regression
// Convex-combination sampler (Section IV, Step I, Example 3): trial tau draws weights uniform on the
// simplex, w_i = e_i / sum_j e_j with e_i = -log u_i, u_i = ((word_i >> 8) + 1/2) 2^-24 from words
// 0..n-1 of stream (5, 0, 0, tau); the candidate is t = sum w_i t_i, R = proj_SO3(sum w_i R_i) (the
// rotation maximising tr(R^T M), Horn's quaternion method), accepted if it lies in the PURSE
// (eq. PURSEreg, FP64).  Table rows: (t_i, beta_i^t), then the rows of R_i with beta_i^R in the first.
__global__ void __launch_bounds__(128)
    convex_seed_kernel(const double* tab, int n, uint32_t k0, uint32_t k1, int trial0, int n_trials, double* pose,
                       uint8_t* acc) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n_trials) return;
  const uint32_t tau = (uint32_t)(trial0 + tid);
  Stream s(k0, k1, kPhaseRansag, 0u, 0u, tau);
  double se = 0.0, t[3] = {0.0, 0.0, 0.0}, M[9];
  for (int k = 0; k < 9; ++k) M[k] = 0.0;
  for (int i = 0; i < n; ++i) {
    const uint32_t w = s.next();
    const double e = -log(((double)(w >> 8) + 0.5) * (1.0 / 16777216.0));
    se += e;
    for (int c = 0; c < 3; ++c) t[c] += e * tab[4 * i + c];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) M[3 * r + c] += e * tab[4 * ((1 + r) * n + i) + c];
  }
  for (int c = 0; c < 3; ++c) t[c] /= se;
  for (int k = 0; k < 9; ++k) M[k] /= se;
  const M3<double> R = qmat(rotation_maximising_trace(M));
  bool ok = true;
  for (int i = 0; i < n && ok; ++i) {
    double e2 = 0.0, d2 = 0.0;
    for (int c = 0; c < 3; ++c) e2 += (t[c] - tab[4 * i + c]) * (t[c] - tab[4 * i + c]);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        const double d = R.m[3 * r + c] - tab[4 * ((1 + r) * n + i) + c];
        d2 += d * d;
      }
    const double bt = tab[4 * i + 3], bR = tab[4 * (n + i) + 3];
    ok = bR - sqrt(d2) >= 0.0 && bt - sqrt(e2) >= 0.0;
  }
  double* o = pose + 12 * (size_t)tid;
  for (int k = 0; k < 9; ++k) o[k] = R.m[k];
  for (int c = 0; c < 3; ++c) o[9 + c] = t[c];
  acc[tid] = ok ? 1 : 0;
}

cudaError_t launch_convex_seeds(purse_t h, uint64_t seed, int trial0, int n_trials, double* d_pose, uint8_t* d_acc,
                                cudaStream_t st) {
  const int threads = 128;
  convex_seed_kernel<<<(n_trials + threads - 1) / threads, threads, 0, st>>>(
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
