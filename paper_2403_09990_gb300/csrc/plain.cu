// Plain per-instance walk samplers: Alg. 3 (dS_R) and Alg. 5 (dS_t) in the paper's own
// parallel form, one kernel per tensor operation of the listing and every intermediate
// tensor in device memory, one PURSE per call.  This is the comparator of the fused walk
// kernel (walk.cu): it draws the same perturbations (the same Philox streams), keeps the
// same decisions (top_k_indices with ties to the lower j; m0 = the smallest feasible rung,
// k0 = the best-ranked feasible k) and writes the same decision trace, but materialises
// per iteration
//   poses  (W, N_P, 12)         R_j, t_j of the perturbed poses      (perturbation)
//   d      (W, N_P)             dist(R_j, t_j, dS), eq. 11            (dist)
//   J      (W, N_P*)            top_k_indices(d, N_P*)                (top_k)
//   cand   (W, N_T, N_P*, 12)   the ladder candidates                 (update_rotation / _translation)
//   I      (W, N_T, N_P*)       in_purse of every candidate           (in_purse)
// and find_farthest updates (R*, t*).  Every constraint of every pose is evaluated (no
// early exit), as in the tensor formulation.  The walk state (q*, t*) lives in the
// caller's output buffers; walks are processed in chunks that bound the intermediates.
#include <cfloat>

#include "dev.cuh"
#include "internal.h"

namespace purse {

constexpr int kPlainThreads = 256;

template <typename T>
__device__ __forceinline__ T ladder_scale(double gamma, int m) {
  T s = T(1);
  for (int k = 0; k < m; ++k) s *= T(gamma);
  return s;
}

// Start pose (walk w from seed w mod s0) and velocity: omega = omega0 (u + u~) (Alg. 3),
// v = v0 S (dir + v~) (Alg. 5); u~, v~ are the first accepted unit lattice draws of the
// walk's velocity stream.
template <typename T>
__global__ void __launch_bounds__(kPlainThreads)
    plain_init_kernel(const double* __restrict__ seed_data, int s0, const WalkStats* __restrict__ st, int w0, int nw,
                      int sampler, double omega0, double v0, uint32_t key0, uint32_t key1, T* q, T* t, T* vel) {
  const int lw = blockIdx.x * blockDim.x + threadIdx.x;
  if (lw >= nw) return;
  const int w = w0 + lw;
  const double* sd = seed_data + (size_t)(w % s0) * kSeedStride;
  Stream s(key0, key1, sampler == 0 ? kPhaseOmega : kPhaseV, 0u, 0u, (uint32_t)w);
  int X, Y, Z;
  lattice_draw<true>(s, X, Y, Z);
  const double nr = sqrt((double)(X * X + Y * Y + Z * Z));
  const double ux = nr > 0 ? X / nr : 0.0, uy = nr > 0 ? Y / nr : 0.0, uz = nr > 0 ? Z / nr : 0.0;
  T* v = vel + 3 * (size_t)lw;
  if (sampler == 0) {
    v[0] = T(omega0 * (sd[7] + ux)), v[1] = T(omega0 * (sd[8] + uy)), v[2] = T(omega0 * (sd[9] + uz));
  } else {
    const double d0 = sd[10] + ux, d1 = sd[11] + uy, d2 = sd[12] + uz;
    v[0] = T(v0 * (st->S[0] * d0 + st->S[1] * d1 + st->S[2] * d2));
    v[1] = T(v0 * (st->S[3] * d0 + st->S[4] * d1 + st->S[5] * d2));
    v[2] = T(v0 * (st->S[6] * d0 + st->S[7] * d1 + st->S[8] * d2));
  }
  T* qo = q + 4 * (size_t)w;
  T* to = t + 3 * (size_t)w;
  qo[0] = T(sd[0]), qo[1] = T(sd[1]), qo[2] = T(sd[2]), qo[3] = T(sd[3]);
  to[0] = T(sd[4]), to[1] = T(sd[5]), to[2] = T(sd[6]);
}

__device__ __forceinline__ void store_pose(float* p, const M3<float>& R, const V3<float>& t) {
  float4* p4 = reinterpret_cast<float4*>(p);  // 48-byte records: 16-byte aligned
  p4[0] = make_float4(R.m[0], R.m[1], R.m[2], R.m[3]);
  p4[1] = make_float4(R.m[4], R.m[5], R.m[6], R.m[7]);
  p4[2] = make_float4(R.m[8], t.x, t.y, t.z);
}
__device__ __forceinline__ void store_pose(double* p, const M3<double>& R, const V3<double>& t) {
  for (int k = 0; k < 9; ++k) p[k] = R.m[k];
  p[9] = t.x, p[10] = t.y, p[11] = t.z;
}
template <typename T>
__device__ __forceinline__ void load_pose(const T* p, M3<T>& R, V3<T>& t) {
  if constexpr (sizeof(T) == 4) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
    const float4 a = p4[0], b = p4[1], c = p4[2];
    R = M3<T>{{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x}};
    t = V3<T>{c.y, c.z, c.w};
  } else {
    for (int k = 0; k < 9; ++k) R.m[k] = p[k];
    t = V3<T>{p[9], p[10], p[11]};
  }
}

// perturbation: pair b of walk w gives perturbations j = 2b, 2b + 1 (the two points of block 0
// of stream (phase, b, i, w)).  dS_R: (R*, t* + delta_j); dS_t: (R_p,j R*, t*), and the unit
// quaternion of R_p,j R* (the state update of Alg. 5 takes it).
template <typename T, int SAMPLER>
__global__ void __launch_bounds__(kPlainThreads)
    plain_perturb_kernel(int w0, int nw, int NP, int it, uint32_t key0, uint32_t key1,
                         const WalkStats* __restrict__ st, const T* __restrict__ q, const T* __restrict__ t, T* pose,
                         T* pq) {
  const int npairs = (NP + 1) / 2;
  const T r_pert = T(SAMPLER == 0 ? st->r_trans : st->r_rot);
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)nw * npairs) return;
  const int lw = (int)(idx / npairs), b = (int)(idx - (long)lw * npairs);
  const int w = w0 + lw;
  const uint4 wd = philox4x32_10(
      make_uint4(0u, ((SAMPLER == 0 ? kPhaseRPerturb : kPhaseTPerturb) << 24) | (uint32_t)b, (uint32_t)it, (uint32_t)w),
      key0, key1);
  const T* qs = q + 4 * (size_t)w;
  const T* ts = t + 3 * (size_t)w;
  const Q4<T> qw{qs[0], qs[1], qs[2], qs[3]};
  const V3<T> tw{ts[0], ts[1], ts[2]};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = 2 * b + h;
    if (j >= NP) break;
    T ux, uy, uz;
    hatbox_point<T>(h ? wd.z : wd.x, h ? wd.w : wd.y, ux, uy, uz);
    const V3<T> dl{r_pert * ux, r_pert * uy, r_pert * uz};
    T* out = pose + 12 * ((size_t)lw * NP + j);
    if (SAMPLER == 0) {
      store_pose(out, qmat(qw), V3<T>{tw.x + dl.x, tw.y + dl.y, tw.z + dl.z});
    } else {
      const Q4<T> qn = qnormalize(qmul(qexp(dl), qw));
      store_pose(out, qmat(qn), tw);
      T* o = pq + 4 * ((size_t)lw * NP + j);
      o[0] = qn.w, o[1] = qn.x, o[2] = qn.y, o[3] = qn.z;
    }
  }
}

// Constraint table into shared memory: 3D-3D / 2D-3D rows (a_i or Z_i, r_i), then (b_i or (u_i, v_i, 0),
// r_i^2), 8 N values; pose regression rows (t_i, beta_i^t), then the rows of R_i with beta_i^R in the first,
// 16 N values.
template <typename T, int KIND>
__device__ __forceinline__ void stage_table(const T* __restrict__ tab, int N, T* s) {
  const int count = (KIND == 2 ? 16 : 8) * N;
  for (int k = threadIdx.x; k < count; k += blockDim.x) s[k] = tab[k];
  __syncthreads();
}

// Pose regression (Example 3): the two margins of hypothesis i, beta_i^R - |R - R_i|_F and
// beta_i^t - |t - t_i|, and whether both constraints hold.
template <typename T>
__device__ __forceinline__ void reg_margins(const T* s, int N, int i, const M3<T>& R, const V3<T>& t, T& mR, T& mt,
                                            bool& ok) {
  const T* ti = s + 4 * i;
  const T ex = t.x - ti[0], ey = t.y - ti[1], ez = t.z - ti[2];
  const T e2 = ex * ex + ey * ey + ez * ez;
  T d2 = T(0);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const T* row = s + 4 * ((1 + r) * N + i);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T d = R.m[3 * r + c] - row[c];
      d2 += d * d;
    }
  }
  const T bR = s[4 * (N + i) + 3];
  mR = bR - sqrt(d2);
  mt = ti[3] - sqrt(e2);
  ok = d2 <= bR * bR && e2 <= ti[3] * ti[3];
}

// |U e|^2 for the noise norm of eq. 4 (Lambda = U^T U, U upper triangular, 8 values per constraint:
// 3D-3D u00 u01 u02 u11 u12 u22, 2D-3D u00 u01 u11).
template <typename T>
__device__ __forceinline__ T lam_norm2_3(const T* u, T e0, T e1, T e2) {
  const T a = u[0] * e0 + u[1] * e1 + u[2] * e2, b = u[3] * e1 + u[4] * e2, c = u[5] * e2;
  return a * a + b * b + c * c;
}
template <typename T>
__device__ __forceinline__ T lam_norm2_2(const T* u, T e0, T e1) {
  const T a = u[0] * e0 + u[1] * e1, b = u[2] * e1;
  return a * a + b * b;
}

// Noise factors (8 N values) after the constraint table in shared memory, or NULL.
template <typename T, int KIND>
__device__ __forceinline__ const T* stage_noise(const T* __restrict__ ell, int N, T* s) {
  if (KIND == 2 || ell == nullptr) return nullptr;
  T* u = s + 8 * N;
  for (int k = threadIdx.x; k < 8 * N; k += blockDim.x) u[k] = ell[k];
  __syncthreads();
  return u;
}

// dist(R, t, dS) of eq. 11: min_i (r_i - |g_i|), -inf when a 2D-3D keypoint is behind the camera;
// |g_i| in the norm of eq. 4 when the PURSE carries noise matrices (ell != NULL).
template <typename T, int KIND>
__global__ void __launch_bounds__(kPlainThreads)
    plain_dist_kernel(const T* __restrict__ tab, const T* __restrict__ ell, int N, T fx, T fy, T cx, T cy,
                      const T* __restrict__ pose, long n, T* d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  stage_table<T, KIND>(tab, N, s);
  const T* u = stage_noise<T, KIND>(ell, N, s);
  const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  M3<T> R;
  V3<T> t;
  load_pose(pose + 12 * p, R, t);
  T best = T(INFINITY);
  if (KIND == 2) {
    for (int i = 0; i < N; ++i) {
      T mR, mt;
      bool ok;
      reg_margins<T>(s, N, i, R, t, mR, mt, ok);
      best = fmin(best, fmin(mR, mt));
    }
    d[p] = best;
    return;
  }
  for (int i = 0; i < N; ++i) {
    const T* a = s + 4 * i;
    const T* o = s + 4 * (N + i);
    const V3<T> X = mul(R, V3<T>{a[0], a[1], a[2]}) + t;
    T m;
    if (KIND == 0) {
      const T ex = X.x - o[0], ey = X.y - o[1], ez = X.z - o[2];
      m = a[3] - sqrt(u ? lam_norm2_3(u + 8 * i, ex, ey, ez) : ex * ex + ey * ey + ez * ez);
    } else if (X.z > T(0)) {
      const T gu = o[0] - (fx * X.x + cx * X.z) / X.z, gv = o[1] - (fy * X.y + cy * X.z) / X.z;
      m = a[3] - sqrt(u ? lam_norm2_2(u + 8 * i, gu, gv) : gu * gu + gv * gv);
    } else {
      m = -T(INFINITY);
    }
    best = fmin(best, m);
  }
  d[p] = best;
}

// top_k_indices(d, N_P*), one warp per walk: lane l holds j = l + 32 s; N_P* rounds of a warp
// arg-max over (d_j, -j), so ties go to the lower j.
template <typename T>
__global__ void __launch_bounds__(kPlainThreads)
    plain_topk_kernel(const T* __restrict__ d, int w0, int nw, int NP, int K, int32_t* J, int16_t* trace, int n_iter,
                      int it) {
  const int lw = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (lw >= nw) return;  // warp-uniform
  T v[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int j = lane + 32 * s;
    v[s] = j < NP ? d[(size_t)lw * NP + j] : -T(INFINITY);
  }
  unsigned taken = 0;  // bit s: slot s already ranked
  const size_t w = (size_t)(w0 + lw);
  for (int r = 0; r < K; ++r) {
    T bv = -T(INFINITY);
    int bj = 1 << 30;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int j = lane + 32 * s;
      if (j < NP && !((taken >> s) & 1u) && (v[s] > bv || bj == (1 << 30))) bv = v[s], bj = j;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const T ov = __shfl_xor_sync(kFullMask, bv, o);
      const int oj = __shfl_xor_sync(kFullMask, bj, o);
      if (oj != (1 << 30) && (bj == (1 << 30) || ov > bv || (ov == bv && oj < bj))) bv = ov, bj = oj;
    }
    if ((bj & 31) == lane) taken |= 1u << (bj >> 5);
    if (lane == 0) {
      J[(size_t)lw * K + r] = bj;
      if (trace) trace[(w * n_iter + it) * (K + 2) + r] = (int16_t)bj;
    }
  }
}

// Ladder candidates (k, m), Delta T = gamma^m (m from 0): dS_R (update_rotation):
// (Exp(Delta T omega) R*, t_{j_k}); dS_t (update_translation): (R_{j_k}, t* + Delta T v).
template <typename T, int SAMPLER>
__global__ void __launch_bounds__(kPlainThreads)
    plain_ladder_kernel(int w0, int nw, int NP, int K, int NT, double gamma, const T* __restrict__ q,
                        const T* __restrict__ t, const T* __restrict__ vel, const int32_t* __restrict__ J,
                        const T* __restrict__ pose, T* cand) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)nw * NT * K) return;
  const int lw = (int)(idx / (NT * K)), rem = (int)(idx - (long)lw * NT * K);
  const int m = rem / K, k = rem - m * K;
  const size_t w = (size_t)(w0 + lw);
  const T sm = ladder_scale<T>(gamma, m);
  const T* v = vel + 3 * (size_t)lw;
  const int jk = J[(size_t)lw * K + k];
  M3<T> Rj;
  V3<T> tj;
  load_pose(pose + 12 * ((size_t)lw * NP + jk), Rj, tj);
  T* out = cand + 12 * (size_t)idx;
  if (SAMPLER == 0) {
    const Q4<T> e = qexp(V3<T>{sm * v[0], sm * v[1], sm * v[2]});
    const T* qs = q + 4 * w;
    store_pose(out, qmat(qnormalize(qmul(Q4<T>{e.w, e.x, e.y, e.z}, Q4<T>{qs[0], qs[1], qs[2], qs[3]}))), tj);
  } else {
    const T* ts = t + 3 * w;
    store_pose(out, Rj, V3<T>{ts[0] + sm * v[0], ts[1] + sm * v[1], ts[2] + sm * v[2]});
  }
}

// in_purse of every candidate: all_i |g_i| <= r_i (2D-3D also P_z > 0), eq. 2/3/5.
template <typename T, int KIND>
__global__ void __launch_bounds__(kPlainThreads)
    plain_in_purse_kernel(const T* __restrict__ tab, const T* __restrict__ ell, int N, T fx, T fy, T cx, T cy,
                          const T* __restrict__ cand, long n, uint8_t* I) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  stage_table<T, KIND>(tab, N, s);
  const T* u = stage_noise<T, KIND>(ell, N, s);
  const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  M3<T> R;
  V3<T> t;
  load_pose(cand + 12 * p, R, t);
  bool ok = true;
  if (KIND == 2) {
    for (int i = 0; i < N; ++i) {
      T mR, mt;
      bool oki;
      reg_margins<T>(s, N, i, R, t, mR, mt, oki);
      ok = ok && oki;
    }
    I[p] = ok ? 1 : 0;
    return;
  }
  for (int i = 0; i < N; ++i) {
    const T* a = s + 4 * i;
    const T* o = s + 4 * (N + i);
    const V3<T> X = mul(R, V3<T>{a[0], a[1], a[2]}) + t;
    if (KIND == 0) {
      const T ex = X.x - o[0], ey = X.y - o[1], ez = X.z - o[2];
      ok = ok && (u ? lam_norm2_3(u + 8 * i, ex, ey, ez) : ex * ex + ey * ey + ez * ez) <= o[3];
    } else {
      const bool front = X.z > T(0);
      const T Pz = front ? X.z : T(1);
      const T gu = o[0] - (fx * X.x + cx * X.z) / Pz, gv = o[1] - (fy * X.y + cy * X.z) / Pz;
      ok = ok && front && (u ? lam_norm2_2(u + 8 * i, gu, gv) : gu * gu + gv * gv) <= o[3];
    }
  }
  I[p] = ok ? 1 : 0;
}

// find_farthest + the state update: m0 = the smallest m with a feasible k, k0 = the best-ranked
// feasible k there; (R*, t*) <- candidate (k0, m0); unchanged when nothing is feasible.
template <typename T, int SAMPLER>
__global__ void __launch_bounds__(kPlainThreads)
    plain_select_kernel(int w0, int nw, int NP, int K, int NT, double gamma, const uint8_t* __restrict__ I,
                        const int32_t* __restrict__ J, const T* __restrict__ pose, const T* __restrict__ pq,
                        const T* __restrict__ vel, T* q, T* t, int16_t* trace, int n_iter, int it) {
  const int lw = blockIdx.x * blockDim.x + threadIdx.x;
  if (lw >= nw) return;
  const size_t w = (size_t)(w0 + lw);
  int m0 = -1, k0 = -1;
  const uint8_t* Iw = I + (size_t)lw * NT * K;
  for (int m = 0; m < NT && m0 < 0; ++m)
    for (int k = 0; k < K; ++k)
      if (Iw[m * K + k]) {
        m0 = m, k0 = k;
        break;
      }
  if (m0 >= 0) {
    const int jk = J[(size_t)lw * K + k0];
    const T sm = ladder_scale<T>(gamma, m0);
    const T* v = vel + 3 * (size_t)lw;
    T* qs = q + 4 * w;
    T* ts = t + 3 * w;
    if (SAMPLER == 0) {
      const Q4<T> e = qexp(V3<T>{sm * v[0], sm * v[1], sm * v[2]});
      const Q4<T> qn = qnormalize(qmul(Q4<T>{e.w, e.x, e.y, e.z}, Q4<T>{qs[0], qs[1], qs[2], qs[3]}));
      M3<T> R;
      V3<T> tj;
      load_pose(pose + 12 * ((size_t)lw * NP + jk), R, tj);
      qs[0] = qn.w, qs[1] = qn.x, qs[2] = qn.y, qs[3] = qn.z;
      ts[0] = tj.x, ts[1] = tj.y, ts[2] = tj.z;
    } else {
      const T* p = pq + 4 * ((size_t)lw * NP + jk);
      qs[0] = p[0], qs[1] = p[1], qs[2] = p[2], qs[3] = p[3];
      ts[0] = ts[0] + sm * v[0], ts[1] = ts[1] + sm * v[1], ts[2] = ts[2] + sm * v[2];
    }
  }
  if (trace) {
    int16_t* tr = trace + (w * n_iter + it) * (K + 2);
    tr[K] = (int16_t)m0;
    tr[K + 1] = (int16_t)k0;
  }
}

__global__ void plain_count_kernel(unsigned long long* evals, unsigned long long n) { *evals = n; }

// Bytes of the intermediates per walk of a chunk.
template <typename T>
static size_t plain_bytes_per_walk(int NP, int K, int NT, int sampler) {
  return sizeof(T) * (12 * (size_t)NP + (sampler ? 4 * (size_t)NP : 0) + NP + 12 * (size_t)NT * K + 3) +
         sizeof(int32_t) * K + (size_t)NT * K + 64;
}

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

static unsigned blocks_for(long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <typename T, int KIND, int SAMPLER>
static cudaError_t run_plain_t(purse_t h, const purse_params* p, const WalkStats* d_stats, const double* d_seed_data,
                               int s0, uint64_t seed, int n_samples, T* q, T* t, int16_t* trace, void* scratch,
                               size_t scratch_bytes, int chunk, cudaStream_t st) {
  const int NP = p->n_perturb, K = p->n_keep, NT = p->n_steps, N = h->n;
  const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
  const T* tab = sizeof(T) == 4 ? (const T*)h->tables.f32 : (const T*)h->tables.f64;
  const T fx = T(h->K.fx), fy = T(h->K.fy), cx = T(h->K.cx), cy = T(h->K.cy);
  const T* ell = sizeof(T) == 4 ? (const T*)h->ell32 : (const T*)h->ell64;
  const size_t tab_smem = ((KIND == 2 ? 16 : 8) + (ell ? 8 : 0)) * (size_t)N * sizeof(T);
  cudaError_t e = cudaSuccess;
  char* base = reinterpret_cast<char*>(scratch);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* ptr = base + off;
    off += a256(bytes);
    return ptr;
  };
  T* pose = reinterpret_cast<T*>(take(sizeof(T) * 12 * (size_t)chunk * NP));
  T* pq = SAMPLER ? reinterpret_cast<T*>(take(sizeof(T) * 4 * (size_t)chunk * NP)) : nullptr;
  T* d = reinterpret_cast<T*>(take(sizeof(T) * (size_t)chunk * NP));
  int32_t* J = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (size_t)chunk * K));
  T* cand = reinterpret_cast<T*>(take(sizeof(T) * 12 * (size_t)chunk * NT * K));
  uint8_t* I = reinterpret_cast<uint8_t*>(take((size_t)chunk * NT * K));
  T* vel = reinterpret_cast<T*>(take(sizeof(T) * 3 * (size_t)chunk));
  if (off > scratch_bytes) return cudaErrorInvalidValue;
  const int TH = kPlainThreads;
  for (int w0 = 0; w0 < n_samples && e == cudaSuccess; w0 += chunk) {
    const int nw = n_samples - w0 < chunk ? n_samples - w0 : chunk;
    plain_init_kernel<T><<<blocks_for(nw, TH), TH, 0, st>>>(d_seed_data, s0, d_stats, w0, nw, SAMPLER, p->omega0,
                                                            p->v0, key0, key1, q, t, vel);
    for (int it = 0; it < p->n_iter; ++it) {
      const long npose = (long)nw * NP, ncand = (long)nw * NT * K;
      plain_perturb_kernel<T, SAMPLER><<<blocks_for((long)nw * ((NP + 1) / 2), TH), TH, 0, st>>>(
          w0, nw, NP, it, key0, key1, d_stats, q, t, pose, pq);
      plain_dist_kernel<T, KIND><<<blocks_for(npose, TH), TH, tab_smem, st>>>(tab, ell, N, fx, fy, cx, cy, pose,
                                                                              npose, d);
      plain_topk_kernel<T><<<blocks_for(32L * nw, TH), TH, 0, st>>>(d, w0, nw, NP, K, J, trace, p->n_iter, it);
      plain_ladder_kernel<T, SAMPLER><<<blocks_for(ncand, TH), TH, 0, st>>>(w0, nw, NP, K, NT, p->gamma, q, t, vel,
                                                                            J, pose, cand);
      plain_in_purse_kernel<T, KIND><<<blocks_for(ncand, TH), TH, tab_smem, st>>>(tab, ell, N, fx, fy, cx, cy, cand,
                                                                                  ncand, I);
      plain_select_kernel<T, SAMPLER><<<blocks_for(nw, TH), TH, 0, st>>>(w0, nw, NP, K, NT, p->gamma, I, J, pose, pq,
                                                                         vel, q, t, trace, p->n_iter, it);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const unsigned long long n_evals = (unsigned long long)n_samples * p->n_iter *
                                       ((unsigned long long)NP + (unsigned long long)NT * K) * (KIND == 2 ? 2 * N : N);
    plain_count_kernel<<<1, 1, 0, st>>>(h->d_evals, n_evals);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_plain_dist(purse_t h, const float* d_poses, long n_poses, float* d_dist, cudaStream_t st) {
  if (n_poses == 0) return cudaSuccess;
  const float* ell = h->kind == 2 ? nullptr : h->ell32;
  const size_t tab_smem = ((h->kind == 2 ? 16 : 8) + (ell ? 8 : 0)) * (size_t)h->n * sizeof(float);
  const float fx = float(h->K.fx), fy = float(h->K.fy), cx = float(h->K.cx), cy = float(h->K.cy);
  const unsigned grid = blocks_for(n_poses, kPlainThreads);
  if (h->kind == 0)
    plain_dist_kernel<float, 0><<<grid, kPlainThreads, tab_smem, st>>>(h->tables.f32, ell, h->n, fx, fy, cx, cy,
                                                                        d_poses, n_poses, d_dist);
  else if (h->kind == 2)
    plain_dist_kernel<float, 2><<<grid, kPlainThreads, tab_smem, st>>>(h->tables.f32, nullptr, h->n, fx, fy, cx, cy,
                                                                        d_poses, n_poses, d_dist);
  else
    plain_dist_kernel<float, 1><<<grid, kPlainThreads, tab_smem, st>>>(h->tables.f32, ell, h->n, fx, fy, cx, cy,
                                                                        d_poses, n_poses, d_dist);
  return cudaGetLastError();
}

size_t plain_scratch_bytes(const purse_params* p, int n_samples, int* chunk) {
  const size_t per = p->precision == 1 ? plain_bytes_per_walk<double>(p->n_perturb, p->n_keep, p->n_steps, p->sampler)
                                       : plain_bytes_per_walk<float>(p->n_perturb, p->n_keep, p->n_steps, p->sampler);
  // intermediates of one chunk bounded by about 2 GB
  long c = (long)((size_t)2 << 30) / (long)per;
  if (c < 1024) c = 1024;
  if (c > n_samples) c = n_samples < 1 ? 1 : n_samples;
  *chunk = (int)c;
  return per * (size_t)c + 16 * 256;
}

cudaError_t launch_plain(purse_t h, const purse_params* p, const WalkStats* d_stats, const double* d_seed_data, int s0,
                         uint64_t seed, int n_samples, void* d_q, void* d_t, int16_t* d_trace, void* scratch,
                         size_t scratch_bytes, int chunk, cudaStream_t st) {
  const int kind = h->kind, smp = p->sampler;
#define PLAIN_RUN(T, KD, SM)                                                                                    \
  return run_plain_t<T, KD, SM>(h, p, d_stats, d_seed_data, s0, seed, n_samples, (T*)d_q, (T*)d_t, d_trace, \
                                scratch, scratch_bytes, chunk, st)
  if (p->precision == 0) {
    if (kind == 0) {
      if (smp == 0) PLAIN_RUN(float, 0, 0);
      PLAIN_RUN(float, 0, 1);
    }
    if (kind == 2) {
      if (smp == 0) PLAIN_RUN(float, 2, 0);
      PLAIN_RUN(float, 2, 1);
    }
    if (smp == 0) PLAIN_RUN(float, 1, 0);
    PLAIN_RUN(float, 1, 1);
  }
  if (kind == 0) {
    if (smp == 0) PLAIN_RUN(double, 0, 0);
    PLAIN_RUN(double, 0, 1);
  }
  if (kind == 2) {
    if (smp == 0) PLAIN_RUN(double, 2, 0);
    PLAIN_RUN(double, 2, 1);
  }
  if (smp == 0) PLAIN_RUN(double, 1, 0);
  PLAIN_RUN(double, 1, 1);
#undef PLAIN_RUN
}

}  // namespace purse
