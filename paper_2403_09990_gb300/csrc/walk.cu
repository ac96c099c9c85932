// Fused strategic random walk (Section IV Step II; Alg. 2/3 for the dS_R
// sampler, Alg. 4/5 for the dS_t sampler), one warp per walk.
//
// Per iteration of a walk:
//   1. tables: Y_i = R* Z_i (and the per-constraint constants of the
//      perturbation phase) into the warp's shared-memory slab;
//   2. perturbation + dist (eq. 11): lane l draws perturbations
//      j = l + 32 s from Philox and evaluates d_j = min_i (r_i - |g_i|);
//   3. top_k_indices: N_P* rounds of warp max (REDUX) over order-preserving
//      keys, ties to the lower j;
//   4. step ladder: candidates (k, m) are laid out lane = m_local * N_P* + k
//      over chunks of 32 / N_P* ladder rungs; in_purse is evaluated
//      division-free; the first chunk with a feasible candidate ends the
//      ladder, and __ffs of the ballot gives m0 (smallest m) then k0
//      (best-ranked k), i.e. find_farthest;
//   5. update (R*, t*).
// Factoring used on the hot loop (same values as the paper's per-pose
// transform, fewer operations):
//   dS_R, 2D-3D: K(R* Z_i + t* + delta_j) = Q_i + K delta_j,
//                K(E_m R* Z_i + t_jk)     = W_mi + K t_jk
//   dS_t, 2D-3D: K(R_p R* Z_i + t*)       = (K R_p) Y_i + K t*
// and the same without K (minus b_i) for 3D-3D.
#include <cfloat>
#include <cstdio>

#include "dev.cuh"
#include "internal.h"

namespace purse {

constexpr int kWalkWarps = 8;
constexpr int kWalkThreads = kWalkWarps * 32;
constexpr int kPertGroup = 4;  // perturbations per lane per pass
constexpr int kPertPasses = 2; // N_P <= 32 * 4 * 2 = 256

template <typename T>
struct alignas(sizeof(T) * 4) T4 {
  T x, y, z, w;
};

template <typename T>
struct KeyOf;
template <>
struct KeyOf<float> {
  using type = uint32_t;
};
template <>
struct KeyOf<double> {
  using type = unsigned long long;
};

__device__ __forceinline__ uint32_t warp_max_key(uint32_t k) { return __reduce_max_sync(kFullMask, k); }
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long k) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(kFullMask, k, o);
    k = v > k ? v : k;
  }
  return k;
}

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
template <typename T>
__device__ __forceinline__ T tiny();
template <>
__device__ __forceinline__ float tiny<float>() {
  return 1e-30f;
}
template <>
__device__ __forceinline__ double tiny<double>() {
  return 1e-300;
}
template <typename T>
__device__ __forceinline__ T inf() {
  return T(INFINITY);
}

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bytes of one warp's slab (must match the carving in the kernel).
template <typename T>
__host__ __device__ inline size_t walk_slab_bytes(int n, int n_perturb, int n_steps, int mc, int sampler) {
  const size_t t4 = 4 * sizeof(T);
  const size_t entries = 2 * (size_t)n + (sampler == 0 ? (size_t)mc * n : 0) + n_perturb + 4 * (size_t)n_steps;
  return align_up(entries * t4 + 32 * sizeof(int), 128);
}

template <typename T>
__host__ __device__ inline size_t walk_table_bytes(int n) {
  return align_up(8 * (size_t)n * sizeof(T), 128);
}

// Margin r - |g| of one 2D-3D constraint at P = K X (pixels), -inf behind the camera.
template <typename T>
__device__ __forceinline__ T margin2d(T Px, T Py, T Pz, T u, T v, T r) {
  const T ex = Px - u * Pz;
  const T ey = Py - v * Pz;
  const T s2 = ex * ex + ey * ey;
  const T q = fmax(s2 * (Pz * Pz), tiny<T>());
  const T m = r - s2 * rsq(q);  // |e| / Pz
  return Pz > T(0) ? m : -inf<T>();
}

template <typename T>
__device__ __forceinline__ T margin3d(T ex, T ey, T ez, T r) {
  const T s2 = ex * ex + ey * ey + ez * ez;
  return r - s2 * rsq(fmax(s2, tiny<T>()));
}

template <typename T, int KIND, int SAMPLER>
__global__ void __launch_bounds__(kWalkThreads) walk_kernel(const WalkArgs a, const int mc, const int slab_bytes) {
  using Key = typename KeyOf<T>::type;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  const int N = a.n;
  const int NP = a.n_perturb, K = a.n_keep, NT = a.n_steps;
  const T4<T>* tab = reinterpret_cast<const T4<T>*>(smem + 128);  // rows [0,N): (a,r); [N,2N): (b or z, r^2)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* slab = smem + 128 + walk_table_bytes<T>(N) + (size_t)warp * slab_bytes;
  T4<T>* Ytab = reinterpret_cast<T4<T>*>(slab);
  T4<T>* Qtab = Ytab + N;
  T4<T>* Wtab = Qtab + N;
  T4<T>* Ptab = Wtab + (SAMPLER == 0 ? mc * N : 0);
  T4<T>* Etab = Ptab + NP;
  int* Jtab = reinterpret_cast<int*>(Etab + 4 * NT);

  // ---- a0: stage the constraint table with a 1-D TMA bulk copy.
  const uint32_t tbytes = 8u * N * sizeof(T);
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, tbytes);
    bulk_copy_g2s(smem + 128, a.table, tbytes, bar);
  }
  if (!mbar_wait_bounded(bar, 0, 1 << 22)) {
    if (threadIdx.x == 0) atomicOr(a.status, kDevErrTimeout);
    return;
  }

  const T fx = T(a.fx), fy = T(a.fy), cx = T(a.cx), cy = T(a.cy);
  const WalkStats* st = a.stats;
  const T r_pert = T((SAMPLER == 0 ? st->r_trans : st->r_rot) / 1024.0);
  const int ncand = mc * K;
  const int cm = lane / K, ck = lane - (lane / K) * K;
  unsigned long long evals = 0;

  for (int w = blockIdx.x * kWalkWarps + warp; w < a.n_samples; w += gridDim.x * kWalkWarps) {
    // ---- a3: start pose and velocity (FP64), ladder table.
    const double* sd = a.seed_data + (size_t)(w % a.s0) * kSeedStride;
    Q4<T> q{T(sd[0]), T(sd[1]), T(sd[2]), T(sd[3])};
    V3<T> t{T(sd[4]), T(sd[5]), T(sd[6])};
    double vel[3];
    {
      Stream s(a.key0, a.key1, SAMPLER == 0 ? kPhaseOmega : kPhaseV, 0u, 0u, (uint32_t)w);
      int X, Y, Z;
      lattice_draw<true>(s, X, Y, Z);
      const double nr = sqrt((double)(X * X + Y * Y + Z * Z));
      const double ut[3] = {nr > 0 ? X / nr : 0.0, nr > 0 ? Y / nr : 0.0, nr > 0 ? Z / nr : 0.0};
      if (SAMPLER == 0) {
        for (int c = 0; c < 3; ++c) vel[c] = a.omega0 * (sd[7 + c] + ut[c]);
      } else {
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = sd[10 + c] + ut[c];
        for (int r = 0; r < 3; ++r)
          vel[r] = a.v0 * (st->S[3 * r] * d[0] + st->S[3 * r + 1] * d[1] + st->S[3 * r + 2] * d[2]);
      }
    }
    for (int m = lane; m < NT; m += 32) {
      const double sm = pow(a.gamma, (double)m);
      if (SAMPLER == 0) {
        const Q4<double> e = qexp(V3<double>{sm * vel[0], sm * vel[1], sm * vel[2]});
        const M3<double> E = qmat(e);
        Etab[4 * m] = T4<T>{T(e.w), T(e.x), T(e.y), T(e.z)};
        for (int r = 0; r < 3; ++r) Etab[4 * m + 1 + r] = T4<T>{T(E.m[3 * r]), T(E.m[3 * r + 1]), T(E.m[3 * r + 2]), T(0)};
      } else {
        Etab[4 * m] = T4<T>{T(sm * vel[0]), T(sm * vel[1]), T(sm * vel[2]), T(0)};
      }
    }
    __syncwarp();

    for (int it = 0; it < a.n_iter; ++it) {
      const M3<T> R = qmat(q);
      // ---- tables for this iteration
      for (int i = lane; i < N; i += 32) {
        const T4<T> mz = tab[i], ob = tab[N + i];
        const V3<T> Y = mul(R, V3<T>{mz.x, mz.y, mz.z});
        Ytab[i] = T4<T>{Y.x, Y.y, Y.z, T(0)};
        if (SAMPLER == 0) {
          if (KIND == 1) {
            const V3<T> X = Y + t;
            Qtab[i] = T4<T>{fx * X.x + cx * X.z, fy * X.y + cy * X.z, X.z, T(0)};
          } else {
            Qtab[i] = T4<T>{Y.x + t.x - ob.x, Y.y + t.y - ob.y, Y.z + t.z - ob.z, T(0)};
          }
        } else if (KIND == 0) {
          Qtab[i] = T4<T>{t.x - ob.x, t.y - ob.y, t.z - ob.z, T(0)};
        }
      }
      __syncwarp();

      // ---- a4: perturbations and their distance to the boundary (eq. 11)
      Key key[kPertGroup * kPertPasses];
#pragma unroll
      for (int p = 0; p < kPertPasses; ++p) {
#pragma unroll
        for (int g = 0; g < kPertGroup; ++g) key[p * kPertGroup + g] = 0;
        if (p * 32 * kPertGroup >= NP) continue;
        T dmin[kPertGroup];
        bool valid[kPertGroup];
        // dS_R: D = translation offset in P units; dS_t: A = rotation (K R_p for 2D-3D)
        V3<T> D[kPertGroup];
        M3<T> A[SAMPLER == 1 ? kPertGroup : 1];
#pragma unroll
        for (int g = 0; g < kPertGroup; ++g) {
          const int j = p * 32 * kPertGroup + g * 32 + lane;
          valid[g] = j < NP;
          dmin[g] = inf<T>();
          D[g] = V3<T>{T(0), T(0), T(0)};
          if constexpr (SAMPLER == 1) A[g] = M3<T>{{T(1), T(0), T(0), T(0), T(1), T(0), T(0), T(0), T(1)}};
          if (valid[g]) {
            Stream s(a.key0, a.key1, SAMPLER == 0 ? kPhaseRPerturb : kPhaseTPerturb, (uint32_t)j, (uint32_t)it,
                     (uint32_t)w);
            int X, Y, Z;
            lattice_draw<false>(s, X, Y, Z);
            const V3<T> dl{r_pert * T(X), r_pert * T(Y), r_pert * T(Z)};
            if constexpr (SAMPLER == 0) {
              Ptab[j] = T4<T>{dl.x, dl.y, dl.z, T(0)};
              D[g] = KIND == 1 ? V3<T>{fx * dl.x + cx * dl.z, fy * dl.y + cy * dl.z, dl.z} : dl;
            } else {
              const Q4<T> pq = qexp(dl);
              Ptab[j] = T4<T>{pq.w, pq.x, pq.y, pq.z};
              M3<T> Rp = qmat(pq);
              if (KIND == 1) {
                for (int c = 0; c < 3; ++c) {
                  Rp.m[c] = fx * Rp.m[c] + cx * Rp.m[6 + c];
                  Rp.m[3 + c] = fy * Rp.m[3 + c] + cy * Rp.m[6 + c];
                }
              }
              A[g] = Rp;
            }
          }
        }
        V3<T> Kt{T(0), T(0), T(0)};
        if (SAMPLER == 1 && KIND == 1) Kt = V3<T>{fx * t.x + cx * t.z, fy * t.y + cy * t.z, t.z};
        for (int i = 0; i < N; ++i) {
          const T4<T> ob = tab[N + i];
          const T r = tab[i].w;
          if constexpr (SAMPLER == 0) {
            const T4<T> Qi = Qtab[i];
#pragma unroll
            for (int g = 0; g < kPertGroup; ++g) {
              const T Px = Qi.x + D[g].x, Py = Qi.y + D[g].y, Pz = Qi.z + D[g].z;
              const T m = KIND == 1 ? margin2d(Px, Py, Pz, ob.x, ob.y, r) : margin3d(Px, Py, Pz, r);
              dmin[g] = fmin(dmin[g], m);
            }
          } else {
            const T4<T> Yi = Ytab[i];
            const V3<T> c0 = KIND == 1 ? Kt : V3<T>{Qtab[i].x, Qtab[i].y, Qtab[i].z};
#pragma unroll
            for (int g = 0; g < kPertGroup; ++g) {
              const M3<T>& M = A[g];
              const T Px = M.m[0] * Yi.x + M.m[1] * Yi.y + M.m[2] * Yi.z + c0.x;
              const T Py = M.m[3] * Yi.x + M.m[4] * Yi.y + M.m[5] * Yi.z + c0.y;
              const T Pz = M.m[6] * Yi.x + M.m[7] * Yi.y + M.m[8] * Yi.z + c0.z;
              const T m = KIND == 1 ? margin2d(Px, Py, Pz, ob.x, ob.y, r) : margin3d(Px, Py, Pz, r);
              dmin[g] = fmin(dmin[g], m);
            }
          }
        }
#pragma unroll
        for (int g = 0; g < kPertGroup; ++g)
          key[p * kPertGroup + g] = valid[g] ? orderable(dmin[g]) : Key(0);
      }
      evals += (unsigned long long)NP * N;

      // ---- a5: top_k_indices (ties to the lower j)
      for (int r = 0; r < K; ++r) {
        Key bk = 0;
        int bs = -1;
#pragma unroll
        for (int s = 0; s < kPertGroup * kPertPasses; ++s)
          if (key[s] > bk) bk = key[s], bs = s;
        const Key wmax = warp_max_key(bk);
        const uint32_t myj = (bs >= 0 && bk == wmax) ? (uint32_t)(lane + 32 * bs) : 0xFFFFu;
        const uint32_t jmin = __reduce_min_sync(kFullMask, myj);
        if (myj == jmin) {
#pragma unroll
          for (int s = 0; s < kPertGroup * kPertPasses; ++s)
            if (s == bs) key[s] = 0;
        }
        if (lane == 0) Jtab[r] = (int)jmin;
      }
      __syncwarp();

      // ---- a6/a7: step ladder + in_purse, find_farthest
      int m0 = -1, k0 = -1;
      V3<T> base{T(0), T(0), T(0)};
      M3<T> Ak;
      if (lane < ncand) {
        const T4<T> pj = Ptab[Jtab[ck]];
        if (SAMPLER == 0) {
          const V3<T> tk{t.x + pj.x, t.y + pj.y, t.z + pj.z};
          base = KIND == 1 ? V3<T>{fx * tk.x + cx * tk.z, fy * tk.y + cy * tk.z, tk.z} : tk;
        } else {
          Ak = qmat(Q4<T>{pj.x, pj.y, pj.z, pj.w});
          if (KIND == 1) {
            for (int c = 0; c < 3; ++c) {
              Ak.m[c] = fx * Ak.m[c] + cx * Ak.m[6 + c];
              Ak.m[3 + c] = fy * Ak.m[3 + c] + cy * Ak.m[6 + c];
            }
          }
        }
      }
      for (int mb = 0; mb < NT; mb += mc) {
        if (SAMPLER == 0) {
          const int npair = mc * N;
          for (int pi = lane; pi < npair; pi += 32) {
            const int mi = pi / N, i = pi - mi * N, m = mb + mi;
            if (m < NT) {
              const T4<T> e0 = Etab[4 * m + 1], e1 = Etab[4 * m + 2], e2 = Etab[4 * m + 3];
              const T4<T> Yi = Ytab[i];
              const T X = e0.x * Yi.x + e0.y * Yi.y + e0.z * Yi.z;
              const T Y = e1.x * Yi.x + e1.y * Yi.y + e1.z * Yi.z;
              const T Z = e2.x * Yi.x + e2.y * Yi.y + e2.z * Yi.z;
              if (KIND == 1) {
                Wtab[pi] = T4<T>{fx * X + cx * Z, fy * Y + cy * Z, Z, T(0)};
              } else {
                const T4<T> ob = tab[N + i];
                Wtab[pi] = T4<T>{X - ob.x, Y - ob.y, Z - ob.z, T(0)};
              }
            }
          }
          __syncwarp();
        }
        const int m = mb + cm;
        bool feas = false;
        if (lane < ncand && m < NT) {
          T cmax = -inf<T>(), zmin = inf<T>();
          V3<T> bm = base;
          if (SAMPLER == 1) {
            const T4<T> sv = Etab[4 * m];
            const V3<T> Tm{t.x + sv.x, t.y + sv.y, t.z + sv.z};
            bm = KIND == 1 ? V3<T>{fx * Tm.x + cx * Tm.z, fy * Tm.y + cy * Tm.z, Tm.z} : Tm;
          }
          for (int i = 0; i < N; ++i) {
            const T4<T> ob = tab[N + i];
            T Px, Py, Pz;
            if (SAMPLER == 0) {
              const T4<T> Wi = Wtab[cm * N + i];
              Px = Wi.x + bm.x, Py = Wi.y + bm.y, Pz = Wi.z + bm.z;
            } else {
              const T4<T> Yi = Ytab[i];
              Px = Ak.m[0] * Yi.x + Ak.m[1] * Yi.y + Ak.m[2] * Yi.z + bm.x;
              Py = Ak.m[3] * Yi.x + Ak.m[4] * Yi.y + Ak.m[5] * Yi.z + bm.y;
              Pz = Ak.m[6] * Yi.x + Ak.m[7] * Yi.y + Ak.m[8] * Yi.z + bm.z;
              if (KIND == 0) Px -= ob.x, Py -= ob.y, Pz -= ob.z;
            }
            T c;
            if (KIND == 1) {
              const T ex = Px - ob.x * Pz, ey = Py - ob.y * Pz;
              const T rz = tab[i].w * Pz;
              c = ex * ex + ey * ey - rz * rz;
              zmin = fmin(zmin, Pz);
            } else {
              c = Px * Px + Py * Py + Pz * Pz - ob.w;
            }
            cmax = fmax(cmax, c);
          }
          feas = cmax <= T(0) && (KIND == 0 || zmin > T(0));
        }
        const unsigned bal = __ballot_sync(kFullMask, feas);
        evals += (unsigned long long)N * K * (unsigned long long)min(mc, NT - mb);
        __syncwarp();
        if (bal) {
          const int l = __ffs(bal) - 1;
          m0 = mb + l / K;
          k0 = l - (l / K) * K;
          break;
        }
      }

      // ---- update (R*, t*)
      if (m0 >= 0) {
        const T4<T> pj = Ptab[Jtab[k0]];
        if (SAMPLER == 0) {
          const T4<T> e = Etab[4 * m0];
          q = qnormalize(qmul(Q4<T>{e.x, e.y, e.z, e.w}, q));
          t = V3<T>{t.x + pj.x, t.y + pj.y, t.z + pj.z};
        } else {
          q = qnormalize(qmul(Q4<T>{pj.x, pj.y, pj.z, pj.w}, q));
          const T4<T> sv = Etab[4 * m0];
          t = V3<T>{t.x + sv.x, t.y + sv.y, t.z + sv.z};
        }
      }
      if (a.trace != nullptr && lane == 0) {
        int16_t* tr = a.trace + ((size_t)w * a.n_iter + it) * (K + 2);
        for (int r = 0; r < K; ++r) tr[r] = (int16_t)Jtab[r];
        tr[K] = (int16_t)m0;
        tr[K + 1] = (int16_t)k0;
      }
      __syncwarp();
    }

    // ---- a8: emit
    if (lane == 0) {
      T* oq = reinterpret_cast<T*>(a.out_q) + 4 * (size_t)w;
      T* ot = reinterpret_cast<T*>(a.out_t) + 3 * (size_t)w;
      oq[0] = q.w, oq[1] = q.x, oq[2] = q.y, oq[3] = q.z;
      ot[0] = t.x, ot[1] = t.y, ot[2] = t.z;
      if (!(isfinite(q.w) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(t.x) && isfinite(t.y) &&
            isfinite(t.z)))
        atomicOr(a.status, kDevErrNumeric);
    }
    __syncwarp();
  }
  if (lane == 0 && evals) atomicAdd(a.evals, evals);
}

template <typename T, int KIND, int SAMPLER>
static cudaError_t launch_walk_t(purse_t h, const purse_params* p, const WalkArgs& a, cudaStream_t st) {
  const int mc = p->n_keep >= 32 ? 1 : 32 / p->n_keep;
  const size_t slab = walk_slab_bytes<T>(a.n, p->n_perturb, p->n_steps, mc, SAMPLER);
  const size_t smem = 128 + walk_table_bytes<T>(a.n) + kWalkWarps * slab;
  auto kern = walk_kernel<T, KIND, SAMPLER>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWalkThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long need = (a.n_samples + kWalkWarps - 1) / kWalkWarps;
  const long cap = (long)per_sm * h->sm_count;
  const int grid = (int)(need < cap ? need : cap);
  kern<<<grid, kWalkThreads, smem, st>>>(a, mc, (int)slab);
  return cudaGetLastError();
}

cudaError_t launch_walk(purse_t h, const purse_params* p, const WalkArgs& a, cudaStream_t st) {
  const bool dbl = p->precision == 1;
  const int kind = h->kind, smp = p->sampler;
  if (!dbl) {
    if (kind == 0) return smp == 0 ? launch_walk_t<float, 0, 0>(h, p, a, st) : launch_walk_t<float, 0, 1>(h, p, a, st);
    return smp == 0 ? launch_walk_t<float, 1, 0>(h, p, a, st) : launch_walk_t<float, 1, 1>(h, p, a, st);
  }
  if (kind == 0) return smp == 0 ? launch_walk_t<double, 0, 0>(h, p, a, st) : launch_walk_t<double, 0, 1>(h, p, a, st);
  return smp == 0 ? launch_walk_t<double, 1, 0>(h, p, a, st) : launch_walk_t<double, 1, 1>(h, p, a, st);
}

}  // namespace purse
