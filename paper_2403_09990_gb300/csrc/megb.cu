// Minimum enclosing geodesic balls of the samples (Step III) by geodesic
// gradient descent (Section II; step rule of Alg. 6):
//   rotation:    f_k = argmax_s |vec(C_{k-1}^* q_s)|^2   (= sin^2 of half the
//                geodesic distance, monotone on [0, pi]),
//                C_k = SLERP(C_{k-1}, q_{f_k}, 1/k)
//   translation: f_k = argmax_s |t_s - c_{k-1}|^2,  c_k = c_{k-1} + (t_f - c_{k-1}) / k
// Every block reduces its slice to a (key, index) partial (FP32 samples: one
// 64-bit atomic maximum per block; FP64 samples: an array of partials).  One
// launch per iteration (megb_backward, the allocation-free solver): the last block
// to finish (atomic ticket, no waiting) takes the farthest sample and the step in
// FP64.  One persistent launch for both balls (megb_solve): after a bounded grid
// barrier every block takes the same step itself.  A final pass computes the
// radius from the farthest sample with an FP64 log map.  Ties go to the lowest
// index.
#include <climits>
#include <mutex>

#include "dev.cuh"
#include "internal.h"

namespace purse {

constexpr int kMegbThreads = 256;

struct MegbState {
  double C[4];
  double c[4];
  unsigned int counter[2];
  int fstar[2];       // farthest sample from the final centre (rotation, translation)
  unsigned int gen[2];  // iterations published by the persistent kernel
  // FP32 samples: farthest (key bits, complement of the index) of the iteration so far, per ball and
  // iteration mod 2 (one launch per iteration: the block that takes the step reads and clears it) or
  // mod 3 (persistent kernel: every block reads it after the barrier, block 0 clears the slot of the
  // iteration after next)
  unsigned long long best[2][3];
  // output rule of Alg. 6 (megb_solve_mean): sums over the last iterates -- of q q^T (upper triangle of
  // the 4 x 4 matrix, 10 values) for the rotation ball and of c for the translation ball
  double acc[13];
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct Part {
  double key;
  int idx;
  int pad;
};

__host__ __device__ inline size_t megb_blocks_cap(int sm_count) { return 4 * (size_t)sm_count; }

size_t megb_scratch_bytes(int n_iters, int sm_count) {
  return sizeof(MegbState) + 2 * megb_blocks_cap(sm_count) * sizeof(Part) + 2 * (size_t)n_iters * sizeof(int32_t) + 256;
}

// The farthest-sample rule (larger key, ties to the lower index) on the bit patterns of keys >= 0, which
// order like the values (an empty entry is (0, INT_MAX), below every sample).
__device__ __forceinline__ bool better_bits(unsigned long long ka, int ia, unsigned long long kb, int ib) {
  return ka > kb || (ka == kb && ia < ib);
}

// Warp reduction of (key bits, index) by that rule with three integer warp maxima.
__device__ __forceinline__ void warp_best64(unsigned long long& kb, int& bi) {
  const bool has = bi != INT_MAX;
  const uint32_t hw = __reduce_max_sync(kFullMask, has ? (uint32_t)(kb >> 32) : 0u);
  const uint32_t lw = __reduce_max_sync(kFullMask, has && (uint32_t)(kb >> 32) == hw ? (uint32_t)kb : 0u);
  const unsigned long long m = ((unsigned long long)hw << 32) | lw;
  const uint32_t mi = __reduce_max_sync(kFullMask, has && kb == m ? ~(uint32_t)bi : 0u);
  kb = m;
  bi = mi ? (int)~mi : INT_MAX;
}

template <typename T>
__global__ void megb_init(const T* q, int nq, const T* t, int nt, MegbState* s) {
  if (threadIdx.x != 0) return;
  if (nq > 0) {
    const Q4<double> c = qnormalize(Q4<double>{(double)q[0], (double)q[1], (double)q[2], (double)q[3]});
    s->C[0] = c.w, s->C[1] = c.x, s->C[2] = c.y, s->C[3] = c.z;
  }
  if (nt > 0) {
    s->c[0] = t[0], s->c[1] = t[1], s->c[2] = t[2];
  }
  s->c[3] = 0.0;
  s->counter[0] = s->counter[1] = 0;
  s->gen[0] = s->gen[1] = 0;
  for (int i = 0; i < 6; ++i) s->best[i / 3][i % 3] = 0ull;
  for (int i = 0; i < 13; ++i) s->acc[i] = 0.0;
}

// Squared sine of half the geodesic distance between centre (cw, cv) and q.
template <typename T>
__device__ __forceinline__ T rot_key(T cw, T cx, T cy, T cz, const T* qs) {
  const T qw = qs[0], qx = qs[1], qy = qs[2], qz = qs[3];
  // vector part of c^* (x) q = cw qv - qw cv - cv x qv
  const T vx = cw * qx - qw * cx - (cy * qz - cz * qy);
  const T vy = cw * qy - qw * cy - (cz * qx - cx * qz);
  const T vz = cw * qz - qw * cz - (cx * qy - cy * qx);
  return vx * vx + vy * vy + vz * vz;
}

// Relative rotation d = C* (x) q_f on the short path (w >= 0), its sine norm and angle.
struct RelRot {
  Q4<double> d;
  double sn, inv_sn, th;
};
__device__ __forceinline__ RelRot rel_rot(const Q4<double>& c, const Q4<double>& qf) {
  RelRot r;
  r.d = qmul(Q4<double>{c.w, -c.x, -c.y, -c.z}, qf);
  if (r.d.w < 0) r.d = Q4<double>{-r.d.w, -r.d.x, -r.d.y, -r.d.z};
  const double s2 = r.d.x * r.d.x + r.d.y * r.d.y + r.d.z * r.d.z;
  r.inv_sn = s2 > 0.0 ? rsqrt(s2) : 0.0;
  r.sn = s2 * r.inv_sn;
  r.th = 2.0 * atan2(r.sn, r.d.w);
  return r;
}

// GGD step k on SO(3): SLERP(C, q_f, 1/k) = C Exp(Log(C^T R_f) / k).  Written for few FP64
// instructions (each costs the same whatever the number of active lanes): one sincos, products by
// reciprocals, and no renormalisation -- both factors are unit quaternions to FP64 rounding, so the
// norm drifts by ~1e-16 per step; only the sign is kept (w >= 0).
__device__ __forceinline__ Q4<double> slerp_step(const Q4<double>& c, const RelRot& r, int k) {
  Q4<double> step{1.0, 0.0, 0.0, 0.0};
  if (r.sn > 0.0) {
    double sh, ch;
    sincos(r.th * (0.5 / k), &sh, &ch);
    sh *= r.inv_sn;
    step = Q4<double>{ch, sh * r.d.x, sh * r.d.y, sh * r.d.z};
  }
  Q4<double> o = qmul(c, step);
  if (o.w < 0.0) o = Q4<double>{-o.w, -o.x, -o.y, -o.z};
  return o;
}

// Output rule of Alg. 6 (the appendix's descent): the centre is the projection onto SO(3) of the sum
// of the rotation matrices of the last navg iterates C_{K-navg+1} .. C_K (all of C_0 .. C_K when there
// are fewer), i.e. the unit quaternion maximising sum (4 (p . C_t)^2 - 1) over p: the eigenvector of the
// largest eigenvalue of sum C_t C_t^T.  Called by the thread that takes step k with the previous and
// the new iterate; adds them to the sums in s->acc and returns, at k == K, the projected mean (the new
// iterate before).  The translation ball averages its last centres the same way (no projection).
__device__ __forceinline__ Q4<double> mean_rule_rotation(MegbState* s, const Q4<double>& prev, const Q4<double>& cn,
                                                         int k, int K, int navg) {
  const int first = K - navg + 1;
  double a[10];
  for (int e = 0; e < 10; ++e) a[e] = s->acc[e];
  auto add = [&](const Q4<double>& q) {
    const double v[4] = {q.w, q.x, q.y, q.z};
    int e = 0;
    for (int i = 0; i < 4; ++i)
      for (int j = i; j < 4; ++j) a[e++] += v[i] * v[j];
  };
  if (k == 1 && first <= 0) add(prev);
  if (k >= first) add(cn);
  if (k < K) {
    for (int e = 0; e < 10; ++e) s->acc[e] = a[e];
    return cn;
  }
  double N[4][4], V[4][4];
  int e = 0;
  for (int i = 0; i < 4; ++i)
    for (int j = i; j < 4; ++j) N[i][j] = N[j][i] = a[e++];
  jacobi_eigen<4>(N, V);
  int best = 0;
  for (int i = 1; i < 4; ++i)
    if (N[i][i] > N[best][best]) best = i;
  Q4<double> q = qnormalize(Q4<double>{V[0][best], V[1][best], V[2][best], V[3][best]});
  if (q.w < 0.0) q = Q4<double>{-q.w, -q.x, -q.y, -q.z};
  return q;
}

__device__ __forceinline__ void mean_rule_translation(MegbState* s, const double* prev, double* cn, int k, int K,
                                                      int navg) {
  const int first = K - navg + 1;
  double a[3];
  for (int d = 0; d < 3; ++d) a[d] = s->acc[10 + d];
  for (int d = 0; d < 3; ++d) {
    if (k == 1 && first <= 0) a[d] += prev[d];
    if (k >= first) a[d] += cn[d];
  }
  if (k < K) {
    for (int d = 0; d < 3; ++d) s->acc[10 + d] = a[d];
    return;
  }
  const double cnt = double(first <= 0 ? K + 1 : navg);
  for (int d = 0; d < 3; ++d) cn[d] = a[d] / cnt;
}

// Key of sample i: squared sine of half the angle to the centre (rotation) or squared distance.
template <typename T, int MODE>
__device__ __forceinline__ T sample_key(const T* __restrict__ x, int i, bool vec, T c0, T c1, T c2, T c3) {
  if (MODE == 0) {
    if (vec) {
      T qv[4];
      if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(x) + i);
        qv[0] = v.x, qv[1] = v.y, qv[2] = v.z, qv[3] = v.w;
      } else {
        const double2 a = __ldg(reinterpret_cast<const double2*>(x) + 2 * (size_t)i);
        const double2 b = __ldg(reinterpret_cast<const double2*>(x) + 2 * (size_t)i + 1);
        qv[0] = a.x, qv[1] = a.y, qv[2] = b.x, qv[3] = b.y;
      }
      return rot_key(c0, c1, c2, c3, qv);
    }
    return rot_key(c0, c1, c2, c3, x + 4 * (size_t)i);
  }
  const T* p = x + 3 * (size_t)i;
  const T dx = __ldg(p) - c0, dy = __ldg(p + 1) - c1, dz = __ldg(p + 2) - c2;
  return dx * dx + dy * dy + dz * dz;
}

// This thread's farthest sample of its slice (samples bid * blockDim.x + threadIdx.x + j * stride) from the
// centre (c0, c1, c2, c3): the largest key in the key precision (its conversion to FP64 is exact and keeps
// the order), ties to the lowest index; (-1, INT_MAX) when the slice is empty.
template <typename T, int MODE>
__device__ __forceinline__ void scan_slice(const T* __restrict__ x, int n, int bid, int stride, T c0, T c1, T c2, T c3,
                                           T& bkt, int& bi) {
  bkt = T(-1);
  bi = INT_MAX;
  // Four samples in flight per thread (indices ascending, so the strict > keeps the lowest index
  // among equal keys); quaternions are read as 16-byte vectors when the array allows it.
  const bool vec = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  int i = bid * blockDim.x + threadIdx.x;
  const bool grouped = MODE == 1 && sizeof(T) == 4 && vec;
  if (grouped) {
    // FP32 translations: groups of four samples = three 16-byte vectors per thread, two groups in
    // flight; the n mod 4 tail is read by the first threads after all groups (indices stay ascending).
    const int ng = n >> 2;
    int gi = i;
    for (; (long)gi + stride < (long)ng; gi += 2 * stride) {
      float4 v[6];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int r = 0; r < 3; ++r) v[3 * u + r] = __ldg(reinterpret_cast<const float4*>(x) + 3 * (size_t)(gi + u * stride) + r);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float f[12] = {v[3 * u].x, v[3 * u].y, v[3 * u].z, v[3 * u].w, v[3 * u + 1].x, v[3 * u + 1].y,
                             v[3 * u + 1].z, v[3 * u + 1].w, v[3 * u + 2].x, v[3 * u + 2].y, v[3 * u + 2].z,
                             v[3 * u + 2].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const T dx = f[3 * e] - c0, dy = f[3 * e + 1] - c1, dz = f[3 * e + 2] - c2;
          const T key = dx * dx + dy * dy + dz * dz;
          if (key > bkt) bkt = key, bi = 4 * (gi + u * stride) + e;
        }
      }
    }
    for (; gi < ng; gi += stride) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(x) + 3 * (size_t)gi);
      const float4 b = __ldg(reinterpret_cast<const float4*>(x) + 3 * (size_t)gi + 1);
      const float4 c = __ldg(reinterpret_cast<const float4*>(x) + 3 * (size_t)gi + 2);
      const float f[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const T dx = f[3 * e] - c0, dy = f[3 * e + 1] - c1, dz = f[3 * e + 2] - c2;
        const T key = dx * dx + dy * dy + dz * dz;
        if (key > bkt) bkt = key, bi = 4 * gi + e;
      }
    }
    i = 4 * ng + i;  // tail
  }
  for (; !grouped && (long)i + 3L * stride < (long)n; i += 4 * stride) {
    T key[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) key[u] = sample_key<T, MODE>(x, i + u * stride, vec, c0, c1, c2, c3);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (key[u] > bkt) bkt = key[u], bi = i + u * stride;
  }
  for (; i < n; i += stride) {
    const T key = sample_key<T, MODE>(x, i, vec, c0, c1, c2, c3);
    if (key > bkt) bkt = key, bi = i;
  }
}

// One GGD iteration of a ball over this block's slice of the samples.  MODE 0: rotation ball, MODE 1:
// translation ball.  k >= 1: GGD step k; k == 0: final radius.  Every block reduces its slice to a
// (key, index) maximum -- FP32 samples: packed into one 64-bit atomic maximum; FP64 samples: a
// partial per block -- and the last block to take a ticket takes the farthest sample and the step in
// FP64 (its thread 0 writes the state).  Returns true in the block that took the step.
template <typename T, int MODE>
__device__ __forceinline__ bool ggd_iter(const T* __restrict__ x, int n, MegbState* s, Part* parts, int k, int K,
                                         int navg, int32_t* f_int, int32_t* f_out, double* result, double* wkey,
                                         int* widx, bool* last, int bid, int nb) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T c0, c1, c2, c3;
  if (MODE == 0)
    c0 = T(s->C[0]), c1 = T(s->C[1]), c2 = T(s->C[2]), c3 = T(s->C[3]);
  else
    c0 = T(s->c[0]), c1 = T(s->c[1]), c2 = T(s->c[2]), c3 = T(0);
  T bkt;
  int bi;
  scan_slice<T, MODE>(x, n, bid, nb * (int)blockDim.x, c0, c1, c2, c3, bkt, bi);
  if constexpr (sizeof(T) == 4) {
    // FP32 keys are >= 0 (or never taken: NaN fails key > bkt), so their bit patterns order like the
    // values; (key bits, complement of the index) packed in 64 bits is largest for the farthest
    // sample, ties to the lowest index -- the rule of better_bits(), reduced with integer operations only
    // (each FP64 instruction of a warp occupies this part's FP64 unit for tens of cycles).  An empty
    // thread packs 0, below every sample.
    const bool has = bi != INT_MAX;
    const uint32_t kb = has ? __float_as_uint(bkt) : 0u;
    const uint32_t mk = __reduce_max_sync(kFullMask, kb);
    const uint32_t mi = __reduce_max_sync(kFullMask, has && kb == mk ? ~(uint32_t)bi : 0u);
    unsigned long long* wpk = reinterpret_cast<unsigned long long*>(wkey);
    if (lane == 0) wpk[warp] = ((unsigned long long)mk << 32) | mi;
    __syncthreads();
    if (tid == 0) {
      unsigned long long b = wpk[0];
      for (int w = 1; w < kMegbThreads / 32; ++w) b = wpk[w] > b ? wpk[w] : b;
      unsigned long long* slot = &s->best[MODE][k & 1];
      atomicMax(slot, b);
      __threadfence();
      const unsigned ticket = atomicAdd(&s->counter[MODE], 1u);
      *last = ticket == (unsigned)nb - 1;
      if (*last) {
        __threadfence();
        // every block's maximum is in (its atomicMax came before its ticket); clear the slot for the
        // iteration after next
        b = atomicExch(slot, 0ull);
        bi = b == 0ull ? 0 : (int)~(uint32_t)b;
      }
    }
    __syncthreads();
    if (!*last) return false;
    if (tid != 0) return true;
  } else {
    // FP64 keys (>= 0) order like their 64-bit patterns: the same rule with integer reductions of
    // (key bits, index) -- the high word, then the low word, then the complement of the index
    unsigned long long kb = bi != INT_MAX ? (unsigned long long)__double_as_longlong(bkt) : 0ull;
    warp_best64(kb, bi);
    unsigned long long* wpk = reinterpret_cast<unsigned long long*>(wkey);
    if (lane == 0) wpk[warp] = kb, widx[warp] = bi;
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < kMegbThreads / 32; ++w)
        if (better_bits(wpk[w], widx[w], kb, bi)) kb = wpk[w], bi = widx[w];
      parts[bid] = Part{__longlong_as_double((long long)kb), bi, 0};
      __threadfence();
      const unsigned ticket = atomicAdd(&s->counter[MODE], 1u);
      *last = ticket == (unsigned)nb - 1;
    }
    __syncthreads();
    if (!*last) return false;
    __threadfence();
    kb = 0ull, bi = INT_MAX;
    for (int b = tid; b < nb; b += blockDim.x) {
      // partials of other blocks: read from L2, bypassing this SM's L1
      const unsigned long long pk = (unsigned long long)__ldcg(reinterpret_cast<const long long*>(&parts[b].key));
      const int pi = __ldcg(&parts[b].idx);
      if (better_bits(pk, pi, kb, bi)) kb = pk, bi = pi;
    }
    warp_best64(kb, bi);
    __syncthreads();  // every warp has read wpk / widx of the first reduction
    if (lane == 0) wpk[warp] = kb, widx[warp] = bi;
    __syncthreads();
    if (tid != 0) return true;
    for (int w = 1; w < kMegbThreads / 32; ++w)
      if (better_bits(wpk[w], widx[w], kb, bi)) kb = wpk[w], bi = widx[w];
  }
  s->counter[MODE] = 0;
  auto ld = [](const double* p) { return *p; };
  if (MODE == 0) {
    const T* qs = x + 4 * (size_t)bi;
    const Q4<double> c{ld(&s->C[0]), ld(&s->C[1]), ld(&s->C[2]), ld(&s->C[3])};
    const Q4<double> qf = qnormalize(Q4<double>{(double)qs[0], (double)qs[1], (double)qs[2], (double)qs[3]});
    const RelRot r = rel_rot(c, qf);
    if (k > 0) {
      Q4<double> cn = slerp_step(c, r, k);
      if (navg > 1) cn = mean_rule_rotation(s, c, cn, k, K, navg);
      s->C[0] = cn.w, s->C[1] = cn.x, s->C[2] = cn.y, s->C[3] = cn.z;
    } else {
      result[0] = c.w, result[1] = c.x, result[2] = c.y, result[3] = c.z;
      result[7] = r.th;
    }
  } else {
    const T* p = x + 3 * (size_t)bi;
    const double c0d = ld(&s->c[0]), c1d = ld(&s->c[1]), c2d = ld(&s->c[2]);
    if (k > 0) {
      const double rk = 1.0 / k;
      double cn[3] = {c0d + ((double)p[0] - c0d) * rk, c1d + ((double)p[1] - c1d) * rk, c2d + ((double)p[2] - c2d) * rk};
      if (navg > 1) {
        const double prev[3] = {c0d, c1d, c2d};
        mean_rule_translation(s, prev, cn, k, K, navg);
      }
      s->c[0] = cn[0], s->c[1] = cn[1], s->c[2] = cn[2];
    } else {
      const double dx = (double)p[0] - c0d, dy = (double)p[1] - c1d, dz = (double)p[2] - c2d;
      result[4] = c0d, result[5] = c1d, result[6] = c2d;
      result[8] = sqrt(dx * dx + dy * dy + dz * dz);
    }
  }
  if (k > 0) {
    f_int[k - 1] = bi;
    if (f_out) f_out[k - 1] = bi;
  } else {
    s->fstar[MODE] = bi;
  }
  return true;
}

// One launch per iteration (the state is complete at every kernel boundary).
template <typename T, int MODE>
__global__ void __launch_bounds__(kMegbThreads)
    ggd_step(const T* __restrict__ x, int n, MegbState* s, Part* parts, int k, int K, int navg, int32_t* f_int,
             int32_t* f_out, double* result) {
  __shared__ double wkey[kMegbThreads / 32];
  __shared__ int widx[kMegbThreads / 32];
  __shared__ bool last;
  ggd_iter<T, MODE>(x, n, s, parts, k, K, navg, f_int, f_out, result, wkey, widx, &last, blockIdx.x, gridDim.x);
}

// The slice of this block's thread kept in shared memory for all iterations of the persistent kernel:
// sample i = bid * blockDim.x + threadIdx.x + j * stride (j < J) in slot j * blockDim.x + threadIdx.x --
// rotations as 4 values per slot, translations as three planes of J * blockDim.x values.  Every thread
// reads back only its own slots.
template <typename T, int MODE>
__device__ __forceinline__ void cache_slice(const T* __restrict__ x, int n, int bid, int stride, int J, T* cache) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = 0; j < J; ++j) {
    const long i = (long)bid * nt + tid + (long)j * stride;
    if (i >= n) break;
    const int slot = j * nt + tid;
    if (MODE == 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) cache[4 * slot + c] = x[4 * i + c];
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) cache[c * J * nt + slot] = x[3 * i + c];
    }
  }
}

// scan_slice over the cached slice: the same keys in the same order (indices ascending, strict >).
template <typename T, int MODE>
__device__ __forceinline__ void scan_cached(const T* cache, int n, int bid, int stride, int J, T c0, T c1, T c2, T c3,
                                            T& bkt, int& bi) {
  const int tid = threadIdx.x, nt = blockDim.x;
  bkt = T(-1);
  bi = INT_MAX;
  const int i0 = bid * nt + tid;
  // slots j < jn hold samples of this thread (i0 + j stride < n)
  const int jn = i0 >= n ? 0 : min(J, (n - 1 - i0) / stride + 1);
#pragma unroll 4
  for (int j = 0; j < jn; ++j) {
    const int slot = j * nt + tid;
    T key;
    if (MODE == 0) {
      T qv[4];
      if constexpr (sizeof(T) == 4) {
        const float4 v = reinterpret_cast<const float4*>(cache)[slot];
        qv[0] = v.x, qv[1] = v.y, qv[2] = v.z, qv[3] = v.w;
      } else {
        const double2 a = reinterpret_cast<const double2*>(cache)[2 * slot];
        const double2 b = reinterpret_cast<const double2*>(cache)[2 * slot + 1];
        qv[0] = a.x, qv[1] = a.y, qv[2] = b.x, qv[3] = b.y;
      }
      key = rot_key(c0, c1, c2, c3, qv);
    } else {
      const T dx = cache[slot] - c0, dy = cache[J * nt + slot] - c1, dz = cache[2 * J * nt + slot] - c2;
      key = dx * dx + dy * dy + dz * dz;
    }
    if (key > bkt) bkt = key, bi = i0 + j * stride;
  }
}

// All K iterations and the radius pass of a ball on blocks [0, nb) of its group in a cooperative launch
// (every block resident).  Every block keeps its own copy of the descent state in shared memory and
// takes every step itself: per iteration it reduces its slice to a farthest (key, index), posts it
// (FP32 keys: one 64-bit atomic maximum of (key bits, complement of the index) into the iteration's
// slot of a ring of three; FP64 keys: its partial), arrives on the group's counter (release) and
// waits (acquire, bounded poll) until all nb blocks of the group have arrived; then it reads the
// farthest sample and takes the FP64 step.  Every block computes the same step from the same values,
// so the copies stay identical, and the farthest sample does not depend on the grid (keys descending,
// indices ascending): the results equal those of the one-launch-per-iteration kernel.  Block 0 writes
// the farthest sequence, the result and the final state.  If the poll limit runs out the block flags
// a timeout in the status word and leaves (the result is then not written).
template <typename T, int MODE>
__device__ __forceinline__ void ggd_ball(const T* __restrict__ x, int n, MegbState* s, Part* parts, int n_iters,
                                         int navg, int32_t* f_int, int32_t* f_out, double* result, int* status, int bid,
                                         int nb, MegbState* loc, unsigned long long* wpk, int* widx, int* fsh,
                                         bool* stop, T* cache, int J) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int stride = nb * (int)blockDim.x;
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) loc->C[i] = __ldcg(&s->C[i]), loc->c[i] = __ldcg(&s->c[i]);
    for (int i = 0; i < 13; ++i) loc->acc[i] = __ldcg(&s->acc[i]);
  }
  if (J > 0) cache_slice<T, MODE>(x, n, bid, stride, J, cache);
  __syncthreads();
  for (int it = 1; it <= n_iters + 1; ++it) {
    const int k = it <= n_iters ? it : 0;
    T c0, c1, c2, c3 = T(0);
    if (MODE == 0)
      c0 = T(loc->C[0]), c1 = T(loc->C[1]), c2 = T(loc->C[2]), c3 = T(loc->C[3]);
    else
      c0 = T(loc->c[0]), c1 = T(loc->c[1]), c2 = T(loc->c[2]);
    T bkt;
    int bi;
    if (J > 0)
      scan_cached<T, MODE>(cache, n, bid, stride, J, c0, c1, c2, c3, bkt, bi);
    else
      scan_slice<T, MODE>(x, n, bid, stride, c0, c1, c2, c3, bkt, bi);
    // the block's farthest (key bits, index): keys >= 0 (NaN is never taken) order like their bit
    // patterns; an empty entry is (0, INT_MAX), below every sample
    const bool has = bi != INT_MAX;
    unsigned long long kb;
    if constexpr (sizeof(T) == 4) {
      const uint32_t k32 = has ? __float_as_uint(bkt) : 0u;
      const uint32_t mk = __reduce_max_sync(kFullMask, k32);
      const uint32_t mi = __reduce_max_sync(kFullMask, has && k32 == mk ? ~(uint32_t)bi : 0u);
      kb = ((unsigned long long)mk << 32) | mi;
    } else {
      kb = has ? (unsigned long long)__double_as_longlong(bkt) : 0ull;
      warp_best64(kb, bi);
    }
    if (lane == 0) wpk[warp] = kb, widx[warp] = bi;
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < kMegbThreads / 32; ++w) {
        if (sizeof(T) == 4) {
          kb = wpk[w] > kb ? wpk[w] : kb;
        } else if (better_bits(wpk[w], widx[w], kb, bi)) {
          kb = wpk[w], bi = widx[w];
        }
      }
      if (sizeof(T) == 4) {
        atomicMax(&s->best[MODE][it % 3], kb);
        // the slot of iteration it + 1 was last read after the barrier of iteration it - 2, before
        // every block arrived at the barrier of iteration it - 1, which this block has passed
        if (bid == 0) s->best[MODE][(it + 1) % 3] = 0ull;
      } else {
        parts[bid] = Part{__longlong_as_double((long long)kb), bi, 0};
      }
      __threadfence();
      atomicAdd(&s->gen[MODE], 1u);
      const unsigned target = (unsigned)nb * (unsigned)it;
      int polls = 0;
      *stop = false;
      while (ld_acquire(&s->gen[MODE]) < target) {
        if (++polls > (1 << 22)) {
          atomicOr(status, kDevErrTimeout);
          *stop = true;
          break;
        }
        __nanosleep(32);
      }
      if (sizeof(T) == 4 && !*stop) {
        const unsigned long long b = __ldcg(&s->best[MODE][it % 3]);
        *fsh = b == 0ull ? 0 : (int)~(uint32_t)b;
      }
    }
    __syncthreads();
    if (*stop) return;
    if constexpr (sizeof(T) == 8) {
      // the partials of every block of the group (read from L2, bypassing this SM's L1)
      kb = 0ull, bi = INT_MAX;
      for (int b = tid; b < nb; b += blockDim.x) {
        const unsigned long long pk = (unsigned long long)__ldcg(reinterpret_cast<const long long*>(&parts[b].key));
        const int pi = __ldcg(&parts[b].idx);
        if (better_bits(pk, pi, kb, bi)) kb = pk, bi = pi;
      }
      warp_best64(kb, bi);
      if (lane == 0) wpk[warp] = kb, widx[warp] = bi;
      __syncthreads();
      if (tid == 0) {
        for (int w = 1; w < kMegbThreads / 32; ++w)
          if (better_bits(wpk[w], widx[w], kb, bi)) kb = wpk[w], bi = widx[w];
        *fsh = bi == INT_MAX ? 0 : bi;
      }
    }
    if (tid == 0) {
      const int f = *fsh;
      if (MODE == 0) {
        const T* qs = x + 4 * (size_t)f;
        const Q4<double> c{loc->C[0], loc->C[1], loc->C[2], loc->C[3]};
        const Q4<double> qf = qnormalize(Q4<double>{(double)qs[0], (double)qs[1], (double)qs[2], (double)qs[3]});
        const RelRot r = rel_rot(c, qf);
        if (k > 0) {
          Q4<double> cn = slerp_step(c, r, k);
          if (navg > 1) cn = mean_rule_rotation(loc, c, cn, k, n_iters, navg);
          loc->C[0] = cn.w, loc->C[1] = cn.x, loc->C[2] = cn.y, loc->C[3] = cn.z;
        } else if (bid == 0) {
          result[0] = c.w, result[1] = c.x, result[2] = c.y, result[3] = c.z;
          result[7] = r.th;
        }
      } else {
        const T* p = x + 3 * (size_t)f;
        const double c0d = loc->c[0], c1d = loc->c[1], c2d = loc->c[2];
        if (k > 0) {
          const double rk = 1.0 / k;
          double cn[3] = {c0d + ((double)p[0] - c0d) * rk, c1d + ((double)p[1] - c1d) * rk,
                          c2d + ((double)p[2] - c2d) * rk};
          if (navg > 1) {
            const double prev[3] = {c0d, c1d, c2d};
            mean_rule_translation(loc, prev, cn, k, n_iters, navg);
          }
          loc->c[0] = cn[0], loc->c[1] = cn[1], loc->c[2] = cn[2];
        } else if (bid == 0) {
          const double dx = (double)p[0] - c0d, dy = (double)p[1] - c1d, dz = (double)p[2] - c2d;
          result[4] = c0d, result[5] = c1d, result[6] = c2d;
          result[8] = sqrt(dx * dx + dy * dy + dz * dz);
        }
      }
      if (bid == 0) {
        if (k > 0) {
          f_int[k - 1] = f;
          if (f_out) f_out[k - 1] = f;
        } else {
          s->fstar[MODE] = f;
          for (int i = 0; i < 4; ++i) {
            if (MODE == 0) s->C[i] = loc->C[i];
            else s->c[i] = loc->c[i];
          }
        }
      }
    }
    __syncthreads();
  }
}

// Both balls in one launch: blocks [0, gq) descend the rotation ball, blocks [gq, gridDim.x) the
// translation ball (each group with its own ticket and iteration counter).
template <typename T>
__global__ void __launch_bounds__(kMegbThreads)
    ggd_persistent(const T* __restrict__ q, int nq, const T* __restrict__ t, int nt, int gq, MegbState* s,
                   Part* parts_q, Part* parts_t, int n_iters, int navg, int32_t* f_int, int32_t* f_out,
                   double* result, int* status, int jq, int jt) {
  __shared__ MegbState loc;
  __shared__ unsigned long long wpk[kMegbThreads / 32];
  __shared__ int widx[kMegbThreads / 32];
  __shared__ int fsh;
  __shared__ bool stop;
  extern __shared__ __align__(16) unsigned char slice[];  // jq / jt > 0: the block's samples, kept
  T* cache = reinterpret_cast<T*>(slice);
  if ((int)blockIdx.x < gq)
    ggd_ball<T, 0>(q, nq, s, parts_q, n_iters, navg, f_int, f_out, result, status, blockIdx.x, gq, &loc, wpk, widx, &fsh,
                   &stop, cache, jq);
  else
    ggd_ball<T, 1>(t, nt, s, parts_t, n_iters, navg, f_int + n_iters, f_out ? f_out + n_iters : nullptr, result, status,
                   blockIdx.x - gq, gridDim.x - gq, &loc, wpk, widx, &fsh, &stop, cache, jt);
}

__global__ void megb_zero_result(double* result, int skip_rot, int skip_tr) {
  if (threadIdx.x != 0) return;
  if (skip_rot) result[0] = result[1] = result[2] = result[3] = result[7] = 0.0;
  if (skip_tr) result[4] = result[5] = result[6] = result[8] = 0.0;
}

template <typename T>
static cudaError_t launch_megb_t(purse_t h, int n_iters, int navg, const T* q, int nq, const T* t, int nt,
                                 double* result, int32_t* f_out, void* scratch, cudaStream_t st) {
  MegbState* s = reinterpret_cast<MegbState*>(scratch);
  Part* parts = reinterpret_cast<Part*>(reinterpret_cast<char*>(scratch) + sizeof(MegbState));
  int32_t* f_int = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(parts) + 2 * megb_blocks_cap(h->sm_count) * sizeof(Part));
  megb_init<T><<<1, 32, 0, st>>>(q, nq, t, nt, s);
  megb_zero_result<<<1, 32, 0, st>>>(result, nq == 0, nt == 0);
  const long cap = (long)megb_blocks_cap(h->sm_count);
  // one cooperative launch for both balls when every block fits on the GPU at once
  static int resident[2] = {-1, -1};  // co-resident ggd_persistent blocks per SM (FP32, FP64)
  int& per_sm = resident[sizeof(T) == 8];
  if (per_sm < 0) {
    int coop = 0, dev = 0, nbk = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess && coop)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbk, ggd_persistent<T>, kMegbThreads, 0);
    if (e != cudaSuccess) return e;
    per_sm = coop ? nbk : 0;
  }
  const long room = (long)per_sm * h->sm_count;
  // FP32 samples: four per thread (the pass streams them); FP64 samples: one per thread, since every
  // FP64 instruction of a warp occupies the SM's FP64 unit for tens of cycles and the keys need
  // spreading over as many SMs as the samples allow
  const int spt = tuned_config(kTuneMegb, h->kind, h->n, nq > nt ? nq : nt, sizeof(T) == 8, sizeof(T) == 8 ? 1 : 4);
  const long per_block = (long)kMegbThreads * (spt < 1 ? 1 : spt);
  const long want_q = nq > 0 ? ((long)nq + per_block - 1) / per_block : 0;
  const long want_t = nt > 0 ? ((long)nt + per_block - 1) / per_block : 0;
  if ((nq > 0 || nt > 0) && room >= 2) {
    // split the resident blocks between the balls (the farthest sample does not depend on the split)
    long gq = nq > 0 ? (want_q < cap ? want_q : cap) : 0, gt = nt > 0 ? (want_t < cap ? want_t : cap) : 0;
    if (gq < 1 && nq > 0) gq = 1;
    if (gt < 1 && nt > 0) gt = 1;
    if (gq + gt > room) {  // each group stays within cap (its partials array)
      if (nq > 0 && nt > 0) {
        const long half = room / 2;
        gq = gq < half ? gq : half;
        gt = gt < room - gq ? gt : room - gq;
      } else if (nq > 0) {
        gq = room;
      } else {
        gt = room;
      }
    }
    // keep every block's samples in shared memory for all iterations when they fit and every block stays
    // resident with that much shared memory
    int jq = gq > 0 ? (int)(((long)nq + gq * kMegbThreads - 1) / (gq * kMegbThreads)) : 0;
    int jt = gt > 0 ? (int)(((long)nt + gt * kMegbThreads - 1) / (gt * kMegbThreads)) : 0;
    const size_t bq = (size_t)jq * kMegbThreads * 4 * sizeof(T), bt = (size_t)jt * kMegbThreads * 3 * sizeof(T);
    size_t dyn = bq > bt ? bq : bt;
    static int smem_optin = -1;
    if (smem_optin < 0) {
      int dev = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (e != cudaSuccess) return e;
    }
    bool keep = dyn > 0 && dyn + 1024 <= (size_t)smem_optin;
    if (keep) {
      cudaError_t e = cudaFuncSetAttribute(ggd_persistent<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ggd_persistent<T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      int nbk = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbk, ggd_persistent<T>, kMegbThreads, dyn);
      if (e != cudaSuccess) return e;
      keep = (long)nbk * h->sm_count >= gq + gt;
    }
    if (!keep) jq = jt = 0, dyn = 0;
    int gqi = (int)gq, nqi = nq, nti = nt, ni = n_iters, na = navg;
    Part* parts_t = parts + cap;
    int* status = h->d_status;
    void* args[] = {(void*)&q, &nqi, (void*)&t, &nti, &gqi, &s, &parts, &parts_t, &ni, &na, &f_int, &f_out, &result,
                    &status, &jq, &jt};
    return cudaLaunchCooperativeKernel((const void*)ggd_persistent<T>, dim3((unsigned)(gq + gt)), dim3(kMegbThreads),
                                       args, dyn, st);
  }
  if (nq > 0) {
    const long want = ((long)nq + kMegbThreads * 4 - 1) / (kMegbThreads * 4);
    const int g = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    for (int k = 1; k <= n_iters; ++k)
      ggd_step<T, 0><<<g, kMegbThreads, 0, st>>>(q, nq, s, parts, k, n_iters, navg, f_int, f_out, result);
    ggd_step<T, 0><<<g, kMegbThreads, 0, st>>>(q, nq, s, parts, 0, n_iters, navg, f_int, f_out, result);
  }
  if (nt > 0) {
    const long want = ((long)nt + kMegbThreads * 4 - 1) / (kMegbThreads * 4);
    const int g = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    Part* parts_t = parts + cap;
    for (int k = 1; k <= n_iters; ++k)
      ggd_step<T, 1><<<g, kMegbThreads, 0, st>>>(t, nt, s, parts_t, k, n_iters, navg, f_int + n_iters,
                                                  f_out ? f_out + n_iters : nullptr, result);
    ggd_step<T, 1><<<g, kMegbThreads, 0, st>>>(t, nt, s, parts_t, 0, n_iters, navg, f_int + n_iters, nullptr, result);
  }
  return cudaGetLastError();
}

cudaError_t launch_megb(purse_t h, int precision, int n_iters, const void* d_q, int n_rot, const void* d_t, int n_tr,
                        double* d_result, int32_t* d_farthest, void* scratch, cudaStream_t st, int navg) {
  if (precision == 0)
    return launch_megb_t<float>(h, n_iters, navg, (const float*)d_q, n_rot, (const float*)d_t, n_tr, d_result, d_farthest,
                                scratch, st);
  return launch_megb_t<double>(h, n_iters, navg, (const double*)d_q, n_rot, (const double*)d_t, n_tr, d_result, d_farthest,
                               scratch, st);
}

// ---------------------------------------------------------------- adjoint
// Reverse-mode derivative of the balls through the boundary snap.  Rotations are perturbed on
// the left, R -> Exp(delta) R.  GGD step k linearises to eps_k = (I - A_k) eps_{k-1} + A_k delta_{f_k}
// with A_k = (1/k) C_k J_r(phi_k / k) J_l(phi_k)^-1 C_{k-1}^T, phi_k = Log(C_{k-1}^T R_{f_k}); the radius
// D = |Log(C_K^T R_f*)| gives dD = (C_K u)^T (delta_f* - eps_K) (u the unit axis; Section II and the
// appendix on geodesic gradient descent give the gradient of the squared distance along it).
// Translation: c_K is an affine combination of the farthest samples (Badoiu-Clarkson).  Each sample
// gradient g then moves its snapped sample along its ray: d tau* = (dr_j* - dh/dy . dy_j*) / h'.

// J_l(phi) y (inverse = false) or J_l(phi)^-1 y (inverse = true); J_l(phi)^T = J_l(-phi).
__device__ __forceinline__ V3<double> jl_apply(const V3<double>& phi, const V3<double>& y, bool inverse) {
  const double th2 = dot(phi, phi), th = sqrt(th2);
  const V3<double> py = cross(phi, y), ppy = cross(phi, py);
  double a, b;
  if (th < 1e-3) {
    a = inverse ? -0.5 : 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    b = inverse ? 1.0 / 12.0 + th2 / 720.0 + th2 * th2 / 30240.0 : 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
  } else if (inverse) {
    a = -0.5;
    b = 1.0 / th2 - 1.0 / (2.0 * th * tan(0.5 * th));
  } else {
    const double sh = sin(0.5 * th);
    a = 2.0 * sh * sh / th2;
    b = (th - sin(th)) / (th2 * th);
  }
  return V3<double>{y.x + a * py.x + b * ppy.x, y.y + a * py.y + b * ppy.y, y.z + a * py.z + b * ppy.z};
}

__device__ __forceinline__ V3<double> mul_t(const M3<double>& R, const V3<double>& a) {
  return V3<double>{R.m[0] * a.x + R.m[3] * a.y + R.m[6] * a.z, R.m[1] * a.x + R.m[4] * a.y + R.m[7] * a.z,
                    R.m[2] * a.x + R.m[5] * a.y + R.m[8] * a.z};
}

template <typename T>
__device__ __forceinline__ Q4<double> load_q(const T* q, int i) {
  const T* p = q + 4 * (size_t)i;
  return qnormalize(Q4<double>{(double)p[0], (double)p[1], (double)p[2], (double)p[3]});
}

// Scatter a sample gradient v (left tangent for rotation-ball samples, R^3 for translation-ball
// samples) through the sample's snap record.  Records whose ray does not move this ball's
// coordinate (ray kind != ball) or that were not snapped (j* < 0) take nothing.
template <typename T>
__device__ __forceinline__ void snap_scatter(const T* rec, int ball, V3<double> v, int n, int dim,
                                             double* gy, double* gr, int* status) {
  const double jd = (double)rec[0];
  if (!(jd >= 0.0) || (int)rec[1] != ball) return;
  const int j = (int)jd;
  const double hp = (double)rec[5];
  if (j >= n || !(hp != 0.0)) {
    atomicOr(status, kDevErrNumeric);
    return;
  }
  const double gt = (v.x * (double)rec[2] + v.y * (double)rec[3] + v.z * (double)rec[4]) / hp;
  gr[j] += gt;
  for (int c = 0; c < dim; ++c) gy[(size_t)dim * j + c] -= gt * (double)rec[6 + c];
}

// Reverse sweep of the rotation ball (one thread, FP64), accumulating into gy / gr.
// q: samples; snap: their records; f: the K farthest indices; fs: farthest from C_K;
// g: dL/d(result) (9); Cs: K + 1 quaternions of scratch.
template <typename T>
__device__ void adjoint_rotation(const T* q, const T* snap, int K, const int32_t* f, int fs, const double* g,
                                 Q4<double>* Cs, int n, int dim, double* gy, double* gr, int* status) {
  // recompute the iterates C_0..C_K from the stored farthest sequence
  Cs[0] = load_q(q, 0);
  for (int k = 1; k <= K; ++k) Cs[k] = slerp_step(Cs[k - 1], rel_rot(Cs[k - 1], load_q(q, f[k - 1])), k);
  const Q4<double> CK = Cs[K];
  const M3<double> RK = qmat(CK);
  // dL/d eps_K from the centre-quaternion gradient: g_C = (w g_v - g_w v + v x g_v) / 2
  const V3<double> vq{CK.x, CK.y, CK.z}, gv{g[1], g[2], g[3]};
  const V3<double> cv = cross(vq, gv);
  V3<double> lam{0.5 * (CK.w * gv.x - g[0] * vq.x + cv.x), 0.5 * (CK.w * gv.y - g[0] * vq.y + cv.y),
                 0.5 * (CK.w * gv.z - g[0] * vq.z + cv.z)};
  const RelRot r = rel_rot(CK, load_q(q, fs));
  if (r.sn > 0.0 && g[7] != 0.0) {
    const V3<double> w = mul(RK, V3<double>{r.d.x / r.sn, r.d.y / r.sn, r.d.z / r.sn});
    snap_scatter(snap + (size_t)kSnapStride * fs, 0, g[7] * w, n, dim, gy, gr, status);
    lam = lam - g[7] * w;
  }
  for (int k = K; k >= 1; --k) {
    const RelRot rk = rel_rot(Cs[k - 1], load_q(q, f[k - 1]));
    V3<double> phi{0.0, 0.0, 0.0};
    if (rk.sn > 0.0) phi = (rk.th / rk.sn) * V3<double>{rk.d.x, rk.d.y, rk.d.z};
    // A_k^T lam = (1/k) C_{k-1} J_l(-phi)^-1 J_l(phi/k) C_k^T lam
    V3<double> y = mul_t(qmat(Cs[k]), lam);
    y = jl_apply((1.0 / k) * phi, y, false);
    y = jl_apply(-1.0 * phi, y, true);
    const V3<double> v = (1.0 / k) * mul(qmat(Cs[k - 1]), y);
    snap_scatter(snap + (size_t)kSnapStride * f[k - 1], 0, v, n, dim, gy, gr, status);
    lam = lam - v;
  }
  snap_scatter(snap, 0, lam, n, dim, gy, gr, status);
}

// Reverse sweep of the translation ball; c: the final centre c_K (3 doubles).
template <typename T>
__device__ void adjoint_translation(const T* t, const T* snap, int K, const int32_t* f, int fs, const double* c,
                                    const double* g, int n, int dim, double* gy, double* gr, int* status) {
  const T* tf = t + 3 * (size_t)fs;
  const V3<double> e{(double)tf[0] - c[0], (double)tf[1] - c[1], (double)tf[2] - c[2]};
  const double dn = sqrt(dot(e, e));
  V3<double> mu{g[4], g[5], g[6]};
  if (dn > 0.0 && g[8] != 0.0) {
    const V3<double> u = (g[8] / dn) * e;
    snap_scatter(snap + (size_t)kSnapStride * fs, 1, u, n, dim, gy, gr, status);
    mu = mu - u;
  }
  for (int k = K; k >= 1; --k) {
    snap_scatter(snap + (size_t)kSnapStride * f[k - 1], 1, (1.0 / k) * mu, n, dim, gy, gr, status);
    mu = (1.0 - 1.0 / k) * mu;
  }
  snap_scatter(snap, 1, mu, n, dim, gy, gr, status);
}

// Both sweeps in parallel (warp 0: rotation into acc, warp 1: translation into acc + n (dim + 1)),
// then gy = rotation part + translation part, gr likewise.  acc: 2 n (dim + 1) zeroed here.
template <typename T>
__device__ void adjoint_both(const T* q, const T* snap_r, int nq, const T* t, const T* snap_t, int nt, int K,
                             const int32_t* f, const int* fstar, const double* result, const double* g,
                             Q4<double>* Cs, int n, int dim, double* acc, double* gy, double* gr, int* status) {
  const int m = n * (dim + 1);
  for (int i = threadIdx.x; i < 2 * m; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0 && nq > 0)
    adjoint_rotation(q, snap_r, K, f, fstar[0], g, Cs, n, dim, acc, acc + n * dim, status);
  if (threadIdx.x == 32 && nt > 0)
    adjoint_translation(t, snap_t, K, f + K, fstar[1], result + 4, g, n, dim, acc + m, acc + m + n * dim, status);
  __syncthreads();
  for (int i = threadIdx.x; i < n * dim; i += blockDim.x) gy[i] = acc[i] + acc[m + i];
  for (int i = threadIdx.x; i < n; i += blockDim.x) gr[i] = acc[n * dim + i] + acc[m + n * dim + i];
}

template <typename T>
__global__ void __launch_bounds__(64)
    megb_adjoint_kernel(const T* q, const T* snap_r, int nq, const T* t, const T* snap_t, int nt, int K,
                        const int32_t* f, const MegbState* s, const double* result, const double* g, Q4<double>* Cs,
                        double* acc, int n, int dim, double* gy, double* gr, int* status) {
  adjoint_both(q, snap_r, nq, t, snap_t, nt, K, f, s->fstar, result, g, Cs, n, dim, acc, gy, gr, status);
}

__global__ void megb_state_from_result(const double* result, MegbState* s) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i < 4; ++i) s->C[i] = result[i];
  for (int i = 0; i < 3; ++i) s->c[i] = result[4 + i];
  s->c[3] = 0.0;
  s->counter[0] = s->counter[1] = 0;
  s->fstar[0] = s->fstar[1] = 0;
  for (int i = 0; i < 6; ++i) s->best[i / 3][i % 3] = 0ull;
  for (int i = 0; i < 13; ++i) s->acc[i] = 0.0;
}

size_t megb_backward_scratch_bytes(int n_iters, int sm_count, int n) {
  return megb_scratch_bytes(n_iters, sm_count) + 16 * sizeof(double) + ((size_t)n_iters + 1) * sizeof(Q4<double>) +
         8 * (size_t)n * sizeof(double);
}

template <typename T>
static cudaError_t launch_megb_backward_t(purse_t h, int K, const T* q, const T* snap_r, int nq, const T* t,
                                          const T* snap_t, int nt, const int32_t* f, const double* result,
                                          const double* g, double* gy, double* gr, void* scratch, cudaStream_t st) {
  MegbState* s = reinterpret_cast<MegbState*>(scratch);
  Part* parts = reinterpret_cast<Part*>(reinterpret_cast<char*>(scratch) + sizeof(MegbState));
  const long cap = (long)megb_blocks_cap(h->sm_count);
  int32_t* f_int = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(parts) + 2 * cap * sizeof(Part));
  char* tail = reinterpret_cast<char*>(scratch) + megb_scratch_bytes(K, h->sm_count);
  double* dummy = reinterpret_cast<double*>(tail);
  Q4<double>* Cs = reinterpret_cast<Q4<double>*>(tail + 16 * sizeof(double));
  double* acc = reinterpret_cast<double*>(Cs + K + 1);
  megb_state_from_result<<<1, 32, 0, st>>>(result, s);
  // farthest sample from the final centres, by the forward's own final pass
  if (nq > 0) {
    const long want = ((long)nq + kMegbThreads * 4 - 1) / (kMegbThreads * 4);
    const int gsz = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    ggd_step<T, 0><<<gsz, kMegbThreads, 0, st>>>(q, nq, s, parts, 0, K, 1, f_int, nullptr, dummy);
  }
  if (nt > 0) {
    const long want = ((long)nt + kMegbThreads * 4 - 1) / (kMegbThreads * 4);
    const int gsz = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    ggd_step<T, 1><<<gsz, kMegbThreads, 0, st>>>(t, nt, s, parts + cap, 0, K, 1, f_int, nullptr, dummy);
  }
  const int dim = h->kind == PURSE_2D3D ? 2 : 3;
  megb_adjoint_kernel<T><<<1, 64, 0, st>>>(q, snap_r, nq, t, snap_t, nt, K, f, s, result, g, Cs, acc, h->n, dim, gy,
                                           gr, h->d_status);
  return cudaGetLastError();
}

cudaError_t launch_megb_backward(purse_t h, int precision, int n_iters, const void* d_q, const void* d_snap_rot,
                                 int n_rot, const void* d_t, const void* d_snap_tr, int n_tr,
                                 const int32_t* d_farthest, const double* d_result, const double* d_grad_result,
                                 double* d_grad_obs, double* d_grad_radii, void* scratch, cudaStream_t st) {
  if (precision == 0)
    return launch_megb_backward_t<float>(h, n_iters, (const float*)d_q, (const float*)d_snap_rot, n_rot,
                                         (const float*)d_t, (const float*)d_snap_tr, n_tr, d_farthest, d_result,
                                         d_grad_result, d_grad_obs, d_grad_radii, scratch, st);
  return launch_megb_backward_t<double>(h, n_iters, (const double*)d_q, (const double*)d_snap_rot, n_rot,
                                        (const double*)d_t, (const double*)d_snap_tr, n_tr, d_farthest, d_result,
                                        d_grad_result, d_grad_obs, d_grad_radii, scratch, st);
}

// ---------------------------------------------------------------- one block per ball
// The same descent with the samples resident in shared memory and all K iterations inside
// one block: per iteration a block argmax (ties to the lowest index) and the FP64 step by
// thread 0.  Used for batches of PURSEs (one block per PURSE and ball).
constexpr int kGgdBlockThreads = 512;

template <typename T, int MODE>
__device__ void ggd_block(const T* __restrict__ x, int n, int K, double* result, int32_t* f_out, int32_t* fstar, T* xs) {
  static_assert(sizeof(T) == 4, "the packed reduction below takes FP32 keys");
  constexpr int D = MODE == 0 ? 4 : 3;
  __shared__ double c[4];
  __shared__ double wkey[kGgdBlockThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = tid; k < n * D; k += blockDim.x) xs[k] = x[k];
  if (tid == 0) {
    if (MODE == 0) {
      const Q4<double> q0 = qnormalize(Q4<double>{(double)x[0], (double)x[1], (double)x[2], (double)x[3]});
      c[0] = q0.w, c[1] = q0.x, c[2] = q0.y, c[3] = q0.z;
    } else {
      c[0] = x[0], c[1] = x[1], c[2] = x[2], c[3] = 0.0;
    }
  }
  __syncthreads();
  for (int k = 1; k <= K + 1; ++k) {  // k = K + 1: final pass for the radius
    const T c0 = T(c[0]), c1 = T(c[1]), c2 = T(c[2]), c3 = T(c[3]);
    T bkt = T(-1);
    int bi = INT_MAX;
    for (int i = tid; i < n; i += blockDim.x) {
      T key;
      if (MODE == 0) {
        key = rot_key(c0, c1, c2, c3, xs + 4 * i);
      } else {
        const T* pp = xs + 3 * i;
        const T dx = pp[0] - c0, dy = pp[1] - c1, dz = pp[2] - c2;
        key = dx * dx + dy * dy + dz * dz;
      }
      if (key > bkt) bkt = key, bi = i;
    }
    // (key bits, complement of the index) in 64 bits, as in ggd_iter: the farthest sample with ties to
    // the lowest index, reduced with integer operations only
    const bool has = bi != INT_MAX;
    const uint32_t kb = has ? __float_as_uint(float(bkt)) : 0u;
    const uint32_t mk = __reduce_max_sync(kFullMask, kb);
    const uint32_t mi = __reduce_max_sync(kFullMask, has && kb == mk ? ~(uint32_t)bi : 0u);
    unsigned long long* wpk = reinterpret_cast<unsigned long long*>(wkey);
    if (lane == 0) wpk[warp] = ((unsigned long long)mk << 32) | mi;
    __syncthreads();
    if (tid == 0) {
      unsigned long long b = wpk[0];
      for (int w2 = 1; w2 < (int)(blockDim.x / 32); ++w2) b = wpk[w2] > b ? wpk[w2] : b;
      bi = b == 0ull ? 0 : (int)~(uint32_t)b;
      if (MODE == 0) {
        const T* qs = x + 4 * (size_t)bi;
        const Q4<double> cq{c[0], c[1], c[2], c[3]};
        const Q4<double> qf = qnormalize(Q4<double>{(double)qs[0], (double)qs[1], (double)qs[2], (double)qs[3]});
        const RelRot r = rel_rot(cq, qf);
        if (k <= K) {
          const Q4<double> cn = slerp_step(cq, r, k);
          c[0] = cn.w, c[1] = cn.x, c[2] = cn.y, c[3] = cn.z;
        } else {
          result[0] = cq.w, result[1] = cq.x, result[2] = cq.y, result[3] = cq.z;
          result[7] = r.th;
        }
      } else {
        const T* pp = x + 3 * (size_t)bi;
        if (k <= K) {
          const double rk = 1.0 / k;  // the same arithmetic as the single-PURSE ball
          for (int d = 0; d < 3; ++d) c[d] = c[d] + ((double)pp[d] - c[d]) * rk;
        } else {
          const double dx = (double)pp[0] - c[0], dy = (double)pp[1] - c[1], dz = (double)pp[2] - c[2];
          result[4] = c[0], result[5] = c[1], result[6] = c[2];
          result[8] = sqrt(dx * dx + dy * dy + dz * dz);
        }
      }
      if (k <= K && f_out) f_out[k - 1] = bi;
      if (k > K && fstar) *fstar = bi;
    }
    __syncthreads();
  }
}

// Batch: block (p, ball) with ball 0 = rotation (dS_R samples), 1 = translation (3D-3D: dS_R
// samples, 2D-3D: dS_t samples).  farthest: n_purses x 2K (rotation then translation sequence).
__global__ void __launch_bounds__(kGgdBlockThreads)
    ggd_batch_kernel(const __grid_constant__ BatchArgs b, int K, double* results, int32_t* farthest) {
  extern __shared__ __align__(16) unsigned char ggd_smem[];
  const int p = blockIdx.x >> 1, ball = blockIdx.x & 1;
  const size_t off = (size_t)p * b.n_samples;
  int32_t* f = farthest ? farthest + (size_t)p * 2 * K + ball * K : nullptr;
  int32_t* fs = b.fstar ? b.fstar + 2 * (size_t)p + ball : nullptr;
  if (ball == 0) {
    ggd_block<float, 0>(b.q_rot + 4 * off, b.n_samples, K, results + 9 * (size_t)p, f, fs,
                        reinterpret_cast<float*>(ggd_smem));
  } else {
    const float* t = (b.info[p].kind == 0 && !b.tr3d ? b.t_rot : b.t_tr) + 3 * off;
    ggd_block<float, 1>(t, b.n_samples, K, results + 9 * (size_t)p, f, fs, reinterpret_cast<float*>(ggd_smem));
  }
}

cudaError_t launch_megb_batch(const BatchArgs& b, int n_iters, double* d_results, int32_t* d_farthest,
                              cudaStream_t st) {
  const size_t smem = (size_t)b.n_samples * 4 * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(ggd_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  ggd_batch_kernel<<<2 * b.n_purses, kGgdBlockThreads, smem, st>>>(b, n_iters, d_results, d_farthest);
  return cudaGetLastError();
}

// Batched adjoint: block p runs both sweeps of PURSE p (warp 0 rotation, warp 1 translation)
// with the accumulators in shared memory, and writes its rows of the CSR gradients
// (grad_obs rows x 3, the third column 0 for 2D-3D; grad_radii rows).
__global__ void __launch_bounds__(64)
    batch_adjoint_kernel(const __grid_constant__ BatchArgs b, int K, const int32_t* far, const double* results,
                         const double* g, Q4<double>* cs, double* gy, double* gr) {
  extern __shared__ __align__(16) unsigned char adj_smem[];
  const int p = blockIdx.x;
  const BatchPurseInfo in = b.info[p];
  const int n = in.n, dim = in.kind == 1 ? 2 : 3;
  const size_t off = (size_t)p * b.n_samples;
  double* acc = reinterpret_cast<double*>(adj_smem);
  double* ly = acc + 2 * n * (dim + 1);  // local gradient rows before the CSR write
  double* lr = ly + n * dim;
  const bool tr = in.kind == 1 || b.tr3d;
  const float* t = (tr ? b.t_tr : b.t_rot) + 3 * off;
  const float* snap_t = (tr ? b.snap_tr : b.snap_rot) + (size_t)kSnapStride * off;
  adjoint_both<float>(b.q_rot + 4 * off, b.snap_rot + (size_t)kSnapStride * off, b.n_samples, t, snap_t, b.n_samples,
                      K, far + (size_t)p * 2 * K, b.fstar + 2 * (size_t)p, results + 9 * (size_t)p,
                      g + 9 * (size_t)p, cs + (size_t)p * (K + 1), n, dim, acc, ly, lr, b.status);
  __syncthreads();
  const int o = in.table_off / 2;  // first keypoint of PURSE p (tables hold 2 rows per keypoint)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    gy[3 * (size_t)(o + i)] = ly[dim * i];
    gy[3 * (size_t)(o + i) + 1] = ly[dim * i + 1];
    gy[3 * (size_t)(o + i) + 2] = dim == 3 ? ly[dim * i + 2] : 0.0;
    gr[o + i] = lr[i];
  }
}

cudaError_t launch_batch_backward(const BatchArgs& b, int n_iters, const int32_t* d_far, const double* d_results,
                                  const double* d_grad_results, void* d_cs, double* d_grad_obs, double* d_grad_radii,
                                  cudaStream_t st) {
  const size_t smem = (size_t)b.nmax * (2 * 4 + 4) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(batch_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  batch_adjoint_kernel<<<b.n_purses, 64, smem, st>>>(b, n_iters, d_far, d_results, d_grad_results,
                                                       reinterpret_cast<Q4<double>*>(d_cs), d_grad_obs, d_grad_radii);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- allocation-free variant
// megb_solve_noalloc runs the same kernels as megb_solve, but its scratch (ball state,
// per-block partial maxima, farthest-sample sequence) lives in one file-scope device array
// instead of handle-owned cudaMalloc memory.  Limits: at most kNoAllocMaxIters GGD
// iterations; the grid is capped at kNoAllocMaxBlocks blocks.
constexpr int kNoAllocMaxIters = 4096;
constexpr int kNoAllocMaxBlocks = 512;
constexpr size_t kNoAllocStateBytes = 256;
constexpr size_t kNoAllocBytes = 65536;
static_assert(sizeof(MegbState) <= kNoAllocStateBytes, "state slot too small");
static_assert(kNoAllocStateBytes + 2 * kNoAllocMaxBlocks * sizeof(Part) + 2 * kNoAllocMaxIters * sizeof(int32_t) <=
                  kNoAllocBytes,
              "no-alloc scratch too small");

// Every GPU that loads the library holds these 64 KiB until the process exits.
static __device__ __align__(256) unsigned char g_megb_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
static int g_noalloc_sms[kNoAllocMaxDevices] = {};

// Device address of the static scratch on the current device (looked up once per device and
// cached; the cache assumes the device's primary context lives as long as the process, i.e. no
// cudaDeviceReset between calls, after which the module and its array are loaded anew).
static cudaError_t noalloc_scratch(void** ptr, int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_megb_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
    g_noalloc_sms[dev] = n;
  }
  *ptr = g_noalloc_ptr[dev];
  *sms = g_noalloc_sms[dev];
  return cudaSuccess;
}

template <typename T>
static cudaError_t launch_megb_noalloc_t(int sms, int n_iters, const T* q, int nq, const T* t, int nt, double* result,
                                         int32_t* f_out, void* scratch, cudaStream_t st) {
  MegbState* s = reinterpret_cast<MegbState*>(scratch);
  Part* parts = reinterpret_cast<Part*>(reinterpret_cast<char*>(scratch) + kNoAllocStateBytes);
  int32_t* f_int = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(parts) + 2 * kNoAllocMaxBlocks * sizeof(Part));
  const long cap = 4L * sms < kNoAllocMaxBlocks ? 4L * sms : kNoAllocMaxBlocks;
  megb_init<T><<<1, 32, 0, st>>>(q, nq, t, nt, s);  // also zeroes the completion counters
  megb_zero_result<<<1, 32, 0, st>>>(result, nq == 0, nt == 0);
  if (nq > 0) {
    const long want = ((long)nq + kMegbThreads * 4 - 1) / (kMegbThreads * 4);
    const int g = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    for (int k = 1; k <= n_iters; ++k)
      ggd_step<T, 0><<<g, kMegbThreads, 0, st>>>(q, nq, s, parts, k, n_iters, 1, f_int, f_out, result);
    ggd_step<T, 0><<<g, kMegbThreads, 0, st>>>(q, nq, s, parts, 0, n_iters, 1, f_int, f_out, result);
  }
  if (nt > 0) {
    const long want = ((long)nt + kMegbThreads * 4 - 1) / (kMegbThreads * 4);
    const int g = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    Part* parts_t = parts + kNoAllocMaxBlocks;
    for (int k = 1; k <= n_iters; ++k)
      ggd_step<T, 1><<<g, kMegbThreads, 0, st>>>(t, nt, s, parts_t, k, n_iters, 1, f_int + n_iters,
                                                  f_out ? f_out + n_iters : nullptr, result);
    ggd_step<T, 1><<<g, kMegbThreads, 0, st>>>(t, nt, s, parts_t, 0, n_iters, 1, f_int + n_iters, nullptr, result);
  }
  return cudaGetLastError();
}

}  // namespace purse

extern "C" purse_status megb_solve_noalloc(int precision, int n_iters, const void* d_q, int n_rot, const void* d_t,
                                           int n_tr, double* d_result, int32_t* d_farthest, purse_stream_t stream) {
  using namespace purse;
  if (precision != 0 && precision != 1) {
    set_error("megb_solve_noalloc: precision must be 0 or 1");
    return PURSE_ERR_ARG;
  }
  if (n_iters < 1 || n_iters > kNoAllocMaxIters) {
    set_error("megb_solve_noalloc: n_iters must be in [1, 4096] (size of the static scratch)");
    return PURSE_ERR_ARG;
  }
  if (n_rot > kMaxBallSamples || n_tr > kMaxBallSamples) {
    set_error("megb_solve_noalloc: more than 2^31 - 2^21 samples (32-bit sample indices)");
    return PURSE_ERR_ARG;
  }
  if (n_rot < 0 || n_tr < 0 || (n_rot > 0 && !d_q) || (n_tr > 0 && !d_t) || !d_result) {
    set_error("megb_solve_noalloc: negative sample count or NULL buffer");
    return PURSE_ERR_ARG;
  }
  if (fault_at("launch")) return injected_fault("launch", "megb_solve_noalloc");
  void* scratch = nullptr;
  int sms = 0;
  cudaError_t e = noalloc_scratch(&scratch, &sms);
  if (e != cudaSuccess) return cuda_fail(e, "megb_solve_noalloc (static scratch address)");
  cudaStream_t st = (cudaStream_t)stream;
  e = precision == 0 ? launch_megb_noalloc_t<float>(sms, n_iters, (const float*)d_q, n_rot, (const float*)d_t, n_tr,
                                                    d_result, d_farthest, scratch, st)
                     : launch_megb_noalloc_t<double>(sms, n_iters, (const double*)d_q, n_rot, (const double*)d_t,
                                                     n_tr, d_result, d_farthest, scratch, st);
  return e == cudaSuccess ? PURSE_OK : cuda_fail(e, "megb_solve_noalloc");
}
