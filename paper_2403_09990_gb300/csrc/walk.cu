// Fused strategic random walk (Section IV Step II; Alg. 2/3 for the dS_R
// sampler, Alg. 4/5 for the dS_t sampler), one warp per walk.
//
// Per iteration of a walk:
//   1. constraint order: the margins of the current pose are sorted across
//      the warp (most nearly violated first) and the warp's tables
//      (Y_i = R* Z_i, observations, perturbation-phase constants) are
//      written in that order into its shared-memory slab;
//   2. perturbation + dist (eq. 11): lane l owns the pairs of perturbations
//      j = 2b, 2b + 1, b = l + 32 P, drawn from one Philox block each, and
//      evaluates d_j = min_i (r_i - |g_i|) for both at once (paired FP32
//      instructions), ceil(N_P / 64) pairs per lane;
//   3. top_k_indices: each lane sorts its own keys once, then N_P* rounds of
//      a warp max (REDUX) pop the best head; ties go to the lower j;
//   4. step ladder: candidates (k, m) are laid out lane = m_local * N_P* + k
//      over chunks of 32 / N_P* rungs; in_purse is evaluated division-free
//      two constraints at a time (paired FP32), and a chunk is left as soon
//      as a warp vote after a pair shows that every candidate has violated
//      one (in_purse is a conjunction, so the order and the early exit do
//      not change it);
//      the first chunk with a feasible candidate ends the ladder and __ffs
//      of the ballot gives m0 (smallest m) then k0 (best-ranked k);
//   5. update (R*, t*).
// Factoring used on the perturbation phase (same values as the per-pose
// transform of Alg. 3, fewer operations):
//   dS_R, 2D-3D: K(R* Z_i + t* + delta_j) = Q_i + K delta_j
//   dS_t, 2D-3D: K(R_p R* Z_i + t*)       = (K R_p) Y_i + K t*
// and the same without K (minus b_i) for 3D-3D.
// Noise matrices (eq. 4, LAM): the residual g_i enters every norm as U_i g_i
// with Lambda_i = U_i^T U_i (upper triangular); for 2D-3D U_i acts on the
// division-free pixel residual (e_x, e_y), which P_z > 0 only scales.
#include <cfloat>
#include <cstdio>

#include "dev.cuh"
#include "internal.h"

namespace purse {

constexpr int kWalkWarps = 8;
constexpr int kWalkThreads = kWalkWarps * 32;
constexpr size_t kMaxSmemPerBlock = 227 * 1024;

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

// Constraint table in shared memory: rows [0, N) (a or Z, r), [N, 2N) (b or z, r^2); with noise
// matrices then two rows per constraint of U_i (3D: u00 u01 u02 u11 | u12 u22; 2D: u00 u01 u11).
template <typename T>
__host__ __device__ inline size_t walk_table_bytes(int n, bool lam = false) {
  return align_up((lam ? 16 : 8) * (size_t)n * sizeof(T), 128);
}

// Pairs per constraint row of the slab tables D and L: 8, or 14 with the U_i entries (slots 8-13;
// 14 rather than 16 keeps rows i and i + 1 in different shared-memory banks).
template <bool LAM>
constexpr int kRow = LAM ? 14 : 8;

template <typename K>
__device__ __forceinline__ void cas_desc(K& a, K& b) {
  const K hi = a > b ? a : b, lo = a > b ? b : a;
  a = hi, b = lo;
}
// Sorting network for 8 keys, descending.
template <typename K>
__device__ __forceinline__ void sort8_desc(K (&k)[8]) {
  cas_desc(k[0], k[1]); cas_desc(k[2], k[3]); cas_desc(k[4], k[5]); cas_desc(k[6], k[7]);
  cas_desc(k[0], k[2]); cas_desc(k[1], k[3]); cas_desc(k[4], k[6]); cas_desc(k[5], k[7]);
  cas_desc(k[1], k[2]); cas_desc(k[5], k[6]); cas_desc(k[0], k[4]); cas_desc(k[3], k[7]);
  cas_desc(k[1], k[5]); cas_desc(k[2], k[6]);
  cas_desc(k[1], k[4]); cas_desc(k[3], k[6]);
  cas_desc(k[2], k[4]); cas_desc(k[3], k[5]);
  cas_desc(k[3], k[4]);
}

// Per-warp view of the shared-memory slab (constraint order of the current iteration).
//  D[r][0..7]  perturbation phase, constraint r broadcast to both halves of a pair:
//              dS_R: (Q_x, Q_y, Q_z, r_i) with Q = K(R* Z + t*) or R* a + t* - b;
//              dS_t: (Y_x, Y_y, Y_z, r_i) with Y = R* Z;
//              then 2D-3D: (-u, -v), 3D-3D dS_t: (t* - b); with noise matrices U_i in slots 8-13.
//  L[q][0..7]  ladder, constraints 2q and 2q + 1 in the two halves of a pair:
//              (Y_x, Y_y, Y_z), then 2D-3D: (-u, -v, -r^2), 3D-3D: (-b_x, -b_y, -b_z, -r^2);
//              with noise matrices U_i in slots 8-13.
//  P[j]        perturbation j: translation offset (dS_R) or unit quaternion (dS_t)
//  E[4m..]     ladder rung m: quaternion and rows of (K) E_m (dS_R) or s_m v (dS_t)
//  S           walk state of FP32 walks: q*, t* as double-float pairs
template <typename T>
struct Slab {
  P2<T>* D;
  P2<T>* L;
  T4<T>* P;
  T4<T>* E;
  typename KeyOf<T>::type* key;
  int* J;
  double* S;
};

__host__ __device__ inline int ladder_pairs(int n) { return (n + 1) / 2; }

// Slab::S of FP32 walks: the pose as double-float pairs (floats 0-3 q* hi, 4-7 q* lo, 8-10 t* hi,
// 11-13 t* lo).
constexpr int kStateDoubles = 8;

template <typename T>
__host__ __device__ inline size_t walk_slab_bytes2(int n, int n_perturb, int n_steps, bool lam = false) {
  const size_t p2 = 2 * sizeof(T), t4 = 4 * sizeof(T), row = lam ? 14 : 8;
  const size_t bytes = row * (size_t)n * p2 + row * (size_t)ladder_pairs(n) * p2 + (n_perturb + 4 * (size_t)n_steps) * t4 +
                       (size_t)n_perturb * sizeof(typename KeyOf<T>::type) + 32 * sizeof(int);
  return align_up(align_up(bytes, 8) + kStateDoubles * sizeof(double), 128);
}

template <typename T, bool LAM = false>
__device__ __forceinline__ Slab<T> carve(unsigned char* base, int N, int NP, int NT) {
  Slab<T> s;
  s.D = reinterpret_cast<P2<T>*>(base);
  s.L = s.D + kRow<LAM> * N;
  s.P = reinterpret_cast<T4<T>*>(s.L + kRow<LAM> * ladder_pairs(N));
  s.E = s.P + NP;
  s.key = reinterpret_cast<typename KeyOf<T>::type*>(s.E + 4 * NT);
  s.J = reinterpret_cast<int*>(s.key + NP);
  s.S = reinterpret_cast<double*>(align_up(reinterpret_cast<size_t>(s.J + 32), 8));
  return s;
}

// Perturbation phase over NPAIR pairs per lane, starting at pair pb: pair P of this lane holds
// perturbations j = 2 b, 2 b + 1 with b = 32 (pb + P) + (lane >> sh), the two points of block 0 of
// stream (phase, b, it, w).  sh > 0 (the ragged last pass, NPAIR = 1): the 2^sh lanes of a pair
// split its constraints (i = sub, sub + 2^sh, ...) and combine their minima by shuffles -- the
// minimum is exact, so the keys are those of one lane taking every constraint.  Writes the keys of
// every valid j.
// ZCHK = false (dS_t, 2D-3D): the caller has bounded P_z away from 0 for every constraint and
// perturbation, so the cheirality minimum is not tracked.
template <typename T, int KIND, int SAMPLER, int NPAIR, bool ZCHK = true, bool LAM = false, class RK>
__device__ __forceinline__ void dist_pass(const RK& rk, int it, int w, const Slab<T>& sl, int N, int NP, int lane,
                                          int pb, T r_pert, const V3<T>& t, T fx, T fy, T cx, T cy, T qzmin,
                                          int sh = 0) {
  using T2 = P2<T>;
  const int pl = lane >> sh, sub = lane & ((1 << sh) - 1), S = 1 << sh;
  T2 dmin[NPAIR], zmin[NPAIR];
  T2 Dx[NPAIR], Dy[NPAIR], Dz[NPAIR];             // dS_R: translation offsets in P units
  T2 A[SAMPLER == 1 ? NPAIR : 1][9];              // dS_t: (K) R_p per slot
#pragma unroll
  for (int p = 0; p < NPAIR; ++p) {
    T dx[2], dy[2], dz[2];
    const int b = 32 * (pb + p) + pl;
    uint4 wd = make_uint4(0u, 0u, 0u, 0u);
    if (2 * b < NP)
      wd = philox4x32_10_rk(make_uint4(0u, ((SAMPLER == 0 ? kPhaseRPerturb : kPhaseTPerturb) << 24) | (uint32_t)b,
                                       (uint32_t)it, (uint32_t)w),
                            rk);
    if constexpr (SAMPLER == 1) {
      // both rotations of the block at once on paired lanes: (K) R_p for the constraint loop
      T2 qw, qx, qy, qz;
      hatbox_quat2<T>(wd, r_pert, qw, qx, qy, qz);
      qmat2<T>(qw, qx, qy, qz, A[p]);
      if (KIND == 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          A[p][c] = fma2(dup(fx), A[p][c], mul2(dup(cx), A[p][6 + c]));
          A[p][3 + c] = fma2(dup(fy), A[p][3 + c], mul2(dup(cy), A[p][6 + c]));
        }
      }
      if (2 * b < NP) sl.P[2 * b] = T4<T>{qw.x, qx.x, qy.x, qz.x};
      if (2 * b + 1 < NP) sl.P[2 * b + 1] = T4<T>{qw.y, qx.y, qy.y, qz.y};
      Dx[p] = Dy[p] = Dz[p] = dup(T(0));
      dmin[p] = dup(inf<T>());
      zmin[p] = dup(inf<T>());
      continue;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // dS_R: the translation offsets K delta_j
      const int j = 2 * b + h;
      dx[h] = dy[h] = dz[h] = T(0);
      if (j < NP) {
        T ux, uy, uz;
        hatbox_point<T>(h ? wd.z : wd.x, h ? wd.w : wd.y, ux, uy, uz);
        const V3<T> dl{r_pert * ux, r_pert * uy, r_pert * uz};
        sl.P[j] = T4<T>{dl.x, dl.y, dl.z, T(0)};
        if (KIND == 1) {
          dx[h] = fx * dl.x + cx * dl.z, dy[h] = fy * dl.y + cy * dl.z, dz[h] = dl.z;
        } else {
          dx[h] = dl.x, dy[h] = dl.y, dz[h] = dl.z;
        }
      }
    }
    Dx[p] = pr(dx[0], dx[1]), Dy[p] = pr(dy[0], dy[1]), Dz[p] = pr(dz[0], dz[1]);
    dmin[p] = dup(inf<T>());
    zmin[p] = dup(inf<T>());
  }
  const T2 neg1 = dup(T(-1)), tiny2 = dup(tiny<T>());
  T2 c0x = dup(T(0)), c0y = c0x, c0z = c0x;
  if (SAMPLER == 1 && KIND == 1) c0x = dup(fx * t.x + cx * t.z), c0y = dup(fy * t.y + cy * t.z), c0z = dup(t.z);
  constexpr int kUnroll = 2;
#pragma unroll kUnroll
  for (int i = sub; i < N; i += S) {
    const T2* Di = sl.D + kRow<LAM> * i;
    const T2 d0 = Di[0], d1 = Di[1], d2 = Di[2], rr = Di[3];
    T2 d4, d5, d6, u0, u1, u2, u3, u4, u5;
    if (KIND == 1 || SAMPLER == 1) d4 = Di[4], d5 = Di[5];
    if (KIND == 0 && SAMPLER == 1) d6 = Di[6];
    if constexpr (LAM) {
      u0 = Di[8], u1 = Di[9], u2 = Di[10];
      if (KIND == 0) u3 = Di[11], u4 = Di[12], u5 = Di[13];
    }
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
      T2 Px, Py, Pz;
      if constexpr (SAMPLER == 0) {
        Px = add2(d0, Dx[p]), Py = add2(d1, Dy[p]), Pz = add2(d2, Dz[p]);
      } else {
        const T2 bx = KIND == 1 ? c0x : d4, by = KIND == 1 ? c0y : d5, bz = KIND == 1 ? c0z : d6;
        Px = fma2(A[p][0], d0, fma2(A[p][1], d1, fma2(A[p][2], d2, bx)));
        Py = fma2(A[p][3], d0, fma2(A[p][4], d1, fma2(A[p][5], d2, by)));
        Pz = fma2(A[p][6], d0, fma2(A[p][7], d1, fma2(A[p][8], d2, bz)));
      }
      T2 s2, qq;
      if (KIND == 1) {
        T2 ex = fma2(d4, Pz, Px), ey = fma2(d5, Pz, Py);
        if constexpr (LAM) ex = fma2(u1, ey, mul2(u0, ex)), ey = mul2(u2, ey);
        s2 = fma2(ey, ey, mul2(ex, ex));
        qq = fma2(s2, mul2(Pz, Pz), tiny2);
        if (SAMPLER == 1 && ZCHK) zmin[p] = min2(zmin[p], Pz);
      } else {
        if constexpr (LAM) {
          const T2 ex = fma2(u2, Pz, fma2(u1, Py, mul2(u0, Px))), ey = fma2(u4, Pz, mul2(u3, Py)), ez = mul2(u5, Pz);
          s2 = fma2(ez, ez, fma2(ey, ey, mul2(ex, ex)));
        } else {
          s2 = fma2(Pz, Pz, fma2(Py, Py, mul2(Px, Px)));
        }
        qq = add2(s2, tiny2);
      }
      T2 m;  // r - |e| (2D-3D: |e| / P_z)
      if constexpr (SAMPLER == 0)
        m = fma2(pr(-s2.x, -s2.y), rsq2(qq), rr);
      else
        m = fma2(mul2(s2, rsq2(qq)), neg1, rr);
      dmin[p] = min2(dmin[p], m);
    }
  }
  for (int o = 1; o < S; o <<= 1) {
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
      dmin[p] = min2(dmin[p], pr(__shfl_xor_sync(kFullMask, dmin[p].x, o), __shfl_xor_sync(kFullMask, dmin[p].y, o)));
      if (SAMPLER == 1 && KIND == 1 && ZCHK)
        zmin[p] = min2(zmin[p], pr(__shfl_xor_sync(kFullMask, zmin[p].x, o), __shfl_xor_sync(kFullMask, zmin[p].y, o)));
    }
  }
#pragma unroll
  for (int p = 0; p < NPAIR; ++p) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * (32 * (pb + p) + pl) + h;
      if (j < NP && sub == 0) {
        T d = h ? dmin[p].y : dmin[p].x;
        if (KIND == 1) {
          // dS_R: P_z = Q_z,i + D_z,j and rounding is monotone, so min_i P_z = min_i Q_z,i + D_z,j
          const T zm = SAMPLER == 0 ? qzmin + (h ? Dz[p].y : Dz[p].x) : ZCHK ? (h ? zmin[p].y : zmin[p].x) : T(1);
          if (!(zm > T(0))) d = -inf<T>();
        }
        sl.key[j] = orderable(d);
      }
    }
  }
}

// top_k_indices of Alg. 3/5 (ties to the lower j): lane l holds keys j = l + 32 s, s < NS (the low
// three bits of a key encode 7 - s), sorts them, and K rounds of a warp maximum pop the best head;
// the winners' indices go to sl.J in rank order.
template <typename Key, int NS, typename T>
__device__ __forceinline__ void top_k(const Slab<T>& sl, int NP, int K, int lane) {
  Key kk[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int j = lane + 32 * s;
    kk[s] = j < NP ? ((sl.key[j] & ~Key(7)) | Key(7 - s)) : Key(0);
  }
  if constexpr (NS == 8) {
    sort8_desc(kk);
  } else {
#pragma unroll
    for (int a = 0; a < NS - 1; ++a)
#pragma unroll
      for (int b = 0; b < NS - 1 - a; ++b) cas_desc(kk[b], kk[b + 1]);
  }
  for (int r = 0; r < K; ++r) {
    const Key mx = warp_max_key(kk[0]);
    const unsigned bal = __ballot_sync(kFullMask, kk[0] == mx);
    const int wl = __ffs(bal) - 1;
    if (lane == wl) {
#pragma unroll
      for (int s = 0; s < NS - 1; ++s) kk[s] = kk[s + 1];
      kk[NS - 1] = Key(0);
    }
    if (lane == 0) sl.J[r] = wl + 32 * (7 - (int)(mx & Key(7)));
  }
}

// in_purse of one ladder candidate against constraint pair Lq (two constraints on the paired
// lanes): the division-free value c (<= 0 inside) of both halves folded into the running maximum
// cmax, and for 2D-3D (Z) P_z into the running minimum zmin.
template <typename T, int KIND, bool Z, bool LAM>
__device__ __forceinline__ void ladder_pair(const P2<T>* Lq, const P2<T> (&M2)[9], P2<T> bx, P2<T> by, P2<T> bz,
                                            P2<T>& cmax, P2<T>& zmin) {
  using T2 = P2<T>;
  const T2 yx = Lq[0], yy = Lq[1], yz = Lq[2], o3 = Lq[3], o4 = Lq[4], o5 = Lq[5];
  const T2 Px = fma2(M2[0], yx, fma2(M2[1], yy, fma2(M2[2], yz, bx)));
  const T2 Py = fma2(M2[3], yx, fma2(M2[4], yy, fma2(M2[5], yz, by)));
  const T2 Pz = fma2(M2[6], yx, fma2(M2[7], yy, fma2(M2[8], yz, bz)));
  T2 c;
  if (KIND == 1) {
    T2 ex = fma2(o3, Pz, Px), ey = fma2(o4, Pz, Py);
    if constexpr (LAM) ex = fma2(Lq[9], ey, mul2(Lq[8], ex)), ey = mul2(Lq[10], ey);
    c = fma2(o5, mul2(Pz, Pz), fma2(ey, ey, mul2(ex, ex)));
    if (Z) zmin = min2(zmin, Pz);
  } else {
    T2 ex = add2(Px, o3), ey = add2(Py, o4), ez = add2(Pz, o5);
    if constexpr (LAM) {
      const T2 gx = fma2(Lq[10], ez, fma2(Lq[9], ey, mul2(Lq[8], ex)));
      const T2 gy = fma2(Lq[12], ez, mul2(Lq[11], ey));
      ez = mul2(Lq[13], ez), ex = gx, ey = gy;
    }
    c = add2(fma2(ez, ez, fma2(ey, ey, mul2(ex, ex))), Lq[6]);
  }
  cmax = max2(cmax, c);
}

// A candidate survives the pairs seen so far while every value is <= 0 (and, 2D-3D, every P_z > 0).
template <typename T, int KIND, bool Z>
__device__ __forceinline__ bool ladder_ok(P2<T> cmax, P2<T> zmin) {
  return fmax(cmax.x, cmax.y) <= T(0) && (KIND == 0 || !Z || fmin(zmin.x, zmin.y) > T(0));
}

// in_purse of one ladder chunk (one candidate per lane) over the constraint pairs q0 .. NQ - 1, a warp
// vote after each pair leaving the chunk once every candidate has violated a constraint.  The
// constraints come in ascending margin at the current pose, so most candidates die on the first
// pairs; a vote per pair measured faster than one per two or more.  The result of a pair range
// started after pairs that a candidate passed equals that of the whole range (running max / min).
// Z: track the cheirality minimum (2D-3D; off when the caller has bounded P_z away from 0).
template <typename T, int KIND, bool Z, bool LAM = false>
__device__ __forceinline__ void ladder_scan(const P2<T>* L, int q0, int NQ, int N, const P2<T> (&M2)[9], P2<T> bx,
                                            P2<T> by, P2<T> bz, P2<T>& cmax, P2<T>& zmin, bool& alive, int& done) {
  for (int qi = q0; qi < NQ; ++qi) {
    ladder_pair<T, KIND, Z, LAM>(L + kRow<LAM> * qi, M2, bx, by, bz, cmax, zmin);
    done = min(N, 2 * (qi + 1));
    alive = alive && ladder_ok<T, KIND, Z>(cmax, zmin);
    if (!__any_sync(kFullMask, alive)) break;
  }
}

// Everything one walk needs about its PURSE and parameters (kept in registers).
template <typename T>
struct WalkCtx {
  int N, NP, K, NT, mc, n_iter;
  T fx, fy, cx, cy, r_pert;
  T rho_max;  // largest model-point radius (bounds P_z from below for the cheirality test)
  double omega0, v0, gamma;
  T om0, vv0, gam;  // the same in T (converted once per block)
  const WalkStats* st;
  const double* seed_data;
  int s0;
  uint32_t key0, key1;
  T* out_q;
  T* out_t;
  int16_t* trace;
  T* out_snap;  // NULL: no snap; else kSnapStride values per walk
  const double* tab64;  // the PURSE's FP64 constraint table (global memory), read by the snap
  const double* kd;     // fx, fy, cx, cy in FP64 (global or parameter memory), read by the snap
  const double* ell64;  // noise factors U_i in FP64 (8 per constraint) or NULL, read by the snap
  int* status;
};

// Philox round keys from the kernel parameters (constant bank) or from memory.
struct RkParam {
  const WalkArgs& a;
  __device__ __forceinline__ uint32_t operator[](int i) const { return a.rk[i]; }
};
struct RkPtr {
  const uint32_t* p;
  __device__ __forceinline__ uint32_t operator[](int i) const { return p[i]; }
};

// Pose on the walk's last-move ray: rotation ray (Exp(tau d) R*, t*) for dS_R, translation ray
// (R*, t* + tau d) for dS_t.
template <typename T, int SAMPLER>
__device__ __forceinline__ void ray_pose(const Q4<T>& q, const V3<T>& t, const V3<T>& d, T tau, Q4<T>& qo, V3<T>& to) {
  if (SAMPLER == 0) {
    qo = qnormalize(qmul(qexp(V3<T>{tau * d.x, tau * d.y, tau * d.z}), q));
    to = t;
  } else {
    qo = q;
    to = V3<T>{t.x + tau * d.x, t.y + tau * d.y, t.z + tau * d.z};
  }
}

// in_purse of one pose, constraints spread over the lanes (warp-uniform result).
template <typename T, int KIND>
__device__ __forceinline__ bool pose_in_purse(const T4<T>* tab, int N, const M3<T>& R, const V3<T>& t, T fx, T fy,
                                              T cx, T cy, int lane) {
  bool ok = true;
  for (int i = lane; i < N; i += 32) {
    const T4<T> mz = tab[i], ob = tab[N + i];
    const V3<T> X = mul(R, V3<T>{mz.x, mz.y, mz.z}) + t;
    if (KIND == 1) {
      const T Pz = X.z, ex = fx * X.x + cx * X.z - ob.x * Pz, ey = fy * X.y + cy * X.z - ob.y * Pz;
      const T rz = mz.w * Pz;
      ok = ok && Pz > T(0) && ex * ex + ey * ey - rz * rz <= T(0);
    } else {
      const T ex = X.x - ob.x, ey = X.y - ob.y, ez = X.z - ob.z;
      ok = ok && ex * ex + ey * ey + ez * ez - ob.w <= T(0);
    }
  }
  return __all_sync(kFullMask, ok);
}

// Boundary snap along the last-move ray (used to differentiate the balls): tau_hi = the
// smallest ladder value whose pose leaves S, bisection of [0, tau_hi] keeping the feasible end,
// j* = the constraint of smallest margin there (ties to the lower index).  Record (kSnapStride
// values): j* (-1: nothing left S along the ladder, pose unchanged), ray kind (0 rotation,
// 1 translation), direction (3), h'(tau*) = d|g_j*|/d tau, d|g_j*|/d y_j* (3; 2 used for 2D-3D).
//
// Rotation rays (dS_R) are evaluated in the walk precision.  Along a translation ray (dS_t) the
// residual of every constraint is affine in tau -- 3D-3D g(tau) = g0 + tau v; 2D-3D
// (e_x, e_y, P_z)(tau) = (e_x0, e_y0, P_z0) + tau (beta_x, beta_y, v_z) for the division-free pixel
// residual e = P_xy - z_i P_z -- so the base residuals and slopes are formed once, in FP64 from the
// FP64 table and pose, and the bisection steps only evaluate the affine model.  In FP32 a direct
// evaluation would subtract projected coordinates of hundreds of px to get residuals of a few px,
// and along the viewing ray of a 2D-3D PURSE that rounding moves the boundary by ~1e-6 m.
// U x for the upper-triangular noise factor U of a constraint (eq. 4): u = (u00 u01 u02 u11 u12 u22)
// in 3D, (u00 u01 u11) in 2D.
__device__ __forceinline__ V3<double> umul3(const double* u, const V3<double>& x) {
  return V3<double>{u[0] * x.x + u[1] * x.y + u[2] * x.z, u[3] * x.y + u[4] * x.z, u[5] * x.z};
}

template <typename T, int KIND, bool LAM>
__device__ __forceinline__ void snap_record(const WalkCtx<T>& c, int j, const Q4<double>& qs, const V3<double>& ts,
                                            const V3<double>& dir, int sampler, T* rec) {
  // In FP64 from the FP64 table and snapped pose: h' = d|g|/d tau is a difference of terms tens of
  // times larger when the ray grazes the boundary, and the adjoint divides by it.
  using D = double;
  const int N = c.N;
  const T4<D>* tab = reinterpret_cast<const T4<D>*>(c.tab64);
  const D fx = c.kd[0], fy = c.kd[1], cx = c.kd[2], cy = c.kd[3];
  const M3<D> R = qmat(qs);
  const T4<D> mz = tab[j], ob = tab[N + j];
  const V3<D> RA = mul(R, V3<D>{mz.x, mz.y, mz.z});
  const V3<D> X = RA + ts;
  // d|g|/de with e = -g: e / |e|, or Lambda e / |e|_Lambda = U^T (U e) / |U e| with noise matrices
  V3<D> wv, dy;  // d|g|/d(translation of the keypoint), d|g|/d y
  const double* u = LAM ? c.ell64 + 8 * (size_t)j : nullptr;
  if (KIND == 1) {
    const D Px = fx * X.x + cx * X.z, Py = fy * X.y + cy * X.z, Pz = X.z;
    const D e0 = Px / Pz - ob.x, e1 = Py / Pz - ob.y;
    D n0, n1;
    if (LAM) {
      const D f0 = u[0] * e0 + u[1] * e1, f1 = u[2] * e1;
      const D nrm = sqrt(f0 * f0 + f1 * f1);
      n0 = u[0] * f0 / nrm, n1 = (u[1] * f0 + u[2] * f1) / nrm;
    } else {
      const D nrm = sqrt(e0 * e0 + e1 * e1);
      n0 = e0 / nrm, n1 = e1 / nrm;
    }
    const V3<D> jn{n0 / Pz, n1 / Pz, -(Px * n0 + Py * n1) / (Pz * Pz)};
    wv = V3<D>{fx * jn.x, fy * jn.y, cx * jn.x + cy * jn.y + jn.z};
    dy = V3<D>{-n0, -n1, D(0)};
  } else {
    const V3<D> e = X - V3<D>{ob.x, ob.y, ob.z};
    if (LAM) {
      const V3<D> f = umul3(u, e);
      const V3<D> g{u[0] * f.x, u[1] * f.x + u[3] * f.y, u[2] * f.x + u[4] * f.y + u[5] * f.z};
      wv = (D(1) / sqrt(dot(f, f))) * g;
    } else {
      wv = (D(1) / sqrt(dot(e, e))) * e;
    }
    dy = D(-1) * wv;
  }
  const D dh = sampler == 0 ? dot(cross(RA, wv), dir) : dot(wv, dir);
  rec[0] = T(j), rec[1] = T(sampler), rec[2] = T(dir.x), rec[3] = T(dir.y), rec[4] = T(dir.z), rec[5] = T(dh);
  rec[6] = T(dy.x), rec[7] = T(dy.y), rec[8] = T(dy.z);
  for (int k = 9; k < kSnapStride; ++k) rec[k] = T(0);
}

// Smallest margin over the constraints spread across the lanes, ties to the lower index.
__device__ __forceinline__ int warp_argmin(double m, int i) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const double om = __shfl_xor_sync(kFullMask, m, o);
    const int oi = __shfl_xor_sync(kFullMask, i, o);
    if (om < m || (om == m && oi < i)) m = om, i = oi;
  }
  return i;
}

// (Exp(theta k) - I) for a unit axis k: sin(theta) [k]x + 2 sin^2(theta / 2) (k k^T - I), written
// without the cancellation of 1 - cos(theta) for small angles.
template <typename T>
__device__ __forceinline__ M3<T> exp_minus_identity(const V3<T>& k, T theta) {
  const T s = sin(theta), h = sin(T(0.5) * theta), c2 = T(2) * h * h;
  return M3<T>{{c2 * (k.x * k.x - T(1)), -s * k.z + c2 * k.x * k.y, s * k.y + c2 * k.x * k.z,
                s * k.z + c2 * k.x * k.y, c2 * (k.y * k.y - T(1)), -s * k.x + c2 * k.y * k.z,
                -s * k.y + c2 * k.x * k.z, s * k.x + c2 * k.y * k.z, c2 * (k.z * k.z - T(1))}};
}

// Rotation ray (Exp(tau omega) R*, t*): X_i(tau) = X_i(0) + (Exp(tau omega) - I) Y_i with
// Y_i = R* Z_i, so the residual is its value at tau = 0 (formed in FP64) plus an increment that
// is small near the sample, evaluated in the walk precision.  (q64, t64, w64) the FP64 pose and
// angular velocity, coef a free area of the warp's slab (10 N values).
template <typename T, int KIND, bool LAM>
__device__ __forceinline__ void snap_rotation(const WalkCtx<T>& c, const T4<T>* tab_s, const Q4<double>& q64,
                                              const V3<double>& t64, const V3<T>& wt, T* coef, Q4<T>& q, V3<T>& t,
                                              int w, int lane) {
  const V3<double> w64{double(wt.x), double(wt.y), double(wt.z)};
  constexpr int kS = LAM ? 16 : 10;  // coefficients per constraint
  using D = double;
  const int N = c.N;
  const T4<D>* tab = reinterpret_cast<const T4<D>*>(c.tab64);
  const D fx = c.kd[0], fy = c.kd[1], cx = c.kd[2], cy = c.kd[3];
  const M3<D> R = qmat(q64);
  // coef[kS i ..]: base residual (3: e_x, e_y, P_z or g), Y_i (3), cx - u, cy - v (2D-3D), r or r^2,
  // then with noise matrices the factor U_i (3 or 6 entries)
  for (int i = lane; i < N; i += 32) {
    const T4<D> mz = tab[i], ob = tab[N + i];
    const V3<D> Y = mul(R, V3<D>{mz.x, mz.y, mz.z});
    const V3<D> X = Y + t64;
    T* k = coef + kS * i;
    if (LAM)
      for (int e = 0; e < (KIND == 1 ? 3 : 6); ++e) k[9 + e] = T(c.ell64[8 * (size_t)i + e]);
    if (KIND == 1) {
      k[0] = T(fx * X.x + (cx - ob.x) * X.z), k[1] = T(fy * X.y + (cy - ob.y) * X.z), k[2] = T(X.z);
      k[6] = T(cx - ob.x), k[7] = T(cy - ob.y), k[8] = T(mz.w);
    } else {
      k[0] = T(X.x - ob.x), k[1] = T(X.y - ob.y), k[2] = T(X.z - ob.z);
      k[8] = T(ob.w);
    }
    k[3] = T(Y.x), k[4] = T(Y.y), k[5] = T(Y.z);
  }
  __syncwarp();
  const D wn = sqrt(dot(w64, w64));
  const V3<T> ax = wn > 0 ? V3<T>{T(w64.x / wn), T(w64.y / wn), T(w64.z / wn)} : V3<T>{T(1), T(0), T(0)};
  const T fxt = T(fx), fyt = T(fy), wnt = T(wn);
  auto residual = [&](const M3<T>& M, int i, T& ex, T& ey, T& ez) {
    const T* k = coef + kS * i;
    const V3<T> dX = mul(M, V3<T>{k[3], k[4], k[5]});
    if (KIND == 1) {
      ex = k[0] + fxt * dX.x + k[6] * dX.z, ey = k[1] + fyt * dX.y + k[7] * dX.z, ez = k[2] + dX.z;
      if (LAM) ex = k[9] * ex + k[10] * ey, ey = k[11] * ey;  // U (e_x, e_y); P_z untouched
    } else {
      ex = k[0] + dX.x, ey = k[1] + dX.y, ez = k[2] + dX.z;
      if (LAM) {
        const T gx = k[9] * ex + k[10] * ey + k[11] * ez, gy = k[12] * ey + k[13] * ez;
        ez = k[14] * ez, ex = gx, ey = gy;
      }
    }
  };
  auto inside = [&](T tau) {
    const M3<T> M = exp_minus_identity(ax, tau * wnt);
    bool ok = true;
    for (int i = lane; i < N; i += 32) {
      T ex, ey, ez;
      residual(M, i, ex, ey, ez);
      const T r = coef[kS * i + 8];
      if (KIND == 1) {
        const T rz = r * ez;
        ok = ok && ez > T(0) && ex * ex + ey * ey - rz * rz <= T(0);
      } else {
        ok = ok && ex * ex + ey * ey + ez * ez - r <= T(0);
      }
    }
    return __all_sync(kFullMask, ok);
  };
  T hi = T(-1);
  for (int m = c.NT - 1; m >= 0 && hi < T(0); --m) {
    T sm = T(1);
    for (int k = 0; k < m; ++k) sm *= c.gam;
    if (!inside(sm)) hi = sm;
  }
  T* rec = c.out_snap + (size_t)kSnapStride * w;
  if (hi < T(0)) {
    if (lane == 0) {
      rec[0] = T(-1), rec[1] = T(0);
      for (int k = 2; k < kSnapStride; ++k) rec[k] = T(0);
    }
    __syncwarp();
    return;
  }
  T lo = T(0);
  const int nb = sizeof(T) == 4 ? 24 : 52;
  for (int b = 0; b < nb; ++b) {
    const T mid = T(0.5) * (lo + hi);
    if (inside(mid))
      lo = mid;
    else
      hi = mid;
  }
  // snapped rotation Exp(tau* omega) R* in FP64, rounded once
  const D th = D(lo) * wn, hs = sin(0.5 * th), hc = cos(0.5 * th);
  const Q4<D> inc = wn > 0 ? Q4<D>{hc, hs * w64.x / wn, hs * w64.y / wn, hs * w64.z / wn} : Q4<D>{1.0, 0.0, 0.0, 0.0};
  Q4<D> qs = qmul(inc, q64);  // both factors unit to FP64 rounding
  if (qs.w < 0) qs = Q4<D>{-qs.w, -qs.x, -qs.y, -qs.z};
  q = Q4<T>{T(qs.w), T(qs.x), T(qs.y), T(qs.z)};
  t = V3<T>{T(t64.x), T(t64.y), T(t64.z)};
  // active constraint at tau* from the same residuals
  const M3<T> M = exp_minus_identity(ax, lo * wnt);
  double bm = INFINITY;
  int bi = 0x7FFFFFFF;
  for (int i = lane; i < N; i += 32) {
    T ex, ey, ez;
    residual(M, i, ex, ey, ez);
    const double r = double(coef[kS * i + 8]);
    const double m = KIND == 1 ? r - sqrt(double(ex) * ex + double(ey) * ey) / double(ez)
                               : sqrt(r) - sqrt(double(ex) * ex + double(ey) * ey + double(ez) * ez);
    if (m < bm) bm = m, bi = i;
  }
  const int j = warp_argmin(bm, bi);
  if (lane == 0) snap_record<T, KIND, LAM>(c, j, qs, t64, w64, 0, rec);
  __syncwarp();
}

// Translation ray (R*, t* + tau v) through the affine residuals; (q64, t64, v64) the FP64 pose and
// direction, coef a free area of the warp's slab (7 N values).  The snapped translation is formed
// in FP64 and rounded once.
template <typename T, int KIND, bool LAM>
__device__ __forceinline__ void snap_translation(const WalkCtx<T>& c, const T4<T>* tab_s, const Q4<double>& q64,
                                                 const V3<double>& t64, const V3<T>& vt, T* coef, Q4<T>& q,
                                                 V3<T>& t, int w, int lane) {
  const V3<double> v64{double(vt.x), double(vt.y), double(vt.z)};
  using D = double;
  const int N = c.N;
  const T4<D>* tab = reinterpret_cast<const T4<D>*>(c.tab64);
  const D fx = c.kd[0], fy = c.kd[1], cx = c.kd[2], cy = c.kd[3];
  const M3<D> R = qmat(q64);
  // coef[7 i ..]: base residual (3), slope (3), r (2D-3D) or r^2 (3D-3D)
  for (int i = lane; i < N; i += 32) {
    const T4<D> mz = tab[i], ob = tab[N + i];
    const V3<D> X = mul(R, V3<D>{mz.x, mz.y, mz.z}) + t64;
    T* k = coef + 7 * i;
    const double* u = LAM ? c.ell64 + 8 * (size_t)i : nullptr;
    if (KIND == 1) {
      // e = (fx X_x + (cx - u) X_z, fy X_y + (cy - v) X_z), P_z = X_z; with noise matrices U e
      D e0 = fx * X.x + (cx - ob.x) * X.z, e1 = fy * X.y + (cy - ob.y) * X.z;
      D b0 = fx * v64.x + (cx - ob.x) * v64.z, b1 = fy * v64.y + (cy - ob.y) * v64.z;
      if (LAM) {
        e0 = u[0] * e0 + u[1] * e1, e1 = u[2] * e1;
        b0 = u[0] * b0 + u[1] * b1, b1 = u[2] * b1;
      }
      k[0] = T(e0), k[1] = T(e1), k[2] = T(X.z);
      k[3] = T(b0), k[4] = T(b1), k[5] = T(v64.z);
      k[6] = T(mz.w);
    } else {
      V3<D> g0 = X - V3<D>{ob.x, ob.y, ob.z}, g1 = v64;
      if (LAM) g0 = umul3(u, g0), g1 = umul3(u, g1);
      k[0] = T(g0.x), k[1] = T(g0.y), k[2] = T(g0.z);
      k[3] = T(g1.x), k[4] = T(g1.y), k[5] = T(g1.z);
      k[6] = T(ob.w);
    }
  }
  __syncwarp();
  auto inside = [&](T tau) {
    bool ok = true;
    for (int i = lane; i < N; i += 32) {
      const T* k = coef + 7 * i;
      const T ex = fma(tau, k[3], k[0]), ey = fma(tau, k[4], k[1]), ez = fma(tau, k[5], k[2]);
      if (KIND == 1) {
        const T rz = k[6] * ez;
        ok = ok && ez > T(0) && ex * ex + ey * ey - rz * rz <= T(0);
      } else {
        ok = ok && ex * ex + ey * ey + ez * ez - k[6] <= T(0);
      }
    }
    return __all_sync(kFullMask, ok);
  };
  T hi = T(-1);
  for (int m = c.NT - 1; m >= 0 && hi < T(0); --m) {
    T sm = T(1);
    for (int k = 0; k < m; ++k) sm *= c.gam;
    if (!inside(sm)) hi = sm;
  }
  T* rec = c.out_snap + (size_t)kSnapStride * w;
  if (hi < T(0)) {
    if (lane == 0) {
      rec[0] = T(-1), rec[1] = T(1);
      for (int k = 2; k < kSnapStride; ++k) rec[k] = T(0);
    }
    return;
  }
  T lo = T(0);
  const int nb = sizeof(T) == 4 ? 24 : 52;
  for (int b = 0; b < nb; ++b) {
    const T mid = T(0.5) * (lo + hi);
    if (inside(mid))
      lo = mid;
    else
      hi = mid;
  }
  const V3<D> ts{t64.x + D(lo) * v64.x, t64.y + D(lo) * v64.y, t64.z + D(lo) * v64.z};
  t = V3<T>{T(ts.x), T(ts.y), T(ts.z)};
  q = Q4<T>{T(q64.w), T(q64.x), T(q64.y), T(q64.z)};
  // active constraint at tau* from the affine model (margins r - |e| / P_z, or r - |g|)
  double bm = INFINITY;
  int bi = 0x7FFFFFFF;
  for (int i = lane; i < N; i += 32) {
    const T* k = coef + 7 * i;
    const T ex = fma(lo, k[3], k[0]), ey = fma(lo, k[4], k[1]), ez = fma(lo, k[5], k[2]);
    const double m = KIND == 1 ? double(k[6]) - sqrt(double(ex) * ex + double(ey) * ey) / double(ez)
                               : sqrt(double(k[6])) - sqrt(double(ex) * ex + double(ey) * ey + double(ez) * ez);
    if (m < bm) bm = m, bi = i;
  }
  const int j = warp_argmin(bm, bi);
  if (lane == 0) snap_record<T, KIND, LAM>(c, j, q64, ts, v64, 1, rec);
  __syncwarp();
}

// Double-float arithmetic (a value carried as an unevaluated sum hi + lo of two floats, ~48
// significant bits) from the error-free transformations of Knuth (two_sum) and of the fused
// multiply-add (two_prod); the file is compiled without contraction, so + and * round as written.
struct DF {
  float h, l;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return DF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = a * b;
  return DF{p, fmaf(a, b, -p)};
}
// a0 b0 + a1 b1 + a2 b2 + a3 b3 for float a and double-float b (the lo parts of b enter once).
__device__ __forceinline__ DF df_dot4(float a0, DF b0, float a1, DF b1, float a2, DF b2, float a3, DF b3) {
  const DF p0 = two_prod(a0, b0.h), p1 = two_prod(a1, b1.h), p2 = two_prod(a2, b2.h), p3 = two_prod(a3, b3.h);
  const DF s1 = two_sum(p0.h, p1.h), s2 = two_sum(s1.h, p2.h), s3 = two_sum(s2.h, p3.h);
  const float lo = ((s1.l + s2.l) + (s3.l + p0.l)) + ((p1.l + p2.l) + p3.l) +
                   (a0 * b0.l + a1 * b1.l + a2 * b2.l + a3 * b3.l);
  return quick_two_sum(s3.h, lo);
}

// One move of an FP32 walk's pose, p (x) q and t + dt, in double-float, spread over the warp: lane
// k < 4 forms quaternion component k, lane 4 + k translation component k.  p is a unit quaternion to
// FP32 rounding, so |p (x) q|^2 = 1 + d with |d| ~ 1e-7, and q (1 - d/2) renormalises to ~d^2 (the
// squared norm is summed over lanes 0-3 with two shuffles); the sign keeps w >= 0.  F: floats of
// Slab::S, read by every lane before any lane writes.
__device__ __forceinline__ void df_move(float* F, int lane, float pw, float px, float py, float pz, float dx, float dy,
                                        float dz) {
  const DF qw{F[0], F[4]}, qx{F[1], F[5]}, qy{F[2], F[6]}, qz{F[3], F[7]};
  // component lane of p (x) q: w = pw qw - px qx - py qy - pz qz, x = pw qx + px qw + py qz - pz qy,
  // y = pw qy + py qw + pz qx - px qz, z = pw qz + pz qw + px qy - py qx
  const int k = lane & 3;
  const float a1 = k == 0 ? -px : k == 1 ? px : k == 2 ? py : pz;
  const float a2 = k == 0 ? -py : k == 1 ? py : k == 2 ? pz : px;
  const float a3 = k == 0 ? -pz : k == 1 ? -pz : k == 2 ? -px : -py;
  const DF b0 = k == 0 ? qw : k == 1 ? qx : k == 2 ? qy : qz;
  const DF b1 = k == 0 ? qx : qw;
  const DF b2 = k == 0 ? qy : k == 1 ? qz : k == 2 ? qx : qy;
  const DF b3 = k == 0 ? qz : k == 1 ? qy : k == 2 ? qz : qx;
  DF r = df_dot4(pw, b0, a1, b1, a2, b2, a3, b3);
  if (lane >= 4) r = DF{0.0f, 0.0f};
  // |r|^2 over lanes 0-3: h^2 exactly (two_prod) plus 2 h l
  DF sq = two_prod(r.h, r.h);
  float lo = sq.l + 2.0f * r.h * r.l;
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    const float oh = __shfl_xor_sync(kFullMask, sq.h, o), ol = __shfl_xor_sync(kFullMask, lo, o);
    const DF t = two_sum(sq.h, oh);
    sq.h = t.h, lo = lo + ol + t.l;
  }
  const float d = (sq.h - 1.0f) + lo;
  const float sg = __shfl_sync(kFullMask, r.h, 0) < 0.0f ? -1.0f : 1.0f;
  float th = 0.0f, tl = 0.0f;
  if (lane >= 4 && lane < 7) {
    const int c = lane - 4;
    const float dt = c == 0 ? dx : c == 1 ? dy : dz;
    const DF s = two_sum(F[8 + c], dt);
    const DF v = quick_two_sum(s.h, s.l + F[11 + c]);
    th = v.h, tl = v.l;
  }
  __syncwarp();
  if (lane < 4) {
    const DF v = quick_two_sum(r.h, r.l - 0.5f * d * r.h);
    F[lane] = sg * v.h, F[4 + lane] = sg * v.l;
  } else if (lane < 7) {
    F[8 + lane - 4] = th, F[11 + lane - 4] = tl;
  }
}

// Start velocity of walk w in FP64: omega = omega0 (u + u~) (Alg. 3) or v = v0 S (dir + v~) (Alg. 5),
// u~ / v~ the first accepted unit lattice draw of the walk's stream.
template <typename T, int SAMPLER>
__device__ __forceinline__ V3<double> start_velocity64(const WalkCtx<T>& c, int w) {
  const double* sd = c.seed_data + (size_t)(w % c.s0) * kSeedStride;
  Stream s(c.key0, c.key1, SAMPLER == 0 ? kPhaseOmega : kPhaseV, 0u, 0u, (uint32_t)w);
  int X, Y, Z;
  lattice_draw<true>(s, X, Y, Z);
  const double nr = sqrt((double)(X * X + Y * Y + Z * Z));
  const double ux = nr > 0 ? X / nr : 0.0, uy = nr > 0 ? Y / nr : 0.0, uz = nr > 0 ? Z / nr : 0.0;
  if (SAMPLER == 0)
    return V3<double>{c.omega0 * (sd[7] + ux), c.omega0 * (sd[8] + uy), c.omega0 * (sd[9] + uz)};
  const WalkStats* st = c.st;
  const double d0 = sd[10] + ux, d1 = sd[11] + uy, d2 = sd[12] + uz;
  return V3<double>{c.v0 * (st->S[0] * d0 + st->S[1] * d1 + st->S[2] * d2),
                    c.v0 * (st->S[3] * d0 + st->S[4] * d1 + st->S[5] * d2),
                    c.v0 * (st->S[6] * d0 + st->S[7] * d1 + st->S[8] * d2)};
}

// Start of walk w: pose of seed (w mod |S0|) and the start velocity, in T.  FP32 walks take the
// rounded seed data and compute the velocity in FP32 (no FP64 instruction: on this part each one
// occupies the FP64 unit for tens of cycles); FP64 walks take start_velocity64.
template <typename T, int SAMPLER>
__device__ __forceinline__ void walk_start(const WalkCtx<T>& c, int w, Q4<T>& q, V3<T>& t, V3<T>& vel) {
  const double* sd = c.seed_data + (size_t)(w % c.s0) * kSeedStride;
  if constexpr (sizeof(T) == 8) {
    q = Q4<T>{sd[0], sd[1], sd[2], sd[3]};
    t = V3<T>{sd[4], sd[5], sd[6]};
    const V3<double> v = start_velocity64<T, SAMPLER>(c, w);
    vel = V3<T>{v.x, v.y, v.z};
  } else {
    const float* f = reinterpret_cast<const float*>(sd + kSeedFloats);
    q = Q4<T>{f[0], f[1], f[2], f[3]};
    t = V3<T>{f[8], f[9], f[10]};
    Stream s(c.key0, c.key1, SAMPLER == 0 ? kPhaseOmega : kPhaseV, 0u, 0u, (uint32_t)w);
    int X, Y, Z;
    lattice_draw<true>(s, X, Y, Z);
    const float nr = sqrtf((float)(X * X + Y * Y + Z * Z));  // the integer is exact in FP32
    const float ux = nr > 0 ? X / nr : 0.0f, uy = nr > 0 ? Y / nr : 0.0f, uz = nr > 0 ? Z / nr : 0.0f;
    if (SAMPLER == 0) {
      vel = V3<T>{c.om0 * (f[14] + ux), c.om0 * (f[15] + uy), c.om0 * (f[16] + uz)};
    } else {
      const float* S = c.st->Sf;
      const float d0 = f[17] + ux, d1 = f[18] + uy, d2 = f[19] + uz;
      vel = V3<T>{c.vv0 * (S[0] * d0 + S[1] * d1 + S[2] * d2), c.vv0 * (S[3] * d0 + S[4] * d1 + S[5] * d2),
                  c.vv0 * (S[6] * d0 + S[7] * d1 + S[8] * d2)};
    }
  }
}

// One walk of Alg. 3 (dS_R) or Alg. 5 (dS_t): N_I iterations from seed (w mod |S0|), then emit.
// tab: the PURSE's constraint table in shared memory; sl: this warp's slab.
// LAM: noise matrices; their factors follow the table (rows 2N + 2i, 2N + 2i + 1).
template <typename T, int KIND, int SAMPLER, bool LAM, class RK>
__device__ __forceinline__ void walk_one(const WalkCtx<T>& c, const RK& rk, int w, const T4<T>* tab,
                                         const Slab<T>& sl, int lane, unsigned long long& evals) {
  using Key = typename KeyOf<T>::type;
  using T2 = P2<T>;
  const int N = c.N, NQ = ladder_pairs(c.N);
  const int NP = c.NP, K = c.K, NT = c.NT, mc = c.mc;
  const T fx = c.fx, fy = c.fy, cx = c.cx, cy = c.cy, r_pert = c.r_pert;
  const int ncand = mc * K;
  const int cm = lane / K, ck = lane - (lane / K) * K;
  // perturbation pairs: nfull passes of 32, then qtail pairs with 2^tsh lanes each
  const int npairs = (NP + 1) / 2, nfull = npairs / 32, qtail = npairs % 32;
  const int tsh = qtail == 0 ? 0 : qtail <= 1 ? 5 : qtail <= 2 ? 4 : qtail <= 4 ? 3 : qtail <= 8 ? 2 : qtail <= 16 ? 1 : 0;
  // ---- a3: start pose and velocity, ladder table of this walk.
  Q4<T> q;
  V3<T> t;
  V3<T> vel;
  // FP32 2D-3D walks whose samples are snapped to the boundary carry their pose in double-float pairs
  // in the slab: the warp applies each move there (lanes 0-6, df_move) and every lane takes the hi
  // parts.  Repeated FP32 pose updates accumulate ~1e-7 rad per move, and the snap places the sample
  // where the ray from that pose meets the boundary -- along the viewing ray of a 2D-3D PURSE ~1e-6 m
  // off.  A 3D-3D PURSE has no such long axis (the same error moves its snapped samples by ~1e-7 m),
  // and without the snap a sample is an interior point chosen by the walk's discrete decisions, so
  // those walks keep the FP32 pose (the double-float moves cost ~9 % of a short batch walk).  (FP64 arithmetic
  // would do, but one FP64 instruction of one lane occupies this part's FP64 unit far longer.)
  constexpr bool kState64 = sizeof(T) == 4 && KIND == 1;
  const bool df = kState64 && c.out_snap != nullptr;
  walk_start<T, SAMPLER>(c, w, q, t, vel);
  if (df && lane == 0) {
    const float* f = reinterpret_cast<const float*>(c.seed_data + (size_t)(w % c.s0) * kSeedStride + kSeedFloats);
    float* F = reinterpret_cast<float*>(sl.S);
    for (int k = 0; k < 14; ++k) F[k] = f[k];
  }
  const T rho_max = c.rho_max;
  for (int m = lane; m < NT; m += 32) {
    T sm = T(1);
    for (int k = 0; k < m; ++k) sm *= c.gam;
    if (SAMPLER == 0) {
      const Q4<T> e = qexp(V3<T>{sm * vel.x, sm * vel.y, sm * vel.z});
      M3<T> E = qmat(e);
      if (KIND == 1) {
        for (int c = 0; c < 3; ++c) {
          E.m[c] = fx * E.m[c] + cx * E.m[6 + c];
          E.m[3 + c] = fy * E.m[3 + c] + cy * E.m[6 + c];
        }
      }
      sl.E[4 * m] = T4<T>{e.w, e.x, e.y, e.z};
      for (int r = 0; r < 3; ++r) sl.E[4 * m + 1 + r] = T4<T>{E.m[3 * r], E.m[3 * r + 1], E.m[3 * r + 2], T(0)};
    } else {
      sl.E[4 * m] = T4<T>{sm * vel.x, sm * vel.y, sm * vel.z, T(0)};
    }
  }
  __syncwarp();

  // The order and the tables depend on (R*, t*) only: an iteration after one that kept the pose
  // reuses them (and qzmin).
  bool moved = true;
  T qzmin = inf<T>();
  for (int it = 0; it < c.n_iter; ++it) {
   if (moved) {
    const M3<T> R = qmat(q);
    // ---- constraint order: ascending margin of the current pose (N <= 32; the order only decides how
    //      soon the ladder's early exit triggers), then the tables
    int perm = lane;
    if (N <= 32) {
      uint32_t kk = 0xFFFFFFFFu;
      if (lane < N) {
        const T4<T> mz = tab[lane], ob = tab[N + lane];
        const V3<T> X = mul(R, V3<T>{mz.x, mz.y, mz.z}) + t;
        float m;
        if (KIND == 1) {
          const T Pz = X.z;
          T ex = fx * X.x + cx * X.z - ob.x * Pz, ey = fy * X.y + cy * X.z - ob.y * Pz;
          if constexpr (LAM) {
            const T4<T> ua = tab[2 * N + 2 * lane];
            ex = ua.x * ex + ua.y * ey, ey = ua.z * ey;
          }
          m = Pz > T(0) ? (float)(mz.w * Pz * mz.w * Pz - ex * ex - ey * ey) : -INFINITY;
        } else {
          T ex = X.x - ob.x, ey = X.y - ob.y, ez = X.z - ob.z;
          if constexpr (LAM) {
            const T4<T> ua = tab[2 * N + 2 * lane], ub = tab[2 * N + 2 * lane + 1];
            const T gx = ua.x * ex + ua.y * ey + ua.z * ez, gy = ua.w * ey + ub.x * ez;
            ex = gx, ey = gy, ez = ub.y * ez;
          }
          m = (float)(ob.w - ex * ex - ey * ey - ez * ez);
        }
        kk = (orderable(m) & ~31u) | (uint32_t)lane;
      }
#pragma unroll
      for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
          const uint32_t o = __shfl_xor_sync(kFullMask, kk, stride);
          const bool up = ((lane & size) == 0);
          const bool lower = (lane & stride) == 0;
          const uint32_t mn = kk < o ? kk : o, mx = kk < o ? o : kk;
          kk = (lower == up) ? mn : mx;
        }
      }
      perm = (int)(kk & 31u);
    }
    qzmin = inf<T>();
    for (int r = lane; r < N; r += 32) {
      const int i = N <= 32 ? perm : r;
      const T4<T> mz = tab[i], ob = tab[N + i];
      const V3<T> Y = mul(R, V3<T>{mz.x, mz.y, mz.z});
      T2* Dr = sl.D + kRow<LAM> * r;
      if (SAMPLER == 0) {
        if (KIND == 1) {
          const V3<T> X = Y + t;
          const T qz = X.z;
          Dr[0] = dup(fx * X.x + cx * X.z), Dr[1] = dup(fy * X.y + cy * X.z), Dr[2] = dup(qz);
          qzmin = fmin(qzmin, qz);
        } else {
          Dr[0] = dup(Y.x + t.x - ob.x), Dr[1] = dup(Y.y + t.y - ob.y), Dr[2] = dup(Y.z + t.z - ob.z);
        }
      } else {
        Dr[0] = dup(Y.x), Dr[1] = dup(Y.y), Dr[2] = dup(Y.z);
      }
      Dr[3] = dup(mz.w);
      if (KIND == 1) {
        Dr[4] = dup(-ob.x), Dr[5] = dup(-ob.y);
      } else if (SAMPLER == 1) {
        Dr[4] = dup(t.x - ob.x), Dr[5] = dup(t.y - ob.y), Dr[6] = dup(t.z - ob.z);
      }
      // ladder table: constraint r in half (r & 1) of pair r / 2
      T* Lq = reinterpret_cast<T*>(sl.L + kRow<LAM> * (r >> 1)) + (r & 1);
      Lq[0] = Y.x, Lq[2] = Y.y, Lq[4] = Y.z;
      if (KIND == 1) {
        Lq[6] = -ob.x, Lq[8] = -ob.y, Lq[10] = -ob.w;
      } else {
        Lq[6] = -ob.x, Lq[8] = -ob.y, Lq[10] = -ob.z, Lq[12] = -ob.w;
      }
      if constexpr (LAM) {  // U_i in slots 8-13 of both tables
        const T4<T> ua = tab[2 * N + 2 * i], ub = tab[2 * N + 2 * i + 1];
        const T u[6] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y};
#pragma unroll
        for (int k = 0; k < (KIND == 1 ? 3 : 6); ++k) Dr[8 + k] = dup(u[k]), Lq[16 + 2 * k] = u[k];
      }
    }
    if ((N & 1) && lane == 0) {  // odd N: the second half of the last pair is always satisfied
      T* Lq = reinterpret_cast<T*>(sl.L + kRow<LAM> * (N >> 1)) + 1;
      Lq[0] = Lq[2] = Lq[4] = T(0);
      Lq[6] = Lq[8] = T(0);
      Lq[10] = T(-1e30);
      if (KIND == 0) Lq[10] = T(0), Lq[12] = T(-1e30);
      if constexpr (LAM) {
#pragma unroll
        for (int k = 0; k < 6; ++k) Lq[16 + 2 * k] = T(0);
      }
    }
    if (SAMPLER == 0 && KIND == 1) {
#pragma unroll
      for (int o = 16; o; o >>= 1) qzmin = fmin(qzmin, __shfl_xor_sync(kFullMask, qzmin, o));
    }
    __syncwarp();
   }

    // ---- a4: perturbations and their distance to the boundary (eq. 11): full passes of 32 pairs
    //      (dS_R: all at once; dS_t keeps one rotation per perturbation in registers: two pairs at
    //      a time), then the ragged remainder of q pairs with 32 / q lanes (a power of two) per pair
    if constexpr (SAMPLER == 0) {
      if (nfull == 4)
        dist_pass<T, KIND, SAMPLER, 4, true, LAM>(rk, it, w, sl, N, NP, lane, 0, r_pert, t, fx, fy, cx, cy, qzmin);
      else if (nfull == 3)
        dist_pass<T, KIND, SAMPLER, 3, true, LAM>(rk, it, w, sl, N, NP, lane, 0, r_pert, t, fx, fy, cx, cy, qzmin);
      else if (nfull == 2)
        dist_pass<T, KIND, SAMPLER, 2, true, LAM>(rk, it, w, sl, N, NP, lane, 0, r_pert, t, fx, fy, cx, cy, qzmin);
      else if (nfull == 1)
        dist_pass<T, KIND, SAMPLER, 1, true, LAM>(rk, it, w, sl, N, NP, lane, 0, r_pert, t, fx, fy, cx, cy, qzmin);
      if (qtail) dist_pass<T, KIND, SAMPLER, 1, true, LAM>(rk, it, w, sl, N, NP, lane, nfull, r_pert, t, fx, fy, cx, cy, qzmin, tsh);
    } else {
      // P_z = (R Z_i)_z + t*_z >= t*_z - max |Z_i| (rotations keep |Z_i|); the margin covers rounding
      if (KIND == 1 && t.z - rho_max > T(1e-3) * (fabs(t.z) + rho_max)) {
        for (int pb = 0; pb < nfull; pb += 2) {
          if (nfull - pb >= 2)
            dist_pass<T, KIND, SAMPLER, 2, false, LAM>(rk, it, w, sl, N, NP, lane, pb, r_pert, t, fx, fy, cx, cy, qzmin);
          else
            dist_pass<T, KIND, SAMPLER, 1, false, LAM>(rk, it, w, sl, N, NP, lane, pb, r_pert, t, fx, fy, cx, cy, qzmin);
        }
        if (qtail)
          dist_pass<T, KIND, SAMPLER, 1, false, LAM>(rk, it, w, sl, N, NP, lane, nfull, r_pert, t, fx, fy, cx, cy, qzmin, tsh);
      } else {
        for (int pb = 0; pb < nfull; pb += 2) {
          if (nfull - pb >= 2)
            dist_pass<T, KIND, SAMPLER, 2, true, LAM>(rk, it, w, sl, N, NP, lane, pb, r_pert, t, fx, fy, cx, cy, qzmin);
          else
            dist_pass<T, KIND, SAMPLER, 1, true, LAM>(rk, it, w, sl, N, NP, lane, pb, r_pert, t, fx, fy, cx, cy, qzmin);
        }
        if (qtail) dist_pass<T, KIND, SAMPLER, 1, true, LAM>(rk, it, w, sl, N, NP, lane, nfull, r_pert, t, fx, fy, cx, cy, qzmin, tsh);
      }
    }
    evals += (unsigned long long)NP * N;
    __syncwarp();

    // ---- a5: top_k_indices (ties to the lower j): per-lane sorted keys, warp max rounds
    if (NP <= 160)
      top_k<Key, 5>(sl, NP, K, lane);
    else
      top_k<Key, 8>(sl, NP, K, lane);
    __syncwarp();

    // ---- a6/a7: step ladder + in_purse with early exit, find_farthest
    int m0 = -1, k0 = -1;
    V3<T> base{T(0), T(0), T(0)};
    M3<T> Ak = M3<T>{{T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)}};  // dS_t: (K) R_{j_k}
    if (lane < ncand) {
      const T4<T> pj = sl.P[sl.J[ck]];
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
    T2 M2t[9];
    if constexpr (SAMPLER == 1) {
#pragma unroll
      for (int c = 0; c < 9; ++c) M2t[c] = dup(Ak.m[c]);
    }
    // Candidate of this lane in the chunk of rungs [mb, mb + mc): the rung's (K) E_m (dS_R) or the
    // kept perturbation's (K) R_{j_k} (dS_t) as M2, and the candidate translation b (projected by K
    // for 2D-3D).
    auto chunk = [&](int mb, T2 (&M2)[9], V3<T>& bm) {
      const int m = mb + cm;
      const bool active = lane < ncand && m < NT;
      M3<T> M = M3<T>{{T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)}};
      bm = base;
      if (active) {
        if (SAMPLER == 0) {
          const T4<T> e0 = sl.E[4 * m + 1], e1 = sl.E[4 * m + 2], e2 = sl.E[4 * m + 3];
          M = M3<T>{{e0.x, e0.y, e0.z, e1.x, e1.y, e1.z, e2.x, e2.y, e2.z}};
        } else {
          const T4<T> sv = sl.E[4 * m];
          const V3<T> Tm{t.x + sv.x, t.y + sv.y, t.z + sv.z};
          bm = KIND == 1 ? V3<T>{fx * Tm.x + cx * Tm.z, fy * Tm.y + cy * Tm.z, Tm.z} : Tm;
        }
      }
#pragma unroll
      for (int c = 0; c < 9; ++c) M2[c] = SAMPLER == 1 ? M2t[c] : dup(M.m[c]);
      return active;
    };
    // First pass: constraint pair 0 (the two constraints of smallest margin at the current pose) for
    // the candidates of every chunk, with no vote between chunks; on the walk workloads almost every
    // candidate fails there.  Bit s of surv: this lane's candidate of chunk s passed it.
    const int nch = (NT + mc - 1) / mc;
    uint32_t surv = 0;
#pragma unroll 2
    for (int s = 0; s < nch; ++s) {
      T2 M2[9];
      V3<T> bm;
      const bool active = chunk(s * mc, M2, bm);
      T2 cmax = dup(-inf<T>()), zmin = dup(inf<T>());
      ladder_pair<T, KIND, true, LAM>(sl.L, M2, dup(bm.x), dup(bm.y), dup(bm.z), cmax, zmin);
      surv |= (uint32_t)(active && ladder_ok<T, KIND, true>(cmax, zmin)) << s;
    }
    evals += (unsigned long long)K * NT * min(N, 2);
    // Then the chunks in rung order, each only if some candidate passed pair 0, over pairs 1 ..; the
    // first chunk with a feasible candidate ends the ladder (the same m0, k0 as scanning every chunk
    // over every pair: in_purse is a conjunction and each value is the same expression).
    for (int s = 0; s < nch; ++s) {
      unsigned bal = __ballot_sync(kFullMask, (surv >> s) & 1u);
      if (!bal) continue;
      const int mb = s * mc;
      if (NQ > 1) {
        T2 M2[9];
        V3<T> bm;
        const bool active = chunk(mb, M2, bm);
        const T2 bx = dup(bm.x), by = dup(bm.y), bz = dup(bm.z);
        T2 cmax = dup(-inf<T>()), zmin = dup(inf<T>());
        bool alive = ((surv >> s) & 1u) != 0;
        const int nact = K * min(mc, NT - mb);
        int done = 2;
        // 2D-3D: P_z >= (candidate translation)_z - max |Z_i| (the rotation rows are unit vectors);
        // when that bound is positive for every candidate of the chunk, cheirality is not tracked
        // (dS_R only: the dS_t kernel measured slower with the second ladder instantiation)
        const bool zsafe = KIND == 1 && SAMPLER == 0 &&
                           __all_sync(kFullMask, !active || bm.z - rho_max > T(1e-3) * (fabs(bm.z) + rho_max));
        if (zsafe)
          ladder_scan<T, KIND, false, LAM>(sl.L, 1, NQ, N, M2, bx, by, bz, cmax, zmin, alive, done);
        else
          ladder_scan<T, KIND, true, LAM>(sl.L, 1, NQ, N, M2, bx, by, bz, cmax, zmin, alive, done);
        evals += (unsigned long long)nact * (done - 2);
        bal = __ballot_sync(kFullMask, alive);
      }
      if (bal) {
        const int l = __ffs(bal) - 1;
        m0 = mb + l / K;
        k0 = l - (l / K) * K;
        break;
      }
    }

    // ---- update (R*, t*)
    moved = m0 >= 0;
    if (m0 >= 0) {
      const T4<T> pj = sl.P[sl.J[k0]];
      if (df) {
        float* F = reinterpret_cast<float*>(sl.S);
        if (SAMPLER == 0) {
          const T4<T> e = sl.E[4 * m0];  // (w, x, y, z) of E_m0
          df_move(F, lane, e.x, e.y, e.z, e.w, pj.x, pj.y, pj.z);
        } else {
          const T4<T> sv = sl.E[4 * m0];  // gamma^m0 v
          df_move(F, lane, pj.x, pj.y, pj.z, pj.w, sv.x, sv.y, sv.z);
        }
        __syncwarp();
        q = Q4<T>{F[0], F[1], F[2], F[3]};
        t = V3<T>{F[8], F[9], F[10]};
      } else if (SAMPLER == 0) {
        const T4<T> e = sl.E[4 * m0];
        q = qnormalize(qmul(Q4<T>{e.x, e.y, e.z, e.w}, q));
        t = V3<T>{t.x + pj.x, t.y + pj.y, t.z + pj.z};
      } else {
        q = qnormalize(qmul(Q4<T>{pj.x, pj.y, pj.z, pj.w}, q));
        const T4<T> sv = sl.E[4 * m0];
        t = V3<T>{t.x + sv.x, t.y + sv.y, t.z + sv.z};
      }
    }
    if (c.trace != nullptr && lane == 0) {
      int16_t* tr = c.trace + ((size_t)w * c.n_iter + it) * (K + 2);
      for (int r = 0; r < K; ++r) tr[r] = (int16_t)sl.J[r];
      tr[K] = (int16_t)m0;
      tr[K + 1] = (int16_t)k0;
    }
    __syncwarp();
  }

  // ---- optional boundary snap (for the adjoint), then a8: emit
  {
    if (c.out_snap) {
      // the ray starts from the pose in FP64 (the double-float state of FP32 walks) and follows the
      // walk's velocity in T (its rounding moves the snapped point by ~1e-7 of the step)
      Q4<double> q64;
      V3<double> t64;
      if constexpr (kState64) {
        const float* F = reinterpret_cast<const float*>(sl.S);
        q64 = Q4<double>{double(F[0]) + F[4], double(F[1]) + F[5], double(F[2]) + F[6], double(F[3]) + F[7]};
        t64 = V3<double>{double(F[8]) + F[11], double(F[9]) + F[12], double(F[10]) + F[13]};
      } else {
        q64 = Q4<double>{double(q.w), double(q.x), double(q.y), double(q.z)};
        t64 = V3<double>{double(t.x), double(t.y), double(t.z)};
      }
      if constexpr (SAMPLER == 0)
        snap_rotation<T, KIND, LAM>(c, tab, q64, t64, vel, reinterpret_cast<T*>(sl.D), q, t, w, lane);
      else
        snap_translation<T, KIND, LAM>(c, tab, q64, t64, vel, reinterpret_cast<T*>(sl.D), q, t, w, lane);
    }
  }
  if (lane == 0) {
    T* oq = c.out_q + 4 * (size_t)w;
    T* ot = c.out_t + 3 * (size_t)w;
    oq[0] = q.w, oq[1] = q.x, oq[2] = q.y, oq[3] = q.z;
    ot[0] = t.x, ot[1] = t.y, ot[2] = t.z;
    if (!(isfinite(q.w) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(t.x) && isfinite(t.y) &&
          isfinite(t.z)))
      atomicOr(c.status, kDevErrNumeric);
  }
  __syncwarp();
}

template <typename T, int KIND, int SAMPLER, bool LAM>
__global__ void __launch_bounds__(kWalkThreads, sizeof(T) == 4 ? 2 : 1)
    walk_kernel(const __grid_constant__ WalkArgs a, const int mc, const int slab_bytes) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  const int N = a.n;
  // rows [0,N): (a, r); [N,2N): (b or z, r^2); with noise matrices [2N,4N): U_i
  const T4<T>* tab = reinterpret_cast<const T4<T>*>(smem + 128);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Slab<T> sl = carve<T, LAM>(smem + 128 + walk_table_bytes<T>(N, LAM) + (size_t)warp * slab_bytes, N,
                                   a.n_perturb, a.n_steps);

  // ---- a0: stage the constraint table (and the noise factors) with 1-D TMA bulk copies.
  const uint32_t tbytes = 8u * N * sizeof(T);
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, LAM ? 2 * tbytes : tbytes);
    bulk_copy_g2s(smem + 128, a.table, tbytes, bar);
    if (LAM) bulk_copy_g2s(smem + 128 + tbytes, a.ell, tbytes, bar);
  }
  if (!mbar_wait_bounded(bar, 0, 1 << 22)) {
    // thread 0 gives the copies still in flight one more bounded wait, so that none lands in this
    // CTA's shared memory after it has exited
    if (threadIdx.x == 0) {
      atomicOr(a.status, kDevErrTimeout);
      mbar_wait_bounded(bar, 0, 1 << 22);
    }
    return;
  }
  if (a.stall_probe) {  // PURSE_FAULT=stall: a second barrier that nothing arrives at, short poll limit
    if (threadIdx.x == 0) mbar_init(bar + 1, 1);
    __syncthreads();
    if (!mbar_wait_bounded(bar + 1, 0, 1 << 10)) {
      if (threadIdx.x == 0) atomicOr(a.status, kDevErrTimeout);
      return;
    }
  }
  WalkCtx<T> c;
  c.N = N, c.NP = a.n_perturb, c.K = a.n_keep, c.NT = a.n_steps, c.mc = mc, c.n_iter = a.n_iter;
  c.fx = T(a.fx), c.fy = T(a.fy), c.cx = T(a.cx), c.cy = T(a.cy);
  c.rho_max = T(a.rho_max);
  c.r_pert = T(SAMPLER == 0 ? a.stats->r_trans : a.stats->r_rot);
  c.omega0 = a.omega0, c.v0 = a.v0, c.gamma = a.gamma;
  c.om0 = T(a.omega0), c.vv0 = T(a.v0), c.gam = T(a.gamma);
  c.st = a.stats, c.seed_data = a.seed_data, c.s0 = a.s0;
  c.key0 = a.key0, c.key1 = a.key1;
  c.out_q = reinterpret_cast<T*>(a.out_q), c.out_t = reinterpret_cast<T*>(a.out_t);
  c.trace = a.trace, c.status = a.status;
  c.out_snap = reinterpret_cast<T*>(a.out_snap);
  c.tab64 = a.table64, c.kd = &a.fx, c.ell64 = a.ell64;
  const RkParam rk{a};
  unsigned long long evals = 0;
  const int nw = blockDim.x >> 5;  // warps per block (fewer than kWalkWarps for large tables)
  for (int w = blockIdx.x * nw + warp; w < a.n_samples; w += gridDim.x * nw)
    walk_one<T, KIND, SAMPLER, LAM>(c, rk, w, tab, sl, lane, evals);
  if (lane == 0 && evals) atomicAdd(a.evals, evals);
}

// ---------------------------------------------------------------- pose-regression walks (Example 3)
// Hypothesis i constrains the rotation, |R - R_i|_F <= beta_i^R, and the translation,
// |t - t_i| <= beta_i^t.  A dS_R perturbation moves only t and a dS_t perturbation only R, so the
// part that stays is evaluated once per iteration and the distance of perturbation j (eq. 11) is
// min(that part's minimum margin, min_i of the moving part's margins); in_purse of a ladder
// candidate (k, m) is the product of a factor of k and a factor of m (dS_R: the rung's rotation
// and the kept perturbation's translation; dS_t the other way round), so the ladder evaluates
// N_T + N_P* half-constraint sets, one rung and one kept perturbation per lane, and m0 / k0 are
// the first set bits of the two warp ballots.  The same draws, decisions and trace as the
// per-operation samplers.  Table (4 rows per hypothesis): [0, N) (t_i, beta_i^t), [N + r N + i)
// row r of R_i with beta_i^R in the w of row 0.
template <typename T>
__host__ __device__ inline size_t reg_table_bytes(int n) {
  return align_up(16 * (size_t)n * sizeof(T), 128);
}
template <typename T>
__host__ __device__ inline size_t reg_slab_bytes(int n, int n_perturb) {
  const size_t t4 = 4 * sizeof(T);
  return align_up((size_t)n * t4 + (size_t)n_perturb * t4 + (size_t)n_perturb * sizeof(typename KeyOf<T>::type) +
                      32 * sizeof(int),
                  128);
}

// |R - R_i|_F^2 of hypothesis i (the order of the per-operation samplers).
template <typename T>
__device__ __forceinline__ T reg_rot_d2(const T4<T>* tab, int N, int i, const M3<T>& R) {
  const T4<T> r0 = tab[N + i], r1 = tab[2 * N + i], r2 = tab[3 * N + i];
  const T g[9] = {r0.x, r0.y, r0.z, r1.x, r1.y, r1.z, r2.x, r2.y, r2.z};
  T d2 = T(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const T d = R.m[k] - g[k];
    d2 += d * d;
  }
  return d2;
}
template <typename T>
__device__ __forceinline__ T reg_trans_e2(const T4<T>* tab, int i, const V3<T>& t) {
  const T4<T> ti = tab[i];
  const T ex = t.x - ti.x, ey = t.y - ti.y, ez = t.z - ti.z;
  return ex * ex + ey * ey + ez * ez;
}
template <typename T>
__device__ __forceinline__ bool reg_rot_ok(const T4<T>* tab, int N, const M3<T>& R) {
  bool ok = true;
  for (int i = 0; i < N; ++i) {
    const T b = tab[N + i].w;
    ok = ok && reg_rot_d2(tab, N, i, R) <= b * b;
  }
  return ok;
}
template <typename T>
__device__ __forceinline__ bool reg_trans_ok(const T4<T>* tab, int N, const V3<T>& t) {
  bool ok = true;
  for (int i = 0; i < N; ++i) {
    const T b = tab[i].w;
    ok = ok && reg_trans_e2(tab, i, t) <= b * b;
  }
  return ok;
}

template <typename T, int SAMPLER, class RK>
__device__ __forceinline__ void reg_walk_one(const WalkCtx<T>& c, const RK& rk, int w, const T4<T>* tab, T4<T>* C,
                                             const Slab<T>& sl, int lane, unsigned long long& evals) {
  using Key = typename KeyOf<T>::type;
  using T2 = P2<T>;
  const int N = c.N, NP = c.NP, K = c.K, NT = c.NT;
  const T r_pert = c.r_pert;
  Q4<T> q;
  V3<T> t;
  V3<T> vel;
  walk_start<T, SAMPLER>(c, w, q, t, vel);
  T sm = T(1);  // this lane's rung scale gamma^lane
  for (int k = 0; k < lane; ++k) sm *= c.gam;
  bool moved = true;
  T fixed_min = inf<T>();  // minimum margin of the part the perturbations do not move
  for (int it = 0; it < c.n_iter; ++it) {
    const M3<T> R = qmat(q);
    if (moved) {
      T mn = inf<T>();
      for (int i = lane; i < N; i += 32) {
        if (SAMPLER == 0) {  // rotation margins of R*; the translation offsets t* - t_i
          mn = fmin(mn, tab[N + i].w - sqrt(reg_rot_d2(tab, N, i, R)));
          const T4<T> ti = tab[i];
          C[i] = T4<T>{t.x - ti.x, t.y - ti.y, t.z - ti.z, ti.w};
        } else {             // translation margins of t*
          mn = fmin(mn, tab[i].w - sqrt(reg_trans_e2(tab, i, t)));
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) mn = fmin(mn, __shfl_xor_sync(kFullMask, mn, o));
      fixed_min = mn;
      evals += (unsigned long long)N;
      __syncwarp();
    }
    // ---- perturbations and their distance (eq. 11), two per lane and pass on paired lanes
    const T2 tiny2 = dup(tiny<T>());
    for (int b = lane; 2 * b < NP; b += 32) {
      const uint4 wd = philox4x32_10_rk(
          make_uint4(0u, ((SAMPLER == 0 ? kPhaseRPerturb : kPhaseTPerturb) << 24) | (uint32_t)b, (uint32_t)it,
                     (uint32_t)w),
          rk);
      T2 dmin = dup(inf<T>());
      if constexpr (SAMPLER == 0) {
        T dx[2], dy[2], dz[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          T ux, uy, uz;
          hatbox_point<T>(h ? wd.z : wd.x, h ? wd.w : wd.y, ux, uy, uz);
          dx[h] = r_pert * ux, dy[h] = r_pert * uy, dz[h] = r_pert * uz;
          if (2 * b + h < NP) sl.P[2 * b + h] = T4<T>{dx[h], dy[h], dz[h], T(0)};
        }
        const T2 Dx = pr(dx[0], dx[1]), Dy = pr(dy[0], dy[1]), Dz = pr(dz[0], dz[1]);
        for (int i = 0; i < N; ++i) {
          const T4<T> ci = C[i];
          const T2 ex = add2(dup(ci.x), Dx), ey = add2(dup(ci.y), Dy), ez = add2(dup(ci.z), Dz);
          const T2 s2 = fma2(ez, ez, fma2(ey, ey, mul2(ex, ex)));
          dmin = min2(dmin, fma2(pr(-s2.x, -s2.y), rsq2(add2(s2, tiny2)), dup(ci.w)));
        }
      } else {
        T2 qw, qx, qy, qz, A[9], Rj[9];
        hatbox_quat2<T>(wd, r_pert, qw, qx, qy, qz);
        if (2 * b < NP) sl.P[2 * b] = T4<T>{qw.x, qx.x, qy.x, qz.x};
        if (2 * b + 1 < NP) sl.P[2 * b + 1] = T4<T>{qw.y, qx.y, qy.y, qz.y};
        qmat2<T>(qw, qx, qy, qz, A);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc)
            Rj[3 * r + cc] = fma2(A[3 * r + 2], dup(R.m[6 + cc]),
                                  fma2(A[3 * r + 1], dup(R.m[3 + cc]), mul2(A[3 * r], dup(R.m[cc]))));
        for (int i = 0; i < N; ++i) {
          const T4<T> r0 = tab[N + i], r1 = tab[2 * N + i], r2 = tab[3 * N + i];
          const T g[9] = {r0.x, r0.y, r0.z, r1.x, r1.y, r1.z, r2.x, r2.y, r2.z};
          T2 d2 = dup(T(0));
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const T2 d = add2(Rj[k], dup(-g[k]));
            d2 = fma2(d, d, d2);
          }
          dmin = min2(dmin, fma2(pr(-d2.x, -d2.y), rsq2(add2(d2, tiny2)), dup(r0.w)));
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (2 * b + h < NP) sl.key[2 * b + h] = orderable(fmin(h ? dmin.y : dmin.x, fixed_min));
    }
    evals += (unsigned long long)NP * N;
    __syncwarp();
    // ---- top_k_indices (ties to the lower j)
    if (NP <= 160)
      top_k<Key, 5>(sl, NP, K, lane);
    else
      top_k<Key, 8>(sl, NP, K, lane);
    __syncwarp();
    // ---- ladder: rung m = lane and kept perturbation k = lane, each against its half of the constraints
    Q4<T> qm{T(1), T(0), T(0), T(0)};  // dS_R: the rung's rotation; dS_t: the kept perturbation's
    V3<T> tm = t;                       // dS_R: the kept perturbation's translation; dS_t: the rung's
    bool ok_m = false, ok_k = false;
    if (lane < NT) {
      if (SAMPLER == 0) {
        qm = qnormalize(qmul(qexp(V3<T>{sm * vel.x, sm * vel.y, sm * vel.z}), q));
        ok_m = reg_rot_ok(tab, N, qmat(qm));
      } else {
        tm = V3<T>{t.x + sm * vel.x, t.y + sm * vel.y, t.z + sm * vel.z};
        ok_m = reg_trans_ok(tab, N, tm);
      }
    }
    Q4<T> qk{T(1), T(0), T(0), T(0)};
    V3<T> tk = t;
    if (lane < K) {
      const T4<T> pj = sl.P[sl.J[lane]];
      if (SAMPLER == 0) {
        tk = V3<T>{t.x + pj.x, t.y + pj.y, t.z + pj.z};
        ok_k = reg_trans_ok(tab, N, tk);
      } else {
        qk = qnormalize(qmul(Q4<T>{pj.x, pj.y, pj.z, pj.w}, q));
        ok_k = reg_rot_ok(tab, N, qmat(qk));
      }
    }
    evals += (unsigned long long)(NT + K) * N;
    const unsigned bm = __ballot_sync(kFullMask, ok_m), bk = __ballot_sync(kFullMask, ok_k);
    int m0 = -1, k0 = -1;
    if (bm && bk) m0 = __ffs(bm) - 1, k0 = __ffs(bk) - 1;
    // ---- update (R*, t*): from lane m0 (the rung) and lane k0 (the kept perturbation)
    moved = m0 >= 0;
    if (moved) {
      const Q4<T> qr = SAMPLER == 0 ? qm : qk;
      const V3<T> tr = SAMPLER == 0 ? tk : tm;
      const int lq = SAMPLER == 0 ? m0 : k0, lt = SAMPLER == 0 ? k0 : m0;
      q = Q4<T>{__shfl_sync(kFullMask, qr.w, lq), __shfl_sync(kFullMask, qr.x, lq), __shfl_sync(kFullMask, qr.y, lq),
                __shfl_sync(kFullMask, qr.z, lq)};
      t = V3<T>{__shfl_sync(kFullMask, tr.x, lt), __shfl_sync(kFullMask, tr.y, lt), __shfl_sync(kFullMask, tr.z, lt)};
    }
    if (c.trace != nullptr && lane == 0) {
      int16_t* trc = c.trace + ((size_t)w * c.n_iter + it) * (K + 2);
      for (int r = 0; r < K; ++r) trc[r] = (int16_t)sl.J[r];
      trc[K] = (int16_t)m0;
      trc[K + 1] = (int16_t)k0;
    }
    __syncwarp();
  }
  if (lane == 0) {
    T* oq = c.out_q + 4 * (size_t)w;
    T* ot = c.out_t + 3 * (size_t)w;
    oq[0] = q.w, oq[1] = q.x, oq[2] = q.y, oq[3] = q.z;
    ot[0] = t.x, ot[1] = t.y, ot[2] = t.z;
    if (!(isfinite(q.w) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(t.x) && isfinite(t.y) &&
          isfinite(t.z)))
      atomicOr(c.status, kDevErrNumeric);
  }
  __syncwarp();
}

template <typename T, int SAMPLER>
__global__ void __launch_bounds__(kWalkThreads, sizeof(T) == 4 ? 2 : 1)
    reg_walk_kernel(const __grid_constant__ WalkArgs a, const int slab_bytes) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  const int N = a.n;
  const T4<T>* tab = reinterpret_cast<const T4<T>*>(smem + 128);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* slab = smem + 128 + reg_table_bytes<T>(N) + (size_t)warp * slab_bytes;
  T4<T>* C = reinterpret_cast<T4<T>*>(slab);
  Slab<T> sl;
  sl.D = nullptr, sl.L = nullptr, sl.E = nullptr, sl.S = nullptr;
  sl.P = C + N;
  sl.key = reinterpret_cast<typename KeyOf<T>::type*>(sl.P + a.n_perturb);
  sl.J = reinterpret_cast<int*>(sl.key + a.n_perturb);
  // ---- stage the hypotheses with a 1-D TMA bulk copy
  const uint32_t tbytes = 16u * N * sizeof(T);
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, tbytes);
    bulk_copy_g2s(smem + 128, a.table, tbytes, bar);
  }
  if (!mbar_wait_bounded(bar, 0, 1 << 22)) {
    // thread 0 gives the copies still in flight one more bounded wait, so that none lands in this
    // CTA's shared memory after it has exited
    if (threadIdx.x == 0) {
      atomicOr(a.status, kDevErrTimeout);
      mbar_wait_bounded(bar, 0, 1 << 22);
    }
    return;
  }
  if (a.stall_probe) {  // PURSE_FAULT=stall: a second barrier that nothing arrives at, short poll limit
    if (threadIdx.x == 0) mbar_init(bar + 1, 1);
    __syncthreads();
    if (!mbar_wait_bounded(bar + 1, 0, 1 << 10)) {
      if (threadIdx.x == 0) atomicOr(a.status, kDevErrTimeout);
      return;
    }
  }
  WalkCtx<T> c;
  c.N = N, c.NP = a.n_perturb, c.K = a.n_keep, c.NT = a.n_steps, c.mc = 1, c.n_iter = a.n_iter;
  c.fx = c.fy = c.cx = c.cy = T(0);
  c.rho_max = T(0);
  c.r_pert = T(SAMPLER == 0 ? a.stats->r_trans : a.stats->r_rot);
  c.omega0 = a.omega0, c.v0 = a.v0, c.gamma = a.gamma;
  c.om0 = T(a.omega0), c.vv0 = T(a.v0), c.gam = T(a.gamma);
  c.st = a.stats, c.seed_data = a.seed_data, c.s0 = a.s0;
  c.key0 = a.key0, c.key1 = a.key1;
  c.out_q = reinterpret_cast<T*>(a.out_q), c.out_t = reinterpret_cast<T*>(a.out_t);
  c.trace = a.trace, c.status = a.status;
  c.out_snap = nullptr;
  c.tab64 = nullptr, c.kd = nullptr, c.ell64 = nullptr;
  const RkParam rk{a};
  unsigned long long evals = 0;
  const int nw = blockDim.x >> 5;
  for (int w = blockIdx.x * nw + warp; w < a.n_samples; w += gridDim.x * nw)
    reg_walk_one<T, SAMPLER>(c, rk, w, tab, C, sl, lane, evals);
  if (lane == 0 && evals) atomicAdd(a.evals, evals);
}

// ---------------------------------------------------------------- batched walks (one persistent launch)
// Work item i = (PURSE p, sampler, walk w) with p = i / (2 S), sampler = (i / S) & 1, w = i mod S;
// the dS_t items of 3D-3D PURSEs are skipped (their two balls use the dS_R samples).  Each warp
// pops chunks of items from one atomic counter; the queue never waits, so the kernel ends when
// the counter passes the last item.  A warp stages the constraint table and Philox round keys of
// its current PURSE into its own shared-memory area when the PURSE changes.  With noise matrices
// (LAM) the warp's table holds the PURSE's factors U_i after its 2N rows, as in walk_kernel.
__host__ __device__ inline size_t batch_warp_bytes(int nmax, int n_perturb, int n_steps, bool lam = false) {
  return walk_table_bytes<float>(nmax, lam) + 128 + walk_slab_bytes2<float>(nmax, n_perturb, n_steps, lam);
}

// Pose-regression batches: the warp's hypothesis table (4N rows), round keys, then reg_walk_one's slab.
__host__ __device__ inline size_t batch_reg_warp_bytes(int nmax, int n_perturb) {
  return reg_table_bytes<float>(nmax) + 128 + reg_slab_bytes<float>(nmax, n_perturb);
}

size_t batch_walk_smem(int nmax, int n_perturb, int n_steps, int warps, bool lam, bool reg) {
  return (size_t)warps * (reg ? batch_reg_warp_bytes(nmax, n_perturb) : batch_warp_bytes(nmax, n_perturb, n_steps, lam));
}

// TR3D: the 3D-3D dS_t walks run too (b.tr3d); a separate instantiation so that batches without
// them keep the smaller kernel.  LAM: the batch carries noise matrices (eq. 4).
template <bool TR3D, bool LAM>
__global__ void __launch_bounds__(kWalkThreads, 2)
    batch_walk_kernel(const __grid_constant__ BatchArgs b, const int chunk, const int np_max, const int nt_max) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem + (size_t)warp * batch_warp_bytes(b.nmax, np_max, nt_max, LAM);
  T4<float>* tab = reinterpret_cast<T4<float>*>(base);
  uint32_t* rkw = reinterpret_cast<uint32_t*>(base + walk_table_bytes<float>(b.nmax, LAM));
  unsigned char* slab_base = base + walk_table_bytes<float>(b.nmax, LAM) + 128;
  const unsigned S = (unsigned)b.n_samples;
  const unsigned long long seed = *b.seed;
  unsigned long long evals = 0;
  int cur = -1;
  WalkCtx<float> c;
  Slab<float> sl;
  const RkPtr rk{rkw};
  for (;;) {
    unsigned head = 0;
    if (lane == 0) head = atomicAdd(b.counter, (unsigned)chunk);
    head = __shfl_sync(kFullMask, head, 0);
    if (head >= b.total_items) break;
    const unsigned end = min(head + (unsigned)chunk, b.total_items);
    for (unsigned item = head; item < end; ++item) {
      const int p = (int)(item / (2 * S));
      const int smp = (int)((item / S) & 1u);
      const int w = (int)(item % S);
      const BatchPurseInfo in = b.info[p];
      if (in.kind == 0 && smp == 1 && !TR3D) continue;
      if (p != cur) {
        __syncwarp();
        const T4<float>* src = reinterpret_cast<const T4<float>*>(b.table) + in.table_off;
        for (int r = lane; r < 2 * in.n; r += 32) tab[r] = src[r];
        if constexpr (LAM) {  // rows [2N, 4N): U_i, two rows of 4 floats per keypoint
          const T4<float>* us = reinterpret_cast<const T4<float>*>(b.ell) + in.table_off;
          for (int r = lane; r < 2 * in.n; r += 32) tab[2 * in.n + r] = us[r];
        }
        const unsigned long long key = seed + (unsigned long long)p;
        if (lane < 10) {
          rkw[2 * lane] = (uint32_t)key + (uint32_t)lane * 0x9E3779B9u;
          rkw[2 * lane + 1] = (uint32_t)(key >> 32) + (uint32_t)lane * 0xBB67AE85u;
        }
        const int kd = in.kind;
        c.N = in.n, c.NP = b.n_perturb[kd], c.K = b.n_keep[kd], c.NT = b.n_steps[kd], c.n_iter = b.n_iter[kd];
        c.mc = c.K >= 32 ? 1 : 32 / c.K;
        c.fx = float(in.fx), c.fy = float(in.fy), c.cx = float(in.cx), c.cy = float(in.cy);
        c.rho_max = float(in.rho_max);
        c.omega0 = b.omega0[kd], c.v0 = b.v0[kd], c.gamma = b.gamma[kd];
        c.om0 = float(b.omega0[kd]), c.vv0 = float(b.v0[kd]), c.gam = float(b.gamma[kd]);
        c.st = b.stats + p, c.seed_data = b.seed_data + (size_t)p * kSeedStride, c.s0 = 1;
        c.key0 = (uint32_t)key, c.key1 = (uint32_t)(key >> 32);
        c.trace = nullptr, c.status = b.status;
        c.tab64 = b.table64 + 4 * (size_t)in.table_off, c.kd = &b.info[p].fx;
        c.ell64 = LAM ? b.ell64 + 4 * (size_t)in.table_off : nullptr;
        sl = carve<float, LAM>(slab_base, c.N, c.NP, c.NT);
        cur = p;
        __syncwarp();
      }
      c.r_pert = float(smp == 0 ? c.st->r_trans : c.st->r_rot);
      const size_t off = (size_t)p * S;
      c.out_q = (smp == 0 ? b.q_rot : b.q_tr) + 4 * off;
      c.out_t = (smp == 0 ? b.t_rot : b.t_tr) + 3 * off;
      float* snap = smp == 0 ? b.snap_rot : b.snap_tr;
      c.out_snap = snap ? snap + (size_t)kSnapStride * off : nullptr;
      if (in.kind == 0 && smp == 0)
        walk_one<float, 0, 0, LAM>(c, rk, w, tab, sl, lane, evals);
      else if (in.kind == 0) {
        if constexpr (TR3D) walk_one<float, 0, 1, LAM>(c, rk, w, tab, sl, lane, evals);
      }
      else if (smp == 0)
        walk_one<float, 1, 0, LAM>(c, rk, w, tab, sl, lane, evals);
      else
        walk_one<float, 1, 1, LAM>(c, rk, w, tab, sl, lane, evals);
    }
  }
  if (lane == 0 && evals) atomicAdd(b.evals, evals);
}

// Batches of pose-regression PURSEs (Example 3): the same work queue over (PURSE, sampler, walk)
// items, both samplers for every PURSE, each walk run by reg_walk_one (the walk of reg_walk_kernel).
__global__ void __launch_bounds__(kWalkThreads, 2)
    batch_reg_walk_kernel(const __grid_constant__ BatchArgs b, const int chunk, const int np_max) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem + (size_t)warp * batch_reg_warp_bytes(b.nmax, np_max);
  T4<float>* tab = reinterpret_cast<T4<float>*>(base);
  uint32_t* rkw = reinterpret_cast<uint32_t*>(base + reg_table_bytes<float>(b.nmax));
  T4<float>* C = reinterpret_cast<T4<float>*>(base + reg_table_bytes<float>(b.nmax) + 128);
  const unsigned S = (unsigned)b.n_samples;
  const unsigned long long seed = *b.seed;
  unsigned long long evals = 0;
  int cur = -1;
  WalkCtx<float> c;
  Slab<float> sl;
  sl.D = nullptr, sl.L = nullptr, sl.E = nullptr, sl.S = nullptr;
  const RkPtr rk{rkw};
  for (;;) {
    unsigned head = 0;
    if (lane == 0) head = atomicAdd(b.counter, (unsigned)chunk);
    head = __shfl_sync(kFullMask, head, 0);
    if (head >= b.total_items) break;
    const unsigned end = min(head + (unsigned)chunk, b.total_items);
    for (unsigned item = head; item < end; ++item) {
      const int p = (int)(item / (2 * S));
      const int smp = (int)((item / S) & 1u);
      const int w = (int)(item % S);
      if (p != cur) {
        const BatchPurseInfo in = b.info[p];
        __syncwarp();
        const T4<float>* src = reinterpret_cast<const T4<float>*>(b.table) + in.table_off;
        for (int r = lane; r < 4 * in.n; r += 32) tab[r] = src[r];
        const unsigned long long key = seed + (unsigned long long)p;
        if (lane < 10) {
          rkw[2 * lane] = (uint32_t)key + (uint32_t)lane * 0x9E3779B9u;
          rkw[2 * lane + 1] = (uint32_t)(key >> 32) + (uint32_t)lane * 0xBB67AE85u;
        }
        c.N = in.n, c.NP = b.n_perturb[0], c.K = b.n_keep[0], c.NT = b.n_steps[0], c.n_iter = b.n_iter[0], c.mc = 1;
        c.fx = c.fy = c.cx = c.cy = 0.0f;
        c.rho_max = 0.0f;
        c.omega0 = b.omega0[0], c.v0 = b.v0[0], c.gamma = b.gamma[0];
        c.om0 = float(b.omega0[0]), c.vv0 = float(b.v0[0]), c.gam = float(b.gamma[0]);
        c.st = b.stats + p, c.seed_data = b.seed_data + (size_t)p * kSeedStride, c.s0 = 1;
        c.key0 = (uint32_t)key, c.key1 = (uint32_t)(key >> 32);
        c.trace = nullptr, c.status = b.status, c.out_snap = nullptr;
        c.tab64 = nullptr, c.kd = nullptr, c.ell64 = nullptr;
        sl.P = C + in.n;
        sl.key = reinterpret_cast<uint32_t*>(sl.P + c.NP);
        sl.J = reinterpret_cast<int*>(sl.key + c.NP);
        cur = p;
        __syncwarp();
      }
      c.r_pert = float(smp == 0 ? c.st->r_trans : c.st->r_rot);
      const size_t off = (size_t)p * S;
      c.out_q = (smp == 0 ? b.q_rot : b.q_tr) + 4 * off;
      c.out_t = (smp == 0 ? b.t_rot : b.t_tr) + 3 * off;
      if (smp == 0)
        reg_walk_one<float, 0>(c, rk, w, tab, C, sl, lane, evals);
      else
        reg_walk_one<float, 1>(c, rk, w, tab, C, sl, lane, evals);
    }
  }
  if (lane == 0 && evals) atomicAdd(b.evals, evals);
}

static cudaError_t launch_batch_reg_walk(const BatchArgs& b, int chunk, int warps, int sm_count, cudaStream_t st) {
  const int np_max = b.n_perturb[0];
  const size_t smem = batch_walk_smem(b.nmax, np_max, b.n_steps[0], warps, false, true);
  cudaError_t e = cudaFuncSetAttribute(batch_reg_walk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_reg_walk_kernel, 32 * warps, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  batch_reg_walk_kernel<<<per_sm * sm_count, 32 * warps, smem, st>>>(b, chunk, np_max);
  return cudaGetLastError();
}

template <bool TR3D, bool LAM>
static cudaError_t launch_batch_walk_t(const BatchArgs& b, int chunk, int warps, int sm_count, cudaStream_t st) {
  const int np_max = max(b.n_perturb[0], b.n_perturb[1]), nt_max = max(b.n_steps[0], b.n_steps[1]);
  const size_t smem = batch_walk_smem(b.nmax, np_max, nt_max, warps, LAM);
  auto kern = batch_walk_kernel<TR3D, LAM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  kern<<<per_sm * sm_count, 32 * warps, smem, st>>>(b, chunk, np_max, nt_max);
  return cudaGetLastError();
}

cudaError_t launch_batch_walk(const BatchArgs& b, int chunk, int warps, int sm_count, cudaStream_t st) {
  if (b.reg) return launch_batch_reg_walk(b, chunk, warps, sm_count, st);
  if (b.ell)
    return b.tr3d ? launch_batch_walk_t<true, true>(b, chunk, warps, sm_count, st)
                  : launch_batch_walk_t<false, true>(b, chunk, warps, sm_count, st);
  return b.tr3d ? launch_batch_walk_t<true, false>(b, chunk, warps, sm_count, st)
                : launch_batch_walk_t<false, false>(b, chunk, warps, sm_count, st);
}

template <typename T, int KIND, int SAMPLER, bool LAM>
static cudaError_t launch_walk_t(purse_t h, const purse_params* p, const WalkArgs& a, cudaStream_t st) {
  const int mc = p->n_keep >= 32 ? 1 : 32 / p->n_keep;
  const size_t slab = walk_slab_bytes2<T>(a.n, p->n_perturb, p->n_steps, LAM);
  const size_t table = walk_table_bytes<T>(a.n, LAM);
  // warps per block: the tuned choice (8 by default), no more than the shared memory holds slabs for
  int warps = tuned_config(kTuneWalk, h->kind, a.n, a.n_samples, p->sampler + 2 * p->precision, kWalkWarps);
  warps = warps < 1 ? 1 : warps > kWalkWarps ? kWalkWarps : warps;
  while (warps > 1 && 128 + table + warps * slab > kMaxSmemPerBlock) --warps;
  const size_t smem = 128 + table + warps * slab;
  if (smem > kMaxSmemPerBlock) return cudaErrorInvalidConfiguration;
  auto kern = walk_kernel<T, KIND, SAMPLER, LAM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long need = (a.n_samples + warps - 1) / warps;
  const long cap = (long)per_sm * h->sm_count;
  const int grid = (int)(need < cap ? need : cap);
  kern<<<grid, 32 * warps, smem, st>>>(a, mc, (int)slab);
  return cudaGetLastError();
}

template <bool LAM>
static cudaError_t launch_walk_l(purse_t h, const purse_params* p, const WalkArgs& a, cudaStream_t st) {
  const bool dbl = p->precision == 1;
  const int kind = h->kind, smp = p->sampler;
  if (!dbl) {
    if (kind == 0)
      return smp == 0 ? launch_walk_t<float, 0, 0, LAM>(h, p, a, st) : launch_walk_t<float, 0, 1, LAM>(h, p, a, st);
    return smp == 0 ? launch_walk_t<float, 1, 0, LAM>(h, p, a, st) : launch_walk_t<float, 1, 1, LAM>(h, p, a, st);
  }
  if (kind == 0)
    return smp == 0 ? launch_walk_t<double, 0, 0, LAM>(h, p, a, st) : launch_walk_t<double, 0, 1, LAM>(h, p, a, st);
  return smp == 0 ? launch_walk_t<double, 1, 0, LAM>(h, p, a, st) : launch_walk_t<double, 1, 1, LAM>(h, p, a, st);
}

template <typename T, int SAMPLER>
static cudaError_t launch_reg_walk_t(purse_t h, const purse_params* p, const WalkArgs& a, cudaStream_t st) {
  const size_t slab = reg_slab_bytes<T>(a.n, p->n_perturb);
  const size_t table = reg_table_bytes<T>(a.n);
  int warps = tuned_config(kTuneWalk, h->kind, a.n, a.n_samples, p->sampler + 2 * p->precision, kWalkWarps);
  warps = warps < 1 ? 1 : warps > kWalkWarps ? kWalkWarps : warps;
  while (warps > 1 && 128 + table + warps * slab > kMaxSmemPerBlock) --warps;
  const size_t smem = 128 + table + warps * slab;
  if (smem > kMaxSmemPerBlock) return cudaErrorInvalidConfiguration;
  auto kern = reg_walk_kernel<T, SAMPLER>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long need = (a.n_samples + warps - 1) / warps;
  const long cap = (long)per_sm * h->sm_count;
  const int grid = (int)(need < cap ? need : cap);
  kern<<<grid, 32 * warps, smem, st>>>(a, (int)slab);
  return cudaGetLastError();
}

cudaError_t launch_walk(purse_t h, const purse_params* p, const WalkArgs& a, cudaStream_t st) {
  if (h->kind == PURSE_REG) {
    if (p->precision == 1)
      return p->sampler == 0 ? launch_reg_walk_t<double, 0>(h, p, a, st) : launch_reg_walk_t<double, 1>(h, p, a, st);
    return p->sampler == 0 ? launch_reg_walk_t<float, 0>(h, p, a, st) : launch_reg_walk_t<float, 1>(h, p, a, st);
  }
  return a.ell ? launch_walk_l<true>(h, p, a, st) : launch_walk_l<false>(h, p, a, st);
}

}  // namespace purse
