// Device-side building blocks of the CLOSURE hot path (sm_103a).
//
// * Philox4x32-10 (Salmon et al., SC'11) and the named random streams the
//   walks draw from, with the one-word lattice rejection draw of a point in
//   the unit ball (uniform perturbations, Section IV Step II).
// * Small fixed-size vector / quaternion / rotation algebra templated on the
//   arithmetic type (float for the FP32 path, double for FP64).
// * TMA 1-D bulk copy + mbarrier helpers (inline PTX) with bounded waits.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace purse {

constexpr unsigned kFullMask = 0xffffffffu;

// Device status bits (the handle's status word).
constexpr int kDevErrTimeout = 1;
constexpr int kDevErrNumeric = 2;

// Random stream phases.
constexpr uint32_t kPhaseRPerturb = 1;
constexpr uint32_t kPhaseTPerturb = 2;
constexpr uint32_t kPhaseOmega = 3;
constexpr uint32_t kPhaseV = 4;
constexpr uint32_t kPhaseRansag = 5;
constexpr int kMaxAttempts = 64;

// ---------------------------------------------------------------- Philox
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1,
                   (uint32_t)p0);
  }
  return c;
}

// Philox4x32-10 with the ten round keys given (rk[2r], rk[2r+1]) = (k0 + r W0, k1 + r W1).
template <class RK>
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const RK& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1],
                   (uint32_t)p0);
  }
  return c;
}

__device__ __forceinline__ void sin_cos_pi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sin_cos_pi(double x, double* s, double* c) { sincospi(x, s, c); }

// Perturbation point from two words (no rejection): hat-box direction with
// z = ((w0 >> 16) + 1/2) 2^-15 - 1 and azimuth pi ((w0 & 0xFFFF) + 1/2) 2^-15, radius
// (max of the three 10-bit fields of w1 + 1/2) 2^-10, whose cube is uniform; so the
// point is uniform in the unit ball.  z, the azimuth fraction and the radius are exact.
template <typename T>
__device__ __forceinline__ void hatbox_point(uint32_t w0, uint32_t w1, T& x, T& y, T& z) {
  const T zz = T((int)(w0 >> 16)) * T(1.0 / 32768) + T(0.5 / 32768 - 1.0);
  const T az = T((int)(w0 & 0xFFFFu)) * T(1.0 / 32768) + T(0.5 / 32768);
  const uint32_t k = max(max(w1 & 1023u, (w1 >> 10) & 1023u), (w1 >> 20) & 1023u);
  const T rho = T((int)k) * T(1.0 / 1024) + T(0.5 / 1024);
  T sp, cp, s;
  const T c2 = T(1) - zz * zz;  // >= 2^-15
  if constexpr (sizeof(T) == 4) {
    // hardware sine/cosine and reciprocal square root: absolute errors ~1e-6 of a unit
    // perturbation direction, far below what changes any walk decision
    __sincosf(3.14159265358979f * az, &sp, &cp);
    s = rho * c2 * rsqrtf(c2);
  } else {
    sin_cos_pi(az, &sp, &cp);
    s = rho * sqrt(c2);
  }
  x = s * cp, y = s * sp, z = rho * zz;
}

// Words of the stream named (phase, j, i, w) under key (k0, k1), in order.
struct Stream {
  uint32_t k0, k1, c1, c2, c3, block;
  uint4 buf;
  int pos;
  __device__ __forceinline__ Stream(uint32_t key0, uint32_t key1, uint32_t phase, uint32_t j, uint32_t i,
                                    uint32_t w)
      : k0(key0), k1(key1), c1((phase << 24) | j), c2(i), c3(w), block(0), pos(4) {}
  __device__ __forceinline__ uint32_t next() {
    if (pos == 4) {
      buf = philox4x32_10(make_uint4(block++, c1, c2, c3), k0, k1);
      pos = 0;
    }
    const uint32_t v = pos == 0 ? buf.x : pos == 1 ? buf.y : pos == 2 ? buf.z : buf.w;
    ++pos;
    return v;
  }
};

// First accepted lattice point of the stream: X_c = 2 ((word >> 10c) & 1023) - 1023,
// accepted when |X|^2 <= 2^20 (and >= 2^14 for unit vectors).  Returns false
// (and X = 0) when every attempt was rejected.
template <bool kUnit>
__device__ __forceinline__ bool lattice_draw(Stream& s, int& x, int& y, int& z) {
  for (int a = 0; a < kMaxAttempts; ++a) {
    const uint32_t wd = s.next();
    const int X = 2 * (int)(wd & 1023u) - 1023;
    const int Y = 2 * (int)((wd >> 10) & 1023u) - 1023;
    const int Z = 2 * (int)((wd >> 20) & 1023u) - 1023;
    const int r2 = X * X + Y * Y + Z * Z;  // <= 3 * 1023^2 < 2^31
    const bool ok = kUnit ? (r2 <= (1 << 20) && r2 >= (1 << 14)) : (r2 <= (1 << 20));
    if (ok) {
      x = X, y = Y, z = Z;
      return true;
    }
  }
  x = y = z = 0;
  return false;
}

// ---------------------------------------------------------------- small algebra
template <typename T>
struct V3 {
  T x, y, z;
};
template <typename T>
struct Q4 {
  T w, x, y, z;
};
template <typename T>
struct M3 {
  T m[9];  // row-major
};

template <typename T>
__host__ __device__ __forceinline__ V3<T> v3(T x, T y, T z) {
  return V3<T>{x, y, z};
}
template <typename T>
__host__ __device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) {
  return v3(a.x + b.x, a.y + b.y, a.z + b.z);
}
template <typename T>
__host__ __device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) {
  return v3(a.x - b.x, a.y - b.y, a.z - b.z);
}
template <typename T>
__host__ __device__ __forceinline__ V3<T> operator*(T s, V3<T> a) {
  return v3(s * a.x, s * a.y, s * a.z);
}
template <typename T>
__host__ __device__ __forceinline__ T dot(V3<T> a, V3<T> b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename T>
__host__ __device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <typename T>
__host__ __device__ __forceinline__ V3<T> mul(const M3<T>& R, V3<T> a) {
  return v3(R.m[0] * a.x + R.m[1] * a.y + R.m[2] * a.z, R.m[3] * a.x + R.m[4] * a.y + R.m[5] * a.z,
            R.m[6] * a.x + R.m[7] * a.y + R.m[8] * a.z);
}
template <typename T>
__host__ __device__ __forceinline__ M3<T> mul(const M3<T>& A, const M3<T>& B) {
  M3<T> C;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      C.m[3 * r + c] = A.m[3 * r] * B.m[c] + A.m[3 * r + 1] * B.m[3 + c] + A.m[3 * r + 2] * B.m[6 + c];
  return C;
}

// Hamilton product.
template <typename T>
__host__ __device__ __forceinline__ Q4<T> qmul(Q4<T> p, Q4<T> q) {
  return Q4<T>{p.w * q.w - p.x * q.x - p.y * q.y - p.z * q.z, p.w * q.x + q.w * p.x + p.y * q.z - p.z * q.y,
               p.w * q.y + q.w * p.y + p.z * q.x - p.x * q.z, p.w * q.z + q.w * p.z + p.x * q.y - p.y * q.x};
}

template <typename T>
__device__ __forceinline__ Q4<T> qnormalize(Q4<T> q) {
  T n = sqrt(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
  T s = (q.w < T(0) ? T(-1) : T(1)) / n;
  return Q4<T>{q.w * s, q.x * s, q.y * s, q.z * s};
}

template <typename T>
__host__ __device__ __forceinline__ M3<T> qmat(Q4<T> q) {
  const T w = q.w, x = q.x, y = q.y, z = q.z;
  M3<T> R;
  R.m[0] = T(1) - T(2) * (y * y + z * z);
  R.m[1] = T(2) * (x * y - z * w);
  R.m[2] = T(2) * (x * z + y * w);
  R.m[3] = T(2) * (x * y + z * w);
  R.m[4] = T(1) - T(2) * (x * x + z * z);
  R.m[5] = T(2) * (y * z - x * w);
  R.m[6] = T(2) * (x * z - y * w);
  R.m[7] = T(2) * (y * z + x * w);
  R.m[8] = T(1) - T(2) * (x * x + y * y);
  return R;
}

__device__ __forceinline__ void sin_cos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sin_cos(double x, double* s, double* c) { sincos(x, s, c); }

// sin and cos of a small angle: for |x| <= 1/4 the Taylor series through x^7 and x^8 (the first
// omitted terms, x^9/9! and x^10/10!, are below 1.1e-11 there), else the library sincos.
template <typename T>
__device__ __forceinline__ void sincos_small(T x, T& s, T& c) {
  if (fabs(x) <= T(0.25)) {
    const T x2 = x * x;
    s = x * fma(-x2, fma(-x2, fma(-x2, T(1.0 / 5040), T(1.0 / 120)), T(1.0 / 6)), T(1));
    c = fma(-x2, fma(-x2, fma(-x2, fma(-x2, T(1.0 / 40320), T(1.0 / 720)), T(1.0 / 24)), T(0.5)), T(1));
  } else {
    sin_cos(x, &s, &c);
  }
}

// Exp(r u) as a unit quaternion for the perturbation point u of hatbox_point(w0, w1): u is rho
// times the unit direction (sqrt(1 - z^2) cos a, sqrt(1 - z^2) sin a, z), so the rotation angle
// is r rho and the axis that direction -- no norm and no division are formed.
template <typename T>
__device__ __forceinline__ Q4<T> hatbox_quat(uint32_t w0, uint32_t w1, T r) {
  const T zz = T((int)(w0 >> 16)) * T(1.0 / 32768) + T(0.5 / 32768 - 1.0);
  const T az = T((int)(w0 & 0xFFFFu)) * T(1.0 / 32768) + T(0.5 / 32768);
  const uint32_t k = max(max(w1 & 1023u, (w1 >> 10) & 1023u), (w1 >> 20) & 1023u);
  const T rho = T((int)k) * T(1.0 / 1024) + T(0.5 / 1024);
  const T c2 = T(1) - zz * zz;  // >= 2^-15
  T sp, cp, sq;
  if constexpr (sizeof(T) == 4) {
    __sincosf(3.14159265358979f * az, &sp, &cp);
    sq = c2 * rsqrtf(c2);
  } else {
    sin_cos_pi(az, &sp, &cp);
    sq = sqrt(c2);
  }
  T sh, ch;
  sincos_small(T(0.5) * r * rho, sh, ch);
  const T f = sh * sq;
  return Q4<T>{ch, f * cp, f * sp, sh * zz};
}

// Unit quaternion of the rotation vector v (Exp of so(3), Rodrigues).
template <typename T>
__device__ __forceinline__ Q4<T> qexp(V3<T> v) {
  const T th = sqrt(dot(v, v));
  T s, c;
  if (th < T(1e-12)) {
    return Q4<T>{T(1), T(0.5) * v.x, T(0.5) * v.y, T(0.5) * v.z};
  }
  sin_cos(T(0.5) * th, &s, &c);
  const T k = s / th;
  return Q4<T>{c, k * v.x, k * v.y, k * v.z};
}

// Unit quaternion (w >= 0) of a rotation matrix, Shepperd's branch choice.
__device__ __forceinline__ Q4<double> quat_from_mat(const double* M) {
  const double tr = M[0] + M[4] + M[8];
  Q4<double> q;
  if (tr >= M[0] && tr >= M[4] && tr >= M[8]) {
    const double s = 2.0 * sqrt(1.0 + tr);
    q = Q4<double>{0.25 * s, (M[7] - M[5]) / s, (M[2] - M[6]) / s, (M[3] - M[1]) / s};
  } else if (M[0] >= M[4] && M[0] >= M[8]) {
    const double s = 2.0 * sqrt(1.0 + M[0] - M[4] - M[8]);
    q = Q4<double>{(M[7] - M[5]) / s, 0.25 * s, (M[1] + M[3]) / s, (M[2] + M[6]) / s};
  } else if (M[4] >= M[8]) {
    const double s = 2.0 * sqrt(1.0 + M[4] - M[0] - M[8]);
    q = Q4<double>{(M[2] - M[6]) / s, (M[1] + M[3]) / s, 0.25 * s, (M[5] + M[7]) / s};
  } else {
    const double s = 2.0 * sqrt(1.0 + M[8] - M[0] - M[4]);
    q = Q4<double>{(M[3] - M[1]) / s, (M[2] + M[6]) / s, (M[5] + M[7]) / s, 0.25 * s};
  }
  return qnormalize(q);
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (n <= 4), FP64.
// A is destroyed (its diagonal holds the eigenvalues), V receives the eigenvectors as columns.
template <int n>
__device__ __forceinline__ void jacobi_eigen(double (&A)[n][n], double (&V)[n][n]) {
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) V[r][c] = r == c ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 16; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        tot += A[r][c] * A[r][c];
        if (r != c) off += A[r][c] * A[r][c];
      }
    if (off <= 1e-34 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p][q];
        if (apq == 0.0) continue;
        const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
}

// Rotation (as unit quaternion, w >= 0) maximising tr(R^T M): the eigenvector of the
// largest eigenvalue of Horn's symmetric 4 x 4 matrix.  Gives the nearest rotation to M
// (the projection onto SO(3)) and, with M = sum (b_i - b)(a_i - a)^T, the least-squares
// rotation of point pairs (the same optimum as Arun's SVD method).
__device__ __forceinline__ Q4<double> rotation_maximising_trace(const double* M) {
  double N[4][4], V[4][4];
  N[0][0] = M[0] + M[4] + M[8];
  N[1][1] = M[0] - M[4] - M[8];
  N[2][2] = -M[0] + M[4] - M[8];
  N[3][3] = -M[0] - M[4] + M[8];
  N[0][1] = N[1][0] = M[7] - M[5];
  N[0][2] = N[2][0] = M[2] - M[6];
  N[0][3] = N[3][0] = M[3] - M[1];
  N[1][2] = N[2][1] = M[1] + M[3];
  N[1][3] = N[3][1] = M[2] + M[6];
  N[2][3] = N[3][2] = M[5] + M[7];
  jacobi_eigen<4>(N, V);
  int best = 0;
  for (int k = 1; k < 4; ++k)
    if (N[k][k] > N[best][best]) best = k;
  return qnormalize(Q4<double>{V[0][best], V[1][best], V[2][best], V[3][best]});
}

// ---------------------------------------------------------------- paired arithmetic
// Two independent lanes of arithmetic per thread: float2 maps to the paired FP32
// instructions of sm_100+ (one issue slot for two FMAs), double2 to two scalar ops.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rsq2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ float2 min2(float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ float2 max2(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 rsq2(double2 a) { return make_double2(rsqrt(a.x), rsqrt(a.y)); }
__device__ __forceinline__ double2 min2(double2 a, double2 b) { return make_double2(fmin(a.x, b.x), fmin(a.y, b.y)); }
__device__ __forceinline__ double2 max2(double2 a, double2 b) { return make_double2(fmax(a.x, b.x), fmax(a.y, b.y)); }

template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};
template <typename T>
using P2 = typename Pair<T>::type;
template <typename T>
__device__ __forceinline__ P2<T> dup(T x) {
  return P2<T>{x, x};
}
template <typename T>
__device__ __forceinline__ P2<T> pr(T x, T y) {
  return P2<T>{x, y};
}

// The two perturbation quaternions of one Philox block -- points (words x, y) and (words z, w) of
// hatbox_quat -- with the floating-point work on paired lanes (.x the first point, .y the second).
template <typename T>
__device__ __forceinline__ void hatbox_quat2(uint4 wd, T r, P2<T>& qw, P2<T>& qx, P2<T>& qy, P2<T>& qz) {
  using T2 = P2<T>;
  const T zz0 = T((int)(wd.x >> 16)) * T(1.0 / 32768) + T(0.5 / 32768 - 1.0);
  const T zz1 = T((int)(wd.z >> 16)) * T(1.0 / 32768) + T(0.5 / 32768 - 1.0);
  const T az0 = T((int)(wd.x & 0xFFFFu)) * T(1.0 / 32768) + T(0.5 / 32768);
  const T az1 = T((int)(wd.z & 0xFFFFu)) * T(1.0 / 32768) + T(0.5 / 32768);
  const uint32_t k0 = max(max(wd.y & 1023u, (wd.y >> 10) & 1023u), (wd.y >> 20) & 1023u);
  const uint32_t k1 = max(max(wd.w & 1023u, (wd.w >> 10) & 1023u), (wd.w >> 20) & 1023u);
  const T2 rho = fma2(pr(T((int)k0), T((int)k1)), dup(T(1.0 / 1024)), dup(T(0.5 / 1024)));
  const T2 zz = pr(zz0, zz1);
  const T2 c2 = fma2(pr(-zz0, -zz1), zz, dup(T(1)));  // >= 2^-15
  T sp0, cp0, sp1, cp1;
  T2 sq;
  if constexpr (sizeof(T) == 4) {
    __sincosf(3.14159265358979f * az0, &sp0, &cp0);
    __sincosf(3.14159265358979f * az1, &sp1, &cp1);
    sq = mul2(c2, rsq2(c2));
  } else {
    sin_cos_pi(az0, &sp0, &cp0);
    sin_cos_pi(az1, &sp1, &cp1);
    sq = pr(sqrt(c2.x), sqrt(c2.y));
  }
  const T2 x = mul2(dup(T(0.5) * r), rho);  // half angles
  T2 sh, ch;
  if (fabs(x.x) <= T(0.25) && fabs(x.y) <= T(0.25)) {  // Taylor series as in sincos_small
    const T2 n2 = mul2(pr(-x.x, -x.y), x);
    sh = mul2(x, fma2(n2, fma2(n2, fma2(n2, dup(T(1.0 / 5040)), dup(T(1.0 / 120))), dup(T(1.0 / 6))), dup(T(1))));
    ch = fma2(n2, fma2(n2, fma2(n2, fma2(n2, dup(T(1.0 / 40320)), dup(T(1.0 / 720))), dup(T(1.0 / 24))),
                       dup(T(0.5))),
              dup(T(1)));
  } else {
    sincos_small(x.x, sh.x, ch.x);
    sincos_small(x.y, sh.y, ch.y);
  }
  const T2 f = mul2(sh, sq);
  qw = ch;
  qx = mul2(f, pr(cp0, cp1));
  qy = mul2(f, pr(sp0, sp1));
  qz = mul2(sh, zz);
}

// Rotation matrices (row-major) of two unit quaternions on paired lanes.
template <typename T>
__device__ __forceinline__ void qmat2(P2<T> w, P2<T> x, P2<T> y, P2<T> z, P2<T> (&m)[9]) {
  using T2 = P2<T>;
  const T2 two = dup(T(2)), m2 = dup(T(-2)), one = dup(T(1));
  const T2 xx = mul2(x, x), yy = mul2(y, y), zq = mul2(z, z);
  const T2 xy = mul2(x, y), xz = mul2(x, z), yz = mul2(y, z);
  const T2 nw = pr(-w.x, -w.y);
  m[0] = fma2(m2, add2(yy, zq), one);
  m[1] = mul2(two, fma2(nw, z, xy));
  m[2] = mul2(two, fma2(w, y, xz));
  m[3] = mul2(two, fma2(w, z, xy));
  m[4] = fma2(m2, add2(xx, zq), one);
  m[5] = mul2(two, fma2(nw, x, yz));
  m[6] = mul2(two, fma2(nw, y, xz));
  m[7] = mul2(two, fma2(w, x, yz));
  m[8] = fma2(m2, add2(xx, yy), one);
}

// Float keys ordered like the values they encode (for warp max reductions).
__device__ __forceinline__ uint32_t orderable(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ unsigned long long orderable(double f) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(f);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// ---------------------------------------------------------------- TMA / mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after max_tries polls and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, int max_tries) {
  for (int k = 0; k < max_tries; ++k)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

}  // namespace purse
