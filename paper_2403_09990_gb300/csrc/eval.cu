// Constraint evaluation for arbitrary poses: margins r_i - |g_i| (eq. 2/3),
// the active constraint of dist(R, t, dS) (eq. 11) and the SE(3) gradient of
// its residual norm under R <- Exp(phi) R, t <- t + rho.  One thread per pose.
#include "dev.cuh"
#include "internal.h"

namespace purse {

template <typename T, int KIND>
__global__ void __launch_bounds__(256)
    eval_kernel(const T* __restrict__ tab, int n, T fx, T fy, T cx, T cy, const T* __restrict__ poses, int n_poses,
                T* margin, int32_t* active, T* grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_poses) return;
  const T* ps = poses + 12 * (size_t)p;
  M3<T> R;
  for (int k = 0; k < 9; ++k) R.m[k] = ps[k];
  const V3<T> t{ps[9], ps[10], ps[11]};
  T best = T(INFINITY);
  int bi = 0;
  for (int i = 0; i < n; ++i) {
    const T* a = tab + 4 * i;
    const T* o = tab + 4 * (n + i);
    const V3<T> X = mul(R, V3<T>{a[0], a[1], a[2]}) + t;
    T m;
    if (KIND == 0) {
      const V3<T> e = X - V3<T>{o[0], o[1], o[2]};
      m = a[3] - sqrt(dot(e, e));
    } else {
      const T Pz = X.z;
      if (Pz > T(0)) {
        const T u = (fx * X.x + cx * X.z) / Pz, v = (fy * X.y + cy * X.z) / Pz;
        const T gu = o[0] - u, gv = o[1] - v;
        m = a[3] - sqrt(gu * gu + gv * gv);
      } else {
        m = -T(INFINITY);
      }
    }
    if (margin) margin[(size_t)p * n + i] = m;
    if (m < best || i == 0) best = m, bi = i;
  }
  if (active) active[p] = bi;
  if (!grad) return;
  T* g = grad + 6 * (size_t)p;
  for (int k = 0; k < 6; ++k) g[k] = T(0);
  const T* a = tab + 4 * bi;
  const T* o = tab + 4 * (n + bi);
  const V3<T> RA = mul(R, V3<T>{a[0], a[1], a[2]});
  const V3<T> X = RA + t;
  V3<T> wv;  // d|g| / d(translation of the transformed point)
  if (KIND == 0) {
    const V3<T> e = X - V3<T>{o[0], o[1], o[2]};
    const T nrm = sqrt(dot(e, e));
    if (!(nrm > T(0))) return;
    wv = (T(1) / nrm) * e;
  } else {
    const T Px = fx * X.x + cx * X.z, Py = fy * X.y + cy * X.z, Pz = X.z;
    if (!(Pz > T(0))) return;
    const T e0 = Px / Pz - o[0], e1 = Py / Pz - o[1];
    const T nrm = sqrt(e0 * e0 + e1 * e1);
    if (!(nrm > T(0))) return;
    const T n0 = e0 / nrm, n1 = e1 / nrm;
    // J_pi^T n, then K^T
    const V3<T> jn{n0 / Pz, n1 / Pz, -(Px * n0 + Py * n1) / (Pz * Pz)};
    wv = V3<T>{fx * jn.x, fy * jn.y, cx * jn.x + cy * jn.y + jn.z};
  }
  const V3<T> gphi = cross(RA, wv);
  g[0] = gphi.x, g[1] = gphi.y, g[2] = gphi.z;
  g[3] = wv.x, g[4] = wv.y, g[5] = wv.z;
}

cudaError_t launch_eval(purse_t h, int precision, const void* d_poses, int n_poses, void* d_margin,
                        int32_t* d_active, void* d_grad, cudaStream_t st) {
  const int threads = 256, blocks = (n_poses + threads - 1) / threads;
  if (n_poses == 0) return cudaSuccess;
  if (precision == 0) {
    auto k = h->kind == 0 ? eval_kernel<float, 0> : eval_kernel<float, 1>;
    k<<<blocks, threads, 0, st>>>(h->tables.f32, h->n, (float)h->K.fx, (float)h->K.fy, (float)h->K.cx,
                                  (float)h->K.cy, (const float*)d_poses, n_poses, (float*)d_margin, d_active,
                                  (float*)d_grad);
  } else {
    auto k = h->kind == 0 ? eval_kernel<double, 0> : eval_kernel<double, 1>;
    k<<<blocks, threads, 0, st>>>(h->tables.f64, h->n, h->K.fx, h->K.fy, h->K.cx, h->K.cy, (const double*)d_poses,
                                  n_poses, (double*)d_margin, d_active, (double*)d_grad);
  }
  return cudaGetLastError();
}

}  // namespace purse
