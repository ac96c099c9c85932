// Step III as the paper states it (Section IV, Step III): the exact minimum enclosing ball of
// the translation samples in R^3, and of the rotation samples embedded as unit quaternions in
// R^4 (each on the side of a reference rotation), its centre projected back to the unit sphere
// and the radius measured as the largest geodesic distance from it.
//
// Exact ball of up to 2^26 points: a candidate set C starts with the first sample; each round
// one pass over all samples finds the farthest from the exact ball of C (FP64 distances, block
// maxima, ties to the lower index), and if it lies outside that ball (beyond a relative 1e-12)
// it joins C and the exact ball of C is recomputed by Welzl's recursion on one thread (FP64,
// support sets of at most d + 1 points, circumballs by Gaussian elimination).  The ball of C
// never shrinks and every added point lies outside it, so the rounds end, in practice after a
// few dozen; when no sample lies outside, the ball of C is the ball of all samples.
#include <algorithm>
#include <cfloat>

#include "dev.cuh"
#include "internal.h"

namespace purse {

constexpr int kExactCap = 96;     // candidate points
constexpr int kExactThreads = 256;

struct ExactState {
  double c[4];    // centre of the exact ball of the candidates
  double r;       // its radius (-1: empty)
  double ref[4];  // reference quaternion (rotations)
  double far_d2;  // squared distance of the farthest sample in the last pass
  int n;          // candidates
  int done;       // the last pass found no sample outside the ball
  int overflow;   // the candidate set filled up before that
  int pad;
  double pts[kExactCap][4];
};

template <int DIM>
__device__ __forceinline__ double dist2(const double* a, const double* c) {
  double s = 0.0;
  for (int k = 0; k < DIM; ++k) s += (a[k] - c[k]) * (a[k] - c[k]);
  return s;
}

// Smallest ball with the points P[R[0..nr)] on its boundary, centre in their affine hull:
// c = P_0 + sum_k lam_k (P_k - P_0) with 2 (D D^T) lam = |D_k|^2 (D_k = P_k - P_0), solved by
// Gaussian elimination with partial pivoting; a pivot below 1e-14 of the diagonal scale (an
// affinely dependent point) leaves its coefficient 0.
template <int DIM>
__device__ __forceinline__ void circumball(const double (*P)[4], const int* R, int nr, double* c, double& r) {
  if (nr == 0) {
    for (int k = 0; k < DIM; ++k) c[k] = 0.0;
    r = -1.0;
    return;
  }
  const double* p0 = P[R[0]];
  for (int k = 0; k < DIM; ++k) c[k] = p0[k];
  r = 0.0;
  if (nr == 1) return;
  const int m = nr - 1;
  double D[DIM + 1][4], G[DIM + 1][DIM + 2];
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < DIM; ++k) D[i][k] = P[R[i + 1]][k] - p0[k];
  double scale = 0.0;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int k = 0; k < DIM; ++k) s += D[i][k] * D[j][k];
      G[i][j] = 2.0 * s;
    }
    double s = 0.0;
    for (int k = 0; k < DIM; ++k) s += D[i][k] * D[i][k];
    G[i][m] = s;
    scale = fmax(scale, G[i][i]);
  }
  int piv_col[DIM + 1];
  bool used[DIM + 1];
  for (int i = 0; i < m; ++i) used[i] = false;
  int rank = 0;
  for (int col = 0; col < m; ++col) {  // elimination by rows, pivot = largest remaining entry in the column
    int best = -1;
    double bv = 1e-14 * scale;
    for (int i = 0; i < m; ++i)
      if (!used[i] && fabs(G[i][col]) > bv) bv = fabs(G[i][col]), best = i;
    piv_col[col] = best;
    if (best < 0) continue;
    used[best] = true;
    ++rank;
    for (int i = 0; i < m; ++i) {
      if (i == best) continue;
      const double f = G[i][col] / G[best][col];
      for (int j = col; j <= m; ++j) G[i][j] -= f * G[best][j];
    }
  }
  for (int col = 0; col < m; ++col) {
    const int i = piv_col[col];
    const double lam = i >= 0 ? G[i][m] / G[i][col] : 0.0;
    for (int k = 0; k < DIM; ++k) c[k] += lam * D[col][k];
  }
  for (int i = 0; i < nr; ++i) r = fmax(r, sqrt(dist2<DIM>(P[R[i]], c)));
}

__device__ __forceinline__ bool inside_ball(double d2, double r) {
  return r >= 0.0 && sqrt(d2) <= r * (1.0 + 1e-12) + 1e-15;
}

// Welzl's recursion, the exact ball of P[0..k_end) with the support R[0..nr) on its boundary,
// run as a loop over an explicit stack of (k_end, k) frames (the support grows by one point per
// level, so at most d + 2 frames): a point outside the current ball joins the support and opens a
// frame over the points before it; a finished frame removes its point again and its caller goes
// on with the ball the frame left.  No recursion, so the thread's stack is known at compile time.
// Returns false if it took more than kWelzlSteps loop steps (the ball is then unfinished).
constexpr int kWelzlSteps = 1 << 22;

template <int DIM>
__device__ __forceinline__ bool welzl(const double (*P)[4], int k_end, int* R, int nr, double* c, double& r) {
  int fk_end[DIM + 2], fk[DIM + 2];
  int depth = 0;
  fk_end[0] = k_end, fk[0] = 0;
  circumball<DIM>(P, R, nr, c, r);
  if (nr == DIM + 1) return true;
  for (int step = 0; depth >= 0; ++step) {
    if (step == kWelzlSteps) return false;
    if (fk[depth] >= fk_end[depth]) {  // frame done: back to the caller, which moves past its point
      --depth;
      if (depth >= 0) --nr, ++fk[depth];
      continue;
    }
    const int k = fk[depth];
    if (inside_ball(dist2<DIM>(P[k], c), r)) {
      ++fk[depth];
      continue;
    }
    R[nr++] = k;
    circumball<DIM>(P, R, nr, c, r);
    if (nr == DIM + 1) {  // a full support: the callee has no points to scan
      --nr, ++fk[depth];
      continue;
    }
    ++depth;
    fk_end[depth] = k, fk[depth] = 0;
  }
  return true;
}

template <typename T, int DIM>
__device__ __forceinline__ void load_point(const T* x, long i, const double* ref, double* p) {
  if (DIM == 3) {
    p[0] = x[3 * i], p[1] = x[3 * i + 1], p[2] = x[3 * i + 2];
  } else {
    const double q0 = x[4 * i], q1 = x[4 * i + 1], q2 = x[4 * i + 2], q3 = x[4 * i + 3];
    const double s = q0 * ref[0] + q1 * ref[1] + q2 * ref[2] + q3 * ref[3] < 0.0 ? -1.0 : 1.0;
    p[0] = s * q0, p[1] = s * q1, p[2] = s * q2, p[3] = s * q3;
  }
}

template <typename T, int DIM>
__global__ void exact_init_kernel(const T* x, const double* ref_in, ExactState* st) {
  double ref[4] = {1.0, 0.0, 0.0, 0.0};
  if (DIM == 4) {
    if (ref_in) {
      for (int k = 0; k < 4; ++k) ref[k] = ref_in[k];
    } else {
      for (int k = 0; k < 4; ++k) ref[k] = x[k];
    }
  }
  for (int k = 0; k < 4; ++k) st->ref[k] = ref[k];
  double p[4] = {0.0, 0.0, 0.0, 0.0};
  load_point<T, DIM>(x, 0, ref, p);
  for (int k = 0; k < 4; ++k) st->pts[0][k] = p[k], st->c[k] = p[k];
  st->r = 0.0;
  st->n = 1;
  st->done = 0;
  st->overflow = 0;
  st->far_d2 = 0.0;
}

// One pass: the farthest sample from the current centre, per block (ties to the lower index).
template <typename T, int DIM>
__global__ void __launch_bounds__(kExactThreads)
    exact_far_kernel(const T* __restrict__ x, long n, const ExactState* st, double* blk_d2, long* blk_idx) {
  if (st->done) return;
  __shared__ double s_c[4], s_ref[4];
  __shared__ double w_d2[kExactThreads / 32];
  __shared__ long w_idx[kExactThreads / 32];
  if (threadIdx.x < 4) s_c[threadIdx.x] = st->c[threadIdx.x], s_ref[threadIdx.x] = st->ref[threadIdx.x];
  __syncthreads();
  double best = -1.0;
  long bi = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double p[4];
    load_point<T, DIM>(x, i, s_ref, p);
    const double d2 = dist2<DIM>(p, s_c);
    if (d2 > best) best = d2, bi = i;
  }
  for (int o = 16; o; o >>= 1) {
    const double od = __shfl_xor_sync(kFullMask, best, o);
    const long oi = __shfl_xor_sync(kFullMask, bi, o);
    if (od > best || (od == best && oi < bi)) best = od, bi = oi;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) w_d2[warp] = best, w_idx[warp] = bi;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (w_d2[w] > best || (w_d2[w] == best && w_idx[w] < bi)) best = w_d2[w], bi = w_idx[w];
    blk_d2[blockIdx.x] = best;
    blk_idx[blockIdx.x] = bi;
  }
}

// The farthest sample of the pass joins the candidates if it lies outside their ball; then the
// exact ball of the candidates (one thread).
template <typename T, int DIM>
__global__ void exact_update_kernel(const T* x, int nblk, const double* blk_d2, const long* blk_idx,
                                    ExactState* st) {
  if (st->done) return;
  double best = -1.0;
  long bi = 0;
  for (int b = 0; b < nblk; ++b)
    if (blk_d2[b] > best || (blk_d2[b] == best && blk_idx[b] < bi)) best = blk_d2[b], bi = blk_idx[b];
  st->far_d2 = best;
  if (inside_ball(best, st->r)) {
    st->done = 1;
    return;
  }
  if (st->n == kExactCap) {
    st->overflow = 1;
    st->done = 1;
    return;
  }
  double p[4] = {0.0, 0.0, 0.0, 0.0};
  load_point<T, DIM>(x, bi, st->ref, p);
  const int n = st->n;
  for (int k = 0; k < 4; ++k) st->pts[n][k] = p[k];
  st->n = n + 1;
  // the new point lies outside the ball of the others, so it is on the boundary of the ball of all
  // (Welzl's lemma): the recursion starts with it in the support
  int R[DIM + 1];
  R[0] = n;
  double c[DIM], r;
  if (!welzl<DIM>(st->pts, n, R, 1, c, r)) {
    st->overflow = 1;
    st->done = 1;
  }
  for (int k = 0; k < DIM; ++k) st->c[k] = c[k];
  st->r = r;
}

// Result: translation centre and radius (the largest distance of the last pass); rotation centre
// projected to the unit sphere (w >= 0) and the largest geodesic distance from it, found as the
// sample of largest 1 - (C . q)^2 = sin^2(theta / 2), its angle from 2 atan2(|vec(C* q)|, |C . q|).
template <typename T>
__global__ void __launch_bounds__(kExactThreads)
    exact_rot_radius_kernel(const T* __restrict__ x, long n, const ExactState* st, double* blk_d2, long* blk_idx) {
  __shared__ double s_C[4];
  __shared__ double w_d2[kExactThreads / 32];
  __shared__ long w_idx[kExactThreads / 32];
  if (threadIdx.x == 0) {
    double nn = 0.0;
    for (int k = 0; k < 4; ++k) nn += st->c[k] * st->c[k];
    const double s = (st->c[0] < 0.0 ? -1.0 : 1.0) / sqrt(nn);
    for (int k = 0; k < 4; ++k) s_C[k] = s * st->c[k];
  }
  __syncthreads();
  double best = -1.0;
  long bi = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double d = s_C[0] * (double)x[4 * i] + s_C[1] * (double)x[4 * i + 1] + s_C[2] * (double)x[4 * i + 2] +
                     s_C[3] * (double)x[4 * i + 3];
    const double key = 1.0 - d * d;
    if (key > best) best = key, bi = i;
  }
  for (int o = 16; o; o >>= 1) {
    const double od = __shfl_xor_sync(kFullMask, best, o);
    const long oi = __shfl_xor_sync(kFullMask, bi, o);
    if (od > best || (od == best && oi < bi)) best = od, bi = oi;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) w_d2[warp] = best, w_idx[warp] = bi;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (w_d2[w] > best || (w_d2[w] == best && w_idx[w] < bi)) best = w_d2[w], bi = w_idx[w];
    blk_d2[blockIdx.x] = best;
    blk_idx[blockIdx.x] = bi;
  }
}

template <typename T>
__global__ void exact_result_kernel(const T* q, int nblk_r, const double* blk_r, const long* idx_r,
                                    const ExactState* st_r, const ExactState* st_t, int has_r, int has_t,
                                    double* result, int* status) {
  if (has_r) {
    double best = -1.0;
    long bi = 0;
    for (int b = 0; b < nblk_r; ++b)
      if (blk_r[b] > best || (blk_r[b] == best && idx_r[b] < bi)) best = blk_r[b], bi = idx_r[b];
    double nn = 0.0;
    for (int k = 0; k < 4; ++k) nn += st_r->c[k] * st_r->c[k];
    const double s = (st_r->c[0] < 0.0 ? -1.0 : 1.0) / sqrt(nn);
    double C[4];
    for (int k = 0; k < 4; ++k) C[k] = s * st_r->c[k], result[k] = C[k];
    const Q4<double> c{C[0], -C[1], -C[2], -C[3]};
    const Q4<double> qq{(double)q[4 * bi], (double)q[4 * bi + 1], (double)q[4 * bi + 2], (double)q[4 * bi + 3]};
    const Q4<double> e = qmul(c, qq);
    result[7] = 2.0 * atan2(sqrt(e.x * e.x + e.y * e.y + e.z * e.z), fabs(e.w));
    if (st_r->overflow) atomicOr(status, kDevErrNumeric);
  }
  if (has_t) {
    for (int k = 0; k < 3; ++k) result[4 + k] = st_t->c[k];
    result[8] = sqrt(st_t->far_d2);
    if (st_t->overflow) atomicOr(status, kDevErrNumeric);
  }
  if (!has_r) result[0] = result[1] = result[2] = result[3] = result[7] = 0.0;
  if (!has_t) result[4] = result[5] = result[6] = result[8] = 0.0;
}

size_t exact_scratch_bytes(int sm_count) {
  const int nblk = 4 * sm_count;
  return 2 * ((sizeof(ExactState) + 255) / 256 * 256) + 2 * (size_t)nblk * (sizeof(double) + sizeof(long)) + 512;
}

template <typename T>
static cudaError_t run_exact_t(purse_t h, const T* q, long n_rot, const T* t, long n_tr, const double* d_ref,
                               double* d_result, void* scratch, cudaStream_t st) {
  const int nblk = 4 * h->sm_count;
  char* base = reinterpret_cast<char*>(scratch);
  const size_t sst = (sizeof(ExactState) + 255) / 256 * 256;
  ExactState* st_r = reinterpret_cast<ExactState*>(base);
  ExactState* st_t = reinterpret_cast<ExactState*>(base + sst);
  double* blk_d2 = reinterpret_cast<double*>(base + 2 * sst);
  long* blk_idx = reinterpret_cast<long*>(blk_d2 + nblk);
  double* blk_d2b = reinterpret_cast<double*>(blk_idx + nblk);
  long* blk_idxb = reinterpret_cast<long*>(blk_d2b + nblk);
  const bool hr = n_rot > 0, ht = n_tr > 0;
  auto grid = [&](long n) { return (int)std::min<long>(nblk, (n + kExactThreads - 1) / kExactThreads); };
  if (hr) exact_init_kernel<T, 4><<<1, 1, 0, st>>>(q, d_ref, st_r);
  if (ht) exact_init_kernel<T, 3><<<1, 1, 0, st>>>(t, nullptr, st_t);
  int done[2] = {hr ? 0 : 1, ht ? 0 : 1};
  cudaError_t e = cudaGetLastError();
  // rounds of eight passes, then the host reads the two done flags
  for (int round = 0; round < kExactCap / 8 + 1 && e == cudaSuccess && !(done[0] && done[1]); ++round) {
    for (int k = 0; k < 8; ++k) {
      if (hr && !done[0]) {
        exact_far_kernel<T, 4><<<grid(n_rot), kExactThreads, 0, st>>>(q, n_rot, st_r, blk_d2, blk_idx);
        exact_update_kernel<T, 4><<<1, 1, 0, st>>>(q, grid(n_rot), blk_d2, blk_idx, st_r);
      }
      if (ht && !done[1]) {
        exact_far_kernel<T, 3><<<grid(n_tr), kExactThreads, 0, st>>>(t, n_tr, st_t, blk_d2b, blk_idxb);
        exact_update_kernel<T, 3><<<1, 1, 0, st>>>(t, grid(n_tr), blk_d2b, blk_idxb, st_t);
      }
    }
    e = cudaGetLastError();
    int hd[2] = {1, 1};
    if (e == cudaSuccess && hr) e = cudaMemcpyAsync(&hd[0], &st_r->done, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ht) e = cudaMemcpyAsync(&hd[1], &st_t->done, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (hr) done[0] = hd[0];
    if (ht) done[1] = hd[1];
  }
  if (e != cudaSuccess) return e;
  if (hr) exact_rot_radius_kernel<T><<<grid(n_rot), kExactThreads, 0, st>>>(q, n_rot, st_r, blk_d2, blk_idx);
  exact_result_kernel<T><<<1, 1, 0, st>>>(q, grid(n_rot), blk_d2, blk_idx, st_r, st_t, hr, ht, d_result,
                                         h->d_status);
  return cudaGetLastError();
}

cudaError_t launch_megb_exact(purse_t h, int precision, const void* d_q, long n_rot, const void* d_t, long n_tr,
                              const double* d_ref, double* d_result, void* scratch, cudaStream_t st) {
  if (precision == 0)
    return run_exact_t<float>(h, (const float*)d_q, n_rot, (const float*)d_t, n_tr, d_ref, d_result, scratch, st);
  return run_exact_t<double>(h, (const double*)d_q, n_rot, (const double*)d_t, n_tr, d_ref, d_result, scratch, st);
}

}  // namespace purse
