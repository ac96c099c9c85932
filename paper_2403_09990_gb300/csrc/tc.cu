// dist(R, t, dS) of eq. 11 for materialised FP32 poses, with the pose transform as a dense
// contraction on the fifth-generation tensor cores (tcgen05, kind::tf32).
//
// A pose is the row p = (R_00 .. R_22, t_0, t_1, t_2, 1, 0, 0, 0) (K = 16).  Every
// constraint i contributes three columns of B (16 x 3 n) such that (p B) holds, for
//   3D-3D (eq. 3): the residual R a_i + t - b_i;
//   2D-3D (eq. 2): e_x = P_x - u_i P_z, e_y = P_y - v_i P_z and P_z of P = K (R Z_i + t)
//                  (the division-free residual; the margin divides once by P_z).
// The epilogue turns each triple into the margin r_i - |g_i| and keeps the minimum.
//
// Precision: a TF32 operand keeps 11 significant bits.  mode 1 splits both operands,
// x = hi + lo with hi = rna_tf32(x) and lo = rna_tf32(x - hi), and accumulates
// hi.hi + hi.lo + lo.hi in FP32 (about 2^-21 relative per product, near FP32); mode 2 takes
// one TF32 pass (2^-11).  B is split from the FP64 constraint table.
//
// Mapping: one CTA of 128 threads per tile of 128 poses (persistent over tiles), M = 128
// rows in TMEM lanes, constraints in rounds of up to 32 (N <= 96 columns per MMA, 128 TMEM
// columns at most, so four CTAs fit an SM).  The raw 6 KB pose tiles stream through a ring of
// four shared-memory stages filled by 1-D bulk copies (cp.async.bulk, one mbarrier per
// stage); the threads split a landed tile into A (hi, lo).  Shared memory holds A and B in
// the K-major no-swizzle canonical layout: core matrices of 8 rows x 16 bytes, the four core
// matrices of a row group along K contiguous (LBO = 128 B), row groups 512 B apart (SBO).
// One thread issues the MMAs and commits them to an mbarrier; all four warps read their 32
// TMEM lanes back with tcgen05.ld.
#include <algorithm>
#include <cfloat>

#include "dev.cuh"
#include "internal.h"

namespace purse {

constexpr int kTcThreads = 128;
constexpr int kTcRoundMax = 32;          // constraints per MMA round (N = 96, 128 TMEM columns)
constexpr int kTcStages = 4;             // raw pose tiles in flight per CTA
constexpr uint32_t kTcTileBytes = 8192;  // 128 rows x 16 fp32
constexpr uint32_t kTcRawBytes = 6144;   // 128 poses x 48 B

__device__ __forceinline__ float rna_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row, k) in a K-major no-swizzle tile with K = 16 (fp32).
__device__ __forceinline__ uint32_t kmaj_off(int row, int k) {
  return (uint32_t)((row >> 3) * 512 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(512u >> 4) << 32) |
         (1ull << 46);
}

// kind::tf32, D = F32, A = B = TF32, both K-major, M = 128.
__device__ __forceinline__ uint32_t idesc_tf32(int n_cols) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n_cols >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Coefficient of pose entry k in output column comp of constraint i (FP64 table rows (a or Z, r),
// (b or (u, v, 0), r^2)).
__device__ double tc_coef(int kind, const double* tab, int n, double fx, double fy, double cx, double cy, int i,
                          int comp, int k) {
  const double* a = tab + 4 * i;
  const double* o = tab + 4 * (n + i);
  if (kind == 0) {  // e_c = sum_j R_cj a_j + t_c - b_c
    if (k >= 3 * comp && k < 3 * comp + 3) return a[k - 3 * comp];
    if (k == 9 + comp) return 1.0;
    if (k == 12) return -o[comp];
    return 0.0;
  }
  // X = R Z + t; e_x = fx X_x + (cx - u) X_z, e_y = fy X_y + (cy - v) X_z, P_z = X_z
  const double s0 = comp == 0 ? fx : 0.0;                                  // weight of X_x
  const double s1 = comp == 1 ? fy : 0.0;                                  // weight of X_y
  const double s2 = comp == 0 ? cx - o[0] : comp == 1 ? cy - o[1] : 1.0;  // weight of X_z
  if (k < 3) return s0 * a[k];
  if (k < 6) return s1 * a[k - 3];
  if (k < 9) return s2 * a[k - 6];
  if (k == 9) return s0;
  if (k == 10) return s1;
  if (k == 11) return s2;
  return 0.0;
}

template <int KIND, int PASSES>
__global__ void __launch_bounds__(kTcThreads, 4)
    tc_dist_kernel(const double* __restrict__ tab, const float* __restrict__ tab32, int n, double fx, double fy,
                   double cx, double cy, const float* __restrict__ poses, long n_poses, float* __restrict__ dist,
                   uint32_t tmem_cols, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // layout: [raw pose tiles, kTcStages x 6 KB][A_hi 8 KB][A_lo 8 KB][B_hi 64 B per column][B_lo][radii]
  //         [mbarriers: MMA completion, one per raw stage][TMEM address]
  const int n_pad = (n + 15) & ~15;
  const int cols = 3 * n_pad;
  unsigned char* raw = smem;
  unsigned char* a_hi = smem + kTcStages * kTcRawBytes;
  unsigned char* a_lo = a_hi + kTcTileBytes;
  unsigned char* b_hi = a_lo + kTcTileBytes;
  unsigned char* b_lo = b_hi + 64 * (size_t)cols;
  float* r_s = reinterpret_cast<float*>(b_lo + 64 * (size_t)cols);
  uint64_t* bar = reinterpret_cast<uint64_t*>(r_s + n_pad);
  uint64_t* full = bar + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(full + kTcStages);
  const int tid = threadIdx.x, warp = tid >> 5;

  // ---- operands that stay: B (hi, lo), radii, the constant column k = 12..15 of A
  for (int e = tid; e < cols * 16; e += kTcThreads) {
    const int c = e >> 4, k = e & 15;
    const int i = c / 3, comp = c - 3 * i;
    const double v = i < n ? tc_coef(KIND, tab, n, fx, fy, cx, cy, i, comp, k) : 0.0;
    const float hi = rna_tf32((float)v);
    const float lo = rna_tf32((float)(v - (double)hi));
    *reinterpret_cast<float*>(b_hi + kmaj_off(c, k)) = hi;
    *reinterpret_cast<float*>(b_lo + kmaj_off(c, k)) = lo;
  }
  for (int i = tid; i < n_pad; i += kTcThreads) r_s[i] = i < n ? tab32[4 * i + 3] : 0.f;
  {
    const int row = tid;  // k = 12..15: (1, 0, 0, 0) in hi, zeros in lo
    *reinterpret_cast<float4*>(a_hi + kmaj_off(row, 12)) = make_float4(1.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4*>(a_lo + kmaj_off(row, 12)) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    for (int s = 0; s < kTcStages; ++s) mbar_init(full + s, 1);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t a_hi_s = smem_addr(a_hi), a_lo_s = smem_addr(a_lo);
  const uint32_t b_hi_s = smem_addr(b_hi), b_lo_s = smem_addr(b_lo);
  uint32_t phase = 0;
  bool failed = false;

  // ---- raw pose tiles: tile k of this CTA (global tile blockIdx.x + k gridDim.x, 48 B per pose,
  //      one 1-D bulk copy) lands in stage k mod kTcStages; thread 0 keeps kTcStages tiles in flight
  const long n_tiles = (n_poses + 127) / 128;
  long issued = 0;  // thread 0: bulk copies issued so far
  auto issue = [&](long k) {
    const long tile = blockIdx.x + k * (long)gridDim.x;
    if (tile >= n_tiles) return;
    const int s = (int)(k % kTcStages);
    const long rows = n_poses - tile * 128 < 128 ? n_poses - tile * 128 : 128;
    const uint32_t bytes = (uint32_t)(rows * 48);
    mbar_arrive_expect_tx(full + s, bytes);
    bulk_copy_g2s(raw + (size_t)s * kTcRawBytes, poses + 12 * (tile * 128), bytes, full + s);
    issued = k + 1;
  };
  if (tid == 0)
    for (int k = 0; k < kTcStages; ++k) issue(k);
  long k = 0;
  for (;; ++k) {
    const long tile = blockIdx.x + k * (long)gridDim.x;
    if (tile >= n_tiles) break;
    const int st = (int)(k % kTcStages);
    const bool okf = mbar_wait_bounded(full + st, (uint32_t)((k / kTcStages) & 1), 1 << 24);
    if (__syncthreads_or(!okf)) {
      failed = true;
      break;
    }
    const long row0 = tile * 128;
    const long avail4 = (n_poses - row0) * 3;
    const float4* src = reinterpret_cast<const float4*>(raw + (size_t)st * kTcRawBytes);
    // ---- A split into hi and lo (K-major core matrices)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int q = tid + kTcThreads * j;
      const int row = q / 3, kb = q - 3 * row;
      const float4 x = q < avail4 ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 h = make_float4(rna_tf32(x.x), rna_tf32(x.y), rna_tf32(x.z), rna_tf32(x.w));
      *reinterpret_cast<float4*>(a_hi + kmaj_off(row, 4 * kb)) = h;
      if (PASSES == 3)
        *reinterpret_cast<float4*>(a_lo + kmaj_off(row, 4 * kb)) =
            make_float4(rna_tf32(x.x - h.x), rna_tf32(x.y - h.y), rna_tf32(x.z - h.z), rna_tf32(x.w - h.w));
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) issue(k + kTcStages);  // every thread has read stage st: refill it
    float best = INFINITY;
    for (int c0 = 0; c0 < n_pad && !failed; c0 += kTcRoundMax) {
      const int nr = min(kTcRoundMax, n_pad - c0);  // constraints of this round (a multiple of 16)
      const int ncol = 3 * nr;
      if (tid == 0) {
        tc_fence_after();
        const uint32_t idesc = idesc_tf32(ncol);
        const uint32_t boff = (uint32_t)(3 * c0 / 8) * 512u;  // first column of the round
#pragma unroll
        for (int s = 0; s < 2; ++s) {  // K = 16 in two steps of 8
          const uint32_t ko = 256u * s;
          tc_mma(tmem, smem_desc(a_hi_s + ko), smem_desc(b_hi_s + boff + ko), idesc, s > 0);
          if (PASSES == 3) {
            tc_mma(tmem, smem_desc(a_hi_s + ko), smem_desc(b_lo_s + boff + ko), idesc, 1);
            tc_mma(tmem, smem_desc(a_lo_s + ko), smem_desc(b_hi_s + boff + ko), idesc, 1);
          }
        }
        tc_commit(bar);
      }
      const bool ok = mbar_wait_bounded(bar, phase, 1 << 24);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc_fence_after();
      const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
      for (int g = 0; g < nr; g += 16) {
        float v0[16], v1[16], v2[16];
        const uint32_t col = (uint32_t)(3 * g);
        tc_ld16(lane_base + col, v0);
        tc_ld16(lane_base + col + 16, v1);
        tc_ld16(lane_base + col + 32, v2);
        tc_wait_ld();
        float v[48];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = v0[u], v[16 + u] = v1[u], v[32 + u] = v2[u];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int i = c0 + g + u;
          if (i < n) {
            const float x = v[3 * u], y = v[3 * u + 1], z = v[3 * u + 2];
            // margin r - |e| (2D-3D: r - |e| / P_z) without a division: |e| = s2 rsqrt(s2 (P_z^2))
            float m;
            if (KIND == 0) {
              const float s2 = fmaf(z, z, fmaf(y, y, x * x));
              m = fmaf(-s2, rsqrtf(s2 + 1e-30f), r_s[i]);
            } else {
              const float s2 = fmaf(y, y, x * x);
              m = z > 0.f ? fmaf(-s2, rsqrtf(fmaf(s2, z * z, 1e-30f)), r_s[i]) : -INFINITY;
            }
            best = fminf(best, m);
          }
        }
      }
      tc_fence_before();
      __syncthreads();  // every warp has read TMEM before the next round overwrites it
    }
    if (failed) break;
    const long row = row0 + tid;
    if (row < n_poses) dist[row] = best;
  }
  if (failed) {
    if (tid == 0) {
      atomicOr(status, kDevErrTimeout);
      // the bulk copies still in flight land before the shared memory is released (bounded)
      for (long kk = k; kk < issued; ++kk)
        mbar_wait_bounded(full + (int)(kk % kTcStages), (uint32_t)((kk / kTcStages) & 1), 1 << 24);
    }
    // and the MMAs still in flight finish before the accumulator is released (bounded)
    mbar_wait_bounded(bar, phase ^ 1u, 1 << 24);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

size_t tc_dist_smem(int n) {
  const int n_pad = (n + 15) & ~15;
  return kTcStages * kTcRawBytes + 2 * kTcTileBytes + 2 * 64 * (size_t)(3 * n_pad) + 4 * (size_t)n_pad +
         8 * (1 + kTcStages) + 16;
}

cudaError_t launch_tc_dist(purse_t h, int passes, const float* d_poses, long n_poses, float* d_dist, cudaStream_t st) {
  if (n_poses == 0) return cudaSuccess;
  const int n = h->n, n_pad = (n + 15) & ~15;
  const int round_cols = 3 * (n_pad < kTcRoundMax ? n_pad : kTcRoundMax);
  uint32_t tcols = 32;
  while (tcols < (uint32_t)round_cols) tcols <<= 1;
  const size_t smem = tc_dist_smem(n);
  void (*kern)(const double*, const float*, int, double, double, double, double, const float*, long, float*,
               uint32_t, int*);
  if (h->kind == 0)
    kern = passes == 3 ? tc_dist_kernel<0, 3> : tc_dist_kernel<0, 1>;
  else
    kern = passes == 3 ? tc_dist_kernel<1, 3> : tc_dist_kernel<1, 1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // several CTAs per SM: the whole configurable shared memory for this kernel
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  // resident CTAs per SM from the register file, the shared memory and the accumulator columns (every
  // resident CTA holds its own, at most 512 per SM)
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  int dev = 0, smem_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e != cudaSuccess) return e;
  const int regs = (fa.numRegs + 7) & ~7;
  int per_sm = 65536 / (regs * kTcThreads);
  per_sm = std::min(per_sm, smem_sm / (int)(smem + 1024));
  per_sm = std::min(per_sm, 2048 / kTcThreads);
  per_sm = std::min(per_sm, (int)(512u / tcols));
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  per_sm = std::max(1, std::min(per_sm, tuned_config(kTuneDist, h->kind, n, n_poses, passes, per_sm)));
  const long tiles = (n_poses + 127) / 128;
  const long cap = (long)per_sm * h->sm_count;
  const int grid = (int)(tiles < cap ? tiles : cap);
  kern<<<grid, kTcThreads, smem, st>>>(h->tables.f64, h->tables.f32, n, h->K.fx, h->K.fy, h->K.cx, h->K.cy, d_poses,
                                       n_poses, d_dist, tcols, h->d_status);
  return cudaGetLastError();
}

}  // namespace purse
