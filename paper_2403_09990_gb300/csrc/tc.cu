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
// Mapping: persistent CTAs of nine warps (two per SM) over tiles of 128 poses, M = 128 rows in
// TMEM lanes, constraints in rounds of 16 (N = 48 columns per MMA).  Split warps load their pose
// rows with 16-byte global loads and write A (hi, lo) into a ring of shared-memory slots; one thread
// issues the MMAs into a ring of TMEM accumulators; epilogue warps read them back with tcgen05.ld.
// The stages hand over through mbarriers (see tc_dist_kernel).  Shared memory holds A and B in the
// K-major no-swizzle canonical layout: core matrices of 8 rows x 16 bytes, the four core matrices of
// a row group along K contiguous (LBO = 128 B), row groups 512 B apart (SBO).
#include <algorithm>
#include <cfloat>

#include "dev.cuh"
#include "internal.h"

namespace purse {

constexpr uint32_t kTcTileBytes = 8192;  // 128 rows x 16 fp32

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

// Byte size of one A slot: hi (and lo for the split passes).
template <int PASSES>
__host__ __device__ constexpr uint32_t tc_abuf() {
  return PASSES == 3 ? 2 * kTcTileBytes : kTcTileBytes;
}

constexpr int kTcThreads = 288;                // 9 warps
constexpr int kTcA = 3, kTcAcc = 4;            // A slots, TMEM accumulators of 64 columns
constexpr int kTcPrefetch = 4;                 // pose tiles in flight per split thread
constexpr uint32_t kTcCols = 64 * kTcAcc;

// Wait for the phase of the given parity with the thread suspended in between (try_wait with a suspend
// time hint: the thread resumes when the phase completes, or after the hint), so that waiting warps take
// no issue slots from the working ones.  Bounded: gives up after about 2^31 SM cycles (about a second)
// or once another role has raised the failure flag.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* fail) {
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try_wait_hint(bar, parity)) return true;
    if (*fail || clock64() - t0 > (1ll << 31)) return false;
    __nanosleep(32);  // the suspending try_wait alone still left the waiting warps busy on the issue slots
  }
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Each CTA is persistent over tiles of 128 poses (tile k of the CTA is
// global tile blockIdx.x + k gridDim.x) and runs each stage on its own warps, linked by mbarrier rings
// (no CTA-wide barrier in the loop):
//   warps 0-3  load the poses of tile k with 16-byte global loads (one pose row of 48 B per thread,
//              kTcPrefetch tiles in flight in registers), split them into A (hi, lo) in a ring of
//              kTcA slots of shared memory and signal the slot;
//   warp 4     (one thread) issues the MMAs of each unit (tile, round of 16 constraints, N = 48) into a
//              ring of kTcAcc accumulators of 64 TMEM columns, committing to the accumulator's barrier
//              and, after a tile's last round, to its A slot's;
//   warps 5-8  read an accumulator back (warp w reads TMEM lanes 32 (w mod 4) ..), release it and turn
//              it into margins, one pose row per thread.
// Padded constraints (i >= n) get radius +inf and, 2D-3D, P_z = 1, so they never lower the minimum; the
// margins use FP32 expressions two constraints per paired instruction.  Every wait is bounded; a role
// that gives up raises a shared flag that ends the others' loops, and the MMAs in flight finish before
// TMEM is released.
template <int KIND, int PASSES>
__global__ void __launch_bounds__(kTcThreads)
    tc_dist_kernel(const double* __restrict__ tab, const float* __restrict__ tab32, int n, double fx, double fy,
                   double cx, double cy, const float* __restrict__ poses, long n_poses, float* __restrict__ dist,
                   int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // layout: [A slots, kTcA x (hi, lo)][B_hi 64 B per column][B_lo][radii]
  //         [barriers: A full, A empty, acc full, acc empty, MMA done][TMEM address][flag]
  constexpr uint32_t abuf = tc_abuf<PASSES>();
  const int n_pad = (n + 15) & ~15;
  const int cols = 3 * n_pad, R = n_pad / 16;
  unsigned char* a0 = smem;
  unsigned char* b_hi = a0 + kTcA * abuf;
  unsigned char* b_lo = b_hi + 64 * (size_t)cols;
  float* r_s = reinterpret_cast<float*>(b_lo + 64 * (size_t)cols);
  uint64_t* a_full = reinterpret_cast<uint64_t*>(r_s + n_pad);
  uint64_t* a_empty = a_full + kTcA;
  uint64_t* t_full = a_empty + kTcA;
  uint64_t* t_empty = t_full + kTcAcc;
  uint64_t* mma_done = t_empty + kTcAcc;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* fail = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- operands that stay: B (hi, lo), radii, the constant columns k = 12..15 of every A slot
  for (int e = tid; e < cols * 16; e += kTcThreads) {
    const int c = e >> 4, k = e & 15;
    const int i = c / 3, comp = c - 3 * i;
    const double v = i < n ? tc_coef(KIND, tab, n, fx, fy, cx, cy, i, comp, k)
                           : (KIND == 1 && comp == 2 && k == 12 ? 1.0 : 0.0);
    const float hi = rna_tf32((float)v);
    const float lo = rna_tf32((float)(v - (double)hi));
    *reinterpret_cast<float*>(b_hi + kmaj_off(c, k)) = hi;
    *reinterpret_cast<float*>(b_lo + kmaj_off(c, k)) = lo;
  }
  for (int i = tid; i < n_pad; i += kTcThreads) r_s[i] = i < n ? tab32[4 * i + 3] : INFINITY;
  for (int e = tid; e < kTcA * 128; e += kTcThreads) {
    unsigned char* ah = a0 + (e >> 7) * abuf;
    *reinterpret_cast<float4*>(ah + kmaj_off(e & 127, 12)) = make_float4(1.f, 0.f, 0.f, 0.f);
    if (PASSES == 3)
      *reinterpret_cast<float4*>(ah + kTcTileBytes + kmaj_off(e & 127, 12)) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (tid == 0) {
    for (int s = 0; s < kTcA; ++s) mbar_init(a_full + s, 4), mbar_init(a_empty + s, 1);
    for (int s = 0; s < kTcAcc; ++s) mbar_init(t_full + s, 1), mbar_init(t_empty + s, 4);
    mbar_init(mma_done, 1);
    *fail = 0;
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();  // B and the constant columns of A, written by the generic proxy, are read by the MMAs
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // tiles of this CTA (32-bit per-CTA counters: a launch takes fewer than 2^31 tiles)
  const int n_tiles = (int)((n_poses + 127) / 128);
  const int T = n_tiles > (int)blockIdx.x ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const long step = (long)gridDim.x * 128;

  if (warp < 4) {
    // ---- split warps: pose row tid of every tile
    long row = (long)blockIdx.x * 128 + tid;
    float4 x[kTcPrefetch][3];
    auto load = [&](float4 (&d)[3], long r) {
      const float4* src = reinterpret_cast<const float4*>(poses) + 3 * r;
#pragma unroll
      for (int kb = 0; kb < 3; ++kb) d[kb] = r < n_poses ? __ldg(src + kb) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
#pragma unroll
    for (int j = 0; j < kTcPrefetch; ++j) load(x[j], row + j * step);
    int as = 0;
    uint32_t aph = 0;
    for (int k0 = 0; k0 < T && !*fail; k0 += kTcPrefetch) {
#pragma unroll
      for (int j = 0; j < kTcPrefetch; ++j) {
        const int k = k0 + j;
        if (k >= T) break;
        if (k >= kTcA && !tc_wait(a_empty + as, aph ^ 1u, fail)) {
          *fail = 1;
          break;
        }
        unsigned char* ah = a0 + (size_t)as * abuf;
#pragma unroll
        for (int kb = 0; kb < 3; ++kb) {
          const float4 v = x[j][kb];
          const float4 h = make_float4(rna_tf32(v.x), rna_tf32(v.y), rna_tf32(v.z), rna_tf32(v.w));
          *reinterpret_cast<float4*>(ah + kmaj_off(tid, 4 * kb)) = h;
          if (PASSES == 3)
            *reinterpret_cast<float4*>(ah + kTcTileBytes + kmaj_off(tid, 4 * kb)) =
                make_float4(rna_tf32(v.x - h.x), rna_tf32(v.y - h.y), rna_tf32(v.z - h.z), rna_tf32(v.w - h.w));
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(a_full + as);
        if (++as == kTcA) as = 0, aph ^= 1u;
        load(x[j], row + (long)(k + kTcPrefetch) * step);  // the tile kTcPrefetch ahead into the freed registers
      }
    }
  } else if (warp == 4) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t a0_s = smem_addr(a0), b_hi_s = smem_addr(b_hi), b_lo_s = smem_addr(b_lo);
      const uint32_t idesc = idesc_tf32(48);
      int as = 0, ts = 0, u = 0;
      uint32_t aph = 0, tph = 0;
      for (int k = 0; k < T && !*fail; ++k) {
        if (!tc_wait(a_full + as, aph, fail)) {
          *fail = 1;
          break;
        }
        const uint32_t ah = a0_s + (uint32_t)as * abuf, al = ah + kTcTileBytes;
        for (int r = 0; r < R; ++r, ++u) {
          if (u >= kTcAcc && !tc_wait(t_empty + ts, tph ^ 1u, fail)) {
            *fail = 1;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + 64u * (uint32_t)ts;
          const uint32_t boff = (uint32_t)(6 * r) * 512u;  // columns 48 r .. 48 r + 47
#pragma unroll
          for (int s = 0; s < 2; ++s) {  // K = 16 in two steps of 8
            const uint32_t ko = 256u * s;
            tc_mma(d, smem_desc(ah + ko), smem_desc(b_hi_s + boff + ko), idesc, s > 0);
            if (PASSES == 3) {
              tc_mma(d, smem_desc(ah + ko), smem_desc(b_lo_s + boff + ko), idesc, 1);
              tc_mma(d, smem_desc(al + ko), smem_desc(b_hi_s + boff + ko), idesc, 1);
            }
          }
          tc_commit(t_full + ts);
          if (++ts == kTcAcc) ts = 0, tph ^= 1u;
        }
        if (*fail) break;
        tc_commit(a_empty + as);  // the tile's MMAs have read A slot as
        if (++as == kTcA) as = 0, aph ^= 1u;
      }
      // every MMA issued has finished before TMEM is released
      tc_commit(mma_done);
      if (!tc_wait(mma_done, 0u, fail)) mbar_wait_bounded(mma_done, 0u, 1 << 24);
    }
  } else {
    // ---- epilogue warps: TMEM lanes 32 (warp mod 4) .. + 31, pose row 32 (warp mod 4) + lane of each tile
    const int q = warp & 3;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    long row = (long)blockIdx.x * 128 + 32 * q + lane;
    const float2 tiny = make_float2(1e-30f, 1e-30f);
    int ts = 0;
    uint32_t tph = 0;
    for (int k = 0; k < T && !*fail; ++k, row += step) {
      float2 best = make_float2(INFINITY, INFINITY), zmin = best, zsum = make_float2(0.f, 0.f);
      for (int r = 0; r < R; ++r) {
        if (!tc_wait(t_full + ts, tph, fail)) {
          *fail = 1;
          break;
        }
        tc_fence_after();
        float v[48];
        {
          float v0[16], v1[16], v2[16];
          const uint32_t col = 64u * (uint32_t)ts;
          tc_ld16(lane_base + col, v0);
          tc_ld16(lane_base + col + 16, v1);
          tc_ld16(lane_base + col + 32, v2);
          tc_wait_ld();
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = v0[e], v[16 + e] = v1[e], v[32 + e] = v2[e];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(t_empty + ts);  // this warp has read its lanes of the accumulator
        if (++ts == kTcAcc) ts = 0, tph ^= 1u;
        const float2* r2 = reinterpret_cast<const float2*>(r_s + 16 * r);
#pragma unroll
        for (int p = 0; p < 8; ++p) {  // constraints 16 r + 2 p and 16 r + 2 p + 1
          const float2 x = make_float2(v[6 * p], v[6 * p + 3]), y = make_float2(v[6 * p + 1], v[6 * p + 4]);
          const float2 z = make_float2(v[6 * p + 2], v[6 * p + 5]);
          float2 m;
          if (KIND == 0) {
            const float2 s2 = fma2(z, z, fma2(y, y, mul2(x, x)));
            m = fma2(make_float2(-s2.x, -s2.y), rsq2(add2(s2, tiny)), r2[p]);
          } else {
            const float2 s2 = fma2(y, y, mul2(x, x));
            m = fma2(make_float2(-s2.x, -s2.y), rsq2(fma2(s2, mul2(z, z), tiny)), r2[p]);
            zmin = min2(zmin, z);
            zsum = add2(zsum, z);  // NaN if some P_z is NaN
          }
          best = min2(best, m);
        }
      }
      if (*fail) break;
      float b = fminf(best.x, best.y);
      if (KIND == 1 && !(fminf(zmin.x, zmin.y) > 0.f && zsum.x == zsum.x && zsum.y == zsum.y)) b = -INFINITY;
      if (row < n_poses) dist[row] = b;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && *fail) atomicOr(status, kDevErrTimeout);
  if (warp == 4)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

size_t tc_dist_smem(int n, int passes) {
  const int n_pad = (n + 15) & ~15;
  return kTcA * (size_t)(passes == 3 ? tc_abuf<3>() : tc_abuf<1>()) + 2 * 64 * (size_t)(3 * n_pad) +
         4 * (size_t)n_pad + 8 * (2 * kTcA + 2 * kTcAcc + 1) + 16;
}

cudaError_t launch_tc_dist(purse_t h, int passes, const float* d_poses, long n_poses, float* d_dist, cudaStream_t st) {
  if (n_poses == 0) return cudaSuccess;
  const int n = h->n;
  const size_t smem = tc_dist_smem(n, passes);
  void (*kern)(const double*, const float*, int, double, double, double, double, const float*, long, float*, int*);
  if (h->kind == 0)
    kern = passes == 3 ? tc_dist_kernel<0, 3> : tc_dist_kernel<0, 1>;
  else
    kern = passes == 3 ? tc_dist_kernel<1, 3> : tc_dist_kernel<1, 1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // several CTAs per SM: the whole configurable shared memory for this kernel
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  // resident CTAs per SM from the register file, the threads, the shared memory and the accumulator
  // columns (every resident CTA holds its own, at most 512 per SM)
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  int dev = 0, smem_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e != cudaSuccess) return e;
  const int regs = (fa.numRegs + 7) & ~7;
  int per_sm = 65536 / (regs * kTcThreads);
  per_sm = std::min(per_sm, 2048 / kTcThreads);
  per_sm = std::min(per_sm, smem_sm / (int)(smem + 1024));
  per_sm = std::min(per_sm, (int)(512u / kTcCols));
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  per_sm = std::max(1, std::min(per_sm, tuned_config(kTuneDist, h->kind, n, n_poses, passes, per_sm)));
  const long tiles = (n_poses + 127) / 128;
  const long cap = (long)per_sm * h->sm_count;
  const int grid = (int)(tiles < cap ? tiles : cap);
  kern<<<grid, kTcThreads, smem, st>>>(h->tables.f64, h->tables.f32, n, h->K.fx, h->K.fy, h->K.cx, h->K.cy, d_poses,
                                       n_poses, d_dist, h->d_status);
  return cudaGetLastError();
}

}  // namespace purse
