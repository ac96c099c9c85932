/*
 * purse.h -- C ABI of the GB300 CLOSURE hot path (arXiv 2403.09990).
 *
 * A PURSE (pose uncertainty set, eq. 5 with Lambda_i = I, beta_i = r_i) is the
 * set of poses (R, t) in SE(3) whose residuals satisfy |g_i(R, t)| <= r_i for
 * every keypoint i, with
 *   3D-3D (Example 2, eq. 3):  g_i = b_i - (R a_i + t)
 *   2D-3D (Example 1, eq. 2):  g_i = z_i - pi(K (R Z_i + t)) in pixels,
 *                              pi(P) = (P_x/P_z, P_y/P_z), and P_z > 0 required.
 * The library samples the PURSE boundary with the strategic random walks of
 * Section IV (Alg. 2-5) and computes minimum enclosing geodesic balls (MEGB,
 * Section II) of the samples by geodesic gradient descent.
 *
 * Conventions for every call
 * - Every call returns a purse_status; PURSE_OK is 0.  On failure
 *   purse_last_error() returns a thread-local message.  Kernels are launched
 *   asynchronously on the given stream; errors detected on the device (a
 *   bounded wait that ran out, non-finite input) are recorded in the
 *   handle's device status word and returned by the next purse_sync().
 * - Pointers named d_* are device pointers owned by the caller; they must
 *   stay valid until the work on the stream completes.  Host pointers are
 *   read before the call returns.
 * - Rotations are unit quaternions (w, x, y, z) with w >= 0; a pose packed
 *   in 12 doubles is R row-major followed by t.
 * - Precision: 0 = FP32 (float buffers), 1 = FP64 (double buffers).
 * - A handle is not thread-safe; different handles are independent.
 * - purse_stream_t is a cudaStream_t (NULL = the legacy default stream).
 */
#ifndef PURSE_H
#define PURSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct purse_s* purse_t;
typedef void* purse_stream_t;

typedef enum { PURSE_3D3D = 0, PURSE_2D3D = 1, PURSE_REG = 2 } purse_kind;

typedef enum {
  PURSE_OK = 0,
  PURSE_ERR_ARG = 1,      /* invalid argument (sizes, NaN/Inf, r_i <= 0, ...) */
  PURSE_ERR_CUDA = 2,     /* a CUDA runtime call failed */
  PURSE_ERR_EMPTY = 3,    /* Step I found no pose inside the PURSE */
  PURSE_ERR_TIMEOUT = 4,  /* a bounded device wait ran out */
  PURSE_ERR_NOMEM = 5,    /* device allocation failed */
  PURSE_ERR_NUMERIC = 6,  /* non-finite value met on the device */
  PURSE_ERR_STATE = 7     /* call out of order (e.g. backward before solve) */
} purse_status;

typedef struct { double fx, fy, cx, cy; } purse_intrinsics;

/* Simulation parameters P of Alg. 1 (names of Alg. 2-5). */
typedef struct {
  int n_iter;           /* N_I   walk iterations, >= 0 */
  int n_perturb;        /* N_P   perturbations per iteration, 1..256 */
  int n_keep;           /* N_P*  kept perturbations, 1..min(32, N_P) */
  int n_steps;          /* N_T   step-ladder length, 1..32 */
  double omega0;        /* omega_0 angular speed [rad] (rotation sampler) */
  double v0;            /* v_0 centre speed [m] (translation sampler) */
  double gamma;         /* time-step decay, ladder Delta T = gamma^(m-1), in (0, 1] */
  double rot_perturb;   /* theta_p (R_p) */
  double trans_perturb; /* t_p */
  int perturb_units;    /* 0: t_p, theta_p relative to the PURSE scale; 1: raw m / rad */
  int sampler;          /* 0: dS_R sampler (Alg. 2/3); 1: dS_t sampler (Alg. 4/5) */
  int precision;        /* 0: FP32 samples and walk arithmetic; 1: FP64 */
} purse_params;

/* Create a handle owning device copies of one PURSE (eq. 5).
 * kind: PURSE_3D3D or PURSE_2D3D.  n: number of constraints, 3..256.
 * model: host n x 3 (a_i or Z_i); obs: host n x 3 (b_i) or n x 2 (pixels z_i);
 * radii: host n, each > 0 (r_i = beta_i); K: intrinsics for 2D-3D, NULL for 3D-3D.
 * All values must be finite.  Allocates device memory (PURSE_ERR_NOMEM). */
purse_status purse_create(int kind, int n, const double* model, const double* obs,
                          const double* radii, const purse_intrinsics* K, purse_t* out);

/* Noise bounded in the general norm of eq. 4, |e|_Lambda = sqrt(e^T Lambda_i e) <= r_i, for the
 * constraints of a 3D-3D (Lambda_i 3 x 3) or 2D-3D (2 x 2, pixels) PURSE: lam (host, n x d x d,
 * row-major, each symmetric positive definite; PURSE_ERR_ARG otherwise); NULL restores the
 * identity.  Each Lambda_i is factored once on the host (Cholesky, Lambda = U^T U) and the factors
 * are kept on the device.  With noise matrices: purse_sample (with or without the snap),
 * megb_backward, purse_sample_plain, purse_ransag (points drawn in the noise ellipsoids, acceptance
 * in that norm) and purse_dist mode 0 use them; purse_eval and purse_dist modes 1-2 return
 * PURSE_ERR_ARG.
 * Allocates device memory on the first call. */
purse_status purse_set_noise(purse_t h, const double* lam);

/* Create a handle of a pose-regression PURSE (Example 3, eq. PURSEreg): n pose hypotheses
 * (R_i, t_i), host n x 12 (R_i row-major, then t_i; each R_i a rotation to 1e-6), and radii
 * beta_rot (host n, the Frobenius distance |vec(R) - vec(R_i)| allowed) and beta_t (host n,
 * metres), each > 0; n in [1, 256].  The PURSE is every (R, t) within both radii of every
 * hypothesis.  Sampled by purse_sample (fused, no snap) or purse_sample_plain;
 * purse_ransag draws its seeds by convex combinations of the hypotheses; purse_dist takes mode 0;
 * megb_solve and megb_solve_exact take its samples like any other.  Allocates device memory. */
purse_status purse_create_regression(int n, const double* hyp, const double* beta_rot,
                                     const double* beta_t, purse_t* out);

purse_status purse_destroy(purse_t h);

/* Constraint evaluation (eq. 2/3, eq. 11).  d_poses: n_poses x 12 poses (R row-major,
 * t) in the given precision.  Outputs (each may be NULL):
 *   d_margin  n_poses x n  r_i - |g_i| (-inf for 2D-3D keypoints behind the camera)
 *   d_active  n_poses      index of the smallest margin (the constraint defining
 *                          dist(R, t, dS) of eq. 11), lowest index on ties
 *   d_grad    n_poses x 6  d|g_a| / d(phi, rho) for that active constraint a, under
 *                          R <- Exp(phi) R, t <- t + rho (0 when |g_a| = 0). */
purse_status purse_eval(purse_t h, int precision, const void* d_poses, int n_poses,
                        void* d_margin, int32_t* d_active, void* d_grad, purse_stream_t stream);

/* dist(R, t, dS) of eq. 11 -- min_i (r_i - |g_i|), -inf when a 2D-3D keypoint is behind the
 * camera -- for n_poses FP32 poses d_poses (n_poses x 12: R row-major, then t; 16-byte aligned),
 * written to d_dist (n_poses floats).  The pose transform of all constraints is one dense
 * contraction [poses x 16] . [16 x 3n] of the pose row (R, t, 1, 0, 0, 0) with a constraint
 * matrix (3D-3D: the residual R a_i + t - b_i; 2D-3D: P_x - u_i P_z, P_y - v_i P_z, P_z of
 * P = K (R Z_i + t)).  mode 0: FP32 on the CUDA cores (the per-pose formula of eq. 2/3);
 * mode 1: tensor cores (tcgen05, TF32) with both operands split into TF32 hi + lo and three
 * passes hi.hi + hi.lo + lo.hi accumulated in FP32 (about 2^-21 relative per product);
 * mode 2: one TF32 pass (about 2^-11).  Asynchronous on the stream. */
purse_status purse_dist(purse_t h, int mode, const float* d_poses, long long n_poses, float* d_dist,
                        purse_stream_t stream);

/* Step I (Section IV, RANSAG), FP64: trials tau = 0..n_trials-1 each pick three distinct
 * constraints (multiply-shift of words 0-2 of Philox stream (5, 0, 0, tau)) and draw one point
 * inside each noise region (stream (5, c, 0, tau), c = 1..3: lattice rejection in the ball for
 * 3D-3D, in the disk of pixels for 2D-3D -- see purse_sample for the word layout).
 * 3D-3D (Example 2): one pose fitted to the three pairs (least-squares rotation, Arun/Horn).
 * 2D-3D (Example 1): the poses of the perspective-three-point problem on the three pixels (up to
 * four; Grunert's quartic in the depth ratio, candidates in ascending order of its real roots).
 * Pose regression (Example 3): one pose per trial, the convex combination of all hypotheses with
 * weights uniform on the simplex (w_i = e_i / sum e, e_i = -log u_i, u_i = ((word_i >> 8) + 1/2)
 * 2^-24 from words 0..n-1 of stream (5, 0, 0, tau)): t = sum w_i t_i, R = proj_SO3(sum w_i R_i).
 * A candidate is accepted if it lies in the PURSE.  The first max_seeds accepted poses in
 * (trial, candidate) order are written to d_seeds (device, max_seeds x 12 doubles); *n_seeds
 * (host) receives their count.  Synchronises the stream.  PURSE_ERR_EMPTY if none. */
purse_status purse_ransag(purse_t h, uint64_t seed, int n_trials, int max_seeds,
                          double* d_seeds, int* n_seeds, purse_stream_t stream);

/* Step II (Alg. 3 or Alg. 5 by p->sampler): n_samples walks, walk w starting from seed pose
 * (w mod s0) of d_seeds (device, s0 x 12 doubles).  Writes the final pose of each walk:
 * d_q n_samples x 4 and d_t n_samples x 3 (precision p->precision).  d_trace (device, may be
 * NULL) receives per walk and iteration n_keep + 2 int16: the top-k perturbation indices in
 * rank order, then m0 and k0 (0-based; -1 when no candidate was feasible).
 * Random draws: Philox4x32-10, key = (low, high 32 bits of seed); word k of the stream named
 * (phase, j, i, w) is output lane k & 3 of counter (k >> 2, phase << 24 | j, i, w).  Phase 1/2:
 * the perturbations of iteration i of walk w in the dS_R / dS_t sampler; perturbations 2b and
 * 2b + 1 are the two points of words 0-1 and 2-3 of stream (phase, b, i, w), a point of words
 * (w0, w1) being rho (sqrt(1 - z^2) cos a, sqrt(1 - z^2) sin a, z) in the unit ball with
 * z = ((w0 >> 16) + 1/2) / 2^15 - 1, a = pi ((w0 & 0xFFFF) + 1/2) / 2^15 and
 * rho = (max of the three 10-bit fields of w1 + 1/2) / 1024 (no rejection), scaled by the
 * perturbation radius.  Phase 3/4: the random unit vector of the initial angular / centre
 * velocity, one word per attempt: X_c = 2 ((word >> 10c) & 1023) - 1023, accepted if
 * 2^14 <= |X|^2 <= 2^20, normalised.
 * d_snap (device, may be NULL): snap every final sample to the PURSE boundary along its walk's
 * last-move ray (rotation ray Exp(tau omega) R* for the dS_R sampler, translation ray t* + tau v for
 * dS_t; the paper has no snap -- it makes the balls differentiable): tau_hi = the smallest ladder
 * value gamma^m leaving S, bisection of [0, tau_hi] (24 steps FP32, 52 FP64) keeping the feasible
 * end, which replaces the sample in d_q / d_t.  Record per walk, 12 values in the sample precision:
 * j* (the active constraint, -1 if no ladder pose left S), ray kind (0 rotation, 1 translation),
 * ray direction (3), h'(tau*) = d|g_j*|/d tau, d|g_j*|/d y_j* (3; 2 used for 2D-3D), 3 unused.
 * Pass the records to megb_backward.  The snap works in the constraints' norm: with noise
 * matrices (purse_set_noise) h = |g_j*|_Lambda and d h / d y = Lambda g / h (eq. 4).  The ray's
 * residuals are formed once per sample in FP64 (from the FP64 table and pose) and the bisection
 * evaluates small increments in the walk precision; the snapped pose is formed in FP64.
 * Regression PURSEs (purse_create_regression) take no snap; their walks evaluate the part of each hypothesis a perturbation moves (dS_R: the
 * translations, dS_t: the rotations) per perturbation and the other part once per iteration, and
 * the ladder's two factors once per rung and kept perturbation, so purse_last_evals counts those
 * half-constraint evaluations. */
purse_status purse_sample(purse_t h, const purse_params* p, uint64_t seed, const double* d_seeds,
                          int s0, int n_samples, void* d_q, void* d_t, int16_t* d_trace, void* d_snap,
                          purse_stream_t stream);

/* Step II by the plain per-operation samplers (Alg. 3 / Alg. 5 in the paper's parallel form):
 * the same walks, draws, decisions, outputs and trace as purse_sample (no snap), computed by one
 * kernel per tensor operation of the listing (perturbation, dist of eq. 11, top_k_indices,
 * update_rotation / update_translation, in_purse, find_farthest) with every intermediate tensor
 * -- perturbed poses (W, N_P, 12), distances (W, N_P), kept indices (W, N_P*), ladder
 * candidates (W, N_T, N_P*, 12), in_purse flags (W, N_T, N_P*) -- in device memory, and every
 * constraint of every pose evaluated.  It is the per-instance comparator of the fused walk
 * kernel.  Arguments as for purse_sample.  The intermediates of up to about 2 GB of walks at a
 * time live in handle-owned scratch (grown with cudaMalloc; PURSE_ERR_NOMEM).
 * purse_last_evals afterwards returns n_samples N_I (N_P + N_T N_P*) n. */
purse_status purse_sample_plain(purse_t h, const purse_params* p, uint64_t seed, const double* d_seeds,
                                int s0, int n_samples, void* d_q, void* d_t, int16_t* d_trace,
                                purse_stream_t stream);

/* Number of (pose, constraint) evaluations the last purse_sample on this handle executed
 * (perturbation distances of eq. 11 plus in_purse checks of the step ladder up to m0).
 * Synchronises the stream; *evals is a host pointer. */
purse_status purse_last_evals(purse_t h, unsigned long long* evals, purse_stream_t stream);

/* Step III (Section II, geodesic gradient descent; step rule of Alg. 6): K iterations on the
 * n_rot rotation samples d_q (n_rot x 4) and on the n_tr translation samples d_t (n_tr x 3),
 * precision as given.  C_0 = first sample; C_k = SLERP(C_{k-1}, farthest sample, 1/k);
 * c_k = c_{k-1} + (farthest - c_{k-1}) / k.  d_result (device, 9 doubles):
 * C (4, w >= 0), c (3), D-hat (rad), d-hat (m).  d_farthest (device, may be NULL):
 * 2K int32, the farthest-sample indices of the rotation then the translation descent.
 * Either ball may be skipped with n = 0 (its result entries are 0); at most 2^31 - 2^21
 * samples per ball (PURSE_ERR_ARG beyond; the same bound holds for megb_solve_exact,
 * megb_backward and megb_solve_noalloc).
 * Uses handle-owned scratch; the input buffers must not change before megb_backward. */
purse_status megb_solve(purse_t h, int precision, int n_iters, const void* d_q, int n_rot,
                        const void* d_t, int n_tr, double* d_result, int32_t* d_farthest,
                        purse_stream_t stream);

/* megb_solve with the output rule of Alg. 6 (the appendix's SDP-based descent, whose listing
 * returns the projection onto SO(3) of the sum of its last 10 iterates): the same K iterations and
 * farthest samples, then the rotation centre is proj_SO3(sum of R(C_t), t = K - n_last + 1 .. K) --
 * computed as the eigenvector of the largest eigenvalue of sum C_t C_t^T, the unit quaternion that
 * maximises the same trace -- and the translation centre the mean of c_t over the same t; when
 * K + 1 < n_last, all iterates C_0 .. C_K are used.  The radii are the largest distances from these
 * centres (a final pass).  n_last = 1 gives megb_solve's result; n_last = 10 is the paper's rule.
 * Arguments and d_result / d_farthest layouts as for megb_solve, plus n_last >= 1 (PURSE_ERR_ARG
 * otherwise).  megb_backward differentiates megb_solve only: after a megb_solve_mean with
 * n_last > 1 on the handle it returns PURSE_ERR_ARG until the next megb_solve. */
purse_status megb_solve_mean(purse_t h, int precision, int n_iters, int n_last, const void* d_q,
                             int n_rot, const void* d_t, int n_tr, double* d_result,
                             int32_t* d_farthest, purse_stream_t stream);

/* Reverse-mode derivative of the balls of megb_solve with respect to the PURSE observations y_i
 * and radii r_i (the paper has no adjoint; the samples come from the discrete walks of Alg. 3/5,
 * so they are differentiated through the boundary snap of purse_sample's d_snap records).
 * Loss L = g . (C (4), c (3), D-hat, d-hat) with g = d_grad_result (device, 9 doubles).
 * Rotations are perturbed on the left, R -> Exp(delta) R.  The descent of Section II is
 * reversed with the SO(3) Jacobians (step k: A_k = (1/k) C_k J_r(phi_k / k) J_l(phi_k)^-1 C_{k-1}^T,
 * phi_k = Log(C_{k-1}^T R_{f_k}); iterates recomputed from d_farthest, not stored); the radius
 * uses dD = (C_K u)^T (delta_f* - eps_K), u the unit axis of C_K^T R_f*, f* the farthest sample
 * from the final centre (found again here with megb_solve's final pass); the translation ball
 * is an affine combination of its farthest samples.  A sample gradient v then moves the
 * sample's snapped ray parameter: d tau* = (d r_j* - dh/dy . d y_j*) / h'(tau*) with
 * tau-gradient v . direction, accumulated onto constraint j* of the sample's record.
 * Inputs: exactly the arguments given to megb_solve (precision, n_iters, d_q, n_rot, d_t, n_tr,
 * its d_result and d_farthest, unchanged since), plus the snap records of the rotation samples
 * (d_snap_rot, n_rot x 12) and of the translation samples (d_snap_tr, n_tr x 12), in the sample
 * precision.  A record whose ray does not move its ball's coordinate (a rotation ray in the
 * translation ball) or with j* = -1 contributes nothing.
 * Outputs (device, overwritten): d_grad_obs n x 3 (3D-3D, metres) or n x 2 (2D-3D, pixels)
 * doubles, d_grad_radii n doubles.  One thread runs the reverse sweep in FP64.  A record whose
 * j* is out of range or whose h' is 0 is skipped and flags PURSE_ERR_NUMERIC at the next
 * purse_sync.  Uses handle-owned scratch ((n_iters + 1) x 32 bytes beyond megb_solve's). */
purse_status megb_backward(purse_t h, int precision, int n_iters, const void* d_q,
                           const void* d_snap_rot, int n_rot, const void* d_t, const void* d_snap_tr,
                           int n_tr, const int32_t* d_farthest, const double* d_result,
                           const double* d_grad_result, double* d_grad_obs, double* d_grad_radii,
                           purse_stream_t stream);

/* Step III exactly as the paper states it (Section IV, Step III, the miniball of the samples):
 * the exact minimum enclosing ball of the n_tr translations d_t (n_tr x 3) in R^3, and of the
 * n_rot rotations d_q (n_rot x 4, unit quaternions) embedded in R^4 -- each quaternion taken on
 * the side of the reference rotation d_ref (device, 4 doubles; NULL: the first rotation sample)
 * -- whose centre is projected back to the unit sphere.  Output d_result (device, 9 doubles,
 * the layout of megb_solve): centre quaternion (w >= 0), centre translation, the largest
 * geodesic distance D from that rotation centre and the largest distance d from the
 * translation centre (0 for an empty set).  Method: a candidate set grown by the farthest
 * sample outside the exact ball of the candidates (FP64 passes over all samples, Welzl's
 * recursion on the candidates) until no sample lies outside (relative 1e-12); at most 96
 * candidates, beyond which the ball of the candidates is returned and PURSE_ERR_NUMERIC is
 * flagged for the next purse_sync.  Synchronises the stream (it reads a flag every eight
 * passes).  Uses handle-owned scratch. */
purse_status megb_solve_exact(purse_t h, int precision, const void* d_q, int n_rot, const void* d_t,
                              int n_tr, const double* d_ref, double* d_result, purse_stream_t stream);

/* megb_solve without any device allocation, for callers that must not allocate device memory
 * once they are running: real-time perception loops that reserve all memory at start-up
 * (cudaMalloc / cudaFree can synchronise the device and take unbounded time), and hosts whose
 * device memory is owned by another allocator.  The paper has no counterpart; the computation
 * and outputs are those of megb_solve, without a PURSE handle.
 * Scratch: one 64 KiB array in the library's device memory, which every GPU that loads the
 * library holds until the process exits.  Limits: n_iters <= 4096 (PURSE_ERR_ARG beyond).
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  The address is cached per device for the
 * life of the process: do not call cudaDeviceReset between calls (the reset unloads the
 * module, and the cached address would then point at freed memory).  The grid of the ball
 * kernels is capped at min(4 x SMs, 512) blocks (megb_solve: 4 x SMs); the farthest samples,
 * centres and radii are the same, ties going to the lowest index in both.  All calls share the one array and a call
 * leaves its contents behind (it re-initialises what must start at zero), so calls whose
 * work overlaps on the GPU (other streams, other host threads) race: serialise them. */
purse_status megb_solve_noalloc(int precision, int n_iters, const void* d_q, int n_rot, const void* d_t, int n_tr,
                                double* d_result, int32_t* d_farthest, purse_stream_t stream);

/* The walks' random streams, exposed for verification: for streams w = w0 .. w0+n_streams-1
 * named (phase, j, i, w) under key = seed, writes their first n_words Philox4x32-10 words to
 * d_words (device, n_streams x n_words uint32) and, if d_lattice is not NULL, the first accepted
 * lattice point of each stream (device, n_streams x 4 int32: X, Y, Z, attempts used; unit != 0
 * selects the unit-vector acceptance region 2^14 <= |X|^2 <= 2^20). */
purse_status purse_rng_words(uint64_t seed, uint32_t phase, uint32_t j, uint32_t i, uint32_t w0, int n_streams,
                             int n_words, uint32_t* d_words, int32_t* d_lattice, int unit, purse_stream_t stream);

/* ---- Autotuner.  Launch shapes chosen by measurement, cached per (operation, PURSE kind,
 * keypoint-count bucket ceil(log2 n), sample-count bucket floor(log2 samples), variant, GPU name).
 * The paper has no counterpart (its experiments fix the CuPy launch shapes).  Operations:
 *   0 walk -- warps per walk block, {8, 4, 2}; used by purse_sample (variant = sampler + 2 precision)
 *   1 megb -- samples per thread of the persistent ball kernel, i.e. blocks per ball, FP32
 *             {1 .. 64}, FP64 {1 .. 8}; used by megb_solve (variant = precision)
 *   2 dist -- resident CTAs per SM of the tensor-core distance kernel, {2, 1}; used by
 *             purse_dist modes 1 and 2 (variant = 3 split passes or 1)
 *   3 batch -- reserved (purse_batch_tune keeps its choice in the batch).
 * No shape changes a result.  The cache lives in the process; if the environment variable
 * PURSE_TUNE_CACHE names a file, it is read at the first lookup and every tuning call appends its
 * choice to it.  Tuning calls run the operation once with the current shape (argument checks and
 * warm-up), then once per candidate with CUDA events on the stream (the faster of two timed runs
 * after one untimed), store the fastest and report it (out may be NULL); they synchronise the
 * stream and leave the outputs of the last run in the buffers. */
typedef struct {
  int op;             /* the operation */
  int config;         /* the chosen shape */
  float ms;           /* its time */
  int default_config; /* the shape used without tuning */
  float default_ms;   /* its time (-1 if not measured) */
  int n_tried;        /* candidates that fitted and ran */
} purse_tune_result;

/* purse_sample's arguments (d_trace and d_snap are not used). */
purse_status purse_tune_walk(purse_t h, const purse_params* p, uint64_t seed, const double* d_seeds, int s0,
                             int n_samples, void* d_q, void* d_t, purse_tune_result* out, purse_stream_t stream);
/* megb_solve's arguments (d_farthest is not used). */
purse_status purse_tune_megb(purse_t h, int precision, int n_iters, const void* d_q, int n_rot, const void* d_t,
                             int n_tr, double* d_result, purse_tune_result* out, purse_stream_t stream);
/* purse_dist's arguments, mode 1 or 2. */
purse_status purse_tune_dist(purse_t h, int mode, const float* d_poses, long long n_poses, float* d_dist,
                             purse_tune_result* out, purse_stream_t stream);
/* Cache access without a GPU call: gpu = NULL means the current device's name.  get returns
 * PURSE_ERR_STATE when there is no entry; clear empties the process cache (the file is read again
 * at the next lookup). */
purse_status purse_tune_cache_get(int op, int kind, int n, long long n_samples, int variant, const char* gpu,
                                  purse_tune_result* out);
purse_status purse_tune_cache_put(int op, int kind, int n, long long n_samples, int variant, const char* gpu,
                                  int config, float ms);
purse_status purse_tune_cache_clear(void);

/* ---- Batches: many PURSEs solved by one graph of three launches (centre statistics, one
 * persistent walk launch over all (PURSE, sampler, walk) items, one block per ball).
 * PURSE p has kind kinds[p] and constraints offsets[p] .. offsets[p+1]-1 (3..256 each) of
 * model (host, x 3), obs (host, x 3; z ignored for 2D-3D) and radii (host, > 0); K (host,
 * n_purses entries) holds the intrinsics of the 2D-3D PURSEs (others ignored; may be NULL if
 * there are none).  2D-3D PURSEs use the dS_R samples for the rotation ball and the dS_t samples
 * for the translation ball.  3D-3D PURSEs use the dS_R samples for both balls when p3d->v0 = 0 (the
 * dS_t walks would not move); with p3d->v0 > 0 their dS_t walks run too and feed the translation
 * ball, as for 2D-3D. */
typedef struct purse_batch_s* purse_batch_t;

purse_status purse_batch_create(int n_purses, const int* kinds, const int* offsets, const double* model,
                                const double* obs, const double* radii, const purse_intrinsics* K,
                                purse_batch_t* out);

/* A batch of pose-regression PURSEs (Example 3, eq. PURSEreg): PURSE p has the hypotheses
 * [offsets[p], offsets[p+1]) (1..256 each) of the host arrays hyp (12 doubles per hypothesis: R_i
 * row-major, then t_i; as purse_create_regression), beta_rot and beta_t (> 0).  purse_batch_solve
 * then runs both samplers of every PURSE (reg_walk_one, the walk of the single-PURSE regression
 * kernel) with the parameter set p3d (p2d must be valid and is not used), one seed pose per PURSE,
 * and the balls as for the other kinds (rotation ball from the dS_R samples, translation ball from
 * the dS_t samples): PURSE p gives exactly purse_sample / megb_solve of a regression handle with key
 * seed + p.  No boundary snap, adjoint or noise matrices (purse_batch_set_grad / _set_noise answer
 * PURSE_ERR_ARG).  Errors and ownership as for purse_batch_create. */
purse_status purse_batch_create_regression(int n_purses, const int* offsets, const double* hyp,
                                           const double* beta_rot, const double* beta_t,
                                           purse_batch_t* out);

purse_status purse_batch_destroy(purse_batch_t b);

/* Noise bounded in the general norm of eq. 4 for every PURSE of the batch (the batched form of
 * purse_set_noise): d_lam is a HOST array of 9 doubles per keypoint in the CSR order of
 * purse_batch_create, the symmetric positive definite Lambda_i row-major as a 3 x 3 block (2D-3D
 * keypoints: its top-left 2 x 2 block is read, in pixels^-2).  The factors Lambda_i = U_i^T U_i are
 * taken on the host and kept in batch-owned device memory; walks, centre statistics, boundary snap
 * and purse_batch_backward then work in the Lambda-norm, with the same samples as purse_sample on
 * a handle given the same matrices by purse_set_noise.  NULL returns the batch to Lambda_i = I.
 * Errors: PURSE_ERR_ARG (non-finite, not symmetric or not positive definite), PURSE_ERR_NOMEM.
 * The next purse_batch_solve captures its graph anew. */
purse_status purse_batch_set_noise(purse_batch_t b, const double* lam);

/* Alg. 1 for every PURSE of the batch, FP32 walks: n_samples walks per PURSE and sampler from the
 * seed pose d_seeds[p] (device, n_purses x 12 doubles), the parameters p3d / p2d by kind (their
 * sampler and precision fields must be 0), Philox key seed + p for PURSE p (so PURSE p gets the
 * samples purse_sample would give with that key), then n_iters GGD iterations per ball.
 * d_results: device, n_purses x 9 doubles as in megb_solve.  n_samples <= 12288.
 * The launch sequence is captured into a CUDA graph on the first call and replayed while
 * parameters, sizes and buffers stay the same (the seed may change). */
purse_status purse_batch_solve(purse_batch_t b, const purse_params* p3d, const purse_params* p2d, uint64_t seed,
                               const double* d_seeds, int n_samples, int n_iters, double* d_results,
                               purse_stream_t stream);

/* Autotuner: times the walk launch for work-queue chunks {1, 4, 16, 64} x {4, 8} warps per block
 * on this batch with n_samples walks per PURSE, keeps the fastest for later solves and reports it
 * (outputs may be NULL).  Synchronises the stream. */
purse_status purse_batch_tune(purse_batch_t b, const purse_params* p3d, const purse_params* p2d, uint64_t seed,
                              const double* d_seeds, int n_samples, int* best_chunk, int* best_warps,
                              float* best_ms, purse_stream_t stream);

/* Copy the farthest-sample sequences of the last solve to d_out (device, n_purses x 2 n_iters int32:
 * rotation then translation sequence per PURSE).  PURSE_ERR_STATE before the first solve. */
purse_status purse_batch_copy_farthest(purse_batch_t b, int32_t* d_out, purse_stream_t stream);

/* Copy PURSE p's samples of the last solve (device, n_samples x 4 / x 3 floats each; any may be NULL):
 * dS_R quaternions and translations, dS_t quaternions and translations (the dS_t buffers are
 * unwritten for 3D-3D PURSEs solved with p3d->v0 = 0). */
purse_status purse_batch_copy_samples(purse_batch_t b, int p, float* d_q_rot, float* d_t_rot, float* d_q_tr,
                                      float* d_t_tr, purse_stream_t stream);

/* Differentiation of batched solves (enable = 1) or not (0, the default).  While enabled, every
 * purse_batch_solve also snaps the final samples to the boundary (as purse_sample's d_snap) and
 * keeps the snap records and the farthest samples of the final centres in batch-owned memory
 * (2 x n_purses x n_samples x 12 floats), for purse_batch_backward.  The paper has no adjoint;
 * see megb_backward.  Changing the flag re-captures the graph at the next solve. */
purse_status purse_batch_set_grad(purse_batch_t b, int enable);

/* Copy PURSE p's snap records of the last solve (device, n_samples x 12 floats each; either may be
 * NULL): dS_R walks, dS_t walks.  PURSE_ERR_STATE unless the last solve had gradients enabled. */
purse_status purse_batch_copy_snap(purse_batch_t b, int p, float* d_snap_rot, float* d_snap_tr,
                                   purse_stream_t stream);

/* megb_backward for every PURSE of the last solve (which must have had gradients enabled):
 * d_results the solve's results (device, n_purses x 9, unchanged since), d_grad_results dL/d
 * results (device, n_purses x 9); writes d_grad_obs (device, total keypoints x 3 doubles in the
 * CSR order of purse_batch_create; the third column is 0 for 2D-3D) and d_grad_radii (device,
 * total keypoints doubles).  One block per PURSE, the two sweeps on two warps, FP64; identical
 * to megb_backward on the PURSE's samples.  PURSE_ERR_STATE without such a solve. */
purse_status purse_batch_backward(purse_batch_t b, const double* d_results, const double* d_grad_results,
                                  double* d_grad_obs, double* d_grad_radii, purse_stream_t stream);

/* Synchronise the stream; *evals (host, may be NULL) receives the executed evaluations of the
 * last batch walk launch; returns the batch's device status. */
purse_status purse_batch_sync(purse_batch_t b, unsigned long long* evals, purse_stream_t stream);

/* Synchronise the stream and return (and clear) the handle's device status. */
purse_status purse_sync(purse_t h, purse_stream_t stream);

/* Thread-local message for the last failing call (never NULL). */
const char* purse_last_error(void);

/* Library build string: version, CUDA target. */
const char* purse_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PURSE_H */
