/*
 * megaparticles.h -- C ABI of the GB300 (sm_103a) implementation of the
 * MegaParticles hot path: Koide, Oishi, Yokozuka, Banno, "MegaParticles:
 * Range-based 6-DoF Monte Carlo Localization with GPU-Accelerated Stein
 * Particle Filter", ICRA 2024 (arXiv 2404.16370).
 *
 * One filter step (mp_step) runs, on the context's CUDA stream and entirely in
 * this library's kernels:
 *   prediction                 Sec. III-B, Eq. 1
 *   scan Gaussians             Sec. III-C, GICP point model
 *   neighbour list update      Sec. III-C, Eq. 9-10, Algorithm 1
 *   likelihood + Gauss-Newton  Sec. III-C, Eq. 2-4 (NNF lookup)
 *   particle state update      Sec. III-C, Eq. 4-8 (GN step, SVGD)
 *   posterior propagation      Sec. III-D, Eq. 11 (+ representative state)
 *
 * Conventions shared by every entry point:
 *  - Pointers may be host or device memory; the library asks the CUDA runtime
 *    (cudaPointerGetAttributes) and copies accordingly. Device pointers must
 *    belong to the device that was current at mp_init_map.
 *  - Ownership: the context owns all device state (a map shared through
 *    mp_init_map_shared: jointly with the other contexts on it). Inputs are copied before the
 *    call returns (or enqueued on the context stream, for device pointers: the
 *    caller keeps them alive until the stream reaches that point). Outputs go
 *    to caller-allocated buffers.
 *  - Synchronisation: mp_init_map, mp_init_particles and the getters
 *    synchronise the context stream; mp_step and mp_run_stages only enqueue.
 *  - Errors: every call returns MP_OK (0) or a negative code; a message is kept
 *    in the context (mp_last_error). No exception crosses the ABI. After
 *    MP_ECUDA the context should be destroyed.
 *  - Poses are float32[7] = (qx, qy, qz, qw, tx, ty, tz), sensor-to-map, unit
 *    quaternion (Hamilton). Twists are (omega, v), rotation first (the order
 *    of W^K in Eq. 7).
 *  - Sizes: n_particles <= 2^26; the NNF grid holds < 2^31 voxels; scans hold
 *    at most params.max_scan points.
 */
#ifndef MEGAPARTICLES_H
#define MEGAPARTICLES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MP_OK 0
#define MP_EINVAL (-1)    /* bad argument, size or state                      */
#define MP_ENOMEM (-2)    /* device allocation failed                         */
#define MP_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed      */
#define MP_ETIMEOUT (-4)  /* a bounded device-side wait gave up               */
#define MP_ENOTINIT (-5)  /* particles not initialised                        */

typedef struct mp_ctx mp_ctx;

/* Filter constants. Printed in the paper: nnf_res (Sec. III-C: 0.1 m indoor,
 * 0.2 m outdoor), sigma_r = 5 rad^-1 and sigma_t = 2.5 m^-1 (Eq. 7), K (Sec.
 * III-C, e.g. 20), post_iters (Sec. III-D, e.g. 10). The others are readings
 * of what the paper leaves open: r_max (NNF search radius), c_max (per-point
 * cost truncation), alpha and lsh_sigma (Eq. 10), lambda/eps (GN damping),
 * eps_cov/r_cov/cov_k/cov_min (GICP covariances), C (bucket window),
 * n_buckets_log2 (N^B = 2^n_buckets_log2). */
typedef struct mp_params {
    float nnf_res, r_max, c_max;
    float sigma_r, sigma_t;
    float alpha, lsh_sigma;
    float lambda, eps;
    float eps_cov, r_cov;
    int32_t K, C;
    int32_t cov_k, cov_min;
    int32_t post_iters;
    int32_t n_buckets_log2;
    int32_t max_scan;
    uint64_t seed;
    /* 0 (default): the SVGD update of Eq. 6 as printed. 1: the repulsive sum
     * of particle i is multiplied by (H_i + lambda diag H_i + eps I)^-1, the
     * matrix of its own Gauss-Newton step, so that it scales like the steps
     * psi_j it is added to (a Stein variational Newton reading; not the
     * paper's printed update); a particle without a step (fewer than 6
     * inliers or a non-positive pivot) gets no repulsion. */
    int32_t svgd_precond;
    /* Floor of the initial posterior (Sec. III-D), in nats: p_i is evaluated
     * as exp(max(l_i - max_j l_j, -post_floor)) with l = log prior +
     * log-likelihood, so that no particle's posterior -- and so no particle's
     * prior at the next step -- is an exact zero (without it, FP64 exp
     * underflows for every particle more than ~745 nats below the best, and
     * those particles could never become the representative state again,
     * whatever their later likelihood). Default 700 (the range of FP64 exp);
     * 0 = no floor (the plain exp(l - max l)). Not printed in the paper. */
    float post_floor;
} mp_params;

#define MP_PRESET_BOX_ROOM 0   /* 0.1 m NNF, r_max 1 m, K = C = 16           */
#define MP_PRESET_OUTDOOR 1    /* 0.2 m NNF, r_max 2 m, K = C = 32           */

/* Fill *p with the defaults of a preset. n_particles sets n_buckets_log2 =
 * ceil(log2(n_particles)). Returns MP_EINVAL for an unknown preset. */
int mp_default_params(mp_params* p, int preset, int64_t n_particles);

/* Map preprocessing (Sec. III-A map M; Sec. III-C point Gaussians and the
 * nearest neighbour field m^nnf). xyz: n_map x 3 float32 map points. Computes
 * each point's GICP normal from its cov_k nearest points within r_cov (fewer
 * than cov_min: the point is unused), then the NNF: for every voxel of the map
 * box padded by r_max, the nearest valid map point to the voxel centre within
 * r_max (-1 if none). cuda_stream: a cudaStream_t the context will use for all
 * its work (NULL = legacy default stream). On success *ctx owns the device
 * memory. Errors: MP_EINVAL (NULL/empty input, bad params, grid too large),
 * MP_ENOMEM, MP_ECUDA; *ctx is NULL on error. */
int mp_init_map(mp_ctx** ctx, const float* xyz, int64_t n_map, const mp_params* p, void* cuda_stream);

/* A context on the map of another (no counterpart in the paper: several
 * filters localising in one map, e.g. the instances of a batch). *ctx gets its
 * own particles, scan buffers, parameters and stream, and reads src's device
 * map (points, normals, records, NNF) without a copy; the map's device memory
 * is freed with the last context that uses it, whichever is destroyed last.
 * The map is read-only after mp_init_map, so contexts sharing it may step on
 * different streams. p may differ from src's parameters except in those that
 * define the map: nnf_res, r_max, r_cov, cov_k and cov_min must be equal.
 * Synchronises src's stream and cuda_stream. Errors: MP_EINVAL (NULL
 * argument, src without a map, map parameters that differ, another device
 * than src's), MP_ENOMEM, MP_ECUDA; *ctx is NULL on error. Creating and
 * destroying contexts that share a map is thread-safe with respect to the
 * count of its users. */
int mp_init_map_shared(mp_ctx** ctx, mp_ctx* src, const mp_params* p, void* cuda_stream);

/* Particle set X_t (Sec. III-A), uniform prior, neighbour lists = {self}.
 * With poses_or_null (n x 7 float32) the poses are copied; otherwise each
 * particle is drawn on the device from Philox(seed): x, y, z, roll, pitch, yaw
 * uniform in [lo, hi] (R = Rz(yaw) Ry(pitch) Rx(roll)), or a uniform SO(3)
 * rotation when all three angle ranges span >= 2 pi (Sec. IV-A, full SO(3)).
 * log_prior_or_null: n float64 log prior weights (state import); NULL =
 * uniform. Resets the step counter. Errors: MP_EINVAL, MP_ENOMEM, MP_ECUDA. */
int mp_init_particles(mp_ctx* ctx, int64_t n_particles, const float lo[6], const float hi[6],
                      const float* poses_or_null, const double* log_prior_or_null);

/* One filter step on one scan P_t (n_scan x 3 float32, sensor frame).
 * odom_T: row-major 4x4 float64 relative motion dT_t (NULL = identity);
 * odom_cov: 6x6 float64 covariance Sigma^dT of the tangent noise (rotation
 * first; NULL = no noise). n_scan = 0 is a blackout step: prediction, the
 * neighbour list update and the posterior smoothing run with a zero
 * log-likelihood; likelihood and SVGD are skipped. Enqueued on the context
 * stream; advances the step counter. Errors: MP_EINVAL (n_scan > max_scan,
 * NULL scan with n_scan > 0), MP_ENOTINIT, MP_ECUDA. */
int mp_step(mp_ctx* ctx, const float* scan_xyz, int32_t n_scan, const double odom_T[16],
            const double odom_cov[36]);

/* Posterior after the last step (Sec. III-D): poses_out (n x 7 float32),
 * prob_out (n float64, sums to 1), best_pose (7 float32: the particle with the
 * highest posterior, smallest index on ties) and best_prob. Any output may be
 * NULL. Synchronises the stream; reports MP_ETIMEOUT if a device-side wait gave
 * up during the step. */
int mp_get_posterior(mp_ctx* ctx, float* poses_out, double* prob_out, float best_pose[7], double* best_prob);

/* Frees every resource of the context (NULL is accepted). */
int mp_destroy(mp_ctx* ctx);

/* Message of the last error of ctx ("" if none). With ctx NULL: the message
 * of the last failure, on the calling thread, of a call that has no context
 * to keep it (mp_init_map, mp_init_map_shared, the batch calls,
 * mp_posterior_init_noalloc, the proposal network's calls). The library
 * prints nothing. */
const char* mp_last_error(const mp_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Stage-level access (the same kernels mp_step runs; used for parity tests,
 * profiling and state import/export).
 * ------------------------------------------------------------------------- */
#define MP_STAGE_PREDICT 0x001u      /* Eq. 1                                   */
#define MP_STAGE_SCAN 0x002u         /* scan Gaussians + compaction             */
#define MP_STAGE_LSH 0x004u          /* Eq. 9-10 keys (draws T^LSH, delta^LSH)  */
#define MP_STAGE_SORT 0x008u         /* Algorithm 1 distribute: stable sort (and the likelihood's visiting order) */
#define MP_STAGE_MERGE 0x010u        /* Algorithm 1 gather + list refinement    */
#define MP_STAGE_LIKELIHOOD 0x020u   /* Eq. 2-4 sums                            */
#define MP_STAGE_SOLVE 0x040u        /* psi = GN step                           */
#define MP_STAGE_SVGD 0x080u         /* Eq. 5-6                                 */
#define MP_STAGE_POSTERIOR 0x100u    /* Eq. 11 + argmax                         */
#define MP_STAGE_ALL 0x1FFu

/* Upload a scan / odometry for the current step without running anything.
 * Same argument rules as mp_step. */
int mp_set_scan(mp_ctx* ctx, const float* scan_xyz, int32_t n_scan);
int mp_set_odometry(mp_ctx* ctx, const double odom_T[16], const double odom_cov[36]);

/* Run the selected stages, in the order of the step, at the current step
 * index (which is not advanced). Enqueued only. */
int mp_run_stages(mp_ctx* ctx, uint32_t stage_mask);

/* Step index used by the random draws of the next stage run (mp_step advances
 * it by one). */
int mp_set_step_index(mp_ctx* ctx, uint64_t step);

/* Buffers readable (and, where noted, writable) as flat arrays, in particle
 * order unless noted. count = number of elements of the stated type. */
#define MP_BUF_POSES 1         /* n x 7 float32          rw                     */
#define MP_BUF_LOG_PRIOR 2     /* n float64               rw                     */
#define MP_BUF_KEYS 3          /* n uint32 LSH keys        r                     */
#define MP_BUF_BUCKETS 4       /* n uint32 key mod N^B     r                     */
#define MP_BUF_SORTED_IDS 5    /* n int32 stable order     rw                    */
#define MP_BUF_SEGMENTS 6      /* n x 2 int32 [lo, hi) of each particle's bucket in the sorted order  r */
#define MP_BUF_NBR_IDS 7       /* n x K int32, -1 padded   rw (current lists)     */
#define MP_BUF_NBR_K 8         /* n x K float32 k_ij       rw                     */
#define MP_BUF_NBR_D 9         /* n x K x 6 float32 d_ij   rw                     */
#define MP_BUF_GN 10           /* n x 29 float32: H (21, upper rows), b (6), log-lik, inliers  r */
#define MP_BUF_PSI 11          /* n x 6 float32 GN steps   rw                     */
#define MP_BUF_POST 12         /* n float64 posterior      r                      */
#define MP_BUF_POST_INIT 13    /* n float64 initial posterior (before Eq. 11)  r  */
#define MP_BUF_LOGLIK 14       /* n float32 log-likelihood rw                     */
#define MP_BUF_SCAN_NORMALS 15 /* n_scan x 3 float32       r                      */
#define MP_BUF_SCAN_VALID 16   /* n_scan uint8             r                      */
#define MP_BUF_MAP_NORMALS 17  /* n_map x 3 float32        r                      */
#define MP_BUF_MAP_VALID 18    /* n_map uint8              r                      */
#define MP_BUF_LSH 19          /* 13 float64: T^LSH q (4), t (3), delta (6)  r    */
#define MP_BUF_PHI 20          /* n x 6 float32 SVGD update r                     */
#define MP_BUF_VISIT_ORDER 21  /* n int32 the likelihood's visiting order: particle ids by the Morton code
                                  of their position's cell (cubes of 2^s NNF voxels, s the smallest
                                  shift leaving at most 32 cubes along every NNF axis, positions
                                  clamped to the grid), LSH order (MP_BUF_SORTED_IDS) within a cell.
                                  Written by MP_STAGE_SORT; no result depends on it (a
                                  permutation set here lasts until the next sort).  rw */

/* Element count of a buffer (0 if not allocated). */
int mp_buffer_size(mp_ctx* ctx, int which, int64_t* count);
/* Copy a buffer out (synchronises the stream). count must equal its size. */
int mp_get_buffer(mp_ctx* ctx, int which, void* dst, int64_t count);
/* Overwrite a writable buffer (synchronises the stream). Index buffers the
 * kernels gather through are checked on the host first: MP_BUF_SORTED_IDS and
 * MP_BUF_VISIT_ORDER must be permutations of [0, n), MP_BUF_NBR_IDS entries
 * must lie in [-1, n); otherwise MP_EINVAL and nothing is written. */
int mp_set_buffer(mp_ctx* ctx, int which, const void* src, int64_t count);

/* NNF values of m voxels (m x 3 int32 integer coordinates; outside the grid:
 * -1). Synchronises. */
int mp_nnf_query(mp_ctx* ctx, const int32_t* vox, int64_t m, int32_t* out);

/* NNF grid geometry: origin o, dims n, inv_res = 1/res and off = -(o*inv_res)
 * (FP32), such that a point q has voxel floor(fma(q, inv_res, off)); n_valid =
 * number of map points with a covariance. */
int mp_map_info(mp_ctx* ctx, float origin[3], int32_t dims[3], float* inv_res, float off[3], int64_t* n_valid);

/* Per-stage device timing with CUDA events on the context stream.
 * mp_set_timing(ctx, 1) enables it and resets every total (0 disables);
 * enabling adds two event records per stage run and no synchronisation.
 * mp_stage_times returns, in stage-bit order, the summed device time (ms_out,
 * 9 floats) and the number of runs (runs_out, 9 int64) of each stage since
 * timing was enabled, and in *pairs (may be NULL) the particle x scan-point
 * pairs the likelihood stage evaluated in that interval. Synchronises. */
int mp_set_timing(mp_ctx* ctx, int enable);
int mp_stage_times(mp_ctx* ctx, float ms_out[9], int64_t runs_out[9], int64_t* pairs);

/* Arithmetic precision of the likelihood stage (the mixed-precision form of
 * Eq. 2-4). MP_PREC_FP32 (default): every per-pair value in FP32.
 * MP_PREC_BF16 / MP_PREC_FP16: the scan-point transform R mu, the normal
 * rotation, the information matrix, the cost and the Jacobian products of
 * each (particle, point) pair are computed in packed 16-bit pairs (bf16x2 /
 * half2); the voxel decision q = (R mu) + t, the residual mu^M - q and the
 * Gauss-Newton sums stay FP32, and the 6x6 solve and the posterior
 * normalisation stay FP64. Results then differ from the FP32 path by the
 * 16-bit rounding (a voxel decision can move by one voxel; sums by ~1e-3
 * relative). Returns MP_EINVAL for any other value. */
#define MP_PREC_FP32 0
#define MP_PREC_BF16 1
#define MP_PREC_FP16 2
int mp_set_precision(mp_ctx* ctx, int precision);

/* Tile knob of the FP32 likelihood stage: the scan is split over `split`
 * CTAs per block of particles (1 to 64; default 1), whose partial sums are
 * added atomically into the Gauss-Newton sums (summation order, so the last
 * bits, then depend on scheduling). Splitting puts more CTAs to work when the
 * particles are few (a 4096-particle instance has 16 particle blocks for 152
 * SMs); mp_batch_create picks it per instance by timing. */
int mp_set_likelihood_split(mp_ctx* ctx, int split);

/* ---- Scan-to-scan GICP odometry (Sec. III-B, prediction step) ----------
 * mp_gicp registers scan src (n_src x 3, sensor frame at t) to scan tgt
 * (n_tgt x 3, sensor frame at t-1), host or device pointers: T_out (4x4
 * row-major) maps src points into the tgt frame, i.e. DeltaT_t = T_{t-1}^-1
 * T_t; cov_out (6x6 row-major, may be NULL) = H^-1, the inverse of the
 * Gauss-Newton Hessian sum J^T Omega J at the last iteration (rotation-first
 * twist). Point Gaussians as for scans (cov_k, cov_min, r_cov, eps_cov);
 * each src point with a Gaussian takes the nearest tgt point with a Gaussian
 * (FP32 decisions on T rounded to float, ties to the smaller index) within
 * r_max; damped Gauss-Newton (lambda, eps) from init_T (NULL: identity) for at
 * most max_iters iterations, stopping once every step component is below
 * 1e-6. n_corr / iters (may be NULL) receive the correspondences and the
 * iterations of the last step. Synchronises. MP_EINVAL when fewer than 6
 * correspondences remain or the system is singular.
 * mp_step_gicp: mp_step with odometry from mp_gicp against the previous
 * scan given to it (first scan, and the first after an empty one: no motion),
 * started from the previous motion estimate, covariance scaled by cov_scale. */
int mp_gicp(mp_ctx* ctx, const float* src, int32_t n_src, const float* tgt, int32_t n_tgt, const double init_T[16],
            int32_t max_iters, double T_out[16], double cov_out[36], int32_t* n_corr, int32_t* iters);
int mp_step_gicp(mp_ctx* ctx, const float* scan, int32_t n_scan, double cov_scale);

/* ---- Batched instances ------------------------------------------------
 * Many independent contexts (each with its own particles and parameters;
 * presets may differ; maps their own or shared through mp_init_map_shared)
 * stepped together. mp_batch_create plans one step of all instances as about
 * thirty grouped launches, each covering the blocks of every instance (one
 * kernel per phase: prediction, scan Gaussians, LSH keys, each radix pass,
 * merge, likelihood, solve, SVGD), and the posterior as one cooperative
 * persistent launch over all instances (bounded grid barriers between its
 * sub-steps; a barrier that gives up is reported as MP_ETIMEOUT by every
 * instance). It captures the plan on cuda_stream into a CUDA graph, twice
 * (two pinned staging slots); mp_batch_step replays one. Per
 * instance the scan size is fixed (n_scan[i] points every step) and every step
 * runs all stages, the prediction included (identity odometry without noise
 * is applied, not skipped). tune_scans (may be NULL; else one host scan per
 * instance) is used to pick, by timing, each instance's likelihood split
 * (mp_set_likelihood_split): alone first, then as a policy over the grouped
 * launch; the pick runs the scan, LSH and sort stages of each instance once on
 * its own stream. Contexts must use the FP32 likelihood and must not have
 * timing enabled; their streams only order other calls on them before and
 * after batch steps (they may be cuda_stream itself). The batch does not own
 * the contexts; destroy it before them, and do not re-initialise their
 * particles while it exists. A context in a batch is stepped only through
 * the batch (mp_batch_step returns MP_EINVAL otherwise); reading it
 * (mp_get_posterior, mp_get_buffer) is fine. */
typedef struct mp_batch mp_batch;
/* A new non-blocking CUDA stream and its release; *stream receives the
 * cudaStream_t. */
int mp_stream_create(void** stream);
int mp_stream_destroy(void* stream);
int mp_batch_create(mp_batch** batch, mp_ctx* const* ctxs, int n, const int32_t* n_scan,
                    const float* const* tune_scans, void* cuda_stream);
/* One step of every instance: scans[i] = n_scan[i] x 3 host floats (copied
 * before return), odom_T = n x 16 and odom_cov = n x 36 host doubles (NULL:
 * identity motion / no noise for all). Asynchronous: later calls on an
 * instance (mp_get_posterior, ...) are ordered after it. */
int mp_batch_step(mp_batch* batch, const float* const* scans, const double* odom_T, const double* odom_cov);
/* The likelihood split picked for instance i. */
int mp_batch_split(mp_batch* batch, int i, int* split);
int mp_batch_destroy(mp_batch* batch);

/* Number of kernels this context has launched so far. */
int mp_kernel_launches(mp_ctx* ctx, int64_t* count);

/* Test knobs of the failure path (no counterpart in the paper).
 * MP_DEBUG_WAIT_BUDGET: SM-clock-cycle limit of every bounded device wait
 * (default about 2 s; value <= 0 restores it). MP_DEBUG_STARVE_TX: when
 * non-zero, the likelihood kernel announces 16 bytes more than it copies for
 * its first scan chunk, so that chunk's barrier never completes and the
 * bounded wait gives up; the kernel then records the error (reported as
 * MP_ETIMEOUT by the next mp_get_posterior) and returns. No copy is left in
 * flight. MP_DEBUG_STARVE_BARRIER: when non-zero, the first grid barrier of
 * the posterior stage (one cooperative launch) waits for one CTA more than the
 * grid has, so every CTA's bounded wait gives up; the kernel records the error
 * for every instance it serves and returns. In a batch the first instance's
 * knob and wait budget when mp_batch_create captures the step apply, to the
 * posterior and to the batch's LSH/sort phase (also one cooperative launch). */
#define MP_DEBUG_WAIT_BUDGET 1
#define MP_DEBUG_STARVE_TX 2
#define MP_DEBUG_STARVE_BARRIER 3
int mp_debug_set(mp_ctx* ctx, int what, int64_t value);

/* ---------------------------------------------------------------------------
 * Allocation-free initial posterior. The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory when they
 * need it -- a real-time loop that allocates only at start-up (cudaMalloc can
 * synchronise the device and stall for milliseconds), or an application whose
 * device memory belongs to another allocator or a fixed budget.
 *
 * Computes, for n particles, p_i = exp(l_i - max l) / sum_j exp(l_j - max l)
 * with l_i = log_prior[i] + loglik[i] (log_prior NULL: 0), and the index of
 * the largest p_i (smallest index on ties): the plain definition, without
 * the posterior stage's floor. These equal that stage's initial posterior
 * (MP_BUF_POST_INIT) when its floor is off (mp_params.post_floor = 0), up to
 * the FP64 rounding of the sum, whose summation order differs; the index is
 * the same. log_prior (n
 * float64), loglik (n float32), post_out (n float64) and best_out (1 int64)
 * are DEVICE pointers of the current device, owned by the caller; host
 * memory (pageable or pinned) and other devices' memory are refused with
 * MP_EINVAL before anything is launched. The work is enqueued on cuda_stream
 * (NULL = legacy default stream) and the call does not synchronise.
 *
 * Degenerate input (every l_i = -inf, or some l_i NaN or +inf): the
 * normaliser is not a finite positive number, so *best_out = -1 and every
 * post_out[i] is NaN. The call still returns MP_OK (it does not wait for the
 * result): check best_out >= 0 before using it as an index.
 *
 * No memory is allocated: block partials live in one static device array of
 * MP_NOALLOC_SCRATCH_BYTES that every device loading the library holds until
 * the process exits. The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress, with the device current) and caches it; with
 * lazy module loading (the CUDA default) that first call also loads the
 * module, which places the array and the kernels on the device. Make that
 * first call a warm-up in the caller's allocation phase, before any stream
 * capture; later calls allocate nothing. All calls share the array, so calls
 * that overlap on the GPU race and must be serialised by the caller.
 * Errors: MP_EINVAL for NULL or non-device pointers and n outside [1,
 * MP_NOALLOC_MAX_PARTICLES], MP_ECUDA for a failed symbol lookup or launch;
 * the message is mp_last_error(NULL). */
#define MP_NOALLOC_MAX_PARTICLES (1 << 24)
#define MP_NOALLOC_SCRATCH_BYTES (262144 + 256)
int mp_posterior_init_noalloc(const double* log_prior, const float* loglik, int64_t n, double* post_out,
                              int64_t* best_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MEGAPARTICLES_H */
