/*
 * pfreg.h -- C ABI of the GB300 (sm_103a) particle-filter 3D-3D rigid
 * registration library (libpfreg.so).
 *
 * The method: a sequential Monte Carlo (particle filter) search for the
 * rigid transform that aligns a source volume or binary mask with a target
 * (Eq. 1, Sec. 3.1), and the warp of every frame of the source sequence by
 * the estimate (Abstract; Sec. 3.3).  Each particle is a 6-DOF pose
 * [rx, ry, rz, tx, ty, tz] (radians, world units; Eq. 3) drawn within the given
 * rotation and translation limits; every iteration runs the cycle of the
 * Fig. 1 caption: prediction (perturbation), measurement (each particle's
 * transform warps the source into the target grid and a similarity is
 * reduced over the voxels), update (weights), estimation and resampling.
 *
 * Conventions
 *   Volumes: uint8, x fastest, index = x + X*(y + Y*z); dims = {X, Y, Z},
 *   each >= 2 and <= 2048.  Every grid carries an origin o (the world
 *   position of voxel (0,0,0)) and a voxel size s per axis (spacing; Table 1
 *   lists anisotropic ones), both in world units (mm; spacing 1 makes world
 *   units voxels).  Voxel p of a grid sits at o + s * p.  Translations and
 *   their limits are in the same world units, rotations in radians.  A pose
 *   maps target voxel p to the source continuous index
 *     q = (R (o_T + s_T * p - c) + c + t - o_S) / s_S
 *   (element-wise products and quotients by the spacings) with
 *   R = Rz(rz) Rx(rx) Ry(ry) and c = o_S + s_S * (dims_S - 1)/2 the world
 *   position of the source centre.  Masks: nonzero voxels are 1.
 *
 * Errors: every call returns PF_OK (0) or a negative PF_E* code and never
 * aborts; pf_last_error() gives the calling thread's last message.
 * Threading: a context belongs to one CUDA stream; calls on one context are
 * not thread-safe.  Different contexts are independent.
 */
#ifndef PFREG_H
#define PFREG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PF_OK 0
#define PF_EINVAL (-1)   /* bad argument: NULL, dims, limits, sizes, non-finite values */
#define PF_ENOMEM (-2)   /* a device or pinned-host allocation failed */
#define PF_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define PF_ETIMEOUT (-4) /* a bounded device-side wait gave up (the tensor-core kernels'
                            mbarrier waits; the registration kernels wait on nothing) */
#define PF_ESTATE (-5)   /* call not valid in the context's current state */

typedef struct pf_ctx pf_ctx;

/* A volume description.  data points to X*Y*Z bytes, x fastest; is_device =
 * 1 when it is a device pointer on the current device, 0 for host memory.
 * origin is the world position of voxel (0,0,0) and spacing the voxel size
 * per axis (Table 1 lists anisotropic ones), both in world units (mm);
 * voxel p sits at origin + spacing * p.  Translations and their limits are
 * in the same world units.  Spacing must be finite and > 0 (1 = voxel units). */
typedef struct {
    const void *data;
    int32_t dims[3];
    float origin[3];
    int32_t is_device;
    float spacing[3];
} pf_volume;

/* Measurement modes (similarity of Sec. 3.3-3.4):
 *   PF_MASK_DICE  nearest-neighbour mask sampling, Dice of Eq. 4 over the
 *                 whole target grid (source taken as 0 outside its grid);
 *   PF_MASK_NCC   nearest-neighbour mask sampling, squared NCC of Eq. 2 over
 *                 the overlap;
 *   PF_IMAGE_NCC  trilinear image sampling, squared NCC of Eq. 2 over the
 *                 overlap;
 *   PF_COMBINED   0.5 * (image NCC^2 + mask Dice), both from one sweep. */
typedef enum { PF_MASK_DICE = 0, PF_MASK_NCC = 1, PF_IMAGE_NCC = 2, PF_COMBINED = 3 } pf_mode;

/* Filter settings.  The paper states only that the method starts from
 * rotation and translation limits (Abstract); the remaining settings are this
 * library's readings of the Fig. 1 cycle:
 *   sigma_k = sigma0_frac * limit * sigma_decay^k   (perturbation scale)
 *   w_i     = (s_i / max s)^(2^gamma_log2)          (likelihood)
 *   score 0 when the overlap has fewer than min_overlap_frac * |target| voxels. */
typedef struct {
    int32_t mode;             /* pf_mode */
    int32_t n_particles;      /* 1 .. 65536 */
    float rot_limit[3];       /* radians, each in (0, pi/2] */
    float trans_limit[3];     /* world units (voxels at unit spacing), each in (0, 2048] */
    float sigma0_frac;        /* (0, 1] */
    float sigma_decay;        /* (0, 1] */
    int32_t gamma_log2;       /* 0 .. 10 */
    uint64_t seed;            /* Philox4x32-10 key */
    float min_overlap_frac;   /* [0, 1] */
    int32_t trace_estimate;   /* 1: after every iteration warp the source mask with the
                                 estimate and log its Dice against the target mask (Sec. 3.2:
                                 the masks validate image-based registration after each
                                 iteration); needs both masks, also in image mode */
    int32_t estimator;        /* pf_estimator: how the estimate's rotation is averaged */
    int32_t autotune;         /* 1: pick the measurement's tile shape (work items per warp)
                                 by timing the candidates on the initial cloud at creation,
                                 cached per (mode, dims, N) for the process; results are
                                 identical for every shape.  0: the default shape */
} pf_config;

/* Estimate of an iteration (Fig. 1 "estimation"), from the measured cloud
 * and its integer weights W (uniform when all W are 0):
 *   PF_EST_MEAN        weighted mean of the six pose parameters;
 *   PF_EST_QUATERNION  translations as above; the rotation is the weighted
 *                      quaternion average, the eigenvector of the largest
 *                      eigenvalue of sum_i W_i q_i q_i^T (sign-free), turned
 *                      back into the R = Rz Rx Ry angles.  Unlike the angle
 *                      mean it is not biased by the curvature of the angle
 *                      parametrisation when the cloud is wide. */
typedef enum { PF_EST_MEAN = 0, PF_EST_QUATERNION = 1 } pf_estimator;

/* Fill cfg with the defaults: PF_MASK_DICE, N = 256, limits 15 deg / 8 voxels,
 * sigma0_frac 0.25, sigma_decay 0.8, gamma_log2 5, seed 0,
 * min_overlap_frac 0.01, trace_estimate 0, estimator PF_EST_MEAN, autotune 0. */
void pf_config_default(pf_config *cfg);

/* Create a registration context (Sec. 3.1 problem statement: source and target
 * volumes or masks, limits, N).  Copies (or bit-packs) the volumes into
 * context-owned device memory on `cuda_stream` (a cudaStream_t; NULL = the
 * legacy default stream), counts the target mask, and draws the initial
 * particles uniformly within the limits (iteration index 0).
 *   Image modes need src/tgt; mask modes need src_mask/tgt_mask; the combined
 *   mode needs all four, with each mask on its image's grid.  Image mode may
 *   also take both masks (on the image grids) to trace the estimate's Dice.
 *   Unused volumes may be NULL.  The caller may free its buffers when the
 *   call returns.
 * Errors: PF_EINVAL (missing volume, dims, limits, N), PF_ENOMEM, PF_ECUDA.
 * On error *out is set to NULL. */
int pf_register_init(pf_ctx **out, const pf_volume *src, const pf_volume *tgt,
                     const pf_volume *src_mask, const pf_volume *tgt_mask,
                     const pf_config *cfg, void *cuda_stream);

/* Run n_iters filter iterations k .. k+n_iters-1 (Fig. 1 cycle): for k > 0
 * perturb every particle, then pose -> matrix, measure, score, weights,
 * estimate, resample.  Asynchronous on the context's stream; each iteration
 * is one CUDA-graph launch.  Errors: PF_EINVAL (n_iters < 0), PF_ECUDA. */
int pf_step(pf_ctx *ctx, int32_t n_iters);

/* Synchronise the stream and return the estimate of the last iteration
 * (Fig. 1 "estimation": the weighted mean pose, or the quaternion average
 * of pf_config.estimator) and, when score_out is not NULL, the score of that
 * pose (one extra measurement).  Errors: PF_EINVAL (NULL ctx or pose_out),
 * PF_ESTATE (before the first pf_step), PF_ECUDA. */
int pf_estimate(pf_ctx *ctx, float pose_out[6], double *score_out);

/* Seed the cloud from a proposal (the learned approach named as future work
 * in Sec. 6: a predicted mean and spread seed and shrink the particle cloud).
 * Replaces the initial particles by x_id = clamp(mean_d + std_d eps_id, -L_d,
 * L_d), eps the bounded unit-variance Irwin-Hall draw (u1+u2+u3+u4-2) sqrt 3
 * of Philox counter (i, 0, 3, d), and makes std the perturbation base:
 * sigma_kd = std_d * sigma_decay^k (instead of sigma0_frac * L_d).  mean /
 * std: [rx ry rz tx ty tz] in radians and world units.  Only before the first
 * pf_step.  Synchronous; re-captures the iteration graph.
 * Errors: PF_EINVAL (NULL, non-finite mean, std outside (0, 1e6]),
 * PF_ESTATE (after the first iteration, or while profiling is armed), PF_ECUDA. */
int pf_seed_gaussian(pf_ctx *ctx, const float mean[6], const float std[6]);

/* Release the context and its device memory (NULL is accepted; no
 * counterpart in the paper).  Waits for the context's stream first. */
int pf_register_destroy(pf_ctx *ctx);

/* Warp every frame of a sequence by one pose (Abstract; Sec. 3.3: the
 * transform found on the end-diastolic frame is applied to all frames).
 * frames_in / frames_out: host arrays of n_frames DEVICE pointers, each frame
 * src_dims resp. tgt_dims bytes.  out(p) = round-half-even of the trilinear
 * sample (interp = 1) or the nearest voxel (interp = 0) of the source at q(p),
 * 0 where q(p) falls outside the source grid.  Spacings may be NULL (1).
 * Allocates nothing; runs asynchronously on cuda_stream.  Errors: PF_EINVAL
 * (NULL, dims, spacing, pose rotation outside [-pi/2, pi/2], non-finite
 * pose), PF_ECUDA. */
int warp_sequence(const uint8_t *const *frames_in, int32_t n_frames, const int32_t src_dims[3],
                  const float src_origin[3], const float src_spacing[3], uint8_t *const *frames_out,
                  const int32_t tgt_dims[3], const float tgt_origin[3], const float tgt_spacing[3],
                  const float pose[6], int32_t interp, void *cuda_stream);

/* ---- batches: many registrations stepped together ---- */

/* A batch steps several registrations (each created by pf_register_init, all
 * on one device and one stream, any mix of modes, volume sizes and particle
 * counts) together.  One batch iteration is one CUDA-graph launch: prediction
 * of every particle of every running registration, their measurements (image,
 * mask and combined registrations as three concurrent launches over their
 * concatenated work items; a registration with at least 120000 measurement
 * work items -- 32 target rows of one particle each, enough to fill the GPU
 * for several waves -- gets its own launch in the same graph instead) and one
 * update/resampling block per registration.
 * n_iters[r] is registration r's total iteration count.  Members are ordered
 * by remaining iterations, so the running ones are a prefix; one graph is
 * captured per such prefix (on first use) and its grids cover only the
 * running members' work.  Every registration
 * follows exactly the arithmetic of pf_step (same results bit for bit).
 * While in a batch, a context must not be stepped on its own (the batch
 * counts the remaining iterations on the host); its state,
 * estimate and log are read with the usual calls.  Tracing is not applied in
 * batches.  The batch borrows the contexts: destroy it before them.
 * Errors: PF_EINVAL (NULL, n outside 1..65536, repeated context, different
 * devices or streams, negative count), PF_ENOMEM, PF_ECUDA. */
typedef struct pf_batch pf_batch;
int pf_batch_create(pf_batch **out, pf_ctx *const *ctxs, int32_t n, const int32_t *n_iters);
/* When every member was created with autotune = 1 and none has run yet,
 * pf_batch_create also picks the tile shape of the batch's measurement
 * launches by timing the candidates on the members' initial clouds.
 * pf_batch_tile_shape reports it (work items per warp). */
int pf_batch_tile_shape(pf_batch *b, int32_t *items_per_warp);
/* Launch n_iters batch iterations, each the Fig. 1 cycle of every running
 * member (asynchronous on the contexts' stream). */
int pf_batch_step(pf_batch *b, int32_t n_iters);
/* Launch as many batch iterations as the longest remaining registration needs. */
int pf_batch_run(pf_batch *b);
int pf_batch_destroy(pf_batch *b);

/* ---- one iteration in two halves: the measurement sharded over processes ---- */

/* The measurement is > 99 % of an iteration and each particle's moments are
 * independent (Fig. 1 "measurement"), so several processes (one per GPU) can
 * share one registration: each creates the same context (same volumes,
 * config and seed), and per iteration
 *   pf_step_measure(ctx, lo_r, hi_r)      on rank r, disjoint slices covering 0..N
 *   element-wise integer SUM of the moment buffers over the ranks
 *   pf_step_update(ctx)                   on every rank
 * The prediction and the update are repeated on every rank (cheap and
 * deterministic), so every rank holds the same cloud, bit for bit equal to
 * pf_step on one GPU: outside its slice a rank's moments stay 0 and exactly
 * one rank contributes each word, so the sum (in uint64 or int64) is exact.
 *
 * pf_step_measure: predict (k > 0: perturb) all N particles, zero all
 * moments, measure particles p_begin .. p_end-1 (0 <= p_begin <= p_end <= N).
 * pf_step_update: scores, weights, estimate, resampling, log (and the traced
 * estimate Dice), k += 1.  Both are asynchronous on the context's stream;
 * they are plain launches, not the iteration graph, and are not timed by
 * pf_profile_*.  Errors: PF_EINVAL (NULL, slice out of range), PF_ECUDA. */
int pf_step_measure(pf_ctx *ctx, int32_t p_begin, int32_t p_end);
int pf_step_update(pf_ctx *ctx);

/* The device address of the context's moment buffer, uint64 [N][12] (layout
 * of pf_get_state), for a collective that sums it in place between the two
 * halves.  Owned by the context; valid until pf_register_destroy.  *n_words =
 * 12 N.  Errors: PF_EINVAL (NULL). */
int pf_moments_device(pf_ctx *ctx, uint64_t **moments, int64_t *n_words);

/* ---- inspection, checkpoint and test exports (host buffers, synchronous) ---- */

/* Number of iterations run so far (the next iteration's index k; Fig. 1
 * iterations).  Synchronous. */
int pf_get_iteration(pf_ctx *ctx, int32_t *k_out);

/* Copy the state of the last iteration to host buffers (any may be NULL):
 *   poses_measured [6][N]  the cloud that was measured (SoA, DOF-major)
 *   moments        [N][12] n S1 S2lo S2hi ST T1 T2 0 | n_nn A B C: image
 *                          moments of the trilinear samples rounded to
 *                          s_q = rint(2^15 s) over the overlap (S2 = sum s_q^2
 *                          as two 64-bit words), then the mask counts
 *   scores [N], weights [N] (W = floor(w * 2^24)), resample_idx [N]
 *   poses_next     [6][N]  the resampled cloud the next iteration starts from */
int pf_get_state(pf_ctx *ctx, float *poses_measured, uint64_t *moments, double *scores,
                 uint64_t *weights, int32_t *resample_idx, float *poses_next);

/* Checkpoint resume: replace the cloud ([6][N] host, within the limits) and
 * set the iteration index to k (the counter-based RNG makes the continuation
 * bit-identical to an uninterrupted run). */
int pf_set_state(pf_ctx *ctx, const float *poses6xN, int32_t k);

/* Per-iteration log of the last min(k, capacity, 4096) iterations, oldest
 * first (any array may be NULL): est [count][6] (fp64 estimate), best [count]
 * (max score), ess [count] (effective sample size from the integer weights),
 * evals [count] (particle-voxel evaluations measured: the summed overlap
 * counts), est_dice [count] (Dice of the masks at the estimate rounded to
 * fp32, -1 unless trace_estimate).  *count_inout: in = capacity of the
 * caller's arrays, out = rows written. */
int pf_get_log(pf_ctx *ctx, double *est, double *best, double *ess, uint64_t *evals, double *est_dice,
               int32_t *count_inout);

/* Measure M given 3x4 matrices (host, [M][12] = r00 r01 r02 b0 | r10 ... b2)
 * with offset a (host float[3]): q = R (p - a) + b.  Writes moments [M][12]
 * (host) in the layout of pf_get_state.  Used to inject exact matrices. */
int pf_measure_matrices(pf_ctx *ctx, const float *mats, int32_t M, const float a[3],
                        uint64_t *moments_out);

/* Allocation-free variant of pf_measure_matrices (no counterpart in the
 * paper: it is a service for callers that cannot allocate device memory once
 * they are running -- an acquisition or control loop that must not stall on
 * the allocator or fail midway, a process held to a fixed device-memory
 * budget after start-up, or code where allocation calls are not permitted).
 * Same inputs and output as pf_measure_matrices (host matrices, host
 * moments [M][12]) with M <= PF_NOALLOC_MAX_MATRICES; larger M returns
 * PF_EINVAL.  It calls no cudaMalloc or cudaFree: the uploaded matrices and
 * the moment accumulators live in one fixed library-wide device array
 * (PF_NOALLOC_MAX_MATRICES x 144 bytes, 576 KiB) that every GPU loading the
 * library holds until the process exits.  The device the context was created
 * on must be the calling thread's current device (else PF_EINVAL, before
 * anything is copied): the array has one copy per device.  The first call on
 * a device looks up that array's device address (once per device); make that
 * first call before any CUDA stream capture.  All calls share the one array:
 * calls that overlap on the GPU (different streams or contexts at the same
 * time) race; the accumulators are cleared at the start of every call.
 * Synchronous. */
#define PF_NOALLOC_MAX_MATRICES 4096
int pf_measure_matrices_noalloc(pf_ctx *ctx, const float *mats, int32_t M, const float a[3],
                                uint64_t *moments_out);

/* Pose -> (matrix [12], offset a [3]) exactly as the filter computes it
 * (Eq. 3 with the spacings: M = diag(1/s_S) R diag(s_T), b and a in source
 * resp. target voxel units).  src_spacing / tgt_spacing may be NULL (1). */
int pf_pose_matrix(const float pose[6], const int32_t src_dims[3], const float src_origin[3],
                   const float src_spacing[3], const float tgt_origin[3], const float tgt_spacing[3],
                   float mat_out[12], float a_out[3]);

/* Host-side fault injection for tests (no counterpart in the paper): cap the
 * device bytes any context created afterwards may allocate (0 = no cap);
 * pf_register_init then fails with PF_ENOMEM, releasing what it allocated.
 * Process-wide.  Errors: PF_EINVAL (bytes < 0). */
int pf_debug_alloc_limit(int64_t bytes);

/* The measurement's tile shape (no counterpart in the paper): target rows per
 * work item (one warp's rows) and consecutive work items per warp (the
 * autotuned parameter). */
int pf_tile_shape(pf_ctx *ctx, int32_t *rows_per_item, int32_t *items_per_warp);

/* Philox4x32-10 (Salmon et al., SC'11; the generator of every random draw of
 * the Fig. 1 cycle) of (ctr, key) computed on the device, for tests of the
 * generator against its published known answers. */
int pf_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Timing of the measurement kernel (the hot loop; no counterpart in the
 * paper) inside the iteration graph:
 * pf_profile_begin arms CUDA events for the next `capacity` iterations run by
 * pf_step (0 disarms); pf_profile_end synchronises and returns the summed
 * device time of those measurement launches (ms) and how many were timed. */
int pf_profile_begin(pf_ctx *ctx, int32_t capacity);
int pf_profile_end(pf_ctx *ctx, double *total_ms, int32_t *n_timed);

/* ---- learned proposal network: tensor-core contractions (test exports) ----
 *
 * The proposal network (a 3-D CNN that predicts the mean and log-variance of
 * the 6-DOF pose to seed the particle cloud; the learned approach Sec. 6 names
 * as future work) is built from strided 3-D convolutions: kernel 4^3, stride 2,
 * padding 1, 32 output channels.  Tensors are bf16 (uint16_t bit patterns) in
 * NDHWC layout, x fastest: element (b, z, y, x, c) of a D^3 x C volume sits at
 * (((b*D + z)*D + y)*D + x)*C + c.  Weights are [32 co][64 taps][Cin], tap =
 * (kz*4 + ky)*4 + kx.  The contractions run on the tcgen05 tensor cores with
 * fp32 accumulation.  All pointers are device pointers; calls are asynchronous
 * on `stream` (a cudaStream_t) and allocate nothing.
 * Errors: PF_EINVAL (NULL, D odd or outside [2, 512], Cin not one of 2, 8, 16,
 * 32, 64, 128, 256, sizes beyond int32 indexing), PF_ECUDA. */

/* C[M][32] (fp32) = A[M][K] B[32][K]^T, A and B row-major bf16, K % 8 == 0. */
int pf_nn_gemm_bf16(const uint16_t *A, const uint16_t *B, float *C, int32_t M, int32_t K, void *stream);

/* y[b, o, co] = relu(bias[co] + sum_{tap, ci} x[b, 2o + k - 1, ci] w[co][tap][ci])
 * (per axis, k the tap's offset 0..3; taps outside the input read 0).
 * x: [batch][D^3][Cin]; y: [batch][(D/2)^3][32] bf16 (rounded to nearest). */
int pf_nn_conv3d_forward(const uint16_t *x, int32_t batch, int32_t D, int32_t Cin, const uint16_t *w,
                         const float *bias, uint16_t *y, void *stream);

/* Gradient with respect to the input of a 32-channel layer (Cin = 32):
 * dx[b, i, ci] = [act[b, i, ci] > 0] * sum over (tap, co) with o = (i + 1 - k)/2
 * integral and inside of dy[b, o, co] w[co][tap][ci]  (per axis).
 * dy: [batch][(D/2)^3][32]; w_t: the weights transposed to [ci][tap][co];
 * act: [batch][D^3][32] ReLU output of the layer below (mask), or NULL for no
 * mask; dx: [batch][D^3][32] bf16. */
int pf_nn_conv3d_backward_data(const uint16_t *dy, int32_t batch, int32_t D, const uint16_t *w_t,
                               const uint16_t *act, uint16_t *dx, void *stream);

/* Gradient with respect to the weights: dw[co][tap][ci] += sum_{b, o}
 * x[b, 2o + k - 1, ci] dy[b, o, co] (fp32 accumulation into dw; partial sums
 * of K-slices are added atomically, so the summation order varies). */
int pf_nn_conv3d_backward_weights(const uint16_t *x, int32_t batch, int32_t D, int32_t Cin, const uint16_t *dy,
                                  float *dw, void *stream);

/* *gave_up = 1 when a tensor-core kernel's bounded wait on an mbarrier ran
 * out since the last clear (its tile was then not written); clear != 0
 * resets the flag.  Synchronous.  The synchronous proposal calls
 * (pf_proposal_train with loss_out, pf_proposal_predict,
 * pf_proposal_backward) check the same flag when they finish: if it is set
 * they return PF_ETIMEOUT and clear it. */
int pf_nn_status(int32_t clear, int32_t *gave_up);

/* Failure-detection self-test (no counterpart in the paper): launches one
 * thread that waits on an mbarrier nothing arrives on, with the same kind of
 * bounded wait the tensor-core kernels use (2^16 polls); when the wait runs
 * out it sets the flag pf_nn_status reports.  Nothing faults or hangs: the
 * kernel returns and the context stays usable.  Asynchronous on `stream`. */
int pf_nn_wait_selftest(void *stream);

/* ---- learned proposal network ----
 *
 * A 3-D CNN that predicts, from a source/target pair, the mean and the
 * log-variance of the 6-DOF pose; the mean and spread seed and shrink the
 * particle cloud (pf_seed_gaussian).  The paper names a learned approach as
 * future work (Sec. 6); this network is not in the paper.  Architecture:
 * input 64^3 x 2 (source and target box-averaged, /64, onto one 64^3 grid over
 * the source's box: the target sits at its own origin), four convolutions
 * 4^3 / stride 2 / padding 1 / 32 channels with ReLU (bf16 activations, fp32
 * accumulation on the tcgen05 tensor cores), then fully connected 2048 -> 128
 * (ReLU) -> 12 in fp32: mean (6) and log-variance (6) in units of the
 * training limits.  464,652 fp32 parameters, Adam.
 * Training data: synthetic echo-like pairs generated on the GPU (speckled
 * left-ventricle shell, per-view gain, random pose within the limits, target
 * field of view slid along x for 35-60 % overlap), labels = generating pose.
 * A proposal object belongs to one stream and is not thread-safe. */
typedef struct pf_proposal pf_proposal;

/* Create a network with parameters drawn from Philox(seed) (uniform, fan-in
 * scaled) for batches of up to max_batch (1..256) pairs.  Device memory:
 * about max_batch * 2.5 MB plus 8 MB.  Errors: PF_EINVAL, PF_ENOMEM, PF_ECUDA. */
int pf_proposal_create(pf_proposal **out, int32_t max_batch, uint64_t seed, void *stream);
int pf_proposal_destroy(pf_proposal *p);

/* Run n_steps Adam steps (learning rate lr) on fresh synthetic batches of
 * `batch` pairs of vol_dims volumes with poses uniform in +-rot_limit (rad,
 * every axis) / +-trans_limit (voxels); batch b of step t is drawn from
 * Philox(data_seed, b, t).  Each step is one CUDA-graph launch.  loss_out
 * (host, n_steps floats, may be NULL) receives the mean Gaussian negative
 * log-likelihood of each step.  The limits are the units of the outputs and
 * must stay the same across calls.  Synchronous when loss_out is given.
 * Errors: PF_EINVAL (sizes, lr outside (0, 1), limits), PF_ENOMEM, PF_ECUDA. */
int pf_proposal_train(pf_proposal *p, int32_t n_steps, int32_t batch, float lr, uint64_t data_seed,
                      const int32_t vol_dims[3], float rot_limit, float trans_limit, float *loss_out);

/* Predict the pose of a pair: mean_out = mean * limits, std_out =
 * exp(log-variance / 2) * limits, per DOF [rx ry rz tx ty tz] (radians,
 * world units).  Volumes as for pf_register_init (host or device).
 * Synchronous.  Errors: PF_EINVAL, PF_ESTATE (not trained), PF_ECUDA. */
int pf_proposal_predict(pf_proposal *p, const pf_volume *src, const pf_volume *tgt, float mean_out[6],
                        float std_out[6]);

/* Checkpoint and inspection (host buffers of *n_params floats, any may be
 * NULL): theta_in replaces the parameters, then theta_out / grad_out receive
 * the parameters and the gradient of the last backward pass.  Synchronous. */
int pf_proposal_params(pf_proposal *p, float *theta_out, float *grad_out, const float *theta_in,
                       int64_t *n_params);

/* Test exports (device buffers, asynchronous on the stream):
 *   forward:  x [batch][64^3][2] bf16 -> out [batch][12], hidden [batch][128] (may be NULL);
 *   backward: gradient of the mean loss for labels y [batch][6] (pose / limits)
 *             after a forward of the same batch; *loss_out (host) = the loss; synchronous;
 *   synth:    a synthetic batch (x, y) of step `step` as pf_proposal_train draws it;
 *   input:    the network input [64^3][2] of one pair, as pf_proposal_predict builds it. */
int pf_proposal_forward(pf_proposal *p, const uint16_t *x, int32_t batch, float *out, float *hidden);
int pf_proposal_backward(pf_proposal *p, const float *y, int32_t batch, float *loss_out);
int pf_proposal_synth(pf_proposal *p, int32_t batch, uint64_t seed, int32_t step, const int32_t vol_dims[3],
                      float rot_limit, float trans_limit, uint16_t *x_out, float *y_out);
int pf_proposal_input(pf_proposal *p, const pf_volume *src, const pf_volume *tgt, uint16_t *x_out);

/* Test export: copy one of the network's device tensors of the last forward /
 * backward pass to host memory (host_out), for layer-by-layer checks:
 *   which 0..3   conv layer l's output after ReLU, a_l, bf16 bits [batch][(32 >> l)^3][32];
 *   which 4..7   the gradient with respect to conv layer (which - 4)'s
 *                pre-activation, d_l, bf16 bits, same shape;
 *   which 8 / 10 the hidden layer's output h / the gradient dh with respect
 *                to its pre-activation, fp32 [batch][128];
 *   which 9 / 11 the output (mean, log-variance) / the loss gradient with
 *                respect to it, fp32 [batch][12].
 * Synchronous.  Errors: PF_EINVAL (NULL, which, batch outside [1, max_batch]), PF_ECUDA. */
int pf_proposal_tensor(pf_proposal *p, int32_t which, int32_t batch, void *host_out);

/* Number of this library's kernels launched in this process so far (each
 * graph replay counts its kernels). */
uint64_t pf_kernel_launches(void);

/* Read-bandwidth probe (no counterpart in the paper; the L2 roof the
 * measurement's gathers are reported against): launches one kernel that reads
 * the device buffer buf (16-byte aligned, `bytes` a multiple of 16) `reps`
 * times with 16-byte loads that bypass L1, so every byte comes from L2 when
 * the buffer fits there (from HBM otherwise).  The caller times it with CUDA
 * events on `stream`; bytes * reps were read.  sink: one device uint64 the
 * kernel may write (it keeps the loads).  Asynchronous.
 * Errors: PF_EINVAL (NULL, size, alignment, reps outside [1, 100000]), PF_ECUDA. */
int pf_probe_read(const void *buf, int64_t bytes, int32_t reps, uint64_t *sink, void *stream);

/* Bounds checks of the debug build (no counterpart in the paper).  The
 * library built with -DPF_DEBUG=1 (libpfreg_debug.so) checks every gather
 * index of the measurement and warp kernels against its buffer before the
 * load; an index outside is counted, the first one is kept and the load is
 * skipped (the value reads 0) -- nothing traps, the context stays usable.
 * Synchronises the device, then *checks_on = 1 in the debug build (0 in the
 * release build, where *hits is always 0), *hits = out-of-bounds indices seen
 * since the last clear, *first_bad = the first of them (an element index of
 * the buffer).  clear != 0 resets the counters.  Errors: PF_EINVAL (NULL),
 * PF_ECUDA. */
int pf_debug_bounds(int32_t clear, int32_t *checks_on, uint64_t *hits, int64_t *first_bad);

/* Number of device allocations (cudaMalloc / cudaMallocAsync calls that
 * succeeded) this library has made in this process so far; a test hook that
 * shows which calls allocate (no counterpart in the paper). */
uint64_t pf_debug_device_allocs(void);

/* The calling thread's last error message ("" if none). */
const char *pf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PFREG_H */
