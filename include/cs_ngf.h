/*
 * cs_ngf.h -- C ABI of the GB300 all-shift NGF similarity library
 *             (hot path of Cross-Sim-NGF global rigid alignment).
 *
 * What it computes (Cross-Sim-NGF, Ofverstedt, Lindblad, Sladoje):
 *   n(x; V)     = grad V / sqrt(|grad V|^2 + eps^2)                  Eq. 1
 *   s_NGF(x)    = <n(x; A), n(x; B)>^2                               Eq. 2
 *   CSNGF(chi)  = sum_x M_A(x) M_B(x+chi) s_NGF(x; A(x), B(x+chi)) / N(chi),
 *   N(chi)      = (M_A star M_B)(chi)                                Eq. 4-5
 * evaluated for every integer shift chi at once through six weighted channel
 * correlations and one mask correlation in the frequency domain, summed
 * before the inverse transform (Eq. 6-8, Section 3.1).  For each candidate
 * rotation the floating volume is resampled, B_hat = B o T_theta, with
 * trilinear interpolation, shifts whose overlap is below gamma are excluded,
 * and the best shift is argmax_chi CSNGF (Section 3.2); the alignment is the
 * maximum over rotations (Fig. 1).
 *
 * Conventions (the paper leaves these open; the library fixes them):
 *   - Volumes are [z][y][x] with x contiguous; dims[] = {nz, ny, nx}, each in
 *     [2, 256].  B has the same dims as A.  The cap comes from the longest
 *     FFT length built, 512 >= 2n - 1 (a rotation whose admitted shifts span
 *     the whole range needs the full linear length).  Volumes up to 512 per
 *     axis would need 1024-point transforms, which are not built (their fixed
 *     spectra take about 30 GB, each rotation's fields about 15 GB); at 1024
 *     per axis the 2048-point fixed spectra alone (about 240 GB) leave no room
 *     for a rotation in HBM.
 *   - Vectors are (x, y, z).  Rotation centre c = (n - 1) / 2 per axis and
 *     B_hat(x) = B(R(q)(x - c) + c), R the Hamilton matrix of the unit
 *     quaternion q = (w, x, y, z), built in FP64 on the host with entries
 *     within 1e-9 of -1, 0, 1 snapped, then rounded to FP32.  Quaternions
 *     are therefore HOST float64 arrays, not device floats: the matrix is
 *     formed once per rotation on the host and uploaded with the batch.
 *   - The rotated mask is [trilinear M_B >= 0.5] at sample points inside
 *     [0, n-1]^3 (1e-4 slack); outside, B_hat = 0 and the mask is 0.
 *   - Gradient: central differences, unit spacing, indices clamped at faces.
 *   - Shift sign: C(chi) = sum_x a(x) b(x + chi); shifts are reported as
 *     (chi_z, chi_y, chi_x) in [-(n-1), n-1].
 *   - A shift is valid iff N(chi) >= max(1, ceil(gamma * min(sum M_A,
 *     sum M_hat))), the product taken in FP64 from the FP32 gamma given.
 *     Masks are 0/1 bytes (nonzero counts as 1).
 *   - Ties: the larger score wins; equal scores go to the smallest
 *     (chi_z, chi_y, chi_x), then to the smallest rotation index.
 *   - FFT lengths: per axis the smallest of {16, 32, 40, 64, 80, 100, 128,
 *     160, 192, 200, 216, 256, 320, 360, 400, 512} that is >= 2n - 1 (full linear
 *     correlation), unless set.  With bound-limited padding (the default,
 *     cs_ngf_pad_mode) a call may use shorter lengths; the results are the
 *     same (see cs_ngf_pad_mode).
 *
 * Memory and streams: array arguments are DEVICE pointers owned by the
 * caller unless a function says "host".  Work is enqueued on `stream` (a
 * cudaStream_t, NULL = legacy default stream); the caller keeps the inputs
 * alive until that work completes.  A handle owns all of its device memory
 * (fixed spectra and per-batch workspace) and is used by one host thread at
 * a time: a call that finds another thread inside a call on the same handle
 * returns CS_NGF_EBUSY at once, without touching the handle.  Calls on one
 * handle may use different streams: each call's work waits for the previous
 * call's (an event recorded on the previous call's stream), so they never
 * overlap on the handle's buffers.  No function aborts the process: each
 * returns a status.
 */
#ifndef CS_NGF_H
#define CS_NGF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cs_ngf_fixed cs_ngf_fixed; /* opaque handle */

typedef enum {
  CS_NGF_OK = 0,
  CS_NGF_EINVAL = 1,      /* bad argument (null pointer, size, eps, gamma, quaternion) */
  CS_NGF_ENOMEM = 2,      /* device or host allocation failed */
  CS_NGF_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  CS_NGF_ENOVALID = 4,    /* no rotation had any valid shift */
  CS_NGF_EUNSUPPORTED = 5, /* FFT length or size not supported */
  CS_NGF_ECANCELED = 6,    /* a served job was cancelled */
  CS_NGF_ETIMEOUT = 7,     /* a wait ended before the job finished */
  CS_NGF_EBUSY = 8         /* another host thread is inside a call on this handle */
} cs_ngf_status;

typedef enum {
  CS_NGF_SQUARED = 0,   /* s_NGF = <n_A, n_B>^2 (Eq. 2), the paper's CSNGF */
  CS_NGF_UNSQUARED = 1  /* s_US-NGF = <n_A, n_B> (Eq. 3), the USNGF method of Section 5.1 */
} cs_ngf_measure;

typedef enum {
  CS_NGF_FP32 = 0,  /* all intermediates FP32 */
  CS_NGF_BF16 = 1,  /* NGF channel intermediates of the forward x and y passes stored as
                       BF16 (FP32 arithmetic); the mask / overlap count path stays FP32 */
  CS_NGF_FP16 = 2   /* the same intermediates stored as FP16 (3 more mantissa bits than
                       BF16, range to 65504): each channel field is scaled by a power of
                       two chosen from its magnitude bound (at most 1 per voxel, times the
                       voxels summed by each transform) to stay below 2^15; the scale is
                       exact and undone on load */
} cs_ngf_precision;

/* FFT lengths per call.  A circular correlation of length P holds at slot
 * chi mod P the sum of the linear correlation over chi, chi - P, chi + P, ...
 * (Eq. 7-8 evaluated with the DFT).  FULL uses P >= 2n - 1 per axis, so every
 * shift in [-(n-1), n-1] has a slot of its own ("a suitable zero padding",
 * Section 3.2).  BOUND uses that a shift can only be valid where the overlap
 * bound of the mask slab counts reaches the gamma threshold (Section 3.2):
 * N(chi) <= sum_i min(a_i, b_{i + chi}) along each axis, a the slab counts of
 * M_A and b those of the rotated mask.  Each scoring call first counts the
 * rotated masks of all its rotations, takes the range [lo, hi] of shifts the
 * bound admits for each of them, and gives each rotation per axis the
 * shortest supported length P >= n + max(-lo, hi) over its own range.
 * Rotations needing the same lengths are scored together (small groups join
 * a larger one, with lengths raised to cover both), and the results come
 * back in the caller's order.  Then for every admitted shift chi the other
 * shifts chi + kP, k != 0, fall outside [-(n-1), n-1] where the linear
 * correlation lives, so its slot holds exactly its own value; shifts outside
 * the range are invalid and reported as such, as with FULL.  Scores agree
 * with FULL up to FP32 rounding.  The call synchronises its stream once to
 * read the ranges, and once more for each further set of lengths, whose
 * fixed spectra it recomputes (about the cost of one rotation each). */
typedef enum {
  CS_NGF_PAD_FULL = 0,  /* P >= 2n - 1 on every call */
  CS_NGF_PAD_BOUND = 1  /* per call, the shortest length the shift bound allows (default) */
} cs_ngf_pad_mode;

typedef struct {
  float eps;         /* Eq. 1 regulariser; the paper uses 1e-5 */
  float gamma;       /* minimum overlap fraction in (0, 1]; the paper uses 0.5 */
  int32_t pad[3];    /* FFT lengths (z, y, x); 0 = automatic */
  int32_t batch;     /* rotations per launch group; 0 = automatic (memory-sized, at
                        most 32); a value above 65535 / (fields x nz) is lowered to
                        that (4 fields for the squared measure, 3 unsquared);
                        an odd value above 1 is rounded down to even, since the
                        masks of rotations 2k and 2k+1 share one transform.
                        Results are bit-identical for every even batch; with
                        batch 1 each mask is transformed alone, which can change
                        scores in the last bit */
  int32_t measure;   /* cs_ngf_measure; default CS_NGF_SQUARED */
  int32_t precision; /* cs_ngf_precision; default CS_NGF_FP32 */
  int32_t pad_mode;  /* cs_ngf_pad_mode; cs_ngf_default_config sets CS_NGF_PAD_BOUND.  The
                        lengths from pad (or automatic) are then the largest a call uses */
  int32_t autotune;  /* 0 (default): every FFT pass uses its built-in radix split.
                        1: the first launch group at a new set of FFT lengths times each
                        pass with each split its length offers (e.g. 200 = 10 x 20 or
                        8 x 25) and keeps the faster for the rest of the process
                        (cs_ngf_tuning lists the choices).  Every split computes the same
                        transform; results differ from the default only by FP32 rounding,
                        and are reproducible within a process, not across processes
                        whose timings choose differently.
                        2: every pass uses the alternative split wherever its length has
                        one, without timing (for tests and comparisons). */
  int32_t tensor_cores; /* 1 (cs_ngf_default_config): in the BF16 and FP16 forms the z pass
                        runs the forward z-axis DFT of the NGF channel fields on the tensor
                        cores (BF16 / FP16 operands, FP32 accumulation; Eq. 7-8 unchanged)
                        wherever the z length is at most 216 (16 ... 216) and the block's
                        operands fit in shared memory (at 200 and 216: z extent at most
                        160); the
                        mask field and every inverse transform stay FP32 on the CUDA cores.
                        The handle then holds one more per-rotation buffer (the spectral sum
                        X, (Px/2+1) Py Pz complex values).  0: the CUDA-core FFT for every
                        field.  Ignored in the FP32 form.  A tensor-core pass that waits more
                        than 2 s for its own MMAs stops; the next synchronous call
                        (cs_ngf_align, cs_ngf_score_rotations_host) then returns ECUDA. */
} cs_ngf_config;

typedef struct {
  int32_t dims[3];              /* nz, ny, nx */
  int32_t pad[3];               /* FFT lengths in use (those of the last call) */
  int32_t batch;                /* rotations per launch group */
  int64_t sum_mask_a;           /* sum of M_A */
  int64_t fixed_bytes;          /* device bytes of the fixed spectra */
  int64_t workspace_bytes;      /* device bytes of the per-batch workspace */
  int32_t max_pad[3];           /* largest FFT lengths (buffers are sized for them) */
  int32_t pad_mode;             /* cs_ngf_pad_mode */
  int32_t length_sets;          /* sets of FFT lengths the last scoring call used */
  int32_t reserved_;
} cs_ngf_info;

/* Fill *cfg with the paper's settings (eps 1e-5, gamma 0.5, automatic pad and
 * batch), bound-limited padding and the tensor-core z pass of the
 * reduced-precision forms. */
void cs_ngf_default_config(cs_ngf_config* cfg);

/* Section 3.1, Eq. 1, 6-8, A side: the NGF of the fixed volume A, its six
 * channels times M_A and M_A itself, their forward 3D FFTs, conjugated and
 * weighted (1,1,1,2,2,2), stored on the device in the new handle.
 *   A      device float32 [nz][ny][nx]
 *   maskA  device uint8   [nz][ny][nx]
 *   dims   host {nz, ny, nx}
 *   cfg    host, NULL = defaults
 *   out    host; receives the handle (NULL on failure)
 * Synchronises `stream` before returning (the handle's sum of M_A is read
 * back).  Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA. */
cs_ngf_status cs_ngf_prepare_fixed(const float* A, const uint8_t* maskA, const int32_t dims[3],
                                   const cs_ngf_config* cfg, void* stream, cs_ngf_fixed** out);

/* Section 3.2 + Eq. 5: for each of R rotations, resample B, compute CSNGF for
 * every valid shift and return its maximum and location.
 *   B, maskB    device, dims of the handle
 *   quats       host float64 [R][4] (w, x, y, z); normalised here; a
 *               quaternion whose norm differs from 1 by more than 1e-3 is EINVAL
 *   best_score  device float32 [R]; -inf where a rotation has no valid shift
 *   best_shift  device int32 [R][3] (chi_z, chi_y, chi_x); 0 where no valid shift
 * Asynchronous on `stream` except for the small host-to-device upload of the
 * rotation matrices, which is staged through the handle, and, with
 * bound-limited padding, one wait for the shift range of the call (the call
 * returns once the scoring work is enqueued).  Errors: EINVAL, EBUSY, ECUDA. */
cs_ngf_status cs_ngf_score_rotations(cs_ngf_fixed* f, const float* B, const uint8_t* maskB,
                                     const double* quats, int32_t R, float* best_score,
                                     int32_t* best_shift, void* stream);

/* cs_ngf_score_rotations with HOST buffers: copies B and maskB (host,
 * [nz][ny][nx]) to the handle's device staging area, scores, and copies the
 * results back to host best_score [R] / best_shift [R][3].  Synchronous.
 * Errors: EINVAL, EBUSY, ENOMEM, ECUDA. */
cs_ngf_status cs_ngf_score_rotations_host(cs_ngf_fixed* f, const float* B, const uint8_t* maskB,
                                          const double* quats, int32_t R, float* best_score,
                                          int32_t* best_shift, void* stream);

/* Fig. 1: the maximum of s_ANGF over all rotations and shifts.
 *   score, rot_index, shift: HOST outputs (score -inf, index -1 if nothing
 *   is valid, with status ENOVALID).  Synchronous.  B, maskB device.
 * Errors: EINVAL, EBUSY, ENOVALID, ENOMEM, ECUDA. */
cs_ngf_status cs_ngf_align(cs_ngf_fixed* f, const float* B, const uint8_t* maskB,
                           const double* quats, int32_t R, float* score, int32_t* rot_index,
                           int32_t shift[3], void* stream);

/* Eq. 5 for one rotation, the full map: map is device float32
 * [2nz-1][2ny-1][2nx-1] indexed by chi + n - 1, holding CSNGF(chi) or -inf
 * where chi is not valid.  quat: host float64 [4].  Errors: EINVAL, EBUSY, ECUDA. */
cs_ngf_status cs_ngf_score_map(cs_ngf_fixed* f, const float* B, const uint8_t* maskB,
                               const double* quat, float* map, void* stream);

/* Section 3.2 resample alone (one rotation): B_hat device float32 and M_hat
 * device uint8, [nz][ny][nx].  quat: host float64 [4].  Errors: EINVAL, EBUSY, ECUDA. */
cs_ngf_status cs_ngf_resample(cs_ngf_fixed* f, const float* B, const uint8_t* maskB,
                              const double* quat, float* Bhat, uint8_t* Mhat, void* stream);

/* Recompute the fixed-volume spectra of an existing handle from a new A and
 * maskA of the same dims (no reallocation).  Synchronises `stream`.
 * Errors: EINVAL, EBUSY, ECUDA. */
cs_ngf_status cs_ngf_update_fixed(cs_ngf_fixed* f, const float* A, const uint8_t* maskA,
                                  void* stream);

/* Per-stage timing.  While profiling is on, every kernel launch of the handle
 * is bracketed by CUDA events recorded on its stream.  cs_ngf_stage_times
 * waits for them and returns, per stage, the summed milliseconds and the
 * number of launches since the previous call (host arrays of
 * CS_NGF_NSTAGES), then forgets them.  Errors: EINVAL, EBUSY, ECUDA.  Stages: */
#define CS_NGF_NSTAGES 8
enum {
  CS_NGF_STAGE_RESAMPLE = 0, /* Section 3.2 trilinear resample + rotated mask */
  CS_NGF_STAGE_FWD_X = 1,    /* Eq. 1, 6: NGF channels + x-axis FFT */
  CS_NGF_STAGE_FWD_Y = 2,    /* y-axis FFT */
  CS_NGF_STAGE_ZMAC = 3,     /* z-axis FFT, Eq. 7-8 spectral sum, z-axis inverse */
  CS_NGF_STAGE_INV_Y = 4,    /* y-axis inverse FFT */
  CS_NGF_STAGE_INV_X = 5,    /* x-axis inverse FFT, Eq. 5 normalisation, argmax */
  CS_NGF_STAGE_FIXED = 6,    /* fixed-volume spectra (prepare / update) */
  CS_NGF_STAGE_OTHER = 7     /* thresholds, result decoding */
};
cs_ngf_status cs_ngf_set_profiling(cs_ngf_fixed* f, int32_t on);
cs_ngf_status cs_ngf_stage_times(cs_ngf_fixed* f, double* ms, int64_t* launches);

/* Number of kernel launches this library has made in the process. */
int64_t cs_ngf_launch_count(void);

/* ---------------------------------------------------------------------------
 * Allocation-free scoring for small volumes.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc.  Examples
 * are code running inside another framework's memory pool or allocator hooks,
 * real-time loops where an allocation may block or fail at the worst moment,
 * and processes held to a fixed device-memory budget.
 *
 * It computes what cs_ngf_prepare_fixed + cs_ngf_score_rotations compute for
 * the same inputs, using the same kernels, one rotation at a time.  It
 * allocates nothing: no cudaMalloc, no cudaFree and no allocating library
 * routine.  All scratch memory is a single file-scope device array of
 * CS_NGF_NOALLOC_SCRATCH_BYTES bytes (about 13.9 MiB).  Every GPU that loads
 * this library holds that array until the process exits.
 *   A, maskA, B, maskB  device, [nz][ny][nx] float32 / uint8
 *   dims                host {nz, ny, nx}, each in [2, CS_NGF_NOALLOC_MAX_DIM];
 *                       larger sizes are rejected with EINVAL and a message
 *   eps, gamma          as in cs_ngf_config
 *   quats               host float64 [R][4] (w, x, y, z), read during the call
 *   best_score          device float32 [R]
 *   best_shift          device int32 [R][3]
 * Every array pointer must be device (or managed) memory of the CURRENT
 * device, which runs the work with its own copy of the scratch array; a host
 * pointer or one on another device is rejected with EINVAL.  The caller
 * guarantees the sizes: the library reads nz*ny*nx elements of each volume
 * and writes R scores and R shifts.
 * Work is enqueued on `stream` and the call returns without waiting for it.
 * The first call on a device does a set-up step with that device current: it
 * looks up the device address of the scratch array.  Make that first call
 * before any stream capture.
 * Every call uses the same scratch array, which keeps the previous call's
 * contents.  What must start at zero is cleared on the stream at the start of
 * each call.  Calls whose GPU work overlaps (several host threads, or several
 * streams without ordering between them) race on the scratch array and give
 * wrong results: serialise them.
 * Errors: EINVAL, ECUDA (detail in cs_ngf_last_error()). */
#define CS_NGF_NOALLOC_MAX_DIM 32
#define CS_NGF_NOALLOC_SCRATCH_BYTES 14583552
cs_ngf_status cs_ngf_score_rotations_noalloc(const float* A, const uint8_t* maskA, const float* B,
                                             const uint8_t* maskB, const int32_t dims[3],
                                             float eps, float gamma, const double* quats,
                                             int32_t R, float* best_score, int32_t* best_shift,
                                             void* stream);

/* ---------------------------------------------------------------------------
 * Serving: a continuous-batching request loop for alignment jobs of mixed
 * sizes (the scoring of Section 3.2 for each job; the paper runs one job at a
 * time).  Jobs arrive at any time.  A worker thread admits them (in arrival
 * order, or shortest expected work first) while their device footprint fits
 * the memory budget and an active slot is free.  Device resources are pooled by volume shape and reused without
 * reallocation.  The fixed-volume spectra of each active job stay resident.
 * The worker feeds each job's rotations one launch group at a time on the
 * job's own stream (at most max_inflight groups per job, round-robin over the
 * active jobs), so work of different jobs overlaps on the GPU.  Each job's
 * results equal those of cs_ngf_score_rotations on the same inputs and batch.
 * All inputs of cs_ngf_server_submit are HOST arrays, copied during the call. */
typedef struct cs_ngf_server cs_ngf_server;

/* Admission order when an active slot is free.  ARRIVAL admits pending jobs
 * in submission order.  SHORTEST admits the pending job with the smallest
 * estimated work minus the time it has waited (estimated work: rotations x
 * padded FFT voxels x 2.5e-8 ms, the per-rotation cost measured on one
 * GB300), so short jobs overtake long ones and a long job's priority grows
 * while it waits.  Under either order, when the chosen job does not fit the
 * memory budget no later job is admitted before it. */
enum { CS_NGF_SERVE_ARRIVAL = 0, CS_NGF_SERVE_SHORTEST = 1 };

typedef struct {
  int64_t memory_budget_bytes;      /* device bytes for job resources; 0 = 80 % of free memory */
  int32_t max_active_jobs;          /* jobs on the GPU at once (default 4) */
  int32_t max_inflight;             /* launch groups in flight per job (default 2) */
  int32_t batch;                    /* rotations per launch group when a job's cfg batch is 0 (default 16) */
  int32_t policy;                   /* admission order: CS_NGF_SERVE_ARRIVAL (default) or
                                       CS_NGF_SERVE_SHORTEST */
  int64_t inject_admission_failure; /* test hook: the job with this id fails admission (ENOMEM); 0 = off */
} cs_ngf_server_config;

typedef struct {
  int32_t status;        /* CS_NGF_OK, ENOVALID, ECANCELED or the error that ended the job */
  int32_t rotations;     /* rotations submitted */
  int32_t scored;        /* rotations scored (less than rotations if cancelled) */
  float score;           /* best score over rotations and shifts (-inf if none) */
  int32_t rot_index;     /* its rotation (-1 if none) */
  int32_t shift[3];      /* its shift (chi_z, chi_y, chi_x) */
  double latency_ms;     /* submit to completion */
  double queue_ms;       /* submit to admission */
} cs_ngf_job_result;

typedef struct {
  int32_t pending, active, slots, reserved_;
  int64_t admitted, completed, bytes_in_use, memory_budget_bytes;
} cs_ngf_server_info;

void cs_ngf_server_default_config(cs_ngf_server_config* cfg);
/* Start a server on the current device.  Errors: EINVAL, ENOMEM, ECUDA. */
cs_ngf_status cs_ngf_server_create(const cs_ngf_server_config* cfg, cs_ngf_server** out);
/* Queue a job (host arrays A, maskA, B, maskB [nz][ny][nx], quats [R][4]);
 * cfg (host, NULL = defaults) sets eps, gamma, pad and batch.  A job whose
 * footprint exceeds the whole budget is refused with ENOMEM. */
cs_ngf_status cs_ngf_server_submit(cs_ngf_server* s, const float* A, const uint8_t* maskA,
                                   const float* B, const uint8_t* maskB, const int32_t dims[3],
                                   const double* quats, int32_t R, const cs_ngf_config* cfg,
                                   int64_t* job_id);
/* Ask a job to stop: a pending job never starts, a running job stops after
 * its launch groups in flight (its result then covers the rotations scored
 * so far: a prefix of the job's rotations, or with bound-limited padding,
 * which scores them grouped by FFT lengths, any subset, the others -inf). */
cs_ngf_status cs_ngf_server_cancel(cs_ngf_server* s, int64_t job_id);
/* Wait up to timeout_s seconds (negative = no limit) for a job; on return OK
 * the job's result is in *res (its own status in res->status) and, if not
 * NULL, its per-rotation results in host best_score [R] / best_shift [R][3]
 * (-inf and (0, 0, 0) for rotations not scored); the job is then forgotten.
 * ETIMEOUT if it did not finish in time. */
cs_ngf_status cs_ngf_server_wait(cs_ngf_server* s, int64_t job_id, double timeout_s,
                                 cs_ngf_job_result* res, float* best_score, int32_t* best_shift);
cs_ngf_status cs_ngf_server_stats(cs_ngf_server* s, cs_ngf_server_info* info);
/* Cancel what is left, stop the worker and free every device resource. */
void cs_ngf_server_destroy(cs_ngf_server* s);

/* ---------------------------------------------------------------------------
 * Global rigid alignment (Section 3.2): rotations by random search around
 * starting points, the shift of each rotation from the all-shift similarity,
 * inside an m-level Gaussian pyramid.  Level k smooths both volumes with a
 * Gaussian of sigma[k] voxels (truncated at 4 sigma, faces clamped), keeps
 * every downsample[k]-th voxel (masks sampled at the same voxels), and scores
 * its starting points plus random_rotations[k] rotations, each a uniformly
 * chosen starting point plus U(-max_step_deg[k], max_step_deg[k]) on each
 * Euler angle (about x, then the resulting y, then the resulting z).  The
 * best starting_points[k+1] become the next level's starting points.
 * Random numbers: SplitMix64 seeded with `seed`; per random rotation one
 * uniform draw picks the starting point, then one per angle (x, y, z).  The paper's
 * schedule (cs_ngf_search_default_config): sigma (5, 3, 2, 1.5), d (4, 2, 2,
 * 1), u (180, 30, 10, 0), a (5000, 3000, 300, 0), p (1, 20, 3, 1), start (0,
 * 0, 0).  Inputs are device arrays of `dims`; the call allocates its level
 * buffers and one handle per level, and synchronises `stream`. */
#define CS_NGF_MAX_LEVELS 8
typedef struct {
  int32_t levels;
  float sigma[CS_NGF_MAX_LEVELS];
  int32_t downsample[CS_NGF_MAX_LEVELS];
  float max_step_deg[CS_NGF_MAX_LEVELS];
  int32_t random_rotations[CS_NGF_MAX_LEVELS];
  int32_t starting_points[CS_NGF_MAX_LEVELS];
  float start_euler_deg[3];
  uint64_t seed;
} cs_ngf_search_config;

typedef struct {
  float score;                          /* best score at the last level */
  float level_best[CS_NGF_MAX_LEVELS];  /* best score found at each level */
  double euler_deg[3];                  /* best rotation (x, y', z'' Euler angles, degrees) */
  double quat[4];                       /* the same rotation as a unit quaternion (w, x, y, z) */
  int32_t shift[3];                     /* best shift (chi_z, chi_y, chi_x) in full-resolution voxels */
  int64_t rotations_scored;             /* rotations scored over all levels */
} cs_ngf_search_result;

void cs_ngf_search_default_config(cs_ngf_search_config* cfg);
cs_ngf_status cs_ngf_global_align(const float* A, const uint8_t* maskA, const float* B,
                                  const uint8_t* maskB, const int32_t dims[3],
                                  const cs_ngf_config* cfg, const cs_ngf_search_config* search,
                                  void* stream, cs_ngf_search_result* out);

/* Sizes and FFT lengths of a handle.  info: host. */
cs_ngf_status cs_ngf_get_info(const cs_ngf_fixed* f, cs_ngf_info* info);

/* The sets of FFT lengths the last scoring call used (bound-limited padding
 * groups rotations by the lengths they need; one set otherwise), in the order
 * they were scored.  Fills up to cap entries of host pads [cap][3] (z, y, x)
 * and counts [cap] (rotations scored with those lengths; either may be NULL)
 * and returns the number of sets (0 for a NULL handle or before any call). */
int32_t cs_ngf_length_sets(const cs_ngf_fixed* f, int32_t cap, int32_t* pads, int32_t* counts);

/* Autotuning choices of this process (cs_ngf_config.autotune), one entry per
 * FFT pass, length, input kind and storage form timed so far. */
typedef struct {
  int32_t pass;        /* 0 x forward, 1 y forward, 2 z forward + spectral sum + z inverse,
                          3 y inverse, 4 x inverse */
  int32_t length;      /* FFT length of the pass's axis */
  int32_t half_input;  /* 1: the input fills at most half the length (pruned first stage) */
  int32_t storage;     /* cs_ngf_precision of the channel fields it reads or writes */
  int32_t variant;     /* the split chosen: 0 built-in, 1 alternative */
  int32_t split[2][2]; /* (N1, N2) of each variant: length = N1 x N2 */
  float ms[2];         /* the best time of each variant on the launch group it was timed on */
} cs_ngf_tuning_entry;
/* Fills up to cap entries of host out (may be NULL) and returns the number of
 * entries.  cs_ngf_tuning_reset forgets them (handles keep the variants they
 * hold until their lengths change). */
int32_t cs_ngf_tuning(int32_t cap, cs_ngf_tuning_entry* out);
void cs_ngf_tuning_reset(void);

/* The length classes bound-limited padding forms, computed on the host
 * alone (what a scoring call does after counting the rotated masks):
 *   dims     {nz, ny, nx}; max_pad the largest lengths (each >= 2n - 1)
 *   cur_pad  the lengths in use (their class is scored first) or NULL
 *   bounds   [R][6] per rotation the admitted shift slots v = chi + n - 1,
 *            {lo_z, hi_z, lo_y, hi_y, lo_x, hi_x} (lo > hi: none on that axis)
 * Each rotation needs per axis the shortest supported length
 * P >= n + max(n - 1 - lo, hi - (n - 1)).  Fills up to cap entries of pads
 * [cap][3] and counts [cap], and order [R] with the rotations in class order
 * (each may be NULL); returns the number of classes, or -1 for bad arguments.
 * No device is touched. */
int32_t cs_ngf_plan_lengths(const int32_t dims[3], const int32_t max_pad[3], const int32_t cur_pad[3],
                            int32_t R, const int32_t* bounds, int32_t cap, int32_t* pads,
                            int32_t* counts, int32_t* order);

/* Free every device allocation of the handle (NULL is a no-op).  The caller
 * makes sure no work that uses the handle is still in flight. */
void cs_ngf_release(cs_ngf_fixed* f);

/* Static description of a status code. */
const char* cs_ngf_status_string(int32_t status);

/* Detail of the last failure on the calling host thread ("" if none). */
const char* cs_ngf_last_error(void);

/* Automatic FFT length for a volume side n (0 if n is unsupported). */
int32_t cs_ngf_auto_pad(int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* CS_NGF_H */
