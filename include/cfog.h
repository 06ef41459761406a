/*
 * cfog.h -- C ABI of the GB300 (sm_103a) CFOG matching library, libcfog.so.
 *
 * The library implements the data-parallel hot path of the matching framework
 * of Ye et al., "Fast and Robust Matching for Multimodal Remote Sensing Image
 * Registration" (arXiv 1808.06194):
 *
 *   image --(cfog_extract)--> CFOG volume D (Sec. III-F, Eq. 2, Fig. 9)
 *   image --(cfog_extract_fhog)--> pixel-wise HOG volume, 36 channels (Sec. III-C)
 *   image --(cfog_detect_cps)--> control points (Sec. IV, block-based Harris)
 *   D_ref, D_sen, CPs --(cfog_match)--> integer + sub-pixel offsets and SSD
 *                                        (Eq. 3-9, Sec. V-B)
 *   CPs, offsets --(cfog_fit_affine)--> least-squares affine model (Sec. IV)
 *   CPs, offsets --(cfog_reject_outliers)--> kept CPs + polynomial model
 *                                        (Sec. IV, iterative outlier rejection)
 *   kept CPs --(cfog_tin_delaunay, host)--> TIN;  sensed image, TIN
 *       --(cfog_tin_rectify)--> sensed image on the reference grid (Sec. IV,
 *                                        piecewise linear rectification)
 *
 * Conventions shared by every entry point:
 *   - Every pointer named *_dev or held in cfog_image / cfog_features /
 *     CP arrays is a DEVICE pointer; structs passed by pointer (params, image
 *     and feature descriptors) live in HOST memory and are read during the
 *     call only.
 *   - The caller owns all buffers.  The library never allocates or frees
 *     caller memory.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream).  Results are valid after the stream
 *     is synchronised.  Host outputs (sizes, plans, out6) are written before
 *     the call returns unless stated otherwise.
 *   - Errors: the return value is a cfog_status.  On a non-OK status the
 *     reason is kept, per host thread, in cfog_last_error().  Invalid
 *     arguments are detected on the host before any launch (CFOG_E_INVAL);
 *     launch failures return CFOG_E_CUDA.  Per-CP problems (a window leaving
 *     the image, a peak on the window edge) do not fail the call: they are
 *     reported in cfog_match_result.status.
 */
#ifndef CFOG_H
#define CFOG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CFOG_API_VERSION 1

typedef enum {
    CFOG_OK = 0,
    CFOG_E_INVAL = 1,        /* bad argument (null pointer, size out of range)  */
    CFOG_E_CUDA = 2,         /* a CUDA launch or API call failed                */
    CFOG_E_NOMEM = 3,        /* caller-provided workspace too small             */
    CFOG_E_TIMEOUT = 4,      /* a bounded device-side wait gave up              */
    CFOG_E_UNSUPPORTED = 5   /* parameter combination not compiled in           */
} cfog_status;

/* Per-CP status in cfog_match_result.status. */
enum {
    CFOG_CP_OK = 0,
    CFOG_CP_OOB = 1,         /* template or search window leaves an image       */
    CFOG_CP_EDGE_PEAK = 2,   /* minimum on the border of the search window:
                                integer offset kept, no sub-pixel refinement    */
    CFOG_CP_FLAT = 3,        /* reserved                                        */
    CFOG_CP_TIMEOUT = 4      /* a bounded wait of the tensor-core path gave up:
                                the result is not valid                         */
};

enum { CFOG_DTYPE_F32 = 0, CFOG_DTYPE_U16 = 1 };
enum { CFOG_PREC_FP32_FFT = 0, CFOG_PREC_BF16_DIRECT = 1 };

/* CFOG parameters (Sec. III-F; defaults of Sec. V-C).
 *   m            number of orientated gradient channels, theta_k = k*pi/m
 *                (compiled for m in {6, 8, 9, 12}; default 9)
 *   sigma        STD of the 2-D Gaussian in x, y (default 0.8)
 *   eps          L2 normalisation guard: D = h / (||h|| + eps) (default 1e-6)
 *   gauss_radius taps t = -R..R of the sampled Gaussian, R in {2, 3, 4}
 *                (default ceil(3 sigma) = 3)
 *   orientation  how the oriented gradient channels are formed (Sec. III-F
 *                gives two schemes):
 *                CFOG_ORIENT_EQ2  (default, the paper's second scheme, Eq. 2):
 *                  g_k = |cos t_k gx + sin t_k gy|
 *                CFOG_ORIENT_BINS (the paper's first scheme, Fig. 7): the
 *                  gradient magnitude sqrt(gx^2 + gy^2) is shared between the
 *                  two bins t_k next to the orientation atan2(gy, gx) folded
 *                  into [0, pi), each with weight 1 - (distance in bin widths);
 *                  bins centred on t_k = k*pi/m, wrapping at pi; compiled for
 *                  gauss_radius 3                                             */
enum { CFOG_ORIENT_EQ2 = 0, CFOG_ORIENT_BINS = 1 };
typedef struct {
    int32_t m;
    float sigma;
    float eps;
    int32_t gauss_radius;
    int32_t orientation;
} cfog_params;

/* A single-channel image in device memory, row-major.
 *   data   device pointer to h rows of `pitch` ELEMENTS (pitch >= w)
 *   dtype  CFOG_DTYPE_F32 (float) or CFOG_DTYPE_U16 (uint16, used as its value) */
typedef struct {
    const void *data;
    int32_t h, w;
    int64_t pitch;
    int32_t dtype;
} cfog_image;

/* A CFOG volume in device memory, planar FP32.
 *   data       channel k, pixel (y, x) at data[k*plane_pitch + y*row_pitch + x]
 *   sqnorm     ||D(y,x)||^2 at sqnorm[y*row_pitch + x] (written by
 *              cfog_extract, read by cfog_match)
 *   row_pitch  in floats, a multiple of 4; plane_pitch in floats, >= h*row_pitch
 * cfog_feature_layout() gives the layout cfog_extract expects.                 */
typedef struct {
    float *data;
    float *sqnorm;
    int32_t m, h, w;
    int64_t row_pitch, plane_pitch;
} cfog_features;

typedef struct {
    int32_t x, y;
} cfog_point;

/* One registration job of a batched match: the CFOG volumes of its reference
 * and sensed images (both with the launch's m).  cfog_match_batched reads an
 * array of these from DEVICE memory. */
typedef struct {
    cfog_features ref;
    cfog_features sen;
} cfog_job;

/* Kernel variants of the FFT matcher (threads per CTA / CTAs per SM / FFT plane
 * bound).  0 lets the library choose. */
enum {
    CFOG_MATCH_VARIANT_AUTO = 0,
    CFOG_MATCH_VARIANT_WIDE = 1,   /* 512 threads, 1 CTA per SM, P_y*P_x <= 16384 */
    CFOG_MATCH_VARIANT_PAIR = 2,   /* 256 threads, 2 CTAs per SM, P_y*P_x <= 9216  */
    CFOG_MATCH_VARIANT_TRIO = 3,   /* 256 threads, 3 CTAs per SM, P_y*P_x <= 7680,
                                      spectrum accumulator in tensor memory         */
    CFOG_MATCH_VARIANT_PAIRT = 4   /* as PAIR, spectrum accumulator in tensor memory
                                      (TRIO and PAIRT: batched path only; cfog_match
                                      uses WIDE)                                    */
};

/* Result of one CP (24 bytes).  dx, dy: total integer offset q + v* from the
 * CP to its match in the sensed image, so that sen(p + (dx, dy)) ~ ref(p)
 * (the paper's D2(x - v) of Eq. 3 with the sign folded into the offset).
 * sub_dx, sub_dy: the offset after sub-pixel refinement.  ssd: S(v*) of Eq. 3. */
typedef struct {
    int32_t dx, dy;
    float sub_dx, sub_dy;
    float ssd;
    int32_t status;
} cfog_match_result;

/* Version of this ABI (CFOG_API_VERSION). */
int32_t cfog_version(void);

/* Reason for the last non-OK status returned on the calling host thread
 * ("" if none).  The string stays valid until the next call on that thread. */
const char *cfog_last_error(void);

/* Fill *p with the paper's defaults (Sec. V-C: m = 9, sigma = 0.8) and the
 * readings eps = 1e-6, gauss_radius = 3, orientation CFOG_ORIENT_EQ2.
 * Returns CFOG_E_INVAL if p is NULL. */
cfog_status cfog_default_params(cfog_params *p);

/* Layout of the CFOG volume of an h x w image: writes the row and plane
 * pitches (floats) and returns the bytes needed for `data`; the sqnorm plane
 * needs h*row_pitch*4 more bytes.  Returns 0 on a bad argument. */
size_t cfog_feature_layout(int32_t h, int32_t w, int32_t m, int64_t *row_pitch,
                           int64_t *plane_pitch);

/* CFOG extraction (Sec. III-F, Eq. 2, Fig. 9), one fused kernel:
 * gx, gy by [-1,0,1] filters (replicate borders); g_k = |cos t_k gx + sin t_k gy|
 * for t_k = k*pi/m (or the binned channels of p->orientation); 2-D Gaussian (sigma, radius R, normalised taps, replicate
 * borders); circular [1,2,1]/4 across k; D = h / (||h||_2 + eps); also the
 * ||D||^2 plane.  img and out must have the same h, w; out->m == p->m.
 * p may be NULL for the defaults.                                             */
cfog_status cfog_extract(const cfog_image *img, const cfog_params *p, const cfog_features *out,
                         void *stream);

/* CFOG of output rows [row0, row1) only, with exactly the values cfog_extract
 * gives for those rows: input rows [row0 - R - 1, row1 + R + 1) (clipped to the
 * image) must hold valid data; borders replicate only at rows 0 and h-1.  For
 * an image streamed into device memory in row bands (the partition strategy of
 * Sec. IV): once a band and the first R+1 rows of the next one are resident,
 * the band's features can be computed.  0 <= row0 <= row1 <= h.               */
cfog_status cfog_extract_rows(const cfog_image *img, const cfog_params *p,
                              const cfog_features *out, int32_t row0, int32_t row1,
                              void *stream);

/* Pixel-wise HOG, the FHOG descriptor of the framework (Sec. III-C): at every
 * pixel, a block centred on it of 2 x 2 cells of cell x cell pixels, the
 * gradient orientation in [0, 180) quantised into 9 bins, each block pixel
 * adding its gradient magnitude to the bins next to its position and
 * orientation by trilinear interpolation, then D = h / (||h||_2 + eps).
 * Conventions: gradients by [-1,0,1] (replicate borders, block pixels outside
 * the image repeat the edge pixel); the two cell centres of an axis at -cell/2
 * and +cell/2 from the pixel, spatial weight 1 - |offset - centre| / cell over
 * block offsets -cell..cell; orientation bins centred on k*pi/9 (the binned
 * scheme of cfog_params.orientation).  out->m must be 36: plane
 * (cy*2 + cx)*9 + k holds cell row cy, cell column cx (0 = the cell at
 * -cell/2) and bin k; the ||D||^2 plane is written too, so the result feeds
 * cfog_match / cfog_match_batched with m = 36.  cell in {4, 8} (HOG's usual
 * cell: 8); eps >= 0.                                                        */
cfog_status cfog_extract_fhog(const cfog_image *img, int32_t cell, float eps,
                              const cfog_features *out, void *stream);

/* Block-based Harris detection (Sec. IV).  The interior box
 * [margin, h-margin) x [margin, w-margin) is cut into grid_y x grid_x cells;
 * in each cell a chip of chip x chip pixels centred on the cell centre
 * (chip <= 0: the whole cell; always clipped to the cell) is searched for
 * the k largest Harris responses det(M) - 0.04 tr(M)^2, M the structure
 * tensor of the [-1,0,1] gradients smoothed by a Gaussian (sigma 1.5,
 * radius 4, replicate borders).  Ties go to the smaller (y, x).
 * out_dev: grid_y*grid_x*k points, cell (j, i) rank s at (j*grid_x + i)*k + s.
 * Limits: 1 <= k <= 8; a chip may not exceed 256 x 256 pixels.              */
cfog_status cfog_detect_cps(const cfog_image *img, int32_t grid_x, int32_t grid_y, int32_t k,
                            int32_t chip, int32_t margin, cfog_point *out_dev, void *stream);

/* SSD template matching of n CPs (Eq. 3-9, Sec. V-B) in one launch, one CTA
 * per CP in CP order (variant CFOG_MATCH_VARIANT_WIDE).
 *   cps_dev[i]      CP position p in the reference image
 *   tmpl_dev[i]     template side N (template pixels p + t,
 *                   t in [-floor(N/2), N-1-floor(N/2)]^2), 8 <= N <= tmpl_max
 *   radius_dev[i]   search radius r: shifts v in [-r, r]^2, 1 <= r <= radius_max
 *   prior_dev       nullable; predicted offset q of the search centre
 *                   (Sec. IV, search region from georeferencing)
 *   tmpl_max        host-side upper bound of tmpl_dev (<= 256)
 *   radius_max      host-side upper bound of radius_dev (<= 32)
 *   precision       CFOG_PREC_FP32_FFT: correlation by FP32 2-D FFTs of the
 *                   (x, y) planes summed over channels -- Eq. 9 at channel
 *                   lag 0 -- with near-ties re-scored directly in FP32.
 *                   CFOG_PREC_BF16_DIRECT: the correlation of Eq. 3 as a
 *                   BF16 GEMM on the tcgen05 tensor cores with FP32
 *                   accumulation (N <= 128, r <= 32); the 8 smallest scores
 *                   and the 3 x 3 neighbourhood of the winner are re-scored
 *                   directly in FP32, so the offsets keep FP32 accuracy; the
 *                   surface output holds the BF16 scores
 *   out_dev         n results
 *   surface_dev     nullable; n * (2*radius_max+1)^2 floats.  CP i's FFT SSD
 *                   surface S(v) is written at
 *                   [i][(dy+radius_max)*(2*radius_max+1) + (dx+radius_max)]
 *                   for |dx|, |dy| <= r; other entries are left untouched.
 * A CP whose N or r lies outside [1, tmpl_max] or [0, radius_max] gets status
 * CFOG_CP_OOB.  The argmin takes the smallest (dy, dx) among equal minima.  Results depend
 * only on each CP's own inputs and (N, r), never on n or on the other CPs.   */
cfog_status cfog_match(const cfog_features *ref, const cfog_features *sen,
                       const cfog_point *cps_dev, int32_t n, const int32_t *tmpl_dev,
                       const int32_t *radius_dev, int32_t tmpl_max, int32_t radius_max,
                       const cfog_point *prior_dev, int32_t precision,
                       cfog_match_result *out_dev, float *surface_dev, void *stream);

/* Workspace (device bytes, 256-byte aligned start) that cfog_match_batched
 * needs for n CPs: a queue counter and the queue order.  0 if n < 0. */
size_t cfog_match_workspace_bytes(int32_t n);

/* Batched SSD matching (same method and per-CP results as cfog_match) of n
 * CPs drawn from n_jobs feature pairs, in ONE persistent launch:
 *   jobs_dev        DEVICE array of n_jobs cfog_job (every volume has m channels)
 *   job_of_cp_dev   nullable; job index of each CP (NULL: all CPs use job 0)
 *   cps_dev .. prior_dev, precision, out_dev: as in cfog_match
 *   m               channel count of every job (host value)
 *   variant         CFOG_MATCH_VARIANT_*; results are identical for a given
 *                   variant whatever the batch holds
 *   workspace_dev   caller-owned device scratch of cfog_match_workspace_bytes(n)
 *                   bytes, 256-byte aligned; overwritten by every call, so calls
 *                   that share it must not overlap on the GPU
 * A first small kernel orders the queue by search-window side N + 2r, largest
 * first; persistent CTAs (as many as fit on the GPU) then take queue slots with
 * one atomic each.  A CP whose job index is out of range, or whose job's
 * volumes do not have m channels, gets status CFOG_CP_OOB.  Returns
 * CFOG_E_NOMEM if the workspace is too small.                               */
cfog_status cfog_match_batched(const cfog_job *jobs_dev, int32_t n_jobs,
                               const int32_t *job_of_cp_dev, const cfog_point *cps_dev,
                               int32_t n, const int32_t *tmpl_dev, const int32_t *radius_dev,
                               int32_t tmpl_max, int32_t radius_max, int32_t m,
                               const cfog_point *prior_dev, int32_t precision, int32_t variant,
                               cfog_match_result *out_dev, void *workspace_dev,
                               size_t workspace_bytes, void *stream);

/* Allocation-free batched matching (the paper has no counterpart: this is a
 * deployment convenience, not part of the method).
 *
 * Some callers cannot allocate device memory: a plugin that runs inside a host
 * application whose own memory pool reserves the GPU (a cudaMalloc from the
 * plugin fails or breaks the pool's accounting), or a latency-critical loop
 * that must not enter the CUDA allocator (cudaMalloc and cudaFree may
 * synchronise the whole device).  Such callers cannot provide the workspace of
 * cfog_match_batched.  This entry point takes the same arguments minus the
 * workspace and computes exactly the same results: its queue scratch is a
 * static device array inside libcfog.so, sized for
 * cfog_match_batched_noalloc_max_cps() = 65536 CPs (256 KiB + 256 B), which
 * every GPU that loads the library holds until the process exits.
 *   - It allocates nothing: no cudaMalloc, no cudaFree, no pool.  The caller
 *     still passes every input and output.
 *   - The first call in a CUDA context looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it under the context's ID; make that
 *     first call before any stream capture.  A device reset or another
 *     context on the same device has a new ID, so its first call looks the
 *     address up again instead of using a stale one.
 *   - Every call, on every stream, shares the one array, which keeps the last
 *     call's contents (the queue counter is reset at the start of each call).
 *     Calls that overlap on the GPU race on it: serialise them (one stream, or
 *     events between streams).
 *   - n above the maximum returns CFOG_E_INVAL with the reason in
 *     cfog_last_error(); split the batch or use cfog_match_batched.          */
int32_t cfog_match_batched_noalloc_max_cps(void);
cfog_status cfog_match_batched_noalloc(const cfog_job *jobs_dev, int32_t n_jobs,
                                       const int32_t *job_of_cp_dev, const cfog_point *cps_dev,
                                       int32_t n, const int32_t *tmpl_dev,
                                       const int32_t *radius_dev, int32_t tmpl_max,
                                       int32_t radius_max, int32_t m, const cfog_point *prior_dev,
                                       int32_t precision, int32_t variant,
                                       cfog_match_result *out_dev, void *stream);

/* Failure-detection test hook of the BF16 tensor-core path (the paper has no
 * counterpart).  Every wait of that kernel on an mbarrier is bounded; when a
 * wait gives up, the CP reports CFOG_CP_TIMEOUT (a commit that is still
 * outstanding also stops the CTA from issuing further MMAs, and its later CPs
 * report CFOG_CP_TIMEOUT).  To test that path without faulting or hanging a
 * GPU, this call makes every later BF16 launch stall CP `cp` (its index in
 * the launch) on a barrier that nothing arrives at, for `wait_cycles` SM
 * cycles, before any MMA of that CP is issued: that CP reports
 * CFOG_CP_TIMEOUT and every other CP is matched as usual.  The same limit
 * then applies to every wait of those launches.  cp = -1 switches the hook
 * off and restores the default limit (about one second).  Host state, read
 * at each launch; 1000 <= wait_cycles <= 2e9.                               */
cfog_status cfog_test_inject_wait_timeout(int32_t cp, int64_t wait_cycles);

/* FP32 fused multiply-add throughput probe (a measurement helper; the paper
 * has no counterpart).  Launches `blocks` CTAs of 256 threads, each running
 * eight independent FMA chains for iters x 16 steps (packed != 0: the same
 * count as four packed f32x2 chains).  The caller times the launch on
 * `stream` (e.g. with CUDA events) and divides *flops (HOST, written before
 * the call returns: the flops the launch performs) by the time to get the
 * FP32 rate that bounds the FFT matcher's arithmetic.  out_dev (DEVICE, one
 * float) is written only in the impossible case that every chain sums to 0.
 * 1 <= blocks <= 2^20, 1 <= iters <= 2^24.                                   */
cfog_status cfog_probe_fp32_fma(int32_t blocks, int32_t iters, int32_t packed, float *out_dev,
                                double *flops, void *stream);

/* The FFT plan the matcher uses for template side N (tmpl), radius r, m
 * channels and a kernel variant, for sizing and roofline accounting (host
 * only, no GPU work).  out8 (HOST) = {nb_y, nb_x, P_y, P_x, b_y, b_x, passes,
 * shared-memory bytes}: the template is cut into nb_y x nb_x blocks of at
 * most b_y x b_x pixels, each correlated with its (b + 2r)-wide window by a
 * P_y x P_x FFT (Eq. 8-9 applied block-wise; the correlation is linear in the
 * template, so block spectra add).  A tuned plan recorded with
 * cfog_match_set_plan is reported in place of the cost model's.  Variant 0
 * reports WIDE.  1 <= N <= 256, 0 <= r <= 32.                               */
cfog_status cfog_plan_info(int32_t tmpl, int32_t radius, int32_t m, int32_t variant,
                           int32_t *out8);

/* ------------------------------------------------------------------------
 * Autotuning of the FFT matcher (the batching pattern: FFT sizes and kernel
 * variants picked by measurement).  Sec. III-G evaluates Eq. 3 through FFT
 * correlation (Eq. 8-9); the FFT size and the template blocking that do it
 * fastest depend on the class (N, r) and on the GPU.  The library keeps two
 * tables that a tuner (the package's autotune module) fills from timings:
 *
 *   - per kernel variant and class (N, r): the plan, named by a code, that a
 *     launch with m channels uses instead of the cost model's choice;
 *   - per launch class (m, tmpl_max, radius_max, precision): the variant that
 *     CFOG_MATCH_VARIANT_AUTO runs.
 *
 * A CP's result still depends only on its inputs, (N, r, m), the variant and
 * these tables, never on its batch.  The plan tables live in device memory
 * and are written on the CURRENT device (a synchronous copy): write them on
 * each device that should use them, and never while a match launch of this
 * library may be running.  Shared-memory sizing covers both the tuned and the
 * cost-model plan of every class, so a device whose table was not written
 * simply runs the cost model's plans.
 * ---------------------------------------------------------------------- */

/* Feasible plans of class (N = tmpl, r = radius, m) in `variant` (1..4),
 * best first by the cost model, distinct plans only.  out9 (HOST, max_out x 9
 * int32) rows: {code, nb_y, nb_x, P_y, P_x, b_y, b_x, passes, shared-memory
 * bytes} (fields 1..8 as in cfog_plan_info); *n_out receives the row count.
 * Host only, no GPU work.                                                   */
cfog_status cfog_plan_candidates(int32_t tmpl, int32_t radius, int32_t m, int32_t variant,
                                 int32_t max_out, int32_t *out9, int32_t *n_out);

/* Record plan `code` (a row of cfog_plan_candidates; -1 clears) for class
 * (N, r) with m channels in `variant` (1..4).  Returns CFOG_E_INVAL for a code
 * that names no feasible plan.                                              */
cfog_status cfog_match_set_plan(int32_t variant, int32_t m, int32_t tmpl, int32_t radius,
                                int32_t code);

/* Record the variant CFOG_MATCH_VARIANT_AUTO runs for batched launches of
 * class (m, tmpl_max, radius_max, precision); variant 0 clears.  Host state
 * only.  Without a record AUTO runs CFOG_MATCH_VARIANT_WIDE.                */
cfog_status cfog_match_set_auto_variant(int32_t m, int32_t tmpl_max, int32_t radius_max,
                                        int32_t precision, int32_t variant);

/* The variant AUTO resolves to for that launch class (1..4).                */
int32_t cfog_match_auto_variant(int32_t m, int32_t tmpl_max, int32_t radius_max,
                                int32_t precision);

/* Forget every tuned plan (on the current device) and every AUTO record.    */
cfog_status cfog_match_clear_tuning(void);

/* Least-squares affine mapping model (Sec. IV) over the CPs whose status is
 * CFOG_CP_OK:  x' = a0 + a1 x + a2 y,  y' = b0 + b1 x + b2 y  with
 * (x', y') = p + (sub_dx, sub_dy).  One kernel reduces the FP64 normal
 * equations into work_dev (caller-owned device scratch of at least
 * CFOG_AFFINE_WORK_DOUBLES doubles, fully overwritten) and solves the 3x3
 * systems by Cholesky in the same kernel; the call then copies the solution
 * to the host and synchronises `stream` (it blocks).  out6 (HOST) = {a0, a1, a2, b0, b1, b2}.  Returns CFOG_E_INVAL
 * when fewer than three independent CPs remain.                              */
#define CFOG_AFFINE_WORK_DOUBLES 16
cfog_status cfog_fit_affine(const cfog_point *cps_dev, const cfog_match_result *res_dev,
                            int32_t n, double *work_dev, double *out6, void *stream);

/* ---------------------------------------------------------------------------
 * Outlier rejection (Sec. IV, the registration system's third step): fit the
 * geometric mapping model to the CPs by least squares, compute the residuals
 * and the RMSE, drop the CP with the largest residual, and repeat until the
 * RMSE is below a threshold.  The paper's system uses the cubic polynomial
 * model (degree 3); degrees 1 and 2 are the first- and second-order models it
 * names as alternatives.
 *
 * Model:  x' = sum_t coef_x[t] phi_t(u, v),  y' = sum_t coef_y[t] phi_t(u, v)
 * with (x', y') = p + (sub_dx, sub_dy), u = (x - cx) / scale,
 * v = (y - cy) / scale, and the monomials of total degree <= degree in the
 * order  1, u, v, u^2, uv, v^2, u^3, u^2 v, u v^2, v^3  (3, 6 or 10 terms).
 * (cx, cy) is the centre of the bounding box of the job's valid CPs and scale
 * its larger half-side (1 if 0).  This change of variables leaves the fitted
 * mapping unchanged (polynomials of degree <= d are closed under it); it only
 * conditions the FP64 normal equations.
 * Residual of a CP: Euclidean distance between (x', y') and the model's
 * prediction; RMSE = sqrt(mean of the squared residuals over the kept CPs).
 * Loop: fit; stop with CFOG_REJECT_OK if RMSE < rmse_threshold; stop with
 * CFOG_REJECT_MIN_KEEP if one more removal would leave fewer than
 * max(min_keep, terms) CPs; else drop the CP with the largest residual (the
 * lowest index among equal residuals) and refit.  A removal after which the
 * normal equations are singular is undone and the loop stops with
 * CFOG_REJECT_SINGULAR; a singular first fit (fewer than `terms` CPs in
 * general position) gives CFOG_REJECT_SINGULAR, rmse = -1, zero coefficients;
 * non-finite residuals (a NaN offset) also stop the loop with it.
 * ------------------------------------------------------------------------- */
enum {
    CFOG_REJECT_OK = 0,          /* final RMSE < rmse_threshold                 */
    CFOG_REJECT_MIN_KEEP = 1,    /* stopped at max(min_keep, terms) kept CPs    */
    CFOG_REJECT_SINGULAR = 2     /* normal equations singular (see above)       */
};

/* Per-job outcome of cfog_reject_outliers (216 bytes, DEVICE memory). */
typedef struct {
    int32_t status;      /* CFOG_REJECT_*                                      */
    int32_t terms;       /* monomials of the model: 3, 6 or 10                 */
    int32_t n_valid;     /* CPs of the job with status CFOG_CP_OK              */
    int32_t n_kept;      /* CPs left after rejection                           */
    int32_t n_removed;   /* n_valid - n_kept                                   */
    int32_t n_fits;      /* least-squares fits performed                       */
    double rmse;         /* RMSE of the final fit over the kept CPs (-1: none) */
    double cx, cy, scale;
    double coef_x[10];   /* first `terms` entries used                         */
    double coef_y[10];
} cfog_poly_model;

/* Device scratch bytes cfog_reject_outliers needs for n_cps = job_start[n_jobs]
 * CP slots and n_jobs jobs. */
size_t cfog_reject_workspace_bytes(int32_t n_cps, int32_t n_jobs);

/* Outlier rejection for n_jobs independent jobs in one launch (one CTA per
 * job).  Job j owns the CPs [job_start[j], job_start[j+1]) of cps_dev and
 * res_dev; job_start is a HOST array of n_jobs + 1 non-decreasing offsets
 * starting at >= 0 (copied into the workspace on `stream`).  Only CPs with
 * status CFOG_CP_OK take part.
 *   degree          1, 2 or 3 (the paper's system: 3)
 *   rmse_threshold  >= 0 pixels (the paper: 1 px in Sec. IV, 3.5 px in its
 *                   comparison runs)
 *   min_keep        >= 0
 *   keep_dev        out, uint8 per CP slot of every job: 1 kept, 0 dropped or
 *                   not valid
 *   order_dev       out, nullable: the first n_removed slots of job j's range
 *                   hold the (global) indices of its dropped CPs in removal order
 *   models_dev      out, n_jobs cfog_poly_model
 *   work_dev        device scratch of work_bytes >= cfog_reject_workspace_bytes
 * FP64 normal equations (updated by removing the dropped CP's terms) and FP64
 * solves; residuals re-evaluated each round as the FP32 change from the first
 * fit's FP64 residuals.  Asynchronous on `stream`.  CFOG_E_INVAL for bad
 * arguments and CFOG_E_NOMEM for a short workspace, both checked on the host
 * before any copy or launch; n_jobs = 0 is a no-op.                          */
cfog_status cfog_reject_outliers(const cfog_point *cps_dev, const cfog_match_result *res_dev,
                                 const int32_t *job_start, int32_t n_jobs, int32_t degree,
                                 double rmse_threshold, int32_t min_keep, uint8_t *keep_dev,
                                 int32_t *order_dev, cfog_poly_model *models_dev, void *work_dev,
                                 size_t work_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Image rectification on a triangulated irregular network (Sec. IV, "Image
 * rectification": a piecewise linear model, one affine map per triangle of a
 * TIN over the CPs).
 * ------------------------------------------------------------------------- */

/* Delaunay triangulation (HOST only, no GPU work) of the points pts[i] (HOST
 * array) with keep[i] != 0 (keep may be NULL: all points).  Equal points count
 * once (the lowest index).  Triangles are written counter-clockwise (y down
 * counts as a left-handed frame: orientation by the sign of
 * (b-a) x (c-a) > 0) as index triples into pts: tris[3*t + 0..2], at most cap
 * triangles; *n_tris receives the count (at most 2*n).  Exact predicates (a
 * floating-point filter backed by integer arithmetic); for co-circular points
 * any of the valid triangulations may be returned.  Fewer than 3 points, or all collinear: 0 triangles.
 * CFOG_E_NOMEM when cap is too small (*n_tris still holds the count).       */
cfog_status cfog_tin_delaunay(const cfog_point *pts, int32_t n, const uint8_t *keep,
                              int32_t *tris, int32_t cap, int32_t *n_tris);

/* Device scratch bytes of cfog_tin_rectify for n_tris triangles and an
 * out_h x out_w output (0 on a bad argument). */
size_t cfog_tin_workspace_bytes(int32_t n_tris, int32_t out_h, int32_t out_w);

/* Piecewise-linear rectification of the sensed image onto the reference grid.
 * Triangle t (tris_dev[3t..3t+2], DEVICE, indices into the n_cps CPs, as
 * cfog_tin_delaunay writes them) maps its reference vertices p = cps_dev[i]
 * to their sensed positions p + (sub_dx, sub_dy) of res_dev[i]; the affine
 * map through these three correspondences sends every reference pixel (x, y)
 * of the triangle (edges included, exact integer tests; a pixel in several
 * triangles takes the lowest index) to a sensed point (u, v).  out(y, x) =
 * bilinear interpolation of the sensed image at (u, v) when 0 <= u <= w-1 and
 * 0 <= v <= h-1, else `nodata`; pixels in no triangle get `nodata` too.
 * out_dev: out_h x out_w FP32, row pitch out_pitch floats (DEVICE).
 * Degenerate or clockwise triangles cover nothing.  work_dev: device scratch
 * of cfog_tin_workspace_bytes bytes, 256-byte aligned (triangle maps and the
 * per-tile triangle lists; overwritten by every call, so calls sharing it
 * must not overlap on the GPU).  Asynchronous on `stream`; argument errors
 * (CFOG_E_INVAL) and a short workspace (CFOG_E_NOMEM) are found before any
 * launch.                                                                    */
cfog_status cfog_tin_rectify(const cfog_image *sen, const cfog_point *cps_dev,
                             const cfog_match_result *res_dev, int32_t n_cps,
                             const int32_t *tris_dev, int32_t n_tris, int32_t out_h,
                             int32_t out_w, float nodata, float *out_dev, int64_t out_pitch,
                             void *work_dev, size_t work_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CFOG_H */
