/*
 * mcubes.h -- C ABI of the GB300 (sm_103a) m-Cubes integrator library (libmcubes.so).
 *
 * m-Cubes (Sakiotis et al.; the integrator of arXiv 2302.05730, Sec. 3.2) is a VEGAS-style
 * Monte Carlo integrator over the unit cube [0,1]^d. Each iteration:
 *   - splits [0,1]^d into m = g^d sub-cubes and draws p samples in each;
 *   - maps every draw through the separable VEGAS importance grid (500 bins per axis);
 *   - evaluates the integrand and forms each sub-cube's mean and variance;
 *   - accumulates per-bin contributions (Algorithm 2, the "V-Sample" kernel).
 * The grid is then refined from the bin contributions (Rebin). The iteration estimates are
 * combined by inverse-variance weighting.
 *
 * Conventions for every call:
 *   - Return value: a status code (MCUBES_OK = 0 on success). Nothing is thrown across the ABI.
 *     Output buffers are written only on MCUBES_OK (a result struct's status field is set
 *     either way).
 *   - Host pointers are owned by the caller. The library copies what it needs and keeps no
 *     pointer after the call returns.
 *   - Device pointers ("d_" prefix) must be device memory of the current CUDA device. They
 *     must not be used by other work while the call's stream runs.
 *   - `stream` is a cudaStream_t, or NULL for a stream the library owns per host thread. The
 *     special handles cudaStreamLegacy and cudaStreamPerThread are accepted as well (use
 *     cudaStreamLegacy to order work with the legacy default stream). "_dev" calls are
 *     asynchronous on that stream; every other call synchronises before it returns.
 *   - Grids are row-major d x (MCUBES_NBINS + 1) doubles: B[i][0] = 0 < B[i][1] < ... <
 *     B[i][500] = 1. Bin contributions are d x MCUBES_NBINS doubles.
 *   - Integrand parameters are 2d doubles: a[0..d-1] then u[0..d-1] (constant: a[0] = c); the
 *     rotated Gaussian takes d^2 + d (see MCUBES_ROTATED_GAUSSIAN).
 *   - Calls from different host threads are safe. Each thread has its own cached workspace,
 *     released by mcubes_shutdown() on that thread.
 *   - Run log: with MCUBES_LOG=<file> in the environment, mcubes_integrate, mcubes_integrate_ex
 *     and mcubes_integrate_range append JSON lines to the file: one per iteration
 *     ({"event": "iteration", "it", "adjust", "I", "sigma", "running_estimate", "running_error",
 *     "running_chi2_dof", "samples"}) and one per call ({"event": "run", "integrand", "d",
 *     "samples_per_iter", "itmax", "iter_adjust", "iterations", "precision", "ms",
 *     "samples_per_s", and for whole runs "estimate", "error", "chi2_dof"}). Non-finite values
 *     are written as null.
 */
#ifndef MCUBES_H
#define MCUBES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* VEGAS bins per axis: Algorithm 2's inputs B[500 d] and C[500 d] (Sec. 3.2). */
#define MCUBES_NBINS 500
/* Largest supported dimension. */
#define MCUBES_DMAX 16

/* Status codes. */
#define MCUBES_OK 0
#define MCUBES_ERR_INVALID_ARG 1      /* a size, count, pointer or flag is out of range */
#define MCUBES_ERR_UNSUPPORTED_DIM 2  /* d < 1 or d > MCUBES_DMAX */
#define MCUBES_ERR_UNKNOWN_INTEGRAND 3
#define MCUBES_ERR_CUDA 4             /* a CUDA runtime call failed; see mcubes_last_cuda_error() */
#define MCUBES_ERR_ALLOC 5            /* device or pinned-host allocation failed */
#define MCUBES_ERR_NONFINITE 6        /* the integrand produced a NaN or infinity */
#define MCUBES_ERR_TIMEOUT 7          /* a bounded device-side wait gave up */
#define MCUBES_ERR_WORKSPACE 8        /* caller-provided workspace too small or misaligned */

/* Integrands: Genz families behind the paper's benchmark integrands (Sec. 5, Eq. 1-6) plus
 * the addition integrand of Sec. 5.3 and a constant. */
#define MCUBES_OSCILLATORY 0    /* cos(2 pi u_0 + sum a_i x_i)          Eq. 1: a_i = i, u_0 = 0 */
#define MCUBES_PRODUCT_PEAK 1   /* prod (a_i^-2 + (x_i - u_i)^2)^-1     Eq. 2: a_i = 50, u_i = 1/2 */
#define MCUBES_CORNER_PEAK 2    /* (1 + sum a_i x_i)^-(d+1)             Eq. 3: a_i = i */
#define MCUBES_GAUSSIAN 3       /* exp(-sum a_i^2 (x_i - u_i)^2)        Eq. 4: a_i = 25, u_i = 1/2 */
#define MCUBES_C0 4             /* exp(-sum a_i |x_i - u_i|)            Eq. 5: a_i = 10, u_i = 1/2 */
#define MCUBES_DISCONTINUOUS 5  /* exp(sum a_i x_i) if x_i < u_i on every axis, else 0
                                                                         Eq. 6: a_i = i+4, u_i = (3+i)/10 */
#define MCUBES_ADDITION 6       /* sum x_i                               Sec. 5.3 */
#define MCUBES_CONSTANT 7       /* a_0 */
/* Correlated and multi-modal cases for the learned proposal (the paper has none):
 *   double Gaussian: exp(-sum a_i^2 (x_i - u_i)^2) + exp(-sum a_i^2 (x_i - 1 + u_i)^2);
 *   rotated Gaussian: exp(-(x - c)^T M (x - c)), params = M (d x d, row-major) then c (d), so
 *     d^2 + d doubles instead of 2d. */
#define MCUBES_DOUBLE_GAUSSIAN 8
#define MCUBES_ROTATED_GAUSSIAN 9
#define MCUBES_N_INTEGRANDS 10

/* Arithmetic of the sampling path.
 *   MCUBES_FP64: the paper's setting. Draws, map, integrand and statistics are all FP64.
 *   MCUBES_FP32_EVAL: the point is formed, and the integrand evaluated, in FP32 with fast
 *     SFU math. The integrand is scaled by a host-computed FP64 factor so that it stays in
 *     range. Per-cube combination, the global sums and Rebin stay FP64. */
#define MCUBES_FP64 0
#define MCUBES_FP32_EVAL 1

typedef struct mcubes_result {
    double estimate;          /* combined integral estimate */
    double error;             /* its standard deviation */
    double chi2_dof;          /* chi^2 per degree of freedom of the iteration estimates */
    int32_t iters_done;
    int32_t status;           /* mirrors the return value */
    int64_t samples_per_iter; /* m * p, the samples actually drawn per iteration */
} mcubes_result;

/* Launch tuning. Zero fields take the defaults. */
typedef struct mcubes_tuning {
    int32_t block_threads;    /* threads per V-Sample block (64..256, multiple of 32). Default: 256;
                                 1024 for FP32 adjusting iterations, whose one block per SM holds the
                                 fixed-point histogram; 512 for the FP64 kernel of the Genz families up to
                                 d = 12 (one block per SM, one copy of its tables) */
    int32_t blocks_per_sm;    /* resident blocks per SM to launch (persistent grid); default: occupancy */
    int32_t fp64_plain;       /* FP64 precision, single-job V-Sample: 0 (default) takes the FP64 kernel with
                                 integer bin extraction and per-bin folded integrand tables for the six Genz
                                 families (the same quantities to FP64 rounding, bins bit-identical; adjusting
                                 launches add half of each sample's bin contributions to C with FP64
                                 reductions, so C's summation order varies from run to run);
                                 1 forces the plain FP64 kernel, which evaluates the definition step by step */
    int32_t reserved[5];
} mcubes_tuning;

/* Stratification (Sec. 3.2: m sub-cubes so that a 2-point MC estimate runs in each while about
 * ncall samples are drawn). g is the largest integer with 2 g^d <= ncall, m = g^d,
 * p = max(2, floor(ncall / m)). Host only.
 * Errors: UNSUPPORTED_DIM; INVALID_ARG if ncall < 2, m >= 2^32, or an output pointer is NULL. */
int mcubes_stratify(int d, int64_t ncall, int64_t *g, int64_t *m, int64_t *p);

/* Whole integration (the paper's problem statement; V-Sample = Algorithm 2, then Rebin).
 * itmax iterations (1..65535). The first iter_adjust (0..itmax) iterations accumulate bin
 * contributions and refine the grid; the rest sample a frozen grid. All iterations are
 * combined by inverse-variance weighting (an iteration with zero variance makes the estimate
 * the mean of such iterations, with error 0). Philox4x32-10 is keyed by seed. FP64 precision,
 * default tuning, library stream.
 * Errors: UNSUPPORTED_DIM, UNKNOWN_INTEGRAND, INVALID_ARG (NULL params/out, ncall < 2,
 * itmax out of range, m >= 2^32), ALLOC, CUDA, NONFINITE. */
int mcubes_integrate(int integrand_id, const double *params, int d, int64_t ncall, int itmax,
                     int iter_adjust, uint64_t seed, mcubes_result *out);

/* mcubes_integrate with every option.
 *   precision: MCUBES_FP64 or MCUBES_FP32_EVAL.
 *   tune: NULL for defaults.
 *   stream: cudaStream_t or NULL.
 *   iter_out: NULL, or 2 * itmax doubles that receive (I_it, Var_it) for each iteration.
 *   grid_in: NULL for the uniform grid, else d x 501 starting grid (host).
 *   grid_out: NULL, or d x 501 doubles that receive the final grid (host).
 * FP32_EVAL additionally requires g <= 2^24 (INVALID_ARG otherwise). */
int mcubes_integrate_ex(int integrand_id, const double *params, int d, int64_t ncall, int itmax,
                        int iter_adjust, uint64_t seed, int precision, const mcubes_tuning *tune,
                        void *stream, double *iter_out, const double *grid_in, double *grid_out,
                        mcubes_result *out);

/* Checkpoint and resume: iterations [it_begin, it_end) of an integration of itmax iterations
 * whose first iter_adjust iterations refine the grid. The Philox counters use the absolute
 * iteration index, so running [0, k) and then [k, itmax) from the returned grid repeats the
 * uninterrupted run, up to the order of floating-point sums.
 *   grid_in: the grid before iteration it_begin (d x 501, host). NULL only for it_begin == 0
 *     (uniform grid).
 *   prev_estimate: the estimate of iteration it_begin - 1, or 0 if none. It only sets the
 *     FP32-eval histogram scale.
 *   grid_out: NULL, or d x 501 doubles that receive the grid after the range.
 *   iter_out: 2 x (it_end - it_begin) doubles: (I_it, Var_it).
 * Combine all iterations with mcubes_combine. FP32_EVAL additionally requires g <= 2^24.
 * Errors: as mcubes_integrate_ex; INVALID_ARG for a bad range, a NULL iter_out, or a NULL
 * grid_in with it_begin > 0. */
int mcubes_integrate_range(int integrand_id, const double *params, int d, int64_t ncall, int itmax,
                           int iter_adjust, int it_begin, int it_end, uint64_t seed, int precision,
                           const double *grid_in, double prev_estimate, double *grid_out, double *iter_out,
                           void *stream);

/* Inverse-variance combination of iterations [skip, n) of iter (n pairs (I_it, Var_it)), as in
 * mcubes_integrate. skip drops early iterations, e.g. those sampled before the grid settled.
 * Host only. Errors: INVALID_ARG (NULL pointers, n < 1, skip outside [0, n), a non-finite or
 * negative entry). */
int mcubes_combine(const double *iter, int n, int skip, mcubes_result *out);

/* One V-Sample pass (Algorithm 2) on a caller-supplied grid, with host buffers. This is the
 * per-iteration parity hook.
 *   iteration (0..65535) and job select the Philox counters (ctr = (t, q, iteration<<16 | j, job)).
 *   adjust != 0: bin contributions are accumulated. Then C_out (d x 500, may be NULL) receives
 *     them, and grid_out (d x 501, may be NULL) receives the Rebin of grid_in by them.
 *   adjust == 0: grid_out and C_out are ignored.
 *   grid_in: NULL for the uniform grid.
 *   I_out, var_out: the iteration's estimate (1/m) sum I_t and variance (1/m^2) sum V_t.
 * Errors: as mcubes_integrate_ex. */
int mcubes_vsample_once(int integrand_id, const double *params, int d, int64_t ncall,
                        uint64_t seed, int iteration, uint32_t job, int adjust, int precision,
                        const double *grid_in, double *grid_out, double *C_out,
                        double *I_out, double *var_out);

/* ---------------------------------------------------------------------------------------
 * Device-level calls: all pointers are device memory, work is queued on `stream` and the call
 * returns without synchronising. Host-side argument errors are reported at once; kernel
 * errors surface at the caller's next synchronisation.
 * --------------------------------------------------------------------------------------- */

/* The V-Sample kernel alone (Algorithm 2). Accumulates into d_sums[0] += sum_t I_t and
 * d_sums[1] += sum_t V_t (not yet divided by m, m^2), and, when adjust != 0, into
 * d_C[i][k] += sum of w^2 (d x 500). The caller zeroes d_sums and d_C first.
 *   d_grid: d x 501.
 *   d_prev: NULL, or the previous iteration's (I, Var) on the device. In FP32_EVAL it sets the
 *     scale of the single-precision histogram; it never changes the result beyond rounding.
 *   d_probe: NULL, or (m >> probe_shift) + 1 pairs of doubles. Sub-cube t with
 *     t mod 2^probe_shift == 0 writes (I_t, V_t) to pair t >> probe_shift.
 * Errors: as mcubes_integrate_ex. INVALID_ARG if d_grid or d_sums is NULL, if adjust is set
 * with d_C NULL, or if probe_shift is outside 0..31. */
int mcubes_vsample_dev(int integrand_id, const double *params, int d, int64_t ncall,
                       uint64_t seed, int iteration, uint32_t job, int adjust, int precision,
                       const double *d_grid, double *d_C, double *d_sums, const double *d_prev,
                       double *d_probe, int probe_shift, const mcubes_tuning *tune, void *stream);

/* Grid refinement (VEGAS, Lepage 1978; m-Cubes delegates to it). Per axis, on the device:
 *   1. 3-point smoothing of C;
 *   2. normalisation;
 *   3. damping r = ((1 - rho)/ln(1/rho))^alpha with alpha = 1.5;
 *   4. new boundaries at equal damped mass, linear inside each old bin.
 * An axis with no contribution keeps its grid. d_grid_out and d_grid_in must be distinct.
 * Errors: UNSUPPORTED_DIM, INVALID_ARG (NULL or aliased pointers), CUDA. */
int mcubes_rebin_dev(int d, const double *d_grid_in, const double *d_C, double *d_grid_out,
                     void *stream);

/* Bytes of device workspace one mcubes_iteration_dev call needs for dimension d (the bin
 * contribution accumulator and the sums; 256-byte aligned). */
size_t mcubes_workspace_bytes(int d);

/* One whole iteration on the device: zero the workspace, V-Sample, and Rebin (when adjust),
 * then write d_result[0] = I = sum I_t / m and d_result[1] = Var = sum V_t / m^2.
 *   d_grid_out: receives the refined grid when adjust != 0, else a copy of d_grid_in; it must
 *     not alias d_grid_in.
 *   d_prev: optional previous (I, Var), as in mcubes_vsample_dev.
 *   d_workspace: at least mcubes_workspace_bytes(d) bytes of scratch, 256-byte aligned. Its
 *     contents are overwritten.
 * Errors: as mcubes_vsample_dev; WORKSPACE if d_workspace is NULL, misaligned or too small. */
int mcubes_iteration_dev(int integrand_id, const double *params, int d, int64_t ncall,
                         uint64_t seed, int iteration, uint32_t job, int adjust, int precision,
                         const double *d_grid_in, double *d_grid_out, double *d_result,
                         const double *d_prev, void *d_workspace, size_t workspace_bytes,
                         const mcubes_tuning *tune, void *stream);

/* mcubes_iteration_dev without caller scratch. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they run an iteration. Examples:
 * an application whose memory pool already owns the whole device, or a latency-critical loop
 * where cudaMalloc/cudaFree would stall or synchronise the device.
 *   - The scratch (bin-contribution accumulator and sums) is a fixed array inside the library
 *     of mcubes_static_scratch_bytes() bytes (64,256: enough for d <= 16). Every GPU that loads
 *     the library holds it until the process exits.
 *   - The call allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress, once
 *     per device, with that device current). Make that first call before any stream capture.
 *   - Under CUDA's default lazy module loading, the first address lookup and the first launch of
 *     each (precision, integrand, d) kernel can make the CUDA driver load code, which takes device
 *     memory. A caller whose pool will own the whole device should make one call of every
 *     configuration it uses before the pool claims the device, or run with
 *     CUDA_MODULE_LOADING=EAGER.
 *   - Every call shares the one array per device. The call clears it before use, but two calls
 *     whose work overlaps on the GPU (different streams, no ordering) race on it.
 *   - `stream` NULL means the legacy default stream here, not the library's own stream (creating
 *     that stream would allocate).
 * Arguments and results as mcubes_iteration_dev.
 * Errors: as mcubes_iteration_dev; WORKSPACE if the iteration needs more scratch than the array
 * holds; CUDA if the address lookup fails. */
int mcubes_iteration_dev_static(int integrand_id, const double *params, int d, int64_t ncall,
                                uint64_t seed, int iteration, uint32_t job, int adjust, int precision,
                                const double *d_grid_in, double *d_grid_out, double *d_result,
                                const double *d_prev, const mcubes_tuning *tune, void *stream);

/* Size in bytes of the fixed scratch array behind mcubes_iteration_dev_static. */
size_t mcubes_static_scratch_bytes(void);

/* ---------------------------------------------------------------------------------------
 * Batches of independent integrations (the target's batched form; the paper runs one
 * integration at a time). Every job runs mcubes_integrate's iteration schedule, all jobs
 * together: each iteration launches one persistent V-Sample kernel per (d, integrand) class and
 * one Rebin kernel for all (job, axis) pairs. The whole schedule is captured once into a CUDA
 * graph and launched as one graph. Job j draws with Philox counter word 3 = j and key = its
 * seed, so it reproduces mcubes_vsample_once(..., job = j) iteration by iteration.
 * --------------------------------------------------------------------------------------- */
typedef struct mcubes_job {
    int32_t integrand_id;
    int32_t d;                 /* 1..MCUBES_DMAX */
    int64_t ncall;             /* samples per iteration (>= 2) */
    const double *params;      /* 2d doubles (host), copied */
    uint64_t seed;
} mcubes_job;

/* Launch shape of the batched V-Sample kernel per dimension d (index d; entry 0 unused).
 * Zero entries take the defaults (256 threads, 4 sub-cubes per thread per tile, block-private
 * histogram). A tile is block_threads x cubes_per_thread consecutive sub-cubes of one job.
 * hist_mode 0: block-private shared-memory histogram, flushed once per job and block.
 * hist_mode 1: FP64 atomics straight into the job's global bin contributions.
 * In FP64, the jobs of one (d, Genz family) class take the fast FP64 V-Sample kernel (the one
 * mcubes_tuning.fp64_plain describes; half of each sample's bin adds as FP64 reductions into the
 * job's C, half into a block-private shared copy; hist_mode not consulted)
 * when every job of the class meets its conditions and its shared memory fits; fp64_plain = 1
 * sends every class to the plain kernels. mcubes_tune_batch leaves it 0. */
typedef struct mcubes_batch_tuning {
    int32_t block_threads[MCUBES_DMAX + 1];
    int32_t cubes_per_thread[MCUBES_DMAX + 1];
    int32_t hist_mode[MCUBES_DMAX + 1];
    int32_t fp64_plain;   /* 0 or 1, else INVALID_ARG */
} mcubes_batch_tuning;

/* Integrate n_jobs independent problems together on the current device.
 *   itmax, iter_adjust: as mcubes_integrate, shared by all jobs.
 *   precision: MCUBES_FP64 or MCUBES_FP32_EVAL.
 *   tune: NULL for defaults, or the output of mcubes_tune_batch.
 *   stream: cudaStream_t the work is ordered after and before (NULL: the library stream). The
 *     graph itself runs on a library stream.
 *   out: n_jobs results.
 *   iter_out: NULL or n_jobs x itmax x 2 doubles (I_it, Var_it), job-major.
 * Device memory for grids, bin contributions and sums is allocated for the call and freed before
 * it returns. Synchronous.
 * Errors: INVALID_ARG (n_jobs < 1, NULL jobs/out, a job's arguments as mcubes_integrate_ex),
 * UNSUPPORTED_DIM, UNKNOWN_INTEGRAND, ALLOC, CUDA, NONFINITE (a job's estimate is not finite; the
 * other jobs' results are still written, and each result's status says which failed). */
int mcubes_integrate_batch(int n_jobs, const mcubes_job *jobs, int itmax, int iter_adjust, int precision,
                           const mcubes_batch_tuning *tune, void *stream, mcubes_result *out,
                           double *iter_out);

/* Autotuner of the batched V-Sample kernel. For every dimension present in the batch, it times
 * one grid-adjusting V-Sample pass over that dimension's jobs on the device. Candidates:
 * block_threads in {128, 256}, cubes_per_thread in {1, 2, 4, 8, 16}, hist_mode in {0, 1}. The
 * fastest of each goes into *out; dimensions not present keep zeros (defaults). Synchronous;
 * allocates and frees its own device memory.
 * Errors: as mcubes_integrate_batch. */
int mcubes_tune_batch(int n_jobs, const mcubes_job *jobs, int precision, mcubes_batch_tuning *out);

/* ---------------------------------------------------------------------------------------
 * PAGANI, the paper's other workload (Sec. 3.1): the region-evaluation kernel (the PAGANI-kernel
 * algorithm) and an adaptive driver around it. FP64 throughout.
 *   Rule (the paper defers it to PAGANI; the reading here): the Genz-Malik fully symmetric rule
 *   of degree 7 with its embedded rule of degree 5 on each region, f_eval = 1 + 4d + 2d(d-1) + 2^d
 *   points, and three lower-degree rules on the same points (degree 3 on the centre and the
 *   +-l2 e_i points, degree 3 on the centre and the +-l3 e_i points, the centre alone): five
 *   rules, as the paper's kernel accumulates. I = the degree-7 estimate; E = |R7 - R5| when the
 *   differences of successive degrees fall at least fourfold (|R7 - R5| <= |R5 - R3| / 4 <=
 *   |R3 - R1| / 16, each difference its largest over the two degree-3 rules), else the largest of
 *   them; the split axis of the region = the
 *   largest fourth divided difference along the axes (ties -- within 1e-12 of the larger
 *   difference and of the largest |f| at the centre and axis points -- go to the longest side,
 *   then the lowest axis).
 *   Regions: row-major n x d arrays of low corners and side lengths.
 * Supported: 2 <= d <= 16 (f_eval grows as 2^d).
 * --------------------------------------------------------------------------------------- */
typedef struct mcubes_pagani_result {
    double estimate, error;
    int64_t regions_evaluated;  /* over all iterations */
    int32_t iterations;
    int32_t status;             /* 0 converged, 1 iteration limit, 2 region limit */
    int64_t active_regions;     /* regions evaluated in the last iteration */
} mcubes_pagani_result;

/* f_eval of the rule at dimension d, or 0 if unsupported. */
int mcubes_pagani_rule_points(int d);

/* The PAGANI kernel on n_regions device regions (d_lo, d_len: n x d FP64): d_I, d_E (FP64) and
 * d_axis (int32) per region. params as mcubes_integrate. Asynchronous on stream (NULL: the legacy
 * default stream). Errors: INVALID_ARG, UNSUPPORTED_DIM (d < 2 or d > 16), UNKNOWN_INTEGRAND, CUDA. */
int mcubes_pagani_evaluate_dev(int integrand_id, const double *params, int d, int64_t n_regions,
                               const double *d_lo, const double *d_len, double *d_I, double *d_E,
                               int32_t *d_axis, void *stream);

/* Adaptive integration over [0,1]^d (reading; the paper describes the kernel only). The cube starts
 * as init_split^d equal regions. Each iteration evaluates every active region; with the running
 * totals I = I_done + sum I_r and E = E_done + sum E_r it stops once E <= rel_tol |I|. Otherwise a
 * region with E_r <= rel_tol |I| V_r is finished (joins I_done, E_done) and every other region is
 * halved along its split axis (lower half first, children in the parents' order). The run also
 * stops after max_iters iterations, when no region is left, or when the next set would exceed
 * max_regions (at most 2^31 - 1). Synchronous; allocates and frees its own device memory
 * (about 32 d max_regions bytes). Errors: as mcubes_pagani_evaluate_dev; INVALID_ARG for
 * rel_tol <= 0, max_iters < 1, init_split < 1 or init_split^d > max_regions; NONFINITE. */
int mcubes_pagani_integrate(int integrand_id, const double *params, int d, double rel_tol, int max_iters,
                            int64_t max_regions, int init_split, mcubes_pagani_result *out);

/* ---------------------------------------------------------------------------------------
 * Learned proposal (the target's extension; the paper's m-Cubes uses the VEGAS grid only): a
 * coupling flow on [0,1]^d (neural importance sampling: coupling layers whose transformed axes
 * go through piecewise-quadratic CDFs computed by a ReLU MLP). The MLPs run on the tensor
 * cores with bf16 operands and FP32 accumulation.
 *   Axis split of layer l: l mod 4 = 0 -> kept axes A = the first floor(d/2); 1 -> the halves
 *   swapped; 2 -> A = the even axes; 3 -> swapped.
 *   Parameters (FP32, flat), per layer: W1 [H x |A|], b1 [H], W2 [H x H], b2 [H],
 *   W3 [|B|(2K+1) x H], b3 [|B|(2K+1)]; output slot s holds K bin-width logits, then K+1
 *   edge-value logits, for axis B[s].
 * Supported: 2 <= d <= 16, 1 <= layers <= 32, hidden in {32, 64, 128}, bins in {4, 8, 16, 32}
 * (large d x bins x hidden combinations may exceed shared memory: CUDA error).
 * Device buffers are row-major n x d FP32 (points), n FP32 (log densities).
 * --------------------------------------------------------------------------------------- */
typedef struct mcubes_flow_shape {
    int32_t d, layers, hidden, bins;
} mcubes_flow_shape;

/* Number of FP32 parameters, or 0 for an unsupported shape. */
int64_t mcubes_flow_param_count(const mcubes_flow_shape *shape);

/* Scratch bytes for n samples (256-byte aligned buffer expected), or 0 if unsupported. */
size_t mcubes_flow_work_bytes(const mcubes_flow_shape *shape, int64_t n);

/* Density direction: d_z = flow(d_x), d_logq = log q(x). Asynchronous on stream.
 * Errors: INVALID_ARG, WORKSPACE, CUDA. */
int mcubes_flow_forward_dev(const mcubes_flow_shape *shape, const float *d_params, int64_t n, const float *d_x,
                            float *d_z, float *d_logq, void *d_work, size_t work_bytes, void *stream);

/* Sampling direction: d_x = flow^-1(d_z), d_logq = log q(x). Asynchronous on stream. */
int mcubes_flow_inverse_dev(const mcubes_flow_shape *shape, const float *d_params, int64_t n, const float *d_z,
                            float *d_x, float *d_logq, void *d_work, size_t work_bytes, void *stream);

/* Loss and gradient on n samples x with weights w (normalised to sum 1 by the caller):
 *   loss_kind 0 (variance, chi^2): L = sum w / q(x)   (w = f^2 J from the grid sampler);
 *   loss_kind 1 (KL):              L = -sum w log q(x) (w = |f| J).
 * d_grad (param_count FP32) and d_loss[0] accumulate; zero them first. Asynchronous.
 * Kernels: widths 64 and 128 (output GEMM at most 256 wide, K <= 16) run on the tcgen05 training
 * kernels (tensor-core MMAs with TMEM accumulators), width 32 and shapes beyond those on the fused
 * mma.sync kernels, and shapes neither fits on the per-layer kernels; the environment variable
 * MCUBES_FLOW_TRAIN=mma or =chain forces the latter two (for comparisons). The tcgen05 kernels'
 * waits are bounded: if one expires they set the int at the workspace's last 256 bytes
 * (mcubes_flow_work_bytes(shape, n) - 256), and the gradient is then invalid; mcubes_flow_integrate
 * checks that word after training (TIMEOUT). */
int mcubes_flow_grad_dev(const mcubes_flow_shape *shape, const float *d_params, int64_t n, const float *d_x,
                         const float *d_w, int loss_kind, float *d_grad, float *d_loss, void *d_work,
                         size_t work_bytes, void *stream);

/* Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; step >= 1) on the FP32 parameters. */
int mcubes_flow_adam_dev(int64_t n_params, float *d_params, const float *d_grad, float *d_m, float *d_v, int step,
                         float lr, void *stream);

/* Scratch bytes of mcubes_flow_sample_dev (the bf16 copy of the weights in the fused kernel's
 * layout), or 0 when the shape is unsupported or has more than 16 layers. */
size_t mcubes_flow_sample_work_bytes(const mcubes_flow_shape *shape);

/* Fused flow-proposal sampling of samples [i0, i0 + n) of one m-Cubes iteration, in one kernel:
 * sample i = t p + q of sub-cube t (stratification of ncall as mcubes_stratify) draws the
 * FP32-layout Philox uniforms u (counter (t, q, iteration << 16 | j, job), key = seed), takes the
 * latent point z = (c + u) / g (the sub-cube's strata in latent space, Sec. 3.2 stratification
 * carried over), then x = flow^-1(z) and q(x), and the weight
 *   d_w[i - i0] = (f(x) / F) / q(x),
 * f evaluated in the FP32-eval form and scaled by the integrand's FP32 factor F (*fscale_out).
 * d_x (n x d) and d_logq (n) are optional (NULL: not written). params: as mcubes_integrate.
 * d_work: mcubes_flow_sample_work_bytes bytes, 256-byte aligned. Asynchronous on stream.
 * Errors: INVALID_ARG (also when the shape needs more shared memory than the device offers),
 * UNSUPPORTED_DIM, UNKNOWN_INTEGRAND, WORKSPACE, CUDA. */
int mcubes_flow_sample_dev(const mcubes_flow_shape *shape, const float *d_params, int integrand_id,
                           const double *params, int64_t ncall, uint64_t seed, int iteration, uint32_t job,
                           int64_t i0, int64_t n, float *d_x, float *d_logq, float *d_w, double *fscale_out,
                           void *d_work, size_t work_bytes, void *stream);

/* Whole learned-proposal run:
 *   1. vegas_iters grid-adjusting m-Cubes iterations (FP32-eval), then flow_iters frozen-grid
 *      iterations as the reference;
 *   2. sets of train_samples points drawn through the adapted grid with their weights (f^2 J for
 *      the variance loss, |f| J for KL) train the flow (train_steps Adam steps of `batch` samples,
 *      starting from the identity flow; a fresh set is drawn for every pass over the previous
 *      one; the rate follows a cosine decay from lr to lr/10);
 *   3. flow_iters m-Cubes iterations sample with the flow: strata in latent space,
 *      x = flow^-1(z), weight f(x)/q(x).
 * All at ncall samples per iteration. params_out: NULL or mcubes_flow_param_count floats.
 * Synchronous; allocates and frees its own device memory.
 * Errors: INVALID_ARG (shape.d != d, unsupported shape, bad counts), as mcubes_integrate_ex,
 * NONFINITE. */
typedef struct mcubes_flow_config {
    mcubes_flow_shape shape;
    int32_t loss_kind;          /* 0: variance (chi^2), 1: KL */
    int32_t vegas_iters;        /* >= 1 */
    int32_t flow_iters;         /* >= 1 */
    int32_t train_steps;        /* >= 0 */
    int32_t batch;              /* >= 64 */
    float lr;
    int64_t ncall;              /* samples per iteration */
    int64_t train_samples;      /* points per training set (one epoch), >= batch */
    uint64_t seed;
} mcubes_flow_config;

typedef struct mcubes_flow_report {
    mcubes_result vegas;        /* frozen adapted-grid iterations */
    mcubes_result flow;         /* flow-proposal iterations */
    double vegas_var_per_sample;   /* mean per-iteration variance x samples per iteration */
    double flow_var_per_sample;
    double train_loss_first, train_loss_last;
    double seconds_vegas, seconds_train, seconds_flow;
} mcubes_flow_report;

int mcubes_flow_integrate(int integrand_id, const double *params, int d, const mcubes_flow_config *cfg,
                          float *params_out, mcubes_flow_report *out);

/* Philox4x32-10 on the device, for checking the generator. out[4j..4j+3] = Philox(ctr[4j..4j+3],
 * key = (seed mod 2^32, seed >> 32)) for j < n.
 *   impl 0: the library's own generator (the flow samplers use it).
 *   impl 1: the CUDA toolkit's cuRAND device function curand_Philox4x32_10.
 *   impl 2: the library's hoisted form (round 0 and part of round 1 precomputed per launch and
 *           per sub-cube), as the single-job V-Sample kernels draw; counter word 2 is split into
 *           its top 29 bits (the launch constant) and its low 3 bits (the draw word j).
 *   impl 3: the hoisted form with its constants in registers, as the batched V-Sample kernel
 *           draws; the same split of counter word 2.
 * Errors: INVALID_ARG (NULL pointers, impl not 0-3), CUDA. */
int mcubes_philox_dev(const uint32_t *d_ctr, uint64_t n, uint64_t seed, int impl,
                      uint32_t *d_out, void *stream);

/* Static description of a status code (never NULL). */
const char *mcubes_status_string(int status);

/* The last cudaError_t the calling thread saw inside the library (0 if none). */
int mcubes_last_cuda_error(void);

/* Release the calling thread's cached device workspace and stream. */
void mcubes_shutdown(void);

/* Unit rates of the current device, measured by microbenchmarks (about 50 ms): the per-SM
 * throughput of the operations the V-Sample kernels are built from, per SM clock at the
 * device's maximum SM clock (cudaDevAttrClockRate). out[0..min(n_out, 12) - 1] receives:
 *   0: FP32 fused multiply-adds (lanes); 1: FP64 fused multiply-adds (lanes);
 *   2: exp2f (lanes); 3: Philox4x32-10 calls;
 *   4: random 8-byte shared-memory gathers from an 8 x 500 table (lanes);
 *   5: random FP32 shared atomics into an 8 x 500 histogram (lanes);
 *   6: random u32 shared atomics with their old value into 8 lane-interleaved copies of an
 *      8 x 500 histogram, carry into a high word (lanes; one 1024-thread block an SM);
 *   7: random u64 shared reductions (no returned value) into one 8 x 500 histogram (lanes; one
 *      1024-thread block an SM); 8: the same into 4 lane-interleaved copies;
 *   9: random u32 shared reductions (no returned value) into 8 lane-interleaved copies;
 *   10: random 8-byte read-only global gathers from an 8 x 500 table (L1-resident; lanes);
 *   11: the same gathers, axes 0-3 from shared memory and 4-7 through L1 (lanes).
 * Errors: INVALID_ARG (NULL out, n_out < 1), ALLOC, CUDA. Synchronous. */
int mcubes_unit_rates(double *out, int n_out);

/* Allocation fault hook (for testing the error paths). After mcubes_fail_alloc(n) with n >= 1,
 * the n-th device or pinned-host allocation the library makes from then on (any thread) fails as
 * if out of memory: the call that needed it returns MCUBES_ERR_ALLOC, having released what it
 * had allocated, and later calls allocate afresh. n = 0 disarms the hook. The environment
 * variable MCUBES_FAULT_ALLOC=n arms it the same way at the library's first allocation.
 * Returns the number of allocations made since the library loaded. */
int64_t mcubes_fail_alloc(int64_t n);

/* Bounds-checked builds (libmcubes_checked.so): the kernels check every computed bin, sub-cube
 * and probe index against its bound; a failed check skips the access and is counted. Returns
 * the count since the last reset (and, if first is not NULL, the first failure as site << 48 |
 * index: site 1 table bin, 2 global bin, 3 sub-cube, 4 probe slot, 5 batch tile range), then
 * resets it when reset != 0. Returns -1 from a normal build. Synchronizes the device. */
int64_t mcubes_checked_violations(int reset, int64_t *first);

#ifdef __cplusplus
}
#endif

#endif /* MCUBES_H */
