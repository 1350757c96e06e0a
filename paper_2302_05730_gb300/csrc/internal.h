// Host-side declarations shared by the translation units of libmcubes.so (not installed).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mcubes {

// One validated problem: integrand, dimension, precision, stratification and the launch
// parameters of its V-Sample kernel (pointers and per-iteration fields left for the caller).
struct Problem {
    int fid, d, prec;
    int64_t g, m, p;
    VsampleParams P;
};

// Number of FP64 parameters integrand fid takes at dimension d (2d, or d^2 + d for the
// rotated Gaussian).
inline int param_len(int fid, int d) { return fid == 9 ? d * d + d : 2 * d; }

// Host helpers of capi.cu, shared with the batched path.
int cuda_status(cudaError_t e);   // MCUBES_* status of a CUDA error (records it per thread)
// Every device / pinned-host allocation of the library goes through these (the fault hook of
// mcubes_fail_alloc sits here).
cudaError_t mc_malloc(void **p, size_t bytes);
cudaError_t mc_malloc_host(void **p, size_t bytes);
int stratify(int d, int64_t n, int64_t *g, int64_t *m, int64_t *p);
int prepare(int fid, const double *params, int d, int64_t ncall, uint64_t seed, int iteration,
            uint32_t job, int adjust, int prec, Problem &pb);

// Launch request of one V-Sample kernel.
struct LaunchReq {
    int threads;          // threads per block
    int user_threads;     // 1: threads was requested (else each kernel takes its default size)
    int blocks_per_sm;    // 0: as many as fit (occupancy)
    int num_sms;          // SMs of the device
    int plain64;          // 1: the plain FP64 V-Sample kernel even where the fast one serves the family
};

}  // namespace mcubes
struct mcubes_tuning;
namespace mcubes {
// Launch request from the public tuning struct (NULL: defaults) on the current device.
int make_req(const mcubes_tuning *tune, LaunchReq &req);

// Per-(precision, integrand) launchers, one translation unit each (vsample_inst.cu).
// Return a cudaError_t value.
#define MCUBES_DECLARE_LAUNCHER(PREC, FID) \
    int launch_vsample_##PREC##_##FID(int d, const VsampleParams &P, const LaunchReq &req, cudaStream_t s);
MCUBES_DECLARE_LAUNCHER(f64, 0)
MCUBES_DECLARE_LAUNCHER(f64, 1)
MCUBES_DECLARE_LAUNCHER(f64, 2)
MCUBES_DECLARE_LAUNCHER(f64, 3)
MCUBES_DECLARE_LAUNCHER(f64, 4)
MCUBES_DECLARE_LAUNCHER(f64, 5)
MCUBES_DECLARE_LAUNCHER(f64, 6)
MCUBES_DECLARE_LAUNCHER(f64, 7)
MCUBES_DECLARE_LAUNCHER(f64, 8)
MCUBES_DECLARE_LAUNCHER(f64, 9)
MCUBES_DECLARE_LAUNCHER(f32, 0)
MCUBES_DECLARE_LAUNCHER(f32, 1)
MCUBES_DECLARE_LAUNCHER(f32, 2)
MCUBES_DECLARE_LAUNCHER(f32, 3)
MCUBES_DECLARE_LAUNCHER(f32, 4)
MCUBES_DECLARE_LAUNCHER(f32, 5)
MCUBES_DECLARE_LAUNCHER(f32, 6)
MCUBES_DECLARE_LAUNCHER(f32, 7)
MCUBES_DECLARE_LAUNCHER(f32, 8)
MCUBES_DECLARE_LAUNCHER(f32, 9)
#undef MCUBES_DECLARE_LAUNCHER

// Batched launchers: one (precision, integrand) slice, any d. hist_mode 0 = block-private
// shared histogram, 1 = FP64 atomics straight into each job's global bin contributions, 2 = the fast
// FP64 kernel of the Genz families (shared histogram; every job's parameters carry its fold).
struct BatchJob;
struct BatchTile;
#define MCUBES_DECLARE_BATCH_LAUNCHER(PREC, FID)                                                   \
    int launch_vsample_batch_##PREC##_##FID(int d, const BatchJob *jobs, const BatchTile *tiles,   \
                                            int n_tiles, int iteration, int parity, int adjust,     \
                                            int hist_mode, const LaunchReq &req, cudaStream_t s);
MCUBES_DECLARE_BATCH_LAUNCHER(f64, 0)
MCUBES_DECLARE_BATCH_LAUNCHER(f64, 1)
MCUBES_DECLARE_BATCH_LAUNCHER(f64, 2)
MCUBES_DECLARE_BATCH_LAUNCHER(f64, 3)
MCUBES_DECLARE_BATCH_LAUNCHER(f64, 4)
MCUBES_DECLARE_BATCH_LAUNCHER(f64, 5)
MCUBES_DECLARE_BATCH_LAUNCHER(f64, 6)
MCUBES_DECLARE_BATCH_LAUNCHER(f64, 7)
MCUBES_DECLARE_BATCH_LAUNCHER(f64, 8)
MCUBES_DECLARE_BATCH_LAUNCHER(f64, 9)
MCUBES_DECLARE_BATCH_LAUNCHER(f32, 0)
MCUBES_DECLARE_BATCH_LAUNCHER(f32, 1)
MCUBES_DECLARE_BATCH_LAUNCHER(f32, 2)
MCUBES_DECLARE_BATCH_LAUNCHER(f32, 3)
MCUBES_DECLARE_BATCH_LAUNCHER(f32, 4)
MCUBES_DECLARE_BATCH_LAUNCHER(f32, 5)
MCUBES_DECLARE_BATCH_LAUNCHER(f32, 6)
MCUBES_DECLARE_BATCH_LAUNCHER(f32, 7)
MCUBES_DECLARE_BATCH_LAUNCHER(f32, 8)
MCUBES_DECLARE_BATCH_LAUNCHER(f32, 9)
#undef MCUBES_DECLARE_BATCH_LAUNCHER

int launch_rebin(int d, const double *d_grid_in, const double *d_C, double *d_grid_out,
                 double alpha, cudaStream_t stream);


// Rebin of many (job, axis) pairs in one launch: block b refines axis axis[b] of job job[b],
// reading grid_in[job] (d_job x 501), C[job] and writing grid_out[job].
int launch_rebin_batch(int n_blocks, const uint32_t *block_job, const uint32_t *block_axis,
                       const double *const *grid_in, const double *const *C, double *const *grid_out,
                       double alpha, cudaStream_t stream);

}  // namespace mcubes
