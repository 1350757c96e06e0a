// Host-side declarations shared by the translation units of libmcubes.so (not installed).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mcubes {

// Launch request of one V-Sample kernel.
struct LaunchReq {
    int threads;          // threads per block
    int blocks_per_sm;    // 0: as many as fit (occupancy)
    int num_sms;          // SMs of the device
};

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
MCUBES_DECLARE_LAUNCHER(f32, 0)
MCUBES_DECLARE_LAUNCHER(f32, 1)
MCUBES_DECLARE_LAUNCHER(f32, 2)
MCUBES_DECLARE_LAUNCHER(f32, 3)
MCUBES_DECLARE_LAUNCHER(f32, 4)
MCUBES_DECLARE_LAUNCHER(f32, 5)
MCUBES_DECLARE_LAUNCHER(f32, 6)
MCUBES_DECLARE_LAUNCHER(f32, 7)
#undef MCUBES_DECLARE_LAUNCHER

int launch_rebin(int d, const double *d_grid_in, const double *d_C, double *d_grid_out,
                 double alpha, cudaStream_t stream);

}  // namespace mcubes
