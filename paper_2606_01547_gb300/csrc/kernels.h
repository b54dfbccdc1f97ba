// Host-visible launchers of the CUDA kernels (internal to liblenssim.so).
#pragma once

#include <cuda_runtime.h>

#include "lens_device.cuh"

namespace ls {

// Launch shape of the fused trace kernel: `nw` warps per CTA split the subhalo list of one
// 8x4-pixel tile; `pts` sub-pixel samples per thread per pass.
struct TraceShape {
  int nw;
  int pts;
};

TraceShape choose_trace_shape(int nx, int ny, int s, int n_sub, int sm_count);

// Per-subhalo constants from a SoA [5][ld] table (cx, cy, Rs, alpha_Rs, r_t).
cudaError_t launch_tnfw_prep(const float* soa, int n, int ld, float4* table, cudaStream_t st);

// Fused ray-trace + subhalo sum + Sersic + supersample bin-down of one system into sys.out.
cudaError_t launch_trace(const DevSystem& sys, TraceShape shape, cudaStream_t st);

// Total deflection at n device points.
cudaError_t launch_deflection(const DevSystem& sys, const float* x, const float* y, int n, float* ax,
                              float* ay, cudaStream_t st);

// Zero-padded 'same' convolution (flip = 1) or correlation (flip = 0) of n_img images.
cudaError_t launch_conv(const float* in, float* out, int n_img, int ny, int nx, const float* K, int k,
                        int flip, cudaStream_t st);

}  // namespace ls
