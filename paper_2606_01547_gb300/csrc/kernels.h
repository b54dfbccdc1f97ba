// Host-visible launchers of the CUDA kernels (internal to liblenssim.so).
#pragma once

#include <cuda_runtime.h>

#include "lens_device.cuh"

namespace ls {

constexpr int kUnitPts = 9;      // samples per lane in a trace unit (a unit is 32 x 9 samples)
constexpr int kPackedPairs = 4;  // of a lane's samples, this many pairs run as FP32x2 instructions
constexpr int kTraceWarps = 8;   // warps per trace CTA, splitting the subhalo list

// One system's subhalo constants for the batched preparation kernel.
struct PrepJob {
  const float* soa;  // SoA [5][ld]
  float4* tab;       // kTableStride float4 per subhalo
  int n, ld;
};

// One image of a batched convolution; `tile0` is the prefix of 32x32 output tiles.
struct ConvJob {
  const float* in;
  float* out;
  const float* K;
  int ny, nx, k, tile0;
};

// Device header of a batched launch; every batch kernel reads its counts, pointers and work
// counters from here, so a captured graph does not depend on the batch.
struct BatchMeta {
  int n_sys, n_prep, n_conv, kmax;
  unsigned int trace_counter, conv_counter, pad0, pad1;  // zeroed by each call's header copy
  const DevSystem* systems;  // ordered by per-unit cost, largest first
  const int* unit_prefix;    // [n_sys + 1]
  const PrepJob* prep;       // [n_prep]
  const ConvJob* conv;       // [n_conv + 1], the last entry's tile0 = total tiles
};

// Per-subhalo constants from a SoA [5][ld] table (cx, cy, Rs, alpha_Rs, r_t).
cudaError_t launch_tnfw_prep(const float* soa, int n, int ld, float4* table, cudaStream_t st);

// Trace units of a system (one CTA per unit in the single-system launch).
int unit_count(int nx, int ny, int s);

// Fused ray-trace + subhalo sum + Sersic + supersample bin-down of one system into sys.out, by
// launch variant (all variants give bitwise-identical images):
// 0 one CTA of 8 warps per unit, 1 one CTA of 4 warps summing the 8 slices in two passes,
// 2 a cluster of 2 CTAs x 4 warps per unit, 3 a cluster of 4 CTAs x 2 warps per unit,
// 4 a cluster of 8 single-warp CTAs per unit.
constexpr int kTraceVariants = 5;
cudaError_t launch_trace_variant(const DevSystem& sys, int variant, cudaStream_t st);
const char* trace_variant_name(int v);

// Persistent batched trace over device descriptors; units are numbered by unit_prefix
// ([n_sys + 1] ints) and handed out through the header's counter (zeroed by each call's header
// copy).  Forms (bitwise-identical images): 0 CTAs of 4 warps in two passes, 1 CTAs of 8 warps,
// 2 clusters of 2 CTAs x 4 warps.
constexpr int kBatchForms = 3;
const char* batch_form_name(int form);
int trace_batch_grid(int sm_count, int form);
cudaError_t launch_trace_batch_meta(const BatchMeta* meta, int form, int grid, bool far, cudaStream_t st);

// Summed subhalo deflection at every sample of the grid (main deflectors excluded), in the
// order ((row * nx + column) * s + sub-row) * s + sub-column; the same sum as the image kernels.
cudaError_t launch_subhalo_field(const DevSystem& sys, float2* out, cudaStream_t st);

// Total deflection at n device points.
cudaError_t launch_deflection(const DevSystem& sys, const float* x, const float* y, int n, float* ax,
                              float* ay, cudaStream_t st);

// Zero-padded 'same' convolution (flip = 1) or correlation (flip = 0) of n_img images.
cudaError_t launch_conv(const float* in, float* out, int n_img, int ny, int nx, const float* K, int k,
                        int flip, cudaStream_t st);

// TMA form of the convolution for batches of equal-size images (odd k <= 31, nx % 4 == 0,
// 16-byte aligned buffers).  `err` is a host-mapped flag raised if a bounded wait expires.
bool conv_tma_supported(const float* in, const float* out, int ny, int nx, int k);
// FFT convolution (psf_fft.cu): padded sizes (false if beyond 1024); the central core x core taps
// the caller convolves directly for large kernels (0: none); workspace per image (the images' half
// spectra); the kernel's spectrum (its wings' half spectrum, then the core taps) and the work
// space that computes it; the convolution, added to `out` when accumulate is set.
bool conv_fft_sizes(int ny, int nx, int k, int* My, int* Mx);
int conv_fft_core(int k);
size_t conv_fft_bytes_per_image(int ny, int Mx);
size_t conv_fft_spectrum_bytes(int My, int Mx, int k);
size_t conv_fft_spectrum_work_bytes(int Mx, int k);
cudaError_t launch_fft_spectrum(const float* K, int k, int My, int Mx, void* work, void* spec, cudaStream_t st);
const float* conv_fft_core_kernel(const void* spec, int My, int Mx);
cudaError_t launch_conv_fft(const float* in, float* out, int n_img, int ny, int nx, int k, int My, int Mx,
                            const void* spec, float2* A, int accumulate, cudaStream_t st);
cudaError_t launch_conv_tma(const float* in, float* out, int n_img, int ny, int nx, const float* K, int k, int* err,
                            int sm_count, cudaStream_t st);

// Persistent batched convolution over device job descriptors; tiles are numbered by
// jobs[i].tile0 (jobs[n_jobs].tile0 = total) and handed out through *counter.
int conv_batch_grid(int sm_count, int kmax);
cudaError_t launch_conv_batch_meta(const BatchMeta* meta, int kmax, int grid, cudaStream_t st);
size_t conv_batch_smem(int kmax);

}  // namespace ls
