// PSF step (image simulation step 3): zero-padded 'same'-size direct convolution with an odd
// k x k kernel, tiled through shared memory.  flip = 1 is the convolution
//   out[i][j] = sum_{a,b} K[a][b] in[i + c - a][j + c - b],  c = (k-1)/2,
// flip = 0 the correlation sum_{a,b} K[a][b] in[i - c + a][j - c + b], its adjoint.
// A CTA computes a 32x32 output tile (32x8 threads, 4 rows each) from a (32+k-1)^2 input tile.
#include "kernels.h"

namespace ls {

constexpr int kConvT = 32;
constexpr int kConvRows = 8;
// From this kernel size on (above the TMA kernel's k <= 31) the direct sum is taken by rows.
constexpr int kConvRowSumMinK = 33;

// The tile sum of one thread's kConvT / kConvRows outputs, shared by the single-image and the
// batched kernels so that both sum in the same order (bitwise equal outputs).
__device__ __forceinline__ void conv_tile_sum(const float* sK, const float* sT, int tw, int k,
                                              float (&acc)[kConvT / kConvRows]) {
#pragma unroll
  for (int q = 0; q < kConvT / kConvRows; ++q) acc[q] = 0.f;
  if (k < kConvRowSumMinK) {
    // one running sum over the k^2 taps, in the order of the TMA kernel (bitwise equal to it)
    for (int a = 0; a < k; ++a) {
      for (int b = 0; b < k; ++b) {
        const float kv = sK[a * k + b];
#pragma unroll
        for (int q = 0; q < kConvT / kConvRows; ++q) {
          const int r = threadIdx.y + q * kConvRows;
          acc[q] = fmaf(kv, sT[(r + a) * tw + threadIdx.x + b], acc[q]);
        }
      }
    }
  } else {
    // large kernels: a partial sum per kernel row, then the sum of the rows.  One running sum
    // over k^2 = 18,225 taps (k = 135) drifts by ~sqrt(k^2) roundings, 1.6e-5 of the image
    // maximum on a lensed image; two levels keep it to ~2 sqrt(k).
    for (int a = 0; a < k; ++a) {
      float row[kConvT / kConvRows];
#pragma unroll
      for (int q = 0; q < kConvT / kConvRows; ++q) row[q] = 0.f;
      for (int b = 0; b < k; ++b) {
        const float kv = sK[a * k + b];
#pragma unroll
        for (int q = 0; q < kConvT / kConvRows; ++q) {
          const int r = threadIdx.y + q * kConvRows;
          row[q] = fmaf(kv, sT[(r + a) * tw + threadIdx.x + b], row[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < kConvT / kConvRows; ++q) acc[q] += row[q];
    }
  }
}

__global__ void __launch_bounds__(kConvT * kConvRows)
conv_kernel(const float* __restrict__ in, float* __restrict__ out, int ny, int nx,
            const float* __restrict__ K, int k, int flip) {
  extern __shared__ float smem[];
  const int tw = kConvT + k - 1;
  float* sK = smem;              // k*k (oriented so that out = sum sK[a][b] T[r+a][c+b])
  float* sT = smem + k * k;      // tw*tw input tile with halo
  const int c = (k - 1) / 2;
  const size_t img = (size_t)blockIdx.z * ny * nx;
  const int i0 = blockIdx.y * kConvT, j0 = blockIdx.x * kConvT;
  const int tid = threadIdx.y * kConvT + threadIdx.x;
  const int nthr = kConvT * kConvRows;
  for (int t = tid; t < k * k; t += nthr) sK[t] = flip ? K[k * k - 1 - t] : K[t];
  for (int t = tid; t < tw * tw; t += nthr) {
    const int r = t / tw, cc = t - r * tw;
    const int gi = i0 - c + r, gj = j0 - c + cc;
    sT[t] = (gi >= 0 && gi < ny && gj >= 0 && gj < nx) ? in[img + (size_t)gi * nx + gj] : 0.f;
  }
  __syncthreads();
  float acc[kConvT / kConvRows];
  conv_tile_sum(sK, sT, tw, k, acc);
#pragma unroll
  for (int q = 0; q < kConvT / kConvRows; ++q) {
    const int gi = i0 + threadIdx.y + q * kConvRows, gj = j0 + threadIdx.x;
    if (gi < ny && gj < nx) out[img + (size_t)gi * nx + gj] = acc[q];
  }
}

cudaError_t launch_conv(const float* in, float* out, int n_img, int ny, int nx, const float* K, int k,
                        int flip, cudaStream_t st) {
  if (n_img <= 0) return cudaSuccess;
  const int tw = kConvT + k - 1;
  const size_t smem = sizeof(float) * ((size_t)k * k + (size_t)tw * tw);
  // The opt-in is an attribute of the kernel on the current device, so it is set before every
  // launch that needs more than the default 48 KB (a cached flag would miss other devices).
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((nx + kConvT - 1) / kConvT, (ny + kConvT - 1) / kConvT, n_img);
  dim3 block(kConvT, kConvRows);
  conv_kernel<<<grid, block, smem, st>>>(in, out, ny, nx, K, k, flip);
  return cudaGetLastError();
}

}  // namespace ls

namespace ls {

size_t conv_batch_smem(int kmax) {
  const int tw = kConvT + kmax - 1;
  return sizeof(float) * ((size_t)kmax * kmax + (size_t)tw * tw);
}

// Persistent form over many images of different sizes and kernels (the batched PSF step).
__global__ void __launch_bounds__(kConvT * kConvRows)
conv_batch_kernel(BatchMeta* __restrict__ meta) {
  extern __shared__ float smem[];
  __shared__ int s_ticket;
  const ConvJob* __restrict__ jobs = meta->conv;
  const int n_jobs = meta->n_conv;
  unsigned int* counter = &meta->conv_counter;
  const int total = jobs[n_jobs].tile0;
  const int tid = threadIdx.y * kConvT + threadIdx.x;
  const int nthr = kConvT * kConvRows;
  for (;;) {
    if (tid == 0) s_ticket = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int u = s_ticket;
    __syncthreads();
    if (u >= total) return;
    int lo = 0, hi = n_jobs;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (jobs[mid].tile0 <= u) lo = mid; else hi = mid;
    }
    const ConvJob J = jobs[lo];
    const int t = u - J.tile0;
    const int tiles_x = (J.nx + kConvT - 1) / kConvT;
    const int i0 = (t / tiles_x) * kConvT, j0 = (t % tiles_x) * kConvT;
    const int k = J.k, c = (k - 1) / 2, tw = kConvT + k - 1;
    float* sK = smem;
    float* sT = smem + k * k;
    for (int q = tid; q < k * k; q += nthr) sK[q] = J.K[k * k - 1 - q];
    for (int q = tid; q < tw * tw; q += nthr) {
      const int r = q / tw, cc = q - r * tw;
      const int gi = i0 - c + r, gj = j0 - c + cc;
      sT[q] = (gi >= 0 && gi < J.ny && gj >= 0 && gj < J.nx) ? J.in[(size_t)gi * J.nx + gj] : 0.f;
    }
    __syncthreads();
    float acc[kConvT / kConvRows];
    conv_tile_sum(sK, sT, tw, k, acc);
#pragma unroll
    for (int q = 0; q < kConvT / kConvRows; ++q) {
      const int gi = i0 + threadIdx.y + q * kConvRows, gj = j0 + threadIdx.x;
      if (gi < J.ny && gj < J.nx) J.out[(size_t)gi * J.nx + gj] = acc[q];
    }
    __syncthreads();
  }
}

int conv_batch_grid(int sm_count, int kmax) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_batch_kernel, kConvT * kConvRows,
                                                    conv_batch_smem(kmax)) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return sm_count * per_sm;
}

cudaError_t launch_conv_batch_meta(const BatchMeta* meta, int kmax, int grid, cudaStream_t st) {
  const size_t smem = conv_batch_smem(kmax);
  if (smem > 48 * 1024) {  // per device, as in launch_conv
    cudaError_t e = cudaFuncSetAttribute(conv_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  conv_batch_kernel<<<grid, dim3(kConvT, kConvRows), smem, st>>>(const_cast<BatchMeta*>(meta));
  return cudaGetLastError();
}

}  // namespace ls
