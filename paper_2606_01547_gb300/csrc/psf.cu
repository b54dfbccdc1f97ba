// PSF step (image simulation step 3): zero-padded 'same'-size direct convolution with an odd
// k x k kernel, tiled through shared memory.  flip = 1 is the convolution
//   out[i][j] = sum_{a,b} K[a][b] in[i + c - a][j + c - b],  c = (k-1)/2,
// flip = 0 the correlation sum_{a,b} K[a][b] in[i - c + a][j - c + b], its adjoint.
// A CTA computes a 32x32 output tile (32x8 threads, 4 rows each) from a (32+k-1)^2 input tile.
#include "kernels.h"

namespace ls {

constexpr int kConvT = 32;
constexpr int kConvRows = 8;

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
#pragma unroll
  for (int q = 0; q < kConvT / kConvRows; ++q) acc[q] = 0.f;
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
  static thread_local size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  dim3 grid((nx + kConvT - 1) / kConvT, (ny + kConvT - 1) / kConvT, n_img);
  dim3 block(kConvT, kConvRows);
  conv_kernel<<<grid, block, smem, st>>>(in, out, ny, nx, K, k, flip);
  return cudaGetLastError();
}

}  // namespace ls
