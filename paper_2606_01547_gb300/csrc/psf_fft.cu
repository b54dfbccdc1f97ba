// PSF step by FFT for large kernels (image simulation step 3, the paper's FFT convolution).
//
// 'same'-size zero-padded true convolution out[i][j] = sum_{a,b} K[a][b] in[i + c - a][j + c - b],
// c = (k-1)/2, as a circular convolution on an My x Mx grid (powers of two, My >= ny + c,
// Mx >= nx + c: the rows and columns the crop keeps, [c, c + n), never receive wrapped terms):
//   1. forward FFT of each image row, zero-padded to Mx           (rows >= ny are zero: skipped)
//   2. per block of kCols columns: forward column FFT, product with the kernel's spectrum,
//      inverse column FFT; only the rows [c, c + ny) are written
//   3. inverse FFT of each kept row, crop of the columns [c, c + nx), scale 1/(Mx My)
// The kernel's spectrum comes from steps 1-2 run on the k x k kernel (spectrum mode).
//
// Radix-2 transforms in shared memory: the forward transform is decimation in time (input in
// bit-reversed order, output natural), the inverse decimation in frequency (input natural,
// output bit-reversed), so no separate permutation pass is needed; each CTA computes its
// twiddles exp(-2 pi i m / M) with sincospif.  All arithmetic is FP32 in a fixed order.
#include "kernels.h"

namespace ls {

namespace {

constexpr int kFftThreads = 256;
constexpr int kCols = 8;            // columns per CTA in the column pass (one 64 B row segment)
constexpr int kFftMaxLog2 = 10;     // M <= 1024

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ int brev(int v, int lg) { return (int)(__brev((unsigned)v) >> (32 - lg)); }

__device__ __forceinline__ void make_twiddles(float2* tw, int M) {
  for (int m = threadIdx.x; m < M / 2; m += blockDim.x) {
    float sn, cs;
    sincospif(-2.f * (float)m / (float)M, &sn, &cs);
    tw[m] = make_float2(cs, sn);
  }
}

// `batch` interleaved transforms of length n (element e of transform b at s[e * batch + b]).
// Forward, decimation in time: bit-reversed input, natural output.
__device__ void fft_dit(float2* s, int n, int batch, const float2* tw) {
  for (int len = 2, lg = 1; len <= n; len <<= 1, ++lg) {
    const int half = len >> 1, step = n / len;
    for (int t = threadIdx.x; t < (n >> 1) * batch; t += blockDim.x) {
      const int b = t % batch, bt = t / batch;
      const int pos = bt & (half - 1), grp = bt >> (lg - 1);
      const int ia = (grp * len + pos) * batch + b, ib = ia + half * batch;
      const float2 u = s[ia], v = cmul(s[ib], tw[pos * step]);
      s[ia] = cadd(u, v);
      s[ib] = csub(u, v);
    }
    __syncthreads();
  }
}

// Inverse (unscaled), decimation in frequency: natural input, bit-reversed output.
__device__ void ifft_dif(float2* s, int n, int batch, const float2* tw) {
  for (int len = n, lg = 0; len >= 2; len >>= 1) {
    (void)lg;
    const int half = len >> 1, step = n / len;
    for (int t = threadIdx.x; t < (n >> 1) * batch; t += blockDim.x) {
      const int b = t % batch, bt = t / batch;
      const int pos = bt % half, grp = bt / half;
      const int ia = (grp * len + pos) * batch + b, ib = ia + half * batch;
      const float2 u = s[ia], v = s[ib];
      s[ia] = cadd(u, v);
      s[ib] = cmulc(csub(u, v), tw[pos * step]);
    }
    __syncthreads();
  }
}

// Step 1: forward FFT of rows [0, ny) of each image (real, zero-padded to Mx) into A[img][row][Mx].
__global__ void __launch_bounds__(kFftThreads)
fft_rows_fwd_kernel(const float* __restrict__ in, int ny, int nx, int Mx, int lgx, float2* __restrict__ A) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* s = sm + Mx / 2;
  const int row = blockIdx.x;
  const size_t img = blockIdx.y;
  make_twiddles(tw, Mx);
  const float* src = in + (img * ny + row) * (size_t)nx;
  for (int j = threadIdx.x; j < Mx; j += blockDim.x) s[brev(j, lgx)] = make_float2(j < nx ? src[j] : 0.f, 0.f);
  __syncthreads();
  fft_dit(s, Mx, 1, tw);
  float2* dst = A + (img * ny + row) * (size_t)Mx;
  for (int j = threadIdx.x; j < Mx; j += blockDim.x) dst[j] = s[j];
}

// Step 2: column transforms of kCols columns.  spectrum = 1: forward only, all My rows of the
// result (natural order) to out[My][Mx].  spectrum = 0: forward, product with Kf, inverse; rows
// [row0, row0 + nrow) to out[img][nrow][Mx].
__global__ void __launch_bounds__(kFftThreads)
fft_cols_kernel(const float2* __restrict__ A, int ny, int Mx, int My, int lgy, const float2* __restrict__ Kf,
                int spectrum, int row0, int nrow, float2* __restrict__ out) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* s = sm + My / 2;
  const int j0 = blockIdx.x * kCols;
  const size_t img = blockIdx.y;
  make_twiddles(tw, My);
  const float2* src = A + img * ny * (size_t)Mx;
  for (int t = threadIdx.x; t < My * kCols; t += blockDim.x) {
    const int r = t / kCols, b = t - r * kCols;
    s[brev(r, lgy) * kCols + b] = r < ny ? src[(size_t)r * Mx + j0 + b] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_dit(s, My, kCols, tw);
  if (spectrum) {
    for (int t = threadIdx.x; t < My * kCols; t += blockDim.x) {
      const int r = t / kCols, b = t - r * kCols;
      out[(size_t)r * Mx + j0 + b] = s[t];
    }
    return;
  }
  for (int t = threadIdx.x; t < My * kCols; t += blockDim.x) {
    const int r = t / kCols, b = t - r * kCols;
    s[t] = cmul(s[t], Kf[(size_t)r * Mx + j0 + b]);
  }
  __syncthreads();
  ifft_dif(s, My, kCols, tw);
  float2* dst = out + img * nrow * (size_t)Mx;
  for (int t = threadIdx.x; t < nrow * kCols; t += blockDim.x) {
    const int r = t / kCols, b = t - r * kCols;
    dst[(size_t)r * Mx + j0 + b] = s[brev(row0 + r, lgy) * kCols + b];
  }
}

// Step 3: inverse FFT of each kept row, crop of columns [col0, col0 + nx), scale.
__global__ void __launch_bounds__(kFftThreads)
ifft_rows_crop_kernel(const float2* __restrict__ B, int ny, int nx, int Mx, int lgx, int col0, float scale,
                      float* __restrict__ out) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* s = sm + Mx / 2;
  const int row = blockIdx.x;
  const size_t img = blockIdx.y;
  make_twiddles(tw, Mx);
  const float2* src = B + (img * ny + row) * (size_t)Mx;
  for (int j = threadIdx.x; j < Mx; j += blockDim.x) s[j] = src[j];
  __syncthreads();
  ifft_dif(s, Mx, 1, tw);
  float* dst = out + (img * ny + row) * (size_t)nx;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) dst[j] = s[brev(col0 + j, lgx)].x * scale;
}

int log2_exact(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

cudaError_t set_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

bool conv_fft_sizes(int ny, int nx, int k, int* My, int* Mx) {
  const int c = (k - 1) / 2;
  int my = 2, mx = kCols;
  while (my < ny + c) my <<= 1;
  while (mx < nx + c) mx <<= 1;
  *My = my;
  *Mx = mx;
  return my <= (1 << kFftMaxLog2) && mx <= (1 << kFftMaxLog2);
}

size_t conv_fft_bytes_per_image(int ny, int Mx) { return 2 * sizeof(float2) * (size_t)ny * Mx; }

cudaError_t launch_fft_spectrum(const float* K, int k, int My, int Mx, float2* work, float2* Kf, cudaStream_t st) {
  const int lgx = log2_exact(Mx), lgy = log2_exact(My);
  const size_t smx = sizeof(float2) * (Mx / 2 + Mx), smy = sizeof(float2) * (My / 2 + (size_t)My * kCols);
  cudaError_t e = set_smem((const void*)fft_cols_kernel, smy);
  if (e != cudaSuccess) return e;
  fft_rows_fwd_kernel<<<dim3(k, 1), kFftThreads, smx, st>>>(K, k, k, Mx, lgx, work);
  fft_cols_kernel<<<dim3(Mx / kCols, 1), kFftThreads, smy, st>>>(work, k, Mx, My, lgy, nullptr, 1, 0, 0, Kf);
  return cudaGetLastError();
}

cudaError_t launch_conv_fft(const float* in, float* out, int n_img, int ny, int nx, int k, int My, int Mx,
                            const float2* Kf, float2* A, float2* B, cudaStream_t st) {
  if (n_img <= 0) return cudaSuccess;
  const int lgx = log2_exact(Mx), lgy = log2_exact(My), c = (k - 1) / 2;
  const size_t smx = sizeof(float2) * (Mx / 2 + Mx), smy = sizeof(float2) * (My / 2 + (size_t)My * kCols);
  cudaError_t e = set_smem((const void*)fft_cols_kernel, smy);
  if (e != cudaSuccess) return e;
  fft_rows_fwd_kernel<<<dim3(ny, n_img), kFftThreads, smx, st>>>(in, ny, nx, Mx, lgx, A);
  fft_cols_kernel<<<dim3(Mx / kCols, n_img), kFftThreads, smy, st>>>(A, ny, Mx, My, lgy, Kf, 0, c, ny, B);
  ifft_rows_crop_kernel<<<dim3(ny, n_img), kFftThreads, smx, st>>>(B, ny, nx, Mx, lgx, c,
                                                                   1.f / ((float)Mx * (float)My), out);
  return cudaGetLastError();
}

}  // namespace ls
