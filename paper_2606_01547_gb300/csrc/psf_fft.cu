// PSF step by FFT for large kernels (image simulation step 3, the paper's FFT convolution).
//
// 'same'-size zero-padded true convolution out[i][j] = sum_{a,b} K[a][b] in[i + c - a][j + c - b],
// c = (k-1)/2, as a circular convolution on an My x Mx grid (powers of two, My >= ny + c,
// Mx >= nx + c: the rows and columns the crop keeps, [c, c + n), never receive wrapped terms).
// The image is real, so its spectrum is Hermitian and half of it (H = Mx/2 + 1 columns) suffices:
//   1. rows: two real rows a, b per complex FFT of z = a + i b, split into their half spectra
//      A_k = (Z_k + conj Z_{-k})/2, B_k = (Z_k - conj Z_{-k})/(2i), k = 0 .. Mx/2, stored as
//      an ny x H array;
//   2. columns: per column of that array, forward FFT (rows >= ny are zero), product with the
//      kernel's spectrum, inverse FFT; the rows [c, c + ny) are written back in place;
//   3. rows: two rows' half spectra recombined into one complex inverse FFT of A + i B (the
//      negative frequencies from conjugates), whose real and imaginary parts, columns
//      [c, c + nx), scaled by 1/(Mx My), are the two output rows.
// The kernel's spectrum comes from steps 1 and 2 run on the zero-padded k x k kernel.
//
// Transforms of length M = N1 N2 (N1 = 2^ceil(L/2), N2 = 2^floor(L/2), L = log2 M) run in the
// four-step form on a group of N1 lanes of one warp: N2 DFTs of length N1 in registers, the
// twiddles W_M^(n2 k1), one exchange through shared memory, N1 DFTs of length N2 in registers,
// in place in a padded buffer; the register DFTs are radix-2 decimation in time with the
// permutation done by renaming.  The twiddles are computed in FP64 on the host and rounded
// once.  Inverse transforms are conj(FFT(conj(x))).
//
// Core and wings: for kernels from LENS_CONV_FFT_MIN_K on, the central kFftCore x kFftCore taps
// are convolved directly (by the caller) and the FFT carries only the rest of the kernel, whose
// amplitude is a small part of a centrally concentrated PSF's: the FFT's rounding error, of order
// eps log2(M) times the kernel's and image's L2 norms, then shrinks with it.
#include <cmath>
#include <mutex>

#include "kernels.h"

namespace ls {

namespace {

constexpr int kFftThreads = 256;
constexpr int kFftMaxLog2 = 10;
constexpr int kFftMax = 1 << kFftMaxLog2;  // M <= 1024
constexpr int kFftCore = 7;                // taps convolved directly when the wings go by FFT

// Twiddles, computed in FP64 on the host and rounded once: g_fft_twr[j] = W_32^j (the register
// DFTs' W_LEN^q = W_32^(32 q / LEN)); for each length M = 2^L, the four-step twiddles
// W_M^(t k1) at g_fft_tw4[(M - 2) + k1 N2 + t] (k1 < N1, t < N2), laid out so that the N2 lanes of
// a group read consecutive entries.
constexpr int kTw4Total = 2 * kFftMax - 2;
__device__ float2 g_fft_twr[32];
__device__ float2 g_fft_tw4[kTw4Total];

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

__host__ __device__ constexpr int log2_int(int v) { return v <= 1 ? 0 : 1 + log2_int(v >> 1); }
__host__ __device__ constexpr int brev_bits(int v, int bits) {
  return bits == 0 ? 0 : (((v & 1) << (bits - 1)) | brev_bits(v >> 1, bits - 1));
}

// The in-register DFT's steps as template recursions, so that every index is a compile-time
// constant and v stays in registers: the bit-reversal permutation (element I), then the radix-2
// butterfly stages of span LEN = 2, 4, .., R.
template <int R, int I>
__device__ __forceinline__ void dft_permute(float2 (&v)[R]) {
  if constexpr (I < R) {
    constexpr int J = brev_bits(I, log2_int(R));
    if constexpr (J > I) {
      const float2 t = v[I];
      v[I] = v[J];
      v[J] = t;
    }
    dft_permute<R, I + 1>(v);
  }
}

template <int R, int LEN>
__device__ __forceinline__ void dft_stages(float2 (&v)[R], const float2* __restrict__ tw) {
  if constexpr (LEN <= R) {
#pragma unroll
    for (int i = 0; i < R; i += LEN) {
#pragma unroll
      for (int q = 0; q < LEN / 2; ++q) {
        const float2 a = v[i + q];
        const float2 b = q == 0 ? v[i + q + LEN / 2] : cmul(v[i + q + LEN / 2], tw[q * (32 / LEN)]);
        v[i + q] = cadd(a, b);
        v[i + q + LEN / 2] = csub(a, b);
      }
    }
    dft_stages<R, LEN * 2>(v, tw);
  }
}

// In-register DFT of length R (a power of two <= 32), natural order in and out: radix-2
// decimation in time on the bit-reversed elements.
template <int R>
__device__ __forceinline__ void dft_regs(float2 (&v)[R], const float2* __restrict__ tw) {
  dft_permute<R, 0>(v);
  dft_stages<R, 2>(v, tw);
}

// FFT of length M = N1 N2 of one group's buffer s (INV: the unscaled inverse), by the group's
// lane t in [0, N1).  s holds element m of the sequence at pad(m) = m + m / N2 (rows of N2
// elements with one slot of padding: N1 (N2 + 1) slots), in and out, so that both the column
// reads of the first step and the row reads of the second are free of bank conflicts; the
// transform runs in place.  twr: W_32^j; tw4: this length's four-step twiddles.  Every lane of
// the warp calls it (the groups of a warp work on their own buffers).
template <int N2>
__device__ __forceinline__ int pad_index(int m) {
  return m + m / N2;
}

template <int N1, int N2, bool INV>
__device__ __forceinline__ void fft_group(float2* s, int t, const float2* __restrict__ twr,
                                          const float2* __restrict__ tw4) {
  constexpr int YS = N2 + 1;
  static_assert(N1 >= N2 && N1 <= 32, "four-step split");
  if (t < N2) {
    float2 v[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const float2 a = s[n1 * YS + t];
      v[n1] = INV ? conj2(a) : a;
    }
    dft_regs<N1>(v, twr);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) s[k1 * YS + t] = k1 == 0 ? v[k1] : cmul(v[k1], tw4[k1 * N2 + t]);
  }
  __syncwarp();
  float2 u[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) u[n2] = s[t * YS + n2];
  __syncwarp();
  dft_regs<N2>(u, twr);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) s[pad_index<N2>(t + N1 * k2)] = INV ? conj2(u[k2]) : u[k2];
  __syncwarp();
}

template <int L>
struct FftShape {
  static constexpr int M = 1 << L;
  static constexpr int N2 = 1 << (L / 2);
  static constexpr int N1 = M / N2;
  static constexpr int G = 32 / N1;                                  // groups per warp
  static constexpr int kGroups = (kFftThreads / 32) * G;            // groups per CTA
  static constexpr int kStride = N1 * (N2 + 1) + 1;                 // float2 per group (odd: no conflicts)
  static constexpr int kTw = 32 + M;                                 // twiddle slots
  static constexpr size_t kSmem = sizeof(float2) * ((size_t)kTw + (size_t)kGroups * kStride);
};

template <int L>
__device__ __forceinline__ void load_twiddles(float2* tw) {
  constexpr int M = 1 << L;
  for (int j = threadIdx.x; j < 32 + M; j += blockDim.x) tw[j] = j < 32 ? g_fft_twr[j] : g_fft_tw4[(M - 2) + j - 32];
}

// Step 1: rows [0, ny) of each image (real, zero-padded to Mx = 2^L), two per transform, into
// their half spectra A[img][row][0 .. H).
template <int L>
__global__ void __launch_bounds__(kFftThreads)
fft_rows_fwd_kernel(const float* __restrict__ in, int ny, int nx, int n_img, float2* __restrict__ A) {
  using S = FftShape<L>;
  constexpr int M = S::M, N1 = S::N1, N2 = S::N2, H = M / 2 + 1;
  extern __shared__ float2 sm[];
  load_twiddles<L>(sm);
  __syncthreads();
  const float2* twr = sm;
  const float2* tw4 = sm + 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = lane % N1, group = warp * S::G + lane / N1;
  float2* s = sm + S::kTw + (size_t)group * S::kStride;
  const int pairs = (ny + 1) / 2;
  const long long total = (long long)pairs * n_img;
  const long long warps_total = (long long)gridDim.x * (kFftThreads / 32);
  for (long long wt = (long long)blockIdx.x * (kFftThreads / 32) + warp; wt * S::G < total; wt += warps_total) {
    const long long task = wt * S::G + lane / N1;
    const bool valid = task < total;
    const int img = valid ? (int)(task / pairs) : 0;
    const int r0 = valid ? 2 * (int)(task % pairs) : 0;
    const bool has1 = valid && r0 + 1 < ny;
    const float* a = in + ((size_t)img * ny + r0) * nx;
#pragma unroll 4
    for (int j = t; j < M; j += N1) {
      const float va = (valid && j < nx) ? a[j] : 0.f;
      const float vb = (has1 && j < nx) ? a[nx + j] : 0.f;
      s[pad_index<N2>(j)] = make_float2(va, vb);
    }
    __syncwarp();
    fft_group<N1, N2, false>(s, t, twr, tw4);
    if (valid) {
      float2* da = A + ((size_t)img * ny + r0) * H;
      for (int k = t; k < H; k += N1) {
        const float2 zk = s[pad_index<N2>(k)], zm = conj2(s[pad_index<N2>((M - k) & (M - 1))]);
        da[k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
        if (has1) da[H + k] = make_float2(0.5f * (zk.y - zm.y), -0.5f * (zk.x - zm.x));
      }
    }
    __syncwarp();
  }
}

// Step 2: column transforms of the half spectra.  spectrum = 1: forward only, all My rows to
// out[col][row] (the kernel spectrum, transposed so that each column is contiguous).
// spectrum = 0: forward, product with Kf[col][row], inverse; rows [c, c + ny) back into
// A[img][0 .. ny)[col] in place.  A CTA takes kGroups consecutive columns of one image.
template <int L>
__global__ void __launch_bounds__(kFftThreads)
fft_cols_kernel(float2* __restrict__ A, int ny, int H, int c, const float2* __restrict__ Kf, int spectrum,
                float2* __restrict__ out) {
  using S = FftShape<L>;
  constexpr int M = S::M, N1 = S::N1, N2 = S::N2, CB = S::kGroups;
  extern __shared__ float2 sm[];
  load_twiddles<L>(sm);
  const float2* twr = sm;
  const float2* tw4 = sm + 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = lane % N1, group = warp * S::G + lane / N1;
  const int col0 = blockIdx.x * CB;
  const size_t img = blockIdx.y;
  float2* cols = sm + S::kTw;  // column g at cols + g * kStride
  float2* src = A + img * (size_t)ny * H;
  for (int q = threadIdx.x; q < M * CB; q += blockDim.x) {
    const int r = q / CB, g = q - r * CB, col = col0 + g;
    cols[(size_t)g * S::kStride + pad_index<N2>(r)] =
        (r < ny && col < H) ? src[(size_t)r * H + col] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2* s = cols + (size_t)group * S::kStride;
  const int col = col0 + group;
  fft_group<N1, N2, false>(s, t, twr, tw4);
  if (spectrum) {
    if (col < H)
      for (int r = t; r < M; r += N1) out[(size_t)col * M + r] = s[pad_index<N2>(r)];
    return;
  }
  if (col < H) {
    const float2* kf = Kf + (size_t)col * M;
    for (int r = t; r < M; r += N1) s[pad_index<N2>(r)] = cmul(s[pad_index<N2>(r)], kf[r]);
  }
  __syncwarp();
  fft_group<N1, N2, true>(s, t, twr, tw4);
  __syncthreads();
  for (int q = threadIdx.x; q < ny * CB; q += blockDim.x) {
    const int r = q / CB, g = q - r * CB, cc = col0 + g;
    if (cc < H) src[(size_t)r * H + cc] = cols[(size_t)g * S::kStride + pad_index<N2>(r + c)];
  }
}

// Step 3: pairs of output rows from their half spectra, columns [c, c + nx), scaled; added to
// `out` when accumulate is set (the FFT then carries the kernel's wings beside a direct core).
template <int L>
__global__ void __launch_bounds__(kFftThreads)
fft_rows_inv_kernel(const float2* __restrict__ A, int ny, int nx, int n_img, int c, float scale, int accumulate,
                    float* __restrict__ out) {
  using S = FftShape<L>;
  constexpr int M = S::M, N1 = S::N1, N2 = S::N2, H = M / 2 + 1;
  extern __shared__ float2 sm[];
  load_twiddles<L>(sm);
  __syncthreads();
  const float2* twr = sm;
  const float2* tw4 = sm + 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = lane % N1, group = warp * S::G + lane / N1;
  float2* s = sm + S::kTw + (size_t)group * S::kStride;
  const int pairs = (ny + 1) / 2;
  const long long total = (long long)pairs * n_img;
  const long long warps_total = (long long)gridDim.x * (kFftThreads / 32);
  for (long long wt = (long long)blockIdx.x * (kFftThreads / 32) + warp; wt * S::G < total; wt += warps_total) {
    const long long task = wt * S::G + lane / N1;
    const bool valid = task < total;
    const int img = valid ? (int)(task / pairs) : 0;
    const int r0 = valid ? 2 * (int)(task % pairs) : 0;
    const bool has1 = valid && r0 + 1 < ny;
    const float2* a = A + ((size_t)img * ny + r0) * H;
#pragma unroll 4
    for (int k = t; k < H; k += N1) {
      const float2 ak = valid ? a[k] : make_float2(0.f, 0.f);
      const float2 bk = has1 ? a[H + k] : make_float2(0.f, 0.f);
      s[pad_index<N2>(k)] = make_float2(ak.x - bk.y, ak.y + bk.x);  // A_k + i B_k
      if (k > 0 && k < M / 2)                                        // conj A_k + i conj B_k
        s[pad_index<N2>(M - k)] = make_float2(ak.x + bk.y, bk.x - ak.y);
    }
    __syncwarp();
    fft_group<N1, N2, true>(s, t, twr, tw4);
    if (valid) {
      float* __restrict__ d0 = out + ((size_t)img * ny + r0) * nx;
      float* __restrict__ d1 = d0 + nx;
      if (accumulate) {
#pragma unroll 4
        for (int j = t; j < nx; j += N1) {
          const float2 z = s[pad_index<N2>(c + j)];
          const float o0 = d0[j], o1 = has1 ? d1[j] : 0.f;
          d0[j] = fmaf(z.x, scale, o0);
          if (has1) d1[j] = fmaf(z.y, scale, o1);
        }
      } else {
#pragma unroll 4
        for (int j = t; j < nx; j += N1) {
          const float2 z = s[pad_index<N2>(c + j)];
          d0[j] = z.x * scale;
          if (has1) d1[j] = z.y * scale;
        }
      }
    }
    __syncwarp();
  }
}

// Host twiddle tables (FP64, rounded once), copied to each device on first use.
std::mutex g_tw_mu;
bool g_tw_done[64] = {};

cudaError_t ensure_twiddles() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_tw_mu);
  if (g_tw_done[dev]) return cudaSuccess;
  static float2 host_twr[32];
  static float2 host_tw4[kTw4Total];
  static bool host_ready = false;
  if (!host_ready) {
    const double pi = 3.14159265358979323846264338327950288;
    for (int j = 0; j < 32; ++j) {
      const double a = -2.0 * pi * (double)j / 32.0;
      host_twr[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    for (int L = 1; L <= kFftMaxLog2; ++L) {
      const int M = 1 << L, N2 = 1 << (L / 2), N1 = M / N2;
      for (int k1 = 0; k1 < N1; ++k1)
        for (int t = 0; t < N2; ++t) {
          const double a = -2.0 * pi * (double)(t * k1) / (double)M;
          host_tw4[(M - 2) + k1 * N2 + t] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    }
    host_ready = true;
  }
  e = cudaMemcpyToSymbol(g_fft_twr, host_twr, sizeof(host_twr));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_fft_tw4, host_tw4, sizeof(host_tw4));
  if (e == cudaSuccess) g_tw_done[dev] = true;
  return e;
}

template <class F>
cudaError_t allow_smem(F* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int grid_for(long long tasks, int groups_per_cta) {
  const long long ctas = (tasks + groups_per_cta - 1) / groups_per_cta;
  return (int)std::min<long long>(std::max<long long>(ctas, 1), 4096);
}

template <int L>
cudaError_t rows_fwd(const float* in, int ny, int nx, int n_img, float2* A, cudaStream_t st) {
  using S = FftShape<L>;
  cudaError_t e = allow_smem(fft_rows_fwd_kernel<L>, S::kSmem);
  if (e != cudaSuccess) return e;
  fft_rows_fwd_kernel<L><<<grid_for((long long)((ny + 1) / 2) * n_img, S::kGroups), kFftThreads, S::kSmem, st>>>(
      in, ny, nx, n_img, A);
  return cudaGetLastError();
}

template <int L>
cudaError_t cols(float2* A, int ny, int H, int c, int n_img, const float2* Kf, int spectrum, float2* out,
                 cudaStream_t st) {
  using S = FftShape<L>;
  cudaError_t e = allow_smem(fft_cols_kernel<L>, S::kSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((H + S::kGroups - 1) / S::kGroups, n_img);
  fft_cols_kernel<L><<<grid, kFftThreads, S::kSmem, st>>>(A, ny, H, c, Kf, spectrum, out);
  return cudaGetLastError();
}

template <int L>
cudaError_t rows_inv(const float2* A, int ny, int nx, int n_img, int c, float scale, int accumulate, float* out,
                     cudaStream_t st) {
  using S = FftShape<L>;
  cudaError_t e = allow_smem(fft_rows_inv_kernel<L>, S::kSmem);
  if (e != cudaSuccess) return e;
  fft_rows_inv_kernel<L><<<grid_for((long long)((ny + 1) / 2) * n_img, S::kGroups), kFftThreads, S::kSmem, st>>>(
      A, ny, nx, n_img, c, scale, accumulate, out);
  return cudaGetLastError();
}

#define LS_FFT_DISPATCH(lg, call)   \
  switch (lg) {                     \
    case 1: { constexpr int L = 1; return call; }  \
    case 2: { constexpr int L = 2; return call; }  \
    case 3: { constexpr int L = 3; return call; }  \
    case 4: { constexpr int L = 4; return call; }  \
    case 5: { constexpr int L = 5; return call; }  \
    case 6: { constexpr int L = 6; return call; }  \
    case 7: { constexpr int L = 7; return call; }  \
    case 8: { constexpr int L = 8; return call; }  \
    case 9: { constexpr int L = 9; return call; }  \
    case 10: { constexpr int L = 10; return call; } \
    default: return cudaErrorInvalidValue;         \
  }

cudaError_t rows_fwd_any(int lg, const float* in, int ny, int nx, int n_img, float2* A, cudaStream_t st) {
  LS_FFT_DISPATCH(lg, (rows_fwd<L>(in, ny, nx, n_img, A, st)))
}
cudaError_t cols_any(int lg, float2* A, int ny, int H, int c, int n_img, const float2* Kf, int spectrum,
                     float2* out, cudaStream_t st) {
  LS_FFT_DISPATCH(lg, (cols<L>(A, ny, H, c, n_img, Kf, spectrum, out, st)))
}
cudaError_t rows_inv_any(int lg, const float2* A, int ny, int nx, int n_img, int c, float scale, int accumulate,
                         float* out, cudaStream_t st) {
  LS_FFT_DISPATCH(lg, (rows_inv<L>(A, ny, nx, n_img, c, scale, accumulate, out, st)))
}
#undef LS_FFT_DISPATCH

int log2_exact(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// The kernel's wings: K with its central core x core taps set to zero (row-major k x k).
__global__ void wings_kernel(const float* __restrict__ K, int k, int core, float* __restrict__ W,
                             float* __restrict__ Kc) {
  const int c = (k - 1) / 2, h = (core - 1) / 2;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k * k; t += gridDim.x * blockDim.x) {
    const int a = t / k, b = t - a * k;
    const bool in_core = core > 0 && a >= c - h && a <= c + h && b >= c - h && b <= c + h;
    W[t] = in_core ? 0.f : K[t];
    if (in_core) Kc[(a - (c - h)) * core + (b - (c - h))] = K[t];
  }
}

}  // namespace

bool conv_fft_sizes(int ny, int nx, int k, int* My, int* Mx) {
  const int c = (k - 1) / 2;
  int my = 2, mx = 2;
  while (my < ny + c) my <<= 1;
  while (mx < nx + c) mx <<= 1;
  *My = my;
  *Mx = mx;
  return my <= kFftMax && mx <= kFftMax;
}

int conv_fft_core(int k) { return k >= LENS_CONV_FFT_MIN_K ? kFftCore : 0; }

size_t conv_fft_bytes_per_image(int ny, int Mx) { return sizeof(float2) * (size_t)ny * (Mx / 2 + 1); }

size_t conv_fft_spectrum_bytes(int My, int Mx, int k) {
  const int core = conv_fft_core(k);
  return sizeof(float2) * (size_t)(Mx / 2 + 1) * My + sizeof(float) * (size_t)core * core;
}

size_t conv_fft_spectrum_work_bytes(int Mx, int k) {
  return sizeof(float2) * (size_t)k * (Mx / 2 + 1) + sizeof(float) * (size_t)k * k;
}

cudaError_t launch_fft_spectrum(const float* K, int k, int My, int Mx, void* work, void* spec, cudaStream_t st) {
  cudaError_t e = ensure_twiddles();
  if (e != cudaSuccess) return e;
  const int H = Mx / 2 + 1, core = conv_fft_core(k);
  float2* Kf = (float2*)spec;
  float* Kc = (float*)(Kf + (size_t)H * My);
  float2* A = (float2*)work;
  float* W = (float*)(A + (size_t)k * H);
  const float* src = K;
  if (core > 0) {
    wings_kernel<<<(k * k + 255) / 256, 256, 0, st>>>(K, k, core, W, Kc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    src = W;
  }
  if ((e = rows_fwd_any(log2_exact(Mx), src, k, k, 1, A, st)) != cudaSuccess) return e;
  return cols_any(log2_exact(My), A, k, H, 0, 1, nullptr, 1, Kf, st);
}

const float* conv_fft_core_kernel(const void* spec, int My, int Mx) {
  return (const float*)((const float2*)spec + (size_t)(Mx / 2 + 1) * My);
}

cudaError_t launch_conv_fft(const float* in, float* out, int n_img, int ny, int nx, int k, int My, int Mx,
                            const void* spec, float2* A, int accumulate, cudaStream_t st) {
  if (n_img <= 0) return cudaSuccess;
  cudaError_t e = ensure_twiddles();
  if (e != cudaSuccess) return e;
  const int lgx = log2_exact(Mx), lgy = log2_exact(My), c = (k - 1) / 2, H = Mx / 2 + 1;
  if ((e = rows_fwd_any(lgx, in, ny, nx, n_img, A, st)) != cudaSuccess) return e;
  if ((e = cols_any(lgy, A, ny, H, c, n_img, (const float2*)spec, 0, nullptr, st)) != cudaSuccess) return e;
  return rows_inv_any(lgx, A, ny, nx, n_img, c, 1.f / ((float)Mx * (float)My), accumulate, out, st);
}

}  // namespace ls
