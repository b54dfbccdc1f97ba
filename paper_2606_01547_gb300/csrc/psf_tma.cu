// PSF step for batches of equal-size images (lens_sim_convolve) on sm_103a: a persistent,
// double-buffered kernel whose input tiles arrive by TMA (cp.async.bulk.tensor) into shared
// memory, completion tracked by an mbarrier.
//
// Each CTA computes tiles of 64 x 32 outputs (64 x 64 for k <= 7), or for images 65..128
// columns wide one tile across the whole row (one thread per 4 columns: no columns computed
// past the edge); its input box is the tile plus the k - 1 halo, with the left edge rounded
// down to a 16-byte boundary (TMA needs an aligned x) and
// out-of-image elements zero-filled by the TMA unit, which is exactly the zero padding of the
// 'same' convolution.  While one tile is computed the next is in flight.  A thread owns 2x4
// outputs: per kernel row it reads float4 windows of the two input rows it needs, so shared
// memory serves one float4 per ~3 FMAs, and it writes its outputs as float4.  The tap order
// (kernel row outer, column inner) is that of the generic kernel, so the two agree bitwise.
// Every mbarrier wait is bounded (1 s of %globaltimer); on expiry the CTA raises a flag in
// host-mapped memory, waits (bounded) for its copies in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "kernels.h"

namespace ls {

namespace {

constexpr int kThreads = 256;  // at most; 16 x 16 threads by default, each 4 columns x rows_per_thread(K) rows
constexpr unsigned long long kWaitNs = 1000000000ull;

// Small kernels (k <= 7, the HBM-bound regime) use 4 output rows per thread (64x64 tiles) with the
// weights in registers; larger kernels (FP32-bound) use 2 rows (64x32 tiles).
constexpr int rows_per_thread(int K) { return K <= 7 ? 4 : 2; }
constexpr int cpad(int K) { return ((K - 1) / 2 + 3) / 4 * 4; }   // left halo rounded up to 4
constexpr int coff(int K) { return cpad(K) - (K - 1) / 2; }        // tile column of the first tap

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for one phase of an mbarrier.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > kWaitNs) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

struct TmaConvArgs {
  float* out;
  const float* K;
  int nx, ny, n_img, tiles_x, tiles_y;
  int tx_n;     // threads across a tile (4 output columns each)
  int tw, th;   // tile width and height in outputs
  int bw, bh;   // input box (shared-memory tile) width and height
  int tile_fl;  // floats per shared-memory tile buffer (a 128-byte multiple)
  int* err;     // host-mapped flag, raised when a bounded wait expires
};

// out[2x? rows][4 cols] of one thread from the tile in shared memory.  Small K: every input row
// the thread needs is read once (float4 window) and applied to each output row it touches, with
// the weights in registers; large K: per kernel row, the two input rows, weights row hoisted.
template <int K>
__device__ __forceinline__ void conv_tile_compute(const float* __restrict__ T, const float* __restrict__ sK,
                                                  const float (&kreg)[K <= 7 ? K * K : 1], int tx, int ty, int BW,
                                                  float (&acc)[rows_per_thread(K)][4]) {
  constexpr int R = rows_per_thread(K), OFF = coff(K);
  constexpr int NV = (OFF + 4 + K - 1 + 3) / 4;  // float4 per window row
#pragma unroll
  for (int rr = 0; rr < R; ++rr)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[rr][c] = 0.f;
  if constexpr (K <= 7) {
#pragma unroll
    for (int t = 0; t < R + K - 1; ++t) {
      const float4* row = reinterpret_cast<const float4*>(T + (R * ty + t) * BW + 4 * tx);
      float w[4 * NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float4 f = row[v];
        w[4 * v] = f.x;
        w[4 * v + 1] = f.y;
        w[4 * v + 2] = f.z;
        w[4 * v + 3] = f.w;
      }
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const int a = t - rr;
        if (a < 0 || a >= K) continue;
#pragma unroll
        for (int b = 0; b < K; ++b)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[rr][c] = fmaf(kreg[a * K + b], w[OFF + c + b], acc[rr][c]);
      }
    }
  } else {
#pragma unroll 1
    for (int a = 0; a < K; ++a) {
      float kr[K];
#pragma unroll
      for (int b = 0; b < K; ++b) kr[b] = sK[a * K + b];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const float4* row = reinterpret_cast<const float4*>(T + (R * ty + rr + a) * BW + 4 * tx);
        float w[4 * NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float4 f = row[v];
          w[4 * v] = f.x;
          w[4 * v + 1] = f.y;
          w[4 * v + 2] = f.z;
          w[4 * v + 3] = f.w;
        }
#pragma unroll
        for (int b = 0; b < K; ++b)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[rr][c] = fmaf(kr[b], w[OFF + c + b], acc[rr][c]);
      }
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads) conv_tma_kernel(const __grid_constant__ CUtensorMap tin,
                                                           const TmaConvArgs A) {
  constexpr int C = (K - 1) / 2, R = rows_per_thread(K);
  const int TW = A.tw, TH = A.th;
  const unsigned kBytes = (unsigned)(A.bw * A.bh) * sizeof(float);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* tile0 = (float*)smem_raw;
  float* tile1 = tile0 + A.tile_fl;
  float* sK = tile1 + A.tile_fl;
  __shared__ __align__(8) unsigned long long bars[2];

  const int tid = threadIdx.x, tx = tid % A.tx_n, ty = tid / A.tx_n;
  for (int q = tid; q < K * K; q += blockDim.x) sK[q] = A.K[K * K - 1 - q];  // flipped: out = sum sK . window
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  float kreg[K <= 7 ? K * K : 1];
  if constexpr (K <= 7) {
#pragma unroll
    for (int q = 0; q < K * K; ++q) kreg[q] = sK[q];
  } else {
    kreg[0] = 0.f;
  }

  const int per_img = A.tiles_x * A.tiles_y;
  const long long total = (long long)per_img * A.n_img;
  auto issue = [&](long long t, int s) {
    const int z = (int)(t / per_img);
    const int r = (int)(t - (long long)z * per_img);
    const int i0 = (r / A.tiles_x) * TH, j0 = (r % A.tiles_x) * TW;
    mbar_expect_tx(&bars[s], kBytes);
    tma_load_3d(s ? tile1 : tile0, &tin, j0 - cpad(K), i0 - C, z, &bars[s]);
  };
  if (tid == 0 && (long long)blockIdx.x < total) issue(blockIdx.x, 0);

  int it = 0;
  for (long long t = blockIdx.x; t < total; t += gridDim.x, ++it) {
    const int s = it & 1;
    const long long tn = t + gridDim.x;
    if (tid == 0 && tn < total) issue(tn, s ^ 1);
    const bool ok = mbar_wait_bounded(&bars[s], (unsigned)((it >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        *A.err = 1;
        __threadfence_system();
        mbar_wait_bounded(&bars[s], (unsigned)((it >> 1) & 1));
        if (tn < total) mbar_wait_bounded(&bars[s ^ 1], (unsigned)(((it + 1) >> 1) & 1));
      }
      __syncthreads();
      return;
    }
    const int z = (int)(t / per_img);
    const int r = (int)(t - (long long)z * per_img);
    const int i0 = (r / A.tiles_x) * TH, j0 = (r % A.tiles_x) * TW;
    float acc[R][4];
    conv_tile_compute<K>(s ? tile1 : tile0, sK, kreg, tx, ty, A.bw, acc);
    const int j = j0 + 4 * tx;
    if (j < A.nx) {
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const int i = i0 + R * ty + rr;
        if (i < A.ny)
          *reinterpret_cast<float4*>(A.out + ((size_t)z * A.ny + i) * A.nx + j) =
              make_float4(acc[rr][0], acc[rr][1], acc[rr][2], acc[rr][3]);
      }
    }
    __syncthreads();  // the buffer is refilled two tiles later
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  });
  return fn;
}

template <int K>
cudaError_t launch_k(const float* in, float* out, int n_img, int ny, int nx, const float* Kw, int* err, int sm_count,
                     cudaStream_t st) {
  auto enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  constexpr int R = rows_per_thread(K);
  TmaConvArgs A;
  // tile shape: 16 x 16 threads (64-column tiles), or for rows of 65..128 columns one thread per
  // 4 columns across the whole row (nx % 4 == 0 here) and as many thread rows as fit 256 threads
  A.tx_n = 16;
  int ty_n = 16;
  if (nx > 64 && nx <= 128) {
    A.tx_n = nx / 4;
    ty_n = kThreads / A.tx_n;
  }
  A.tw = 4 * A.tx_n;
  A.th = ty_n * R;
  A.bw = (coff(K) + A.tw + K - 1 + 3) / 4 * 4;
  A.bh = A.th + K - 1;
  A.tile_fl = (A.bw * A.bh + 31) / 32 * 32;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)n_img};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)nx * ny * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)A.bw, (cuuint32_t)A.bh, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)in, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float) * ((size_t)2 * A.tile_fl + (size_t)K * K);
  const int threads = A.tx_n * ty_n;
  // an attribute of the kernel on the current device: set before every launch that needs it
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(conv_tma_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_tma_kernel<K>, threads, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  A.out = out;
  A.K = Kw;
  A.nx = nx;
  A.ny = ny;
  A.n_img = n_img;
  A.tiles_x = (nx + A.tw - 1) / A.tw;
  A.tiles_y = (ny + A.th - 1) / A.th;
  A.err = err;
  const long long total = (long long)A.tiles_x * A.tiles_y * n_img;
  const int grid = (int)std::min<long long>(total, (long long)sm_count * per_sm);
  conv_tma_kernel<K><<<grid, threads, smem, st>>>(map, A);
  return cudaGetLastError();
}

}  // namespace

bool conv_tma_supported(const float* in, const float* out, int ny, int nx, int k) {
  (void)ny;
  return (k % 2) == 1 && k >= 1 && k <= 31 && (nx % 4) == 0 && ((uintptr_t)in % 16) == 0 &&
         ((uintptr_t)out % 16) == 0 && encode_fn() != nullptr;
}

cudaError_t launch_conv_tma(const float* in, float* out, int n_img, int ny, int nx, const float* K, int k, int* err,
                            int sm_count, cudaStream_t st) {
  switch (k) {
    case 1: return launch_k<1>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 3: return launch_k<3>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 5: return launch_k<5>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 7: return launch_k<7>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 9: return launch_k<9>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 11: return launch_k<11>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 13: return launch_k<13>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 15: return launch_k<15>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 17: return launch_k<17>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 19: return launch_k<19>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 21: return launch_k<21>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 23: return launch_k<23>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 25: return launch_k<25>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 27: return launch_k<27>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 29: return launch_k<29>(in, out, n_img, ny, nx, K, err, sm_count, st);
    case 31: return launch_k<31>(in, out, n_img, ny, nx, K, err, sm_count, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ls
