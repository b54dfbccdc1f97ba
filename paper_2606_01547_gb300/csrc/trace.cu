// Fused image-simulation kernel (image simulation steps 1 and 2 plus the supersample bin-down):
// every thread owns one pixel of an 8x4 tile and up to PTS of its s*s sub-pixel samples; the
// NW warps of a CTA split the subhalo list (an N-body-like all-pairs sum staged through
// shared memory), their partial deflections are reduced in a fixed warp order, then the
// main deflectors, the lens equation beta = theta - alpha, the Sersic source and the
// bin-down run on chip.  Traced coordinates never leave registers/shared memory; only the
// binned image is written.
#include <algorithm>

#include "kernels.h"

namespace ls {

constexpr int kTileW = 8;
constexpr int kTileH = 4;

__global__ void tnfw_prep_kernel(const float* __restrict__ soa, int n, int ld, float4* __restrict__ tab) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float4 a, b;
  tnfw_constants(soa[j], soa[ld + j], soa[2 * ld + j], soa[3 * ld + j], soa[4 * ld + j], a, b);
  tab[2 * j] = a;
  tab[2 * j + 1] = b;
}

cudaError_t launch_tnfw_prep(const float* soa, int n, int ld, float4* table, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  tnfw_prep_kernel<<<(n + 255) / 256, 256, 0, st>>>(soa, n, ld, table);
  return cudaGetLastError();
}

template <int PTS, int NW>
__global__ void __launch_bounds__(32 * NW) trace_image_kernel(const __grid_constant__ DevSystem sys) {
  __shared__ float4 s_sub[NW][32][2];
  __shared__ float2 s_part[NW][PTS][32];
  __shared__ float s_I[PTS][32];

  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int tiles_x = (sys.nx + kTileW - 1) / kTileW;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int j = tx * kTileW + (lane & (kTileW - 1));
  const int i = ty * kTileH + (lane / kTileW);
  const int s = sys.s, s2 = s * s;
  const int passes = (s2 + PTS - 1) / PTS;
  const int n = sys.n_sub;
  const int lo = (int)(((long long)n * w) / NW);
  const int hi = (int)(((long long)n * (w + 1)) / NW);
  const float4* __restrict__ tab = sys.sub;

  float pix = 0.f;
  for (int pass = 0; pass < passes; ++pass) {
    float px[PTS], py[PTS], ax[PTS], ay[PTS];
#pragma unroll
    for (int k = 0; k < PTS; ++k) {
      int pt = pass * PTS + k;
      if (pt >= s2) pt = 0;
      const int a = pt / s, b = pt - a * s;
      px[k] = grid_coord(sys.x0, j, sys.nx, b, s, sys.dpix);
      py[k] = grid_coord(sys.y0, i, sys.ny, a, s, sys.dpix);
      ax[k] = 0.f;
      ay[k] = 0.f;
    }
    // Subhalo sum over this warp's slice [lo, hi), 32 subhalos per shared-memory stage.
    for (int base = lo; base < hi; base += 32) {
      const int idx = base + lane;
      if (idx < hi) {
        s_sub[w][lane][0] = __ldg(tab + 2 * idx);
        s_sub[w][lane][1] = __ldg(tab + 2 * idx + 1);
      }
      __syncwarp();
      const int cnt = min(32, hi - base);
      for (int q = 0; q < cnt; ++q) {
        const float4 A = s_sub[w][q][0];
        const float4 B = s_sub[w][q][1];
#pragma unroll
        for (int k = 0; k < PTS; ++k) tnfw_pair(px[k], py[k], A, B, ax[k], ay[k]);
      }
      __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < PTS; ++k) s_part[w][k][lane] = make_float2(ax[k], ay[k]);
    __syncthreads();
    // Per sample: fixed-order reduction over warps, main deflectors, lens equation, source.
    for (int idx = threadIdx.x; idx < 32 * PTS; idx += 32 * NW) {
      const int k = idx >> 5, l = idx & 31;
      const int pt = pass * PTS + k;
      float I = 0.f;
      if (pt < s2) {
        float sx = 0.f, sy = 0.f;
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) {
          const float2 v = s_part[ww][k][l];
          sx += v.x;
          sy += v.y;
        }
        const int jj = tx * kTileW + (l & (kTileW - 1));
        const int ii = ty * kTileH + (l / kTileW);
        const int a = pt / s, b = pt - a * s;
        const float x = grid_coord(sys.x0, jj, sys.nx, b, s, sys.dpix);
        const float y = grid_coord(sys.y0, ii, sys.ny, a, s, sys.dpix);
        for (int d = 0; d < sys.n_defl; ++d) {
          float dax, day;
          alpha_profile(sys.defl[d], x, y, dax, day);
          sx += dax;
          sy += day;
        }
        I = source_light(sys.src_type, sys.src, x - sx, y - sy);
      }
      s_I[k][l] = I;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
      for (int k = 0; k < PTS; ++k) pix += s_I[k][lane];
    }
    __syncthreads();
  }
  if (w == 0 && i < sys.ny && j < sys.nx)
    sys.out[(size_t)i * sys.nx + j] = pix * (sys.dpix * sys.dpix / (float)s2);
}

TraceShape choose_trace_shape(int nx, int ny, int s, int n_sub, int sm_count) {
  TraceShape sh;
  sh.pts = (s == 1) ? 1 : (s == 2) ? 4 : (s == 3) ? 9 : 8;
  const long long tiles = (long long)((nx + kTileW - 1) / kTileW) * ((ny + kTileH - 1) / kTileH);
  if (n_sub < 64) {
    sh.nw = 1;
  } else {
    // aim for ~32 resident warps per SM across the tiles
    long long want = (long long)sm_count * 32;
    int nw = 1;
    while (nw < 8 && tiles * nw < want) nw *= 2;
    sh.nw = nw;
  }
  return sh;
}

template <int PTS>
static cudaError_t launch_trace_pts(const DevSystem& sys, int nw, int grid, cudaStream_t st) {
  switch (nw) {
    case 1: trace_image_kernel<PTS, 1><<<grid, 32, 0, st>>>(sys); break;
    case 2: trace_image_kernel<PTS, 2><<<grid, 64, 0, st>>>(sys); break;
    case 4: trace_image_kernel<PTS, 4><<<grid, 128, 0, st>>>(sys); break;
    default: trace_image_kernel<PTS, 8><<<grid, 256, 0, st>>>(sys); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_trace(const DevSystem& sys, TraceShape shape, cudaStream_t st) {
  const int grid = ((sys.nx + kTileW - 1) / kTileW) * ((sys.ny + kTileH - 1) / kTileH);
  switch (shape.pts) {
    case 1: return launch_trace_pts<1>(sys, shape.nw, grid, st);
    case 4: return launch_trace_pts<4>(sys, shape.nw, grid, st);
    case 9: return launch_trace_pts<9>(sys, shape.nw, grid, st);
    default: return launch_trace_pts<8>(sys, shape.nw, grid, st);
  }
}

// Ray-shooting at arbitrary points: one thread per point, per-warp staging of the subhalos.
__global__ void __launch_bounds__(256) deflection_kernel(const __grid_constant__ DevSystem sys,
                                                         const float* __restrict__ xs,
                                                         const float* __restrict__ ys, int n,
                                                         float* __restrict__ axs, float* __restrict__ ays) {
  __shared__ float4 s_sub[8][32][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int warp_first = blockIdx.x * blockDim.x + w * 32;
  if (warp_first >= n) return;
  const int idx = warp_first + lane;
  const bool valid = idx < n;
  const float px = valid ? xs[idx] : 0.f;
  const float py = valid ? ys[idx] : 0.f;
  float ax = 0.f, ay = 0.f;
  for (int base = 0; base < sys.n_sub; base += 32) {
    const int t = base + lane;
    if (t < sys.n_sub) {
      s_sub[w][lane][0] = __ldg(sys.sub + 2 * t);
      s_sub[w][lane][1] = __ldg(sys.sub + 2 * t + 1);
    }
    __syncwarp();
    const int cnt = min(32, sys.n_sub - base);
    for (int q = 0; q < cnt; ++q) tnfw_pair(px, py, s_sub[w][q][0], s_sub[w][q][1], ax, ay);
    __syncwarp();
  }
  for (int d = 0; d < sys.n_defl; ++d) {
    float dax, day;
    alpha_profile(sys.defl[d], px, py, dax, day);
    ax += dax;
    ay += day;
  }
  if (valid) {
    axs[idx] = ax;
    ays[idx] = ay;
  }
}

cudaError_t launch_deflection(const DevSystem& sys, const float* x, const float* y, int n, float* ax,
                              float* ay, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  deflection_kernel<<<(n + 255) / 256, 256, 0, st>>>(sys, x, y, n, ax, ay);
  return cudaGetLastError();
}

}  // namespace ls
