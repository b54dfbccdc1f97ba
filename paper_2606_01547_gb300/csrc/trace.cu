// Fused image-simulation kernel (image simulation steps 1 and 2 plus the supersample bin-down).
//
// Work unit: 288 sub-pixel samples = 32 lanes x 9 samples, covering a pixel block whose shape
// depends on the supersampling factor s (24x12 pixels at s=1, 12x6 at s=2, 8x4 at s=3, ...), so
// every s keeps all lanes busy.  The NW warps of a CTA split the subhalo list of the unit (an
// N-body-like all-pairs sum staged through shared memory); their partial deflections are
// reduced in a fixed warp order, then the main deflectors, the lens equation
// beta = theta - alpha, the Sersic source and the bin-down run on chip.  Traced coordinates
// never leave registers and shared memory; only the binned image is written.
//
// Two launch forms share the unit body: one CTA per unit of a single system, and a persistent
// kernel that pulls units of many systems from a device-side queue (largest cost first).
#include <algorithm>

#include "kernels.h"

namespace ls {

__global__ void tnfw_prep_kernel(const float* __restrict__ soa, int n, int ld, float4* __restrict__ tab) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float4 v0, v1, v2, v3;
  tnfw_constants(soa[j], soa[ld + j], soa[2 * ld + j], soa[3 * ld + j], soa[4 * ld + j], v0, v1, v2, v3);
  float4* t = tab + (size_t)kSubStride * j;
  t[0] = v0;
  t[1] = v1;
  t[2] = v2;
  t[3] = v3;
}

cudaError_t launch_tnfw_prep(const float* soa, int n, int ld, float4* table, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  tnfw_prep_kernel<<<(n + 255) / 256, 256, 0, st>>>(soa, n, ld, table);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- unit geometry
__host__ __device__ inline void unit_shape(int s, int& bw, int& bh) {
  switch (s) {
    case 1: bw = 24; bh = 12; break;
    case 2: bw = 12; bh = 6; break;
    case 3: bw = 8; bh = 4; break;
    case 4: bw = 6; bh = 3; break;
    case 5: bw = 5; bh = 2; break;
    case 6: bw = 4; bh = 2; break;
    case 7: bw = 5; bh = 1; break;
    default: bw = 2; bh = 2; break;
  }
}

int unit_count(int nx, int ny, int s) {
  int bw, bh;
  unit_shape(s, bw, bh);
  return ((nx + bw - 1) / bw) * ((ny + bh - 1) / bh);
}

template <int NW>
struct TraceSmem {
  float4 sub[NW][32][kSubStride];
  float2 part[NW][kUnitPts][32];
  float I[kUnitPts * 32];
};

// One unit of one system.  All threads of the CTA call it; it ends with a CTA barrier.
template <int NW>
__device__ __forceinline__ void trace_unit(const DevSystem& sys, int blk, TraceSmem<NW>& sm) {
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int s = sys.s, s2 = s * s;
  int bw, bh;
  unit_shape(s, bw, bh);
  const int nbx = (sys.nx + bw - 1) / bw;
  const int bx = blk % nbx, by = blk / nbx;
  const int nsamp = bw * bh * s2;
  const int n = sys.n_sub;
  const int lo = (int)(((long long)n * w) / NW);
  const int hi = (int)(((long long)n * (w + 1)) / NW);
  const float4* __restrict__ tab = sys.sub;

  float px[kUnitPts], py[kUnitPts], ax[kUnitPts], ay[kUnitPts];
#pragma unroll
  for (int k = 0; k < kUnitPts; ++k) {
    int q = lane * kUnitPts + k;
    if (q >= nsamp) q = 0;
    const int p = q / s2, sub = q - p * s2;
    const int a = sub / s, b = sub - a * s;
    const int i = by * bh + p / bw, j = bx * bw + p % bw;
    px[k] = grid_coord(sys.x0, j, sys.nx, b, s, sys.dpix);
    py[k] = grid_coord(sys.y0, i, sys.ny, a, s, sys.dpix);
    ax[k] = 0.f;
    ay[k] = 0.f;
  }
  // Subhalo sum over this warp's slice [lo, hi), 32 subhalos per shared-memory stage.  Per
  // subhalo the warp votes: if no sample of any lane is inside the far-field radius, every
  // pair takes the straight-line series path; otherwise each sample picks its own form.
  for (int base = lo; base < hi; base += 32) {
    const int idx = base + lane;
    if (idx < hi) {
#pragma unroll
      for (int c = 0; c < kSubStride; ++c) sm.sub[w][lane][c] = __ldg(tab + (size_t)kSubStride * idx + c);
    }
    __syncwarp();
    const int cnt = min(32, hi - base);
    for (int q = 0; q < cnt; ++q) {
      const float4 v0 = sm.sub[w][q][0];
      const float4 v1 = sm.sub[w][q][1];
      const float4 v2 = sm.sub[w][q][2];
      const float4 v3 = sm.sub[w][q][3];
      float dx[kUnitPts], dy[kUnitPts], x2[kUnitPts];
      bool inner = false;
#pragma unroll
      for (int k = 0; k < kUnitPts; ++k) {
        dx[k] = px[k] - v0.x;
        dy[k] = py[k] - v0.y;
        x2[k] = fmaf(dx[k], dx[k], dy[k] * dy[k]) * v0.z;
        inner |= x2[k] < v0.w;
      }
      if (!__any_sync(0xffffffffu, inner)) {
#pragma unroll
        for (int k = 0; k < kUnitPts; ++k) {
          const float g = tnfw_series(x2[k], v1, v2, v3);
          ax[k] = fmaf(g, dx[k], ax[k]);
          ay[k] = fmaf(g, dy[k], ay[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < kUnitPts; ++k) {
          const float g = tnfw_ag(x2[k], v0, v1, v2, v3);
          ax[k] = fmaf(g, dx[k], ax[k]);
          ay[k] = fmaf(g, dy[k], ay[k]);
        }
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int k = 0; k < kUnitPts; ++k) sm.part[w][k][lane] = make_float2(ax[k], ay[k]);
  __syncthreads();
  // Per sample: fixed-order reduction over warps, main deflectors, lens equation, source.
  for (int idx = threadIdx.x; idx < 32 * kUnitPts; idx += 32 * NW) {
    const int k = idx >> 5, l = idx & 31;
    const int q = l * kUnitPts + k;
    if (q >= nsamp) continue;
    float sx = 0.f, sy = 0.f;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) {
      const float2 v = sm.part[ww][k][l];
      sx += v.x;
      sy += v.y;
    }
    const int p = q / s2, sub = q - p * s2;
    const int a = sub / s, b = sub - a * s;
    const int i = by * bh + p / bw, j = bx * bw + p % bw;
    const float x = grid_coord(sys.x0, j, sys.nx, b, s, sys.dpix);
    const float y = grid_coord(sys.y0, i, sys.ny, a, s, sys.dpix);
    for (int d = 0; d < sys.n_defl; ++d) {
      float dax, day;
      alpha_profile(sys.defl[d], x, y, dax, day);
      sx += dax;
      sy += day;
    }
    sm.I[q] = source_light(sys.src_type, sys.src, x - sx, y - sy);
  }
  __syncthreads();
  // Bin-down: dpix^2 times the mean of each pixel's s^2 samples, summed in sample order.
  const float wgt = sys.dpix * sys.dpix / (float)s2;
  for (int p = threadIdx.x; p < bw * bh; p += 32 * NW) {
    const int i = by * bh + p / bw, j = bx * bw + p % bw;
    if (i < sys.ny && j < sys.nx) {
      float acc = 0.f;
      for (int t = 0; t < s2; ++t) acc += sm.I[p * s2 + t];
      sys.out[(size_t)i * sys.nx + j] = acc * wgt;
    }
  }
  __syncthreads();
}

template <int NW>
__global__ void __launch_bounds__(32 * NW) trace_image_kernel(const __grid_constant__ DevSystem sys) {
  __shared__ TraceSmem<NW> sm;
  trace_unit<NW>(sys, blockIdx.x, sm);
}

// Persistent form: CTAs pull unit tickets from the header's counter; ticket u belongs to the
// system whose prefix range [unit_prefix[i], unit_prefix[i+1]) contains it.  Systems arrive
// ordered by per-unit cost (largest first), so the queue hands out the longest units first.
template <int NW>
__global__ void __launch_bounds__(32 * NW) trace_batch_kernel(BatchMeta* __restrict__ meta) {
  __shared__ TraceSmem<NW> sm;
  __shared__ int s_ticket;
  const int n_sys = meta->n_sys;
  const int* __restrict__ unit_prefix = meta->unit_prefix;
  const DevSystem* __restrict__ systems = meta->systems;
  const int total = unit_prefix[n_sys];
  for (;;) {
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(&meta->trace_counter, 1u);
    __syncthreads();
    const int u = s_ticket;
    __syncthreads();
    if (u >= total) return;
    int lo = 0, hi = n_sys;  // largest i with unit_prefix[i] <= u
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (unit_prefix[mid] <= u) lo = mid; else hi = mid;
    }
    trace_unit<NW>(systems[lo], u - unit_prefix[lo], sm);
  }
}

TraceShape choose_trace_shape(int nx, int ny, int s, int n_sub, int sm_count) {
  (void)nx; (void)ny; (void)s; (void)n_sub; (void)sm_count;
  // Fixed for every system so that a system's image does not depend on the launch form or on
  // the other systems of a batch: eight warps split the subhalo list of each unit.
  TraceShape sh;
  sh.nw = kTraceWarps;
  sh.pts = kUnitPts;
  return sh;
}

cudaError_t launch_trace(const DevSystem& sys, TraceShape shape, cudaStream_t st) {
  (void)shape;
  const int grid = unit_count(sys.nx, sys.ny, sys.s);
  trace_image_kernel<kTraceWarps><<<grid, 32 * kTraceWarps, 0, st>>>(sys);
  return cudaGetLastError();
}

int trace_batch_grid(int sm_count) {
  static int blocks_per_sm = 0;
  if (!blocks_per_sm) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, trace_batch_kernel<kTraceWarps>,
                                                      32 * kTraceWarps, 0) != cudaSuccess || blocks_per_sm < 1) {
      cudaGetLastError();
      blocks_per_sm = 1;
    }
  }
  return sm_count * blocks_per_sm;
}

cudaError_t launch_trace_batch_meta(const BatchMeta* meta, int grid, cudaStream_t st) {
  trace_batch_kernel<kTraceWarps><<<grid, 32 * kTraceWarps, 0, st>>>(const_cast<BatchMeta*>(meta));
  return cudaGetLastError();
}

// Ray-shooting at arbitrary points: one thread per point, per-warp staging of the subhalos.
__global__ void __launch_bounds__(256) deflection_kernel(const __grid_constant__ DevSystem sys,
                                                         const float* __restrict__ xs,
                                                         const float* __restrict__ ys, int n,
                                                         float* __restrict__ axs, float* __restrict__ ays) {
  __shared__ float4 s_sub[8][32][kSubStride];
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
#pragma unroll
      for (int c = 0; c < kSubStride; ++c) s_sub[w][lane][c] = __ldg(sys.sub + (size_t)kSubStride * t + c);
    }
    __syncwarp();
    const int cnt = min(32, sys.n_sub - base);
    for (int q = 0; q < cnt; ++q)
      tnfw_pair(px, py, s_sub[w][q][0], s_sub[w][q][1], s_sub[w][q][2], s_sub[w][q][3], ax, ay);
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
