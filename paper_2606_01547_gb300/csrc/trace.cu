// Fused image-simulation kernels, exact subhalo sum: the per-subhalo table prep, the single-system
// launch forms and the batched persistent forms (their device code in trace_unit.cuh; the
// far-field instantiations in trace_far.cu), the likelihood's subhalo field and ray shooting at
// arbitrary points.
#include <algorithm>
#include <type_traits>

#include <cooperative_groups.h>

#include "trace_unit.cuh"

namespace ls {

__global__ void tnfw_prep_kernel(const float* __restrict__ soa, int n, int ld, float4* __restrict__ tab) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  tnfw_write_table(soa[j], soa[ld + j], soa[2 * ld + j], soa[3 * ld + j], soa[4 * ld + j], j, n, tab);
}

cudaError_t launch_tnfw_prep(const float* soa, int n, int ld, float4* table, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  tnfw_prep_kernel<<<(n + 255) / 256, 256, 0, st>>>(soa, n, ld, table);
  return cudaGetLastError();
}

int unit_count(int nx, int ny, int s) {
  int bw, bh;
  unit_shape(s, bw, bh);
  return ((nx + bw - 1) / bw) * ((ny + bh - 1) / bh);
}

// Subhalo deflection field of a grid (the likelihood's fixed field): the units, slices and
// packed pair loop of the image kernels, then each sample's 8 slice partials summed in slice
// order and stored at out[((i * nx + j) * s + a) * s + b] for sub-sample (a, b) of pixel (i, j).
__global__ void __launch_bounds__(32 * kTraceWarps, 2) subhalo_field_kernel(const __grid_constant__ DevSystem sys,
                                                                            float2* __restrict__ out) {
  __shared__ TraceSmem<kTraceWarps> sm;
  const UnitGeom g = unit_geom(sys, blockIdx.x);
  if (block_layout(g.s)) unit_partials<kTraceWarps, false, true>(sys, g, 0, sm);
  else unit_partials<kTraceWarps, false, false>(sys, g, 0, sm);
  __syncthreads();
  for (int idx = threadIdx.x; idx < 32 * kUnitPts; idx += 32 * kTraceWarps) {
    const int k = idx >> 5, l = idx & 31;
    const int q = unit_sample_index(g, l, k);
    if (q >= g.nsamp) continue;
    const int p = q / g.s2, sub = q - p * g.s2;
    const int a = sub / g.s, b = sub - a * g.s;
    const int i = g.by * g.bh + p / g.bw, j = g.bx * g.bw + p % g.bw;
    if (i >= sys.ny || j >= sys.nx) continue;
    float sx = 0.f, sy = 0.f;
#pragma unroll
    for (int sl = 0; sl < kTraceWarps; ++sl) {
      const float2 v = sm.wa[sl].part[k][l];
      sx += v.x;
      sy += v.y;
    }
    out[(((size_t)i * sys.nx + j) * g.s + a) * g.s + b] = make_float2(sx, sy);
  }
}

const char* trace_variant_name(int v) {
  switch (v) {
    case 0: return "cta8";
    case 1: return "cta4x2pass";
    case 2: return "cluster2x4";
    case 3: return "cluster4x2";
    case 4: return "cluster8x1";
    default: return "?";
  }
}

// Every launch takes the block layout where the unit allows it (the finalisation maps samples by
// block_layout(s), so the layout is a function of s alone; the batched launch's persistent
// kernels choose it per unit).  Each sample's arithmetic is the same in both layouts.
cudaError_t launch_trace_variant(const DevSystem& sys, int variant, cudaStream_t st) {
  const int units = unit_count(sys.nx, sys.ny, sys.s);
  const bool far = sys.far_kappa > 0.f, blk = block_layout(sys.s);
  if (far) launch_trace_far(sys, variant, units, st);
  else if (blk) launch_trace_form<false, true>(sys, variant, units, st);
  else launch_trace_form<false, false>(sys, variant, units, st);
  return cudaGetLastError();
}

cudaError_t launch_subhalo_field(const DevSystem& sys, float2* out, cudaStream_t st) {
  subhalo_field_kernel<<<unit_count(sys.nx, sys.ny, sys.s), 32 * kTraceWarps, 0, st>>>(sys, out);
  return cudaGetLastError();
}


const char* batch_form_name(int form) {
  switch (form) {
    case 0: return "cta4x2pass";
    case 1: return "cta8";
    case 2: return "cluster2x4";
    default: return "?";
  }
}

int trace_batch_grid(int sm_count, int form) {
  static int per_sm[kBatchForms] = {0, 0, 0};
  if (form < 0 || form >= kBatchForms) form = 0;
  if (!per_sm[form]) {
    int v = 0;
    cudaError_t e = cudaSuccess;
    // the FAR instantiations have the same launch bounds and shared memory
    if (form == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, trace_batch_kernel<false>, 32 * kHalfWarps, 0);
    if (form == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, trace_batch8_kernel<false>, 32 * kTraceWarps, 0);
    if (form == 2)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, trace_batch_cluster_kernel<false>, 32 * kHalfWarps, 0);
    if (e != cudaSuccess || v < 1) {
      cudaGetLastError();
      v = form == 1 ? 1 : 2;
    }
    if (form == 2) v &= ~1;  // whole clusters
    per_sm[form] = v < 1 ? 2 : v;
  }
  return sm_count * per_sm[form];
}

cudaError_t launch_trace_batch_meta(const BatchMeta* meta, int form, int grid, bool far, cudaStream_t st) {
  BatchMeta* m = const_cast<BatchMeta*>(meta);
  if (far) launch_trace_batch_far(m, form, grid, st);
  else launch_batch_form<false>(m, form, grid, st);
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
  const float4* __restrict__ mid_tab = sys.sub + (size_t)kSubStride * sys.n_sub;
  for (int base = 0; base < sys.n_sub; base += 32) {
    const int t = base + lane;
    if (t < sys.n_sub) {
#pragma unroll
      for (int c = 0; c < kSubStride; ++c) s_sub[w][lane][c] = __ldg(sys.sub + (size_t)kSubStride * t + c);
    }
    __syncwarp();
    const int cnt = min(32, sys.n_sub - base);
    for (int q = 0; q < cnt; ++q)
      tnfw_pair(px, py, s_sub[w][q], mid_tab + (size_t)kMidStride * (base + q), ax, ay);
    __syncwarp();
  }
  for (int d = 0; d < sys.n_defl; ++d) {
    float dax, day;
    alpha_profile(sys.defl[d], sys.ell_c, sys.ell_K, px, py, dax, day);
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
