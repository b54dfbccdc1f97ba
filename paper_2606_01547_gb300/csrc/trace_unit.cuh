// Device code of the fused image-simulation kernels (image simulation steps 1 and 2 plus the
// supersample bin-down), shared by the translation units that instantiate them: trace.cu (the
// exact subhalo sum) and trace_far.cu (the optional far-field interpolation), compiled in
// parallel.
//
// Work unit: 288 sub-pixel samples = 32 lanes x 9 samples, covering a pixel block whose shape
// depends on the supersampling factor s (24x12 pixels at s=1, 12x6 at s=2, 8x4 at s=3, ...), so
// every s keeps all lanes busy.  The NW warps of a CTA split the subhalo list of the unit (an
// N-body-like all-pairs sum staged through shared memory); their partial deflections are
// reduced in a fixed warp order, then the main deflectors, the lens equation
// beta = theta - alpha, the Sersic source and the bin-down run on chip.  Traced coordinates
// never leave registers and shared memory; only the binned image is written.
//
// Two launch forms share the unit body: one CTA (or cluster) per unit of a single system, and
// persistent kernels that pull units of many systems from a device-side queue.
#pragma once
#include <type_traits>

#include <cooperative_groups.h>

#include "kernels.h"

namespace ls {
namespace cg = cooperative_groups;

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


// A warp stages 32 subhalos at a time, record q in lane q's slot, and lists them by class -- 6-,
// 4-, 3-term far-field series, then the marked near-field subhalos -- in subhalo order within
// the class, so each class is a counted loop over consecutive list entries (whose loads the
// compiler can issue ahead) rather than a scan of a ballot mask.  Every class but the last
// (marked) one starts on an even list position (one pad each at most), so a pair of entries
// loads as one int2.  With the far-field interpolation, far subhalos form three more classes
// (summed at the Chebyshev nodes) between the sample classes and the marked ones.
constexpr int kStageList = 38;
constexpr int kFarRec = 4;                 // t0, t2, t3, t4: centre and series coefficients
constexpr int kNearRec = 2 + kMidStride;   // t1, t6 and the annulus block
static_assert(kUnitPts > 2 * kPackedPairs, "a lane runs kPackedPairs sample pairs and at least one scalar sample");

// Far-field interpolation (optional, changes results): a subhalo at least kappa times the box's
// larger half-width from the unit's sample box is summed at the 8 x 8 Chebyshev nodes of the box
// (first kind, x_i = cos(pi (i + 1/2) / 8) scaled to the box) rather than at its 288 samples,
// and the unit's summed node values are interpolated to the samples with the tensor Lagrange
// basis -- the local-expansion step of a black-box fast multipole method (Fong and Darve 2009).
// Node n = 8 i + j sits at (x_i, y_j); lane l holds nodes 2l and 2l + 1 as one packed pair.
constexpr int kFarNodes1 = 8;
constexpr int kFarNodes = kFarNodes1 * kFarNodes1;
static_assert(kFarNodes == 2 * 32, "a lane evaluates two nodes");
static __constant__ float c_cheb8[kFarNodes1] = {9.807852804e-01f, 8.314696123e-01f, 5.555702330e-01f, 1.950903220e-01f,
                                          -1.950903220e-01f, -5.555702330e-01f, -8.314696123e-01f, -9.807852804e-01f};
// 1 / prod_{k != i} (x_i - x_k): the Lagrange basis is L_i(t) = w_i prod_{k != i} (t - x_k)
static __constant__ float c_cheb8_w[kFarNodes1] = {3.121445152e+00f, -8.889123728e+00f, 1.330351380e+01f, -1.569256449e+01f,
                                            1.569256449e+01f, -1.330351380e+01f, 8.889123728e+00f, -3.121445152e+00f};

__device__ __forceinline__ void cheb8_lagrange(float t, float* L) {
  float d[kFarNodes1], pre[kFarNodes1], suf[kFarNodes1];
#pragma unroll
  for (int k = 0; k < kFarNodes1; ++k) d[k] = t - c_cheb8[k];
  pre[0] = 1.f;
#pragma unroll
  for (int k = 1; k < kFarNodes1; ++k) pre[k] = pre[k - 1] * d[k - 1];
  suf[kFarNodes1 - 1] = 1.f;
#pragma unroll
  for (int k = kFarNodes1 - 2; k >= 0; --k) suf[k] = suf[k + 1] * d[k + 1];
#pragma unroll
  for (int k = 0; k < kFarNodes1; ++k) L[k] = c_cheb8_w[k] * (pre[k] * suf[k]);
}

template <int NW>
struct TraceSmem {
  // Per warp: the staged records of one stage, reused for the warp's partials once its subhalo
  // loop has ended (so a warp never overwrites what another warp is still reading).
  union WarpArea {
    struct {
      float4 sub[32][kFarRec];
      float4 marked[32][kNearRec];
      int list[kStageList];
      float4 box;  // the unit's bounding box (kept here rather than in registers)
      // per stage: the far-field node classes' compact records (float4 x 2 per lane), then the
      // closed-form arguments and values of one marked subhalo at a time; at the end, the
      // slice's far-field node sums (float2 x 64)
      alignas(16) float queue[kUnitPts * 32];
    };
    float2 part[kUnitPts][32];
  } wa[NW];
  float I[kUnitPts * 32];
  float2 nodes[kFarNodes];  // the unit's far-field node sums (interpolation only)
};

struct UnitGeom {
  int s, s2, bw, bh, bx, by, nsamp;
};

__device__ __forceinline__ UnitGeom unit_geom(const DevSystem& sys, int blk) {
  UnitGeom g;
  g.s = sys.s;
  g.s2 = g.s * g.s;
  unit_shape(g.s, g.bw, g.bh);
  const int nbx = (sys.nx + g.bw - 1) / g.bw;
  g.bx = blk % nbx;
  g.by = blk / nbx;
  g.nsamp = g.bw * g.bh * g.s2;
  return g;
}

__device__ __forceinline__ void sample_xy(const DevSystem& sys, const UnitGeom& g, int q, float& x, float& y) {
  const int p = q / g.s2, sub = q - p * g.s2;
  const int a = sub / g.s, b = sub - a * g.s;
  const int i = g.by * g.bh + p / g.bw, j = g.bx * g.bw + p % g.bw;
  x = grid_coord(sys.x0, j, sys.nx, b, g.s, sys.dpix);
  y = grid_coord(sys.y0, i, sys.ny, a, g.s, sys.dpix);
}

// Block layout: at s = 1, 2, 3, 4 and 6 a unit is 24 x 12 samples, and lane l holds the 3 x 3
// block of samples at sample columns 3 (l mod 8) + b and rows 3 (l div 8) + a (k = 3a + b; at
// s = 3 the block is the lane's pixel, its 9 sub-samples).  unit_sample_index maps lane l's
// sample k to the unit's sample index q (pixel q / s^2 of the unit's pixel block, sub-sample
// q mod s^2) in either layout, so partials, finalisation and bin-down agree.
__host__ __device__ constexpr bool block_layout(int s) { return s == 1 || s == 2 || s == 3 || s == 4 || s == 6; }

__device__ __forceinline__ int unit_sample_index(const UnitGeom& g, int l, int k) {
  if (!block_layout(g.s)) return l * kUnitPts + k;
  const int sc = 3 * (l & 7) + k % 3, sr = 3 * (l >> 3) + k / 3;
  const int pc = sc / g.s, pr = sr / g.s;
  return (pr * g.bw + pc) * g.s2 + (sr - pr * g.s) * g.s + (sc - pc * g.s);
}

// Coordinate of a block-layout sample column c (0 .. 23 of the unit) or row r (0 .. 11): the
// sample_xy value of every sample in it, from one division by s.
__device__ __forceinline__ float block_x(const DevSystem& sys, const UnitGeom& g, int c) {
  const int pc = c / g.s;
  return grid_coord(sys.x0, g.bx * g.bw + pc, sys.nx, c - pc * g.s, g.s, sys.dpix);
}
__device__ __forceinline__ float block_y(const DevSystem& sys, const UnitGeom& g, int r) {
  const int pr = r / g.s;
  return grid_coord(sys.y0, g.by * g.bh + pr, sys.ny, r - pr * g.s, g.s, sys.dpix);
}

// In the block layout a lane's packed pairs are {(0,b),(1,b)} for the columns b = 0, 1, 2, then
// {(2,0),(2,1)}, and the scalar sample (2,2).  The three column pairs share their rows, so one
// (dy, dy^2) pair serves them, and each pair's dx is one column's: per subhalo the 3 column
// offsets and the 3 row offsets and squares are computed once, and the scalar sample takes
// column 2's and row 2's.
__host__ __device__ constexpr int s3_pair_of(int k) { return k / 3 < 2 ? k % 3 : (k % 3 < 2 ? 3 : -1); }
__host__ __device__ constexpr int s3_half_of(int k) { return k / 3 < 2 ? k / 3 : k % 3; }
__host__ __device__ constexpr int s3_k_of(int i, int e) { return i < 3 ? 3 * e + i : 6 + e; }

// Partial subhalo deflections of one unit: warp w of this CTA sums slice (slice0 + w) of the
// kTraceWarps-way split of the subhalo list and writes its 288 partials to wa[area0 + w].part.
//
// A lane's first 2 kPackedPairs samples run as packed pairs (FP32x2 instructions, two samples
// per issue slot, on the heavy FMA pipe), the rest as scalars; both kinds draw on the same
// FP32 capacity, so the packing saves issue slots, not lane operations.  The packed operations
// are element-wise the same IEEE operations as the scalar ones, so every sample's deflection
// is the same whichever kind it is.  With BLK (block_layout(s) only) the
// samples take the block layout above: each sample's arithmetic is unchanged, only shared terms
// are computed once, so every sample's partial is bitwise that of the generic layout.
template <int NWC, bool FAR = false, bool BLK = false>
__device__ __forceinline__ void unit_partials(const DevSystem& sys, const UnitGeom& g, int slice0,
                                              TraceSmem<NWC>& sm, int area0 = 0) {
  constexpr int kP = kPackedPairs;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int n = sys.n_sub;
  const int slice = slice0 + w;
  const int lo = (int)(((long long)n * slice) / kTraceWarps);
  const int hi = (int)(((long long)n * (slice + 1)) / kTraceWarps);
  const float4* __restrict__ rec_tab = sys.sub;
  const float4* __restrict__ mid_tab = sys.sub + (size_t)kSubStride * n;
  const float4* __restrict__ far_tab = sys.sub + (size_t)(kSubStride + kMidStride) * n;
  auto& area = sm.wa[area0 + w];

  // generic layout: the packed pairs' and scalar samples' coordinates (px2, py2, po_*); block
  // layout: the lane's three columns and rows (bxs, bys); both: the sums (ax2, ay2, ao_*)
  float2 px2[kP], py2[kP], ax2[kP], ay2[kP];
  constexpr int kS = kUnitPts - 2 * kP;  // scalar samples
  static_assert(!BLK || (kP == 4 && kS == 1), "the block layout pairs a lane's 3 x 3 samples");
  float po_x[kS], po_y[kS], ao_x[kS], ao_y[kS];  // the scalar samples and their sums
  // sample k's place: packed pair pair_of(k) (-1: scalar k - 2 kP), half half_of(k); and back
  auto pair_of = [](int k) { return BLK ? s3_pair_of(k) : (k < 2 * kP ? k >> 1 : -1); };
  auto half_of = [](int k) { return BLK ? s3_half_of(k) : (k & 1); };
  auto k_of = [](int i, int e) { return BLK ? s3_k_of(i, e) : 2 * i + e; };
  float xmin = 3.0e38f, xmax = -3.0e38f, ymin = 3.0e38f, ymax = -3.0e38f;
  float bxs[3], bys[3];  // block layout: the lane's three sample columns and rows
  if constexpr (BLK) {
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      bxs[e] = block_x(sys, g, 3 * (lane & 7) + e);
      bys[e] = block_y(sys, g, 3 * (lane >> 3) + e);
    }
  }
#pragma unroll
  for (int k = 0; k < kUnitPts; ++k) {
    float x, y;
    if constexpr (BLK) {
      x = bxs[k % 3];
      y = bys[k / 3];
    } else {
      int q = lane * kUnitPts + k;
      if (q >= g.nsamp) q = 0;
      sample_xy(sys, g, q, x, y);
    }
    xmin = fminf(xmin, x); xmax = fmaxf(xmax, x);
    ymin = fminf(ymin, y); ymax = fmaxf(ymax, y);
    if constexpr (BLK) continue;
    const int pr = pair_of(k);
    if (pr < 0) {
      po_x[k - 2 * kP] = x;
      po_y[k - 2 * kP] = y;
    } else if (half_of(k)) {
      px2[pr].y = x;
      py2[pr].y = y;
    } else {
      px2[pr].x = x;
      py2[pr].x = y;
    }
  }
#pragma unroll
  for (int i = 0; i < kP; ++i) {
    ax2[i] = make_float2(0.f, 0.f);
    ay2[i] = make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int i = 0; i < kS; ++i) {
    ao_x[i] = 0.f;
    ao_y[i] = 0.f;
  }
  // bounding box of the unit's samples (uniform across the warp)
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    xmin = fminf(xmin, __shfl_xor_sync(0xffffffffu, xmin, off));
    xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, off));
    ymin = fminf(ymin, __shfl_xor_sync(0xffffffffu, ymin, off));
    ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, off));
  }
  if (lane == 0) area.box = make_float4(xmin, xmax, ymin, ymax);
  __syncwarp();
  // far-field interpolation: the lane's two nodes and their sums
  float2 pn_x = make_float2(0.f, 0.f), pn_y = pn_x, an_x = pn_x, an_y = pn_x;
  float far_d2 = 3.0e38f;
  if constexpr (FAR) {
    const float hx = 0.5f * (xmax - xmin), hy = 0.5f * (ymax - ymin);
    const float cxb = 0.5f * (xmin + xmax), cyb = 0.5f * (ymin + ymax);
    const float hf = sys.far_kappa * fmaxf(hx, hy);
    far_d2 = hf * hf;
    const int ni = lane >> 2, nj = 2 * (lane & 3);
    const float xn = fmaf(hx, c_cheb8[ni], cxb);
    pn_x = make_float2(xn, xn);
    pn_y = make_float2(fmaf(hy, c_cheb8[nj], cyb), fmaf(hy, c_cheb8[nj + 1], cyb));
  }
  // offsets of the lane's samples from record t's centre: packed pairs' dx, dy, dy^2, and the
  // scalar samples' (dx = x - cx, dy = y - cy).  In the block layout the 3 columns' dx and the
  // 3 rows' dy and dy^2 are computed once each as scalars and then paired: an FP32x2 operation
  // on a duplicated pair spends two lane operations of the FP32 pipe on one value (9 scalar
  // operations per subhalo instead of 8 FP32x2 ones, i.e. 16 lane operations; the same IEEE
  // results)
  auto deltas = [&](const float4* t, float2* dx, float2* dy, float2* dy2, float* sdx, float* sdy, float* sdy2) {
    if constexpr (BLK) {
      const float ex0 = bxs[0] + t[0].x, ex1 = bxs[1] + t[0].x, ex2 = bxs[2] + t[0].x;
      const float ey0 = bys[0] + t[0].z, ey1 = bys[1] + t[0].z, ey2 = bys[2] + t[0].z;
      const float qy0 = ey0 * ey0, qy1 = ey1 * ey1, qy2 = ey2 * ey2;
      dx[0] = make_float2(ex0, ex0);
      dx[1] = make_float2(ex1, ex1);
      dx[2] = make_float2(ex2, ex2);
      dx[3] = make_float2(ex0, ex1);
      const float2 dya = make_float2(ey0, ey1), dyc = make_float2(ey2, ey2);
      const float2 dy2a = make_float2(qy0, qy1), dy2c = make_float2(qy2, qy2);
      dy[0] = dya; dy[1] = dya; dy[2] = dya; dy[3] = dyc;
      dy2[0] = dy2a; dy2[1] = dy2a; dy2[2] = dy2a; dy2[3] = dy2c;
      sdx[0] = ex2;   // sample (2, 2): column 2
      sdy[0] = ey2;   // row 2
      sdy2[0] = qy2;
    } else {
      const float2 ncx = make_float2(t[0].x, t[0].y), ncy = make_float2(t[0].z, t[0].w);
#pragma unroll
      for (int i = 0; i < kP; ++i) {
        dx[i] = __fadd2_rn(px2[i], ncx);
        dy[i] = __fadd2_rn(py2[i], ncy);
        dy2[i] = __fmul2_rn(dy[i], dy[i]);
      }
#pragma unroll
      for (int j = 0; j < kS; ++j) {
        sdx[j] = po_x[j] + t[0].x;
        sdy[j] = po_y[j] + t[0].z;
        sdy2[j] = sdy[j] * sdy[j];
      }
    }
  };
  // far-field series truncated after d_K for record t, every sample of the lane
  auto far_all = [&](const float4* t, auto Kc) {
    constexpr int K = decltype(Kc)::value;
    float2 dx[kP], dy[kP], dy2[kP];
    float sdx[kS], sdy[kS], sdy2[kS];
    deltas(t, dx, dy, dy2, sdx, sdy, sdy2);
#pragma unroll
    for (int i = 0; i < kP; ++i) {
      const float2 r2 = __ffma2_rn(dx[i], dx[i], dy2[i]);
      const float2 u = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
      const float2 gg = tnfw_series2_k<K>(u, __fmul2_rn(u, u), t);
      ax2[i] = __ffma2_rn(gg, dx[i], ax2[i]);
      ay2[i] = __ffma2_rn(gg, dy[i], ay2[i]);
    }
#pragma unroll
    for (int j = 0; j < kS; ++j) {
      const float u = rsqrt_ftz(fmaf(sdx[j], sdx[j], sdy2[j]));
      const float gg = tnfw_series_k<K>(u, u * u, t);
      ao_x[j] = fmaf(gg, sdx[j], ao_x[j]);
      ao_y[j] = fmaf(gg, sdy[j], ao_y[j]);
    }
  };
  auto load_far = [&](int q, float4* t) {
    t[0] = area.sub[q][0];
#pragma unroll
    for (int c = 1; c < kFarRec; ++c) t[1 + c] = area.sub[q][c];
  };
  // a class of far subhalos at list positions [b, e), b even: two per basic block (four for the
  // shortest series, the most common class, in the exact kernels; the far-field ones measured
  // slower with it), so the scheduler overlaps one's reciprocal square roots and loads with
  // another's polynomial; the subhalos are summed in list order either way
  auto far_class = [&](int b, int e, auto Kc) {
    int q = b;
    if constexpr (decltype(Kc)::value == 3 && !FAR) {
#pragma unroll 1
      for (; q + 3 < e; q += 4) {
        float4 ta[5], tb[5], tc[5], td[5];
        const int2 qa = *reinterpret_cast<const int2*>(&area.list[q]);
        const int2 qb = *reinterpret_cast<const int2*>(&area.list[q + 2]);
        load_far(qa.x, ta);
        load_far(qa.y, tb);
        load_far(qb.x, tc);
        load_far(qb.y, td);
        far_all(ta, Kc);
        far_all(tb, Kc);
        far_all(tc, Kc);
        far_all(td, Kc);
      }
    }
#pragma unroll 1
    for (; q + 1 < e; q += 2) {
      float4 ta[5], tb[5];
      const int2 qq = *reinterpret_cast<const int2*>(&area.list[q]);
      load_far(qq.x, ta);
      load_far(qq.y, tb);
      far_all(ta, Kc);
      far_all(tb, Kc);
    }
    if (q < e) {
      float4 ta[5];
      load_far(area.list[q], ta);
      far_all(ta, Kc);
    }
  };
  // sample k's coordinates (k static) and its accumulators
  auto sample_at = [&](int k, float& x, float& y) {
    if constexpr (BLK) {  // the lane's column b and row a
      x = bxs[k % 3];
      y = bys[k / 3];
      return;
    }
    const int pr = pair_of(k);
    if (pr < 0) { x = po_x[k - 2 * kP]; y = po_y[k - 2 * kP]; }
    else if (half_of(k)) { x = px2[pr].y; y = py2[pr].y; }
    else { x = px2[pr].x; y = py2[pr].x; }
  };
  auto accumulate_at = [&](int k, float g, float dx, float dy) {
    const int pr = pair_of(k);
    if (pr < 0) {
      ao_x[k - 2 * kP] = fmaf(g, dx, ao_x[k - 2 * kP]);
      ao_y[k - 2 * kP] = fmaf(g, dy, ao_y[k - 2 * kP]);
    }
    else if (half_of(k)) { ax2[pr].y = fmaf(g, dx, ax2[pr].y); ay2[pr].y = fmaf(g, dy, ay2[pr].y); }
    else { ax2[pr].x = fmaf(g, dx, ax2[pr].x); ay2[pr].x = fmaf(g, dy, ay2[pr].x); }
  };
  // The closed forms of a marked subhalo's samples inside r_in (bit k of `inner`), spread over
  // the whole warp: the samples of a few lanes' pixels would otherwise run them one sample
  // position at a time with the other lanes idle.  Each lane queues its samples' arguments in
  // sample order, the warp evaluates the queue 32 at a time, and each lane adds its values
  // where the pair loop left them out, so every accumulator sees the same sequence of FMAs.
  auto near_inner = [&](const float4* t, unsigned inner) {
    const int c = __popc(inner);
    int pre = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, pre, off);
      if (lane >= off) pre += v;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    float* qv = area.queue;
    int o = pre - c;
#pragma unroll
    for (int k = 0; k < kUnitPts; ++k) {
      if ((inner >> k) & 1u) {
        float x, y;
        sample_at(k, x, y);
        const float dx = x + t[0].x, dy = y + t[0].z;
        qv[o++] = fmaf(dx, dx, dy * dy) * t[1].y;
      }
    }
    __syncwarp();
#pragma unroll 1
    for (int e = lane; e < total; e += 32) qv[e] = tnfw_g_inner(qv[e], t[1].z, t[1].w, t[6].w);
    __syncwarp();
    o = pre - c;
#pragma unroll
    for (int k = 0; k < kUnitPts; ++k) {
      if ((inner >> k) & 1u) {
        float x, y;
        sample_at(k, x, y);
        const float dx = x + t[0].x, dy = y + t[0].z;
        accumulate_at(k, qv[o++], dx, dy);
      }
    }
    __syncwarp();  // the queue is free for the next subhalo
  };
  // far-field interpolation: a class of far subhalos at list positions [b, e), b even, summed
  // at the lane's two nodes
  //
  // A node pair is one subhalo's work against one packed pair of a sample subhalo's nine, so
  // the node classes read each record in the compact form (-cx, -cy, d_0, d_2), (d_3 .. d_6)
  // that staging left in the queue area (2 broadcast loads instead of 3-4) and evaluate the
  // lane's two nodes, which share their x, as scalars on the light FMA pipe.
  auto node_pair = [&](const float4* compact, int q, auto Kc) {
    constexpr int K = decltype(Kc)::value;
    const float4 c0 = compact[2 * q], c1 = compact[2 * q + 1];
    const float d[7] = {c0.z, 0.f, c0.w, c1.x, c1.y, c1.z, c1.w};  // d_0, -, d_2 .. d_6
    const float dx = pn_x.x + c0.x, dy0 = pn_y.x + c0.y, dy1 = pn_y.y + c0.y;
    const float dx2 = dx * dx;
    const float u0 = rsqrt_ftz(fmaf(dy0, dy0, dx2)), u1 = rsqrt_ftz(fmaf(dy1, dy1, dx2));
    const float v0 = u0 * u0, v1 = u1 * u1;
    float p0 = fmaf(d[K], u0, d[K - 1]), p1 = fmaf(d[K], u1, d[K - 1]);
#pragma unroll
    for (int k = K - 2; k >= 2; --k) {
      p0 = fmaf(p0, u0, d[k]);
      p1 = fmaf(p1, u1, d[k]);
    }
    const float g0 = fmaf(p0, v0, d[0]) * v0, g1 = fmaf(p1, v1, d[0]) * v1;
    an_x.x = fmaf(g0, dx, an_x.x);
    an_y.x = fmaf(g0, dy0, an_y.x);
    an_x.y = fmaf(g1, dx, an_x.y);
    an_y.y = fmaf(g1, dy1, an_y.y);
  };
  auto node_class = [&](int b, int e, auto Kc) {
    const float4* compact = reinterpret_cast<const float4*>(area.queue);
    int q = b;
#pragma unroll 1
    for (; q + 1 < e; q += 2) {
      const int2 qq = *reinterpret_cast<const int2*>(&area.list[q]);
      node_pair(compact, qq.x, Kc);
      node_pair(compact, qq.y, Kc);
    }
    if (q < e) node_pair(compact, area.list[q], Kc);
  };
  // subhalos the bounding-box test marked: series and annulus polynomial for every sample
  // (packed, branch-free), each sample then keeps the form of its distance; samples inside
  // r_in add nothing here and take the closed form through the queue
  auto near_pairs = [&](const float4* t, const float4* m) {
    const float r_far2 = t[1].x, r_in2 = t[6].z;
    auto pick = [&](float r2, float gs, float gm) { return r2 >= r_far2 ? gs : (r2 >= r_in2 ? gm : 0.f); };
    unsigned inner = 0u;
    float2 dx[kP], dy[kP], dy2[kP];
    float sdx[kS], sdy[kS], sdy2[kS];
    deltas(t, dx, dy, dy2, sdx, sdy, sdy2);
#pragma unroll
    for (int i = 0; i < kP; ++i) {
      const float2 r2 = __ffma2_rn(dx[i], dx[i], dy2[i]);
      const float2 u = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
      const float2 u2 = __fmul2_rn(u, u);
      const float2 gs = tnfw_series2_u(u, u2, t);
      const float2 gm = tnfw_mid2_u(u, u2, t, m);
      const float2 gg = make_float2(pick(r2.x, gs.x, gm.x), pick(r2.y, gs.y, gm.y));
      inner |= (r2.x < r_in2 ? 1u : 0u) << k_of(i, 0);
      inner |= (r2.y < r_in2 ? 1u : 0u) << k_of(i, 1);
      ax2[i] = __ffma2_rn(gg, dx[i], ax2[i]);
      ay2[i] = __ffma2_rn(gg, dy[i], ay2[i]);
    }
#pragma unroll
    for (int j = 0; j < kS; ++j) {
      const float r2 = fmaf(sdx[j], sdx[j], sdy2[j]);
      const float u = rsqrt_ftz(r2), u2 = u * u;
      const float gg = pick(r2, tnfw_series_u(u, u2, t), tnfw_mid_u(u, u2, t, m));
      inner |= (r2 < r_in2 ? 1u : 0u) << (2 * kP + j);
      ao_x[j] = fmaf(gg, sdx[j], ao_x[j]);
      ao_y[j] = fmaf(gg, sdy[j], ao_y[j]);
    }
    if (__any_sync(0xffffffffu, inner != 0u)) near_inner(t, inner);
  };
  // While staging, each lane tests its subhalo against the unit's bounding box: subhalos some
  // sample might see inside the far-field radius are marked (near); the others take the
  // shortest far-field series whose range holds the whole box (6 terms from 7, 4 from 20, 3 from
  // 40 max(tau, 1) Rs).  Marked subhalos let every sample pick its own form (the 6-term series
  // again beyond the radius).  The stage is summed class by class (6-, 4-, 3-term, then marked),
  // each in subhalo order: an order fixed by the unit, so every launch form gives the same sums.
  for (int base = lo; base < hi; base += 32) {
    const int idx = base + lane;
    const bool alive = idx < hi;
    bool near = false, interp = false;
    int tier = 0;  // 0: 6-term series, 1: 4-term, 2: 3-term
    if (alive) {
      // the compact block, written out as the record's duplicated pairs
      const float4 f0 = __ldg(far_tab + (size_t)kFarStride * idx);
      const float4 f1 = __ldg(far_tab + (size_t)kFarStride * idx + 1);
      const float4 f2 = __ldg(far_tab + (size_t)kFarStride * idx + 2);
      area.sub[lane][0] = make_float4(f0.x, f0.x, f0.y, f0.y);
      area.sub[lane][1] = make_float4(f1.y, f1.y, f1.z, f1.z);
      area.sub[lane][2] = make_float4(f1.w, f1.w, f2.x, f2.x);
      area.sub[lane][3] = make_float4(f2.y, f2.y, f2.z, f2.z);
      // f0.xy hold the negated centre
      const float4 bx = area.box;
      const float xmin = bx.x, xmax = bx.y, ymin = bx.z, ymax = bx.w;
      const float ddx = fmaxf(fmaxf(xmin + f0.x, -f0.x - xmax), 0.f);
      const float ddy = fmaxf(fmaxf(ymin + f0.y, -f0.y - ymax), 0.f);
      const float d2 = fmaf(ddx, ddx, ddy * ddy);
      near = d2 < f0.z;
      tier = d2 >= f1.x ? 2 : (d2 >= f0.w ? 1 : 0);
      if constexpr (FAR) {
        interp = !near && d2 >= far_d2;  // marked subhalos always run at the samples
        if (interp) {  // the compact record of the node classes (queue area, free until the near field)
          float4* compact = reinterpret_cast<float4*>(area.queue);
          compact[2 * lane] = make_float4(f0.x, f0.y, f1.y, f1.z);
          compact[2 * lane + 1] = make_float4(f1.w, f2.x, f2.y, f2.z);
        }
      }
      if (near) {
        area.marked[lane][0] = __ldg(rec_tab + (size_t)kSubStride * idx + 1);
        area.marked[lane][1] = __ldg(rec_tab + (size_t)kSubStride * idx + 6);
#pragma unroll
        for (int c = 0; c < kMidStride; ++c) area.marked[lane][2 + c] = __ldg(mid_tab + (size_t)kMidStride * idx + c);
      }
    }
    const bool direct = alive && !near && !interp;
    const unsigned mn = __ballot_sync(0xffffffffu, alive && near);
    const unsigned m3 = __ballot_sync(0xffffffffu, direct && tier == 2);
    const unsigned m4 = __ballot_sync(0xffffffffu, direct && tier == 1);
    const unsigned m6 = __ballot_sync(0xffffffffu, direct && tier == 0);
    const int n6 = __popc(m6), n4 = __popc(m4), n3 = __popc(m3), nn = __popc(mn);
    const int b4 = (n6 + 1) & ~1, b3 = b4 + ((n4 + 1) & ~1);
    int bn = b3 + n3;
    unsigned f3 = 0u, f4 = 0u, f6 = 0u;
    int nf6 = 0, nf4 = 0, nf3 = 0, bf6 = bn, bf4 = bn, bf3 = bn;
    if constexpr (FAR) {
      f3 = __ballot_sync(0xffffffffu, interp && tier == 2);
      f4 = __ballot_sync(0xffffffffu, interp && tier == 1);
      f6 = __ballot_sync(0xffffffffu, interp && tier == 0);
      nf6 = __popc(f6); nf4 = __popc(f4); nf3 = __popc(f3);
      bf6 = b3 + ((n3 + 1) & ~1);
      bf4 = bf6 + ((nf6 + 1) & ~1);
      bf3 = bf4 + ((nf4 + 1) & ~1);
      bn = bf3 + nf3;
    }
    if (alive) {
      const unsigned below = (1u << lane) - 1u;
      int pos;
      if (near) pos = bn + __popc(mn & below);
      else if (interp) pos = tier == 2 ? bf3 + __popc(f3 & below) : (tier == 1 ? bf4 + __popc(f4 & below) : bf6 + __popc(f6 & below));
      else pos = tier == 2 ? b3 + __popc(m3 & below) : (tier == 1 ? b4 + __popc(m4 & below) : __popc(m6 & below));
      area.list[pos] = lane;
    }
    __syncwarp();
    far_class(0, n6, std::integral_constant<int, kFarTerms>{});
    far_class(b4, b4 + n4, std::integral_constant<int, 4>{});
    far_class(b3, b3 + n3, std::integral_constant<int, 3>{});
    if constexpr (FAR) {
      node_class(bf6, bf6 + nf6, std::integral_constant<int, kFarTerms>{});
      node_class(bf4, bf4 + nf4, std::integral_constant<int, 4>{});
      node_class(bf3, bf3 + nf3, std::integral_constant<int, 3>{});
    }
#pragma unroll 1
    for (int i = bn; i < bn + nn; ++i) {
      const int q = area.list[i];
      float4 t[kSubStride], m[kMidStride];
      t[0] = area.sub[q][0];
      t[1] = area.marked[q][0];
#pragma unroll
      for (int c = 1; c < kFarRec; ++c) t[1 + c] = area.sub[q][c];
      t[5] = make_float4(0.f, 0.f, 0.f, 0.f);
      t[6] = area.marked[q][1];
      t[7] = t[5];
#pragma unroll
      for (int c = 0; c < kMidStride; ++c) m[c] = area.marked[q][2 + c];
      near_pairs(t, m);
    }
    __syncwarp();
  }
  // the warp's staged records are dead from here on: its partials take their place
#pragma unroll
  for (int i = 0; i < kP; ++i) {
    area.part[k_of(i, 0)][lane] = make_float2(ax2[i].x, ay2[i].x);
    area.part[k_of(i, 1)][lane] = make_float2(ax2[i].y, ay2[i].y);
  }
#pragma unroll
  for (int i = 0; i < kS; ++i) area.part[2 * kP + i][lane] = make_float2(ao_x[i], ao_y[i]);
  if constexpr (FAR) {  // the slice's node sums, for the unit's interpolation
    float2* nv = reinterpret_cast<float2*>(area.queue);
    nv[2 * lane] = make_float2(an_x.x, an_y.x);
    nv[2 * lane + 1] = make_float2(an_x.y, an_y.y);
  }
}

// Far-field interpolation: the unit's node sums from its kTraceWarps slices' (node(slice, n), in
// slice order) into `nodes`.  Executed by `nthr` threads, ends with a CTA barrier.
template <class NodeFn>
__device__ __forceinline__ void unit_sum_nodes(float2* nodes, int nthr, NodeFn node) {
  for (int n = threadIdx.x; n < kFarNodes; n += nthr) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int sl = 0; sl < kTraceWarps; ++sl) {
      const float2 v = node(sl, n);
      acc.x += v.x;
      acc.y += v.y;
    }
    nodes[n] = acc;
  }
  __syncthreads();
}

// Finalise a unit from its kTraceWarps slice partials (part(slice, k, lane) in slice order):
// main deflectors, lens equation, source, then the bin-down.  Executed by `nthr` threads.  With
// FAR, each sample adds the interpolant of the node sums (`nodes`, over the box `box`).
template <bool FAR = false, class PartFn>
__device__ __forceinline__ void unit_finalize(const DevSystem& sys, const UnitGeom& g, float* I, int nthr,
                                              PartFn part, const float2* nodes = nullptr,
                                              float4 box = make_float4(0.f, 0.f, 0.f, 0.f)) {
  float cxb = 0.f, cyb = 0.f, ihx = 0.f, ihy = 0.f;
  if constexpr (FAR) {
    const float hx = 0.5f * (box.y - box.x), hy = 0.5f * (box.w - box.z);
    cxb = 0.5f * (box.x + box.y);
    cyb = 0.5f * (box.z + box.w);
    ihx = hx > 0.f ? 1.f / hx : 0.f;  // a box one sample wide: every sample at t = 0
    ihy = hy > 0.f ? 1.f / hy : 0.f;
  }
  for (int idx = threadIdx.x; idx < 32 * kUnitPts; idx += nthr) {
    const int k = idx >> 5, l = idx & 31;
    int q;
    float x, y;
    if (block_layout(g.s)) {  // the sample's index and coordinates from its column and row
      const int sc = 3 * (l & 7) + k % 3, sr = 3 * (l >> 3) + k / 3;
      const int pc = sc / g.s, pr = sr / g.s;
      q = (pr * g.bw + pc) * g.s2 + (sr - pr * g.s) * g.s + (sc - pc * g.s);
      x = grid_coord(sys.x0, g.bx * g.bw + pc, sys.nx, sc - pc * g.s, g.s, sys.dpix);
      y = grid_coord(sys.y0, g.by * g.bh + pr, sys.ny, sr - pr * g.s, g.s, sys.dpix);
    } else {
      q = l * kUnitPts + k;
      if (q >= g.nsamp) continue;
      sample_xy(sys, g, q, x, y);
    }
    float sx = 0.f, sy = 0.f;
#pragma unroll
    for (int sl = 0; sl < kTraceWarps; ++sl) {
      const float2 v = part(sl, k, l);
      sx += v.x;
      sy += v.y;
    }
    if constexpr (FAR) {
      float lx[kFarNodes1], ly[kFarNodes1];
      cheb8_lagrange((x - cxb) * ihx, lx);
      cheb8_lagrange((y - cyb) * ihy, ly);
      float fx = 0.f, fy = 0.f;
#pragma unroll
      for (int i = 0; i < kFarNodes1; ++i) {
        float rx = 0.f, ry = 0.f;
#pragma unroll
        for (int j = 0; j < kFarNodes1; ++j) {
          const float2 v = nodes[kFarNodes1 * i + j];
          rx = fmaf(ly[j], v.x, rx);
          ry = fmaf(ly[j], v.y, ry);
        }
        fx = fmaf(lx[i], rx, fx);
        fy = fmaf(lx[i], ry, fy);
      }
      sx += fx;
      sy += fy;
    }
    for (int d = 0; d < sys.n_defl; ++d) {
      float dax, day;
      alpha_profile(sys.defl[d], sys.ell_c, sys.ell_K, x, y, dax, day);
      sx += dax;
      sy += day;
    }
    I[q] = source_light(sys.src_type, sys.src, sys.src_coef, x - sx, y - sy);
  }
}

__device__ __forceinline__ void unit_bin_down(const DevSystem& sys, const UnitGeom& g, const float* I, int nthr) {
  // dpix^2 times the mean of each pixel's s^2 samples, summed in sample order
  const float wgt = sys.dpix * sys.dpix / (float)g.s2;
  for (int p = threadIdx.x; p < g.bw * g.bh; p += nthr) {
    const int i = g.by * g.bh + p / g.bw, j = g.bx * g.bw + p % g.bw;
    if (i < sys.ny && j < sys.nx) {
      float acc = 0.f;
      for (int t = 0; t < g.s2; ++t) acc += I[p * g.s2 + t];
      sys.out[(size_t)i * sys.nx + j] = acc * wgt;
    }
  }
}

// The slices' node sums as written by unit_partials<FAR = true>
template <int NW>
__device__ __forceinline__ float2 slice_node(const TraceSmem<NW>& sm, int w, int n) {
  return reinterpret_cast<const float2*>(sm.wa[w].queue)[n];
}

// One unit of one system by one CTA of kTraceWarps warps; ends with a CTA barrier.
template <bool FAR = false, bool BLK = false>
__device__ __forceinline__ void trace_unit(const DevSystem& sys, int blk, TraceSmem<kTraceWarps>& sm) {
  const UnitGeom g = unit_geom(sys, blk);
  unit_partials<kTraceWarps, FAR, BLK>(sys, g, 0, sm);
  __syncthreads();
  if constexpr (FAR) unit_sum_nodes(sm.nodes, 32 * kTraceWarps, [&](int sl, int n) { return slice_node(sm, sl, n); });
  unit_finalize<FAR>(sys, g, sm.I, 32 * kTraceWarps, [&](int sl, int k, int l) { return sm.wa[sl].part[k][l]; },
                     sm.nodes, sm.wa[0].box);
  __syncthreads();
  unit_bin_down(sys, g, sm.I, 32 * kTraceWarps);
  __syncthreads();
}

template <int MINB, bool FAR = false, bool BLK = false>
__global__ void __launch_bounds__(32 * kTraceWarps, MINB) trace_image_kernel(const __grid_constant__ DevSystem sys) {
  __shared__ TraceSmem<kTraceWarps> sm;
  trace_unit<FAR, BLK>(sys, blockIdx.x, sm);
}


// Two-pass form: a CTA of kTraceWarps/2 warps sums the 8 slices in two passes (warp w takes
// slices w and w + 4) into the same per-slice areas, then reduces them in slice order like the
// one-CTA form, so its images are bitwise the same; the smaller CTA fits three per SM.
constexpr int kHalfWarps = kTraceWarps / 2;
template <bool FAR = false, bool BLK = false>
__device__ __forceinline__ void trace_unit_2pass(const DevSystem& sys, int blk, TraceSmem<kTraceWarps>& sm) {
  const UnitGeom g = unit_geom(sys, blk);
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass)
    unit_partials<kTraceWarps, FAR, BLK>(sys, g, pass * kHalfWarps, sm, pass * kHalfWarps);
  __syncthreads();
  if constexpr (FAR) unit_sum_nodes(sm.nodes, 32 * kHalfWarps, [&](int sl, int n) { return slice_node(sm, sl, n); });
  unit_finalize<FAR>(sys, g, sm.I, 32 * kHalfWarps, [&](int sl, int k, int l) { return sm.wa[sl].part[k][l]; },
                     sm.nodes, sm.wa[0].box);
  __syncthreads();
  unit_bin_down(sys, g, sm.I, 32 * kHalfWarps);
  __syncthreads();
}

template <bool FAR = false, bool BLK = false>
__global__ void __launch_bounds__(32 * kHalfWarps, 4) trace_image_2pass_kernel(const __grid_constant__ DevSystem sys) {
  __shared__ TraceSmem<kTraceWarps> sm;
  trace_unit_2pass<FAR, BLK>(sys, blockIdx.x, sm);
}

// Cluster form: CL CTAs of kTraceWarps/CL warps share one unit (register budget for 16 warps
// per SM: measured faster than fewer warps with no spills).  CTA r computes slices
// [r*NWC, (r+1)*NWC) of the same split; the leader reads every CTA's partials through
// distributed shared memory in slice order, so the image is bitwise that of the one-CTA form,
// while the finer CTAs balance the tail of the grid across the SMs.
template <int CL, bool FAR = false, bool BLK = false>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(32 * (kTraceWarps / CL), 4 * CL / 2)
trace_cluster_kernel(const __grid_constant__ DevSystem sys) {
  constexpr int NWC = kTraceWarps / CL;
  __shared__ TraceSmem<NWC> sm;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const UnitGeom g = unit_geom(sys, blockIdx.x / CL);
  unit_partials<NWC, FAR, BLK>(sys, g, rank * NWC, sm);
  cluster.sync();
  if (rank == 0) {
    const TraceSmem<NWC>* peers[CL];
#pragma unroll
    for (int r = 0; r < CL; ++r) peers[r] = cluster.map_shared_rank(&sm, r);
    if constexpr (FAR)
      unit_sum_nodes(sm.nodes, 32 * NWC, [&](int sl, int n) { return slice_node(*peers[sl / NWC], sl % NWC, n); });
    unit_finalize<FAR>(sys, g, sm.I, 32 * NWC,
                       [&](int sl, int k, int l) { return peers[sl / NWC]->wa[sl % NWC].part[k][l]; },
                       sm.nodes, sm.wa[0].box);
    __syncthreads();
    unit_bin_down(sys, g, sm.I, 32 * NWC);
  }
  cluster.sync();  // peers keep their shared memory alive until the leader has read it
}

// Persistent forms of the batched launch: CTAs (or clusters) pull unit tickets from the
// header's counter; ticket u belongs to the system whose prefix range [unit_prefix[i],
// unit_prefix[i+1]) contains it.  Every form sums a unit's 8 slices with the same warps' code and
// reduces them in slice order, so a system's image is bitwise that of its single-system call.
//   form 0: CTAs of 4 warps summing the 8 slices in two passes (4 CTAs per SM);
//   form 1: CTAs of 8 warps, one slice each (2 CTAs per SM);
//   form 2: clusters of 2 CTAs x 4 warps, the leader finishing the unit through distributed
//           shared memory (the single-image cluster2x4 form made persistent).
__device__ __forceinline__ int batch_system_of(const int* __restrict__ unit_prefix, int n_sys, int u) {
  int lo = 0, hi = n_sys;  // largest i with unit_prefix[i] <= u
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (unit_prefix[mid] <= u) lo = mid; else hi = mid;
  }
  return lo;
}

template <bool FAR>
__global__ void __launch_bounds__(32 * kHalfWarps, 4) trace_batch_kernel(BatchMeta* __restrict__ meta) {
  __shared__ TraceSmem<kTraceWarps> sm;
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
    const int i = batch_system_of(unit_prefix, n_sys, u);
    const DevSystem& sys = systems[i];
    if (block_layout(sys.s)) trace_unit_2pass<FAR, true>(sys, u - unit_prefix[i], sm);
    else trace_unit_2pass<FAR, false>(sys, u - unit_prefix[i], sm);
  }
}

template <bool FAR>
__global__ void __launch_bounds__(32 * kTraceWarps, 2) trace_batch8_kernel(BatchMeta* __restrict__ meta) {
  __shared__ TraceSmem<kTraceWarps> sm;
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
    const int i = batch_system_of(unit_prefix, n_sys, u);
    const DevSystem& sys = systems[i];
    if (block_layout(sys.s)) trace_unit<FAR, true>(sys, u - unit_prefix[i], sm);
    else trace_unit<FAR, false>(sys, u - unit_prefix[i], sm);
  }
}

template <bool FAR>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(32 * kHalfWarps, 4)
trace_batch_cluster_kernel(BatchMeta* __restrict__ meta) {
  constexpr int NWC = kHalfWarps;
  __shared__ TraceSmem<NWC> sm;
  __shared__ int s_ticket;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int* leader_ticket = cluster.map_shared_rank(&s_ticket, 0);
  const int n_sys = meta->n_sys;
  const int* __restrict__ unit_prefix = meta->unit_prefix;
  const DevSystem* __restrict__ systems = meta->systems;
  const int total = unit_prefix[n_sys];
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) s_ticket = (int)atomicAdd(&meta->trace_counter, 1u);
    cluster.sync();
    const int u = *leader_ticket;
    cluster.sync();  // both CTAs hold the ticket before the leader takes the next one
    if (u >= total) return;
    const int i = batch_system_of(unit_prefix, n_sys, u);
    const DevSystem& sys = systems[i];
    const UnitGeom g = unit_geom(sys, u - unit_prefix[i]);
    if (block_layout(sys.s)) unit_partials<NWC, FAR, true>(sys, g, rank * NWC, sm);
    else unit_partials<NWC, FAR, false>(sys, g, rank * NWC, sm);
    cluster.sync();
    if (rank == 0) {
      const TraceSmem<NWC>* peers[2] = {cluster.map_shared_rank(&sm, 0), cluster.map_shared_rank(&sm, 1)};
      if constexpr (FAR)
        unit_sum_nodes(sm.nodes, 32 * NWC, [&](int sl, int n) { return slice_node(*peers[sl / NWC], sl % NWC, n); });
      unit_finalize<FAR>(sys, g, sm.I, 32 * NWC,
                         [&](int sl, int k, int l) { return peers[sl / NWC]->wa[sl % NWC].part[k][l]; },
                         sm.nodes, sm.wa[0].box);
      __syncthreads();
      unit_bin_down(sys, g, sm.I, 32 * NWC);
    }
    cluster.sync();  // the peer keeps its partials until the leader has read them
  }
}

// Launch of a single-system form (variant) and of a batched form, per instantiation.
template <bool FAR, bool BLK>
inline void launch_trace_form(const DevSystem& sys, int variant, int units, cudaStream_t st) {
  switch (variant) {
    case 1: trace_image_2pass_kernel<FAR, BLK><<<units, 32 * kHalfWarps, 0, st>>>(sys); break;
    case 2: trace_cluster_kernel<2, FAR, BLK><<<units * 2, 32 * (kTraceWarps / 2), 0, st>>>(sys); break;
    case 3: trace_cluster_kernel<4, FAR, BLK><<<units * 4, 32 * (kTraceWarps / 4), 0, st>>>(sys); break;
    case 4: trace_cluster_kernel<8, FAR, BLK><<<units * 8, 32 * (kTraceWarps / 8), 0, st>>>(sys); break;
    default: trace_image_kernel<2, FAR, BLK><<<units, 32 * kTraceWarps, 0, st>>>(sys); break;
  }
}

template <bool FAR>
inline void launch_batch_form(BatchMeta* m, int form, int grid, cudaStream_t st) {
  switch (form) {
    case 1: trace_batch8_kernel<FAR><<<grid, 32 * kTraceWarps, 0, st>>>(m); break;
    case 2: trace_batch_cluster_kernel<FAR><<<grid, 32 * kHalfWarps, 0, st>>>(m); break;
    default: trace_batch_kernel<FAR><<<grid, 32 * kHalfWarps, 0, st>>>(m); break;
  }
}

// The far-field instantiations, compiled in trace_far.cu.
void launch_trace_far(const DevSystem& sys, int variant, int units, cudaStream_t st);
void launch_trace_batch_far(BatchMeta* m, int form, int grid, cudaStream_t st);

}  // namespace ls
