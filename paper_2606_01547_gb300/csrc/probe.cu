// Pipe-rate probes: the measured denominators of the ALU-bound kernels' rooflines.
//
// Each probe kernel runs independent dependency chains of one instruction kind, enough of
// them per thread and enough warps per SM (32) that the pipe, not the chain latency, sets
// the rate.  Every block times its own chains with the SM clock (clock64) between two block
// barriers and records the SM it ran on, so a rate is per SM clock and per SM, whatever the
// clock the GPU ran at: the lane operations of the blocks an SM held over the longest of their
// times.  All blocks of a launch are resident at once (2 x 512 threads per SM, ~40 registers).
#include <algorithm>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.h"
#include "sim_internal.h"

namespace ls {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeBlocksPerSm = 2;
constexpr int kProbeUnroll = 4;

enum ProbeOp { kOpFfma2 = 0, kOpFfma, kOpRsqrt, kOpEx2, kOpLg2, kOpRcp, kProbeOps };
// chains per thread and the lane operations one chain step counts for
__host__ __device__ constexpr int probe_chains(int op) { return op == kOpFfma ? 16 : 8; }
__host__ __device__ constexpr int probe_lane_ops(int op) { return op == kOpFfma2 ? 2 : 1; }

__device__ __forceinline__ float mufu_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One chain step per op.  The MUFU chains stay bounded: rsqrt iterates towards 1, ex2 of a
// negated value towards 0.64, lg2(x + 2) towards 2, rcp(x + 1) towards 0.618 (each MUFU
// chain step with an FP32 operation that keeps the compiler from folding the chain, and that
// runs on another pipe); the FMA chains towards c / (1 - m).
template <int OP>
__global__ void __launch_bounds__(kProbeThreads) pipe_probe_kernel(int iters, float m, float c, float* sink,
                                                                   long long* cycles) {
  constexpr int C = probe_chains(OP);
  float a[C];
  float2 a2[C];
  const float t0v = 1.0f + 1e-6f * (float)threadIdx.x;
#pragma unroll
  for (int i = 0; i < C; ++i) {
    a[i] = t0v + 0.125f * i;
    a2[i] = make_float2(a[i], a[i] + 0.0625f);
  }
  const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < C; ++i) {
        if constexpr (OP == kOpFfma2) a2[i] = __ffma2_rn(a2[i], m2, c2);
        else if constexpr (OP == kOpFfma) a[i] = fmaf(a[i], m, c);
        else if constexpr (OP == kOpRsqrt) a[i] = mufu_rsqrt(a[i]);
        else if constexpr (OP == kOpEx2) a[i] = mufu_ex2(-a[i]);
        else if constexpr (OP == kOpLg2) a[i] = mufu_lg2(a[i] + 2.0f);
        else a[i] = mufu_rcp(a[i] + 1.0f);
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float acc = 0.f;
#pragma unroll
  for (int i = 0; i < C; ++i) acc += (OP == kOpFfma2) ? a2[i].x + a2[i].y : a[i];
  sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = acc;
  if (threadIdx.x == 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    cycles[2 * blockIdx.x] = t1 - t0;
    cycles[2 * blockIdx.x + 1] = (long long)smid;
  }
}

template <int OP>
cudaError_t launch_probe(int blocks, int iters, float* sink, long long* cycles, cudaStream_t st) {
  pipe_probe_kernel<OP><<<blocks, kProbeThreads, 0, st>>>(iters, 0.9999f, 1e-4f, sink, cycles);
  return cudaGetLastError();
}

cudaError_t launch_probe_op(int op, int blocks, int iters, float* sink, long long* cycles, cudaStream_t st) {
  switch (op) {
    case kOpFfma2: return launch_probe<kOpFfma2>(blocks, iters, sink, cycles, st);
    case kOpFfma: return launch_probe<kOpFfma>(blocks, iters, sink, cycles, st);
    case kOpRsqrt: return launch_probe<kOpRsqrt>(blocks, iters, sink, cycles, st);
    case kOpEx2: return launch_probe<kOpEx2>(blocks, iters, sink, cycles, st);
    case kOpLg2: return launch_probe<kOpLg2>(blocks, iters, sink, cycles, st);
    default: return launch_probe<kOpRcp>(blocks, iters, sink, cycles, st);
  }
}

}  // namespace
}  // namespace ls

using namespace ls;

extern "C" int lens_sim_pipe_rates(lens_sim* s, double* rates, int n_rates) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (!rates || n_rates < 1) return fail(s, LENS_ERR_INVALID_ARG, "rates must hold at least one value");
  DeviceGuard g(s->device);
  const int blocks = kProbeBlocksPerSm * (s->sm_count > 0 ? s->sm_count : 1);
  const size_t sink_bytes = (size_t)blocks * kProbeThreads * sizeof(float);  // a multiple of 8
  DevBuffer buf;
  int rc = ensure(s, buf, sink_bytes + (size_t)blocks * 2 * sizeof(long long));
  if (rc) return rc;
  float* sink = (float*)buf.p;
  long long* cycles = (long long*)((char*)buf.p + sink_bytes);
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  std::vector<long long> h(2 * (size_t)blocks);
  const int n = std::min(n_rates, (int)kProbeOps);
  for (int op = 0; op < n && e == cudaSuccess; ++op) {
    // about a million SM clocks per launch at the expected rates; the first launch warms up
    const int iters = op <= kOpFfma ? 2000 : 500;
    e = launch_probe_op(op, blocks, iters / 10, sink, cycles, st);
    if (e == cudaSuccess) e = launch_probe_op(op, blocks, iters, sink, cycles, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h.data(), cycles, h.size() * sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) break;
    // per SM: its blocks' lane operations over the longest of their times; the median over SMs
    const double ops_per_block = (double)kProbeThreads * iters * kProbeUnroll * probe_chains(op) * probe_lane_ops(op);
    std::vector<std::pair<long long, long long>> by_sm(blocks);  // (SM, cycles)
    for (int b = 0; b < blocks; ++b) by_sm[b] = {h[2 * b + 1], std::max(1LL, h[2 * b])};
    std::sort(by_sm.begin(), by_sm.end());
    std::vector<double> per_sm;
    for (size_t i = 0; i < by_sm.size();) {
      size_t j = i;
      long long mx = 1;
      for (; j < by_sm.size() && by_sm[j].first == by_sm[i].first; ++j) mx = std::max(mx, by_sm[j].second);
      per_sm.push_back(ops_per_block * (double)(j - i) / (double)mx);
      i = j;
    }
    std::sort(per_sm.begin(), per_sm.end());
    rates[op] = per_sm[per_sm.size() / 2];
  }
  if (st) cudaStreamDestroy(st);
  release(s, buf);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(s, e, "pipe-rate probe");
  }
  for (int op = n; op < n_rates; ++op) rates[op] = 0.0;
  return LENS_OK;
}
