// Batched image simulation: many lens systems of uneven sizes in one persistent fused launch.
//
// Per call the host packs one metadata block -- system descriptors ordered by per-unit cost
// (largest first), the unit prefix, the subhalo-preparation jobs and the PSF jobs -- copies it
// to the device with one cudaMemcpyAsync, and replays a CUDA graph of three persistent kernels
// (subhalo constants, trace units, PSF tiles).  The kernels read every count and pointer from
// the device header, so one captured graph serves every batch; it is re-captured only when the
// workspace moves, the largest PSF grows, or the persistent trace form or the far-field on/off
// setting changes (the far-field kappa itself travels in each system's descriptor).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "kernels.h"
#include "lens_sim.h"
#include "sim_internal.h"

namespace ls {

// Persistent subhalo preparation over the header's jobs (grid-stride over jobs, then subhalos).
__global__ void prep_batch_meta_kernel(const BatchMeta* __restrict__ meta) {
  const int n_jobs = meta->n_prep;
  for (int jb = blockIdx.x; jb < n_jobs; jb += gridDim.x) {
    const PrepJob j = meta->prep[jb];
    for (int t = threadIdx.x; t < j.n; t += blockDim.x) {
      tnfw_write_table(j.soa[t], j.soa[j.ld + t], j.soa[2 * j.ld + t], j.soa[3 * j.ld + t], j.soa[4 * j.ld + t], t,
                       j.n, j.tab);
    }
  }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Host-side estimate of one unit's cost in pair evaluations: 288 samples x (subhalos + the
// per-sample finalise, worth about eight pairs).
static double unit_cost(const lens_system& y, int n_sub) {
  (void)y;
  return (double)kUnitPts * 32.0 * ((double)n_sub + 8.0);
}

int capture_batch_graph(lens_sim* s, int kmax) {
  if (s->graph_exec) {
    cudaGraphExecDestroy(s->graph_exec);
    s->graph_exec = nullptr;
  }
  if (!s->cap_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(s, e, "create capture stream");
  }
  const BatchMeta* meta = (const BatchMeta*)s->batch_meta.p;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(s, e, "begin capture");
  prep_batch_meta_kernel<<<s->sm_count * 4, 256, 0, s->cap_stream>>>(meta);
  cudaError_t e1 = cudaGetLastError();
  const bool far = s->far_kappa > 0.f;
  cudaError_t e2 = launch_trace_batch_meta(meta, s->batch_form, trace_batch_grid(s->sm_count, s->batch_form), far,
                                           s->cap_stream);
  cudaError_t e3 = launch_conv_batch_meta(meta, kmax, conv_batch_grid(s->sm_count, kmax), s->cap_stream);
  e = cudaStreamEndCapture(s->cap_stream, &graph);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(s, e != cudaSuccess ? e : (e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3)),
                     "capture batch graph");
  }
  e = cudaGraphInstantiate(&s->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    s->graph_exec = nullptr;
    return cuda_fail(s, e, "instantiate batch graph");
  }
  s->graph_meta = s->batch_meta.p;
  s->graph_kmax = kmax;
  s->graph_form = s->batch_form;
  s->graph_far = far;
  return LENS_OK;
}

int run_image_batch(lens_sim* s, const lens_system* systems, int n, float* const* outs, cudaStream_t st) {
  // ---- sizes and order
  std::vector<int> nsub(n), units(n), order(n);
  std::vector<double> cost(n);
  std::vector<bool> dev_out(n);
  size_t pix_total = 0, raw_total = 0, tab_total = 0, stage_total = 0;
  int kmax = 1, n_prep = 0, n_conv = 0;
  for (int i = 0; i < n; ++i) {
    const lens_system& y = systems[i];
    nsub[i] = sub_count(s, y);
    units[i] = unit_count(y.grid.nx, y.grid.ny, y.grid.supersample);
    cost[i] = unit_cost(y, nsub[i]);
    dev_out[i] = is_device_ptr(outs[i]);
    const size_t npix = (size_t)y.grid.nx * y.grid.ny;
    if (y.psf_id >= 0) {
      pix_total += align256(npix * sizeof(float));
      PsfEntry pe;
      if (s->res->psf(y.psf_id, &pe)) kmax = std::max(kmax, pe.k);
      ++n_conv;
    }
    if (!dev_out[i]) stage_total += align256(npix * sizeof(float));
    if (y.subhalo_table < 0 && nsub[i] > 0) {
      tab_total += align256((size_t)kTableStride * sizeof(float4) * nsub[i]);
      if (!is_device_ptr(y.subhalos)) raw_total += align256(5 * sizeof(float) * (size_t)nsub[i]);
      ++n_prep;
    }
  }
  kmax = std::max(kmax, s->res->kmax());  // graph smem covers every registered PSF
  std::iota(order.begin(), order.end(), 0);
  if (s->batch_order == 0)  // the longest units first (otherwise the queue keeps the given order)
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });

  // ---- device workspace (metadata block, tables, raw copies, unconvolved images, staging)
  // systems with an elliptical multipole carry their harmonics in a side region of the block
  int n_ell = 0;
  for (int i = 0; i < n; ++i) n_ell += count_deflectors(systems[i], LENS_MULTIPOLE_ELL) > 0;
  const size_t ell_bytes = align256(sizeof(float) * kEllTableFloats * (size_t)n_ell);
  const size_t meta_bytes = align256(sizeof(BatchMeta)) + align256(sizeof(DevSystem) * n) +
                            align256(sizeof(int) * (n + 1)) + align256(sizeof(PrepJob) * (n + 1)) +
                            align256(sizeof(ConvJob) * (n + 1)) + ell_bytes;
  int rc;
  const size_t meta_cap = std::max(meta_bytes, align256(sizeof(BatchMeta)) + align256(sizeof(DevSystem) * s->max_batch) +
                          align256(sizeof(int) * (s->max_batch + 1)) + align256(sizeof(PrepJob) * (s->max_batch + 1)) +
                          align256(sizeof(ConvJob) * (s->max_batch + 1)));
  if ((rc = ensure(s, s->batch_meta, meta_cap))) return rc;
  if ((rc = ensure(s, s->batch_data, std::max<size_t>(256, tab_total + raw_total + pix_total + stage_total)))) return rc;
  if (!s->pinned || s->pinned_cap < meta_bytes) {
    if (s->pinned) {
      cudaEventSynchronize(s->pinned_ready);
      cudaFreeHost(s->pinned);
      s->pinned = nullptr;
    }
    cudaError_t e = cudaMallocHost(&s->pinned, meta_cap);
    if (e != cudaSuccess) { s->pinned = nullptr; return fail(s, LENS_ERR_OOM, "pinned staging: %s", cudaGetErrorString(e)); }
    s->pinned_cap = meta_cap;
  }
  if (!s->pinned_ready) {
    cudaError_t e = cudaEventCreateWithFlags(&s->pinned_ready, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(s, e, "create event");
  } else {
    cudaError_t e = cudaEventSynchronize(s->pinned_ready);  // the previous call's copy has read the staging
    if (e != cudaSuccess) return cuda_fail(s, e, "staging event");
  }

  // ---- carve the data region
  char* dbase = (char*)s->batch_data.p;
  std::vector<float4*> tabs(n, nullptr);
  std::vector<const float*> soas(n, nullptr);
  std::vector<float*> raw_img(n, nullptr), stage(n, nullptr);
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    const lens_system& y = systems[i];
    if (y.subhalo_table < 0 && nsub[i] > 0) {
      tabs[i] = (float4*)(dbase + off);
      off += align256((size_t)kTableStride * sizeof(float4) * nsub[i]);
    }
  }
  for (int i = 0; i < n; ++i) {
    const lens_system& y = systems[i];
    if (y.subhalo_table < 0 && nsub[i] > 0) {
      if (is_device_ptr(y.subhalos)) {
        soas[i] = y.subhalos;
      } else {
        float* dst = (float*)(dbase + off);
        off += align256(5 * sizeof(float) * (size_t)nsub[i]);
        cudaError_t e = cudaMemcpyAsync(dst, y.subhalos, 5 * sizeof(float) * (size_t)nsub[i],
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(s, e, "copy subhalos to device");
        soas[i] = dst;
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    const size_t npix = (size_t)systems[i].grid.nx * systems[i].grid.ny;
    if (systems[i].psf_id >= 0) {
      raw_img[i] = (float*)(dbase + off);
      off += align256(npix * sizeof(float));
    }
    if (!dev_out[i]) {
      stage[i] = (float*)(dbase + off);
      off += align256(npix * sizeof(float));
    }
  }

  // ---- pack the metadata block in pinned memory (device addresses computed from the base)
  char* hb = (char*)s->pinned;
  char* db = (char*)s->batch_meta.p;
  size_t o_hdr = 0, o_sys = align256(sizeof(BatchMeta));
  size_t o_pre = o_sys + align256(sizeof(DevSystem) * n);
  size_t o_prep = o_pre + align256(sizeof(int) * (n + 1));
  size_t o_conv = o_prep + align256(sizeof(PrepJob) * (n + 1));
  size_t o_ell = o_conv + align256(sizeof(ConvJob) * (n + 1));
  BatchMeta* hm = (BatchMeta*)(hb + o_hdr);
  DevSystem* hsys = (DevSystem*)(hb + o_sys);
  int* hpre = (int*)(hb + o_pre);
  PrepJob* hprep = (PrepJob*)(hb + o_prep);
  ConvJob* hconv = (ConvJob*)(hb + o_conv);
  std::memset(hm, 0, sizeof(BatchMeta));
  int u = 0, ip = 0, ic = 0, tiles = 0;
  for (int r = 0; r < n; ++r) {
    const int i = order[r];
    const lens_system& y = systems[i];
    DevSystem& d = hsys[r];
    fill_dev_system(y, d);
    d.far_kappa = s->far_kappa;
    if (count_deflectors(y, LENS_MULTIPOLE_ELL) > 0) {
      d.ell_K = ell_table(y, (float*)(hb + o_ell));
      d.ell_c = (const float*)(db + o_ell);
      o_ell += sizeof(float) * kEllTableFloats;
    }
    if (y.subhalo_table >= 0) {
      SubTable t;
      s->res->table(y.subhalo_table, &t);
      d.sub = t.d;
      d.n_sub = t.n;
    } else {
      d.sub = tabs[i];
      d.n_sub = nsub[i];
      if (nsub[i] > 0) hprep[ip++] = PrepJob{soas[i], tabs[i], nsub[i], nsub[i]};
    }
    float* final_dst = dev_out[i] ? outs[i] : stage[i];
    d.out = (y.psf_id >= 0) ? raw_img[i] : final_dst;
    hpre[r] = u;
    u += units[i];
    if (y.psf_id >= 0) {
      PsfEntry p;
      s->res->psf(y.psf_id, &p);
      hconv[ic++] = ConvJob{raw_img[i], final_dst, p.d, y.grid.ny, y.grid.nx, p.k, tiles};
      tiles += ((y.grid.nx + 31) / 32) * ((y.grid.ny + 31) / 32);
    }
  }
  hpre[n] = u;
  hconv[ic] = ConvJob{nullptr, nullptr, nullptr, 0, 0, 0, tiles};
  hm->n_sys = n;
  hm->n_prep = ip;
  hm->n_conv = ic;
  hm->kmax = kmax;
  hm->systems = (const DevSystem*)(db + o_sys);
  hm->unit_prefix = (const int*)(db + o_pre);
  hm->prep = (const PrepJob*)(db + o_prep);
  hm->conv = (const ConvJob*)(db + o_conv);
  cudaError_t e = cudaMemcpyAsync(db, hb, meta_bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(s, e, "copy batch metadata");
  e = cudaEventRecord(s->pinned_ready, st);
  if (e != cudaSuccess) return cuda_fail(s, e, "record staging event");

  // ---- launch the captured graph (re-captured if the workspace moved or a PSF grew)
  if (!s->graph_exec || s->graph_meta != s->batch_meta.p || s->graph_kmax < kmax || s->graph_form != s->batch_form ||
      s->graph_far != (s->far_kappa > 0.f)) {
    if ((rc = capture_batch_graph(s, std::max(kmax, s->graph_kmax)))) return rc;
  }
  e = cudaGraphLaunch(s->graph_exec, st);
  if (e != cudaSuccess) return cuda_fail(s, e, "launch batch graph");

  // ---- host outputs
  bool host_out = false;
  for (int i = 0; i < n; ++i) {
    if (dev_out[i]) continue;
    const size_t npix = (size_t)systems[i].grid.nx * systems[i].grid.ny;
    e = cudaMemcpyAsync(outs[i], stage[i], npix * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "copy image to host");
    host_out = true;
  }
  if (host_out) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(s, e, "stream synchronize");
  }
  return LENS_OK;
}

}  // namespace ls

extern "C" {

int lens_sim_set_batch_schedule(lens_sim* s, int form, int order) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (form < 0 || form >= ls::kBatchForms || order < 0 || order > 1)
    return ls::fail(s, LENS_ERR_INVALID_ARG, "batch schedule (%d, %d) not in [0, %d) x [0, 1]", form, order,
                    ls::kBatchForms);
  s->batch_form = form;
  s->batch_order = order;
  return LENS_OK;
}

int lens_sim_autotune_batch(lens_sim* s, const lens_system* systems, int n_sys, float* const* out_images, int reps,
                            int* best_form, int* best_order, float* ms, void* stream) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (!systems || !out_images || !best_form || !best_order || n_sys < 2 || reps < 1 || reps > 1000)
    return ls::fail(s, LENS_ERR_INVALID_ARG, "bad batch autotune arguments (at least 2 systems)");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return ls::cuda_fail(s, cudaGetLastError(), "create event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ls::cuda_fail(s, cudaGetLastError(), "create event");
  }
  const int form0 = s->batch_form, order0 = s->batch_order;
  float best = 3.0e38f;
  int bf = form0, bo = order0, rc = LENS_OK;
  for (int f = 0; f < ls::kBatchForms && rc == LENS_OK; ++f) {
    for (int o = 0; o < 2 && rc == LENS_OK; ++o) {
      s->batch_form = f;
      s->batch_order = o;
      rc = lens_sim_image(s, systems, n_sys, out_images, stream);  // warm-up (captures the graph)
      if (rc) break;
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && rc == LENS_OK; ++r) rc = lens_sim_image(s, systems, n_sys, out_images, stream);
      cudaEventRecord(e1, st);
      if (rc) break;
      cudaError_t e = cudaEventSynchronize(e1);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e != cudaSuccess) {
        rc = ls::cuda_fail(s, e, "batch autotune timing");
        break;
      }
      t /= (float)reps;
      if (ms) ms[f * 2 + o] = t;
      if (t < best) {
        best = t;
        bf = f;
        bo = o;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->batch_form = rc ? form0 : bf;
  s->batch_order = rc ? order0 : bo;
  if (rc) return rc;
  *best_form = bf;
  *best_order = bo;
  return LENS_OK;
}

}  // extern "C"
