// Serving loop (lens_serve_*): continuous batching of image-simulation and likelihood+gradient
// requests on one GPU.
//
// Requests enter a FIFO queue.  A worker thread admits them by an estimated device-memory
// budget into idle stream slots; each slot owns a lens_sim handle (its own workspace and
// captured batch graph) that shares the server's resident PSFs and subhalo tables, plus
// pinned staging for asynchronous copies.  The images of one admission go out as one batched
// launch, the likelihood requests as lens_sim_grad calls on the same stream, and a host
// callback at the end of the stream's work wakes the worker, which copies results to the
// caller's buffers and records latency.  Requests that arrive while slots are busy are
// admitted as soon as a slot and budget free up, so their work overlaps on the device.
// Every host-side wait is bounded; nothing spins on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "lens_sim.h"
#include "sim_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { kQueued, kRunning, kDone, kCancelled, kFailed };

struct Req {
  unsigned long long ticket = 0;
  lens_request r{};
  std::vector<lens_profile> defl;
  std::vector<float> coef;  // source amplitudes (SHAPELETS), copied at submit
  size_t est_bytes = 0;
  Clock::time_point t_submit, t_done;
  int state = kQueued;
  int status = LENS_OK;
  size_t out_off = 0;  // offset (floats) of this request's outputs in the slot buffers
  size_t in_off = 0;   // offset (floats) of its inputs (likelihood)
  size_t sub_off = 0;  // offset (floats) of its subhalo arrays in the packed batch copy
  const float* sub_dev = nullptr;
};

struct Slot {
  lens_sim* sim = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<Req*> batch;
  bool busy = false;
  bool complete = false;
  size_t est_bytes = 0;
  float* d_out = nullptr;
  float* h_out = nullptr;
  size_t out_cap = 0;
  float* d_in = nullptr;
  float* h_in = nullptr;
  size_t in_cap = 0;
  float* d_sub = nullptr;  // the batch's subhalo arrays, packed (pinned copy -> one async H2D)
  float* h_sub = nullptr;
  size_t sub_cap = 0;
};

size_t npix_of(const lens_request& r) { return (size_t)r.sys.grid.nx * (size_t)r.sys.grid.ny; }

}  // namespace

struct lens_server {
  lens_sim* main = nullptr;
  std::vector<Slot*> slots;
  int max_inflight = 0;
  int max_batch = 64;
  size_t budget = 0;
  size_t in_use = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::unordered_map<unsigned long long, Req*> reqs;
  unsigned long long next_ticket = 1;
  int outstanding = 0;
  bool paused = false;
  std::atomic<bool> stop{false};
  std::thread worker;
  std::vector<double> lat_ms;
  Clock::time_point t_first, t_last;
  bool have_first = false;
  std::mutex err_mu;
  std::string last_err;  // text of the most recent failed request
};

namespace {

void note_error(lens_server* srv, const char* what) {
  std::lock_guard<std::mutex> lk(srv->err_mu);
  srv->last_err = what ? what : "unknown error";
}

// Estimated device bytes of one request while it runs.
size_t estimate_bytes(lens_server* srv, const lens_request& r) {
  const size_t npix = npix_of(r);
  const size_t s2 = (size_t)r.sys.grid.supersample * r.sys.grid.supersample;
  const size_t nsub = r.sys.subhalo_table >= 0 ? 0 : (size_t)std::max(r.sys.n_subhalos, 0);
  (void)srv;
  if (r.kind == 0) return npix * 4 * 3 + nsub * (20 + 176) + 4096;
  return npix * 4 * 6 + npix * s2 * 8 + nsub * (20 + 176) + 64 * 4 * 16 + 4096;
}

int grow(float** d, float** h, size_t* cap, size_t need) {
  if (need <= *cap) return LENS_OK;
  size_t want = std::max(need, *cap * 2);
  if (*d) cudaFree(*d);
  if (*h) cudaFreeHost(*h);
  *d = nullptr;
  *h = nullptr;
  *cap = 0;
  if (cudaMalloc((void**)d, want * sizeof(float)) != cudaSuccess) { cudaGetLastError(); return LENS_ERR_OOM; }
  if (cudaMallocHost((void**)h, want * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(*d);
    *d = nullptr;
    return LENS_ERR_OOM;
  }
  *cap = want;
  return LENS_OK;
}

void CUDART_CB slot_done_cb(void* arg);

struct CbArg {
  lens_server* srv;
  Slot* slot;
};

// Issue one admitted batch on an idle slot (worker thread, no lock held).
void issue(lens_server* srv, Slot* sl, CbArg* cb) {
  size_t out_need = 0, in_need = 0;
  for (Req* q : sl->batch) {
    q->out_off = out_need;
    out_need += (q->r.kind == 0) ? npix_of(q->r) : 16;
    q->in_off = in_need;
    if (q->r.kind == 1) in_need += npix_of(q->r) + 16;
  }
  size_t sub_need = 0;
  for (Req* q : sl->batch) {
    q->sub_off = sub_need;
    q->sub_dev = nullptr;
    if (q->r.sys.subhalo_table < 0 && q->r.sys.n_subhalos > 0 && !ls::is_device_ptr(q->r.sys.subhalos))
      sub_need += 5 * (size_t)q->r.sys.n_subhalos;
  }
  int rc = grow(&sl->d_out, &sl->h_out, &sl->out_cap, std::max<size_t>(out_need, 1));
  if (rc == LENS_OK) rc = grow(&sl->d_in, &sl->h_in, &sl->in_cap, std::max<size_t>(in_need, 1));
  if (rc == LENS_OK) rc = grow(&sl->d_sub, &sl->h_sub, &sl->sub_cap, std::max<size_t>(sub_need, 1));
  if (rc == LENS_OK && sub_need > 0) {
    // host subhalo arrays: pack into pinned memory, one asynchronous copy for the batch
    for (Req* q : sl->batch) {
      if (q->r.sys.subhalo_table < 0 && q->r.sys.n_subhalos > 0 && !ls::is_device_ptr(q->r.sys.subhalos)) {
        std::memcpy(sl->h_sub + q->sub_off, q->r.sys.subhalos, 5 * sizeof(float) * q->r.sys.n_subhalos);
        q->sub_dev = sl->d_sub + q->sub_off;
      }
    }
    if (cudaMemcpyAsync(sl->d_sub, sl->h_sub, sub_need * sizeof(float), cudaMemcpyHostToDevice, sl->stream) !=
        cudaSuccess) {
      cudaGetLastError();
      rc = LENS_ERR_CUDA;
    }
  }
  if (rc != LENS_OK) {
    for (Req* q : sl->batch) q->status = rc;
    note_error(srv, "staging the batch's inputs failed");
  } else {
    // images: one (batched) call
    std::vector<lens_system> sys;
    std::vector<float*> outs;
    std::vector<Req*> img;
    for (Req* q : sl->batch)
      if (q->r.kind == 0) {
        lens_system y = q->r.sys;
        y.deflectors = q->defl.data();
        y.source_coeffs = q->coef.empty() ? nullptr : q->coef.data();
        if (q->sub_dev) y.subhalos = q->sub_dev;
        sys.push_back(y);
        outs.push_back(sl->d_out + q->out_off);
        img.push_back(q);
      }
    if (!img.empty()) {
      int st = lens_sim_image(sl->sim, sys.data(), (int)sys.size(), outs.data(), sl->stream);
      if (st != LENS_OK) {
        // re-issue one by one so that one bad request does not fail the others
        for (size_t k = 0; k < img.size(); ++k) {
          img[k]->status = lens_sim_image(sl->sim, &sys[k], 1, &outs[k], sl->stream);
          if (img[k]->status != LENS_OK) note_error(srv, lens_sim_last_error(sl->sim));
        }
      }
      for (Req* q : img)
        if (q->status == LENS_OK)
          cudaMemcpyAsync(sl->h_out + q->out_off, sl->d_out + q->out_off, npix_of(q->r) * sizeof(float),
                          cudaMemcpyDeviceToHost, sl->stream);
    }
    // likelihood + gradient: one call per request on the same stream
    for (Req* q : sl->batch) {
      if (q->r.kind != 1) continue;
      const size_t npix = npix_of(q->r);
      float* hin = sl->h_in + q->in_off;
      float* din = sl->d_in + q->in_off;
      std::memcpy(hin, q->r.data, npix * sizeof(float));
      std::memcpy(hin + npix, q->r.params, LENS_N_FREE_PARAMS * sizeof(float));
      cudaMemcpyAsync(din, hin, (npix + LENS_N_FREE_PARAMS) * sizeof(float), cudaMemcpyHostToDevice, sl->stream);
      lens_system y = q->r.sys;
      y.deflectors = q->defl.data();
      y.source_coeffs = q->coef.empty() ? nullptr : q->coef.data();
      if (q->sub_dev) y.subhalos = q->sub_dev;
      float* dout = sl->d_out + q->out_off;
      q->status = lens_sim_grad(sl->sim, &y, din, q->r.sigma_bkg, q->r.t_exp, din + npix, 1, dout,
                                q->r.out_grad ? dout + 1 : nullptr, sl->stream);
      if (q->status != LENS_OK) note_error(srv, lens_sim_last_error(sl->sim));
      if (q->status == LENS_OK)
        cudaMemcpyAsync(sl->h_out + q->out_off, dout, 16 * sizeof(float), cudaMemcpyDeviceToHost, sl->stream);
    }
  }
  cb->srv = srv;
  cb->slot = sl;
  if (cudaLaunchHostFunc(sl->stream, slot_done_cb, cb) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(sl->stream);
    slot_done_cb(cb);
  }
}

void CUDART_CB slot_done_cb(void* arg) {
  CbArg* cb = (CbArg*)arg;
  std::lock_guard<std::mutex> lk(cb->srv->mu);
  cb->slot->complete = true;
  cb->srv->cv_work.notify_all();
}

// Completion of a slot (worker thread, lock held on entry and exit): results to the caller,
// latency, budget.  The copies to the callers' buffers run with the lock released, so that
// submits and waits are not held up by them (only the worker touches a running batch).
void finish(lens_server* srv, Slot* sl, std::unique_lock<std::mutex>& lk) {
  // The host callback ran after every earlier operation of the stream completed; while the
  // callback itself retires the stream may still report "not ready", which is no error.
  cudaError_t e = cudaStreamQuery(sl->stream);
  if (e == cudaErrorNotReady) {
    cudaGetLastError();  // "not ready" must not linger as this thread's last error
    e = cudaSuccess;
  }
  if (e != cudaSuccess) note_error(srv, cudaGetErrorString(e));
  lk.unlock();
  for (Req* q : sl->batch) {
    if (q->status == LENS_OK && e != cudaSuccess) q->status = LENS_ERR_CUDA;
    if (q->status == LENS_OK) {
      if (q->r.kind == 0) {
        std::memcpy(q->r.out, sl->h_out + q->out_off, npix_of(q->r) * sizeof(float));
      } else {
        q->r.out[0] = sl->h_out[q->out_off];
        if (q->r.out_grad) std::memcpy(q->r.out_grad, sl->h_out + q->out_off + 1, LENS_N_FREE_PARAMS * sizeof(float));
      }
    }
  }
  lk.lock();
  const auto now = Clock::now();
  for (Req* q : sl->batch) {
    q->state = q->status == LENS_OK ? kDone : kFailed;
    q->t_done = now;
    srv->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - q->t_submit).count());
    srv->t_last = now;
    srv->outstanding--;
  }
  srv->in_use -= sl->est_bytes;
  sl->est_bytes = 0;
  sl->batch.clear();
  sl->busy = false;
  sl->complete = false;
  srv->cv_done.notify_all();
}

void worker_main(lens_server* srv) {
  cudaSetDevice(srv->main->device);
  std::vector<CbArg> cbs(srv->slots.size());
  std::unique_lock<std::mutex> lk(srv->mu);
  while (!srv->stop.load()) {
    for (Slot* sl : srv->slots)
      if (sl->busy && sl->complete) finish(srv, sl, lk);
    bool issued = false;
    if (!srv->paused) {
      for (size_t si = 0; si < srv->slots.size() && !srv->queue.empty(); ++si) {
        Slot* sl = srv->slots[si];
        if (sl->busy) continue;
        // admit from the queue front while the budget allows (always at least one request)
        while (!srv->queue.empty() && (int)sl->batch.size() < srv->max_batch) {
          Req* q = srv->queue.front();
          if (!sl->batch.empty() && srv->in_use + q->est_bytes > srv->budget) break;
          if (sl->batch.empty() && srv->in_use > 0 && srv->in_use + q->est_bytes > srv->budget) break;
          srv->queue.pop_front();
          q->state = kRunning;
          srv->in_use += q->est_bytes;
          sl->est_bytes += q->est_bytes;
          sl->batch.push_back(q);
        }
        if (sl->batch.empty()) break;
        sl->busy = true;
        lk.unlock();
        issue(srv, sl, &cbs[si]);
        lk.lock();
        issued = true;
      }
    }
    if (!issued) srv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
  }
  // drain: wait (bounded) for the slots' work, then release
  for (Slot* sl : srv->slots)
    if (sl->busy) {
      lk.unlock();
      cudaStreamSynchronize(sl->stream);
      lk.lock();
      if (!sl->complete) sl->complete = true;
      finish(srv, sl, lk);
    }
}

}  // namespace

extern "C" {

int lens_serve_create(const lens_sim_config* config, int max_inflight, lens_server** out) {
  if (!out || max_inflight < 1) return LENS_ERR_INVALID_ARG;
  *out = nullptr;
  lens_sim_config c{0, 0, 0, 0};
  if (config) c = *config;
  lens_server* srv = new (std::nothrow) lens_server();
  if (!srv) return LENS_ERR_OOM;
  int rc = lens_sim_create(&c, &srv->main);
  if (rc != LENS_OK) {
    delete srv;
    return rc;
  }
  cudaSetDevice(c.device);
  srv->max_inflight = max_inflight;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  srv->budget = c.mem_budget_bytes ? c.mem_budget_bytes : (size_t)(0.5 * (double)free_b);
  const int n_slots = 4;
  for (int i = 0; i < n_slots; ++i) {
    Slot* sl = new Slot();
    lens_sim_config sc = c;
    sc.mem_budget_bytes = 0;
    if (lens_sim_create(&sc, &sl->sim) != LENS_OK || cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      if (sl->sim) lens_sim_destroy(sl->sim);
      delete sl;
      lens_serve_destroy(srv);
      return LENS_ERR_CUDA;
    }
    sl->sim->res = srv->main->res;  // share registered PSFs and subhalo tables
    sl->sim->owns_resident = false;
    srv->slots.push_back(sl);
  }
  srv->worker = std::thread(worker_main, srv);
  *out = srv;
  return LENS_OK;
}

lens_sim* lens_serve_sim(lens_server* srv) { return srv ? srv->main : nullptr; }

const char* lens_serve_last_error(lens_server* srv) {
  static thread_local std::string copy;
  if (!srv) return "null server";
  std::lock_guard<std::mutex> lk(srv->err_mu);
  copy = srv->last_err;
  return copy.c_str();
}

int lens_serve_pause(lens_server* srv, int paused) {
  if (!srv) return LENS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->paused = paused != 0;
  srv->cv_work.notify_all();
  return LENS_OK;
}

int lens_serve_submit(lens_server* srv, const lens_request* req, unsigned long long* ticket) {
  if (!srv || !req || !ticket) return LENS_ERR_INVALID_ARG;
  if (req->kind != 0 && req->kind != 1) return LENS_ERR_INVALID_ARG;
  if (!req->out) return LENS_ERR_INVALID_ARG;
  if (req->kind == 1 && (!req->data || !req->params)) return LENS_ERR_INVALID_ARG;
  if (req->sys.grid.nx < 1 || req->sys.grid.ny < 1 || req->sys.grid.nx > 16384 || req->sys.grid.ny > 16384)
    return LENS_ERR_INVALID_ARG;
  if (req->sys.n_deflectors < 0 || req->sys.n_deflectors > LENS_MAX_DEFLECTORS ||
      (req->sys.n_deflectors > 0 && !req->sys.deflectors))
    return LENS_ERR_INVALID_ARG;
  Req* q = new (std::nothrow) Req();
  if (!q) return LENS_ERR_OOM;
  q->r = *req;
  q->defl.assign(req->sys.deflectors, req->sys.deflectors + req->sys.n_deflectors);
  if (req->sys.source_coeffs && req->sys.n_source_coeffs > 0 && req->sys.n_source_coeffs <= LENS_MAX_SHAPELET_COEFFS)
    q->coef.assign(req->sys.source_coeffs, req->sys.source_coeffs + req->sys.n_source_coeffs);
  q->est_bytes = estimate_bytes(srv, *req);
  std::lock_guard<std::mutex> lk(srv->mu);
  if (q->est_bytes > srv->budget) {
    delete q;
    return LENS_ERR_OOM;
  }
  if (srv->outstanding >= srv->max_inflight) {
    delete q;
    return LENS_ERR_BUSY;
  }
  q->ticket = srv->next_ticket++;
  q->t_submit = Clock::now();
  if (!srv->have_first) {
    srv->t_first = q->t_submit;
    srv->have_first = true;
  }
  srv->reqs[q->ticket] = q;
  srv->queue.push_back(q);
  srv->outstanding++;
  *ticket = q->ticket;
  srv->cv_work.notify_all();
  return LENS_OK;
}

static int final_status(Req* q) { return q->state == kCancelled ? LENS_ERR_CANCELLED : q->status; }

int lens_serve_wait(lens_server* srv, unsigned long long ticket, int timeout_ms) {
  if (!srv || timeout_ms < 0) return LENS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return LENS_ERR_INVALID_ARG;
  Req* q = it->second;
  const bool ok = srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
    return q->state == kDone || q->state == kFailed || q->state == kCancelled;
  });
  if (!ok) return LENS_ERR_TIMEOUT;
  const int st = final_status(q);
  srv->reqs.erase(ticket);
  delete q;
  return st;
}

int lens_serve_poll(lens_server* srv, unsigned long long ticket) {
  if (!srv) return LENS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return LENS_ERR_INVALID_ARG;
  Req* q = it->second;
  if (q->state == kQueued || q->state == kRunning) return LENS_ERR_BUSY;
  const int st = final_status(q);
  srv->reqs.erase(ticket);
  delete q;
  return st;
}

int lens_serve_cancel(lens_server* srv, unsigned long long ticket) {
  if (!srv) return LENS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return LENS_ERR_INVALID_ARG;
  Req* q = it->second;
  if (q->state == kRunning) return LENS_ERR_BUSY;
  if (q->state != kQueued) return LENS_OK;
  srv->queue.erase(std::remove(srv->queue.begin(), srv->queue.end(), q), srv->queue.end());
  q->state = kCancelled;
  srv->outstanding--;
  srv->cv_done.notify_all();
  return LENS_OK;
}

int lens_serve_stats(lens_server* srv, double* p50_ms, double* p99_ms, double* requests_per_s) {
  if (!srv) return LENS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  std::vector<double> v = srv->lat_ms;
  double p50 = 0, p99 = 0, rate = 0;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    p50 = v[(size_t)(0.50 * (v.size() - 1))];
    p99 = v[(size_t)(0.99 * (v.size() - 1))];
    const double span = std::chrono::duration<double>(srv->t_last - srv->t_first).count();
    rate = span > 0 ? (double)v.size() / span : 0.0;
  }
  if (p50_ms) *p50_ms = p50;
  if (p99_ms) *p99_ms = p99;
  if (requests_per_s) *requests_per_s = rate;
  return LENS_OK;
}

int lens_serve_reset_stats(lens_server* srv) {
  if (!srv) return LENS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->lat_ms.clear();
  srv->have_first = false;
  return LENS_OK;
}

void lens_serve_destroy(lens_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop.store(true);
    srv->paused = false;
    srv->cv_work.notify_all();
  }
  if (srv->worker.joinable()) srv->worker.join();
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    for (Req* q : srv->queue) {
      q->state = kCancelled;
    }
    srv->queue.clear();
    for (auto& kv : srv->reqs) delete kv.second;
    srv->reqs.clear();
    srv->cv_done.notify_all();
  }
  for (Slot* sl : srv->slots) {
    if (sl->stream) cudaStreamSynchronize(sl->stream);
    if (sl->d_out) cudaFree(sl->d_out);
    if (sl->h_out) cudaFreeHost(sl->h_out);
    if (sl->d_in) cudaFree(sl->d_in);
    if (sl->h_in) cudaFreeHost(sl->h_in);
    if (sl->d_sub) cudaFree(sl->d_sub);
    if (sl->h_sub) cudaFreeHost(sl->h_sub);
    if (sl->stream) cudaStreamDestroy(sl->stream);
    if (sl->sim) lens_sim_destroy(sl->sim);
    delete sl;
  }
  srv->slots.clear();
  if (srv->main) lens_sim_destroy(srv->main);
  delete srv;
}

}  // extern "C"
