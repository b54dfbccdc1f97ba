// Internal state of a lens_sim handle (shared by the ABI translation units).
#pragma once

#include <algorithm>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "lens_device.cuh"
#include "lens_sim.h"

namespace ls {

struct DevBuffer {
  void* p = nullptr;
  size_t cap = 0;
};

struct PsfEntry {
  float* d = nullptr;
  int k = 0;
  float* dflip = nullptr;  // the kernel turned by 180 degrees: correlation as a convolution
};

struct SubTable {
  float4* d = nullptr;
  int n = 0;
};

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev);
  ~DeviceGuard();

 private:
  int prev_ = 0;
  int dev_ = 0;
};

int fail(lens_sim* s, int code, const char* fmt, ...);
int cuda_fail(lens_sim* s, cudaError_t e, const char* what);
bool is_device_ptr(const void* p);
// True for device memory of a GPU other than the current one (a kernel launched here would
// read it through a peer mapping, or fault without one).
bool on_other_device(const void* p);
// Grid checks of validate_system: 1..16384 pixels per side, supersampling in
// [1, LENS_MAX_SUPERSAMPLE], a finite positive pixel scale and a finite centre.
int validate_grid(lens_sim* s, const lens_grid& g);
int ensure(lens_sim* s, DevBuffer& b, size_t bytes);
void release(lens_sim* s, DevBuffer& b);
int validate_system(lens_sim* s, const lens_system& y, bool need_grid);
// Host-mapped flag of the TMA convolution's bounded waits: allocated on first use; returns
// LENS_ERR_TIMEOUT (and clears it) if an earlier wait expired.
int ensure_wait_flag(lens_sim* s);
int sub_count(lens_sim* s, const lens_system& y);
int prepare_subhalos(lens_sim* s, const lens_system& y, float4* tab_buf, float* raw_buf, const float4** out_tab,
                     int* out_n, cudaStream_t st);
void fill_dev_system(const lens_system& y, DevSystem& d);
// The elliptical-multipole harmonics of a system into `host` (kEllTableFloats floats); returns
// the highest harmonic K (0 if the system has no LENS_MULTIPOLE_ELL).
int ell_table(const lens_system& y, float* host);
// For the single-system launches of a handle: the table copied to the handle's device buffer
// (from its pinned staging, on the stream) and d.ell_c / d.ell_K set; no-op without the profile.
int upload_ell_table(lens_sim* s, const lens_system& y, DevSystem& d, cudaStream_t st);
// Deflectors of the given type in a system.
int count_deflectors(const lens_system& y, int type);
int run_image_batch(lens_sim* s, const lens_system* systems, int n, float* const* outs, cudaStream_t st);

}  // namespace ls

namespace ls {
// Resident state (registered PSFs and subhalo tables).  A server's slot handles share their
// parent's resident state; only the owner frees it.
// Registered PSFs and subhalo tables, shared by a server's slot handles.  Registration may
// append from another thread while requests run, so entries are read as copies under the lock
// (a reference into the vectors would dangle when they grow).
struct Resident {
  mutable std::mutex mu;
  std::vector<PsfEntry> psfs;
  std::vector<SubTable> tables;

  bool psf(int id, PsfEntry* out) const {
    std::lock_guard<std::mutex> lk(mu);
    if (id < 0 || id >= (int)psfs.size()) return false;
    *out = psfs[id];
    return true;
  }
  bool table(int id, SubTable* out) const {
    std::lock_guard<std::mutex> lk(mu);
    if (id < 0 || id >= (int)tables.size()) return false;
    *out = tables[id];
    return true;
  }
  int kmax() const {
    std::lock_guard<std::mutex> lk(mu);
    int k = 0;
    for (const auto& p : psfs) k = p.k > k ? p.k : k;
    return k;
  }
  int add_psf(const PsfEntry& e) {
    std::lock_guard<std::mutex> lk(mu);
    psfs.push_back(e);
    return (int)psfs.size() - 1;
  }
  int add_table(const SubTable& t) {
    std::lock_guard<std::mutex> lk(mu);
    tables.push_back(t);
    return (int)tables.size() - 1;
  }
};
}  // namespace ls

struct lens_sim {
  int device = 0;
  size_t budget = 0;
  size_t allocated = 0;
  int max_batch = 4096;
  int sm_count = 0;
  int trace_variant = 0;  // launch variant of the single-system trace kernel
  float far_kappa = 0.f;  // far-field interpolation of the subhalo sum (0: exact)
  int batch_form = 0;     // persistent trace kernel of the batched launch (kBatchForms)
  int batch_order = 0;    // unit queue: 0 systems by per-unit cost (largest first), 1 as given
  int conv_method = 0;    // LENS_CONV_AUTO / _DIRECT / _FFT
  int* wait_flag_h = nullptr;  // host-mapped flag raised by an expired bounded device wait
  int* wait_flag_d = nullptr;
  std::string err;
  std::shared_ptr<ls::Resident> res = std::make_shared<ls::Resident>();
  bool owns_resident = true;
  ls::DevBuffer raw_sub;  // device copy of a host subhalo SoA
  ls::DevBuffer tab;      // per-call subhalo constants
  ls::DevBuffer img;      // unconvolved (binned) image
  ls::DevBuffer ell_dev;  // elliptical-multipole harmonics of the current single-system call
  float* ell_pinned = nullptr;        // their host staging
  cudaEvent_t ell_ready = nullptr;    // recorded after the staging's last copy
  ls::DevBuffer stage;    // device staging of host outputs
  ls::DevBuffer grad_ws;  // likelihood / adjoint workspace
  ls::DevBuffer fft_ws;   // FFT convolution workspace (row and column spectra of a chunk of images)
  // Subhalo deflection field at every sample of a grid, for a registered (immutable) subhalo
  // table: computed once per (table, grid) and reused by the likelihood calls that follow.
  ls::DevBuffer sub_field;
  struct FieldKey {
    int table = -1, nx = 0, ny = 0, s = 0;
    float dpix = 0.f, x0 = 0.f, y0 = 0.f;
    bool operator==(const FieldKey& o) const {
      return table == o.table && nx == o.nx && ny == o.ny && s == o.s && dpix == o.dpix && x0 == o.x0 && y0 == o.y0;
    }
  } field_key;
  struct FftSpectrum {
    int psf_id, My, Mx;
    ls::DevBuffer buf;
  };
  std::vector<FftSpectrum> spectra;  // kernel spectra per (psf, padded size)
  // batched launch
  ls::DevBuffer batch_meta;   // packed header + descriptors + prefix + jobs
  ls::DevBuffer batch_data;   // subhalo tables, raw copies, unconvolved images, output staging
  void* pinned = nullptr;     // host staging of the metadata block
  size_t pinned_cap = 0;
  cudaEvent_t pinned_ready = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  void* graph_meta = nullptr;
  int graph_kmax = 0;
  int graph_form = -1;
  bool graph_far = false;  // the captured graph runs the far-field interpolation
};
