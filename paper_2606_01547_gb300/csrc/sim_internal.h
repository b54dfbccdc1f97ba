// Internal state of a lens_sim handle (shared by the ABI translation units).
#pragma once

#include <algorithm>
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
int ensure(lens_sim* s, DevBuffer& b, size_t bytes);
void release(lens_sim* s, DevBuffer& b);
int validate_system(lens_sim* s, const lens_system& y, bool need_grid);
int sub_count(lens_sim* s, const lens_system& y);
int prepare_subhalos(lens_sim* s, const lens_system& y, float4* tab_buf, float* raw_buf, const float4** out_tab,
                     int* out_n, cudaStream_t st);
void fill_dev_system(const lens_system& y, DevSystem& d);

}  // namespace ls

struct lens_sim {
  int device = 0;
  size_t budget = 0;
  size_t allocated = 0;
  int max_batch = 4096;
  int sm_count = 0;
  std::string err;
  std::vector<ls::PsfEntry> psfs;
  std::vector<ls::SubTable> tables;
  ls::DevBuffer raw_sub;  // device copy of a host subhalo SoA
  ls::DevBuffer tab;      // per-call subhalo constants
  ls::DevBuffer img;      // unconvolved (binned) image
  ls::DevBuffer stage;    // device staging of host outputs
  ls::DevBuffer grad_ws;  // likelihood / adjoint workspace
};
