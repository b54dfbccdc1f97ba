// Allocation-free single-image entry point (lens_sim_image_noalloc).
//
// Some callers cannot call cudaMalloc: applications that reserve the device's memory up front
// for their own pool allocator (a library's cudaMalloc would fail or fragment that pool), and
// latency-critical loops that forbid allocation after start-up because cudaMalloc/cudaFree can
// synchronise the whole device.  This entry point serves them.  It runs the single-system
// kernels of lens_sim_image (subhalo constants, the fused trace kernel, and the direct PSF
// convolution for every k) with no handle: its scratch -- the per-subhalo constants, the
// unconvolved image and an elliptical multipole's harmonics -- lives in one fixed file-scope
// device array instead of a handle's workspace.  It calls no cudaMalloc, cudaFree or allocating
// library routine.
#include "kernels.h"
#include "lens_sim.h"
#include "sim_internal.h"

namespace ls {
int validate_profile(lens_sim* s, const lens_profile& p);
int validate_light(lens_sim* s, const light_profile& p, const float* coeffs, int n_coeffs);
}  // namespace ls

namespace {

constexpr size_t kTableBytes = (size_t)LENS_NOALLOC_MAX_SUBHALOS * ls::kTableStride * sizeof(float4);
constexpr size_t kImageBytes = (size_t)LENS_NOALLOC_MAX_PIXELS * sizeof(float);
constexpr size_t kEllBytes = (size_t)ls::kEllTableFloats * sizeof(float);  // elliptical-multipole harmonics
static_assert(kTableBytes + kImageBytes + kEllBytes == LENS_NOALLOC_SCRATCH_BYTES, "scratch size mismatch");

// The scratch array: every device that loads the library holds one copy until the process
// exits.  Host code must not pass `g_scratch` itself to a kernel (on the host it names a
// stand-in, not device memory); it uses the address looked up below.
static __device__ __align__(256) unsigned char g_scratch[LENS_NOALLOC_SCRATCH_BYTES];

// Device address of g_scratch in the current device's context.  Looked up on every call:
// cudaGetSymbolAddress allocates nothing, and a fresh lookup stays right after the context has
// been re-created (for instance after cudaDeviceReset reloads the module).
int scratch_address(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return LENS_ERR_CUDA;
  }
  *out = p;
  return LENS_OK;
}

}  // namespace

extern "C" int lens_sim_image_noalloc(const lens_system* sys, const float* psf, int k, float* out_image,
                                      void* stream) {
  using namespace ls;
  if (!sys || !out_image) return LENS_ERR_INVALID_ARG;
  const lens_system& y = *sys;
  const lens_grid& g = y.grid;
  if (validate_grid(nullptr, g) != LENS_OK) return LENS_ERR_INVALID_ARG;
  if (y.subhalo_table != -1 || y.n_subhalos < 0 || (y.n_subhalos > 0 && !y.subhalos)) return LENS_ERR_INVALID_ARG;
  if (y.n_deflectors < 0 || y.n_deflectors > LENS_MAX_DEFLECTORS || (y.n_deflectors > 0 && !y.deflectors))
    return LENS_ERR_INVALID_ARG;
  for (int d = 0; d < y.n_deflectors; ++d)
    if (validate_profile(nullptr, y.deflectors[d]) != LENS_OK) return LENS_ERR_INVALID_ARG;
  if (count_deflectors(y, LENS_MULTIPOLE_ELL) > 1) return LENS_ERR_INVALID_ARG;
  if (validate_light(nullptr, y.source, y.source_coeffs, y.n_source_coeffs) != LENS_OK) return LENS_ERR_INVALID_ARG;
  const bool with_psf = psf != nullptr && k != 0;
  if (with_psf && (k < 1 || k > LENS_MAX_PSF || (k % 2) == 0)) return LENS_ERR_INVALID_ARG;
  // sizes beyond the fixed scratch are refused before anything is launched
  if (y.n_subhalos > LENS_NOALLOC_MAX_SUBHALOS || (long long)g.nx * g.ny > (long long)LENS_NOALLOC_MAX_PIXELS)
    return LENS_ERR_OOM;
  // every buffer must be memory of the current device, where the kernels run
  const bool has_sub = y.n_subhalos > 0;
  if (!is_device_ptr(out_image) || (has_sub && !is_device_ptr(y.subhalos)) || (with_psf && !is_device_ptr(psf)))
    return LENS_ERR_INVALID_ARG;
  if (on_other_device(out_image) || (has_sub && on_other_device(y.subhalos)) || (with_psf && on_other_device(psf)))
    return LENS_ERR_INVALID_ARG;

  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != LENS_OK) return rc;
  float4* table = (float4*)base;
  float* raw = (float*)((char*)base + kTableBytes);
  cudaStream_t st = (cudaStream_t)stream;

  // Every byte read below is written first by this call: the table by the constants kernel,
  // the unconvolved image by the trace kernel, the harmonics by the copy.  Nothing needs clearing.
  DevSystem d;
  fill_dev_system(y, d);
  if (count_deflectors(y, LENS_MULTIPOLE_ELL) > 0) {
    // the harmonics go to the scratch from pageable host memory: the copy waits for the
    // stream's earlier work, and the host buffer is free again when the call returns
    float host_ell[kEllTableFloats];
    d.ell_K = ell_table(y, host_ell);
    float* ell = (float*)((char*)base + kTableBytes + kImageBytes);
    if (cudaMemcpyAsync(ell, host_ell, kEllBytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      cudaGetLastError();
      return LENS_ERR_CUDA;
    }
    d.ell_c = ell;
  }
  d.sub = table;
  d.n_sub = y.n_subhalos;
  d.out = with_psf ? raw : out_image;
  cudaError_t e = launch_tnfw_prep(y.subhalos, y.n_subhalos, y.n_subhalos, table, st);
  if (e == cudaSuccess) e = launch_trace_variant(d, 0, st);
  if (e == cudaSuccess && with_psf) e = launch_conv(raw, out_image, 1, g.ny, g.nx, psf, k, 1, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LENS_ERR_CUDA;
  }
  return LENS_OK;
}
