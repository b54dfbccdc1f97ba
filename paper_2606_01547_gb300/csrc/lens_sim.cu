// Host implementation of the C ABI in include/lens_sim.h: argument validation, device
// workspace management, resident PSF/subhalo state, and the per-system launch sequence
//   subhalo constants -> fused trace/source/bin-down kernel -> PSF convolution.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "lens_sim.h"
#include "sim_internal.h"

using namespace ls;

namespace ls {

int fail(lens_sim* s, int code, const char* fmt, ...) {
  if (s) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    s->err = buf;
  }
  return code;
}

int cuda_fail(lens_sim* s, cudaError_t e, const char* what) {
  return fail(s, LENS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool on_other_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type != cudaMemoryTypeDevice) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.device != dev;
}

int ensure(lens_sim* s, DevBuffer& b, size_t bytes) {
  if (bytes <= b.cap) return LENS_OK;
  size_t want = bytes + bytes / 4;  // geometric growth
  if (s->budget && s->allocated - b.cap + want > s->budget) {
    want = bytes;
    if (s->allocated - b.cap + want > s->budget)
      return fail(s, LENS_ERR_OOM, "workspace of %zu bytes exceeds the memory budget (%zu of %zu used)",
                  bytes, s->allocated, s->budget);
  }
  if (b.p) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaDeviceSynchronize");
    cudaFree(b.p);
    s->allocated -= b.cap;
    b.p = nullptr;
    b.cap = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(s, LENS_ERR_OOM, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
  }
  b.cap = want;
  s->allocated += want;
  return LENS_OK;
}

void release(lens_sim* s, DevBuffer& b) {
  if (b.p) {
    cudaFree(b.p);
    s->allocated -= b.cap;
  }
  b.p = nullptr;
  b.cap = 0;
}

static bool finite(float v) { return v == v && v < 3.0e38f && v > -3.0e38f; }

static bool is_integer_in(float v, int lo, int hi) {
  return v >= (float)lo && v <= (float)hi && v == (float)(int)v;
}

int validate_profile(lens_sim* s, const lens_profile& p) {
  for (int k = 0; k < LENS_PROFILE_PARAMS; ++k)
    if (!finite(p.p[k])) return fail(s, LENS_ERR_INVALID_ARG, "deflector parameter %d is not finite", k);
  switch (p.type) {
    case LENS_SIS: case LENS_SHEAR: case LENS_POINT_MASS: return LENS_OK;
    case LENS_SIE:
      if (!(p.p[1] > 0.f && p.p[1] <= 1.f)) return fail(s, LENS_ERR_INVALID_ARG, "SIE q=%g not in (0,1]", p.p[1]);
      return LENS_OK;
    case LENS_EPL:
      if (!(p.p[2] > 0.f && p.p[2] <= 1.f)) return fail(s, LENS_ERR_INVALID_ARG, "EPL q=%g not in (0,1]", p.p[2]);
      if (!(p.p[1] > 1.f && p.p[1] < 3.f)) return fail(s, LENS_ERR_INVALID_ARG, "EPL gamma=%g not in (1,3)", p.p[1]);
      return LENS_OK;
    case LENS_EPL_E1E2:
      if (!(p.p[1] > 1.f && p.p[1] < 3.f)) return fail(s, LENS_ERR_INVALID_ARG, "EPL gamma=%g not in (1,3)", p.p[1]);
      if (!(p.p[2] * p.p[2] + p.p[3] * p.p[3] < 1.f)) return fail(s, LENS_ERR_INVALID_ARG, "EPL |e| >= 1");
      return LENS_OK;
    case LENS_SIE_E1E2:
      if (!(p.p[1] * p.p[1] + p.p[2] * p.p[2] < 1.f)) return fail(s, LENS_ERR_INVALID_ARG, "SIE |e| >= 1");
      return LENS_OK;
    case LENS_NFW:
      if (!(p.p[0] > 0.f)) return fail(s, LENS_ERR_INVALID_ARG, "NFW Rs must be > 0");
      return LENS_OK;
    case LENS_TNFW:
      if (!(p.p[0] > 0.f && p.p[2] > 0.f)) return fail(s, LENS_ERR_INVALID_ARG, "TNFW Rs and r_t must be > 0");
      return LENS_OK;
    case LENS_MULTIPOLE:
      if (!is_integer_in(p.p[0], 1, LENS_MAX_MULTIPOLE_ORDER))
        return fail(s, LENS_ERR_INVALID_ARG, "multipole order m=%g not an integer in [1, %d]", p.p[0],
                    LENS_MAX_MULTIPOLE_ORDER);
      if (!(p.p[5] > 0.f)) return fail(s, LENS_ERR_INVALID_ARG, "multipole r_E must be > 0");
      return LENS_OK;
    case LENS_MULTIPOLE_ELL:
      if (!is_integer_in(p.p[0], 1, LENS_MAX_MULTIPOLE_ELL_ORDER))
        return fail(s, LENS_ERR_INVALID_ARG, "elliptical multipole order m=%g not an integer in [1, %d]", p.p[0],
                    LENS_MAX_MULTIPOLE_ELL_ORDER);
      if (!(p.p[3] >= 0.2f && p.p[3] <= 1.f))
        return fail(s, LENS_ERR_INVALID_ARG, "elliptical multipole q=%g not in [0.2, 1]", p.p[3]);
      if (!(p.p[7] > 0.f)) return fail(s, LENS_ERR_INVALID_ARG, "elliptical multipole r_E must be > 0");
      return LENS_OK;
    case LENS_NFW_ELLIPSE_CSE:
    case LENS_HERNQUIST_ELLIPSE_CSE:
      if (!(p.p[p.type == LENS_NFW_ELLIPSE_CSE ? 0 : 1] > 0.f)) return fail(s, LENS_ERR_INVALID_ARG, "Rs must be > 0");
      if (!(p.p[2] * p.p[2] + p.p[3] * p.p[3] < 1.f)) return fail(s, LENS_ERR_INVALID_ARG, "|e| >= 1");
      return LENS_OK;
    case LENS_CSE:
      if (!(p.p[1] > 0.f)) return fail(s, LENS_ERR_INVALID_ARG, "CSE core s must be > 0");
      if (!(p.p[2] * p.p[2] + p.p[3] * p.p[3] < 1.f)) return fail(s, LENS_ERR_INVALID_ARG, "CSE |e| >= 1");
      return LENS_OK;
    case LENS_EPL_MULTIPOLE_M1M3M4:
      if (!(p.p[0] > 0.f)) return fail(s, LENS_ERR_INVALID_ARG, "EPL theta_E must be > 0");
      if (!(p.p[1] > 1.f && p.p[1] < 3.f)) return fail(s, LENS_ERR_INVALID_ARG, "EPL gamma=%g not in (1,3)", p.p[1]);
      if (!(p.p[2] * p.p[2] + p.p[3] * p.p[3] < 1.f)) return fail(s, LENS_ERR_INVALID_ARG, "EPL |e| >= 1");
      return LENS_OK;
    default: return fail(s, LENS_ERR_INVALID_ARG, "unknown deflector type %d", p.type);
  }
}

int validate_light(lens_sim* s, const light_profile& p, const float* coeffs, int n_coeffs) {
  for (int k = 0; k < 8; ++k)
    if (!finite(p.p[k])) return fail(s, LENS_ERR_INVALID_ARG, "source parameter %d is not finite", k);
  if (p.type == LIGHT_SHAPELETS) {
    if (!is_integer_in(p.p[0], 0, LENS_MAX_SHAPELET_NMAX))
      return fail(s, LENS_ERR_INVALID_ARG, "shapelet n_max=%g not an integer in [0, %d]", p.p[0],
                  LENS_MAX_SHAPELET_NMAX);
    if (!(p.p[1] > 0.f)) return fail(s, LENS_ERR_INVALID_ARG, "shapelet beta must be > 0");
    const int nm = (int)p.p[0], want = (nm + 1) * (nm + 2) / 2;
    if (!coeffs || n_coeffs != want)
      return fail(s, LENS_ERR_INVALID_ARG, "shapelets need %d amplitudes in source_coeffs, got %d", want,
                  coeffs ? n_coeffs : 0);
    for (int k = 0; k < n_coeffs; ++k)
      if (!finite(coeffs[k])) return fail(s, LENS_ERR_INVALID_ARG, "shapelet amplitude %d is not finite", k);
    return LENS_OK;
  }
  if (!(p.p[1] > 0.f) || !(p.p[2] > 0.f)) return fail(s, LENS_ERR_INVALID_ARG, "Sersic R and n must be > 0");
  switch (p.type) {
    case LIGHT_SERSIC: return LENS_OK;
    case LIGHT_SERSIC_ELLIPSE_Q_PHI:
      if (!(p.p[3] > 0.f && p.p[3] <= 1.f)) return fail(s, LENS_ERR_INVALID_ARG, "Sersic q=%g not in (0,1]", p.p[3]);
      return LENS_OK;
    case LIGHT_SERSIC_ELLIPSE:
      if (!(p.p[3] * p.p[3] + p.p[4] * p.p[4] < 1.f)) return fail(s, LENS_ERR_INVALID_ARG, "Sersic |e| >= 1");
      return LENS_OK;
    default: return fail(s, LENS_ERR_INVALID_ARG, "unknown light type %d", p.type);
  }
}

int validate_grid(lens_sim* s, const lens_grid& g) {
  if (g.nx < 1 || g.ny < 1 || g.nx > 16384 || g.ny > 16384)
    return fail(s, LENS_ERR_INVALID_ARG, "grid %dx%d out of range [1, 16384]", g.nx, g.ny);
  if (g.supersample < 1 || g.supersample > LENS_MAX_SUPERSAMPLE)
    return fail(s, LENS_ERR_INVALID_ARG, "supersample %d not in [1, %d]", g.supersample, LENS_MAX_SUPERSAMPLE);
  if (!(g.pixel_scale > 0.f) || !finite(g.pixel_scale) || !finite(g.x0) || !finite(g.y0))
    return fail(s, LENS_ERR_INVALID_ARG, "bad pixel scale or grid centre");
  return LENS_OK;
}

int validate_system(lens_sim* s, const lens_system& y, bool need_grid) {
  if (need_grid) {
    if (int rg = validate_grid(s, y.grid)) return rg;
    int rc = validate_light(s, y.source, y.source_coeffs, y.n_source_coeffs);
    if (rc) return rc;
    PsfEntry pe;
    if (y.psf_id < -1 || (y.psf_id >= 0 && (!s->res->psf(y.psf_id, &pe) || !pe.d)))
      return fail(s, LENS_ERR_INVALID_ARG, "unknown psf_id %d", y.psf_id);
  }
  if (y.n_deflectors < 0 || y.n_deflectors > LENS_MAX_DEFLECTORS)
    return fail(s, LENS_ERR_INVALID_ARG, "n_deflectors %d not in [0, %d]", y.n_deflectors, LENS_MAX_DEFLECTORS);
  if (y.n_deflectors > 0 && !y.deflectors) return fail(s, LENS_ERR_INVALID_ARG, "deflectors is NULL");
  for (int d = 0; d < y.n_deflectors; ++d) {
    int rc = validate_profile(s, y.deflectors[d]);
    if (rc) return rc;
  }
  if (count_deflectors(y, LENS_MULTIPOLE_ELL) > 1)
    return fail(s, LENS_ERR_INVALID_ARG, "at most one elliptical multipole per system");
  if (y.subhalo_table >= 0) {
    SubTable t;
    if (!s->res->table(y.subhalo_table, &t) || (!t.d && t.n))
      return fail(s, LENS_ERR_INVALID_ARG, "unknown subhalo_table %d", y.subhalo_table);
  } else {
    if (y.subhalo_table != -1) return fail(s, LENS_ERR_INVALID_ARG, "subhalo_table must be -1 or a table id");
    if (y.n_subhalos < 0) return fail(s, LENS_ERR_INVALID_ARG, "n_subhalos < 0");
    if (y.n_subhalos > 0 && !y.subhalos) return fail(s, LENS_ERR_INVALID_ARG, "subhalos is NULL");
  }
  return LENS_OK;
}

int sub_count(lens_sim* s, const lens_system& y) {
  if (y.subhalo_table < 0) return y.n_subhalos;
  SubTable t;
  return s->res->table(y.subhalo_table, &t) ? t.n : 0;
}

// Resolve the subhalo table of a system into device constants (kTableStride float4 per subhalo).
// `tab_buf` must hold 16 * kTableStride * n bytes when the system carries raw subhalos.
int prepare_subhalos(lens_sim* s, const lens_system& y, float4* tab_buf, float* raw_buf,
                     const float4** out_tab, int* out_n, cudaStream_t st) {
  if (y.subhalo_table >= 0) {
    SubTable t;
    if (!s->res->table(y.subhalo_table, &t)) return fail(s, LENS_ERR_INVALID_ARG, "unknown subhalo_table %d", y.subhalo_table);
    *out_tab = t.d;
    *out_n = t.n;
    return LENS_OK;
  }
  const int n = y.n_subhalos;
  *out_n = n;
  *out_tab = tab_buf;
  if (n == 0) return LENS_OK;
  const float* src = y.subhalos;
  if (!is_device_ptr(src)) {
    cudaError_t e = cudaMemcpyAsync(raw_buf, src, sizeof(float) * 5 * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "copy subhalos to device");
    src = raw_buf;
  }
  cudaError_t e = launch_tnfw_prep(src, n, n, tab_buf, st);
  if (e != cudaSuccess) return cuda_fail(s, e, "tnfw_prep launch");
  return LENS_OK;
}

int count_deflectors(const lens_system& y, int type) {
  int n = 0;
  for (int k = 0; k < y.n_deflectors; ++k) n += y.deflectors[k].type == type;
  return n;
}

// LENS_MULTIPOLE_ELL: the Fourier coefficients c_k of 2 kappa r / (a_m r_E), a function of the
// polar angle alone, by the trapezoid rule on 1024 points (geometric convergence for this
// analytic periodic function; 1024 points resolve the at most 320 harmonics kept without
// aliasing), kept up to the last harmonic above 1e-8 of the largest (at most kEllMaxK) and stored
// scaled by a_m r_E as (Re, Im) pairs.  Host FP64; the cosine and sine tables are computed once.
static int ell_coefficients(const float* p, float* out) {
  constexpr int N = 1024;
  constexpr double kTwoPi = 6.283185307179586476925;
  static double cs[N], sn[N];
  static std::once_flag once;
  std::call_once(once, [] {
    for (int j = 0; j < N; ++j) {
      cs[j] = std::cos(kTwoPi * j / N);
      sn[j] = std::sin(kTwoPi * j / N);
    }
  });
  const int m = (int)std::lround(p[0]);
  const double q = p[3], dphi = (double)p[2] - (double)p[4], scale = (double)p[1] * (double)p[7];
  const double sq = std::sqrt(q);
  std::vector<double> h(N), re(kEllMaxK + 1), im(kEllMaxK + 1);
  for (int j = 0; j < N; ++j) {
    const double g = std::sqrt(q * cs[j] * cs[j] + sn[j] * sn[j] / q);  // R / r
    h[j] = std::cos(m * (std::atan2(sn[j] / sq, sq * cs[j]) - dphi)) / g;
  }
  double amax = 0.0;
  for (int k = 0; k <= kEllMaxK; ++k) {
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < N; ++j) {
      const int idx = (k * j) % N;
      sr += h[j] * cs[idx];
      si -= h[j] * sn[idx];
    }
    re[k] = sr / N;
    im[k] = si / N;
    amax = std::max(amax, std::hypot(re[k], im[k]));
  }
  int K = 1;
  for (int k = 2; k <= kEllMaxK; ++k)
    if (std::hypot(re[k], im[k]) > 1e-8 * amax) K = k;
  for (int k = 0; k <= kEllMaxK; ++k) {
    out[2 * k] = k <= K ? (float)(scale * re[k]) : 0.f;
    out[2 * k + 1] = k <= K ? (float)(scale * im[k]) : 0.f;
  }
  return K;
}

int ell_table(const lens_system& y, float* host) {
  for (int k = 0; k < y.n_deflectors; ++k)
    if (y.deflectors[k].type == LENS_MULTIPOLE_ELL) return ell_coefficients(y.deflectors[k].p, host);
  return 0;
}

int upload_ell_table(lens_sim* s, const lens_system& y, DevSystem& d, cudaStream_t st) {
  d.ell_K = 0;
  d.ell_c = nullptr;
  if (count_deflectors(y, LENS_MULTIPOLE_ELL) == 0) return LENS_OK;
  int rc = ensure(s, s->ell_dev, sizeof(float) * kEllTableFloats);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (!s->ell_pinned) {
    e = cudaMallocHost((void**)&s->ell_pinned, sizeof(float) * kEllTableFloats);
    if (e != cudaSuccess) {
      s->ell_pinned = nullptr;
      return fail(s, LENS_ERR_OOM, "pinned staging: %s", cudaGetErrorString(e));
    }
    if ((e = cudaEventCreateWithFlags(&s->ell_ready, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(s, e, "create event");
  } else if ((e = cudaEventSynchronize(s->ell_ready)) != cudaSuccess) {  // the last copy has read it
    return cuda_fail(s, e, "staging event");
  }
  d.ell_K = ell_table(y, s->ell_pinned);
  e = cudaMemcpyAsync(s->ell_dev.p, s->ell_pinned, sizeof(float) * kEllTableFloats, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(s->ell_ready, st);
  if (e != cudaSuccess) return cuda_fail(s, e, "copy elliptical-multipole table");
  d.ell_c = (const float*)s->ell_dev.p;
  return LENS_OK;
}

void fill_dev_system(const lens_system& y, DevSystem& d) {
  std::memset(&d, 0, sizeof(d));
  d.nx = y.grid.nx;
  d.ny = y.grid.ny;
  d.s = y.grid.supersample;
  d.dpix = y.grid.pixel_scale;
  d.x0 = y.grid.x0;
  d.y0 = y.grid.y0;
  d.n_defl = y.n_deflectors;
  for (int k = 0; k < y.n_deflectors; ++k) {
    d.defl[k].type = y.deflectors[k].type;
    for (int q = 0; q < LENS_PROFILE_PARAMS; ++q) d.defl[k].p[q] = y.deflectors[k].p[q];
  }
  d.src_type = y.source.type;
  for (int q = 0; q < 8; ++q) d.src[q] = y.source.p[q];
  if (y.source.type == LIGHT_SHAPELETS && y.source_coeffs)
    for (int q = 0; q < y.n_source_coeffs && q < LENS_MAX_SHAPELET_COEFFS; ++q) d.src_coef[q] = y.source_coeffs[q];
}

// PSF step of a stack of n_img equal-size device images (method per the handle; in != out).
int psf_apply(lens_sim* s, const float* in, float* out, int n_img, int ny, int nx, int psf_id, cudaStream_t st,
              bool allow_tma) {
  PsfEntry p;
  if (!s->res->psf(psf_id, &p)) return fail(s, LENS_ERR_INVALID_ARG, "unknown psf_id %d", psf_id);
  int My = 0, Mx = 0;
  const bool fits = conv_fft_sizes(ny, nx, p.k, &My, &Mx);
  if (s->conv_method == LENS_CONV_FFT && !fits)
    return fail(s, LENS_ERR_UNSUPPORTED, "FFT convolution needs padded sizes <= 1024 (got %dx%d)", My, Mx);
  const bool use_fft = fits && (s->conv_method == LENS_CONV_FFT ||
                                (s->conv_method == LENS_CONV_AUTO && p.k >= LENS_CONV_FFT_MIN_K));
  cudaError_t e;
  if (use_fft) {
    lens_sim::FftSpectrum* spec = nullptr;
    for (auto& f : s->spectra)
      if (f.psf_id == psf_id && f.My == My && f.Mx == Mx) spec = &f;
    const size_t per_img = conv_fft_bytes_per_image(ny, Mx);
    const size_t want_ws = std::max(per_img * (size_t)std::min(n_img, 64), conv_fft_spectrum_work_bytes(Mx, p.k));
    int rc;
    if ((rc = ensure(s, s->fft_ws, want_ws))) return rc;
    if (!spec) {
      s->spectra.push_back({psf_id, My, Mx, DevBuffer{}});
      spec = &s->spectra.back();
      if ((rc = ensure(s, spec->buf, conv_fft_spectrum_bytes(My, Mx, p.k)))) {
        s->spectra.pop_back();
        return rc;
      }
      e = launch_fft_spectrum(p.d, p.k, My, Mx, s->fft_ws.p, spec->buf.p, st);
      if (e != cudaSuccess) return cuda_fail(s, e, "FFT spectrum of the PSF");
    }
    // large kernels: the central core directly (exact-order sum), the wings by FFT, added
    const int core = conv_fft_core(p.k);
    if (core > 0) {
      const float* kc = conv_fft_core_kernel(spec->buf.p, My, Mx);
      if (allow_tma && conv_tma_supported(in, out, ny, nx, core))
        e = launch_conv_tma(in, out, n_img, ny, nx, kc, core, s->wait_flag_d, s->sm_count, st);
      else
        e = launch_conv(in, out, n_img, ny, nx, kc, core, 1, st);
      if (e != cudaSuccess) return cuda_fail(s, e, "PSF core launch");
    }
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_img, s->fft_ws.cap / per_img));
    float2* A = (float2*)s->fft_ws.p;
    for (int i0 = 0; i0 < n_img; i0 += chunk) {
      const int n = std::min(chunk, n_img - i0);
      e = launch_conv_fft(in + (size_t)i0 * ny * nx, out + (size_t)i0 * ny * nx, n, ny, nx, p.k, My, Mx,
                          spec->buf.p, A, core > 0 ? 1 : 0, st);
      if (e != cudaSuccess) return cuda_fail(s, e, "FFT convolution launch");
    }
    return LENS_OK;
  }
  if (allow_tma && conv_tma_supported(in, out, ny, nx, p.k))
    e = launch_conv_tma(in, out, n_img, ny, nx, p.d, p.k, s->wait_flag_d, s->sm_count, st);
  else
    e = launch_conv(in, out, n_img, ny, nx, p.d, p.k, 1, st);
  if (e != cudaSuccess) return cuda_fail(s, e, "psf kernel launch");
  return LENS_OK;
}

int ensure_wait_flag(lens_sim* s) {
  if (!s->wait_flag_h) {
    if (cudaHostAlloc((void**)&s->wait_flag_h, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&s->wait_flag_d, s->wait_flag_h, 0) != cudaSuccess) {
      cudaGetLastError();
      if (s->wait_flag_h) cudaFreeHost(s->wait_flag_h);
      s->wait_flag_h = nullptr;
      return fail(s, LENS_ERR_OOM, "host-mapped wait flag");
    }
    *s->wait_flag_h = 0;
  }
  if (*(volatile int*)s->wait_flag_h) {
    *s->wait_flag_h = 0;
    return fail(s, LENS_ERR_TIMEOUT, "a bounded wait of an earlier convolution expired");
  }
  return LENS_OK;
}

DeviceGuard::DeviceGuard(int dev) {
  // A non-fatal status left by an earlier call on this thread (e.g. "not ready" from a query)
  // would otherwise be read back by the launch checks below as a launch failure.
  cudaGetLastError();
  cudaGetDevice(&prev_);
  if (prev_ != dev) cudaSetDevice(dev);
  dev_ = dev;
}
DeviceGuard::~DeviceGuard() {
  if (prev_ != dev_) cudaSetDevice(prev_);
}

}  // namespace ls

// ============================================================================ C ABI
extern "C" {

int lens_sim_create(const lens_sim_config* cfg, lens_sim** out) {
  if (!out) return LENS_ERR_INVALID_ARG;
  *out = nullptr;
  lens_sim_config c{0, 0, 0, 0};
  if (cfg) c = *cfg;
  if (c.flags != 0 || c.max_batch < 0) return LENS_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return LENS_ERR_CUDA;
  }
  if (c.device < 0 || c.device >= ndev) return LENS_ERR_INVALID_ARG;
  lens_sim* s = new (std::nothrow) lens_sim();
  if (!s) return LENS_ERR_OOM;
  s->device = c.device;
  s->budget = c.mem_budget_bytes;
  s->max_batch = c.max_batch ? c.max_batch : 4096;
  DeviceGuard g(s->device);
  cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  *out = s;
  return LENS_OK;
}

void lens_sim_destroy(lens_sim* s) {
  if (!s) return;
  {
    DeviceGuard g(s->device);
    cudaDeviceSynchronize();
    if (s->owns_resident) {
      std::lock_guard<std::mutex> lk(s->res->mu);
      for (auto& p : s->res->psfs) if (p.d) cudaFree(p.d);
      for (auto& t : s->res->tables) if (t.d) cudaFree(t.d);
      s->res->psfs.clear();
      s->res->tables.clear();
    }
    release(s, s->raw_sub);
    release(s, s->tab);
    release(s, s->img);
    release(s, s->ell_dev);
    if (s->ell_ready) cudaEventDestroy(s->ell_ready);
    if (s->ell_pinned) cudaFreeHost(s->ell_pinned);
    release(s, s->stage);
    release(s, s->grad_ws);
    release(s, s->fft_ws);
    release(s, s->sub_field);
    for (auto& f : s->spectra) release(s, f.buf);
    s->spectra.clear();
    release(s, s->batch_meta);
    release(s, s->batch_data);
    if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->pinned_ready) cudaEventDestroy(s->pinned_ready);
    if (s->pinned) cudaFreeHost(s->pinned);
    if (s->wait_flag_h) cudaFreeHost(s->wait_flag_h);
  }
  delete s;
}

const char* lens_sim_last_error(const lens_sim* s) { return s ? s->err.c_str() : "null handle"; }

int lens_sim_register_psf(lens_sim* s, const float* kernel, int k, int* psf_id) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (!kernel || !psf_id) return fail(s, LENS_ERR_INVALID_ARG, "NULL kernel or psf_id");
  if (k < 1 || k > LENS_MAX_PSF || (k % 2) == 0) return fail(s, LENS_ERR_INVALID_ARG, "PSF size %d must be odd in [1, %d]", k, LENS_MAX_PSF);
  DeviceGuard g(s->device);
  size_t bytes = sizeof(float) * (size_t)k * k;
  if (s->budget && s->allocated + 2 * bytes > s->budget) return fail(s, LENS_ERR_OOM, "PSF exceeds the memory budget");
  std::vector<float> h((size_t)k * k), hf((size_t)k * k);
  cudaError_t e = cudaMemcpy(h.data(), kernel, bytes, is_device_ptr(kernel) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
  if (e != cudaSuccess) return cuda_fail(s, e, "read PSF");
  for (size_t t = 0; t < h.size(); ++t) hf[t] = h[h.size() - 1 - t];
  float* d = nullptr;
  float* df = nullptr;
  e = cudaMalloc(&d, 2 * bytes);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(s, LENS_ERR_OOM, "cudaMalloc PSF: %s", cudaGetErrorString(e)); }
  df = d + (size_t)k * k;
  e = cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(df, hf.data(), bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(d); return cuda_fail(s, e, "copy PSF"); }
  s->allocated += 2 * bytes;
  *psf_id = s->res->add_psf({d, k, df});
  return LENS_OK;
}

int lens_sim_register_subhalos(lens_sim* s, const float* soa, int n, int* table_id) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (!table_id || n < 0 || (n > 0 && !soa)) return fail(s, LENS_ERR_INVALID_ARG, "bad subhalo table arguments");
  DeviceGuard g(s->device);
  SubTable t{nullptr, n};
  if (n > 0) {
    size_t bytes = kTableStride * sizeof(float4) * (size_t)n;
    if (s->budget && s->allocated + bytes > s->budget) return fail(s, LENS_ERR_OOM, "subhalo table exceeds the memory budget");
    cudaError_t e = cudaMalloc(&t.d, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(s, LENS_ERR_OOM, "cudaMalloc subhalo table: %s", cudaGetErrorString(e)); }
    const float* src = soa;
    float* tmp = nullptr;
    if (!is_device_ptr(soa)) {
      e = cudaMalloc(&tmp, sizeof(float) * 5 * (size_t)n);
      if (e == cudaSuccess) e = cudaMemcpy(tmp, soa, sizeof(float) * 5 * (size_t)n, cudaMemcpyHostToDevice);
      src = tmp;
    }
    if (e == cudaSuccess) e = launch_tnfw_prep(src, n, n, t.d, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) { cudaFree(t.d); return cuda_fail(s, e, "subhalo table"); }
    s->allocated += bytes;
  }
  *table_id = s->res->add_table(t);
  return LENS_OK;
}

int lens_sim_image(lens_sim* s, const lens_system* systems, int n_sys, float* const* out_images, void* stream) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (n_sys < 0 || n_sys > s->max_batch) return fail(s, LENS_ERR_INVALID_ARG, "n_sys %d not in [0, %d]", n_sys, s->max_batch);
  if (n_sys == 0) return LENS_OK;
  if (!systems || !out_images) return fail(s, LENS_ERR_INVALID_ARG, "NULL systems or out_images");
  DeviceGuard g(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  size_t max_pix = 0, max_sub = 0;
  for (int i = 0; i < n_sys; ++i) {
    int rc = validate_system(s, systems[i], true);
    if (rc) return fail(s, rc, "system %d: %s", i, s->err.c_str());
    if (!out_images[i]) return fail(s, LENS_ERR_INVALID_ARG, "system %d: NULL output", i);
    max_pix = std::max(max_pix, (size_t)systems[i].grid.nx * systems[i].grid.ny);
    if (systems[i].subhalo_table < 0) max_sub = std::max(max_sub, (size_t)systems[i].n_subhalos);
  }
  if (n_sys > 1) return run_image_batch(s, systems, n_sys, out_images, st);
  int rc;
  if ((rc = ensure(s, s->img, sizeof(float) * max_pix))) return rc;
  if ((rc = ensure(s, s->stage, sizeof(float) * max_pix))) return rc;
  if (max_sub) {
    if ((rc = ensure(s, s->tab, kTableStride * sizeof(float4) * max_sub))) return rc;
    if ((rc = ensure(s, s->raw_sub, 5 * sizeof(float) * max_sub))) return rc;
  }
  bool host_out = false;
  for (int i = 0; i < n_sys; ++i) {
    const lens_system& y = systems[i];
    DevSystem d;
    fill_dev_system(y, d);
    if ((rc = upload_ell_table(s, y, d, st))) return rc;
    if ((rc = prepare_subhalos(s, y, (float4*)s->tab.p, (float*)s->raw_sub.p, &d.sub, &d.n_sub, st))) return rc;
    const bool dev_out = is_device_ptr(out_images[i]);
    float* final_dst = dev_out ? out_images[i] : (float*)s->stage.p;
    d.out = (y.psf_id >= 0) ? (float*)s->img.p : final_dst;
    d.far_kappa = s->far_kappa;
    cudaError_t e = launch_trace_variant(d, s->trace_variant, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "trace kernel launch");
    if (y.psf_id >= 0 && (rc = psf_apply(s, (float*)s->img.p, final_dst, 1, d.ny, d.nx, y.psf_id, st, false)))
      return rc;
    if (!dev_out) {
      e = cudaMemcpyAsync(out_images[i], final_dst, sizeof(float) * d.nx * d.ny, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return cuda_fail(s, e, "copy image to host");
      host_out = true;
    }
  }
  if (host_out) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(s, e, "stream synchronize");
  }
  return LENS_OK;
}

int lens_sim_deflection(lens_sim* s, const lens_system* sys, const float* x, const float* y, int n, float* ax,
                        float* ay, void* stream) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (!sys || n < 0) return fail(s, LENS_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return LENS_OK;
  if (!x || !y || !ax || !ay) return fail(s, LENS_ERR_INVALID_ARG, "NULL point arrays");
  DeviceGuard g(s->device);
  int rc = validate_system(s, *sys, false);
  if (rc) return rc;
  if (!is_device_ptr(x) || !is_device_ptr(y) || !is_device_ptr(ax) || !is_device_ptr(ay))
    return fail(s, LENS_ERR_INVALID_ARG, "point arrays must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  if (sys->subhalo_table < 0 && sys->n_subhalos > 0) {
    if ((rc = ensure(s, s->tab, kTableStride * sizeof(float4) * sys->n_subhalos))) return rc;
    if ((rc = ensure(s, s->raw_sub, 5 * sizeof(float) * sys->n_subhalos))) return rc;
  }
  DevSystem d;
  lens_system tmp = *sys;
  tmp.grid = lens_grid{1, 1, 1, 1.f, 0.f, 0.f};
  fill_dev_system(tmp, d);
  if ((rc = upload_ell_table(s, tmp, d, st))) return rc;
  if ((rc = prepare_subhalos(s, *sys, (float4*)s->tab.p, (float*)s->raw_sub.p, &d.sub, &d.n_sub, st))) return rc;
  cudaError_t e = launch_deflection(d, x, y, n, ax, ay, st);
  if (e != cudaSuccess) return cuda_fail(s, e, "deflection kernel launch");
  return LENS_OK;
}

int lens_sim_convolve(lens_sim* s, const float* in, int n_img, int ny, int nx, int psf_id, float* out, void* stream) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (n_img < 0 || ny < 1 || nx < 1 || ny > 16384 || nx > 16384) return fail(s, LENS_ERR_INVALID_ARG, "bad image sizes");
  PsfEntry pe;
  if (!s->res->psf(psf_id, &pe)) return fail(s, LENS_ERR_INVALID_ARG, "unknown psf_id %d", psf_id);
  if (n_img == 0) return LENS_OK;
  if (!in || !out || in == out) return fail(s, LENS_ERR_INVALID_ARG, "NULL or aliased buffers");
  DeviceGuard g(s->device);
  if (!is_device_ptr(in) || !is_device_ptr(out)) return fail(s, LENS_ERR_INVALID_ARG, "images must be device memory");
  const int rc = ensure_wait_flag(s);
  if (rc) return rc;
  return psf_apply(s, in, out, n_img, ny, nx, psf_id, (cudaStream_t)stream, true);
}

int lens_sim_set_conv_method(lens_sim* s, int method) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (method != LENS_CONV_AUTO && method != LENS_CONV_DIRECT && method != LENS_CONV_FFT)
    return fail(s, LENS_ERR_INVALID_ARG, "unknown convolution method %d", method);
  s->conv_method = method;
  return LENS_OK;
}

int lens_sim_set_variant(lens_sim* s, int variant) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (variant < 0 || variant >= kTraceVariants) return fail(s, LENS_ERR_INVALID_ARG, "variant %d not in [0, %d)", variant, kTraceVariants);
  s->trace_variant = variant;
  return LENS_OK;
}

int lens_sim_set_far_field(lens_sim* s, float kappa) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (!std::isfinite(kappa) || kappa < 0.f || (kappa > 0.f && kappa < 3.f))
    return fail(s, LENS_ERR_INVALID_ARG, "far-field kappa must be 0 or >= 3 (got %g)", (double)kappa);
  s->far_kappa = kappa;
  return LENS_OK;
}

int lens_sim_autotune(lens_sim* s, const lens_system* sample, int reps, int* best_variant, float* ms_per_variant,
                      int n_ms, void* stream) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (!sample || !best_variant || reps < 1 || reps > 1000) return fail(s, LENS_ERR_INVALID_ARG, "bad autotune arguments");
  DeviceGuard g(s->device);
  int rc = validate_system(s, *sample, true);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t npix = (size_t)sample->grid.nx * sample->grid.ny;
  if ((rc = ensure(s, s->img, sizeof(float) * npix))) return rc;
  if (sample->subhalo_table < 0 && sample->n_subhalos > 0) {
    if ((rc = ensure(s, s->tab, kTableStride * sizeof(float4) * sample->n_subhalos))) return rc;
    if ((rc = ensure(s, s->raw_sub, 5 * sizeof(float) * sample->n_subhalos))) return rc;
  }
  DevSystem d;
  fill_dev_system(*sample, d);
  if ((rc = upload_ell_table(s, *sample, d, st))) return rc;
  if ((rc = prepare_subhalos(s, *sample, (float4*)s->tab.p, (float*)s->raw_sub.p, &d.sub, &d.n_sub, st))) return rc;
  d.out = (float*)s->img.p;
  d.far_kappa = s->far_kappa;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 3.0e38f;
  int bi = 0;
  cudaError_t e = cudaSuccess;
  for (int v = 0; v < kTraceVariants && e == cudaSuccess; ++v) {
    e = launch_trace_variant(d, v, st);  // warm-up
    if (e != cudaSuccess) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_trace_variant(d, v, st);
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)reps;
    if (ms_per_variant && v < n_ms) ms_per_variant[v] = ms;
    if (e == cudaSuccess && ms < best) { best = ms; bi = v; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(s, e, "autotune");
  s->trace_variant = bi;
  *best_variant = bi;
  return LENS_OK;
}

}  // extern "C"
