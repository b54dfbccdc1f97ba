// Forward-mode dual numbers (FP32 value + N FP32 tangents) for the per-sample local
// Jacobians of the likelihood adjoint: d alpha_EPL / d(6 lens parameters) and
// d I_Sersic / d(7 source parameters, beta_x, beta_y).
#pragma once

#include <cuda_runtime.h>

namespace ls {

template <int N>
struct Dn {
  float v;
  float d[N];
};

template <int N> __device__ __forceinline__ Dn<N> dconst(float v) {
  Dn<N> r; r.v = v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = 0.f;
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> dvar(float v, int k) {
  Dn<N> r = dconst<N>(v);
  r.d[k] = 1.f;
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator+(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator-(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator-(const Dn<N>& a) {
  Dn<N> r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator*(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = fmaf(a.d[i], b.v, a.v * b.d[i]);
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator*(const Dn<N>& a, float b) {
  Dn<N> r; r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator*(float b, const Dn<N>& a) { return a * b; }
template <int N> __device__ __forceinline__ Dn<N> operator+(const Dn<N>& a, float b) { Dn<N> r = a; r.v += b; return r; }
template <int N> __device__ __forceinline__ Dn<N> operator+(float b, const Dn<N>& a) { Dn<N> r = a; r.v += b; return r; }
template <int N> __device__ __forceinline__ Dn<N> operator-(const Dn<N>& a, float b) { Dn<N> r = a; r.v -= b; return r; }
template <int N> __device__ __forceinline__ Dn<N> operator-(float b, const Dn<N>& a) { return (-a) + b; }
template <int N> __device__ __forceinline__ Dn<N> inv(const Dn<N>& a) {
  float iv = 1.f / a.v, g = -iv * iv;
  Dn<N> r; r.v = iv;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = g * a.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator/(const Dn<N>& a, const Dn<N>& b) { return a * inv(b); }
template <int N> __device__ __forceinline__ Dn<N> operator/(const Dn<N>& a, float b) { return a * (1.f / b); }
template <int N> __device__ __forceinline__ Dn<N> operator/(float a, const Dn<N>& b) { return inv(b) * a; }

// f(a) with f(a.v) = val and f'(a.v) = der
template <int N> __device__ __forceinline__ Dn<N> dapply(const Dn<N>& a, float val, float der) {
  Dn<N> r; r.v = val;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = der * a.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> dsqrt(const Dn<N>& a) {
  float s = sqrtf(a.v);
  return dapply(a, s, 0.5f / s);
}
template <int N> __device__ __forceinline__ Dn<N> dexp(const Dn<N>& a) {
  float e = expf(a.v);
  return dapply(a, e, e);
}
template <int N> __device__ __forceinline__ Dn<N> dlog(const Dn<N>& a) { return dapply(a, logf(a.v), 1.f / a.v); }
template <int N> __device__ __forceinline__ Dn<N> dsin(const Dn<N>& a) { return dapply(a, sinf(a.v), cosf(a.v)); }
template <int N> __device__ __forceinline__ Dn<N> dcos(const Dn<N>& a) { return dapply(a, cosf(a.v), -sinf(a.v)); }
template <int N> __device__ __forceinline__ Dn<N> datan2(const Dn<N>& y, const Dn<N>& x) {
  float den = 1.f / (x.v * x.v + y.v * y.v);
  Dn<N> r; r.v = atan2f(y.v, x.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) * den;
  return r;
}

}  // namespace ls
