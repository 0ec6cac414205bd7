// Device math for the batched rigid-body step.
//
// Two scalar flavours:
//   * `nf` -- FP32 where every +,-,*,/ and sqrt is an IEEE round-to-nearest
//     operation that is never contracted into an FMA (__fadd_rn & co.). The
//     collision stages (AABB, broadphase, narrowphase) use it so that pair
//     lists and contact counts are reproducible bit for bit by any IEEE FP32
//     evaluation of the same expressions in the same order.
//   * plain `float` -- the solver and integrator, where the compiler is free to
//     fuse multiply-adds.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace msh {

struct nf {
  float v;
  __device__ __forceinline__ nf() {}
  __device__ __forceinline__ constexpr nf(float x) : v(x) {}
};
__device__ __forceinline__ nf operator+(nf a, nf b) { return nf(__fadd_rn(a.v, b.v)); }
__device__ __forceinline__ nf operator-(nf a, nf b) { return nf(__fsub_rn(a.v, b.v)); }
__device__ __forceinline__ nf operator*(nf a, nf b) { return nf(__fmul_rn(a.v, b.v)); }
__device__ __forceinline__ nf operator/(nf a, nf b) { return nf(__fdiv_rn(a.v, b.v)); }
__device__ __forceinline__ nf operator-(nf a) { return nf(-a.v); }
__device__ __forceinline__ bool operator<(nf a, nf b) { return a.v < b.v; }
__device__ __forceinline__ bool operator>(nf a, nf b) { return a.v > b.v; }
__device__ __forceinline__ bool operator<=(nf a, nf b) { return a.v <= b.v; }
__device__ __forceinline__ bool operator>=(nf a, nf b) { return a.v >= b.v; }
__device__ __forceinline__ bool operator==(nf a, nf b) { return a.v == b.v; }
__device__ __forceinline__ bool operator!=(nf a, nf b) { return a.v != b.v; }
__device__ __forceinline__ nf sqrt_(nf a) { return nf(__fsqrt_rn(a.v)); }
__device__ __forceinline__ nf abs_(nf a) { return nf(fabsf(a.v)); }
__device__ __forceinline__ float fl(nf a) { return a.v; }

__device__ __forceinline__ float sqrt_(float a) { return sqrtf(a); }
__device__ __forceinline__ float abs_(float a) { return fabsf(a); }
__device__ __forceinline__ float fl(float a) { return a; }

// Single-tangent forward-mode dual number (value v, derivative d). The
// adjoint evaluates the row set-up and the narrowphase with it, one input
// direction at a time, to get exact local Jacobians with the branch decisions
// (clamps, contact features) of the primal values.
struct d1 {
  float v, d;
  __device__ __forceinline__ d1() {}
  __device__ __forceinline__ constexpr d1(float x) : v(x), d(0.f) {}
  __device__ __forceinline__ constexpr d1(float x, float t) : v(x), d(t) {}
};
__device__ __forceinline__ d1 operator+(d1 a, d1 b) { return d1(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ d1 operator-(d1 a, d1 b) { return d1(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ d1 operator*(d1 a, d1 b) { return d1(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ d1 operator/(d1 a, d1 b) { float q = a.v / b.v; return d1(q, (a.d - q * b.d) / b.v); }
__device__ __forceinline__ d1 operator-(d1 a) { return d1(-a.v, -a.d); }
__device__ __forceinline__ bool operator<(d1 a, d1 b) { return a.v < b.v; }
__device__ __forceinline__ bool operator>(d1 a, d1 b) { return a.v > b.v; }
__device__ __forceinline__ bool operator<=(d1 a, d1 b) { return a.v <= b.v; }
__device__ __forceinline__ bool operator>=(d1 a, d1 b) { return a.v >= b.v; }
__device__ __forceinline__ bool operator==(d1 a, d1 b) { return a.v == b.v; }
__device__ __forceinline__ bool operator!=(d1 a, d1 b) { return a.v != b.v; }
__device__ __forceinline__ d1 sqrt_(d1 a) { float r = sqrtf(a.v); return d1(r, r > 0.f ? a.d / (2.f * r) : 0.f); }
__device__ __forceinline__ d1 abs_(d1 a) { return a.v < 0.f ? -a : a; }
__device__ __forceinline__ float fl(d1 a) { return a.v; }
__device__ __forceinline__ d1 atan2_(d1 y, d1 x) {
  float den = x.v * x.v + y.v * y.v;
  return d1(atan2f(y.v, x.v), den > 0.f ? (x.v * y.d - y.v * x.d) / den : 0.f);
}
__device__ __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }

template <class T> __device__ __forceinline__ T clampv(T x, T lo, T hi) { return x < lo ? lo : (x > hi ? hi : x); }
template <class T> __device__ __forceinline__ T maxv(T a, T b) { return a > b ? a : b; }
template <class T> __device__ __forceinline__ T minv(T a, T b) { return a < b ? a : b; }

template <class T> struct V3 { T x, y, z; };
template <class T> struct Q4 { T w, x, y, z; };
template <class T> struct M3 { T m[3][3]; };

template <class T> __device__ __forceinline__ V3<T> v3(T x, T y, T z) { V3<T> r; r.x = x; r.y = y; r.z = z; return r; }
template <class T> __device__ __forceinline__ V3<T> operator+(const V3<T>& a, const V3<T>& b) { return v3<T>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class T> __device__ __forceinline__ V3<T> operator-(const V3<T>& a, const V3<T>& b) { return v3<T>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class T> __device__ __forceinline__ V3<T> operator-(const V3<T>& a) { return v3<T>(-a.x, -a.y, -a.z); }
template <class T> __device__ __forceinline__ V3<T> operator*(const V3<T>& a, T s) { return v3<T>(a.x * s, a.y * s, a.z * s); }
template <class T> __device__ __forceinline__ T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> __device__ __forceinline__ V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return v3<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
template <class T> __device__ __forceinline__ T comp(const V3<T>& a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }
template <class T> __device__ __forceinline__ void setc(V3<T>& a, int k, T v) { if (k == 0) a.x = v; else if (k == 1) a.y = v; else a.z = v; }
template <class T> __device__ __forceinline__ V3<T> unit(int k) { V3<T> r = v3<T>(T(0.f), T(0.f), T(0.f)); setc(r, k, T(1.f)); return r; }

template <class T> __device__ __forceinline__ M3<T> qmat(const Q4<T>& q) {
  T xx = q.x * q.x, yy = q.y * q.y, zz = q.z * q.z;
  T xy = q.x * q.y, xz = q.x * q.z, yz = q.y * q.z;
  T wx = q.w * q.x, wy = q.w * q.y, wz = q.w * q.z;
  const T one = T(1.f), two = T(2.f);
  M3<T> M;
  M.m[0][0] = one - two * (yy + zz); M.m[0][1] = two * (xy - wz); M.m[0][2] = two * (xz + wy);
  M.m[1][0] = two * (xy + wz); M.m[1][1] = one - two * (xx + zz); M.m[1][2] = two * (yz - wx);
  M.m[2][0] = two * (xz - wy); M.m[2][1] = two * (yz + wx); M.m[2][2] = one - two * (xx + yy);
  return M;
}
template <class T> __device__ __forceinline__ V3<T> mul(const M3<T>& M, const V3<T>& v) {
  return v3<T>(M.m[0][0] * v.x + M.m[0][1] * v.y + M.m[0][2] * v.z,
               M.m[1][0] * v.x + M.m[1][1] * v.y + M.m[1][2] * v.z,
               M.m[2][0] * v.x + M.m[2][1] * v.y + M.m[2][2] * v.z); }
template <class T> __device__ __forceinline__ V3<T> mulT(const M3<T>& M, const V3<T>& v) {
  return v3<T>(M.m[0][0] * v.x + M.m[1][0] * v.y + M.m[2][0] * v.z,
               M.m[0][1] * v.x + M.m[1][1] * v.y + M.m[2][1] * v.z,
               M.m[0][2] * v.x + M.m[1][2] * v.y + M.m[2][2] * v.z); }
template <class T> __device__ __forceinline__ V3<T> col(const M3<T>& M, int k) { return v3<T>(M.m[0][k], M.m[1][k], M.m[2][k]); }

template <class T> __device__ __forceinline__ Q4<T> qmul(const Q4<T>& a, const Q4<T>& b) {
  Q4<T> r;
  r.w = a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z;
  r.x = a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y;
  r.y = a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x;
  r.z = a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w;
  return r; }
template <class T> __device__ __forceinline__ Q4<T> qconj(const Q4<T>& a) { Q4<T> r; r.w = a.w; r.x = -a.x; r.y = -a.y; r.z = -a.z; return r; }

// float <-> nf vector conversions
__device__ __forceinline__ V3<nf> to_nf(const V3<float>& a) { return v3<nf>(nf(a.x), nf(a.y), nf(a.z)); }
__device__ __forceinline__ V3<float> to_f(const V3<nf>& a) { return v3<float>(a.x.v, a.y.v, a.z.v); }
__device__ __forceinline__ V3<float> f3(float4 a) { return v3<float>(a.x, a.y, a.z); }
__device__ __forceinline__ float4 f4(const V3<float>& a, float w) { return make_float4(a.x, a.y, a.z, w); }

// Explicitly fused float helpers for the solver's hot loops. The library is
// compiled with -fmad=false, so these are the only fused multiply-adds: one
// correctly rounded fmaf does not depend on the surrounding code, which keeps
// every execution form of the step bitwise identical.
__device__ __forceinline__ float dotf(const V3<float>& a, const V3<float>& b) {
  return fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)); }
__device__ __forceinline__ V3<float> crossf(const V3<float>& a, const V3<float>& b) {
  return v3<float>(fmaf(a.y, b.z, -(a.z * b.y)), fmaf(a.z, b.x, -(a.x * b.z)), fmaf(a.x, b.y, -(a.y * b.x))); }
__device__ __forceinline__ V3<float> axpyf(const V3<float>& y, const V3<float>& x, float s) {
  return v3<float>(fmaf(x.x, s, y.x), fmaf(x.y, s, y.y), fmaf(x.z, s, y.z)); }

// symmetric 3x3 stored as (xx, xy, xz, yy) + (yz, zz)
struct Sym3 { float xx, xy, xz, yy, yz, zz; };
__device__ __forceinline__ V3<float> smul(const Sym3& S, const V3<float>& v) {
  return v3<float>(S.xx * v.x + S.xy * v.y + S.xz * v.z,
                   S.xy * v.x + S.yy * v.y + S.yz * v.z,
                   S.xz * v.x + S.yz * v.y + S.zz * v.z);
}
__device__ __forceinline__ V3<float> smulf(const Sym3& S, const V3<float>& v) {
  return v3<float>(fmaf(S.xz, v.z, fmaf(S.xy, v.y, S.xx * v.x)),
                   fmaf(S.yz, v.z, fmaf(S.yy, v.y, S.xy * v.x)),
                   fmaf(S.zz, v.z, fmaf(S.yz, v.y, S.xz * v.x)));
}

}  // namespace msh
