// Per-precision 16-byte vector arithmetic used by the stencil sweep and projector kernels.
//
// complex128: one thread vector = one double2 (re, im).
// complex64 : one thread vector = two complex64, held as two packed 64-bit registers
//             (re0, im0), (re1, im1); arithmetic uses the paired-FP32 instructions of
//             sm_100+ (add/sub/mul/fma .f32x2), which halve the instruction count of the
//             FP32 stencil.
#pragma once
#include <cuda_runtime.h>
#include "tdks_internal.cuh"

namespace tdks {

typedef unsigned long long u64;

__device__ __forceinline__ u64 pk2(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 up2(u64 a) {
  float2 r;
  asm("mov.b64 {%0,%1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a));
  return r;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {  // a * b + c
  u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// (-im, re): multiply by +i
__device__ __forceinline__ u64 ipos2(u64 a) {
  float2 f = up2(a);
  return pk2(-f.y, f.x);
}

template <int P> struct VT;

template <> struct VT<P_C128> {
  typedef double2 V;
  typedef double S;   // broadcast scalar
  typedef double R;   // scalar type of the potential arrays
  static __device__ __forceinline__ V zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ S bc(double s) { return s; }
  static __device__ __forceinline__ V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ V sub(V a, V b) { return make_double2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ V mul(S s, V a) { return make_double2(s * a.x, s * a.y); }
  static __device__ __forceinline__ V fma(S s, V a, V c) {
    return make_double2(__fma_rn(s, a.x, c.x), __fma_rn(s, a.y, c.y));
  }
  // (cr + i ci) * a
  static __device__ __forceinline__ V cmul(S cr, S ci, V a) {
    return make_double2(cr * a.x - ci * a.y, cr * a.y + ci * a.x);
  }
  // -i a
  static __device__ __forceinline__ V negi(V a) { return make_double2(a.y, -a.x); }
  static __device__ __forceinline__ V ld(const V *p) { return __ldg(p); }
  // state storage (complex128) -> compute vector
  static __device__ __forceinline__ V ld_state(const double2 *psi, long pt, int v) {
    return __ldg(psi + pt * OVC + v);
  }
  // sum over the vector's complex entries of w * |a|^2, and the vector as doubles
  static __device__ __forceinline__ void to_d(V a, double2 *o) { o[0] = a; }
  static constexpr int CPV = 1;  // complex values per vector
};

template <> struct VT<P_C64> {
  typedef ulonglong2 V;
  typedef u64 S;
  typedef float R;
  static __device__ __forceinline__ V zero() { return make_ulonglong2(0ull, 0ull); }
  static __device__ __forceinline__ S bc(double s) { float f = (float)s; return pk2(f, f); }
  static __device__ __forceinline__ V add(V a, V b) { return make_ulonglong2(add2(a.x, b.x), add2(a.y, b.y)); }
  static __device__ __forceinline__ V sub(V a, V b) { return make_ulonglong2(sub2(a.x, b.x), sub2(a.y, b.y)); }
  static __device__ __forceinline__ V mul(S s, V a) { return make_ulonglong2(mul2(s, a.x), mul2(s, a.y)); }
  static __device__ __forceinline__ V fma(S s, V a, V c) { return make_ulonglong2(fma2(s, a.x, c.x), fma2(s, a.y, c.y)); }
  static __device__ __forceinline__ V cmul(S cr, S ci, V a) {
    return make_ulonglong2(fma2(ci, ipos2(a.x), mul2(cr, a.x)), fma2(ci, ipos2(a.y), mul2(cr, a.y)));
  }
  static __device__ __forceinline__ V negi(V a) {
    float2 p = up2(a.x), q = up2(a.y);
    return make_ulonglong2(pk2(p.y, -p.x), pk2(q.y, -q.x));
  }
  static __device__ __forceinline__ V ld(const V *p) { return __ldg(p); }
  static __device__ __forceinline__ V ld_state(const double2 *psi, long pt, int v) {
    const double2 *b = psi + pt * (2 * OVC) + 2 * v;
    double2 a = __ldg(b), c = __ldg(b + 1);
    return make_ulonglong2(pk2((float)a.x, (float)a.y), pk2((float)c.x, (float)c.y));
  }
  static __device__ __forceinline__ void to_d(V a, double2 *o) {
    float2 p = up2(a.x), q = up2(a.y);
    o[0] = make_double2(p.x, p.y);
    o[1] = make_double2(q.x, q.y);
  }
  static constexpr int CPV = 2;
};

}  // namespace tdks
