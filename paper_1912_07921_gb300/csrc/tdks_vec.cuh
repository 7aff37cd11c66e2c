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
constexpr u64 SIGN2 = 0x8000000080000000ull;

// Double-float arithmetic (a value is the unevaluated sum hi + lo of two FP32 numbers,
// |lo| <= ulp(hi)/2, ~48-bit significand), from the error-free transformations of
// Knuth (TwoSum) and Dekker (FastTwoSum); lane-wise on packed pairs.
// (hi, lo) + d  ->  (ho, lout)
__device__ __forceinline__ void df_add2(u64 hi, u64 lo, u64 d, u64 &ho, u64 &lout) {
  const u64 s = add2(hi, d);
  const u64 bb = sub2(s, hi);
  u64 e = add2(sub2(hi, sub2(s, bb)), sub2(d, bb));
  e = add2(e, lo);
  ho = add2(s, e);
  lout = sub2(e, sub2(ho, s));
}
// scalar TwoSum: s + e = a + b exactly
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
  const float s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
  return s;
}
// (h, l) += (bh, bl), both double-float
__device__ __forceinline__ void df_add_df(float &h, float &l, float bh, float bl) {
  float e;
  const float s = two_sum(h, bh, e);
  e += l + bl;
  h = s + e;
  l = e - (h - s);
}
// accumulate x into the double-float (h, l)
__device__ __forceinline__ void df_acc(float &h, float &l, float x) {
  float e;
  const float s = two_sum(h, x, e);
  l += e;
  h = s + l;
  l = l - (h - s);
}

template <int P> struct VT;

template <> struct VT<P_C128> {
  typedef double2 V;
  typedef double S;   // broadcast scalar
  typedef double R;   // scalar type of the potential arrays
  static __device__ __forceinline__ V zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ S bc(double s) { return s; }
  // a coefficient from its FP64 value (the FP32 copy is for complex64)
  static __device__ __forceinline__ S coef(double d, float) { return d; }
  // diagonal (V_eff(r) + w0) broadcast, in the compute precision
  static __device__ __forceinline__ S diag(R ve, double w0) { return ve + w0; }
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
  static __device__ __forceinline__ void to_d(V a, double2 *o) { o[0] = a; }
  static constexpr int CPV = 1;  // complex values per vector
  static constexpr int OV = 4;   // vectors per (point, batch): 64 bytes
};

template <> struct VT<P_C64> {
  typedef ulonglong2 V;
  typedef u64 S;
  typedef float R;
  static __device__ __forceinline__ V zero() { return make_ulonglong2(0ull, 0ull); }
  static __device__ __forceinline__ S bc(double s) { float f = (float)s; return pk2(f, f); }
  // a coefficient from its FP32 copy (no FP64 conversion in the kernel)
  static __device__ __forceinline__ S coef(double, float f) { return pk2(f, f); }
  static __device__ __forceinline__ S diag(R ve, float w0) { const float d = ve + w0; return pk2(d, d); }
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
  static __device__ __forceinline__ void to_d(V a, double2 *o) {
    float2 p = up2(a.x), q = up2(a.y);
    o[0] = make_double2(p.x, p.y);
    o[1] = make_double2(q.x, q.y);
  }
  static constexpr int CPV = 2;
  static constexpr int OV = 4;
};

// complex64 with one complex value per thread vector (one packed 64-bit register); the
// same per-component arithmetic as VT<P_C64>, on half the data per thread.
template <> struct VT<P_C64S> {
  typedef u64 V;
  typedef u64 S;
  typedef float R;
  static __device__ __forceinline__ V zero() { return 0ull; }
  static __device__ __forceinline__ S bc(double s) { float f = (float)s; return pk2(f, f); }
  static __device__ __forceinline__ S coef(double, float f) { return pk2(f, f); }
  static __device__ __forceinline__ S diag(R ve, float w0) { const float d = ve + w0; return pk2(d, d); }
  static __device__ __forceinline__ V add(V a, V b) { return add2(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return sub2(a, b); }
  static __device__ __forceinline__ V mul(S s, V a) { return mul2(s, a); }
  static __device__ __forceinline__ V fma(S s, V a, V c) { return fma2(s, a, c); }
  static __device__ __forceinline__ V cmul(S cr, S ci, V a) { return fma2(ci, ipos2(a), mul2(cr, a)); }
  static __device__ __forceinline__ V negi(V a) {
    const float2 p = up2(a);
    return pk2(p.y, -p.x);
  }
  static __device__ __forceinline__ V ld(const V *p) { return __ldg(reinterpret_cast<const unsigned long long *>(p)); }
  static __device__ __forceinline__ void to_d(V a, double2 *o) {
    const float2 p = up2(a);
    o[0] = make_double2(p.x, p.y);
  }
  static constexpr int CPV = 1;
  static constexpr int OV = 8;
};

// ---------------------------------------------------------------------------------
// Taylor combine of the last sweep and the point's density contribution.
//   complex128: psi' = (((psi + t1) + t2) + t3) + t4 in FP64;
//   complex64 : the state is the double-float pair (hi, lo); delta = t1+t2+t3+t4 in FP32,
//               psi' = (hi, lo) + delta by TwoSum/FastTwoSum; |psi'|^2 as a double-float
//               partial (hi^2 exactly by FMA, + 2 hi lo), no FP64 instruction per value.
// dens_hi + dens_lo receives sum over the thread's complex entries of |psi'|^2.
// ---------------------------------------------------------------------------------
template <int P> struct Combine;

template <> struct Combine<P_C128> {
  typedef double2 V;
  typedef double A;
  static __device__ __forceinline__ void run(V &psi, V lo_unused, V t1, V t2, V t3, V t4, V &lo_out,
                                             A &dh, A &dl) {
    (void)lo_unused;
    double re = psi.x + t1.x, im = psi.y + t1.y;
    re += t2.x; im += t2.y;
    re += t3.x; im += t3.y;
    re += t4.x; im += t4.y;
    psi = make_double2(re, im);
    lo_out = make_double2(0.0, 0.0);
    dh = re * re + im * im;
    dl = 0.0;
  }
  // sum over the 4 consecutive lanes that hold one (point, batch)
  static __device__ __forceinline__ void reduce_point(A &h, A &l) {
    h += __shfl_xor_sync(0xffffffffu, h, 1);
    h += __shfl_xor_sync(0xffffffffu, h, 2);
    (void)l;
  }
  static __device__ __forceinline__ double value(A h, A l) { (void)l; return h; }
  // the point's density partial: w_k f sum |psi|^2 in FP64
  static __device__ __forceinline__ void store_density(double *slot, double wocc, A h, A l) {
    (void)l;
    *slot = wocc * h;
  }
};

template <> struct Combine<P_C64> {
  typedef ulonglong2 V;
  typedef float A;
  static __device__ __forceinline__ float sq_parts(u64 h, u64 l, float &err) {
    // sum of the two lanes' |x|^2 = (h + l)^2 ~ h^2 + 2 h l, returned as s + err
    const u64 p = mul2(h, h);
    const u64 e = fma2(add2(h, h), l, fma2(h, h, p ^ SIGN2));
    const float2 pp = up2(p), ee = up2(e);
    float e2;
    const float s = two_sum(pp.x, pp.y, e2);
    err = e2 + ee.x + ee.y;
    return s;
  }
  static __device__ __forceinline__ void run(V &hi, V lo, V t1, V t2, V t3, V t4, V &lo_out,
                                             A &dh, A &dl) {
    const u64 dx = add2(add2(add2(t1.x, t2.x), t3.x), t4.x);
    const u64 dy = add2(add2(add2(t1.y, t2.y), t3.y), t4.y);
    u64 hx, lx, hy, ly;
    df_add2(hi.x, lo.x, dx, hx, lx);
    df_add2(hi.y, lo.y, dy, hy, ly);
    hi = make_ulonglong2(hx, hy);
    lo_out = make_ulonglong2(lx, ly);
    float ea, eb, ec;
    const float sa = sq_parts(hx, lx, ea), sb = sq_parts(hy, ly, eb);
    dh = two_sum(sa, sb, ec);
    dl = ea + eb + ec;
  }
  // sum over the 4 consecutive lanes that hold one (point, batch)
  static __device__ __forceinline__ void reduce_point(A &h, A &l) {
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
      float e;
      h = two_sum(h, oh, e);
      l = l + ol + e;
    }
  }
  static __device__ __forceinline__ double value(A h, A l) { return (double)h + (double)l; }
  // the point's density partial: sum |psi|^2 unweighted, as the pair (h, l) in the 8-byte
  // slot (the LDA kernel forms w_k f ((double)h + (double)l)); no FP64 instruction here
  static __device__ __forceinline__ void store_density(double *slot, double wocc, A h, A l) {
    (void)wocc;
    *reinterpret_cast<float2 *>(slot) = make_float2(h, l);
  }
};

// One complex value per lane: the same state update as Combine<P_C64> per component, the
// density summed over the 8 lanes of a (point, batch).
template <> struct Combine<P_C64S> {
  typedef u64 V;
  typedef float A;
  static __device__ __forceinline__ void run(V &hi, V lo, V t1, V t2, V t3, V t4, V &lo_out, A &dh, A &dl) {
    const u64 d = add2(add2(add2(t1, t2), t3), t4);
    u64 h, l;
    df_add2(hi, lo, d, h, l);
    hi = h;
    lo_out = l;
    dh = Combine<P_C64>::sq_parts(h, l, dl);
  }
  static __device__ __forceinline__ void reduce_point(A &h, A &l) {
#pragma unroll
    for (int o = 1; o <= 4; o <<= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
      float e;
      h = two_sum(h, oh, e);
      l = l + ol + e;
    }
  }
  static __device__ __forceinline__ double value(A h, A l) { return (double)h + (double)l; }
  static __device__ __forceinline__ void store_density(double *slot, double wocc, A h, A l) {
    Combine<P_C64>::store_density(slot, wocc, h, l);
  }
};

}  // namespace tdks
