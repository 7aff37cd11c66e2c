// Per-point work shared by the stencil sweeps: H applied at one output vector from its
// z-column queue (registers) and its x/y neighbours (shared-memory plane), the projector
// scatter, and the mode's epilogue (store a Taylor term, or combine the series and emit
// the density; optional energy/current partial sums).
//
// H t(r) = (w0 + V_eff(r)) t(r) + sum_m w_m [sum of the 6 neighbours at distance m]
//          [- i A . grad_h t(r)]  (velocity gauge, periodic cells)
//          + sum_(a,j) beta_aj(r) phase* q_aj    (Kleinman-Bylander term, precomputed per
//                                                 sphere point by the projector step)
// with w0 = -3 c_0 / (2 h^2), w_m = -c_m / (2 h^2) (central FD weights c_m of order 2M).
#pragma once
#include "tdks_internal.cuh"
#include "tdks_vec.cuh"

namespace tdks {

// Energy / current partial sums of one thread.  complex128: FP64; complex64: FP32
// products accumulated as double-float (no FP64 instruction per value).
template <int P> struct ObsAcc;
template <> struct ObsAcc<P_C128> {
  double e = 0.0, j[3] = {0.0, 0.0, 0.0};
  __device__ __forceinline__ void add_e(double2 c, double2 h) { e += c.x * h.x + c.y * h.y; }
  __device__ __forceinline__ void add_j(int a, double2 c, double2 g) { j[a] += c.x * g.y - c.y * g.x; }
  __device__ __forceinline__ double get_e() const { return e; }
  __device__ __forceinline__ double get_j(int a) const { return j[a]; }
};
template <> struct ObsAcc<P_C64> {
  float eh = 0.f, el = 0.f, jh[3] = {0.f, 0.f, 0.f}, jl[3] = {0.f, 0.f, 0.f};
  __device__ __forceinline__ void add_e(ulonglong2 c, ulonglong2 h) {
    const float2 c0 = up2(c.x), c1 = up2(c.y), h0 = up2(h.x), h1 = up2(h.y);
    df_acc(eh, el, (c0.x * h0.x + c0.y * h0.y) + (c1.x * h1.x + c1.y * h1.y));
  }
  __device__ __forceinline__ void add_j(int a, ulonglong2 c, ulonglong2 g) {
    const float2 c0 = up2(c.x), c1 = up2(c.y), g0 = up2(g.x), g1 = up2(g.y);
    df_acc(jh[a], jl[a], (c0.x * g0.y - c0.y * g0.x) + (c1.x * g1.y - c1.y * g1.x));
  }
  __device__ __forceinline__ double get_e() const { return (double)eh + (double)el; }
  __device__ __forceinline__ double get_j(int a) const { return (double)jh[a] + (double)jl[a]; }
};

template <> struct ObsAcc<P_C64S> {
  float eh = 0.f, el = 0.f, jh[3] = {0.f, 0.f, 0.f}, jl[3] = {0.f, 0.f, 0.f};
  __device__ __forceinline__ void add_e(u64 c, u64 h) {
    const float2 c0 = up2(c), h0 = up2(h);
    df_acc(eh, el, c0.x * h0.x + c0.y * h0.y);
  }
  __device__ __forceinline__ void add_j(int a, u64 c, u64 g) {
    const float2 c0 = up2(c), g0 = up2(g);
    df_acc(jh[a], jl[a], c0.x * g0.y - c0.y * g0.x);
  }
  __device__ __forceinline__ double get_e() const { return (double)eh + (double)el; }
  __device__ __forceinline__ double get_j(int a) const { return (double)jh[a] + (double)jl[a]; }
};

// Diagonal weight w0 in the compute precision.
template <int P> struct W0T { typedef float type; };
template <> struct W0T<P_C128> { typedef double type; };

// H applied at one point.  The z-column queue is the circular register array Q of QN
// (>= 2M+1) entries; plane z+j (j = -M..M) sits in Q[(QB + M + j) % QN] (QB: compile-time
// rotation, so no register moves per plane).  Sp = shared plane z (vectors, row stride SXO
// vectors), csl = own slot.  Returns H t; gax receives the three FD gradients when `grads`
// is set (observables of periodic cells).
template <int M, int P, int BLOCH, int QB = 0, int QN = 2 * M + 1>
__device__ __forceinline__ typename VT<P>::V
stencil_point(const SweepParams &p, const typename VT<P>::S *W, typename W0T<P>::type w0,
              const typename VT<P>::V *Q, const typename VT<P>::V *Sp, int csl, int SXO,
              typename VT<P>::R ve, bool need_grad, bool grads, typename VT<P>::V *gax) {
  typedef VT<P> T;
  typedef typename T::V V;
  const V c0 = Q[(QB + M) % QN];
  V acc = T::mul(T::diag(ve, w0), c0);
  V gsum = T::zero();
#pragma unroll
  for (int m = 1; m <= M; m++) {
    const V zm = Q[(QB + M - m) % QN], zp = Q[(QB + M + m) % QN];
    const V xm = Sp[csl - m * OVC], xp = Sp[csl + m * OVC];
    const V ym = Sp[csl - m * SXO], yp = Sp[csl + m * SXO];
    const V s6 = T::add(T::add(T::add(zm, zp), T::add(xm, xp)), T::add(ym, yp));
    acc = T::fma(W[m], s6, acc);
    if (BLOCH && need_grad) {
      const V dx = T::sub(xp, xm), dy = T::sub(yp, ym), dz = T::sub(zp, zm);
      gsum = T::fma(T::bc(p.A[0] * p.gw[m]), dx,
                    T::fma(T::bc(p.A[1] * p.gw[m]), dy, T::fma(T::bc(p.A[2] * p.gw[m]), dz, gsum)));
      if (grads) {
        const typename T::S gm = T::bc(p.gw[m]);
        gax[0] = T::fma(gm, dx, gax[0]);
        gax[1] = T::fma(gm, dy, gax[1]);
        gax[2] = T::fma(gm, dz, gax[2]);
      }
    }
  }
  if (BLOCH && need_grad) acc = T::add(acc, T::negi(gsum));
  return acc;
}

// Non-local (Kleinman-Bylander) term of a point, precomputed per sphere point by the
// projector step: nlk = the item's (kb, v) column of nl; row r0 for points with entries,
// the zero row n_ent for the others (a branch-free load that can be issued early).
template <int P>
__device__ __forceinline__ typename VT<P>::V nl_term(const typename VT<P>::V *nlk, int n_ent, int r0, int r1) {
  return VT<P>::ld(nlk + (long)(r1 > r0 ? r0 : n_ent) * VT<P>::OV);
}
template <int P>
__device__ __forceinline__ const typename VT<P>::V *nl_column(const SweepParams &p, int kb, int v) {
  return reinterpret_cast<const typename VT<P>::V *>(p.nl) + (long)kb * (p.n_ent + 1) * VT<P>::OV + v;
}

// Own-point operands of the last sweep (state parts and earlier terms).
template <int P> struct LastOperands {
  typename VT<P>::V hi, lo, t1, t2;
};

template <int P>
__device__ __forceinline__ void load_last(const SweepParams &p, long idx, LastOperands<P> &o) {
  typedef typename VT<P>::V V;
  o.hi = VT<P>::ld(reinterpret_cast<const V *>(p.psi) + idx);
  o.lo = P != P_C128 ? VT<P>::ld(reinterpret_cast<const V *>(p.psi_lo) + idx) : VT<P>::zero();
  o.t1 = VT<P>::ld(reinterpret_cast<const V *>(p.t1) + idx);
  o.t2 = VT<P>::ld(reinterpret_cast<const V *>(p.t2) + idx);
}

// Per-item epilogue operands, read from the parameters once per work item (inside the
// plane loop every asm memory clobber would make the compiler load them again).
struct Epi {
  void *out, *psi, *psi_lo;
  double *dens_part;
  double wocc;  // k-weight times occupation of the item's k-point
};
__device__ __forceinline__ Epi make_epi(const SweepParams &p, int kidx) {
  return Epi{p.out, p.psi, p.psi_lo, p.dens_part, p.wocc[kidx]};
}

// Epilogue of one output vector.  idx = vector index ((kb*N + pt)*OVC + v); (CR, CI) = the
// Taylor coefficient, converted to the compute precision once per work item.
template <int P, int MODE>
__device__ __forceinline__ void finish_point(const Epi &ep, typename VT<P>::S CR, typename VT<P>::S CI, bool own,
                                             long idx, int v, typename VT<P>::V c0, typename VT<P>::V acc,
                                             const LastOperands<P> &lo_ops) {
  typedef VT<P> T;
  typedef typename T::V V;
  const V outv = T::cmul(CR, CI, acc);
  if (MODE != MODE_LAST) {
    if (own) reinterpret_cast<V *>(ep.out)[idx] = outv;
  } else {
    V hi = lo_ops.hi, lo_out;
    typename Combine<P>::A dh, dl;
    Combine<P>::run(hi, lo_ops.lo, lo_ops.t1, lo_ops.t2, c0, outv, lo_out, dh, dl);
    if (own) {
      reinterpret_cast<V *>(ep.psi)[idx] = hi;
      if (P != P_C128) reinterpret_cast<V *>(ep.psi_lo)[idx] = lo_out;
    }
    Combine<P>::reduce_point(dh, dl);
    if (own && v == 0) Combine<P>::store_density(ep.dens_part + idx / T::OV, ep.wocc, dh, dl);
  }
}

template <int P, int MODE>
__device__ __forceinline__ void finish_point(const SweepParams &p, typename VT<P>::S CR, typename VT<P>::S CI,
                                             bool own, long idx, int v, int kidx, typename VT<P>::V c0,
                                             typename VT<P>::V acc, const LastOperands<P> &lo_ops) {
  finish_point<P, MODE>(make_epi(p, kidx), CR, CI, own, idx, v, c0, acc, lo_ops);
}

// Block reduction of the observable partials of one work item into obs_part[item].
template <int P, int NT>
__device__ __forceinline__ void reduce_obs(const SweepParams &p, const ObsAcc<P> &oa, long item, int kidx,
                                           double (*red)[4]) {
  const int tid = threadIdx.x;
  double vals[4] = {oa.get_e(), oa.get_j(0), oa.get_j(1), oa.get_j(2)};
#pragma unroll
  for (int i = 0; i < 4; i++) {
    double x = vals[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((tid & 31) == 0) red[tid >> 5][i] = x;
  }
  __syncthreads();
  if (tid < 4) {
    double x = 0.0;
    for (int w = 0; w < NT / 32; w++) x += red[w][tid];
    p.obs_part[item * 4 + tid] = p.wocc[kidx] * x;
  }
}

}  // namespace tdks
