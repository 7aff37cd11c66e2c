// Auxiliary kernels of the TDKS library: Kleinman-Bylander gather-dot, density, LDA
// exchange + effective potential, observable finalisation, layout packing.
#include "tdks_internal.cuh"
#include "tdks_vec.cuh"

namespace tdks {

// ---------------------------------------------------------------------------------
// Projector gather-dot: q[kb][a][j][v] = D_aj h^3 sum_{u in S_a} beta_aj(u - R_a)
//                                         exp(+i (k.T_u + A.d_u)) in(cell(u))[v]
// (the <beta_aj|psi> of V_NL = sum |beta> D <beta|; the paper's norm-conserving
// pseudopotentials, Sec. "Magneto-optics" and Sec. "Periodic systems", with synthetic
// Gaussian-times-polynomial projectors).  Stage 1: n_chunks CTAs per (atom, kb), each
// summing a contiguous share of the sphere with 64 point lanes x OVC vectors (warp
// shuffles, then warps through shared memory in a fixed order); stage 2 adds the chunks in
// order and applies D_aj h^3.  No atomics: the result does not depend on timing.
// ---------------------------------------------------------------------------------
constexpr int GATHER_THREADS = 256;

int gather_chunks(long units) {
  const long want = (152L * 4 + units - 1) / units;
  return (int)(want < 1 ? 1 : (want > 16 ? 16 : want));
}

template <int P, int BLOCH>
__device__ __forceinline__ void gather_body(const GatherParams &p, int a, int kb, int chunk) {
  typedef VT<P> T;
  typedef typename T::V V;
  const int kidx = kb / p.n_batches;
  const int tid = threadIdx.x, v = tid % OVC, lane = tid / OVC;
  constexpr int LANES = GATHER_THREADS / OVC;
  // per-lane sums: FP64 for complex128 systems, FP32 for complex64 systems; the cross-lane
  // sums below are FP64 for both.
  double2 accd[4] = {};
  float2 accf[4][2] = {};
  const int a0 = p.atom_begin[a], a1 = p.atom_begin[a + 1];
  const int len = (a1 - a0 + p.n_chunks - 1) / p.n_chunks;
  const int e0 = a0 + chunk * len, e1 = min(a1, e0 + len);
  const bool phase = BLOCH || (p.A[0] != 0.0 || p.A[1] != 0.0 || p.A[2] != 0.0);
  for (int e = e0 + lane; e < e1; e += LANES) {
    if constexpr (P == P_C64) {
      // compact entry arrays: 8 + 16 bytes per entry instead of the full record
      const int2 ca = p.ent_ca[e];
      const float4 b4 = p.ent_beta[e];
      const V x = T::ld(reinterpret_cast<const V *>(p.in) + ((long)kb * p.N + ca.x) * OVC + v);
      float c = 1.f, s = 0.f;
      if (phase) {
        if (p.phase) {
          const float2 ph = p.phase[(long)kidx * p.n_ent + e];
          c = ph.x;
          s = ph.y;
        } else {
          const ProjEntry &E = p.ent[e];
          double ang = p.A[0] * E.d[0] + p.A[1] * E.d[1] + p.A[2] * E.d[2];
          if (BLOCH) ang += p.kvec[3 * kidx] * E.T[0] + p.kvec[3 * kidx + 1] * E.T[1] + p.kvec[3 * kidx + 2] * E.T[2];
          sincosf((float)ang, &s, &c);
        }
      }
      const float2 x0 = up2(x.x), x1 = up2(x.y);
      const float2 y0 = make_float2(c * x0.x - s * x0.y, c * x0.y + s * x0.x);
      const float2 y1 = make_float2(c * x1.x - s * x1.y, c * x1.y + s * x1.x);
      const float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int j = 0; j < 4; j++) {
        accf[j][0].x = fmaf(b[j], y0.x, accf[j][0].x); accf[j][0].y = fmaf(b[j], y0.y, accf[j][0].y);
        accf[j][1].x = fmaf(b[j], y1.x, accf[j][1].x); accf[j][1].y = fmaf(b[j], y1.y, accf[j][1].y);
      }
    } else {
      const ProjEntry &E = p.ent[e];
      const long pt = (long)kb * p.N + E.cell;
      const V x = T::ld(reinterpret_cast<const V *>(p.in) + pt * OVC + v);
      double c = 1.0, s = 0.0;
      if (phase) {
        double ang = p.A[0] * E.d[0] + p.A[1] * E.d[1] + p.A[2] * E.d[2];
        if (BLOCH) ang += p.kvec[3 * kidx] * E.T[0] + p.kvec[3 * kidx + 1] * E.T[1] + p.kvec[3 * kidx + 2] * E.T[2];
        sincos(ang, &s, &c);
      }
      const double2 xd = *reinterpret_cast<const double2 *>(&x);
      const double xr = c * xd.x - s * xd.y, xi = c * xd.y + s * xd.x;
#pragma unroll
      for (int j = 0; j < 4; j++) {
        accd[j].x += E.betad[j] * xr;
        accd[j].y += E.betad[j] * xi;
      }
    }
  }
  // reduce over lanes with equal v (they differ in bits 2..4 of the lane id), then over the
  // warps in a fixed order.  complex64: the lane sums are FP32 (as the per-lane sums), so
  // the shuffles stay off GB300's slow FP64 pipe; the warp partials are FP64.
  __shared__ double2 red[GATHER_THREADS / 32][4][OVC][2];
#pragma unroll
  for (int j = 0; j < 4; j++)
#pragma unroll
    for (int cc = 0; cc < 2; cc++) {
      if constexpr (P == P_C64) {
        float2 x = accf[j][cc];
        for (int o = 4; o < 32; o <<= 1) {
          x.x += __shfl_xor_sync(0xffffffffu, x.x, o);
          x.y += __shfl_xor_sync(0xffffffffu, x.y, o);
        }
        if ((tid & 31) < OVC) red[tid >> 5][j][v][cc] = make_double2(x.x, x.y);
      } else if (cc == 0) {
        double2 x = accd[j];
        for (int o = 4; o < 32; o <<= 1) {
          x.x += __shfl_xor_sync(0xffffffffu, x.x, o);
          x.y += __shfl_xor_sync(0xffffffffu, x.y, o);
        }
        if ((tid & 31) < OVC) {
          red[tid >> 5][j][v][0] = x;
          red[tid >> 5][j][v][1] = make_double2(0.0, 0.0);
        }
      }
    }
  __syncthreads();
  if (tid < 4 * OVC) {
    const int j = tid / OVC, vv = tid % OVC;
    double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
    for (int w = 0; w < GATHER_THREADS / 32; w++) {
      s0.x += red[w][j][vv][0].x; s0.y += red[w][j][vv][0].y;
      s1.x += red[w][j][vv][1].x; s1.y += red[w][j][vv][1].y;
    }
    double2 *qp = p.qpart + ((((long)(kb * p.n_atoms + a) * p.n_chunks + chunk) * 4 + j) * OVC + vv) * 2;
    qp[0] = s0;
    qp[1] = s1;
  }
}

// Stage 2 for one (atom, kb): thread (j, v) adds the chunk partials in order, times D h^3.
template <int P>
__device__ __forceinline__ void gather_finish(const GatherParams &p, int a, int kb, int t) {
  typedef typename VT<P>::V V;
  const int j = t / OVC, vv = t % OVC;
  double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
  for (int c = 0; c < p.n_chunks; c++) {
    const double2 *qp = p.qpart + ((((long)(kb * p.n_atoms + a) * p.n_chunks + c) * 4 + j) * OVC + vv) * 2;
    s0.x += qp[0].x; s0.y += qp[0].y;
    s1.x += qp[1].x; s1.y += qp[1].y;
  }
  const double f = p.D[4 * a + j] * p.h3;
  V *q = reinterpret_cast<V *>(p.q) + ((long)(kb * p.n_atoms + a) * 4 + j) * OVC + vv;
  if constexpr (P == P_C64) {
    *q = make_ulonglong2(pk2((float)(f * s0.x), (float)(f * s0.y)), pk2((float)(f * s1.x), (float)(f * s1.y)));
  } else {
    *q = make_double2(f * s0.x, f * s0.y);
  }
}

template <int P, int BLOCH>
__global__ void __launch_bounds__(GATHER_THREADS) gather_kernel(const GatherParams p) {
  gather_body<P, BLOCH>(p, blockIdx.x / p.n_chunks, blockIdx.y, blockIdx.x % p.n_chunks);
}

// 16 threads per (atom, kb) unit, 8 units per CTA
template <int P>
__global__ void __launch_bounds__(128) gather_finish_kernel(const GatherParams p) {
  const long u = blockIdx.x * 8L + threadIdx.x / 16;
  if (u >= (long)p.n_atoms * p.n_kb) return;
  gather_finish<P>(p, (int)(u % p.n_atoms), (int)(u / p.n_atoms), threadIdx.x % 16);
}

// Non-local term at every point inside a sphere (the scatter half of V_nl):
//   nl(r) = sum over the point's entries (a, j) of beta_aj(r) e^{-i phi} q_aj,
//   phi = k . T + A . d (Bloch cells / velocity gauge), q_aj = D_aj h^3 <beta_aj|in>,
// summed in entry order from zero and stored at row r0 (the point's first entry) of
// nl[kb]; the sweeps add it to H in at the point.  Thread = (sphere point, v).
template <int P, int BLOCH>
__device__ __forceinline__ void nl_body(const GatherParams &p, long t, int kb) {
  typedef VT<P> T;
  typedef typename T::V V;
  const long sidx = t / OVC;
  const int v = (int)(t % OVC);
  if (sidx >= p.n_sp) return;
  const int2 r = p.sp[sidx];
  const int kidx = kb / p.n_batches;
  const bool phase = BLOCH || (p.A[0] != 0.0 || p.A[1] != 0.0 || p.A[2] != 0.0);
  V acc = T::zero();
  for (int e = r.x; e < r.y; e++) {
    const int ei = p.rowent[e];
    V x;
    if constexpr (P == P_C64) {
      const int2 ca = p.ent_ca[ei];
      const float4 b4 = p.ent_beta[ei];
      const V *qa = reinterpret_cast<const V *>(p.q) + ((long)(kb * p.n_atoms + ca.y) * 4) * OVC + v;
      x = T::mul(T::coef(0.0, b4.x), T::ld(qa));
      x = T::fma(T::coef(0.0, b4.y), T::ld(qa + OVC), x);
      x = T::fma(T::coef(0.0, b4.z), T::ld(qa + 2 * OVC), x);
      x = T::fma(T::coef(0.0, b4.w), T::ld(qa + 3 * OVC), x);
      if (phase) {
        float sn, cs;
        if (p.phase) {
          const float2 ph = p.phase[(long)kidx * p.n_ent + ei];
          cs = ph.x;
          sn = ph.y;
        } else {
          const ProjEntry &E = p.ent[ei];
          double ang = p.A[0] * E.d[0] + p.A[1] * E.d[1] + p.A[2] * E.d[2];
          if (BLOCH) ang += p.kvec[3 * kidx] * E.T[0] + p.kvec[3 * kidx + 1] * E.T[1] + p.kvec[3 * kidx + 2] * E.T[2];
          sincosf((float)ang, &sn, &cs);
        }
        x = T::cmul(pk2(cs, cs), pk2(-sn, -sn), x);
      }
    } else {
      const ProjEntry &E = p.ent[ei];
      const V *qa = reinterpret_cast<const V *>(p.q) + ((long)(kb * p.n_atoms + E.atom) * 4) * OVC + v;
      x = T::mul(E.betad[0], T::ld(qa));
#pragma unroll
      for (int j = 1; j < 4; j++) x = T::fma(E.betad[j], T::ld(qa + j * OVC), x);
      if (phase) {
        double ang = p.A[0] * E.d[0] + p.A[1] * E.d[1] + p.A[2] * E.d[2];
        if (BLOCH) ang += p.kvec[3 * kidx] * E.T[0] + p.kvec[3 * kidx + 1] * E.T[1] + p.kvec[3 * kidx + 2] * E.T[2];
        double sn, cs;
        sincos(ang, &sn, &cs);
        x = T::cmul(cs, -sn, x);
      }
    }
    acc = T::add(acc, x);
  }
  reinterpret_cast<V *>(p.nl)[((long)kb * (p.n_ent + 1) + r.x) * OVC + v] = acc;
}

// (with many k-batches each thread takes its (sphere point, vector) through a run of them: the
// point's entry data stays in L1 across the run, and a periodic cell's 64 k-batches need 8x
// fewer CTAs; a molecule's few k-batches keep one per CTA row, for parallelism)
constexpr int NL_KB_RUN = 8;
inline unsigned nl_kb_rows(int n_kb) { return n_kb >= 4 * NL_KB_RUN ? (n_kb + NL_KB_RUN - 1) / NL_KB_RUN : n_kb; }
template <int P, int BLOCH>
__global__ void __launch_bounds__(NL_THREADS) nl_kernel(const GatherParams p) {
  const long t = (long)blockIdx.x * NL_THREADS + threadIdx.x;
  if ((int)gridDim.y == p.n_kb) {
    nl_body<P, BLOCH>(p, t, blockIdx.y);
    return;
  }
  const int run = (p.n_kb + gridDim.y - 1) / gridDim.y;
  const int kb0 = blockIdx.y * run, kb1 = min(p.n_kb, kb0 + run);
  for (int kb = kb0; kb < kb1; kb++) nl_body<P, BLOCH>(p, t, kb);
}

// Batched gather: stage 1 over every system's (atom, kb, chunk) CTAs, stage 2 over every
// system's (atom, kb) units.  The system of a CTA (or unit) comes from a table.
template <int P>
__global__ void __launch_bounds__(GATHER_THREADS)
gather_batch_kernel(const GatherParams *gp, const long *begin, const int *sys_of) {
  const int s = sys_of[blockIdx.x];
  const GatherParams &p = gp[s];
  const long u = blockIdx.x - begin[s];
  const long unit = u / p.n_chunks;
  gather_body<P, 0>(p, (int)(unit % p.n_atoms), (int)(unit / p.n_atoms), (int)(u % p.n_chunks));
}

template <int P>
__global__ void __launch_bounds__(128)
gather_finish_batch_kernel(const GatherParams *gp, const long *ubegin, const int *sys_of, long total_units) {
  const long u = blockIdx.x * 8L + threadIdx.x / 16;
  if (u >= total_units) return;
  const int s = sys_of[u];
  const GatherParams &p = gp[s];
  const long local = u - ubegin[s];
  gather_finish<P>(p, (int)(local % p.n_atoms), (int)(local / p.n_atoms), threadIdx.x % 16);
}

// CTA c of the batched non-local kernel: system s with nbegin[s] <= c < nbegin[s+1]; within
// it, kb = local / chunks, chunk = local % chunks.
template <int P>
__global__ void __launch_bounds__(NL_THREADS)
nl_batch_kernel(const GatherParams *gp, const long *nbegin, const int *sys_of) {
  const int s = sys_of[blockIdx.x];
  const GatherParams &p = gp[s];
  const long local = blockIdx.x - nbegin[s];
  constexpr long RUN = (long)NL_THREADS * NL_BATCH_RUNS;
  const long chunks = ((long)p.n_sp * OVC + RUN - 1) / RUN;
  const int kb = (int)(local / chunks);
  const long t0 = (local % chunks) * RUN + threadIdx.x;
#pragma unroll 2
  for (int i = 0; i < NL_BATCH_RUNS; i++) nl_body<P, 0>(p, t0 + (long)i * NL_THREADS, kb);
}

cudaError_t launch_gather_batch(int prec, const GatherParams *gp, const long *begin, const long *ubegin,
                                const long *nbegin, const int *gsys, const int *usys, const int *nsys,
                                long total, long total_units, long total_nl, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const unsigned fgrid = (unsigned)((total_units + 7) / 8);
  if (prec == P_C64) {
    gather_batch_kernel<P_C64><<<(unsigned)total, GATHER_THREADS, 0, s>>>(gp, begin, gsys);
    gather_finish_batch_kernel<P_C64><<<fgrid, 128, 0, s>>>(gp, ubegin, usys, total_units);
    if (total_nl > 0) nl_batch_kernel<P_C64><<<(unsigned)total_nl, NL_THREADS, 0, s>>>(gp, nbegin, nsys);
  } else {
    gather_batch_kernel<P_C128><<<(unsigned)total, GATHER_THREADS, 0, s>>>(gp, begin, gsys);
    gather_finish_batch_kernel<P_C128><<<fgrid, 128, 0, s>>>(gp, ubegin, usys, total_units);
    if (total_nl > 0) nl_batch_kernel<P_C128><<<(unsigned)total_nl, NL_THREADS, 0, s>>>(gp, nbegin, nsys);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Projectors' share of the periodic cell's current (Sec. "Conductivities", eqn.
// current_density: the velocity operator i[H, r] includes i[V_NL, r]).  For one atom, one
// k-batch and the BS orbitals of the batch, with d = (sphere point, unwrapped) - R_a and the
// Bloch and gauge phase e^{i(k.T + A.d)} of each entry,
//   p_j = sum beta_j(d) e^{i..} phi,   q_jx = sum d_x beta_j(d) e^{i..} phi   (times h^3 each),
//   <phi| i[V_NL, r_x] |phi> = sum_j D_j i (p_j^* q_jx - q_jx^* p_j) = sum_j D_j (-2 Im(p_j^* q_jx)).
// Written as extra partial records (energy 0, three current sums in the units of the sweep's
// partials: w_k f times the velocity, over h^3) that the record's finalise adds in order.
// Once per record; complex128 systems in FP64, complex64 systems with FP32 lane sums.
// ---------------------------------------------------------------------------------
constexpr int NLC_THREADS = 128;

// per-lane sums of one orbital over a strided share of the atom's entries: FP64 for complex128
// systems; FP32 products and sums for complex64 systems (the FP64 pipe of GB300 is a small
// fraction of its FP32 one; the lane sums meet in FP64)
template <typename F>
__device__ __forceinline__ void nl_current_lane(const NlCurrentParams &p, int a, int kb, int o, int lane, int lanes,
                                                double *r) {
  const int kidx = kb / p.n_batches;
  const double kx = p.kvec[3 * kidx], ky = p.kvec[3 * kidx + 1], kz = p.kvec[3 * kidx + 2];
  F pr[4] = {}, pi[4] = {}, qr[4][3] = {}, qi[4][3] = {};
  for (int e = p.atom_begin[a] + lane; e < p.atom_begin[a + 1]; e += lanes) {
    const ProjEntry &E = p.ent[e];
    const long i = ((long)kb * p.N + E.cell) * p.BS + o;
    F xr, xi;
    if constexpr (sizeof(F) == 8) {
      const double2 v = reinterpret_cast<const double2 *>(p.psi)[i];
      xr = v.x;
      xi = v.y;
    } else {
      const float2 hi = reinterpret_cast<const float2 *>(p.psi)[i], lo = reinterpret_cast<const float2 *>(p.psi_lo)[i];
      xr = hi.x + lo.x;
      xi = hi.y + lo.y;
    }
    const double ang = kx * E.T[0] + ky * E.T[1] + kz * E.T[2] + p.A[0] * E.d[0] + p.A[1] * E.d[1] + p.A[2] * E.d[2];
    F sn, cs;
    if constexpr (sizeof(F) == 8) sincos(ang, &sn, &cs); else sincosf((float)ang, &sn, &cs);
    const F vr = cs * xr - sn * xi, vi = cs * xi + sn * xr;
    F b[4], d[3];
#pragma unroll
    for (int j = 0; j < 4; j++) b[j] = sizeof(F) == 8 ? (F)E.betad[j] : (F)E.beta[j];
#pragma unroll
    for (int x = 0; x < 3; x++) d[x] = (F)E.d[x];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      pr[j] += b[j] * vr;
      pi[j] += b[j] * vi;
#pragma unroll
      for (int x = 0; x < 3; x++) {
        qr[j][x] += d[x] * b[j] * vr;
        qi[j][x] += d[x] * b[j] * vi;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; j++) {
    r[8 * j] = pr[j];
    r[8 * j + 1] = pi[j];
#pragma unroll
    for (int x = 0; x < 3; x++) {
      r[8 * j + 2 + 2 * x] = qr[j][x];
      r[8 * j + 3 + 2 * x] = qi[j][x];
    }
  }
}

__global__ void __launch_bounds__(NLC_THREADS) nl_current_kernel(const NlCurrentParams p) {
  const int a = blockIdx.x, kb = blockIdx.y, t = threadIdx.x;
  const int o = t % p.BS, lane = t / p.BS, lanes = NLC_THREADS / p.BS;
  const int kidx = kb / p.n_batches;
  // sum over the lanes of each orbital in a fixed order
  __shared__ double red[NLC_THREADS][32];
  if (p.prec == P_C128) nl_current_lane<double>(p, a, kb, o, lane, lanes, red[t]);
  else nl_current_lane<float>(p, a, kb, o, lane, lanes, red[t]);
  __syncthreads();
  if (t < p.BS) {
    double sum[32];
    for (int c = 0; c < 32; c++) sum[c] = 0.0;
    for (int l = 0; l < lanes; l++)
      for (int c = 0; c < 32; c++) sum[c] += red[l * p.BS + t][c];
    double vel[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < 4; j++)
      for (int x = 0; x < 3; x++) {
        // Im(p^* q) = p_r q_i - p_i q_r
        const double im = sum[8 * j] * sum[8 * j + 3 + 2 * x] - sum[8 * j + 1] * sum[8 * j + 2 + 2 * x];
        vel[x] += p.D[4 * a + j] * (-2.0 * im);
      }
    double *out = p.out + ((long)kb * p.n_atoms * p.BS + (long)a * p.BS + t) * 4;
    const double f = p.wocc[kidx] * p.h3;  // (h^3)^2 of p and q, over the h^3 the finalise applies
    out[0] = 0.0;
    out[1] = f * vel[0];
    out[2] = f * vel[1];
    out[3] = f * vel[2];
  }
}

cudaError_t launch_nl_current(const NlCurrentParams &p, cudaStream_t s) {
  nl_current_kernel<<<dim3(p.n_atoms, p.n_kb), NLC_THREADS, 0, s>>>(p);
  return cudaGetLastError();
}

__global__ void phase_table_kernel(const ProjEntry *ent, int n_ent, int n_k, const double *kvec, double Ax,
                                   double Ay, double Az, int bloch, float2 *out) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)n_ent * n_k) return;
  const int e = (int)(i % n_ent), k = (int)(i / n_ent);
  const ProjEntry &E = ent[e];
  double ang = Ax * E.d[0] + Ay * E.d[1] + Az * E.d[2];
  if (bloch) ang += kvec[3 * k] * E.T[0] + kvec[3 * k + 1] * E.T[1] + kvec[3 * k + 2] * E.T[2];
  float sn, cs;
  sincosf((float)ang, &sn, &cs);
  out[i] = make_float2(cs, sn);
}

cudaError_t launch_phase_table(const ProjEntry *ent, int n_ent, int n_k, const double *kvec, const double A[3],
                               int bloch, float2 *out, cudaStream_t s) {
  const long n = (long)n_ent * n_k;
  if (n <= 0) return cudaSuccess;
  phase_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ent, n_ent, n_k, kvec, A[0], A[1], A[2], bloch,
                                                                 out);
  return cudaGetLastError();
}

cudaError_t launch_gather(int prec, int bloch, const GatherParams &p, cudaStream_t s) {
  if (p.n_atoms <= 0) return cudaSuccess;
  dim3 grid(p.n_atoms * p.n_chunks, p.n_kb);
  const unsigned fgrid = (unsigned)(((long)p.n_atoms * p.n_kb + 7) / 8);
  const dim3 ngrid((unsigned)(((long)p.n_sp * OVC + NL_THREADS - 1) / NL_THREADS), nl_kb_rows(p.n_kb));
  if (prec == P_C64) {
    if (bloch) gather_kernel<P_C64, 1><<<grid, GATHER_THREADS, 0, s>>>(p);
    else gather_kernel<P_C64, 0><<<grid, GATHER_THREADS, 0, s>>>(p);
    gather_finish_kernel<P_C64><<<fgrid, 128, 0, s>>>(p);
    if (p.n_sp > 0 && bloch) nl_kernel<P_C64, 1><<<ngrid, NL_THREADS, 0, s>>>(p);
    else if (p.n_sp > 0) nl_kernel<P_C64, 0><<<ngrid, NL_THREADS, 0, s>>>(p);
  } else {
    if (bloch) gather_kernel<P_C128, 1><<<grid, GATHER_THREADS, 0, s>>>(p);
    else gather_kernel<P_C128, 0><<<grid, GATHER_THREADS, 0, s>>>(p);
    gather_finish_kernel<P_C128><<<fgrid, 128, 0, s>>>(p);
    if (p.n_sp > 0 && bloch) nl_kernel<P_C128, 1><<<ngrid, NL_THREADS, 0, s>>>(p);
    else if (p.n_sp > 0) nl_kernel<P_C128, 0><<<ngrid, NL_THREADS, 0, s>>>(p);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Density contribution of each (k, batch) block (n(r) = sum_k w_k sum_i f_i |phi_ik(r)|^2,
// with closed-shell f_i = 2):
//   complex128 systems: dens_part[kb][r] = w_k f sum_j |psi|^2 (double);
//   complex64 systems (state hi + lo): the 8-byte slot holds sum_j |psi|^2 unweighted, as a
//   double-float pair (float hi, float lo); the LDA kernel weights and adds the blocks as
//   double-float, so neither the kernels that produce it nor the LDA run FP64 per point.
// ---------------------------------------------------------------------------------
__global__ void density_c128_kernel(long N, int n_kb, int n_batches, const double2 *psi, const double *wocc,
                                    double *dens_part) {
  const long total = (long)n_kb * N;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const double2 *b = psi + i * OVC;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < OVC; j++) {
      const double2 x = b[j];
      s += x.x * x.x + x.y * x.y;
    }
    dens_part[i] = wocc[(int)(i / N) / n_batches] * s;
  }
}

// |psi|^2 of one complex64 value held as the double-float pair (h, l), as s + e with FP32
// operations only (h^2 exactly by FMA, + 2 h l), then summed over the 2 * OVC lanes of a
// (point, batch) block with an xor tree (1, 2, 4) of double-float additions.  Lane 0 of the
// block returns the block's sum.  pack_in_kernel and density_c64_kernel both use it, so a
// state's density partials do not depend on which of them wrote them.
__device__ __forceinline__ void block_sq_c64(float hx, float hy, float lx, float ly, float &sh, float &sl) {
  float e;
  sh = Combine<P_C64>::sq_parts(pk2(hx, hy), pk2(lx, ly), e);
  sl = e;
#pragma unroll
  for (int o = 1; o < 2 * OVC; o <<= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
    float t;
    sh = two_sum(sh, oh, t);
    sl = sl + ol + t;
  }
}

// Thread = one complex value of one (k-batch, point): 8 adjacent lanes per block.
__global__ void density_c64_kernel(long N, int n_kb, int n_batches, const float2 *hi, const float2 *lo,
                                   const double *wocc, double *dens_part) {
  const long total = (long)n_kb * N * 2 * OVC;
  (void)wocc;
  (void)n_batches;
  const long stride = (long)gridDim.x * blockDim.x;  // a multiple of 32, so lanes keep their value index
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i - threadIdx.x % 32 < total; i += stride) {
    const bool live = i < total;
    const float2 a = live ? hi[i] : make_float2(0.f, 0.f), b = live ? lo[i] : make_float2(0.f, 0.f);
    float sh, sl;
    block_sq_c64(a.x, a.y, b.x, b.y, sh, sl);
    if (live && i % (2 * OVC) == 0) reinterpret_cast<float2 *>(dens_part)[i / (2 * OVC)] = make_float2(sh, sl);
  }
}

cudaError_t launch_density(int prec, long N, int n_kb, int n_batches, const void *psi, const void *psi_lo,
                           const double *wocc, double *dens_part, cudaStream_t s) {
  const long total = (long)n_kb * N * (prec == P_C64 ? 2 * OVC : 1);
  int grid = (int)((total + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  if (prec == P_C64)
    density_c64_kernel<<<grid, 256, 0, s>>>(N, n_kb, n_batches, (const float2 *)psi, (const float2 *)psi_lo, wocc,
                                            dens_part);
  else
    density_c128_kernel<<<grid, 256, 0, s>>>(N, n_kb, n_batches, (const double2 *)psi, wocc, dens_part);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// n(r) = sum_kb dens_part (fixed order); LDA exchange v_x = -(3n/pi)^(1/3),
// e_x = 3/4 v_x (Sec. "Local domains": E_xc = int n e_xc(n)); adiabatic: from the
// current density only (Sec. "New propagators").  V_eff = V_loc + v_x + E.r (length
// gauge, finite box) + |A|^2/2 (velocity gauge).  Per-block partial sums for the
// observables: [int n, int n e_x, int n v_x, int x n, int y n, int z n] (before h^3).
// ---------------------------------------------------------------------------------
constexpr int LDA_THREADS = 256;

int lda_blocks(long N) {
  long g = (N + LDA_THREADS - 1) / LDA_THREADS;
  return (int)(g < 152 * 4 ? g : 152 * 4);
}

// complex128 systems: everything in FP64.
// complex64 systems (V_eff is FP32 there): the density is summed over the k-point batches
// as double-float (two FP32 numbers, ~44-bit significand) and weighted by w_k f split into
// two floats; v_x and V_eff in FP32; the per-point terms of the observables in FP32
// accumulated as double-float per thread; the sums across threads in FP64.  This keeps
// GB300's slow FP64 pipe out of the per-point loop.
constexpr int LDA_MAXK = 256;  // k-points whose split weights are staged in shared memory

template <typename R>
__device__ __forceinline__ void lda_body(long N, int nx, int ny, int nz, double h, int bloch, int n_kb,
                                         int n_batches, const double *wocc, const double *dens_part,
                                         const double *vloc, int xc, double Ex, double Ey, double Ez,
                                         double half_A2, PointAux *aux, double *lda_part, int blk, int nblk,
                                         const double *n_in = nullptr, const double *vh = nullptr,
                                         bool sums = true) {
  constexpr bool F32 = sizeof(R) == 4;
  const int n_k = n_kb / n_batches;
  __shared__ float2 s_w[LDA_MAXK];  // complex64: w_k f = hi + lo
  if constexpr (F32) {
    for (int k = threadIdx.x; k < n_k && k < LDA_MAXK; k += blockDim.x) {
      const float hi = (float)wocc[k];
      s_w[k] = make_float2(hi, (float)(wocc[k] - (double)hi));
    }
    __syncthreads();
  }
  double acc[6] = {0, 0, 0, 0, 0, 0};
  float fh[6] = {0, 0, 0, 0, 0, 0}, fl[6] = {0, 0, 0, 0, 0, 0};
  const double cx = bloch ? 0.0 : 0.5 * (nx - 1), cy = bloch ? 0.0 : 0.5 * (ny - 1),
               cz = bloch ? 0.0 : 0.5 * (nz - 1);
  const float hf = (float)h, cxf = (float)cx, cyf = (float)cy, czf = (float)cz;
  const float Exf = (float)Ex, Eyf = (float)Ey, Ezf = (float)Ez, hA2f = (float)half_A2;
  for (long p = blk * (long)blockDim.x + threadIdx.x; p < N; p += (long)nblk * blockDim.x) {
    double n = 0.0;
    float nh = 0.f, nl = 0.f;  // complex64: n = nh + nl
    if (n_in) {
      // the density summed over every rank's states (state-parallel propagation)
      n = n_in[p];
      nh = (float)n;
      nl = (float)(n - (double)nh);
    } else if constexpr (F32) {
      const float2 *d2 = reinterpret_cast<const float2 *>(dens_part);
      for (int k = 0; k < n_k; k++) {
        float sh = 0.f, sl = 0.f;  // sum over the k-point's batches of sum |psi|^2
        for (int b = 0; b < n_batches; b++) {
          const float2 d = d2[(long)(k * n_batches + b) * N + p];
          df_add_df(sh, sl, d.x, d.y);
        }
        float2 w;
        if (k < LDA_MAXK) {
          w = s_w[k];
        } else {
          const float hi = (float)wocc[k];
          w = make_float2(hi, (float)(wocc[k] - (double)hi));
        }
        // (sh + sl)(w.x + w.y): the leading product exactly (FMA residual), the cross terms rounded
        const float ph = sh * w.x;
        const float pl = fmaf(sh, w.x, -ph) + (sh * w.y + sl * w.x);
        df_add_df(nh, nl, ph, pl);
      }
    } else {
      for (int kb = 0; kb < n_kb; kb++) n += dens_part[(long)kb * N + p];
    }
    // (32-bit index arithmetic: a 64-bit division per coordinate cost more than the point's
    // arithmetic; the grids here have far fewer than 2^32 points)
    const unsigned up = (unsigned)p, unx = (unsigned)nx, uny = (unsigned)ny;
    const int ix = (int)(up % unx), iy = (int)((up / unx) % uny), iz = (int)(up / (unx * uny));
    if constexpr (F32) {
      const float nf = nh;
      const float x = (ix - cxf) * hf, y = (iy - cyf) * hf, z = (iz - czf) * hf;
      const float vx = xc ? -cbrtf(3.0f * nf * 0.318309886f) : 0.0f;
      const float vhf = vh ? (float)vh[p] : 0.0f;
      float v = (float)vloc[p] + vx + vhf + hA2f;
      if (!bloch) v += Exf * x + Eyf * y + Ezf * z;
      *reinterpret_cast<float *>(&aux[p].veff) = v;
      if (sums) {
        // (with the Hartree potential the record subtracts int n (v_x + v_H) and adds E_H =
        // 1/2 int n v_H: the third sum is int n (v_x + v_H / 2))
        const float t[6] = {nf, nf * 0.75f * vx, nf * (vx + 0.5f * vhf), x * nf, y * nf, z * nf};
#pragma unroll
        for (int c = 0; c < 6; c++) df_acc(fh[c], fl[c], t[c]);
        fl[0] += nl;  // the electron count keeps the double-float density in full
      }
    } else {
      const double x = (ix - cx) * h, y = (iy - cy) * h, z = (iz - cz) * h;
      double vx = 0.0;
      if (xc) vx = -cbrt(3.0 * n * 0.31830988618379067154);  // 1/pi
      const double vhd = vh ? vh[p] : 0.0;
      double v = vloc[p] + vx + vhd + half_A2;
      if (!bloch) v += Ex * x + Ey * y + Ez * z;
      *reinterpret_cast<double *>(&aux[p].veff) = v;
      if (sums) {
        acc[0] += n;
        acc[1] += n * 0.75 * vx;
        acc[2] += n * (vx + 0.5 * vhd);
        acc[3] += x * n;
        acc[4] += y * n;
        acc[5] += z * n;
      }
    }
  }
  if (!sums) return;  // (uniform over the grid: V_eff only, no record follows)
  if constexpr (F32) {
#pragma unroll
    for (int c = 0; c < 6; c++) acc[c] = (double)fh[c] + (double)fl[c];
  }
  __shared__ double red[LDA_THREADS / 32][6];
  for (int i = 0; i < 6; i++) {
    double x = acc[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][i] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double x = 0.0;
    for (int w = 0; w < LDA_THREADS / 32; w++) x += red[w][threadIdx.x];
    lda_part[blk * 6 + threadIdx.x] = x;
  }
}

template <typename R>
__global__ void __launch_bounds__(LDA_THREADS)
lda_kernel(long N, int nx, int ny, int nz, double h, int bloch, int n_kb, int n_batches, const double *wocc,
           const double *dens_part, const double *vloc, int xc, double Ex, double Ey, double Ez, double half_A2,
           PointAux *aux, double *lda_part, const double *n_in, const double *vh, int sums) {
  lda_body<R>(N, nx, ny, nz, h, bloch, n_kb, n_batches, wocc, dens_part, vloc, xc, Ex, Ey, Ez, half_A2, aux,
              lda_part, blockIdx.x, gridDim.x, n_in, vh, sums != 0);
}

// The density of this system's states at every point, n(r) = sum_k w_k f sum_i |psi|^2, as
// FP64 (the LDA kernel's sum: in order over the batches, complex64 partials as double-float),
// for a state-parallel run to sum over ranks before the LDA kernel reads it back.
template <typename R>
__global__ void __launch_bounds__(LDA_THREADS)
density_sum_kernel(long N, int n_kb, int n_batches, const double *wocc, const double *dens_part, double *n_out) {
  constexpr bool F32 = sizeof(R) == 4;
  const int n_k = n_kb / n_batches;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < N; p += (long)gridDim.x * blockDim.x) {
    if constexpr (F32) {
      const float2 *d2 = reinterpret_cast<const float2 *>(dens_part);
      float nh = 0.f, nl = 0.f;
      for (int k = 0; k < n_k; k++) {
        float sh = 0.f, sl = 0.f;
        for (int b = 0; b < n_batches; b++) {
          const float2 d = d2[(long)(k * n_batches + b) * N + p];
          df_add_df(sh, sl, d.x, d.y);
        }
        const float wh = (float)wocc[k], wl = (float)(wocc[k] - (double)wh);
        const float ph = sh * wh;
        const float pl = fmaf(sh, wh, -ph) + (sh * wl + sl * wh);
        df_add_df(nh, nl, ph, pl);
      }
      n_out[p] = (double)nh + (double)nl;
    } else {
      double n = 0.0;
      for (int kb = 0; kb < n_kb; kb++) n += dens_part[(long)kb * N + p];
      n_out[p] = n;
    }
  }
}

// Runge-Kutta stage updates: element-wise over the packed state, one double2 per thread
// and grid-stride loop (HBM-bound: 48 or 64 bytes per value).
__global__ void rk4_stage_kernel(long n, const double2 *psi, const double2 *k, double a, double2 *stage, double2 *acc,
                                 double b, int init) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double2 kv = k[i], pv = psi[i];
    stage[i] = make_double2(pv.x + a * kv.x, pv.y + a * kv.y);
    const double2 av = init ? make_double2(0.0, 0.0) : acc[i];
    acc[i] = make_double2(av.x + b * kv.x, av.y + b * kv.y);
  }
}

__global__ void rk4_finish_kernel(long n, double2 *psi, const double2 *acc, const double2 *k, double b) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double2 kv = k[i], av = acc[i], pv = psi[i];
    psi[i] = make_double2(pv.x + (av.x + b * kv.x), pv.y + (av.y + b * kv.y));
  }
}

static int elementwise_blocks(long n) {
  const long want = (n + 255) / 256;
  return (int)(want < 1 ? 1 : (want > 152L * 16 ? 152L * 16 : want));
}

cudaError_t launch_rk4_stage(long n, const void *psi, const void *k, double a, void *stage, void *acc, double b,
                             int init, cudaStream_t s) {
  rk4_stage_kernel<<<elementwise_blocks(n), 256, 0, s>>>(n, (const double2 *)psi, (const double2 *)k, a,
                                                         (double2 *)stage, (double2 *)acc, b, init);
  return cudaGetLastError();
}

cudaError_t launch_rk4_finish(long n, void *psi, const void *acc, const void *k, double b, cudaStream_t s) {
  rk4_finish_kernel<<<elementwise_blocks(n), 256, 0, s>>>(n, (double2 *)psi, (const double2 *)acc,
                                                          (const double2 *)k, b);
  return cudaGetLastError();
}

cudaError_t launch_density_sum(int prec, long N, int n_kb, int n_batches, const double *wocc,
                               const double *dens_part, double *n_out, cudaStream_t s) {
  if (prec == P_C64)
    density_sum_kernel<float><<<lda_blocks(N), LDA_THREADS, 0, s>>>(N, n_kb, n_batches, wocc, dens_part, n_out);
  else
    density_sum_kernel<double><<<lda_blocks(N), LDA_THREADS, 0, s>>>(N, n_kb, n_batches, wocc, dens_part, n_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// CFM4 (Sec. "New propagators for real-time TDDFT"): the effective potential of one of the
// two exponentials, V_eff = V_loc + sum_j w_j v_x,j + E.r, where v_x,j is the exchange
// potential at the start of the j-th latest sub-step (the history) and the w_j extrapolate
// it to the Gauss points (the host forms them).  push: first store v_x of the current
// density (dens_part, summed as the LDA kernel does) into hist.v[0], the slot the host has
// rotated to the front.  The history is FP64; complex64 systems compute v_x in FP32 as their
// LDA kernel does and round V_eff to FP32.
// ---------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(LDA_THREADS)
cfm_veff_kernel(long N, int nx, int ny, int nz, double h, int bloch, int n_kb, int n_batches, const double *wocc,
                const double *dens_part, const double *vloc, int xc, int push, CfmHist hist, double Ex, double Ey,
                double Ez, PointAux *aux, const double *vh, const double *n_in) {
  constexpr bool F32 = sizeof(R) == 4;
  const int n_k = n_kb / n_batches;
  __shared__ float2 s_w[LDA_MAXK];
  if constexpr (F32) {
    for (int k = threadIdx.x; k < n_k && k < LDA_MAXK; k += blockDim.x) {
      const float hi = (float)wocc[k];
      s_w[k] = make_float2(hi, (float)(wocc[k] - (double)hi));
    }
    __syncthreads();
  }
  const double cx = bloch ? 0.0 : 0.5 * (nx - 1), cy = bloch ? 0.0 : 0.5 * (ny - 1), cz = bloch ? 0.0 : 0.5 * (nz - 1);
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < N; p += (long)gridDim.x * blockDim.x) {
    if (push && xc) {
      double vx;
      if (n_in) {
        // the density summed in FP64 (every rank's states, or the Hartree source)
        if constexpr (F32) {
          vx = (double)(-cbrtf(3.0f * (float)n_in[p] * 0.318309886f));
        } else {
          vx = -cbrt(3.0 * n_in[p] * 0.31830988618379067154);
        }
      } else if constexpr (F32) {
        const float2 *d2 = reinterpret_cast<const float2 *>(dens_part);
        float nh = 0.f, nl = 0.f;
        for (int k = 0; k < n_k; k++) {
          float sh = 0.f, sl = 0.f;
          for (int b = 0; b < n_batches; b++) {
            const float2 d = d2[(long)(k * n_batches + b) * N + p];
            df_add_df(sh, sl, d.x, d.y);
          }
          float2 w;
          if (k < LDA_MAXK) {
            w = s_w[k];
          } else {
            const float hi = (float)wocc[k];
            w = make_float2(hi, (float)(wocc[k] - (double)hi));
          }
          const float ph = sh * w.x;
          const float pl = fmaf(sh, w.x, -ph) + (sh * w.y + sl * w.x);
          df_add_df(nh, nl, ph, pl);
        }
        vx = (double)(-cbrtf(3.0f * nh * 0.318309886f));
      } else {
        double n = 0.0;
        for (int kb = 0; kb < n_kb; kb++) n += dens_part[(long)kb * N + p];
        vx = -cbrt(3.0 * n * 0.31830988618379067154);
      }
      if (vh) vx += vh[p];  // the Hartree potential of the same density
      hist.v[0][p] = vx;
    }
    // (32-bit index arithmetic: a 64-bit division per coordinate cost more than the point's
    // arithmetic; the grids here have far fewer than 2^32 points)
    const unsigned up = (unsigned)p, unx = (unsigned)nx, uny = (unsigned)ny;
    const int ix = (int)(up % unx), iy = (int)((up / unx) % uny), iz = (int)(up / (unx * uny));
    double v = vloc[p];
    for (int j = 0; j < hist.nh; j++) v += hist.w[j] * hist.v[j][p];
    v += Ex * ((ix - cx) * h) + Ey * ((iy - cy) * h) + Ez * ((iz - cz) * h);
    *reinterpret_cast<R *>(&aux[p].veff) = (R)v;
  }
}

cudaError_t launch_cfm_veff(int prec, int bloch, long N, int nx, int ny, int nz, double h, int n_kb, int n_batches,
                            const double *wocc, const double *dens_part, const double *vloc, int xc, int push,
                            const CfmHist &hist, const double E[3], PointAux *aux, cudaStream_t s,
                            const double *vh, const double *n_in) {
  const int blocks = lda_blocks(N);
  if (prec == P_C64)
    cfm_veff_kernel<float><<<blocks, LDA_THREADS, 0, s>>>(N, nx, ny, nz, h, bloch, n_kb, n_batches, wocc, dens_part,
                                                          vloc, xc, push, hist, E[0], E[1], E[2], aux, vh, n_in);
  else
    cfm_veff_kernel<double><<<blocks, LDA_THREADS, 0, s>>>(N, nx, ny, nz, h, bloch, n_kb, n_batches, wocc, dens_part,
                                                           vloc, xc, push, hist, E[0], E[1], E[2], aux, vh, n_in);
  return cudaGetLastError();
}

// Laser field of a batched system at time t (finite boxes: length gauge or none).
__device__ __forceinline__ double batch_field(const BatchAux &a, double t) {
  if (a.gauge != 1) return 0.0;
  double env = 1.0;
  if (a.envelope == 1) {
    if (t < 0.0 || t > a.t_total) return 0.0;
    const double x = sin(3.14159265358979323846 * t / a.t_total);
    env = x * x;
  }
  return a.amp * env * sin(a.omega * t);
}

// Batched LDA: the systems' CTA ranges are concatenated; the field is evaluated at each
// system's current sub-step midpoint from its device clock.
template <typename R>
__global__ void __launch_bounds__(LDA_THREADS)
lda_batch_kernel(const BatchAux *aux, const BatchClock *clk, const long *begin, int n_sys) {
  __shared__ double f;
  // the CTA's system: a binary search over the systems' CTA ranges (a table lookup, as the
  // projector kernels use, measured 1.3% slower on the batched step here)
  int lo = 0, hi = n_sys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (begin[mid] <= (long)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const int s = lo;
  const BatchAux &a = aux[s];
  if (threadIdx.x == 0) {
    const BatchClock c = clk[s];
    f = batch_field(a, c.t + (c.j + 0.5) * c.dt / c.substeps);
  }
  __syncthreads();
  const double E = f;
  lda_body<R>(a.N, a.nx, a.ny, a.nz, a.h, 0, a.n_kb, a.n_batches, a.wocc, a.dens_part, a.vloc, a.xc,
              E * a.pol[0], E * a.pol[1], E * a.pol[2], 0.0, a.aux, a.lda_part, (int)(blockIdx.x - begin[s]),
              a.n_lda);
}

cudaError_t launch_lda_batch(int prec, const BatchAux *aux, const BatchClock *clk, const long *begin, int n_sys,
                             long total, cudaStream_t s) {
  if (prec == P_C64) lda_batch_kernel<float><<<(unsigned)total, LDA_THREADS, 0, s>>>(aux, clk, begin, n_sys);
  else lda_batch_kernel<double><<<(unsigned)total, LDA_THREADS, 0, s>>>(aux, clk, begin, n_sys);
  return cudaGetLastError();
}

cudaError_t launch_lda(int prec, int bloch, long N, int nx, int ny, int nz, double h, int n_kb, int n_batches,
                       const double *wocc, const double *dens_part, const double *vloc, int xc, const double E[3],
                       double half_A2, PointAux *aux, double *lda_part, int n_blocks, cudaStream_t s,
                       const double *n_in, const double *vh, int sums) {
  if (prec == P_C64)
    lda_kernel<float><<<n_blocks, LDA_THREADS, 0, s>>>(N, nx, ny, nz, h, bloch, n_kb, n_batches, wocc, dens_part,
                                                       vloc, xc, E[0], E[1], E[2], half_A2, aux, lda_part, n_in, vh,
                                                       sums);
  else
    lda_kernel<double><<<n_blocks, LDA_THREADS, 0, s>>>(N, nx, ny, nz, h, bloch, n_kb, n_batches, wocc, dens_part,
                                                        vloc, xc, E[0], E[1], E[2], half_A2, aux, lda_part, n_in, vh,
                                                        sums);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Observable record [t, norm, E, E_x, o_x, o_y, o_z, field]:
//   norm = int n / f;  E = sum_k w_k f <phi|H|phi> - int n v_x + E_x;
//   o = dipole int r n (finite box, Sec. "Local domains") or the current
//       J = -(1/Omega) (sum w f <phi|-i grad|phi> + A int n) (Sec. "Conductivities").
// One CTA; partials are summed in index order.
// ---------------------------------------------------------------------------------
// The record from the summed partials O (energy, current x, y, z) and Lq (LDA sums).
__device__ __forceinline__ void write_record(const double O[4], const double Lq[6], double *rec, double t_state,
                                             double h3, double occ, int bloch, double omega_cell, double Ax,
                                             double Ay, double Az, double field_val) {
  const double nint = Lq[0] * h3, ex = Lq[1] * h3, nvx = Lq[2] * h3;
  rec[0] = t_state;
  rec[1] = nint / occ;
  rec[2] = O[0] * h3 - nvx + ex;
  rec[3] = ex;
  if (!bloch) {
    rec[4] = Lq[3] * h3;
    rec[5] = Lq[4] * h3;
    rec[6] = Lq[5] * h3;
  } else {
    rec[4] = -(O[1] * h3 + Ax * nint) / omega_cell;
    rec[5] = -(O[2] * h3 + Ay * nint) / omega_cell;
    rec[6] = -(O[3] * h3 + Az * nint) / omega_cell;
  }
  rec[7] = field_val;
}

// Sum of the 10 per-thread values v over the CTA (FIN_THREADS threads): a fixed xor tree
// within each warp, then the warps in order; thread c < 10 returns component c.
constexpr int FIN_THREADS = 128;
__device__ __forceinline__ double block_sum10(double v[10], int t) {
  __shared__ double red[FIN_THREADS / 32][10];
#pragma unroll
  for (int c = 0; c < 10; c++) {
    double x = v[c];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((t & 31) == 0) red[t >> 5][c] = x;
  }
  __syncthreads();
  double x = 0.0;
  if (t < 10)
    for (int w = 0; w < FIN_THREADS / 32; w++) x += red[w][t];
  return x;
}

// Partials of records [i0, i1) and LDA blocks [l0, l1), summed by one CTA.
__device__ __forceinline__ double partial_sums(const double *obs_part, long i0, long i1, const double *lda_part,
                                               long l0, long l1, int t) {
  double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (long i = i0 + t; i < i1; i += FIN_THREADS)
    for (int c = 0; c < 4; c++) v[c] += obs_part[i * 4 + c];
  for (long i = l0 + t; i < l1; i += FIN_THREADS)
    for (int c = 0; c < 6; c++) v[4 + c] += lda_part[i * 6 + c];
  return block_sum10(v, t);
}

// One CTA of FIN_THREADS threads (batched systems: one CTA per system).
__device__ __forceinline__ void finalize_body(const double *obs_part, long n_items, const double *lda_part,
                                              int n_lda, double *rec, double t_state, double h3, double occ,
                                              int bloch, double omega_cell, double Ax, double Ay, double Az,
                                              double field_val) {
  __shared__ double tot[10];
  const int t = threadIdx.x;
  const double x = partial_sums(obs_part, 0, n_items, lda_part, 0, n_lda, t);
  if (t < 10) tot[t] = x;
  __syncthreads();
  if (t == 0) write_record(tot, tot + 4, rec, t_state, h3, occ, bloch, omega_cell, Ax, Ay, Az, field_val);
}

// Two stages for one system: CTA b of stage 1 sums the b-th contiguous share of the
// partials; stage 2 adds the CTAs' sums in order.  The shares depend only on the counts,
// so the record is the same on every run.
__global__ void __launch_bounds__(FIN_THREADS)
finalize_stage1_kernel(const double *obs_part, long n_items, const double *lda_part, int n_lda, double *fin_part) {
  const long b = blockIdx.x, nb = gridDim.x;
  const double x = partial_sums(obs_part, n_items * b / nb, n_items * (b + 1) / nb, lda_part, n_lda * b / nb,
                                n_lda * (b + 1) / nb, threadIdx.x);
  if (threadIdx.x < 10) fin_part[b * 10 + threadIdx.x] = x;
}

__global__ void __launch_bounds__(32)
finalize_stage2_kernel(const double *fin_part, int nb, double *rec, double t_state, double h3, double occ,
                       int bloch, double omega_cell, double Ax, double Ay, double Az, double field_val) {
  __shared__ double tot[10];
  const int t = threadIdx.x;
  if (t < 10) {
    double x = 0.0;
    for (int b = 0; b < nb; b++) x += fin_part[b * 10 + t];
    tot[t] = x;
  }
  __syncwarp();
  if (t == 0) write_record(tot, tot + 4, rec, t_state, h3, occ, bloch, omega_cell, Ax, Ay, Az, field_val);
}

// Batched observable records: one CTA per system, at the first sub-step of each step.
__global__ void finalize_batch_kernel(const BatchAux *aux, const BatchClock *clk, int n_sys) {
  const int s = blockIdx.x;
  const BatchClock c = clk[s];
  if (c.j != 0) return;
  const BatchAux &a = aux[s];
  const double h3 = a.h * a.h * a.h;
  const double fv = batch_field(a, c.t + 0.5 * c.dt / c.substeps);
  const double fpol = fv * (a.pol[0] * a.pol[0] + a.pol[1] * a.pol[1] + a.pol[2] * a.pol[2]);
  finalize_body(a.obs_part, a.n_items, a.lda_part, a.n_lda, a.ring + (c.step % a.ring_len) * 8, c.t, h3, a.occ, 0,
                (double)a.N * h3, 0.0, 0.0, 0.0, fpol);
}

// Advance every batched system's clock by one sub-step.
__global__ void clock_batch_kernel(BatchClock *clk, int n_sys) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_sys) return;
  BatchClock c = clk[s];
  if (++c.j == c.substeps) {
    c.j = 0;
    c.step++;
    c.t += c.dt;
  }
  clk[s] = c;
}

cudaError_t launch_batch_tail(const BatchAux *aux, BatchClock *clk, int n_sys, int which, cudaStream_t s) {
  if (which == 0) finalize_batch_kernel<<<n_sys, FIN_THREADS, 0, s>>>(aux, clk, n_sys);
  else clock_batch_kernel<<<(n_sys + 127) / 128, 128, 0, s>>>(clk, n_sys);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(32) finalize_sums_kernel(const double *fin_part, int nb, double *sums) {
  const int t = threadIdx.x;
  if (t < 10) {
    double x = 0.0;
    for (int b = 0; b < nb; b++) x += fin_part[b * 10 + t];
    sums[t] = x;
  }
}

__global__ void __launch_bounds__(32)
record_from_sums_kernel(const double *sums, double *rec, double t_state, double h3, double occ, int bloch,
                        double omega_cell, double Ax, double Ay, double Az, double field_val) {
  if (threadIdx.x == 0) write_record(sums, sums + 4, rec, t_state, h3, occ, bloch, omega_cell, Ax, Ay, Az, field_val);
}

static int finalize_blocks(long n_items, int n_lda) {
  const long want = (n_items + n_lda + 4L * FIN_THREADS - 1) / (4L * FIN_THREADS);
  return (int)(want < 1 ? 1 : (want > FIN_BLOCKS ? FIN_BLOCKS : want));
}

cudaError_t launch_finalize_sums(const double *obs_part, long n_items, const double *lda_part, int n_lda,
                                 double *fin_part, double *sums, cudaStream_t s) {
  const int nb = finalize_blocks(n_items, n_lda);
  finalize_stage1_kernel<<<nb, FIN_THREADS, 0, s>>>(obs_part, n_items, lda_part, n_lda, fin_part);
  finalize_sums_kernel<<<1, 32, 0, s>>>(fin_part, nb, sums);
  return cudaGetLastError();
}

cudaError_t launch_record_from_sums(const double *sums, double *record, double t_state, double h3, double occ,
                                    int bloch, double omega_cell, const double A[3], double field_val,
                                    cudaStream_t s) {
  record_from_sums_kernel<<<1, 32, 0, s>>>(sums, record, t_state, h3, occ, bloch, omega_cell, A[0], A[1], A[2],
                                           field_val);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double *obs_part, long n_items, const double *lda_part, int n_lda,
                            double *record, double t_state, double h3, double occ, int bloch,
                            double omega_cell, const double A[3], double field_val, double *fin_part,
                            cudaStream_t s) {
  const int nb = finalize_blocks(n_items, n_lda);
  finalize_stage1_kernel<<<nb, FIN_THREADS, 0, s>>>(obs_part, n_items, lda_part, n_lda, fin_part);
  finalize_stage2_kernel<<<1, 32, 0, s>>>(fin_part, nb, record, t_state, h3, occ, bloch, omega_cell, A[0], A[1],
                                          A[2], field_val);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Layout conversion between the host layout [k][r][n_orb] (complex128) and the packed
// state [k][batch][r][BS] (zero-padded orbitals).  complex64 systems split each value
// into hi = fl32(x) and lo = fl32(x - hi) (the double-float state); unpacking returns
// hi + lo in FP64.
// ---------------------------------------------------------------------------------
__global__ void pack_kernel(int to_internal, int c64, long N, int n_k, int n_orb, int n_batches, int BS,
                            void *internal, void *internal_lo, double2 *plain) {
  const long total = (long)n_k * n_batches * N * BS;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int j = (int)(i % BS);
    long r = i / BS;
    const long pt = r % N;
    r /= N;
    const int b = (int)(r % n_batches);
    const int k = (int)(r / n_batches);
    const int o = b * BS + j;
    const long pidx = ((long)k * N + pt) * n_orb + o;
    if (to_internal) {
      const double2 x = o < n_orb ? plain[pidx] : make_double2(0.0, 0.0);
      if (c64) {
        const float hx = (float)x.x, hy = (float)x.y;
        reinterpret_cast<float2 *>(internal)[i] = make_float2(hx, hy);
        reinterpret_cast<float2 *>(internal_lo)[i] = make_float2((float)(x.x - (double)hx), (float)(x.y - (double)hy));
      } else {
        reinterpret_cast<double2 *>(internal)[i] = x;
      }
    } else if (o < n_orb) {
      if (c64) {
        const float2 h = reinterpret_cast<const float2 *>(internal)[i];
        const float2 l = reinterpret_cast<const float2 *>(internal_lo)[i];
        plain[pidx] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
      } else {
        plain[pidx] = reinterpret_cast<const double2 *>(internal)[i];
      }
    }
  }
}

// Host layout -> internal layout for the points [pt0, pt0 + npts) of k-point k, with the
// density partials of those points (the values launch_density would write), so a state
// set from the host needs no separate density pass.  Thread = one orbital value of one
// (batch, point): the BS threads of a point are adjacent lanes, so reads and writes are
// contiguous, and they add their |psi|^2 with shuffles in the density kernel's order.
__global__ void pack_in_kernel(int c64, long N, int k, long pt0, long npts, int n_orb, int n_batches, int BS,
                               const double2 *plain, void *internal, void *internal_lo, const double *wocc,
                               double *dens_part) {
  const long total = (long)n_batches * npts * BS;
  const long stride = (long)gridDim.x * blockDim.x;  // a multiple of 32, so lanes keep their j
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i - threadIdx.x % 32 < total; i += stride) {
    const bool live = i < total;
    const int j = (int)(i % BS);
    const long q = i / BS;
    const long pt = pt0 + q % npts;
    const int b = (int)(q / npts);
    const long kb = (long)k * n_batches + b;
    const int o = b * BS + j;
    const double2 x = live && o < n_orb ? plain[((long)k * N + pt) * n_orb + o] : make_double2(0.0, 0.0);
    const long dst = (kb * N + pt) * BS + j;
    if (c64) {
      // the value as a double-float pair, and the block's density partial with FP32
      // operations only (GB300's FP64 pipe would otherwise bound this kernel)
      const float hx = (float)x.x, hy = (float)x.y;
      const float lx = (float)(x.x - (double)hx), ly = (float)(x.y - (double)hy);
      if (live) {
        reinterpret_cast<float2 *>(internal)[dst] = make_float2(hx, hy);
        reinterpret_cast<float2 *>(internal_lo)[dst] = make_float2(lx, ly);
      }
      float sh, sl;
      block_sq_c64(hx, hy, lx, ly, sh, sl);
      if (live && j == 0) reinterpret_cast<float2 *>(dens_part)[kb * N + pt] = make_float2(sh, sl);
    } else {
      if (live) reinterpret_cast<double2 *>(internal)[dst] = x;
      const double s = x.x * x.x + x.y * x.y;
      // lane j of the point gathers the sum over the point's values in index order
      double acc = 0.0;
      for (int t = 0; t < BS; t++) acc += __shfl_sync(0xffffffffu, s, (threadIdx.x & 31 & ~(BS - 1)) + t);
      if (live && j == 0) dens_part[kb * N + pt] = wocc[k] * acc;
    }
  }
}

cudaError_t launch_pack_in(int prec, long N, int k, long pt0, long npts, int n_orb, int n_batches,
                           const double *plain, void *internal, void *internal_lo, const double *wocc,
                           double *dens_part, cudaStream_t s) {
  const int BS = prec == P_C64 ? 2 * OVC : OVC;
  const long total = (long)n_batches * npts * BS;
  long g = (total + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (g <= 0) return cudaSuccess;
  pack_in_kernel<<<(int)g, 256, 0, s>>>(prec == P_C64, N, k, pt0, npts, n_orb, n_batches, BS,
                                        reinterpret_cast<const double2 *>(plain), internal, internal_lo, wocc,
                                        dens_part);
  return cudaGetLastError();
}

cudaError_t launch_pack(int prec, int to_internal, long N, int n_k, int n_orb, int n_batches, void *internal,
                        void *internal_lo, double *plain, cudaStream_t s) {
  const int BS = prec == P_C64 ? 2 * OVC : OVC;
  const long total = (long)n_k * n_batches * N * BS;
  long g = (total + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  pack_kernel<<<(int)g, 256, 0, s>>>(to_internal, prec == P_C64, N, n_k, n_orb, n_batches, BS, internal,
                                     internal_lo, (double2 *)plain);
  return cudaGetLastError();
}

}  // namespace tdks
