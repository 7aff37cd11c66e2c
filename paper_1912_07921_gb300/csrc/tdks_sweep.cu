// Fused Taylor-term sweep: t_k = (cr + i ci) * H t_(k-1) on the packed-batch layout.
//
// H = -1/2 Lap_h + V_eff(r) [+ velocity-gauge terms] + V_NL, with the star stencil of
// order 2M (Sec. "Maxwell ... coupling" and Sec. "Periodic systems": high-order finite
// differences on the real-space grid), V_eff = V_loc + v_x[n] + E(t).r (+ |A|^2/2)
// prepared once per sub-step, and V_NL the Kleinman-Bylander scatter of the projections
// D_aj h^3 <beta_aj|t_(k-1)> gathered just before this sweep.  The exponential is the
// 4th-order Taylor series t_0 = psi, t_k = (-i dt / k) H t_(k-1), psi' = sum t_k
// (the TDKS step of Sec. "New propagators"; H frozen over the step).
//
// Data movement (GB300: HBM-bound for complex64):
//   * one CTA owns a TX x TY tile of one (k, batch) block and marches a z-chunk;
//   * each thread owns one 16-byte vector (1 complex128 or 2 complex64 orbitals) of one
//     (x, y) column and keeps the 2M+1 z-neighbours of its column in registers, so the
//     z-arm of the stencil costs no shared-memory traffic;
//   * the x/y arms come from a double-buffered shared-memory plane holding the tile plus
//     a cross-shaped halo (no corners: the star stencil never reads them); the centre of
//     plane z+1 is written from registers, only the halo is loaded from global memory
//     (mostly L2 hits: concurrently running CTAs march the same z range);
//   * next-plane loads are issued before the barrier of the current plane, so their
//     latency overlaps the current plane's arithmetic; one __syncthreads per plane;
//   * MODE_FIRST reads the state (the hi part of a complex64 system's double-float state)
//     and optionally accumulates the energy and current partial sums; MODE_LAST adds
//     psi + t1 + t2 + t3 + t4 in place (FP64, or double-float for complex64 systems) and
//     writes each point's density contribution for the next sub-step.
// This is the general path (any boundary, loads through L1/L2); finite boxes use the
// TMA-fed sweep of tdks_sweep_tma.cu.
#include "tdks_internal.cuh"
#include "tdks_sweep_common.cuh"

namespace tdks {

// floor(i / n) for possibly negative i
__device__ __forceinline__ int floordiv(int i, int n) { return i >= 0 ? i / n : -((-i - 1) / n) - 1; }

template <int M, int P, int MODE, int BLOCH, int TX, int TY>
__global__ void __launch_bounds__(OVC * TX * TY)
sweep_kernel(const SweepParams p) {
  typedef VT<P> T;
  typedef typename T::V V;
  typedef typename T::S S;
  typedef typename T::R R;
  constexpr int NT = OVC * TX * TY;
  constexpr int SX = TX + 2 * M;
  constexpr int SY = TY + 2 * M;
  constexpr int PLANE = SX * SY * OVC;
  constexpr int NHP = 2 * M * (TX + TY);
  constexpr int NHV = NHP * OVC;
  constexpr int HPT = (NHV + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V *sm = reinterpret_cast<V *>(smem_raw);
  __shared__ double red[NT / 32][4];

  const int tid = threadIdx.x;
  const int v = tid % OVC;
  const int lx = (tid / OVC) % TX;
  const int ly = tid / (OVC * TX);
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const long N = (long)nx * ny * nz;

  S W[M + 1];
#pragma unroll
  for (int m = 0; m <= M; m++) W[m] = T::coef(p.w[m], p.wf[m]);
  const typename W0T<P>::type w0 = P == P_C64 ? (typename W0T<P>::type)p.wf[0] : (typename W0T<P>::type)p.w[0];
  const S CR = T::coef(p.cr, p.crf), CI = T::coef(p.ci, p.cif);
  const bool need_grad = BLOCH && (p.grad_mask != 0);
  const bool grads = BLOCH && MODE == MODE_FIRST && (p.grad_mask & 8);

  for (long item = blockIdx.x; item < p.n_items; item += gridDim.x) {
    long it = item;
    const int tx = (int)(it % p.n_tx); it /= p.n_tx;
    const int ty = (int)(it % p.n_ty); it /= p.n_ty;
    const int kb = (int)(it % p.n_kb); it /= p.n_kb;
    const int zc = (int)it;
    const int kidx = kb / p.n_batches;
    const V *nlk = nl_column<P>(p, kb, v);
    const int z0 = zc * p.zc;
    const int z1 = min(z0 + p.zc, nz);
    const long kbN = (long)kb * N;
    double kL[3] = {0.0, 0.0, 0.0};
    if (BLOCH) {
      kL[0] = p.kvec[3 * kidx + 0] * p.L[0];
      kL[1] = p.kvec[3 * kidx + 1] * p.L[1];
      kL[2] = p.kvec[3 * kidx + 2] * p.L[2];
    }
    const V *in = reinterpret_cast<const V *>(p.in);

    // boundary-extended load of the stencil input at grid position (x, y, z)
    auto load = [&](int x, int y, int z) -> V {
      if ((unsigned)x < (unsigned)nx && (unsigned)y < (unsigned)ny && (unsigned)z < (unsigned)nz)
        return T::ld(in + (kbN + ((long)z * ny + y) * nx + x) * OVC + v);
      if (!BLOCH) return T::zero();
      const int wx = floordiv(x, nx), wy = floordiv(y, ny), wz = floordiv(z, nz);
      x -= wx * nx; y -= wy * ny; z -= wz * nz;
      const V a = T::ld(in + (kbN + ((long)z * ny + y) * nx + x) * OVC + v);
      const double ang = kL[0] * wx + kL[1] * wy + kL[2] * wz;
      if constexpr (P == P_C64) {
        float s, c;
        sincosf((float)ang, &s, &c);
        return T::cmul(pk2(c, c), pk2(s, s), a);
      } else {
        double s, c;
        sincos(ang, &s, &c);
        return T::cmul(T::bc(c), T::bc(s), a);
      }
    };

    const int gx = tx * TX + lx, gy = ty * TY + ly;
    const bool own = gx < nx && gy < ny;

    int hgx[HPT], hgy[HPT], hsl[HPT];
#pragma unroll
    for (int j = 0; j < HPT; j++) {
      const int s = tid + j * NT;
      int hlx = 0, hly = 0;
      hsl[j] = -1;
      if (s < NHV) {
        const int hp = s / OVC;
        if (hp < 2 * M * TY) {
          const int row = hp / (2 * M), c = hp % (2 * M);
          hlx = c < M ? c - M : TX + c - M;
          hly = row;
        } else {
          const int q = hp - 2 * M * TY;
          const int col = q % TX, r = q / TX;
          hly = r < M ? r - M : TY + r - M;
          hlx = col;
        }
        hsl[j] = ((hly + M) * SX + (hlx + M)) * OVC + v;
      }
      hgx[j] = tx * TX + hlx;
      hgy[j] = ty * TY + hly;
    }
    const int csl = ((ly + M) * SX + (lx + M)) * OVC + v;

    V Q[2 * M + 1];
#pragma unroll
    for (int j = 0; j < 2 * M; j++) Q[j] = load(gx, gy, z0 - M + j);
    V H[HPT];
#pragma unroll
    for (int j = 0; j < HPT; j++)
      if (hsl[j] >= 0) H[j] = load(hgx[j], hgy[j], z0);
    sm[csl] = Q[M];
#pragma unroll
    for (int j = 0; j < HPT; j++)
      if (hsl[j] >= 0) sm[hsl[j]] = H[j];

    ObsAcc<P> oa;

    for (int z = z0; z < z1; z++) {
      const int buf = (z - z0) & 1;
      Q[2 * M] = load(gx, gy, z + M);
#pragma unroll
      for (int j = 0; j < HPT; j++)
        if (hsl[j] >= 0) H[j] = load(hgx[j], hgy[j], z + 1);
      const long pt = ((long)z * ny + gy) * nx + gx;
      const long idx = (kbN + pt) * OVC + v;
      R ve = R(0);
      int r0 = 0, r1 = 0;
      LastOperands<P> lop;
      lop.hi = lop.lo = lop.t1 = lop.t2 = T::zero();
      if (own) {
        const PointAux a = p.aux[pt];
        ve = *reinterpret_cast<const R *>(&a.veff);
        if (p.has_proj) { r0 = a.r0; r1 = a.r1; }
        if (MODE == MODE_LAST) load_last<P>(p, idx, lop);
      }
      __syncthreads();
      V gax[3] = {T::zero(), T::zero(), T::zero()};
      V acc = stencil_point<M, P, BLOCH>(p, W, w0, Q, sm + buf * PLANE, csl, SX * OVC, ve, need_grad, grads, gax);
      if (own && r1 > r0) acc = T::add(acc, T::ld(nlk + (long)r0 * OVC));
      if (MODE == MODE_FIRST && p.do_obs && own) {
        oa.add_e(Q[M], acc);
        if (grads) {
#pragma unroll
          for (int a = 0; a < 3; a++) oa.add_j(a, Q[M], gax[a]);
        }
      }
      finish_point<P, MODE>(p, CR, CI, own, idx, v, kidx, Q[M], acc, lop);
      // plane z+1 into the other buffer
      V *Sn = sm + (buf ^ 1) * PLANE;
      Sn[csl] = Q[M + 1];
#pragma unroll
      for (int j = 0; j < HPT; j++)
        if (hsl[j] >= 0) Sn[hsl[j]] = H[j];
#pragma unroll
      for (int j = 0; j < 2 * M; j++) Q[j] = Q[j + 1];
    }
    if (MODE == MODE_FIRST && p.do_obs) reduce_obs<P, NT>(p, oa, item, kidx, red);
    __syncthreads();
  }
}

template <int M, int P, int MODE, int BLOCH, int TX, int TY>
static cudaError_t launch_t(const SweepParams &p, int grid, cudaStream_t s) {
  const size_t smem = sweep_smem(M, TX, TY);
  auto k = sweep_kernel<M, P, MODE, BLOCH, TX, TY>;
  static std::atomic<unsigned> attr_done{0};
  if (cudaError_t e = ensure_smem_attr(k, smem, attr_done)) return e;
  if (grid <= 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, OVC * TX * TY, smem);
    if (per < 1) per = 1;
    long g = (long)sms * per;
    grid = (int)(p.n_items < g ? p.n_items : g);
  }
  k<<<grid, OVC * TX * TY, smem, s>>>(p);
  return cudaGetLastError();
}

int sweep_threads(int tx, int ty) { return OVC * tx * ty; }
size_t sweep_smem(int M, int tx, int ty) {
  return (size_t)2 * (tx + 2 * M) * (ty + 2 * M) * OVC * 16;
}

template <int M, int P, int MODE, int BLOCH>
static cudaError_t by_tile(int tx, int ty, const SweepParams &p, int grid, cudaStream_t s) {
  if (tx == 16 && ty == 8) return launch_t<M, P, MODE, BLOCH, 16, 8>(p, grid, s);
  if (tx == 32 && ty == 4) return launch_t<M, P, MODE, BLOCH, 32, 4>(p, grid, s);
  if (tx == 8 && ty == 8) return launch_t<M, P, MODE, BLOCH, 8, 8>(p, grid, s);
  return cudaErrorInvalidValue;
}

template <int M, int P, int MODE>
static cudaError_t by_bc(int bloch, int tx, int ty, const SweepParams &p, int grid, cudaStream_t s) {
  return bloch ? by_tile<M, P, MODE, 1>(tx, ty, p, grid, s) : by_tile<M, P, MODE, 0>(tx, ty, p, grid, s);
}

template <int M, int P>
static cudaError_t by_mode(int mode, int bloch, int tx, int ty, const SweepParams &p, int grid, cudaStream_t s) {
  switch (mode) {
    case MODE_FIRST: return by_bc<M, P, MODE_FIRST>(bloch, tx, ty, p, grid, s);
    case MODE_MID: return by_bc<M, P, MODE_MID>(bloch, tx, ty, p, grid, s);
    case MODE_LAST: return by_bc<M, P, MODE_LAST>(bloch, tx, ty, p, grid, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep(int M, int prec, int mode, int bloch, int tx, int ty,
                         const SweepParams &p, int grid, cudaStream_t s) {
  if (M == 2) return prec == P_C64 ? by_mode<2, P_C64>(mode, bloch, tx, ty, p, grid, s)
                                   : by_mode<2, P_C128>(mode, bloch, tx, ty, p, grid, s);
  if (M == 4) return prec == P_C64 ? by_mode<4, P_C64>(mode, bloch, tx, ty, p, grid, s)
                                   : by_mode<4, P_C128>(mode, bloch, tx, ty, p, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace tdks
