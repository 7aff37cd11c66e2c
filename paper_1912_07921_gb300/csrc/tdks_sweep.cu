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
//   * MODE_FIRST reads the complex128 state and (optionally) accumulates the energy and
//     current partial sums; MODE_LAST adds psi + t1 + t2 + t3 + t4 in FP64 in place and
//     writes each point's density contribution for the next sub-step.
#include "tdks_internal.cuh"
#include "tdks_vec.cuh"

namespace tdks {

template <int P, int MODE>
struct InLoad {
  typedef typename VT<P>::V V;
  static __device__ __forceinline__ V ld(const void *base, long pt, int v) {
    if (MODE == MODE_FIRST) return VT<P>::ld_state(reinterpret_cast<const double2 *>(base), pt, v);
    return VT<P>::ld(reinterpret_cast<const V *>(base) + pt * OVC + v);
  }
};

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
  for (int m = 0; m <= M; m++) W[m] = T::bc(p.w[m]);
  const S CR = T::bc(p.cr), CI = T::bc(p.ci);
  const bool need_grad = BLOCH && (p.grad_mask != 0);

  for (long item = blockIdx.x; item < p.n_items; item += gridDim.x) {
    long it = item;
    const int tx = (int)(it % p.n_tx); it /= p.n_tx;
    const int ty = (int)(it % p.n_ty); it /= p.n_ty;
    const int kb = (int)(it % p.n_kb); it /= p.n_kb;
    const int zc = (int)it;
    const int kidx = kb / p.n_batches;
    const int z0 = zc * p.zc;
    const int z1 = min(z0 + p.zc, nz);
    const long kbN = (long)kb * N;
    double kL[3] = {0.0, 0.0, 0.0};
    if (BLOCH) {
      kL[0] = p.kvec[3 * kidx + 0] * p.L[0];
      kL[1] = p.kvec[3 * kidx + 1] * p.L[1];
      kL[2] = p.kvec[3 * kidx + 2] * p.L[2];
    }

    // boundary-extended load of the stencil input at grid position (x, y, z)
    auto load = [&](int x, int y, int z) -> V {
      if ((unsigned)x < (unsigned)nx && (unsigned)y < (unsigned)ny && (unsigned)z < (unsigned)nz)
        return InLoad<P, MODE>::ld(p.in, kbN + ((long)z * ny + y) * nx + x, v);
      if (!BLOCH) return T::zero();
      const int wx = floordiv(x, nx), wy = floordiv(y, ny), wz = floordiv(z, nz);
      x -= wx * nx; y -= wy * ny; z -= wz * nz;
      V a = InLoad<P, MODE>::ld(p.in, kbN + ((long)z * ny + y) * nx + x, v);
      double s, c;
      sincos(kL[0] * wx + kL[1] * wy + kL[2] * wz, &s, &c);
      return T::cmul(T::bc(c), T::bc(s), a);
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

    V Q[2 * M];
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

    double acc_e = 0.0, acc_j[3] = {0.0, 0.0, 0.0};

    for (int z = z0; z < z1; z++) {
      const int buf = (z - z0) & 1;
      const V Qn = load(gx, gy, z + M);
#pragma unroll
      for (int j = 0; j < HPT; j++)
        if (hsl[j] >= 0) H[j] = load(hgx[j], hgy[j], z + 1);
      const long pt = ((long)z * ny + gy) * nx + gx;
      R ve = R(0);
      int r0 = 0, r1 = 0;
      V T1 = T::zero(), T2 = T::zero();
      double2 PS[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
      if (own) {
        ve = reinterpret_cast<const R *>(p.veff)[pt];
        if (p.rowptr) { r0 = __ldg(p.rowptr + pt); r1 = __ldg(p.rowptr + pt + 1); }
        if (MODE == MODE_LAST) {
          T1 = T::ld(reinterpret_cast<const V *>(p.t1) + (kbN + pt) * OVC + v);
          T2 = T::ld(reinterpret_cast<const V *>(p.t2) + (kbN + pt) * OVC + v);
          const double2 *ps = reinterpret_cast<const double2 *>(p.psi) + (kbN + pt) * (OVC * T::CPV) + T::CPV * v;
#pragma unroll
          for (int c = 0; c < T::CPV; c++) PS[c] = ps[c];
        }
      }
      __syncthreads();
      const V *Sp = sm + buf * PLANE;
      const V c0 = Q[M];
      V acc = T::mul(T::bc((double)ve + p.w[0]), c0);
      V gsum = T::zero();
      V gax[3] = {T::zero(), T::zero(), T::zero()};
#pragma unroll
      for (int m = 1; m <= M; m++) {
        const V zm = Q[M - m];
        const V zp = (M + m < 2 * M) ? Q[M + m] : Qn;
        const V xm = Sp[csl - m * OVC], xp = Sp[csl + m * OVC];
        const V ym = Sp[csl - m * SX * OVC], yp = Sp[csl + m * SX * OVC];
        const V s6 = T::add(T::add(T::add(zm, zp), T::add(xm, xp)), T::add(ym, yp));
        acc = T::fma(W[m], s6, acc);
        if (need_grad) {
          const V dx = T::sub(xp, xm), dy = T::sub(yp, ym), dz = T::sub(zp, zm);
          gsum = T::fma(T::bc(p.A[0] * p.gw[m]), dx,
                        T::fma(T::bc(p.A[1] * p.gw[m]), dy, T::fma(T::bc(p.A[2] * p.gw[m]), dz, gsum)));
          if (MODE == MODE_FIRST && (p.grad_mask & 8)) {
            const S gm = T::bc(p.gw[m]);
            gax[0] = T::fma(gm, dx, gax[0]);
            gax[1] = T::fma(gm, dy, gax[1]);
            gax[2] = T::fma(gm, dz, gax[2]);
          }
        }
      }
      if (need_grad) acc = T::add(acc, T::negi(gsum));
      // Kleinman-Bylander scatter: sum_aj beta_aj(r) phase* q_aj
      if (own && r1 > r0) {
        for (int e = r0; e < r1; e++) {
          const ProjEntry &E = p.ent[__ldg(p.rowent + e)];
          const V *qa = reinterpret_cast<const V *>(p.q) + ((long)(kb * p.n_atoms + E.atom) * 4) * OVC + v;
          V nl;
          if (P == P_C64) {
            nl = T::mul(T::bc(E.beta[0]), T::ld(qa));
#pragma unroll
            for (int j = 1; j < 4; j++) nl = T::fma(T::bc(E.beta[j]), T::ld(qa + j * OVC), nl);
          } else {
            nl = T::mul(T::bc(E.betad[0]), T::ld(qa));
#pragma unroll
            for (int j = 1; j < 4; j++) nl = T::fma(T::bc(E.betad[j]), T::ld(qa + j * OVC), nl);
          }
          if (BLOCH || p.grad_mask) {
            double ang = 0.0;
            if (BLOCH)
              ang += p.kvec[3 * kidx] * E.T[0] + p.kvec[3 * kidx + 1] * E.T[1] + p.kvec[3 * kidx + 2] * E.T[2];
            ang += p.A[0] * E.d[0] + p.A[1] * E.d[1] + p.A[2] * E.d[2];
            double s, c;
            sincos(ang, &s, &c);
            nl = T::cmul(T::bc(c), T::bc(-s), nl);
          }
          acc = T::add(acc, nl);
        }
      }
      if (MODE == MODE_FIRST && p.do_obs && own) {
        double2 cd[2], hd[2];
        T::to_d(c0, cd);
        T::to_d(acc, hd);
#pragma unroll
        for (int c = 0; c < T::CPV; c++) acc_e += cd[c].x * hd[c].x + cd[c].y * hd[c].y;
        if (BLOCH && (p.grad_mask & 8)) {
#pragma unroll
          for (int a = 0; a < 3; a++) {
            double2 gd[2];
            T::to_d(gax[a], gd);
#pragma unroll
            for (int c = 0; c < T::CPV; c++) acc_j[a] += cd[c].x * gd[c].y - cd[c].y * gd[c].x;
          }
        }
      }
      const V outv = T::cmul(CR, CI, acc);
      if (MODE != MODE_LAST) {
        if (own) reinterpret_cast<V *>(p.out)[(kbN + pt) * OVC + v] = outv;
      } else {
        double2 a1[2], a2[2], a3[2], a4[2];
        T::to_d(T1, a1);
        T::to_d(T2, a2);
        T::to_d(c0, a3);
        T::to_d(outv, a4);
        double dsum = 0.0;
#pragma unroll
        for (int c = 0; c < T::CPV; c++) {
          double re = PS[c].x + a1[c].x;
          double im = PS[c].y + a1[c].y;
          re += a2[c].x; im += a2[c].y;
          re += a3[c].x; im += a3[c].y;
          re += a4[c].x; im += a4[c].y;
          PS[c] = make_double2(re, im);
          dsum += re * re + im * im;
        }
        if (own) {
          double2 *ps = reinterpret_cast<double2 *>(p.psi) + (kbN + pt) * (OVC * T::CPV) + T::CPV * v;
#pragma unroll
          for (int c = 0; c < T::CPV; c++) ps[c] = PS[c];
        }
        // lanes 4j..4j+3 hold the OVC vectors of one point
        dsum += __shfl_xor_sync(0xffffffffu, dsum, 1);
        dsum += __shfl_xor_sync(0xffffffffu, dsum, 2);
        if (own && v == 0) p.dens_part[kbN + pt] = p.wocc[kidx] * dsum;
      }
      // plane z+1 into the other buffer
      V *Sn = sm + (buf ^ 1) * PLANE;
      Sn[csl] = (M + 1 < 2 * M) ? Q[M + 1] : Qn;
#pragma unroll
      for (int j = 0; j < HPT; j++)
        if (hsl[j] >= 0) Sn[hsl[j]] = H[j];
#pragma unroll
      for (int j = 0; j < 2 * M - 1; j++) Q[j] = Q[j + 1];
      Q[2 * M - 1] = Qn;
    }
    if (MODE == MODE_FIRST && p.do_obs) {
      double vals[4] = {acc_e, acc_j[0], acc_j[1], acc_j[2]};
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
    __syncthreads();
  }
}

template <int M, int P, int MODE, int BLOCH, int TX, int TY>
static cudaError_t launch_t(const SweepParams &p, int grid, cudaStream_t s) {
  const size_t smem = sweep_smem(M, TX, TY);
  auto k = sweep_kernel<M, P, MODE, BLOCH, TX, TY>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
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
