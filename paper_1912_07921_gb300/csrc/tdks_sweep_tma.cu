// TMA-fed Taylor-term sweep for finite boxes (zero boundary).
//
// Same arithmetic as the general sweep (tdks_sweep.cu; see tdks_sweep_common.cuh), with
// the stencil input streamed by the Tensor Memory Accelerator:
//   * a 5D tensor map views the input as {16 floats, nx, ny, nz, k*batch}; one
//     cp.async.bulk.tensor copy brings a whole (TX+2M) x (TY+2M) plane tile with its halo
//     into shared memory, and out-of-box coordinates arrive as zeros, which is exactly
//     the zero boundary condition of a finite box;
//   * a ring of S plane buffers, each completed by an mbarrier transaction count, runs
//     S - M planes ahead of the plane being computed, so several planes of HBM traffic
//     are in flight per SM without any thread waiting on a load;
//   * the stream of plane loads continues across the CTA's work items (persistent grid,
//     one CTA per SM), so the pipeline never drains between items;
//   * each thread keeps its z-column (2M+1 planes) in registers; x/y neighbours are read
//     from the ring buffer of the output plane.
// Every wait is bounded: a wait that runs out sets the error word, waits (bounded) for
// the copies still in flight, and the CTA returns.
#include "tdks_tma.cuh"

namespace tdks {

template <int M, int P, int MODE, int TX, int TY, int U, bool BATCH, class Src>
__device__ __forceinline__ void tma_sweep_body(const Src &src) {
  typedef VT<P> T;
  typedef typename T::V V;
  typedef typename T::S S_;
  typedef typename T::R R;
  constexpr bool OPS = MODE == MODE_LAST;
  typedef TmaGeom<M, TX, TY, U, OPS> G;
  static_assert(M % U == 0, "M must be a multiple of U");
  static_assert(!OPS || U == 1, "the last Taylor term takes one plane per iteration");
  constexpr int NT = OVC * TX * TY;
  constexpr int SC = G::SC, SH = G::SH;
  constexpr int SO = G::SO > 0 ? G::SO : 1;
  constexpr int QN = 2 * M + U;   // z-queue entries
  constexpr int LP = 2 * M / U;   // priming centre loads per item
  extern __shared__ unsigned char smem_raw[];
  unsigned char *cbase = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  unsigned char *hbase = cbase + (size_t)SC * G::CSLOT_BYTES;
  unsigned char *obase = hbase + (size_t)SH * G::HSLOT_BYTES;
  __shared__ __align__(8) uint64_t cfull[SC];
  __shared__ __align__(8) uint64_t hfull[SH];
  __shared__ __align__(8) uint64_t ofull[SO];
  __shared__ double red[NT / 32][4];
  __shared__ int s_abort;
  __shared__ SweepParams s_params;  // batch: parameters of the current item's system

  const int tid = threadIdx.x;
  const int v = tid % OVC;
  const int lx = (tid / OVC) % TX;
  const int ly = tid / (OVC * TX);
  const int hsl = ((ly + M) * G::SX + (lx + M)) * OVC + v;  // own vector in a halo plane
  const int tsl = ly * TX + lx;                              // own point in a tile
  const int csl = tsl * OVC + v;                             // own vector in a centre plane
  const long n_items_all = src.n_items();
  const long n_my = (long)blockIdx.x < n_items_all ? (n_items_all - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (n_my == 0) return;

  if (tid == 0) {
    for (int s = 0; s < SC; s++) mbar_init(&cfull[s], 1);
    for (int s = 0; s < SH; s++) mbar_init(&hfull[s], 1);
    for (int s = 0; s < SO; s++) mbar_init(&ofull[s], 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const Loader<M, TX, TY, U, G, SC, SH, SO, Src> ld{src, n_my, cbase, hbase, obase, cfull, hfull, ofull};
  // the cursors live in shared memory: only thread 0 uses them, and registers are scarce
  __shared__ LoadCursor cur[3];
  LoadCursor &cc = cur[0], &hc = cur[1], &oc = cur[2];
  if (tid == 0) {
    for (int k = 0; k < 3; k++) cur[k] = LoadCursor{-1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int s = 0; s < SC; s++) ld.issue(cc, 0);
    for (int s = 0; s < SH; s++) ld.issue(hc, 1);
    if (OPS)
      for (int s = 0; s < SO; s++) ld.issue(oc, 2);
  }

  long gc = 0, gh = 0;  // centre / halo (and operand) loads consumed
  RingPos rc, rh, ro;   // their ring positions
  for (long ii = 0; ii < n_my; ii++) {
    const long item = blockIdx.x + ii * gridDim.x;
    const SweepParams *pp;
    const SweepMaps *mp_unused;
    long local;
    src.item(item, pp, mp_unused, local);
    if constexpr (BATCH) {
      __syncthreads();  // everyone is done with the previous item's parameters
      if (tid == 0) s_params = *pp;
      __syncthreads();
      pp = &s_params;
    }
    const SweepParams &p = *pp;
    const int nx = p.nx, ny = p.ny;
    const long N = (long)nx * ny * p.nz;
    const long plane_pts = (long)nx * ny;
    S_ W[M + 1];
#pragma unroll
    for (int m = 0; m <= M; m++) W[m] = T::coef(p.w[m], p.wf[m]);
    const typename W0T<P>::type w0 = P == P_C64 ? (typename W0T<P>::type)p.wf[0] : (typename W0T<P>::type)p.w[0];
    const S_ CR = T::coef(p.cr, p.crf), CI = T::coef(p.ci, p.cif);
    int tx, ty, kb, z0, z1;
    item_geom(p, local, tx, ty, kb, z0, z1);
    const int kidx = kb / p.n_batches;
    const Epi epi = make_epi(p, kidx);
    const bool has_proj = p.has_proj != 0, do_obs = p.do_obs != 0;
    const V *nlk = nl_column<P>(p, kb, v);
    const int n_ent = p.n_ent;
    const int gx = tx * TX + lx, gy = ty * TY + ly;
    const bool own = gx < nx && gy < ny;
    const int nl = loads_of<M, U>(0, z0, z1);
    // vector index of the own point in the first output plane (advances one plane per output)
    long idx = ((long)kb * N + ((long)z0 * ny + gy) * nx + gx) * OVC + v;
    V Q[QN];
#pragma unroll
    for (int j = 0; j < QN; j++) Q[j] = T::zero();
    ObsAcc<P> oa;

    int l = 0;
    bool aborted = false;
    // one centre load (and, past the priming loads, one halo load); RQ = compile-time
    // queue position of its first plane
    auto iteration = [&](auto rq) {
      constexpr int RQ = decltype(rq)::value;
      const int cs = rc.slot;
      if (!mbar_wait_bounded(&cfull[cs], rc.phase)) s_abort = 1;
      const V *cslot = reinterpret_cast<const V *>(cbase + (size_t)cs * G::CSLOT_BYTES);
#pragma unroll
      for (int u = 0; u < U; u++) Q[(RQ + u) % QN] = cslot[u * G::CPLANE + csl];
      const bool out = l >= LP;
      if (out) {
        const int zf = z0 + U * (l - LP);
        const int hs = rh.slot;
        if (!mbar_wait_bounded(&hfull[hs], rh.phase)) s_abort = 1;
        const unsigned char *hslot = hbase + (size_t)hs * G::HSLOT_BYTES;
        const V *xs = reinterpret_cast<const V *>(hslot);
        const PointAux *ax = reinterpret_cast<const PointAux *>(hslot + G::IN_BYTES);
        LastOperands<P> lop;
        lop.hi = lop.lo = lop.t1 = lop.t2 = T::zero();
        if constexpr (OPS) {
          const int os = ro.slot;
          if (!mbar_wait_bounded(&ofull[os], ro.phase)) s_abort = 1;
          const V *ob = reinterpret_cast<const V *>(obase + (size_t)os * G::OP_BYTES);
          lop.hi = ob[csl];
          lop.lo = ob[G::CPLANE + csl];
          lop.t1 = ob[2 * G::CPLANE + csl];
          lop.t2 = ob[3 * G::CPLANE + csl];
        }
        static_for<0, U>([&](auto uc) {
          constexpr int u = decltype(uc)::value;
          constexpr int QB = (RQ + U + u) % QN;  // queue position of plane (zf + u) - M
          const PointAux a = ax[u * TX * TY + tsl];
          const R ve = *reinterpret_cast<const R *>(&a.veff);
          const V nlv = has_proj ? nl_term<P>(nlk, n_ent, a.r0, a.r1) : T::zero();
          V gax[3];
          V acc = stencil_point<M, P, 0, QB, QN>(p, W, w0, Q, xs + u * G::PLANE, hsl, G::SX * OVC, ve, false,
                                                 false, gax);
          const bool live = own && (zf + u < z1);
          if (has_proj) acc = T::add(acc, nlv);
          const V c0 = Q[(QB + M) % QN];
          if (MODE == MODE_FIRST && do_obs && live) oa.add_e(c0, acc);
          finish_point<P, MODE>(epi, CR, CI, live, idx + (long)u * plane_pts * OVC, v, c0, acc, lop);
        });
        idx += U * plane_pts * OVC;
      }
      __syncthreads();
      if (s_abort) {
        aborted = true;
        return;
      }
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ld.issue(cc, 0);
        if (out) {
          ld.issue(hc, 1);
          if (OPS) ld.issue(oc, 2);
        }
      }
      gc++;
      rc.next<SC>();
      if (out) {
        gh++;
        rh.next<SH>();
        if (OPS) ro.next<SO>();
      }
      l++;
    };
    int rq = 0;
    while (l < nl && !aborted) {
      switch (rq) {
#define TDKS_CASE(k)                                                  \
  case k:                                                             \
    if constexpr (k % U == 0 && k < QN) iteration(std::integral_constant<int, k>{}); \
    break;
        TDKS_CASE(0) TDKS_CASE(1) TDKS_CASE(2) TDKS_CASE(3) TDKS_CASE(4)
        TDKS_CASE(5) TDKS_CASE(6) TDKS_CASE(7) TDKS_CASE(8) TDKS_CASE(9)
#undef TDKS_CASE
      }
      rq = rq + U >= QN ? rq + U - QN : rq + U;
    }
    if (aborted) {
      if (tid == 0) {  // (the cursors are thread 0's; nobody else reads them)
        if (p.err) atomicExch(p.err, 1);
        for (long j = gc; j < cc.issued; j++)
          mbar_wait_bounded(&cfull[j % SC], (uint32_t)((j / SC) & 1), DRAIN_LIMIT_CYCLES);
        for (long j = gh; j < hc.issued; j++)
          mbar_wait_bounded(&hfull[j % SH], (uint32_t)((j / SH) & 1), DRAIN_LIMIT_CYCLES);
        for (long j = gh; j < oc.issued; j++)
          mbar_wait_bounded(&ofull[j % SO], (uint32_t)((j / SO) & 1), DRAIN_LIMIT_CYCLES);
      }
      return;
    }
    if (MODE == MODE_FIRST && p.do_obs) reduce_obs<P, NT>(p, oa, local, kidx, red);
  }
}

template <int M, int P, int MODE, int TX, int TY, int U>
__global__ void __launch_bounds__(OVC * TX * TY, 1)
tma_sweep_kernel(const __grid_constant__ SweepMaps maps, const __grid_constant__ SweepParams p) {
  const SingleSrc src{&p, &maps};
  tma_sweep_body<M, P, MODE, TX, TY, U, false>(src);
}

template <int M, int P, int MODE, int TX, int TY, int U>
__global__ void __launch_bounds__(OVC * TX * TY, 1)
tma_sweep_batch_kernel(const __grid_constant__ BatchSweepArgs a) {
  const BatchSrc src{&a};
  tma_sweep_body<M, P, MODE, TX, TY, U, true>(src);
}

// Planes per TMA copy of a sweep mode (the z depth of its tensor-map boxes): the lockstep
// kernel takes two planes per iteration in the complex64 term sweeps, everything else one.
int tma_planes(int prec, int mode, bool lockstep) { return (lockstep && prec == P_C64 && mode != MODE_LAST) ? 2 : 1; }

bool tma_supported(int M, int tx, int ty) { return (M == 2 || M == 4) && tx == 16 && ty == 8; }

// Lockstep kernel (16x8 tiles; complex64 term sweeps take two planes per iteration).
template <int M, int P, int MODE, int U>
static cudaError_t launch_lockstep_t(const SweepMaps &maps, const SweepParams &p, int grid, cudaStream_t s) {
  typedef TmaGeom<M, 16, 8, U, MODE == MODE_LAST> G;
  auto k = tma_sweep_kernel<M, P, MODE, 16, 8, U>;
  static std::atomic<unsigned> attr_done{0};
  if (cudaError_t e = ensure_smem_attr(k, G::SMEM, attr_done)) return e;
  if (grid <= 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = (int)(p.n_items < sms ? p.n_items : sms);
  }
  k<<<grid, OVC * 16 * 8, G::SMEM, s>>>(maps, p);
  return cudaGetLastError();
}

extern template cudaError_t launch_ws_batch_shape<1>(int, int, int, const BatchSweepArgs &, cudaStream_t);
extern template cudaError_t launch_ws_batch_shape<2>(int, int, int, const BatchSweepArgs &, cudaStream_t);
extern template cudaError_t launch_ws_batch_shape<3>(int, int, int, const BatchSweepArgs &, cudaStream_t);
extern template cudaError_t launch_ws_batch_shape<4>(int, int, int, const BatchSweepArgs &, cudaStream_t);
extern template cudaError_t launch_ws_batch_shape<5>(int, int, int, const BatchSweepArgs &, cudaStream_t);
template cudaError_t launch_ws_batch_shape<0>(int, int, int, const BatchSweepArgs &, cudaStream_t);

cudaError_t launch_sweep_tma_batch(int M, int prec, int mode, const BatchSweepArgs &a, cudaStream_t s, int shape) {
  if (M != 2 && M != 4) return cudaErrorInvalidValue;
  switch (shape) {
    case 0: return launch_ws_batch_shape<0>(M, prec, mode, a, s);
    case 1: return launch_ws_batch_shape<1>(M, prec, mode, a, s);
    case 2: return launch_ws_batch_shape<2>(M, prec, mode, a, s);
    case 3: return launch_ws_batch_shape<3>(M, prec, mode, a, s);
    case 4: return launch_ws_batch_shape<4>(M, prec, mode, a, s);
    case 5: return launch_ws_batch_shape<5>(M, prec, mode, a, s);
  }
  return cudaErrorInvalidValue;
}

template <int M, int P>
static cudaError_t lockstep_by_mode(int mode, const SweepMaps &maps, const SweepParams &p, int grid, cudaStream_t s) {
  switch (mode) {
    case MODE_FIRST: return launch_lockstep_t<M, P, MODE_FIRST, P == P_C64 ? 2 : 1>(maps, p, grid, s);
    case MODE_MID: return launch_lockstep_t<M, P, MODE_MID, P == P_C64 ? 2 : 1>(maps, p, grid, s);
    case MODE_LAST: return launch_lockstep_t<M, P, MODE_LAST, 1>(maps, p, grid, s);
  }
  return cudaErrorInvalidValue;
}

// Shapes 1..4 are compiled in translation units of their own (tdks_sweep_ws*.cu).
extern template cudaError_t launch_ws_shape<1>(int, int, int, int, const SweepMaps &, const SweepParams &, int,
                                                 cudaStream_t);
extern template cudaError_t launch_ws_shape<2>(int, int, int, int, const SweepMaps &, const SweepParams &, int,
                                                 cudaStream_t);
extern template cudaError_t launch_ws_shape<3>(int, int, int, int, const SweepMaps &, const SweepParams &, int,
                                                 cudaStream_t);
extern template cudaError_t launch_ws_shape<4>(int, int, int, int, const SweepMaps &, const SweepParams &, int,
                                                 cudaStream_t);
extern template cudaError_t launch_ws_shape<5>(int, int, int, int, const SweepMaps &, const SweepParams &, int,
                                                 cudaStream_t);
template cudaError_t launch_ws_shape<0>(int, int, int, int, const SweepMaps &, const SweepParams &, int, cudaStream_t);

template <int SHAPE>
static void shape_of(int *tx, int *ty, int *rows, int *warps) {
  typedef WsShape<SHAPE> S;
  if (tx) *tx = S::TX;
  if (ty) *ty = S::TY;
  if (rows) *rows = S::R;
  if (warps) *warps = WsWarps<S::TX, S::TY, S::R>::CW;
}

bool ws_shape_info(int shape, int *tx, int *ty, int *rows, int *warps) {
  switch (shape) {
    case 0: shape_of<0>(tx, ty, rows, warps); return true;
    case 1: shape_of<1>(tx, ty, rows, warps); return true;
    case 2: shape_of<2>(tx, ty, rows, warps); return true;
    case 3: shape_of<3>(tx, ty, rows, warps); return true;
    case 4: shape_of<4>(tx, ty, rows, warps); return true;
    case 5: {
      // complex64 systems: 8 one-complex vectors per point (complex128 runs shape 2, also 12 warps)
      typedef WsShape<5> S;
      if (tx) *tx = S::TX;
      if (ty) *ty = S::TY;
      if (rows) *rows = S::R;
      if (warps) *warps = WsWarps<S::TX, S::TY, S::R, 8>::CW;
      return true;
    }
  }
  return false;
}

cudaError_t launch_sweep_tma(int M, int prec, int mode, int tx, int ty, const SweepMaps &maps, const SweepParams &p,
                             int grid, cudaStream_t s, bool lockstep, int shape) {
  if (!tma_supported(M, tx, ty)) return cudaErrorInvalidValue;
  if (lockstep && p.bloch) return cudaErrorInvalidValue;  // periodic cells: warp-specialised sweep only
  const int b = p.bloch;
  if (lockstep) {
    if (M == 2) return prec == P_C64 ? lockstep_by_mode<2, P_C64>(mode, maps, p, grid, s)
                                     : lockstep_by_mode<2, P_C128>(mode, maps, p, grid, s);
    return prec == P_C64 ? lockstep_by_mode<4, P_C64>(mode, maps, p, grid, s)
                         : lockstep_by_mode<4, P_C128>(mode, maps, p, grid, s);
  }
  switch (shape) {
    case 0: return launch_ws_shape<0>(M, prec, mode, b, maps, p, grid, s);
    case 1: return launch_ws_shape<1>(M, prec, mode, b, maps, p, grid, s);
    case 2: return launch_ws_shape<2>(M, prec, mode, b, maps, p, grid, s);
    case 3: return launch_ws_shape<3>(M, prec, mode, b, maps, p, grid, s);
    case 4: return launch_ws_shape<4>(M, prec, mode, b, maps, p, grid, s);
    case 5: return launch_ws_shape<5>(M, prec, mode, b, maps, p, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace tdks

