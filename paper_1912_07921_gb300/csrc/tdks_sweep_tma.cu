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
#include <cuda.h>

#include <type_traits>

#include "tdks_internal.cuh"
#include "tdks_sweep_common.cuh"

namespace tdks {

namespace {

constexpr long long WAIT_LIMIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > WAIT_LIMIT_CYCLES) return false;
  return true;
}
__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *tmap, uint64_t *bar, int c0, int c1,
                                            int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace

// Compile-time loop: f(integral_constant<int, 0>) ... f(integral_constant<int, N-1>).
template <int I, int N, class F>
__device__ __forceinline__ void static_for(F &&f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// U planes per copy (box depth U in z) and per loop iteration; each thread computes U
// independent outputs per iteration, which halves the per-output cost of the barrier,
// the waits and the address arithmetic and doubles the independent work in flight.
// The ring holds 8 planes.
template <int M, int TX, int TY, int U>
struct TmaGeom {
  static constexpr int SX = TX + 2 * M, SY = TY + 2 * M;
  static constexpr int PLANE = SX * SY * OVC;  // 16-byte vectors per plane
  static constexpr int SLOT = PLANE * U;       // vectors per ring slot
  static constexpr uint32_t SLOT_BYTES = SLOT * 16;
  static constexpr int S = 8 / U;              // ring depth (slots)
  static constexpr size_t SMEM = (size_t)S * SLOT_BYTES + 128;
};

// Work sources: a single system (parameters and tensor map are kernel parameters), or a
// batch of systems (per-system parameters and tensor maps in device arrays; a CTA stages
// the parameters of its current item in shared memory).
struct SingleSrc {
  const SweepParams *p;
  const CUtensorMap *tmap;
  __device__ __forceinline__ long n_items() const { return p->n_items; }
  __device__ __forceinline__ void item(long it, const SweepParams *&pp, const CUtensorMap *&tm, long &local) const {
    pp = p;
    tm = tmap;
    local = it;
  }
};

__device__ __forceinline__ int find_item_sys(const long *begin, int n, long u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (begin[mid] <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct BatchSrc {
  const BatchSweepArgs *a;
  __device__ __forceinline__ long n_items() const { return a->total_items; }
  __device__ __forceinline__ void item(long it, const SweepParams *&pp, const CUtensorMap *&tm, long &local) const {
    const int s = find_item_sys(a->item_begin, a->n_sys, it);
    pp = a->params + s;
    tm = reinterpret_cast<const CUtensorMap *>(a->tmaps) + 4 * s + a->which;
    local = it - a->item_begin[s];
  }
};

template <int M, int P, int MODE, int TX, int TY, int U, bool BATCH, class Src>
__device__ __forceinline__ void tma_sweep_body(const Src &src) {
  typedef VT<P> T;
  typedef typename T::V V;
  typedef typename T::S S_;
  typedef typename T::R R;
  typedef TmaGeom<M, TX, TY, U> G;
  static_assert(M % U == 0, "M must be a multiple of U");
  constexpr int NT = OVC * TX * TY;
  constexpr int S = G::S;
  constexpr int QN = 2 * M + U;   // z-queue entries
  constexpr int LP = 2 * M / U;   // priming loads per item
  constexpr int MU = M / U;       // loads between a plane's arrival and its output
  extern __shared__ unsigned char smem_raw[];
  V *ring = reinterpret_cast<V *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  __shared__ __align__(8) uint64_t full[S];
  __shared__ double red[NT / 32][4];
  __shared__ int s_abort;
  __shared__ SweepParams s_params;  // batch: parameters of the current item's system

  const int tid = threadIdx.x;
  const int v = tid % OVC;
  const int lx = (tid / OVC) % TX;
  const int ly = tid / (OVC * TX);
  const int csl = ((ly + M) * G::SX + (lx + M)) * OVC + v;
  const long n_items_all = src.n_items();
  const long n_my = (long)blockIdx.x < n_items_all ? (n_items_all - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (n_my == 0) return;

  if (tid == 0) {
    for (int s = 0; s < S; s++) mbar_init(&full[s], 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  auto geom = [&](const SweepParams &q, long it, int &tx, int &ty, int &kb, int &z0, int &z1) {
    tx = (int)(it % q.n_tx); it /= q.n_tx;
    ty = (int)(it % q.n_ty); it /= q.n_ty;
    kb = (int)(it % q.n_kb); it /= q.n_kb;
    z0 = (int)it * q.zc;
    z1 = min(z0 + q.zc, q.nz);
  };
  auto loads_of = [&](int z0, int z1) { return (z1 - z0 + 2 * M + U - 1) / U; };

  // producer cursor (thread 0 only): the slot loads of all this CTA's items, in order
  long pi = 0, issued = 0;
  int pl = 0;
  auto issue_next = [&]() {
    if (pi >= n_my) return;
    const SweepParams *qp;
    const CUtensorMap *tm;
    long local;
    src.item(blockIdx.x + pi * gridDim.x, qp, tm, local);
    int tx, ty, kb, z0, z1;
    geom(*qp, local, tx, ty, kb, z0, z1);
    const int slot = (int)(issued % S);
    mbar_expect_tx(&full[slot], G::SLOT_BYTES);
    tma_load_5d(ring + (size_t)slot * G::SLOT, tm, &full[slot], 0, tx * TX - M, ty * TY - M,
                z0 - M + U * pl, kb);
    issued++;
    if (++pl >= loads_of(z0, z1)) { pl = 0; pi++; }
  };
  if (tid == 0)
    for (int s = 0; s < S; s++) issue_next();

  long g = 0;  // slot loads consumed
  for (long ii = 0; ii < n_my; ii++) {
    const long item = blockIdx.x + ii * gridDim.x;
    const SweepParams *pp;
    const CUtensorMap *tm_unused;
    long local;
    src.item(item, pp, tm_unused, local);
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
    for (int m = 0; m <= M; m++) W[m] = T::bc(p.w[m]);
    const typename W0T<P>::type w0 = (typename W0T<P>::type)p.w[0];
    const S_ CR = T::bc(p.cr), CI = T::bc(p.ci);
    int tx, ty, kb, z0, z1;
    geom(p, local, tx, ty, kb, z0, z1);
    const int kidx = kb / p.n_batches;
    const int gx = tx * TX + lx, gy = ty * TY + ly;
    const bool own = gx < nx && gy < ny;
    const int nl = loads_of(z0, z1);
    // own point of the next output plane: grid index and vector index
    long pt = ((long)z0 * ny + gy) * nx + gx;
    long idx = ((long)kb * N + pt) * OVC + v;
    V Q[QN];
#pragma unroll
    for (int j = 0; j < QN; j++) Q[j] = T::zero();
    ObsAcc<P> oa;
    // own-point operands of the next U output planes (prefetched one iteration ahead)
    R ve[U];
    int r0[U], r1[U];
    LastOperands<P> lop[U];
    auto prefetch = [&](int zfirst) {
#pragma unroll
      for (int u = 0; u < U; u++) {
        ve[u] = R(0);
        r0[u] = r1[u] = 0;
        lop[u].hi = lop[u].lo = lop[u].t1 = lop[u].t2 = T::zero();
        if (own && zfirst + u < z1) {
          const long q = pt + u * plane_pts;
          ve[u] = reinterpret_cast<const R *>(p.veff)[q];
          if (p.rowptr) { r0[u] = __ldg(p.rowptr + q); r1[u] = __ldg(p.rowptr + q + 1); }
          if (MODE == MODE_LAST) load_last<P>(p, idx + u * plane_pts * OVC, lop[u]);
        }
      }
    };
    prefetch(z0);

    int l = 0;
    bool aborted = false;
    // one slot load; RQ = compile-time queue position of its first plane
    auto iteration = [&](auto rq) {
      constexpr int RQ = decltype(rq)::value;
      const int slot = (int)(g & (S - 1));
      if (!mbar_wait_bounded(&full[slot], (uint32_t)((g / S) & 1))) s_abort = 1;
      const V *in_slot = ring + (size_t)slot * G::SLOT;
#pragma unroll
      for (int u = 0; u < U; u++) Q[(RQ + u) % QN] = in_slot[u * G::PLANE + csl];
      if (l >= LP) {
        const int zf = z0 + U * (l - LP);
        const V *xs = ring + (size_t)((g - MU) & (S - 1)) * G::SLOT;
        R ve_c[U];
        int r0_c[U], r1_c[U];
        LastOperands<P> cur[U];
#pragma unroll
        for (int u = 0; u < U; u++) { ve_c[u] = ve[u]; r0_c[u] = r0[u]; r1_c[u] = r1[u]; cur[u] = lop[u]; }
        const long cidx = idx;
        pt += U * plane_pts;
        idx += U * plane_pts * OVC;
        prefetch(zf + U);
        static_for<0, U>([&](auto uc) {
          constexpr int u = decltype(uc)::value;
          constexpr int QB = (RQ + U + u) % QN;  // queue position of plane (zf + u) - M
          V gax[3];
          V acc = stencil_point<M, P, 0, QB, QN>(p, W, w0, Q, xs + u * G::PLANE, csl, G::SX * OVC, ve_c[u], false,
                                                 false, gax);
          const bool live = own && (zf + u < z1);
          if (live && r1_c[u] > r0_c[u]) acc = kb_scatter<P, 0>(p, kb, kidx, v, r0_c[u], r1_c[u], acc);
          const V c0 = Q[(QB + M) % QN];
          if (MODE == MODE_FIRST && p.do_obs && live) oa.add_e(c0, acc);
          finish_point<P, MODE>(p, CR, CI, live, cidx + (long)u * plane_pts * OVC, v, kidx, c0, acc, cur[u]);
        });
      }
      __syncthreads();
      if (s_abort) {
        aborted = true;
        return;
      }
      if (tid == 0 && g >= MU) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_next();
      }
      g++;
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
      if (tid == 0) {
        if (p.err) atomicExch(p.err, 1);
        for (long j = g; j < issued; j++) mbar_wait_bounded(&full[j & (S - 1)], (uint32_t)((j / S) & 1));
      }
      return;
    }
    if (MODE == MODE_FIRST && p.do_obs) reduce_obs<P, NT>(p, oa, local, kidx, red);
  }
}

template <int M, int P, int MODE, int TX, int TY, int U>
__global__ void __launch_bounds__(OVC * TX * TY, 1)
tma_sweep_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ SweepParams p) {
  const SingleSrc src{&p, &tmap};
  tma_sweep_body<M, P, MODE, TX, TY, U, false>(src);
}

template <int M, int P, int MODE, int TX, int TY, int U>
__global__ void __launch_bounds__(OVC * TX * TY, 1)
tma_sweep_batch_kernel(const __grid_constant__ BatchSweepArgs a) {
  const BatchSrc src{&a};
  tma_sweep_body<M, P, MODE, TX, TY, U, true>(src);
}

// Planes per TMA copy of a sweep mode (the z depth of its tensor-map box): complex64 term
// sweeps take two planes per iteration, everything else one.
int tma_planes(int prec, int mode) { return (prec == P_C64 && mode != MODE_LAST) ? 2 : 1; }

bool tma_supported(int M, int tx, int ty) { return (M == 2 || M == 4) && tx == 16 && ty == 8; }

template <int M, int P, int MODE, int TX, int TY, int U>
static cudaError_t launch_tma_t(const void *tmap, const SweepParams &p, int grid, cudaStream_t s) {
  typedef TmaGeom<M, TX, TY, U> G;
  auto k = tma_sweep_kernel<M, P, MODE, TX, TY, U>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (grid <= 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = (int)(p.n_items < sms ? p.n_items : sms);
  }
  k<<<grid, OVC * TX * TY, G::SMEM, s>>>(*reinterpret_cast<const CUtensorMap *>(tmap), p);
  return cudaGetLastError();
}

template <int M, int P, int MODE, int TX, int TY, int U>
static cudaError_t launch_tma_batch_t(const BatchSweepArgs &a, cudaStream_t s) {
  typedef TmaGeom<M, TX, TY, U> G;
  auto k = tma_sweep_batch_kernel<M, P, MODE, TX, TY, U>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)(a.total_items < sms ? a.total_items : sms);
  if (grid <= 0) return cudaSuccess;
  k<<<grid, OVC * TX * TY, G::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int M, int P>
static cudaError_t tma_batch_by_mode(int mode, const BatchSweepArgs &a, cudaStream_t s) {
  switch (mode) {
    case MODE_FIRST: return launch_tma_batch_t<M, P, MODE_FIRST, 16, 8, P == P_C64 ? 2 : 1>(a, s);
    case MODE_MID: return launch_tma_batch_t<M, P, MODE_MID, 16, 8, P == P_C64 ? 2 : 1>(a, s);
    case MODE_LAST: return launch_tma_batch_t<M, P, MODE_LAST, 16, 8, 1>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_tma_batch(int M, int prec, int mode, const BatchSweepArgs &a, cudaStream_t s) {
  if (M == 2) return prec == P_C64 ? tma_batch_by_mode<2, P_C64>(mode, a, s) : tma_batch_by_mode<2, P_C128>(mode, a, s);
  if (M == 4) return prec == P_C64 ? tma_batch_by_mode<4, P_C64>(mode, a, s) : tma_batch_by_mode<4, P_C128>(mode, a, s);
  return cudaErrorInvalidValue;
}

template <int M, int P>
static cudaError_t tma_by_mode(int mode, const void *tmap, const SweepParams &p, int grid, cudaStream_t s) {
  switch (mode) {
    // complex64: two planes per iteration in the term sweeps; complex128 (FP64-bound, and
    // twice the registers per value) one plane
    case MODE_FIRST: return launch_tma_t<M, P, MODE_FIRST, 16, 8, P == P_C64 ? 2 : 1>(tmap, p, grid, s);
    case MODE_MID: return launch_tma_t<M, P, MODE_MID, 16, 8, P == P_C64 ? 2 : 1>(tmap, p, grid, s);  // = tma_planes
    case MODE_LAST: return launch_tma_t<M, P, MODE_LAST, 16, 8, 1>(tmap, p, grid, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_tma(int M, int prec, int mode, int tx, int ty, const void *tmap, const SweepParams &p,
                             int grid, cudaStream_t s) {
  if (!tma_supported(M, tx, ty)) return cudaErrorInvalidValue;
  if (M == 2) return prec == P_C64 ? tma_by_mode<2, P_C64>(mode, tmap, p, grid, s)
                                   : tma_by_mode<2, P_C128>(mode, tmap, p, grid, s);
  return prec == P_C64 ? tma_by_mode<4, P_C64>(mode, tmap, p, grid, s)
                       : tma_by_mode<4, P_C128>(mode, tmap, p, grid, s);
}

}  // namespace tdks
