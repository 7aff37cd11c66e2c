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

template <int M, int TX, int TY>
struct TmaGeom {
  static constexpr int SX = TX + 2 * M, SY = TY + 2 * M;
  static constexpr int PLANE = SX * SY * OVC;  // 16-byte vectors
  static constexpr uint32_t PLANE_BYTES = PLANE * 16;
  static constexpr int S = 8;                  // ring depth (planes)
  static constexpr size_t SMEM = (size_t)S * PLANE_BYTES + 128;
};

template <int M, int P, int MODE, int TX, int TY>
__global__ void __launch_bounds__(OVC * TX * TY, 1)
tma_sweep_kernel(const __grid_constant__ CUtensorMap tmap, const SweepParams p) {
  typedef VT<P> T;
  typedef typename T::V V;
  typedef typename T::S S_;
  typedef typename T::R R;
  typedef TmaGeom<M, TX, TY> G;
  constexpr int NT = OVC * TX * TY;
  constexpr int S = G::S;
  constexpr int QN = 2 * M + 1;
  extern __shared__ unsigned char smem_raw[];
  V *ring = reinterpret_cast<V *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  __shared__ __align__(8) uint64_t full[S];
  __shared__ double red[NT / 32][4];
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int v = tid % OVC;
  const int lx = (tid / OVC) % TX;
  const int ly = tid / (OVC * TX);
  const int csl = ((ly + M) * G::SX + (lx + M)) * OVC + v;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const long N = (long)nx * ny * nz;
  const long plane_pts = (long)nx * ny;
  const long n_my = (long)blockIdx.x < p.n_items ? (p.n_items - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (n_my == 0) return;

  S_ W[M + 1];
#pragma unroll
  for (int m = 0; m <= M; m++) W[m] = T::bc(p.w[m]);
  const typename W0T<P>::type w0 = (typename W0T<P>::type)p.w[0];

  if (tid == 0) {
    for (int s = 0; s < S; s++) mbar_init(&full[s], 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  auto geom = [&](long item, int &tx, int &ty, int &kb, int &z0, int &z1) {
    long it = item;
    tx = (int)(it % p.n_tx); it /= p.n_tx;
    ty = (int)(it % p.n_ty); it /= p.n_ty;
    kb = (int)(it % p.n_kb); it /= p.n_kb;
    z0 = (int)it * p.zc;
    z1 = min(z0 + p.zc, nz);
  };

  // producer cursor (thread 0 only): the plane loads of all this CTA's items, in order
  long pi = 0, issued = 0;
  int pl = 0;
  auto issue_next = [&]() {
    if (pi >= n_my) return;
    int tx, ty, kb, z0, z1;
    geom(blockIdx.x + pi * gridDim.x, tx, ty, kb, z0, z1);
    const int slot = (int)(issued % S);
    mbar_expect_tx(&full[slot], G::PLANE_BYTES);
    tma_load_5d(ring + (size_t)slot * G::PLANE, &tmap, &full[slot], 0, tx * TX - M, ty * TY - M, z0 - M + pl, kb);
    issued++;
    if (++pl >= (z1 - z0) + 2 * M) { pl = 0; pi++; }
  };
  if (tid == 0)
    for (int s = 0; s < S; s++) issue_next();

  long g = 0;  // loads consumed
  for (long ii = 0; ii < n_my; ii++) {
    const long item = blockIdx.x + ii * gridDim.x;
    int tx, ty, kb, z0, z1;
    geom(item, tx, ty, kb, z0, z1);
    const int kidx = kb / p.n_batches;
    const int gx = tx * TX + lx, gy = ty * TY + ly;
    const bool own = gx < nx && gy < ny;
    const int nl = (z1 - z0) + 2 * M;
    // own point of the next output plane: grid index and vector index (advance one plane
    // per output)
    long pt = ((long)z0 * ny + gy) * nx + gx;
    long idx = ((long)kb * N + pt) * OVC + v;
    V Q[QN];
#pragma unroll
    for (int j = 0; j < QN; j++) Q[j] = T::zero();
    ObsAcc<P> oa;
    R ve = R(0);
    int r0 = 0, r1 = 0;
    LastOperands<P> lop;
    lop.hi = lop.lo = lop.t1 = lop.t2 = T::zero();
    auto prefetch = [&](bool valid) {
      if (own && valid) {
        ve = reinterpret_cast<const R *>(p.veff)[pt];
        if (p.rowptr) { r0 = __ldg(p.rowptr + pt); r1 = __ldg(p.rowptr + pt + 1); }
        if (MODE == MODE_LAST) load_last<P>(p, idx, lop);
      }
    };
    prefetch(true);

    // one plane load; RQ = compile-time slot of the arriving plane in the queue
    int l = 0;
    bool aborted = false;
    auto iteration = [&](auto rq) {
      constexpr int RQ = decltype(rq)::value;
      const int slot = (int)(g & (S - 1));
      if (!mbar_wait_bounded(&full[slot], (uint32_t)((g / S) & 1))) s_abort = 1;
      Q[RQ] = ring[(size_t)slot * G::PLANE + csl];
      if (l >= 2 * M) {
        const V *Sp = ring + (size_t)((g - M) & (S - 1)) * G::PLANE;
        V gax[3];
        constexpr int QB = (RQ + 1) % QN;  // oldest entry = plane z - M
        V acc = stencil_point<M, P, 0, QB>(p, W, w0, Q, Sp, csl, G::SX * OVC, ve, false, false, gax);
        if (own && r1 > r0) acc = kb_scatter<P, 0>(p, kb, kidx, v, r0, r1, acc);
        const V c0 = Q[(QB + M) % QN];
        if (MODE == MODE_FIRST && p.do_obs && own) oa.add_e(c0, acc);
        const LastOperands<P> cur = lop;
        const long cidx = idx;
        pt += plane_pts;
        idx += plane_pts * OVC;
        prefetch(l + 1 < nl);
        finish_point<P, MODE>(p, own, cidx, v, kidx, c0, acc, cur);
      }
      __syncthreads();
      if (s_abort) {
        aborted = true;
        return;
      }
      if (tid == 0 && g >= M) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_next();
      }
      g++;
      l++;
    };
    int rq = 0;
    while (l < nl && !aborted) {
      switch (rq) {
        case 0: iteration(std::integral_constant<int, 0>{}); break;
        case 1: iteration(std::integral_constant<int, 1>{}); break;
        case 2: iteration(std::integral_constant<int, 2>{}); break;
        case 3: iteration(std::integral_constant<int, 3>{}); break;
        case 4: iteration(std::integral_constant<int, 4 % QN>{}); break;
        case 5: iteration(std::integral_constant<int, 5 % QN>{}); break;
        case 6: iteration(std::integral_constant<int, 6 % QN>{}); break;
        case 7: iteration(std::integral_constant<int, 7 % QN>{}); break;
        case 8: iteration(std::integral_constant<int, 8 % QN>{}); break;
      }
      rq = rq + 1 == QN ? 0 : rq + 1;
    }
    if (aborted) {
      if (tid == 0) {
        atomicExch(p.err, 1);
        for (long j = g; j < issued; j++) mbar_wait_bounded(&full[j & (S - 1)], (uint32_t)((j / S) & 1));
      }
      return;
    }
    if (MODE == MODE_FIRST && p.do_obs) reduce_obs<P, NT>(p, oa, item, kidx, red);
  }
}

bool tma_supported(int M, int tx, int ty) { return (M == 2 || M == 4) && tx == 16 && ty == 8; }

template <int M, int P, int MODE, int TX, int TY>
static cudaError_t launch_tma_t(const void *tmap, const SweepParams &p, int grid, cudaStream_t s) {
  typedef TmaGeom<M, TX, TY> G;
  auto k = tma_sweep_kernel<M, P, MODE, TX, TY>;
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

template <int M, int P>
static cudaError_t tma_by_mode(int mode, const void *tmap, const SweepParams &p, int grid, cudaStream_t s) {
  switch (mode) {
    case MODE_FIRST: return launch_tma_t<M, P, MODE_FIRST, 16, 8>(tmap, p, grid, s);
    case MODE_MID: return launch_tma_t<M, P, MODE_MID, 16, 8>(tmap, p, grid, s);
    case MODE_LAST: return launch_tma_t<M, P, MODE_LAST, 16, 8>(tmap, p, grid, s);
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
