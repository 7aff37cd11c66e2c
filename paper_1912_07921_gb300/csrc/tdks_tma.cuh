// Shared pieces of the TMA-fed stencil sweeps: mbarrier and bulk-tensor-copy wrappers,
// the ring geometry, work sources (one system or a batch), the producer's load cursors
// and the warp-specialised sweep body, whose tile shape (rows of 16 points, points per
// consumer thread, consumer warps) is a template parameter so that each shape can be
// compiled in a translation unit of its own.
#pragma once
#include <cuda.h>

#include <type_traits>

#include "tdks_internal.cuh"
#include "tdks_sweep_common.cuh"

namespace tdks {

namespace {

constexpr long long WAIT_LIMIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz
constexpr long long DRAIN_LIMIT_CYCLES = 200000000LL;  // ~0.1 s per copy on the error path

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
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long limit = WAIT_LIMIT_CYCLES) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 16-byte asynchronous global -> shared copy (L2 only), and an arrive on an mbarrier that
// fires once every cp.async this thread has issued so far has landed (the barrier's pending
// count is raised by one at issue, so its expected count stays as initialised).
__device__ __forceinline__ void cp_async_16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar) {
  asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Consumer wait: bounded, and gives up at once when another warp has given up.  (Reading
// the abort flag only every 16 polls, or taking the bound from shared memory, measured 1-3%
// slower sweeps: the flag's load paces the polling.)
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity, const volatile int *abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > WAIT_LIMIT_CYCLES) return false;
  }
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

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *tmap, uint64_t *bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
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

// Position in a ring of S slots: slot index and the parity of the slot's current use.
struct RingPos {
  int slot = 0;
  uint32_t phase = 0;
  template <int S>
  __device__ __forceinline__ void next() {
    if (++slot == S) {
      slot = 0;
      phase ^= 1u;
    }
  }
};

// Shared-memory plan: three TMA-fed rings, each slot completed by one mbarrier.
//   centre ring (SC slots): U planes of the input tile (no halo), which feed the per-thread
//     register z-queue; a slot is free again as soon as its planes are in registers;
//   halo ring (SH slots): U output planes of the input with their x/y halo, followed by the
//     U planes' per-point records; read when those planes are computed;
//   operand ring (SO slots, last Taylor term only): the four own-point operand tiles of one
//     output plane (state hi, state lo, t1, t2).
// Keeping the z history in registers (not in the ring) lets every ring run several slots
// ahead of the plane being computed.
//   periodic cells (BL): each halo slot also holds the four periodic-image strips a boundary
//     tile needs (the M columns beyond each x face over the slot's SY rows, the M rows beyond
//     each y face over the tile's TX columns), loaded by TMA from the opposite faces, and (first
//     Taylor term) the non-local rows of the plane's sphere points (one per point, in tile
//     order), which the patcher warp copies in with cp.async so that no consumer waits on a
//     global load.
template <int M, int TX, int TY, int U, bool OPS, bool BL = false, bool NLG = false>
struct TmaGeom {
  static constexpr int SX = TX + 2 * M, SY = TY + 2 * M;
  static constexpr int PLANE = SX * SY * OVC;                        // vectors per halo plane
  static constexpr int CPLANE = TX * TY * OVC;                       // vectors per centre plane
  static constexpr uint32_t CSLOT_BYTES = (uint32_t)CPLANE * 16 * U;
  static constexpr uint32_t IN_BYTES = (uint32_t)PLANE * 16 * U;
  static constexpr uint32_t AUX_BYTES = (uint32_t)TX * TY * 16 * U;
  static constexpr uint32_t STRIPX_BYTES = (uint32_t)M * SY * OVC * 16;   // beyond x = 0 or x = nx - 1
  static constexpr uint32_t STRIPY_BYTES = (uint32_t)TX * M * OVC * 16;   // beyond y = 0 or y = ny - 1
  static constexpr uint32_t STRIP_BYTES = BL ? 2 * (STRIPX_BYTES + STRIPY_BYTES) : 0;
  static constexpr uint32_t OPT_BYTES = (uint32_t)CPLANE * 16;       // one operand tile
  static constexpr uint32_t OP_BYTES = 4 * OPT_BYTES;
  static constexpr int SO = OPS ? 2 : 0;
  // (the last term's 4 operand tiles leave taller tiles room for few centre slots)
  static constexpr int SC = U == 1 ? (OPS ? (TX * TY > 128 ? 2 : 4) : 6) : 4;
  static constexpr size_t BUDGET = 227 * 1024 - 2048;                // dynamic smem available
  static constexpr size_t HALO_ROOM = BUDGET - 128 - (size_t)SO * OP_BYTES - (size_t)SC * CSLOT_BYTES;
  // periodic cells, first Taylor term (NLG): the non-local rows of the plane's sphere points,
  // gathered into the slot by the patcher warp, where two slots still fit (else the consumers
  // load them).  (The larger slot leaves fewer halo slots: the faster middle and last sweeps
  // measured slower with it, the first sweep, with its current gradients, faster.)
  static constexpr uint32_t NL_STAGE = (uint32_t)TX * TY * OVC * 16;
  static constexpr bool NLS = BL && NLG && HALO_ROOM / (IN_BYTES + AUX_BYTES + STRIP_BYTES + NL_STAGE) >= 2;
  static constexpr uint32_t NL_BYTES = NLS ? NL_STAGE : 0;
  static constexpr uint32_t HSLOT_BYTES = IN_BYTES + AUX_BYTES + STRIP_BYTES + NL_BYTES;
  static_assert(!BL || U == 1, "periodic cells take one plane per iteration");
  static constexpr int SH_FIT = (int)(HALO_ROOM / HSLOT_BYTES);
  static constexpr int SH = SH_FIT < 8 ? SH_FIT : 8;
  static constexpr size_t SMEM = (size_t)SC * CSLOT_BYTES + (size_t)SH * HSLOT_BYTES + (size_t)SO * OP_BYTES + 128;
  static_assert(SH >= 2, "halo ring too small");
};

// Work sources: a single system (parameters and tensor maps are kernel parameters), or a
// batch of systems (per-system parameters and tensor maps in device arrays; a CTA stages
// the parameters of its current item in shared memory).
struct SingleSrc {
  const SweepParams *p;
  const SweepMaps *maps;
  __device__ __forceinline__ long n_items() const { return p->n_items; }
  __device__ __forceinline__ void item(long it, const SweepParams *&pp, const SweepMaps *&mp, long &local) const {
    pp = p;
    mp = maps;
    local = it;
  }
  __device__ __forceinline__ int sys_of(long) const { return 0; }
  __device__ __forceinline__ const SweepMaps *maps_of(int) const { return maps; }
  __device__ __forceinline__ int *err0() const { return p->err; }
  __device__ __forceinline__ bool withhold() const { return p->withhold != 0; }
};

// (the system of an item comes from a table: one load where a binary search over the systems'
// item ranges took a chain of them at the start of every item, in every warp)
struct BatchSrc {
  const BatchSweepArgs *a;
  __device__ __forceinline__ long n_items() const { return a->total_items; }
  __device__ __forceinline__ void item(long it, const SweepParams *&pp, const SweepMaps *&mp, long &local) const {
    const int s = a->item_sys[it];
    pp = a->params + s;
    mp = a->maps + 4 * s + a->which;
    local = it - a->item_begin[s];
  }
  __device__ __forceinline__ int sys_of(long it) const { return a->item_sys[it]; }
  __device__ __forceinline__ const SweepMaps *maps_of(int s) const { return a->maps + 4 * s + a->which; }
  __device__ __forceinline__ int *err0() const { return a->params[0].err; }
  __device__ __forceinline__ bool withhold() const { return a->params[0].withhold != 0; }
};

// Sequential cursor over one kind of load of the CTA's items (thread 0 only).  The item's
// geometry is decoded once, when the cursor enters the item, so issuing a load costs a few
// instructions: the other threads wait for thread 0 at the next barrier.
struct LoadCursor {
  long ii;     // item index among the CTA's items (-1: not entered yet)
  int l;       // load index within the item
  int n;       // loads of this kind in the item
  int tx, ty, kb, z0;
  int sys;     // system of the item (batch)
  long issued; // loads issued so far
  int nx, ny, nz, wrap;  // periodic cell: centre planes outside [0, nz) are loaded wrapped, and
                         // the halo slots of boundary tiles get their periodic-image strips
};

// floor(i / n) for possibly negative i
__device__ __forceinline__ int floordiv_i(int i, int n) { return i >= 0 ? i / n : -((-i - 1) / n) - 1; }

// Work item -> tile (tx, ty), orbital block kb and z chunk [z0, z1).
__device__ __forceinline__ void item_geom(const SweepParams &q, long it, int &tx, int &ty, int &kb, int &z0,
                                          int &z1) {
  // z chunks fastest: consecutive items are the chunks of one column, which run at about the
  // same time on different SMs and share the planes at their boundaries through L2
  z0 = (int)(it % q.n_zc) * q.zc;
  it /= q.n_zc;
  tx = (int)(it % q.n_tx);
  it /= q.n_tx;
  ty = (int)(it % q.n_ty);
  it /= q.n_ty;
  kb = (int)it;
  z1 = min(z0 + q.zc, q.nz);
}

// Loads per item: 0 = centre (queue planes z0-M .. z1+M-1, U per load), 1 = halo (output
// planes, U per load), 2 = operands (one per output plane).
template <int M, int U>
__device__ __forceinline__ int loads_of(int kind, int z0, int z1) {
  if (kind == 0) return (z1 - z0 + 2 * M + U - 1) / U;
  if (kind == 1) return (z1 - z0 + U - 1) / U;
  return z1 - z0;
}

// The producer side of the rings (thread 0 only).
template <int M, int TX, int TY, int U, class G, int SC, int SH, int SO, class Src>
struct Loader {
  Src src;
  long n_my;
  unsigned char *cbase, *hbase, *obase;
  uint64_t *cfull, *hfull, *ofull;

  // move the cursor onto its next load (decoding the geometry of an item it enters)
  __device__ __forceinline__ void advance(LoadCursor &c, int kind) const {
    while (c.ii < n_my && (c.ii < 0 || c.l >= c.n)) {
      c.ii += 1;
      c.l = 0;
      c.n = 0;
      if (c.ii < n_my) {
        const SweepParams *qp = nullptr;
        const SweepMaps *mq = nullptr;
        long local = 0;
        src.item(blockIdx.x + c.ii * gridDim.x, qp, mq, local);
        int z1 = 0;
        item_geom(*qp, local, c.tx, c.ty, c.kb, c.z0, z1);
        c.sys = src.sys_of(blockIdx.x + c.ii * gridDim.x);
        c.n = loads_of<M, U>(kind, c.z0, z1);
        c.nx = qp->nx;
        c.ny = qp->ny;
        c.nz = qp->nz;
        c.wrap = qp->bloch;
      }
    }
  }

  // issue the next load of `kind`; nothing past the CTA's last item
  __device__ __forceinline__ void issue(LoadCursor &c, int kind) const {
    advance(c, kind);
    if (c.ii >= n_my) return;
    emit(c, kind);
  }

  // issue the load the cursor is positioned on
  __device__ __forceinline__ void emit(LoadCursor &c, int kind) const {
    const SweepMaps *mp = src.maps_of(c.sys);
    if (kind == 0) {
      const int slot = (int)(c.issued % SC);
      mbar_expect_tx(&cfull[slot], G::CSLOT_BYTES);
      int zc = c.z0 - M + U * c.l;
      if (c.wrap) zc -= floordiv_i(zc, c.nz) * c.nz;  // (U = 1 for periodic cells)
      tma_load_5d(cbase + (size_t)slot * G::CSLOT_BYTES, &mp->ctr, &cfull[slot], 0, c.tx * TX, c.ty * TY, zc,
                  c.kb);
    } else if (kind == 1) {
      const int slot = (int)(c.issued % SH);
      unsigned char *dst = hbase + (size_t)slot * G::HSLOT_BYTES;
      const int zp = c.z0 + U * c.l;
      const int x0 = c.tx * TX, y0 = c.ty * TY;
      // periodic cell: the strips this tile's halo crosses (the slot holds zeros there)
      const bool sl = G::STRIP_BYTES && c.wrap && x0 - M < 0, sr = G::STRIP_BYTES && c.wrap && x0 + TX + M > c.nx;
      const bool st = G::STRIP_BYTES && c.wrap && y0 - M < 0, sb = G::STRIP_BYTES && c.wrap && y0 + TY + M > c.ny;
      const uint32_t bytes = G::IN_BYTES + G::AUX_BYTES + (uint32_t)(sl + sr) * G::STRIPX_BYTES +
                             (uint32_t)(st + sb) * G::STRIPY_BYTES;
      mbar_expect_tx(&hfull[slot], bytes);
      tma_load_5d(dst, &mp->in, &hfull[slot], 0, x0 - M, y0 - M, zp, c.kb);
      tma_load_4d(dst + G::IN_BYTES, &mp->aux, &hfull[slot], 0, x0, y0, zp);
      if constexpr (G::STRIP_BYTES > 0) {
        unsigned char *sd = dst + G::IN_BYTES + G::AUX_BYTES;
        if (sl) tma_load_5d(sd, &mp->sx, &hfull[slot], 0, c.nx - M, y0 - M, zp, c.kb);
        if (sr) tma_load_5d(sd + G::STRIPX_BYTES, &mp->sx, &hfull[slot], 0, 0, y0 - M, zp, c.kb);
        if (st) tma_load_5d(sd + 2 * G::STRIPX_BYTES, &mp->sy, &hfull[slot], 0, x0, c.ny - M, zp, c.kb);
        if (sb) tma_load_5d(sd + 2 * G::STRIPX_BYTES + G::STRIPY_BYTES, &mp->sy, &hfull[slot], 0, x0, 0, zp, c.kb);
      }
    } else {
      const int slot = (int)(c.issued % SO);
      unsigned char *dst = obase + (size_t)slot * G::OP_BYTES;
      mbar_expect_tx(&ofull[slot], G::OP_BYTES);
      for (int j = 0; j < 4; j++)
        tma_load_5d(dst + j * G::OPT_BYTES, &mp->op[j], &ofull[slot], 0, c.tx * TX, c.ty * TY, c.z0 + c.l, c.kb);
    }
    c.issued++;
    c.l++;
  }
};

// ---------------------------------------------------------------------------------------
// Warp-specialised variant: one producer warp keeps the three rings full, CW consumer
// warps compute.  A ring slot is handed back by an "empty" mbarrier that each consumer
// warp arrives on once it has read the slot, so the consumer warps never wait for one
// another inside a work item: while some warps read their shared-memory neighbours,
// others do arithmetic or store.  Each consumer thread computes one 16-byte vector of R
// y-adjacent points, which share the y-column values they read (R points need 2M+R column
// loads instead of 2M R).
//
// Shapes (tile TX x TY points of one orbital block; R y-adjacent points per consumer
// thread; CW = 4 TX TY / (32 R) consumer warps, plus the producer warp).  More points per
// thread share more y-column loads and give each warp more independent arithmetic; more
// warps hide more latency.  The register budget of a thread is set by the warps that share
// one of the SM's four scheduler partitions (16K registers each): 7 or 8 warps in all leave
// 255 registers per thread, 9 leave 168, 13 leave 128, 17 leave 96.  tdks_autotune times
// the shapes on the system's own data.
//
// Shape 5 computes complex64 systems with one complex value per thread vector (8 bytes, 8
// vectors per point, P_C64S): at the same register budget a thread then holds the z queues
// of 4 y-adjacent points, which share their y-column loads, while a warp still spans 4
// consecutive points in x (conflict-free 256-byte shared loads).  Per output value that is
// 2M x-arm loads, 2M/4 y-arm loads and one queue load of 8 bytes, against 2M, (2M+2)/2 and
// one of 16 bytes for two values in the two-complex shapes: about a third fewer shared-memory
// bytes per value.  Complex128 systems and periodic cells run shape 5 as shape 2.
template <int SHAPE> struct WsShape;
template <> struct WsShape<0> { static constexpr int TX = 16, TY = 8, R = 2; };   //  8 consumer warps
template <> struct WsShape<1> { static constexpr int TX = 16, TY = 12, R = 4; };  //  6
template <> struct WsShape<2> { static constexpr int TX = 16, TY = 12, R = 2; };  // 12
template <> struct WsShape<3> { static constexpr int TX = 16, TY = 8, R = 1; };   // 16
template <> struct WsShape<4> { static constexpr int TX = 14, TY = 8, R = 2; };   //  7
template <> struct WsShape<5> { static constexpr int TX = 16, TY = 12, R = 4; };  // 12 (complex64, 8-byte vectors)
template <int TX, int TY, int R, int OV = OVC> struct WsWarps {
  static constexpr int CW = OV * TX * TY / (32 * R);       // consumer warps
  static constexpr int THREADS = 32 * CW + 32;             // + the producer warp
  // consumer thread t owns vector t % OV of point (t / OV) % TX of row group t / (OV TX), whose
  // R rows are y-adjacent: the row groups must fill the tile and the warps exactly
  static_assert(TY % R == 0 && CW * 32 == OV * TX * (TY / R), "row groups must fill the tile and the warps");
};

// H at R y-adjacent points (rows 0 .. R-1) of one plane, from their z queues Q[r] and
// the halo plane Sp (row 0's own vector at hs0, row stride SXO vectors).  Same terms and
// summation order as stencil_point.
template <int M, int P, int QB, int QN, int R>
__device__ __forceinline__ void stencil_rows(const typename VT<P>::S *W, typename W0T<P>::type w0,
                                             const typename VT<P>::V (*Q)[QN], const typename VT<P>::V *Sp, int hs0,
                                             int SXO, const typename VT<P>::R *ve, typename VT<P>::V *acc) {
  typedef VT<P> T;
  typedef typename T::V V;
  V col[2 * M + R];  // Sp[hs0 + k SXO], k = -M .. M+R-1
#pragma unroll
  for (int k = 0; k < 2 * M + R; k++) col[k] = Sp[hs0 + (k - M) * SXO];
#pragma unroll
  for (int r = 0; r < R; r++) acc[r] = T::mul(T::diag(ve[r], w0), Q[r][(QB + M) % QN]);
#pragma unroll
  for (int m = 1; m <= M; m++) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int hr = hs0 + r * SXO;
      const V s = T::add(T::add(T::add(Q[r][(QB + M - m) % QN], Q[r][(QB + M + m) % QN]),
                                T::add(Sp[hr - m * T::OV], Sp[hr + m * T::OV])),
                         T::add(col[M + r - m], col[M + r + m]));
      acc[r] = T::fma(W[m], s, acc[r]);
    }
  }
}

// Bloch phase of one wrap, e^{i ang} = c + i s, in the compute precision.
template <int P>
__device__ __forceinline__ void bloch_phase(double ang, typename VT<P>::S &c, typename VT<P>::S &s) {
  if constexpr (P == P_C64) {
    float sn, cs;
    sincosf((float)ang, &sn, &cs);
    c = pk2(cs, cs);
    s = pk2(sn, sn);
  } else {
    double sn, cs;
    sincos(ang, &sn, &cs);
    c = cs;
    s = sn;
  }
}
// a times the phase of w wraps, (c + i s)^w (w = +-1 except in grids smaller than the stencil)
template <int P>
__device__ __forceinline__ typename VT<P>::V apply_phase(typename VT<P>::S c, typename VT<P>::S s, int w,
                                                         typename VT<P>::V a) {
  typedef VT<P> T;
  if (w < 0) {
    if constexpr (P == P_C64) s ^= SIGN2; else s = -s;
  }
  for (int i = w < 0 ? -w : w; i > 0; i--) a = T::cmul(c, s, a);
  return a;
}

// Periodic (Bloch) cell: as stencil_rows, with the velocity-gauge gradient term -i A.grad_h
// (and, for the current, the three gradients gax) in the order of stencil_point.  The halo
// slot S already holds the phased periodic images beyond the faces (the patcher warp wrote
// them), so the neighbours are read as in a finite box.
template <int M, int P, int QB, int QN, int R>
__device__ __forceinline__ void stencil_rows_bloch(const SweepParams &p, const typename VT<P>::S *W,
                                                   typename W0T<P>::type w0, const typename VT<P>::V (*Q)[QN],
                                                   const typename VT<P>::V *S, int hs0, int SXO,
                                                   const typename VT<P>::R *ve, typename VT<P>::V *acc,
                                                   typename VT<P>::V (*gax)[3], bool need_grad, bool grads) {
  typedef VT<P> T;
  typedef typename T::V V;
  V col[2 * M + R];  // y = gy0 - M + k
#pragma unroll
  for (int k = 0; k < 2 * M + R; k++) col[k] = S[hs0 + (k - M) * SXO];
  // gradient term as sum_m gw_m (A . d_m): 3 + M coefficients live instead of 3 M
  typename T::S A3[3] = {};
  if (need_grad) {
#pragma unroll
    for (int a = 0; a < 3; a++) A3[a] = T::bc(p.A[a]);
  }
  V gsum[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    acc[r] = T::mul(T::diag(ve[r], w0), Q[r][(QB + M) % QN]);
    gsum[r] = T::zero();
    gax[r][0] = gax[r][1] = gax[r][2] = T::zero();
  }
#pragma unroll
  for (int m = 1; m <= M; m++) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const V xm = S[hs0 + r * SXO - m * T::OV], xp = S[hs0 + r * SXO + m * T::OV];
      const V zm = Q[r][(QB + M - m) % QN], zp = Q[r][(QB + M + m) % QN];
      const V ym = col[M + r - m], yp = col[M + r + m];
      const V s6 = T::add(T::add(T::add(zm, zp), T::add(xm, xp)), T::add(ym, yp));
      acc[r] = T::fma(W[m], s6, acc[r]);
      if (need_grad) {
        const V dx = T::sub(xp, xm), dy = T::sub(yp, ym), dz = T::sub(zp, zm);
        const typename T::S gm = T::bc(p.gw[m]);
        const V dA = T::fma(A3[0], dx, T::fma(A3[1], dy, T::mul(A3[2], dz)));
        gsum[r] = T::fma(gm, dA, gsum[r]);
        if (grads) {
          gax[r][0] = T::fma(gm, dx, gax[r][0]);
          gax[r][1] = T::fma(gm, dy, gax[r][1]);
          gax[r][2] = T::fma(gm, dz, gax[r][2]);
        }
      }
    }
  }
  if (need_grad) {
#pragma unroll
    for (int r = 0; r < R; r++) acc[r] = T::add(acc[r], T::negi(gsum[r]));
  }
}

template <int M, int P, int MODE, int TX, int TY, int R, int U, bool BATCH, int BLOCH, class Src>
__device__ __forceinline__ void ws_sweep_body(const Src &src, unsigned int *work) {
  typedef VT<P> T;
  typedef typename T::V V;
  typedef typename T::S S_;
  typedef typename T::R Rv;
  constexpr bool OPS = MODE == MODE_LAST;
  typedef TmaGeom<M, TX, TY, U, OPS, BLOCH != 0, MODE == MODE_FIRST> G;
  static_assert(M % U == 0, "M must be a multiple of U");
  static_assert(!OPS || U == 1, "the last Taylor term takes one plane per iteration");
  constexpr int OV = T::OV;       // thread vectors per (point, batch)
  constexpr int CPL = TX * TY * OV;  // thread vectors per centre plane or operand tile
  constexpr int CW = WsWarps<TX, TY, R, OV>::CW;
  constexpr int SC = G::SC, SH = G::SH;
  constexpr int SO = G::SO > 0 ? G::SO : 1;
  constexpr int QN = 2 * M + U;   // z-queue entries
  constexpr int LP = 2 * M / U;   // priming centre loads per item
  constexpr int IR = 16;          // claimed-item ring (the producer runs at most a few items ahead)
  extern __shared__ unsigned char smem_raw[];
  unsigned char *cbase = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  unsigned char *hbase = cbase + (size_t)SC * G::CSLOT_BYTES;
  unsigned char *obase = hbase + (size_t)SH * G::HSLOT_BYTES;
  __shared__ __align__(8) uint64_t cfull[SC], cempty[SC];
  __shared__ __align__(8) uint64_t hfull[SH], hempty[SH];
  __shared__ __align__(8) uint64_t hready[BLOCH ? SH : 1];  // periodic cells: face images written
  __shared__ __align__(8) uint64_t ofull[SO], oempty[SO];
  __shared__ __align__(8) uint64_t ibar[IR];  // completes when s_item[seq % IR] is written
  __shared__ long s_item[IR];                 // item of the CTA's seq-th claim (-1: no more)
  __shared__ int s_abort;
  volatile int *abort_flag = &s_abort;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const long n_items_all = src.n_items();

  if (tid == 0) {
    for (int s = 0; s < SC; s++) { mbar_init(&cfull[s], 1); mbar_init(&cempty[s], CW); }
    for (int s = 0; s < SH; s++) { mbar_init(&hfull[s], 1); mbar_init(&hempty[s], CW); }
    if (BLOCH)
      for (int s = 0; s < SH; s++) mbar_init(&hready[s], 1);
    for (int s = 0; s < SO; s++) { mbar_init(&ofull[s], 1); mbar_init(&oempty[s], CW); }
    for (int s = 0; s < IR; s++) mbar_init(&ibar[s], 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();  // the only CTA-wide barrier: from here on the warps run decoupled

  if (warp == CW) {
    // ---- producer: claim items, and issue every ring's loads as soon as a slot is free ----
    // (failure injection: a withholding producer does nothing, so the other warps' waits
    // run out; no copy is in flight and nothing needs draining)
    if (lane == 0 && !src.withhold()) {
      const Loader<M, TX, TY, U, G, SC, SH, SO, Src> ld{src, 0, cbase, hbase, obase, cfull, hfull, ofull};
      LoadCursor c[3];
      bool done[3] = {false, false, !OPS};
      for (int k = 0; k < 3; k++) c[k] = LoadCursor{-1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      long claimed = 0;  // claims made (their items are in s_item)
      // position cursor k on its next load; false if it has none yet (or none at all)
      auto position = [&](int k) -> bool {
        LoadCursor &cu = c[k];
        while (!done[k] && cu.l >= cu.n) {
          const long ns = cu.ii + 1;
          if (ns >= claimed) {
            if (k != 0) return false;  // the centre cursor, always ahead, makes the claims
            const unsigned int t = atomicAdd(work, 1u);
            // every CTA ends with one claim past the last item: the launch's last claim
            // returns the counter to zero for the next launch
            if ((long)t == n_items_all + (long)gridDim.x - 1) atomicExch(work, 0u);
            s_item[claimed % IR] = (long)t < n_items_all ? (long)t : -1;
            mbar_arrive(&ibar[claimed % IR]);
            claimed++;
          }
          const long it = s_item[ns % IR];
          if (it < 0) {
            done[k] = true;
            break;
          }
          const SweepParams *qp = nullptr;
          const SweepMaps *mq = nullptr;
          long local = 0;
          src.item(it, qp, mq, local);
          int z1 = 0;
          item_geom(*qp, local, cu.tx, cu.ty, cu.kb, cu.z0, z1);
          cu.sys = src.sys_of(it);
          cu.ii = ns;
          cu.l = 0;
          cu.n = loads_of<M, U>(k, cu.z0, z1);
          cu.nx = qp->nx;
          cu.ny = qp->ny;
          cu.nz = qp->nz;
          cu.wrap = qp->bloch;
        }
        return !done[k];
      };
      long long idle_since = clock64();
      for (;;) {
        bool left = false, progressed = false;
#pragma unroll
        for (int k = 0; k < 3; k++) {
          if (done[k]) continue;
          left = true;
          if (!position(k)) continue;
          const int S = k == 0 ? SC : (k == 1 ? SH : SO);
          uint64_t *empty = k == 0 ? cempty : (k == 1 ? hempty : oempty);
          const long n = c[k].issued;
          // slot n % S is free once the consumers have released its previous use
          if (n >= S && !mbar_test(&empty[n % S], (uint32_t)(((n / S) - 1) & 1))) continue;
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          ld.emit(c[k], k);
          progressed = true;
        }
        if (!left) break;
        if (progressed) {
          idle_since = clock64();
        } else {
          if (*abort_flag || clock64() - idle_since > WAIT_LIMIT_CYCLES) {
            *abort_flag = 1;
            break;
          }
          __nanosleep(32);
        }
      }
      // copies still in flight must land before the CTA's shared memory goes away
      for (int k = 0; k < 3; k++) {
        if (k == 2 && !OPS) continue;
        const int S = k == 0 ? SC : (k == 1 ? SH : SO);
        uint64_t *full = k == 0 ? cfull : (k == 1 ? hfull : ofull);
        const long n = c[k].issued;
        for (long j = n > S ? n - S : 0; j < n; j++)
          mbar_wait_bounded(&full[j % S], (uint32_t)((j / S) & 1), DRAIN_LIMIT_CYCLES);
      }
    }
    return;
  }

  if (BLOCH && warp == CW + 1) {
    // ---- patcher (periodic cells): for each output plane of each item, once the halo slot
    // has landed, write the Bloch-phased periodic images of the strips beyond the cell's
    // x and y faces into the halo box (where the TMA box holds zeros), then release the
    // slot to the consumers -----------------------------------------------------------------
    RingPos rp;
    for (long seq = 0;; seq++) {
      if (!mbar_wait_or_abort(&ibar[seq % IR], (uint32_t)((seq / IR) & 1), abort_flag)) {
        *abort_flag = 1;
        break;
      }
      const long item = s_item[seq % IR];
      if (item < 0) break;
      const SweepParams *pp;
      const SweepMaps *mp_unused;
      long local;
      src.item(item, pp, mp_unused, local);
      const SweepParams &p = *pp;
      int tx, ty, kb, z0, z1;
      item_geom(p, local, tx, ty, kb, z0, z1);
      const int nx = p.nx, ny = p.ny, x0 = tx * TX, y0 = ty * TY;
      const bool sl = x0 - M < 0, sr = x0 + TX + M > nx, st = y0 - M < 0, sb = y0 + TY + M > ny;
      const int kidx = kb / p.n_batches;
      S_ cx, sx, cy, sy;
      bloch_phase<P>(p.kvec[3 * kidx] * p.L[0], cx, sx);
      bloch_phase<P>(p.kvec[3 * kidx + 1] * p.L[1], cy, sy);
      constexpr int VB = (int)sizeof(V);  // bytes per thread vector
      constexpr int SLB = (int)((G::IN_BYTES + G::AUX_BYTES) / VB);
      constexpr int SRB = SLB + (int)(G::STRIPX_BYTES / VB);
      constexpr int STB = SRB + (int)(G::STRIPX_BYTES / VB);
      constexpr int SBB = STB + (int)(G::STRIPY_BYTES / VB);
      bool gave_up = false;
      for (int z = z0; z < z1; z++) {
        const int hs = rp.slot;
        if (!mbar_wait_or_abort(&hfull[hs], rp.phase, abort_flag)) {
          gave_up = true;
          break;
        }
        V *box = reinterpret_cast<V *>(hbase + (size_t)hs * G::HSLOT_BYTES);
        if (sl || sr) {
          // box columns c with grid x = x0 - M + c beyond x = 0 (c < M) or beyond x = nx - 1
          const int cr0 = nx - x0 + M;  // first box column past the last grid column
          for (int i = lane; i < 2 * G::SY * M * OV; i += 32) {
            const int v = i % OV, j = (i / OV) % M, row = (i / (OV * M)) % G::SY, side = i / (OV * M * G::SY);
            if (side == 0 ? !sl : !sr) continue;
            const int c = side == 0 ? j : cr0 + j;
            if (c >= G::SX) continue;
            const V a = box[(side == 0 ? SLB : SRB) + (row * M + j) * OV + v];
            box[(row * G::SX + c) * OV + v] = apply_phase<P>(cx, sx, side == 0 ? -1 : 1, a);
          }
        }
        if (st || sb) {
          // box rows rr with grid y = y0 - M + rr beyond y = 0 (rr < M) or beyond y = ny - 1,
          // over the tile's columns (the star stencil never reads the corners)
          const int rb0 = ny - y0 + M;
          for (int i = lane; i < 2 * M * TX * OV; i += 32) {
            const int v = i % OV, c = (i / OV) % TX, j = (i / (OV * TX)) % M, side = i / (OV * TX * M);
            if (side == 0 ? !st : !sb) continue;
            const int rr = side == 0 ? j : rb0 + j;
            if (rr >= G::SY) continue;
            const V a = box[(side == 0 ? STB : SBB) + (j * TX + c) * OV + v];
            box[(rr * G::SX + c + M) * OV + v] = apply_phase<P>(cy, sy, side == 0 ? -1 : 1, a);
          }
        }
        if (G::NLS && p.has_proj) {
          // the plane's non-local rows: row r0 of each sphere point (points outside every
          // sphere are never read from here)
          const PointAux *ax = reinterpret_cast<const PointAux *>(hbase + (size_t)hs * G::HSLOT_BYTES + G::IN_BYTES);
          V *nla = box + (G::IN_BYTES + G::AUX_BYTES + G::STRIP_BYTES) / VB;
          const V *nlk = reinterpret_cast<const V *>(p.nl) + (long)kb * (p.n_ent + 1) * OV;
          for (int i = lane; i < TX * TY * OV; i += 32) {
            const PointAux a = ax[i / OV];
            if (a.r1 > a.r0) cp_async_16(nla + i, nlk + (long)a.r0 * OV + i % OV);
          }
          cp_async_arrive(&hready[hs]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&hready[hs]);
        rp.next<SH>();
      }
      if (gave_up) {
        *abort_flag = 1;
        break;
      }
    }
    cp_async_wait_all();  // no copy may land after the CTA's shared memory is gone
    return;
  }

  // ---- consumers: no barrier between warps; a warp that gives up stops, and the others
  // give up at their next wait ----------------------------------------------------------------
  const int v = tid % OV;
  const int lx = (tid / OV) % TX;
  const int ly0 = R * (tid / (OV * TX));
  const int hs0 = ((ly0 + M) * G::SX + (lx + M)) * OV + v;   // row 0's vector in a halo plane
  const int tsl0 = ly0 * TX + lx;                             // row 0's point in a tile
  const int csl0 = tsl0 * OV + v;                             // row 0's vector in a centre plane
  constexpr int SXO = G::SX * OV;

  RingPos rc, rh, ro;  // ring positions of the next centre / halo / operand load
  bool aborted = false;
  int *errp = src.err0();  // then the current item's system's
  for (long seq = 0;; seq++) {
    if (!mbar_wait_or_abort(&ibar[seq % IR], (uint32_t)((seq / IR) & 1), abort_flag)) {
      aborted = true;
      break;
    }
    const long item = s_item[seq % IR];
    if (item < 0) break;
    const SweepParams *pp;
    const SweepMaps *mp_unused;
    long local;
    src.item(item, pp, mp_unused, local);
    const SweepParams &p = *pp;  // (batch: read from the parameter array, once per item)
    errp = p.err;
    const int nx = p.nx, ny = p.ny;
    const long N = (long)nx * ny * p.nz;
    const long plane_pts = (long)nx * ny;
    S_ W[M + 1];
#pragma unroll
    for (int m = 0; m <= M; m++) W[m] = T::coef(p.w[m], p.wf[m]);
    const typename W0T<P>::type w0 = P != P_C128 ? (typename W0T<P>::type)p.wf[0] : (typename W0T<P>::type)p.w[0];
    const S_ CR = T::coef(p.cr, p.crf), CI = T::coef(p.ci, p.cif);
    int tx, ty, kb, z0, z1;
    item_geom(p, local, tx, ty, kb, z0, z1);
    const int kidx = kb / p.n_batches;
    const Epi epi = make_epi(p, kidx);
    const bool has_proj = p.has_proj != 0, do_obs = p.do_obs != 0;
    const V *nlk = nl_column<P>(p, kb, v);
    const int n_ent = p.n_ent;
    const int gx = tx * TX + lx, gy0 = ty * TY + ly0;
    // periodic cell: the Bloch phase of one wrap along z, e^{i k_z L_z} = cz + i sz, applied to
    // the queue planes loaded from beyond a z face (the patcher warp handles x and y)
    S_ cz{}, sz{};
    if constexpr (BLOCH) bloch_phase<P>(p.kvec[3 * kidx + 2] * p.L[2], cz, sz);
    const bool need_grad = BLOCH && p.grad_mask != 0;
    const bool grads = BLOCH && MODE == MODE_FIRST && (p.grad_mask & 8);
    bool own[R];
#pragma unroll
    for (int r = 0; r < R; r++) own[r] = gx < nx && gy0 + r < ny;
    const int nl = loads_of<M, U>(0, z0, z1);
    // vector index of row 0's point in the first output plane (advances one plane per output)
    long idx = ((long)kb * N + ((long)z0 * ny + gy0) * nx + gx) * OV + v;
    const long row = (long)nx * OV;
    V Q[R][QN];
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
      for (int j = 0; j < QN; j++) Q[r][j] = T::zero();
    ObsAcc<P> oa;

    int l = 0;
    // one centre load (and, past the priming loads, one halo load); RQ = compile-time
    // queue position of its first plane
    auto iteration = [&](auto rq) {
      constexpr int RQ = decltype(rq)::value;
      const int cs = rc.slot;
      if (!mbar_wait_or_abort(&cfull[cs], rc.phase, abort_flag)) {
        aborted = true;
        return;
      }
      const V *cslot = reinterpret_cast<const V *>(cbase + (size_t)cs * G::CSLOT_BYTES);
#pragma unroll
      for (int u = 0; u < U; u++) {
#pragma unroll
        for (int r = 0; r < R; r++) Q[r][(RQ + u) % QN] = cslot[u * CPL + csl0 + r * TX * OV];
        if constexpr (BLOCH) {
          // a plane beyond a z face was loaded from its periodic image: apply the Bloch phase
          const int zq = z0 - M + U * l + u;
          if ((unsigned)zq >= (unsigned)p.nz) {
            const int wz = floordiv_i(zq, p.nz);
#pragma unroll
            for (int r = 0; r < R; r++) Q[r][(RQ + u) % QN] = apply_phase<P>(cz, sz, wz, Q[r][(RQ + u) % QN]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&cempty[cs]);
      rc.next<SC>();
      if (l >= LP) {
        const int zf = z0 + U * (l - LP);
        const int hs = rh.slot;
        // periodic cells: the slot is ready once the patcher warp has written the face images
        if (!mbar_wait_or_abort(BLOCH ? &hready[hs] : &hfull[hs], rh.phase, abort_flag)) {
          aborted = true;
          return;
        }
        const unsigned char *hslot = hbase + (size_t)hs * G::HSLOT_BYTES;
        const V *xs = reinterpret_cast<const V *>(hslot);
        const PointAux *ax = reinterpret_cast<const PointAux *>(hslot + G::IN_BYTES);
        const V *ob = nullptr;  // last term: the operand slot, read row by row at the epilogue
        int os = 0;
        if constexpr (OPS) {
          os = ro.slot;
          if (!mbar_wait_or_abort(&ofull[os], ro.phase, abort_flag)) {
            aborted = true;
            return;
          }
          ob = reinterpret_cast<const V *>(obase + (size_t)os * G::OP_BYTES);
        }
        (void)ob;
        (void)os;
        auto operands = [&](int c) {
          LastOperands<P> o;
          if constexpr (OPS) {
            o.hi = ob[c];
            o.lo = ob[CPL + c];
            o.t1 = ob[2 * CPL + c];
            o.t2 = ob[3 * CPL + c];
          } else {
            (void)c;
            o.hi = o.lo = o.t1 = o.t2 = T::zero();
          }
          return o;
        };
        static_for<0, U>([&](auto uc) {
          constexpr int u = decltype(uc)::value;
          constexpr int QB = (RQ + U + u) % QN;  // queue position of plane (zf + u) - M
          Rv ve[R];
          V nlv[R], acc[R];
#pragma unroll
          for (int r = 0; r < R; r++) {
            const PointAux a = ax[u * TX * TY + tsl0 + r * TX];
            ve[r] = *reinterpret_cast<const Rv *>(&a.veff);
            if constexpr (G::NLS) {
              // (gathered into the slot by the patcher warp)
              const V *nla = reinterpret_cast<const V *>(hslot + G::IN_BYTES + G::AUX_BYTES + G::STRIP_BYTES);
              nlv[r] = has_proj && a.r1 > a.r0 ? nla[(tsl0 + r * TX) * OV + v] : T::zero();
            } else {
              nlv[r] = has_proj ? nl_term<P>(nlk, n_ent, a.r0, a.r1) : T::zero();
            }
          }
          V gax[BLOCH ? R : 1][3];
          if constexpr (BLOCH) {
            stencil_rows_bloch<M, P, QB, QN, R>(p, W, w0, Q, xs, hs0, SXO, ve, acc, gax, need_grad, grads);
          } else {
            stencil_rows<M, P, QB, QN, R>(W, w0, Q, xs + u * G::SX * G::SY * OV, hs0, SXO, ve, acc);
          }
          const long iu = idx + (long)u * plane_pts * OV;
#pragma unroll
          for (int r = 0; r < R; r++) {
            const bool live = own[r] && (zf + u < z1);
            if (has_proj) acc[r] = T::add(acc[r], nlv[r]);
            const V c0 = Q[r][(QB + M) % QN];
            if (MODE == MODE_FIRST && do_obs && live) {
              oa.add_e(c0, acc[r]);
              if constexpr (BLOCH) {
                if (grads) {
#pragma unroll
                  for (int a = 0; a < 3; a++) oa.add_j(a, c0, gax[r][a]);
                }
              }
            }
            finish_point<P, MODE>(epi, CR, CI, live, iu + r * row, v, c0, acc[r], operands(csl0 + r * TX * OV));
          }
        });
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&hempty[hs]);
          if constexpr (OPS) mbar_arrive(&oempty[os]);
        }
        idx += U * plane_pts * OV;
        rh.next<SH>();
        if (OPS) ro.next<SO>();
      }
      l++;
    };
    // every item starts at queue rotation 0, so the plane loop runs in unrolled blocks of
    // QN / U iterations (one full turn of the queue), each with its compile-time rotation
    while (l < nl && !aborted) {
      static_for<0, QN / U>([&](auto j) {
        if (l < nl && !aborted) iteration(std::integral_constant<int, decltype(j)::value * U>{});
      });
    }
    if (aborted) break;
    if (MODE == MODE_FIRST && do_obs) {
      // this warp's partials of the item: record local * CW + warp
      double vals[4] = {oa.get_e(), oa.get_j(0), oa.get_j(1), oa.get_j(2)};
#pragma unroll
      for (int i = 0; i < 4; i++) {
        double x = vals[i];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) p.obs_part[(local * CW + warp) * 4 + i] = epi.wocc * x;
      }
    }
  }
  if (aborted) {
    *abort_flag = 1;
    if (lane == 0 && errp) atomicExch(errp, 1);
  }
}

template <int M, int P, int MODE, int TX, int TY, int R, int U, int BLOCH>
__global__ void __launch_bounds__(WsWarps<TX, TY, R, VT<P>::OV>::THREADS + 32 * BLOCH, 1)
ws_sweep_kernel(const __grid_constant__ SweepMaps maps, const __grid_constant__ SweepParams p) {
  const SingleSrc src{&p, &maps};
  ws_sweep_body<M, P, MODE, TX, TY, R, U, false, BLOCH>(src, p.work);
}

template <int M, int P, int MODE, int TX, int TY, int R, int U>
__global__ void __launch_bounds__(WsWarps<TX, TY, R, VT<P>::OV>::THREADS, 1)
ws_sweep_batch_kernel(const __grid_constant__ BatchSweepArgs a) {
  const BatchSrc src{&a};
  ws_sweep_body<M, P, MODE, TX, TY, R, U, true, 0>(src, a.work);
}

// Launch of the warp-specialised sweep of shape SHAPE for one system (one plane per
// iteration; grid <= 0: one CTA per SM, at most one per work item).
template <int SHAPE, int M, int P, int MODE, int BLOCH>
static cudaError_t launch_ws_t(const SweepMaps &maps, const SweepParams &p, int grid, cudaStream_t s) {
  constexpr int TX = WsShape<SHAPE>::TX, TY = WsShape<SHAPE>::TY, R = WsShape<SHAPE>::R;
  typedef TmaGeom<M, TX, TY, 1, MODE == MODE_LAST, BLOCH != 0, MODE == MODE_FIRST> G;
  auto k = ws_sweep_kernel<M, P, MODE, TX, TY, R, 1, BLOCH>;
  static std::atomic<unsigned> attr_done{0};
  if (cudaError_t e = ensure_smem_attr(k, G::SMEM, attr_done)) return e;
  if (grid <= 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = (int)(p.n_items < sms ? p.n_items : sms);
  }
  k<<<grid, WsWarps<TX, TY, R, VT<P>::OV>::THREADS + 32 * BLOCH, G::SMEM, s>>>(maps, p);  // (+ the patcher warp)
  return cudaGetLastError();
}

// Launch of the batched warp-specialised sweep of shape SHAPE: 152 persistent CTAs (one per
// SM, at most one per work item) walk the items of every system of the batch.
template <int SHAPE, int M, int P, int MODE>
static cudaError_t launch_ws_batch_t(const BatchSweepArgs &a, cudaStream_t s) {
  constexpr int TX = WsShape<SHAPE>::TX, TY = WsShape<SHAPE>::TY, R = WsShape<SHAPE>::R;
  typedef TmaGeom<M, TX, TY, 1, MODE == MODE_LAST> G;
  auto k = ws_sweep_batch_kernel<M, P, MODE, TX, TY, R, 1>;
  static std::atomic<unsigned> attr_done{0};
  if (cudaError_t e = ensure_smem_attr(k, G::SMEM, attr_done)) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)(a.total_items < sms ? a.total_items : sms);
  if (grid <= 0) return cudaSuccess;
  k<<<grid, WsWarps<TX, TY, R, VT<P>::OV>::THREADS, G::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int SHAPE>
cudaError_t launch_ws_batch_shape(int M, int prec, int mode, const BatchSweepArgs &a, cudaStream_t s) {
#define TDKS_WSB_MODES(MM, PP)                                                    \
  switch (mode) {                                                                 \
    case MODE_FIRST: return launch_ws_batch_t<SHAPE, MM, PP, MODE_FIRST>(a, s);   \
    case MODE_MID: return launch_ws_batch_t<SHAPE, MM, PP, MODE_MID>(a, s);       \
    case MODE_LAST: return launch_ws_batch_t<SHAPE, MM, PP, MODE_LAST>(a, s);     \
  }                                                                               \
  return cudaErrorInvalidValue;
  if constexpr (SHAPE == 5) {
    // complex64: one complex value per thread vector; complex128 runs shape 2
    if (prec != P_C64) return launch_ws_batch_shape<2>(M, prec, mode, a, s);
    if (M == 2) { TDKS_WSB_MODES(2, P_C64S) }
    if (M == 4) { TDKS_WSB_MODES(4, P_C64S) }
  } else {
    if (M == 2) {
      if (prec == P_C64) { TDKS_WSB_MODES(2, P_C64) } else { TDKS_WSB_MODES(2, P_C128) }
    }
    if (M == 4) {
      if (prec == P_C64) { TDKS_WSB_MODES(4, P_C64) } else { TDKS_WSB_MODES(4, P_C128) }
    }
  }
#undef TDKS_WSB_MODES
  return cudaErrorInvalidValue;
}

// One boundary kind of one shape: every mode, FD order and precision.
template <int SHAPE, int BLOCH>
static cudaError_t launch_ws_bc(int M, int prec, int mode, const SweepMaps &maps, const SweepParams &p, int grid,
                                cudaStream_t s) {
#define TDKS_WS_MODES(MM, PP)                                                                \
  switch (mode) {                                                                            \
    case MODE_FIRST: return launch_ws_t<SHAPE, MM, PP, MODE_FIRST, BLOCH>(maps, p, grid, s); \
    case MODE_MID: return launch_ws_t<SHAPE, MM, PP, MODE_MID, BLOCH>(maps, p, grid, s);     \
    case MODE_LAST: return launch_ws_t<SHAPE, MM, PP, MODE_LAST, BLOCH>(maps, p, grid, s);   \
  }                                                                                          \
  return cudaErrorInvalidValue;
  if (M == 2) {
    if (prec == P_C64) { TDKS_WS_MODES(2, P_C64) } else { TDKS_WS_MODES(2, P_C128) }
  }
  if (M == 4) {
    if (prec == P_C64) { TDKS_WS_MODES(4, P_C64) } else { TDKS_WS_MODES(4, P_C128) }
  }
#undef TDKS_WS_MODES
  return cudaErrorInvalidValue;
}

// Every mode, FD order, precision and boundary (finite box or periodic cell) of one shape
// (instantiated once per shape, in a translation unit of its own).
template <int SHAPE>
cudaError_t launch_ws_shape(int M, int prec, int mode, int bloch, const SweepMaps &maps, const SweepParams &p,
                            int grid, cudaStream_t s) {
  if constexpr (SHAPE == 5) {
    // complex64 finite boxes: one complex value per thread vector; the rest run shape 2
    if (bloch || prec != P_C64) return launch_ws_shape<2>(M, prec, mode, bloch, maps, p, grid, s);
#define TDKS_WS5_MODES(MM)                                                                       \
  switch (mode) {                                                                                \
    case MODE_FIRST: return launch_ws_t<5, MM, P_C64S, MODE_FIRST, 0>(maps, p, grid, s);         \
    case MODE_MID: return launch_ws_t<5, MM, P_C64S, MODE_MID, 0>(maps, p, grid, s);             \
    case MODE_LAST: return launch_ws_t<5, MM, P_C64S, MODE_LAST, 0>(maps, p, grid, s);           \
  }                                                                                              \
  return cudaErrorInvalidValue;
    if (M == 2) { TDKS_WS5_MODES(2) }
    if (M == 4) { TDKS_WS5_MODES(4) }
#undef TDKS_WS5_MODES
    return cudaErrorInvalidValue;
  } else {
    return bloch ? launch_ws_bc<SHAPE, 1>(M, prec, mode, maps, p, grid, s)
                 : launch_ws_bc<SHAPE, 0>(M, prec, mode, maps, p, grid, s);
  }
}

}  // namespace tdks
