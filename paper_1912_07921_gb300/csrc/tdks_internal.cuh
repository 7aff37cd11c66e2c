// Internal declarations of the GB300 TDKS library (not part of the C interface).
//
// Device layout of one system ("packed batches", the paper's Sec. "Memory layout": the
// state index is innermost so every thread of a warp runs the same stencil on
// neighbouring orbitals):
//
//   orbitals  [k][batch][z][y][x][j],  orbital o = batch * BS + j,  BS orbitals per batch
//   vectors   one thread owns one 16-byte vector: complex128 -> 1 orbital,
//             complex64 -> 2 orbitals; OVC = 4 vectors per (point, batch), i.e. 64 B.
//
// complex128 systems: BS = 4, the state and the Taylor terms are complex128.
// complex64  systems: BS = 8, the Taylor terms are complex64; the state (the running sum
//                     of the series) is a double-float pair hi + lo of two complex64
//                     arrays (~48-bit significand), updated with error-free FP32
//                     transformations, because GB300 runs FP64 at a small fraction of its
//                     FP32 rate; density, potentials and reductions are FP64.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace tdks {

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per device for kernel k; `done`
// (one per kernel instantiation) records the devices already set, safely across host
// threads that drive systems at the same time.
template <typename K>
inline cudaError_t ensure_smem_attr(K k, size_t smem, std::atomic<unsigned> &done) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned bit = dev < 32 ? 1u << dev : 0u;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

constexpr int OVC = 4;        // 16-byte vectors per (point, batch)
constexpr int MAXM = 4;       // largest FD half-width (8th order)

enum Mode { MODE_FIRST = 0, MODE_MID = 1, MODE_LAST = 2 };
// Compute precisions of the sweeps.  P_C64S is complex64 storage computed with one complex
// value per thread vector (8 bytes, 8 vectors per (point, batch)) instead of two (16 bytes,
// 4 vectors): the tile shapes that use it keep more points per thread in registers.
enum Prec { P_C128 = 0, P_C64 = 1, P_C64S = 2 };

// Per-entry projector data (one grid point of one atom's sphere).
struct ProjEntry {
  int cell;        // flat grid index of the (wrapped) point
  int atom;
  float beta[4];   // beta_aj at the point (c64 path)
  double betad[4]; // same, double (c128 path)
  double T[3];     // lattice translation of the unwrapped point
  double d[3];     // unwrapped point minus atom centre
};

// One point of one face of the t-SURFF surface: its flat grid index, the face's normal
// axis, the trapezoid weight times the sign of the outward normal, and its position.
struct TsEntry {
  long cell;
  int ax;
  double ws;
  double r[3];
};

// Per-point record read by the sweeps (16 bytes): the diagonal potential V_eff (double
// for complex128 systems; float in the first 4 bytes for complex64 systems) and the point's
// range [r0, r1) in the point-major projector entry list.
struct __align__(16) PointAux {
  double veff;
  int r0, r1;
};

struct SweepParams {
  int nx, ny, nz;
  int n_tx, n_ty, n_zc, zc;   // x/y tiles and z chunks
  int n_kb, n_batches;        // kb = k * n_batches + batch
  long n_items;
  // stencil: H = w0 c + sum_m w[m] (sum of the 6 neighbours at distance m) + ...
  double w[MAXM + 1];         // w[0] = -3 c_0 / (2 h^2), w[m] = -c_m / (2 h^2)
  double gw[MAXM + 1];        // gradient weights d_m / h
  double cr, ci;              // out = (cr + i ci) * (H in)
  float wf[MAXM + 1];         // w rounded to FP32 (complex64 sweeps)
  float crf, cif;             // cr, ci rounded to FP32
  const void *in;             // stencil input (psi storage in MODE_FIRST, term storage else)
  void *out;                  // term output (MODE_FIRST / MODE_MID)
  void *psi;                  // MODE_LAST: state (complex128, or the hi part of a complex64
                              // system's double-float state), read and written in place
  void *psi_lo;               // MODE_LAST, complex64 systems: lo part of the state
  const void *t1, *t2;        // MODE_LAST: earlier terms
  const PointAux *aux;        // [N] V_eff and projector entry ranges
  // projectors
  int has_proj;               // the system has projector entries
  const void *nl;             // [kb][n_ent + 1][OVC] vectors: sum_aj beta_aj(r) phase q_aj at the
                              // sphere point whose entries start at r0; row n_ent is zero
  int n_ent;                  // projector entries
  // Bloch boundary
  int bloch;                  // periodic cell: values across a face carry exp(i k.L) per wrap
  const double *kvec;         // [n_k][3]
  double L[3];
  double A[3];                // vector potential (velocity gauge)
  int grad_mask;              // bit a: add -i A_a grad_a; bit 3: observables need all grads
  // reductions
  int do_obs;
  double *obs_part;           // [n_items][4]: <psi|H psi> weighted, current x,y,z
  const double *wocc;         // [n_k] k-weight times occupation
  double *dens_part;          // [n_kb][N] (MODE_LAST): w_k f sum |psi|^2 (complex128); for
                              // complex64, the unweighted sum as a (float hi, float lo) pair
  int *err;                   // device error word (bounded waits that ran out set it)
  int withhold;               // failure injection (tests): the producer makes no claim and no
                              // copy, so every other warp's first wait runs out
  unsigned int *work;         // work-item counter of the warp-specialised TMA sweep (zero
                              // between launches: the launch's last claim resets it)
};

// Sets the Taylor coefficient (cr + i ci) with its FP32 copies.
inline void set_coef(SweepParams &p, double cr, double ci) {
  p.cr = cr;
  p.ci = ci;
  p.crf = (float)cr;
  p.cif = (float)ci;
}

struct GatherParams {
  int n_kb, n_batches, n_atoms;
  long N;
  const void *in;             // stencil input (state or hi part of the state, or a term)
  const int *atom_begin;      // [n_atoms+1] entry ranges (atom-major)
  const ProjEntry *ent;
  const float4 *ent_beta;     // [n_ent] beta_aj of each entry in FP32 (complex64 kernels)
  const int2 *ent_ca;         // [n_ent] (cell, atom) of each entry
  const double *D;            // [n_atoms][4]
  double h3;
  const double *kvec;
  double A[3];
  void *q;                    // [kb][atom][4][OVC] vectors
  int n_chunks;               // CTAs per (atom, kb): each sums a contiguous share of the sphere
  double2 *qpart;             // [kb][atom][chunk][4][OVC][2] partial sums (FP64)
  // scatter side: the non-local term at every sphere point
  const int2 *sp;             // [n_sp] entry range [r0, r1) of each point inside a sphere
  int n_sp;
  const int *rowent;          // entry indices, point-major
  int n_ent;
  void *nl;                   // [kb][n_ent + 1][OVC] vectors, row r0 of each sphere point
  const float2 *phase;        // complex64: [k][n_ent] (cos, sin) of k.T + A.d, or null
};

// The projectors' share of a periodic cell's current (record time): partial records
// out[(kb * n_atoms + a) * BS + o][4] for every atom, k-batch and orbital of the batch.
struct NlCurrentParams {
  int prec, BS, n_batches, n_kb, n_atoms;
  long N;
  const void *psi, *psi_lo;   // the state (complex64: hi and lo parts)
  const int *atom_begin;      // [n_atoms + 1] entry ranges
  const ProjEntry *ent;
  const double *D;            // [n_atoms][4]
  const double *kvec;         // [n_k][3]
  const double *wocc;         // [n_k] k-weight times occupation
  double A[3], h3;
  double *out;
};
cudaError_t launch_nl_current(const NlCurrentParams &p, cudaStream_t s);

// Per-system data of a batch (device copies), for the batched LDA and finalise kernels.
struct BatchAux {
  long N;
  int nx, ny, nz, n_kb, n_batches, xc;
  double h, occ;
  const double *wocc;       // [n_k] k-weight times occupation
  int gauge, envelope;
  double pol[3], amp, omega, t_total;
  const double *dens_part;
  const double *vloc;
  PointAux *aux;
  double *lda_part;
  int n_lda;
  double *obs_part;
  long n_items;
  double *ring;
  long long ring_len;
};

// Device clock of a batched system: state time t of the current step, step length dt,
// sub-steps per step, current sub-step j, steps completed.
struct BatchClock {
  double t, dt;
  long long step;
  int substeps, j;
};

// Tensor maps of one TMA sweep launch: the stencil input with halo (z depth = planes per
// copy), the stencil input as tiles without halo (same depth), the per-point records (tile
// box, same depth) and, for the last Taylor term, the four own-point operands state hi,
// state lo, t1, t2 (tile boxes, depth 1).
struct SweepMaps {
  CUtensorMap in, ctr, aux, op[4];
  CUtensorMap sx, sy;  // periodic cells: the input as M x (TY + 2M) and TX x M strip boxes
};

// Batched stencil sweep over many systems (tdks_sweep_tma.cu): params[s] and
// maps[4*s + which] of system s; item_begin[s] = first work item of system s.
struct BatchSweepArgs {
  const SweepParams *params;
  const SweepMaps *maps;  // 4 per system (one per Taylor term)
  int which;
  const long *item_begin;
  int n_sys;
  long total_items;
  unsigned int *work;     // work-item counter (zero between launches)
  const int *item_sys;    // the system of every work item
};


// Launchers (tdks_sweep.cu)
cudaError_t launch_sweep(int M, int prec, int mode, int bloch, int tx, int ty,
                         const SweepParams &p, int grid, cudaStream_t s);
int sweep_threads(int tx, int ty);
size_t sweep_smem(int M, int tx, int ty);

// Launchers (tdks_aux.cu).  The projector step is three kernels: the gather-dot (stages 1
// and 2) and the non-local term at every sphere point (skipped when no point is in a sphere).
constexpr int NL_THREADS = 256;
cudaError_t launch_gather(int prec, int bloch, const GatherParams &p, cudaStream_t s);
// out[k * n_ent + e] = (cos, sin) of A.d_e (+ k.T_e in a periodic cell), as the complex64
// projector kernels would form it per entry
cudaError_t launch_phase_table(const ProjEntry *ent, int n_ent, int n_k, const double *kvec, const double A[3],
                               int bloch, float2 *out, cudaStream_t s);
// chunks per (atom, k-batch) that fill the GPU for n_atoms * n_kb units
int gather_chunks(long units);
cudaError_t launch_density(int prec, long N, int n_kb, int n_batches, const void *psi, const void *psi_lo,
                           const double *wocc, double *dens_part, cudaStream_t s);
cudaError_t launch_lda(int prec, int bloch, long N, int nx, int ny, int nz, double h,
                       int n_kb, int n_batches, const double *wocc, const double *dens_part,
                       const double *vloc, int xc,
                       const double E[3], double half_A2, PointAux *aux, double *lda_part,
                       int n_blocks, cudaStream_t s, const double *n_in = nullptr, const double *vh = nullptr,
                       int sums = 1);
// Classical Runge-Kutta stage update over n complex128 values (complex128 systems):
//   stage = psi + a k,  acc = (init ? 0 : acc) + b k,
// and the last stage's psi <- psi + acc + b k (rk4_finish).
cudaError_t launch_rk4_stage(long n, const void *psi, const void *k, double a, void *stage, void *acc, double b,
                             int init, cudaStream_t s);
cudaError_t launch_rk4_finish(long n, void *psi, const void *acc, const void *k, double b, cudaStream_t s);
// n_out[r] = sum over this system's states of w_k f |psi_ik(r)|^2 (FP64), from dens_part
cudaError_t launch_density_sum(int prec, long N, int n_kb, int n_batches, const double *wocc,
                               const double *dens_part, double *n_out, cudaStream_t s);
// fin_part: device scratch of FIN_BLOCKS * 10 doubles for the first of the two stages
constexpr int FIN_BLOCKS = 64;
// CFM4 exchange history: v[j] is v_x at the start of the j-th latest sub-step (v[0] the
// newest), w[j] its weight in an exponential's effective potential, nh the points in use.
struct CfmHist {
  double *v[4];
  double w[4];
  int nh;
};
cudaError_t launch_cfm_veff(int prec, int bloch, long N, int nx, int ny, int nz, double h, int n_kb, int n_batches,
                            const double *wocc, const double *dens_part, const double *vloc, int xc, int push,
                            const CfmHist &hist, const double E[3], PointAux *aux, cudaStream_t s,
                            const double *vh = nullptr, const double *n_in = nullptr);
cudaError_t launch_finalize(const double *obs_part, long n_items, const double *lda_part,
                            int n_lda_blocks, double *record, double t_state, double h3,
                            double occ, int bloch, double omega_cell, const double A[3],
                            double field_val, double *fin_part, cudaStream_t s);
// The same record in two parts, for state-parallel runs: the 10 sums into sums[0..9]
// (sums[0..3]: this rank's band energy and current; sums[4..9]: from the summed density),
// then, once the caller has summed sums[0..3] over the ranks, the record from sums.
cudaError_t launch_finalize_sums(const double *obs_part, long n_items, const double *lda_part, int n_lda_blocks,
                                 double *fin_part, double *sums, cudaStream_t s);
cudaError_t launch_record_from_sums(const double *sums, double *record, double t_state, double h3, double occ,
                                    int bloch, double omega_cell, const double A[3], double field_val,
                                    cudaStream_t s);
// host layout -> internal layout and density partials, points [pt0, pt0 + npts) of k-point k
cudaError_t launch_pack_in(int prec, long N, int k, long pt0, long npts, int n_orb, int n_batches,
                           const double *plain, void *internal, void *internal_lo, const double *wocc,
                           double *dens_part, cudaStream_t s);
cudaError_t launch_pack(int prec, int to_internal, long N, int n_k, int n_orb, int n_batches,
                        void *internal, void *internal_lo, double *plain, cudaStream_t s);

// TMA sweep for finite boxes (tdks_sweep_tma.cu).  maps.in: dims {16 floats, nx, ny, nz,
// n_kb}, box {16, TX+2M, TY+2M, tma_planes(prec, mode), 1} (TY: the shape's tile height); maps.aux: dims {4, nx, ny, nz}
// (4-byte words), box {4, TX, TY, tma_planes}; maps.op[i]: dims as maps.in, box
// {16, TX, TY, 1, 1}; maps.ctr: as maps.op with tma_planes planes.  Default: the
// warp-specialised kernel (a producer warp and eight consumer warps); lockstep: the variant
// in which all warps of a CTA advance plane by plane together.
cudaError_t launch_sweep_tma(int M, int prec, int mode, int tx, int ty, const SweepMaps &maps,
                             const SweepParams &p, int grid, cudaStream_t s, bool lockstep = false,
                             int shape = 0);
// Tile shapes of the warp-specialised sweep: shape s covers tx x ty points of one orbital
// block with `warps` consumer warps, each thread computing `rows` y-adjacent points.
// Shape 0 (16 x 8, two points per thread, eight consumer warps) is the default and the one
// the batched sweep uses.  Null outputs are skipped; false for a shape out of range.
constexpr int WS_SHAPES = 6;
bool ws_shape_info(int shape, int *tx, int *ty, int *rows, int *warps);
bool tma_supported(int M, int tx, int ty);
int tma_planes(int prec, int mode, bool lockstep = false);
int lda_blocks(long N);
cudaError_t launch_sweep_tma_batch(int M, int prec, int mode, const BatchSweepArgs &a, cudaStream_t s,
                                   int shape = 0);
// begin: prefix sums of n_atoms * n_kb * n_chunks (stage 1 CTAs); ubegin: of n_atoms * n_kb;
// nbegin: of the non-local kernel's CTAs, n_kb * ceil(n_sp * OVC / NL_THREADS).  gsys, usys,
// nsys: the system of each stage-1 CTA, unit and non-local CTA (one table load instead of a
// binary search over the prefix sums in every CTA).
cudaError_t launch_gather_batch(int prec, const GatherParams *gp, const long *begin, const long *ubegin,
                                const long *nbegin, const int *gsys, const int *usys, const int *nsys,
                                long total, long total_units, long total_nl, cudaStream_t s);
// CTAs of the non-local kernel of one system; in a batch each CTA covers NL_BATCH_RUNS runs of
// NL_THREADS (sphere point, vector) pairs, so that its setup is paid once per several runs
inline long nl_blocks(int n_sp, int n_kb) { return (long)n_kb * (((long)n_sp * OVC + NL_THREADS - 1) / NL_THREADS); }
constexpr int NL_BATCH_RUNS = 8;
inline long nl_batch_blocks(int n_sp, int n_kb) {
  return (long)n_kb * (((long)n_sp * OVC + NL_THREADS * NL_BATCH_RUNS - 1) / (NL_THREADS * NL_BATCH_RUNS));
}
cudaError_t launch_lda_batch(int prec, const BatchAux *aux, const BatchClock *clk, const long *begin, int n_sys,
                             long total, cudaStream_t s);
// which = 0: observable records (first sub-step of a step); 1: advance the clocks
cudaError_t launch_batch_tail(const BatchAux *aux, BatchClock *clk, int n_sys, int which, cudaStream_t s);

}  // namespace tdks
