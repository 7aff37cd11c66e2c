// Host-side system object and helpers shared by the C interface translation units
// (not part of the public interface).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/tdks.h"
#include "tdks_internal.cuh"

namespace tdks_host {

int fail(int code, const std::string &msg);

#define CU(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return tdks_host::fail(e_ == cudaErrorMemoryAllocation ? TDKS_ENOMEM : TDKS_EDEVICE,   \
                             std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

}  // namespace tdks_host

struct tdks_system {
  int nx, ny, nz, M, bc, prec, n_orb, n_k, BS, n_batches, n_kb;
  long N;
  double h;
  std::vector<double> kpts, kw;
  cudaStream_t stream;
  int dev;
  // physics parameters
  int xc = TDKS_XC_LDA_X;
  double occ = 2.0;
  int gauge = TDKS_GAUGE_NONE, envelope = TDKS_ENV_NONE;
  double pol[3] = {0, 0, 1}, amp = 0, omega = 0, t_total = 0;
  int n_atoms = 0;
  std::vector<double> pos, D;
  double r_c = 0.0, r_cut = 0.0;  // projector width and support radius (tdks_set_atoms_projectors)
  double vloc_absmax = 0.0, vnl_bound = 0.0;
  // device buffers
  void *psi = nullptr;          // packed state: complex128, or the hi part (complex64) of a
                                // complex64 system's double-float state
  void *psi_lo = nullptr;       // lo part of a complex64 system's state
  void *term[3] = {nullptr, nullptr, nullptr};
  double *vloc = nullptr;
  tdks::PointAux *aux = nullptr;   // V_eff and projector entry range per point
  double *dens_part = nullptr;
  double *lda_part = nullptr;
  double *obs_part = nullptr;
  long obs_cap = 0;            // records obs_part holds (sweep partials, then the projectors' current)
  long obs_base = 0;           // of which the sweep partials
  double *ring = nullptr;
  double *obs_rec = nullptr;    // single record for tdks_observe
  double *d_kvec = nullptr, *d_wocc = nullptr, *d_D = nullptr;
  int *d_rowent = nullptr, *d_atom_begin = nullptr;
  int2 *d_sp = nullptr;       // entry ranges of the points inside a sphere
  void *d_nl = nullptr;       // non-local term per sphere point, [n_kb][n_ent + 1][OVC]
  int n_sp = 0, n_ent = 0;
  tdks::ProjEntry *d_ent = nullptr;
  float4 *d_ent_beta = nullptr;  // compact copies of the entries' FP32 beta and (cell, atom)
  int2 *d_ent_ca = nullptr;
  // complex64 projector phases e^{i (k.T + A.d)} of every entry and k-point, built once per
  // vector potential (a sub-step's Taylor terms share one)
  float2 *d_phase = nullptr;
  double phase_A[3] = {0.0, 0.0, 0.0};
  bool phase_ok = false;
  double *fin_part = nullptr;    // first-stage partials of the observable record
  void *d_q = nullptr;
  double2 *d_qpart = nullptr;   // gather partial sums, gchunks per (atom, k-batch)
  int gchunks = 1;
  double *staging = nullptr;
  cudaStream_t copy_stream = nullptr;  // host uploads, chunked so that packing overlaps them
  cudaEvent_t ev_staging_free = nullptr;  // recorded after the last kernel that reads the staging buffer
  bool staging_pending = false;            // ev_staging_free has been recorded
  std::vector<cudaEvent_t> ev_chunk;
  // two upload buffers (tdks_set_upload_buffers): each upload packs the next state into these
  // spares on pack_stream while earlier work runs, and then they swap with psi / psi_lo / dens_part
  int upload_buffers = 1;
  void *psi_b = nullptr, *psi_lo_b = nullptr;
  double *dens_b = nullptr;
  cudaStream_t pack_stream = nullptr;
  cudaEvent_t ev_spare_free = nullptr;  // recorded on the stream when the spares were swapped out
  cudaEvent_t ev_packed = nullptr;      // recorded on pack_stream after an upload's packing
  bool spare_pending = false;
  int *d_err = nullptr;       // [0]: error word of the bounded waits; [1]: sweep work counter
  int withhold = 0;           // failure injection: the sweeps' producers withhold their copies
  long obs_count = 0;         // energy/current partial records written by the last first sweep
  // TMA tensor maps over the four sweep inputs (state, t1, t2, t3) for the current tile
  tdks::SweepMaps smaps[4];   // TMA maps of the four Taylor-term sweeps
  bool tmaps_ok = false;
  int path = 0;                 // 0: TMA sweep where possible, 1: general sweep
  size_t state_bytes = 0, term_bytes = 0;
  bool have_orbitals = false, dens_valid = false;
  long long steps = 0;
  // propagator (tdks_set_propagator); CFM4 keeps v_x of the last four sub-step starts
  int prop = TDKS_PROP_TAYLOR4;
  double *vx_hist[4] = {nullptr, nullptr, nullptr, nullptr};  // [0] the newest
  void *etrs_save = nullptr, *etrs_save_lo = nullptr;         // ETRS: the state during the trial
  int n_hist = 0;
  // state-parallel runs (tdks_set_exchange): hook, its context, the summed density
  // (N doubles) and the record's 10 sums
  tdks_exchange_fn xfn = nullptr;
  void *xctx = nullptr;
  double *n_total = nullptr, *fin_sum = nullptr;
  // t-SURFF (tdks_set_tsurff): surface entries, momenta, gathered surface values, amplitudes,
  // the Volkov parameters a, alpha, beta and the time since the accumulation started
  tdks::TsEntry *d_ts_ent = nullptr;
  double *d_ts_p = nullptr;
  double2 *d_ts_G = nullptr, *d_ts_b = nullptr;
  int ts_np = 0, ts_ne = 0;
  double ts_vol[7] = {0, 0, 0, 0, 0, 0, 0};
  double ts_trel = 0.0, ts_t0 = 0.0;
  bool ts_started = false;
  // Hartree term (xc = TDKS_XC_LDA_X_HARTREE): padded transform buffer and transformed kernel
  // (hp[] points per axis), the potential v_H (N doubles); the density goes through n_total
  double2 *d_hbuf = nullptr, *d_hkern = nullptr;
  double *d_vh = nullptr;
  int hp[3] = {0, 0, 0};
  // clock used by batched propagation: state time, step length, sub-steps per step
  double clock_t = 0.0, clock_dt = 0.0;
  int clock_substeps = 1;
  static constexpr long long RING = 65536;
  // stencil configuration
  int tx = 16, ty = 8, zc = 0;
  int wshape[4] = {0, 0, 0, 0};  // warp-specialised TMA sweep: tile shape of each Taylor term
  long long launches = 0;
  // profiling
  bool profile = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
  std::vector<cudaEvent_t> ev_free;
  double prof_ms[7] = {0, 0, 0, 0, 0, 0, 0};  // kinds of tdks_kernel_time
  long long prof_n[7] = {0, 0, 0, 0, 0, 0, 0};
};

namespace tdks_host {

void fd_weights(int M, double *lap, double *grad);
void field_at(const tdks_system *s, double t, double E[3], double A[3]);
double envelope_of(const tdks_system *s, double t, double *denv);
// sweep: which of the four Taylor-term sweeps (0..3) the parameters are for, so that the
// warp-specialised TMA sweep takes that sweep's tile shape; -1: the system's tile (16x8 on
// the TMA path)
bool ws_path(const tdks_system *s);
void sweep_geometry(const tdks_system *s, tdks::SweepParams &p, int sweep = -1);
void sweep_common(const tdks_system *s, tdks::SweepParams &p, const double A[3], int sweep = -1);
long n_items_of(const tdks_system *s);
bool encode_map(const tdks_system *s, const void *ptr, int mode, CUtensorMap *out, bool lockstep, int tx, int ty);
// tile box (no halo) of z depth `depth` over a packed array
bool encode_op_map(const tdks_system *s, const void *ptr, CUtensorMap *out, int tx, int ty, int depth = 1);
// all maps of a TMA sweep of `mode` over input `in` (the operand maps only for the last term)
// lockstep: box depths for the lockstep TMA kernel (tdks_set_sweep_path 2), else for the
// warp-specialised one
bool encode_sweep_maps(const tdks_system *s, const void *in, int mode, tdks::SweepMaps *out, bool lockstep,
                       int sweep = -1);
int ensure_density(tdks_system *s);
// t-SURFF (tdks_tsurff.cu): add weight x the flux of the current state to the amplitudes;
// advance a, alpha, beta and the accumulation time by dt from t; free the buffers
int tsurff_accumulate(tdks_system *s, double weight);
void tsurff_advance(tdks_system *s, double t, double dt);
void tsurff_free(tdks_system *s);
// Hartree potential (tdks_hartree.cu): workspace and transformed kernel; v_H of n_total into d_vh
int hartree_setup(tdks_system *s);
int hartree_solve(tdks_system *s);
void hartree_free(tdks_system *s);
int check_err(tdks_system *s);
double kinetic_max(const tdks_system *s);

}  // namespace tdks_host
