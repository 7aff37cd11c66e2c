// C interface of the TDKS library: system objects, host-side set-up (finite-difference
// weights, projector spheres, field, sub-step policy) and the propagation driver.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tdks_system.h"

using namespace tdks;
using namespace tdks_host;

namespace tdks_host {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn lookup_encode_fn() {
  void *f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    return reinterpret_cast<EncodeTiledFn>(f);
  return nullptr;
}
EncodeTiledFn encode_fn() {
  static const EncodeTiledFn fn = lookup_encode_fn();  // initialised once, thread-safe
  return fn;
}

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}



// Finite-difference weights by Fornberg's recursion (weights of derivatives 0..2 at
// x = 0 from the nodes -M..M); central, order 2M.
void fd_weights(int M, double *lap, double *grad) {
  const int n = 2 * M;
  std::vector<double> x(n + 1);
  for (int i = 0; i <= n; i++) x[i] = (double)(i - M);
  std::vector<std::vector<double>> c(n + 1, std::vector<double>(3, 0.0));
  double c1 = 1.0, c4 = x[0];
  c[0][0] = 1.0;
  for (int i = 1; i <= n; i++) {
    const int mn = std::min(i, 2);
    double c2 = 1.0;
    const double c5 = c4;
    c4 = x[i];
    for (int j = 0; j < i; j++) {
      const double c3 = x[i] - x[j];
      c2 *= c3;
      if (j == i - 1) {
        for (int k = mn; k > 0; k--) c[i][k] = c1 * (k * c[i - 1][k - 1] - c5 * c[i - 1][k]) / c2;
        c[i][0] = -c1 * c5 * c[i - 1][0] / c2;
      }
      for (int k = mn; k > 0; k--) c[j][k] = (c4 * c[j][k] - k * c[j][k - 1]) / c3;
      c[j][0] = c4 * c[j][0] / c3;
    }
    c1 = c2;
  }
  for (int m = 0; m <= M; m++) {
    lap[m] = c[M + m][2];
    grad[m] = m == 0 ? 0.0 : c[M + m][1];
  }
}

}  // namespace

namespace tdks_host {

double envelope_of(const tdks_system *s, double t, double *denv) {
  if (s->envelope == TDKS_ENV_SIN2) {
    if (t < 0.0 || t > s->t_total) { *denv = 0.0; return 0.0; }
    const double a = M_PI * t / s->t_total;
    *denv = 2.0 * std::sin(a) * std::cos(a) * M_PI / s->t_total;
    return std::sin(a) * std::sin(a);
  }
  *denv = 0.0;
  return 1.0;
}

// E(t), A(t) of the configured laser
void field_at(const tdks_system *s, double t, double E[3], double A[3]) {
  double denv;
  const double env = envelope_of(s, t, &denv);
  const double f = s->amp * env * std::sin(s->omega * t);
  const double df = s->amp * (denv * std::sin(s->omega * t) + env * s->omega * std::cos(s->omega * t));
  for (int a = 0; a < 3; a++) {
    E[a] = A[a] = 0.0;
    if (s->gauge == TDKS_GAUGE_LENGTH) E[a] = f * s->pol[a];
    if (s->gauge == TDKS_GAUGE_VELOCITY) { A[a] = f * s->pol[a]; E[a] = -df * s->pol[a]; }
  }
}

int ev_get(tdks_system *s, cudaEvent_t *e) {
  if (!s->ev_free.empty()) { *e = s->ev_free.back(); s->ev_free.pop_back(); return 0; }
  return cudaEventCreate(e) == cudaSuccess ? 0 : -1;
}

struct Timed {
  tdks_system *s;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  Timed(tdks_system *s_, int k) : s(s_), kind(k) {
    if (s->profile && ev_get(s, &a) == 0 && ev_get(s, &b) == 0) cudaEventRecord(a, s->stream);
    else a = b = nullptr;
  }
  ~Timed() {
    if (a && b) {
      cudaEventRecord(b, s->stream);
      s->ev_used.push_back({kind, {a, b}});
    }
  }
};

// The warp-specialised TMA sweep serves finite boxes and periodic cells (path 0, 16x8 system
// tile); the lockstep TMA sweep (path 2) serves finite boxes only.
bool ws_path(const tdks_system *s) { return s->path == 0 && tma_supported(s->M, s->tx, s->ty); }

static bool tma_path(const tdks_system *s) {
  return ws_path(s) || (s->path == 2 && s->bc == TDKS_BC_ZERO && tma_supported(s->M, s->tx, s->ty));
}

// Tile of a sweep: the warp-specialised TMA sweep's shape, else the system's tile.
static void sweep_tile(const tdks_system *s, int sweep, int &tx, int &ty) {
  tx = s->tx;
  ty = s->ty;
  if (sweep >= 0 && ws_path(s)) ws_shape_info(s->wshape[sweep], &tx, &ty, nullptr, nullptr);
}

void sweep_geometry(const tdks_system *s, SweepParams &p, int sweep) {
  int tx, ty;
  sweep_tile(s, sweep, tx, ty);
  p.nx = s->nx; p.ny = s->ny; p.nz = s->nz;
  p.n_tx = (s->nx + tx - 1) / tx;
  p.n_ty = (s->ny + ty - 1) / ty;
  p.n_kb = s->n_kb;
  p.n_batches = s->n_batches;
  int zc = s->zc;
  const bool dynamic = ws_path(s);
  if (zc <= 0 && dynamic) {
    // warp-specialised TMA sweep: CTAs claim items from a counter, so the cost is the total
    // work spread over the SMs (the 2M priming planes of an item only load a centre tile,
    // about a quarter of an output plane each) plus half an item of tail; the items of
    // one column's z chunks are claimed one after another and share their halo planes in L2.
    const long per_plane = (long)p.n_tx * p.n_ty * p.n_kb;
    double best = -1.0;
    for (int c = 1; c <= s->nz; c++) {
      const long items = per_plane * ((s->nz + c - 1) / c);
      const double cost = (double)items * (c + 0.25 * 2 * s->M) / 152.0 + 0.5 * c;
      if (best < 0.0 || cost < best) { best = cost; zc = c; }
    }
  } else if (zc <= 0) {
    // z-chunk length minimising (waves of work items) x (planes per item, including the
    // 2M planes that prime each item's z-queue); one resident CTA per SM.
    const long per_plane = (long)p.n_tx * p.n_ty * p.n_kb;
    const long slots = 152;
    long best = -1;
    for (int c = 1; c <= s->nz; c++) {
      const long items = per_plane * ((s->nz + c - 1) / c);
      const long cost = ((items + slots - 1) / slots) * (c + 2 * s->M);
      if (best < 0 || cost < best) { best = cost; zc = c; }
    }
  }
  p.zc = zc;
  p.n_zc = (s->nz + zc - 1) / zc;
  p.n_items = (long)p.n_tx * p.n_ty * p.n_kb * p.n_zc;
}

long n_items_of(const tdks_system *s) {
  SweepParams p{};
  sweep_geometry(s, p);
  return p.n_items;
}

void sweep_common(const tdks_system *s, SweepParams &p, const double A[3], int sweep) {
  sweep_geometry(s, p, sweep);
  double c[MAXM + 1], d[MAXM + 1];
  fd_weights(s->M, c, d);
  for (int m = 0; m <= MAXM; m++) { p.w[m] = 0.0; p.gw[m] = 0.0; }
  p.w[0] = -1.5 * c[0] / (s->h * s->h);
  for (int m = 1; m <= s->M; m++) {
    p.w[m] = -0.5 * c[m] / (s->h * s->h);
    p.gw[m] = d[m] / s->h;
  }
  for (int m = 0; m <= MAXM; m++) p.wf[m] = (float)p.w[m];
  set_coef(p, 1.0, 0.0);
  p.aux = s->aux;
  p.has_proj = s->n_atoms > 0;
  p.withhold = s->withhold;
  p.nl = s->d_nl;
  p.n_ent = s->n_ent;
  p.kvec = s->d_kvec;
  p.bloch = s->bc == TDKS_BC_BLOCH;
  p.L[0] = s->nx * s->h; p.L[1] = s->ny * s->h; p.L[2] = s->nz * s->h;
  for (int a = 0; a < 3; a++) p.A[a] = A[a];
  p.grad_mask = 0;
  if (s->bc == TDKS_BC_BLOCH)
    for (int a = 0; a < 3; a++) if (A[a] != 0.0) p.grad_mask |= 1 << a;
  p.wocc = s->d_wocc;
  p.obs_part = s->obs_part;
  p.work = s->d_err ? reinterpret_cast<unsigned int *>(s->d_err + 1) : nullptr;
  p.dens_part = s->dens_part;
  p.do_obs = 0;
}

// Tensor map over a packed array for the TMA sweep of `mode` (box depth = planes per copy).
bool encode_map(const tdks_system *s, const void *ptr, int mode, CUtensorMap *out, bool lockstep, int tx, int ty) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(ptr) & 15) != 0) return false;
  const cuuint64_t dims[5] = {16, (cuuint64_t)s->nx, (cuuint64_t)s->ny, (cuuint64_t)s->nz, (cuuint64_t)s->n_kb};
  const cuuint64_t strides[4] = {64, 64ull * s->nx, 64ull * s->nx * s->ny, 64ull * (cuuint64_t)s->N};
  const cuuint32_t box[5] = {16, (cuuint32_t)(tx + 2 * s->M), (cuuint32_t)(ty + 2 * s->M),
                             (cuuint32_t)tma_planes(s->prec, mode, lockstep), 1};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void *>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Map over the per-point records, tile box of the mode's depth.
bool encode_aux_map(const tdks_system *s, int mode, CUtensorMap *out, bool lockstep, int tx, int ty) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(s->aux) & 15) != 0) return false;
  const cuuint64_t dims[4] = {4, (cuuint64_t)s->nx, (cuuint64_t)s->ny, (cuuint64_t)s->nz};
  const cuuint64_t strides[3] = {16, 16ull * s->nx, 16ull * s->nx * s->ny};
  const cuuint32_t box[4] = {4, (cuuint32_t)tx, (cuuint32_t)ty, (cuuint32_t)tma_planes(s->prec, mode, lockstep)};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, s->aux, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Map over a packed array with the tile box (no halo) of z depth `depth`.
bool encode_op_map(const tdks_system *s, const void *ptr, CUtensorMap *out, int tx, int ty, int depth) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(ptr) & 15) != 0) return false;
  const cuuint64_t dims[5] = {16, (cuuint64_t)s->nx, (cuuint64_t)s->ny, (cuuint64_t)s->nz, (cuuint64_t)s->n_kb};
  const cuuint64_t strides[4] = {64, 64ull * s->nx, 64ull * s->nx * s->ny, 64ull * (cuuint64_t)s->N};
  const cuuint32_t box[5] = {16, (cuuint32_t)tx, (cuuint32_t)ty, (cuuint32_t)depth, 1};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void *>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_sweep_maps(const tdks_system *s, const void *in, int mode, SweepMaps *out, bool lockstep, int sweep) {
  int tx = s->tx, ty = s->ty;
  if (!lockstep) sweep_tile(s, sweep, tx, ty);
  if (!encode_map(s, in, mode, &out->in, lockstep, tx, ty) || !encode_aux_map(s, mode, &out->aux, lockstep, tx, ty) ||
      !encode_op_map(s, in, &out->ctr, tx, ty, tma_planes(s->prec, mode, lockstep)))
    return false;
  if (s->bc == TDKS_BC_BLOCH) {
    // periodic-image strips of boundary tiles: M columns over the slot's rows, M rows over
    // the tile's columns
    if (!encode_op_map(s, in, &out->sx, s->M, ty + 2 * s->M) || !encode_op_map(s, in, &out->sy, tx, s->M))
      return false;
  } else {
    out->sx = out->sy = out->in;  // unused
  }
  if (mode == MODE_LAST) {
    const void *ops[4] = {s->psi, s->psi_lo ? s->psi_lo : s->psi, s->term[0], s->term[1]};
    for (int j = 0; j < 4; j++)
      if (!encode_op_map(s, ops[j], &out->op[j], tx, ty)) return false;
  } else {
    for (int j = 0; j < 4; j++) out->op[j] = out->in;  // unused
  }
  return true;
}

void build_tmaps(tdks_system *s) {
  s->tmaps_ok = false;
  if (!tma_path(s)) return;
  const void *ins[4] = {s->psi, s->term[0], s->term[1], s->term[2]};
  const int modes[4] = {MODE_FIRST, MODE_MID, MODE_MID, MODE_LAST};
  for (int i = 0; i < 4; i++)
    if (!encode_sweep_maps(s, ins[i], modes[i], &s->smaps[i], s->path == 2, i)) return;
  s->tmaps_ok = true;
}

// tm: tensor maps of the sweep (or null): finite boxes with a 16x8 tile take the TMA sweep.
// sweep: which Taylor-term sweep (0..3; its tile shape on the warp-specialised TMA path), or
// -1 for the default shape
int run_sweep(tdks_system *s, int mode, SweepParams &p, const SweepMaps *tm, int sweep = -1) {
  Timed tmr(s, sweep >= 0 && sweep < 4 ? 3 + sweep : 0);  // (kinds 3..6 also count as kind 0)
  p.err = s->d_err;
  cudaError_t e;
  const bool tma = tm && tma_path(s);
  const bool ws = tma && s->path == 0;
  const int shape = (ws && sweep >= 0) ? s->wshape[sweep] : 0;
  if (tma)
    e = launch_sweep_tma(s->M, s->prec, mode, s->tx, s->ty, *tm, p, 0, s->stream, !ws, shape);
  else
    e = launch_sweep(s->M, s->prec, mode, s->bc == TDKS_BC_BLOCH, s->tx, s->ty, p, 0, s->stream);
  if (mode == MODE_FIRST && p.do_obs) {
    int warps = 1;
    if (ws) ws_shape_info(shape, nullptr, nullptr, nullptr, &warps);
    s->obs_count = p.n_items * warps;
  }
  s->launches++;
  if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("stencil sweep: ") + cudaGetErrorString(e));
  return TDKS_OK;
}

int run_gather(tdks_system *s, const void *in, const double A[3]) {
  if (s->n_atoms <= 0) return TDKS_OK;
  GatherParams g{};
  g.n_kb = s->n_kb; g.n_batches = s->n_batches; g.n_atoms = s->n_atoms; g.N = s->N;
  g.in = in;
  g.atom_begin = s->d_atom_begin; g.ent = s->d_ent; g.D = s->d_D;
  g.ent_beta = s->d_ent_beta; g.ent_ca = s->d_ent_ca;
  g.h3 = s->h * s->h * s->h;
  g.kvec = s->d_kvec;
  for (int a = 0; a < 3; a++) g.A[a] = s->gauge == TDKS_GAUGE_VELOCITY ? A[a] : 0.0;
  g.q = s->d_q;
  g.n_chunks = s->gchunks;
  g.qpart = s->d_qpart;
  g.sp = s->d_sp; g.n_sp = s->n_sp;
  g.rowent = s->d_rowent; g.n_ent = s->n_ent;
  g.nl = s->d_nl;
  g.phase = nullptr;
  const bool bloch = s->bc == TDKS_BC_BLOCH;
  if (s->prec == TDKS_C64 && (bloch || g.A[0] != 0.0 || g.A[1] != 0.0 || g.A[2] != 0.0)) {
    // the entries' phases for this vector potential, once for the Taylor terms that share it
    if (!s->d_phase) CU(cudaMalloc((void **)&s->d_phase, (size_t)s->n_ent * s->n_k * sizeof(float2)));
    if (!s->phase_ok || g.A[0] != s->phase_A[0] || g.A[1] != s->phase_A[1] || g.A[2] != s->phase_A[2]) {
      CU(launch_phase_table(s->d_ent, s->n_ent, s->n_k, s->d_kvec, g.A, bloch, s->d_phase, s->stream));
      s->launches++;
      for (int a = 0; a < 3; a++) s->phase_A[a] = g.A[a];
      s->phase_ok = true;
    }
    g.phase = s->d_phase;
  }
  Timed tm(s, 1);
  cudaError_t e = launch_gather(s->prec, bloch, g, s->stream);
  s->launches += s->n_sp > 0 ? 3 : 2;  // gather stages 1 and 2, the non-local term
  if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("projector gather: ") + cudaGetErrorString(e));
  return TDKS_OK;
}

int ensure_density(tdks_system *s) {
  if (!s->have_orbitals) return fail(TDKS_ESTATE, "orbitals not set");
  if (s->dens_valid) return TDKS_OK;
  Timed tm(s, 2);
  cudaError_t e = launch_density(s->prec, s->N, s->n_kb, s->n_batches, s->psi, s->psi_lo, s->d_wocc,
                                 s->dens_part, s->stream);
  s->launches++;
  if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("density: ") + cudaGetErrorString(e));
  s->dens_valid = true;
  return TDKS_OK;
}

int run_lda(tdks_system *s, const double E[3], const double A[3], bool sums = true) {
  const double half_A2 = s->gauge == TDKS_GAUGE_VELOCITY ? 0.5 * (A[0] * A[0] + A[1] * A[1] + A[2] * A[2]) : 0.0;
  const double El[3] = {s->gauge == TDKS_GAUGE_LENGTH ? E[0] : 0.0, s->gauge == TDKS_GAUGE_LENGTH ? E[1] : 0.0,
                        s->gauge == TDKS_GAUGE_LENGTH ? E[2] : 0.0};
  const bool hartree = s->xc == TDKS_XC_LDA_X_HARTREE;
  if (s->xfn || hartree) {  // the density as one FP64 array: every rank's states, or the Hartree source
    cudaError_t e = launch_density_sum(s->prec, s->N, s->n_kb, s->n_batches, s->d_wocc, s->dens_part, s->n_total,
                                       s->stream);
    s->launches++;
    if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("density sum: ") + cudaGetErrorString(e));
    if (s->xfn)
      if (int r = s->xfn(s->n_total, (long long)s->N, (void *)s->stream, s->xctx))
        return fail(TDKS_EDEVICE, "exchange hook failed on the density (" + std::to_string(r) + ")");
  }
  if (hartree)
    if (int rc = hartree_solve(s)) return rc;
  Timed tm(s, 2);
  cudaError_t e = launch_lda(s->prec, s->bc == TDKS_BC_BLOCH, s->N, s->nx, s->ny, s->nz, s->h, s->n_kb,
                             s->n_batches, s->d_wocc, s->dens_part, s->vloc, s->xc != TDKS_XC_NONE, El, half_A2,
                             s->aux, s->lda_part, lda_blocks(s->N), s->stream,
                             (s->xfn || hartree) ? s->n_total : nullptr, hartree ? s->d_vh : nullptr, sums ? 1 : 0);
  s->launches++;
  if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("lda: ") + cudaGetErrorString(e));
  return TDKS_OK;
}

int run_finalize(tdks_system *s, double *rec, double t_state, const double E[3], const double A[3]) {
  const double h3 = s->h * s->h * s->h;
  const double omega_cell = (double)s->N * h3;
  long n_part = s->obs_count;
  if (s->bc == TDKS_BC_BLOCH && s->n_atoms > 0) {
    // the projectors' commutator in the current: partial records after the sweep's
    const long extra = (long)s->n_atoms * s->n_kb * s->BS;
    if (n_part + extra > s->obs_cap) return fail(TDKS_EDEVICE, "observable partials exceed their buffer");
    NlCurrentParams q{};
    q.prec = s->prec; q.BS = s->BS; q.n_batches = s->n_batches; q.n_kb = s->n_kb; q.n_atoms = s->n_atoms;
    q.N = s->N; q.psi = s->psi; q.psi_lo = s->psi_lo; q.atom_begin = s->d_atom_begin; q.ent = s->d_ent;
    q.D = s->d_D; q.kvec = s->d_kvec; q.wocc = s->d_wocc; q.h3 = h3;
    for (int a = 0; a < 3; a++) q.A[a] = s->gauge == TDKS_GAUGE_VELOCITY ? A[a] : 0.0;
    q.out = s->obs_part + n_part * 4;
    cudaError_t e = launch_nl_current(q, s->stream);
    s->launches++;
    if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("non-local current: ") + cudaGetErrorString(e));
    n_part += extra;
  }
  double fv = 0.0;
  for (int a = 0; a < 3; a++) fv += (s->gauge == TDKS_GAUGE_VELOCITY ? A[a] : E[a]) * s->pol[a];
  const double Az[3] = {0, 0, 0};
  if (s->xfn) {  // state-parallel: band energy and currents summed over the ranks
    cudaError_t e = launch_finalize_sums(s->obs_part, n_part, s->lda_part, lda_blocks(s->N), s->fin_part,
                                         s->fin_sum, s->stream);
    s->launches += 2;
    if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("finalize: ") + cudaGetErrorString(e));
    if (int r = s->xfn(s->fin_sum, 4, (void *)s->stream, s->xctx))
      return fail(TDKS_EDEVICE, "exchange hook failed on the record sums (" + std::to_string(r) + ")");
    e = launch_record_from_sums(s->fin_sum, rec, t_state, h3, s->occ, s->bc == TDKS_BC_BLOCH, omega_cell,
                                s->gauge == TDKS_GAUGE_VELOCITY ? A : Az, fv, s->stream);
    s->launches++;
    if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("record: ") + cudaGetErrorString(e));
    return TDKS_OK;
  }
  Timed tm(s, 2);
  cudaError_t e = launch_finalize(s->obs_part, n_part, s->lda_part, lda_blocks(s->N), rec, t_state, h3,
                                  s->occ, s->bc == TDKS_BC_BLOCH, omega_cell,
                                  s->gauge == TDKS_GAUGE_VELOCITY ? A : Az, fv, s->fin_part, s->stream);
  s->launches += 2;
  if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("finalize: ") + cudaGetErrorString(e));
  return TDKS_OK;
}

// Sweep 1 of a sub-step (or an observation): term[0] = coef * H psi, with the energy
// and current partial sums when `obs` is set.
int first_sweep(tdks_system *s, double cr, double ci, const double A[3], bool obs) {
  int rc = run_gather(s, s->psi, A);
  if (rc) return rc;
  SweepParams p{};
  sweep_common(s, p, A, 0);
  set_coef(p, cr, ci);
  p.in = s->psi;
  p.out = s->term[0];
  p.do_obs = obs ? 1 : 0;
  if (obs && s->bc == TDKS_BC_BLOCH) p.grad_mask |= 8;
  // without observables the first term is a middle-term sweep over the state: the same
  // arithmetic, without the energy accumulators (whose registers cost the sweep ~8%)
  return run_sweep(s, obs ? MODE_FIRST : MODE_MID, p, s->tmaps_ok ? &s->smaps[0] : nullptr, 0);
}

// Gershgorin-type bound on |lambda| of H: kinetic maximum (the +/- alternating mode of
// the stencil), |V_loc|, exchange of a dense region, field terms, projector norms.
double h_bound(const tdks_system *s, double dt_hint) {
  double c[MAXM + 1], d[MAXM + 1];
  fd_weights(s->M, c, d);
  double smax = -c[0];
  for (int m = 1; m <= s->M; m++) smax -= 2.0 * c[m] * ((m % 2) ? -1.0 : 1.0);
  double dmax = 0.0;
  for (int m = 1; m <= s->M; m++) dmax += std::fabs(d[m]);
  dmax *= 2.0 / s->h;
  double kin = 3.0 * smax / (2.0 * s->h * s->h);
  double bound = kin + s->vloc_absmax + s->vnl_bound + 2.0;  // 2 Ha covers v_x at n <= 10
  const double Lmax = 0.5 * std::max(s->nx, std::max(s->ny, s->nz)) * s->h * std::sqrt(3.0);
  if (s->gauge == TDKS_GAUGE_LENGTH) bound += std::fabs(s->amp) * Lmax;
  if (s->gauge == TDKS_GAUGE_VELOCITY) bound += std::fabs(s->amp) * dmax + 0.5 * s->amp * s->amp;
  (void)dt_hint;
  return bound;
}

double kinetic_max(const tdks_system *s) {
  double c[MAXM + 1], d[MAXM + 1];
  fd_weights(s->M, c, d);
  double smax = -c[0];
  for (int m = 1; m <= s->M; m++) smax -= 2.0 * c[m] * ((m % 2) ? -1.0 : 1.0);
  return 3.0 * smax / (2.0 * s->h * s->h);
}

void free_proj(tdks_system *s) {
  cudaFree(s->d_rowent); cudaFree(s->d_atom_begin);
  cudaFree(s->d_ent); cudaFree(s->d_q); cudaFree(s->d_D); cudaFree(s->d_qpart);
  cudaFree(s->d_ent_beta); cudaFree(s->d_ent_ca); cudaFree(s->d_phase);
  s->d_ent_beta = nullptr; s->d_ent_ca = nullptr; s->d_phase = nullptr;
  s->phase_ok = false;
  cudaFree(s->d_sp); cudaFree(s->d_nl);
  s->d_rowent = s->d_atom_begin = nullptr;
  s->d_sp = nullptr; s->d_nl = nullptr;
  s->n_sp = s->n_ent = 0;
  if (s->aux) cudaMemsetAsync(s->aux, 0, s->N * sizeof(PointAux), s->stream);  // no entries anywhere
  s->d_ent = nullptr; s->d_q = nullptr; s->d_D = nullptr; s->d_qpart = nullptr;
  s->n_atoms = 0;
  s->vnl_bound = 0.0;
}

// After a stream synchronise: report a kernel that gave up a bounded wait.
int check_err(tdks_system *s) {
  int h = 0;
  CU(cudaMemcpy(&h, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    CU(cudaMemset(s->d_err, 0, 2 * sizeof(int)));  // and the work counter an aborted sweep left
    return fail(TDKS_ETIMEOUT, "a sweep kernel gave up waiting for its TMA copies");
  }
  return TDKS_OK;
}

double coord_of(const tdks_system *s, int axis, int i) {
  const int n = axis == 0 ? s->nx : (axis == 1 ? s->ny : s->nz);
  if (s->bc == TDKS_BC_ZERO) return ((double)i - 0.5 * (double)(n - 1)) * s->h;
  return (double)i * s->h;
}

}  // namespace

extern "C" {

const char *tdks_last_error(void) { return g_err.c_str(); }

int tdks_create_grid(int nx, int ny, int nz, double h, int fd_order, int bc, int prec, int n_orb, int n_k,
                     const double *kpts, const double *kweights, void *stream, tdks_sys *out) {
  if (!out) return fail(TDKS_EINVAL, "out is NULL");
  *out = nullptr;
  if (fd_order != 4 && fd_order != 8) return fail(TDKS_EINVAL, "fd_order must be 4 or 8");
  const int M = fd_order / 2;
  if (bc != TDKS_BC_ZERO && bc != TDKS_BC_BLOCH) return fail(TDKS_EINVAL, "bc must be TDKS_BC_ZERO or TDKS_BC_BLOCH");
  if (prec != TDKS_C128 && prec != TDKS_C64) return fail(TDKS_EINVAL, "prec must be TDKS_C128 or TDKS_C64");
  const int nmin = bc == TDKS_BC_BLOCH ? M : M + 1;
  if (nx < nmin || ny < nmin || nz < nmin) return fail(TDKS_EINVAL, "grid too small for the stencil");
  if (!(h > 0.0)) return fail(TDKS_EINVAL, "h must be > 0");
  if (n_orb < 1 || n_k < 1) return fail(TDKS_EINVAL, "n_orb and n_k must be >= 1");
  if (bc == TDKS_BC_ZERO && n_k != 1) return fail(TDKS_EINVAL, "a finite box takes exactly one k-point");
  const long N = (long)nx * ny * nz;
  if (N > (1L << 30)) return fail(TDKS_EINVAL, "grid larger than 2^30 points");
  tdks_system *s = new (std::nothrow) tdks_system();
  if (!s) return fail(TDKS_ENOMEM, "host allocation");
  s->nx = nx; s->ny = ny; s->nz = nz; s->h = h; s->M = M; s->bc = bc; s->prec = prec;
  s->n_orb = n_orb; s->n_k = n_k; s->N = N;
  s->BS = prec == TDKS_C64 ? 2 * OVC : OVC;
  s->n_batches = (n_orb + s->BS - 1) / s->BS;
  s->n_kb = n_k * s->n_batches;
  s->stream = (cudaStream_t)stream;
  s->kpts.assign(3 * n_k, 0.0);
  s->kw.assign(n_k, 1.0 / n_k);
  if (kpts) for (int i = 0; i < 3 * n_k; i++) s->kpts[i] = kpts[i];
  if (kweights) for (int i = 0; i < n_k; i++) s->kw[i] = kweights[i];
  cudaGetDevice(&s->dev);
  const size_t pts = (size_t)s->n_kb * N;
  s->term_bytes = pts * OVC * 16;
  s->state_bytes = s->term_bytes;
  const int nlda = lda_blocks(N);
  auto cleanup = [&](int code, const std::string &m) { tdks_destroy(s); return fail(code, m); };
#define ALLOC(ptr, bytes)                                                                    \
  do {                                                                                       \
    cudaError_t e_ = cudaMalloc((void **)&(ptr), (bytes));                                   \
    if (e_ != cudaSuccess) { cudaGetLastError(); return cleanup(TDKS_ENOMEM, std::string("cudaMalloc ") + #ptr); } \
  } while (0)
  ALLOC(s->psi, s->state_bytes);
  if (prec == TDKS_C64) ALLOC(s->psi_lo, s->state_bytes);
  for (int i = 0; i < 3; i++) ALLOC(s->term[i], s->term_bytes);
  ALLOC(s->d_err, 2 * sizeof(int));
  ALLOC(s->vloc, N * sizeof(double));
  ALLOC(s->aux, N * sizeof(PointAux));
  ALLOC(s->dens_part, pts * sizeof(double));
  ALLOC(s->lda_part, (size_t)nlda * 6 * sizeof(double));
  s->zc = 0;
  // obs partials sized for the most records a first sweep can write: the smallest tile of
  // the general sweep, or the warp-specialised sweep's per-warp records (z chunks of 1 plane)
  {
    const long items_gen = (long)((nx + 7) / 8) * ((ny + 3) / 4) * s->n_kb * nz;
    long items_ws = 0;
    for (int sh = 0; sh < WS_SHAPES; sh++) {
      int tx = 16, ty = 8, warps = 8;
      ws_shape_info(sh, &tx, &ty, nullptr, &warps);
      items_ws = std::max(items_ws, (long)((nx + tx - 1) / tx) * ((ny + ty - 1) / ty) * s->n_kb * nz * warps);
    }
    s->obs_cap = s->obs_base = std::max(items_gen, items_ws);
    ALLOC(s->obs_part, (size_t)s->obs_cap * 4 * sizeof(double));
  }
  ALLOC(s->ring, (size_t)tdks_system::RING * TDKS_RECORD * sizeof(double));
  ALLOC(s->fin_part, (size_t)FIN_BLOCKS * 10 * sizeof(double));
  ALLOC(s->obs_rec, TDKS_RECORD * sizeof(double));
  ALLOC(s->d_kvec, 3 * n_k * sizeof(double));
  ALLOC(s->d_wocc, n_k * sizeof(double));
#undef ALLOC
  if (cudaMemcpy(s->d_kvec, s->kpts.data(), 3 * n_k * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemsetAsync(s->vloc, 0, N * sizeof(double), s->stream) != cudaSuccess ||
      cudaMemsetAsync(s->aux, 0, N * sizeof(PointAux), s->stream) != cudaSuccess ||
      cudaMemsetAsync(s->psi, 0, s->state_bytes, s->stream) != cudaSuccess ||
      (s->psi_lo && cudaMemsetAsync(s->psi_lo, 0, s->state_bytes, s->stream) != cudaSuccess) ||
      cudaMemsetAsync(s->d_err, 0, 2 * sizeof(int), s->stream) != cudaSuccess)
    return cleanup(TDKS_EDEVICE, "initial copies");
  build_tmaps(s);
  std::vector<double> wocc(n_k);
  for (int i = 0; i < n_k; i++) wocc[i] = s->kw[i] * s->occ;
  if (cudaMemcpy(s->d_wocc, wocc.data(), n_k * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return cleanup(TDKS_EDEVICE, "initial copies");
  *out = s;
  return TDKS_OK;
}

int tdks_destroy(tdks_sys s) {
  if (!s) return TDKS_OK;
  cudaStreamSynchronize(s->stream);
  free_proj(s);
  cudaFree(s->psi);
  cudaFree(s->psi_lo);
  cudaFree(s->d_err);
  for (int i = 0; i < 3; i++) cudaFree(s->term[i]);
  cudaFree(s->vloc); cudaFree(s->aux); cudaFree(s->dens_part); cudaFree(s->lda_part);
  cudaFree(s->obs_part); cudaFree(s->ring); cudaFree(s->fin_part);
  for (int j = 0; j < 4; j++) cudaFree(s->vx_hist[j]);
  cudaFree(s->etrs_save); cudaFree(s->etrs_save_lo);
  cudaFree(s->n_total); cudaFree(s->fin_sum);
  cudaFree(s->obs_rec); cudaFree(s->d_kvec); cudaFree(s->d_wocc);
  cudaFree(s->staging);
  tsurff_free(s);
  hartree_free(s);
  if (s->pack_stream) cudaStreamSynchronize(s->pack_stream);
  cudaFree(s->psi_b); cudaFree(s->psi_lo_b); cudaFree(s->dens_b);
  if (s->pack_stream) cudaStreamDestroy(s->pack_stream);
  if (s->ev_spare_free) cudaEventDestroy(s->ev_spare_free);
  if (s->ev_packed) cudaEventDestroy(s->ev_packed);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->ev_staging_free) cudaEventDestroy(s->ev_staging_free);
  for (auto e : s->ev_chunk) cudaEventDestroy(e);
  for (auto &u : s->ev_used) { cudaEventDestroy(u.second.first); cudaEventDestroy(u.second.second); }
  for (auto e : s->ev_free) cudaEventDestroy(e);
  delete s;
  return TDKS_OK;
}

int tdks_set_local_potential(tdks_sys s, const double *v) {
  if (!s || !v) return fail(TDKS_EINVAL, "NULL argument");
  double mx = 0.0;
  for (long i = 0; i < s->N; i++) mx = std::max(mx, std::fabs(v[i]));
  s->vloc_absmax = mx;
  CU(cudaMemcpyAsync(s->vloc, v, s->N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  CU(cudaStreamSynchronize(s->stream));
  return TDKS_OK;
}

static int ensure_staging(tdks_system *s) {
  if (s->staging) return TDKS_OK;
  CU(cudaMalloc((void **)&s->staging, (size_t)s->n_k * s->N * s->n_orb * 16));
  return TDKS_OK;
}

// The upload runs in chunks (point ranges of each k-point) on a copy stream; each chunk is
// packed into the internal layout, with its density partials, on the system stream as soon
// as it has landed, so packing overlaps the remaining copies.
constexpr int UPLOAD_CHUNKS = 8;

int tdks_set_orbitals(tdks_sys s, const double *psi) {
  if (!s || !psi) return fail(TDKS_EINVAL, "NULL argument");
  int rc = ensure_staging(s);
  if (rc) return rc;
  const int per_k = std::max(1, (UPLOAD_CHUNKS + s->n_k - 1) / s->n_k);
  const int n_chunks = per_k * s->n_k;
  if (!s->copy_stream) {
    CU(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&s->ev_staging_free, cudaEventDisableTiming));
  }
  while ((int)s->ev_chunk.size() < n_chunks) {
    cudaEvent_t e;
    CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    s->ev_chunk.push_back(e);
  }
  // With two upload buffers the upload packs into the spares on their own stream, so that the
  // packing too overlaps the work enqueued before this call; the system then switches to them
  // for the work enqueued after it.  With one, it packs in place on the system's stream.
  const bool twin = s->upload_buffers == 2;
  cudaStream_t ps = twin ? s->pack_stream : s->stream;
  void *dst = twin ? s->psi_b : s->psi, *dst_lo = twin ? s->psi_lo_b : s->psi_lo;
  double *dst_dens = twin ? s->dens_b : s->dens_part;
  // the spares are written only once the work that used them as the state is done
  if (twin && s->spare_pending) CU(cudaStreamWaitEvent(ps, s->ev_spare_free, 0));
  // the copies overwrite the staging buffer only once the kernels that read it (the previous
  // upload's packing) are done; they do not wait for other work of the system, so an upload
  // issued right after tdks_propagate_n overlaps that propagation
  if (s->staging_pending) CU(cudaStreamWaitEvent(s->copy_stream, s->ev_staging_free, 0));
  const long len = (s->N + per_k - 1) / per_k;
  int c = 0;
  for (int k = 0; k < s->n_k; k++)
    for (long pt0 = 0; pt0 < s->N; pt0 += len, c++) {
      const long npts = std::min(len, s->N - pt0);
      const size_t off = ((size_t)k * s->N + pt0) * s->n_orb * 2;  // doubles
      CU(cudaMemcpyAsync(s->staging + off, psi + off, (size_t)npts * s->n_orb * 16, cudaMemcpyHostToDevice,
                         s->copy_stream));
      CU(cudaEventRecord(s->ev_chunk[c], s->copy_stream));
      CU(cudaStreamWaitEvent(ps, s->ev_chunk[c], 0));
      CU(launch_pack_in(s->prec, s->N, k, pt0, npts, s->n_orb, s->n_batches, s->staging, dst, dst_lo, s->d_wocc,
                        dst_dens, ps));
      s->launches++;
    }
  CU(cudaEventRecord(s->ev_staging_free, ps));
  s->staging_pending = true;
  if (twin) {
    // work enqueued from now on reads the new state once it is packed; the old state becomes
    // the spare once the work enqueued so far is done
    CU(cudaEventRecord(s->ev_packed, ps));
    CU(cudaStreamWaitEvent(s->stream, s->ev_packed, 0));
    std::swap(s->psi, s->psi_b);
    std::swap(s->psi_lo, s->psi_lo_b);
    std::swap(s->dens_part, s->dens_b);
    CU(cudaEventRecord(s->ev_spare_free, s->stream));
    s->spare_pending = true;
    build_tmaps(s);
  }
  // the host buffer has been read once the copies are done ("copied")
  CU(cudaStreamSynchronize(s->copy_stream));
  s->have_orbitals = true;
  s->dens_valid = true;
  s->n_hist = 0;  // a new state starts a new CFM4 exchange history
  return TDKS_OK;
}

int tdks_set_upload_buffers(tdks_sys s, int n) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (n != 1 && n != 2) return fail(TDKS_EINVAL, "upload buffers must be 1 or 2");
  if (n == s->upload_buffers) return TDKS_OK;
  CU(cudaStreamSynchronize(s->stream));
  if (s->pack_stream) CU(cudaStreamSynchronize(s->pack_stream));
  if (n == 2) {
    CU(cudaMalloc(&s->psi_b, s->state_bytes));
    if (s->psi_lo) CU(cudaMalloc(&s->psi_lo_b, s->state_bytes));
    CU(cudaMalloc((void **)&s->dens_b, (size_t)s->n_kb * s->N * sizeof(double)));
    if (!s->pack_stream) {
      CU(cudaStreamCreateWithFlags(&s->pack_stream, cudaStreamNonBlocking));
      CU(cudaEventCreateWithFlags(&s->ev_spare_free, cudaEventDisableTiming));
      CU(cudaEventCreateWithFlags(&s->ev_packed, cudaEventDisableTiming));
    }
  } else {
    cudaFree(s->psi_b); cudaFree(s->psi_lo_b); cudaFree(s->dens_b);
    s->psi_b = s->psi_lo_b = nullptr;
    s->dens_b = nullptr;
  }
  s->spare_pending = false;
  s->upload_buffers = n;
  return TDKS_OK;
}

int tdks_get_orbitals(tdks_sys s, double *psi_out) {
  if (!s || !psi_out) return fail(TDKS_EINVAL, "NULL argument");
  int rc = ensure_staging(s);
  if (rc) return rc;
  CU(launch_pack(s->prec, 0, s->N, s->n_k, s->n_orb, s->n_batches, s->psi, s->psi_lo, s->staging, s->stream));
  s->launches++;
  CU(cudaMemcpyAsync(psi_out, s->staging, (size_t)s->n_k * s->N * s->n_orb * 16, cudaMemcpyDeviceToHost,
                     s->stream));
  CU(cudaStreamSynchronize(s->stream));
  return check_err(s);
}

int tdks_set_atoms_projectors(tdks_sys s, int n_atoms, const double *pos, const double *D, double r_c,
                              double r_cut) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (n_atoms < 0) return fail(TDKS_EINVAL, "n_atoms < 0");
  CU(cudaStreamSynchronize(s->stream));
  free_proj(s);
  if (n_atoms == 0) return TDKS_OK;
  if (!pos || !D || !(r_c > 0.0) || !(r_cut > 0.0)) return fail(TDKS_EINVAL, "bad projector arguments");
  const int n[3] = {s->nx, s->ny, s->nz};
  std::vector<ProjEntry> ent;
  std::vector<int> atom_begin(n_atoms + 1, 0);
  double vnl = 0.0;
  const double h3 = s->h * s->h * s->h;
  for (int a = 0; a < n_atoms; a++) {
    atom_begin[a] = (int)ent.size();
    const double *R = pos + 3 * a;
    int lo[3], hi[3];
    for (int ax = 0; ax < 3; ax++) {
      if (s->bc == TDKS_BC_ZERO) {
        const double c0 = 0.5 * (n[ax] - 1);
        lo[ax] = std::max(0, (int)std::floor((R[ax] - r_cut) / s->h + c0) - 1);
        hi[ax] = std::min(n[ax] - 1, (int)std::ceil((R[ax] + r_cut) / s->h + c0) + 1);
      } else {
        lo[ax] = (int)std::floor((R[ax] - r_cut) / s->h) - 1;
        hi[ax] = (int)std::ceil((R[ax] + r_cut) / s->h) + 1;
      }
    }
    double nb[4] = {0, 0, 0, 0};
    for (int iz = lo[2]; iz <= hi[2]; iz++)
      for (int iy = lo[1]; iy <= hi[1]; iy++)
        for (int ix = lo[0]; ix <= hi[0]; ix++) {
          const int ii[3] = {ix, iy, iz};
          double dd[3], r2 = 0.0;
          for (int ax = 0; ax < 3; ax++) {
            const double u = s->bc == TDKS_BC_ZERO ? coord_of(s, ax, ii[ax]) : (double)ii[ax] * s->h;
            dd[ax] = u - R[ax];
            r2 += dd[ax] * dd[ax];
          }
          if (r2 > r_cut * r_cut) continue;
          ProjEntry e{};
          int cc[3];
          for (int ax = 0; ax < 3; ax++) {
            int w = ii[ax] >= 0 ? ii[ax] / n[ax] : -((-ii[ax] - 1) / n[ax]) - 1;
            cc[ax] = ii[ax] - w * n[ax];
            e.T[ax] = (double)(w * n[ax]) * s->h;
            e.d[ax] = dd[ax];
          }
          e.cell = (cc[2] * s->ny + cc[1]) * s->nx + cc[0];
          e.atom = a;
          const double g = std::exp(-r2 / (2.0 * r_c * r_c));
          const double b[4] = {g, dd[0] * g, dd[1] * g, dd[2] * g};
          for (int j = 0; j < 4; j++) {
            e.betad[j] = b[j];
            e.beta[j] = (float)b[j];
            nb[j] += b[j] * b[j] * h3;
          }
          ent.push_back(e);
        }
    for (int j = 0; j < 4; j++) vnl += std::fabs(D[4 * a + j]) * nb[j];
  }
  atom_begin[n_atoms] = (int)ent.size();
  if (ent.empty()) return TDKS_OK;
  // point-major CSR for the scatter (entries in ascending entry order per point)
  std::vector<int> rowptr(s->N + 1, 0), rowent(ent.size());
  for (auto &e : ent) rowptr[e.cell + 1]++;
  for (long i = 0; i < s->N; i++) rowptr[i + 1] += rowptr[i];
  {
    std::vector<int> fill(rowptr.begin(), rowptr.end() - 1);
    for (size_t i = 0; i < ent.size(); i++) rowent[fill[ent[i].cell]++] = (int)i;
  }
  CU(cudaMalloc((void **)&s->d_rowent, ent.size() * sizeof(int)));
  CU(cudaMalloc((void **)&s->d_atom_begin, (n_atoms + 1) * sizeof(int)));
  CU(cudaMalloc((void **)&s->d_ent, ent.size() * sizeof(ProjEntry)));
  CU(cudaMalloc((void **)&s->d_q, (size_t)s->n_kb * n_atoms * 4 * OVC * 16));
  s->gchunks = gather_chunks((long)n_atoms * s->n_kb);
  CU(cudaMalloc((void **)&s->d_qpart, (size_t)s->n_kb * n_atoms * s->gchunks * 4 * OVC * 2 * sizeof(double2)));
  CU(cudaMalloc((void **)&s->d_D, (size_t)n_atoms * 4 * sizeof(double)));
  {
    // per-point entry ranges (V_eff is rewritten by the LDA kernel before every sweep)
    std::vector<PointAux> aux(s->N);
    std::vector<int2> sp;
    for (long i = 0; i < s->N; i++) {
      aux[i] = PointAux{0.0, rowptr[i], rowptr[i + 1]};
      if (rowptr[i + 1] > rowptr[i]) sp.push_back(make_int2(rowptr[i], rowptr[i + 1]));
    }
    CU(cudaMemcpy(s->aux, aux.data(), s->N * sizeof(PointAux), cudaMemcpyHostToDevice));
    s->n_sp = (int)sp.size();
    s->n_ent = (int)ent.size();
    CU(cudaMalloc((void **)&s->d_sp, sp.size() * sizeof(int2)));
    CU(cudaMemcpy(s->d_sp, sp.data(), sp.size() * sizeof(int2), cudaMemcpyHostToDevice));
    // one 16-byte vector per (kb, entry row, v) plus a zero row per kb
    const size_t nl_bytes = (size_t)s->n_kb * (s->n_ent + 1) * OVC * 16;
    CU(cudaMalloc(&s->d_nl, nl_bytes));
    CU(cudaMemset(s->d_nl, 0, nl_bytes));
  }
  CU(cudaMemcpy(s->d_rowent, rowent.data(), ent.size() * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(s->d_atom_begin, atom_begin.data(), (n_atoms + 1) * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(s->d_ent, ent.data(), ent.size() * sizeof(ProjEntry), cudaMemcpyHostToDevice));
  {
    std::vector<float4> eb(ent.size());
    std::vector<int2> eca(ent.size());
    for (size_t i = 0; i < ent.size(); i++) {
      eb[i] = make_float4(ent[i].beta[0], ent[i].beta[1], ent[i].beta[2], ent[i].beta[3]);
      eca[i] = make_int2(ent[i].cell, ent[i].atom);
    }
    CU(cudaMalloc((void **)&s->d_ent_beta, ent.size() * sizeof(float4)));
    CU(cudaMalloc((void **)&s->d_ent_ca, ent.size() * sizeof(int2)));
    CU(cudaMemcpy(s->d_ent_beta, eb.data(), ent.size() * sizeof(float4), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(s->d_ent_ca, eca.data(), ent.size() * sizeof(int2), cudaMemcpyHostToDevice));
  }
  CU(cudaMemcpy(s->d_D, D, (size_t)n_atoms * 4 * sizeof(double), cudaMemcpyHostToDevice));
  if (s->bc == TDKS_BC_BLOCH) {
    // room for the projectors' current records after the sweep partials
    const long need = s->obs_base + (long)n_atoms * s->n_kb * s->BS;
    double *grown = nullptr;
    CU(cudaMalloc((void **)&grown, (size_t)need * 4 * sizeof(double)));
    cudaFree(s->obs_part);
    s->obs_part = grown;
    s->obs_cap = need;
  }
  s->n_atoms = n_atoms;
  s->pos.assign(pos, pos + 3 * n_atoms);
  s->D.assign(D, D + 4 * n_atoms);
  s->r_c = r_c;
  s->r_cut = r_cut;
  s->vnl_bound = vnl;
  return TDKS_OK;
}

int tdks_set_field(tdks_sys s, int gauge, const double pol[3], double amp, double omega, int envelope,
                   double t_total) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (gauge < 0 || gauge > 2) return fail(TDKS_EINVAL, "bad gauge");
  if (gauge == TDKS_GAUGE_LENGTH && s->bc != TDKS_BC_ZERO)
    return fail(TDKS_EINVAL, "the length gauge needs a finite box (E.r is not periodic)");
  if (gauge == TDKS_GAUGE_VELOCITY && s->bc != TDKS_BC_BLOCH)
    return fail(TDKS_EINVAL, "the velocity gauge is implemented for periodic cells");
  if (envelope != TDKS_ENV_NONE && envelope != TDKS_ENV_SIN2) return fail(TDKS_EINVAL, "bad envelope");
  if (envelope == TDKS_ENV_SIN2 && !(t_total > 0.0)) return fail(TDKS_EINVAL, "t_total must be > 0");
  s->gauge = gauge;
  if (pol) for (int a = 0; a < 3; a++) s->pol[a] = pol[a];
  s->amp = amp; s->omega = omega; s->envelope = envelope; s->t_total = t_total;
  return TDKS_OK;
}

int tdks_set_xc(tdks_sys s, int xc, double occupation) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (xc != TDKS_XC_NONE && xc != TDKS_XC_LDA_X && xc != TDKS_XC_LDA_X_HARTREE) return fail(TDKS_EINVAL, "bad xc");
  if (!(occupation > 0.0)) return fail(TDKS_EINVAL, "occupation must be > 0");
  if (xc == TDKS_XC_LDA_X_HARTREE)
    if (int rc = hartree_setup(s)) return rc;
  s->xc = xc;
  s->occ = occupation;
  std::vector<double> wocc(s->n_k);
  for (int i = 0; i < s->n_k; i++) wocc[i] = s->kw[i] * s->occ;
  CU(cudaMemcpyAsync(s->d_wocc, wocc.data(), s->n_k * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  CU(cudaStreamSynchronize(s->stream));
  s->dens_valid = false;
  return TDKS_OK;
}

int tdks_layout(tdks_sys s, int *bs, int *n_batches, int *elem_bytes, long long *bytes) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (bs) *bs = s->BS;
  if (n_batches) *n_batches = s->n_batches;
  if (elem_bytes) *elem_bytes = s->prec == TDKS_C64 ? 8 : 16;
  if (bytes) *bytes = (long long)s->term_bytes;
  return TDKS_OK;
}

int tdks_set_tile(tdks_sys s, int tx, int ty, int zc) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  const bool ok = (tx == 16 && ty == 8) || (tx == 32 && ty == 4) || (tx == 8 && ty == 8);
  if (!ok) return fail(TDKS_EINVAL, "tile must be one of 16x8, 32x4, 8x8");
  if (zc < 0) return fail(TDKS_EINVAL, "zc < 0");
  CU(cudaStreamSynchronize(s->stream));
  s->tx = tx; s->ty = ty; s->zc = zc;
  build_tmaps(s);
  return TDKS_OK;
}

int tdks_set_failure_injection(tdks_sys s, int withhold) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  CU(cudaStreamSynchronize(s->stream));
  s->withhold = withhold ? 1 : 0;
  return TDKS_OK;
}

int tdks_set_sweep_path(tdks_sys s, int path) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (path < 0 || path > 2)
    return fail(TDKS_EINVAL, "path must be 0 (TMA where possible), 1 (general) or 2 (TMA, lockstep warps)");
  s->path = path;
  build_tmaps(s);  // the box depth of the maps depends on the kernel variant
  return TDKS_OK;
}

int tdks_sweep_shape_info(int shape, int *count, int *tx, int *ty, int *rows, int *warps) {
  if (count) *count = WS_SHAPES;
  if (!ws_shape_info(shape, tx, ty, rows, warps)) return fail(TDKS_EINVAL, "no such sweep shape");
  return TDKS_OK;
}

int tdks_set_sweep_shape(tdks_sys s, int sweep, int shape) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (sweep < -1 || sweep > 3) return fail(TDKS_EINVAL, "sweep must be 0..3 or -1");
  if (!ws_shape_info(shape, nullptr, nullptr, nullptr, nullptr)) return fail(TDKS_EINVAL, "no such sweep shape");
  CU(cudaStreamSynchronize(s->stream));
  for (int i = 0; i < 4; i++)
    if (sweep < 0 || sweep == i) s->wshape[i] = shape;
  build_tmaps(s);
  return TDKS_OK;
}

int tdks_get_sweep_shape(tdks_sys s, int sweep, int *shape) {
  if (!s || !shape) return fail(TDKS_EINVAL, "NULL argument");
  if (sweep < 0 || sweep > 3) return fail(TDKS_EINVAL, "sweep must be 0..3");
  *shape = s->wshape[sweep];
  return TDKS_OK;
}

// One timed Taylor-term sweep of the autotuner: sweep 0 reads the state and writes t1,
// sweeps 1 and 2 read t(k-1) and write t(k); sweep 3 reads t3 and combines into t1/t2 in
// place of the state (state hi <- t1, state lo <- t2), so the state itself is untouched.
static int tune_launch(tdks_system *s, int sweep) {
  // in the velocity gauge, a vector potential along the field's polarisation, so that the
  // timed sweeps carry the gauge term the propagation's sweeps carry
  double At[3] = {0.0, 0.0, 0.0};
  if (s->gauge == TDKS_GAUGE_VELOCITY)
    for (int a = 0; a < 3; a++) At[a] = s->amp * s->pol[a];
  const int modes[4] = {MODE_FIRST, MODE_MID, MODE_MID, MODE_LAST};
  const int mode = modes[sweep];
  SweepParams p{};
  sweep_common(s, p, At, sweep);
  set_coef(p, 0.0, -0.01 / (sweep + 1));
  p.in = sweep == 0 ? s->psi : s->term[sweep - 1];
  SweepMaps tm;
  if (!encode_sweep_maps(s, p.in, mode, &tm, false, sweep)) return fail(TDKS_EDEVICE, "tensor map encoding failed");
  if (mode == MODE_LAST) {
    int tx = 16, ty = 8;
    ws_shape_info(s->wshape[sweep], &tx, &ty, nullptr, nullptr);
    const void *ops[4] = {s->term[0], s->term[1], s->term[0], s->term[1]};
    for (int j = 0; j < 4; j++)
      if (!encode_op_map(s, ops[j], &tm.op[j], tx, ty)) return fail(TDKS_EDEVICE, "tensor map encoding failed");
    p.psi = s->term[0];
    p.psi_lo = s->term[1];
    p.t1 = s->term[0];
    p.t2 = s->term[1];
  } else {
    p.out = s->term[sweep];
  }
  return run_sweep(s, mode, p, &tm, sweep);
}

int tdks_autotune(tdks_sys s, int reps, double *ms) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (reps < 1) return fail(TDKS_EINVAL, "reps < 1");
  if (ms)
    for (int i = 0; i < WS_SHAPES * 4; i++) ms[i] = -1.0;
  if (!ws_path(s)) return TDKS_OK;
  CU(cudaStreamSynchronize(s->stream));
  const int saved[4] = {s->wshape[0], s->wshape[1], s->wshape[2], s->wshape[3]};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(TDKS_EDEVICE, "cudaEventCreate");
  }
  double best[4] = {-1.0, -1.0, -1.0, -1.0};
  int pick[4] = {saved[0], saved[1], saved[2], saved[3]};
  int rc = TDKS_OK;
  for (int sh = 0; sh < WS_SHAPES && rc == TDKS_OK; sh++) {
    for (int i = 0; i < 4; i++) s->wshape[i] = sh;
    for (int sw = 0; sw < 4 && rc == TDKS_OK; sw++) {
      if ((rc = tune_launch(s, sw))) break;  // warm-up (and fills this sweep's output)
      cudaEventRecord(e0, s->stream);
      for (int r = 0; r < reps && rc == TDKS_OK; r++) rc = tune_launch(s, sw);
      cudaEventRecord(e1, s->stream);
      if (rc) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(TDKS_EDEVICE, "autotune timing"); break; }
      if ((rc = check_err(s))) break;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      const double per = (double)t / reps;
      if (ms) ms[sh * 4 + sw] = per;
      if (best[sw] < 0.0 || per < best[sw]) { best[sw] = per; pick[sw] = sh; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < 4; i++) s->wshape[i] = rc == TDKS_OK ? pick[i] : saved[i];
  build_tmaps(s);
  s->dens_valid = false;  // the last sweeps overwrote the density partials
  return rc;
}

int tdks_apply_H(tdks_sys s, double t, const void *dev_in, void *dev_out) {
  if (!s || !dev_in || !dev_out) return fail(TDKS_EINVAL, "NULL argument");
  if (dev_in == dev_out) return fail(TDKS_EINVAL, "dev_in and dev_out must differ");
  double E[3], A[3];
  field_at(s, t, E, A);
  int rc = TDKS_OK;
  if (s->have_orbitals) rc = ensure_density(s);
  else if (s->xc == TDKS_XC_LDA_X) return fail(TDKS_ESTATE, "LDA exchange needs the density of set orbitals");
  else CU(cudaMemsetAsync(s->dens_part, 0, (size_t)s->n_kb * s->N * sizeof(double), s->stream));
  if (rc) return rc;
  if ((rc = run_lda(s, E, A))) return rc;
  if ((rc = run_gather(s, dev_in, A))) return rc;
  SweepParams p{};
  sweep_common(s, p, A, 1);
  set_coef(p, 1.0, 0.0);
  p.in = dev_in;
  p.out = dev_out;
  SweepMaps tm;
  const bool have_tm = tma_path(s) && encode_sweep_maps(s, dev_in, MODE_MID, &tm, s->path == 2, 1);
  return run_sweep(s, MODE_MID, p, have_tm ? &tm : nullptr, 1);
}

int tdks_auto_substeps(tdks_sys s, double dt, int *substeps) {
  if (!s || !substeps) return fail(TDKS_EINVAL, "NULL argument");
  const double b = h_bound(s, dt);
  *substeps = std::max(1, (int)std::ceil(std::fabs(dt) * b / 2.5));
  return TDKS_OK;
}

// CFM4 constants (Sec. "New propagators for real-time TDDFT"): weights a1, a2 and the Gauss
// points t + theta_i ds of the two Hamiltonians.
static void cfm4_constants(double a[2], double theta[2]) {
  const double r3 = std::sqrt(3.0);
  a[0] = (3.0 - 2.0 * r3) / 12.0;
  a[1] = (3.0 + 2.0 * r3) / 12.0;
  theta[0] = 0.5 - r3 / 6.0;
  theta[1] = 0.5 + r3 / 6.0;
}

// One exponential factor of a sub-step ds of an exponential propagator: exp(-i tau H_eff)
// with tau = frac * ds and H_eff = H0 + v_eff + E_eff.r, where
//   E_eff = sum_i c[i] E(t + th[i] ds),  v_eff = sum_i c[i] v_x(t + th[i] ds),
// v_x at t + th ds extrapolated from its values at the starts of the last sub-steps.
struct ExpFactor {
  double frac;
  int n;
  double th[2], c[2];
};
struct ExpScheme {
  int n_exp;
  ExpFactor f[2];
  const char *name;
};

// CFM4: exp(-i ds (a1 H[t1] + a2 H[t2])) exp(-i ds (a2 H[t1] + a1 H[t2])), a1 + a2 = 1/2, so
// each factor is an exponential of ds/2 of 2 (a H[t1] + a' H[t2]).  EMR: exp(-i ds H[t + ds/2]).
// AETRS: exp(-i ds/2 H[t + ds]) exp(-i ds/2 H[t]).  (Factors listed in the order applied.)
static ExpScheme exp_scheme(int prop) {
  ExpScheme e{};
  if (prop == TDKS_PROP_CFM4) {
    double a[2], th[2];
    cfm4_constants(a, th);
    e.n_exp = 2;
    e.f[0] = ExpFactor{0.5, 2, {th[0], th[1]}, {2.0 * a[1], 2.0 * a[0]}};
    e.f[1] = ExpFactor{0.5, 2, {th[0], th[1]}, {2.0 * a[0], 2.0 * a[1]}};
    e.name = "CFM4";
  } else if (prop == TDKS_PROP_EMR) {
    e.n_exp = 1;
    e.f[0] = ExpFactor{1.0, 1, {0.5, 0.0}, {1.0, 0.0}};
    e.name = "EMR";
  } else {
    e.n_exp = 2;
    e.f[0] = ExpFactor{0.5, 1, {0.0, 0.0}, {1.0, 0.0}};
    e.f[1] = ExpFactor{0.5, 1, {1.0, 0.0}, {1.0, 0.0}};
    e.name = "AETRS";
  }
  return e;
}

// Weights of the exchange history (v_x at offsets 0, -1, .., -(nh-1) sub-steps, [0] the
// newest) in a factor's v_eff: sum_i c[i] times the Lagrange basis polynomials through the
// nh offsets, evaluated at th[i].
static void factor_history_weights(const ExpFactor &f, int nh, double w[4]) {
  for (int j = 0; j < 4; j++) w[j] = 0.0;
  for (int j = 0; j < nh; j++) {
    double acc = 0.0;
    for (int q = 0; q < f.n; q++) {
      double l = 1.0;
      for (int i = 0; i < nh; i++) {
        if (i == j) continue;
        l *= (f.th[q] + i) / (double)(i - j);
      }
      acc += f.c[q] * l;
    }
    w[j] = acc;
  }
}

// Taylor terms 2..4 of a sub-step of length dts (term 1 is already in term[0]); the last
// sweep adds the series into the state and writes its density.
static int taylor_tail(tdks_system *s, double dts, const double A[3]) {
  int rc = TDKS_OK;
  for (int k = 2; k <= 4; k++) {
    const void *in = s->term[k - 2];
    if ((rc = run_gather(s, in, A))) return rc;
    SweepParams p{};
    sweep_common(s, p, A, k - 1);
    set_coef(p, 0.0, -dts / k);
    p.in = in;
    if (k < 4) {
      p.out = s->term[k - 1];
      if ((rc = run_sweep(s, MODE_MID, p, s->tmaps_ok ? &s->smaps[k - 1] : nullptr, k - 1))) return rc;
    } else {
      p.psi = s->psi;
      p.psi_lo = s->psi_lo;
      p.t1 = s->term[0];
      p.t2 = s->term[1];
      if ((rc = run_sweep(s, MODE_LAST, p, s->tmaps_ok ? &s->smaps[3] : nullptr, 3))) return rc;
    }
  }
  return rc;
}

// V_eff of one CFM4 exponential (push: first store v_x of the current density as the newest
// history entry).
static int run_cfm_veff(tdks_system *s, bool push, int nh, const double w[4], const double E[3]) {
  const bool hartree = s->xc == TDKS_XC_LDA_X_HARTREE;
  // the pushed potential from the density as one FP64 array: every rank's states
  // (state-parallel propagation), and the source of v_H, which joins the pushed v_x
  const bool total = push && s->xc != TDKS_XC_NONE && (s->xfn || hartree);
  if (total) {
    cudaError_t e = launch_density_sum(s->prec, s->N, s->n_kb, s->n_batches, s->d_wocc, s->dens_part, s->n_total,
                                       s->stream);
    s->launches++;
    if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("density sum: ") + cudaGetErrorString(e));
    if (s->xfn)
      if (int r = s->xfn(s->n_total, (long long)s->N, (void *)s->stream, s->xctx))
        return fail(TDKS_EDEVICE, "exchange hook failed on the density (" + std::to_string(r) + ")");
    if (hartree)
      if (int rc = hartree_solve(s)) return rc;
  }
  CfmHist h{};
  for (int j = 0; j < 4; j++) h.v[j] = s->vx_hist[j];
  h.nh = s->xc != TDKS_XC_NONE ? nh : 0;
  for (int j = 0; j < 4; j++) h.w[j] = j < h.nh ? w[j] : 0.0;
  const double El[3] = {s->gauge == TDKS_GAUGE_LENGTH ? E[0] : 0.0, s->gauge == TDKS_GAUGE_LENGTH ? E[1] : 0.0,
                        s->gauge == TDKS_GAUGE_LENGTH ? E[2] : 0.0};
  Timed tm(s, 2);
  cudaError_t e = launch_cfm_veff(s->prec, s->bc == TDKS_BC_BLOCH, s->N, s->nx, s->ny, s->nz, s->h, s->n_kb,
                                  s->n_batches, s->d_wocc, s->dens_part, s->vloc, s->xc != TDKS_XC_NONE,
                                  push ? 1 : 0, h, El, s->aux, s->stream, total && hartree ? s->d_vh : nullptr,
                                  total ? s->n_total : nullptr);
  s->launches++;
  if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("cfm4 potential: ") + cudaGetErrorString(e));
  return TDKS_OK;
}

// Steps of an exponential propagator other than Taylor-4 (CFM4, EMR, AETRS; see
// tdks_set_propagator): per sub-step, v_x of the current state is pushed into the history,
// then each factor sets its effective potential and applies a Taylor-4 exponential.
static int propagate_exp(tdks_system *s, double t0, double dt, int n_steps, int substeps) {
  const ExpScheme sc = exp_scheme(s->prop);
  if (s->gauge == TDKS_GAUGE_VELOCITY)
    return fail(TDKS_EINVAL, std::string(sc.name) + " needs a field that enters H linearly (length gauge or no field)");
  const double ds = dt / substeps;
  double fmax = 0.0;
  for (int f = 0; f < sc.n_exp; f++) fmax = std::max(fmax, sc.f[f].frac);
  if (std::fabs(fmax * ds) * kinetic_max(s) > 2.0 * std::sqrt(2.0))
    return fail(TDKS_EUNSTABLE, std::string(sc.name) +
                                    " exponential beyond the Taylor-4 stability limit (tau * K_max > 2 sqrt 2)");
  int rc = ensure_density(s);
  if (rc) return rc;
  const double A0[3] = {0.0, 0.0, 0.0};
  const bool xc = s->xc != TDKS_XC_NONE;  // a density-dependent potential (v_x, v_x + v_H)
  for (int st = 0; st < n_steps; st++) {
    const double t = t0 + st * dt;
    for (int j = 0; j < substeps; j++) {
      const double tj = t + j * ds;
      if (j == 0) {
        // record of the state at t: the Hamiltonian of t + ds/2 with v_x of this state
        double E[3], A[3];
        field_at(s, tj + 0.5 * ds, E, A);
        if ((rc = run_lda(s, E, A))) return rc;
        if ((rc = first_sweep(s, 1.0, 0.0, A, true))) return rc;
        double *slot = s->ring + (s->steps % tdks_system::RING) * TDKS_RECORD;
        if ((rc = run_finalize(s, slot, t, E, A))) return rc;
      }
      if (xc) {  // the oldest history slot becomes the newest
        double *oldest = s->vx_hist[3];
        for (int q = 3; q > 0; q--) s->vx_hist[q] = s->vx_hist[q - 1];
        s->vx_hist[0] = oldest;
        s->n_hist = std::min(s->n_hist + 1, 4);
      }
      for (int f = 0; f < sc.n_exp; f++) {
        const ExpFactor &fa = sc.f[f];
        double Ef[3] = {0.0, 0.0, 0.0}, w[4] = {0, 0, 0, 0};
        for (int q = 0; q < fa.n; q++) {
          double Eq[3], Aq[3];
          field_at(s, tj + fa.th[q] * ds, Eq, Aq);
          for (int ax = 0; ax < 3; ax++) Ef[ax] += fa.c[q] * Eq[ax];
        }
        if (xc) factor_history_weights(fa, s->n_hist, w);
        if ((rc = run_cfm_veff(s, xc && f == 0, s->n_hist, w, Ef))) return rc;
        const double tau = fa.frac * ds;
        if ((rc = first_sweep(s, 0.0, -tau, A0, false))) return rc;
        if ((rc = taylor_tail(s, tau, A0))) return rc;
      }
      s->dens_valid = true;  // the last sweep wrote the density of the new state
    }
    s->steps++;
  }
  s->clock_t = t0 + n_steps * dt;
  s->clock_dt = dt;
  s->clock_substeps = substeps;
  return TDKS_OK;
}

// Enforced time-reversal symmetry with its trial state (see tdks_set_propagator): per sub-step
// ds, H[t] takes v_x of the current state; the trial exp(-i ds H[t]) phi runs on the state
// itself (saved first), and its density gives v_x at t + ds; then the saved state takes
// exp(-i ds/2 H[t]) and exp(-i ds/2 H[t + ds]).  History slots: [0] the newest v_x, [1] v_x(t)
// while the trial's is computed.
static int propagate_etrs(tdks_system *s, double t0, double dt, int n_steps, int substeps) {
  if (s->gauge == TDKS_GAUGE_VELOCITY)
    return fail(TDKS_EINVAL, "ETRS needs a field that enters H linearly (length gauge or no field)");
  const double ds = dt / substeps;
  if (std::fabs(ds) * kinetic_max(s) > 2.0 * std::sqrt(2.0))
    return fail(TDKS_EUNSTABLE, "ETRS trial exponential beyond the Taylor-4 stability limit (tau * K_max > 2 sqrt 2)");
  int rc = ensure_density(s);
  if (rc) return rc;
  const double A0[3] = {0.0, 0.0, 0.0};
  const bool xc = s->xc != TDKS_XC_NONE;  // a density-dependent potential (v_x, v_x + v_H)
  const double w_new[4] = {1.0, 0.0, 0.0, 0.0}, w_old[4] = {0.0, 1.0, 0.0, 0.0};
  auto exponential = [&](double tau) -> int {
    int r;
    if ((r = first_sweep(s, 0.0, -tau, A0, false))) return r;
    return taylor_tail(s, tau, A0);
  };
  auto copy_state = [&](void *dst, void *dst_lo, const void *src, const void *src_lo) -> int {
    CU(cudaMemcpyAsync(dst, src, s->state_bytes, cudaMemcpyDeviceToDevice, s->stream));
    if (src_lo) CU(cudaMemcpyAsync(dst_lo, src_lo, s->state_bytes, cudaMemcpyDeviceToDevice, s->stream));
    return TDKS_OK;
  };
  for (int st = 0; st < n_steps; st++) {
    const double t = t0 + st * dt;
    for (int j = 0; j < substeps; j++) {
      const double tj = t + j * ds;
      double E[3], A[3];
      if (j == 0) {
        // record of the state at t: the Hamiltonian of t + ds/2 with v_x of this state
        field_at(s, tj + 0.5 * ds, E, A);
        if ((rc = run_lda(s, E, A))) return rc;
        if ((rc = first_sweep(s, 1.0, 0.0, A, true))) return rc;
        double *slot = s->ring + (s->steps % tdks_system::RING) * TDKS_RECORD;
        if ((rc = run_finalize(s, slot, t, E, A))) return rc;
      }
      field_at(s, tj, E, A);
      // H[t]: v_x of the current state into slot 0
      if ((rc = run_cfm_veff(s, xc, 1, w_new, E))) return rc;
      if (xc) {
        if ((rc = copy_state(s->etrs_save, s->etrs_save_lo, s->psi, s->psi_lo))) return rc;
        if ((rc = exponential(ds))) return rc;  // the trial; its density now in dens_part
        std::swap(s->vx_hist[0], s->vx_hist[1]);
        // v_x of the trial into slot 0; V_eff stays H[t] (slot 1)
        if ((rc = run_cfm_veff(s, true, 2, w_old, E))) return rc;
        if ((rc = copy_state(s->psi, s->psi_lo, s->etrs_save, s->etrs_save_lo))) return rc;
      }
      if ((rc = exponential(0.5 * ds))) return rc;
      field_at(s, tj + ds, E, A);
      if ((rc = run_cfm_veff(s, false, 1, w_new, E))) return rc;  // H[t + ds]
      if ((rc = exponential(0.5 * ds))) return rc;
      s->dens_valid = true;  // the last sweep wrote the density of the new state
    }
    s->steps++;
  }
  s->clock_t = t0 + n_steps * dt;
  s->clock_dt = dt;
  s->clock_substeps = substeps;
  return TDKS_OK;
}

// (cr + i ci) H[n, t] in -> out, with n the density now in dens_part: LDA, projector step
// and a middle-term sweep (the shape of Taylor term 2).
static int apply_scaled(tdks_system *s, const void *in, void *out, double cr, double ci, double t) {
  double E[3], A[3];
  field_at(s, t, E, A);
  int rc;
  if ((rc = run_lda(s, E, A))) return rc;
  if ((rc = run_gather(s, in, A))) return rc;
  SweepParams p{};
  sweep_common(s, p, A, 1);
  set_coef(p, cr, ci);
  p.in = in;
  p.out = out;
  SweepMaps tm;
  const bool have_tm = tma_path(s) && encode_sweep_maps(s, in, MODE_MID, &tm, s->path == 2, 1);
  return run_sweep(s, MODE_MID, p, have_tm ? &tm : nullptr, 1);
}

// Classical fourth-order Runge-Kutta on d psi/dt = -i H[n(psi), t] psi (complex128 systems):
// every stage rebuilds the density of its own stage vector, so H follows the state within the
// sub-step.  term[0] accumulates the weighted slopes, term[1] holds the stage vector, term[2]
// the slope k = -i H psi_stage.
static int propagate_rk4(tdks_system *s, double t0, double dt, int n_steps, int substeps) {
  const double ds = dt / substeps;
  if (std::fabs(ds) * kinetic_max(s) > 2.0 * std::sqrt(2.0))
    return fail(TDKS_EUNSTABLE, "RK4 sub-step beyond its stability limit on the imaginary axis (dt_sub * K_max > 2 sqrt 2)");
  const long n = (long)(s->state_bytes / 16);
  void *acc = s->term[0], *stage = s->term[1], *k = s->term[2];
  int rc;
  auto stage_density = [&](const void *v) -> int {
    cudaError_t e = launch_density(s->prec, s->N, s->n_kb, s->n_batches, v, nullptr, s->d_wocc, s->dens_part,
                                   s->stream);
    s->launches++;
    s->dens_valid = false;  // dens_part now holds a stage vector's density
    return e == cudaSuccess ? TDKS_OK : fail(TDKS_EDEVICE, std::string("density: ") + cudaGetErrorString(e));
  };
  auto check = [&](cudaError_t e) {
    s->launches++;
    return e == cudaSuccess ? TDKS_OK : fail(TDKS_EDEVICE, std::string("rk4 update: ") + cudaGetErrorString(e));
  };
  for (int st = 0; st < n_steps; st++) {
    const double t = t0 + st * dt;
    for (int j = 0; j < substeps; j++) {
      const double tj = t + j * ds;
      if ((rc = ensure_density(s))) return rc;
      if (j == 0) {
        // record of the state at t: the Hamiltonian of t + ds/2 with v_x of this state
        double E[3], A[3];
        field_at(s, tj + 0.5 * ds, E, A);
        if ((rc = run_lda(s, E, A))) return rc;
        if ((rc = first_sweep(s, 1.0, 0.0, A, true))) return rc;
        double *slot = s->ring + (s->steps % tdks_system::RING) * TDKS_RECORD;
        if ((rc = run_finalize(s, slot, t, E, A))) return rc;
      }
      if ((rc = apply_scaled(s, s->psi, k, 0.0, -1.0, tj))) return rc;  // k1
      if ((rc = check(launch_rk4_stage(n, s->psi, k, 0.5 * ds, stage, acc, ds / 6.0, 1, s->stream)))) return rc;
      if ((rc = stage_density(stage)) || (rc = apply_scaled(s, stage, k, 0.0, -1.0, tj + 0.5 * ds))) return rc;  // k2
      if ((rc = check(launch_rk4_stage(n, s->psi, k, 0.5 * ds, stage, acc, ds / 3.0, 0, s->stream)))) return rc;
      if ((rc = stage_density(stage)) || (rc = apply_scaled(s, stage, k, 0.0, -1.0, tj + 0.5 * ds))) return rc;  // k3
      if ((rc = check(launch_rk4_stage(n, s->psi, k, ds, stage, acc, ds / 3.0, 0, s->stream)))) return rc;
      if ((rc = stage_density(stage)) || (rc = apply_scaled(s, stage, k, 0.0, -1.0, tj + ds))) return rc;  // k4
      if ((rc = check(launch_rk4_finish(n, s->psi, acc, k, ds / 6.0, s->stream)))) return rc;
      s->dens_valid = false;
    }
    s->steps++;
  }
  s->clock_t = t0 + n_steps * dt;
  s->clock_dt = dt;
  s->clock_substeps = substeps;
  return TDKS_OK;
}

int tdks_set_propagator(tdks_sys s, int propagator) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (propagator < TDKS_PROP_TAYLOR4 || propagator > TDKS_PROP_ETRS)
    return fail(TDKS_EINVAL, "propagator must be TDKS_PROP_TAYLOR4, _CFM4, _EMR, _AETRS, _RK4 or _ETRS");
  if (propagator == TDKS_PROP_RK4 && s->prec != TDKS_C128)
    return fail(TDKS_EINVAL, "RK4 runs on complex128 systems");
  CU(cudaStreamSynchronize(s->stream));
  if (propagator != TDKS_PROP_TAYLOR4 && propagator != TDKS_PROP_RK4 && !s->vx_hist[0])
    for (int j = 0; j < 4; j++) CU(cudaMalloc((void **)&s->vx_hist[j], (size_t)s->N * sizeof(double)));
  if (propagator == TDKS_PROP_ETRS && !s->etrs_save) {
    CU(cudaMalloc(&s->etrs_save, s->state_bytes));
    if (s->psi_lo) CU(cudaMalloc(&s->etrs_save_lo, s->state_bytes));
  }
  s->prop = propagator;
  s->n_hist = 0;
  return TDKS_OK;
}

int tdks_set_exchange(tdks_sys s, tdks_exchange_fn fn, void *ctx) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (fn && !s->n_total) {
    CU(cudaMalloc((void **)&s->n_total, (size_t)s->N * sizeof(double)));
    CU(cudaMalloc((void **)&s->fin_sum, 10 * sizeof(double)));
  }
  s->xfn = fn;
  s->xctx = fn ? ctx : nullptr;
  return TDKS_OK;
}

static int propagate_steps(tdks_system *s, double t0, double dt, int n_steps, int substeps);

int tdks_propagate_n(tdks_sys s, double t0, double dt, int n_steps, int substeps) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (n_steps < 0 || substeps < 0) return fail(TDKS_EINVAL, "negative count");
  if (!s->have_orbitals) return fail(TDKS_ESTATE, "orbitals not set");
  if (substeps == 0) tdks_auto_substeps(s, dt, &substeps);
  if (s->ts_np == 0) return propagate_steps(s, t0, dt, n_steps, substeps);
  // t-SURFF: the flux of the state at the start of every step, by the trapezoid rule in time
  // (dt/2 at this call's first and last states), the Volkov parameters advanced per step
  if (!s->ts_started) {
    s->ts_started = true;
    s->ts_t0 = t0;
  } else if (std::fabs(t0 - (s->ts_t0 + s->ts_trel)) > 1e-9 * std::max(1.0, std::fabs(t0))) {
    return fail(TDKS_EINVAL, "t-SURFF accumulation: t0 must continue from the last propagation's end");
  }
  int rc = TDKS_OK;
  for (int st = 0; st <= n_steps; st++) {
    const double t = t0 + st * dt;
    if ((rc = tsurff_accumulate(s, (st == 0 || st == n_steps) ? 0.5 * dt : dt))) return rc;
    if (st == n_steps) break;
    if ((rc = propagate_steps(s, t, dt, 1, substeps))) return rc;
    tsurff_advance(s, t, dt);
  }
  s->clock_t = t0 + n_steps * dt;
  return TDKS_OK;
}

static int propagate_steps(tdks_system *s, double t0, double dt, int n_steps, int substeps) {
  if (s->prop == TDKS_PROP_RK4) return propagate_rk4(s, t0, dt, n_steps, substeps);
  if (s->prop == TDKS_PROP_ETRS) return propagate_etrs(s, t0, dt, n_steps, substeps);
  if (s->prop != TDKS_PROP_TAYLOR4) return propagate_exp(s, t0, dt, n_steps, substeps);
  const double dts = dt / substeps;
  if (std::fabs(dts) * kinetic_max(s) > 2.0 * std::sqrt(2.0))
    return fail(TDKS_EUNSTABLE, "sub-step beyond the Taylor-4 stability limit (dt_sub * K_max > 2 sqrt 2)");
  int rc = ensure_density(s);
  if (rc) return rc;
  for (int st = 0; st < n_steps; st++) {
    const double t = t0 + st * dt;
    for (int j = 0; j < substeps; j++) {
      const double tj = t + j * dts, tm = tj + 0.5 * dts;
      double E[3], A[3];
      field_at(s, tm, E, A);
      const bool rec = (j == 0);
      if ((rc = run_lda(s, E, A, rec))) return rc;  // (the record's sums on record sub-steps only)
      if ((rc = first_sweep(s, 0.0, -dts, A, rec))) return rc;
      if (rec) {
        double *slot = s->ring + (s->steps % tdks_system::RING) * TDKS_RECORD;
        if ((rc = run_finalize(s, slot, t, E, A))) return rc;
      }
      if ((rc = taylor_tail(s, dts, A))) return rc;
      s->dens_valid = true;  // MODE_LAST wrote the density of the new state
    }
    s->steps++;
  }
  s->clock_t = t0 + n_steps * dt;
  s->clock_dt = dt;
  s->clock_substeps = substeps;
  return TDKS_OK;
}

int tdks_reductions(tdks_sys s, long long step_from, int n, double *out) {
  if (!s || (!out && n > 0)) return fail(TDKS_EINVAL, "NULL argument");
  if (n < 0 || step_from < 0 || step_from + n > s->steps || step_from < s->steps - tdks_system::RING)
    return fail(TDKS_EINVAL, "record range outside the stored ring");
  CU(cudaStreamSynchronize(s->stream));
  if (int rc = check_err(s)) return rc;
  for (int i = 0; i < n;) {
    const long long slot = (step_from + i) % tdks_system::RING;
    const int cnt = (int)std::min<long long>(n - i, tdks_system::RING - slot);
    CU(cudaMemcpy(out + (size_t)i * TDKS_RECORD, s->ring + slot * TDKS_RECORD, (size_t)cnt * TDKS_RECORD * sizeof(double),
                  cudaMemcpyDeviceToHost));
    i += cnt;
  }
  return TDKS_OK;
}

int tdks_step_count(tdks_sys s, long long *count) {
  if (!s || !count) return fail(TDKS_EINVAL, "NULL argument");
  *count = s->steps;
  return TDKS_OK;
}

int tdks_observe(tdks_sys s, double t_state, double t_field, double *out) {
  if (!s || !out) return fail(TDKS_EINVAL, "NULL argument");
  int rc = ensure_density(s);
  if (rc) return rc;
  double E[3], A[3];
  field_at(s, t_field, E, A);
  if ((rc = run_lda(s, E, A))) return rc;
  if ((rc = first_sweep(s, 1.0, 0.0, A, true))) return rc;
  if ((rc = run_finalize(s, s->obs_rec, t_state, E, A))) return rc;
  CU(cudaMemcpyAsync(out, s->obs_rec, TDKS_RECORD * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CU(cudaStreamSynchronize(s->stream));
  return check_err(s);
}

int tdks_set_profiling(tdks_sys s, int on) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  s->profile = on != 0;
  return TDKS_OK;
}

int tdks_kernel_time(tdks_sys s, int kind, double *ms, long long *launches) {
  if (!s || kind < 0 || kind > 6) return fail(TDKS_EINVAL, "bad argument");
  CU(cudaStreamSynchronize(s->stream));
  for (auto &u : s->ev_used) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, u.second.first, u.second.second) == cudaSuccess) {
      s->prof_ms[u.first] += t;
      s->prof_n[u.first]++;
      if (u.first >= 3) {  // a Taylor term's sweep is also a stencil sweep
        s->prof_ms[0] += t;
        s->prof_n[0]++;
      }
    }
    s->ev_free.push_back(u.second.first);
    s->ev_free.push_back(u.second.second);
  }
  s->ev_used.clear();
  if (ms) *ms = s->prof_ms[kind];
  if (launches) *launches = s->prof_n[kind];
  s->prof_ms[kind] = 0.0;
  s->prof_n[kind] = 0;
  return TDKS_OK;
}

int tdks_launch_count(tdks_sys s, long long *count) {
  if (!s || !count) return fail(TDKS_EINVAL, "NULL argument");
  *count = s->launches;
  return TDKS_OK;
}

}  // extern "C"
