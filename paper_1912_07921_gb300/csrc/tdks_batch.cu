// Batched propagation: many independent finite-box systems advanced together with one
// persistent TMA sweep launch per Taylor term (plus one batched projector gather, one
// batched LDA/V_eff and the record/clock kernels), the whole sub-step captured once as a
// CUDA graph and replayed.  Every system keeps its own device clock (time, step length,
// sub-step counter), so the graph needs no host-side parameter change between replays.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "tdks_system.h"

using namespace tdks;
using namespace tdks_host;

struct tdks_batch {
  std::vector<tdks_system *> sys;
  cudaStream_t stream = nullptr;   // the caller's stream
  cudaStream_t work = nullptr;     // private stream the batch captures and runs on
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int M = 0, prec = 0, substeps = 0;
  int shape[4] = {0, 0, 0, 0};     // sweep tile shape of each Taylor term (tdks_batch_autotune)
  // device arrays
  SweepParams *d_sweep[4] = {nullptr, nullptr, nullptr, nullptr};   // per Taylor term
  GatherParams *d_gather[4] = {nullptr, nullptr, nullptr, nullptr};
  SweepMaps *d_maps = nullptr;                                      // 4 per system
  long *d_item_begin[4] = {nullptr, nullptr, nullptr, nullptr};     // per Taylor term
  int *d_item_sys[4] = {nullptr, nullptr, nullptr, nullptr};        // the system of every item
  long *d_gather_begin = nullptr, *d_unit_begin = nullptr, *d_lda_begin = nullptr;
  long *d_nl_begin = nullptr;
  int *d_gather_sys = nullptr, *d_unit_sys = nullptr, *d_nl_sys = nullptr;
  unsigned int *d_work = nullptr;  // work-item counter of the batched sweep (zero between launches)
  BatchAux *d_aux = nullptr;
  std::vector<BatchAux> aux_h;     // host copy (the record count follows the first term's shape)
  BatchClock *d_clock = nullptr;
  long total_items[4] = {0, 0, 0, 0};
  long total_gather = 0, total_units = 0, total_lda = 0, total_nl = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;
};

namespace {

void batch_free(tdks_batch *b) {
  for (int k = 0; k < 4; k++) {
    cudaFree(b->d_sweep[k]); cudaFree(b->d_gather[k]); cudaFree(b->d_item_begin[k]); cudaFree(b->d_item_sys[k]);
  }
  cudaFree(b->d_maps); cudaFree(b->d_gather_begin); cudaFree(b->d_lda_begin);
  cudaFree(b->d_nl_begin); cudaFree(b->d_work);
  cudaFree(b->d_unit_begin);
  cudaFree(b->d_gather_sys); cudaFree(b->d_unit_sys); cudaFree(b->d_nl_sys);
  cudaFree(b->d_aux); cudaFree(b->d_clock);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->work) cudaStreamDestroy(b->work);
}

// CTAs of one system in the batched LDA launch: a sixteenth of the single-system count (whose
// partial buffer it fills), i.e. ~16 points per thread, so that the launch over all systems pays
// each CTA's setup (system lookup, field, weight staging) a few times per SM rather than once per
// CTA-sized run of points.
static int lda_batch_blocks(long N) { return std::max(1, (lda_blocks(N) + 15) / 16); }

// Kernels one sub-step launches: the LDA/V_eff kernel, per Taylor term the projector step
// (gather stages 1 and 2 and the non-local term, where any system has atoms) and the sweep,
// and the record and clock kernels.
long long substep_launches(const tdks_batch *b) {
  const int proj = b->total_gather > 0 ? 2 + (b->total_nl > 0 ? 1 : 0) : 0;
  return 1 + 4 * (proj + 1) + 2;
}

// Enqueue one sub-step of every system of the batch.
int enqueue_substep(tdks_batch *b) {
  const int n = (int)b->sys.size();
  cudaError_t e = launch_lda_batch(b->prec, b->d_aux, b->d_clock, b->d_lda_begin, n, b->total_lda, b->work);
  if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("batched lda: ") + cudaGetErrorString(e));
  for (int k = 0; k < 4; k++) {
    e = launch_gather_batch(b->prec, b->d_gather[k], b->d_gather_begin, b->d_unit_begin, b->d_nl_begin,
                            b->d_gather_sys, b->d_unit_sys, b->d_nl_sys, b->total_gather, b->total_units,
                            b->total_nl, b->work);
    if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("batched gather: ") + cudaGetErrorString(e));
    BatchSweepArgs a{b->d_sweep[k], b->d_maps, k, b->d_item_begin[k],
                      n, b->total_items[k], b->d_work, b->d_item_sys[k]};
    const int mode = k == 0 ? MODE_FIRST : (k == 3 ? MODE_LAST : MODE_MID);
    e = launch_sweep_tma_batch(b->M, b->prec, mode, a, b->work, b->shape[k]);
    if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("batched sweep: ") + cudaGetErrorString(e));
    if (k == 0) {
      e = launch_batch_tail(b->d_aux, b->d_clock, n, 0, b->work);
      if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("batched records: ") + cudaGetErrorString(e));
    }
  }
  e = launch_batch_tail(b->d_aux, b->d_clock, n, 1, b->work);
  if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("batched clocks: ") + cudaGetErrorString(e));
  b->launches += substep_launches(b);
  return TDKS_OK;
}

template <class T>
int upload(T **dst, const std::vector<T> &v) {
  CU(cudaMalloc((void **)dst, std::max<size_t>(1, v.size()) * sizeof(T)));
  if (!v.empty()) CU(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return TDKS_OK;
}

// Sweep tables of the batch for its current shapes: per Taylor term the systems' sweep
// parameters, tensor maps (one per system and term) and work-item prefix sums; whole z
// columns per item (many systems already balance the grid).  tune: the last term's
// tables point the state operands at the Taylor-term buffers (state hi <- t1, lo <- t2), so
// the autotuner can time it without touching any state.  The captured graph, which holds
// the old tables, is dropped.
int build_sweep_tables(tdks_batch *b, bool tune) {
  const int n = (int)b->sys.size();
  std::vector<SweepParams> sp[4];
  std::vector<SweepMaps> maps(4 * (size_t)n);
  std::vector<long> ib[4];
  for (int k = 0; k < 4; k++) ib[k].assign(n + 1, 0);
  const int modes[4] = {MODE_FIRST, MODE_MID, MODE_MID, MODE_LAST};
  const double A0[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < n; i++) {
    tdks_system *s = b->sys[i];
    const int save_tx = s->tx, save_ty = s->ty, save_zc = s->zc;
    const void *ins[4] = {s->psi, s->term[0], s->term[1], s->term[2]};
    const double dts = s->clock_dt / s->clock_substeps;
    bool ok = true;
    for (int k = 0; k < 4 && ok; k++) {
      int tx = 16, ty = 8;
      ws_shape_info(b->shape[k], &tx, &ty, nullptr, nullptr);
      s->tx = tx; s->ty = ty; s->zc = s->nz;
      ok = encode_sweep_maps(s, ins[k], modes[k], &maps[4 * i + k], false);
      SweepParams p{};
      sweep_common(s, p, A0);
      set_coef(p, 0.0, -dts / (k + 1));
      p.in = ins[k];
      p.do_obs = k == 0;
      p.err = s->d_err;
      if (k < 3) {
        p.out = s->term[k];
      } else if (!tune) {
        p.psi = s->psi; p.psi_lo = s->psi_lo; p.t1 = s->term[0]; p.t2 = s->term[1];
      } else {
        p.psi = s->term[0]; p.psi_lo = s->term[1]; p.t1 = s->term[0]; p.t2 = s->term[1];
        const void *ops[4] = {s->term[0], s->term[1], s->term[0], s->term[1]};
        for (int j = 0; j < 4 && ok; j++) ok = encode_op_map(s, ops[j], &maps[4 * i + k].op[j], tx, ty);
      }
      sp[k].push_back(p);
      ib[k][i + 1] = ib[k][i] + p.n_items;
    }
    s->tx = save_tx; s->ty = save_ty; s->zc = save_zc;
    if (!ok) return fail(TDKS_EDEVICE, "tensor map encoding failed");
    // the warp-specialised sweep writes one partial record per consumer warp and item
    int warps = 8;
    ws_shape_info(b->shape[0], nullptr, nullptr, nullptr, &warps);
    b->aux_h[i].n_items = sp[0].back().n_items * warps;
  }
  for (int k = 0; k < 4; k++) {
    cudaFree(b->d_sweep[k]); b->d_sweep[k] = nullptr;
    cudaFree(b->d_item_begin[k]); b->d_item_begin[k] = nullptr;
    cudaFree(b->d_item_sys[k]); b->d_item_sys[k] = nullptr;
  }
  cudaFree(b->d_maps); b->d_maps = nullptr;
  int rc = TDKS_OK;
  for (int k = 0; k < 4 && !rc; k++) {
    rc = upload(&b->d_sweep[k], sp[k]);
    if (!rc) rc = upload(&b->d_item_begin[k], ib[k]);
    b->total_items[k] = ib[k][n];
    std::vector<int> owner((size_t)ib[k][n]);
    for (int i = 0; i < n; i++)
      for (long it = ib[k][i]; it < ib[k][i + 1]; it++) owner[(size_t)it] = i;
    if (!rc) rc = upload(&b->d_item_sys[k], owner);
  }
  if (!rc) rc = upload(&b->d_maps, maps);
  if (!rc && b->d_aux) CU(cudaMemcpy(b->d_aux, b->aux_h.data(), n * sizeof(BatchAux), cudaMemcpyHostToDevice));
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  return rc;
}

}  // namespace

extern "C" {

int tdks_set_clock(tdks_sys s, double t, double dt, int substeps) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (substeps < 1) return fail(TDKS_EINVAL, "substeps must be >= 1");
  if (std::fabs(dt / substeps) * kinetic_max(s) > 2.0 * std::sqrt(2.0))
    return fail(TDKS_EUNSTABLE, "sub-step beyond the Taylor-4 stability limit (dt_sub * K_max > 2 sqrt 2)");
  s->clock_t = t;
  s->clock_dt = dt;
  s->clock_substeps = substeps;
  return TDKS_OK;
}

int tdks_get_clock(tdks_sys s, double *t, long long *steps) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (t) *t = s->clock_t;
  if (steps) *steps = s->steps;
  return TDKS_OK;
}

int tdks_batch_create(const tdks_sys *systems, int n, void *stream, tdks_batch_t *out) {
  if (!systems || n < 1 || !out) return fail(TDKS_EINVAL, "bad arguments");
  *out = nullptr;
  tdks_batch *b = new (std::nothrow) tdks_batch();
  if (!b) return fail(TDKS_ENOMEM, "host allocation");
  b->stream = (cudaStream_t)stream;
  b->sys.assign(systems, systems + n);
  tdks_system *s0 = b->sys[0];
  b->M = s0->M;
  b->prec = s0->prec;
  b->substeps = s0->clock_substeps;
  auto bad = [&](const char *m) { delete b; return fail(TDKS_EINVAL, m); };
  for (tdks_system *s : b->sys) {
    if (!s) return bad("NULL system in batch");
    if (s->bc != TDKS_BC_ZERO) return bad("batched propagation takes finite boxes only");
    if (s->M != b->M || s->prec != b->prec) return bad("a batch shares the FD order and the precision");
    if (s->clock_substeps != b->substeps) return bad("a batch shares the sub-step count (tdks_set_clock)");
    if (s->gauge == TDKS_GAUGE_VELOCITY) return bad("velocity gauge is not batched");
    if (!s->have_orbitals) return bad("orbitals not set");
    if (!tma_supported(s->M, 16, 8)) return bad("no TMA sweep for this FD order");
    if (s->prop != TDKS_PROP_TAYLOR4) return bad("batched propagation uses the Taylor-4 propagator");
    if (s->xfn) return bad("a state-parallel system (exchange hook set) cannot join a batch");
    if (s->xc == TDKS_XC_LDA_X_HARTREE) return bad("a system with the Hartree term cannot join a batch");
    if (s->upload_buffers != 1) return bad("a system with two upload buffers cannot join a batch");
  }
  std::vector<GatherParams> gp[4];
  std::vector<long> gather_begin(n + 1, 0), unit_begin(n + 1, 0), lda_begin(n + 1, 0);
  std::vector<long> nl_begin(n + 1, 0);
  std::vector<BatchAux> &aux = b->aux_h;
  aux.assign(n, BatchAux{});
  std::vector<BatchClock> clk(n);
  // the projector gather's chunks per (atom, k-batch) unit are sized for the whole batch's
  // units (a system alone splits each unit into up to 16 chunks to fill the GPU; a batch has
  // the units to fill it without the per-chunk reductions); never more than the system's
  // partial-sum buffer holds
  long batch_units = 0;
  for (tdks_system *s : b->sys) batch_units += (long)s->n_atoms * s->n_kb;
  const int bchunks = gather_chunks(std::max(batch_units, 1L));
  for (int i = 0; i < n; i++) {
    tdks_system *s = b->sys[i];
    const void *ins[4] = {s->psi, s->term[0], s->term[1], s->term[2]};
    const int nch = std::min(s->gchunks, bchunks);
    for (int k = 0; k < 4; k++) {
      GatherParams g{};
      g.n_kb = s->n_kb; g.n_batches = s->n_batches; g.n_atoms = s->n_atoms; g.N = s->N;
      g.in = ins[k]; g.atom_begin = s->d_atom_begin; g.ent = s->d_ent; g.D = s->d_D;
      g.ent_beta = s->d_ent_beta; g.ent_ca = s->d_ent_ca;
      g.h3 = s->h * s->h * s->h; g.kvec = s->d_kvec; g.q = s->d_q;
      g.n_chunks = nch; g.qpart = s->d_qpart;
      g.sp = s->d_sp; g.n_sp = s->n_sp; g.rowent = s->d_rowent; g.n_ent = s->n_ent; g.nl = s->d_nl;
      gp[k].push_back(g);
    }
    gather_begin[i + 1] = gather_begin[i] + (long)s->n_atoms * s->n_kb * (s->n_atoms > 0 ? nch : 0);
    unit_begin[i + 1] = unit_begin[i] + (long)s->n_atoms * s->n_kb;
    nl_begin[i + 1] = nl_begin[i] + (s->n_atoms > 0 ? nl_batch_blocks(s->n_sp, s->n_kb) : 0);
    const int nl = lda_batch_blocks(s->N);
    lda_begin[i + 1] = lda_begin[i] + nl;
    BatchAux &a = aux[i];
    a.N = s->N; a.nx = s->nx; a.ny = s->ny; a.nz = s->nz; a.n_kb = s->n_kb; a.xc = s->xc;
    a.n_batches = s->n_batches; a.wocc = s->d_wocc;
    a.h = s->h; a.occ = s->occ; a.gauge = s->gauge; a.envelope = s->envelope;
    for (int d = 0; d < 3; d++) a.pol[d] = s->pol[d];
    a.amp = s->amp; a.omega = s->omega; a.t_total = s->t_total;
    a.dens_part = s->dens_part; a.vloc = s->vloc; a.aux = s->aux; a.lda_part = s->lda_part; a.n_lda = nl;
    a.obs_part = s->obs_part; a.ring = s->ring;  // a.n_items: set with the sweep tables
    a.ring_len = tdks_system::RING;
  }
  int rc = build_sweep_tables(b, false);
  b->total_gather = gather_begin[n];
  b->total_units = unit_begin[n];
  b->total_lda = lda_begin[n];
  b->total_nl = nl_begin[n];
  for (int k = 0; k < 4 && !rc; k++) rc = upload(&b->d_gather[k], gp[k]);
  if (!rc) rc = upload(&b->d_gather_begin, gather_begin);
  if (!rc) rc = upload(&b->d_unit_begin, unit_begin);
  if (!rc) rc = upload(&b->d_lda_begin, lda_begin);
  if (!rc) rc = upload(&b->d_nl_begin, nl_begin);
  // the system of every CTA (or unit) of the batched projector launches
  auto owners = [&](const std::vector<long> &beg) {
    std::vector<int> o((size_t)beg[n]);
    for (int i = 0; i < n; i++)
      for (long c = beg[i]; c < beg[i + 1]; c++) o[(size_t)c] = i;
    return o;
  };
  if (!rc) rc = upload(&b->d_gather_sys, owners(gather_begin));
  if (!rc) rc = upload(&b->d_unit_sys, owners(unit_begin));
  if (!rc) rc = upload(&b->d_nl_sys, owners(nl_begin));
  if (!rc) rc = upload(&b->d_work, std::vector<unsigned int>(1, 0u));
  if (!rc) rc = upload(&b->d_aux, aux);
  if (!rc) rc = upload(&b->d_clock, clk);
  if (!rc && (cudaStreamCreateWithFlags(&b->work, cudaStreamNonBlocking) != cudaSuccess ||
              cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
              cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess))
    rc = fail(TDKS_EDEVICE, "batch stream/event creation");
  if (rc) {
    batch_free(b);
    delete b;
    return rc;
  }
  *out = b;
  return TDKS_OK;
}

int tdks_batch_destroy(tdks_batch_t b) {
  if (!b) return TDKS_OK;
  cudaStreamSynchronize(b->stream);
  if (b->work) cudaStreamSynchronize(b->work);
  batch_free(b);
  delete b;
  return TDKS_OK;
}

int tdks_batch_propagate(tdks_batch_t b, int n_steps, int use_graph) {
  if (!b || n_steps < 0) return fail(TDKS_EINVAL, "bad arguments");
  const int n = (int)b->sys.size();
  // densities of the current states, and the device clocks from each system's clock
  std::vector<BatchClock> clk(n);
  for (int i = 0; i < n; i++) {
    tdks_system *s = b->sys[i];
    if (s->stream != b->stream) CU(cudaStreamSynchronize(s->stream));
    if (int rc = ensure_density(s)) return rc;
    if (s->stream != b->stream) CU(cudaStreamSynchronize(s->stream));
    clk[i] = BatchClock{s->clock_t, s->clock_dt, s->steps, s->clock_substeps, 0};
  }
  // the batch's work follows everything enqueued on the caller's stream
  CU(cudaEventRecord(b->ev_in, b->stream));
  CU(cudaStreamWaitEvent(b->work, b->ev_in, 0));
  CU(cudaMemcpyAsync(b->d_clock, clk.data(), n * sizeof(BatchClock), cudaMemcpyHostToDevice, b->work));
  if (use_graph && !b->exec) {
    CU(cudaStreamBeginCapture(b->work, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_substep(b);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->work, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("graph capture: ") + cudaGetErrorString(e));
    b->graph = g;
    CU(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->launches -= substep_launches(b);
  }
  const long long subs = (long long)n_steps * b->substeps;
  for (long long i = 0; i < subs; i++) {
    if (use_graph) {
      CU(cudaGraphLaunch(b->exec, b->work));
      b->launches += substep_launches(b);
    } else if (int rc = enqueue_substep(b)) {
      return rc;
    }
  }
  // and everything enqueued on the caller's stream afterwards follows the batch
  CU(cudaEventRecord(b->ev_out, b->work));
  CU(cudaStreamWaitEvent(b->stream, b->ev_out, 0));
  for (tdks_system *s : b->sys) {
    s->steps += n_steps;
    s->clock_t += n_steps * s->clock_dt;
    s->dens_valid = true;
  }
  return TDKS_OK;
}

int tdks_batch_set_shape(tdks_batch_t b, int term, int shape) {
  if (!b) return fail(TDKS_EINVAL, "NULL batch");
  if (term < -1 || term > 3) return fail(TDKS_EINVAL, "term must be 0..3 or -1");
  if (!ws_shape_info(shape, nullptr, nullptr, nullptr, nullptr)) return fail(TDKS_EINVAL, "no such sweep shape");
  CU(cudaStreamSynchronize(b->stream));
  CU(cudaStreamSynchronize(b->work));
  for (int k = 0; k < 4; k++)
    if (term < 0 || term == k) b->shape[k] = shape;
  return build_sweep_tables(b, false);
}

int tdks_batch_get_shape(tdks_batch_t b, int term, int *shape) {
  if (!b || !shape) return fail(TDKS_EINVAL, "NULL argument");
  if (term < 0 || term > 3) return fail(TDKS_EINVAL, "term must be 0..3");
  *shape = b->shape[term];
  return TDKS_OK;
}

int tdks_batch_autotune(tdks_batch_t b, int reps, double *ms) {
  if (!b) return fail(TDKS_EINVAL, "NULL batch");
  if (reps < 1) return fail(TDKS_EINVAL, "reps < 1");
  if (ms)
    for (int i = 0; i < WS_SHAPES * 4; i++) ms[i] = -1.0;
  CU(cudaStreamSynchronize(b->stream));
  CU(cudaStreamSynchronize(b->work));
  const int n = (int)b->sys.size();
  const int saved[4] = {b->shape[0], b->shape[1], b->shape[2], b->shape[3]};
  int pick[4] = {saved[0], saved[1], saved[2], saved[3]};
  double best[4] = {-1.0, -1.0, -1.0, -1.0};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(TDKS_EDEVICE, "cudaEventCreate");
  }
  int rc = TDKS_OK;
  const int modes[4] = {MODE_FIRST, MODE_MID, MODE_MID, MODE_LAST};
  for (int sh = 0; sh < WS_SHAPES && !rc; sh++) {
    for (int k = 0; k < 4; k++) b->shape[k] = sh;
    if ((rc = build_sweep_tables(b, true))) break;
    for (int k = 0; k < 4 && !rc; k++) {
      BatchSweepArgs a{b->d_sweep[k], b->d_maps, k, b->d_item_begin[k],
                      n, b->total_items[k], b->d_work, b->d_item_sys[k]};
      cudaError_t e = launch_sweep_tma_batch(b->M, b->prec, modes[k], a, b->work, sh);  // warm-up
      cudaEventRecord(e0, b->work);
      for (int r = 0; r < reps && e == cudaSuccess; r++)
        e = launch_sweep_tma_batch(b->M, b->prec, modes[k], a, b->work, sh);
      cudaEventRecord(e1, b->work);
      if (e != cudaSuccess) { rc = fail(TDKS_EDEVICE, std::string("batched sweep: ") + cudaGetErrorString(e)); break; }
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(TDKS_EDEVICE, "batch autotune timing"); break; }
      for (tdks_system *s : b->sys)
        if ((rc = check_err(s))) break;
      if (rc) break;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      const double per = (double)t / reps;
      if (ms) ms[sh * 4 + k] = per;
      if (best[k] < 0.0 || per < best[k]) { best[k] = per; pick[k] = sh; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int k = 0; k < 4; k++) b->shape[k] = rc ? saved[k] : pick[k];
  const int rc2 = build_sweep_tables(b, false);
  for (tdks_system *s : b->sys) s->dens_valid = false;  // the timed last terms wrote density partials
  return rc ? rc : rc2;
}

int tdks_batch_launch_count(tdks_batch_t b, long long *count) {
  if (!b || !count) return fail(TDKS_EINVAL, "NULL argument");
  *count = b->launches;
  return TDKS_OK;
}

}  // extern "C"
