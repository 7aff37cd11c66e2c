/*
 * tdks.h — C interface of the GB300 real-time TDDFT propagation library.
 *
 * The library integrates the time-dependent Kohn-Sham equations in the form the paper
 * states them (arXiv:1912.07921, Sec. "New propagators for real-time TDDFT", first three
 * equations):  d phi_i / dt = -i H[n(t), t] phi_i,  phi(t0) = phi^0,  i = 1..N_orb,
 * in the adiabatic approximation (the exchange potential depends on n(t) only).
 *
 * H = -1/2 Lap_h + V_loc(r) + v_x[n](r) + E(t).r  (length gauge, finite box), or
 * H = 1/2 (-i grad_h + A(t))^2 + V_loc + v_x[n]    (velocity gauge, periodic cell,
 *     E = -dA/dt, Sec. "Conductivities"),
 * plus Kleinman-Bylander projectors V_NL = sum_aj |beta_aj> D_aj <beta_aj|.
 * Lap_h and grad_h are central finite differences of order 4 or 8 on a uniform grid
 * (Sec. "Maxwell ... coupling" and Sec. "Periodic systems"); v_x is LDA exchange
 * (Sec. "Local domains", E_xc = int n e_xc(n)); orbitals are doubly occupied by default
 * (closed shells, Sec. "t-SURFF").  The exponential exp(-i dt H) is a 4th-order Taylor
 * series with H frozen over each sub-step: t_0 = psi, t_k = (-i dt/k) H t_(k-1),
 * psi(t+dt) = t_0 + ... + t_4; the density is rebuilt and the field is taken at the
 * sub-step midpoint.
 *
 * Conventions
 *   - Every function returns a tdks_status and never aborts; tdks_last_error() returns a
 *     thread-local message for the last failure on the calling thread.
 *   - The system object owns all its device memory.  Host arrays passed in are copied;
 *     host arrays passed out are filled before the call returns.
 *   - Work is enqueued on the stream given to tdks_create_grid (a cudaStream_t, or NULL
 *     for the legacy default stream) and may still run when a call returns, except for
 *     calls documented as synchronising.
 *   - Host orbital layout: complex128 as interleaved (re, im) doubles, index
 *     [k][z][y][x][orb], the state index innermost (Sec. "Memory layout").
 *   - Device (packed) layout used by tdks_apply_H: [k][batch][z][y][x][j], orbital
 *     o = batch * BS + j, BS = 4 (complex128 systems) or 8 (complex64 systems),
 *     zero-padded to a whole number of batches; elements are complex128 or complex64
 *     as the system's precision.  tdks_layout() reports BS, the batch count and sizes.
 *   - Grid coordinates: finite box x_i = (i - (nx-1)/2) h; periodic cell x_i = i h,
 *     cell side L = nx h; the same for y and z.
 *   - Errors: TDKS_EINVAL for bad arguments, TDKS_ENOMEM for failed device or host
 *     allocation, TDKS_EUNSTABLE when a requested sub-step is beyond the stability
 *     limit of the 4th-order Taylor series, TDKS_EDEVICE for a CUDA error (the message
 *     names it), TDKS_ESTATE when a call needs data not set yet (e.g. orbitals).
 */
#ifndef TDKS_H
#define TDKS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdks_system *tdks_sys;

typedef enum {
  TDKS_OK = 0,
  TDKS_EINVAL = 1,
  TDKS_ENOMEM = 2,
  TDKS_EUNSTABLE = 3,
  TDKS_ETIMEOUT = 4,
  TDKS_EDEVICE = 5,
  TDKS_ESTATE = 6
} tdks_status;

enum { TDKS_BC_ZERO = 0, TDKS_BC_BLOCH = 1 };
enum { TDKS_C128 = 0, TDKS_C64 = 1 };
enum { TDKS_GAUGE_NONE = 0, TDKS_GAUGE_LENGTH = 1, TDKS_GAUGE_VELOCITY = 2 };
enum { TDKS_ENV_NONE = 0, TDKS_ENV_SIN2 = 1 };
enum { TDKS_XC_NONE = 0, TDKS_XC_LDA_X = 1, TDKS_XC_LDA_X_HARTREE = 2 };

/* Number of doubles in one observable record. */
#define TDKS_RECORD 8

/*
 * Create a system on the current CUDA device.
 *   nx, ny, nz  grid points per axis (each >= fd_order/2 + 1; for bc = TDKS_BC_BLOCH each >= fd_order/2)
 *   h           grid spacing (bohr), > 0
 *   fd_order    4 or 8 (13- or 25-point star Laplacian)
 *   bc          TDKS_BC_ZERO: orbitals vanish outside the box (finite systems);
 *               TDKS_BC_BLOCH: periodic cell whose orbitals obey the Bloch condition
 *               psi(r + L e_a) = exp(i k_a L) psi(r) (Sec. "Periodic systems": Bloch theorem)
 *   prec        TDKS_C128: all of H psi and the series in complex128;
 *               TDKS_C64: H psi and the Taylor terms in complex64, the state (the sum of the
 *               series), density, potentials and all reductions in FP64
 *   n_orb       orbitals per k-point (>= 1)
 *   n_k         k-points (1 for TDKS_BC_ZERO)
 *   kpts        [n_k][3] k-vectors (bohr^-1), or NULL for k = 0
 *   kweights    [n_k] weights, or NULL for 1/n_k each
 *   stream      cudaStream_t on which all work of this system is enqueued (NULL: default)
 *   out         receives the handle
 * The local potential starts at zero, no projectors, no field, LDA exchange on with
 * occupation 2.  Allocates all device buffers of the system.
 */
int tdks_create_grid(int nx, int ny, int nz, double h, int fd_order, int bc, int prec, int n_orb, int n_k,
                     const double *kpts, const double *kweights, void *stream, tdks_sys *out);

/* Free the system and its device memory (synchronises its stream first). */
int tdks_destroy(tdks_sys sys);

/* V_loc: host array [nz][ny][nx] of doubles (Ha), copied. */
int tdks_set_local_potential(tdks_sys sys, const double *v);

/* Orbitals: host array in the host layout (2 * n_k * N * n_orb doubles), copied (the call
 * returns once the buffer has been read; pinned memory gives the fastest upload) and packed
 * on the device in chunks that overlap the copy, together with the density of the new
 * state.  The new state replaces the old one for all work enqueued on the system's stream
 * after the call; work enqueued before it still sees the old state.  The copy waits only for
 * the previous upload's packing, so an upload issued while a propagation runs overlaps it.
 * The packing runs on the system's stream, after the work enqueued there, unless the system
 * has two upload buffers (tdks_set_upload_buffers). */
int tdks_set_orbitals(tdks_sys sys, const double *psi);

/* Upload buffers of a system: 1 (default), or 2 for a stream of uploads (one per step, say):
 * each tdks_set_orbitals then packs the new state into a second state buffer (one more state
 * and density array, allocated here) on a stream of its own, so that the packing overlaps
 * the work enqueued before the call too, and the system switches buffers for the work
 * enqueued after it.  A system with two buffers cannot join a batch (TDKS_EINVAL from
 * tdks_batch_create).  n = 1 frees the second buffer.  Synchronises the system's stream. */
int tdks_set_upload_buffers(tdks_sys sys, int n);

/* Copy the current orbitals out into the host layout.  Synchronises. */
int tdks_get_orbitals(tdks_sys sys, double *psi_out);

/*
 * Kleinman-Bylander projectors (the paper's norm-conserving pseudopotentials carry
 * non-local parts, Sec. "Magneto-optics"; their shape is not printed there, so the
 * projectors are Gaussian-times-polynomial): for atom a at R_a and d = r - R_a,
 *   beta_a1 = g, beta_a2..4 = (d_x, d_y, d_z) g,  g = exp(-|d|^2 / (2 r_c^2)),  |d| <= r_cut.
 *   pos  [n_atoms][3] positions (bohr), D [n_atoms][4] strengths D_aj (Ha), both copied.
 * In a periodic cell the sphere points are taken over the neighbouring images with the
 * Bloch phase exp(i k.T); in the velocity gauge beta carries exp(-i A.d).
 * n_atoms = 0 removes the projectors.
 */
int tdks_set_atoms_projectors(tdks_sys sys, int n_atoms, const double *pos, const double *D, double r_c,
                              double r_cut);

/*
 * External field (forward coupling to a classical laser, Sec. "Maxwell ... coupling").
 *   gauge     TDKS_GAUGE_NONE; TDKS_GAUGE_LENGTH (finite box only): +E(t).r with
 *             E(t) = amp env(t) sin(omega t) pol; TDKS_GAUGE_VELOCITY (periodic cell only):
 *             A(t) = amp env(t) sin(omega t) pol, E = -dA/dt.
 *   envelope  TDKS_ENV_NONE (env = 1) or TDKS_ENV_SIN2: env = sin^2(pi t / t_total) on
 *             [0, t_total], 0 outside.
 */
int tdks_set_field(tdks_sys sys, int gauge, const double pol[3], double amp, double omega, int envelope,
                   double t_total);

/* Exchange-correlation term: TDKS_XC_NONE or TDKS_XC_LDA_X (spin-unpolarised LDA
 * exchange, v_x = -(3n/pi)^(1/3)); occupation f > 0 of every orbital (2 for closed shells).
 * TDKS_XC_LDA_X_HARTREE adds the Hartree potential of the density (the other density-dependent
 * part of the Kohn-Sham potential, which CFM4 of Sec. "New propagators for real-time TDDFT"
 * extrapolates with exchange): finite box, the Coulomb sum over grid cells
 * v_H(r_i) = h^3 sum_j n_j / |r_i - r_j| with a cell's own term n_i h^2 c0,
 * c0 = 3 ln(2 + sqrt 3) - pi/2, computed exactly by a zero-padded FFT; periodic cell,
 * v_H(G) = 4 pi n(G) / |G|^2 on the grid's plane waves (G = 0 dropped, neutralising
 * background).  The record's energy then adds E_H = 1/2 int n v_H.  Every propagator takes v_H
 * with v_x (CFM4, EMR and AETRS extrapolate their sum, ETRS takes both from the trial's density,
 * RK4 rebuilds both at every stage); TDKS_EINVAL from tdks_batch_create; grid edges with prime factors <= 13
 * (periodic cells) and transforms of at most 1024 points per axis (TDKS_EINVAL otherwise).
 * Allocates the transform workspace (two complex arrays of the padded grid) once. */
int tdks_set_xc(tdks_sys sys, int xc, double occupation);

/*
 * Packed device layout: *bs = orbitals per batch, *n_batches per k-point,
 * *elem_bytes = 16 (complex128) or 8 (complex64), *bytes = size of one packed array.
 * Any output pointer may be NULL.
 */
int tdks_layout(tdks_sys sys, int *bs, int *n_batches, int *elem_bytes, long long *bytes);

/*
 * dev_out = H[n, t] dev_in for every orbital and k-point, where n is the density of the
 * system's current orbitals and the field is taken at time t.  dev_in and dev_out are
 * device arrays in the packed layout (see tdks_layout), distinct, owned by the caller.
 * Asynchronous on the system's stream.
 */
int tdks_apply_H(tdks_sys sys, double t, const void *dev_in, void *dev_out);

/*
 * Advance the orbitals by n_steps steps of length dt from time t0.  Each step is split
 * into `substeps` equal Taylor sub-steps (0: automatic, from a bound on |H|, so that
 * dt_sub * |lambda_max| <= 2.5 < 2 sqrt 2, the stability limit of the 4th-order Taylor
 * series).  A sub-step whose kinetic part alone exceeds the limit is refused with
 * TDKS_EUNSTABLE.  One observable record is stored per step for the state at the start
 * of that step (see tdks_reductions).  Asynchronous on the system's stream.
 */
int tdks_propagate_n(tdks_sys sys, double t0, double dt, int n_steps, int substeps);

/*
 * Propagator of tdks_propagate_n.  TDKS_PROP_TAYLOR4 (default): the 4th-order Taylor series
 * above.  TDKS_PROP_CFM4: the order-four commutator-free Magnus expansion of Sec. "New
 * propagators for real-time TDDFT",
 *   phi(t + ds) = exp(-i ds (a1 H[t1] + a2 H[t2])) exp(-i ds (a2 H[t1] + a1 H[t2])) phi(t),
 *   a1,2 = (3 -+ 2 sqrt3)/12,  t1,2 = t + (1/2 -+ sqrt3/6) ds,
 * per sub-step ds = dt / substeps.  As a1 + a2 = 1/2, each factor is a Taylor-4
 * exponential of ds/2 of H with the field 2 (a2 E(t1) + a1 E(t2)) (first factor; a1 and
 * a2 swapped in the second) and the exchange potential extrapolated the same way to t1 and
 * t2 from its values at the starts of the last four sub-steps (Lagrange, order four; fewer
 * points while the history fills).  The paper also names the exponential midpoint rule and
 * the enforced time-reversal symmetry scheme among the propagators in use (same section)
 * without stating them; their usual forms, with the exchange potential extrapolated the
 * same way (the explicit variant of the time-reversal scheme, "approximate ETRS"):
 *   TDKS_PROP_EMR:   phi(t + ds) = exp(-i ds H[t + ds/2]) phi(t),
 *   TDKS_PROP_AETRS: phi(t + ds) = exp(-i ds/2 H[t + ds]) exp(-i ds/2 H[t]) phi(t),
 * where H[t] uses v_x of the current state exactly.  Each exponential is a Taylor-4 series.
 * The history is cleared by tdks_set_orbitals and by this call.  Length gauge or no field
 * (TDKS_EINVAL with the velocity gauge at propagation); the stability limit applies to each
 * exponential's length (ds/2, or ds for EMR).  Records as for Taylor-4.  Batches propagate
 * with Taylor-4.
 */
#define TDKS_PROP_TAYLOR4 0
#define TDKS_PROP_CFM4 1
#define TDKS_PROP_EMR 2
#define TDKS_PROP_AETRS 3
/*
 * TDKS_PROP_RK4: the classical fourth-order Runge-Kutta method (the same section's list of
 * propagators names Runge-Kutta) on d phi/dt = -i H[n(phi), t] phi, with the density rebuilt at every
 * stage from the stage vector and the field at the stage times t, t + ds/2, t + ds/2, t + ds;
 * the slope weights 1/6, 1/3, 1/3, 1/6.  Fourth order also in the density coupling, at four
 * H applications per sub-step: a reference integrator.  Complex128 systems only (TDKS_EINVAL
 * for complex64); any gauge; its stability limit on the imaginary axis is the Taylor-4 one.
 */
#define TDKS_PROP_RK4 4
/*
 * TDKS_PROP_ETRS: enforced time-reversal symmetry with its trial state, as the propagator
 * review that the same section cites defines it (the scheme of the hydrogen-fluoride dimer run
 * of Sec. "vdW-TS" and of the first GPU port of Sec. "GPUs"):
 *   trial:  phi~ = exp(-i ds H[t]) phi(t),
 *   step:   phi(t + ds) = exp(-i ds/2 H[t + ds]) exp(-i ds/2 H[t]) phi(t),
 * H[t] with v_x of phi(t) and E(t), H[t + ds] with v_x of the trial's density and E(t + ds).
 * Three Taylor-4 exponentials per sub-step (lengths ds, ds/2, ds/2; the stability limit
 * applies to ds); without exchange the trial is skipped and the step is the AETRS step.  One
 * extra state-sized buffer (allocated here).  Length gauge or no field, as AETRS.
 */
#define TDKS_PROP_ETRS 5
int tdks_set_propagator(tdks_sys sys, int propagator);

/*
 * State-parallel propagation (one molecule over several GPUs, each holding a slice of the
 * orbitals).  The Hamiltonian couples the orbitals only through the density
 * n(r) = sum_i f_i |phi_i(r)|^2 in v_x[n] (Sec. "New propagators for real-time TDDFT":
 * H[n(t), t]); everything else in a Taylor sub-step acts on each orbital alone.  A system
 * created with its slice's n_orb becomes one rank of such a run once an exchange hook is
 * set: wherever the library needs n (every sub-step of tdks_propagate_n, tdks_observe,
 * tdks_apply_H) it sums its own states' density into a device buffer of N doubles
 * (N = nx ny nz; the k-points' weights already applied) and calls
 *     fn(dev_buf, N, stream, ctx),
 * which must replace dev_buf, in place, with the sum of all ranks' buffers (an allreduce)
 * before work later enqueued on `stream` (the system's cudaStream_t) reads it; v_x and the
 * density terms of the record are then built from that sum.  For each observable record
 * it calls fn once more with n = 4 (this rank's band energy sum_i f_i <phi_i|H|phi_i> and
 * its three current sums) to get the whole system's.  Every rank must make the same calls
 * in the same order with the same arguments (times, fields, steps), and every rank's
 * record is then the whole system's.  fn returns 0 on success; any other value stops the
 * call with TDKS_EDEVICE.  fn runs on the calling thread, while earlier work may still run
 * on the stream.  Every rank holds the same k-points, grid, potentials, projectors and
 * field.  Every propagator: the density behind each potential it builds (the pushed v_x of
 * CFM4, EMR and AETRS, the state's and the trial's in ETRS, each RK4 stage's) is exchanged
 * first, so a sub-step calls fn once per such density.  fn = NULL detaches the hook.  ctx is
 * passed through untouched.
 */
typedef int (*tdks_exchange_fn)(double *dev_buf, long long n, void *stream, void *ctx);
int tdks_set_exchange(tdks_sys sys, tdks_exchange_fn fn, void *ctx);

/*
 * Checkpoint and resume.  tdks_save writes everything a propagation continues from: grid,
 * precision, k-points, potential, projectors, field, exchange settings, propagator (with its
 * exchange history), tile and sweep-shape choices, the device state exactly as stored (the
 * hi and lo parts of a complex64 state), the density of that state, the step count, the
 * clock of tdks_set_clock and the stored records (the last min(steps, 65536)).  It waits for
 * the system's stream, writes `path` + ".tmp" and renames it to `path` once complete (an
 * existing file is replaced only by a whole checkpoint).  The exchange hook is not saved.
 * tdks_load creates a new system on `stream` (a cudaStream_t, or NULL) from such a file; it
 * continues bit for bit as the saved system would have, with the same records and step
 * count.  TDKS_EINVAL for a file that cannot be opened or written, is not a checkpoint, is
 * truncated, or fails its checksum; the other codes as for the calls that set each part.
 * The file is little-endian and holds doubles as stored in memory.
 */
int tdks_save(tdks_sys sys, const char *path);
int tdks_load(const char *path, void *stream, tdks_sys *out);

/* Sub-step count the automatic policy of tdks_propagate_n picks for step dt. */
int tdks_auto_substeps(tdks_sys sys, double dt, int *substeps);

/*
 * Copy n observable records, starting at step index step_from (counted over the life of
 * the system), into out[n][TDKS_RECORD]:
 *   [0] t       state time t0 + s dt
 *   [1] norm    sum_k w_k sum_i ||phi_ik||^2 h^3
 *   [2] E       sum_k w_k f <phi|H|phi> - int n v_x + E_x  (field of the step's first
 *               sub-step, i.e. at t + dt_sub/2)
 *   [3] E_x     LDA exchange energy (0 when exchange is off)
 *   [4..6]      finite box: dipole d = int r n(r) dr (Sec. "Local domains");
 *               periodic cell: current J = -(1/Omega)(sum_k w_k f <phi|-i grad_h|phi> + A int n)
 *               (eqn. current_density, local part)
 *   [7]         field along pol at t + dt_sub/2 (E in length gauge, A in velocity gauge)
 * Records are kept in a ring of 65536 steps.  Synchronises.
 */
int tdks_reductions(tdks_sys sys, long long step_from, int n, double *out);

/* Number of steps recorded so far. */
int tdks_step_count(tdks_sys sys, long long *count);

/* Observable record of the current state at t_state with the field at t_field
 * (layout as in tdks_reductions).  Synchronises. */
int tdks_observe(tdks_sys sys, double t_state, double t_field, double *out);

/*
 * Kernel accounting.  tdks_set_profiling(sys, 1) brackets every stencil-sweep launch
 * with CUDA events on the system's stream; tdks_kernel_time(sys, kind, &ms, &n) then
 * returns the summed device time and launch count since the last call and resets them
 * (kind 0: stencil sweeps, 1: projector gathers, 2: density/LDA/finalise; 3..6: the stencil
 * sweeps of Taylor terms 1..4, which kind 0 counts too).  Synchronises.
 * tdks_launch_count returns the number of kernels this system has launched.
 */
int tdks_set_profiling(tdks_sys sys, int on);
int tdks_kernel_time(tdks_sys sys, int kind, double *ms, long long *launches);
int tdks_launch_count(tdks_sys sys, long long *count);

/* Stencil tile shape (x, y points per CTA; one of 16x8, 32x4, 8x8) and z-chunk
 * length (0: automatic).  Results do not depend on the choice except in the last bits of
 * the energy and current sums. */
int tdks_set_tile(tdks_sys sys, int tx, int ty, int zc);

/*
 * Failure detection of the warp-specialised TMA sweeps.  Every wait in them is bounded (4e9
 * GPU clock cycles, ~2 s).  A wait that runs out (a copy that does not land, a ring slot that
 * is not released, a claimed work item that does not arrive) makes its CTA give up: its other
 * warps stop at their next wait, its producer waits (at most ~0.1 s each) for the copies it
 * has in flight, the error word is set, and the next synchronising call (tdks_reductions,
 * tdks_get_orbitals, tdks_observe, tdks_autotune, tdks_get_tsurff) returns TDKS_ETIMEOUT and
 * clears it; the orbitals are then undefined until set again.  withhold = 1 injects that
 * failure for tests: the sweeps' producer warps make no claim and issue no copy, so every
 * consumer warp's first wait runs out after the bound (nothing is read or written by those
 * sweeps, no copy is in flight); withhold = 0 restores normal sweeps.  No passage of the
 * paper defines this: it is the library's own failure handling.  Synchronises the system's
 * stream; applies to launches made after the call (batches: to batches created after it).
 */
int tdks_set_failure_injection(tdks_sys sys, int withhold);

/* Stencil sweep implementation: 0 (default) streams the input planes with TMA bulk
 * tensor copies where that applies (finite boxes, 16x8 tiles) into a warp-specialised
 * kernel (one producer warp, eight consumer warps); 1 always uses the general sweep (loads
 * through L1/L2; the only one for periodic cells); 2 is the TMA sweep in which all warps of
 * a CTA advance plane by plane together.  All compute the same values (to the last bits of
 * FP64 rounding in the energy and current sums). */
int tdks_set_sweep_path(tdks_sys sys, int path);

/*
 * Tile shapes of the warp-specialised TMA sweep (path 0, finite boxes, 16x8 system tile)
 * and the autotuner that picks one per Taylor-term sweep.  No passage of the paper
 * defines these: they choose how the stencil (Sec. "Maxwell ... coupling", finite
 * differences on a uniform grid) is tiled on the GPU and do not change its values (each
 * point's arithmetic and order of terms is the same in every shape; energy and current
 * partial sums are grouped per consumer warp, so those change in the last bits).
 *
 * tdks_sweep_shape_info: shape s (0 .. count-1) covers tx x ty points of one orbital batch
 * per work item with `warps` consumer warps, each thread computing `rows` y-adjacent
 * points of one 16-byte vector (two complex64 or one complex128 values; 4 vectors per point,
 * so warps x 32 = 4 tx ty / rows).  Shape 5 computes complex64 finite boxes with one
 * complex64 value (8 bytes) per thread vector, 8 vectors per point (warps x 32 = 8 tx ty /
 * rows): fewer shared-memory bytes per value at the same register budget; complex128
 * systems and periodic cells run it as shape 2 (the same tile and warp count).  *count (if
 * not NULL) receives the number of shapes; tx/ty/rows/warps may be NULL.  TDKS_EINVAL for a
 * shape out of range.
 */
int tdks_sweep_shape_info(int shape, int *count, int *tx, int *ty, int *rows, int *warps);
/* Shape of Taylor-term sweep `sweep` (0 = t1 from psi, 1 = t2, 2 = t3, 3 = t4 and the
 * combine), or of all four when sweep = -1.  Synchronises the system's stream. */
int tdks_set_sweep_shape(tdks_sys sys, int sweep, int shape);
int tdks_get_sweep_shape(tdks_sys sys, int sweep, int *shape);
/* Autotuner: times every shape on each of the four Taylor-term sweeps of this system, on
 * its own grid, orbitals and projectors (in the velocity gauge with a vector potential
 * amp * pol, so that the gauge term is timed too; reps launches each after one warm-up
 * launch, CUDA events on the system's stream), and keeps the fastest shape per sweep.  The state psi is
 * not changed; the Taylor-term buffers and the density partials are overwritten (the next
 * propagation or H application rebuilds them).  ms (if not NULL) receives the mean
 * milliseconds per launch as ms[shape * 4 + sweep] (count * 4 values).  Systems that do not
 * take the warp-specialised sweep keep their settings and ms is filled with -1.
 * Synchronises; TDKS_ETIMEOUT if a sweep gave up waiting for its copies. */
int tdks_autotune(tdks_sys sys, int reps, double *ms);

/*
 * Batched propagation of many independent finite-box systems (uneven grids, orbital and
 * atom counts), the many-systems workload: per Taylor term one persistent sweep launch
 * walks the work items of every system, with one batched projector gather, one batched
 * LDA/V_eff launch and the record/clock kernels; a sub-step is captured once as a CUDA
 * graph and replayed.  Each system advances from its own clock.  Results equal those of
 * tdks_propagate_n on each system alone (the same per-point arithmetic and reduction
 * order).
 */
typedef struct tdks_batch *tdks_batch_t;

/* Clock of a system for batched propagation: state time t, step length dt, sub-steps
 * per step (checked against the stability limit like tdks_propagate_n).
 * tdks_propagate_n also leaves the clock at t0 + n_steps dt. */
int tdks_set_clock(tdks_sys sys, double t, double dt, int substeps);
int tdks_get_clock(tdks_sys sys, double *t, long long *steps);

/* systems[n]: finite boxes sharing fd_order, precision and sub-step count, with orbitals
 * set; they must outlive the batch and use the batch's stream (their work is enqueued
 * there).  Device parameter tables are built here; the systems' potentials, projectors
 * and fields must not change while the batch exists. */
int tdks_batch_create(const tdks_sys *systems, int n, void *stream, tdks_batch_t *out);
/* Advance every system of the batch by n_steps steps of its own dt (one observable record
 * per step, as tdks_propagate_n).  use_graph = 1 replays a captured CUDA graph per
 * sub-step.  Asynchronous on the batch's stream. */
int tdks_batch_propagate(tdks_batch_t batch, int n_steps, int use_graph);
int tdks_batch_launch_count(tdks_batch_t batch, long long *count);
/* Sweep tile shape of Taylor term `term` (0..3, or -1 for all) of the batched sweep (see
 * tdks_sweep_shape_info); synchronises the batch's streams.  No passage of the paper
 * defines tiles; results do not depend on the choice except in the last bits of the
 * energy sums. */
int tdks_batch_set_shape(tdks_batch_t batch, int term, int shape);
int tdks_batch_get_shape(tdks_batch_t batch, int term, int *shape);
/* Autotuner of the batched sweep: times every shape on each Taylor term's batched sweep
 * over all the batch's systems (reps launches after one warm-up, CUDA events) and keeps
 * the fastest per term.  No system's state changes; the Taylor-term buffers and density
 * partials are overwritten and rebuilt by the next tdks_batch_propagate.  ms (if not NULL):
 * mean milliseconds per launch as ms[shape * 4 + term].  Synchronises. */
int tdks_batch_autotune(tdks_batch_t batch, int reps, double *ms);
int tdks_batch_destroy(tdks_batch_t batch);

/*
 * H applied without allocating device memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc, such as code running inside a
 * host framework that owns all device memory through its own pool, or a real-time loop
 * that cannot afford the device-wide synchronisation an allocation or free may cause.
 *
 * dev_out = (-1/2 Lap_h + V_loc) dev_in on a finite box (zero boundary), for one k-point:
 * no exchange term, no projectors, no field.  nx, ny, nz, h, fd_order, prec and n_orb as in
 * tdks_create_grid; dev_vloc: device array [nz][ny][nx] of doubles; dev_in / dev_out:
 * distinct device arrays in the packed layout of such a system (BS = 4 for TDKS_C128,
 * 8 for TDKS_C64, zero-padded batches); stream: cudaStream_t or NULL.  The caller owns all
 * three buffers.  The call synchronises the stream before it returns.
 *
 * Scratch (one 16-byte record per point with the potential, an error word and a work-item
 * counter) lives in a fixed file-scope device array of 16 MiB + 256 B that every GPU loading the library holds until
 * the process exits; grids above 2^20 = 1,048,576 points are rejected with TDKS_EINVAL.
 * All calls on a device share that array and each call overwrites it, so calls whose work
 * overlaps on the GPU (several streams or host threads) race: serialise them.  The first
 * call on a device looks up the array's device address on that device.  Returns
 * TDKS_ETIMEOUT if a sweep gave up waiting for its copies.
 */
int tdks_apply_H_noalloc(int nx, int ny, int nz, double h, int fd_order, int prec, int n_orb,
                         const double *dev_vloc, const void *dev_in, void *dev_out, void *stream);

/*
 * Kinetic heat current of a periodic cell (Sec. "Conductivities", eqn. KEcurrent), cell-averaged:
 *   J_t = (1/Omega) sum_k w_k f int [J_t(r)] dr,
 *   [J_t]_i = (i/8) ([d_i phi^*][Lap phi] - [Lap phi^*][d_i phi] - [d_i grad phi^*].[grad phi]
 *              + [grad phi^*].[d_i grad phi]),
 * the printed last pair taken with the sign that makes J_t real (a plane wave then carries minus
 * its kinetic energy times its velocity, the sign convention of the charge current J of the
 * record); derivatives as in H (central differences of the system's order with Bloch images,
 * covariant d + i A with the vector potential at t_field in the velocity gauge).  out[3]
 * receives J_t of the current state.  Periodic cells only (TDKS_EINVAL otherwise).  Synchronises.
 */
int tdks_heat_current(tdks_sys sys, double t_field, double *out);

/*
 * t-SURFF photoelectron amplitudes (Sec. "t-SURFF": the expansion coefficients b_i(p, t) of
 * the orbitals on Volkov states, obtained from the continuity equation as the time integral
 * of the current through a surface S):
 *   b_i(p, T) = int dt oint_S ds n . <chi_p| j |phi_i>,  <chi_p| j |phi> = 1/2 chi_p^* (k_p phi - i grad_h phi),
 *   chi_p = (2 pi)^(-3/2) exp(i k_p.r - i Phi_p),  k_p = p + a(t),  a = -int E,
 *   Phi_p = 1/2 int |k_p|^2  (Volkov states of -1/2 Lap + E(t).r, the length gauge of the
 *   finite boxes; the section prints the velocity-gauge form).
 * S is the surface of the box of grid planes x = x[box[0]], x[box[1]], y = y[box[2]], y[box[3]],
 * z = z[box[4]], z[box[5]], integrated face by face with the two-dimensional trapezoid rule and
 * the outward normal n; grad_h is the central difference of the system's order; time runs
 * from the start of the first tdks_propagate_n after this call, and the time integral is the
 * trapezoid rule over the configured steps (the flux of the state at the start of each step;
 * a(t), int a and int |a|^2 advanced per step by the classical Runge-Kutta method).  Later
 * propagations must continue in time from where the last one ended (TDKS_EINVAL otherwise).
 *   box  six plane indices with fd_order/2 <= lo < hi <= n - 1 - fd_order/2 on each axis
 *   p    [n_p][3] momenta (bohr^-1), copied; n_p = 0 turns t-SURFF off
 * Finite boxes with one k-point only (TDKS_EINVAL otherwise).  Resets the amplitudes to zero.
 * The amplitudes are not part of a checkpoint.  Synchronises.
 */
int tdks_set_tsurff(tdks_sys sys, const int box[6], int n_p, const double *p);
/* b [n_orb][n_p] complex amplitudes (interleaved re, im doubles) accumulated so far, and the
 * time since the accumulation started (either pointer may be NULL).  Synchronises;
 * TDKS_ESTATE when t-SURFF is not set. */
int tdks_get_tsurff(tdks_sys sys, double *b, double *t_rel);

/*
 * Fused multiply-add throughput of the current device, measured by the library's own probe
 * kernel: prec = TDKS_C128 for FP64 FMAs, TDKS_C64 for FP32 ones; *fma_per_s receives FMA
 * instructions (thread-level) per second, 2 FLOP each.  The paper has no counterpart: it
 * gives the denominator of the complex128 path's roofline, whose stencil sweeps are bound
 * by the FP64 pipe rather than by HBM on GPUs with a low FP64 rate.  Allocates a small
 * buffer, runs on the legacy default stream and synchronises.
 */
int tdks_fma_rate(int prec, double *fma_per_s);

const char *tdks_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TDKS_H */
