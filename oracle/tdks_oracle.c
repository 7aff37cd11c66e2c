/*
 * FP64 CPU oracle for real-time TDDFT propagation on a uniform 3D grid.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this file's library.  It shares no code, header, table or helper
 * with the CUDA library; the two meet only in the seeded inputs.
 *
 * What it computes follows the paper's statement of the problem (arXiv:1912.07921):
 *   - the TDKS system  dphi_i/dt = -i H[n(t), t] phi_i,  phi(t0) = phi^0
 *     (Sec. "New propagators for real-time TDDFT", first three equations);
 *   - the adiabatic approximation: the exchange potential depends on the current
 *     density only (same section);
 *   - the high-order finite-difference Laplacian and gradient on the real-space grid
 *     (Sec. "Maxwell ... coupling", discretisation paragraph; Sec. "Periodic systems");
 *   - the LDA exchange energy E_x = int n e_x(n) (Sec. "Local domains", LDA equation);
 *   - the Hartree potential of the density, for an exchange-plus-Hartree mode (the
 *     density-dependent potentials that CFM4 extrapolates, Sec. "New propagators for
 *     real-time TDDFT");
 *   - the time-dependent dipole d(t) = int r n(r,t) dr (Sec. "Local domains");
 *   - the macroscopic current J = -(i/Omega) int sum_i phi_i [H, r] phi_i
 *     (Sec. "Conductivities", eqn. current_density), with the projectors' commutator;
 *   - the velocity-gauge field E = -dA/dt (same section);
 *   - closed-shell occupations f_i = 2 (Sec. "t-SURFF", closed shells);
 *   - the t-SURFF photoelectron amplitudes: the time integral of the Volkov-state
 *     current through a surface (Sec. "t-SURFF", eqns. for chi_p, b_i and the current);
 *   - the kinetic heat current (Sec. "Conductivities", eqn. KEcurrent).
 * The exponential is a 4th-order Taylor series with H frozen over a (sub-)step; the
 * paper does not print this propagator, so the oracle takes the readings listed at each
 * function.  Everything is plain loops in double precision; OpenMP only splits the
 * outermost independent loop.
 *
 * Layout: orbitals are complex doubles, index [k][z][y][x][orb] (state index innermost,
 * Sec. "Memory layout").  Every function is pinned, in tests/test_oracle_pins.py, by closed
 * forms, invariants, brute force or library routines.  The paper prints no worked-example
 * numbers for this path; the printed values used as pins are the CFM4 constants and (through
 * the cited literature) the finite-difference weights, both under tests/golden/.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
  int nx, ny, nz;
  double h;
  int fd_order;       /* 2M: 4 or 8 */
  int bc;             /* 0: psi = 0 outside the box; 1: Bloch-twisted periodic cell */
  int n_orb;
  int n_k;
  const double *kpts; /* [n_k][3] */
  const double *kw;   /* [n_k] */
  const double *vloc; /* [nz][ny][nx] */
  int xc;             /* 0: none; 1: LDA exchange; 2: LDA exchange and Hartree */
  double occ;         /* occupation of every orbital */
  int gauge;          /* 0: no field; 1: length gauge E(t).r; 2: velocity gauge A(t) */
  double pol[3];
  double amp, omega;
  int envelope;       /* 0: none; 1: sin^2(pi t / t_total) on [0, t_total] */
  double t_total;
  int n_atoms;
  const double *pos;  /* [n_atoms][3] */
  const double *D;    /* [n_atoms][4] */
  double r_c, r_cut;
} oracle_sys;

static long npts(const oracle_sys *s) { return (long)s->nx * s->ny * s->nz; }

/* Compensated (Kahan) running sum.  The grid integrals below add up to ~10^8 terms; a
 * plain running sum of that many positive terms drifts by ~1e-11 relative, which would
 * swamp the 1e-12 parity tolerance, while the compensated sum stays at rounding level.
 * The paper defines these quantities as integrals; the order of summation is not part
 * of the method. */
typedef struct { double s, c; } ksum;
static void kadd(ksum *k, double x) {
  double y = x - k->c;
  double t = k->s + y;
  k->c = (t - k->s) - y;
  k->s = t;
}

/* --------------------------------------------------------------------------------
 * Finite-difference weights.  Central differences of order 2M on a uniform grid; the
 * paper takes its weights from its Ref. (PRB 78, 075109) without printing them.  Closed
 * forms: second derivative c_m = 2(-1)^(m+1) (M!)^2 / (m^2 (M-m)! (M+m)!),
 * c_0 = -2 sum c_m; first derivative d_m = (-1)^(m+1) (M!)^2 / (m (M-m)! (M+m)!).
 * ------------------------------------------------------------------------------ */
static double fact(int n) { double f = 1.0; for (int i = 2; i <= n; i++) f *= i; return f; }

void oracle_fd_laplacian_weights(int M, double *c) {
  double s = 0.0;
  for (int m = 1; m <= M; m++) {
    double sign = (m % 2 == 1) ? 1.0 : -1.0;
    c[m] = 2.0 * sign * fact(M) * fact(M) / ((double)m * m * fact(M - m) * fact(M + m));
    s += c[m];
  }
  c[0] = -2.0 * s;
}

void oracle_fd_gradient_weights(int M, double *d) {
  d[0] = 0.0;
  for (int m = 1; m <= M; m++) {
    double sign = (m % 2 == 1) ? 1.0 : -1.0;
    d[m] = sign * fact(M) * fact(M) / ((double)m * fact(M - m) * fact(M + m));
  }
}

/* Grid coordinates: centred box for finite systems, cell from the origin for solids. */
static double coord(const oracle_sys *s, int axis, int i) {
  int n = axis == 0 ? s->nx : (axis == 1 ? s->ny : s->nz);
  if (s->bc == 0) return ((double)i - 0.5 * (double)(n - 1)) * s->h;
  return (double)i * s->h;
}

/* --------------------------------------------------------------------------------
 * External field.  Length gauge: E(t) = amp env(t) sin(omega t) pol, coupling +E.r
 * (electron charge -1).  Velocity gauge: A(t) = amp env(t) sin(omega t) pol and
 * E = -dA/dt (Sec. "Conductivities"; c absorbed into A).
 * ------------------------------------------------------------------------------ */
static double envelope(const oracle_sys *s, double t, double *denv) {
  if (s->envelope == 1) {
    if (t < 0.0 || t > s->t_total) { *denv = 0.0; return 0.0; }
    double a = M_PI * t / s->t_total;
    *denv = 2.0 * sin(a) * cos(a) * M_PI / s->t_total;
    return sin(a) * sin(a);
  }
  *denv = 0.0;
  return 1.0;
}

void oracle_field(const oracle_sys *s, double t, double *E, double *A) {
  double denv, env = envelope(s, t, &denv);
  double f = s->amp * env * sin(s->omega * t);
  double df = s->amp * (denv * sin(s->omega * t) + env * s->omega * cos(s->omega * t));
  for (int a = 0; a < 3; a++) {
    E[a] = 0.0;
    A[a] = 0.0;
    if (s->gauge == 1) E[a] = f * s->pol[a];
    if (s->gauge == 2) { A[a] = f * s->pol[a]; E[a] = -df * s->pol[a]; }
  }
}

/* --------------------------------------------------------------------------------
 * Boundary extension.  Value of orbital (k, o) at integer grid position (ix, iy, iz),
 * which may lie outside the box: zero for finite systems; for a periodic cell the
 * Bloch condition psi(r + L e_a) = exp(i k_a L_a) psi(r) folds it back.
 * ------------------------------------------------------------------------------ */
static cplx fetch(const oracle_sys *s, const cplx *psi, int k, int o, int ix, int iy, int iz) {
  int n[3] = {s->nx, s->ny, s->nz};
  int i[3] = {ix, iy, iz};
  cplx phase = 1.0;
  for (int a = 0; a < 3; a++) {
    if (i[a] >= 0 && i[a] < n[a]) continue;
    if (s->bc == 0) return 0.0;
    int w = (int)floor((double)i[a] / (double)n[a]);
    i[a] -= w * n[a];
    double L = n[a] * s->h;
    phase *= cexp(I * s->kpts[3 * k + a] * L * (double)w);
  }
  long p = ((long)i[2] * s->ny + i[1]) * s->nx + i[0];
  return phase * psi[((long)k * npts(s) + p) * s->n_orb + o];
}

/* --------------------------------------------------------------------------------
 * Density n(r) = sum_k w_k sum_i f_i |phi_ik(r)|^2  (TDKS density; f_i = occ).
 * ------------------------------------------------------------------------------ */
void oracle_density(const oracle_sys *s, const cplx *psi, double *n) {
  long N = npts(s);
#pragma omp parallel for
  for (long p = 0; p < N; p++) {
    double acc = 0.0;
    for (int k = 0; k < s->n_k; k++)
      for (int o = 0; o < s->n_orb; o++) {
        cplx v = psi[((long)k * N + p) * s->n_orb + o];
        acc += s->kw[k] * s->occ * (creal(v) * creal(v) + cimag(v) * cimag(v));
      }
    n[p] = acc;
  }
}

/* --------------------------------------------------------------------------------
 * LDA exchange, spin-unpolarised: e_x(n) = -(3/4)(3 n / pi)^(1/3) per particle,
 * v_x = d(n e_x)/dn = -(3 n / pi)^(1/3);  E_x = sum_r n e_x(n) h^3.
 * ------------------------------------------------------------------------------ */
double oracle_lda_x(const oracle_sys *s, const double *n, double *vx) {
  long N = npts(s);
  double h3 = s->h * s->h * s->h;
  ksum ex = {0.0, 0.0};
  for (long p = 0; p < N; p++) {
    double c = cbrt(3.0 * n[p] / M_PI);
    if (vx) vx[p] = -c;
    kadd(&ex, n[p] * (-0.75 * c) * h3);
  }
  return ex.s;
}

double oracle_hartree(const oracle_sys *s, const double *n, double *vh); /* defined below */

/* The density-dependent potential of the xc setting: v = v_x (xc 1, exchange) or
 * v = v_x + v_H (xc 2, exchange and Hartree); returns E_x and puts E_H (0 without
 * Hartree) in *eh when eh is not NULL. */
static int has_density_potential(const oracle_sys *s) { return s->xc == 1 || s->xc == 2; }
static double density_potential(const oracle_sys *s, const double *n, double *v, double *eh) {
  const double ex = oracle_lda_x(s, n, v);
  double e = 0.0;
  if (s->xc == 2) {
    const long N = npts(s);
    double *vh = (double *)malloc(sizeof(double) * (size_t)N);
    e = oracle_hartree(s, n, vh);
    for (long p = 0; p < N; p++) v[p] += vh[p];
    free(vh);
  }
  if (eh) *eh = e;
  return ex;
}

/* --------------------------------------------------------------------------------
 * Kleinman-Bylander projectors.  The paper uses norm-conserving pseudopotentials with
 * non-local parts but prints no projector formula, so these are synthetic:
 *   beta_a1 = g(d), beta_a2..4 = (d_x, d_y, d_z) g(d),  g = exp(-|d|^2 / (2 r_c^2)),
 *   d = r - R_a, support |d| <= r_cut,   V_NL = sum_aj |beta_aj> D_aj <beta_aj|.
 * In a Bloch cell the sphere points are unwrapped positions u = cell point + T and carry
 * exp(i k.T); in the velocity gauge beta is dressed by exp(-i A.d) so that V_NL is the
 * gauge transform exp(-iA.r) V_NL exp(iA.r) and stays Hermitian.
 * ------------------------------------------------------------------------------ */
typedef struct {
  long cell;      /* flat cell index */
  double d[3];    /* u - R_a */
  double T[3];    /* lattice translation u - cell position */
} sphere_pt;

static int sphere_points(const oracle_sys *s, int a, sphere_pt **out) {
  int n[3] = {s->nx, s->ny, s->nz};
  int lo[3], hi[3];
  const double *R = s->pos + 3 * a;
  for (int ax = 0; ax < 3; ax++) {
    if (s->bc == 0) { lo[ax] = 0; hi[ax] = n[ax] - 1; }
    else {
      lo[ax] = (int)floor((R[ax] - s->r_cut) / s->h) - 1;
      hi[ax] = (int)ceil((R[ax] + s->r_cut) / s->h) + 1;
    }
  }
  long cap = (long)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
  sphere_pt *pts = (sphere_pt *)malloc(sizeof(sphere_pt) * (size_t)cap);
  int cnt = 0;
  for (int iz = lo[2]; iz <= hi[2]; iz++)
    for (int iy = lo[1]; iy <= hi[1]; iy++)
      for (int ix = lo[0]; ix <= hi[0]; ix++) {
        int ii[3] = {ix, iy, iz}, cc[3];
        double u[3], d[3], r2 = 0.0;
        for (int ax = 0; ax < 3; ax++) {
          if (s->bc == 0) u[ax] = coord(s, ax, ii[ax]);
          else u[ax] = (double)ii[ax] * s->h;
          d[ax] = u[ax] - R[ax];
          r2 += d[ax] * d[ax];
        }
        if (r2 > s->r_cut * s->r_cut) continue;
        sphere_pt *q = &pts[cnt++];
        for (int ax = 0; ax < 3; ax++) {
          int w = (int)floor((double)ii[ax] / (double)n[ax]);
          cc[ax] = ii[ax] - w * n[ax];
          q->T[ax] = (double)(w * n[ax]) * s->h;
          q->d[ax] = d[ax];
        }
        q->cell = ((long)cc[2] * s->ny + cc[1]) * s->nx + cc[0];
      }
  *out = pts;
  return cnt;
}

static void beta_values(const oracle_sys *s, const double *d, double *b) {
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double g = exp(-r2 / (2.0 * s->r_c * s->r_c));
  b[0] = g;
  b[1] = d[0] * g;
  b[2] = d[1] * g;
  b[3] = d[2] * g;
}

/* Number of grid points in the projector sphere of atom a (for tests). */
int oracle_sphere_count(const oracle_sys *s, int a) {
  sphere_pt *p;
  int c = sphere_points(s, a, &p);
  free(p);
  return c;
}

/* --------------------------------------------------------------------------------
 * H psi for every orbital and k-point.  H = -1/2 Lap_h + V_loc + v_x + E(t).r
 * (length gauge) or H = 1/2 (-i grad_h + A(t))^2 + V_loc + v_x (velocity gauge),
 * plus V_NL.  vx may be NULL (no exchange term).  The field is taken at time t.
 * ------------------------------------------------------------------------------ */
static void apply_H_field(const oracle_sys *s, const double *E, const double *A, const double *vx, const cplx *in,
                          cplx *out);

void oracle_apply_H(const oracle_sys *s, double t, const double *vx, const cplx *in, cplx *out) {
  double E[3], A[3];
  oracle_field(s, t, E, A);
  apply_H_field(s, E, A, vx, in, out);
}

/* H psi with the field given explicitly (E in the length gauge, A in the velocity gauge). */
static void apply_H_field(const oracle_sys *s, const double *E, const double *A, const double *vx, const cplx *in,
                          cplx *out) {
  int M = s->fd_order / 2;
  double c[5], d[5];
  oracle_fd_laplacian_weights(M, c);
  oracle_fd_gradient_weights(M, d);
  double h = s->h, h2 = h * h, h3 = h * h * h;
  long N = npts(s);
  int B = s->n_orb;
  double A2 = A[0] * A[0] + A[1] * A[1] + A[2] * A[2];

  /* local part: kinetic stencil, potential, field */
#pragma omp parallel for collapse(2)
  for (int k = 0; k < s->n_k; k++)
    for (int iz = 0; iz < s->nz; iz++)
      for (int iy = 0; iy < s->ny; iy++)
        for (int ix = 0; ix < s->nx; ix++) {
          long p = ((long)iz * s->ny + iy) * s->nx + ix;
          double v = s->vloc[p] + (vx ? vx[p] : 0.0);
          if (s->gauge == 1)
            v += E[0] * coord(s, 0, ix) + E[1] * coord(s, 1, iy) + E[2] * coord(s, 2, iz);
          if (s->gauge == 2) v += 0.5 * A2;
          for (int o = 0; o < B; o++) {
            cplx psi0 = fetch(s, in, k, o, ix, iy, iz);
            cplx lap = 3.0 * c[0] * psi0;
            cplx grad[3] = {0.0, 0.0, 0.0};
            for (int m = 1; m <= M; m++) {
              cplx xp = fetch(s, in, k, o, ix + m, iy, iz), xm = fetch(s, in, k, o, ix - m, iy, iz);
              cplx yp = fetch(s, in, k, o, ix, iy + m, iz), ym = fetch(s, in, k, o, ix, iy - m, iz);
              cplx zp = fetch(s, in, k, o, ix, iy, iz + m), zm = fetch(s, in, k, o, ix, iy, iz - m);
              lap += c[m] * (xp + xm + yp + ym + zp + zm);
              grad[0] += d[m] * (xp - xm);
              grad[1] += d[m] * (yp - ym);
              grad[2] += d[m] * (zp - zm);
            }
            cplx r = -0.5 * lap / h2 + v * psi0;
            if (s->gauge == 2)
              r += -I * (A[0] * grad[0] + A[1] * grad[1] + A[2] * grad[2]) / h;
            out[((long)k * N + p) * B + o] = r;
          }
        }

  /* non-local part: gather <beta_aj|psi>, then scatter beta_aj D_aj <beta_aj|psi> */
  if (s->n_atoms <= 0 || s->D == NULL) return;
  for (int a = 0; a < s->n_atoms; a++) {
    sphere_pt *pts;
    int np = sphere_points(s, a, &pts);
    for (int k = 0; k < s->n_k; k++) {
      const double *kk = s->kpts + 3 * k;
      cplx *proj = (cplx *)calloc((size_t)4 * B, sizeof(cplx));
      for (int q = 0; q < np; q++) {
        double b[4];
        beta_values(s, pts[q].d, b);
        double ph = 0.0;
        for (int ax = 0; ax < 3; ax++) ph += kk[ax] * pts[q].T[ax] + A[ax] * pts[q].d[ax];
        cplx phase = (s->bc == 1 || s->gauge == 2) ? cexp(I * ph) : 1.0;
        for (int j = 0; j < 4; j++)
          for (int o = 0; o < B; o++)
            proj[j * B + o] += h3 * b[j] * phase * in[((long)k * N + pts[q].cell) * B + o];
      }
      for (int q = 0; q < np; q++) {
        double b[4];
        beta_values(s, pts[q].d, b);
        double ph = 0.0;
        for (int ax = 0; ax < 3; ax++) ph += kk[ax] * pts[q].T[ax] + A[ax] * pts[q].d[ax];
        cplx phase = (s->bc == 1 || s->gauge == 2) ? cexp(-I * ph) : 1.0;
        for (int j = 0; j < 4; j++)
          for (int o = 0; o < B; o++)
            out[((long)k * N + pts[q].cell) * B + o] += b[j] * phase * s->D[4 * a + j] * proj[j * B + o];
      }
      free(proj);
    }
    free(pts);
  }
}

/* --------------------------------------------------------------------------------
 * One Taylor (sub-)step t -> t + dt with H frozen: density and v_x from psi(t), field at
 * the midpoint t + dt/2;  t_0 = psi,  t_k = (-i dt / k) H t_(k-1),  psi <- sum_(k=0..4) t_k.
 * ------------------------------------------------------------------------------ */
void oracle_taylor_substep(const oracle_sys *s, double t, double dt, cplx *psi) {
  long tot = (long)s->n_k * npts(s) * s->n_orb;
  double *n = NULL, *vx = NULL;
  if (has_density_potential(s)) {
    n = (double *)malloc(sizeof(double) * (size_t)npts(s));
    vx = (double *)malloc(sizeof(double) * (size_t)npts(s));
    oracle_density(s, psi, n);
    density_potential(s, n, vx, NULL);
  }
  cplx *term = (cplx *)malloc(sizeof(cplx) * (size_t)tot);
  cplx *next = (cplx *)malloc(sizeof(cplx) * (size_t)tot);
  cplx *acc = (cplx *)malloc(sizeof(cplx) * (size_t)tot);
  memcpy(term, psi, sizeof(cplx) * (size_t)tot);
  memcpy(acc, psi, sizeof(cplx) * (size_t)tot);
  for (int k = 1; k <= 4; k++) {
    oracle_apply_H(s, t + 0.5 * dt, vx, term, next);
    cplx coef = -I * dt / (double)k;
    for (long i = 0; i < tot; i++) {
      term[i] = coef * next[i];
      acc[i] += term[i];
    }
  }
  memcpy(psi, acc, sizeof(cplx) * (size_t)tot);
  free(term); free(next); free(acc); free(n); free(vx);
}

/* The projectors' part of sum_k w_k f <phi| i[V_NL, r] |phi> h^3 per axis, added to acc:
 * per atom, k-point and orbital, p_j = <b_j|phi> and q_jx = <d_x b_j|phi> (sphere points
 * unwrapped, r - R_a = d, with the Bloch and gauge phases), and
 * <phi| i[V_NL, r_x] |phi> = sum_j D_j i (p_j^* q_jx - q_jx^* p_j)  (the atom's position cancels). */
static void nonlocal_velocity(const oracle_sys *s, const double *A, const cplx *psi, ksum *acc) {
  if (s->n_atoms <= 0 || s->D == NULL) return;
  const long N = npts(s);
  const int B = s->n_orb;
  const double h3 = s->h * s->h * s->h;
  for (int a = 0; a < s->n_atoms; a++) {
    sphere_pt *pts;
    const int np = sphere_points(s, a, &pts);
    for (int k = 0; k < s->n_k; k++) {
      const double *kk = s->kpts + 3 * k;
      for (int o = 0; o < B; o++) {
        cplx p[4] = {0.0, 0.0, 0.0, 0.0}, q[4][3];
        for (int j = 0; j < 4; j++) q[j][0] = q[j][1] = q[j][2] = 0.0;
        for (int t = 0; t < np; t++) {
          double b[4];
          beta_values(s, pts[t].d, b);
          double ph = 0.0;
          for (int ax = 0; ax < 3; ax++) ph += kk[ax] * pts[t].T[ax] + A[ax] * pts[t].d[ax];
          const cplx val = h3 * cexp(I * ph) * psi[((long)k * N + pts[t].cell) * B + o];
          for (int j = 0; j < 4; j++) {
            p[j] += b[j] * val;
            for (int ax = 0; ax < 3; ax++) q[j][ax] += pts[t].d[ax] * b[j] * val;
          }
        }
        for (int j = 0; j < 4; j++)
          for (int ax = 0; ax < 3; ax++) {
            const cplx c = I * (conj(p[j]) * q[j][ax] - conj(q[j][ax]) * p[j]);
            kadd(&acc[ax], s->kw[k] * s->occ * s->D[4 * a + j] * creal(c));
          }
      }
    }
    free(pts);
  }
}

/* --------------------------------------------------------------------------------
 * Observables of the state psi (recorded at state time t_state) with the field of the
 * Hamiltonian taken at t_field.  obs = [t_state, norm, E, E_x, o_x, o_y, o_z, f] with
 *   norm = sum_k w_k sum_i ||phi_ik||^2 h^3,
 *   E    = sum_k w_k f_i <phi|H(t_field)|phi> - int n v_x + E_x,
 *          with Hartree (xc 2): v_x -> v_x + v_H and + E_H,
 *   o    = dipole int r n (finite systems) or the current
 *          J = -(1/Omega) sum_k w_k f_i <phi| i[H, r] |phi> (periodic cells): the local part
 *          <phi|(-i grad_h + A)|phi> and the projectors' commutator <phi| i[V_NL, r] |phi>,
 *   f    = field component along pol at t_field (E in length gauge, A in velocity gauge).
 * ------------------------------------------------------------------------------ */
void oracle_observables(const oracle_sys *s, double t_state, double t_field, const cplx *psi,
                        double *obs) {
  long N = npts(s), tot = (long)s->n_k * N * s->n_orb;
  int B = s->n_orb, M = s->fd_order / 2;
  double h = s->h, h3 = h * h * h;
  double *n = (double *)malloc(sizeof(double) * (size_t)N);
  double *vx = (double *)malloc(sizeof(double) * (size_t)N);
  oracle_density(s, psi, n);
  double ex = 0.0, eh = 0.0;
  ksum nvx = {0.0, 0.0};
  if (has_density_potential(s)) {
    ex = density_potential(s, n, vx, &eh);
    for (long p = 0; p < N; p++) kadd(&nvx, n[p] * vx[p] * h3);
  }
  cplx *hp = (cplx *)malloc(sizeof(cplx) * (size_t)tot);
  oracle_apply_H(s, t_field, has_density_potential(s) ? vx : NULL, psi, hp);
  ksum norm = {0.0, 0.0}, eband = {0.0, 0.0};
  for (int k = 0; k < s->n_k; k++)
    for (long p = 0; p < N; p++)
      for (int o = 0; o < B; o++) {
        long i = ((long)k * N + p) * B + o;
        kadd(&norm, s->kw[k] * creal(conj(psi[i]) * psi[i]) * h3);
        kadd(&eband, s->kw[k] * s->occ * creal(conj(psi[i]) * hp[i]) * h3);
      }
  double E[3], A[3];
  oracle_field(s, t_field, E, A);
  double o3[3] = {0.0, 0.0, 0.0};
  if (s->bc == 0) {
    ksum dip[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    for (int iz = 0; iz < s->nz; iz++)
      for (int iy = 0; iy < s->ny; iy++)
        for (int ix = 0; ix < s->nx; ix++) {
          long p = ((long)iz * s->ny + iy) * s->nx + ix;
          kadd(&dip[0], coord(s, 0, ix) * n[p] * h3);
          kadd(&dip[1], coord(s, 1, iy) * n[p] * h3);
          kadd(&dip[2], coord(s, 2, iz) * n[p] * h3);
        }
    for (int ax = 0; ax < 3; ax++) o3[ax] = dip[ax].s;
  } else {
    double d[5];
    oracle_fd_gradient_weights(M, d);
    double omega_cell = (double)s->nx * s->ny * s->nz * h3;
    ksum pexp[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}}, nel = {0.0, 0.0};
    for (int k = 0; k < s->n_k; k++)
      for (int iz = 0; iz < s->nz; iz++)
        for (int iy = 0; iy < s->ny; iy++)
          for (int ix = 0; ix < s->nx; ix++)
            for (int o = 0; o < B; o++) {
              long p = ((long)iz * s->ny + iy) * s->nx + ix;
              cplx v = psi[((long)k * N + p) * B + o];
              cplx g[3] = {0.0, 0.0, 0.0};
              for (int m = 1; m <= M; m++) {
                g[0] += d[m] * (fetch(s, psi, k, o, ix + m, iy, iz) - fetch(s, psi, k, o, ix - m, iy, iz));
                g[1] += d[m] * (fetch(s, psi, k, o, ix, iy + m, iz) - fetch(s, psi, k, o, ix, iy - m, iz));
                g[2] += d[m] * (fetch(s, psi, k, o, ix, iy, iz + m) - fetch(s, psi, k, o, ix, iy, iz - m));
              }
              for (int ax = 0; ax < 3; ax++)
                kadd(&pexp[ax], s->kw[k] * s->occ * creal(conj(v) * (-I) * g[ax] / h) * h3);
              kadd(&nel, s->kw[k] * s->occ * creal(conj(v) * v) * h3);
            }
    nonlocal_velocity(s, A, psi, pexp);
    for (int ax = 0; ax < 3; ax++) o3[ax] = -(pexp[ax].s + A[ax] * nel.s) / omega_cell;
  }
  obs[0] = t_state;
  obs[1] = norm.s;
  obs[2] = eband.s - nvx.s + ex + eh;
  obs[3] = ex;
  obs[4] = o3[0];
  obs[5] = o3[1];
  obs[6] = o3[2];
  obs[7] = (s->gauge == 2 ? A[0] * s->pol[0] + A[1] * s->pol[1] + A[2] * s->pol[2]
                          : E[0] * s->pol[0] + E[1] * s->pol[1] + E[2] * s->pol[2]);
  free(n); free(vx); free(hp);
}

/* --------------------------------------------------------------------------------
 * n_steps configured steps of length dt, each split into `substeps` equal Taylor
 * sub-steps.  Record s holds the observables of psi(t0 + s dt), the state at the start
 * of step s, with the field of the step's first sub-step (its midpoint).
 * ------------------------------------------------------------------------------ */
void oracle_propagate(const oracle_sys *s, double t0, double dt, int n_steps, int substeps,
                      cplx *psi, double *obs) {
  double dts = dt / (double)substeps;
  for (int st = 0; st < n_steps; st++) {
    double t = t0 + (double)st * dt;
    if (obs) oracle_observables(s, t, t + 0.5 * dts, psi, obs + 8 * st);
    for (int j = 0; j < substeps; j++) oracle_taylor_substep(s, t + (double)j * dts, dts, psi);
  }
}

/* --------------------------------------------------------------------------------
 * CFM4 (Sec. "New propagators for real-time TDDFT": the order-four commutator-free Magnus
 * expansion with two exponentials),
 *   phi(t + ds) = exp(-i ds (a1 H[t1] + a2 H[t2])) exp(-i ds (a2 H[t1] + a1 H[t2])) phi(t),
 *   a1 = (3 - 2 sqrt3)/12, a2 = (3 + 2 sqrt3)/12, t1,2 = t + (1/2 -+ sqrt3/6) ds.
 * In the length gauge H[t] = H0 + v_x(t) + E(t).r, and a1 + a2 = 1/2, so each exponential is
 * exp(-i (ds/2) H_eff) with H_eff = H0 + v_eff + E_eff.r:
 *   first  (applied first):  E_eff = 2 (a2 E(t1) + a1 E(t2)),  v_eff = 2 (a2 v_x(t1) + a1 v_x(t2)),
 *   second:                  E_eff = 2 (a1 E(t1) + a2 E(t2)),  v_eff = 2 (a1 v_x(t1) + a2 v_x(t2)).
 * v_x at t1, t2 is not known (it depends on the states); as the paper does for the
 * exchange-correlation part, it is extrapolated from earlier sub-steps: the Lagrange
 * polynomial through v_x at the starts of the last nh <= 4 sub-steps (offsets 0, -1, -2, -3
 * in units of ds; order four with four points).  Each exponential is applied with the
 * Taylor-4 series of this file.
 * ------------------------------------------------------------------------------ */
/* Lagrange weights of the nh history points at offsets 0, -1, .., -(nh-1), evaluated at x. */
static void lagrange_weights(int nh, double x, double *L) {
  for (int j = 0; j < nh; j++) {
    double w = 1.0;
    for (int i = 0; i < nh; i++)
      if (i != j) w *= (x - (double)(-i)) / ((double)(-j) - (double)(-i));
    L[j] = w;
  }
}

/* CFM4 constants: a[0] = a1, a[1] = a2, theta[0,1] = offsets of t1, t2 in units of ds. */
void oracle_cfm4_constants(double *a, double *theta) {
  const double r3 = sqrt(3.0);
  a[0] = (3.0 - 2.0 * r3) / 12.0;
  a[1] = (3.0 + 2.0 * r3) / 12.0;
  theta[0] = 0.5 - r3 / 6.0;
  theta[1] = 0.5 + r3 / 6.0;
}

/* Weights of the history v_x[j] (j = 0 the newest) in the effective potentials of the first
 * (wf) and second (ws) exponential. */
void oracle_cfm4_weights(int nh, double *wf, double *ws) {
  double a[2], th[2], L1[4], L2[4];
  oracle_cfm4_constants(a, th);
  lagrange_weights(nh, th[0], L1);
  lagrange_weights(nh, th[1], L2);
  for (int j = 0; j < nh; j++) {
    wf[j] = 2.0 * (a[1] * L1[j] + a[0] * L2[j]);
    ws[j] = 2.0 * (a[0] * L1[j] + a[1] * L2[j]);
  }
}

/* psi <- sum_(k=0..4) (-i tau H)^k / k! psi with H = H0 + v + E.r (v may be NULL). */
static void taylor_exp_field(const oracle_sys *s, const double *E, const double *v, double tau, cplx *psi) {
  long tot = (long)s->n_k * npts(s) * s->n_orb;
  const double A0[3] = {0.0, 0.0, 0.0};
  cplx *term = (cplx *)malloc(sizeof(cplx) * (size_t)tot);
  cplx *next = (cplx *)malloc(sizeof(cplx) * (size_t)tot);
  cplx *acc = (cplx *)malloc(sizeof(cplx) * (size_t)tot);
  memcpy(term, psi, sizeof(cplx) * (size_t)tot);
  memcpy(acc, psi, sizeof(cplx) * (size_t)tot);
  for (int k = 1; k <= 4; k++) {
    apply_H_field(s, E, A0, v, term, next);
    cplx coef = -I * tau / (double)k;
    for (long i = 0; i < tot; i++) {
      term[i] = coef * next[i];
      acc[i] += term[i];
    }
  }
  memcpy(psi, acc, sizeof(cplx) * (size_t)tot);
  free(term); free(next); free(acc);
}

/* n_steps configured steps of CFM4, each split into `substeps` equal CFM4 sub-steps ds; the
 * v_x history starts empty at t0.  Records as oracle_propagate (state at the start of each
 * step, Hamiltonian of t + ds/2 with v_x of that state).  Length gauge or no field only. */
void oracle_propagate_cfm4(const oracle_sys *s, double t0, double dt, int n_steps, int substeps, cplx *psi,
                           double *obs) {
  if (s->gauge == 2) return;  /* the effective-Hamiltonian form needs a field linear in H */
  const long N = npts(s);
  const double ds = dt / (double)substeps;
  double a[2], th[2];
  oracle_cfm4_constants(a, th);
  double *hist[4] = {NULL, NULL, NULL, NULL};
  int nh = 0;
  double *n = (double *)malloc(sizeof(double) * (size_t)N);
  double *vf = (double *)malloc(sizeof(double) * (size_t)N);
  double *vs = (double *)malloc(sizeof(double) * (size_t)N);
  for (int j = 0; j < 4; j++) hist[j] = (double *)malloc(sizeof(double) * (size_t)N);
  for (int st = 0; st < n_steps; st++) {
    double t = t0 + (double)st * dt;
    if (obs) oracle_observables(s, t, t + 0.5 * ds, psi, obs + 8 * st);
    for (int j = 0; j < substeps; j++) {
      const double tj = t + (double)j * ds;
      const double *pf = NULL, *ps = NULL;
      if (has_density_potential(s)) {
        /* push v_x (and v_H) of the current state as the newest history entry */
        double *oldest = hist[3];
        for (int q = 3; q > 0; q--) hist[q] = hist[q - 1];
        hist[0] = oldest;
        oracle_density(s, psi, n);
        density_potential(s, n, hist[0], NULL);
        if (nh < 4) nh++;
        double wf[4], wsw[4];
        oracle_cfm4_weights(nh, wf, wsw);
        for (long p = 0; p < N; p++) {
          double x = 0.0, y = 0.0;
          for (int q = 0; q < nh; q++) {
            x += wf[q] * hist[q][p];
            y += wsw[q] * hist[q][p];
          }
          vf[p] = x;
          vs[p] = y;
        }
        pf = vf;
        ps = vs;
      }
      double E1[3], E2[3], A[3], Ef[3], Es[3];
      oracle_field(s, tj + th[0] * ds, E1, A);
      oracle_field(s, tj + th[1] * ds, E2, A);
      for (int ax = 0; ax < 3; ax++) {
        Ef[ax] = 2.0 * (a[1] * E1[ax] + a[0] * E2[ax]);
        Es[ax] = 2.0 * (a[0] * E1[ax] + a[1] * E2[ax]);
      }
      taylor_exp_field(s, Ef, pf, 0.5 * ds, psi);
      taylor_exp_field(s, Es, ps, 0.5 * ds, psi);
    }
  }
  for (int j = 0; j < 4; j++) free(hist[j]);
  free(n); free(vf); free(vs);
}

/* --------------------------------------------------------------------------------
 * Exponential midpoint rule and approximate enforced time-reversal symmetry.  The paper
 * lists both among the propagators in use (Sec. "New propagators for real-time TDDFT"; the
 * time-reversal scheme also in the hydrogen-fluoride dimer run of Sec. "vdW-TS" and in the
 * first GPU port of Sec. "GPUs") without writing them out.  Their usual forms, per sub-step ds:
 *   EMR:   phi(t + ds) = exp(-i ds H[t + ds/2]) phi(t)
 *   AETRS: phi(t + ds) = exp(-i ds/2 H[t + ds]) exp(-i ds/2 H[t]) phi(t)
 * with H[t] = H0 + v_x(t) + E(t).r.  v_x(t) is that of the current state; v_x at t + ds/2
 * and t + ds is not known, and, as for CFM4, it is extrapolated from the values at the
 * starts of the last nh <= 4 sub-steps (Lagrange, offsets 0, -1, .., -(nh-1)).  Each
 * exponential is the Taylor-4 series.  Records and history as oracle_propagate_cfm4.
 * ------------------------------------------------------------------------------ */

/* Push v_x of psi into the history (hist[0] the newest) and return the new count. */
static int push_vx(const oracle_sys *s, const cplx *psi, double **hist, int nh, double *n) {
  double *oldest = hist[3];
  for (int q = 3; q > 0; q--) hist[q] = hist[q - 1];
  hist[0] = oldest;
  oracle_density(s, psi, n);
  density_potential(s, n, hist[0], NULL);
  return nh < 4 ? nh + 1 : 4;
}

/* v(p) = sum_j L_j(x) hist[j][p]: the history extrapolated to offset x (in sub-steps). */
static void extrapolate_vx(const oracle_sys *s, double **hist, int nh, double x, double *v) {
  double L[4];
  lagrange_weights(nh, x, L);
  for (long p = 0; p < npts(s); p++) {
    double acc = 0.0;
    for (int j = 0; j < nh; j++) acc += L[j] * hist[j][p];
    v[p] = acc;
  }
}

static void propagate_two_point(const oracle_sys *s, int aetrs, double t0, double dt, int n_steps, int substeps,
                                cplx *psi, double *obs) {
  if (s->gauge == 2) return;  /* the field must enter H linearly */
  const long N = npts(s);
  const double ds = dt / (double)substeps;
  double *hist[4];
  int nh = 0;
  double *n = (double *)malloc(sizeof(double) * (size_t)N);
  double *v = (double *)malloc(sizeof(double) * (size_t)N);
  for (int j = 0; j < 4; j++) hist[j] = (double *)malloc(sizeof(double) * (size_t)N);
  for (int st = 0; st < n_steps; st++) {
    double t = t0 + (double)st * dt;
    if (obs) oracle_observables(s, t, t + 0.5 * ds, psi, obs + 8 * st);
    for (int j = 0; j < substeps; j++) {
      const double tj = t + (double)j * ds;
      double E[3], A[3];
      if (has_density_potential(s)) nh = push_vx(s, psi, hist, nh, n);
      if (!aetrs) {
        if (has_density_potential(s)) extrapolate_vx(s, hist, nh, 0.5, v);
        oracle_field(s, tj + 0.5 * ds, E, A);
        taylor_exp_field(s, E, has_density_potential(s) ? v : NULL, ds, psi);
      } else {
        oracle_field(s, tj, E, A);
        taylor_exp_field(s, E, has_density_potential(s) ? hist[0] : NULL, 0.5 * ds, psi);
        if (has_density_potential(s)) extrapolate_vx(s, hist, nh, 1.0, v);
        oracle_field(s, tj + ds, E, A);
        taylor_exp_field(s, E, has_density_potential(s) ? v : NULL, 0.5 * ds, psi);
      }
    }
  }
  for (int j = 0; j < 4; j++) free(hist[j]);
  free(n); free(v);
}

/* --------------------------------------------------------------------------------
 * Enforced time-reversal symmetry with its trial state (the scheme of the propagator review
 * the paper cites in Sec. "New propagators for real-time TDDFT"; used in the hydrogen-fluoride
 * dimer run of Sec. "vdW-TS" and the first GPU port of Sec. "GPUs").  Per sub-step ds:
 *   trial:  phi~ = exp(-i ds H[t]) phi(t)                     (H[t] frozen over the step)
 *   step:   phi(t + ds) = exp(-i ds/2 H[t + ds]) exp(-i ds/2 H[t]) phi(t)
 * with H[t] = H0 + v_x(n(phi(t))) + E(t).r and H[t + ds] = H0 + v_x(n(phi~)) + E(t + ds).r.
 * Each exponential is the Taylor-4 series.  Without a density-dependent potential the trial
 * changes nothing and the step is the AETRS step.  Records as oracle_propagate.
 * ------------------------------------------------------------------------------ */
void oracle_propagate_etrs(const oracle_sys *s, double t0, double dt, int n_steps, int substeps, cplx *psi,
                           double *obs) {
  if (s->gauge == 2) return;  /* the field must enter H linearly */
  const long N = npts(s);
  const long tot = (long)s->n_k * N * s->n_orb;
  const double ds = dt / (double)substeps;
  const int dp = has_density_potential(s);
  double *n = (double *)malloc(sizeof(double) * (size_t)N);
  double *v_t = (double *)malloc(sizeof(double) * (size_t)N);
  double *v_next = (double *)malloc(sizeof(double) * (size_t)N);
  cplx *trial = (cplx *)malloc(sizeof(cplx) * (size_t)tot);
  for (int st = 0; st < n_steps; st++) {
    double t = t0 + (double)st * dt;
    if (obs) oracle_observables(s, t, t + 0.5 * ds, psi, obs + 8 * st);
    for (int j = 0; j < substeps; j++) {
      const double tj = t + (double)j * ds;
      double E[3], A[3];
      oracle_field(s, tj, E, A);
      if (dp) {
        oracle_density(s, psi, n);
        density_potential(s, n, v_t, NULL);
        memcpy(trial, psi, sizeof(cplx) * (size_t)tot);
        taylor_exp_field(s, E, v_t, ds, trial);
        oracle_density(s, trial, n);
        density_potential(s, n, v_next, NULL);
      }
      taylor_exp_field(s, E, dp ? v_t : NULL, 0.5 * ds, psi);
      oracle_field(s, tj + ds, E, A);
      taylor_exp_field(s, E, dp ? v_next : NULL, 0.5 * ds, psi);
    }
  }
  free(n); free(v_t); free(v_next); free(trial);
}

void oracle_propagate_emr(const oracle_sys *s, double t0, double dt, int n_steps, int substeps, cplx *psi,
                          double *obs) {
  propagate_two_point(s, 0, t0, dt, n_steps, substeps, psi, obs);
}

void oracle_propagate_aetrs(const oracle_sys *s, double t0, double dt, int n_steps, int substeps, cplx *psi,
                            double *obs) {
  propagate_two_point(s, 1, t0, dt, n_steps, substeps, psi, obs);
}

/* --------------------------------------------------------------------------------
 * Classical fourth-order Runge-Kutta on the TDKS system d phi/dt = -i H[n(phi), t] phi
 * (Sec. "New propagators for real-time TDDFT" lists Runge-Kutta among the propagators in
 * use).  Per sub-step ds, with every stage's Hamiltonian built from that stage's own density:
 *   k1 = -i H[n(phi), t] phi,                      k2 = -i H[n(p2), t + ds/2] p2, p2 = phi + ds/2 k1,
 *   k3 = -i H[n(p3), t + ds/2] p3, p3 = phi + ds/2 k2,  k4 = -i H[n(p4), t + ds] p4, p4 = phi + ds k3,
 *   phi(t + ds) = phi + ds/6 (k1 + 2 k2 + 2 k3 + k4).
 * Records as oracle_propagate.
 * ------------------------------------------------------------------------------ */
/* k = -i H[n(v), t] v */
static void rk4_slope(const oracle_sys *s, double t, const cplx *v, double *n, double *vx, cplx *k) {
  const long tot = (long)s->n_k * npts(s) * s->n_orb;
  double E[3], A[3];
  oracle_field(s, t, E, A);
  if (has_density_potential(s)) {
    oracle_density(s, v, n);
    density_potential(s, n, vx, NULL);
  }
  apply_H_field(s, E, A, has_density_potential(s) ? vx : NULL, v, k);
  for (long i = 0; i < tot; i++) k[i] *= -I;
}

void oracle_propagate_rk4(const oracle_sys *s, double t0, double dt, int n_steps, int substeps, cplx *psi,
                          double *obs) {
  const long N = npts(s), tot = (long)s->n_k * N * s->n_orb;
  const double ds = dt / (double)substeps;
  double *n = (double *)malloc(sizeof(double) * (size_t)N);
  double *vx = (double *)malloc(sizeof(double) * (size_t)N);
  cplx *k = (cplx *)malloc(sizeof(cplx) * (size_t)tot);
  cplx *stage = (cplx *)malloc(sizeof(cplx) * (size_t)tot);
  cplx *sum = (cplx *)malloc(sizeof(cplx) * (size_t)tot);
  for (int st = 0; st < n_steps; st++) {
    double t = t0 + (double)st * dt;
    if (obs) oracle_observables(s, t, t + 0.5 * ds, psi, obs + 8 * st);
    for (int j = 0; j < substeps; j++) {
      const double tj = t + (double)j * ds;
      rk4_slope(s, tj, psi, n, vx, k);
      for (long i = 0; i < tot; i++) {
        sum[i] = k[i];
        stage[i] = psi[i] + 0.5 * ds * k[i];
      }
      rk4_slope(s, tj + 0.5 * ds, stage, n, vx, k);
      for (long i = 0; i < tot; i++) {
        sum[i] += 2.0 * k[i];
        stage[i] = psi[i] + 0.5 * ds * k[i];
      }
      rk4_slope(s, tj + 0.5 * ds, stage, n, vx, k);
      for (long i = 0; i < tot; i++) {
        sum[i] += 2.0 * k[i];
        stage[i] = psi[i] + ds * k[i];
      }
      rk4_slope(s, tj + ds, stage, n, vx, k);
      for (long i = 0; i < tot; i++) psi[i] += ds / 6.0 * (sum[i] + k[i]);
    }
  }
  free(n); free(vx); free(k); free(stage); free(sum);
}

/* --------------------------------------------------------------------------------
 * Hartree potential v_H(r) = int n(r') / |r - r'| dr' (atomic units), with the energy
 * E_H = 1/2 int n v_H.  The paper's TDDFT Hamiltonian carries the Hartree term among the
 * density-dependent potentials it extrapolates for CFM4 (Sec. "New propagators for
 * real-time TDDFT"); the propagation path built here takes exchange only, and these
 * functions are the definition a Hartree kernel is checked against.
 *
 * Finite box: the integral as a sum over grid cells, n taken constant over each cell:
 *   v_H(r_i) = h^3 sum_j n_j G(r_i - r_j),  G(d) = 1/|d| for d != 0,
 *   G(0) = (1/h^3) int over the cell centred at 0 of 1/|r| = c0 / h,
 *   c0 = int over the unit cube [-1/2, 1/2]^3 of 1/|r| = 3 ln(2 + sqrt 3) - pi/2
 * (the cell's own contribution; the other cells by their centre value).
 * Periodic cell: the Poisson equation -Lap v_H = 4 pi (n - <n>) solved exactly on the
 * grid's plane waves, v_H = sum_(G != 0) 4 pi n(G) / |G|^2 e^(i G.r), with the neutralising
 * background removing G = 0 and each G the shortest of its aliases.
 * Returns E_H = 1/2 h^3 sum_i n_i v_H(r_i).
 * ------------------------------------------------------------------------------ */
double oracle_hartree_self_cell(void) { return 3.0 * log(2.0 + sqrt(3.0)) - 0.5 * M_PI; }

/* wavenumber of index k on an n-point periodic axis of length L: the alias nearest zero */
static double grid_wavenumber(int k, int n, double L) {
  const int kk = (k <= n / 2) ? k : k - n;
  return 2.0 * M_PI * (double)kk / L;
}

double oracle_hartree(const oracle_sys *s, const double *n, double *vh) {
  const long N = npts(s);
  const double h = s->h, h3 = h * h * h;
  if (s->bc == 0) {
    const double g0 = oracle_hartree_self_cell() / h;
#pragma omp parallel for
    for (long i = 0; i < N; i++) {
      const int ix = (int)(i % s->nx), iy = (int)((i / s->nx) % s->ny), iz = (int)(i / ((long)s->nx * s->ny));
      double acc = 0.0;
      for (long j = 0; j < N; j++) {
        const int jx = (int)(j % s->nx), jy = (int)((j / s->nx) % s->ny), jz = (int)(j / ((long)s->nx * s->ny));
        const double dx = (ix - jx) * h, dy = (iy - jy) * h, dz = (iz - jz) * h;
        const double d = sqrt(dx * dx + dy * dy + dz * dz);
        acc += n[j] * (j == i ? g0 : 1.0 / d);
      }
      vh[i] = h3 * acc;
    }
  } else {
    /* plain discrete Fourier transform over all grid points (small cells only) */
    const double L[3] = {s->nx * h, s->ny * h, s->nz * h};
    const long NG = N;
    cplx *nG = (cplx *)malloc(sizeof(cplx) * (size_t)NG);
#pragma omp parallel for
    for (long g = 0; g < NG; g++) {
      const int kx = (int)(g % s->nx), ky = (int)((g / s->nx) % s->ny), kz = (int)(g / ((long)s->nx * s->ny));
      cplx acc = 0.0;
      for (long j = 0; j < N; j++) {
        const int jx = (int)(j % s->nx), jy = (int)((j / s->nx) % s->ny), jz = (int)(j / ((long)s->nx * s->ny));
        const double ph = 2.0 * M_PI * ((double)kx * jx / s->nx + (double)ky * jy / s->ny + (double)kz * jz / s->nz);
        acc += n[j] * cexp(-I * ph);
      }
      nG[g] = acc;
    }
#pragma omp parallel for
    for (long i = 0; i < N; i++) {
      const int ix = (int)(i % s->nx), iy = (int)((i / s->nx) % s->ny), iz = (int)(i / ((long)s->nx * s->ny));
      cplx acc = 0.0;
      for (long g = 1; g < NG; g++) { /* g = 0 is the background */
        const int kx = (int)(g % s->nx), ky = (int)((g / s->nx) % s->ny), kz = (int)(g / ((long)s->nx * s->ny));
        const double Gx = grid_wavenumber(kx, s->nx, L[0]), Gy = grid_wavenumber(ky, s->ny, L[1]),
                     Gz = grid_wavenumber(kz, s->nz, L[2]);
        const double G2 = Gx * Gx + Gy * Gy + Gz * Gz;
        const double ph = 2.0 * M_PI * ((double)kx * ix / s->nx + (double)ky * iy / s->ny + (double)kz * iz / s->nz);
        acc += 4.0 * M_PI / G2 * nG[g] * cexp(I * ph);
      }
      vh[i] = creal(acc) / (double)N;
    }
    free(nG);
  }
  ksum e = {0.0, 0.0};
  for (long i = 0; i < N; i++) kadd(&e, 0.5 * n[i] * vh[i] * h3);
  return e.s;
}

/* OpenMP runtime calls (libgomp, linked by -fopenmp) */
int omp_get_max_threads(void);
void omp_set_num_threads(int n);

/* Host threads of the oracle's parallel loops (for timing it on one core and on all);
 * returns the count in use before the call. */
int oracle_set_threads(int n) {
  const int old = omp_get_max_threads();
  if (n > 0) omp_set_num_threads(n);
  return old;
}

/* --------------------------------------------------------------------------------
 * Velocity expectation and band energy at an explicit vector potential (periodic cells,
 * velocity gauge).  The macroscopic current of Sec. "Conductivities" is
 * J = -(1/Omega) sum_k w_k f_i <phi| v |phi> with the velocity operator v = i[H, r]:
 *   local part     (-i grad_h + A),
 *   non-local part i[V_NL, r], with r inside a projector sphere the unwrapped position of
 *                  the sphere point (its atom's position cancels in the commutator):
 *                  <phi| i[V_NL, r] |phi> = sum_aj D_aj i (<phi|b_aj><b_aj| d phi> - <phi| d b_aj><b_aj|phi>)
 *                  with b_aj the dressed projector (Bloch and gauge phases) and d = r - R_a.
 * The observable record carries both parts; oracle_velocity_expectation returns
 * sum_k w_k f_i <phi|v|phi> h^3 per axis, with the non-local part when `nonlocal` is set.
 * oracle_band_energy returns sum_k w_k f_i <phi|H(A)|phi> h^3 (no exchange, no other field).
 * ------------------------------------------------------------------------------ */
double oracle_band_energy(const oracle_sys *s, const double *A, const cplx *psi) {
  const long N = npts(s), tot = (long)s->n_k * N * s->n_orb;
  const double h3 = s->h * s->h * s->h, E0[3] = {0.0, 0.0, 0.0};
  cplx *hp = (cplx *)malloc(sizeof(cplx) * (size_t)tot);
  apply_H_field(s, E0, A, NULL, psi, hp);
  ksum e = {0.0, 0.0};
  for (int k = 0; k < s->n_k; k++)
    for (long i = (long)k * N * s->n_orb; i < (long)(k + 1) * N * s->n_orb; i++)
      kadd(&e, s->kw[k] * s->occ * creal(conj(psi[i]) * hp[i]) * h3);
  free(hp);
  return e.s;
}

void oracle_velocity_expectation(const oracle_sys *s, const double *A, const cplx *psi, int nonlocal, double *out) {
  const long N = npts(s);
  const int M = s->fd_order / 2, B = s->n_orb;
  const double h = s->h, h3 = h * h * h;
  double d[5];
  oracle_fd_gradient_weights(M, d);
  ksum acc[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
  for (int k = 0; k < s->n_k; k++)
    for (int iz = 0; iz < s->nz; iz++)
      for (int iy = 0; iy < s->ny; iy++)
        for (int ix = 0; ix < s->nx; ix++)
          for (int o = 0; o < B; o++) {
            const cplx v = fetch(s, psi, k, o, ix, iy, iz);
            cplx g[3] = {0.0, 0.0, 0.0};
            for (int m = 1; m <= M; m++) {
              g[0] += d[m] * (fetch(s, psi, k, o, ix + m, iy, iz) - fetch(s, psi, k, o, ix - m, iy, iz));
              g[1] += d[m] * (fetch(s, psi, k, o, ix, iy + m, iz) - fetch(s, psi, k, o, ix, iy - m, iz));
              g[2] += d[m] * (fetch(s, psi, k, o, ix, iy, iz + m) - fetch(s, psi, k, o, ix, iy, iz - m));
            }
            for (int ax = 0; ax < 3; ax++)
              kadd(&acc[ax], s->kw[k] * s->occ * creal(conj(v) * (-I * g[ax] / h + A[ax] * v)) * h3);
          }
  if (nonlocal) nonlocal_velocity(s, A, psi, acc);
  for (int ax = 0; ax < 3; ax++) out[ax] = acc[ax].s;
}

/* --------------------------------------------------------------------------------
 * t-SURFF flux (Sec. "t-SURFF": the photoelectron amplitude b_i(p, t) as the time
 * integral of the current of the Volkov state chi_p and the orbital through a surface S
 * that separates the inner region from the outer one).
 *
 * Readings (the section prints the velocity-gauge forms; finite systems here couple the
 * field in the length gauge, +E(t).r):
 *   - S is the surface of a box of grid planes x = x_i0, x_i1, y = y_j0, y_j1, z = z_k0,
 *     z_k1 (the section leaves the shape of S free; planes of the grid need no
 *     interpolation).  Each face is integrated with the two-dimensional trapezoid rule over
 *     its grid points (weight h^2, halved on its edges, quartered at its corners) and
 *     carries the outward unit normal n.
 *   - Volkov states of the free length-gauge Hamiltonian -1/2 Lap + E(t).r:
 *       chi_p(r, t) = (2 pi)^(-3/2) exp(i k_p(t).r - i Phi_p(t)),  k_p(t) = p + a(t),
 *       a(t) = -int_0^t E,  Phi_p(t) = 1/2 int_0^t |k_p|^2 = 1/2 (|p|^2 t + 2 p.alpha(t) + beta(t)),
 *       alpha(t) = int_0^t a,  beta(t) = int_0^t |a|^2;
 *     (the printed phase lacks the 1/2 and has the opposite sign; only this form solves the
 *     Volkov equation), with times counted from the start of the accumulation.
 *   - the current matrix element is the length-gauge one (no vector-potential term):
 *       <chi_p| j |phi> = 1/2 (i phi grad chi_p^* - i chi_p^* grad phi) = 1/2 chi_p^* (k_p phi - i grad_h phi),
 *     with grad_h the central difference of order 2M (psi = 0 outside the box);
 *   - b_i(p, T) = int_0^T F_i(p, t) dt, F_i = oint_S n . <chi_p| j |phi_i> ds with the outward
 *     normal (the projection of phi_i on chi_p in the outer region, from the continuity
 *     equation; the printed minus sign belongs to the inward normal).
 * F_i(p) is returned as F[i * n_p + pidx]; one k-point (finite systems).
 * ------------------------------------------------------------------------------ */
void oracle_tsurff_flux(const oracle_sys *s, const int *box, int n_p, const double *p, const double *a,
                        const double *alpha, double beta, double t_rel, const cplx *psi, cplx *F) {
  const int M = s->fd_order / 2, B = s->n_orb;
  const double h = s->h;
  double d[5];
  oracle_fd_gradient_weights(M, d);
  const double pref = 0.5 * pow(2.0 * M_PI, -1.5);
  for (long i = 0; i < (long)B * n_p; i++) F[i] = 0.0;
  for (int face = 0; face < 6; face++) {
    const int ax = face / 2;                 /* normal axis */
    const double sgn = (face % 2) ? 1.0 : -1.0;
    const int c = box[2 * ax + (face % 2)];  /* the face's plane index along ax */
    const int ua = (ax + 1) % 3, va = (ax + 2) % 3;
    for (int u = box[2 * ua]; u <= box[2 * ua + 1]; u++)
      for (int v = box[2 * va]; v <= box[2 * va + 1]; v++) {
        double w = h * h;
        if (u == box[2 * ua] || u == box[2 * ua + 1]) w *= 0.5;
        if (v == box[2 * va] || v == box[2 * va + 1]) w *= 0.5;
        int ii[3];
        ii[ax] = c;
        ii[ua] = u;
        ii[va] = v;
        double r[3];
        for (int q = 0; q < 3; q++) r[q] = coord(s, q, ii[q]);
        for (int o = 0; o < B; o++) {
          const cplx phi = fetch(s, psi, 0, o, ii[0], ii[1], ii[2]);
          cplx g = 0.0;
          for (int m = 1; m <= M; m++) {
            int ip[3] = {ii[0], ii[1], ii[2]}, im[3] = {ii[0], ii[1], ii[2]};
            ip[ax] += m;
            im[ax] -= m;
            g += d[m] * (fetch(s, psi, 0, o, ip[0], ip[1], ip[2]) - fetch(s, psi, 0, o, im[0], im[1], im[2]));
          }
          g /= h;
          for (int q = 0; q < n_p; q++) {
            const double *pp = p + 3 * q;
            double kr = 0.0, phase = 0.5 * (pp[0] * pp[0] + pp[1] * pp[1] + pp[2] * pp[2]) * t_rel + 0.5 * beta;
            for (int x = 0; x < 3; x++) {
              kr += (pp[x] + a[x]) * r[x];
              phase += pp[x] * alpha[x];
            }
            const cplx chi_conj = cexp(I * (phase - kr));
            const double kn = pp[ax] + a[ax];
            F[(long)o * n_p + q] += w * sgn * pref * chi_conj * (kn * phi - I * g);
          }
        }
      }
  }
}

/* a(t), alpha(t), beta(t) advanced over one step dt by the classical Runge-Kutta method on
 * a' = -E(t), alpha' = a, beta' = |a|^2 (y = a[3], alpha[3], beta). */
static void volkov_rhs(const oracle_sys *s, double t, const double *y, double *f) {
  double E[3], A[3];
  oracle_field(s, t, E, A);
  for (int x = 0; x < 3; x++) {
    f[x] = s->gauge == 1 ? -E[x] : 0.0;
    f[3 + x] = y[x];
  }
  f[6] = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
}
void oracle_volkov_step(const oracle_sys *s, double t, double dt, double *y) {
  double k1[7], k2[7], k3[7], k4[7], tmp[7];
  volkov_rhs(s, t, y, k1);
  for (int i = 0; i < 7; i++) tmp[i] = y[i] + 0.5 * dt * k1[i];
  volkov_rhs(s, t + 0.5 * dt, tmp, k2);
  for (int i = 0; i < 7; i++) tmp[i] = y[i] + 0.5 * dt * k2[i];
  volkov_rhs(s, t + 0.5 * dt, tmp, k3);
  for (int i = 0; i < 7; i++) tmp[i] = y[i] + dt * k3[i];
  volkov_rhs(s, t + dt, tmp, k4);
  for (int i = 0; i < 7; i++) y[i] += dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* Taylor-4 propagation (as oracle_propagate) with the t-SURFF amplitudes accumulated by the
 * trapezoid rule in time over the configured steps: b += dt (F(t0)/2 + F(t1) + ... +
 * F(t_(n-1)) + F(t_n)/2), so that consecutive calls add up to one trapezoid sum.  vol
 * (a, alpha, beta) and t_rel (time since the accumulation started) are read and advanced. */
void oracle_tsurff_propagate(const oracle_sys *s, const int *box, int n_p, const double *p, double t0, double dt,
                             int n_steps, int substeps, cplx *psi, double *obs, double *vol, double *t_rel, cplx *b) {
  const int B = s->n_orb;
  cplx *F = (cplx *)malloc(sizeof(cplx) * (size_t)B * (size_t)n_p);
  const double dts = dt / (double)substeps;
  for (int st = 0; st <= n_steps; st++) {
    const double t = t0 + (double)st * dt;
    oracle_tsurff_flux(s, box, n_p, p, vol, vol + 3, vol[6], *t_rel, psi, F);
    const double w = (st == 0 || st == n_steps) ? 0.5 * dt : dt;
    for (long i = 0; i < (long)B * n_p; i++) b[i] += w * F[i];
    if (st == n_steps) break;
    if (obs) oracle_observables(s, t, t + 0.5 * dts, psi, obs + 8 * st);
    for (int j = 0; j < substeps; j++) oracle_taylor_substep(s, t + (double)j * dts, dts, psi);
    oracle_volkov_step(s, t, dt, vol);
    *t_rel += dt;
  }
  free(F);
}

/* --------------------------------------------------------------------------------
 * Kinetic heat current (Sec. "Conductivities", eqn. KEcurrent): the macroscopic (cell-averaged)
 *   J_t = (1/Omega) sum_k w_k f int [J_t(r)] dr,
 *   [J_t(r)]_i = (i/8) ( [d_i phi^*][Lap phi] - [Lap phi^*][d_i phi] - [d_i grad phi^*].[grad phi]
 *                        + [grad phi^*].[d_i grad phi] ).
 * Reading: the printed last pair has equal signs, which makes its (i/8) multiple imaginary; with
 * the pair antisymmetric, as the first one, J_t is real, and a plane wave gives
 * -(1/2)|k|^2 k: minus its kinetic energy times its velocity, the sign convention of the charge
 * current J of eqn. current_density (electron charge -1).  Derivatives as in H: covariant in the
 * velocity gauge, d_j -> d_j + i A_j with d_j the central difference of order 2M (Bloch images in a
 * periodic cell, zeros outside a box); Lap -> Lap_h + 2 i A.grad_h - |A|^2 with Lap_h the star
 * Laplacian; d_i grad phi -> the covariant first differences composed.  Plain loops, every
 * neighbour fetched.
 * ------------------------------------------------------------------------------ */
static void cov_grad(const oracle_sys *s, const double *d, const double *A, const cplx *psi, int k, int o, int ix,
                     int iy, int iz, cplx *g) {
  const int M = s->fd_order / 2;
  const cplx v = fetch(s, psi, k, o, ix, iy, iz);
  for (int j = 0; j < 3; j++) {
    cplx acc = 0.0;
    for (int m = 1; m <= M; m++) {
      int p[3] = {ix, iy, iz}, q[3] = {ix, iy, iz};
      p[j] += m;
      q[j] -= m;
      acc += d[m] * (fetch(s, psi, k, o, p[0], p[1], p[2]) - fetch(s, psi, k, o, q[0], q[1], q[2]));
    }
    g[j] = acc / s->h + I * A[j] * v;
  }
}

void oracle_heat_current(const oracle_sys *s, const double *A, const cplx *psi, double *out) {
  const int M = s->fd_order / 2, B = s->n_orb;
  const double h = s->h, h2 = h * h, h3 = h * h * h;
  double c[5], d[5];
  oracle_fd_laplacian_weights(M, c);
  oracle_fd_gradient_weights(M, d);
  const double A2 = A[0] * A[0] + A[1] * A[1] + A[2] * A[2];
  const double omega_cell = (double)s->nx * s->ny * s->nz * h3;
  ksum acc[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
  for (int k = 0; k < s->n_k; k++)
    for (int iz = 0; iz < s->nz; iz++)
      for (int iy = 0; iy < s->ny; iy++)
        for (int ix = 0; ix < s->nx; ix++)
          for (int o = 0; o < B; o++) {
            const cplx v = fetch(s, psi, k, o, ix, iy, iz);
            cplx g[3];
            cov_grad(s, d, A, psi, k, o, ix, iy, iz, g);
            /* covariant Laplacian: the star Laplacian, 2 i A.grad_h, -|A|^2 */
            cplx lap = 3.0 * c[0] * v, adg = 0.0;
            for (int j = 0; j < 3; j++)
              for (int m = 1; m <= M; m++) {
                int p[3] = {ix, iy, iz}, q[3] = {ix, iy, iz};
                p[j] += m;
                q[j] -= m;
                const cplx a = fetch(s, psi, k, o, p[0], p[1], p[2]), b = fetch(s, psi, k, o, q[0], q[1], q[2]);
                lap += c[m] * (a + b);
                adg += A[j] * d[m] * (a - b);
              }
            lap = lap / h2 + 2.0 * I * adg / h - A2 * v;
            /* G[i][j] = (d_i + i A_i)(d_j + i A_j) phi: the covariant gradient at the neighbours along i */
            cplx G[3][3];
            for (int i = 0; i < 3; i++) {
              cplx gi[3] = {0.0, 0.0, 0.0};
              for (int m = 1; m <= M; m++) {
                int p[3] = {ix, iy, iz}, q[3] = {ix, iy, iz};
                p[i] += m;
                q[i] -= m;
                cplx gp[3], gq[3];
                cov_grad(s, d, A, psi, k, o, p[0], p[1], p[2], gp);
                cov_grad(s, d, A, psi, k, o, q[0], q[1], q[2], gq);
                for (int j = 0; j < 3; j++) gi[j] += d[m] * (gp[j] - gq[j]);
              }
              for (int j = 0; j < 3; j++) G[i][j] = gi[j] / h + I * A[i] * g[j];
            }
            for (int i = 0; i < 3; i++) {
              const cplx t1 = conj(g[i]) * lap, t2 = conj(lap) * g[i];
              cplx t3 = 0.0, t4 = 0.0;
              for (int j = 0; j < 3; j++) {
                t3 += conj(G[i][j]) * g[j];
                t4 += conj(g[j]) * G[i][j];
              }
              const cplx jt = (I / 8.0) * (t1 - t2 - t3 + t4);
              kadd(&acc[i], s->kw[k] * s->occ * creal(jt) * h3);
            }
          }
  for (int i = 0; i < 3; i++) out[i] = acc[i].s / omega_cell;
}
