// t-SURFF photoelectron amplitudes (Sec. "t-SURFF"): the amplitude of orbital i on the
// Volkov state of momentum p is the time integral of the current of chi_p and phi_i through
// a surface S between the inner region and the outer one,
//   b_i(p, T) = int_0^T dt oint_S ds n . <chi_p| j |phi_i>,
//   <chi_p| j |phi> = 1/2 chi_p^* (k_p phi - i grad_h phi)   (length gauge),
//   chi_p(r, t) = (2 pi)^(-3/2) exp(i k_p(t).r - i Phi_p(t)),  k_p = p + a(t),  a = -int E,
//   Phi_p = 1/2 (|p|^2 t + 2 p.alpha + beta),  alpha = int a,  beta = int |a|^2,
// with S the surface of a box of grid planes (each face by the two-dimensional trapezoid rule,
// outward normal), the gradient the central difference of order 2M, and the time integral
// the trapezoid rule over the configured steps.  The section notes that the method only
// needs the gradient on the surface points: per step a gather kernel forms, at every surface
// entry and orbital, w n.(phi, -i grad_h phi), and a flux kernel contracts them with the
// Volkov factors of every momentum.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "tdks_system.h"

using namespace tdks;
using namespace tdks_host;

namespace {

struct TsGather {
  int prec, BS, n_orb, ax_unused;
  long N;
  long stride[3];          // point strides along x, y, z
  const void *psi, *psi_lo;
  const TsEntry *ent;
  int n_e, M;
  double d[MAXM + 1];      // gradient weights over h
  double2 *G0, *G1;        // [n_e][n_orb]
};

// value of orbital o at point pt, in FP64 (complex64 systems: hi + lo of the state)
__device__ __forceinline__ double2 ts_value(const TsGather &g, int o, long pt) {
  const long i = ((long)(o / g.BS) * g.N + pt) * g.BS + (o % g.BS);
  if (g.prec == P_C128) return reinterpret_cast<const double2 *>(g.psi)[i];
  const float2 hi = reinterpret_cast<const float2 *>(g.psi)[i], lo = reinterpret_cast<const float2 *>(g.psi_lo)[i];
  return make_double2((double)hi.x + (double)lo.x, (double)hi.y + (double)lo.y);
}

__global__ void tsurff_gather_kernel(const TsGather g) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)g.n_e * g.n_orb) return;
  const int e = (int)(t / g.n_orb), o = (int)(t % g.n_orb);
  const TsEntry en = g.ent[e];
  const long st = g.stride[en.ax];
  const double2 phi = ts_value(g, o, en.cell);
  double gx = 0.0, gy = 0.0;
  for (int m = 1; m <= g.M; m++) {
    const double2 a = ts_value(g, o, en.cell + m * st), b = ts_value(g, o, en.cell - m * st);
    gx += g.d[m] * (a.x - b.x);
    gy += g.d[m] * (a.y - b.y);
  }
  // w n (phi) and w n (-i grad phi); -i (gx + i gy) = gy - i gx
  g.G0[t] = make_double2(en.ws * phi.x, en.ws * phi.y);
  g.G1[t] = make_double2(en.ws * gy, -en.ws * gx);
}

struct TsFlux {
  int n_e, n_orb, n_p;
  const TsEntry *ent;
  const double2 *G0, *G1;
  const double *p;         // [n_p][3]
  double a[3], alpha[3], beta, t_rel, weight;
  double2 *b;              // [n_orb][n_p]
};

constexpr int TS_THREADS = 128;

// One momentum per CTA; threads over orbitals.  The Volkov factor exp(-i k_p.r_e) of a tile
// of entries is formed once per CTA in shared memory.
__global__ void __launch_bounds__(TS_THREADS) tsurff_flux_kernel(const TsFlux f) {
  __shared__ double2 sW[TS_THREADS];
  __shared__ double sK[TS_THREADS];
  const int pi = blockIdx.x, tid = threadIdx.x;
  const double px = f.p[3 * pi], py = f.p[3 * pi + 1], pz = f.p[3 * pi + 2];
  const double k[3] = {px + f.a[0], py + f.a[1], pz + f.a[2]};
  const double phase = 0.5 * ((px * px + py * py + pz * pz) * f.t_rel +
                              2.0 * (px * f.alpha[0] + py * f.alpha[1] + pz * f.alpha[2]) + f.beta);
  for (int o0 = 0; o0 < f.n_orb; o0 += TS_THREADS) {
    const int o = o0 + tid;
    double ar = 0.0, ai = 0.0;
    for (int e0 = 0; e0 < f.n_e; e0 += TS_THREADS) {
      const int e = e0 + tid;
      if (e < f.n_e) {
        const TsEntry en = f.ent[e];
        double sn, cs;
        sincos(k[0] * en.r[0] + k[1] * en.r[1] + k[2] * en.r[2], &sn, &cs);
        sW[tid] = make_double2(cs, -sn);
        sK[tid] = k[en.ax];
      }
      __syncthreads();
      if (o < f.n_orb) {
        const int ne = min(TS_THREADS, f.n_e - e0);
        for (int j = 0; j < ne; j++) {
          const long gi = (long)(e0 + j) * f.n_orb + o;
          const double2 g0 = f.G0[gi], g1 = f.G1[gi], w = sW[j];
          const double tr = sK[j] * g0.x + g1.x, ti = sK[j] * g0.y + g1.y;
          ar += w.x * tr - w.y * ti;
          ai += w.x * ti + w.y * tr;
        }
      }
      __syncthreads();
    }
    if (o < f.n_orb) {
      double sn, cs;
      sincos(phase, &sn, &cs);
      const double pref = 0.5 * f.weight * 0.063493635934240969;  // (2 pi)^(-3/2)
      double2 &bo = f.b[(long)o * f.n_p + pi];
      bo.x += pref * (cs * ar - sn * ai);
      bo.y += pref * (cs * ai + sn * ar);
    }
  }
}

}  // namespace

namespace tdks_host {

void tsurff_free(tdks_system *s) {
  cudaFree(s->d_ts_p); cudaFree(s->d_ts_ent); cudaFree(s->d_ts_G); cudaFree(s->d_ts_b);
  s->d_ts_p = nullptr; s->d_ts_ent = nullptr; s->d_ts_G = nullptr; s->d_ts_b = nullptr;
  s->ts_np = 0;
  s->ts_ne = 0;
}

// The flux of the current state with trapezoid weight `weight` (dt or dt/2) into b.
int tsurff_accumulate(tdks_system *s, double weight) {
  double c[MAXM + 1], d[MAXM + 1];
  fd_weights(s->M, c, d);
  TsGather g{};
  g.prec = s->prec; g.BS = s->BS; g.n_orb = s->n_orb; g.N = s->N;
  g.stride[0] = 1; g.stride[1] = s->nx; g.stride[2] = (long)s->nx * s->ny;
  g.psi = s->psi; g.psi_lo = s->psi_lo; g.ent = s->d_ts_ent; g.n_e = s->ts_ne; g.M = s->M;
  for (int m = 0; m <= MAXM; m++) g.d[m] = m <= s->M ? d[m] / s->h : 0.0;
  g.G0 = s->d_ts_G;
  g.G1 = s->d_ts_G + (size_t)s->ts_ne * s->n_orb;
  const long n = (long)s->ts_ne * s->n_orb;
  tsurff_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s->stream>>>(g);
  TsFlux f{};
  f.n_e = s->ts_ne; f.n_orb = s->n_orb; f.n_p = s->ts_np; f.ent = s->d_ts_ent;
  f.G0 = g.G0; f.G1 = g.G1; f.p = s->d_ts_p;
  for (int x = 0; x < 3; x++) { f.a[x] = s->ts_vol[x]; f.alpha[x] = s->ts_vol[3 + x]; }
  f.beta = s->ts_vol[6];
  f.t_rel = s->ts_trel;
  f.weight = weight;
  f.b = s->d_ts_b;
  tsurff_flux_kernel<<<s->ts_np, TS_THREADS, 0, s->stream>>>(f);
  s->launches += 2;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("t-SURFF flux: ") + cudaGetErrorString(e));
  return TDKS_OK;
}

// a, alpha, beta from t to t + dt: the classical Runge-Kutta method on a' = -E (length
// gauge; zero otherwise), alpha' = a, beta' = |a|^2.
void tsurff_advance(tdks_system *s, double t, double dt) {
  auto rhs = [&](double tt, const double *y, double *f) {
    double E[3], A[3];
    field_at(s, tt, E, A);
    for (int x = 0; x < 3; x++) {
      f[x] = s->gauge == TDKS_GAUGE_LENGTH ? -E[x] : 0.0;
      f[3 + x] = y[x];
    }
    f[6] = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
  };
  double *y = s->ts_vol, k1[7], k2[7], k3[7], k4[7], tmp[7];
  rhs(t, y, k1);
  for (int i = 0; i < 7; i++) tmp[i] = y[i] + 0.5 * dt * k1[i];
  rhs(t + 0.5 * dt, tmp, k2);
  for (int i = 0; i < 7; i++) tmp[i] = y[i] + 0.5 * dt * k2[i];
  rhs(t + 0.5 * dt, tmp, k3);
  for (int i = 0; i < 7; i++) tmp[i] = y[i] + dt * k3[i];
  rhs(t + dt, tmp, k4);
  for (int i = 0; i < 7; i++) y[i] += dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  s->ts_trel += dt;
}

}  // namespace tdks_host

extern "C" int tdks_set_tsurff(tdks_sys s, const int *box, int n_p, const double *p) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (n_p < 0) return fail(TDKS_EINVAL, "n_p < 0");
  CU(cudaStreamSynchronize(s->stream));
  tsurff_free(s);
  if (n_p == 0) return TDKS_OK;
  if (!box || !p) return fail(TDKS_EINVAL, "NULL argument");
  if (s->bc != TDKS_BC_ZERO || s->n_k != 1) return fail(TDKS_EINVAL, "t-SURFF needs a finite box with one k-point");
  const int n[3] = {s->nx, s->ny, s->nz};
  for (int a = 0; a < 3; a++)
    if (box[2 * a] < s->M || box[2 * a] >= box[2 * a + 1] || box[2 * a + 1] > n[a] - 1 - s->M)
      return fail(TDKS_EINVAL, "t-SURFF box planes must satisfy M <= lo < hi <= n - 1 - M on every axis");
  for (int i = 0; i < 3 * n_p; i++)
    if (!std::isfinite(p[i])) return fail(TDKS_EINVAL, "momenta must be finite");
  // surface entries: every grid point of each face (trapezoid weight h^2, halved on the face's
  // edges) with the face's outward normal; points on edges and corners belong to each face
  std::vector<TsEntry> ent;
  for (int face = 0; face < 6; face++) {
    const int ax = face / 2, ua = (ax + 1) % 3, va = (ax + 2) % 3;
    const double sgn = (face % 2) ? 1.0 : -1.0;
    for (int u = box[2 * ua]; u <= box[2 * ua + 1]; u++)
      for (int v = box[2 * va]; v <= box[2 * va + 1]; v++) {
        int ii[3];
        ii[ax] = box[2 * ax + (face % 2)];
        ii[ua] = u;
        ii[va] = v;
        double w = s->h * s->h;
        if (u == box[2 * ua] || u == box[2 * ua + 1]) w *= 0.5;
        if (v == box[2 * va] || v == box[2 * va + 1]) w *= 0.5;
        TsEntry e{};
        e.cell = ((long)ii[2] * s->ny + ii[1]) * s->nx + ii[0];
        e.ax = ax;
        e.ws = sgn * w;
        for (int q = 0; q < 3; q++) e.r[q] = (ii[q] - 0.5 * (n[q] - 1)) * s->h;
        ent.push_back(e);
      }
  }
  s->ts_ne = (int)ent.size();
  CU(cudaMalloc((void **)&s->d_ts_ent, ent.size() * sizeof(TsEntry)));
  CU(cudaMemcpy(s->d_ts_ent, ent.data(), ent.size() * sizeof(TsEntry), cudaMemcpyHostToDevice));
  CU(cudaMalloc((void **)&s->d_ts_p, (size_t)n_p * 3 * sizeof(double)));
  CU(cudaMemcpy(s->d_ts_p, p, (size_t)n_p * 3 * sizeof(double), cudaMemcpyHostToDevice));
  CU(cudaMalloc((void **)&s->d_ts_G, 2 * ent.size() * (size_t)s->n_orb * sizeof(double2)));
  CU(cudaMalloc((void **)&s->d_ts_b, (size_t)s->n_orb * n_p * sizeof(double2)));
  CU(cudaMemset(s->d_ts_b, 0, (size_t)s->n_orb * n_p * sizeof(double2)));
  s->ts_np = n_p;
  for (int i = 0; i < 7; i++) s->ts_vol[i] = 0.0;
  s->ts_trel = 0.0;
  s->ts_started = false;
  return TDKS_OK;
}

extern "C" int tdks_get_tsurff(tdks_sys s, double *b, double *t_rel) {
  if (!s) return fail(TDKS_EINVAL, "NULL system");
  if (s->ts_np == 0) return fail(TDKS_ESTATE, "t-SURFF is not set");
  CU(cudaStreamSynchronize(s->stream));
  if (int rc = check_err(s)) return rc;
  if (b) CU(cudaMemcpy(b, s->d_ts_b, (size_t)s->n_orb * s->ts_np * sizeof(double2), cudaMemcpyDeviceToHost));
  if (t_rel) *t_rel = s->ts_trel;
  return TDKS_OK;
}
