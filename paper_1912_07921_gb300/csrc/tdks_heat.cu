// Kinetic heat current of a periodic cell (Sec. "Conductivities", eqn. KEcurrent): the
// macroscopic J_t = (1/Omega) sum_k w_k f int [J_t(r)] dr with
//   [J_t]_i = (i/8) ( [d_i phi^*][Lap phi] - [Lap phi^*][d_i phi] - [d_i grad phi^*].[grad phi]
//                     + [grad phi^*].[d_i grad phi] )
// (the printed last pair with the sign that makes J_t real), derivatives covariant in the
// velocity gauge: D_j = d_j + i A_j (d_j the central difference of order 2M, Bloch images),
// Lap -> the star Laplacian + 2 i A.d - |A|^2.  Over the cell the D_j are anti-Hermitian and
// commute, so int [d_i grad phi^*].[grad phi] = int (sum_j D_j D_j phi)^* D_i phi: the cell integral
// needs only star stencils at each point (radius M for d and the Laplacian, radius 2M for
// sum_j D_j^2, whose 1D weights are the first-difference weights composed), and
//   J_t,i = (1/Omega) sum_k w_k f h^3 sum_r 1/4 ( Im[(D^2 phi)^* D_i phi] - Im[(D_i phi)^* Lap phi] ).
// Computed on demand (tdks_heat_current), FP64, one thread per (point, orbital), per-CTA
// partial sums added on the host in order.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "tdks_system.h"

using namespace tdks;
using namespace tdks_host;

namespace {

constexpr int HC_THREADS = 256;
constexpr int HC_MAXS = 2 * MAXM;  // widest offset of the composed second difference

struct HeatParams {
  int prec, BS, n_batches, n_kb, nx, ny, nz, M;
  long N;
  const void *psi, *psi_lo;
  const double *kvec, *wocc;
  double L[3], A[3];
  double c[MAXM + 1];      // star Laplacian weights over h^2
  double d[MAXM + 1];      // first-difference weights over h
  double dd[HC_MAXS + 1];  // composed second-difference weights (offset s >= 0; symmetric)
  double scale;            // h^3 / (4 Omega)
  double *part;            // [gridDim.x][3]
};

__device__ __forceinline__ double2 value(const HeatParams &p, int kb, int j, long pt) {
  const long i = ((long)kb * p.N + pt) * p.BS + j;
  if (p.prec == P_C128) return reinterpret_cast<const double2 *>(p.psi)[i];
  const float2 hi = reinterpret_cast<const float2 *>(p.psi)[i], lo = reinterpret_cast<const float2 *>(p.psi_lo)[i];
  return make_double2((double)hi.x + (double)lo.x, (double)hi.y + (double)lo.y);
}

// phi at grid offset s along axis a from (x, y, z): the periodic image with its Bloch phase
__device__ __forceinline__ double2 neighbour(const HeatParams &p, int kb, int j, int x, int y, int z, int a, int s,
                                            const double *kk) {
  int c[3] = {x, y, z};
  const int n[3] = {p.nx, p.ny, p.nz};
  c[a] += s;
  const int w = c[a] >= 0 ? c[a] / n[a] : -((-c[a] - 1) / n[a]) - 1;
  c[a] -= w * n[a];
  const double2 v = value(p, kb, j, ((long)c[2] * p.ny + c[1]) * p.nx + c[0]);
  if (w == 0) return v;
  double sn, cs;
  sincos(kk[a] * p.L[a] * (double)w, &sn, &cs);
  return make_double2(cs * v.x - sn * v.y, cs * v.y + sn * v.x);
}

__global__ void __launch_bounds__(HC_THREADS) heat_current_kernel(const HeatParams p) {
  const long total = (long)p.n_kb * p.N * p.BS;
  double acc[3] = {0.0, 0.0, 0.0};
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int j = (int)(t % p.BS);
    const long pt = (t / p.BS) % p.N;
    const int kb = (int)(t / ((long)p.BS * p.N));
    const int kidx = kb / p.n_batches;
    const double *kk = p.kvec + 3 * kidx;
    const int x = (int)(pt % p.nx), y = (int)((pt / p.nx) % p.ny), z = (int)(pt / ((long)p.nx * p.ny));
    const double2 v = value(p, kb, j, pt);
    double2 g[3], lap = make_double2(3.0 * p.c[0] * v.x, 3.0 * p.c[0] * v.y), dd = make_double2(0.0, 0.0);
    double adr = 0.0, adi = 0.0;  // A . d phi
    for (int a = 0; a < 3; a++) {
      double gx = 0.0, gy = 0.0;
      for (int s = 1; s <= 2 * p.M; s++) {
        const double2 f = neighbour(p, kb, j, x, y, z, a, s, kk), b = neighbour(p, kb, j, x, y, z, a, -s, kk);
        if (s <= p.M) {
          gx += p.d[s] * (f.x - b.x);
          gy += p.d[s] * (f.y - b.y);
          lap.x += p.c[s] * (f.x + b.x);
          lap.y += p.c[s] * (f.y + b.y);
        }
        dd.x += p.dd[s] * (f.x + b.x);
        dd.y += p.dd[s] * (f.y + b.y);
      }
      dd.x += p.dd[0] * v.x;
      dd.y += p.dd[0] * v.y;
      adr += p.A[a] * gx;
      adi += p.A[a] * gy;
      // covariant gradient: d phi + i A phi
      g[a] = make_double2(gx - p.A[a] * v.y, gy + p.A[a] * v.x);
    }
    // covariant Laplacians: + 2 i A.d phi - |A|^2 phi
    const double A2 = p.A[0] * p.A[0] + p.A[1] * p.A[1] + p.A[2] * p.A[2];
    lap = make_double2(lap.x - 2.0 * adi - A2 * v.x, lap.y + 2.0 * adr - A2 * v.y);
    dd = make_double2(dd.x - 2.0 * adi - A2 * v.x, dd.y + 2.0 * adr - A2 * v.y);
    const double w = p.wocc[kidx];
    for (int a = 0; a < 3; a++) {
      // Im(conj(u) v) = u.x v.y - u.y v.x
      const double c1 = dd.x * g[a].y - dd.y * g[a].x;
      const double c2 = g[a].x * lap.y - g[a].y * lap.x;
      acc[a] += w * (c1 - c2);
    }
  }
  __shared__ double red[HC_THREADS / 32][3];
  for (int a = 0; a < 3; a++) {
    double s = acc[a];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][a] = s;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < HC_THREADS / 32; w++) s += red[w][threadIdx.x];
    p.part[blockIdx.x * 3 + threadIdx.x] = p.scale * s;
  }
}

}  // namespace

extern "C" int tdks_heat_current(tdks_sys s, double t_field, double *out) {
  if (!s || !out) return fail(TDKS_EINVAL, "NULL argument");
  if (s->bc != TDKS_BC_BLOCH) return fail(TDKS_EINVAL, "the heat current is defined for periodic cells");
  if (!s->have_orbitals) return fail(TDKS_ESTATE, "orbitals not set");
  double c[MAXM + 1], d[MAXM + 1];
  fd_weights(s->M, c, d);
  HeatParams p{};
  p.prec = s->prec; p.BS = s->BS; p.n_batches = s->n_batches; p.n_kb = s->n_kb;
  p.nx = s->nx; p.ny = s->ny; p.nz = s->nz; p.M = s->M; p.N = s->N;
  p.psi = s->psi; p.psi_lo = s->psi_lo; p.kvec = s->d_kvec; p.wocc = s->d_wocc;
  p.L[0] = s->nx * s->h; p.L[1] = s->ny * s->h; p.L[2] = s->nz * s->h;
  double E[3], A[3];
  field_at(s, t_field, E, A);
  for (int a = 0; a < 3; a++) p.A[a] = s->gauge == TDKS_GAUGE_VELOCITY ? A[a] : 0.0;
  const double h = s->h;
  for (int m = 0; m <= MAXM; m++) {
    p.c[m] = m <= s->M ? c[m] / (h * h) : 0.0;
    p.d[m] = m <= s->M ? d[m] / h : 0.0;
  }
  // composed second difference: sum_{m,m'} d_m d_m' (phi(x+m+m') - phi(x+m-m') - phi(x-m+m') + phi(x-m-m'))
  double w[2 * HC_MAXS + 1] = {};
  for (int m = 1; m <= s->M; m++)
    for (int q = 1; q <= s->M; q++) {
      const double dm = d[m] * d[q] / (h * h);
      w[HC_MAXS + m + q] += dm;
      w[HC_MAXS + m - q] -= dm;
      w[HC_MAXS - m + q] -= dm;
      w[HC_MAXS - m - q] += dm;
    }
  for (int t = 0; t <= HC_MAXS; t++) p.dd[t] = w[HC_MAXS + t];
  const double omega = (double)s->N * h * h * h;
  p.scale = h * h * h / (4.0 * omega);
  const int blocks = 152 * 8;
  double *part = nullptr;
  CU(cudaMalloc((void **)&part, (size_t)blocks * 3 * sizeof(double)));
  p.part = part;
  heat_current_kernel<<<blocks, HC_THREADS, 0, s->stream>>>(p);
  s->launches++;
  std::vector<double> hp((size_t)blocks * 3);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(part);
  if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("heat current: ") + cudaGetErrorString(e));
  for (int a = 0; a < 3; a++) {
    double sum = 0.0;
    for (int b = 0; b < blocks; b++) sum += hp[(size_t)b * 3 + a];
    out[a] = sum;
  }
  return check_err(s);
}
