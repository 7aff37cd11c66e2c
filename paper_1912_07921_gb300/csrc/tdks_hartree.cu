// Hartree potential of the density (the density-dependent potential beside exchange in the
// Kohn-Sham Hamiltonian, which CFM4 of Sec. "New propagators for real-time TDDFT"
// extrapolates as part of Hxc):
//   finite box:     v_H(r_i) = h^3 sum_j K(r_i - r_j) n_j,  K(d) = 1/|d|,  K(0) = c0 / h,
//                   c0 = 3 ln(2 + sqrt 3) - pi/2 (the Coulomb integral of a cell over itself);
//                   a linear convolution, computed exactly by a zero-padded FFT (Hockney):
//                   v = IFFT(FFT(n padded) FFT(K padded)) on a grid of >= 2n - 1 points per axis;
//   periodic cell:  v_H(G) = 4 pi n(G) / |G|^2 on the grid's plane waves (G the alias nearest
//                   zero), G = 0 dropped (neutralising background).
// The FFTs are the library's own: one CTA per line of a 3D array, the line in shared memory,
// mixed-radix Stockham passes (Govindaraju et al., SC 2008: each pass takes R values N/R
// apart, twiddles them, does an R-point DFT and stores them in autosorted order), radices the
// prime factors of the line length (all <= 13), FP64 throughout.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "tdks_system.h"

using namespace tdks;
using namespace tdks_host;

namespace {

constexpr int FFT_THREADS = 128;
constexpr int FFT_MAXR = 13;      // largest radix (prime factor of a line length)
constexpr int FFT_MAXN = 1024;    // longest line

struct FftAxis {
  int n;             // line length
  int nrad, rad[12]; // radices, in the order the passes take them
  long stride;       // element stride along the line
  long d0, d1;       // the other two dimensions' sizes (line index = i0 + d0 i1)
  long s0, s1;       // and their strides
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place transform of every line along one axis: sign -1 forward, +1 inverse; scale applied
// on the way out.
__global__ void __launch_bounds__(FFT_THREADS) fft_lines_kernel(double2 *data, const FftAxis ax, int sign,
                                                                 double scale) {
  extern __shared__ double2 sm[];
  double2 *a = sm, *b = sm + ax.n;
  const long l = blockIdx.x;
  const long start = (l % ax.d0) * ax.s0 + (l / ax.d0) * ax.s1;
  const int n = ax.n, tid = threadIdx.x;
  for (int i = tid; i < n; i += FFT_THREADS) a[i] = data[start + i * ax.stride];
  __syncthreads();
  int Ns = 1;
  for (int pass = 0; pass < ax.nrad; pass++) {
    const int R = ax.rad[pass], m = n / R;
    for (int j = tid; j < m; j += FFT_THREADS) {
      const int k = j % Ns;
      double2 v[FFT_MAXR];
      for (int r = 0; r < R; r++) {
        double sn, cs;
        sincospi((double)sign * 2.0 * (double)(k * r) / (double)(Ns * R), &sn, &cs);
        v[r] = cmul(a[j + r * m], make_double2(cs, sn));
      }
      const int base = (j / Ns) * Ns * R + k;
      for (int q = 0; q < R; q++) {
        double2 w = make_double2(0.0, 0.0);
        for (int r = 0; r < R; r++) {
          double sn, cs;
          sincospi((double)sign * 2.0 * (double)((r * q) % R) / (double)R, &sn, &cs);
          const double2 t = cmul(v[r], make_double2(cs, sn));
          w.x += t.x;
          w.y += t.y;
        }
        b[base + q * Ns] = w;
      }
    }
    __syncthreads();
    double2 *t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  for (int i = tid; i < n; i += FFT_THREADS)
    data[start + i * ax.stride] = make_double2(scale * a[i].x, scale * a[i].y);
}

// density into the padded complex array (zeros elsewhere)
__global__ void hartree_pad_kernel(const double *n, int nx, int ny, int nz, int px, int py, long P, double2 *buf) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < P; i += (long)gridDim.x * blockDim.x) {
    const int x = (int)(i % px), y = (int)((i / px) % py), z = (int)(i / ((long)px * py));
    double v = 0.0;
    if (x < nx && y < ny && z < nz) v = n[((long)z * ny + y) * nx + x];
    buf[i] = make_double2(v, 0.0);
  }
}

// transformed density times the transformed kernel
__global__ void hartree_mul_kernel(double2 *buf, const double2 *kern, long P) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < P; i += (long)gridDim.x * blockDim.x)
    buf[i] = cmul(buf[i], kern[i]);
}

// v_H on the grid: the real part of the box region, times `scale`
__global__ void hartree_crop_kernel(const double2 *buf, int nx, int ny, int nz, int px, int py, double scale,
                                    double *vh) {
  const long N = (long)nx * ny * nz;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long)nx * ny));
    vh[i] = scale * buf[((long)z * py + y) * px + x].x;
  }
}

// the sampled kernel on the padded grid: offsets 0..n-1 at indices 0..n-1, offsets -(n-1)..-1
// at indices P-(n-1)..P-1, zero in between (never met by a linear convolution of n points)
__global__ void hartree_kernel_box(int nx, int ny, int nz, int px, int py, int pz, double h, double self,
                                   double2 *kern) {
  const long P = (long)px * py * pz;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < P; i += (long)gridDim.x * blockDim.x) {
    const int x = (int)(i % px), y = (int)((i / px) % py), z = (int)(i / ((long)px * py));
    const int dx = x < nx ? x : (x > px - nx ? x - px : INT32_MAX);
    const int dy = y < ny ? y : (y > py - ny ? y - py : INT32_MAX);
    const int dz = z < nz ? z : (z > pz - nz ? z - pz : INT32_MAX);
    double v = 0.0;
    if (dx != INT32_MAX && dy != INT32_MAX && dz != INT32_MAX) {
      if (dx == 0 && dy == 0 && dz == 0) v = self / h;
      else v = 1.0 / (h * sqrt((double)dx * dx + (double)dy * dy + (double)dz * dz));
    }
    kern[i] = make_double2(v, 0.0);
  }
}

// periodic cell: 4 pi / |G|^2 with G the alias of each index nearest zero, 0 at G = 0, over
// the number of points (the inverse transform is unscaled)
__global__ void hartree_kernel_cell(int nx, int ny, int nz, double Lx, double Ly, double Lz, double2 *kern) {
  const long N = (long)nx * ny * nz;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long)nx * ny));
    const int ax = x <= nx / 2 ? x : x - nx, ay = y <= ny / 2 ? y : y - ny, az = z <= nz / 2 ? z : z - nz;
    const double gx = 2.0 * M_PI * ax / Lx, gy = 2.0 * M_PI * ay / Ly, gz = 2.0 * M_PI * az / Lz;
    const double g2 = gx * gx + gy * gy + gz * gz;
    kern[i] = make_double2(i == 0 ? 0.0 : 4.0 * M_PI / g2 / (double)N, 0.0);
  }
}

bool factor(int n, FftAxis &ax) {
  ax.n = n;
  ax.nrad = 0;
  int m = n;
  for (int p = 2; p <= FFT_MAXR && m > 1; p++)
    while (m % p == 0) {
      if (ax.nrad == 12) return false;
      ax.rad[ax.nrad++] = p;
      m /= p;
    }
  return m == 1 && n <= FFT_MAXN;
}

// smallest length >= m whose prime factors are 2 and 3
int smooth_at_least(int m) {
  for (int c = m;; c++) {
    int r = c;
    while (r % 2 == 0) r /= 2;
    while (r % 3 == 0) r /= 3;
    if (r == 1) return c;
  }
}

int grid_blocks(long n) {
  const long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152L * 16 ? 152L * 16 : b));
}

// the three axis descriptions of a P0 x P1 x P2 array (x fastest)
bool axes(int p0, int p1, int p2, FftAxis ax[3]) {
  if (!factor(p0, ax[0]) || !factor(p1, ax[1]) || !factor(p2, ax[2])) return false;
  const long P01 = (long)p0 * p1;
  ax[0].stride = 1;   ax[0].d0 = p1; ax[0].s0 = p0;  ax[0].d1 = p2; ax[0].s1 = P01;
  ax[1].stride = p0;  ax[1].d0 = p0; ax[1].s0 = 1;   ax[1].d1 = p2; ax[1].s1 = P01;
  ax[2].stride = P01; ax[2].d0 = p0; ax[2].s0 = 1;   ax[2].d1 = p1; ax[2].s1 = p0;
  return true;
}

cudaError_t fft3(double2 *buf, const FftAxis ax[3], int sign, double scale, cudaStream_t s) {
  for (int a = 0; a < 3; a++) {
    const long lines = ax[a].d0 * ax[a].d1;
    fft_lines_kernel<<<(unsigned)lines, FFT_THREADS, 2 * ax[a].n * sizeof(double2), s>>>(buf, ax[a], sign,
                                                                                       a == 2 ? scale : 1.0);
  }
  return cudaGetLastError();
}

}  // namespace

namespace tdks_host {

void hartree_free(tdks_system *s) {
  cudaFree(s->d_hbuf); cudaFree(s->d_hkern); cudaFree(s->d_vh);
  s->d_hbuf = s->d_hkern = nullptr;
  s->d_vh = nullptr;
}

// Workspace and the transformed kernel of the system's grid (once, when the Hartree term is
// turned on).
int hartree_setup(tdks_system *s) {
  if (s->d_vh) return TDKS_OK;
  int p[3];
  const int n[3] = {s->nx, s->ny, s->nz};
  for (int a = 0; a < 3; a++) p[a] = s->bc == TDKS_BC_ZERO ? smooth_at_least(2 * n[a] - 1) : n[a];
  FftAxis ax[3];
  if (!axes(p[0], p[1], p[2], ax))
    return fail(TDKS_EINVAL, "Hartree term: grid edges need prime factors <= 13 and transforms of <= 1024 points");
  s->hp[0] = p[0]; s->hp[1] = p[1]; s->hp[2] = p[2];
  const long P = (long)p[0] * p[1] * p[2];
  CU(cudaMalloc((void **)&s->d_hbuf, P * sizeof(double2)));
  CU(cudaMalloc((void **)&s->d_hkern, P * sizeof(double2)));
  CU(cudaMalloc((void **)&s->d_vh, s->N * sizeof(double)));
  if (!s->n_total) CU(cudaMalloc((void **)&s->n_total, (size_t)s->N * sizeof(double)));
  if (s->bc == TDKS_BC_ZERO) {
    const double self = 3.0 * std::log(2.0 + std::sqrt(3.0)) - 0.5 * M_PI;
    hartree_kernel_box<<<grid_blocks(P), 256, 0, s->stream>>>(s->nx, s->ny, s->nz, p[0], p[1], p[2], s->h, self,
                                                              s->d_hkern);
    CU(cudaGetLastError());
    CU(fft3(s->d_hkern, ax, -1, 1.0, s->stream));
  } else {
    hartree_kernel_cell<<<grid_blocks(P), 256, 0, s->stream>>>(s->nx, s->ny, s->nz, s->nx * s->h, s->ny * s->h,
                                                               s->nz * s->h, s->d_hkern);
    CU(cudaGetLastError());
  }
  CU(cudaStreamSynchronize(s->stream));
  return TDKS_OK;
}

// v_H of the density in n_total (FP64, N points) into d_vh.
int hartree_solve(tdks_system *s) {
  FftAxis ax[3];
  axes(s->hp[0], s->hp[1], s->hp[2], ax);
  const long P = (long)s->hp[0] * s->hp[1] * s->hp[2];
  hartree_pad_kernel<<<grid_blocks(P), 256, 0, s->stream>>>(s->n_total, s->nx, s->ny, s->nz, s->hp[0], s->hp[1], P,
                                                            s->d_hbuf);
  cudaError_t e = fft3(s->d_hbuf, ax, -1, 1.0, s->stream);
  if (e == cudaSuccess) {
    hartree_mul_kernel<<<grid_blocks(P), 256, 0, s->stream>>>(s->d_hbuf, s->d_hkern, P);
    // box: the unscaled inverse transform is P times the convolution; cell: the kernel
    // already holds 1/N
    const double h3 = s->h * s->h * s->h;
    e = fft3(s->d_hbuf, ax, +1, s->bc == TDKS_BC_ZERO ? h3 / (double)P : 1.0, s->stream);
  }
  if (e == cudaSuccess) {
    hartree_crop_kernel<<<grid_blocks(s->N), 256, 0, s->stream>>>(s->d_hbuf, s->nx, s->ny, s->nz, s->hp[0],
                                                                  s->hp[1], 1.0, s->d_vh);
    e = cudaGetLastError();
  }
  s->launches += 11;
  if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("Hartree: ") + cudaGetErrorString(e));
  return TDKS_OK;
}

}  // namespace tdks_host
