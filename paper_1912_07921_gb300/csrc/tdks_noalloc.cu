// H applied without allocating device memory, for callers that may not allocate.
//
// Some callers cannot call cudaMalloc: code that runs inside a host framework which owns
// all device memory through its own pool and forbids other allocations, or a real-time
// loop in which a cudaMalloc/cudaFree (which can synchronise the device and stall other
// streams) is not acceptable.  tdks_apply_H_noalloc serves them.  The caller passes the
// potential, the input orbitals and the output buffer; the only scratch this path needs
// (a per-point record with the potential in the compute precision, an error word and the
// sweep's work counter) lives in a file-scope
// __device__ array of fixed size, which every GPU that loads the library holds until the
// process exits.
//
// The scratch array is shared by all calls on a device and keeps the last call's
// contents.  Calls whose work overlaps on the GPU (several streams, or several host
// threads) race on it; serialise them.  The first call on a device looks up the array's
// device address (cudaGetSymbolAddress) with that device current.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "tdks_system.h"

using namespace tdks;
using namespace tdks_host;

namespace {

// Largest grid served: 2^20 points (e.g. 96^3 = 884,736 fits; 128^3 does not).
constexpr long NOALLOC_MAX_POINTS = 1L << 20;
constexpr int NOALLOC_MAX_DEVICES = 64;

// [0, 16 * NOALLOC_MAX_POINTS): one 16-byte record per point (the potential in the compute
// precision, an empty projector range); then the error word and the sweep's work counter.
static __device__ __align__(256) unsigned char g_noalloc_scratch[16 * NOALLOC_MAX_POINTS + 256];

std::mutex g_addr_mutex;
void *g_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(void **out) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(TDKS_EDEVICE, "device index out of range");
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return TDKS_OK;
}

template <typename R>
__global__ void noalloc_prepare(long N, const double *vloc, PointAux *aux, int *err) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i == 0) {  // the error word and the sweep's work counter must start at zero on every call
    err[0] = 0;
    err[1] = 0;
  }
  if (i < N) {
    PointAux a{0.0, 0, 0};
    *reinterpret_cast<R *>(&a.veff) = (R)vloc[i];
    aux[i] = a;
  }
}

}  // namespace

extern "C" int tdks_apply_H_noalloc(int nx, int ny, int nz, double h, int fd_order, int prec, int n_orb,
                                    const double *dev_vloc, const void *dev_in, void *dev_out, void *stream) {
  if (fd_order != 4 && fd_order != 8) return fail(TDKS_EINVAL, "fd_order must be 4 or 8");
  if (prec != TDKS_C128 && prec != TDKS_C64) return fail(TDKS_EINVAL, "bad precision");
  const int M = fd_order / 2;
  if (nx < M + 1 || ny < M + 1 || nz < M + 1 || !(h > 0.0) || n_orb < 1)
    return fail(TDKS_EINVAL, "bad grid or orbital count");
  if (!dev_vloc || !dev_in || !dev_out || dev_in == dev_out) return fail(TDKS_EINVAL, "bad buffers");
  const long N = (long)nx * ny * nz;
  if (N > NOALLOC_MAX_POINTS)
    return fail(TDKS_EINVAL, "grid has " + std::to_string(N) + " points; tdks_apply_H_noalloc serves at most " +
                                 std::to_string(NOALLOC_MAX_POINTS));
  void *scratch = nullptr;
  if (int rc = scratch_address(&scratch)) return rc;
  unsigned char *base = static_cast<unsigned char *>(scratch);
  int *err = reinterpret_cast<int *>(base + 16 * NOALLOC_MAX_POINTS);
  PointAux *aux = reinterpret_cast<PointAux *>(base);
  cudaStream_t st = (cudaStream_t)stream;

  // a host-side description of the grid (no device memory behind it)
  tdks_system s;
  s.nx = nx; s.ny = ny; s.nz = nz; s.h = h; s.M = M; s.bc = TDKS_BC_ZERO; s.prec = prec; s.n_orb = n_orb;
  s.n_k = 1; s.N = N;
  s.BS = prec == TDKS_C64 ? 2 * OVC : OVC;
  s.n_batches = (n_orb + s.BS - 1) / s.BS;
  s.n_kb = s.n_batches;
  s.aux = aux;
  s.stream = st;

  const int blocks = (int)((N + 255) / 256);
  if (prec == TDKS_C64) noalloc_prepare<float><<<blocks, 256, 0, st>>>(N, dev_vloc, aux, err);
  else noalloc_prepare<double><<<blocks, 256, 0, st>>>(N, dev_vloc, aux, err);
  CU(cudaGetLastError());

  const double A0[3] = {0.0, 0.0, 0.0};
  SweepParams p{};
  sweep_common(&s, p, A0);
  set_coef(p, 1.0, 0.0);
  p.in = dev_in;
  p.out = dev_out;
  p.err = err;
  p.work = reinterpret_cast<unsigned int *>(err + 1);
  SweepMaps tm;
  cudaError_t e;
  if (tma_supported(M, s.tx, s.ty) && encode_sweep_maps(&s, dev_in, MODE_MID, &tm, false))
    e = launch_sweep_tma(M, prec, MODE_MID, s.tx, s.ty, tm, p, 0, st);
  else
    e = launch_sweep(M, prec, MODE_MID, 0, s.tx, s.ty, p, 0, st);
  if (e != cudaSuccess) return fail(TDKS_EDEVICE, std::string("stencil sweep: ") + cudaGetErrorString(e));
  // wait for the result and report a sweep that gave up waiting for its copies; the error
  // word is read on the caller's stream, so no other stream of the device is waited for
  int h_err = 0;
  CU(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (h_err) return fail(TDKS_ETIMEOUT, "the sweep gave up waiting for its TMA copies");
  return TDKS_OK;
}
