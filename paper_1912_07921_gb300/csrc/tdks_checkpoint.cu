// Checkpoint and resume of one system (tdks_save / tdks_load): the configuration, the
// device state exactly as stored (complex128, or the hi and lo parts of a complex64 state),
// the density partials of that state, the propagator and its exchange history, the clock
// and the stored observable records, so that a loaded system continues bit for bit as the
// saved one would have.
//
// File layout (little-endian, as both supported hosts are): the 8-byte magic "TDKSCKP1";
// a header of 32 int64 and 16 double fields; then the arrays in a fixed order, each a raw
// block of the length the header implies; last, a 64-bit checksum over everything before it.
// The file is written under path + ".tmp" and renamed into place once complete.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tdks_system.h"

using namespace tdks;
using namespace tdks_host;

namespace {

constexpr char MAGIC[8] = {'T', 'D', 'K', 'S', 'C', 'K', 'P', '1'};
constexpr int NI = 32, ND = 16;
enum {  // int64 header fields
  H_NX, H_NY, H_NZ, H_ORDER, H_BC, H_PREC, H_NORB, H_NK, H_XC, H_GAUGE, H_ENV, H_NATOMS, H_PROP, H_NHIST,
  H_STEPS, H_CSUB, H_PATH, H_TX, H_TY, H_ZC, H_WS0, H_WS1, H_WS2, H_WS3, H_HAVE, H_NREC
};
enum {  // double header fields
  D_H, D_OCC, D_POLX, D_POLY, D_POLZ, D_AMP, D_OMEGA, D_TTOT, D_RC, D_RCUT, D_CT, D_CDT
};

// 64-bit checksum: FNV-1a over the bytes, fed in any split (the writer and the reader see
// the same byte stream).
struct Checksum {
  uint64_t h = 1469598103934665603ull;
  void add(const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; i++) h = (h ^ b[i]) * 1099511628211ull;
  }
};

struct Writer {
  FILE *f = nullptr;
  Checksum ck;
  bool ok = true;
  void put(const void *p, size_t n) {
    if (!ok || n == 0) return;
    ck.add(p, n);
    ok = std::fwrite(p, 1, n, f) == n;
  }
};

struct Reader {
  FILE *f = nullptr;
  Checksum ck;
  bool ok = true;
  void get(void *p, size_t n) {
    if (!ok || n == 0) return;
    ok = std::fread(p, 1, n, f) == n;
    if (ok) ck.add(p, n);
  }
};

constexpr size_t CHUNK = 64u << 20;  // device <-> host staging per copy

// Device array -> file, through a host buffer of at most CHUNK bytes.
// The ring positions of `count` consecutive records starting at step `from`: at most two
// contiguous spans (the second where the ring wraps); `first` is the span's offset among
// the records.
struct RingSpan {
  long long first, slot, count;
};
std::vector<RingSpan> ring_spans(long long from, long long count) {
  std::vector<RingSpan> out;
  long long done = 0;
  while (done < count) {
    const long long slot = (from + done) % tdks_system::RING;
    const long long n = std::min(count - done, tdks_system::RING - slot);
    out.push_back(RingSpan{done, slot, n});
    done += n;
  }
  return out;
}

int put_device(Writer &w, const void *dev, size_t bytes, cudaStream_t st, std::vector<unsigned char> &buf) {
  buf.resize(std::min(bytes, CHUNK));
  for (size_t off = 0; off < bytes; off += CHUNK) {
    const size_t n = std::min(CHUNK, bytes - off);
    CU(cudaMemcpyAsync(buf.data(), static_cast<const unsigned char *>(dev) + off, n, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    w.put(buf.data(), n);
  }
  return w.ok ? TDKS_OK : fail(TDKS_EINVAL, "checkpoint write failed");
}

int get_device(Reader &r, void *dev, size_t bytes, cudaStream_t st, std::vector<unsigned char> &buf) {
  buf.resize(std::min(bytes, CHUNK));
  for (size_t off = 0; off < bytes; off += CHUNK) {
    const size_t n = std::min(CHUNK, bytes - off);
    r.get(buf.data(), n);
    if (!r.ok) return fail(TDKS_EINVAL, "checkpoint file is truncated");
    CU(cudaMemcpyAsync(static_cast<unsigned char *>(dev) + off, buf.data(), n, cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));
  }
  return TDKS_OK;
}

}  // namespace

extern "C" {

int tdks_save(tdks_sys s, const char *path) {
  if (!s || !path) return fail(TDKS_EINVAL, "NULL argument");
  int rc = TDKS_OK;
  if (s->have_orbitals && (rc = ensure_density(s))) return rc;
  CU(cudaStreamSynchronize(s->stream));
  if ((rc = check_err(s))) return rc;
  const long long n_rec = std::min<long long>(s->steps, tdks_system::RING);
  int64_t hi[NI] = {0};
  double hd[ND] = {0};
  hi[H_NX] = s->nx; hi[H_NY] = s->ny; hi[H_NZ] = s->nz; hi[H_ORDER] = 2 * s->M; hi[H_BC] = s->bc;
  hi[H_PREC] = s->prec; hi[H_NORB] = s->n_orb; hi[H_NK] = s->n_k; hi[H_XC] = s->xc; hi[H_GAUGE] = s->gauge;
  hi[H_ENV] = s->envelope; hi[H_NATOMS] = s->n_atoms; hi[H_PROP] = s->prop;
  hi[H_NHIST] = s->prop != TDKS_PROP_TAYLOR4 ? s->n_hist : 0;
  hi[H_STEPS] = s->steps; hi[H_CSUB] = s->clock_substeps; hi[H_PATH] = s->path;
  hi[H_TX] = s->tx; hi[H_TY] = s->ty; hi[H_ZC] = s->zc;
  for (int i = 0; i < 4; i++) hi[H_WS0 + i] = s->wshape[i];
  hi[H_HAVE] = s->have_orbitals ? 1 : 0;
  hi[H_NREC] = n_rec;
  hd[D_H] = s->h; hd[D_OCC] = s->occ;
  for (int a = 0; a < 3; a++) hd[D_POLX + a] = s->pol[a];
  hd[D_AMP] = s->amp; hd[D_OMEGA] = s->omega; hd[D_TTOT] = s->t_total; hd[D_RC] = s->r_c; hd[D_RCUT] = s->r_cut;
  hd[D_CT] = s->clock_t; hd[D_CDT] = s->clock_dt;

  const std::string tmp = std::string(path) + ".tmp";
  Writer w;
  w.f = std::fopen(tmp.c_str(), "wb");
  if (!w.f) return fail(TDKS_EINVAL, "cannot open " + tmp + " for writing");
  std::vector<unsigned char> buf;
  std::vector<double> vloc(s->N), recs((size_t)n_rec * TDKS_RECORD);
  auto body = [&]() -> int {
    w.put(MAGIC, sizeof MAGIC);
    w.put(hi, sizeof hi);
    w.put(hd, sizeof hd);
    w.put(s->kpts.data(), s->kpts.size() * sizeof(double));
    w.put(s->kw.data(), s->kw.size() * sizeof(double));
    CU(cudaMemcpyAsync(vloc.data(), s->vloc, s->N * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    // records of steps [steps - n_rec, steps), in order: at most two contiguous spans of the ring
    for (const RingSpan &sp : ring_spans(s->steps - n_rec, n_rec))
      CU(cudaMemcpyAsync(recs.data() + sp.first * TDKS_RECORD, s->ring + sp.slot * TDKS_RECORD,
                         sp.count * TDKS_RECORD * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    w.put(vloc.data(), vloc.size() * sizeof(double));
    w.put(s->pos.data(), s->pos.size() * sizeof(double));
    w.put(s->D.data(), s->D.size() * sizeof(double));
    int r;
    if ((r = put_device(w, s->psi, s->state_bytes, s->stream, buf))) return r;
    if (s->psi_lo && (r = put_device(w, s->psi_lo, s->state_bytes, s->stream, buf))) return r;
    if ((r = put_device(w, s->dens_part, (size_t)s->n_kb * s->N * sizeof(double), s->stream, buf))) return r;
    for (int j = 0; j < hi[H_NHIST]; j++)
      if ((r = put_device(w, s->vx_hist[j], (size_t)s->N * sizeof(double), s->stream, buf))) return r;
    w.put(recs.data(), recs.size() * sizeof(double));
    const uint64_t sum = w.ck.h;
    if (w.ok) w.ok = std::fwrite(&sum, sizeof sum, 1, w.f) == 1;
    return w.ok ? TDKS_OK : fail(TDKS_EINVAL, "checkpoint write failed");
  };
  rc = body();
  const bool closed = std::fclose(w.f) == 0;
  if (rc == TDKS_OK && !closed) rc = fail(TDKS_EINVAL, "checkpoint write failed");
  if (rc == TDKS_OK && std::rename(tmp.c_str(), path) != 0) rc = fail(TDKS_EINVAL, std::string("cannot rename to ") + path);
  if (rc != TDKS_OK) std::remove(tmp.c_str());
  return rc;
}

int tdks_load(const char *path, void *stream, tdks_sys *out) {
  if (!path || !out) return fail(TDKS_EINVAL, "NULL argument");
  *out = nullptr;
  Reader r;
  r.f = std::fopen(path, "rb");
  if (!r.f) return fail(TDKS_EINVAL, std::string("cannot open ") + path);
  tdks_sys s = nullptr;
  auto body = [&]() -> int {
    char magic[8];
    int64_t hi[NI];
    double hd[ND];
    r.get(magic, sizeof magic);
    if (!r.ok || std::memcmp(magic, MAGIC, sizeof MAGIC) != 0) return fail(TDKS_EINVAL, "not a checkpoint file");
    r.get(hi, sizeof hi);
    r.get(hd, sizeof hd);
    if (!r.ok) return fail(TDKS_EINVAL, "checkpoint file is truncated");
    const int64_t nk = hi[H_NK], na = hi[H_NATOMS], nrec = hi[H_NREC], nh = hi[H_NHIST];
    if (nk < 1 || nk > (1 << 20) || na < 0 || na > (1 << 20) || nrec < 0 || nrec > tdks_system::RING || nh < 0 ||
        nh > 4 || (nh > 0 && hi[H_PROP] == TDKS_PROP_TAYLOR4) || hi[H_STEPS] < nrec)
      return fail(TDKS_EINVAL, "checkpoint header out of range");
    std::vector<double> kpts(3 * nk), kw(nk);
    r.get(kpts.data(), kpts.size() * sizeof(double));
    r.get(kw.data(), kw.size() * sizeof(double));
    if (!r.ok) return fail(TDKS_EINVAL, "checkpoint file is truncated");
    int rc = tdks_create_grid((int)hi[H_NX], (int)hi[H_NY], (int)hi[H_NZ], hd[D_H], (int)hi[H_ORDER], (int)hi[H_BC],
                              (int)hi[H_PREC], (int)hi[H_NORB], (int)nk, kpts.data(), kw.data(), stream, &s);
    if (rc) return rc;
    std::vector<double> vloc(s->N), pos(3 * na), D(4 * na), recs((size_t)nrec * TDKS_RECORD);
    r.get(vloc.data(), vloc.size() * sizeof(double));
    r.get(pos.data(), pos.size() * sizeof(double));
    r.get(D.data(), D.size() * sizeof(double));
    if (!r.ok) return fail(TDKS_EINVAL, "checkpoint file is truncated");
    if ((rc = tdks_set_local_potential(s, vloc.data()))) return rc;
    if (na > 0 && (rc = tdks_set_atoms_projectors(s, (int)na, pos.data(), D.data(), hd[D_RC], hd[D_RCUT]))) return rc;
    if ((rc = tdks_set_field(s, (int)hi[H_GAUGE], hd + D_POLX, hd[D_AMP], hd[D_OMEGA], (int)hi[H_ENV], hd[D_TTOT])))
      return rc;
    if ((rc = tdks_set_xc(s, (int)hi[H_XC], hd[D_OCC]))) return rc;
    if ((rc = tdks_set_propagator(s, (int)hi[H_PROP]))) return rc;
    if ((rc = tdks_set_tile(s, (int)hi[H_TX], (int)hi[H_TY], (int)hi[H_ZC]))) return rc;
    if ((rc = tdks_set_sweep_path(s, (int)hi[H_PATH]))) return rc;
    for (int i = 0; i < 4; i++)
      if ((rc = tdks_set_sweep_shape(s, i, (int)hi[H_WS0 + i]))) return rc;
    std::vector<unsigned char> buf;
    if ((rc = get_device(r, s->psi, s->state_bytes, s->stream, buf))) return rc;
    if (s->psi_lo && (rc = get_device(r, s->psi_lo, s->state_bytes, s->stream, buf))) return rc;
    if ((rc = get_device(r, s->dens_part, (size_t)s->n_kb * s->N * sizeof(double), s->stream, buf))) return rc;
    for (int j = 0; j < nh; j++)
      if ((rc = get_device(r, s->vx_hist[j], (size_t)s->N * sizeof(double), s->stream, buf))) return rc;
    r.get(recs.data(), recs.size() * sizeof(double));
    uint64_t want = 0;
    const uint64_t got = r.ck.h;
    if (r.ok) r.ok = std::fread(&want, sizeof want, 1, r.f) == 1;
    if (!r.ok) return fail(TDKS_EINVAL, "checkpoint file is truncated");
    if (want != got) return fail(TDKS_EINVAL, "checkpoint checksum mismatch (corrupt file)");
    for (const RingSpan &sp : ring_spans(hi[H_STEPS] - nrec, nrec))
      CU(cudaMemcpyAsync(s->ring + sp.slot * TDKS_RECORD, recs.data() + sp.first * TDKS_RECORD,
                         sp.count * TDKS_RECORD * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    s->n_hist = (int)nh;
    s->steps = hi[H_STEPS];
    s->clock_t = hd[D_CT];
    s->clock_dt = hd[D_CDT];
    s->clock_substeps = (int)hi[H_CSUB];
    s->have_orbitals = hi[H_HAVE] != 0;
    s->dens_valid = s->have_orbitals;
    return TDKS_OK;
  };
  const int rc = body();
  std::fclose(r.f);
  if (rc != TDKS_OK) {
    if (s) tdks_destroy(s);
    return rc;
  }
  *out = s;
  return TDKS_OK;
}

}  // extern "C"
