// Checkpoint and resume of a tracked bunch (host code only; the paper has no
// counterpart, but its runs reach ~5e5 turns, so a run must be able to stop
// and go on).  Resuming is bit-exact: the state is written as the raw float64
// bits, tracking is deterministic (integer charge, fixed reduction orders)
// and a captured turn depends only on the state, the beam and the lattice,
// which the file records (the beam bit for bit, the lattice by a hash).
//
// File layout (little-endian, as both hosts of this library are):
//   magic "SCCKPT" 0 1 (8 bytes), u32 version = 1, u32 zero,
//   i64 n, i64 turn, sc_beam (6 float64), u64 lattice hash,
//   x, px, y, py, sigma, psigma (n float64 each),
//   u64 checksum of every byte before it.
// Hashes: 64-bit FNV-1a (offset basis 0xcbf29ce484222325, prime 0x100000001b3).
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sc_internal.cuh"

namespace sc {
namespace {

constexpr unsigned char kMagic[8] = {'S', 'C', 'C', 'K', 'P', 'T', 0, 1};
constexpr uint32_t kVersion = 1;
constexpr uint64_t kFnvBasis = 0xcbf29ce484222325ull, kFnvPrime = 0x100000001b3ull;

struct Header {
  unsigned char magic[8];
  uint32_t version, zero;
  int64_t n, turn;
  sc_beam beam;
  uint64_t lattice_hash;
};
static_assert(sizeof(Header) == 8 + 4 + 4 + 8 + 8 + 48 + 8, "packed header");

uint64_t fnv1a(uint64_t h, const void* data, size_t bytes) {
  const unsigned char* c = (const unsigned char*)data;
  for (size_t k = 0; k < bytes; ++k) h = (h ^ c[k]) * kFnvPrime;
  return h;
}

uint64_t lattice_hash(const sc_element* lattice, int n_elems) {
  const int64_t n = n_elems;
  uint64_t h = fnv1a(kFnvBasis, &n, sizeof n);
  return n_elems > 0 ? fnv1a(h, lattice, (size_t)n_elems * sizeof(sc_element)) : h;
}

sc_status check_host_bunch(const sc_particles* p) {
  if (!p) return set_error(SC_ERR_ARG, "particles is NULL");
  if (p->n <= 0) return set_error(SC_ERR_ARG, "a checkpoint needs at least one particle");
  if (!p->x || !p->px || !p->y || !p->py || !p->sigma || !p->psigma)
    return set_error(SC_ERR_ARG, "particle array pointer is NULL");
  return SC_OK;
}

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};

}  // namespace
}  // namespace sc

extern "C" sc_status sc_checkpoint_write(const char* path, const sc_particles* host, int64_t turn, const sc_beam* b,
                                         const sc_element* lattice, int n_elems) {
  using namespace sc;
  if (!path || !b) return set_error(SC_ERR_ARG, "path or beam is NULL");
  sc_status st = check_host_bunch(host);
  if (st) return st;
  if (n_elems < 0 || (n_elems > 0 && !lattice)) return set_error(SC_ERR_ARG, "bad element list");
  Header hd;
  std::memset(&hd, 0, sizeof hd);
  std::memcpy(hd.magic, kMagic, sizeof kMagic);
  hd.version = kVersion;
  hd.n = host->n;
  hd.turn = turn;
  hd.beam = *b;
  hd.lattice_hash = lattice_hash(lattice, n_elems);
  const std::string tmp = std::string(path) + ".tmp";
  uint64_t sum = fnv1a(kFnvBasis, &hd, sizeof hd);
  {
    File out;
    out.f = std::fopen(tmp.c_str(), "wb");
    if (!out.f) return set_error(SC_ERR_ARG, "cannot open " + tmp + " for writing");
    bool ok = std::fwrite(&hd, sizeof hd, 1, out.f) == 1;
    const double* arr[6] = {host->x, host->px, host->y, host->py, host->sigma, host->psigma};
    for (int a = 0; a < 6 && ok; ++a) {
      ok = std::fwrite(arr[a], sizeof(double), (size_t)host->n, out.f) == (size_t)host->n;
      sum = fnv1a(sum, arr[a], (size_t)host->n * sizeof(double));
    }
    ok = ok && std::fwrite(&sum, sizeof sum, 1, out.f) == 1;
    const int closed = std::fclose(out.f);
    out.f = nullptr;
    if (!ok || closed != 0) {
      std::remove(tmp.c_str());
      return set_error(SC_ERR_ARG, "writing " + tmp + " failed");
    }
  }
  // the finished file replaces any previous checkpoint in one step
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return set_error(SC_ERR_ARG, std::string("cannot rename the checkpoint to ") + path);
  }
  return SC_OK;
}

extern "C" sc_status sc_checkpoint_read(const char* path, const sc_particles* host, int64_t* turn, const sc_beam* b,
                                        const sc_element* lattice, int n_elems) {
  using namespace sc;
  if (!path || !b) return set_error(SC_ERR_ARG, "path or beam is NULL");
  sc_status st = check_host_bunch(host);
  if (st) return st;
  if (n_elems < 0 || (n_elems > 0 && !lattice)) return set_error(SC_ERR_ARG, "bad element list");
  File in;
  in.f = std::fopen(path, "rb");
  if (!in.f) return set_error(SC_ERR_ARG, std::string("cannot open ") + path);
  Header hd;
  if (std::fread(&hd, sizeof hd, 1, in.f) != 1 || std::memcmp(hd.magic, kMagic, sizeof kMagic) != 0)
    return set_error(SC_ERR_ARG, std::string(path) + " is not a checkpoint of this library");
  if (hd.version != kVersion) return set_error(SC_ERR_ARG, "unsupported checkpoint version");
  if (hd.n != host->n)
    return set_error(SC_ERR_ARG, "the checkpoint holds " + std::to_string(hd.n) + " particles, the bunch " +
                                     std::to_string(host->n));
  if (std::memcmp(&hd.beam, b, sizeof(sc_beam)) != 0)
    return set_error(SC_ERR_ARG, "the checkpoint was written with other beam constants");
  if (hd.lattice_hash != lattice_hash(lattice, n_elems))
    return set_error(SC_ERR_ARG, "the checkpoint was written with another lattice");
  // first pass: the checksum over the whole file, so that a damaged file
  // leaves the caller's arrays untouched
  const size_t body = (size_t)hd.n * 6 * sizeof(double);
  uint64_t sum = fnv1a(kFnvBasis, &hd, sizeof hd);
  std::vector<unsigned char> buf(size_t(1) << 20);
  for (size_t done = 0; done < body;) {
    const size_t want = body - done < buf.size() ? body - done : buf.size();
    if (std::fread(buf.data(), 1, want, in.f) != want) return set_error(SC_ERR_ARG, "the checkpoint is truncated");
    sum = fnv1a(sum, buf.data(), want);
    done += want;
  }
  uint64_t stored = 0;
  if (std::fread(&stored, sizeof stored, 1, in.f) != 1) return set_error(SC_ERR_ARG, "the checkpoint is truncated");
  if (std::fgetc(in.f) != EOF) return set_error(SC_ERR_ARG, "the checkpoint has trailing bytes");
  if (stored != sum) return set_error(SC_ERR_ARG, "the checkpoint's checksum does not match its contents");
  // second pass: the state into the caller's arrays
  if (std::fseek(in.f, (long)sizeof hd, SEEK_SET) != 0) return set_error(SC_ERR_ARG, "cannot seek in the checkpoint");
  double* arr[6] = {host->x, host->px, host->y, host->py, host->sigma, host->psigma};
  for (int a = 0; a < 6; ++a)
    if (std::fread(arr[a], sizeof(double), (size_t)hd.n, in.f) != (size_t)hd.n)
      return set_error(SC_ERR_ARG, "the checkpoint changed while it was read");
  if (turn) *turn = hd.turn;
  return SC_OK;
}
