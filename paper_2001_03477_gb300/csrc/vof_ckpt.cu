// vof_ckpt.cu -- checkpoint and resume of the state of a run (host code;
// the paper has no counterpart): the grid, the step index, the time and
// the two fields c and e, in one little-endian binary file.
//
// Layout: the 8-byte magic "VOFGBCK1", a fixed header (format version,
// header size, grid, step, time, cell count), c[N] and e[N] as doubles, then
// an FNV-1a 64-bit checksum of everything before it.  The file is written to
// a temporary name and renamed into place, so a crash mid-write leaves the
// previous checkpoint intact.  Loading checks the magic, the version, the
// sizes and the checksum before it copies anything out.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/vofgb.h"

namespace {

constexpr char kMagic[8] = {'V', 'O', 'F', 'G', 'B', 'C', 'K', '1'};
constexpr uint32_t kVersion = 1;

#pragma pack(push, 1)
struct CkptHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int32_t n[3];
  int32_t bc[3];
  int32_t precision;
  int32_t scheme;
  double h, Cp_l, Cp_g, T_sat, eps_mixed;
  int64_t step;
  double t;
  uint64_t cells;
};
#pragma pack(pop)

uint64_t fnv1a(const void* data, size_t n, uint64_t h) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

constexpr uint64_t kFnvBasis = 14695981039346656037ull;

bool little_endian() {
  const uint16_t one = 1;
  unsigned char b;
  std::memcpy(&b, &one, 1);
  return b == 1;
}

}  // namespace

extern "C" {

vof_status vof_checkpoint_save(const char* path, const vof_grid* g, const double* c, const double* e, long step,
                               double t) {
  if (!path || !g || !c || !e || !little_endian()) return VOF_EINVAL;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return VOF_EINVAL;
  const uint64_t N = (uint64_t)g->nx * g->ny * g->nz;
  CkptHeader hd;
  std::memset(&hd, 0, sizeof hd);
  std::memcpy(hd.magic, kMagic, 8);
  hd.version = kVersion;
  hd.header_bytes = sizeof(CkptHeader);
  hd.n[0] = g->nx; hd.n[1] = g->ny; hd.n[2] = g->nz;
  for (int a = 0; a < 3; ++a) hd.bc[a] = g->bc[a];
  hd.precision = g->precision;
  hd.scheme = g->scheme;
  hd.h = g->h; hd.Cp_l = g->Cp_l; hd.Cp_g = g->Cp_g; hd.T_sat = g->T_sat; hd.eps_mixed = g->eps_mixed;
  hd.step = step;
  hd.t = t;
  hd.cells = N;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return VOF_EINVAL;
  uint64_t sum = fnv1a(&hd, sizeof hd, kFnvBasis);
  sum = fnv1a(c, N * sizeof(double), sum);
  sum = fnv1a(e, N * sizeof(double), sum);
  bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1 && std::fwrite(c, sizeof(double), N, f) == N &&
            std::fwrite(e, sizeof(double), N, f) == N && std::fwrite(&sum, sizeof sum, 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return VOF_EINVAL;
  }
  return VOF_OK;
}

vof_status vof_checkpoint_info(const char* path, vof_grid* g, long* step, double* t) {
  if (!path || !g || !little_endian()) return VOF_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return VOF_EINVAL;
  CkptHeader hd;
  const bool ok = std::fread(&hd, sizeof hd, 1, f) == 1;
  std::fclose(f);
  if (!ok || std::memcmp(hd.magic, kMagic, 8) != 0 || hd.version != kVersion || hd.header_bytes != sizeof hd)
    return VOF_EINVAL;
  if (hd.n[0] < 1 || hd.n[1] < 1 || hd.n[2] < 1 || hd.cells != (uint64_t)hd.n[0] * hd.n[1] * hd.n[2])
    return VOF_EINVAL;
  g->nx = hd.n[0]; g->ny = hd.n[1]; g->nz = hd.n[2];
  for (int a = 0; a < 3; ++a) g->bc[a] = hd.bc[a];
  g->precision = hd.precision;
  g->scheme = hd.scheme;
  g->h = hd.h; g->Cp_l = hd.Cp_l; g->Cp_g = hd.Cp_g; g->T_sat = hd.T_sat; g->eps_mixed = hd.eps_mixed;
  // the network parameters of a learned-normal run are not in the file
  g->normal = VOF_NORMAL_MYC;
  g->mlp = nullptr;
  if (step) *step = (long)hd.step;
  if (t) *t = hd.t;
  return VOF_OK;
}

vof_status vof_checkpoint_load(const char* path, size_t cells, double* c, double* e) {
  if (!path || !c || !e || !little_endian()) return VOF_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return VOF_EINVAL;
  CkptHeader hd;
  bool ok = std::fread(&hd, sizeof hd, 1, f) == 1 && std::memcmp(hd.magic, kMagic, 8) == 0 &&
            hd.version == kVersion && hd.header_bytes == sizeof hd && hd.cells == (uint64_t)cells &&
            hd.n[0] >= 1 && hd.n[1] >= 1 && hd.n[2] >= 1 &&
            hd.cells == (uint64_t)hd.n[0] * hd.n[1] * hd.n[2];
  std::vector<double> bc_, be_;
  uint64_t stored = 0;
  if (ok) {
    bc_.resize(cells);
    be_.resize(cells);
    ok = std::fread(bc_.data(), sizeof(double), cells, f) == cells &&
         std::fread(be_.data(), sizeof(double), cells, f) == cells && std::fread(&stored, sizeof stored, 1, f) == 1;
    unsigned char extra;
    ok = ok && std::fread(&extra, 1, 1, f) == 0;  // nothing after the checksum
  }
  std::fclose(f);
  if (!ok) return VOF_EINVAL;
  uint64_t sum = fnv1a(&hd, sizeof hd, kFnvBasis);
  sum = fnv1a(bc_.data(), cells * sizeof(double), sum);
  sum = fnv1a(be_.data(), cells * sizeof(double), sum);
  if (sum != stored) return VOF_EINVAL;
  std::memcpy(c, bc_.data(), cells * sizeof(double));
  std::memcpy(e, be_.data(), cells * sizeof(double));
  return VOF_OK;
}

}  // extern "C"
