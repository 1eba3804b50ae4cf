// vof_tiles.cu -- the tile pass at the start of an in-place time step: which
// 8^3 tiles are quiet (no cell of them can change in this step, so the
// streaming kernels skip them), and the sums of c and e over the grid.
//
// A tile is uniform when all its cells hold the same (c, e) bits; it is quiet
// when it is uniform with c exactly 0 or 1 and every one of its 26 neighbour
// tiles is uniform with the same bits.  The neighbours then contain the 3-cell
// halo of the tile, so every 7-cell sweep window of a tile cell, and every
// window the earlier sweeps of the step use for the cells those windows
// reach, sees one value: the cells are no-ops in all three sweeps (a cell
// that does not change is not marked in the frozen state either) and remain
// pure for the shift.  Beyond a zero-gradient boundary the halo repeats the
// boundary cells, so a missing neighbour tile counts as equal; a periodic
// axis wraps.  On a periodic axis whose last tile holds fewer than 3 cells
// the halo can reach two tiles away, and no tile is skipped (tiles_usable).
#include "vof_launch.h"
#include "vof_sums.cuh"

namespace vofgb {

namespace {

constexpr unsigned kFullT = 0xffffffffu;

__device__ __forceinline__ bool same_bits_t(double a, double b) { return dbits(a) == dbits(b); }

__device__ __noinline__ void add_tile_cells(const double (&cv)[kTile], const double (&ev)[kTile], bool on,
                                           double (&v)[kNSums]) {
  if (!on) return;
#pragma unroll
  for (int zi = 0; zi < kTile; ++zi) {
    v[kSumC] += cv[zi];
    v[kSumE] += ev[zi];
  }
}

// CTA: 32 x 8 threads covering four tiles along x (32 cells), one along y
// and one along z (the threads walk its 8 planes).
__device__ __forceinline__ void k_tiles_body(const GridDev& g, const double* __restrict__ c, const double* __restrict__ e, const TileScratch& ts, int ntx, int nty, const SumOut& sums, uint8_t* __restrict__ state, int* __restrict__ counters, const VB vb) {
  __shared__ unsigned uni_w[8];
  __shared__ double ref[4][2];
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int j = tx >> 3;  // tile of this thread within the CTA
  const int x = vb.bx * 32 + tx, y = vb.by * kTile + ty, z0 = vb.bz * kTile;
  const int xt = vb.bx * 4 + j;
  const bool tile_ok = xt * kTile < nx;
  double cv[kTile], ev[kTile];
  const bool xy_ok = x < nx && y < ny;
#pragma unroll
  for (int zi = 0; zi < kTile; ++zi) {
    const int z = z0 + zi;
    const bool ok = xy_ok && z < nz;
    const size_t id = ((size_t)z * ny + y) * nx + x;
    cv[zi] = ok ? __ldg(c + id) : 0.0;
    ev[zi] = ok ? __ldg(e + id) : 0.0;
    if (ok && state) state[id] = 0;  // the step's frozen-state flags start clear
  }
  if (counters && (vb.bx | vb.by | vb.bz) == 0 && ty == 0 && tx < kStepCounters) counters[tx] = 0;
  // reference of each tile: its first cell, which this CTA's thread
  // (8 j, 0) holds as its first value
  if (ty == 0 && (tx & 7) == 0 && tile_ok) {
    ref[j][0] = cv[0];
    ref[j][1] = ev[0];
  }
  __syncthreads();
  const double cr = tile_ok ? ref[j][0] : 0.0, er = tile_ok ? ref[j][1] : 0.0;
  bool uniform = true;
#pragma unroll
  for (int zi = 0; zi < kTile; ++zi)
    if (xy_ok && z0 + zi < nz) uniform = uniform && same_bits_t(cv[zi], cr) && same_bits_t(ev[zi], er);
  const unsigned b = __ballot_sync(kFullT, uniform);
  if (tx == 0) uni_w[ty] = b;
  __syncthreads();
  unsigned all = 0xffffffffu;
#pragma unroll
  for (int w = 0; w < 8; ++w) all &= uni_w[w];
  const bool tile_uni = ((all >> (8 * j)) & 0xFFu) == 0xFFu;
  double v[kNSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (tile_ok) {
    if (tile_uni) {
      // one thread per tile: (cells of the tile) x value
      if (ty == 0 && (tx & 7) == 0) {
        const int cx = min(kTile, nx - xt * kTile), cy = min(kTile, ny - (int)vb.by * kTile),
                  cz = min(kTile, nz - z0);
        const double n = (double)(cx * cy * cz);
        v[kSumC] = n * cr;
        v[kSumE] = n * er;
        const size_t t = ((size_t)vb.bz * nty + vb.by) * ntx + xt;
        ts.uni[t] = 1;
        ts.vc[t] = cr;
        ts.ve[t] = er;
      }
    } else if (ty == 0 && (tx & 7) == 0) {
      ts.uni[((size_t)vb.bz * nty + vb.by) * ntx + xt] = 0;
    }
  }
  // cell by cell only in the tiles that are not uniform; the branch is
  // taken per warp so that the adds are not executed (predicated) for the
  // uniform majority -- an FP64 add costs ~80 cycles of the SM partition's
  // FP64 unit per warp on this part
  const bool add_cells = tile_ok && !tile_uni && xy_ok;
  if (__any_sync(kFullT, add_cells)) add_tile_cells(cv, ev, add_cells, v);

  block_sums(v, sums, vb.bx + vb.gx * (vb.by + vb.gy * vb.bz));
}

__global__ void __launch_bounds__(256)
k_tiles(GridDev g, const double* __restrict__ c, const double* __restrict__ e,
                                               TileScratch ts, int ntx, int nty, SumOut sums, uint8_t* state,
                                               int* counters) {
  k_tiles_body(g, c, e, ts, ntx, nty, sums, state, counters, vb_self());
}

__device__ __forceinline__ void k_quiet_body(const GridDev& g, const TileScratch& ts, int ntx, int nty, int ntz, const VB vb) {
  const long long nt = (long long)ntx * nty * ntz;
  for (long long t = vb.bx * (long long)blockDim.x + threadIdx.x; t < nt; t += (long long)vb.gx * blockDim.x) {
    const int tx = (int)(t % ntx), ty = (int)((t / ntx) % nty), tz = (int)(t / ((long long)ntx * nty));
    bool q = ts.uni[t] != 0;
    double cr = 0.0, er = 0.0;
    if (q) {
      cr = ts.vc[t];
      er = ts.ve[t];
      const long long cb = dbits(cr);
      q = cb == 0 || cb == 0x3FF0000000000000LL;
    }
    const int ntv[3] = {ntx, nty, ntz};
    for (int oz = -1; oz <= 1 && q; ++oz)
      for (int oy = -1; oy <= 1 && q; ++oy)
        for (int ox = -1; ox <= 1 && q; ++ox) {
          if (!ox && !oy && !oz) continue;
          int p[3] = {tx + ox, ty + oy, tz + oz};
          bool skip = false;
          for (int a = 0; a < 3; ++a) {
            if (p[a] < 0 || p[a] >= ntv[a]) {
              if (g.bc[a] != 0) skip = true;  // zero-gradient: the halo repeats the boundary
              else p[a] = (p[a] + ntv[a]) % ntv[a];
            }
          }
          if (skip) continue;
          const size_t u = ((size_t)p[2] * nty + p[1]) * ntx + p[0];
          q = ts.uni[u] != 0 && same_bits_t(ts.vc[u], cr) && same_bits_t(ts.ve[u], er);
        }
    ts.quiet[t] = q ? 1 : 0;
  }
}

__global__ void __launch_bounds__(256)
k_quiet(GridDev g, TileScratch ts, int ntx, int nty, int ntz) {
  k_quiet_body(g, ts, ntx, nty, ntz, vb_self());
}

size_t al256t(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

void tile_counts(const GridDev& g, int nt[3]) {
  for (int a = 0; a < 3; ++a) nt[a] = (g.n[a] + kTile - 1) / kTile;
}

bool tiles_usable(const GridDev& g) {
  for (int a = 0; a < 3; ++a) {
    const int r = g.n[a] % kTile;
    if (g.bc[a] == 0 && (r == 1 || r == 2) && g.n[a] > 2 * kTile) return false;
  }
  return true;
}

int tile_blocks(const GridDev& g) {
  int nt[3];
  tile_counts(g, nt);
  return ((nt[0] + 3) / 4) * nt[1] * nt[2];
}

size_t tile_scratch_bytes(const GridDev& g) {
  int nt[3];
  tile_counts(g, nt);
  const size_t T = (size_t)nt[0] * nt[1] * nt[2];
  return al256t(T) + al256t(T * 8) + al256t(T * 8) + al256t(T);
}

TileScratch carve_tile_scratch(const GridDev& g, void* ws) {
  int nt[3];
  tile_counts(g, nt);
  const size_t T = (size_t)nt[0] * nt[1] * nt[2];
  char* b = static_cast<char*>(ws);
  TileScratch s;
  s.uni = reinterpret_cast<uint8_t*>(b);   b += al256t(T);
  s.vc = reinterpret_cast<double*>(b);     b += al256t(T * 8);
  s.ve = reinterpret_cast<double*>(b);     b += al256t(T * 8);
  s.quiet = reinterpret_cast<uint8_t*>(b);
  return s;
}

__global__ void __launch_bounds__(256) k_tiles_grp(GroupMap m, const TileArgs* __restrict__ args) {
  unsigned b;
  const VB vb = vb_group(m, b);
  const TileArgs A = args[b];
  k_tiles_body(A.g, A.c, A.e, A.ts, A.nt[0], A.nt[1], A.sums, A.state, A.counters, vb);
}
__global__ void __launch_bounds__(256) k_quiet_grp(GroupMap m, const TileArgs* __restrict__ args) {
  unsigned b;
  const VB vb = vb_group(m, b);
  const TileArgs A = args[b];
  k_quiet_body(A.g, A.ts, A.nt[0], A.nt[1], A.nt[2], vb);
}

cudaError_t launch_tiles_grp(const GroupMap& mt, const GroupMap& mq, const TileArgs* a, unsigned ct, unsigned cq,
                             cudaStream_t st) {
  if (ct) k_tiles_grp<<<ct, dim3(32, 8), 0, st>>>(mt, a);
  prof_mark("group.tiles", st);
  if (cq) k_quiet_grp<<<cq, 256, 0, st>>>(mq, a);
  prof_mark("group.quiet", st);
  return cudaGetLastError();
}

unsigned quiet_blocks(const GridDev& g) {
  int nt[3];
  tile_counts(g, nt);
  const long long T = (long long)nt[0] * nt[1] * nt[2];
  return (unsigned)((T + 255) / 256 < 152 * 8 ? (T + 255) / 256 : 152 * 8);
}

cudaError_t launch_tiles(const GridDev& g, const double* c, const double* e, TileScratch ts, SumOut sums,
                         uint8_t* state, int* counters, cudaStream_t st) {
  int nt[3];
  tile_counts(g, nt);
  k_tiles<<<dim3((unsigned)((nt[0] + 3) / 4), (unsigned)nt[1], (unsigned)nt[2]), dim3(32, 8), 0, st>>>(
      g, c, e, ts, nt[0], nt[1], sums, state, counters);
  prof_mark("tiles", st);
  k_quiet<<<quiet_blocks(g), 256, 0, st>>>(g, ts, nt[0], nt[1], nt[2]);
  prof_mark("tiles.quiet", st);
  return cudaGetLastError();
}

}  // namespace vofgb
