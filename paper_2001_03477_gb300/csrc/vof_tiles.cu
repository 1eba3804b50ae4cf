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

// Sums of the tiles that are not uniform.  These helpers are not inlined
// and are called under warp-uniform branches, so that the compiler cannot
// turn a branch into predicated FP64 adds that every warp would issue (an
// FP64 instruction costs its full issue time whatever its active lanes; a
// by-value form was measured to lose the branch).
//
// this thread's 8 cells, then over the 8 lanes of its tile's x-row (lane 8j
// of the warp ends with the row's sums); every lane of the warp calls it
__device__ __noinline__ void tile_row_sums(const double (&cv)[kTile], const double (&ev)[kTile], bool on,
                                           double (&s)[2]) {
  double sc = 0.0, se = 0.0;
  if (on) {
#pragma unroll
    for (int zi = 0; zi < kTile; ++zi) {
      sc += cv[zi];
      se += ev[zi];
    }
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    sc += __shfl_down_sync(kFullT, sc, o, 8);
    se += __shfl_down_sync(kFullT, se, o, 8);
  }
  s[0] = sc;
  s[1] = se;
}
// the 8 rows of a tile (its y extent), from shared memory, in order
__device__ __noinline__ void tile_sum_rows(const double (*rows)[2], double (&s)[2]) {
  double sc = 0.0, se = 0.0;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    sc += rows[r][0];
    se += rows[r][1];
  }
  s[0] = sc;
  s[1] = se;
}

// CTA: 32 x 8 threads covering four tiles along x (32 cells), one along y
// and one along z (the threads walk its 8 planes).  Each tile writes one
// sum row (4 rows per CTA): a uniform tile (cells) x value, another its
// cells' sum (threads over z, lanes over x, warps over y).
__device__ __forceinline__ void k_tiles_body(const GridDev& g, const double* __restrict__ c, const double* __restrict__ e, const TileScratch& ts, int ntx, int nty, const SumOut& sums, uint8_t* __restrict__ state, int* __restrict__ counters, const VB vb) {
  __shared__ unsigned uni_w[8];
  __shared__ double ref[4][2];
  __shared__ double rows[4][8][2];  // non-uniform tiles: [tile][y row][c, e]
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
  // non-uniform tiles: each warp's x-row sums into shared memory
  const bool add_cells = tile_ok && !tile_uni && xy_ok;
  const bool warp_adds = __any_sync(kFullT, tile_ok && !tile_uni);
  if (warp_adds) {
    double rs[2];
    tile_row_sums(cv, ev, add_cells, rs);
    if ((tx & 7) == 0) {
      rows[j][ty][0] = rs[0];
      rows[j][ty][1] = rs[1];
    }
  }
  __syncthreads();
  if (ty == 0 && (tx & 7) == 0) {
    const size_t t = ((size_t)vb.bz * nty + vb.by) * ntx + xt;
    double sc = 0.0, se = 0.0;  // a slot beyond the grid: a zero row
    if (!tile_ok) {
    } else if (tile_uni) {
      const int cx = min(kTile, nx - xt * kTile), cy = min(kTile, ny - (int)vb.by * kTile),
                cz = min(kTile, nz - z0);
      const double n = (double)(cx * cy * cz);
      sc = n * cr;
      se = n * er;
      ts.uni[t] = 1;
      ts.vc[t] = cr;
      ts.ve[t] = er;
    } else {
      ts.uni[t] = 0;
      double s2[2];
      tile_sum_rows(rows[j], s2);  // rows beyond ny hold 0
      sc = s2[0];
      se = s2[1];
    }
    if (sums.partials) {
      double* row = sums.partials + ((size_t)(vb.bx + vb.gx * (vb.by + vb.gy * vb.bz)) * 4 + j) * sums.stride;
      row[kSumC] = sc;
      row[kSumE] = se;
      row[kSumClip] = 0.0;
      row[kSumShDc] = 0.0;
      row[kSumUnpl] = 0.0;
      row[kSumShDe] = 0.0;
    }
  }
}

__global__ void __launch_bounds__(256)
k_tiles(GridDev g, const double* __restrict__ c, const double* __restrict__ e,
                                               TileScratch ts, int ntx, int nty, SumOut sums, uint8_t* state,
                                               int* counters) {
  k_tiles_body(g, c, e, ts, ntx, nty, sums, state, counters, vb_self());
}

// neighbour tile index along one axis: -1 when it lies beyond a
// zero-gradient boundary (the halo repeats the boundary: counts as equal),
// wrapped on a periodic axis
__device__ __forceinline__ int tile_nb(int p, int n, int bc) {
  if (p < 0) return bc ? -1 : p + n;
  if (p >= n) return bc ? -1 : p - n;
  return p;
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
    if (q) {
      // the 26 neighbours' flags and values, loaded independently (no
      // early exit: one round trip instead of a chain of 26)
      bool all = true;
#pragma unroll
      for (int o = 0; o < 27; ++o) {
        if (o == 13) continue;
        const int px = tile_nb(tx + o % 3 - 1, ntx, g.bc[0]), py = tile_nb(ty + (o / 3) % 3 - 1, nty, g.bc[1]),
                  pz = tile_nb(tz + o / 9 - 1, ntz, g.bc[2]);
        if ((px | py | pz) < 0) continue;
        const size_t u = ((size_t)pz * nty + py) * ntx + px;
        all = all & (ts.uni[u] != 0) & same_bits_t(ts.vc[u], cr) & same_bits_t(ts.ve[u], er);
      }
      q = all;
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

// sum rows of the tile pass: 4 per CTA (one per tile slot along x)
int tile_blocks(const GridDev& g) {
  int nt[3];
  tile_counts(g, nt);
  return ((nt[0] + 3) / 4) * nt[1] * nt[2] * 4;
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
