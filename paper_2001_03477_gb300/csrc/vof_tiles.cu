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


// CTA: 32 x 8 threads covering four tiles along x (32 cells), one along y
// and one along z (the threads walk its 8 planes).  Each tile's flag and
// reference values; integer compares only (no FP64 work and nothing kept
// beyond registers), so the pass streams c and e at the memory's rate.
__device__ __forceinline__ void k_tiles_body(const GridDev& g, const double* __restrict__ c, const double* __restrict__ e, const TileScratch& ts, int ntx, int nty, uint8_t* __restrict__ state, int* __restrict__ counters, const VB vb) {
  __shared__ unsigned uni_w[8];
  __shared__ double ref[4][2];
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int j = tx >> 3;  // tile of this thread within the CTA
  const int x = vb.bx * 32 + tx, y = vb.by * kTile + ty, z0 = vb.bz * kTile;
  const int xt = vb.bx * 4 + j;
  const bool tile_ok = xt * kTile < nx;
  long long cb[kTile], eb[kTile];
  const bool xy_ok = x < nx && y < ny;
#pragma unroll
  for (int zi = 0; zi < kTile; ++zi) {
    const int z = z0 + zi;
    const bool ok = xy_ok && z < nz;
    const size_t id = ((size_t)z * ny + y) * nx + x;
    cb[zi] = ok ? dbits(__ldg(c + id)) : 0;
    eb[zi] = ok ? dbits(__ldg(e + id)) : 0;
    if (ok && state) state[id] = 0;  // the step's frozen-state flags start clear
  }
  if (counters && (vb.bx | vb.by | vb.bz) == 0 && ty == 0 && tx < kStepCounters) counters[tx] = 0;
  // reference of each tile: its first cell, which this CTA's thread
  // (8 j, 0) holds as its first value
  if (ty == 0 && (tx & 7) == 0 && tile_ok) {
    ref[j][0] = __longlong_as_double(cb[0]);
    ref[j][1] = __longlong_as_double(eb[0]);
  }
  __syncthreads();
  const long long cr = tile_ok ? dbits(ref[j][0]) : 0, er = tile_ok ? dbits(ref[j][1]) : 0;
  bool uniform = true;
#pragma unroll
  for (int zi = 0; zi < kTile; ++zi)
    if (xy_ok && z0 + zi < nz) uniform = uniform && cb[zi] == cr && eb[zi] == er;
  const unsigned bal = __ballot_sync(kFullT, uniform);
  if (tx == 0) uni_w[ty] = bal;
  __syncthreads();
  if (ty == 0 && (tx & 7) == 0 && tile_ok) {
    unsigned all = 0xffffffffu;
#pragma unroll
    for (int w = 0; w < 8; ++w) all &= uni_w[w];
    const bool tile_uni = ((all >> (8 * j)) & 0xFFu) == 0xFFu;
    const size_t t = ((size_t)vb.bz * nty + vb.by) * ntx + xt;
    ts.uni[t] = tile_uni ? 1 : 0;
    ts.vc[t] = __longlong_as_double(cr);
    ts.ve[t] = __longlong_as_double(er);
  }
}

__global__ void __launch_bounds__(256)
k_tiles(GridDev g, const double* __restrict__ c, const double* __restrict__ e, TileScratch ts, int ntx, int nty,
        uint8_t* state, int* counters) {
  pdl_wait();
  k_tiles_body(g, c, e, ts, ntx, nty, state, counters, vb_self());
}

// neighbour tile index along one axis: -1 when it lies beyond a
// zero-gradient boundary (the halo repeats the boundary: counts as equal),
// wrapped on a periodic axis
__device__ __forceinline__ int tile_nb(int p, int n, int bc) {
  if (p < 0) return bc ? -1 : p + n;
  if (p >= n) return bc ? -1 : p - n;
  return p;
}

// Sums of c and e over a tile whose cells differ: each lane its cells
// q = lane + 32 r (x fastest within the tile) in order, then the lanes in a
// fixed tree; lane 0 holds the result.  Not inlined and called under a
// warp-uniform branch, so that uniform tiles issue none of its FP64 adds
// (an FP64 instruction costs its full issue time whatever its active lanes).
__device__ __noinline__ double2 tile_cell_sums(int nx, int ny, int nz, const double* __restrict__ c,
                                               const double* __restrict__ e, int x0, int y0, int z0) {
  const int lane = threadIdx.x & 31;
  double sc = 0.0, se = 0.0;
#pragma unroll 4
  for (int r = 0; r < kTile * kTile * kTile / 32; ++r) {
    const int q = lane + 32 * r;
    const int x = x0 + (q & 7), y = y0 + ((q >> 3) & 7), z = z0 + (q >> 6);
    if (x < nx && y < ny && z < nz) {
      const size_t id = ((size_t)z * ny + y) * nx + x;
      sc += __ldg(c + id);
      se += __ldg(e + id);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sc += __shfl_down_sync(kFullT, sc, o);
    se += __shfl_down_sync(kFullT, se, o);
  }
  return make_double2(sc, se);
}

// n x v for the bit pattern v (the same for every lane of the warp): a
// whole tile (n = 512 = 2^9) by adding 9 to the exponent when the product is
// a normal number, and +-0 as itself -- both exact, as the FP64 product is,
// and without an FP64 instruction; otherwise the FP64 product, in a call
// under a warp vote so that the common case issues no predicated multiply
__device__ __noinline__ double times_cells_mul(int n, long long v) { return (double)n * __longlong_as_double(v); }
__device__ __forceinline__ double times_cells(int n, long long v) {
  const int ex = (int)((v >> 52) & 0x7FF);
  const bool shift = n == kTile * kTile * kTile && ex >= 1 && ex <= 0x7FE - 9;
  const bool zero = ((unsigned long long)v << 1) == 0ull;
  double r = __longlong_as_double(shift ? v + (9LL << 52) : v);
  if (__any_sync(kFullT, !shift && !zero)) r = times_cells_mul(n, v);
  return r;
}

// One warp per tile: quiet flag (lanes 0..26 check the tile and its 26
// neighbours at once) and the tile's sum row -- a uniform tile's is
// (cells) x value, another's the sum of its cells.  Rows are placed at
// (tz nty + ty) 4 ceil(ntx / 4) + tx; the slots past the last tile of an
// x-row of tiles hold zero rows.
__device__ __forceinline__ void k_quiet_body(const GridDev& g, const double* __restrict__ c, const double* __restrict__ e, const TileScratch& ts, int ntx, int nty, int ntz, const SumOut& sums, const VB vb) {
  const long long nt = (long long)ntx * nty * ntz;
  const int lane = threadIdx.x & 31;
  const long long wpb = blockDim.x >> 5;
  const int rstride = 4 * ((ntx + 3) / 4);
  // tile t goes to CTA t mod gx: neighbouring tiles (the interface's, whose
  // sums take FP64 adds) spread over the SMs
  for (long long t = vb.bx + (long long)vb.gx * (threadIdx.x >> 5); t < nt; t += (long long)vb.gx * wpb) {
    const int tx = (int)(t % ntx), ty = (int)((t / ntx) % nty), tz = (int)(t / ((long long)ntx * nty));
    // lane o < 27: the tile at offset (o % 3 - 1, o / 3 % 3 - 1, o / 9 - 1);
    // one beyond a zero-gradient boundary counts as equal
    bool nb_ok = true, nb_uni = true;
    long long nb_c = 0, nb_e = 0;
    if (lane < 27) {
      const int px = tile_nb(tx + lane % 3 - 1, ntx, g.bc[0]), py = tile_nb(ty + (lane / 3) % 3 - 1, nty, g.bc[1]),
                pz = tile_nb(tz + lane / 9 - 1, ntz, g.bc[2]);
      nb_ok = (px | py | pz) >= 0;
      if (nb_ok) {
        const size_t u = ((size_t)pz * nty + py) * ntx + px;
        nb_uni = ts.uni[u] != 0;
        nb_c = dbits(ts.vc[u]);
        nb_e = dbits(ts.ve[u]);
      }
    }
    const bool uni = __shfl_sync(kFullT, nb_uni ? 1 : 0, 13) != 0;  // lane 13: the tile itself
    const long long cr = __shfl_sync(kFullT, nb_c, 13), er = __shfl_sync(kFullT, nb_e, 13);
    const bool same = !nb_ok || (nb_uni && nb_c == cr && nb_e == er);
    const bool all = __all_sync(kFullT, lane >= 27 || same);
    const bool q = uni && (cr == 0 || cr == 0x3FF0000000000000LL) && all;
    if (lane == 0) ts.quiet[t] = q ? 1 : 0;
    if (!sums.partials) continue;
    double sc, se;
    if (uni) {
      const int cx = min(kTile, g.n[0] - tx * kTile), cy = min(kTile, g.n[1] - ty * kTile),
                cz = min(kTile, g.n[2] - tz * kTile);
      const int n = cx * cy * cz;
      sc = times_cells(n, cr);
      se = times_cells(n, er);
    } else {
      const double2 s2 = tile_cell_sums(g.n[0], g.n[1], g.n[2], c, e, tx * kTile, ty * kTile, tz * kTile);
      sc = s2.x;
      se = s2.y;
    }
    const size_t slot = ((size_t)tz * nty + ty) * rstride + tx;
    if (lane == 0) {
      double* row = sums.partials + slot * sums.stride;
      row[kSumC] = sc;
      row[kSumE] = se;
      row[kSumClip] = 0.0;
      row[kSumShDc] = 0.0;
      row[kSumUnpl] = 0.0;
      row[kSumShDe] = 0.0;
    }
    if (tx == ntx - 1 && lane >= 1 && lane < rstride - ntx + 1) {
      // zero rows of the slots past the row's last tile
      double* row = sums.partials + (slot + lane) * sums.stride;
      for (int k = 0; k < kNSums; ++k) row[k] = 0.0;
    }
  }
}

__global__ void __launch_bounds__(256)
k_quiet(GridDev g, const double* __restrict__ c, const double* __restrict__ e, TileScratch ts, int ntx, int nty,
        int ntz, SumOut sums) {
  pdl_wait();
  k_quiet_body(g, c, e, ts, ntx, nty, ntz, sums, vb_self());
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
  __shared__ TileArgs sA;
  const TileArgs& A = cta_args(args, b, sA);
  k_tiles_body(A.g, A.c, A.e, A.ts, A.nt[0], A.nt[1], A.state, A.counters, vb);
}
__global__ void __launch_bounds__(256) k_quiet_grp(GroupMap m, const TileArgs* __restrict__ args) {
  unsigned b;
  const VB vb = vb_group(m, b);
  __shared__ TileArgs sA;
  const TileArgs& A = cta_args(args, b, sA);
  k_quiet_body(A.g, A.c, A.e, A.ts, A.nt[0], A.nt[1], A.nt[2], A.sums, vb);
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
  // one warp per tile, 8 per CTA
  return (unsigned)((T + 7) / 8 < 152 * 8 ? (T + 7) / 8 : 152 * 8);
}

cudaError_t launch_tiles(const GridDev& g, const double* c, const double* e, TileScratch ts, SumOut sums,
                         uint8_t* state, int* counters, cudaStream_t st) {
  int nt[3];
  tile_counts(g, nt);
  launch_pdl(k_tiles, dim3((unsigned)((nt[0] + 3) / 4), (unsigned)nt[1], (unsigned)nt[2]), dim3(32, 8), st,
             g, c, e, ts, nt[0], nt[1], state, counters);
  prof_mark("tiles", st);
  launch_pdl(k_quiet, quiet_blocks(g), 256, st, g, c, e, ts, nt[0], nt[1], nt[2], sums);
  prof_mark("tiles.quiet", st);
  return cudaGetLastError();
}

}  // namespace vofgb
