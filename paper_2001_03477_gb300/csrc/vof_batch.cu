// vof_batch.cu -- many independent subdomains stepped together (host code).
//
// The paper steps one domain.  Workloads made of thousands of small, uneven
// domains (separate droplets, each in its own periodic box) leave most of
// the GPU idle when their steps run one after the other: a 24^3 box fills a
// few dozen CTAs.  Here each box is still one vof_step() -- the same
// kernels, sums and results as a call of its own -- but the boxes are spread
// over several streams ("lanes") that the GPU runs concurrently, joined back
// into the caller's stream by events.  Under stream capture the lanes become
// parallel branches of one CUDA graph, so a replay issues every box's
// kernels without the host.
//
// Lane assignment is longest-processing-time first by cell count, which
// keeps the lanes' loads within one box of each other; each lane reuses one
// step workspace sized for its largest box, since its boxes run in order.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/vofgb.h"
#include "vof_launch.h"

namespace {

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t box_cells(const vof_box& b) { return (size_t)b.grid.nx * b.grid.ny * b.grid.nz; }

struct Plan {
  std::vector<int> lane;        // lane of each box
  std::vector<int> order;       // boxes in queueing order (decreasing cells, then index)
  std::vector<size_t> offset;   // workspace offset of each lane
  size_t total = 0;
};

// Checks the boxes' grids (through vof_step_workspace_bytes) and builds the
// plan; false for a bad argument.
bool make_plan(const vof_box* boxes, int nbox, int lanes, Plan* p) {
  if (nbox < 0 || lanes < 1 || (nbox > 0 && !boxes)) return false;
  std::vector<size_t> ws(nbox), n(nbox);
  for (int b = 0; b < nbox; ++b) {
    ws[b] = vof_step_workspace_bytes(&boxes[b].grid);
    if (ws[b] == 0) return false;
    n[b] = box_cells(boxes[b]);
  }
  p->order.resize(nbox);
  std::iota(p->order.begin(), p->order.end(), 0);
  std::stable_sort(p->order.begin(), p->order.end(), [&](int a, int b) { return n[a] > n[b]; });
  p->lane.assign(nbox, 0);
  std::vector<unsigned long long> load(lanes, 0);
  std::vector<size_t> need(lanes, 0);
  for (int b : p->order) {
    int best = 0;
    for (int l = 1; l < lanes; ++l)
      if (load[l] < load[best]) best = l;
    p->lane[b] = best;
    load[best] += n[b];
    need[best] = std::max(need[best], ws[b]);
  }
  p->offset.assign(lanes, 0);
  size_t off = 0;
  for (int l = 0; l < lanes; ++l) {
    p->offset[l] = off;
    off += align256(need[l]);
  }
  p->total = off;
  return true;
}

struct Span {
  const char* lo;
  const char* hi;
};

// true when two of the spans overlap: in order of their starts, a span
// overlaps an earlier one exactly when it starts before the furthest end
// seen so far
bool any_overlap(std::vector<Span>& s) {
  std::sort(s.begin(), s.end(), [](const Span& a, const Span& b) { return a.lo < b.lo; });
  const char* reach = nullptr;
  for (size_t i = 0; i < s.size(); ++i) {
    if (i > 0 && s[i].lo < reach) return true;
    if (i == 0 || s[i].hi > reach) reach = s[i].hi;
  }
  return false;
}

}  // namespace

extern "C" {

vof_status vof_batched_plan(const vof_box* boxes, int nbox, int lanes, int* lane_of_box, size_t* lane_offset,
                            size_t* workspace_bytes) {
  Plan p;
  if (!make_plan(boxes, nbox, lanes, &p)) return VOF_EINVAL;
  if (lane_of_box)
    for (int b = 0; b < nbox; ++b) lane_of_box[b] = p.lane[b];
  if (lane_offset)
    for (int l = 0; l < lanes; ++l) lane_offset[l] = p.offset[l];
  if (workspace_bytes) *workspace_bytes = p.total;
  return VOF_OK;
}

size_t vof_batched_workspace_bytes(const vof_box* boxes, int nbox, int lanes) {
  Plan p;
  if (!make_plan(boxes, nbox, lanes, &p)) return 0;
  return p.total;
}

vof_status vof_batched_step(const vof_box* boxes, int nbox, long step_index, double* sums, int lanes,
                            void* const* lane_streams, void* workspace, size_t workspace_bytes, void* stream) {
  if (nbox == 0 && lanes >= 1) return VOF_OK;
  if (step_index < 0) return VOF_EINVAL;
  if (lanes > 1 && !lane_streams) return VOF_EINVAL;
  Plan p;
  if (!make_plan(boxes, nbox, lanes, &p)) return VOF_EINVAL;
  if (!workspace || ((uintptr_t)workspace & 255) != 0 || workspace_bytes < p.total) return VOF_EINVAL;
  // every box checked before anything is queued
  std::vector<Span> spans;
  spans.reserve(2 * (size_t)nbox + 1);
  for (int b = 0; b < nbox; ++b) {
    const vof_box& x = boxes[b];
    if (!x.c || !x.e || !x.u || !x.v || !x.w || !(x.dt >= 0.0)) return VOF_EINVAL;
    const size_t B = box_cells(x) * sizeof(double);
    spans.push_back({reinterpret_cast<const char*>(x.c), reinterpret_cast<const char*>(x.c) + B});
    spans.push_back({reinterpret_cast<const char*>(x.e), reinterpret_cast<const char*>(x.e) + B});
  }
  if (p.total > 0)
    spans.push_back({static_cast<const char*>(workspace), static_cast<const char*>(workspace) + p.total});
  if (any_overlap(spans)) return VOF_EINVAL;
  if (sums) {
    const char* s0 = reinterpret_cast<const char*>(sums);
    const char* s1 = s0 + (size_t)nbox * VOF_NSUMS * sizeof(double);
    for (const Span& s : spans)
      if (s0 < s.hi && s.lo < s1) return VOF_EINVAL;
  }

  cudaStream_t main = (cudaStream_t)stream;
  std::vector<cudaStream_t> ls(lanes, main);
  if (lane_streams)
    for (int l = 0; l < lanes; ++l) ls[l] = (cudaStream_t)lane_streams[l];

  // fork: every lane waits for the work queued on the caller's stream
  std::vector<cudaEvent_t> ev(lanes + 1, nullptr);
  cudaError_t err = cudaSuccess;
  for (int i = 0; i <= lanes && err == cudaSuccess; ++i) err = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
  if (err == cudaSuccess) err = cudaEventRecord(ev[lanes], main);
  for (int l = 0; l < lanes && err == cudaSuccess; ++l)
    if (ls[l] != main) err = cudaStreamWaitEvent(ls[l], ev[lanes], 0);
  vof_status st = VOF_OK;
  if (err != cudaSuccess) {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    vofgb::set_last_cuda_error((int)err);
    return VOF_ECUDA;
  }
  char* ws = static_cast<char*>(workspace);
  for (int b : p.order) {
    const vof_box& x = boxes[b];
    const int l = p.lane[b];
    const size_t need = vof_step_workspace_bytes(&x.grid);
    st = vof_step(&x.grid, x.c, x.e, x.u, x.v, x.w, x.dt, step_index, x.dd, x.dd_uniform,
                  sums ? sums + (size_t)VOF_NSUMS * b : nullptr, ws + p.offset[l], need, ls[l]);
    if (st != VOF_OK) break;
  }
  // join: the caller's stream waits for every lane (also after a failure,
  // so that nothing of the call is left running unordered)
  for (int l = 0; l < lanes; ++l) {
    if (ls[l] == main) continue;
    cudaError_t e1 = cudaEventRecord(ev[l], ls[l]);
    cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(main, ev[l], 0) : e1;
    if (e2 != cudaSuccess && err == cudaSuccess) err = e2;
  }
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
  if (st != VOF_OK) return st;
  if (err != cudaSuccess) {
    vofgb::set_last_cuda_error((int)err);
    return VOF_ECUDA;
  }
  return VOF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Grouped batch: one launch per kernel of the time step covers every box.
// vof_group_create() carves each box's own step workspace out of the
// caller's buffer, builds every kernel's per-box arguments (exactly as
// vof_step would) and the CTA -> box maps of every grouped launch, and copies
// them into the same buffer once; vof_group_step() then issues ~22 launches
// whatever the number of boxes (no host work per box, capturable).
// ---------------------------------------------------------------------------
namespace {

using namespace vofgb;

struct Launch {
  GroupMap m;
  unsigned ctas = 0;
};

// host side of one grouped launch while planning: per box its launch shape
struct LaunchPlan {
  std::vector<uint3> gdim;
  std::vector<uint32_t> first;
  unsigned total = 0;
  void add(unsigned x, unsigned y, unsigned z) {
    x = x ? x : 1;
    y = y ? y : 1;
    z = z ? z : 1;
    first.push_back(total);
    gdim.push_back(make_uint3(x, y, z));
    total += x * y * z;
  }
  size_t bytes() const { return align256(gdim.size() * sizeof(uint3)) + 2 * align256(gdim.size() * 4) +
                                align256((size_t)total * 4); }
};

}  // namespace

struct vof_group {
  int nbox = 0;
  int f32 = 0, youngs = 0;
  const TileArgs* tiles = nullptr;
  const SweepArgs* sweep[3] = {nullptr, nullptr, nullptr};
  const ShiftArgs* shift = nullptr;
  const ReduceBox* red = nullptr;
  Launch l_tiles, l_quiet, l_stream[3], l_prep[3], l_faces[3], l_update[3], l_sh[5], l_red1;
  bool sums = false;
};

namespace {

unsigned div_up(unsigned long long a, unsigned long long b) { return (unsigned)((a + b - 1) / b); }

// CTAs of a grid-stride kernel for a box of n cells: about one per `work`
// cells, at most the single-grid launch's count
unsigned gs_ctas(size_t n, int work, int cap) {
  unsigned long long k = (n + (unsigned long long)work - 1) / (unsigned long long)work;
  if (k < 1) k = 1;
  if (k > (unsigned long long)cap) k = (unsigned long long)cap;
  return (unsigned)k;
}

}  // namespace

extern "C" {

size_t vof_group_workspace_bytes(const vof_box* boxes, int nbox, int work_per_cta);

// Plans (host) and, when `dev` is not null, builds the group in `dev`.
static vof_status group_plan(const vof_box* boxes, int nbox, double* sums, int work, char* dev, size_t dev_bytes,
                             cudaStream_t st, vof_group* out, size_t* need) {
  if (nbox < 1 || !boxes || work < 32) return VOF_EINVAL;
  const int prec = boxes[0].grid.precision, nrm = boxes[0].grid.normal;
  std::vector<size_t> ws(nbox);
  size_t off = 0;
  for (int b = 0; b < nbox; ++b) {
    if (boxes[b].grid.precision != prec || boxes[b].grid.normal != nrm || nrm == VOF_NORMAL_MLP) return VOF_EINVAL;
    ws[b] = vof_step_workspace_bytes(&boxes[b].grid);
    if (ws[b] == 0) return VOF_EINVAL;
    off += align256(ws[b]);
  }
  const size_t tables = off;
  std::vector<StepBox> sb(nbox);
  // launch plans
  LaunchPlan p_tiles, p_quiet, p_stream[3], p_prep[3], p_faces[3], p_update[3], p_sh[5], p_red1;
  size_t base = 0;
  for (int b = 0; b < nbox; ++b) {
    const vof_box& x = boxes[b];
    if (!x.c || !x.e || !x.u || !x.v || !x.w || !(x.dt >= 0.0)) return VOF_EINVAL;
    char* wsb = dev ? dev + base : reinterpret_cast<char*>(256);  // planning: any non-null address
    if (!step_box(&x.grid, x.c, x.e, x.u, x.v, x.w, x.dt, x.dd, x.dd_uniform,
                  sums ? sums + (size_t)VOF_NSUMS * b : nullptr, wsb, &sb[b]))
      return VOF_EINVAL;
    base += align256(ws[b]);
    const StepBox& B = sb[b];
    p_tiles.add(B.grid_tiles.x, B.grid_tiles.y, B.grid_tiles.z);
    p_quiet.add(B.grid_quiet, 1, 1);
    for (int a = 0; a < 3; ++a) {
      p_stream[a].add(B.grid_stream[a].x, B.grid_stream[a].y, B.grid_stream[a].z);
      p_prep[a].add(gs_ctas(B.cells, work, prep_ctas()), 1, 1);
      p_faces[a].add(gs_ctas(B.cells, work, prep_ctas()), 1, 1);
      p_update[a].add(B.grid_update[a], 1, 1);
    }
    p_sh[0].add(B.grid_shift_stream.x, B.grid_shift_stream.y, 1);
    for (int k = 1; k < 4; ++k) p_sh[k].add(gs_ctas(B.cells, work, shift_list_ctas()), 1, 1);
    p_sh[4].add(B.grid_shift_sums, 1, 1);
    p_red1.add(kReduceCTAs, 1, 1);
  }
  // table region after the boxes' workspaces
  LaunchPlan* plans[] = {&p_tiles,     &p_quiet,     &p_stream[0], &p_stream[1], &p_stream[2], &p_prep[0],
                         &p_prep[1],   &p_prep[2],   &p_faces[0],  &p_faces[1],  &p_faces[2],  &p_update[0],
                         &p_update[1], &p_update[2], &p_sh[0],     &p_sh[1],     &p_sh[2],     &p_sh[3],
                         &p_sh[4],     &p_red1};
  const size_t nb = (size_t)nbox;
  size_t t = tables;
  const size_t o_tiles = t;  t += align256(nb * sizeof(TileArgs));
  size_t o_sweep[3];
  for (int a = 0; a < 3; ++a) { o_sweep[a] = t; t += align256(nb * sizeof(SweepArgs)); }
  const size_t o_shift = t;  t += align256(nb * sizeof(ShiftArgs));
  const size_t o_red = t;    t += align256(nb * sizeof(ReduceBox));
  const size_t o_maps = t;
  for (LaunchPlan* lp : plans) t += lp->bytes();
  if (need) *need = t;
  if (!dev) return VOF_OK;
  if (dev_bytes < t) return VOF_EINVAL;

  // host image of the table region, one copy
  std::vector<unsigned char> img(t - tables, 0);
  auto put = [&](size_t o, const void* src, size_t n) { std::memcpy(img.data() + (o - tables), src, n); };
  {
    std::vector<TileArgs> ta(nb);
    std::vector<SweepArgs> sa(nb);
    std::vector<ShiftArgs> sh(nb);
    std::vector<ReduceBox> rb(nb);
    for (size_t b = 0; b < nb; ++b) ta[b] = sb[b].tiles;
    put(o_tiles, ta.data(), nb * sizeof(TileArgs));
    for (int a = 0; a < 3; ++a) {
      for (size_t b = 0; b < nb; ++b) sa[b] = sb[b].sweep[a];
      put(o_sweep[a], sa.data(), nb * sizeof(SweepArgs));
    }
    for (size_t b = 0; b < nb; ++b) sh[b] = sb[b].shift;
    put(o_shift, sh.data(), nb * sizeof(ShiftArgs));
    for (size_t b = 0; b < nb; ++b) rb[b] = sb[b].red;
    put(o_red, rb.data(), nb * sizeof(ReduceBox));
  }
  Launch* launches[] = {&out->l_tiles,     &out->l_quiet,     &out->l_stream[0], &out->l_stream[1],
                        &out->l_stream[2], &out->l_prep[0],   &out->l_prep[1],   &out->l_prep[2],
                        &out->l_faces[0],  &out->l_faces[1],  &out->l_faces[2],  &out->l_update[0],
                        &out->l_update[1], &out->l_update[2], &out->l_sh[0],     &out->l_sh[1],
                        &out->l_sh[2],     &out->l_sh[3],     &out->l_sh[4],     &out->l_red1};
  size_t o = o_maps;
  for (size_t i = 0; i < sizeof(plans) / sizeof(plans[0]); ++i) {
    const LaunchPlan& lp = *plans[i];
    const size_t nent = lp.gdim.size();
    const size_t o_gdim = o, o_first = o_gdim + align256(nent * sizeof(uint3)), o_cta = o_first + align256(nent * 4);
    put(o_gdim, lp.gdim.data(), nent * sizeof(uint3));
    put(o_first, lp.first.data(), nent * 4);
    std::vector<uint32_t> cta(lp.total);
    for (size_t e = 0; e < nent; ++e) {
      const unsigned n = lp.gdim[e].x * lp.gdim[e].y * lp.gdim[e].z;
      for (unsigned k = 0; k < n; ++k) cta[lp.first[e] + k] = (uint32_t)e;
    }
    put(o_cta, cta.data(), cta.size() * 4);
    Launch& L = *launches[i];
    L.m.gdim = reinterpret_cast<const uint3*>(dev + o_gdim);
    L.m.box_first = reinterpret_cast<const uint32_t*>(dev + o_first);
    L.m.cta_box = reinterpret_cast<const uint32_t*>(dev + o_cta);
    L.ctas = lp.total;
    o += lp.bytes();
  }
  cudaError_t err = cudaMemcpyAsync(dev + tables, img.data(), img.size(), cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) {
    set_last_cuda_error((int)err);
    return VOF_ECUDA;
  }
  out->nbox = nbox;
  out->f32 = prec == VOF_F32_FLUX ? 1 : 0;
  out->youngs = nrm == VOF_NORMAL_YOUNGS ? 1 : 0;
  out->tiles = reinterpret_cast<const TileArgs*>(dev + o_tiles);
  for (int a = 0; a < 3; ++a) out->sweep[a] = reinterpret_cast<const SweepArgs*>(dev + o_sweep[a]);
  out->shift = reinterpret_cast<const ShiftArgs*>(dev + o_shift);
  out->red = reinterpret_cast<const ReduceBox*>(dev + o_red);
  out->sums = sums != nullptr;
  return VOF_OK;
}

size_t vof_group_workspace_bytes(const vof_box* boxes, int nbox, int work_per_cta) {
  size_t need = 0;
  vof_group tmp;
  if (group_plan(boxes, nbox, nullptr, work_per_cta, nullptr, 0, nullptr, &tmp, &need) != VOF_OK) return 0;
  return need;
}

vof_status vof_group_create(const vof_box* boxes, int nbox, double* sums, int work_per_cta, void* workspace,
                            size_t workspace_bytes, void* stream, vof_group** out) {
  if (!out || !workspace || ((uintptr_t)workspace & 255) != 0) return VOF_EINVAL;
  *out = nullptr;
  vof_group* grp = new (std::nothrow) vof_group();
  if (!grp) return VOF_EINVAL;
  // the boxes' fields must not overlap one another or the buffer
  size_t need = 0;
  vof_status st = group_plan(boxes, nbox, sums, work_per_cta, nullptr, 0, nullptr, grp, &need);
  if (st == VOF_OK) {
    std::vector<Span> spans;
    for (int b = 0; b < nbox; ++b) {
      const size_t B = box_cells(boxes[b]) * sizeof(double);
      spans.push_back({reinterpret_cast<const char*>(boxes[b].c), reinterpret_cast<const char*>(boxes[b].c) + B});
      spans.push_back({reinterpret_cast<const char*>(boxes[b].e), reinterpret_cast<const char*>(boxes[b].e) + B});
    }
    spans.push_back({static_cast<const char*>(workspace), static_cast<const char*>(workspace) + need});
    if (any_overlap(spans)) st = VOF_EINVAL;
  }
  if (st == VOF_OK)
    st = group_plan(boxes, nbox, sums, work_per_cta, static_cast<char*>(workspace), workspace_bytes,
                    (cudaStream_t)stream, grp, &need);
  if (st != VOF_OK) {
    delete grp;
    return st;
  }
  *out = grp;
  return VOF_OK;
}

vof_status vof_group_step(vof_group* grp, long step_index, void* stream) {
  if (!grp || grp->nbox < 1 || step_index < 0) return VOF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // the tile pass also clears every box's frozen-state flags and counters
  cudaError_t err =
      launch_tiles_grp(grp->l_tiles.m, grp->l_quiet.m, grp->tiles, grp->l_tiles.ctas, grp->l_quiet.ctas, st);
  for (int s = 0; s < 3 && err == cudaSuccess; ++s) {
    const int ax = (step_index % 2 == 0) ? s : 2 - s;
    const GroupMap maps[4] = {grp->l_stream[ax].m, grp->l_prep[ax].m, grp->l_faces[ax].m, grp->l_update[ax].m};
    const unsigned ctas[4] = {grp->l_stream[ax].ctas, grp->l_prep[ax].ctas, grp->l_faces[ax].ctas,
                              grp->l_update[ax].ctas};
    err = launch_sweep_grp(ax, grp->f32, grp->youngs, maps, grp->sweep[ax], ctas, st);
  }
  if (err == cudaSuccess) {
    GroupMap maps[5];
    unsigned ctas[5];
    for (int k = 0; k < 5; ++k) {
      maps[k] = grp->l_sh[k].m;
      ctas[k] = grp->l_sh[k].ctas;
    }
    err = launch_shift_grp(maps, grp->shift, ctas, st);
  }
  if (err == cudaSuccess && grp->sums)
    err = launch_reduce_grp(grp->l_red1.m, grp->red, grp->l_red1.ctas, (unsigned)grp->nbox, st);
  if (err != cudaSuccess) {
    set_last_cuda_error((int)err);
    return VOF_ECUDA;
  }
  return VOF_OK;
}

void vof_group_destroy(vof_group* grp) { delete grp; }

}  // extern "C"
