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
