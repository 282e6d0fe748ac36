// Batched engine: many independent lattices (uneven sizes, their own EOS and
// relaxation times, one collision kind) advanced together.
//
// Work is partitioned by blocks, not by instances: the density/psi pass runs one
// 256-node block per work item; the collision pass runs one 256-thread tile per
// work item, with a tile shape (tw x th, tw*th = 256) chosen per instance so that
// narrow lattices (the 4-wide planar ones) do not leave threads idle. A
// device-resident table maps each work item to its instance. Three ways to run a
// step, chosen by the autotuner:
//   PLAN_LAUNCHES   two launches per step covering every instance;
//   PLAN_GRAPH      the same two launches, two steps captured in a CUDA graph that
//                   is replayed;
//   PLAN_PERSISTENT one cooperative launch for all steps of a call: a grid-stride
//                   loop over work items with a grid barrier between the passes.
//                   Every barrier wait is bounded: after the spin limit the block
//                   sets the error word (PPLBM_ERR_TIMEOUT) and returns.
//   PLAN_PIPELINED  the instances in two groups of about equal node counts, group B
//                   half a step behind group A inside a call: each launch runs the
//                   density pass of one group with the collision pass of the other
//                   (work items interleaved), so that the FP64-bound and the
//                   integer-bound pass share the SMs; a prologue (density pass of A)
//                   and an epilogue (collision pass of B) bring every instance to the
//                   same step at the end of the call; two-step CUDA graphs in between.
// The per-node arithmetic is the single-lattice kernels' (step_device.cuh), so a
// batched step is bitwise identical to stepping each lattice alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pplbm.h"
#include "batch_kernels.cuh"

namespace pplbm {
namespace {

int ilog2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

bool lattice_ok(const pplbm_lattice* l) {
  if (!l || l->nx < 1 || l->ny < 1 || l->reserved != 0) return false;
  if (9 * (int64_t)l->nx * l->ny >= ((int64_t)1 << 31)) return false;
  if (!(l->bc & PPLBM_BC_PERIODIC_X)) return false;
  const uint32_t walls = l->bc & (PPLBM_BC_WALL_BOTTOM | PPLBM_BC_WALL_TOP);
  if (l->bc & PPLBM_BC_PERIODIC_Y) return walls == 0;
  return walls == (PPLBM_BC_WALL_BOTTOM | PPLBM_BC_WALL_TOP);
}

size_t inst_doubles(const pplbm_lattice& l, int kind) {
  const size_t n = (size_t)l.nx * l.ny;
  const size_t d = n * (20 + (size_t)moment_planes(kind));  // f x 2, psi, moments, guard snapshot
  return (d + 31) & ~(size_t)31;  // 256-byte aligned instances
}

// tile width for a lattice: the power of two in [4, 256] that wastes the fewest
// threads on partial tiles (ties go to the width closest to 32)
int model_tile_width(int nx, int ny) {
  int best = 32;
  long long best_waste = -1;
  for (int tw = 4; tw <= 256; tw *= 2) {
    const int th = 256 / tw;
    const long long tiles = (long long)((nx + tw - 1) / tw) * ((ny + th - 1) / th);
    const long long waste = tiles * 256 - (long long)nx * ny;
    const int dist = std::abs(ilog2(tw) - 5);
    if (best_waste < 0 || waste < best_waste || (waste == best_waste && dist < std::abs(ilog2(best) - 5))) {
      best = tw;
      best_waste = waste;
    }
  }
  return best;
}

}  // namespace
}  // namespace pplbm

using namespace pplbm;

struct pplbm_batch {
  int n;
  int kind;
  bool st;  // some instance has the surface-tension source
  std::vector<pplbm_lattice> lat;
  std::vector<pplbm_relax> relax;
  std::vector<pplbm_eos_derived> eos;
  std::vector<BatchInst> host_inst;
  std::vector<double*> bufA, bufB;  // per instance: the two f buffers
  int parity;                       // state of every instance is in buffer `parity`
  cudaStream_t stream;
  cudaStream_t capture_stream;
  void* dev_block;                  // owned: instance table, owners, barrier, error word
  BatchInst* d_inst;
  int* d_owner1;
  int* d_owner2;
  int n1, n2;
  GridBarrier* d_bar;
  int* d_err;                       // batch-wide word (grid-barrier timeout)
  unsigned* d_queue;                // the mixed kernel's item counter and finished-block count
  int* d_ierr;                      // one word per instance (divergence)
  int* d_snap_valid;                // one word per instance: guard snapshot holds a density
  double* d_gpart;                  // guard partials, 4 per density-pass work item
  double* d_gout;                   // guard output, 4 per instance
  bool isolate;                     // diverged instances do not stop the batch
  std::vector<int> diverged;
  int persistent_grid;
  pplbm_batch_plan plan;
  cudaGraphExec_t graph[2];  // graph[p]: two steps starting from parity p
  // pipelined plan: item tables (instance | pass bit, then the density block or the
  // collision tile's log2 width and origin) of M1 = collision of A + density of B, M2 =
  // density of A + collision of B, the prologue PA = density of A and the epilogue EB =
  // collision of B; pgraph[p] replays M1, M2, M1, M2 from parity p; mixed_grid = the
  // mixed kernel's resident blocks
  int4* d_mix[4];
  int nmix[4];
  int mixed_grid;
  cudaGraphExec_t pgraph[2];
  int64_t steps;
  pplbm_status sticky;
  std::string msg;
  bool timing;
  std::vector<cudaEvent_t> ev;
  size_t ev_used;
  int64_t timed_steps;
  // per-pass timing: event pairs around every launch of each pass (0: density/psi,
  // 1: collision). Under the launches plan every step is two plain launches bracketed
  // by events; under the graph plan each two-step graph replay uses one of
  // `timed_graphs` graphs that record their own events between the launches.
  bool pass_timing;
  int64_t pass_capacity;
  std::vector<cudaEvent_t> pev[2];
  size_t pev_used[2];
  struct TimedGraph {
    cudaGraphExec_t exec;
    cudaEvent_t ev[5];  // before pass 1, between the four launches, after the last
  };
  std::vector<TimedGraph> timed_graphs[2];  // by the parity the two steps start from
  size_t timed_used[2];                     // replayed since the last read
};

namespace {

pplbm_status bfail(pplbm_batch* b, pplbm_status s, const char* fmt, ...) {
  if (b) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    b->msg = buf;
  }
  return s;
}

#define BTRY(b, call)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return bfail((b), PPLBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

bool is_dev(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// rebuild the per-instance tile shapes and the owner tables for a tile-width policy
pplbm_status build_tables(pplbm_batch* b, int tile_width) {
  std::vector<int> o1, o2;
  for (int i = 0; i < b->n; ++i) {
    BatchInst& I = b->host_inst[i];
    const int nx = b->lat[i].nx, ny = b->lat[i].ny;
    const int tw = tile_width > 0 ? tile_width : model_tile_width(nx, ny);
    I.tw = tw;
    I.th = 256 / tw;
    I.log2tw = ilog2(tw);
    I.tiles_x = (nx + tw - 1) / tw;
    const int tiles = I.tiles_x * ((ny + I.th - 1) / I.th);
    const int64_t n = (int64_t)nx * ny;
    I.k1_start = (int)o1.size();
    for (int64_t k = 0; k < (n + kThreads - 1) / kThreads; ++k) o1.push_back(i);
    I.k2_start = (int)o2.size();
    for (int k = 0; k < tiles; ++k) o2.push_back(i);
  }
  if (o1.size() > (size_t)INT32_MAX / 2 || o2.size() > (size_t)INT32_MAX / 2)
    return bfail(b, PPLBM_ERR_ARG, "batch too large");
  b->n1 = (int)o1.size();
  b->n2 = (int)o2.size();
  // pipelined plan: two groups by node count (largest instance first to the lighter
  // group), then the four item tables
  std::vector<int> order(b->n);
  for (int i = 0; i < b->n; ++i) order[i] = i;
  auto nodes = [&](int i) { return (int64_t)b->lat[i].nx * b->lat[i].ny; };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return nodes(x) > nodes(y); });
  std::vector<int> group(b->n, 0);
  int64_t load[2] = {0, 0};
  for (int i : order) {
    const int g = load[1] < load[0] ? 1 : 0;
    group[i] = g;
    load[g] += nodes(i);
  }
  std::vector<int4> k1[2], k2[2];
  for (int i = 0; i < b->n; ++i) {
    const BatchInst& I = b->host_inst[i];
    const int nb = (int)((nodes(i) + kThreads - 1) / kThreads);
    const int ty_n = (b->lat[i].ny + I.th - 1) / I.th;
    for (int j = 0; j < nb; ++j) k1[group[i]].push_back(make_int4(i, j, 0, 0));
    for (int ty = 0; ty < ty_n; ++ty)
      for (int tx = 0; tx < I.tiles_x; ++tx)
        k2[group[i]].push_back(make_int4(i | (int)0x80000000u, I.log2tw, tx * I.tw, ty * I.th));
  }
  // evenly interleaved: item i of x sits at (i + 1/2)/|x| of the table, likewise for y
  auto interleave = [](const std::vector<int4>& x, const std::vector<int4>& y) {
    std::vector<int4> m;
    m.reserve(x.size() + y.size());
    size_t i = 0, j = 0;
    while (i < x.size() || j < y.size()) {
      const bool take_x = j == y.size() || (i < x.size() && (2 * i + 1) * y.size() <= (2 * j + 1) * x.size());
      m.push_back(take_x ? x[i++] : y[j++]);
    }
    return m;
  };
  const std::vector<int4> mix[4] = {interleave(k2[0], k1[1]), interleave(k1[0], k2[1]), k1[0], k2[1]};
  for (int k = 0; k < 4; ++k) {
    b->nmix[k] = (int)mix[k].size();
    if (!mix[k].empty())
      BTRY(b, cudaMemcpyAsync(b->d_mix[k], mix[k].data(), sizeof(int4) * mix[k].size(), cudaMemcpyHostToDevice,
                              b->stream));
  }
  // owner tables live in a device block sized at create for the worst case (tw = 4 or 256)
  BTRY(b, cudaMemcpyAsync(b->d_inst, b->host_inst.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice,
                          b->stream));
  BTRY(b, cudaMemcpyAsync(b->d_owner1, o1.data(), sizeof(int) * o1.size(), cudaMemcpyHostToDevice, b->stream));
  BTRY(b, cudaMemcpyAsync(b->d_owner2, o2.data(), sizeof(int) * o2.size(), cudaMemcpyHostToDevice, b->stream));
  BTRY(b, cudaStreamSynchronize(b->stream));
  return PPLBM_OK;
}

void destroy_graphs(pplbm_batch* b) {
  for (int p = 0; p < 2; ++p) {
    if (b->graph[p]) {
      cudaGraphExecDestroy(b->graph[p]);
      b->graph[p] = nullptr;
    }
    if (b->pgraph[p]) {
      cudaGraphExecDestroy(b->pgraph[p]);
      b->pgraph[p] = nullptr;
    }
  }
}

// pipelined plan: M1 (collision of A and density of B, both at parity p) and M2
// (density of A at 1 - p, collision of B at p) advance both groups by one step
void launch_mixed_step(pplbm_batch* b, int p, cudaStream_t s) {
  launch_mixed(b->kind, b->st, b->d_inst, b->d_mix[0], b->nmix[0], b->mixed_grid, p, p, b->d_queue, s);
  launch_mixed(b->kind, b->st, b->d_inst, b->d_mix[1], b->nmix[1], b->mixed_grid, 1 - p, p, b->d_queue, s);
}

pplbm_status build_pipelined_graphs(pplbm_batch* b) {
  for (int p = 0; p < 2; ++p) {
    cudaGraph_t g;
    BTRY(b, cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
    launch_mixed_step(b, p, b->capture_stream);
    launch_mixed_step(b, 1 - p, b->capture_stream);
    BTRY(b, cudaStreamEndCapture(b->capture_stream, &g));
    cudaError_t e = cudaGraphInstantiate(&b->pgraph[p], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, PPLBM_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  return PPLBM_OK;
}

pplbm_status build_graphs(pplbm_batch* b) {
  destroy_graphs(b);
  for (int p = 0; p < 2; ++p) {
    cudaGraph_t g;
    BTRY(b, cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
    launch_pair(b->kind, b->st, b->d_inst, b->d_owner1, b->n1, b->d_owner2, b->n2, p, b->capture_stream);
    launch_pair(b->kind, b->st, b->d_inst, b->d_owner1, b->n1, b->d_owner2, b->n2, 1 - p, b->capture_stream);
    BTRY(b, cudaStreamEndCapture(b->capture_stream, &g));
    cudaError_t e = cudaGraphInstantiate(&b->graph[p], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, PPLBM_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  return PPLBM_OK;
}

void destroy_timed_graphs(pplbm_batch* b) {
  for (int p = 0; p < 2; ++p) {
    for (auto& g : b->timed_graphs[p]) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      for (cudaEvent_t e : g.ev)
        if (e) cudaEventDestroy(e);
    }
    b->timed_graphs[p].clear();
    b->timed_used[p] = 0;
  }
}

// count graphs of two steps from each parity, each recording its own events between
// the launches (event-record nodes: a replay overwrites them, so a graph is used at
// most once between two reads)
pplbm_status build_timed_graphs(pplbm_batch* b, int64_t count) {
  destroy_timed_graphs(b);
  for (int p = 0; p < 2; ++p) {
    for (int64_t k = 0; k < count; ++k) {
      b->timed_graphs[p].push_back(pplbm_batch::TimedGraph{});  // owned from here, filled below
      pplbm_batch::TimedGraph& g = b->timed_graphs[p].back();
      for (cudaEvent_t& e : g.ev) BTRY(b, cudaEventCreate(&e));
      cudaStream_t cs = b->capture_stream;
      cudaGraph_t graph;
      BTRY(b, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      int e = 0;
      for (int step = 0; step < 2; ++step) {
        const int par = (p + step) & 1;
        if (step == 0) cudaEventRecordWithFlags(g.ev[e++], cs, cudaEventRecordExternal);
        launch_density_pass(b->kind, b->d_inst, b->d_owner1, b->n1, par, cs);
        cudaEventRecordWithFlags(g.ev[e++], cs, cudaEventRecordExternal);
        launch_collision_pass(b->kind, b->st, b->d_inst, b->d_owner2, b->n2, par, cs);
        cudaEventRecordWithFlags(g.ev[e++], cs, cudaEventRecordExternal);
      }
      BTRY(b, cudaStreamEndCapture(cs, &graph));
      const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) return bfail(b, PPLBM_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
    }
  }
  return PPLBM_OK;
}

pplbm_status apply_plan(pplbm_batch* b, int mode, int tile_width) {
  if (mode != PPLBM_PLAN_LAUNCHES && mode != PPLBM_PLAN_GRAPH && mode != PPLBM_PLAN_PERSISTENT &&
      mode != PPLBM_PLAN_PIPELINED)
    return bfail(b, PPLBM_ERR_ARG, "unknown plan mode %d", mode);
  if (tile_width != 0 && (tile_width < 4 || tile_width > 256 || (tile_width & (tile_width - 1))))
    return bfail(b, PPLBM_ERR_ARG, "tile width must be 0 or a power of two in [4, 256]");
  if (pplbm_status s = build_tables(b, tile_width)) return s;
  destroy_graphs(b);
  destroy_timed_graphs(b);
  if (mode == PPLBM_PLAN_GRAPH)
    if (pplbm_status s = build_graphs(b)) return s;
  if (mode == PPLBM_PLAN_PIPELINED)
    if (pplbm_status s = build_pipelined_graphs(b)) return s;
  if (mode == PPLBM_PLAN_GRAPH && b->pass_timing)
    if (pplbm_status s = build_timed_graphs(b, (b->pass_capacity + 1) / 2)) return s;
  b->plan.mode = mode;
  b->plan.tile_width = tile_width;
  b->plan.k1_blocks = b->n1;
  b->plan.k2_tiles = b->n2;
  return PPLBM_OK;
}

pplbm_status poll(pplbm_batch* b) {
  int h = 0;
  std::vector<int> hi(b->n, 0);
  BTRY(b, cudaMemcpyAsync(&h, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BTRY(b, cudaMemcpyAsync(hi.data(), b->d_ierr, sizeof(int) * b->n, cudaMemcpyDeviceToHost, b->stream));
  BTRY(b, cudaStreamSynchronize(b->stream));
  int first = -1;
  for (int i = 0; i < b->n; ++i)
    if (hi[i]) {
      b->diverged[i] = 1;
      if (first < 0) first = i;
    }
  if (b->sticky == PPLBM_OK) {
    if (h & kErrTimeout) {
      b->sticky = PPLBM_ERR_TIMEOUT;
      b->msg = "a grid-barrier wait of the persistent kernel gave up";
    } else if (first >= 0 && !b->isolate) {
      b->sticky = PPLBM_ERR_DIVERGED;
      char buf[160];
      snprintf(buf, sizeof(buf), "instance %d met a non-finite or non-positive density, or psi^2 <= 0", first);
      b->msg = buf;
    }
  }
  return b->sticky;
}

pplbm_status launch_persistent(pplbm_batch* b, int64_t nsteps, cudaStream_t s, unsigned spin_limit, int absent) {
  BTRY(b, cudaMemsetAsync(b->d_bar, 0, sizeof(GridBarrier), s));
  int parity0 = b->parity;
  long long ns = nsteps;
  void* args[] = {(void*)&b->d_inst, (void*)&b->d_owner1, (void*)&b->n1,     (void*)&b->d_owner2,
                  (void*)&b->n2,     (void*)&parity0,     (void*)&ns,        (void*)&b->d_bar,
                  (void*)&b->d_err,  (void*)&spin_limit,  (void*)&absent};
  BTRY(b, cudaLaunchCooperativeKernel(persistent_kernel(b->kind, b->st), dim3(b->persistent_grid), dim3(kThreads), args, 0,
                                      s));
  return PPLBM_OK;
}

pplbm_status grow_pass_events(pplbm_batch* b, int k, size_t need) {
  while (b->pev[k].size() < need) {
    cudaEvent_t e;
    BTRY(b, cudaEventCreate(&e));
    b->pev[k].push_back(e);
  }
  return PPLBM_OK;
}

// one step as two plain launches, each bracketed by an event pair
pplbm_status issue_timed_step(pplbm_batch* b, cudaStream_t s) {
  for (int k = 0; k < 2; ++k) {
    if (pplbm_status st = grow_pass_events(b, k, b->pev_used[k] + 2)) return st;
    BTRY(b, cudaEventRecord(b->pev[k][b->pev_used[k]], s));
    if (k == 0)
      launch_density_pass(b->kind, b->d_inst, b->d_owner1, b->n1, b->parity, s);
    else
      launch_collision_pass(b->kind, b->st, b->d_inst, b->d_owner2, b->n2, b->parity, s);
    BTRY(b, cudaEventRecord(b->pev[k][b->pev_used[k] + 1], s));
    b->pev_used[k] += 2;
  }
  b->parity ^= 1;
  return PPLBM_OK;
}

pplbm_status issue_steps(pplbm_batch* b, int64_t nsteps, cudaStream_t s) {
  int64_t k = 0;
  if (b->pass_timing) {
    if (b->plan.mode == PPLBM_PLAN_GRAPH) {
      for (; k + 2 <= nsteps; k += 2) {
        auto& tg = b->timed_graphs[b->parity];
        size_t& used = b->timed_used[b->parity];
        if (used >= tg.size()) break;  // every timed graph is waiting to be read
        BTRY(b, cudaGraphLaunch(tg[used].exec, s));
        ++used;
      }
    }
    for (; k < nsteps; ++k)
      if (pplbm_status st = issue_timed_step(b, s)) return st;
    BTRY(b, cudaGetLastError());
    return PPLBM_OK;
  }
  if (b->plan.mode == PPLBM_PLAN_PIPELINED && nsteps > 0) {
    // prologue, then M1 M2 per step with the last M2 left out, then the epilogue
    const int p0 = b->parity;
    launch_mixed(b->kind, b->st, b->d_inst, b->d_mix[2], b->nmix[2], b->mixed_grid, p0, p0, b->d_queue, s);
    int64_t j = 0;
    for (; j + 2 <= nsteps - 1; j += 2) BTRY(b, cudaGraphLaunch(b->pgraph[(p0 + j) & 1], s));
    for (; j < nsteps - 1; ++j) launch_mixed_step(b, (int)((p0 + j) & 1), s);
    const int pl = (int)((p0 + nsteps - 1) & 1);
    launch_mixed(b->kind, b->st, b->d_inst, b->d_mix[0], b->nmix[0], b->mixed_grid, pl, pl, b->d_queue, s);
    launch_mixed(b->kind, b->st, b->d_inst, b->d_mix[3], b->nmix[3], b->mixed_grid, pl, pl, b->d_queue, s);
    BTRY(b, cudaGetLastError());
    b->parity = (int)((p0 + nsteps) & 1);
    return PPLBM_OK;
  }
  if (b->plan.mode == PPLBM_PLAN_PERSISTENT && nsteps > 0) {
    if (pplbm_status st = launch_persistent(b, nsteps, s, kSpinLimit, -1)) return st;
    b->parity = (int)((b->parity + nsteps) & 1);
    return PPLBM_OK;
  }
  if (b->plan.mode == PPLBM_PLAN_GRAPH) {
    for (; k + 2 <= nsteps; k += 2) BTRY(b, cudaGraphLaunch(b->graph[b->parity], s));
  }
  for (; k < nsteps; ++k) {
    launch_pair(b->kind, b->st, b->d_inst, b->d_owner1, b->n1, b->d_owner2, b->n2, b->parity, s);
    b->parity ^= 1;
  }
  BTRY(b, cudaGetLastError());
  return PPLBM_OK;
}

// StepArgs of instance i reading buffer `parity`
StepArgs& args_of(pplbm_batch* b, int i) { return b->host_inst[i].a[b->parity]; }

}  // namespace

extern "C" {

size_t pplbm_batch_workspace_bytes(int32_t n, const pplbm_lattice* lattices, const pplbm_relax* relax) {
  if (n < 1 || !lattices || !relax) return 0;
  size_t total = 0;
  const int k0 = collision_kind(&relax[0]);
  for (int i = 0; i < n; ++i) {
    const int k = collision_kind(&relax[i]);
    if (k < 0 || k != k0 || !lattice_ok(&lattices[i])) return 0;
    total += inst_doubles(lattices[i], k);
  }
  return total * sizeof(double);
}

pplbm_status pplbm_batch_create(pplbm_batch** out, int32_t n, const pplbm_lattice* lattices,
                                const pplbm_eos_params* eos, const pplbm_relax* relax, double G, void* workspace,
                                size_t workspace_bytes, void* stream) {
  if (!out) return PPLBM_ERR_ARG;
  *out = nullptr;
  if (n < 1 || !lattices || !eos || !relax || !workspace) return PPLBM_ERR_ARG;
  const size_t need = pplbm_batch_workspace_bytes(n, lattices, relax);
  if (need == 0 || workspace_bytes < need || ((uintptr_t)workspace & 255u)) return PPLBM_ERR_ARG;
  pplbm_batch* b = new (std::nothrow) pplbm_batch();
  if (!b) return PPLBM_ERR_ARG;
  b->n = n;
  b->kind = collision_kind(&relax[0]);
  b->st = false;
  for (int i = 0; i < n; ++i) b->st = b->st || relax[i].kappa != 0.0;
  b->lat.assign(lattices, lattices + n);
  b->relax.assign(relax, relax + n);
  b->eos.resize(n);
  b->host_inst.resize(n);
  b->bufA.resize(n);
  b->bufB.resize(n);
  b->stream = (cudaStream_t)stream;
  b->sticky = PPLBM_OK;
  for (int i = 0; i < n; ++i) {
    const pplbm_status st = pplbm_eos_setup(&eos[i], G, &b->eos[i]);
    if (st != PPLBM_OK) {
      delete b;
      return st;
    }
  }
  // the largest owner tables any tile width can produce
  size_t max1 = 0, max2 = 0;
  for (int i = 0; i < n; ++i) {
    const int64_t nn = (int64_t)lattices[i].nx * lattices[i].ny;
    max1 += (nn + kThreads - 1) / kThreads;
    size_t worst = 0;
    for (int tw = 4; tw <= 256; tw *= 2)
      worst = std::max(worst, (size_t)((lattices[i].nx + tw - 1) / tw) * ((lattices[i].ny + 256 / tw - 1) / (256 / tw)));
    max2 += worst;
  }
  const size_t inst_bytes = ((sizeof(BatchInst) * n + 255) / 256) * 256;
  const size_t o1_bytes = ((sizeof(int) * max1 + 255) / 256) * 256;
  const size_t o2_bytes = ((sizeof(int) * max2 + 255) / 256) * 256;
  const size_t ierr_bytes = ((sizeof(int) * n + 255) / 256) * 256;
  const size_t gpart_bytes = ((sizeof(double) * kGuardQ * max1 + 255) / 256) * 256;
  const size_t gout_bytes = ((sizeof(double) * kGuardQ * n + 255) / 256) * 256;
  const size_t mix_bytes = ((sizeof(int4) * (max1 + max2) + 255) / 256) * 256;  // each pipelined table
  const size_t block =
      inst_bytes + o1_bytes + o2_bytes + 256 + 256 + 2 * ierr_bytes + gpart_bytes + gout_bytes + 4 * mix_bytes + 256;
  if (cudaMalloc(&b->dev_block, block) != cudaSuccess) {
    delete b;
    return PPLBM_ERR_CUDA;
  }
  char* p = (char*)b->dev_block;
  b->d_inst = (BatchInst*)p;
  b->d_owner1 = (int*)(p + inst_bytes);
  b->d_owner2 = (int*)(p + inst_bytes + o1_bytes);
  b->d_bar = (GridBarrier*)(p + inst_bytes + o1_bytes + o2_bytes);
  b->d_err = (int*)(p + inst_bytes + o1_bytes + o2_bytes + 256);
  b->d_ierr = (int*)(p + inst_bytes + o1_bytes + o2_bytes + 512);
  b->d_snap_valid = (int*)(p + inst_bytes + o1_bytes + o2_bytes + 512 + ierr_bytes);
  b->d_gpart = (double*)(p + inst_bytes + o1_bytes + o2_bytes + 512 + 2 * ierr_bytes);
  b->d_gout = (double*)(p + inst_bytes + o1_bytes + o2_bytes + 512 + 2 * ierr_bytes + gpart_bytes);
  for (int k = 0; k < 4; ++k)
    b->d_mix[k] = (int4*)(p + inst_bytes + o1_bytes + o2_bytes + 512 + 2 * ierr_bytes + gpart_bytes + gout_bytes +
                          k * mix_bytes);
  b->d_queue = (unsigned*)(p + inst_bytes + o1_bytes + o2_bytes + 512 + 2 * ierr_bytes + gpart_bytes + gout_bytes +
                           4 * mix_bytes);
  b->diverged.assign(n, 0);
  if (cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(b->dev_block);
    delete b;
    return PPLBM_ERR_CUDA;
  }
  cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
  cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(unsigned), b->stream);
  cudaMemsetAsync(b->d_ierr, 0, sizeof(int) * n, b->stream);
  cudaMemsetAsync(b->d_snap_valid, 0, sizeof(int) * n, b->stream);
  double* w = (double*)workspace;
  for (int i = 0; i < n; ++i) {
    const pplbm_lattice& L = lattices[i];
    const pplbm_relax& r = relax[i];
    const pplbm_eos_derived& d = b->eos[i];
    const int64_t nn = (int64_t)L.nx * L.ny;
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = w + 18 * nn;
    a.mom = w + 19 * nn;
    a.err = b->d_ierr + i;
    a.nx = L.nx;
    a.ny = L.ny;
    a.n = nn;
    a.walls = (L.bc & PPLBM_BC_PERIODIC_Y) ? 0 : 1;
    a.kind = b->kind;
    a.eos = make_eos_const(d);
    a.G = G;
    a.half_force = -G / 24.0;
    a.psi_ghost_bottom = d.psi_l;
    a.psi_ghost_top = d.psi_v;
    set_collision_args(a, b->kind, r, d, G);
    b->bufA[i] = w;
    b->bufB[i] = w + 9 * nn;
    BatchInst& I = b->host_inst[i];
    I.snap = w + (19 + moment_planes(b->kind)) * nn;
    I.a[0] = a;
    I.a[0].f_in = b->bufA[i];
    I.a[0].f_out = b->bufB[i];
    I.a[1] = a;
    I.a[1].f_in = b->bufB[i];
    I.a[1].f_out = b->bufA[i];
    w += inst_doubles(L, b->kind);
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_kernel(b->kind, b->st), kThreads, 0);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->persistent_grid = std::max(1, occ * sms);
  occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mixed_kernel(b->kind, b->st), kThreads, 0);
  b->mixed_grid = std::max(1, occ * sms);
  pplbm_status s = apply_plan(b, PPLBM_PLAN_LAUNCHES, 0);
  if (s != PPLBM_OK) {
    pplbm_batch_destroy(b);
    return s;
  }
  b->persistent_grid = std::min(b->persistent_grid, std::max(b->n1, b->n2));
  *out = b;
  return PPLBM_OK;
}

pplbm_status pplbm_batch_init_equilibrium(pplbm_batch* b, int32_t i, const double* rho0, const double* ux0,
                                          const double* uy0) {
  if (!b || i < 0 || i >= b->n || !rho0) return bfail(b, PPLBM_ERR_ARG, "bad instance or NULL rho0");
  if (b->sticky) return b->sticky;
  StepArgs& a = args_of(b, i);
  const double* src[3] = {rho0, ux0, uy0};
  const double* dev[3];
  for (int k = 0; k < 3; ++k) {
    if (!src[k] || is_dev(src[k])) {
      dev[k] = src[k];
    } else {  // stage host data in the other f buffer, unused between steps
      double* dst = const_cast<double*>(a.f_out) + (int64_t)k * a.n;
      BTRY(b, cudaMemcpyAsync(dst, src[k], sizeof(double) * a.n, cudaMemcpyHostToDevice, b->stream));
      dev[k] = dst;
    }
  }
  launch_init_eq(a, const_cast<double*>(a.f_in), dev[0], dev[1], dev[2], b->stream);
  BTRY(b, cudaGetLastError());
  BTRY(b, cudaMemsetAsync(b->d_snap_valid + i, 0, sizeof(int), b->stream));
  return poll(b);
}

pplbm_status pplbm_batch_step(pplbm_batch* b, int64_t nsteps) {
  if (!b || nsteps < 0) return bfail(b, PPLBM_ERR_ARG, "nsteps < 0");
  if (b->sticky) return b->sticky;
  if (b->timing) {
    while (b->ev.size() < b->ev_used + 2) {
      cudaEvent_t e;
      BTRY(b, cudaEventCreate(&e));
      b->ev.push_back(e);
    }
    BTRY(b, cudaEventRecord(b->ev[b->ev_used], b->stream));
  }
  if (pplbm_status s = issue_steps(b, nsteps, b->stream)) return s;
  if (b->timing) {
    BTRY(b, cudaEventRecord(b->ev[b->ev_used + 1], b->stream));
    b->ev_used += 2;
    b->timed_steps += nsteps;
  }
  b->steps += nsteps;
  return PPLBM_OK;
}

pplbm_status pplbm_batch_get_fields(pplbm_batch* b, int32_t i, double* rho, double* ux, double* uy, double* psi) {
  if (!b || i < 0 || i >= b->n) return bfail(b, PPLBM_ERR_ARG, "bad instance");
  if (b->sticky) return b->sticky;
  StepArgs a = args_of(b, i);
  launch_rho_psi(a, b->stream);
  double* outs[4] = {rho, ux, uy, psi};
  double* dst[4];
  bool host[4];
  for (int k = 0; k < 4; ++k) {
    host[k] = outs[k] && !is_dev(outs[k]);
    dst[k] = host[k] ? a.f_out + (int64_t)k * a.n : outs[k];
  }
  launch_fields(a, dst[0], dst[1], dst[2], dst[3], b->stream);
  BTRY(b, cudaGetLastError());
  for (int k = 0; k < 4; ++k)
    if (host[k]) BTRY(b, cudaMemcpyAsync(outs[k], dst[k], sizeof(double) * a.n, cudaMemcpyDeviceToHost, b->stream));
  return poll(b);
}

pplbm_status pplbm_batch_run_host(pplbm_batch* b, const double* const* rho0, int64_t nsteps,
                                  double* const* rho_out) {
  if (!b || !rho0 || !rho_out || nsteps < 0) return bfail(b, PPLBM_ERR_ARG, "NULL arrays or nsteps < 0");
  if (b->sticky) return b->sticky;
  for (int i = 0; i < b->n; ++i)
    if (!rho0[i] || !rho_out[i]) return bfail(b, PPLBM_ERR_ARG, "NULL density array for instance %d", i);
  // host densities in: staged in each instance's second f buffer, then f = f^eq
  for (int i = 0; i < b->n; ++i) {
    StepArgs& a = args_of(b, i);
    double* stage = const_cast<double*>(a.f_out);
    BTRY(b, cudaMemcpyAsync(stage, rho0[i], sizeof(double) * a.n, cudaMemcpyHostToDevice, b->stream));
    launch_init_eq(a, const_cast<double*>(a.f_in), stage, nullptr, nullptr, b->stream);
  }
  BTRY(b, cudaGetLastError());
  BTRY(b, cudaMemsetAsync(b->d_snap_valid, 0, sizeof(int) * b->n, b->stream));
  if (pplbm_status st = issue_steps(b, nsteps, b->stream)) return st;
  b->steps += nsteps;
  // densities out: the density pass over the final state, one copy per instance
  launch_density_pass(b->kind, b->d_inst, b->d_owner1, b->n1, b->parity, b->stream);
  for (int i = 0; i < b->n; ++i) {
    const StepArgs& a = args_of(b, i);
    BTRY(b, cudaMemcpyAsync(rho_out[i], a.mom, sizeof(double) * a.n, cudaMemcpyDeviceToHost, b->stream));
  }
  BTRY(b, cudaStreamSynchronize(b->stream));
  return poll(b);
}

pplbm_status pplbm_batch_get_f(pplbm_batch* b, int32_t i, double* f) {
  if (!b || i < 0 || i >= b->n || !f) return bfail(b, PPLBM_ERR_ARG, "bad instance or NULL f");
  const StepArgs& a = args_of(b, i);
  BTRY(b, cudaMemcpyAsync(f, a.f_in, sizeof(double) * 9 * a.n, cudaMemcpyDefault, b->stream));
  if (!is_dev(f)) BTRY(b, cudaStreamSynchronize(b->stream));
  return PPLBM_OK;
}

pplbm_status pplbm_batch_set_f(pplbm_batch* b, int32_t i, const double* f) {
  if (!b || i < 0 || i >= b->n || !f) return bfail(b, PPLBM_ERR_ARG, "bad instance or NULL f");
  if (b->sticky) return b->sticky;
  const StepArgs& a = args_of(b, i);
  BTRY(b, cudaMemcpyAsync(const_cast<double*>(a.f_in), f, sizeof(double) * 9 * a.n, cudaMemcpyDefault, b->stream));
  BTRY(b, cudaMemsetAsync(b->d_snap_valid + i, 0, sizeof(int), b->stream));
  if (!is_dev(f)) BTRY(b, cudaStreamSynchronize(b->stream));
  return PPLBM_OK;
}

pplbm_status pplbm_batch_set_plan(pplbm_batch* b, int32_t mode, int32_t tile_width) {
  if (!b) return PPLBM_ERR_ARG;
  if (b->pass_timing && (mode == PPLBM_PLAN_PERSISTENT || mode == PPLBM_PLAN_PIPELINED))
    return bfail(b, PPLBM_ERR_STATE, "per-pass timing is on: the persistent and pipelined plans mix the passes");
  BTRY(b, cudaStreamSynchronize(b->stream));
  return apply_plan(b, mode, tile_width);
}

pplbm_status pplbm_batch_get_plan(const pplbm_batch* b, pplbm_batch_plan* out) {
  if (!b || !out) return PPLBM_ERR_ARG;
  *out = b->plan;
  return PPLBM_OK;
}

pplbm_status pplbm_batch_autotune(pplbm_batch* b, int32_t trial_steps, pplbm_batch_plan* chosen) {
  if (!b || trial_steps < 2) return bfail(b, PPLBM_ERR_ARG, "trial_steps < 2");
  if (b->sticky) return b->sticky;
  // keep the state: copy every instance's current f aside, restore it afterwards
  size_t total = 0;
  for (int i = 0; i < b->n; ++i) total += 9 * (size_t)b->lat[i].nx * b->lat[i].ny;
  double* backup = nullptr;
  BTRY(b, cudaMalloc(&backup, total * sizeof(double)));
  const int parity0 = b->parity;
  size_t off = 0;
  for (int i = 0; i < b->n; ++i) {
    const StepArgs& a = args_of(b, i);
    cudaMemcpyAsync(backup + off, a.f_in, sizeof(double) * 9 * a.n, cudaMemcpyDeviceToDevice, b->stream);
    off += 9 * (size_t)a.n;
  }
  const bool pass_timing = b->pass_timing;  // the trials time whole steps, each plan as it runs
  b->pass_timing = false;
  const int modes[4] = {PPLBM_PLAN_LAUNCHES, PPLBM_PLAN_GRAPH, PPLBM_PLAN_PERSISTENT, PPLBM_PLAN_PIPELINED};
  const int widths[2] = {0, 32};
  // three interleaved rounds over the six candidates; each keeps its best time, so a
  // transient (a clock change, another process) does not decide the plan
  double per[4][2];
  for (auto& r : per) r[0] = r[1] = 1e300;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  pplbm_status st = PPLBM_OK;
  for (int round = 0; round < 3 && st == PPLBM_OK; ++round) {
    for (int mi = 0; mi < 4 && st == PPLBM_OK; ++mi) {
      for (int wi = 0; wi < 2; ++wi) {
        if ((st = apply_plan(b, modes[mi], widths[wi])) != PPLBM_OK) break;
        if ((st = issue_steps(b, 2, b->stream)) != PPLBM_OK) break;  // warm-up
        cudaEventRecord(e0, b->stream);
        if ((st = issue_steps(b, trial_steps, b->stream)) != PPLBM_OK) break;
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          st = bfail(b, PPLBM_ERR_CUDA, "autotune timing failed");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        per[mi][wi] = std::min(per[mi][wi], (double)ms / trial_steps);
      }
    }
  }
  double best = 1e300;
  int best_mode = PPLBM_PLAN_LAUNCHES, best_w = 0;
  for (int mi = 0; mi < 4; ++mi)
    for (int wi = 0; wi < 2; ++wi)
      if (per[mi][wi] < best) {
        best = per[mi][wi];
        best_mode = modes[mi];
        best_w = widths[wi];
      }
  b->plan.ms_launches = std::min(per[0][0], per[0][1]);
  b->plan.ms_graph = std::min(per[1][0], per[1][1]);
  b->plan.ms_persistent = std::min(per[2][0], per[2][1]);
  b->plan.ms_pipelined = std::min(per[3][0], per[3][1]);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore the state into buffer parity0
  b->parity = parity0;
  off = 0;
  for (int i = 0; i < b->n; ++i) {
    const StepArgs& a = args_of(b, i);
    cudaMemcpyAsync(const_cast<double*>(a.f_in), backup + off, sizeof(double) * 9 * a.n, cudaMemcpyDeviceToDevice,
                    b->stream);
    off += 9 * (size_t)a.n;
  }
  cudaStreamSynchronize(b->stream);
  cudaFree(backup);
  b->pass_timing = pass_timing && best_mode != PPLBM_PLAN_PERSISTENT && best_mode != PPLBM_PLAN_PIPELINED;
  if (st != PPLBM_OK) return st;
  if (pplbm_status s = poll(b)) return s;
  const double keep_l = b->plan.ms_launches, keep_g = b->plan.ms_graph, keep_p = b->plan.ms_persistent;
  const double keep_q = b->plan.ms_pipelined;
  if (pplbm_status s = apply_plan(b, best_mode, best_w)) return s;
  b->plan.ms_launches = keep_l;
  b->plan.ms_graph = keep_g;
  b->plan.ms_persistent = keep_p;
  b->plan.ms_pipelined = keep_q;
  b->plan.ms_chosen = best;
  if (chosen) *chosen = b->plan;
  return PPLBM_OK;
}

pplbm_status pplbm_batch_sync(pplbm_batch* b, int64_t* steps_done) {
  if (!b) return PPLBM_ERR_ARG;
  const pplbm_status s = poll(b);
  if (steps_done) *steps_done = b->steps;
  return s;
}

pplbm_status pplbm_batch_get_derived(const pplbm_batch* b, int32_t i, pplbm_eos_derived* out) {
  if (!b || i < 0 || i >= b->n || !out) return PPLBM_ERR_ARG;
  *out = b->eos[i];
  return PPLBM_OK;
}

pplbm_status pplbm_batch_enable_timing(pplbm_batch* b, int64_t capacity) {
  if (!b || capacity < 0) return PPLBM_ERR_ARG;
  b->timing = capacity > 0;
  while (b->ev.size() < 2 * (size_t)capacity) {
    cudaEvent_t e;
    BTRY(b, cudaEventCreate(&e));
    b->ev.push_back(e);
  }
  b->ev_used = 0;
  b->timed_steps = 0;
  return PPLBM_OK;
}

pplbm_status pplbm_batch_times(pplbm_batch* b, double* ms, int64_t* steps) {
  if (!b || !ms || !steps) return PPLBM_ERR_ARG;
  BTRY(b, cudaStreamSynchronize(b->stream));
  double acc = 0.0;
  for (size_t k = 0; k + 1 < b->ev_used; k += 2) {
    float t = 0.f;
    BTRY(b, cudaEventElapsedTime(&t, b->ev[k], b->ev[k + 1]));
    acc += t;
  }
  *ms = acc;
  *steps = b->timed_steps;
  b->ev_used = 0;
  b->timed_steps = 0;
  return PPLBM_OK;
}

pplbm_status pplbm_batch_enable_pass_timing(pplbm_batch* b, int64_t capacity) {
  if (!b || capacity < 0) return PPLBM_ERR_ARG;
  if (capacity > 0 && (b->plan.mode == PPLBM_PLAN_PERSISTENT || b->plan.mode == PPLBM_PLAN_PIPELINED))
    return bfail(b, PPLBM_ERR_STATE,
                 "per-pass timing needs the launches or graph plan (the persistent and pipelined plans mix the passes)");
  BTRY(b, cudaStreamSynchronize(b->stream));
  b->pass_timing = capacity > 0;
  b->pass_capacity = capacity;
  for (int k = 0; k < 2; ++k) {
    if (pplbm_status st = grow_pass_events(b, k, 2 * (size_t)capacity)) return st;
    b->pev_used[k] = 0;
  }
  destroy_timed_graphs(b);
  if (b->pass_timing && b->plan.mode == PPLBM_PLAN_GRAPH)
    if (pplbm_status st = build_timed_graphs(b, (capacity + 1) / 2)) return st;
  return PPLBM_OK;
}

pplbm_status pplbm_batch_pass_times(pplbm_batch* b, double ms[2], int64_t launches[2]) {
  if (!b || !ms || !launches) return PPLBM_ERR_ARG;
  BTRY(b, cudaStreamSynchronize(b->stream));
  for (int k = 0; k < 2; ++k) {
    double acc = 0.0;
    for (size_t i = 0; i + 1 < b->pev_used[k]; i += 2) {
      float t = 0.f;
      BTRY(b, cudaEventElapsedTime(&t, b->pev[k][i], b->pev[k][i + 1]));
      acc += t;
    }
    ms[k] = acc;
    launches[k] = (int64_t)(b->pev_used[k] / 2);
    b->pev_used[k] = 0;
  }
  // replayed timed graphs: events 0..4 bracket density, collision, density, collision
  for (int p = 0; p < 2; ++p) {
    for (size_t g = 0; g < b->timed_used[p]; ++g) {
      const auto& tg = b->timed_graphs[p][g];
      for (int j = 0; j < 4; ++j) {
        float t = 0.f;
        BTRY(b, cudaEventElapsedTime(&t, tg.ev[j], tg.ev[j + 1]));
        ms[j & 1] += t;
        launches[j & 1] += 1;
      }
    }
    b->timed_used[p] = 0;
  }
  return PPLBM_OK;
}

pplbm_status pplbm_batch_barrier_selftest(pplbm_batch* b, uint32_t spin_limit) {
  if (!b || spin_limit < 1) return PPLBM_ERR_ARG;
  if (b->sticky) return b->sticky;
  if (b->persistent_grid < 2) return bfail(b, PPLBM_ERR_STATE, "barrier self-test needs at least two blocks");
  if (pplbm_status s = launch_persistent(b, 1, b->stream, spin_limit, b->persistent_grid - 1)) return s;
  int h = 0;
  BTRY(b, cudaMemcpyAsync(&h, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BTRY(b, cudaStreamSynchronize(b->stream));
  // the waits gave up before the collision pass, so no distribution was written:
  // clear the word and keep the batch usable
  BTRY(b, cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
  BTRY(b, cudaStreamSynchronize(b->stream));
  return (h & kErrTimeout) ? PPLBM_ERR_TIMEOUT : PPLBM_OK;
}

pplbm_status pplbm_batch_set_isolation(pplbm_batch* b, int32_t on) {
  if (!b) return PPLBM_ERR_ARG;
  b->isolate = on != 0;
  return PPLBM_OK;
}

pplbm_status pplbm_batch_guard(pplbm_batch* b, double* out) {
  if (!b || !out) return bfail(b, PPLBM_ERR_ARG, "NULL batch or output");
  if (b->sticky) return b->sticky;
  launch_density_pass(b->kind, b->d_inst, b->d_owner1, b->n1, b->parity, b->stream);
  k_batch_guard_partial<<<b->n1, kThreads, 0, b->stream>>>(b->d_inst, b->d_owner1, b->parity, b->d_snap_valid,
                                                            b->d_gpart);
  k_batch_guard_final<<<b->n, kThreads, 0, b->stream>>>(b->d_inst, b->d_gpart, b->d_snap_valid, b->d_gout);
  BTRY(b, cudaGetLastError());
  BTRY(b, cudaMemcpyAsync(out, b->d_gout, sizeof(double) * kGuardQ * b->n, cudaMemcpyDefault, b->stream));
  BTRY(b, cudaStreamSynchronize(b->stream));
  return poll(b);
}

pplbm_status pplbm_batch_instance_status(pplbm_batch* b, int32_t* status) {
  if (!b || !status) return PPLBM_ERR_ARG;
  const pplbm_status s = poll(b);
  for (int i = 0; i < b->n; ++i) status[i] = b->diverged[i] ? PPLBM_ERR_DIVERGED : PPLBM_OK;
  return s;
}

const char* pplbm_batch_last_error(const pplbm_batch* b) { return b ? b->msg.c_str() : ""; }

void pplbm_batch_destroy(pplbm_batch* b) {
  if (!b) return;
  destroy_graphs(b);
  destroy_timed_graphs(b);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  for (int k = 0; k < 2; ++k)
    for (cudaEvent_t e : b->pev[k]) cudaEventDestroy(e);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  if (b->dev_block) cudaFree(b->dev_block);
  delete b;
}

}  // extern "C"
