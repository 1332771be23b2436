// gbmd_api.cu -- the C ABI of libgbmd (include/gbmd.h): systems, batches, CUDA
// graphs with a device-decided rebuild, overflow recovery, readouts, autotuning.
//
// A "group" is the unit that is stepped: one system alone, or a batch of systems.
// Its step is a CUDA graph per block of steps; per step:
//   step kernel (pair force K5 + integration K6) -> IF(any system needs a rebuild)
//   { bin -> scan -> scatter -> cellsort -> permute -> copyback -> [blocks] -> nlist }.
// The IF is a graph conditional node whose value the step kernel's last block sets
// on the device, so a step never returns to the host.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "launch.cuh"

using namespace gbmd;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? GBMD_ERR_OOM : GBMD_ERR_CUDA,          \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    }                                                                                    \
  } while (0)

#define RET(x)                 \
  do {                         \
    int r_ = (x);              \
    if (r_ != GBMD_OK) return r_; \
  } while (0)

constexpr int STEPS_PER_GRAPH = 16;
constexpr int STAGED_WINDOW_CAP = 3072;   // window particles in 48 KB of shared memory

size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

// NVTX range over a host call (the timeline of a profiler shows the library's
// calls: enqueues, rebuild recoveries, readouts); a no-op unless a tool is attached
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

}  // namespace

struct Group;

struct gbmd_system {
  int device = 0;             // CUDA ordinal every call on this system uses
  SysDev h{};                 // master descriptor (device pointers)
  Flags* d_flags = nullptr;
  cudaStream_t stream = nullptr;     // the caller's stream
  std::vector<void*> allocs;
  size_t footprint = 0;
  Group* own = nullptr;       // the system alone
  Group* batch = nullptr;
  int batch_slot = -1;
  long long target_step = 0;  // steps requested so far (absolute), host bookkeeping
  long long step_limit = -1;
  double cell_min = 0;        // smallest allowed cell width: r_list,max (cell list) or
                              // r_list,min (tree list, whose cells only order particles)
  double cell_scale = 1.0;    // cell width >= cell_scale * cell_min (autotuned)
  bool want_staged = false;   // GBMD_PATH_STAGED requested
  // staging for import/export (device)
  double *d_pos = nullptr, *d_vel = nullptr, *d_frc = nullptr;
  int *d_img = nullptr, *d_type = nullptr, *d_misc = nullptr;
  double *d_ppu = nullptr, *d_ppw = nullptr;   // per-particle readout staging (lazy)
  double* d_thermo = nullptr;
};

struct Group {
  int device = 0;
  std::vector<gbmd_system*> members;   // may contain nullptr (free slots of a batch)
  bool is_batch = false;
  int precision = GBMD_MIXED;
  int multi = 0;   // pair-table mode: 0 one type, 1 at most two, 2 more
  bool rel = true;     // every member has at least 3 cells on every axis
  cudaStream_t stream = nullptr;
  int tpp = 2, fblock = 128;
  // device tables
  SysDev* d_desc = nullptr;
  Tile *d_tp = nullptr, *d_tf = nullptr, *d_tc = nullptr, *d_ts = nullptr;
  Tile *d_tb = nullptr, *d_tbk = nullptr;   // staged force blocks; their window kernel
  Tile* d_te = nullptr;   // energy/virial launches: EV_TILE_P particles per tile, whatever
                          // the tuning, so the FP64 sums do not depend on it
  Tile* d_tt = nullptr;   // tree-list systems: tiles over their trees' leaves
  int ntp = 0, ntf = 0, ntc = 0, nts = 0, ntb = 0, ntbk = 0, nte = 0, ntt = 0;
  size_t cap_desc = 0, cap_tp = 0, cap_tf = 0, cap_tc = 0, cap_ts = 0, cap_part = 0;
  size_t cap_tb = 0, cap_tbk = 0, cap_te = 0, cap_tt = 0;
  bool any_cell = true;   // some member builds its list from cells
  int window_cap = 0;                        // largest staged window among members
  bool nvt = false;                          // the members integrate NVT (all or none)
  int eval = EVAL_LJ;                        // the members' pair evaluator (all the same)
  double* d_nhpart = nullptr;                // NVT: per-step-tile v.v partial sums
  size_t cap_nhpart = 0;
  double* d_partials = nullptr;
  GroupCtl* d_ctl = nullptr;
  cudaGraphExec_t exec_many = nullptr, exec_one = nullptr;
  // optional event records around the force kernel of the single-step graph
  cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
  cudaGraph_t graph_one = nullptr;                 // kept alive for node updates
  cudaGraphNode_t node_ev_begin = nullptr, node_ev_end = nullptr;
  bool layout_dirty = true;
  bool graphs_dirty = true;
  bool use_graphs = true;
};

namespace {

// make `dev` current for this thread in this library's CUDA runtime
int use_device(int dev) {
  int cur = -1;
  if (cudaGetDevice(&cur) == cudaSuccess && cur == dev) return GBMD_OK;
  CK(cudaSetDevice(dev));
  return GBMD_OK;
}

std::vector<gbmd_system*> live(const Group* g) {
  std::vector<gbmd_system*> v;
  for (auto* s : g->members)
    if (s) v.push_back(s);
  return v;
}

template <typename T>
int grow(T** p, size_t* cap, size_t need) {
  if (*cap >= need && *p) return GBMD_OK;
  if (*p) CK(cudaFree(*p));
  *p = nullptr;
  size_t n = std::max<size_t>(need, 1);
  CK(cudaMalloc((void**)p, n * sizeof(T)));
  *cap = n;
  return GBMD_OK;
}

void destroy_graphs(Group* g) {
  if (g->exec_many) cudaGraphExecDestroy(g->exec_many);
  if (g->exec_one) cudaGraphExecDestroy(g->exec_one);
  if (g->graph_one) cudaGraphDestroy(g->graph_one);
  g->exec_many = g->exec_one = nullptr;
  g->graph_one = nullptr;
  g->node_ev_begin = g->node_ev_end = nullptr;
  g->graphs_dirty = true;
}

// Rebuild descriptor copies and tile tables for the group's current members.
int sync_layout(Group* g) {
  if (!g->layout_dirty) return GBMD_OK;
  std::vector<gbmd_system*> m = live(g);
  std::vector<SysDev> desc;
  std::vector<Tile> tp, tf, tc, ts, tb, tbk, te, tt;
  const int per_f = g->fblock / g->tpp;
  g->multi = 0;
  g->rel = true;
  g->window_cap = 0;
  g->nvt = !m.empty() && m[0]->h.nvt;
  g->eval = m.empty() ? EVAL_LJ : m[0]->h.eval;
  g->any_cell = false;
  for (size_t k = 0; k < m.size(); ++k) {
    SysDev d = m[k]->h;
    const int n = d.n;
    for (int f = 0; f < n; f += TILE_P) tp.push_back({(int)k, f, std::min(TILE_P, n - f), 0});
    if (d.staged) {   // one force tile per 2x2x2 block of cells
      d.tile_first_f = (int)tb.size();   // shifted past the global tiles below
      for (int b = 0; b < d.nblocks; ++b) tb.push_back({(int)k, b, 1, 0});
      d.tile_count_f = d.nblocks;
      for (int b = 0; b < d.nblocks; b += 8) tbk.push_back({(int)k, b, std::min(8, d.nblocks - b), 0});
      g->window_cap = std::max(g->window_cap, d.window_cap);
    } else {
      d.tile_first_s = (int)tf.size();
      for (int f = 0; f < n; f += per_f) tf.push_back({(int)k, f, std::min(per_f, n - f), 0});
      d.tile_count_s = (int)tf.size() - d.tile_first_s;
      d.tile_first_f = (int)te.size();   // partial sums come from the energy launches
      for (int f = 0; f < n; f += EV_TILE_P) te.push_back({(int)k, f, std::min(EV_TILE_P, n - f), 0});
      d.tile_count_f = (int)te.size() - d.tile_first_f;
    }
    for (int c = 0; c < d.nbins; c += CELLS_PER_TILE)
      tc.push_back({(int)k, c, std::min(CELLS_PER_TILE, d.nbins - c), 0});
    ts.push_back({(int)k, 0, 0, 0});
    if (d.tree)
      for (int f = 0; f < d.tree_leaves_total; f += TILE_P)
        tt.push_back({(int)k, f, std::min(TILE_P, d.tree_leaves_total - f), 0});
    desc.push_back(d);
    if (d.ntypes > 1) g->multi = std::max(g->multi, d.ntypes > 2 ? 2 : 1);
    if (!d.tree) {
      g->any_cell = true;
      if (d.nc[0] < 3 || d.nc[1] < 3 || d.nc[2] < 3) g->rel = false;
    }
  }
  for (auto& d : desc)
    if (d.staged) d.tile_first_f += (int)te.size();   // staged partial sums follow the global ones
  RET(grow(&g->d_partials, &g->cap_part, 8 * std::max<size_t>(te.size() + tb.size(), 1)));
  RET(grow(&g->d_nhpart, &g->cap_nhpart, std::max<size_t>(tf.size(), 1)));
  for (auto& d : desc) {
    d.partials = g->d_partials;
    d.nh_part = g->d_nhpart;
  }
  RET(grow(&g->d_desc, &g->cap_desc, desc.size()));
  RET(grow(&g->d_tp, &g->cap_tp, tp.size()));
  RET(grow(&g->d_tf, &g->cap_tf, tf.size()));
  RET(grow(&g->d_tc, &g->cap_tc, tc.size()));
  RET(grow(&g->d_ts, &g->cap_ts, ts.size()));
  RET(grow(&g->d_tb, &g->cap_tb, tb.size()));
  RET(grow(&g->d_tbk, &g->cap_tbk, tbk.size()));
  RET(grow(&g->d_te, &g->cap_te, te.size()));
  RET(grow(&g->d_tt, &g->cap_tt, tt.size()));
  if (!g->d_ctl) {
    CK(cudaMalloc(&g->d_ctl, sizeof(GroupCtl)));
    CK(cudaMemsetAsync(g->d_ctl, 0, sizeof(GroupCtl), g->stream));
  }
  auto up = [&](void* dst, const std::vector<Tile>& v) -> cudaError_t {
    if (v.empty()) return cudaSuccess;
    return cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(Tile), cudaMemcpyHostToDevice, g->stream);
  };
  if (!desc.empty()) CK(cudaMemcpyAsync(g->d_desc, desc.data(), desc.size() * sizeof(SysDev), cudaMemcpyHostToDevice, g->stream));
  CK(up(g->d_tp, tp));
  CK(up(g->d_tf, tf));
  CK(up(g->d_tc, tc));
  CK(up(g->d_ts, ts));
  CK(up(g->d_tb, tb));
  CK(up(g->d_tbk, tbk));
  CK(up(g->d_te, te));
  CK(up(g->d_tt, tt));
  CK(cudaStreamSynchronize(g->stream));   // host vectors die here
  g->ntp = (int)tp.size();
  g->ntf = (int)tf.size();
  g->ntc = (int)tc.size();
  g->nts = (int)ts.size();
  g->ntb = (int)tb.size();
  g->ntbk = (int)tbk.size();
  g->nte = (int)te.size();
  g->ntt = (int)tt.size();
  g->layout_dirty = false;
  destroy_graphs(g);
  return GBMD_OK;
}

// update one member's descriptor in every group it belongs to (pointer/size change)
int refresh_desc(gbmd_system* s) {
  for (Group* g : {s->own, s->batch}) {
    if (!g) continue;
    g->layout_dirty = true;
    RET(sync_layout(g));
  }
  return GBMD_OK;
}

// the rebuild: cell sort (and re-sort), then the lists -- cell-list members by
// k_nlist (after the staged windows, if any), tree-list members by k_tree_*
std::vector<KernelCall> rebuild_calls(const Group* g) {
  std::vector<KernelCall> v = {bin_call(g->d_desc, g->d_tp, g->ntp, g->d_ctl),
                               scan_call(g->d_desc, g->d_ts, g->nts, g->d_ctl),
                               scatter_call(g->d_desc, g->d_tp, g->ntp, g->d_ctl),
                               cellsort_call(g->d_desc, g->d_tc, g->ntc, g->d_ctl),
                               permute_call(g->d_desc, g->d_tp, g->ntp, g->d_ctl),
                               copyback_call(g->d_desc, g->d_tp, g->ntp, g->d_ctl)};
  if (g->ntbk > 0) v.push_back(blocks_call(g->d_desc, g->d_tbk, g->ntbk, g->d_ctl));
  if (g->any_cell)
    v.push_back(nlist_call(g->d_desc, g->d_tc, g->ntc, g->d_ctl, g->rel, g->multi, g->ntbk > 0));
  if (g->ntt > 0) {
    v.push_back(tree_build_call(g->d_desc, g->d_tt, g->ntt, g->d_ctl));
    v.push_back(tree_nlist_call(g->d_desc, g->d_tp, g->ntp, g->d_ctl));
  }
  return v;
}

// forces at the current positions, outside the step (autotuning, readouts)
KernelCall plain_force_call(const Group* g) {
  return force_call(g->precision, g->multi, MODE_FORCE, g->tpp, g->fblock, g->d_desc, g->d_tf,
                    g->ntf, g->d_ctl, StepArgs{}, g->eval);
}

// energy/virial launch of the global-list systems: the step's threads per particle
// (so the FP32 forces it writes are bitwise the step's), EV_TILE_P particles per block
KernelCall ev_force_call(const Group* g, const SysDev* desc) {
  return force_call(g->precision, g->multi, MODE_EV, g->tpp, EV_TILE_P * g->tpp, desc, g->d_te,
                    g->nte, g->d_ctl, StepArgs{}, g->eval);
}

// readout force launches (ev = 0 forces, 1 also energy/virial): global-list systems,
// then staged ones
std::vector<KernelCall> force_calls(const Group* g, int ev) {
  std::vector<KernelCall> v;
  if (g->ntf > 0) v.push_back(ev ? ev_force_call(g, g->d_desc) : plain_force_call(g));
  if (g->ntb > 0)
    v.push_back(force_staged_call(g->multi, ev ? MODE_EV : MODE_FORCE, g->d_desc, g->d_tb, g->ntb,
                                  g->d_ctl, g->nte, g->window_cap, StepArgs{}));
  return v;
}

// the step kernels: force + integrate of every member, global-list systems then
// staged ones; the last of all their blocks makes the step's decisions and sets
// `cond` (when use_cond) for the rebuild that follows
std::vector<KernelCall> step_calls(const Group* g, cudaGraphConditionalHandle cond, int use_cond) {
  StepArgs sa;
  sa.nsys = (int)live(g).size();
  sa.total_blocks = g->ntf + g->ntb;
  sa.cond = cond;
  sa.use_cond = use_cond;
  std::vector<KernelCall> v;
  if (g->nvt) {   // forces + closing half + thermostat, then the opening half and drift
    StepArgs a = sa;
    a.total_blocks = g->ntf;
    a.cond = 0;
    a.use_cond = 0;
    v.push_back(force_call(g->precision, g->multi, MODE_NVT_A, g->tpp, g->fblock, g->d_desc, g->d_tf,
                           g->ntf, g->d_ctl, a, g->eval));
    StepArgs b = sa;
    b.total_blocks = g->ntp;
    v.push_back(nvt_b_call(g->precision, g->d_desc, g->d_tp, g->ntp, g->d_ctl, b));
    return v;
  }
  if (g->ntf > 0)
    v.push_back(force_call(g->precision, g->multi, MODE_STEP, g->tpp, g->fblock, g->d_desc, g->d_tf,
                           g->ntf, g->d_ctl, sa, g->eval));
  if (g->ntb > 0)
    v.push_back(force_staged_call(g->multi, MODE_STEP, g->d_desc, g->d_tb, g->ntb, g->d_ctl, g->nte,
                                  g->window_cap, sa));
  return v;
}

int add_kernel(cudaGraph_t graph, const cudaGraphNode_t* dep, const KernelCall& k,
               cudaGraphNode_t* out) {
  cudaKernelNodeParams p{};
  p.func = k.func;
  p.gridDim = k.grid;
  p.blockDim = k.block;
  p.sharedMemBytes = (unsigned)k.smem;
  void* a[10];
  args_of(k, a);
  p.kernelParams = a;
  p.extra = nullptr;
  CK(cudaGraphAddKernelNode(out, graph, dep, dep ? 1 : 0, &p));
  return GBMD_OK;
}

int build_graph(Group* g, int nsteps, cudaGraphExec_t* exec) {
  cudaGraph_t graph;
  CK(cudaGraphCreate(&graph, 0));
  const bool events = nsteps == 1 && g->ev_begin && g->ev_end;
  cudaGraphNode_t prev = nullptr;
  const int nsys = (int)live(g).size();
  int rc = GBMD_OK;
  for (int st = 0; st < nsteps && rc == GBMD_OK; ++st) {
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { rc = fail(GBMD_ERR_CUDA, "conditional handle: %s", cudaGetErrorString(e)); break; }
    // force + integrate (event nodes around them when asked), then IF(rebuild){lists}
    cudaGraphNode_t before = prev;
    if (events) {
      e = cudaGraphAddEventRecordNode(&g->node_ev_begin, graph, before ? &before : nullptr, before ? 1 : 0,
                                      g->ev_begin);
      if (e != cudaSuccess) { rc = fail(GBMD_ERR_CUDA, "event node: %s", cudaGetErrorString(e)); break; }
      before = g->node_ev_begin;
    }
    for (const KernelCall& k : step_calls(g, h, 1)) {
      cudaGraphNode_t n5;
      rc = add_kernel(graph, before ? &before : nullptr, k, &n5);
      if (rc) break;
      before = n5;
    }
    if (rc) break;
    if (events) {
      e = cudaGraphAddEventRecordNode(&g->node_ev_end, graph, &before, 1, g->ev_end);
      if (e != cudaSuccess) { rc = fail(GBMD_ERR_CUDA, "event node: %s", cudaGetErrorString(e)); break; }
      before = g->node_ev_end;
    }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t nc;
    e = cudaGraphAddNode(&nc, graph, &before, nullptr, 1, &cp);
    if (e != cudaSuccess) { rc = fail(GBMD_ERR_CUDA, "conditional node: %s", cudaGetErrorString(e)); break; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaGraphNode_t bprev = nullptr;
    for (const KernelCall& k : rebuild_calls(g)) {
      cudaGraphNode_t bn;
      rc = add_kernel(body, bprev ? &bprev : nullptr, k, &bn);
      if (rc) break;
      bprev = bn;
    }
    if (rc) break;
    prev = nc;
  }
  if (rc == GBMD_OK) {
    cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
    if (e != cudaSuccess) rc = fail(GBMD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  if (events && rc == GBMD_OK) g->graph_one = graph;   // node handles stay valid
  else cudaGraphDestroy(graph);
  return rc;
}

int ensure_graphs(Group* g) {
  RET(sync_layout(g));
  if (!g->graphs_dirty) return GBMD_OK;
  RET(build_graph(g, STEPS_PER_GRAPH, &g->exec_many));
  RET(build_graph(g, 1, &g->exec_one));
  g->graphs_dirty = false;
  return GBMD_OK;
}

// enqueue n steps of the group (graphs, or direct launches when graphs are off)
int enqueue_steps(Group* g, long long n) {
  if (n <= 0 || live(g).empty()) return GBMD_OK;
  RET(sync_layout(g));
  if (g->use_graphs) {
    RET(ensure_graphs(g));
    for (long long k = 0; k < n / STEPS_PER_GRAPH; ++k) CK(cudaGraphLaunch(g->exec_many, g->stream));
    for (long long k = 0; k < n % STEPS_PER_GRAPH; ++k) CK(cudaGraphLaunch(g->exec_one, g->stream));
    return GBMD_OK;
  }
  for (long long k = 0; k < n; ++k) {
    const bool events = n == 1 && g->ev_begin && g->ev_end;
    if (events) CK(cudaEventRecord(g->ev_begin, g->stream));
    {
      Range r("gbmd step kernel launches");
      for (const KernelCall& c : step_calls(g, 0, 0)) CK(launch(c, g->stream));
    }
    if (events) CK(cudaEventRecord(g->ev_end, g->stream));
    Range r("gbmd rebuild kernel launches");
    for (const KernelCall& c : rebuild_calls(g)) CK(launch(c, g->stream));
  }
  return GBMD_OK;
}

int read_flags(gbmd_system* s, Flags* f, cudaStream_t st) {
  CK(cudaMemcpyAsync(f, s->d_flags, sizeof(Flags), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return GBMD_OK;
}

int write_flags(gbmd_system* s, const Flags* f, cudaStream_t st) {
  CK(cudaMemcpyAsync(s->d_flags, f, sizeof(Flags), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return GBMD_OK;
}

cudaStream_t cur_stream(gbmd_system* s) { return s->own->stream; }

// rebuild lists (when flags->do_rebuild) + forces, outside any graph, for the system alone
int rebuild_and_force(gbmd_system* s, int ev) {
  Group* g = s->own;
  RET(sync_layout(g));
  for (const KernelCall& c : rebuild_calls(g)) CK(launch(c, g->stream));
  for (const KernelCall& c : force_calls(g, ev)) CK(launch(c, g->stream));
  return GBMD_OK;
}

int dalloc(gbmd_system* s, void** p, size_t bytes) {
  bytes = std::max<size_t>(bytes, 16);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return fail(GBMD_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  s->allocs.push_back(*p);
  s->footprint += bytes;
  return GBMD_OK;
}

// Grow the neighbour list to hold `need` neighbours per particle.
int grow_nlist(gbmd_system* s, int need) {
  const int cap = (int)round_up((size_t)need + need / 4 + 8, 8);
  CK(cudaStreamSynchronize(cur_stream(s)));
  auto it = std::find(s->allocs.begin(), s->allocs.end(), (void*)s->h.nl);
  if (it != s->allocs.end()) {
    s->allocs.erase(it);
    s->footprint -= (size_t)s->h.nl_stride * s->h.cap * sizeof(int);
  }
  CK(cudaFree(s->h.nl));
  s->h.nl = nullptr;
  RET(dalloc(s, (void**)&s->h.nl, (size_t)s->h.nl_stride * cap * sizeof(int)));
  s->h.cap = cap;
  return refresh_desc(s);
}

// Wait for the system's work; recover from overflow; run what remains of its steps.
int sync_system(gbmd_system* s) {
  cudaStream_t st = cur_stream(s);
  for (int round = 0; round < 64; ++round) {
    CK(cudaStreamSynchronize(st));
    Flags f;
    RET(read_flags(s, &f, st));
    if (f.error == DEV_NONFINITE)
      return fail(GBMD_ERR_NONFINITE, "non-finite coordinate or a particle moved more than L/2 in one step (step %lld)", f.step);
    if (f.error == DEV_WINDOW) {   // a staged window outgrew shared memory
      s->h.staged = 0;
      RET(refresh_desc(s));
      f.error = 0;
      f.do_rebuild = 1;
      RET(write_flags(s, &f, st));
      RET(rebuild_and_force(s, 0));
      continue;
    }
    if (f.error == DEV_OVERFLOW) {
      Range r("gbmd neighbour-list overflow recovery");
      RET(grow_nlist(s, std::max(f.overflow_need, s->h.cap + 1)));
      f.error = 0;
      f.overflow_need = 0;
      f.do_rebuild = 1;
      RET(write_flags(s, &f, st));
      RET(rebuild_and_force(s, 0));   // finishes the interrupted step
      continue;
    }
    if (f.error == DEV_TREE)
      return fail(GBMD_ERR_TIMEOUT, "a tree traversal passed its node bound (step %lld)", f.step);
    if (f.error) return fail(GBMD_ERR_CUDA, "unknown device error %d", f.error);
    long long want = s->target_step;
    if (s->step_limit >= 0) want = std::min(want, s->step_limit);
    if (f.step < want) {
      RET(enqueue_steps(s->own, want - f.step));
      continue;
    }
    return GBMD_OK;
  }
  return fail(GBMD_ERR_NLIST_OVERFLOW, "neighbour list kept overflowing");
}

// the cut-off radius of type pair p: the rcut table, except WCA's 2^(1/6) sigma
double cut_of(const gbmd_desc* d, int p) {
  return d->potential == GBMD_POT_WCA ? std::pow(2.0, 1.0 / 6.0) * d->sigma[p] : d->rcut[p];
}

// the pair tables the potential reads: present, finite, in range and symmetric
int validate_pairs(const gbmd_desc* d, double* rmax_out) {
  const int pot = d->potential;
  if (pot < GBMD_POT_LJ || pot > GBMD_POT_GAUSS) return fail(GBMD_ERR_BAD_ARG, "potential must be a gbmd_potential (0..4)");
  const bool need_sigma = pot != GBMD_POT_YUKAWA, need_rcut = pot != GBMD_POT_WCA;
  const bool signed_eps = pot == GBMD_POT_YUKAWA || pot == GBMD_POT_GAUSS;
  if (!d->eps || (need_sigma && !d->sigma) || (need_rcut && !d->rcut))
    return fail(GBMD_ERR_BAD_ARG, "a pair table the potential reads (eps, sigma, rcut) is NULL");
  if (pot == GBMD_POT_MIE && (!d->mie_n || !d->mie_m)) return fail(GBMD_ERR_BAD_ARG, "Mie needs mie_n and mie_m");
  if (pot == GBMD_POT_YUKAWA && !d->kappa) return fail(GBMD_ERR_BAD_ARG, "Yukawa needs kappa");
  const int nt = d->ntypes;
  double rmax = 0;
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      const int p = a * nt + b, q = b * nt + a;
      auto sym = [&](const double* t) { return !t || t[p] == t[q]; };
      const double e = d->eps[p];
      if (!std::isfinite(e) || (signed_eps ? e == 0 : !(e > 0)))
        return fail(GBMD_ERR_BAD_ARG, "eps must be finite and %s", signed_eps ? "nonzero" : "positive");
      if (need_sigma && (!(d->sigma[p] > 0) || !std::isfinite(d->sigma[p])))
        return fail(GBMD_ERR_BAD_ARG, "sigma must be positive and finite");
      if (need_rcut && (!(d->rcut[p] > 0) || !std::isfinite(d->rcut[p])))
        return fail(GBMD_ERR_BAD_ARG, "rcut must be positive and finite");
      if (pot == GBMD_POT_MIE && !(d->mie_m[p] > 0 && d->mie_n[p] > d->mie_m[p] && std::isfinite(d->mie_n[p])))
        return fail(GBMD_ERR_BAD_ARG, "Mie exponents need 0 < m < n (finite)");
      if (pot == GBMD_POT_YUKAWA && !(d->kappa[p] >= 0 && std::isfinite(d->kappa[p])))
        return fail(GBMD_ERR_BAD_ARG, "kappa must be >= 0 and finite");
      const bool s = sym(d->eps) && (!need_sigma || sym(d->sigma)) && (!need_rcut || sym(d->rcut)) &&
                     (pot != GBMD_POT_MIE || (sym(d->mie_n) && sym(d->mie_m))) &&
                     (pot != GBMD_POT_YUKAWA || sym(d->kappa));
      if (!s) return fail(GBMD_ERR_BAD_ARG, "pair parameter tables must be symmetric");
      rmax = std::max(rmax, cut_of(d, p));
    }
  *rmax_out = rmax;
  return GBMD_OK;
}

int validate(const gbmd_desc* d, bool device) {
  if (!d) return fail(GBMD_ERR_BAD_ARG, "desc is NULL");
  if (d->n < 1 || d->n > (1LL << 30)) return fail(GBMD_ERR_BAD_ARG, "n must be in [1, 2^30], got %lld", (long long)d->n);
  if (!d->pos || !d->vel) return fail(GBMD_ERR_BAD_ARG, "pos and vel must not be NULL");
  if (d->ntypes < 1 || d->ntypes > GBMD_MAX_TYPES) return fail(GBMD_ERR_BAD_ARG, "ntypes must be in [1, %d]", GBMD_MAX_TYPES);
  for (int a = 0; a < 3; ++a)
    if (!(d->box[a] > 0) || !std::isfinite(d->box[a])) return fail(GBMD_ERR_BAD_ARG, "box edges must be positive and finite");
  if (!(d->dt > 0) || !(d->mass > 0) || !(d->r_buff >= 0) || !std::isfinite(d->dt) || !std::isfinite(d->r_buff))
    return fail(GBMD_ERR_BAD_ARG, "need dt > 0, mass > 0, r_buff >= 0");
  if (d->precision != GBMD_FP64 && d->precision != GBMD_MIXED) return fail(GBMD_ERR_BAD_ARG, "precision must be GBMD_FP64 or GBMD_MIXED");
  if (d->sort_period < 0 || d->nlist_capacity < 0) return fail(GBMD_ERR_BAD_ARG, "sort_period and nlist_capacity must be >= 0");
  if (d->threads_per_particle != 0 && !tpp_supported(d->threads_per_particle))
    return fail(GBMD_ERR_BAD_ARG, "threads_per_particle must be 0, 1, 2 or 4");
  if (d->force_path != GBMD_PATH_GLOBAL && d->force_path != GBMD_PATH_STAGED)
    return fail(GBMD_ERR_BAD_ARG, "force_path must be GBMD_PATH_GLOBAL or GBMD_PATH_STAGED");
  if (d->integrator != GBMD_NVE && d->integrator != GBMD_NVT)
    return fail(GBMD_ERR_BAD_ARG, "integrator must be GBMD_NVE or GBMD_NVT");
  if (d->nlist != GBMD_NLIST_CELL && d->nlist != GBMD_NLIST_TREE)
    return fail(GBMD_ERR_BAD_ARG, "nlist must be GBMD_NLIST_CELL or GBMD_NLIST_TREE");
  if (d->integrator == GBMD_NVT &&
      (!(d->kT > 0) || !(d->tau > 0) || !std::isfinite(d->kT) || !std::isfinite(d->tau) || d->n < 2))
    return fail(GBMD_ERR_BAD_ARG, "NVT needs kT > 0, tau > 0 and at least 2 particles");
  if (d->n_ghost < 0 || d->n_ghost >= d->n) return fail(GBMD_ERR_BAD_ARG, "n_ghost must be in [0, n)");
  if (d->n_ghost > 0 && (d->integrator != GBMD_NVE || d->force_path != GBMD_PATH_GLOBAL))
    return fail(GBMD_ERR_BAD_ARG, "ghosts need the NVE integrator and the global force path");
  const int nt = d->ntypes;
  double rmax = 0;
  RET(validate_pairs(d, &rmax));
  const double rl = rmax + d->r_buff;
  for (int a = 0; a < 3; ++a)
    if (d->box[a] < 2.0 * rl)
      return fail(GBMD_ERR_BOX_TOO_SMALL, "box edge %d (%g) < 2 (r_cut,max + r_buff) = %g", a, d->box[a], 2 * rl);
  if (!device) {
    for (int64_t i = 0; i < 3 * d->n; ++i)
      if (!std::isfinite(d->pos[i]) || !std::isfinite(d->vel[i])) return fail(GBMD_ERR_BAD_ARG, "non-finite position or velocity");
    if (d->type)
      for (int64_t i = 0; i < d->n; ++i)
        if (d->type[i] < 0 || d->type[i] >= nt) return fail(GBMD_ERR_BAD_ARG, "type id out of range at %lld", (long long)i);
  }
  return GBMD_OK;
}

// the evaluator coefficients of type pair p (PairD's p0..p4 and the unshifted
// V(r_cut) as `shift`), cut at rc
void pair_coefficients(const gbmd_desc* d, int p, double rc, PairD* c) {
  const double e = d->eps[p];
  switch (d->potential) {
    case GBMD_POT_MIE: {
      const double sg = d->sigma[p], n = d->mie_n[p], m = d->mie_m[p];
      const double ce = n / (n - m) * std::pow(n / m, m / (n - m)) * e;
      const double x = sg * sg / (rc * rc);
      c->p0 = sg * sg;
      c->p1 = 0.5 * n;
      c->p2 = 0.5 * m;
      c->p3 = ce;
      c->shift = ce * (std::pow(x, 0.5 * n) - std::pow(x, 0.5 * m));
      break;
    }
    case GBMD_POT_YUKAWA: {
      const double k = d->kappa[p];
      c->p0 = e;
      c->p1 = k;
      c->shift = e * std::exp(-k * rc) / rc;
      break;
    }
    case GBMD_POT_GAUSS: {
      const double sg = d->sigma[p];
      c->p0 = e;
      c->p1 = 1.0 / (2.0 * sg * sg);
      c->p2 = e / (sg * sg);
      c->shift = e * std::exp(-rc * rc / (2.0 * sg * sg));
      break;
    }
    default: {   // LJ; WCA with rc = 2^(1/6) sigma
      const double sg = d->sigma[p];
      const double s6 = std::pow(sg, 6.0), s12 = s6 * s6;
      const double c2 = sg * sg / (rc * rc), c6 = c2 * c2 * c2, c12 = c6 * c6;
      c->p0 = 48.0 * e * s12;
      c->p1 = 24.0 * e * s6;
      c->p3 = 4.0 * e * s12;
      c->p4 = 4.0 * e * s6;
      c->shift = 4.0 * e * (c12 - c6);
    }
  }
}

struct Geometry {
  int nc[3];
  int ncells;
  int nbins;        // sort bins: ncells, or ntypes * ncells on the tree list
  int cap;
  double rl_max;
  double cell_min;  // smallest cell width
};

// cells per axis: as many as fit with a width of at least scale * cell_min (for the
// cell list cell_min = r_list,max: the 27-cell stencil then holds every neighbour),
// at most 1024
int cells_along(double L, double cell_min, double scale) {
  const int c = (int)std::floor(L / (cell_min * scale * (1.0 + 1e-6)));
  return std::min(std::max(c, 1), 1024);
}

// type_counts (particles per type, or NULL when unknown) refines the default list
// capacity of the tree list: sum over types t of rho_t (4/3) pi r_list(i, t)^3 for the
// worst type i, instead of rho (4/3) pi r_list,max^3
Geometry geometry(const gbmd_desc* d, const int64_t* type_counts = nullptr) {
  Geometry g;
  const int nt = d->ntypes;
  const bool tree = d->nlist == GBMD_NLIST_TREE;
  double rmax = 0, rmin = 1e300;
  for (int p = 0; p < nt * nt; ++p) {
    rmax = std::max(rmax, cut_of(d, p));
    rmin = std::min(rmin, cut_of(d, p));
  }
  const double vol = d->box[0] * d->box[1] * d->box[2];
  g.rl_max = rmax + d->r_buff;
  // the tree list's cells only order the particles (by Morton code inside a cell):
  // about 32 particles per cell, and no finer than the smallest r_list
  g.cell_min = tree ? std::max(rmin + d->r_buff, std::cbrt(32.0 * vol / (double)d->n)) : g.rl_max;
  g.ncells = 1;
  for (int a = 0; a < 3; ++a) {
    g.nc[a] = cells_along(d->box[a], g.cell_min, 1.0);
    g.ncells *= g.nc[a];
  }
  g.nbins = tree ? nt * g.ncells : g.ncells;
  if (d->nlist_capacity > 0) {
    g.cap = (int)round_up((size_t)d->nlist_capacity, 4);   // whole slot groups
  } else {
    const double rho = (double)d->n / vol;
    double nexp = rho * 4.0 / 3.0 * M_PI * g.rl_max * g.rl_max * g.rl_max;
    if (tree && type_counts) {
      nexp = 0;
      for (int a = 0; a < nt; ++a) {
        double e = 0;
        for (int b = 0; b < nt; ++b) {
          const double rl = cut_of(d, a * nt + b) + d->r_buff;
          e += (double)type_counts[b] / vol * 4.0 / 3.0 * M_PI * rl * rl * rl;
        }
        if (type_counts[a] > 0) nexp = std::max(nexp, e);
      }
    }
    g.cap = (int)round_up((size_t)(nexp * 1.4 + 24), 8);
    g.cap = std::min<int>(g.cap, (int)std::max<int64_t>(8, round_up((size_t)d->n, 8)));
  }
  return g;
}

uint32_t spread3(uint32_t v) {   // 10 bits -> every third bit
  v &= 0x3ff;
  v = (v | (v << 16)) & 0x030000FF;
  v = (v | (v << 8)) & 0x0300F00F;
  v = (v | (v << 4)) & 0x030C30C3;
  v = (v | (v << 2)) & 0x09249249;
  return v;
}

size_t footprint_of(const gbmd_desc* d, const Geometry& g) {
  const size_t n = (size_t)d->n;
  size_t b = 0;
  b += n * (8 * 3 * 2);          // x, v
  b += n * 4 * 3 + n * 4 * 3;    // img, rtag/tag/type
  b += n * 16 * 3;               // q (two step-parity buffers), q_build
  if (d->precision == GBMD_FP64) b += n * 32 * 2;   // p64 (two buffers)
  b += n * (d->precision == GBMD_FP64 ? 32 : 16);   // force
  b += n * 4 + round_up(n, 32) * 4 * (size_t)g.cap;  // nn, nl (ELL4)
  b += n * (4 * 5 + 16) + (size_t)(g.nbins + 1) * 4 * 3 + (size_t)g.ncells * 4 * 2;   // cells, keys
  if (d->nlist == GBMD_NLIST_TREE)   // tree boxes and arrival counters (<= n + 4 ntypes
    b += (n + 4 * (size_t)d->ntypes) * (sizeof(TreeBox) + 4) + n * 16;  // nodes), leaves
  b += (size_t)((g.nc[0] + 1) / 2) * ((g.nc[1] + 1) / 2) * ((g.nc[2] + 1) / 2) *
       (WIN_CELLS * 8 + 16);                                                      // staged blocks
  b += n * (8 * 3 * 2 + 4 * 3 + 4 * 2 + 16);         // re-sort scratch
  b += n * (8 * 3 * 3 + 4 * 3 + 4 * 2);              // import/export staging
  b += 4096;
  return b;
}

// staged force path possible: mixed precision, >= 4 cells per axis, expected windows
// well inside shared memory (a larger one at a rebuild falls back, see sync_system)
bool staged_ok(const SysDev& h, const int nc[3]) {
  const double per_cell = (double)h.n / ((double)nc[0] * nc[1] * nc[2]);
  return h.precision == GBMD_MIXED && nc[0] >= 4 && nc[1] >= 4 && nc[2] >= 4 &&
         WIN_CELLS * per_cell * 1.35 + 96 <= STAGED_WINDOW_CAP;
}

void dfree(gbmd_system* s, void* p, size_t bytes) {
  if (!p) return;
  auto it = std::find(s->allocs.begin(), s->allocs.end(), p);
  if (it != s->allocs.end()) {
    s->allocs.erase(it);
    s->footprint -= std::max<size_t>(bytes, 16);
  }
  cudaFree(p);
}

// The cell grid: nc cells per axis, the arrays sized by the cell count and the
// Morton rank of every cell.  Replaces an existing grid (its arrays are freed).
int setup_cells(gbmd_system* s, const int nc[3], cudaStream_t st) {
  SysDev& h = s->h;
  CK(cudaStreamSynchronize(st));
  if (h.cell_cnt) {
    const size_t oc = (size_t)h.ncells, ob = (size_t)h.nblocks, obins = (size_t)h.nbins;
    dfree(s, h.cell_cnt, (obins + 1) * 4); dfree(s, h.cell_start, (obins + 1) * 4);
    dfree(s, h.cell_cursor, (obins + 1) * 4);
    dfree(s, const_cast<int*>(h.rank2lin), oc * 4); dfree(s, const_cast<int*>(h.lin2rank), oc * 4);
    dfree(s, h.blk_win, ob * WIN_CELLS * sizeof(int2)); dfree(s, h.blk_info, ob * sizeof(int4));
    h.cell_cnt = h.cell_start = h.cell_cursor = nullptr;
    h.rank2lin = h.lin2rank = nullptr;
    h.blk_win = nullptr;
    h.blk_info = nullptr;
  }
  int ncells = 1, nblocks = 1;
  for (int a = 0; a < 3; ++a) {
    h.nc[a] = nc[a];
    ncells *= nc[a];
    h.nb[a] = (nc[a] + 1) / 2;
    nblocks *= h.nb[a];
  }
  h.ncells = ncells;
  h.nblocks = nblocks;
  h.nbins = h.tree ? h.ntypes * ncells : ncells;   // the tree list sorts type-major
  const size_t nbins = (size_t)h.nbins;
  int rc = GBMD_OK;
  auto A = [&](void** p, size_t bytes) {
    if (rc == GBMD_OK) rc = dalloc(s, p, bytes);
  };
  A((void**)&h.blk_win, (size_t)nblocks * WIN_CELLS * sizeof(int2));
  A((void**)&h.blk_info, (size_t)nblocks * sizeof(int4));
  A((void**)&h.cell_cnt, (nbins + 1) * 4); A((void**)&h.cell_start, (nbins + 1) * 4);
  A((void**)&h.cell_cursor, (nbins + 1) * 4);
  int *r2l = nullptr, *l2r = nullptr;
  A((void**)&r2l, (size_t)ncells * 4); A((void**)&l2r, (size_t)ncells * 4);
  h.rank2lin = r2l;
  h.lin2rank = l2r;
  if (rc != GBMD_OK) return rc;
  std::vector<std::pair<uint32_t, int>> code(ncells);
  for (int z = 0; z < nc[2]; ++z)
    for (int y = 0; y < nc[1]; ++y)
      for (int x = 0; x < nc[0]; ++x) {
        const int lin = (z * nc[1] + y) * nc[0] + x;
        code[lin] = {spread3(x) | (spread3(y) << 1) | (spread3(z) << 2), lin};
      }
  std::sort(code.begin(), code.end());
  std::vector<int> rl(ncells), lr(ncells);
  for (int r = 0; r < ncells; ++r) {
    rl[r] = code[r].second;
    lr[code[r].second] = r;
  }
  CK(cudaMemcpyAsync(r2l, rl.data(), (size_t)ncells * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(l2r, lr.data(), (size_t)ncells * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(h.cell_cnt, 0, (nbins + 1) * 4, st));
  CK(cudaStreamSynchronize(st));   // the host tables die here
  return GBMD_OK;
}

int create_impl(const gbmd_desc* d, gbmd_system** out, bool device) {
  if (!out) return fail(GBMD_ERR_BAD_ARG, "out is NULL");
  *out = nullptr;
  RET(validate(d, device));
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return fail(GBMD_ERR_NO_DEVICE, "no CUDA device");
  int dev = d->device;
  if (dev < 0) CK(cudaGetDevice(&dev));
  if (dev >= ndev) return fail(GBMD_ERR_BAD_ARG, "device %d does not exist (%d devices)", dev, ndev);
  RET(use_device(dev));
  const bool tree = d->nlist == GBMD_NLIST_TREE;
  int64_t tcount[GBMD_MAX_TYPES] = {0, 0, 0, 0};   // particles per type (tree list)
  if (tree) {
    std::vector<int32_t> ty;
    const int32_t* tp = d->type;
    if (tp && device) {   // the tree layout is fixed by the type counts: read them once
      ty.resize((size_t)d->n);
      CK(cudaMemcpy(ty.data(), tp, (size_t)d->n * 4, cudaMemcpyDeviceToHost));
      tp = ty.data();
    }
    for (int64_t i = 0; i < d->n; ++i) {
      const int t = tp ? tp[i] : 0;
      if (t < 0 || t >= d->ntypes) return fail(GBMD_ERR_BAD_ARG, "type id out of range at %lld", (long long)i);
      ++tcount[t];
    }
  }
  const Geometry geo = geometry(d, tree ? tcount : nullptr);
  gbmd_system* s = new gbmd_system();
  s->device = dev;
  s->stream = (cudaStream_t)d->stream;
  SysDev& h = s->h;
  const int n = (int)d->n, nt = d->ntypes;
  h.n = n;
  h.n_ghost = (int)d->n_ghost;
  h.ntypes = nt;
  h.precision = d->precision;
  h.sort_period = d->sort_period;
  h.cap = geo.cap;
  h.nl_stride = (int)round_up((size_t)n, 32);
  h.dt = d->dt;
  h.mass = d->mass;
  h.h = 0.5 * d->dt / d->mass;
  s->cell_min = geo.cell_min;
  s->want_staged = d->force_path == GBMD_PATH_STAGED && d->integrator == GBMD_NVE &&
                   eval_of(d->potential) == EVAL_LJ && !tree;
  h.tree = tree ? 1 : 0;
  int nodes = 0;
  if (tree) {   // type t: particles [first, first + n) of the sorted order, P leaves
    int first = 0, leaves = 0;
    for (int t = 0; t < nt; ++t) {
      h.tree_first[t] = first;
      h.tree_n[t] = (int)tcount[t];
      h.tree_P[t] = tree_leaves((int)tcount[t]);
      h.tree_leaf0[t] = leaves;
      h.tree_node0[t] = nodes;
      first += (int)tcount[t];
      leaves += h.tree_P[t];
      nodes += 2 * h.tree_P[t];   // boxes 1 .. 2P - 1 (0 unused)
    }
    h.tree_leaves_total = leaves;
    // query order: the types by decreasing expected work per particle
    double work[GBMD_MAX_TYPES];
    int ord[GBMD_MAX_TYPES];
    for (int t = 0; t < nt; ++t) {
      work[t] = 0;
      for (int u = 0; u < nt; ++u) {
        const double rl = cut_of(d, t * nt + u) + d->r_buff;
        work[t] += (double)tcount[u] * rl * rl * rl;
      }
      ord[t] = t;
    }
    std::stable_sort(ord, ord + nt, [&](int a, int b) { return work[a] > work[b]; });
    int qpos = 0;
    for (int k = 0; k < nt; ++k) {
      h.tree_qtype[k] = ord[k];
      h.tree_qpos[k] = qpos;
      qpos += (int)tcount[ord[k]];
    }
    h.tree_qpos[nt] = qpos;
  }
  h.nvt = d->integrator == GBMD_NVT;
  h.kT = d->kT;
  h.tau = d->tau;
  h.gdof = 3.0 * (double)n - 3.0;
  h.staged = s->want_staged && staged_ok(h, geo.nc);
  h.window_cap = STAGED_WINDOW_CAP;
  for (int a = 0; a < 3; ++a) {
    h.L[a] = d->box[a];
    h.halfL[a] = 0.5 * d->box[a];
    h.qscale[a] = 4294967296.0 / d->box[a];
    h.dtq[a] = d->dt * h.qscale[a];
    h.fscale[a] = (float)(d->box[a] / 4294967296.0);
  }
  const double hb = 0.5 * d->r_buff;
  h.rbuff_half2 = (float)(hb * hb * (1.0 - 1e-5));
  h.eval = eval_of(d->potential);
  for (int p = 0; p < nt * nt; ++p) {
    const double rc = cut_of(d, p), rl = rc + d->r_buff;
    PairD& pd = h.pd[p];
    pd = PairD{};
    pair_coefficients(d, p, rc, &pd);
    pd.rc2 = rc * rc;
    pd.rl2 = rl * rl;
    PairF& pf = h.pf[p];
    pf.p0 = (float)pd.p0;
    pf.p1 = (float)pd.p1;
    pf.p2 = (float)pd.p2;
    pf.p3 = (float)pd.p3;
    pf.p4 = (float)pd.p4;
    pf.rc2 = (float)pd.rc2;
    pf.shift = (float)pd.shift;
    pf.rl2 = (float)pd.rl2;
  }
  int rc = GBMD_OK;
  auto A = [&](void** p, size_t bytes) {
    if (rc == GBMD_OK) rc = dalloc(s, p, bytes);
  };
  const size_t N = (size_t)n;
  A((void**)&h.x, N * 24); A((void**)&h.v, N * 24); A((void**)&h.img, N * 12);
  A((void**)&h.type, N * 4); A((void**)&h.tag, N * 4); A((void**)&h.rtag, N * 4);
  A((void**)&h.q, N * 16); A((void**)&h.q1, N * 16); A((void**)&h.q_build, N * 16);
  if (d->precision == GBMD_FP64) {
    A((void**)&h.p64, N * 32); A((void**)&h.p64b, N * 32);
  }
  if (d->precision == GBMD_FP64) A((void**)&h.f64, N * 32); else A((void**)&h.f32, N * 16);
  A((void**)&h.nn, N * 4); A((void**)&h.nl, round_up(N, 32) * 4 * (size_t)geo.cap);
  A((void**)&h.key, N * 4); A((void**)&h.members, N * 4); A((void**)&h.members_tmp, N * 4);
  A((void**)&h.rmember, N * 4);
  A((void**)&h.x_alt, N * 24); A((void**)&h.v_alt, N * 24); A((void**)&h.img_alt, N * 12);
  A((void**)&h.type_alt, N * 4); A((void**)&h.tag_alt, N * 4); A((void**)&h.q_alt, N * 16);
  A((void**)&h.fkey, N * 4);   // fine Morton keys: the order inside a cell
  A((void**)&h.cpos, N * 16);  // positions in cell order (the list build's candidates)
  A((void**)&h.thermo, 16 * 8);
  A((void**)&h.nh, 4 * 8);
  if (tree) {
    A((void**)&h.tree_box, (size_t)nodes * sizeof(TreeBox));
    A((void**)&h.tree_arrive, (size_t)nodes * 4);
    A((void**)&h.tree_q, N * 16);
  }
  A((void**)&s->d_flags, sizeof(Flags));
  A((void**)&s->d_pos, N * 24); A((void**)&s->d_vel, N * 24); A((void**)&s->d_frc, N * 24);
  A((void**)&s->d_img, N * 12); A((void**)&s->d_type, N * 4); A((void**)&s->d_misc, 64);
  h.flags = s->d_flags;
  s->d_thermo = h.thermo;
  if (rc != GBMD_OK) { gbmd_destroy(s); return rc; }
  cudaStream_t st = s->stream;
  rc = setup_cells(s, geo.nc, st);
  if (rc != GBMD_OK) { std::string m = g_err; gbmd_destroy(s); g_err = m; return rc; }
  {
    const double nh0[4] = {0.0, 0.0, 1.0, 0.0};   // xi, eta, exp(-xi dt/2)
    cudaError_t e5 = cudaMemsetAsync(s->d_flags, 0, sizeof(Flags), st);
    cudaError_t e6 = cudaMemsetAsync(h.nn, 0, N * 4, st);
    if (tree && e6 == cudaSuccess) e6 = cudaMemsetAsync(h.tree_arrive, 0, (size_t)nodes * 4, st);
    cudaError_t e7 = cudaMemcpyAsync(h.nh, nh0, sizeof(nh0), cudaMemcpyHostToDevice, st);
    cudaError_t e4 = cudaStreamSynchronize(st);
    if (e7) { gbmd_destroy(s); return fail(GBMD_ERR_CUDA, "thermostat upload failed"); }
    if (e4 || e5 || e6) { gbmd_destroy(s); return fail(GBMD_ERR_CUDA, "clearing the flags failed"); }
  }
  // own group
  s->own = new Group();
  s->own->device = dev;
  s->own->stream = st;
  s->own->precision = d->precision;
  s->own->members.push_back(s);
  // default tuning (measured on GB300 with the L2 flushed between steps).  Mixed
  // precision: one lane per particle once there are enough particles to fill every
  // SM several times over, two below that; 128-thread blocks.  FP64 (bound by the
  // FP64 pipe): one lane in 64-thread blocks from 32k particles (the 64k fluid
  // steps 10% faster than with two lanes in 128-thread blocks), four lanes in
  // 128-thread blocks below (the 4,000-particle fluid 29% faster)
  const bool fp64 = d->precision == GBMD_FP64;
  const int auto_tpp = fp64 ? (d->n >= 32768 ? 1 : 4) : (d->n >= (1 << 19) ? 1 : 2);
  s->own->tpp = d->threads_per_particle ? d->threads_per_particle : auto_tpp;
  s->own->fblock = fp64 && s->own->tpp == 1 ? 64 : 128;
  if (const char* ev = getenv("GBMD_NO_GRAPHS")) s->own->use_graphs = ev[0] != '1';
  *out = s;
  return GBMD_OK;
}

// Upload positions/velocities/types/images (tag order, host or device memory),
// then build the lists (with the initial Morton sort) and compute the forces.
int load_state(gbmd_system* s, const double* pos, const double* vel, const int32_t* type,
               const int32_t* image, bool device, long long step) {
  cudaStream_t st = cur_stream(s);
  const size_t N = (size_t)s->h.n;
  const double *dp = pos, *dv = vel;
  const int *dt = type, *di = image;
  if (!device) {
    CK(cudaMemcpyAsync(s->d_pos, pos, N * 24, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s->d_vel, vel, N * 24, cudaMemcpyHostToDevice, st));
    dp = s->d_pos;
    dv = s->d_vel;
    if (type) {
      CK(cudaMemcpyAsync(s->d_type, type, N * 4, cudaMemcpyHostToDevice, st));
      dt = s->d_type;
    }
    if (image) {
      CK(cudaMemcpyAsync(s->d_img, image, N * 12, cudaMemcpyHostToDevice, st));
      di = s->d_img;
    }
  }
  Group* g = s->own;
  RET(sync_layout(g));
  CK(launch(import_call(g->d_desc, g->d_tp, g->ntp, dp, dv, dt, di), st));
  Flags f{};
  f.do_rebuild = 1;
  f.do_sort = 1;
  f.v_full = 1;
  f.active = 1;
  f.step = step;
  f.step_limit = s->step_limit;
  f.last_sort = step;
  Flags old{};
  CK(cudaMemcpyAsync(&old, s->d_flags, sizeof(Flags), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (old.error == DEV_BADTYPE) return fail(GBMD_ERR_BAD_ARG, "type id out of range in the device type array");
  f.n_rebuilds = old.n_rebuilds;
  f.n_sorts = old.n_sorts + 1;
  f.launches = old.launches;
  RET(write_flags(s, &f, st));
  s->target_step = step;
  RET(rebuild_and_force(s, 0));
  CK(cudaStreamSynchronize(st));
  Flags after;
  RET(read_flags(s, &after, st));
  if (after.error == DEV_WINDOW) {
    s->h.staged = 0;
    RET(refresh_desc(s));
    after.error = 0;
    after.do_rebuild = 1;
    RET(write_flags(s, &after, st));
    RET(rebuild_and_force(s, 0));
    RET(read_flags(s, &after, st));
  }
  if (after.error == DEV_OVERFLOW) {
    RET(grow_nlist(s, after.overflow_need));
    after.error = 0;
    after.overflow_need = 0;
    after.do_rebuild = 1;
    RET(write_flags(s, &after, st));
    RET(rebuild_and_force(s, 0));
    RET(read_flags(s, &after, st));
    if (after.error) return fail(GBMD_ERR_NLIST_OVERFLOW, "neighbour list overflow at creation");
  }
  return GBMD_OK;
}

// NVT readout of the thermostat, as the state after the last completed step: the
// stored xi / eta are those of the step's opening half; the closing half adds
// dt/2 G(K) to xi and dt/2 xi to eta (nothing right after create / set_state).
// h_ext = K + U (+ g kT (tau^2 xi^2 / 2 + eta) for NVT) is the conserved quantity.
int fill_thermostat(gbmd_system* s, const Flags& f, gbmd_thermo* out) {
  out->xi = 0.0;
  out->eta = 0.0;
  out->h_ext = out->ke + out->pe;
  if (!s->h.nvt) return GBMD_OK;
  double nh[2];
  cudaStream_t st = cur_stream(s);
  CK(cudaMemcpyAsync(nh, s->h.nh, sizeof(nh), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const SysDev& h = s->h;
  double xi = nh[0], eta = nh[1];
  if (!f.v_full) {
    const double G = (2.0 * out->ke / (h.gdof * h.kT) - 1.0) / (h.tau * h.tau);
    eta += 0.5 * h.dt * xi;
    xi += 0.5 * h.dt * G;
  }
  out->xi = xi;
  out->eta = eta;
  out->h_ext += h.gdof * h.kT * (0.5 * h.tau * h.tau * xi * xi + eta);
  return GBMD_OK;
}

int thermo_impl(gbmd_system* s, double out[8]) {
  Group* g = s->own;
  RET(sync_layout(g));
  cudaStream_t st = cur_stream(s);
  for (const KernelCall& c : force_calls(g, 1)) CK(launch(c, st));
  CK(launch(thermo_call(g->d_desc, g->d_ts, g->nts, g->d_ctl), st));
  CK(cudaMemcpyAsync(out, s->d_thermo, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return GBMD_OK;
}

int export_impl(gbmd_system* s, double* pos, double* vel, int32_t* image, double* force,
                double* pp_u, double* pp_w) {
  Group* g = s->own;
  RET(sync_layout(g));
  cudaStream_t st = cur_stream(s);
  const size_t N = (size_t)s->h.n;
  if ((pp_u || pp_w) && !s->d_ppw) return fail(GBMD_ERR_STATE, "per-particle arrays not allocated");
  // forces and full-step velocities need F at the current positions: the step kernel
  // does not store its force, so evaluate it here
  if (vel || force)
    for (const KernelCall& c : force_calls(g, 0)) CK(launch(c, st));
  CK(launch(export_call(g->d_desc, g->d_tp, g->ntp, pos ? s->d_pos : nullptr,
                        vel ? s->d_vel : nullptr, image ? s->d_img : nullptr,
                        force ? s->d_frc : nullptr, pp_u ? s->d_ppu : nullptr,
                        pp_w ? s->d_ppw : nullptr), st));
  if (pos) CK(cudaMemcpyAsync(pos, s->d_pos, N * 24, cudaMemcpyDeviceToHost, st));
  if (vel) CK(cudaMemcpyAsync(vel, s->d_vel, N * 24, cudaMemcpyDeviceToHost, st));
  if (image) CK(cudaMemcpyAsync(image, s->d_img, N * 12, cudaMemcpyDeviceToHost, st));
  if (force) CK(cudaMemcpyAsync(force, s->d_frc, N * 24, cudaMemcpyDeviceToHost, st));
  if (pp_u) CK(cudaMemcpyAsync(pp_u, s->d_ppu, N * 8, cudaMemcpyDeviceToHost, st));
  if (pp_w) CK(cudaMemcpyAsync(pp_w, s->d_ppw, N * 48, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return GBMD_OK;
}

int time_force(Group* g, float* ms) {
  RET(sync_layout(g));
  if (g->ntf == 0) {
    *ms = 0.f;
    return GBMD_OK;
  }
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  for (int k = 0; k < 2; ++k) CK(launch(plain_force_call(g), g->stream));
  CK(cudaEventRecord(a, g->stream));
  const int reps = 5;
  for (int k = 0; k < reps; ++k) CK(launch(plain_force_call(g), g->stream));
  CK(cudaEventRecord(b, g->stream));
  CK(cudaEventSynchronize(b));
  float t = 0;
  CK(cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t / reps;
  return GBMD_OK;
}

// Cells at least scale * r_list,max wide: a new cell grid, then the lists (with a
// re-sort into the new Morton order) and the forces at the current positions.  The
// neighbour sets do not change (r_list does not); the order of a particle's
// neighbours, and so the FP32 summation order of its force, may.
int regrid(gbmd_system* s, double scale) {
  if (!(scale >= 1.0 && scale <= 4.0)) return fail(GBMD_ERR_BAD_ARG, "cell scale must be in [1, 4]");
  SysDev& h = s->h;
  int nc[3];
  for (int a = 0; a < 3; ++a) nc[a] = cells_along(h.L[a], s->cell_min, scale);
  s->cell_scale = scale;
  if (nc[0] == h.nc[0] && nc[1] == h.nc[1] && nc[2] == h.nc[2]) return GBMD_OK;
  RET(sync_system(s));   // nothing in flight, nothing owed
  cudaStream_t st = cur_stream(s);
  RET(setup_cells(s, nc, st));
  h.staged = s->want_staged && staged_ok(h, nc);
  RET(refresh_desc(s));
  for (int round = 0; round < 2; ++round) {
    Flags f;
    RET(read_flags(s, &f, st));
    if (round == 1 && f.error != DEV_WINDOW) break;
    if (f.error == DEV_WINDOW) {   // a staged window outgrew shared memory
      h.staged = 0;
      RET(refresh_desc(s));
      f.error = 0;
    }
    f.do_rebuild = 1;
    f.do_sort = 1;
    f.last_sort = f.step;
    f.n_sorts += 1;
    RET(write_flags(s, &f, st));
    RET(rebuild_and_force(s, 0));
    CK(cudaStreamSynchronize(st));
  }
  Flags f;
  RET(read_flags(s, &f, st));
  if (f.error) return fail(GBMD_ERR_STATE, "device error %d after a new cell grid", f.error);
  f.do_rebuild = 0;
  f.do_sort = 0;
  return write_flags(s, &f, st);
}

// Mean time of one full list rebuild (no re-sort) of every member of the group.
int time_rebuild(Group* g, float* ms) {
  RET(sync_layout(g));
  std::vector<gbmd_system*> m = live(g);
  for (auto* s : m) {
    Flags f;
    RET(read_flags(s, &f, g->stream));
    f.do_rebuild = 1;
    f.do_sort = 0;
    RET(write_flags(s, &f, g->stream));
  }
  const std::vector<KernelCall> calls = rebuild_calls(g);
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  for (const KernelCall& c : calls) CK(launch(c, g->stream));
  CK(cudaEventRecord(a, g->stream));
  const int reps = 3;
  for (int k = 0; k < reps; ++k)
    for (const KernelCall& c : calls) CK(launch(c, g->stream));
  CK(cudaEventRecord(b, g->stream));
  CK(cudaEventSynchronize(b));
  float t = 0;
  CK(cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t / reps;
  for (auto* s : m) {   // the lists stand for the current positions
    Flags f;
    RET(read_flags(s, &f, g->stream));
    if (f.error) return fail(GBMD_ERR_STATE, "device error %d while timing a rebuild", f.error);
    f.do_rebuild = 0;
    RET(write_flags(s, &f, g->stream));
  }
  return GBMD_OK;
}

std::string tune_key(const Group* g) {
  std::vector<gbmd_system*> m = live(g);
  long long np = 0;
  double vol = 0;
  for (auto* s : m) {
    np += s->h.n;
    vol += s->h.L[0] * s->h.L[1] * s->h.L[2];
  }
  const int lg = np > 0 ? (int)std::floor(std::log2((double)np)) : 0;
  const int rho10 = vol > 0 ? (int)std::lround(10.0 * np / vol) : 0;
  char buf[512];
  cudaDeviceProp p{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&p, dev);
  snprintf(buf, sizeof(buf), "%s|prec=%d|multi=%d|eval=%d|members=%d|log2n=%d|rho10=%d", p.name,
           g->precision, g->multi, g->eval, (int)m.size(), lg, rho10);
  for (char* c = buf; *c; ++c)
    if (*c == ' ') *c = '_';
  return buf;
}

int set_tuning(Group* g, int tpp, int block) {
  if (!tpp_supported(tpp) || block < 32 || block > 512 || block % 32 || block % tpp)
    return fail(GBMD_ERR_BAD_ARG, "bad tuning tpp=%d block=%d", tpp, block);
  if (g->tpp == tpp && g->fblock == block) return GBMD_OK;
  g->tpp = tpp;
  g->fblock = block;
  g->layout_dirty = true;
  return sync_layout(g);
}

int autotune_group(Group* g, const char* cache) {
  RET(sync_layout(g));
  if (g->ntf == 0) return GBMD_OK;   // every member on the staged path (nothing to tune)
  const std::string key = tune_key(g);
  if (cache) {
    std::ifstream in(cache);
    std::string line;
    int bt = 0, bb = 0;
    double bs = 1.0;
    while (std::getline(in, line)) {
      std::istringstream ls(line);
      std::string k;
      int t, b;
      if (ls >> k >> t >> b && k == key) {
        bt = t;
        bb = b;
        double sc;
        bs = (ls >> sc) ? sc : 1.0;
      }
    }
    if (bt) {
      for (auto* s : live(g)) RET(regrid(s, bs));
      return set_tuning(g, bt, bb);
    }
  }
  // cell width: the list rebuild at each candidate width (the global force path does
  // not depend on it); a wider cell only wins if it is clearly faster
  double best_s = 1.0;
  {
    bool any_staged = false;
    for (auto* s : live(g)) any_staged |= s->h.staged != 0;
    if (!any_staged) {
      float best_r = 1e30f;
      std::vector<std::vector<int>> seen;
      for (double sc : {1.0, 1.1, 1.2, 1.35}) {
        std::vector<int> grid;
        for (auto* s : live(g))
          for (int a = 0; a < 3; ++a) grid.push_back(cells_along(s->h.L[a], s->cell_min, sc));
        if (std::find(seen.begin(), seen.end(), grid) != seen.end()) continue;
        seen.push_back(grid);
        for (auto* s : live(g)) RET(regrid(s, sc));
        float ms;
        RET(time_rebuild(g, &ms));
        if (getenv("GBMD_VERBOSE")) fprintf(stderr, "gbmd autotune %s cell_scale=%.2f rebuild %.4f ms\n", key.c_str(), sc, ms);
        if (ms < 0.97f * best_r) { best_r = ms; best_s = sc; }
      }
      for (auto* s : live(g)) RET(regrid(s, best_s));
    }
  }
  int best_t = g->tpp, best_b = g->fblock;
  float best = 1e30f;
  // FP64 also tries 64-thread blocks (its best step shape from 32k particles on)
  const bool fp64 = g->precision == GBMD_FP64;
  for (int tpp : {1, 2, 4})
    for (int block : {64, 128, 256, 512}) {
      if (block == 64 && !fp64) continue;
      RET(set_tuning(g, tpp, block));
      float ms;
      RET(time_force(g, &ms));
      if (getenv("GBMD_VERBOSE")) fprintf(stderr, "gbmd autotune %s tpp=%d block=%d %.4f ms\n", key.c_str(), tpp, block, ms);
      if (ms < best) { best = ms; best_t = tpp; best_b = block; }
    }
  RET(set_tuning(g, best_t, best_b));
  if (cache) {
    std::ofstream o(cache, std::ios::app);
    o << key << " " << best_t << " " << best_b << " " << best_s << "\n";
  }
  return GBMD_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char* gbmd_last_error(void) { return g_err.c_str(); }

int gbmd_abi_version(void) { return GBMD_ABI_VERSION; }

int gbmd_probe_arith(int32_t kind, int32_t iters, void* stream, double* ops, float* ms) {
  if (!ops || !ms) return fail(GBMD_ERR_BAD_ARG, "NULL output");
  if (kind != GBMD_PROBE_DFMA && kind != GBMD_PROBE_FFMA && kind != GBMD_PROBE_DRCP)
    return fail(GBMD_ERR_BAD_ARG, "unknown probe kind %d", kind);
  if (iters < 1) return fail(GBMD_ERR_BAD_ARG, "iters must be >= 1");
  CK(probe_run(kind, static_cast<cudaStream_t>(stream), iters, ops, ms));
  return GBMD_OK;
}

int gbmd_create(const gbmd_desc* d, gbmd_system** out) {
  Range nvtx_range("gbmd_create");
  RET(create_impl(d, out, false));
  int rc = load_state(*out, d->pos, d->vel, d->type, d->image, false, 0);
  if (rc != GBMD_OK) {
    std::string msg = g_err;
    gbmd_destroy(*out);
    *out = nullptr;
    g_err = msg;
  }
  return rc;
}

int gbmd_create_device(const gbmd_desc* d, gbmd_system** out) {
  Range nvtx_range("gbmd_create_device");
  RET(create_impl(d, out, true));
  int rc = load_state(*out, d->pos, d->vel, d->type, d->image, true, 0);
  if (rc != GBMD_OK) {
    std::string msg = g_err;
    gbmd_destroy(*out);
    *out = nullptr;
    g_err = msg;
  }
  return rc;
}

int gbmd_destroy(gbmd_system* s) {
  if (!s) return fail(GBMD_ERR_BAD_ARG, "system is NULL");
  use_device(s->device);
  if (s->batch) {
    Group* b = s->batch;
    for (auto& m : b->members)
      if (m == s) m = nullptr;
    b->layout_dirty = true;
    s->batch = nullptr;
  }
  if (s->own) cudaStreamSynchronize(s->own->stream);
  for (void* p : s->allocs) cudaFree(p);
  if (s->own) {
    Group* g = s->own;
    destroy_graphs(g);
    cudaFree(g->d_desc); cudaFree(g->d_tp); cudaFree(g->d_tf); cudaFree(g->d_tc); cudaFree(g->d_te); cudaFree(g->d_nhpart);
    cudaFree(g->d_ts); cudaFree(g->d_tb); cudaFree(g->d_tbk); cudaFree(g->d_tt); cudaFree(g->d_partials);
    cudaFree(g->d_ctl);
    delete g;
  }
  delete s;
  return GBMD_OK;
}

int gbmd_step(gbmd_system* s, int64_t nsteps) {
  Range nvtx_range("gbmd_step");
  if (!s || nsteps < 0) return fail(GBMD_ERR_BAD_ARG, "bad system or nsteps");
  RET(use_device(s->device));
  if (s->batch) return fail(GBMD_ERR_STATE, "system belongs to a batch; use gbmd_batch_step");
  s->target_step += nsteps;
  return enqueue_steps(s->own, nsteps);
}

int gbmd_sync(gbmd_system* s) {
  Range nvtx_range("gbmd_sync");
  if (!s) return fail(GBMD_ERR_BAD_ARG, "system is NULL");
  RET(use_device(s->device));
  return sync_system(s);
}

int gbmd_get_forces(gbmd_system* s, double* out) {
  Range nvtx_range("gbmd_get_forces");
  if (!s || !out) return fail(GBMD_ERR_BAD_ARG, "NULL argument");
  RET(use_device(s->device));
  RET(sync_system(s));
  return export_impl(s, nullptr, nullptr, nullptr, out, nullptr, nullptr);
}

int gbmd_get_thermo(gbmd_system* s, gbmd_thermo* out) {
  Range nvtx_range("gbmd_get_thermo");
  if (!s || !out) return fail(GBMD_ERR_BAD_ARG, "NULL argument");
  RET(use_device(s->device));
  RET(sync_system(s));
  double t[8];
  RET(thermo_impl(s, t));
  Flags f;
  RET(read_flags(s, &f, cur_stream(s)));
  const double n = (double)s->h.n;
  const double vol = s->h.L[0] * s->h.L[1] * s->h.L[2];
  out->step = f.step;
  out->pe = t[0];
  out->ke = 0.5 * s->h.mass * t[1];
  out->temperature = n > 1 ? 2.0 * out->ke / (3.0 * n - 3.0) : 0.0;
  for (int c = 0; c < 6; ++c) out->virial[c] = t[2 + c];
  out->w = t[2] + t[5] + t[7];
  out->pressure = (n * out->temperature + out->w / 3.0) / vol;
  out->n_rebuilds = f.n_rebuilds;
  return fill_thermostat(s, f, out);
}

int gbmd_get_per_particle(gbmd_system* s, double* energy, double* virial) {
  Range nvtx_range("gbmd_get_per_particle");
  if (!s) return fail(GBMD_ERR_BAD_ARG, "system is NULL");
  RET(use_device(s->device));
  RET(sync_system(s));
  if (!s->h.pp_u) {
    const size_t N = (size_t)s->h.n;
    RET(dalloc(s, (void**)&s->h.pp_u, N * 8));
    RET(dalloc(s, (void**)&s->h.pp_w, N * 48));
    RET(dalloc(s, (void**)&s->d_ppu, N * 8));
    RET(dalloc(s, (void**)&s->d_ppw, N * 48));
    RET(refresh_desc(s));
  }
  double t[8];
  RET(thermo_impl(s, t));   // the energy pass fills the per-particle arrays
  return export_impl(s, nullptr, nullptr, nullptr, nullptr, energy, virial);
}

int gbmd_get_state(gbmd_system* s, double* pos, double* vel, int32_t* image, int64_t* step) {
  Range nvtx_range("gbmd_get_state");
  if (!s) return fail(GBMD_ERR_BAD_ARG, "system is NULL");
  RET(use_device(s->device));
  RET(sync_system(s));
  RET(export_impl(s, pos, vel, image, nullptr, nullptr, nullptr));
  if (step) {
    Flags f;
    RET(read_flags(s, &f, cur_stream(s)));
    *step = f.step;
  }
  return GBMD_OK;
}

int gbmd_set_state(gbmd_system* s, const double* pos, const double* vel, const int32_t* image,
                   int64_t step) {
  Range nvtx_range("gbmd_set_state");
  if (!s || !pos || !vel || step < 0) return fail(GBMD_ERR_BAD_ARG, "bad argument");
  RET(use_device(s->device));
  if (s->batch) return fail(GBMD_ERR_STATE, "remove the system from its batch first");
  RET(sync_system(s));
  const size_t N = (size_t)s->h.n;
  cudaStream_t st = cur_stream(s);
  Group* g = s->own;
  RET(sync_layout(g));
  // The new state goes to the staging buffers; its finiteness and the current types
  // in tag order are taken there on the device, and nothing of the system is
  // replaced unless every value is finite.
  CK(cudaMemcpyAsync(s->d_pos, pos, N * 24, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(s->d_vel, vel, N * 24, cudaMemcpyHostToDevice, st));
  if (image) CK(cudaMemcpyAsync(s->d_img, image, N * 12, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(s->d_misc, 0, 4, st));
  CK(launch(prep_state_call(g->d_desc, g->d_tp, g->ntp, s->d_pos, s->d_vel, s->d_type, s->d_misc),
            st));
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, s->d_misc, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad) return fail(GBMD_ERR_BAD_ARG, "non-finite state");
  return load_state(s, s->d_pos, s->d_vel, s->d_type, image ? s->d_img : nullptr, true, step);
}

int gbmd_get_neighbors(gbmd_system* s, int32_t* counts, int32_t* idx, int64_t cap) {
  Range nvtx_range("gbmd_get_neighbors");
  if (!s || !counts || !idx || cap < 1 || cap > (1 << 20)) return fail(GBMD_ERR_BAD_ARG, "bad argument");
  RET(use_device(s->device));
  RET(sync_system(s));
  Group* g = s->own;
  RET(sync_layout(g));
  cudaStream_t st = cur_stream(s);
  const size_t N = (size_t)s->h.n;
  int *dc = nullptr, *di = nullptr, *dflag = s->d_misc;
  CK(cudaMalloc(&dc, N * 4));
  cudaError_t e = cudaMalloc(&di, N * (size_t)cap * 4);
  if (e != cudaSuccess) {
    cudaFree(dc);
    return fail(GBMD_ERR_OOM, "no room for the neighbour readout");
  }
  int too_many = 0;
  int rc = GBMD_OK;
  if (cudaMemsetAsync(dflag, 0, 4, st) != cudaSuccess ||
      launch(nlist_export_call(g->d_desc, g->d_tp, g->ntp, dc, di, (int)cap, dflag), st) != cudaSuccess ||
      cudaMemcpyAsync(counts, dc, N * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(idx, di, N * (size_t)cap * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&too_many, dflag, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    rc = fail(GBMD_ERR_CUDA, "neighbour readout failed");
  cudaFree(dc);
  cudaFree(di);
  if (rc == GBMD_OK && too_many) rc = fail(GBMD_ERR_BAD_ARG, "some particle has more than cap neighbours");
  return rc;
}

int gbmd_get_info(gbmd_system* s, gbmd_info* out) {
  if (!s || !out) return fail(GBMD_ERR_BAD_ARG, "NULL argument");
  RET(use_device(s->device));
  RET(sync_system(s));
  Flags f;
  RET(read_flags(s, &f, cur_stream(s)));
  Group* g = s->batch ? s->batch : s->own;
  out->n = s->h.n;
  out->precision = s->h.precision;
  out->ntypes = s->h.ntypes;
  for (int a = 0; a < 3; ++a) out->cells[a] = s->h.nc[a];
  out->nlist_capacity = s->h.cap;
  out->threads_per_particle = g->tpp;
  out->force_block = g->fblock;
  out->step = f.step;
  out->n_rebuilds = f.n_rebuilds;
  out->n_sorts = f.n_sorts;
  out->kernel_launches = (int64_t)f.launches;
  out->neighbors_total = (int64_t)f.nb_total;
  out->footprint_bytes = (int64_t)s->footprint;
  out->force_path = s->h.staged ? 1 : 0;
  out->max_window = f.max_window;
  out->cell_scale = s->cell_scale;
  out->nlist = s->h.tree ? GBMD_NLIST_TREE : GBMD_NLIST_CELL;
  out->rebuild_pending = s->h.n_ghost > 0 && f.rebuild_req ? 1 : 0;
  out->n_ghost = s->h.n_ghost;
  return GBMD_OK;
}

int gbmd_set_ghost_positions(gbmd_system* s, const double* pos, int32_t device) {
  if (!s || !pos) return fail(GBMD_ERR_BAD_ARG, "NULL argument");
  if (s->h.n_ghost <= 0) return fail(GBMD_ERR_BAD_ARG, "the system has no ghosts");
  if (s->batch) return fail(GBMD_ERR_STATE, "the system is in a batch");
  RET(use_device(s->device));
  Group* g = s->own;
  RET(sync_layout(g));
  cudaStream_t st = cur_stream(s);
  const double* dp = pos;
  if (!device) {   // staging: the import buffer holds n >= n_ghost rows
    CK(cudaMemcpyAsync(s->d_pos, pos, (size_t)s->h.n_ghost * 24, cudaMemcpyHostToDevice, st));
    dp = s->d_pos;
  }
  CK(launch(ghost_set_call(g->d_desc, s->h.n_ghost, dp), st));
  return GBMD_OK;
}

int gbmd_get_positions(gbmd_system* s, const int32_t* tags, int64_t m, double* out,
                       int32_t device) {
  if (!s || !tags || !out) return fail(GBMD_ERR_BAD_ARG, "NULL argument");
  if (m < 0 || m > s->h.n) return fail(GBMD_ERR_BAD_ARG, "m must be in [0, n]");
  if (!device)
    for (int64_t k = 0; k < m; ++k)
      if (tags[k] < 0 || tags[k] >= s->h.n) return fail(GBMD_ERR_BAD_ARG, "tag %d out of range", tags[k]);
  RET(use_device(s->device));
  RET(sync_system(s));
  if (m == 0) return GBMD_OK;
  Group* g = s->batch ? s->batch : s->own;
  RET(sync_layout(g));
  int idx = 0;   // the system's slot in its group's descriptor array
  for (size_t k = 0; k < g->members.size(); ++k)
    if (g->members[k] == s) idx = (int)k;
  cudaStream_t st = cur_stream(s);
  const int* dt = tags;
  double* dout = out;
  if (!device) {   // staging: the import buffers hold n >= m rows
    CK(cudaMemcpyAsync(s->d_type, tags, (size_t)m * 4, cudaMemcpyHostToDevice, st));
    dt = s->d_type;
    dout = s->d_pos;
  }
  CK(launch(gather_pos_call(g->d_desc + idx, dt, (int)m, dout), st));
  if (!device) CK(cudaMemcpyAsync(out, s->d_pos, (size_t)m * 24, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return GBMD_OK;
}

int64_t gbmd_footprint_bytes(const gbmd_desc* d) {
  if (!d || d->n < 1 || d->ntypes < 1 || d->ntypes > GBMD_MAX_TYPES)
    return fail(GBMD_ERR_BAD_ARG, "bad description");
  double rmax = 0;
  RET(validate_pairs(d, &rmax));
  for (int a = 0; a < 3; ++a)
    if (!(d->box[a] > 0)) return fail(GBMD_ERR_BAD_ARG, "bad box");
  return (int64_t)footprint_of(d, geometry(d));
}

int gbmd_set_step_limit(gbmd_system* s, int64_t step) {
  if (!s || step < -1) return fail(GBMD_ERR_BAD_ARG, "bad argument");
  RET(use_device(s->device));
  cudaStream_t st = cur_stream(s);
  CK(cudaStreamSynchronize(st));
  Flags f;
  RET(read_flags(s, &f, st));
  f.step_limit = step;
  s->step_limit = step;
  return write_flags(s, &f, st);
}

int gbmd_set_thermostat(gbmd_system* s, double xi, double eta) {
  if (!s) return fail(GBMD_ERR_BAD_ARG, "system is NULL");
  if (!s->h.nvt) return fail(GBMD_ERR_BAD_ARG, "not an NVT system");
  if (!std::isfinite(xi) || !std::isfinite(eta)) return fail(GBMD_ERR_BAD_ARG, "non-finite thermostat");
  RET(use_device(s->device));
  RET(sync_system(s));
  cudaStream_t st = cur_stream(s);
  // the state of a completed step, as gbmd_get_thermo reports it: valid where the
  // velocities are full-step ones too (after create / set_state, before stepping)
  Flags f;
  RET(read_flags(s, &f, st));
  if (!f.v_full) return fail(GBMD_ERR_STATE, "set the thermostat after gbmd_set_state, before stepping");
  const double nh[3] = {xi, eta, std::exp(-0.5 * s->h.dt * xi)};
  CK(cudaMemcpyAsync(s->h.nh, nh, sizeof(nh), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return GBMD_OK;
}

int gbmd_set_cell_scale(gbmd_system* s, double scale) {
  if (!s) return fail(GBMD_ERR_BAD_ARG, "system is NULL");
  RET(use_device(s->device));
  return regrid(s, scale);
}

int gbmd_set_force_events(gbmd_system* s, void* ev_begin, void* ev_end) {
  if (!s || (!ev_begin) != (!ev_end)) return fail(GBMD_ERR_BAD_ARG, "bad argument");
  RET(use_device(s->device));
  Group* g = s->batch ? s->batch : s->own;
  cudaEvent_t b = (cudaEvent_t)ev_begin, e = (cudaEvent_t)ev_end;
  const bool had = g->ev_begin != nullptr;
  g->ev_begin = b;
  g->ev_end = e;
  if (had && b && g->exec_one && g->node_ev_begin && !g->graphs_dirty) {
    CK(cudaGraphExecEventRecordNodeSetEvent(g->exec_one, g->node_ev_begin, b));
    CK(cudaGraphExecEventRecordNodeSetEvent(g->exec_one, g->node_ev_end, e));
    return GBMD_OK;
  }
  destroy_graphs(g);   // rebuilt with (or without) the records at the next step
  return GBMD_OK;
}

int gbmd_autotune(gbmd_system* s, const char* cache_path) {
  Range nvtx_range("gbmd_autotune");
  if (!s) return fail(GBMD_ERR_BAD_ARG, "system is NULL");
  RET(use_device(s->device));
  if (s->batch) return fail(GBMD_ERR_STATE, "system belongs to a batch");
  RET(sync_system(s));
  return autotune_group(s->own, cache_path);
}

int gbmd_set_tuning(gbmd_system* s, int32_t tpp, int32_t block) {
  if (!s) return fail(GBMD_ERR_BAD_ARG, "system is NULL");
  RET(use_device(s->device));
  RET(sync_system(s));
  return set_tuning(s->own, tpp, block);
}

// ---- batches ----

int gbmd_batch_create(int32_t precision, void* stream, int32_t device, gbmd_batch** out) {
  if (!out || (precision != GBMD_FP64 && precision != GBMD_MIXED)) return fail(GBMD_ERR_BAD_ARG, "bad argument");
  int dev = device;
  if (dev < 0) CK(cudaGetDevice(&dev));
  RET(use_device(dev));
  Group* g = new Group();
  g->device = dev;
  g->is_batch = true;
  g->precision = precision;
  g->stream = (cudaStream_t)stream;
  if (const char* ev = getenv("GBMD_NO_GRAPHS")) g->use_graphs = ev[0] != '1';
  *out = reinterpret_cast<gbmd_batch*>(g);
  return GBMD_OK;
}

// A member's own readouts (forces, thermo, state) run on its single-system group;
// they take the batch's tuning, so that (with FP64 sums depending on the lanes per
// particle) a member reads back what a system stepped alone at that tuning does.
static void follow_batch_tuning(Group* b) {
  for (auto* m : live(b)) {
    if (m->own->tpp != b->tpp || m->own->fblock != b->fblock) {
      m->own->tpp = b->tpp;
      m->own->fblock = b->fblock;
      m->own->layout_dirty = true;
    }
  }
}

int gbmd_batch_add(gbmd_batch* bh, gbmd_system* s, int32_t* slot) {
  Group* b = reinterpret_cast<Group*>(bh);
  if (!b || !s || !slot) return fail(GBMD_ERR_BAD_ARG, "NULL argument");
  RET(use_device(reinterpret_cast<Group*>(bh)->device));
  if (s->batch) return fail(GBMD_ERR_STATE, "system already in a batch");
  if (s->h.n_ghost > 0) return fail(GBMD_ERR_BAD_ARG, "a system with ghosts cannot join a batch");
  if (s->h.precision != b->precision) return fail(GBMD_ERR_BAD_ARG, "precision mismatch");
  for (auto* m : live(b)) {
    if (m->h.nvt != s->h.nvt) return fail(GBMD_ERR_BAD_ARG, "a batch holds NVE or NVT systems, not both");
    if (m->h.eval != s->h.eval)
      return fail(GBMD_ERR_BAD_ARG, "a batch holds systems of one pair evaluator (LJ and WCA share one)");
  }
  if (s->device != b->device) return fail(GBMD_ERR_BAD_ARG, "system and batch are on different devices");
  RET(sync_system(s));
  CK(cudaStreamSynchronize(b->stream));
  int k = -1;
  for (size_t i = 0; i < b->members.size(); ++i)
    if (!b->members[i]) { k = (int)i; break; }
  if (k < 0) {
    k = (int)b->members.size();
    b->members.push_back(nullptr);
  }
  b->members[k] = s;
  s->batch = b;
  s->batch_slot = k;
  s->own->stream = b->stream;
  b->layout_dirty = true;
  follow_batch_tuning(b);
  *slot = k;
  return GBMD_OK;
}

int gbmd_batch_remove(gbmd_batch* bh, int32_t slot) {
  Group* b = reinterpret_cast<Group*>(bh);
  if (!b || slot < 0 || slot >= (int)b->members.size() || !b->members[slot])
    return fail(GBMD_ERR_BAD_ARG, "bad slot");
  RET(use_device(reinterpret_cast<Group*>(bh)->device));
  gbmd_system* s = b->members[slot];
  RET(sync_system(s));
  CK(cudaStreamSynchronize(b->stream));
  b->members[slot] = nullptr;
  s->batch = nullptr;
  s->batch_slot = -1;
  s->own->stream = s->stream;
  b->layout_dirty = true;
  return GBMD_OK;
}

int gbmd_batch_step(gbmd_batch* bh, int64_t nsteps) {
  Range nvtx_range("gbmd_batch_step");
  Group* b = reinterpret_cast<Group*>(bh);
  if (!b || nsteps < 0) return fail(GBMD_ERR_BAD_ARG, "bad argument");
  RET(use_device(reinterpret_cast<Group*>(bh)->device));
  for (auto* s : live(b)) s->target_step += nsteps;
  return enqueue_steps(b, nsteps);
}

int gbmd_batch_sync(gbmd_batch* bh) {
  Range nvtx_range("gbmd_batch_sync");
  Group* b = reinterpret_cast<Group*>(bh);
  if (!b) return fail(GBMD_ERR_BAD_ARG, "NULL batch");
  RET(use_device(reinterpret_cast<Group*>(bh)->device));
  CK(cudaStreamSynchronize(b->stream));
  int first = GBMD_OK;
  std::string msg;
  for (auto* s : live(b)) {
    int rc = sync_system(s);
    if (rc != GBMD_OK && first == GBMD_OK) {
      first = rc;
      msg = g_err;
    }
  }
  if (first != GBMD_OK) g_err = msg;
  return first;
}

int gbmd_batch_autotune(gbmd_batch* bh, const char* cache_path) {
  Range nvtx_range("gbmd_batch_autotune");
  Group* b = reinterpret_cast<Group*>(bh);
  if (!b) return fail(GBMD_ERR_BAD_ARG, "NULL batch");
  RET(use_device(reinterpret_cast<Group*>(bh)->device));
  RET(gbmd_batch_sync(bh));
  if (live(b).empty()) return GBMD_OK;
  RET(autotune_group(b, cache_path));
  follow_batch_tuning(b);
  return GBMD_OK;
}

int gbmd_batch_set_tuning(gbmd_batch* bh, int32_t tpp, int32_t block) {
  Group* b = reinterpret_cast<Group*>(bh);
  if (!b) return fail(GBMD_ERR_BAD_ARG, "NULL batch");
  RET(use_device(reinterpret_cast<Group*>(bh)->device));
  RET(gbmd_batch_sync(bh));
  RET(set_tuning(b, tpp, block));
  follow_batch_tuning(b);
  return GBMD_OK;
}

int gbmd_batch_info(gbmd_batch* bh, int32_t* members, int64_t* particles, int64_t* launches) {
  Group* b = reinterpret_cast<Group*>(bh);
  if (!b) return fail(GBMD_ERR_BAD_ARG, "NULL batch");
  RET(use_device(reinterpret_cast<Group*>(bh)->device));
  std::vector<gbmd_system*> m = live(b);
  if (members) *members = (int32_t)m.size();
  if (particles) {
    int64_t np = 0;
    for (auto* s : m) np += s->h.n;
    *particles = np;
  }
  if (launches) {
    GroupCtl c{};
    if (b->d_ctl) {
      CK(cudaMemcpyAsync(&c, b->d_ctl, sizeof(c), cudaMemcpyDeviceToHost, b->stream));
      CK(cudaStreamSynchronize(b->stream));
    }
    *launches = (int64_t)c.launches;
  }
  return GBMD_OK;
}

int gbmd_batch_destroy(gbmd_batch* bh) {
  Group* b = reinterpret_cast<Group*>(bh);
  if (!b) return fail(GBMD_ERR_BAD_ARG, "NULL batch");
  use_device(b->device);
  cudaStreamSynchronize(b->stream);
  for (auto* s : live(b)) {
    s->batch = nullptr;
    s->batch_slot = -1;
    s->own->stream = s->stream;
  }
  destroy_graphs(b);
  cudaFree(b->d_desc); cudaFree(b->d_tp); cudaFree(b->d_tf); cudaFree(b->d_tc); cudaFree(b->d_te); cudaFree(b->d_nhpart);
  cudaFree(b->d_ts); cudaFree(b->d_tb); cudaFree(b->d_tbk); cudaFree(b->d_tt); cudaFree(b->d_partials);
  cudaFree(b->d_ctl);
  delete b;
  return GBMD_OK;
}

}  // extern "C"

// ============================================================================
// Allocation-free thermo readout (gbmd_get_thermo_noalloc)
//
// For callers that may not allocate GPU memory.  The scratch the energy/virial
// kernels need -- per-tile FP64 partial sums and the descriptor copy they read --
// lives in the static device arrays below; host code only ever passes their
// device addresses (looked up once per device with cudaGetSymbolAddress), never
// the symbols themselves.
// ============================================================================
namespace {

constexpr int kNoallocMaxTiles = GBMD_NOALLOC_MAX_TILES;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[8 * kNoallocMaxTiles];   // 2 MiB
static __device__ __align__(256) SysDev g_noalloc_desc;

struct NoallocAddrs {
  bool ready = false;
  double* partials = nullptr;
  SysDev* desc = nullptr;
};
NoallocAddrs g_noalloc_addrs[kNoallocMaxDevices];
std::mutex g_noalloc_mutex;

// once per device, with that device current
int noalloc_setup(int dev, NoallocAddrs* out) {
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(GBMD_ERR_BAD_ARG, "device ordinal %d too large", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoallocAddrs& a = g_noalloc_addrs[dev];
  if (!a.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return fail(GBMD_ERR_CUDA, "cudaGetSymbolAddress(partials): %s", cudaGetErrorString(e));
    a.partials = static_cast<double*>(p);
    e = cudaGetSymbolAddress(&p, g_noalloc_desc);
    if (e != cudaSuccess) return fail(GBMD_ERR_CUDA, "cudaGetSymbolAddress(descriptor): %s", cudaGetErrorString(e));
    a.desc = static_cast<SysDev*>(p);
    a.ready = true;
  }
  *out = a;
  return GBMD_OK;
}

}  // namespace

extern "C" int gbmd_get_thermo_noalloc(gbmd_system* s, gbmd_thermo* out) {
  if (!s || !out) return fail(GBMD_ERR_BAD_ARG, "NULL argument");
  RET(use_device(s->device));
  NoallocAddrs addr;
  RET(noalloc_setup(s->device, &addr));
  Group* g = s->own;
  cudaStream_t st = g->stream;
  // finish queued work without any recovery that could allocate
  CK(cudaStreamSynchronize(st));
  Flags f;
  RET(read_flags(s, &f, st));
  if (f.error == DEV_NONFINITE) return fail(GBMD_ERR_NONFINITE, "non-finite state (step %lld)", f.step);
  if (f.error) return fail(GBMD_ERR_STATE, "pending device error %d: call gbmd_sync first", f.error);
  long long want = s->target_step;
  if (s->step_limit >= 0) want = std::min(want, s->step_limit);
  if (f.step < want) return fail(GBMD_ERR_STATE, "steps still owed after a recovery: call gbmd_sync first");
  if (g->layout_dirty) return fail(GBMD_ERR_STATE, "layout changed: call gbmd_sync or gbmd_get_thermo first");
  if (g->nte + g->ntb > kNoallocMaxTiles)
    return fail(GBMD_ERR_BAD_ARG, "%d energy tiles exceed the allocation-free limit of %d",
                g->nte + g->ntb, kNoallocMaxTiles);
  // the system's descriptor, pointed at the static partials (own group: tiles from 0)
  SysDev d = s->h;
  d.tile_first_f = 0;
  d.tile_count_f = g->nte + g->ntb;   // the system alone: one of the two is zero
  d.partials = addr.partials;
  CK(cudaMemcpyAsync(addr.desc, &d, sizeof(SysDev), cudaMemcpyHostToDevice, st));
  if (g->ntf > 0) CK(launch(ev_force_call(g, addr.desc), st));
  if (g->ntb > 0)
    CK(launch(force_staged_call(g->multi, MODE_EV, addr.desc, g->d_tb, g->ntb, g->d_ctl, 0,
                                g->window_cap, StepArgs{}), st));
  CK(launch(thermo_call(addr.desc, g->d_ts, g->nts, g->d_ctl), st));
  double t[8];
  CK(cudaMemcpyAsync(t, s->d_thermo, sizeof(t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));   // `d` and `t` are host stack memory
  const double n = (double)s->h.n;
  const double vol = s->h.L[0] * s->h.L[1] * s->h.L[2];
  out->step = f.step;
  out->pe = t[0];
  out->ke = 0.5 * s->h.mass * t[1];
  out->temperature = n > 1 ? 2.0 * out->ke / (3.0 * n - 3.0) : 0.0;
  for (int c = 0; c < 6; ++c) out->virial[c] = t[2 + c];
  out->w = t[2] + t[5] + t[7];
  out->pressure = (n * out->temperature + out->w / 3.0) / vol;
  out->n_rebuilds = f.n_rebuilds;
  return fill_thermostat(s, f, out);
}
