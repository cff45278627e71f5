// C ABI of the HHG library (include/hhg.h): device storage, the V-cycle
// driver, the fault / recovery paths and the solve loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "../../include/hhg.h"
#include "hhg_kernels.h"

using namespace hhg;

namespace {

thread_local std::string g_err;
thread_local int g_err_code = HHG_OK;

int fail(int code, const std::string& msg) {
  g_err = msg;
  g_err_code = code;
  return code;
}

#define HHG_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? HHG_ERR_OOM : HHG_ERR_CUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

#define HHG_TRY(expr)            \
  do {                           \
    int rc_ = (expr);            \
    if (rc_ != HHG_OK) return rc_; \
  } while (0)

// Timing events of one call, destroyed on every return path.
struct CallEvents {
  cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
  CallEvents() = default;
  CallEvents(const CallEvents&) = delete;
  CallEvents& operator=(const CallEvents&) = delete;
  ~CallEvents() {
    for (cudaEvent_t x : e)
      if (x) cudaEventDestroy(x);
  }
  cudaError_t create(int n) {
    for (int i = 0; i < n; ++i) {
      const cudaError_t r = cudaEventCreate(&e[i]);
      if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
  }
};

template <class T>
struct Prec {
  std::vector<DevLevel<T>> lv;
  std::vector<T*> Winv;
};

}  // namespace

struct hhg_mesh {
  HostMesh host;
  int device = 0;
  int precision = 64;
  std::vector<DevLevelTables> tab;
  Prec<double> d64;
  // 7-point stencils: the finest level's f and interior weights divided by
  // each macro's centre weight (the FP64 volume Gauss-Seidel reads these)
  double* fs_top = nullptr;
  double* wsc_top = nullptr;
  // general connectivity: every interface copy of the finest level (block
  // offset, master), to fill the ghost shells after an import
  int64_t* gen_copy_off = nullptr;
  int* gen_copy_master = nullptr;
  int n_gen_copy = 0;
  Prec<float> d32;
  MacroGeo* geo = nullptr;
  DevProblem global, faulty, healthy;
  std::vector<unsigned char> fault_set;
  bool has_fault = false;
  // fault bookkeeping on the finest level
  int* fault_zero_ids = nullptr;
  int n_fault_zero = 0;
  int64_t* fault_restore_off = nullptr;
  int* fault_restore_master = nullptr;
  int n_fault_restore = 0;
  // Dirichlet-Neumann recovery (§4.3, Algorithm 2) on the finest level:
  // the Omega_I problem (kind 3), its interface right-hand side with the
  // frozen flux on Gamma, the Gamma masters, the copies of Gamma inside the
  // faulty blocks, and two snapshots of the masters
  DevProblem dn;
  std::vector<unsigned char> dn_set;
  bool has_dn = false;
  int* dn_gamma = nullptr;
  int n_dn_gamma = 0;
  int64_t* dn_off = nullptr;
  int* dn_master = nullptr;
  int n_dn_copy = 0;
  double* dn_snap[2] = {nullptr, nullptr};
  cudaEvent_t ev_dn_e = nullptr, ev_dn_r[2] = {nullptr, nullptr};
  double* staging = nullptr;
  cudaStream_t side = nullptr;       // highest priority: the Omega_F side of a recovery
  int prio_hi = 0;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // one recovery cycle of the faulty problem captured as a CUDA graph and
  // replayed for the later cycles of a recovery (few macros, many small
  // launches); valid for the current fault set and cycle parameters
  cudaStream_t cap = nullptr;
  cudaGraphExec_t local_exec = nullptr;
  long long local_kernels = 0;  // kernels in the captured cycle
  bool local_failed = false;
  bool local_mixed = false;
  int local_pre = 0, local_post = 0, local_maxit = 0;
  double local_rtol = 0.0;
  std::vector<void*> allocs;
  std::unordered_map<void*, int64_t> alloc_bytes;
  // allocations of the current fault set (its sub-problems and lists), freed
  // when another set replaces it; `collect`, when set, receives new ones
  std::vector<void*> fault_allocs, dn_allocs;
  std::vector<void*>* collect = nullptr;
  int batch_refs = 0;              // batch graphs that hold this mesh's buffers
  int64_t bytes = 0;
  double* host_scalar = nullptr;   // pinned
  double* grad_partial = nullptr;  // coefficient-gradient partial sums
  double* grad_out = nullptr;
  // CTAs per fused launch at most (0: as many as are resident; hhg_set_launch_limit)
  int grid_cap = 0;
  // streaming 7-point Gauss-Seidel (hhg_set_streaming) and the bounded device
  // waits: their error flag (device) and tries (hhg_set_wait_limit)
  int stream_gs = 0;
  int* dev_err = nullptr;
  int wait_limit = 1 << 24;
  int* host_flag = nullptr;        // pinned
  // phase breakdown of the global cycles (hhg_profile_enable bit 1): an event
  // at every phase boundary and the phase that starts there
  bool bd_on = false;
  std::vector<cudaEvent_t> bd_ev;
  std::vector<int> bd_cat;
  size_t bd_used = 0;
  bool coeff_dirty = false;   // host coefficients changed, device stencils not yet
  // profiling of the finest-level Gauss-Seidel volume kernel of the global problem
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;
  size_t prof_used = 0;
};

struct hhg_batch {
  struct Task {
    hhg_mesh* mesh;
    int cycles;
    cudaStream_t stream;
    cudaEvent_t done;       // join dependency inside the capture
    cudaEvent_t done_time;  // event-record node: completion time of the task
  };
  std::vector<Task> tasks;       // recovery tasks, then (optionally) the global one
  bool mixed = false;
  cudaStream_t origin = nullptr;
  cudaEvent_t start = nullptr, fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;  // kernels in the graph
  // persistent executor (hhg_batch_launch_persistent): every task's
  // operations in order, run by one launch of the scheduler kernel
  std::vector<BOp> ops;
  std::vector<int> op_off;               // task t: ops [op_off[t], op_off[t + 1])
  BOp* d_ops = nullptr;
  int* d_op_off = nullptr;
  int* d_state = nullptr;                // phase[n] | issued[n_ops] | done[n_ops] | tasks_done
  size_t state_bytes = 0;
  unsigned long long* d_ns = nullptr;    // start | completion of task t (globaltimer ns)
  int* d_err = nullptr;
  int* d_order = nullptr;                // tasks by priority class, highest first
  int* d_seg = nullptr;                  // class c: d_order[d_seg[c] .. d_seg[c + 1])
  int n_seg = 1;
  int wait_limit = 1 << 24;
};

namespace {

template <class T>
int dalloc(hhg_mesh* m, T** p, size_t n) {
  *p = nullptr;
  if (n == 0) return HHG_OK;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(HHG_ERR_OOM, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed: " +
                                 cudaGetErrorString(e));
  }
  m->allocs.push_back(q);
  m->alloc_bytes[q] = (int64_t)(n * sizeof(T));
  if (m->collect) m->collect->push_back(q);
  m->bytes += (int64_t)(n * sizeof(T));
  *p = static_cast<T*>(q);
  return HHG_OK;
}

// Free the allocations in `list` (cudaFree waits for the device), unless a
// batch graph still refers to the mesh's buffers (then they stay until the
// mesh is destroyed).
void release(hhg_mesh* m, std::vector<void*>& list) {
  if (m->batch_refs > 0) {
    list.clear();
    return;
  }
  if (!list.empty()) cudaDeviceSynchronize();   // nothing in flight may still use them
  for (void* q : list) {
    cudaFree(q);
    m->bytes -= m->alloc_bytes[q];
    m->alloc_bytes.erase(q);
    m->allocs.erase(std::find(m->allocs.begin(), m->allocs.end(), q));
  }
  list.clear();
}

// Collect the allocations made while this object lives into `list`.
struct Collect {
  hhg_mesh* m;
  std::vector<void*>* prev;
  Collect(hhg_mesh* mm, std::vector<void*>& list) : m(mm), prev(mm->collect) { m->collect = &list; }
  ~Collect() { m->collect = prev; }
};

template <class T>
int upload(hhg_mesh* m, T** p, const std::vector<T>& v) {
  HHG_TRY(dalloc(m, p, v.size()));
  if (!v.empty()) HHG_CUDA(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HHG_OK;
}

void free_all(hhg_mesh* m) {
  for (void* p : m->allocs) cudaFree(p);
  m->allocs.clear();
  m->alloc_bytes.clear();
}

LevelArgs largs(const hhg_mesh* m, int l) {
  const HostLevel& H = m->host.lv[l];
  const DevLevelTables& t = m->tab[l];
  LevelArgs a;
  a.N = H.N;
  a.rs = t.SL;
  a.block = H.block;
  a.if_gid = t.if_gid;
  a.cptr = t.if_cptr;
  a.cps = t.if_copy;
  a.cp_off = t.cp_off;
  a.tiles_int = t.tiles_int;
  a.n_tiles_int = t.n_tiles_int;
  a.tiles_all = t.tiles_all;
  a.n_tiles_all = t.n_tiles_all;
  a.tiles_stream = t.tiles_stream;
  a.n_tiles_stream = t.n_tiles_stream;
  a.stream_band = H.stream_band;
  a.tiles_stream32 = t.tiles_stream32;
  a.n_tiles_stream32 = t.n_tiles_stream32;
  a.stream_band32 = H.stream_band32;
  a.gs_items64 = t.gs_items64;
  a.gs_items32 = t.gs_items32;
  for (int c = 0; c < 5; ++c) {
    a.gs_off64[c] = t.gs_off64[c];
    a.gs_off32[c] = t.gs_off32[c];
  }
  a.slot_items = t.slot_items;
  a.n_slots = t.n_slots;
  a.gs_flat = t.gs_flat;
  return a;
}

// Level arguments seen by problem p: kind 3 reaches interface nodes through
// its own (healthy) copies only.
LevelArgs plargs(const hhg_mesh* m, const DevProblem& p, int l) {
  LevelArgs a = largs(m, l);
  if (p.lv[l].cptr) {
    a.cptr = p.lv[l].cptr;
    a.cps = p.lv[l].cps;
    a.cp_off = p.lv[l].cp_off;
  }
  return a;
}

// Interface right-hand side of level l (the finest one may be replaced by
// the problem's own, FP64 only).
template <class T>
const T* level_fI(const DevLevel<T>& D, const DevProblem&, bool) {
  return D.fI;
}
template <>
const double* level_fI<double>(const DevLevel<double>& D, const DevProblem& p, bool top) {
  return top && p.fI_top ? p.fI_top : D.fI;
}

ProbArgs pargs(const DevProblem& p, int l) {
  ProbArgs a;
  a.act = p.act;
  a.n_act = p.n_act;
  const DevProblemLevel& q = p.lv[l];
  a.free_if = q.free_if;
  for (int c = 0; c < 5; ++c) a.col_off[c] = q.col_off[c];
  a.zero_off = q.zero_off;
  a.n_zero = q.n_zero;
  a.gather = q.gather;
  a.sched = p.sched;
  a.grid_cap = p.grid_cap;
  a.tnb = q.tnb;
  a.tw64 = q.tw64;
  a.td64 = q.td64;
  a.ti64 = q.ti64;
  a.tw32 = q.tw32;
  a.td32 = q.td32;
  a.ti32 = q.ti32;
  a.tn = q.tn;
  a.stream_gs = p.stream_gs;
  a.err = p.err;
  a.wait_limit = p.wait_limit;
  return a;
}

// Interface stencil tables (weights, diagonal, inverse diagonal) of problem
// level l from the current stencils; allocates on the first call (device
// pointers null), else overwrites the weights in place (new coefficients).
// Levels of general meshes, the coarsest level and meshes whose offsets need
// more than 32 bits keep the per-copy path (tables null).
int upload_if_tables(hhg_mesh* m, DevProblemLevel& q, int l, int kind, const std::vector<int>& free_if,
                     const std::vector<int>& pcptr, const std::vector<Copy>& pcopies) {
  if (l == 0 || free_if.empty()) return HHG_OK;
  const HostLevel& H = m->host.lv[l];
  const std::vector<int>& cptr = kind == 3 ? pcptr : H.if_cptr;
  const std::vector<Copy>& copies = kind == 3 ? pcopies : H.if_copy;
  const int K = m->host.seven_point ? 6 : 14;
  std::vector<uint32_t> nb;
  std::vector<double> w, dg;
  if (!build_if_tables(m->host, l, free_if, cptr, copies, K, nb, w, dg)) return HHG_OK;
  const size_t n = free_if.size();
  std::vector<double> di(n);
  for (size_t i = 0; i < n; ++i) di[i] = 1.0 / dg[i];
  const bool fresh = q.tnb == nullptr;
  if (fresh) {
    HHG_TRY(upload(m, &q.tnb, nb));
    HHG_TRY(dalloc(m, &q.tw64, w.size()));
    HHG_TRY(dalloc(m, &q.td64, n));
    HHG_TRY(dalloc(m, &q.ti64, n));
    if (m->precision == 32) {
      HHG_TRY(dalloc(m, &q.tw32, w.size()));
      HHG_TRY(dalloc(m, &q.td32, n));
      HHG_TRY(dalloc(m, &q.ti32, n));
    }
    q.tn = (int)n;
  } else if ((size_t)q.tn != n) {
    return fail(HHG_ERR_STATE, "interface table changed shape");
  }
  HHG_CUDA(cudaMemcpy(q.tw64, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
  HHG_CUDA(cudaMemcpy(q.td64, dg.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  HHG_CUDA(cudaMemcpy(q.ti64, di.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  if (q.tw32) {
    std::vector<float> w32(w.begin(), w.end()), d32(dg.begin(), dg.end()), i32(n);
    for (size_t i = 0; i < n; ++i) i32[i] = (float)(1.0 / (double)d32[i]);
    HHG_CUDA(cudaMemcpy(q.tw32, w32.data(), w32.size() * sizeof(float), cudaMemcpyHostToDevice));
    HHG_CUDA(cudaMemcpy(q.td32, d32.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    HHG_CUDA(cudaMemcpy(q.ti32, i32.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  }
  return HHG_OK;
}

int upload_problem(hhg_mesh* m, const HostProblem& h, DevProblem& d) {
  d.kind = h.kind;
  d.act_host = h.act;
  d.macro_active_host = h.macro_active;
  d.free0_host = h.lv.empty() ? std::vector<int>() : h.lv[0].free_if;
  d.free_host.clear();
  for (const HostProblemLevel& q : h.lv) d.free_host.push_back(q.free_if);
  d.n_act = (int)h.act.size();
  HHG_TRY(upload(m, &d.act, h.act));
  d.lv.assign(h.lv.size(), DevProblemLevel());
  for (size_t l = 0; l < h.lv.size(); ++l) {
    HHG_TRY(upload(m, &d.lv[l].free_if, h.lv[l].free_if));
    for (int c = 0; c < 5; ++c) d.lv[l].col_off[c] = h.lv[l].col_off[c];
    HHG_TRY(upload(m, &d.lv[l].zero_off, h.lv[l].zero_off));
    d.lv[l].n_zero = (int)h.lv[l].zero_off.size();
    HHG_TRY(upload(m, &d.lv[l].gather, h.lv[l].gather));
    HHG_TRY(upload(m, &d.lv[l].cptr, h.lv[l].cptr));
    HHG_TRY(upload(m, &d.lv[l].cps, h.lv[l].copies));
    if (!h.lv[l].copies.empty()) {
      std::vector<uint32_t> off;
      if (copy_offsets(m->host, (int)l, h.lv[l].copies, off)) HHG_TRY(upload(m, &d.lv[l].cp_off, off));
    }
    HHG_TRY(upload_if_tables(m, d.lv[l], (int)l, h.kind, h.lv[l].free_if, h.lv[l].cptr, h.lv[l].copies));
    HHG_TRY(upload(m, &d.lv[l].gptr, h.lv[l].gptr));
    HHG_TRY(upload(m, &d.lv[l].goff, h.lv[l].goff));
    d.lv[l].class_off = h.lv[l].class_off;
  }
  d.n_cg = h.n_cg;
  d.nnz = (int64_t)h.val.size();
  HHG_TRY(upload(m, &d.rowptr, h.rowptr));
  HHG_TRY(upload(m, &d.col, h.col));
  HHG_TRY(upload(m, &d.val, h.val));
  HHG_TRY(upload(m, &d.fsrc, h.fsrc));
  HHG_TRY(upload(m, &d.uptr, h.uptr));
  HHG_TRY(upload(m, &d.udst, h.udst));
  HHG_TRY(upload(m, &d.umaster, h.umaster));
  HHG_TRY(dalloc(m, &d.cg_work, (size_t)4 * std::max(1, h.n_cg)));
  const int L = (int)m->host.lv.size() - 1;
  d.n_partial = m->tab[L].n_tiles_int * std::max(1, d.n_act) + (m->host.lv[L].n_if + 127) / 128 + 64;
  HHG_TRY(dalloc(m, &d.partial, (size_t)d.n_partial));
  HHG_TRY(dalloc(m, &d.scalar, 8));
  HHG_TRY(dalloc(m, &d.cg_iters, 4));
  HHG_TRY(dalloc(m, &d.sched, 4));
  HHG_CUDA(cudaMemset(d.sched, 0, 4 * sizeof(int)));
  d.grid_cap = m->grid_cap;
  d.stream_gs = m->stream_gs;
  d.err = m->dev_err;
  d.wait_limit = m->wait_limit;
  return HHG_OK;
}

template <class T>
int alloc_levels(hhg_mesh* m, Prec<T>& P, bool with_r_on_finest) {
  const int nl = (int)m->host.lv.size();
  P.lv.assign(nl, DevLevel<T>());
  P.Winv.assign(nl, nullptr);
  for (int l = 0; l < nl; ++l) {
    const HostLevel& H = m->host.lv[l];
    DevLevel<T>& D = P.lv[l];
    D.N = H.N;
    D.block = H.block;
    D.n_if = H.n_if;
    const size_t nb = (size_t)m->host.n_macro * H.block;
    HHG_TRY(dalloc(m, &D.u, nb));
    HHG_TRY(dalloc(m, &D.f, nb));
    if (l < nl - 1 || with_r_on_finest) HHG_TRY(dalloc(m, &D.r, nb));
    HHG_TRY(dalloc(m, &D.uI, (size_t)std::max(1, H.n_if)));
    HHG_TRY(dalloc(m, &D.fI, (size_t)std::max(1, H.n_if)));
    HHG_CUDA(cudaMemset(D.u, 0, nb * sizeof(T)));
    HHG_CUDA(cudaMemset(D.f, 0, nb * sizeof(T)));
    if (D.r) HHG_CUDA(cudaMemset(D.r, 0, nb * sizeof(T)));
    HHG_CUDA(cudaMemset(D.uI, 0, std::max(1, H.n_if) * sizeof(T)));
    HHG_CUDA(cudaMemset(D.fI, 0, std::max(1, H.n_if) * sizeof(T)));
    std::vector<T> w(H.W.size()), winv(m->host.n_macro);
    for (size_t q = 0; q < w.size(); ++q) w[q] = (T)H.W[q];
    for (int t = 0; t < m->host.n_macro; ++t) winv[t] = (T)(1.0 / H.W[(size_t)t * 16 * NDIR]);
    HHG_TRY(upload(m, &D.W, w));
    HHG_TRY(upload(m, &P.Winv[l], winv));
  }
  return HHG_OK;
}

// The finest level's interior weights divided by the centre weight, per macro
// (same table layout as W, other node classes zero), uploaded to wsc_top, and
// fs_top = f scaled the same way (on the legacy stream, after the copies).
int refresh_scaled(hhg_mesh* m) {
  if (!m->wsc_top) return HHG_OK;
  const int L = (int)m->host.lv.size() - 1;
  const HostLevel& H = m->host.lv[L];
  std::vector<double> w(H.W.size(), 0.0);
  for (int t = 0; t < m->host.n_macro; ++t) {
    const size_t o = (size_t)t * 16 * NDIR;
    const double inv = 1.0 / H.W[o];
    for (int d = 0; d < NDIR; ++d) w[o + d] = H.W[o + d] * inv;
  }
  HHG_CUDA(cudaMemcpy(m->wsc_top, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
  HHG_CUDA(scale_blocks(m->d64.lv[L].f, m->d64.Winv[L], m->fs_top, m->host.n_macro, H.block, 0));
  HHG_CUDA(cudaStreamSynchronize(0));
  return HHG_OK;
}

int alloc_scaled(hhg_mesh* m) {
  if (!m->host.seven_point) return HHG_OK;
  const int L = (int)m->host.lv.size() - 1;
  const HostLevel& H = m->host.lv[L];
  HHG_TRY(dalloc(m, &m->fs_top, (size_t)m->host.n_macro * H.block));
  HHG_TRY(dalloc(m, &m->wsc_top, H.W.size()));
  return refresh_scaled(m);
}

// One V(pre, post) cycle of problem p on the arrays of precision T.
// A pair of events bracketing the next profiled launch (none when profiling
// is off).
int prof_pair(hhg_mesh* m, cudaEvent_t* b, cudaEvent_t* e) {
  *b = *e = nullptr;
  if (!m->prof_on) return HHG_OK;
  while (m->prof_ev.size() < m->prof_used + 2) {
    cudaEvent_t ev;
    HHG_CUDA(cudaEventCreate(&ev));
    m->prof_ev.push_back(ev);
  }
  *b = m->prof_ev[m->prof_used];
  *e = m->prof_ev[m->prof_used + 1];
  m->prof_used += 2;
  return HHG_OK;
}

// profile = false keeps the profiling hook (which creates events) out.
// Phases of the breakdown: fine-level smoothing, fine residual, restriction
// from and prolongation to the fine level, the levels below (smoothing,
// residuals, transfers), coarse CG, the stopping test's residual and norm
// (with iterative refinement: the FP64 residual), the time until the host
// issues the next work (read-back of the norm, launch), fault injection and
// recovery, and the FP32 correction's zeroing and addition (mixed precision).
enum { BD_FINE_SMOOTH, BD_FINE_RES, BD_RESTRICT, BD_PROLONG, BD_COARSE, BD_CG, BD_NORM, BD_HOST, BD_RECOVERY,
       BD_IR, BD_N };

// Start of phase `cat` on stream s (breakdown enabled, global problem only).
int bd_mark(hhg_mesh* m, cudaStream_t s, int cat) {
  if (!m->bd_on) return HHG_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  HHG_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return HHG_OK;
  if (m->bd_ev.size() <= m->bd_used) {
    cudaEvent_t ev;
    HHG_CUDA(cudaEventCreate(&ev));
    m->bd_ev.push_back(ev);
    m->bd_cat.push_back(0);
  }
  HHG_CUDA(cudaEventRecord(m->bd_ev[m->bd_used], s));
  m->bd_cat[m->bd_used] = cat;
  ++m->bd_used;
  return HHG_OK;
}

template <class T>
int smooth(hhg_mesh* m, Prec<T>& P, DevProblem& p, int l, int steps, cudaStream_t s, bool profile = true) {
  const int L = (int)P.lv.size() - 1;
  DevLevel<T>& D = P.lv[l];
  const LevelArgs a = plargs(m, p, l);
  const ProbArgs q = pargs(p, l);
  const T* fI = level_fI<T>(D, p, l == L);
  const bool prof = profile && l == L && p.kind == 0;
  const T* fs = nullptr;
  const T* wsc = nullptr;
  if constexpr (std::is_same<T, double>::value)
    if (l == L) {
      fs = m->fs_top;
      wsc = m->wsc_top;
    }
  if (m->host.general) {
    // general connectivity: the four volume colours without interface nodes,
    // then the interface classes, each an interface-only launch
    ProbArgs qv = q;
    qv.col_off[4] = 0;
    ProbArgs qi = q;
    qi.n_act = 0;
    const std::vector<int>& co = p.lv[l].class_off;
    for (int it = 0; it < steps; ++it) {
      for (int c = 0; c < 4; ++c)
        HHG_CUDA(gs_colour<T>(a, qv, D.u, D.uI, D.f, fI, D.W, P.Winv[l], c, false, s));
      for (size_t c = 0; c + 1 < co.size(); ++c) {
        if (co[c + 1] == co[c]) continue;
        qi.col_off[0] = co[c];
        qi.col_off[1] = co[c + 1];
        HHG_CUDA(gs_colour<T>(a, qi, D.u, D.uI, D.f, fI, D.W, P.Winv[l], 0, false, s));
      }
    }
    return HHG_OK;
  }
  for (int it = 0; it < steps; ++it)
    for (int c = 0; c < 4; ++c) {
      cudaEvent_t b = nullptr, e = nullptr;
      if (prof) HHG_TRY(prof_pair(m, &b, &e));
      HHG_CUDA(gs_colour<T>(a, q, D.u, D.uI, D.f, fI, D.W, P.Winv[l], c, m->host.seven_point, s, b, e, fs, wsc));
    }
  return HHG_OK;
}

// Options of one cycle beyond the problem's own state: cg_work (not null)
// replaces the problem's coarse CG work vectors (4 n_cg doubles); profile =
// false leaves the cycle's Gauss-Seidel launches out of hhg_profile_enable's
// record.
struct CycleOpts {
  double* cg_work = nullptr;
  bool profile = true;
};

template <class T>
int vcycle_T(hhg_mesh* m, Prec<T>& P, DevProblem& p, int pre, int post, double cg_rtol, int cg_maxit,
             cudaStream_t s, const CycleOpts& co = CycleOpts()) {
  const int L = (int)P.lv.size() - 1;
  const bool s7 = m->host.seven_point;
  const bool bd = co.profile && p.kind == 0;
  auto mark = [&](int cat) { return bd ? bd_mark(m, s, cat) : HHG_OK; };
  for (int l = L; l >= 1; --l) {
    DevLevel<T>& D = P.lv[l];
    const LevelArgs a = plargs(m, p, l);
    const ProbArgs q = pargs(p, l);
    HHG_TRY(mark(l == L ? BD_FINE_SMOOTH : BD_COARSE));
    HHG_TRY(smooth<T>(m, P, p, l, pre, s, co.profile));
    if (l == L) HHG_TRY(mark(BD_FINE_RES));
    // after a smoothing step the last colour's residual vanishes (cube family:
    // colour 3 is smoothed last, interface nodes included)
    const int skip = pre > 0 && !m->host.general ? 3 : -1;
    HHG_CUDA(residual<T>(a, q, D.u, D.uI, D.f, level_fI<T>(D, p, l == L), D.r, D.W, s7, true, nullptr, nullptr, s,
                         skip));
    DevLevel<T>& C = P.lv[l - 1];
    if (l == L) HHG_TRY(mark(BD_RESTRICT));
    if (m->host.general) {
      // volume part as usual, interface part through the variable-length gathers
      ProbArgs qc = pargs(p, l - 1);
      ProbArgs qv = qc;
      qv.col_off[4] = 0;
      qv.n_zero = 0;
      HHG_CUDA(restrict_to<T>(plargs(m, p, l - 1), a, qv, D.r, C.f, C.fI, C.u, C.uI, s));
      HHG_CUDA(general_restrict_if<T>(plargs(m, p, l - 1), qc, p.lv[l - 1].gptr, p.lv[l - 1].goff, D.r, C.fI, C.u,
                                      C.uI, s));
      continue;
    }
    HHG_CUDA(restrict_to<T>(plargs(m, p, l - 1), a, pargs(p, l - 1), D.r, C.f, C.fI, C.u, C.uI, s));
  }
  HHG_TRY(mark(BD_CG));
  HHG_CUDA(coarse_cg<T>(p, P.lv[0].f, P.lv[0].fI, P.lv[0].u, P.lv[0].uI, cg_rtol, cg_maxit, s, co.cg_work));
  HHG_TRY(mark(BD_COARSE));
  for (int l = 1; l <= L; ++l) {
    DevLevel<T>& D = P.lv[l];
    const LevelArgs a = plargs(m, p, l);
    const ProbArgs q = pargs(p, l);
    if (l == L) HHG_TRY(mark(BD_PROLONG));
    // the first post-smoothing colour (0) overwrites its nodes without
    // reading them: their correction is not formed (interface entries of
    // colour 0 too, where the list is sorted by colour: the cube family)
    const int pskip = post > 0 ? 0 : -1;
    const int if_hi = post > 0 && !m->host.general ? q.col_off[1] : 0;
    HHG_CUDA(prolong_add<T>(a, plargs(m, p, l - 1), q, D.u, D.uI, P.lv[l - 1].u, s, pskip, q.col_off[0], if_hi));
    if (l == L) HHG_TRY(mark(BD_FINE_SMOOTH));
    HHG_TRY(smooth<T>(m, P, p, l, post, s, co.profile));
  }
  return HHG_OK;
}

// ||f - A u||^2 of problem p on the finest FP64 level, left in p.scalar[0].
// after_smoothing: the iterate comes straight from an FP64 cycle with post-
// smoothing, so the last colour's residual vanishes and is skipped.
int norm2_async(hhg_mesh* m, DevProblem& p, cudaStream_t s, bool after_smoothing = false) {
  const int L = (int)m->d64.lv.size() - 1;
  DevLevel<double>& D = m->d64.lv[L];
  int np = 0;
  const int skip = after_smoothing && !m->host.general ? 3 : -1;
  HHG_CUDA(residual<double>(plargs(m, p, L), pargs(p, L), D.u, D.uI, D.f, level_fI<double>(D, p, true), nullptr, D.W,
                            m->host.seven_point, false, p.partial, &np, s, skip));
  HHG_CUDA(reduce_partials(p.partial, np, p.scalar, s));
  return HHG_OK;
}

// Reads a device scalar (synchronising s) together with the mesh's error
// flag; a set flag (a bounded device wait ran out in an earlier kernel) is
// cleared and reported as HHG_ERR_TIMEOUT.
int read_scalar(hhg_mesh* m, const double* dev, double* out, cudaStream_t s) {
  HHG_CUDA(cudaMemcpyAsync(m->host_scalar, dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  HHG_CUDA(cudaMemcpyAsync(m->host_flag, m->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  HHG_CUDA(cudaStreamSynchronize(s));
  *out = *m->host_scalar;
  if (*m->host_flag != 0) {
    const int code = *m->host_flag;
    HHG_CUDA(cudaMemsetAsync(m->dev_err, 0, sizeof(int), s));
    HHG_CUDA(cudaStreamSynchronize(s));
    return fail(HHG_ERR_TIMEOUT, code == 1 ? "a bounded device wait ran out (the iterate is incomplete)"
                                           : "a staging range exceeded its shared-memory slot");
  }
  return HHG_OK;
}

int resnorm(hhg_mesh* m, double* out, cudaStream_t s) {
  HHG_TRY(norm2_async(m, m->global, s));
  double v = 0.0;
  HHG_TRY(read_scalar(m, m->global.scalar, &v, s));
  *out = std::sqrt(v);
  return HHG_OK;
}

// Mixed precision: one FP64 iterative-refinement step of problem p with an
// FP32 inner V-cycle.  The FP64 residual r = f - A u is formed on the finest
// level and handed to the FP32 cycle as its right-hand side (its squared norm
// is left in p.scalar[0]); the FP32 correction e (zero initial guess) is then
// added to u in FP64.
int ir_residual(hhg_mesh* m, DevProblem& p, cudaStream_t s) {
  const int L = (int)m->d64.lv.size() - 1;
  DevLevel<double>& D = m->d64.lv[L];
  DevLevel<float>& E = m->d32.lv[L];
  int np = 0;
  HHG_CUDA(residual_to_f32(plargs(m, p, L), pargs(p, L), D.u, D.uI, D.f, level_fI<double>(D, p, true), E.f, E.fI, D.W,
                           m->host.seven_point, p.partial, &np, s));
  HHG_CUDA(reduce_partials(p.partial, np, p.scalar, s));
  return HHG_OK;
}

int ir_cycle(hhg_mesh* m, DevProblem& p, int pre, int post, double cg_rtol, int cg_maxit, cudaStream_t s) {
  const int L = (int)m->d64.lv.size() - 1;
  DevLevel<float>& E = m->d32.lv[L];
  HHG_TRY(ir_residual(m, p, s));
  HHG_CUDA(zero_problem_blocks<float>(plargs(m, p, L), pargs(p, L), E.u, E.uI, s));
  HHG_TRY(vcycle_T<float>(m, m->d32, p, pre, post, cg_rtol, cg_maxit, s));
  DevLevel<double>& D = m->d64.lv[L];
  HHG_CUDA(add_correction(plargs(m, p, L), pargs(p, L), D.u, D.uI, E.u, E.uI, s));
  return HHG_OK;
}

int cycle(hhg_mesh* m, DevProblem& p, bool mixed, int pre, int post, double cg_rtol, int cg_maxit, cudaStream_t s) {
  if (mixed) return ir_cycle(m, p, pre, post, cg_rtol, cg_maxit, s);
  return vcycle_T<double>(m, m->d64, p, pre, post, cg_rtol, cg_maxit, s);
}

// Every kernel node of g runs at stream priority prio (the replayed local
// cycles keep the high priority of the stream they were captured on).
cudaError_t set_kernel_priority(cudaGraph_t g, int prio) {
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
  if (e != cudaSuccess || n == 0) return e;
  std::vector<cudaGraphNode_t> nodes(n);
  e = cudaGraphGetNodes(g, nodes.data(), &n);
  if (e != cudaSuccess) return e;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    e = cudaGraphNodeGetType(nd, &t);
    if (e != cudaSuccess) return e;
    if (t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeAttrValue v;
    std::memset(&v, 0, sizeof(v));
    v.priority = prio;
    e = cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributePriority, &v);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void drop_local_graph(hhg_mesh* m) {
  if (m->local_exec) cudaGraphExecDestroy(m->local_exec);
  m->local_exec = nullptr;
  m->local_failed = false;
}

// n cycles of the faulty problem on stream ls: the first one directly (it
// also fills the launch-shape caches), the others as replays of one captured
// cycle (captured on the mesh's own stream, so ls may be the legacy stream).
// Where capture is not possible the cycles run directly.
int local_cycles(hhg_mesh* m, int n, bool mixed, int pre, int post, double cg_rtol, int cg_maxit, cudaStream_t ls) {
  if (n <= 0) return HHG_OK;
  HHG_TRY(cycle(m, m->faulty, mixed, pre, post, cg_rtol, cg_maxit, ls));
  if (n == 1) return HHG_OK;
  const bool same = m->local_mixed == mixed && m->local_pre == pre && m->local_post == post &&
                    m->local_rtol == cg_rtol && m->local_maxit == cg_maxit;
  if (!same) drop_local_graph(m);
  // inside a caller's own stream capture the cycles are recorded directly
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  HHG_CUDA(cudaStreamIsCapturing(ls, &cs));
  if (cs != cudaStreamCaptureStatusNone) {
    for (int c = 1; c < n; ++c) HHG_TRY(cycle(m, m->faulty, mixed, pre, post, cg_rtol, cg_maxit, ls));
    return HHG_OK;
  }
  if (!m->local_exec && !m->local_failed) {
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int rc = HHG_OK;
    // captured kernels are counted as launches when the graph replays them
    const long long k0 = g_kernel_launches.load();
    if (ok) rc = cycle(m, m->faulty, mixed, pre, post, cg_rtol, cg_maxit, m->cap);
    m->local_kernels = g_kernel_launches.load() - k0;
    g_kernel_launches -= m->local_kernels;
    if (ok) ok = cudaStreamEndCapture(m->cap, &g) == cudaSuccess && rc == HHG_OK && g;
    if (ok) ok = set_kernel_priority(g, m->prio_hi) == cudaSuccess;
    if (ok) ok = cudaGraphInstantiate(&m->local_exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      cudaGetLastError();
      m->local_exec = nullptr;
      m->local_failed = true;
    }
    m->local_mixed = mixed;
    m->local_pre = pre;
    m->local_post = post;
    m->local_rtol = cg_rtol;
    m->local_maxit = cg_maxit;
  }
  for (int c = 1; c < n; ++c) {
    if (m->local_exec) {
      HHG_CUDA(cudaGraphLaunch(m->local_exec, ls));
      g_kernel_launches += m->local_kernels;
    } else HHG_TRY(cycle(m, m->faulty, mixed, pre, post, cg_rtol, cg_maxit, ls));
  }
  return HHG_OK;
}

// Entries of a global vector: the grid nodes of the cube family; for general
// connectivity the interface nodes plus every macro's volume nodes.
int64_t global_nodes(const hhg_mesh* m) {
  if (m->host.general) {
    const HostLevel& L = m->host.lv.back();
    return (int64_t)L.n_if + (int64_t)m->host.n_macro * (L.N - 1) * (L.N - 2) * (L.N - 3) / 6;
  }
  return (m->host.nx + 1) * (m->host.ny + 1) * (m->host.nz + 1);
}

int64_t global_dof(const hhg_mesh* m) {
  if (m->host.general) {
    const HostLevel& L = m->host.lv.back();
    int64_t dir = 0;
    for (unsigned char d : L.if_dirichlet) dir += d;
    return global_nodes(m) - dir;
  }
  return (m->host.nx - 1) * (m->host.ny - 1) * (m->host.nz - 1);
}

int refuse_general(const hhg_mesh* m, const char* what) {
  if (m && m->host.general)
    return fail(HHG_ERR_STATE, std::string(what) + " is not available for meshes of general connectivity");
  return HHG_OK;
}

// Every call on a mesh runs on the device the mesh was created on: that
// device must be current (the mesh's buffers, streams and the static scratch
// address of the allocation-free cycle belong to it).
int check_device(const hhg_mesh* m) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(HHG_ERR_CUDA, "cudaGetDevice failed");
  }
  if (dev != m->device)
    return fail(HHG_ERR_STATE, "the current device (" + std::to_string(dev) + ") is not the mesh's device (" +
                                   std::to_string(m->device) + ")");
  return HHG_OK;
}

const double* stage_in(hhg_mesh* m, const double* g, cudaStream_t s, int* rc) {
  *rc = HHG_OK;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, g);
  if (e != cudaSuccess) cudaGetLastError();
  if (e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) return g;
  const int64_t n = global_nodes(m);
  if (!m->staging) {
    *rc = dalloc(m, &m->staging, (size_t)n);
    if (*rc != HHG_OK) return nullptr;
  }
  e = cudaMemcpyAsync(m->staging, g, (size_t)n * sizeof(double), cudaMemcpyDefault, s);
  if (e != cudaSuccess) {
    *rc = fail(HHG_ERR_CUDA, std::string("copy of a global vector to the device: ") + cudaGetErrorString(e));
    return nullptr;
  }
  return m->staging;
}

int check_ids(const hhg_mesh* m, const int* ids, int n, std::vector<unsigned char>& set) {
  if (n <= 0 || !ids) return fail(HHG_ERR_ARG, "empty macro id list");
  set.assign(m->host.n_macro, 0);
  for (int q = 0; q < n; ++q) {
    if (ids[q] < 0 || ids[q] >= m->host.n_macro) return fail(HHG_ERR_ARG, "macro id out of range");
    if (set[ids[q]]) return fail(HHG_ERR_ARG, "duplicate macro id");
    set[ids[q]] = 1;
  }
  return HHG_OK;
}

// A problem of either mesh family (kinds as for build_problem).
void build_any_problem(const HostMesh& h, int kind, const std::vector<unsigned char>& set, HostProblem& p) {
  if (h.general) build_general_problem(h, kind, set, p);
  else build_problem(h, kind, set, p);
}

int setup_fault(hhg_mesh* m, const std::vector<unsigned char>& set) {
  if (m->has_fault && set == m->fault_set) return HHG_OK;
  HostProblem hf, hh;
  try {
    build_any_problem(m->host, 1, set, hf);
    build_any_problem(m->host, 2, set, hh);
  } catch (const std::exception& e) {
    return fail(HHG_ERR_ARG, std::string("fault set: ") + e.what());
  }
  // the previous set's sub-problems and lists (and the DN problem built on
  // them) are replaced
  drop_local_graph(m);
  release(m, m->dn_allocs);
  m->has_dn = false;
  release(m, m->fault_allocs);
  Collect keep(m, m->fault_allocs);
  HHG_TRY(upload_problem(m, hf, m->faulty));
  HHG_TRY(upload_problem(m, hh, m->healthy));
  // finest-level fault bookkeeping: masters inside Omega_F are erased; every
  // interface copy inside a lost block is restored from its master
  const int L = (int)m->host.lv.size() - 1;
  const HostLevel& H = m->host.lv[L];
  std::vector<int> zero_ids(hf.lv[L].free_if);
  std::vector<int64_t> off;
  std::vector<int> mst;
  for (int n = 0; n < H.n_if; ++n)
    for (int c = H.if_cptr[n]; c < H.if_cptr[n + 1]; ++c) {
      const Copy& cp = H.if_copy[c];
      if (!set[cp.macro]) continue;
      off.push_back((int64_t)cp.macro * H.block + lidx(H.SL.data(), H.N, cp.i, cp.j, cp.k));
      mst.push_back(n);
    }
  HHG_TRY(upload(m, &m->fault_zero_ids, zero_ids));
  m->n_fault_zero = (int)zero_ids.size();
  HHG_TRY(upload(m, &m->fault_restore_off, off));
  HHG_TRY(upload(m, &m->fault_restore_master, mst));
  m->n_fault_restore = (int)off.size();
  m->fault_set = set;
  m->has_fault = true;
  return HHG_OK;
}

int inject(hhg_mesh* m, cudaStream_t s) {
  const int L = (int)m->host.lv.size() - 1;
  DevLevel<double>& D = m->d64.lv[L];
  for (int t = 0; t < m->host.n_macro; ++t)
    if (m->fault_set[t]) HHG_CUDA(memset16(D.u + (size_t)t * D.block, D.block * sizeof(double), s));
  HHG_CUDA(set_masters_zero(D.uI, m->fault_zero_ids, m->n_fault_zero, s));
  HHG_CUDA(restore_copies(D.u, D.uI, m->fault_restore_off, m->fault_restore_master, m->n_fault_restore, s));
  return HHG_OK;
}

// LR (n_global = 0): the Omega_F cycles on s.  DD: the Omega_F cycles on the
// mesh's high-priority stream, forked from s, and the Omega_I cycles on s;
// the block scheduler serves the small local kernels first, so Omega_F runs
// ahead (the superman of §4.1) while Omega_I fills the rest of the GPU.
int recover(hhg_mesh* m, int n_local, int n_global, bool mixed, int pre, int post, double cg_rtol, int cg_maxit,
            double* t_local, double* t_global, cudaStream_t s) {
  const bool timed = t_local || t_global;
  CallEvents ev;
  if (timed) HHG_CUDA(ev.create(4));
  cudaEvent_t a0 = ev.e[0], a1 = ev.e[1], b0 = ev.e[2], b1 = ev.e[3];
  cudaStream_t ls = s;
  if (n_global > 0) {
    ls = m->side;
    HHG_CUDA(cudaEventRecord(m->ev_fork, s));
    HHG_CUDA(cudaStreamWaitEvent(ls, m->ev_fork, 0));
  }
  if (timed) HHG_CUDA(cudaEventRecord(a0, ls));
  HHG_TRY(local_cycles(m, n_local, mixed, pre, post, cg_rtol, cg_maxit, ls));
  if (timed) HHG_CUDA(cudaEventRecord(a1, ls));
  if (n_global > 0) {
    if (timed) HHG_CUDA(cudaEventRecord(b0, s));
    for (int c = 0; c < n_global; ++c) HHG_TRY(cycle(m, m->healthy, mixed, pre, post, cg_rtol, cg_maxit, s));
    if (timed) HHG_CUDA(cudaEventRecord(b1, s));
    HHG_CUDA(cudaEventRecord(m->ev_join, ls));
    HHG_CUDA(cudaStreamWaitEvent(s, m->ev_join, 0));
  }
  if (timed) {
    HHG_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    HHG_CUDA(cudaEventElapsedTime(&ms, a0, a1));
    if (t_local) *t_local = ms * 1e-3;
    if (t_global) {
      *t_global = 0.0;
      if (n_global > 0) {
        HHG_CUDA(cudaEventElapsedTime(&ms, b0, b1));
        *t_global = ms * 1e-3;
      }
    }
  }
  return HHG_OK;
}

// Dirichlet-Neumann recovery (§4.3, Algorithm 2).  Omega_I (kind 3) frees
// every node with a healthy copy, Gamma included, under A_I; Omega_F (kind 1)
// is the Dirichlet problem of the lost nodes.  Gamma is the set of free
// kind-3 interface nodes that also have a faulty copy.
int setup_dn(hhg_mesh* m, const std::vector<unsigned char>& set) {
  HHG_TRY(setup_fault(m, set));
  if (m->has_dn && set == m->dn_set) return HHG_OK;
  HostProblem hd;
  try {
    build_any_problem(m->host, 3, set, hd);
  } catch (const std::exception& e) {
    return fail(HHG_ERR_ARG, std::string("fault set: ") + e.what());
  }
  const size_t nI = (size_t)std::max(1, m->host.lv.back().n_if);
  for (int b = 0; b < 2; ++b)       // the snapshots live as long as the mesh
    if (!m->dn_snap[b]) HHG_TRY(dalloc(m, &m->dn_snap[b], nI));
  release(m, m->dn_allocs);
  Collect keep(m, m->dn_allocs);
  m->dn = DevProblem();
  HHG_TRY(upload_problem(m, hd, m->dn));
  const int L = (int)m->host.lv.size() - 1;
  const HostLevel& H = m->host.lv[L];
  std::vector<int> gamma;
  std::vector<int64_t> off;
  std::vector<int> mst;
  for (int n : hd.lv[L].free_if) {
    bool any_f = false;
    for (int c = H.if_cptr[n]; c < H.if_cptr[n + 1]; ++c) {
      const Copy& cp = H.if_copy[c];
      if (!set[cp.macro]) continue;
      any_f = true;
      off.push_back((int64_t)cp.macro * H.block + lidx(H.SL.data(), H.N, cp.i, cp.j, cp.k));
      mst.push_back(n);
    }
    if (any_f) gamma.push_back(n);
  }
  HHG_TRY(upload(m, &m->dn_gamma, gamma));
  m->n_dn_gamma = (int)gamma.size();
  HHG_TRY(upload(m, &m->dn_off, off));
  HHG_TRY(upload(m, &m->dn_master, mst));
  m->n_dn_copy = (int)off.size();
  HHG_TRY(dalloc(m, &m->dn.fI_top, nI));
  if (!m->ev_dn_e) {
    HHG_CUDA(cudaEventCreateWithFlags(&m->ev_dn_e, cudaEventDisableTiming));
    for (int b = 0; b < 2; ++b) HHG_CUDA(cudaEventCreateWithFlags(&m->ev_dn_r[b], cudaEventDisableTiming));
  }
  m->dn_set = set;
  m->has_dn = true;
  return HHG_OK;
}

// n_global cycles on Omega_I; before cycle j, block j of Omega_F cycles
// (ceil(j eta) - ceil((j - 1) eta) of them) starts on the side stream from the
// Gamma values left by Omega_I cycle j - 1 (the copies inside the faulty
// blocks are the Dirichlet data of Omega_F, rewritten from a snapshot of the
// masters), so Omega_F block j runs concurrently with Omega_I cycle j.  The
// healthy side keeps, as the right-hand side of its Gamma rows, the flux
// (A_I u)_Gamma of the iterate at the time of the fault.  Returns the number
// of Omega_F cycles in *n_f.
int recover_dn(hhg_mesh* m, int n_global, double eta, bool mixed, int pre, int post, double cg_rtol, int cg_maxit,
               int* n_f, double* t_local, double* t_global, cudaStream_t s) {
  const int L = (int)m->host.lv.size() - 1;
  DevLevel<double>& D = m->d64.lv[L];
  const size_t nI = (size_t)std::max(1, D.n_if) * sizeof(double);
  const bool timed = t_local || t_global;
  CallEvents ev;
  if (timed) HHG_CUDA(ev.create(4));
  cudaEvent_t a0 = ev.e[0], a1 = ev.e[1], b0 = ev.e[2], b1 = ev.e[3];
  HHG_CUDA(cudaMemcpyAsync(m->dn.fI_top, D.fI, nI, cudaMemcpyDeviceToDevice, s));
  HHG_CUDA(apply_if_nodes(plargs(m, m->dn, L), D.u, D.uI, D.W, m->host.seven_point, m->dn_gamma, m->n_dn_gamma,
                          m->dn.fI_top, s));
  HHG_CUDA(cudaEventRecord(m->ev_dn_e, s));
  if (timed) HHG_CUDA(cudaEventRecord(b0, s));
  int total = 0;
  for (int j = 1; j <= n_global; ++j) {
    const int cyc = (int)std::ceil(j * eta) - (int)std::ceil((j - 1) * eta);
    // Omega_F, block j: after Omega_I cycle j - 1 and its snapshot
    HHG_CUDA(cudaStreamWaitEvent(m->side, m->ev_dn_e, 0));
    if (j == 1 && timed) HHG_CUDA(cudaEventRecord(a0, m->side));
    if (j >= 2)
      HHG_CUDA(restore_copies(D.u, m->dn_snap[(j - 1) & 1], m->dn_off, m->dn_master, m->n_dn_copy, m->side));
    HHG_CUDA(cudaEventRecord(m->ev_dn_r[j & 1], m->side));
    HHG_TRY(local_cycles(m, cyc, mixed, pre, post, cg_rtol, cg_maxit, m->side));
    total += cyc;
    // Omega_I, cycle j; its snapshot overwrites the one block j - 1 read
    HHG_TRY(cycle(m, m->dn, mixed, pre, post, cg_rtol, cg_maxit, s));
    if (j >= 3) HHG_CUDA(cudaStreamWaitEvent(s, m->ev_dn_r[(j - 1) & 1], 0));
    HHG_CUDA(copy_listed(D.uI, m->dn_snap[j & 1], m->dn_gamma, m->n_dn_gamma, s));
    HHG_CUDA(cudaEventRecord(m->ev_dn_e, s));
  }
  if (timed) {
    HHG_CUDA(cudaEventRecord(b1, s));
    HHG_CUDA(cudaEventRecord(a1, m->side));
  }
  // join; the copies of Gamma inside the faulty blocks take the final values
  HHG_CUDA(cudaEventRecord(m->ev_join, m->side));
  HHG_CUDA(cudaStreamWaitEvent(s, m->ev_join, 0));
  HHG_CUDA(restore_copies(D.u, D.uI, m->dn_off, m->dn_master, m->n_dn_copy, s));
  if (n_f) *n_f = total;
  if (timed) {
    HHG_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    if (t_local) {
      *t_local = 0.0;
      if (n_global > 0) {
        HHG_CUDA(cudaEventElapsedTime(&ms, a0, a1));
        *t_local = ms * 1e-3;
      }
    }
    if (t_global) {
      HHG_CUDA(cudaEventElapsedTime(&ms, b0, b1));
      *t_global = ms * 1e-3;
    }
  }
  return HHG_OK;
}

// Stencils of all levels, the coarse CG matrices and the pre-divided finest
// level arrays for new coefficients.
int update_coefficients(hhg_mesh* m, const double* coeff) {
  try {
    set_coefficients(m->host, coeff);
  } catch (const std::exception& e) {
    return fail(HHG_ERR_ARG, std::string("coefficients: ") + e.what());
  }
  const int nl = (int)m->host.lv.size();
  for (int l = 0; l < nl; ++l) {
    const HostLevel& H = m->host.lv[l];
    std::vector<double> winv(m->host.n_macro);
    for (int t = 0; t < m->host.n_macro; ++t) winv[t] = 1.0 / H.W[(size_t)t * 16 * NDIR];
    HHG_CUDA(cudaMemcpy(m->d64.lv[l].W, H.W.data(), H.W.size() * sizeof(double), cudaMemcpyHostToDevice));
    HHG_CUDA(cudaMemcpy(m->d64.Winv[l], winv.data(), winv.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (m->precision == 32) {
      std::vector<float> w32(H.W.begin(), H.W.end()), wi32(winv.begin(), winv.end());
      HHG_CUDA(cudaMemcpy(m->d32.lv[l].W, w32.data(), w32.size() * sizeof(float), cudaMemcpyHostToDevice));
      HHG_CUDA(cudaMemcpy(m->d32.Winv[l], wi32.data(), wi32.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
  }
  HHG_TRY(refresh_scaled(m));
  // the Neumann-side problem of DN recovery (operator A_I, coarse matrix,
  // interface flux) is rebuilt from the new coefficients on its next use
  m->has_dn = false;
  std::vector<DevProblem*> probs = {&m->global};
  if (m->has_fault) {
    probs.push_back(&m->faulty);
    probs.push_back(&m->healthy);
  }
  for (DevProblem* d : probs) {
    HostProblem h;
    h.kind = d->kind;
    h.act = d->act_host;
    h.macro_active = d->macro_active_host;
    h.lv.resize(1);
    h.lv[0].free_if = d->free0_host;
    assemble_coarse(m->host, h);
    if ((int64_t)h.val.size() != d->nnz || h.n_cg != d->n_cg)
      return fail(HHG_ERR_STATE, "coarse system changed shape");
    if (!h.val.empty())
      HHG_CUDA(cudaMemcpy(d->val, h.val.data(), h.val.size() * sizeof(double), cudaMemcpyHostToDevice));
    // the interface tables hold summed stencil weights (kinds 0-2 use the
    // level's own copy lists)
    for (size_t l = 1; l < d->lv.size() && l < d->free_host.size(); ++l)
      if (d->lv[l].tnb)
        HHG_TRY(upload_if_tables(m, d->lv[l], (int)l, d->kind, d->free_host[l], std::vector<int>(),
                                 std::vector<Copy>()));
  }
  return HHG_OK;
}

// Candidate shapes of the interior tiles: (nodes of one colour per tile in its
// first slice, consecutive slices per tile).
const int TUNE_CAND[][2] = {{256, 4}, {512, 8}, {1024, 8}, {2048, 16}};
constexpr int N_TUNE_CAND = 4;

// Flat Gauss-Seidel on level l (7-point meshes of the cube family): build and
// upload its item tables (FP64, and FP32 on precision-32 meshes) when
// switching it on, free them when switching it off.
// Whether the flat kernels can run level l: 4 .. 1024 intervals per macro edge
// (the packed items hold j, k and the group in 10 bits each) and every item
// count times the macros below 2^31 (the kernels' thread indices are 32-bit;
// the largest counts are the slots and the FP64 items of all four colours).
bool flat_fits(const hhg_mesh* m, int l) {
  const int N = m->host.lv[l].N;
  if (N > 1024 || N < 4) return false;
  int64_t items = 0, slots = 0;
  for (int k = 1; k <= N - 3; ++k)
    for (int j = 1; j <= N - 2 - k; ++j) {
      const int L = N - 1 - j - k;
      slots += (L >> 2) + 1;
      for (int c = 0; c < 4; ++c) {
        const int ic = (c - 2 * j - 3 * k) & 3, mlo = ic == 0;
        const int n = L >= ic ? ((L - ic) >> 2) - mlo + 1 : 0;
        items += n > 0 ? (mlo + n - 1) / 2 + 1 : 0;
      }
    }
  const int64_t limit = (int64_t)INT32_MAX - 1024;
  return std::max(items, slots) * m->host.n_macro <= limit;
}

int set_flat(hhg_mesh* m, int l, bool on) {
  DevLevelTables& tb = m->tab[l];
  const HostLevel& H = m->host.lv[l];
  if (!on) {
    std::vector<void*> unused;
    for (void* q : {(void*)tb.gs_items64, (void*)tb.gs_items32, (void*)tb.slot_items})
      if (q) unused.push_back(q);
    release(m, unused);
    tb.gs_items64 = tb.gs_items32 = nullptr;
    tb.slot_items = nullptr;
    tb.n_slots = 0;
    for (int c = 0; c < 5; ++c) tb.gs_off64[c] = tb.gs_off32[c] = 0;
    tb.gs_flat = 0;
    return HHG_OK;
  }
  if (!flat_fits(m, l))
    return fail(HHG_ERR_ARG, "the flat kernels need 4 .. 1024 intervals per macro edge and fewer than 2^31 "
                             "items per launch");
  for (int vw : {2, 4}) {
    if (vw == 4 && m->precision != 32) continue;
    uint32_t*& dst = vw == 2 ? tb.gs_items64 : tb.gs_items32;
    if (dst) continue;
    std::vector<uint32_t> items;
    int off[5];
    build_gs_items(H.N, vw, items, off);
    HHG_TRY(upload(m, &dst, items));
    for (int c = 0; c < 5; ++c) (vw == 2 ? tb.gs_off64 : tb.gs_off32)[c] = off[c];
  }
  if (!tb.slot_items) {
    std::vector<uint32_t> slots;
    build_slot_items(H.N, slots);
    HHG_TRY(upload(m, &tb.slot_items, slots));
    tb.n_slots = (int)slots.size();
  }
  tb.gs_flat = 1;
  return HHG_OK;
}

// Device time of `reps` Gauss-Seidel steps of the global problem on level l
// in precision T (after one warm-up step).
template <class T>
int time_smooth(hhg_mesh* m, Prec<T>& P, int l, int reps, cudaStream_t s, cudaEvent_t a, cudaEvent_t b, float* ms) {
  HHG_TRY(smooth<T>(m, P, m->global, l, 1, s, false));
  HHG_CUDA(cudaEventRecord(a, s));
  HHG_TRY(smooth<T>(m, P, m->global, l, reps, s, false));
  HHG_CUDA(cudaEventRecord(b, s));
  HHG_CUDA(cudaEventSynchronize(b));
  HHG_CUDA(cudaEventElapsedTime(ms, a, b));
  return HHG_OK;
}

int tune_level(hhg_mesh* m, int l, int reps, cudaStream_t s, int* best_out) {
  const HostLevel& H = m->host.lv[l];
  DevLevelTables& tb = m->tab[l];
  HHG_TRY(set_flat(m, l, false));   // the tile candidates are timed with the tile kernel
  Tile* const before = tb.tiles_int;
  double best_ms = 1e30;
  int best = -1;
  std::vector<Tile*> dev(N_TUNE_CAND, nullptr);
  std::vector<int> ndev(N_TUNE_CAND, 0);
  CallEvents ev;
  HHG_CUDA(ev.create(2));
  cudaEvent_t a = ev.e[0], b = ev.e[1];
  for (int c = 0; c < N_TUNE_CAND; ++c) {
    std::vector<Tile> tiles;
    build_pair_tiles(H.N, tiles, TUNE_CAND[c][0], TUNE_CAND[c][1]);
    HHG_TRY(upload(m, &dev[c], tiles));
    ndev[c] = (int)tiles.size();
    tb.tiles_int = dev[c];
    tb.n_tiles_int = ndev[c];
    // both precisions' sweeps use the level's tiles: the FP64 one always,
    // the FP32 one on precision-32 meshes
    float ms = 0.f, ms32 = 0.f;
    HHG_TRY(time_smooth<double>(m, m->d64, l, reps, s, a, b, &ms));
    if (m->precision == 32) HHG_TRY(time_smooth<float>(m, m->d32, l, reps, s, a, b, &ms32));
    ms += ms32;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  tb.tiles_int = dev[best];
  tb.n_tiles_int = ndev[best];
  *best_out = best;
  // the flat Gauss-Seidel kernel against the best tile shape (7-point
  // levels); the level's other kernels keep the tiles either way
  if (m->host.seven_point && flat_fits(m, l)) {
    HHG_TRY(set_flat(m, l, true));
    float ms = 0.f, ms32 = 0.f;
    HHG_TRY(time_smooth<double>(m, m->d64, l, reps, s, a, b, &ms));
    if (m->precision == 32) HHG_TRY(time_smooth<float>(m, m->d32, l, reps, s, a, b, &ms32));
    if (ms + ms32 < best_ms) *best_out = best + N_TUNE_CAND;
    else HHG_TRY(set_flat(m, l, false));
  }
  // the other candidates' tiles and the level's previous tiles are unused now
  std::vector<void*> unused;
  for (int c = 0; c < N_TUNE_CAND; ++c)
    if (c != best && dev[c]) unused.push_back(dev[c]);
  if (before && before != dev[best]) unused.push_back(before);
  release(m, unused);
  return HHG_OK;
}

int capture_task(hhg_mesh* m, int cycles, bool recovery, bool mixed, cudaStream_t s) {
  if (recovery) {
    HHG_TRY(inject(m, s));
    for (int c = 0; c < cycles; ++c) HHG_TRY(cycle(m, m->faulty, mixed, 3, 3, 1e-12, 1000, s));
  } else {
    for (int c = 0; c < cycles; ++c) HHG_TRY(cycle(m, m->global, mixed, 3, 3, 1e-12, 1000, s));
  }
  return HHG_OK;
}

// The operations of one task as the persistent executor runs them: while
// recording, the launchers append the launch they would make (its kind,
// arguments and number of work units) to `out` and launch nothing.  The
// profiling hooks are off meanwhile (they would record events).
int record_task(hhg_mesh* m, int cycles, bool recovery, bool mixed, std::vector<BOp>& out) {
  const bool prof = m->prof_on, bd = m->bd_on;
  m->prof_on = m->bd_on = false;
  record_ops(&out);
  const int rc = capture_task(m, cycles, recovery, mixed, nullptr);
  record_ops(nullptr);
  m->prof_on = prof;
  m->bd_on = bd;
  return rc;
}

void free_persistent(hhg_batch* b) {
  for (void* q : {(void*)b->d_ops, (void*)b->d_op_off, (void*)b->d_state, (void*)b->d_ns, (void*)b->d_err,
                  (void*)b->d_order, (void*)b->d_seg})
    if (q) cudaFree(q);
  b->d_order = nullptr;
  b->d_seg = nullptr;
  b->d_ops = nullptr;
  b->d_op_off = nullptr;
  b->d_state = nullptr;
  b->d_ns = nullptr;
  b->d_err = nullptr;
}

// Priority classes of the persistent executor: the tasks ordered by
// decreasing priority (ties in task order), one class per distinct value.
int upload_priorities(hhg_batch* b, const std::vector<int>& prio) {
  const int n = (int)prio.size();
  std::vector<int> order(n), seg;
  for (int t = 0; t < n; ++t) order[t] = t;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return prio[a] > prio[c]; });
  for (int q = 0; q < n; ++q)
    if (q == 0 || prio[order[q]] != prio[order[q - 1]]) seg.push_back(q);
  seg.push_back(n);
  b->n_seg = (int)seg.size() - 1;
  if (n > 0) HHG_CUDA(cudaMemcpy(b->d_order, order.data(), n * sizeof(int), cudaMemcpyHostToDevice));
  HHG_CUDA(cudaMemcpy(b->d_seg, seg.data(), seg.size() * sizeof(int), cudaMemcpyHostToDevice));
  return HHG_OK;
}

// Records every task's program and uploads it with the scheduler's counters.
int setup_persistent(hhg_batch* b, size_t n_rec) {
  b->op_off.assign(1, 0);
  for (size_t t = 0; t < b->tasks.size(); ++t) {
    HHG_TRY(record_task(b->tasks[t].mesh, b->tasks[t].cycles, t < n_rec, b->mixed, b->ops));
    b->op_off.push_back((int)b->ops.size());
  }
  const size_t n = b->tasks.size(), n_ops = b->ops.size();
  b->state_bytes = (n + 2 * n_ops + 1) * sizeof(int);
  auto alloc = [&](void** q, size_t bytes) {
    const cudaError_t e = cudaMalloc(q, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) cudaGetLastError();
    return e;
  };
  if (alloc((void**)&b->d_ops, n_ops * sizeof(BOp)) != cudaSuccess ||
      alloc((void**)&b->d_op_off, (n + 1) * sizeof(int)) != cudaSuccess ||
      alloc((void**)&b->d_state, b->state_bytes) != cudaSuccess ||
      alloc((void**)&b->d_ns, (n + 1) * sizeof(unsigned long long)) != cudaSuccess ||
      alloc((void**)&b->d_err, sizeof(int)) != cudaSuccess || alloc((void**)&b->d_order, n * sizeof(int)) != cudaSuccess ||
      alloc((void**)&b->d_seg, (n + 1) * sizeof(int)) != cudaSuccess)
    return fail(HHG_ERR_OOM, "allocation of the persistent executor's program failed");
  if (n_ops) HHG_CUDA(cudaMemcpy(b->d_ops, b->ops.data(), n_ops * sizeof(BOp), cudaMemcpyHostToDevice));
  HHG_CUDA(cudaMemcpy(b->d_op_off, b->op_off.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice));
  HHG_CUDA(cudaMemset(b->d_err, 0, sizeof(int)));
  if (!b->tasks.empty()) b->wait_limit = b->tasks[0].mesh->global.wait_limit;
  return upload_priorities(b, std::vector<int>(n, 0));
}

// ---------------------------------------------------------------------------
// Allocation-free V-cycle: the coarse-grid CG keeps its work vectors (x, r, p,
// A p) in this file-scope static device array instead of the mesh's own
// scratch.  Every GPU that loads the library holds the array until the
// process exits.
// ---------------------------------------------------------------------------
constexpr int NOALLOC_MAX_COARSE = 16384;
static __device__ __align__(256) double g_noalloc_cg_scratch[4 * NOALLOC_MAX_COARSE];
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_cg_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the static array on the current device, looked up once
// per device (with that device current).
int noalloc_scratch(double** out) {
  int dev = 0;
  HHG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(HHG_ERR_ARG, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_cg_ptr[dev]) {
    void* p = nullptr;
    HHG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_cg_scratch));
    g_noalloc_cg_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_cg_ptr[dev];
  return HHG_OK;
}

}  // namespace

extern "C" {

int hhg_vcycle_noalloc(hhg_mesh* m, int pre, int post, void* stream) {
  if (!m || pre < 0 || post < 0) return fail(HHG_ERR_ARG, "invalid argument");
  HHG_TRY(check_device(m));
  if (m->global.n_cg > NOALLOC_MAX_COARSE)
    return fail(HHG_ERR_ARG, "coarse problem has " + std::to_string(m->global.n_cg) +
                                 " unknowns; the allocation-free V-cycle holds at most " +
                                 std::to_string(NOALLOC_MAX_COARSE));
  // the mesh's device is current (checked above), so this is its copy
  double* scratch = nullptr;
  HHG_TRY(noalloc_scratch(&scratch));
  // the ordinary cycle with the coarse CG's work vectors in the static array
  // and without the profiling hook (which creates events)
  CycleOpts co;
  co.cg_work = scratch;
  co.profile = false;
  return vcycle_T<double>(m, m->d64, m->global, pre, post, 1e-12, 1000, (cudaStream_t)stream, co);
}

int hhg_last_error(char* buf, size_t len) {
  if (buf && len > 0) {
    size_t n = std::min(len - 1, g_err.size());
    std::memcpy(buf, g_err.data(), n);
    buf[n] = '\0';
  }
  return g_err_code;
}

// Device side of a new mesh (after its host mesh is built): level tables,
// arrays of both precisions, the global problem, streams and events.  On
// failure everything allocated is freed.
int setup_device(hhg_mesh* m) {
  int rc = HHG_OK;
  auto cleanup = [&](int code) {
    free_all(m);
    return code;
  };
  if (cudaGetDevice(&m->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(HHG_ERR_CUDA, "no CUDA device");
  }
  const int nl = (int)m->host.lv.size();
  m->tab.assign(nl, DevLevelTables());
  for (int l = 0; l < nl && rc == HHG_OK; ++l) {
    const HostLevel& H = m->host.lv[l];
    DevLevelTables& t = m->tab[l];
    if ((rc = upload(m, &t.SL, H.SL)) != HHG_OK) break;
    if ((rc = upload(m, &t.if_gid, H.if_gid)) != HHG_OK) break;
    if ((rc = upload(m, &t.if_cptr, H.if_cptr)) != HHG_OK) break;
    if ((rc = upload(m, &t.if_copy, H.if_copy)) != HHG_OK) break;
    {
      std::vector<uint32_t> off;
      if (copy_offsets(m->host, l, H.if_copy, off) && (rc = upload(m, &t.cp_off, off)) != HHG_OK) break;
    }
    if ((rc = upload(m, &t.tiles_int, H.tiles_int)) != HHG_OK) break;
    if ((rc = upload(m, &t.tiles_all, H.tiles_all)) != HHG_OK) break;
    if ((rc = upload(m, &t.tiles_stream, H.tiles_stream)) != HHG_OK) break;
    if ((rc = upload(m, &t.tiles_stream32, H.tiles_stream32)) != HHG_OK) break;
    t.n_tiles_int = (int)H.tiles_int.size();
    t.n_tiles_all = (int)H.tiles_all.size();
    t.n_tiles_stream = (int)H.tiles_stream.size();
    t.n_tiles_stream32 = (int)H.tiles_stream32.size();
  }
  if (rc == HHG_OK) rc = upload(m, &m->geo, m->host.geo);
  if (rc == HHG_OK) rc = dalloc(m, &m->dev_err, 4);
  if (rc == HHG_OK && cudaMemset(m->dev_err, 0, 4 * sizeof(int)) != cudaSuccess)
    rc = fail(HHG_ERR_CUDA, "cudaMemset failed");
  if (rc == HHG_OK) rc = alloc_levels<double>(m, m->d64, true);
  if (rc == HHG_OK) rc = alloc_scaled(m);
  if (rc == HHG_OK && m->precision == 32) rc = alloc_levels<float>(m, m->d32, true);
  if (rc == HHG_OK) {
    HostProblem hg;
    try {
      if (m->host.general) build_general_problem(m->host, 0, std::vector<unsigned char>(m->host.n_macro, 0), hg);
      else build_problem(m->host, 0, std::vector<unsigned char>(m->host.n_macro, 0), hg);
    } catch (const std::exception& e) {
      rc = fail(HHG_ERR_ARG, std::string("problem: ") + e.what());
    }
    if (rc == HHG_OK) rc = upload_problem(m, hg, m->global);
  }
  if (rc == HHG_OK && m->host.general) {
    const HostLevel& H = m->host.lv.back();
    std::vector<int64_t> off;
    std::vector<int> master;
    for (int n = 0; n < H.n_if; ++n)
      for (int c = H.if_cptr[n]; c < H.if_cptr[n + 1]; ++c) {
        const Copy& cp = H.if_copy[c];
        off.push_back((int64_t)cp.macro * H.block + lidx(H.SL.data(), H.N, cp.i, cp.j, cp.k));
        master.push_back(n);
      }
    m->n_gen_copy = (int)off.size();
    rc = upload(m, &m->gen_copy_off, off);
    if (rc == HHG_OK) rc = upload(m, &m->gen_copy_master, master);
  }
  if (rc != HHG_OK) return cleanup(rc);
  // the recovery's Omega_F side (and the capture of its cycle) run at the
  // device's highest stream priority
  int prio_lo = 0, prio_hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
    cudaGetLastError();
    prio_hi = 0;
  }
  m->prio_hi = prio_hi;
  if (cudaStreamCreateWithPriority(&m->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaStreamCreateWithPriority(&m->cap, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&m->host_scalar, sizeof(double) * 8) != cudaSuccess ||
      cudaMallocHost(&m->host_flag, sizeof(int) * 4) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(HHG_ERR_CUDA, "stream / event creation failed"));
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return cleanup(fail(HHG_ERR_CUDA, "device error during setup"));
  return HHG_OK;
}

int hhg_mesh_create(const hhg_mesh_desc* desc, hhg_mesh** out) {
  if (!desc || !out) return fail(HHG_ERR_ARG, "null argument");
  *out = nullptr;
  const int r0 = desc->coarsest > 0 ? desc->coarsest : 2;
  for (int a = 0; a < 3; ++a)
    if (desc->subcubes[a] < 1 || desc->subcubes[a] > 64) return fail(HHG_ERR_ARG, "subcubes must be in [1, 64]");
  if (r0 < 2) return fail(HHG_ERR_ARG, "coarsest refinement must be >= 2");
  if (desc->levels <= r0 || desc->levels > 10) return fail(HHG_ERR_ARG, "levels must be in (coarsest, 10]");
  if (desc->precision != 64 && desc->precision != 32) return fail(HHG_ERR_ARG, "precision must be 64 or 32");
  if (desc->coeff)
    for (int t = 0; t < 6 * desc->subcubes[0] * desc->subcubes[1] * desc->subcubes[2]; ++t)
      if (!(desc->coeff[t] > 0.0)) return fail(HHG_ERR_ARG, "coefficients must be positive");
  if (desc->affine && desc->vertex_pos) return fail(HHG_ERR_ARG, "give affine or vertex_pos, not both");
  std::unique_ptr<hhg_mesh> m(new (std::nothrow) hhg_mesh());
  if (!m) return fail(HHG_ERR_OOM, "host allocation failed");
  try {
    build_host_mesh(m->host, desc->subcubes, desc->levels, r0, desc->coeff, desc->affine, desc->vertex_pos);
  } catch (const std::bad_alloc&) {
    return fail(HHG_ERR_OOM, "host allocation failed while building the mesh");
  } catch (const std::exception& e) {
    return fail(HHG_ERR_ARG, std::string("mesh: ") + e.what());
  }
  m->precision = desc->precision;
  HHG_TRY(setup_device(m.get()));
  *out = m.release();
  return HHG_OK;
}

int hhg_mesh_create_general(const hhg_general_desc* desc, hhg_mesh** out) {
  if (!desc || !out) return fail(HHG_ERR_ARG, "null argument");
  *out = nullptr;
  const int r0 = desc->coarsest > 0 ? desc->coarsest : 2;
  if (!desc->vertices || !desc->macros || desc->n_vertices < 4 || desc->n_macros < 1)
    return fail(HHG_ERR_ARG, "need vertices and macros");
  if (r0 < 2) return fail(HHG_ERR_ARG, "coarsest refinement must be >= 2");
  if (desc->levels <= r0 || desc->levels > 10) return fail(HHG_ERR_ARG, "levels must be in (coarsest, 10]");
  if (desc->precision != 64 && desc->precision != 32) return fail(HHG_ERR_ARG, "precision must be 64 or 32");
  if (desc->coeff)
    for (int t = 0; t < desc->n_macros; ++t)
      if (!(desc->coeff[t] > 0.0)) return fail(HHG_ERR_ARG, "coefficients must be positive");
  std::unique_ptr<hhg_mesh> m(new (std::nothrow) hhg_mesh());
  if (!m) return fail(HHG_ERR_OOM, "host allocation failed");
  try {
    build_general_mesh(m->host, desc->vertices, desc->n_vertices, desc->macros, desc->n_macros, desc->levels, r0,
                       desc->coeff);
  } catch (const std::bad_alloc&) {
    return fail(HHG_ERR_OOM, "host allocation failed while building the mesh");
  } catch (const std::exception& e) {
    return fail(HHG_ERR_ARG, std::string("mesh: ") + e.what());
  }
  m->precision = desc->precision;
  HHG_TRY(setup_device(m.get()));
  *out = m.release();
  return HHG_OK;
}

int hhg_mesh_destroy(hhg_mesh* m) {
  if (!m) return HHG_OK;
  // the mesh's device is made current for the release and the caller's
  // current device is put back afterwards
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    cur = -1;
  }
  if (cur != m->device) cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  free_all(m);
  if (m->local_exec) cudaGraphExecDestroy(m->local_exec);
  if (m->side) cudaStreamDestroy(m->side);
  if (m->cap) cudaStreamDestroy(m->cap);
  if (m->ev_fork) cudaEventDestroy(m->ev_fork);
  if (m->ev_join) cudaEventDestroy(m->ev_join);
  if (m->ev_dn_e) cudaEventDestroy(m->ev_dn_e);
  for (int b = 0; b < 2; ++b)
    if (m->ev_dn_r[b]) cudaEventDestroy(m->ev_dn_r[b]);
  if (m->host_scalar) cudaFreeHost(m->host_scalar);
  if (m->host_flag) cudaFreeHost(m->host_flag);
  for (cudaEvent_t ev : m->prof_ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : m->bd_ev) cudaEventDestroy(ev);
  const int dev = m->device;
  delete m;
  if (cur >= 0 && cur != dev) cudaSetDevice(cur);
  return HHG_OK;
}

int hhg_mesh_info(const hhg_mesh* m, int64_t* n_nodes, int64_t* n_dof, int* n_macro) {
  if (!m) return fail(HHG_ERR_ARG, "null mesh");
  if (n_nodes) *n_nodes = global_nodes(m);
  if (n_dof) *n_dof = global_dof(m);
  if (n_macro) *n_macro = m->host.n_macro;
  return HHG_OK;
}

int hhg_mesh_bytes(const hhg_mesh* m, int64_t* bytes) {
  if (!m || !bytes) return fail(HHG_ERR_ARG, "null argument");
  *bytes = m->bytes;
  return HHG_OK;
}

int hhg_set_problem(hhg_mesh* m, const double* f, const double* u0, void* stream) {
  if (!m) return fail(HHG_ERR_ARG, "null mesh");
  HHG_TRY(check_device(m));
  cudaStream_t s = (cudaStream_t)stream;
  const int L = (int)m->host.lv.size() - 1;
  const LevelArgs a = largs(m, L);
  DevLevel<double>& D = m->d64.lv[L];
  int rc;
  const bool gen = m->host.general;
  const int64_t n_if = m->host.lv[L].n_if;
  if (f) {
    const double* g = stage_in(m, f, s, &rc);
    if (!g) return rc;
    if (gen) HHG_CUDA(general_import_vol<double>(a, m->host.n_macro, n_if, g, D.f, s));
    else HHG_CUDA(import_vec<double>(a, m->geo, m->host.n_macro, m->host.nx, m->host.ny, g, D.f, D.fI, false, s));
    HHG_CUDA(import_masters<double>(a.if_gid, m->host.lv[L].n_if, g, D.fI, s));
    if (m->fs_top)
      HHG_CUDA(scale_blocks(D.f, m->d64.Winv[L], m->fs_top, m->host.n_macro, m->host.lv[L].block, s));
  }
  if (u0) {
    const double* g = stage_in(m, u0, s, &rc);
    if (!g) return rc;
    if (gen) {
      HHG_CUDA(general_import_vol<double>(a, m->host.n_macro, n_if, g, D.u, s));
      HHG_CUDA(import_masters<double>(a.if_gid, m->host.lv[L].n_if, g, D.uI, s));
      HHG_CUDA(restore_copies(D.u, D.uI, m->gen_copy_off, m->gen_copy_master, m->n_gen_copy, s));
    } else {
      HHG_CUDA(import_vec<double>(a, m->geo, m->host.n_macro, m->host.nx, m->host.ny, g, D.u, D.uI, true, s));
      HHG_CUDA(import_masters<double>(a.if_gid, m->host.lv[L].n_if, g, D.uI, s));
    }
  }
  return HHG_OK;
}

int hhg_get_solution(hhg_mesh* m, double* u, void* stream) {
  if (!m || !u) return fail(HHG_ERR_ARG, "null argument");
  HHG_TRY(check_device(m));
  cudaStream_t s = (cudaStream_t)stream;
  const int L = (int)m->host.lv.size() - 1;
  const LevelArgs a = largs(m, L);
  DevLevel<double>& D = m->d64.lv[L];
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, u);
  if (e != cudaSuccess) cudaGetLastError();
  const bool dev = e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
  double* g = u;
  const int64_t n = global_nodes(m);
  if (!dev) {
    if (!m->staging) HHG_TRY(dalloc(m, &m->staging, (size_t)n));
    g = m->staging;
  }
  if (m->host.general)
    HHG_CUDA(general_export_vol<double>(a, m->host.n_macro, m->host.lv[L].n_if, D.u, g, s));
  else
    HHG_CUDA(export_vec<double>(a, m->geo, m->host.n_macro, m->host.nx, m->host.ny, D.u, D.uI, g, s));
  HHG_CUDA(export_masters<double>(a.if_gid, m->host.lv[L].n_if, D.uI, g, s));
  if (!dev) {
    HHG_CUDA(cudaMemcpyAsync(u, g, (size_t)n * sizeof(double), cudaMemcpyDefault, s));
    HHG_CUDA(cudaStreamSynchronize(s));
  }
  return HHG_OK;
}

int hhg_vcycle(hhg_mesh* m, int pre, int post, double* resid_out, void* stream) {
  if (!m || pre < 0 || post < 0) return fail(HHG_ERR_ARG, "invalid argument");
  HHG_TRY(check_device(m));
  cudaStream_t s = (cudaStream_t)stream;
  HHG_TRY(vcycle_T<double>(m, m->d64, m->global, pre, post, 1e-12, 1000, s));
  if (resid_out) HHG_TRY(resnorm(m, resid_out, s));
  return HHG_OK;
}

int hhg_residual_norm(hhg_mesh* m, double* out, void* stream) {
  if (!m || !out) return fail(HHG_ERR_ARG, "null argument");
  HHG_TRY(check_device(m));
  return resnorm(m, out, (cudaStream_t)stream);
}

int hhg_inject_fault(hhg_mesh* m, const int* ids, int n, void* stream) {
  if (!m) return fail(HHG_ERR_ARG, "null mesh");
  HHG_TRY(check_device(m));
  std::vector<unsigned char> set;
  HHG_TRY(check_ids(m, ids, n, set));
  HHG_TRY(setup_fault(m, set));
  return inject(m, (cudaStream_t)stream);
}

int hhg_recover_local(hhg_mesh* m, const int* ids, int n, int n_local, int n_global, double* seconds_local,
                      double* seconds_global, void* stream) {
  if (!m || n_local < 0 || n_global < 0) return fail(HHG_ERR_ARG, "invalid argument");
  HHG_TRY(check_device(m));
  std::vector<unsigned char> set;
  HHG_TRY(check_ids(m, ids, n, set));
  HHG_TRY(setup_fault(m, set));
  return recover(m, n_local, n_global, false, 3, 3, 1e-12, 1000, seconds_local, seconds_global,
                 (cudaStream_t)stream);
}

int hhg_recover_dn(hhg_mesh* m, const int* ids, int n, int n_global, double eta, int* n_local_run,
                   double* seconds_local, double* seconds_global, void* stream) {
  if (!m || n_global < 0 || !(eta >= 0.0)) return fail(HHG_ERR_ARG, "invalid argument");
  HHG_TRY(check_device(m));
  std::vector<unsigned char> set;
  HHG_TRY(check_ids(m, ids, n, set));
  HHG_TRY(setup_dn(m, set));
  return recover_dn(m, n_global, eta, false, 3, 3, 1e-12, 1000, n_local_run, seconds_local, seconds_global,
                    (cudaStream_t)stream);
}

int hhg_set_coefficients(hhg_mesh* m, const double* coeff, void* stream) {
  if (!m || !coeff) return fail(HHG_ERR_ARG, "null argument");
  HHG_TRY(check_device(m));
  HHG_TRY(refuse_general(m, "changing coefficients"));
  for (int t = 0; t < m->host.n_macro; ++t)
    if (!(coeff[t] > 0.0)) return fail(HHG_ERR_ARG, "coefficients must be positive");
  HHG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  // the same coefficients again (an adjoint solve after its forward solve):
  // the stencils, tables and coarse matrices already hold them
  if (!m->coeff_dirty && std::equal(coeff, coeff + m->host.n_macro, m->host.coeff.begin())) return HHG_OK;
  m->coeff_dirty = true;   // until the device holds them (a failed update is redone)
  HHG_TRY(update_coefficients(m, coeff));
  m->coeff_dirty = false;
  return HHG_OK;
}

int hhg_grad_coeff(hhg_mesh* m, const double* u, const double* lam, double* grad, void* stream) {
  if (!m || !u || !lam || !grad) return fail(HHG_ERR_ARG, "null argument");
  HHG_TRY(check_device(m));
  HHG_TRY(refuse_general(m, "the coefficient gradient"));
  cudaStream_t s = (cudaStream_t)stream;
  const int L = (int)m->host.lv.size() - 1;
  const LevelArgs a = largs(m, L);
  DevLevel<double>& D = m->d64.lv[L];
  const int n_macro = m->host.n_macro;
  if (!m->grad_partial) {
    HHG_TRY(dalloc(m, &m->grad_partial, (size_t)n_macro * std::max(1, a.n_tiles_all)));
    HHG_TRY(dalloc(m, &m->grad_out, (size_t)n_macro));
  }
  int rc;
  const double* g = stage_in(m, u, s, &rc);
  if (!g) return rc;
  HHG_CUDA(import_vec<double>(a, m->geo, n_macro, m->host.nx, m->host.ny, g, D.u, D.uI, true, s));
  HHG_CUDA(import_masters<double>(a.if_gid, m->host.lv[L].n_if, g, D.uI, s));
  const double* gl = stage_in(m, lam, s, &rc);
  if (!gl) return rc;
  HHG_CUDA(import_vec<double>(a, m->geo, n_macro, m->host.nx, m->host.ny, gl, D.r, nullptr, true, s));
  HHG_CUDA(grad_partials(a, n_macro, D.u, D.r, D.W, m->grad_partial, s));
  HHG_CUDA(reduce_per_macro(m->grad_partial, a.n_tiles_all, n_macro, m->grad_out, s));
  std::vector<double> out(n_macro);
  HHG_CUDA(cudaMemcpyAsync(out.data(), m->grad_out, n_macro * sizeof(double), cudaMemcpyDeviceToHost, s));
  HHG_CUDA(cudaStreamSynchronize(s));
  for (int t = 0; t < n_macro; ++t) grad[t] = -out[t] / m->host.coeff[t];
  return HHG_OK;
}

int hhg_autotune(hhg_mesh* m, int reps, int* chosen, void* stream) {
  if (!m || reps < 1) return fail(HHG_ERR_ARG, "invalid argument");
  HHG_TRY(check_device(m));
  HHG_TRY(refuse_general(m, "autotuning"));
  cudaStream_t s = (cudaStream_t)stream;
  const int nl = (int)m->host.lv.size();
  drop_local_graph(m);
  for (int l = 1; l < nl; ++l) {
    int best = 0;
    HHG_TRY(tune_level(m, l, reps, s, &best));
    if (chosen) chosen[l] = best;
  }
  if (chosen) chosen[0] = -1;
  return HHG_OK;
}

int hhg_batch_create(hhg_mesh* global, int global_cycles, hhg_mesh* const* meshes, const int* const* ids,
                     const int* n_ids, const int* cycles, int n_tasks, int mixed, hhg_batch** out) {
  if (!out || n_tasks < 0 || (n_tasks > 0 && (!meshes || !ids || !n_ids || !cycles)) ||
      (global && global_cycles < 0))
    return fail(HHG_ERR_ARG, "invalid argument");
  *out = nullptr;
  std::unique_ptr<hhg_batch> b(new (std::nothrow) hhg_batch());
  if (!b) return fail(HHG_ERR_OOM, "host allocation failed");
  b->mixed = mixed != 0;
  if (global) HHG_TRY(refuse_general(global, "batched recovery"));
  if (global) HHG_TRY(check_device(global));
  for (int t = 0; t < n_tasks; ++t) {
    hhg_mesh* m = meshes[t];
    if (!m || cycles[t] < 0) return fail(HHG_ERR_ARG, "invalid task");
    HHG_TRY(check_device(m));
    HHG_TRY(refuse_general(m, "batched recovery"));
    if (b->mixed && m->precision != 32) return fail(HHG_ERR_STATE, "mixed precision needs precision-32 meshes");
    for (int q = 0; q < t; ++q)
      if (meshes[q] == m) return fail(HHG_ERR_ARG, "a mesh may appear in one task only");
    std::vector<unsigned char> set;
    HHG_TRY(check_ids(m, ids[t], n_ids[t], set));
    HHG_TRY(setup_fault(m, set));
    b->tasks.push_back({m, cycles[t], nullptr, nullptr, nullptr});
  }
  if (global) {
    if (b->mixed && global->precision != 32) return fail(HHG_ERR_STATE, "mixed precision needs precision-32 meshes");
    for (int t = 0; t < n_tasks; ++t)
      if (meshes[t] == global) return fail(HHG_ERR_ARG, "the global mesh may not also be a task");
    b->tasks.push_back({global, global_cycles, nullptr, nullptr, nullptr});
  }
  auto cleanup = [&](int rc) {
    for (auto& t : b->tasks) {
      if (t.stream) cudaStreamDestroy(t.stream);
      if (t.done) cudaEventDestroy(t.done);
      if (t.done_time) cudaEventDestroy(t.done_time);
    }
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->start) cudaEventDestroy(b->start);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->graph) cudaGraphDestroy(b->graph);
    free_persistent(b.get());
    return rc;
  };
  if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&b->start) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(fail(HHG_ERR_CUDA, "stream / event creation failed"));
  for (auto& t : b->tasks)
    if (cudaStreamCreateWithFlags(&t.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&t.done_time) != cudaSuccess)
      return cleanup(fail(HHG_ERR_CUDA, "stream / event creation failed"));
  // one uncaptured pass (fills the launch-shape caches; same work as the graph)
  const size_t n_rec = (size_t)n_tasks;
  for (size_t t = 0; t < b->tasks.size(); ++t) {
    int rc = capture_task(b->tasks[t].mesh, b->tasks[t].cycles, t < n_rec, b->mixed, b->origin);
    if (rc != HHG_OK) return cleanup(rc);
  }
  if (cudaStreamSynchronize(b->origin) != cudaSuccess) return cleanup(fail(HHG_ERR_CUDA, "warm-up pass failed"));
  // capture: fork one branch per task from the origin stream, join at the end
  if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return cleanup(fail(HHG_ERR_CUDA, "cudaStreamBeginCapture failed"));
  int rc = HHG_OK;
  const long long k0 = g_kernel_launches.load();
  // timing events are captured as event-record nodes (External); fork and
  // join events only order the branches
  if (cudaEventRecordWithFlags(b->start, b->origin, cudaEventRecordExternal) != cudaSuccess ||
      cudaEventRecord(b->fork, b->origin) != cudaSuccess)
    rc = fail(HHG_ERR_CUDA, "event record in capture failed");
  for (size_t t = 0; t < b->tasks.size() && rc == HHG_OK; ++t) {
    auto& task = b->tasks[t];
    if (cudaStreamWaitEvent(task.stream, b->fork, 0) != cudaSuccess) {
      rc = fail(HHG_ERR_CUDA, "fork in capture failed");
      break;
    }
    rc = capture_task(task.mesh, task.cycles, t < n_rec, b->mixed, task.stream);
    if (rc == HHG_OK && (cudaEventRecordWithFlags(task.done_time, task.stream, cudaEventRecordExternal) != cudaSuccess ||
                         cudaEventRecord(task.done, task.stream) != cudaSuccess ||
                         cudaStreamWaitEvent(b->origin, task.done, 0) != cudaSuccess))
      rc = fail(HHG_ERR_CUDA, "join in capture failed");
  }
  // captured kernels are counted as launches when the graph runs
  b->kernels = g_kernel_launches.load() - k0;
  g_kernel_launches -= b->kernels;
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(b->origin, &g);
  if (rc != HHG_OK) {
    if (g) cudaGraphDestroy(g);
    return cleanup(rc);
  }
  if (ec != cudaSuccess) return cleanup(fail(HHG_ERR_CUDA, std::string("capture failed: ") + cudaGetErrorString(ec)));
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
    return cleanup(fail(HHG_ERR_CUDA, "cudaGraphInstantiate failed"));
  rc = setup_persistent(b.get(), n_rec);
  if (rc != HHG_OK) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    return cleanup(rc);
  }
  // the graph holds the meshes' buffers: a new fault set may not free them
  for (auto& t : b->tasks) ++t.mesh->batch_refs;
  *out = b.release();
  return HHG_OK;
}

int hhg_batch_launch(hhg_batch* b, double* task_ms, void* stream) {
  if (!b) return fail(HHG_ERR_ARG, "null batch");
  if (!b->tasks.empty()) HHG_TRY(check_device(b->tasks[0].mesh));
  cudaStream_t s = (cudaStream_t)stream;
  HHG_CUDA(cudaGraphLaunch(b->exec, s));
  g_kernel_launches += b->kernels;
  if (task_ms) {
    HHG_CUDA(cudaStreamSynchronize(s));
    for (size_t t = 0; t < b->tasks.size(); ++t) {
      float ms = 0.f;
      HHG_CUDA(cudaEventElapsedTime(&ms, b->start, b->tasks[t].done_time));
      task_ms[t] = ms;
    }
  }
  return HHG_OK;
}

int hhg_batch_launch_persistent(hhg_batch* b, double* task_ms, void* stream) {
  if (!b) return fail(HHG_ERR_ARG, "null batch");
  if (b->tasks.empty()) return HHG_OK;
  HHG_TRY(check_device(b->tasks[0].mesh));
  cudaStream_t s = (cudaStream_t)stream;
  const int n = (int)b->tasks.size();
  const int n_ops = (int)b->ops.size();
  HHG_CUDA(cudaMemsetAsync(b->d_state, 0, b->state_bytes, s));
  HHG_CUDA(cudaMemsetAsync(b->d_ns, 0xff, sizeof(unsigned long long), s));   // start: atomicMin over the CTAs
  BatchState st;
  st.phase = b->d_state;
  st.issued = b->d_state + n;
  st.done = b->d_state + n + n_ops;
  st.tasks_done = b->d_state + n + 2 * n_ops;
  st.start_ns = b->d_ns;
  st.task_ns = b->d_ns + 1;
  int n_live = 0;
  for (int t = 0; t < n; ++t) n_live += b->op_off[t + 1] > b->op_off[t] ? 1 : 0;
  HHG_CUDA(run_batch(b->d_ops, b->d_op_off, b->d_order, b->d_seg, b->n_seg, n_live, st, b->wait_limit, b->d_err, s));
  if (task_ms) {
    std::vector<unsigned long long> ns(n + 1);
    int err = 0;
    HHG_CUDA(cudaMemcpyAsync(ns.data(), b->d_ns, (n + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    HHG_CUDA(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    HHG_CUDA(cudaStreamSynchronize(s));
    if (err != 0) {
      HHG_CUDA(cudaMemsetAsync(b->d_err, 0, sizeof(int), s));
      HHG_CUDA(cudaStreamSynchronize(s));
      return fail(HHG_ERR_TIMEOUT, "the persistent batch found no work for longer than its wait limit");
    }
    for (int t = 0; t < n; ++t)
      task_ms[t] = b->op_off[t + 1] > b->op_off[t] ? (double)(ns[t + 1] - ns[0]) * 1e-6 : 0.0;
  }
  return HHG_OK;
}

int hhg_batch_set_priority(hhg_batch* b, const int* prio) {
  if (!b) return fail(HHG_ERR_ARG, "null batch");
  if (b->tasks.empty()) return HHG_OK;
  HHG_TRY(check_device(b->tasks[0].mesh));
  std::vector<int> p(b->tasks.size(), 0);
  if (prio) p.assign(prio, prio + b->tasks.size());
  HHG_CUDA(cudaDeviceSynchronize());   // no launch may still read the old order
  return upload_priorities(b, p);
}

int hhg_batch_info(hhg_batch* b, int64_t* info) {
  if (!b || !info) return fail(HHG_ERR_ARG, "invalid argument");
  int64_t units = 0;
  for (const BOp& op : b->ops) units += op.n_units;
  info[0] = (int64_t)b->tasks.size();
  info[1] = (int64_t)b->ops.size();
  info[2] = units;
  info[3] = b->kernels;
  return HHG_OK;
}

int hhg_batch_destroy(hhg_batch* b) {
  if (!b) return HHG_OK;
  cudaDeviceSynchronize();
  free_persistent(b);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto& t : b->tasks) {
    --t.mesh->batch_refs;
    if (t.stream) cudaStreamDestroy(t.stream);
    if (t.done) cudaEventDestroy(t.done);
    if (t.done_time) cudaEventDestroy(t.done_time);
  }
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->start) cudaEventDestroy(b->start);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
  return HHG_OK;
}

int hhg_profile_enable(hhg_mesh* m, int enable) {
  if (!m) return fail(HHG_ERR_ARG, "null mesh");
  m->prof_on = (enable & 1) != 0;
  m->prof_used = 0;
  m->bd_on = (enable & 2) != 0;
  m->bd_used = 0;
  return HHG_OK;
}

int hhg_profile_breakdown(hhg_mesh* m, double* ms, int n) {
  if (!m || !ms || n < BD_N) return fail(HHG_ERR_ARG, "invalid argument");
  HHG_TRY(check_device(m));
  HHG_CUDA(cudaDeviceSynchronize());
  for (int c = 0; c < n; ++c) ms[c] = 0.0;
  for (size_t q = 0; q + 1 < m->bd_used; ++q) {
    float t = 0.f;
    HHG_CUDA(cudaEventElapsedTime(&t, m->bd_ev[q], m->bd_ev[q + 1]));
    ms[m->bd_cat[q]] += t;
  }
  m->bd_used = 0;
  return HHG_OK;
}

int hhg_profile_read(hhg_mesh* m, int64_t* launches, double* total_ms) {
  if (!m) return fail(HHG_ERR_ARG, "null mesh");
  HHG_TRY(check_device(m));
  HHG_CUDA(cudaDeviceSynchronize());
  double t = 0.0;
  for (size_t q = 0; q + 1 < m->prof_used; q += 2) {
    float ms = 0.f;
    HHG_CUDA(cudaEventElapsedTime(&ms, m->prof_ev[q], m->prof_ev[q + 1]));
    t += ms;
  }
  if (launches) *launches = (int64_t)(m->prof_used / 2);
  if (total_ms) *total_ms = t;
  m->prof_used = 0;
  return HHG_OK;
}

int hhg_profile_info(const hhg_mesh* m, int64_t* volume_nodes, int* seven_point) {
  if (!m) return fail(HHG_ERR_ARG, "null mesh");
  const int N = m->host.lv.back().N;
  if (volume_nodes) *volume_nodes = (int64_t)m->host.n_macro * (N - 1) * (N - 2) * (N - 3) / 6;
  if (seven_point) *seven_point = m->host.seven_point ? 1 : 0;
  return HHG_OK;
}

int hhg_set_launch_limit(hhg_mesh* m, int max_ctas) {
  if (!m || max_ctas < 0) return fail(HHG_ERR_ARG, "invalid argument");
  HHG_TRY(check_device(m));
  m->grid_cap = max_ctas;
  for (DevProblem* p : {&m->global, &m->faulty, &m->healthy, &m->dn}) p->grid_cap = max_ctas;
  // captured recovery cycles hold the old launch shapes
  drop_local_graph(m);
  return HHG_OK;
}

int hhg_set_streaming(hhg_mesh* m, int enable) {
  if (!m) return fail(HHG_ERR_ARG, "null mesh");
  HHG_TRY(check_device(m));
  m->stream_gs = enable ? 1 : 0;
  for (DevProblem* p : {&m->global, &m->faulty, &m->healthy, &m->dn}) p->stream_gs = m->stream_gs;
  drop_local_graph(m);
  return HHG_OK;
}

int hhg_set_flat_gs(hhg_mesh* m, int enable) {
  if (!m) return fail(HHG_ERR_ARG, "null mesh");
  HHG_TRY(check_device(m));
  HHG_TRY(refuse_general(m, "the flat Gauss-Seidel kernel"));
  if (!m->host.seven_point) return HHG_OK;   // the flat kernels serve the 7-point structure only
  const int nl = (int)m->host.lv.size();
  if (enable)
    for (int l = 1; l < nl; ++l)
      if (!flat_fits(m, l))
        return fail(HHG_ERR_ARG, "the flat kernels need 4 .. 1024 intervals per macro edge and fewer than 2^31 "
                                 "items per launch");
  drop_local_graph(m);
  for (int l = 1; l < nl; ++l) HHG_TRY(set_flat(m, l, enable != 0));
  return HHG_OK;
}

int hhg_set_wait_limit(hhg_mesh* m, int tries) {
  if (!m) return fail(HHG_ERR_ARG, "null mesh");
  HHG_TRY(check_device(m));
  m->wait_limit = tries >= 0 ? tries : (1 << 24);
  for (DevProblem* p : {&m->global, &m->faulty, &m->healthy, &m->dn}) p->wait_limit = m->wait_limit;
  drop_local_graph(m);
  return HHG_OK;
}

int hhg_walk_counts(hhg_mesh* m, int64_t* counts) {
  if (!m || !counts) return fail(HHG_ERR_ARG, "null argument");
  HHG_TRY(check_device(m));
  const DevProblem* probs[4] = {&m->global, &m->faulty, &m->healthy, &m->dn};
  int v[4] = {0, 0, 0, 0};
  HHG_CUDA(cudaDeviceSynchronize());
  for (int q = 0; q < 4; ++q)
    if (probs[q]->sched) HHG_CUDA(cudaMemcpy(&v[q], probs[q]->sched + 2, sizeof(int), cudaMemcpyDeviceToHost));
  for (int q = 0; q < 4; ++q) counts[q] = v[q];
  return HHG_OK;
}

int hhg_measure_fp64_peak(double* tflops) {
  if (!tflops) return fail(HHG_ERR_ARG, "null argument");
  int dev = 0, sms = 0;
  HHG_CUDA(cudaGetDevice(&dev));
  HHG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 8 * sms, iters = 1 << 14;
  double* out = nullptr;
  HHG_CUDA(cudaMalloc(&out, sizeof(double) * 256 * (size_t)blocks));
  CallEvents ev;
  cudaError_t e = ev.create(2);
  double best = 0.0;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(ev.e[0], 0);
    if (e == cudaSuccess) e = fma_probe(out, blocks, iters, 0);
    if (e == cudaSuccess) e = cudaEventRecord(ev.e[1], 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev.e[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]);
    if (e == cudaSuccess && rep > 0 && ms > 0.f)   // the first launch is a warm-up
      best = std::max(best, 2.0 * 8.0 * iters * 256.0 * blocks / (ms * 1e-3) / 1e12);
  }
  cudaFree(out);
  if (e != cudaSuccess) return fail(HHG_ERR_CUDA, std::string("FP64 probe: ") + cudaGetErrorString(e));
  *tflops = best;
  return HHG_OK;
}

int hhg_launch_count(int64_t* count) {
  if (!count) return fail(HHG_ERR_ARG, "null argument");
  *count = (int64_t)g_kernel_launches.load();
  return HHG_OK;
}

int hhg_solve(hhg_mesh* m, const hhg_solve_opts* o, double* hist, int* n_hist, int* cycles, void* stream) {
  if (!m || !o) return fail(HHG_ERR_ARG, "null argument");
  HHG_TRY(check_device(m));
  if (o->max_cycles < 0 || !(o->rtol >= 0.0)) return fail(HHG_ERR_ARG, "invalid rtol / max_cycles");
  if (o->mixed_precision) HHG_TRY(refuse_general(m, "mixed precision"));
  const bool mixed = o->mixed_precision != 0;
  if (mixed && m->precision != 32) return fail(HHG_ERR_STATE, "mixed precision needs a precision-32 mesh");
  const int pre = o->pre > 0 ? o->pre : 3, post = o->post > 0 ? o->post : 3;
  const double cg_rtol = o->coarse_rtol > 0 ? o->coarse_rtol : 1e-12;
  const int cg_maxit = o->coarse_maxit > 0 ? o->coarse_maxit : 1000;
  // fault events: (cycle, id set) in the order they are handled
  struct Event {
    int cycle;
    std::vector<unsigned char> set;
  };
  std::vector<Event> events;
  if (o->n_faults < 0 || (o->n_faults > 0 && !o->faults)) return fail(HHG_ERR_ARG, "invalid fault list");
  for (int q = -1; q < o->n_faults; ++q) {
    const int cyc = q < 0 ? o->fault_cycle : o->faults[q].cycle;
    if (cyc <= 0) {
      if (q < 0) continue;
      return fail(HHG_ERR_ARG, "fault cycle must be positive");
    }
    Event ev;
    ev.cycle = cyc;
    if (q < 0) HHG_TRY(check_ids(m, o->fault_ids, o->n_fault_ids, ev.set));
    else HHG_TRY(check_ids(m, o->faults[q].macro_ids, o->faults[q].n_ids, ev.set));
    events.push_back(std::move(ev));
  }
  if (!events.empty()) {
    if (o->recovery < HHG_RECOVERY_NONE || o->recovery > HHG_RECOVERY_DN)
      return fail(HHG_ERR_ARG, "unknown recovery strategy");
    if (o->recovery == HHG_RECOVERY_DN && (o->n_global < 0 || !(o->eta >= 0.0)))
      return fail(HHG_ERR_ARG, "invalid n_global / eta");
    // the first fault's sub-problems are built before the timed iteration
    if (o->recovery == HHG_RECOVERY_DN) HHG_TRY(setup_dn(m, events[0].set));
    else HHG_TRY(setup_fault(m, events[0].set));
  }
  cudaStream_t s = (cudaStream_t)stream;
  int nh = 0;
  auto push = [&](double v) {
    if (hist) hist[nh] = v;
    ++nh;
  };
  // residual norm of the current iterate
  double r0 = 0.0, v = 0.0;
  if (mixed) {
    HHG_TRY(ir_residual(m, m->global, s));
    HHG_TRY(read_scalar(m, m->global.scalar, &v, s));
    r0 = std::sqrt(v);
  } else {
    HHG_TRY(resnorm(m, &r0, s));
  }
  push(1.0);
  int k = 0;
  double rel = 1.0;
  while (k < o->max_cycles) {
    if (mixed) {
      // the residual of the current iterate is already the FP32 right-hand side
      const int L = (int)m->d64.lv.size() - 1;
      DevLevel<float>& E = m->d32.lv[L];
      HHG_TRY(bd_mark(m, s, BD_IR));
      HHG_CUDA(zero_problem_blocks<float>(largs(m, L), pargs(m->global, L), E.u, E.uI, s));
      HHG_TRY(vcycle_T<float>(m, m->d32, m->global, pre, post, cg_rtol, cg_maxit, s));
      DevLevel<double>& D = m->d64.lv[L];
      HHG_TRY(bd_mark(m, s, BD_IR));
      HHG_CUDA(add_correction(largs(m, L), pargs(m->global, L), D.u, D.uI, E.u, E.uI, s));
      HHG_TRY(bd_mark(m, s, BD_NORM));
      HHG_TRY(ir_residual(m, m->global, s));
      HHG_TRY(bd_mark(m, s, BD_HOST));
      HHG_TRY(read_scalar(m, m->global.scalar, &v, s));
    } else {
      HHG_TRY(vcycle_T<double>(m, m->d64, m->global, pre, post, cg_rtol, cg_maxit, s));
      HHG_TRY(bd_mark(m, s, BD_NORM));
      HHG_TRY(norm2_async(m, m->global, s, post > 0));
      HHG_TRY(bd_mark(m, s, BD_HOST));
      HHG_TRY(read_scalar(m, m->global.scalar, &v, s));
    }
    ++k;
    rel = r0 > 0 ? std::sqrt(v) / r0 : 0.0;
    push(rel);
    for (const Event& ev : events) {
      if (ev.cycle != k) continue;
      if (o->recovery == HHG_RECOVERY_DN) HHG_TRY(setup_dn(m, ev.set));
      else HHG_TRY(setup_fault(m, ev.set));
      HHG_TRY(bd_mark(m, s, BD_RECOVERY));
      HHG_TRY(inject(m, s));
      if (o->recovery == HHG_RECOVERY_DN) {
        HHG_TRY(recover_dn(m, o->n_global, o->eta, mixed, pre, post, cg_rtol, cg_maxit, nullptr, nullptr, nullptr, s));
      } else if (o->recovery != HHG_RECOVERY_NONE) {
        const int n_global = o->recovery == HHG_RECOVERY_DD ? o->n_global : 0;
        int n_local = o->n_local;
        if (n_local <= 0 && o->recovery == HHG_RECOVERY_DD) n_local = (int)std::ceil(o->eta * o->n_global);
        HHG_TRY(recover(m, n_local, n_global, mixed, pre, post, cg_rtol, cg_maxit, nullptr, nullptr, s));
      }
      HHG_TRY(bd_mark(m, s, BD_NORM));
      if (mixed) HHG_TRY(ir_residual(m, m->global, s));
      else HHG_TRY(norm2_async(m, m->global, s));
      HHG_TRY(bd_mark(m, s, BD_HOST));
      HHG_TRY(read_scalar(m, m->global.scalar, &v, s));
      rel = r0 > 0 ? std::sqrt(v) / r0 : 0.0;
      push(rel);
    }
    if (rel <= o->rtol) break;
  }
  if (n_hist) *n_hist = nh;
  if (cycles) *cycles = k;
  if (rel > o->rtol) return fail(HHG_ERR_NOT_CONVERGED, "rtol not reached within max_cycles");
  return HHG_OK;
}

}  // extern "C"
