// Launchers of the HHG CUDA kernels (kernels.cu).  T is the arithmetic type of
// the cycle (double, or float for the inner cycles of mixed-precision
// iterative refinement).
#pragma once

#include <vector>

#include "hhg_internal.h"

namespace hhg {

struct LevelArgs {
  int N;
  const int* rs;   // slice-start table of the block layout (N + 3 entries)
  int64_t block;
  const int64_t* if_gid;
  const int* cptr;
  const Copy* cps;
  const uint32_t* cp_off;   // block offsets of the copies cps (null: computed)
  const Tile* tiles_int;
  int n_tiles_int;
  const Tile* tiles_all;
  int n_tiles_all;
  const StreamTile* tiles_stream;   // streaming Gauss-Seidel units of the FP64 cycles (none below
  int n_tiles_stream;               // STREAM_MIN_N) and their rows per band
  int stream_band;
  const StreamTile* tiles_stream32; // the same for the FP32 cycles
  int n_tiles_stream32;
  int stream_band32;
  const uint32_t* gs_items64;       // flat Gauss-Seidel items (build_gs_items), FP64 and FP32,
  const uint32_t* gs_items32;       // with their per-colour offsets; used when gs_flat is set
  int gs_off64[5];
  int gs_off32[5];
  const uint32_t* slot_items;       // the flat restriction's items on this (coarse) level
  int n_slots;
  int gs_flat;
};

struct ProbArgs {
  const int* act;
  int n_act;
  const int* free_if;
  int col_off[5];
  const int64_t* zero_off;
  int n_zero;
  const int64_t* gather;
  int* sched;      // the problem's dynamic-walk counters: [0] next unit, [1] finished CTAs (both
                   // zero between launches), [2] dynamic launches completed
  int grid_cap;    // > 0: at most this many CTAs per fused launch (0: as many as are resident)
  // interface stencil tables of free_if (DevProblemLevel; tnb null: none)
  const uint32_t* tnb;
  const double* tw64;
  const double* td64;
  const double* ti64;
  const float* tw32;
  const float* td32;
  const float* ti32;
  int tn;
  int stream_gs;   // 1: 7-point Gauss-Seidel uses the streaming kernel where the level has units
  int* err;        // device flag: set to 1 when a bounded wait of a kernel runs out
  int wait_limit;  // tries of such a wait (about 64 ns apart)
};

// One colour of multicolour Gauss-Seidel on the volume interiors and the free
// interface nodes of a problem.
// If ev_begin / ev_end are not null they are recorded on s right before and
// after the volume kernel (profiling of the dominant kernel).  With the
// 7-point stencil, fs and Wsc (both non-null) are f and the interior weights
// divided by each macro's centre weight: the volume nodes are then updated as
// u = fs - sum Wsc u (no final scaling); the interface nodes always use fI, W.
template <class T>
cudaError_t gs_colour(const LevelArgs& L, const ProbArgs& p, T* u, T* uI, const T* f, const T* fI,
                      const T* W, const T* Winv, int colour, bool seven_point, cudaStream_t s,
                      cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr, const T* fs = nullptr,
                      const T* Wsc = nullptr);

// out[t * block + o] = f[t * block + o] * winv[t] for the n_macro blocks.
cudaError_t scale_blocks(const double* f, const double* winv, double* out, int n_macro, int64_t block,
                         cudaStream_t s);

// r = f - A u on the free nodes (written to the blocks' r), zero at the
// problem's frozen copies.  If partial != NULL each CTA also writes its
// partial sum of r^2 (volume CTAs first, then interface CTAs) and write_r may
// be false (norm only).  Returns the number of partials written in *n_part.
// skip (0..3, cube-family meshes only): the colour smoothed last, whose
// nodes' residual vanishes (all their neighbours have other colours and were
// updated before them); it is written as zero without evaluating the stencil.
template <class T>
cudaError_t residual(const LevelArgs& L, const ProbArgs& p, const T* u, const T* uI, const T* f,
                     const T* fI, T* r, const T* W, bool seven_point, bool write_r, double* partial,
                     int* n_part, cudaStream_t s, int skip = -1);

// Coarse right-hand side f_c = P^T r_f on the free coarse nodes; the coarse
// correction u_c is set to zero on the problem's nodes of the coarse level.
template <class T>
cudaError_t restrict_to(const LevelArgs& C, const LevelArgs& F, const ProbArgs& pc, const T* rf, T* fc,
                        T* fIc, T* uc, T* uIc, cudaStream_t s);

// u_f += P u_c on the free fine nodes.  skip (0..3): the volume nodes of that
// colour are left out, and the interface list entries [if_lo, if_hi) too --
// for nodes the next Gauss-Seidel colour overwrites without reading them.
template <class T>
cudaError_t prolong_add(const LevelArgs& F, const LevelArgs& C, const ProbArgs& pf, T* uf, T* uIf,
                        const T* uc, cudaStream_t s, int skip = -1, int if_lo = 0, int if_hi = 0);

// Coarse CG (FP64) on the compact free nodes of level 0; reads the level's
// right-hand side (type T), writes the solution into u / uI.  work (4 n_cg
// doubles) replaces the problem's own work vectors when not null.
template <class T>
cudaError_t coarse_cg(const DevProblem& p, const T* f, const T* fI, T* u, T* uI, double rtol, int maxit,
                      cudaStream_t s, double* work = nullptr);

cudaError_t reduce_partials(const double* partial, int n, double* out, cudaStream_t s);

// FP64 FMA throughput probe: `blocks` CTAs of 256 threads, 8 x iters FMAs per
// thread; out holds blocks * 256 doubles.
cudaError_t fma_probe(double* out, int blocks, int iters, cudaStream_t s);

// Global vector <-> blocked storage of one level.
template <class T>
cudaError_t import_vec(const LevelArgs& L, const MacroGeo* geo, int n_macro, int64_t nx, int64_t ny,
                       const double* g, T* blocks, T* masters, bool closed, cudaStream_t s);
template <class T>
cudaError_t export_vec(const LevelArgs& L, const MacroGeo* geo, int n_macro, int64_t nx, int64_t ny,
                       const T* blocks, const T* masters, double* g, cudaStream_t s);

template <class T>
cudaError_t import_masters(const int64_t* gid, int n, const double* g, T* m, cudaStream_t s);
template <class T>
cudaError_t export_masters(const int64_t* gid, int n, const T* m, double* g, cudaStream_t s);

// Coefficient gradient: partial[macro * n_tiles_all + tile] = sum over the
// closed-lattice nodes p of the tile of lam_p (sub-stencil of the macro at p
// applied to u); reduce_per_macro sums them into out[macro].
cudaError_t grad_partials(const LevelArgs& L, int n_macro, const double* u, const double* lam, const double* W,
                          double* partial, cudaStream_t s);
cudaError_t reduce_per_macro(const double* partial, int n_per, int n_macro, double* out, cudaStream_t s);

// Fault support.
// out[list[q]] = (A u) at interface node list[q], summed over the copies that
// L's copy lists hold for it (FP64, finest level).
cudaError_t apply_if_nodes(const LevelArgs& L, const double* u, const double* uI, const double* W, bool seven_point,
                           const int* list, int n, double* out, cudaStream_t s);
// dst[idx[q]] = src[idx[q]] for q < n.
cudaError_t copy_listed(const double* src, double* dst, const int* idx, int n, cudaStream_t s);
cudaError_t set_masters_zero(double* uI, const int* ids, int n, cudaStream_t s);
cudaError_t restore_copies(double* u, const double* uI, const int64_t* off, const int* master, int n,
                           cudaStream_t s);

// Mixed precision: fine FP64 residual written as the FP32 right-hand side of
// the correction problem (blocks and masters), with its norm partials.
cudaError_t residual_to_f32(const LevelArgs& L, const ProbArgs& p, const double* u, const double* uI,
                            const double* f, const double* fI, float* f32, float* fI32, const double* W,
                            bool seven_point, double* partial, int* n_part, cudaStream_t s);
// u64 += e32 on the free nodes (volume interiors and interface masters + copies).
cudaError_t add_correction(const LevelArgs& L, const ProbArgs& p, double* u, double* uI, const float* e,
                           const float* eI, cudaStream_t s);
template <class T>
cudaError_t zero_problem_blocks(const LevelArgs& L, const ProbArgs& p, T* u, T* uI, cudaStream_t s);

// ---------------------------------------------------------------------------
// Persistent batch executor (kernels.cu).  A program is the list of the
// level-wide operations one task issues (fault injection, Gauss-Seidel
// colours, residuals, transfers, coarse CG, the FP64/FP32 hand-over of
// iterative refinement), each split into the work units its kernel would
// walk.  While a recording is open, the launchers of this header append an
// operation instead of launching; run_batch then executes the programs of
// many tasks in one launch.
// ---------------------------------------------------------------------------
enum BOpKind : int {
  BOP_GS, BOP_RES, BOP_RESTRICT, BOP_PROLONG, BOP_CG, BOP_ZERO_BLOCKS, BOP_ZERO_LIST, BOP_RES_F32,
  BOP_ADD_BLOCKS, BOP_ADD_MASTERS, BOP_MEMSET, BOP_SET_ZERO, BOP_RESTORE
};

struct BOp {
  int kind;            // BOpKind
  int fp32;            // arithmetic type of the arrays: 1 float, 0 double
  int n_units;
  int n_if_units;      // interface chunks, first (GS, RES, RESTRICT, PROLONG, RES_F32)
  int seven_point, scaled, colour, skip, skip_lo, skip_hi;
  LevelArgs L;         // the level (the fine one of a transfer)
  LevelArgs C;         // the coarse level of a transfer
  ProbArgs P;          // the problem on L (on C for a restriction)
  int list_off;        // first entry of P.free_if the operation walks
  int n_list;
  int n_zero;          // frozen copies zeroed after the list (RES, RESTRICT)
  // arrays (float or double by fp32; FP64 + FP32 for the hand-over)
  void* u;
  void* uI;
  const void* f;
  const void* fI;
  void* r;
  const void* W;       // stencil weights (interface sub-stencils)
  const void* Wv;      // the volume's weights (GS: divided by the centre weight when scaled)
  const void* Winv;
  void* fc;
  void* fIc;
  void* uc;
  void* uIc;
  void* o32;           // RES_F32 output, ADD_* correction (FP32)
  void* oI32;
  int64_t n;           // element count (ZERO_LIST, MEMSET in 16-byte words, SET_ZERO, RESTORE, ADD_MASTERS)
  const int* ids;      // ZERO_LIST, SET_ZERO, ADD_MASTERS: index list; RESTORE: master per copy
  const int64_t* offs; // RESTORE: block offsets
  // coarse CG (level 0 of the problem)
  int n_cg;
  const int* rowptr;
  const int* col;
  const double* val;
  const int64_t* fsrc;
  const int* uptr;
  const int64_t* udst;
  const int* umaster;
  double* work;
  int* iters;
  double rtol;
  int maxit;
};

// While rec != null the launchers append to *rec instead of launching.
void record_ops(std::vector<BOp>* rec);
bool recording();
// Zero `bytes` bytes at p (a multiple of 16; recorded as BOP_MEMSET).
cudaError_t memset16(void* p, size_t bytes, cudaStream_t s);
// Runs the programs ops[op_off[t] .. op_off[t + 1]) of the tasks in one
// launch (grid = resident CTAs).  order[seg[c] .. seg[c + 1]) lists the
// tasks of priority class c (n_seg classes, highest first; every task in
// exactly one class); n_live tasks have at least one operation.  The
// counters (phase per task, issued and done per operation, tasks done) must
// be zero and *start_ns ~0 before the launch.  task_ns[t] receives the
// global timer when task t finished, *start_ns the earliest start.
struct BatchState {
  int* phase;
  int* issued;
  int* done;
  int* tasks_done;
  unsigned long long* start_ns;
  unsigned long long* task_ns;
};
cudaError_t run_batch(const BOp* ops, const int* op_off, const int* order, const int* seg, int n_seg, int n_live,
                      const BatchState& st, int wait_limit, int* err, cudaStream_t s);

// Macro meshes of general connectivity (general.cu).  Global vectors list
// the interface nodes first (their masters move with import_masters /
// export_masters) and then the volume nodes macro by macro in local
// (k, j, i) order, which these two move into / out of the blocks.
template <class T>
cudaError_t general_import_vol(const LevelArgs& L, int n_macro, int64_t n_if, const double* g, T* blocks,
                               cudaStream_t s);
template <class T>
cudaError_t general_export_vol(const LevelArgs& L, int n_macro, int64_t n_if, const T* blocks, double* g,
                               cudaStream_t s);
// Restriction onto the free coarse interface nodes through variable-length
// gathers (gptr over pc.free_if, fine block offsets goff, the node itself
// first) and zeroing of the coarse correction there, on their copies and at
// the frozen copies pc.zero_off; the volume part is restrict_to's.
template <class T>
cudaError_t general_restrict_if(const LevelArgs& C, const ProbArgs& pc, const int* gptr, const int64_t* goff,
                                const T* rf, T* fIc, T* uc, T* uIc, cudaStream_t s);

}  // namespace hhg
