/*
 * hhg.h - C ABI of the GB300 resilient hierarchical-hybrid multigrid library.
 *
 * Method: Huber, Gmeiner, Ruede, Wohlmuth, "Resilience for Multigrid Software
 * at the Extreme Scale".  The library solves the P1 finite-element Poisson
 * problem of §2.1 (Eq. (1), discretised as Eq. (2)) on the unit cube split
 * into sub-cubes of six Kuhn macro-tetrahedra (the base mesh T_-2, §2.1),
 * refined uniformly, with matrix-free multigrid V-cycles (linear
 * interpolation, its adjoint, multicolour Gauss-Seidel smoothing, CG on the
 * coarsest level; §2.1), and recovers from the loss of the volume unknowns
 * of some macro-tetrahedra (the fault model of §2.2) with local Dirichlet
 * multigrid cycles (local recovery LR, §4.4) running, for the
 * Dirichlet-Dirichlet strategy (§4.2, Algorithm 1), concurrently with
 * global cycles on the healthy sub-domain.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - Every call returns an int status (HHG_OK on success).  Nothing throws
 *   across the ABI.  hhg_last_error() gives a message for the last failure
 *   of the calling thread.  A NULL handle or a NULL required pointer is
 *   rejected with HHG_ERR_ARG before any device use; destroying a NULL
 *   handle is a no-op that returns HHG_OK.
 * - A mesh handle owns all device storage it allocates; the caller owns the
 *   vectors it passes in.  Handles are not thread-safe: one thread at a time.
 * - A mesh lives on the device that was current when it was created.  Every
 *   call that takes a mesh (or a batch) needs that device current and
 *   returns HHG_ERR_STATE otherwise; hhg_mesh_destroy makes the mesh's device
 *   current by itself for the release and restores the caller's device.
 * - Global vectors (right-hand side, solution) are laid out over the global
 *   node grid, x fastest: node (x, y, z) of a grid with nx, ny, nz intervals
 *   has index (z * (ny + 1) + y) * (nx + 1) + x, nx = subcubes[0] * 2^levels
 *   etc.; there are (nx + 1)(ny + 1)(nz + 1) entries.  A vector pointer may
 *   be host memory (pageable or pinned) or device memory of the current
 *   device; the library tells them apart itself.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Calls that return values to the host synchronise that stream.
 * - The right-hand side is the algebraic load vector f_l of Eq. (2) (one
 *   value per node); its Dirichlet-node entries are ignored.  The solution
 *   vector carries the Dirichlet values g on the boundary nodes.
 */
#ifndef HHG_H
#define HHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HHG_OK = 0,
  HHG_ERR_ARG = 1,            /* invalid argument (sizes, ids, null pointer) */
  HHG_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  HHG_ERR_OOM = 3,            /* device or host allocation failed */
  HHG_ERR_TIMEOUT = 4,        /* a bounded device-side wait ran out
                                 (hhg_set_wait_limit) */
  HHG_ERR_NOT_CONVERGED = 5,  /* hhg_solve stopped at max_cycles above rtol */
  HHG_ERR_STATE = 6           /* call not valid in the mesh's current state */
};

/* Recovery strategies after a fault (§2.2 job classes, §4). */
enum {
  HHG_RECOVERY_NONE = 0,      /* do-nothing: zero re-initialisation only */
  HHG_RECOVERY_LR = 1,        /* n_F local cycles on Omega_F, Omega_I idle */
  HHG_RECOVERY_DD = 2,        /* Algorithm 1: n_F local cycles on Omega_F and,
                                 concurrently, n_I cycles on Omega_I with the
                                 interface frozen */
  HHG_RECOVERY_DN = 3         /* Algorithm 2 (§4.3): n_I cycles of a Neumann
                                 problem on Omega_I and the interface, with
                                 Dirichlet cycles on Omega_F interleaved */
};

typedef struct hhg_mesh hhg_mesh;

typedef struct {
  int subcubes[3];        /* sub-cubes per axis; 6 macro-tetrahedra each */
  int levels;             /* finest refinement R: 2^R intervals per macro edge */
  int coarsest;           /* coarsest refinement r0 (>= 2, < levels; 0 = 2) */
  int precision;          /* 64: FP64 cycles; 32: also allocate the FP32
                             inner-cycle arrays used by mixed-precision
                             iterative refinement (hhg_solve_opts) */
  const double* coeff;    /* host, one diffusion coefficient k_T per macro
                             (macro id = 6 * subcube + Kuhn type, sub-cubes x
                             fastest, Kuhn types in lexicographic axis order);
                             NULL = all ones */
  const double* affine;   /* host, 3x3 row-major linear map applied to the
                             unit cube's node positions; NULL = identity */
  const double* vertex_pos; /* host, physical positions of the
                             (sx+1)(sy+1)(sz+1) sub-cube corners, 3 doubles
                             each, corner (a, b, c) at index
                             (c (sy+1) + b)(sx+1) + a; NULL = the unit cube's
                             corners (mapped by affine).  Moved corners make
                             every macro a general tetrahedron of a polyhedral
                             domain with the cube family's connectivity (§2.1:
                             unstructured base mesh, uniform refinement per
                             macro); each macro must keep its Kuhn simplex's
                             orientation (else HHG_ERR_ARG).  Not together
                             with affine. */
} hhg_mesh_desc;

/* Build the macro mesh, all levels coarsest..levels, the per-macro stencils
 * (15 weights per node class, interface sub-stencils summed per node, §3.2
 * Fig. 4) and the device storage (per-macro blocks with a ghost shell and
 * face/edge/vertex interface containers, §3.1).  *out receives the handle. */
int hhg_mesh_create(const hhg_mesh_desc* desc, hhg_mesh** out);
int hhg_mesh_destroy(hhg_mesh* mesh);

/* A macro mesh of general connectivity (§2.1: an unstructured tetrahedral
 * base mesh of a polyhedral domain, refined uniformly inside every macro).
 * vertices: host, n_vertices x 3 doubles; macros: host, n_macros x 4 vertex
 * ids (any order, a conforming mesh: a face belongs to at most two macros);
 * coeff: host, one positive coefficient per macro or NULL.  The Dirichlet
 * boundary is every face of a single macro.  Global vectors of such a mesh
 * list first the interface nodes (vertex, edge and face nodes of the macro
 * mesh) sorted by key - the number of macro vertices with a positive
 * barycentric weight, then the values vertex id * (2^levels + 1) + weight of
 * those vertices in ascending order - and then the volume nodes macro by
 * macro, node (i, j, k) of a macro (weights (N-i-j-k, i, j, k) on its
 * vertices in the given order) in the order k, then j, then i; hhg_mesh_info
 * gives their count.  One Gauss-Seidel step visits the volume nodes by their
 * macro's colour (i + 2j + 3k) mod 4 and then the interface nodes in the
 * classes of a greedy colouring of their couplings in key order.
 * V-cycles (also the allocation-free one), solves, fault injection and LR /
 * DD / DN recovery (FP64) are available; mixed precision, coefficient changes
 * and gradients, batching and autotuning return HHG_ERR_STATE for these
 * meshes.  Errors: HHG_ERR_ARG for invalid sizes, ids, degenerate macros or
 * a non-conforming mesh (found before any device use). */
typedef struct {
  int n_vertices;
  const double* vertices;
  int n_macros;
  const int* macros;
  int levels;             /* finest refinement R: 2^R intervals per macro edge */
  int coarsest;           /* coarsest refinement r0 (>= 2, < levels; 0 = 2) */
  int precision;          /* 64 or 32, as for hhg_mesh_desc */
  const double* coeff;
} hhg_general_desc;
int hhg_mesh_create_general(const hhg_general_desc* desc, hhg_mesh** out);

/* n_nodes: entries of a global vector; n_dof: non-Dirichlet fine nodes;
 * n_macro: macro-tetrahedra.  Any output pointer may be NULL. */
int hhg_mesh_info(const hhg_mesh* mesh, int64_t* n_nodes, int64_t* n_dof, int* n_macro);

/* Device bytes held by the mesh (all levels, interface tables, scratch). */
int hhg_mesh_bytes(const hhg_mesh* mesh, int64_t* bytes);

/* Load the right-hand side f (may be NULL: keep the current one, initially
 * zero) and the initial guess u0 including Dirichlet values (may be NULL:
 * keep the current iterate, initially zero) from global vectors.  With the
 * 7-point stencil the mesh also keeps f divided by each macro's centre weight
 * for the finest level's FP64 Gauss-Seidel; it is refreshed here and by
 * hhg_set_coefficients. */
int hhg_set_problem(hhg_mesh* mesh, const double* f, const double* u0, void* stream);

/* Write the current fine-level iterate into the global vector u. */
int hhg_get_solution(hhg_mesh* mesh, double* u, void* stream);

/* One global V(pre, post) cycle (§2.1) on the current iterate.  If resid_out
 * is not NULL it receives ||f - A u||_2 over the non-Dirichlet fine nodes
 * after the cycle (synchronises the stream). */
int hhg_vcycle(hhg_mesh* mesh, int pre, int post, double* resid_out, void* stream);

/* ||f - A u||_2 over the non-Dirichlet fine nodes (synchronises). */
int hhg_residual_norm(hhg_mesh* mesh, double* out, void* stream);

/* Fault model of §2.2: the macro-tetrahedra macro_ids[0..n_ids) lose their
 * volume storage (block and ghost shell) and every unknown strictly inside
 * their union Omega_F is re-initialised with zero.  The interface values on
 * Gamma survive in the face/edge/vertex containers and are written back into
 * the ghost shells of the lost blocks (Eq. (4), row 4; Algorithm 1 step 4).
 * Ids must be distinct and in [0, n_macro).  The first call for a set builds
 * the set's recovery sub-problems on the device; a call with another set
 * replaces them and frees the previous ones (after synchronising the
 * device), except while a batch (hhg_batch_create) refers to the mesh. */
int hhg_inject_fault(hhg_mesh* mesh, const int* macro_ids, int n_ids, void* stream);

/* Recovery after hhg_inject_fault on the same ids.  n_local V-cycles of the
 * Dirichlet problem A_FF u_F = f_F - A_FG u_G on Omega_F (Algorithm 1 step
 * a).  n_global = 0: local recovery (LR), Omega_I idles.  n_global > 0:
 * Dirichlet-Dirichlet recovery, n_global V-cycles of A_II u_I = f_I -
 * A_IG u_G on Omega_I with the interface frozen (step b) run on the caller's
 * stream concurrently with the Omega_F cycles, which run on a stream of the
 * device's highest priority (forked from and joined back into `stream`).  If seconds_local / seconds_global are not NULL they
 * receive the device time of the two cycle sequences (synchronises).  With
 * n_local >= 2 the first Omega_F cycle runs directly and the others replay a
 * CUDA graph of one cycle, captured on the first such call for the fault set
 * and kept until the set, the cycle parameters or the tile shapes change
 * (inside a caller's stream capture the cycles are recorded directly). */
int hhg_recover_local(hhg_mesh* mesh, const int* macro_ids, int n_ids, int n_local,
                      int n_global, double* seconds_local, double* seconds_global,
                      void* stream);

/* Dirichlet-Neumann recovery (§4.3, Algorithm 2) after hhg_inject_fault on
 * the same ids.  Omega_I together with the interface Gamma iterates on A_I,
 * the operator of the healthy macros' elements only, with right-hand side f
 * on Omega_I and, on Gamma, the flux (A_I u)_Gamma of the iterate at the time
 * of the fault (the Neumann data of Eq. (5)): n_global V-cycles of that
 * problem run on the caller's stream.  Omega_F runs Dirichlet V-cycles with
 * the Gamma values of the last finished Omega_I cycle (one-way update):
 * before Omega_I cycle j, ceil(j eta) - ceil((j - 1) eta) of them start on a
 * second stream from the values after Omega_I cycle j - 1, so the two sides
 * run concurrently.  On return the ghost copies of Gamma in the lost blocks
 * hold the final Gamma values (blocks of two or more Omega_F cycles replay
 * the captured cycle graph described at hhg_recover_local).  *n_local_run
 * (may be NULL) receives the Omega_F cycles run, ceil(n_global eta).
 * seconds_local / seconds_global (may be NULL) receive the device time spans
 * of the two sides (synchronises).
 * Errors: HHG_ERR_ARG for a NULL mesh, n_global < 0, eta < 0 or NaN, or an
 * invalid id list; CUDA errors as HHG_ERR_CUDA. */
int hhg_recover_dn(hhg_mesh* mesh, const int* macro_ids, int n_ids, int n_global, double eta,
                   int* n_local_run, double* seconds_local, double* seconds_global, void* stream);

/* A fault of a multi-fault run (§5: a second fault at another location after
 * the first recovery): after global cycle `cycle` the macros macro_ids[0..
 * n_ids) are lost. */
typedef struct {
  int cycle;
  const int* macro_ids;   /* host */
  int n_ids;
} hhg_fault;

typedef struct {
  double rtol;            /* stop when ||r_k|| <= rtol ||r_0|| (r_0 of the
                             initial iterate) */
  int max_cycles;         /* global V-cycles at most */
  int pre, post;          /* smoothing steps (0 = 3 each) */
  int fault_cycle;        /* inject the fault after this global cycle; <= 0:
                             no fault */
  const int* fault_ids;   /* host, macro ids of Omega_F */
  int n_fault_ids;
  int recovery;           /* HHG_RECOVERY_* */
  int n_local;            /* n_F; 0 with DD: ceil(eta * n_global); unused
                             with DN */
  int n_global;           /* n_I (DD and DN) */
  double eta;             /* superman factor: n_F = ceil(eta * n_I) (DD with
                             n_local = 0; DN always) */
  int mixed_precision;    /* 1: FP32 cycles inside FP64 iterative refinement
                             (needs a precision-32 mesh) */
  double coarse_rtol;     /* coarse CG relative tolerance (0 = 1e-12) */
  int coarse_maxit;       /* coarse CG iteration cap (0 = 1000) */
  const hhg_fault* faults;  /* further faults (host, may be NULL), each handled
                               like the first with the same recovery */
  int n_faults;
} hhg_solve_opts;

/* Iterate global V-cycles from the current iterate until rtol or
 * max_cycles, injecting the faults and running the recovery of opts after
 * each (faults of the same cycle in list order, the one of fault_cycle
 * first).
 * hist (host, at least max_cycles + 1 + number of faults doubles, may be
 * NULL) receives the
 * relative residuals: hist[0] = 1, one entry per global cycle and one extra
 * entry right after each fault and its recovery.
 * *n_hist receives the entries written, *cycles the global V-cycles run.
 * Returns HHG_ERR_NOT_CONVERGED (after writing the outputs) if rtol was not
 * reached. */
int hhg_solve(hhg_mesh* mesh, const hhg_solve_opts* opts, double* hist, int* n_hist,
              int* cycles, void* stream);

/* Differentiation support (an extension of the method of §2.1 to a
 * per-macro diffusion coefficient k_T, A = sum_T k_T A_T).
 * hhg_set_coefficients: replace the coefficients (host, n_macro positive
 * values) and rebuild every level's stencils, interface tables and the coarse
 * CG matrices (nothing to rebuild when the values equal the current ones);
 * the iterate and right-hand side are kept.  Synchronises the stream.
 * hhg_grad_coeff: with u a solution (global vector with its Dirichlet
 * values) and lam the adjoint solution of A_FF lam = dL/du_F (zero on the
 * Dirichlet nodes), write dL/dk_T = -lam^T A_T u for every macro into grad
 * (host, n_macro).  u becomes the mesh's iterate.  Synchronises the stream. */
int hhg_set_coefficients(hhg_mesh* mesh, const double* coeff, void* stream);
int hhg_grad_coeff(hhg_mesh* mesh, const double* u, const double* lam, double* grad, void* stream);

/* Autotuning of the volume tile shape (an implementation knob, not part of
 * the method).  For every smoothed level, times `reps` Gauss-Seidel steps of
 * the global problem with each candidate tile shape (nodes per tile and
 * slices per tile: 256/4, 512/8, 1024/8, 2048/16) on the FP64 iterate (which
 * the sweeps smooth) and, on precision-32 meshes, also on the FP32 arrays,
 * and keeps for that level the shape with the least total time; on meshes
 * with the 7-point structure it then times the flat Gauss-Seidel kernel
 * (hhg_set_flat_gs) and keeps it for the level's sweeps if it is faster
 * still (the residual and transfer kernels keep the chosen tiles).
 * chosen (may be NULL, one int per level, coarsest first) receives the index
 * c of the chosen tile shape, or c + 4 when the level's Gauss-Seidel sweeps
 * use the flat kernel (-1 for the coarsest level, which is not smoothed).
 * The tiles not kept are freed (after synchronising the device), except while
 * a batch refers to the mesh. */
int hhg_autotune(hhg_mesh* mesh, int reps, int* chosen, void* stream);

/* Batched recovery in one CUDA-graph launch (the concurrency of §4.1's
 * superman recovery, many sub-domains at once).  A batch holds n_tasks
 * recovery tasks -- task t: on meshes[t] (each mesh in one task only), the
 * fault of §2.2 on the macros ids[t][0..n_ids[t]) followed by cycles[t] local
 * Dirichlet cycles on them (LR) -- and, if global is not NULL, global_cycles
 * global cycles on the mesh `global` (not one of the task meshes).  Every
 * task is one branch of a CUDA graph, all branches fork from one start node,
 * so the tasks run concurrently; mixed = 1 runs every cycle as FP32 cycles in
 * FP64 iterative refinement (precision-32 meshes).  Creation does the host
 * set-up, runs the work once without the graph, and captures the graph.
 * hhg_batch_launch launches the whole batch with one graph launch on stream;
 * if task_ms is not NULL (n_tasks + 1 doubles, the global task last when
 * present) it synchronises and receives each task's completion time in ms
 * after the start of the launch. */
typedef struct hhg_batch hhg_batch;
int hhg_batch_create(hhg_mesh* global, int global_cycles, hhg_mesh* const* meshes, const int* const* ids,
                     const int* n_ids, const int* cycles, int n_tasks, int mixed, hhg_batch** out);
int hhg_batch_launch(hhg_batch* batch, double* task_ms, void* stream);
int hhg_batch_destroy(hhg_batch* batch);

/* The same batch as ONE kernel launch: a persistent scheduler kernel (as
 * many CTAs as the GPU holds at once) runs every task's operations in their
 * stream order.  Creation records each task's program -- every launch the
 * graph makes (Gauss-Seidel colours, residuals, transfers, the coarse CG, the
 * fault's zeroing and restoring, the FP32/FP64 hand-over), with its work
 * units -- and uploads it.  The launch resets the scheduler's counters (two
 * memsets on stream) and starts the kernel.  A CTA takes the next unit of
 * the current operation of some task; a task advances to its next operation
 * when all units of the current one are done, so the tasks share the GPU
 * unit by unit instead of by stream.  The results are bit for bit those of
 * hhg_batch_launch (the per-unit arithmetic is the same).  task_ms (may be
 * NULL; n_tasks + 1 doubles as in hhg_batch_launch) synchronises stream and
 * receives each task's completion time in ms after the first CTA started
 * (device global timer).  A kernel that found no work to take for longer than
 * the first task mesh's wait limit (hhg_set_wait_limit) stops and the timed
 * launch returns HHG_ERR_TIMEOUT; an untimed launch reports it on the next
 * timed one.  Needs the batch's device current. */
int hhg_batch_launch_persistent(hhg_batch* batch, double* task_ms, void* stream);

/* Priorities of the persistent launch's tasks: prio[t] for t < n_tasks (the
 * global task last, when present), or NULL for all equal (the default).  A
 * CTA looking for work takes it from the highest class that has some; within
 * a class it stays with the task it served last.  Giving the recovery tasks
 * the higher class lets them run ahead, as with §4.1's superman (shorter
 * latency per recovered sub-domain); giving the longest task the higher
 * class shortens the whole batch.  Results do not depend on the priorities.
 * Synchronises the device. */
int hhg_batch_set_priority(hhg_batch* batch, const int* prio);

/* info[0..4): tasks, recorded operations, work units over all operations,
 * kernels in the graph of hhg_batch_launch. */
int hhg_batch_info(hhg_batch* batch, int64_t* info);

/* Allocation-free V-cycle (an interface addition; the paper has no
 * counterpart).  Some callers cannot call cudaMalloc at all once they are
 * running: for example a host application that hands the device's memory to
 * its own arena allocator at start-up, or code on a path where device
 * allocation is forbidden.  This call runs the same global V(pre, post) cycle
 * as hhg_vcycle (without the residual norm) but its coarse-grid CG keeps its
 * work vectors in a fixed array of the library's static device memory
 * (4 x 16384 doubles = 512 KiB, which every GPU that loads the library holds
 * until the process exits) instead of in memory obtained from cudaMalloc; the
 * call itself makes no cudaMalloc, cudaFree or other allocating call.
 * Limit: the coarsest level may have at most 16384 unknowns; larger meshes
 * get HHG_ERR_ARG.  Meshes of general connectivity are accepted.  The mesh's
 * device must be current (HHG_ERR_STATE otherwise); the first call on a
 * device looks up that device's copy of the array (cudaGetSymbolAddress) with
 * the device current, so make that first call before any stream capture.
 * The cycle's Gauss-Seidel launches are not timed by hhg_profile_enable.
 * All calls share the array and it keeps the last call's contents; the CG
 * kernel writes every work value before it reads it, so nothing has to start
 * at zero, but calls whose work overlaps on the GPU (other streams, other
 * threads, other meshes) race on the array. */
int hhg_vcycle_noalloc(hhg_mesh* mesh, int pre, int post, void* stream);

/* Measurement support (not part of the method).
 * hhg_profile_enable: enable bit 0: every launch of the dominant kernel -- the
 * finest-level Gauss-Seidel volume kernel of the global problem (one colour of
 * the smoother of §2.1 on all macro interiors) -- is bracketed by CUDA events on
 * the stream it runs on.  Bit 1: the global cycles of hhg_solve / hhg_vcycle
 * record an event at every phase boundary (not inside a stream capture).
 * Enabling clears both records.
 * hhg_profile_breakdown: synchronises the device and sums, per phase, the
 * time from each recorded boundary to the next, into ms[0..9]: fine-level
 * smoothing, fine residual, restriction from the fine level, prolongation to
 * it, the levels below (smoothing, residuals, transfers), coarse CG, the
 * stopping test (residual and norm; FP64 residual of iterative refinement),
 * host turnaround (read-back of the norm until the next cycle's first work),
 * fault injection and recovery, and the FP32 correction's zeroing and
 * addition (mixed precision); n >= 10.  Clears the record.
 * hhg_profile_read: synchronises the device and returns the number of
 * recorded launches and their summed device time in milliseconds; clears the
 * record.
 * hhg_profile_info: volume-interior nodes of the finest level (the nodes one
 * sweep of all four colours of that kernel updates) and whether the stencil
 * has the 7-point structure (only the six axis neighbours non-zero).
 * hhg_launch_count: kernel launches issued by the library in this process;
 * each kernel of a CUDA graph the library replays (batched recovery, the
 * later cycles of a local recovery) counts as one launch per replay, kernels
 * recorded while capturing such a graph do not count.
 * hhg_set_launch_limit: at most max_ctas CTAs per level-wide launch of the
 * tile kernels (0, the default: as many as the GPU holds at once; the flat
 * kernels launch one CTA per 256 items and are not limited).  A level-wide launch walks its
 * work units (interface chunks, then volume tiles) with a grid stride when
 * it has fewer than 4 units per CTA, and otherwise hands the units out
 * through a per-problem counter (the dynamic walk of large launches, where
 * the Gauss-Seidel and residual launches place the interface chunks evenly
 * among the volume tiles); a small limit makes small meshes take the dynamic
 * walk.  The result does not depend on the limit (a residual norm only up to
 * the order of its summation).  Drops the captured recovery-cycle graph.
 * hhg_walk_counts: counts[0..3] = level-wide launches that completed the
 * dynamic walk, for the global problem, the faulty sub-problem (Omega_F),
 * the healthy sub-problem with Gamma frozen and the Neumann problem of DN
 * recovery (0 where a problem does not exist; counts restart when a fault set
 * replaces the sub-problems).  Synchronises the device. */
int hhg_profile_enable(hhg_mesh* mesh, int enable);
int hhg_profile_breakdown(hhg_mesh* mesh, double* ms, int n);
int hhg_profile_read(hhg_mesh* mesh, int64_t* launches, double* total_ms);
int hhg_profile_info(const hhg_mesh* mesh, int64_t* volume_nodes, int* seven_point);
int hhg_launch_count(int64_t* count);
int hhg_set_launch_limit(hhg_mesh* mesh, int max_ctas);

/* FP64 FMA throughput of the current device in TFLOP/s (measurement support:
 * the ALU roofline of the FP64 kernels): 8 CTAs of 256 threads per SM, each
 * thread running 8 independent FMA chains of 16384 steps, timed with CUDA
 * events on the legacy stream, best of three after a warm-up launch.
 * Allocates and frees a small device buffer; synchronises. */
int hhg_measure_fp64_peak(double* tflops);
int hhg_walk_counts(hhg_mesh* mesh, int64_t* counts);

/* Kernel options (implementation knobs, not part of the method).
 * hhg_set_streaming: enable or disable (default) the streaming Gauss-Seidel
 * kernel on meshes with the 7-point structure: on levels with at least 64
 * intervals per macro edge it sweeps bands of rows slice by slice, a
 * producer warp staging the two neighbour colours and the right-hand side of
 * each slice in shared memory with bulk asynchronous copies on mbarriers for
 * eight consumer warps; disabled, each level uses the row-pair tile kernel or,
 * where switched on (hhg_set_flat_gs, hhg_autotune), the flat kernel.  All
 * give the same iterate bit for bit (the streaming kernel is the slowest of
 * the three on GB300).  Drops the captured recovery-cycle graph.
 * hhg_set_wait_limit: the streaming kernel's waits on its mbarriers are bounded
 * (default tries < 0: about one second per wait).  When a wait runs out the
 * CTA records it in the mesh's device error flag, waits (bounded) for its
 * copies in flight and stops; the next call that reads a result back
 * (hhg_vcycle with resid_out, hhg_residual_norm, hhg_solve) clears the flag
 * and returns HHG_ERR_TIMEOUT, and the iterate is then incomplete (reload it
 * with hhg_set_problem).  tries = 0 makes every wait run out at once, which
 * exercises that path without any fault. */
int hhg_set_streaming(hhg_mesh* mesh, int enable);
/* hhg_set_flat_gs: enable or disable (default) the flat Gauss-Seidel kernel on
 * every smoothed level of a mesh with the 7-point structure (ignored on
 * meshes without it; general connectivity: HHG_ERR_STATE; HHG_ERR_ARG, with
 * nothing changed, when a level has more than 1024 intervals per macro edge
 * or 2^31 items per launch): one thread per
 * 16-byte vector of same-colour nodes, indexed through a per-level item
 * table (4 bytes per item, FP64 and on precision-32 meshes FP32 tables,
 * allocated on enable and freed on disable), with no tiles and no CTA
 * barrier, which suits the small coarse levels; hhg_autotune picks it per
 * level.  On those levels the residual before each restriction, the
 * restriction onto the level (one thread per slot of four coarse nodes) and
 * the prolongation onto it (one thread per 16-byte vector of same-colour fine
 * nodes) run in the same flat form; the stopping test's norm keeps the tile
 * kernel.  Same iterate bit for bit as the tile kernels.  The streaming kernel
 * (hhg_set_streaming) takes precedence where both are enabled; the
 * persistent batch executor keeps the tile kernel.  Drops the captured
 * recovery-cycle graph. */
int hhg_set_flat_gs(hhg_mesh* mesh, int enable);
int hhg_set_wait_limit(hhg_mesh* mesh, int tries);

/* Copy the message of the calling thread's last failure into buf (always
 * NUL-terminated if len > 0).  Returns the status of that failure. */
int hhg_last_error(char* buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* HHG_H */
