// Internal structures of the HHG library: the blocked per-macro layout, the
// interface (face / edge / vertex) containers, per-problem work lists, and the
// declarations shared by the host mesh builder and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

namespace hhg {

// Kernel launches issued by the library (all meshes, all streams).
extern std::atomic<long long> g_kernel_launches;

// ---------------------------------------------------------------------------
// 15-point stencil directions in a macro-tetrahedron's local lattice.
//
// Local node (i, j, k), i, j, k >= 0, i + j + k <= N, sits at
// V0 + (i (V1 - V0) + j (V2 - V0) + k (V3 - V0)) / N.  In "chain" coordinates
// (a, b, c) = (i + j + k, j + k, k) the macro is the Kuhn simplex
// N >= a >= b >= c >= 0 and its uniform (Bey) refinement is the Freudenthal
// triangulation of the chain lattice, whose edges are the 7 non-zero 0/1
// chain vectors.  Index 0 is the centre, 1..7 those chain vectors mapped to
// (di, dj, dk) = (da - db, db - dc, dc), 8..14 their negatives.
// ---------------------------------------------------------------------------
constexpr int NDIR = 15;

__host__ __device__ __forceinline__ void dir_ijk(int d, int& di, int& dj, int& dk) {
  // chain (1,0,0) (0,1,0) (0,0,1) (1,1,0) (0,1,1) (1,0,1) (1,1,1)
  int s = 1;
  if (d > 7) { s = -1; d -= 7; }
  switch (d) {
    case 1: di = 1;  dj = 0;  dk = 0; break;
    case 2: di = -1; dj = 1;  dk = 0; break;
    case 3: di = 0;  dj = -1; dk = 1; break;
    case 4: di = 0;  dj = 1;  dk = 0; break;
    case 5: di = -1; dj = 0;  dk = 1; break;
    case 6: di = 1;  dj = -1; dk = 1; break;
    case 7: di = 0;  dj = 0;  dk = 1; break;
    default: di = 0; dj = 0; dk = 0; s = 1; break;
  }
  di *= s; dj *= s; dk *= s;
}

// Node class of a local lattice node: bit 0: k == 0, bit 1: j == 0,
// bit 2: i == 0, bit 3: i + j + k == N (the four faces of the macro).
// 0 = volume interior, one bit = face, two = edge, three = vertex.
__host__ __device__ __forceinline__ int node_class(int i, int j, int k, int N) {
  return (k == 0) | ((j == 0) << 1) | ((i == 0) << 2) | ((i + j + k == N) << 3);
}

__host__ __device__ __forceinline__ bool in_lattice(int i, int j, int k, int N) {
  return i >= 0 && j >= 0 && k >= 0 && i + j + k <= N;
}

// ---------------------------------------------------------------------------
// Blocked colour-split layout of one macro's closed lattice at refinement N.
// The colour of node (i, j, k) is (i + 2j + 3k) mod 4, equal to (x + y + z)
// mod 4 of its global grid coordinates.  A block holds four colour arrays of
// CS slots each (block = 4 CS).  Inside each colour array the rows (j, k)
// follow each other (k major); row (j, k) has L = N + 1 - j - k nodes, node i
// sitting in slot i >> 2 of the row of its colour, and the row gets
// 4 ceil(L / 16) slots: a multiple of four, so that every row starts on a
// 16-byte boundary (FP32) and consecutive same-colour nodes of a row can be
// moved as one vector.  With S(m) = sum_{l=1..m} 4 ceil(l / 16)
// = 4 (a + 1)(8a + b) for m = 16a + b, the rows of slice k before row j take
// S(M) - S(M - j) slots (M = N + 1 - k), and the per-level table
// SL[k] = sum_{k' < k} S(N + 1 - k') gives the slice starts:
//   offset(i, j, k) = c CS + SL[k] + S(M) - S(M - j) + (i >> 2).
// The arrays are dense up to at most 3 idle slots per row plus the padding
// to four, and a sweep of one colour streams exactly the arrays it reads and
// writes.  SL has N + 3 entries; SL[N + 2] holds CS.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int slot_prefix(int m) {
  const int a = m >> 4, b = m & 15;
  return 4 * (a + 1) * (8 * a + b);
}

// Slots of a row of L nodes (one colour).
__host__ __device__ __forceinline__ int row_slots(int L) { return 4 * ((L + 15) >> 4); }

__host__ __device__ __forceinline__ int lidx(const int* SL, int N, int i, int j, int k) {
  const int M = N + 1 - k;
  return ((i + 2 * j + 3 * k) & 3) * SL[N + 2] + SL[k] + slot_prefix(M) - slot_prefix(M - j) + (i >> 2);
}

// Walk position u of a launch with n_if interface chunks and n_vol volume
// units, chunks spread evenly among the volume units: one chunk after every
// R = n_vol / n_if volume units (chunks left over when n_vol < n_if follow,
// then the remaining volume units).  Returns the chunk index, or -1 with the
// volume unit's index in vol.  A bijection of [0, n_if + n_vol) onto the
// chunks and the volume units, both in their own order.
__host__ __device__ __forceinline__ int spread_position(int u, int n_if, int n_vol, int& vol) {
  if (n_if == 0) {
    vol = u;
    return -1;
  }
  const int R = n_vol / n_if > 1 ? n_vol / n_if : 1;
  const int m = n_if < n_vol / R ? n_if : n_vol / R;   // chunks placed among the volume units
  const int span = m * (R + 1);
  if (u < span) {
    const int q = u / (R + 1), r = u - q * (R + 1);
    if (r == R) return q;
    vol = q * R + r;
    return -1;
  }
  u -= span;
  if (u < n_if - m) return m + u;
  vol = m * R + (u - (n_if - m));
  return -1;
}

// Slice-start table (N + 3 entries, last = CS) and block size (4 CS, CS a
// multiple of 64) of refinement N.
inline int64_t build_slice_starts(int N, std::vector<int>& SL) {
  SL.assign((size_t)N + 3, 0);
  int64_t off = 0;
  for (int k = 0; k <= N + 1; ++k) {
    SL[k] = (int)off;
    if (k <= N) off += slot_prefix(N + 1 - k);
  }
  const int64_t cs = (off + 63) & ~int64_t(63);
  SL[N + 2] = (int)cs;
  return 4 * cs;
}

// Work tile of the volume kernels.  Interior tiles: slices k .. k + pad - 1,
// row pairs j0 .. j0 + m0 - 1 (see build_pair_tiles).  Closed-lattice tiles:
// 8 rows (j0..j0+7) x 32 slots (m0..m0+31) of slice k.
struct Tile {
  int k, j0, m0, pad;
};
constexpr int TILE_ROWS = 8;
constexpr int TILE_SLABS = 8;
constexpr int TILE_TARGET_DEFAULT = 512;
constexpr int TILE_SLOTS = 32;

// Work unit of the streaming Gauss-Seidel kernel (7-point structure): the
// interior rows j0..j1 of slices ka..kb of one macro, swept slice by slice
// with the neighbour colours staged in shared memory (kernels.cu).
struct StreamTile {
  int j0, j1, ka, kb;
};
constexpr int STREAM_BAND = 16;      // rows per band of the FP64 units (8 from 512 intervals on)
constexpr int STREAM_BAND32 = 32;    // rows per band of the FP32 units (16 from 512 intervals on)
constexpr int STREAM_SLICES = 16;    // slices per unit at most
constexpr int STREAM_MIN_N = 64;     // levels with at least this many intervals stream

// A copy of an interface node inside one macro block.
struct Copy {
  int macro, i, j, k;
};

// Macro geometry used by device kernels: global fine coordinates of local
// node (i, j, k) at refinement N are N * v0 + i * e1 + j * e2 + k * e3.
struct MacroGeo {
  int v0[3], e1[3], e2[3], e3[3];
};

// ---------------------------------------------------------------------------
// Host-side mesh description (built by mesh.cpp).
// ---------------------------------------------------------------------------
struct HostLevel {
  int r = 0, N = 0;
  int64_t block = 0;
  std::vector<int> SL;                // slice-start table of the block layout
  int n_if = 0;
  std::vector<int64_t> if_gid;        // global id of each interface node (grid id
                                      // on the cube family; general meshes: its
                                      // rank, interface nodes coming first)
  std::vector<int> if_cptr;           // copies CSR
  std::vector<Copy> if_copy;
  std::vector<unsigned char> if_colour, if_dirichlet;   // general meshes: if_colour
                                      // holds the interface smoother class
  int n_if_classes = 0;               // general meshes: number of interface classes
  std::vector<double> W;              // [n_macro][16][15] stencil weights
  std::vector<Tile> tiles_int;        // row-pair tiles of the volume interior
  std::vector<Tile> tiles_all;        // tiles covering the closed lattice
  std::vector<StreamTile> tiles_stream;  // streaming units (N >= STREAM_MIN_N), FP64 cycles
  int stream_band = 0;                // their rows per band
  std::vector<StreamTile> tiles_stream32;  // the same for the FP32 cycles (wider bands)
  int stream_band32 = 0;
};

struct HostMesh {
  int sub[3] = {0, 0, 0};
  int R = 0, r0 = 2;
  int n_macro = 0;
  int64_t nx = 0, ny = 0, nz = 0;     // finest-level intervals per axis
  std::vector<MacroGeo> geo;
  std::vector<double> coeff;
  double G[9];
  // General connectivity (build_general_mesh): the four vertex ids of every
  // macro, positions in vpos; global node order = interface nodes by key,
  // then the volume nodes macro by macro in local (k, j, i) order.
  bool general = false;
  std::vector<std::array<int, 4>> mverts;
  // Physical positions of the sub-cube corners ((sx+1)(sy+1)(sz+1) x 3, x
  // fastest); empty = the corners of the unit cube mapped by G.  With moved
  // corners every macro is a general tetrahedron, refined through its own
  // affine map.
  std::vector<double> vpos;
  std::vector<HostLevel> lv;          // index 0 = coarsest (r0)
  std::vector<std::vector<int>> node_macros;   // not used on device
  bool seven_point = false;           // all volume stencils have only the 6
                                      // chain-axis neighbours non-zero
};

// Problem: which nodes are unknowns.  kind 0 = global, 1 = faulty sub-domain,
// 2 = healthy sub-domain (interface frozen), 3 = healthy sub-domain with the
// interface free and only the healthy macros' elements in the operator (A_I,
// the Neumann side of Dirichlet-Neumann recovery, §4.3 Algorithm 2).
struct HostProblemLevel {
  std::vector<int> free_if;           // free interface nodes grouped by colour
  int col_off[5] = {0, 0, 0, 0, 0};
  std::vector<int64_t> zero_off;      // frozen copies in active blocks
  std::vector<int64_t> gather;        // [free_if.size()][15] fine offsets of the
                                      // restriction onto this level (-1 = none)
  // Interface copies restricted to the active macros (kind 3 only; empty
  // otherwise, where every copy of a free node is active): CSR over all
  // interface nodes of the level.
  std::vector<int> cptr;
  std::vector<Copy> copies;
  // General meshes: free_if grouped by interface class (class_off, one entry
  // per class + 1; col_off then only holds the total in col_off[4]) and the
  // restriction gathers as CSR (gptr over free_if, block offsets goff of the
  // distinct fine nodes, the coarse node itself first with weight 1, the
  // others weight 1/2) instead of the 15-entry rows of gather.
  std::vector<int> class_off;
  std::vector<int> gptr;
  std::vector<int64_t> goff;
};

struct HostProblem {
  int kind = 0;
  std::vector<int> act;               // active macros
  std::vector<unsigned char> macro_active;
  std::vector<HostProblemLevel> lv;
  // coarse CG (level 0): compact free nodes
  int n_cg = 0;
  std::vector<int> rowptr, col;
  std::vector<double> val;
  std::vector<int64_t> fsrc;          // >= 0: block offset of f; < 0: -1 - master
  std::vector<int> uptr;              // scatter CSR
  std::vector<int64_t> udst;          // block offsets to write
  std::vector<int> umaster;           // master index or -1
};

void build_host_mesh(HostMesh& m, const int sub[3], int R, int r0, const double* coeff,
                     const double* affine, const double* vertex_pos = nullptr);
// open: all adjacent macros faulty (and not Dirichlet); closed: any faulty.
void build_problem(const HostMesh& m, int kind, const std::vector<unsigned char>& faulty,
                   HostProblem& p);
bool macro_in_set(const std::vector<unsigned char>& s, int m);
// Interior row-pair tiles of refinement N (see mesh.cpp).
void build_pair_tiles(int N, std::vector<Tile>& out, int target, int slabs);
// Streaming units of refinement N: bands of `band` interior rows, each split
// into runs of at most `slices` slices, largest first.
void build_stream_tiles(int N, int band, int slices, std::vector<StreamTile>& out);
// Work items of the flat Gauss-Seidel kernel on refinement N (N <= 1024) for
// vectors of vw same-colour slots: for each colour c, the groups g of every
// interior row (j, k) of one macro holding colour-c nodes, packed as
// (j << 20) | (k << 10) | g, slice by slice, row by row, group by group;
// colour c's items are items[off[c] .. off[c + 1]).
void build_gs_items(int N, int vw, std::vector<uint32_t>& items, int off[5]);
// Slots of four consecutive nodes (one per colour array) of every interior
// row (j, k) of one macro, m = 0 .. (N - 1 - j - k) >> 2, packed as
// (j << 20) | (k << 10) | m, slice by slice, row by row: the flat
// restriction's items on the coarse level.
void build_slot_items(int N, std::vector<uint32_t>& items);
// Recompute every level's stencils for new per-macro coefficients.
void set_coefficients(HostMesh& m, const double* coeff);
// A macro mesh of general connectivity: nv vertex positions (3 doubles each),
// nt macros (4 vertex ids each, any order), refinement levels r0..R, one
// coefficient per macro (NULL = ones).  Throws std::invalid_argument for a
// degenerate macro, an id out of range or a face shared by more than two
// macros.
void build_general_mesh(HostMesh& m, const double* verts, int nv, const int* tets, int nt, int R, int r0,
                        const double* coeff);
// A problem of a general mesh (kinds as for build_problem: 0 global, 1
// faulty sub-domain, 2 healthy with the interface frozen, 3 healthy with the
// interface free under A_I): free interface nodes by class, frozen copies,
// variable-length restriction gathers, coarse CSR.
void build_general_problem(const HostMesh& m, int kind, const std::vector<unsigned char>& faulty,
                           HostProblem& p);
// Global id of the volume node (i, j, k) (all positive, i + j + k < N) of a
// macro of a general mesh at level L: n_if + macro * (N-1)(N-2)(N-3)/6 + its
// index in the local (k, j, i) order.
int64_t general_volume_id(const HostLevel& L, int macro, int i, int j, int k);
// (Re)assemble a problem's coarse-level CG system from the current stencils
// (needs p.act, p.macro_active and p.lv[0].free_if).
void assemble_coarse(const HostMesh& m, HostProblem& p);

// Block offsets (macro * block + local offset) of the copies of level l,
// or of a given copy list; false if an offset does not fit 32 bits.
bool copy_offsets(const HostMesh& m, int l, const std::vector<Copy>& copies, std::vector<uint32_t>& out);

// Interface stencil tables of one problem level of a cube-family mesh.  For
// the interface nodes free_if[q] (in that order) the stencil - the sum of the
// sub-stencils of the node's copies listed in cptr / copies (§3.2, Fig. 4) -
// is stored per distinct neighbour: its summed weight w and the block offset
// nb of a copy of it inside the block of a macro whose sub-stencil reaches
// it, K entries per node direction-major (entry e of node q at e * n + q,
// n = free_if.size()), padded with weight 0 and the node's own first copy;
// diag[q] is the summed centre weight.  Returns false (tables empty) for
// general connectivity, for a node with more than K neighbours or for an
// offset beyond 32 bits.
bool build_if_tables(const HostMesh& m, int l, const std::vector<int>& free_if, const std::vector<int>& cptr,
                     const std::vector<Copy>& copies, int K, std::vector<uint32_t>& nb, std::vector<double>& w,
                     std::vector<double>& diag);

// ---------------------------------------------------------------------------
// Device-side structures.
// ---------------------------------------------------------------------------
template <class T>
struct DevLevel {
  int N = 0;
  int64_t block = 0;
  int n_if = 0;
  T* u = nullptr;   // blocks [n_macro * block]
  T* f = nullptr;
  T* r = nullptr;
  T* uI = nullptr;  // interface masters [n_if]
  T* fI = nullptr;
  T* W = nullptr;   // [n_macro][16][15]
};

struct DevLevelTables {
  int* SL = nullptr;                  // slice-start table of the block layout
  int64_t* if_gid = nullptr;
  int* if_cptr = nullptr;
  Copy* if_copy = nullptr;
  uint32_t* cp_off = nullptr;         // block offset of every copy (null: computed from if_copy)
  Tile* tiles_int = nullptr;
  int n_tiles_int = 0;
  Tile* tiles_all = nullptr;
  int n_tiles_all = 0;
  StreamTile* tiles_stream = nullptr;
  int n_tiles_stream = 0;
  StreamTile* tiles_stream32 = nullptr;
  int n_tiles_stream32 = 0;
  // flat Gauss-Seidel (7-point levels, on request): build_gs_items for FP64
  // (2 slots per item) and FP32 (4), and whether the level uses it
  uint32_t* gs_items64 = nullptr;
  int gs_off64[5] = {0, 0, 0, 0, 0};
  uint32_t* gs_items32 = nullptr;
  int gs_off32[5] = {0, 0, 0, 0, 0};
  uint32_t* slot_items = nullptr;    // build_slot_items
  int n_slots = 0;
  int gs_flat = 0;
};

struct DevProblemLevel {
  int* gptr = nullptr;                // general meshes: restriction gathers (CSR)
  int64_t* goff = nullptr;
  std::vector<int> class_off;         // general meshes: interface classes in free_if
  int* free_if = nullptr;
  int col_off[5] = {0, 0, 0, 0, 0};
  int64_t* zero_off = nullptr;
  int n_zero = 0;
  int64_t* gather = nullptr;
  int* cptr = nullptr;                // active copies (kind 3), else null
  Copy* cps = nullptr;
  uint32_t* cp_off = nullptr;         // block offsets of those copies (kind 3)
  // interface stencil tables of the free interface nodes (build_if_tables;
  // null for general meshes and on level 0): tK entries per node,
  // direction-major with stride tn = free_if size; weights, diagonal and its
  // inverse in both precisions (FP32 only on precision-32 meshes)
  uint32_t* tnb = nullptr;
  double* tw64 = nullptr;
  double* td64 = nullptr;
  double* ti64 = nullptr;
  float* tw32 = nullptr;
  float* td32 = nullptr;
  float* ti32 = nullptr;
  int tn = 0;
};

struct DevProblem {
  int kind = 0;
  int* sched = nullptr;               // counters of the dynamic walks (kernels.cu): next unit,
                                      // finished CTAs, completed dynamic launches
  int grid_cap = 0;                   // CTAs per fused launch at most (0: resident CTAs)
  int stream_gs = 0;                  // streaming 7-point Gauss-Seidel where a level has units
  int* err = nullptr;                 // the mesh's device error flag (bounded waits)
  int wait_limit = 1 << 24;           // tries of a bounded device wait
  int* act = nullptr;
  int n_act = 0;
  std::vector<int> act_host;
  std::vector<unsigned char> macro_active_host;
  std::vector<int> free0_host;        // free interface nodes of level 0
  std::vector<std::vector<int>> free_host;  // free interface nodes of every level
                                      // (rebuilding the interface tables for new
                                      // coefficients)
  std::vector<DevProblemLevel> lv;
  int n_cg = 0;
  int64_t nnz = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* val = nullptr;
  int64_t* fsrc = nullptr;
  int* uptr = nullptr;
  int64_t* udst = nullptr;
  int* umaster = nullptr;
  double* cg_work = nullptr;        // 4 * n_cg scratch
  double* partial = nullptr;        // per-CTA partial sums of the norm
  int n_partial = 0;
  double* scalar = nullptr;         // [4]: norm^2 result, cg info
  int* cg_iters = nullptr;
  double* fI_top = nullptr;         // finest-level FP64 interface right-hand
                                    // side replacing the mesh's (kind 3)
  cudaStream_t stream = nullptr;    // stream owned by the problem (DD half)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

}  // namespace hhg
