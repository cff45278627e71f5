// CUDA kernels of the HHG multigrid for sm_103a.
//
// Every level-wide operation is one launch of 256-thread CTAs (32 x 8), as many
// as the GPU holds at once, walking a list of work units: chunks of free
// interface (face / edge / vertex) nodes, one node per thread, and row-pair
// tiles of the volume interiors of the active macros (the chunks first, or in
// large stencil launches spread evenly among the tiles).
//
// Volume work: in slice k of a macro's lattice the interior rows are
// j = 1..J (J = N - 2 - k) and row j holds N - 1 - j - k nodes.  Rows are
// paired as (1 + p, J - p), whose lengths add up to N - 1 - k, and a tile
// holds enough pairs for about 512 nodes of one colour in 8 consecutive
// slices; per slice the CTA flattens the nodes (or 4-node slots) of all its
// pairs into one index range, so lanes stay busy although the rows shrink
// across the triangle, and the rows it loads for one slice are still in L1
// when it processes the next.  On GB300 the FP64 pipe
// retires 2 DFMA per clock per SM and is charged per warp instruction, so
// idle lanes cost as much as busy ones.  Consecutive lanes read consecutive
// slots of one colour segment, so stencil neighbours are contiguous accesses.
//
// Flat kernels (k_gs_flat, k_res_flat, k_restrict_flat, k_prolong_flat; the
// autotuner's choice per level on meshes with the 7-point structure): no
// tiles, one work item per thread from a per-level table (a 16-byte vector of
// same-colour slots, or a slot of four nodes), one CTA per 256 items, so a
// launch has no CTA barrier and no CTA walking a long tile; the per-item
// arithmetic is the tile kernels', hence the same results bit for bit.
//
// Interface work: a node's stencil is the sum of the sub-stencils of the
// macros around it (§3.2, Fig. 4); the kernel updates the master in the
// interface container and writes the value into the ghost shell of every
// adjacent block (the local half of the ghost update of §3.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <map>
#include <mutex>
#include <utility>

#include "hhg_kernels.h"

namespace hhg {

std::atomic<long long> g_kernel_launches{0};

namespace {

constexpr int CTA = TILE_ROWS * TILE_SLOTS;   // 256 threads, 32 x 8

// 7-point structure: only the three chain axes (and negatives) are non-zero.
__host__ __device__ constexpr bool used_dir(int d, bool s7) {
  return !s7 || d == 1 || d == 2 || d == 3 || d == 8 || d == 9 || d == 10;
}

// Offset of node (i, j, k) inside a macro block (32-bit: a block holds fewer
// than 2^31 nodes for N <= 1024); rs is the level's slice-start table.
__device__ __forceinline__ int lidx32(const int* __restrict__ rs, int N, int i, int j, int k) {
  const int M = N + 1 - k;
  return ((i + 2 * j + 3 * k) & 3) * __ldg(rs + N + 2) + __ldg(rs + k) + slot_prefix(M) - slot_prefix(M - j) +
         (i >> 2);
}

// Base slot of row j of slice k of a level (colour array 0).
__device__ __forceinline__ int row_base(const int* __restrict__ rs, int N, int j, int k) {
  const int M = N + 1 - k;
  return __ldg(rs + k) + slot_prefix(M) - slot_prefix(M - j);
}

// Offsets of the 7-point neighbourhood of node (i, j, k), colour c, in one
// go: the five rows involved are derived from a single slot_prefix(M - j).
// nb[d] for d in {1, 2, 3, 8, 9, 10}; me = the node itself.
struct Slice {
  int N, k, M, CS, SLm, SL0, SLp, SMm, SM0, SMp;
};
__device__ __forceinline__ Slice slice_consts(const int* __restrict__ rs, int N, int k) {
  Slice s;
  s.N = N;
  s.k = k;
  s.M = N + 1 - k;
  s.CS = __ldg(rs + N + 2);
  s.SLm = k > 0 ? __ldg(rs + k - 1) : 0;
  s.SL0 = __ldg(rs + k);
  s.SLp = __ldg(rs + k + 1);
  s.SMm = slot_prefix(s.M - 1);
  s.SM0 = slot_prefix(s.M);
  s.SMp = slot_prefix(s.M + 1);
  return s;
}
struct Nb7 {
  int me, nb1, nb8, nb2, nb9, nb3, nb10;
};
__device__ __forceinline__ Nb7 nb7(const Slice& s, int i, int j) {
  const int X = slot_prefix(s.M - j);
  const int L = s.M - j;
  const int r0 = s.SL0 + s.SM0 - X;           // row (j, k)
  const int rjp = r0 + row_slots(L);          // row (j + 1, k)
  const int rjm = r0 - row_slots(L + 1);      // row (j - 1, k)
  const int rkp = s.SLp + s.SMm - X;          // row (j - 1, k + 1)
  const int rkm = s.SLm + s.SMp - X;          // row (j + 1, k - 1)
  const int c = (i + 2 * j + 3 * s.k) & 3;
  const int cp = ((c + 1) & 3) * s.CS, cm = ((c + 3) & 3) * s.CS;
  Nb7 n;
  n.me = c * s.CS + r0 + (i >> 2);
  n.nb1 = cp + r0 + ((i + 1) >> 2);           // ( 1,  0, 0)
  n.nb8 = cm + r0 + ((i - 1) >> 2);           // (-1,  0, 0)
  n.nb2 = cp + rjp + ((i - 1) >> 2);          // (-1,  1, 0)
  n.nb9 = cm + rjm + ((i + 1) >> 2);          // ( 1, -1, 0)
  n.nb3 = cp + rkp + (i >> 2);                // ( 0, -1, 1)
  n.nb10 = cm + rkm + (i >> 2);               // ( 0,  1, -1)
  return n;
}

__device__ __forceinline__ int tid256() { return threadIdx.y * TILE_SLOTS + threadIdx.x; }

// Sum over the CTA (any shape up to 1024 threads); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthreads = blockDim.x * blockDim.y;
  __syncthreads();
  if ((lane & 31) == 0) sh[lane >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (lane < 32) {
    s = (lane < (nthreads + 31) / 32) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

// Colour-c nodes of interior row j of slice k: slots m = mlo .. mlo + n - 1
// (i = 4m + ic, 1 <= i <= N - 1 - j - k).
__device__ __forceinline__ void colour_row(int N, int j, int k, int c, int& ic, int& mlo, int& n) {
  ic = (c - 2 * j - 3 * k) & 3;
  const int L = N - 1 - j - k;
  mlo = ic == 0;
  n = L >= ic ? ((L - ic) >> 2) - mlo + 1 : 0;
}

// Work items of interior row j: its colour-c nodes (colour kernels; with
// vw > 1 its groups of vw consecutive slots holding them, slots vw g .. vw g
// + vw - 1) or its slots of four consecutive nodes (all-colour kernels).
__device__ __forceinline__ int row_items(int N, int j, int k, int c, bool colour, int vw = 1) {
  if (colour) {
    int ic, mlo, n;
    colour_row(N, j, k, c, ic, mlo, n);
    if (vw == 1) return n;
    return n > 0 ? (mlo + n - 1) / vw + 1 : 0;
  }
  return ((N - 1 - j - k) >> 2) + 1;
}

// An interior tile holds row pairs p = t.j0 .. t.j0 + t.m0 - 1 of slices t.k ..
// t.k + t.pad - 1, pair p being rows 1 + p and J - p of a slice (J = N - 2 -
// k).  The CTA flattens the items of all its pairs and slices into one range
// so that every lane has work: s_pre[s][q] = items of pairs t.j0 .. t.j0 + q -
// 1 in slice t.k + s (one warp per slice computes it with a warp scan), and
// s_tot[s] the items of slices t.k .. t.k + s - 1.  One CTA barrier for the
// whole tile, so that the threads stream through the items of all its slices
// without waiting for each other.  Returns the tile's item count.  All
// threads must call it.
constexpr int MAX_SLABS = 16;
__device__ __forceinline__ int flat_setup_slabs(const Tile& t, int N, int c, bool colour, int vw,
                                                int (*s_pre)[33], int* s_tot) {
  const int J0 = N - 2;
  for (int sl = threadIdx.y; sl < t.pad; sl += TILE_ROWS) {
    const int k = t.k + sl, J = J0 - k;
    const int q = threadIdx.x;
    int len = 0;
    if (q < t.m0) {
      const int j1 = 1 + t.j0 + q, j2 = J - t.j0 - q;
      if (j1 <= j2) {
        len = row_items(N, j1, k, c, colour, vw);
        if (j2 > j1) len += row_items(N, j2, k, c, colour, vw);
      }
    }
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, len, o);
      if (q >= o) len += y;
    }
    s_pre[sl][q + 1] = len;
    if (q == 0) s_pre[sl][0] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int acc = 0;
    for (int sl = 0; sl < t.pad; ++sl) {
      s_tot[sl] = acc;
      acc += s_pre[sl][t.m0];
    }
    s_tot[t.pad] = acc;
  }
  __syncthreads();
  return s_tot[t.pad];
}

// Item tt of a flattened tile -> its row j and index v within the row.
__device__ __forceinline__ void flat_item(const Tile& t, int N, int c, bool colour, const int* s_pre, int tt, int& j,
                                          int& v, int vw = 1) {
  int lo = 0, hi = t.m0;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (s_pre[mid] <= tt) lo = mid;
    else hi = mid;
  }
  const int j1 = 1 + t.j0 + lo;
  const int w = tt - s_pre[lo];
  const int n1 = row_items(N, j1, t.k, c, colour, vw);
  if (w < n1) {
    j = j1;
    v = w;
  } else {
    j = N - 2 - t.k - t.j0 - lo;
    v = w - n1;
  }
}

// Loop over the interior nodes of a tile, four consecutive nodes
// i = 4m .. 4m + 3 (one per colour array) per item, the items of all the
// tile's slices in one range (one CTA barrier per tile); the body sees i, j, k
// and the slice constants sc of the iterated level.  The kernel declares
// s_pre2[MAX_SLABS][33] and s_pre_tot[MAX_SLABS + 1] in shared memory.
#define HHG_TILE_NODES(NN, RS, t, s_pre, ...)                                        \
  {                                                                                  \
    const int total_ = flat_setup_slabs((t), (NN), 0, false, 1, s_pre##2, s_pre##_tot); \
    int sl_ = 0;                                                                     \
    for (int tt = tid256(); tt < total_; tt += CTA) {                                \
      while (tt >= s_pre##_tot[sl_ + 1]) ++sl_;                                      \
      const int k = (t).k + sl_;                                                     \
      const Tile ts_{k, (t).j0, (t).m0, 1};                                          \
      int j, m;                                                                      \
      flat_item(ts_, (NN), 0, false, s_pre##2[sl_], tt - s_pre##_tot[sl_], j, m);    \
      const Slice sc = slice_consts((RS), (NN), k);                                  \
      (void)sc;                                                                      \
      const int L = (NN) - 1 - j - k;                                                \
      _Pragma("unroll") for (int qq = 0; qq < 4; ++qq) {                             \
        const int i = 4 * m + qq;                                                    \
        if (i < 1 || i > L) continue;                                                \
        __VA_ARGS__                                                                  \
      }                                                                              \
    }                                                                                \
    __syncthreads();                                                                 \
  }

// Work units of a fused launch: units [0, n_if_units) are chunks of 256
// interface list entries, the rest (tile, active macro) pairs (large stencil
// launches map walk positions to units through spread_unit instead).  CTAs
// walk the units with a grid stride, so a launch has a few CTAs per SM
// whatever the level size.
#define HHG_UNITS(n_if_units, n_tiles, n_act)                                                     \
  for (int unit = blockIdx.x, n_units_ = (n_if_units) + (n_tiles) * (n_act); unit < n_units_;     \
       unit += gridDim.x)

// Interface chunk at position u of the walk (-1: a volume unit).
__device__ __forceinline__ int if_chunk(int u, int n_if_units) { return u < n_if_units ? u : -1; }
// Index of the volume unit at position u (not an interface chunk).
__device__ __forceinline__ int vol_index(int u, int n_if_units) { return u - n_if_units; }

// Walk over the same units, dynamic for large launches: CTA b starts with
// unit b; with at least DYN_UNITS_PER_CTA units per CTA, later units come from
// the problem's counter sched[0] (unit = gridDim.x + counter), so the units
// (tiles by decreasing work, the interface chunks spread among them, see
// spread_unit) are handed out greedily and the launch ends with the smallest
// tiles; smaller launches keep the grid
// stride (measured faster there, e.g. the local recovery cycles of a few
// macros).  Thread 0 takes the next unit one unit ahead, so the atomic's
// latency hides behind the work.  The CTA that finishes last (counted in
// sched[1]) puts both counters back to zero for the problem's next launch and
// counts the completed dynamic launch in sched[2] (read back by tests to show
// that the dynamic branch ran); a problem's kernels run one after another on
// one stream, so launches never share a counter.
constexpr int DYN_UNITS_PER_CTA = 4;
__device__ __forceinline__ bool walk_dynamic(int n_units) { return n_units >= DYN_UNITS_PER_CTA * (int)gridDim.x; }
__device__ __forceinline__ int walk_after(int cur, int n_units, int* sched) {
  if (cur >= n_units) return n_units;
  return walk_dynamic(n_units) ? (int)gridDim.x + atomicAdd(sched, 1) : cur + (int)gridDim.x;
}
__device__ __forceinline__ int walk_first(int n_units, int* sched, int* s_unit, int& nxt) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    nxt = walk_after((int)blockIdx.x, n_units, sched);
    *s_unit = blockIdx.x;
  }
  __syncthreads();
  return *s_unit;
}
__device__ __forceinline__ int walk_next(int n_units, int* sched, int* s_unit, int& nxt) {
  __syncthreads();                              // every thread has read the last unit
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int cur = nxt;
    nxt = walk_after(cur, n_units, sched);
    *s_unit = cur;
  }
  __syncthreads();
  return *s_unit;
}
__device__ __forceinline__ void finish_units(int* sched, int n_units) {
  if (!walk_dynamic(n_units)) return;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    if (atomicAdd(sched + 1, 1) == (int)gridDim.x - 1) {
      atomicExch(sched, 0);
      atomicExch(sched + 1, 0);
      atomicAdd(sched + 2, 1);
    }
  }
}
#define HHG_UNITS_DYN(n_if_units, n_tiles, n_act, sched, s_unit)                                      \
  for (int n_units_ = (n_if_units) + (n_tiles) * (n_act), nxt_ = 0,                                    \
           unit = walk_first(n_units_, (sched), (s_unit), nxt_);                                       \
       unit < n_units_; unit = walk_next(n_units_, (sched), (s_unit), nxt_))

// Position u of a stencil launch's walk -> its interface chunk (returned, or
// -1 for a volume unit, whose index is written to vol).  Launches that take
// the dynamic walk interleave the n_if interface chunks with the n_vol volume
// units (spread_position in hhg_internal.h: one chunk after every
// R = n_vol / n_if volume units).  An interface chunk gathers scattered
// neighbours and does little arithmetic, a volume tile streams contiguous
// rows through the FP64 (or load) pipe, so CTAs of the two kinds side by side
// on an SM keep the pipe busier than a launch whose first units are all
// interface chunks (finest FP64 Gauss-Seidel launch at refinement 8: 0.416
// against 0.442 ms).  Smaller launches keep the chunks first (measured faster
// on the coarse levels).  Every unit still runs once.
__device__ __forceinline__ int spread_unit(int u, int n_if, int n_vol, int& vol) {
  if (!walk_dynamic(n_if + n_vol)) {
    vol = u - n_if;
    return u < n_if ? u : -1;
  }
  return spread_position(u, n_if, n_vol, vol);
}

// Volume unit -> (tile, macro).  The macro index runs fastest and the tile
// lists are sorted by decreasing work, so the last units of a grid-stride walk
// are the smallest tiles of all macros (a short tail).
__device__ __forceinline__ void vol_unit(int b, int n_act, const Tile* __restrict__ tiles,
                                         const int* __restrict__ act, Tile& t, int& macro) {
  t = tiles[b / n_act];
  macro = act[b % n_act];
}

// The restriction walks each coarse tile as RESTRICT_SPLIT units of
// consecutive slices: a coarse level has an eighth of the fine level's nodes
// and its tiles give a few heavy units per CTA, whose tail left SMs idle.
constexpr int RESTRICT_SPLIT = 4;

// Volume unit b of a walk over split tiles: part (b / n_act) % split of tile
// (b / n_act) / split, for active macro b % n_act.
__device__ __forceinline__ void vol_subunit(int b, int n_act, int split, const Tile* __restrict__ tiles,
                                            const int* __restrict__ act, Tile& t, int& macro) {
  const int tp = b / n_act;
  macro = act[b % n_act];
  t = tiles[tp / split];
  const int part = tp % split;
  const int s0 = t.pad * part / split, s1 = t.pad * (part + 1) / split;
  t.k += s0;
  t.pad = s1 - s0;
}

// Off-diagonal part of an interface node's stencil applied to u, and the sum
// of the diagonal weights, over all copies of the node.
template <class T, bool S7>
__device__ __forceinline__ void if_stencil(int N, const int* __restrict__ rs, int64_t block, const T* __restrict__ u,
                                           const T* __restrict__ W, const Copy* __restrict__ cps, int c0, int c1,
                                           T& off, T& diag) {
  for (int c = c0; c < c1; ++c) {
    const Copy cp = cps[c];
    const T* w = W + ((size_t)cp.macro * 16 + node_class(cp.i, cp.j, cp.k, N)) * NDIR;
    const T* ub = u + (size_t)cp.macro * block;
    diag += w[0];
#pragma unroll
    for (int d = 1; d < NDIR; ++d) {
      if (!used_dir(d, S7)) continue;
      const T wd = w[d];
      // 15-point: skip the many zero weights; 7-point: no load waits on a weight
      if (!S7 && wd == T(0)) continue;
      int di, dj, dk;
      dir_ijk(d, di, dj, dk);
      const int ni = cp.i + di, nj = cp.j + dj, nk = cp.k + dk;
      if (!in_lattice(ni, nj, nk, N)) continue;
      off += wd * ub[lidx32(rs, N, ni, nj, nk)];
    }
  }
}

// Writes val into the copies c0 .. c1 - 1 of an interface node: at their
// precomputed block offsets cpo when given, else at the offsets computed from
// (macro, i, j, k).
template <class T>
__device__ __forceinline__ void write_copies(int N, const int* __restrict__ rs, int64_t block, T* __restrict__ u,
                                             const Copy* __restrict__ cps, const uint32_t* __restrict__ cpo, int c0,
                                             int c1, T val) {
  if (cpo) {
    for (int c = c0; c < c1; ++c) u[cpo[c]] = val;
    return;
  }
  for (int c = c0; c < c1; ++c) {
    const Copy cp = cps[c];
    u[(size_t)cp.macro * block + lidx32(rs, N, cp.i, cp.j, cp.k)] = val;
  }
}

// Interface stencil table of a problem level (build_if_tables): for list
// entry q the K distinct neighbours of the node's summed stencil, entry e at
// e * n + q (block offset nb, weight w), its diagonal and inverse diagonal.
template <class T>
struct IfTab {
  const uint32_t* nb;
  const T* w;
  const T* diag;
  const T* dinv;
  int n;
};
constexpr int if_tab_k(bool s7) { return s7 ? 6 : 14; }

// Off-diagonal part of the stencil of list entry q applied to u.
template <class T, int K>
__device__ __forceinline__ T if_offdiag(const IfTab<T>& t, const T* __restrict__ u, int q) {
  T s = T(0);
#pragma unroll
  for (int e = 0; e < K; ++e) s += t.w[(size_t)e * t.n + q] * u[t.nb[(size_t)e * t.n + q]];
  return s;
}

// ---------------------------------------------------------------------------
// Gauss-Seidel, one colour (§2.1 smoother)
// ---------------------------------------------------------------------------
// 16-byte vectors of a row: 4 FP32 or 2 FP64 consecutive slots.
template <class T>
struct Vec;
// load<true>() goes through the read-only path: a Gauss-Seidel colour
// kernel reads only arrays it does not write (the other colours and f).
// load<false>() is a plain coherent load, for code that reads data written
// earlier in the same launch (the persistent batch executor).
template <>
struct Vec<float> {
  static constexpr int n = 4;
  template <bool NC = true>
  __device__ static void load(const float* p, float* v) {
    const float4 q = NC ? __ldg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  }
  __device__ static void store(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Vec<double> {
  static constexpr int n = 2;
  template <bool NC = true>
  __device__ static void load(const double* p, double* v) {
    const double2 q = NC ? __ldg(reinterpret_cast<const double2*>(p)) : *reinterpret_cast<const double2*>(p);
    v[0] = q.x;
    v[1] = q.y;
  }
  __device__ static void store(double* p, const double* v) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

// Slots m0 + s .. m0 + s + VW - 1 (s = +1 when up, -1 when dn, else 0) of a
// row, from the aligned vector at p = &row[m0] and one extra element.
template <class T, bool NC = true>
__device__ __forceinline__ void load_shifted(const T* __restrict__ p, bool up, bool dn, T* v) {
  constexpr int VW = Vec<T>::n;
  Vec<T>::template load<NC>(p, v);
  if (up) {
    const T e = NC ? __ldg(p + VW) : p[VW];
#pragma unroll
    for (int t = 0; t < VW - 1; ++t) v[t] = v[t + 1];
    v[VW - 1] = e;
  } else if (dn) {
    const T e = NC ? __ldg(p - 1) : p[-1];
#pragma unroll
    for (int t = VW - 1; t > 0; --t) v[t] = v[t - 1];
    v[0] = e;
  }
}

// 7-point update of the colour-c nodes in slots m0 .. m0 + VW - 1 of interior
// row j of slice k (one aligned vector per stencil direction, plus one element
// where the neighbour's slot is shifted by one); only the interior nodes among
// them are written.  SCALED: the weights w and the load fb are already divided
// by the centre weight (u = f~ - sum w~ u, six FMAs per node), else the sum is
// multiplied by inv, the inverse centre weight.
template <class T, bool SCALED, bool NC = true>
__device__ __forceinline__ void gs_group7(const Slice& sc, int N, int j, int g, int c, T* __restrict__ ub,
                                          const T* __restrict__ fb, const T* __restrict__ w, T inv) {
  constexpr int VW = Vec<T>::n;
  int ic, mlo, n;
  colour_row(N, j, sc.k, c, ic, mlo, n);
  const int m0 = g * VW;
  const int X = slot_prefix(sc.M - j);
  const int L = sc.M - j;
  const int r0 = sc.SL0 + sc.SM0 - X;           // row (j, k)
  const int rjp = r0 + row_slots(L);             // row (j + 1, k)
  const int rjm = r0 - row_slots(L + 1);         // row (j - 1, k)
  const int rkp = sc.SLp + sc.SMm - X;           // row (j - 1, k + 1)
  const int rkm = sc.SLm + sc.SMp - X;           // row (j + 1, k - 1)
  const int cc = c * sc.CS, cp = ((c + 1) & 3) * sc.CS, cm = ((c + 3) & 3) * sc.CS;
  const bool e1 = ic == 3, e0 = ic == 0;         // slot of i + 1 is m + e1, of i - 1 is m - e0
  T acc[VW], a[VW];
  Vec<T>::template load<NC>(fb + cc + r0 + m0, acc);
  load_shifted<T, NC>(ub + cp + r0 + m0, e1, false, a);    // ( 1,  0,  0)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[1] * a[t];
  load_shifted<T, NC>(ub + cp + rjp + m0, false, e0, a);   // (-1,  1,  0)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[2] * a[t];
  Vec<T>::template load<NC>(ub + cp + rkp + m0, a);              // ( 0, -1,  1)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[3] * a[t];
  load_shifted<T, NC>(ub + cm + r0 + m0, false, e0, a);    // (-1,  0,  0)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[8] * a[t];
  load_shifted<T, NC>(ub + cm + rjm + m0, e1, false, a);   // ( 1, -1,  0)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[9] * a[t];
  Vec<T>::template load<NC>(ub + cm + rkm + m0, a);              // ( 0,  1, -1)
#pragma unroll
  for (int t = 0; t < VW; ++t) {
    if (SCALED) acc[t] -= w[10] * a[t];         // weights and f already divided by the centre weight
    else acc[t] = (acc[t] - w[10] * a[t]) * inv;
  }
  T* out = ub + cc + r0 + m0;
  const int lo = max(mlo - m0, 0), hi = min(mlo + n - m0, VW);
  if (lo == 0 && hi == VW) {
    Vec<T>::store(out, acc);
  } else {
#pragma unroll
    for (int t = 0; t < VW; ++t)
      if (t >= lo && t < hi) out[t] = acc[t];
  }
}

// 7-point residual r = f - A u of the colour-c nodes in slots m0 .. m0 + VW - 1
// of interior row j of slice k (same vectors as gs_group7 plus the centre);
// writes the interior nodes among them to rb and/or adds their squares to ss.
// ZERO: the residual of these nodes is known to vanish (their colour was the
// last one smoothed); zeros are written and nothing is read.
// Stores the lanes lo .. hi - 1 of a VW-vector (all lanes at once when the
// vector is complete).
template <class T>
__device__ __forceinline__ void store_lanes(T* __restrict__ out, const T* acc, int lo, int hi) {
  constexpr int VW = Vec<T>::n;
  if (lo == 0 && hi == VW) {
    Vec<T>::store(out, acc);
  } else {
#pragma unroll
    for (int t = 0; t < VW; ++t)
      if (t >= lo && t < hi) out[t] = acc[t];
  }
}

template <class T, bool WRITE, bool NORM, bool ZERO = false, bool NC = true>
__device__ __forceinline__ void res_group7(const Slice& sc, int N, int j, int g, int c, const T* __restrict__ ub,
                                           const T* __restrict__ fb, T* __restrict__ rb, const T* __restrict__ w,
                                           double& ss) {
  constexpr int VW = Vec<T>::n;
  int ic, mlo, n;
  colour_row(N, j, sc.k, c, ic, mlo, n);
  const int m0 = g * VW;
  const int X = slot_prefix(sc.M - j);
  const int L = sc.M - j;
  const int r0 = sc.SL0 + sc.SM0 - X;
  const int rjp = r0 + row_slots(L);
  const int rjm = r0 - row_slots(L + 1);
  const int rkp = sc.SLp + sc.SMm - X;
  const int rkm = sc.SLm + sc.SMp - X;
  const int cc = c * sc.CS, cp = ((c + 1) & 3) * sc.CS, cm = ((c + 3) & 3) * sc.CS;
  const bool e1 = ic == 3, e0 = ic == 0;
  T acc[VW], a[VW];
  if (ZERO) {
#pragma unroll
    for (int t = 0; t < VW; ++t) acc[t] = T(0);
    if (WRITE) store_lanes(rb + cc + r0 + m0, acc, max(mlo - m0, 0), min(mlo + n - m0, VW));
    return;
  }
  Vec<T>::template load<NC>(fb + cc + r0 + m0, acc);
  Vec<T>::template load<NC>(ub + cc + r0 + m0, a);               // centre
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[0] * a[t];
  load_shifted<T, NC>(ub + cp + r0 + m0, e1, false, a);    // ( 1,  0,  0)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[1] * a[t];
  load_shifted<T, NC>(ub + cp + rjp + m0, false, e0, a);   // (-1,  1,  0)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[2] * a[t];
  Vec<T>::template load<NC>(ub + cp + rkp + m0, a);              // ( 0, -1,  1)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[3] * a[t];
  load_shifted<T, NC>(ub + cm + r0 + m0, false, e0, a);    // (-1,  0,  0)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[8] * a[t];
  load_shifted<T, NC>(ub + cm + rjm + m0, e1, false, a);   // ( 1, -1,  0)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[9] * a[t];
  Vec<T>::template load<NC>(ub + cm + rkm + m0, a);              // ( 0,  1, -1)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[10] * a[t];
  const int lo = max(mlo - m0, 0), hi = min(mlo + n - m0, VW);
  if (NORM) {
#pragma unroll
    for (int t = 0; t < VW; ++t)
      if (t >= lo && t < hi) ss += (double)acc[t] * (double)acc[t];
  }
  if (WRITE) store_lanes(rb + cc + r0 + m0, acc, lo, hi);
}

// The 7-point colour-c items of one tile: groups of VW consecutive same-colour
// slots per thread, the items of all the tile's slices streamed in one pass.
template <class T, bool SCALED, bool NC = true>
__device__ __forceinline__ void gs_tile7(const Tile& t, int N, const int* __restrict__ rs, int colour,
                                         T* __restrict__ ub, const T* __restrict__ fb, const T* __restrict__ w, T inv,
                                         int (*s_pre2)[33], int* s_pre_tot) {
  constexpr int VW = Vec<T>::n;
  const T wr[11] = {T(0), w[1], w[2], w[3], T(0), T(0), T(0), T(0), w[8], w[9], w[10]};
  const int total = flat_setup_slabs(t, N, colour, true, VW, s_pre2, s_pre_tot);
  int sl = 0;
  for (int tt = tid256(); tt < total; tt += CTA) {
    while (tt >= s_pre_tot[sl + 1]) ++sl;    // items only grow: the slice only advances
    const int k = t.k + sl;
    const Tile ts{k, t.j0, t.m0, 1};
    int j, g;
    flat_item(ts, N, colour, true, s_pre2[sl], tt - s_pre_tot[sl], j, g, VW);
    gs_group7<T, SCALED, NC>(slice_consts(rs, N, k), N, j, g, colour, ub, fb, wr, inv);
  }
}

// fs / Wsc (7-point only, may be null): the volume nodes read f and the
// interior weights already divided by their macro's centre weight.
template <class T, bool S7>
__global__ void __launch_bounds__(CTA, 5) k_gs(int N, const int* __restrict__ rs, int64_t block, T* __restrict__ u, T* __restrict__ uI,
                                            const T* __restrict__ f, const T* __restrict__ fI,
                                            const T* __restrict__ W, const T* __restrict__ Winv,
                                            const T* __restrict__ fs, const T* __restrict__ Wsc,
                                            const Tile* __restrict__ tiles, int n_tiles, const int* __restrict__ act,
                                            int n_act, int colour, const int* __restrict__ cptr,
                                            const Copy* __restrict__ cps, const uint32_t* __restrict__ cpo,
                                            const int* __restrict__ list, int n_list, IfTab<T> tab,
                                            int n_if_units, int* __restrict__ sched) {
  __shared__ int s_pre2[MAX_SLABS][33];
  __shared__ int s_pre_tot[MAX_SLABS + 1];
  __shared__ int s_unit;
  HHG_UNITS_DYN(n_if_units, n_tiles, n_act, sched, &s_unit) {
    int vol_ = 0;
    if (const int ic_ = spread_unit(unit, n_if_units, n_tiles * n_act, vol_); ic_ >= 0) {
      const int q = ic_ * CTA + tid256();
      if (q < n_list) {
        const int node = list[q];
        const int c0 = cptr[node], c1 = cptr[node + 1];
        T val;
        if (tab.nb) {
          val = (fI[node] - if_offdiag<T, if_tab_k(S7)>(tab, u, q)) * tab.dinv[q];
        } else {
          T off = T(0), diag = T(0);
          if_stencil<T, S7>(N, rs, block, u, W, cps, c0, c1, off, diag);
          val = (fI[node] - off) / diag;
        }
        uI[node] = val;
        write_copies(N, rs, block, u, cps, cpo, c0, c1, val);
      }
      continue;
    }
    Tile t;
    int macro;
    vol_unit(vol_, n_act, tiles, act, t, macro);
    T* ub = u + (size_t)macro * block;
    const T* fb = f + (size_t)macro * block;
    const T* w = W + (size_t)macro * 16 * NDIR;
    const T inv = Winv[macro];
    if (S7) {
      if (Wsc)
        gs_tile7<T, true>(t, N, rs, colour, ub, fs + (size_t)macro * block, Wsc + (size_t)macro * 16 * NDIR, T(1),
                          s_pre2, s_pre_tot);
      else
        gs_tile7<T, false>(t, N, rs, colour, ub, fb, w, inv, s_pre2, s_pre_tot);
    } else {
      // 15-point: one colour-c node per item
      const int total = flat_setup_slabs(t, N, colour, true, 1, s_pre2, s_pre_tot);
      int sl = 0;
      for (int tt = tid256(); tt < total; tt += CTA) {
        while (tt >= s_pre_tot[sl + 1]) ++sl;
        const int k = t.k + sl;
        const Tile ts{k, t.j0, t.m0, 1};
        int j, v, ic, mlo, n;
        flat_item(ts, N, colour, true, s_pre2[sl], tt - s_pre_tot[sl], j, v);
        colour_row(N, j, k, colour, ic, mlo, n);
        const int i = 4 * (mlo + v) + ic;
        const int me = lidx32(rs, N, i, j, k);
        T acc = fb[me];
#pragma unroll
        for (int d = 1; d < NDIR; ++d) {
          int di, dj, dk;
          dir_ijk(d, di, dj, dk);
          acc -= w[d] * ub[lidx32(rs, N, i + di, j + dj, k + dk)];
        }
        ub[me] = acc * inv;
      }
    }
    __syncthreads();
  }
  finish_units(sched, n_if_units + n_tiles * n_act);
}

// Flat Gauss-Seidel, one colour, 7-point structure: one work item (one
// 16-byte vector of same-colour slots of one row) per thread, no tiles, no
// CTA barrier.  items[it] = (j << 20) | (k << 10) | g lists the colour's
// items of one macro interior, slice by slice and row by row, so consecutive
// threads take consecutive vectors of a row; a thread's global index runs
// over the active macros (item it of macro act[a]).  CTAs of interface nodes
// (one node per thread, as in k_gs) are spread among the volume CTAs
// (spread_position over CTAs).  fv / Wv: the volume's load and weights (f and
// W, or with SCALED both divided by the centre weight).  On a coarse level the tile kernel's launch
// waits for a few CTAs each walking a whole tile; here every thread has one
// item and the launch lasts about one item's latency.  Same arithmetic per
// item as gs_tile7, so the iterate equals the tile kernel's bit for bit.
// Resident CTAs per SM: the FP64 form is held to 8 (32 registers; measured
// 1.2% faster at refinement 8); the FP32 form is left to the compiler (0: no
// bound; 3% slower held to 8, 6% slower held to 6).
template <class T>
struct FlatMinCtas {
  static constexpr int value = sizeof(T) == 8 ? 8 : 0;
};
template <class T, bool SCALED>
__global__ void __launch_bounds__(CTA, FlatMinCtas<T>::value) k_gs_flat(int N, const int* __restrict__ rs, int64_t block, T* __restrict__ u,
                                                 T* __restrict__ uI, const T* __restrict__ fI,
                                                 const T* __restrict__ W, const T* __restrict__ Winv,
                                                 const T* __restrict__ fv, const T* __restrict__ Wv,
                                                 const uint32_t* __restrict__ items, int n_items,
                                                 const int* __restrict__ act, int n_act, int colour,
                                                 const int* __restrict__ cptr, const Copy* __restrict__ cps,
                                                 const uint32_t* __restrict__ cpo, const int* __restrict__ list,
                                                 int n_list, IfTab<T> tab, int n_if_ctas, int n_vol_ctas) {
  int vb = 0;
  const int ib = spread_position((int)blockIdx.x, n_if_ctas, n_vol_ctas, vb);
  if (ib >= 0) {
    const int q = ib * CTA + tid256();
    if (q < n_list) {
      const int node = list[q];
      const int c0 = cptr[node], c1 = cptr[node + 1];
      T val;
      if (tab.nb) {
        val = (fI[node] - if_offdiag<T, 6>(tab, u, q)) * tab.dinv[q];
      } else {
        T off = T(0), diag = T(0);
        if_stencil<T, true>(N, rs, block, u, W, cps, c0, c1, off, diag);
        val = (fI[node] - off) / diag;
      }
      uI[node] = val;
      write_copies(N, rs, block, u, cps, cpo, c0, c1, val);
    }
    return;
  }
  const int v = vb * CTA + tid256();
  if (v >= n_items * n_act) return;
  const int a = v / n_items, it = v - a * n_items;
  const int macro = act[a];
  const uint32_t d = items[it];
  const int j = (int)(d >> 20), k = (int)((d >> 10) & 1023u), g = (int)(d & 1023u);
  const T* w = Wv + (size_t)macro * 16 * NDIR;
  const T wr[11] = {T(0), w[1], w[2], w[3], T(0), T(0), T(0), T(0), w[8], w[9], w[10]};
  gs_group7<T, SCALED>(slice_consts(rs, N, k), N, j, g, colour, u + (size_t)macro * block,
                       fv + (size_t)macro * block, wr, SCALED ? T(1) : Winv[macro]);
}

// ---------------------------------------------------------------------------
// Streaming Gauss-Seidel, one colour, 7-point structure (levels with at least
// STREAM_MIN_N intervals).  In the colour-split layout the rows of a slice
// follow each other, so a band of rows of one slice and colour is one
// contiguous range of memory.  A unit (StreamTile) sweeps the band j0..j1 of
// one macro through the slices ka..kb.  The colour-c update of slice k reads
// colour c+1 in slices k and k+1, colour c-1 in slices k-1 and k, and f of
// colour c in slice k.  A producer warp copies these ranges into shared
// memory with bulk asynchronous copies (rings of three slices per neighbour
// colour, two for f) that complete on a "full" mbarrier per step; eight
// consumer warps wait on it, update their share of the slice's colour-c
// nodes straight into global memory and arrive on the step's "empty"
// mbarrier, which frees the slots the producer refills two steps later.  No
// CTA-wide barrier separates the steps of a unit, so warps and copies
// overlap; each neighbour value crosses HBM about once per launch (plus one
// row on either side of the band and one slice at either end of the unit).
// Interface chunks are updated by the consumer threads as in k_gs.  Every
// wait on an mbarrier is bounded: when one runs out the CTA sets *err, lets
// its copies in flight land (bounded) and stops taking units.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of bar with the given parity; false after `limit`
// unsuccessful tries (the first 32 back to back, then about 64 ns apart).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    if (mbar_test(bar, parity)) return true;
    if (it >= 32) __nanosleep(64);
  }
  return false;
}
constexpr int DRAIN_LIMIT = 1 << 24;

// First slot and slot count, inside one colour array, of rows ja..jb of
// slice k (clipped to the slice's closed lattice, rows 0..N-k).
__device__ __forceinline__ void band_range(const int* __restrict__ rs, int N, int k, int ja, int jb, int& off,
                                           int& len) {
  const int M = N + 1 - k;
  jb = min(jb, N - k);
  off = __ldg(rs + k) + slot_prefix(M) - slot_prefix(M - ja);
  len = jb >= ja ? slot_prefix(M - ja) - slot_prefix(M - jb - 1) : 0;
}

// 16-byte vector of a staged row in shared memory (16-byte aligned), shifted
// by one slot as in load_shifted.
template <class T>
struct SVec;
template <>
struct SVec<float> {
  __device__ static void load(const float* p, float* v) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  }
};
template <>
struct SVec<double> {
  __device__ static void load(const double* p, double* v) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x;
    v[1] = q.y;
  }
};
template <class T>
__device__ __forceinline__ void lds_shifted(const T* p, bool up, bool dn, T* v) {
  constexpr int VW = Vec<T>::n;
  SVec<T>::load(p, v);
  if (up) {
    const T e = p[VW];
#pragma unroll
    for (int t = 0; t < VW - 1; ++t) v[t] = v[t + 1];
    v[VW - 1] = e;
  } else if (dn) {
    const T e = p[-1];
#pragma unroll
    for (int t = VW - 1; t > 0; --t) v[t] = v[t - 1];
    v[0] = e;
  }
}

// The update of gs_group7 with its operands read from the staged rows: a0 /
// a0p = colour c+1 rows j and j+1 of slice k, a1m = colour c+1 row j-1 of
// slice k+1, b0 / b0m = colour c-1 rows j and j-1 of slice k, bmp = colour
// c-1 row j+1 of slice k-1, fr = row j of f (all pointing at slot m0); out
// is row j of colour c in global memory at slot m0.  Same operations in the
// same order as gs_group7.
template <class T, bool SCALED>
__device__ __forceinline__ void gs_group7_staged(const T* a0, const T* a0p, const T* a1m, const T* b0, const T* b0m,
                                                 const T* bmp, const T* fr, T* __restrict__ out, bool e0, bool e1,
                                                 int lo, int hi, const T* w, T inv) {
  constexpr int VW = Vec<T>::n;
  T acc[VW], a[VW];
  SVec<T>::load(fr, acc);
  lds_shifted(a0, e1, false, a);    // ( 1,  0,  0)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[1] * a[t];
  lds_shifted(a0p, false, e0, a);   // (-1,  1,  0)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[2] * a[t];
  SVec<T>::load(a1m, a);            // ( 0, -1,  1)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[3] * a[t];
  lds_shifted(b0, false, e0, a);    // (-1,  0,  0)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[8] * a[t];
  lds_shifted(b0m, e1, false, a);   // ( 1, -1,  0)
#pragma unroll
  for (int t = 0; t < VW; ++t) acc[t] -= w[9] * a[t];
  SVec<T>::load(bmp, a);            // ( 0,  1, -1)
#pragma unroll
  for (int t = 0; t < VW; ++t) {
    if (SCALED) acc[t] -= w[10] * a[t];
    else acc[t] = (acc[t] - w[10] * a[t]) * inv;
  }
  if (lo == 0 && hi == VW) {
    Vec<T>::store(out, acc);
  } else {
#pragma unroll
    for (int t = 0; t < VW; ++t)
      if (t >= lo && t < hi) out[t] = acc[t];
  }
}

// Shared memory of the streaming kernel: 8 staging slots of `slot` elements
// (3 for colour c+1, 3 for colour c-1, 2 for f) between pads of STREAM_PAD
// elements, so that the one-slot shifts of lanes outside the interior stay
// inside the allocation.  The CTA is 8 consumer warps and 1 producer warp.
constexpr int STREAM_PAD = 32;
constexpr int STREAM_NSLOT = 8;
constexpr int STREAM_CONSUMERS = 8;
constexpr int STREAM_CTA = 32 * (STREAM_CONSUMERS + 1);

template <class T, bool SCALED>
__global__ void __launch_bounds__(STREAM_CTA) k_gs_stream(
    int N, const int* __restrict__ rs, int64_t block, T* __restrict__ u, T* __restrict__ uI,
    const T* __restrict__ fI, const T* __restrict__ W, const T* __restrict__ Winv, const T* __restrict__ fv,
    const T* __restrict__ Wv, const StreamTile* __restrict__ tiles, int n_tiles, const int* __restrict__ act,
    int n_act, int colour, const int* __restrict__ cptr, const Copy* __restrict__ cps,
    const uint32_t* __restrict__ cpo, const int* __restrict__ list, int n_list, IfTab<T> tab, int n_if_units,
    int* __restrict__ sched, int slot, int wait_limit, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char s_dyn[];
  T* const buf = reinterpret_cast<T*>(s_dyn) + STREAM_PAD;
  __shared__ __align__(8) uint64_t full[3], empty[3];
  __shared__ int s_pre[STREAM_SLICES][STREAM_BAND32 + 1];
  __shared__ int s_unit;
  __shared__ int s_fail;
  const int tid = tid256();
  const int warp = threadIdx.y, lane = threadIdx.x;
  const bool producer = warp == STREAM_CONSUMERS;
  if (tid == 0) s_fail = 0;
  constexpr int VW = Vec<T>::n;
  const int CS = __ldg(rs + N + 2);
  const int c = colour, cA = (c + 1) & 3, cB = (c + 3) & 3;
  bool failed = false;
  HHG_UNITS_DYN(n_if_units, n_tiles, n_act, sched, &s_unit) {
    if (const int ic_ = if_chunk(unit, n_if_units); ic_ >= 0) {
      const int q = ic_ * CTA + tid;
      if (!producer && q < n_list) {
        const int node = list[q];
        const int c0 = cptr[node], c1 = cptr[node + 1];
        T val;
        if (tab.nb) {
          val = (fI[node] - if_offdiag<T, 6>(tab, u, q)) * tab.dinv[q];
        } else {
          T off = T(0), diag = T(0);
          if_stencil<T, true>(N, rs, block, u, W, cps, c0, c1, off, diag);
          val = (fI[node] - off) / diag;
        }
        uI[node] = val;
        write_copies(N, rs, block, u, cps, cpo, c0, c1, val);
      }
      continue;
    }
    const int vb = vol_index(unit, n_if_units);
    const StreamTile st = tiles[vb / n_act];
    const int macro = act[vb % n_act];
    const int nst = st.kb - st.ka + 1;
    // fresh barriers per unit (every phase of the previous unit completed:
    // its steps were all consumed and released), and the items per row of
    // every step of the unit
    if (tid == 0)
      for (int b = 0; b < 3; ++b) {
        mbar_init(&full[b], 1);
        mbar_init(&empty[b], STREAM_CONSUMERS);
      }
    for (int sidx = warp; sidx < nst; sidx += STREAM_CONSUMERS + 1) {
      const int k = st.ka + sidx;
      const int nr = min(st.j1, N - 2 - k) - st.j0 + 1;
      int len = lane < nr ? row_items(N, st.j0 + lane, k, c, true, VW) : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, len, o);
        if (lane >= o) len += y;
      }
      if (lane < nr) s_pre[sidx][lane + 1] = len;
      if (lane == 0) s_pre[sidx][0] = 0;
    }
    __syncthreads();
    T* ub = u + (size_t)macro * block;
    const int ja = st.j0 - 1, jbA = st.j1 + 1;
    if (producer) {
      if (lane == 0) {
        const T* gA = ub + (size_t)cA * CS;
        const T* gB = ub + (size_t)cB * CS;
        const T* gF = fv + (size_t)macro * block + (size_t)c * CS;
        int issued = 0;
        for (int sidx = 0; sidx < nst; ++sidx) {
          // step sidx refills the slots of step sidx - 2 (released on its empty barrier)
          if (sidx >= 2 && !mbar_wait(&empty[(sidx - 2) % 3], ((sidx - 2) / 3) & 1, wait_limit)) {
            atomicExch(err, 1);
            atomicExch(&s_fail, 1);
          }
          if (*(volatile int*)&s_fail) break;
          const int k = st.ka + sidx;
          int oA1, lA1, oB0, lB0, oF, lF, oA0 = 0, lA0 = 0, oBm = 0, lBm = 0;
          band_range(rs, N, k + 1, ja, jbA, oA1, lA1);
          band_range(rs, N, k, ja, jbA, oB0, lB0);
          band_range(rs, N, k, st.j0, min(st.j1, N - 2 - k), oF, lF);
          if (sidx == 0) {
            band_range(rs, N, k, ja, jbA, oA0, lA0);
            band_range(rs, N, k - 1, ja, jbA, oBm, lBm);
          }
          if (max(max(max(lA1, lB0), max(lF, lA0)), lBm) > slot) {   // never for the host's slot size
            atomicExch(err, 2);
            lA1 = min(lA1, slot);
            lB0 = min(lB0, slot);
            lF = min(lF, slot);
            lA0 = min(lA0, slot);
            lBm = min(lBm, slot);
          }
          fence_async_shared();
          uint64_t* b = &full[sidx % 3];
          mbar_expect(b, (uint32_t)(lA1 + lB0 + lF + lA0 + lBm) * (uint32_t)sizeof(T));
          if (lA1) bulk_load(buf + ((k + 1) % 3) * slot, gA + oA1, lA1 * (uint32_t)sizeof(T), b);
          if (lB0) bulk_load(buf + (3 + k % 3) * slot, gB + oB0, lB0 * (uint32_t)sizeof(T), b);
          if (lF) bulk_load(buf + (6 + k % 2) * slot, gF + oF, lF * (uint32_t)sizeof(T), b);
          if (lA0) bulk_load(buf + (k % 3) * slot, gA + oA0, lA0 * (uint32_t)sizeof(T), b);
          if (lBm) bulk_load(buf + (3 + (k + 2) % 3) * slot, gB + oBm, lBm * (uint32_t)sizeof(T), b);
          issued = sidx + 1;
        }
        if (*(volatile int*)&s_fail) {
          // the copies of the last step issued on each barrier may still be in flight
          for (int b = 0; b < 3; ++b) {
            int last = -1;
            for (int q = 0; q < issued; ++q)
              if (q % 3 == b) last = q;
            if (last >= 0) mbar_wait(&full[b], (last / 3) & 1, DRAIN_LIMIT);
          }
        }
      }
    } else {
      T* gU = ub + (size_t)c * CS;
      const T* wm = Wv + (size_t)macro * 16 * NDIR;
      const T w[11] = {T(0), wm[1], wm[2], wm[3], T(0), T(0), T(0), T(0), wm[8], wm[9], wm[10]};
      const T inv = SCALED ? T(1) : Winv[macro];
      for (int sidx = 0; sidx < nst; ++sidx) {
        if (!mbar_wait(&full[sidx % 3], (sidx / 3) & 1, wait_limit)) {
          if (lane == 0) {
            atomicExch(err, 1);
            atomicExch(&s_fail, 1);
          }
          break;   // no arrival on empty: the producer stops at its next wait
        }
        const int k = st.ka + sidx;
        const int nr = min(st.j1, N - 2 - k) - st.j0 + 1;
        const int* pre = s_pre[sidx];
        const int total = pre[nr];
        const int M = N + 1 - k, M1 = N - k, Mm = N + 2 - k;
        const T* sA0 = buf + (k % 3) * slot;
        const T* sA1 = buf + ((k + 1) % 3) * slot;
        const T* sB0 = buf + (3 + k % 3) * slot;
        const T* sBm = buf + (3 + (k + 2) % 3) * slot;
        const T* sF = buf + (6 + k % 2) * slot;
        const int PA = slot_prefix(M - ja), PA1 = slot_prefix(M1 - ja), PAm = slot_prefix(Mm - ja);
        const int PF = slot_prefix(M - st.j0);
        const int gbase = __ldg(rs + k) + slot_prefix(M);
        for (int tt = tid; tt < total; tt += CTA) {
          int lo_r = 0, hi_r = nr;
          while (hi_r - lo_r > 1) {
            const int mid = (lo_r + hi_r) >> 1;
            if (pre[mid] <= tt) lo_r = mid;
            else hi_r = mid;
          }
          const int j = st.j0 + lo_r;
          const int g = tt - pre[lo_r];
          int ic, mlo, n;
          colour_row(N, j, k, c, ic, mlo, n);
          const int m0 = g * VW;
          const int X = slot_prefix(M - j);
          const T* a0 = sA0 + (PA - X) + m0;
          const T* a0p = sA0 + (PA - slot_prefix(M - j - 1)) + m0;
          const T* a1m = sA1 + (PA1 - slot_prefix(M1 - j + 1)) + m0;
          const T* b0 = sB0 + (PA - X) + m0;
          const T* b0m = sB0 + (PA - slot_prefix(M - j + 1)) + m0;
          const T* bmp = sBm + (PAm - slot_prefix(Mm - j - 1)) + m0;
          const T* fr = sF + (PF - X) + m0;
          const int lo = max(mlo - m0, 0), hi = min(mlo + n - m0, VW);
          gs_group7_staged<T, SCALED>(a0, a0p, a1m, b0, b0m, bmp, fr, gU + (gbase - X) + m0, ic == 0, ic == 3,
                                      lo, hi, w, inv);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[sidx % 3]);
      }
    }
    __syncthreads();
    if (*(volatile int*)&s_fail) {
      failed = true;
      break;
    }
  }
  (void)failed;
  finish_units(sched, n_if_units + n_tiles * n_act);
}

// ---------------------------------------------------------------------------
// Residual r = f - A u on the free nodes (all colours); optional write of r
// (zero at the problem's frozen ghost copies) and per-CTA partial sums of r^2
// ---------------------------------------------------------------------------
template <class T, bool S7, bool WRITE, bool NORM>
__global__ void __launch_bounds__(CTA, 4) k_res(int N, const int* __restrict__ rs, int64_t block, const T* __restrict__ u,
                                             const T* __restrict__ uI, const T* __restrict__ f,
                                             const T* __restrict__ fI, T* __restrict__ r, const T* __restrict__ W,
                                             const Tile* __restrict__ tiles, int n_tiles, const int* __restrict__ act,
                                             int n_act, const int* __restrict__ cptr, const Copy* __restrict__ cps,
                                             const uint32_t* __restrict__ cpo, const int* __restrict__ list,
                                             int n_list, IfTab<T> tab,
                                             const int64_t* __restrict__ zero_off, int n_zero, int n_if_units,
                                             double* __restrict__ partial, int* __restrict__ sched, int skip,
                                             int skip_lo, int skip_hi) {
  __shared__ int s_pre2[MAX_SLABS][33];
  __shared__ int s_pre_tot[MAX_SLABS + 1];
  __shared__ double sh[32];
  double ss = 0.0;
  __shared__ int s_unit;
  HHG_UNITS_DYN(n_if_units, n_tiles, n_act, sched, &s_unit) {
    int vol_ = 0;
    if (const int ic_ = spread_unit(unit, n_if_units, n_tiles * n_act, vol_); ic_ >= 0) {
      const int q = ic_ * CTA + tid256();
      if (q < n_list) {
        const int node = list[q];
        const int c0 = cptr[node], c1 = cptr[node + 1];
        T res;
        if (q >= skip_lo && q < skip_hi) {
          res = T(0);                              // the colour smoothed last
        } else if (tab.nb) {
          res = fI[node] - tab.diag[q] * uI[node] - if_offdiag<T, if_tab_k(S7)>(tab, u, q);
        } else {
          T off = T(0), diag = T(0);
          if_stencil<T, S7>(N, rs, block, u, W, cps, c0, c1, off, diag);
          res = fI[node] - diag * uI[node] - off;
        }
        if (WRITE) write_copies(N, rs, block, r, cps, cpo, c0, c1, res);
        if (NORM) ss += (double)res * (double)res;
      } else if (WRITE && q < n_list + n_zero) {
        r[zero_off[q - n_list]] = T(0);
      }
      continue;
    }
    Tile t;
    int macro;
    vol_unit(vol_, n_act, tiles, act, t, macro);
    const T* ub = u + (size_t)macro * block;
    const T* fb = f + (size_t)macro * block;
    T* rb = r + (size_t)macro * block;
    const T* w = W + (size_t)macro * 16 * NDIR;
    if (S7) {
      // one colour after another, groups of VW same-colour slots per thread
      constexpr int VW = Vec<T>::n;
      const T wr[11] = {w[0], w[1], w[2], w[3], T(0), T(0), T(0), T(0), w[8], w[9], w[10]};
      for (int c = 0; c < 4; ++c) {
        if (!WRITE && c == skip) continue;         // norm only: the skipped colour adds nothing
        const int total = flat_setup_slabs(t, N, c, true, VW, s_pre2, s_pre_tot);
        int sl = 0;
        for (int tt = tid256(); tt < total; tt += CTA) {
          while (tt >= s_pre_tot[sl + 1]) ++sl;
          const int k = t.k + sl;
          const Tile ts{k, t.j0, t.m0, 1};
          int j, g;
          flat_item(ts, N, c, true, s_pre2[sl], tt - s_pre_tot[sl], j, g, VW);
          if (c == skip)
            res_group7<T, WRITE, NORM, true>(slice_consts(rs, N, k), N, j, g, c, ub, fb, rb, wr, ss);
          else
            res_group7<T, WRITE, NORM>(slice_consts(rs, N, k), N, j, g, c, ub, fb, rb, wr, ss);
        }
        __syncthreads();
      }
      continue;
    }
    // 15-point: four nodes of one slot per item
    HHG_TILE_NODES(N, rs, t, s_pre, {
      const int me = lidx32(rs, N, i, j, k);
      T acc = T(0);
      if (((i + 2 * j + 3 * k) & 3) != skip) {
        acc = fb[me] - w[0] * ub[me];
_Pragma("unroll")
        for (int d = 1; d < NDIR; ++d) {
          int di, dj, dk;
          dir_ijk(d, di, dj, dk);
          acc -= w[d] * ub[lidx32(rs, N, i + di, j + dj, k + dk)];
        }
      }
      if (WRITE) rb[me] = acc;
      if (NORM) ss += (double)acc * (double)acc;
    })
  }
  finish_units(sched, n_if_units + n_tiles * n_act);
  if (NORM) {
    const double s = block_sum(ss, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.x] = s;
  }
}

// Flat residual, 7-point structure: the items of all four colours of the flat
// Gauss-Seidel tables (colour c's at off[c] .. off[c + 1]) for every active
// macro, and the interface entries, in chunks of 256 walked with a grid
// stride (launched with one chunk per CTA), interface chunks spread among the
// volume chunks; no tiles and no CTA barrier before the final norm
// reduction.  Same arithmetic per item as k_res (res_group7), so r is the
// same bit for bit; the norm's partial sums would follow the grid.  n_items:
// items per macro taken (off[4], or off[3] for a norm-only launch that skips
// colour 3).
template <class T, bool WRITE, bool NORM>
__global__ void __launch_bounds__(CTA) k_res_flat(int N, const int* __restrict__ rs, int64_t block,
                                                  const T* __restrict__ u, const T* __restrict__ uI,
                                                  const T* __restrict__ f, const T* __restrict__ fI, T* __restrict__ r,
                                                  const T* __restrict__ W, const uint32_t* __restrict__ items,
                                                  int4 off, int n_items, const int* __restrict__ act, int n_act,
                                                  const int* __restrict__ cptr, const Copy* __restrict__ cps,
                                                  const uint32_t* __restrict__ cpo, const int* __restrict__ list,
                                                  int n_list, IfTab<T> tab, const int64_t* __restrict__ zero_off,
                                                  int n_zero, int n_if_chunks, int n_vol_chunks,
                                                  double* __restrict__ partial, int skip, int skip_lo, int skip_hi) {
  __shared__ double sh[32];
  double ss = 0.0;
  const int n_vol = n_items * n_act;
  for (int chunk = blockIdx.x; chunk < n_if_chunks + n_vol_chunks; chunk += gridDim.x) {
    int vc = 0;
    const int ic = spread_position(chunk, n_if_chunks, n_vol_chunks, vc);
    if (ic >= 0) {
      const int q = ic * CTA + tid256();
      if (q < n_list) {
        const int node = list[q];
        const int c0 = cptr[node], c1 = cptr[node + 1];
        T res;
        if (q >= skip_lo && q < skip_hi) {
          res = T(0);                              // the colour smoothed last
        } else if (tab.nb) {
          res = fI[node] - tab.diag[q] * uI[node] - if_offdiag<T, 6>(tab, u, q);
        } else {
          T off_ = T(0), diag = T(0);
          if_stencil<T, true>(N, rs, block, u, W, cps, c0, c1, off_, diag);
          res = fI[node] - diag * uI[node] - off_;
        }
        if (WRITE) write_copies(N, rs, block, r, cps, cpo, c0, c1, res);
        if (NORM) ss += (double)res * (double)res;
      } else if (WRITE && q < n_list + n_zero) {
        r[zero_off[q - n_list]] = T(0);
      }
      continue;
    }
    const int v = vc * CTA + tid256();
    if (v >= n_vol) continue;
    const int a = v / n_items, it = v - a * n_items;
    const int c = it < off.y ? 0 : it < off.z ? 1 : it < off.w ? 2 : 3;
    if (!WRITE && c == skip) continue;             // norm only: the skipped colour adds nothing
    const int macro = act[a];
    const uint32_t d = items[it];
    const int j = (int)(d >> 20), k = (int)((d >> 10) & 1023u), g = (int)(d & 1023u);
    const T* w = W + (size_t)macro * 16 * NDIR;
    const T wr[11] = {w[0], w[1], w[2], w[3], T(0), T(0), T(0), T(0), w[8], w[9], w[10]};
    const size_t mb = (size_t)macro * block;
    if (c == skip)
      res_group7<T, WRITE, NORM, true>(slice_consts(rs, N, k), N, j, g, c, u + mb, f + mb, r + mb, wr, ss);
    else
      res_group7<T, WRITE, NORM>(slice_consts(rs, N, k), N, j, g, c, u + mb, f + mb, r + mb, wr, ss);
  }
  if (NORM) {
    const double s = block_sum(ss, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Restriction R = P^T onto the coarse level (§2.1); zero the coarse correction
// ---------------------------------------------------------------------------
// Calls body(j, k, m) for every item of a tile: slot m of interior row j of
// slice k, i.e. the nodes i = 4m .. 4m + 3 (one per colour array), the items
// of all the tile's slices in one range (one CTA barrier per tile, as for the
// stencil kernels); ends with a CTA barrier.  The kernel declares
// s_pre2[MAX_SLABS][33] and s_pre_tot[MAX_SLABS + 1] in shared memory.
template <class F>
__device__ __forceinline__ void for_tile_slots(const Tile& t, int N, int (*s_pre2)[33], int* s_pre_tot, F&& body) {
  const int total = flat_setup_slabs(t, N, 0, false, 1, s_pre2, s_pre_tot);
  int sl = 0;
  for (int tt = tid256(); tt < total; tt += CTA) {
    while (tt >= s_pre_tot[sl + 1]) ++sl;
    const int k = t.k + sl;
    const Tile ts{k, t.j0, t.m0, 1};
    int j, m;
    flat_item(ts, N, 0, false, s_pre2[sl], tt - s_pre_tot[sl], j, m);
    body(j, k, m);
  }
  __syncthreads();
}

// Full-weighting restriction f_c = r(2I) + 1/2 sum_d r(2I + d) (d over the 14
// stencil directions, summed in their order) of the coarse nodes I = 4M ..
// 4M + 3 of interior row J of coarse slice K (one per colour array); the
// coarse correction there is zeroed.  The seven fine rows (2J + dj, 2K + dk)
// are located once per item; fine node i' = 8M + 2q + di lies in colour
// array (2q + di + 2 jf + 3 kf) & 3 at slot 2M + ((2q + di) >> 2), so every
// load is a row base plus constants.  All colours of the item in one pass
// keep the fine rows in cache for the four coarse nodes.  Plain loads when
// NC is false (data written in this launch).
template <class T, bool NC>
__device__ __forceinline__ void restrict_slot(int Nc, const int* __restrict__ rsc, int Nf,
                                              const int* __restrict__ rsf, int J, int K, int M,
                                              const T* __restrict__ rb, T* __restrict__ fcb, T* __restrict__ ucb) {
  const int Lc = Nc - 1 - J - K;
  const int CSf = __ldg(rsf + Nf + 2);
  int base[NDIR], col[NDIR];
#pragma unroll
  for (int d = 0; d < NDIR; ++d) {
    int di, dj, dk;
    dir_ijk(d, di, dj, dk);
    const int jf = 2 * J + dj, kf = 2 * K + dk;
    base[d] = row_base(rsf, Nf, jf, kf) + 2 * M;
    col[d] = 2 * jf + 3 * kf;
  }
  const int CSc = __ldg(rsc + Nc + 2);
  const int rbc = row_base(rsc, Nc, J, K) + M;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int I = 4 * M + q;
    if (I < 1 || I > Lc) continue;
    T cen = T(0), acc = T(0);
#pragma unroll
    for (int d = 0; d < NDIR; ++d) {
      int di, dj, dk;
      dir_ijk(d, di, dj, dk);
      const int o = ((2 * q + di + col[d]) & 3) * CSf + base[d] + ((2 * q + di) >> 2);
      const T x = NC ? __ldg(rb + o) : rb[o];
      if (d == 0) cen = x;
      else acc += x;
    }
    const int me = ((q + 2 * J + 3 * K) & 3) * CSc + rbc;
    fcb[me] = fma(T(0.5), acc, cen);   // the halving is exact: same value as a separate multiply
    ucb[me] = T(0);
  }
}

// Volume restriction of a coarse tile.
template <class T, bool NC>
__device__ __forceinline__ void restrict_tile(const Tile& t, int Nc, const int* __restrict__ rsc, int Nf,
                                              const int* __restrict__ rsf, const T* __restrict__ rb,
                                              T* __restrict__ fcb, T* __restrict__ ucb, int (*s_pre2)[33],
                                              int* s_pre_tot) {
  for_tile_slots(t, Nc, s_pre2, s_pre_tot, [&](int J, int K, int M) {
    restrict_slot<T, NC>(Nc, rsc, Nf, rsf, J, K, M, rb, fcb, ucb);
  });
}

template <class T>
__global__ void __launch_bounds__(CTA, 4) k_restrict(int Nc, const int* __restrict__ rsc, int64_t bc, T* __restrict__ fc, T* __restrict__ fIc,
                                                  T* __restrict__ uc, T* __restrict__ uIc, int Nf, const int* __restrict__ rsf, int64_t bf,
                                                  const T* __restrict__ rf, const Tile* __restrict__ tiles, int n_tiles,
                                                  const int* __restrict__ act, int n_act,
                                                  const int* __restrict__ cptr, const Copy* __restrict__ cps,
                                                  const uint32_t* __restrict__ cpo,
                                                  const int* __restrict__ list, int n_list,
                                                  const int64_t* __restrict__ gather,
                                                  const int64_t* __restrict__ zero_off, int n_zero, int n_if_units, int* __restrict__ sched) {
  __shared__ int s_pre2[MAX_SLABS][33];
  __shared__ int s_pre_tot[MAX_SLABS + 1];
  __shared__ int s_unit;
  HHG_UNITS_DYN(n_if_units, n_tiles * RESTRICT_SPLIT, n_act, sched, &s_unit) {
    if (const int ic_ = if_chunk(unit, n_if_units); ic_ >= 0) {
      const int q = ic_ * CTA + tid256();
      if (q < n_list) {
        const int node = list[q];
        const int64_t* g = gather + (size_t)q * NDIR;
        T acc = T(0);
        for (int e = 1; e < NDIR; ++e) {
          const int64_t o = g[e];
          if (o >= 0) acc += rf[o];
        }
        fIc[node] = rf[g[0]] + T(0.5) * acc;
        uIc[node] = T(0);
        write_copies(Nc, rsc, bc, uc, cps, cpo, cptr[node], cptr[node + 1], T(0));
      } else if (q < n_list + n_zero) {
        uc[zero_off[q - n_list]] = T(0);
      }
      continue;
    }
    Tile t;
    int macro;
    vol_subunit(vol_index(unit, n_if_units), n_act, RESTRICT_SPLIT, tiles, act, t, macro);
    restrict_tile<T, true>(t, Nc, rsc, Nf, rsf, rf + (size_t)macro * bf, fc + (size_t)macro * bc,
                           uc + (size_t)macro * bc, s_pre2, s_pre_tot);
  }
  finish_units(sched, n_if_units + n_tiles * RESTRICT_SPLIT * n_act);
}

// ---------------------------------------------------------------------------
// Prolongation u_f += P u_c (linear interpolation, §2.1)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T interp(const T* __restrict__ cb, int Nc, const int* __restrict__ rsc, int i, int j, int k) {
  const int pi = i & 1, pj = j & 1, pk = k & 1;
  if (!(pi | pj | pk)) return cb[lidx32(rsc, Nc, i >> 1, j >> 1, k >> 1)];
  // the coarse edge through a fine midpoint: parity -> local direction
  int di, dj, dk;
  const int code = pi | (pj << 1) | (pk << 2);
  switch (code) {
    case 1: di = 1; dj = 0; dk = 0; break;
    case 2: di = 0; dj = 1; dk = 0; break;
    case 4: di = 0; dj = 0; dk = 1; break;
    case 3: di = -1; dj = 1; dk = 0; break;
    case 5: di = -1; dj = 0; dk = 1; break;
    case 6: di = 0; dj = -1; dk = 1; break;
    default: di = 1; dj = -1; dk = 1; break;
  }
  const T a = cb[lidx32(rsc, Nc, (i - di) >> 1, (j - dj) >> 1, (k - dk) >> 1)];
  const T b = cb[lidx32(rsc, Nc, (i + di) >> 1, (j + dj) >> 1, (k + dk) >> 1)];
  return T(0.5) * (a + b);
}

// Coarse edge through a fine node of parities (pi, pj, pk), not all zero: the
// fine node is the midpoint of coarse nodes (i -+ di, j -+ dj, k -+ dk) / 2.
__device__ __forceinline__ void edge_dir(int code, int& di, int& dj, int& dk) {
  switch (code) {
    case 1: di = 1; dj = 0; dk = 0; break;
    case 2: di = 0; dj = 1; dk = 0; break;
    case 4: di = 0; dj = 0; dk = 1; break;
    case 3: di = -1; dj = 1; dk = 0; break;
    case 5: di = -1; dj = 0; dk = 1; break;
    case 6: di = 0; dj = -1; dk = 1; break;
    default: di = 1; dj = -1; dk = 1; break;
  }
}

// Prolongation u_f += P u_c of the fine nodes i = 4m .. 4m + 3 of interior
// row j of fine slice k (one per colour array; fine block fb, coarse block
// cb).  The parities of a node are (q & 1, j & 1, k & 1), so an item has two
// interpolation cases (even and odd i): the coarse node (i/2, j/2, k/2) when
// all parities are even, else the mean of the coarse edge's two ends.  Their
// coarse rows are located once per item; coarse node I = 2m + const lies in
// colour array (I + 2J + 3K) & 3 at slot I >> 2.  Plain loads for the fine
// values (written by this launch), the read-only path for the coarse ones
// when NC.  Nodes of colour skip are left out (-1: none).
template <class T, bool NC>
__device__ __forceinline__ void prolong_slot(int Nf, const int* __restrict__ rsf, int Nc, const int* __restrict__ rsc,
                                             int j, int k, int m, T* __restrict__ fb, const T* __restrict__ cb,
                                             int skip) {
  const int L = Nf - 1 - j - k;
  const int CSf = __ldg(rsf + Nf + 2), CSc = __ldg(rsc + Nc + 2);
  const int rbf = row_base(rsf, Nf, j, k) + m;
  const int cf = 2 * j + 3 * k;
  // per parity of i: direction, the two coarse rows and their colour terms
  int di[2], rba[2], rbb[2], ca[2], cbb[2], code[2];
#pragma unroll
  for (int par = 0; par < 2; ++par) {
    code[par] = par | ((j & 1) << 1) | ((k & 1) << 2);
    int dj = 0, dk = 0;
    di[par] = 0;
    if (code[par]) edge_dir(code[par], di[par], dj, dk);
    const int JA = (j - dj) >> 1, KA = (k - dk) >> 1, JB = (j + dj) >> 1, KB = (k + dk) >> 1;
    rba[par] = row_base(rsc, Nc, JA, KA);
    rbb[par] = row_base(rsc, Nc, JB, KB);
    ca[par] = 2 * JA + 3 * KA;
    cbb[par] = 2 * JB + 3 * KB;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 4 * m + q;
    if (i < 1 || i > L || ((q + cf) & 3) == skip) continue;
    const int par = q & 1;
    T* out = fb + ((q + cf) & 3) * CSf + rbf;
    const T u = *out;
    if (code[par] == 0) {
      const int I = 2 * m + (q >> 1);
      const int o = ((I + ca[par]) & 3) * CSc + rba[par] + (I >> 2);
      *out = u + (NC ? __ldg(cb + o) : cb[o]);
    } else {
      const int IA = 2 * m + ((q - di[par]) >> 1), IB = 2 * m + ((q + di[par]) >> 1);
      const int oa = ((IA + ca[par]) & 3) * CSc + rba[par] + (IA >> 2);
      const int ob = ((IB + cbb[par]) & 3) * CSc + rbb[par] + (IB >> 2);
      const T a = NC ? __ldg(cb + oa) : cb[oa];
      const T b = NC ? __ldg(cb + ob) : cb[ob];
      *out = fma(T(0.5), a + b, u);   // the halving is exact: same value as a separate multiply
    }
  }
}

// The same prolongation for the colour-c nodes in slots m0 .. m0 + VW - 1 of
// interior row j of fine slice k, one 16-byte vector of fine values: all
// nodes i = 4m + ic of a colour row share their parities, hence one case.
template <class T, bool NC>
__device__ __forceinline__ void prolong_group(int Nf, const int* __restrict__ rsf, int Nc, const int* __restrict__ rsc,
                                              int j, int k, int g, int c, T* __restrict__ fb,
                                              const T* __restrict__ cb) {
  constexpr int VW = Vec<T>::n;
  int ic, mlo, n;
  colour_row(Nf, j, k, c, ic, mlo, n);
  const int m0 = g * VW;
  const int lo = max(mlo - m0, 0), hi = min(mlo + n - m0, VW);
  T* out = fb + c * __ldg(rsf + Nf + 2) + row_base(rsf, Nf, j, k) + m0;
  T v[VW];
  Vec<T>::template load<false>(out, v);
  const int CSc = __ldg(rsc + Nc + 2);
  const int code = (ic & 1) | ((j & 1) << 1) | ((k & 1) << 2);
  int di = 0, dj = 0, dk = 0;
  if (code) edge_dir(code, di, dj, dk);
  const int JA = (j - dj) >> 1, KA = (k - dk) >> 1, ia = (ic - di) >> 1;
  const int JB = (j + dj) >> 1, KB = (k + dk) >> 1, ib = (ic + di) >> 1;
  const int rba = row_base(rsc, Nc, JA, KA), rbb = row_base(rsc, Nc, JB, KB);
  const int ca = ia + 2 * JA + 3 * KA, cbb = ib + 2 * JB + 3 * KB;
#pragma unroll
  for (int q = 0; q < VW; ++q) {
    if (q < lo || q >= hi) continue;
    const int two_m = 2 * (m0 + q);
    const int oa = ((ca + two_m) & 3) * CSc + rba + ((two_m + ia) >> 2);
    const T a = NC ? __ldg(cb + oa) : cb[oa];
    if (code == 0) {
      v[q] += a;
    } else {
      const int ob = ((cbb + two_m) & 3) * CSc + rbb + ((two_m + ib) >> 2);
      const T b = NC ? __ldg(cb + ob) : cb[ob];
      v[q] = fma(T(0.5), a + b, v[q]);   // the halving is exact: same value as a separate multiply
    }
  }
  store_lanes(out, v, lo, hi);
}

// Volume prolongation of a fine tile: FP64 one item per slot (four nodes,
// all colours), FP32 colour by colour in 16-byte vectors (measured faster for
// each precision); colour skip left out (-1: none).
template <class T, bool NC>
__device__ __forceinline__ void prolong_tile(const Tile& t, int Nf, const int* __restrict__ rsf, int Nc,
                                             const int* __restrict__ rsc, T* __restrict__ fb, const T* __restrict__ cb,
                                             int skip, int (*s_pre2)[33], int* s_pre_tot) {
  if constexpr (std::is_same<T, float>::value) {
    constexpr int VW = Vec<T>::n;
    for (int c = 0; c < 4; ++c) {
      if (c == skip) continue;
      const int total = flat_setup_slabs(t, Nf, c, true, VW, s_pre2, s_pre_tot);
      int sl = 0;
      for (int tt = tid256(); tt < total; tt += CTA) {
        while (tt >= s_pre_tot[sl + 1]) ++sl;
        const int k = t.k + sl;
        const Tile ts{k, t.j0, t.m0, 1};
        int j, g;
        flat_item(ts, Nf, c, true, s_pre2[sl], tt - s_pre_tot[sl], j, g, VW);
        prolong_group<T, NC>(Nf, rsf, Nc, rsc, j, k, g, c, fb, cb);
      }
      __syncthreads();
    }
  } else {
    for_tile_slots(t, Nf, s_pre2, s_pre_tot, [&](int j, int k, int m) {
      prolong_slot<T, NC>(Nf, rsf, Nc, rsc, j, k, m, fb, cb, skip);
    });
  }
}

template <class T>
__global__ void __launch_bounds__(CTA) k_prolong(int Nf, const int* __restrict__ rsf, int64_t bf, T* __restrict__ uf, T* __restrict__ uIf,
                                                 int Nc, const int* __restrict__ rsc, int64_t bc, const T* __restrict__ uc,
                                                 const Tile* __restrict__ tiles, int n_tiles,
                                                 const int* __restrict__ act, int n_act, const int* __restrict__ cptr,
                                                 const Copy* __restrict__ cps, const uint32_t* __restrict__ cpo,
                                                 const int* __restrict__ list,
                                                 int n_list, int n_if_units, int* __restrict__ sched, int skip,
                                                 int if_lo, int if_hi) {
  __shared__ int s_pre2[MAX_SLABS][33];
  __shared__ int s_pre_tot[MAX_SLABS + 1];
  __shared__ int s_unit;
  HHG_UNITS_DYN(n_if_units, n_tiles, n_act, sched, &s_unit) {
    if (const int ic_ = if_chunk(unit, n_if_units); ic_ >= 0) {
      const int q = ic_ * CTA + tid256();
      if (q < n_list && (q < if_lo || q >= if_hi)) {
        const int node = list[q];
        const int c0 = cptr[node], c1 = cptr[node + 1];
        const Copy cp = cps[c0];
        const T val = uIf[node] + interp(uc + (size_t)cp.macro * bc, Nc, rsc, cp.i, cp.j, cp.k);
        uIf[node] = val;
        write_copies(Nf, rsf, bf, uf, cps, cpo, c0, c1, val);
      }
      continue;
    }
    Tile t;
    int macro;
    vol_unit(vol_index(unit, n_if_units), n_act, tiles, act, t, macro);
    prolong_tile<T, true>(t, Nf, rsf, Nc, rsc, uf + (size_t)macro * bf, uc + (size_t)macro * bc, skip, s_pre2,
                          s_pre_tot);
  }
  finish_units(sched, n_if_units + n_tiles * n_act);
}

// Flat transfers (levels on the flat kernels): one thread per item, no tiles
// and no CTA barrier, CTAs of interface nodes spread among the volume CTAs.
// The restriction takes the coarse level's slot items (four coarse nodes of
// one row per thread, restrict_slot); the prolongation takes the fine level's
// Gauss-Seidel items of the colours it updates (one 16-byte vector of
// same-colour fine nodes per thread, prolong_group).  Same arithmetic per
// node as k_restrict / k_prolong, so the same values bit for bit.
template <class T>
__global__ void __launch_bounds__(CTA) k_restrict_flat(int Nc, const int* __restrict__ rsc, int64_t bc,
                                                       T* __restrict__ fc, T* __restrict__ fIc, T* __restrict__ uc,
                                                       T* __restrict__ uIc, int Nf, const int* __restrict__ rsf,
                                                       int64_t bf, const T* __restrict__ rf,
                                                       const uint32_t* __restrict__ slots, int n_slots,
                                                       const int* __restrict__ act, int n_act,
                                                       const int* __restrict__ cptr, const Copy* __restrict__ cps,
                                                       const uint32_t* __restrict__ cpo, const int* __restrict__ list,
                                                       int n_list, const int64_t* __restrict__ gather,
                                                       const int64_t* __restrict__ zero_off, int n_zero,
                                                       int n_if_ctas, int n_vol_ctas) {
  int vb = 0;
  const int ib = spread_position((int)blockIdx.x, n_if_ctas, n_vol_ctas, vb);
  if (ib >= 0) {
    const int q = ib * CTA + tid256();
    if (q < n_list) {
      const int node = list[q];
      const int64_t* g = gather + (size_t)q * NDIR;
      T acc = T(0);
      for (int e = 1; e < NDIR; ++e) {
        const int64_t o = g[e];
        if (o >= 0) acc += rf[o];
      }
      fIc[node] = rf[g[0]] + T(0.5) * acc;
      uIc[node] = T(0);
      write_copies(Nc, rsc, bc, uc, cps, cpo, cptr[node], cptr[node + 1], T(0));
    } else if (q < n_list + n_zero) {
      uc[zero_off[q - n_list]] = T(0);
    }
    return;
  }
  const int v = vb * CTA + tid256();
  if (v >= n_slots * n_act) return;
  const int a = v / n_slots, it = v - a * n_slots;
  const int macro = act[a];
  const uint32_t d = slots[it];
  restrict_slot<T, true>(Nc, rsc, Nf, rsf, (int)(d >> 20), (int)((d >> 10) & 1023u), (int)(d & 1023u),
                         rf + (size_t)macro * bf, fc + (size_t)macro * bc, uc + (size_t)macro * bc);
}

// items / n_items: the fine level's Gauss-Seidel items of colours first_c ..
// 3 (colour-major, from off[first_c] on); off holds the starts of the later
// colours relative to that (n_items where there is none), to find an item's
// colour.
template <class T>
__global__ void __launch_bounds__(CTA) k_prolong_flat(int Nf, const int* __restrict__ rsf, int64_t bf,
                                                      T* __restrict__ uf, T* __restrict__ uIf, int Nc,
                                                      const int* __restrict__ rsc, int64_t bc,
                                                      const T* __restrict__ uc, const uint32_t* __restrict__ items,
                                                      int n_items, int first_c, int3 off,
                                                      const int* __restrict__ act, int n_act,
                                                      const int* __restrict__ cptr, const Copy* __restrict__ cps,
                                                      const uint32_t* __restrict__ cpo,
                                                      const int* __restrict__ list, int n_list, int if_lo, int if_hi,
                                                      int n_if_ctas, int n_vol_ctas) {
  int vb = 0;
  const int ib = spread_position((int)blockIdx.x, n_if_ctas, n_vol_ctas, vb);
  if (ib >= 0) {
    const int q = ib * CTA + tid256();
    if (q < n_list && (q < if_lo || q >= if_hi)) {
      const int node = list[q];
      const int c0 = cptr[node], c1 = cptr[node + 1];
      const Copy cp = cps[c0];
      const T val = uIf[node] + interp(uc + (size_t)cp.macro * bc, Nc, rsc, cp.i, cp.j, cp.k);
      uIf[node] = val;
      write_copies(Nf, rsf, bf, uf, cps, cpo, c0, c1, val);
    }
    return;
  }
  const int v = vb * CTA + tid256();
  if (v >= n_items * n_act) return;
  const int a = v / n_items, it = v - a * n_items;
  const int c = first_c + (it >= off.x) + (it >= off.y) + (it >= off.z);
  const int macro = act[a];
  const uint32_t d = items[it];
  prolong_group<T, true>(Nf, rsf, Nc, rsc, (int)(d >> 20), (int)((d >> 10) & 1023u), (int)(d & 1023u), c,
                         uf + (size_t)macro * bf, uc + (size_t)macro * bc);
}

// ---------------------------------------------------------------------------
// Mixed precision: FP64 residual handed to the FP32 cycle as its right-hand
// side (with partial sums of r^2), and the FP64 update u += e
// ---------------------------------------------------------------------------
template <bool S7>
__global__ void __launch_bounds__(CTA) k_res_f32(int N, const int* __restrict__ rs, int64_t block, const double* __restrict__ u,
                                                 const double* __restrict__ uI, const double* __restrict__ f,
                                                 const double* __restrict__ fI, float* __restrict__ f32,
                                                 float* __restrict__ fI32, const double* __restrict__ W,
                                                 const Tile* __restrict__ tiles, int n_tiles,
                                                 const int* __restrict__ act, int n_act,
                                                 const int* __restrict__ cptr, const Copy* __restrict__ cps,
                                                 const int* __restrict__ list, int n_list, IfTab<double> tab,
                                                 int n_if_units, double* __restrict__ partial,
                                                 int* __restrict__ sched) {
  __shared__ int s_pre2[MAX_SLABS][33];
  __shared__ int s_pre_tot[MAX_SLABS + 1];
  __shared__ double sh[32];
  double ss = 0.0;
  __shared__ int s_unit;
  HHG_UNITS_DYN(n_if_units, n_tiles, n_act, sched, &s_unit) {
    int vol_ = 0;
    if (const int ic_ = spread_unit(unit, n_if_units, n_tiles * n_act, vol_); ic_ >= 0) {
      const int q = ic_ * CTA + tid256();
      if (q < n_list) {
        const int node = list[q];
        double res;
        if (tab.nb) {
          res = fI[node] - tab.diag[q] * uI[node] - if_offdiag<double, if_tab_k(S7)>(tab, u, q);
        } else {
          double off = 0.0, diag = 0.0;
          if_stencil<double, S7>(N, rs, block, u, W, cps, cptr[node], cptr[node + 1], off, diag);
          res = fI[node] - diag * uI[node] - off;
        }
        fI32[node] = (float)res;
        ss += res * res;
      }
      continue;
    }
    Tile t;
    int macro;
    vol_unit(vol_, n_act, tiles, act, t, macro);
    const double* ub = u + (size_t)macro * block;
    const double* fb = f + (size_t)macro * block;
    float* ob = f32 + (size_t)macro * block;
    const double* w = W + (size_t)macro * 16 * NDIR;
    HHG_TILE_NODES(N, rs, t, s_pre, {
      int me;
      double acc;
      if (S7) {
        const Nb7 q = nb7(sc, i, j);
        me = q.me;
        acc = fb[me] - w[0] * ub[me];
        acc -= w[1] * ub[q.nb1];
        acc -= w[2] * ub[q.nb2];
        acc -= w[3] * ub[q.nb3];
        acc -= w[8] * ub[q.nb8];
        acc -= w[9] * ub[q.nb9];
        acc -= w[10] * ub[q.nb10];
      } else {
        me = lidx32(rs, N, i, j, k);
        acc = fb[me] - w[0] * ub[me];
_Pragma("unroll")
        for (int d = 1; d < NDIR; ++d) {
          int di, dj, dk;
          dir_ijk(d, di, dj, dk);
          acc -= w[d] * ub[lidx32(rs, N, i + di, j + dj, k + dk)];
        }
      }
      ob[me] = (float)acc;
      ss += acc * acc;
    })
  }
  finish_units(sched, n_if_units + n_tiles * n_act);
  const double s = block_sum(ss, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.x] = s;
}

// u64 += e32 over whole active blocks, two slots per thread and step: the
// FP32 correction is zero at every slot the cycle does not own (Dirichlet and
// frozen copies, padding; the blocks are cleared before the cycle), and each
// ghost copy of a free interface node holds the master's correction, so the
// copies stay equal to their masters.  Blocks are multiples of 256 slots.
__global__ void __launch_bounds__(256) k_add_corr_blocks(double* __restrict__ u, const float* __restrict__ e,
                                                        int64_t block, const int* __restrict__ act) {
  const size_t base = (size_t)act[blockIdx.y] * block;
  double2* ub = reinterpret_cast<double2*>(u + base);
  const float2* eb = reinterpret_cast<const float2*>(e + base);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < block / 2; q += (int64_t)gridDim.x * blockDim.x) {
    double2 x = ub[q];
    const float2 d = __ldg(eb + q);
    x.x += (double)d.x;
    x.y += (double)d.y;
    ub[q] = x;
  }
}

// uI[list[q]] += eI[list[q]] for the free interface masters.
__global__ void k_add_corr_masters(double* __restrict__ uI, const float* __restrict__ eI, const int* __restrict__ list,
                                   int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) {
    const int node = list[q];
    uI[node] += (double)eI[node];
  }
}

// ---------------------------------------------------------------------------
// Coarse-level CG, one CTA (FP64; §2.1 coarse solver)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cta_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    // only the first blockDim.x / 32 entries were written
    double s = threadIdx.x < (blockDim.x + 31) / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) sh[32] = s;
  }
  __syncthreads();
  return sh[32];
}

constexpr int CG_THREADS = 256;

// Sum of v over the CTA (CG_THREADS threads), returned to every thread in the
// same order (warp partials 0..7); buf holds the warp partials.  Consecutive
// reductions alternate between two buffers.
__device__ __forceinline__ double cg_allreduce(double v, double* buf) {
  const int t = threadIdx.y * blockDim.x + threadIdx.x;   // 1-D or (32, 8) CTAs
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((t & 31) == 0) buf[t >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < CG_THREADS / 32; ++w) s += buf[w];
  return s;
}

// CG on the compact free nodes of the coarsest level from x = 0 until
// ||r|| <= rtol ||b|| or maxit iterations.  x, r, p and A p live in shared
// memory (smem != 0) or in the global work array (4 n doubles).  Each
// iteration: A p and p.Ap (one reduction), the updates of x and r and r.r
// (one reduction), the new direction; row q belongs to thread q mod
// CG_THREADS throughout.
template <class T>
__global__ void __launch_bounds__(CG_THREADS) k_cg(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                                   const double* __restrict__ val, const int64_t* __restrict__ fsrc,
                                                   const T* __restrict__ f, const T* __restrict__ fI,
                                                   const int* __restrict__ uptr, const int64_t* __restrict__ udst,
                                                   const int* __restrict__ umaster, T* __restrict__ u,
                                                   T* __restrict__ uI, double* __restrict__ work, double rtol,
                                                   int maxit, int* __restrict__ iters, int smem) {
  extern __shared__ double s_cg[];
  __shared__ double red[2][CG_THREADS / 32];
  double* x = smem ? s_cg : work;
  double* r = x + n;
  double* p = r + n;
  double* Ap = p + n;
  double part = 0.0;
  for (int q = threadIdx.x; q < n; q += CG_THREADS) {
    const int64_t s = fsrc[q];
    const double b = s >= 0 ? (double)f[s] : (double)fI[-1 - s];
    x[q] = 0.0;
    r[q] = b;
    p[q] = b;
    part += b * b;
  }
  double rr = cg_allreduce(part, red[0]);
  int rb = 1;
  const double bnorm = sqrt(rr);
  int it = 0;
  while (bnorm > 0.0 && sqrt(rr) > rtol * bnorm && it < maxit) {
    __syncthreads();   // every p entry written before A p reads it
    part = 0.0;
    for (int q = threadIdx.x; q < n; q += CG_THREADS) {
      double a = 0.0;
      for (int e = __ldg(rowptr + q); e < __ldg(rowptr + q + 1); ++e) a += __ldg(val + e) * p[__ldg(col + e)];
      Ap[q] = a;
      part += p[q] * a;
    }
    const double pAp = cg_allreduce(part, red[rb]);
    rb ^= 1;
    const double alpha = rr / pAp;
    part = 0.0;
    for (int q = threadIdx.x; q < n; q += CG_THREADS) {
      x[q] += alpha * p[q];
      const double rq = r[q] - alpha * Ap[q];
      r[q] = rq;
      part += rq * rq;
    }
    const double rr_new = cg_allreduce(part, red[rb]);
    rb ^= 1;
    const double beta = rr_new / rr;
    for (int q = threadIdx.x; q < n; q += CG_THREADS) p[q] = r[q] + beta * p[q];
    rr = rr_new;
    ++it;
  }
  for (int q = threadIdx.x; q < n; q += CG_THREADS) {
    const T v = (T)x[q];
    for (int e = uptr[q]; e < uptr[q + 1]; ++e) u[udst[e]] = v;
    if (umaster[q] >= 0) uI[umaster[q]] = v;
  }
  if (threadIdx.x == 0 && iters) *iters = it;
}

// Coefficient gradient (per macro, closed lattice): sum of lam_p times the
// macro's own sub-stencil at p applied to u, i.e. lam^T (A_T u) up to the
// factor k_T.
__global__ void __launch_bounds__(CTA) k_grad(int N, const int* __restrict__ rs, int64_t block,
                                              const double* __restrict__ u, const double* __restrict__ lam,
                                              const double* __restrict__ W, const Tile* __restrict__ tiles,
                                              double* __restrict__ partial) {
  __shared__ double sh[32];
  const Tile t = tiles[blockIdx.x];
  const int macro = blockIdx.y;
  const int k = t.k;
  const int j = t.j0 + threadIdx.y;
  const int m = t.m0 + threadIdx.x;
  const double* ub = u + (size_t)macro * block;
  const double* lb = lam + (size_t)macro * block;
  const double* Wm = W + (size_t)macro * 16 * NDIR;
  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 4 * m + q;
    if (i + j + k > N) continue;
    const int me = lidx32(rs, N, i, j, k);
    const double l = lb[me];
    if (l == 0.0) continue;
    const double* w = Wm + node_class(i, j, k, N) * NDIR;
    double sv = w[0] * ub[me];
    for (int d = 1; d < NDIR; ++d) {
      const double wd = w[d];
      if (wd == 0.0) continue;
      int di, dj, dk;
      dir_ijk(d, di, dj, dk);
      if (!in_lattice(i + di, j + dj, k + dk, N)) continue;
      sv += wd * ub[lidx32(rs, N, i + di, j + dj, k + dk)];
    }
    acc += l * sv;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[(size_t)macro * gridDim.x + blockIdx.x] = s;
}

__global__ void k_reduce_per_macro(const double* __restrict__ partial, int n_per, double* __restrict__ out) {
  __shared__ double sh[33];
  double s = 0.0;
  const double* p = partial + (size_t)blockIdx.x * n_per;
  for (int q = threadIdx.x; q < n_per; q += blockDim.x) s += p[q];
  s = cta_sum(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

__global__ void k_reduce(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double sh[33];
  double s = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += partial[q];
  s = cta_sum(s, sh);
  if (threadIdx.x == 0) out[0] = s;
}

// FP64 FMA throughput probe (measurement support): every thread runs eight
// independent FMA chains of `iters` steps and writes their sum.
__global__ void __launch_bounds__(256) k_fma_probe(double* __restrict__ out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = threadIdx.x * 1e-3 + q;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ---------------------------------------------------------------------------
// Global vector <-> blocks (closed-lattice tiles: 8 rows x 32 slots)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t dev_gid(const MacroGeo& g, int N, int i, int j, int k, int64_t nx, int64_t ny) {
  const int64_t X = (int64_t)N * g.v0[0] + (int64_t)i * g.e1[0] + (int64_t)j * g.e2[0] + (int64_t)k * g.e3[0];
  const int64_t Y = (int64_t)N * g.v0[1] + (int64_t)i * g.e1[1] + (int64_t)j * g.e2[1] + (int64_t)k * g.e3[1];
  const int64_t Z = (int64_t)N * g.v0[2] + (int64_t)i * g.e1[2] + (int64_t)j * g.e2[2] + (int64_t)k * g.e3[2];
  return (Z * (ny + 1) + Y) * (nx + 1) + X;
}

template <class T>
__global__ void __launch_bounds__(CTA) k_import_vol(int N, const int* __restrict__ rs, int64_t block, const MacroGeo* __restrict__ geo,
                                                    int64_t nx, int64_t ny, const double* __restrict__ g,
                                                    T* __restrict__ dst, const Tile* __restrict__ tiles, bool closed) {
  const Tile t = tiles[blockIdx.x];
  const int macro = blockIdx.y;
  const int k = t.k;
  const int j = t.j0 + threadIdx.y;
  const int m = t.m0 + threadIdx.x;
  const MacroGeo gm = geo[macro];
  T* b = dst + (size_t)macro * block;
  const int lo = closed ? 0 : 1, top = closed ? N : N - 1;
  if (j < lo) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 4 * m + q;
    if (i < lo || i + j + k > top) continue;
    b[lidx32(rs, N, i, j, k)] = (T)g[dev_gid(gm, N, i, j, k, nx, ny)];
  }
}

template <class T>
__global__ void __launch_bounds__(CTA) k_export_vol(int N, const int* __restrict__ rs, int64_t block, const MacroGeo* __restrict__ geo,
                                                    int64_t nx, int64_t ny, const T* __restrict__ src,
                                                    double* __restrict__ g, const Tile* __restrict__ tiles) {
  const Tile t = tiles[blockIdx.x];
  const int macro = blockIdx.y;
  const int k = t.k;
  const int j = t.j0 + threadIdx.y;
  const int m = t.m0 + threadIdx.x;
  const MacroGeo gm = geo[macro];
  const T* b = src + (size_t)macro * block;
  if (j < 1 || k < 1) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 4 * m + q;
    if (i < 1 || i + j + k > N - 1) continue;
    g[dev_gid(gm, N, i, j, k, nx, ny)] = (double)b[lidx32(rs, N, i, j, k)];
  }
}

template <class T>
__global__ void k_import_if(const int64_t* __restrict__ gid, int n, const double* __restrict__ g, T* __restrict__ m) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) m[q] = (T)g[gid[q]];
}

template <class T>
__global__ void k_export_if(const int64_t* __restrict__ gid, int n, const T* __restrict__ m, double* __restrict__ g) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) g[gid[q]] = (double)m[q];
}

// out[node] = (A u)_node over the copies listed for each node (the healthy
// copies give A_I, the flux of the healthy side at an interface node).
template <bool S7>
__global__ void k_if_apply(int N, const int* __restrict__ rs, int64_t block, const double* __restrict__ u,
                           const double* __restrict__ uI, const double* __restrict__ W, const int* __restrict__ cptr,
                           const Copy* __restrict__ cps, const int* __restrict__ list, int n, double* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int node = list[q];
  double off = 0.0, diag = 0.0;
  if_stencil<double, S7>(N, rs, block, u, W, cps, cptr[node], cptr[node + 1], off, diag);
  out[node] = diag * uI[node] + off;
}

__global__ void k_copy_listed(const double* __restrict__ src, double* __restrict__ dst, const int* __restrict__ idx,
                              int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) dst[idx[q]] = src[idx[q]];
}

__global__ void k_scale_blocks(const double* __restrict__ f, const double* __restrict__ winv,
                               double* __restrict__ out, int n_macro, int64_t block) {
  const int64_t total = (int64_t)n_macro * block;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
    out[q] = f[q] * winv[q / block];
}

__global__ void k_set_masters_zero(double* __restrict__ uI, const int* __restrict__ ids, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) uI[ids[q]] = 0.0;
}

__global__ void k_restore(double* __restrict__ u, const double* __restrict__ uI, const int64_t* __restrict__ off,
                          const int* __restrict__ master, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) u[off[q]] = uI[master[q]];
}

template <class T>
__global__ void k_zero_blocks(T* __restrict__ u, int64_t block, const int* __restrict__ act) {
  T* b = u + (size_t)act[blockIdx.y] * block;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < block; q += (int64_t)gridDim.x * blockDim.x)
    b[q] = T(0);
}

template <class T>
__global__ void k_zero_list(T* __restrict__ uI, const int* __restrict__ list, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) uI[list[q]] = T(0);
}

inline unsigned lin_grid(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// The problem's interface table in precision T, starting at list entry off.
template <class T>
IfTab<T> if_tab(const ProbArgs& p, int off);
template <>
IfTab<double> if_tab<double>(const ProbArgs& p, int off) {
  IfTab<double> t{nullptr, nullptr, nullptr, nullptr, 0};
  if (p.tnb && p.tw64) t = IfTab<double>{p.tnb + off, p.tw64 + off, p.td64 + off, p.ti64 + off, p.tn};
  return t;
}
template <>
IfTab<float> if_tab<float>(const ProbArgs& p, int off) {
  IfTab<float> t{nullptr, nullptr, nullptr, nullptr, 0};
  if (p.tnb && p.tw32) t = IfTab<float>{p.tnb + off, p.tw32 + off, p.td32 + off, p.ti32 + off, p.tn};
  return t;
}
inline dim3 cta_shape() { return dim3(TILE_SLOTS, TILE_ROWS); }

// Grid of a fused launch: interface units first, then tiles x active macros;
// at most as many CTAs as the GPU holds at once (occupancy of the kernel
// times the SM count), each walking the units with a grid stride.
struct Units {
  int n_if_units, total;
};
inline Units units(int n_if_items, int n_tiles, int n_act) {
  Units g;
  g.n_if_units = (int)lin_grid(n_if_items, CTA);
  g.total = g.n_if_units + (n_act > 0 ? n_tiles * n_act : 0);
  return g;
}

std::mutex g_occ_mu;
std::map<std::pair<const void*, int>, int> g_occ;   // (kernel, device) -> resident CTAs

// cap > 0 limits the grid further (a smaller grid makes a launch take the
// dynamic walk at smaller sizes).
inline unsigned resident_grid(const void* kernel, int total, int cap_limit = 0) {
  int dev = 0;
  cudaGetDevice(&dev);
  int cap = 0;
  {
    std::lock_guard<std::mutex> lock(g_occ_mu);
    auto it = g_occ.find({kernel, dev});
    if (it != g_occ.end()) {
      cap = it->second;
    } else {
      int sms = 0, per_sm = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, CTA, 0);
      cap = std::max(1, sms * std::max(1, per_sm));
      g_occ[{kernel, dev}] = cap;
    }
  }
  if (cap_limit > 0) cap = std::min(cap, cap_limit);
  return (unsigned)std::min(total, cap);
}

// ---------------------------------------------------------------------------
// Persistent batch executor.  One launch runs the programs of many tasks (a
// program is the list of level-wide operations one task issues, recorded
// from the launchers; see hhg_kernels.h).  A CTA takes the next unit of the
// current operation of some task (per-operation counters of units handed out
// and finished); the CTA that finishes an operation's last unit publishes the
// task's next operation.  Units of one operation are independent, as in the
// level kernels; the publishing thread fences after the CTA's writes, and a
// CTA fences after reading a task's operation index and before reading its
// data (no read-only-path loads of data written in the launch), so every
// operation sees its predecessors' results.  A CTA never waits inside a
// unit, so some CTA always makes progress; a CTA that finds no work waits
// (bounded) and retries, and stops when every task has finished.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <class T>
__device__ __forceinline__ IfTab<T> dev_if_tab(const ProbArgs& p, int off);
template <>
__device__ __forceinline__ IfTab<double> dev_if_tab<double>(const ProbArgs& p, int off) {
  IfTab<double> t{nullptr, nullptr, nullptr, nullptr, 0};
  if (p.tnb && p.tw64) t = IfTab<double>{p.tnb + off, p.tw64 + off, p.td64 + off, p.ti64 + off, p.tn};
  return t;
}
template <>
__device__ __forceinline__ IfTab<float> dev_if_tab<float>(const ProbArgs& p, int off) {
  IfTab<float> t{nullptr, nullptr, nullptr, nullptr, 0};
  if (p.tnb && p.tw32) t = IfTab<float>{p.tnb + off, p.tw32 + off, p.td32 + off, p.ti32 + off, p.tn};
  return t;
}

// Unit `unit` of a Gauss-Seidel colour (k_gs).
template <class T, bool S7>
__device__ void unit_gs(const BOp& op, int unit, int (*s_pre2)[33], int* s_pre_tot) {
  const LevelArgs& L = op.L;
  const ProbArgs& p = op.P;
  const int N = L.N;
  const int* rs = L.rs;
  const int64_t block = L.block;
  T* u = (T*)op.u;
  if (unit < op.n_if_units) {
    const int q = unit * CTA + tid256();
    if (q < op.n_list) {
      T* uI = (T*)op.uI;
      const T* fI = (const T*)op.fI;
      const int node = p.free_if[op.list_off + q];
      const int c0 = L.cptr[node], c1 = L.cptr[node + 1];
      const IfTab<T> tab = dev_if_tab<T>(p, op.list_off);
      T val;
      if (tab.nb) {
        val = (fI[node] - if_offdiag<T, if_tab_k(S7)>(tab, u, q)) * tab.dinv[q];
      } else {
        T off = T(0), diag = T(0);
        if_stencil<T, S7>(N, rs, block, u, (const T*)op.W, L.cps, c0, c1, off, diag);
        val = (fI[node] - off) / diag;
      }
      uI[node] = val;
      write_copies(N, rs, block, u, L.cps, L.cp_off, c0, c1, val);
    }
    return;
  }
  const int vb = unit - op.n_if_units;
  const Tile t = L.tiles_int[vb / p.n_act];
  const int macro = p.act[vb % p.n_act];
  T* ub = u + (size_t)macro * block;
  const T* w = (const T*)op.Wv + (size_t)macro * 16 * NDIR;
  const T inv = ((const T*)op.Winv)[macro];
  const T* fb = (const T*)op.f + (size_t)macro * block;
  if (S7) {
    if (op.scaled) gs_tile7<T, true, false>(t, N, rs, op.colour, ub, fb, w, T(1), s_pre2, s_pre_tot);
    else gs_tile7<T, false, false>(t, N, rs, op.colour, ub, fb, w, inv, s_pre2, s_pre_tot);
    return;
  }
  const int total = flat_setup_slabs(t, N, op.colour, true, 1, s_pre2, s_pre_tot);
  int sl = 0;
  for (int tt = tid256(); tt < total; tt += CTA) {
    while (tt >= s_pre_tot[sl + 1]) ++sl;
    const int k = t.k + sl;
    const Tile ts{k, t.j0, t.m0, 1};
    int j, v, ic, mlo, n;
    flat_item(ts, N, op.colour, true, s_pre2[sl], tt - s_pre_tot[sl], j, v);
    colour_row(N, j, k, op.colour, ic, mlo, n);
    const int i = 4 * (mlo + v) + ic;
    const int me = lidx32(rs, N, i, j, k);
    T acc = fb[me];
#pragma unroll
    for (int d = 1; d < NDIR; ++d) {
      int di, dj, dk;
      dir_ijk(d, di, dj, dk);
      acc -= w[d] * ub[lidx32(rs, N, i + di, j + dj, k + dk)];
    }
    ub[me] = acc * inv;
  }
}

// Unit of the residual r = f - A u written to r (k_res, no norm).
template <class T, bool S7>
__device__ void unit_res(const BOp& op, int unit, int (*s_pre2)[33], int* s_pre_tot) {
  const LevelArgs& L = op.L;
  const ProbArgs& p = op.P;
  const int N = L.N;
  const int* rs = L.rs;
  const int64_t block = L.block;
  const T* u = (const T*)op.u;
  T* r = (T*)op.r;
  double ss = 0.0;
  if (unit < op.n_if_units) {
    const int q = unit * CTA + tid256();
    if (q < op.n_list) {
      const T* uI = (const T*)op.uI;
      const T* fI = (const T*)op.fI;
      const int node = p.free_if[q];
      const int c0 = L.cptr[node], c1 = L.cptr[node + 1];
      const IfTab<T> tab = dev_if_tab<T>(p, 0);
      T res;
      if (q >= op.skip_lo && q < op.skip_hi) {
        res = T(0);
      } else if (tab.nb) {
        res = fI[node] - tab.diag[q] * uI[node] - if_offdiag<T, if_tab_k(S7)>(tab, u, q);
      } else {
        T off = T(0), diag = T(0);
        if_stencil<T, S7>(N, rs, block, u, (const T*)op.W, L.cps, c0, c1, off, diag);
        res = fI[node] - diag * uI[node] - off;
      }
      write_copies(N, rs, block, r, L.cps, L.cp_off, c0, c1, res);
    } else if (q < op.n_list + op.n_zero) {
      r[p.zero_off[q - op.n_list]] = T(0);
    }
    return;
  }
  const int vb = unit - op.n_if_units;
  const Tile t = L.tiles_int[vb / p.n_act];
  const int macro = p.act[vb % p.n_act];
  const T* ub = u + (size_t)macro * block;
  const T* fb = (const T*)op.f + (size_t)macro * block;
  T* rb = r + (size_t)macro * block;
  const T* w = (const T*)op.W + (size_t)macro * 16 * NDIR;
  if (S7) {
    constexpr int VW = Vec<T>::n;
    const T wr[11] = {w[0], w[1], w[2], w[3], T(0), T(0), T(0), T(0), w[8], w[9], w[10]};
    for (int c = 0; c < 4; ++c) {
      const int total = flat_setup_slabs(t, N, c, true, VW, s_pre2, s_pre_tot);
      int sl = 0;
      for (int tt = tid256(); tt < total; tt += CTA) {
        while (tt >= s_pre_tot[sl + 1]) ++sl;
        const int k = t.k + sl;
        const Tile ts{k, t.j0, t.m0, 1};
        int j, g;
        flat_item(ts, N, c, true, s_pre2[sl], tt - s_pre_tot[sl], j, g, VW);
        if (c == op.skip)
          res_group7<T, true, false, true, false>(slice_consts(rs, N, k), N, j, g, c, ub, fb, rb, wr, ss);
        else
          res_group7<T, true, false, false, false>(slice_consts(rs, N, k), N, j, g, c, ub, fb, rb, wr, ss);
      }
      __syncthreads();
    }
    return;
  }
  HHG_TILE_NODES(N, rs, t, s_pre, {
    const int me = lidx32(rs, N, i, j, k);
    T acc = T(0);
    if (((i + 2 * j + 3 * k) & 3) != op.skip) {
      acc = fb[me] - w[0] * ub[me];
_Pragma("unroll")
      for (int d = 1; d < NDIR; ++d) {
        int di, dj, dk;
        dir_ijk(d, di, dj, dk);
        acc -= w[d] * ub[lidx32(rs, N, i + di, j + dj, k + dk)];
      }
    }
    rb[me] = acc;
  })
}

// Unit of the restriction onto the coarse level C (k_restrict).
template <class T>
__device__ void unit_restrict(const BOp& op, int unit, int (*s_pre2)[33], int* s_pre_tot) {
  const LevelArgs& F = op.L;
  const LevelArgs& C = op.C;
  const ProbArgs& pc = op.P;
  const T* rf = (const T*)op.r;
  T* fc = (T*)op.fc;
  T* uc = (T*)op.uc;
  if (unit < op.n_if_units) {
    const int q = unit * CTA + tid256();
    if (q < op.n_list) {
      T* fIc = (T*)op.fIc;
      T* uIc = (T*)op.uIc;
      const int node = pc.free_if[q];
      const int64_t* g = pc.gather + (size_t)q * NDIR;
      T acc = T(0);
      for (int e = 1; e < NDIR; ++e) {
        const int64_t o = g[e];
        if (o >= 0) acc += rf[o];
      }
      fIc[node] = rf[g[0]] + T(0.5) * acc;
      uIc[node] = T(0);
      write_copies(C.N, C.rs, C.block, uc, C.cps, C.cp_off, C.cptr[node], C.cptr[node + 1], T(0));
    } else if (q < op.n_list + op.n_zero) {
      uc[pc.zero_off[q - op.n_list]] = T(0);
    }
    return;
  }
  Tile t;
  int macro;
  vol_subunit(unit - op.n_if_units, pc.n_act, RESTRICT_SPLIT, C.tiles_int, pc.act, t, macro);
  restrict_tile<T, false>(t, C.N, C.rs, F.N, F.rs, rf + (size_t)macro * F.block, fc + (size_t)macro * C.block,
                          uc + (size_t)macro * C.block, s_pre2, s_pre_tot);
}

// Unit of the prolongation u_f += P u_c (k_prolong).
template <class T>
__device__ void unit_prolong(const BOp& op, int unit, int (*s_pre2)[33], int* s_pre_tot) {
  const LevelArgs& F = op.L;
  const LevelArgs& C = op.C;
  const ProbArgs& pf = op.P;
  T* uf = (T*)op.u;
  const T* uc = (const T*)op.uc;
  if (unit < op.n_if_units) {
    const int q = unit * CTA + tid256();
    if (q < op.n_list && (q < op.skip_lo || q >= op.skip_hi)) {
      T* uIf = (T*)op.uI;
      const int node = pf.free_if[q];
      const int c0 = F.cptr[node], c1 = F.cptr[node + 1];
      const Copy cp = F.cps[c0];
      const T val = uIf[node] + interp(uc + (size_t)cp.macro * C.block, C.N, C.rs, cp.i, cp.j, cp.k);
      uIf[node] = val;
      write_copies(F.N, F.rs, F.block, uf, F.cps, F.cp_off, c0, c1, val);
    }
    return;
  }
  const int vb = unit - op.n_if_units;
  const Tile t = F.tiles_int[vb / pf.n_act];
  const int macro = pf.act[vb % pf.n_act];
  prolong_tile<T, false>(t, F.N, F.rs, C.N, C.rs, uf + (size_t)macro * F.block, uc + (size_t)macro * C.block, op.skip,
                         s_pre2, s_pre_tot);
}

// Unit of the FP64 residual handed to the FP32 cycle (k_res_f32, no norm).
template <bool S7>
__device__ void unit_res_f32(const BOp& op, int unit, int (*s_pre2)[33], int* s_pre_tot) {
  const LevelArgs& L = op.L;
  const ProbArgs& p = op.P;
  const int N = L.N;
  const int* rs = L.rs;
  const int64_t block = L.block;
  const double* u = (const double*)op.u;
  if (unit < op.n_if_units) {
    const int q = unit * CTA + tid256();
    if (q < op.n_list) {
      const double* uI = (const double*)op.uI;
      const double* fI = (const double*)op.fI;
      const int node = p.free_if[q];
      const IfTab<double> tab = dev_if_tab<double>(p, 0);
      double res;
      if (tab.nb) {
        res = fI[node] - tab.diag[q] * uI[node] - if_offdiag<double, if_tab_k(S7)>(tab, u, q);
      } else {
        double off = 0.0, diag = 0.0;
        if_stencil<double, S7>(N, rs, block, u, (const double*)op.W, L.cps, L.cptr[node], L.cptr[node + 1], off,
                               diag);
        res = fI[node] - diag * uI[node] - off;
      }
      ((float*)op.oI32)[node] = (float)res;
    }
    return;
  }
  const int vb = unit - op.n_if_units;
  const Tile t = L.tiles_int[vb / p.n_act];
  const int macro = p.act[vb % p.n_act];
  const double* ub = u + (size_t)macro * block;
  const double* fb = (const double*)op.f + (size_t)macro * block;
  float* ob = (float*)op.o32 + (size_t)macro * block;
  const double* w = (const double*)op.W + (size_t)macro * 16 * NDIR;
  HHG_TILE_NODES(N, rs, t, s_pre, {
    int me;
    double acc;
    if (S7) {
      const Nb7 q = nb7(sc, i, j);
      me = q.me;
      acc = fb[me] - w[0] * ub[me];
      acc -= w[1] * ub[q.nb1];
      acc -= w[2] * ub[q.nb2];
      acc -= w[3] * ub[q.nb3];
      acc -= w[8] * ub[q.nb8];
      acc -= w[9] * ub[q.nb9];
      acc -= w[10] * ub[q.nb10];
    } else {
      me = lidx32(rs, N, i, j, k);
      acc = fb[me] - w[0] * ub[me];
_Pragma("unroll")
      for (int d = 1; d < NDIR; ++d) {
        int di, dj, dk;
        dir_ijk(d, di, dj, dk);
        acc -= w[d] * ub[lidx32(rs, N, i + di, j + dj, k + dk)];
      }
    }
    ob[me] = (float)acc;
  })
}

// Coarse CG (k_cg with its vectors in the problem's global work array).
template <class T>
__device__ void unit_cg(const BOp& op, double* red) {
  const int n = op.n_cg;
  const T* f = (const T*)op.f;
  const T* fI = (const T*)op.fI;
  T* u = (T*)op.u;
  T* uI = (T*)op.uI;
  double* x = op.work;
  double* r = x + n;
  double* p = r + n;
  double* Ap = p + n;
  const int tid = tid256();
  double part = 0.0;
  for (int q = tid; q < n; q += CTA) {
    const int64_t s = op.fsrc[q];
    const double b = s >= 0 ? (double)f[s] : (double)fI[-1 - s];
    x[q] = 0.0;
    r[q] = b;
    p[q] = b;
    part += b * b;
  }
  double rr = cg_allreduce(part, red);
  int rb = 1;
  const double bnorm = sqrt(rr);
  int it = 0;
  while (bnorm > 0.0 && sqrt(rr) > op.rtol * bnorm && it < op.maxit) {
    __syncthreads();
    part = 0.0;
    for (int q = tid; q < n; q += CTA) {
      double a = 0.0;
      for (int e = op.rowptr[q]; e < op.rowptr[q + 1]; ++e) a += op.val[e] * p[op.col[e]];
      Ap[q] = a;
      part += p[q] * a;
    }
    const double pAp = cg_allreduce(part, red + 8 * rb);
    rb ^= 1;
    const double alpha = rr / pAp;
    part = 0.0;
    for (int q = tid; q < n; q += CTA) {
      x[q] += alpha * p[q];
      const double rq = r[q] - alpha * Ap[q];
      r[q] = rq;
      part += rq * rq;
    }
    const double rr_new = cg_allreduce(part, red + 8 * rb);
    rb ^= 1;
    const double beta = rr_new / rr;
    for (int q = tid; q < n; q += CTA) p[q] = r[q] + beta * p[q];
    rr = rr_new;
    ++it;
  }
  for (int q = tid; q < n; q += CTA) {
    const T v = (T)x[q];
    for (int e = op.uptr[q]; e < op.uptr[q + 1]; ++e) u[op.udst[e]] = v;
    if (op.umaster[q] >= 0) uI[op.umaster[q]] = v;
  }
  if (tid == 0 && op.iters) *op.iters = it;
}

// 16384 elements per unit of the block-wise operations (zeroing, the FP32
// correction added in FP64, memsets): tens of microseconds of streaming per
// unit, like a stencil tile, so that the claims stay cheap by comparison
constexpr int BATCH_CHUNK = CTA * 64;

__device__ void run_unit(const BOp& op, int unit, int (*s_pre2)[33], int* s_pre_tot, double* red) {
  const int tid = tid256();
  switch (op.kind) {
    case BOP_GS:
      if (op.fp32) {
        if (op.seven_point) unit_gs<float, true>(op, unit, s_pre2, s_pre_tot);
        else unit_gs<float, false>(op, unit, s_pre2, s_pre_tot);
      } else {
        if (op.seven_point) unit_gs<double, true>(op, unit, s_pre2, s_pre_tot);
        else unit_gs<double, false>(op, unit, s_pre2, s_pre_tot);
      }
      break;
    case BOP_RES:
      if (op.fp32) {
        if (op.seven_point) unit_res<float, true>(op, unit, s_pre2, s_pre_tot);
        else unit_res<float, false>(op, unit, s_pre2, s_pre_tot);
      } else {
        if (op.seven_point) unit_res<double, true>(op, unit, s_pre2, s_pre_tot);
        else unit_res<double, false>(op, unit, s_pre2, s_pre_tot);
      }
      break;
    case BOP_RESTRICT:
      if (op.fp32) unit_restrict<float>(op, unit, s_pre2, s_pre_tot);
      else unit_restrict<double>(op, unit, s_pre2, s_pre_tot);
      break;
    case BOP_PROLONG:
      if (op.fp32) unit_prolong<float>(op, unit, s_pre2, s_pre_tot);
      else unit_prolong<double>(op, unit, s_pre2, s_pre_tot);
      break;
    case BOP_CG:
      if (op.fp32) unit_cg<float>(op, red);
      else unit_cg<double>(op, red);
      break;
    case BOP_RES_F32:
      if (op.seven_point) unit_res_f32<true>(op, unit, s_pre2, s_pre_tot);
      else unit_res_f32<false>(op, unit, s_pre2, s_pre_tot);
      break;
    case BOP_ZERO_BLOCKS: {
      // unit = (active macro, chunk of BATCH_CHUNK elements)
      const int64_t chunks = (op.L.block + BATCH_CHUNK - 1) / BATCH_CHUNK;
      const int macro = op.P.act[unit / chunks];
      const int64_t c0 = (unit % chunks) * BATCH_CHUNK;
      const int64_t c1 = min((int64_t)BATCH_CHUNK + c0, op.L.block);
      for (int64_t q = c0 + tid; q < c1; q += CTA) {
        if (op.fp32) ((float*)op.u)[(size_t)macro * op.L.block + q] = 0.f;
        else ((double*)op.u)[(size_t)macro * op.L.block + q] = 0.0;
      }
      break;
    }
    case BOP_ZERO_LIST: {
      const int64_t q = (int64_t)unit * CTA + tid;
      if (q < op.n) {
        if (op.fp32) ((float*)op.uI)[op.ids[q]] = 0.f;
        else ((double*)op.uI)[op.ids[q]] = 0.0;
      }
      break;
    }
    case BOP_ADD_BLOCKS: {
      // unit = (active macro, chunk of BATCH_CHUNK FP64 slots); u64 += e32
      const int64_t chunks = (op.L.block + BATCH_CHUNK - 1) / BATCH_CHUNK;
      const int macro = op.P.act[unit / chunks];
      const int64_t c0 = (unit % chunks) * BATCH_CHUNK;
      const int64_t c1 = min((int64_t)BATCH_CHUNK + c0, op.L.block);
      double* ub = (double*)op.u + (size_t)macro * op.L.block;
      const float* eb = (const float*)op.o32 + (size_t)macro * op.L.block;
      for (int64_t q = c0 + 2 * tid; q < c1; q += 2 * CTA) {
        double2 x = *reinterpret_cast<double2*>(ub + q);
        const float2 d = *reinterpret_cast<const float2*>(eb + q);
        x.x += (double)d.x;
        x.y += (double)d.y;
        *reinterpret_cast<double2*>(ub + q) = x;
      }
      break;
    }
    case BOP_ADD_MASTERS: {
      const int64_t q = (int64_t)unit * CTA + tid;
      if (q < op.n) {
        const int node = op.ids[q];
        ((double*)op.uI)[node] += (double)((const float*)op.oI32)[node];
      }
      break;
    }
    case BOP_MEMSET: {
      // 16-byte words [unit * BATCH_CHUNK, ...) of op.u
      const int64_t c0 = (int64_t)unit * BATCH_CHUNK;
      const int64_t c1 = min((int64_t)BATCH_CHUNK + c0, op.n);
      for (int64_t q = c0 + tid; q < c1; q += CTA) reinterpret_cast<double2*>(op.u)[q] = make_double2(0.0, 0.0);
      break;
    }
    case BOP_SET_ZERO: {
      const int64_t q = (int64_t)unit * CTA + tid;
      if (q < op.n) ((double*)op.uI)[op.ids[q]] = 0.0;
      break;
    }
    case BOP_RESTORE: {
      const int64_t q = (int64_t)unit * CTA + tid;
      if (q < op.n) ((double*)op.u)[op.offs[q]] = ((const double*)op.uI)[op.ids[q]];
      break;
    }
    default:
      break;
  }
}

// Persistent executor of a batch: task t runs ops [op_off[t], op_off[t + 1])
// in order; n_live tasks have at least one operation.  Every CTA repeatedly
// claims a unit of the current operation of some task, runs it and counts it
// done; the CTA that completes an operation's last unit publishes the task's
// next phase.
//   * Claims: warp 0 scans the tasks 32 at a time in priority classes (the
//     tasks order[seg[c] .. seg[c + 1]) form class c, highest first); within
//     a class it starts at the task it served last, and the first lane that
//     sees unissued units of its task's current operation takes one with an
//     atomic.  While the CTA runs a unit, thread 0 already claims the next
//     unit of the same operation (the atomic's latency hides behind the
//     work), except near the end of the operation; a unit taken there is
//     valid because an operation with unissued units is still its task's
//     current one.
//   * Memory order: a unit's writes precede its done count (CTA barrier, then
//     a device fence by the counting thread); a CTA reads a published phase
//     before the data (device fence by the scanning warp, then a CTA
//     barrier); the units read that data with plain coherent loads.
//   * A CTA that finds no unit for wait_limit rounds in a row sets *err = 1
//     and stops; the CTA that completes an operation always finds the next
//     one, so the work still finishes.
//   * Time stamps: st.start_ns (first CTA), st.task_ns[t] (the task's last
//     unit done).
// One unit per claim: a large operation gives each CTA only a few units
// (a Gauss-Seidel tile takes tens of microseconds), so claiming several at
// once lengthens the operation's tail by more than the claims cost.
__device__ __forceinline__ int batch_claim_size(int) { return 1; }

// Scheduler state of a CTA, in shared memory so that no register stays live
// across a unit's body.
struct BatchCtl {
  int state, task, gi, unit, cnt;   // the claim to run (written by warp 0)
  int cur_gi, cur_task;             // operation held in the CTA's op copy
  int next;                         // first task of the next scan
  int pf_u, pf_k;                   // chunk claimed ahead on cur_gi (-1: none)
  int idle;                         // scans in a row that found nothing
};

__global__ void __launch_bounds__(CTA, 5) k_batch(const BOp* __restrict__ ops, const int* __restrict__ op_off,
                                                  const int* __restrict__ order, const int* __restrict__ seg, int n_seg,
                                                  int n_live, BatchState st, int wait_limit, int* __restrict__ err) {
  __shared__ int s_pre2[MAX_SLABS][33];
  __shared__ int s_pre_tot[MAX_SLABS + 1];
  __shared__ double red[16];
  __shared__ BatchCtl ctl;
  __shared__ __align__(16) BOp s_op;
  if (tid256() == 0) {
    atomicMin(st.start_ns, global_ns());
    ctl.cur_gi = -1;
    ctl.cur_task = 0;
    ctl.next = -1;
    ctl.pf_u = -1;
    ctl.pf_k = 0;
    ctl.idle = 0;
  }
  __syncthreads();
  for (;;) {
    if (tid256() < 32) {
      const int lane = tid256();
      int state = 0, task = 0, gi = 0, u = 0, cnt = 0;
      if (ctl.pf_u >= 0) {
        state = 1;
        task = ctl.cur_task;
        gi = ctl.cur_gi;
        u = ctl.pf_u;
        cnt = ctl.pf_k;
      } else if (*(volatile int*)st.tasks_done >= n_live) {
        state = 2;
      } else {
        int pos_taken = 0;
        for (int c = 0; c < n_seg && state == 0; ++c) {
          const int lo = seg[c], len = seg[c + 1] - lo;
          const int cur = ctl.next;   // position in order[] of the task served last
          const int start = cur >= lo && cur < lo + len ? cur - lo : (int)(blockIdx.x % (unsigned)len);
          for (int base = 0; base < len && state == 0; base += 32) {
            const int q = base + lane;
            int pos = start + q;
            if (pos >= len) pos -= len;
            bool avail = false;
            int g = 0, nu = 0, t = 0;
            if (q < len) {
              t = order[lo + pos];
              const int ph = *(volatile int*)(st.phase + t);
              const int o0 = op_off[t];
              if (ph < op_off[t + 1] - o0) {
                g = o0 + ph;
                nu = ops[g].n_units;
                avail = *(volatile int*)(st.issued + g) < nu;
              }
            }
            unsigned mask = __ballot_sync(0xffffffffu, avail);
            while (mask) {
              const int src = __ffs(mask) - 1;
              mask &= mask - 1;
              int claim = -1, k = 0;
              if (lane == src) {
                k = batch_claim_size(nu);
                const int u0 = atomicAdd(st.issued + g, k);
                if (u0 < nu) {
                  claim = u0;
                  k = min(k, nu - u0);
                }
              }
              claim = __shfl_sync(0xffffffffu, claim, src);
              if (claim >= 0) {
                state = 1;
                task = __shfl_sync(0xffffffffu, t, src);
                gi = __shfl_sync(0xffffffffu, g, src);
                cnt = __shfl_sync(0xffffffffu, k, src);
                pos_taken = lo + __shfl_sync(0xffffffffu, pos, src);
                u = claim;
                break;
              }
            }
          }
        }
        if (state == 1 && lane == 0) ctl.next = pos_taken;
        __threadfence();   // what the earlier operations wrote is read after this
      }
      __syncwarp();
      if (lane == 0) {
        ctl.state = state;
        ctl.task = task;
        ctl.gi = gi;
        ctl.unit = u;
        ctl.cnt = cnt;
      }
    }
    __syncthreads();
    if (ctl.state == 2) break;
    if (ctl.state == 0) {
      __syncthreads();   // every thread has read the state
      if (tid256() == 0) {
        if (++ctl.idle > wait_limit) {
          atomicExch(err, 1);
          ctl.state = 2;
        } else {
          __nanosleep(256);
        }
      }
      __syncthreads();
      if (ctl.state == 2) break;
      continue;
    }
    if (ctl.gi != ctl.cur_gi) {
      const int* src = reinterpret_cast<const int*>(ops + ctl.gi);
      int* dst = reinterpret_cast<int*>(&s_op);
      for (int q = tid256(); q < (int)(sizeof(BOp) / sizeof(int)); q += CTA) dst[q] = src[q];
      __syncthreads();
    }
    if (tid256() == 0) {
      ctl.idle = 0;
      ctl.cur_gi = ctl.gi;
      ctl.cur_task = ctl.task;
      // claim the next unit of this operation while this one runs, unless
      // the operation nears its end (a unit held back there lengthens the
      // operation's tail)
      const int nu = s_op.n_units;
      ctl.pf_k = batch_claim_size(nu);
      ctl.pf_u = ctl.unit + ctl.cnt + 2 * (int)gridDim.x * ctl.pf_k < nu ? atomicAdd(st.issued + ctl.gi, ctl.pf_k) : nu;
    }
    for (int c = 0; c < ctl.cnt; ++c) {
      run_unit(s_op, ctl.unit + c, s_pre2, s_pre_tot, red);
      __syncthreads();
    }
    if (tid256() == 0) {
      const int nu = s_op.n_units;
      if (ctl.pf_u >= nu) ctl.pf_u = -1;
      else ctl.pf_k = min(ctl.pf_k, nu - ctl.pf_u);
      const int gi = ctl.gi, cnt = ctl.cnt;
      __threadfence();   // the CTA's writes before its units count as done
      const int d = atomicAdd(st.done + gi, cnt);
      if (d + cnt == nu) {
        const int t = ctl.task;
        const int ph = gi - op_off[t] + 1;
        __threadfence();
        atomicExch(st.phase + t, ph);
        if (ph == op_off[t + 1] - op_off[t]) {
          st.task_ns[t] = global_ns();
          __threadfence();
          atomicAdd(st.tasks_done, 1);
        }
      }
    }
    // the next scan (warp 0) reads ctl after thread 0 wrote it: same warp,
    // ordered by __syncwarp at the top of the scan
    __syncwarp();
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
namespace {
thread_local std::vector<BOp>* g_rec = nullptr;

// A batch operation of kind k in the arithmetic type T.
template <class T>
BOp new_op(int kind) {
  BOp op;
  std::memset(&op, 0, sizeof(op));
  op.kind = kind;
  op.fp32 = sizeof(T) == 4 ? 1 : 0;
  return op;
}

int64_t block_chunks(int64_t block) { return (block + BATCH_CHUNK - 1) / BATCH_CHUNK; }
}  // namespace

void record_ops(std::vector<BOp>* rec) { g_rec = rec; }
bool recording() { return g_rec != nullptr; }

cudaError_t memset16(void* p, size_t bytes, cudaStream_t s) {
  if (g_rec) {
    if (bytes % 16 != 0 || reinterpret_cast<uintptr_t>(p) % 16 != 0) return cudaErrorInvalidValue;
    BOp op = new_op<double>(BOP_MEMSET);
    op.u = p;
    op.n = (int64_t)(bytes / 16);
    op.n_units = (int)((op.n + BATCH_CHUNK - 1) / BATCH_CHUNK);
    if (op.n_units > 0) g_rec->push_back(op);
    return cudaSuccess;
  }
  return cudaMemsetAsync(p, 0, bytes, s);
}

cudaError_t run_batch(const BOp* ops, const int* op_off, const int* order, const int* seg, int n_seg, int n_live,
                      const BatchState& st, int wait_limit, int* err, cudaStream_t s) {
  if (n_live <= 0) return cudaSuccess;
  const unsigned grid = resident_grid((const void*)k_batch, 1 << 30);
  ++g_kernel_launches;
  k_batch<<<grid, cta_shape(), 0, s>>>(ops, op_off, order, seg, n_seg, n_live, st, wait_limit, err);
  return cudaGetLastError();
}
// Elements of one staging slot of the streaming kernel on a level: the
// largest band range, rows 0..band+1 of slice 0, rounded up to 32 elements.
inline int stream_slot(int N, int band) {
  const int M = N + 1;
  const int len = slot_prefix(M) - slot_prefix(std::max(0, M - (band + 2)));
  return (len + 31) & ~31;
}

template <class T, bool SCALED>
cudaError_t launch_gs_stream(const LevelArgs& L, const ProbArgs& p, T* u, T* uI, const T* fI, const T* W,
                             const T* Winv, const T* fv, const T* Wv, int colour, int n, cudaStream_t s) {
  const bool wide = sizeof(T) == 4;   // FP32 cycles: wider bands
  const StreamTile* tiles = wide ? L.tiles_stream32 : L.tiles_stream;
  const int n_tiles = wide ? L.n_tiles_stream32 : L.n_tiles_stream;
  const Units g = units(n, n_tiles, p.n_act);
  if (g.total == 0) return cudaSuccess;
  const int slot = stream_slot(L.N, wide ? L.stream_band32 : L.stream_band);
  const size_t smem = (size_t)(STREAM_NSLOT * slot + 2 * STREAM_PAD) * sizeof(T);
  auto kern = k_gs_stream<T, SCALED>;
  // the kernel may use up to the device's opt-in shared memory per CTA (set
  // once per device; a smaller setting would refuse later, larger launches)
  static std::mutex mu;
  static std::map<int, int> attr_max;   // device -> bytes allowed
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = attr_max.find(dev);
    if (it == attr_max.end()) {
      int optin = 0;
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      const int static_bytes = 4096;   // the kernel's own shared arrays, with room
      const int allow = std::max(0, optin - static_bytes);
      const cudaError_t e =
          cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, allow);
      if (e != cudaSuccess) return e;
      it = attr_max.emplace(dev, allow).first;
    }
    if ((size_t)it->second < smem) return cudaErrorInvalidConfiguration;
  }
  int per_sm = 0, sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)kern, STREAM_CTA, smem);
  int cap = std::max(1, sms * std::max(1, per_sm));
  if (p.grid_cap > 0) cap = std::min(cap, p.grid_cap);
  const unsigned grid = (unsigned)std::min(g.total, cap);
  ++g_kernel_launches;
  kern<<<grid, dim3(32, STREAM_CONSUMERS + 1), smem, s>>>(L.N, L.rs, L.block, u, uI, fI, W, Winv, fv, Wv, tiles,
                                                         n_tiles, p.act, p.n_act, colour, L.cptr, L.cps, L.cp_off,
                                       p.free_if + p.col_off[colour], n, if_tab<T>(p, p.col_off[colour]),
                                       g.n_if_units, p.sched, slot, p.wait_limit, p.err);
  return cudaGetLastError();
}

template <class T>
cudaError_t gs_colour(const LevelArgs& L, const ProbArgs& p, T* u, T* uI, const T* f, const T* fI, const T* W,
                      const T* Winv, int colour, bool seven_point, cudaStream_t s, cudaEvent_t ev_begin,
                      cudaEvent_t ev_end, const T* fs, const T* Wsc) {
  if (g_rec) {
    if (!seven_point || !fs || !Wsc) fs = Wsc = nullptr;
    const int nl = p.col_off[colour + 1] - p.col_off[colour];
    const Units g = units(nl, L.n_tiles_int, p.n_act);
    if (g.total == 0) return cudaSuccess;
    BOp op = new_op<T>(BOP_GS);
    op.seven_point = seven_point ? 1 : 0;
    op.scaled = fs ? 1 : 0;
    op.colour = colour;
    op.L = L;
    op.P = p;
    op.list_off = p.col_off[colour];
    op.n_list = nl;
    op.n_if_units = g.n_if_units;
    op.n_units = g.total;
    op.u = u;
    op.uI = uI;
    op.f = fs ? fs : f;
    op.fI = fI;
    op.W = W;
    op.Wv = Wsc ? Wsc : W;
    op.Winv = Winv;
    g_rec->push_back(op);
    return cudaSuccess;
  }
  if (!seven_point) fs = Wsc = nullptr;
  if (!fs || !Wsc) fs = Wsc = nullptr;
  const int n = p.col_off[colour + 1] - p.col_off[colour];
  if (seven_point && p.stream_gs && L.n_tiles_stream > 0 && p.err) {
    if (ev_begin) cudaEventRecord(ev_begin, s);
    const cudaError_t e = fs ? launch_gs_stream<T, true>(L, p, u, uI, fI, W, Winv, fs, Wsc, colour, n, s)
                             : launch_gs_stream<T, false>(L, p, u, uI, fI, W, Winv, f, W, colour, n, s);
    if (ev_end) cudaEventRecord(ev_end, s);
    return e;
  }
  const uint32_t* items = sizeof(T) == 8 ? L.gs_items64 : L.gs_items32;
  if (seven_point && L.gs_flat && items) {
    const int* off = sizeof(T) == 8 ? L.gs_off64 : L.gs_off32;
    const int n_items = off[colour + 1] - off[colour];
    const int n_if_ctas = (int)lin_grid(n, CTA);
    const int n_vol_ctas = p.n_act > 0 ? (int)lin_grid((int64_t)n_items * p.n_act, CTA) : 0;
    if (n_if_ctas + n_vol_ctas == 0) return cudaSuccess;
    auto kern = fs ? k_gs_flat<T, true> : k_gs_flat<T, false>;
    if (ev_begin) cudaEventRecord(ev_begin, s);
    ++g_kernel_launches;
    kern<<<n_if_ctas + n_vol_ctas, cta_shape(), 0, s>>>(
        L.N, L.rs, L.block, u, uI, fI, W, Winv, fs ? fs : f, Wsc ? Wsc : W, items + off[colour], n_items, p.act,
        p.n_act, colour, L.cptr, L.cps, L.cp_off, p.free_if + p.col_off[colour], n, if_tab<T>(p, p.col_off[colour]),
        n_if_ctas, n_vol_ctas);
    if (ev_end) cudaEventRecord(ev_end, s);
    return cudaGetLastError();
  }
  const Units g = units(n, L.n_tiles_int, p.n_act);
  if (g.total == 0) return cudaSuccess;
  auto kern = seven_point ? k_gs<T, true> : k_gs<T, false>;
  const unsigned grid = resident_grid((const void*)kern, g.total, p.grid_cap);
  if (ev_begin) cudaEventRecord(ev_begin, s);
  ++g_kernel_launches;
  kern<<<grid, cta_shape(), 0, s>>>(L.N, L.rs, L.block, u, uI, f, fI, W, Winv, fs, Wsc, L.tiles_int, L.n_tiles_int, p.act,
                                    p.n_act, colour, L.cptr, L.cps, L.cp_off, p.free_if + p.col_off[colour], n,
                                    if_tab<T>(p, p.col_off[colour]), g.n_if_units, p.sched);
  if (ev_end) cudaEventRecord(ev_end, s);
  return cudaGetLastError();
}

template <class T>
cudaError_t residual(const LevelArgs& L, const ProbArgs& p, const T* u, const T* uI, const T* f, const T* fI, T* r,
                     const T* W, bool seven_point, bool write_r, double* partial, int* n_part, cudaStream_t s,
                     int skip) {
  if (g_rec) {
    if (partial || !write_r) return cudaErrorNotSupported;   // norms are not part of a batch
    const int nl = p.col_off[4];
    const Units g = units(nl + p.n_zero, L.n_tiles_int, p.n_act);
    if (g.total == 0) return cudaSuccess;
    BOp op = new_op<T>(BOP_RES);
    op.seven_point = seven_point ? 1 : 0;
    op.skip = skip >= 0 && skip < 4 ? skip : -1;
    op.skip_lo = op.skip >= 0 ? p.col_off[op.skip] : 0;
    op.skip_hi = op.skip >= 0 ? p.col_off[op.skip + 1] : 0;
    op.L = L;
    op.P = p;
    op.n_list = nl;
    op.n_zero = p.n_zero;
    op.n_if_units = g.n_if_units;
    op.n_units = g.total;
    op.u = (void*)u;
    op.uI = (void*)uI;
    op.f = f;
    op.fI = fI;
    op.r = r;
    op.W = W;
    g_rec->push_back(op);
    return cudaSuccess;
  }
  const bool norm = partial != nullptr;
  const int n = p.col_off[4];
  const int n_zero = write_r ? p.n_zero : 0;
  const Units g = units(n + n_zero, L.n_tiles_int, p.n_act);
  if (n_part) *n_part = 0;
  if (g.total == 0) return cudaSuccess;
  const uint32_t* items = sizeof(T) == 8 ? L.gs_items64 : L.gs_items32;
  if (seven_point && L.gs_flat && items && write_r && !norm) {
    // the residual before a restriction, on levels whose Gauss-Seidel runs
    // flat: one chunk per CTA (norm launches keep the tile kernel, whose
    // partial sums per CTA measured faster)
    const int* off = sizeof(T) == 8 ? L.gs_off64 : L.gs_off32;
    const int sk = skip >= 0 && skip < 4 ? skip : -1;
    const int n_items = off[4];
    const int n_if_chunks = (int)lin_grid(n + n_zero, CTA);
    const int n_vol_chunks = p.n_act > 0 ? (int)lin_grid((int64_t)n_items * p.n_act, CTA) : 0;
    ++g_kernel_launches;
    k_res_flat<T, true, false><<<n_if_chunks + n_vol_chunks, cta_shape(), 0, s>>>(
        L.N, L.rs, L.block, u, uI, f, fI, r, W, items, make_int4(off[0], off[1], off[2], off[3]), n_items, p.act,
        p.n_act, L.cptr, L.cps, L.cp_off, p.free_if, n, if_tab<T>(p, 0), p.zero_off, n_zero, n_if_chunks,
        n_vol_chunks, nullptr, sk, sk >= 0 ? p.col_off[sk] : 0, sk >= 0 ? p.col_off[sk + 1] : 0);
    return cudaGetLastError();
  }
  void (*kern)(int, const int*, int64_t, const T*, const T*, const T*, const T*, T*, const T*, const Tile*, int, const int*,
               int, const int*, const Copy*, const uint32_t*, const int*, int, IfTab<T>, const int64_t*, int, int,
               double*, int*, int, int, int);
  const int skip_lo = skip >= 0 && skip < 4 ? p.col_off[skip] : 0;
  const int skip_hi = skip >= 0 && skip < 4 ? p.col_off[skip + 1] : 0;
  if (seven_point)
    kern = write_r ? (norm ? k_res<T, true, true, true> : k_res<T, true, true, false>) : k_res<T, true, false, true>;
  else
    kern = write_r ? (norm ? k_res<T, false, true, true> : k_res<T, false, true, false>) : k_res<T, false, false, true>;
  const unsigned grid = resident_grid((const void*)kern, g.total, p.grid_cap);
  if (n_part && norm) *n_part = (int)grid;
  ++g_kernel_launches;
  kern<<<grid, cta_shape(), 0, s>>>(L.N, L.rs, L.block, u, uI, f, fI, r, W, L.tiles_int, L.n_tiles_int, p.act,
                                    p.n_act, L.cptr, L.cps, L.cp_off, p.free_if, n, if_tab<T>(p, 0), p.zero_off, n_zero,
                                    g.n_if_units, partial, p.sched, skip >= 0 && skip < 4 ? skip : -1, skip_lo, skip_hi);
  return cudaGetLastError();
}

template <class T>
cudaError_t restrict_to(const LevelArgs& C, const LevelArgs& F, const ProbArgs& pc, const T* rf, T* fc, T* fIc, T* uc,
                        T* uIc, cudaStream_t s) {
  if (g_rec) {
    const int nl = pc.col_off[4];
    const Units g = units(nl + pc.n_zero, C.n_tiles_int * RESTRICT_SPLIT, pc.n_act);
    if (g.total == 0) return cudaSuccess;
    BOp op = new_op<T>(BOP_RESTRICT);
    op.L = F;
    op.C = C;
    op.P = pc;
    op.n_list = nl;
    op.n_zero = pc.n_zero;
    op.n_if_units = g.n_if_units;
    op.n_units = g.total;
    op.r = (void*)rf;
    op.fc = fc;
    op.fIc = fIc;
    op.uc = uc;
    op.uIc = uIc;
    g_rec->push_back(op);
    return cudaSuccess;
  }
  const int n = pc.col_off[4];
  const Units g = units(n + pc.n_zero, C.n_tiles_int * RESTRICT_SPLIT, pc.n_act);
  if (g.total == 0) return cudaSuccess;
  if (C.gs_flat && C.slot_items) {
    const int n_if_ctas = (int)lin_grid(n + pc.n_zero, CTA);
    const int n_vol_ctas = pc.n_act > 0 ? (int)lin_grid((int64_t)C.n_slots * pc.n_act, CTA) : 0;
    ++g_kernel_launches;
    k_restrict_flat<T><<<n_if_ctas + n_vol_ctas, cta_shape(), 0, s>>>(
        C.N, C.rs, C.block, fc, fIc, uc, uIc, F.N, F.rs, F.block, rf, C.slot_items, C.n_slots, pc.act, pc.n_act,
        C.cptr, C.cps, C.cp_off, pc.free_if, n, pc.gather, pc.zero_off, pc.n_zero, n_if_ctas, n_vol_ctas);
    return cudaGetLastError();
  }
  const unsigned grid = resident_grid((const void*)k_restrict<T>, g.total, pc.grid_cap);
  ++g_kernel_launches;
  k_restrict<T><<<grid, cta_shape(), 0, s>>>(C.N, C.rs, C.block, fc, fIc, uc, uIc, F.N, F.rs, F.block, rf, C.tiles_int,
                                             C.n_tiles_int, pc.act, pc.n_act, C.cptr, C.cps, C.cp_off, pc.free_if, n,
                                             pc.gather, pc.zero_off, pc.n_zero, g.n_if_units, pc.sched);
  return cudaGetLastError();
}

template <class T>
cudaError_t prolong_add(const LevelArgs& F, const LevelArgs& C, const ProbArgs& pf, T* uf, T* uIf, const T* uc,
                        cudaStream_t s, int skip, int if_lo, int if_hi) {
  skip = skip >= 0 && skip < 4 ? skip : -1;
  if (if_hi <= if_lo) if_lo = if_hi = 0;
  if (g_rec) {
    const int nl = pf.col_off[4];
    const Units g = units(nl, F.n_tiles_int, pf.n_act);
    if (g.total == 0) return cudaSuccess;
    BOp op = new_op<T>(BOP_PROLONG);
    op.skip = skip;
    op.skip_lo = if_lo;
    op.skip_hi = if_hi;
    op.L = F;
    op.C = C;
    op.P = pf;
    op.n_list = nl;
    op.n_if_units = g.n_if_units;
    op.n_units = g.total;
    op.u = uf;
    op.uI = uIf;
    op.uc = (void*)uc;
    g_rec->push_back(op);
    return cudaSuccess;
  }
  const int n = pf.col_off[4];
  const Units g = units(n, F.n_tiles_int, pf.n_act);
  if (g.total == 0) return cudaSuccess;
  const uint32_t* items = sizeof(T) == 8 ? F.gs_items64 : F.gs_items32;
  if (F.gs_flat && items && (skip == -1 || skip == 0)) {
    // the fine level's items of the colours updated: all, or 1..3 when the
    // first post-smoothing sweep overwrites colour 0
    const int* off = sizeof(T) == 8 ? F.gs_off64 : F.gs_off32;
    const int first_c = skip == 0 ? 1 : 0;
    const int n_items = off[4] - off[first_c];
    int rel[3];   // starts of the colours after first_c, relative to off[first_c]
    for (int t = 0; t < 3; ++t) {
      const int cc = first_c + 1 + t;
      rel[t] = cc <= 3 ? off[cc] - off[first_c] : n_items;
    }
    const int n_if_ctas = (int)lin_grid(n, CTA);
    const int n_vol_ctas = pf.n_act > 0 ? (int)lin_grid((int64_t)n_items * pf.n_act, CTA) : 0;
    ++g_kernel_launches;
    k_prolong_flat<T><<<n_if_ctas + n_vol_ctas, cta_shape(), 0, s>>>(
        F.N, F.rs, F.block, uf, uIf, C.N, C.rs, C.block, uc, items + off[first_c], n_items, first_c,
        make_int3(rel[0], rel[1], rel[2]), pf.act,
        pf.n_act, F.cptr, F.cps, F.cp_off, pf.free_if, n, if_lo, if_hi, n_if_ctas, n_vol_ctas);
    return cudaGetLastError();
  }
  const unsigned grid = resident_grid((const void*)k_prolong<T>, g.total, pf.grid_cap);
  ++g_kernel_launches;
  k_prolong<T><<<grid, cta_shape(), 0, s>>>(F.N, F.rs, F.block, uf, uIf, C.N, C.rs, C.block, uc, F.tiles_int,
                                            F.n_tiles_int, pf.act, pf.n_act, F.cptr, F.cps, F.cp_off, pf.free_if, n,
                                            g.n_if_units, pf.sched, skip, if_lo, if_hi);
  return cudaGetLastError();
}

template <class T>
cudaError_t coarse_cg(const DevProblem& p, const T* f, const T* fI, T* u, T* uI, double rtol, int maxit,
                      cudaStream_t s, double* work) {
  if (g_rec) {
    if (p.n_cg == 0) return cudaSuccess;
    BOp op = new_op<T>(BOP_CG);
    op.n_units = 1;
    op.n_cg = p.n_cg;
    op.rowptr = p.rowptr;
    op.col = p.col;
    op.val = p.val;
    op.fsrc = p.fsrc;
    op.uptr = p.uptr;
    op.udst = p.udst;
    op.umaster = p.umaster;
    op.work = work ? work : p.cg_work;
    op.iters = p.cg_iters;
    op.rtol = rtol;
    op.maxit = maxit;
    op.f = f;
    op.fI = fI;
    op.u = u;
    op.uI = uI;
    g_rec->push_back(op);
    return cudaSuccess;
  }
  if (p.n_cg == 0) return cudaSuccess;
  // the vectors live in shared memory when they fit and no work array is
  // imposed (the allocation-free cycle passes its static array)
  static std::mutex mu;
  static std::map<int, int> allow;   // device -> dynamic shared bytes allowed
  int dev = 0;
  cudaGetDevice(&dev);
  int lim = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = allow.find(dev);
    if (it == allow.end()) {
      int optin = 0;
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      const int a = std::max(0, optin - 4096);
      const cudaError_t e = cudaFuncSetAttribute((const void*)k_cg<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, a);
      if (e != cudaSuccess) return e;
      it = allow.emplace(dev, a).first;
    }
    lim = it->second;
  }
  const size_t bytes = (size_t)4 * p.n_cg * sizeof(double);
  const bool in_smem = !work && bytes <= (size_t)lim;
  ++g_kernel_launches;
  k_cg<T><<<1, CG_THREADS, in_smem ? bytes : 0, s>>>(p.n_cg, p.rowptr, p.col, p.val, p.fsrc, f, fI, p.uptr, p.udst,
                                                     p.umaster, u, uI, work ? work : p.cg_work, rtol, maxit,
                                                     p.cg_iters, in_smem ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t fma_probe(double* out, int blocks, int iters, cudaStream_t s) {
  ++g_kernel_launches;
  k_fma_probe<<<blocks, 256, 0, s>>>(out, iters, 0.999999, 1e-7);
  return cudaGetLastError();
}

cudaError_t reduce_partials(const double* partial, int n, double* out, cudaStream_t s) {
  if (g_rec) return cudaSuccess;   // a batch needs no norms
  ++g_kernel_launches;
  k_reduce<<<1, 1024, 0, s>>>(partial, n, out);
  return cudaGetLastError();
}

template <class T>
cudaError_t import_vec(const LevelArgs& L, const MacroGeo* geo, int n_macro, int64_t nx, int64_t ny, const double* g,
                       T* blocks, T* masters, bool closed, cudaStream_t s) {
  (void)masters;
  // interior imports also go through the closed-lattice tiles (the kernel
  // filters to the interior)
  if (L.n_tiles_all > 0) {
    ++g_kernel_launches;
    k_import_vol<T><<<dim3((unsigned)L.n_tiles_all, (unsigned)n_macro), cta_shape(), 0, s>>>(
        L.N, L.rs, L.block, geo, nx, ny, g, blocks, L.tiles_all, closed);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t export_vec(const LevelArgs& L, const MacroGeo* geo, int n_macro, int64_t nx, int64_t ny, const T* blocks,
                       const T* masters, double* g, cudaStream_t s) {
  (void)masters;
  if (L.n_tiles_all > 0) {
    ++g_kernel_launches;
    k_export_vol<T><<<dim3((unsigned)L.n_tiles_all, (unsigned)n_macro), cta_shape(), 0, s>>>(
        L.N, L.rs, L.block, geo, nx, ny, blocks, g, L.tiles_all);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t import_masters(const int64_t* gid, int n, const double* g, T* m, cudaStream_t s) {
  if (n > 0) {
    ++g_kernel_launches;
    k_import_if<T><<<lin_grid(n, 256), 256, 0, s>>>(gid, n, g, m);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t export_masters(const int64_t* gid, int n, const T* m, double* g, cudaStream_t s) {
  if (n > 0) {
    ++g_kernel_launches;
    k_export_if<T><<<lin_grid(n, 256), 256, 0, s>>>(gid, n, m, g);
  }
  return cudaGetLastError();
}

cudaError_t grad_partials(const LevelArgs& L, int n_macro, const double* u, const double* lam, const double* W,
                          double* partial, cudaStream_t s) {
  if (L.n_tiles_all > 0 && n_macro > 0) {
    ++g_kernel_launches;
    k_grad<<<dim3((unsigned)L.n_tiles_all, (unsigned)n_macro), cta_shape(), 0, s>>>(L.N, L.rs, L.block, u, lam, W,
                                                                                   L.tiles_all, partial);
  }
  return cudaGetLastError();
}

cudaError_t reduce_per_macro(const double* partial, int n_per, int n_macro, double* out, cudaStream_t s) {
  if (n_macro > 0) {
    ++g_kernel_launches;
    k_reduce_per_macro<<<n_macro, 256, 0, s>>>(partial, n_per, out);
  }
  return cudaGetLastError();
}

cudaError_t apply_if_nodes(const LevelArgs& L, const double* u, const double* uI, const double* W, bool seven_point,
                           const int* list, int n, double* out, cudaStream_t s) {
  if (n > 0) {
    ++g_kernel_launches;
    if (seven_point)
      k_if_apply<true><<<lin_grid(n, 128), 128, 0, s>>>(L.N, L.rs, L.block, u, uI, W, L.cptr, L.cps, list, n, out);
    else
      k_if_apply<false><<<lin_grid(n, 128), 128, 0, s>>>(L.N, L.rs, L.block, u, uI, W, L.cptr, L.cps, list, n, out);
  }
  return cudaGetLastError();
}

cudaError_t copy_listed(const double* src, double* dst, const int* idx, int n, cudaStream_t s) {
  if (n > 0) {
    ++g_kernel_launches;
    k_copy_listed<<<lin_grid(n, 256), 256, 0, s>>>(src, dst, idx, n);
  }
  return cudaGetLastError();
}

cudaError_t set_masters_zero(double* uI, const int* ids, int n, cudaStream_t s) {
  if (g_rec) {
    if (n <= 0) return cudaSuccess;
    BOp op = new_op<double>(BOP_SET_ZERO);
    op.uI = uI;
    op.ids = ids;
    op.n = n;
    op.n_units = (int)lin_grid(n, CTA);
    g_rec->push_back(op);
    return cudaSuccess;
  }
  if (n > 0) {
    ++g_kernel_launches;
    k_set_masters_zero<<<lin_grid(n, 256), 256, 0, s>>>(uI, ids, n);
  }
  return cudaGetLastError();
}

cudaError_t scale_blocks(const double* f, const double* winv, double* out, int n_macro, int64_t block,
                         cudaStream_t s) {
  const int64_t total = (int64_t)n_macro * block;
  if (total > 0) {
    ++g_kernel_launches;
    k_scale_blocks<<<(unsigned)std::min<int64_t>(lin_grid(total, 256), 152 * 16), 256, 0, s>>>(f, winv, out, n_macro,
                                                                                               block);
  }
  return cudaGetLastError();
}

cudaError_t restore_copies(double* u, const double* uI, const int64_t* off, const int* master, int n, cudaStream_t s) {
  if (g_rec) {
    if (n <= 0) return cudaSuccess;
    BOp op = new_op<double>(BOP_RESTORE);
    op.u = u;
    op.uI = (void*)uI;
    op.offs = off;
    op.ids = master;
    op.n = n;
    op.n_units = (int)lin_grid(n, CTA);
    g_rec->push_back(op);
    return cudaSuccess;
  }
  if (n > 0) {
    ++g_kernel_launches;
    k_restore<<<lin_grid(n, 256), 256, 0, s>>>(u, uI, off, master, n);
  }
  return cudaGetLastError();
}

cudaError_t residual_to_f32(const LevelArgs& L, const ProbArgs& p, const double* u, const double* uI, const double* f,
                            const double* fI, float* f32, float* fI32, const double* W, bool seven_point,
                            double* partial, int* n_part, cudaStream_t s) {
  if (g_rec) {
    const int nl = p.col_off[4];
    const Units g = units(nl, L.n_tiles_int, p.n_act);
    if (n_part) *n_part = 0;
    if (g.total == 0) return cudaSuccess;
    BOp op = new_op<double>(BOP_RES_F32);
    op.seven_point = seven_point ? 1 : 0;
    op.L = L;
    op.P = p;
    op.n_list = nl;
    op.n_if_units = g.n_if_units;
    op.n_units = g.total;
    op.u = (void*)u;
    op.uI = (void*)uI;
    op.f = f;
    op.fI = fI;
    op.o32 = f32;
    op.oI32 = fI32;
    op.W = W;
    g_rec->push_back(op);
    return cudaSuccess;
  }
  const int n = p.col_off[4];
  const Units g = units(n, L.n_tiles_int, p.n_act);
  if (n_part) *n_part = 0;
  if (g.total == 0) return cudaSuccess;
  auto kern = seven_point ? k_res_f32<true> : k_res_f32<false>;
  const unsigned grid = resident_grid((const void*)kern, g.total, p.grid_cap);
  if (n_part) *n_part = (int)grid;
  ++g_kernel_launches;
  kern<<<grid, cta_shape(), 0, s>>>(L.N, L.rs, L.block, u, uI, f, fI, f32, fI32, W, L.tiles_int, L.n_tiles_int, p.act,
                                    p.n_act, L.cptr, L.cps, p.free_if, n, if_tab<double>(p, 0), g.n_if_units, partial,
                                    p.sched);
  return cudaGetLastError();
}

cudaError_t add_correction(const LevelArgs& L, const ProbArgs& p, double* u, double* uI, const float* e,
                           const float* eI, cudaStream_t s) {
  if (g_rec) {
    if (p.n_act > 0) {
      BOp op = new_op<double>(BOP_ADD_BLOCKS);
      op.L = L;
      op.P = p;
      op.u = u;
      op.o32 = (void*)e;
      op.n_units = (int)(p.n_act * block_chunks(L.block));
      g_rec->push_back(op);
    }
    if (p.col_off[4] > 0) {
      BOp op = new_op<double>(BOP_ADD_MASTERS);
      op.uI = uI;
      op.oI32 = (void*)eI;
      op.ids = p.free_if;
      op.n = p.col_off[4];
      op.n_units = (int)lin_grid(op.n, CTA);
      g_rec->push_back(op);
    }
    return cudaSuccess;
  }
  if (p.n_act > 0) {
    const int64_t per = 256 * 8;
    const unsigned gx = (unsigned)std::min<int64_t>((L.block / 2 + per - 1) / per, 4096);
    ++g_kernel_launches;
    k_add_corr_blocks<<<dim3(gx, (unsigned)p.n_act), 256, 0, s>>>(u, e, L.block, p.act);
  }
  const int n = p.col_off[4];
  if (n > 0) {
    ++g_kernel_launches;
    k_add_corr_masters<<<lin_grid(n, 256), 256, 0, s>>>(uI, eI, p.free_if, n);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t zero_problem_blocks(const LevelArgs& L, const ProbArgs& p, T* u, T* uI, cudaStream_t s) {
  if (g_rec) {
    if (p.n_act > 0) {
      BOp op = new_op<T>(BOP_ZERO_BLOCKS);
      op.L = L;
      op.P = p;
      op.u = u;
      op.n_units = (int)(p.n_act * block_chunks(L.block));
      g_rec->push_back(op);
    }
    if (p.col_off[4] > 0) {
      BOp op = new_op<T>(BOP_ZERO_LIST);
      op.uI = uI;
      op.ids = p.free_if;
      op.n = p.col_off[4];
      op.n_units = (int)lin_grid(op.n, CTA);
      g_rec->push_back(op);
    }
    return cudaSuccess;
  }
  if (p.n_act > 0) {
    const int64_t per = 256 * 8;
    unsigned gx = (unsigned)std::min<int64_t>((L.block + per - 1) / per, 4096);
    ++g_kernel_launches;
    k_zero_blocks<T><<<dim3(gx, p.n_act), 256, 0, s>>>(u, L.block, p.act);
  }
  const int n = p.col_off[4];
  if (n > 0) {
    ++g_kernel_launches;
    k_zero_list<T><<<lin_grid(n, 256), 256, 0, s>>>(uI, p.free_if, n);
  }
  return cudaGetLastError();
}

#define HHG_INSTANTIATE(T)                                                                                        \
  template cudaError_t gs_colour<T>(const LevelArgs&, const ProbArgs&, T*, T*, const T*, const T*, const T*,   \
                                    const T*, int, bool, cudaStream_t, cudaEvent_t, cudaEvent_t, const T*,      \
                                    const T*);                                                                  \
  template cudaError_t residual<T>(const LevelArgs&, const ProbArgs&, const T*, const T*, const T*, const T*, T*, \
                                   const T*, bool, bool, double*, int*, cudaStream_t, int);                    \
  template cudaError_t restrict_to<T>(const LevelArgs&, const LevelArgs&, const ProbArgs&, const T*, T*, T*, T*, \
                                      T*, cudaStream_t);                                                       \
  template cudaError_t prolong_add<T>(const LevelArgs&, const LevelArgs&, const ProbArgs&, T*, T*, const T*,     \
                                      cudaStream_t, int, int, int);                                            \
  template cudaError_t coarse_cg<T>(const DevProblem&, const T*, const T*, T*, T*, double, int, cudaStream_t,     \
                                    double*);                                                                  \
  template cudaError_t import_vec<T>(const LevelArgs&, const MacroGeo*, int, int64_t, int64_t, const double*,    \
                                     T*, T*, bool, cudaStream_t);                                              \
  template cudaError_t export_vec<T>(const LevelArgs&, const MacroGeo*, int, int64_t, int64_t, const T*,         \
                                     const T*, double*, cudaStream_t);                                         \
  template cudaError_t import_masters<T>(const int64_t*, int, const double*, T*, cudaStream_t);                  \
  template cudaError_t export_masters<T>(const int64_t*, int, const T*, double*, cudaStream_t);                  \
  template cudaError_t zero_problem_blocks<T>(const LevelArgs&, const ProbArgs&, T*, T*, cudaStream_t);

HHG_INSTANTIATE(double)
HHG_INSTANTIATE(float)

}  // namespace hhg
