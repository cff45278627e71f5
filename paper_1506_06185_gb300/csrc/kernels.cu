// CUDA kernels of the HHG multigrid for sm_103a.
//
// Volume kernels run over 8 x 32 tiles of one slice of a macro block (rows j,
// slots m of the colour-split layout) with one CTA per (tile, active macro);
// a warp reads 32 consecutive slots of one colour segment, so every stencil
// neighbour is a contiguous, sector-aligned access.  Interface kernels run one
// thread per face / edge / vertex node: they sum the sub-stencils of the
// macros around the node (§3.2, Fig. 4), update the master in the interface
// container and write the new value into the ghost shell of every adjacent
// block (the local half of the ghost update of §3.1).
#include <cuda_runtime.h>

#include <algorithm>

#include "hhg_kernels.h"

namespace hhg {

std::atomic<long long> g_kernel_launches{0};

namespace {

constexpr int VOL_THREADS = TILE_ROWS * TILE_SLOTS;   // 256

// 7-point structure: only the three chain axes (and negatives) are non-zero.
__host__ __device__ constexpr bool used_dir(int d, bool s7) {
  return !s7 || d == 1 || d == 2 || d == 3 || d == 8 || d == 9 || d == 10;
}

// 32-bit local index (a block holds fewer than 2^31 slots for N <= 1024);
// 64-bit integer arithmetic is kept out of the per-node work entirely.
__device__ __forceinline__ int slice32(int N, int P, int k) {
  return 4 * P * (k * (N + 1) - ((k * (k - 1)) >> 1));
}
__device__ __forceinline__ int lidx32(int N, int P, int i, int j, int k) {
  return slice32(N, P, k) + (4 * j + ((i + 2 * j + 3 * k) & 3)) * P + (i >> 2);
}

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
  return s;   // valid in thread 0
}

// ---------------------------------------------------------------------------
// Gauss-Seidel, one colour
// ---------------------------------------------------------------------------
template <class T, bool S7>
__global__ void __launch_bounds__(VOL_THREADS) k_gs_vol(int N, int P, int64_t block, T* __restrict__ u,
                                                        const T* __restrict__ f, const T* __restrict__ W,
                                                        const T* __restrict__ Winv, const Tile* __restrict__ tiles,
                                                        const int* __restrict__ act, int colour) {
  const Tile t = tiles[blockIdx.x];
  const int macro = act[blockIdx.y];
  const int k = t.k;
  const int j = t.j0 + threadIdx.y;
  const int m = t.m0 + threadIdx.x;
  const int i = 4 * m + ((colour - 2 * j - 3 * k) & 3);
  if (j < 1 || i < 1 || i + j + k > N - 1) return;
  T* ub = u + (size_t)macro * block;
  const T* fb = f + (size_t)macro * block;
  const T* w = W + (size_t)macro * 16 * NDIR;
  const int me = lidx32(N, P, i, j, k);
  T acc = fb[me];
#pragma unroll
  for (int d = 1; d < NDIR; ++d) {
    if (!used_dir(d, S7)) continue;
    int di, dj, dk;
    dir_ijk(d, di, dj, dk);
    acc -= w[d] * ub[lidx32(N, P, i + di, j + dj, k + dk)];
  }
  ub[me] = acc * Winv[macro];
}

template <class T>
__global__ void k_gs_if(int N, int P, int64_t block, T* __restrict__ u, T* __restrict__ uI,
                        const T* __restrict__ fI, const T* __restrict__ W, const int* __restrict__ cptr,
                        const Copy* __restrict__ cps, const int* __restrict__ list, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int node = list[q];
  T acc = fI[node];
  T diag = T(0);
  const int c0 = cptr[node], c1 = cptr[node + 1];
  for (int c = c0; c < c1; ++c) {
    const Copy cp = cps[c];
    const T* w = W + ((size_t)cp.macro * 16 + node_class(cp.i, cp.j, cp.k, N)) * NDIR;
    const T* ub = u + (size_t)cp.macro * block;
    diag += w[0];
#pragma unroll
    for (int d = 1; d < NDIR; ++d) {
      const T wd = w[d];
      if (wd == T(0)) continue;
      int di, dj, dk;
      dir_ijk(d, di, dj, dk);
      const int ni = cp.i + di, nj = cp.j + dj, nk = cp.k + dk;
      if (!in_lattice(ni, nj, nk, N)) continue;
      acc -= wd * ub[lidx32(N, P, ni, nj, nk)];
    }
  }
  const T val = acc / diag;
  uI[node] = val;
  for (int c = c0; c < c1; ++c) {
    const Copy cp = cps[c];
    u[(size_t)cp.macro * block + lidx32(N, P, cp.i, cp.j, cp.k)] = val;
  }
}

// ---------------------------------------------------------------------------
// Residual (all colours); optional write and norm partials
// ---------------------------------------------------------------------------
template <class T, bool S7, bool WRITE, bool NORM>
__global__ void __launch_bounds__(VOL_THREADS) k_res_vol(int N, int P, int64_t block, const T* __restrict__ u,
                                                         const T* __restrict__ f, T* __restrict__ r,
                                                         const T* __restrict__ W, const Tile* __restrict__ tiles,
                                                         const int* __restrict__ act, double* __restrict__ partial) {
  __shared__ double sh[32];
  const Tile t = tiles[blockIdx.x];
  const int macro = act[blockIdx.y];
  const int k = t.k;
  const int j = t.j0 + threadIdx.y;
  const int m = t.m0 + threadIdx.x;
  const T* ub = u + (size_t)macro * block;
  const T* fb = f + (size_t)macro * block;
  T* rb = r + (size_t)macro * block;
  const T* w = W + (size_t)macro * 16 * NDIR;
  double ss = 0.0;
  if (j >= 1) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = 4 * m + q;
      if (i < 1 || i + j + k > N - 1) continue;
      const int me = lidx32(N, P, i, j, k);
      T acc = fb[me] - w[0] * ub[me];
#pragma unroll
      for (int d = 1; d < NDIR; ++d) {
        if (!used_dir(d, S7)) continue;
        int di, dj, dk;
        dir_ijk(d, di, dj, dk);
        acc -= w[d] * ub[lidx32(N, P, i + di, j + dj, k + dk)];
      }
      if (WRITE) rb[me] = acc;
      if (NORM) ss += (double)acc * (double)acc;
    }
  }
  if (NORM) {
    double s = block_sum(ss, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

template <class T, bool WRITE, bool NORM>
__global__ void k_res_if(int N, int P, int64_t block, const T* __restrict__ u, const T* __restrict__ fI,
                         T* __restrict__ r, const T* __restrict__ W, const int* __restrict__ cptr,
                         const Copy* __restrict__ cps, const int* __restrict__ list, int n,
                         const int64_t* __restrict__ zero_off, int n_zero, double* __restrict__ partial) {
  __shared__ double sh[32];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  double ss = 0.0;
  if (q < n) {
    const int node = list[q];
    T acc = fI[node];
    const int c0 = cptr[node], c1 = cptr[node + 1];
    for (int c = c0; c < c1; ++c) {
      const Copy cp = cps[c];
      const T* w = W + ((size_t)cp.macro * 16 + node_class(cp.i, cp.j, cp.k, N)) * NDIR;
      const T* ub = u + (size_t)cp.macro * block;
      acc -= w[0] * ub[lidx32(N, P, cp.i, cp.j, cp.k)];
#pragma unroll
      for (int d = 1; d < NDIR; ++d) {
        const T wd = w[d];
        if (wd == T(0)) continue;
        int di, dj, dk;
        dir_ijk(d, di, dj, dk);
        const int ni = cp.i + di, nj = cp.j + dj, nk = cp.k + dk;
        if (!in_lattice(ni, nj, nk, N)) continue;
        acc -= wd * ub[lidx32(N, P, ni, nj, nk)];
      }
    }
    if (WRITE)
      for (int c = c0; c < c1; ++c) {
        const Copy cp = cps[c];
        r[(size_t)cp.macro * block + lidx32(N, P, cp.i, cp.j, cp.k)] = acc;
      }
    if (NORM) ss = (double)acc * (double)acc;
  } else if (WRITE && q < n + n_zero) {
    r[zero_off[q - n]] = T(0);
  }
  if (NORM) {
    double s = block_sum(ss, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Restriction R = P^T onto the coarse level; zero the coarse correction
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(VOL_THREADS) k_restrict_vol(int Nc, int Pc, int64_t bc, T* __restrict__ fc,
                                                              T* __restrict__ uc, int Nf, int Pf, int64_t bf,
                                                              const T* __restrict__ rf, const Tile* __restrict__ tiles,
                                                              const int* __restrict__ act) {
  const Tile t = tiles[blockIdx.x];
  const int macro = act[blockIdx.y];
  const int k = t.k;
  const int j = t.j0 + threadIdx.y;
  const int m = t.m0 + threadIdx.x;
  if (j < 1) return;
  const T* rb = rf + (size_t)macro * bf;
  T* fb = fc + (size_t)macro * bc;
  T* ub = uc + (size_t)macro * bc;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 4 * m + q;
    if (i < 1 || i + j + k > Nc - 1) continue;
    const int fi = 2 * i, fj = 2 * j, fk = 2 * k;
    T acc = T(0);
#pragma unroll
    for (int d = 1; d < NDIR; ++d) {
      int di, dj, dk;
      dir_ijk(d, di, dj, dk);
      acc += rb[lidx32(Nf, Pf, fi + di, fj + dj, fk + dk)];
    }
    const int me = lidx32(Nc, Pc, i, j, k);
    fb[me] = rb[lidx32(Nf, Pf, fi, fj, fk)] + T(0.5) * acc;
    ub[me] = T(0);
  }
}

template <class T>
__global__ void k_restrict_if(int Nc, int Pc, int64_t bc, const T* __restrict__ rf, T* __restrict__ fIc,
                              T* __restrict__ uc, T* __restrict__ uIc, const int* __restrict__ cptr,
                              const Copy* __restrict__ cps, const int* __restrict__ list, int n,
                              const int64_t* __restrict__ gather, const int64_t* __restrict__ zero_off, int n_zero) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) {
    const int node = list[q];
    const int64_t* g = gather + (size_t)q * NDIR;
    T acc = T(0);
    for (int e = 1; e < NDIR; ++e) acc += rf[g[e]];
    fIc[node] = rf[g[0]] + T(0.5) * acc;
    uIc[node] = T(0);
    for (int c = cptr[node]; c < cptr[node + 1]; ++c) {
      const Copy cp = cps[c];
      uc[(size_t)cp.macro * bc + lidx32(Nc, Pc, cp.i, cp.j, cp.k)] = T(0);
    }
  } else if (q < n + n_zero) {
    uc[zero_off[q - n]] = T(0);
  }
}

// ---------------------------------------------------------------------------
// Prolongation u_f += P u_c
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T interp(const T* __restrict__ cb, int Nc, int Pc, int i, int j, int k) {
  const int pi = i & 1, pj = j & 1, pk = k & 1;
  if (!(pi | pj | pk)) return cb[lidx32(Nc, Pc, i >> 1, j >> 1, k >> 1)];
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
  const T a = cb[lidx32(Nc, Pc, (i - di) >> 1, (j - dj) >> 1, (k - dk) >> 1)];
  const T b = cb[lidx32(Nc, Pc, (i + di) >> 1, (j + dj) >> 1, (k + dk) >> 1)];
  return T(0.5) * (a + b);
}

template <class T>
__global__ void __launch_bounds__(VOL_THREADS) k_prolong_vol(int Nf, int Pf, int64_t bf, T* __restrict__ uf, int Nc,
                                                             int Pc, int64_t bc, const T* __restrict__ uc,
                                                             const Tile* __restrict__ tiles,
                                                             const int* __restrict__ act) {
  const Tile t = tiles[blockIdx.x];
  const int macro = act[blockIdx.y];
  const int k = t.k;
  const int j = t.j0 + threadIdx.y;
  const int m = t.m0 + threadIdx.x;
  if (j < 1) return;
  T* fb = uf + (size_t)macro * bf;
  const T* cb = uc + (size_t)macro * bc;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 4 * m + q;
    if (i < 1 || i + j + k > Nf - 1) continue;
    const int me = lidx32(Nf, Pf, i, j, k);
    fb[me] += interp(cb, Nc, Pc, i, j, k);
  }
}

template <class T>
__global__ void k_prolong_if(int Nf, int Pf, int64_t bf, T* __restrict__ uf, T* __restrict__ uIf, int Nc, int Pc,
                             int64_t bc, const T* __restrict__ uc, const int* __restrict__ cptr,
                             const Copy* __restrict__ cps, const int* __restrict__ list, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int node = list[q];
  const int c0 = cptr[node], c1 = cptr[node + 1];
  const Copy c0p = cps[c0];
  const T corr = interp(uc + (size_t)c0p.macro * bc, Nc, Pc, c0p.i, c0p.j, c0p.k);
  const T val = uIf[node] + corr;
  uIf[node] = val;
  for (int c = c0; c < c1; ++c) {
    const Copy cp = cps[c];
    uf[(size_t)cp.macro * bf + lidx32(Nf, Pf, cp.i, cp.j, cp.k)] = val;
  }
}

// ---------------------------------------------------------------------------
// Coarse-level CG, one CTA (FP64; §2.1 coarse solver)
// ---------------------------------------------------------------------------
constexpr int CG_THREADS = 1024;

__device__ __forceinline__ double cta_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = sh[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) sh[32] = s;
  }
  __syncthreads();
  return sh[32];
}

template <class T>
__global__ void __launch_bounds__(CG_THREADS) k_cg(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                                   const double* __restrict__ val, const int64_t* __restrict__ fsrc,
                                                   const T* __restrict__ f, const T* __restrict__ fI,
                                                   const int* __restrict__ uptr, const int64_t* __restrict__ udst,
                                                   const int* __restrict__ umaster, T* __restrict__ u,
                                                   T* __restrict__ uI, double* __restrict__ work, double rtol,
                                                   int maxit, int* __restrict__ iters) {
  __shared__ double sh[33];
  double* x = work;
  double* r = work + n;
  double* p = work + 2 * (size_t)n;
  double* Ap = work + 3 * (size_t)n;
  double part = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int64_t s = fsrc[q];
    const double b = s >= 0 ? (double)f[s] : (double)fI[-1 - s];
    x[q] = 0.0;
    r[q] = b;
    p[q] = b;
    part += b * b;
  }
  double rr = cta_sum(part, sh);
  const double bnorm = sqrt(rr);
  int it = 0;
  while (bnorm > 0.0 && sqrt(rr) > rtol * bnorm && it < maxit) {
    part = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      double a = 0.0;
      for (int e = rowptr[q]; e < rowptr[q + 1]; ++e) a += val[e] * p[col[e]];
      Ap[q] = a;
      part += p[q] * a;
    }
    const double pAp = cta_sum(part, sh);
    const double alpha = rr / pAp;
    part = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      x[q] += alpha * p[q];
      const double rq = r[q] - alpha * Ap[q];
      r[q] = rq;
      part += rq * rq;
    }
    const double rr_new = cta_sum(part, sh);
    const double beta = rr_new / rr;
    for (int q = threadIdx.x; q < n; q += blockDim.x) p[q] = r[q] + beta * p[q];
    rr = rr_new;
    ++it;
    __syncthreads();
  }
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const T v = (T)x[q];
    for (int e = uptr[q]; e < uptr[q + 1]; ++e) u[udst[e]] = v;
    if (umaster[q] >= 0) uI[umaster[q]] = v;
  }
  if (threadIdx.x == 0 && iters) *iters = it;
}

__global__ void k_reduce(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double sh[33];
  double s = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += partial[q];
  s = cta_sum(s, sh);
  if (threadIdx.x == 0) out[0] = s;
}

// ---------------------------------------------------------------------------
// Global vector <-> blocks
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t dev_gid(const MacroGeo& g, int N, int i, int j, int k, int64_t nx, int64_t ny) {
  const int64_t X = (int64_t)N * g.v0[0] + (int64_t)i * g.e1[0] + (int64_t)j * g.e2[0] + (int64_t)k * g.e3[0];
  const int64_t Y = (int64_t)N * g.v0[1] + (int64_t)i * g.e1[1] + (int64_t)j * g.e2[1] + (int64_t)k * g.e3[1];
  const int64_t Z = (int64_t)N * g.v0[2] + (int64_t)i * g.e1[2] + (int64_t)j * g.e2[2] + (int64_t)k * g.e3[2];
  return (Z * (ny + 1) + Y) * (nx + 1) + X;
}

template <class T>
__global__ void __launch_bounds__(VOL_THREADS) k_import_vol(int N, int P, int64_t block, const MacroGeo* __restrict__ geo,
                                                            int64_t nx, int64_t ny, const double* __restrict__ g,
                                                            T* __restrict__ dst, const Tile* __restrict__ tiles,
                                                            bool closed) {
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
    b[lidx32(N, P, i, j, k)] = (T)g[dev_gid(gm, N, i, j, k, nx, ny)];
  }
}

template <class T>
__global__ void __launch_bounds__(VOL_THREADS) k_export_vol(int N, int P, int64_t block, const MacroGeo* __restrict__ geo,
                                                            int64_t nx, int64_t ny, const T* __restrict__ src,
                                                            double* __restrict__ g, const Tile* __restrict__ tiles) {
  const Tile t = tiles[blockIdx.x];
  const int macro = blockIdx.y;
  const int k = t.k;
  const int j = t.j0 + threadIdx.y;
  const int m = t.m0 + threadIdx.x;
  const MacroGeo gm = geo[macro];
  const T* b = src + (size_t)macro * block;
  if (j < 1) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 4 * m + q;
    if (i < 1 || i + j + k > N - 1) continue;
    g[dev_gid(gm, N, i, j, k, nx, ny)] = (double)b[lidx32(N, P, i, j, k)];
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

__global__ void k_set_masters_zero(double* __restrict__ uI, const int* __restrict__ ids, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) uI[ids[q]] = 0.0;
}

__global__ void k_restore(double* __restrict__ u, const double* __restrict__ uI, const int64_t* __restrict__ off,
                          const int* __restrict__ master, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) u[off[q]] = uI[master[q]];
}

// ---------------------------------------------------------------------------
// Mixed precision helpers
// ---------------------------------------------------------------------------
template <bool S7>
__global__ void __launch_bounds__(VOL_THREADS) k_res_vol_f32(int N, int P, int64_t block, const double* __restrict__ u,
                                                             const double* __restrict__ f, float* __restrict__ f32,
                                                             const double* __restrict__ W, const Tile* __restrict__ tiles,
                                                             const int* __restrict__ act, double* __restrict__ partial) {
  __shared__ double sh[32];
  const Tile t = tiles[blockIdx.x];
  const int macro = act[blockIdx.y];
  const int k = t.k;
  const int j = t.j0 + threadIdx.y;
  const int m = t.m0 + threadIdx.x;
  const double* ub = u + (size_t)macro * block;
  const double* fb = f + (size_t)macro * block;
  float* ob = f32 + (size_t)macro * block;
  const double* w = W + (size_t)macro * 16 * NDIR;
  double ss = 0.0;
  if (j >= 1) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = 4 * m + q;
      if (i < 1 || i + j + k > N - 1) continue;
      const int me = lidx32(N, P, i, j, k);
      double acc = fb[me] - w[0] * ub[me];
#pragma unroll
      for (int d = 1; d < NDIR; ++d) {
        if (!used_dir(d, S7)) continue;
        int di, dj, dk;
        dir_ijk(d, di, dj, dk);
        acc -= w[d] * ub[lidx32(N, P, i + di, j + dj, k + dk)];
      }
      ob[me] = (float)acc;
      ss += acc * acc;
    }
  }
  double s = block_sum(ss, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

__global__ void k_res_if_f32(int N, int P, int64_t block, const double* __restrict__ u, const double* __restrict__ fI,
                             float* __restrict__ fI32, const double* __restrict__ W, const int* __restrict__ cptr,
                             const Copy* __restrict__ cps, const int* __restrict__ list, int n,
                             double* __restrict__ partial) {
  __shared__ double sh[32];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  double ss = 0.0;
  if (q < n) {
    const int node = list[q];
    double acc = fI[node];
    for (int c = cptr[node]; c < cptr[node + 1]; ++c) {
      const Copy cp = cps[c];
      const double* w = W + ((size_t)cp.macro * 16 + node_class(cp.i, cp.j, cp.k, N)) * NDIR;
      const double* ub = u + (size_t)cp.macro * block;
      acc -= w[0] * ub[lidx32(N, P, cp.i, cp.j, cp.k)];
      for (int d = 1; d < NDIR; ++d) {
        const double wd = w[d];
        if (wd == 0.0) continue;
        int di, dj, dk;
        dir_ijk(d, di, dj, dk);
        const int ni = cp.i + di, nj = cp.j + dj, nk = cp.k + dk;
        if (!in_lattice(ni, nj, nk, N)) continue;
        acc -= wd * ub[lidx32(N, P, ni, nj, nk)];
      }
    }
    fI32[node] = (float)acc;
    ss = acc * acc;
  }
  double s = block_sum(ss, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(VOL_THREADS) k_add_corr_vol(int N, int P, int64_t block, double* __restrict__ u,
                                                              const float* __restrict__ e, const Tile* __restrict__ tiles,
                                                              const int* __restrict__ act) {
  const Tile t = tiles[blockIdx.x];
  const int macro = act[blockIdx.y];
  const int k = t.k;
  const int j = t.j0 + threadIdx.y;
  const int m = t.m0 + threadIdx.x;
  if (j < 1) return;
  double* ub = u + (size_t)macro * block;
  const float* eb = e + (size_t)macro * block;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 4 * m + q;
    if (i < 1 || i + j + k > N - 1) continue;
    const int me = lidx32(N, P, i, j, k);
    ub[me] += (double)eb[me];
  }
}

__global__ void k_add_corr_if(int N, int P, int64_t block, double* __restrict__ u, double* __restrict__ uI,
                              const float* __restrict__ eI, const int* __restrict__ cptr, const Copy* __restrict__ cps,
                              const int* __restrict__ list, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int node = list[q];
  const double val = uI[node] + (double)eI[node];
  uI[node] = val;
  for (int c = cptr[node]; c < cptr[node + 1]; ++c) {
    const Copy cp = cps[c];
    u[(size_t)cp.macro * block + lidx32(N, P, cp.i, cp.j, cp.k)] = val;
  }
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

inline dim3 vol_grid(int n_tiles, int n_macro) { return dim3((unsigned)n_tiles, (unsigned)n_macro); }
inline dim3 vol_block() { return dim3(TILE_SLOTS, TILE_ROWS); }
inline unsigned lin_grid(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class T>
cudaError_t gs_colour(const LevelArgs& L, const ProbArgs& p, T* u, T* uI, const T* f, const T* fI, const T* W,
                      const T* Winv, int colour, bool seven_point, cudaStream_t s, cudaEvent_t ev_begin,
                      cudaEvent_t ev_end) {
  if (p.n_act > 0 && L.n_tiles_int > 0) {
    if (ev_begin) cudaEventRecord(ev_begin, s);
    if (seven_point)
      { ++g_kernel_launches; k_gs_vol<T, true><<<vol_grid(L.n_tiles_int, p.n_act), vol_block(), 0, s>>>(L.N, L.P, L.block, u, f, W, Winv,
                                                                                  L.tiles_int, p.act, colour); }
    else
      { ++g_kernel_launches; k_gs_vol<T, false><<<vol_grid(L.n_tiles_int, p.n_act), vol_block(), 0, s>>>(L.N, L.P, L.block, u, f, W, Winv,
                                                                                   L.tiles_int, p.act, colour); }
    if (ev_end) cudaEventRecord(ev_end, s);
  }
  const int n = p.col_off[colour + 1] - p.col_off[colour];
  if (n > 0)
    { ++g_kernel_launches; k_gs_if<T><<<lin_grid(n, 128), 128, 0, s>>>(L.N, L.P, L.block, u, uI, fI, W, L.cptr, L.cps,
                                                p.free_if + p.col_off[colour], n); }
  return cudaGetLastError();
}

template <class T>
cudaError_t residual(const LevelArgs& L, const ProbArgs& p, const T* u, const T* uI, const T* f, const T* fI, T* r,
                     const T* W, bool seven_point, bool write_r, double* partial, int* n_part, cudaStream_t s) {
  (void)uI;
  int np = 0;
  const bool norm = partial != nullptr;
  if (p.n_act > 0 && L.n_tiles_int > 0) {
    dim3 g = vol_grid(L.n_tiles_int, p.n_act);
#define HHG_RES_VOL(S7, WR, NO)                                                                          \
  do {                                                                                                    \
    ++g_kernel_launches;                                                                                  \
    k_res_vol<T, S7, WR, NO><<<g, vol_block(), 0, s>>>(L.N, L.P, L.block, u, f, r, W, L.tiles_int, p.act, \
                                                       partial);                                          \
  } while (0)
    if (seven_point) {
      if (write_r && norm) HHG_RES_VOL(true, true, true);
      else if (write_r) HHG_RES_VOL(true, true, false);
      else if (norm) HHG_RES_VOL(true, false, true);
    } else {
      if (write_r && norm) HHG_RES_VOL(false, true, true);
      else if (write_r) HHG_RES_VOL(false, true, false);
      else if (norm) HHG_RES_VOL(false, false, true);
    }
#undef HHG_RES_VOL
    np = (int)(g.x * g.y);
  }
  const int n = p.col_off[4];
  const int total = n + (write_r ? p.n_zero : 0);
  if (total > 0) {
    const unsigned gb = lin_grid(total, 128);
    double* pp = norm ? partial + np : nullptr;
    if (write_r && norm)
      { ++g_kernel_launches; k_res_if<T, true, true><<<gb, 128, 0, s>>>(L.N, L.P, L.block, u, fI, r, W, L.cptr, L.cps, p.free_if, n,
                                                 p.zero_off, p.n_zero, pp); }
    else if (write_r)
      { ++g_kernel_launches; k_res_if<T, true, false><<<gb, 128, 0, s>>>(L.N, L.P, L.block, u, fI, r, W, L.cptr, L.cps, p.free_if, n,
                                                  p.zero_off, p.n_zero, pp); }
    else
      { ++g_kernel_launches; k_res_if<T, false, true><<<gb, 128, 0, s>>>(L.N, L.P, L.block, u, fI, r, W, L.cptr, L.cps, p.free_if, n,
                                                  p.zero_off, p.n_zero, pp); }
    if (norm) np += (int)gb;
  }
  if (n_part) *n_part = np;
  return cudaGetLastError();
}

template <class T>
cudaError_t restrict_to(const LevelArgs& C, const LevelArgs& F, const ProbArgs& pc, const T* rf, T* fc, T* fIc, T* uc,
                        T* uIc, cudaStream_t s) {
  if (pc.n_act > 0 && C.n_tiles_int > 0)
    { ++g_kernel_launches; k_restrict_vol<T><<<vol_grid(C.n_tiles_int, pc.n_act), vol_block(), 0, s>>>(C.N, C.P, C.block, fc, uc, F.N, F.P,
                                                                                 F.block, rf, C.tiles_int, pc.act); }
  const int n = pc.col_off[4];
  const int total = n + pc.n_zero;
  if (total > 0)
    { ++g_kernel_launches; k_restrict_if<T><<<lin_grid(total, 128), 128, 0, s>>>(C.N, C.P, C.block, rf, fIc, uc, uIc, C.cptr, C.cps,
                                                          pc.free_if, n, pc.gather, pc.zero_off, pc.n_zero); }
  return cudaGetLastError();
}

template <class T>
cudaError_t prolong_add(const LevelArgs& F, const LevelArgs& C, const ProbArgs& pf, T* uf, T* uIf, const T* uc,
                        cudaStream_t s) {
  if (pf.n_act > 0 && F.n_tiles_int > 0)
    { ++g_kernel_launches; k_prolong_vol<T><<<vol_grid(F.n_tiles_int, pf.n_act), vol_block(), 0, s>>>(F.N, F.P, F.block, uf, C.N, C.P,
                                                                                C.block, uc, F.tiles_int, pf.act); }
  const int n = pf.col_off[4];
  if (n > 0)
    { ++g_kernel_launches; k_prolong_if<T><<<lin_grid(n, 128), 128, 0, s>>>(F.N, F.P, F.block, uf, uIf, C.N, C.P, C.block, uc, F.cptr,
                                                     F.cps, pf.free_if, n); }
  return cudaGetLastError();
}

template <class T>
cudaError_t coarse_cg(const DevProblem& p, const T* f, const T* fI, T* u, T* uI, double rtol, int maxit,
                      cudaStream_t s) {
  if (p.n_cg == 0) return cudaSuccess;
  { ++g_kernel_launches; k_cg<T><<<1, CG_THREADS, 0, s>>>(p.n_cg, p.rowptr, p.col, p.val, p.fsrc, f, fI, p.uptr, p.udst, p.umaster, u, uI,
                                   p.cg_work, rtol, maxit, p.cg_iters); }
  return cudaGetLastError();
}

cudaError_t reduce_partials(const double* partial, int n, double* out, cudaStream_t s) {
  { ++g_kernel_launches; k_reduce<<<1, 1024, 0, s>>>(partial, n, out); }
  return cudaGetLastError();
}

template <class T>
cudaError_t import_vec(const LevelArgs& L, const MacroGeo* geo, int n_macro, int64_t nx, int64_t ny, const double* g,
                       T* blocks, T* masters, bool closed, cudaStream_t s) {
  const Tile* tl = closed ? L.tiles_all : L.tiles_int;
  const int nt = closed ? L.n_tiles_all : L.n_tiles_int;
  if (nt > 0)
    { ++g_kernel_launches; k_import_vol<T><<<vol_grid(nt, n_macro), vol_block(), 0, s>>>(L.N, L.P, L.block, geo, nx, ny, g, blocks, tl,
                                                                   closed); }
  (void)masters;
  return cudaGetLastError();
}

template <class T>
cudaError_t export_vec(const LevelArgs& L, const MacroGeo* geo, int n_macro, int64_t nx, int64_t ny, const T* blocks,
                       const T* masters, double* g, cudaStream_t s) {
  (void)masters;
  if (L.n_tiles_int > 0)
    { ++g_kernel_launches; k_export_vol<T><<<vol_grid(L.n_tiles_int, n_macro), vol_block(), 0, s>>>(L.N, L.P, L.block, geo, nx, ny, blocks,
                                                                              g, L.tiles_int); }
  return cudaGetLastError();
}

template <class T>
cudaError_t import_masters(const int64_t* gid, int n, const double* g, T* m, cudaStream_t s) {
  if (n > 0) { ++g_kernel_launches; k_import_if<T><<<lin_grid(n, 256), 256, 0, s>>>(gid, n, g, m); }
  return cudaGetLastError();
}

template <class T>
cudaError_t export_masters(const int64_t* gid, int n, const T* m, double* g, cudaStream_t s) {
  if (n > 0) { ++g_kernel_launches; k_export_if<T><<<lin_grid(n, 256), 256, 0, s>>>(gid, n, m, g); }
  return cudaGetLastError();
}

cudaError_t set_masters_zero(double* uI, const int* ids, int n, cudaStream_t s) {
  if (n > 0) { ++g_kernel_launches; k_set_masters_zero<<<lin_grid(n, 256), 256, 0, s>>>(uI, ids, n); }
  return cudaGetLastError();
}

cudaError_t restore_copies(double* u, const double* uI, const int64_t* off, const int* master, int n, cudaStream_t s) {
  if (n > 0) { ++g_kernel_launches; k_restore<<<lin_grid(n, 256), 256, 0, s>>>(u, uI, off, master, n); }
  return cudaGetLastError();
}

cudaError_t residual_to_f32(const LevelArgs& L, const ProbArgs& p, const double* u, const double* uI, const double* f,
                            const double* fI, float* f32, float* fI32, const double* W, bool seven_point,
                            double* partial, int* n_part, cudaStream_t s) {
  (void)uI;
  int np = 0;
  if (p.n_act > 0 && L.n_tiles_int > 0) {
    dim3 g = vol_grid(L.n_tiles_int, p.n_act);
    if (seven_point)
      { ++g_kernel_launches; k_res_vol_f32<true><<<g, vol_block(), 0, s>>>(L.N, L.P, L.block, u, f, f32, W, L.tiles_int, p.act, partial); }
    else
      { ++g_kernel_launches; k_res_vol_f32<false><<<g, vol_block(), 0, s>>>(L.N, L.P, L.block, u, f, f32, W, L.tiles_int, p.act, partial); }
    np = (int)(g.x * g.y);
  }
  const int n = p.col_off[4];
  if (n > 0) {
    const unsigned gb = lin_grid(n, 128);
    { ++g_kernel_launches; k_res_if_f32<<<gb, 128, 0, s>>>(L.N, L.P, L.block, u, fI, fI32, W, L.cptr, L.cps, p.free_if, n, partial + np); }
    np += (int)gb;
  }
  if (n_part) *n_part = np;
  return cudaGetLastError();
}

cudaError_t add_correction(const LevelArgs& L, const ProbArgs& p, double* u, double* uI, const float* e,
                           const float* eI, cudaStream_t s) {
  if (p.n_act > 0 && L.n_tiles_int > 0)
    { ++g_kernel_launches; k_add_corr_vol<<<vol_grid(L.n_tiles_int, p.n_act), vol_block(), 0, s>>>(L.N, L.P, L.block, u, e, L.tiles_int,
                                                                             p.act); }
  const int n = p.col_off[4];
  if (n > 0)
    { ++g_kernel_launches; k_add_corr_if<<<lin_grid(n, 128), 128, 0, s>>>(L.N, L.P, L.block, u, uI, eI, L.cptr, L.cps, p.free_if, n); }
  return cudaGetLastError();
}

template <class T>
cudaError_t zero_problem_blocks(const LevelArgs& L, const ProbArgs& p, T* u, T* uI, cudaStream_t s) {
  if (p.n_act > 0) {
    const int64_t per = 256 * 8;
    unsigned gx = (unsigned)std::min<int64_t>((L.block + per - 1) / per, 4096);
    { ++g_kernel_launches; k_zero_blocks<T><<<dim3(gx, p.n_act), 256, 0, s>>>(u, L.block, p.act); }
  }
  const int n = p.col_off[4];
  if (n > 0) { ++g_kernel_launches; k_zero_list<T><<<lin_grid(n, 256), 256, 0, s>>>(uI, p.free_if, n); }
  return cudaGetLastError();
}

#define HHG_INSTANTIATE(T)                                                                                        \
  template cudaError_t gs_colour<T>(const LevelArgs&, const ProbArgs&, T*, T*, const T*, const T*, const T*,   \
                                    const T*, int, bool, cudaStream_t, cudaEvent_t, cudaEvent_t);               \
  template cudaError_t residual<T>(const LevelArgs&, const ProbArgs&, const T*, const T*, const T*, const T*, T*, \
                                   const T*, bool, bool, double*, int*, cudaStream_t);                         \
  template cudaError_t restrict_to<T>(const LevelArgs&, const LevelArgs&, const ProbArgs&, const T*, T*, T*, T*, \
                                      T*, cudaStream_t);                                                       \
  template cudaError_t prolong_add<T>(const LevelArgs&, const LevelArgs&, const ProbArgs&, T*, T*, const T*,     \
                                      cudaStream_t);                                                           \
  template cudaError_t coarse_cg<T>(const DevProblem&, const T*, const T*, T*, T*, double, int, cudaStream_t);   \
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
