// Kernels of macro meshes of general connectivity (§2.1: an unstructured base
// mesh, refined uniformly): moving global vectors in the library's node order
// (interface nodes first, then the volume nodes macro by macro in local
// (k, j, i) order) into and out of the macro blocks, and the restriction
// onto coarse interface nodes whose fine neighbourhood has a variable size
// (a node at a macro-mesh vertex of high valence has more than 14 fine
// neighbours).  The volume kernels, interface stencils and coarse solver are
// those of kernels.cu.
#include <cuda_runtime.h>

#include "hhg_kernels.h"

namespace hhg {

namespace {

constexpr int GCTA = 256;

// One thread per volume node of every macro: t = q / nvol, and the local
// index q % nvol (order k, then j, then i; slice k holds T(N - 2 - k) nodes,
// T(m) = m (m + 1) / 2, row j of it N - 1 - j - k) mapped back to (i, j, k)
// by walking slices and rows.
__device__ __forceinline__ void vol_ijk(int N, int64_t l, int& i, int& j, int& k) {
  k = 1;
  for (;;) {
    const int64_t M = N - 2 - k;
    const int64_t sz = M * (M + 1) / 2;
    if (l < sz) break;
    l -= sz;
    ++k;
  }
  j = 1;
  for (;;) {
    const int64_t len = N - 1 - j - k;
    if (l < len) break;
    l -= len;
    ++j;
  }
  i = 1 + (int)l;
}

template <class T>
__global__ void __launch_bounds__(GCTA) k_gen_import_vol(int N, const int* __restrict__ rs, int64_t block,
                                                          int64_t n_if, int64_t nvol, int64_t total,
                                                          const double* __restrict__ g, T* __restrict__ blocks) {
  for (int64_t q = (int64_t)blockIdx.x * GCTA + threadIdx.x; q < total; q += (int64_t)gridDim.x * GCTA) {
    const int64_t t = q / nvol;
    int i, j, k;
    vol_ijk(N, q - t * nvol, i, j, k);
    blocks[t * block + lidx(rs, N, i, j, k)] = (T)g[n_if + q];
  }
}

template <class T>
__global__ void __launch_bounds__(GCTA) k_gen_export_vol(int N, const int* __restrict__ rs, int64_t block,
                                                          int64_t n_if, int64_t nvol, int64_t total,
                                                          const T* __restrict__ blocks, double* __restrict__ g) {
  for (int64_t q = (int64_t)blockIdx.x * GCTA + threadIdx.x; q < total; q += (int64_t)gridDim.x * GCTA) {
    const int64_t t = q / nvol;
    int i, j, k;
    vol_ijk(N, q - t * nvol, i, j, k);
    g[n_if + q] = (double)blocks[t * block + lidx(rs, N, i, j, k)];
  }
}

// Restriction onto the free coarse interface nodes (R = P^T: the coarse node
// itself with weight 1, the midpoints of its coarse edges with weight 1/2);
// the coarse correction starts from zero on them and on their copies, and at
// the problem's frozen copies.
template <class T>
__global__ void __launch_bounds__(GCTA) k_gen_restrict_if(int Nc, const int* __restrict__ rsc, int64_t bc,
                                                           T* __restrict__ fIc, T* __restrict__ uc,
                                                           T* __restrict__ uIc, const T* __restrict__ rf,
                                                           const int* __restrict__ cptr, const Copy* __restrict__ cps,
                                                           const int* __restrict__ list, int n_list,
                                                           const int* __restrict__ gptr,
                                                           const int64_t* __restrict__ goff,
                                                           const int64_t* __restrict__ zero_off, int n_zero) {
  const int q = blockIdx.x * GCTA + threadIdx.x;
  if (q < n_list) {
    const int node = list[q];
    const int e0 = gptr[q], e1 = gptr[q + 1];
    T acc = T(0);
    for (int e = e0 + 1; e < e1; ++e) acc += rf[goff[e]];
    fIc[node] = rf[goff[e0]] + T(0.5) * acc;
    uIc[node] = T(0);
    for (int c = cptr[node]; c < cptr[node + 1]; ++c) {
      const Copy cp = cps[c];
      uc[(int64_t)cp.macro * bc + lidx(rsc, Nc, cp.i, cp.j, cp.k)] = T(0);
    }
  } else if (q < n_list + n_zero) {
    uc[zero_off[q - n_list]] = T(0);
  }
}

inline unsigned gen_grid(int64_t n) {
  const int64_t g = (n + GCTA - 1) / GCTA;
  return (unsigned)(g < 152 * 16 ? (g > 0 ? g : 1) : 152 * 16);
}

}  // namespace

template <class T>
cudaError_t general_import_vol(const LevelArgs& L, int n_macro, int64_t n_if, const double* g, T* blocks,
                               cudaStream_t s) {
  const int64_t nvol = (int64_t)(L.N - 1) * (L.N - 2) * (L.N - 3) / 6;
  const int64_t total = nvol * n_macro;
  if (total == 0) return cudaSuccess;
  ++g_kernel_launches;
  k_gen_import_vol<T><<<gen_grid(total), GCTA, 0, s>>>(L.N, L.rs, L.block, n_if, nvol, total, g, blocks);
  return cudaGetLastError();
}

template <class T>
cudaError_t general_export_vol(const LevelArgs& L, int n_macro, int64_t n_if, const T* blocks, double* g,
                               cudaStream_t s) {
  const int64_t nvol = (int64_t)(L.N - 1) * (L.N - 2) * (L.N - 3) / 6;
  const int64_t total = nvol * n_macro;
  if (total == 0) return cudaSuccess;
  ++g_kernel_launches;
  k_gen_export_vol<T><<<gen_grid(total), GCTA, 0, s>>>(L.N, L.rs, L.block, n_if, nvol, total, blocks, g);
  return cudaGetLastError();
}

template <class T>
cudaError_t general_restrict_if(const LevelArgs& C, const ProbArgs& pc, const int* gptr, const int64_t* goff,
                                const T* rf, T* fIc, T* uc, T* uIc, cudaStream_t s) {
  const int n = pc.col_off[4];
  const int64_t total = (int64_t)n + pc.n_zero;
  if (total == 0) return cudaSuccess;
  ++g_kernel_launches;
  k_gen_restrict_if<T><<<(unsigned)((total + GCTA - 1) / GCTA), GCTA, 0, s>>>(
      C.N, C.rs, C.block, fIc, uc, uIc, rf, C.cptr, C.cps, pc.free_if, n, gptr, goff, pc.zero_off, pc.n_zero);
  return cudaGetLastError();
}

#define HHG_GENERAL_INSTANTIATE(T)                                                                              \
  template cudaError_t general_import_vol<T>(const LevelArgs&, int, int64_t, const double*, T*, cudaStream_t); \
  template cudaError_t general_export_vol<T>(const LevelArgs&, int, int64_t, const T*, double*, cudaStream_t); \
  template cudaError_t general_restrict_if<T>(const LevelArgs&, const ProbArgs&, const int*, const int64_t*,   \
                                              const T*, T*, T*, T*, cudaStream_t);

HHG_GENERAL_INSTANTIATE(double)
HHG_GENERAL_INSTANTIATE(float)

}  // namespace hhg
