// Host-side check of the mesh builder (csrc/mesh.cpp) against the oracle,
// driven by tests/test_host_mesh.py: for every level it applies the per-macro
// stencils and the interface sub-stencil sums to a global vector (as the CUDA
// kernels do, through the macro blocks and the copy lists), and for every
// problem kind it applies the restriction gathers and dumps the coarse CG
// matrix.  Runs on the CPU; makes no CUDA call.
//
// usage: mesh_check sx sy sz R geometry dir n_faulty id...
// geometry: 0 = unit cube, 1 = sheared cube, 2 = moved sub-cube corners read
// from dir/vpos.bin ((sx+1)(sy+1)(sz+1) x 3 doubles, x fastest).
// dir holds coeff.bin (n_macro doubles), in_<l>.bin (level-l grid vectors) and
// r_<kind>_<l>.bin (fine residual of problem kind on level l); the program
// writes Ag_<l>.bin, rc_<kind>_<l>.bin (pairs grid id, value),
// csr_<kind>.bin (n, then per row: grid id, nnz, (column grid id, value)...)
// and, where the interface stencil tables exist, At_<kind>_<l>.bin (pairs
// grid id, (A in_l) at the problem's free interface nodes through the tables:
// diagonal times the node's value plus the summed weights times the values
// at the tables' block offsets).  Exit code 4: a copy offset differs from
// the one computed from (macro, i, j, k).
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../paper_1506_06185_gb300/csrc/hhg_internal.h"

using namespace hhg;

static std::vector<double> readv(const std::string& fn, size_t n) {
  std::vector<double> v(n);
  FILE* f = fopen(fn.c_str(), "rb");
  if (!f || fread(v.data(), 8, n, f) != n) {
    fprintf(stderr, "cannot read %s\n", fn.c_str());
    exit(2);
  }
  fclose(f);
  return v;
}

static void writev(const std::string& fn, const std::vector<double>& v) {
  FILE* f = fopen(fn.c_str(), "wb");
  fwrite(v.data(), 8, v.size(), f);
  fclose(f);
}

// Global grid id of local node (i, j, k) of macro t at refinement N.
static int64_t gid(const HostMesh& m, int t, int N, int i, int j, int k) {
  const MacroGeo& g = m.geo[t];
  int64_t X[3];
  for (int a = 0; a < 3; ++a)
    X[a] = (int64_t)N * g.v0[a] + (int64_t)i * g.e1[a] + (int64_t)j * g.e2[a] + (int64_t)k * g.e3[a];
  const int64_t nx = (int64_t)m.sub[0] * N, ny = (int64_t)m.sub[1] * N;
  return (X[2] * (ny + 1) + X[1]) * (nx + 1) + X[0];
}

static std::vector<double> to_blocks(const HostMesh& m, const HostLevel& L, const std::vector<double>& g) {
  const int N = L.N;
  std::vector<double> blk((size_t)m.n_macro * L.block, 0.0);
  for (int t = 0; t < m.n_macro; ++t)
    for (int k = 0; k <= N; ++k)
      for (int j = 0; j + k <= N; ++j)
        for (int i = 0; i + j + k <= N; ++i)
          blk[(size_t)t * L.block + lidx(L.SL.data(), N, i, j, k)] = g[gid(m, t, N, i, j, k)];
  return blk;
}

int main(int argc, char** argv) {
  if (argc < 8) return 1;
  const int sub[3] = {atoi(argv[1]), atoi(argv[2]), atoi(argv[3])};
  const int R = atoi(argv[4]);
  const int geometry = atoi(argv[5]);
  const std::string dir = argv[6];
  const int nf = atoi(argv[7]);
  const int n_macro = 6 * sub[0] * sub[1] * sub[2];
  std::vector<unsigned char> faulty(n_macro, 0);
  for (int q = 0; q < nf; ++q) faulty[atoi(argv[8 + q])] = 1;
  const double G[9] = {1.0, 0.3, -0.2, 0.1, 0.9, 0.25, -0.15, 0.2, 1.1};
  const std::vector<double> coeff = readv(dir + "/coeff.bin", n_macro);
  std::vector<double> vpos;
  if (geometry == 2) vpos = readv(dir + "/vpos.bin", (size_t)3 * (sub[0] + 1) * (sub[1] + 1) * (sub[2] + 1));
  HostMesh m;
  build_host_mesh(m, sub, R, 2, coeff.data(), geometry == 1 ? G : nullptr, geometry == 2 ? vpos.data() : nullptr);
  // A g on every level: volume nodes with their macro's interior stencil,
  // interface nodes with the sum of the sub-stencils of their copies
  for (size_t l = 0; l < m.lv.size(); ++l) {
    const HostLevel& L = m.lv[l];
    const int N = L.N;
    const size_t nn = (size_t)(m.sub[0] * N + 1) * (m.sub[1] * N + 1) * (m.sub[2] * N + 1);
    const std::vector<double> g = readv(dir + "/in_" + std::to_string(l) + ".bin", nn);
    const std::vector<double> blk = to_blocks(m, L, g);
    std::vector<double> out(nn, 0.0);
    for (int t = 0; t < m.n_macro; ++t) {
      const double* w = &L.W[(size_t)t * 16 * NDIR];
      for (int k = 1; k <= N; ++k)
        for (int j = 1; j + k <= N - 1; ++j)
          for (int i = 1; i + j + k <= N - 1; ++i) {
            double a = 0.0;
            for (int d = 0; d < NDIR; ++d) {
              int di, dj, dk;
              dir_ijk(d, di, dj, dk);
              a += w[d] * blk[(size_t)t * L.block + lidx(L.SL.data(), N, i + di, j + dj, k + dk)];
            }
            out[gid(m, t, N, i, j, k)] = a;
          }
    }
    for (int n = 0; n < L.n_if; ++n) {
      double a = 0.0;
      for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c) {
        const Copy& cp = L.if_copy[c];
        const double* w = &L.W[((size_t)cp.macro * 16 + node_class(cp.i, cp.j, cp.k, N)) * NDIR];
        for (int d = 0; d < NDIR; ++d) {
          if (w[d] == 0.0) continue;
          int di, dj, dk;
          dir_ijk(d, di, dj, dk);
          if (!in_lattice(cp.i + di, cp.j + dj, cp.k + dk, N)) return 3;   // a weight leaves the lattice
          a += w[d] * blk[(size_t)cp.macro * L.block + lidx(L.SL.data(), N, cp.i + di, cp.j + dj, cp.k + dk)];
        }
      }
      out[L.if_gid[n]] = a;
    }
    writev(dir + "/Ag_" + std::to_string(l) + ".bin", out);
  }
  // per problem kind: restriction gathers onto the free coarse interface
  // nodes, and the compact coarse matrix
  for (int kind = 0; kind < 4; ++kind) {
    if (kind > 0 && nf == 0) break;
    HostProblem p;
    build_problem(m, kind, faulty, p);
    for (size_t l = 0; l + 1 < m.lv.size(); ++l) {
      const HostLevel& C = m.lv[l];
      const HostLevel& F = m.lv[l + 1];
      const int Nf = F.N;
      const size_t nn = (size_t)(m.sub[0] * Nf + 1) * (m.sub[1] * Nf + 1) * (m.sub[2] * Nf + 1);
      const std::vector<double> g =
          readv(dir + "/r_" + std::to_string(kind) + "_" + std::to_string(l + 1) + ".bin", nn);
      const std::vector<double> blk = to_blocks(m, F, g);
      const HostProblemLevel& P = p.lv[l];
      std::vector<double> res;
      for (size_t q = 0; q < P.free_if.size(); ++q) {
        double b = 0.0;
        for (int e = 1; e < NDIR; ++e)
          if (P.gather[q * NDIR + e] >= 0) b += blk[P.gather[q * NDIR + e]];
        res.push_back((double)C.if_gid[P.free_if[q]]);
        res.push_back(blk[P.gather[q * NDIR]] + 0.5 * b);
      }
      writev(dir + "/rc_" + std::to_string(kind) + "_" + std::to_string(l) + ".bin", res);
    }
    const HostLevel& L0 = m.lv[0];
    std::vector<int64_t> dgid(p.n_cg);
    for (int q = 0; q < p.n_cg; ++q) {
      const int64_t s = p.fsrc[q];
      if (s < 0) {
        dgid[q] = L0.if_gid[-1 - s];
        continue;
      }
      const int t = (int)(s / L0.block);
      const int64_t off = s % L0.block;
      for (int k = 1; k <= L0.N; ++k)
        for (int j = 1; j + k <= L0.N - 1; ++j)
          for (int i = 1; i + j + k <= L0.N - 1; ++i)
            if (lidx(L0.SL.data(), L0.N, i, j, k) == off) dgid[q] = gid(m, t, L0.N, i, j, k);
    }
    std::vector<double> dump;
    dump.push_back(p.n_cg);
    for (int q = 0; q < p.n_cg; ++q) {
      dump.push_back((double)dgid[q]);
      dump.push_back(p.rowptr[q + 1] - p.rowptr[q]);
      for (int e = p.rowptr[q]; e < p.rowptr[q + 1]; ++e) {
        dump.push_back((double)dgid[p.col[e]]);
        dump.push_back(p.val[e]);
      }
    }
    writev(dir + "/csr_" + std::to_string(kind) + ".bin", dump);
    // interface stencil tables (levels above the coarsest) applied to in_l
    for (size_t l = 1; l < m.lv.size(); ++l) {
      const HostLevel& L = m.lv[l];
      const HostProblemLevel& P = p.lv[l];
      const std::vector<int>& cptr = kind == 3 ? P.cptr : L.if_cptr;
      const std::vector<Copy>& copies = kind == 3 ? P.copies : L.if_copy;
      std::vector<uint32_t> off;
      if (copy_offsets(m, (int)l, copies, off))
        for (size_t c = 0; c < copies.size(); ++c)
          if (off[c] != (uint32_t)((int64_t)copies[c].macro * L.block +
                                   lidx(L.SL.data(), L.N, copies[c].i, copies[c].j, copies[c].k)))
            return 4;
      const int K = m.seven_point ? 6 : 14;
      std::vector<uint32_t> nb;
      std::vector<double> w, dg;
      if (!build_if_tables(m, (int)l, P.free_if, cptr, copies, K, nb, w, dg)) continue;
      const size_t nn = (size_t)(m.sub[0] * L.N + 1) * (m.sub[1] * L.N + 1) * (m.sub[2] * L.N + 1);
      const std::vector<double> g = readv(dir + "/in_" + std::to_string(l) + ".bin", nn);
      const std::vector<double> blk = to_blocks(m, L, g);
      const size_t n = P.free_if.size();
      std::vector<double> res;
      for (size_t q = 0; q < n; ++q) {
        const int node = P.free_if[q];
        double a = dg[q] * g[L.if_gid[node]];
        for (int e = 0; e < K; ++e) a += w[(size_t)e * n + q] * blk[nb[(size_t)e * n + q]];
        res.push_back((double)L.if_gid[node]);
        res.push_back(a);
      }
      writev(dir + "/At_" + std::to_string(kind) + "_" + std::to_string(l) + ".bin", res);
    }
  }
  return 0;
}
