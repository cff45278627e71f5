// Host-side check of the general-connectivity mesh builder (csrc/mesh.cpp,
// build_general_mesh / build_general_problem), driven by
// tests/test_host_general.py.  Runs on the CPU; makes no CUDA call.
//
// usage: general_check nv nt R dir [n_faulty id...]
// dir holds verts.bin (nv x 3 doubles) and tets.bin (nt x 4 int32), and
// receives per level l: keys_<l>.bin (node keys, 5 int64 per node, in the
// library's node order), g_<l>.bin and Ag_<l>.bin (a test vector and A g
// applied through the macro blocks and copy lists as the kernels do),
// cls_<l>.bin (interface class per interface node, -1 = Dirichlet); and per
// problem kind (0 global; with faulty macros also 1 faulty, 2 healthy with
// the interface frozen, 3 healthy under A_I) and level l below the finest
// r_<kind>_<l+1>.bin and rc_<kind>_<l>.bin (a fine residual, zero off the
// problem's free nodes, and its restriction through the gathers, pairs node
// id / value), and csr_<kind>.bin (the coarse CG matrix: n, then per row id,
// nnz, (column id, value)...).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../paper_1506_06185_gb300/csrc/hhg_internal.h"

using namespace hhg;

template <class T>
static std::vector<T> readv(const std::string& fn, size_t n) {
  std::vector<T> v(n);
  FILE* f = fopen(fn.c_str(), "rb");
  if (!f || fread(v.data(), sizeof(T), n, f) != n) {
    fprintf(stderr, "cannot read %s\n", fn.c_str());
    exit(2);
  }
  fclose(f);
  return v;
}

template <class T>
static void writev(const std::string& fn, const std::vector<T>& v) {
  FILE* f = fopen(fn.c_str(), "wb");
  fwrite(v.data(), sizeof(T), v.size(), f);
  fclose(f);
}

// test values in [-1, 1] from a 64-bit mix of the node id and a salt
static double testval(int64_t id, uint64_t salt) {
  uint64_t z = (uint64_t)id * 0x9e3779b97f4a7c15ull + salt;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (double)(z >> 11) / (double)(1ull << 52) - 1.0;
}

static std::array<int64_t, 5> key_of(const HostMesh& m, int t, int N, int i, int j, int k) {
  const int w[4] = {N - i - j - k, i, j, k};
  int64_t v[4];
  int64_t nz = 0;
  for (int q = 0; q < 4; ++q) {
    v[q] = w[q] > 0 ? (int64_t)m.mverts[t][q] * (N + 1) + w[q] : -1;
    nz += w[q] > 0;
  }
  std::sort(v, v + 4);
  return {nz, v[0], v[1], v[2], v[3]};
}

struct LevelIds {
  std::unordered_map<int64_t, int64_t> slot_id;   // macro * block + slot -> node id (boundary points)
  int64_t n_nodes = 0;
};

static LevelIds level_ids(const HostMesh& m, const HostLevel& L) {
  LevelIds ids;
  for (int n = 0; n < L.n_if; ++n)
    for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c) {
      const Copy& cp = L.if_copy[c];
      ids.slot_id[(int64_t)cp.macro * L.block + lidx(L.SL.data(), L.N, cp.i, cp.j, cp.k)] = L.if_gid[n];
    }
  const int64_t nvol = (int64_t)(L.N - 1) * (L.N - 2) * (L.N - 3) / 6;
  ids.n_nodes = L.n_if + (int64_t)m.n_macro * nvol;
  return ids;
}

static int64_t id_of(const HostMesh& m, const HostLevel& L, const LevelIds& ids, int t, int i, int j, int k) {
  if (node_class(i, j, k, L.N) == 0) return general_volume_id(L, t, i, j, k);
  return ids.slot_id.at((int64_t)t * L.block + lidx(L.SL.data(), L.N, i, j, k));
}

static std::vector<double> to_blocks(const HostMesh& m, const HostLevel& L, const LevelIds& ids,
                                     const std::vector<double>& g) {
  std::vector<double> blk((size_t)m.n_macro * L.block, 0.0);
  const int N = L.N;
  for (int t = 0; t < m.n_macro; ++t)
    for (int k = 0; k <= N; ++k)
      for (int j = 0; j + k <= N; ++j)
        for (int i = 0; i + j + k <= N; ++i)
          blk[(size_t)t * L.block + lidx(L.SL.data(), N, i, j, k)] = g[id_of(m, L, ids, t, i, j, k)];
  return blk;
}

int main(int argc, char** argv) {
  if (argc < 5) return 1;
  const int nv = atoi(argv[1]), nt = atoi(argv[2]), R = atoi(argv[3]);
  const std::string dir = argv[4];
  const std::vector<double> verts = readv<double>(dir + "/verts.bin", 3 * (size_t)nv);
  const std::vector<int> tets = readv<int>(dir + "/tets.bin", 4 * (size_t)nt);
  const std::vector<double> coeff = readv<double>(dir + "/coeff.bin", (size_t)nt);
  std::vector<unsigned char> faulty(nt, 0);
  const int nf = argc > 5 ? atoi(argv[5]) : 0;
  for (int q = 0; q < nf; ++q) faulty[atoi(argv[6 + q])] = 1;
  HostMesh m;
  build_general_mesh(m, verts.data(), nv, tets.data(), nt, R, 2, coeff.data());
  std::vector<LevelIds> all;
  for (size_t l = 0; l < m.lv.size(); ++l) all.push_back(level_ids(m, m.lv[l]));
  for (size_t l = 0; l < m.lv.size(); ++l) {
    const HostLevel& L = m.lv[l];
    const LevelIds& ids = all[l];
    const int N = L.N;
    // keys in node order
    std::vector<int64_t> keys((size_t)ids.n_nodes * 5, 0);
    for (int n = 0; n < L.n_if; ++n) {
      const Copy& cp = L.if_copy[L.if_cptr[n]];
      auto kk = key_of(m, cp.macro, N, cp.i, cp.j, cp.k);
      for (int q = 0; q < 5; ++q) keys[(size_t)L.if_gid[n] * 5 + q] = kk[q];
    }
    for (int t = 0; t < m.n_macro; ++t)
      for (int k = 1; k <= N; ++k)
        for (int j = 1; j + k <= N - 1; ++j)
          for (int i = 1; i + j + k <= N - 1; ++i) {
            auto kk = key_of(m, t, N, i, j, k);
            const int64_t id = general_volume_id(L, t, i, j, k);
            for (int q = 0; q < 5; ++q) keys[(size_t)id * 5 + q] = kk[q];
          }
    writev(dir + "/keys_" + std::to_string(l) + ".bin", keys);
    // A g through blocks and copies
    std::vector<double> g(ids.n_nodes);
    for (int64_t q = 0; q < ids.n_nodes; ++q) g[q] = testval(q, 17 + l);
    const std::vector<double> blk = to_blocks(m, L, ids, g);
    std::vector<double> out(ids.n_nodes, 0.0);
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
            out[general_volume_id(L, t, i, j, k)] = a;
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
          if (!in_lattice(cp.i + di, cp.j + dj, cp.k + dk, N)) return 3;
          a += w[d] * blk[(size_t)cp.macro * L.block + lidx(L.SL.data(), N, cp.i + di, cp.j + dj, cp.k + dk)];
        }
      }
      out[L.if_gid[n]] = a;
    }
    writev(dir + "/g_" + std::to_string(l) + ".bin", g);
    writev(dir + "/Ag_" + std::to_string(l) + ".bin", out);
    std::vector<int> cls(L.n_if);
    for (int n = 0; n < L.n_if; ++n) cls[L.if_gid[n]] = L.if_dirichlet[n] ? -1 : (int)L.if_colour[n];
    writev(dir + "/cls_" + std::to_string(l) + ".bin", cls);
  }
  for (int kind = 0; kind < 4; ++kind) {
    if (kind > 0 && nf == 0) break;
    HostProblem p;
    build_general_problem(m, kind, faulty, p);
    const std::string ks = std::to_string(kind);
    // restriction through the gathers
    for (size_t l = 0; l + 1 < m.lv.size(); ++l) {
      const HostLevel& C = m.lv[l];
      const HostLevel& F = m.lv[l + 1];
      const LevelIds& fids = all[l + 1];
      std::vector<double> r(fids.n_nodes);
      for (int64_t q = 0; q < fids.n_nodes; ++q) r[q] = testval(q, 101 + l + 7 * kind);
      // zero off the free nodes: interface nodes not in the problem's lists,
      // volume nodes of inactive macros
      std::vector<unsigned char> fr(F.n_if, 0);
      for (int n : p.lv[l + 1].free_if) fr[n] = 1;
      for (int n = 0; n < F.n_if; ++n)
        if (!fr[n]) r[F.if_gid[n]] = 0.0;
      const int64_t nvol = (int64_t)(F.N - 1) * (F.N - 2) * (F.N - 3) / 6;
      for (int t = 0; t < m.n_macro; ++t)
        if (!p.macro_active[t])
          for (int64_t q = 0; q < nvol; ++q) r[F.n_if + (int64_t)t * nvol + q] = 0.0;
      writev(dir + "/r_" + ks + "_" + std::to_string(l + 1) + ".bin", r);
      const std::vector<double> blk = to_blocks(m, F, fids, r);
      const HostProblemLevel& P = p.lv[l];
      std::vector<double> res;
      for (size_t q = 0; q < P.free_if.size(); ++q) {
        double b = 0.0;
        for (int e = P.gptr[q] + 1; e < P.gptr[q + 1]; ++e) b += blk[P.goff[e]];
        res.push_back((double)C.if_gid[P.free_if[q]]);
        res.push_back(blk[P.goff[P.gptr[q]]] + 0.5 * b);
      }
      writev(dir + "/rc_" + ks + "_" + std::to_string(l) + ".bin", res);
    }
    // coarse CG matrix with node ids
    const HostLevel& L0 = m.lv[0];
    std::unordered_map<int64_t, int64_t> off_id;
    for (int t = 0; t < m.n_macro; ++t)
      for (int k = 1; k <= L0.N; ++k)
        for (int j = 1; j + k <= L0.N - 1; ++j)
          for (int i = 1; i + j + k <= L0.N - 1; ++i)
            off_id[(int64_t)t * L0.block + lidx(L0.SL.data(), L0.N, i, j, k)] = general_volume_id(L0, t, i, j, k);
    std::vector<int64_t> did(p.n_cg);
    for (int q = 0; q < p.n_cg; ++q) {
      const int64_t sidx = p.fsrc[q];
      did[q] = sidx < 0 ? L0.if_gid[-1 - sidx] : off_id.at(sidx);
    }
    std::vector<double> dump;
    dump.push_back(p.n_cg);
    for (int q = 0; q < p.n_cg; ++q) {
      dump.push_back((double)did[q]);
      dump.push_back(p.rowptr[q + 1] - p.rowptr[q]);
      for (int e = p.rowptr[q]; e < p.rowptr[q + 1]; ++e) {
        dump.push_back((double)did[p.col[e]]);
        dump.push_back(p.val[e]);
      }
    }
    writev(dir + "/csr_" + ks + ".bin", dump);
  }
  return 0;
}
