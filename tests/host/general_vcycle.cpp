// Host model of the device V-cycle on a macro mesh of general connectivity,
// driven by tests/test_host_general.py: the same tables the library uploads
// (build_general_mesh / build_general_problem) and the same per-node
// arithmetic and order as its kernels (volume Gauss-Seidel by local colour,
// then the interface classes; residual written to every copy; restriction
// through the volume stencil and the variable-length interface gathers;
// coarse CG; interpolation along the coarse edge through each fine node),
// executed one node at a time.  Runs on the CPU; makes no CUDA call.
//
// usage: general_vcycle nv nt R cycles dir [fault_cycle recovery n_local n_global n_faulty id... [eta]]
// dir holds verts.bin, tets.bin (int32), coeff.bin, f.bin and u0.bin (global
// vectors in the library's node order); writes u_<c>.bin after every global
// cycle and hist.bin (relative residual after every global cycle and, with a
// fault, one entry right after the fault and its recovery: recovery 1 = LR,
// n_local cycles on the faulty sub-domain; 2 = DD, also n_global cycles on
// the healthy one with the interface frozen; 3 = DN, n_global Neumann-side
// cycles with Omega_F blocks of ceil(j eta) - ceil((j - 1) eta) cycles).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
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

struct Lev {
  std::vector<double> u, f, r, uI, fI;
};

struct Model {
  HostMesh m;
  HostProblem glob, loc, heal, neum;          // global, faulty sub-domain, healthy (interface
                                              // frozen), healthy under A_I (interface free)
  std::vector<Lev> lv;

  size_t at(const HostLevel& L, int t, int i, int j, int k) const {
    return (size_t)t * L.block + lidx(L.SL.data(), L.N, i, j, k);
  }

  // the copy lists a problem works with: its own (the Neumann side keeps
  // only the healthy copies) or the level's
  struct Cps {
    const int* ptr;
    const Copy* cps;
  };
  Cps copies(const HostProblem& p, int l) const {
    const HostProblemLevel& P = p.lv[l];
    if (!P.cptr.empty()) return {P.cptr.data(), P.copies.data()};
    return {m.lv[l].if_cptr.data(), m.lv[l].if_copy.data()};
  }
  Cps all_copies(int l) const { return {m.lv[l].if_cptr.data(), m.lv[l].if_copy.data()}; }

  void write_copies(const HostLevel& L, Cps cl, std::vector<double>& b, int n, double v) const {
    for (int c = cl.ptr[n]; c < cl.ptr[n + 1]; ++c) {
      const Copy& cp = cl.cps[c];
      b[at(L, cp.macro, cp.i, cp.j, cp.k)] = v;
    }
  }
  // sum over the copies of the sub-stencils: off-diagonal part and diagonal
  void if_stencil(const HostLevel& L, Cps cl, const std::vector<double>& u, int n, double& off, double& diag) const {
    off = diag = 0.0;
    for (int c = cl.ptr[n]; c < cl.ptr[n + 1]; ++c) {
      const Copy& cp = cl.cps[c];
      const double* w = &L.W[((size_t)cp.macro * 16 + node_class(cp.i, cp.j, cp.k, L.N)) * NDIR];
      diag += w[0];
      for (int d = 1; d < NDIR; ++d) {
        if (w[d] == 0.0) continue;
        int di, dj, dk;
        dir_ijk(d, di, dj, dk);
        off += w[d] * u[at(L, cp.macro, cp.i + di, cp.j + dj, cp.k + dk)];
      }
    }
  }

  void smooth(const HostProblem& p, int l, int steps, const std::vector<double>& fI) {
    const HostLevel& L = m.lv[l];
    Lev& D = lv[l];
    const HostProblemLevel& P = p.lv[l];
    const Cps cl = copies(p, l);
    const int N = L.N;
    for (int it = 0; it < steps; ++it) {
      for (int c = 0; c < 4; ++c)
        for (int t : p.act) {
          const double* w = &L.W[(size_t)t * 16 * NDIR];
          for (int k = 1; k <= N; ++k)
            for (int j = 1; j + k <= N - 1; ++j)
              for (int i = 1; i + j + k <= N - 1; ++i) {
                if (((i + 2 * j + 3 * k) & 3) != c) continue;
                double acc = D.f[at(L, t, i, j, k)];
                for (int d = 1; d < NDIR; ++d) {
                  int di, dj, dk;
                  dir_ijk(d, di, dj, dk);
                  acc -= w[d] * D.u[at(L, t, i + di, j + dj, k + dk)];
                }
                D.u[at(L, t, i, j, k)] = acc * (1.0 / w[0]);
              }
        }
      for (size_t c = 0; c + 1 < P.class_off.size(); ++c)
        for (int q = P.class_off[c]; q < P.class_off[c + 1]; ++q) {
          const int n = P.free_if[q];
          double off, diag;
          if_stencil(L, cl, D.u, n, off, diag);
          const double v = (fI[n] - off) / diag;
          D.uI[n] = v;
          write_copies(L, cl, D.u, n, v);
        }
    }
  }

  void residual(const HostProblem& p, int l, const std::vector<double>& fI) {
    const HostLevel& L = m.lv[l];
    Lev& D = lv[l];
    const HostProblemLevel& P = p.lv[l];
    const Cps cl = copies(p, l);
    const int N = L.N;
    for (int t : p.act) {
      const double* w = &L.W[(size_t)t * 16 * NDIR];
      for (int k = 1; k <= N; ++k)
        for (int j = 1; j + k <= N - 1; ++j)
          for (int i = 1; i + j + k <= N - 1; ++i) {
            double acc = D.f[at(L, t, i, j, k)];
            for (int d = 0; d < NDIR; ++d) {
              int di, dj, dk;
              dir_ijk(d, di, dj, dk);
              acc -= w[d] * D.u[at(L, t, i + di, j + dj, k + dk)];
            }
            D.r[at(L, t, i, j, k)] = acc;
          }
    }
    for (int n : P.free_if) {
      double off, diag;
      if_stencil(L, cl, D.u, n, off, diag);
      write_copies(L, cl, D.r, n, fI[n] - diag * D.uI[n] - off);
    }
    for (int64_t o : P.zero_off) D.r[o] = 0.0;
  }

  void restrict_to(const HostProblem& p, int l) {   // level l -> l - 1
    const HostLevel& F = m.lv[l];
    const HostLevel& C = m.lv[l - 1];
    Lev& Df = lv[l];
    Lev& Dc = lv[l - 1];
    const HostProblemLevel& P = p.lv[l - 1];
    const int Nc = C.N;
    for (int t : p.act)
      for (int k = 1; k <= Nc; ++k)
        for (int j = 1; j + k <= Nc - 1; ++j)
          for (int i = 1; i + j + k <= Nc - 1; ++i) {
            double acc = 0.0;
            for (int d = 1; d < NDIR; ++d) {
              int di, dj, dk;
              dir_ijk(d, di, dj, dk);
              acc += Df.r[at(F, t, 2 * i + di, 2 * j + dj, 2 * k + dk)];
            }
            Dc.f[at(C, t, i, j, k)] = Df.r[at(F, t, 2 * i, 2 * j, 2 * k)] + 0.5 * acc;
            Dc.u[at(C, t, i, j, k)] = 0.0;
          }
    for (size_t q = 0; q < P.free_if.size(); ++q) {
      const int n = P.free_if[q];
      double acc = 0.0;
      for (int e = P.gptr[q] + 1; e < P.gptr[q + 1]; ++e) acc += Df.r[P.goff[e]];
      Dc.fI[n] = Df.r[P.goff[P.gptr[q]]] + 0.5 * acc;
      Dc.uI[n] = 0.0;
      write_copies(C, copies(p, l - 1), Dc.u, n, 0.0);
    }
    for (int64_t o : P.zero_off) Dc.u[o] = 0.0;
  }

  double interp(const HostLevel& C, const std::vector<double>& uc, int t, int i, int j, int k) const {
    const int pi = i & 1, pj = j & 1, pk = k & 1;
    if (!(pi | pj | pk)) return uc[at(C, t, i >> 1, j >> 1, k >> 1)];
    // the fine node is the midpoint of a coarse edge; in chain coordinates
    // (a, b, c) = (i + j + k, j + k, k) its end points are floor and ceil of half
    const int a = i + j + k, b = j + k, c = k;
    const int la = a >> 1, lb = b >> 1, lc = c >> 1, ha = (a + 1) >> 1, hb = (b + 1) >> 1, hc = (c + 1) >> 1;
    return 0.5 * (uc[at(C, t, la - lb, lb - lc, lc)] + uc[at(C, t, ha - hb, hb - hc, hc)]);
  }

  void prolong(const HostProblem& p, int l) {   // level l - 1 -> l
    const HostLevel& F = m.lv[l];
    const HostLevel& C = m.lv[l - 1];
    Lev& Df = lv[l];
    const Lev& Dc = lv[l - 1];
    const int N = F.N;
    for (int t : p.act)
      for (int k = 1; k <= N; ++k)
        for (int j = 1; j + k <= N - 1; ++j)
          for (int i = 1; i + j + k <= N - 1; ++i) Df.u[at(F, t, i, j, k)] += interp(C, Dc.u, t, i, j, k);
    const Cps cl = copies(p, l);
    for (int n : p.lv[l].free_if) {
      const Copy& cp = cl.cps[cl.ptr[n]];
      const double v = Df.uI[n] + interp(C, Dc.u, cp.macro, cp.i, cp.j, cp.k);
      Df.uI[n] = v;
      write_copies(F, cl, Df.u, n, v);
    }
  }

  void coarse_solve(const HostProblem& p) {
    // CG on the compact free nodes of level 0, from zero, to 1e-12 relative
    Lev& D = lv[0];
    const int n = p.n_cg;
    std::vector<double> b(n), x(n, 0.0), r, pv, Ap(n);
    for (int q = 0; q < n; ++q) {
      const int64_t s = p.fsrc[q];
      b[q] = s < 0 ? D.fI[-1 - s] : D.f[s];
    }
    auto mv = [&](const std::vector<double>& v, std::vector<double>& out) {
      for (int q = 0; q < n; ++q) {
        double a = 0.0;
        for (int e = p.rowptr[q]; e < p.rowptr[q + 1]; ++e) a += p.val[e] * v[p.col[e]];
        out[q] = a;
      }
    };
    r = b;
    pv = r;
    double rr = 0.0;
    for (double v : r) rr += v * v;
    const double stop = 1e-24 * rr;
    for (int it = 0; it < 10 * n + 100 && rr > stop && rr > 0.0; ++it) {
      mv(pv, Ap);
      double pAp = 0.0;
      for (int q = 0; q < n; ++q) pAp += pv[q] * Ap[q];
      const double al = rr / pAp;
      double rn = 0.0;
      for (int q = 0; q < n; ++q) {
        x[q] += al * pv[q];
        r[q] -= al * Ap[q];
        rn += r[q] * r[q];
      }
      for (int q = 0; q < n; ++q) pv[q] = r[q] + (rn / rr) * pv[q];
      rr = rn;
    }
    for (int q = 0; q < n; ++q) {
      for (int e = p.uptr[q]; e < p.uptr[q + 1]; ++e) D.u[p.udst[e]] = x[q];
      if (p.umaster[q] >= 0) D.uI[p.umaster[q]] = x[q];
    }
  }

  // fI_top: the interface right-hand side of the finest level (the Neumann
  // side's, with the flux on Gamma), else the level's own
  void vcycle(const HostProblem& p, const std::vector<double>* fI_top = nullptr) {
    const int top = (int)m.lv.size() - 1;
    auto fI = [&](int l) -> const std::vector<double>& { return l == top && fI_top ? *fI_top : lv[l].fI; };
    for (int l = top; l >= 1; --l) {
      smooth(p, l, 3, fI(l));
      residual(p, l, fI(l));
      restrict_to(p, l);
    }
    coarse_solve(p);
    for (int l = 1; l <= top; ++l) {
      prolong(p, l);
      smooth(p, l, 3, fI(l));
    }
  }

  // ||f - A u|| over the free nodes of the global problem (finest level)
  double resnorm() {
    const int top = (int)m.lv.size() - 1;
    residual(glob, top, lv[top].fI);
    const HostLevel& L = m.lv[top];
    const Lev& D = lv[top];
    double ss = 0.0;
    for (int t = 0; t < m.n_macro; ++t)
      for (int k = 1; k <= L.N; ++k)
        for (int j = 1; j + k <= L.N - 1; ++j)
          for (int i = 1; i + j + k <= L.N - 1; ++i) ss += D.r[at(L, t, i, j, k)] * D.r[at(L, t, i, j, k)];
    for (int n : glob.lv[top].free_if) {
      const Copy& cp = L.if_copy[L.if_cptr[n]];
      const double v = D.r[at(L, cp.macro, cp.i, cp.j, cp.k)];
      ss += v * v;
    }
    return std::sqrt(ss);
  }

  // Dirichlet-Neumann recovery as the device schedules it (Algorithm 2): the
  // Neumann side's interface right-hand side takes the flux (A_I u) on Gamma
  // (the interface nodes free on the Neumann side with a faulty copy); block j
  // of ceil(j eta) - ceil((j - 1) eta) Omega_F cycles starts from the Gamma
  // values after Omega_I cycle j - 1 (copied into the faulty blocks), Omega_I
  // cycle j follows (the two touch disjoint data, so the device runs them
  // concurrently); at the end the faulty blocks take the final Gamma values.
  void recover_dn(const std::vector<unsigned char>& faulty, int n_global, double eta) {
    const int top = (int)m.lv.size() - 1;
    const HostLevel& L = m.lv[top];
    Lev& D = lv[top];
    const Cps cn = copies(neum, top);
    std::vector<int> gamma;
    for (int n : neum.lv[top].free_if) {
      bool any_f = false;
      for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c) any_f = any_f || faulty[L.if_copy[c].macro];
      if (any_f) gamma.push_back(n);
    }
    std::vector<double> fI_dn = D.fI;
    for (int n : gamma) {
      double off, diag;
      if_stencil(L, cn, D.u, n, off, diag);
      fI_dn[n] = diag * D.uI[n] + off;
    }
    auto to_faulty_blocks = [&](const std::vector<double>& val) {
      for (size_t q = 0; q < gamma.size(); ++q)
        for (int c = L.if_cptr[gamma[q]]; c < L.if_cptr[gamma[q] + 1]; ++c) {
          const Copy& cp = L.if_copy[c];
          if (faulty[cp.macro]) D.u[at(L, cp.macro, cp.i, cp.j, cp.k)] = val[q];
        }
    };
    std::vector<double> snap(gamma.size());
    for (size_t q = 0; q < gamma.size(); ++q) snap[q] = D.uI[gamma[q]];
    for (int j = 1; j <= n_global; ++j) {
      const int cyc = (int)std::ceil(j * eta) - (int)std::ceil((j - 1) * eta);
      if (j >= 2) to_faulty_blocks(snap);
      for (int c = 0; c < cyc; ++c) vcycle(loc);
      vcycle(neum, &fI_dn);
      for (size_t q = 0; q < gamma.size(); ++q) snap[q] = D.uI[gamma[q]];
    }
    to_faulty_blocks(snap);
  }

  // fault (§2.2): the faulty blocks lose everything, the masters inside
  // Omega_F are erased, the copies in the lost blocks come back from masters
  void inject(const std::vector<unsigned char>& faulty) {
    const int top = (int)m.lv.size() - 1;
    const HostLevel& L = m.lv[top];
    Lev& D = lv[top];
    for (int t = 0; t < m.n_macro; ++t)
      if (faulty[t]) std::fill(D.u.begin() + (size_t)t * L.block, D.u.begin() + (size_t)(t + 1) * L.block, 0.0);
    for (int n : loc.lv[top].free_if) D.uI[n] = 0.0;
    for (int n = 0; n < L.n_if; ++n)
      for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c)
        if (faulty[L.if_copy[c].macro]) {
          const Copy& cp = L.if_copy[c];
          D.u[at(L, cp.macro, cp.i, cp.j, cp.k)] = D.uI[n];
        }
  }
};

int main(int argc, char** argv) {
  if (argc < 6) return 1;
  const int nv = atoi(argv[1]), nt = atoi(argv[2]), R = atoi(argv[3]), cycles = atoi(argv[4]);
  const std::string dir = argv[5];
  const auto verts = readv<double>(dir + "/verts.bin", 3 * (size_t)nv);
  const auto tets = readv<int>(dir + "/tets.bin", 4 * (size_t)nt);
  const auto coeff = readv<double>(dir + "/coeff.bin", (size_t)nt);
  Model M;
  build_general_mesh(M.m, verts.data(), nv, tets.data(), nt, R, 2, coeff.data());
  std::vector<unsigned char> faulty(nt, 0);
  const int fault_cycle = argc > 6 ? atoi(argv[6]) : -1;
  const int recovery = argc > 7 ? atoi(argv[7]) : 0;
  const int n_local = argc > 8 ? atoi(argv[8]) : 0;
  const int n_global = argc > 9 ? atoi(argv[9]) : 0;
  const int nf = argc > 10 ? atoi(argv[10]) : 0;
  for (int q = 0; q < nf; ++q) faulty[atoi(argv[11 + q])] = 1;
  build_general_problem(M.m, 0, std::vector<unsigned char>(nt, 0), M.glob);
  if (nf > 0) {
    build_general_problem(M.m, 1, faulty, M.loc);
    build_general_problem(M.m, 2, faulty, M.heal);
    build_general_problem(M.m, 3, faulty, M.neum);
  }
  const double eta = argc > 11 + nf ? atof(argv[11 + nf]) : 1.0;
  M.lv.resize(M.m.lv.size());
  for (size_t l = 0; l < M.m.lv.size(); ++l) {
    const HostLevel& L = M.m.lv[l];
    const size_t nb = (size_t)nt * L.block;
    M.lv[l].u.assign(nb, 0.0);
    M.lv[l].f.assign(nb, 0.0);
    M.lv[l].r.assign(nb, 0.0);
    M.lv[l].uI.assign(std::max(1, L.n_if), 0.0);
    M.lv[l].fI.assign(std::max(1, L.n_if), 0.0);
  }
  // import f and u0 at the finest level (volume nodes, masters, copies)
  const HostLevel& T = M.m.lv.back();
  const int N = T.N;
  const int64_t nvol = (int64_t)(N - 1) * (N - 2) * (N - 3) / 6;
  const int64_t nn = T.n_if + (int64_t)nt * nvol;
  const auto f = readv<double>(dir + "/f.bin", (size_t)nn);
  const auto u0 = readv<double>(dir + "/u0.bin", (size_t)nn);
  Lev& D = M.lv.back();
  for (int t = 0; t < nt; ++t)
    for (int k = 1; k <= N; ++k)
      for (int j = 1; j + k <= N - 1; ++j)
        for (int i = 1; i + j + k <= N - 1; ++i) {
          const int64_t id = general_volume_id(T, t, i, j, k);
          D.f[M.at(T, t, i, j, k)] = f[id];
          D.u[M.at(T, t, i, j, k)] = u0[id];
        }
  for (int n = 0; n < T.n_if; ++n) {
    D.fI[n] = f[T.if_gid[n]];
    D.uI[n] = u0[T.if_gid[n]];
    M.write_copies(T, M.all_copies((int)M.m.lv.size() - 1), D.u, n, D.uI[n]);
  }
  std::vector<double> hist = {1.0};
  const double r0 = M.resnorm();
  for (int c = 0; c < cycles; ++c) {
    M.vcycle(M.glob);
    hist.push_back(M.resnorm() / r0);
    if (c + 1 == fault_cycle) {
      M.inject(faulty);
      if (recovery == 1 || recovery == 2)
        for (int q = 0; q < n_local; ++q) M.vcycle(M.loc);
      if (recovery == 2)
        for (int q = 0; q < n_global; ++q) M.vcycle(M.heal);
      if (recovery == 3) M.recover_dn(faulty, n_global, eta);
      hist.push_back(M.resnorm() / r0);
    }
    std::vector<double> out(nn);
    for (int t = 0; t < nt; ++t)
      for (int k = 1; k <= N; ++k)
        for (int j = 1; j + k <= N - 1; ++j)
          for (int i = 1; i + j + k <= N - 1; ++i) out[general_volume_id(T, t, i, j, k)] = D.u[M.at(T, t, i, j, k)];
    for (int n = 0; n < T.n_if; ++n) out[T.if_gid[n]] = D.uI[n];
    FILE* fo = fopen((dir + "/u_" + std::to_string(c) + ".bin").c_str(), "wb");
    fwrite(out.data(), 8, out.size(), fo);
    fclose(fo);
  }
  FILE* fh = fopen((dir + "/hist.bin").c_str(), "wb");
  fwrite(hist.data(), 8, hist.size(), fh);
  fclose(fh);
  return 0;
}
