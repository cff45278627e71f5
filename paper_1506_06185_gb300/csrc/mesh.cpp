// Host-side construction of the macro mesh, its refinement levels, the
// per-macro stencils and the interface containers (§2.1 base mesh and
// uniform refinement; §3.1 volume / face / edge / vertex containers; §3.2 and
// Fig. 4: a node on a macro face, edge or vertex gets its stencil as the sum
// of the sub-stencils of the macros around it).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <stdexcept>
#include <unordered_map>

#include "hhg_internal.h"

namespace hhg {

namespace {

const int PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

struct Prim {
  int type = 0;                         // 0 vertex, 1 edge, 2 face
  std::vector<int> gv;                  // sorted global vertex ids
  std::vector<std::array<int, 3>> X;    // their integer sub-cube coordinates
  std::vector<std::pair<int, std::array<int, 3>>> adj;  // (macro, local vertex of gv[t])
  bool boundary = false;
};

// Key of a lattice node of a general mesh, the same from every macro that
// contains it: the number of positive barycentric weights, then the values
// vertex id * (N + 1) + weight of the positive weights in ascending order,
// -1 padding first.  Sorting nodes by key orders them by primitive dimension
// (vertex, edge, face, volume) and then by their vertices and weights.
using NodeKey = std::array<int64_t, 5>;

struct KeyHash {
  size_t operator()(const NodeKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int64_t x : k) {
      h ^= (uint64_t)x;
      h *= 1099511628211ull;
    }
    return (size_t)h;
  }
};

NodeKey node_key(const HostMesh& m, int macro, int N, int i, int j, int k) {
  const int w[4] = {N - i - j - k, i, j, k};
  int64_t v[4];
  int64_t nz = 0;
  for (int q = 0; q < 4; ++q) {
    v[q] = w[q] > 0 ? (int64_t)m.mverts[macro][q] * (N + 1) + w[q] : -1;
    nz += w[q] > 0;
  }
  std::sort(v, v + 4);
  return NodeKey{nz, v[0], v[1], v[2], v[3]};
}

int64_t grid_gid(const HostMesh& m, int N, int64_t x, int64_t y, int64_t z) {
  int64_t nx = (int64_t)m.sub[0] * N, ny = (int64_t)m.sub[1] * N;
  return (z * (ny + 1) + y) * (nx + 1) + x;
}

void local_to_fine(const MacroGeo& g, int N, int i, int j, int k, int64_t X[3]) {
  for (int a = 0; a < 3; ++a)
    X[a] = (int64_t)N * g.v0[a] + (int64_t)i * g.e1[a] + (int64_t)j * g.e2[a] + (int64_t)k * g.e3[a];
}

int64_t node_gid(const HostMesh& m, int macro, int N, int i, int j, int k) {
  int64_t X[3];
  local_to_fine(m.geo[macro], N, i, j, k, X);
  return grid_gid(m, N, X[0], X[1], X[2]);
}

// Physical position of the sub-cube corner c (integer corner coordinates).
const double* corner_pos(const HostMesh& m, const int c[3]) {
  return &m.vpos[(((size_t)c[2] * (m.sub[1] + 1) + c[1]) * (m.sub[0] + 1) + c[0]) * 3];
}

// Physical position of a local lattice node of a macro at refinement N: the
// macro's corners P0..P3 (moved corners), P0 + (i (P1-P0) + j (P2-P0) +
// k (P3-P0)) / N; else the unit-cube grid position mapped by G.
void position(const HostMesh& m, int macro, int N, int i, int j, int k, double out[3]) {
  if (!m.mverts.empty()) {
    const double* P[4];
    for (int q = 0; q < 4; ++q) P[q] = &m.vpos[3 * (size_t)m.mverts[macro][q]];
    for (int a = 0; a < 3; ++a)
      out[a] = P[0][a] + (i * (P[1][a] - P[0][a]) + j * (P[2][a] - P[0][a]) + k * (P[3][a] - P[0][a])) / N;
    return;
  }
  if (!m.vpos.empty()) {
    const MacroGeo& g = m.geo[macro];
    int c[4][3];
    for (int a = 0; a < 3; ++a) {
      c[0][a] = g.v0[a];
      c[1][a] = g.v0[a] + g.e1[a];
      c[2][a] = g.v0[a] + g.e2[a];
      c[3][a] = g.v0[a] + g.e3[a];
    }
    const double* P0 = corner_pos(m, c[0]);
    const double* P1 = corner_pos(m, c[1]);
    const double* P2 = corner_pos(m, c[2]);
    const double* P3 = corner_pos(m, c[3]);
    for (int a = 0; a < 3; ++a)
      out[a] = P0[a] + (i * (P1[a] - P0[a]) + j * (P2[a] - P0[a]) + k * (P3[a] - P0[a])) / N;
    return;
  }
  int64_t X[3];
  local_to_fine(m.geo[macro], N, i, j, k, X);
  double p[3] = {double(X[0]) / (double(m.sub[0]) * N), double(X[1]) / (double(m.sub[1]) * N),
                 double(X[2]) / (double(m.sub[2]) * N)};
  for (int a = 0; a < 3; ++a) out[a] = m.G[3 * a] * p[0] + m.G[3 * a + 1] * p[1] + m.G[3 * a + 2] * p[2];
}

// P1 stiffness of one tetrahedron with unit coefficient: gradients of the
// barycentric coordinates from the inverse edge matrix, times the volume.
void tet_stiffness(const double X[4][3], double K[4][4]) {
  double E[3][3];
  for (int q = 0; q < 3; ++q)
    for (int a = 0; a < 3; ++a) E[a][q] = X[q + 1][a] - X[0][a];
  double det = E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) -
               E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
               E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
  double inv[3][3];
  inv[0][0] = (E[1][1] * E[2][2] - E[1][2] * E[2][1]) / det;
  inv[0][1] = (E[0][2] * E[2][1] - E[0][1] * E[2][2]) / det;
  inv[0][2] = (E[0][1] * E[1][2] - E[0][2] * E[1][1]) / det;
  inv[1][0] = (E[1][2] * E[2][0] - E[1][0] * E[2][2]) / det;
  inv[1][1] = (E[0][0] * E[2][2] - E[0][2] * E[2][0]) / det;
  inv[1][2] = (E[0][2] * E[1][0] - E[0][0] * E[1][2]) / det;
  inv[2][0] = (E[1][0] * E[2][1] - E[1][1] * E[2][0]) / det;
  inv[2][1] = (E[0][1] * E[2][0] - E[0][0] * E[2][1]) / det;
  inv[2][2] = (E[0][0] * E[1][1] - E[0][1] * E[1][0]) / det;
  double D[4][3];
  for (int a = 0; a < 3; ++a) {
    D[1][a] = inv[0][a];
    D[2][a] = inv[1][a];
    D[3][a] = inv[2][a];
    D[0][a] = -(inv[0][a] + inv[1][a] + inv[2][a]);
  }
  double vol = std::fabs(det) / 6.0;
  for (int p = 0; p < 4; ++p)
    for (int q = 0; q < 4; ++q) K[p][q] = vol * (D[p][0] * D[q][0] + D[p][1] * D[q][1] + D[p][2] * D[q][2]);
}

int dir_index(int di, int dj, int dk) {
  for (int d = 0; d < NDIR; ++d) {
    int a, b, c;
    dir_ijk(d, a, b, c);
    if (a == di && b == dj && c == dk) return d;
  }
  return -1;
}

// Representative local node of a node class at refinement N (N >= 4).
bool class_representative(int mask, int N, int& i, int& j, int& k) {
  bool k0 = mask & 1, j0 = mask & 2, i0 = mask & 4, top = mask & 8;
  if (mask == 15) return false;
  i = i0 ? 0 : 1;
  j = j0 ? 0 : 1;
  k = k0 ? 0 : 1;
  if (top) {
    if (!i0) i = N - j - k;
    else if (!j0) j = N - k;
    else if (!k0) k = N;
    else return false;
  }
  if (!in_lattice(i, j, k, N) || node_class(i, j, k, N) != mask) return false;
  return true;
}

// Sub-stencil of macro `macro` at a node of class `mask`: the sum over the
// fine tetrahedra of the macro that contain the node (Kuhn simplices of the
// chain lattice inside N >= a >= b >= c >= 0) of their element stiffness row.
void class_weights(const HostMesh& m, int macro, int N, int mask, double w[NDIR]) {
  for (int d = 0; d < NDIR; ++d) w[d] = 0.0;
  int i, j, k;
  if (!class_representative(mask, N, i, j, k)) return;
  const int pa = i + j + k, pb = j + k, pc = k;
  const double kT = m.coeff[macro];
  for (int o = 0; o < 8; ++o) {
    const int oa = o & 1, ob = (o >> 1) & 1, oc = (o >> 2) & 1;
    const int ca = pa - oa, cb = pb - ob, cc = pc - oc;
    for (int s = 0; s < 6; ++s) {
      int V[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 1}};
      V[1][PERM[s][0]] = 1;
      V[2][PERM[s][0]] = 1;
      V[2][PERM[s][1]] = 1;
      int self = -1;
      for (int q = 0; q < 4; ++q)
        if (V[q][0] == oa && V[q][1] == ob && V[q][2] == oc) self = q;
      if (self < 0) continue;
      bool inside = true;
      double X[4][3];
      int L[4][3];
      for (int q = 0; q < 4; ++q) {
        int a = ca + V[q][0], b = cb + V[q][1], c = cc + V[q][2];
        if (!(N >= a && a >= b && b >= c && c >= 0)) { inside = false; break; }
        L[q][0] = a - b;
        L[q][1] = b - c;
        L[q][2] = c;
        position(m, macro, N, L[q][0], L[q][1], L[q][2], X[q]);
      }
      if (!inside) continue;
      double K[4][4];
      tet_stiffness(X, K);
      for (int q = 0; q < 4; ++q) {
        int d = dir_index(L[q][0] - i, L[q][1] - j, L[q][2] - k);
        if (d < 0) throw std::runtime_error("stencil direction outside the 15-point set");
        w[d] += kT * K[self][q];
      }
    }
  }
}

void compute_level_weights(const HostMesh& m, HostLevel& L) {
  L.W.assign((size_t)m.n_macro * 16 * NDIR, 0.0);
  for (int t = 0; t < m.n_macro; ++t)
    for (int mask = 0; mask < 15; ++mask) class_weights(m, t, L.N, mask, &L.W[((size_t)t * 16 + mask) * NDIR]);
}

void build_tiles(int N, bool interior, std::vector<Tile>& out) {
  out.clear();
  const int lo = interior ? 1 : 0;
  const int top = interior ? N - 1 : N;     // i + j + k <= top
  for (int k = lo; k <= top; ++k) {
    int jmax = top - k - lo;                // need i >= lo
    for (int j0 = lo; j0 <= jmax; j0 += TILE_ROWS) {
      int imax = top - j0 - k;
      int mmax = imax >> 2;
      for (int m0 = 0; m0 <= mmax; m0 += TILE_SLOTS) out.push_back(Tile{k, j0, m0, 0});
    }
  }
}

}  // namespace

// Row-pair tiles of the volume interior: in slice k the interior rows are
// j = 1..J, J = N - 2 - k; pair p joins rows 1 + p and J - p, whose lengths add
// up to N - 1 - k nodes.  A tile covers pairs j0 .. j0 + m0 - 1 (about
// `target` nodes of one colour in its first slice, at most 32 pairs) in the
// `slabs` consecutive slices k .. k + pad - 1, so that the CTA that loads a
// slice's rows reuses them for the next slice (pairs beyond a slice's count
// are empty).
// Renumber the interface nodes of a level colour by colour and, within a
// colour, by the block offset of a "home" copy: the first copy that lies in
// the plane j = 0 or k = 0 of its macro (whose rows are contiguous in the
// block; the planes i = 0 and i + j + k = N cut across the rows), else the
// first copy.  The home copy is moved to the front of the node's copy list,
// so the interface stencil tables read shared neighbours from the home block.
// A colour's Gauss-Seidel launch then touches the masters, loads and copy
// pointers of consecutive node ids, and on a face lying in a contiguous plane
// the neighbour gathers and the home copy's write of consecutive nodes land
// on consecutive slots.
static void number_if_by_colour(HostLevel& L) {
  const int n_if = L.n_if;
  std::vector<int> home(n_if);
  std::vector<int64_t> home_off(n_if);
  for (int n = 0; n < n_if; ++n) {
    int h = L.if_cptr[n];
    for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c)
      if (L.if_copy[c].j == 0 || L.if_copy[c].k == 0) {
        h = c;
        break;
      }
    home[n] = h;
    const Copy& cp = L.if_copy[h];
    home_off[n] = (int64_t)cp.macro * L.block + lidx(L.SL.data(), L.N, cp.i, cp.j, cp.k);
  }
  std::vector<int> order(n_if);
  for (int n = 0; n < n_if; ++n) order[n] = n;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (L.if_colour[a] != L.if_colour[b]) return L.if_colour[a] < L.if_colour[b];
    return home_off[a] < home_off[b];
  });
  std::vector<int64_t> gid(n_if);
  std::vector<unsigned char> col(n_if), dir(n_if);
  std::vector<int> cptr(1, 0);
  std::vector<Copy> copies;
  copies.reserve(L.if_copy.size());
  for (int n = 0; n < n_if; ++n) {
    const int o = order[n];
    gid[n] = L.if_gid[o];
    col[n] = L.if_colour[o];
    dir[n] = L.if_dirichlet[o];
    copies.push_back(L.if_copy[home[o]]);
    for (int c = L.if_cptr[o]; c < L.if_cptr[o + 1]; ++c)
      if (c != home[o]) copies.push_back(L.if_copy[c]);
    cptr.push_back((int)copies.size());
  }
  L.if_gid.swap(gid);
  L.if_colour.swap(col);
  L.if_dirichlet.swap(dir);
  L.if_cptr.swap(cptr);
  L.if_copy.swap(copies);
}

void build_pair_tiles(int N, std::vector<Tile>& out, int target, int slabs) {
  out.clear();
  for (int k0 = 1; k0 <= N - 3; k0 += slabs) {
    const int nk = std::min(slabs, N - 2 - k0);
    const int J = N - 2 - k0;
    const int pairs = (J + 1) / 2;
    const int per_pair = std::max(1, (N - 1 - k0) / 4);
    const int np = std::min(32, std::max(1, (target + per_pair - 1) / per_pair));
    for (int p0 = 0; p0 < pairs; p0 += np) out.push_back(Tile{k0, p0, std::min(np, pairs - p0), nk});
  }
  // largest tiles first (interior nodes of the tile's pairs in its slices)
  auto work = [N](const Tile& t) {
    int64_t w = 0;
    for (int k = t.k; k < t.k + t.pad; ++k)
      for (int q = 0; q < t.m0; ++q) {
        const int j1 = 1 + t.j0 + q, j2 = N - 2 - k - t.j0 - q;
        if (j1 < j2) w += N - 1 - k;
        else if (j1 == j2) w += N - 1 - j1 - k;
      }
    return w;
  };
  std::stable_sort(out.begin(), out.end(), [&](const Tile& a, const Tile& b) { return work(a) > work(b); });
}

void build_gs_items(int N, int vw, std::vector<uint32_t>& items, int off[5]) {
  items.clear();
  for (int c = 0; c < 4; ++c) {
    off[c] = (int)items.size();
    for (int k = 1; k <= N - 3; ++k)
      for (int j = 1; j <= N - 2 - k; ++j) {
        // colour-c nodes of the row: i = 4 m + ic for slots m = mlo .. mlo + n - 1
        const int ic = (c - 2 * j - 3 * k) & 3;
        const int L = N - 1 - j - k;
        const int mlo = ic == 0;
        const int n = L >= ic ? ((L - ic) >> 2) - mlo + 1 : 0;
        const int groups = n > 0 ? (mlo + n - 1) / vw + 1 : 0;
        for (int g = 0; g < groups; ++g) items.push_back(((uint32_t)j << 20) | ((uint32_t)k << 10) | (uint32_t)g);
      }
  }
  off[4] = (int)items.size();
}

void build_slot_items(int N, std::vector<uint32_t>& items) {
  items.clear();
  for (int k = 1; k <= N - 3; ++k)
    for (int j = 1; j <= N - 2 - k; ++j)
      for (int m = 0; m <= (N - 1 - j - k) >> 2; ++m)
        items.push_back(((uint32_t)j << 20) | ((uint32_t)k << 10) | (uint32_t)m);
}

void build_stream_tiles(int N, int band, int slices, std::vector<StreamTile>& out) {
  out.clear();
  // interior rows j = 1..N-2-k of slice k = 1..N-3; band [j0, j1] has
  // interior rows in slices k <= N - 2 - j0
  for (int j0 = 1; j0 <= N - 3; j0 += band) {
    const int j1 = std::min(j0 + band - 1, N - 3);
    for (int ka = 1; ka <= N - 2 - j0; ka += slices)
      out.push_back(StreamTile{j0, j1, ka, std::min(ka + slices - 1, N - 2 - j0)});
  }
  auto work = [N](const StreamTile& t) {
    int64_t w = 0;
    for (int k = t.ka; k <= t.kb; ++k)
      for (int j = t.j0; j <= std::min(t.j1, N - 2 - k); ++j) w += N - 1 - j - k;
    return w;
  };
  std::stable_sort(out.begin(), out.end(),
                   [&](const StreamTile& a, const StreamTile& b) { return work(a) > work(b); });
}

void set_coefficients(HostMesh& m, const double* coeff) {
  for (int t = 0; t < m.n_macro; ++t) m.coeff[t] = coeff[t];
  for (auto& L : m.lv) compute_level_weights(m, L);
}

bool macro_in_set(const std::vector<unsigned char>& s, int m) { return m >= 0 && m < (int)s.size() && s[m]; }

void build_host_mesh(HostMesh& m, const int sub[3], int R, int r0, const double* coeff,
                     const double* affine, const double* vertex_pos) {
  for (int a = 0; a < 3; ++a) m.sub[a] = sub[a];
  m.R = R;
  m.r0 = r0;
  m.n_macro = 6 * sub[0] * sub[1] * sub[2];
  const int N_f = 1 << R;
  m.nx = (int64_t)sub[0] * N_f;
  m.ny = (int64_t)sub[1] * N_f;
  m.nz = (int64_t)sub[2] * N_f;
  for (int a = 0; a < 9; ++a) m.G[a] = affine ? affine[a] : (a % 4 == 0 ? 1.0 : 0.0);
  m.coeff.assign(m.n_macro, 1.0);
  if (coeff)
    for (int t = 0; t < m.n_macro; ++t) m.coeff[t] = coeff[t];

  // macro-tetrahedra: sub-cube (a, b, c), x fastest, six Kuhn types each
  m.geo.resize(m.n_macro);
  std::vector<std::array<std::array<int, 3>, 4>> V(m.n_macro);
  for (int c = 0; c < sub[2]; ++c)
    for (int b = 0; b < sub[1]; ++b)
      for (int a = 0; a < sub[0]; ++a)
        for (int p = 0; p < 6; ++p) {
          int t = ((c * sub[1] + b) * sub[0] + a) * 6 + p;
          std::array<int, 3> v0 = {a, b, c}, v1 = v0, v2, v3 = {a + 1, b + 1, c + 1};
          v1[PERM[p][0]] += 1;
          v2 = v1;
          v2[PERM[p][1]] += 1;
          V[t] = {v0, v1, v2, v3};
          for (int q = 0; q < 3; ++q) {
            m.geo[t].v0[q] = v0[q];
            m.geo[t].e1[q] = v1[q] - v0[q];
            m.geo[t].e2[q] = v2[q] - v0[q];
            m.geo[t].e3[q] = v3[q] - v0[q];
          }
        }
  auto vid = [&](const std::array<int, 3>& x) { return (x[2] * (sub[1] + 1) + x[1]) * (sub[0] + 1) + x[0]; };

  // moved corners: every macro must keep the orientation of its Kuhn simplex
  // and a volume bounded away from zero
  m.vpos.clear();
  if (vertex_pos) {
    const size_t nv = (size_t)(sub[0] + 1) * (sub[1] + 1) * (sub[2] + 1);
    m.vpos.assign(vertex_pos, vertex_pos + 3 * nv);
    for (double x : m.vpos)
      if (!std::isfinite(x)) throw std::invalid_argument("vertex positions must be finite");
    for (int t = 0; t < m.n_macro; ++t) {
      double E[3][3], R3[3][3];
      for (int q = 0; q < 3; ++q) {
        const double* P = &m.vpos[3 * (size_t)vid(V[t][q + 1])];
        const double* P0 = &m.vpos[3 * (size_t)vid(V[t][0])];
        for (int a = 0; a < 3; ++a) {
          E[a][q] = P[a] - P0[a];
          R3[a][q] = (double)(V[t][q + 1][a] - V[t][0][a]) / sub[a];
        }
      }
      auto det3 = [](const double A[3][3]) {
        return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
               A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
      };
      const double d = det3(E), ref = det3(R3);
      if (!(d * ref > 0.0) || std::fabs(d) < 1e-6 * std::fabs(ref))
        throw std::invalid_argument("macro " + std::to_string(t) + " is inverted or degenerate");
    }
  }

  // interface primitives (faces, edges, vertices) with their adjacent macros
  std::map<std::vector<int>, int> key;
  std::vector<Prim> prims;
  auto add = [&](int t, const std::vector<int>& loc) {
    std::vector<std::pair<int, int>> gl;
    for (int l : loc) gl.push_back({vid(V[t][l]), l});
    std::sort(gl.begin(), gl.end());
    std::vector<int> g;
    for (auto& x : gl) g.push_back(x.first);
    auto it = key.find(g);
    int id;
    if (it == key.end()) {
      id = (int)prims.size();
      key[g] = id;
      Prim pr;
      pr.type = (int)loc.size() - 1;
      pr.gv = g;
      for (auto& x : gl) pr.X.push_back(V[t][x.second]);
      prims.push_back(pr);
    } else {
      id = it->second;
    }
    std::array<int, 3> lv = {-1, -1, -1};
    for (size_t q = 0; q < gl.size(); ++q) lv[q] = gl[q].second;
    prims[id].adj.push_back({t, lv});
  };
  for (int t = 0; t < m.n_macro; ++t) {
    for (int q = 0; q < 4; ++q) add(t, {q});
    for (int q = 0; q < 4; ++q)
      for (int s = q + 1; s < 4; ++s) add(t, {q, s});
    for (int o = 0; o < 4; ++o) {
      std::vector<int> loc;
      for (int q = 0; q < 4; ++q)
        if (q != o) loc.push_back(q);
      add(t, loc);
    }
  }
  for (auto& pr : prims) {
    for (int a = 0; a < 3 && !pr.boundary; ++a)
      for (int side : {0, sub[a]}) {
        bool all = true;
        for (auto& x : pr.X) all = all && (x[a] == side);
        if (all) pr.boundary = true;
      }
  }
  std::vector<int> order(prims.size());
  for (size_t q = 0; q < prims.size(); ++q) order[q] = (int)q;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return prims[a].type < prims[b].type; });

  m.lv.clear();
  m.seven_point = true;
  for (int r = r0; r <= R; ++r) {
    HostLevel L;
    L.r = r;
    L.N = 1 << r;
    L.block = build_slice_starts(L.N, L.SL);
    const int N = L.N;
    // stencils
    compute_level_weights(m, L);
    // 7-point structure: every class (volume and sub-stencils) of every macro
    // has zero weights off the three chain axes
    for (size_t q = 0; q < L.W.size(); ++q) {
      const int d = (int)(q % NDIR);
      const int dd = d > 7 ? d - 7 : d;
      if (dd > 3 && L.W[q] != 0.0) m.seven_point = false;
    }
    // interface nodes: vertices, edges, faces
    L.if_cptr.push_back(0);
    for (int id : order) {
      const Prim& pr = prims[id];
      const int nv = (int)pr.gv.size();
      std::vector<std::array<int, 3>> alphas;
      if (nv == 1) alphas.push_back({N, 0, 0});
      if (nv == 2)
        for (int a = 1; a <= N - 1; ++a) alphas.push_back({a, N - a, 0});
      if (nv == 3)
        for (int a = 1; a <= N - 2; ++a)
          for (int b = 1; a + b <= N - 1; ++b) alphas.push_back({a, b, N - a - b});
      for (auto& al : alphas) {
        int64_t X[3] = {0, 0, 0};
        for (int q = 0; q < nv; ++q)
          for (int a = 0; a < 3; ++a) X[a] += (int64_t)al[q] * pr.X[q][a];
        L.if_gid.push_back(grid_gid(m, N, X[0], X[1], X[2]));
        L.if_colour.push_back((unsigned char)((X[0] + X[1] + X[2]) & 3));
        L.if_dirichlet.push_back(pr.boundary ? 1 : 0);
        for (auto& ad : pr.adj) {
          int lam[4] = {0, 0, 0, 0};
          for (int q = 0; q < nv; ++q) lam[ad.second[q]] = al[q];
          Copy cp{ad.first, lam[1], lam[2], lam[3]};
          if (((cp.i + 2 * cp.j + 3 * cp.k) & 3) != L.if_colour.back())
            throw std::runtime_error("inconsistent colouring across macros");
          L.if_copy.push_back(cp);
        }
        L.if_cptr.push_back((int)L.if_copy.size());
      }
    }
    L.n_if = (int)L.if_gid.size();
    number_if_by_colour(L);
    build_pair_tiles(N, L.tiles_int, TILE_TARGET_DEFAULT, TILE_SLABS);
    build_tiles(N, false, L.tiles_all);
    if (N >= STREAM_MIN_N) {
      L.stream_band = N >= 512 ? STREAM_BAND / 2 : STREAM_BAND;
      build_stream_tiles(N, L.stream_band, STREAM_SLICES, L.tiles_stream);
      L.stream_band32 = N >= 512 ? STREAM_BAND32 / 2 : STREAM_BAND32;
      build_stream_tiles(N, L.stream_band32, STREAM_SLICES, L.tiles_stream32);
    }
    m.lv.push_back(std::move(L));
  }
}

// Coarse-level CG system of a problem (level 0): compact numbering of its
// free nodes (volume interiors of the active macros, then free interface
// nodes), the matrix assembled from the per-macro sub-stencils, and the maps
// that gather the right-hand side and scatter the solution.
template <class IdFn>
void assemble_coarse_ids(const HostMesh& m, HostProblem& p, IdFn node_id) {
  p.n_cg = 0;
  p.rowptr.clear();
  p.col.clear();
  p.val.clear();
  p.fsrc.clear();
  p.uptr.clear();
  p.udst.clear();
  p.umaster.clear();

    const HostLevel& L = m.lv[0];
    const int N = L.N;
    std::unordered_map<int64_t, int> cidx;
    struct Dof { std::vector<Copy> cps; int master; };
    std::vector<Dof> dofs;
    for (int t : p.act)
      for (int k = 1; k <= N - 3; ++k)
        for (int j = 1; j + k <= N - 2; ++j)
          for (int i = 1; i + j + k <= N - 1; ++i) {
            cidx[node_id(t, i, j, k)] = (int)dofs.size();
            dofs.push_back(Dof{{Copy{t, i, j, k}}, -1});
          }
    for (int n : p.lv[0].free_if) {
      Dof d;
      d.master = n;
      for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c)
        if (p.macro_active[L.if_copy[c].macro]) d.cps.push_back(L.if_copy[c]);
      cidx[L.if_gid[n]] = (int)dofs.size();
      dofs.push_back(d);
    }
    p.n_cg = (int)dofs.size();
    p.rowptr.push_back(0);
    p.uptr.push_back(0);
    for (auto& d : dofs) {
      std::map<int, double> row;
      for (const Copy& cp : d.cps) {
        int mask = node_class(cp.i, cp.j, cp.k, N);
        const double* w = &L.W[((size_t)cp.macro * 16 + mask) * NDIR];
        for (int e = 0; e < NDIR; ++e) {
          if (w[e] == 0.0) continue;
          int di, dj, dk;
          dir_ijk(e, di, dj, dk);
          int ni = cp.i + di, nj = cp.j + dj, nk = cp.k + dk;
          if (!in_lattice(ni, nj, nk, N)) continue;
          auto it = cidx.find(node_id(cp.macro, ni, nj, nk));
          if (it == cidx.end()) continue;
          row[it->second] += w[e];
        }
        p.udst.push_back((int64_t)cp.macro * L.block + lidx(L.SL.data(), N, cp.i, cp.j, cp.k));
      }
      for (auto& kv : row) {
        p.col.push_back(kv.first);
        p.val.push_back(kv.second);
      }
      p.rowptr.push_back((int)p.col.size());
      p.uptr.push_back((int)p.udst.size());
      p.umaster.push_back(d.master);
      if (d.master >= 0) p.fsrc.push_back(-1 - (int64_t)d.master);
      else p.fsrc.push_back(p.udst.back());
    }
  }

int64_t general_volume_id(const HostLevel& L, int macro, int i, int j, int k) {
  const int64_t N = L.N;
  // interior slices k' < k hold T(N - 2 - k') nodes, T(m) = m (m + 1) / 2;
  // rows j' < j of slice k hold N - 1 - j' - k nodes each
  int64_t before = 0;
  for (int64_t kk = 1; kk < k; ++kk) {
    const int64_t M = N - 2 - kk;
    before += M * (M + 1) / 2;
  }
  before += (int64_t)(j - 1) * (N - 1 - k) - (int64_t)(j - 1) * j / 2;
  const int64_t nvol = (N - 1) * (N - 2) * (N - 3) / 6;
  return (int64_t)L.n_if + (int64_t)macro * nvol + before + (i - 1);
}

void assemble_coarse(const HostMesh& m, HostProblem& p) {
  if (m.general) {
    const HostLevel& L = m.lv[0];
    std::unordered_map<NodeKey, int64_t, KeyHash> if_id;
    for (int n = 0; n < L.n_if; ++n) {
      const Copy& cp = L.if_copy[L.if_cptr[n]];
      if_id[node_key(m, cp.macro, L.N, cp.i, cp.j, cp.k)] = L.if_gid[n];
    }
    assemble_coarse_ids(m, p, [&](int t, int i, int j, int k) -> int64_t {
      if (node_class(i, j, k, L.N) == 0) return general_volume_id(L, t, i, j, k);
      return if_id.at(node_key(m, t, L.N, i, j, k));
    });
    return;
  }
  const int N = m.lv[0].N;
  assemble_coarse_ids(m, p, [&](int t, int i, int j, int k) { return node_gid(m, t, N, i, j, k); });
}

bool copy_offsets(const HostMesh& m, int l, const std::vector<Copy>& copies, std::vector<uint32_t>& out) {
  const HostLevel& L = m.lv[l];
  out.clear();
  if ((uint64_t)m.n_macro * (uint64_t)L.block > 0xffffffffull) return false;
  out.reserve(copies.size());
  for (const Copy& cp : copies)
    out.push_back((uint32_t)((int64_t)cp.macro * L.block + lidx(L.SL.data(), L.N, cp.i, cp.j, cp.k)));
  return true;
}

bool build_if_tables(const HostMesh& m, int l, const std::vector<int>& free_if, const std::vector<int>& cptr,
                     const std::vector<Copy>& copies, int K, std::vector<uint32_t>& nb, std::vector<double>& w,
                     std::vector<double>& diag) {
  nb.clear();
  w.clear();
  diag.clear();
  const HostLevel& L = m.lv[l];
  const int N = L.N;
  const size_t n = free_if.size();
  if (m.general || (uint64_t)m.n_macro * (uint64_t)L.block > 0xffffffffull) return false;
  nb.assign((size_t)K * n, 0);
  w.assign((size_t)K * n, 0.0);
  diag.assign(n, 0.0);
  struct Ent {
    int64_t gid;
    double w;
    uint32_t off;
  };
  std::vector<Ent> ent;
  for (size_t q = 0; q < n; ++q) {
    const int node = free_if[q];
    ent.clear();
    double dg = 0.0;
    uint32_t self = 0;
    for (int c = cptr[node]; c < cptr[node + 1]; ++c) {
      const Copy& cp = copies[c];
      const double* wm = &L.W[((size_t)cp.macro * 16 + node_class(cp.i, cp.j, cp.k, N)) * NDIR];
      if (c == cptr[node]) self = (uint32_t)((int64_t)cp.macro * L.block + lidx(L.SL.data(), N, cp.i, cp.j, cp.k));
      dg += wm[0];
      for (int d = 1; d < NDIR; ++d) {
        if (wm[d] == 0.0) continue;
        int di, dj, dk;
        dir_ijk(d, di, dj, dk);
        const int ni = cp.i + di, nj = cp.j + dj, nk = cp.k + dk;
        if (!in_lattice(ni, nj, nk, N)) continue;
        const int64_t g = node_gid(m, cp.macro, N, ni, nj, nk);
        bool found = false;
        for (Ent& e : ent)
          if (e.gid == g) {
            e.w += wm[d];
            found = true;
            break;
          }
        if (!found)
          ent.push_back(Ent{g, wm[d], (uint32_t)((int64_t)cp.macro * L.block + lidx(L.SL.data(), N, ni, nj, nk))});
      }
    }
    if ((int)ent.size() > K) {
      nb.clear();
      w.clear();
      diag.clear();
      return false;
    }
    diag[q] = dg;
    for (int e = 0; e < K; ++e) {
      nb[(size_t)e * n + q] = e < (int)ent.size() ? ent[e].off : self;
      w[(size_t)e * n + q] = e < (int)ent.size() ? ent[e].w : 0.0;
    }
  }
  return true;
}

void build_problem(const HostMesh& m, int kind, const std::vector<unsigned char>& faulty, HostProblem& p) {
  p = HostProblem();
  p.kind = kind;
  p.macro_active.assign(m.n_macro, 0);
  for (int t = 0; t < m.n_macro; ++t) {
    bool f = macro_in_set(faulty, t);
    bool a = kind == 0 ? true : (kind == 1 ? f : !f);
    p.macro_active[t] = a;
    if (a) p.act.push_back(t);
  }
  const int nl = (int)m.lv.size();
  p.lv.resize(nl);
  std::vector<std::vector<unsigned char>> is_free(nl);
  for (int l = 0; l < nl; ++l) {
    const HostLevel& L = m.lv[l];
    HostProblemLevel& P = p.lv[l];
    is_free[l].assign(L.n_if, 0);
    std::vector<int> bycol[4];
    for (int n = 0; n < L.n_if; ++n) {
      bool any_f = false, all_f = true;
      for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c) {
        bool f = macro_in_set(faulty, L.if_copy[c].macro);
        any_f = any_f || f;
        all_f = all_f && f;
      }
      bool fr = !L.if_dirichlet[n];
      if (kind == 1) fr = fr && all_f;
      if (kind == 2) fr = fr && !any_f;
      if (kind == 3) fr = fr && !all_f;
      is_free[l][n] = fr;
      if (fr) {
        bycol[L.if_colour[n]].push_back(n);
      } else {
        for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c) {
          const Copy& cp = L.if_copy[c];
          if (p.macro_active[cp.macro])
            P.zero_off.push_back((int64_t)cp.macro * L.block + lidx(L.SL.data(), L.N, cp.i, cp.j, cp.k));
        }
      }
    }
    P.col_off[0] = 0;
    for (int c = 0; c < 4; ++c) {
      P.free_if.insert(P.free_if.end(), bycol[c].begin(), bycol[c].end());
      P.col_off[c + 1] = (int)P.free_if.size();
    }
    if (kind == 3) {
      // only the healthy copies take part: their sub-stencils sum to A_I, and
      // the copies inside the faulty blocks keep the other side's values
      P.cptr.assign(1, 0);
      for (int n = 0; n < L.n_if; ++n) {
        for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c)
          if (p.macro_active[L.if_copy[c].macro]) P.copies.push_back(L.if_copy[c]);
        P.cptr.push_back((int)P.copies.size());
      }
    }
  }
  // restriction gathers onto every level below the finest
  for (int l = 0; l + 1 < nl; ++l) {
    const HostLevel& C = m.lv[l];
    const HostLevel& F = m.lv[l + 1];
    HostProblemLevel& P = p.lv[l];
    P.gather.assign(P.free_if.size() * NDIR, -1);
    for (size_t q = 0; q < P.free_if.size(); ++q) {
      int n = P.free_if[q];
      std::vector<int64_t> seen;
      int cnt = 0;
      for (int c = C.if_cptr[n]; c < C.if_cptr[n + 1]; ++c) {
        const Copy& cp = C.if_copy[c];
        if (!p.macro_active[cp.macro]) continue;
        for (int d = 0; d < NDIR; ++d) {
          int di, dj, dk;
          dir_ijk(d, di, dj, dk);
          int fi = 2 * cp.i + di, fj = 2 * cp.j + dj, fk = 2 * cp.k + dk;
          if (!in_lattice(fi, fj, fk, F.N)) continue;
          int64_t g = node_gid(m, cp.macro, F.N, fi, fj, fk);
          if (std::find(seen.begin(), seen.end(), g) != seen.end()) continue;
          seen.push_back(g);
          if (cnt >= NDIR) throw std::runtime_error("restriction stencil has more than 15 points");
          int64_t off = (int64_t)cp.macro * F.block + lidx(F.SL.data(), F.N, fi, fj, fk);
          // the centre (the coarse node itself, weight 1) comes first; the 14
          // edge midpoints follow (weight 1/2)
          if (d == 0 && cnt != 0) throw std::runtime_error("restriction centre not first");
          P.gather[q * NDIR + cnt] = off;
          ++cnt;
        }
      }
      // with the interface free next to inactive macros (kind 3) the fine
      // points inside those macros are not reachable; their residual is zero
      if (cnt != NDIR && !(kind == 3 && cnt > 0)) throw std::runtime_error("restriction stencil incomplete");
    }
  }
  assemble_coarse(m, p);
}


// ---------------------------------------------------------------------------
// Macro meshes of general connectivity (§2.1: an unstructured base mesh of a
// polyhedral domain, refined uniformly).  The per-macro blocks, stencils and
// copy lists are the cube family's; what differs is how nodes are named (keys
// from the macro vertices instead of grid coordinates), which nodes are
// Dirichlet (those on faces of a single macro), and the smoother order of the
// interface nodes: neighbouring macros' local colourings need not agree, so
// the interface nodes get classes of their own (a greedy colouring of their
// coupling graph in key order), visited after the four volume colours.
// ---------------------------------------------------------------------------
void build_general_mesh(HostMesh& m, const double* verts, int nv, const int* tets, int nt, int R, int r0,
                        const double* coeff) {
  if (nv < 4 || nt < 1 || !verts || !tets) throw std::invalid_argument("need vertices and macros");
  m = HostMesh();
  m.general = true;
  m.R = R;
  m.r0 = r0;
  m.n_macro = nt;
  for (int a = 0; a < 9; ++a) m.G[a] = a % 4 == 0 ? 1.0 : 0.0;
  m.vpos.assign(verts, verts + 3 * (size_t)nv);
  for (double x : m.vpos)
    if (!std::isfinite(x)) throw std::invalid_argument("vertex positions must be finite");
  m.coeff.assign(nt, 1.0);
  if (coeff)
    for (int t = 0; t < nt; ++t) m.coeff[t] = coeff[t];
  m.mverts.resize(nt);
  double scale = 0.0;
  for (double x : m.vpos) scale = std::max(scale, std::fabs(x));
  for (int t = 0; t < nt; ++t) {
    for (int q = 0; q < 4; ++q) {
      const int g = tets[4 * (size_t)t + q];
      if (g < 0 || g >= nv) throw std::invalid_argument("macro " + std::to_string(t) + ": vertex id out of range");
      m.mverts[t][q] = g;
    }
    double E[3][3];
    for (int q = 0; q < 3; ++q)
      for (int a = 0; a < 3; ++a) E[a][q] = m.vpos[3 * (size_t)m.mverts[t][q + 1] + a] - m.vpos[3 * (size_t)m.mverts[t][0] + a];
    const double det = E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) -
                       E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
                       E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
    if (!(std::fabs(det) > 1e-12 * scale * scale * scale))
      throw std::invalid_argument("macro " + std::to_string(t) + " is degenerate");
  }

  // primitives keyed by their sorted vertex ids, with the adjacent macros
  std::map<std::vector<int>, int> key;
  std::vector<Prim> prims;
  auto add = [&](int t, const std::vector<int>& loc) {
    std::vector<std::pair<int, int>> gl;
    for (int l : loc) gl.push_back({m.mverts[t][l], l});
    std::sort(gl.begin(), gl.end());
    std::vector<int> g;
    for (auto& x : gl) g.push_back(x.first);
    for (size_t q = 1; q < g.size(); ++q)
      if (g[q] == g[q - 1]) throw std::invalid_argument("macro " + std::to_string(t) + " repeats a vertex");
    auto it = key.find(g);
    int id;
    if (it == key.end()) {
      id = (int)prims.size();
      key[g] = id;
      Prim pr;
      pr.type = (int)loc.size() - 1;
      pr.gv = g;
      prims.push_back(pr);
    } else {
      id = it->second;
    }
    std::array<int, 3> lv = {-1, -1, -1};
    for (size_t q = 0; q < gl.size(); ++q) lv[q] = gl[q].second;
    prims[id].adj.push_back({t, lv});
  };
  for (int t = 0; t < nt; ++t) {
    for (int q = 0; q < 4; ++q) add(t, {q});
    for (int q = 0; q < 4; ++q)
      for (int r = q + 1; r < 4; ++r) add(t, {q, r});
    for (int o = 0; o < 4; ++o) {
      std::vector<int> loc;
      for (int q = 0; q < 4; ++q)
        if (q != o) loc.push_back(q);
      add(t, loc);
    }
  }
  // Dirichlet boundary: the faces of a single macro, their edges and vertices
  for (auto& pr : prims) {
    if (pr.type != 2) continue;
    if (pr.adj.size() > 2) throw std::invalid_argument("a face is shared by more than two macros");
    if (pr.adj.size() != 1) continue;
    pr.boundary = true;
    for (int a = 0; a < 3; ++a) {
      prims[key.at({pr.gv[a]})].boundary = true;
      for (int b = a + 1; b < 3; ++b) prims[key.at({pr.gv[a], pr.gv[b]})].boundary = true;
    }
  }

  m.lv.clear();
  m.seven_point = false;
  for (int r = r0; r <= R; ++r) {
    HostLevel L;
    L.r = r;
    L.N = 1 << r;
    L.block = build_slice_starts(L.N, L.SL);
    const int N = L.N;
    compute_level_weights(m, L);
    // interface nodes in key order
    struct INode { NodeKey k; int prim; std::array<int, 3> al; };
    std::vector<INode> nodes;
    for (int id = 0; id < (int)prims.size(); ++id) {
      const Prim& pr = prims[id];
      const int nvp = (int)pr.gv.size();
      std::vector<std::array<int, 3>> alphas;
      if (nvp == 1) alphas.push_back({N, 0, 0});
      if (nvp == 2)
        for (int a = 1; a <= N - 1; ++a) alphas.push_back({a, N - a, 0});
      if (nvp == 3)
        for (int a = 1; a <= N - 2; ++a)
          for (int b = 1; a + b <= N - 1; ++b) alphas.push_back({a, b, N - a - b});
      for (auto& al : alphas) {
        int64_t v[4] = {-1, -1, -1, -1};
        for (int q = 0; q < nvp; ++q) v[4 - nvp + q] = (int64_t)pr.gv[q] * (N + 1) + al[q];
        nodes.push_back({NodeKey{nvp, v[0], v[1], v[2], v[3]}, id, al});
      }
    }
    std::sort(nodes.begin(), nodes.end(), [](const INode& a, const INode& b) { return a.k < b.k; });
    L.if_cptr.push_back(0);
    for (size_t n = 0; n < nodes.size(); ++n) {
      const Prim& pr = prims[nodes[n].prim];
      L.if_gid.push_back((int64_t)n);
      L.if_dirichlet.push_back(pr.boundary ? 1 : 0);
      for (auto& ad : pr.adj) {
        int lam[4] = {0, 0, 0, 0};
        for (size_t q = 0; q < pr.gv.size(); ++q) lam[ad.second[q]] = nodes[n].al[q];
        L.if_copy.push_back(Copy{ad.first, lam[1], lam[2], lam[3]});
      }
      L.if_cptr.push_back((int)L.if_copy.size());
    }
    L.n_if = (int)nodes.size();
    // interface classes: greedy colouring of the coupling graph of the free
    // interface nodes (lattice neighbours inside some macro), in key order
    std::unordered_map<int64_t, int> at;               // macro * block + slot -> interface node
    for (int n = 0; n < L.n_if; ++n)
      for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c) {
        const Copy& cp = L.if_copy[c];
        at[(int64_t)cp.macro * L.block + lidx(L.SL.data(), N, cp.i, cp.j, cp.k)] = n;
      }
    std::vector<int> cls(L.n_if, -1);
    int n_cls = 0;
    for (int n = 0; n < L.n_if; ++n) {
      if (L.if_dirichlet[n]) continue;
      std::vector<char> used(64, 0);
      for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c) {
        const Copy& cp = L.if_copy[c];
        for (int d = 1; d < NDIR; ++d) {
          int di, dj, dk;
          dir_ijk(d, di, dj, dk);
          const int ni = cp.i + di, nj = cp.j + dj, nk = cp.k + dk;
          if (!in_lattice(ni, nj, nk, N) || node_class(ni, nj, nk, N) == 0) continue;
          auto it = at.find((int64_t)cp.macro * L.block + lidx(L.SL.data(), N, ni, nj, nk));
          if (it != at.end() && cls[it->second] >= 0) {
            if (cls[it->second] >= (int)used.size()) used.resize(cls[it->second] + 1, 0);
            used[cls[it->second]] = 1;
          }
        }
      }
      int c = 0;
      while (c < (int)used.size() && used[c]) ++c;
      if (c > 250) throw std::invalid_argument("too many interface classes");
      cls[n] = c;
      n_cls = std::max(n_cls, c + 1);
    }
    L.if_colour.resize(L.n_if);
    for (int n = 0; n < L.n_if; ++n) L.if_colour[n] = (unsigned char)(cls[n] < 0 ? 0 : cls[n]);
    L.n_if_classes = n_cls;
    build_pair_tiles(N, L.tiles_int, TILE_TARGET_DEFAULT, TILE_SLABS);
    build_tiles(N, false, L.tiles_all);
    if (N >= STREAM_MIN_N) {
      L.stream_band = N >= 512 ? STREAM_BAND / 2 : STREAM_BAND;
      build_stream_tiles(N, L.stream_band, STREAM_SLICES, L.tiles_stream);
      L.stream_band32 = N >= 512 ? STREAM_BAND32 / 2 : STREAM_BAND32;
      build_stream_tiles(N, L.stream_band32, STREAM_SLICES, L.tiles_stream32);
    }
    m.lv.push_back(std::move(L));
  }
}

void build_general_problem(const HostMesh& m, int kind, const std::vector<unsigned char>& faulty,
                           HostProblem& p) {
  p = HostProblem();
  p.kind = kind;
  p.macro_active.assign(m.n_macro, 0);
  for (int t = 0; t < m.n_macro; ++t) {
    const bool f = macro_in_set(faulty, t);
    const bool a = kind == 0 ? true : (kind == 1 ? f : !f);
    p.macro_active[t] = a;
    if (a) p.act.push_back(t);
  }
  const int nl = (int)m.lv.size();
  p.lv.resize(nl);
  for (int l = 0; l < nl; ++l) {
    const HostLevel& L = m.lv[l];
    HostProblemLevel& P = p.lv[l];
    std::vector<std::vector<int>> bycls(std::max(1, L.n_if_classes));
    for (int n = 0; n < L.n_if; ++n) {
      // free as for the cube family: all copies faulty (kind 1), none (kind
      // 2), not all (kind 3, the Neumann side with its interface free)
      bool any_f = false, all_f = true;
      for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c) {
        const bool f = macro_in_set(faulty, L.if_copy[c].macro);
        any_f = any_f || f;
        all_f = all_f && f;
      }
      bool fr = !L.if_dirichlet[n];
      if (kind == 1) fr = fr && all_f;
      if (kind == 2) fr = fr && !any_f;
      if (kind == 3) fr = fr && !all_f;
      if (fr) {
        bycls[L.if_colour[n]].push_back(n);
      } else {
        for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c) {
          const Copy& cp = L.if_copy[c];
          if (p.macro_active[cp.macro])
            P.zero_off.push_back((int64_t)cp.macro * L.block + lidx(L.SL.data(), L.N, cp.i, cp.j, cp.k));
        }
      }
    }
    P.class_off.assign(1, 0);
    for (auto& b : bycls) {
      P.free_if.insert(P.free_if.end(), b.begin(), b.end());
      P.class_off.push_back((int)P.free_if.size());
    }
    P.col_off[4] = (int)P.free_if.size();
    if (kind == 3) {
      P.cptr.assign(1, 0);
      for (int n = 0; n < L.n_if; ++n) {
        for (int c = L.if_cptr[n]; c < L.if_cptr[n + 1]; ++c)
          if (p.macro_active[L.if_copy[c].macro]) P.copies.push_back(L.if_copy[c]);
        P.cptr.push_back((int)P.copies.size());
      }
    }
  }
  // restriction gathers: the distinct fine nodes 2 (i, j, k) + d over the
  // active copies of each free coarse interface node, the node itself first
  for (int l = 0; l + 1 < nl; ++l) {
    const HostLevel& F = m.lv[l + 1];
    const HostLevel& C = m.lv[l];
    HostProblemLevel& P = p.lv[l];
    P.gptr.assign(1, 0);
    for (int n : P.free_if) {
      std::vector<NodeKey> seen;
      for (int pass = 0; pass < 2; ++pass)
        for (int c = C.if_cptr[n]; c < C.if_cptr[n + 1]; ++c) {
          const Copy& cp = C.if_copy[c];
          if (!p.macro_active[cp.macro]) continue;
          for (int d = (pass == 0 ? 0 : 1); d < (pass == 0 ? 1 : NDIR); ++d) {
            int di, dj, dk;
            dir_ijk(d, di, dj, dk);
            const int fi = 2 * cp.i + di, fj = 2 * cp.j + dj, fk = 2 * cp.k + dk;
            if (!in_lattice(fi, fj, fk, F.N)) continue;
            const NodeKey kf = node_key(m, cp.macro, F.N, fi, fj, fk);
            if (std::find(seen.begin(), seen.end(), kf) != seen.end()) continue;
            seen.push_back(kf);
            P.goff.push_back((int64_t)cp.macro * F.block + lidx(F.SL.data(), F.N, fi, fj, fk));
          }
        }
      P.gptr.push_back((int)P.goff.size());
    }
  }
  assemble_coarse(m, p);
}

}  // namespace hhg
