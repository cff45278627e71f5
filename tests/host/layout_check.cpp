// Host-side check of the blocked colour-split layout (hhg_internal.h) and of
// the row-pair work tiles of the volume kernels (csrc/mesh.cpp), driven by
// tests/test_host_layout.py.  Runs on the CPU; makes no CUDA call.
//
// usage: layout_check N_max
// Checks every refinement N = 2 .. N_max and N = 256, 512, and prints one
// line per failed property (exit status 1), else "ok".
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1506_06185_gb300/csrc/hhg_internal.h"

using namespace hhg;

static int failures = 0;

#define CHECK(cond, ...)                    \
  do {                                      \
    if (!(cond)) {                          \
      if (failures < 20) {                  \
        std::printf("N=%d: ", N);           \
        std::printf(__VA_ARGS__);           \
        std::printf("\n");                  \
      }                                     \
      ++failures;                           \
    }                                       \
  } while (0)

// S(m) by its definition: the slots of rows of 1 .. m nodes, 4 ceil(l / 16) each.
static int64_t slots_by_definition(int m) {
  int64_t s = 0;
  for (int l = 1; l <= m; ++l) s += 4 * ((l + 15) / 16);
  return s;
}

static void check_layout(int N) {
  std::vector<int> SL;
  const int64_t block = build_slice_starts(N, SL);
  const int CS = SL[N + 2];
  CHECK(block == 4 * (int64_t)CS, "block %lld != 4 CS", (long long)block);
  CHECK(CS % 64 == 0, "CS %d not a multiple of 64", CS);
  // every lattice node gets its own slot, inside its colour's array; rows
  // start on a multiple of four slots (16 bytes in FP32, two FP64 vectors)
  std::vector<unsigned char> used((size_t)block, 0);
  for (int k = 0; k <= N; ++k)
    for (int j = 0; j + k <= N; ++j) {
      const int M = N + 1 - k;
      const int row = SL[k] + slot_prefix(M) - slot_prefix(M - j);
      CHECK(row % 4 == 0, "row (%d, %d) starts at slot %d", j, k, row);
      const int L = M - j;
      CHECK(row + row_slots(L) <= CS, "row (%d, %d) ends past CS", j, k);
      for (int i = 0; i + j + k <= N; ++i) {
        const int c = (i + 2 * j + 3 * k) & 3;
        const int o = lidx(SL.data(), N, i, j, k);
        CHECK(o >= c * CS && o < (c + 1) * CS, "node (%d, %d, %d) outside colour array %d", i, j, k, c);
        CHECK(o == c * CS + row + (i >> 2), "node (%d, %d, %d) not in slot i >> 2 of its row", i, j, k);
        if (o >= 0 && o < block) {
          CHECK(!used[o], "node (%d, %d, %d) shares slot %d", i, j, k, o);
          used[o] = 1;
        }
      }
      // the neighbour rows the vector kernels address from row (j, k):
      // (j + 1, k) follows after row_slots(L), (j - 1, k) precedes by row_slots(L + 1)
      if (j + k < N) CHECK(SL[k] + slot_prefix(M) - slot_prefix(M - j - 1) == row + row_slots(L), "row (%d+1, %d)", j, k);
      if (j > 0) CHECK(SL[k] + slot_prefix(M) - slot_prefix(M - j + 1) == row - row_slots(L + 1), "row (%d-1, %d)", j, k);
    }
  // slice starts: slice k + 1 begins where slice k's S(N + 1 - k) slots end
  for (int k = 0; k <= N; ++k) CHECK(SL[k + 1] - SL[k] == slot_prefix(N + 1 - k), "slice %d length", k);
}

static void check_pair_tiles(int N, int target, int slabs) {
  if (N < 4) return;
  std::vector<Tile> tiles;
  build_pair_tiles(N, tiles, target, slabs);
  // cover[k][j]: how often interior row j of slice k is covered
  std::vector<std::vector<int>> cover(N + 1, std::vector<int>(N + 1, 0));
  int64_t prev_work = -1;
  for (size_t q = 0; q < tiles.size(); ++q) {
    const Tile& t = tiles[q];
    // the kernels' shared tables hold 16 slices of 32 pairs per tile
    CHECK(t.pad >= 1 && t.pad <= 16, "tile %zu: %d slices (target %d, slabs %d)", q, t.pad, target, slabs);
    CHECK(t.m0 >= 1 && t.m0 <= 32, "tile %zu: %d pairs", q, t.m0);
    CHECK(t.k >= 1 && t.k + t.pad - 1 <= N - 3, "tile %zu: slices %d .. %d", q, t.k, t.k + t.pad - 1);
    int64_t work = 0;
    for (int k = t.k; k < t.k + t.pad && k <= N; ++k)
      for (int p = t.j0; p < t.j0 + t.m0; ++p) {
        const int j1 = 1 + p, j2 = N - 2 - k - p;
        if (j1 > j2) continue;                      // beyond this slice's pairs: empty
        ++cover[k][j1];
        work += N - 1 - j1 - k;
        if (j2 != j1) {
          ++cover[k][j2];
          work += N - 1 - j2 - k;
        }
      }
    // largest tiles first
    if (prev_work >= 0) CHECK(work <= prev_work, "tile %zu: work %lld after %lld", q, (long long)work, (long long)prev_work);
    prev_work = work;
  }
  for (int k = 1; k <= N - 3; ++k)
    for (int j = 1; j + k <= N - 2; ++j)
      CHECK(cover[k][j] == 1, "interior row (%d, %d) covered %d times (target %d, slabs %d)", j, k, cover[k][j],
            target, slabs);
}

// The streaming Gauss-Seidel kernel (k_gs_stream) on refinement N with bands
// of `band` rows and vectors of VW slots: every staged range (colour c+1
// rows j0-1 .. j1+1 of slices k and k+1, colour c-1 of slices k-1 and k, f
// rows j0 .. of slice k) fits one slot of the shared-memory ring and starts
// and ends on 16 bytes; every neighbour read of every interior colour-c node
// a unit updates lands, inside its staged range, on the right lattice node;
// the one-slot shifts of the other lanes stay inside the padded buffer; and
// the units update every interior node of every colour exactly once.  The
// offset expressions are the kernel's.
static int colour_first(int j, int k, int c) { return (c - 2 * j - 3 * k) & 3; }

static void check_stream_tiles(int N, int band, int VW) {
  std::vector<int> SL;
  const int64_t block = build_slice_starts(N, SL);
  (void)block;
  std::vector<StreamTile> tiles;
  build_stream_tiles(N, band, STREAM_SLICES, tiles);
  const int M0 = N + 1;
  const int slot = ((slot_prefix(M0) - slot_prefix(std::max(0, M0 - (band + 2)))) + 31) & ~31;
  const int PAD = 32;
  auto S = [](int m) { return slot_prefix(m); };
  auto range = [&](int k, int ja, int jb, int& off, int& len) {
    const int M = N + 1 - k;
    jb = std::min(jb, N - k);
    off = SL[k] + S(M) - S(M - ja);
    len = jb >= ja ? S(M - ja) - S(M - jb - 1) : 0;
  };
  auto inner = [&](int i, int j, int k) { return lidx(SL.data(), N, i, j, k) - ((i + 2 * j + 3 * k) & 3) * SL[N + 2]; };
  std::vector<unsigned char> hits((size_t)(N + 1) * (N + 1) * (N + 1), 0);
  for (int c = 0; c < 4; ++c) {
    std::fill(hits.begin(), hits.end(), 0);
    for (const StreamTile& t : tiles) {
      CHECK(t.ka >= 1 && t.kb <= N - 2 - t.j0 && t.kb - t.ka < STREAM_SLICES && t.j1 - t.j0 < band,
            "unit (%d..%d, %d..%d)", t.j0, t.j1, t.ka, t.kb);
      const int ja = t.j0 - 1, jbA = t.j1 + 1;
      for (int k = t.ka; k <= t.kb; ++k) {
        int oA0, lA0, oA1, lA1, oB0, lB0, oBm, lBm, oF, lF;
        range(k, ja, jbA, oA0, lA0);
        range(k + 1, ja, jbA, oA1, lA1);
        range(k, ja, jbA, oB0, lB0);
        range(k - 1, ja, jbA, oBm, lBm);
        const int je = std::min(t.j1, N - 2 - k);
        range(k, t.j0, je, oF, lF);
        for (int len : {lA0, lA1, lBm, lF}) CHECK(len <= slot && len % 4 == 0, "staged range %d, slot %d", len, slot);
        for (int off : {oA0, oA1, oBm, oF}) CHECK(off % 4 == 0, "staged range starts at %d", off);
        const int M = N + 1 - k, M1 = N - k, Mm = N + 2 - k;
        const int PA = S(M - ja), PA1 = S(M1 - ja), PAm = S(Mm - ja), PF = S(M - t.j0);
        for (int j = t.j0; j <= je; ++j) {
          const int ic = colour_first(j, k, c);
          const int L = N - 1 - j - k;
          const int mlo = ic == 0;
          const int n = L >= ic ? ((L - ic) >> 2) - mlo + 1 : 0;
          const int X = S(M - j);
          const int groups = n > 0 ? (mlo + n - 1) / VW + 1 : 0;
          for (int g = 0; g < groups; ++g) {
            const int m0 = g * VW;
            struct Rd { int off0, lo, len, shift_lo, shift_hi; } rd[7] = {
                {PA - X, oA0, lA0, 0, ic == 3},               {PA - S(M - j - 1), oA0, lA0, -(ic == 0), 0},
                {PA1 - S(M1 - j + 1), oA1, lA1, 0, 0},        {PA - X, oB0, lB0, -(ic == 0), 0},
                {PA - S(M - j + 1), oB0, lB0, 0, ic == 3},    {PAm - S(Mm - j - 1), oBm, lBm, 0, 0},
                {PF - X, oF, lF, 0, 0}};
            for (const Rd& r : rd)
              CHECK(r.off0 + m0 - 1 >= -PAD && r.off0 + m0 + VW < slot + PAD, "vector read outside the buffer");
            const int lo = std::max(mlo - m0, 0), hi = std::min(mlo + n - m0, VW);
            for (int q = lo; q < hi; ++q) {
              const int m = m0 + q, i = 4 * m + ic;
              CHECK(i >= 1 && i + j + k <= N - 1, "lane outside the interior");
              CHECK(SL[k] + S(M) - X + m == inner(i, j, k), "store slot of (%d, %d, %d)", i, j, k);
              const int nb[7][3] = {{i + 1, j, k}, {i - 1, j + 1, k}, {i, j - 1, k + 1}, {i - 1, j, k},
                                    {i + 1, j - 1, k}, {i, j + 1, k - 1}, {i, j, k}};
              const int sh[7] = {ic == 3, -(ic == 0), 0, -(ic == 0), ic == 3, 0, 0};
              for (int d = 0; d < 7; ++d) {
                const int e = rd[d].off0 + m + sh[d];
                CHECK(e >= 0 && e < rd[d].len, "read %d of (%d, %d, %d) outside its range", d, i, j, k);
                CHECK(rd[d].lo + e == inner(nb[d][0], nb[d][1], nb[d][2]), "read %d of (%d, %d, %d)", d, i, j, k);
              }
              unsigned char& h = hits[((size_t)k * (N + 1) + j) * (N + 1) + i];
              CHECK(h == 0, "(%d, %d, %d) updated twice", i, j, k);
              h = 1;
            }
          }
        }
      }
    }
    for (int k = 1; k <= N; ++k)
      for (int j = 1; j + k <= N - 1; ++j)
        for (int i = 1; i + j + k <= N - 1; ++i)
          if (((i + 2 * j + 3 * k) & 3) == c)
            CHECK(hits[((size_t)k * (N + 1) + j) * (N + 1) + i], "(%d, %d, %d) of colour %d not updated", i, j, k, c);
  }
}

// The flat restriction's slot items (build_slot_items): every interior node
// of a macro lies in exactly one slot of four (i = 4m .. 4m + 3 of its row),
// and every slot holds at least one interior node.
static void check_slot_items(int N) {
  std::vector<uint32_t> items;
  build_slot_items(N, items);
  std::vector<int> seen((size_t)(N + 1) * (N + 1) * (N + 1), 0);
  auto at = [&](int i, int j, int k) { return ((size_t)k * (N + 1) + j) * (N + 1) + i; };
  for (uint32_t d : items) {
    const int j = (int)(d >> 20), k = (int)((d >> 10) & 1023u), m = (int)(d & 1023u);
    CHECK(k >= 1 && k <= N - 3 && j >= 1 && j <= N - 2 - k, "slot items: row (%d, %d) not interior", j, k);
    if (!(k >= 1 && k <= N - 3 && j >= 1 && j <= N - 2 - k)) continue;
    int here = 0;
    for (int q = 0; q < 4; ++q) {
      const int i = 4 * m + q;
      if (i >= 1 && i <= N - 1 - j - k) {
        ++seen[at(i, j, k)];
        ++here;
      }
    }
    CHECK(here > 0, "slot items: slot (%d, %d, %d) holds no node", j, k, m);
  }
  for (int k = 1; k <= N - 3; ++k)
    for (int j = 1; j <= N - 2 - k; ++j)
      for (int i = 1; i <= N - 1 - j - k; ++i)
        CHECK(seen[at(i, j, k)] == 1, "slot items: node (%d, %d, %d) covered %d times", i, j, k, seen[at(i, j, k)]);
}

// The walk order of the large stencil launches (spread_position): every
// interface chunk and every volume unit exactly once, each kind in its own
// order, and while volume units remain no more than R = n_vol / n_if of them
// between two chunks.
static void check_spread(int n_if, int n_vol) {
  const int N = -1;   // for the CHECK message
  std::vector<int> seen_if(n_if, 0), seen_vol(n_vol, 0);
  int last_if = -1, last_vol = -1, run = 0, max_run = 0;
  for (int u = 0; u < n_if + n_vol; ++u) {
    int vol = -1;
    const int c = spread_position(u, n_if, n_vol, vol);
    if (c >= 0) {
      CHECK(c < n_if && c == last_if + 1, "spread %d/%d: position %d gives chunk %d after %d", n_if, n_vol, u, c,
            last_if);
      if (c < n_if) ++seen_if[c];
      last_if = c;
      max_run = std::max(max_run, run);
      run = 0;
    } else {
      CHECK(vol >= 0 && vol < n_vol && vol == last_vol + 1, "spread %d/%d: position %d gives unit %d after %d", n_if,
            n_vol, u, vol, last_vol);
      if (vol >= 0 && vol < n_vol) ++seen_vol[vol];
      last_vol = vol;
      ++run;
    }
  }
  for (int q = 0; q < n_if; ++q) CHECK(seen_if[q] == 1, "spread %d/%d: chunk %d seen %d times", n_if, n_vol, q, seen_if[q]);
  for (int b = 0; b < n_vol; ++b)
    CHECK(seen_vol[b] == 1, "spread %d/%d: unit %d seen %d times", n_if, n_vol, b, seen_vol[b]);
  if (n_if > 0) {
    const int R = std::max(1, n_vol / n_if);
    CHECK(max_run <= R, "spread %d/%d: %d volume units between two chunks (R = %d)", n_if, n_vol, max_run, R);
  }
}

// The flat Gauss-Seidel items (build_gs_items): for each colour, the slots of
// every item hold at least one colour-c interior node, and every colour-c
// interior node of every slice lies in exactly one item's slots.
static void check_gs_items(int N, int vw) {
  std::vector<uint32_t> items;
  int off[5];
  build_gs_items(N, vw, items, off);
  CHECK(off[0] == 0 && off[4] == (int)items.size(), "gs items: offsets %d .. %d of %zu", off[0], off[4], items.size());
  std::vector<int> seen;
  auto at = [&](int i, int j, int k) { return ((size_t)k * (N + 1) + j) * (N + 1) + i; };
  for (int c = 0; c < 4; ++c) {
    CHECK(off[c] <= off[c + 1], "gs items: colour %d offsets decrease", c);
    seen.assign((size_t)(N + 1) * (N + 1) * (N + 1), 0);
    for (int q = off[c]; q < off[c + 1]; ++q) {
      const uint32_t d = items[q];
      const int j = (int)(d >> 20), k = (int)((d >> 10) & 1023u), g = (int)(d & 1023u);
      CHECK(k >= 1 && k <= N - 3 && j >= 1 && j <= N - 2 - k, "gs items vw %d: row (%d, %d) not interior", vw, j, k);
      if (!(k >= 1 && k <= N - 3 && j >= 1 && j <= N - 2 - k)) continue;
      const int L = N - 1 - j - k, ic = (c - 2 * j - 3 * k) & 3;
      int here = 0;
      for (int m = g * vw; m < g * vw + vw; ++m) {
        const int i = 4 * m + ic;
        if (i >= 1 && i <= L) {
          ++seen[at(i, j, k)];
          ++here;
        }
      }
      CHECK(here > 0, "gs items vw %d: item (%d, %d, %d) of colour %d holds no node", vw, j, k, g, c);
    }
    for (int k = 1; k <= N - 3; ++k)
      for (int j = 1; j <= N - 2 - k; ++j)
        for (int i = 1; i <= N - 1 - j - k; ++i)
          if (((i + 2 * j + 3 * k) & 3) == c)
            CHECK(seen[at(i, j, k)] == 1, "gs items vw %d: node (%d, %d, %d) covered %d times", vw, i, j, k,
                  seen[at(i, j, k)]);
  }
}

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const int n_max = std::atoi(argv[1]);
  // S(m) in closed form against its definition
  for (int m = 0; m <= 1100; ++m) {
    const int N = m;
    CHECK(slot_prefix(m) == slots_by_definition(m), "S(%d) = %d, definition %lld", m, slot_prefix(m),
          (long long)slots_by_definition(m));
    if (m > 0) CHECK(slot_prefix(m) - slot_prefix(m - 1) == row_slots(m), "row_slots(%d)", m);
  }
  std::vector<int> ns;
  for (int N = 2; N <= n_max; ++N) ns.push_back(N);
  if (n_max < 256) ns.push_back(256);
  if (n_max < 512) ns.push_back(512);
  // default tiles and the autotuner's candidates (target nodes, slices)
  const int cand[][2] = {{TILE_TARGET_DEFAULT, TILE_SLABS}, {256, 4}, {512, 8}, {1024, 8}, {2048, 16}};
  for (int N : ns) {
    check_layout(N);
    for (const auto& c : cand) check_pair_tiles(N, c[0], c[1]);
  }
  // streaming units on the levels that have them (64 intervals and more),
  // FP64 (two slots per vector) and FP32 (four) bands
  for (int N : {64, 128, 256, 512}) {
    check_stream_tiles(N, N >= 512 ? STREAM_BAND / 2 : STREAM_BAND, 2);
    check_stream_tiles(N, N >= 512 ? STREAM_BAND32 / 2 : STREAM_BAND32, 4);
  }
  for (int N : {4, 5, 8, 13, 16, 32, 64, 128})
    for (int vw : {2, 4}) check_gs_items(N, vw);
  for (int N : {4, 5, 8, 13, 16, 32, 64, 128}) check_slot_items(N);
  for (int n_if = 0; n_if <= 40; ++n_if)
    for (int n_vol = 0; n_vol <= 130; ++n_vol) check_spread(n_if, n_vol);
  // the finest launches of the bench's mesh (refinement 8: about 2300 chunks
  // per colour, 5000 .. 31000 tiles) and of its residual (four colours)
  for (const auto& c : {std::array<int, 2>{2284, 5040}, {2284, 8784}, {2284, 30912}, {9136, 8784}, {9136, 5040}})
    check_spread(c[0], c[1]);
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
