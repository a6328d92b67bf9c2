// Consistency check of the host symbolic pass (no GPU): every position the
// kernels will dereference points at the DOF it claims, and the group counts
// match the closed forms c^3, 3(c-1)c^2, 3(c-1)^2 c, (c-1)^3 (Dirichlet) or
// c^3, 3c^3, 3c^3, c^3 (periodic grid: third argument "p").
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "symbolic.h"

using namespace hif;

static int fails = 0;
#define CHECK(c, ...)                      \
  do {                                     \
    if (!(c)) {                            \
      if (fails < 20) {                    \
        std::printf("FAIL %s: ", #c);      \
        std::printf(__VA_ARGS__);          \
        std::printf("\n");                 \
      }                                    \
      ++fails;                             \
    }                                      \
  } while (0)

static bool periodic = false;
static int L = 0;
static bool is_sep(int x, int s, int level) {
  return periodic ? (level < L && x % s == 0) : (x != 0 && x % s == 0);
}

int main(int argc, char** argv) {
  int n = argc > 1 ? std::atoi(argv[1]) : 16;
  int m = argc > 2 ? std::atoi(argv[2]) : 4;
  periodic = argc > 3 && argv[3][0] == 'p';
  Symbolic sym(n, m, periodic);
  L = sym.levels();
  const int64_t N = (int64_t)n * n * n;
  CellPlan prev;
  long long rows_total = 0;
  for (int level = 0; level <= L; ++level) {
    CellPlan cp;
    sym.build_cells(level, cp);
    const int s = cp.s, C = cp.C;
    // each active DOF: in exactly one interior, or in >= 1 boundary list
    std::vector<int> seenI(N, 0), seenB(N, 0);
    for (int c = 0; c < cp.ncell; ++c) {
      const int cx = c % C, cy = (c / C) % C, cz = c / (C * C);
      for (int64_t t = cp.off[c]; t < cp.off[c + 1]; ++t) {
        const int g = cp.dofs[t];
        const int x[3] = {g % n, (g / n) % n, g / (n * n)};
        const int cc[3] = {cx, cy, cz};
        bool interior = t < cp.off[c] + cp.p[c];
        for (int d = 0; d < 3; ++d) {
          const int lo = s * cc[d], hi = std::min(s * (cc[d] + 1), n - 1);
          if (periodic)   // the closure runs from plane lo to plane lo + s, wrapping
            CHECK(((x[d] - lo) % n + n) % n <= s, "dof %d outside closure of cell %d", g, c);
          else
            CHECK(x[d] >= lo && x[d] <= hi, "dof %d outside closure of cell %d", g, c);
          if (interior) CHECK(!is_sep(x[d], s, level), "interior dof %d on a separator", g);
        }
        if (interior) seenI[g]++;
        else {
          seenB[g]++;
          const int b = (int)(t - cp.off[c] - cp.p[c]);
          CHECK(sym.pos_in_cell(cp, g, cx, cy, cz) == b, "posB mismatch dof %d cell %d", g, c);
        }
      }
    }
    for (int32_t g : cp.active) CHECK((seenI[g] == 1) != (seenB[g] > 0), "dof %d coverage", g);
    // merge maps
    if (level > 0) {
      std::vector<int64_t> moff;
      PlanVec32 map;
      sym.merge_maps(prev, cp, moff, map);
      for (int c = 0; c < cp.ncell; ++c) {
        const int64_t nn = cp.off[c + 1] - cp.off[c];
        const int px = c % C, py = (c / C) % C, pz = c / (C * C);
        int covered_pairs_ok = 1;
        for (int q = 0; q < 8; ++q) {
          const int cx = 2 * px + (q & 1), cy = 2 * py + ((q >> 1) & 1), cz = 2 * pz + ((q >> 2) & 1);
          for (int64_t a = 0; a < nn; ++a) {
            const int32_t pos = map[moff[c] + q * nn + a];
            if (pos < 0) continue;
            const int ch = cx + prev.C * (cy + prev.C * cz);
            const int64_t nb = prev.off[ch + 1] - prev.off[ch] - prev.p[ch];
            CHECK(pos < nb, "merge pos out of range");
            CHECK(prev.dofs[prev.off[ch] + prev.p[ch] + pos] == cp.dofs[cp.off[c] + a],
                  "merge map mismatch");
          }
        }
        (void)covered_pairs_ok;
        // every parent DOF comes from at least one child
        for (int64_t a = 0; a < nn; ++a) {
          bool any = false;
          for (int q = 0; q < 8; ++q) any = any || map[moff[c] + q * nn + a] >= 0;
          CHECK(any, "parent dof without a child");
        }
      }
    }
    if (level == L) {
      CHECK(cp.ncell == 1 && (int64_t)cp.p[0] == (int64_t)cp.dofs.size(), "root is one interior");
      std::printf("level %d (root): %lld dofs\n", level, (long long)cp.dofs.size());
      break;
    }
    // faces then edges with every boundary DOF alive (exact mode)
    std::vector<uint8_t> alive(N, 0);
    for (int32_t g : cp.active) alive[g] = 1;
    for (int c = 0; c < cp.ncell; ++c)
      for (int64_t t = cp.off[c]; t < cp.off[c] + cp.p[c]; ++t) alive[cp.dofs[t]] = 0;
    int counts[3] = {cp.ncell, 0, 0};
    for (int kind = 1; kind <= 2; ++kind) {
      SkelPlan sp;
      sym.build_skel(cp, kind, alive, sp);
      counts[kind] = sp.nfront;
      const int ncp = sp.ncellPer;
      for (int f = 0; f < sp.nfront; ++f) {
        for (int64_t r = sp.rowOff[f]; r < sp.rowOff[f + 1]; ++r) {
          const int g = sp.rowDof[r];
          bool anyp = false;
          for (int i = 0; i < ncp; ++i) {
            const int cell = sp.cells[(size_t)f * ncp + i];
            const int32_t pos = sp.rowPos[r * ncp + i];
            if (r < sp.rowOff[f] + sp.nF[f]) CHECK(pos >= 0, "front dof missing in one of its cells");
            if (pos < 0) continue;
            anyp = true;
            const int64_t nb = cp.off[cell + 1] - cp.off[cell] - cp.p[cell];
            CHECK(pos < nb, "row pos out of range");
            CHECK(cp.dofs[cp.off[cell] + cp.p[cell] + pos] == g, "row pos mismatch");
          }
          CHECK(anyp, "row in no cell");
        }
        rows_total += sp.rowOff[f + 1] - sp.rowOff[f];
      }
    }
    // an edge plan built before some face DOFs die, then filtered, equals a
    // plan built afterwards
    {
      std::vector<uint8_t> alive_pre = alive, alive_post = alive;
      int t = 0;
      for (int32_t g : cp.active) {
        const int x[3] = {g % n, (g / n) % n, g / (n * n)};
        int ns = 0;
        for (int d = 0; d < 3; ++d) ns += is_sep(x[d], s, level);
        if (ns == 1 && alive_post[g] && (t++ % 3 == 0)) alive_post[g] = 0;
      }
      SkelPlan a, b;
      sym.build_skel(cp, 2, alive_pre, a);
      sym.filter_rows(a, alive_post);
      sym.build_skel(cp, 2, alive_post, b);
      CHECK(a.nfront == b.nfront && a.rowOff == b.rowOff && a.rowDof == b.rowDof &&
                a.rowPos == b.rowPos && a.nR == b.nR && a.cells == b.cells,
            "filtered edge plan differs at level %d", level);
    }
    const int c = C;
    CHECK(counts[1] == (periodic ? 3 * c * c * c : 3 * (c - 1) * c * c), "face count");
    CHECK(counts[2] == (periodic ? 3 * c * c * c : 3 * (c - 1) * (c - 1) * c), "edge count");
    std::printf("level %d: %d cells, %d faces, %d edges\n", level, counts[0], counts[1], counts[2]);
    std::vector<int32_t> next;
    for (int32_t g : cp.active)
      if (alive[g]) next.push_back(g);
    // building from an explicit list equals building from the stored set
    {
      CellPlan x, y;
      sym.build_cells_from(level + 1, next, x);
      sym.set_active(next);
      sym.build_cells(level + 1, y);
      CHECK(x.dofs == y.dofs && x.off == y.off && x.p == y.p && x.posB == y.posB,
            "build_cells_from differs");
    }
    sym.set_active(next);
    prev = std::move(cp);
  }
  std::printf("rows %lld\n", rows_total);
  std::printf(fails ? "FAILED %d\n" : "OK\n", fails);
  return fails ? 1 : 0;
}
