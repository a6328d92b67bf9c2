// Host-side symbolic pass (geometry of §2.1 with a Dirichlet boundary).
#include "symbolic.h"

#include <algorithm>
#include <thread>

namespace hif {

namespace {

template <class F>
void parallel_for(int64_t n, F&& f) {
  unsigned hw = std::thread::hardware_concurrency();
  if (hw == 0) hw = 1;
  int64_t nt = std::min<int64_t>(hw, (n + 255) / 256);
  if (nt <= 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int64_t t = 0; t < nt; ++t) {
    th.emplace_back([&, t] {
      int64_t a = n * t / nt, b = n * (t + 1) / nt;
      for (int64_t i = a; i < b; ++i) f(i);
    });
  }
  for (auto& x : th) x.join();
}

// f(t, a, b) on nt contiguous chunks [a, b) of [0, n), in parallel; the
// chunks are in index order, so per-chunk results combine deterministically
template <class F>
int parallel_chunks(int64_t n, F&& f) {
  unsigned hw = std::thread::hardware_concurrency();
  if (hw == 0) hw = 1;
  const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(hw, n / 4096));
  if (nt == 1) {
    f(0, (int64_t)0, n);
    return 1;
  }
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] { f(t, n * t / nt, n * (t + 1) / nt); });
  for (auto& x : th) x.join();
  return nt;
}

inline int popc3(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1); }

}  // namespace

int hif_num_levels(int n, int m) {
  if (n <= 0 || m <= 0 || n % m) return -1;
  int q = n / m, L = 0;
  while ((1 << L) < q) ++L;
  return (1 << L) == q ? L : -1;
}

Symbolic::Symbolic(int n, int m, bool periodic)
    : n_(n), m_(m), L_(hif_num_levels(n, m)), periodic_(periodic) {
  active_.resize((size_t)n * n * n);
  for (size_t i = 0; i < active_.size(); ++i) active_[i] = (int32_t)i;
}

namespace {
// Boundary position in cell c (coordinates) of the DOF at active slot sl
// with packed geometry pk, or -1 if the cell's closure does not hold it.
inline int32_t pos_at(const CellPlan& cp, int32_t sl, int64_t pk, const int* c) {
  const int sep = (int)(pk >> 48);
  int q = 0;
  for (int d = 0; d < 3; ++d) {
    const int lc = (int)((pk >> (16 * d)) & 0xffff);
    if (c[d] == lc) continue;
    // the upper cell of a separator (wrapping on the periodic grid; with a
    // Dirichlet boundary lc + 1 < C always holds)
    if (((sep >> d) & 1) && c[d] == (lc + 1 == cp.C ? 0 : lc + 1)) {
      q |= 1 << d;
      continue;
    }
    return -1;
  }
  return cp.posB[(int64_t)sl * 8 + q];
}
}  // namespace

int32_t Symbolic::pos_in_cell(const CellPlan& cp, int32_t g, int cx, int cy, int cz) const {
  const int32_t sl = cp.slot[g];
  if (sl < 0) return -1;
  const int c[3] = {cx, cy, cz};
  return pos_at(cp, sl, cp.packed[sl], c);
}

void Symbolic::build_cells(int level, CellPlan& cp) const { build_cells_from(level, active_, cp); }

void Symbolic::filter_rows(SkelPlan& sp, const std::vector<uint8_t>& alive) const {
  SkelPlan out;
  filter_rows(sp, alive, out);
  sp = std::move(out);
}

void Symbolic::filter_rows(const SkelPlan& sp, const std::vector<uint8_t>& alive,
                           SkelPlan& out) const {
  const int ncp = sp.ncellPer;
  const int nf = sp.nfront;
  out.kind = sp.kind;
  out.ncellPer = sp.ncellPer;
  out.nfront = sp.nfront;
  out.cells = sp.cells;
  out.nF = sp.nF;
  out.nR.assign(nf, 0);
  std::vector<int64_t> kept(nf, 0);
  parallel_for(nf, [&](int64_t f) {
    int64_t k = 0;
    for (int64_t r = sp.rowOff[f]; r < sp.rowOff[f + 1]; ++r)
      if (r < sp.rowOff[f] + sp.nF[f] || alive[sp.rowDof[r]]) ++k;
    kept[f] = k;
  });
  std::vector<int64_t> off(nf + 1, 0);
  for (int f = 0; f < nf; ++f) off[f + 1] = off[f] + kept[f];
  PlanVec32 dof(off[nf]);
  PlanVec32 pos(off[nf] * ncp);
  parallel_for(nf, [&](int64_t f) {
    int64_t o = off[f];
    for (int64_t r = sp.rowOff[f]; r < sp.rowOff[f + 1]; ++r) {
      if (!(r < sp.rowOff[f] + sp.nF[f] || alive[sp.rowDof[r]])) continue;
      dof[o] = sp.rowDof[r];
      for (int i = 0; i < ncp; ++i) pos[o * ncp + i] = sp.rowPos[r * ncp + i];
      ++o;
    }
    out.nR[f] = (int32_t)(kept[f] - sp.nF[f]);
  });
  out.rowOff = std::move(off);
  out.rowDof = std::move(dof);
  out.rowPos = std::move(pos);
}

void Symbolic::build_cells_from(int level, const std::vector<int32_t>& active, CellPlan& cp) const {
  const int n = n_;
  const int s = m_ << level;
  const int C = n / s;
  const int64_t N = (int64_t)n * n * n;
  cp.level = level;
  cp.s = s;
  cp.C = C;
  cp.ncell = C * C * C;
  cp.active = active;
  const int64_t na = (int64_t)cp.active.size();
  cp.slot.resize(N);
  parallel_for(N, [&](int64_t g) { cp.slot[g] = -1; });
  cp.packed.resize(na);
  parallel_for(na, [&](int64_t i) {
    int32_t g = cp.active[i];
    cp.slot[g] = (int32_t)i;
    int x[3] = {g % n, (g / n) % n, g / (n * n)};
    int64_t pk = 0;
    int sep = 0;
    for (int d = 0; d < 3; ++d) {
      // periodic: the top level (one cell) has no separators; below it the
      // cell under plane 0 is the last one
      bool sd = periodic_ ? (level < L_ && x[d] % s == 0) : (x[d] != 0 && x[d] % s == 0);
      int lc = sd ? (x[d] / s + C - 1) % C : x[d] / s;
      if (sd) sep |= 1 << d;
      pk |= (int64_t)lc << (16 * d);
    }
    cp.packed[i] = pk | ((int64_t)sep << 48);
  });
  auto cell_of = [&](int64_t pk, int q) {
    int c0 = ((int)(pk & 0xffff) + (q & 1)) % C;
    int c1 = ((int)((pk >> 16) & 0xffff) + ((q >> 1) & 1)) % C;
    int c2 = ((int)((pk >> 32) & 0xffff) + ((q >> 2) & 1)) % C;
    return c0 + C * (c1 + C * c2);
  };
  // interior / boundary counts per cell, per chunk of the active list; the
  // chunks then fill the lists at their running offsets, so the lists keep
  // ascending global order within each part, as a sequential pass would
  unsigned hw = std::thread::hardware_concurrency();
  const int ntmax = (int)std::max<int64_t>(1, std::min<int64_t>(hw == 0 ? 1 : hw, na / 4096));
  std::vector<std::vector<int32_t>> cntI(ntmax), cntB(ntmax);
  const int nt = parallel_chunks(na, [&](int t, int64_t a, int64_t b) {
    std::vector<int32_t>& ci = cntI[t];
    std::vector<int32_t>& cb = cntB[t];
    ci.assign(cp.ncell, 0);
    cb.assign(cp.ncell, 0);
    for (int64_t i = a; i < b; ++i) {
      int64_t pk = cp.packed[i];
      int sep = (int)(pk >> 48);
      if (sep == 0) {
        ci[cell_of(pk, 0)]++;
      } else {
        for (int q = 0; q < 8; ++q)
          if ((q & ~sep) == 0) cb[cell_of(pk, q)]++;
      }
    }
  });
  cp.off.assign(cp.ncell + 1, 0);
  cp.p.assign(cp.ncell, 0);
  for (int c = 0; c < cp.ncell; ++c) {
    int32_t ti = 0, tb = 0;
    for (int t = 0; t < nt; ++t) {   // counts become each chunk's start within the cell
      const int32_t xi = cntI[t][c], xb = cntB[t][c];
      cntI[t][c] = ti;
      cntB[t][c] = tb;
      ti += xi;
      tb += xb;
    }
    cp.off[c + 1] = cp.off[c] + ti + tb;
    cp.p[c] = ti;
  }
  cp.dofs.resize(cp.off[cp.ncell]);
  cp.dofSlot.resize(cp.off[cp.ncell]);
  cp.dofPk.resize(cp.off[cp.ncell]);
  cp.posB.resize(na * 8);
  parallel_chunks(na, [&](int t, int64_t a, int64_t b) {
    std::vector<int32_t>& curI = cntI[t];
    std::vector<int32_t>& curB = cntB[t];
    for (int64_t i = a; i < b; ++i) {
      int64_t pk = cp.packed[i];
      int sep = (int)(pk >> 48);
      int32_t g = cp.active[i];
      int32_t* pb = &cp.posB[i * 8];
      for (int q = 0; q < 8; ++q) pb[q] = -1;
      if (sep == 0) {
        int c = cell_of(pk, 0);
        const int64_t e = cp.off[c] + curI[c]++;
        cp.dofs[e] = g;
        cp.dofSlot[e] = (int32_t)i;
        cp.dofPk[e] = pk;
      } else {
        for (int q = 0; q < 8; ++q) {
          if (q & ~sep) continue;
          int c = cell_of(pk, q);
          int bpos = curB[c]++;
          const int64_t e = cp.off[c] + cp.p[c] + bpos;
          cp.dofs[e] = g;
          cp.dofSlot[e] = (int32_t)i;
          cp.dofPk[e] = pk;
          pb[q] = bpos;
        }
      }
    }
  });
}

void Symbolic::merge_maps(const CellPlan& child, const CellPlan& parent,
                          std::vector<int64_t>& mapOff, PlanVec32& map) const {
  const int C = parent.C, Cc = child.C;
  mapOff.assign(parent.ncell + 1, 0);
  for (int c = 0; c < parent.ncell; ++c)
    mapOff[c + 1] = mapOff[c] + 8 * (parent.off[c + 1] - parent.off[c]);
  map.resize(mapOff[parent.ncell]);
  parallel_for(parent.ncell, [&](int64_t c) {
    int px = (int)(c % C), py = (int)((c / C) % C), pz = (int)(c / ((int64_t)C * C));
    int64_t o = parent.off[c];
    int64_t nn = parent.off[c + 1] - o;
    // each DOF's slot and geometry in the child plan are looked up once for
    // all 8 children
    int cc[8][3];
    bool has[8];
    for (int q = 0; q < 8; ++q) {
      cc[q][0] = 2 * px + (q & 1);
      cc[q][1] = 2 * py + ((q >> 1) & 1);
      cc[q][2] = 2 * pz + ((q >> 2) & 1);
      has[q] = cc[q][0] < Cc && cc[q][1] < Cc && cc[q][2] < Cc;
    }
    int32_t* out = &map[mapOff[c]];
    for (int64_t e = 0; e < 8 * nn; ++e) out[e] = -1;
    for (int64_t a = 0; a < nn; ++a) {
      const int32_t sl = child.slot[parent.dofs[o + a]];
      if (sl < 0) continue;
      const int64_t pk = child.packed[sl];
      for (int q = 0; q < 8; ++q)
        if (has[q]) out[(int64_t)q * nn + a] = pos_at(child, sl, pk, cc[q]);
    }
  });
}

void Symbolic::build_skel(const CellPlan& cp, int kind, const std::vector<uint8_t>& alive,
                          SkelPlan& sp) const {
  const int C = cp.C;
  const int64_t na = (int64_t)cp.active.size();
  sp.kind = kind;
  sp.ncellPer = kind == 1 ? 2 : 4;
  const int ncp = sp.ncellPer;
  // group id = sep mask (3 bits) * C^3 + low-cell index
  auto gkey = [&](int64_t pk) -> int64_t {
    int64_t c0 = pk & 0xffff, c1 = (pk >> 16) & 0xffff, c2 = (pk >> 32) & 0xffff;
    return (pk >> 48) * (int64_t)C * C * C + c0 + C * (c1 + C * c2);
  };
  // group id -> front number through a dense table (8 separator masks x C^3
  // low cells); fronts are numbered in order of their lowest global index
  const int64_t C3 = (int64_t)C * C * C;
  std::vector<int32_t> fid(8 * C3, -1);
  std::vector<int64_t> keys;
  std::vector<int32_t> fcount;
  std::vector<int32_t> front_of(na, -1);
  for (int64_t i = 0; i < na; ++i) {
    int32_t g = cp.active[i];
    if (!alive[g]) continue;
    int64_t pk = cp.packed[i];
    if (popc3((int)(pk >> 48)) != kind) continue;
    const int64_t k = gkey(pk);
    int32_t f = fid[k];
    if (f < 0) {
      f = (int32_t)keys.size();
      fid[k] = f;
      keys.push_back(k);
      fcount.push_back(0);
    }
    fcount[f]++;
    front_of[i] = f;
  }
  const int nf = (int)keys.size();
  // members of each front (ascending global index), CSR
  std::vector<int64_t> moff(nf + 1, 0);
  for (int f = 0; f < nf; ++f) moff[f + 1] = moff[f] + fcount[f];
  std::vector<int32_t> mem(moff[nf]);
  {
    std::vector<int64_t> cur(moff.begin(), moff.end() - 1);
    for (int64_t i = 0; i < na; ++i)
      if (front_of[i] >= 0) mem[cur[front_of[i]]++] = cp.active[i];
  }
  sp.nfront = nf;
  sp.cells.assign((size_t)nf * ncp, -1);
  sp.nF.assign(nf, 0);
  sp.nR.assign(nf, 0);
  // cells of each front: corners over its separator dimensions
  std::vector<int32_t> cellxyz((size_t)nf * ncp * 3);
  for (int f = 0; f < nf; ++f) {
    int64_t pk = cp.packed[cp.slot[mem[moff[f]]]];
    int sep = (int)(pk >> 48);
    int lc[3] = {(int)(pk & 0xffff), (int)((pk >> 16) & 0xffff), (int)((pk >> 32) & 0xffff)};
    int j = 0;
    for (int q = 0; q < 8; ++q) {
      if (q & ~sep) continue;
      int c[3] = {(lc[0] + (q & 1)) % C, (lc[1] + ((q >> 1) & 1)) % C, (lc[2] + ((q >> 2) & 1)) % C};
      sp.cells[(size_t)f * ncp + j] = c[0] + C * (c[1] + C * c[2]);
      for (int d = 0; d < 3; ++d) cellxyz[((size_t)f * ncp + j) * 3 + d] = c[d];
      ++j;
    }
  }
  // rows: the front's DOFs, then the alive boundary DOFs of its cells not in
  // the front, each once (first cell in corner order that holds it).
  // emit(g, pos) gets the row's position in each of the front's cells
  // (-1 = not in that cell); it is called with pos = nullptr when only the
  // count is wanted, which skips the positions after the first cell.
  auto for_rows = [&](int f, bool want_pos, auto&& emit) {
    const int64_t fk = keys[f];
    const int32_t* cx = &cellxyz[(size_t)f * ncp * 3];
    int32_t pos[4];
    for (int64_t u = moff[f]; u < moff[f + 1]; ++u) {
      const int32_t g = mem[u];
      if (want_pos) {
        const int32_t sl = cp.slot[g];
        const int64_t pk = cp.packed[sl];
        for (int j = 0; j < ncp; ++j) pos[j] = pos_at(cp, sl, pk, cx + 3 * j);
      }
      emit(g, pos);
    }
    for (int i = 0; i < ncp; ++i) {
      const int cell = sp.cells[(size_t)f * ncp + i];
      const int64_t o = cp.off[cell] + cp.p[cell], e = cp.off[cell + 1];
      for (int64_t t = o; t < e; ++t) {
        const int32_t g = cp.dofs[t];
        if (!alive[g]) continue;
        const int32_t sl = cp.dofSlot[t];
        const int64_t pk = cp.dofPk[t];
        if (gkey(pk) == fk) continue;
        bool earlier = false;
        for (int j = 0; j < i && !earlier; ++j) {
          pos[j] = pos_at(cp, sl, pk, cx + 3 * j);
          earlier = pos[j] >= 0;
        }
        if (earlier) continue;
        if (want_pos) {
          pos[i] = (int32_t)(t - o);
          for (int j = i + 1; j < ncp; ++j) pos[j] = pos_at(cp, sl, pk, cx + 3 * j);
        }
        emit(g, pos);
      }
    }
  };
  std::vector<int64_t> cnt(nf, 0);
  parallel_for(nf, [&](int64_t f) {
    int64_t c = 0;
    for_rows((int)f, false, [&](int32_t, const int32_t*) { ++c; });
    cnt[f] = c;
    sp.nF[f] = (int32_t)(moff[f + 1] - moff[f]);
    sp.nR[f] = (int32_t)(c - sp.nF[f]);
  });
  sp.rowOff.assign(nf + 1, 0);
  for (int f = 0; f < nf; ++f) sp.rowOff[f + 1] = sp.rowOff[f] + cnt[f];
  sp.rowDof.resize(sp.rowOff[nf]);
  sp.rowPos.resize(sp.rowOff[nf] * ncp);
  parallel_for(nf, [&](int64_t f) {
    int64_t r = sp.rowOff[f];
    for_rows((int)f, true, [&](int32_t g, const int32_t* pos) {
      sp.rowDof[r] = g;
      for (int i = 0; i < ncp; ++i) sp.rowPos[r * ncp + i] = pos[i];
      ++r;
    });
  });
}

}  // namespace hif
