// Host-side symbolic pass of the HIF level loop: which DOFs form each front.
//
// Geometry (§2.1, read for a zero Dirichlet boundary): at level l the cell
// side is s = m 2^l; coordinate x is a separator iff x % s == 0 and x != 0.
// On the periodic grid every multiple of s below the top level is a
// separator (x = 0 included, each cell owning its first frame as in §2.1)
// and cell indices wrap: the cell below plane 0 is the last one.
// A DOF with 0 / 1 / 2 / 3 separator coordinates is a cell-interior / face /
// edge / vertex point.  The lowest cell holding coordinate x along a dimension
// is x/s - 1 for a separator and x/s otherwise; a separator coordinate also
// lies in the next cell.  So a DOF lies in the closure of up to 8 cells,
// numbered by a 3-bit "corner" (bit d set = the higher cell along dimension d).
//
// Each cell of a level keeps a dense frontal matrix over its closure: the
// active interior DOFs first (eliminated by the cell step, §2.2), then the
// active boundary DOFs.  The matrix of the level is the sum of the cells'
// frontal matrices, so faces and edges (skeletonized in §2.3) read their
// blocks by summing over the 2 or 4 cells that hold them.
#pragma once

#include <stdint.h>

#include <memory>
#include <new>
#include <utility>
#include <vector>

namespace hif {

// Allocator whose value-less construct leaves the element uninitialized: the
// large plan arrays are written in full by parallel loops, so zero-filling
// them first on one thread would only cost time (and touch every page from
// that thread).
template <class T>
struct DefaultInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = DefaultInitAlloc<U>;
  };
  DefaultInitAlloc() = default;
  template <class U>
  DefaultInitAlloc(const DefaultInitAlloc<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... Args>
  void construct(U* p, Args&&... args) {
    ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
  }
};
using PlanVec32 = std::vector<int32_t, DefaultInitAlloc<int32_t>>;

struct CellPlan {
  int level = 0, s = 0, C = 0;   // cell side, cells per dimension
  int ncell = 0;
  std::vector<int32_t> active;   // sorted global ids active at the start of the level
  PlanVec32 slot;                // global id -> index in `active`, -1 if inactive
  std::vector<int64_t> off;      // per cell offset into dofs (ncell + 1)
  PlanVec32 dofs;                // frontal lists: interior, then boundary
  PlanVec32 dofSlot;             // per dofs entry: its active slot
  std::vector<int64_t, DefaultInitAlloc<int64_t>> dofPk;   // per dofs entry: its packed geometry
  std::vector<int32_t> p;        // interior count per cell
  PlanVec32 posB;                // per active slot, 8 corners: position in that cell's boundary list
  std::vector<int64_t> packed;   // per active slot: low cells (3 x 16 bit) | separator mask << 48
};

struct SkelPlan {
  int kind = 0;                  // 1 = faces, 2 = edges
  int ncellPer = 0;              // 2 for faces, 4 for edges
  int nfront = 0;
  std::vector<int32_t> cells;    // nfront * ncellPer cell ids
  std::vector<int32_t> nF, nR;   // front size and number of coupled rows
  std::vector<int64_t> rowOff;   // per front offset into rowDof (nfront + 1)
  PlanVec32 rowDof;              // global ids: the front's DOFs first, then R
  PlanVec32 rowPos;              // per row, ncellPer boundary positions (-1 = absent)
};

class Symbolic {
 public:
  Symbolic(int n, int m, bool periodic = false);
  int n() const { return n_; }
  int m() const { return m_; }
  int levels() const { return L_; }
  bool periodic() const { return periodic_; }

  // Build the cell plan of `level` from the current active set.
  void build_cells(int level, CellPlan& cp) const;
  // Merge maps from the children (plan `child`, level l-1) into `parent`
  // (level l): for each parent cell, 8 x n_parent entries (child corner q
  // major) giving the child's boundary position of the parent's DOF, or -1.
  void merge_maps(const CellPlan& child, const CellPlan& parent,
                  std::vector<int64_t>& mapOff, PlanVec32& map) const;
  // Faces (kind 1) or edges (kind 2) of the level with their coupled rows.
  // `alive` marks DOFs still active (redundant DOFs of faces are dropped
  // before the edges are planned).
  void build_skel(const CellPlan& cp, int kind, const std::vector<uint8_t>& alive,
                  SkelPlan& sp) const;

  // Drop the R rows whose DOF is no longer alive (the plan keeps its order),
  // in place or into a new plan.
  void filter_rows(SkelPlan& sp, const std::vector<uint8_t>& alive) const;
  void filter_rows(const SkelPlan& sp, const std::vector<uint8_t>& alive, SkelPlan& out) const;
  // build_cells from an explicit active list (sorted global ids).
  void build_cells_from(int level, const std::vector<int32_t>& active, CellPlan& cp) const;

  // Position of global DOF g in the boundary list of cell (cx,cy,cz) of plan cp.
  int32_t pos_in_cell(const CellPlan& cp, int32_t g, int cx, int cy, int cz) const;

  void set_active(std::vector<int32_t> act) { active_ = std::move(act); }
  const std::vector<int32_t>& active() const { return active_; }

 private:
  int n_, m_, L_;
  bool periodic_;
  std::vector<int32_t> active_;
};

// L with n = m 2^L, or -1.
int hif_num_levels(int n, int m);

}  // namespace hif
