// Kernels that move matrix entries between the fronts of the level loop.
#pragma once

#include "common.cuh"

namespace hif {

// Per-cell frontal matrix of a level: K (n x n, ld = n) at offset K of the arena.
struct CellDesc {
  int64_t K;
  int64_t list;   // offset of the frontal DOF list (global ids) in the level's index array
  int n;
  int p;          // interior count; the boundary block K' = K[p:n, p:n]
};

// Seven-point operator (§2.4): coupling to +e_d neighbours and diagonal.
// cpl[d*N + j] = a_{j+e_d/2}/h^2 (Dirichlet: 0 on the last plane; periodic:
// the coupling to the first plane), diag[j] = sum/h^2 + b_j.  *d_bad is set
// for a <= 0, b < 0 (b <= 0 when periodic) or non-finite values.
void stencil_coefficients(const double* a, const double* b, double b_const, int n, int periodic,
                          double* cpl, double* diag, int* d_bad, cudaStream_t st);

// Level-0 frontal matrices from the stencil (each coupling counted in exactly
// one cell: the lowest cell whose closure holds both points).
template <typename T>
void assemble_level0(const CellDesc* d_cells, int ncell, const int32_t* lists, int n, int s,
                     int periodic,
                     const double* cpl, const double* diag, T* Karena, int maxbox,
                     cudaStream_t st);

// Parent frontal matrices as the sum of the children's boundary blocks.
struct MergeDesc {
  int64_t K;        // parent K offset
  int64_t map;      // offset of 8 x n maps (child corner major)
  int n;
  int child[8];     // child cell index in the previous level's table (-1 = none)
};
template <typename T>
void merge_children(const MergeDesc* d_par, const MergeDesc* h_par, int npar,
                    const CellDesc* d_child, const int32_t* maps, const T* Kchild,
                    T* Kpar, cudaStream_t st);

// Skeleton front (face: 2 cells, edge: 4 cells).
struct SkelDesc {
  int64_t G;        // offset of the (nF+nR) x nF gather buffer (ld = nF + nR)
  int64_t rows;     // offset of its rows in rowPos (times ncellPer)
  int64_t Z;        // offset of the nF x nF frontal matrix (ld = nF)
  int64_t P;        // factor panel offset (nF x p)
  int64_t Tm;       // offset of T (k x p, ld = k) in the factor arena
  int64_t perm;     // offset of the nF-entry permutation
  int nF, nR;
  int k;            // rank (skeleton count) found by the ID
  int cell[4];
  // matrix the ID factors: idm x nF at offset idoff (ld = idld) of the arena
  // given to the ID; either the R rows of the gather buffer (idm = nR) or the
  // triangular factor of their unpivoted QR (idm = nF)
  int64_t idoff;
  int idm, idld;
};
// the kernel that took a front's ID: the streaming cluster kernel (matrix in
// global memory), one CTA with the matrix in its shared memory, or a cluster
// with the matrix spread over its CTAs' shared memory
enum : int8_t { ID_ROUTE_STREAM = 0, ID_ROUTE_SMEM = 1, ID_ROUTE_CLUSTER_SMEM = 2 };
template <typename T>
void skel_gather(const SkelDesc* d_f, const SkelDesc* h_f, int nf, int ncp,
                 const int32_t* rowPos, const CellDesc* d_cells, const T* Karena, T* Garena,
                 cudaStream_t st);
// Z = A_FF permuted to (redundant, skeleton) order.
template <typename T>
void skel_permute(const SkelDesc* d_f, const SkelDesc* h_f, int nf, const int32_t* perm,
                  const T* Garena, T* Zarena, cudaStream_t st);
// B_{F^F^} (trailing block of Z) into the first cell's boundary block; zero in the others.
template <typename T>
void skel_writeback(const SkelDesc* d_f, const SkelDesc* h_f, int nf, int ncp,
                    const int32_t* rowPos, const int32_t* perm, const CellDesc* d_cells,
                    const T* Zarena, T* Karena, cudaStream_t st);

}  // namespace hif
