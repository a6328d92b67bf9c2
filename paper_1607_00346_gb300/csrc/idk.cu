// Interpolative decomposition of A_RF for a batch of faces or edges (§2.3):
// column-pivoted Householder QR stopped at |R_ii| <= eps |R_11|, then
// T_F = R11^{-1} R12.  Three kernels, by the size of the front's matrix:
//   * k_cpqr_smem: the matrix fits one CTA's shared memory;
//   * k_cpqr_dsm: it fits the shared memory of a 2-16 CTA cluster;
//   * k_cpqr (below): the matrix stays in global memory and streams through
//     the cluster once per pivot step.
// k_cpqr_smem forms T itself; after the other two, k_id_solve_t forms T from
// the R they leave in the matrix (blocked back substitution, many CTAs per
// front).
//
// k_cpqr: one thread-block cluster per front (1 to 16 CTAs, chosen from the
// front's size and the batch).  Column j of the gather buffer belongs to CTA
// j % CS of the cluster and never moves: the pivot order is kept as a
// permutation.
//
// Blocked with deferred updates (the xLAQPS scheme of LAPACK's pivoted QR):
// within a block of NBK steps the remaining columns keep their block-start
// values; with V the block's reflectors and F(c,:) = tau-weighted products of
// column c with them, the current column is a_c - V F(c,:)^T.  Each step
//   1. every CTA proposes the largest remaining (downdated) column norm among
//      its columns; the proposals meet in distributed shared memory and every
//      CTA picks the same winner (largest norm, lowest column index on ties);
//   2. the owner of the pivot column brings it up to date, builds the
//      Householder reflector in place and the products g_l = v_l^T v_j;
//   3. every CTA computes F(c, j) = tau_j (v_j^T a_c - sum_l g_l F(c,l)) for
//      its remaining columns (one read of each column), updates row i of them
//      (their R entries) and downdates their norms.
// After the block, each CTA applies a_c -= V F(c,:)^T below the block to its
// columns (one read and one write per column).  So each step reads the
// trailing columns once instead of reading them twice and writing them.
//
// Reflectors and products run in the factor precision T.  Column norms are
// kept in double and downdated after every step (|a_j|^2 -= R_ij^2); when the
// downdate has lost most of the value the norm is recomputed from the current
// column (the LAPACK xGEQP3 safeguard).  Rows are never permuted, so R_{l,j}
// sits in row l of column j.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "front.cuh"
#include "tune.h"
#include "warp.cuh"

namespace cg = cooperative_groups;

namespace hif {

namespace {

constexpr int ID_THREADS = 512;
constexpr int ID_WARPS = ID_THREADS / 32;
constexpr int NBK = 16;   // steps per block of deferred updates
constexpr int RC = 128;   // rows of V staged in shared memory by the block update
constexpr int CPQR_SMEM_MAX = 200 * 1024;   // dynamic shared memory of k_cpqr, bytes
// Per-CTA state of its own columns, in dynamic shared memory (local index q
// of column c = rank + CS q): the downdated squared norm and its reference
// (double), the F row of the current block, and the step at which the column
// became a pivot (-1 while it remains).
template <typename T>
__host__ __device__ constexpr size_t cpqr_col_bytes() {
  return 2 * sizeof(double) + NBK * sizeof(T) + sizeof(int);
}

template <typename T>
__global__ void __launch_bounds__(ID_THREADS, 2) k_cpqr(SkelDesc* fr, const int* __restrict__ list,
                                                     T* Gar, int32_t* permAr, int32_t* stepAr,
                                                     double eps) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int fidx = list[blockIdx.x / CS];
  SkelDesc& fref = fr[fidx];
  const SkelDesc f = fref;
  const int nF = f.nF, m = f.idm, ld = f.idld;
  T* M = Gar + f.idoff;             // column c at M + c*ld
  int32_t* pv = permAr + f.perm;
  int32_t* stepOf = stepAr + f.perm;
  const int ncq = (nF + CS - 1) / CS;   // local columns (an upper bound for every rank)
  extern __shared__ __align__(16) unsigned char colsm[];
  double* nrm = reinterpret_cast<double*>(colsm);   // nrm[q]
  double* ref = nrm + ncq;
  T* Fm = reinterpret_cast<T*>(ref + ncq);          // F(c, l) at Fm[q*NBK + l]
  int* stepq = reinterpret_cast<int*>(Fm + (size_t)ncq * NBK);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  __shared__ double s_val[ID_WARPS];
  __shared__ int s_idx[ID_WARPS];
  __shared__ double s_cand_val;
  __shared__ int s_cand_idx;
  __shared__ double s_tau_own, s_v0_own;     // written by the pivot's owner
  __shared__ T s_g_own[NBK];                 // g_l = v_l^T v_j, written by the owner
  __shared__ T s_g[NBK];
  __shared__ T s_vrow[NBK];                  // V[i, l] of the current step
  __shared__ int s_pl[NBK];                  // pivot columns of the block
  __shared__ T s_v0[NBK], s_tau[NBK];
  __shared__ int s_piv, s_stop;
  __shared__ double s_r11;
  __shared__ T s_V[RC][NBK + 1];
  __shared__ T s_fp[NBK];

  for (int c = rank + CS * warp; c < nF; c += CS * ID_WARPS) {
    const double s = warp_sumsq(M + (int64_t)c * ld, 0, m, lane);
    if (lane == 0) {
      const int q = (c - rank) / CS;
      nrm[q] = s;
      ref[q] = s;
      stepq[q] = -1;
    }
  }
  __syncthreads();
  const int kmax = min(m, nF);
  int k = kmax;
  int i = 0;
  bool stopped = false;
  while (i < kmax && !stopped) {
    int jdone = 0;
    for (int j = 0; j < NBK && i < kmax; ++j) {
      // 1. proposals
      double bv = -1.0;
      int bi = nF;
      for (int c = rank + CS * tid; c < nF; c += CS * ID_THREADS) {
        const int q = (c - rank) / CS;
        if (stepq[q] >= 0) continue;
        const double v = nrm[q];
        if (v > bv || (v == bv && c < bi)) {
          bv = v;
          bi = c;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_val[warp] = bv;
        s_idx[warp] = bi;
      }
      __syncthreads();
      if (tid == 0) {
        double v = s_val[0];
        int ix = s_idx[0];
        for (int w = 1; w < ID_WARPS; ++w)
          if (s_val[w] > v || (s_val[w] == v && s_idx[w] < ix)) {
            v = s_val[w];
            ix = s_idx[w];
          }
        s_cand_val = v;
        s_cand_idx = ix;
      }
      cl.sync();
      if (warp == 0) {
        // lane q reads CTA q's proposal; a shuffle reduction picks the winner
        double v = -1.0;
        int ix = nF;
        if (lane < CS) {
          v = *cl.map_shared_rank(&s_cand_val, lane);
          ix = *cl.map_shared_rank(&s_cand_idx, lane);
        }
        for (int o = 16; o > 0; o >>= 1) {
          const double ov = __shfl_xor_sync(0xffffffffu, v, o);
          const int oi = __shfl_xor_sync(0xffffffffu, ix, o);
          if (ov > v || (ov == v && oi < ix)) {
            v = ov;
            ix = oi;
          }
        }
        if (lane == 0) {
          const double nv = sqrt(fmax(v, 0.0));
          if (i == 0) s_r11 = nv;
          s_stop = (ix >= nF) || ((i == 0) ? (nv == 0.0) : !(nv > eps * s_r11));
          s_piv = ix;
        }
      }
      __syncthreads();
      if (s_stop) {
        k = i;
        stopped = true;
        break;
      }
      const int piv = s_piv;
      const int owner = piv % CS;
      T* cp = M + (int64_t)piv * ld;
      // 2. the owner: bring the pivot column up to date, build the reflector
      if (owner == rank) {
        const int qp = (piv - rank) / CS;
        if (j > 0) {
          if (tid < NBK) s_fp[tid] = tid < j ? Fm[(int64_t)qp * NBK + tid] : T(0);
          __syncthreads();
          for (int r = i + tid; r < m; r += ID_THREADS) {
            T vv[NBK];
#pragma unroll
            for (int l = 0; l < NBK; ++l) vv[l] = l < j ? M[r + (int64_t)s_pl[l] * ld] : T(0);
            T a = cp[r];
#pragma unroll
            for (int l = 0; l < NBK; ++l) a = fma(-vv[l], s_fp[l], a);
            cp[r] = a;
          }
          __syncthreads();
        }
        double s = 0.0;
        for (int r = i + 1 + tid; r < m; r += ID_THREADS) {
          const double v = (double)cp[r];
          s += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) s_val[warp] = s;
        __syncthreads();
        if (tid == 0) {
          double tail = 0.0;
          for (int w = 0; w < ID_WARPS; ++w) tail += s_val[w];
          const double x0 = (double)cp[i];
          const double nx = sqrt(x0 * x0 + tail);
          const double alpha = x0 >= 0.0 ? -nx : nx;
          const double v0 = x0 - alpha;
          const double vtv = v0 * v0 + tail;
          s_tau_own = vtv > 0.0 ? 2.0 / vtv : 0.0;
          s_v0_own = v0;
          cp[i] = (T)alpha;    // R_ii; v0 lives in shared memory
          pv[i] = piv;
          stepq[qp] = i;
        }
        __syncthreads();
        // g_l = v_l^T v_j over rows i..m-1 (v_l is nonzero there, v_j starts at row i)
        const T v0 = (T)s_v0_own;
        for (int l = warp; l < j; l += ID_WARPS) {
          const T* vl = M + (int64_t)s_pl[l] * ld;
          T g = warp_dot(vl, cp, i + 1, m, lane);
          g = fma(vl[i], v0, g);
          if (lane == 0) s_g_own[l] = g;
        }
      }
      cl.sync();
      // 3. every CTA: the step's reflector scalars, then its own columns
      if (tid == 0) {
        s_pl[j] = piv;
        s_v0[j] = (T)*cl.map_shared_rank(&s_v0_own, owner);
        s_tau[j] = (T)*cl.map_shared_rank(&s_tau_own, owner);
      }
      if (tid < j) {
        s_g[tid] = *cl.map_shared_rank(&s_g_own[tid], owner);
        s_vrow[tid] = M[i + (int64_t)s_pl[tid] * ld];
      }
      __syncthreads();
      if (tid == 0) s_vrow[j] = s_v0[j];
      __syncthreads();
      const T v0 = s_v0[j], tau = s_tau[j];
      for (int c = rank + CS * warp; c < nF; c += CS * ID_WARPS) {
        const int q = (c - rank) / CS;
        if (stepq[q] >= 0) continue;
        T* cc = M + (int64_t)c * ld;
        T* Fc = Fm + (int64_t)q * NBK;
        T fl[NBK];
#pragma unroll
        for (int l = 0; l < NBK; ++l) fl[l] = l < j ? Fc[l] : T(0);
        const T aci = cc[i];
        T dot = warp_dot(cp, cc, i + 1, m, lane);
        dot = fma(v0, aci, dot);
        T corr = T(0), rv = aci;
#pragma unroll
        for (int l = 0; l < NBK; ++l) {
          if (l < j) {
            corr = fma(s_g[l], fl[l], corr);
            rv = fma(-s_vrow[l], fl[l], rv);
          }
        }
        const T fcj = tau * (dot - corr);
        rv = fma(-s_vrow[j], fcj, rv);
        __syncwarp();
        if (lane == 0) {
          Fc[j] = fcj;
          cc[i] = rv;
        }
        // downdate |a_c|^2 by R_ic^2 in double; recompute when mostly cancelled
        double nv = nrm[q] - (double)rv * (double)rv;
        if (nv <= 1e-2 * ref[q]) {
          double s = 0.0;
          for (int r = i + 1 + lane; r < m; r += 32) {
            T a = cc[r];
            for (int l = 0; l < j; ++l) a = fma(-M[r + (int64_t)s_pl[l] * ld], fl[l], a);
            a = fma(-cp[r], fcj, a);
            s += (double)a * (double)a;
          }
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          nv = s;
          if (lane == 0) ref[q] = s;
        }
        if (lane == 0) nrm[q] = fmax(nv, 0.0);
      }
      __syncthreads();
      ++i;
      jdone = j + 1;
    }
    // block update of my remaining columns below the block: a_c -= V F(c,:)^T
    if (!stopped && i < kmax && jdone > 0) {
      for (int r0 = i; r0 < m; r0 += RC) {
        const int rn = min(RC, m - r0);
        for (int e = tid; e < RC * NBK; e += ID_THREADS) {
          const int rr = e % RC, l = e / RC;
          s_V[rr][l] = (rr < rn && l < jdone) ? M[r0 + rr + (int64_t)s_pl[l] * ld] : T(0);
        }
        __syncthreads();
        for (int c = rank + CS * warp; c < nF; c += CS * ID_WARPS) {
          const int q = (c - rank) / CS;
          if (stepq[q] >= 0) continue;
          T* cc = M + (int64_t)c * ld;
          const T* Fc = Fm + (int64_t)q * NBK;
          T fl[NBK];
#pragma unroll
          for (int l = 0; l < NBK; ++l) fl[l] = l < jdone ? Fc[l] : T(0);
          for (int rr = lane; rr < rn; rr += 32) {
            T a = cc[r0 + rr];
#pragma unroll
            for (int l = 0; l < NBK; ++l) a = fma(-s_V[rr][l], fl[l], a);
            cc[r0 + rr] = a;
          }
        }
        __syncthreads();
      }
    }
  }
  // redundant columns, in increasing column order, follow the pivots in pv
  for (int c = rank + CS * tid; c < nF; c += CS * ID_THREADS) stepOf[c] = stepq[(c - rank) / CS];
  __threadfence();
  cl.sync();
  if (rank == 0 && tid == 0) {
    int t = k;
    for (int c = 0; c < nF; ++c)
      if (stepOf[c] < 0 || stepOf[c] >= k) pv[t++] = c;
    fref.k = k;
  }
  // T = R11^{-1} R12 follows in k_id_solve_t (R_{l,j} sits in row l of column pv[j])
}

// ---- fronts whose ID matrix fits in shared memory ---------------------------------
// One CTA per front: the idm x nF matrix is copied into shared memory and
// factored there by unblocked Householder QR with column pivoting.  Columns
// stay in place (ties go to the lowest column index, as in the cluster
// kernel).  The pass that applies step i's reflector to a column also
// recomputes, from the updated entries, the column's norm below row i + 1
// and its row i + 1 entry, and every warp keeps the best candidate among its
// columns; so each step needs a single barrier, and the norms involve no
// downdating (no cancellation), which lets them run in the factor precision
// (FP64 arithmetic is a small fraction of the FP32 rate on this part).
constexpr int SMEM_ID_MAX = 220 * 1024;   // dynamic shared memory per CTA, bytes

__host__ __device__ inline size_t smem_id_bytes(int m, int nF, int tsize) {
  // tail norms (T), R diagonal (T), done flags (int) + the matrix
  return (((size_t)nF * (2 * tsize + 4) + 15) / 16) * 16 + (size_t)m * nF * tsize;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_cpqr_smem(SkelDesc* fr, const int* __restrict__ list,
                                                    const T* __restrict__ Gar, int32_t* permAr,
                                                    T* Far, double eps) {
  const int fidx = list[blockIdx.x];
  SkelDesc& fref = fr[fidx];
  const SkelDesc f = fref;
  const int nF = f.nF, m = f.idm, ldg = f.idld;
  const T* Mg = Gar + f.idoff;
  int32_t* pv = permAr + f.perm;
  T* Tm = Far + f.Tm;
  extern __shared__ __align__(16) unsigned char sm[];
  T* tail = reinterpret_cast<T*>(sm);          // |a_c[i+1:]|^2 before step i
  T* rdiag = tail + nF;                        // R_ii
  int* done = reinterpret_cast<int*>(rdiag + nF);
  T* A = reinterpret_cast<T*>(sm + ((size_t)nF * (2 * sizeof(T) + 4) + 15) / 16 * 16);
  // per-warp candidates for the next pivot, |a_c[i:]|^2 and the column;
  // double-buffered by step parity so that one barrier per step suffices
  __shared__ T s_cv[2][32];
  __shared__ int s_ci[2][32];
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid / 32, lane = tid % 32, nw = nt / 32;

  // copy, and the norms for step 0
  {
    T bv = T(-1);
    int bc = nF;
    for (int c = warp; c < nF; c += nw) {
      const T* src = Mg + (int64_t)c * ldg;
      T* dst = A + (int64_t)c * m;
      T s = T(0), head = T(0);
      for (int r = lane; r < m; r += 32) {
        const T x = src[r];
        dst[r] = x;
        if (r == 0) head = x;
        else s = fma(x, x, s);
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      head = __shfl_sync(0xffffffffu, head, 0);
      const T full = fma(head, head, s);
      if (lane == 0) {
        tail[c] = s;
        done[c] = 0;
      }
      if (full > bv) {
        bv = full;
        bc = c;
      }
    }
    if (lane == 0) {
      s_cv[0][warp] = bv;
      s_ci[0][warp] = bc;
    }
  }
  __syncthreads();
  const int kmax = min(m, nF);
  int k = kmax;
  T r11 = T(0);
  for (int i = 0; i < kmax; ++i) {
    // pivot: the best of the warps' candidates (largest norm, lowest column)
    const int cur = i & 1;
    T bv = s_cv[cur][0];
    int p = s_ci[cur][0];
    for (int w = 1; w < nw; ++w) {
      const T v = s_cv[cur][w];
      const int c = s_ci[cur][w];
      if (v > bv || (v == bv && c < p)) {
        bv = v;
        p = c;
      }
    }
    const T nv = sqrt(fmax(bv, T(0)));
    if (i == 0) r11 = nv;
    if (p >= nF || (i == 0 ? nv == T(0) : !((double)nv > eps * (double)r11))) {
      k = i;
      break;
    }
    // reflector of column p over rows i..m-1: v = (x0 - alpha, a_p[i+1:])
    const T* ap = A + (int64_t)p * m;
    const T x0 = ap[i], tl = tail[p];
    const T nx = sqrt(fma(x0, x0, tl));
    const T alpha = x0 >= T(0) ? -nx : nx;
    const T v0 = x0 - alpha;
    const T vtv = fma(v0, v0, tl);
    const T tau = vtv > T(0) ? T(2) / vtv : T(0);
    if (tid == 0) {
      rdiag[i] = alpha;
      pv[i] = p;
    }
    // the other remaining columns: a_c -= tau v (v^T a_c)
    T cbv = T(-1);
    int cbc = nF;
    for (int c = warp; c < nF; c += nw) {
      if (c == p || done[c]) continue;
      T* ac = A + (int64_t)c * m;
      T w0 = T(0), w1 = T(0);
      int r = i + 1 + lane;
      for (; r + 32 < m; r += 64) {
        w0 = fma(ap[r], ac[r], w0);
        w1 = fma(ap[r + 32], ac[r + 32], w1);
      }
      if (r < m) w0 = fma(ap[r], ac[r], w0);
      T w = w0 + w1;
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      w = fma(v0, ac[i], w);
      const T tw = tau * w;
      T s = T(0), head = T(0);
      for (int r2 = i + 1 + lane; r2 < m; r2 += 32) {
        const T x = fma(-ap[r2], tw, ac[r2]);
        ac[r2] = x;
        if (r2 == i + 1) head = x;
        else s = fma(x, x, s);
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      head = __shfl_sync(0xffffffffu, head, 0);
      const T full = fma(head, head, s);
      __syncwarp();
      if (lane == 0) {
        ac[i] = fma(-v0, tw, ac[i]);   // R_ic
        tail[c] = s;
      }
      if (full > cbv) {
        cbv = full;
        cbc = c;
      }
    }
    if (lane == 0) {
      s_cv[cur ^ 1][warp] = cbv;
      s_ci[cur ^ 1][warp] = cbc;
    }
    if (tid == 0) done[p] = 1;
    __syncthreads();
  }
  if (tid == 0) fref.k = k;
  // T = R11^{-1} R12 (k x (nF-k), ld = k): one warp per redundant column,
  // back substitution in place in shared memory; R_{l,j} sits in row l of
  // column pv[j], R_jj in rdiag[j]; redundant columns follow the pivots in
  // increasing column order
  for (int c = warp; c < nF; c += nw) {
    if (done[c]) continue;
    int rk = 0;
    for (int q2 = 0; q2 < c; ++q2) rk += done[q2] == 0;
    T* b = A + (int64_t)c * m;
    for (int ii = k - 1; ii >= 0; --ii) {
      const T xi = b[ii] / rdiag[ii];
      const T* rc = A + (int64_t)pv[ii] * m;
      __syncwarp();
      if (lane == 0) b[ii] = xi;
      for (int r = lane; r < ii; r += 32) b[r] = fma(-xi, rc[r], b[r]);
      __syncwarp();
    }
    T* out = Tm + (int64_t)rk * k;
    for (int r = lane; r < k; r += 32) out[r] = b[r];
    if (lane == 0) pv[k + rk] = c;
  }
}

// ---- fronts whose ID matrix fits in the shared memory of one cluster ---------------
// One cluster of CS CTAs (1 to 16) per front.  Column c sits in the shared
// memory of CTA c % CS (local column c / CS) for the whole factorization, so
// the pivot steps read and write the matrix on chip instead of streaming it
// from L2 or HBM once per step.  Unblocked Householder QR with column
// pivoting, as in k_cpqr_smem: the tail norms are recomputed from the updated
// entries in the factor precision (no downdating), and the pivot is the
// largest norm, lowest column index on ties.  Each step:
//   1. a cluster barrier makes the CTAs' proposals for this step (their best
//      column with its norm, row-i entry and tail norm, pushed into every
//      CTA's shared memory) and their column updates of the last step visible;
//   2. every warp takes the winner among the CS proposals; every CTA copies
//      the pivot column's rows below the step from its owner into a local
//      buffer;
//   3. the warps share the CTA's remaining columns (a compacted list, so the
//      warps stay balanced as columns become pivots) and apply the reflector
//      to them: each column segment is read into registers as 16-byte
//      vectors, kept there between the dot product and the update, and
//      written back once; the reflector sits in registers for all of the
//      warp's columns; only the vectors that still hold rows below the step
//      are touched;
//   4. the warps' best columns meet in this CTA's proposal for the next step.
// The proposals are double-buffered by step parity, so one cluster barrier
// per step orders every exchange.  RPL rows per lane bound m (m <= 32 RPL).
// At the end each CTA writes rows 0..k-1 of its columns (R, with R_jj in row
// i of the column pivoted at step i) back to the matrix for k_id_solve_t.
// Fronts of 64-220 KB, which fit one CTA, run here with CS = 1 (the column
// passes from registers beat k_cpqr_smem's on them).
constexpr int DSM_THREADS = 512;
constexpr int DSM_WARPS = DSM_THREADS / 32;
constexpr int DSM_SMEM_MAX = 224 * 1024;   // dynamic shared memory per CTA, bytes
constexpr int DSM_MAX_CS = 16;

// rows of a column padded to whole 16-byte vectors
__host__ __device__ inline int dsm_ld(int m, int tsize) {
  const int ve = 16 / tsize;
  return (m + ve - 1) / ve * ve;
}

// dynamic shared memory of one CTA of a CS-CTA cluster: its columns (ncq x
// ldm), the pivot-column buffer (ldm), tail norms (ncq), R diagonal (kmax),
// pivot columns (kmax ints), the list of remaining local columns and their
// places in it (ncq ints each), and done flags (one byte per front column)
__host__ __device__ inline size_t dsm_id_bytes(int m, int nF, int CS, int tsize) {
  const size_t ncq = (size_t)((nF + CS - 1) / CS);
  const size_t kmax = (size_t)(m < nF ? m : nF);
  const size_t ldm = (size_t)dsm_ld(m, tsize);
  const size_t b = (ncq * ldm + ldm + ncq + kmax) * tsize + (kmax + 2 * ncq) * 4 + nF;
  return (b + 15) / 16 * 16;
}

// one 16-byte vector of shared memory <-> VE values
__device__ __forceinline__ void ld16(float (&x)[4], const float* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x[0] = v.x;
  x[1] = v.y;
  x[2] = v.z;
  x[3] = v.w;
}
__device__ __forceinline__ void ld16(double (&x)[2], const double* p) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  x[0] = v.x;
  x[1] = v.y;
}
__device__ __forceinline__ void st16(float* p, const float (&x)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
__device__ __forceinline__ void st16(double* p, const double (&x)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
}

template <typename T, int RPL>
__global__ void __launch_bounds__(DSM_THREADS, 1) k_cpqr_dsm(SkelDesc* fr, const int* __restrict__ list,
                                                          T* Gar, int32_t* permAr, double eps) {
  constexpr int VE = 16 / (int)sizeof(T);   // values per 16-byte vector
  constexpr int NV = RPL / VE;              // vectors per lane
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int fidx = list[blockIdx.x / CS];
  SkelDesc& fref = fr[fidx];
  const SkelDesc f = fref;
  const int nF = f.nF, m = f.idm, ldg = f.idld;
  T* Mg = Gar + f.idoff;
  int32_t* pv = permAr + f.perm;
  const int ncq = (nF + CS - 1) / CS;   // local columns (an upper bound on every rank)
  const int kmax = min(m, nF);
  const int ldm = dsm_ld(m, (int)sizeof(T)), nvc = ldm / VE;
  extern __shared__ __align__(16) unsigned char dsm[];
  T* A = reinterpret_cast<T*>(dsm);              // local column q at A + q ldm
  T* vbuf = A + (size_t)ncq * ldm;               // pivot column, row r at vbuf[r]
  T* tail = vbuf + ldm;                          // |a_c[i+1:]|^2 of local column q
  T* rdiag = tail + ncq;                         // R_ii
  int* pvl = reinterpret_cast<int*>(rdiag + kmax);   // pivot column of step i
  int* lst = pvl + kmax;                             // remaining local columns
  int* lpos = lst + ncq;                             // place of local column q in lst
  unsigned char* done = reinterpret_cast<unsigned char*>(lpos + ncq);   // per front column
  __shared__ T s_wv[DSM_WARPS], s_wh[DSM_WARPS], s_wt[DSM_WARPS];
  __shared__ int s_wc[DSM_WARPS];
  // the CTAs' proposals, by step parity and CTA: norm, column, row-i entry,
  // tail norm (each CTA writes its own slot in every CTA of the cluster)
  __shared__ T s_qv[2][DSM_MAX_CS], s_qh[2][DSM_MAX_CS], s_qt[2][DSM_MAX_CS];
  __shared__ int s_qc[2][DSM_MAX_CS];
  __shared__ int s_nrem;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  constexpr int nw = DSM_WARPS;

  // the warps' candidates -> this CTA's proposal (largest norm, lowest
  // column), pushed to every CTA of the cluster
  auto propose = [&](int par, T cbv, int cbc, T cbh, T cbt) {
    if (lane == 0) {
      s_wv[warp] = cbv;
      s_wc[warp] = cbc;
      s_wh[warp] = cbh;
      s_wt[warp] = cbt;
    }
    __syncthreads();
    if (warp == 0) {
      T v = T(-1), h = T(0), t = T(0);
      int c = nF;
      if (lane < nw) {
        v = s_wv[lane];
        c = s_wc[lane];
        h = s_wh[lane];
        t = s_wt[lane];
      }
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oc = __shfl_xor_sync(0xffffffffu, c, o);
        const T oh = __shfl_xor_sync(0xffffffffu, h, o);
        const T ot = __shfl_xor_sync(0xffffffffu, t, o);
        if (ov > v || (ov == v && oc < c)) {
          v = ov;
          c = oc;
          h = oh;
          t = ot;
        }
      }
      if (lane < CS) {
        *cl.map_shared_rank(&s_qv[par][rank], lane) = v;
        *cl.map_shared_rank(&s_qc[par][rank], lane) = c;
        *cl.map_shared_rank(&s_qh[par][rank], lane) = h;
        *cl.map_shared_rank(&s_qt[par][rank], lane) = t;
      }
    }
  };

  // copy the local columns in (zero rows up to ldm), and the norms for step 0
  for (int e = tid; e < nF; e += DSM_THREADS) done[e] = 0;
  for (int e = tid; e < ncq; e += DSM_THREADS) {
    lst[e] = e;
    lpos[e] = e;
  }
  if (tid == 0) s_nrem = max(0, (nF - rank + CS - 1) / CS);   // columns rank, rank + CS, ...
  {
    T bv = T(-1), bh = T(0), bt = T(0);
    int bc = nF;
    for (int q = warp; q < ncq; q += nw) {
      const int c = rank + CS * q;
      if (c >= nF) break;
      const T* src = Mg + (int64_t)c * ldg;
      T* dst = A + (size_t)q * ldm;
      T s = T(0), head = T(0);
      for (int r = lane; r < ldm; r += 32) {
        const T x = r < m ? src[r] : T(0);
        dst[r] = x;
        if (r == 0) head = x;
        else s = fma(x, x, s);
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      head = __shfl_sync(0xffffffffu, head, 0);
      const T full = fma(head, head, s);
      if (lane == 0) tail[q] = s;
      if (full > bv) {
        bv = full;
        bc = c;
        bh = head;
        bt = s;
      }
    }
    for (int r = m + tid; r < ldm; r += DSM_THREADS) vbuf[r] = T(0);
    cl.sync();   // every CTA of the cluster runs before the first proposal is pushed
    propose(0, bv, bc, bh, bt);
  }
  int k = kmax;
  T r11 = T(0);
  for (int i = 0; i < kmax; ++i) {
    const int cur = i & 1;
    cl.sync();
    // 2. the pivot: the best of the CTAs' proposals (every warp, same result)
    T bv = T(-1), x0 = T(0), tl = T(0);
    int p = nF;
    if (lane < CS) {
      bv = s_qv[cur][lane];
      p = s_qc[cur][lane];
      x0 = s_qh[cur][lane];
      tl = s_qt[cur][lane];
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oc = __shfl_xor_sync(0xffffffffu, p, o);
      const T oh = __shfl_xor_sync(0xffffffffu, x0, o);
      const T ot = __shfl_xor_sync(0xffffffffu, tl, o);
      if (ov > bv || (ov == bv && oc < p)) {
        bv = ov;
        p = oc;
        x0 = oh;
        tl = ot;
      }
    }
    const T nv = sqrt(fmax(bv, T(0)));
    if (i == 0) r11 = nv;
    if (p >= nF || (i == 0 ? nv == T(0) : !((double)nv > eps * (double)r11))) {
      k = i;
      break;
    }
    // reflector of column p over rows i..m-1: v = (x0 - alpha, a_p[i+1:])
    const T nx = sqrt(fma(x0, x0, tl));
    const T alpha = x0 >= T(0) ? -nx : nx;
    const T v0 = x0 - alpha;
    const T vtv = fma(v0, v0, tl);
    const T tau = vtv > T(0) ? T(2) / vtv : T(0);
    const int owner = p % CS, qp = p / CS;
    {
      // whole 16-byte vectors from the one holding row i + 1 (rows above it
      // are masked below; the column's padding rows are zero)
      const T* src = cl.map_shared_rank(A + (size_t)qp * ldm, owner);
      for (int g = (i + 1) / VE + tid; g < nvc; g += DSM_THREADS) {
        T x[VE];
        ld16(x, src + (size_t)g * VE);
        st16(vbuf + (size_t)g * VE, x);
      }
    }
    if (tid == 0) {
      rdiag[i] = alpha;
      pvl[i] = p;
      done[p] = 1;
      if (owner == rank) {   // drop the pivot from the remaining columns
        const int at = lpos[qp], last = lst[s_nrem - 1];
        lst[at] = last;
        lpos[last] = at;
        --s_nrem;
      }
    }
    __syncthreads();
    // 3. the remaining local columns: a_c -= tau v (v^T a_c), new tail norms;
    //    vectors b0 + lane + 32 t (t < tmax) hold the rows from i + 1 on, the
    //    first lo rows of vector b0 lie above them
    const int b0 = (i + 1) / VE, lo = i + 1 - VE * b0;
    const int tmax = (nvc - b0 + 31) / 32;
    T vr[NV][VE];
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int g = b0 + lane + 32 * t;
      if (t < tmax && g < nvc) {
        ld16(vr[t], vbuf + (size_t)g * VE);
      } else {
#pragma unroll
        for (int e = 0; e < VE; ++e) vr[t][e] = T(0);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int e = 0; e < VE; ++e)
        if (e < lo) vr[0][e] = T(0);
    }
    T cbv = T(-1), cbh = T(0), cbt = T(0);
    int cbc = nF;
    const int nrem = s_nrem;
    for (int li = warp; li < nrem; li += nw) {
      const int q = lst[li];
      const int c = rank + CS * q;
      T* ac = A + (size_t)q * ldm;
      T ar[NV][VE];
#pragma unroll
      for (int t = 0; t < NV; ++t) {
        const int g = b0 + lane + 32 * t;
        if (t < tmax && g < nvc) {
          ld16(ar[t], ac + (size_t)g * VE);
        } else {
#pragma unroll
          for (int e = 0; e < VE; ++e) ar[t][e] = T(0);
        }
      }
      const T aci = ac[i];
      T acc[VE];
#pragma unroll
      for (int e = 0; e < VE; ++e) acc[e] = T(0);
#pragma unroll
      for (int t = 0; t < NV; ++t) {
        if (t >= tmax) break;
#pragma unroll
        for (int e = 0; e < VE; ++e) acc[e] = fma(vr[t][e], ar[t][e], acc[e]);
      }
      T w = acc[0];
#pragma unroll
      for (int e = 1; e < VE; ++e) w += acc[e];
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      w = fma(v0, aci, w);
      const T tw = tau * w;
      T sacc[VE];
#pragma unroll
      for (int e = 0; e < VE; ++e) sacc[e] = T(0);
      T head = T(0);
#pragma unroll
      for (int t = 0; t < NV; ++t) {
        if (t >= tmax) break;
        T x[VE];
#pragma unroll
        for (int e = 0; e < VE; ++e) x[e] = fma(-vr[t][e], tw, ar[t][e]);
        if (t == 0) {
          // lane 0: rows above i + 1 keep their values, row i + 1 is the head
#pragma unroll
          for (int e = 0; e < VE; ++e) {
            const bool above = lane == 0 && e < lo, hd = lane == 0 && e == lo;
            if (above) x[e] = ar[0][e];
            if (hd) head = x[e];
            if (!above && !hd) sacc[e] = fma(x[e], x[e], sacc[e]);
          }
        } else {
#pragma unroll
          for (int e = 0; e < VE; ++e) sacc[e] = fma(x[e], x[e], sacc[e]);
        }
        const int g = b0 + lane + 32 * t;
        if (g < nvc) st16(ac + (size_t)g * VE, x);
      }
      T s = sacc[0];
#pragma unroll
      for (int e = 1; e < VE; ++e) s += sacc[e];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      head = __shfl_sync(0xffffffffu, head, 0);
      const T full = fma(head, head, s);
      __syncwarp();
      if (lane == 0) {
        ac[i] = fma(-v0, tw, aci);   // R_ic
        tail[q] = s;
      }
      if (full > cbv || (full == cbv && c < cbc)) {
        cbv = full;
        cbc = c;
        cbh = head;
        cbt = s;
      }
    }
    // 4. this CTA's proposal for step i + 1
    propose(cur ^ 1, cbv, cbc, cbh, cbt);
  }
  // the last step's copies and proposals are done: from here on no CTA
  // touches another's shared memory (so each may leave when it is done)
  cl.sync();
  if (rank == 0) {
    if (tid == 0) fref.k = k;
    for (int e = tid; e < k; e += DSM_THREADS) pv[e] = pvl[e];
  }
  // R back to the matrix in global memory, for k_id_solve_t: rows 0..k-1 of
  // every local column (R_{l,j} in row l of column pvl[j]), with R_jj in row j
  // of the local pivot columns; the redundant columns follow the pivots in
  // increasing column order
  for (int e = tid; e < k; e += DSM_THREADS)
    if (pvl[e] % CS == rank) A[(size_t)(pvl[e] / CS) * ldm + e] = rdiag[e];
  __syncthreads();
  for (int q = warp; q < ncq; q += nw) {
    const int c = rank + CS * q;
    if (c >= nF) break;
    T* dst = Mg + (int64_t)c * ldg;
    const T* src = A + (size_t)q * ldm;
    for (int r = lane; r < k; r += 32) dst[r] = src[r];
  }
  const int nred = s_nrem;
  for (int li = warp; li < nred; li += nw) {
    const int c = rank + CS * lst[li];
    int rk = 0;
    for (int c2 = lane; c2 < c; c2 += 32) rk += done[c2] == 0;
    for (int o = 16; o > 0; o >>= 1) rk += __shfl_xor_sync(0xffffffffu, rk, o);
    if (lane == 0) pv[k + rk] = c;
  }
}


// ---- T = R11^{-1} R12 for the fronts of the cluster kernels --------------------------
// Blocked back substitution, one CTA per front and block of NC redundant
// columns, after the ID kernel has left R in the matrix (R_{l,j} in row l of
// column pv[j]; the redundant columns are pv[k..nF-1]).  The block of R12 (k
// rows) sits in shared memory; from the last block of 32 rows up, the 32 x 32
// diagonal block of R11 is solved for every column (a warp per column, lanes
// over rows), then the solved rows update the rows above them (a thread per
// row with its NC sums in registers, R11 read from the matrix, the solved
// rows read from shared memory as 16-byte vectors).  Factor precision.
constexpr int TS_THREADS = 256;
constexpr int TS_SMEM_MAX = 200 * 1024;

template <typename T, int NC>
__host__ __device__ constexpr int ts_pitch() {
  return NC + 16 / (int)sizeof(T);   // row pitch of the block: 16-byte rows
}

template <typename T, int NC>
__global__ void __launch_bounds__(TS_THREADS) k_id_solve_t(const SkelDesc* __restrict__ fr,
                                                           const int* __restrict__ list, int cbpf,
                                                           const T* __restrict__ Gar,
                                                           const int32_t* __restrict__ permAr,
                                                           T* Far) {
  constexpr int VE = 16 / (int)sizeof(T);
  constexpr int BP = ts_pitch<T, NC>();
  const int fidx = list[blockIdx.x / cbpf];
  const int cb = (int)(blockIdx.x % cbpf);
  const SkelDesc f = fr[fidx];
  const int nF = f.nF, k = f.k, ld = f.idld;
  const int nr = nF - k, t0 = cb * NC;
  if (k == 0 || t0 >= nr) return;
  const int nc = min(NC, nr - t0);
  const T* M = Gar + f.idoff;
  const int32_t* pv = permAr + f.perm;
  T* Tm = Far + f.Tm;
  extern __shared__ __align__(16) unsigned char tsm[];
  T* B = reinterpret_cast<T*>(tsm);   // B[r BP + c]: row r < k of the block's column c
  __shared__ T s_D[32][33];           // diagonal block of R11
  __shared__ int s_pc[32];            // its columns
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  constexpr int nw = TS_THREADS / 32;
  for (int c = warp; c < NC; c += nw) {
    const T* src = M + (int64_t)pv[k + t0 + min(c, nc - 1)] * ld;
    for (int r = lane; r < k; r += 32) B[(size_t)r * BP + c] = c < nc ? src[r] : T(0);
  }
  for (int r0 = ((k - 1) / 32) * 32; r0 >= 0; r0 -= 32) {
    const int rn = min(32, k - r0);
    __syncthreads();   // the last block's updates are done
    if (tid < 32) s_pc[tid] = pv[r0 + min(tid, rn - 1)];
    __syncthreads();
    for (int e = tid; e < 32 * 32; e += TS_THREADS) {
      const int i = e % 32, j = e / 32;
      s_D[i][j] = (i < rn && j < rn && i <= j) ? M[(r0 + i) + (int64_t)s_pc[j] * ld] : T(0);
    }
    __syncthreads();
    // D X = B[r0 : r0 + rn, :]
    for (int c = warp; c < nc; c += nw) {
      T b = lane < rn ? B[(size_t)(r0 + lane) * BP + c] : T(0);
      for (int j = rn - 1; j >= 0; --j) {
        const T xj = __shfl_sync(0xffffffffu, b, j) / s_D[j][j];
        if (lane == j) b = xj;
        else if (lane < j) b = fma(-xj, s_D[lane][j], b);
      }
      if (lane < rn) B[(size_t)(r0 + lane) * BP + c] = b;
    }
    __syncthreads();
    // the rows above: B[r, :] -= sum_j R_{r, r0 + j} X[j, :]
    for (int r = tid; r < r0; r += TS_THREADS) {
      T acc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = B[(size_t)r * BP + c];
      for (int j = 0; j < rn; ++j) {
        const T rv = M[r + (int64_t)s_pc[j] * ld];
        const T* x = B + (size_t)(r0 + j) * BP;
#pragma unroll
        for (int c = 0; c < NC; c += VE) {
          T xv[VE];
          ld16(xv, x + c);
#pragma unroll
          for (int e = 0; e < VE; ++e) acc[c + e] = fma(-rv, xv[e], acc[c + e]);
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) B[(size_t)r * BP + c] = acc[c];
    }
  }
  __syncthreads();
  for (int c = warp; c < nc; c += nw) {
    T* dst = Tm + (int64_t)(t0 + c) * k;
    for (int r = lane; r < k; r += 32) dst[r] = B[(size_t)r * BP + c];
  }
}

// k_cpqr_dsm's rows per lane for a front of m rows (0: too tall for it); the
// widest class holds 64 registers of column data per lane, which FP64 fronts
// would spill
inline int dsm_rows_per_lane(int m, int tsize) {
  return m <= 256 ? 8 : m <= 512 ? 16 : (m <= 1024 && tsize == 4) ? 32 : 0;
}

// the smallest cluster whose CTAs' shared memory holds the front (0: none)
inline int dsm_min_cluster(int m, int nF, int tsize, int cs_from = 2) {
  for (int cs = cs_from; cs <= DSM_MAX_CS; ++cs)
    if (dsm_id_bytes(m, nF, cs, tsize) <= (size_t)DSM_SMEM_MAX) return cs;
  return 0;
}

template <typename T, int RPL>
void dsm_attributes() {
  static const bool set = [] {
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_cpqr_dsm<T, RPL>,
                                      cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_cpqr_dsm<T, RPL>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, DSM_SMEM_MAX));
    return true;
  }();
  (void)set;
}

// whether clusters of CS CTAs with `smem` bytes of dynamic shared memory each
// can be placed on this GPU (asked once per shape)
template <typename T, int RPL>
bool dsm_placeable(int CS, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, bool> known;
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_pair(CS, smem);
  const auto it = known.find(key);
  if (it != known.end()) return it->second;
  dsm_attributes<T, RPL>();
  cudaLaunchConfig_t q = {};
  q.gridDim = dim3((unsigned)CS);
  q.blockDim = dim3(DSM_THREADS);
  q.dynamicSmemBytes = smem;
  cudaLaunchAttribute qa[1];
  qa[0].id = cudaLaunchAttributeClusterDimension;
  qa[0].val.clusterDim.x = CS;
  qa[0].val.clusterDim.y = 1;
  qa[0].val.clusterDim.z = 1;
  q.attrs = qa;
  q.numAttrs = 1;
  int ncl = 0;
  const bool ok = cudaOccupancyMaxActiveClusters(&ncl, k_cpqr_dsm<T, RPL>, &q) == cudaSuccess && ncl > 0;
  cudaGetLastError();
  known[key] = ok;
  return ok;
}

// one launch of k_cpqr_dsm over `fronts` (all of one rows-per-lane class):
// the smallest cluster (at least cs_min CTAs) that holds each of them and can
// be placed; false if there is none (the caller takes the fronts elsewhere)
template <typename T, int RPL>
bool launch_cpqr_dsm(const std::vector<int>& fronts, const SkelDesc* h_f, SkelDesc* d_f, T* G,
                     int32_t* perm, double eps, int cs_min, cudaStream_t st) {
  if (fronts.empty()) return true;
  int CS = std::max(1, cs_min);
  for (int f : fronts)
    CS = std::max(CS, dsm_min_cluster(h_f[f].idm, h_f[f].nF, (int)sizeof(T), std::max(1, cs_min)));
  for (; CS <= DSM_MAX_CS; ++CS) {
    size_t smem = 0;
    for (int f : fronts)
      smem = std::max(smem, dsm_id_bytes(h_f[f].idm, h_f[f].nF, CS, (int)sizeof(T)));
    smem = (smem + 4095) / 4096 * 4096;
    if (smem > (size_t)DSM_SMEM_MAX || !dsm_placeable<T, RPL>(CS, smem)) continue;
    int* d_list = nullptr;
    HIF_CUDA_TRY(cudaMallocAsync(&d_list, sizeof(int) * fronts.size(), st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_list, fronts.data(), sizeof(int) * fronts.size(),
                                 cudaMemcpyHostToDevice, st));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(fronts.size() * CS));
    cfg.blockDim = dim3(DSM_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    {
      ProfScope ps("id_cpqr_dsm", st);   // counts added by the caller (they need k)
      HIF_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_cpqr_dsm<T, RPL>, d_f, (const int*)d_list, G, perm,
                                      eps));
      HIF_CHECK_LAUNCH();
    }
    HIF_CUDA_TRY(cudaFreeAsync(d_list, st));
    return true;
  }
  return false;
}
}  // namespace


template <typename T>
void interpolative_decomposition(SkelDesc* d_f, const SkelDesc* h_f, int nf, T* Garena,
                                 size_t arena_elems, int32_t* perm, T* Farena, int32_t* stepAr,
                                 double eps, cudaStream_t st, int8_t* route) {
  if (nf == 0) return;
  int nsm = 0, dev = 0;
  HIF_CUDA_TRY(cudaGetDevice(&dev));
  HIF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // fronts whose matrix fits in shared memory: one CTA each, in three size
  // classes (128, 256 or 1024 threads; dynamic shared memory of the class's
  // largest front)
  // once per precision; a function-local static is initialised once even
  // when several host threads factor at the same time
  static const bool smem_attr = [] {
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_cpqr_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      SMEM_ID_MAX));
    return true;
  }();
  (void)smem_attr;
  constexpr size_t class_max[3] = {16 * 1024, 64 * 1024, (size_t)SMEM_ID_MAX};
  constexpr int class_threads[3] = {128, 256, 1024};
  std::vector<int> small[3], rest;
  size_t small_bytes[3] = {0, 0, 0};
  // fronts of the widest one-CTA class go to k_cpqr_dsm on one CTA when
  // they fit it (its column passes hold the column in registers as 16-byte
  // vectors)
  std::vector<int> one[3];
  for (int f = 0; f < nf; ++f) {
    const size_t by = smem_id_bytes(h_f[f].idm, h_f[f].nF, (int)sizeof(T));
    int cl = 0;
    while (cl < 3 && by > class_max[cl]) ++cl;
    const int rpl = dsm_rows_per_lane(h_f[f].idm, (int)sizeof(T));
    if (cl == 2 && rpl > 0 &&
        dsm_id_bytes(h_f[f].idm, h_f[f].nF, 1, (int)sizeof(T)) <= (size_t)DSM_SMEM_MAX) {
      one[rpl == 8 ? 0 : rpl == 16 ? 1 : 2].push_back(f);
    } else if (cl == 3) {
      rest.push_back(f);
    } else {
      small[cl].push_back(f);
      small_bytes[cl] = std::max(small_bytes[cl], by);
      if (route) route[f] = ID_ROUTE_SMEM;
    }
  }
  for (int cl = 0; cl < 3; ++cl) {
    if (small[cl].empty()) continue;
    int* d_list = nullptr;
    HIF_CUDA_TRY(cudaMallocAsync(&d_list, sizeof(int) * small[cl].size(), st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_list, small[cl].data(), sizeof(int) * small[cl].size(),
                                 cudaMemcpyHostToDevice, st));
    {
      ProfScope ps("id_cpqr_smem", st);   // counts added by the caller (they need k)
      k_cpqr_smem<T><<<(unsigned)small[cl].size(), class_threads[cl], small_bytes[cl], st>>>(
          d_f, d_list, Garena, perm, Farena, eps);
      HIF_CHECK_LAUNCH();
    }
    HIF_CUDA_TRY(cudaFreeAsync(d_list, st));
  }
  {
    bool placed[3] = {launch_cpqr_dsm<T, 8>(one[0], h_f, d_f, Garena, perm, eps, 1, st),
                      launch_cpqr_dsm<T, 16>(one[1], h_f, d_f, Garena, perm, eps, 1, st), true};
    if constexpr (sizeof(T) == 4)
      placed[2] = launch_cpqr_dsm<T, 32>(one[2], h_f, d_f, Garena, perm, eps, 1, st);
    for (int c = 0; c < 3; ++c)
      for (int f : one[c]) {
        if (placed[c]) {
          if (route) route[f] = ID_ROUTE_CLUSTER_SMEM;
        } else {
          rest.push_back(f);   // not expected: a one-CTA cluster always fits
        }
      }
  }
  // fronts that fit the shared memory of one cluster: k_cpqr_dsm, one launch
  // per rows-per-lane class; the rest (and any class whose cluster cannot be
  // placed) go to the streaming cluster kernel
  {
    std::vector<int> dsm[3], keep;
    for (int f : rest) {
      const int rpl = dsm_rows_per_lane(h_f[f].idm, (int)sizeof(T));
      if (rpl > 0 && dsm_min_cluster(h_f[f].idm, h_f[f].nF, (int)sizeof(T)) > 0)
        dsm[rpl == 8 ? 0 : rpl == 16 ? 1 : 2].push_back(f);
      else
        keep.push_back(f);
    }
    bool placed[3] = {launch_cpqr_dsm<T, 8>(dsm[0], h_f, d_f, Garena, perm, eps, 2, st),
                      launch_cpqr_dsm<T, 16>(dsm[1], h_f, d_f, Garena, perm, eps, 2, st),
                      true};   // the widest class is FP32 only
    if constexpr (sizeof(T) == 4)
      placed[2] = launch_cpqr_dsm<T, 32>(dsm[2], h_f, d_f, Garena, perm, eps, 2, st);
    for (int c = 0; c < 3; ++c)
      for (int f : dsm[c]) {
        if (placed[c]) {
          if (route) route[f] = ID_ROUTE_CLUSTER_SMEM;
        } else {
          keep.push_back(f);
        }
      }
    rest.swap(keep);
  }
  if (route)
    for (int f : rest) route[f] = ID_ROUTE_STREAM;
  if (rest.empty()) return;
  static const bool attr_set = [] {
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_cpqr<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_cpqr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      CPQR_SMEM_MAX));
    return true;
  }();
  (void)attr_set;
  // the largest cluster of at most b CTAs that the GPU can place
  static int placeable[17] = {0};
  static std::once_flag place_once;
  std::call_once(place_once, [] {
    for (int b = 1; b <= 16; ++b) {
      int CS = b;
      while (CS > 1) {
        cudaLaunchConfig_t q = {};
        q.gridDim = dim3((unsigned)CS);
        q.blockDim = dim3(ID_THREADS);
        cudaLaunchAttribute qa[1];
        qa[0].id = cudaLaunchAttributeClusterDimension;
        qa[0].val.clusterDim.x = CS;
        qa[0].val.clusterDim.y = 1;
        qa[0].val.clusterDim.z = 1;
        q.attrs = qa;
        q.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, k_cpqr<T>, &q) == cudaSuccess && ncl > 0) break;
        cudaGetLastError();
        --CS;
      }
      placeable[b] = CS;
    }
  });
  // one launch per chunk of `wave` fronts (0: all), clusters of CS CTAs
  auto launch = [&](const std::vector<int>& fronts, int CS, int wave, SkelDesc* df, T* arena) {
    CS = placeable[std::max(1, std::min(16, CS))];
    const int w = wave > 0 ? wave : (int)fronts.size();
    for (size_t f0 = 0; f0 < fronts.size(); f0 += (size_t)w) {
      const int cnt = (int)std::min<size_t>((size_t)w, fronts.size() - f0);
      int nfm = 1;
      for (int q = 0; q < cnt; ++q) nfm = std::max(nfm, h_f[fronts[f0 + q]].nF);
      // the CTAs' column state must fit their shared memory (a wider
      // cluster if not); a cluster that cannot be placed with it shrinks
      auto smem_for = [&](int cs) { return (size_t)((nfm + cs - 1) / cs) * cpqr_col_bytes<T>(); };
      while (CS < 16 && smem_for(CS) > (size_t)CPQR_SMEM_MAX) CS = placeable[std::min(16, 2 * CS)];
      size_t smem = 0;
      for (;;) {
        smem = smem_for(CS);
        if (smem > (size_t)CPQR_SMEM_MAX)
          throw Error{HIF_ERR_INVALID_ARG, "interpolative decomposition front too wide"};
        if (CS == 1) break;
        cudaLaunchConfig_t q = {};
        q.gridDim = dim3((unsigned)CS);
        q.blockDim = dim3(ID_THREADS);
        q.dynamicSmemBytes = smem;
        cudaLaunchAttribute qa[1];
        qa[0].id = cudaLaunchAttributeClusterDimension;
        qa[0].val.clusterDim.x = CS;
        qa[0].val.clusterDim.y = 1;
        qa[0].val.clusterDim.z = 1;
        q.attrs = qa;
        q.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, k_cpqr<T>, &q) == cudaSuccess && ncl > 0) break;
        cudaGetLastError();
        --CS;
      }
      int* d_list = nullptr;
      HIF_CUDA_TRY(cudaMallocAsync(&d_list, sizeof(int) * cnt, st));
      HIF_CUDA_TRY(cudaMemcpyAsync(d_list, fronts.data() + f0, sizeof(int) * cnt,
                                   cudaMemcpyHostToDevice, st));
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(cnt * CS));
      cfg.blockDim = dim3(ID_THREADS);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = CS;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      {
        ProfScope ps("id_cpqr", st);
        HIF_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_cpqr<T>, df, (const int*)d_list, arena, perm,
                                        stepAr, eps));
        HIF_CHECK_LAUNCH();
      }
      HIF_CUDA_TRY(cudaFreeAsync(d_list, st));
    }
  };
  // built-in rule: small fronts get one CTA; large fronts (work per step
  // nF x nR above ~1e6) spread their columns over as many SMs as the batch
  // leaves free (two CTAs per SM), up to 16, at least 8 columns per CTA
  int nbig = 0;
  for (int f : rest)
    if ((double)h_f[f].nF * (h_f[f].nF + h_f[f].idm) > 1.0e6) ++nbig;
  const int cs_big = std::max(1, std::min(16, 2 * nsm / std::max(1, nbig)));
  // one bucket per call: the width class of its widest cluster front and the
  // count class of its cluster fronts; one shape (cluster size, fronts per
  // launch) for all of them, the cluster size capped per front at nF / 8
  // CTAs; fronts with the same effective shape share launches
  int nfmax = 0, nfmin = 1 << 30;
  size_t maxbytes = 0;
  for (int f : rest) {
    nfmax = std::max(nfmax, h_f[f].nF);
    nfmin = std::min(nfmin, h_f[f].nF);
    maxbytes = std::max(maxbytes, sizeof(T) * (size_t)h_f[f].idm * h_f[f].nF);
  }
  const int wcls = id_width_class(nfmax), ccls = id_count_class((int)rest.size());
  auto run_all = [&](int cs_choice, int wave, SkelDesc* df, T* arena) {
    std::map<int, std::vector<int>> by_cs;
    for (int f : rest) {
      int cs = cs_choice;
      if (cs <= 0) {   // built-in rule
        const double work = (double)h_f[f].nF * (h_f[f].nF + h_f[f].idm);
        cs = work > 1.0e6 ? cs_big : 1;
      }
      by_cs[std::min(cs, std::max(1, h_f[f].nF / 8))].push_back(f);
    }
    for (auto& [cs, fronts] : by_cs) launch(fronts, cs, wave, df, arena);
  };
  IdChoice tuned;
  if (!tune_id_lookup(wcls, ccls, &tuned) && tune_session_active() && arena_elems > 0) {
    // time the candidate shapes in place: every run starts from a copy of
    // the matrices and descriptors as they are now (the ID overwrites them)
    T* pristine = nullptr;
    T* work = nullptr;
    SkelDesc* dwork = nullptr;
    HIF_CUDA_TRY(cudaMallocAsync(&pristine, sizeof(T) * arena_elems, st));
    HIF_CUDA_TRY(cudaMallocAsync(&work, sizeof(T) * arena_elems, st));
    HIF_CUDA_TRY(cudaMallocAsync(&dwork, sizeof(SkelDesc) * nf, st));
    HIF_CUDA_TRY(cudaMemcpyAsync(pristine, Garena, sizeof(T) * arena_elems, cudaMemcpyDeviceToDevice, st));
    cudaEvent_t e0, e1;
    HIF_CUDA_TRY(cudaEventCreate(&e0));
    HIF_CUDA_TRY(cudaEventCreate(&e1));
    // fronts resident in L2 together (129 MB, with room to spare)
    const int l2fit = (int)std::max<size_t>(1, (size_t)(96u << 20) / std::max<size_t>(1, maxbytes));
    std::vector<int> waves = {0};
    if (l2fit < (int)rest.size()) waves.push_back(l2fit);
    std::vector<std::pair<IdChoice, double>> tried;
    double best = 1e30;
    for (int cs : {0, 1, 2, 4, 8, 16}) {   // 0: the built-in rule
      if (cs > 1 && (cs > nfmin / 8 || placeable[cs] != cs)) continue;
      if (cs > 0 && (size_t)((nfmax + cs - 1) / cs) * cpqr_col_bytes<T>() > (size_t)CPQR_SMEM_MAX)
        continue;
      for (int wv : waves) {
        HIF_CUDA_TRY(cudaMemcpyAsync(work, pristine, sizeof(T) * arena_elems, cudaMemcpyDeviceToDevice, st));
        HIF_CUDA_TRY(cudaMemcpyAsync(dwork, d_f, sizeof(SkelDesc) * nf, cudaMemcpyDeviceToDevice, st));
        HIF_CUDA_TRY(cudaEventRecord(e0, st));
        run_all(cs, wv, dwork, work);
        HIF_CUDA_TRY(cudaEventRecord(e1, st));
        HIF_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        HIF_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        tried.push_back({IdChoice{cs, wv}, 1e-3 * ms});
        if (ms < best) {
          best = ms;
          tuned.cs = cs;
          tuned.wave = wv;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    HIF_CUDA_TRY(cudaFreeAsync(dwork, st));
    HIF_CUDA_TRY(cudaFreeAsync(work, st));
    HIF_CUDA_TRY(cudaFreeAsync(pristine, st));
    tune_id_set(wcls, ccls, tuned, tried);
  }
  run_all(tuned.cs, tuned.wave, d_f, Garena);
}

template void interpolative_decomposition<float>(SkelDesc*, const SkelDesc*, int, float*, size_t,
                                                 int32_t*, float*, int32_t*, double, cudaStream_t,
                                                 int8_t*);
template void interpolative_decomposition<double>(SkelDesc*, const SkelDesc*, int, double*,
                                                  size_t, int32_t*, double*, int32_t*, double,
                                                  cudaStream_t, int8_t*);


template <typename T>
void id_solve_t(const SkelDesc* d_f, const SkelDesc* h_f, const std::vector<int>& fronts,
                const T* Garena, const int32_t* perm, T* Farena, cudaStream_t st) {
  if (fronts.empty()) return;
  int kmax = 1, nrmax = 1;
  for (int f : fronts) {
    kmax = std::max(kmax, h_f[f].k);
    nrmax = std::max(nrmax, h_f[f].nF - h_f[f].k);
  }
  auto bytes = [&](int pitch) { return (size_t)kmax * pitch * sizeof(T); };
  int* d_list = nullptr;
  HIF_CUDA_TRY(cudaMallocAsync(&d_list, sizeof(int) * fronts.size(), st));
  HIF_CUDA_TRY(cudaMemcpyAsync(d_list, fronts.data(), sizeof(int) * fronts.size(),
                               cudaMemcpyHostToDevice, st));
  auto run = [&](auto kern, int nc, size_t smem) {
    static std::mutex mu;
    std::lock_guard<std::mutex> g(mu);
    HIF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TS_SMEM_MAX));
    const int cbpf = ceil_div(nrmax, nc);
    // k^2 (nF - k) flops; R11 and R12 read, T written
    double fl = 0.0, by = 0.0;
    if (prof_enabled())
      for (int f : fronts) {
        const double k = h_f[f].k, nr = h_f[f].nF - h_f[f].k;
        fl += k * k * nr;
        by += sizeof(T) * (0.5 * k * k + 2.0 * k * nr);
      }
    ProfScope ps("id_solve_t", st, fl, by);
    kern<<<(unsigned)(fronts.size() * cbpf), TS_THREADS, smem, st>>>(d_f, d_list, cbpf, Garena,
                                                                     perm, Farena);
    HIF_CHECK_LAUNCH();
  };
  if (bytes(ts_pitch<T, 32>()) <= (size_t)TS_SMEM_MAX)
    run(k_id_solve_t<T, 32>, 32, bytes(ts_pitch<T, 32>()));
  else if (bytes(ts_pitch<T, 16>()) <= (size_t)TS_SMEM_MAX)
    run(k_id_solve_t<T, 16>, 16, bytes(ts_pitch<T, 16>()));
  else if (bytes(ts_pitch<T, 8>()) <= (size_t)TS_SMEM_MAX)
    run(k_id_solve_t<T, 8>, 8, bytes(ts_pitch<T, 8>()));
  else if (bytes(ts_pitch<T, 4>()) <= (size_t)TS_SMEM_MAX)
    run(k_id_solve_t<T, 4>, 4, bytes(ts_pitch<T, 4>()));
  else
    throw Error{HIF_ERR_INVALID_ARG, "interpolative decomposition rank too large"};
  HIF_CUDA_TRY(cudaFreeAsync(d_list, st));
}

template void id_solve_t<float>(const SkelDesc*, const SkelDesc*, const std::vector<int>&,
                                const float*, const int32_t*, float*, cudaStream_t);
template void id_solve_t<double>(const SkelDesc*, const SkelDesc*, const std::vector<int>&,
                                 const double*, const int32_t*, double*, cudaStream_t);

}  // namespace hif
