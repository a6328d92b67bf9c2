// Interpolative decomposition of A_RF for a batch of faces or edges (§2.3):
// column-pivoted Householder QR stopped at |R_ii| <= eps |R_11|, then
// T_F = R11^{-1} R12.
//
// One thread-block cluster per front (1 to 16 CTAs, chosen from the front's
// size and the batch).  Column j of the gather buffer belongs to CTA j % CS of
// the cluster and never moves: the pivot order is kept as a permutation.
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
                                                     T* Gar, int32_t* permAr, T* Far,
                                                     int32_t* stepAr, double eps) {
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
  cl.sync();
  // T = R11^{-1} R12 (k x (nF-k), ld = k): column-oriented back substitution,
  // one warp per redundant column
  T* Tm = Far + f.Tm;
  for (int t = rank + CS * warp; t < nF - k; t += CS * ID_WARPS) {
    T* b = Tm + (int64_t)t * k;
    const T* cj = M + (int64_t)pv[k + t] * ld;
    for (int r = lane; r < k; r += 32) b[r] = cj[r];
    __syncwarp();
    for (int ii = k - 1; ii >= 0; --ii) {
      const T* rc = M + (int64_t)pv[ii] * ld;   // R[0:ii+1, ii] lives in column pv[ii]
      const T xi = b[ii] / rc[ii];
      __syncwarp();
      if (lane == 0) b[ii] = xi;
      for (int r = lane; r < ii; r += 32) b[r] = fma(-xi, rc[r], b[r]);
      __syncwarp();
    }
  }
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

}  // namespace


bool id_in_shared_memory(int m, int nF, int tsize) {
  return smem_id_bytes(m, nF, tsize) <= (size_t)SMEM_ID_MAX;
}

template <typename T>
void interpolative_decomposition(SkelDesc* d_f, const SkelDesc* h_f, int nf, T* Garena,
                                 size_t arena_elems, int32_t* perm, T* Farena, int32_t* stepAr,
                                 double eps, cudaStream_t st) {
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
  for (int f = 0; f < nf; ++f) {
    const size_t by = smem_id_bytes(h_f[f].idm, h_f[f].nF, (int)sizeof(T));
    int cl = 0;
    while (cl < 3 && by > class_max[cl]) ++cl;
    if (cl == 3) {
      rest.push_back(f);
    } else {
      small[cl].push_back(f);
      small_bytes[cl] = std::max(small_bytes[cl], by);
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
                                        Farena, stepAr, eps));
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
                                                 int32_t*, float*, int32_t*, double, cudaStream_t);
template void interpolative_decomposition<double>(SkelDesc*, const SkelDesc*, int, double*,
                                                  size_t, int32_t*, double*, int32_t*, double,
                                                  cudaStream_t);

}  // namespace hif
