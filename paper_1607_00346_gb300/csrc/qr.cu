// Row reduction before the interpolative decomposition of large fronts.
//
// The ID of A_RF (§2.3) depends on A_RF only through the norms of the linear
// combinations of its columns: with A_RF = Q R (Q orthonormal, R square upper
// triangular) ||A_RF x|| = ||R x|| for every x, so column-pivoted QR of R makes
// the same pivots and the same R factor as column-pivoted QR of A_RF.  For a
// front with many more coupled rows than DOFs (the faces of the upper levels:
// ~10^4 rows for ~10^3 columns) R is computed first by an unpivoted blocked
// Householder QR, whose work is in batched matrix products, and the pivoted QR
// then runs on the small square R.
//
// Blocked Householder QR, panel by panel (32 columns):
//   * the panel: Householder reflectors of its columns, the explicit
//     reflector matrix V and the triangular T of the compact form
//     Q = I - V T V^T (forward accumulation: T_{j+1} = [T_j, -tau_j T_j
//     V_j^T v_j; 0, tau_j]); k_qr_panel_cluster keeps the panel in the shared
//     memory of a cluster (row slices, one exchange per column), k_qr_panel
//     (one CTA per front, the panel in global memory, norms in double) takes
//     panels too tall for 16 CTAs;
//   * the columns right of the panel inside its 128-column block: W = T^T
//     V^T A and A -= V W, two kernels that stream those columns once each
//     (k_qr_w1/k_qr_w2, k_qr_update);
//   * after a block's last panel, the columns right of the block, once per
//     block, by tensor-core products: G = V^T V, the block's T from G and
//     the panels' tau (k_qr_tblk), W' = V^T A_t, W = T^T W', A_t -= V W.
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "dense.cuh"
#include "front.cuh"
#include "warp.cuh"

#include <cooperative_groups.h>

namespace hif {

namespace cg = cooperative_groups;

namespace {

constexpr int QB = 32;          // panel width
constexpr int QB2 = 128;        // block width: trailing columns are updated once per block

// Panel p (32 columns) of the block starting at p0 keeps its reflectors in
// the block's V (rows relative to p0, ld = m): column p - p0 on, row p - p0 on,
// so V(r, j) of the panel (r relative to p) sits at V + voff + r + j m; its T
// is the ((p - p0) / 32)-th 32 x 32 matrix of the block's four.
__host__ __device__ inline int64_t qr_voff(int p, int p0, int m) { return (int64_t)(p - p0) * (m + 1); }
__host__ __device__ inline int64_t qr_toff(int p, int p0) { return (int64_t)((p - p0) / QB) * QB * QB; }
constexpr int QR_THREADS = 512;
constexpr int QR_WARPS = QR_THREADS / 32;

struct QRDesc {
  int64_t A;     // matrix (m x n, ld) offset in the gather arena
  int64_t V;     // reflector block (m x QB, ld = m) offset in the V arena
  int64_t W;     // QB x n work block (ld = QB) offset in the W arena
  int64_t Tt;    // QB x QB offset in the T arena
  int m, n, ld;
  int pad;
};

template <typename T>
__global__ void __launch_bounds__(QR_THREADS) k_qr_panel(const QRDesc* __restrict__ ds, T* Gar,
                                                         T* Var, T* Tar, int p, int p0) {
  const QRDesc d = ds[blockIdx.x];
  if (p >= d.n) return;
  const int jb = min(QB, d.n - p);
  const int m = d.m, ld = d.ld;
  T* A = Gar + d.A;
  T* V = Var + d.V + qr_voff(p, p0, m);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  __shared__ double s_red[QR_WARPS];
  __shared__ double s_tau[QB], s_v0[QB];
  __shared__ double s_G[QB][QB + 1];
  __shared__ double s_T[QB][QB + 1];
  for (int j = 0; j < jb; ++j) {
    const int c = p + j;
    T* col = A + (int64_t)c * ld;
    // tail norm: warps take interleaved row chunks
    double s = 0.0;
    {
      const int span = (m - c - 1 + QR_WARPS - 1) / QR_WARPS;
      const int r0 = c + 1 + warp * span, r1 = min(m, r0 + span);
      if (r0 < r1) s = warp_sumsq(col, r0, r1, lane);
    }
    if (lane == 0) s_red[warp] = s;
    __syncthreads();
    if (tid == 0) {
      double tail = 0.0;
      for (int w = 0; w < QR_WARPS; ++w) tail += s_red[w];
      const double x0 = (double)col[c];
      const double nx = sqrt(x0 * x0 + tail);
      const double alpha = x0 >= 0.0 ? -nx : nx;
      const double v0 = x0 - alpha;
      const double vtv = v0 * v0 + tail;
      s_tau[j] = vtv > 0.0 ? 2.0 / vtv : 0.0;
      s_v0[j] = v0;
      col[c] = (T)alpha;          // R_cc; v0 lives in shared memory
    }
    __syncthreads();
    const T v0 = (T)s_v0[j], tau = (T)s_tau[j];
    // explicit reflector column j of V (rows p0..m-1 of the block's V)
    for (int r = p0 + tid; r < m; r += QR_THREADS)
      V[(r - p) + (int64_t)j * m] = r < c ? T(0) : (r == c ? v0 : col[r]);
    // the rest of the panel
    for (int jj = j + 1 + warp; jj < jb; jj += QR_WARPS) {
      T* a = A + (int64_t)(p + jj) * ld;
      T w = warp_dot(col, a, c + 1, m, lane);
      w = fma(v0, a[c], w);
      const T tw = tau * w;
      warp_axpy(tw, col, a, c + 1, m, lane);
      __syncwarp();
      if (lane == 0) a[c] = fma(-tw, v0, a[c]);
    }
    __syncthreads();
  }
  // Gram matrix of the reflectors, then T column by column
  for (int e = warp; e < jb * jb; e += QR_WARPS) {
    const int a = e % jb, b = e / jb;
    if (a > b) continue;
    const T* va = V + (int64_t)a * m;
    const T* vb = V + (int64_t)b * m;
    const double s = (double)warp_dot(va, vb, 0, m - p, lane);
    if (lane == 0) {
      s_G[a][b] = s;
      s_G[b][a] = s;
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < jb; ++j) {
      for (int i = 0; i < QB; ++i) s_T[i][j] = 0.0;
      s_T[j][j] = s_tau[j];
      for (int i = 0; i < j; ++i) {
        double t = 0.0;
        for (int l = i; l < j; ++l) t += s_T[i][l] * s_G[l][j];
        s_T[i][j] = -s_tau[j] * t;
      }
    }
  }
  __syncthreads();
  T* Tt = Tar + d.Tt + qr_toff(p, p0);
  for (int e = tid; e < QB * QB; e += QR_THREADS) {
    const int i = e % QB, j = e / QB;
    Tt[e] = (i < jb && j < jb) ? (T)s_T[i][j] : T(0);
  }
}

// The same panel factorization spread over a thread-block cluster: the
// panel's active rows (p..m-1) are split into CS contiguous slices held in
// the shared memory of the cluster's CTAs.  One exchange per column: before
// column j is reduced, every CTA holds its slice's parts (rows below j) of
// the tail norm |a_j|^2, of the products a_j^T a_jj with the remaining panel
// columns (jj > j) and of v_l^T a_j with the earlier reflectors (l < j), and
// pushes them into every CTA's shared memory (the owner of row j also pushes
// that row).  After one cluster barrier every CTA adds the CS parts in the
// same order and forms the same reflector, the same w_jj = v^T a_jj =
// v0 a_jj[j] + (a_j^T a_jj below j) and the same column j of T
// (T[0:j, j] = -tau_j T[0:j, 0:j] V^T v_j, with v_l^T v_j = v_l[j] v0 +
// (v_l^T a_j below j); the products are kept and T is formed once after the
// column loop).  The pass that then updates the slice (a_jj -= tau w_jj v)
// also takes the parts for column j + 1 from the updated entries; each row is
// read in two halves whose loads are in flight together.  Per column: one
// cluster barrier, two CTA barriers, one read and write of the slice; the
// parts are double-buffered by column parity.  Sums run in the factor
// precision (FP64 arithmetic is slow here).
constexpr int QRC_MAX_CS = 16;
constexpr int QRC_MAX_WARPS = 16;
// threads per CTA: 512 in FP32; 256 in FP64 (each thread keeps 32 partial
// sums and half a row of the panel in registers)
template <typename T>
__host__ __device__ constexpr int qrc_threads() {
  return sizeof(T) == 4 ? 512 : 256;
}

template <typename T>
__global__ void __launch_bounds__(qrc_threads<T>()) k_qr_panel_cluster(const QRDesc* __restrict__ ds,
                                                                      T* Gar, T* Var, T* Tar,
                                                                      int p, int p0, int rb) {
  constexpr int QRC_THREADS = qrc_threads<T>();
  constexpr int QRC_WARPS = QRC_THREADS / 32;
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const QRDesc d = ds[blockIdx.x / CS];
  if (p >= d.n) return;   // the whole cluster returns (same front)
  const int jb = min(QB, d.n - p);
  const int m = d.m, ld = d.ld, mp = m - p;
  const int r0 = rank * rb, r1 = min(mp, r0 + rb);   // this CTA's rows, relative to p
  T* A = Gar + d.A;
  T* V = Var + d.V + qr_voff(p, p0, m);
  extern __shared__ __align__(16) unsigned char qsm[];
  T* P = reinterpret_cast<T*>(qsm);                  // slice: P[i + j rb], i = row - p - r0
  // parts pushed by every CTA, by column parity: [CTA][jj] = the slice's sum
  // below row j of a_j a_jj (jj > j), a_j^2 (jj = j) or v_jj a_j (jj < j)
  __shared__ T s_part[2][QRC_MAX_CS][QB];
  __shared__ T s_row[2][QB];                         // row j of the panel
  __shared__ T s_red[QRC_MAX_WARPS][QB];
  __shared__ T s_sum[QB];
  __shared__ T s_tw[QB];                             // tau w_jj of the current column
  __shared__ T s_v0[QB];
  __shared__ T s_tau[QB];
  __shared__ T s_T[QB][QB + 1];                      // V^T V above the diagonal, then T
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int nr = max(0, r1 - r0);
  // the slice, eight loads in flight per thread
  for (int e0 = 0; e0 < nr * jb; e0 += 8 * QRC_THREADS) {
    T x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + tid + u * QRC_THREADS;
      x[u] = e < nr * jb ? A[(p + r0 + e % nr) + (int64_t)(p + e / nr) * ld] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + tid + u * QRC_THREADS;
      if (e < nr * jb) P[e % nr + (e / nr) * rb] = x[u];
    }
  }
  for (int e = tid; e < QB * (QB + 1); e += QRC_THREADS) (&s_T[0][0])[e] = T(0);
  cl.sync();   // every CTA runs (and holds its slice) before the first push

  // sum acc[] over the warp (lane l ends with entry l), then over the warps;
  // push column c's parts (and row c from its owner) into every CTA
  T acc[QB];
  auto push = [&](int c, int par, T r_prev) {
#pragma unroll
    for (int o = QB / 2; o > 0; o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int q = 0; q < o; ++q) {
        const T send = up ? acc[q] : acc[q + o];
        const T keep = up ? acc[q + o] : acc[q];
        acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    s_red[warp][lane] = acc[0];
    __syncthreads();
    if (tid == 2 * QB && c >= 1 && c - 1 >= r0 && c - 1 < r1)   // R of the column just reduced
      P[(c - 1 - r0) + (c - 1) * rb] = r_prev;
    if (tid < QB) {
      T t = T(0);
      for (int w = 0; w < QRC_WARPS; ++w) t += s_red[w][tid];
      for (int q = 0; q < CS; ++q) *cl.map_shared_rank(&s_part[par][rank][tid], q) = t;
    } else if (tid < 2 * QB && c >= r0 && c < r1) {
      const int jj = tid - QB;
      const T x = jj < jb ? P[(c - r0) + jj * rb] : T(0);
      for (int q = 0; q < CS; ++q) *cl.map_shared_rank(&s_row[par][jj], q) = x;
    }
  };

  // parts of column 0
#pragma unroll
  for (int jj = 0; jj < QB; ++jj) acc[jj] = T(0);
  for (int i = tid; i < nr; i += QRC_THREADS) {
    if (r0 + i == 0) continue;
    const T x = P[i];
    acc[0] = fma(x, x, acc[0]);
#pragma unroll
    for (int jj = 1; jj < QB; ++jj)
      if (jj < jb) acc[jj] = fma(x, P[i + jj * rb], acc[jj]);
  }
  push(0, 0, T(0));
  for (int j = 0; j < jb; ++j) {
    const int par = j & 1;
    cl.sync();   // column j's parts are in every CTA
    if (tid < QB) {
      T t = T(0);
      for (int q = 0; q < CS; ++q) t += s_part[par][q][tid];
      s_sum[tid] = t;
    }
    __syncthreads();
    const T x0 = s_row[par][j], tail = s_sum[j];
    const T nx = sqrt(fma(x0, x0, tail));
    const T alpha = x0 >= T(0) ? -nx : nx;
    const T v0 = x0 - alpha;
    const T vtv = fma(v0, v0, tail);
    const T tau = vtv > T(0) ? T(2) / vtv : T(0);
    if (tid < QB) {
      s_tw[tid] = (tid > j && tid < jb) ? tau * fma(v0, s_row[par][tid], s_sum[tid]) : T(0);
    } else if (tid < 2 * QB) {
      // v_l^T v_j = v_l[j] v0 + (v_l^T a_j below row j), kept for T
      const int l = tid - QB;
      if (l < j) {
        s_T[l][j] = fma(s_row[par][l], v0, s_sum[l]);
      } else if (l == j) {
        s_tau[j] = tau;
        s_v0[j] = v0;
      }
    }
    __syncthreads();
    if (j + 1 == jb) {
      if (tid == 0 && j >= r0 && j < r1) P[(j - r0) + j * rb] = alpha;   // R_jj
      break;
    }
    // a_jj -= (tau w_jj) v on the slice's rows from j on, and the parts of
    // column j + 1 from the updated entries (rows below j + 1)
#pragma unroll
    for (int jj = 0; jj < QB; ++jj) acc[jj] = T(0);
    T tl = T(0);
    for (int i = tid; i < nr; i += QRC_THREADS) {
      const int row = r0 + i;
      if (row < j) continue;
      // column j + 1 first (its updated entry weights the products), then
      // the other columns in two halves: each half's loads in flight
      // together, then its update (columns > j) and products
      const T vi = row == j ? v0 : P[i + j * rb];
      const T xj1 = fma(-s_tw[j + 1], vi, P[i + (j + 1) * rb]);
      P[i + (j + 1) * rb] = xj1;
      const T xn = row > j + 1 ? xj1 : T(0);
      tl = fma(xn, xn, tl);
#pragma unroll
      for (int h = 0; h < QB; h += QB / 2) {
        T x[QB / 2];
#pragma unroll
        for (int u = 0; u < QB / 2; ++u) {
          const int jj = h + u;
          x[u] = (jj < jb && jj != j + 1) ? P[i + jj * rb] : T(0);
        }
#pragma unroll
        for (int u = 0; u < QB / 2; ++u) {
          const int jj = h + u;
          if (jj > j + 1 && jj < jb) {
            x[u] = fma(-s_tw[jj], vi, x[u]);
            P[i + jj * rb] = x[u];
          }
          if (jj < jb && jj != j + 1) acc[jj] = fma(xn, x[u], acc[jj]);
        }
      }
    }
#pragma unroll
    for (int jj = 0; jj < QB; ++jj)
      if (jj == j + 1) acc[jj] = tl;
    push(j + 1, par ^ 1, alpha);   // also R_jj = alpha
  }
  __syncthreads();
  // reflectors to V (rows p..m-1, zeros above each diagonal), the slice back
  // to A, and T from the first CTA
  for (int e = tid; e < nr * QB; e += QRC_THREADS) {
    const int i = e % nr, j = e / nr, row = r0 + i;
    T v = T(0);
    if (j < jb) {
      if (row == j) v = s_v0[j];
      else if (row > j) v = P[i + j * rb];
      A[(p + row) + (int64_t)(p + j) * ld] = P[i + j * rb];
    }
    V[row + (int64_t)j * m] = v;
  }
  if (rank == 0) {
    // the block's rows above the panel: zero in the panel's reflectors
    const int vtop = p - p0;
    for (int e = tid; e < vtop * QB; e += QRC_THREADS) V[(e % vtop - vtop) + (int64_t)(e / vtop) * m] = T(0);
    // T column by column from the products kept above its diagonal:
    // T[l][j] = -tau_j sum_{i=l}^{j-1} T[l][i] (v_i^T v_j), T[j][j] = tau_j
    for (int j = 0; j < jb; ++j) {
      T t = T(0);
      if (tid < j)
        for (int i2 = tid; i2 < j; ++i2) t = fma(s_T[tid][i2], s_T[i2][j], t);
      __syncthreads();
      if (tid < j) s_T[tid][j] = -s_tau[j] * t;
      else if (tid == j) s_T[j][j] = s_tau[j];
      __syncthreads();
    }
    T* Tt = Tar + d.Tt + qr_toff(p, p0);
    for (int e = tid; e < QB * QB; e += QRC_THREADS) {
      const int i = e % QB, j = e / QB;
      Tt[e] = (i < jb && j < jb) ? s_T[i][j] : T(0);
    }
  }
}

// R (n x n, ld = n, zeros below the diagonal) from rows 0..n-1 of the factored matrix
template <typename T>
__global__ void k_extract_r(const QRDesc* __restrict__ ds, const int64_t* __restrict__ roff,
                            const T* __restrict__ Gar, T* Rar) {
  const QRDesc d = ds[blockIdx.y];
  const int64_t tot = (int64_t)d.n * d.n;
  const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (e >= tot) return;
  const int r = (int)(e % d.n), c = (int)(e / d.n);
  Rar[roff[blockIdx.y] + e] = r <= c ? Gar[d.A + r + (int64_t)c * d.ld] : T(0);
}

// ---- trailing columns of a panel: W = T^T V^T A_t, A_t -= V W ---------------
// Both products stream A_t (the (m-p) x nt columns right of the panel) from
// HBM once; V (m-p) x jb and W (jb x nt) are small and come from L2.
//
// eight consecutive values from 16-byte aligned shared memory
__device__ __forceinline__ void load8(float (&x)[8], const float* p) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 4);
  x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
  x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}
__device__ __forceinline__ void load8(double (&x)[8], const double* p) {
#pragma unroll
  for (int i = 0; i < 8; i += 2) {
    const double2 a = *reinterpret_cast<const double2*>(p + i);
    x[i] = a.x;
    x[i + 1] = a.y;
  }
}

// asynchronous copy of one element global -> shared (zero when !ok)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool ok) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(ok ? 4 : 0)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
                 "r"(ok ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// k_qr_w1: partial V^T A_t over one split of the rows.  A CTA owns 64
// columns and a contiguous range of 32-row chunks, streamed through a ring
// of W1_ST shared-memory stages by asynchronous copies (W1_ST - 1 chunks in
// flight while one is multiplied).  Its 8 warps take 4 rows of each chunk,
// every lane an 8 x 8 block of the 32 x 64 partial (8 consecutive V columns
// by 8 consecutive A columns, read as 16-byte vectors), and the 8 warps'
// partials are added in warp order at the end.  Partial s of front f goes
// to Wp + wpo[f] + s QB nt (QB x nt, ld = QB).
constexpr int W1_NC = 64;
constexpr int W1_KC = 32;
constexpr int W1_ST = 4;
constexpr int W1_THREADS = 256;
constexpr int W1_AP = W1_NC + 4;   // row pitches of a staged chunk (16-byte rows)
constexpr int W1_VP = QB + 4;
constexpr int W1_STAGE = W1_KC * (W1_AP + W1_VP);   // elements per stage

template <typename T>
constexpr size_t w1_smem_bytes() {
  const size_t ring = sizeof(T) * (size_t)W1_ST * W1_STAGE;
  const size_t red = sizeof(T) * (size_t)(W1_THREADS / 32) * QB * W1_NC;
  return ring > red ? ring : red;
}

template <typename T>
__global__ void __launch_bounds__(W1_THREADS, sizeof(T) == 4 ? 2 : 1)
    k_qr_w1(const QRDesc* __restrict__ ds, const T* __restrict__ Gar, const T* __restrict__ Var,
            T* Wp, const int64_t* __restrict__ wpo, int p, int p0, int S) {
  const QRDesc d = ds[blockIdx.y];
  if (p >= d.n) return;
  const int jb = min(QB, d.n - p);
  const int nt = min(d.n, p0 + QB2) - p - jb;   // the block's columns right of the panel
  const int c0 = (int)(blockIdx.x / S) * W1_NC, s = (int)(blockIdx.x % S);
  if (nt <= 0 || c0 >= nt) return;
  const int mp = d.m - p;
  const int nch = (mp + W1_KC - 1) / W1_KC;
  const int kc0 = (int)((int64_t)nch * s / S), kc1 = (int)((int64_t)nch * (s + 1) / S);
  const T* A = Gar + d.A + p + (int64_t)(p + jb) * d.ld;   // A_t(0, 0)
  const T* V = Var + d.V + qr_voff(p, p0, d.m);            // V(r, j) = V[r + j m]
  extern __shared__ __align__(16) unsigned char w1sm[];
  T* ring = reinterpret_cast<T*>(w1sm);   // stage: As[k W1_AP + c], then Vs[k W1_VP + j]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lv = lane & 3, la = lane >> 2;                  // V columns lv*8+i, A columns la*8+jj
  // thread tid copies row sk of a chunk, A and V columns sc + CS q: a warp
  // covers 8 consecutive rows of 4 columns, so its global reads fill whole
  // 32-byte sectors and its shared-memory stores (row pitch = 4 mod 32 banks)
  // hit 32 different banks
  static_assert(W1_KC == 32 && W1_THREADS == 256, "staging map assumes 32 rows, 8 warps");
  constexpr int NQA = W1_NC * W1_KC / W1_THREADS, NQV = W1_KC * QB / W1_THREADS;
  constexpr int CS = W1_THREADS / W1_KC;
  const int sk = (lane & 7) + 8 * (warp & 3), sc = (lane >> 3) + 4 * (warp >> 2);
  auto issue = [&](int kc) {
    if (kc < kc1) {
      T* As = ring + (size_t)((kc - kc0) % W1_ST) * W1_STAGE;
      T* Vs = As + W1_KC * W1_AP;
      const int r = kc * W1_KC + sk;
#pragma unroll
      for (int q = 0; q < NQA; ++q) {
        const int cc = c0 + sc + CS * q;
        const bool ok = r < mp && cc < nt;
        cp_async_elem(As + sk * W1_AP + sc + CS * q, ok ? A + r + (int64_t)cc * d.ld : A, ok);
      }
#pragma unroll
      for (int q = 0; q < NQV; ++q) {
        const int j = sc + CS * q;
        const bool ok = r < mp && j < jb;
        cp_async_elem(Vs + sk * W1_VP + j, ok ? V + r + (int64_t)j * d.m : V, ok);
      }
    }
    cp_async_commit();   // one group per chunk slot, empty past the end
  };
  T acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) acc[i][jj] = T(0);
#pragma unroll
  for (int i = 0; i < W1_ST - 1; ++i) issue(kc0 + i);
  for (int kc = kc0; kc < kc1; ++kc) {
    cp_async_wait<W1_ST - 2>();   // this thread's copies of chunk kc are done
    __syncthreads();              // everyone's are; stage (kc - 1) is free again
    issue(kc + W1_ST - 1);
    const T* As = ring + (size_t)((kc - kc0) % W1_ST) * W1_STAGE;
    const T* Vs = As + W1_KC * W1_AP;
#pragma unroll 1
    for (int kk = 0; kk < W1_KC / 8; ++kk) {
      const int k = warp * (W1_KC / 8) + kk;
      T v[8], a[8];
      load8(v, Vs + k * W1_VP + lv * 8);
      load8(a, As + k * W1_AP + la * 8);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[i][jj] = fma(v[i], a[jj], acc[i][jj]);
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // the 8 warps' partials, added in warp order
  T* R = reinterpret_cast<T*>(w1sm);   // R[w QB W1_NC + i + QB c]
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj)
      R[(size_t)warp * QB * W1_NC + (lv * 8 + i) + QB * (la * 8 + jj)] = acc[i][jj];
  __syncthreads();
  T* out = Wp + wpo[blockIdx.y] + (int64_t)s * QB * nt;
  for (int e = tid; e < QB * W1_NC; e += W1_THREADS) {
    const int i = e % QB, c = e / QB;
    if (c0 + c >= nt) continue;
    T t = R[e];
    for (int w = 1; w < W1_THREADS / 32; ++w) t += R[(size_t)w * QB * W1_NC + e];
    out[i + (int64_t)(c0 + c) * QB] = t;
  }
}

// k_qr_w2: W = T^T (sum of the S partials, in split order), one thread per
// column; W goes to the front's work block (War + W, ld = QB).
template <typename T>
__global__ void __launch_bounds__(128) k_qr_w2(const QRDesc* __restrict__ ds,
                                               const T* __restrict__ Wp,
                                               const int64_t* __restrict__ wpo,
                                               const T* __restrict__ Tar, T* War, int p, int p0,
                                               int S) {
  const QRDesc d = ds[blockIdx.y];
  if (p >= d.n) return;
  const int jb = min(QB, d.n - p);
  const int nt = min(d.n, p0 + QB2) - p - jb;
  __shared__ T Ts[QB][QB + 1];   // Ts[i][j] = T(i, j)
  const T* Tt = Tar + d.Tt + qr_toff(p, p0);
  for (int e = threadIdx.x; e < QB * QB; e += 128) Ts[e % QB][e / QB] = Tt[e];
  __syncthreads();
  const int c = blockIdx.x * 128 + threadIdx.x;
  if (c >= nt) return;
  T w1[QB];
#pragma unroll
  for (int i = 0; i < QB; ++i) w1[i] = T(0);
  const T* src = Wp + wpo[blockIdx.y] + (int64_t)c * QB;
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int i = 0; i < QB; ++i) w1[i] += src[(int64_t)s * QB * nt + i];
  T* dst = War + d.W + (int64_t)c * QB;
#pragma unroll
  for (int i = 0; i < QB; ++i) {
    T t = T(0);
#pragma unroll
    for (int j = 0; j <= i; ++j) t = fma(Ts[j][i], w1[j], t);   // T upper triangular
    dst[i] = i < jb ? t : T(0);
  }
}

// k_qr_update: A_t -= V W over 128 x 64 tiles; lane l of warp w holds rows
// l + 32 i (i < 4) and columns 8 w + jj (jj < 8) of the tile.
template <typename T>
__global__ void __launch_bounds__(256) k_qr_update(const QRDesc* __restrict__ ds, T* Gar,
                                                   const T* __restrict__ Var,
                                                   const T* __restrict__ War, int p, int p0) {
  const QRDesc d = ds[blockIdx.y];
  if (p >= d.n) return;
  const int jb = min(QB, d.n - p);
  const int nt = min(d.n, p0 + QB2) - p - jb;
  const int mp = d.m - p;
  const int tm = (mp + 127) / 128, tn = (nt + 63) / 64;
  if (nt <= 0 || (int)blockIdx.x >= tm * tn) return;
  const int rb = (int)(blockIdx.x % tm) * 128, cb = (int)(blockIdx.x / tm) * 64;
  T* A = Gar + d.A + p + (int64_t)(p + jb) * d.ld;
  const T* V = Var + d.V + qr_voff(p, p0, d.m);
  const T* W = War + d.W;
  __shared__ __align__(16) T Vs[QB][128];
  __shared__ __align__(16) T Ws[QB][64 + 4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // this thread's entries of A_t, loaded before the staging so that their
  // latency overlaps it
  T a[4][8];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int c = cb + warp * 8 + jj;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rb + lane + 32 * i;
      a[i][jj] = (r < mp && c < nt) ? A[r + (int64_t)c * d.ld] : T(0);
    }
  }
  // V rows rb.. and W columns cb.. of the tile, all loads issued before the
  // shared-memory stores
  {
    T sv[QB * 128 / 256], sw[QB * 64 / 256];
    const int r = threadIdx.x % 128, j0 = threadIdx.x / 128;
#pragma unroll
    for (int q = 0; q < QB * 128 / 256; ++q) {
      const int j = j0 + 2 * q;
      sv[q] = (rb + r < mp && j < jb) ? V[rb + r + (int64_t)j * d.m] : T(0);
    }
    const int k = threadIdx.x % QB, c0 = threadIdx.x / QB;
#pragma unroll
    for (int q = 0; q < QB * 64 / 256; ++q) {
      const int c = c0 + 8 * q;
      sw[q] = (cb + c < nt) ? W[k + (int64_t)(cb + c) * QB] : T(0);
    }
#pragma unroll
    for (int q = 0; q < QB * 128 / 256; ++q) Vs[j0 + 2 * q][r] = sv[q];
#pragma unroll
    for (int q = 0; q < QB * 64 / 256; ++q) Ws[k][c0 + 8 * q] = sw[q];
  }
  __syncthreads();
#pragma unroll 4
  for (int k = 0; k < QB; ++k) {
    T v[4], w[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = Vs[k][lane + 32 * i];
    load8(w, &Ws[k][warp * 8]);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) a[i][jj] = fma(-v[i], w[jj], a[i][jj]);
  }
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int c = cb + warp * 8 + jj;
    if (c >= nt) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rb + lane + 32 * i;
      if (r < mp) A[r + (int64_t)c * d.ld] = a[i][jj];
    }
  }
}


// T of a 128-column block from the Gram matrix G = V^T V of its reflectors
// (G[l + j 128]) and their tau (the diagonals of its four panel T's): T[j][j]
// = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] G[0:j, j], column by column; thread
// i owns row i.  One CTA per front.
template <typename T>
__global__ void __launch_bounds__(QB2) k_qr_tblk(const QRDesc* __restrict__ ds,
                                                 const T* __restrict__ Gb,
                                                 const T* __restrict__ Tar, T* Tb) {
  const QRDesc d = ds[blockIdx.x];
  const T* G = Gb + (int64_t)blockIdx.x * QB2 * QB2;
  const T* Tp = Tar + d.Tt;
  T* To = Tb + (int64_t)blockIdx.x * QB2 * QB2;
  extern __shared__ __align__(16) unsigned char tbs[];
  T* sT = reinterpret_cast<T*>(tbs);   // sT[i (QB2 + 1) + j]
  __shared__ T s_g[QB2], s_tau[QB2];
  const int i = threadIdx.x;
  s_tau[i] = Tp[(i / QB) * QB * QB + (i % QB) * (QB + 1)];
  for (int j = 0; j < QB2; ++j) sT[i * (QB2 + 1) + j] = T(0);
  for (int j = 0; j < QB2; ++j) {
    __syncthreads();
    s_g[i] = G[i + (int64_t)j * QB2];
    __syncthreads();
    const T tau = s_tau[j];
    if (i < j) {
      T t = T(0);
      for (int l = i; l < j; ++l) t = fma(sT[i * (QB2 + 1) + l], s_g[l], t);
      sT[i * (QB2 + 1) + j] = -tau * t;
    } else if (i == j) {
      sT[i * (QB2 + 1) + j] = tau;
    }
  }
  __syncthreads();
  for (int j = 0; j < QB2; ++j) To[i + (int64_t)j * QB2] = sT[i * (QB2 + 1) + j];
}
}  // namespace

constexpr size_t QRC_SMEM_MAX = 160 * 1024;

// How many clusters of cs CTAs with rb panel rows each the GPU holds at once
// (0: none; asked once per shape; the first call per precision also lifts
// the kernel's cluster-size and shared memory limits).
template <typename T>
int panel_clusters_active_t(int cs, int rb) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> known;
  std::lock_guard<std::mutex> g(mu);
  static const bool attr = [] {
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_qr_panel_cluster<T>,
                                      cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_qr_panel_cluster<T>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)QRC_SMEM_MAX));
    return true;
  }();
  (void)attr;
  const size_t smem = (size_t)rb * QB * sizeof(T);
  if (smem > QRC_SMEM_MAX) return 0;
  const auto key = std::make_pair(cs, rb);
  const auto it = known.find(key);
  if (it != known.end()) return it->second;
  cudaLaunchConfig_t q = {};
  q.gridDim = dim3((unsigned)cs);
  q.blockDim = dim3(qrc_threads<T>());
  q.dynamicSmemBytes = smem;
  cudaLaunchAttribute qa[1];
  qa[0].id = cudaLaunchAttributeClusterDimension;
  qa[0].val.clusterDim.x = cs;
  qa[0].val.clusterDim.y = 1;
  qa[0].val.clusterDim.z = 1;
  q.attrs = qa;
  q.numAttrs = 1;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, k_qr_panel_cluster<T>, &q) != cudaSuccess) {
    cudaGetLastError();
    ncl = 0;
  }
  known[key] = std::max(0, ncl);
  return known[key];
}

inline int panel_clusters_active(int cs, int rb, int tsize) {
  return tsize == 8 ? panel_clusters_active_t<double>(cs, rb)
                    : panel_clusters_active_t<float>(cs, rb);
}

// The cluster size for a panel launch over nact fronts of at most maxmp rows
// (0: none fits, the panel streams through k_qr_panel): the one that
// minimises waves x (per-column cost of a CTA), the cost of a column being a
// fixed part (barriers, exchange) worth QRC_FIXED_ROWS rows plus its rows.
constexpr int QRC_FIXED_ROWS = 256;
inline int panel_cluster_size(int nact, int maxmp, int tsize) {
  int best = 0;
  double best_cost = 0.0;
  for (int cs = 1; cs <= QRC_MAX_CS; ++cs) {
    const int rb = ceil_div(maxmp, cs);
    const int act = panel_clusters_active(cs, rb, tsize);
    if (act <= 0) continue;
    const double cost = (double)ceil_div(nact, act) * (QRC_FIXED_ROWS + rb);
    if (best == 0 || cost < best_cost) {
      best = cs;
      best_cost = cost;
    }
  }
  return best;
}

// Unpivoted QR of the R rows of fronts `which` (in place in the gather
// arena); their n x n triangular factors go to Rout at rOff (ld = n).
template <typename T>
void reduce_rows_qr(const SkelDesc* h_f, const std::vector<int>& which, T* Garena, T* Rout,
                    const std::vector<int64_t>& rOff, int* d_flags, bool tensor_cores,
                    cudaStream_t st) {
  const int nq = (int)which.size();
  if (nq == 0) return;
  // fronts sorted by n (largest first) so that the fronts still factoring a
  // panel are a prefix
  std::vector<int> ord(nq);
  for (int i = 0; i < nq; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(),
                   [&](int a, int b) { return h_f[which[a]].nF > h_f[which[b]].nF; });
  std::vector<QRDesc> qd(nq);
  std::vector<int64_t> ro(nq);
  int64_t voff = 0, woff = 0, toff = 0;
  for (int i = 0; i < nq; ++i) {
    const SkelDesc& s = h_f[which[ord[i]]];
    QRDesc& d = qd[i];
    d.A = s.G + s.nF;
    d.m = s.nR;
    d.n = s.nF;
    d.ld = s.nF + s.nR;
    d.V = voff;
    d.W = woff;
    d.Tt = toff;
    d.pad = 0;
    voff += (int64_t)d.m * QB2;          // the block's reflectors
    woff += (int64_t)QB * d.n;
    toff += (QB2 / QB) * QB * QB;         // the block's four panel T's
    ro[i] = rOff[ord[i]];
  }
  T *Var = nullptr, *War = nullptr, *Tar = nullptr;
  QRDesc* d_qd = nullptr;
  int64_t* d_ro = nullptr;
  HIF_CUDA_TRY(cudaMallocAsync(&Var, sizeof(T) * voff, st));
  HIF_CUDA_TRY(cudaMallocAsync(&War, sizeof(T) * woff, st));
  HIF_CUDA_TRY(cudaMallocAsync(&Tar, sizeof(T) * toff, st));
  HIF_CUDA_TRY(cudaMallocAsync(&d_qd, sizeof(QRDesc) * nq, st));
  HIF_CUDA_TRY(cudaMallocAsync(&d_ro, sizeof(int64_t) * nq, st));
  HIF_CUDA_TRY(cudaMemcpyAsync(d_qd, qd.data(), sizeof(QRDesc) * nq, cudaMemcpyHostToDevice, st));
  HIF_CUDA_TRY(cudaMemcpyAsync(d_ro, ro.data(), sizeof(int64_t) * nq, cudaMemcpyHostToDevice, st));
  const int nmax = qd[0].n;
  int nsm = 0, dev = 0;
  HIF_CUDA_TRY(cudaGetDevice(&dev));
  HIF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // split of the rows of W = V^T A_t: enough CTAs for two waves at two per
  // SM; the partials' workspace holds the largest split of any panel
  constexpr int W1_SPLIT_MAX = 8;
  // the block's columns right of panel p (block start p0)
  auto nt_in = [&](const QRDesc& d, int p, int p0) {
    return std::min(d.n, p0 + QB2) - p - std::min(QB, d.n - p);
  };
  auto w1_split = [&](int p, int p0) {
    int tiles = 0;
    for (int i = 0; i < nq && qd[i].n > p; ++i) {
      const int nt = nt_in(qd[i], p, p0);
      if (nt > 0) tiles += ceil_div(nt, W1_NC);
    }
    return tiles == 0 ? 0 : std::max(1, std::min(W1_SPLIT_MAX, ceil_div(4 * nsm, tiles)));
  };
  int smax = 0;
  for (int p = 0; p < nmax; p += QB) smax = std::max(smax, w1_split(p, p / QB2 * QB2));
  std::vector<int64_t> wpo(nq);
  int64_t wptot = 0;
  for (int i = 0; i < nq; ++i) {
    wpo[i] = wptot;
    wptot += (int64_t)smax * QB * qd[i].n;
  }
  T* Wp = nullptr;
  int64_t* d_wpo = nullptr;
  HIF_CUDA_TRY(cudaMallocAsync(&Wp, sizeof(T) * std::max<int64_t>(1, wptot), st));
  HIF_CUDA_TRY(cudaMallocAsync(&d_wpo, sizeof(int64_t) * nq, st));
  HIF_CUDA_TRY(cudaMemcpyAsync(d_wpo, wpo.data(), sizeof(int64_t) * nq, cudaMemcpyHostToDevice, st));
  static const bool w1_attr = [] {
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_qr_w1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)w1_smem_bytes<T>()));
    return true;
  }();
  (void)w1_attr;
  // the block update's workspace: the Gram matrix of the block's
  // reflectors, the block's T, and W' = V^T A_t, W = T^T W'
  int64_t w2tot = 0;
  std::vector<int64_t> w2o(nq);
  for (int i = 0; i < nq; ++i) {
    w2o[i] = w2tot;
    w2tot += (int64_t)QB2 * qd[i].n;
  }
  const bool blocks = nmax > QB2;
  T *Gb = nullptr, *Tb = nullptr, *W1b = nullptr, *W2b = nullptr;
  if (blocks) {
    HIF_CUDA_TRY(cudaMallocAsync(&Gb, sizeof(T) * nq * QB2 * QB2, st));
    HIF_CUDA_TRY(cudaMallocAsync(&Tb, sizeof(T) * nq * QB2 * QB2, st));
    HIF_CUDA_TRY(cudaMallocAsync(&W1b, sizeof(T) * w2tot, st));
    HIF_CUDA_TRY(cudaMallocAsync(&W2b, sizeof(T) * w2tot, st));
  }
  for (int p = 0; p < nmax; p += QB) {
    const int p0 = p / QB2 * QB2;
    int nact = 0;
    while (nact < nq && qd[nact].n > p) ++nact;
    {
      // algorithmic counts: Householder QR of the (m - p) x jb panel
      // (2 (m-p) jb^2 flops), read and written once, reflectors written to V
      double pf = 0, pb = 0;
      int maxmp = 0;
      for (int i = 0; i < nact; ++i) maxmp = std::max(maxmp, qd[i].m - p);
      if (prof_enabled())
        for (int i = 0; i < nact; ++i) {
          const double mp = qd[i].m - p, jb = std::min(QB, qd[i].n - p);
          pf += 2.0 * mp * jb * jb;
          pb += 3.0 * sizeof(T) * mp * jb;
        }
      ProfScope ps("id_rowreduce_panel", st, pf, pb);
      // each panel in the shared memory of a cluster (the size that
      // finishes the batch first); panels too tall for 16 CTAs stream from
      // L2 (k_qr_panel)
      const int cs = panel_cluster_size(nact, maxmp, (int)sizeof(T));
      const int rb = ceil_div(maxmp, std::max(1, cs));
      const size_t smem = (size_t)rb * QB * sizeof(T);
      if (cs > 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nact * cs));
        cfg.blockDim = dim3(qrc_threads<T>());
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        HIF_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_qr_panel_cluster<T>, (const QRDesc*)d_qd, Garena,
                                        Var, Tar, p, p0, rb));
      } else {
        k_qr_panel<T><<<nact, QR_THREADS, 0, st>>>(d_qd, Garena, Var, Tar, p, p0);
      }
      HIF_CHECK_LAUNCH();
    }
    // the block's columns right of the panel: W = T^T V^T A_t (partials
    // over row splits, then their sum and T^T), A_t -= V W
    const int S = w1_split(p, p0);
    if (S > 0) {
      int ct = 0, ntmax = 0, ut = 0;
      double f1 = 0, b1 = 0, b2 = 0;
      for (int i = 0; i < nact; ++i) {
        const int jb = std::min(QB, qd[i].n - p), nt = nt_in(qd[i], p, p0), mp = qd[i].m - p;
        if (nt <= 0) continue;
        ct = std::max(ct, ceil_div(nt, W1_NC));
        ntmax = std::max(ntmax, nt);
        ut = std::max(ut, ceil_div(mp, 128) * ceil_div(nt, 64));
        f1 += 2.0 * jb * (double)nt * mp;
        b1 += sizeof(T) * ((double)mp * nt + (double)mp * jb);
        b2 += 2.0 * sizeof(T) * (double)mp * nt;
      }
      {
        ProfScope ps("id_rowreduce_w1", st, f1, b1);
        k_qr_w1<T><<<dim3((unsigned)(ct * S), nact), W1_THREADS, w1_smem_bytes<T>(), st>>>(
            d_qd, Garena, Var, Wp, d_wpo, p, p0, S);
        HIF_CHECK_LAUNCH();
        k_qr_w2<T><<<dim3((unsigned)ceil_div(ntmax, 128), nact), 128, 0, st>>>(d_qd, Wp, d_wpo, Tar,
                                                                             War, p, p0, S);
        HIF_CHECK_LAUNCH();
      }
      {
        ProfScope ps("id_rowreduce_update", st, f1, b2);
        k_qr_update<T><<<dim3((unsigned)ut, nact), 256, 0, st>>>(d_qd, Garena, Var, War, p, p0);
        HIF_CHECK_LAUNCH();
      }
    }
    // after the block's last panel: the columns right of the block, once
    // per block, by matrix products (tensor cores in FP32):
    // G = V^T V -> the block's T;  W' = V^T A_t;  W = T^T W';  A_t -= V W
    if (p + QB < p0 + QB2 && p + QB < nmax) continue;
    int nb = 0;
    while (nb < nq && qd[nb].n > p0 + QB2) ++nb;
    if (nb == 0) continue;
    std::vector<GemmOp> og(nb), o1(nb), o2(nb), ou(nb);
    for (int i = 0; i < nb; ++i) {
      const QRDesc& d = qd[i];
      const int mp0 = d.m - p0, nt = d.n - p0 - QB2;
      const int64_t at = d.A + p0 + (int64_t)(p0 + QB2) * d.ld;   // A_t(0, 0)
      og[i] = GemmOp{d.V, d.V, (int64_t)i * QB2 * QB2, QB2, QB2, mp0, d.m, d.m, QB2, 1, 0, 1.f, 0.f, 0, 0};
      o1[i] = GemmOp{d.V, at, w2o[i], QB2, nt, mp0, d.m, d.ld, QB2, 1, 0, 1.f, 0.f, 0, 0};
      o2[i] = GemmOp{(int64_t)i * QB2 * QB2, w2o[i], w2o[i], QB2, nt, QB2, QB2, QB2, QB2, 1, 0, 1.f, 0.f, 0, 0};
      ou[i] = GemmOp{d.V, w2o[i], at, mp0, nt, QB2, d.m, QB2, d.ld, 0, 0, -1.f, 1.f, 0, 0};
    }
    GemmOp* d_ops = nullptr;
    HIF_CUDA_TRY(cudaMallocAsync(&d_ops, sizeof(GemmOp) * 4 * nb, st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_ops, og.data(), sizeof(GemmOp) * nb, cudaMemcpyHostToDevice, st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_ops + nb, o1.data(), sizeof(GemmOp) * nb, cudaMemcpyHostToDevice, st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_ops + 2 * nb, o2.data(), sizeof(GemmOp) * nb, cudaMemcpyHostToDevice, st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_ops + 3 * nb, ou.data(), sizeof(GemmOp) * nb, cudaMemcpyHostToDevice, st));
    auto gemm = [&](const GemmOp* dop, const GemmOp* hop, const T* Ab, const T* Bb, T* Cb,
                    const char* tc_name, const char* name) {
      if constexpr (std::is_same<T, float>::value) {
        if (tensor_cores) {
          gemm_tc(dop, hop, nb, Ab, Bb, Cb, d_flags, st, tc_name);
          return;
        }
      }
      gemm_batched<T>(dop, hop, nb, Ab, Bb, Cb, st, name);
    };
    gemm(d_ops, og.data(), Var, Var, Gb, "id_rowreduce_gram_tc", "id_rowreduce_gram");
    {
      static const bool tb_attr = [] {
        HIF_CUDA_TRY(cudaFuncSetAttribute(k_qr_tblk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sizeof(T) * QB2 * (QB2 + 1))));
        return true;
      }();
      (void)tb_attr;
      ProfScope ps("id_rowreduce_blockt", st, (double)nb * QB2 * QB2 * QB2 / 3.0, 0.0);
      k_qr_tblk<T><<<nb, QB2, sizeof(T) * QB2 * (QB2 + 1), st>>>(d_qd, Gb, Tar, Tb);
      HIF_CHECK_LAUNCH();
    }
    gemm(d_ops + nb, o1.data(), Var, Garena, W1b, "id_rowreduce_vta_tc", "id_rowreduce_vta");
    gemm(d_ops + 2 * nb, o2.data(), Tb, W1b, W2b, "id_rowreduce_tw_tc", "id_rowreduce_tw");
    gemm(d_ops + 3 * nb, ou.data(), Var, W2b, Garena, "id_rowreduce_block_tc", "id_rowreduce_block");
    HIF_CUDA_TRY(cudaFreeAsync(d_ops, st));
  }
  if (blocks) {
    HIF_CUDA_TRY(cudaFreeAsync(W2b, st));
    HIF_CUDA_TRY(cudaFreeAsync(W1b, st));
    HIF_CUDA_TRY(cudaFreeAsync(Tb, st));
    HIF_CUDA_TRY(cudaFreeAsync(Gb, st));
  }
  {
    ProfScope ps("id_rowreduce_extract", st);
    const int64_t mx = (int64_t)nmax * nmax;
    k_extract_r<T><<<dim3(ceil_div(mx, 256), nq), 256, 0, st>>>(d_qd, d_ro, Garena, Rout);
    HIF_CHECK_LAUNCH();
  }
  HIF_CUDA_TRY(cudaFreeAsync(d_wpo, st));
  HIF_CUDA_TRY(cudaFreeAsync(Wp, st));
  HIF_CUDA_TRY(cudaFreeAsync(d_ro, st));
  HIF_CUDA_TRY(cudaFreeAsync(d_qd, st));
  HIF_CUDA_TRY(cudaFreeAsync(Tar, st));
  HIF_CUDA_TRY(cudaFreeAsync(War, st));
  HIF_CUDA_TRY(cudaFreeAsync(Var, st));
}

template void reduce_rows_qr<float>(const SkelDesc*, const std::vector<int>&, float*, float*,
                                    const std::vector<int64_t>&, int*, bool, cudaStream_t);
template void reduce_rows_qr<double>(const SkelDesc*, const std::vector<int>&, double*, double*,
                                     const std::vector<int64_t>&, int*, bool, cudaStream_t);

}  // namespace hif
