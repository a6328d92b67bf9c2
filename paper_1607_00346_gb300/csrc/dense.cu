// Batched dense kernels over uneven fronts: partial Cholesky (panel factor +
// triangular solve + trailing rank-NB update), inverse of the Cholesky factor,
// generic batched GEMM and the batched GEMV of the apply sweeps.
//
// Every kernel takes a descriptor array (one entry per front or problem) and a
// 2-D grid: blockIdx.y = descriptor, blockIdx.x = tile / chunk inside it.
// Fronts whose work is finished, and tiles outside a front, exit at once.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <type_traits>
#include <vector>

#include "dense.cuh"

namespace hif {

namespace {

constexpr int PANEL_ROWS = 128;   // rows solved per CTA in the panel kernel
constexpr int KC = 16;            // inner-dimension chunk of the tile products
constexpr int MAX_GRID_Y = 65535;

__device__ __forceinline__ void flag_front(int* flags, int which, int id) {
  atomicCAS(&flags[which], -1, id);
}

// ---- tile micro-kernel ---------------------------------------------------------
// 256 threads, 64 x 64 output, thread t owns rows (t % 16)*4 .. +4 and columns
// (t / 16)*4 .. +4.  As[k][r] and Bs[k][c] hold a KC-deep slice.
template <typename T>
struct TileAcc {
  T v[4][4];
  __device__ void zero() {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) v[i][j] = T(0);
  }
  __device__ void mma(const T (*As)[TILE + 4], const T (*Bs)[TILE + 4], int kdepth) {
    const int tr = (threadIdx.x % 16) * 4, tc = (threadIdx.x / 16) * 4;
    for (int k = 0; k < kdepth; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tr + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tc + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) v[i][j] = fma(a[i], b[j], v[i][j]);
    }
  }
};

// ---- panel: Cholesky of the diagonal block, then triangular solve of the rows below
// k_chol_diag: one CTA per front factors the jb x jb diagonal block (jb <= 64)
// right-looking with the block in registers: thread (ty, tx) of a 16 x 16 grid
// holds rows ty + 16 i and columns tx + 16 j (i, j < 4).  Per column c the
// threads holding column c scale it by the pivot and publish it to shared
// memory; every thread then updates its entries right of c, and the holder
// of entry (c+1, c+1) publishes the next pivot.  L goes to the factor panel
// (zeros above the diagonal); a non-positive or non-finite pivot flags the
// front and continues with 1.
//
// With growth > 0 (FP32 fronts that may be retried in FP64), the panel's
// diagonal holds the front's original diagonal A_jj on entry, and a pivot
// d_j with A_jj / d_j > growth (cancellation has eaten all but a few bits of
// it), or one that is not positive or not finite, marks the front in
// fflag[blockIdx.x] instead of failing it.
template <typename T>
__global__ void __launch_bounds__(256) k_chol_diag(const DFront* __restrict__ fr, const T* Kar,
                                                   T* Par, int j0, int* flags, float growth,
                                                   int* fflag) {
  const DFront d = fr[blockIdx.x];
  if (j0 >= d.p) return;
  const int jb = min(NB, d.p - j0);
  const int64_t ld = d.ld;
  const T* K = Kar + d.K + (int64_t)j0 + (int64_t)j0 * ld;
  T* P = Par + d.P + (int64_t)j0 + (int64_t)j0 * ld;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  __shared__ T colv[2][NB];
  __shared__ T diagv[NB];
  __shared__ T origv[NB];
  if (growth > 0.f && threadIdx.x < jb) origv[threadIdx.x] = P[threadIdx.x + (int64_t)threadIdx.x * ld];
  T a[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      a[i][j] = (r < jb && c < jb && r >= c) ? K[r + (int64_t)c * ld] : T(0);
      if (r == c && r == 0) diagv[0] = a[i][j];
    }
  __syncthreads();
  for (int c = 0; c < jb; ++c) {
    const int par = c & 1;
    if (tx == c % 16) {
      const int j = c / 16;
      T dv = diagv[c];
      if (growth > 0.f) {
        if (!(dv > T(0)) || !isfinite(dv) || dv * (T)growth < origv[c]) {
          if (ty == 0) fflag[blockIdx.x] = 1;
          if (!(dv > T(0)) || !isfinite(dv)) dv = T(1);
        }
      } else if (!(dv > T(0)) || !isfinite(dv)) {
        if (ty == 0) flag_front(flags, FLAG_NOT_SPD, d.id);
        dv = T(1);
      }
      const T piv = sqrt(dv), inv = T(1) / piv;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = ty + 16 * i;
        if (r > c) {
          a[i][j] *= inv;
          colv[par][r] = a[i][j];
        } else if (r == c) {
          a[i][j] = piv;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = ty + 16 * i;
      if (r <= c) continue;
      const T lr = colv[par][r];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cc = tx + 16 * j;
        if (cc > c && cc <= r) {
          a[i][j] = fma(-lr, colv[par][cc], a[i][j]);
          if (r == cc && r == c + 1) diagv[r] = a[i][j];
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      if (r < jb && c < jb) P[r + (int64_t)c * ld] = r >= c ? a[i][j] : T(0);
    }
}

// k_panel: the rows below the diagonal block, L21 = A21 L11^{-T}, by forward
// substitution per row (one thread per row) with L11 read from the factor
// panel; rows past the leading block also go to the panel.
template <typename T>
__global__ void __launch_bounds__(PANEL_ROWS) k_panel(const DFront* __restrict__ fr, T* Kar,
                                                      T* Par, int j0) {
  const DFront d = fr[blockIdx.y];
  if (j0 >= d.p) return;
  const int jb = min(NB, d.p - j0);
  const int j1 = j0 + jb;
  const int n = d.n;
  const int64_t ld = d.ld;
  const int r0 = j1 + blockIdx.x * PANEL_ROWS;
  if (r0 >= n) return;
  T* K = Kar + d.K;
  T* P = Par + d.P;
  __shared__ T D[NB][NB + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += PANEL_ROWS) {
    int r = e % NB, c = e / NB;
    D[r][c] = (r < jb && c < jb && r >= c) ? P[(int64_t)(j0 + r) + (int64_t)(j0 + c) * ld] : T(0);
  }
  __syncthreads();
  const int r = r0 + tid;
  if (r >= n) return;
  T x[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) x[c] = c < jb ? K[(int64_t)r + (int64_t)(j0 + c) * ld] : T(0);
  // four partial sums per dot product shorten the dependent chains
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (c < jb) {
      T s[4] = {x[c], T(0), T(0), T(0)};
#pragma unroll
      for (int l = 0; l < c; ++l) s[l & 3] = fma(-x[l], D[c][l], s[l & 3]);
      x[c] = ((s[0] + s[1]) + (s[2] + s[3])) / D[c][c];
    }
  }
  const bool toP = r >= d.p;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (c < jb) {
      const int64_t o = (int64_t)r + (int64_t)(j0 + c) * ld;
      K[o] = x[c];
      if (toP) P[o] = x[c];
    }
  }
}

__device__ __forceinline__ void tri_index(int t, int& ti, int& tj) {
  int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  ti = i;
  tj = t - i * (i + 1) / 2;
}

// ---- trailing update: K[j1:n, j1:n] -= K[j1:n, j0:j1] K[j1:n, j0:j1]^T (lower tiles)
// (jmax < n: only the columns below jmax, i.e. the rest of an outer block;
// the tiles then form nrow x ncol rectangles, strictly upper ones skipped)
template <typename T>
__global__ void __launch_bounds__(256) k_syrk(const DFront* __restrict__ fr, T* Kar, int j0,
                                              int jmax) {
  const DFront d = fr[blockIdx.y];
  if (j0 >= d.p) return;
  const int jb = min(NB, d.p - j0);
  const int j1 = j0 + jb;
  const int n = d.n;
  const int64_t ld = d.ld;
  const int nt = (n - j1 + TILE - 1) / TILE;
  int ti, tj;
  if (jmax >= n) {
    if ((int)blockIdx.x >= nt * (nt + 1) / 2) return;
    tri_index(blockIdx.x, ti, tj);
  } else {
    const int nct = (jmax - j1 + TILE - 1) / TILE;
    if (nct <= 0 || (int)blockIdx.x >= nt * nct) return;
    ti = blockIdx.x % nt;
    tj = blockIdx.x / nt;
    if (tj > ti) return;
  }
  const int rb = j1 + ti * TILE, cb = j1 + tj * TILE;
  T* K = Kar + d.K;
  __shared__ T As[KC][TILE + 4];
  __shared__ T Bs[KC][TILE + 4];
  TileAcc<T> acc;
  acc.zero();
  for (int k0 = 0; k0 < jb; k0 += KC) {
    for (int e = threadIdx.x; e < KC * TILE; e += 256) {
      int rr = e % TILE, kk = e / TILE;
      int col = j0 + k0 + kk;
      bool kin = k0 + kk < jb;
      As[kk][rr] = (kin && rb + rr < n) ? K[(int64_t)(rb + rr) + (int64_t)col * ld] : T(0);
      Bs[kk][rr] = (kin && cb + rr < n) ? K[(int64_t)(cb + rr) + (int64_t)col * ld] : T(0);
    }
    __syncthreads();
    acc.mma(As, Bs, KC);
    __syncthreads();
  }
  const int tr = (threadIdx.x % 16) * 4, tc = (threadIdx.x / 16) * 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = cb + tc + j;
    if (c >= n || c >= jmax) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rb + tr + i;
      if (r < n && r >= c) K[(int64_t)r + (int64_t)c * ld] -= acc.v[i][j];
    }
  }
}

// ---- inverse of the diagonal NB x NB blocks of L (held in P) in place ----------
template <typename T>
__global__ void __launch_bounds__(NB) k_trtri_diag(const DFront* __restrict__ fr, T* Par) {
  const DFront d = fr[blockIdx.y];
  const int i0 = blockIdx.x * NB;
  if (i0 >= d.p) return;
  const int ib = min(NB, d.p - i0);
  const int64_t n = d.ld;
  T* P = Par + d.P;
  __shared__ T Ls[NB][NB + 1];
  __shared__ T Zs[NB][NB + 1];
  for (int e = threadIdx.x; e < NB * NB; e += NB) {
    int r = e % NB, c = e / NB;
    Ls[r][c] = (r < ib && c < ib && r >= c) ? P[(int64_t)(i0 + r) + (int64_t)(i0 + c) * n] : T(0);
  }
  __syncthreads();
  const int c = threadIdx.x;   // one column of the inverse per thread
  if (c < ib) {
    for (int r = 0; r < c; ++r) Zs[r][c] = T(0);
    Zs[c][c] = T(1) / Ls[c][c];
    for (int r = c + 1; r < ib; ++r) {
      T s = T(0);
      for (int l = c; l < r; ++l) s = fma(Ls[r][l], Zs[l][c], s);
      Zs[r][c] = -s / Ls[r][r];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ib * ib; e += NB) {
    int r = e % ib, cc = e / ib;
    P[(int64_t)(i0 + r) + (int64_t)(i0 + cc) * n] = Zs[r][cc];
  }
}


// ---- FP64 retry of FP32 fronts flagged by the leading-block Cholesky ----------
// Before the leading block is factored: its p x p entries are copied to a
// snapshot S (column-major, ld = p) and its diagonal to the panel's diagonal
// (where k_chol_diag reads the original A_jj).
template <typename T>
__global__ void __launch_bounds__(256) k_retry_prep(const DFront* __restrict__ fr, const T* Kar,
                                                    T* Par, T* S, const int64_t* __restrict__ soff) {
  const DFront d = fr[blockIdx.y];
  const int64_t pp = (int64_t)d.p * d.p;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < pp; e += (int64_t)gridDim.x * 256) {
    const int r = (int)(e % d.p), c = (int)(e / d.p);
    const T v = Kar[d.K + r + (int64_t)c * d.ld];
    S[soff[blockIdx.y] + e] = v;
    if (r == c) Par[d.P + r + (int64_t)c * d.ld] = v;
  }
}

// A flagged front in the FP32 arenas and its FP64 copy.
struct RetryMap {
  int64_t Kf, Pf;   // offsets in the FP32 K and panel arenas
  int64_t Kd, Pd;   // offsets in the FP64 copies
  int64_t S;        // offset of its leading-block snapshot
  int p, ld;        // eliminated count, size (= leading dimension)
};

// FP64 copy of the original front: the leading block from the snapshot, the
// rest (A_NI, A_NN: untouched by the leading-block Cholesky) from K.
__global__ void __launch_bounds__(256) k_retry_build(const RetryMap* __restrict__ mp,
                                                     const float* Kar, const float* S,
                                                     double* Kd) {
  const RetryMap m = mp[blockIdx.y];
  const int64_t tot = (int64_t)m.ld * m.ld;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < tot; e += (int64_t)gridDim.x * 256) {
    const int r = (int)(e % m.ld), c = (int)(e / m.ld);
    const float v = (r < m.p && c < m.p) ? S[m.S + r + (int64_t)c * m.p] : Kar[m.Kf + e];
    Kd[m.Kd + e] = (double)v;
  }
}

// Results of the FP64 partial Cholesky back in FP32: the whole panel
// [Linv; X^T] and the Schur complement (trailing block of K).
__global__ void __launch_bounds__(256) k_retry_writeback(const RetryMap* __restrict__ mp,
                                                         const double* Kd, const double* Pd,
                                                         float* Kar, float* Par) {
  const RetryMap m = mp[blockIdx.y];
  const int64_t np = (int64_t)m.ld * m.p;
  const int nb = m.ld - m.p;
  const int64_t nn = (int64_t)nb * nb;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < np + nn;
       e += (int64_t)gridDim.x * 256) {
    if (e < np) {
      Par[m.Pf + e] = (float)Pd[m.Pd + e];
    } else {
      const int64_t q = e - np;
      const int r = m.p + (int)(q % nb), c = m.p + (int)(q / nb);
      const int64_t o = r + (int64_t)c * m.ld;
      Kar[m.Kf + o] = (float)Kd[m.Kd + o];
    }
  }
}

// ---- generic batched GEMM ------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_gemm(const GemmOp* __restrict__ ops, const T* Ab,
                                              const T* Bb, T* Cb) {
  const GemmOp o = ops[blockIdx.y];
  const int tm = (o.m + TILE - 1) / TILE, tn = (o.n + TILE - 1) / TILE;
  if ((int)blockIdx.x >= tm * tn) return;
  const int rb = (blockIdx.x % tm) * TILE, cb = (blockIdx.x / tm) * TILE;
  if (o.lower && cb >= rb + TILE) return;
  const T* A = Ab + o.A;
  const T* B = Bb + o.B;
  T* C = Cb + o.C;
  __shared__ T As[KC][TILE + 4];
  __shared__ T Bs[KC][TILE + 4];
  TileAcc<T> acc;
  acc.zero();
  for (int k0 = 0; k0 < o.k; k0 += KC) {
    for (int e = threadIdx.x; e < KC * TILE; e += 256) {
      int rr, kk;
      // choose the thread mapping that reads memory contiguously
      if (!o.transA) { rr = e % TILE; kk = e / TILE; } else { kk = e % KC; rr = e / KC; }
      int r = rb + rr, k = k0 + kk;
      T v = T(0);
      if (r < o.m && k < o.k)
        v = o.transA ? A[(int64_t)k + (int64_t)r * o.lda] : A[(int64_t)r + (int64_t)k * o.lda];
      As[kk][rr] = v;
      int cc;
      if (o.transB) { cc = e % TILE; kk = e / TILE; } else { kk = e % KC; cc = e / KC; }
      int c = cb + cc;
      k = k0 + kk;
      v = T(0);
      if (c < o.n && k < o.k)
        v = o.transB ? B[(int64_t)c + (int64_t)k * o.ldb] : B[(int64_t)k + (int64_t)c * o.ldb];
      Bs[kk][cc] = v;
    }
    __syncthreads();
    acc.mma(As, Bs, KC);
    __syncthreads();
  }
  const int tr = (threadIdx.x % 16) * 4, tc = (threadIdx.x / 16) * 4;
  const T alpha = (T)o.alpha, beta = (T)o.beta;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = cb + tc + j;
    if (c >= o.n) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rb + tr + i;
      if (r >= o.m) continue;
      T* cp = &C[(int64_t)r + (int64_t)c * o.ldc];
      *cp = (beta == T(0) ? T(0) : beta * *cp) + alpha * acc.v[i][j];
    }
  }
}

// ---- batched GEMV --------------------------------------------------------------
constexpr int GEMV_ROWS = 128;   // rows of y per CTA (N form)
constexpr int GEMV_WARPS = 8;    // column classes per CTA (N form)

// y = alpha M x (+ y): a CTA owns 128 rows; its 8 warps take the columns
// c = w, w + 8, ... (each warp reads 128 contiguous rows of a column, 4 per
// lane), and the 8 partial sums are added in warp order in shared memory,
// so the result does not depend on timing.  x and y hold R right-hand sides
// vs apart.  The same body serves one handle's ops (offsets from the
// factor's arenas) and grouped ops of several handles (absolute pointers),
// so a grouped apply is bitwise the handle's own.
template <typename T, int R>
__device__ __forceinline__ void gemv_n_body(const T* __restrict__ M, const T* xw, T* yw, int64_t vs,
                                            int rows, int cols, int ld, int tri, float alpha,
                                            int beta_one) {
  const int r0 = blockIdx.x * GEMV_ROWS;
  if (r0 >= rows) return;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __shared__ T red[GEMV_WARPS][GEMV_ROWS];
  T acc[4][R];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int q = 0; q < R; ++q) acc[j][q] = T(0);
  const int cend = tri ? min(cols, r0 + GEMV_ROWS) : cols;
  for (int c = warp; c < cend; c += GEMV_WARPS) {
    T xv[R];
#pragma unroll
    for (int q = 0; q < R; ++q) xv[q] = xw[q * vs + c];
    const T* mc = M + (int64_t)c * ld;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + lane + 32 * j;
      if (r < rows && (!tri || c <= r)) {
        const T mv = mc[r];
#pragma unroll
        for (int q = 0; q < R; ++q) acc[j][q] = fma(mv, xv[q], acc[j][q]);
      }
    }
  }
  const T al = (T)alpha;
#pragma unroll
  for (int q = 0; q < R; ++q) {
#pragma unroll
    for (int j = 0; j < 4; ++j) red[warp][lane + 32 * j] = acc[j][q];
    __syncthreads();
    if (threadIdx.x < GEMV_ROWS) {
      const int r = r0 + threadIdx.x;
      T s = red[0][threadIdx.x];
#pragma unroll
      for (int w = 1; w < GEMV_WARPS; ++w) s += red[w][threadIdx.x];
      if (r < rows) {
        T* yp = &yw[q * vs + r];
        *yp = (beta_one ? *yp : T(0)) + al * s;
      }
    }
    __syncthreads();
  }
}

// y = alpha M^T x (+ y): one warp per output column, lanes stride the rows,
// butterfly reduction.
template <typename T, int R>
__device__ __forceinline__ void gemv_t_body(const T* __restrict__ M, const T* xw, T* yw, int64_t vs,
                                            int rows, int cols, int ld, int tri, float alpha,
                                            int beta_one) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int c = blockIdx.x * 8 + warp;
  if (c >= cols) return;
  const T* Mc = M + (int64_t)c * ld;
  T acc[R];
#pragma unroll
  for (int q = 0; q < R; ++q) acc[q] = T(0);
  for (int r = (tri ? c : 0) + lane; r < rows; r += 32) {
    const T mv = Mc[r];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] = fma(mv, xw[q * vs + r], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) {
    T v = acc[q];
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    acc[q] = v;
  }
  if (lane == 0) {
    const T al = (T)alpha;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      T* yp = &yw[q * vs + c];
      *yp = (beta_one ? *yp : T(0)) + al * acc[q];
    }
  }
}

template <typename T, int R>
__global__ void __launch_bounds__(GEMV_ROWS * 2) k_gemv_n(const GemvOp* __restrict__ ops,
                                                          const T* __restrict__ Mar, T* work,
                                                          int64_t vs) {
  const GemvOp o = ops[blockIdx.y];
  gemv_n_body<T, R>(Mar + o.M, work + o.x, work + o.y, vs, o.rows, o.cols, o.ld, o.tri, o.alpha,
                    o.beta_one);
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_gemv_t(const GemvOp* __restrict__ ops,
                                                const T* __restrict__ Mar, T* work, int64_t vs) {
  const GemvOp o = ops[blockIdx.y];
  gemv_t_body<T, R>(Mar + o.M, work + o.x, work + o.y, vs, o.rows, o.cols, o.ld, o.tri, o.alpha,
                    o.beta_one);
}

// Grouped launches: blockIdx.y (plus y0) runs op j of the launch, which is op
// j - first of the segment that holds it (one factor's mat-vec list for one
// block of right-hand sides).
template <typename T>
__device__ __forceinline__ const GemvSeg<T>& find_seg(const GemvSeg<T>* segs, int nseg, int64_t j) {
  int k = 0;
  while (k + 1 < nseg && segs[k + 1].first <= j) ++k;
  return segs[k];
}

template <typename T, int R>
__global__ void __launch_bounds__(GEMV_ROWS * 2) k_gemv_n_seg(const GemvSeg<T>* __restrict__ segs,
                                                              int nseg, int64_t y0) {
  const int64_t j = y0 + blockIdx.y;
  const GemvSeg<T> sg = find_seg(segs, nseg, j);
  const GemvOp o = sg.ops[j - sg.first];
  gemv_n_body<T, R>(sg.M + o.M, sg.w + o.x, sg.w + o.y, sg.vs, o.rows, o.cols, o.ld, o.tri,
                    o.alpha, o.beta_one);
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_gemv_t_seg(const GemvSeg<T>* __restrict__ segs, int nseg,
                                                    int64_t y0) {
  const int64_t j = y0 + blockIdx.y;
  const GemvSeg<T> sg = find_seg(segs, nseg, j);
  const GemvOp o = sg.ops[j - sg.first];
  gemv_t_body<T, R>(sg.M + o.M, sg.w + o.x, sg.w + o.y, sg.vs, o.rows, o.cols, o.ld, o.tri,
                    o.alpha, o.beta_one);
}

}  // namespace

// ---- host wrappers ---------------------------------------------------------------

// products at least this large (rows of X^T) go to the tensor cores (FP32)
constexpr int TC_MIN_ROWS = 256;

template <typename T>
void finish_fronts(const DFront* d_fronts, const DFront* h_fronts, int nfront, T* Karena,
                   T* Parena, int* d_flags, bool use_tc, cudaStream_t st);

// Refactor the flagged FP32 fronts entirely in FP64 (from the snapshot of
// their leading blocks and their untouched A_NI, A_NN) and store the results
// in the FP32 arenas.
static void retry_fronts_fp64(const std::vector<int>& bad, const DFront* h_fronts,
                       const std::vector<int64_t>& soff, float* Karena, float* Parena,
                       const float* snap, int* d_flags, cudaStream_t st) {
  const int nb = (int)bad.size();
  std::vector<DFront> dl;
  std::vector<RetryMap> maps;
  int64_t kt = 0, pt = 0, mx = 0;
  for (int f : bad) {
    const DFront& h = h_fronts[f];
    dl.push_back(DFront{kt, pt, h.n, h.p, h.id, h.ld});
    maps.push_back(RetryMap{h.K, h.P, kt, pt, soff[f], h.p, h.ld});
    kt += (int64_t)h.ld * h.ld;
    pt += (int64_t)h.ld * h.p;
    mx = std::max<int64_t>(mx, (int64_t)h.ld * h.ld);
  }
  double* Kd = nullptr;
  double* Pd = nullptr;
  RetryMap* d_maps = nullptr;
  DFront* d_dl = nullptr;
  HIF_CUDA_TRY(cudaMallocAsync(&Kd, sizeof(double) * kt, st));
  HIF_CUDA_TRY(cudaMallocAsync(&Pd, sizeof(double) * std::max<int64_t>(1, pt), st));
  HIF_CUDA_TRY(cudaMallocAsync(&d_maps, sizeof(RetryMap) * nb, st));
  HIF_CUDA_TRY(cudaMallocAsync(&d_dl, sizeof(DFront) * nb, st));
  HIF_CUDA_TRY(cudaMemsetAsync(Pd, 0, sizeof(double) * std::max<int64_t>(1, pt), st));
  HIF_CUDA_TRY(cudaMemcpyAsync(d_maps, maps.data(), sizeof(RetryMap) * nb, cudaMemcpyHostToDevice, st));
  HIF_CUDA_TRY(cudaMemcpyAsync(d_dl, dl.data(), sizeof(DFront) * nb, cudaMemcpyHostToDevice, st));
  const int gx = std::max(1, std::min(1024, ceil_div(mx, 256)));
  for (int f0 = 0; f0 < nb; f0 += MAX_GRID_Y) {
    const int c = std::min(MAX_GRID_Y, nb - f0);
    ProfScope ps("chol_retry_fp64", st);
    k_retry_build<<<dim3(gx, c), 256, 0, st>>>(d_maps + f0, Karena, snap, Kd);
    HIF_CHECK_LAUNCH();
  }
  partial_cholesky<double>(d_dl, dl.data(), nb, Kd, Pd, d_flags, false, st, nullptr);
  for (int f0 = 0; f0 < nb; f0 += MAX_GRID_Y) {
    const int c = std::min(MAX_GRID_Y, nb - f0);
    ProfScope ps("chol_retry_fp64", st);
    k_retry_writeback<<<dim3(gx, c), 256, 0, st>>>(d_maps + f0, Kd, Pd, Karena, Parena);
    HIF_CHECK_LAUNCH();
  }
  HIF_CUDA_TRY(cudaFreeAsync(d_dl, st));
  HIF_CUDA_TRY(cudaFreeAsync(d_maps, st));
  HIF_CUDA_TRY(cudaFreeAsync(Pd, st));
  HIF_CUDA_TRY(cudaFreeAsync(Kd, st));
}

template <typename T>
void partial_cholesky(const DFront* d_fronts, const DFront* h_fronts, int nfront, T* Karena,
                      T* Parena, int* d_flags, bool tensor_cores, cudaStream_t st,
                      const RetryOpts* retry) {
  if (nfront == 0) return;
  const bool use_tc = std::is_same<T, float>::value && tensor_cores;
  const int pmax = h_fronts[0].p;
  // FP32 fronts that may be retried in FP64: snapshot of every leading block,
  // original diagonal in the panel, one flag per front
  const bool growth_on = std::is_same<T, float>::value && retry && retry->growth > 0.0;
  int* d_fflag = nullptr;
  T* snap = nullptr;
  int64_t* d_soff = nullptr;
  std::vector<int64_t> soff;
  if (growth_on) {
    soff.resize(nfront);
    int64_t tot = 0, mx = 1;
    for (int f = 0; f < nfront; ++f) {
      soff[f] = tot;
      tot += (int64_t)h_fronts[f].p * h_fronts[f].p;
      mx = std::max<int64_t>(mx, (int64_t)h_fronts[f].p * h_fronts[f].p);
    }
    HIF_CUDA_TRY(cudaMallocAsync(&d_fflag, sizeof(int) * nfront, st));
    HIF_CUDA_TRY(cudaMallocAsync(&snap, sizeof(T) * std::max<int64_t>(1, tot), st));
    HIF_CUDA_TRY(cudaMallocAsync(&d_soff, sizeof(int64_t) * nfront, st));
    HIF_CUDA_TRY(cudaMemsetAsync(d_fflag, 0, sizeof(int) * nfront, st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_soff, soff.data(), sizeof(int64_t) * nfront,
                                 cudaMemcpyHostToDevice, st));
    const int gx = std::max(1, std::min(1024, ceil_div(mx, 256)));
    for (int f0 = 0; f0 < nfront; f0 += MAX_GRID_Y) {
      const int c = std::min(MAX_GRID_Y, nfront - f0);
      ProfScope ps("chol_retry_snapshot", st, 0.0, 2.0 * sizeof(T) * tot);
      k_retry_prep<T><<<dim3(gx, c), 256, 0, st>>>(d_fronts + f0, Karena, Parena, snap, d_soff + f0);
      HIF_CHECK_LAUNCH();
    }
  }
  // 1. Cholesky of the leading p x p block (right-looking, panels of NB):
  //    the kernels see extent p, leading dimension n
  std::vector<DFront> lead(h_fronts, h_fronts + nfront);
  for (auto& f : lead) f.n = f.p;
  DFront* d_lead = nullptr;
  HIF_CUDA_TRY(cudaMallocAsync(&d_lead, sizeof(DFront) * nfront, st));
  HIF_CUDA_TRY(cudaMemcpyAsync(d_lead, lead.data(), sizeof(DFront) * nfront,
                               cudaMemcpyHostToDevice, st));
  // two levels: inner panels of NB factor an outer block of NB2 columns and
  // update only its remaining columns; the rows and columns right of the
  // outer block then get one rank-NB2 update A22 -= L21 L21^T as a batched
  // product (tensor cores for FP32)
  constexpr int NB2 = 256;
  const bool outer = pmax > NB2;
  for (int J0 = 0; J0 < pmax; J0 += NB2) {
    const int jend = outer ? J0 + NB2 : INT_MAX;
    for (int j0 = J0; j0 < std::min(pmax, J0 + NB2); j0 += NB) {
      int nact = 0;
      while (nact < nfront && lead[nact].p > j0) ++nact;
      const int nm = lead[0].p;   // fronts are sorted by p, largest first
      const int j1min = j0 + 1;   // smallest possible j1 among active fronts
      const int chunks = ceil_div(std::max(0, nm - j1min), PANEL_ROWS);
      const int ntile = ceil_div(std::max(0, nm - j1min), TILE);
      const int nctile = outer ? std::max(1, ceil_div(std::max(0, jend - j1min), TILE)) : 0;
      const int grid = outer ? std::max(1, ntile * nctile) : std::max(1, ntile * (ntile + 1) / 2);
      // algorithmic counts of this step (only while profiling)
      double pf = 0, pb = 0, sf = 0, sb = 0;
      if (prof_enabled()) {
        for (int f = 0; f < nact; ++f) {
          const double jb = std::min(NB, lead[f].p - j0);
          const double rest = lead[f].p - j0 - jb;
          const double cols = std::min<double>(rest, (double)std::min(jend, lead[f].p) - j0 - jb);
          pf += jb * jb * jb / 3.0 + rest * jb * jb;
          pb += sizeof(T) * (jb * jb / 2.0 + 2.0 * rest * jb);
          sf += (2.0 * rest - cols + 1.0) * cols * jb;
          sb += sizeof(T) * (rest * jb + (2.0 * rest - cols + 1.0) * cols);
        }
      }
      for (int f0 = 0; f0 < nact; f0 += MAX_GRID_Y) {
        const int nb = std::min(MAX_GRID_Y, nact - f0);
        {
          ProfScope ps("chol_panel", st, pf, pb);
          k_chol_diag<T><<<nb, 256, 0, st>>>(d_lead + f0, Karena, Parena, j0, d_flags,
                                             growth_on ? (float)retry->growth : 0.f,
                                             growth_on ? d_fflag + f0 : nullptr);
          HIF_CHECK_LAUNCH();
          if (chunks > 0) {
            k_panel<T><<<dim3(chunks, nb), PANEL_ROWS, 0, st>>>(d_lead + f0, Karena, Parena, j0);
            HIF_CHECK_LAUNCH();
          }
        }
        {
          ProfScope ps("chol_trailing_update", st, sf, sb);
          k_syrk<T><<<dim3(grid, nb), 256, 0, st>>>(d_lead + f0, Karena, j0,
                                                     outer ? jend : INT_MAX);
          HIF_CHECK_LAUNCH();
        }
      }
    }
    if (!outer) break;
    // A22 -= L21 L21^T for the fronts that extend past the outer block
    std::vector<GemmOp> uo;
    for (int f = 0; f < nfront && lead[f].p > jend; ++f) {
      const DFront& h = lead[f];
      const int64_t ld = h.ld;
      const int rest = h.p - jend;
      uo.push_back(GemmOp{h.K + jend + (int64_t)J0 * ld, h.K + jend + (int64_t)J0 * ld,
                          h.K + jend + (int64_t)jend * ld, rest, rest, NB2, (int)ld, (int)ld,
                          (int)ld, 0, 1, -1.f, 1.f, 1, 0});
    }
    if (uo.empty()) continue;
    GemmOp* d_uo = nullptr;
    HIF_CUDA_TRY(cudaMallocAsync(&d_uo, sizeof(GemmOp) * uo.size(), st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_uo, uo.data(), sizeof(GemmOp) * uo.size(),
                                 cudaMemcpyHostToDevice, st));
    if constexpr (std::is_same<T, float>::value) {
      if (use_tc) {
        gemm_tc(d_uo, uo.data(), (int)uo.size(), reinterpret_cast<const float*>(Karena),
                reinterpret_cast<const float*>(Karena), reinterpret_cast<float*>(Karena), d_flags,
                st, "chol_block_update_tc");
      } else {
        gemm_batched<T>(d_uo, uo.data(), (int)uo.size(), Karena, Karena, Karena, st,
                        "chol_block_update");
      }
    } else {
      gemm_batched<T>(d_uo, uo.data(), (int)uo.size(), Karena, Karena, Karena, st,
                      "chol_block_update");
    }
    HIF_CUDA_TRY(cudaFreeAsync(d_uo, st));
  }
  HIF_CUDA_TRY(cudaFreeAsync(d_lead, st));
  // flagged fronts: redone in FP64 now; the others go on in FP32
  std::vector<DFront> keep;
  DFront* d_keep = nullptr;
  if (growth_on) {
    std::vector<int> hf(nfront), bad;
    HIF_CUDA_TRY(cudaMemcpyAsync(hf.data(), d_fflag, sizeof(int) * nfront, cudaMemcpyDeviceToHost, st));
    HIF_CUDA_TRY(cudaStreamSynchronize(st));
    for (int f = 0; f < nfront; ++f) {
      if (hf[f]) bad.push_back(f);
      else keep.push_back(h_fronts[f]);
    }
    if (!bad.empty()) {
      if constexpr (std::is_same<T, float>::value)
        retry_fronts_fp64(bad, h_fronts, soff, Karena, Parena, snap, d_flags, st);
      if (retry->retried) *retry->retried += (int64_t)bad.size();
      if (!keep.empty()) {
        HIF_CUDA_TRY(cudaMallocAsync(&d_keep, sizeof(DFront) * keep.size(), st));
        HIF_CUDA_TRY(cudaMemcpyAsync(d_keep, keep.data(), sizeof(DFront) * keep.size(),
                                     cudaMemcpyHostToDevice, st));
      }
      d_fronts = d_keep;
      h_fronts = keep.data();
      nfront = (int)keep.size();
    }
    HIF_CUDA_TRY(cudaFreeAsync(d_soff, st));
    HIF_CUDA_TRY(cudaFreeAsync(snap, st));
    HIF_CUDA_TRY(cudaFreeAsync(d_fflag, st));
    if (nfront == 0) return;
  }
  finish_fronts(d_fronts, h_fronts, nfront, Karena, Parena, d_flags, use_tc, st);
  if (d_keep) HIF_CUDA_TRY(cudaFreeAsync(d_keep, st));
}

// Steps 2-4 of the partial Cholesky once the leading blocks hold L.
template <typename T>
void finish_fronts(const DFront* d_fronts, const DFront* h_fronts, int nfront, T* Karena,
                   T* Parena, int* d_flags, bool use_tc, cudaStream_t st) {
  const int pmax = h_fronts[0].p;
  // 2. Linv = L^{-1}: invert the NB x NB diagonal blocks, then merge
  //    neighbouring inverted blocks pairwise up a binary tree of widths
  //    s = NB, 2 NB, 4 NB, ...:  inv([A 0; B C]) = [A^-1 0; -C^-1 B A^-1  C^-1]
  //    (two batched products per width: T = B A^-1, then -C^-1 T)
  const int nblk = ceil_div(pmax, NB);
  for (int f0 = 0; f0 < nfront; f0 += MAX_GRID_Y) {
    const int nb = std::min(MAX_GRID_Y, nfront - f0);
    double fl = 0;
    if (prof_enabled())
      for (int f = f0; f < f0 + nb; ++f) fl += (double)h_fronts[f].p * NB * NB / 3.0;
    ProfScope ps("trtri_diag", st, fl, 0.0);
    k_trtri_diag<T><<<dim3(nblk, nb), NB, 0, st>>>(d_fronts + f0, Parena);
    HIF_CHECK_LAUNCH();
  }
  for (int s = NB; s < pmax; s *= 2) {
    std::vector<GemmOp> tops, rops;
    int64_t scr = 0;
    for (int f = 0; f < nfront && h_fronts[f].p > s; ++f) {
      const DFront& h = h_fronts[f];
      const int ld = h.ld;
      for (int i0 = 0; i0 + s < h.p; i0 += 2 * s) {
        const int rs = std::min(2 * s, h.p - i0) - s;   // rows of the right part
        const int64_t boff = (i0 + s) + (int64_t)i0 * ld;
        const int64_t aoff = i0 + (int64_t)i0 * ld;
        const int64_t coff = (i0 + s) + (int64_t)(i0 + s) * ld;
        tops.push_back(GemmOp{h.K + boff, h.P + aoff, scr, rs, s, s, ld, ld, rs, 0, 0, 1.f, 0.f, 0, 0});
        rops.push_back(GemmOp{h.P + coff, scr, h.P + boff, rs, s, rs, ld, rs, ld, 0, 0, -1.f, 0.f, 0, 0});
        scr += (int64_t)rs * s;
      }
    }
    if (tops.empty()) break;
    const size_t cnt = tops.size();
    GemmOp* d_ops = nullptr;
    T* d_scr = nullptr;
    HIF_CUDA_TRY(cudaMallocAsync(&d_ops, sizeof(GemmOp) * 2 * cnt, st));
    HIF_CUDA_TRY(cudaMallocAsync(&d_scr, sizeof(T) * scr, st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_ops, tops.data(), sizeof(GemmOp) * cnt, cudaMemcpyHostToDevice, st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_ops + cnt, rops.data(), sizeof(GemmOp) * cnt,
                                 cudaMemcpyHostToDevice, st));
    if constexpr (std::is_same<T, float>::value) {
      if (use_tc && s >= 128) {
        gemm_tc(d_ops, tops.data(), (int)cnt, Karena, Parena, d_scr, d_flags, st, "trtri_merge_tc");
        gemm_tc(d_ops + cnt, rops.data(), (int)cnt, Parena, d_scr, Parena, d_flags, st, "trtri_merge_tc");
      } else {
        gemm_batched<T>(d_ops, tops.data(), (int)cnt, Karena, Parena, d_scr, st, "trtri_merge");
        gemm_batched<T>(d_ops + cnt, rops.data(), (int)cnt, Parena, d_scr, Parena, st, "trtri_merge");
      }
    } else {
      gemm_batched<T>(d_ops, tops.data(), (int)cnt, Karena, Parena, d_scr, st, "trtri_merge");
      gemm_batched<T>(d_ops + cnt, rops.data(), (int)cnt, Parena, d_scr, Parena, st, "trtri_merge");
    }
    HIF_CUDA_TRY(cudaFreeAsync(d_scr, st));
    HIF_CUDA_TRY(cudaFreeAsync(d_ops, st));
  }
  // 3. X^T = A_NI L^{-T} (into the panel below Linv) and 4. the Schur
  //    complement A_NN -= X^T X (lower tiles), each one deep product per front
  std::vector<GemmOp> xo, so;
  int maxrows = 0;
  for (int f = 0; f < nfront; ++f) {
    const DFront& h = h_fronts[f];
    const int nb = h.n - h.p;
    if (nb <= 0 || h.p <= 0) continue;
    const int ld = h.ld;
    GemmOp x{h.K + h.p, h.P, h.P + h.p, nb, h.p, h.p, ld, ld, ld, 0, 1, 1.f, 0.f, 0, 0};
    GemmOp s{h.P + h.p, h.P + h.p, h.K + h.p + (int64_t)h.p * ld, nb, nb, h.p, ld, ld, ld, 0, 1,
             -1.f, 1.f, 1, 0};
    xo.push_back(x);
    so.push_back(s);
    maxrows = std::max(maxrows, nb);
  }
  if (!xo.empty()) {
    GemmOp* d_ops = nullptr;
    const size_t cnt = xo.size();
    HIF_CUDA_TRY(cudaMallocAsync(&d_ops, sizeof(GemmOp) * 2 * cnt, st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_ops, xo.data(), sizeof(GemmOp) * cnt, cudaMemcpyHostToDevice, st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_ops + cnt, so.data(), sizeof(GemmOp) * cnt,
                                 cudaMemcpyHostToDevice, st));
    if (use_tc && maxrows >= TC_MIN_ROWS) {
      gemm_tc(d_ops, xo.data(), (int)cnt, reinterpret_cast<const float*>(Karena),
              reinterpret_cast<const float*>(Parena), reinterpret_cast<float*>(Parena), d_flags, st);
      gemm_tc(d_ops + cnt, so.data(), (int)cnt, reinterpret_cast<const float*>(Parena),
              reinterpret_cast<const float*>(Parena), reinterpret_cast<float*>(Karena), d_flags, st);
    } else {
      gemm_batched<T>(d_ops, xo.data(), (int)cnt, Karena, Parena, Parena, st);
      gemm_batched<T>(d_ops + cnt, so.data(), (int)cnt, Parena, Parena, Karena, st);
    }
    HIF_CUDA_TRY(cudaFreeAsync(d_ops, st));
  }
}

template <typename T>
void gemm_batched(const GemmOp* d_ops, const GemmOp* h_ops, int nops, const T* Abase,
                  const T* Bbase, T* Cbase, cudaStream_t st, const char* name) {
  if (nops == 0) return;
  int mt = 1;
  for (int i = 0; i < nops; ++i)
    mt = std::max(mt, ceil_div(h_ops[i].m, TILE) * ceil_div(h_ops[i].n, TILE));
  for (int f0 = 0; f0 < nops; f0 += MAX_GRID_Y) {
    const int nb = std::min(MAX_GRID_Y, nops - f0);
    double fl = 0;
    if (prof_enabled())
      for (int i = f0; i < f0 + nb; ++i) fl += 2.0 * h_ops[i].m * (double)h_ops[i].n * h_ops[i].k;
    ProfScope ps(name, st, fl, 0.0);
    k_gemm<T><<<dim3(mt, nb), 256, 0, st>>>(d_ops + f0, Abase, Bbase, Cbase);
    HIF_CHECK_LAUNCH();
  }
}

template <typename T>
void gemv_batched(const GemvOp* d_ops, const GemvOp* h_ops, int nops, int trans,
                  const T* Marena, T* work, int64_t vstride, int nrhs, cudaStream_t st) {
  if (nops == 0) return;
  int mx = 1;
  for (int i = 0; i < nops; ++i)
    mx = std::max(mx, trans ? ceil_div(h_ops[i].cols, 8) : ceil_div(h_ops[i].rows, GEMV_ROWS));
  // right-hand sides in blocks of 16, 8, 4, 2, 1: each block reads the
  // factor once, and every column sees the same arithmetic in any block
  for (int q0 = 0; q0 < nrhs;) {
    const int left = nrhs - q0;
    const int R = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    T* w = work + (int64_t)q0 * vstride;
    for (int f0 = 0; f0 < nops; f0 += MAX_GRID_Y) {
      const int nb = std::min(MAX_GRID_Y, nops - f0);
      dim3 grid(mx, nb);
      double by = 0, fl = 0;
      if (prof_enabled()) {
        for (int i = f0; i < f0 + nb; ++i) {
          const GemvOp& o = h_ops[i];
          double ent = (double)o.rows * o.cols;
          if (o.tri) ent = 0.5 * (double)o.cols * (o.cols + 1);
          by += sizeof(T) * (ent + (double)R * (o.rows + o.cols) * (o.beta_one ? 1.5 : 1.0));
          fl += 2.0 * ent * R;
        }
      }
      ProfScope ps(trans ? "apply_gemv_t" : "apply_gemv_n", st, fl, by);
      if (trans) {
        switch (R) {
          case 16: k_gemv_t<T, 16><<<grid, 256, 0, st>>>(d_ops + f0, Marena, w, vstride); break;
          case 8: k_gemv_t<T, 8><<<grid, 256, 0, st>>>(d_ops + f0, Marena, w, vstride); break;
          case 4: k_gemv_t<T, 4><<<grid, 256, 0, st>>>(d_ops + f0, Marena, w, vstride); break;
          case 2: k_gemv_t<T, 2><<<grid, 256, 0, st>>>(d_ops + f0, Marena, w, vstride); break;
          default: k_gemv_t<T, 1><<<grid, 256, 0, st>>>(d_ops + f0, Marena, w, vstride);
        }
      } else {
        constexpr int TH = GEMV_ROWS * 2;
        switch (R) {
          case 16: k_gemv_n<T, 16><<<grid, TH, 0, st>>>(d_ops + f0, Marena, w, vstride); break;
          case 8: k_gemv_n<T, 8><<<grid, TH, 0, st>>>(d_ops + f0, Marena, w, vstride); break;
          case 4: k_gemv_n<T, 4><<<grid, TH, 0, st>>>(d_ops + f0, Marena, w, vstride); break;
          case 2: k_gemv_n<T, 2><<<grid, TH, 0, st>>>(d_ops + f0, Marena, w, vstride); break;
          default: k_gemv_n<T, 1><<<grid, TH, 0, st>>>(d_ops + f0, Marena, w, vstride);
        }
      }
      HIF_CHECK_LAUNCH();
      }
    q0 += R;
  }
}

template <typename T>
void gemv_segments(const GemvSeg<T>* d_segs, int nseg, int64_t nops, int mx, int trans, int R,
                   double flops, double bytes, cudaStream_t st) {
  if (nops == 0) return;
  ProfScope ps(trans ? "apply_grouped_gemv_t" : "apply_grouped_gemv_n", st, flops, bytes);
  for (int64_t f0 = 0; f0 < nops; f0 += MAX_GRID_Y) {
    const dim3 grid(std::max(1, mx), (unsigned)std::min<int64_t>(MAX_GRID_Y, nops - f0));
    if (trans) {
      switch (R) {
        case 16: k_gemv_t_seg<T, 16><<<grid, 256, 0, st>>>(d_segs, nseg, f0); break;
        case 8: k_gemv_t_seg<T, 8><<<grid, 256, 0, st>>>(d_segs, nseg, f0); break;
        case 4: k_gemv_t_seg<T, 4><<<grid, 256, 0, st>>>(d_segs, nseg, f0); break;
        case 2: k_gemv_t_seg<T, 2><<<grid, 256, 0, st>>>(d_segs, nseg, f0); break;
        default: k_gemv_t_seg<T, 1><<<grid, 256, 0, st>>>(d_segs, nseg, f0);
      }
    } else {
      constexpr int TH = GEMV_ROWS * 2;
      switch (R) {
        case 16: k_gemv_n_seg<T, 16><<<grid, TH, 0, st>>>(d_segs, nseg, f0); break;
        case 8: k_gemv_n_seg<T, 8><<<grid, TH, 0, st>>>(d_segs, nseg, f0); break;
        case 4: k_gemv_n_seg<T, 4><<<grid, TH, 0, st>>>(d_segs, nseg, f0); break;
        case 2: k_gemv_n_seg<T, 2><<<grid, TH, 0, st>>>(d_segs, nseg, f0); break;
        default: k_gemv_n_seg<T, 1><<<grid, TH, 0, st>>>(d_segs, nseg, f0);
      }
    }
    HIF_CHECK_LAUNCH();
  }
}

int gemv_tiles(const GemvOp* h_ops, int nops, int trans) {
  int mx = 1;
  for (int i = 0; i < nops; ++i)
    mx = std::max(mx, trans ? ceil_div(h_ops[i].cols, 8) : ceil_div(h_ops[i].rows, GEMV_ROWS));
  return mx;
}

#define HIF_INST(T)                                                                          \
  template void partial_cholesky<T>(const DFront*, const DFront*, int, T*, T*, int*, bool,  \
                                    cudaStream_t, const RetryOpts*);                         \
  template void gemm_batched<T>(const GemmOp*, const GemmOp*, int, const T*, const T*, T*,  \
                                cudaStream_t, const char*);                                  \
  template void gemv_batched<T>(const GemvOp*, const GemvOp*, int, int, const T*, T*,       \
                                int64_t, int, cudaStream_t);                                 \
  template void gemv_segments<T>(const GemvSeg<T>*, int, int64_t, int, int, int, double,     \
                                 double, cudaStream_t);
HIF_INST(float)
HIF_INST(double)
#undef HIF_INST

}  // namespace hif
