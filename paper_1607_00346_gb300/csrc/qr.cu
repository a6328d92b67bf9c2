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
//   * k_qr_panel (one CTA per front): Householder reflectors of the panel's
//     columns (norms accumulated in double), the explicit reflector matrix V
//     and the triangular T of the compact form Q = I - V T V^T (forward
//     accumulation: T_{j+1} = [T_j, -tau_j T_j V_j^T v_j; 0, tau_j]);
//   * trailing columns: W = V^T A, W = T^T W, A -= V W (batched GEMMs).
#include <algorithm>
#include <cstdlib>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "dense.cuh"
#include "front.cuh"
#include "warp.cuh"

namespace hif {

namespace {

constexpr int QB = 32;          // panel width
constexpr int QR_THREADS = 512;
constexpr int QR_WARPS = QR_THREADS / 32;

struct QRDesc {
  int64_t A;     // matrix (m x n, ld) offset in the gather arena
  int64_t V;     // reflector block (m x QB, ld = m) offset in the V arena
  int64_t W;     // two QB x n work blocks (ld = QB) offset in the W arena
  int64_t Tt;    // QB x QB offset in the T arena
  int m, n, ld;
  int pad;
};

template <typename T>
__global__ void __launch_bounds__(QR_THREADS) k_qr_panel(const QRDesc* __restrict__ ds, T* Gar,
                                                         T* Var, T* Tar, int p) {
  const QRDesc d = ds[blockIdx.x];
  if (p >= d.n) return;
  const int jb = min(QB, d.n - p);
  const int m = d.m, ld = d.ld;
  T* A = Gar + d.A;
  T* V = Var + d.V;
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
    // explicit reflector column j of V (rows p..m-1)
    for (int r = p + tid; r < m; r += QR_THREADS)
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
  T* Tt = Tar + d.Tt;
  for (int e = tid; e < QB * QB; e += QR_THREADS) {
    const int i = e % QB, j = e / QB;
    Tt[e] = (i < jb && j < jb) ? (T)s_T[i][j] : T(0);
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

}  // namespace

// Unpivoted QR of the R rows of fronts `which` (in place in the gather
// arena); their n x n triangular factors go to Rout at rOff (ld = n).
template <typename T>
void reduce_rows_qr(const SkelDesc* h_f, const std::vector<int>& which, T* Garena, T* Rout,
                    const std::vector<int64_t>& rOff, int* d_flags, bool tensor_cores,
                    cudaStream_t st) {
  const int nq = (int)which.size();
  if (nq == 0) return;
  const bool use_tc = std::is_same<T, float>::value && tensor_cores;
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
    voff += (int64_t)d.m * QB;
    woff += 2LL * QB * d.n;
    toff += QB * QB;
    ro[i] = rOff[ord[i]];
  }
  T *Var = nullptr, *War = nullptr, *Tar = nullptr;
  QRDesc* d_qd = nullptr;
  int64_t* d_ro = nullptr;
  GemmOp* d_ops = nullptr;
  HIF_CUDA_TRY(cudaMallocAsync(&Var, sizeof(T) * voff, st));
  HIF_CUDA_TRY(cudaMallocAsync(&War, sizeof(T) * woff, st));
  HIF_CUDA_TRY(cudaMallocAsync(&Tar, sizeof(T) * toff, st));
  HIF_CUDA_TRY(cudaMallocAsync(&d_qd, sizeof(QRDesc) * nq, st));
  HIF_CUDA_TRY(cudaMallocAsync(&d_ro, sizeof(int64_t) * nq, st));
  HIF_CUDA_TRY(cudaMemcpyAsync(d_qd, qd.data(), sizeof(QRDesc) * nq, cudaMemcpyHostToDevice, st));
  HIF_CUDA_TRY(cudaMemcpyAsync(d_ro, ro.data(), sizeof(int64_t) * nq, cudaMemcpyHostToDevice, st));
  const int nmax = qd[0].n;
  // GEMM descriptors of every panel, uploaded once
  std::vector<GemmOp> ops;
  std::vector<int64_t> opOff;   // per panel: start of its 3 lists
  std::vector<int> opCnt;
  for (int p = 0; p < nmax; p += QB) {
    opOff.push_back((int64_t)ops.size());
    int cnt = 0;
    for (int i = 0; i < nq; ++i) {
      const QRDesc& d = qd[i];
      if (p >= d.n) break;
      const int jb = std::min(QB, d.n - p);
      const int nt = d.n - p - jb;
      if (nt <= 0) continue;
      ++cnt;
    }
    opCnt.push_back(cnt);
    for (int which_gemm = 0; which_gemm < 3; ++which_gemm) {
      for (int i = 0; i < nq; ++i) {
        const QRDesc& d = qd[i];
        if (p >= d.n) break;
        const int jb = std::min(QB, d.n - p);
        const int nt = d.n - p - jb;
        if (nt <= 0) continue;
        const int mp = d.m - p;
        const int64_t At = d.A + p + (int64_t)(p + jb) * d.ld;
        GemmOp o;
        if (which_gemm == 0)        // W1 = V^T A_t
          o = GemmOp{d.V, At, d.W, jb, nt, mp, d.m, d.ld, QB, 1, 0, 1.f, 0.f};
        else if (which_gemm == 1)   // W2 = T^T W1
          o = GemmOp{d.Tt, d.W, d.W + (int64_t)QB * d.n, jb, nt, jb, QB, QB, QB, 1, 0, 1.f, 0.f};
        else                        // A_t -= V W2
          o = GemmOp{d.V, d.W + (int64_t)QB * d.n, At, mp, nt, jb, d.m, QB, d.ld, 0, 0, -1.f, 1.f};
        ops.push_back(o);
      }
    }
  }
  if (!ops.empty()) {
    HIF_CUDA_TRY(cudaMallocAsync(&d_ops, sizeof(GemmOp) * ops.size(), st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_ops, ops.data(), sizeof(GemmOp) * ops.size(),
                                 cudaMemcpyHostToDevice, st));
  }
  int pi = 0;
  for (int p = 0; p < nmax; p += QB, ++pi) {
    int nact = 0;
    while (nact < nq && qd[nact].n > p) ++nact;
    {
      // algorithmic counts: Householder QR of the (m - p) x jb panel
      // (2 (m-p) jb^2 flops), read and written once, reflectors written to V
      double pf = 0, pb = 0;
      if (prof_enabled())
        for (int i = 0; i < nact; ++i) {
          const double mp = qd[i].m - p, jb = std::min(QB, qd[i].n - p);
          pf += 2.0 * mp * jb * jb;
          pb += 3.0 * sizeof(T) * mp * jb;
        }
      ProfScope ps("id_rowreduce_panel", st, pf, pb);
      k_qr_panel<T><<<nact, QR_THREADS, 0, st>>>(d_qd, Garena, Var, Tar, p);
      HIF_CHECK_LAUNCH();
    }
    const int cnt = opCnt[pi];
    if (cnt == 0) continue;
    const int64_t o0 = opOff[pi];
    // W1 = V^T A_t (deep K) goes to the tensor cores for FP32 fronts; the
    // rank-QB update A_t -= V W2 is a read-modify-write of A_t with K = QB and
    // runs faster on the SIMT kernel, which keeps more CTAs resident per SM
    auto product = [&](int which_gemm, const T* A, const T* B, T* C) {
      const int64_t oi = o0 + (int64_t)which_gemm * cnt;
      if constexpr (std::is_same<T, float>::value) {
        if (use_tc && which_gemm == 0) {
          gemm_tc(d_ops + oi, ops.data() + oi, cnt, A, B, C, d_flags, st);
          return;
        }
      }
      gemm_batched<T>(d_ops + oi, ops.data() + oi, cnt, A, B, C, st);
    };
    product(0, Var, Garena, War);
    product(1, Tar, War, War);
    product(2, Var, War, Garena);
  }
  {
    ProfScope ps("id_rowreduce_extract", st);
    const int64_t mx = (int64_t)nmax * nmax;
    k_extract_r<T><<<dim3(ceil_div(mx, 256), nq), 256, 0, st>>>(d_qd, d_ro, Garena, Rout);
    HIF_CHECK_LAUNCH();
  }
  if (d_ops) HIF_CUDA_TRY(cudaFreeAsync(d_ops, st));
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
