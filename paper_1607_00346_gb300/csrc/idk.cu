// Interpolative decomposition of A_RF for a batch of faces or edges (§2.3):
// column-pivoted Householder QR stopped at |R_ii| <= eps |R_11|, then
// T_F = R11^{-1} R12.
//
// One thread-block cluster per front (1 to 16 CTAs, chosen from the front's
// size).  Column j of the gather buffer belongs to CTA j % CS of the cluster
// and never moves: the pivot order is kept as a permutation.  Each step
//   1. every CTA proposes the largest remaining column norm among its columns;
//      the proposals meet in distributed shared memory and every CTA picks the
//      same winner (largest norm, lowest column index on ties);
//   2. the owner of the pivot column builds the Householder reflector in place;
//   3. every CTA applies it to its own remaining columns and downdates their
//      norms.
// Reflectors and products run in the factor precision T.  Column norms are
// kept in double and downdated after every step (|a_j|^2 -= R_ij^2); when the
// downdate has lost most of the value the norm is recomputed from the column
// (the LAPACK xGEQP3 safeguard).  Rows are never permuted, so R_{l,j} sits in
// row l of column j.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "front.cuh"

namespace cg = cooperative_groups;

namespace hif {

namespace {

constexpr int ID_THREADS = 512;
constexpr int ID_WARPS = ID_THREADS / 32;

constexpr int UNR = 8;   // independent loads in flight per lane in the column passes

// sum_{r in [r0, r1)} a[r] b[r] over one warp (result in every lane)
template <typename T>
__device__ __forceinline__ T warp_dot(const T* __restrict__ a, const T* __restrict__ b, int r0,
                                      int r1, int lane) {
  T acc[4] = {T(0), T(0), T(0), T(0)};
  int r = r0 + lane;
  for (; r + 32 * (UNR - 1) < r1; r += 32 * UNR) {
    T x[UNR], y[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      x[u] = a[r + 32 * u];
      y[u] = b[r + 32 * u];
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) acc[u & 3] = fma(x[u], y[u], acc[u & 3]);
  }
  for (; r < r1; r += 32) acc[0] = fma(a[r], b[r], acc[0]);
  T s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// b[r] -= t a[r] for r in [r0, r1), one warp
template <typename T>
__device__ __forceinline__ void warp_axpy(T t, const T* __restrict__ a, T* __restrict__ b, int r0,
                                          int r1, int lane) {
  int r = r0 + lane;
  for (; r + 32 * (UNR - 1) < r1; r += 32 * UNR) {
    T x[UNR], y[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      x[u] = a[r + 32 * u];
      y[u] = b[r + 32 * u];
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) b[r + 32 * u] = fma(-t, x[u], y[u]);
  }
  for (; r < r1; r += 32) b[r] = fma(-t, a[r], b[r]);
}

// sum of squares (double) of a[r0:r1], one warp
template <typename T>
__device__ __forceinline__ double warp_sumsq(const T* __restrict__ a, int r0, int r1, int lane) {
  double acc[2] = {0.0, 0.0};
  int r = r0 + lane;
  for (; r + 32 * (UNR - 1) < r1; r += 32 * UNR) {
    T x[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) x[u] = a[r + 32 * u];
#pragma unroll
    for (int u = 0; u < UNR; ++u) acc[u & 1] += (double)x[u] * (double)x[u];
  }
  for (; r < r1; r += 32) acc[0] += (double)a[r] * (double)a[r];
  double s = acc[0] + acc[1];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <typename T>
__global__ void __launch_bounds__(ID_THREADS) k_cpqr(SkelDesc* fr, const int* __restrict__ list,
                                                     T* Gar, int32_t* permAr, T* Far,
                                                     double* scratch, int32_t* stepAr, double eps) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int fidx = list[blockIdx.x / CS];
  SkelDesc& fref = fr[fidx];
  const SkelDesc f = fref;
  const int nF = f.nF, m = f.nR, ld = nF + m;
  T* M = Gar + f.G + nF;            // the R rows; column c at M + c*ld
  int32_t* pv = permAr + f.perm;
  int32_t* stepOf = stepAr + f.perm;
  double* nrm = scratch + 2 * f.perm;
  double* ref = nrm + nF;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  __shared__ double s_val[ID_WARPS];
  __shared__ int s_idx[ID_WARPS];
  __shared__ double s_cand_val;
  __shared__ int s_cand_idx;
  __shared__ double s_tau, s_v0;
  __shared__ int s_piv, s_stop;
  __shared__ double s_r11;

  // initial norms of my columns
  for (int c = rank + CS * warp; c < nF; c += CS * ID_WARPS) {
    const double s = warp_sumsq(M + (int64_t)c * ld, 0, m, lane);
    if (lane == 0) {
      nrm[c] = s;
      ref[c] = s;
      stepOf[c] = -1;
    }
  }
  __syncthreads();
  const int kmax = min(m, nF);
  int k = kmax;
  for (int i = 0; i < kmax; ++i) {
    // 1. local proposal
    double bv = -1.0;
    int bi = nF;
    for (int c = rank + CS * tid; c < nF; c += CS * ID_THREADS) {
      if (stepOf[c] >= 0) continue;
      const double v = nrm[c];
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
    // 2. the cluster-wide winner (same in every CTA)
    if (tid == 0) {
      double v = -1.0;
      int ix = nF;
      for (int q = 0; q < CS; ++q) {
        const double ov = *cl.map_shared_rank(&s_cand_val, q);
        const int oi = *cl.map_shared_rank(&s_cand_idx, q);
        if (ov > v || (ov == v && oi < ix)) {
          v = ov;
          ix = oi;
        }
      }
      const double nv = sqrt(fmax(v, 0.0));
      if (i == 0) s_r11 = nv;
      s_stop = (ix >= nF) || ((i == 0) ? (nv == 0.0) : !(nv > eps * s_r11));
      s_piv = ix;
    }
    __syncthreads();
    if (s_stop) {
      k = i;
      break;
    }
    const int piv = s_piv;
    const int owner = piv % CS;
    T* cp = M + (int64_t)piv * ld;
    if (owner == rank) {
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
        s_tau = vtv > 0.0 ? 2.0 / vtv : 0.0;
        s_v0 = v0;
        cp[i] = (T)alpha;    // R_ii; v0 lives in shared memory
        pv[i] = piv;
        stepOf[piv] = i;
      }
    }
    cl.sync();
    // 3. apply the reflector v = [v0; cp[i+1:m]] to my remaining columns
    const double tau_d = *cl.map_shared_rank(&s_tau, owner);
    const T v0 = (T)*cl.map_shared_rank(&s_v0, owner);
    const T tau = (T)tau_d;
    for (int j = rank + CS * warp; j < nF; j += CS * ID_WARPS) {
      if (stepOf[j] >= 0) continue;
      T* cj = M + (int64_t)j * ld;
      T w = warp_dot(cp, cj, i + 1, m, lane);
      w = fma(v0, cj[i], w);
      const T tw = tau * w;
      warp_axpy(tw, cp, cj, i + 1, m, lane);
      __syncwarp();
      if (lane == 0) cj[i] = fma(-tw, v0, cj[i]);
      __syncwarp();
      // downdate |a_j|^2 by R_ij^2 in double; recompute when mostly cancelled
      const double rij = (double)cj[i];
      double nv = nrm[j] - rij * rij;
      if (nv <= 1e-2 * ref[j]) {
        nv = warp_sumsq(cj, i + 1, m, lane);
        if (lane == 0) ref[j] = nv;
      }
      if (lane == 0) nrm[j] = fmax(nv, 0.0);
    }
    __syncthreads();
  }
  // redundant columns, in increasing column order, follow the pivots in pv
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

}  // namespace

template <typename T>
void interpolative_decomposition(SkelDesc* d_f, const SkelDesc* h_f, int nf, T* Garena,
                                 int32_t* perm, T* Farena, double* scratch, int32_t* stepAr,
                                 double eps, cudaStream_t st) {
  if (nf == 0) return;
  int nsm = 0, dev = 0;
  HIF_CUDA_TRY(cudaGetDevice(&dev));
  HIF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // cluster size per front from its work per step (nF x nR), so that the
  // large fronts of the upper levels spread over up to 16 SMs each
  std::vector<std::vector<int>> bucket(5);
  const int sizes[5] = {1, 2, 4, 8, 16};
  for (int f = 0; f < nf; ++f) {
    const double work = (double)h_f[f].nF * (h_f[f].nF + h_f[f].nR);
    int b = 0;
    if (work > 2.0e5) b = 1;
    if (work > 1.0e6) b = 2;
    if (work > 4.0e6) b = 3;
    if (work > 1.6e7) b = 4;
    // do not spread a few fronts wider than the GPU
    while (b > 0 && (int64_t)nf * sizes[b] > 2 * nsm) --b;
    bucket[b].push_back(f);
  }
  static bool attr_set[2] = {false, false};
  if (!attr_set[sizeof(T) == 8]) {
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_cpqr<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    attr_set[sizeof(T) == 8] = true;
  }
  for (int b = 0; b < 5; ++b) {
    if (bucket[b].empty()) continue;
    const int CS = sizes[b];
    int* d_list = nullptr;
    HIF_CUDA_TRY(cudaMallocAsync(&d_list, sizeof(int) * bucket[b].size(), st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_list, bucket[b].data(), sizeof(int) * bucket[b].size(),
                                 cudaMemcpyHostToDevice, st));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(bucket[b].size() * CS));
    cfg.blockDim = dim3(ID_THREADS);
    cfg.dynamicSmemBytes = 0;
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
      HIF_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_cpqr<T>, d_f, (const int*)d_list, Garena, perm,
                                      Farena, scratch, stepAr, eps));
      HIF_CHECK_LAUNCH();
    }
    HIF_CUDA_TRY(cudaFreeAsync(d_list, st));
  }
}

template void interpolative_decomposition<float>(SkelDesc*, const SkelDesc*, int, float*, int32_t*,
                                                 float*, double*, int32_t*, double, cudaStream_t);
template void interpolative_decomposition<double>(SkelDesc*, const SkelDesc*, int, double*,
                                                  int32_t*, double*, double*, int32_t*, double,
                                                  cudaStream_t);

}  // namespace hif
