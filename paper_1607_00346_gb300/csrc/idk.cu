// Interpolative decomposition of A_RF for a batch of faces or edges (§2.3):
// column-pivoted Householder QR stopped at |R_ii| <= eps |R_11|, then
// T_F = R11^{-1} R12.
//
// One CTA per front; the R rows of the gather buffer are factored in place.
// Reflectors and products run in the factor precision T.  Column norms are
// kept in double and downdated after every step (|a_j|^2 -= R_ij^2); when the
// downdate has lost most of the value the norm is recomputed from the column
// (the LAPACK xGEQP3 safeguard).  Ties between equal norms go to the lowest
// current column index.
#include <algorithm>

#include "common.cuh"
#include "front.cuh"

namespace hif {

namespace {

constexpr int ID_THREADS = 256;
constexpr int ID_WARPS = ID_THREADS / 32;

template <typename T>
__global__ void __launch_bounds__(ID_THREADS) k_cpqr(SkelDesc* fr, T* Gar, int32_t* permAr,
                                                     T* Far, double* scratch, double eps) {
  SkelDesc& fref = fr[blockIdx.x];
  const SkelDesc f = fref;
  const int nF = f.nF, m = f.nR, ld = nF + m;
  T* M = Gar + f.G + nF;            // the R rows; column c at M + c*ld
  int32_t* pv = permAr + f.perm;
  double* nrm = scratch + 2 * f.perm;
  double* ref = nrm + nF;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  __shared__ double s_val[ID_WARPS];
  __shared__ int s_idx[ID_WARPS];
  __shared__ double s_r11, s_alpha, s_tau;
  __shared__ int s_piv, s_stop;

  for (int c = tid; c < nF; c += ID_THREADS) pv[c] = c;
  for (int c = warp; c < nF; c += ID_WARPS) {
    double s = 0.0;
    for (int r = lane; r < m; r += 32) {
      const double v = (double)M[r + (int64_t)c * ld];
      s += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      nrm[c] = s;
      ref[c] = s;
    }
  }
  __syncthreads();
  const int kmax = min(m, nF);
  int k = kmax;
  for (int i = 0; i < kmax; ++i) {
    // pivot: largest remaining norm, lowest index on ties
    double bv = -1.0;
    int bi = nF;
    for (int c = i + tid; c < nF; c += ID_THREADS) {
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
      const double nv = sqrt(fmax(v, 0.0));
      if (i == 0) s_r11 = nv;
      s_stop = (i == 0) ? (nv == 0.0) : !(nv > eps * s_r11);
      s_piv = ix;
    }
    __syncthreads();
    if (s_stop) {
      k = i;
      break;
    }
    const int piv = s_piv;
    if (piv != i) {
      for (int r = tid; r < m; r += ID_THREADS) {
        const T t0 = M[r + (int64_t)i * ld];
        M[r + (int64_t)i * ld] = M[r + (int64_t)piv * ld];
        M[r + (int64_t)piv * ld] = t0;
      }
      if (tid == 0) {
        double t = nrm[i]; nrm[i] = nrm[piv]; nrm[piv] = t;
        t = ref[i]; ref[i] = ref[piv]; ref[piv] = t;
        const int32_t q = pv[i]; pv[i] = pv[piv]; pv[piv] = q;
      }
      __syncthreads();
    }
    // Householder reflector of column i, rows i..m-1
    T* ci = M + (int64_t)i * ld;
    {
      double s = 0.0;
      for (int r = i + 1 + tid; r < m; r += ID_THREADS) {
        const double v = (double)ci[r];
        s += v * v;
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) s_val[warp] = s;
      __syncthreads();
      if (tid == 0) {
        double tail = 0.0;
        for (int w = 0; w < ID_WARPS; ++w) tail += s_val[w];
        const double x0 = (double)ci[i];
        const double nx = sqrt(x0 * x0 + tail);
        const double alpha = x0 >= 0.0 ? -nx : nx;
        const double v0 = x0 - alpha;
        const double vtv = v0 * v0 + tail;
        s_alpha = alpha;
        s_tau = vtv > 0.0 ? 2.0 / vtv : 0.0;
        ci[i] = (T)v0;   // column i now holds v (its R entry is restored below)
      }
      __syncthreads();
    }
    const T tau = (T)s_tau;
    for (int j = i + 1 + warp; j < nF; j += ID_WARPS) {
      T* cj = M + (int64_t)j * ld;
      T w = T(0);
      for (int r = i + lane; r < m; r += 32) w = fma(ci[r], cj[r], w);
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      const T tw = tau * w;
      for (int r = i + lane; r < m; r += 32) cj[r] = fma(-tw, ci[r], cj[r]);
      __syncwarp();
      // downdate |a_j|^2 by R_ij^2 in double; recompute when mostly cancelled
      const double rij = (double)cj[i];
      double nv = nrm[j] - rij * rij;
      if (nv <= 1e-2 * ref[j]) {
        double s = 0.0;
        for (int r = i + 1 + lane; r < m; r += 32) {
          const double v = (double)cj[r];
          s += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        nv = s;
        if (lane == 0) ref[j] = s;
      }
      if (lane == 0) nrm[j] = fmax(nv, 0.0);
    }
    __syncthreads();
    if (tid == 0) ci[i] = (T)s_alpha;
    // column i below the diagonal still holds the reflector; R needs rows <= i only
    __syncthreads();
  }
  if (tid == 0) fref.k = k;
  // T = R11^{-1} R12 (k x (nF-k), ld = k): column-oriented back substitution,
  // one warp per column of R12
  T* Tm = Far + f.Tm;
  for (int j = k + warp; j < nF; j += ID_WARPS) {
    T* b = Tm + (int64_t)(j - k) * k;
    const T* cj = M + (int64_t)j * ld;
    for (int r = lane; r < k; r += 32) b[r] = cj[r];
    __syncwarp();
    for (int ii = k - 1; ii >= 0; --ii) {
      const T xi = b[ii] / M[ii + (int64_t)ii * ld];
      __syncwarp();
      if (lane == 0) b[ii] = xi;
      const T* rc = M + (int64_t)ii * ld;
      for (int r = lane; r < ii; r += 32) b[r] = fma(-xi, rc[r], b[r]);
      __syncwarp();
    }
  }
}

}  // namespace

template <typename T>
void interpolative_decomposition(SkelDesc* d_f, int nf, T* Garena, int32_t* perm, T* Farena,
                                 double* scratch, double eps, cudaStream_t st) {
  if (nf == 0) return;
  k_cpqr<T><<<nf, ID_THREADS, 0, st>>>(d_f, Garena, perm, Farena, scratch, eps);
  HIF_CHECK_LAUNCH();
}

template void interpolative_decomposition<float>(SkelDesc*, int, float*, int32_t*, float*,
                                                 double*, double, cudaStream_t);
template void interpolative_decomposition<double>(SkelDesc*, int, double*, int32_t*, double*,
                                                  double*, double, cudaStream_t);

}  // namespace hif
