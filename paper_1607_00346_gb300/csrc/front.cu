// Moving matrix entries between fronts: stencil coefficients (§2.4), level-0
// frontal matrices, extend-add of the children into a parent cell (the merge
// of §3.2, done in device memory), the gather of A_{[F;R],F} for a face or
// edge (§2.3) and the write-back of B_{F^F^}.
//
// Frontal matrices are symmetric; only their lower triangle is read or written
// (entry (a,b) lives at K[max(a,b) + min(a,b)*n]).
#include <algorithm>

#include "front.cuh"

namespace hif {

namespace {

constexpr int MAX_GRID_Y = 65535;

__device__ __forceinline__ double harmonic(double p, double q) { return 2.0 * p * q / (p + q); }

// Dirichlet: h = 1/(n+1), a neighbour outside the grid adds its coupling
// (a_j) to the diagonal only.  Periodic: h = 1/n, the last plane couples to
// the first, and b must be positive (otherwise the constant is a null vector).
__global__ void k_stencil(const double* __restrict__ a, const double* __restrict__ b,
                          double b_const, int n, int periodic, double* cpl, double* diag,
                          int* bad) {
  const int64_t N = (int64_t)n * n * n;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const int x[3] = {(int)(j % n), (int)((j / n) % n), (int)(j / ((int64_t)n * n))};
  const int64_t stride[3] = {1, n, (int64_t)n * n};
  const double h = periodic ? 1.0 / n : 1.0 / (n + 1);
  const double ih2 = 1.0 / (h * h);
  const double aj = a[j];
  const double bj = b ? b[j] : b_const;
  if (!(aj > 0.0) || !isfinite(aj) || !(bj >= 0.0) || !isfinite(bj) || (periodic && !(bj > 0.0)))
    atomicExch(bad, 1);
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    double cm, cp;
    if (periodic) {
      const int64_t jm = x[d] > 0 ? j - stride[d] : j + (int64_t)(n - 1) * stride[d];
      const int64_t jp = x[d] + 1 < n ? j + stride[d] : j - (int64_t)(n - 1) * stride[d];
      cm = harmonic(a[jm], aj);
      cp = harmonic(aj, a[jp]);
      cpl[d * N + j] = cp * ih2;
    } else {
      cm = x[d] > 0 ? harmonic(a[j - stride[d]], aj) : aj;
      cp = x[d] + 1 < n ? harmonic(aj, a[j + stride[d]]) : aj;
      cpl[d * N + j] = x[d] + 1 < n ? cp * ih2 : 0.0;
    }
    s += cm + cp;
  }
  diag[j] = s * ih2 + bj;
}

// The cell (coordinate along one dimension) that owns point x at cell side
// s: a separator plane belongs to the cell below it (wrapping to the last
// cell on the periodic grid, where plane 0 is a separator too).
__device__ __forceinline__ int lowcell(int x, int s, int C, int periodic) {
  if (periodic) return x % s == 0 ? (x / s + C - 1) % C : x / s;
  return (x != 0 && x % s == 0) ? x / s - 1 : x / s;
}

// The cell's closure is the box [s c, s (c+1)] per dimension (clipped to the
// grid with a Dirichlet boundary, wrapping to plane 0 on the periodic grid);
// points are addressed by their offset from the box's low corner.
template <typename T>
__global__ void k_assemble0(const CellDesc* __restrict__ cells, const int32_t* __restrict__ lists,
                            int n, int s, int periodic, const double* __restrict__ cpl,
                            const double* __restrict__ diag, T* Kar) {
  extern __shared__ int boxmap[];
  const CellDesc cd = cells[blockIdx.x];
  const int C = n / s;
  const int c[3] = {(int)(blockIdx.x % C), (int)((blockIdx.x / C) % C), (int)(blockIdx.x / (C * C))};
  int lo[3], B[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = s * c[d];
    B[d] = periodic ? s + 1 : min(s * (c[d] + 1), n - 1) - lo[d] + 1;
  }
  const int32_t* lst = lists + cd.list;
  const int64_t N = (int64_t)n * n * n;
  for (int a = threadIdx.x; a < cd.n; a += blockDim.x) {
    const int g = lst[a];
    const int x[3] = {g % n, (g / n) % n, g / (n * n)};
    int xl[3];
    for (int d = 0; d < 3; ++d) xl[d] = (x[d] - lo[d] + n) % n;
    boxmap[xl[0] + B[0] * (xl[1] + B[1] * xl[2])] = a;
  }
  __syncthreads();
  T* K = Kar + cd.K;
  const int nc = cd.n;
  for (int a = threadIdx.x; a < nc; a += blockDim.x) {
    const int g = lst[a];
    const int x[3] = {g % n, (g / n) % n, g / (n * n)};
    int xl[3];
    for (int d = 0; d < 3; ++d) xl[d] = (x[d] - lo[d] + n) % n;
    bool own = true;
    for (int d = 0; d < 3; ++d) own = own && lowcell(x[d], s, C, periodic) == c[d];
    if (own) K[(int64_t)a + (int64_t)a * nc] = (T)diag[g];
    for (int d = 0; d < 3; ++d) {
      // the coupling of x with its +e_d neighbour, if the box holds both
      if (xl[d] + 1 >= B[d]) continue;
      bool ownp = x[d] / s == c[d];
      for (int e = 0; e < 3; ++e)
        if (e != d) ownp = ownp && lowcell(x[e], s, C, periodic) == c[e];
      if (!ownp) continue;
      int y[3] = {xl[0], xl[1], xl[2]};
      y[d] += 1;
      const int b = boxmap[y[0] + B[0] * (y[1] + B[1] * y[2])];
      const int hi_ = max(a, b), lo_ = min(a, b);
      K[(int64_t)hi_ + (int64_t)lo_ * nc] = (T)(-cpl[d * N + g]);
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

template <typename T>
__global__ void __launch_bounds__(256) k_merge(const MergeDesc* __restrict__ par,
                                               const CellDesc* __restrict__ child,
                                               const int32_t* __restrict__ maps,
                                               const T* __restrict__ Kc, T* Kp) {
  const MergeDesc pd = par[blockIdx.y];
  const int n = pd.n;
  const int nt = (n + 63) / 64;
  if ((int)blockIdx.x >= nt * (nt + 1) / 2) return;
  int ti, tj;
  tri_index(blockIdx.x, ti, tj);
  __shared__ int rmap[8][64];
  __shared__ int cmap[8][64];
  __shared__ int64_t cK[8];
  __shared__ int cn[8], cp[8];
  const int32_t* mp = maps + pd.map;
  for (int e = threadIdx.x; e < 8 * 64; e += 256) {
    const int q = e / 64, i = e % 64;
    const int a = ti * 64 + i, b = tj * 64 + i;
    const bool has = pd.child[q] >= 0;
    rmap[q][i] = (has && a < n) ? mp[(int64_t)q * n + a] : -1;
    cmap[q][i] = (has && b < n) ? mp[(int64_t)q * n + b] : -1;
  }
  if (threadIdx.x < 8) {
    const int ch = pd.child[threadIdx.x];
    if (ch >= 0) {
      const CellDesc cd = child[ch];
      cK[threadIdx.x] = cd.K;
      cn[threadIdx.x] = cd.n;
      cp[threadIdx.x] = cd.p;
    } else {
      cK[threadIdx.x] = 0;
      cn[threadIdx.x] = 0;
      cp[threadIdx.x] = 0;
    }
  }
  __syncthreads();
  // the children that hold row i / column j of the tile (bit q): an entry
  // visits only the children that hold both, in increasing q as before
  __shared__ unsigned s_rm[64], s_cm[64];
  if (threadIdx.x < 64) {
    unsigned r = 0u, c = 0u;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      r |= (rmap[q][threadIdx.x] >= 0 ? 1u : 0u) << q;
      c |= (cmap[q][threadIdx.x] >= 0 ? 1u : 0u) << q;
    }
    s_rm[threadIdx.x] = r;
    s_cm[threadIdx.x] = c;
  }
  __syncthreads();
  T* K = Kp + pd.K;
  for (int e = threadIdx.x; e < 64 * 64; e += 256) {
    const int i = e % 64, j = e / 64;
    const int a = ti * 64 + i, b = tj * 64 + j;
    if (a >= n || b >= n || a < b) continue;
    T sum = T(0);
    for (unsigned msk = s_rm[i] & s_cm[j]; msk != 0u; msk &= msk - 1u) {
      const int q = __ffs(msk) - 1;
      const int x = rmap[q][i], y = cmap[q][j];
      const int hi_ = max(x, y), lo_ = min(x, y);
      const int64_t ncq = cn[q], pq = cp[q];
      sum += Kc[cK[q] + (pq + hi_) + (pq + lo_) * ncq];
    }
    K[(int64_t)a + (int64_t)b * n] = sum;
  }
}

// One CTA per 32 x 32 tile of a front's gather block.  The cells' frontal
// matrices hold only their lower triangles, so an entry (x, y) with x < y is
// read as (y, x): the tile is accumulated in shared memory in two passes per
// cell, lanes over the tile's rows for the entries read down a column
// (x >= y) and lanes over its columns for the transposed ones (x < y), so
// both read consecutive addresses; the cells are added in order.
constexpr int GT = 32;   // gather tile

template <typename T>
__global__ void __launch_bounds__(256) k_skel_gather(const SkelDesc* __restrict__ fr, int ncp,
                                                     const int32_t* __restrict__ rowPos,
                                                     const CellDesc* __restrict__ cells,
                                                     const T* __restrict__ Kar, T* Gar) {
  const SkelDesc f = fr[blockIdx.y];
  const int rows = f.nF + f.nR, cols = f.nF;
  const int tr = (rows + GT - 1) / GT, tc = (cols + GT - 1) / GT;
  if ((int)blockIdx.x >= tr * tc) return;
  const int r0 = (int)(blockIdx.x % tr) * GT, c0 = (int)(blockIdx.x / tr) * GT;
  __shared__ T tile[GT][GT + 1];   // tile[c][r]
  __shared__ int xr[4][GT], yc[4][GT];
  __shared__ int64_t cK[4];
  __shared__ int cn[4], cp[4];
  const int tx = threadIdx.x % GT, ty = threadIdx.x / GT;   // ty < 8
  const int32_t* rp = rowPos + f.rows;
  if (threadIdx.x < ncp) {
    const CellDesc cd = cells[f.cell[threadIdx.x]];
    cK[threadIdx.x] = cd.K;
    cn[threadIdx.x] = cd.n;
    cp[threadIdx.x] = cd.p;
  }
  if (ty < ncp) {
    xr[ty][tx] = r0 + tx < rows ? rp[(int64_t)(r0 + tx) * ncp + ty] : -1;
    yc[ty][tx] = c0 + tx < cols ? rp[(int64_t)(c0 + tx) * ncp + ty] : -1;
  }
  for (int q = ty; q < GT; q += 8) tile[q][tx] = T(0);
  __syncthreads();
  for (int i = 0; i < ncp; ++i) {
    const T* K = Kar + cK[i];
    const int64_t nc = cn[i], p = cp[i];
    for (int q = ty; q < GT; q += 8) {   // lanes over rows: (x, y) with x >= y
      const int x = xr[i][tx], y = yc[i][q];
      if (x >= 0 && y >= 0 && x >= y) tile[q][tx] += K[(p + x) + (p + y) * nc];
    }
    __syncthreads();
    for (int q = ty; q < GT; q += 8) {   // lanes over columns: (x, y) with x < y, read as (y, x)
      const int x = xr[i][q], y = yc[i][tx];
      if (x >= 0 && y >= 0 && x < y) tile[tx][q] += K[(p + y) + (p + x) * nc];
    }
    __syncthreads();
  }
  for (int q = ty; q < GT; q += 8)
    if (r0 + tx < rows && c0 + q < cols) Gar[f.G + (r0 + tx) + (int64_t)(c0 + q) * rows] = tile[q][tx];
}

template <typename T>
__global__ void __launch_bounds__(256) k_skel_permute(const SkelDesc* __restrict__ fr,
                                                      const int32_t* __restrict__ perm,
                                                      const T* __restrict__ Gar, T* Zar) {
  const SkelDesc f = fr[blockIdx.y];
  const int nF = f.nF;
  const int64_t tot = (int64_t)nF * nF;
  const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (e >= tot) return;
  const int r = (int)(e % nF), c = (int)(e / nF);
  const int p = nF - f.k;
  const int32_t* pm = perm + f.perm;
  const int orr = r < p ? pm[f.k + r] : pm[r - p];
  const int occ = c < p ? pm[f.k + c] : pm[c - p];
  const int ld = nF + f.nR;
  Zar[f.Z + e] = Gar[f.G + orr + (int64_t)occ * ld];
}

template <typename T>
__global__ void __launch_bounds__(256) k_skel_writeback(const SkelDesc* __restrict__ fr, int ncp,
                                                        const int32_t* __restrict__ rowPos,
                                                        const int32_t* __restrict__ perm,
                                                        const CellDesc* __restrict__ cells,
                                                        const T* __restrict__ Zar, T* Kar) {
  const SkelDesc f = fr[blockIdx.y];
  const int k = f.k, nF = f.nF, p = nF - k;
  const int64_t tot = (int64_t)k * k;
  const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (e >= tot) return;
  const int r = (int)(e % k), c = (int)(e / k);
  if (r < c) return;
  const T v = Zar[f.Z + (p + r) + (int64_t)(p + c) * nF];
  const int32_t* pm = perm + f.perm;
  const int32_t* rp = rowPos + f.rows;
  const int gr = pm[r], gc = pm[c];
  for (int i = 0; i < ncp; ++i) {
    const CellDesc cd = cells[f.cell[i]];
    const int x = rp[(int64_t)gr * ncp + i], y = rp[(int64_t)gc * ncp + i];
    if (x < 0 || y < 0) continue;
    const int hi_ = max(x, y), lo_ = min(x, y);
    Kar[cd.K + (cd.p + hi_) + (int64_t)(cd.p + lo_) * cd.n] = i == 0 ? v : T(0);
  }
}

}  // namespace

void stencil_coefficients(const double* a, const double* b, double b_const, int n, int periodic,
                          double* cpl, double* diag, int* d_bad, cudaStream_t st) {
  const int64_t N = (int64_t)n * n * n;
  ProfScope ps("stencil_coefficients", st, 0.0, 8.0 * N * (b ? 6.0 : 5.0));
  k_stencil<<<ceil_div(N, 256), 256, 0, st>>>(a, b, b_const, n, periodic, cpl, diag, d_bad);
  HIF_CHECK_LAUNCH();
}

template <typename T>
void assemble_level0(const CellDesc* d_cells, int ncell, const int32_t* lists, int n, int s,
                     int periodic, const double* cpl, const double* diag, T* Karena, int maxbox,
                     cudaStream_t st) {
  const size_t smem = (size_t)maxbox * sizeof(int);
  if (smem > 48 * 1024)
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_assemble0<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  ProfScope ps("assemble_level0", st);
  k_assemble0<T><<<ncell, 128, smem, st>>>(d_cells, lists, n, s, periodic, cpl, diag, Karena);
  HIF_CHECK_LAUNCH();
}

template <typename T>
void merge_children(const MergeDesc* d_par, const MergeDesc* h_par, int npar,
                    const CellDesc* d_child, const int32_t* maps, const T* Kchild, T* Kpar,
                    cudaStream_t st) {
  int nmax = 1;
  for (int i = 0; i < npar; ++i) nmax = std::max(nmax, h_par[i].n);
  const int nt = ceil_div(nmax, 64);
  for (int f0 = 0; f0 < npar; f0 += MAX_GRID_Y) {
    const int nb = std::min(MAX_GRID_Y, npar - f0);
    double by = 0;
    if (prof_enabled())
      for (int i = f0; i < f0 + nb; ++i) by += sizeof(T) * 0.5 * (double)h_par[i].n * (h_par[i].n + 1);
    ProfScope ps("merge_children", st, 0.0, by);
    k_merge<T><<<dim3(nt * (nt + 1) / 2, nb), 256, 0, st>>>(d_par + f0, d_child, maps, Kchild,
                                                            Kpar);
    HIF_CHECK_LAUNCH();
  }
}

template <typename T>
void skel_gather(const SkelDesc* d_f, const SkelDesc* h_f, int nf, int ncp,
                 const int32_t* rowPos, const CellDesc* d_cells, const T* Karena, T* Garena,
                 cudaStream_t st) {
  int64_t mx = 1;
  for (int i = 0; i < nf; ++i)
    mx = std::max<int64_t>(mx, (int64_t)ceil_div(h_f[i].nF + h_f[i].nR, GT) * ceil_div(h_f[i].nF, GT));
  for (int f0 = 0; f0 < nf; f0 += MAX_GRID_Y) {
    const int nb = std::min(MAX_GRID_Y, nf - f0);
    double by = 0;
    if (prof_enabled())
      for (int i = f0; i < f0 + nb; ++i) by += sizeof(T) * (double)(h_f[i].nF + h_f[i].nR) * h_f[i].nF;
    ProfScope ps("skel_gather", st, 0.0, by);
    k_skel_gather<T><<<dim3((unsigned)mx, nb), 256, 0, st>>>(d_f + f0, ncp, rowPos, d_cells,
                                                             Karena, Garena);
    HIF_CHECK_LAUNCH();
  }
}

template <typename T>
void skel_permute(const SkelDesc* d_f, const SkelDesc* h_f, int nf, const int32_t* perm,
                  const T* Garena, T* Zarena, cudaStream_t st) {
  int64_t mx = 1;
  for (int i = 0; i < nf; ++i) mx = std::max<int64_t>(mx, (int64_t)h_f[i].nF * h_f[i].nF);
  for (int f0 = 0; f0 < nf; f0 += MAX_GRID_Y) {
    const int nb = std::min(MAX_GRID_Y, nf - f0);
    ProfScope ps("skel_permute", st);
    k_skel_permute<T><<<dim3(ceil_div(mx, 256), nb), 256, 0, st>>>(d_f + f0, perm, Garena, Zarena);
    HIF_CHECK_LAUNCH();
  }
}

template <typename T>
void skel_writeback(const SkelDesc* d_f, const SkelDesc* h_f, int nf, int ncp,
                    const int32_t* rowPos, const int32_t* perm, const CellDesc* d_cells,
                    const T* Zarena, T* Karena, cudaStream_t st) {
  int64_t mx = 1;
  for (int i = 0; i < nf; ++i) mx = std::max<int64_t>(mx, (int64_t)h_f[i].k * h_f[i].k);
  for (int f0 = 0; f0 < nf; f0 += MAX_GRID_Y) {
    const int nb = std::min(MAX_GRID_Y, nf - f0);
    ProfScope ps("skel_writeback", st);
    k_skel_writeback<T><<<dim3(ceil_div(mx, 256), nb), 256, 0, st>>>(d_f + f0, ncp, rowPos, perm,
                                                                     d_cells, Zarena, Karena);
    HIF_CHECK_LAUNCH();
  }
}

#define HIF_INST(T)                                                                          \
  template void assemble_level0<T>(const CellDesc*, int, const int32_t*, int, int, int,     \
                                   const double*, const double*, T*, int, cudaStream_t);    \
  template void merge_children<T>(const MergeDesc*, const MergeDesc*, int, const CellDesc*, \
                                  const int32_t*, const T*, T*, cudaStream_t);              \
  template void skel_gather<T>(const SkelDesc*, const SkelDesc*, int, int, const int32_t*,  \
                               const CellDesc*, const T*, T*, cudaStream_t);                \
  template void skel_permute<T>(const SkelDesc*, const SkelDesc*, int, const int32_t*,      \
                                const T*, T*, cudaStream_t);                                \
  template void skel_writeback<T>(const SkelDesc*, const SkelDesc*, int, int,               \
                                  const int32_t*, const int32_t*, const CellDesc*,          \
                                  const T*, T*, cudaStream_t);
HIF_INST(float)
HIF_INST(double)
#undef HIF_INST

}  // namespace hif
