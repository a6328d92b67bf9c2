// Vector kernels: gathers and scatters of the apply sweeps (deterministic, no
// atomics), the seven-point residual in double, dot products and updates of
// the preconditioned conjugate gradients.
#include <algorithm>

#include "solve.cuh"

namespace hif {

namespace {

constexpr int VT = 256;
constexpr int DOT_BLOCKS = 1024;

template <typename T>
__global__ void k_gather(const int32_t* __restrict__ idx, int64_t cnt, const T* __restrict__ y,
                         int64_t ys, T* work, int64_t vs, int64_t voff, int nrhs) {
  const int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x;
  if (i >= cnt) return;
  const int64_t g = idx[i];
  for (int q = 0; q < nrhs; ++q) work[q * vs + voff + i] = y[q * ys + g];
}

template <typename T>
__global__ void k_set(const int32_t* __restrict__ gi, const int32_t* __restrict__ pos, int64_t cnt,
                      T* y, int64_t ys, const T* __restrict__ work, int64_t vs, int nrhs) {
  const int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x;
  if (i >= cnt) return;
  const int64_t g = gi[i], p = pos[i];
  for (int q = 0; q < nrhs; ++q) y[q * ys + g] = work[q * vs + p];
}

template <typename T>
__global__ void k_acc(const int32_t* __restrict__ tgt, const int64_t* __restrict__ ptr,
                      const int32_t* __restrict__ src, int64_t ntgt, T* y, int64_t ys,
                      const T* __restrict__ work, int64_t vs, int nrhs) {
  const int64_t t = (int64_t)blockIdx.x * VT + threadIdx.x;
  if (t >= ntgt) return;
  const int64_t g = tgt[t];
  for (int q = 0; q < nrhs; ++q) {
    T s = T(0);
    for (int64_t e = ptr[t]; e < ptr[t + 1]; ++e) s += work[q * vs + src[e]];
    y[q * ys + g] -= s;
  }
}

// Grouped forms: blockIdx.y = one factor's part (VecJob), the same
// per-element work as k_gather, k_set and k_acc.
template <typename T>
__global__ void k_gather_grouped(const VecJob<T>* __restrict__ jobs) {
  const VecJob<T> jb = jobs[blockIdx.y];
  const int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x;
  if (i >= jb.cnt) return;
  const int64_t g = jb.a[i];
  for (int q = 0; q < jb.nrhs; ++q) jb.w[q * jb.vs + i] = jb.y[q * jb.ys + g];
}

template <typename T>
__global__ void k_set_grouped(const VecJob<T>* __restrict__ jobs) {
  const VecJob<T> jb = jobs[blockIdx.y];
  const int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x;
  if (i >= jb.cnt) return;
  const int64_t g = jb.a[i], p = jb.b[i];
  for (int q = 0; q < jb.nrhs; ++q) jb.y[q * jb.ys + g] = jb.w[q * jb.vs + p];
}

template <typename T>
__global__ void k_acc_grouped(const VecJob<T>* __restrict__ jobs) {
  const VecJob<T> jb = jobs[blockIdx.y];
  const int64_t t = (int64_t)blockIdx.x * VT + threadIdx.x;
  if (t >= jb.cnt) return;
  const int64_t g = jb.a[t];
  for (int q = 0; q < jb.nrhs; ++q) {
    T s = T(0);
    for (int64_t e = jb.ptr[t]; e < jb.ptr[t + 1]; ++e) s += jb.w[q * jb.vs + jb.b[e]];
    jb.y[q * jb.ys + g] -= s;
  }
}

template <typename T>
__global__ void k_cin(const double* __restrict__ x, T* y, int64_t cnt) {
  const int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x;
  if (i < cnt) y[i] = (T)x[i];
}

template <typename T>
__global__ void k_cout(const T* __restrict__ y, double* x, int64_t cnt) {
  const int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x;
  if (i < cnt) x[i] = (double)y[i];
}

// y = A u (mode 0) or y = f - A u (mode 1).  Dirichlet: neighbours outside
// the grid are zero; periodic: index arithmetic wraps around every dimension.
__global__ void k_stencil_apply(const double* __restrict__ cpl, const double* __restrict__ diag,
                                int n, int periodic, const double* __restrict__ f,
                                const double* __restrict__ u, double* out, int nrhs, int mode) {
  const int64_t N = (int64_t)n * n * n;
  const int64_t j = (int64_t)blockIdx.x * VT + threadIdx.x;
  if (j >= N) return;
  const int x0 = (int)(j % n), x1 = (int)((j / n) % n), x2 = (int)(j / ((int64_t)n * n));
  const int64_t nn = (int64_t)n * n;
  if (!periodic) {
    for (int q = 0; q < nrhs; ++q) {
      const double* uq = u + q * N;
      double s = diag[j] * uq[j];
      if (x0 + 1 < n) s -= cpl[j] * uq[j + 1];
      if (x0 > 0) s -= cpl[j - 1] * uq[j - 1];
      if (x1 + 1 < n) s -= cpl[N + j] * uq[j + n];
      if (x1 > 0) s -= cpl[N + j - n] * uq[j - n];
      if (x2 + 1 < n) s -= cpl[2 * N + j] * uq[j + nn];
      if (x2 > 0) s -= cpl[2 * N + j - nn] * uq[j - nn];
      out[q * N + j] = mode ? f[q * N + j] - s : s;
    }
    return;
  }
  // neighbour offsets with wrap-around
  const int64_t p0 = x0 + 1 < n ? 1 : -(int64_t)(n - 1), m0 = x0 > 0 ? -1 : (int64_t)(n - 1);
  const int64_t p1 = x1 + 1 < n ? n : -(int64_t)(n - 1) * n, m1 = x1 > 0 ? -n : (int64_t)(n - 1) * n;
  const int64_t p2 = x2 + 1 < n ? nn : -(int64_t)(n - 1) * nn,
                m2 = x2 > 0 ? -nn : (int64_t)(n - 1) * nn;
  for (int q = 0; q < nrhs; ++q) {
    const double* uq = u + q * N;
    double s = diag[j] * uq[j];
    s -= cpl[j] * uq[j + p0];
    s -= cpl[j + m0] * uq[j + m0];
    s -= cpl[N + j] * uq[j + p1];
    s -= cpl[N + j + m1] * uq[j + m1];
    s -= cpl[2 * N + j] * uq[j + p2];
    s -= cpl[2 * N + j + m2] * uq[j + m2];
    out[q * N + j] = mode ? f[q * N + j] - s : s;
  }
}

__global__ void k_dot_part(const double* __restrict__ x, const double* __restrict__ y, int64_t N,
                           double* part) {
  const int c = blockIdx.y;
  const double* xc = x + c * N;
  const double* yc = y + c * N;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x; i < N; i += (int64_t)gridDim.x * VT)
    s += xc[i] * yc[i];
  __shared__ double red[VT / 32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < VT / 32; ++w) t += red[w];
    part[c * DOT_BLOCKS + blockIdx.x] = t;
  }
}

__global__ void k_dot_final(const double* __restrict__ part, double* out) {
  const int c = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < DOT_BLOCKS; i += VT) s += part[c * DOT_BLOCKS + i];
  __shared__ double red[VT / 32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < VT / 32; ++w) t += red[w];
    out[c] = t;
  }
}

__global__ void k_axpy(const double* __restrict__ a, double sign, const double* __restrict__ x,
                       double* y, int64_t N) {
  const int c = blockIdx.y;
  const double al = sign * a[c];
  for (int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x; i < N; i += (int64_t)gridDim.x * VT)
    y[c * N + i] += al * x[c * N + i];
}

__global__ void k_xpby(const double* __restrict__ z, const double* __restrict__ b, double* p,
                       int64_t N) {
  const int c = blockIdx.y;
  const double bb = b[c];
  for (int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x; i < N; i += (int64_t)gridDim.x * VT)
    p[c * N + i] = z[c * N + i] + bb * p[c * N + i];
}

inline int grid1(int64_t cnt) { return (int)((cnt + VT - 1) / VT); }

}  // namespace

template <typename T>
void vec_gather(const int32_t* idx, int64_t cnt, const T* y, int64_t ys, T* work, int64_t vs,
                int64_t voff, int nrhs, cudaStream_t st) {
  if (cnt == 0) return;
  ProfScope ps("apply_gather", st, 0.0, (double)cnt * (4.0 + 2.0 * sizeof(T) * nrhs));
  k_gather<T><<<grid1(cnt), VT, 0, st>>>(idx, cnt, y, ys, work, vs, voff, nrhs);
  HIF_CHECK_LAUNCH();
}

template <typename T>
void vec_set(const int32_t* g, const int32_t* pos, int64_t cnt, T* y, int64_t ys,
             const T* work, int64_t vs, int nrhs, cudaStream_t st) {
  if (cnt == 0) return;
  ProfScope ps("apply_scatter", st, 0.0, (double)cnt * (8.0 + 2.0 * sizeof(T) * nrhs));
  k_set<T><<<grid1(cnt), VT, 0, st>>>(g, pos, cnt, y, ys, work, vs, nrhs);
  HIF_CHECK_LAUNCH();
}

template <typename T>
void vec_accumulate(const int32_t* tgt, const int64_t* ptr, const int32_t* src, int64_t ntgt,
                    T* y, int64_t ys, const T* work, int64_t vs, int nrhs, cudaStream_t st) {
  if (ntgt == 0) return;
  ProfScope ps("apply_accumulate", st);
  k_acc<T><<<grid1(ntgt), VT, 0, st>>>(tgt, ptr, src, ntgt, y, ys, work, vs, nrhs);
  HIF_CHECK_LAUNCH();
}

template <typename T>
void vec_convert_in(const double* x, T* y, int64_t cnt, cudaStream_t st) {
  if (cnt == 0) return;
  ProfScope ps("convert", st, 0.0, (double)cnt * (8.0 + sizeof(T)));
  k_cin<T><<<grid1(cnt), VT, 0, st>>>(x, y, cnt);
  HIF_CHECK_LAUNCH();
}

template <typename T>
void vec_grouped(int kind, const VecJob<T>* d_jobs, const VecJob<T>* h_jobs, int njobs,
                 cudaStream_t st) {
  int64_t mx = 0;
  double by = 0;
  for (int i = 0; i < njobs; ++i) {
    mx = std::max(mx, h_jobs[i].cnt);
    by += (double)h_jobs[i].cnt * ((kind == 0 ? 4.0 : 8.0) + 2.0 * sizeof(T) * h_jobs[i].nrhs);
  }
  if (mx == 0) return;
  static const char* names[3] = {"apply_grouped_gather", "apply_grouped_scatter",
                                 "apply_grouped_accumulate"};
  ProfScope ps(names[kind], st, 0.0, kind == 2 ? 0.0 : by);
  for (int f0 = 0; f0 < njobs; f0 += 65535) {
    const dim3 grid((unsigned)grid1(mx), (unsigned)std::min(65535, njobs - f0));
    if (kind == 0) k_gather_grouped<T><<<grid, VT, 0, st>>>(d_jobs + f0);
    else if (kind == 1) k_set_grouped<T><<<grid, VT, 0, st>>>(d_jobs + f0);
    else k_acc_grouped<T><<<grid, VT, 0, st>>>(d_jobs + f0);
    HIF_CHECK_LAUNCH();
  }
}

template <typename T>
void vec_convert_out(const T* y, double* x, int64_t cnt, cudaStream_t st) {
  if (cnt == 0) return;
  ProfScope ps("convert", st, 0.0, (double)cnt * (8.0 + sizeof(T)));
  k_cout<T><<<grid1(cnt), VT, 0, st>>>(y, x, cnt);
  HIF_CHECK_LAUNCH();
}

void residual(const double* cpl, const double* diag, int n, int periodic, const double* f,
              const double* u, double* r, int nrhs, cudaStream_t st) {
  const int64_t N = (int64_t)n * n * n;
  ProfScope ps("residual", st, 14.0 * N * nrhs, 8.0 * N * (4.0 + 3.0 * nrhs));
  k_stencil_apply<<<grid1(N), VT, 0, st>>>(cpl, diag, n, periodic, f, u, r, nrhs, 1);
  HIF_CHECK_LAUNCH();
}

void matvec(const double* cpl, const double* diag, int n, int periodic, const double* p,
            double* q, int nrhs, cudaStream_t st) {
  const int64_t N = (int64_t)n * n * n;
  ProfScope ps("spmv", st, 13.0 * N * nrhs, 8.0 * N * (4.0 + 2.0 * nrhs));
  k_stencil_apply<<<grid1(N), VT, 0, st>>>(cpl, diag, n, periodic, nullptr, p, q, nrhs, 0);
  HIF_CHECK_LAUNCH();
}

void dots(const double* x, const double* y, int64_t N, int ncol, double* part, double* out,
          cudaStream_t st) {
  ProfScope ps("dots", st, 2.0 * N * ncol, 16.0 * N * ncol);
  k_dot_part<<<dim3(DOT_BLOCKS, ncol), VT, 0, st>>>(x, y, N, part);
  HIF_CHECK_LAUNCH();
  k_dot_final<<<ncol, VT, 0, st>>>(part, out);
  HIF_CHECK_LAUNCH();
}

void axpy_cols(const double* a, double sign, const double* x, double* y, int64_t N, int ncol,
               cudaStream_t st) {
  ProfScope ps("axpy", st, 2.0 * N * ncol, 24.0 * N * ncol);
  k_axpy<<<dim3(std::min<int64_t>(grid1(N), 2048), ncol), VT, 0, st>>>(a, sign, x, y, N);
  HIF_CHECK_LAUNCH();
}

void xpby_cols(const double* z, const double* b, double* p, int64_t N, int ncol, cudaStream_t st) {
  ProfScope ps("axpy", st, 2.0 * N * ncol, 24.0 * N * ncol);
  k_xpby<<<dim3(std::min<int64_t>(grid1(N), 2048), ncol), VT, 0, st>>>(z, b, p, N);
  HIF_CHECK_LAUNCH();
}

#define HIF_INST(T)                                                                           \
  template void vec_gather<T>(const int32_t*, int64_t, const T*, int64_t, T*, int64_t,       \
                              int64_t, int, cudaStream_t);                                   \
  template void vec_set<T>(const int32_t*, const int32_t*, int64_t, T*, int64_t, const T*,   \
                           int64_t, int, cudaStream_t);                                      \
  template void vec_accumulate<T>(const int32_t*, const int64_t*, const int32_t*, int64_t,   \
                                  T*, int64_t, const T*, int64_t, int, cudaStream_t);        \
  template void vec_convert_in<T>(const double*, T*, int64_t, cudaStream_t);                 \
  template void vec_convert_out<T>(const T*, double*, int64_t, cudaStream_t);                \
  template void vec_grouped<T>(int, const VecJob<T>*, const VecJob<T>*, int, cudaStream_t);
HIF_INST(float)
HIF_INST(double)
#undef HIF_INST

}  // namespace hif
