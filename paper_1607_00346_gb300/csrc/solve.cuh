// Vector kernels of the apply sweeps and of the preconditioned solve.
#pragma once

#include "common.cuh"

namespace hif {

// work[q*vs + voff + i] = y[q*ys + idx[i]]
template <typename T>
void vec_gather(const int32_t* idx, int64_t cnt, const T* y, int64_t ys, T* work, int64_t vs,
                int64_t voff, int nrhs, cudaStream_t st);
// y[q*ys + g[i]] = work[q*vs + pos[i]]
template <typename T>
void vec_set(const int32_t* g, const int32_t* pos, int64_t cnt, T* y, int64_t ys,
             const T* work, int64_t vs, int nrhs, cudaStream_t st);
// y[q*ys + tgt[t]] -= sum_{e = ptr[t]}^{ptr[t+1]-1} work[q*vs + src[e]]  (fixed order)
template <typename T>
void vec_accumulate(const int32_t* tgt, const int64_t* ptr, const int32_t* src, int64_t ntgt,
                    T* y, int64_t ys, const T* work, int64_t vs, int nrhs, cudaStream_t st);
// One factor's part of a grouped gather (kind 0: w[q vs + i] = y[q ys + a[i]]),
// set (kind 1: y[q ys + a[i]] = w[q vs + b[i]]) or accumulate (kind 2:
// y[q ys + a[t]] -= sum_{e = ptr[t]}^{ptr[t+1]-1} w[q vs + b[e]]), i < cnt,
// q < nrhs: the parts of several factors in one launch.
template <typename T>
struct VecJob {
  const int32_t* a;
  const int32_t* b;
  const int64_t* ptr;
  int64_t cnt;
  T* y;
  int64_t ys;
  T* w;
  int64_t vs;
  int nrhs;
};
template <typename T>
void vec_grouped(int kind, const VecJob<T>* d_jobs, const VecJob<T>* h_jobs, int njobs,
                 cudaStream_t st);
// y = (T) x
template <typename T>
void vec_convert_in(const double* x, T* y, int64_t cnt, cudaStream_t st);
// x = (double) y
template <typename T>
void vec_convert_out(const T* y, double* x, int64_t cnt, cudaStream_t st);

// r = f - A u for nrhs columns of length n^3 (seven-point operator, double;
// periodic: neighbours wrap around).
void residual(const double* cpl, const double* diag, int n, int periodic, const double* f,
              const double* u, double* r, int nrhs, cudaStream_t st);
// q = A p
void matvec(const double* cpl, const double* diag, int n, int periodic, const double* p,
            double* q, int nrhs, cudaStream_t st);
// out[c] = sum_i x[c*N + i] * y[c*N + i] for c < ncol; `part` holds
// ncol * 1024 partial sums.
void dots(const double* x, const double* y, int64_t N, int ncol, double* part, double* out,
          cudaStream_t st);
// y[c] = y[c] + a[c] x[c]   (a: device array of ncol scalars; sign applied)
void axpy_cols(const double* a, double sign, const double* x, double* y, int64_t N, int ncol,
               cudaStream_t st);
// p[c] = z[c] + b[c] p[c]
void xpby_cols(const double* z, const double* b, double* p, int64_t N, int ncol, cudaStream_t st);

}  // namespace hif
