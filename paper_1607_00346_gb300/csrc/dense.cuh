// Batched dense kernels over uneven fronts (host launch wrappers).
#pragma once

#include "common.cuh"

namespace hif {

constexpr int NB = 64;      // panel width of the partial Cholesky and of the triangular inverse
constexpr int TILE = 64;    // output tile of the trailing update / batched GEMM

// FP64 retry of FP32 fronts (the LDL^T of §2.2 / §2.3 read as Cholesky, redone
// in double when the FP32 one breaks down): a front whose leading-block
// Cholesky meets a pivot d_j with A_jj / d_j > growth (or d_j not positive)
// is refactored entirely in FP64; growth = 0 turns this off (such a pivot
// then fails the factorization with HIF_ERR_NOT_SPD).  *retried counts them.
struct RetryOpts {
  double growth;
  int64_t* retried;
};

// Partial Cholesky of a batch of fronts (§2.2 and §2.3: A_II = L L^T,
// X = L^{-1} A_IN, A_NN -= X^T X).  Fronts must be sorted by p, largest first.
// On return: trailing blocks of K hold the Schur complements, P holds
// [Linv; X^T] (Linv = L^{-1}, lower triangular) for each front.  With
// tensor_cores (FP32 only) the deep products run on gemm_tc.  With retry
// (FP32 only) the host waits once after the leading blocks are factored to
// read the per-front flags.
template <typename T>
void partial_cholesky(const DFront* d_fronts, const DFront* h_fronts, int nfront, T* Karena,
                      T* Parena, int* d_flags, bool tensor_cores, cudaStream_t st,
                      const RetryOpts* retry = nullptr);

// C = beta C + alpha op(A) op(B) on the tensor cores (tcgen05, 3xTF32; see
// tc.cu): GemmOp semantics as gemm_batched, beta 0 or 1, FP32 data.
// `name` labels the launches in the kernel profile.
void gemm_tc(const GemmOp* d_ops, const GemmOp* h_ops, int nops, const float* Abase,
             const float* Bbase, float* Cbase, int* d_flags, cudaStream_t st,
             const char* name = "gemm_tc");

// Autotuning of gemm_tc's tile shape: time the variants on the product
// shapes recorded during a tuning factorization (tune.h).
void tune_gemm_from_records(cudaStream_t st);

// C = beta C + alpha op(A) op(B) for a batch of independent problems.
template <typename T>
void gemm_batched(const GemmOp* d_ops, const GemmOp* h_ops, int nops, const T* Abase,
                  const T* Bbase, T* Cbase, cudaStream_t st, const char* name = "gemm_batched");

// y = alpha op(M) x (+ y), batched (see GemvOp).  trans = 0: y (rows) = M x;
// trans = 1: y (cols) = M^T x.  nrhs vectors with stride `vstride` in `work`.
template <typename T>
void gemv_batched(const GemvOp* d_ops, const GemvOp* h_ops, int nops, int trans,
                  const T* Marena, T* work, int64_t vstride, int nrhs, cudaStream_t st);

// Grouped apply: one launch runs the mat-vec lists of several factors (one
// segment per factor's list and block of right-hand sides).  Segment k owns
// ops first_k .. first_{k+1}-1 of the launch; op j reads ops[j - first] of
// its device list, its matrix at M + op.M and its vectors at w + op.x,
// w + op.y (w already shifted to the block's first column, vs apart).
template <typename T>
struct GemvSeg {
  const GemvOp* ops;
  const T* M;
  T* w;
  int64_t vs;
  int64_t first;
};

// gemv_batched over the segments (trans as there, R right-hand sides per op:
// 16, 8, 4, 2 or 1; nops = all ops of the launch; mx = the widest op's row
// tiles (trans 0) or column groups (trans 1), from gemv_tiles).  Per op the
// arithmetic is gemv_batched's, so a grouped apply is bitwise the factor's
// own apply.
template <typename T>
void gemv_segments(const GemvSeg<T>* d_segs, int nseg, int64_t nops, int mx, int trans, int R,
                   double flops, double bytes, cudaStream_t st);
int gemv_tiles(const GemvOp* h_ops, int nops, int trans);

}  // namespace hif
