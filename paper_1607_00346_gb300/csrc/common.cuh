// Internal definitions shared by the HIF CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/hif.h"

namespace hif {

// ---- error plumbing ---------------------------------------------------------

struct Error {
  hif_status code;
  std::string msg;
};

void set_last_error(const std::string& msg);

#define HIF_CUDA_TRY(expr)                                                        \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      throw ::hif::Error{e_ == cudaErrorMemoryAllocation ? HIF_ERR_OOM            \
                                                          : HIF_ERR_CUDA,         \
                         std::string(#expr) + ": " + cudaGetErrorString(e_)};     \
    }                                                                             \
  } while (0)

// Every kernel launch is followed by HIF_CHECK_LAUNCH(), which also counts it.
int64_t& launch_counter();
// Profiling: while hif_profile_begin() is in force, a ProfScope records CUDA
// events around the launches made during its lifetime, attributed to `name`
// with the given algorithmic flops and bytes.
bool prof_enabled();
// Add algorithmic counts to a kernel's record without a launch (used when the
// counts are only known after the launch, e.g. the ranks found by the ID).
void prof_add(const char* name, double flops, double bytes);
// A scope also counts the kernels launched inside it (this thread's launch
// counter; a CUDA graph replay adds the kernels of the graph).  While a
// ProfSuspend is alive on this thread (a stream capture), scopes record
// nothing.
class ProfScope {
 public:
  ProfScope(const char* name, cudaStream_t st, double flops = 0.0, double bytes = 0.0);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  cudaStream_t st_;
  bool active_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
  std::string name_;
  double flops_ = 0.0, bytes_ = 0.0;
  int64_t k0_ = 0;
};
class ProfSuspend {
 public:
  ProfSuspend();
  ~ProfSuspend();
  ProfSuspend(const ProfSuspend&) = delete;
  ProfSuspend& operator=(const ProfSuspend&) = delete;

 private:
  bool prev_;
};

#define HIF_CHECK_LAUNCH()                 \
  do {                                     \
    ++::hif::launch_counter();             \
    HIF_CUDA_TRY(cudaGetLastError());      \
  } while (0)

// ---- device-side error flags -------------------------------------------------
// Kernels never trap.  A failed Cholesky pivot (not positive or not finite)
// records the front index in flags[FLAG_NOT_SPD] (first failure wins) and the
// kernel carries on with a harmless value so that the launch finishes
// normally; a bounded wait that ran out records the front in
// flags[FLAG_TIMEOUT] and the kernel returns early.
enum : int { FLAG_NOT_SPD = 0, FLAG_TIMEOUT = 1, FLAG_COUNT = 4 };

// ---- work descriptors ---------------------------------------------------------

// A dense front: an n x n column-major frontal matrix K (ld = n) whose first p
// columns are eliminated (partial Cholesky), and an n x p factor panel P
// (ld = n) that receives [Linv; X^T] (Linv = L^{-1} of the leading p x p block).
struct DFront {
  int64_t K;     // element offset of K in the K arena
  int64_t P;     // element offset of P in the factor arena
  int n;         // extent handled by the kernel (rows/columns 0..n-1)
  int p;
  int id;        // front number (reported on failure)
  int ld;        // leading dimension of K and P (the front's full size)
};

// Batched matrix product C (m x n) = beta C + alpha op(A) op(B) with k inner.
struct GemmOp {
  int64_t A, B, C;   // element offsets from the A, B and C base pointers of the launch
  int m, n, k;
  int lda, ldb, ldc;
  int transA, transB;
  float alpha, beta;
  int lower;         // 1: C is symmetric, only tiles touching its lower triangle are computed
  int pad;
};

// Batched matrix-vector product on a front of the apply (see apply kernels).
struct GemvOp {
  int64_t M;      // element offset of the matrix in the factor arena
  int64_t x;      // offset of the input vector in the work arena
  int64_t y;      // offset of the output vector in the work arena
  int rows, cols; // matrix shape (column-major)
  int ld;
  int tri;        // 1: matrix is lower triangular (only r >= c read)
  float alpha;
  int beta_one;   // 1: y += alpha op(M) x ; 0: y = alpha op(M) x
};

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace hif
