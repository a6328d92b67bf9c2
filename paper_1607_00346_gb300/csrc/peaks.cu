// Measured arithmetic peaks of the current GPU: dense FMA loops (FP32, FP64)
// and back-to-back tensor-core products (tcgen05 kind::tf32 and kind::f16
// with BF16), each timed with CUDA events.  These are the denominators of the
// roofline fractions of the FMA-bound and tensor-bound kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <string>

#include "../../include/hif_peaks.h"
#include "common.cuh"
#include "tcgen05.cuh"

namespace hif {
namespace {

constexpr int FMA_THREADS = 256;
constexpr int FMA_CHAINS = 8;      // independent dependency chains per thread
constexpr int FMA_UNROLL = 16;     // FMAs per chain per loop trip

template <typename T>
__global__ void __launch_bounds__(FMA_THREADS) k_peak_fma(T* out, int iters, T seed) {
  T a[FMA_CHAINS];
#pragma unroll
  for (int i = 0; i < FMA_CHAINS; ++i) a[i] = seed + T(threadIdx.x % 7 + i);
  const T mul = T(0.9999), add = T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < FMA_UNROLL; ++u)
#pragma unroll
      for (int i = 0; i < FMA_CHAINS; ++i) a[i] = fma(a[i], mul, add);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < FMA_CHAINS; ++i) s += a[i];
  if (s == T(-1234.5)) out[blockIdx.x] = s;   // never true; keeps the chains live
}

// Tensor-core loop: one thread issues `iters` x 4 products D += A B^T
// (M = 128, N = 256) from fixed shared-memory operands into one TMEM
// accumulator of 256 columns, then commits; every thread waits for the
// commit with an iteration limit.  100 KB of shared memory keeps at most two
// CTAs on an SM, so the two accumulators fit the SM's 512 TMEM columns.
constexpr int MMA_SMEM = 100 * 1024;
constexpr int MMA_N = 256;
constexpr long long MMA_WAIT_LIMIT = 200000000;

template <bool BF16>
__global__ void __launch_bounds__(128) k_peak_mma(int iters, int* flags) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid / 32;
  // operands: A 128 rows x 32 bytes per K step, B 256 rows; 4 K steps of
  // 32 bytes each (TF32: K = 8, BF16: K = 16 per instruction); small values
  uint32_t* w = reinterpret_cast<uint32_t*>(smem);
  for (int i = tid; i < 48 * 1024 / 4; i += blockDim.x)
    w[i] = BF16 ? 0x3c003c00u ^ (uint32_t)(i & 0x00ff00ff) : 0x3c000000u ^ (uint32_t)(i & 0xffff);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     tc5::smem_u32(&s_tmem)),
                 "r"(MMA_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc5::smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("fence.proxy.async.shared::cta;\n");
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = s_tmem;
  if (tid == 0) {
    const uint32_t a = tc5::smem_u32(smem), b = a + 16 * 1024;
    constexpr uint32_t SBO = 8 * 128;    // 8 rows x 128 bytes (4 K steps of 32 bytes)
    const uint32_t id = BF16 ? tc5::idesc_bf16(128, MMA_N) : tc5::idesc_tf32(128, MMA_N);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint64_t da = tc5::sdesc(a + ks * 256, 128, SBO), db = tc5::sdesc(b + ks * 256, 128, SBO);
        if (BF16) tc5::mma_bf16(tmem, da, db, id, (it | ks) ? 1u : 0u);
        else tc5::mma_tf32(tmem, da, db, id, (it | ks) ? 1u : 0u);
      }
    }
    tc5::commit(&mbar);
  }
  bool done = false;
  for (long long k = 0; k < MMA_WAIT_LIMIT && !done; ++k) done = tc5::mbar_test(&mbar, 0);
  if (!__syncthreads_and(done)) {
    // bounded second wait so that nothing writes the accumulator once freed
    if (!done)
      for (long long k = 0; k < MMA_WAIT_LIMIT && !done; ++k) done = tc5::mbar_test(&mbar, 0);
    if (tid == 0) atomicCAS(&flags[FLAG_TIMEOUT], -1, (int)blockIdx.x);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(MMA_N));
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    HIF_CUDA_TRY(cudaEventCreate(&a));
    HIF_CUDA_TRY(cudaEventCreate(&b));
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// Best-of-three seconds of launch(iters) after one warm-up launch, with
// iters grown until one launch takes at least `target` seconds.
template <typename F>
double time_loop(F launch, int iters0, double target, cudaStream_t st, int* iters_out) {
  Timer t;
  int iters = iters0;
  double best = 0.0;
  for (int round = 0; round < 12; ++round) {
    launch(iters);   // warm-up at this size
    best = 1e30;
    for (int r = 0; r < 3; ++r) {
      HIF_CUDA_TRY(cudaEventRecord(t.a, st));
      launch(iters);
      HIF_CUDA_TRY(cudaEventRecord(t.b, st));
      HIF_CUDA_TRY(cudaEventSynchronize(t.b));
      float ms = 0.f;
      HIF_CUDA_TRY(cudaEventElapsedTime(&ms, t.a, t.b));
      best = std::min(best, 1e-3 * ms);
    }
    if (best >= target) break;
    const double grow = std::min(16.0, std::max(1.5, 1.2 * target / std::max(best, 1e-6)));
    iters = (int)std::min(1e9, iters * grow);
  }
  *iters_out = iters;
  return best;
}

}  // namespace
}  // namespace hif

extern "C" hif_status hif_measure_peaks(hif_peaks* out, hif_stream stream) {
  using hif::Error;
  try {
    if (!out) throw Error{HIF_ERR_INVALID_ARG, "out must not be NULL"};
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0, clk = 0;
    HIF_CUDA_TRY(cudaGetDevice(&dev));
    HIF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    HIF_CUDA_TRY(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev));
    out->sm_count = nsm;
    out->sm_clock_khz = clk;
    float* d32 = nullptr;
    double* d64 = nullptr;
    int* flags = nullptr;
    HIF_CUDA_TRY(cudaMalloc(&d32, sizeof(float) * 64 * 1024));
    HIF_CUDA_TRY(cudaMalloc(&d64, sizeof(double) * 64 * 1024));
    HIF_CUDA_TRY(cudaMalloc(&flags, sizeof(int) * hif::FLAG_COUNT));
    struct Free {
      void* p[3];
      ~Free() {
        for (void* q : p) cudaFree(q);
      }
    } fr{{d32, d64, flags}};
    HIF_CUDA_TRY(cudaMemsetAsync(flags, 0xff, sizeof(int) * hif::FLAG_COUNT, st));
    const int fblocks = nsm * 8;   // 2048 threads per SM
    const double fthreads = (double)fblocks * hif::FMA_THREADS;
    const double per_iter = 2.0 * hif::FMA_CHAINS * hif::FMA_UNROLL;
    int it = 0;
    double s = hif::time_loop(
        [&](int iters) {
          hif::k_peak_fma<float><<<fblocks, hif::FMA_THREADS, 0, st>>>(d32, iters, 1.0f);
          HIF_CHECK_LAUNCH();
        },
        64, 0.02, st, &it);
    out->fp32_fma_tflops = fthreads * per_iter * it / s / 1e12;
    s = hif::time_loop(
        [&](int iters) {
          hif::k_peak_fma<double><<<fblocks, hif::FMA_THREADS, 0, st>>>(d64, iters, 1.0);
          HIF_CHECK_LAUNCH();
        },
        4, 0.02, st, &it);
    out->fp64_fma_tflops = fthreads * per_iter * it / s / 1e12;
    static const bool attr = [] {
      HIF_CUDA_TRY(cudaFuncSetAttribute(hif::k_peak_mma<false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        hif::MMA_SMEM));
      HIF_CUDA_TRY(cudaFuncSetAttribute(hif::k_peak_mma<true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        hif::MMA_SMEM));
      return true;
    }();
    (void)attr;
    const int mblocks = 2 * nsm;
    for (int bf = 0; bf < 2; ++bf) {
      s = hif::time_loop(
          [&](int iters) {
            if (bf)
              hif::k_peak_mma<true><<<mblocks, 128, hif::MMA_SMEM, st>>>(iters, flags);
            else
              hif::k_peak_mma<false><<<mblocks, 128, hif::MMA_SMEM, st>>>(iters, flags);
            HIF_CHECK_LAUNCH();
          },
          16, 0.02, st, &it);
      const double kinst = bf ? 16.0 : 8.0;
      const double fl = (double)mblocks * it * 4.0 * 2.0 * 128.0 * hif::MMA_N * kinst;
      (bf ? out->bf16_mma_tflops : out->tf32_mma_tflops) = fl / s / 1e12;
    }
    int hflags[hif::FLAG_COUNT];
    HIF_CUDA_TRY(cudaMemcpy(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost));
    if (hflags[hif::FLAG_TIMEOUT] >= 0)
      throw Error{HIF_ERR_TIMEOUT, "a tensor-core wait of the peak loop expired"};
    out->seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return HIF_OK;
  } catch (const Error& e) {
    hif::set_last_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    hif::set_last_error(e.what());
    return HIF_ERR_CUDA;
  }
}
