// Batched matrix products on the sm_103a tensor cores: the Schur complements
// of the partial Cholesky (A_NN -= X^T X, §2.2 / §2.3: the only dense
// contraction of the method) and X^T = A_NI L^{-T}.  FP32 accuracy from TF32
// tensor cores by the 3xTF32 split: x = hi + lo with hi = tf32(x),
// lo = tf32(x - hi), and A B^T ~= hi_A hi_B^T + hi_A lo_B^T + lo_A hi_B^T
// (FP32 accumulation in tensor memory).
//
// Per CTA (one 128 x TN output tile, TN = 128 or 256; 128 + TN threads):
//   * K is walked in chunks of KC (16, or 32 for products with few rows):
//     thread t loads one row of the chunk of A (t < 128) or of B (t >= 128)
//     into registers two chunks ahead, splits it and stores it in the K-major,
//     no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix;
//     LBO = 128 B between K-adjacent core matrices, SBO = 8 KC bytes between
//     8-row groups) of one of two shared buffers;
//   * one thread issues tcgen05.mma.cta_group::1.kind::tf32 (M = 128, N = TN,
//     K = 8 per instruction) into a TN-column TMEM accumulator and commits
//     to the buffer's mbarrier; the wait on it has an iteration limit (on
//     expiry the CTA agrees on the failure with a block-wide vote, waits
//     once more, again bounded, for its commits still in flight, records
//     FLAG_TIMEOUT, frees its TMEM and returns without reading it);
//   * with KC = 16 a 128 x 128 CTA holds 64 KB of shared memory and three
//     share an SM (384 of its 512 TMEM columns); a 128 x 256 CTA holds 96 KB
//     and two share an SM (all 512 columns), so one CTA's loads overlap the
//     others' products, and no mix of resident CTAs can ask for more than
//     512 columns;
//   * warps 0-7 read the accumulator back with tcgen05.ld (warp w owns TMEM
//     lanes 32 (w % 4) .. = tile rows, and half w / 4 of the columns) and
//     write alpha times it to C (added to C when beta = 1).
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "dense.cuh"
#include "tcgen05.cuh"
#include "tune.h"

namespace hif {

namespace {

constexpr int TC_M = 128;        // tile rows (TMEM lanes)
constexpr long long WAIT_LIMIT = 20000000;     // mbarrier polls before giving up

using tc5::idesc_tf32;
using tc5::mma_tf32;
using tc5::sdesc;
using tc5::smem_u32;

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of element (row, k) of a TC_M x KC K-major operand
template <int KC>
__device__ __forceinline__ int core_off(int row, int k) {
  return ((row >> 3) * (KC / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// C (M x N) = beta C + alpha op(A) op(B) for a batch of problems (GemmOp
// semantics: op(A)[r][k] = transA ? A[k + r lda] : A[r + k lda],
// op(B)[k][c] = transB ? B[c + k ldb] : B[k + c ldb]).  Operands are read in
// K chunks of KC, split into TF32 hi/lo parts and staged in one of two
// shared-memory buffers while the tensor cores work on the other.  beta is 0
// or 1.  `lower` skips tiles strictly above the diagonal of a symmetric C.
template <int KC, int TN>
__global__ void __launch_bounds__(TC_M + TN, KC == 16 ? (TN == 128 ? 3 : 2) : 1)
    k_gemm_tc(const GemmOp* __restrict__ ops, const float* __restrict__ Ab,
              const float* __restrict__ Bb, float* Cb, int* flags,
              const int64_t* __restrict__ woff, float* Wk) {
  constexpr int TILE_A = TC_M * KC * 4;   // A operand, one split
  constexpr int TILE_B = TN * KC * 4;     // B operand, one split
  constexpr int STAGE = 2 * TILE_A + 2 * TILE_B;
  const GemmOp o = ops[blockIdx.y];
  const int tm_n = (o.m + TC_M - 1) / TC_M, tn_n = (o.n + TN - 1) / TN;
  if ((int)blockIdx.x >= tm_n * tn_n) return;
  const int rb = (blockIdx.x % tm_n) * TC_M, cb = (blockIdx.x / tm_n) * TN;
  if (o.lower && cb >= rb + TC_M) return;
  const float* A = Ab + o.A;
  const float* B = Bb + o.B;
  float* C = Cb + o.C;

  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = idesc_tf32(TC_M, TN);
  // split K (gridDim.z > 1): this CTA takes chunks [cbeg, cbeg + nchunk) of
  // the product and leaves its partial tile in the work space Wk
  const int nch_all = (o.k + KC - 1) / KC;
  const int cbeg = (int)(((int64_t)nch_all * blockIdx.z) / gridDim.z);
  const int nchunk = (int)(((int64_t)nch_all * (blockIdx.z + 1)) / gridDim.z) - cbeg;
  uint32_t phase[2] = {0u, 0u};
  // outstanding[s]: products committed on buffer s whose completion this
  // thread has not yet seen (at most one commit per buffer is in flight)
  bool outstanding[2] = {false, false};
  bool ok = true;

  // bounded wait for the products issued on buffer s; the phase advances
  // only when the commit has arrived, so an expired wait can be retried
  auto wait_buf = [&](int s) {
    long long it = 0;
    uint32_t done = 0;
    while (!done) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(&mbar[s])), "r"(phase[s]));
      if (++it > WAIT_LIMIT) break;
    }
    if (done) {
      phase[s] ^= 1u;
      outstanding[s] = false;
    }
    return done != 0;
  };

  // staging registers of two chunks: chunk c lives in va (c even) or vb (c
  // odd); the loads of chunk c + 2 are issued as soon as chunk c is stored
  const bool isA = tid < TC_M;
  const int row = isA ? tid : tid - TC_M;
  const float* X = isA ? A : B;
  const int base = isA ? rb : cb;
  const int lim = isA ? o.m : o.n;
  const int64_t ldx = isA ? o.lda : o.ldb;
  const bool kfast = isA ? (o.transA != 0) : (o.transB == 0);   // k contiguous in memory
  const bool rin = base + row < lim;
  // K contiguous in memory: value q of a thread is (kr(q), kk(q)) so that
  // one warp instruction reads 8 rows x 4 consecutive k (16 bytes per row)
  // and stores 32 consecutive words of the core-matrix layout; otherwise a
  // thread owns one row (consecutive threads read consecutive rows)
  const int gw = isA ? warp : warp - TC_M / 32;   // warp within the operand's group
  constexpr int GA = TC_M / 32, GB = TN / 32;
  const int G = isA ? GA : GB;
  auto kr = [&](int q) { return (q / (KC / 4)) * (G * 8) + gw * 8 + lane / 4; };
  auto kq = [&](int q) { return (q % (KC / 4)) * 4 + lane % 4; };
  auto load = [&](int ch, float (&v)[KC]) {
    const int k0 = (cbeg + ch) * KC;
    if (kfast) {
#pragma unroll
      for (int q = 0; q < KC; ++q) {
        const int r = kr(q), kk = k0 + kq(q);
        v[q] = (base + r < lim && kk < o.k) ? X[(int64_t)kk + (int64_t)(base + r) * ldx] : 0.f;
      }
    } else {
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const int kk = k0 + k;
        v[k] = (rin && kk < o.k) ? X[(int64_t)(base + row) + (int64_t)kk * ldx] : 0.f;
      }
    }
  };
  auto step = [&](int ch, float (&v)[KC]) -> bool {
    const int s = ch & 1;
    unsigned char* buf = smem + s * STAGE;
    if (ch >= 2 && !wait_buf(s)) s_fail = 1;   // buffer s is free again
    __syncthreads();
    if (s_fail) return false;
    if (kfast) {
      unsigned char* hi = buf + (isA ? 0 : 2 * TILE_A);
      unsigned char* lo = hi + (isA ? TILE_A : TILE_B);
#pragma unroll
      for (int q = 0; q < KC; ++q) {
        const float h = tf32_hi(v[q]);
        const int off = core_off<KC>(kr(q), kq(q));
        *reinterpret_cast<float*>(hi + off) = h;
        *reinterpret_cast<float*>(lo + off) = tf32_hi(v[q] - h);
      }
    } else {
      unsigned char* hi = buf + (isA ? 0 : 2 * TILE_A);
      unsigned char* lo = hi + (isA ? TILE_A : TILE_B);
#pragma unroll
      for (int k = 0; k < KC; k += 4) {
        float4 h, l;
        h.x = tf32_hi(v[k]);
        h.y = tf32_hi(v[k + 1]);
        h.z = tf32_hi(v[k + 2]);
        h.w = tf32_hi(v[k + 3]);
        l.x = tf32_hi(v[k] - h.x);
        l.y = tf32_hi(v[k + 1] - h.y);
        l.z = tf32_hi(v[k + 2] - h.z);
        l.w = tf32_hi(v[k + 3] - h.w);
        const int off = core_off<KC>(row, k);
        *reinterpret_cast<float4*>(hi + off) = h;
        *reinterpret_cast<float4*>(lo + off) = l;
      }
    }
    if (ch + 2 < nchunk) load(ch + 2, v);
    asm volatile("fence.proxy.async.shared::cta;\n");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      const uint32_t ah = smem_u32(buf), al = ah + TILE_A, bh = ah + 2 * TILE_A,
                     bl = bh + TILE_B;
      for (int ks = 0; ks < KC / 8; ++ks) {
        const uint32_t off = ks * 256;   // two core matrices of K per instruction
        const uint32_t acc0 = (ch > 0 || ks > 0) ? 1u : 0u;
        constexpr uint32_t SBO = KC * 32;   // 8 rows x KC floats
        mma_tf32(tmem, sdesc(ah + off, 128, SBO), sdesc(bh + off, 128, SBO), idesc, acc0);
        mma_tf32(tmem, sdesc(ah + off, 128, SBO), sdesc(bl + off, 128, SBO), idesc, 1u);
        mma_tf32(tmem, sdesc(al + off, 128, SBO), sdesc(bh + off, 128, SBO), idesc, 1u);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_u32(&mbar[s])));
    }
    outstanding[s] = true;
    return true;
  };
  float va[KC], vb[KC];
  if (nchunk > 0) load(0, va);
  if (nchunk > 1) load(1, vb);
  for (int ch = 0; ch < nchunk && ok; ch += 2) {
    if (!step(ch, va)) ok = false;
    else if (ch + 1 < nchunk && !step(ch + 1, vb)) ok = false;
  }
  // the last one or two chunks are still in flight
  if (ok) {
    for (int ch = max(0, nchunk - 2); ch < nchunk; ++ch)
      if (!wait_buf(ch & 1)) ok = false;
  }
  // one verdict for the whole CTA: the epilogue's tcgen05.ld is warp-collective
  ok = __syncthreads_and(ok) != 0;
  if (!ok) {
    // drain: wait once more (bounded) for every commit this thread has not
    // seen complete, so that no product is still writing the accumulator
    // when it is freed below; a commit that never arrives is left behind
    for (int s = 0; s < 2; ++s)
      if (outstanding[s]) wait_buf(s);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  if (ok && nchunk > 0 && warp < 8) {
    // warps 0-7: warp w reads TMEM lanes 32 (w % 4) .. (tile rows) and half
    // w / 4 of the columns
    const int r = rb + (warp % 4) * 32 + lane;
    const float al = o.alpha;
    const int ch0 = (warp / 4) * (TN / 2);
    for (int c0 = ch0; c0 < ch0 + TN / 2; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)((warp % 4) * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
          "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n");
      if (r < o.m) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = cb + c0 + j;
          if (c < o.n) {
            if (gridDim.z > 1) {
              Wk[woff[blockIdx.y] + (int64_t)blockIdx.z * o.m * o.n + r + (int64_t)c * o.m] =
                  __uint_as_float(v[j]);
            } else {
              float* cp = &C[(int64_t)r + (int64_t)c * o.ldc];
              const float x = al * __uint_as_float(v[j]);
              *cp = o.beta != 0.f ? *cp + x : x;
            }
          }
        }
      }
    }
  } else if (ok && nchunk == 0 && gridDim.z > 1 && warp < 4) {
    // an empty share of a split product contributes zero
    const int r = rb + warp * 32 + lane;
    if (r < o.m)
      for (int c = cb; c < min(o.n, cb + TN); ++c)
        Wk[woff[blockIdx.y] + (int64_t)blockIdx.z * o.m * o.n + r + (int64_t)c * o.m] = 0.f;
  } else if (!ok && tid == 0) {
    atomicCAS(&flags[FLAG_TIMEOUT], -1, (int)blockIdx.y);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TN));
}

// C = beta C + alpha (sum of the split partial tiles), summed in split order
__global__ void k_splitk_reduce(const GemmOp* __restrict__ ops, const int64_t* __restrict__ woff,
                                const float* __restrict__ Wk, int S, float* Cb) {
  const GemmOp o = ops[blockIdx.y];
  const int64_t mn = (int64_t)o.m * o.n;
  const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (e >= mn) return;
  const float* w = Wk + woff[blockIdx.y] + e;
  float s = 0.f;
  for (int z = 0; z < S; ++z) s += w[z * mn];
  const int r = (int)(e % o.m), c = (int)(e / o.m);
  float* cp = Cb + o.C + r + (int64_t)c * o.ldc;
  const float x = o.alpha * s;
  *cp = o.beta != 0.f ? *cp + x : x;
}

}  // namespace

template <int KC, int TN>
void launch_tc(const GemmOp* d_ops, int nops, int mt, const float* Abase, const float* Bbase,
               float* Cbase, int* d_flags, cudaStream_t st, int S = 1,
               const int64_t* d_woff = nullptr, float* Wk = nullptr) {
  constexpr size_t smem = 2 * (size_t)(2 * TC_M * KC * 4 + 2 * TN * KC * 4);
  static const bool attr = [] {   // initialised once, also under concurrent factorizations
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc<KC, TN>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return true;
  }();
  (void)attr;
  for (int f0 = 0; f0 < nops; f0 += 65535) {
    const int nb = std::min(65535, nops - f0);
    k_gemm_tc<KC, TN><<<dim3(mt, nb, S), TC_M + TN, smem, st>>>(
        d_ops + f0, Abase, Bbase, Cbase, d_flags, d_woff ? d_woff + f0 : nullptr, Wk);
    HIF_CHECK_LAUNCH();
  }
}

namespace {

// tile variants (see tune.h): 0 = KC 16 / 128 x 128, 1 = 16 / 128 x 256,
// 2 = 32 / 128 x 128
constexpr int VAR_KC[3] = {16, 16, 32};
constexpr int VAR_TN[3] = {128, 256, 128};
constexpr int VAR_PER_SM[3] = {3, 2, 1};

int sm_count() {
  static const int nsm = [] {
    int dev = 0, count = 0;
    HIF_CUDA_TRY(cudaGetDevice(&dev));
    HIF_CUDA_TRY(cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev));
    return count;
  }();
  return nsm;
}

void launch_variant(int v, const GemmOp* d_ops, int nops, int mt, const float* Abase,
                    const float* Bbase, float* Cbase, int* d_flags, cudaStream_t st, int S,
                    const int64_t* d_woff, float* Wk) {
  if (v == 2) launch_tc<32, 128>(d_ops, nops, mt, Abase, Bbase, Cbase, d_flags, st, S, d_woff, Wk);
  else if (v == 1) launch_tc<16, 256>(d_ops, nops, mt, Abase, Bbase, Cbase, d_flags, st, S, d_woff, Wk);
  else launch_tc<16, 128>(d_ops, nops, mt, Abase, Bbase, Cbase, d_flags, st, S, d_woff, Wk);
}

// Output tiles of the batch for tile width tn, and the widest product's.
void tile_counts(const GemmOp* h_ops, int nops, int tn, int* tiles, int* mt) {
  *tiles = 0;
  *mt = 1;
  for (int i = 0; i < nops; ++i) {
    const int t = ceil_div(h_ops[i].m, TC_M) * ceil_div(h_ops[i].n, tn);
    *tiles += t;
    *mt = std::max(*mt, t);
  }
}

// Split of K: S minimises the waves per unit of work, ceil(tiles S /
// capacity) / S, with at least 16 chunks of K per share; only for launches
// that leave SMs idle, never for triangular (lower) products.  Computed from
// the built-in variant so that a tuned tile shape never changes it.
int split_k(const GemmOp* h_ops, int nops, int v) {
  int tiles = 0, mt = 1, kmin = 1 << 30;
  bool any_lower = false;
  tile_counts(h_ops, nops, VAR_TN[v], &tiles, &mt);
  for (int i = 0; i < nops; ++i) {
    kmin = std::min(kmin, h_ops[i].k);
    any_lower = any_lower || h_ops[i].lower;
  }
  const int cap = VAR_PER_SM[v] * sm_count();
  int S = 1;
  if (!any_lower && nops <= 65535 && tiles < cap) {
    const int smax =
        std::max(1, std::min({8, kmin / (16 * VAR_KC[v]), ceil_div(2 * cap, std::max(1, tiles))}));
    double best = 1e30;
    for (int q = 1; q <= smax; ++q) {
      const double cost = (double)ceil_div(tiles * q, cap) / q;
      if (cost < best - 1e-9) {
        best = cost;
        S = q;
      }
    }
  }
  return S;
}

}  // namespace

void gemm_tc(const GemmOp* d_ops, const GemmOp* h_ops, int nops, const float* Abase,
             const float* Bbase, float* Cbase, int* d_flags, cudaStream_t st, const char* name) {
  if (nops == 0) return;
  int mmax = 0, nmax = 0, kmax = 0;
  double fl = 0;
  for (int i = 0; i < nops; ++i) {
    mmax = std::max(mmax, h_ops[i].m);
    nmax = std::max(nmax, h_ops[i].n);
    kmax = std::max(kmax, h_ops[i].k);
    fl += 2.0 * h_ops[i].m * (double)h_ops[i].n * h_ops[i].k * (h_ops[i].lower ? 0.5 : 1.0);
  }
  // built-in rule: few rows (one tile, mostly padding): fewer, longer
  // chunks; wide products: 128 x 256 tiles (half the A staging per product)
  const bool narrow = mmax <= 64;
  const int vdef = narrow ? 2 : (nmax >= 256 ? 1 : 0);
  const int S = split_k(h_ops, nops, vdef);
  int tiles = 0, mt = 1;
  tile_counts(h_ops, nops, 128, &tiles, &mt);
  const int scls = gemm_shape_class(mmax, nmax, kmax), wcls = gemm_waves_class(tiles, sm_count());
  if (tune_session_active()) tune_record_gemm(scls, wcls, h_ops, nops, fl);
  // a tuned tile shape (every variant accumulates each entry in the same
  // order; with K split, only variants with the same K chunk keep the split)
  int v = vdef, vt = -1;
  if (tune_gemm_lookup(scls, wcls, &vt) && (S == 1 || VAR_KC[vt] == VAR_KC[vdef])) v = vt;
  tile_counts(h_ops, nops, VAR_TN[v], &tiles, &mt);
  ProfScope ps(name, st, fl, 0.0);
  int64_t* d_woff = nullptr;
  float* Wk = nullptr;
  if (S > 1) {
    std::vector<int64_t> woff(nops);
    int64_t tot = 0;
    int64_t mnmax = 1;
    for (int i = 0; i < nops; ++i) {
      woff[i] = tot;
      tot += (int64_t)S * h_ops[i].m * h_ops[i].n;
      mnmax = std::max<int64_t>(mnmax, (int64_t)h_ops[i].m * h_ops[i].n);
    }
    HIF_CUDA_TRY(cudaMallocAsync(&d_woff, sizeof(int64_t) * nops, st));
    HIF_CUDA_TRY(cudaMallocAsync(&Wk, sizeof(float) * tot, st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_woff, woff.data(), sizeof(int64_t) * nops,
                                 cudaMemcpyHostToDevice, st));
    launch_variant(v, d_ops, nops, mt, Abase, Bbase, Cbase, d_flags, st, S, d_woff, Wk);
    k_splitk_reduce<<<dim3((unsigned)ceil_div(mnmax, 256), nops), 256, 0, st>>>(d_ops, d_woff, Wk,
                                                                                S, Cbase);
    HIF_CHECK_LAUNCH();
    HIF_CUDA_TRY(cudaFreeAsync(Wk, st));
    HIF_CUDA_TRY(cudaFreeAsync(d_woff, st));
    return;
  }
  launch_variant(v, d_ops, nops, mt, Abase, Bbase, Cbase, d_flags, st, 1, nullptr, nullptr);
}

// Time the tile variants on the product shapes recorded during a tuning
// factorization (one batch per bucket, the one with the most flops), on
// synthetic operands of those shapes, and keep the fastest per bucket.
void tune_gemm_from_records(cudaStream_t st) {
  std::vector<GemmShapeRec> recs = tune_take_gemm_records();
  int* d_flags = nullptr;
  HIF_CUDA_TRY(cudaMallocAsync(&d_flags, sizeof(int) * FLAG_COUNT, st));
  HIF_CUDA_TRY(cudaMemsetAsync(d_flags, 0xff, sizeof(int) * FLAG_COUNT, st));
  cudaEvent_t e0, e1;
  HIF_CUDA_TRY(cudaEventCreate(&e0));
  HIF_CUDA_TRY(cudaEventCreate(&e1));
  for (GemmShapeRec& r : recs) {
    // compact operand arenas of the recorded shapes
    std::vector<GemmOp> ops = r.ops;
    int64_t na = 0, nb = 0, nc = 0;
    int mmax = 0, nmax = 0;
    for (GemmOp& o : ops) {
      const int64_t asz = (int64_t)o.lda * (o.transA ? o.m : o.k);
      const int64_t bsz = (int64_t)o.ldb * (o.transB ? o.k : o.n);
      const int64_t csz = (int64_t)o.ldc * o.n;
      o.A = na;
      o.B = nb;
      o.C = nc;
      na += asz;
      nb += bsz;
      nc += csz;
      mmax = std::max(mmax, o.m);
      nmax = std::max(nmax, o.n);
    }
    float *A = nullptr, *B = nullptr, *C = nullptr;
    GemmOp* d_ops = nullptr;
    HIF_CUDA_TRY(cudaMallocAsync(&A, sizeof(float) * std::max<int64_t>(1, na), st));
    HIF_CUDA_TRY(cudaMallocAsync(&B, sizeof(float) * std::max<int64_t>(1, nb), st));
    HIF_CUDA_TRY(cudaMallocAsync(&C, sizeof(float) * std::max<int64_t>(1, nc), st));
    HIF_CUDA_TRY(cudaMallocAsync(&d_ops, sizeof(GemmOp) * ops.size(), st));
    HIF_CUDA_TRY(cudaMemsetAsync(A, 0, sizeof(float) * std::max<int64_t>(1, na), st));
    HIF_CUDA_TRY(cudaMemsetAsync(B, 0, sizeof(float) * std::max<int64_t>(1, nb), st));
    HIF_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(float) * std::max<int64_t>(1, nc), st));
    HIF_CUDA_TRY(cudaMemcpyAsync(d_ops, ops.data(), sizeof(GemmOp) * ops.size(),
                                 cudaMemcpyHostToDevice, st));
    const int nops = (int)ops.size();
    const bool narrow = mmax <= 64;
    const int vdef = narrow ? 2 : (nmax >= 256 ? 1 : 0);
    const int S = split_k(ops.data(), nops, vdef);
    double best = 1e30;
    int vbest = vdef;
    double secs[3] = {0, 0, 0};
    for (int v = 0; v < 3; ++v) {
      if (S > 1 && VAR_KC[v] != VAR_KC[vdef]) continue;
      int tiles = 0, mt = 1;
      tile_counts(ops.data(), nops, VAR_TN[v], &tiles, &mt);
      std::vector<float> ms;
      for (int rep = 0; rep < 4; ++rep) {
        int64_t* d_woff = nullptr;
        float* Wk = nullptr;
        std::vector<int64_t> woff(nops);
        if (S > 1) {
          int64_t tot = 0;
          for (int i = 0; i < nops; ++i) {
            woff[i] = tot;
            tot += (int64_t)S * ops[i].m * ops[i].n;
          }
          HIF_CUDA_TRY(cudaMallocAsync(&d_woff, sizeof(int64_t) * nops, st));
          HIF_CUDA_TRY(cudaMallocAsync(&Wk, sizeof(float) * tot, st));
          HIF_CUDA_TRY(cudaMemcpyAsync(d_woff, woff.data(), sizeof(int64_t) * nops,
                                       cudaMemcpyHostToDevice, st));
        }
        HIF_CUDA_TRY(cudaEventRecord(e0, st));
        launch_variant(v, d_ops, nops, mt, A, B, C, d_flags, st, S, d_woff, Wk);
        HIF_CUDA_TRY(cudaEventRecord(e1, st));
        HIF_CUDA_TRY(cudaEventSynchronize(e1));
        float t = 0.f;
        HIF_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
        if (rep > 0) ms.push_back(t);   // the first run warms up
        if (Wk) HIF_CUDA_TRY(cudaFreeAsync(Wk, st));
        if (d_woff) HIF_CUDA_TRY(cudaFreeAsync(d_woff, st));
      }
      std::sort(ms.begin(), ms.end());
      secs[v] = 1e-3 * ms[ms.size() / 2];
      if (secs[v] < best) {
        best = secs[v];
        vbest = v;
      }
    }
    tune_gemm_set(r.shape_cls, r.waves_cls, vbest, secs);
    HIF_CUDA_TRY(cudaFreeAsync(d_ops, st));
    HIF_CUDA_TRY(cudaFreeAsync(C, st));
    HIF_CUDA_TRY(cudaFreeAsync(B, st));
    HIF_CUDA_TRY(cudaFreeAsync(A, st));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int hflags[FLAG_COUNT];
  HIF_CUDA_TRY(cudaMemcpyAsync(hflags, d_flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
  HIF_CUDA_TRY(cudaStreamSynchronize(st));
  HIF_CUDA_TRY(cudaFree(d_flags));
  if (hflags[FLAG_TIMEOUT] >= 0) throw Error{HIF_ERR_TIMEOUT, "a tensor-core wait expired while tuning"};
}

}  // namespace hif
