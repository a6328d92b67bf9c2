// C ABI of the GB300 HIF library: factorization driver (level loop of §2.4),
// application of F^{-1} (forward / backward sweeps) and the preconditioned
// conjugate-gradient solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <future>
#include <memory>
#include <mutex>
#include <numeric>
#include <type_traits>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "dense.cuh"
#include "front.cuh"
#include "solve.cuh"
#include "symbolic.h"
#include "tune.h"

namespace hif {

template <typename T>
void interpolative_decomposition(SkelDesc* d_f, const SkelDesc* h_f, int nf, T* Garena,
                                 size_t arena_elems, int32_t* perm, T* Farena, int32_t* stepAr,
                                 double eps, cudaStream_t st, int8_t* route);
template <typename T>
void id_solve_t(const SkelDesc* d_f, const SkelDesc* h_f, const std::vector<int>& fronts,
                const T* Garena, const int32_t* perm, T* Farena, cudaStream_t st);
template <typename T>
void reduce_rows_qr(const SkelDesc* h_f, const std::vector<int>& which, T* Garena, T* Rout,
                    const std::vector<int64_t>& rOff, int* d_flags, bool tensor_cores,
                    cudaStream_t st);

namespace {
thread_local std::string g_last_error;
thread_local int64_t g_launches = 0;
}  // namespace

void set_last_error(const std::string& msg) { g_last_error = msg; }
int64_t& launch_counter() { return g_launches; }

namespace {

using Clock = std::chrono::steady_clock;
double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

// HIF_TRACE=1 prints the wall time of each host phase of hif_factor to stderr.
// HIF_TRACE=2 also drains the stream at every mark and prints how long the
// drain took: a phase whose drain is near zero left the GPU idle while the
// host worked (the drains serialize host and GPU, so the total grows).
struct Trace {
  int mode = std::getenv("HIF_TRACE") ? std::atoi(std::getenv("HIF_TRACE")) : 0;
  bool on = mode > 0;
  cudaStream_t st = nullptr;
  Clock::time_point t = Clock::now();
  void mark(int level, const char* what) {
    if (!on) return;
    const double ms = 1e3 * seconds_since(t);
    double drain = 0.0;
    if (mode >= 2) {
      const auto t1 = Clock::now();
      cudaStreamSynchronize(st);
      drain = 1e3 * seconds_since(t1);
    }
    std::fprintf(stderr, "[hif] level %d %-28s %9.2f ms  drain %8.2f ms\n", level, what, ms, drain);
    t = Clock::now();
  }
};

// ---- device memory --------------------------------------------------------------

struct MemStats {
  size_t cur = 0, peak = 0;
};

class DevBuf {
 public:
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { swap(o); }
  DevBuf& operator=(DevBuf&& o) noexcept {
    release();
    swap(o);
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t bytes, MemStats* ms) {
    release();
    ms_ = ms;
    if (bytes == 0) return;
    HIF_CUDA_TRY(cudaMalloc(&p_, bytes));
    bytes_ = bytes;
    if (ms_) {
      ms_->cur += bytes;
      ms_->peak = std::max(ms_->peak, ms_->cur);
    }
  }
  // Stream-ordered: allocated and later freed in order on `st` (no device
  // synchronisation); for the temporaries of one factorization.
  void alloc_async(size_t bytes, MemStats* ms, cudaStream_t st) {
    release();
    ms_ = ms;
    if (bytes == 0) return;
    HIF_CUDA_TRY(cudaMallocAsync(&p_, bytes, st));
    st_ = st;
    async_ = true;
    bytes_ = bytes;
    if (ms_) {
      ms_->cur += bytes;
      ms_->peak = std::max(ms_->peak, ms_->cur);
    }
  }
  void release() {
    if (p_) {
      if (async_) cudaFreeAsync(p_, st_);
      else cudaFree(p_);
      if (ms_) ms_->cur -= bytes_;
    }
    p_ = nullptr;
    bytes_ = 0;
    async_ = false;
  }
  template <typename U>
  U* as() const { return static_cast<U*>(p_); }
  size_t bytes() const { return bytes_; }

 private:
  void swap(DevBuf& o) {
    std::swap(p_, o.p_);
    std::swap(bytes_, o.bytes_);
    std::swap(ms_, o.ms_);
    std::swap(st_, o.st_);
    std::swap(async_, o.async_);
  }
  void* p_ = nullptr;
  size_t bytes_ = 0;
  MemStats* ms_ = nullptr;
  cudaStream_t st_ = nullptr;
  bool async_ = false;
};

template <typename U, typename A>
void upload_async(DevBuf& b, const std::vector<U, A>& h, MemStats* ms, cudaStream_t st) {
  b.alloc_async(h.size() * sizeof(U), ms, st);
  if (!h.empty())
    HIF_CUDA_TRY(cudaMemcpyAsync(b.as<void>(), h.data(), h.size() * sizeof(U),
                                 cudaMemcpyHostToDevice, st));
}

template <typename U, typename A>
void upload(DevBuf& b, const std::vector<U, A>& h, MemStats* ms, cudaStream_t st) {
  b.alloc(h.size() * sizeof(U), ms);
  if (!h.empty())
    HIF_CUDA_TRY(cudaMemcpyAsync(b.as<void>(), h.data(), h.size() * sizeof(U),
                                 cudaMemcpyHostToDevice, st));
}

// Device of a device (or managed) pointer; -1 for host memory.
int pointer_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return -1;
  return at.device;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ---- apply stages ----------------------------------------------------------------
// One stage per front batch (cells of a level, faces, edges, root).  The
// forward sweep runs the stages in order, the backward sweep in reverse.
// Work layout of a stage (per right-hand side): v = gathered values of every
// front's DOFs (front f at voff_f), t = a second vector of the same size at
// offset nidx.
struct GemvList {
  std::vector<GemvOp> h;
  DevBuf d;
  int trans = 0;
  int mat = 0;   // 0: panel arena, 1: interpolation-matrix arena
  int tiles = -1;   // widest op's CTA count along x (cached for grouped launches)
  int get_tiles() {
    if (tiles < 0) tiles = gemv_tiles(h.data(), (int)h.size(), trans);
    return tiles;
  }
};

struct Stage {
  int kind = 0;                 // 0 = cells (or root), 1 = faces / edges
  int level = 0;
  int64_t nidx = 0;
  DevBuf idx;                   // gather list (global DOF per work slot)
  DevBuf panels;                // [Linv; X^T] per front
  DevBuf tmats;                 // T per front (skeleton stages)
  std::vector<GemvList> fwd, bwd;
  DevBuf set_g, set_p;          // y[g] = work[p] (both sweeps)
  int64_t nset = 0;
  DevBuf acc_tgt, acc_ptr, acc_src;   // forward, cells: y[g] -= sum work[src]
  int64_t nacc = 0;
  int64_t entries = 0;          // factor entries read per sweep
};

struct FactorBase {
  virtual ~FactorBase() = default;
  virtual void apply(const double* f_dev, double* u_dev, int nrhs, cudaStream_t st) = 0;
  // Bytes of work space the sweeps need for nrhs right-hand sides, and the
  // sweeps run in caller-provided work space (nothing is allocated).
  virtual size_t sweep_scratch_bytes(int nrhs) const = 0;
  virtual void apply_in_scratch(const double* f_dev, double* u_dev, int nrhs, void* scratch,
                                cudaStream_t st) = 0;
  int n = 0, m = 0, L = 0, precision = 0;
  int bc = 0;                   // 0: zero Dirichlet, 1: periodic
  int device = -1;              // CUDA device holding every buffer of the factor
  double eps = 0;
  MemStats mem;
  DevBuf cpl, diag;             // operator for the residual
  // active[l]: sorted grid indices of the DOFs still active after level l
  // (Sigma^{l+1} of §2.4); active[L-1] is the root set
  std::vector<std::vector<int32_t>> active;
  hif_stats stats{};
  hif_options opt{};
};

template <typename T>
struct Factor : FactorBase {
  std::vector<Stage> stages;
  DevBuf y, work;               // apply buffers (grown on demand)
  int64_t work_cap = 0, y_cap = 0;
  int64_t work_stride = 0;
  // with opt.use_graphs: the two sweeps of an apply (every stage forward,
  // then backward) captured once per nrhs on a private stream and replayed
  // on the caller's stream; the graphs name y and work, so they are dropped
  // whenever those buffers grow
  struct SweepGraph {
    int nrhs;
    cudaGraphExec_t exec;
    int64_t kernels;             // kernels one replay runs
  };
  std::vector<SweepGraph> graphs;
  cudaStream_t cap_st = nullptr;

  ~Factor() override {
    drop_graphs();
    if (cap_st) cudaStreamDestroy(cap_st);
  }
  void drop_graphs() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
  }
  void sweeps(T* yv, T* w, int nrhs, cudaStream_t st) {
    const int64_t N = (int64_t)n * n * n;
    for (auto& s : stages) run_stage(s, true, yv, N, w, work_stride, nrhs, st);
    for (auto it = stages.rbegin(); it != stages.rend(); ++it)
      run_stage(*it, false, yv, N, w, work_stride, nrhs, st);
  }
  // Algorithmic counts of the two sweeps for nrhs right-hand sides: every
  // stored factor entry is read once per sweep and per block of right-hand
  // sides (blocks of 16, 8, 4, 2, 1) and used in one multiply-add per
  // column; gathers and sets move an index and the values in and out.
  void sweep_counts(int nrhs, double* flops, double* bytes) const {
    int64_t ent = 0, slots = 0;
    for (const Stage& s : stages) {
      ent += s.entries;
      slots += s.nidx + s.nset;
    }
    int blocks = 0;
    for (int left = nrhs; left > 0;) {
      const int R = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
      left -= R;
      ++blocks;
    }
    *flops = 2.0 * 2.0 * (double)ent * nrhs;
    *bytes = 2.0 * ((double)ent * sizeof(T) * blocks + (double)slots * (6.0 + 2.0 * sizeof(T) * nrhs));
  }
  void sweeps_maybe_graph(T* yv, T* w, int nrhs, cudaStream_t st) {
    if (!opt.use_graphs) {
      sweeps(yv, w, nrhs, st);
      return;
    }
    const SweepGraph* g = nullptr;
    for (auto& x : graphs)
      if (x.nrhs == nrhs) g = &x;
    if (!g) {
      if (!cap_st) HIF_CUDA_TRY(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      const int64_t l0 = launch_counter();
      {
        // the kernel profile times the replay as a whole, not the captured launches
        ProfSuspend quiet;
        HIF_CUDA_TRY(cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeThreadLocal));
        sweeps(yv, w, nrhs, cap_st);
        HIF_CUDA_TRY(cudaStreamEndCapture(cap_st, &graph));
      }
      const int64_t nk = launch_counter() - l0;
      launch_counter() = l0;   // counted again at every replay
      const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      HIF_CUDA_TRY(e);
      graphs.push_back(SweepGraph{nrhs, exec, nk});
      g = &graphs.back();
    }
    double fl = 0.0, by = 0.0;
    if (prof_enabled()) sweep_counts(nrhs, &fl, &by);
    ProfScope ps("apply_sweeps_graph", st, fl, by);
    HIF_CUDA_TRY(cudaGraphLaunch(g->exec, st));
    launch_counter() += g->kernels;
  }

  void run_stage(Stage& s, bool fwd, T* yv, int64_t ys, T* w, int64_t vs, int nrhs,
                 cudaStream_t st) {
    vec_gather<T>(s.idx.as<int32_t>(), s.nidx, yv, ys, w, vs, 0, nrhs, st);
    auto& lists = fwd ? s.fwd : s.bwd;
    for (auto& gl : lists) {
      if (gl.h.empty()) continue;
      const T* M = gl.mat ? s.tmats.as<T>() : s.panels.as<T>();
      gemv_batched<T>(gl.d.as<GemvOp>(), gl.h.data(), (int)gl.h.size(), gl.trans, M, w, vs, nrhs,
                      st);
    }
    vec_set<T>(s.set_g.as<int32_t>(), s.set_p.as<int32_t>(), s.nset, yv, ys, w, vs, nrhs, st);
    if (fwd && s.nacc)
      vec_accumulate<T>(s.acc_tgt.as<int32_t>(), s.acc_ptr.as<int64_t>(), s.acc_src.as<int32_t>(),
                        s.nacc, yv, ys, w, vs, nrhs, st);
  }

  // the apply's vectors for nrhs right-hand sides (grown on demand; the
  // captured graphs name them, so they are dropped when the buffers grow)
  void ensure_apply_buffers(int nrhs) {
    const int64_t N = (int64_t)n * n * n;
    if (y_cap < N * nrhs) {
      drop_graphs();
      y.alloc(sizeof(T) * N * nrhs, &mem);
      y_cap = N * nrhs;
    }
    if (work_cap < work_stride * nrhs) {
      drop_graphs();
      work.alloc(sizeof(T) * std::max<int64_t>(1, work_stride * nrhs), &mem);
      work_cap = work_stride * nrhs;
    }
  }

  void apply(const double* f_dev, double* u_dev, int nrhs, cudaStream_t st) override {
    const int64_t N = (int64_t)n * n * n;
    ensure_apply_buffers(nrhs);
    T* yv = y.as<T>();
    T* w = work.as<T>();
    vec_convert_in<T>(f_dev, yv, N * nrhs, st);
    sweeps_maybe_graph(yv, w, nrhs, st);
    vec_convert_out<T>(yv, u_dev, N * nrhs, st);
  }

  static size_t round256(size_t b) { return (b + 255) / 256 * 256; }

  size_t sweep_scratch_bytes(int nrhs) const override {
    const int64_t N = (int64_t)n * n * n;
    return round256(sizeof(T) * N * nrhs) +
           round256(sizeof(T) * std::max<int64_t>(1, work_stride * nrhs));
  }

  void apply_in_scratch(const double* f_dev, double* u_dev, int nrhs, void* scratch,
                        cudaStream_t st) override {
    const int64_t N = (int64_t)n * n * n;
    T* yv = static_cast<T*>(scratch);
    T* w = reinterpret_cast<T*>(static_cast<char*>(scratch) + round256(sizeof(T) * N * nrhs));
    vec_convert_in<T>(f_dev, yv, N * nrhs, st);
    sweeps(yv, w, nrhs, st);
    vec_convert_out<T>(yv, u_dev, N * nrhs, st);
  }
};

// ---- grouped apply over several factors --------------------------------------
// The sweeps of several factors of one precision run in shared launches.  At
// step t of the forward sweep every factor that has a stage t contributes
// its gather, its mat-vec lists, its set and its accumulate to one launch
// each (a mat-vec list: one launch per transpose form and block size of
// right-hand sides); the backward sweep aligns the factors' stages from the
// last one.  Each factor keeps its own buffers and its own kernels'
// arithmetic, so its result is bitwise that of its own apply.
template <typename T>
void grouped_sweeps(const std::vector<Factor<T>*>& Fs, const std::vector<int>& nrhs,
                    cudaStream_t st) {
  struct Launch {
    int kind;              // 0 gather, 1 set, 2 accumulate, 3 mat-vec
    int trans, R, count;   // count: jobs or segments
    size_t off;            // byte offset of the descriptors in the upload
    int64_t nops;
    int mx;
    double fl, by;
  };
  std::vector<unsigned char> blob;
  std::vector<Launch> seq;
  auto push = [&](const void* p, size_t bytes) {
    const size_t off = (blob.size() + 255) / 256 * 256;
    blob.resize(off + bytes);
    std::memcpy(blob.data() + off, p, bytes);
    return off;
  };
  const int nh = (int)Fs.size();
  std::vector<T*> yv(nh), wv(nh);
  std::vector<int64_t> ys(nh), vs(nh);
  std::vector<std::vector<std::pair<int, int>>> blocks(nh);   // (first column, R)
  size_t S = 0;
  for (int h = 0; h < nh; ++h) {
    yv[h] = Fs[h]->y.template as<T>();
    wv[h] = Fs[h]->work.template as<T>();
    ys[h] = (int64_t)Fs[h]->n * Fs[h]->n * Fs[h]->n;
    vs[h] = Fs[h]->work_stride;
    for (int q0 = 0; q0 < nrhs[h];) {
      const int left = nrhs[h] - q0;
      const int R = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
      blocks[h].push_back({q0, R});
      q0 += R;
    }
    S = std::max(S, Fs[h]->stages.size());
  }
  const bool prof = prof_enabled();
  for (int dir = 0; dir < 2; ++dir) {
    for (size_t t = 0; t < S; ++t) {
      std::vector<std::pair<int, Stage*>> at;
      for (int h = 0; h < nh; ++h) {
        const size_t sh = Fs[h]->stages.size();
        if (t < sh) at.push_back({h, &Fs[h]->stages[dir == 0 ? t : sh - 1 - t]});
      }
      auto vec_launch = [&](int kind) {
        std::vector<VecJob<T>> jobs;
        for (auto& [h, st_] : at) {
          VecJob<T> j{};
          j.y = yv[h];
          j.ys = ys[h];
          j.w = wv[h];
          j.vs = vs[h];
          j.nrhs = nrhs[h];
          if (kind == 0) {
            j.a = st_->idx.template as<int32_t>();
            j.cnt = st_->nidx;
          } else if (kind == 1) {
            j.a = st_->set_g.template as<int32_t>();
            j.b = st_->set_p.template as<int32_t>();
            j.cnt = st_->nset;
          } else {
            j.a = st_->acc_tgt.template as<int32_t>();
            j.b = st_->acc_src.template as<int32_t>();
            j.ptr = st_->acc_ptr.template as<int64_t>();
            j.cnt = st_->nacc;
          }
          if (j.cnt) jobs.push_back(j);
        }
        if (jobs.empty()) return;
        Launch l{kind, 0, 0, (int)jobs.size(), push(jobs.data(), sizeof(VecJob<T>) * jobs.size()),
                 0, 0, 0.0, 0.0};
        seq.push_back(l);
      };
      vec_launch(0);
      size_t nl = 0;
      for (auto& [h, st_] : at) nl = std::max(nl, (dir ? st_->bwd : st_->fwd).size());
      for (size_t i = 0; i < nl; ++i) {
        std::map<std::pair<int, int>, std::vector<GemvSeg<T>>> buckets;
        std::map<std::pair<int, int>, Launch> meta;
        for (auto& [h, st_] : at) {
          auto& lists = dir ? st_->bwd : st_->fwd;
          if (i >= lists.size() || lists[i].h.empty()) continue;
          GemvList& gl = lists[i];
          const T* M = gl.mat ? st_->tmats.template as<T>() : st_->panels.template as<T>();
          double ent = 0.0, vecs = 0.0;
          if (prof)
            for (const GemvOp& o : gl.h) {
              ent += o.tri ? 0.5 * (double)o.cols * (o.cols + 1) : (double)o.rows * o.cols;
              vecs += (double)(o.rows + o.cols) * (o.beta_one ? 1.5 : 1.0);
            }
          for (auto [q0, R] : blocks[h]) {
            const auto key = std::make_pair(gl.trans, R);
            Launch& l = meta[key];
            l.kind = 3;
            l.trans = gl.trans;
            l.R = R;
            buckets[key].push_back(
                GemvSeg<T>{gl.d.as<GemvOp>(), M, wv[h] + (int64_t)q0 * vs[h], vs[h], l.nops});
            l.nops += (int64_t)gl.h.size();
            l.mx = std::max(l.mx, gl.get_tiles());
            l.fl += 2.0 * ent * R;
            l.by += sizeof(T) * (ent + R * vecs);
          }
        }
        for (auto& [key, segs] : buckets) {
          Launch l = meta[key];
          l.count = (int)segs.size();
          l.off = push(segs.data(), sizeof(GemvSeg<T>) * segs.size());
          seq.push_back(l);
        }
      }
      vec_launch(1);
      if (dir == 0) vec_launch(2);
    }
  }
  if (seq.empty()) return;
  DevBuf d;
  d.alloc_async(blob.size(), nullptr, st);
  HIF_CUDA_TRY(cudaMemcpyAsync(d.as<void>(), blob.data(), blob.size(), cudaMemcpyHostToDevice, st));
  const unsigned char* base = d.as<unsigned char>();
  for (const Launch& l : seq) {
    if (l.kind == 3) {
      gemv_segments<T>(reinterpret_cast<const GemvSeg<T>*>(base + l.off), l.count, l.nops, l.mx,
                       l.trans, l.R, l.fl, l.by, st);
    } else {
      vec_grouped<T>(l.kind, reinterpret_cast<const VecJob<T>*>(base + l.off),
                     reinterpret_cast<const VecJob<T>*>(blob.data() + l.off), l.count, st);
    }
  }
}

// u_h = F_h^{-1} f_h for several factors of one precision, sweeps grouped.
template <typename T>
void grouped_apply(const std::vector<Factor<T>*>& Fs, const std::vector<const double*>& f,
                   const std::vector<double*>& u, const std::vector<int>& nrhs, cudaStream_t st) {
  for (size_t h = 0; h < Fs.size(); ++h) {
    Fs[h]->ensure_apply_buffers(nrhs[h]);
    const int64_t N = (int64_t)Fs[h]->n * Fs[h]->n * Fs[h]->n;
    vec_convert_in<T>(f[h], Fs[h]->y.template as<T>(), N * nrhs[h], st);
  }
  grouped_sweeps<T>(Fs, nrhs, st);
  for (size_t h = 0; h < Fs.size(); ++h) {
    const int64_t N = (int64_t)Fs[h]->n * Fs[h]->n * Fs[h]->n;
    vec_convert_out<T>(Fs[h]->y.template as<T>(), u[h], N * nrhs[h], st);
  }
}

void grouped_apply_any(const std::vector<FactorBase*>& Fs, const std::vector<const double*>& f,
                       const std::vector<double*>& u, const std::vector<int>& nrhs,
                       cudaStream_t st) {
  if (Fs.empty()) return;
  if (Fs[0]->precision == HIF_PREC_FP32) {
    std::vector<Factor<float>*> v;
    for (FactorBase* F : Fs) v.push_back(static_cast<Factor<float>*>(F));
    grouped_apply<float>(v, f, u, nrhs, st);
  } else {
    std::vector<Factor<double>*> v;
    for (FactorBase* F : Fs) v.push_back(static_cast<Factor<double>*>(F));
    grouped_apply<double>(v, f, u, nrhs, st);
  }
}

// ---- the factorization ---------------------------------------------------------

template <typename T>
class Builder {
 public:
  Builder(Factor<T>& F, cudaStream_t st) : F_(F), st_(st), sym_(F.n, F.m, F.bc == 1) {
    tr_.st = st;
    retry_.growth = std::is_same<T, float>::value ? F.opt.retry_growth : 0.0;
    retry_.retried = &F.stats.retried_fronts;
  }
  ~Builder() {
    jobs_.clear();   // waits for the host workers
    if (up_st_) {
      cudaStreamSynchronize(up_st_);
      cudaStreamDestroy(up_st_);
    }
  }

  void run(const double* a_dev, const double* b_dev, double b_const);

 private:
  void check_flags(const char* where);
  void cell_step(std::shared_ptr<const CellPlan> cpp, DevBuf& Kar, DevBuf& cdesc_d,
                 std::vector<CellDesc>& cdesc, DevBuf& lists_d);
  // returns the number of DOFs the step eliminated (marked dead in alive)
  int64_t skel_step(const CellPlan& cp, int kind, std::vector<uint8_t>& alive, DevBuf& Kar,
                    DevBuf& cdesc_d, std::shared_ptr<const SkelPlan> plan);

  // Host side of an apply stage (gather list, mat-vec lists, set and
  // accumulate lists).  It depends only on the plan and, for faces and edges,
  // on the ID's ranks and pivots, so a worker thread builds it while the GPU
  // factors; finished stages are uploaded on a side stream whenever the host
  // waits for the GPU anyway, and the rest when the factorization ends.
  struct StageHost {
    std::vector<int32_t> idx;        // empty: the list is already on the device
    std::vector<GemvOp> fwd[3], bwd[3];
    int nfwd = 0, nbwd = 0;
    int fwd_trans[3] = {0, 0, 0}, fwd_mat[3] = {0, 0, 0};
    int bwd_trans[3] = {0, 0, 0}, bwd_mat[3] = {0, 0, 0};
    std::vector<int32_t> set_g, set_p;
    std::vector<int32_t> acc_tgt, acc_src;
    std::vector<int64_t> acc_ptr;
    int64_t entries_add = 0;
  };
  std::vector<std::pair<size_t, std::future<StageHost>>> jobs_;
  // cell stages wait until the level's plans are joined (they would compete
  // with the planning threads for the host cores)
  std::vector<std::pair<size_t, std::function<StageHost()>>> unstarted_;
  void start_stage_jobs() {
    for (auto& u : unstarted_) jobs_.emplace_back(u.first, std::async(std::launch::async, std::move(u.second)));
    unstarted_.clear();
  }
  cudaStream_t up_st_ = nullptr;
  void upload_stages(bool all);
  static StageHost cell_stage_host(std::shared_ptr<const CellPlan> cpp,
                                   std::vector<CellDesc> cdesc, std::vector<int64_t> poff,
                                   int64_t N, int64_t nidx);

  Factor<T>& F_;
  cudaStream_t st_;
  RetryOpts retry_{};
  Symbolic sym_;
  DevBuf flags_;
  int level_ = 0;
  Trace tr_;
  // next level's symbolic plan built ahead of time
  bool have_spec_ = false;
  CellPlan spec_cells_;
  std::vector<int64_t> spec_mapOff_;
  PlanVec32 spec_map_;
};

template <typename T>
void Builder<T>::check_flags(const char* where) {
  int h[FLAG_COUNT];
  HIF_CUDA_TRY(cudaMemcpyAsync(h, flags_.as<int>(), sizeof(h), cudaMemcpyDeviceToHost, st_));
  HIF_CUDA_TRY(cudaStreamSynchronize(st_));
  if (h[FLAG_TIMEOUT] >= 0)
    throw Error{HIF_ERR_TIMEOUT, std::string("a bounded device wait expired in ") + where +
                                     " at level " + std::to_string(level_) + ", front " +
                                     std::to_string(h[FLAG_TIMEOUT])};
  if (h[FLAG_NOT_SPD] >= 0)
    throw Error{HIF_ERR_NOT_SPD, std::string("non-positive Cholesky pivot in ") + where +
                                     " at level " + std::to_string(level_) + ", front " +
                                     std::to_string(h[FLAG_NOT_SPD])};
}

template <typename T>
void Builder<T>::run(const double* a_dev, const double* b_dev, double b_const) {
  const int n = F_.n;
  const int64_t N = (int64_t)n * n * n;
  auto t0 = Clock::now();
  {
    // keep the stream-ordered pool's memory between levels instead of
    // returning it to the driver at every synchronisation
    int dev = 0;
    cudaMemPool_t pool;
    HIF_CUDA_TRY(cudaGetDevice(&dev));
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  }
  F_.cpl.alloc(sizeof(double) * 3 * N, &F_.mem);
  F_.diag.alloc(sizeof(double) * N, &F_.mem);
  DevBuf bad;
  bad.alloc_async(sizeof(int), &F_.mem, st_);
  HIF_CUDA_TRY(cudaMemsetAsync(bad.as<int>(), 0, sizeof(int), st_));
  stencil_coefficients(a_dev, b_dev, b_const, n, F_.bc, F_.cpl.template as<double>(), F_.diag.template as<double>(),
                       bad.as<int>(), st_);
  int hbad = 0;
  HIF_CUDA_TRY(cudaMemcpyAsync(&hbad, bad.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, st_));
  HIF_CUDA_TRY(cudaStreamSynchronize(st_));
  if (hbad)
    throw Error{HIF_ERR_INVALID_ARG, F_.bc ? "a must be finite and > 0, b finite and > 0 (periodic grid)"
                                           : "a must be finite and > 0, b finite and >= 0"};
  flags_.alloc_async(sizeof(int) * FLAG_COUNT, &F_.mem, st_);
  HIF_CUDA_TRY(cudaMemsetAsync(flags_.as<int>(), 0xff, sizeof(int) * FLAG_COUNT, st_));

  HIF_CUDA_TRY(cudaStreamCreateWithFlags(&up_st_, cudaStreamNonBlocking));
  const int L = F_.L;
  std::shared_ptr<const CellPlan> prevp;
  DevBuf prevK, prevDesc;
  for (int level = 0; level <= L; ++level) {
    level_ = level;
    auto tl = Clock::now();
    std::shared_ptr<const CellPlan> cpp;
    tr_.mark(level, "start");
    std::vector<int64_t> mapOff;
    PlanVec32 map;
    {
      auto built = std::make_shared<CellPlan>();
      if (have_spec_) {
        *built = std::move(spec_cells_);
        mapOff = std::move(spec_mapOff_);
        map = std::move(spec_map_);
        have_spec_ = false;
      } else {
        sym_.build_cells(level, *built);
        if (level > 0) sym_.merge_maps(*prevp, *built, mapOff, map);
      }
      cpp = std::move(built);
    }
    const CellPlan& cp = *cpp;
    tr_.mark(level, "symbolic cells + merge maps");
    // frontal matrices of the level's cells
    std::vector<CellDesc> cdesc(cp.ncell);
    int64_t koff = 0;
    for (int c = 0; c < cp.ncell; ++c) {
      const int nc = (int)(cp.off[c + 1] - cp.off[c]);
      cdesc[c] = CellDesc{koff, cp.off[c], nc, cp.p[c]};
      koff += (int64_t)nc * nc;
    }
    DevBuf Kar, cdesc_d, lists_d;
    Kar.alloc_async(sizeof(T) * std::max<int64_t>(1, koff), &F_.mem, st_);
    upload_async(cdesc_d, cdesc, &F_.mem, st_);
    upload(lists_d, cp.dofs, &F_.mem, st_);
    if (level == 0) {
      HIF_CUDA_TRY(cudaMemsetAsync(Kar.as<T>(), 0, sizeof(T) * koff, st_));
      const int maxbox = (cp.s + 1) * (cp.s + 1) * (cp.s + 1);
      assemble_level0<T>(cdesc_d.as<CellDesc>(), cp.ncell, lists_d.as<int32_t>(), n, cp.s, F_.bc,
                         F_.cpl.template as<double>(), F_.diag.template as<double>(), Kar.as<T>(), maxbox, st_);
    } else {
      DevBuf map_d, mdesc_d;
      upload_async(map_d, map, &F_.mem, st_);
      std::vector<MergeDesc> md(cp.ncell);
      const int C = cp.C, Cc = prevp->C;
      for (int c = 0; c < cp.ncell; ++c) {
        md[c].K = cdesc[c].K;
        md[c].map = mapOff[c];
        md[c].n = cdesc[c].n;
        const int px = c % C, py = (c / C) % C, pz = c / (C * C);
        for (int q = 0; q < 8; ++q) {
          const int cx = 2 * px + (q & 1), cy = 2 * py + ((q >> 1) & 1), cz = 2 * pz + ((q >> 2) & 1);
          md[c].child[q] = (cx < Cc && cy < Cc && cz < Cc) ? cx + Cc * (cy + Cc * cz) : -1;
        }
      }
      upload_async(mdesc_d, md, &F_.mem, st_);
      merge_children<T>(mdesc_d.as<MergeDesc>(), md.data(), cp.ncell, prevDesc.as<CellDesc>(),
                        map_d.as<int32_t>(), prevK.as<T>(), Kar.as<T>(), st_);
      prevK.release();
      prevDesc.release();
    }
    tr_.mark(level, "frontal matrices");
    // after the cell step the interiors are gone; the face and edge plans
    // depend only on that set, so two host threads build them while the
    // cells are eliminated on the GPU (the edge rows are filtered again once
    // the faces have dropped their redundant DOFs)
    std::vector<uint8_t> alive(N, 0);
    for (int32_t g : cp.active) alive[g] = 1;
    for (int c = 0; c < cp.ncell; ++c)
      for (int64_t t = cp.off[c]; t < cp.off[c] + cp.p[c]; ++t) alive[cp.dofs[t]] = 0;
    // the planners read their own copy of `alive` (the face step changes
    // it while the edge plan is still being built); declared before the
    // futures, so it outlives them
    std::vector<uint8_t> alive_plan;
    auto fbuild = std::make_shared<SkelPlan>(), ebuild = std::make_shared<SkelPlan>();
    std::shared_ptr<const SkelPlan> fplan, eplan;
    std::future<void> face_plan, edge_plan;
    if (level < L && F_.eps > 0.0) {
      alive_plan = alive;
      face_plan = std::async(std::launch::async, [&]() { sym_.build_skel(cp, 1, alive_plan, *fbuild); });
      edge_plan = std::async(std::launch::async, [&]() { sym_.build_skel(cp, 2, alive_plan, *ebuild); });
    }
    cell_step(cpp, Kar, cdesc_d, cdesc, lists_d);
    tr_.mark(level, "cell elimination");
    F_.stats.fronts[level][0] = cp.ncell;
    if (level == L) {
      start_stage_jobs();
      F_.stats.root_size = (int)cp.dofs.size();
      check_flags("the root factorization");
      F_.stats.level_seconds[level] = seconds_since(tl);
      break;
    }
    if (F_.eps > 0.0) {
      // the face step starts once its plan is ready; the edge plan goes on
      // meanwhile and is joined after the face step
      face_plan.get();
      fplan = fbuild;
      tr_.mark(level, "face plan joined");
      const int64_t dropped = skel_step(cp, 1, alive, Kar, cdesc_d, fplan);
      tr_.mark(level, "faces");
      edge_plan.get();
      eplan = ebuild;
      start_stage_jobs();
      tr_.mark(level, "edge plan joined");
      if (dropped) {
        auto filtered = std::make_shared<SkelPlan>();
        sym_.filter_rows(*eplan, alive, *filtered);
        eplan = std::move(filtered);
      }
      // the next level's cells, assuming the edges keep every DOF (they
      // usually do), are planned on a host thread while the edges run;
      // rebuilt at the next level if an edge lost DOFs
      std::vector<int32_t> spec_act;
      spec_act.reserve(cp.active.size());
      for (int32_t g : cp.active)
        if (alive[g]) spec_act.push_back(g);
      const std::vector<uint8_t> alive_faces = alive;
      auto spec = std::async(std::launch::async, [&, act = std::move(spec_act)]() {
        sym_.build_cells_from(level + 1, act, spec_cells_);
        sym_.merge_maps(cp, spec_cells_, spec_mapOff_, spec_map_);
      });
      skel_step(cp, 2, alive, Kar, cdesc_d, eplan);
      spec.get();
      have_spec_ = (alive == alive_faces);
      tr_.mark(level, "edges");
    } else {
      start_stage_jobs();
    }
    check_flags("level factorization");
    std::vector<int32_t> next;
    next.reserve(cp.active.size());
    for (int32_t g : cp.active)
      if (alive[g]) next.push_back(g);
    F_.stats.active_after[level] = (int64_t)next.size();
    F_.active.push_back(next);
    sym_.set_active(std::move(next));
    prevp = std::move(cpp);
    prevK = std::move(Kar);
    prevDesc = std::move(cdesc_d);
    F_.stats.level_seconds[level] = seconds_since(tl);
  }
  start_stage_jobs();
  upload_stages(true);
  HIF_CUDA_TRY(cudaStreamSynchronize(up_st_));
  HIF_CUDA_TRY(cudaStreamSynchronize(st_));
  F_.stats.factor_seconds = seconds_since(t0);
}

template <typename T>
void Builder<T>::cell_step(std::shared_ptr<const CellPlan> cpp, DevBuf& Kar, DevBuf& cdesc_d,
                           std::vector<CellDesc>& cdesc, DevBuf& lists_d) {
  (void)cdesc_d;
  const CellPlan& cp = *cpp;
  Stage s;
  s.kind = 0;
  s.level = level_;
  // panels for the cells with an interior, sorted by p (largest first)
  std::vector<int> order;
  for (int c = 0; c < cp.ncell; ++c)
    if (cp.p[c] > 0) order.push_back(c);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cp.p[x] > cp.p[y]; });
  std::vector<DFront> fr;
  std::vector<int64_t> poff(cp.ncell, -1);
  int64_t pcur = 0;
  for (int c : order) {
    poff[c] = pcur;
    fr.push_back(DFront{cdesc[c].K, pcur, cdesc[c].n, cdesc[c].p, c, cdesc[c].n});
    pcur += (int64_t)cdesc[c].n * cdesc[c].p;
    F_.stats.flops += std::pow((double)cdesc[c].p, 3) / 3.0 +
                      (double)cdesc[c].p * cdesc[c].p * (cdesc[c].n - cdesc[c].p) +
                      (double)(cdesc[c].n - cdesc[c].p) * (cdesc[c].n - cdesc[c].p) * cdesc[c].p;
  }
  s.panels.alloc(sizeof(T) * std::max<int64_t>(1, pcur), &F_.mem);
  // zero: the products read L^{-1} as a dense block (zeros above the diagonal)
  HIF_CUDA_TRY(cudaMemsetAsync(s.panels.as<void>(), 0, sizeof(T) * std::max<int64_t>(1, pcur), st_));
  s.entries = pcur;
  DevBuf fr_d;
  upload_async(fr_d, fr, &F_.mem, st_);
  partial_cholesky<T>(fr_d.as<DFront>(), fr.data(), (int)fr.size(), Kar.as<T>(), s.panels.as<T>(),
                      flags_.as<int>(), F_.opt.tensor_cores != 0, st_, &retry_);
  tr_.mark(level_, " cells: partial Cholesky queued");
  // apply stage: gather the whole frontal list of every cell (already on
  // the device); the rest is built on a worker thread
  s.nidx = (int64_t)cp.dofs.size();
  s.idx = std::move(lists_d);
  const size_t si = F_.stages.size();
  F_.stages.push_back(std::move(s));
  const int64_t N = (int64_t)F_.n * F_.n * F_.n;
  const int64_t nidx = (int64_t)cp.dofs.size();
  unstarted_.emplace_back(si, [cpp, cdesc, poff = std::move(poff), N, nidx]() mutable {
    return cell_stage_host(cpp, std::move(cdesc), std::move(poff), N, nidx);
  });
}

template <typename T>
typename Builder<T>::StageHost Builder<T>::cell_stage_host(std::shared_ptr<const CellPlan> cpp,
                                                           std::vector<CellDesc> cdesc,
                                                           std::vector<int64_t> poff, int64_t N,
                                                           int64_t nidx) {
  const CellPlan& cp = *cpp;
  StageHost h;
  for (int c = 0; c < cp.ncell; ++c) {
    const int nc = cdesc[c].n, p = cdesc[c].p;
    if (p == 0) continue;
    const int64_t vo = cp.off[c], to = nidx + cp.off[c], P = poff[c];
    // forward: t_I = Linv v_I ; t_B = X^T t_I
    h.fwd[0].push_back(GemvOp{P, vo, to, p, p, nc, 1, 1.0f, 0});
    if (nc > p) h.fwd[1].push_back(GemvOp{P + p, to, to + p, nc - p, p, nc, 0, 1.0f, 0});
    // backward: v_I -= X v_B ; t_I = Linv^T v_I
    if (nc > p) h.bwd[0].push_back(GemvOp{P + p, vo + p, vo, nc - p, p, nc, 0, -1.0f, 1});
    h.bwd[1].push_back(GemvOp{P, vo, to, p, p, nc, 1, 1.0f, 0});
    for (int a = 0; a < p; ++a) {
      h.set_g.push_back(cp.dofs[cp.off[c] + a]);
      h.set_p.push_back((int32_t)(to + a));
    }
  }
  h.nfwd = h.nbwd = 2;
  h.bwd_trans[0] = h.bwd_trans[1] = 1;
  // deterministic accumulation of the boundary updates: per DOF, contributions
  // in cell order (counting sort on the global index)
  std::vector<int64_t> cnt(N + 1, 0);
  int64_t npair = 0;
  for (int c = 0; c < cp.ncell; ++c) {
    if (cp.p[c] == 0) continue;
    for (int64_t t = cp.off[c] + cp.p[c]; t < cp.off[c + 1]; ++t) {
      cnt[cp.dofs[t] + 1]++;
      ++npair;
    }
  }
  if (npair) {
    for (int64_t g = 0; g < N; ++g)
      if (cnt[g + 1]) h.acc_tgt.push_back((int32_t)g);
    std::vector<int64_t> start(N + 1, 0);
    for (int64_t g = 0; g < N; ++g) start[g + 1] = start[g] + cnt[g + 1];
    h.acc_src.resize(npair);
    std::vector<int64_t> cur(start.begin(), start.end() - 1);
    for (int c = 0; c < cp.ncell; ++c) {
      if (cp.p[c] == 0) continue;
      for (int64_t t = cp.off[c] + cp.p[c]; t < cp.off[c + 1]; ++t)
        h.acc_src[cur[cp.dofs[t]]++] = (int32_t)(nidx + t);
    }
    h.acc_ptr.reserve(h.acc_tgt.size() + 1);
    h.acc_ptr.push_back(0);
    for (int32_t g : h.acc_tgt) h.acc_ptr.push_back(start[g + 1]);
  }
  return h;
}

template <typename T>
void Builder<T>::upload_stages(bool all) {
  for (size_t jj = 0; jj < jobs_.size();) {
    auto& job = jobs_[jj];
    if (!all && job.second.wait_for(std::chrono::seconds(0)) != std::future_status::ready) {
      ++jj;
      continue;
    }
    StageHost h = job.second.get();
    Stage& s = F_.stages[job.first];
    if (!h.idx.empty()) upload(s.idx, h.idx, &F_.mem, up_st_);
    s.fwd.resize(h.nfwd);
    s.bwd.resize(h.nbwd);
    for (int i = 0; i < h.nfwd; ++i) {
      s.fwd[i].h = std::move(h.fwd[i]);
      s.fwd[i].trans = h.fwd_trans[i];
      s.fwd[i].mat = h.fwd_mat[i];
      upload(s.fwd[i].d, s.fwd[i].h, &F_.mem, up_st_);
    }
    for (int i = 0; i < h.nbwd; ++i) {
      s.bwd[i].h = std::move(h.bwd[i]);
      s.bwd[i].trans = h.bwd_trans[i];
      s.bwd[i].mat = h.bwd_mat[i];
      upload(s.bwd[i].d, s.bwd[i].h, &F_.mem, up_st_);
    }
    s.nset = (int64_t)h.set_g.size();
    upload(s.set_g, h.set_g, &F_.mem, up_st_);
    upload(s.set_p, h.set_p, &F_.mem, up_st_);
    s.nacc = (int64_t)h.acc_tgt.size();
    if (s.nacc) {
      upload(s.acc_tgt, h.acc_tgt, &F_.mem, up_st_);
      upload(s.acc_ptr, h.acc_ptr, &F_.mem, up_st_);
      upload(s.acc_src, h.acc_src, &F_.mem, up_st_);
    }
    s.entries += h.entries_add;
    F_.work_stride = std::max(F_.work_stride, 2 * s.nidx);
    jobs_.erase(jobs_.begin() + (std::ptrdiff_t)jj);
  }
}

template <typename T>
int64_t Builder<T>::skel_step(const CellPlan& cp, int kind, std::vector<uint8_t>& alive,
                              DevBuf& Kar, DevBuf& cdesc_d, std::shared_ptr<const SkelPlan> plan) {
  const SkelPlan& sp = *plan;
  tr_.mark(level_, kind == 1 ? " symbolic faces" : " symbolic edges");
  const int nf = sp.nfront;
  if (nf == 0) return 0;
  const int ncp = sp.ncellPer;
  std::vector<SkelDesc> sd(nf);
  int64_t goff = 0, poff = 0, toff = 0;
  for (int f = 0; f < nf; ++f) {
    SkelDesc& d = sd[f];
    std::memset(&d, 0, sizeof(d));
    d.nF = sp.nF[f];
    d.nR = sp.nR[f];
    d.G = goff;
    d.idoff = goff + sp.nF[f];
    d.idm = sp.nR[f];
    d.idld = sp.nF[f] + sp.nR[f];
    d.rows = sp.rowOff[f] * ncp;
    d.perm = poff;
    d.Tm = toff;
    for (int i = 0; i < ncp; ++i) d.cell[i] = sp.cells[(size_t)f * ncp + i];
    goff += (int64_t)(d.nF + d.nR) * d.nF;
    poff += d.nF;
    toff += (int64_t)(d.nF / 2) * (d.nF - d.nF / 2);
    F_.stats.flops += 2.0 * d.nR * (double)d.nF * d.nF;
  }
  DevBuf rowpos_d, sd_d, G, perm_d, steps, tm;
  upload_async(rowpos_d, sp.rowPos, &F_.mem, st_);
  upload_async(sd_d, sd, &F_.mem, st_);
  G.alloc_async(sizeof(T) * std::max<int64_t>(1, goff), &F_.mem, st_);
  perm_d.alloc_async(sizeof(int32_t) * poff, &F_.mem, st_);
  steps.alloc_async(sizeof(int32_t) * poff, &F_.mem, st_);
  tm.alloc(sizeof(T) * std::max<int64_t>(1, toff), &F_.mem);
  skel_gather<T>(sd_d.as<SkelDesc>(), sd.data(), nf, ncp, rowpos_d.as<int32_t>(),
                 cdesc_d.as<CellDesc>(), Kar.as<T>(), G.as<T>(), st_);
  // fronts with many more coupled rows than DOFs: reduce the rows by an
  // unpivoted QR first; their ID then runs on the square triangular factor
  std::vector<int> sel[2];   // 0: ID on the gathered rows, 1: ID on R
  for (int f = 0; f < nf; ++f)
    sel[(sd[f].nR > 2 * sd[f].nF && sd[f].nF >= 96) ? 1 : 0].push_back(f);
  DevBuf Rbuf;
  if (!sel[1].empty()) {
    std::vector<int64_t> roff(sel[1].size());
    int64_t rtot = 0;
    for (size_t i = 0; i < sel[1].size(); ++i) {
      roff[i] = rtot;
      rtot += (int64_t)sd[sel[1][i]].nF * sd[sel[1][i]].nF;
    }
    Rbuf.alloc_async(sizeof(T) * rtot, &F_.mem, st_);
    reduce_rows_qr<T>(sd.data(), sel[1], G.as<T>(), Rbuf.as<T>(), roff, flags_.as<int>(),
                      F_.opt.tensor_cores != 0, st_);
    for (size_t i = 0; i < sel[1].size(); ++i) {
      SkelDesc& d = sd[sel[1][i]];
      d.idoff = roff[i];
      d.idm = d.nF;
      d.idld = d.nF;
    }
  }
  if (tr_.on) {
    for (int g = 0; g < 2; ++g) {
      if (sel[g].empty()) continue;
      int64_t mxF = 0, mxM = 0, sF = 0, sM = 0;
      for (int f : sel[g]) {
        mxF = std::max<int64_t>(mxF, sd[f].nF);
        mxM = std::max<int64_t>(mxM, sd[f].idm);
        sF += sd[f].nF;
        sM += sd[f].idm;
      }
      std::fprintf(stderr, "[hif] level %d %s ID%s: %zu fronts, nF max %lld mean %.1f, rows max %lld mean %.1f\n",
                   level_, kind == 1 ? "faces" : "edges", g ? " on R" : "", sel[g].size(),
                   (long long)mxF, (double)sF / sel[g].size(), (long long)mxM,
                   (double)sM / sel[g].size());
    }
  }
  tr_.mark(level_, " gather + row reduction queued");
  std::vector<SkelDesc> sub[2];
  std::vector<int8_t> route[2];
  DevBuf sub_d[2];
  for (int g = 0; g < 2; ++g) {
    if (sel[g].empty()) continue;
    for (int f : sel[g]) sub[g].push_back(sd[f]);
    route[g].assign(sel[g].size(), ID_ROUTE_STREAM);
    upload_async(sub_d[g], sub[g], &F_.mem, st_);
    interpolative_decomposition<T>(sub_d[g].as<SkelDesc>(), sub[g].data(), (int)sub[g].size(),
                                   g == 0 ? G.as<T>() : Rbuf.as<T>(),
                                   (g == 0 ? G.bytes() : Rbuf.bytes()) / sizeof(T),
                                   perm_d.as<int32_t>(), tm.as<T>(), steps.as<int32_t>(), F_.eps,
                                   st_, route[g].data());
    HIF_CUDA_TRY(cudaMemcpyAsync(sub[g].data(), sub_d[g].as<void>(),
                                 sizeof(SkelDesc) * sub[g].size(), cudaMemcpyDeviceToHost, st_));
  }
  std::vector<int32_t> perm(poff);
  HIF_CUDA_TRY(cudaMemcpyAsync(perm.data(), perm_d.as<void>(), sizeof(int32_t) * poff,
                               cudaMemcpyDeviceToHost, st_));
  upload_stages(false);   // while the GPU runs the ID
  HIF_CUDA_TRY(cudaStreamSynchronize(st_));
  for (int g = 0; g < 2; ++g)
    for (size_t i = 0; i < sel[g].size(); ++i) sd[sel[g][i]].k = sub[g][i].k;
  tr_.mark(level_, " gather + ID");
  // T = R11^{-1} R12 of the fronts the cluster kernels took (the shared-memory
  // kernel forms its own)
  for (int g = 0; g < 2; ++g) {
    std::vector<int> need;
    for (size_t i = 0; i < sel[g].size(); ++i)
      if (route[g][i] != ID_ROUTE_SMEM && sub[g][i].k > 0 && sub[g][i].k < sub[g][i].nF)
        need.push_back((int)i);
    id_solve_t<T>(sub_d[g].as<SkelDesc>(), sub[g].data(), need, g == 0 ? G.as<T>() : Rbuf.as<T>(),
                  perm_d.as<int32_t>(), tm.as<T>(), st_);
  }
  if (tr_.on) {
    int64_t kmx = 0, ks = 0, fs = 0;
    for (int f = 0; f < nf; ++f) {
      kmx = std::max<int64_t>(kmx, sd[f].k);
      ks += sd[f].k;
      fs += sd[f].nF;
    }
    std::fprintf(stderr, "[hif] level %d %s ranks: max %lld mean %.1f (%.1f%% of the DOFs kept)\n",
                 level_, kind == 1 ? "faces" : "edges", (long long)kmx, (double)ks / nf,
                 100.0 * (double)ks / std::max<int64_t>(1, fs));
  }
  steps.release();
  Rbuf.release();
  if (prof_enabled()) {
    // algorithmic counts of the ID (§2.3): Householder pivoted QR, 4 flops
    // per entry of the trailing (idm - i) x (nF - i - 1) block at each of
    // the k steps; in the shared-memory kernel also T = R11^{-1} R12
    // (k^2 (nF - k) flops; id_solve_t counts it for the others); bytes: the
    // matrix read once, T (or R) and the pivots written once
    double fl[3] = {0.0, 0.0, 0.0}, by[3] = {0.0, 0.0, 0.0};
    for (int g = 0; g < 2; ++g)
      for (size_t j = 0; j < sel[g].size(); ++j) {
        const int f = sel[g][j], sm = route[g][j];
        const double k = sd[f].k, nF = sd[f].nF;
        for (int i = 0; i < sd[f].k; ++i)
          fl[sm] += 4.0 * (double)(sd[f].idm - i) * (sd[f].nF - i - 1);
        if (sm == ID_ROUTE_SMEM) {
          fl[sm] += k * k * (nF - k);
          by[sm] += sizeof(T) * ((double)sd[f].idm * nF + k * (nF - k)) + 4.0 * nF;
        } else {   // the matrix read once, R (k rows) written back, pivots written
          by[sm] += sizeof(T) * ((double)sd[f].idm * nF + (sm == ID_ROUTE_CLUSTER_SMEM ? k * nF : 0.0)) + 4.0 * nF;
        }
      }
    prof_add("id_cpqr", fl[ID_ROUTE_STREAM], by[ID_ROUTE_STREAM]);
    prof_add("id_cpqr_smem", fl[ID_ROUTE_SMEM], by[ID_ROUTE_SMEM]);
    prof_add("id_cpqr_dsm", fl[ID_ROUTE_CLUSTER_SMEM], by[ID_ROUTE_CLUSTER_SMEM]);
  }
  // fronts with redundant DOFs are eliminated; the others keep every DOF
  std::vector<int> act;
  for (int f = 0; f < nf; ++f)
    if (sd[f].k < sd[f].nF) act.push_back(f);
  F_.stats.fronts[level_][kind] = (int64_t)act.size();
  int64_t dropped = 0;
  for (int f : act) {
    const int32_t* pm = &perm[sd[f].perm];
    for (int i = sd[f].k; i < sd[f].nF; ++i) alive[sp.rowDof[sp.rowOff[f] + pm[i]]] = 0;
    dropped += sd[f].nF - sd[f].k;
  }
  if (act.empty()) return 0;
  // frontal matrices Z = Q^T A_FF Q in (redundant, skeleton) order
  int64_t zoff = 0, pnl = 0;
  std::vector<DFront> fr;
  for (int f : act) {
    SkelDesc& d = sd[f];
    d.Z = zoff;
    d.P = pnl;
    const int p = d.nF - d.k;
    fr.push_back(DFront{d.Z, d.P, d.nF, p, f, d.nF});
    zoff += (int64_t)d.nF * d.nF;
    pnl += (int64_t)d.nF * p;
    F_.stats.flops += 4.0 * d.nF * (double)d.k * p + std::pow((double)p, 3) / 3.0 +
                      (double)p * p * d.k + (double)d.k * d.k * p;
  }
  upload_async(sd_d, sd, &F_.mem, st_);
  DevBuf Z;
  Z.alloc_async(sizeof(T) * std::max<int64_t>(1, zoff), &F_.mem, st_);
  // permute only the active fronts: build a compact descriptor list
  std::vector<SkelDesc> sda;
  for (int f : act) sda.push_back(sd[f]);
  DevBuf sda_d;
  upload_async(sda_d, sda, &F_.mem, st_);
  skel_permute<T>(sda_d.as<SkelDesc>(), sda.data(), (int)sda.size(), perm_d.as<int32_t>(),
                  G.as<T>(), Z.as<T>(), st_);
  // B_{F^F~} = A_{F^F~} - A_{F^F^} T ;  B_{F~F~} = A_{F~F~} - A_{F~F^} T - T^T B_{F^F~}
  std::vector<GemmOp> g1, g2, g3;
  for (const SkelDesc& d : sda) {
    const int k = d.k, p = d.nF - k, nF = d.nF;
    if (k == 0) continue;
    g1.push_back(GemmOp{d.Z + p + (int64_t)p * nF, d.Tm, d.Z + p, k, p, k, nF, k, nF, 0, 0, -1.f, 1.f, 0, 0});
    g2.push_back(GemmOp{d.Z + (int64_t)p * nF, d.Tm, d.Z, p, p, k, nF, k, nF, 0, 0, -1.f, 1.f, 0, 0});
    g3.push_back(GemmOp{d.Tm, d.Z + p, d.Z, p, p, k, k, nF, nF, 1, 0, -1.f, 1.f, 0, 0});
  }
  DevBuf g1d, g2d, g3d;
  upload_async(g1d, g1, &F_.mem, st_);
  upload_async(g2d, g2, &F_.mem, st_);
  upload_async(g3d, g3, &F_.mem, st_);
  gemm_batched<T>(g1d.as<GemmOp>(), g1.data(), (int)g1.size(), Z.as<T>(), tm.as<T>(), Z.as<T>(), st_,
                  "skel_z_products");
  gemm_batched<T>(g2d.as<GemmOp>(), g2.data(), (int)g2.size(), Z.as<T>(), tm.as<T>(), Z.as<T>(), st_,
                  "skel_z_products");
  gemm_batched<T>(g3d.as<GemmOp>(), g3.data(), (int)g3.size(), tm.as<T>(), Z.as<T>(), Z.as<T>(), st_,
                  "skel_z_products");
  // partial Cholesky of Z: eliminate the redundant DOFs
  Stage s;
  s.kind = 1;
  s.level = level_;
  s.panels.alloc(sizeof(T) * std::max<int64_t>(1, pnl), &F_.mem);
  HIF_CUDA_TRY(cudaMemsetAsync(s.panels.as<void>(), 0, sizeof(T) * std::max<int64_t>(1, pnl), st_));
  std::vector<DFront> frs = fr;
  std::stable_sort(frs.begin(), frs.end(), [](const DFront& x, const DFront& y) { return x.p > y.p; });
  DevBuf fr_d;
  upload_async(fr_d, frs, &F_.mem, st_);
  partial_cholesky<T>(fr_d.as<DFront>(), frs.data(), (int)frs.size(), Z.as<T>(), s.panels.as<T>(),
                      flags_.as<int>(), F_.opt.tensor_cores != 0, st_, &retry_);
  tr_.mark(level_, " Z products + Cholesky queued");
  skel_writeback<T>(sda_d.as<SkelDesc>(), sda.data(), (int)sda.size(), ncp, rowpos_d.as<int32_t>(),
                    perm_d.as<int32_t>(), cdesc_d.as<CellDesc>(), Z.as<T>(), Kar.as<T>(), st_);
  // apply stage: the lists are built on a worker thread
  int64_t totalF = 0;
  for (const SkelDesc& d : sda) totalF += d.nF;
  s.nidx = totalF;
  s.tmats = std::move(tm);
  const size_t si = F_.stages.size();
  F_.stages.push_back(std::move(s));
  auto job = [sda, perm = std::move(perm), act, plan, totalF]() {
    const auto& rowDof = plan->rowDof;
    const auto& rowOff = plan->rowOff;
    StageHost h;
    int64_t vo = 0;
    for (const SkelDesc& d : sda) {
      const int k = d.k, nF = d.nF, p = nF - k;
      const int32_t* pm = &perm[d.perm];
      const int src = act[&d - sda.data()];
      const int64_t base = (int64_t)h.idx.size();
      for (int i = 0; i < p; ++i) h.idx.push_back(rowDof[rowOff[src] + pm[k + i]]);
      for (int i = 0; i < k; ++i) h.idx.push_back(rowDof[rowOff[src] + pm[i]]);
      const int64_t to = totalF + vo;
      // forward: v_c -= T^T v_h ; t_c = Linv v_c ; v_h -= X^T t_c
      if (k) h.fwd[0].push_back(GemvOp{d.Tm, vo + p, vo, k, p, k, 0, -1.0f, 1});
      h.fwd[1].push_back(GemvOp{d.P, vo, to, p, p, nF, 1, 1.0f, 0});
      if (k) h.fwd[2].push_back(GemvOp{d.P + p, to, vo + p, k, p, nF, 0, -1.0f, 1});
      // backward: v_c -= X v_h ; t_c = Linv^T v_c ; v_h -= T t_c
      if (k) h.bwd[0].push_back(GemvOp{d.P + p, vo + p, vo, k, p, nF, 0, -1.0f, 1});
      h.bwd[1].push_back(GemvOp{d.P, vo, to, p, p, nF, 1, 1.0f, 0});
      if (k) h.bwd[2].push_back(GemvOp{d.Tm, to, vo + p, k, p, k, 0, -1.0f, 1});
      for (int i = 0; i < p; ++i) {
        h.set_g.push_back(h.idx[base + i]);
        h.set_p.push_back((int32_t)(to + i));
      }
      for (int i = 0; i < k; ++i) {
        h.set_g.push_back(h.idx[base + p + i]);
        h.set_p.push_back((int32_t)(vo + p + i));
      }
      h.entries_add += (int64_t)nF * p + (int64_t)k * p;
      vo += nF;
    }
    h.nfwd = h.nbwd = 3;
    h.fwd_trans[0] = 1;
    h.fwd_mat[0] = 1;
    h.bwd_trans[0] = h.bwd_trans[1] = 1;
    h.bwd_mat[2] = 1;
    return h;
  };
  jobs_.emplace_back(si, std::async(std::launch::async, std::move(job)));
  return dropped;
}

// ---- PCG ------------------------------------------------------------------------

struct SolveBufs {
  DevBuf r, z, p, q, rold, part, dots, scal;
};

// One factor's system in a PCG run: its right-hand sides f (nrhs columns),
// solution u, work vectors and the per-column state of the iteration.
struct PcgItem {
  FactorBase* F = nullptr;
  const double* f = nullptr;
  double* u = nullptr;
  int nrhs = 0;
  SolveBufs b;
  std::vector<double> fn, rz, tmp, tmp2, al, be, rel;
  std::vector<int> it, done;
  bool all = false;
};

// z = F^{-1} r for the listed items (their b.r into b.z).
using PcgApply = std::function<void(const std::vector<PcgItem*>&, cudaStream_t)>;

// Preconditioned conjugate gradients for several systems in lockstep
// (Polak-Ribiere beta; FP64 residual with the seven-point operator).  Every
// item runs exactly the kernels and the scalar arithmetic it would run alone:
// the items only share the host waits and, through `apply`, the launches of
// the preconditioner.  An item stops when all its columns reached its
// pcg_tol or after its max_iter iterations.  Returns HIF_OK if every column
// converged.
hif_status pcg_many(std::vector<PcgItem>& items, cudaStream_t st, const PcgApply& apply) {
  for (PcgItem& I : items) {
    const int64_t N = (int64_t)I.F->n * I.F->n * I.F->n;
    MemStats* ms = &I.F->mem;
    for (DevBuf* x : {&I.b.r, &I.b.z, &I.b.p, &I.b.q, &I.b.rold}) x->alloc(sizeof(double) * N * I.nrhs, ms);
    I.b.part.alloc(sizeof(double) * 1024 * I.nrhs, ms);
    I.b.dots.alloc(sizeof(double) * 2 * I.nrhs, ms);
    I.b.scal.alloc(sizeof(double) * I.nrhs, ms);
    for (auto* v : {&I.fn, &I.rz, &I.tmp, &I.tmp2, &I.al, &I.be, &I.rel}) v->assign(I.nrhs, 0.0);
    I.it.assign(I.nrhs, 0);
    I.done.assign(I.nrhs, 0);
  }
  auto N_of = [](const PcgItem& I) { return (int64_t)I.F->n * I.F->n * I.F->n; };
  // out[c] = x_c . y_c for each column (queued; read after the next wait)
  auto qdots = [&](PcgItem& I, const double* x, const double* y, std::vector<double>& out) {
    dots(x, y, N_of(I), I.nrhs, I.b.part.as<double>(), I.b.dots.as<double>(), st);
    HIF_CUDA_TRY(cudaMemcpyAsync(out.data(), I.b.dots.as<double>(), sizeof(double) * I.nrhs,
                                 cudaMemcpyDeviceToHost, st));
  };
  auto wait = [&]() { HIF_CUDA_TRY(cudaStreamSynchronize(st)); };
  auto put = [&](PcgItem& I, const std::vector<double>& v) {
    HIF_CUDA_TRY(cudaMemcpyAsync(I.b.scal.as<double>(), v.data(), sizeof(double) * I.nrhs,
                                 cudaMemcpyHostToDevice, st));
  };
  auto all_of = [](const std::vector<int>& d) {
    return std::all_of(d.begin(), d.end(), [](int x) { return x; });
  };
  for (PcgItem& I : items) {
    const int64_t N = N_of(I);
    HIF_CUDA_TRY(cudaMemsetAsync(I.u, 0, sizeof(double) * N * I.nrhs, st));
    HIF_CUDA_TRY(cudaMemcpyAsync(I.b.r.as<double>(), I.f, sizeof(double) * N * I.nrhs,
                                 cudaMemcpyDeviceToDevice, st));
    qdots(I, I.b.r.as<double>(), I.b.r.as<double>(), I.fn);
  }
  wait();
  std::vector<PcgItem*> act;
  for (PcgItem& I : items) {
    for (int c = 0; c < I.nrhs; ++c) {
      I.fn[c] = std::sqrt(I.fn[c]);
      I.rel[c] = I.fn[c] > 0 ? 1.0 : 0.0;
      if (I.fn[c] == 0) I.done[c] = 1;
    }
    act.push_back(&I);
  }
  apply(act, st);
  for (PcgItem& I : items) {
    HIF_CUDA_TRY(cudaMemcpyAsync(I.b.p.as<double>(), I.b.z.as<double>(),
                                 sizeof(double) * N_of(I) * I.nrhs, cudaMemcpyDeviceToDevice, st));
    qdots(I, I.b.r.as<double>(), I.b.z.as<double>(), I.rz);
  }
  wait();
  for (PcgItem& I : items) I.all = all_of(I.done);
  for (int k = 1;; ++k) {
    // the items still iterating at this step
    act.clear();
    for (PcgItem& I : items)
      if (!I.all && k <= I.F->opt.max_iter) act.push_back(&I);
    if (act.empty()) break;
    for (PcgItem* I : act) {
      matvec(I->F->cpl.as<double>(), I->F->diag.as<double>(), I->F->n, I->F->bc,
             I->b.p.as<double>(), I->b.q.as<double>(), I->nrhs, st);
      qdots(*I, I->b.p.as<double>(), I->b.q.as<double>(), I->tmp);
    }
    wait();
    for (PcgItem* I : act) {
      const int64_t N = N_of(*I);
      for (int c = 0; c < I->nrhs; ++c)
        I->al[c] = I->done[c] || I->tmp[c] == 0 ? 0.0 : I->rz[c] / I->tmp[c];
      put(*I, I->al);
      double* r = I->b.r.as<double>();
      axpy_cols(I->b.scal.as<double>(), 1.0, I->b.p.as<double>(), I->u, N, I->nrhs, st);
      HIF_CUDA_TRY(cudaMemcpyAsync(I->b.rold.as<double>(), r, sizeof(double) * N * I->nrhs,
                                   cudaMemcpyDeviceToDevice, st));
      axpy_cols(I->b.scal.as<double>(), -1.0, I->b.q.as<double>(), r, N, I->nrhs, st);
      qdots(*I, r, r, I->tmp);
    }
    wait();
    std::vector<PcgItem*> next;
    for (PcgItem* I : act) {
      for (int c = 0; c < I->nrhs; ++c) {
        if (I->done[c]) continue;
        I->rel[c] = std::sqrt(I->tmp[c]) / I->fn[c];
        I->it[c] = k;
        if (I->rel[c] <= I->F->opt.pcg_tol) I->done[c] = 1;
      }
      I->all = all_of(I->done);
      if (!I->all) next.push_back(I);
    }
    if (next.empty()) continue;
    apply(next, st);
    for (PcgItem* I : next) {
      qdots(*I, I->b.r.as<double>(), I->b.z.as<double>(), I->tmp);       // r_new . z
      qdots(*I, I->b.rold.as<double>(), I->b.z.as<double>(), I->tmp2);   // r_old . z
    }
    wait();
    for (PcgItem* I : next) {
      const int64_t N = N_of(*I);
      for (int c = 0; c < I->nrhs; ++c) {
        I->be[c] = I->done[c] || I->rz[c] == 0 ? 0.0 : (I->tmp[c] - I->tmp2[c]) / I->rz[c];   // Polak-Ribiere
        if (!I->done[c]) I->rz[c] = I->tmp[c];
      }
      put(*I, I->be);
      double* pp = I->b.p.as<double>();
      xpby_cols(I->b.z.as<double>(), I->b.scal.as<double>(), pp, N, I->nrhs, st);
      // converged columns keep p = 0 so that later updates leave them alone
      for (int c = 0; c < I->nrhs; ++c)
        if (I->done[c]) HIF_CUDA_TRY(cudaMemsetAsync(pp + c * N, 0, sizeof(double) * N, st));
    }
  }
  wait();
  bool ok = true;
  for (PcgItem& I : items) ok = ok && I.all;
  return ok ? HIF_OK : HIF_ERR_NO_CONVERGENCE;
}

hif_status do_solve(FactorBase& F, const double* f, double* u, int nrhs, cudaStream_t st,
                    int* iters, double* relres) {
  std::vector<PcgItem> items(1);
  items[0].F = &F;
  items[0].f = f;
  items[0].u = u;
  items[0].nrhs = nrhs;
  const hif_status s = pcg_many(items, st, [](const std::vector<PcgItem*>& v, cudaStream_t s2) {
    for (PcgItem* I : v) I->F->apply(I->b.r.as<double>(), I->b.z.as<double>(), I->nrhs, s2);
  });
  for (int c = 0; c < nrhs; ++c) {
    if (iters) iters[c] = items[0].it[c];
    if (relres) relres[c] = items[0].rel[c];
  }
  return s;
}

}  // namespace
}  // namespace hif

// ---- C ABI ------------------------------------------------------------------------

struct hif_handle_s {
  std::unique_ptr<hif::FactorBase> f;
};

using hif::Error;

#define HIF_API_BEGIN try {
#define HIF_API_END                                                  \
  }                                                                  \
  catch (const Error& e) {                                           \
    hif::set_last_error(e.msg);                                      \
    return e.code;                                                   \
  }                                                                  \
  catch (const std::bad_alloc&) {                                    \
    hif::set_last_error("host allocation failed");                   \
    return HIF_ERR_OOM;                                              \
  }                                                                  \
  catch (const std::exception& e) {                                  \
    hif::set_last_error(e.what());                                   \
    return HIF_ERR_CUDA;                                             \
  }

namespace {

// Input array: device pointer as given, or a device copy of host data.
struct InArray {
  const double* p = nullptr;
  hif::DevBuf tmp;
  void set(const double* src, int64_t cnt, cudaStream_t st) {
    if (src == nullptr || hif::is_device_ptr(src)) {
      p = src;
      return;
    }
    tmp.alloc(sizeof(double) * cnt, nullptr);
    HIF_CUDA_TRY(cudaMemcpyAsync(tmp.as<void>(), src, sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
    p = tmp.as<double>();
  }
};

struct OutArray {
  double* user = nullptr;
  double* p = nullptr;
  hif::DevBuf tmp;
  int64_t cnt = 0;
  void set(double* dst, int64_t c) {
    user = dst;
    cnt = c;
    if (hif::is_device_ptr(dst)) {
      p = dst;
    } else {
      tmp.alloc(sizeof(double) * c, nullptr);
      p = tmp.as<double>();
    }
  }
  void finish(cudaStream_t st) {
    if (p != user) {
      HIF_CUDA_TRY(cudaMemcpyAsync(user, p, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
      HIF_CUDA_TRY(cudaStreamSynchronize(st));
    }
  }
};

}  // namespace

namespace {

// Work space of hif_apply_noalloc: one fixed array in device memory, present
// on every GPU that loads the library, shared by all calls.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code the
// array's name only stands for it; the address is asked from the runtime once
// per device, with that device current.
void* noalloc_scratch_address() {
  int dev = 0;
  HIF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw Error{HIF_ERR_INVALID_ARG, "device index out of range"};
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    HIF_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = p;
  }
  return g_noalloc_addr[dev];
}

}  // namespace

namespace hif {
namespace {

// ---- factor files: a versioned binary image of a handle ------------------------
// Layout: "HIFF", format version, sizes of the option/stats structs (a file
// is read only by the build that wrote it), the scalars of the factor, the
// operator, then every stage: its scalars, its device arrays (byte count +
// bytes) and its mat-vec lists (count + descriptors).
constexpr uint32_t kFileVersion = 2;

struct FileOut {
  std::FILE* f = nullptr;
  explicit FileOut(const char* path) : f(std::fopen(path, "wb")) {
    if (!f) throw Error{HIF_ERR_INVALID_ARG, std::string("cannot open ") + path + " for writing"};
  }
  ~FileOut() { if (f) std::fclose(f); }
  void raw(const void* p, size_t n) {
    if (n && std::fwrite(p, 1, n, f) != n) throw Error{HIF_ERR_INVALID_ARG, "write failed"};
  }
  template <typename U> void put(const U& v) { raw(&v, sizeof(U)); }
  void buf(const DevBuf& b) {
    const uint64_t n = b.bytes();
    put(n);
    if (!n) return;
    std::vector<unsigned char> h(n);
    HIF_CUDA_TRY(cudaMemcpy(h.data(), b.as<void>(), n, cudaMemcpyDeviceToHost));
    raw(h.data(), n);
  }
  void list(const GemvList& gl) {
    put(gl.trans);
    put(gl.mat);
    const uint64_t c = gl.h.size();
    put(c);
    raw(gl.h.data(), sizeof(GemvOp) * c);
  }
};

struct FileIn {
  std::FILE* f = nullptr;
  explicit FileIn(const char* path) : f(std::fopen(path, "rb")) {
    if (!f) throw Error{HIF_ERR_INVALID_ARG, std::string("cannot open ") + path};
  }
  ~FileIn() { if (f) std::fclose(f); }
  void raw(void* p, size_t n) {
    if (n && std::fread(p, 1, n, f) != n) throw Error{HIF_ERR_INVALID_ARG, "truncated factor file"};
  }
  template <typename U> U get() {
    U v;
    raw(&v, sizeof(U));
    return v;
  }
  // a device array; with `keep`, its bytes also stay on the host (for the
  // consistency checks of load_factor)
  void buf(DevBuf& b, MemStats* ms, std::vector<unsigned char>* keep = nullptr) {
    const uint64_t n = get<uint64_t>();
    if (n > (uint64_t(1) << 40)) throw Error{HIF_ERR_INVALID_ARG, "corrupt factor file"};
    b.alloc(n, ms);
    std::vector<unsigned char> local;
    std::vector<unsigned char>& h = keep ? *keep : local;
    h.assign(n, 0);
    if (!n) return;
    raw(h.data(), n);
    HIF_CUDA_TRY(cudaMemcpy(b.as<void>(), h.data(), n, cudaMemcpyHostToDevice));
  }
  void list(GemvList& gl, MemStats* ms) {
    gl.trans = get<int>();
    gl.mat = get<int>();
    const uint64_t c = get<uint64_t>();
    if (c > (uint64_t(1) << 32)) throw Error{HIF_ERR_INVALID_ARG, "corrupt factor file"};
    gl.h.resize(c);
    raw(gl.h.data(), sizeof(GemvOp) * c);
    gl.d.alloc(sizeof(GemvOp) * c, ms);
    if (c)
      HIF_CUDA_TRY(cudaMemcpy(gl.d.as<void>(), gl.h.data(), sizeof(GemvOp) * c,
                              cudaMemcpyHostToDevice));
  }
};

template <typename T>
void save_factor(const Factor<T>& F, FileOut& o) {
  o.put(F.n);
  o.put(F.m);
  o.put(F.L);
  o.put(F.precision);
  o.put(F.eps);
  o.put(F.bc);
  o.put(F.opt);
  o.put(F.stats);
  o.put(F.work_stride);
  o.buf(F.cpl);
  o.buf(F.diag);
  const uint64_t ns = F.stages.size();
  o.put(ns);
  for (const Stage& s : F.stages) {
    o.put(s.kind);
    o.put(s.level);
    o.put(s.nidx);
    o.put(s.nset);
    o.put(s.nacc);
    o.put(s.entries);
    o.buf(s.idx);
    o.buf(s.panels);
    o.buf(s.tmats);
    o.buf(s.set_g);
    o.buf(s.set_p);
    o.buf(s.acc_tgt);
    o.buf(s.acc_ptr);
    o.buf(s.acc_src);
    o.put((uint32_t)s.fwd.size());
    for (const auto& gl : s.fwd) o.list(gl);
    o.put((uint32_t)s.bwd.size());
    for (const auto& gl : s.bwd) o.list(gl);
  }
  o.put((uint64_t)F.active.size());
  for (const auto& a : F.active) {
    o.put((uint64_t)a.size());
    o.raw(a.data(), sizeof(int32_t) * a.size());
  }
}

[[noreturn]] void corrupt(const char* what) {
  throw Error{HIF_ERR_INVALID_ARG, std::string("corrupt factor file: ") + what};
}

// The host bytes of an int array read from a factor file, as values.
template <typename I>
std::vector<I> as_values(const std::vector<unsigned char>& b, int64_t count, const char* what) {
  if ((int64_t)b.size() != count * (int64_t)sizeof(I)) corrupt(what);
  std::vector<I> v((size_t)count);
  if (count) std::memcpy(v.data(), b.data(), b.size());
  return v;
}

// Every index and mat-vec extent of a loaded stage must stay inside the
// arrays the apply sweeps give it: the gather list and set / accumulate
// targets inside the grid (N), their work positions inside the stage's two
// work vectors (2 nidx), and every matrix inside its arena.
template <typename T>
void check_stage(const Stage& s, int64_t N, const std::vector<unsigned char>& idx_b,
                 const std::vector<unsigned char>& setg_b, const std::vector<unsigned char>& setp_b,
                 const std::vector<unsigned char>& tgt_b, const std::vector<unsigned char>& ptr_b,
                 const std::vector<unsigned char>& src_b) {
  if (s.nidx < 0 || s.nidx > (int64_t(1) << 30) || s.nset < 0 || s.nacc < 0)
    corrupt("stage counts");
  const int64_t W = 2 * s.nidx;   // work entries of the stage, per right-hand side
  for (int32_t g : as_values<int32_t>(idx_b, s.nidx, "gather list"))
    if (g < 0 || g >= N) corrupt("gather index");
  const auto sg = as_values<int32_t>(setg_b, s.nset, "set list");
  const auto sp = as_values<int32_t>(setp_b, s.nset, "set positions");
  for (int64_t i = 0; i < s.nset; ++i)
    if (sg[i] < 0 || sg[i] >= N || sp[i] < 0 || sp[i] >= W) corrupt("set entry");
  if (s.nacc) {
    const auto tg = as_values<int32_t>(tgt_b, s.nacc, "accumulate targets");
    const auto pt = as_values<int64_t>(ptr_b, s.nacc + 1, "accumulate pointers");
    const int64_t nsrc = (int64_t)(src_b.size() / sizeof(int32_t));
    const auto sr = as_values<int32_t>(src_b, nsrc, "accumulate sources");
    if (pt[0] != 0 || pt[s.nacc] != nsrc) corrupt("accumulate pointers");
    for (int64_t t = 0; t < s.nacc; ++t) {
      if (tg[t] < 0 || tg[t] >= N || pt[t + 1] < pt[t]) corrupt("accumulate entry");
    }
    for (int32_t q : sr)
      if (q < 0 || q >= W) corrupt("accumulate source");
  } else if (!tgt_b.empty() || !ptr_b.empty() || !src_b.empty()) {
    corrupt("accumulate lists");
  }
  const int64_t npan = (int64_t)(s.panels.bytes() / sizeof(T));
  const int64_t ntm = (int64_t)(s.tmats.bytes() / sizeof(T));
  auto lists_ok = [&](const std::vector<GemvList>& lists) {
    for (const GemvList& gl : lists) {
      if ((gl.trans != 0 && gl.trans != 1) || (gl.mat != 0 && gl.mat != 1)) corrupt("mat-vec list");
      const int64_t arena = gl.mat ? ntm : npan;
      for (const GemvOp& o : gl.h) {
        if (o.rows < 0 || o.cols < 0 || o.ld < std::max(1, o.rows) || o.M < 0 || o.x < 0 ||
            o.y < 0 || (o.tri != 0 && o.tri != 1) || (o.beta_one != 0 && o.beta_one != 1))
          corrupt("mat-vec shape");
        if (o.rows && o.cols && o.M + (int64_t)(o.cols - 1) * o.ld + o.rows > arena)
          corrupt("mat-vec matrix extent");
        const int64_t xin = gl.trans ? o.rows : o.cols, yout = gl.trans ? o.cols : o.rows;
        if (o.x + xin > W || o.y + yout > W) corrupt("mat-vec vector extent");
      }
    }
  };
  lists_ok(s.fwd);
  lists_ok(s.bwd);
}

template <typename T>
void load_factor(Factor<T>& F, FileIn& in) {
  F.n = in.get<int>();
  F.m = in.get<int>();
  F.L = in.get<int>();
  F.precision = in.get<int>();
  F.eps = in.get<double>();
  F.bc = in.get<int>();
  if (F.bc != 0 && F.bc != 1) corrupt("boundary condition");
  F.opt = in.get<hif_options>();
  F.stats = in.get<hif_stats>();
  const int64_t stride_in_file = in.get<int64_t>();
  if (F.n < 1 || F.n > 1024 || F.L < 0 || F.L > 16) corrupt("grid");
  const int64_t N = (int64_t)F.n * F.n * F.n;
  in.buf(F.cpl, &F.mem);
  in.buf(F.diag, &F.mem);
  if (F.cpl.bytes() != sizeof(double) * 3 * N || F.diag.bytes() != sizeof(double) * N)
    corrupt("operator size");
  const uint64_t ns = in.get<uint64_t>();
  if (ns > 4096) corrupt("stage count");
  F.stages.resize(ns);
  F.work_stride = 0;
  for (Stage& s : F.stages) {
    s.kind = in.get<int>();
    s.level = in.get<int>();
    s.nidx = in.get<int64_t>();
    s.nset = in.get<int64_t>();
    s.nacc = in.get<int64_t>();
    s.entries = in.get<int64_t>();
    std::vector<unsigned char> idx_b, setg_b, setp_b, tgt_b, ptr_b, src_b;
    in.buf(s.idx, &F.mem, &idx_b);
    in.buf(s.panels, &F.mem);
    in.buf(s.tmats, &F.mem);
    in.buf(s.set_g, &F.mem, &setg_b);
    in.buf(s.set_p, &F.mem, &setp_b);
    in.buf(s.acc_tgt, &F.mem, &tgt_b);
    in.buf(s.acc_ptr, &F.mem, &ptr_b);
    in.buf(s.acc_src, &F.mem, &src_b);
    const uint32_t nf = in.get<uint32_t>();
    if (nf > 8) corrupt("mat-vec list count");
    s.fwd.resize(nf);
    for (auto& gl : s.fwd) in.list(gl, &F.mem);
    const uint32_t nb = in.get<uint32_t>();
    if (nb > 8) corrupt("mat-vec list count");
    s.bwd.resize(nb);
    for (auto& gl : s.bwd) in.list(gl, &F.mem);
    check_stage<T>(s, N, idx_b, setg_b, setp_b, tgt_b, ptr_b, src_b);
    // the sweeps' work stride follows from the stages, as in hif_factor
    F.work_stride = std::max(F.work_stride, 2 * s.nidx);
  }
  if (F.work_stride != stride_in_file) corrupt("work stride");
  const uint64_t na = in.get<uint64_t>();
  if (na > 16) corrupt("active set count");
  F.active.resize(na);
  for (auto& a : F.active) {
    const uint64_t c = in.get<uint64_t>();
    if (c > (uint64_t)N) corrupt("active set size");
    a.resize(c);
    in.raw(a.data(), sizeof(int32_t) * c);
    for (size_t i = 0; i < a.size(); ++i)
      if (a[i] < 0 || a[i] >= N || (i && a[i] <= a[i - 1])) corrupt("active set");
  }
  F.stats.factor_bytes = F.mem.cur;
}

}  // namespace
}  // namespace hif

extern "C" {

void hif_default_options(hif_options* o) {
  if (!o) return;
  o->eps = 1e-6;
  o->precision = HIF_PREC_FP64;
  o->use_graphs = 1;
  o->pcg_tol = 1e-10;
  o->max_iter = 200;
  o->tensor_cores = 1;
  o->retry_growth = 1e5;
}

const char* hif_version(void) { return "hif-gb300 0.1"; }

const char* hif_last_error(void) { return hif::g_last_error.c_str(); }

hif_status hif_factor(const hif_grid* grid, const double* a, const double* b, double b_const,
                      const hif_options* opt, hif_stream stream, hif_handle* out) {
  if (out) *out = nullptr;
  HIF_API_BEGIN
  if (!grid || !a || !out) throw Error{HIF_ERR_INVALID_ARG, "grid, a and out must not be NULL"};
  hif_options o;
  hif_default_options(&o);
  if (opt) o = *opt;
  const int n = grid->n, m = grid->m;
  const int L = hif::hif_num_levels(n, m);
  if (grid->bc != 0 && grid->bc != 1)
    throw Error{HIF_ERR_INVALID_ARG, "bc must be 0 (zero Dirichlet) or 1 (periodic)"};
  if (m < 2 || L < 0 || n > 1024)
    throw Error{HIF_ERR_INVALID_ARG, "need n = m 2^L with m >= 2 and n <= 1024"};
  if (!(o.eps >= 0.0) || !(o.eps < 1.0)) throw Error{HIF_ERR_INVALID_ARG, "eps must be in [0, 1)"};
  if (o.precision != HIF_PREC_FP64 && o.precision != HIF_PREC_FP32)
    throw Error{HIF_ERR_INVALID_ARG, "precision must be HIF_PREC_FP64 or HIF_PREC_FP32"};
  if (o.tensor_cores != 0 && o.tensor_cores != 1)
    throw Error{HIF_ERR_INVALID_ARG, "tensor_cores must be 0 or 1"};
  if (!std::isfinite(o.retry_growth) || o.retry_growth < 0)
    throw Error{HIF_ERR_INVALID_ARG, "retry_growth must be finite and >= 0"};
  if (!std::isfinite(b_const) || b_const < 0) throw Error{HIF_ERR_INVALID_ARG, "b_const must be finite and >= 0"};
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t N = (int64_t)n * n * n;
  hif::launch_counter() = 0;
  InArray ain, bin;
  ain.set(a, N, st);
  bin.set(b, N, st);
  auto h = std::make_unique<hif_handle_s>();
  int dev = 0;
  HIF_CUDA_TRY(cudaGetDevice(&dev));
  auto build = [&](auto* F) {
    F->device = dev;
    F->n = n;
    F->m = m;
    F->L = L;
    F->bc = grid->bc;
    F->eps = o.eps;
    F->precision = o.precision;
    F->opt = o;
    using FT = std::remove_pointer_t<decltype(F)>;
    using TT = std::conditional_t<std::is_same<FT, hif::Factor<float>>::value, float, double>;
    hif::Builder<TT> bld(*F, st);
    bld.run(ain.p, bin.p, b_const);
    F->stats.n = n;
    F->stats.m = m;
    F->stats.levels = L;
    F->stats.precision = o.precision;
    F->stats.eps = o.eps;
    F->stats.kernel_launches = (int)hif::launch_counter();
    int64_t ent = 0;
    for (auto& s : F->stages) ent += s.entries;
    F->stats.stored_entries = ent;
  };
  if (o.precision == HIF_PREC_FP32) {
    auto* F = new hif::Factor<float>();
    h->f.reset(F);
    build(F);
  } else {
    auto* F = new hif::Factor<double>();
    h->f.reset(F);
    build(F);
  }
  h->f->stats.factor_bytes = h->f->mem.cur;
  h->f->stats.peak_bytes = h->f->mem.peak;
  *out = h.release();
  return HIF_OK;
  HIF_API_END
}

hif_status hif_apply(hif_handle h, const double* f, double* u, int nrhs, hif_stream stream) {
  HIF_API_BEGIN
  if (!h || !f || !u || nrhs < 1) throw Error{HIF_ERR_INVALID_ARG, "bad handle, pointer or nrhs"};
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t N = (int64_t)h->f->n * h->f->n * h->f->n;
  InArray fin;
  fin.set(f, N * nrhs, st);
  OutArray uo;
  uo.set(u, N * nrhs);
  const int64_t l0 = hif::launch_counter();
  h->f->apply(fin.p, uo.p, nrhs, st);
  if (nrhs == 1) h->f->stats.apply_launches = (int)(hif::launch_counter() - l0);
  uo.finish(st);
  if (fin.tmp.bytes()) HIF_CUDA_TRY(cudaStreamSynchronize(st));
  return HIF_OK;
  HIF_API_END
}

hif_status hif_apply_noalloc(hif_handle h, const double* f, double* u, int nrhs,
                             hif_stream stream) {
  HIF_API_BEGIN
  if (!h || !f || !u || nrhs < 1) throw Error{HIF_ERR_INVALID_ARG, "bad handle, pointer or nrhs"};
  if (hif::prof_enabled())
    throw Error{HIF_ERR_INVALID_ARG, "hif_apply_noalloc cannot run while kernel profiling is on"};
  if (!hif::is_device_ptr(f) || !hif::is_device_ptr(u))
    throw Error{HIF_ERR_INVALID_ARG, "hif_apply_noalloc needs f and u in device memory"};
  {
    // the work array used is the current device's copy: the factor, f and u
    // must all live on that device
    int cur = -1;
    HIF_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != h->f->device || hif::pointer_device(f) != cur || hif::pointer_device(u) != cur)
      throw Error{HIF_ERR_INVALID_ARG,
                  "hif_apply_noalloc: the factor (device " + std::to_string(h->f->device) +
                      "), f and u must be on the current device (" + std::to_string(cur) + ")"};
  }
  const size_t need = h->f->sweep_scratch_bytes(nrhs);
  if (need > kNoAllocScratchBytes)
    throw Error{HIF_ERR_INVALID_ARG,
                "hif_apply_noalloc: this grid and nrhs need " + std::to_string(need) +
                    " bytes of work space, more than its fixed " +
                    std::to_string(kNoAllocScratchBytes) + " bytes"};
  void* scratch = noalloc_scratch_address();
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  h->f->apply_in_scratch(f, u, nrhs, scratch, st);
  return HIF_OK;
  HIF_API_END
}

hif_status hif_residual(hif_handle h, const double* f, const double* u, double* r, int nrhs,
                        hif_stream stream) {
  HIF_API_BEGIN
  if (!h || !f || !u || !r || nrhs < 1) throw Error{HIF_ERR_INVALID_ARG, "bad handle, pointer or nrhs"};
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t N = (int64_t)h->f->n * h->f->n * h->f->n;
  InArray fin, uin;
  fin.set(f, N * nrhs, st);
  uin.set(u, N * nrhs, st);
  OutArray ro;
  ro.set(r, N * nrhs);
  hif::residual(h->f->cpl.as<double>(), h->f->diag.as<double>(), h->f->n, h->f->bc, fin.p, uin.p,
                ro.p, nrhs, st);
  ro.finish(st);
  HIF_CUDA_TRY(cudaStreamSynchronize(st));
  return HIF_OK;
  HIF_API_END
}

hif_status hif_solve(hif_handle h, const double* f, double* u, int nrhs, hif_stream stream,
                     int* iters, double* relres) {
  HIF_API_BEGIN
  if (!h || !f || !u || nrhs < 1) throw Error{HIF_ERR_INVALID_ARG, "bad handle, pointer or nrhs"};
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t N = (int64_t)h->f->n * h->f->n * h->f->n;
  InArray fin;
  fin.set(f, N * nrhs, st);
  OutArray uo;
  uo.set(u, N * nrhs);
  hif_status s = hif::do_solve(*h->f, fin.p, uo.p, nrhs, st, iters, relres);
  uo.finish(st);
  if (s != HIF_OK) hif::set_last_error("PCG did not reach the tolerance within max_iter");
  return s;
  HIF_API_END
}

namespace {

// Checks shared by the batch entry points; returns the factors.
std::vector<hif::FactorBase*> batch_factors(const hif_handle* hs, int nh, const int* nrhs) {
  if (!hs || nh < 1 || !nrhs) throw Error{HIF_ERR_INVALID_ARG, "need nh >= 1 handles and nrhs"};
  std::vector<hif::FactorBase*> Fs;
  for (int i = 0; i < nh; ++i) {
    if (!hs[i] || nrhs[i] < 1) throw Error{HIF_ERR_INVALID_ARG, "bad handle or nrhs in the batch"};
    hif::FactorBase* F = hs[i]->f.get();
    if (std::find(Fs.begin(), Fs.end(), F) != Fs.end())
      throw Error{HIF_ERR_INVALID_ARG, "a handle appears twice in the batch"};
    if (!Fs.empty() && (F->precision != Fs[0]->precision || F->device != Fs[0]->device))
      throw Error{HIF_ERR_INVALID_ARG, "the batch's factors must share precision and device"};
    Fs.push_back(F);
  }
  return Fs;
}

}  // namespace

hif_status hif_apply_batch(const hif_handle* hs, int nh, const double* const* f,
                           double* const* u, const int* nrhs, hif_stream stream) {
  HIF_API_BEGIN
  std::vector<hif::FactorBase*> Fs = batch_factors(hs, nh, nrhs);
  if (!f || !u) throw Error{HIF_ERR_INVALID_ARG, "f and u must not be NULL"};
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::vector<InArray> fin(nh);
  std::vector<OutArray> uo(nh);
  std::vector<const double*> fp(nh);
  std::vector<double*> up(nh);
  std::vector<int> nr(nrhs, nrhs + nh);
  for (int i = 0; i < nh; ++i) {
    if (!f[i] || !u[i]) throw Error{HIF_ERR_INVALID_ARG, "f and u must not be NULL"};
    const int64_t N = (int64_t)Fs[i]->n * Fs[i]->n * Fs[i]->n;
    fin[i].set(f[i], N * nrhs[i], st);
    uo[i].set(u[i], N * nrhs[i]);
    fp[i] = fin[i].p;
    up[i] = uo[i].p;
  }
  hif::grouped_apply_any(Fs, fp, up, nr, st);
  bool staged = false;
  for (int i = 0; i < nh; ++i) {
    uo[i].finish(st);
    staged = staged || fin[i].tmp.bytes();
  }
  if (staged) HIF_CUDA_TRY(cudaStreamSynchronize(st));
  return HIF_OK;
  HIF_API_END
}

hif_status hif_solve_batch(const hif_handle* hs, int nh, const double* const* f, double* const* u,
                           const int* nrhs, hif_stream stream, int* iters, double* relres) {
  HIF_API_BEGIN
  std::vector<hif::FactorBase*> Fs = batch_factors(hs, nh, nrhs);
  if (!f || !u) throw Error{HIF_ERR_INVALID_ARG, "f and u must not be NULL"};
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::vector<InArray> fin(nh);
  std::vector<OutArray> uo(nh);
  std::vector<hif::PcgItem> items(nh);
  for (int i = 0; i < nh; ++i) {
    if (!f[i] || !u[i]) throw Error{HIF_ERR_INVALID_ARG, "f and u must not be NULL"};
    const int64_t N = (int64_t)Fs[i]->n * Fs[i]->n * Fs[i]->n;
    fin[i].set(f[i], N * nrhs[i], st);
    uo[i].set(u[i], N * nrhs[i]);
    items[i].F = Fs[i];
    items[i].f = fin[i].p;
    items[i].u = uo[i].p;
    items[i].nrhs = nrhs[i];
  }
  const hif_status s = hif::pcg_many(items, st, [](const std::vector<hif::PcgItem*>& v, cudaStream_t s2) {
    std::vector<hif::FactorBase*> F;
    std::vector<const double*> r;
    std::vector<double*> z;
    std::vector<int> nr;
    for (hif::PcgItem* I : v) {
      F.push_back(I->F);
      r.push_back(I->b.r.as<double>());
      z.push_back(I->b.z.as<double>());
      nr.push_back(I->nrhs);
    }
    hif::grouped_apply_any(F, r, z, nr, s2);
  });
  int col = 0;
  for (int i = 0; i < nh; ++i) {
    uo[i].finish(st);
    for (int c = 0; c < nrhs[i]; ++c, ++col) {
      if (iters) iters[col] = items[i].it[c];
      if (relres) relres[col] = items[i].rel[c];
    }
  }
  if (s != HIF_OK) hif::set_last_error("PCG did not reach the tolerance within max_iter");
  return s;
  HIF_API_END
}

hif_status hif_autotune(const hif_grid* grid, const double* a, const double* b, double b_const,
                        const hif_options* opt, const char* path, int force, hif_stream stream) {
  HIF_API_BEGIN
  if (path && !force) {
    if (std::FILE* fh = std::fopen(path, "rb")) {
      std::string text;
      char buf[4096];
      size_t got;
      while ((got = std::fread(buf, 1, sizeof(buf), fh)) > 0) text.append(buf, got);
      std::fclose(fh);
      std::string why;
      if (hif::tune_parse(text, &why)) return HIF_OK;   // a table for this device
    }
  }
  hif::tune_clear();
  {
    // one factorization measures: the cluster IDs time their shapes in
    // place, the tensor-core products record theirs
    hif::TuneSession session;
    hif_handle h = nullptr;
    const hif_status s = hif_factor(grid, a, b, b_const, opt, stream, &h);
    if (s != HIF_OK) return s;
    hif_destroy(h);
  }
  hif::tune_gemm_from_records(reinterpret_cast<cudaStream_t>(stream));
  if (path) {
    const std::string text = hif::tune_serialize();
    std::FILE* fh = std::fopen(path, "wb");
    if (!fh) throw Error{HIF_ERR_INVALID_ARG, std::string("cannot write ") + path};
    const size_t put = std::fwrite(text.data(), 1, text.size(), fh);
    std::fclose(fh);
    if (put != text.size()) throw Error{HIF_ERR_INVALID_ARG, std::string("cannot write ") + path};
  }
  return HIF_OK;
  HIF_API_END
}

hif_status hif_autotune_load(const char* path) {
  HIF_API_BEGIN
  if (!path) throw Error{HIF_ERR_INVALID_ARG, "path must not be NULL"};
  std::FILE* fh = std::fopen(path, "rb");
  if (!fh) throw Error{HIF_ERR_INVALID_ARG, std::string("cannot open ") + path};
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), fh)) > 0) text.append(buf, got);
  std::fclose(fh);
  std::string why;
  if (!hif::tune_parse(text, &why)) throw Error{HIF_ERR_INVALID_ARG, "tuning table rejected: " + why};
  return HIF_OK;
  HIF_API_END
}

void hif_autotune_clear(void) { hif::tune_clear(); }

hif_status hif_autotune_table(char* buf, size_t cap, size_t* len) {
  HIF_API_BEGIN
  const std::string text = hif::tune_serialize();
  if (len) *len = text.size();
  if (buf && cap) {
    const size_t n = std::min(cap - 1, text.size());
    std::memcpy(buf, text.data(), n);
    buf[n] = 0;
  }
  return HIF_OK;
  HIF_API_END
}

hif_status hif_query_stats(hif_handle h, hif_stats* st) {
  if (!h || !st) {
    hif::set_last_error("NULL handle or stats");
    return HIF_ERR_INVALID_ARG;
  }
  *st = h->f->stats;
  st->factor_bytes = h->f->mem.cur;
  return HIF_OK;
}

hif_status hif_query_active(hif_handle h, int level, int32_t* out, int64_t cap,
                            int64_t* count) {
  HIF_API_BEGIN
  if (!h || !count) throw Error{HIF_ERR_INVALID_ARG, "NULL handle or count"};
  const auto& act = h->f->active;
  if (level < 0 || level >= (int)act.size())
    throw Error{HIF_ERR_INVALID_ARG, "level must be in [0, L)"};
  const auto& a = act[(size_t)level];
  *count = (int64_t)a.size();
  if (out) {
    if (cap < (int64_t)a.size()) throw Error{HIF_ERR_INVALID_ARG, "out holds fewer than count entries"};
    std::memcpy(out, a.data(), sizeof(int32_t) * a.size());
  }
  return HIF_OK;
  HIF_API_END
}

size_t hif_predict_bytes(const hif_grid* grid, const hif_options* opt) {
  if (!grid || hif::hif_num_levels(grid->n, grid->m) < 0) return 0;
  const double N = (double)grid->n * grid->n * grid->n;
  const int prec = opt ? opt->precision : HIF_PREC_FP64;
  const double word = prec == HIF_PREC_FP32 ? 4.0 : 8.0;
  // Peak device bytes of hif_factor: the operator (32 B per DOF) plus factor
  // words per DOF growing with log2 n, fitted to measured peaks at eps = 1e-6
  // (64^3: ~2000 words per DOF, 128^3: ~3000) with a 25% margin, and at
  // least 400 words per DOF for small grids.  A larger eps keeps fewer
  // skeletons: the measured peaks shrink by ~0.56 per decade of eps above
  // 1e-6 (64^3: 2.1 / 1.2 / 0.7 GB at 1e-6 / 1e-5 / 1e-4; 256^3 at 1e-4:
  // 74 GB), taken here as 0.6 per decade, at most four decades.
  const double lg = std::log2((double)grid->n);
  double words = std::max(400.0, -3718.0 + 955.0 * lg);
  const double eps = opt ? opt->eps : 1e-6;
  if (eps > 1e-6) words *= std::pow(0.6, std::min(4.0, std::log10(eps / 1e-6)));
  return (size_t)(N * (32.0 + 1.25 * words * word) + (64u << 20));
}

void hif_destroy(hif_handle h) { delete h; }

hif_status hif_save(hif_handle h, const char* path) {
  HIF_API_BEGIN
  if (!h || !path) throw Error{HIF_ERR_INVALID_ARG, "handle and path must not be NULL"};
  HIF_CUDA_TRY(cudaDeviceSynchronize());
  hif::FileOut o(path);
  o.raw("HIFF", 4);
  o.put(hif::kFileVersion);
  o.put((uint32_t)sizeof(hif_options));
  o.put((uint32_t)sizeof(hif_stats));
  if (h->f->precision == HIF_PREC_FP32)
    hif::save_factor(*static_cast<hif::Factor<float>*>(h->f.get()), o);
  else
    hif::save_factor(*static_cast<hif::Factor<double>*>(h->f.get()), o);
  return HIF_OK;
  HIF_API_END
}

hif_status hif_load(const char* path, hif_handle* out) {
  if (out) *out = nullptr;
  HIF_API_BEGIN
  if (!path || !out) throw Error{HIF_ERR_INVALID_ARG, "path and out must not be NULL"};
  hif::FileIn in(path);
  char magic[4];
  in.raw(magic, 4);
  if (std::memcmp(magic, "HIFF", 4) != 0) throw Error{HIF_ERR_INVALID_ARG, "not a factor file"};
  if (in.get<uint32_t>() != hif::kFileVersion || in.get<uint32_t>() != sizeof(hif_options) ||
      in.get<uint32_t>() != sizeof(hif_stats))
    throw Error{HIF_ERR_INVALID_ARG, "factor file written by another version"};
  auto hh = std::make_unique<hif_handle_s>();
  int dev = 0;
  HIF_CUDA_TRY(cudaGetDevice(&dev));
  // the precision decides the factor's word size: peek at it after n, m, L
  const long pos = std::ftell(in.f);
  in.get<int>();
  in.get<int>();
  in.get<int>();
  const int prec = in.get<int>();
  std::fseek(in.f, pos, SEEK_SET);
  if (prec == HIF_PREC_FP32) {
    auto* F = new hif::Factor<float>();
    hh->f.reset(F);
    F->device = dev;
    hif::load_factor(*F, in);
  } else if (prec == HIF_PREC_FP64) {
    auto* F = new hif::Factor<double>();
    hh->f.reset(F);
    F->device = dev;
    hif::load_factor(*F, in);
  } else {
    throw Error{HIF_ERR_INVALID_ARG, "corrupt factor file"};
  }
  *out = hh.release();
  return HIF_OK;
  HIF_API_END
}

}  // extern "C"
