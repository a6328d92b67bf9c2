// Autotuning table: launch shapes of the batched kernels per size bucket,
// chosen by timing on the device (hif_autotune) among shapes that give
// bitwise the same results.  Process-wide; host code only.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "common.cuh"

namespace hif {

// Tensor-core products (gemm_tc): bucket = (shape class, waves class).
//   shape class: 0 narrow (<= 64 rows), 1 fewer than 256 columns, 2 wider;
//   waves class: output tiles against 2 CTAs per SM: < 1/2, < 2, >= 2 waves.
// Variant: 0 = K chunks of 16 with 128 x 128 tiles, 1 = 16 / 128 x 256,
// 2 = 32 / 128 x 128.  Every variant accumulates each output entry with the
// same sequence of K = 8 tensor-core steps, so they agree bitwise (when K
// is split across CTAs only variants with the default chunk are allowed).
int gemm_shape_class(int mmax, int nmax, int kmax);
int gemm_waves_class(int tiles, int nsm);

// Cluster ID (k_cpqr): bucket = (width class of the call's widest cluster
// front, count class of the call's cluster fronts).  width: nF < 512, < 1024,
// < 2048, >= 2048; count: <= 16, <= 64, <= 256, > 256.  Choice: cluster size
// (CTAs per front; 0 = the built-in rule) and fronts per launch (0 = all).  A column's arithmetic does not
// depend on which CTA of the cluster owns it, nor on which fronts share a
// launch, so every choice agrees bitwise.
int id_width_class(int nF);
int id_count_class(int nfronts);
struct IdChoice {
  int cs = -1;    // -1: no entry; 0: the built-in rule; 1-16: CTAs per front
  int wave = 0;   // fronts per launch, 0 = all
};

bool tune_gemm_lookup(int shape_cls, int waves_cls, int* variant);
// seconds: the measured time of each candidate (kept as comments of the table)
void tune_gemm_set(int shape_cls, int waves_cls, int variant, const double seconds[3]);
bool tune_id_lookup(int width_cls, int count_cls, IdChoice* c);
void tune_id_set(int width_cls, int count_cls, IdChoice c,
                 const std::vector<std::pair<IdChoice, double>>& tried);
void tune_clear();
std::string tune_serialize();
// Parse a table written by tune_serialize for this device; false (and the
// table unchanged) if it is malformed or for another device.
bool tune_parse(const std::string& text, std::string* why);
std::string tune_device_tag();

// While a TuneSession is alive on this thread, hif_factor measures: the ID
// times its candidate shapes in place for buckets without an entry, and the
// tensor-core products record their shapes for a later replay.
struct GemmShapeRec {
  int shape_cls, waves_cls;
  double flops;
  std::vector<GemmOp> ops;
};
bool tune_session_active();
void tune_record_gemm(int shape_cls, int waves_cls, const GemmOp* ops, int nops, double flops);
std::vector<GemmShapeRec> tune_take_gemm_records();
class TuneSession {
 public:
  TuneSession();
  ~TuneSession();
  TuneSession(const TuneSession&) = delete;
  TuneSession& operator=(const TuneSession&) = delete;
};

}  // namespace hif
