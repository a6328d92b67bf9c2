// Autotuning table (see tune.h).
#include "tune.h"

#include <cuda_runtime.h>

#include <cstdio>
#include <map>
#include <mutex>
#include <sstream>

namespace hif {

namespace {

struct Table {
  std::mutex mu;
  std::map<std::pair<int, int>, int> gemm;
  std::map<std::pair<int, int>, IdChoice> id;
  std::map<std::pair<int, int>, GemmShapeRec> rec;
  std::vector<std::string> notes;   // measured candidates, as comment lines
};

Table& table() {
  static Table t;
  return t;
}

thread_local int t_session = 0;

}  // namespace

int gemm_shape_class(int mmax, int nmax, int kmax) {
  // rows and width of the widest product; + 3 for shallow batches (K <= 256),
  // whose tiles are dominated by the C read and write rather than the K loop
  return (mmax <= 64 ? 0 : (nmax < 256 ? 1 : 2)) + (kmax <= 256 ? 3 : 0);
}

int gemm_waves_class(int tiles, int nsm) {
  const double w = (double)tiles / (2.0 * nsm);
  return w < 0.5 ? 0 : (w < 2.0 ? 1 : 2);
}

int id_width_class(int nF) { return nF < 512 ? 0 : nF < 1024 ? 1 : nF < 2048 ? 2 : 3; }

int id_count_class(int n) { return n <= 16 ? 0 : n <= 64 ? 1 : n <= 256 ? 2 : 3; }

bool tune_gemm_lookup(int s, int w, int* variant) {
  Table& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  auto it = t.gemm.find({s, w});
  if (it == t.gemm.end()) return false;
  *variant = it->second;
  return true;
}

void tune_gemm_set(int s, int w, int variant, const double* seconds) {
  Table& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  t.gemm[{s, w}] = variant;
  std::string line = "# gemm " + std::to_string(s) + " " + std::to_string(w) + ":";
  for (int v = 0; v < 3; ++v) {
    char buf[48];
    if (seconds[v] > 0.0) std::snprintf(buf, sizeof(buf), " variant %d %.3f ms", v, 1e3 * seconds[v]);
    else std::snprintf(buf, sizeof(buf), " variant %d not a candidate", v);
    line += buf;
  }
  t.notes.push_back(line);
}

bool tune_id_lookup(int wc, int cc, IdChoice* c) {
  Table& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  auto it = t.id.find({wc, cc});
  if (it == t.id.end()) return false;
  *c = it->second;
  return true;
}

void tune_id_set(int wc, int cc, IdChoice c, const std::vector<std::pair<IdChoice, double>>& tried) {
  Table& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  t.id[{wc, cc}] = c;
  std::string line = "# id " + std::to_string(wc) + " " + std::to_string(cc) + ":";
  for (auto& [ch, sec] : tried) {
    char buf[64];
    std::snprintf(buf, sizeof(buf), " cs%d/w%d %.2f ms", ch.cs, ch.wave, 1e3 * sec);
    line += buf;
  }
  t.notes.push_back(line);
}

void tune_clear() {
  Table& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  t.gemm.clear();
  t.id.clear();
  t.rec.clear();
  t.notes.clear();
}

std::string tune_device_tag() {
  int dev = 0;
  cudaDeviceProp p{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string name = p.name;
  for (char& ch : name)
    if (ch == ' ') ch = '_';
  return name + "_sm" + std::to_string(p.multiProcessorCount) + "_cc" + std::to_string(p.major) +
         std::to_string(p.minor);
}

std::string tune_serialize() {
  Table& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  std::ostringstream o;
  o << "# hif autotune table: launch shapes per size bucket, chosen by timing\n";
  o << "device " << tune_device_tag() << "\n";
  for (auto& n : t.notes) o << n << "\n";
  for (auto& kv : t.gemm)
    o << "gemm " << kv.first.first << " " << kv.first.second << " " << kv.second << "\n";
  for (auto& kv : t.id)
    o << "id " << kv.first.first << " " << kv.first.second << " " << kv.second.cs << " "
      << kv.second.wave << "\n";
  return o.str();
}

bool tune_parse(const std::string& text, std::string* why) {
  std::istringstream in(text);
  std::string line;
  std::map<std::pair<int, int>, int> g;
  std::map<std::pair<int, int>, IdChoice> id;
  bool dev_ok = false;
  while (std::getline(in, line)) {
    if (line.empty() || line[0] == '#') continue;
    std::istringstream ls(line);
    std::string kind;
    ls >> kind;
    if (kind == "device") {
      std::string tag;
      ls >> tag;
      if (tag != tune_device_tag()) {
        if (why) *why = "table written for " + tag + ", this device is " + tune_device_tag();
        return false;
      }
      dev_ok = true;
    } else if (kind == "gemm") {
      int s = -1, w = -1, v = -1;
      ls >> s >> w >> v;
      if (!ls || s < 0 || s > 5 || w < 0 || w > 2 || v < 0 || v > 2) {
        if (why) *why = "bad line: " + line;
        return false;
      }
      g[{s, w}] = v;
    } else if (kind == "id") {
      int a = -1, b = -1;
      IdChoice c;
      ls >> a >> b >> c.cs >> c.wave;
      if (!ls || a < 0 || a > 3 || b < 0 || b > 3 || c.cs < 0 || c.cs > 16 || c.wave < 0) {
        if (why) *why = "bad line: " + line;
        return false;
      }
      id[{a, b}] = c;
    } else {
      if (why) *why = "bad line: " + line;
      return false;
    }
  }
  if (!dev_ok) {
    if (why) *why = "no device line";
    return false;
  }
  Table& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  t.gemm = std::move(g);
  t.id = std::move(id);
  return true;
}

bool tune_session_active() { return t_session > 0; }

void tune_record_gemm(int s, int w, const GemmOp* ops, int nops, double flops) {
  Table& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  auto& r = t.rec[{s, w}];
  if (flops > r.flops) {
    r.shape_cls = s;
    r.waves_cls = w;
    r.flops = flops;
    r.ops.assign(ops, ops + nops);
  }
}

std::vector<GemmShapeRec> tune_take_gemm_records() {
  Table& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  std::vector<GemmShapeRec> out;
  for (auto& kv : t.rec) out.push_back(std::move(kv.second));
  t.rec.clear();
  return out;
}

TuneSession::TuneSession() { ++t_session; }
TuneSession::~TuneSession() { --t_session; }

}  // namespace hif
