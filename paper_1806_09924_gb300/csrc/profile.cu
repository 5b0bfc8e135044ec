// Opt-in per-kernel timing with CUDA events and a process-wide launch counter.
//
// When enabled (pff_profile_enable), every instrumented launcher records an
// event pair on the stream it launches on, together with the algorithmic
// bytes of that launch (the bytes the operation must move at minimum: each
// input and output array once).  pff_profile_report synchronizes, resolves the
// pending events and returns per-kernel totals as JSON.  The launch counter
// counts every kernel the library launches, instrumented or not.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pff_internal.h"

namespace pff {

std::atomic<long long> g_launches{0};

namespace {

struct Pending {
  const char* name;
  double bytes;
  cudaEvent_t a, b;
};

struct Acc {
  long long count = 0;
  double ms = 0.0;
  double bytes = 0.0;
};

struct Profiler {
  std::mutex mu;
  bool on = false;
  std::vector<std::string> only;   // when not empty, only launches of these names are timed
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, Acc> acc;

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }

  // resolve completed records (all of them when `all`, after a device sync)
  void flush(bool all) {
    std::vector<Pending> keep;
    for (auto& p : pending) {
      if (!all && cudaEventQuery(p.b) != cudaSuccess) {
        keep.push_back(p);
        continue;
      }
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        Acc& a = acc[p.name];
        a.count += 1;
        a.ms += ms;
        a.bytes += p.bytes;
      }
      cudaGetLastError();
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.swap(keep);
  }
};

Profiler& prof() {
  static Profiler* p = new Profiler();
  return *p;
}

}  // namespace

bool verbose() {
  static const bool v = std::getenv("PFF_VERBOSE") != nullptr;
  return v;
}

namespace {
thread_local bool t_capturing = false;
thread_local double t_capture_bytes = 0.0;
}

void set_capturing(bool on) {
  if (on && !t_capturing) t_capture_bytes = 0.0;
  t_capturing = on;
}

double captured_bytes() { return t_capture_bytes; }

void count_launch(int k) {
  if (!t_capturing) g_launches.fetch_add(k, std::memory_order_relaxed);
}

ProfScope::ProfScope(const char* name, double bytes, cudaStream_t s, int kernels)
    : name_(name), bytes_(bytes), s_(s), a_(nullptr) {
  count_launch(kernels);
  if (t_capturing) {
    t_capture_bytes += bytes;
    return;
  }
  Profiler& P = prof();
  if (!P.on) return;
  if (!P.only.empty() && std::find(P.only.begin(), P.only.end(), name_) == P.only.end()) return;
  std::lock_guard<std::mutex> g(P.mu);
  if (P.pending.size() > 4096) P.flush(false);
  a_ = P.get();
  cudaEventRecord(static_cast<cudaEvent_t>(a_), s_);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  Profiler& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  cudaEvent_t b = P.get();
  cudaEventRecord(b, s_);
  P.pending.push_back({name_, bytes_, static_cast<cudaEvent_t>(a_), b});
}

// --------------------------------------------------- persistent tuning record --
// The autotuners (sparse-kernel formats, element-kernel tiles, Jacobian apply
// variant) time their candidates with CUDA events.  Under a profiler that
// serialises and instruments every launch those timings mean nothing, and a
// profiled run would execute different kernels than the run it documents.  With
// PFF_TUNE_CACHE naming a file, every choice made is written there, and choices
// found there are reused without timing: a plain run of a command records them,
// the same command under the profiler replays them.
namespace {
struct TuneRecord {
  std::mutex mu;
  bool loaded = false;
  std::string path;
  std::map<std::string, int> entries;

  void load() {   // mu held
    if (loaded) return;
    loaded = true;
    const char* e = std::getenv("PFF_TUNE_CACHE");
    if (!e || !*e) return;
    path = e;
    if (FILE* f = std::fopen(path.c_str(), "r")) {
      char key[256];
      int v = 0;
      while (std::fscanf(f, "%255s %d", key, &v) == 2) entries[key] = v;
      std::fclose(f);
    }
  }
};

TuneRecord& tune_record() {
  static TuneRecord* t = new TuneRecord();
  return *t;
}
}  // namespace

bool tune_lookup(const std::string& key, int* value) {
  TuneRecord& t = tune_record();
  std::lock_guard<std::mutex> g(t.mu);
  t.load();
  auto it = t.entries.find(key);
  if (it == t.entries.end()) return false;
  *value = it->second;
  return true;
}

void tune_store(const std::string& key, int value) {
  TuneRecord& t = tune_record();
  std::lock_guard<std::mutex> g(t.mu);
  t.load();
  t.entries[key] = value;
  if (t.path.empty()) return;
  if (FILE* f = std::fopen(t.path.c_str(), "w")) {
    for (const auto& kv : t.entries) std::fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
    std::fclose(f);
  }
}

}  // namespace pff

extern "C" {

int pff_profile_enable(int on) {
  auto& P = pff::prof();
  std::lock_guard<std::mutex> g(P.mu);
  cudaDeviceSynchronize();
  P.flush(true);
  P.acc.clear();
  P.on = on != 0;
  return PFF_OK;
}

int pff_profile_select(const char* name) {
  auto& P = pff::prof();
  std::lock_guard<std::mutex> g(P.mu);
  P.only.clear();
  if (name) {
    const std::string all(name);
    size_t a = 0;
    while (a <= all.size()) {
      size_t b = all.find(',', a);
      if (b == std::string::npos) b = all.size();
      if (b > a) P.only.push_back(all.substr(a, b - a));
      a = b + 1;
    }
  }
  return PFF_OK;
}

int pff_profile_report(char* buf, int buflen) {
  auto& P = pff::prof();
  std::lock_guard<std::mutex> g(P.mu);
  cudaDeviceSynchronize();
  P.flush(true);
  std::string s = "{";
  bool first = true;
  for (auto& kv : P.acc) {
    char tmp[256];
    std::snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"count\": %lld, \"ms\": %.6f, \"bytes\": %.0f}",
                  first ? "" : ", ", kv.first.c_str(), kv.second.count, kv.second.ms,
                  kv.second.bytes);
    s += tmp;
    first = false;
  }
  s += "}";
  if (buf && buflen > 0) {
    const size_t n = std::min<size_t>(s.size(), (size_t)buflen - 1);
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return (int)s.size() + 1;
}

long long pff_launch_count(void) { return pff::g_launches.load(); }

}  // extern "C"
