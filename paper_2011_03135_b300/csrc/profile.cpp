// Launch accounting and an optional per-kernel timer.
//
// Every kernel launch site of the library is wrapped by gpm_prof_begin /
// gpm_prof_end. The launch counter always runs; when profiling is enabled the
// pair also records CUDA events on the launching stream, and
// gpm_profile_report() (after the caller has synchronised) sums the elapsed
// time per kernel name.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gpm_internal.h"

namespace {

std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_enabled{0};
std::mutex g_mu;

struct Pending {
  std::string name;
  cudaEvent_t start, stop;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
struct Stat {
  uint64_t launches = 0;
  double ms = 0.0;
};
std::map<std::string, Stat> g_stats;
thread_local std::vector<Pending> t_open;

cudaEvent_t take_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void drain_locked() {
  for (auto &p : g_pending) {
    float ms = 0.f;
    if (p.start && p.stop && cudaEventSynchronize(p.stop) == cudaSuccess &&
        cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
      Stat &s = g_stats[p.name];
      s.launches++;
      s.ms += ms;
    } else {
      cudaGetLastError();
    }
    if (p.start) g_free.push_back(p.start);
    if (p.stop) g_free.push_back(p.stop);
  }
  g_pending.clear();
}

}  // namespace

void gpm_note_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

static thread_local uint64_t t_captured = 0;
uint64_t gpm_captured_launches() { return t_captured; }

void gpm_prof_begin(const char *name, cudaStream_t st) {
  if (capturing(st)) {
    t_open.push_back(Pending{name, nullptr, nullptr});  // launches inside a graph are counted at replay
    ++t_captured;
    return;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_enabled.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Pending p{name, take_event(), take_event()};
  if (p.start) cudaEventRecord(p.start, st);
  t_open.push_back(p);
}

void gpm_prof_end(cudaStream_t st) {
  if (t_open.empty()) return;
  if (!t_open.back().start && !t_open.back().stop) {
    t_open.pop_back();
    return;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  Pending p = t_open.back();
  t_open.pop_back();
  if (p.stop) cudaEventRecord(p.stop, st);
  g_pending.push_back(p);
}

extern "C" {

uint64_t gpm_kernel_launches(void) { return g_launches.load(); }

int gpm_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_enabled.store(on ? 1 : 0);
  return GPM_OK;
}

int gpm_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  g_stats.clear();
  return GPM_OK;
}

int gpm_profile_report(char *buf, size_t len, size_t *needed) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  std::string s = "{";
  bool first = true;
  for (auto &kv : g_stats) {
    if (!first) s += ",";
    first = false;
    char tmp[96];
    snprintf(tmp, sizeof(tmp), "\":{\"launches\":%llu,\"ms\":%.6f}", (unsigned long long)kv.second.launches,
             kv.second.ms);
    s += "\"" + kv.first + tmp;
  }
  s += "}";
  if (needed) *needed = s.size() + 1;
  if (buf && len) {
    size_t n = std::min(len - 1, s.size());
    memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return GPM_OK;
}

}  // extern "C"
