// trace.cu -- launch counters and CUDA-event timers per kernel class.
//
// The paper's codes report timing breakdowns from CUDA events (Sec. 4,
// Table 1).  Here every library launch passes through a TraceScope: when
// tracing is on it counts the launch under its class name ("ax_f64_N7",
// "gs_f32_N3", ...), and for classes whose name contains the timing filter it
// records an event pair on the launching stream.  Elapsed times are resolved
// when the trace is read, so timing adds no host synchronisation.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "trace.cuh"

namespace sem {

namespace {
struct ClassStats {
  int64_t launches = 0;
  int64_t timed = 0;
  double ms = 0.0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};
struct Tracer {
  std::atomic<bool> on{false};
  std::mutex mu;
  std::string filter;
  std::map<std::string, ClassStats> cls;
  std::vector<cudaEvent_t> pool;
};
Tracer &tracer() {
  static Tracer *t = new Tracer();  // never destroyed: events may outlive static teardown order
  return *t;
}
cudaEvent_t take_event(Tracer &T) {
  if (!T.pool.empty()) {
    cudaEvent_t e = T.pool.back();
    T.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  SEM_CHECK_CUDA(cudaEventCreate(&e));
  return e;
}
}  // namespace

bool trace_on() { return tracer().on.load(std::memory_order_relaxed); }

// "*" matches every class; otherwise the filter is a '|'-separated list of
// substrings, any of which selects a class.
static bool filter_matches(const std::string &filter, const char *name) {
  if (filter.empty()) return false;
  if (filter == "*") return true;
  size_t start = 0;
  while (start <= filter.size()) {
    size_t end = filter.find('|', start);
    if (end == std::string::npos) end = filter.size();
    if (end > start && std::strstr(name, filter.substr(start, end - start).c_str()) != nullptr)
      return true;
    start = end + 1;
  }
  return false;
}

namespace {
// Kernels per class captured by this thread while a tally is open.
thread_local std::map<std::string, int64_t> *t_tally = nullptr;
}  // namespace

void trace_tally_begin(std::map<std::string, int64_t> *tally) { t_tally = tally; }
void trace_tally_end() { t_tally = nullptr; }

TraceScope::TraceScope(const char *name, int N, cudaStream_t st, int kernels) : st_(st) {
  Tracer &T = tracer();
  if (!T.on.load(std::memory_order_relaxed) && !t_tally) return;
  char buf[64];
  snprintf(buf, sizeof(buf), "%s_N%d", name, N);
  // launches captured into a CUDA graph run later, once per replay: the
  // capture's tally holds them and the graph's owner counts the replays
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    if (t_tally) (*t_tally)[buf] += kernels;
    return;
  }
  if (!T.on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lock(T.mu);
  ClassStats &c = T.cls[buf];
  c.launches += kernels;
  if (filter_matches(T.filter, buf)) {
    e0_ = take_event(T);
    e1_ = take_event(T);
    SEM_CHECK_CUDA(cudaEventRecord(e0_, st_));
    key_ = buf;
    active_ = true;
  }
}

TraceScope::~TraceScope() {
  if (!active_) return;
  Tracer &T = tracer();
  cudaEventRecord(e1_, st_);
  std::lock_guard<std::mutex> lock(T.mu);
  T.cls[key_].pending.emplace_back(e0_, e1_);
}

void trace_count(const char *name, int N, int64_t launches) {
  char buf[64];
  snprintf(buf, sizeof(buf), "%s_N%d", name, N);
  trace_count_key(buf, launches);
}

void trace_count_key(const std::string &key, int64_t launches) {
  Tracer &T = tracer();
  if (!T.on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lock(T.mu);
  T.cls[key].launches += launches;
}

void trace_enable(bool on, const char *filter) {
  Tracer &T = tracer();
  std::lock_guard<std::mutex> lock(T.mu);
  T.filter = filter ? filter : "";
  T.on.store(on);
}

int trace_read(sem_trace_entry *out, int max_entries, bool reset) {
  Tracer &T = tracer();
  std::lock_guard<std::mutex> lock(T.mu);
  int n = 0;
  for (auto &kv : T.cls) {
    ClassStats &c = kv.second;
    for (auto &pr : c.pending) {
      SEM_CHECK_CUDA(cudaEventSynchronize(pr.second));
      float ms = 0.f;
      SEM_CHECK_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
      c.ms += ms;
      c.timed += 1;
      T.pool.push_back(pr.first);
      T.pool.push_back(pr.second);
    }
    c.pending.clear();
    if (out && n < max_entries) {
      sem_trace_entry &e = out[n];
      std::memset(&e, 0, sizeof(e));
      std::strncpy(e.name, kv.first.c_str(), sizeof(e.name) - 1);
      e.launches = c.launches;
      e.timed = c.timed;
      e.total_ms = c.ms;
    }
    ++n;
  }
  if (reset) T.cls.clear();
  return n;
}

}  // namespace sem

extern "C" {

sem_status sem_trace_enable(int32_t enable, const char *timed_filter) {
  try {
    sem::trace_enable(enable != 0, timed_filter);
    return SEM_OK;
  } catch (const sem::Failure &f) {
    return f.status;
  }
}

sem_status sem_trace_read(sem_trace_entry *out, int32_t max_entries, int32_t *n_entries,
                          int32_t reset) {
  try {
    if (max_entries < 0 || (max_entries > 0 && !out)) {
      sem::set_error_message("bad output array");
      return SEM_EINVAL;
    }
    int n = sem::trace_read(out, max_entries, reset != 0);
    if (n_entries) *n_entries = n;
    return SEM_OK;
  } catch (const sem::Failure &f) {
    return f.status;
  }
}

}  // extern "C"
