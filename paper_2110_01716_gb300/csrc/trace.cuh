// trace.cuh -- per-class launch counters and event timers (see trace.cu).
#pragma once

#include <map>
#include <string>

#include "common.cuh"

namespace sem {

// Counts one launch of class "<name>_N<order>" and, when the class matches
// the timing filter, brackets it with CUDA events on `st`.  Construct it just
// before the launch; it records the closing event when it goes out of scope.
class TraceScope {
 public:
  // `kernels`: how many kernels the scope launches (counted as launches)
  TraceScope(const char *name, int N, cudaStream_t st, int kernels = 1);
  ~TraceScope();
  TraceScope(const TraceScope &) = delete;
  TraceScope &operator=(const TraceScope &) = delete;

 private:
  cudaStream_t st_;
  cudaEvent_t e0_{}, e1_{};
  bool active_ = false;
  std::string key_;
};

// Adds `launches` kernel launches to class "<name>_N<order>" (or to the class
// named `key`) without timing (kernels that ran inside a graph launch).
void trace_count(const char *name, int N, int64_t launches);
void trace_count_key(const std::string &key, int64_t launches);

// While a tally is open, the TraceScopes this thread meets on a capturing
// stream add their kernels to (*tally)[class] instead of counting them: the
// per-class kernels of a captured graph, for trace_count_key per replay.
void trace_tally_begin(std::map<std::string, int64_t> *tally);
void trace_tally_end();

}  // namespace sem
