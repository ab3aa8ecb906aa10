// Launch accounting: construct a ProfScope right before a kernel launch and
// let it go out of scope right after; it counts the launch and, when
// profiling is enabled, brackets it with CUDA events on its stream.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace slos {

class ProfScope {
  public:
    ProfScope(const char *name, double algorithmic_bytes, cudaStream_t s);
    ~ProfScope();
    ProfScope(const ProfScope &) = delete;
    ProfScope &operator=(const ProfScope &) = delete;

  private:
    bool active_;
    size_t idx_ = 0;
    cudaStream_t stream_;
};

// Counts a launch that is timed inside another kernel's scope.
void count_launch();

}  // namespace slos
