// Helper for the pass-kernel instantiation units: each unit instantiates the
// kernel for one (mode, precision) over every supported length and exposes
// a lookup from log2 N to the kernel entry point.
#pragma once
#include "pass_kernel.cuh"

namespace tcfft {

template <int MODE, bool SPLIT, int LOG2N>
const void* pass_fn_upto(int log2N) {
  if constexpr (LOG2N < kMinLog2Pass) {
    return nullptr;
  } else {
    if (log2N == LOG2N) return reinterpret_cast<const void*>(&pass_kernel<LOG2N, MODE, SPLIT>);
    return pass_fn_upto<MODE, SPLIT, LOG2N - 1>(log2N);
  }
}

}  // namespace tcfft

#define TCFFT_PASS_UNIT(MODE, SPLIT, NAME)                                               \
  namespace tcfft {                                                                      \
  const void* NAME(int log2N) {                                                          \
    return pass_fn_upto<MODE, SPLIT, max_log2_pass(MODE, SPLIT)>(log2N);                 \
  }                                                                                      \
  }
