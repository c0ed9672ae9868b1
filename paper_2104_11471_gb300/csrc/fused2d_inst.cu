// Fused 2D kernels for square matrices of side 2^4 .. 2^9 (plain) and
// 2^4 .. 2^8 (split precision), and their entry-point lookup.
#include "fused2d_kernel.cuh"
#include "pass_setup.h"

namespace tcfft {

namespace {
template <bool SPLIT, int LOG2S>
const void* fused_upto(int log2S) {
  if constexpr (LOG2S < kMinLog2Pass) {
    return nullptr;
  } else {
    if (log2S == LOG2S) return reinterpret_cast<const void*>(&fused2d_kernel<LOG2S, SPLIT>);
    return fused_upto<SPLIT, LOG2S - 1>(log2S);
  }
}
}  // namespace

const void* fused2d_fn(int log2S, bool split) {
  if (log2S < kMinLog2Pass || log2S > (split ? kMaxLog2Fused2DSplit : kMaxLog2Fused2D)) return nullptr;
  return split ? fused_upto<true, kMaxLog2Fused2DSplit>(log2S) : fused_upto<false, kMaxLog2Fused2D>(log2S);
}

}  // namespace tcfft
