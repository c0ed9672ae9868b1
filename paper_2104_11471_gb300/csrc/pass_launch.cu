// Instantiates the fused pass kernel for every leading radix (1, 2, 4, 8)
// and both precisions, and dispatches launches to them.
#include <cuda_runtime.h>

#include "pass_kernel.cuh"

namespace tcfft {

namespace {
template <bool SPLIT>
cudaError_t set_smem(int bytes) {
  cudaError_t e = cudaSuccess, r;
  r = cudaFuncSetAttribute(pass_kernel<1, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (r != cudaSuccess) e = r;
  r = cudaFuncSetAttribute(pass_kernel<2, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (r != cudaSuccess) e = r;
  r = cudaFuncSetAttribute(pass_kernel<4, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (r != cudaSuccess) e = r;
  r = cudaFuncSetAttribute(pass_kernel<8, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (r != cudaSuccess) e = r;
  return e;
}

template <bool SPLIT>
void launch(const PassParams& p, dim3 grid, size_t smem, cudaStream_t s) {
  switch (p.R) {
    case 1: pass_kernel<1, SPLIT><<<grid, kThreads, smem, s>>>(p); break;
    case 2: pass_kernel<2, SPLIT><<<grid, kThreads, smem, s>>>(p); break;
    case 4: pass_kernel<4, SPLIT><<<grid, kThreads, smem, s>>>(p); break;
    default: pass_kernel<8, SPLIT><<<grid, kThreads, smem, s>>>(p); break;
  }
}
}  // namespace

cudaError_t configure_pass_kernel(bool split, size_t smem) {
  const int bytes = (int)(smem > 227 * 1024 ? 227 * 1024 : smem);
  return split ? set_smem<true>(bytes) : set_smem<false>(bytes);
}

cudaError_t launch_pass(const PassParams& p, bool split, dim3 grid, size_t smem, cudaStream_t s) {
  if (split)
    launch<true>(p, grid, smem, s);
  else
    launch<false>(p, grid, smem, s);
  return cudaGetLastError();
}

}  // namespace tcfft
