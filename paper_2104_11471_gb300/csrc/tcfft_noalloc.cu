// Allocation-free entry point for large batched 1D transforms.
//
// The plan-based path (tcfft_plan_1d + tcfft_exec) allocates its twiddle
// tables, DFT-matrix images, status word and -- for n > 16384 -- a workspace
// that the two passes of the transform exchange data through.  Some callers
// cannot allocate device memory at the time they need a transform: processes
// that reserved their whole device-memory budget up front (a framework's
// caching allocator or a serving process holding a fixed pool), where a
// library allocation would fail or take memory the caller has promised
// elsewhere, and latency-sensitive loops where cudaMalloc / cudaFree may
// synchronise the device.  tcfft_exec_1d_noalloc serves them: the workspace,
// tables and status word live in file-scope __device__ arrays of fixed size,
// loaded with the library and held by every GPU that loads it until exit.
//
// Limits: plain FP16, n a power of two in [2^15, 2^24], n * batch <= 2^24
// points (the 64 MiB workspace below).  Larger requests are rejected with
// TCFFT_ERR_INVALID_SIZE.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/tcfft.h"
#include "pass_params.h"
#include "pass_setup.h"
#include "tables.cuh"

namespace {

constexpr int64_t kNoAllocMaxPoints = int64_t(1) << 24;  // complex FP16 points (64 MiB)
constexpr int kMinLog2 = 15, kMaxLog2 = 24;
constexpr int kTwHalf = 4096;      // float2 entries per half of a factored W table
constexpr int kStageSlot = 4096;   // float4 entries of epilogue twiddles per pass length
constexpr int kMaxDevices = 64;
constexpr int64_t kNoLevel = int64_t(1) << 40;

}  // namespace

// Workspace between the two passes: pass 1 writes all of it that a call
// uses before pass 2 reads it, so nothing needs clearing between calls.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocMaxPoints];
// Factored W_M tables for log2 M = 0..24: [log2 M][lo (kTwHalf) | hi (kTwHalf)].
static __device__ __align__(256) float2 g_noalloc_tw[(kMaxLog2 + 1) * 2 * kTwHalf];
// Epilogue twiddles per pass length log2 L = 0..12.
static __device__ __align__(256) float4 g_noalloc_stage[13 * kStageSlot];
// DFT-matrix images for leading radix 1, 2, 4, 8 (16 images of 1024 halves each).
static __device__ __align__(256) __half g_noalloc_dftb[4 * 16 * 1024];
// Error word the pass kernels require (they write TCFFT_ERR_TIMEOUT into it
// when a bounded wait expires).  Here it is write-only: zeroed once at set-up,
// never read or cleared afterwards, because this entry point has no plan to
// report device-side timeouts through.
static __device__ __align__(256) int g_noalloc_status;

namespace {

struct DeviceTables {
  bool ready = false;
  uint32_t* scratch = nullptr;
  float2* tw = nullptr;
  float4* stage = nullptr;
  __half* dftb = nullptr;
  int* status = nullptr;
};

DeviceTables g_dev[kMaxDevices];
std::mutex g_mu;

template <class T>
tcfft_status symbol_address(T** out, const void* symbol) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, symbol) != cudaSuccess || p == nullptr) return TCFFT_ERR_CUDA;
  *out = static_cast<T*>(p);
  return TCFFT_OK;
}

int stage_rows(int log2N) {
  const int S = log2N / 4, RX = 1 << (log2N % 4);
  int rows = (S >= 2) ? (RX << (4 * (S - 1))) : 0;
  for (int j = 2; j < S; ++j) rows += 1 << (4 * (S - j));
  return rows;
}

// Once per device, with that device current: resolve the device addresses
// of the arrays above and fill the tables.  Synchronises the device.
tcfft_status setup_device(DeviceTables& d) {
  tcfft_status st;
  if ((st = symbol_address(&d.scratch, g_noalloc_scratch)) != TCFFT_OK) return st;
  if ((st = symbol_address(&d.tw, g_noalloc_tw)) != TCFFT_OK) return st;
  if ((st = symbol_address(&d.stage, g_noalloc_stage)) != TCFFT_OK) return st;
  if ((st = symbol_address(&d.dftb, g_noalloc_dftb)) != TCFFT_OK) return st;
  if ((st = symbol_address(&d.status, &g_noalloc_status)) != TCFFT_OK) return st;
  if (cudaMemset(d.status, 0, sizeof(int)) != cudaSuccess) return TCFFT_ERR_CUDA;
  for (int lg = 1; lg <= kMaxLog2; ++lg) {
    const int log2S = (lg + 1) / 2;
    float2* lo = d.tw + (size_t)lg * 2 * kTwHalf;
    const int64_t n = (int64_t(1) << log2S) + (int64_t(1) << (lg - log2S));
    tcfft::twiddle_table_kernel<<<(int)((n + 255) / 256), 256>>>(lo, lo + kTwHalf, lg, log2S);
  }
  for (int lg = tcfft::kMinLog2Pass; lg <= 12; ++lg) {
    const int rows = stage_rows(lg);
    if (rows > 0)  // kStageSlots float4 per key: at most 272 * 9 = 2448 <= kStageSlot for lengths to 2^12
      tcfft::stage_twiddle_kernel<<<(rows * tcfft::kStageSlots + 255) / 256, 256>>>(
          d.stage + (size_t)lg * kStageSlot, lg, rows);
  }
  for (int r = 0; r < 4; ++r) tcfft::dft_b_kernel<<<1 << r, 1024>>>(d.dftb + (size_t)r * 16 * 1024, 1 << r);
  if (cudaGetLastError() != cudaSuccess) return TCFFT_ERR_LAUNCH;
  if (cudaDeviceSynchronize() != cudaSuccess) return TCFFT_ERR_CUDA;
  d.ready = true;
  return TCFFT_OK;
}

// Points pass tables at the arrays above (no allocation).
void bind_tables(const DeviceTables& d, tcfft::PassParams& p, int log2L, int otw_log2M) {
  const int ls = (log2L + 1) / 2;
  p.tw_lo = reinterpret_cast<const float*>(d.tw + (size_t)log2L * 2 * kTwHalf);
  p.tw_hi = reinterpret_cast<const float*>(d.tw + (size_t)log2L * 2 * kTwHalf + kTwHalf);
  p.tw_log2S = ls;
  p.stw = d.stage + (size_t)log2L * kStageSlot;
  p.dft_b = reinterpret_cast<const uint16_t*>(d.dftb + (size_t)(log2L % 4) * 16 * 1024);
  p.otw_level = otw_log2M ? 1 : 0;
  if (otw_log2M) {
    p.otw_log2M = otw_log2M;
    p.otw_log2S = (otw_log2M + 1) / 2;
    p.otw_lo = reinterpret_cast<const float*>(d.tw + (size_t)otw_log2M * 2 * kTwHalf);
    p.otw_hi = reinterpret_cast<const float*>(d.tw + (size_t)otw_log2M * 2 * kTwHalf + kTwHalf);
  }
  p.status = d.status;
}

}  // namespace

extern "C" tcfft_status tcfft_exec_1d_noalloc(int64_t n, int64_t batch, const void* in, void* out,
                                              void* stream) {
  if (!in || !out) return TCFFT_ERR_INVALID_VALUE;
  if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
    return TCFFT_ERR_INVALID_VALUE;
  if (!tcfft::is_pow2(n) || n < (int64_t(1) << kMinLog2) || n > (int64_t(1) << kMaxLog2) || batch < 1 ||
      batch > kNoAllocMaxPoints / n)
    return TCFFT_ERR_INVALID_SIZE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TCFFT_ERR_UNSUPPORTED;
  cudaDeviceProp prop;
  DeviceTables& d = g_dev[dev];
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!d.ready) {
      if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return TCFFT_ERR_UNSUPPORTED;
      if (prop.major != 10 || prop.minor != 3) return TCFFT_ERR_UNSUPPORTED;
      const tcfft_status st = setup_device(d);
      if (st != TCFFT_OK) return st;
    }
  }
  // n = N1 N2: pass 1 = N1-point DFTs of the columns x[N2 n1 + n2] times
  // W_n^{n2 k1}, into the workspace; pass 2 = N2-point DFTs of the rows,
  // written to X[k1 + N1 k2] (the same split as the plan-based path).
  const int lg = tcfft::ilog2(n);
  const int64_t N1 = int64_t(1) << ((lg + 1) / 2), N2 = n / N1;
  tcfft::PassLaunch ps[2];
  const tcfft::Side c1{1, n, 0, N2};
  tcfft_status st = tcfft::pass_geometry(ps[0], N1, batch * N2, N2, kNoLevel, c1, c1, false);
  if (st != TCFFT_OK) return st;
  const tcfft::Side in2{N2, n, 0, 1}, out2{1, n, 0, N1};
  st = tcfft::pass_geometry(ps[1], N2, batch * N1, N1, kNoLevel, in2, out2, false);
  if (st != TCFFT_OK) return st;
  bind_tables(d, ps[0].p, tcfft::ilog2(N1), lg);
  bind_tables(d, ps[1].p, tcfft::ilog2(N2), 0);
  ps[0].p.in = static_cast<const uint32_t*>(in);
  ps[0].p.out = d.scratch;
  ps[1].p.in = d.scratch;
  ps[1].p.out = static_cast<uint32_t*>(out);
  tcfft::encode_in_map(ps[0].p, false);
  tcfft::encode_in_map(ps[1].p, false);
  tcfft::encode_out_map(ps[0].p, false);
  tcfft::encode_out_map(ps[1].p, false);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int i = 0; i < 2; ++i) {
    void* args[1] = {&ps[i].p};
    if (tcfft::launch_pass(ps[i].fn, ps[i].grid, ps[i].threads, ps[i].smem, s, args) != cudaSuccess)
      return TCFFT_ERR_LAUNCH;
  }
  return TCFFT_OK;
}
