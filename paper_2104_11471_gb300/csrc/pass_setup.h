// Launch geometry of one fused pass (shared by the plan-based C ABI and the
// allocation-free entry point): kernel choice, transforms per CTA, MMA tiles,
// TMEM columns, shared memory, CTAs per SM and the persistent grid.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/tcfft.h"
#include "pass_params.h"

namespace tcfft {

// One side (input or output) of a pass, in complex elements (see SideLayout).
struct Side {
  int64_t s1, s2, s3, es;
  const int64_t* toff = nullptr;  // optional transform-offset table (device)
};

struct PassLaunch {
  PassParams p;
  const void* fn = nullptr;  // kernel entry point
  dim3 grid;
  size_t smem = 0;
  int occ = 0;   // CTAs per SM the grid was sized for
  int regs = 0;  // registers per thread of the kernel
  int threads = kThreads;  // threads per CTA (a multiple of 128: one warp per TMEM lane quarter)
};

// Launches one pass kernel on `s` with programmatic stream serialization: its
// CTAs may start their prologue while the previous kernel in the stream
// finishes; the kernel waits (griddepcontrol.wait) before reading its input.
cudaError_t launch_pass(const void* fn, dim3 grid, int threads, size_t smem, cudaStream_t s, void** args);

// Encodes p.in_map for the input pointer bound in p (strided-input passes
// planned with p.in_tma); clears p.in_tma when the map cannot be encoded, and
// the kernel then gathers with per-thread 16-byte copies.  Call after every
// change of p.in, p.T or p.in_plane.
void encode_in_map(PassParams& p, bool split);
// The same for p.out_map (strided-output two-stage passes planned with
// p.out_tma); clears p.out_tma when the map cannot be encoded.
void encode_out_map(PassParams& p, bool split);

int ilog2(int64_t v);
bool is_pow2(int64_t v);
// Integer from the environment (debugging and tuning overrides), or dflt.
int env_int(const char* name, int dflt);
// Kernel entry point for one (length, mode, precision), or null.
const void* pass_fn(int log2N, int mode, bool split);

// Fills the geometry of a pass computing DFTs of length L on T transforms
// indexed by (t1 < I1, t2 < I2, t3) with layouts `in` and `out`, and sets
// the kernel's shared-memory attributes.  Leaves tables, status word,
// buffers, planes and output twiddle to the caller.  Allocates nothing.
// target_points (0 = default) overrides the points per CTA aimed at: the
// transforms-per-CTA target of contiguous passes, the cap of strided ones.
// target_points > 0 asks for that many points per CTA (autotuner);
// force_threads (128 or 256) and force_async (0 or 1) fix the CTA size and
// the load mode instead of the planner's choice.
tcfft_status pass_geometry(PassLaunch& ps, int64_t L, int64_t T, int64_t I1, int64_t I2, Side in,
                           Side out, bool split, int64_t target_points = 0, int force_threads = 0,
                           int force_async = -1, bool share_sm = false);

// ------------------------------------------------------------ fused 2D
// One fused 2D pass (Fused2DParams): S x S matrices, a cluster of 2^log2K
// CTAs per matrix.
struct Fused2DLaunch {
  Fused2DParams f;
  const void* fn = nullptr;
  dim3 grid;
  int threads = kThreads;
  size_t smem = 0;
  int occ = 0;  // CTAs per SM
  int regs = 0;
};

// Kernel entry point of the persistent work-queue executor.
const void* queue_fn();

// Kernel entry point of the fused 2D pass for S = 2^log2S, or null.
const void* fused2d_fn(int log2S, bool split);

// Fills the geometry of a fused 2D pass over `batch` S x S matrices: the
// smallest cluster (2^log2K CTAs, at most 16) whose CTAs hold at most 8192
// points each (4096 split; 16384 plain when 16 CTAs of 8192 do not suffice)
// and at least 8 columns each; tables, buffers and direction flags are left
// to the caller.  TCFFT_ERR_INVALID_SIZE when the matrix does not fit (or
// force_log2K >= 0 names an impossible cluster).
tcfft_status fused2d_geometry(Fused2DLaunch& fl, int64_t S, int64_t batch, bool split, int force_log2K = -1);

// Launches a fused 2D pass (cluster dimension and programmatic stream
// serialization attributes) on `s`.
cudaError_t launch_fused2d(const Fused2DLaunch& fl, const Fused2DParams& f, cudaStream_t s);

}  // namespace tcfft
