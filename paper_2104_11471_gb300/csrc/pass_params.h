// Parameters of one "pass": a batch of DFTs of one length N = R * 16^S that a
// single kernel launch computes entirely on chip (shared memory + TMEM).
// Host code (planner) and device code (pass kernel) both include this file.
#pragma once
#include <cuda.h>  // CUtensorMap

#include <cstdint>

namespace tcfft {

// Transform t of a pass is split into three index levels
//   t1 = t & (I1 - 1), t2 = (t >> log2I1) & (I2 - 1), t3 = t >> (log2I1 + log2I2)
// and its first element sits at t1*s1 + t2*s2 + t3*s3 (complex elements).
// Element e of the transform sits at first + e*es.  A side is "contiguous"
// when es == 1 (then s1 == N: the C transforms of a CTA form one block of
// C*N elements); otherwise it is "strided" (s1 == 1: element e of the CTA's
// C transforms is one run of C adjacent complex values).  The C transforms
// of a CTA never straddle a t1 run (C divides I1).
// With a transform-offset table (toff != null) the t2/t3 part of the first
// element is toff[t >> log2I1] instead: transforms of a ragged batch sit at
// arbitrary 16-byte-aligned offsets of one buffer.  With I1 == 1 on a
// contiguous side every transform of a CTA has its own offset ("gather").
struct SideLayout {
  int64_t s1, s2, s3;
  uint32_t es;
  const int64_t* toff;
};

// Pass modes (input side / output side).
enum PassMode : int {
  kModeContig = 0,    // contiguous in, contiguous out
  kModeStrided = 1,   // strided in, strided out
  kModeToStrided = 2  // contiguous in, strided out
};

struct PassParams {
  const uint32_t* in;   // interleaved FP16 complex (re in low half)
  uint32_t* out;
  int64_t in_plane;     // split precision: element offset of the lo plane
  int64_t out_plane;
  int log2N;            // transform length of the pass (must match the kernel)
  int log2C;            // transforms per CTA
  int tiles;            // 128-butterfly MMA tiles per stage = ceil(C*N/2048)
  int tmem_cols;        // TMEM columns allocated per CTA
  int64_t T;            // transforms in the pass
  int log2I1, log2I2;
  SideLayout in_l, out_l;
  // Epilogue twiddles of radix-16 stages 1..S-1 (stage_twiddle_kernel): one
  // float4 (a, b) per row key, then 8 float4 per key holding its 16
  // twiddles a b^k as packed pairs.
  const float4* stw;
  // W_N table for this pass (factored: W_N^a = hi[a >> log2S] * lo[a & (S-1)])
  const float* tw_lo;   // float2 pairs
  const float* tw_hi;
  int tw_log2S;
  // optional output twiddle W_M^{col * k} of a multi-pass transform; col is
  // t1 (level 1) or t2 (level 2) of the transform, k its output index.
  int otw_level;        // 0 = none
  int otw_log2M;
  int otw_log2S;
  const float* otw_lo;
  const float* otw_hi;
  int conj_in;            // negate imaginary parts on load (first pass of an inverse)
  int conj_out;           // negate imaginary parts of the results (last pass of an inverse)
  float prescale;         // factor on the leading radix-R step (1/R when the pass is scaled)
  // split kernels only: this side is interleaved FP32 complex (8 B per point,
  // one buffer) instead of the hi / lo FP16 planes; offsets stay in points
  int in_f32;
  int out_f32;
  // strided input through the tensor-memory accelerator: one tensor map of
  // the input side (dims t1, element, t2, t3, plane; boxes of C x <= 256
  // elements), encoded at exec time for the bound pointer; 0 = per-thread
  // 16-byte cp.async gathers
  int in_tma;
  // swizzle of the strided input boxes in shared memory (0 none; 1, 2, 3 =
  // 32-, 64-, 128-byte spans matching rows of C = 8, 16, 32 columns): the
  // 16-byte slot index of byte offset b within the raw buffer is XORed with
  // (b >> 7) & (2^in_swz - 1), so the stage-1 reads of a quarter-warp spread
  // over all bank groups
  int in_swz;
  CUtensorMap in_map;  // 128-byte aligned by its type
  // strided output of a two-stage pass (length 256..1024, C in {8, 16, 32})
  // through tensor-map stores: the staging copy is written in the map's swizzle
  // (16-byte chunk XOR 128-byte line, over C * 4-byte rows) and one thread
  // stores C x 256-element boxes per plane; 0 = per-thread 16-byte stores
  int out_tma;
  CUtensorMap out_map;
  int in_gather;          // contiguous input, one offset per transform (see SideLayout)
  int out_scatter;        // contiguous output, one offset per transform
  int async_load;         // 1: prefetch the next chunk with cp.async into a raw buffer
  int64_t nchunks;        // CTA work items: ceil(T / C); CTAs loop over them
  const uint16_t* dft_b;  // radix-16 DFT matrix image(s) in the MMA B layout
  int* status;            // device error word (0 = ok)
};

// A fused 2D pass: S x S matrices, one per cluster of 2^log2K CTAs.  CTA r
// of a cluster transforms rows r*S/K .. (r+1)*S/K - 1 of its matrix (phase 1,
// `row`: contiguous rows read from row.in), hands every row output to the CTA
// that owns its column through distributed shared memory, then transforms
// columns r*S/K .. (r+1)*S/K - 1 (phase 2, `col`: strided output to col.out).
// One read and one write of every matrix in HBM.
struct Fused2DParams {
  PassParams row;
  PassParams col;
  int log2K;      // CTAs per cluster (log2)
  int64_t batch;  // matrices
};

// A persistent launch over a device work queue (ragged batches): items are
// (pass, slot) pairs in dependency order -- slot s of a pass runs its chunks
// s, s + G, ... (G = nchunks[pass] slots); a CTA claims the next item, waits
// (bounded) until every slot of the pass it depends on is done, runs the slot
// and counts it done.  Counters are zero at launch.
struct QueueParams {
  const PassParams* passes;  // per pass, buffers bound (tensor maps encoded)
  const int* dep;            // per pass: the pass that must be complete first, or -1
  const int* nchunks;        // per pass: slots
  const int2* items;         // (pass, slot)
  int nitems;
  int* head;                 // next item to claim
  int* done;                 // per pass: slots completed
  int* abort;                // set once a dependency wait timed out: later items are skipped
  int* status;               // device error word
  long long wait_limit;      // SM clock cycles a dependency wait may take
  int a_bytes;               // operand area of the largest pass (A, raw buffer, DFT images)
  int b_bytes;               // unused (kept 0)
  int tmem_cols;
};

constexpr int kTileRows = 128;        // butterflies per MMA tile (M)
constexpr int kTileBytes = 8192;      // one tile of A: 128 rows x 32 halves
constexpr int kBImageBytes = 2048;    // 32 x 32 halves, K-major, no swizzle
constexpr int kStageSlots = 9;        // float4 entries per epilogue-twiddle key: (a, b) and 8 twiddle pairs
constexpr int kThreads = 256;        // 8 warps: two per TMEM lane quarter
constexpr long long kWaitLimitCycles = 2000000000LL;  // ~1 s at 2 GHz

// Device status codes written by kernels (mirror tcfft_status values).
constexpr int kDevErrTimeout = 5;

// Largest side (log2) of the fused 2D kernels: 2^18 points over at most 16
// CTAs of 16384 points (plain), 2^16 over 16 CTAs of 4096 (split).
constexpr int kMaxLog2Fused2D = 9;
constexpr int kMaxLog2Fused2DSplit = 8;

// Supported pass lengths per mode and precision (log2 N).
constexpr int kMinLog2Pass = 4;
constexpr int max_log2_pass(int mode, bool split) {
  return mode == kModeContig ? 14 : (split ? 11 : 12);
}

}  // namespace tcfft
