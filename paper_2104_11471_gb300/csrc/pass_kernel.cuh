// The fused pass kernel: one CTA computes C complete DFTs of length
// N = R * 16^S on chip.
//
// Method (arXiv 2104.11471, Sec. 2.1 and 3.2).  A length-L DFT, L = 16^S, is
// computed by S merging processes of radix 16, Eq. (dft_mm):
//     X_out = F_16 . (T (.) X_in),
// written here in the equivalent "twiddle after the butterfly" order.  With
// input index n = n_1 16^{S-1} + n^(2) (n_1 the most significant base-16
// digit) stage 1 forms, for every n^(2),
//     Y[k_1][n^(2)] = W_L^{k_1 n^(2)} sum_{n_1} x[n_1 16^{S-1} + n^(2)] W_16^{n_1 k_1}
// and stage j repeats this on the length-16^{S-j+1} sub-sequences, so that
// after stage S the output index is k = k_1 + 16 k_2 + ... + 16^{S-1} k_S.
// A leading radix-R step (R in {1,2,4,8}, Sec. 3.1 "radix 2 and radix 4 on
// CUDA cores") splits N = R L the same way before the first radix-16 stage:
// sub-transform k0 gets y_k0[n'] = W_N^{k0 n'} sum_{n0} x[n0 L + n'] W_R^{n0 k0}
// and X[k0 + R k'] = DFT_L(y_k0)[k'].
//
// GB300 mapping.
//  * Every radix-16 butterfly column is one row of an MMA A operand:
//    16 complex inputs stored as 32 halves, K = [re_0..re_15 | im_0..im_15].
//    B is the real 32 x 32 form of F_16:
//        [Re out | Im out] = [Re in | Im in] . [[Fr, Fi], [-Fi, Fr]].
//    One tcgen05.mma (M = 128 butterflies, N = 32, K = 16) per K half, FP16
//    operands, FP32 accumulation in TMEM.  The whole stage of all C
//    transforms is issued at once; its FP32 result (<= 512 columns) stays in
//    TMEM until the epilogue has consumed it, so A is rewritten in place.
//  * A is MN-major with the 128-byte swizzle.  The epilogue thread that owns
//    one butterfly holds its 16 outputs k_j; in the next stage those are 16
//    consecutive rows (k_j is the fastest row digit there) at one K, so the
//    thread writes them as four 16-byte vector stores (re lo/hi, im lo/hi).
//  * The twiddle W_{L_j}^{k_j n^(j+1)} is applied in FP32 registers between
//    tcgen05.ld and the FP16 conversion (the paper does it in FP16 on the
//    fragments, Alg. 2); the 16 factors of one thread are powers of one
//    base read from a factored FP32 table generated in FP64.
//  * The final stage writes natural-order results into a swizzled staging
//    copy in shared memory, which is then stored with 16-byte coalesced
//    writes ("continuous size", Sec. 4.2, Table gbw).
//  * Sizes, radices and layouts are template parameters: all index
//    arithmetic is shifts and masks on 32-bit offsets from per-CTA bases.
// Split precision (hi + 2^-11 lo, FP32 accumulation, three products per
// stage) follows the paper's "precision recovery" future work (Sec. 7).
#pragma once
#include <cuda_fp16.h>
#include <cstdint>

#include "pass_params.h"
#include "tc_ptx.cuh"

namespace tcfft {

template <int LOG2N_, int MODE, bool SPLIT_>
struct PassCfg {
  static constexpr int S = LOG2N_ / 4;         // radix-16 stages
  static constexpr int LOG2RX = LOG2N_ % 4;     // leading radix on CUDA cores
  static constexpr int RX = 1 << LOG2RX;
  static constexpr int LOG2N = LOG2N_;
  static constexpr int N = 1 << LOG2N;
  static constexpr int LOG2L = 4 * S;          // radix-16 sub-transform length
  static constexpr int L = 1 << LOG2L;
  static constexpr int LOG2LQ = 4 * (S - 1);   // 16^{S-1}
  static constexpr int LQ = 1 << LOG2LQ;
  static constexpr bool IN_C = MODE != kModeStrided;
  static constexpr bool OUT_C = MODE == kModeContig;
  static constexpr bool SPLIT = SPLIT_;
  static constexpr int PLANES = SPLIT ? 2 : 1;
  // With two or more radix-16 stages the leading radix-RX twiddle W_N^{k0 n'}
  // is folded out of the load: its factor W_{16 RX}^{k0 n_1} goes into a
  // per-k0 copy of the stage-1 DFT matrix (every MMA tile then holds one k0)
  // and its factor W_N^{k0 n^(2)} into the stage-1 epilogue twiddle.
  static constexpr bool FOLD = S >= 2 && RX > 1;
  // final outputs go straight to global memory when the lanes of a warp hold
  // consecutive output indices (two radix-16 stages, no leading radix,
  // contiguous output)
  static constexpr bool DIRECT_OUT = OUT_C && S == 2 && RX == 1;
  // keys of the epilogue-twiddle table: RX 16^{S-1} for stage 1, then
  // 16^{S-j} for stage j = 2..S-1
  static constexpr int STAGE_KEYS = S >= 2 ? RX * LQ + (S == 3 ? 16 : 0) : 0;
  // CTAs per SM the register budget is sized for (the kernel is latency-bound:
  // more resident warps hide the TMEM, barrier and memory waits).  Plain
  // lengths fit 80 registers (3 CTAs of 256 threads) without spills except
  // those with a radix-8 leading step or a single radix-16 stage after a
  // radix 2/4 step, which keep 2.  Split kernels keep their full register
  // budget (a 128-register cap measured slower: more 128-thread CTAs of the
  // unconstrained kernel win).
  static constexpr int MINB = SPLIT ? 1 : ((LOG2N_ % 4 == 3 || (LOG2N_ > 4 && LOG2N_ < 8)) ? 2 : 3);
  static_assert(S >= 1 && S <= 3, "pass length out of range");
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Byte offset of A element (m, k): m = butterfly row in [0, tiles*128),
// k in [0, 32).  MN-major, 128-byte swizzle: per 8 KB tile two M-atoms of 64
// rows (4096 B apart); each holds four K-atoms (8 k-rows of 128 B, 1024 B
// apart); 16-byte chunk index XOR (k mod 8).
__device__ __forceinline__ uint32_t a_off(uint32_t m, uint32_t k) {
  const uint32_t mm = m & 127u;
  return (m >> 7) * kTileBytes + ((mm >> 6) << 12) + ((k >> 3) << 10) + ((k & 7u) << 7) +
         ((((mm & 63u) >> 3) ^ (k & 7u)) << 4) + ((mm & 7u) << 1);
}

// MMA row order.  Logical row r (a butterfly's identity at the current
// stage) sits at physical row (TMEM lane, A row) rp(r) = r ^ (bit 6 of r) << 3,
// an involution that swaps the two 8-row groups of each 16-row block in the
// upper half of every 128-row tile.  Writers whose lanes fill consecutive
// 16-row blocks at one K (the epilogues, the strided stage-1 load) then put
// the first 8-row chunk of lanes 0-3 and of lanes 4-7 of a quarter-warp in
// 16-byte slots of opposite parity: all eight 16-byte stores of a
// quarter-warp land in distinct bank groups instead of two-way conflicts.
// Tiles (rows >> 7) are unchanged, so per-tile DFT matrices still apply.
__device__ __forceinline__ uint32_t rp(uint32_t r) { return r ^ (((r >> 6) & 1u) << 3); }

__device__ __forceinline__ int64_t side_base(const SideLayout& l, int64_t t, int log2I1,
                                             int log2I2) {
  const int64_t t1 = t & ((int64_t(1) << log2I1) - 1);
  const int64_t t23 = t >> log2I1;
  if (l.toff) return t1 * l.s1 + __ldg(l.toff + t23);
  const int64_t t2 = t23 & ((int64_t(1) << log2I2) - 1);
  const int64_t t3 = t23 >> log2I2;
  return t1 * l.s1 + t2 * l.s2 + t3 * l.s3;
}

__device__ __forceinline__ float2 tw_lookup(const float* lo, const float* hi, uint32_t a,
                                            int log2M, int log2S) {
  a &= (1u << log2M) - 1u;
  const float2 h = __ldg(reinterpret_cast<const float2*>(hi) + (a >> log2S));
  const float2 l = __ldg(reinterpret_cast<const float2*>(lo) + (a & ((1u << log2S) - 1u)));
  return cmulf(h, l);
}

__device__ __forceinline__ float2 h2f(uint32_t u) {
  __half2 h = *reinterpret_cast<__half2*>(&u);
  return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2h2(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
// low part of the split pair: fp16((v - fp16(v)) * 2^11), per component
__device__ __forceinline__ uint32_t split_lo(float a, float b, uint32_t hi) {
  const float2 hf = h2f(hi);
  return f2h2((a - hf.x) * 2048.0f, (b - hf.y) * 2048.0f);
}

// In-place DFT of length RX (1, 2, 4, 8) on FP32 complex values.
template <int RX>
__device__ __forceinline__ void small_dft(float2 (&v)[RX]) {
  if constexpr (RX == 2) {
    float2 a = v[0], b = v[1];
    v[0] = make_float2(a.x + b.x, a.y + b.y);
    v[1] = make_float2(a.x - b.x, a.y - b.y);
  } else if constexpr (RX == 4) {
    // y_k = sum_n x_n W_4^{nk}, W_4 = -i
    float2 s02 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
    float2 d02 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
    float2 s13 = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
    float2 d13 = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);
    v[0] = make_float2(s02.x + s13.x, s02.y + s13.y);
    v[2] = make_float2(s02.x - s13.x, s02.y - s13.y);
    v[1] = make_float2(d02.x + d13.y, d02.y - d13.x);  // d02 - i d13
    v[3] = make_float2(d02.x - d13.y, d02.y + d13.x);  // d02 + i d13
  } else if constexpr (RX == 8) {
    // radix-2 split of a length-8 DFT: two length-4 DFTs on even/odd inputs
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    small_dft<4>(e);
    small_dft<4>(o);
    const float h = 0.70710678118654752f;
    // W_8^k for k = 0..3: 1, (1-i)/sqrt2, -i, (-1-i)/sqrt2
    const float2 t0 = o[0], t1 = cmulf(o[1], make_float2(h, -h)), t2 = make_float2(o[2].y, -o[2].x),
                 t3 = cmulf(o[3], make_float2(-h, -h));
    v[0] = make_float2(e[0].x + t0.x, e[0].y + t0.y);
    v[4] = make_float2(e[0].x - t0.x, e[0].y - t0.y);
    v[1] = make_float2(e[1].x + t1.x, e[1].y + t1.y);
    v[5] = make_float2(e[1].x - t1.x, e[1].y - t1.y);
    v[2] = make_float2(e[2].x + t2.x, e[2].y + t2.y);
    v[6] = make_float2(e[2].x - t2.x, e[2].y - t2.y);
    v[3] = make_float2(e[3].x + t3.x, e[3].y + t3.y);
    v[7] = make_float2(e[3].x - t3.x, e[3].y - t3.y);
  }
}

// Writes 8 consecutive logical butterfly rows (m0 multiple of 8) of input k
// of A from 8 packed complex values: re halves at K = k, im halves at K = 16 + k.
__device__ __forceinline__ void a_store8c(uint8_t* A, uint32_t m0, uint32_t k,
                                          const uint32_t (&v)[8]) {
  m0 = rp(m0);
  const uint4 re = make_uint4(__byte_perm(v[0], v[1], 0x5410), __byte_perm(v[2], v[3], 0x5410),
                              __byte_perm(v[4], v[5], 0x5410), __byte_perm(v[6], v[7], 0x5410));
  const uint4 im = make_uint4(__byte_perm(v[0], v[1], 0x7632), __byte_perm(v[2], v[3], 0x7632),
                              __byte_perm(v[4], v[5], 0x7632), __byte_perm(v[6], v[7], 0x7632));
  // K = 16 + k lies two K-atoms (2048 bytes) after K = k, same swizzle phase
  uint8_t* a = A + a_off(m0, k);
  *reinterpret_cast<uint4*>(a) = re;
  *reinterpret_cast<uint4*>(a + 2048) = im;
}

// Staging-buffer swizzle for the final stage.  Output word (c, ko) of the
// chunk lives at logical index c*N + ko (contiguous output) or ko*C + c
// (strided output); its 16-byte chunk index inside each 128-byte line is
// XORed with a key.  The key depends only on c and on ko bits below the
// k_S digit (so one thread's 16 words share it), is constant inside a line
// (so the XOR permutes whole chunks within their line), and is taken from
// the digit that differs between the lanes of a warp, so the single-word
// writes of one warp spread over the shared-memory banks.
template <class K>
__device__ __forceinline__ uint32_t stg_key(uint32_t c, uint32_t ko, int log2C) {
  constexpr int KSLO = K::LOG2RX + 4 * (K::S - 1);  // lowest bit of the k_S digit in ko
  ko &= (1u << KSLO) - 1u;
  if constexpr (K::OUT_C) {
    constexpr int LANE = (K::S >= 2) ? (K::LOG2RX + 4 * (K::S - 2)) : 0;
    constexpr int KS = LANE > 5 ? LANE : 5;
    constexpr int W = (KSLO - KS) < 3 ? (KSLO - KS) : 3;
    if constexpr (K::S >= 2 && W > 0) {
      return (ko >> KS) & ((1u << W) - 1u);
    } else {
      constexpr int CS = K::LOG2N >= 5 ? 0 : 5 - K::LOG2N;
      return (c >> CS) & 7u;
    }
  } else {
    if constexpr (K::S == 1) {
      return 0u;
    } else {
      constexpr int LANE = K::LOG2RX + 4 * (K::S - 2);
      const int line_min = log2C >= 5 ? 0 : 5 - log2C;
      const int ks = LANE > line_min ? LANE : line_min;
      const int w = (KSLO - ks) < 3 ? (KSLO - ks) : 3;
      return w > 0 ? ((ko >> ks) & ((1u << w) - 1u)) : 0u;
    }
  }
}

// 32-bit words per point on a side: 2 for interleaved FP32 complex (split
// kernels with in_f32 / out_f32), else 1 (FP16 complex or one FP16 plane)
template <class K>
__device__ __forceinline__ uint32_t in_words(const PassParams& p) {
  return (K::SPLIT && p.in_f32) ? 2u : 1u;
}
template <class K>
__device__ __forceinline__ uint32_t out_words(const PassParams& p) {
  return (K::SPLIT && p.out_f32) ? 2u : 1u;
}

// ------------------------------------------------------------------ loads
__device__ __forceinline__ void cp_async16(uint32_t dst_smem, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst_smem), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Issues the asynchronous copy of one chunk (C transforms) into the raw
// buffer, keeping the global element order: contiguous input -> raw[c*N + e]
// (one bulk copy per plane, completion on `lbar`), strided input ->
// raw[e*C + c] (16-byte cp.async per thread).  Transforms past the end of
// the batch are not copied: their rows only feed outputs that are dropped.
template <class K>
__device__ __forceinline__ void issue_raw_copy(const PassParams& p, uint32_t raw_s, uint32_t lbar,
                                               const uint32_t* gin, int64_t t0, int log2C, int nvalid,
                                               const PassParams* maps = nullptr) {
  const CUtensorMap* in_map = maps ? &maps->in_map : &p.in_map;  // param or global memory
  const uint32_t P = (uint32_t)1 << (log2C + K::LOG2N);
  if constexpr (K::IN_C) {
    if (!p.in_gather) {
      if (threadIdx.x == 0) {
        const uint32_t bytes = ((uint32_t)nvalid << K::LOG2N) * 4u;
        mbar_arrive_expect_tx(lbar, bytes * K::PLANES);
        if (K::SPLIT && p.in_f32) {
          bulk_g2s(raw_s, gin, bytes * 2u, lbar);  // FP32 complex: raw[c*N + e] at 8 B per point
        } else {
          bulk_g2s(raw_s, gin, bytes, lbar);
          if constexpr (K::SPLIT) bulk_g2s(raw_s + P * 4u, gin + p.in_plane, bytes, lbar);
        }
      }
    } else if (threadIdx.x < 32) {
      // one bulk copy per transform, from its own offset (ragged batches)
      const uint32_t bytes = (uint32_t)K::N * 4u;
      if (threadIdx.x == 0) mbar_arrive_expect_tx(lbar, bytes * K::PLANES * (uint32_t)nvalid);
      __syncwarp();
      for (int c = threadIdx.x; c < nvalid; c += 32) {
        const uint32_t* src = p.in + in_words<K>(p) * side_base(p.in_l, t0 + c, p.log2I1, p.log2I2);
        if (K::SPLIT && p.in_f32) {
          bulk_g2s(raw_s + (uint32_t)c * bytes * 2u, src, bytes * 2u, lbar);
        } else {
          bulk_g2s(raw_s + (uint32_t)c * bytes, src, bytes, lbar);
          if constexpr (K::SPLIT) bulk_g2s(raw_s + P * 4u + (uint32_t)c * bytes, src + p.in_plane, bytes, lbar);
        }
      }
    }
  } else if (p.in_tma) {
    // tensor-map boxes of C columns x up to 256 elements per plane, issued by
    // one thread; completion on `lbar` like the contiguous copies
    if (threadIdx.x == 0) {
      const uint32_t wpp = in_words<K>(p);  // 32-bit words per point of a plane
      const uint32_t planes = (K::SPLIT && !p.in_f32) ? 2u : 1u;
      mbar_arrive_expect_tx(lbar, P * 4u * wpp * planes);
      const int bl = K::N < 256 ? K::N : 256;
      const int64_t t1 = t0 & ((int64_t(1) << p.log2I1) - 1);
      const int64_t t23 = t0 >> p.log2I1;
      const int t2 = (int)(t23 & ((int64_t(1) << p.log2I2) - 1));
      const int t3 = (int)(t23 >> p.log2I2);
      for (uint32_t pl = 0; pl < planes; ++pl)
        for (int e0 = 0; e0 < K::N; e0 += bl)
          tma_load_5d(raw_s + pl * (P * 4u) + (uint32_t)e0 * ((uint32_t)1 << log2C) * 4u * wpp, in_map,
                      (int)t1, e0, t2, t3, (int)pl, lbar);
    }
  } else if (K::SPLIT && p.in_f32) {
    // FP32 complex: 16-byte copies of two adjacent columns, raw[e*C + c] at 8 B per point
    const uint32_t nq = P >> 1;
    const int cq = log2C - 1;
    for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
      const uint32_t off = (q >> cq) * p.in_l.es + ((q & ((1u << cq) - 1u)) << 1);
      cp_async16(raw_s + (q << 4), gin + 2u * off, 16);
    }
    cp_async_commit();
  } else {
    const uint32_t nq = P >> 2;  // 16-byte chunks per plane
    const int cq = log2C - 2;
#pragma unroll 1
    for (int pl = 0; pl < K::PLANES; ++pl) {
      const uint32_t* g = gin + (pl ? p.in_plane : 0);
      const uint32_t dst0 = raw_s + pl * (P * 4u);
      for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
        const uint32_t off = (q >> cq) * p.in_l.es + ((q & ((1u << cq) - 1u)) << 2);
        cp_async16(dst0 + (q << 4), g + off, 16);
      }
    }
    cp_async_commit();
  }
}

// Reads the CTA's C transforms, applies the leading radix-RX step (if any)
// and writes the stage-1 A operand(s).  Sub-transform g = k0*C + c.
//   contiguous input: stage-1 row g*16^{S-1} + n^(2)
//   strided input:    stage-1 row (k0*16^{S-1} + n^(2))*C + c
// (k0 is the slowest row digit, so with FOLD every 128-row tile has one k0).
// Without FOLD (one radix-16 stage) the twiddle W_N^{k0 n'} is applied here.
// Source: global memory (SMEM = false; element e of transform c at
// c*N + e or c + e*es) or the raw shared buffer (SMEM = true; es = C).
// CG: global loads through L2 only (ld.global.cg), for inputs that other CTAs
// of the same launch wrote (the non-coherent read-only path could return
// stale lines then).
template <class K, bool SMEM, bool CG = false>
__device__ __forceinline__ void load_stage1(const PassParams& p, uint8_t* A, const uint32_t* src,
                                            const uint32_t* src_lo, uint32_t es, int log2C,
                                            int nvalid, int64_t t0 = 0) {
  constexpr int RX = K::RX;
  uint8_t* Alo = A + p.tiles * kTileBytes;
  const int C = 1 << log2C;
  // items: 8 points (contiguous: of one transform; strided: of 8 transforms)
  constexpr int BLOG = K::LOG2L - 3;
  const int items = K::IN_C ? (C << BLOG) : (K::L << (log2C - 3));
  for (int it = threadIdx.x; it < items; it += (int)blockDim.x) {
    int c, np;  // transform (first of 8 when strided), point n' in [0, L)
    uint32_t off0, step;
    bool valid = true;
    if constexpr (K::IN_C) {
      c = it >> BLOG;
      np = (it & ((1 << BLOG) - 1)) << 3;
      off0 = ((uint32_t)c << K::LOG2N) + np;
      step = K::L;
      if constexpr (!SMEM) {
        valid = c < nvalid;
        if (p.in_gather && valid) {
          // ragged batch read from global memory: transform c has its own offset
          src = p.in + in_words<K>(p) * side_base(p.in_l, t0 + c, p.log2I1, p.log2I2);
          src_lo = src + p.in_plane;
          off0 = np;
        }
      }
    } else {
      const int cbm = (1 << (log2C - 3)) - 1;
      c = (it & cbm) << 3;
      np = it >> (log2C - 3);
      off0 = (uint32_t)c + (uint32_t)np * es;
      step = (uint32_t)K::L * es;
    }
    uint32_t hv[RX][8], lv[RX][8];
    if (K::SPLIT && p.in_f32) {
      // interleaved FP32 complex (shared or global memory, 8 B per point):
      // split each value into hi = fp16(v), lo = fp16((v - hi) 2^11)
      const float* srcf = reinterpret_cast<const float*>(src);
#pragma unroll
      for (int n0 = 0; n0 < RX; ++n0) {
        const float4* f4 = reinterpret_cast<const float4*>(srcf + 2u * (off0 + n0 * step));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float4 f = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          if constexpr (SMEM) {
            f = f4[q];
          } else if (valid) {
            f = CG ? __ldcg(f4 + q) : __ldg(f4 + q);
          }
          hv[n0][2 * q] = f2h2(f.x, f.y);
          lv[n0][2 * q] = split_lo(f.x, f.y, hv[n0][2 * q]);
          hv[n0][2 * q + 1] = f2h2(f.z, f.w);
          lv[n0][2 * q + 1] = split_lo(f.z, f.w, hv[n0][2 * q + 1]);
        }
      }
    } else {
    // strided raw buffer written by swizzled tensor-map boxes: 16-byte slot
    // index XOR (byte offset >> 7) & swm (swm = 0: plain layout)
    const uint32_t swm = (SMEM && !K::IN_C) ? ((1u << p.in_swz) - 1u) : 0u;
#pragma unroll
    for (int n0 = 0; n0 < RX; ++n0) {
      uint4 a = make_uint4(0, 0, 0, 0), b = a;
      const uint4* s4 = reinterpret_cast<const uint4*>(src + off0 + n0 * step);
      if constexpr (SMEM) {
        if constexpr (!K::IN_C) {
          uint32_t bo = (off0 + n0 * step) << 2;
          bo ^= ((bo >> 7) & swm) << 4;
          a = *reinterpret_cast<const uint4*>(reinterpret_cast<const uint8_t*>(src) + bo);
          b = *reinterpret_cast<const uint4*>(reinterpret_cast<const uint8_t*>(src) + (bo ^ 16u));
        } else {
          a = s4[0];
          b = s4[1];
        }
      } else if (valid) {
        a = CG ? __ldcg(s4) : __ldg(s4);
        b = CG ? __ldcg(s4 + 1) : __ldg(s4 + 1);
      }
      hv[n0][0] = a.x; hv[n0][1] = a.y; hv[n0][2] = a.z; hv[n0][3] = a.w;
      hv[n0][4] = b.x; hv[n0][5] = b.y; hv[n0][6] = b.z; hv[n0][7] = b.w;
      if constexpr (K::SPLIT) {
        uint4 c2 = make_uint4(0, 0, 0, 0), d = c2;
        const uint4* l4 = reinterpret_cast<const uint4*>(src_lo + off0 + n0 * step);
        if constexpr (SMEM) {
          if constexpr (!K::IN_C) {
            uint32_t bo = (off0 + n0 * step) << 2;
            bo ^= ((bo >> 7) & swm) << 4;
            c2 = *reinterpret_cast<const uint4*>(reinterpret_cast<const uint8_t*>(src_lo) + bo);
            d = *reinterpret_cast<const uint4*>(reinterpret_cast<const uint8_t*>(src_lo) + (bo ^ 16u));
          } else {
            c2 = l4[0];
            d = l4[1];
          }
        } else if (valid) {
          c2 = CG ? __ldcg(l4) : __ldg(l4);
          d = CG ? __ldcg(l4 + 1) : __ldg(l4 + 1);
        }
        lv[n0][0] = c2.x; lv[n0][1] = c2.y; lv[n0][2] = c2.z; lv[n0][3] = c2.w;
        lv[n0][4] = d.x; lv[n0][5] = d.y; lv[n0][6] = d.z; lv[n0][7] = d.w;
      }
    }
    }
    if (p.conj_in) {
      // inverse transform: conj(x) on the way in (sign bit of each imaginary half)
#pragma unroll
      for (int n0 = 0; n0 < RX; ++n0)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          hv[n0][i] ^= 0x80000000u;
          if constexpr (K::SPLIT) lv[n0][i] ^= 0x80000000u;
        }
    }
    if constexpr (RX > 1) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float2 v[RX];
#pragma unroll
        for (int n0 = 0; n0 < RX; ++n0) {
          v[n0] = h2f(hv[n0][i]);
          if constexpr (K::SPLIT) {
            const float2 l = h2f(lv[n0][i]);
            v[n0].x = fmaf(l.x, 1.0f / 2048.0f, v[n0].x);
            v[n0].y = fmaf(l.y, 1.0f / 2048.0f, v[n0].y);
          }
        }
        small_dft<RX>(v);
        if (p.prescale != 1.0f) {
#pragma unroll
          for (int k0 = 0; k0 < RX; ++k0) v[k0] = make_float2(v[k0].x * p.prescale, v[k0].y * p.prescale);
        }
        const uint32_t npi = K::IN_C ? (uint32_t)(np + i) : (uint32_t)np;
#pragma unroll
        for (int k0 = 0; k0 < RX; ++k0) {
          float2 y = v[k0];
          if (!K::FOLD && k0)
            y = cmulf(y, tw_lookup(p.tw_lo, p.tw_hi, (uint32_t)k0 * npi, K::LOG2N, p.tw_log2S));
          hv[k0][i] = f2h2(y.x, y.y);
          if constexpr (K::SPLIT) lv[k0][i] = split_lo(y.x, y.y, hv[k0][i]);
        }
      }
    }
    if constexpr (K::IN_C) {
#pragma unroll
      for (int k0 = 0; k0 < RX; ++k0) {
        const uint32_t g = ((uint32_t)k0 << log2C) + c;
        if constexpr (K::LQ >= 8) {
          const uint32_t m0 = (g << K::LOG2LQ) + (np & (K::LQ - 1));
          const uint32_t n1 = (uint32_t)np >> K::LOG2LQ;
          a_store8c(A, m0, n1, hv[k0]);
          if constexpr (K::SPLIT) a_store8c(Alo, m0, n1, lv[k0]);
        } else {
          // S == 1: the 8 points are 8 different inputs of butterfly row g
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const uint32_t k = (uint32_t)(np + i);
            const uint32_t gp = rp(g);
            *reinterpret_cast<uint16_t*>(A + a_off(gp, k)) = (uint16_t)(hv[k0][i] & 0xFFFFu);
            *reinterpret_cast<uint16_t*>(A + a_off(gp, 16 + k)) = (uint16_t)(hv[k0][i] >> 16);
            if constexpr (K::SPLIT) {
              *reinterpret_cast<uint16_t*>(Alo + a_off(gp, k)) = (uint16_t)(lv[k0][i] & 0xFFFFu);
              *reinterpret_cast<uint16_t*>(Alo + a_off(gp, 16 + k)) = (uint16_t)(lv[k0][i] >> 16);
            }
          }
        }
      }
    } else {
      const uint32_t n1 = (uint32_t)np >> K::LOG2LQ;
      const uint32_t nrest = (uint32_t)np & (K::LQ - 1);
#pragma unroll
      for (int k0 = 0; k0 < RX; ++k0) {
        const uint32_t m0 = ((((uint32_t)k0 << K::LOG2LQ) + nrest) << log2C) + c;
        a_store8c(A, m0, n1, hv[k0]);
        if constexpr (K::SPLIT) a_store8c(Alo, m0, n1, lv[k0]);
      }
    }
  }
}

// ---------------------------------------------------------------- epilogue
// Packed FP32x2 complex multiply of two adjacent outputs by their twiddles:
// (x + i y) (c + i d) = (x c - y d) + i (x d + y c), with nd = -d.
__device__ __forceinline__ void cmul2(float2& x, float2& y, float2 c, float2 d, float2 nd) {
  const float2 xr = __ffma2_rn(y, nd, __fmul2_rn(x, c));
  const float2 xi = __ffma2_rn(y, c, __fmul2_rn(x, d));
  x = xr;
  y = xi;
}

// Byte offsets of the four 16-byte chunks a thread writes for one butterfly
// (16 consecutive logical rows m0..m0+15 at input k of the next stage): re/im
// halves of rows m0..m0+7 and m0+8..m0+15.  m0 is a multiple of 16; the two
// 8-row groups sit in adjacent 16-byte slots (slot index ^ 1) whichever of
// them rp() puts first.
struct RowChunks {
  uint32_t re0, re1;  // im chunks are 2048 bytes further (K + 16)
};
__device__ __forceinline__ RowChunks row_chunks(uint32_t m0, uint32_t k) {
  RowChunks r;
  r.re0 = a_off(rp(m0), k);
  r.re1 = r.re0 ^ 16u;
  return r;
}

// Final-stage outputs of one butterfly into the natural-order staging copy
// at A (P points per plane): word c*N + k (contiguous output) or k*C + c
// (strided output), XORed with the bank-spreading key, or with the tensor
// map's swizzle when the chunk leaves through tensor-map stores.
template <class K>
__device__ __forceinline__ void staging_store(const PassParams& p, uint8_t* A, uint32_t P, int log2C, uint32_t c,
                                              uint32_t kbase, const float2 (&X)[8], const float2 (&Y)[8]) {
  constexpr uint32_t kstep = (uint32_t)K::LQ << K::LOG2RX;  // output index step per k_S
  uint32_t* stg = reinterpret_cast<uint32_t*>(A);
  const uint32_t base = K::OUT_C ? ((c << K::LOG2N) + kbase) : ((kbase << log2C) + c);
  // bank-spreading key; for tensor-map stores the map's swizzle (the
  // 16-byte chunk index XOR the 128-byte line index, over rows of
  // C * 4 bytes), which is constant over a thread's 16 words here
  uint32_t key = stg_key<K>(c, kbase, log2C) << 2;
  if constexpr (K::OUT_C) {
    if (K::S == 3 && p.out_tma) key = ((base >> 5) & 7u) << 2;  // rows of 32 points
  } else {
    if (p.out_tma) key = ((base >> 5) & ((1u << (log2C - 2)) - 1u)) << 2;
  }
  const uint32_t wstep = K::OUT_C ? kstep : (kstep << log2C);
  // The key changes bits 2..4 of the word index only, so with a step that is
  // a multiple of 32 words (base + n step) ^ key = (base ^ key) + n step: the
  // 16 stores then share one address and differ by constant offsets.  Taken
  // where the step is a compile-time constant (contiguous output) and for
  // the strided output of 256-point passes (step 16 C); for 512- and
  // 1024-point passes with their run-time step it measured slower.
  auto put = [&](uint32_t* s0, auto idx) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t i0 = idx(2 * i), i1 = idx(2 * i + 1);
      if (K::SPLIT && p.out_f32) {
        // FP32 output: the two staging planes hold re and im
        s0[i0] = __float_as_uint(X[i].x);
        s0[i1] = __float_as_uint(X[i].y);
        s0[P + i0] = __float_as_uint(Y[i].x);
        s0[P + i1] = __float_as_uint(Y[i].y);
        continue;
      }
      const uint32_t h0 = f2h2(X[i].x, Y[i].x), h1 = f2h2(X[i].y, Y[i].y);
      s0[i0] = h0;
      s0[i1] = h1;
      if constexpr (K::SPLIT) {
        s0[P + i0] = split_lo(X[i].x, Y[i].x, h0);
        s0[P + i1] = split_lo(X[i].y, Y[i].y, h1);
      }
    }
  };
  if constexpr (K::OUT_C && (kstep & 31u) == 0u) {
    put(stg + (base ^ key), [&](int n) { return (uint32_t)n * kstep; });
  } else if (!K::OUT_C && K::LOG2N == 8 && (wstep & 31u) == 0u) {
    put(stg + (base ^ key), [&](int n) { return ((uint32_t)n * kstep) << log2C; });
  } else {
    put(stg, [&](int n) { return (base + (uint32_t)n * wstep) ^ key; });
  }
}

// Staging copy (natural order, chunk-swizzled, at A) -> global memory for
// the chunk of transforms t0 .. t0 + nvalid - 1 whose output starts at gout:
// tensor-map stores issued by one thread (which waits until they have read
// the staging copy) or 16-byte stores by every thread.
template <class K>
__device__ __forceinline__ void copy_out(const PassParams& p, uint8_t* A, uint32_t* gout, int64_t t0, int nvalid,
                                         int log2C, const PassParams* maps = nullptr, bool wait_read = true) {
  const CUtensorMap* out_map = maps ? &maps->out_map : &p.out_map;  // param or global memory
  const int tid = threadIdx.x;
  const uint32_t P = (uint32_t)1 << (log2C + K::LOG2N);
  const uint32_t ow = out_words<K>(p);
  const uint4* stg = reinterpret_cast<const uint4*>(A);
  const uint32_t nch = P >> 2;
  if (K::OUT_C && K::S == 3 && p.out_tma) {
    // rows of 32 points in the 128-byte swizzle, up to 256 rows per box;
    // rows past the end of the output are not written
    if (tid == 0) {
      const int row0 = (int)((gout - p.out) >> 5);
      const uint32_t a0 = smem_u32(A);
      for (int pl = 0; pl < K::PLANES; ++pl)
        for (uint32_t r0 = 0; r0 < (P >> 5); r0 += 256)
          tma_store_5d(out_map, a0 + (uint32_t)pl * (P * 4u) + r0 * 128u, 0, row0 + (int)r0, pl, 0, 0);
      bulk_commit();
      if (wait_read) bulk_wait_read();  // the staging copy (= A) is rewritten by the next chunk
    }
  } else if constexpr (K::OUT_C) {
    const uint32_t vchunks = ((uint32_t)nvalid << K::LOG2N) >> 2;
    for (uint32_t q = tid; q < vchunks; q += blockDim.x) {
      const uint32_t c = (q << 2) >> K::LOG2N;
      const uint32_t ko = (q << 2) & (K::N - 1);
      const uint32_t pq = q ^ stg_key<K>(c, ko, log2C);
      uint32_t* o = p.out_scatter ? p.out + ow * (side_base(p.out_l, t0 + c, p.log2I1, p.log2I2) + ko)
                                  : gout + ow * (q << 2);
      if (K::SPLIT && p.out_f32) {
        // four points: re and im planes -> interleaved FP32 complex
        const uint4 re = stg[pq], im = stg[nch + pq];
        reinterpret_cast<uint4*>(o)[0] = make_uint4(re.x, im.x, re.y, im.y);
        reinterpret_cast<uint4*>(o)[1] = make_uint4(re.z, im.z, re.w, im.w);
        continue;
      }
      *reinterpret_cast<uint4*>(o) = stg[pq];
      if constexpr (K::SPLIT) *reinterpret_cast<uint4*>(o + p.out_plane) = stg[nch + pq];
    }
  } else if (p.out_tma) {
    // tensor-map boxes of C columns x 256 elements per plane, one thread
    if (tid == 0) {
      const int64_t t1 = t0 & ((int64_t(1) << p.log2I1) - 1);
      const int64_t t23 = t0 >> p.log2I1;
      const int t2 = (int)(t23 & ((int64_t(1) << p.log2I2) - 1));
      const int t3 = (int)(t23 >> p.log2I2);
      const uint32_t a0 = smem_u32(A);
      for (int pl = 0; pl < K::PLANES; ++pl)
        for (int e0 = 0; e0 < K::N; e0 += 256)
          tma_store_5d(out_map, a0 + (uint32_t)pl * (P * 4u) + ((uint32_t)e0 << log2C) * 4u, (int)t1, e0,
                       t2, t3, pl);
      bulk_commit();
      if (wait_read) bulk_wait_read();  // the staging copy (= A) is rewritten by the next chunk
    }
  } else {
    const int cq = log2C - 2;  // log2 of the chunks per output element index
    const uint32_t es = p.out_l.es;
    for (uint32_t q = tid; q < nch; q += blockDim.x) {
      const uint32_t ko = q >> cq;
      const uint32_t cc = (q & ((1u << cq) - 1u)) << 2;
      const uint32_t off = ko * es + cc;
      const uint32_t pq = q ^ stg_key<K>(cc, ko, log2C);
      if (K::SPLIT && p.out_f32) {
        const uint4 re = stg[pq], im = stg[nch + pq];
        uint4* o = reinterpret_cast<uint4*>(gout + 2u * off);
        o[0] = make_uint4(re.x, im.x, re.y, im.y);
        o[1] = make_uint4(re.z, im.z, re.w, im.w);
        continue;
      }
      *reinterpret_cast<uint4*>(gout + off) = stg[pq];
      if constexpr (K::SPLIT) *reinterpret_cast<uint4*>(gout + p.out_plane + off) = stg[nch + pq];
    }
  }
}

// DFT matrix images -> shared memory at Bs (the global table holds 8 hi then
// 8 lo images): plain, hi image k0 in slot k0; split, hi image k0 in slot 2 k0
// and its lo image in slot 2 k0 + 1, so that [B_hi | B_lo] is one N = 64
// operand.  FOLD kernels take one image per leading-radix digit k0.
template <class K>
__device__ __forceinline__ void load_dft_images(const PassParams& p, uint8_t* Bs) {
  constexpr int NB = K::FOLD ? K::RX : 1;
  const uint4* src = reinterpret_cast<const uint4*>(p.dft_b);
  uint4* dst = reinterpret_cast<uint4*>(Bs);
  constexpr int per = kBImageBytes / 16;
  for (int i = threadIdx.x; i < K::PLANES * NB * per; i += (int)blockDim.x) {
    const int slot = i / per, r = i - slot * per;
    const int plane = K::SPLIT ? (slot & 1) : 0, k0 = K::SPLIT ? (slot >> 1) : slot;
    dst[i] = __ldg(src + (plane * 8 + k0) * per + r);
  }
}

// ------------------------------------------------------------ stage loop
// The S radix-16 stages of one chunk whose stage-1 A operand is in shared
// memory: per stage, one thread issues the MMAs of every tile (stage 1 with
// FOLD: the DFT image of the tile's k0) and commits them to the MMA barrier;
// the epilogue warps read the accumulators, apply the stage twiddle and write
// the next stage's A in place.  After the last stage each butterfly's 16
// outputs go to fin(c, kbase, X, Y): transform c of the chunk, output index
// kbase + (2i) kstep in X[i].x / Y[i].x (re / im) and kbase + (2i+1) kstep in
// X[i].y / Y[i].y, kstep = 16^{S-1} R.  Returns false (status written) when
// an MMA wait times out.
struct StageCtx {
  uint8_t* A;       // stage operand tiles (1 KB aligned); split: lo plane follows
  uint32_t a_base;  // shared-memory address of A
  uint32_t b_base;  // shared-memory address of the DFT-matrix images
  uint32_t tmem;    // TMEM base address
  uint32_t mbar_s;  // MMA completion barrier
  uint32_t phase;   // its current parity
};

template <class K, class Final>
__device__ __forceinline__ bool run_stages(const PassParams& p, StageCtx& cx, int tiles, int log2C, Final& fin) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3;  // TMEM lane quarter of this warp
  const int half = warp >> 2;    // which tiles this warp takes in the epilogue
  const int halves = (int)(blockDim.x >> 7);  // warps per TMEM lane quarter
  const uint32_t rows_valid = (uint32_t)1 << (log2C + K::LOG2N - 4);  // butterflies per stage
  const uint32_t idesc = make_idesc_f16(128, 32, 1, 0);
  const uint32_t idesc64 = make_idesc_f16(128, 64, 1, 0);  // split: [B_hi | B_lo]
  uint8_t* A = cx.A;
  const uint32_t a_base = cx.a_base, b_base = cx.b_base, tmem = cx.tmem, mbar_s = cx.mbar_s;
  uint32_t& phase = cx.phase;
#pragma unroll
  for (int j = 1; j <= K::S; ++j) {
    if (tid == 0) {
      tc_fence_after_sync();
      for (int t = 0; t < tiles; ++t) {
        const uint32_t a = a_base + t * kTileBytes;
        // stage 1 with FOLD: the DFT matrix of this tile's k0
        const uint32_t kb = (K::FOLD && j == 1) ? ((uint32_t)(t * 128) >> (log2C + K::LOG2LQ)) : 0u;
        if constexpr (!K::SPLIT) {
          const uint32_t d = tmem + 32u * t;
          const uint32_t bb = b_base + kb * kBImageBytes;
          mma_f16(d, make_smem_desc(a, 4096, 1024, 2), make_smem_desc(bb, 128, 512, 0), idesc, 0);
          mma_f16(d, make_smem_desc(a + 2048, 4096, 1024, 2),
                  make_smem_desc(bb + 256, 128, 512, 0), idesc, 1);
        } else {
          // tile t owns TMEM columns [64 t, 64 t + 64): the main product
          // A_hi B_hi in the first 32, the correction A_hi B_lo + A_lo B_hi in
          // the second.  One N = 64 MMA forms A_hi [B_hi | B_lo] (the lo image
          // follows its hi image, at the same 512-byte group stride), one
          // N = 32 MMA adds A_lo B_hi; per K half.
          const uint32_t dm = tmem + 64u * t;
          const uint32_t bb = b_base + 2u * kb * kBImageBytes;
          const uint32_t alo = a + tiles * kTileBytes;
          mma_f16(dm, make_smem_desc(a, 4096, 1024, 2), make_smem_desc(bb, 128, 512, 0), idesc64, 0);
          mma_f16(dm + 32u, make_smem_desc(alo, 4096, 1024, 2), make_smem_desc(bb, 128, 512, 0), idesc, 1);
          mma_f16(dm, make_smem_desc(a + 2048, 4096, 1024, 2), make_smem_desc(bb + 256, 128, 512, 0),
                  idesc64, 1);
          mma_f16(dm + 32u, make_smem_desc(alo + 2048, 4096, 1024, 2),
                  make_smem_desc(bb + 256, 128, 512, 0), idesc, 1);
        }
      }
      mma_commit(mbar_s);
    }
    // the issuing thread polls the MMA barrier; the others sleep in the
    // CTA barrier, ordered after the MMAs by the tcgen05 fence pair
    bool got = true;
    if (tid == 0) got = mbar_wait_bounded(mbar_s, phase, kWaitLimitCycles);
    phase ^= 1u;
    tc_fence_before_sync();
    if (__syncthreads_or(!got)) {
      if (tid == 0) atomicExch(p.status, kDevErrTimeout);
      return false;
    }
    tc_fence_after_sync();

    const bool last = (j == K::S);
    for (int t = half; t < tiles; t += halves) {
      const uint32_t row = rp((uint32_t)t * 128u + 32u * quarter + lane);  // logical row of this lane
      // X[i] = (Re out 2i, Re out 2i+1), Y[i] = (Im out 2i, Im out 2i+1)
      float2 X[8], Y[8];
      {
        const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (K::SPLIT ? 64u : 32u) * t;
        float v[32];
        tmem_ld32_wait(taddr, v);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          X[i] = make_float2(v[2 * i], v[2 * i + 1]);
          Y[i] = make_float2(v[16 + 2 * i], v[16 + 2 * i + 1]);
        }
        if constexpr (K::SPLIT) {
          tmem_ld32_wait(taddr + 32u, v);
          const float2 s = make_float2(1.0f / 2048.0f, 1.0f / 2048.0f);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            X[i] = __ffma2_rn(make_float2(v[2 * i], v[2 * i + 1]), s, X[i]);
            Y[i] = __ffma2_rn(make_float2(v[16 + 2 * i], v[16 + 2 * i + 1]), s, Y[i]);
          }
        }
      }
      if (row >= rows_valid) continue;  // padding rows of a partial last tile

      // butterfly identity of this row at stage j: sub-transform g, the
      // digits kk = (k_1 .. k_{j-1}) already produced, and nrest = n^(j+1)
      uint32_t g, nrest, kk;
      uint32_t k0row = 0;  // k0 of the row (stage 1)
      if (j == 1) {
        kk = 0;
        const uint32_t lk = (uint32_t)log2C + K::LOG2LQ;  // rows per k0
        k0row = row >> lk;
        const uint32_t rem = row & ((1u << lk) - 1u);
        uint32_t c1;
        if constexpr (K::IN_C) {
          c1 = rem >> K::LOG2LQ;
          nrest = rem & (K::LQ - 1);
        } else {
          nrest = rem >> log2C;
          c1 = rem & ((1u << log2C) - 1u);
        }
        g = (k0row << log2C) + c1;
      } else {
        const int sj = 4 * (j - 1);
        kk = row & ((1u << sj) - 1u);
        const uint32_t q = row >> sj;
        const int sr = 4 * (K::S - j);
        g = q >> sr;
        nrest = q & ((1u << sr) - 1u);
      }

      if (!last) {
        // twiddle of output k: a b^k, stage 1: a = W_N^{k0 nrest}, b =
        // W_{L}^{nrest}; stage j >= 2: a = 1, b = W_{L_j}^{nrest}, as pairs
        // (a b^{2i}, a b^{2i+1}) in packed FP32x2 arithmetic
        {
          int toff = 0;
          if (j >= 2) toff = K::RX << K::LOG2LQ;
#pragma unroll
          for (int i = 2; i < j; ++i) toff += 1 << (4 * (K::S - i));
          const int ent = toff + (j == 1 ? (int)((k0row << K::LOG2LQ) + nrest) : (int)nrest);
          if (!K::IN_C || (j >= 2 && K::RX == 1)) {
            // the lanes of a warp share a few keys here (their rows differ in
            // the transform of a strided chunk, or in the digits already
            // produced), so the 16 twiddles come from the table as 8 packed
            // pairs: measured 2-3 % faster on strided passes and N = 4096.
            // Stage 1 of a contiguous chunk (one key per lane) and the later
            // stages of N = 16384 keep the multiply chain, which measured
            // faster there.
            const float4* tw = p.stw + K::STAGE_KEYS + 8 * ent;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float4 w = __ldg(tw + i);
              cmul2(X[i], Y[i], make_float2(w.x, w.y), make_float2(w.z, w.w), make_float2(-w.z, -w.w));
            }
          } else {
            // the pairs advanced from (a, b) by packed multiplies
            const float4 e = __ldg(p.stw + ent);
            const float2 a = make_float2(e.x, e.y), b = make_float2(e.z, e.w);
            const float2 ab = cmulf(a, b), b2 = cmulf(b, b);
            float2 c2 = make_float2(a.x, ab.x), d2 = make_float2(a.y, ab.y);
            const float2 sc = make_float2(b2.x, b2.x), sd = make_float2(b2.y, b2.y);
            const float2 snd = make_float2(-b2.y, -b2.y);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              cmul2(X[i], Y[i], c2, d2, make_float2(-d2.x, -d2.y));
              if (i < 7) {
                float2 cn = c2, dn = d2;
                cmul2(cn, dn, sc, sd, snd);
                c2 = cn;
                d2 = dn;
              }
            }
          }
        }
        const int sh = 4 * (K::S - j - 1);
        const uint32_t nnext = nrest >> sh;
        const uint32_t nlow = nrest & ((1u << sh) - 1u);
        const uint32_t dr = ((((g << sh) + nlow) << (4 * j)) + (kk << 4));
        const RowChunks rc = row_chunks(dr, nnext);
        uint32_t hr[8], hi[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          hr[i] = f2h2(X[i].x, X[i].y);
          hi[i] = f2h2(Y[i].x, Y[i].y);
        }
        *reinterpret_cast<uint4*>(A + rc.re0) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
        *reinterpret_cast<uint4*>(A + rc.re0 + 2048) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(A + rc.re1) = make_uint4(hr[4], hr[5], hr[6], hr[7]);
        *reinterpret_cast<uint4*>(A + rc.re1 + 2048) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
        if constexpr (K::SPLIT) {
          uint32_t lr[8], li[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            lr[i] = split_lo(X[i].x, X[i].y, hr[i]);
            li[i] = split_lo(Y[i].x, Y[i].y, hi[i]);
          }
          uint8_t* Alo = A + tiles * kTileBytes;
          *reinterpret_cast<uint4*>(Alo + rc.re0) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
          *reinterpret_cast<uint4*>(Alo + rc.re0 + 2048) = make_uint4(li[0], li[1], li[2], li[3]);
          *reinterpret_cast<uint4*>(Alo + rc.re1) = make_uint4(lr[4], lr[5], lr[6], lr[7]);
          *reinterpret_cast<uint4*>(Alo + rc.re1 + 2048) = make_uint4(li[4], li[5], li[6], li[7]);
        }
      } else {
        // final stage: the output identity of this butterfly
        uint32_t rev = 0;
        {
          uint32_t x = kk;
#pragma unroll
          for (int d = 0; d < K::S - 1; ++d) {
            rev = (rev << 4) | (x & 15u);
            x >>= 4;
          }
        }
        const uint32_t k0 = g >> log2C;
        const uint32_t c = g & ((1u << log2C) - 1u);
        fin(c, k0 + (rev << K::LOG2RX), X, Y);
      }
    }
    fence_proxy_async_smem();
    tc_fence_before_sync();
    __syncthreads();
  }
  return true;
}

// Final-stage output of one butterfly of a pass (transform c of the chunk
// starting at transform t0, output index kbase at k_S = 0): the optional
// multi-pass output twiddle, the inverse's conjugation, then straight to
// global memory (DIRECT_OUT) or into the staging copy at A.
template <class K>
__device__ __forceinline__ void final_out(const PassParams& p, uint8_t* A, uint32_t* gout, int64_t t0, int nvalid,
                                          int log2C, uint32_t c, uint32_t kbase, float2 (&X)[8], float2 (&Y)[8]) {
  const uint32_t ow = out_words<K>(p);
  constexpr uint32_t kstep = (uint32_t)K::LQ << K::LOG2RX;  // output index step per k_S
  if (p.otw_level) {
    // W_M^{col (kbase + kstep k)}: powers of ws = W_M^{col kstep} from
    // w0 = W_M^{col kbase}, advanced two outputs at a time
    const int64_t t = t0 + c;
    const uint32_t col = (p.otw_level == 1)
                             ? (uint32_t)(t & ((int64_t(1) << p.log2I1) - 1))
                             : (uint32_t)((t >> p.log2I1) & ((int64_t(1) << p.log2I2) - 1));
    const float2 w0 = tw_lookup(p.otw_lo, p.otw_hi, col * kbase, p.otw_log2M, p.otw_log2S);
    const float2 ws = tw_lookup(p.otw_lo, p.otw_hi, col * kstep, p.otw_log2M, p.otw_log2S);
    const float2 w1 = cmulf(w0, ws), ws2 = cmulf(ws, ws);
    float2 c2 = make_float2(w0.x, w1.x), d2 = make_float2(w0.y, w1.y);
    const float2 sc = make_float2(ws2.x, ws2.x), sd = make_float2(ws2.y, ws2.y);
    const float2 snd = make_float2(-ws2.y, -ws2.y);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      cmul2(X[i], Y[i], c2, d2, make_float2(-d2.x, -d2.y));
      if (i < 7) {
        float2 cn = c2, dn = d2;
        cmul2(cn, dn, sc, sd, snd);
        c2 = cn;
        d2 = dn;
      }
    }
  }
  if (p.conj_out) {
    // inverse transform: conj() of the result
#pragma unroll
    for (int i = 0; i < 8; ++i) Y[i] = make_float2(-Y[i].x, -Y[i].y);
  }
  if constexpr (K::DIRECT_OUT) {
    // lanes hold consecutive output indices: store straight to global
    if ((int)c < nvalid) {
      uint32_t* o = (p.out_scatter ? p.out + ow * side_base(p.out_l, t0 + c, p.log2I1, p.log2I2)
                                   : gout + ow * (c << K::LOG2N)) + ow * kbase;
      if (K::SPLIT && p.out_f32) {
        // interleaved FP32 complex straight from the accumulator
        float2* of = reinterpret_cast<float2*>(o);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          of[(2 * i) * kstep] = make_float2(X[i].x, Y[i].x);
          of[(2 * i + 1) * kstep] = make_float2(X[i].y, Y[i].y);
        }
        return;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint32_t h0 = f2h2(X[i].x, Y[i].x), h1 = f2h2(X[i].y, Y[i].y);
        o[(2 * i) * kstep] = h0;
        o[(2 * i + 1) * kstep] = h1;
        if constexpr (K::SPLIT) {
          o[p.out_plane + (2 * i) * kstep] = split_lo(X[i].x, Y[i].x, h0);
          o[p.out_plane + (2 * i + 1) * kstep] = split_lo(X[i].y, Y[i].y, h1);
        }
      }
    }
    return;
  }
  staging_store<K>(p, A, (uint32_t)1 << (log2C + K::LOG2N), log2C, c, kbase, X, Y);
}

// ------------------------------------------------------------ pass body
// Per-CTA resources the pass body runs on: the operand area (1 KB aligned:
// A tiles, raw prefetch buffer and DFT images, laid out per pass), the MMA
// and copy barriers with their parities, TMEM.
struct PassCta {
  uint8_t* A;
  uint64_t* mbar;
  uint64_t* lbar;
  uint32_t tmem;
  uint32_t phase, lphase;
};

// Chunks slot, slot + nslots, ... of pass p on this CTA (C transforms each).
// With async_load, the raw input of the next chunk is copied into shared
// memory (bulk copy, tensor-map boxes or cp.async) while the current chunk
// runs its MMA stages, epilogues and stores.  `maps` holds the tensor maps in
// param or global memory (p may be a shared-memory copy); load_images: copy
// the pass's DFT images into place first; launch_dependents: trigger the
// programmatic dependent launch at the CTA's last chunk; CG: synchronous
// loads through L2 only (inputs written by other CTAs of the same launch).
// Returns false when a wait timed out (status written); on return no copy
// targets shared memory and every tensor-map store has completed.
template <class K, bool CG>
__device__ __forceinline__ bool pass_body(const PassParams& p, const PassParams& maps, int64_t slot, int64_t nslots,
                                          PassCta& cta, bool load_images, bool launch_dependents) {
  const int tid = threadIdx.x;
  uint8_t* A = cta.A;
  const int tiles = p.tiles;
  const int log2C = p.log2C;
  const int C = 1 << log2C;
  const uint32_t P = (uint32_t)C << K::LOG2N;  // points per chunk and plane
  uint8_t* RAW = A + K::PLANES * tiles * kTileBytes;
  uint8_t* Bs = RAW + (p.async_load ? K::PLANES * P * 4u : 0u);
  if (load_images) load_dft_images<K>(p, Bs);
  const uint32_t raw_s = smem_u32(RAW);
  const uint32_t lbar_s = smem_u32(cta.lbar);
  const uint32_t* raw32 = reinterpret_cast<const uint32_t*>(RAW);
  uint32_t lphase = cta.lphase;
  bool ok = true, pending = false;  // pending: a bulk copy into RAW is in flight
  StageCtx cx{A, smem_u32(A), smem_u32(Bs), cta.tmem, smem_u32(cta.mbar), cta.phase};

  auto chunk_in = [&](int64_t ch) {
    return p.in + in_words<K>(p) * side_base(p.in_l, ch << log2C, p.log2I1, p.log2I2);
  };
  auto chunk_valid = [&](int64_t ch) {
    const int64_t left = p.T - (ch << log2C);
    return left < C ? (int)left : C;
  };

  int64_t chunk = slot;
  if (p.async_load && chunk < p.nchunks) {
    issue_raw_copy<K>(p, raw_s, lbar_s, chunk_in(chunk), chunk << log2C, log2C, chunk_valid(chunk), &maps);
    pending = K::IN_C || p.in_tma;
  }

  for (; chunk < p.nchunks; chunk += nslots) {
    // last chunk of this CTA: the next kernel may start its prologue
    if (launch_dependents && chunk + nslots >= p.nchunks) griddep_launch_dependents();
    const int64_t t0 = chunk << log2C;
    const int nvalid = chunk_valid(chunk);
    const uint32_t ow = out_words<K>(p);
    uint32_t* gout = p.out + ow * side_base(p.out_l, t0, p.log2I1, p.log2I2);

    if (p.async_load) {
      if (K::IN_C || p.in_tma) {
        // one thread polls the copy's barrier; the others sleep in the CTA
        // barrier (no issue slots spent spinning) and see the copied bytes
        // through it
        bool got = true;
        if (tid == 0) {
          got = mbar_wait_bounded(lbar_s, lphase, kWaitLimitCycles);
          if (p.out_tma) bulk_wait_read();  // the previous chunk's stores have read the staging copy (= A)
        }
        if (__syncthreads_or(!got)) {
          if (tid == 0) atomicExch(p.status, kDevErrTimeout);
          ok = false;
          break;
        }
        lphase ^= 1u;
        pending = false;
      } else {
        cp_async_wait_all();
        if (tid == 0 && p.out_tma) bulk_wait_read();
        __syncthreads();
      }
      load_stage1<K, true>(p, A, raw32, raw32 + P, K::IN_C ? 1u : (uint32_t)C, log2C, nvalid);
      __syncthreads();  // raw buffer consumed: prefetch the next chunk into it
      const int64_t next = chunk + nslots;
      if (next < p.nchunks) {
        issue_raw_copy<K>(p, raw_s, lbar_s, chunk_in(next), next << log2C, log2C, chunk_valid(next), &maps);
        pending = K::IN_C || p.in_tma;
      }
    } else {
      const uint32_t* gin = chunk_in(chunk);
      load_stage1<K, false, CG>(p, A, gin, gin + p.in_plane, p.in_l.es, log2C, nvalid, t0);
    }

    fence_proxy_async_smem();
    tc_fence_before_sync();
    __syncthreads();

    auto fin = [&](uint32_t c, uint32_t kbase, float2 (&X)[8], float2 (&Y)[8]) {
      final_out<K>(p, A, gout, t0, nvalid, log2C, c, kbase, X, Y);
    };
    ok = run_stages<K>(p, cx, tiles, log2C, fin);
    if (!ok) break;

    // copy-out: staging (natural order, chunk-swizzled) -> global.  With
    // prefetching, the wait for the tensor-map stores to read the staging
    // copy moves to the next chunk's input wait, just before load_stage1
    // rewrites A, so the issuing thread does not poll for it here.
    if constexpr (!K::DIRECT_OUT) copy_out<K>(p, A, gout, t0, nvalid, log2C, &maps, !p.async_load);
    __syncthreads();  // staging (= A) is rewritten by the next chunk
  }

  if (p.out_tma && tid == 0) bulk_wait_all();
  // unwind: no copy may still target this CTA's shared memory
  if (p.async_load) {
    if (K::IN_C || p.in_tma) {
      if (pending && mbar_wait_bounded(lbar_s, lphase, kWaitLimitCycles)) lphase ^= 1u;
    } else {
      cp_async_wait_all();
    }
  }
  cta.phase = cx.phase;
  cta.lphase = lphase;
  return ok;
}

// ---------------------------------------------------------------- kernel
// Persistent: CTA b processes chunks b, b + gridDim.x, ... (C transforms
// each).  With async_load, the raw input of the next chunk is copied into
// shared memory (bulk copy or cp.async) while the current chunk runs its
// MMA stages, epilogues and stores.
template <int LOG2N, int MODE, bool SPLIT>
__global__ void __launch_bounds__(kThreads, (PassCfg<LOG2N, MODE, SPLIT>::MINB))
    pass_kernel(const __grid_constant__ PassParams p) {
  using K = PassCfg<LOG2N, MODE, SPLIT>;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* A = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                          ~uintptr_t(1023));
  const int tiles = p.tiles;
  const int log2C = p.log2C;
  const int C = 1 << log2C;
  const uint32_t P = (uint32_t)C << LOG2N;  // points per chunk and plane
  uint8_t* RAW = A + K::PLANES * tiles * kTileBytes;
  constexpr int NB = K::FOLD ? K::RX : 1;  // DFT matrix images per plane
  uint8_t* Bs = RAW + (p.async_load ? K::PLANES * P * 4u : 0u);
  // barrier words and the TMEM slot (64 bytes) sit in the 1 KB alignment
  // slack below A when it has room, else after the B images; the host
  // reserves 1008 bytes of slack (the base is 16-byte aligned)
  const uint32_t slack = (uint32_t)(A - smem_raw);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(slack >= 64 ? A - 64 : Bs + K::PLANES * NB * kBImageBytes);
  uint64_t* lbar = mbar + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);

  const int tid = threadIdx.x;
  const int warp = tid >> 5;

  load_dft_images<K>(p, Bs);
  if (tid == 0) {
    mbar_init(smem_u32(mbar), 1);
    mbar_init(smem_u32(lbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tslot), (uint32_t)p.tmem_cols);
    tmem_relinquish();
  }

  PassCta cta{A, mbar, lbar, 0u, 0u, 0u};
  tc_fence_before_sync();
  __syncthreads();  // barriers initialised, TMEM address published
  tc_fence_after_sync();
  cta.tmem = *tslot;
  const uint32_t tmem = cta.tmem;

  // everything above reads only plan-time tables; the pass input may be the
  // previous kernel's output
  griddep_wait();
  (void)pass_body<K, false>(p, p, blockIdx.x, gridDim.x, cta, false, true);

  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after_sync();
    tmem_dealloc(tmem, (uint32_t)p.tmem_cols);
  }
}

}  // namespace tcfft
