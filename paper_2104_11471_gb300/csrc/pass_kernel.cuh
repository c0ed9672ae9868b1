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
// CUDA cores") splits N = R L the same way before the first radix-16 stage.
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
//    copy of shared memory, which is then stored with 16-byte coalesced
//    writes ("continuous size", Sec. 4.2, Table gbw).
// Split precision (hi + 2^-11 lo, FP32 accumulation, three products per
// stage) follows the paper's "precision recovery" future work (Sec. 7).
#pragma once
#include <cuda_fp16.h>
#include <cstdint>

#include "pass_params.h"
#include "tc_ptx.cuh"

namespace tcfft {

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

// Staging buffer word (one complex = 4 bytes) with a 16-byte-chunk XOR
// swizzle inside each 128-byte line.
__device__ __forceinline__ uint32_t stg_word(uint32_t idx) {
  const uint32_t q = idx >> 2;
  return ((q ^ ((q >> 3) & 7u)) << 2) | (idx & 3u);
}

__device__ __forceinline__ int64_t side_base(const SideLayout& l, int64_t t, int log2I1,
                                             int log2I2) {
  const int64_t t1 = t & ((int64_t(1) << log2I1) - 1);
  const int64_t t23 = t >> log2I1;
  const int64_t t2 = t23 & ((int64_t(1) << log2I2) - 1);
  const int64_t t3 = t23 >> log2I2;
  return t1 * l.s1 + t2 * l.s2 + t3 * l.s3;
}

__device__ __forceinline__ float2 tw_lookup(const float* lo, const float* hi, uint64_t a,
                                            int log2M, int log2S) {
  a &= (uint64_t(1) << log2M) - 1;
  const float2 h = __ldg(reinterpret_cast<const float2*>(hi) + (a >> log2S));
  const float2 l = __ldg(reinterpret_cast<const float2*>(lo) + (a & ((uint64_t(1) << log2S) - 1)));
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
__device__ __forceinline__ uint32_t f2h1(float a) {
  __half h = __float2half_rn(a);
  return (uint32_t)(*reinterpret_cast<uint16_t*>(&h));
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
    float2 w1 = make_float2(h, -h), w3 = make_float2(-h, -h);
    float2 t0 = o[0], t1 = cmulf(o[1], w1), t2 = make_float2(o[2].y, -o[2].x), t3 = cmulf(o[3], w3);
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

// Writes 8 consecutive butterfly rows (m0 multiple of 8) of input k of A:
// re halves at K = k, im halves at K = 16 + k.
__device__ __forceinline__ void a_store8(uint8_t* A, uint32_t m0, uint32_t k, uint4 re8,
                                         uint4 im8) {
  *reinterpret_cast<uint4*>(A + a_off(m0, k)) = re8;
  *reinterpret_cast<uint4*>(A + a_off(m0, 16 + k)) = im8;
}

// ------------------------------------------------------------------ loads
// Reads the CTA's C transforms, applies the leading radix-RX step (if any)
// and writes the stage-1 A operand(s).
//   contiguous input: sub-transform g = c*RX + k0, stage-1 row g*16^{S-1} + n^(2)
//   strided input:    sub-transform g = k0*C + c, stage-1 row n^(2)*G + g
template <int RX, bool SPLIT>
__device__ __forceinline__ void load_stage1(const PassParams& p, uint8_t* A, int64_t t0) {
  const int L = 1 << (4 * p.S);     // sub-transform length
  const int Lq = L >> 4;            // 16^{S-1}
  const int C = p.C;
  uint8_t* Alo = A + p.tiles * kTileBytes;
  const float inv = 1.0f / 2048.0f;
  if (p.in_contig) {
    const int blocks = L >> 3;  // 8-point blocks per sub-transform
    const int items = C * blocks;
    for (int it = threadIdx.x; it < items; it += kThreads) {
      const int c = it / blocks;
      const int nb = (it - c * blocks) << 3;
      const int64_t t = t0 + c;
      const bool valid = t < p.T;
      const int64_t base = valid ? side_base(p.in_l, t, p.log2I1, p.log2I2) : 0;
      uint32_t hv[RX][8], lv[RX][8];
#pragma unroll
      for (int n0 = 0; n0 < RX; ++n0) {
        uint4 a = make_uint4(0, 0, 0, 0), b = a, c2 = a, d = a;
        if (valid) {
          const uint4* src = reinterpret_cast<const uint4*>(p.in + base + n0 * L + nb);
          a = __ldg(src);
          b = __ldg(src + 1);
          if constexpr (SPLIT) {
            const uint4* s2 = reinterpret_cast<const uint4*>(p.in + p.in_plane + base + n0 * L + nb);
            c2 = __ldg(s2);
            d = __ldg(s2 + 1);
          }
        }
        hv[n0][0] = a.x; hv[n0][1] = a.y; hv[n0][2] = a.z; hv[n0][3] = a.w;
        hv[n0][4] = b.x; hv[n0][5] = b.y; hv[n0][6] = b.z; hv[n0][7] = b.w;
        lv[n0][0] = c2.x; lv[n0][1] = c2.y; lv[n0][2] = c2.z; lv[n0][3] = c2.w;
        lv[n0][4] = d.x; lv[n0][5] = d.y; lv[n0][6] = d.z; lv[n0][7] = d.w;
      }
      if constexpr (RX > 1) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float2 v[RX];
#pragma unroll
          for (int n0 = 0; n0 < RX; ++n0) {
            v[n0] = h2f(hv[n0][i]);
            if constexpr (SPLIT) {
              float2 l = h2f(lv[n0][i]);
              v[n0].x = fmaf(l.x, inv, v[n0].x);
              v[n0].y = fmaf(l.y, inv, v[n0].y);
            }
          }
          small_dft<RX>(v);
          const int np = nb + i;  // n' of this point
#pragma unroll
          for (int k0 = 0; k0 < RX; ++k0) {
            float2 y = v[k0];
            if (k0) y = cmulf(y, tw_lookup(p.tw_lo, p.tw_hi, (uint64_t)k0 * np, p.log2N, p.tw_log2S));
            hv[k0][i] = f2h2(y.x, y.y);
            if constexpr (SPLIT) {
              float2 hf = h2f(hv[k0][i]);
              lv[k0][i] = f2h2((y.x - hf.x) * 2048.0f, (y.y - hf.y) * 2048.0f);
            }
          }
        }
      }
      const int n1 = nb / Lq;  // valid when Lq >= 8
#pragma unroll
      for (int k0 = 0; k0 < RX; ++k0) {
        const int g = c * RX + k0;
        if (Lq >= 8) {
          const uint32_t m0 = (uint32_t)g * Lq + (nb & (Lq - 1));
          uint4 re = make_uint4(__byte_perm(hv[k0][0], hv[k0][1], 0x5410), __byte_perm(hv[k0][2], hv[k0][3], 0x5410),
                                __byte_perm(hv[k0][4], hv[k0][5], 0x5410), __byte_perm(hv[k0][6], hv[k0][7], 0x5410));
          uint4 im = make_uint4(__byte_perm(hv[k0][0], hv[k0][1], 0x7632), __byte_perm(hv[k0][2], hv[k0][3], 0x7632),
                                __byte_perm(hv[k0][4], hv[k0][5], 0x7632), __byte_perm(hv[k0][6], hv[k0][7], 0x7632));
          a_store8(A, m0, n1, re, im);
          if constexpr (SPLIT) {
            uint4 re2 = make_uint4(__byte_perm(lv[k0][0], lv[k0][1], 0x5410), __byte_perm(lv[k0][2], lv[k0][3], 0x5410),
                                   __byte_perm(lv[k0][4], lv[k0][5], 0x5410), __byte_perm(lv[k0][6], lv[k0][7], 0x5410));
            uint4 im2 = make_uint4(__byte_perm(lv[k0][0], lv[k0][1], 0x7632), __byte_perm(lv[k0][2], lv[k0][3], 0x7632),
                                   __byte_perm(lv[k0][4], lv[k0][5], 0x7632), __byte_perm(lv[k0][6], lv[k0][7], 0x7632));
            a_store8(Alo, m0, n1, re2, im2);
          }
        } else {
          // S == 1: the 8 points are 8 different inputs of butterfly row g
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const uint32_t k = (uint32_t)(nb + i);
            *reinterpret_cast<uint16_t*>(A + a_off(g, k)) = (uint16_t)(hv[k0][i] & 0xFFFFu);
            *reinterpret_cast<uint16_t*>(A + a_off(g, 16 + k)) = (uint16_t)(hv[k0][i] >> 16);
            if constexpr (SPLIT) {
              *reinterpret_cast<uint16_t*>(Alo + a_off(g, k)) = (uint16_t)(lv[k0][i] & 0xFFFFu);
              *reinterpret_cast<uint16_t*>(Alo + a_off(g, 16 + k)) = (uint16_t)(lv[k0][i] >> 16);
            }
          }
        }
      }
    }
  } else {
    // strided input: 8 adjacent transforms per 32-byte read
    const int cb_n = C >> 3;
    const int items = cb_n * L;
    const int G = C * RX;
    const int64_t base0 = side_base(p.in_l, t0, p.log2I1, p.log2I2);
    for (int it = threadIdx.x; it < items; it += kThreads) {
      const int cb = it % cb_n;
      const int np = it / cb_n;  // n' in [0, L)
      const int c0 = cb << 3;
      uint32_t hv[RX][8], lv[RX][8];
#pragma unroll
      for (int n0 = 0; n0 < RX; ++n0) {
        const int64_t off = base0 + c0 + (int64_t)(n0 * L + np) * p.in_l.es;
        const uint4* src = reinterpret_cast<const uint4*>(p.in + off);
        uint4 a = __ldg(src), b = __ldg(src + 1);
        hv[n0][0] = a.x; hv[n0][1] = a.y; hv[n0][2] = a.z; hv[n0][3] = a.w;
        hv[n0][4] = b.x; hv[n0][5] = b.y; hv[n0][6] = b.z; hv[n0][7] = b.w;
        if constexpr (SPLIT) {
          const uint4* s2 = reinterpret_cast<const uint4*>(p.in + p.in_plane + off);
          uint4 c2 = __ldg(s2), d = __ldg(s2 + 1);
          lv[n0][0] = c2.x; lv[n0][1] = c2.y; lv[n0][2] = c2.z; lv[n0][3] = c2.w;
          lv[n0][4] = d.x; lv[n0][5] = d.y; lv[n0][6] = d.z; lv[n0][7] = d.w;
        }
      }
      if constexpr (RX > 1) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float2 v[RX];
#pragma unroll
          for (int n0 = 0; n0 < RX; ++n0) {
            v[n0] = h2f(hv[n0][i]);
            if constexpr (SPLIT) {
              float2 l = h2f(lv[n0][i]);
              v[n0].x = fmaf(l.x, inv, v[n0].x);
              v[n0].y = fmaf(l.y, inv, v[n0].y);
            }
          }
          small_dft<RX>(v);
#pragma unroll
          for (int k0 = 0; k0 < RX; ++k0) {
            float2 y = v[k0];
            if (k0) y = cmulf(y, tw_lookup(p.tw_lo, p.tw_hi, (uint64_t)k0 * np, p.log2N, p.tw_log2S));
            hv[k0][i] = f2h2(y.x, y.y);
            if constexpr (SPLIT) {
              float2 hf = h2f(hv[k0][i]);
              lv[k0][i] = f2h2((y.x - hf.x) * 2048.0f, (y.y - hf.y) * 2048.0f);
            }
          }
        }
      }
      const int n1 = np / Lq;
      const int nrest = np & (Lq - 1);
#pragma unroll
      for (int k0 = 0; k0 < RX; ++k0) {
        const uint32_t m0 = (uint32_t)nrest * G + k0 * C + c0;
        uint4 re = make_uint4(__byte_perm(hv[k0][0], hv[k0][1], 0x5410), __byte_perm(hv[k0][2], hv[k0][3], 0x5410),
                              __byte_perm(hv[k0][4], hv[k0][5], 0x5410), __byte_perm(hv[k0][6], hv[k0][7], 0x5410));
        uint4 im = make_uint4(__byte_perm(hv[k0][0], hv[k0][1], 0x7632), __byte_perm(hv[k0][2], hv[k0][3], 0x7632),
                              __byte_perm(hv[k0][4], hv[k0][5], 0x7632), __byte_perm(hv[k0][6], hv[k0][7], 0x7632));
        a_store8(A, m0, n1, re, im);
        if constexpr (SPLIT) {
          uint4 re2 = make_uint4(__byte_perm(lv[k0][0], lv[k0][1], 0x5410), __byte_perm(lv[k0][2], lv[k0][3], 0x5410),
                                 __byte_perm(lv[k0][4], lv[k0][5], 0x5410), __byte_perm(lv[k0][6], lv[k0][7], 0x5410));
          uint4 im2 = make_uint4(__byte_perm(lv[k0][0], lv[k0][1], 0x7632), __byte_perm(lv[k0][2], lv[k0][3], 0x7632),
                                 __byte_perm(lv[k0][4], lv[k0][5], 0x7632), __byte_perm(lv[k0][6], lv[k0][7], 0x7632));
          a_store8(Alo, m0, n1, re2, im2);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- kernel
template <int RX, bool SPLIT>
__global__ void __launch_bounds__(kThreads, SPLIT ? 2 : 4) pass_kernel(const PassParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* A = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                          ~uintptr_t(1023));
  const int tiles = p.tiles;
  const int planes = SPLIT ? 2 : 1;
  uint8_t* Bs = A + planes * tiles * kTileBytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Bs + planes * kBImageBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  int* sflag = reinterpret_cast<int*>(tslot + 1);

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int64_t t0 = (int64_t)blockIdx.x * p.C;

  // DFT matrix image(s) -> shared memory
  {
    const uint4* src = reinterpret_cast<const uint4*>(p.dft_b);
    uint4* dst = reinterpret_cast<uint4*>(Bs);
    for (int i = tid; i < planes * kBImageBytes / 16; i += kThreads) dst[i] = __ldg(src + i);
  }
  if (tid == 0) {
    mbar_init(smem_u32(mbar), 1);
    *sflag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tslot), (uint32_t)p.tmem_cols);
    tmem_relinquish();
  }

  load_stage1<RX, SPLIT>(p, A, t0);

  const int S = p.S;
  constexpr int log2RX = (RX == 1) ? 0 : (RX == 2) ? 1 : (RX == 4) ? 2 : 3;
  const int N = 1 << p.log2N;
  const int C = p.C;
  const int G = C * RX;
  const uint32_t Lq = 1u << (4 * (S - 1));
  const uint32_t rows_valid = ((uint32_t)C << p.log2N) >> 4;  // butterflies per stage

  fence_proxy_async_smem();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = make_idesc_f16(128, 32, 1, 0);
  const uint32_t a_base = smem_u32(A), b_base = smem_u32(Bs);
  bool ok = true;

  for (int j = 1; j <= S; ++j) {
    if (tid == 0) {
      tc_fence_after_sync();
      for (int t = 0; t < tiles; ++t) {
        const uint32_t a = a_base + t * kTileBytes;
        const uint32_t d = tmem + 32u * t;
        mma_f16(d, make_smem_desc(a, 4096, 1024, 2), make_smem_desc(b_base, 128, 512, 0), idesc, 0);
        mma_f16(d, make_smem_desc(a + 2048, 4096, 1024, 2), make_smem_desc(b_base + 256, 128, 512, 0),
                idesc, 1);
        if constexpr (SPLIT) {
          const uint32_t alo = a + tiles * kTileBytes;
          const uint32_t blo = b_base + kBImageBytes;
          const uint32_t d2 = tmem + 32u * (tiles + t);
          mma_f16(d2, make_smem_desc(alo, 4096, 1024, 2), make_smem_desc(b_base, 128, 512, 0), idesc, 0);
          mma_f16(d2, make_smem_desc(alo + 2048, 4096, 1024, 2),
                  make_smem_desc(b_base + 256, 128, 512, 0), idesc, 1);
          mma_f16(d2, make_smem_desc(a, 4096, 1024, 2), make_smem_desc(blo, 128, 512, 0), idesc, 1);
          mma_f16(d2, make_smem_desc(a + 2048, 4096, 1024, 2), make_smem_desc(blo + 256, 128, 512, 0),
                  idesc, 1);
        }
      }
      mma_commit(smem_u32(mbar));
    }
    const bool got = mbar_wait_bounded(smem_u32(mbar), (uint32_t)((j - 1) & 1), kWaitLimitCycles);
    if (__syncthreads_or(!got)) {
      if (tid == 0) atomicExch(p.status, kDevErrTimeout);
      ok = false;
      break;
    }
    tc_fence_after_sync();

    const bool last = (j == S);
    for (int t = 0; t < tiles; ++t) {
      const uint32_t row = (uint32_t)t * 128u + 32u * warp + lane;
      float re[16], im[16];
      {
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + 32u * t;
        float v[32];
        tmem_ld32_wait(taddr, v);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          re[k] = v[k];
          im[k] = v[16 + k];
        }
        if constexpr (SPLIT) {
          tmem_ld32_wait(taddr + 32u * tiles, v);
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            re[k] = fmaf(v[k], 1.0f / 2048.0f, re[k]);
            im[k] = fmaf(v[16 + k], 1.0f / 2048.0f, im[k]);
          }
        }
      }

      if (row >= rows_valid) continue;  // padding rows of a partial last tile

      // butterfly identity of this row at stage j
      uint32_t g, nrest, kk;
      if (j == 1) {
        kk = 0;
        if (p.in_contig) {
          g = row >> (4 * (S - 1));
          nrest = row & (Lq - 1);
        } else {
          nrest = row / (uint32_t)G;
          g = row - nrest * (uint32_t)G;
        }
      } else {
        const uint32_t kkmask = (1u << (4 * (j - 1))) - 1u;
        kk = row & kkmask;
        const uint32_t q = row >> (4 * (j - 1));
        g = q >> (4 * (S - j));
        nrest = q & ((1u << (4 * (S - j))) - 1u);
      }

      if (!last) {
        // twiddle W_{L_j}^{k nrest}, L_j = 16^{S-j+1}; table is W_N
        const uint64_t e1 = (uint64_t)nrest << (log2RX + 4 * (j - 1));
        const float2 w = tw_lookup(p.tw_lo, p.tw_hi, e1, p.log2N, p.tw_log2S);
        float2 tw = w;
#pragma unroll
        for (int k = 1; k < 16; ++k) {
          const float xr = re[k], xi = im[k];
          re[k] = fmaf(xr, tw.x, -xi * tw.y);
          im[k] = fmaf(xr, tw.y, xi * tw.x);
          tw = cmulf(tw, w);
        }
        const int sh = 4 * (S - j - 1);
        const uint32_t nnext = nrest >> sh;
        const uint32_t nlow = nrest & ((1u << sh) - 1u);
        const uint32_t dr = ((((g << sh) + nlow) << (4 * j)) + (kk << 4));
        if constexpr (!SPLIT) {
          uint4 r0 = make_uint4(f2h2(re[0], re[1]), f2h2(re[2], re[3]), f2h2(re[4], re[5]), f2h2(re[6], re[7]));
          uint4 r1 = make_uint4(f2h2(re[8], re[9]), f2h2(re[10], re[11]), f2h2(re[12], re[13]), f2h2(re[14], re[15]));
          uint4 i0 = make_uint4(f2h2(im[0], im[1]), f2h2(im[2], im[3]), f2h2(im[4], im[5]), f2h2(im[6], im[7]));
          uint4 i1 = make_uint4(f2h2(im[8], im[9]), f2h2(im[10], im[11]), f2h2(im[12], im[13]), f2h2(im[14], im[15]));
          a_store8(A, dr, nnext, r0, i0);
          a_store8(A, dr + 8, nnext, r1, i1);
        } else {
          uint32_t hr[8], hi_[8], lr[8], li[8];
#pragma unroll
          for (int q2 = 0; q2 < 8; ++q2) {
            hr[q2] = f2h2(re[2 * q2], re[2 * q2 + 1]);
            hi_[q2] = f2h2(im[2 * q2], im[2 * q2 + 1]);
            float2 a = h2f(hr[q2]), b = h2f(hi_[q2]);
            lr[q2] = f2h2((re[2 * q2] - a.x) * 2048.0f, (re[2 * q2 + 1] - a.y) * 2048.0f);
            li[q2] = f2h2((im[2 * q2] - b.x) * 2048.0f, (im[2 * q2 + 1] - b.y) * 2048.0f);
          }
          uint8_t* Alo = A + tiles * kTileBytes;
          a_store8(A, dr, nnext, make_uint4(hr[0], hr[1], hr[2], hr[3]), make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]));
          a_store8(A, dr + 8, nnext, make_uint4(hr[4], hr[5], hr[6], hr[7]), make_uint4(hi_[4], hi_[5], hi_[6], hi_[7]));
          a_store8(Alo, dr, nnext, make_uint4(lr[0], lr[1], lr[2], lr[3]), make_uint4(li[0], li[1], li[2], li[3]));
          a_store8(Alo, dr + 8, nnext, make_uint4(lr[4], lr[5], lr[6], lr[7]), make_uint4(li[4], li[5], li[6], li[7]));
        }
      } else {
        // final stage: natural-order outputs into the staging copy
        uint32_t rev = 0;
        {
          uint32_t x = kk;
          for (int d = 0; d < S - 1; ++d) {
            rev = (rev << 4) | (x & 15u);
            x >>= 4;
          }
        }
        uint32_t c, k0;
        if (p.in_contig) {
          c = g >> log2RX;
          k0 = g & (RX - 1);
        } else {
          k0 = g / (uint32_t)C;
          c = g - k0 * (uint32_t)C;
        }
        const uint32_t kbase = k0 + (rev << log2RX);       // output index for k_S = 0
        const uint32_t kstep = Lq << log2RX;               // output index step per k_S
        if (p.otw_level) {
          const int64_t t = t0 + c;
          const int64_t col = (p.otw_level == 1) ? (t & ((int64_t(1) << p.log2I1) - 1))
                                                 : ((t >> p.log2I1) & ((int64_t(1) << p.log2I2) - 1));
          const float2 w0 = tw_lookup(p.otw_lo, p.otw_hi, (uint64_t)col * kbase, p.otw_log2M, p.otw_log2S);
          const float2 ws = tw_lookup(p.otw_lo, p.otw_hi, (uint64_t)col * kstep, p.otw_log2M, p.otw_log2S);
          float2 tw = w0;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float xr = re[k], xi = im[k];
            re[k] = fmaf(xr, tw.x, -xi * tw.y);
            im[k] = fmaf(xr, tw.y, xi * tw.x);
            tw = cmulf(tw, ws);
          }
        }
        uint32_t* stg = reinterpret_cast<uint32_t*>(A);
        const uint32_t P = (uint32_t)C * (uint32_t)N;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const uint32_t ko = kbase + kstep * k;
          const uint32_t idx = p.out_contig ? (c * (uint32_t)N + ko) : (ko * (uint32_t)C + c);
          if constexpr (!SPLIT) {
            stg[stg_word(idx)] = f2h2(re[k], im[k]);
          } else {
            const uint32_t h = f2h2(re[k], im[k]);
            const float2 hf = h2f(h);
            stg[stg_word(idx)] = h;
            stg[P + stg_word(idx)] = f2h2((re[k] - hf.x) * 2048.0f, (im[k] - hf.y) * 2048.0f);
          }
        }
      }
    }
    fence_proxy_async_smem();
    tc_fence_before_sync();
    __syncthreads();
  }

  if (ok) {
    // copy-out: staging (natural order, chunk-swizzled) -> global, 16-byte stores
    const uint4* stg = reinterpret_cast<const uint4*>(A);
    const uint32_t P = (uint32_t)C * (uint32_t)N;
    const uint32_t nchunks = P >> 2;
    if (p.out_contig) {
      const uint32_t cpt = (uint32_t)N >> 2;  // chunks per transform
      for (uint32_t q = tid; q < nchunks; q += kThreads) {
        const uint32_t c = q / cpt;
        const uint32_t e0 = (q - c * cpt) << 2;
        const int64_t t = t0 + c;
        if (t < p.T) {
          const int64_t off = side_base(p.out_l, t, p.log2I1, p.log2I2) + e0;
          const uint32_t pq = q ^ ((q >> 3) & 7u);
          *reinterpret_cast<uint4*>(p.out + off) = stg[pq];
          if constexpr (SPLIT) *reinterpret_cast<uint4*>(p.out + p.out_plane + off) = stg[nchunks + pq];
        }
      }
    } else {
      const uint32_t cpr = (uint32_t)C >> 2;  // chunks per output element index
      const int64_t base0 = side_base(p.out_l, t0, p.log2I1, p.log2I2);
      for (uint32_t q = tid; q < nchunks; q += kThreads) {
        const uint32_t k = q / cpr;
        const uint32_t cc = (q - k * cpr) << 2;
        const int64_t off = base0 + cc + (int64_t)k * p.out_l.es;
        const uint32_t pq = q ^ ((q >> 3) & 7u);
        *reinterpret_cast<uint4*>(p.out + off) = stg[pq];
        if constexpr (SPLIT) *reinterpret_cast<uint4*>(p.out + p.out_plane + off) = stg[nchunks + pq];
      }
    }
  }

  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after_sync();
    tmem_dealloc(tmem, (uint32_t)p.tmem_cols);
  }
}

}  // namespace tcfft
