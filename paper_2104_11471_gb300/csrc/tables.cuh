// Plan-time table generators (FP64 on the GPU, rounded once): twiddle
// tables, per-stage epilogue twiddles and the radix-16 DFT matrix images.
// Included by each translation unit that builds tables (internal linkage).
#pragma once
#include <cuda_fp16.h>
#include <cstdint>

#include "pass_params.h"

namespace tcfft {

// W_M^m = exp(-2 pi i m / M) in FP64 (sincospi), rounded once to FP32.
static __global__ void twiddle_table_kernel(float2* lo, float2* hi, int log2M, int log2S) {
  const int64_t S = int64_t(1) << log2S;
  const int64_t H = int64_t(1) << (log2M - log2S);
  const int64_t M = int64_t(1) << log2M;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S + H;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = (i < S) ? i : (i - S) * S;  // exponent
    double s, c;
    sincospi(-2.0 * (double)m / (double)M, &s, &c);
    const float2 w = make_float2((float)c, (float)s);
    if (i < S) lo[i] = w; else hi[i - S] = w;
  }
}

// Epilogue twiddles of a pass of length N = RX * 16^S (L = 16^S, LQ = L/16):
// the twiddle of output k of a butterfly row is a * b^k, per row key
//   stage 1, key k0 * LQ + nrest (k0 < RX, nrest < LQ):
//       a = W_N^{k0 nrest}, b = W_L^{nrest}, so a b^k = W_N^{nrest (k0 + RX k)}
//   stage j = 2..S-1, key RX*LQ + sum_{2<=i<j} 16^{S-i} + nrest:
//       a = 1, b = W_{L_j}^{nrest}, L_j = 16^{S-j+1}.
// Two parts: rows float4 (a, b), one per key, for the epilogues that advance
// a b^k by packed multiplies (consecutive keys 16 bytes apart, as the lanes
// of a contiguous chunk read them); then 8 float4 per key, entry
// rows + 8 key + i = (Re w_{2i}, Re w_{2i+1}, Im w_{2i}, Im w_{2i+1}) with
// w_k = a b^k, for the epilogues whose lanes share keys (loads then
// broadcast).  Exponents reduced exactly in integers, FP64 sincospi, each
// value rounded once to FP32.  One thread per entry.
static __global__ void stage_twiddle_kernel(float4* out, int log2N, int rows) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * kStageSlots) return;
  const int row = idx < rows ? idx : (idx - rows) >> 3;
  const int slot = idx < rows ? 0 : 1 + ((idx - rows) & 7);
  const int S = log2N / 4, RX = 1 << (log2N % 4), LQ = 1 << (4 * (S - 1));
  int64_t k0, nrest, n;  // stage 1: a b^k = W_n^{nrest (k0 + RX k)}; else W_n^{nrest k}
  int64_t step;          // exponent step per output k: RX nrest (stage 1) or nrest
  if (row < RX * LQ) {
    k0 = row / LQ;
    nrest = row % LQ;
    n = (int64_t)RX * 16 * LQ;
    step = (int64_t)RX * nrest;
  } else {
    int j = 2, off = RX * LQ;
    while (j < S - 1 && row >= off + (1 << (4 * (S - j)))) {
      off += 1 << (4 * (S - j));
      ++j;
    }
    k0 = 0;
    nrest = row - off;
    n = int64_t(1) << (4 * (S - j + 1));
    step = nrest;
  }
  const int64_t e_a = (k0 * nrest) % n;  // exponent of a (w_0)
  double s0, c0, s1, c1;
  if (slot == 0) {
    sincospi(-2.0 * (double)e_a / (double)n, &s0, &c0);         // a
    sincospi(-2.0 * (double)(step % n) / (double)n, &s1, &c1);  // b = W_n^{step}
    out[idx] = make_float4((float)c0, (float)s0, (float)c1, (float)s1);
    return;
  }
  const int i = slot - 1;
  const int64_t e0 = (e_a + step * (2 * i)) % n, e1 = (e_a + step * (2 * i + 1)) % n;
  sincospi(-2.0 * (double)e0 / (double)n, &s0, &c0);
  sincospi(-2.0 * (double)e1 / (double)n, &s1, &c1);
  out[idx] = make_float4((float)c0, (float)c1, (float)s0, (float)s1);
}

// B operands of the radix-16 stage: the real 32 x 32 form of a complex
// 16 x 16 matrix M,
//   B[k][n]: k < 16 -> Re of input k, k >= 16 -> Im of input k-16;
//            n < 16 -> Re of output n, n >= 16 -> Im of output n-16;
//   [[Re M, Im M], [-Im M, Re M]].
// Scaled plans (1/N spread over the stages) use M / 16.
// Image k0 (k0 < RX) holds M[m][l] = W_16^{l m} W_{16 RX}^{k0 m}
// = W_{16 RX}^{m (RX l + k0)}: the DFT matrix F_16 with the leading-radix
// twiddle factor of input n_1 = m folded in (image 0 is plain F_16).
// Stored K-major without swizzle: core matrices of 8 (n) x 8 (k) halves,
// K-groups 128 B apart, N-groups 512 B apart.  Images 0..7 hold the FP16
// values, images 8..15 the low parts fp16((v - hi) * 2^11) for split precision.
static __global__ void dft_b_kernel(__half* img, int RX, double scale = 1.0) {
  const int k0 = blockIdx.x;    // one block per image
  const int idx = threadIdx.x;  // 1024 threads: one per (k, n)
  const int k = idx >> 5, n = idx & 31;
  const int m = k & 15, l = n & 15;
  const int den = 16 * RX;
  double s, c;
  sincospi(-2.0 * (double)((m * (RX * l + k0)) % den) / (double)den, &s, &c);  // W = c + i s
  double v;
  if (k < 16) v = (n < 16) ? c : s;
  else v = (n < 16) ? -s : c;
  v *= scale;  // 1/16 for scaled plans: exact in FP16
  const int off = k0 * 1024 + (n >> 3) * 256 + (k >> 3) * 64 + (n & 7) * 8 + (k & 7);  // halves
  const __half h = __double2half(v);
  img[off] = h;
  img[8 * 1024 + off] = __float2half_rn((float)((v - (double)__half2float(h)) * 2048.0));
}

}  // namespace tcfft
