// Fused 2D pass: a whole S x S matrix (S = 2^LOG2S) per cluster of CTAs, its
// rows and columns transformed on chip between one HBM read and one write.
//
// Method (arXiv 2104.11471, Sec. 3.1 "Support batched FFT and 2D FFT"): the
// 2D DFT is the 1D DFT of every row followed by the 1D DFT of every column.
// The paper runs the two as separate strided batched passes through global
// memory; on GB300 a matrix of up to 2^18 points fits the distributed shared
// memory of one cluster (at most 16 CTAs), so the row results go to the
// columns' owners directly:
//  * phase 1: CTA r (of K) bulk-copies its S/K contiguous rows into RAW and
//    runs the row stages (pass kernel stage loop, radix-16 on the tensor
//    cores); each final output (row e, column ky) is stored straight into
//    the RAW buffer of CTA ky / (S/K), word e * (S/K) + ky mod (S/K), with
//    st.shared::cluster (the 16-byte slot XOR the 128-byte line index
//    modulo 8 spreads the column-phase reads over the banks);
//  * cluster barrier;
//  * phase 2: every CTA runs the column stages on its S/K columns (strided
//    stage-1 reads from RAW) and stores them through the staging copy.
// Every CTA of a cluster iterates over the same matrices and calls the
// cluster barrier the same number of times; a timed-out wait only skips
// work, never a barrier.
#pragma once
#include "pass_kernel.cuh"

namespace tcfft {

template <int LOG2S, bool SPLIT>
__global__ void __launch_bounds__(kThreads, (PassCfg<LOG2S, kModeContig, SPLIT>::MINB)) fused2d_kernel(const __grid_constant__ Fused2DParams f) {
  using K1 = PassCfg<LOG2S, kModeContig, SPLIT>;   // rows
  using K2 = PassCfg<LOG2S, kModeStrided, SPLIT>;  // columns
  const PassParams& p1 = f.row;
  const PassParams& p2 = f.col;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* A = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tiles = p1.tiles;                        // both phases: P points per CTA
  const int log2C = p1.log2C;                        // rows (phase 1) = columns (phase 2) per CTA
  const int C = 1 << log2C;
  const uint32_t P = (uint32_t)C << LOG2S;           // points per CTA and plane
  uint8_t* RAW = A + K1::PLANES * tiles * kTileBytes;
  uint8_t* Bs = RAW + K1::PLANES * P * 4u;           // one image set: both phases have length S
  constexpr int NB = K1::FOLD ? K1::RX : 1;
  const uint32_t slack = (uint32_t)(A - smem_raw);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(slack >= 64 ? A - 64 : Bs + K1::PLANES * NB * kBImageBytes);
  uint64_t* lbar = mbar + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x;

  load_dft_images<K1>(p1, Bs);
  if (tid == 0) {
    mbar_init(smem_u32(mbar), 1);
    mbar_init(smem_u32(lbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((tid >> 5) == 0) {
    tmem_alloc(smem_u32(tslot), (uint32_t)p1.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  StageCtx cx{A, smem_u32(A), smem_u32(Bs), *tslot, smem_u32(mbar), 0u};
  const uint32_t raw_s = smem_u32(RAW), lbar_s = smem_u32(lbar);
  const uint32_t* raw32 = reinterpret_cast<const uint32_t*>(RAW);
  const uint32_t rank = cluster_ctarank();
  const int64_t cid = blockIdx.x >> f.log2K, ncl = gridDim.x >> f.log2K;
  uint32_t lphase = 0;
  bool ok = true, pending = false;

  griddep_wait();  // the input may be the previous kernel's output

  for (int64_t m = cid; m < f.batch; m += ncl) {
    if (m + ncl >= f.batch) griddep_launch_dependents();
    // first element of matrix m: dense batch, or a transform-offset table
    // (ragged batches)
    const int64_t mb_in = p1.in_l.toff ? __ldg(p1.in_l.toff + m) : (m << (2 * LOG2S));
    const int64_t mb_out = p2.out_l.toff ? __ldg(p2.out_l.toff + m) : (m << (2 * LOG2S));
    // ---- phase 1: rows rank*C .. rank*C + C - 1 of matrix m
    const int64_t t0r = (m << LOG2S) + ((int64_t)rank << log2C);
    if (ok) {
      fence_proxy_async_smem();  // RAW was read by this CTA's last column load
      __syncthreads();
      issue_raw_copy<K1>(p1, raw_s, lbar_s, p1.in + in_words<K1>(p1) * (mb_in + ((int64_t)rank << (log2C + LOG2S))),
                         t0r, log2C, C);
      pending = true;
      bool got = true;
      if (tid == 0) got = mbar_wait_bounded(lbar_s, lphase, kWaitLimitCycles);
      if (__syncthreads_or(!got)) {
        if (tid == 0) atomicExch(p1.status, kDevErrTimeout);
        ok = false;
      } else {
        lphase ^= 1u;
        pending = false;
        load_stage1<K1, true>(p1, A, raw32, raw32 + P, 1u, log2C, C);
      }
    }
    fence_proxy_async_smem();
    tc_fence_before_sync();
    cluster_sync();  // every CTA has consumed its RAW: peers may write into it
    tc_fence_after_sync();
    if (ok) {
      // row e = rank*C + c, output column ky -> CTA ky >> log2C, RAW word
      // e * C + (ky & (C - 1)), 16-byte slot ^= (byte offset >> 7) & 7
      auto fin1 = [&](uint32_t c, uint32_t kbase, float2 (&X)[8], float2 (&Y)[8]) {
        constexpr uint32_t kstep = (uint32_t)K1::LQ << K1::LOG2RX;
        const uint32_t e = (rank << log2C) + c;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const uint32_t ky = kbase + (uint32_t)i * kstep;
          const float re = (i & 1) ? X[i >> 1].y : X[i >> 1].x;
          const float im = (i & 1) ? Y[i >> 1].y : Y[i >> 1].x;
          uint32_t bo = ((e << log2C) + (ky & (uint32_t)(C - 1))) << 2;
          bo ^= ((bo >> 7) & 7u) << 4;
          const uint32_t dst = mapa_shared(raw_s + bo, ky >> log2C);
          const uint32_t h = f2h2(re, im);
          st_cluster_u32(dst, h);
          if constexpr (SPLIT) st_cluster_u32(dst + P * 4u, split_lo(re, im, h));
        }
      };
      ok = run_stages<K1>(p1, cx, tiles, log2C, fin1);
    }
    cluster_sync();  // every row output has reached its column's owner
    // ---- phase 2: columns rank*C .. rank*C + C - 1 of matrix m
    if (ok) {
      load_stage1<K2, true>(p2, A, raw32, raw32 + P, (uint32_t)C, log2C, C);
      fence_proxy_async_smem();
      tc_fence_before_sync();
      __syncthreads();
      auto fin2 = [&](uint32_t c, uint32_t kbase, float2 (&X)[8], float2 (&Y)[8]) {
        if (p2.conj_out) {
#pragma unroll
          for (int i = 0; i < 8; ++i) Y[i] = make_float2(-Y[i].x, -Y[i].y);
        }
        staging_store<K2>(p2, A, P, log2C, c, kbase, X, Y);
      };
      ok = run_stages<K2>(p2, cx, tiles, log2C, fin2);
    }
    if (ok) {
      const int64_t t0c = (m << LOG2S) + ((int64_t)rank << log2C);
      uint32_t* gout = p2.out + out_words<K2>(p2) * (mb_out + ((int64_t)rank << log2C));
      copy_out<K2>(p2, A, gout, t0c, C, log2C);
    }
    __syncthreads();  // staging (= A) is rewritten by the next matrix
  }

  if (p2.out_tma && tid == 0) bulk_wait_all();
  if (pending) (void)mbar_wait_bounded(lbar_s, lphase, kWaitLimitCycles);
  cluster_sync();  // no peer writes into this CTA's shared memory any more
  tc_fence_before_sync();
  __syncthreads();
  if ((tid >> 5) == 0) {
    tc_fence_after_sync();
    tmem_dealloc(cx.tmem, (uint32_t)p1.tmem_cols);
  }
}

}  // namespace tcfft
