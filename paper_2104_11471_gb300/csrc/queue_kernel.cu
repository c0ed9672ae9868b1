// Persistent ragged executor: every pass of a ragged plan in one launch.
//
// A plan's passes (Sec. 3.1: the execution function runs the chosen merging
// kernels in turn) become items of a device work queue: item (pass, slot) is
// the share of the pass that one CTA of that pass's own launch would run --
// chunks slot, slot + G, slot + 2G, ... (G = the pass's grid), with the pass
// kernel's prefetching loads and tensor-map stores.  Items are laid out level
// by level: every slot of the first pass of every shape group, then of the
// second, and so on.  A CTA claims the next item with an atomic counter,
// waits until every slot of the pass it depends on (the previous pass of its
// group) is counted done, runs the slot and counts it done.  Items are
// claimed in queue order and every dependency points to earlier items, so a
// claimed item only ever waits on items already held by running CTAs.  Each
// wait is bounded: when it runs out the launch reports TCFFT_ERR_TIMEOUT,
// raises an abort flag, and every later item is skipped instead of waited for.
//
// Cross-CTA ordering: a slot's outputs (per-thread stores, or tensor-map
// stores waited for) are fenced (async proxy, then device scope) before the
// slot is counted; a dependent slot acquires the counter and fences the async
// proxy before its first tensor-map load; synchronous loads go through L2
// (ld.global.cg).  Plain FP16 passes of every length and layout mode.
#include "pass_kernel.cuh"
#include "pass_setup.h"

namespace tcfft {

namespace {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int LOG2N, int MODE>
__device__ __noinline__ bool queue_slot(const PassParams& p, const PassParams& maps, int64_t slot, int64_t nslots,
                                        PassCta& cta, bool new_images) {
  return pass_body<PassCfg<LOG2N, MODE, false>, true>(p, maps, slot, nslots, cta, new_images, false);
}

template <int MODE, int LOG2N>
__device__ __forceinline__ bool queue_dispatch(const PassParams& p, const PassParams& maps, int64_t slot,
                                               int64_t nslots, PassCta& cta, bool new_images) {
  if constexpr (LOG2N < kMinLog2Pass) {
    return false;
  } else {
    if (p.log2N == LOG2N) return queue_slot<LOG2N, MODE>(p, maps, slot, nslots, cta, new_images);
    return queue_dispatch<MODE, LOG2N - 1>(p, maps, slot, nslots, cta, new_images);
  }
}

__global__ void __launch_bounds__(128, 4) queue_kernel(const __grid_constant__ QueueParams q) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* A = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  PassParams* sp = reinterpret_cast<PassParams*>(A + q.a_bytes);  // 1 KB aligned
  int* s_item = reinterpret_cast<int*>(sp + 1);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(s_item + 4);
  uint64_t* lbar = mbar + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(smem_u32(mbar), 1);
    mbar_init(smem_u32(lbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((tid >> 5) == 0) {
    tmem_alloc(smem_u32(tslot), (uint32_t)q.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  PassCta cta{A, mbar, lbar, *tslot, 0u, 0u};
  griddep_wait();

  int last = -1;
  for (;;) {
    if (tid == 0) *s_item = atomicAdd(q.head, 1);
    __syncthreads();
    const int it = *s_item;
    if (it >= q.nitems) break;
    const int2 item = q.items[it];
    const int pass = item.x;
    bool skip = false;
    if (tid == 0) {
      skip = *reinterpret_cast<volatile const int*>(q.abort) != 0;
      const int d = q.dep[pass];
      if (!skip && d >= 0) {
        const int need = q.nchunks[d];
        const long long t0 = clock64();
        while (ld_acquire(q.done + d) < need) {
          if (*reinterpret_cast<volatile const int*>(q.abort) != 0) {
            skip = true;
            break;
          }
          if (clock64() - t0 > q.wait_limit) {
            atomicExch(q.status, kDevErrTimeout);
            atomicExch(q.abort, 1);
            skip = true;
            break;
          }
        }
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");  // before tensor-map loads of that data
      }
    }
    skip = __syncthreads_or(skip);
    if (!skip) {
      const bool fresh = pass != last;
      if (fresh) {
        // the pass's parameters into shared memory (read often by every thread)
        const uint32_t* src = reinterpret_cast<const uint32_t*>(q.passes + pass);
        uint32_t* dst = reinterpret_cast<uint32_t*>(sp);
        for (int i = tid; i < (int)(sizeof(PassParams) / 4); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
      }
      const PassParams& p = *sp;
      const PassParams& maps = q.passes[pass];  // tensor maps in global memory
      const int mode = (p.in_l.es == 1) ? ((p.out_l.es == 1) ? kModeContig : kModeToStrided) : kModeStrided;
      bool ok;
      if (mode == kModeContig)
        ok = queue_dispatch<kModeContig, max_log2_pass(kModeContig, false)>(p, maps, item.y, q.nchunks[pass], cta, fresh);
      else if (mode == kModeStrided)
        ok = queue_dispatch<kModeStrided, max_log2_pass(kModeStrided, false)>(p, maps, item.y, q.nchunks[pass], cta,
                                                                             fresh);
      else
        ok = queue_dispatch<kModeToStrided, max_log2_pass(kModeToStrided, false)>(p, maps, item.y, q.nchunks[pass],
                                                                                 cta, fresh);
      if (!ok && tid == 0) atomicExch(q.abort, 1);  // the timed-out wait wrote the status
      last = pass;
    }
    // this slot's outputs (tensor-map stores completed in the body) are
    // visible before the slot is counted
    if (tid == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(q.done + pass, 1);
  }

  tc_fence_before_sync();
  __syncthreads();
  if ((tid >> 5) == 0) {
    tc_fence_after_sync();
    tmem_dealloc(cta.tmem, (uint32_t)q.tmem_cols);
  }
}

}  // namespace

const void* queue_fn() { return reinterpret_cast<const void*>(&queue_kernel); }

}  // namespace tcfft
