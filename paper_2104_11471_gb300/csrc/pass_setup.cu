// Launch geometry of fused passes: see pass_setup.h.
#include "pass_setup.h"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

namespace tcfft {

const void* pass_fn_m0_plain(int log2N);
const void* pass_fn_m1_plain(int log2N);
const void* pass_fn_m2_plain(int log2N);
const void* pass_fn_m0_split(int log2N);
const void* pass_fn_m1_split(int log2N);
const void* pass_fn_m2_split(int log2N);

namespace {
// points per CTA (C * N) limits: shared memory holds 4 B (plain) or 8 B
// (split) per point and TMEM 32 (plain) or 64 (split) FP32 columns per 2048.
constexpr int64_t kCapPlain = 32768;
constexpr int64_t kCapSplit = 16384;
}  // namespace

cudaError_t launch_pass(const void* fn, dim3 grid, int threads, size_t smem, cudaStream_t s, void** args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}
}  // namespace

namespace {
// 5-D tensor map (t1, element, t2, t3, plane) of one strided side; boxes of
// C x min(L, 256) elements; false when the layout does not fit a map
bool encode_side_map(CUtensorMap* map, const PassParams& p, const SideLayout& l, const void* base,
                     int64_t plane, bool f32, bool split, CUtensorMapSwizzle swz) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  const uint64_t elem = f32 ? 8 : 4;
  const int64_t I1 = int64_t(1) << p.log2I1;
  const bool lvl2 = p.log2I2 < 40;  // a bounded second index level
  const int64_t I2 = lvl2 ? (int64_t(1) << p.log2I2) : 0;
  const int64_t L = int64_t(1) << p.log2N;
  const int64_t T = p.T;
  // dims (innermost first): t1, element, t2, t3, plane; size-1 dims get a
  // 16-byte stride that is never stepped
  cuuint64_t dims[5], strides[4];
  dims[0] = (cuuint64_t)I1;
  dims[1] = (cuuint64_t)L;
  strides[0] = (cuuint64_t)l.es * elem;
  if (lvl2) {
    dims[2] = (cuuint64_t)I2;
    dims[3] = (cuuint64_t)(T / (I1 * I2));
  } else {
    dims[2] = (cuuint64_t)(T / I1);
    dims[3] = 1;
  }
  strides[1] = (cuuint64_t)l.s2 * elem;
  strides[2] = (cuuint64_t)l.s3 * elem;
  dims[4] = (split && !f32) ? 2 : 1;
  strides[3] = (cuuint64_t)plane * 4;
  for (int i = 2; i <= 4; ++i)
    if (dims[i] == 1) strides[i - 1] = 16;
  bool ok = enc != nullptr && T % I1 == 0 && (!lvl2 || T % (I1 * I2) == 0);
  for (int i = 0; i < 4 && ok; ++i) ok = strides[i] % 16 == 0 && strides[i] > 0 && strides[i] < (1ull << 40);
  for (int i = 0; i < 5 && ok; ++i) ok = dims[i] >= 1 && dims[i] <= (1ull << 32);
  const cuuint32_t box[5] = {(cuuint32_t)(1u << p.log2C), (cuuint32_t)std::min<int64_t>(L, 256), 1, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  ok = ok && box[0] <= 256 && (box[0] * elem) % 16 == 0;
  if (!ok) return false;
  return enc(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 5,
             const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

void encode_out_map(PassParams& p, bool split) {
  if (!p.out_tma) return;
  if (p.out_l.es == 1) {
    // contiguous output: the output buffer as rows of 32 points (128 bytes) in
    // the 128-byte swizzle; boxes of up to 256 rows per plane
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    const uint64_t points = (uint64_t)p.T << p.log2N;
    const uint64_t P = (uint64_t)1 << (p.log2C + p.log2N);
    const cuuint64_t dims[5] = {32, points / 32, (cuuint64_t)(split ? 2 : 1), 1, 1};
    const cuuint64_t strides[4] = {128, split ? (cuuint64_t)p.out_plane * 4 : 16, 16, 16};
    const cuuint32_t box[5] = {32, (cuuint32_t)std::min<uint64_t>(P / 32, 256), 1, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const bool ok = enc != nullptr && !(split && p.out_f32) && points % 32 == 0 && P % 32 == 0 &&
                    points / 32 < (1ull << 31) &&  // row coordinates are 32-bit
                    strides[1] % 16 == 0 && strides[1] < (1ull << 40) &&
                    enc(&p.out_map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 5, p.out, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    if (!ok) p.out_tma = 0;
    return;
  }
  // the staging rows are C * 4 bytes; the swizzle span matches them
  const int rowb = 4 << p.log2C;
  const CUtensorMapSwizzle swz = rowb == 32    ? CU_TENSOR_MAP_SWIZZLE_32B
                                 : rowb == 64  ? CU_TENSOR_MAP_SWIZZLE_64B
                                 : rowb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                               : CU_TENSOR_MAP_SWIZZLE_NONE;
  const bool ok = !(split && p.out_f32) && swz != CU_TENSOR_MAP_SWIZZLE_NONE && p.log2N >= 8 &&
                  encode_side_map(&p.out_map, p, p.out_l, p.out, p.out_plane, false, split, swz);
  if (!ok) p.out_tma = 0;
}

void encode_in_map(PassParams& p, bool split) {
  p.in_swz = 0;
  if (!p.in_tma) return;
  // FP16 planes: rows of C x 4 bytes land in the matching 32/64/128-byte
  // swizzle when every box and plane of the raw buffer starts on a 1 KB line
  const bool f32 = split && p.in_f32;
  const int rowb = 4 << p.log2C;
  const int64_t P = int64_t(1) << (p.log2C + p.log2N);
  int swz = 0;
  if (!f32 && p.log2N >= 6 && (P * 4) % 1024 == 0) swz = rowb == 32 ? 1 : (rowb == 64 ? 2 : (rowb == 128 ? 3 : 0));
  if (env_int("TCFFT_NO_IN_SWIZZLE", 0)) swz = 0;  // debugging override
  const CUtensorMapSwizzle mode = swz == 1   ? CU_TENSOR_MAP_SWIZZLE_32B
                                  : swz == 2 ? CU_TENSOR_MAP_SWIZZLE_64B
                                  : swz == 3 ? CU_TENSOR_MAP_SWIZZLE_128B
                                             : CU_TENSOR_MAP_SWIZZLE_NONE;
  if (encode_side_map(&p.in_map, p, p.in_l, p.in, p.in_plane, f32, split, mode)) {
    p.in_swz = swz;
    return;
  }
  if (swz && encode_side_map(&p.in_map, p, p.in_l, p.in, p.in_plane, f32, split, CU_TENSOR_MAP_SWIZZLE_NONE))
    return;
  p.in_tma = 0;
}

int ilog2(int64_t v) {
  int r = 0;
  while ((int64_t(1) << r) < v) ++r;
  return r;
}
bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return (v && *v) ? std::atoi(v) : dflt;
}

const void* pass_fn(int log2N, int mode, bool split) {
  if (log2N < kMinLog2Pass || log2N > max_log2_pass(mode, split)) return nullptr;
  switch (mode) {
    case kModeContig: return split ? pass_fn_m0_split(log2N) : pass_fn_m0_plain(log2N);
    case kModeStrided: return split ? pass_fn_m1_split(log2N) : pass_fn_m1_plain(log2N);
    default: return split ? pass_fn_m2_split(log2N) : pass_fn_m2_plain(log2N);
  }
}

namespace {
// One candidate geometry: `threads` per CTA (256 or 128), prefetching the next
// chunk into a raw buffer (async = 1) or loading synchronously (async = 0).
tcfft_status geometry_try(PassLaunch& ps, int64_t L, int64_t T, int64_t I1, int64_t I2, Side in, Side out,
                          bool split, int64_t target_points, int threads, int async, bool share_sm) {

  std::memset(&ps.p, 0, sizeof(ps.p));
  PassParams& p = ps.p;
  const int log2L = ilog2(L);
  p.log2N = log2L;
  const bool in_contig = in.es == 1, out_contig = out.es == 1;
  int mode;
  if (in_contig && out_contig) mode = kModeContig;
  else if (!in_contig && !out_contig) mode = kModeStrided;
  else if (in_contig) mode = kModeToStrided;
  else return TCFFT_ERR_INVALID_SIZE;
  // layout contract of the kernel (see SideLayout); a contiguous side with a
  // transform-offset table and I1 == 1 gathers/scatters transform by transform
  // per-transform ("gather"/"scatter") mode: the transforms of a CTA are not
  // one contiguous block -- each has its own offset (table) or they sit s1 != L apart
  const bool in_gather = in_contig && ((in.toff && I1 == 1) || (!in.toff && in.s1 != L));
  const bool out_scatter = out_contig && ((out.toff && I1 == 1) || (!out.toff && out.s1 != L));
  if ((in_contig && in.s1 != L && !in_gather) || (!in_contig && in.s1 != 1)) return TCFFT_ERR_INVALID_SIZE;
  if ((out_contig && out.s1 != L && !out_scatter) || (!out_contig && out.s1 != 1))
    return TCFFT_ERR_INVALID_SIZE;
  if (in.es * L >= (int64_t(1) << 31) || out.es * L >= (int64_t(1) << 31)) return TCFFT_ERR_INVALID_SIZE;
  ps.fn = pass_fn(log2L, mode, split);
  if (!ps.fn) return TCFFT_ERR_INVALID_SIZE;
  const int64_t cap = split ? kCapSplit : kCapPlain;
  // the default chunk sizes scale with the threads per CTA
  ps.threads = threads;
  const int64_t tscale = ps.threads / 128;  // 1 or 2
  int64_t C;
  if (mode == kModeContig) {
    int64_t target = (split ? 2048 : 4096) * tscale;
    const int tgt_env = env_int("TCFFT_POINTS_PER_CTA", 0);  // tuning override
    if (tgt_env >= 2048 && is_pow2(tgt_env)) target = tgt_env;
    if (target_points >= 2048 && is_pow2(target_points)) target = target_points;
    C = std::max<int64_t>(1, target / L);
    if (!(in_gather || out_scatter))
      while (C > 1 && I1 % C != 0) C /= 2;
  } else {
    // strided side: C adjacent transforms per element index, C | I1, C >= 8
    int64_t soft = (split ? 2048 : 4096) * tscale;
    const int soft_env = env_int("TCFFT_STRIDED_POINTS", 0);  // tuning override
    if (soft_env >= 1024 && is_pow2(soft_env)) soft = soft_env;
    if (target_points >= 1024 && is_pow2(target_points)) soft = target_points;
    C = 0;
    for (int64_t c : {32, 16, 8}) {
      if (I1 % c == 0 && c * L <= soft) {
        C = c;
        break;
      }
    }
    if (C == 0 && I1 % 8 == 0 && 8 * L <= cap) C = 8;
    if (C == 0) return TCFFT_ERR_INVALID_SIZE;
    // bring small transforms up to at least one full MMA tile when possible
    while (C * L < 2048 && I1 % (2 * C) == 0 && 2 * C * L <= cap) C *= 2;
  }
  // small plans: fewer transforms per CTA until every SM has a chunk (down
  // to the layout minimum), so that a single large transform spreads over
  // the GPU and each CTA's chunk latency is short
  {
    int sms_now = 0, dev_now = 0;
    cudaGetDevice(&dev_now);
    cudaDeviceGetAttribute(&sms_now, cudaDevAttrMultiProcessorCount, dev_now);
    const int64_t cmin = (mode == kModeContig) ? 1 : 8;
    while (C > cmin && (T + C - 1) / C < sms_now && target_points == 0) C /= 2;
  }
  // with two or more radix-16 stages and a leading radix, every 128-row
  // MMA tile must hold one k0: C * 16^{S-1} >= 128
  const int S = log2L / 4, RX = 1 << (log2L % 4);
  const bool fold = S >= 2 && RX > 1;
  if (fold) {
    const int64_t need = std::max<int64_t>(1, 128 >> (4 * (S - 1)));
    if (C < need) {
      if (I1 % need != 0 && !(in_gather || out_scatter)) return TCFFT_ERR_INVALID_SIZE;
      C = need;
    }
  }
  if (C * L > cap) return TCFFT_ERR_INVALID_SIZE;
  const int64_t P = C * L;
  p.log2C = ilog2(C);
  p.tiles = (int)((P + 2047) / 2048);
  const int planes = split ? 2 : 1;
  int cols = 32;
  while (cols < 32 * p.tiles * planes) cols *= 2;
  if (cols > 512) return TCFFT_ERR_INVALID_SIZE;
  p.tmem_cols = cols;
  p.T = T;
  p.log2I1 = ilog2(I1);
  p.log2I2 = ilog2(I2);
  p.in_l = SideLayout{in.s1, in.s2, in.s3, (uint32_t)in.es, in.toff};
  p.out_l = SideLayout{out.s1, out.s2, out.s3, (uint32_t)out.es, out.toff};
  p.prescale = 1.0f;
  p.in_gather = in_gather;
  p.out_scatter = out_scatter;
  p.nchunks = (T + C - 1) / C;
  // shared memory: A tiles (x planes), raw prefetch buffer (x planes, when it
  // fits), B image(s) and up to 1008 bytes of slack that aligns A to 1 KB
  // (the dynamic base is 16-byte aligned) and holds the two mbarriers and the
  // TMEM slot when it has 64 bytes to spare (else they follow the B images,
  // within the same 1008 bytes); padded so that shared memory, not TMEM
  // allocation, limits CTAs per SM.
  const size_t nb = fold ? (size_t)RX : 1;  // DFT matrix images per plane
  const size_t base = 1008 + (size_t)planes * p.tiles * kTileBytes + (size_t)planes * nb * kBImageBytes;
  const size_t raw = (size_t)planes * P * 4;
  const int ctas_tmem = 512 / cols;
  const size_t sm_total = 228 * 1024;
  const size_t per_cta_max = sm_total / ctas_tmem - 1024;
  // padded so that shared memory, not TMEM allocation, limits CTAs per SM
  auto padded = [&](size_t sm) { return sm < per_cta_max ? std::min<size_t>(per_cta_max, 227 * 1024) : sm; };
  // the attribute is a per-kernel upper bound shared by every pass (and plan)
  // that launches this kernel: always the largest, never the pass's own size
  if (cudaFuncSetAttribute(ps.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
    return TCFFT_ERR_CUDA;
  // ask for the largest shared-memory carveout so that several CTAs fit per SM
  if (cudaFuncSetAttribute(ps.fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
    return TCFFT_ERR_CUDA;
  // CTAs per SM from the kernel's registers, shared memory and threads
  // (register file allocated per warp in units of 256 registers)
  int dev = 0, sms = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaFuncAttributes fa0;
  if (cudaFuncGetAttributes(&fa0, ps.fn) != cudaSuccess) return TCFFT_ERR_CUDA;
  const int warp_regs = ((fa0.numRegs * 32 + 255) / 256) * 256;
  const int by_regs = regs_sm / (warp_regs * (ps.threads / 32));
  const int by_thr = thr_sm / ps.threads;
  auto occupancy = [&](size_t sm) {
    const int by_smem = smem_sm / (int)(sm + fa0.sharedSizeBytes + 1024);
    return std::min(ctas_tmem, std::min(by_regs, std::min(by_smem, by_thr)));
  };
  if (async && base + raw > 227 * 1024) return TCFFT_ERR_INVALID_SIZE;
  p.async_load = async;
  // strided input (no offset table) through tensor-map boxes when prefetching
  p.in_tma = (mode == kModeStrided && async && !in.toff && !env_int("TCFFT_NO_TMA", 0)) ? 1 : 0;
  // strided output of a two-stage pass through tensor-map stores (rows of
  // C * 4 = 32, 64 or 128 bytes in the map's swizzle).  Measured at 2^28
  // points: 256-point passes 9-13 % faster, 512 13 %, 1024 6 %; at 2048 the
  // swizzle's staging bank conflicts outweigh the saved stores (19 % slower).
  p.out_tma = (mode != kModeContig && log2L >= 8 && log2L <= env_int("TCFFT_TMA_STORE_MAX_LOG2", 10) &&
               !out.toff && !out_scatter && C >= 8 && C <= 32 && !env_int("TCFFT_NO_TMA", 0))
                  ? 1
                  : 0;
  // contiguous output of a three-stage pass (N >= 4096): the staging key is the
  // 128-byte swizzle there, so the chunk leaves through tensor-map stores too
  if (mode == kModeContig && log2L >= 12 && !out.toff && !out_scatter && !env_int("TCFFT_NO_TMA", 0) &&
      !env_int("TCFFT_NO_TMA_CONTIG_STORE", 0))
    p.out_tma = 1;
  const size_t smem = padded(async ? base + raw : base);
  if (smem > 227 * 1024) return TCFFT_ERR_INVALID_SIZE;
  ps.smem = smem;
  int occ = occupancy(smem);
  if (occ < 1) return TCFFT_ERR_INVALID_SIZE;
  const int occ_env = env_int("TCFFT_CTAS_PER_SM", 0);  // tuning override
  if (occ_env > 0) occ = std::min(occ, occ_env);
  if (share_sm) occ = std::max(1, occ / 2);  // leave room for other streams' kernels
  ps.grid = dim3((unsigned)std::min<int64_t>(p.nchunks, (int64_t)occ * sms));
  ps.occ = occ;
  ps.regs = fa0.numRegs;
  return TCFFT_OK;
}
}  // namespace

tcfft_status pass_geometry(PassLaunch& ps, int64_t L, int64_t T, int64_t I1, int64_t I2, Side in,
                           Side out, bool split, int64_t target_points, int force_threads, int force_async,
                           bool share_sm) {
  // The pass is latency-bound (each CTA runs a serial chain per chunk: load,
  // then per stage MMA issue, MMA completion, TMEM loads, epilogue, barrier):
  // pick the candidate with the most resident CTAs per SM (independent
  // chains), a synchronous load counting 0.75 of a prefetching CTA, then the
  // most resident warps.  Measured at 2^28 points: N = 256 at 6 x 128 threads
  // 0.38 ms vs 3 x 256 0.43 ms; N = 16384 at 2 x 256 synchronous 0.82 ms vs
  // 1 x 256 prefetching 1.11 ms and 2 x 128 synchronous 0.96 ms; split 4096-point
  // rows at 3 x 128 beat 2 x 256; 2^18 (length-512 passes) 3 x 256 prefetching
  // 1.25 ms vs 6 x 128 synchronous 1.51 ms.
  const int thr_env = force_threads ? force_threads : env_int("TCFFT_THREADS", 0);  // tuning override
  const int sync_env = force_async == 0 || env_int("TCFFT_SYNC_LOAD", 0);           // debugging override
  PassLaunch best;
  double best_score = -1.0;
  tcfft_status last = TCFFT_ERR_INVALID_SIZE;
  for (int thr : {256, 128}) {
    if ((thr_env == 128 || thr_env == 256) && thr != thr_env) continue;
    for (int as : {1, 0}) {
      if (as && sync_env) continue;
      if (!as && force_async == 1) continue;
      PassLaunch c = ps;
      const tcfft_status st = geometry_try(c, L, T, I1, I2, in, out, split, target_points, thr, as, share_sm);
      if (st != TCFFT_OK) {
        last = st;
        continue;
      }
      const double score = c.occ * (as ? 10.0 : 7.5) + c.occ * thr / 320.0;
      if (score > best_score) {
        best = c;
        best_score = score;
      }
    }
  }
  if (best_score < 0) return last;
  ps = best;
  return TCFFT_OK;
}

// ------------------------------------------------------------ fused 2D
tcfft_status fused2d_geometry(Fused2DLaunch& fl, int64_t S, int64_t batch, bool split, int force_log2K) {
  std::memset(&fl.f, 0, sizeof(fl.f));
  const int log2S = ilog2(S);
  fl.fn = fused2d_fn(log2S, split);
  if (!fl.fn || !is_pow2(S) || batch < 1) return TCFFT_ERR_INVALID_SIZE;
  const int64_t pts = S * S;
  const int64_t pmax = split ? 4096 : 8192;
  int log2K = 0;
  if (force_log2K >= 0) {
    log2K = force_log2K;
  } else {
    while ((pts >> log2K) > pmax && log2K < 4) ++log2K;
    if ((pts >> log2K) > pmax && (split || (pts >> log2K) > 2 * pmax)) return TCFFT_ERR_INVALID_SIZE;
  }
  const int64_t K = int64_t(1) << log2K, C = S / K, P = pts / K;
  if (log2K > 4 || C < 8 || P > (split ? pmax : 2 * pmax)) return TCFFT_ERR_INVALID_SIZE;
  const int planes = split ? 2 : 1;
  const int S1 = log2S / 4, RX = 1 << (log2S % 4);
  if (S1 >= 2 && RX > 1 && (C << (4 * (S1 - 1))) < 128) return TCFFT_ERR_INVALID_SIZE;  // one k0 per MMA tile
  const int tiles = (int)((P + 2047) / 2048);
  int cols = 32;
  while (cols < 32 * tiles * planes) cols *= 2;
  if (cols > 512) return TCFFT_ERR_INVALID_SIZE;
  for (PassParams* p : {&fl.f.row, &fl.f.col}) {
    p->log2N = log2S;
    p->log2C = ilog2(C);
    p->tiles = tiles;
    p->tmem_cols = cols;
    p->T = batch * S;
    p->prescale = 1.0f;
    p->nchunks = batch;
  }
  // rows: contiguous transforms of length S; columns: element e of column c
  // at c + e S (matrix m at m S^2), the stage-1 reads from the row phase's
  // exchange buffer in its 128-byte-line swizzle
  fl.f.row.log2I1 = 40;
  fl.f.row.in_l = SideLayout{S, 0, 0, 1, nullptr};
  fl.f.row.out_l = fl.f.row.in_l;
  fl.f.row.async_load = 1;
  fl.f.col.log2I1 = log2S;
  fl.f.col.log2I2 = 40;
  fl.f.col.in_l = SideLayout{1, pts, 0, (uint32_t)S, nullptr};
  fl.f.col.out_l = fl.f.col.in_l;
  fl.f.col.in_swz = 3;
  fl.f.col.out_tma = (log2S >= 8 && C <= 32 && !env_int("TCFFT_NO_TMA", 0)) ? 1 : 0;
  fl.f.log2K = log2K;
  fl.f.batch = batch;
  const int nb = (S1 >= 2 && RX > 1) ? RX : 1;
  fl.smem = 1008 + (size_t)planes * tiles * kTileBytes + (size_t)planes * P * 4 + (size_t)planes * nb * kBImageBytes;
  if (fl.smem > 227 * 1024) return TCFFT_ERR_INVALID_SIZE;
  fl.threads = tiles >= 2 ? 256 : 128;
  if (cudaFuncSetAttribute(fl.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
    return TCFFT_ERR_CUDA;
  if (cudaFuncSetAttribute(fl.fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
    return TCFFT_ERR_CUDA;
  if (K > 8 && cudaFuncSetAttribute(fl.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    (void)cudaGetLastError();
    return TCFFT_ERR_UNSUPPORTED;
  }
  // clusters that can be resident at once: the persistent grid
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(K * std::min<int64_t>(batch, 65536)));
  cfg.blockDim = dim3((unsigned)fl.threads);
  cfg.dynamicSmemBytes = fl.smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)K;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, fl.fn, &cfg) != cudaSuccess || nclusters < 1) {
    (void)cudaGetLastError();
    return TCFFT_ERR_INVALID_SIZE;  // the cluster cannot be placed at all
  }
  // CTAs per SM from registers, shared memory, threads and TMEM columns (as
  // for the pass kernels); clusters never wait on one another, so a grid
  // larger than what is resident at once only queues clusters
  int dev = 0, sms = 1, smem_sm = 0, regs_sm = 0, thr_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, fl.fn) != cudaSuccess) return TCFFT_ERR_CUDA;
  fl.regs = fa.numRegs;
  const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
  const int occ = std::min(std::min(512 / cols, regs_sm / (warp_regs * (fl.threads / 32))),
                           std::min(smem_sm / (int)(fl.smem + fa.sharedSizeBytes + 1024), thr_sm / fl.threads));
  fl.occ = std::max(1, occ);
  const int64_t est = std::max<int64_t>(nclusters, (int64_t)fl.occ * sms / K);
  fl.grid = dim3((unsigned)(K * std::min<int64_t>(batch, est)));
  return TCFFT_OK;
}

cudaError_t launch_fused2d(const Fused2DLaunch& fl, const Fused2DParams& f, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = fl.grid;
  cfg.blockDim = dim3((unsigned)fl.threads);
  cfg.dynamicSmemBytes = fl.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1u << f.log2K;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  void* args[1] = {const_cast<Fused2DParams*>(&f)};
  return cudaLaunchKernelExC(&cfg, fl.fn, args);
}

}  // namespace tcfft
