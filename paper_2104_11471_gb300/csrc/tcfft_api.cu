// C ABI of libtcfft: plans, the execution function, twiddle generation.
//
// A plan (Sec. 3.1, "Architecture") is the list of merging-kernel launches
// ("passes") that together compute the requested transform:
//  * 1D, n <= single-pass limit: one fused pass (all radix-16 stages of the
//    transform in one CTA, Sec. 3.2 "Combine multiple mergings").
//  * 1D, larger n: n = N1 N2, two passes exchanging data through global
//    memory (Sec. 3.2: "data exchanges between blocks ... can only be done
//    through global memory").  Pass 1: N1-point DFTs of the strided columns
//    x[N2 n1 + n2], times W_n^{n2 k1}, into a workspace; pass 2: N2-point
//    DFTs of the workspace rows, written to X[k1 + N1 k2].
//  * 2D (Sec. 3.1, "Support batched FFT and 2D FFT"): a pass over the rows
//    (length ny, contiguous), then a pass over the columns (length nx,
//    stride ny), the latter split in two passes as above for large nx.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <sys/stat.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/tcfft.h"
#include "pass_params.h"
#include "pass_setup.h"
#include "tables.cuh"
#include "tc_ptx.cuh"


using namespace tcfft;

namespace {

constexpr int64_t kMaxLog2_1D = 27;       // three passes of <= 1024 points
constexpr int64_t kMaxLog2_Ragged1D = 24;  // ragged groups use the four-step split
constexpr int64_t kMaxLog2_2D = 13;

// points per CTA on a strided side (8 transforms per CTA)
constexpr int64_t kCapPlain = 32768;
constexpr int64_t kCapSplit = 16384;
// largest single-pass transform (contiguous side)
constexpr int64_t kSinglePlain = 16384;
constexpr int64_t kSingleSplit = 16384;
// largest single-pass 1D plan in split precision: a 16384-point split pass
// holds one CTA per SM (shared memory), and 32 x 512 in two passes is faster
// (2^28 points: 2.01 ms against 2.19 ms)
constexpr int64_t kSingleSplit1D = 8192;

enum Buf { BUF_IN = 0, BUF_OUT = 1, BUF_WS = 2 };

struct TwTable {
  float* lo = nullptr;
  float* hi = nullptr;
  int log2S = 0;
};

struct Pass : PassLaunch {
  Buf src, dst;
  int64_t src_off = 0, dst_off = 0;  // element offsets into the workspace
  int group = 0;                     // independent branch of a ragged plan
  // fused 2D pass (one launch for rows and columns): p is the row phase, p2
  // the column phase, 2^log2K CTAs per cluster (one matrix per cluster)
  int fused = 0;
  PassParams p2;
  int log2K = 0;
};

struct GraphEntry {
  const void* in;
  void* out;
  cudaGraphExec_t exec;
};

// Persistent execution of a ragged plan (TCFFT_PLAN_PERSISTENT): the queue
// (items, dependencies, chunk counts), its counters and one device copy of
// the passes' parameters per (in, out) pair.
struct QueueBinding {
  const void* in;
  void* out;
  PassParams* d_passes;
};
struct QueueState {
  int2* d_items = nullptr;
  int* d_dep = nullptr;
  int* d_nchunks = nullptr;
  int* d_counters = nullptr;  // head, abort, done[passes]
  int nitems = 0;
  int a_bytes = 0, b_bytes = 0, tmem_cols = 32;
  size_t smem = 0;
  dim3 grid;
  long long wait_limit = kWaitLimitCycles;
  std::vector<QueueBinding> bindings;
};

tcfft_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TCFFT_OK;
  if (e == cudaErrorMemoryAllocation) return TCFFT_ERR_ALLOC;
  return TCFFT_ERR_CUDA;
}

}  // namespace

constexpr int kHostSlices = 8;  // tcfft_exec_host: batch slices in flight

struct tcfft_plan_s {
  int dims = 1;
  int64_t n = 0, nx = 0, ny = 0, batch = 0;
  bool split = false;
  bool fp32 = false;      // TCFFT_FP32: user buffers are interleaved FP32 complex (split kernels inside)
  bool share_sm = false;  // TCFFT_PLAN_SHARE_SM
  bool fused_2d = false;  // TCFFT_PLAN_FUSED_2D
  int64_t points = 0;  // total complex points per plane
  std::vector<Pass> passes;
  std::map<int, TwTable> tables;
  std::map<int, __half*> dft_b;  // by 2 * leading radix RX + scaled
  int* d_status = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* h_in_dev = nullptr;
  void* h_out_dev = nullptr;
  // tcfft_exec_host pipeline: upload and download streams, one event pair per slice
  cudaStream_t h_up = nullptr, h_down = nullptr;
  cudaEvent_t h_entry = nullptr;
  cudaEvent_t h_ev_up[kHostSlices] = {}, h_ev_done[kHostSlices] = {};
  size_t table_bytes = 0;
  bool autotune = false;              // time candidate geometries at plan time
  bool inverse = false;               // sign + (TCFFT_PLAN_INVERSE)
  bool normalise = false;             // results times 1/N (TCFFT_PLAN_SCALE)
  bool use_graph = false;             // exec replays a captured CUDA graph
  std::vector<int64_t*> toff_tables;  // device transform-offset tables (ragged)
  std::vector<GraphEntry> graphs;     // instantiated graphs by (in, out)
  void* tune_buf = nullptr;           // scratch for autotuning
  size_t tune_bytes = 0;
  bool queue = false;                 // TCFFT_PLAN_PERSISTENT: one launch over a work queue
  QueueState q;

  ~tcfft_plan_s() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    for (auto& b : q.bindings) cudaFree(b.d_passes);
    cudaFree(q.d_items);
    cudaFree(q.d_dep);
    cudaFree(q.d_nchunks);
    cudaFree(q.d_counters);
    for (auto* t : toff_tables) cudaFree(t);
    cudaFree(tune_buf);
    for (auto& kv : tables) {
      cudaFree(kv.second.lo);
      cudaFree(kv.second.hi);
    }
    for (auto& kv : stage_tables) cudaFree(kv.second);
    for (auto& kv : dft_b) cudaFree(kv.second);
    cudaFree(d_status);
    cudaFree(ws);
    cudaFree(h_in_dev);
    cudaFree(h_out_dev);
    if (h_up) cudaStreamDestroy(h_up);
    if (h_down) cudaStreamDestroy(h_down);
    if (h_entry) cudaEventDestroy(h_entry);
    for (int i = 0; i < kHostSlices; ++i) {
      if (h_ev_up[i]) cudaEventDestroy(h_ev_up[i]);
      if (h_ev_done[i]) cudaEventDestroy(h_ev_done[i]);
    }
  }

  size_t io_bytes() const { return (size_t)points * 4u * (split ? 2u : 1u); }

  std::map<int, float*> stage_tables;  // by log2 of the pass length

  tcfft_status b_images(int RX, const __half** out, bool scaled = false) {
    const int key = RX * 2 + (scaled ? 1 : 0);
    auto it = dft_b.find(key);
    if (it != dft_b.end()) {
      *out = it->second;
      return TCFFT_OK;
    }
    __half* b = nullptr;
    if (cudaMalloc(&b, 16 * kBImageBytes) != cudaSuccess) return TCFFT_ERR_ALLOC;
    cudaMemset(b, 0, 16 * kBImageBytes);
    table_bytes += 16 * kBImageBytes;
    dft_b_kernel<<<RX, 1024>>>(b, RX, scaled ? 1.0 / 16.0 : 1.0);
    if (cudaGetLastError() != cudaSuccess) {
      cudaFree(b);
      return TCFFT_ERR_LAUNCH;
    }
    dft_b[key] = b;
    *out = b;
    return TCFFT_OK;
  }

  tcfft_status stage_table(int log2N, const float** out) {
    auto it = stage_tables.find(log2N);
    if (it != stage_tables.end()) {
      *out = it->second;
      return TCFFT_OK;
    }
    const int S = log2N / 4, RX = 1 << (log2N % 4);
    int rows = 0;
    if (S >= 2) rows = RX << (4 * (S - 1));
    for (int j = 2; j < S; ++j) rows += 1 << (4 * (S - j));
    float* t = nullptr;
    const size_t bytes = (size_t)std::max(rows, 1) * kStageSlots * 4 * sizeof(float);
    if (cudaMalloc(&t, bytes) != cudaSuccess) return TCFFT_ERR_ALLOC;
    table_bytes += bytes;
    if (rows > 0) {
      stage_twiddle_kernel<<<(rows * kStageSlots + 255) / 256, 256>>>(reinterpret_cast<float4*>(t), log2N, rows);
      if (cudaGetLastError() != cudaSuccess) {
        cudaFree(t);
        return TCFFT_ERR_LAUNCH;
      }
    }
    stage_tables[log2N] = t;
    *out = t;
    return TCFFT_OK;
  }

  tcfft_status table(int log2M, TwTable** out) {
    auto it = tables.find(log2M);
    if (it != tables.end()) {
      *out = &it->second;
      return TCFFT_OK;
    }
    TwTable t;
    t.log2S = (log2M + 1) / 2;
    const int64_t S = int64_t(1) << t.log2S, H = int64_t(1) << (log2M - t.log2S);
    if (cudaMalloc(&t.lo, S * 8) != cudaSuccess) return TCFFT_ERR_ALLOC;
    if (cudaMalloc(&t.hi, H * 8) != cudaSuccess) {
      cudaFree(t.lo);
      return TCFFT_ERR_ALLOC;
    }
    table_bytes += (size_t)(S + H) * 8;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((S + H + threads - 1) / threads, 1024);
    twiddle_table_kernel<<<blocks, threads>>>((float2*)t.lo, (float2*)t.hi, log2M, t.log2S);
    if (cudaGetLastError() != cudaSuccess) return TCFFT_ERR_LAUNCH;
    tables[log2M] = t;
    *out = &tables[log2M];
    return TCFFT_OK;
  }
};

namespace {

// Adds one fused pass computing DFTs of length L on T transforms indexed by
// (t1 < I1, t2 < I2, t3), reading `src` with layout `in` and writing `dst`
// with layout `out`.  otw_level / log2M: optional output twiddle W_M^{col k}.
tcfft_status bind_tables(tcfft_plan_s* pl, Pass& ps, int log2L, int otw_level, int log2M);
tcfft_status tune_pass(tcfft_plan_s* pl, Pass& ps, int64_t L, int64_t T, int64_t I1, int64_t I2, Side in,
                       Side out, int otw_level, int log2M);

PassParams bound_params(const tcfft_plan_s* plan, const Pass& ps, const void* in, void* out);

// Operand area of a pass in shared memory (A tiles, raw prefetch buffer, DFT
// images) and the cap a persistent queue gives every pass.
constexpr int64_t kQueueArea = 40 * 1024;
int64_t queue_area(const Pass& ps) {
  const int S = ps.p.log2N / 4, RX = 1 << (ps.p.log2N % 4);
  const int64_t P = int64_t(1) << (ps.p.log2C + ps.p.log2N);
  return (int64_t)ps.p.tiles * kTileBytes + (ps.p.async_load ? 4 * P : 0) +
         ((S >= 2 && RX > 1) ? RX : 1) * kBImageBytes;
}

cudaError_t launch_plan_pass(const tcfft_plan_s* plan, const Pass& ps, const void* in, void* out, cudaStream_t s,
                             int64_t batch = 0);

tcfft_status add_pass(tcfft_plan_s* pl, int64_t L, int64_t T, int64_t I1, int64_t I2, Side in,
                      Side out, Buf src, Buf dst, int otw_level, int log2M, int group = 0,
                      int64_t src_off = 0, int64_t dst_off = 0) {
  Pass ps;
  tcfft_status st = TCFFT_ERR_INVALID_SIZE;
  if (pl->queue) {
    // passes of a persistent queue share one CTA shape: 128 threads, at most
    // kQueueArea bytes of operands and 128 TMEM columns (3 CTAs per SM), so
    // large chunks fall back to smaller ones and then to synchronous loads
    bool fits = false;
    for (int64_t tgt : {int64_t(0), int64_t(8192), int64_t(4096), int64_t(2048)}) {
      for (int as : {-1, 0}) {
        st = pass_geometry(ps, L, T, I1, I2, in, out, pl->split, tgt, 128, as, pl->share_sm);
        if (st == TCFFT_OK && queue_area(ps) <= kQueueArea && ps.p.tmem_cols <= 128) {
          fits = true;
          break;
        }
      }
      if (fits) break;
    }
    if (!fits) {
      if (env_int("TCFFT_DEBUG", 0))
        std::fprintf(stderr, "persistent plan: pass of length %lld (T %lld) fits no queue geometry (last %d)\n",
                     (long long)L, (long long)T, (int)st);
      return TCFFT_ERR_INVALID_SIZE;
    }
  } else {
    st = pass_geometry(ps, L, T, I1, I2, in, out, pl->split, 0, 0, -1, pl->share_sm);
  }
  if (st != TCFFT_OK) return st;
  ps.src = src;
  ps.dst = dst;
  ps.src_off = src_off;
  ps.dst_off = dst_off;
  ps.group = group;
  st = bind_tables(pl, ps, ilog2(L), otw_level, log2M);
  if (st != TCFFT_OK) return st;
  if (!pl->queue && pl->autotune) {
    st = tune_pass(pl, ps, L, T, I1, I2, in, out, otw_level, log2M);
    if (st != TCFFT_OK) return st;
  }
  pl->passes.push_back(ps);
  return TCFFT_OK;
}

// Adds one fused 2D pass over B matrices of S x S (rows and columns in one
// launch, Sec. 3.1), reading `src` and writing `dst`; toff: optional table of
// the matrices' first elements (ragged batches).
tcfft_status add_fused_pass(tcfft_plan_s* pl, int64_t S, int64_t B, Buf src, Buf dst, int group = 0,
                            const int64_t* toff = nullptr) {
  Fused2DLaunch fl;
  tcfft_status st = fused2d_geometry(fl, S, B, pl->split);
  if (st != TCFFT_OK) return st;
  if (pl->share_sm) fl.grid.x = std::max(1u << fl.f.log2K, (fl.grid.x / 2) & ~((1u << fl.f.log2K) - 1u));
  Pass ps;
  ps.fused = 1;
  ps.fn = fl.fn;
  ps.grid = fl.grid;
  ps.threads = fl.threads;
  ps.smem = fl.smem;
  ps.occ = fl.occ;
  ps.regs = fl.regs;
  ps.p = fl.f.row;
  ps.p2 = fl.f.col;
  ps.log2K = fl.f.log2K;
  ps.src = src;
  ps.dst = dst;
  ps.group = group;
  st = bind_tables(pl, ps, ilog2(S), 0, 0);
  if (st != TCFFT_OK) return st;
  // both phases have length S: the same tables and DFT images
  PassParams& c = ps.p2;
  c.tw_lo = ps.p.tw_lo;
  c.tw_hi = ps.p.tw_hi;
  c.tw_log2S = ps.p.tw_log2S;
  c.stw = ps.p.stw;
  c.dft_b = ps.p.dft_b;
  c.status = ps.p.status;
  c.in_plane = ps.p.in_plane;
  c.out_plane = ps.p.out_plane;
  if (toff) {
    ps.p.in_l.toff = toff;
    c.out_l.toff = toff;
    c.out_tma = 0;
  }
  pl->passes.push_back(ps);
  return TCFFT_OK;
}

// Points the pass at the plan's tables (generated on first use).
tcfft_status bind_tables(tcfft_plan_s* pl, Pass& ps, int log2L, int otw_level, int log2M) {
  tcfft_status st;
  PassParams& p = ps.p;
  TwTable* tw = nullptr;
  st = pl->table(log2L, &tw);
  if (st != TCFFT_OK) return st;
  p.tw_lo = tw->lo;
  p.tw_hi = tw->hi;
  p.tw_log2S = tw->log2S;
  const float* stw = nullptr;
  st = pl->stage_table(log2L, &stw);
  if (st != TCFFT_OK) return st;
  p.stw = reinterpret_cast<const float4*>(stw);
  const __half* bimg = nullptr;
  st = pl->b_images(1 << (log2L % 4), &bimg, pl->normalise);
  if (st != TCFFT_OK) return st;
  p.dft_b = reinterpret_cast<const uint16_t*>(bimg);
  p.otw_level = otw_level;
  if (otw_level) {
    TwTable* ot = nullptr;
    st = pl->table(log2M, &ot);
    if (st != TCFFT_OK) return st;
    p.otw_log2M = log2M;
    p.otw_log2S = ot->log2S;
    p.otw_lo = ot->lo;
    p.otw_hi = ot->hi;
  }
  p.status = pl->d_status;
  p.in_plane = pl->points;
  p.out_plane = pl->points;
  return TCFFT_OK;
}

// ------------------------------------------------------------- autotuner
// Chooses, per pass, the points per CTA (transforms per CTA of contiguous
// passes, the column-block cap of strided ones) among a few candidates by
// timing each on scratch memory.  Results are cached in a text file
// (TCFFT_TUNE_CACHE, default $HOME/.cache/tcfft_tune.txt), one
// "key target" pair per line; the key names length, layout, precision and
// the size of the batch.
std::mutex g_tune_mu;
std::map<std::string, int64_t> g_tune_cache;
bool g_tune_loaded = false;

std::string tune_path() {
  const char* e = std::getenv("TCFFT_TUNE_CACHE");
  if (e && *e) return e;
  const char* h = std::getenv("HOME");
  return std::string(h ? h : "/tmp") + "/.cache/tcfft_tune.txt";
}

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  FILE* f = std::fopen(tune_path().c_str(), "r");
  if (!f) return;
  char key[128];
  long long v;
  while (std::fscanf(f, "%127s %lld", key, &v) == 2) g_tune_cache[key] = v;
  std::fclose(f);
}

void tune_store() {
  const std::string path = tune_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {
    const std::string dir = path.substr(0, slash);
    std::string cmd;  // create the cache directory if missing (mkdir -p semantics)
    for (size_t i = 1; i <= dir.size(); ++i)
      if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
  }
  FILE* f = std::fopen(path.c_str(), "w");
  if (!f) return;
  for (auto& kv : g_tune_cache) std::fprintf(f, "%s %lld\n", kv.first.c_str(), (long long)kv.second);
  std::fclose(f);
}

tcfft_status tune_pass(tcfft_plan_s* pl, Pass& ps, int64_t L, int64_t T, int64_t I1, int64_t I2, Side in,
                       Side out, int otw_level, int log2M) {
  const int mode = (in.es == 1) ? ((out.es == 1) ? 0 : 2) : 1;
  char key[128];
  std::snprintf(key, sizeof(key), "v3_L%d_m%d_s%d_T%d_g%d_h%d", ilog2(L), mode, pl->split ? 1 : 0, ilog2(T),
                (in.toff || out.toff) ? 1 : 0, pl->share_sm ? 1 : 0);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load();
  auto it = g_tune_cache.find(key);
  int64_t best = -1;
  if (it != g_tune_cache.end()) {
    best = it->second;
  } else {
    // scratch: one buffer serves as input and output (in place), sized for
    // the plan's largest buffer; its contents do not matter for timing
    const size_t need = std::max(pl->io_bytes(), pl->ws_bytes) + 4096;
    if (pl->tune_bytes < need) {
      cudaFree(pl->tune_buf);
      pl->tune_buf = nullptr;
      pl->tune_bytes = 0;
      if (cudaMalloc(&pl->tune_buf, need) != cudaSuccess) return TCFFT_ERR_ALLOC;
      cudaMemset(pl->tune_buf, 0, need);
      pl->tune_bytes = need;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    // candidates: points per CTA (0 = the planner's) x threads per CTA x load
    // mode; cached as points | threads << 20 | (async + 1) << 30.  Ragged
    // groups (offset tables) run concurrently in one graph, where a geometry
    // timed alone can lose to the planner's: they vary the points only.
    const bool grouped = in.toff || out.toff;
    std::vector<int64_t> cands;
    for (int64_t pts : {0, 2048, 4096, 8192, 16384, 32768}) {
      if (grouped) {
        if (pts) cands.push_back(pts);
        continue;
      }
      for (int64_t thr : {256, 128})
        for (int64_t as : {1, 0}) cands.push_back(pts | (thr << 20) | ((as + 1) << 30));
    }
    for (int64_t cand : cands) {
      Pass c;
      if (pass_geometry(c, L, T, I1, I2, in, out, pl->split, cand & 0xFFFFF, (int)((cand >> 20) & 1023),
                        (int)((cand >> 30) & 3) - 1, pl->share_sm) != TCFFT_OK)
        continue;
      c.src = ps.src;
      c.dst = ps.dst;
      if (bind_tables(pl, c, ilog2(L), otw_level, log2M) != TCFFT_OK) continue;
      c.p.in = reinterpret_cast<const uint32_t*>(pl->tune_buf);
      c.p.out = reinterpret_cast<uint32_t*>(pl->tune_buf);
      encode_in_map(c.p, pl->split);
      encode_out_map(c.p, pl->split);
      void* args[1] = {&c.p};
      float ms = 0.0f;
      bool okc = true;
      for (int rep = 0; rep < 4 && okc; ++rep) {  // first run is a warm-up
        cudaEventRecord(e0);
        okc = cudaLaunchKernel(c.fn, c.grid, dim3(c.threads), args, c.smem, 0) == cudaSuccess;
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0) ms += t;
      }
      if (okc && ms < best_ms) {
        best_ms = ms;
        best = cand;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0) return TCFFT_OK;  // keep the default geometry
    g_tune_cache[key] = best;
    tune_store();
  }
  Pass c;
  if (pass_geometry(c, L, T, I1, I2, in, out, pl->split, best & 0xFFFFF, (int)((best >> 20) & 1023),
                    (int)((best >> 30) & 3) - 1, pl->share_sm) != TCFFT_OK)
    return TCFFT_OK;
  const PassParams keep = ps.p;
  ps.fn = c.fn;
  ps.grid = c.grid;
  ps.smem = c.smem;
  ps.occ = c.occ;
  ps.regs = c.regs;
  ps.threads = c.threads;
  ps.p = c.p;
  // tables, buffers and output twiddle stay those of the bound pass
  ps.p.tw_lo = keep.tw_lo;
  ps.p.tw_hi = keep.tw_hi;
  ps.p.tw_log2S = keep.tw_log2S;
  ps.p.stw = keep.stw;
  ps.p.dft_b = keep.dft_b;
  ps.p.otw_level = keep.otw_level;
  ps.p.otw_log2M = keep.otw_log2M;
  ps.p.otw_log2S = keep.otw_log2S;
  ps.p.otw_lo = keep.otw_lo;
  ps.p.otw_hi = keep.otw_hi;
  ps.p.status = keep.status;
  ps.p.in_plane = keep.in_plane;
  ps.p.out_plane = keep.out_plane;
  return TCFFT_OK;
}

constexpr int64_t kNoLevel = int64_t(1) << 40;  // "unbounded" index level

// Longest strided pass (log2) for the plan's precision: split kernels keep
// two planes per point, so their strided passes stop one length earlier.
int max_strided_log2(const tcfft_plan_s* pl) { return max_log2_pass(kModeStrided, pl->split); }

tcfft_status alloc_ws(tcfft_plan_s* pl, size_t bytes) {
  if (pl->ws && pl->ws_bytes >= bytes) return TCFFT_OK;
  cudaFree(pl->ws);
  pl->ws = nullptr;
  pl->ws_bytes = 0;
  if (cudaMalloc(&pl->ws, bytes) != cudaSuccess) {
    pl->ws = nullptr;
    return TCFFT_ERR_ALLOC;
  }
  pl->ws_bytes = bytes;
  return TCFFT_OK;
}

// The passes of a 1D transform n = 2^l[0] (one pass), 2^l[0] 2^l[1] (two
// passes) or 2^l[0] 2^l[1] 2^l[2] (three passes); the workspace must exist
// for more than one pass.
tcfft_status build_1d(tcfft_plan_s* pl, const int* l, int np) {
  const int64_t n = pl->n, B = pl->batch;
  if (np == 1) {
    Side s{n, 0, 0, 1};
    return add_pass(pl, n, B, kNoLevel, 1, s, s, BUF_IN, BUF_OUT, 0, 0);
  }
  const int lg = ilog2(n);
  if (np == 3) {
    // n = N1 N2 N3 (M = N2 N3) in three passes of short transforms, so that
    // every pass keeps small per-CTA tiles with prefetch:
    //  A: N1-point DFTs of the columns x[M n1 + m], times W_n^{m k1} -> ws
    //  B: N2-point DFTs of ws[k1 M + N3 n2 + n3], times W_M^{n3 k2}, in place
    //  C: N3-point DFTs of ws rows (k1, k2) -> X[k1 + N1 k2 + N1 N2 k3]
    const int64_t N1 = int64_t(1) << l[0], N2 = int64_t(1) << l[1], N3 = int64_t(1) << l[2], M = N2 * N3;
    Side a{1, n, 0, M};
    tcfft_status st = add_pass(pl, N1, B * M, M, kNoLevel, a, a, BUF_IN, BUF_WS, 1, lg);
    if (st != TCFFT_OK) return st;
    Side b{1, M, n, N3};
    st = add_pass(pl, N2, B * N1 * N3, N3, N1, b, b, BUF_WS, BUF_WS, 1, l[1] + l[2]);
    if (st != TCFFT_OK) return st;
    Side cin{M, N3, n, 1}, cout{1, N1, n, N1 * N2};
    return add_pass(pl, N3, B * N1 * N2, N1, N2, cin, cout, BUF_WS, BUF_OUT, 0, 0);
  }
  const int64_t N1 = int64_t(1) << l[0], N2 = n / N1;
  // pass 1: columns n2 of length N1 (stride N2), times W_n^{n2 k1}
  Side c1{1, n, 0, N2};
  tcfft_status st = add_pass(pl, N1, B * N2, N2, kNoLevel, c1, c1, BUF_IN, BUF_WS, 1, lg);
  if (st != TCFFT_OK) return st;
  // pass 2: rows k1 of length N2, written to X[k1 + N1 k2]
  Side in2{N2, n, 0, 1}, out2{1, n, 0, N1};
  return add_pass(pl, N2, B * N1, N1, kNoLevel, in2, out2, BUF_WS, BUF_OUT, 0, 0);
}

// Times the plan's current passes on the autotuning scratch (in = out =
// scratch, the workspace between them): mean of three runs after a warm-up,
// in ms; a negative value when a launch fails.
float time_passes(tcfft_plan_s* pl) {
  const size_t need = pl->io_bytes() + 4096;
  if (pl->tune_bytes < need) {
    cudaFree(pl->tune_buf);
    pl->tune_buf = nullptr;
    pl->tune_bytes = 0;
    if (cudaMalloc(&pl->tune_buf, need) != cudaSuccess) {
      (void)cudaGetLastError();
      return -1.0f;
    }
    cudaMemset(pl->tune_buf, 0, need);
    pl->tune_bytes = need;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float total = 0.0f;
  bool ok = true;
  for (int rep = 0; rep < 4 && ok; ++rep) {
    cudaEventRecord(e0);
    for (const Pass& ps : pl->passes)
      if (launch_plan_pass(pl, ps, pl->tune_buf, pl->tune_buf, 0) != cudaSuccess) ok = false;
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0) total += t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) {
    (void)cudaGetLastError();
    return -1.0f;
  }
  return total / 3.0f;
}

// The pass splits the planner may use for a multi-pass 1D transform of
// 2^lg points: two passes N1 x N2 near the square root, three passes
// N1 x N2 x N3 with N1 from 16 to 256 and N2 ~ N3, every factor a pass
// length the strided kernels have (16 .. 4096 plain, .. 2048 split).
std::vector<std::vector<int>> split_candidates(const tcfft_plan_s* pl, int lg) {
  const int mx = max_strided_log2(pl);
  std::vector<std::vector<int>> c;
  for (int l1 = std::max(4, lg - mx); l1 <= std::min(mx, lg - 4); ++l1)
    if (std::abs(2 * l1 - lg) <= 4) c.push_back({l1, lg - l1});
  if (lg >= 20) {
    for (int l1 = 4; l1 <= 8; ++l1) {
      const int l2 = (lg - l1 + 1) / 2, l3 = lg - l1 - l2;
      if (l3 >= 4 && l2 <= mx) c.push_back({l1, l2, l3});
    }
  }
  return c;
}

// The split the planner takes without autotuning (measured at 2^28 points):
// one pass to 16384 (split precision: to 8192); two passes N1 x N2, N1 = 2^ceil(lg/2), to 2^21; three
// passes from 2^22 (tuning override TCFFT_THREE_PASS_MIN), always beyond
// 2^24 and for split precision beyond 2^22 (the four-step split would need
// strided passes longer than the split kernels' 2^11).  2^22 as 16 x 512 x
// 512 1.53 ms (2048 x 2048: 1.92 ms, 64 x 256 x 256: 1.62 ms); 2^23 as 128 x
// 256 x 256 1.61 ms (two passes: 2.65 ms); 2^24 as 256^3 1.45 ms (16 x 1024 x
// 1024: 1.75 ms).
std::vector<int> default_split(const tcfft_plan_s* pl, int lg) {
  const bool three = lg >= env_int("TCFFT_THREE_PASS_MIN", 22) || lg > 24 || (pl->split && lg > 22);
  if (three) {
    const int l1_default = lg == 22 ? 4 : (lg == 23 ? 7 : 8);
    const int l1 = std::max(4, std::min(8, env_int("TCFFT_THREE_PASS_L1", l1_default)));  // tuning override
    const int l2 = (lg - l1 + 1) / 2;
    return {l1, l2, lg - l1 - l2};
  }
  // split 2^14: 32 x 512, the autotuner's pick among 32 x 512 ... 512 x 32
  const int l1 = env_int("TCFFT_FOUR_STEP_L1", (pl->split && lg == 14) ? 5 : (lg + 1) / 2);  // tuning override
  return {l1, lg - l1};
}

tcfft_status plan_1d(tcfft_plan_s* pl) {
  const int64_t n = pl->n, B = pl->batch;
  const int64_t single = std::min<int64_t>(pl->split ? kSingleSplit1D : kSinglePlain,
                                           int64_t(1) << env_int("TCFFT_SINGLE_MAX_LOG2", 14));  // tuning override
  const int lg = ilog2(n);
  if (n <= single) {
    const int l[1] = {lg};
    return build_1d(pl, l, 1);
  }
  tcfft_status st = alloc_ws(pl, (size_t)B * n * 4 * (pl->split ? 2 : 1));
  if (st != TCFFT_OK) return st;
  std::vector<int> best = default_split(pl, lg);
  if (pl->autotune) {
    // time every candidate split (each pass with its own tuned geometry) on
    // the plan's sizes; the winner is cached per (length, precision, batch)
    char key[128];
    std::snprintf(key, sizeof(key), "split_v1_lg%d_s%d_T%d_h%d", lg, pl->split ? 1 : 0, ilog2(B),
                  pl->share_sm ? 1 : 0);
    int64_t code = -1;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      tune_load();
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) code = it->second;
    }
    if (code < 0) {
      float best_ms = 1e30f;
      for (const std::vector<int>& c : split_candidates(pl, lg)) {
        pl->passes.clear();
        if (build_1d(pl, c.data(), (int)c.size()) != TCFFT_OK) continue;
        const float ms = time_passes(pl);
        if (ms > 0.0f && ms < best_ms) {
          best_ms = ms;
          code = 0;
          for (size_t i = 0; i < c.size(); ++i) code |= (int64_t)c[i] << (8 * i);
        }
      }
      pl->passes.clear();
      if (code >= 0) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = code;
        tune_store();
      }
    }
    if (code > 0) {
      best.clear();
      for (int i = 0; i < 3 && ((code >> (8 * i)) & 255); ++i) best.push_back((int)((code >> (8 * i)) & 255));
    }
  }
  return build_1d(pl, best.data(), (int)best.size());
}

// The passes of a 2D transform: rows, then columns in one strided pass
// (col_l1 == 0) or in two passes nx = N1 N2 with N1 = 2^col_l1 (the
// workspace must exist then).
tcfft_status build_2d(tcfft_plan_s* pl, int col_l1) {
  const int64_t nx = pl->nx, ny = pl->ny, B = pl->batch;
  const int64_t mat = nx * ny;
  // rows: nx * B transforms of length ny, contiguous
  Side r{ny, 0, 0, 1};
  tcfft_status st = add_pass(pl, ny, B * nx, kNoLevel, 1, r, r, BUF_IN, BUF_OUT, 0, 0);
  if (st != TCFFT_OK) return st;
  if (col_l1 == 0) {
    // columns: ny * B transforms of length nx, stride ny, in place on out
    Side c{1, mat, 0, ny};
    return add_pass(pl, nx, B * ny, ny, kNoLevel, c, c, BUF_OUT, BUF_OUT, 0, 0);
  }
  const int lg = ilog2(nx);
  const int64_t N1 = int64_t(1) << col_l1, N2 = nx / N1;
  // pass A: element n1 of column (iy, n2) at (N2 n1 + n2) ny + iy
  Side a{1, ny, mat, N2 * ny};
  st = add_pass(pl, N1, B * ny * N2, ny, N2, a, a, BUF_OUT, BUF_WS, 2, lg);
  if (st != TCFFT_OK) return st;
  // pass B: row k1 (elements n2 at (N2 k1 + n2) ny + iy) -> X[k1 + N1 k2]
  Side bi{1, N2 * ny, mat, ny}, bo{1, ny, mat, N1 * ny};
  return add_pass(pl, N2, B * ny * N1, ny, N1, bi, bo, BUF_WS, BUF_OUT, 0, 0);
}

bool fused_2d_available(const tcfft_plan_s* pl, int64_t nx, int64_t ny, int64_t B) {
  if (!pl->fused_2d || nx != ny || env_int("TCFFT_NO_FUSED_2D", 0)) return false;  // tuning override
  Fused2DLaunch fl;
  return fused2d_geometry(fl, nx, B, pl->split) == TCFFT_OK;
}

tcfft_status plan_2d(tcfft_plan_s* pl) {
  const int64_t nx = pl->nx, B = pl->batch;
  const int64_t mat = nx * pl->ny;
  // TCFFT_PLAN_FUSED_2D, square matrices up to 512^2 (256^2 split): rows and
  // columns in one fused launch, one HBM read and one write per matrix
  // (Sec. 3.1); with autotuning the fused launch competes with the two-pass
  // plan.  Measured at 2^28 points: 256^2 fused 1.71 ms, two passes 0.79 ms;
  // 64^2 1.66 vs 1.34 ms (the stages are bound by on-chip work, not HBM)
  if (fused_2d_available(pl, nx, pl->ny, B)) {
    bool fused = true;
    if (pl->autotune) {
      char key[128];
      std::snprintf(key, sizeof(key), "fused_v1_s%d_p%d_T%d_h%d", ilog2(nx), pl->split ? 1 : 0, ilog2(B),
                    pl->share_sm ? 1 : 0);
      int64_t code = -1;
      {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_load();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) code = it->second;
      }
      if (code < 0) {
        float tf = -1.0f, tu = -1.0f;
        if (add_fused_pass(pl, nx, B, BUF_IN, BUF_OUT) == TCFFT_OK) tf = time_passes(pl);
        pl->passes.clear();
        const int64_t cap = pl->split ? kCapSplit : kCapPlain;
        if (8 * nx <= cap && ilog2(nx) <= max_strided_log2(pl) && build_2d(pl, 0) == TCFFT_OK) tu = time_passes(pl);
        pl->passes.clear();
        code = (tf > 0.0f && (tu <= 0.0f || tf <= tu)) ? 1 : 0;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = code;
        tune_store();
      }
      fused = code == 1;
    }
    if (fused) return add_fused_pass(pl, nx, B, BUF_IN, BUF_OUT);
  }
  const int64_t cap = pl->split ? kCapSplit : kCapPlain;
  const int lg = ilog2(nx);
  const size_t ws = (size_t)B * mat * 4 * (pl->split ? 2 : 1);
  // one column pass up to 2048 rows; longer columns in two passes, 16 x nx/16
  // (measured at 2^28 points: 4096^2 plain 2.27 -> 1.48 ms, split 3.81 ->
  // 2.97 ms; 8192^2 plain 1.91 -> 1.64 ms against 128 x 64, split 4.88 -> 3.70;
  // 1024^2 keeps its single pass, 1.16 ms against 1.61 ms for 16 x 64)
  const int col_max = env_int("TCFFT_2D_COL_MAX_LOG2", 11);  // tuning override
  const bool one_ok = 8 * nx <= cap && lg <= std::min(col_max, max_strided_log2(pl));
  int col_l1 = one_ok ? 0 : env_int("TCFFT_2D_COL_L1", 4);  // tuning override
  if (pl->autotune) {
    // candidates: one column pass (where it fits) and two passes N1 x N2
    // with N1 = 16 .. 128, each timed with its passes' tuned geometry
    std::vector<int> cands;
    if (8 * nx <= cap && lg <= max_strided_log2(pl)) cands.push_back(0);
    for (int l1 = 4; l1 <= 7; ++l1)
      if (lg - l1 >= 4 && lg - l1 <= max_strided_log2(pl) && lg >= 8) cands.push_back(l1);
    if (cands.size() > 1) {
      char key[128];
      std::snprintf(key, sizeof(key), "col_v1_nx%d_ny%d_s%d_T%d_h%d", lg, ilog2(pl->ny), pl->split ? 1 : 0,
                    ilog2(B), pl->share_sm ? 1 : 0);
      int64_t code = -1;
      {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_load();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) code = it->second;
      }
      if (code < 0 && alloc_ws(pl, ws) == TCFFT_OK) {
        float best_ms = 1e30f;
        for (int c : cands) {
          pl->passes.clear();
          if (build_2d(pl, c) != TCFFT_OK) continue;
          const float ms = time_passes(pl);
          if (ms > 0.0f && ms < best_ms) {
            best_ms = ms;
            code = c;
          }
        }
        pl->passes.clear();
        if (code >= 0) {
          std::lock_guard<std::mutex> lock(g_tune_mu);
          g_tune_cache[key] = code;
          tune_store();
        }
      }
      if (code >= 0) col_l1 = (int)code;
    }
  }
  if (col_l1 > 0) {
    tcfft_status st = alloc_ws(pl, ws);
    if (st != TCFFT_OK) return st;
  } else if (pl->ws) {
    cudaFree(pl->ws);  // candidates needed it; the chosen plan does not
    pl->ws = nullptr;
    pl->ws_bytes = 0;
  }
  return build_2d(pl, col_l1);
}

// Ragged batch: transform i is 1D of length n0[i] (n1 == null or n1[i] == 0)
// or 2D n0[i] x n1[i]; its data starts at the sum of the sizes of the
// transforms before it.  Transforms of one shape form a group with its own
// offset table; each group's passes gather and scatter through that table,
// and the groups are independent branches of the plan's graph.
tcfft_status plan_many(tcfft_plan_s* pl, int64_t count, const int64_t* n0, const int64_t* n1) {
  std::map<std::pair<int64_t, int64_t>, std::vector<int64_t>> groups;
  int64_t acc = 0;
  for (int64_t i = 0; i < count; ++i) {
    const int64_t a = n0[i], b = n1 ? n1[i] : 0;
    groups[{a, b}].push_back(acc);
    acc += b ? a * b : a;
  }
  pl->points = acc;
  // persistent queues keep every pass within 8192 points per CTA: longer 1D
  // transforms run as two passes
  const int64_t single = pl->queue ? 8192 : (pl->split ? kSingleSplit : kSinglePlain);
  const int64_t cap = pl->split ? kCapSplit : kCapPlain;
  bool need_ws = false;
  for (auto& g : groups)
    if (g.first.second == 0 && (g.first.first > single || pl->queue)) need_ws = true;
  if (need_ws) {
    pl->ws_bytes = (size_t)acc * 4 * (pl->split ? 2 : 1);
    if (cudaMalloc(&pl->ws, pl->ws_bytes) != cudaSuccess) {
      pl->ws = nullptr;
      return TCFFT_ERR_ALLOC;
    }
  }
  int gid = 0;
  int64_t ws_off = 0;
  for (auto& g : groups) {
    const int64_t a = g.first.first, b = g.first.second;
    const int64_t k = (int64_t)g.second.size();
    int64_t* toff = nullptr;
    if (cudaMalloc(&toff, sizeof(int64_t) * k) != cudaSuccess) return TCFFT_ERR_ALLOC;
    pl->toff_tables.push_back(toff);
    if (cudaMemcpy(toff, g.second.data(), sizeof(int64_t) * k, cudaMemcpyHostToDevice) != cudaSuccess)
      return TCFFT_ERR_CUDA;
    tcfft_status st;
    if (b == 0) {
      const int64_t n = a;
      st = TCFFT_ERR_INVALID_SIZE;
      if (n <= single) {
        Side sd{n, 0, 0, 1, toff};
        st = add_pass(pl, n, k, 1, kNoLevel, sd, sd, BUF_IN, BUF_OUT, 0, 0, gid);
      }
      // a persistent queue's CTA shape cannot hold every single-pass length
      // (2048 points: eight transforms per MMA tile): two passes then
      if (n > single || (st == TCFFT_ERR_INVALID_SIZE && pl->queue)) {
        const int lg = ilog2(n);
        const int64_t N1 = int64_t(1) << ((lg + 1) / 2), N2 = n / N1;
        Side in1{1, 0, 0, N2, toff}, out1{1, n, 0, N2};
        st = add_pass(pl, N1, k * N2, N2, kNoLevel, in1, out1, BUF_IN, BUF_WS, 1, lg, gid, 0, ws_off);
        if (st != TCFFT_OK) return st;
        Side in2{N2, n, 0, 1}, out2{1, 0, 0, N1, toff};
        st = add_pass(pl, N2, k * N1, N1, kNoLevel, in2, out2, BUF_WS, BUF_OUT, 0, 0, gid, ws_off, 0);
        ws_off += k * n;
      }
    } else if (fused_2d_available(pl, a, b, k)) {
      // square matrices: rows and columns in one fused launch
      st = add_fused_pass(pl, a, k, BUF_IN, BUF_OUT, gid, toff);
    } else {
      const int64_t nx = a, ny = b;
      if (8 * nx > cap) return TCFFT_ERR_INVALID_SIZE;  // ragged 2D keeps columns in one pass
      Side r{ny, 0, 0, 1, toff};
      st = add_pass(pl, ny, k * nx, nx, kNoLevel, r, r, BUF_IN, BUF_OUT, 0, 0, gid);
      if (st != TCFFT_OK) return st;
      Side c{1, 0, 0, ny, toff};
      st = add_pass(pl, nx, k * ny, ny, kNoLevel, c, c, BUF_OUT, BUF_OUT, 0, 0, gid);
    }
    if (st != TCFFT_OK) return st;
    ++gid;
  }
  return TCFFT_OK;
}

// The work queue of a persistent plan: items (pass, slot) level by level
// (every slot of the first pass of every group, then of the second, ...),
// each pass depending on the previous pass of its group; counters, geometry
// of the launch.  A slot runs the chunks slot, slot + G, ... of its pass (G =
// the pass's slots = min(chunks, the launch's CTAs)).
tcfft_status build_queue(tcfft_plan_s* pl) {
  QueueState& q = pl->q;
  const int np = (int)pl->passes.size();
  std::vector<int> dep(np, -1), nslot(np), level(np, 0);
  int maxlevel = 0;
  for (int i = 0; i < np; ++i) {
    const Pass& ps = pl->passes[i];
    if (ps.fused || pl->split) return TCFFT_ERR_UNSUPPORTED;
    if (i > 0 && pl->passes[i - 1].group == ps.group) {
      dep[i] = i - 1;
      level[i] = level[i - 1] + 1;
    }
    maxlevel = std::max(maxlevel, level[i]);
    // the pass body's operand area: A tiles, raw prefetch buffer, DFT images
    q.a_bytes = (int)std::max<int64_t>(q.a_bytes, (queue_area(ps) + 1023) & ~int64_t(1023));
    q.tmem_cols = std::max(q.tmem_cols, ps.p.tmem_cols);
  }
  q.b_bytes = 0;
  // one CTA shape for every pass: 128 threads, the largest operand area and
  // TMEM allocation; CTAs per SM from the launch bounds (4), shared memory
  // and TMEM
  const void* fn = queue_fn();
  q.smem = 1008 + (size_t)q.a_bytes + sizeof(PassParams) + 64;
  if (q.smem > 227 * 1024) return TCFFT_ERR_INVALID_SIZE;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess ||
      cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
    return TCFFT_ERR_CUDA;
  int dev = 0, sms = 1, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const int occ = std::max(1, std::min(std::min(4, 512 / q.tmem_cols), smem_sm / (int)(q.smem + 1024)));
  const int64_t ctas = (int64_t)occ * sms;
  std::vector<int2> items;
  for (int i = 0; i < np; ++i) nslot[i] = (int)std::min<int64_t>(pl->passes[i].p.nchunks, ctas);
  for (int lv = 0; lv <= maxlevel; ++lv)
    for (int i = 0; i < np; ++i)
      if (level[i] == lv)
        for (int c = 0; c < nslot[i]; ++c) items.push_back(make_int2(i, c));
  q.nitems = (int)items.size();
  q.grid = dim3((unsigned)std::min<int64_t>(ctas, q.nitems));
  if (cudaMalloc(&q.d_items, sizeof(int2) * items.size()) != cudaSuccess ||
      cudaMalloc(&q.d_dep, sizeof(int) * np) != cudaSuccess || cudaMalloc(&q.d_nchunks, sizeof(int) * np) != cudaSuccess ||
      cudaMalloc(&q.d_counters, sizeof(int) * (2 + np)) != cudaSuccess)
    return TCFFT_ERR_ALLOC;
  if (cudaMemcpy(q.d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(q.d_dep, dep.data(), sizeof(int) * np, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(q.d_nchunks, nslot.data(), sizeof(int) * np, cudaMemcpyHostToDevice) != cudaSuccess)
    return TCFFT_ERR_CUDA;
  return TCFFT_OK;
}

// Runs a persistent plan: counters to zero, then one launch of the queue
// kernel over the passes' parameters bound to (in, out).
tcfft_status exec_queue(tcfft_plan_s* plan, const void* in, void* out, cudaStream_t s) {
  QueueState& q = plan->q;
  PassParams* d_passes = nullptr;
  for (const QueueBinding& b : q.bindings)
    if (b.in == in && b.out == out) d_passes = b.d_passes;
  if (!d_passes) {
    std::vector<PassParams> hp;
    for (const Pass& ps : plan->passes) hp.push_back(bound_params(plan, ps, in, out));
    if (cudaMalloc(&d_passes, sizeof(PassParams) * hp.size()) != cudaSuccess) {
      (void)cudaGetLastError();
      return TCFFT_ERR_ALLOC;
    }
    if (cudaMemcpy(d_passes, hp.data(), sizeof(PassParams) * hp.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(d_passes);
      return TCFFT_ERR_CUDA;
    }
    if (q.bindings.size() >= 8) {  // keep a few buffer pairs
      cudaFree(q.bindings.front().d_passes);
      q.bindings.erase(q.bindings.begin());
    }
    q.bindings.push_back(QueueBinding{in, out, d_passes});
  }
  const int np = (int)plan->passes.size();
  if (cudaMemsetAsync(q.d_counters, 0, sizeof(int) * (2 + np), s) != cudaSuccess) return TCFFT_ERR_CUDA;
  QueueParams qp;
  qp.passes = d_passes;
  qp.dep = q.d_dep;
  qp.nchunks = q.d_nchunks;
  qp.items = q.d_items;
  qp.nitems = q.nitems;
  qp.head = q.d_counters;
  qp.abort = q.d_counters + 1;
  qp.done = q.d_counters + 2;
  qp.status = plan->d_status;
  qp.wait_limit = q.wait_limit;
  qp.a_bytes = q.a_bytes;
  qp.b_bytes = q.b_bytes;
  qp.tmem_cols = q.tmem_cols;
  void* args[1] = {&qp};
  return launch_pass(queue_fn(), q.grid, 128, q.smem, s, args) == cudaSuccess ? TCFFT_OK : TCFFT_ERR_LAUNCH;
}

constexpr unsigned kPlanFlags = TCFFT_PLAN_AUTOTUNE | TCFFT_PLAN_GRAPH | TCFFT_PLAN_INVERSE | TCFFT_PLAN_SCALE |
                                TCFFT_PLAN_SHARE_SM | TCFFT_PLAN_FUSED_2D | TCFFT_PLAN_PERSISTENT;

void apply_flags(tcfft_plan_s* pl, unsigned flags) {
  pl->autotune = (flags & TCFFT_PLAN_AUTOTUNE) || env_int("TCFFT_AUTOTUNE", 0);
  pl->use_graph = (flags & TCFFT_PLAN_GRAPH) != 0;
  pl->inverse = (flags & TCFFT_PLAN_INVERSE) != 0;
  pl->normalise = (flags & TCFFT_PLAN_SCALE) != 0;
  pl->share_sm = (flags & TCFFT_PLAN_SHARE_SM) != 0;
  pl->fused_2d = (flags & TCFFT_PLAN_FUSED_2D) != 0;
}

// Direction and scaling: the inverse DFT is conj(DFT(conj(x))), so the first
// pass of each transform conjugates its input and the last conjugates (and,
// with TCFFT_PLAN_SCALE, scales by 1/N) its output.  In a ragged plan the
// passes of each group are consecutive; the scale is per group.
void apply_direction(tcfft_plan_s* pl) {
  if (!pl->inverse && !pl->normalise) return;
  size_t i = 0;
  while (i < pl->passes.size()) {
    size_t j = i;
    while (j + 1 < pl->passes.size() && pl->passes[j + 1].group == pl->passes[i].group) ++j;
    pl->passes[i].p.conj_in = pl->inverse ? 1 : 0;
    (pl->passes[j].fused ? pl->passes[j].p2 : pl->passes[j].p).conj_out = pl->inverse ? 1 : 0;
    // 1/N is spread over the transform: every radix-16 stage uses F_16 / 16
    // (scaled DFT-matrix images, bound in bind_tables) and every leading
    // radix-R step scales by 1/R, so intermediates keep the input's magnitude
    if (pl->normalise)
      for (size_t k = i; k <= j; ++k) {
        pl->passes[k].p.prescale = 1.0f / (float)(1 << (pl->passes[k].p.log2N % 4));
        pl->passes[k].p2.prescale = pl->passes[k].p.prescale;
      }
    i = j + 1;
  }
}

// TCFFT_FP32 plans run the split kernels; every pass side on a user buffer
// (input or output, which 2D plans also use between their passes) reads or
// writes interleaved FP32 complex, the workspace keeps the hi / lo planes.
void apply_io(tcfft_plan_s* pl) {
  for (Pass& ps : pl->passes) {
    ps.p.in_f32 = (pl->fp32 && ps.src != BUF_WS) ? 1 : 0;
    (ps.fused ? ps.p2 : ps.p).out_f32 = (pl->fp32 && ps.dst != BUF_WS) ? 1 : 0;
  }
}

bool valid_precision(tcfft_precision pr) {
  return pr == TCFFT_FP16 || pr == TCFFT_FP16_SPLIT || pr == TCFFT_FP32;
}

void set_precision(tcfft_plan_s* pl, tcfft_precision pr) {
  pl->split = pr != TCFFT_FP16;
  pl->fp32 = pr == TCFFT_FP32;
}

tcfft_status check_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TCFFT_ERR_UNSUPPORTED;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return TCFFT_ERR_UNSUPPORTED;
  if (prop.major != 10 || prop.minor != 3) return TCFFT_ERR_UNSUPPORTED;
  return TCFFT_OK;
}

tcfft_status common_init(tcfft_plan_s* pl) {
  if (cudaMalloc(&pl->d_status, sizeof(int)) != cudaSuccess) return TCFFT_ERR_ALLOC;
  if (cudaMemset(pl->d_status, 0, sizeof(int)) != cudaSuccess) return TCFFT_ERR_CUDA;
  return TCFFT_OK;
}

tcfft_status finish(tcfft_plan_s* pl, tcfft_status st, tcfft_plan* out) {
  if (st == TCFFT_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = from_cuda(e);
  }
  if (st != TCFFT_OK) {
    delete pl;
    *out = nullptr;
    // a failed allocation leaves the runtime's last-error state set; clear it
    // so that later launch checks (of this or other plans) do not report it
    (void)cudaGetLastError();
    return st;
  }
  *out = pl;
  return TCFFT_OK;
}

}  // namespace

namespace {
// The pass's parameters with the exec's buffers filled in.
PassParams bound_params(const tcfft_plan_s* plan, const Pass& ps, const void* in, void* out) {
  PassParams p = ps.p;
  uint32_t* bufs[3] = {reinterpret_cast<uint32_t*>(const_cast<void*>(in)),
                       reinterpret_cast<uint32_t*>(out), reinterpret_cast<uint32_t*>(plan->ws)};
  p.in = bufs[ps.src] + (ps.src == BUF_WS ? ps.src_off : 0);
  p.out = bufs[ps.dst] + (ps.dst == BUF_WS ? ps.dst_off : 0);
  encode_in_map(p, plan->split);
  encode_out_map(p, plan->split);
  return p;
}

// A fused pass's parameters with the exec's buffers: the rows read `in`'s
// side of the pass, the columns write its output side; batch > 0 runs the
// first `batch` matrices of a dense plan (user buffers of `batch` matrices).
Fused2DParams bound_fused(const tcfft_plan_s* plan, const Pass& ps, const void* in, void* out, int64_t batch = 0) {
  Fused2DParams f;
  f.row = ps.p;
  f.col = ps.p2;
  f.log2K = ps.log2K;
  f.batch = ps.p.nchunks;
  uint32_t* bufs[3] = {reinterpret_cast<uint32_t*>(const_cast<void*>(in)),
                       reinterpret_cast<uint32_t*>(out), reinterpret_cast<uint32_t*>(plan->ws)};
  f.row.in = bufs[ps.src] + (ps.src == BUF_WS ? ps.src_off : 0);
  f.col.out = bufs[ps.dst] + (ps.dst == BUF_WS ? ps.dst_off : 0);
  f.row.out = f.col.out;
  f.col.in = f.row.in;
  if (batch > 0) {
    const int64_t S = int64_t(1) << ps.p.log2N;
    f.batch = batch;
    f.row.T = f.col.T = batch * S;
    f.row.nchunks = f.col.nchunks = batch;
    if (ps.src != BUF_WS) f.row.in_plane = batch * S * S;
    if (ps.dst != BUF_WS) f.col.out_plane = batch * S * S;
  }
  encode_out_map(f.col, plan->split);
  return f;
}

// Launches pass ps of the plan on `s` with the exec's buffers (the first
// `batch` transforms of a dense plan when batch > 0).
cudaError_t launch_plan_pass(const tcfft_plan_s* plan, const Pass& ps, const void* in, void* out, cudaStream_t s,
                             int64_t batch) {
  if (ps.fused) {
    Fused2DLaunch fl;
    fl.fn = ps.fn;
    fl.grid = ps.grid;
    fl.threads = ps.threads;
    fl.smem = ps.smem;
    const Fused2DParams f = bound_fused(plan, ps, in, out, batch);
    const unsigned K = 1u << ps.log2K;
    if (batch > 0) fl.grid.x = (unsigned)std::min<int64_t>(ps.grid.x, K * batch);
    return launch_fused2d(fl, f, s);
  }
  PassParams p = bound_params(plan, ps, in, out);
  dim3 grid = ps.grid;
  if (batch > 0) {
    const int64_t per = plan->points / plan->batch;  // points of one transform
    // every pass's transforms are the batch's transforms times a fixed count
    p.T = ps.p.T / plan->batch * batch;
    const int64_t C = int64_t(1) << p.log2C;
    p.nchunks = (p.T + C - 1) / C;
    // user buffers hold `batch` transforms per plane; the workspace keeps its layout
    if (ps.src != BUF_WS) p.in_plane = per * batch;
    if (ps.dst != BUF_WS) p.out_plane = per * batch;
    grid = dim3((unsigned)std::min<int64_t>(p.nchunks, (int64_t)ps.grid.x));
    p.in_tma = ps.p.in_tma;  // re-encode for the shorter batch
    p.out_tma = ps.p.out_tma;
    encode_in_map(p, plan->split);
    encode_out_map(p, plan->split);
  }
  void* args[1] = {&p};
  return launch_pass(ps.fn, grid, ps.threads, ps.smem, s, args);
}

// Replays the plan as one CUDA graph: passes of a group form a chain, the
// groups of a ragged plan are independent branches that the GPU may run
// concurrently.  One instantiated graph is kept per (in, out) pair.
tcfft_status exec_graph(tcfft_plan_s* plan, const void* in, void* out, cudaStream_t s) {
  for (const GraphEntry& g : plan->graphs)
    if (g.in == in && g.out == out)
      return cudaGraphLaunch(g.exec, s) == cudaSuccess ? TCFFT_OK : TCFFT_ERR_LAUNCH;
  cudaGraph_t graph;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return TCFFT_ERR_CUDA;
  std::map<int, cudaGraphNode_t> last;  // last node of each group
  tcfft_status st = TCFFT_OK;
  for (const Pass& ps : plan->passes) {
    PassParams p = ps.fused ? ps.p : bound_params(plan, ps, in, out);
    Fused2DParams f;
    if (ps.fused) f = bound_fused(plan, ps, in, out);
    void* args[1] = {ps.fused ? static_cast<void*>(&f) : static_cast<void*>(&p)};
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(ps.fn);
    kp.gridDim = ps.grid;
    kp.blockDim = dim3(ps.threads);
    kp.sharedMemBytes = (unsigned)ps.smem;
    kp.kernelParams = args;
    cudaGraphNode_t node;
    auto it = last.find(ps.group);
    if (cudaGraphAddKernelNode(&node, graph, nullptr, 0, &kp) != cudaSuccess) {
      st = TCFFT_ERR_CUDA;
      break;
    }
    if (ps.fused) {
      cudaKernelNodeAttrValue v = {};
      v.clusterDim.x = 1u << ps.log2K;
      v.clusterDim.y = 1;
      v.clusterDim.z = 1;
      if (cudaGraphKernelNodeSetAttribute(node, cudaKernelNodeAttributeClusterDimension, &v) != cudaSuccess) {
        st = TCFFT_ERR_CUDA;
        break;
      }
    }
    if (it != last.end()) {
      // programmatic edge: the pass starts its prologue while the previous
      // pass of the group finishes and waits (griddepcontrol.wait) before
      // reading its input; a plain edge where that is not available
      cudaGraphEdgeData e = {};
      e.from_port = cudaGraphKernelNodePortProgrammatic;
      e.type = cudaGraphDependencyTypeProgrammatic;
      if (cudaGraphAddDependencies(graph, &it->second, &node, &e, 1) != cudaSuccess) {
        (void)cudaGetLastError();
        if (cudaGraphAddDependencies(graph, &it->second, &node, nullptr, 1) != cudaSuccess) {
          st = TCFFT_ERR_CUDA;
          break;
        }
      }
    }
    last[ps.group] = node;
  }
  cudaGraphExec_t exec = nullptr;
  if (st == TCFFT_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) st = TCFFT_ERR_CUDA;
  cudaGraphDestroy(graph);
  if (st != TCFFT_OK) return st;
  if (plan->graphs.size() >= 8) {  // keep a few buffer pairs
    cudaGraphExecDestroy(plan->graphs.front().exec);
    plan->graphs.erase(plan->graphs.begin());
  }
  plan->graphs.push_back(GraphEntry{in, out, exec});
  return cudaGraphLaunch(exec, s) == cudaSuccess ? TCFFT_OK : TCFFT_ERR_LAUNCH;
}

// Waits on an mbarrier that no thread or copy ever completes, with the same
// bounded wait the pass kernels use, and reports the outcome.
__global__ void wait_timeout_selftest_kernel(long long limit_cycles, int* status) {
  __shared__ uint64_t bar;
  const uint32_t b = tcfft::smem_u32(&bar);
  if (threadIdx.x == 0) tcfft::mbar_init(b, 1);
  __syncthreads();
  const bool got = tcfft::mbar_wait_bounded(b, 0, limit_cycles);
  if (__syncthreads_or(!got) && threadIdx.x == 0) atomicExch(status, kDevErrTimeout);
}
}  // namespace

extern "C" {

tcfft_status tcfft_selftest_wait_timeout(long long limit_cycles) {
  if (limit_cycles < 0 || limit_cycles > 4000000000LL) return TCFFT_ERR_INVALID_VALUE;
  tcfft_status st = check_device();
  if (st != TCFFT_OK) return st;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return TCFFT_ERR_ALLOC;
  int v = 0;
  cudaMemset(d, 0, sizeof(int));
  wait_timeout_selftest_kernel<<<1, 32>>>(limit_cycles, d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return from_cuda(e);
  return (tcfft_status)v;
}

tcfft_status tcfft_selftest_queue_timeout(long long limit_cycles) {
  if (limit_cycles < 0 || limit_cycles > 4000000000LL) return TCFFT_ERR_INVALID_VALUE;
  // a persistent plan of one two-pass transform whose queue keeps only the
  // second pass's items: their producer is never enqueued, so the first
  // dependency wait runs out
  const int64_t n0[1] = {int64_t(1) << 16};
  tcfft_plan pl = nullptr;
  tcfft_status st = tcfft_plan_many(&pl, 1, n0, nullptr, TCFFT_FP16, TCFFT_PLAN_PERSISTENT);
  if (st != TCFFT_OK) return st;
  void* buf = nullptr;
  QueueState& q = pl->q;
  std::vector<int2> items(q.nitems);
  st = TCFFT_ERR_CUDA;
  if (pl->passes.size() == 2 &&
      cudaMemcpy(items.data(), q.d_items, sizeof(int2) * items.size(), cudaMemcpyDeviceToHost) == cudaSuccess) {
    std::vector<int2> kept;
    for (const int2& it : items)
      if (it.x == 1) kept.push_back(it);
    if (!kept.empty() && cudaMemcpy(q.d_items, kept.data(), sizeof(int2) * kept.size(), cudaMemcpyHostToDevice) ==
                             cudaSuccess &&
        cudaMalloc(&buf, pl->io_bytes()) == cudaSuccess && cudaMemset(buf, 0, pl->io_bytes()) == cudaSuccess) {
      q.nitems = (int)kept.size();
      q.wait_limit = limit_cycles;
      st = exec_queue(pl, buf, buf, nullptr);
      if (st == TCFFT_OK) st = tcfft_plan_last_error(pl);
    }
  }
  cudaFree(buf);
  tcfft_destroy(pl);
  (void)cudaGetLastError();
  return st;
}

tcfft_status tcfft_plan_1d_ex(tcfft_plan* plan, int64_t n, int64_t batch, tcfft_precision precision,
                              unsigned flags) {
  if (!plan) return TCFFT_ERR_INVALID_VALUE;
  *plan = nullptr;
  if ((flags & ~kPlanFlags) != 0 || !valid_precision(precision)) return TCFFT_ERR_INVALID_VALUE;
  if (!is_pow2(n) || n < 16 || ilog2(n) > kMaxLog2_1D || batch < 1) return TCFFT_ERR_INVALID_SIZE;
  if (batch > (int64_t(1) << 40) / n) return TCFFT_ERR_INVALID_SIZE;
  tcfft_status st = check_device();
  if (st != TCFFT_OK) return st;
  tcfft_plan_s* pl = new (std::nothrow) tcfft_plan_s();
  if (!pl) return TCFFT_ERR_ALLOC;
  pl->dims = 1;
  pl->n = n;
  pl->batch = batch;
  set_precision(pl, precision);
  pl->points = n * batch;
  apply_flags(pl, flags);
  st = common_init(pl);
  if (st == TCFFT_OK) st = plan_1d(pl);
  if (st == TCFFT_OK) apply_direction(pl);
  if (st == TCFFT_OK) apply_io(pl);
  return finish(pl, st, plan);
}

tcfft_status tcfft_plan_1d(tcfft_plan* plan, int64_t n, int64_t batch) {
  return tcfft_plan_1d_ex(plan, n, batch, TCFFT_FP16, 0);
}

tcfft_status tcfft_plan_2d_ex(tcfft_plan* plan, int64_t nx, int64_t ny, int64_t batch,
                              tcfft_precision precision, unsigned flags) {
  if (!plan) return TCFFT_ERR_INVALID_VALUE;
  *plan = nullptr;
  if ((flags & ~kPlanFlags) != 0 || !valid_precision(precision)) return TCFFT_ERR_INVALID_VALUE;
  if (!is_pow2(nx) || !is_pow2(ny) || nx < 16 || ny < 16 || ilog2(nx) > kMaxLog2_2D ||
      ilog2(ny) > kMaxLog2_2D || batch < 1)
    return TCFFT_ERR_INVALID_SIZE;
  if (batch > (int64_t(1) << 40) / (nx * ny)) return TCFFT_ERR_INVALID_SIZE;
  tcfft_status st = check_device();
  if (st != TCFFT_OK) return st;
  tcfft_plan_s* pl = new (std::nothrow) tcfft_plan_s();
  if (!pl) return TCFFT_ERR_ALLOC;
  pl->dims = 2;
  pl->nx = nx;
  pl->ny = ny;
  pl->batch = batch;
  set_precision(pl, precision);
  pl->points = nx * ny * batch;
  apply_flags(pl, flags);
  st = common_init(pl);
  if (st == TCFFT_OK) st = plan_2d(pl);
  if (st == TCFFT_OK) apply_direction(pl);
  if (st == TCFFT_OK) apply_io(pl);
  return finish(pl, st, plan);
}

tcfft_status tcfft_plan_many(tcfft_plan* plan, int64_t count, const int64_t* n0, const int64_t* n1,
                             tcfft_precision precision, unsigned flags) {
  if (!plan) return TCFFT_ERR_INVALID_VALUE;
  *plan = nullptr;
  if (!n0 || (flags & ~kPlanFlags) != 0 || !valid_precision(precision)) return TCFFT_ERR_INVALID_VALUE;
  if (count < 1 || count > (int64_t(1) << 24)) return TCFFT_ERR_INVALID_SIZE;
  int64_t total = 0;
  for (int64_t i = 0; i < count; ++i) {
    const int64_t a = n0[i], b = n1 ? n1[i] : 0;
    if (b == 0) {
      if (!is_pow2(a) || a < 16 || ilog2(a) > kMaxLog2_Ragged1D) return TCFFT_ERR_INVALID_SIZE;
      if (precision != TCFFT_FP16 && ilog2(a) > 22) return TCFFT_ERR_INVALID_SIZE;
    } else {
      if (!is_pow2(a) || !is_pow2(b) || a < 16 || b < 16 || ilog2(a) > kMaxLog2_2D || ilog2(b) > kMaxLog2_2D)
        return TCFFT_ERR_INVALID_SIZE;
    }
    total += b ? a * b : a;
    if (total > (int64_t(1) << 40)) return TCFFT_ERR_INVALID_SIZE;
  }
  tcfft_status st = check_device();
  if (st != TCFFT_OK) return st;
  tcfft_plan_s* pl = new (std::nothrow) tcfft_plan_s();
  if (!pl) return TCFFT_ERR_ALLOC;
  pl->dims = 0;
  pl->batch = count;
  set_precision(pl, precision);
  apply_flags(pl, flags);
  // TCFFT_PLAN_PERSISTENT: plain FP16 ragged plans run as one persistent
  // launch over a work queue (other precisions keep one launch per pass)
  pl->queue = (flags & TCFFT_PLAN_PERSISTENT) && precision == TCFFT_FP16;
  if (pl->queue) pl->fused_2d = false;
  st = common_init(pl);
  if (st == TCFFT_OK) st = plan_many(pl, count, n0, n1);
  if (st == TCFFT_OK) apply_direction(pl);
  if (st == TCFFT_OK) apply_io(pl);
  if (st == TCFFT_OK && pl->queue) st = build_queue(pl);
  return finish(pl, st, plan);
}

tcfft_status tcfft_plan_2d(tcfft_plan* plan, int64_t nx, int64_t ny, int64_t batch) {
  return tcfft_plan_2d_ex(plan, nx, ny, batch, TCFFT_FP16, 0);
}

tcfft_status tcfft_exec(tcfft_plan plan, const void* in, void* out, void* stream) {
  if (!plan || !in || !out) return TCFFT_ERR_INVALID_VALUE;
  if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
    return TCFFT_ERR_INVALID_VALUE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (plan->queue) return exec_queue(plan, in, out, s);
  if (plan->use_graph) return exec_graph(plan, in, out, s);
  for (const Pass& ps : plan->passes) {
    cudaError_t e = launch_plan_pass(plan, ps, in, out, s);
    if (e != cudaSuccess) {
      if (env_int("TCFFT_DEBUG", 0))
        std::fprintf(stderr, "tcfft_exec: launch of pass (log2n %d, grid %u, smem %zu) failed: %s\n",
                     ps.p.log2N, ps.grid.x, ps.smem, cudaGetErrorString(e));
      return TCFFT_ERR_LAUNCH;
    }
  }
  return TCFFT_OK;
}

tcfft_status tcfft_exec_batch(tcfft_plan plan, const void* in, void* out, int64_t batch, void* stream) {
  if (!plan || !in || !out) return TCFFT_ERR_INVALID_VALUE;
  if (plan->dims == 0) return TCFFT_ERR_UNSUPPORTED;  // ragged plans run as planned
  if (batch < 1 || batch > plan->batch) return TCFFT_ERR_INVALID_SIZE;
  if (batch == plan->batch) return tcfft_exec(plan, in, out, stream);
  if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
    return TCFFT_ERR_INVALID_VALUE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (const Pass& ps : plan->passes)
    if (launch_plan_pass(plan, ps, in, out, s, batch) != cudaSuccess) return TCFFT_ERR_LAUNCH;
  return TCFFT_OK;
}

tcfft_status tcfft_exec_host(tcfft_plan plan, const void* host_in, void* host_out, void* stream) {
  if (!plan || !host_in || !host_out) return TCFFT_ERR_INVALID_VALUE;
  const size_t bytes = plan->io_bytes();
  if (!plan->h_in_dev) {
    if (cudaMalloc(&plan->h_in_dev, bytes) != cudaSuccess) {
      plan->h_in_dev = nullptr;
      (void)cudaGetLastError();  // not a sticky error: clear it for later checks
      return TCFFT_ERR_ALLOC;
    }
    if (cudaMalloc(&plan->h_out_dev, bytes) != cudaSuccess) {
      cudaFree(plan->h_in_dev);
      plan->h_in_dev = nullptr;
      plan->h_out_dev = nullptr;
      (void)cudaGetLastError();
      return TCFFT_ERR_ALLOC;
    }
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // Single-plane batches (plain or FP32) run as up to kHostSlices slices of
  // whole transforms: slice j's upload (upload stream), transform (the
  // caller's stream, so that slices share the workspace in turn) and download
  // (download stream) are chained by events, so uploads, transforms and
  // downloads of different slices overlap on the copy engines and the SMs.
  int slices = 1;
  if (plan->dims != 0 && (!plan->split || plan->fp32) && plan->batch >= 2 && plan->points >= (int64_t(1) << 22)) {
    while (slices < kHostSlices && plan->batch % (2 * slices) == 0 &&
           plan->points / (2 * slices) >= (int64_t(1) << 21))
      slices *= 2;
  }
  if (slices > 1 && !plan->h_up) {
    bool ok = cudaStreamCreateWithFlags(&plan->h_up, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&plan->h_down, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&plan->h_entry, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < kHostSlices && ok; ++i)
      ok = cudaEventCreateWithFlags(&plan->h_ev_up[i], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&plan->h_ev_done[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) slices = 1;  // the handles made so far are released with the plan
  }
  if (slices == 1 || !plan->h_up) {
    cudaError_t e = cudaMemcpyAsync(plan->h_in_dev, host_in, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return from_cuda(e);
    tcfft_status st = tcfft_exec(plan, plan->h_in_dev, plan->h_out_dev, stream);
    if (st != TCFFT_OK) return st;
    e = cudaMemcpyAsync(host_out, plan->h_out_dev, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return from_cuda(e);
    return from_cuda(cudaStreamSynchronize(s));
  }
  const int64_t per_slice = plan->batch / slices;
  const size_t sbytes = bytes / (size_t)slices;
  const char* hin = static_cast<const char*>(host_in);
  char* hout = static_cast<char*>(host_out);
  char* din = static_cast<char*>(plan->h_in_dev);
  char* dout = static_cast<char*>(plan->h_out_dev);
  // the slices start after the caller's earlier work on `stream`
  cudaError_t e = cudaEventRecord(plan->h_entry, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->h_up, plan->h_entry, 0);
  for (int j = 0; j < slices && e == cudaSuccess; ++j) {
    const size_t off = (size_t)j * sbytes;
    e = cudaMemcpyAsync(din + off, hin + off, sbytes, cudaMemcpyHostToDevice, plan->h_up);
    if (e == cudaSuccess) e = cudaEventRecord(plan->h_ev_up[j], plan->h_up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->h_ev_up[j], 0);
    if (e != cudaSuccess) break;
    tcfft_status st = tcfft_exec_batch(plan, din + off, dout + off, per_slice, stream);
    if (st != TCFFT_OK) {
      cudaStreamSynchronize(plan->h_up);
      cudaStreamSynchronize(s);
      return st;
    }
    e = cudaEventRecord(plan->h_ev_done[j], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->h_down, plan->h_ev_done[j], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hout + off, dout + off, sbytes, cudaMemcpyDeviceToHost, plan->h_down);
  }
  const cudaError_t e1 = cudaStreamSynchronize(plan->h_up);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  const cudaError_t e3 = cudaStreamSynchronize(plan->h_down);
  if (e != cudaSuccess) return from_cuda(e);
  if (e1 != cudaSuccess) return from_cuda(e1);
  if (e2 != cudaSuccess) return from_cuda(e2);
  return from_cuda(e3);
}

tcfft_status tcfft_destroy(tcfft_plan plan) {
  delete plan;
  return TCFFT_OK;
}

tcfft_status tcfft_plan_last_error(tcfft_plan plan) {
  if (!plan) return TCFFT_ERR_INVALID_VALUE;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return from_cuda(e);
  int v = 0;
  e = cudaMemcpy(&v, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return from_cuda(e);
  cudaMemset(plan->d_status, 0, sizeof(int));
  return (tcfft_status)v;
}

size_t tcfft_io_bytes(tcfft_plan plan) { return plan ? plan->io_bytes() : 0; }

size_t tcfft_workspace_bytes(tcfft_plan plan) {
  if (!plan) return 0;
  size_t b = plan->ws_bytes + plan->table_bytes + sizeof(int);
  if (plan->h_in_dev) b += 2 * plan->io_bytes();
  return b;
}

int tcfft_plan_num_launches(tcfft_plan plan) {
  if (!plan) return 0;
  return plan->queue ? 1 : (int)plan->passes.size();
}

size_t tcfft_plan_describe(tcfft_plan plan, char* buf, size_t len) {
  if (!plan) return 0;
  std::string out = "[";
  for (size_t i = 0; i < plan->passes.size(); ++i) {
    const Pass& ps = plan->passes[i];
    const PassParams& p = ps.p;
    const char* modes[4] = {"contig", "strided", "contig_to_strided", "fused_2d"};
    const int mode = ps.fused ? 3 : ((p.in_l.es == 1) ? ((p.out_l.es == 1) ? 0 : 2) : 1);
    char tmp[512];
    std::snprintf(tmp, sizeof(tmp),
                  "%s{\"log2n\": %d, \"mode\": \"%s\", \"transforms\": %lld, \"per_cta\": %d, "
                  "\"tiles\": %d, \"tmem_cols\": %d, \"smem\": %zu, \"async_load\": %d, \"grid\": %u, "
                  "\"chunks\": %lld, \"out_twiddle\": %d, \"ctas_per_sm\": %d, \"regs\": %d, "
                  "\"threads\": %d, \"cluster\": %d, \"queue\": %d}",
                  i ? ", " : "", p.log2N, modes[mode], (long long)p.T, 1 << p.log2C, p.tiles, p.tmem_cols,
                  ps.smem, p.async_load, ps.grid.x, (long long)p.nchunks, p.otw_level, ps.occ, ps.regs,
                  ps.threads, 1 << ps.log2K, plan->queue ? 1 : 0);
    out += tmp;
  }
  out += "]";
  if (buf && len) {
    std::strncpy(buf, out.c_str(), len - 1);
    buf[len - 1] = 0;
  }
  return out.size() + 1;
}

const char* tcfft_status_string(tcfft_status s) {
  switch (s) {
    case TCFFT_OK: return "TCFFT_OK";
    case TCFFT_ERR_INVALID_SIZE: return "TCFFT_ERR_INVALID_SIZE";
    case TCFFT_ERR_INVALID_VALUE: return "TCFFT_ERR_INVALID_VALUE";
    case TCFFT_ERR_ALLOC: return "TCFFT_ERR_ALLOC";
    case TCFFT_ERR_LAUNCH: return "TCFFT_ERR_LAUNCH";
    case TCFFT_ERR_TIMEOUT: return "TCFFT_ERR_TIMEOUT";
    case TCFFT_ERR_UNSUPPORTED: return "TCFFT_ERR_UNSUPPORTED";
    case TCFFT_ERR_NOT_IMPLEMENTED: return "TCFFT_ERR_NOT_IMPLEMENTED";
    case TCFFT_ERR_CUDA: return "TCFFT_ERR_CUDA";
  }
  return "TCFFT_ERR_UNKNOWN";
}

}  // extern "C"
