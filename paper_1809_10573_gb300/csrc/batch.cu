// An uneven batch of IDBF applies (operators of different N, each with its own number of
// right-hand sides) in ONE persistent kernel launch, captured in a CUDA graph.
//
// Work items are (operator, level, run of nodes, block of right-hand sides). They are queued in
// the order of the levels (all level-0 items of every operator, then all level-1 items, ...),
// and persistent CTAs take them from the queue with an atomic counter. Before starting an item
// of level l, a CTA waits until every item of level l-1 of the same operator has finished (a
// per-(operator, level) completion counter). Those items are earlier in the queue, so they have
// already been taken by CTAs that are running, and the wait ends: there is no cycle, whatever the
// number of resident CTAs. Every wait is bounded in time; on a timeout the item is counted as done
// (its results are invalid), bit 0 of the status word is set, and idbf_batch_sync_status reports
// IDBF_ETIMEOUT.
//
// Each node is computed by fwd_node (right-hand sides per thread) or fwd_node_tiled (register
// tiles), the bodies of the per-level kernels (level_kernels.cuh); the tile, or a per-level mix
// of the two by block height, is autotuned.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "idbf_internal.h"
#include "level_kernels.cuh"

namespace idbf {
namespace bat {

struct OpLevel {
  DevLevel d;
  const void* mat;
  int gcap, rcap, max_in, max_out, max_rows;
  int body;  // mixed tiling: 1 = tiled body (16 right-hand sides per item), 0 = per-thread body (8)
};
struct OpDesc {
  int L, R, level_base, pad;
  void* ws0;
  void* ws1;
};
struct Item {
  int op, level, node0, nodes, r0, pad;
};

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int NT = 256;

// Tiles: right-hand sides per work item (RB); then either right-hand sides per thread (RPT, the
// per-node body fwd_node, all precisions) or TC > 0: the tiled body fwd_node_tiled with TR x TC
// register tiles and streamed factor columns (FP32 and FP64), or TC < 0: mixed, per level: the
// tiled body with 16 right-hand sides per item where the level's blocks have more than a
// threshold of rows, else the per-thread body with 8 per item, 4 per thread (FP32 and FP64).
struct Tile {
  int rb, rpt, tc;
};
constexpr Tile kTiles[] = {{1, 1, 0}, {4, 2, 0}, {8, 2, 0}, {8, 4, 0}, {8, 0, 4}, {16, 0, 4}, {32, 0, 8}, {16, 4, -1}};
constexpr int kNumTiles = 8;
constexpr int kMixedSmallRB = 8;
template <class P>
__host__ __device__ constexpr int max_rb() {
  return std::is_same<P, FP32P>::value ? 32 : std::is_same<P, FP64P>::value ? 16 : 8;
}
template <class P>
__host__ __device__ constexpr bool tiled_ok() {
  return std::is_same<typename P::vec_t, typename P::gv_t>::value;
}
template <class P, int T>
constexpr bool instantiated() {
  return kTiles[T].rb <= max_rb<P>() && (kTiles[T].tc == 0 || tiled_ok<P>());
}

template <class P, int RB, int RPT, int TC>
__global__ void __launch_bounds__(NT, TC == 8 ? 1 : 2) k_batch(const OpDesc* __restrict__ ops, const OpLevel* __restrict__ lv,
                                              const Item* __restrict__ items, int nitems, const void* const* xs,
                                              void* const* ys, const int64_t* lds, int* head, int* done,
                                              const int* __restrict__ target, int* status, uint64_t limit_ns) {
  using V = typename P::vec_t;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int sidx, sfail;
  for (;;) {
    __syncthreads();  // the previous item's shared memory and sidx are no longer in use
    if (threadIdx.x == 0) sidx = atomicAdd(head, 1);
    __syncthreads();
    const int i = sidx;
    if (i >= nitems) break;
    const Item w = items[i];
    const OpDesc od = ops[w.op];
    const int li = od.level_base + w.level;
    if (threadIdx.x == 0) {
      sfail = 0;
      if (w.level > 0) {
        volatile int* dp = done + (li - 1);
        const int need = target[li - 1];
        if (*dp < need) {
          const uint64_t t0 = gtimer();
          while (*dp < need) {
            if (gtimer() - t0 > limit_ns) {
              sfail = 1;
              atomicOr(status, 1);
              break;
            }
          }
        }
        __threadfence();  // acquire: the previous level's outputs are visible
      }
    }
    __syncthreads();
    if (!sfail) {
      const OpLevel ol = lv[li];
      IO<V> io;
      io.x = (const V*)xs[w.op];
      io.ldx = lds[w.op];
      io.y = (V*)ys[w.op];
      io.ldy = lds[w.op];
      io.R = od.R;
      V* wb[2] = {(V*)od.ws0, (V*)od.ws1};
      io.win = w.level > 0 ? wb[(w.level - 1) & 1] : nullptr;
      io.wout = w.level < od.L ? wb[w.level & 1] : nullptr;
      for (int n = 0; n < w.nodes; ++n) {
        if (n) __syncthreads();
        if constexpr (TC > 0) {
          fwd_node_tiled<P, RB, TC>(ol.d, (const typename P::mat_t*)ol.mat, io, ol.max_rows, ol.max_in, ol.max_out,
                                    (int64_t)(w.node0 + n), w.r0, smem);
        } else if constexpr (TC < 0) {
          if (ol.body)
            fwd_node_tiled<P, RB, 4>(ol.d, (const typename P::mat_t*)ol.mat, io, ol.max_rows, ol.max_in, ol.max_out,
                                     (int64_t)(w.node0 + n), w.r0, smem);
          else
            fwd_node<P, kMixedSmallRB, RPT>(ol.d, (const typename P::mat_t*)ol.mat, io, ol.gcap, ol.rcap, ol.max_in,
                                            (int64_t)(w.node0 + n), w.r0, smem);
        } else {
          fwd_node<P, RB, RPT>(ol.d, (const typename P::mat_t*)ol.mat, io, ol.gcap, ol.rcap, ol.max_in,
                               (int64_t)(w.node0 + n), w.r0, smem);
        }
      }
    }
    __threadfence();  // release: this item's outputs before its completion count
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(done + li, 1);
  }
}

template <class P, int RB, int RPT, int TC>
size_t node_smem(const LevelInfo& li, bool tiled_body) {
  const int gcap = std::max(std::max(li.max_cols, li.max_rows), li.max_in);
  const int rcap = std::max(li.max_rows, li.max_cols);
  if constexpr (TC > 0)
    return tiled::smem_bytes<P, RB, TC>(li.max_in, li.max_out, li.max_rows, NT);
  else if constexpr (TC < 0)
    return tiled_body ? tiled::smem_bytes<P, RB, 4>(li.max_in, li.max_out, li.max_rows, NT)
                      : fwd_node_smem<P, kMixedSmallRB, RPT>(li.max_in, gcap, rcap, NT);
  else
    return fwd_node_smem<P, RB, RPT>(li.max_in, gcap, rcap, NT);
}

}  // namespace bat
}  // namespace idbf

using namespace idbf;

struct idbf_batch_s {
  int device = 0, nops = 0, mode = 0, fmt = 0;
  std::vector<idbf_plan> plans;
  std::vector<int64_t> R;
  std::vector<void*> ws;
  bat::OpDesc* d_ops = nullptr;
  bat::OpLevel* d_lv = nullptr;
  int nlevels_total = 0;
  bat::Item* d_items = nullptr;
  int nitems = 0;
  int* d_counters = nullptr;  // head, then done[nlevels_total]
  int* d_target = nullptr;
  int* d_status = nullptr;
  void** d_ptrs = nullptr;    // xs[nops], ys[nops], then lds[nops] (int64)
  int tile = 1, rb = 4, npi = 1;  // tile: index into bat::kTiles
  int mix_rows = 64;              // mixed tiling: levels with at most this many rows per block use the per-thread body
  std::vector<bat::OpLevel> h_lv; // host copy of the level table (the body flags change with mix_rows)
  size_t smem = 0;
  int ctas = 0;
  uint64_t limit_ns = 2000000000ull;
  int debug_extra = 0;  // fault injection: added to the first operator's level-0 completion target
  int64_t split_n = INT64_MAX;  // operators with N >= split_n run through idbf_apply, not the launch
  bool split_auto = true;       // idbf_batch_autotune chooses split_n
  std::vector<char> sep;        // per operator: runs through idbf_apply
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
};

namespace {

void free_layout(idbf_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_target) cudaFree(b->d_target);
  if (b->d_counters) cudaFree(b->d_counters);
  b->d_items = nullptr;
  b->d_target = nullptr;
  b->d_counters = nullptr;
}

template <class P, int T>
idbf_status launch_batch(idbf_batch_s* b, cudaStream_t st) {
  constexpr int RB = bat::kTiles[T].rb, RPT = bat::kTiles[T].rpt, TC = bat::kTiles[T].tc;
  if constexpr (!bat::instantiated<P, T>()) {
    return IDBF_EUNSUPPORTED;
  } else {
    if (b->smem > 48 * 1024)
      IDBF_CUDA_TRY(cudaFuncSetAttribute(bat::k_batch<P, RB, RPT, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)b->smem));
    const void* const* xs = (const void* const*)b->d_ptrs;
    void* const* ys = (void* const*)(b->d_ptrs + b->nops);
    const int64_t* lds = (const int64_t*)(b->d_ptrs + 2 * b->nops);
    IDBF_CUDA_TRY(cudaMemsetAsync(b->d_counters, 0, sizeof(int) * (1 + b->nlevels_total), st));
    bat::k_batch<P, RB, RPT, TC><<<b->ctas, bat::NT, b->smem, st>>>(b->d_ops, b->d_lv, b->d_items, b->nitems, xs, ys, lds,
                                                                 b->d_counters, b->d_counters + 1, b->d_target,
                                                                 b->d_status, b->limit_ns);
    IDBF_CUDA_TRY(cudaGetLastError());
    return IDBF_OK;
  }
}

// shared memory per CTA: the largest node of any level of any operator (0 if the tile is not
// instantiated for this precision)
template <class P, int T>
size_t smem_for(idbf_batch_s* b) {
  constexpr int RB = bat::kTiles[T].rb, RPT = bat::kTiles[T].rpt, TC = bat::kTiles[T].tc;
  if constexpr (!bat::instantiated<P, T>()) {
    return 0;
  } else {
    size_t sm = 0;
    for (int o = 0; o < b->nops; ++o) {
      if (b->sep[o]) continue;
      for (const LevelInfo& li : b->plans[o]->p.lv)
        sm = std::max(sm, bat::node_smem<P, RB, RPT, TC>(li, li.max_rows > b->mix_rows));
    }
    return sm;
  }
}

template <class P, int T>
int occupancy(idbf_batch_s* b) {
  constexpr int RB = bat::kTiles[T].rb, RPT = bat::kTiles[T].rpt, TC = bat::kTiles[T].tc;
  if constexpr (!bat::instantiated<P, T>()) {
    return 1;
  } else {
    int n = 0;
    if (b->smem > 48 * 1024)
      cudaFuncSetAttribute(bat::k_batch<P, RB, RPT, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bat::k_batch<P, RB, RPT, TC>, bat::NT, b->smem);
    return std::max(n, 1);
  }
}

// calls F<P, tile>::run(b, args...) for the batch's precision and current tile
#define IDBF_BATCH_DISPATCH(FN, RET_ON_BAD, ...)                                               \
  [&]() {                                                                                      \
    switch (b->mode) {                                                                         \
      case IDBF_MODE_FP64: switch (b->tile) {                                                  \
          case 0: return FN<FP64P, 0>(__VA_ARGS__); case 1: return FN<FP64P, 1>(__VA_ARGS__);  \
          case 2: return FN<FP64P, 2>(__VA_ARGS__); case 3: return FN<FP64P, 3>(__VA_ARGS__);  \
          case 4: return FN<FP64P, 4>(__VA_ARGS__); case 5: return FN<FP64P, 5>(__VA_ARGS__);  \
          case 6: return FN<FP64P, 6>(__VA_ARGS__); case 7: return FN<FP64P, 7>(__VA_ARGS__);  \
          default: return RET_ON_BAD; }                                                        \
      case IDBF_MODE_DF64: switch (b->tile) {                                                  \
          case 0: return FN<DF64P, 0>(__VA_ARGS__); case 1: return FN<DF64P, 1>(__VA_ARGS__);  \
          case 2: return FN<DF64P, 2>(__VA_ARGS__); case 3: return FN<DF64P, 3>(__VA_ARGS__);  \
          case 4: return FN<DF64P, 4>(__VA_ARGS__); case 5: return FN<DF64P, 5>(__VA_ARGS__);  \
          case 6: return FN<DF64P, 6>(__VA_ARGS__); case 7: return FN<DF64P, 7>(__VA_ARGS__);  \
          default: return RET_ON_BAD; }                                                        \
      default: switch (b->tile) {                                                              \
          case 0: return FN<FP32P, 0>(__VA_ARGS__); case 1: return FN<FP32P, 1>(__VA_ARGS__);  \
          case 2: return FN<FP32P, 2>(__VA_ARGS__); case 3: return FN<FP32P, 3>(__VA_ARGS__);  \
          case 4: return FN<FP32P, 4>(__VA_ARGS__); case 5: return FN<FP32P, 5>(__VA_ARGS__);  \
          case 6: return FN<FP32P, 6>(__VA_ARGS__); case 7: return FN<FP32P, 7>(__VA_ARGS__);  \
          default: return RET_ON_BAD; }                                                        \
    }                                                                                          \
  }()

idbf_status launch(idbf_batch_s* b, cudaStream_t st) {
  return IDBF_BATCH_DISPATCH(launch_batch, IDBF_EINVAL, b, st);
}

bool tile_valid(int mode, int tile) {
  if (tile < 0 || tile >= bat::kNumTiles) return false;
  const bat::Tile t = bat::kTiles[tile];
  switch (mode) {
    case IDBF_MODE_FP64: return t.rb <= bat::max_rb<FP64P>();
    case IDBF_MODE_DF64: return t.rb <= bat::max_rb<DF64P>() && t.tc == 0;
    default: return t.rb <= bat::max_rb<FP32P>();
  }
}

// Queue of items, completion targets and the captured graph for the current (rb, npi).
idbf_status layout(idbf_batch_s* b) {
  free_layout(b);
  if (!tile_valid(b->mode, b->tile)) return IDBF_EUNSUPPORTED;
  b->rb = bat::kTiles[b->tile].rb;
  const bool mixed = bat::kTiles[b->tile].tc < 0;
  b->sep.assign(b->nops, 0);
  for (int o = 0; o < b->nops; ++o) b->sep[o] = b->plans[o]->p.N >= b->split_n ? 1 : 0;
  // level bodies of the mixed tiling (ignored by the others)
  for (int o = 0, li = 0; o < b->nops; ++o)
    for (const LevelInfo& lvi : b->plans[o]->p.lv) b->h_lv[li++].body = lvi.max_rows > b->mix_rows ? 1 : 0;
  IDBF_CUDA_TRY(cudaMemcpy(b->d_lv, b->h_lv.data(), sizeof(bat::OpLevel) * b->h_lv.size(), cudaMemcpyHostToDevice));
  std::vector<bat::Item> items;
  std::vector<int> target(b->nlevels_total, 0);
  int maxL = 0, base = 0;
  std::vector<int> lbase(b->nops);
  for (int o = 0; o < b->nops; ++o) {
    lbase[o] = base;
    base += b->plans[o]->p.L + 1;
    maxL = std::max(maxL, b->plans[o]->p.L);
  }
  for (int l = 0; l <= maxL; ++l)
    for (int o = 0; o < b->nops; ++o) {
      const Plan& p = b->plans[o]->p;
      if (l > p.L || b->sep[o]) continue;
      // the right-hand-side blocks of a run of nodes are neighbours in the queue, so the
      // blocks' second and later reads of the factors come from L2
      const int rbl = mixed && !b->h_lv[lbase[o] + l].body ? bat::kMixedSmallRB : b->rb;
      for (int n0 = 0; n0 < p.m; n0 += b->npi)
        for (int r0 = 0; r0 < b->R[o]; r0 += rbl) {
          bat::Item it;
          it.op = o;
          it.level = l;
          it.node0 = n0;
          it.nodes = std::min(b->npi, p.m - n0);
          it.r0 = r0;
          it.pad = 0;
          items.push_back(it);
          ++target[lbase[o] + l];
        }
    }
  b->nitems = (int)items.size();
  if (b->debug_extra > 0 && b->nlevels_total > 0) target[0] += b->debug_extra;
  if (!tile_valid(b->mode, b->tile)) return IDBF_EUNSUPPORTED;
  if (b->nitems == 0) {  // every operator runs through idbf_apply: no persistent launch
    b->smem = 0;
    b->ctas = 0;
    return IDBF_OK;
  }
  b->smem = IDBF_BATCH_DISPATCH(smem_for, (size_t)0, b);
  if (b->smem == 0 || b->smem > 200 * 1024) return IDBF_EUNSUPPORTED;
  const int occ = IDBF_BATCH_DISPATCH(occupancy, 1, b);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  b->ctas = std::max(1, std::min(occ * sms, b->nitems));
  IDBF_CUDA_TRY(cudaMalloc((void**)&b->d_items, sizeof(bat::Item) * std::max(1, b->nitems)));
  IDBF_CUDA_TRY(cudaMalloc((void**)&b->d_target, sizeof(int) * b->nlevels_total));
  IDBF_CUDA_TRY(cudaMalloc((void**)&b->d_counters, sizeof(int) * (1 + b->nlevels_total)));
  IDBF_CUDA_TRY(cudaMemcpy(b->d_items, items.data(), sizeof(bat::Item) * b->nitems, cudaMemcpyHostToDevice));
  IDBF_CUDA_TRY(cudaMemcpy(b->d_target, target.data(), sizeof(int) * b->nlevels_total, cudaMemcpyHostToDevice));
  // capture: reset the counters, run the persistent kernel
  IDBF_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  idbf_status s = launch(b, b->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (s != IDBF_OK) { if (g) cudaGraphDestroy(g); return s; }
  if (e != cudaSuccess) { set_cuda_error(e); return IDBF_ECUDA; }
  b->graph = g;
  IDBF_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
  return IDBF_OK;
}

}  // namespace

extern "C" {

idbf_status idbf_batch_create(const idbf_plan* plans, int32_t nops, const int64_t* nrhs, int32_t mode, idbf_batch* out) {
  if (!out) return IDBF_EINVAL;
  *out = nullptr;
  if (!plans || !nrhs || nops < 1 || nops > (1 << 16)) return IDBF_EINVAL;
  if (mode != IDBF_MODE_FP64 && mode != IDBF_MODE_DF64 && mode != IDBF_MODE_FP32) return IDBF_EINVAL;
  const int fmt = mode == IDBF_MODE_FP64 ? IDBF_STORE_C128 : mode == IDBF_MODE_DF64 ? IDBF_STORE_DF64 : IDBF_STORE_C64;
  int dev = 0;
  cudaGetDevice(&dev);
  for (int o = 0; o < nops; ++o) {
    if (!plans[o] || nrhs[o] < 1 || nrhs[o] > (1 << 16) || plans[o]->p.device != dev) return IDBF_EINVAL;
    if (!plans[o]->p.has_format(fmt) || plans[o]->p.uneven) return IDBF_EUNSUPPORTED;
  }
  idbf_batch_s* b = new (std::nothrow) idbf_batch_s();
  if (!b) return IDBF_ENOMEM;
  b->device = dev;
  b->nops = nops;
  b->mode = mode;
  b->fmt = fmt;
  b->plans.assign(plans, plans + nops);
  b->R.assign(nrhs, nrhs + nops);
  std::vector<bat::OpDesc> ods(nops);
  std::vector<bat::OpLevel> lvs;
  idbf_status s = IDBF_OK;
  for (int o = 0; o < nops && s == IDBF_OK; ++o) {
    const Plan& p = plans[o]->p;
    const size_t half = (size_t)p.max_seg_total * nrhs[o] * 16;
    void* w = nullptr;
    cudaError_t e = cudaMalloc(&w, 2 * half);
    if (e != cudaSuccess) { set_cuda_error(e); s = IDBF_ENOMEM; break; }
    b->ws.push_back(w);
    ods[o].L = p.L;
    ods[o].R = (int)nrhs[o];
    ods[o].level_base = (int)lvs.size();
    ods[o].pad = 0;
    ods[o].ws0 = w;
    ods[o].ws1 = (char*)w + half;
    for (int l = 0; l <= p.L; ++l) {
      const LevelInfo& li = p.lv[l];
      bat::OpLevel ol;
      ol.d = p.level(l);
      ol.mat = p.lmat[fmt][l];
      ol.gcap = std::max(std::max(li.max_cols, li.max_rows), li.max_in);
      ol.rcap = std::max(li.max_rows, li.max_cols);
      ol.max_in = li.max_in;
      ol.max_out = li.max_out;
      ol.max_rows = li.max_rows;
      ol.body = 1;
      lvs.push_back(ol);
    }
  }
  b->nlevels_total = (int)lvs.size();
  if (s == IDBF_OK) {
    cudaError_t e = cudaMalloc((void**)&b->d_ops, sizeof(bat::OpDesc) * nops);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_lv, sizeof(bat::OpLevel) * lvs.size());
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_ptrs, sizeof(void*) * 3 * nops);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_ops, ods.data(), sizeof(bat::OpDesc) * nops, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_lv, lvs.data(), sizeof(bat::OpLevel) * lvs.size(), cudaMemcpyHostToDevice);
    b->h_lv = lvs;
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) { set_cuda_error(e); s = e == cudaErrorMemoryAllocation ? IDBF_ENOMEM : IDBF_ECUDA; }
  }
  if (s == IDBF_OK) {
    // default tile: the largest preferred one whose shared memory fits
    static const int pref_df[] = {3, 2, 1, 0}, pref_other[] = {5, 4, 3, 1, 0};
    const int* pref = mode == IDBF_MODE_DF64 ? pref_df : pref_other;
    const int npref = mode == IDBF_MODE_DF64 ? 4 : 5;
    for (int k = 0; k < npref; ++k) {
      b->tile = pref[k];
      s = layout(b);
      if (s != IDBF_EUNSUPPORTED) break;
    }
  }
  if (s != IDBF_OK) {
    idbf_batch_destroy(b);
    return s;
  }
  *out = b;
  return IDBF_OK;
}

idbf_status idbf_batch_apply(idbf_batch b, const void* const* x, void* const* y, const int64_t* ld, void* stream) {
  if (!b || !x || !y || !ld) return IDBF_EINVAL;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != b->device) return IDBF_EINVAL;
  std::vector<void*> tab(3 * b->nops);
  for (int o = 0; o < b->nops; ++o) {
    if (!x[o] || !y[o] || ld[o] < b->plans[o]->p.N) return IDBF_EINVAL;
    tab[o] = (void*)x[o];
    tab[b->nops + o] = y[o];
    memcpy(&tab[2 * b->nops + o], &ld[o], sizeof(int64_t));
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (b->exec) {
    // pageable source: the copy is staged before the call returns, so tab may go out of scope
    IDBF_CUDA_TRY(cudaMemcpyAsync(b->d_ptrs, tab.data(), sizeof(void*) * tab.size(), cudaMemcpyHostToDevice, st));
    IDBF_CUDA_TRY(cudaGraphLaunch(b->exec, st));
  }
  // the operators above the split: their own per-level kernels, after the persistent launch
  for (int o = 0; o < b->nops; ++o) {
    if (!b->sep[o]) continue;
    const idbf_status s = idbf_apply(b->plans[o], x[o], y[o], b->R[o], ld[o], b->mode, stream);
    if (s != IDBF_OK) return s;
  }
  return IDBF_OK;
}

idbf_status idbf_batch_autotune(idbf_batch b, const void* const* x, void* const* y, const int64_t* ld, int32_t reps,
                                void* stream, float* best_ms) {
  if (!b || reps < 1) return IDBF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int btile = b->tile, bnpi = b->npi, bmix = b->mix_rows;
  int64_t bsplit = b->split_n;
  idbf_status s = IDBF_OK;
  // time the current layout (a warm-up launch, then reps launches); EUNSUPPORTED layouts are skipped
  auto trial = [&]() {
    idbf_status r = layout(b);
    if (r == IDBF_EUNSUPPORTED) return;
    if (r != IDBF_OK) { s = r; return; }
    if ((s = idbf_batch_apply(b, x, y, ld, stream)) != IDBF_OK) return;
    cudaEventRecord(e0, st);
    for (int k = 0; k < reps && s == IDBF_OK; ++k) s = idbf_batch_apply(b, x, y, ld, stream);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (s == IDBF_OK && ms < best) {
      best = ms;
      btile = b->tile;
      bnpi = b->npi;
      bmix = b->mix_rows;
      bsplit = b->split_n;
    }
  };
  // every tiling at the current split
  auto tilings = [&]() {
    const int npis[3] = {1, 2, 4};
    const int mixes[5] = {32, 64, 96, 128, 192};  // mixed tiling: row threshold of the per-thread body
    const int mix0 = bmix;
    for (int a = 0; a < bat::kNumTiles && s == IDBF_OK; ++a)
      for (int c = 0; c < 3 * 5 && s == IDBF_OK; ++c) {
        if (!tile_valid(b->mode, a)) continue;
        const bool mixed = bat::kTiles[a].tc < 0;
        if (!mixed && c >= 3) continue;
        b->tile = a;
        b->npi = npis[c % 3];
        b->mix_rows = mixed ? mixes[c / 3] : mix0;
        trial();
      }
  };
  if (b->split_auto) {
    b->split_n = INT64_MAX;
    bsplit = INT64_MAX;
  }
  tilings();
  // then, with the best tiling, every split: all operators in the persistent launch, or those of
  // N >= n for each N of the batch through their own per-level kernels; the tilings again if the
  // best split changed
  const int64_t split0 = bsplit;
  if (s == IDBF_OK && b->split_auto) {
    std::vector<int64_t> cand = {INT64_MAX};
    for (const idbf_plan pl : b->plans) cand.push_back(pl->p.N);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    for (const int64_t c : cand) {
      if (s != IDBF_OK) break;
      b->tile = btile;
      b->npi = bnpi;
      b->mix_rows = bmix;
      b->split_n = c;
      trial();
    }
  }
  if (s == IDBF_OK && bsplit != split0) {
    b->split_n = bsplit;
    tilings();
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tile = btile;
  b->npi = bnpi;
  b->mix_rows = bmix;
  b->split_n = bsplit;
  if (s == IDBF_OK) s = layout(b);
  if (best_ms) *best_ms = best;
  return s;
}

idbf_status idbf_batch_set_split(idbf_batch b, int64_t min_separate_n) {
  if (!b || min_separate_n < 0) return IDBF_EINVAL;
  if (min_separate_n == 0) {  // the autotuner chooses; until then every operator stays in the launch
    b->split_auto = true;
    if (b->split_n == INT64_MAX) return IDBF_OK;
    b->split_n = INT64_MAX;
    return layout(b);
  }
  const int64_t old = b->split_n;
  b->split_n = min_separate_n;
  idbf_status s = layout(b);
  if (s == IDBF_EUNSUPPORTED) {
    b->split_n = old;
    const idbf_status r = layout(b);
    return r == IDBF_OK ? s : r;
  }
  b->split_auto = false;
  return s;
}

idbf_status idbf_batch_split(idbf_batch b, int64_t* min_separate_n, int32_t* separate_ops) {
  if (!b) return IDBF_EINVAL;
  if (min_separate_n) *min_separate_n = b->split_n;
  if (separate_ops) {
    int32_t n = 0;
    for (const char c : b->sep) n += c ? 1 : 0;
    *separate_ops = n;
  }
  return IDBF_OK;
}

idbf_status idbf_batch_set_tiling(idbf_batch b, int32_t tile, int32_t nodes_per_item) {
  if (!b || tile < 0 || tile >= bat::kNumTiles) return IDBF_EINVAL;
  if (nodes_per_item != 1 && nodes_per_item != 2 && nodes_per_item != 4) return IDBF_EINVAL;
  if (!tile_valid(b->mode, tile)) return IDBF_EUNSUPPORTED;
  const int old_tile = b->tile, old_npi = b->npi;
  b->tile = tile;
  b->npi = nodes_per_item;
  idbf_status s = layout(b);
  if (s == IDBF_EUNSUPPORTED) {
    b->tile = old_tile;
    b->npi = old_npi;
    const idbf_status r = layout(b);
    return r == IDBF_OK ? s : r;
  }
  return s;
}

idbf_status idbf_batch_debug_set_wait(idbf_batch b, uint64_t limit_ns, int32_t extra_target) {
  if (!b || limit_ns == 0 || extra_target < 0) return IDBF_EINVAL;
  b->limit_ns = limit_ns;
  b->debug_extra = extra_target;
  return layout(b);  // the limit and the targets are captured in the graph
}

idbf_status idbf_batch_info(idbf_batch b, int32_t* rhs_per_item, int32_t* nodes_per_item, int32_t* items, int32_t* ctas) {
  if (!b) return IDBF_EINVAL;
  if (rhs_per_item) *rhs_per_item = b->rb;
  if (nodes_per_item) *nodes_per_item = b->npi;
  if (items) *items = b->nitems;
  if (ctas) *ctas = b->ctas;
  return IDBF_OK;
}

idbf_status idbf_batch_sync_status(idbf_batch b, void* stream) {
  if (!b) return IDBF_EINVAL;
  int v = 0;
  cudaStream_t st = (cudaStream_t)stream;
  IDBF_CUDA_TRY(cudaMemcpyAsync(&v, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  IDBF_CUDA_TRY(cudaStreamSynchronize(st));
  idbf_status res = IDBF_OK;
  if (v) {
    IDBF_CUDA_TRY(cudaMemset(b->d_status, 0, sizeof(int)));
    res = IDBF_ETIMEOUT;
  }
  // the operators applied through idbf_apply report their own bounded waits
  for (int o = 0; o < b->nops; ++o) {
    if (!b->sep[o]) continue;
    const idbf_status r = idbf_sync_status(b->plans[o], stream);
    if (r != IDBF_OK && res == IDBF_OK) res = r;
  }
  return res;
}

void idbf_batch_destroy(idbf_batch b) {
  if (!b) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != b->device) cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  free_layout(b);
  for (void* w : b->ws) cudaFree(w);
  if (b->d_ops) cudaFree(b->d_ops);
  if (b->d_lv) cudaFree(b->d_lv);
  if (b->d_ptrs) cudaFree(b->d_ptrs);
  if (b->d_status) cudaFree(b->d_status);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (cur != b->device) cudaSetDevice(cur);
  delete b;
}

}  // extern "C"
