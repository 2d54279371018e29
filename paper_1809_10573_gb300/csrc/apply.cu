// Apply of the IDBF, y = U^L ... U^h S^h V^h ... V^L x (Eq. 1 of the paper), and its adjoint.
//
// One launch per butterfly level. A node reads two vector segments, applies its two dense
// blocks and writes two segments (Secs. 2.3-2.4: the fractal 2 x 2 structure of every factor).
// The arithmetic policies (FP64, double-float, FP32) are in level_kernels.cuh.
// Forward levels: thread per output row, blocks column-major so that a warp's loads of one
// column are consecutive; adjoint levels: warp per output column (a contiguous run of the
// block) with a warp-shuffle reduction.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "idbf_internal.h"
#include "level_kernels.cuh"

namespace idbf {

template <class P, int RB, int RPT = 0>
__global__ void __launch_bounds__(512) k_level_fwd(DevLevel d, const typename P::mat_t* __restrict__ mat,
                                                   IO<typename P::vec_t> io, int gcap, int rcap, int max_in) {
  extern __shared__ __align__(16) unsigned char smem[];
  fwd_node<P, RB, RPT>(d, mat, io, gcap, rcap, max_in, (int64_t)blockIdx.x, (int)blockIdx.y * RB, smem);
}

// Several right-hand sides, FP32 / FP64 (fwd_node_tiled): node blockIdx.x, right-hand sides
// blockIdx.y * RB ...
template <class P>
__host__ __device__ constexpr bool tiled_ok() {
  return std::is_same<typename P::vec_t, typename P::gv_t>::value;
}
// The right-hand-side blocks of a node are adjacent CTAs (blockIdx.x = node * nblk + block), so
// that their reads of the node's factors meet in L2.
template <class P, int RB, int TC, int MINB>
__global__ void __launch_bounds__(256, MINB) k_level_fwd_tiled(DevLevel d, const typename P::mat_t* __restrict__ mat,
                                                         IO<typename P::vec_t> io, int max_rows, int max_in,
                                                         int max_out, int nblk) {
  extern __shared__ __align__(16) unsigned char smem[];
  if constexpr (tiled_ok<P>())
    fwd_node_tiled<P, RB, TC>(d, mat, io, max_rows, max_in, max_out, (int64_t)(blockIdx.x / nblk),
                              (int)(blockIdx.x % nblk) * RB, smem);
}

// Several right-hand sides, FP32 / FP64 adjoint (adj_node_tiled): node blockIdx.x / nblk,
// right-hand-side block blockIdx.x % nblk.
template <class P, int RB, int MINB>
__global__ void __launch_bounds__(256, MINB) k_level_adj_tiled(DevLevel d, const typename P::mat_t* __restrict__ mat,
                                                               IO<typename P::vec_t> io, int max_in, int max_out,
                                                               int max_rows, int max_cols, int nblk) {
  extern __shared__ __align__(16) unsigned char smem[];
  if constexpr (tiled_ok<P>())
    adj_node_tiled<P, RB>(d, mat, io, max_in, max_out, max_rows, max_cols, (int64_t)(blockIdx.x / nblk),
                          (int)(blockIdx.x % nblk) * RB, smem);
}

// ---------------------------------------------------------------------------------------------
// adjoint level kernel: reads the forward outputs of node j, writes its forward inputs.
// Shared memory: v[max_out][RB], g[2][gcap][RB], res[2][rcap][RB], ub[max_in][RB].
template <class P, int RB>
__global__ void __launch_bounds__(256) k_level_adj(DevLevel d, const typename P::mat_t* __restrict__ mat,
                                                   IO<typename P::vec_t> io, int gcap, int rcap, int max_out) {
  using V = typename P::vec_t;
  using G = typename P::gv_t;
  using M = typename P::mat_t;
  extern __shared__ __align__(16) unsigned char smem[];
  V* v = (V*)smem;
  G* g = (G*)(v + (size_t)max_out * RB);
  V* res = (V*)(g + (size_t)2 * gcap * RB);
  V* ub = res + (size_t)2 * rcap * RB;
  const int64_t j = blockIdx.x;
  const int r0 = blockIdx.y * RB;
  const int nrb = min(RB, io.R - r0);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

  // phase 1: adjoint inputs (forward outputs) -> v
  int o0len, o1len;
  if (d.lev == d.L) {
    o0len = leaf_len(d, j);
    o1len = 0;
    const int64_t x0 = leaf_start(d, j);
    for (int i = tid; i < o0len * RB; i += nt) {
      const int e = i / RB, rb = i % RB;
      v[i] = rb < nrb ? io.x[x0 + e + (int64_t)(r0 + rb) * io.ldx] : P::zero();
    }
  } else {
    const int64_t s0 = out_seg_id(d, j, 0), s1 = out_seg_id(d, j, 1);
    o0len = d.out_len[s0];
    o1len = d.out_len[s1];
    const int64_t b0 = d.out_off[s0], b1 = d.out_off[s1];
    for (int i = tid; i < (o0len + o1len) * RB; i += nt) {
      const int e = i / RB, rb = i % RB;
      const int64_t off = e < o0len ? b0 + e : b1 + (e - o0len);
      v[i] = rb < nrb ? io.win[off * io.R + r0 + rb] : P::zero();
    }
  }
  const int rows0 = d.rows[2 * j], rows1 = d.rows[2 * j + 1];
  const int cols0 = d.cols[2 * j], cols1 = d.cols[2 * j + 1];
  const int64_t mo0 = d.moff[2 * j], mo1 = d.moff[2 * j + 1];
  const int32_t* ix0 = d.idx + d.ioff[2 * j];
  const int32_t* ix1 = d.idx + d.ioff[2 * j + 1];
  __syncthreads();

  // phase 2: operands of the conjugate-transposed products (indexed by block row r)
  if (d.kind == KIND_U) {  // g_c[r] = v[p_c[r]]
    for (int i = tid; i < rows0 * RB; i += nt) g[i] = P::cvt(v[ix0[cols0 + i / RB] * RB + i % RB]);
    for (int i = tid; i < rows1 * RB; i += nt) g[gcap * RB + i] = P::cvt(v[ix1[cols1 + i / RB] * RB + i % RB]);
  } else {  // g_c = v_c (the c-th forward output)
    for (int i = tid; i < rows0 * RB; i += nt) g[i] = P::cvt(v[i]);
    for (int i = tid; i < rows1 * RB; i += nt) g[gcap * RB + i] = P::cvt(v[o0len * RB + i]);
  }
  __syncthreads();

  // phase 3: res_c[i] = sum_r conj(M_c(r, i)) g_c[r]; a warp per column i (contiguous in r)
  const int items = d.kind == KIND_S ? cols0 : cols0 + cols1;
  for (int it = warp; it < items; it += nw) {
    typename P::acc_t acc[RB];
#pragma unroll
    for (int rb = 0; rb < RB; ++rb) P::init(acc[rb]);
    const int cfirst = d.kind == KIND_S ? 0 : (it >= cols0);
    const int clast = d.kind == KIND_S ? 1 : cfirst;
    const int i = (d.kind != KIND_S && cfirst) ? it - cols0 : it;
    for (int c = cfirst; c <= clast; ++c) {
      const int rows = c ? rows1 : rows0;
      const M* col = mat + (c ? mo1 : mo0) + (int64_t)i * rows;
      const G* gc = g + c * gcap * RB;
      int cnt = 0;
      for (int r = lane; r < rows; r += 32) {
        const M mv = P::ld(col + r);
#pragma unroll
        for (int rb = 0; rb < RB; ++rb) P::macc(acc[rb], mv, gc[r * RB + rb]);
        if (++cnt == P::CHUNK) {
#pragma unroll
          for (int rb = 0; rb < RB; ++rb) P::flush(acc[rb]);
          cnt = 0;
        }
      }
    }
#pragma unroll
    for (int rb = 0; rb < RB; ++rb) {
      P::warp_sum(acc[rb]);
      if (lane == 0) res[(cfirst * rcap + i) * RB + rb] = P::fin(acc[rb]);
    }
  }
  __syncthreads();

  // phase 4: combine and write the forward inputs
  int nin;
  if (d.kind == KIND_U) {
    // out_c[i] = v[q_c[i]] + res_c[i]  ->  forward input segment c
    for (int c = 0; c < 2; ++c) {
      const int cols = c ? cols1 : cols0;
      const int32_t* q = c ? ix1 : ix0;
      const int64_t ob = d.in_off[2 * j + c];
      for (int k = tid; k < cols * nrb; k += nt) {
        const int i = k / nrb, rb = k % nrb;
        io.wout[(ob + i) * io.R + r0 + rb] = P::add(v[q[i] * RB + rb], res[(c * rcap + i) * RB + rb]);
      }
    }
    return;
  }
  if (d.kind == KIND_S) {
    nin = cols0;
    for (int k = tid; k < nin * RB; k += nt) ub[k] = res[k];
  } else {
    nin = rows0 + cols0;
    for (int k = tid; k < nin * RB; k += nt) ub[k] = P::zero();
    __syncthreads();
    for (int k = tid; k < rows0 * RB; k += nt) { V* dst = &ub[ix0[k / RB] * RB + k % RB]; *dst = P::add(*dst, v[k]); }
    __syncthreads();
    for (int k = tid; k < rows1 * RB; k += nt) { V* dst = &ub[ix1[k / RB] * RB + k % RB]; *dst = P::add(*dst, v[o0len * RB + k]); }
    __syncthreads();
    for (int k = tid; k < cols0 * RB; k += nt) { V* dst = &ub[ix0[rows0 + k / RB] * RB + k % RB]; *dst = P::add(*dst, res[k]); }
    __syncthreads();
    for (int k = tid; k < cols1 * RB; k += nt) { V* dst = &ub[ix1[rows1 + k / RB] * RB + k % RB]; *dst = P::add(*dst, res[rcap * RB + k]); }
  }
  __syncthreads();
  if (d.lev == 0) {
    const int64_t y0 = leaf_start(d, j);
    for (int k = tid; k < nin * nrb; k += nt) {
      const int e = k / nrb, rb = k % nrb;
      io.y[y0 + e + (int64_t)(r0 + rb) * io.ldy] = ub[e * RB + rb];
    }
  } else {
    const int len0 = d.in_len[2 * j];
    const int64_t b0 = d.in_off[2 * j], b1 = d.in_off[2 * j + 1];
    for (int k = tid; k < nin * nrb; k += nt) {
      const int e = k / nrb, rb = k % nrb;
      const int64_t off = e < len0 ? b0 + e : b1 + (e - len0);
      io.wout[off * io.R + r0 + rb] = ub[e * RB + rb];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Streaming forward level kernel (one right-hand side). Persistent CTAs (one to four per SM,
// by ring layout), each a producer warp and TEAMS consumer teams of TCW warps. The producer
// copies every block of its nodes, a few whole columns at a time, with cp.async.bulk into a
// ring of STAGES shared-memory stages (mbarrier full / empty pairs), and each node's inputs,
// index lists and description into double buffers; the consumers, one output row per thread
// (or per thread group, with the column split), multiply the staged columns with the gathered
// input held in shared memory. Each block is read from HBM once, in large contiguous pieces,
// while the arithmetic runs from shared memory.
// Every wait is bounded (globaltimer): on a timeout the CTA sets bit 0 of *status, lets its
// copies in flight land, and leaves; the host reads the status with idbf_sync_status.
namespace strm {
constexpr int TCW = 6;                   // warps per consumer team
constexpr int TCT = TCW * 32;            // threads per team (one output row each)
constexpr int MAX_RPT = 2;               // output rows per team thread: rows <= MAX_RPT * TCT
constexpr int FLUSH_TERMS = 16;          // double-float partial sums are folded after >= 16 terms
// A block with rows <= TCT / 2 would leave most of a team idle: its columns are then split
// between up to MAX_GROUPS groups of `rows` threads (group g takes columns g, g + G, ... of every
// chunk), and the groups' partial sums are folded in the epilogue.
constexpr int MAX_GROUPS = 4;
// Ring of stages and team layout per arithmetic. Chunk i (counted over the whole launch) goes to
// stage i % STAGES and to team i % TEAMS, so with STAGES a multiple of TEAMS every stage is read
// by one team only, and a team never waits for a phase of a stage more than one phase ahead of
// the last one it consumed there (an mbarrier parity wait cannot tell phase k from k + 2).
// The autotuner picks the layout per level; on the FIO at N = 2^20 RingA takes the levels of
// tall blocks and RingD most levels of short blocks, in double-float and in FP32 alike.
struct RingA {  // two CTAs per SM, two teams each
  static constexpr int TEAMS = 2, STAGES = 4, STAGE_BYTES = 18 * 1024, CTAS = 2;
  static constexpr int NCT = TEAMS * TCT, NTHREADS = NCT + 32;
};
struct RingB {  // two CTAs per SM, one team each, fewer and larger stages
  static constexpr int TEAMS = 1, STAGES = 3, STAGE_BYTES = 24 * 1024, CTAS = 2;
  static constexpr int NCT = TEAMS * TCT, NTHREADS = NCT + 32;
};
struct RingC {  // one CTA per SM, four teams, eight stages
  static constexpr int TEAMS = 4, STAGES = 8, STAGE_BYTES = 22 * 1024, CTAS = 1;
  static constexpr int NCT = TEAMS * TCT, NTHREADS = NCT + 32;
};
struct RingD {  // four CTAs per SM, one team each, small stages: levels of short blocks
  static constexpr int TEAMS = 1, STAGES = 3, STAGE_BYTES = 12 * 1024, CTAS = 4;
  static constexpr int NCT = TEAMS * TCT, NTHREADS = NCT + 32;
};
static_assert(RingA::STAGES % RingA::TEAMS == 0 && RingB::STAGES % RingB::TEAMS == 0 &&
                  RingC::STAGES % RingC::TEAMS == 0 && RingD::STAGES % RingD::TEAMS == 0,
              "every stage must belong to one team");

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(tx) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(sa(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sa(dst)),
               "l"(src), "r"(bytes), "r"(sa(bar))
               : "memory");
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
template <int NCT>
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NCT) : "memory"); }

// Wait until phase `parity` of barrier b has completed, giving up after limit_ns or when
// another warp has flagged an abort. The timer and the flag are read every 256 polls only, so
// that a waiting warp takes few issue slots from the warps that compute.
__device__ __forceinline__ bool wait_bounded(uint64_t* b, uint32_t parity, uint64_t limit_ns, volatile int* abort_flag) {
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t n = 1;; ++n) {
    if (mbar_try_wait(b, parity)) return true;
    if ((n & 255) == 0 && (*abort_flag || gtimer() - t0 > limit_ns)) return false;
  }
}

// columns per chunk for a block with `rows` rows and elements of es bytes; 8-byte elements may
// start 8 bytes past a 16-byte boundary, which costs up to two elements of slack
__host__ __device__ __forceinline__ int cols_per_chunk(int rows, int es, int stage_bytes) {
  const int cap = stage_bytes / es - (es == 8 ? 2 : 0);
  return max(1, cap / max(rows, 1));
}

// A node's description: input segment (offset, lengths), index-list and block offsets, block
// shapes, and where the outputs go. The producer loads it one node ahead and publishes it in
// shared memory before its arrival on the node's input barrier, so that the consumers start a
// node without a global-memory round trip.
struct NodeMeta {
  int64_t in0, io[2], mo[2], ob[2];
  int64_t j;  // node index on its level
  int l0, l1, rows[2], cols[2], olen0;
  int sel;    // level pairs: 0 = the first level (outputs to shared memory), 1 = the second
};

struct Geo {
  size_t vec_off, ibuf_off, g_off, t_off, red_off, mid_off, bar_off, total;
  int ucap, icap;  // elements of one input buffer, ints of one index buffer
};
// Shared memory: the stage ring, two input buffers (node inputs, copied by the producer), two
// index buffers (q and p lists of both blocks), the gathered operands, the row-ID accumulator t,
// the reduction buffer and the mbarriers. The reduction buffer holds one partial sum per thread of
// teams 1.. (and, with the column split, of team 0 too).
template <class P, class RG>
__host__ __device__ inline Geo geometry(int max_in, int max_out, int max_cols_pair, int rpt, int split,
                                        int mid_elems = 0) {
  using V = typename P::vec_t;
  using G = typename P::gv_t;
  constexpr int STAGES = RG::STAGES, STAGE_BYTES = RG::STAGE_BYTES;
  Geo q;
  // capacities rounded to 16 bytes so that buffer 1 starts 16-byte aligned (bulk-copy destination);
  // + room for a start shifted within 16 bytes and a length rounded up to 16 bytes
  q.ucap = (max_in + 16 / (int)sizeof(V) + 1 + 3) & ~3;
  q.icap = (2 * (max_in > max_out ? max_in : max_out) + 16 + 3) & ~3;
  const int gsz = max_cols_pair > max_in ? max_cols_pair : max_in;
  q.vec_off = (size_t)STAGES * STAGE_BYTES;
  q.ibuf_off = q.vec_off + ((2 * (size_t)q.ucap * sizeof(V) + 127) & ~(size_t)127);
  q.g_off = q.ibuf_off + ((2 * (size_t)q.icap * sizeof(int32_t) + 127) & ~(size_t)127);
  q.t_off = q.g_off + (((size_t)gsz * sizeof(G) + 127) & ~(size_t)127);
  q.red_off = q.t_off + (((size_t)max_out * sizeof(V) + 127) & ~(size_t)127);
  const int slots = split ? RG::TEAMS : (RG::TEAMS > 1 ? RG::TEAMS - 1 : 1);
  q.mid_off = q.red_off + (((size_t)slots * rpt * TCT * sizeof(typename P::part_t) + 127) & ~(size_t)127);
  q.bar_off = q.mid_off + (((size_t)mid_elems * sizeof(V) + 127) & ~(size_t)127);
  q.total = q.bar_off + 4 * STAGES * sizeof(uint64_t);
  return q;
}
}  // namespace strm

// PAIR: the launch runs two consecutive levels l (d, mat) and l + 1 (d1, mat1) as a radix-2
// fusion (the closed groups of Eq. expressUSV, as in an FFT): work unit u is the group of level-l
// nodes j0 = aH + r and j0 + 1 (H = 2^(L-l), r = 2 (u mod H/2), a = u div H/2), whose four
// output segments are exactly the inputs of level-(l+1) nodes aH + r/2 and aH + r/2 + H/2. The
// four segments stay in shared memory (mid): level l writes them there, level l + 1 reads them
// there; boundary l never reaches global memory. Without PAIR a unit is one node of level l.
template <class P, class RG, int RPT, bool SPLIT, bool PAIR>
__global__ void __launch_bounds__(RG::NTHREADS, RG::CTAS)
    k_level_stream(DevLevel d, const typename P::mat_t* __restrict__ mat, DevLevel d1,
                   const typename P::mat_t* __restrict__ mat1, IO<typename P::vec_t> io, int max_in, int max_out,
                   int max_cols_pair, int mid_elems, int x_bulk, int* __restrict__ status, uint64_t limit_ns,
                   int producer_enabled) {
  using namespace strm;
  using V = typename P::vec_t;
  using G = typename P::gv_t;
  using M = typename P::mat_t;
  // vectors between levels: the double-float policy keeps them in its own format (Bnd)
  using BP = Bnd<P, std::is_same<P, DF64P>::value>;
  using B = typename BP::b_t;
  constexpr int ES = (int)sizeof(M);
  constexpr int VS = (int)sizeof(V);
  constexpr int STAGES = RG::STAGES, STAGE_BYTES = RG::STAGE_BYTES;
  constexpr int TEAMS = RG::TEAMS, NCT = RG::NCT;
  constexpr int NSUB = PAIR ? 4 : 1;  // nodes per work unit
  extern __shared__ __align__(128) unsigned char smem[];
  static_assert(RPT == 1 || !SPLIT, "the column split is for one output row per thread");
  const Geo geo = geometry<P, RG>(max_in, max_out, max_cols_pair, RPT, SPLIT, PAIR ? mid_elems : 0);
  unsigned char* stages = smem;
  V* ubuf = (V*)(smem + geo.vec_off);              // [2][ucap]
  int32_t* ibuf = (int32_t*)(smem + geo.ibuf_off);  // [2][icap]
  G* g = (G*)(smem + geo.g_off);
  V* t = (V*)(smem + geo.t_off);
  B* tb = (B*)t;  // row-ID accumulator (U levels), in the boundary format
  typename P::part_t* red = (typename P::part_t*)(smem + geo.red_off);
  V* mid = (V*)(smem + geo.mid_off);                // level pairs: the four shared segments
  uint64_t* full = (uint64_t*)(smem + geo.bar_off);
  uint64_t* empty = full + STAGES;
  uint64_t* in_full = empty + STAGES;   // [2]
  uint64_t* in_empty = in_full + 2;     // [2]
  // abort_flag: any warp, only shortens waits. cons_abort: written by consumers before a
  // consumer barrier and read after it, so that all consumer warps leave the loop together.
  __shared__ int abort_flag;
  __shared__ int cons_abort;
  __shared__ NodeMeta nmeta[2];  // description of the node in input buffer b
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nunits = PAIR ? d.m / 2 : d.m;
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], strm::TCW);  // a stage is consumed by the warps of one team
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&in_full[i], 1);
      mbar_init(&in_empty[i], 1);
    }
    abort_flag = 0;
    cons_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool inputs_bulk = x_bulk != 0;  // producer copies node inputs (else consumers load them)

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane != 0) return;
    uint32_t it = 0, nn = 0;
    bool ok = true;
    // node description of node jj on level dl; outputs to global memory
    auto meta_of = [&](const DevLevel& dl, int64_t jj) {
      NodeMeta m;
      m.j = jj;
      m.sel = 0;
      m.in0 = dl.lev == 0 ? leaf_start(dl, jj) : dl.in_off[2 * jj];  // level 0: the leaf's first row of x
      m.l0 = dl.lev == 0 ? leaf_len(dl, jj) : dl.in_len[2 * jj];
      m.l1 = dl.lev == 0 ? 0 : dl.in_len[2 * jj + 1];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        m.io[c] = dl.ioff[2 * jj + c];
        m.mo[c] = dl.moff[2 * jj + c];
        m.rows[c] = dl.rows[2 * jj + c];
        m.cols[c] = dl.cols[2 * jj + c];
      }
      m.ob[0] = m.ob[1] = 0;
      m.olen0 = 0;
      if (dl.lev < dl.L) {
        const int64_t s0 = out_seg_id(dl, jj, 0), s1 = out_seg_id(dl, jj, 1);
        m.ob[0] = dl.out_off[s0];
        m.ob[1] = dl.out_off[s1];
        m.olen0 = dl.out_len[s0];
      }
      return m;
    };
    // node v of work unit un (node descriptions are loaded one node ahead, so that no copy
    // waits for them); for level pairs the shared-memory offsets replace the segment offsets
    auto meta = [&](int64_t un, int v) {
      if (!PAIR) return meta_of(d, un);
      const int64_t hh = (int64_t)d.H >> 1, a = un / hh, r = 2 * (un % hh);
      const int64_t sA = a * 2 * d.H + r, sB = sA + d.H;  // segments of level l written by j0, j0 + 1
      const int lA0 = d.out_len[sA], lA1 = d.out_len[sA + 1], lB0 = d.out_len[sB];
      NodeMeta m;
      if (v < 2) {
        m = meta_of(d, a * d.H + r + v);
        m.ob[0] = v == 0 ? 0 : lA0;
        m.ob[1] = v == 0 ? lA0 + lA1 : lA0 + lA1 + lB0;
      } else {
        m = meta_of(d1, a * d.H + (r >> 1) + (v - 2) * hh);
        m.in0 = v == 2 ? 0 : lA0 + lA1;
        m.sel = 1;
      }
      return m;
    };
    int64_t un = blockIdx.x;
    int v = 0;
    NodeMeta nxt = meta(un < nunits ? un : 0, 0);
    for (; un < nunits && ok; ++nn) {
      const NodeMeta cur = nxt;
      const bool second = PAIR && cur.sel;
      const DevLevel& dl = second ? d1 : d;
      const typename P::mat_t* ml = second ? mat1 : mat;
      // the next node: the next of this unit, else the first of the next unit
      if (v + 1 < NSUB) ++v;
      else { v = 0; un += gridDim.x; }
      if (un < nunits) nxt = meta(un, v);
      // node inputs and index lists into buffer nn & 1 (released by the consumers of node nn-2)
      const int b = nn & 1;
      if (!wait_bounded(&in_empty[b], ((nn >> 1) & 1) ^ 1, limit_ns, &abort_flag)) { ok = false; break; }
      const unsigned char* usrc = nullptr;
      uint32_t ubytes = 0;
      if (second) {
        // inputs already in shared memory (mid)
      } else if (dl.lev == 0) {
        usrc = (const unsigned char*)(io.x + cur.in0);
        ubytes = inputs_bulk ? (uint32_t)(cur.l0 * VS) : 0;
      } else {
        usrc = (const unsigned char*)(io.win + cur.in0);
        ubytes = inputs_bulk ? (uint32_t)((cur.l0 + cur.l1) * VS) : 0;
      }
      const unsigned char* ua = (const unsigned char*)((uintptr_t)usrc & ~(uintptr_t)15);
      const uint32_t ucopy = ubytes ? (uint32_t)((((uintptr_t)usrc + ubytes + 15) & ~(uintptr_t)15) - (uintptr_t)ua) : 0;
      uint32_t icopy[2] = {0, 0};
      const unsigned char* ia[2] = {nullptr, nullptr};
      if (dl.kind != KIND_S && inputs_bulk) {
        for (int c = 0; c < 2; ++c) {
          const unsigned char* is = (const unsigned char*)(dl.idx + cur.io[c]);
          const uint32_t ib = (uint32_t)((cur.rows[c] + cur.cols[c]) * 4);
          ia[c] = (const unsigned char*)((uintptr_t)is & ~(uintptr_t)15);
          icopy[c] = (uint32_t)((((uintptr_t)is + ib + 15) & ~(uintptr_t)15) - (uintptr_t)ia[c]);
        }
      }
      nmeta[b] = cur;  // visible to the consumers through the release of the arrival below
      if (producer_enabled) {
        mbar_expect_tx(&in_full[b], ucopy + icopy[0] + icopy[1]);
        if (ucopy) bulk_g2s(ubuf + (size_t)b * geo.ucap, ua, ucopy, &in_full[b]);
        int32_t* ib0 = ibuf + (size_t)b * geo.icap;
        if (icopy[0]) bulk_g2s(ib0, ia[0], icopy[0], &in_full[b]);
        if (icopy[1]) bulk_g2s(ib0 + ((icopy[0] / 4 + 3) & ~3), ia[1], icopy[1], &in_full[b]);
      }
      // the blocks, a few whole columns per stage
      for (int c = 0; c < 2 && ok; ++c) {
        const int rows = cur.rows[c], cols = cur.cols[c];
        if (rows == 0 || cols == 0) continue;
        const int cpc = cols_per_chunk(rows, ES, STAGE_BYTES);
        const unsigned char* base = (const unsigned char*)(ml + cur.mo[c]);
        for (int j0 = 0; j0 < cols; j0 += cpc, ++it) {
          const int nc = min(cpc, cols - j0);
          const int stg = it % STAGES;
          const uint32_t use = it / STAGES;
          if (!wait_bounded(&empty[stg], (use & 1) ^ 1, limit_ns, &abort_flag)) { ok = false; break; }
          const unsigned char* src = base + (size_t)j0 * rows * ES;
          const unsigned char* src_al = (const unsigned char*)((uintptr_t)src & ~(uintptr_t)15);
          const unsigned char* end = src + (size_t)nc * rows * ES;
          const uint32_t bytes = (uint32_t)((((uintptr_t)end + 15) & ~(uintptr_t)15) - (uintptr_t)src_al);
          if (producer_enabled) {
            mbar_expect_tx(&full[stg], bytes);
            bulk_g2s(stages + (size_t)stg * STAGE_BYTES, src_al, bytes, &full[stg]);
          }
        }
      }
    }
    if (!ok) {
      atomicOr(status, 1);
      abort_flag = 1;
      // let the copies already issued land before the CTA's shared memory goes away
      const uint64_t t0 = gtimer();
      for (uint32_t k = it > STAGES ? it - STAGES : 0; k < it; ++k)
        while (!mbar_try_wait(&full[k % STAGES], (k / STAGES) & 1) && gtimer() - t0 < limit_ns) {
        }
      for (uint32_t k = nn > 2 ? nn - 2 : 0; k <= nn; ++k)
        while (!mbar_try_wait(&in_full[k & 1], (k >> 1) & 1) && gtimer() - t0 < limit_ns) {
        }
    }
    return;
  }

  // ---------------- consumers ----------------
  const int tc = threadIdx.x - 32;      // 0 .. NCT-1: prologue / epilogue index
  const int team = tc / TCT;
  const int tr = tc - team * TCT;       // row index within the team
  uint32_t it = 0, nn = 0;
  bool failed = false;
  for (int64_t un = blockIdx.x; un < nunits; un += gridDim.x) {
  for (int sub = 0; sub < NSUB; ++sub, ++nn) {
    consumer_sync<NCT>();
    if (*(volatile int*)&cons_abort) break;
    const int b = nn & 1;
    if (!failed && !wait_bounded(&in_full[b], (nn >> 1) & 1, limit_ns, &abort_flag)) failed = true;
    // the node's description from the producer (acquired by the wait above); after a failed wait
    // it may be incomplete, so every size is zero and the loops below do nothing
    const NodeMeta& nm = nmeta[b];
    const bool second = PAIR && sub >= 2;   // level l + 1 of a pair: inputs from mid
    const bool to_mid = PAIR && sub < 2;    // level l of a pair: outputs to mid
    const int kind = second ? d1.kind : d.kind;
    const int lev = second ? d1.lev : d.lev;
    const int Lv = d.L;
    const int32_t* lidx = second ? d1.idx : d.idx;
    const int64_t j = nm.j;
    const int l0 = failed ? 0 : nm.l0, l1 = failed ? 0 : nm.l1;
    const int rows0 = failed ? 0 : nm.rows[0], rows1 = failed ? 0 : nm.rows[1];
    const int cols0 = failed ? 0 : nm.cols[0], cols1 = failed ? 0 : nm.cols[1];
    const int64_t obv[2] = {nm.ob[0], nm.ob[1]};
    const int olen0 = failed ? 0 : nm.olen0;
    const int64_t in0 = nm.in0;
    const int64_t iov[2] = {kind != KIND_S ? nm.io[0] : 0, kind != KIND_S ? nm.io[1] : 0};
    const int64_t mov[2] = {nm.mo[0], nm.mo[1]};
    const M* ml = second ? mat1 : mat;
    V* const outp = to_mid ? mid : io.wout;  // where this node's output segments go
    B* const outb = (B*)outp;
    // inputs (shifted within 16 bytes of the copy) and index lists in shared memory
    const V* u;
    if (second) {
      u = mid + in0;
    } else {
      const uintptr_t usrc = lev == 0 ? (uintptr_t)(io.x + in0) : (uintptr_t)(io.win + in0);
      u = ubuf + (size_t)b * geo.ucap + (int)((usrc & 15) / VS);
      if (!inputs_bulk) {  // plain loads by the consumers
        V* uw = ubuf + (size_t)b * geo.ucap;
        if (lev == 0) {
          for (int i = tc; i < l0; i += NCT) uw[i] = io.x[in0 + i];
        } else {
          const B* src = (const B*)(io.win + in0);
          for (int i = tc; i < l0 + l1; i += NCT) ((B*)uw)[i] = src[i];
        }
        u = uw;
      }
    }
    const B* ub = (const B*)u;  // the inputs of a level > 0 (and of the second level of a pair)
    // gathered operand and pass-through term of input element e: level 0 converts x, later
    // levels read the boundary format
    auto gin = [&](int e) -> G { return lev == 0 ? P::cvt(u[e]) : BP::g_of(ub[e]); };
    auto bin = [&](int e) -> B { return lev == 0 ? BP::of_v(u[e]) : ub[e]; };
    const int32_t* ix0 = nullptr;
    const int32_t* ix1 = nullptr;
    if (kind != KIND_S) {
      int32_t* ib0 = ibuf + (size_t)b * geo.icap;
      if (inputs_bulk) {
        const uintptr_t s0 = (uintptr_t)(lidx + iov[0]), s1 = (uintptr_t)(lidx + iov[1]);
        const uint32_t c0 = (uint32_t)((((s0 + (rows0 + cols0) * 4 + 15) & ~(uintptr_t)15)) - (s0 & ~(uintptr_t)15));
        ix0 = ib0 + (int)((s0 & 15) / 4);
        ix1 = ib0 + ((c0 / 4 + 3) & ~3) + (int)((s1 & 15) / 4);
      } else {
        const int32_t* g0 = lidx + iov[0];
        const int32_t* g1 = lidx + iov[1];
        for (int i = tc; i < rows0 + cols0; i += NCT) ib0[i] = g0[i];
        for (int i = tc; i < rows1 + cols1; i += NCT) ib0[rows0 + cols0 + i] = g1[i];
        ix0 = ib0;
        ix1 = ib0 + rows0 + cols0;
      }
    }
    consumer_sync<NCT>();
    // gathered operands: V: g = [u[p_0], u[p_1]]; S and U: g = u
    if (!failed) {
      if (kind == KIND_V) {
        for (int i = tc; i < cols0; i += NCT) g[i] = gin(ix0[rows0 + i]);
        for (int i = tc; i < cols1; i += NCT) g[cols0 + i] = gin(ix1[rows1 + i]);
      } else {
        for (int i = tc; i < l0 + l1; i += NCT) g[i] = gin(i);
      }
      if (kind == KIND_U)  // t[q_0] = in_0; t[p_0] comes from the block-0 products
        for (int i = tc; i < l0; i += NCT) tb[ix0[i]] = bin(i);
    }
    consumer_sync<NCT>();
    const int tl = l0 + rows0;  // row-ID levels: |t| = |q_0| + |p_0|
    for (int c = 0; c < 2; ++c) {
      const int rows = c ? rows1 : rows0, cols = c ? cols1 : cols0;
      const int32_t* ix = c ? ix1 : ix0;
      const G* gc = g + (kind == KIND_S ? 0 : (kind == KIND_V ? c * cols0 : c * l0));
      if (kind == KIND_U && c == 1 && !failed) {  // block 0 has written all of t
        for (int i = tc; i < l1; i += NCT) { B* q = &tb[ix1[i]]; *q = BP::add(*q, bin(l0 + i)); }
      }
      typename P::acc_t acc[RPT];
#pragma unroll
      for (int k = 0; k < RPT; ++k) P::init(acc[k]);
      const bool work = rows > 0 && cols > 0;
      // column split of short blocks: this thread takes row rr of the block in column group grp
      const int ngrp = (SPLIT && rows > 0) ? min(MAX_GROUPS, max(1, TCT / rows)) : 1;
      const int grp = ngrp > 1 ? tr / rows : 0;
      const int rr = tr - grp * rows;
      if (work) {
        const int cpc = cols_per_chunk(rows, ES, STAGE_BYTES);
        const uintptr_t base = (uintptr_t)(ml + mov[c]);
        const uint32_t chunk_bytes = (uint32_t)cpc * rows * ES;
        int since = 0;
        uintptr_t src = base;
        for (int j0 = 0; j0 < cols; j0 += cpc, ++it, src += chunk_bytes) {
          if ((int)(it % TEAMS) != team) continue;  // the other team's chunk (stage it % STAGES)
          const int nc = min(cpc, cols - j0);
          const int stg = it % STAGES;
          if (!failed && !wait_bounded(&full[stg], (it / STAGES) & 1, limit_ns, &abort_flag)) failed = true;
          if (!failed) {
            const int shift = ES == 16 ? 0 : (int)((src & 15) / ES);  // 16-byte entries are never shifted
            const M* st = (const M*)(stages + (size_t)stg * STAGE_BYTES) + shift + tr;
            if (RPT == 1) {
              if (ngrp > 1) {
                if (grp < ngrp) {
                  const M* sg = st - tr + rr;
#pragma unroll 4
                  for (int jj = grp; jj < nc; jj += ngrp) P::mac(acc[0], sg[jj * rows], gc[j0 + jj]);
                }
              } else if (tr < rows) {
#pragma unroll 4
                for (int jj = 0; jj < nc; ++jj) P::mac(acc[0], st[jj * rows], gc[j0 + jj]);
              }
            } else {
#pragma unroll 2
              for (int jj = 0; jj < nc; ++jj) {
                const G gv = gc[j0 + jj];
#pragma unroll
                for (int k = 0; k < RPT; ++k)
                  if (tr + k * TCT < rows) P::mac(acc[k], st[jj * rows + k * TCT], gv);
              }
            }
            since += nc;
            if (since >= FLUSH_TERMS) {
#pragma unroll
              for (int k = 0; k < RPT; ++k) P::flush(acc[k]);
              since = 0;
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[stg]);
        }
#pragma unroll
        for (int k = 0; k < RPT; ++k) P::flush(acc[k]);
        // teams 1.. hand their partial sums to team 0; with the column split, team 0's groups
        // 1.. too (slot team * TCT + tr; without it, slot (team - 1) * RPT * TCT + tr)
        if (ngrp > 1) {
          if ((team > 0 || grp > 0) && grp < ngrp) red[team * TCT + tr] = P::part(acc[0]);
        } else if (team > 0) {
          const int slot = SPLIT ? team : team - 1;
#pragma unroll
          for (int k = 0; k < RPT; ++k)
            if (tr + k * TCT < rows) red[(slot * RPT + k) * TCT + tr] = P::part(acc[k]);
        }
      }
      consumer_sync<NCT>();
      // no early exit here: every consumer warp must reach the barriers of this block
      const int64_t ob = obv[c];
      if (work && team == 0 && !failed) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          const int r = tr + k * TCT;
          if (r >= rows) continue;
          if (ngrp > 1) {
            for (int tm = 0; tm < TEAMS; ++tm)
              for (int gq = tm == 0 ? 1 : 0; gq < ngrp; ++gq) P::combine(acc[0], red[tm * TCT + gq * rows + tr]);
          } else {
            for (int tm = 1; tm < TEAMS; ++tm)
              P::combine(acc[k], red[((SPLIT ? tm : tm - 1) * RPT + k) * TCT + tr]);
          }
          const B v = BP::of_acc(acc[k]);
          if (kind == KIND_U) {
            B* q = &tb[ix[(c ? l1 : l0) + r]];
            *q = c ? BP::add(*q, v) : v;
          } else {
            outb[ob + r] = kind == KIND_V ? BP::add(v, bin(ix[r])) : v;
          }
        }
      }
      if (kind == KIND_V && cols == 0 && !failed) {  // all skeleton: out = u[q]
        for (int r = tc; r < rows; r += NCT) outb[ob + r] = bin(ix[r]);
      }
      // a block with rows but no columns (an empty node of a coordinate-based tree) multiplies
      // nothing: its product is zero (row IDs: block 0 sets t[p_0], block 1 adds nothing)
      if (rows > 0 && cols == 0 && !failed) {
        if (kind == KIND_S)
          for (int r = tc; r < rows; r += NCT) outb[ob + r] = BP::zero();
        else if (kind == KIND_U && c == 0)
          for (int r = tc; r < rows; r += NCT) tb[ix[l0 + r]] = BP::zero();
      }
      consumer_sync<NCT>();  // red is reused by the next block; t must be complete before c = 1
    }
    // the node's inputs and index lists are no longer read: release the buffer
    if (tc == 0) mbar_arrive(&in_empty[b]);
    if (failed) {
      atomicOr(status, 1);
      abort_flag = 1;
      cons_abort = 1;
    }
    if (kind == KIND_U) {
      consumer_sync<NCT>();
      if (*(volatile int*)&cons_abort) break;
      if (lev == Lv) {
        const int64_t y0 = second ? leaf_start(d1, j) : leaf_start(d, j);
        for (int i = tc; i < tl; i += NCT) io.y[y0 + i] = BP::v_of(tb[i]);
      } else {
        for (int i = tc; i < tl; i += NCT) outb[i < olen0 ? obv[0] + i : obv[1] + (i - olen0)] = tb[i];
      }
    }
  }
  if (*(volatile int*)&cons_abort) break;
  }
}

// ---------------------------------------------------------------------------------------------
// Warp-per-node forward level kernel (one right-hand side, short blocks): warp w of the grid
// takes nodes w, w + W, ... (fwd_node_warp in level_kernels.cuh).
constexpr int kWarpNodeWarps = 8;  // warps per CTA
template <class P, int RPL>
__global__ void __launch_bounds__(kWarpNodeWarps * 32) k_level_warp(DevLevel d, const typename P::mat_t* __restrict__ mat,
                                                                   IO<typename P::vec_t> io, int max_in, int gcap,
                                                                   int max_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int w = threadIdx.x >> 5;
  unsigned char* wsm = smem + (size_t)w * warp_node_smem<P>(max_in, gcap, max_out);
  const int64_t nw = (int64_t)gridDim.x * kWarpNodeWarps;
  for (int64_t j = (int64_t)blockIdx.x * kWarpNodeWarps + w; j < d.m; j += nw) {
    fwd_node_warp<P, RPL>(d, mat, io, max_in, gcap, j, wsm);
    __syncwarp();  // the next node's inputs overwrite this node's shared memory
  }
}

// ---------------------------------------------------------------------------------------------
// Forward level kernels for one right-hand side. Variant 0: the per-node kernel; variants
// 1..6: the streaming kernel with ring layout A, B or C (see strm::Ring*), each with the node
// inputs copied by the producer (odd variants) or loaded by the consumers (even variants);
// variant 7: the warp-per-node kernel (levels whose blocks have at most 128 rows); variants
// 8..13: variants 1..6 with the column split of blocks of at most 96 rows (strm::MAX_GROUPS);
// variants 14, 15: ring layout D (four CTAs per SM) with the column split, inputs copied by the
// producer or loaded by the consumers.
constexpr int kNumFwdVariants = IDBF_NUM_FWD_VARIANTS;
// variants kFirstPairVariant .. + 3 on level l run levels l and l + 1 in one launch (radix-2
// level fusion; streaming kernel with ring layout A, B, C or D, inputs copied by the producer,
// column split of short blocks)
constexpr int kFirstPairVariant = 16;
static_assert(kFirstPairVariant + 4 == kNumFwdVariants, "pair variants close the list");
static bool is_pair_variant(int v) { return v >= kFirstPairVariant && v < kNumFwdVariants; }

static int default_variant(int fmt) { return fmt == IDBF_STORE_C128 ? 0 : 1; }

// One level l (pair = false) or the fused pair of levels l, l + 1 (pair = true) with the
// streaming kernel and ring layout RG.
template <class P, class RG>
static idbf_status launch_stream(Plan* p, int l, bool pair, bool bulk, bool split_short, const void* x,
                                 IO<typename P::vec_t> io, cudaStream_t st) {
  using V = typename P::vec_t;
  if (pair && (l + 1 > p->L)) return IDBF_EUNSUPPORTED;
  const LevelInfo& li = p->lv[l];
  const LevelInfo& lj = p->lv[pair ? l + 1 : l];
  const int max_rows = std::max(li.max_rows, lj.max_rows);
  if (!p->d_status || max_rows > strm::MAX_RPT * strm::TCT ||
      max_rows * (int)sizeof(typename P::mat_t) > RG::STAGE_BYTES - 32)
    return IDBF_EUNSUPPORTED;
  const int max_in = std::max(li.max_in, lj.max_in), max_out = std::max(li.max_out, lj.max_out);
  const int max_cols_pair = std::max(li.max_cols_pair, lj.max_cols_pair);
  const int mid_elems = pair ? 2 * li.max_out : 0;  // the outputs of two level-l nodes
  const int rpt = max_rows <= strm::TCT ? 1 : 2;
  // per-SM shared memory 228 KB: each CTA also reserves 1 KB and < 1 KB of static storage
  const size_t cap = (size_t)(228 / RG::CTAS - 2) * 1024;
  // the column split of short blocks (one output row per thread only) if its buffer fits
  int split = rpt == 1 && split_short ? 1 : 0;
  strm::Geo geo = strm::geometry<P, RG>(max_in, max_out, max_cols_pair, rpt, split, mid_elems);
  if (split && geo.total > cap) {
    split = 0;
    geo = strm::geometry<P, RG>(max_in, max_out, max_cols_pair, rpt, split, mid_elems);
  }
  if (geo.total > cap) return IDBF_EUNSUPPORTED;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t units = pair ? p->m / 2 : p->m;
  const unsigned ctas = (unsigned)std::min<int64_t>(units, (int64_t)RG::CTAS * sms);
  // bulk copies of the level-0 inputs read whole 16-byte granules: every leaf of x must start and
  // end on one (uneven leaves: only with 16-byte elements), else the consumers load them
  const int x_ok = ((uintptr_t)x % 16 == 0) &&
                   (p->uneven ? sizeof(V) % 16 == 0 : (p->n0 * (int)sizeof(V)) % 16 == 0);
  const int use_bulk = bulk && (l > 0 || x_ok);
  const DevLevel d = p->level(l);
  const DevLevel d1 = p->level(pair ? l + 1 : l);
  const typename P::mat_t* mat = (const typename P::mat_t*)p->lmat[fmt_of<P>()][l];
  const typename P::mat_t* mat1 = (const typename P::mat_t*)p->lmat[fmt_of<P>()][pair ? l + 1 : l];
  auto go = [&](auto kern) -> idbf_status {
    IDBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geo.total));
    kern<<<ctas, RG::NTHREADS, geo.total, st>>>(d, mat, d1, mat1, io, max_in, max_out, max_cols_pair, mid_elems,
                                                use_bulk, p->d_status, p->wait_limit_ns, p->producer_enabled);
    return IDBF_OK;
  };
  idbf_status s;
  if (pair) {
    s = rpt == 2 ? go(k_level_stream<P, RG, 2, false, true>)
        : split  ? go(k_level_stream<P, RG, 1, true, true>)
                 : go(k_level_stream<P, RG, 1, false, true>);
  } else {
    s = rpt == 2 ? go(k_level_stream<P, RG, 2, false, false>)
        : split  ? go(k_level_stream<P, RG, 1, true, false>)
                 : go(k_level_stream<P, RG, 1, false, false>);
  }
  if (s != IDBF_OK) return s;
  IDBF_CUDA_TRY(cudaGetLastError());
  return IDBF_OK;
}

template <class P>
static idbf_status launch_warp_node(Plan* p, int l, IO<typename P::vec_t> io, cudaStream_t st, int fmt) {
  const LevelInfo& li = p->lv[l];
  const int gcap = std::max(li.max_cols, li.max_in);
  const size_t per = warp_node_smem<P>(li.max_in, gcap, li.max_out);
  if (li.max_rows > 128 || per > 24 * 1024) return IDBF_EUNSUPPORTED;
  const size_t sm = per * kWarpNodeWarps;
  const DevLevel d = p->level(l);
  const typename P::mat_t* mat = (const typename P::mat_t*)p->lmat[fmt][l];
  const unsigned grid = (unsigned)((p->m + kWarpNodeWarps - 1) / kWarpNodeWarps);
  auto go = [&](auto kern) -> idbf_status {
    if (sm > 48 * 1024) IDBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    kern<<<grid, kWarpNodeWarps * 32, sm, st>>>(d, mat, io, li.max_in, gcap, li.max_out);
    IDBF_CUDA_TRY(cudaGetLastError());
    return IDBF_OK;
  };
  if (li.max_rows <= 32) return go(k_level_warp<P, 1>);
  if (li.max_rows <= 64) return go(k_level_warp<P, 2>);
  return go(k_level_warp<P, 4>);
}

template <class P>
static idbf_status launch_fwd_variant(Plan* p, int l, int v, const void* x, void* y, const typename P::vec_t* win,
                                      typename P::vec_t* wout, cudaStream_t st, int fmt) {
  using V = typename P::vec_t;
  IO<V> io;
  io.x = (const V*)x; io.ldx = p->N; io.y = (V*)y; io.ldy = p->N; io.R = 1;
  io.win = win; io.wout = wout;
  if (v == 7 && p->uneven) return IDBF_EUNSUPPORTED;  // uneven leaves: per-node and streaming kernels
  if (v == 7) return launch_warp_node<P>(p, l, io, st, fmt);
  if (v != 0 && fmt == IDBF_STORE_C128) return IDBF_EUNSUPPORTED;  // FP64: per-node or warp-per-node kernel
  if (v >= kFirstPairVariant) {  // levels l and l + 1 fused (win: boundary l - 1, wout: boundary l + 1)
    switch (v - kFirstPairVariant) {
      case 0: return launch_stream<P, strm::RingA>(p, l, true, true, true, x, io, st);
      case 1: return launch_stream<P, strm::RingB>(p, l, true, true, true, x, io, st);
      case 2: return launch_stream<P, strm::RingC>(p, l, true, true, true, x, io, st);
      default: return launch_stream<P, strm::RingD>(p, l, true, true, true, x, io, st);
    }
  }
  if (v == 14 || v == 15) return launch_stream<P, strm::RingD>(p, l, false, v == 14, true, x, io, st);
  const bool split = v >= 8;
  switch (split ? v - 7 : v) {
    case 1: return launch_stream<P, strm::RingA>(p, l, false, true, split, x, io, st);
    case 2: return launch_stream<P, strm::RingA>(p, l, false, false, split, x, io, st);
    case 3: return launch_stream<P, strm::RingB>(p, l, false, true, split, x, io, st);
    case 4: return launch_stream<P, strm::RingB>(p, l, false, false, split, x, io, st);
    case 5: return launch_stream<P, strm::RingC>(p, l, false, true, split, x, io, st);
    case 6: return launch_stream<P, strm::RingC>(p, l, false, false, split, x, io, st);
    default: break;
  }
  const LevelInfo& li = p->lv[l];
  const DevLevel d = p->level(l);
  const typename P::mat_t* mat = (const typename P::mat_t*)p->lmat[fmt][l];
  const int gcap = std::max(std::max(li.max_cols, li.max_rows), li.max_in);
  const int rcap = std::max(li.max_rows, li.max_cols);
  const size_t sm = li.max_in * sizeof(V) + 2 * gcap * sizeof(typename P::gv_t) + 2 * rcap * sizeof(V) + li.max_out * sizeof(V);
  if (sm > 200 * 1024) return IDBF_EUNSUPPORTED;
  if (sm > 48 * 1024) IDBF_CUDA_TRY(cudaFuncSetAttribute(k_level_fwd<P, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int threads = ((li.max_rows_pair + 31) / 32) * 32;
  threads = std::max(64, std::min(512, threads));
  k_level_fwd<P, 1><<<dim3((unsigned)p->m, 1), threads, sm, st>>>(d, mat, io, gcap, rcap, li.max_in);
  IDBF_CUDA_TRY(cudaGetLastError());
  return IDBF_OK;
}

// ---------------------------------------------------------------------------------------------
idbf_status ensure_workspace(Plan* p, int64_t nrhs) {
  const size_t need = (size_t)2 * p->max_seg_total * nrhs * 16;
  if (need <= p->ws_bytes) return IDBF_OK;
  if (p->d_ws) {
    IDBF_CUDA_TRY(cudaDeviceSynchronize());
    IDBF_CUDA_TRY(cudaFree(p->d_ws));
    p->d_ws = nullptr;
    p->ws_bytes = 0;
  }
  IDBF_CUDA_TRY(cudaMalloc(&p->d_ws, need));
  p->ws_bytes = need;
  return IDBF_OK;
}

// Forward apply of one right-hand side: per level the autotuned variant (else the default). A
// pair variant on level l runs levels l and l + 1 in one launch. Each launch reads the buffer the
// previous one wrote and writes the other one.
template <class P>
static idbf_status run_fwd1(Plan* p, const void* x, void* y, int64_t ld, cudaStream_t st, int fmt) {
  using V = typename P::vec_t;
  V* wb[2] = {(V*)p->d_ws, (V*)((char*)p->d_ws + (size_t)p->max_seg_total * 16)};
  int cur = 1;  // buffer holding the last boundary written (boundary b in b % 2 without pairs)
  for (int l = 0; l <= p->L;) {
    int v = p->tuned[fmt].size() > (size_t)l && p->tuned[fmt][l] >= 0 ? p->tuned[fmt][l] : default_variant(fmt);
    const bool pair = is_pair_variant(v) && l < p->L;
    const int last = pair ? l + 1 : l;  // level whose outputs this launch writes
    const V* win = l > 0 ? wb[cur] : nullptr;
    V* wout = last < p->L ? wb[cur ^ 1] : nullptr;
    (void)ld;
    idbf_status s = IDBF_EUNSUPPORTED;
    if (is_pair_variant(v) && !pair) v = default_variant(fmt);  // a pair variant on level L: one level
    s = launch_fwd_variant<P>(p, l, v, x, y, win, wout, st, fmt);
    if (s == IDBF_EUNSUPPORTED && pair) {  // the pair does not fit: level l alone, into the next buffer
      V* wout1 = wb[cur ^ 1];               // l < L here, so level l writes a workspace boundary
      s = launch_fwd_variant<P>(p, l, default_variant(fmt), x, y, win, wout1, st, fmt);
      if (s == IDBF_EUNSUPPORTED) s = launch_fwd_variant<P>(p, l, 0, x, y, win, wout1, st, fmt);
      if (s != IDBF_OK) return s;
      if (l < p->L) cur ^= 1;
      ++l;
      continue;
    }
    if (s == IDBF_EUNSUPPORTED && v != 0) s = launch_fwd_variant<P>(p, l, 0, x, y, win, wout, st, fmt);
    if (s != IDBF_OK) return s;
    if (last < p->L) cur ^= 1;
    l = last + 1;
  }
  return IDBF_OK;
}

template <class P, int RB>
static idbf_status run_levels(Plan* p, const void* x, void* y, int64_t R, int64_t ld, bool adjoint, cudaStream_t st,
                              int fmt) {
  using V = typename P::vec_t;
  if constexpr (RB == 1) {
    if (!adjoint && R == 1) return run_fwd1<P>(p, x, y, ld, st, fmt);
  }
  V* ws0 = (V*)p->d_ws;
  V* ws1 = (V*)((char*)p->d_ws + (size_t)p->max_seg_total * R * 16);
  const int nlev = p->L + 1;
  for (int step = 0; step < nlev; ++step) {
    const int l = adjoint ? p->L - step : step;
    const LevelInfo& li = p->lv[l];
    const DevLevel d = p->level(l);
    const typename P::mat_t* mat = (const typename P::mat_t*)p->lmat[fmt][l];
    IO<V> io;
    io.x = (const V*)x; io.ldx = ld; io.y = (V*)y; io.ldy = ld; io.R = (int)R;
    // boundary b lives in buffer b % 2; forward level l reads b = l-1 and writes b = l,
    // adjoint level l reads b = l and writes b = l-1.
    V* wb[2] = {ws0, ws1};
    if (!adjoint) {
      io.win = l > 0 ? wb[(l - 1) & 1] : nullptr;
      io.wout = l < p->L ? wb[l & 1] : nullptr;
    } else {
      io.win = l < p->L ? wb[l & 1] : nullptr;
      io.wout = l > 0 ? wb[(l - 1) & 1] : nullptr;
    }
    const int gcap = std::max(std::max(li.max_cols, li.max_rows), li.max_in);
    const int rcap = std::max(li.max_rows, li.max_cols);
    dim3 grid((unsigned)p->m, (unsigned)((R + RB - 1) / RB));
    if (!adjoint && RB == 1) {
      // one right-hand side, forward: the per-level variant (autotuned, else the default)
      const int v = p->uneven ? 0
                    : p->tuned[fmt].size() > (size_t)l && p->tuned[fmt][l] >= 0 ? p->tuned[fmt][l] : default_variant(fmt);
      idbf_status s = launch_fwd_variant<P>(p, l, v, x, y, io.win, io.wout, st, fmt);
      if (s == IDBF_EUNSUPPORTED && v != 0) s = launch_fwd_variant<P>(p, l, 0, x, y, io.win, io.wout, st, fmt);
      if (s != IDBF_OK) return s;
      continue;
    }
    if constexpr (RB >= 8 && tiled_ok<P>()) {
      if (!adjoint && !p->uneven) {
      // several right-hand sides, FP32 / FP64: register tiles over streamed factor columns
      // short blocks: 128 threads per CTA, so that more nodes (each a chain of dependent memory
      // accesses) are in flight per SM
      // (FP32: up to 85 registers per thread there), else 256 threads (FP32: up to 128 registers;
      // FP64: unbounded, its tiles need more)
      constexpr bool f32 = sizeof(V) == 8;
      const bool small = f32 && li.max_rows <= 64;
      const int nt = small ? 128 : 256;
      const size_t sm = tiled::smem_bytes<P, RB, 4>(li.max_in, li.max_out, li.max_rows, nt);
      if (sm <= 200 * 1024) {
        auto kern = !f32 ? k_level_fwd_tiled<P, RB, 4, 1> : small ? k_level_fwd_tiled<P, RB, 4, f32 ? 3 : 1>
                                                                  : k_level_fwd_tiled<P, RB, 4, f32 ? 2 : 1>;
        if (sm > 48 * 1024)
          IDBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const int nblk = (int)((R + RB - 1) / RB);
        kern<<<(unsigned)(p->m * nblk), nt, sm, st>>>(d, mat, io, li.max_rows, li.max_in, li.max_out, nblk);
        IDBF_CUDA_TRY(cudaGetLastError());
        continue;
      }
      }
    }
    if (!adjoint) {
      // several right-hand sides: (row, pair of right-hand sides, column slice) per thread
      constexpr int RPT = RB >= 2 ? 2 : 1;
      constexpr int NT = 256;
      const size_t sm = fwd_node_smem<P, RB, RPT>(li.max_in, gcap, rcap, NT);
      if (sm > 200 * 1024) return IDBF_EUNSUPPORTED;
      if (sm > 48 * 1024)
        IDBF_CUDA_TRY(cudaFuncSetAttribute(k_level_fwd<P, RB, RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_level_fwd<P, RB, RPT><<<grid, NT, sm, st>>>(d, mat, io, gcap, rcap, li.max_in);
    } else {
      if constexpr (RB >= 8 && tiled_ok<P>()) {
        // several right-hand sides, FP32 / FP64: register tiles over streamed row chunks
        const size_t sm = tadj::smem_bytes<P, RB>(li.max_in, li.max_out, li.max_rows, li.max_cols);
        if (sm <= 200 * 1024 && !p->uneven) {
          constexpr bool f32 = sizeof(V) == 8;
          auto kern = k_level_adj_tiled<P, RB, f32 ? 2 : 1>;
          if (sm > 48 * 1024) IDBF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
          const int nblk = (int)((R + RB - 1) / RB);
          kern<<<(unsigned)(p->m * nblk), 256, sm, st>>>(d, mat, io, li.max_in, li.max_out, li.max_rows, li.max_cols,
                                                          nblk);
          IDBF_CUDA_TRY(cudaGetLastError());
          continue;
        }
      }
      const size_t sm = (size_t)RB * (li.max_out * sizeof(V) + 2 * gcap * sizeof(typename P::gv_t) +
                                      2 * rcap * sizeof(V) + li.max_in * sizeof(V));
      if (sm > 200 * 1024) return IDBF_EUNSUPPORTED;
      if (sm > 48 * 1024) IDBF_CUDA_TRY(cudaFuncSetAttribute(k_level_adj<P, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_level_adj<P, RB><<<grid, 256, sm, st>>>(d, mat, io, gcap, rcap, li.max_out);
    }
    IDBF_CUDA_TRY(cudaGetLastError());
  }
  return IDBF_OK;
}

static idbf_status apply_common(idbf_plan h, const void* x, void* y, int64_t nrhs, int64_t ld, int32_t mode,
                                void* stream, bool adjoint) {
  if (!h || !x || !y || nrhs < 1 || nrhs > (1 << 20)) return IDBF_EINVAL;
  Plan* p = &h->p;
  if (ld < p->N) return IDBF_EINVAL;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != p->device) return IDBF_EINVAL;
  int fmt;
  switch (mode) {
    case IDBF_MODE_FP64: fmt = IDBF_STORE_C128; break;
    case IDBF_MODE_DF64: fmt = IDBF_STORE_DF64; break;
    case IDBF_MODE_FP32: fmt = IDBF_STORE_C64; break;
    case IDBF_MODE_TF32X3: fmt = IDBF_STORE_C64; break;
    case IDBF_MODE_TF32X3_S64: fmt = IDBF_STORE_C64; break;
    default: return IDBF_EINVAL;
  }
  const bool tensor = mode == IDBF_MODE_TF32X3 || mode == IDBF_MODE_TF32X3_S64;
  if (mode == IDBF_MODE_TF32X3_S64) {
    // complex64 on every level but the middle one, which needs C128 or DF64
    for (int l = 0; l <= p->L; ++l)
      if (l != p->hV && p->lmat_len[l] > 0 && !p->lmat[IDBF_STORE_C64][l]) return IDBF_EUNSUPPORTED;
    if (p->lmat_len[p->hV] > 0 && !p->lmat[IDBF_STORE_C128][p->hV] && !p->lmat[IDBF_STORE_DF64][p->hV])
      return IDBF_EUNSUPPORTED;
  } else if (!p->has_format(fmt)) {
    return IDBF_EUNSUPPORTED;
  }
  if (tensor && adjoint) return IDBF_EUNSUPPORTED;
  idbf_status s = ensure_workspace(p, nrhs);
  if (s != IDBF_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (tensor) return apply_tf32x3(p, x, y, nrhs, ld, st, mode == IDBF_MODE_TF32X3_S64);
  const bool one = nrhs == 1;
  // several right-hand sides in FP32 / FP64 (forward and adjoint): 16 per tile from 16 on, else 8
  const bool wide = nrhs >= 16, mid = nrhs > 1;
  idbf_status s2 = IDBF_EUNSUPPORTED;
  switch (mode) {
    case IDBF_MODE_FP64:
      if (one) return run_levels<FP64P, 1>(p, x, y, nrhs, ld, adjoint, st, fmt);
      if (wide) s2 = run_levels<FP64P, 16>(p, x, y, nrhs, ld, adjoint, st, fmt);
      else if (mid) s2 = run_levels<FP64P, 8>(p, x, y, nrhs, ld, adjoint, st, fmt);
      // a level too large for the wide tiles' shared memory: all levels again with 4 per tile
      return s2 != IDBF_EUNSUPPORTED ? s2 : run_levels<FP64P, 4>(p, x, y, nrhs, ld, adjoint, st, fmt);
    case IDBF_MODE_DF64: return one ? run_levels<DF64P, 1>(p, x, y, nrhs, ld, adjoint, st, fmt)
                                    : run_levels<DF64P, 4>(p, x, y, nrhs, ld, adjoint, st, fmt);
    default:
      if (one) return run_levels<FP32P, 1>(p, x, y, nrhs, ld, adjoint, st, fmt);
      if (wide) s2 = run_levels<FP32P, 16>(p, x, y, nrhs, ld, adjoint, st, fmt);
      else if (mid) s2 = run_levels<FP32P, 8>(p, x, y, nrhs, ld, adjoint, st, fmt);
      return s2 != IDBF_EUNSUPPORTED ? s2 : run_levels<FP32P, 4>(p, x, y, nrhs, ld, adjoint, st, fmt);
  }
}

// ---------------------------------------------------------------------------------------------
// The middle factor S^h of IDBF_MODE_TF32X3_S64 (the other levels run on the tensor cores): the
// complex64 boundaries h_V - 1 and h_V of the workspace, the products and sums in double-float
// (DF64 storage of the level, preferred: FP32 issue) or FP64 (C128 storage: the FP64 pipes), four
// right-hand sides per CTA, two per thread.
idbf_status apply_middle_wide(Plan* p, const void* win, void* wout, int64_t R, cudaStream_t st) {
  const int l = p->hV;
  const LevelInfo& li = p->lv[l];
  const bool df = p->lmat[IDBF_STORE_DF64][l] != nullptr;
  if (!df && !p->lmat[IDBF_STORE_C128][l]) return IDBF_EUNSUPPORTED;
  constexpr int RPT = 2, NT = 256;
  const int gcap = std::max(std::max(li.max_cols, li.max_rows), li.max_in);
  const int rcap = std::max(li.max_rows, li.max_cols);
  const DevLevel d = p->level(l);
  IO<float2> io;
  io.x = nullptr; io.ldx = p->N; io.y = nullptr; io.ldy = p->N; io.R = (int)R;
  io.win = (const float2*)win; io.wout = (float2*)wout;
  // four right-hand sides per CTA: two CTAs per SM (eight per CTA halve the re-reads of the
  // node's blocks but leave one CTA per SM: 348 ms against 200 ms for this level at N = 2^18 with
  // 256 right-hand sides)
  auto go = [&](auto pol, auto rbc, const void* mat) -> idbf_status {
    using Pol = decltype(pol);
    constexpr int RB = decltype(rbc)::value;
    const size_t sm = fwd_node_smem<Pol, RB, RPT>(li.max_in, gcap, rcap, NT);
    if (sm > 200 * 1024) return IDBF_EUNSUPPORTED;
    if (sm > 48 * 1024)
      IDBF_CUDA_TRY(cudaFuncSetAttribute(k_level_fwd<Pol, RB, RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const dim3 grid((unsigned)p->m, (unsigned)((R + RB - 1) / RB));
    k_level_fwd<Pol, RB, RPT><<<grid, NT, sm, st>>>(d, (const typename Pol::mat_t*)mat, io, gcap, rcap, li.max_in);
    IDBF_CUDA_TRY(cudaGetLastError());
    return IDBF_OK;
  };
  using RB4 = std::integral_constant<int, 4>;
  if (df) return go(DF64S32P(), RB4(), p->lmat[IDBF_STORE_DF64][l]);
  return go(FP64S32P(), RB4(), p->lmat[IDBF_STORE_C128][l]);
}

// ---------------------------------------------------------------------------------------------
// Allocation-free forward apply (idbf_apply_noalloc). The level-to-level workspace is a fixed
// array compiled into the library instead of the plan's cudaMalloc'ed workspace. In host code
// the symbol below is only a host-side stand-in: its device address is looked up once per
// device with cudaGetSymbolAddress and cached.
static __device__ __align__(256) unsigned char g_noalloc_scratch[IDBF_NOALLOC_SCRATCH_BYTES];

static constexpr int kNoallocMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static void* g_noalloc_addr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on first use).
static idbf_status noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kNoallocMaxDevices) return IDBF_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      set_cuda_error(e);
      return IDBF_ECUDA;
    }
    g_noalloc_addr[dev] = ptr;
  }
  *out = g_noalloc_addr[dev];
  return IDBF_OK;
}

// Shared memory of the per-node forward kernel k_level_fwd<P, RB> on level l.
template <class P, int RB>
static size_t scratch_level_smem(const Plan* p, int l) {
  using V = typename P::vec_t;
  const LevelInfo& li = p->lv[l];
  const int gcap = std::max(std::max(li.max_cols, li.max_rows), li.max_in);
  const int rcap = std::max(li.max_rows, li.max_cols);
  return (size_t)RB * (li.max_in * sizeof(V) + 2 * gcap * sizeof(typename P::gv_t) + 2 * rcap * sizeof(V) +
                       li.max_out * sizeof(V));
}

// The forward level loop of run_levels with the two ping-pong buffers placed in `ws`. Every
// level's shared memory is checked before the first launch, so that a refused request leaves
// y untouched.
template <class P, int RB>
static idbf_status run_levels_scratch(Plan* p, const void* x, void* y, int64_t R, int64_t ld, cudaStream_t st,
                                      int fmt, void* ws) {
  using V = typename P::vec_t;
  for (int l = 0; l <= p->L; ++l)
    if (scratch_level_smem<P, RB>(p, l) > 200 * 1024) return IDBF_EUNSUPPORTED;
  V* wb[2] = {(V*)ws, (V*)((char*)ws + (size_t)p->max_seg_total * R * 16)};
  for (int l = 0; l <= p->L; ++l) {
    const LevelInfo& li = p->lv[l];
    const DevLevel d = p->level(l);
    const typename P::mat_t* mat = (const typename P::mat_t*)p->lmat[fmt][l];
    IO<V> io;
    io.x = (const V*)x; io.ldx = ld; io.y = (V*)y; io.ldy = ld; io.R = (int)R;
    io.win = l > 0 ? wb[(l - 1) & 1] : nullptr;
    io.wout = l < p->L ? wb[l & 1] : nullptr;
    const int gcap = std::max(std::max(li.max_cols, li.max_rows), li.max_in);
    const int rcap = std::max(li.max_rows, li.max_cols);
    dim3 grid((unsigned)p->m, (unsigned)((R + RB - 1) / RB));
    const size_t sm = scratch_level_smem<P, RB>(p, l);
    if (sm > 48 * 1024) IDBF_CUDA_TRY(cudaFuncSetAttribute(k_level_fwd<P, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int threads = ((li.max_rows_pair + 31) / 32) * 32;
    threads = std::max(64, std::min(512, threads));
    k_level_fwd<P, RB><<<grid, threads, sm, st>>>(d, mat, io, gcap, rcap, li.max_in);
    IDBF_CUDA_TRY(cudaGetLastError());
  }
  return IDBF_OK;
}

// ---------------------------------------------------------------------------------------------
// Autotuner: time every forward variant of every level (one right-hand side) and keep the fastest.
template <class P>
static idbf_status autotune_fmt(Plan* p, int fmt, cudaStream_t st, int reps, float* best_ms_out) {
  using V = typename P::vec_t;
  idbf_status s = ensure_workspace(p, 1);
  if (s != IDBF_OK) return s;
  void *x = nullptr, *y = nullptr;
  IDBF_CUDA_TRY(cudaMalloc(&x, p->N * sizeof(V)));
  if (cudaMalloc(&y, p->N * sizeof(V)) != cudaSuccess) { cudaFree(x); return IDBF_ENOMEM; }
  cudaMemsetAsync(x, 0x3e, p->N * sizeof(V), st);
  V* wb[2] = {(V*)p->d_ws, (V*)((char*)p->d_ws + (size_t)p->max_seg_total * 16)};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // workspace filled with real values: every level once, boundary b left in buffer b % 2
  p->tuned[fmt].assign(p->L + 1, -1);
  s = run_levels<P, 1>(p, x, y, 1, p->N, false, st, fmt);
  // best time of one variant (single level: v < kFirstPairVariant; else the pair l, l + 1)
  auto time_variant = [&](int l, int v, float* ms_out) -> idbf_status {
    const V* win = l > 0 ? wb[(l - 1) & 1] : nullptr;
    const int last = is_pair_variant(v) ? l + 1 : l;
    V* wout = last < p->L ? wb[l & 1] : nullptr;  // a pair's output goes to the other buffer too
    idbf_status r = launch_fwd_variant<P>(p, l, v, x, y, win, wout, st, fmt);
    if (r != IDBF_OK) return r;
    cudaEventRecord(e0, st);
    for (int k = 0; k < reps; ++k) launch_fwd_variant<P>(p, l, v, x, y, win, wout, st, fmt);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return IDBF_ECUDA;
    cudaEventElapsedTime(ms_out, e0, e1);
    return IDBF_OK;
  };
  const int nl = p->L + 1;
  std::vector<float> one(nl, 1e30f), two(nl, 1e30f);
  std::vector<int> one_v(nl, default_variant(fmt)), two_v(nl, -1);
  for (int l = 0; l < nl && s == IDBF_OK; ++l) {
    for (int v = 0; v < kNumFwdVariants && s == IDBF_OK; ++v) {
      if (is_pair_variant(v) && l == p->L) continue;
      float ms = 0.f;
      const idbf_status r = time_variant(l, v, &ms);
      if (r == IDBF_EUNSUPPORTED) continue;
      if (r != IDBF_OK) { s = r; break; }
      if (is_pair_variant(v)) {
        if (ms < two[l]) { two[l] = ms; two_v[l] = v; }
      } else if (ms < one[l]) {
        one[l] = ms; one_v[l] = v;
      }
    }
  }
  // the cheapest way to cover levels 0..L with single levels and fused pairs (left to right, as
  // run_fwd1 reads the choices)
  std::vector<float> cost(nl + 1, 0.f);
  std::vector<int> take_pair(nl, 0);
  for (int l = nl - 1; l >= 0; --l) {
    cost[l] = one[l] + cost[l + 1];
    if (l + 1 < nl && two_v[l] >= 0 && two[l] + cost[l + 2] < cost[l]) {
      cost[l] = two[l] + cost[l + 2];
      take_pair[l] = 1;
    }
  }
  p->tuned[fmt].assign(nl, -1);
  for (int l = 0; l < nl;) {
    if (take_pair[l]) {
      p->tuned[fmt][l] = p->tuned[fmt][l + 1] = two_v[l];
      l += 2;
    } else {
      p->tuned[fmt][l] = one_v[l];
      l += 1;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(x);
  cudaFree(y);
  if (best_ms_out) *best_ms_out = cost[0] / reps;
  return s;
}

}  // namespace idbf

extern "C" {

idbf_status idbf_apply(idbf_plan h, const void* x, void* y, int64_t nrhs, int64_t ld, int32_t mode, void* stream) {
  return idbf::apply_common(h, x, y, nrhs, ld, mode, stream, false);
}

idbf_status idbf_apply_adjoint(idbf_plan h, const void* x, void* y, int64_t nrhs, int64_t ld, int32_t mode,
                               void* stream) {
  return idbf::apply_common(h, x, y, nrhs, ld, mode, stream, true);
}

idbf_status idbf_autotune(idbf_plan h, int32_t mode, int32_t reps, void* stream, float* apply_ms) {
  using namespace idbf;
  if (!h || reps < 1) return IDBF_EINVAL;
  Plan* p = &h->p;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != p->device) return IDBF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  switch (mode) {
    case IDBF_MODE_FP64: return p->has_format(IDBF_STORE_C128) ? autotune_fmt<FP64P>(p, IDBF_STORE_C128, st, reps, apply_ms) : IDBF_EUNSUPPORTED;
    case IDBF_MODE_DF64: return p->has_format(IDBF_STORE_DF64) ? autotune_fmt<DF64P>(p, IDBF_STORE_DF64, st, reps, apply_ms) : IDBF_EUNSUPPORTED;
    case IDBF_MODE_FP32: return p->has_format(IDBF_STORE_C64) ? autotune_fmt<FP32P>(p, IDBF_STORE_C64, st, reps, apply_ms) : IDBF_EUNSUPPORTED;
    default: return IDBF_EINVAL;
  }
}

idbf_status idbf_set_level_variants(idbf_plan h, int32_t mode, const int32_t* variants, int32_t n) {
  using namespace idbf;
  if (!h || n < 0 || (n > 0 && !variants)) return IDBF_EINVAL;
  Plan* p = &h->p;
  if (n != 0 && n != p->L + 1) return IDBF_EINVAL;
  const int fmt = mode == IDBF_MODE_FP64 ? IDBF_STORE_C128 : mode == IDBF_MODE_DF64 ? IDBF_STORE_DF64
                : mode == IDBF_MODE_FP32 ? IDBF_STORE_C64 : -1;
  if (fmt < 0) return IDBF_EINVAL;
  for (int i = 0; i < n; ++i)
    if (variants[i] < -1 || variants[i] >= kNumFwdVariants) return IDBF_EINVAL;
  p->tuned[fmt].assign(variants, variants + n);
  return IDBF_OK;
}

idbf_status idbf_apply_noalloc(idbf_plan h, const void* x, void* y, int64_t nrhs, int64_t ld, int32_t mode,
                               void* stream) {
  using namespace idbf;
  if (!h || !x || !y || nrhs < 1 || nrhs > (1 << 20)) return IDBF_EINVAL;
  Plan* p = &h->p;
  if (ld < p->N) return IDBF_EINVAL;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != p->device) return IDBF_EINVAL;
  int fmt;
  switch (mode) {
    case IDBF_MODE_FP64: fmt = IDBF_STORE_C128; break;
    case IDBF_MODE_DF64: fmt = IDBF_STORE_DF64; break;
    case IDBF_MODE_FP32: fmt = IDBF_STORE_C64; break;
    default: return IDBF_EINVAL;
  }
  if (!p->has_format(fmt)) return IDBF_EUNSUPPORTED;
  // two ping-pong buffers of the largest boundary, 16 bytes per element and right-hand side
  const unsigned long long need = 2ull * (unsigned long long)p->max_seg_total * (unsigned long long)nrhs * 16ull;
  if (need > IDBF_NOALLOC_SCRATCH_BYTES) return IDBF_EUNSUPPORTED;
  void* ws = nullptr;
  const idbf_status s = noalloc_scratch(cur, &ws);
  if (s != IDBF_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const bool one = nrhs == 1;
  switch (mode) {
    case IDBF_MODE_FP64: return one ? run_levels_scratch<FP64P, 1>(p, x, y, nrhs, ld, st, fmt, ws)
                                    : run_levels_scratch<FP64P, 4>(p, x, y, nrhs, ld, st, fmt, ws);
    case IDBF_MODE_DF64: return one ? run_levels_scratch<DF64P, 1>(p, x, y, nrhs, ld, st, fmt, ws)
                                    : run_levels_scratch<DF64P, 4>(p, x, y, nrhs, ld, st, fmt, ws);
    default: return one ? run_levels_scratch<FP32P, 1>(p, x, y, nrhs, ld, st, fmt, ws)
                        : run_levels_scratch<FP32P, 4>(p, x, y, nrhs, ld, st, fmt, ws);
  }
}

}  // extern "C"
