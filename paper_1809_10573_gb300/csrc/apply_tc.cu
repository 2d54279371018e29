// Multi-right-hand-side apply on the tensor cores (tcgen05, kind::tf32, split precision).
//
// With R right-hand sides every butterfly block product M_c G (M_c: rows x cols complex, G:
// cols x R) becomes a dense GEMM (Eq. 1 applied to a block of vectors). The complex product is
// embedded in real arithmetic with interleaved real / imaginary parts and computed transposed,
// D^T = G^T M_c^T, so that the tensor core's M dimension is 128 right-hand sides and its N
// dimension 128 of the block's 2 x rows real output rows per pass (accumulators in TMEM):
//   A (M = 128 rhs x K = 2 cols):  A(n, 2k) = Re G(k, n),  A(n, 2k+1) = Im G(k, n)
//   B (N = 2 rows x K = 2 cols):   B(2r, 2k) = Re M(r,k), B(2r, 2k+1) = -Im M(r,k),
//                                  B(2r+1, 2k) = Im M(r,k), B(2r+1, 2k+1) = Re M(r,k)
//   D (128 x 2 rows):              D(n, 2r) = Re (M G)(r, n), D(n, 2r+1) = Im (M G)(r, n).
// Split precision (3xTF32, Ootomo and Yokota, "Recovering single precision accuracy from Tensor
// Cores while surpassing the FP32 theoretical peak performance", IJHPCA 2022): x = x_hi + x_lo with
// x_hi = rna_tf32(x), x_lo = x - x_hi, and A B ~ A_hi B_hi + (A_hi B_lo + A_lo B_hi). The tensor
// core accumulates in FP32 with its own rounding of every addition, so the error of one long
// accumulation grows with the number of K steps: the main products of chunk k go to one of
// NACC = 3 TMEM accumulators (k mod 3), each of which sums a third of the terms, and the two
// correction products (~2^-11 of the main ones, which would lose their low bits in the main
// accumulators) to a fourth; the four are summed in round-to-nearest FP32 in the epilogue. With
// 4 x 128 TMEM columns a pass covers 128 real (64 complex) output rows; a block takes up to four
// passes. Eight warps stage the operands: each thread copies with cp.async, four chunks ahead,
// exactly the values it later converts, splits them into TF32 hi / lo and stores them in the
// K-major, no-swizzle canonical layout (8-row x 16-byte core matrices), 16 bytes at a time (two
// complex columns of one row) so that a warp's stores fill 512 contiguous bytes; four stages
// over K. A ninth warp issues the MMAs as soon as a stage is full (mbarrier), and
// tcgen05.commit frees the stage; the staging warps read the accumulators out after each pass.
#include <cuda_runtime.h>

#include <algorithm>

#include "idbf_internal.h"

namespace idbf {
namespace tc {

constexpr int NT = 256;          // threads per CTA (8 warps)
constexpr int MR = 128;          // right-hand sides per tile (MMA M)
constexpr int KC = 8;            // complex columns per staged chunk (16 real K)
constexpr int NH = 128;          // real output rows per pass (MMA N)
constexpr int MAXPASS = 4;
constexpr int MAXROWS = MAXPASS * NH / 2;  // complex rows per block supported
constexpr int NACC = 3;          // main accumulators (chunks dealt round robin)
constexpr uint32_t SBO = 128;    // byte step between 8-row core-matrix groups
constexpr uint32_t A_BYTES = MR * 2 * KC * 4;     // 8 KB
constexpr uint32_t B_BYTES = NH * 2 * KC * 4;     // 8 KB
constexpr uint32_t LBO_A = (MR / 8) * 128;        // byte step between 4-element K groups
constexpr uint32_t LBO_B = (NH / 8) * 128;
constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;  // hi and lo of both operands: 32 KB
constexpr int NSTAGE = 4;
constexpr int PFR = 4;           // chunks whose global operands are in flight (cp.async raw ring)
constexpr int RAWV = 8;          // raw complex values per thread per chunk (A: 2 items x 2, B: 2 x 2)
constexpr uint32_t RAW_BYTES = RAWV * NT * 8;          // one raw chunk: 16 KB, value-major
constexpr int GIXCAP = 1024;     // columns per block supported (gather indices in shared memory)
constexpr size_t RAW_OFF = NSTAGE * (size_t)STAGE;
constexpr size_t GIX_OFF = RAW_OFF + PFR * (size_t)RAW_BYTES;
constexpr size_t QIX_OFF = GIX_OFF + GIXCAP * sizeof(int32_t);
constexpr size_t BAR_OFF = QIX_OFF + MAXROWS * sizeof(int32_t);
constexpr size_t SMEM = BAR_OFF + 128;                 // stages, raw ring, indices, barriers
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t D_CORR = NACC * NH;                 // TMEM column of the correction accumulator
constexpr int A_PER_T = MR * (KC / 2) / NT;            // 2 (rhs, column pair) items per thread per chunk
constexpr int B_PER_T = NH * (KC / 2) / NT;            // 2 (real row, column pair) items per thread per chunk
static_assert(D_CORR + NH <= TMEM_COLS, "accumulators fit in TMEM");
static_assert(A_PER_T * NT == MR * (KC / 2) && B_PER_T * NT == NH * (KC / 2), "whole items per thread");
static_assert(RAWV == 2 * (A_PER_T + B_PER_T), "raw values per thread");
static_assert(SMEM <= 227 * 1024, "shared memory per CTA");

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok)
               : "r"(sa(b)), "r"(parity)
               : "memory");
  return ok != 0;
}
// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte offsets, version 1,
// no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor: D = F32, A = B = TF32, both K-major, N and M
__device__ __forceinline__ uint32_t idesc_tf32(uint32_t n, uint32_t m) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                   tmem),
               "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
               : "memory");
}
__device__ __forceinline__ void commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(b)) : "memory");
}
// byte offset of element (row, k) of a K-major no-swizzle tile with 4-byte elements
__device__ __forceinline__ uint32_t koff(int row, int k, uint32_t lbo) {
  return (uint32_t)((k >> 2) * lbo + (row >> 3) * SBO + (row & 7) * 16 + (k & 3) * 4);
}
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// four consecutive K elements of one row (two complex columns): one 16-byte store per split;
// the lo part is rounded to TF32 as well (rna) when round_lo is set, else left for the hardware
// to narrow
__device__ __forceinline__ void put4(unsigned char* hi, unsigned char* lo, uint32_t off, float4 v, int round_lo) {
  const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
  *(float4*)(hi + off) = h;
  float4 l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
  if (round_lo) l = make_float4(tf32_hi(l.x), tf32_hi(l.y), tf32_hi(l.z), tf32_hi(l.w));
  *(float4*)(lo + off) = l;
}

// 32 lanes x 16 consecutive 32-bit TMEM columns starting at taddr (warp-wide)
__device__ __forceinline__ void tmem_ld16(uint32_t (&v)[16], uint32_t taddr) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// 8-byte asynchronous copy global -> shared; src_bytes = 0 writes zeros (src is not read)
__device__ __forceinline__ void cp_async8(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(sa(dst)), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
// the staging / epilogue warps only (the MMA warp does not take part)
__device__ __forceinline__ void staging_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); }
// bounded wait that also gives up as soon as another warp has flagged a failure
__device__ __forceinline__ bool wait_abortable(uint64_t* b, uint32_t parity, uint64_t limit_ns, volatile int* abort_flag) {
  if (try_wait(b, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t n = 1;; ++n) {
    if (try_wait(b, parity)) return true;
    if ((n & 255) == 0 && (*abort_flag || gtimer() - t0 > limit_ns)) return false;
  }
}

// One launch per level; persistent CTAs over nodes. x / y: user blocks (column-major, ld);
// win / wout: workspace boundaries, element e of a segment at (off + e) * R + rhs.
// Warp roles: warps 0-7 stage operands (and read the accumulators out after each pass), warp 8
// issues the MMAs (its lane 0). Per stage s: full[s] (NT arrivals: staged), empty[s] (commit: the
// MMAs reading it are done); per pass: done (commit: accumulators final), tfree (NT arrivals:
// accumulators read out, the next pass may overwrite them). Every wait is bounded; on a failure a
// thread stops waiting and working but keeps walking the same loops, so that every warp meets the
// same named barriers, and bit 0 of *status is set.
__global__ void __launch_bounds__(NT + 32, 1)
    k_level_tc(DevLevel d, const float2* __restrict__ mat, const float2* __restrict__ x, int64_t ldx,
               float2* __restrict__ y, int64_t ldy, const float2* __restrict__ win, float2* __restrict__ wout, int R,
               int* __restrict__ status, uint64_t limit_ns, int split_mode) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  uint64_t* full = (uint64_t*)(sm + BAR_OFF);
  float2* raw = (float2*)(sm + RAW_OFF);     // [PFR][RAWV][NT]: each thread's own values
  int32_t* gix = (int32_t*)(sm + GIX_OFF);   // node-input element of each column of the block
  int32_t* qix = (int32_t*)(sm + QIX_OFF);   // per block row: V pass-through element, U output element
  uint64_t* empty = full + NSTAGE;
  uint64_t* done = empty + NSTAGE;
  uint64_t* tfree = done + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool mma_warp = warp == NT / 32;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < NSTAGE; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(&full[i])), "r"(NT) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(&empty[i])), "r"(1) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(done)), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(tfree)), "r"(NT) : "memory");
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  uint32_t kcg = 0, passes = 0;  // chunks and passes so far (mbarrier phases), same on every thread
  uint32_t issued = 0;           // chunks whose MMAs this thread committed (MMA thread)
  bool failed = false;
  volatile int* abortp = &abort_flag;
  auto fail = [&]() {
    failed = true;
    *abortp = 1;
  };
  const int nrt = (R + MR - 1) / MR;
  // this thread's staging items (the same in every chunk): A items (rhs n, column pair kp),
  // B items (real row rr, column pair kp); NT = 2 MR = 2 NH, so n = rr = tid % 128
  static_assert(NT == 2 * MR && NT == 2 * NH && A_PER_T == 2 && B_PER_T == 2, "item map");
  const int it_n = tid & (MR - 1), it_kp0 = tid >> 7;  // items t = 0, 1: column pairs kp0, kp0 + 2
  uint32_t offA[2], offB[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    offA[t] = koff(it_n, 4 * (it_kp0 + 2 * t), LBO_A);
    offB[t] = koff(it_n, 4 * (it_kp0 + 2 * t), LBO_B);
  }

  for (int64_t j = blockIdx.x; j < d.m; j += gridDim.x) {
    int l0, l1;
    int64_t ib0 = 0;
    if (d.lev == 0) { l0 = d.n0; l1 = 0; }
    else { l0 = d.in_len[2 * j]; l1 = d.in_len[2 * j + 1]; ib0 = d.in_off[2 * j]; }
    const int32_t* ix0 = d.idx + d.ioff[2 * j];
    const int32_t* ix1 = d.idx + d.ioff[2 * j + 1];
    // element e (of concat(in_0, in_1)), right-hand side n of the node input
    auto in_at = [&](int e, int n) -> float2 {
      return d.lev == 0 ? x[(j * d.n0 + e) + (int64_t)n * ldx] : win[(ib0 + e) * R + n];
    };
    // output element e of t = concat(out_0, out_1) (or of the leaf of y), right-hand side n
    int len_o0 = 0;
    int64_t ob0 = 0, ob1 = 0;
    if (d.lev < d.L) {
      const int64_t s0 = (j / d.H) * 2 * d.H + j % d.H, s1 = s0 + d.H;
      len_o0 = d.out_len[s0];
      ob0 = d.out_off[s0];
      ob1 = d.out_off[s1];
    }
    auto out_ptr = [&](int e, int n) -> float2* {
      if (d.lev == d.L) return y + (j * d.n0 + e) + (int64_t)n * ldy;
      return wout + ((e < len_o0 ? ob0 + e : ob1 + (e - len_o0)) * R + n);
    };
    if (d.kind == KIND_U && !mma_warp) {
      // t[q_0] = in_0 (t[p_0] comes from the block-0 products); q_1 part added with block 1
      if (!failed)
        for (int i = tid; i < l0 * R; i += NT) *out_ptr(ix0[i / R], i % R) = in_at(i / R, i % R);
      staging_sync();
    }
    for (int c = 0; c < 2; ++c) {
      const int rows = d.rows[2 * j + c], cols = d.cols[2 * j + c];
      const int32_t* ix = c ? ix1 : ix0;
      const float2* M = mat + d.moff[2 * j + c];
      // column k of the gathered operand G: which element of the node input
      auto g_elem = [&](int k) -> int {
        if (d.kind == KIND_V) return ix[rows + k];
        if (d.kind == KIND_U) return (c ? l0 : 0) + k;
        return k;  // S: all of concat(in_0, in_1)
      };
      if (d.kind == KIND_U && c == 1 && !mma_warp) {
        staging_sync();
        if (!failed)
          for (int i = tid; i < l1 * R; i += NT) {
            float2* q = out_ptr(ix1[i / R], i % R);
            const float2 a = *q, b = in_at(l0 + i / R, i % R);
            *q = make_float2(a.x + b.x, a.y + b.y);
          }
        staging_sync();
      }
      if (rows == 0) continue;
      if (cols == 0) {  // V block that keeps every column: out = u[q]
        if (!mma_warp && !failed)
          for (int i = tid; i < rows * R; i += NT) {
            const int r = i / R, n = i % R;
            *out_ptr((c ? len_o0 : 0) + r, n) = in_at(ix[r], n);
          }
        continue;
      }
      if (!mma_warp) {  // column k of the block multiplies node-input element gix[k]
        staging_sync();  // the previous block's copies are all issued
        for (int k = tid; k < cols; k += NT) gix[k] = g_elem(k);
        if (d.kind != KIND_S)
          for (int r = tid; r < rows; r += NT) qix[r] = d.kind == KIND_V ? ix[r] : ix[(c ? l1 : l0) + r];
        staging_sync();
      }
      const int nkc = (cols + KC - 1) / KC;
      const int npass = (rows + NH / 2 - 1) / (NH / 2);
      for (int rt = 0; rt < nrt; ++rt) {
        const int nr = min(MR, R - rt * MR);
        for (int ps = 0; ps < npass; ++ps, ++passes) {
          const int r0 = ps * (NH / 2);                       // first complex row of the pass
          const int prow = min(NH / 2, rows - r0);            // complex rows of the pass
          const int nreal = (2 * prow + 15) & ~15;            // MMA N (multiple of 16)
          if (mma_warp) {
            if (lane == 0) {
              // the previous pass's accumulators must have been read out
              if (!failed && passes > 0 && !wait_abortable(tfree, (passes - 1) & 1, limit_ns, abortp)) fail();
              const uint32_t id = idesc_tf32((uint32_t)nreal, MR);
              for (int kc = 0; kc < nkc; ++kc) {
                const uint32_t g = kcg + (uint32_t)kc;
                const int s = (int)(g % NSTAGE);
                if (failed) continue;
                if (!wait_abortable(&full[s], (g / NSTAGE) & 1, limit_ns, abortp)) { fail(); continue; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t Ah = sa(sm + (size_t)s * STAGE), Al = Ah + A_BYTES, Bh = Al + A_BYTES, Bl = Bh + B_BYTES;
                const uint32_t dmain = tmem + (uint32_t)(kc % NACC) * NH;
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {  // K = 8 real per MMA: two 4-element core groups
                  const uint32_t ao = 2 * ks * LBO_A, bo = 2 * ks * LBO_B;
                  const uint64_t ah = sdesc(Ah + ao, LBO_A, SBO), al = sdesc(Al + ao, LBO_A, SBO);
                  const uint64_t bh = sdesc(Bh + bo, LBO_B, SBO), bl = sdesc(Bl + bo, LBO_B, SBO);
                  const uint32_t first_main = (kc < NACC && ks == 0) ? 0u : 1u;
                  const uint32_t first_corr = (kc == 0 && ks == 0) ? 0u : 1u;
                  mma_tf32(dmain, ah, bh, id, first_main);            // main: hi * hi
                  mma_tf32(tmem + D_CORR, ah, bl, id, first_corr);    // corrections: hi * lo + lo * hi
                  mma_tf32(tmem + D_CORR, al, bh, id, 1u);
                  if (split_mode == 2) mma_tf32(tmem + D_CORR, al, bl, id, 1u);
                }
                commit(&empty[s]);
                ++issued;
                if (kc == nkc - 1) commit(done);
              }
            }
            kcg += (uint32_t)nkc;
            continue;
          }
          // ---- staging warps: each thread copies (cp.async, PFR chunks ahead) exactly the values
          // it later converts, into its own slots of the raw ring, so no barrier is needed
          // between the copies and their use. Items: (right-hand side n or real row rr, pair of
          // complex columns), four real K each.
          // where this thread's values of column k live: A: a_base + gix[k] * a_step (node input
          // element gix[k], right-hand side rt*MR + it_n); B: b_base + k * rows (block row r0 + it_n/2)
          const bool okA = it_n < nr, okB = (it_n >> 1) < prow;
          const float2* a_base = d.lev == 0 ? x + j * d.n0 + (int64_t)(rt * MR + it_n) * ldx : win + ib0 * R + rt * MR + it_n;
          const int64_t a_step = d.lev == 0 ? 1 : R;
          const float2* b_base = M + r0 + (it_n >> 1);
          auto issue_raw = [&](int kc) {
            if (kc < nkc && !failed) {
              float2* rs = raw + (size_t)(kc % PFR) * (RAWV * NT) + tid;
#pragma unroll
              for (int t = 0; t < 2; ++t)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const int k = kc * KC + 2 * (it_kp0 + 2 * t) + h;
                  const bool inb = k < cols;
                  const bool oa = okA && inb, ob = okB && inb;
                  cp_async8(rs + (2 * t + h) * NT, oa ? a_base + gix[k] * a_step : M, oa ? 8u : 0u);
                  cp_async8(rs + (4 + 2 * t + h) * NT, ob ? b_base + (int64_t)k * rows : M, ob ? 8u : 0u);
                }
            }
            cp_async_commit();  // one group per chunk (empty past the end), so that the counts match
          };
#pragma unroll
          for (int f = 0; f < PFR; ++f) issue_raw(f);
          for (int kc = 0; kc < nkc; ++kc) {
            const uint32_t g = kcg + (uint32_t)kc;
            const int s = (int)(g % NSTAGE);
            cp_async_wait<PFR - 1>();  // this thread's copies of chunk kc have landed
            // the MMAs that last read stage s must be done
            if (!failed && !wait_abortable(&empty[s], ((g / NSTAGE) & 1) ^ 1, limit_ns, abortp)) fail();
            if (!failed) {
              const float2* rs = raw + (size_t)(kc % PFR) * (RAWV * NT) + tid;
              unsigned char* Ah = sm + (size_t)s * STAGE;
              unsigned char* Al = Ah + A_BYTES;
              unsigned char* Bh = Al + A_BYTES;
              unsigned char* Bl = Bh + B_BYTES;
#pragma unroll
              for (int t = 0; t < 2; ++t) {
                const float2 g0 = rs[(2 * t) * NT], g1 = rs[(2 * t + 1) * NT];
                put4(Ah, Al, offA[t], make_float4(g0.x, g0.y, g1.x, g1.y), split_mode >= 1);
                const float2 m0 = rs[(4 + 2 * t) * NT], m1 = rs[(4 + 2 * t + 1) * NT];
                // real row 2r holds (Re M, -Im M) per column, real row 2r+1 (Im M, Re M)
                const float4 bv = (it_n & 1) ? make_float4(m0.y, m0.x, m1.y, m1.x) : make_float4(m0.x, -m0.y, m1.x, -m1.y);
                put4(Bh, Bl, offB[t], bv, split_mode >= 1);
              }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&full[s]);
            issue_raw(kc + PFR);  // into the slot just consumed
          }
          cp_async_wait<0>();
          kcg += (uint32_t)nkc;
          // ---- epilogue: lane quadrant of warp w % 4 = 32 rhs; warps w and w + 4 split the columns.
          // The terms added to the products (V: the pass-through input u[q]; U, block 1: block 0's
          // output) do not depend on the MMAs: they are loaded one column group ahead, the first
          // group before the wait for the pass's MMAs.
          const int q = warp & 3, half = warp >> 2;
          const int n = rt * MR + q * 32 + lane;
          float2 pre[8], nxt[8];
          auto load_terms = [&](int c0, float2 (&tv)[8]) {
#pragma unroll
            for (int h = 0; h < 8; ++h) {
              tv[h] = make_float2(0.f, 0.f);
              const int r = r0 + (c0 >> 1) + h;
              if (failed || n >= R || c0 >= nreal || (c0 >> 1) + h >= prow) continue;
              if (d.kind == KIND_V) tv[h] = in_at(qix[r], n);
              else if (d.kind == KIND_U && c == 1) tv[h] = *out_ptr(qix[r], n);
            }
          };
          load_terms(half * 16, pre);
          if (!failed && !wait_abortable(done, passes & 1, limit_ns, abortp)) fail();
          if (__any_sync(0xffffffffu, failed)) failed = true;  // warp-uniform from here (tcgen05.ld)
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          if (!failed) {
            const int nacc = min(NACC, nkc);  // main accumulators written in this pass
            for (int c0 = half * 16; c0 < nreal; c0 += 32) {
              load_terms(c0 + 32, nxt);
              const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
              uint32_t v[16], w[16];
              float acc[16];
              tmem_ld16(v, taddr);
              tmem_ld16(w, taddr + D_CORR);
              asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
              for (int e = 0; e < 16; ++e) acc[e] = __uint_as_float(v[e]);
              for (int a = 1; a < nacc; ++a) {  // the other main accumulators, in order
                tmem_ld16(v, taddr + (uint32_t)a * NH);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[e] += __uint_as_float(v[e]);
              }
#pragma unroll
              for (int e = 0; e < 16; ++e) acc[e] += __uint_as_float(w[e]);
              if (n < R) {
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                  const int r = r0 + (c0 >> 1) + h;  // complex output row of the block
                  if ((c0 >> 1) + h >= prow) break;
                  const float2 res = make_float2(acc[2 * h] + pre[h].x, acc[2 * h + 1] + pre[h].y);
                  if (d.kind == KIND_U) *out_ptr(qix[r], n) = res;  // block 1: pre = block 0's term
                  else *out_ptr((c ? len_o0 : 0) + r, n) = res;
                }
              }
#pragma unroll
              for (int h = 0; h < 8; ++h) pre[h] = nxt[h];
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(tfree);  // the next pass's MMAs may overwrite the accumulators
        }
      }
    }
  }
  if (failed && lane == 0) atomicOr(status, 1);
  // the last MMAs must have completed before the accumulators and stages are released
  if (mma_warp && lane == 0 && issued > 0) {
    const uint64_t t0 = gtimer();
    while (!try_wait(&empty[(issued - 1) % NSTAGE], ((issued - 1) / NSTAGE) & 1) && gtimer() - t0 < limit_ns) {
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace tc

// the 3xTF32 apply of all levels (forward); returns EUNSUPPORTED if a block is too large. With
// wide_middle the middle factor S^h runs on the CUDA cores in FP64 or double-float instead.
idbf_status apply_tf32x3(Plan* p, const void* x, void* y, int64_t R, int64_t ld, cudaStream_t st, bool wide_middle) {
  if (p->uneven) return IDBF_EUNSUPPORTED;  // leaves of n0 points only
  for (int l = 0; l <= p->L; ++l) {
    if (wide_middle && l == p->hV) continue;
    if (p->lv[l].max_rows > tc::MAXROWS || p->lv[l].max_cols > tc::GIXCAP) return IDBF_EUNSUPPORTED;
  }
  IDBF_CUDA_TRY(cudaFuncSetAttribute(tc::k_level_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM));
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  float2* ws0 = (float2*)p->d_ws;
  float2* ws1 = (float2*)((char*)p->d_ws + (size_t)p->max_seg_total * R * 16);
  float2* wb[2] = {ws0, ws1};
  for (int l = 0; l <= p->L; ++l) {
    const DevLevel d = p->level(l);
    const float2* win = l > 0 ? wb[(l - 1) & 1] : nullptr;
    float2* wout = l < p->L ? wb[l & 1] : nullptr;
    if (wide_middle && l == p->hV) {  // h_V >= 1: both sides are workspace boundaries
      const idbf_status s = apply_middle_wide(p, win, wout, R, st);
      if (s != IDBF_OK) return s;
      continue;
    }
    const unsigned ctas = (unsigned)std::min<int64_t>(p->m, sms);
    tc::k_level_tc<<<ctas, tc::NT + 32, tc::SMEM, st>>>(d, (const float2*)p->lmat[IDBF_STORE_C64][l], (const float2*)x, ld,
                                                  (float2*)y, ld, win, wout, (int)R, p->d_status, p->wait_limit_ns,
                                                  p->tc_split_mode);
    IDBF_CUDA_TRY(cudaGetLastError());
  }
  return IDBF_OK;
}

}  // namespace idbf
