// Multi-right-hand-side apply on the tensor cores (tcgen05, kind::tf32, split precision).
//
// With R right-hand sides every butterfly block product M_c G (M_c: rows x cols complex, G:
// cols x R) becomes a dense GEMM (Eq. 1 applied to a block of vectors). The complex product is
// embedded in real arithmetic with interleaved real / imaginary parts and computed transposed,
// D^T = G^T M_c^T, so that the tensor core's M dimension is 128 right-hand sides and its N
// dimension the 2 rows real output rows of the block (accumulators in TMEM, up to 384 columns):
//   A (M = 128 rhs x K = 2 cols):  A(n, 2k) = Re G(k, n),  A(n, 2k+1) = Im G(k, n)
//   B (N = 2 rows x K = 2 cols):   B(2r, 2k) = Re M(r,k), B(2r, 2k+1) = -Im M(r,k),
//                                  B(2r+1, 2k) = Im M(r,k), B(2r+1, 2k+1) = Re M(r,k)
//   D (128 x 2 rows):              D(n, 2r) = Re (M G)(r, n), D(n, 2r+1) = Im (M G)(r, n).
// Split precision (3xTF32, Ootomo and Yokota, "Recovering single precision accuracy from Tensor
// Cores while surpassing the FP32 theoretical peak performance", IJHPCA 2022): x = x_hi + x_lo with
// x_hi = rna_tf32(x), x_lo = x - x_hi, and A B ~ A_hi B_hi + (A_hi B_lo + A_lo B_hi). The main
// product and the two correction products go to separate TMEM accumulators (the correction terms
// are ~2^-11 of the main ones and lose their low bits when added into the main accumulator) and
// are summed in FP32 in the epilogue. The output rows of a block are covered in passes of at most
// 192 real rows so that both accumulators fit in TMEM. Operands are staged by the CTA's warps
// into shared memory in the K-major, no-swizzle canonical layout (8-row x 16-byte core
// matrices), three stages over K with the next chunk's global loads issued before the current
// chunk is written; one thread issues the MMAs and tcgen05.commit on an mbarrier tracks their
// completion.
#include <cuda_runtime.h>

#include <algorithm>

#include "idbf_internal.h"

namespace idbf {
namespace tc {

constexpr int NT = 256;          // threads per CTA (8 warps)
constexpr int MR = 128;          // right-hand sides per tile (MMA M)
constexpr int KC = 8;            // complex columns per staged chunk (16 real K)
constexpr int NH = 192;          // real output rows per pass (MMA N <= 192; two passes cover 384)
constexpr int MAXROWS = NH;      // complex rows per block supported (2 passes x 96)
constexpr uint32_t SBO = 128;    // byte step between 8-row core-matrix groups
constexpr uint32_t A_BYTES = MR * 2 * KC * 4;     // 8 KB
constexpr uint32_t B_BYTES = NH * 2 * KC * 4;     // 12 KB
constexpr uint32_t LBO_A = (MR / 8) * 128;        // byte step between 4-element K groups
constexpr uint32_t LBO_B = (NH / 8) * 128;
constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;  // hi and lo of both operands: 40 KB
constexpr int NSTAGE = 3;
constexpr size_t SMEM = NSTAGE * (size_t)STAGE + 64;   // stages + barriers
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t D_CORR = 256;                       // TMEM column of the correction accumulator
constexpr int A_PER_T = MR * KC / NT;                  // 4 complex A values per thread per chunk
constexpr int B_PER_T = (NH / 2) * KC / NT;            // 3 complex B values per thread per chunk

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
__device__ __forceinline__ bool wait_bounded(uint64_t* b, uint32_t parity, uint64_t limit_ns) {
  if (try_wait(b, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t n = 1;; ++n) {
    if (try_wait(b, parity)) return true;
    if ((n & 255) == 0 && gtimer() - t0 > limit_ns) return false;
  }
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
// two consecutive K elements (2k', 2k'+1) of one row: one 8-byte store per split; the lo part
// is rounded to TF32 as well (rna) when round_lo is set, else left for the hardware to narrow
__device__ __forceinline__ void put2(unsigned char* hi, unsigned char* lo, uint32_t off, float a, float b, int round_lo) {
  const float ah = tf32_hi(a), bh = tf32_hi(b);
  *(float2*)(hi + off) = make_float2(ah, bh);
  float al = a - ah, bl = b - bh;
  if (round_lo) { al = tf32_hi(al); bl = tf32_hi(bl); }
  *(float2*)(lo + off) = make_float2(al, bl);
}

// One launch per level; persistent CTAs over nodes. x / y: user blocks (column-major, ld);
// win / wout: workspace boundaries, element e of a segment at (off + e) * R + rhs.
__global__ void __launch_bounds__(NT, 1)
    k_level_tc(DevLevel d, const float2* __restrict__ mat, const float2* __restrict__ x, int64_t ldx,
               float2* __restrict__ y, int64_t ldy, const float2* __restrict__ win, float2* __restrict__ wout, int R,
               int* __restrict__ status, uint64_t limit_ns, int split_mode) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base;
  uint64_t* bars = (uint64_t*)(sm + NSTAGE * STAGE);  // [0, NSTAGE): stage free; [NSTAGE]: pass done
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i <= NSTAGE; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(&bars[i])), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  uint32_t kcg = 0, passes = 0;  // chunks and passes issued by this CTA (mbarrier phases)
  bool failed = false;
  const int nrt = (R + MR - 1) / MR;

  for (int64_t j = blockIdx.x; j < d.m && !failed; j += gridDim.x) {
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
    if (d.kind == KIND_U) {
      // t[q_0] = in_0 (t[p_0] comes from the block-0 products); q_1 part added with block 1
      for (int i = tid; i < l0 * R; i += NT) *out_ptr(ix0[i / R], i % R) = in_at(i / R, i % R);
      __syncthreads();
    }
    for (int c = 0; c < 2 && !failed; ++c) {
      const int rows = d.rows[2 * j + c], cols = d.cols[2 * j + c];
      const int32_t* ix = c ? ix1 : ix0;
      const float2* M = mat + d.moff[2 * j + c];
      // column k of the gathered operand G: which element of the node input
      auto g_elem = [&](int k) -> int {
        if (d.kind == KIND_V) return ix[rows + k];
        if (d.kind == KIND_U) return (c ? l0 : 0) + k;
        return k;  // S: all of concat(in_0, in_1)
      };
      if (d.kind == KIND_U && c == 1) {
        __syncthreads();
        for (int i = tid; i < l1 * R; i += NT) {
          float2* q = out_ptr(ix1[i / R], i % R);
          const float2 a = *q, b = in_at(l0 + i / R, i % R);
          *q = make_float2(a.x + b.x, a.y + b.y);
        }
        __syncthreads();
      }
      if (rows == 0) continue;
      if (cols == 0) {  // V block that keeps every column: out = u[q]
        for (int i = tid; i < rows * R; i += NT) {
          const int r = i / R, n = i % R;
          *out_ptr((c ? len_o0 : 0) + r, n) = in_at(ix[r], n);
        }
        continue;
      }
      const int nkc = (cols + KC - 1) / KC;
      const int npass = rows > NH / 2 ? 2 : 1;
      for (int rt = 0; rt < nrt && !failed; ++rt) {
        const int nr = min(MR, R - rt * MR);
        for (int ps = 0; ps < npass && !failed; ++ps) {
          const int r0 = ps * (NH / 2);                       // first complex row of the pass
          const int prow = min(NH / 2, rows - r0);            // complex rows of the pass
          const int nreal = (2 * prow + 15) & ~15;            // MMA N (multiple of 16)
          // registers for one chunk's global operands (prefetched one chunk ahead)
          float2 av[A_PER_T], bv[B_PER_T];
          auto load = [&](int kc) {
#pragma unroll
            for (int t = 0; t < A_PER_T; ++t) {
              const int i = tid + t * NT, kk = i / MR, n = i % MR, k = kc * KC + kk;
              av[t] = (k < cols && n < nr) ? in_at(g_elem(k), rt * MR + n) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int t = 0; t < B_PER_T; ++t) {
              const int i = tid + t * NT, kk = i / (NH / 2), r = i % (NH / 2), k = kc * KC + kk;
              bv[t] = (k < cols && r < prow) ? M[(int64_t)k * rows + r0 + r] : make_float2(0.f, 0.f);
            }
          };
          load(0);
          for (int kc = 0; kc < nkc; ++kc, ++kcg) {
            const int s = kcg % NSTAGE;
            unsigned char* Ah = sm + (size_t)s * STAGE;
            unsigned char* Al = Ah + A_BYTES;
            unsigned char* Bh = Al + A_BYTES;
            unsigned char* Bl = Bh + B_BYTES;
            // the MMAs that last read stage s must be done
            if (!wait_bounded(&bars[s], ((kcg / NSTAGE) & 1) ^ 1, limit_ns)) { failed = true; break; }
#pragma unroll
            for (int t = 0; t < A_PER_T; ++t) {
              const int i = tid + t * NT, kk = i / MR, n = i % MR;
              put2(Ah, Al, koff(n, 2 * kk, LBO_A), av[t].x, av[t].y, split_mode >= 1);
            }
#pragma unroll
            for (int t = 0; t < B_PER_T; ++t) {
              const int i = tid + t * NT, kk = i / (NH / 2), r = i % (NH / 2);
              put2(Bh, Bl, koff(2 * r, 2 * kk, LBO_B), bv[t].x, -bv[t].y, split_mode >= 1);
              put2(Bh, Bl, koff(2 * r + 1, 2 * kk, LBO_B), bv[t].y, bv[t].x, split_mode >= 1);
            }
            if (kc + 1 < nkc) load(kc + 1);  // in flight while this chunk's MMAs run
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              const uint32_t id = idesc_tf32((uint32_t)nreal, MR);
              for (int ks = 0; ks < 2; ++ks) {  // K = 8 real per MMA: two 4-element core groups
                const uint32_t ao = 2 * ks * LBO_A, bo = 2 * ks * LBO_B;
                const uint64_t ah = sdesc(sa(Ah) + ao, LBO_A, SBO), al = sdesc(sa(Al) + ao, LBO_A, SBO);
                const uint64_t bh = sdesc(sa(Bh) + bo, LBO_B, SBO), bl = sdesc(sa(Bl) + bo, LBO_B, SBO);
                const uint32_t first = (kc == 0 && ks == 0) ? 0u : 1u;
                mma_tf32(tmem, ah, bh, id, first);             // main: hi * hi
                mma_tf32(tmem + D_CORR, ah, bl, id, first);    // corrections: hi * lo + lo * hi
                mma_tf32(tmem + D_CORR, al, bh, id, 1u);
                if (split_mode == 2) mma_tf32(tmem + D_CORR, al, bl, id, 1u);
              }
              commit(&bars[s]);
              if (kc == nkc - 1) commit(&bars[NSTAGE]);
            }
          }
          if (failed) break;
          // epilogue: lane quadrant of warp w % 4 = 32 rhs; warps w and w + 4 split the columns
          if (!wait_bounded(&bars[NSTAGE], passes & 1, limit_ns)) { failed = true; break; }
          ++passes;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int q = warp & 3, half = warp >> 2;
          const int n = rt * MR + q * 32 + lane;
          for (int c0 = half * 16; c0 < nreal; c0 += 32) {
            uint32_t v[16], w[16];
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]),
                  "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15])
                : "r"(taddr + D_CORR));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (n >= R) continue;
#pragma unroll
            for (int h = 0; h < 8; ++h) {
              const int r = r0 + (c0 >> 1) + h;  // complex output row of the block
              if ((c0 >> 1) + h >= prow) break;
              const float2 res = make_float2(__uint_as_float(v[2 * h]) + __uint_as_float(w[2 * h]),
                                             __uint_as_float(v[2 * h + 1]) + __uint_as_float(w[2 * h + 1]));
              if (d.kind == KIND_V) {
                const float2 uq = in_at(ix[r], n);
                *out_ptr((c ? len_o0 : 0) + r, n) = make_float2(res.x + uq.x, res.y + uq.y);
              } else if (d.kind == KIND_S) {
                *out_ptr((c ? len_o0 : 0) + r, n) = res;
              } else {
                float2* p = out_ptr(ix[(c ? l1 : l0) + r], n);
                if (c == 0) *p = res;
                else { const float2 a = *p; *p = make_float2(a.x + res.x, a.y + res.y); }
              }
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncthreads();  // TMEM read out before the next pass's MMAs overwrite it
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
      }
    }
    __syncthreads();
  }
  if (failed && (tid & 31) == 0) atomicOr(status, 1);
  // the last MMAs must have completed before the accumulators are released
  if (tid == 0 && kcg > 0) {
    const uint64_t t0 = gtimer();
    while (!try_wait(&bars[(kcg - 1) % NSTAGE], ((kcg - 1) / NSTAGE) & 1) && gtimer() - t0 < limit_ns) {
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace tc

// the 3xTF32 apply of all levels (forward); returns EUNSUPPORTED if a block is too large
idbf_status apply_tf32x3(Plan* p, const void* x, void* y, int64_t R, int64_t ld, cudaStream_t st) {
  for (int l = 0; l <= p->L; ++l)
    if (p->lv[l].max_rows > tc::MAXROWS) return IDBF_EUNSUPPORTED;
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
    const unsigned ctas = (unsigned)std::min<int64_t>(p->m, sms);
    tc::k_level_tc<<<ctas, tc::NT, tc::SMEM, st>>>(d, (const float2*)p->lmat[IDBF_STORE_C64][l], (const float2*)x, ld,
                                                  (float2*)y, ld, win, wout, (int)R, p->d_status, p->wait_limit_ns,
                                                  p->tc_split_mode);
    IDBF_CUDA_TRY(cudaGetLastError());
  }
  return IDBF_OK;
}

}  // namespace idbf
