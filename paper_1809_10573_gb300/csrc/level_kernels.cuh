// Arithmetic policies and the per-node forward body shared by the per-level kernels (apply.cu)
// and the persistent batch kernel (batch.cu). Three policies:
//   FP64P - complex128 factors and vectors, FP64 FMA;
//   DF64P - factors stored as double-float pairs (hi, lo) of binary32, complex128 vectors;
//           products formed exactly with FMA (Dekker's product), sums accumulated with Knuth's
//           TwoSum in chunks (the compensated dot product of Ogita, Rump and Oishi, "Accurate sum
//           and dot product", SIAM J. Sci. Comput. 26, 2005) and folded into a normalised
//           double-float total (Joldes, Muller and Popescu, "Tight and rigorous error bounds for
//           basic building blocks of double-word arithmetic", ACM TOMS 44, 2017);
//   FP32P - complex64 factors and vectors, FP32 FMA.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "idbf_internal.h"

namespace idbf {

// ---------------------------------------------------------------------------------------------
// arithmetic policies
struct FP64P {
  using mat_t = double2;
  using vec_t = double2;
  using gv_t = double2;
  struct acc_t { double re, im; };
  static constexpr int CHUNK = 16;
  __device__ static __forceinline__ mat_t ld(const mat_t* p) { return __ldcs(p); }
  __device__ static __forceinline__ gv_t cvt(vec_t v) { return v; }
  __device__ static __forceinline__ void init(acc_t& a) { a.re = 0.0; a.im = 0.0; }
  __device__ static __forceinline__ void mac(acc_t& a, const mat_t& m, const gv_t& g) {
    a.re = fma(m.x, g.x, a.re);
    a.re = fma(-m.y, g.y, a.re);
    a.im = fma(m.x, g.y, a.im);
    a.im = fma(m.y, g.x, a.im);
  }
  __device__ static __forceinline__ void macc(acc_t& a, const mat_t& m, const gv_t& g) {  // conj(m) g
    a.re = fma(m.x, g.x, a.re);
    a.re = fma(m.y, g.y, a.re);
    a.im = fma(m.x, g.y, a.im);
    a.im = fma(-m.y, g.x, a.im);
  }
  __device__ static __forceinline__ void flush(acc_t&) {}
  __device__ static __forceinline__ vec_t fin(const acc_t& a) { return make_double2(a.re, a.im); }
  __device__ static __forceinline__ void warp_sum(acc_t& a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a.re += __shfl_xor_sync(0xffffffffu, a.re, o);
      a.im += __shfl_xor_sync(0xffffffffu, a.im, o);
    }
  }
  __device__ static __forceinline__ vec_t add(vec_t a, vec_t b) { return make_double2(a.x + b.x, a.y + b.y); }
  __device__ static __forceinline__ vec_t zero() { return make_double2(0.0, 0.0); }
  using part_t = double2;  // a flushed accumulator, for combining partial sums
  __device__ static __forceinline__ part_t part(const acc_t& a) { return make_double2(a.re, a.im); }
  __device__ static __forceinline__ void combine(acc_t& a, const part_t& b) { a.re += b.x; a.im += b.y; }
};

struct FP32P {
  using mat_t = float2;
  using vec_t = float2;
  using gv_t = float2;
  struct acc_t { float re, im; };
  static constexpr int CHUNK = 16;
  __device__ static __forceinline__ mat_t ld(const mat_t* p) { return __ldcs(p); }
  __device__ static __forceinline__ gv_t cvt(vec_t v) { return v; }
  __device__ static __forceinline__ void init(acc_t& a) { a.re = 0.f; a.im = 0.f; }
  __device__ static __forceinline__ void mac(acc_t& a, const mat_t& m, const gv_t& g) {
    a.re = fmaf(m.x, g.x, a.re);
    a.re = fmaf(-m.y, g.y, a.re);
    a.im = fmaf(m.x, g.y, a.im);
    a.im = fmaf(m.y, g.x, a.im);
  }
  __device__ static __forceinline__ void macc(acc_t& a, const mat_t& m, const gv_t& g) {
    a.re = fmaf(m.x, g.x, a.re);
    a.re = fmaf(m.y, g.y, a.re);
    a.im = fmaf(m.x, g.y, a.im);
    a.im = fmaf(-m.y, g.x, a.im);
  }
  __device__ static __forceinline__ void flush(acc_t&) {}
  __device__ static __forceinline__ vec_t fin(const acc_t& a) { return make_float2(a.re, a.im); }
  __device__ static __forceinline__ void warp_sum(acc_t& a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a.re += __shfl_xor_sync(0xffffffffu, a.re, o);
      a.im += __shfl_xor_sync(0xffffffffu, a.im, o);
    }
  }
  __device__ static __forceinline__ vec_t add(vec_t a, vec_t b) { return make_float2(a.x + b.x, a.y + b.y); }
  __device__ static __forceinline__ vec_t zero() { return make_float2(0.f, 0.f); }
  using part_t = float2;
  __device__ static __forceinline__ part_t part(const acc_t& a) { return make_float2(a.re, a.im); }
  __device__ static __forceinline__ void combine(acc_t& a, const part_t& b) { a.re += b.x; a.im += b.y; }
};

// ---- double-float helpers (round-to-nearest intrinsics: never contracted into FMA) ----------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// (hi, lo) += (s, c): the "sloppy" double-word addition (TwoSum of the high parts, the low
// parts added, then renormalised with Fast2Sum).
__device__ __forceinline__ void dw_accumulate(float& hi, float& lo, float s, float c) {
  float t, e;
  two_sum(hi, s, t, e);
  e = __fadd_rn(e, __fadd_rn(lo, c));
  fast_two_sum(t, e, hi, lo);
}
// s + c += a * b for double-float a = (ah, al), b = (bh, bl): the product of the high parts is
// split exactly (p + e, e = fma(ah, bh, -p)); the cross terms ah bl + al bh enter the
// compensation; p enters the running sum through TwoSum whose error also goes to c.
__device__ __forceinline__ void dot2_step(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  float t, err;
  two_sum(s, p, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

struct DF64P {
  using mat_t = float4;   // (re_hi, re_lo, im_hi, im_lo)
  using vec_t = double2;
  using gv_t = float4;
  struct acc_t { float sr, cr, si, ci, hr, lr, hi, li; };
  static constexpr int CHUNK = 16;
  __device__ static __forceinline__ mat_t ld(const mat_t* p) { return __ldcs(p); }
  __device__ static __forceinline__ gv_t cvt(vec_t v) {
    const float rh = (float)v.x, ih = (float)v.y;
    return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
  }
  __device__ static __forceinline__ void init(acc_t& a) {
    a.sr = a.cr = a.si = a.ci = 0.f;
    a.hr = a.lr = a.hi = a.li = 0.f;
  }
  __device__ static __forceinline__ void mac(acc_t& a, const mat_t& m, const gv_t& g) {
    dot2_step(a.sr, a.cr, m.x, m.y, g.x, g.y);
    dot2_step(a.sr, a.cr, -m.z, -m.w, g.z, g.w);
    dot2_step(a.si, a.ci, m.x, m.y, g.z, g.w);
    dot2_step(a.si, a.ci, m.z, m.w, g.x, g.y);
  }
  __device__ static __forceinline__ void macc(acc_t& a, const mat_t& m, const gv_t& g) {
    dot2_step(a.sr, a.cr, m.x, m.y, g.x, g.y);
    dot2_step(a.sr, a.cr, m.z, m.w, g.z, g.w);
    dot2_step(a.si, a.ci, m.x, m.y, g.z, g.w);
    dot2_step(a.si, a.ci, -m.z, -m.w, g.x, g.y);
  }
  __device__ static __forceinline__ void flush(acc_t& a) {
    dw_accumulate(a.hr, a.lr, a.sr, a.cr);
    dw_accumulate(a.hi, a.li, a.si, a.ci);
    a.sr = a.cr = a.si = a.ci = 0.f;
  }
  __device__ static __forceinline__ vec_t fin(const acc_t& a) {
    return make_double2((double)a.hr + (double)a.lr, (double)a.hi + (double)a.li);
  }
  __device__ static __forceinline__ void warp_sum(acc_t& a) {
    flush(a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float hr = __shfl_xor_sync(0xffffffffu, a.hr, o), lr = __shfl_xor_sync(0xffffffffu, a.lr, o);
      const float hi = __shfl_xor_sync(0xffffffffu, a.hi, o), li = __shfl_xor_sync(0xffffffffu, a.li, o);
      dw_accumulate(a.hr, a.lr, hr, lr);
      dw_accumulate(a.hi, a.li, hi, li);
    }
  }
  __device__ static __forceinline__ vec_t add(vec_t a, vec_t b) { return make_double2(a.x + b.x, a.y + b.y); }
  __device__ static __forceinline__ vec_t zero() { return make_double2(0.0, 0.0); }
  using part_t = float4;  // (re_hi, re_lo, im_hi, im_lo) of a flushed accumulator
  __device__ static __forceinline__ part_t part(const acc_t& a) { return make_float4(a.hr, a.lr, a.hi, a.li); }
  __device__ static __forceinline__ void combine(acc_t& a, const part_t& b) {
    dw_accumulate(a.hr, a.lr, b.x, b.y);
    dw_accumulate(a.hi, a.li, b.z, b.w);
  }
};

// The middle factor S^h of the split-precision tensor form (IDBF_MODE_TF32X3_S64): complex64
// vectors on both sides, as on the tensor-core levels around it, with the products and sums in
// FP64 (C128 storage of S^h) or in double-float (DF64 storage). Each FP32 input is exact in the
// wider format; the output is rounded to FP32 once.
struct FP64S32P : FP64P {
  using vec_t = float2;
  __device__ static __forceinline__ gv_t cvt(vec_t v) { return make_double2((double)v.x, (double)v.y); }
  __device__ static __forceinline__ vec_t fin(const acc_t& a) { return make_float2((float)a.re, (float)a.im); }
  __device__ static __forceinline__ vec_t add(vec_t a, vec_t b) { return make_float2(a.x + b.x, a.y + b.y); }
  __device__ static __forceinline__ vec_t zero() { return make_float2(0.f, 0.f); }
};
struct DF64S32P : DF64P {
  using vec_t = float2;
  __device__ static __forceinline__ gv_t cvt(vec_t v) { return make_float4(v.x, 0.f, v.y, 0.f); }
  __device__ static __forceinline__ vec_t fin(const acc_t& a) {
    return make_float2((float)((double)a.hr + (double)a.lr), (float)((double)a.hi + (double)a.li));
  }
  __device__ static __forceinline__ vec_t add(vec_t a, vec_t b) { return make_float2(a.x + b.x, a.y + b.y); }
  __device__ static __forceinline__ vec_t zero() { return make_float2(0.f, 0.f); }
};

// Vectors between levels of the single-vector forward path. With DF set the double-float
// policy keeps them in its own format, (re_hi, re_lo, im_hi, im_lo) floats (16 bytes, like
// complex128), so that gathering a level's operands, adding its pass-through terms and writing its
// outputs take no FP64 arithmetic (GB300 issues FP64 at a small fraction of the FP32 rate); only
// level 0 converts the complex128 x and level L the complex128 y. Otherwise the boundary vectors
// are the policy's vec_t.
template <class P, bool DF>
struct Bnd {
  using b_t = typename P::vec_t;
  __device__ static __forceinline__ b_t of_v(typename P::vec_t v) { return v; }
  __device__ static __forceinline__ typename P::vec_t v_of(b_t b) { return b; }
  __device__ static __forceinline__ typename P::gv_t g_of(b_t b) { return P::cvt(b); }
  __device__ static __forceinline__ b_t of_acc(const typename P::acc_t& a) { return P::fin(a); }
  __device__ static __forceinline__ b_t add(b_t a, b_t b) { return P::add(a, b); }
  __device__ static __forceinline__ b_t zero() { return P::zero(); }
};
template <>
struct Bnd<DF64P, true> {
  using b_t = float4;
  __device__ static __forceinline__ b_t of_v(double2 v) { return DF64P::cvt(v); }  // exact split
  __device__ static __forceinline__ double2 v_of(b_t b) {  // exact: 48 bits in a double
    return make_double2((double)b.x + (double)b.y, (double)b.z + (double)b.w);
  }
  __device__ static __forceinline__ float4 g_of(b_t b) { return b; }
  // a flushed accumulator: its (hi, lo) pairs, of the value fin() rounds exactly into a double
  __device__ static __forceinline__ b_t of_acc(const DF64P::acc_t& a) { return DF64P::part(a); }
  __device__ static __forceinline__ b_t add(b_t a, b_t b) {
    dw_accumulate(a.x, a.y, b.x, b.y);
    dw_accumulate(a.z, a.w, b.z, b.w);
    return a;
  }
  __device__ static __forceinline__ b_t zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
// the single-vector forward bodies of the double-float policy use its own boundary format
template <class P, int RB, int RPT>
constexpr bool df_boundary() {
  return std::is_same<P, DF64P>::value && RB == 1 && RPT == 0;
}
static_assert(sizeof(Bnd<DF64P, true>::b_t) == sizeof(DF64P::vec_t), "boundary elements keep their size");

template <class P> constexpr int fmt_of();
template <> constexpr int fmt_of<FP64P>() { return IDBF_STORE_C128; }
template <> constexpr int fmt_of<DF64P>() { return IDBF_STORE_DF64; }
template <> constexpr int fmt_of<FP32P>() { return IDBF_STORE_C64; }
template <> constexpr int fmt_of<FP64S32P>() { return IDBF_STORE_C128; }
template <> constexpr int fmt_of<DF64S32P>() { return IDBF_STORE_DF64; }

// ---------------------------------------------------------------------------------------------
// addressing of a node's input and output segments
struct Seg {
  int64_t base;  // element offset of element 0, rhs 0
  int64_t es;    // element stride
  int64_t rs;    // rhs stride
  int len;
};

template <class V>
struct IO {
  const V* x;  // user input (forward: level 0; adjoint: level L)
  int64_t ldx;
  V* y;        // user output (forward: level L; adjoint: level 0)
  int64_t ldy;
  const V* win;  // workspace boundary read
  V* wout;       // workspace boundary written
  int R;
};

__device__ __forceinline__ int64_t out_seg_id(const DevLevel& d, int64_t j, int c) {
  return (j / d.H) * 2 * d.H + j % d.H + c * d.H;
}

// Phase 3 of fwd_node for RPT > 0 (see there). Threads take tasks (slice s, group q, row gr) with
// the row fastest, so a warp's loads of one column of a block are consecutive.
template <class P, int RB, int RPT>
__device__ __forceinline__ void block_products_split(const DevLevel& d, const typename P::mat_t* __restrict__ mat,
                                                     const typename P::gv_t* g, typename P::vec_t* res,
                                                     typename P::part_t* pbuf, int gcap, int rcap, int rows0,
                                                     int rows1, int cols0, int cols1, int64_t mo0, int64_t mo1,
                                                     int nrb) {
  using M = typename P::mat_t;
  using G = typename P::gv_t;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nrows = rows0 + rows1;
  const int ng = (nrb + RPT - 1) / RPT;
  const int tasks = nrows * ng;
  const int maxc = max(cols0, cols1);
  int S = 1;
  while (S < 8 && 2 * S * tasks <= nt && maxc >= 16 * S) S *= 2;
  for (int w = tid; w < tasks * S; w += nt) {
    const int s = w / tasks, rem = w - s * tasks;
    const int q = rem / nrows, gr = rem - q * nrows;
    const int c = gr >= rows0;
    const int r = c ? gr - rows0 : gr;
    const int rows = c ? rows1 : rows0;
    const int cols = c ? cols1 : cols0;
    const int cb = (cols * s) / S, ce = (cols * (s + 1)) / S;
    const M* Mc = mat + (c ? mo1 : mo0) + r;
    const G* gc = g + (d.kind == KIND_S ? 0 : c * gcap * RB) + q * RPT;
    typename P::acc_t acc[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) P::init(acc[k]);
    int jj = cb;
    for (; jj + P::CHUNK <= ce; jj += P::CHUNK) {
#pragma unroll 8
      for (int e = 0; e < P::CHUNK; ++e) {
        const M mv = P::ld(Mc + (int64_t)(jj + e) * rows);
#pragma unroll
        for (int k = 0; k < RPT; ++k) P::mac(acc[k], mv, gc[(jj + e) * RB + k]);
      }
#pragma unroll
      for (int k = 0; k < RPT; ++k) P::flush(acc[k]);
    }
    for (; jj < ce; ++jj) {
      const M mv = P::ld(Mc + (int64_t)jj * rows);
#pragma unroll
      for (int k = 0; k < RPT; ++k) P::mac(acc[k], mv, gc[jj * RB + k]);
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) P::flush(acc[k]);
    if (S == 1) {
#pragma unroll
      for (int k = 0; k < RPT; ++k) res[(c * rcap + r) * RB + q * RPT + k] = P::fin(acc[k]);
    } else {
#pragma unroll
      for (int k = 0; k < RPT; ++k) pbuf[(size_t)w * RPT + k] = P::part(acc[k]);
    }
  }
  if (S > 1) {
    __syncthreads();
    for (int i = tid; i < nrows * nrb; i += nt) {
      const int gr = i / nrb, rb = i - gr * nrb;
      const int q = rb / RPT, k = rb - q * RPT;
      const int rem = q * nrows + gr;
      typename P::acc_t a;
      P::init(a);
      for (int s = 0; s < S; ++s) P::combine(a, pbuf[(size_t)(s * tasks + rem) * RPT + k]);
      const int c = gr >= rows0;
      const int r = c ? gr - rows0 : gr;
      res[(c * rcap + r) * RB + rb] = P::fin(a);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// forward level kernel. Shared memory: u[max_in][RB] (inputs), g[2][gcap][RB] (gathered
// operands), res[2][rcap][RB] (block products), and for RPT > 0 a partial-sum buffer of
// blockDim.x * RPT part_t (fwd_node_smem gives the total). The row-ID accumulation t[|t|][RB]
// of a U level reuses g once the block products are done: |t| = |q_0| + |p_0| <= max_in +
// max_rows <= 2 gcap, and sizeof(vec_t) <= sizeof(gv_t).
// One node j of a level, right-hand sides r0 .. r0+RB-1, by the whole CTA (used by the per-level
// kernels and by the persistent batch kernel).
//
// The block products (phase 3) are mapped one of two ways:
//   RPT == 0: one thread per output row, all RB right-hand sides in registers;
//   RPT  > 0: one thread per (output row, group of RPT right-hand sides, column slice). When the
//             node has fewer (row, group) tasks than half the CTA, the columns are cut into
//             S = 2, 4 or 8 slices whose partial sums are combined through shared memory, so
//             that small blocks and single vectors still occupy the CTA.
template <class P, int RB, int RPT>
__host__ __device__ constexpr size_t fwd_node_smem(int max_in, int gcap, int rcap, int nthreads) {
  static_assert(sizeof(typename P::vec_t) <= sizeof(typename P::gv_t), "t reuses g");
  return (size_t)RB * (max_in * sizeof(typename P::vec_t) + 2 * gcap * sizeof(typename P::gv_t) +
                       2 * rcap * sizeof(typename P::vec_t)) +
         (RPT > 0 ? (size_t)nthreads * RPT * sizeof(typename P::part_t) : 0);
}

template <class P, int RB, int RPT = 0>
__device__ __forceinline__ void fwd_node(const DevLevel& d, const typename P::mat_t* __restrict__ mat,
                                         const IO<typename P::vec_t>& io, int gcap, int rcap, int max_in, int64_t j,
                                         int r0, unsigned char* smem) {
  static_assert(RPT == 0 || RB % RPT == 0, "RB must be a multiple of RPT");
  using V = typename P::vec_t;
  using G = typename P::gv_t;
  using M = typename P::mat_t;
  using BP = Bnd<P, df_boundary<P, RB, RPT>()>;
  using B = typename BP::b_t;
  V* u = (V*)smem;
  B* ub = (B*)u;  // the inputs of a level > 0, in the boundary format
  G* g = (G*)(u + (size_t)max_in * RB);
  B* res = (B*)(g + (size_t)2 * gcap * RB);
  B* t = (B*)g;  // phase 4 of a U level only, after the last read of g
  const B* winb = (const B*)io.win;
  B* woutb = (B*)io.wout;
  const int nrb = min(RB, io.R - r0);
  const int tid = threadIdx.x, nt = blockDim.x;

  // phase 1: inputs -> u
  int l0, l1;
  if (d.lev == 0) {
    l0 = leaf_len(d, j);
    l1 = 0;
    const int64_t x0 = leaf_start(d, j);
    for (int i = tid; i < l0 * RB; i += nt) {
      const int e = i / RB, rb = i % RB;
      u[i] = rb < nrb ? io.x[x0 + e + (int64_t)(r0 + rb) * io.ldx] : P::zero();
    }
  } else {
    l0 = d.in_len[2 * j];
    l1 = d.in_len[2 * j + 1];
    const int64_t o0 = d.in_off[2 * j], o1 = d.in_off[2 * j + 1];
    for (int i = tid; i < (l0 + l1) * RB; i += nt) {
      const int e = i / RB, rb = i % RB;
      const int64_t off = e < l0 ? o0 + e : o1 + (e - l0);
      ub[i] = rb < nrb ? winb[off * io.R + r0 + rb] : BP::zero();
    }
  }
  const bool lev0 = d.lev == 0;
  // gathered operand of input element e: level 0 converts x, later levels read the boundary
  auto gin = [&](int e) -> G { return lev0 ? P::cvt(u[e]) : BP::g_of(ub[e]); };
  // pass-through term of input element e, in the boundary format
  auto bin = [&](int e) -> B { return lev0 ? BP::of_v(u[e]) : ub[e]; };
  const int rows0 = d.rows[2 * j], rows1 = d.rows[2 * j + 1];
  const int cols0 = d.cols[2 * j], cols1 = d.cols[2 * j + 1];
  const int64_t mo0 = d.moff[2 * j], mo1 = d.moff[2 * j + 1];
  const int32_t* ix0 = d.idx + d.ioff[2 * j];
  const int32_t* ix1 = d.idx + d.ioff[2 * j + 1];
  __syncthreads();

  // phase 2: gathered operands
  if (d.kind == KIND_V) {
    for (int i = tid; i < cols0 * RB; i += nt) g[i] = gin(ix0[rows0 + i / RB] * RB + i % RB);
    for (int i = tid; i < cols1 * RB; i += nt) g[gcap * RB + i] = gin(ix1[rows1 + i / RB] * RB + i % RB);
  } else if (d.kind == KIND_S) {
    for (int i = tid; i < (l0 + l1) * RB; i += nt) g[i] = gin(i);
  } else {
    for (int i = tid; i < (l0 + l1) * RB; i += nt) g[i < l0 * RB ? i : gcap * RB + i - l0 * RB] = gin(i);
  }
  __syncthreads();

  // phase 3: block products
  if constexpr (RPT > 0) {
    block_products_split<P, RB, RPT>(d, mat, g, res, (typename P::part_t*)(res + (size_t)2 * rcap * RB), gcap, rcap,
                                     rows0, rows1, cols0, cols1, mo0, mo1, nrb);
  } else {
  for (int gr = tid; gr < rows0 + rows1; gr += nt) {
    const int c = gr >= rows0;
    const int r = c ? gr - rows0 : gr;
    const int rows = c ? rows1 : rows0;
    const int cols = c ? cols1 : cols0;
    const M* Mc = mat + (c ? mo1 : mo0) + r;
    const G* gc = g + (d.kind == KIND_S ? 0 : c * gcap * RB);
    typename P::acc_t acc[RB];
#pragma unroll
    for (int rb = 0; rb < RB; ++rb) P::init(acc[rb]);
    int jj = 0;
    for (; jj + P::CHUNK <= cols; jj += P::CHUNK) {
#pragma unroll 4
      for (int q = 0; q < P::CHUNK; ++q) {
        const M mv = P::ld(Mc + (int64_t)(jj + q) * rows);
#pragma unroll
        for (int rb = 0; rb < RB; ++rb) P::mac(acc[rb], mv, gc[(jj + q) * RB + rb]);
      }
#pragma unroll
      for (int rb = 0; rb < RB; ++rb) P::flush(acc[rb]);
    }
    for (; jj < cols; ++jj) {
      const M mv = P::ld(Mc + (int64_t)jj * rows);
#pragma unroll
      for (int rb = 0; rb < RB; ++rb) P::mac(acc[rb], mv, gc[jj * RB + rb]);
    }
#pragma unroll
    for (int rb = 0; rb < RB; ++rb) {
      P::flush(acc[rb]);
      res[(c * rcap + r) * RB + rb] = BP::of_acc(acc[rb]);
    }
  }
  }
  __syncthreads();

  // phase 4: combine and write
  if (d.kind != KIND_U) {
    for (int c = 0; c < 2; ++c) {
      const int rows = c ? rows1 : rows0;
      const int32_t* q = c ? ix1 : ix0;
      const int64_t s = out_seg_id(d, j, c);
      const int64_t ob = d.out_off[s];
      for (int i = tid; i < rows * nrb; i += nt) {
        const int r = i / nrb, rb = i % nrb;
        B v = res[(c * rcap + r) * RB + rb];
        if (d.kind == KIND_V) v = BP::add(v, bin(q[r] * RB + rb));
        woutb[(ob + r) * io.R + r0 + rb] = v;
      }
    }
    return;
  }
  // row-ID level: t[q_c] += in_c, t[p_c] += res_c. q_0 and p_0 partition t, so block 0
  // initialises every position once; block 1 (q_1, p_1 also a partition) then adds.
  const int tl = l0 + rows0;  // |t| = |q_0| + |p_0|
  for (int i = tid; i < l0 * RB; i += nt) t[ix0[i / RB] * RB + i % RB] = bin(i);
  for (int i = tid; i < rows0 * RB; i += nt) t[ix0[l0 + i / RB] * RB + i % RB] = res[i];
  __syncthreads();
  for (int i = tid; i < l1 * RB; i += nt) {
    B* dst = &t[ix1[i / RB] * RB + i % RB];
    *dst = BP::add(*dst, bin(l0 * RB + i));
  }
  for (int i = tid; i < rows1 * RB; i += nt) {
    B* dst = &t[ix1[l1 + i / RB] * RB + i % RB];
    *dst = BP::add(*dst, res[rcap * RB + i]);
  }
  __syncthreads();
  if (d.lev == d.L) {
    const int64_t y0 = leaf_start(d, j);
    for (int i = tid; i < tl * nrb; i += nt) {
      const int e = i / nrb, rb = i % nrb;
      io.y[y0 + e + (int64_t)(r0 + rb) * io.ldy] = BP::v_of(t[e * RB + rb]);
    }
  } else {
    const int64_t s0 = out_seg_id(d, j, 0), s1 = out_seg_id(d, j, 1);
    const int len0 = d.out_len[s0];
    const int64_t b0 = d.out_off[s0], b1 = d.out_off[s1];
    for (int i = tid; i < tl * nrb; i += nt) {
      const int e = i / nrb, rb = i % nrb;
      const int64_t off = e < len0 ? b0 + e : b1 + (e - len0);
      woutb[off * io.R + r0 + rb] = t[e * RB + rb];
    }
  }
}


// ---------------------------------------------------------------------------------------------
// Tiled forward node for several right-hand sides (FP32 and FP64 policies, whose operands need
// no conversion). One CTA computes node j for right-hand sides r0 .. r0+nrb-1 (nrb <= RB):
//   - the node's inputs u[max_in][RB] and index lists are staged in shared memory once;
//   - the columns of both blocks, block 0 then block 1, flow as one sequence of chunks of KC
//     whole columns (contiguous in a column-major block) through a ring of STAGES shared-memory
//     stages filled with cp.async, so the copies of the next chunks, also across the change of
//     block, overlap the arithmetic of the current one;
//   - every thread accumulates a TR x TC tile (TR rows interleaved by the number of row tiles,
//     so that a warp reads consecutive rows of a staged column; TC consecutive right-hand sides
//     read as one vector from u); when a block has fewer tiles than half the CTA, the columns of
//     each chunk are dealt to S = 2, 4 or 8 slices held by neighbouring lanes, whose partial sums
//     meet through warp shuffles;
//   - outputs leave from registers: V and S levels write out_c = M_c u_c (+ u[q_c]) directly;
//     a U level writes block 0's contributions to its output segment first and block 1 adds its
//     own after a barrier (every output position receives exactly one term from each block, so
//     the order of the two additions does not change the sum).
namespace tiled {
constexpr int TR = 4, KC = 16, STAGES = 2;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// bytes of one stage: KC columns of the tallest block (max_rows rows), plus room for a start
// moved down to a 16-byte boundary and an end rounded up to one
template <class P>
__host__ __device__ constexpr size_t stage_bytes(int max_rows) {
  return (((size_t)max_rows * KC * sizeof(typename P::mat_t) + 32) + 15) & ~(size_t)15;
}
// shared memory: u | ring | index lists
template <class P, int RB, int TC>
__host__ __device__ constexpr size_t smem_bytes(int max_in, int max_out, int max_rows, int nthreads) {
  return (((size_t)max_in * RB * sizeof(typename P::vec_t) + 15) & ~(size_t)15) + STAGES * stage_bytes<P>(max_rows) +
         2 * (size_t)((max_in > max_out ? max_in : max_out) + 4) * sizeof(int32_t) + 0 * nthreads;
}

// TC consecutive operands u[0 .. TC-1] (16-byte aligned)
template <class P, int TC>
__device__ __forceinline__ void load_ops(const typename P::vec_t* p, typename P::gv_t (&b)[TC]) {
  if constexpr (sizeof(typename P::vec_t) == 8) {
    static_assert(TC % 2 == 0, "pairs of complex64");
#pragma unroll
    for (int c = 0; c < TC; c += 2) {
      const float4 v = *reinterpret_cast<const float4*>(p + c);
      b[c] = make_float2(v.x, v.y);
      b[c + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int c = 0; c < TC; ++c) b[c] = p[c];
  }
}

// work split of one block over the CTA
struct Split {
  int rows, cols, nch;  // chunks of the block (0 if the block is empty)
  int nrt, tasks;       // row tiles, (row tile, rhs group) tasks
  int S, rounds;        // column slices per task (neighbouring lanes), passes over the block
};
__device__ __forceinline__ Split split_of(int rows, int cols, int nrb, int TC, int nt) {
  Split q;
  q.rows = rows;
  q.cols = cols;
  q.nch = (rows > 0 && cols > 0) ? (cols + KC - 1) / KC : 0;
  q.nrt = (rows + TR - 1) / TR;
  q.tasks = q.nrt * ((nrb + TC - 1) / TC);
  q.S = 1;
  while (q.S < 8 && q.S < KC && 2 * q.S * q.tasks <= nt) q.S *= 2;
  q.rounds = q.S > 1 ? 1 : (q.tasks + nt - 1) / nt;
  return q;
}
}  // namespace tiled

template <class P, int RB, int TC>
__device__ __forceinline__ void fwd_node_tiled(const DevLevel& d, const typename P::mat_t* __restrict__ mat,
                                               const IO<typename P::vec_t>& io, int max_rows, int max_in,
                                               int max_out, int64_t j, int r0, unsigned char* smem) {
  using namespace tiled;
  using V = typename P::vec_t;
  using G = typename P::gv_t;
  using M = typename P::mat_t;
  using A = typename P::acc_t;
  static_assert(std::is_same<V, G>::value, "operands used as stored (FP32 and FP64 policies)");
  static_assert(RB % TC == 0 && (RB * sizeof(V)) % 16 == 0, "16-byte aligned operand rows");
  constexpr int ES = (int)sizeof(M);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nrb = min(RB, io.R - r0);
  V* u = (V*)smem;
  unsigned char* ring = smem + (((size_t)max_in * RB * sizeof(V) + 15) & ~(size_t)15);
  const size_t sbytes = stage_bytes<P>(max_rows);
  int32_t* ixs = (int32_t*)(ring + STAGES * sbytes);
  const int icap = (max_in > max_out ? max_in : max_out) + 4;

  // node description
  int l0, l1;
  int64_t o0 = 0, o1 = 0;
  if (d.lev == 0) {
    l0 = d.n0;
    l1 = 0;
  } else {
    l0 = d.in_len[2 * j];
    l1 = d.in_len[2 * j + 1];
    o0 = d.in_off[2 * j];
    o1 = d.in_off[2 * j + 1];
  }
  const int64_t mov[2] = {d.moff[2 * j], d.moff[2 * j + 1]};
  const Split sp[2] = {split_of(d.rows[2 * j], d.cols[2 * j], nrb, TC, nt),
                       split_of(d.rows[2 * j + 1], d.cols[2 * j + 1], nrb, TC, nt)};
  const int tot0 = sp[0].nch * sp[0].rounds;                // chunks of block 0 over all its passes
  const int tot = tot0 + sp[1].nch * sp[1].rounds;

  // stream chunk g of the node's sequence into stage g % STAGES (all threads; one commit group).
  // Chunks are issued in order, so the block and chunk within it are tracked incrementally.
  int ic = 0, iq = 0, ir = 0;  // block, chunk and pass of the next chunk to issue
  if (sp[0].nch == 0) ic = 1;
  auto issue = [&](int g) {
    const int c = ic, q = iq;
    if (++iq == sp[c].nch) {
      iq = 0;
      if (++ir == sp[c].rounds) { ir = 0; ic = 1; }
    }
    const int rows = sp[c].rows;
    const int k0 = q * KC, kc = min(KC, sp[c].cols - k0);
    const unsigned char* src = (const unsigned char*)(mat + mov[c] + (int64_t)k0 * rows);
    const unsigned char* al = (const unsigned char*)((uintptr_t)src & ~(uintptr_t)15);
    const unsigned char* end = (const unsigned char*)(((uintptr_t)(src + (size_t)kc * rows * ES) + 15) & ~(uintptr_t)15);
    unsigned char* dst = ring + (size_t)(g % STAGES) * sbytes;
    const int pieces = (int)((end - al) >> 4);
    for (int p = tid; p < pieces; p += nt) cp_async16(dst + 16 * p, al + 16 * p);
  };
  // the first chunks go out before the inputs are loaded
#pragma unroll
  for (int g = 0; g < STAGES - 1; ++g) {
    if (g < tot) issue(g);
    cp_async_commit();
  }

  // inputs -> u (level 0: consecutive threads read consecutive elements of one column of x),
  // index lists -> ixs
  if (d.lev == 0) {
    for (int i = tid; i < l0 * RB; i += nt) {
      const int rb = i / l0, e = i - rb * l0;
      u[e * RB + rb] = rb < nrb ? io.x[j * d.n0 + e + (int64_t)(r0 + rb) * io.ldx] : P::zero();
    }
  } else {
    for (int i = tid; i < (l0 + l1) * RB; i += nt) {
      const int e = i / RB, rb = i % RB;
      const int64_t off = e < l0 ? o0 + e : o1 + (e - l0);
      u[i] = rb < nrb ? io.win[off * io.R + r0 + rb] : P::zero();
    }
  }
  if (d.kind != KIND_S) {
    for (int c = 0; c < 2; ++c) {
      const int n = sp[c].rows + (d.kind == KIND_V ? sp[c].cols : (c ? l1 : l0));
      const int32_t* ix = d.idx + d.ioff[2 * j + c];
      for (int i = tid; i < n; i += nt) ixs[c * icap + i] = ix[i];
    }
  }
  __syncthreads();

  // U levels: where output position e of the node lives
  int len0 = 0;
  int64_t b0 = 0, b1 = 0;
  if (d.kind == KIND_U && d.lev < d.L) {
    const int64_t s0 = out_seg_id(d, j, 0), s1 = out_seg_id(d, j, 1);
    len0 = d.out_len[s0];
    b0 = d.out_off[s0];
    b1 = d.out_off[s1];
  }
  auto u_out = [&](int e, int rb) -> V* {
    if (d.lev == d.L) return io.y + j * d.n0 + e + (int64_t)(r0 + rb) * io.ldy;
    const int64_t off = e < len0 ? b0 + e : b1 + (e - len0);
    return io.wout + off * io.R + r0 + rb;
  };

  int g = 0;  // position in the node's chunk sequence
  for (int c = 0; c < 2; ++c) {
    const Split bc = sp[c];
    const int rows = bc.rows;
    const int32_t* ixc = ixs + c * icap;
    const int lc = c ? l1 : l0;
    const int opbase = (d.kind == KIND_U && c) ? l0 : 0;  // U: block c multiplies in_c; S: all of u
    int64_t ob = 0;
    if (d.kind != KIND_U) ob = d.out_off[out_seg_id(d, j, c)];
    const int S = bc.S;
    for (int rd = 0; rd < bc.rounds && bc.tasks > 0; ++rd) {
      const int w = S > 1 ? tid / S : rd * nt + tid;
      const int sl = S > 1 ? tid - w * S : 0;
      const bool active = w < bc.tasks;
      const int ct = active ? w / bc.nrt : 0;
      const int rt = active ? w - ct * bc.nrt : 0;
      A acc[TR][TC];
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int cc = 0; cc < TC; ++cc) P::init(acc[i][cc]);
      int roff[TR];
#pragma unroll
      for (int i = 0; i < TR; ++i) roff[i] = max(0, min(rt + i * bc.nrt, rows - 1));
      for (int q = 0; q < bc.nch; ++q, ++g) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();  // chunk g landed for every thread; the stage of chunk g-1 is free again
        if (g + STAGES - 1 < tot) issue(g + STAGES - 1);
        cp_async_commit();
        if (active) {
          const int k0 = q * KC, kc = min(KC, bc.cols - k0);
          const unsigned char* stg = ring + (size_t)(g % STAGES) * sbytes;
          const M* mc = (const M*)(stg + ((uintptr_t)(mat + mov[c] + (int64_t)k0 * rows) & 15));
          auto column = [&](int kk) {
            const int k = k0 + kk;
            const int er = d.kind == KIND_V ? ixc[rows + k] : opbase + k;
            G b[TC];
            load_ops<P, TC>(u + (size_t)er * RB + ct * TC, b);
            const M* mcol = mc + kk * rows;
#pragma unroll
            for (int i = 0; i < TR; ++i) {
              const M mv = mcol[roff[i]];
#pragma unroll
              for (int cc = 0; cc < TC; ++cc) P::mac(acc[i][cc], mv, b[cc]);
            }
          };
          if (S == 1 && kc == KC) {
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) column(kk);
          } else {
            for (int kk = sl; kk < kc; kk += S) column(kk);
          }
        }
      }
      // the S slices of a task are neighbouring lanes: combine their partial sums
      for (int o = 1; o < S; o <<= 1) {
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
          for (int cc = 0; cc < TC; ++cc) {
            acc[i][cc].re += __shfl_xor_sync(0xffffffffu, acc[i][cc].re, o);
            acc[i][cc].im += __shfl_xor_sync(0xffffffffu, acc[i][cc].im, o);
          }
      }
      if (active && sl == 0) {
#pragma unroll
        for (int i = 0; i < TR; ++i) {
          const int r = rt + i * bc.nrt;
          if (r >= rows) continue;
#pragma unroll
          for (int cc = 0; cc < TC; ++cc) {
            const int rb = ct * TC + cc;
            if (rb >= nrb) continue;
            V v = P::fin(acc[i][cc]);
            if (d.kind == KIND_U) {
              V* dst = u_out(ixc[lc + r], rb);
              *dst = c ? P::add(*dst, v) : v;
            } else {
              if (d.kind == KIND_V) v = P::add(v, u[(size_t)ixc[r] * RB + rb]);
              io.wout[(ob + r) * io.R + r0 + rb] = v;
            }
          }
        }
      }
    }
    if (d.kind == KIND_U) {
      // the inputs pass through to positions q_c
      for (int i = tid; i < lc * nrb; i += nt) {
        const int e = i / nrb, rb = i - e * nrb;
        V* dst = u_out(ixc[e], rb);
        const V v = u[(size_t)(opbase + e) * RB + rb];
        *dst = c ? P::add(*dst, v) : v;
      }
      if (c == 0) __syncthreads();  // block 0's terms are in place before block 1 adds to them
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------------------------
// Warp-per-node forward body, one right-hand side, for levels of short blocks (the outer levels
// of the butterfly: leaves and their neighbours). Every phase of a node (inputs, gathered operands,
// block products, combination) is done by one warp with __syncwarp between phases, so a CTA has
// as many nodes in flight as it has warps and no phase waits for another warp. Lanes cover the
// rows of a block, RPL rows each (rows <= 32 RPL); a column of a block is read by the warp as
// consecutive entries. Shared memory per warp: u[max_in] (inputs), g[2][gcap] (gathered
// operands), t[max_out] (row-ID accumulation of a U level).
template <class P>
__host__ __device__ constexpr size_t warp_node_smem(int max_in, int gcap, int max_out) {
  return (((size_t)max_in * sizeof(typename P::vec_t) + 2 * (size_t)gcap * sizeof(typename P::gv_t) +
           (size_t)max_out * sizeof(typename P::vec_t)) + 15) & ~(size_t)15;
}

template <class P, int RPL>
__device__ __forceinline__ void fwd_node_warp(const DevLevel& d, const typename P::mat_t* __restrict__ mat,
                                              const IO<typename P::vec_t>& io, int max_in, int gcap, int64_t j,
                                              unsigned char* wsm) {
  using V = typename P::vec_t;
  using G = typename P::gv_t;
  using M = typename P::mat_t;
  using BP = Bnd<P, df_boundary<P, 1, 0>()>;
  using B = typename BP::b_t;
  V* u = (V*)wsm;
  B* ub = (B*)u;  // the inputs of a level > 0, in the boundary format
  G* g = (G*)(u + max_in);
  B* t = (B*)(g + 2 * (size_t)gcap);
  const B* winb = (const B*)io.win;
  B* woutb = (B*)io.wout;
  const int lane = threadIdx.x & 31;

  // inputs -> u
  int l0, l1;
  if (d.lev == 0) {
    l0 = d.n0;
    l1 = 0;
    for (int e = lane; e < l0; e += 32) u[e] = io.x[j * d.n0 + e];
  } else {
    l0 = d.in_len[2 * j];
    l1 = d.in_len[2 * j + 1];
    const int64_t o0 = d.in_off[2 * j], o1 = d.in_off[2 * j + 1];
    for (int e = lane; e < l0 + l1; e += 32) ub[e] = winb[(e < l0 ? o0 + e : o1 + (e - l0)) * io.R];
  }
  const bool lev0 = d.lev == 0;
  auto gin = [&](int e) -> G { return lev0 ? P::cvt(u[e]) : BP::g_of(ub[e]); };
  auto bin = [&](int e) -> B { return lev0 ? BP::of_v(u[e]) : ub[e]; };
  const int rowsv[2] = {d.rows[2 * j], d.rows[2 * j + 1]};
  const int colsv[2] = {d.cols[2 * j], d.cols[2 * j + 1]};
  const int64_t mov[2] = {d.moff[2 * j], d.moff[2 * j + 1]};
  const int32_t* ixv[2] = {d.idx + d.ioff[2 * j], d.idx + d.ioff[2 * j + 1]};
  __syncwarp();

  // gathered operands -> g
  if (d.kind == KIND_V) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
      for (int k = lane; k < colsv[c]; k += 32) g[c * gcap + k] = gin(ixv[c][rowsv[c] + k]);
  } else if (d.kind == KIND_S) {
    for (int e = lane; e < l0 + l1; e += 32) g[e] = gin(e);
  } else {
    for (int e = lane; e < l0; e += 32) g[e] = gin(e);
    for (int e = lane; e < l1; e += 32) g[gcap + e] = gin(l0 + e);
  }
  __syncwarp();

  // block products: lane owns rows lane + 32 i
  B res[2][RPL];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int rows = rowsv[c], cols = colsv[c];
    const M* Mc = mat + mov[c];
    const G* gc = g + (d.kind == KIND_S ? 0 : c * gcap);
    // two accumulators per row (even and odd columns): two independent dependency chains
    typename P::acc_t acc0[RPL], acc1[RPL];
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      P::init(acc0[i]);
      P::init(acc1[i]);
    }
    auto pair = [&](int kk) {  // columns kk (into acc0) and kk + 1 (into acc1)
      const G g0 = gc[kk], g1 = gc[kk + 1];
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        const int r = lane + 32 * i;
        if (r < rows) {
          P::mac(acc0[i], P::ld(Mc + (int64_t)kk * rows + r), g0);
          P::mac(acc1[i], P::ld(Mc + (int64_t)(kk + 1) * rows + r), g1);
        }
      }
    };
    int k = 0;
    for (; k + 2 * P::CHUNK <= cols; k += 2 * P::CHUNK) {
#pragma unroll 4
      for (int q = 0; q < 2 * P::CHUNK; q += 2) pair(k + q);
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        P::flush(acc0[i]);
        P::flush(acc1[i]);
      }
    }
    for (; k + 1 < cols; k += 2) pair(k);
    if (k < cols) {
      const G g0 = gc[k];
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        const int r = lane + 32 * i;
        if (r < rows) P::mac(acc0[i], P::ld(Mc + (int64_t)k * rows + r), g0);
      }
    }
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      P::flush(acc0[i]);
      P::flush(acc1[i]);
      P::combine(acc0[i], P::part(acc1[i]));
      res[c][i] = BP::of_acc(acc0[i]);
    }
    if (d.kind != KIND_U) {
      const int64_t ob = d.out_off[out_seg_id(d, j, c)];
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        const int r = lane + 32 * i;
        if (r >= rows) continue;
        B v = res[c][i];
        if (d.kind == KIND_V) v = BP::add(v, bin(ixv[c][r]));
        woutb[(ob + r) * io.R] = v;
      }
    }
  }
  if (d.kind != KIND_U) return;
  // row-ID level: t[q_c] = in_c, t[p_c] = res_c, block 0 first (q_0, p_0 partition t), then
  // block 1 adds (q_1, p_1 also a partition)
  const int tl = l0 + rowsv[0];
  for (int e = lane; e < l0; e += 32) t[ixv[0][e]] = bin(e);
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    const int r = lane + 32 * i;
    if (r < rowsv[0]) t[ixv[0][l0 + r]] = res[0][i];
  }
  __syncwarp();
  for (int e = lane; e < l1; e += 32) {
    B* dst = &t[ixv[1][e]];
    *dst = BP::add(*dst, bin(l0 + e));
  }
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    const int r = lane + 32 * i;
    if (r < rowsv[1]) {
      B* dst = &t[ixv[1][l1 + r]];
      *dst = BP::add(*dst, res[1][i]);
    }
  }
  __syncwarp();
  if (d.lev == d.L) {
    for (int e = lane; e < tl; e += 32) io.y[j * d.n0 + e] = BP::v_of(t[e]);
  } else {
    const int64_t s0 = out_seg_id(d, j, 0), s1 = out_seg_id(d, j, 1);
    const int len0 = d.out_len[s0];
    const int64_t b0 = d.out_off[s0], b1 = d.out_off[s1];
    for (int e = lane; e < tl; e += 32) woutb[(e < len0 ? b0 + e : b1 + (e - len0)) * io.R] = t[e];
  }
}

// ---------------------------------------------------------------------------------------------
// Tiled adjoint node for several right-hand sides (FP32 and FP64 policies). The adjoint of a
// block product y_c = M_c g_c is res_c = M_c^* y_c: a reduction over the block's rows whose
// outputs are its columns. One CTA computes node j for right-hand sides r0 .. r0+nrb-1:
//   - the adjoint inputs v (the forward outputs of the node) are staged once, with, per block,
//     the element of v that each block row multiplies (gsrc) and the block's index lists;
//   - chunks of KR whole rows of a block (all its columns; in a column-major block a row chunk is
//     one short piece per column) flow through a ring of STAGES stages filled with cp.async and
//     laid out row-major with a padded row stride, so a thread's TI consecutive columns are one
//     vector load and a warp's stores and loads spread over the banks;
//   - every thread keeps a TI x TC tile (columns x right-hand sides) in registers over all the
//     chunks; blocks with few column tiles split their rows over S = 2 .. 16 neighbouring lanes,
//     combined by warp shuffles once per block;
//   - outputs are the forward inputs of the node. U level: segment c gets v[q_c] + res_c (each
//     block its own segment). S level: res_0 + res_1 over the same columns. V level: every input
//     element receives one term from each block (v_c[r] at q_c[r] and res_c[i] at p_c[i]). Where
//     two blocks meet, block 0 stores and block 1 adds after a barrier (two terms: the order of
//     the addition cannot change the sum).
namespace tadj {
constexpr int TI = 8, TC = 4, KR = 8, STAGES = 2;
// row stride of a staged chunk: even (16-byte aligned vectors of two complex64 columns) and
// = 2 mod 16 columns, so that the rows of a chunk start in different banks
__host__ __device__ constexpr int col_pad(int cols) {
  return (cols + 15) / 16 * 16 + 2;  // >= the last column tile's end (TI = 8 divides 16)
}
template <class P>
__host__ __device__ constexpr size_t stage_bytes(int max_cols) {
  return ((size_t)KR * col_pad(max_cols) * sizeof(typename P::mat_t) + 15) & ~(size_t)15;
}
// shared memory: v[max_out][RB] | ring | gsrc[2][max_rows] | lists[2][icap]
template <class P, int RB>
__host__ __device__ constexpr size_t smem_bytes(int max_in, int max_out, int max_rows, int max_cols) {
  return (((size_t)max_out * RB * sizeof(typename P::vec_t) + 15) & ~(size_t)15) + STAGES * stage_bytes<P>(max_cols) +
         2 * (size_t)(max_rows + 4) * sizeof(int32_t) +
         2 * (size_t)((max_in > max_out ? max_in : max_out) + 4) * sizeof(int32_t);
}
template <int ES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src),
               "n"(ES)
               : "memory");
}
// TI consecutive staged entries (16-byte aligned)
template <class P>
__device__ __forceinline__ void load_cols(const typename P::mat_t* p, typename P::mat_t (&m)[TI]) {
  if constexpr (sizeof(typename P::mat_t) == 8) {
#pragma unroll
    for (int c = 0; c < TI; c += 2) {
      const float4 v = *reinterpret_cast<const float4*>(p + c);
      m[c] = make_float2(v.x, v.y);
      m[c + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int c = 0; c < TI; ++c) m[c] = p[c];
  }
}
}  // namespace tadj

template <class P, int RB>
__device__ __forceinline__ void adj_node_tiled(const DevLevel& d, const typename P::mat_t* __restrict__ mat,
                                               const IO<typename P::vec_t>& io, int max_in, int max_out,
                                               int max_rows, int max_cols, int64_t j, int r0, unsigned char* smem) {
  using namespace tadj;
  using V = typename P::vec_t;
  using G = typename P::gv_t;
  using M = typename P::mat_t;
  using A = typename P::acc_t;
  static_assert(std::is_same<V, G>::value, "operands used as stored (FP32 and FP64 policies)");
  static_assert(RB % TC == 0 && (RB * sizeof(V)) % 16 == 0, "16-byte aligned operand rows");
  constexpr int ES = (int)sizeof(M);
  constexpr int TCN = TC;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nrb = min(RB, io.R - r0);
  V* v = (V*)smem;
  unsigned char* ring = smem + (((size_t)max_out * RB * sizeof(V) + 15) & ~(size_t)15);
  const size_t sbytes = stage_bytes<P>(max_cols);
  int32_t* gsrc = (int32_t*)(ring + STAGES * sbytes);
  int32_t* lists = gsrc + 2 * (max_rows + 4);
  const int icap = (max_in > max_out ? max_in : max_out) + 4;

  // adjoint inputs (the forward outputs of node j) -> v
  int o0len, o1len;
  if (d.lev == d.L) {
    o0len = d.n0;
    o1len = 0;
    for (int i = tid; i < o0len * RB; i += nt) {
      const int rb = i / o0len, e = i - rb * o0len;
      v[e * RB + rb] = rb < nrb ? io.x[j * d.n0 + e + (int64_t)(r0 + rb) * io.ldx] : P::zero();
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
  const int rowsv[2] = {d.rows[2 * j], d.rows[2 * j + 1]};
  const int colsv[2] = {d.cols[2 * j], d.cols[2 * j + 1]};
  const int64_t mov[2] = {d.moff[2 * j], d.moff[2 * j + 1]};
  // block lists and the element of v each block row multiplies
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int32_t* ix = d.idx + d.ioff[2 * j + c];
    const int nl = d.kind == KIND_S ? 0 : rowsv[c] + colsv[c];
    for (int i = tid; i < nl; i += nt) lists[c * icap + i] = ix[i];
    for (int r = tid; r < rowsv[c]; r += nt)
      gsrc[c * (max_rows + 4) + r] = d.kind == KIND_U ? ix[colsv[c] + r] : (c ? o0len : 0) + r;
  }
  // forward input element e of the node (the adjoint's output), right-hand side rb
  int len0 = 0;
  int64_t ib0 = 0, ib1 = 0;
  if (d.lev > 0) {
    len0 = d.in_len[2 * j];
    ib0 = d.in_off[2 * j];
    ib1 = d.in_off[2 * j + 1];
  }
  auto in_ptr = [&](int e, int rb) -> V* {
    if (d.lev == 0) return io.y + j * d.n0 + e + (int64_t)(r0 + rb) * io.ldy;
    return io.wout + (e < len0 ? ib0 + e : ib1 + (e - len0)) * io.R + r0 + rb;
  };
  __syncthreads();
  const int nct = (nrb + TCN - 1) / TCN;
  for (int c = 0; c < 2; ++c) {
    const int rows = rowsv[c], cols = colsv[c];
    const int32_t* lst = lists + c * icap;
    const int32_t* gs = gsrc + c * (max_rows + 4);
    const M* Mc = mat + mov[c];
    const int cp = col_pad(cols);
    const bool add = c == 1 && d.kind != KIND_U;  // second term of an S or V output
    if (add) __syncthreads();                      // block 0's terms are in place
    if (d.kind == KIND_V) {  // pass-through: v_c[r] -> input element q_c[r]
      for (int i = tid; i < rows * nrb; i += nt) {
        const int r = i / nrb, rb = i - r * nrb;
        V* dst = in_ptr(lst[r], rb);
        const V val = v[(size_t)((c ? o0len : 0) + r) * RB + rb];
        *dst = add ? P::add(*dst, val) : val;
      }
    }
    const int nit = (cols + TI - 1) / TI;
    const int tasks = nit * nct;
    if (tasks == 0) continue;
    int S = 1;
    while (S < 16 && 2 * S * tasks <= nt) S *= 2;
    const int rounds = S > 1 ? 1 : (tasks + nt - 1) / nt;
    const int nch = rows > 0 ? (rows + KR - 1) / KR : 0;
    // rows q*KR .. of the block, all columns, into stage q % STAGES (row-major, stride cp)
    auto issue = [&](int q) {
      const int kr = min(KR, rows - q * KR);
      unsigned char* st = ring + (size_t)(q % STAGES) * sbytes;
      for (int e = tid; e < kr * cols; e += nt) {
        const int col = e / kr, r = e - col * kr;
        cp_async_elem<ES>(st + ((size_t)r * cp + col) * ES, Mc + (int64_t)col * rows + q * KR + r);
      }
    };
    for (int rd = 0; rd < rounds; ++rd) {
      const int w = S > 1 ? tid / S : rd * nt + tid;
      const int sl = S > 1 ? tid - w * S : 0;
      const bool active = w < tasks;
      const int it = active ? w % nit : 0;
      const int ct = active ? w / nit : 0;
      A acc[TI][TCN];
#pragma unroll
      for (int ti = 0; ti < TI; ++ti)
#pragma unroll
        for (int cc = 0; cc < TCN; ++cc) P::init(acc[ti][cc]);
#pragma unroll
      for (int q = 0; q < STAGES - 1; ++q) {
        if (q < nch) issue(q);
        tiled::cp_async_commit();
      }
      for (int q = 0; q < nch; ++q) {
        tiled::cp_async_wait<STAGES - 2>();
        __syncthreads();  // chunk q landed for every thread; the stage of chunk q-1 is free again
        if (q + STAGES - 1 < nch) issue(q + STAGES - 1);
        tiled::cp_async_commit();
        if (active) {
          const int kr = min(KR, rows - q * KR);
          const M* st = (const M*)(ring + (size_t)(q % STAGES) * sbytes);
          for (int r = sl; r < kr; r += S) {
            G b[TCN];
            tiled::load_ops<P, TCN>(v + (size_t)gs[q * KR + r] * RB + ct * TCN, b);
            M m[TI];
            load_cols<P>(st + (size_t)r * cp + it * TI, m);
#pragma unroll
            for (int ti = 0; ti < TI; ++ti)
#pragma unroll
              for (int cc = 0; cc < TCN; ++cc) P::macc(acc[ti][cc], m[ti], b[cc]);
          }
        }
      }
      __syncthreads();  // the ring is free for the next pass
      // the S row slices of a task are neighbouring lanes
      for (int o = 1; o < S; o <<= 1) {
#pragma unroll
        for (int ti = 0; ti < TI; ++ti)
#pragma unroll
          for (int cc = 0; cc < TCN; ++cc) {
            acc[ti][cc].re += __shfl_xor_sync(0xffffffffu, acc[ti][cc].re, o);
            acc[ti][cc].im += __shfl_xor_sync(0xffffffffu, acc[ti][cc].im, o);
          }
      }
      if (active && sl == 0) {
#pragma unroll
        for (int ti = 0; ti < TI; ++ti) {
          const int i = it * TI + ti;
          if (i >= cols) continue;
#pragma unroll
          for (int cc = 0; cc < TCN; ++cc) {
            const int rb = ct * TCN + cc;
            if (rb >= nrb) continue;
            V val = P::fin(acc[ti][cc]);
            V* dst;
            if (d.kind == KIND_U) {  // forward input segment c: v[q_c[i]] + res_c[i]
              val = P::add(val, v[(size_t)lst[i] * RB + rb]);
              dst = in_ptr((c ? colsv[0] : 0) + i, rb);
            } else {
              dst = in_ptr(d.kind == KIND_S ? i : lst[rows + i], rb);
              if (add) val = P::add(*dst, val);
            }
            *dst = val;
          }
        }
      }
    }
  }
  tiled::cp_async_wait<0>();
}

}  // namespace idbf
