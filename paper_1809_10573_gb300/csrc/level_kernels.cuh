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

template <class P> constexpr int fmt_of();
template <> constexpr int fmt_of<FP64P>() { return IDBF_STORE_C128; }
template <> constexpr int fmt_of<DF64P>() { return IDBF_STORE_DF64; }
template <> constexpr int fmt_of<FP32P>() { return IDBF_STORE_C64; }

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

// ---------------------------------------------------------------------------------------------
// forward level kernel. Shared memory: u[max_in][RB] (inputs), g[2][gcap][RB] (gathered
// operands), res[2][rcap][RB] (block products), t[max_out][RB] (row-ID accumulation).
// One node j of a level, right-hand sides r0 .. r0+RB-1, by the whole CTA (used by the per-level
// kernel below and by the persistent batch kernel).
template <class P, int RB>
__device__ __forceinline__ void fwd_node(const DevLevel& d, const typename P::mat_t* __restrict__ mat,
                                         const IO<typename P::vec_t>& io, int gcap, int rcap, int max_in, int64_t j,
                                         int r0, unsigned char* smem) {
  using V = typename P::vec_t;
  using G = typename P::gv_t;
  using M = typename P::mat_t;
  V* u = (V*)smem;
  G* g = (G*)(u + (size_t)max_in * RB);
  V* res = (V*)(g + (size_t)2 * gcap * RB);
  V* t = res + (size_t)2 * rcap * RB;
  const int nrb = min(RB, io.R - r0);
  const int tid = threadIdx.x, nt = blockDim.x;

  // phase 1: inputs -> u
  int l0, l1;
  if (d.lev == 0) {
    l0 = d.n0;
    l1 = 0;
    for (int i = tid; i < l0 * RB; i += nt) {
      const int e = i / RB, rb = i % RB;
      u[i] = rb < nrb ? io.x[j * d.n0 + e + (int64_t)(r0 + rb) * io.ldx] : P::zero();
    }
  } else {
    l0 = d.in_len[2 * j];
    l1 = d.in_len[2 * j + 1];
    const int64_t o0 = d.in_off[2 * j], o1 = d.in_off[2 * j + 1];
    for (int i = tid; i < (l0 + l1) * RB; i += nt) {
      const int e = i / RB, rb = i % RB;
      const int64_t off = e < l0 ? o0 + e : o1 + (e - l0);
      u[i] = rb < nrb ? io.win[off * io.R + r0 + rb] : P::zero();
    }
  }
  const int rows0 = d.rows[2 * j], rows1 = d.rows[2 * j + 1];
  const int cols0 = d.cols[2 * j], cols1 = d.cols[2 * j + 1];
  const int64_t mo0 = d.moff[2 * j], mo1 = d.moff[2 * j + 1];
  const int32_t* ix0 = d.idx + d.ioff[2 * j];
  const int32_t* ix1 = d.idx + d.ioff[2 * j + 1];
  __syncthreads();

  // phase 2: gathered operands
  if (d.kind == KIND_V) {
    for (int i = tid; i < cols0 * RB; i += nt) g[i] = P::cvt(u[ix0[rows0 + i / RB] * RB + i % RB]);
    for (int i = tid; i < cols1 * RB; i += nt) g[gcap * RB + i] = P::cvt(u[ix1[rows1 + i / RB] * RB + i % RB]);
  } else if (d.kind == KIND_S) {
    for (int i = tid; i < (l0 + l1) * RB; i += nt) g[i] = P::cvt(u[i]);
  } else {
    for (int i = tid; i < (l0 + l1) * RB; i += nt) g[i < l0 * RB ? i : gcap * RB + i - l0 * RB] = P::cvt(u[i]);
  }
  __syncthreads();

  // phase 3: block products, one thread per output row
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
      res[(c * rcap + r) * RB + rb] = P::fin(acc[rb]);
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
        V v = res[(c * rcap + r) * RB + rb];
        if (d.kind == KIND_V) v = P::add(v, u[q[r] * RB + rb]);
        io.wout[(ob + r) * io.R + r0 + rb] = v;
      }
    }
    return;
  }
  // row-ID level: t[q_c] += in_c, t[p_c] += res_c. q_0 and p_0 partition t, so block 0
  // initialises every position once; block 1 (q_1, p_1 also a partition) then adds.
  const int tl = l0 + rows0;  // |t| = |q_0| + |p_0|
  for (int i = tid; i < l0 * RB; i += nt) t[ix0[i / RB] * RB + i % RB] = u[i];
  for (int i = tid; i < rows0 * RB; i += nt) t[ix0[l0 + i / RB] * RB + i % RB] = res[i];
  __syncthreads();
  for (int i = tid; i < l1 * RB; i += nt) {
    V* dst = &t[ix1[i / RB] * RB + i % RB];
    *dst = P::add(*dst, u[l0 * RB + i]);
  }
  for (int i = tid; i < rows1 * RB; i += nt) {
    V* dst = &t[ix1[l1 + i / RB] * RB + i % RB];
    *dst = P::add(*dst, res[rcap * RB + i]);
  }
  __syncthreads();
  if (d.lev == d.L) {
    for (int i = tid; i < tl * nrb; i += nt) {
      const int e = i / nrb, rb = i % nrb;
      io.y[j * d.n0 + e + (int64_t)(r0 + rb) * io.ldy] = t[e * RB + rb];
    }
  } else {
    const int64_t s0 = out_seg_id(d, j, 0), s1 = out_seg_id(d, j, 1);
    const int len0 = d.out_len[s0];
    const int64_t b0 = d.out_off[s0], b1 = d.out_off[s1];
    for (int i = tid; i < tl * nrb; i += nt) {
      const int e = i / nrb, rb = i % nrb;
      const int64_t off = e < len0 ? b0 + e : b1 + (e - len0);
      io.wout[off * io.R + r0 + rb] = t[e * RB + rb];
    }
  }
}


}  // namespace idbf
