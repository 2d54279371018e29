// On-device construction of the IDBF (Secs. 2.1-2.4 of the paper).
//
// The construction runs step by step as the leaf-root complementary skeletonization (Sec. 2.2)
// recursed by matrix splitting (Secs. 2.3-2.4): U step 1, V step 1, U step 2, V step 2, ...
//   U step s, every (rho at depth L-s+1, kappa at depth s): a row ID of K(rows, columns) with
//     rows    = the leaf rows of rho (s = 1) or rhat(2rho, kappa/2) u rhat(2rho+1, kappa/2);
//     columns = the columns of kappa (s = 1) or the skeleton columns chat(tau, sigma) of the
//               column nodes sigma at depth L-s+2 below kappa, tau the ancestor of rho at
//               depth s-1.
//   V step s, every (tau at depth s, sigma at depth L-s+1): a column ID with
//     columns = the leaf columns of sigma (s = 1) or chat(tau/2, 2sigma) u chat(tau/2, 2sigma+1);
//     rows    = the skeleton rows rhat(rho, kappa) of the row nodes rho at depth L-s+1 below
//               tau, kappa the ancestor of sigma at depth s.
//   Middle factor: S(rho, sigma) = K(rhat(rho, sigma/2), chat(rho/2, sigma)).
// Each ID (Sec. 2.1): t*k candidates sampled (Mock-Chebyshev or uniform random), the sampled
// block filled with kernel entries, an FP64 column-pivoted Householder QR run until
// |R_jj| <= eps |R_11| or the rank parameter is reached, and T = R11^{-1} R12 by FP64 back
// substitution. Skeletons are kept in increasing index order (the rows of T permuted to match),
// so that the skeleton lists of consecutive nodes concatenate into sorted candidate lists.
//
// Storage of the result: the butterfly layout of include/idbf.h, one arena per level.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "idbf_internal.h"

namespace idbf {
namespace bld {

struct KDesc {
  int kind, sign, prof;
};

// (a b) mod 1 with the rounding error of the product kept: p = fl(ab), e = fma(a, b, -p) is
// exact (the FMA-based two-product), and p - rint(p) is exact for |p| < 2^52.
__device__ __forceinline__ double frac_prod(double a, double b) {
  const double p = __dmul_rn(a, b);
  const double e = fma(a, b, -p);
  return __dadd_rn(__dsub_rn(p, rint(p)), e);
}

// c(x) of the FIO kernels (Example 1)
__global__ void k_cprofile(const double* __restrict__ x, double* __restrict__ cx, int64_t n, int prof) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    double c = 0.0;
    if (prof == 0) c = (2.0 + sinpi(2.0 * v) * sinpi(4.0 * v)) / 3.0;
    else if (prof == 1) c = (2.0 + 0.2 * sinpi(2.0 * v)) / 16.0;
    cx[i] = c;
  }
}

__device__ __forceinline__ double2 kentry(const KDesc& K, double x, double cx, double xi) {
  if (K.kind == IDBF_KERNEL_J0) return make_double2(j0(x * xi), 0.0);  // Example 2
  double ph;
  if (K.kind == IDBF_KERNEL_FIO1D) ph = frac_prod(x, xi) + frac_prod(cx, fabs(xi));
  else ph = (double)K.sign * frac_prod(x, xi);
  double s, c;
  sincospi(2.0 * ph, &s, &c);
  return make_double2(c, s);
}

// ---- per-ID descriptors ---------------------------------------------------------------------
struct IDDesc {
  // the interpolated side ("b" list: rows of a row ID, columns of a column ID)
  int64_t b_range;   // >= 0: the list is b_range .. b_range + b - 1
  int64_t b_a_off;   // else: concatenation of prev[b_a_off .. +b_a) and prev[b_b_off .. +b_b)
  int64_t b_b_off;
  int32_t b_a, b_b;
  int32_t b;
  // candidates on the sampled side
  int64_t c_range;   // >= 0: candidates c_range .. c_range + n_c - 1; else list[c_off ..]
  int64_t c_off;
  int64_t n_c;
  int32_t ns;        // samples
  int32_t kmax;      // max rank (min(ns, b, k))
  int32_t pad0;
  int32_t pad;
  uint64_t key;      // random sampling stream
  // scratch offsets (batch-relative)
  int64_t a_off;     // QR matrix (complex), column-major, ld = ns
  int64_t bl_off;    // b list (global indices)
  int64_t sp_off;    // samples (global indices)
};

__device__ __forceinline__ int64_t cand_index(const IDDesc& d, const int32_t* list, int64_t i) {
  return d.c_range >= 0 ? d.c_range + i : (int64_t)list[d.c_off + i];
}

__global__ void k_make_blist(const IDDesc* __restrict__ D, const int32_t* __restrict__ prev, int32_t* __restrict__ bl) {
  const IDDesc d = D[blockIdx.x];
  for (int i = threadIdx.x; i < d.b; i += blockDim.x) {
    int64_t v;
    if (d.b_range >= 0) v = d.b_range + i;
    else v = i < d.b_a ? prev[d.b_a_off + i] : prev[d.b_b_off + (i - d.b_a)];
    bl[d.bl_off + i] = (int32_t)v;
  }
}

// ---- sampling (Sec. 2.1): one warp per ID ----------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// open-addressing set / map of candidate indices in shared memory (key + 1 stored; 0 = empty)
__device__ __forceinline__ int hs_find(const int32_t* keys, int cap, int32_t k) {
  uint32_t h = ((uint32_t)k * 2654435761u) & (cap - 1);
  while (keys[h] != 0 && keys[h] != k + 1) h = (h + 1) & (cap - 1);
  return (int)h;
}

// Mock-Chebyshev (sampling == 0), random (1), all (2). Output: sorted global indices.
// Shared memory per warp: keys[cap], vals[cap], picks[nsmax]; cap is a power of two larger than
// twice the number of keys inserted (ns for Mock-Chebyshev, up to 2 ns for the shuffle).
__global__ void k_sample(const IDDesc* __restrict__ D, int64_t nid, const int32_t* __restrict__ list,
                         const double* __restrict__ coord, int32_t* __restrict__ samp, int sampling, int cap,
                         int nsmax) {
  extern __shared__ int32_t sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int64_t id = (int64_t)blockIdx.x * nwarps + warp;
  if (id >= nid) return;
  int32_t* keys = sm + (size_t)warp * (cap * 2 + nsmax);
  int32_t* vals = keys + cap;
  int32_t* picks = vals + cap;
  const IDDesc d = D[id];
  const int ns = d.ns;
  int32_t* out = samp + d.sp_off;
  if (sampling == 2 || d.n_c <= ns) {
    for (int i = lane; i < ns; i += 32) out[i] = (int32_t)cand_index(d, list, i);
    return;
  }
  for (int i = lane; i < cap; i += 32) keys[i] = 0;
  __syncwarp();
  if (sampling == 0) {
    // nearest candidate position of every Chebyshev node (lower bound), in parallel
    const double lo = coord[cand_index(d, list, 0)], hi = coord[cand_index(d, list, d.n_c - 1)];
    for (int j = lane; j < ns; j += 32) {
      const double t = (1.0 - cospi((2.0 * j + 1.0) / (2.0 * ns))) * 0.5;
      const double y = lo + t * (hi - lo);
      int64_t a = 0, b = d.n_c;  // first index with coord >= y
      while (a < b) {
        const int64_t mid = (a + b) >> 1;
        if (coord[cand_index(d, list, mid)] < y) a = mid + 1; else b = mid;
      }
      picks[j] = (int32_t)a;
    }
    __syncwarp();
    if (lane == 0) {
      for (int j = 0; j < ns; ++j) {
        const double t = (1.0 - cospi((2.0 * j + 1.0) / (2.0 * ns))) * 0.5;
        const double y = lo + t * (hi - lo);
        const int64_t pos = picks[j];
        int64_t left = pos - 1, right = pos;
        while (left >= 0 && keys[hs_find(keys, cap, (int32_t)left)] != 0) --left;
        while (right < d.n_c && keys[hs_find(keys, cap, (int32_t)right)] != 0) ++right;
        int64_t pick;
        if (left < 0) pick = right;
        else if (right >= d.n_c) pick = left;
        else pick = (y - coord[cand_index(d, list, left)]) <= (coord[cand_index(d, list, right)] - y) ? left : right;
        keys[hs_find(keys, cap, (int32_t)pick)] = (int32_t)pick + 1;
        picks[j] = (int32_t)pick;
      }
    }
  } else {
    // partial Fisher-Yates over a virtual array 0..n_c-1; draw i uses splitmix64 at counter i
    if (lane == 0) {
      for (int i = 0; i < ns; ++i) {
        const uint64_t r = splitmix64_mix(d.key + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull);
        const int64_t j = i + (int64_t)(r % (uint64_t)(d.n_c - i));
        const int hi_ = hs_find(keys, cap, i), hj = hs_find(keys, cap, (int32_t)j);
        const int32_t vi = keys[hi_] ? vals[hi_] : i;
        const int32_t vj = keys[hj] ? vals[hj] : (int32_t)j;
        keys[hj] = (int32_t)j + 1;
        vals[hj] = vi;
        const int hi2 = hs_find(keys, cap, i);
        keys[hi2] = i + 1;
        vals[hi2] = vj;
        picks[i] = vj;
      }
    }
  }
  __syncwarp();
  // sort the picks (distinct positions) by rank and emit global indices
  for (int i = lane; i < ns; i += 32) {
    const int32_t v = picks[i];
    int rank = 0;
    for (int l = 0; l < ns; ++l) rank += picks[l] < v;
    out[rank] = (int32_t)cand_index(d, list, v);
  }
}

// ---- kernel entries of the sampled block ----------------------------------------------------
// row ID (side 0): QR matrix A(i, c) = K(x[b_c], xi[s_i]) (the transpose of the sampled block)
// column ID (side 1): A(i, c) = K(x[s_i], xi[b_c])
// Entries are FP64 (double2) or, for the double-float QR, split into (re_hi, re_lo, im_hi, im_lo)
// binary32 parts (float4, the same 16 bytes): hi = fl32(v), lo = fl32(v - hi).
__device__ __forceinline__ float4 df_split(double2 v) {
  const float rh = (float)v.x, ih = (float)v.y;
  return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}
__device__ __forceinline__ double2 df_join(float4 v) {
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

template <bool DF>
__global__ void k_fill(const IDDesc* __restrict__ D, const int32_t* __restrict__ bl, const int32_t* __restrict__ sp,
                       const double* __restrict__ x, const double* __restrict__ cx, const double* __restrict__ xi,
                       double2* __restrict__ A, KDesc K, int side) {
  const IDDesc d = D[blockIdx.x];
  double2* a = A + d.a_off;
  const int32_t* b = bl + d.bl_off;
  const int32_t* s = sp + d.sp_off;
  for (int c = blockIdx.y; c < d.b; c += gridDim.y) {
    const int32_t bc = b[c];
    for (int i = threadIdx.x; i < d.ns; i += blockDim.x) {
      const int32_t si = s[i];
      const double2 v = side == 0 ? kentry(K, x[bc], cx[bc], xi[si]) : kentry(K, x[si], cx[si], xi[bc]);
      if constexpr (DF) ((float4*)a)[(int64_t)c * d.ns + i] = df_split(v);
      else a[(int64_t)c * d.ns + i] = v;
    }
  }
}

// ---- FP64 column-pivoted Householder QR and the interpolation matrix -------------------------
__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

template <int NT>
__device__ __forceinline__ void block_argmax(double& v, int& idx, double* rv, int* ri) {
  // max value, ties to the lowest index
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { rv[w] = v; ri[w] = idx; }
  __syncthreads();
  if (w == 0) {
    v = lane < NT / 32 ? rv[lane] : -1.0;
    idx = lane < NT / 32 ? ri[lane] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if (lane == 0) { rv[0] = v; ri[0] = idx; }
  }
  __syncthreads();
  v = rv[0];
  idx = ri[0];
  __syncthreads();
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* rv) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) rv[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < NT / 32 ? rv[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) rv[0] = v;
  }
  __syncthreads();
  v = rv[0];
  __syncthreads();
  return v;
}

// On exit: kout[id] = k_eps; perm (b entries, pivot order) in pscr; A(0:k, k:b) holds T.
template <int NT>
__global__ void __launch_bounds__(NT) k_qr(const IDDesc* __restrict__ D, double2* __restrict__ Aall,
                                           int32_t* __restrict__ pscr, int32_t* __restrict__ kout,
                                           int32_t* __restrict__ satur, double eps) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const IDDesc d = D[blockIdx.x];
  const int ns = d.ns, b = d.b, kmax = d.kmax;
  double2* A = Aall + d.a_off;
  double2* v = (double2*)smraw;               // Householder vector, ns
  double* nrm = (double*)(v + ns);            // column norms^2, b
  int* perm = (int*)(nrm + b);                // b
  __shared__ double rv[NT / 32];
  __shared__ int ri[NT / 32];
  __shared__ double2 sh_beta;
  __shared__ double sh_coef;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  for (int c = tid; c < b; c += NT) perm[c] = c;
  for (int c = warp; c < b; c += NW) {
    const double2* col = A + (int64_t)c * ns;
    double s = 0.0;
    for (int i = lane; i < ns; i += 32) { const double2 z = col[i]; s = fma(z.x, z.x, fma(z.y, z.y, s)); }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nrm[c] = s;
  }
  __syncthreads();
  double r11 = 0.0;
  int k = 0;
  bool zero_block = false;
  for (int j = 0; j < kmax; ++j) {
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int c = j + tid; c < b; c += NT)
      if (nrm[c] > best) { best = nrm[c]; bi = c; }
    block_argmax<NT>(best, bi, rv, ri);
    const double rjj = sqrt(best);
    if (j == 0) {
      r11 = rjj;
      if (!(r11 > 0.0)) { zero_block = true; break; }
    } else if (rjj <= eps * r11) {
      break;
    }
    // move the pivot column to position j
    if (bi != j) {
      double2* cj = A + (int64_t)j * ns;
      double2* cp = A + (int64_t)bi * ns;
      for (int i = tid; i < ns; i += NT) { const double2 t = cj[i]; cj[i] = cp[i]; cp[i] = t; }
      __syncthreads();
      if (tid == 0) {
        const double tn = nrm[j]; nrm[j] = nrm[bi]; nrm[bi] = tn;
        const int tp = perm[j]; perm[j] = perm[bi]; perm[bi] = tp;
      }
    }
    __syncthreads();
    // Householder reflector H = I - 2 v v^* / (v^* v) with H x = beta e_1, x = A(j:ns, j)
    double2* cj = A + (int64_t)j * ns;
    double a2 = 0.0;
    for (int i = j + tid; i < ns; i += NT) { const double2 z = cj[i]; a2 = fma(z.x, z.x, fma(z.y, z.y, a2)); }
    a2 = block_sum<NT>(a2, rv);
    if (tid == 0) {
      const double alpha = sqrt(a2);
      const double2 x0 = cj[j];
      const double ax0 = hypot(x0.x, x0.y);
      const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
      const double2 beta = make_double2(-ph.x * alpha, -ph.y * alpha);
      sh_beta = beta;
      v[0] = make_double2(x0.x - beta.x, x0.y - beta.y);
      sh_coef = 2.0 / (2.0 * a2 + 2.0 * alpha * ax0);  // 2 / (v^* v)
    }
    for (int i = j + 1 + tid; i < ns; i += NT) v[i - j] = cj[i];
    __syncthreads();
    const double coef = sh_coef;
    // trailing columns: a -= coef v (v^* a); norms of rows j+1.. recomputed
    for (int c = j + 1 + warp; c < b; c += NW) {
      double2* col = A + (int64_t)c * ns;
      double2 dot = make_double2(0.0, 0.0);
      for (int i = j + lane; i < ns; i += 32) {
        const double2 z = col[i], w = v[i - j];
        dot.x = fma(w.x, z.x, fma(w.y, z.y, dot.x));
        dot.y = fma(w.x, z.y, fma(-w.y, z.x, dot.y));
      }
      for (int o = 16; o > 0; o >>= 1) {
        dot.x += __shfl_xor_sync(0xffffffffu, dot.x, o);
        dot.y += __shfl_xor_sync(0xffffffffu, dot.y, o);
      }
      const double2 f = make_double2(coef * dot.x, coef * dot.y);
      double s = 0.0;
      for (int i = j + lane; i < ns; i += 32) {
        const double2 w = v[i - j];
        double2 z = col[i];
        z.x = fma(-w.x, f.x, fma(w.y, f.y, z.x));
        z.y = fma(-w.x, f.y, fma(-w.y, f.x, z.y));
        col[i] = z;
        if (i > j) s = fma(z.x, z.x, fma(z.y, z.y, s));
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) nrm[c] = s;
    }
    if (tid == 0) cj[j] = sh_beta;
    __syncthreads();
    k = j + 1;
  }
  int32_t* pout = pscr + d.bl_off;  // same offsets as the b list
  for (int c = tid; c < b; c += NT) pout[c] = perm[c];
  if (zero_block) {
    k = 1;
    for (int c = 1 + tid; c < b; c += NT) A[(int64_t)c * ns] = make_double2(0.0, 0.0);
  }
  if (tid == 0) {
    kout[blockIdx.x] = k;
    // stopped at the cap, not by eps (an empty block, kmax = 0, has rank 0 by definition)
    satur[blockIdx.x] = (!zero_block && kmax > 0 && k == kmax && kmax < b) ? 1 : 0;
  }
  __syncthreads();
  if (zero_block) return;
  // T = R11^{-1} R12 by column-oriented back substitution, a warp per column of R12
  for (int c = k + warp; c < b; c += NW) {
    double2* col = A + (int64_t)c * ns;
    for (int i = k - 1; i >= 0; --i) {
      __syncwarp();
      const double2 rii = A[(int64_t)i * ns + i];
      const double2 num = col[i];
      const double den = rii.x * rii.x + rii.y * rii.y;
      const double2 t = make_double2((num.x * rii.x + num.y * rii.y) / den, (num.y * rii.x - num.x * rii.y) / den);
      const double2* ci = A + (int64_t)i * ns;
      for (int l = lane; l < i; l += 32) {
        const double2 r = ci[l];
        double2 z = col[l];
        z.x -= r.x * t.x - r.y * t.y;
        z.y -= r.x * t.y + r.y * t.x;
        col[l] = z;
      }
      __syncwarp();
      if (lane == 0) col[i] = t;
    }
  }
}

// ---- the same QR in double-float arithmetic ---------------------------------------------------
// GB300 runs FP32 at ~63x its FP64 rate (cuBLAS: 69.7 against 1.10 TFLOP/s), and the Householder
// updates above keep its FP64 pipe ~93 % busy. Here every O(ns b) loop runs in double-float:
// each complex entry is (re_hi, re_lo, im_hi, im_lo) binary32 parts (48 significant bits, Dekker
// 1971), products are formed exactly with FMA and sums with Knuth's TwoSum (Ogita, Rump and Oishi
// 2005; Joldes, Muller and Popescu 2017). The per-step and per-column scalars (norm, reflector
// coefficients, the back-substitution quotients) are computed in FP64 from the double-float
// values, O(b) and O(k b) operations per ID, not O(ns b k). Pivoting compares FP32 column norms;
// the rank test uses the double-float norm of the pivot column. The result (R and T in A) has
// double-float accuracy, far below any ID tolerance eps >= 1e-12.
__device__ __forceinline__ void df2_sum(float a, float b, float& s, float& e) {  // TwoSum (Knuth)
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void df2_fast(float a, float b, float& s, float& e) {  // Fast2Sum, |a| >= |b|
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// (s, c) accumulates a * b for double-float a = (ah, al), b = (bh, bl): the high product exactly
// (p + e), the cross terms into the compensation, p into s by TwoSum
__device__ __forceinline__ void df2_dot(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  float t, err;
  df2_sum(s, p, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}
// (h, l) += (s, c), renormalised
__device__ __forceinline__ void df2_acc(float& h, float& l, float s, float c) {
  float t, e;
  df2_sum(h, s, t, e);
  e = __fadd_rn(e, __fadd_rn(l, c));
  df2_fast(t, e, h, l);
}
__device__ __forceinline__ float4 df_neg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
// z - f w for double-float complex z, f, w (real parts .x/.y, imaginary .z/.w)
__device__ __forceinline__ float4 df_cmsub(float4 z, float4 f, float4 w) {
  float sr = z.x, cr = z.y, si = z.z, ci = z.w;
  df2_dot(sr, cr, -f.x, -f.y, w.x, w.y);
  df2_dot(sr, cr, f.z, f.w, w.z, w.w);
  df2_dot(si, ci, -f.x, -f.y, w.z, w.w);
  df2_dot(si, ci, -f.z, -f.w, w.x, w.y);
  float4 r;
  df2_fast(sr, cr, r.x, r.y);
  df2_fast(si, ci, r.z, r.w);
  return r;
}

template <int NT>
__device__ __forceinline__ double block_sum_d(double v, double* rv) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) rv[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < NT / 32 ? rv[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) rv[0] = v;
  }
  __syncthreads();
  v = rv[0];
  __syncthreads();
  return v;
}

// As k_qr, on double-float entries (float4); same outputs: kout, perm in pscr, T in A(0:k, k:b).
template <int NT>
__global__ void __launch_bounds__(NT) k_qr_df(const IDDesc* __restrict__ D, double2* __restrict__ Araw,
                                              int32_t* __restrict__ pscr, int32_t* __restrict__ kout,
                                              int32_t* __restrict__ satur, double eps) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const IDDesc d = D[blockIdx.x];
  const int ns = d.ns, b = d.b, kmax = d.kmax;
  float4* A = (float4*)(Araw + d.a_off);
  float4* v = (float4*)smraw;                 // Householder vector, ns (double-float complex)
  float* nrm = (float*)(v + ns);              // FP32 squared column norms (pivot choice), b
  int* perm = (int*)(nrm + b);                // b
  __shared__ double rv[NT / 32];
  __shared__ float rvf[NT / 32];
  __shared__ int ri[NT / 32];
  __shared__ float4 sh_beta;
  __shared__ double sh_coef;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  for (int c = tid; c < b; c += NT) perm[c] = c;
  for (int c = warp; c < b; c += NW) {
    const float4* col = A + (int64_t)c * ns;
    float s = 0.f;
    for (int i = lane; i < ns; i += 32) { const float4 z = col[i]; s = fmaf(z.x, z.x, fmaf(z.z, z.z, s)); }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nrm[c] = s;
  }
  __syncthreads();
  double r11 = 0.0;
  int k = 0;
  bool zero_block = false;
  for (int j = 0; j < kmax; ++j) {
    // pivot: the largest FP32 column norm (ties to the lowest index)
    float best = -1.f;
    int bi = 0x7fffffff;
    for (int c = j + tid; c < b; c += NT)
      if (nrm[c] > best) { best = nrm[c]; bi = c; }
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { rvf[warp] = best; ri[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      best = lane < NW ? rvf[lane] : -1.f;
      bi = lane < NW ? ri[lane] : 0x7fffffff;
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) ri[0] = bi;
    }
    __syncthreads();
    bi = ri[0];
    __syncthreads();
    // move the pivot column to position j
    if (bi != j) {
      float4* cj = A + (int64_t)j * ns;
      float4* cp = A + (int64_t)bi * ns;
      for (int i = tid; i < ns; i += NT) { const float4 t = cj[i]; cj[i] = cp[i]; cp[i] = t; }
      __syncthreads();
      if (tid == 0) {
        const float tn = nrm[j]; nrm[j] = nrm[bi]; nrm[bi] = tn;
        const int tp = perm[j]; perm[j] = perm[bi]; perm[bi] = tp;
      }
    }
    __syncthreads();
    // the pivot column's norm in double-float, then the rank test (Eq. acc) in FP64
    float4* cj = A + (int64_t)j * ns;
    double a2;
    {
      float sh = 0.f, sc = 0.f;
      for (int i = j + tid; i < ns; i += NT) {
        const float4 z = cj[i];
        df2_dot(sh, sc, z.x, z.y, z.x, z.y);
        df2_dot(sh, sc, z.z, z.w, z.z, z.w);
      }
      a2 = block_sum_d<NT>((double)sh + (double)sc, rv);
    }
    const double rjj = sqrt(a2);
    if (j == 0) {
      r11 = rjj;
      if (!(r11 > 0.0)) { zero_block = true; break; }
    } else if (rjj <= eps * r11) {
      break;
    }
    // Householder reflector H = I - 2 v v^* / (v^* v) with H x = beta e_1, x = A(j:ns, j)
    if (tid == 0) {
      const double alpha = rjj;
      const double2 x0 = df_join(cj[j]);
      const double ax0 = hypot(x0.x, x0.y);
      const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
      const double2 beta = make_double2(-ph.x * alpha, -ph.y * alpha);
      sh_beta = df_split(beta);
      v[0] = df_split(make_double2(x0.x - beta.x, x0.y - beta.y));
      sh_coef = 2.0 / (2.0 * a2 + 2.0 * alpha * ax0);  // 2 / (v^* v)
    }
    for (int i = j + 1 + tid; i < ns; i += NT) v[i - j] = cj[i];
    __syncthreads();
    const double coef = sh_coef;
    // trailing columns: a -= coef v (v^* a); FP32 norms of rows j+1.. recomputed
    for (int c = j + 1 + warp; c < b; c += NW) {
      float4* col = A + (int64_t)c * ns;
      float dr = 0.f, er = 0.f, di = 0.f, ei = 0.f;  // v^* a: (sum, compensation) per part
      for (int i = j + lane; i < ns; i += 32) {
        const float4 z = col[i], w = v[i - j];
        df2_dot(dr, er, w.x, w.y, z.x, z.y);   // Re: wr zr + wi zi
        df2_dot(dr, er, w.z, w.w, z.z, z.w);
        df2_dot(di, ei, w.x, w.y, z.z, z.w);   // Im: wr zi - wi zr
        df2_dot(di, ei, -w.z, -w.w, z.x, z.y);
      }
      float hr, lr, hi, li;
      df2_fast(dr, er, hr, lr);
      df2_fast(di, ei, hi, li);
      for (int o = 16; o > 0; o >>= 1) {
        const float ohr = __shfl_xor_sync(0xffffffffu, hr, o), olr = __shfl_xor_sync(0xffffffffu, lr, o);
        const float ohi = __shfl_xor_sync(0xffffffffu, hi, o), oli = __shfl_xor_sync(0xffffffffu, li, o);
        df2_acc(hr, lr, ohr, olr);
        df2_acc(hi, li, ohi, oli);
      }
      const double2 f = make_double2(coef * ((double)hr + (double)lr), coef * ((double)hi + (double)li));
      const float4 fd = df_split(f);
      float s = 0.f;
      for (int i = j + lane; i < ns; i += 32) {
        const float4 z = df_cmsub(col[i], fd, v[i - j]);
        col[i] = z;
        if (i > j) s = fmaf(z.x, z.x, fmaf(z.z, z.z, s));
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) nrm[c] = s;
    }
    if (tid == 0) cj[j] = sh_beta;
    __syncthreads();
    k = j + 1;
  }
  int32_t* pout = pscr + d.bl_off;  // same offsets as the b list
  for (int c = tid; c < b; c += NT) pout[c] = perm[c];
  if (zero_block) {
    k = 1;
    for (int c = 1 + tid; c < b; c += NT) A[(int64_t)c * ns] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (tid == 0) {
    kout[blockIdx.x] = k;
    // stopped at the cap, not by eps (an empty block, kmax = 0, has rank 0 by definition)
    satur[blockIdx.x] = (!zero_block && kmax > 0 && k == kmax && kmax < b) ? 1 : 0;
  }
  __syncthreads();
  if (zero_block) return;
  // T = R11^{-1} R12 by column-oriented back substitution, a warp per column of R12; the
  // quotient in FP64, the updates in double-float
  for (int c = k + warp; c < b; c += NW) {
    float4* col = A + (int64_t)c * ns;
    for (int i = k - 1; i >= 0; --i) {
      __syncwarp();
      const double2 rii = df_join(A[(int64_t)i * ns + i]);
      const double2 num = df_join(col[i]);
      const double den = rii.x * rii.x + rii.y * rii.y;
      const double2 t = make_double2((num.x * rii.x + num.y * rii.y) / den, (num.y * rii.x - num.x * rii.y) / den);
      const float4 td = df_split(t);
      const float4* ci = A + (int64_t)i * ns;
      for (int l = lane; l < i; l += 32) col[l] = df_cmsub(col[l], ci[l], td);
      __syncwarp();
      if (lane == 0) col[i] = td;
    }
  }
}

// ---- emit: sorted skeleton, index lists and the interpolation block -------------------------
struct EmitDesc {
  int64_t t_off;    // output block offset (complex entries) in the batch result
  int64_t i_off;    // output index offset
  int64_t s_off;    // output skeleton offset
};

// side 0 (row ID): block M = T^T (n_p x k), column-major: M(c, r') at r' n_p + c
// side 1 (column ID): block M = T (k x n_p), column-major: M(r', c) at c k + r'
template <bool DF>
__global__ void k_emit(const IDDesc* __restrict__ D, const EmitDesc* __restrict__ E, const double2* __restrict__ Aall,
                       const int32_t* __restrict__ pscr, const int32_t* __restrict__ bl, const int32_t* __restrict__ kin,
                       double2* __restrict__ Tout, int32_t* __restrict__ Iout, int32_t* __restrict__ Sout, int side) {
  extern __shared__ int32_t sq[];  // q[k], order[k]
  const IDDesc d = D[blockIdx.x];
  const EmitDesc e = E[blockIdx.x];
  const int k = kin[blockIdx.x], b = d.b, np = b - k, ns = d.ns;
  const int32_t* perm = pscr + d.bl_off;
  int32_t* order = sq + k;
  for (int i = threadIdx.x; i < k; i += blockDim.x) sq[i] = perm[i];
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const int32_t v = sq[i];
    int rank = 0;
    for (int l = 0; l < k; ++l) rank += sq[l] < v;
    order[rank] = i;  // sorted position rank holds original skeleton i
  }
  __syncthreads();
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    const int32_t q = sq[order[r]];
    Iout[e.i_off + r] = q;
    Sout[e.s_off + r] = bl[d.bl_off + q];
  }
  for (int c = threadIdx.x; c < np; c += blockDim.x) Iout[e.i_off + k + c] = perm[k + c];
  const double2* A = Aall + d.a_off;
  auto at = [&](int64_t i) -> double2 { return DF ? df_join(((const float4*)A)[i]) : A[i]; };
  for (int64_t t = threadIdx.x; t < (int64_t)k * np; t += blockDim.x) {
    if (side == 0) {
      const int r = (int)(t / np), c = (int)(t % np);
      Tout[e.t_off + t] = at((int64_t)(k + c) * ns + order[r]);
    } else {
      const int c = (int)(t / k), r = (int)(t % k);
      Tout[e.t_off + t] = at((int64_t)(k + c) * ns + order[r]);
    }
  }
}

// skeleton lists: batch order (ID order) -> list order
__global__ void k_gather_lists(const int32_t* __restrict__ src, const int64_t* __restrict__ src_off,
                               const int64_t* __restrict__ dst_off, const int32_t* __restrict__ len,
                               int32_t* __restrict__ dst) {
  const int64_t id = blockIdx.x;
  for (int i = threadIdx.x; i < len[id]; i += blockDim.x) dst[dst_off[id] + i] = src[src_off[id] + i];
}

// middle factor: node j = tau 2^hU + kappa, block c: rows rhat(2tau+c, kappa), columns
// chat(tau, 2kappa) u chat(tau, 2kappa+1); column-major.
struct SDesc {
  int64_t moff;
  int64_t r_off;   // rhat list offset
  int64_t c0_off, c1_off;
  int32_t rows, c0, c1, pad;
};
__global__ void k_fill_S(const SDesc* __restrict__ Sd, const int32_t* __restrict__ rl, const int32_t* __restrict__ cl,
                         const double* __restrict__ x, const double* __restrict__ cx, const double* __restrict__ xi,
                         double2* __restrict__ M, KDesc K) {
  const SDesc s = Sd[blockIdx.x];
  const int cols = s.c0 + s.c1;
  for (int c = blockIdx.y; c < cols; c += gridDim.y) {
    const int32_t col = c < s.c0 ? cl[s.c0_off + c] : cl[s.c1_off + (c - s.c0)];
    for (int r = threadIdx.x; r < s.rows; r += blockDim.x) {
      const int32_t row = rl[s.r_off + r];
      M[s.moff + (int64_t)c * s.rows + r] = kentry(K, x[row], cx[row], xi[col]);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// host side
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  ~DevBuf() { if (p) cudaFree(p); }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n) return cudaSuccess;
    if (p) { cudaFree(p); p = nullptr; n = 0; }
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) n = bytes;
    return e;
  }
};

struct StepOut {
  int side = 0, s = 0;
  int64_t nid = 0;
  std::vector<int32_t> k, b;
  int32_t* d_list = nullptr;           // skeletons in list order
  std::vector<int64_t> list_off;       // [nid + 1], list order
  void* d_T = nullptr;                 // blocks in ID order
  std::vector<int64_t> T_off;          // [nid]
  int64_t T_len = 0;
  int32_t* d_idx = nullptr;
  std::vector<int64_t> idx_off;        // [nid]
  int64_t idx_len = 0;
  int saturated = 0;
};

struct Builder {
  Plan* p;
  KDesc K;
  idbf_params prm;
  cudaStream_t st;
  double *d_x = nullptr, *d_xi = nullptr, *d_cx = nullptr;
  std::vector<StepOut> U, V;  // index s - 1
  DevBuf A, blist, samp, pscr, descs, emits, kbuf, satbuf, Tb, Ib, Sb, lofs;
  size_t budget = 0;
  int sms = 152;

  ~Builder() {
    if (d_x) cudaFree(d_x);
    if (d_xi) cudaFree(d_xi);
    if (d_cx) cudaFree(d_cx);
    for (auto* v : {&U, &V})
      for (auto& o : *v) {
        if (o.d_list) cudaFree(o.d_list);
        if (o.d_T) cudaFree(o.d_T);
        if (o.d_idx) cudaFree(o.d_idx);
      }
  }

  // list-order position of ID id of step (side, s)
  int64_t list_pos(int side, int s, int64_t id) const {
    if (side == 1) return id;  // V: tau-major, natural
    const int L = p->L;
    const int64_t rho = id >> s, kappa = id & ((1LL << s) - 1);
    return kappa * (1LL << (L - s + 1)) + rho;  // U: kappa-major
  }

  idbf_status run_step(int side, int s);
  idbf_status assemble();
};

#define TRY_CUDA(x)                                                                          \
  do {                                                                                       \
    cudaError_t _e = (x);                                                                    \
    if (_e != cudaSuccess) {                                                                 \
      set_cuda_error(_e);                                                                    \
      return _e == cudaErrorMemoryAllocation ? IDBF_ENOMEM : IDBF_ECUDA;                     \
    }                                                                                        \
  } while (0)

static uint64_t splitmix64_host(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint64_t stream_key(uint64_t seed, int side, int step, int64_t node) {
  return splitmix64_host(splitmix64_host(seed) ^ ((uint64_t)side << 56) ^ ((uint64_t)step << 40) ^ (uint64_t)node);
}

idbf_status Builder::run_step(int side, int s) {
  const int L = p->L, n0 = p->n0;
  const int64_t N = p->N;
  // leaf j of the rows (x points) and of the columns (xi points): offsets when uneven
  auto row_leaf = [&](int64_t j, int64_t* first) -> int32_t {
    if (!p->uneven) { *first = j * n0; return n0; }
    *first = p->h_leaf_y[j];
    return (int32_t)(p->h_leaf_y[j + 1] - p->h_leaf_y[j]);
  };
  auto col_leaves = [&](int64_t j0, int64_t j1, int64_t* first) -> int64_t {  // leaves j0 .. j1-1
    if (!p->uneven) { *first = j0 * n0; return (j1 - j0) * n0; }
    *first = p->h_leaf_x[j0];
    return p->h_leaf_x[j1] - p->h_leaf_x[j0];
  };
  const int64_t nid = 2LL * p->m;
  StepOut out;
  out.side = side;
  out.s = s;
  out.nid = nid;
  out.k.assign(nid, 0);
  out.b.assign(nid, 0);
  // ---- descriptors
  std::vector<IDDesc> D(nid);
  const StepOut* prevU = s > 1 ? &U[s - 2] : nullptr;  // rhat_{s-1}
  const StepOut* prevV = s > 1 ? &V[s - 2] : nullptr;  // chat_{s-1}
  const StepOut* curU = side == 1 ? &U[s - 1] : nullptr;  // rhat_s for V step s
  const double t = (s == 1 && prm.oversample_leaf > 0) ? prm.oversample_leaf : prm.oversample;
  for (int64_t id = 0; id < nid; ++id) {
    IDDesc& d = D[id];
    memset(&d, 0, sizeof(d));
    if (side == 0) {
      const int64_t rho = id >> s, kappa = id & ((1LL << s) - 1);
      if (s == 1) {
        d.b = row_leaf(rho, &d.b_range);
        const int64_t half = p->m / 2;
        d.n_c = col_leaves(kappa * half, (kappa + 1) * half, &d.c_range);
      } else {
        const int64_t kp = kappa >> 1;
        const int64_t ia = list_pos(0, s - 1, (2 * rho) * (1LL << (s - 1)) + kp);
        const int64_t ib = list_pos(0, s - 1, (2 * rho + 1) * (1LL << (s - 1)) + kp);
        d.b_range = -1;
        d.b_a_off = prevU->list_off[ia];
        d.b_a = (int32_t)(prevU->list_off[ia + 1] - prevU->list_off[ia]);
        d.b_b_off = prevU->list_off[ib];
        d.b_b = (int32_t)(prevU->list_off[ib + 1] - prevU->list_off[ib]);
        d.b = d.b_a + d.b_b;
        const int sh = L - 2 * s + 2;
        const int64_t tau = rho >> sh;
        const int64_t lo = tau * (1LL << (L - s + 2)) + (kappa << sh), hi = lo + (1LL << sh);
        d.c_range = -1;
        d.c_off = prevV->list_off[lo];
        d.n_c = prevV->list_off[hi] - prevV->list_off[lo];
      }
      d.key = stream_key(prm.seed, 0, s, id);
    } else {
      const int64_t tau = id >> (L - s + 1), sigma = id & ((1LL << (L - s + 1)) - 1);
      if (s == 1) {
        d.b = (int32_t)col_leaves(sigma, sigma + 1, &d.b_range);
      } else {
        const int64_t ia = (tau >> 1) * (1LL << (L - s + 2)) + 2 * sigma;
        d.b_range = -1;
        d.b_a_off = prevV->list_off[ia];
        d.b_a = (int32_t)(prevV->list_off[ia + 1] - prevV->list_off[ia]);
        d.b_b_off = prevV->list_off[ia + 1];
        d.b_b = (int32_t)(prevV->list_off[ia + 2] - prevV->list_off[ia + 1]);
        d.b = d.b_a + d.b_b;
      }
      const int sh = L - 2 * s + 1;
      const int64_t kappa = sigma >> sh;
      const int64_t lo = kappa * (1LL << (L - s + 1)) + (tau << sh), hi = lo + (1LL << sh);
      d.c_range = -1;
      d.c_off = curU->list_off[lo];
      d.n_c = curU->list_off[hi] - curU->list_off[lo];
      d.key = stream_key(prm.seed, 1, s, id);
    }
    const int64_t kp = prm.rank_cap > 0 ? prm.rank_cap : std::min<int64_t>(d.b, d.n_c);
    const int64_t want = (int64_t)ceil(t * (double)kp);
    (void)N;
    d.ns = (int32_t)std::min<int64_t>(d.n_c, std::max<int64_t>(1, want));
    if (prm.sampling == IDBF_SAMPLE_ALL) d.ns = (int32_t)d.n_c;
    d.kmax = (int32_t)std::min<int64_t>(std::min<int64_t>(d.ns, d.b), kp);
    out.b[id] = d.b;
  }
  // ---- batches
  struct Batch { int64_t lo, hi; };
  std::vector<Batch> batches;
  {
    int64_t lo = 0, bytes = 0;
    for (int64_t id = 0; id < nid; ++id) {
      const int64_t need = (int64_t)D[id].ns * D[id].b * 16 + (int64_t)(2 * D[id].b + D[id].ns) * 4;
      if (id > lo && (bytes + need > (int64_t)budget || id - lo >= 65535)) {
        batches.push_back({lo, id});
        lo = id;
        bytes = 0;
      }
      bytes += need;
    }
    batches.push_back({lo, nid});
  }
  struct BatchRes { int64_t lo, hi; void* T; int32_t* I; int32_t* S; std::vector<int64_t> toff, ioff, soff; };
  std::vector<BatchRes> res;
  auto free_res = [&]() {
    for (auto& r : res) { if (r.T) cudaFree(r.T); if (r.I) cudaFree(r.I); if (r.S) cudaFree(r.S); }
    res.clear();
  };
  const int32_t* prev_list = side == 0 ? (s > 1 ? prevU->d_list : nullptr) : (s > 1 ? prevV->d_list : nullptr);
  const int32_t* cand_list = side == 0 ? (s > 1 ? prevV->d_list : nullptr) : curU->d_list;
  const double* cand_coord = side == 0 ? d_xi : d_x;
  for (const Batch& bt : batches) {
    const int64_t nb = bt.hi - bt.lo;
    std::vector<IDDesc> Db(D.begin() + bt.lo, D.begin() + bt.hi);
    int64_t a = 0, bo = 0, so = 0;
    int maxns = 1, maxb = 1;
    for (auto& d : Db) {
      d.a_off = a; a += (int64_t)d.ns * d.b;
      d.bl_off = bo; bo += d.b;
      d.sp_off = so; so += d.ns;
      maxns = std::max(maxns, d.ns);
      maxb = std::max(maxb, d.b);
    }
    cudaError_t e;
    if ((e = A.ensure(std::max<int64_t>(a, 1) * 16)) != cudaSuccess ||
        (e = blist.ensure(std::max<int64_t>(bo, 1) * 4)) != cudaSuccess ||
        (e = pscr.ensure(std::max<int64_t>(bo, 1) * 4)) != cudaSuccess ||
        (e = samp.ensure(std::max<int64_t>(so, 1) * 4)) != cudaSuccess ||
        (e = descs.ensure(nb * sizeof(IDDesc))) != cudaSuccess ||
        (e = kbuf.ensure(nb * 4)) != cudaSuccess || (e = satbuf.ensure(nb * 4)) != cudaSuccess) {
      free_res();
      set_cuda_error(e);
      return IDBF_ENOMEM;
    }
    IDDesc* dD = (IDDesc*)descs.p;
    TRY_CUDA(cudaMemcpyAsync(dD, Db.data(), nb * sizeof(IDDesc), cudaMemcpyHostToDevice, st));
    k_make_blist<<<(unsigned)nb, 128, 0, st>>>(dD, prev_list, (int32_t*)blist.p);
    TRY_CUDA(cudaGetLastError());
    // sampling: one ID per warp; hash capacity a power of two >= 4 ns (load factor <= 1/2)
    int cap = 64;
    while (cap < 4 * maxns) cap <<= 1;
    const size_t per_warp = ((size_t)cap * 2 + maxns) * 4;
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(4, (200u * 1024) / per_warp));
    const size_t smS = (size_t)wpb * per_warp;
    if (smS > 200 * 1024) { free_res(); return IDBF_EUNSUPPORTED; }
    TRY_CUDA(cudaFuncSetAttribute(k_sample, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smS));
    k_sample<<<(unsigned)((nb + wpb - 1) / wpb), wpb * 32, smS, st>>>(dD, nb, cand_list, cand_coord, (int32_t*)samp.p,
                                                                    prm.sampling, cap, maxns);
    TRY_CUDA(cudaGetLastError());
    dim3 gf((unsigned)nb, (unsigned)std::min(maxb, 64));
    const bool df = prm.qr_arith == IDBF_QR_DF64;
    if (df) k_fill<true><<<gf, 256, 0, st>>>(dD, (int32_t*)blist.p, (int32_t*)samp.p, d_x, d_cx, d_xi, (double2*)A.p, K, side);
    else k_fill<false><<<gf, 256, 0, st>>>(dD, (int32_t*)blist.p, (int32_t*)samp.p, d_x, d_cx, d_xi, (double2*)A.p, K, side);
    TRY_CUDA(cudaGetLastError());
    const size_t smQ = (size_t)maxns * 16 + (size_t)maxb * 12 + 16;
    if (smQ > 200 * 1024) { free_res(); return IDBF_EUNSUPPORTED; }
    if (df) {
      TRY_CUDA(cudaFuncSetAttribute(k_qr_df<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smQ));
      k_qr_df<256><<<(unsigned)nb, 256, smQ, st>>>(dD, (double2*)A.p, (int32_t*)pscr.p, (int32_t*)kbuf.p,
                                                  (int32_t*)satbuf.p, prm.eps);
    } else {
      TRY_CUDA(cudaFuncSetAttribute(k_qr<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smQ));
      k_qr<256><<<(unsigned)nb, 256, smQ, st>>>(dD, (double2*)A.p, (int32_t*)pscr.p, (int32_t*)kbuf.p,
                                               (int32_t*)satbuf.p, prm.eps);
    }
    TRY_CUDA(cudaGetLastError());
    std::vector<int32_t> kb(nb), sb(nb);
    TRY_CUDA(cudaMemcpyAsync(kb.data(), kbuf.p, nb * 4, cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaMemcpyAsync(sb.data(), satbuf.p, nb * 4, cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaStreamSynchronize(st));
    BatchRes r;
    r.lo = bt.lo; r.hi = bt.hi; r.T = nullptr; r.I = nullptr; r.S = nullptr;
    std::vector<EmitDesc> E(nb);
    int64_t to = 0, io = 0, sk = 0;
    int maxk = 1;
    for (int64_t i = 0; i < nb; ++i) {
      const int k = kb[i], b = Db[i].b;
      out.k[bt.lo + i] = k;
      out.saturated += sb[i];
      E[i].t_off = to; to += (int64_t)k * (b - k);
      E[i].i_off = io; io += b;
      E[i].s_off = sk; sk += k;
      maxk = std::max(maxk, k);
      r.toff.push_back(E[i].t_off); r.ioff.push_back(E[i].i_off); r.soff.push_back(E[i].s_off);
    }
    r.toff.push_back(to); r.ioff.push_back(io); r.soff.push_back(sk);
    cudaError_t e1 = cudaMalloc(&r.T, std::max<int64_t>(to, 1) * 16);
    cudaError_t e2 = cudaMalloc((void**)&r.I, std::max<int64_t>(io, 1) * 4);
    cudaError_t e3 = cudaMalloc((void**)&r.S, std::max<int64_t>(sk, 1) * 4);
    res.push_back(r);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) { free_res(); cudaGetLastError(); return IDBF_ENOMEM; }
    if ((e = emits.ensure(nb * sizeof(EmitDesc))) != cudaSuccess) { free_res(); return IDBF_ENOMEM; }
    TRY_CUDA(cudaMemcpyAsync(emits.p, E.data(), nb * sizeof(EmitDesc), cudaMemcpyHostToDevice, st));
    auto emit = df ? k_emit<true> : k_emit<false>;
    emit<<<(unsigned)nb, 256, (size_t)maxk * 8, st>>>(dD, (EmitDesc*)emits.p, (double2*)A.p, (int32_t*)pscr.p,
                                                    (int32_t*)blist.p, (int32_t*)kbuf.p, (double2*)res.back().T,
                                                    res.back().I, res.back().S, side);
    TRY_CUDA(cudaGetLastError());
    TRY_CUDA(cudaStreamSynchronize(st));
  }
  // ---- concatenate the batches: blocks and index lists in ID order, skeletons in list order
  out.T_off.assign(nid, 0);
  out.idx_off.assign(nid, 0);
  for (int64_t id = 0; id < nid; ++id) {
    out.T_off[id] = out.T_len;
    out.T_len += (int64_t)out.k[id] * (out.b[id] - out.k[id]);
    out.idx_off[id] = out.idx_len;
    out.idx_len += out.b[id];
  }
  out.list_off.assign(nid + 1, 0);
  std::vector<int32_t> klist(nid);
  for (int64_t id = 0; id < nid; ++id) klist[list_pos(side, s, id)] = out.k[id];
  for (int64_t i = 0; i < nid; ++i) out.list_off[i + 1] = out.list_off[i] + klist[i];
  cudaError_t e1 = cudaMalloc(&out.d_T, std::max<int64_t>(out.T_len, 1) * 16);
  // +16 bytes: the apply copies index lists in 16-byte granules and may read up to 12 bytes past the end
  cudaError_t e2 = cudaMalloc((void**)&out.d_idx, std::max<int64_t>(out.idx_len, 1) * 4 + 16);
  cudaError_t e3 = cudaMalloc((void**)&out.d_list, std::max<int64_t>(out.list_off[nid], 1) * 4);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    cudaGetLastError();
    free_res();
    if (out.d_T) cudaFree(out.d_T);
    if (out.d_idx) cudaFree(out.d_idx);
    if (out.d_list) cudaFree(out.d_list);
    return IDBF_ENOMEM;
  }
  std::vector<int64_t> srcoff(nid), dstoff(nid);
  std::vector<int32_t> lens(nid);
  int64_t sbase = 0;
  for (auto& r : res) {
    const int64_t nb = r.hi - r.lo;
    TRY_CUDA(cudaMemcpyAsync((double2*)out.d_T + out.T_off[r.lo], r.T, r.toff[nb] * 16, cudaMemcpyDeviceToDevice, st));
    TRY_CUDA(cudaMemcpyAsync(out.d_idx + out.idx_off[r.lo], r.I, r.ioff[nb] * 4, cudaMemcpyDeviceToDevice, st));
    (void)sbase;
  }
  // skeletons: gather each batch's lists into list order
  for (auto& r : res) {
    const int64_t nb = r.hi - r.lo;
    for (int64_t i = 0; i < nb; ++i) {
      const int64_t id = r.lo + i;
      srcoff[id] = r.soff[i];
      dstoff[id] = out.list_off[list_pos(side, s, id)];
      lens[id] = out.k[id];
    }
    cudaError_t e;
    if ((e = lofs.ensure(nb * (8 + 8 + 4))) != cudaSuccess) { free_res(); return IDBF_ENOMEM; }
    char* q = (char*)lofs.p;
    TRY_CUDA(cudaMemcpyAsync(q, srcoff.data() + r.lo, nb * 8, cudaMemcpyHostToDevice, st));
    TRY_CUDA(cudaMemcpyAsync(q + nb * 8, dstoff.data() + r.lo, nb * 8, cudaMemcpyHostToDevice, st));
    TRY_CUDA(cudaMemcpyAsync(q + nb * 16, lens.data() + r.lo, nb * 4, cudaMemcpyHostToDevice, st));
    k_gather_lists<<<(unsigned)nb, 128, 0, st>>>(r.S, (int64_t*)q, (int64_t*)(q + nb * 8), (int32_t*)(q + nb * 16), out.d_list);
    TRY_CUDA(cudaGetLastError());
    TRY_CUDA(cudaStreamSynchronize(st));
  }
  free_res();
  (side == 0 ? U : V).push_back(std::move(out));
  return IDBF_OK;
}

// Turn the step results into the butterfly layout of the plan (include/idbf.h).
idbf_status Builder::assemble() {
  Plan& P = *p;
  const int L = P.L, hV = P.hV, hU = P.hU;
  const int64_t m = P.m, nbl = 2 * m;
  P.init_levels();
  P.h_rows.assign((L + 1) * nbl, 0);
  P.h_cols.assign((L + 1) * nbl, 0);
  P.h_moff.assign((L + 1) * nbl, 0);
  P.h_ioff.assign((L + 1) * nbl, 0);
  P.h_seg_len.assign((int64_t)L * nbl, 0);
  // segment lengths: boundary b < hV: z_{b+1} (V step b+1, id order); b >= hV: w_s, s = hU - (b - hV)
  for (int b = 0; b < L; ++b) {
    const StepOut& o = b < hV ? V[b] : U[hU - (b - hV) - 1];
    for (int64_t i = 0; i < nbl; ++i) P.h_seg_len[b * nbl + i] = o.k[i];
  }
  for (int l = 0; l <= L; ++l) {
    if (l == hV) continue;
    const bool isV = l < hV;
    StepOut& o = isV ? V[l] : U[hU - (l - hV - 1) - 1];
    const int s = o.s;
    for (int64_t j = 0; j < m; ++j)
      for (int c = 0; c < 2; ++c) {
        int64_t id;
        if (isV) {
          const int64_t H = 1LL << (L - s + 1);
          id = (j / H) * 2 * H + j % H + c * H;  // (2 tau_p + c) H + sigma
        } else {
          id = 2 * j + c;                         // rho 2^s + 2 kappa_p + c
        }
        const int64_t ob = l * nbl + 2 * j + c;
        const int k = o.k[id], b = o.b[id];
        P.h_rows[ob] = isV ? k : b - k;
        P.h_cols[ob] = isV ? b - k : k;
        P.h_moff[ob] = o.T_off[id];
        P.h_ioff[ob] = o.idx_off[id];
      }
    P.lmat_len[l] = o.T_len;
    P.lidx_len[l] = o.idx_len;
    P.lmat[IDBF_STORE_C128][l] = o.T_len > 0 ? o.d_T : nullptr;
    if (o.T_len == 0 && o.d_T) cudaFree(o.d_T);
    o.d_T = nullptr;
    P.lidx[l] = o.d_idx;
    o.d_idx = nullptr;
    P.mat_len += o.T_len;
    P.idx_len += o.idx_len;
  }
  // middle factor
  {
    const StepOut& u = U[hU - 1];
    const StepOut& v = V[hV - 1];
    std::vector<SDesc> Sd(nbl);
    int64_t tot = 0;
    int maxcols = 1;
    for (int64_t j = 0; j < m; ++j)
      for (int c = 0; c < 2; ++c) {
        const int64_t tau = j >> hU, kappa = j & ((1LL << hU) - 1);
        const int64_t rho = 2 * tau + c;
        SDesc& d = Sd[2 * j + c];
        const int64_t ru = list_pos(0, hU, rho * (1LL << hU) + kappa);
        d.r_off = u.list_off[ru];
        d.rows = (int32_t)(u.list_off[ru + 1] - u.list_off[ru]);
        const int64_t v0 = tau * (1LL << (hU + 1)) + 2 * kappa;  // chat(tau, 2kappa), V step hV ids
        d.c0_off = v.list_off[v0];
        d.c0 = (int32_t)(v.list_off[v0 + 1] - v.list_off[v0]);
        d.c1_off = v.list_off[v0 + 1];
        d.c1 = (int32_t)(v.list_off[v0 + 2] - v.list_off[v0 + 1]);
        d.moff = tot;
        const int64_t ob = hV * nbl + 2 * j + c;
        P.h_rows[ob] = d.rows;
        P.h_cols[ob] = d.c0 + d.c1;
        P.h_moff[ob] = tot;
        P.h_ioff[ob] = 0;
        tot += (int64_t)d.rows * (d.c0 + d.c1);
        maxcols = std::max(maxcols, d.c0 + d.c1);
      }
    void* M = nullptr;
    TRY_CUDA(cudaMalloc(&M, std::max<int64_t>(tot, 1) * 16));
    P.lmat[IDBF_STORE_C128][hV] = M;
    P.lmat_len[hV] = tot;
    P.mat_len += tot;
    DevBuf sd;
    TRY_CUDA(sd.ensure(nbl * sizeof(SDesc)));
    TRY_CUDA(cudaMemcpyAsync(sd.p, Sd.data(), nbl * sizeof(SDesc), cudaMemcpyHostToDevice, st));
    dim3 g((unsigned)nbl, (unsigned)std::min(maxcols, 64));
    k_fill_S<<<g, 128, 0, st>>>((SDesc*)sd.p, u.d_list, v.d_list, d_x, d_cx, d_xi, (double2*)M, K);
    TRY_CUDA(cudaGetLastError());
    TRY_CUDA(cudaStreamSynchronize(st));
  }
  finalize_structure(&P);
  return upload_structure(&P, st);
}

// dense ground-truth rows: y[r] = sum_j K(x[rows[r]], xi[j]) v[j], FP64, a block per row
__global__ void k_dense_rows(KDesc K, const double* __restrict__ x, const double* __restrict__ xi, int64_t N,
                             const int64_t* __restrict__ rows, const double2* __restrict__ v, double2* __restrict__ y) {
  __shared__ double2 red[32];
  const int64_t r = rows[blockIdx.x];
  const double xr = x[r];
  double c = 0.0;
  if (K.kind == IDBF_KERNEL_FIO1D) {
    if (K.prof == 0) c = (2.0 + sinpi(2.0 * xr) * sinpi(4.0 * xr)) / 3.0;
    else if (K.prof == 1) c = (2.0 + 0.2 * sinpi(2.0 * xr)) / 16.0;
  }
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
    const double2 k = kentry(K, xr, c, xi[j]);
    const double2 b = v[j];
    acc.x = fma(k.x, b.x, fma(-k.y, b.y, acc.x));
    acc.y = fma(k.x, b.y, fma(k.y, b.x, acc.y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = make_double2(0.0, 0.0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t.x += red[w].x; t.y += red[w].y; }
    y[blockIdx.x] = t;
  }
}

}  // namespace bld
}  // namespace idbf

using namespace idbf;

extern "C" idbf_status idbf_kernel_matvec_rows(const idbf_kernel* kernel, const double* x, const double* xi, int64_t N,
                                               const int64_t* rows, int64_t nrows, const void* v, void* y,
                                               void* stream) {
  if (!kernel || !x || !xi || !rows || !v || !y || N < 1 || nrows < 0 || nrows > (1LL << 31) - 1) return IDBF_EINVAL;
  if (kernel->kind != IDBF_KERNEL_FIO1D && kernel->kind != IDBF_KERNEL_DFT && kernel->kind != IDBF_KERNEL_J0)
    return IDBF_EINVAL;
  if (nrows == 0) return IDBF_OK;
  bld::KDesc K{kernel->kind, kernel->sign, kernel->c_profile};
  bld::k_dense_rows<<<(unsigned)nrows, 256, 0, (cudaStream_t)stream>>>(K, x, xi, N, rows, (const double2*)v, (double2*)y);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_cuda_error(e); return IDBF_ECUDA; }
  return IDBF_OK;
}

// The construction for uniform leaves (ro = co = nullptr, leaf size params->leaf) or for leaves
// given by offsets (2^L + 1 each; params->leaf unused).
static idbf_status build_plan(const idbf_kernel* kernel, const double* x_host, const double* xi_host, int64_t N,
                              int L, const int64_t* ro, const int64_t* co, const idbf_params* params, void* stream,
                              idbf_plan* out) {
  if (!out) return IDBF_EINVAL;
  *out = nullptr;
  if (!kernel || !x_host || !xi_host || !params) return IDBF_EINVAL;
  const idbf_params& pr = *params;
  const bool uneven = ro != nullptr;
  if (N < 1 || N > (1LL << 31) - 1 || L < 2 || L > 30) return IDBF_EINVAL;
  const int64_t m = 1LL << L;
  if (!uneven && (pr.leaf < 1 || N != (int64_t)pr.leaf * m)) return IDBF_EINVAL;
  if (uneven) {
    for (const int64_t* o : {ro, co}) {
      if (o[0] != 0 || o[m] != N) return IDBF_EINVAL;
      for (int64_t j = 0; j < m; ++j)
        if (o[j + 1] < o[j]) return IDBF_EINVAL;
    }
  }
  if (!(pr.eps >= 0.0) || !(pr.oversample >= 1.0) || pr.rank_cap < 0 || pr.sampling < 0 || pr.sampling > 2 ||
      pr.storage < 0 || pr.storage > 2 || (pr.qr_arith != IDBF_QR_FP64 && pr.qr_arith != IDBF_QR_DF64))
    return IDBF_EINVAL;
  if (kernel->kind == IDBF_KERNEL_FIO1D) {
    if (kernel->c_profile < 0 || kernel->c_profile > 2) return IDBF_EINVAL;
  } else if (kernel->kind == IDBF_KERNEL_DFT) {
    if (kernel->sign != 1 && kernel->sign != -1) return IDBF_EINVAL;
  } else if (kernel->kind != IDBF_KERNEL_J0) {
    return IDBF_EINVAL;
  }
  for (int64_t i = 1; i < N; ++i)
    if (!(x_host[i] >= x_host[i - 1]) || !(xi_host[i] >= xi_host[i - 1])) return IDBF_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  idbf_plan_s* h = new (std::nothrow) idbf_plan_s();
  if (!h) return IDBF_ENOMEM;
  Plan& P = h->p;
  cudaGetDevice(&P.device);
  P.N = N;
  P.n0 = uneven ? 0 : pr.leaf;
  P.L = L;
  P.m = (int)m; P.hV = P.L / 2; P.hU = P.L - P.hV;
  P.uneven = uneven;
  if (uneven) {
    P.h_leaf_x.assign(co, co + m + 1);  // columns: the leaves of the vector x that K multiplies
    P.h_leaf_y.assign(ro, ro + m + 1);  // rows: the leaves of y
  }
  P.init_levels();
  idbf_status s = IDBF_OK;
  {
    bld::Builder B;
    B.p = &P;
    B.K = {kernel->kind, kernel->sign, kernel->c_profile};
    B.prm = pr;
    B.st = (cudaStream_t)stream;
    cudaDeviceGetAttribute(&B.sms, cudaDevAttrMultiProcessorCount, P.device);
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    B.budget = std::max<size_t>(256u << 20, std::min<size_t>(fr / 4, (size_t)24 << 30));
    cudaError_t e = cudaMalloc((void**)&B.d_x, N * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&B.d_xi, N * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&B.d_cx, N * 8);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.d_x, x_host, N * 8, cudaMemcpyHostToDevice, B.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.d_xi, xi_host, N * 8, cudaMemcpyHostToDevice, B.st);
    if (e != cudaSuccess) { set_cuda_error(e); s = e == cudaErrorMemoryAllocation ? IDBF_ENOMEM : IDBF_ECUDA; }
    if (s == IDBF_OK) {
      bld::k_cprofile<<<256, 256, 0, B.st>>>(B.d_x, B.d_cx, N, kernel->kind == IDBF_KERNEL_FIO1D ? kernel->c_profile : 2);
      e = cudaGetLastError();
      if (e != cudaSuccess) { set_cuda_error(e); s = IDBF_ECUDA; }
    }
    for (int st = 1; st <= P.hU && s == IDBF_OK; ++st) {
      s = B.run_step(0, st);
      if (s == IDBF_OK && st <= P.hV) s = B.run_step(1, st);
    }
    if (s == IDBF_OK) s = B.assemble();
    if (s == IDBF_OK) {
      for (auto& o : B.U) P.rank_saturated += o.saturated;
      for (auto& o : B.V) P.rank_saturated += o.saturated;
    }
  }
  if (s == IDBF_OK && pr.storage != IDBF_STORE_C128) s = convert_storage(&P, 1u << pr.storage, (cudaStream_t)stream);
  if (s == IDBF_OK) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) { set_cuda_error(e); s = IDBF_ECUDA; }
  }
  if (s != IDBF_OK) {
    idbf_destroy(h);
    return s;
  }
  P.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = h;
  return P.rank_saturated > 0 ? IDBF_ERANKCAP : IDBF_OK;
}

extern "C" idbf_status idbf_build(const idbf_kernel* kernel, const double* x_host, const double* xi_host, int64_t N,
                                  const idbf_params* params, void* stream, idbf_plan* out) {
  if (!out) return IDBF_EINVAL;
  *out = nullptr;
  if (!params || params->leaf < 1 || N < 4 * (int64_t)params->leaf || N % params->leaf) return IDBF_EINVAL;
  const int64_t m = N / params->leaf;
  if (m & (m - 1)) return IDBF_EINVAL;
  int L = 0;
  while ((1LL << L) < m) ++L;
  return build_plan(kernel, x_host, xi_host, N, L, nullptr, nullptr, params, stream, out);
}

extern "C" idbf_status idbf_build_leaves(const idbf_kernel* kernel, const double* x_host, const double* xi_host,
                                         int64_t N, int32_t L, const int64_t* row_leaf_off,
                                         const int64_t* col_leaf_off, const idbf_params* params, void* stream,
                                         idbf_plan* out) {
  if (!out) return IDBF_EINVAL;
  *out = nullptr;
  if (!row_leaf_off || !col_leaf_off) return IDBF_EINVAL;
  return build_plan(kernel, x_host, xi_host, N, L, row_leaf_off, col_leaf_off, params, stream, out);
}

extern "C" idbf_status idbf_dyadic_leaves(const double* points, int64_t n, double lo, double hi, int32_t L,
                                          int64_t* off) {
  if (!off || n < 0 || (n > 0 && !points) || L < 0 || L > 30 || !(hi > lo)) return IDBF_EINVAL;
  for (int64_t i = 0; i < n; ++i)
    if (!(points[i] >= lo) || !(points[i] < hi) || (i > 0 && !(points[i] >= points[i - 1]))) return IDBF_EINVAL;
  const int64_t m = 1LL << L;
  // edge j = lo + (hi - lo) (j / 2^L); off[j] = number of points below edge j (binary search)
  for (int64_t j = 0; j < m; ++j) {
    const double edge = lo + (hi - lo) * ((double)j / (double)m);
    int64_t a = 0, b = n;
    while (a < b) {
      const int64_t mid = (a + b) / 2;
      if (points[mid] < edge) a = mid + 1; else b = mid;
    }
    off[j] = a;
  }
  off[m] = n;
  return IDBF_OK;
}
