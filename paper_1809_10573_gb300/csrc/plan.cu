// Plan lifecycle, factor import, storage formats, statistics and checkpoints.
//
// The factors are held in the butterfly layout documented in include/idbf.h: L + 1 levels of
// m nodes with two dense blocks each (T blocks of the column IDs on the V side, the middle
// factor S, T^T blocks of the row IDs on the U side; Secs. 2.1-2.4 of the paper). On the
// device every block is stored column-major, M(r, j) at offset j * rows + r, so that the
// threads of a forward level kernel, one per output row, read consecutive addresses.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "idbf_internal.h"

namespace idbf {

static thread_local char g_last_cuda[256] = "";

void set_cuda_error(cudaError_t e) {
  snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
}

DevLevel Plan::level(int l) const {
  DevLevel d;
  d.kind = lv[l].kind;
  d.lev = l;
  d.L = L;
  d.H = (int)(1LL << (L - l));
  d.m = m;
  d.n0 = n0;
  const int64_t nb = (int64_t)m * 2;
  d.rows = d_rows + l * nb;
  d.cols = d_cols + l * nb;
  d.moff = d_moff + l * nb;
  d.ioff = d_ioff + l * nb;
  d.idx = lidx[l];
  d.in_off = l > 0 ? d_seg_off + (l - 1) * nb : nullptr;
  d.in_len = l > 0 ? d_seg_len + (l - 1) * nb : nullptr;
  d.out_off = l < L ? d_seg_off + l * nb : nullptr;
  d.out_len = l < L ? d_seg_len + l * nb : nullptr;
  d.leaf = !uneven ? nullptr : l == 0 ? d_leaf : l == L ? d_leaf + (m + 1) : nullptr;
  return d;
}

size_t Plan::device_bytes() const {
  size_t b = ws_bytes;
  const int64_t nb = (int64_t)(L + 1) * m * 2;
  b += nb * (2 * sizeof(int32_t) + 2 * sizeof(int64_t));
  b += (size_t)L * 2 * m * (sizeof(int32_t) + sizeof(int64_t));
  b += idx_len * sizeof(int32_t);
  if (uneven) b += 2 * (size_t)(m + 1) * sizeof(int64_t);
  for (int f = 0; f < 3; ++f)
    for (int l = 0; l <= L && l < (int)lmat[f].size(); ++l)
      if (lmat[f][l]) b += lmat_len[l] * (f == IDBF_STORE_C64 ? 8 : 16);
  return b;
}

bool Plan::has_format(int f) const {
  for (int l = 0; l <= L; ++l)
    if (lmat_len[l] > 0 && !lmat[f][l]) return false;
  return true;
}

void Plan::init_levels() {
  lmat_len.assign(L + 1, 0);
  lidx_len.assign(L + 1, 0);
  for (int f = 0; f < 3; ++f) lmat[f].assign(L + 1, nullptr);
  lidx.assign(L + 1, nullptr);
}

idbf_status finalize_structure(Plan* p) {
  const int64_t m = p->m;
  p->h_seg_off.assign((size_t)p->L * 2 * m, 0);
  p->seg_total.assign(p->L, 0);
  p->max_seg_total = 0;
  for (int b = 0; b < p->L; ++b) {
    int64_t acc = 0;
    for (int64_t i = 0; i < 2 * m; ++i) {
      p->h_seg_off[b * 2 * m + i] = acc;
      acc += p->h_seg_len[b * 2 * m + i];
    }
    p->seg_total[b] = acc;
    p->max_seg_total = std::max(p->max_seg_total, acc);
  }
  p->lv.assign(p->L + 1, LevelInfo());
  for (int l = 0; l <= p->L; ++l) {
    LevelInfo& li = p->lv[l];
    li.kind = l < p->hV ? KIND_V : (l == p->hV ? KIND_S : KIND_U);
    const int64_t H = 1LL << (p->L - l);
    li.kmin = 1 << 30;
    for (int64_t j = 0; j < m; ++j) {
      const int64_t o = (l * m + j) * 2;
      const int leaf_x = p->uneven ? (int)(p->h_leaf_x[j + 1] - p->h_leaf_x[j]) : p->n0;
      const int leaf_y = p->uneven ? (int)(p->h_leaf_y[j + 1] - p->h_leaf_y[j]) : p->n0;
      int in = l == 0 ? leaf_x : p->h_seg_len[(l - 1) * 2 * m + 2 * j] + p->h_seg_len[(l - 1) * 2 * m + 2 * j + 1];
      int out = 0;
      if (l == p->L) {
        out = leaf_y;
        li.kmin = std::min(li.kmin, leaf_y);
        li.kmax = std::max(li.kmax, leaf_y);
      } else {
        for (int c = 0; c < 2; ++c) {
          const int64_t s = (j / H) * 2 * H + j % H + c * H;
          const int len = p->h_seg_len[l * 2 * m + s];
          out += len;
          li.kmin = std::min(li.kmin, len);
          li.kmax = std::max(li.kmax, len);
        }
      }
      li.max_rows_pair = std::max(li.max_rows_pair, p->h_rows[o] + p->h_rows[o + 1]);
      li.max_cols_pair = std::max(li.max_cols_pair, p->h_cols[o] + p->h_cols[o + 1]);
      li.max_in = std::max(li.max_in, in);
      li.max_out = std::max(li.max_out, out);
      for (int c = 0; c < 2; ++c) {
        li.entries += (int64_t)p->h_rows[o + c] * p->h_cols[o + c];
        li.max_rows = std::max(li.max_rows, p->h_rows[o + c]);
        li.max_cols = std::max(li.max_cols, p->h_cols[o + c]);
        if (li.kind == KIND_V) li.idx_entries += p->h_rows[o + c] + p->h_cols[o + c];
        if (li.kind == KIND_U) li.idx_entries += p->h_rows[o + c] + p->h_cols[o + c];
      }
    }
    if (li.kmin > li.kmax) li.kmin = li.kmax;
  }
  return IDBF_OK;
}

idbf_status upload_structure(Plan* p, cudaStream_t st) {
  const int64_t nb = (int64_t)(p->L + 1) * p->m * 2;
  const int64_t ns = (int64_t)p->L * 2 * p->m;
  size_t bytes = nb * (2 * sizeof(int32_t) + 2 * sizeof(int64_t)) + ns * (sizeof(int32_t) + sizeof(int64_t));
  IDBF_CUDA_TRY(cudaMalloc(&p->d_meta, bytes));
  char* q = (char*)p->d_meta;
  p->d_moff = (int64_t*)q; q += nb * sizeof(int64_t);
  p->d_ioff = (int64_t*)q; q += nb * sizeof(int64_t);
  p->d_seg_off = (int64_t*)q; q += ns * sizeof(int64_t);
  p->d_rows = (int32_t*)q; q += nb * sizeof(int32_t);
  p->d_cols = (int32_t*)q; q += nb * sizeof(int32_t);
  p->d_seg_len = (int32_t*)q;
  IDBF_CUDA_TRY(cudaMemcpyAsync(p->d_moff, p->h_moff.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  IDBF_CUDA_TRY(cudaMemcpyAsync(p->d_ioff, p->h_ioff.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  IDBF_CUDA_TRY(cudaMemcpyAsync(p->d_seg_off, p->h_seg_off.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  IDBF_CUDA_TRY(cudaMemcpyAsync(p->d_rows, p->h_rows.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  IDBF_CUDA_TRY(cudaMemcpyAsync(p->d_cols, p->h_cols.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  IDBF_CUDA_TRY(cudaMemcpyAsync(p->d_seg_len, p->h_seg_len.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if (p->uneven && !p->d_leaf) {
    const size_t lb = 2 * (size_t)(p->m + 1) * sizeof(int64_t);
    IDBF_CUDA_TRY(cudaMalloc((void**)&p->d_leaf, lb));
    IDBF_CUDA_TRY(cudaMemcpyAsync(p->d_leaf, p->h_leaf_x.data(), (p->m + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    IDBF_CUDA_TRY(cudaMemcpyAsync(p->d_leaf + p->m + 1, p->h_leaf_y.data(), (p->m + 1) * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, st));
  }
  if (!p->d_status) {
    IDBF_CUDA_TRY(cudaMalloc((void**)&p->d_status, sizeof(int)));
    IDBF_CUDA_TRY(cudaMemsetAsync(p->d_status, 0, sizeof(int), st));
  }
  return IDBF_OK;
}

// ---- storage conversion kernels ------------------------------------------------------------
// double-float split of a binary64 value: hi = fl32(d), lo = fl32(d - hi); hi + lo carries
// 48 significant bits (Dekker 1971 double-length representation with binary32 parts).
__global__ void k_c128_to_df64(const double2* __restrict__ src, float4* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    const float rh = (float)v.x, ih = (float)v.y;
    dst[i] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
  }
}
__global__ void k_df64_to_c128(const float4* __restrict__ src, double2* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = src[i];
    dst[i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
  }
}
__global__ void k_c128_to_c64(const double2* __restrict__ src, float2* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    dst[i] = make_float2((float)v.x, (float)v.y);
  }
}
__global__ void k_df64_to_c64(const float4* __restrict__ src, float2* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = src[i];
    dst[i] = make_float2((float)((double)v.x + (double)v.y), (float)((double)v.z + (double)v.w));
  }
}
// In place: each thread reads its element before writing the same element (same 16 bytes).
__global__ void k_c128_to_df64_inplace(void* buf, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = ((const double2*)buf)[i];
    const float rh = (float)v.x, ih = (float)v.y;
    ((float4*)buf)[i] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
  }
}
__global__ void k_df64_to_c128_inplace(void* buf, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = ((const float4*)buf)[i];
    ((double2*)buf)[i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
  }
}

static int conv_grid(int64_t n) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
}

static idbf_status convert_level(Plan* p, int l, uint32_t mask, cudaStream_t st) {
  const int64_t n = p->lmat_len[l];
  void** m = nullptr;
  void* mm[3] = {p->lmat[0][l], p->lmat[1][l], p->lmat[2][l]};
  m = mm;
  const bool has128 = m[IDBF_STORE_C128], hasdf = m[IDBF_STORE_DF64];
  const bool want128 = mask & (1u << IDBF_STORE_C128), wantdf = mask & (1u << IDBF_STORE_DF64),
             want64 = mask & (1u << IDBF_STORE_C64);
  if (n > 0) {
    if (!has128 && !hasdf) return IDBF_EUNSUPPORTED;  // C64 alone cannot be widened
    const int g = conv_grid(n);
    if (want64 && !m[IDBF_STORE_C64]) {
      void* d = nullptr;
      IDBF_CUDA_TRY(cudaMalloc(&d, n * sizeof(float2) + 16));  // 16 B tail: bulk copies round up to 16 B
      if (has128) k_c128_to_c64<<<g, 256, 0, st>>>((const double2*)m[IDBF_STORE_C128], (float2*)d, n);
      else k_df64_to_c64<<<g, 256, 0, st>>>((const float4*)m[IDBF_STORE_DF64], (float2*)d, n);
      IDBF_CUDA_TRY(cudaGetLastError());
      m[IDBF_STORE_C64] = d;
    }
    if (want128 && wantdf && !(has128 && hasdf)) {
      void* d = nullptr;
      IDBF_CUDA_TRY(cudaMalloc(&d, n * 16));
      if (has128) { k_c128_to_df64<<<g, 256, 0, st>>>((const double2*)m[IDBF_STORE_C128], (float4*)d, n); m[IDBF_STORE_DF64] = d; }
      else { k_df64_to_c128<<<g, 256, 0, st>>>((const float4*)m[IDBF_STORE_DF64], (double2*)d, n); m[IDBF_STORE_C128] = d; }
      IDBF_CUDA_TRY(cudaGetLastError());
    } else if (want128 && !has128) {  // only DF64 present: convert in place
      k_df64_to_c128_inplace<<<g, 256, 0, st>>>(m[IDBF_STORE_DF64], n);
      IDBF_CUDA_TRY(cudaGetLastError());
      m[IDBF_STORE_C128] = m[IDBF_STORE_DF64];
      m[IDBF_STORE_DF64] = nullptr;
    } else if (wantdf && !hasdf) {  // only C128 present: convert in place
      k_c128_to_df64_inplace<<<g, 256, 0, st>>>(m[IDBF_STORE_C128], n);
      IDBF_CUDA_TRY(cudaGetLastError());
      m[IDBF_STORE_DF64] = m[IDBF_STORE_C128];
      m[IDBF_STORE_C128] = nullptr;
    }
    IDBF_CUDA_TRY(cudaStreamSynchronize(st));
  }
  for (int f = 0; f < 3; ++f) {
    if (!(mask & (1u << f)) && m[f]) {
      IDBF_CUDA_TRY(cudaFree(m[f]));
      m[f] = nullptr;
    }
    p->lmat[f][l] = m[f];
  }
  return IDBF_OK;
}

idbf_status convert_storage(Plan* p, uint32_t mask, cudaStream_t st) {
  for (int l = 0; l <= p->L; ++l) {
    idbf_status s = convert_level(p, l, mask, st);
    if (s != IDBF_OK) return s;
  }
  return IDBF_OK;
}

// ---- import ---------------------------------------------------------------------------------
static bool is_perm(const int32_t* a, int64_t na, const int32_t* b, int64_t nb, int64_t n, std::vector<char>& seen) {
  if (na + nb != n) return false;
  seen.assign(n, 0);
  for (int64_t i = 0; i < na; ++i) { if (a[i] < 0 || a[i] >= n || seen[a[i]]) return false; seen[a[i]] = 1; }
  for (int64_t i = 0; i < nb; ++i) { if (b[i] < 0 || b[i] >= n || seen[b[i]]) return false; seen[b[i]] = 1; }
  return true;
}

// Leaf offsets of an import: both NULL (leaves of n0 points) or both valid (m + 1 entries rising
// from 0 to N). Sets *uniform_n0 to the common leaf size when every leaf has the same positive size
// (the uniform case, whatever way it was given), else to 0.
static idbf_status leaf_layout(const idbf_host_factors* f, int* uniform_n0) {
  const int64_t m = 1LL << f->L;
  if (!f->row_leaf_off && !f->col_leaf_off) {
    if (f->n0 < 1 || f->N != ((int64_t)f->n0 << f->L)) return IDBF_EINVAL;
    *uniform_n0 = f->n0;
    return IDBF_OK;
  }
  if (!f->row_leaf_off || !f->col_leaf_off || f->N < 1) return IDBF_EINVAL;
  for (const int64_t* o : {f->row_leaf_off, f->col_leaf_off}) {
    if (o[0] != 0 || o[m] != f->N) return IDBF_EINVAL;
    for (int64_t j = 0; j < m; ++j)
      if (o[j + 1] < o[j] || o[j + 1] - o[j] > (1 << 30)) return IDBF_EINVAL;
  }
  int64_t n0 = f->N / m;
  bool same = n0 >= 1 && n0 * m == f->N;
  for (int64_t j = 0; j < m && same; ++j)
    same = f->row_leaf_off[j + 1] - f->row_leaf_off[j] == n0 && f->col_leaf_off[j + 1] - f->col_leaf_off[j] == n0;
  if (same && f->n0 != 0 && f->n0 != n0) return IDBF_EINVAL;
  *uniform_n0 = same ? (int)n0 : 0;
  return IDBF_OK;
}

static idbf_status validate(const idbf_host_factors* f) {
  if (!f || !f->seg_len || !f->blk_rows || !f->blk_cols || !f->blk_moff || !f->blk_ioff) return IDBF_EINVAL;
  if (f->L < 2 || f->L > 40 || f->n0 < 0) return IDBF_EINVAL;
  int un0 = 0;
  const idbf_status ls = leaf_layout(f, &un0);
  if (ls != IDBF_OK) return ls;
  if (f->mat_len < 0 || f->idx_len < 0 || (f->mat_len > 0 && !f->mat) || (f->idx_len > 0 && !f->idx)) return IDBF_EINVAL;
  const int L = f->L, hV = L / 2;
  const int64_t m = 1LL << L;
  const int min_seg = un0 > 0 ? 1 : 0;  // uneven leaves: empty segments are allowed
  for (int64_t i = 0; i < (int64_t)L * 2 * m; ++i)
    if (f->seg_len[i] < min_seg) return IDBF_EFORMAT;
  std::vector<char> seen;
  for (int l = 0; l <= L; ++l) {
    const int kind = l < hV ? KIND_V : (l == hV ? KIND_S : KIND_U);
    const int64_t H = 1LL << (L - l);
    for (int64_t j = 0; j < m; ++j) {
      int64_t inl[2] = {0, 0}, outl[2] = {0, 0};
      if (l == 0) inl[0] = un0 > 0 ? un0 : f->col_leaf_off[j + 1] - f->col_leaf_off[j];
      else { inl[0] = f->seg_len[(l - 1) * 2 * m + 2 * j]; inl[1] = f->seg_len[(l - 1) * 2 * m + 2 * j + 1]; }
      if (l == L) outl[0] = un0 > 0 ? un0 : f->row_leaf_off[j + 1] - f->row_leaf_off[j];
      else for (int c = 0; c < 2; ++c) outl[c] = f->seg_len[l * 2 * m + (j / H) * 2 * H + j % H + c * H];
      const int64_t nin = inl[0] + inl[1], nout = outl[0] + outl[1];
      for (int c = 0; c < 2; ++c) {
        const int64_t o = (l * m + j) * 2 + c;
        const int64_t r = f->blk_rows[o], cc = f->blk_cols[o], mo = f->blk_moff[o], io = f->blk_ioff[o];
        if (r < 0 || cc < 0 || mo < 0 || io < 0 || mo + r * cc > f->mat_len) return IDBF_EFORMAT;
        if (kind == KIND_V) {
          if (l == L) return IDBF_EFORMAT;
          if (r != outl[c] || r + cc != nin || io + r + cc > f->idx_len) return IDBF_EFORMAT;
          if (!is_perm(f->idx + io, r, f->idx + io + r, cc, nin, seen)) return IDBF_EFORMAT;
        } else if (kind == KIND_S) {
          if (r != outl[c] || cc != nin) return IDBF_EFORMAT;
        } else {
          if (l == 0) return IDBF_EFORMAT;
          if (cc != inl[c] || r + cc != nout || io + r + cc > f->idx_len) return IDBF_EFORMAT;
          if (!is_perm(f->idx + io, cc, f->idx + io + cc, r, nout, seen)) return IDBF_EFORMAT;
        }
      }
    }
  }
  return IDBF_OK;
}

}  // namespace idbf

using namespace idbf;

extern "C" {

void idbf_default_params(idbf_params* p) {
  if (!p) return;
  p->eps = 1e-6;
  p->oversample = 1.0;
  p->oversample_leaf = 0.0;
  p->leaf = 64;
  p->rank_cap = 0;
  p->sampling = IDBF_SAMPLE_MOCK_CHEBYSHEV;
  p->storage = IDBF_STORE_C128;
  p->seed = 0;
  p->qr_arith = IDBF_QR_FP64;
  p->reserved = 0;
}

const char* idbf_strerror(idbf_status s) {
  switch (s) {
    case IDBF_OK: return "ok";
    case IDBF_EINVAL: return "invalid argument";
    case IDBF_ENOMEM: return "out of memory";
    case IDBF_ECUDA: return "CUDA error";
    case IDBF_ERANKCAP: return "an ID reached the rank parameter";
    case IDBF_ETIMEOUT: return "a bounded device wait timed out";
    case IDBF_EFORMAT: return "inconsistent factor data";
    case IDBF_EUNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

const char* idbf_last_cuda_error(void) { return g_last_cuda; }

idbf_status idbf_import_factors(const idbf_host_factors* f, int32_t storage, void* stream, idbf_plan* out) {
  if (!out) return IDBF_EINVAL;
  *out = nullptr;
  if (storage < 0 || storage > 2) return IDBF_EINVAL;
  idbf_status s = validate(f);
  if (s != IDBF_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  idbf_plan_s* h = new (std::nothrow) idbf_plan_s();
  if (!h) return IDBF_ENOMEM;
  Plan& p = h->p;
  cudaGetDevice(&p.device);
  int un0 = 0;
  leaf_layout(f, &un0);
  p.N = f->N; p.n0 = un0; p.L = f->L; p.m = 1 << f->L; p.hV = f->L / 2; p.hU = f->L - p.hV;
  p.uneven = un0 == 0;
  if (p.uneven) {
    p.h_leaf_x.assign(f->col_leaf_off, f->col_leaf_off + p.m + 1);
    p.h_leaf_y.assign(f->row_leaf_off, f->row_leaf_off + p.m + 1);
  }
  p.init_levels();
  const int64_t nb = (int64_t)(p.L + 1) * p.m * 2, nbl = (int64_t)p.m * 2;
  p.h_rows.assign(f->blk_rows, f->blk_rows + nb);
  p.h_cols.assign(f->blk_cols, f->blk_cols + nb);
  p.h_seg_len.assign(f->seg_len, f->seg_len + (int64_t)p.L * 2 * p.m);
  p.h_moff.resize(nb);
  p.h_ioff.resize(nb);
  finalize_structure(&p);
  // per level: compact column-major copy of the blocks (the host blocks are row-major) and the
  // level's index lists (q_c then p_c per block)
  for (int l = 0; l <= p.L && s == IDBF_OK; ++l) {
    int64_t tot = 0, itot = 0;
    for (int64_t o = l * nbl; o < (l + 1) * nbl; ++o) {
      p.h_moff[o] = tot;
      tot += (int64_t)p.h_rows[o] * p.h_cols[o];
      p.h_ioff[o] = itot;
      if (p.lv[l].kind != KIND_S) itot += p.h_rows[o] + p.h_cols[o];
    }
    p.lmat_len[l] = tot;
    p.lidx_len[l] = itot;
    p.mat_len += tot;
    p.idx_len += itot;
    std::vector<double> colmajor;
    std::vector<int32_t> idx;
    try { colmajor.resize(2 * (size_t)tot); idx.resize(itot); } catch (...) { s = IDBF_ENOMEM; break; }
    for (int64_t o = l * nbl; o < (l + 1) * nbl; ++o) {
      const int64_t r = p.h_rows[o], c = p.h_cols[o];
      const double* src = f->mat + 2 * f->blk_moff[o];
      double* dst = colmajor.data() + 2 * p.h_moff[o];
      for (int64_t i = 0; i < r; ++i)
        for (int64_t j = 0; j < c; ++j) {
          dst[2 * (j * r + i)] = src[2 * (i * c + j)];
          dst[2 * (j * r + i) + 1] = src[2 * (i * c + j) + 1];
        }
      if (p.lv[l].kind != KIND_S)
        memcpy(idx.data() + p.h_ioff[o], f->idx + f->blk_ioff[o], (r + c) * sizeof(int32_t));
    }
    cudaError_t e = cudaSuccess;
    if (tot > 0) {
      e = cudaMalloc(&p.lmat[IDBF_STORE_C128][l], tot * 16);
      if (e == cudaSuccess) e = cudaMemcpyAsync(p.lmat[IDBF_STORE_C128][l], colmajor.data(), tot * 16, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && itot > 0) {
      e = cudaMalloc(&p.lidx[l], itot * sizeof(int32_t) + 16);  // 16-byte granule reads may pass the end
      if (e == cudaSuccess) e = cudaMemcpyAsync(p.lidx[l], idx.data(), itot * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host staging buffers go out of scope
    if (e != cudaSuccess) { set_cuda_error(e); s = e == cudaErrorMemoryAllocation ? IDBF_ENOMEM : IDBF_ECUDA; }
  }
  if (s == IDBF_OK) s = upload_structure(&p, st);
  if (s == IDBF_OK && storage != IDBF_STORE_C128) s = convert_storage(&p, 1u << storage, st);
  if (s == IDBF_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_cuda_error(e); s = IDBF_ECUDA; }
  }
  if (s != IDBF_OK) { idbf_destroy(h); return s; }
  *out = h;
  return IDBF_OK;
}

idbf_status idbf_set_storage(idbf_plan h, uint32_t mask, void* stream) {
  if (!h || mask == 0 || (mask & ~7u)) return IDBF_EINVAL;
  return convert_storage(&h->p, mask, (cudaStream_t)stream);
}

idbf_status idbf_clone(idbf_plan h, void* stream, idbf_plan* out) {
  if (!h || !out) return IDBF_EINVAL;
  *out = nullptr;
  const Plan& a = h->p;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != a.device) return IDBF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  idbf_plan_s* c = new (std::nothrow) idbf_plan_s();
  if (!c) return IDBF_ENOMEM;
  Plan& b = c->p;
  b.device = a.device;
  b.N = a.N; b.n0 = a.n0; b.L = a.L; b.m = a.m; b.hV = a.hV; b.hU = a.hU;
  b.init_levels();
  b.h_rows = a.h_rows; b.h_cols = a.h_cols; b.h_moff = a.h_moff; b.h_ioff = a.h_ioff;
  b.h_seg_len = a.h_seg_len;
  b.uneven = a.uneven;
  b.h_leaf_x = a.h_leaf_x;
  b.h_leaf_y = a.h_leaf_y;
  finalize_structure(&b);
  b.mat_len = a.mat_len; b.idx_len = a.idx_len;
  b.lmat_len = a.lmat_len; b.lidx_len = a.lidx_len;
  for (int f = 0; f < 3; ++f) b.tuned[f] = a.tuned[f];
  b.tc_split_mode = a.tc_split_mode;
  b.wait_limit_ns = a.wait_limit_ns;
  b.rank_saturated = a.rank_saturated;
  b.build_seconds = 0.0;
  idbf_status s = upload_structure(&b, st);
  for (int l = 0; l <= a.L && s == IDBF_OK; ++l) {
    for (int f = 0; f < 3 && s == IDBF_OK; ++f) {
      if (!a.lmat[f][l]) continue;
      const size_t bytes = (size_t)a.lmat_len[l] * (f == IDBF_STORE_C64 ? 8 : 16) + (f == IDBF_STORE_C64 ? 16 : 0);
      cudaError_t e = cudaMalloc(&b.lmat[f][l], bytes);
      if (e == cudaSuccess) e = cudaMemcpyAsync(b.lmat[f][l], a.lmat[f][l], bytes, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) { set_cuda_error(e); s = e == cudaErrorMemoryAllocation ? IDBF_ENOMEM : IDBF_ECUDA; }
    }
    if (s == IDBF_OK && a.lidx[l]) {
      const size_t bytes = (size_t)a.lidx_len[l] * sizeof(int32_t) + 16;
      cudaError_t e = cudaMalloc((void**)&b.lidx[l], bytes);
      if (e == cudaSuccess) e = cudaMemcpyAsync(b.lidx[l], a.lidx[l], bytes, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) { set_cuda_error(e); s = e == cudaErrorMemoryAllocation ? IDBF_ENOMEM : IDBF_ECUDA; }
    }
  }
  if (s == IDBF_OK) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_cuda_error(e); s = IDBF_ECUDA; }
  }
  if (s != IDBF_OK) { idbf_destroy(c); return s; }
  *out = c;
  return IDBF_OK;
}

idbf_status idbf_set_level_storage(idbf_plan h, int32_t level, uint32_t mask, void* stream) {
  if (!h || mask == 0 || (mask & ~7u) || level < 0 || level > h->p.L) return IDBF_EINVAL;
  return convert_level(&h->p, level, mask, (cudaStream_t)stream);
}

idbf_status idbf_sync_status(idbf_plan h, void* stream) {
  if (!h) return IDBF_EINVAL;
  Plan& p = h->p;
  if (!p.d_status) return IDBF_OK;
  int v = 0;
  cudaStream_t st = (cudaStream_t)stream;
  IDBF_CUDA_TRY(cudaMemcpyAsync(&v, p.d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  IDBF_CUDA_TRY(cudaStreamSynchronize(st));
  if (v) {
    IDBF_CUDA_TRY(cudaMemsetAsync(p.d_status, 0, sizeof(int), st));
    IDBF_CUDA_TRY(cudaStreamSynchronize(st));
    return IDBF_ETIMEOUT;
  }
  return IDBF_OK;
}

idbf_status idbf_set_tc_split(idbf_plan h, int32_t split_mode) {
  if (!h || split_mode < 0 || split_mode > 2) return IDBF_EINVAL;
  h->p.tc_split_mode = split_mode;
  return IDBF_OK;
}

idbf_status idbf_debug_set_wait(idbf_plan h, uint64_t limit_ns, int32_t producer_enabled) {
  if (!h || limit_ns == 0) return IDBF_EINVAL;
  h->p.wait_limit_ns = limit_ns;
  h->p.producer_enabled = producer_enabled ? 1 : 0;
  return IDBF_OK;
}

idbf_status idbf_reserve(idbf_plan h, int64_t nrhs) {
  if (!h || nrhs < 1) return IDBF_EINVAL;
  return ensure_workspace(&h->p, nrhs);
}

idbf_status idbf_stats(idbf_plan h, idbf_stats_t* s) {
  if (!h || !s) return IDBF_EINVAL;
  const Plan& p = h->p;
  memset(s, 0, sizeof(*s));
  s->N = p.N; s->n0 = p.n0; s->L = p.L; s->h_v = p.hV; s->h_u = p.hU;
  for (int f = 0; f < 3; ++f) if (p.has_format(f)) s->storage_mask |= 1u << f;
  s->rank_saturated = p.rank_saturated;
  s->entries = p.mat_len;
  s->index_entries = p.idx_len;
  for (int l = 0; l <= p.L && l < IDBF_MAX_LEVELS; ++l) {
    s->level_entries[l] = p.lv[l].entries;
    s->level_kmin[l] = p.lv[l].kmin;
    s->level_kmax[l] = p.lv[l].kmax;
  }
  s->segment_entries = p.max_seg_total;
  s->build_seconds = p.build_seconds;
  s->device_bytes = (int64_t)p.device_bytes();
  for (int f = 0; f < 3; ++f)
    for (int l = 0; l < IDBF_MAX_LEVELS; ++l)
      s->level_variant[f][l] = (l < (int)p.tuned[f].size()) ? p.tuned[f][l] : -1;
  for (int l = 0; l <= p.L && l < IDBF_MAX_LEVELS; ++l)
    for (int f = 0; f < 3; ++f)
      if (p.lmat[f][l] || p.lmat_len[l] == 0) s->level_storage[l] |= 1u << f;
  for (int b = 0; b < p.L && b < IDBF_MAX_LEVELS; ++b) s->boundary_entries[b] = p.seg_total[b];
  return IDBF_OK;
}

// ---- checkpoint: "IDBFv001" header, then the butterfly-layout arrays (row-major complex128) --
struct FileHeader {
  char magic[8];
  int64_t N;
  int32_t n0, L;
  int64_t mat_len, idx_len;
};

idbf_status idbf_save(idbf_plan h, const char* path) {
  if (!h || !path) return IDBF_EINVAL;
  const Plan& p = h->p;
  const bool have128 = p.has_format(IDBF_STORE_C128), havedf = p.has_format(IDBF_STORE_DF64);
  if ((p.mat_len > 0 && !have128 && !havedf) || p.uneven) return IDBF_EUNSUPPORTED;
  const int64_t nbl = (int64_t)p.m * 2, nb = (int64_t)(p.L + 1) * nbl;
  // file layout: global (not per-level) offsets, row-major blocks
  std::vector<int64_t> gmoff(nb), gioff(nb);
  std::vector<double> rowmajor(2 * (size_t)p.mat_len);
  std::vector<int32_t> idx(p.idx_len);
  int64_t mbase = 0, ibase = 0;
  for (int l = 0; l <= p.L; ++l) {
    const int64_t n = p.lmat_len[l];
    std::vector<double> dev(2 * (size_t)n);
    if (n > 0) {
      if (have128) {
        IDBF_CUDA_TRY(cudaMemcpy(dev.data(), p.lmat[IDBF_STORE_C128][l], n * 16, cudaMemcpyDeviceToHost));
      } else {
        std::vector<float> t(4 * (size_t)n);
        IDBF_CUDA_TRY(cudaMemcpy(t.data(), p.lmat[IDBF_STORE_DF64][l], n * 16, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i) {
          dev[2 * i] = (double)t[4 * i] + (double)t[4 * i + 1];
          dev[2 * i + 1] = (double)t[4 * i + 2] + (double)t[4 * i + 3];
        }
      }
    }
    if (p.lidx_len[l] > 0)
      IDBF_CUDA_TRY(cudaMemcpy(idx.data() + ibase, p.lidx[l], p.lidx_len[l] * 4, cudaMemcpyDeviceToHost));
    for (int64_t o = l * nbl; o < (l + 1) * nbl; ++o) {
      const int64_t r = p.h_rows[o], c = p.h_cols[o], base = p.h_moff[o];
      gmoff[o] = mbase + base;
      gioff[o] = ibase + p.h_ioff[o];
      for (int64_t i = 0; i < r; ++i)
        for (int64_t j = 0; j < c; ++j) {
          rowmajor[2 * (mbase + base + i * c + j)] = dev[2 * (base + j * r + i)];
          rowmajor[2 * (mbase + base + i * c + j) + 1] = dev[2 * (base + j * r + i) + 1];
        }
    }
    mbase += n;
    ibase += p.lidx_len[l];
  }
  FILE* fp = fopen(path, "wb");
  if (!fp) return IDBF_EINVAL;
  FileHeader hd;
  memcpy(hd.magic, "IDBFv001", 8);
  hd.N = p.N; hd.n0 = p.n0; hd.L = p.L; hd.mat_len = p.mat_len; hd.idx_len = p.idx_len;
  bool ok = fwrite(&hd, sizeof(hd), 1, fp) == 1;
  const int64_t ns = (int64_t)p.L * 2 * p.m;
  ok = ok && fwrite(p.h_seg_len.data(), 4, ns, fp) == (size_t)ns;
  ok = ok && fwrite(p.h_rows.data(), 4, nb, fp) == (size_t)nb;
  ok = ok && fwrite(p.h_cols.data(), 4, nb, fp) == (size_t)nb;
  ok = ok && fwrite(gmoff.data(), 8, nb, fp) == (size_t)nb;
  ok = ok && fwrite(gioff.data(), 8, nb, fp) == (size_t)nb;
  ok = ok && fwrite(rowmajor.data(), 16, p.mat_len, fp) == (size_t)p.mat_len;
  ok = ok && fwrite(idx.data(), 4, p.idx_len, fp) == (size_t)p.idx_len;
  ok = (fclose(fp) == 0) && ok;
  return ok ? IDBF_OK : IDBF_EINVAL;
}

idbf_status idbf_load(const char* path, int32_t storage, void* stream, idbf_plan* out) {
  if (!path || !out) return IDBF_EINVAL;
  *out = nullptr;
  FILE* fp = fopen(path, "rb");
  if (!fp) return IDBF_EINVAL;
  FileHeader hd;
  if (fread(&hd, sizeof(hd), 1, fp) != 1 || memcmp(hd.magic, "IDBFv001", 8) != 0 || hd.L < 2 || hd.L > 40 ||
      hd.n0 < 1 || hd.N != ((int64_t)hd.n0 << hd.L) || hd.mat_len < 0 || hd.idx_len < 0) {
    fclose(fp);
    return IDBF_EFORMAT;
  }
  const int64_t m = 1LL << hd.L, nb = (int64_t)(hd.L + 1) * m * 2, ns = (int64_t)hd.L * 2 * m;
  std::vector<int32_t> seg(ns), rows(nb), cols(nb), idx(hd.idx_len);
  std::vector<int64_t> moff(nb), ioff(nb);
  std::vector<double> mat;
  try { mat.resize(2 * (size_t)hd.mat_len); } catch (...) { fclose(fp); return IDBF_ENOMEM; }
  bool ok = fread(seg.data(), 4, ns, fp) == (size_t)ns && fread(rows.data(), 4, nb, fp) == (size_t)nb &&
            fread(cols.data(), 4, nb, fp) == (size_t)nb && fread(moff.data(), 8, nb, fp) == (size_t)nb &&
            fread(ioff.data(), 8, nb, fp) == (size_t)nb &&
            fread(mat.data(), 16, hd.mat_len, fp) == (size_t)hd.mat_len &&
            fread(idx.data(), 4, hd.idx_len, fp) == (size_t)hd.idx_len;
  fclose(fp);
  if (!ok) return IDBF_EFORMAT;
  idbf_host_factors f;
  f.N = hd.N; f.n0 = hd.n0; f.L = hd.L;
  f.seg_len = seg.data(); f.blk_rows = rows.data(); f.blk_cols = cols.data();
  f.blk_moff = moff.data(); f.blk_ioff = ioff.data();
  f.mat = mat.data(); f.mat_len = hd.mat_len; f.idx = idx.data(); f.idx_len = hd.idx_len;
  f.row_leaf_off = nullptr; f.col_leaf_off = nullptr;
  return idbf_import_factors(&f, storage, stream, out);
}

void idbf_destroy(idbf_plan h) {
  if (!h) return;
  Plan& p = h->p;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != p.device) cudaSetDevice(p.device);
  cudaDeviceSynchronize();
  for (int f = 0; f < 3; ++f)
    for (void* q : p.lmat[f]) if (q) cudaFree(q);
  for (int32_t* q : p.lidx) if (q) cudaFree(q);
  if (p.d_meta) cudaFree(p.d_meta);
  if (p.d_leaf) cudaFree(p.d_leaf);
  if (p.d_ws) cudaFree(p.d_ws);
  if (p.d_status) cudaFree(p.d_status);
  if (cur != p.device) cudaSetDevice(cur);
  delete h;
}

}  // extern "C"
