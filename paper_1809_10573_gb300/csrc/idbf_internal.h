// Internal structures of the IDBF library (not part of the C interface).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "idbf.h"

namespace idbf {

// Level kinds of the butterfly layout (apply order).
enum LevelKind { KIND_V = 0, KIND_S = 1, KIND_U = 2 };

// Everything a level kernel needs, passed by value.
struct DevLevel {
  int kind;
  int lev;
  int L;
  int H;   // 2^(L - lev): output c of node j is segment (j / H) 2H + j % H + c H
  int m;
  int n0;
  const int32_t* rows;    // [m][2]
  const int32_t* cols;    // [m][2]
  const int64_t* moff;    // [m][2] entry offset of M_c (column-major: M(r, j) at j*rows + r)
  const int64_t* ioff;    // [m][2] offset of the index lists in idx
  const int32_t* idx;
  const int64_t* in_off;  // boundary lev-1 segment offsets (nullptr at lev 0)
  const int32_t* in_len;
  const int64_t* out_off; // boundary lev segment offsets (nullptr at lev L)
  const int32_t* out_len;
  const int64_t* leaf;    // uneven leaves only: [m+1] offsets of the leaves of x (lev 0) or y
                          // (lev L); nullptr for leaves of n0 points and on the inner levels
};

#ifdef __CUDACC__
// first row and size of leaf j of the user vector read (forward level 0, adjoint level L) or
// written (forward level L, adjoint level 0) by level d
__device__ __forceinline__ int64_t leaf_start(const DevLevel& d, int64_t j) { return d.leaf ? d.leaf[j] : j * d.n0; }
__device__ __forceinline__ int leaf_len(const DevLevel& d, int64_t j) {
  return d.leaf ? (int)(d.leaf[j + 1] - d.leaf[j]) : d.n0;
}
#endif

struct LevelInfo {
  int kind = 0;
  int64_t entries = 0;
  int64_t idx_entries = 0;
  int max_rows = 0;      // max rows of one block
  int max_cols = 0;      // max cols of one block
  int max_in = 0;        // max summed input length of a node
  int max_out = 0;       // max summed output length of a node
  int max_rows_pair = 0; // max rows_0 + rows_1 of a node
  int max_cols_pair = 0; // max cols_0 + cols_1 of a node
  int kmin = 0, kmax = 0;  // output segment lengths
};

struct Plan {
  int device = 0;
  int64_t N = 0;
  int n0 = 0, L = 0, m = 0, hV = 0, hU = 0;
  std::vector<LevelInfo> lv;           // L + 1
  // host copy of the structure
  std::vector<int32_t> h_rows, h_cols;  // [(L+1) m 2]
  std::vector<int64_t> h_moff, h_ioff;
  std::vector<int32_t> h_seg_len;       // [L][2m]
  std::vector<int64_t> h_seg_off;       // [L][2m]
  std::vector<int64_t> seg_total;       // [L]
  int64_t max_seg_total = 0;
  // leaves of uneven size (coordinate-based trees, Example 3): offsets of the column leaves (x,
  // read by level 0) and of the row leaves (y, written by level L); n0 = 0 then
  bool uneven = false;
  std::vector<int64_t> h_leaf_x, h_leaf_y;  // [m+1] each (uneven only)
  int64_t* d_leaf = nullptr;                // device copy: x offsets, then y offsets
  int64_t mat_len = 0;                  // entries over all levels
  int64_t idx_len = 0;                  // indices over all levels
  // device: one matrix arena per level and format (offsets moff are relative to the level),
  // one index array per level (ioff relative to the level)
  void* d_meta = nullptr;
  int32_t* d_rows = nullptr;
  int32_t* d_cols = nullptr;
  int64_t* d_moff = nullptr;
  int64_t* d_ioff = nullptr;
  int32_t* d_seg_len = nullptr;
  int64_t* d_seg_off = nullptr;
  std::vector<int64_t> lmat_len;        // [L+1] entries
  std::vector<int64_t> lidx_len;        // [L+1]
  std::vector<void*> lmat[3];           // [format][L+1]
  std::vector<int32_t*> lidx;           // [L+1]
  void* d_ws = nullptr;
  int* d_status = nullptr;              // device status word: bit 0 = a bounded wait timed out
  uint64_t wait_limit_ns = 2000000000ull;  // limit of every device-side wait (2 s)
  int producer_enabled = 1;             // 0 only in the timeout test (waits that nothing satisfies)
  std::vector<int> tuned[3];            // per storage format: forward kernel variant per level (-1: default)
  int tc_split_mode = 0;                // tensor-core split: 0 three products, 1 lo rounded, 2 four products
  size_t ws_bytes = 0;
  int rank_saturated = 0;
  double build_seconds = 0.0;

  DevLevel level(int l) const;
  size_t device_bytes() const;
  bool has_format(int f) const;         // every non-empty level holds format f
  void init_levels();                   // size the per-level vectors (L set)
};

// error bookkeeping (thread-local last CUDA error name)
void set_cuda_error(cudaError_t e);
#define IDBF_CUDA_TRY(call)                       \
  do {                                            \
    cudaError_t _e = (call);                      \
    if (_e != cudaSuccess) {                      \
      ::idbf::set_cuda_error(_e);                 \
      return _e == cudaErrorMemoryAllocation ? IDBF_ENOMEM : IDBF_ECUDA; \
    }                                             \
  } while (0)

// Level infos and segment offsets from the host structure (h_rows, h_cols, h_seg_len).
idbf_status finalize_structure(Plan* p);
// Copy the host structure (block shapes and offsets, segment lengths and offsets) to the device.
idbf_status upload_structure(Plan* p, cudaStream_t st);

// storage conversion kernels (plan.cu)
idbf_status convert_storage(Plan* p, uint32_t mask, cudaStream_t st);

// workspace (apply.cu)
idbf_status ensure_workspace(Plan* p, int64_t nrhs);

// 3xTF32 tensor-core forward apply of all levels (apply_tc.cu); workspace must be reserved.
// wide_middle: the middle factor in FP64 / double-float on the CUDA cores (apply_middle_wide).
idbf_status apply_tf32x3(Plan* p, const void* x, void* y, int64_t R, int64_t ld, cudaStream_t st, bool wide_middle);
// The middle factor of IDBF_MODE_TF32X3_S64 between complex64 workspace boundaries (apply.cu).
idbf_status apply_middle_wide(Plan* p, const void* win, void* wout, int64_t R, cudaStream_t st);

inline int64_t boundary_index(int b, int64_t m) { return (int64_t)b * 2 * m; }

}  // namespace idbf

struct idbf_plan_s {
  idbf::Plan p;
};
