// Descriptor of one matrix of a batched product (shared by api.cu, which
// fills it on the host, and batched.cu, whose persistent kernel reads it).
#pragma once
#include <cuda_runtime.h>

namespace gbs {

template <typename T>
struct BatchDesc {
  int m, n, nnz, k;
  const int* row_ptr;
  const int* col_idx;
  const T* vals;
  const T* X;
  T* Y;
  long long ldx, ldy;
  int variant;     // GBS_VARIANT_ROWS or GBS_VARIANT_MERGE
  int lanes;       // ROWS: lanes per row (k == 1) or column lanes (k > 1)
  int tile;        // ROWS: nonzeros staged per pass
  int items;       // MERGE: items per merge thread
  int item_begin;  // first work item of this matrix in the batch's work list
  int nitems;      // its work items: row blocks (ROWS) or merge tiles (MERGE)
  int2* coords;    // MERGE scratch (plan-owned)
  int* carry_row;
  T* carry_val;
  int* done;       // MERGE: tiles finished in the current launch (0 between launches)
  int aligned_vals, aligned_cols;
};

}  // namespace gbs
