// Tensor-core projection C = V^dag X against a bf16 basis (tc_proj.cu).
#pragma once

#include "internal.cuh"

namespace seedcg {

// columns of the B operand for nvec complex vectors (2 per vector, padded to 16/32/48/64)
int tc_cols(int nvec);
// bytes of the B operand workspace for vectors of n complex entries
size_t tc_b_bytes(long n, int nvec);

// C[a][j] = v_a^dag x_j for a < rows, j < nvec.
//   V: bf16 basis, rows_alloc rows of n complex entries (rows valid: `rows`)
//   X: nvec FP32 vectors (x_j = X + j*ldx), rounded to bf16 for the product
//   Bm: workspace of tc_b_bytes(n, nvec); part: FP32 split partials (part_elems floats)
//   C: double2 [rows][ldc]; err: device int set to SEEDCG_ERR_TIMEOUT if a wait expired
void tc_project(const __nv_bfloat162* V, int rows_alloc, int rows, const float2* X, long ldx,
                int nvec, long n, __nv_bfloat162* Bm, float* part, size_t part_elems,
                double2* C, int ldc, int* err, cudaStream_t st);

}  // namespace seedcg
