/* FP64 CSR Gram application for the oracle.
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle; never linked into the
 * library.  It restates one application of the sparse operator of the paper's
 * Sec. IV (Alg. 4 on one device): y = A v, w = A^T y, ||y||^2, all in
 * double precision, with plain loops in row order.
 *
 * row_ptr: m+1 int64 offsets; col_idx: nnz int32; values: nnz float.
 * rows [r0, r1) are applied (r0 = 0, r1 = m for the whole matrix); w (length n)
 * is accumulated into, not cleared.  Returns ||y||^2 over those rows.
 */
#include <stdint.h>

double oracle_csr_gram_apply(int64_t r0, int64_t r1, const int64_t *row_ptr,
                             const int32_t *col_idx, const float *values,
                             const double *v, double *w) {
  double ss = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    double y = 0.0;
    for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p)
      y += (double)values[p] * v[col_idx[p]];
    ss += y * y;
    for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p)
      w[col_idx[p]] += (double)values[p] * y;
  }
  return ss;
}
