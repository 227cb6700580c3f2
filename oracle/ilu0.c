/* ILU(0) for the oracle (test infrastructure only; never linked by the product).
 *
 * Paper Sec. 3.3: the subdomain solver of the restricted additive Schwarz
 * preconditioner is "ILU with no fill-in", ILU(0), on both mesh levels.
 * Plain textbook IKJ ILU(0) on a CSR matrix whose rows have sorted column
 * indices and an explicit diagonal: for row i, for each lower column k in
 * ascending order, l_ik = a_ik / u_kk and a_ij -= l_ik u_kj for every j > k
 * that is in the pattern of both rows; entries outside the pattern are
 * dropped.  L has a unit diagonal; L and U overwrite the matrix.
 */
#include <stdlib.h>

/* returns 0, or 1 + row of the first zero pivot */
int ilu0_factor(int n, const int *indptr, const int *indices, double *a, int *diag) {
  int *iw = (int *)malloc(sizeof(int) * (size_t)n);
  if (!iw) return -1;
  for (int i = 0; i < n; ++i) iw[i] = -1;
  for (int i = 0; i < n; ++i) {
    int b = indptr[i], e = indptr[i + 1];
    diag[i] = -1;
    for (int p = b; p < e; ++p) iw[indices[p]] = p;
    for (int p = b; p < e; ++p) {
      int k = indices[p];
      if (k >= i) {
        if (k == i) diag[i] = p;
        break;
      }
      a[p] /= a[diag[k]];
      double lik = a[p];
      for (int q = diag[k] + 1; q < indptr[k + 1]; ++q) {
        int w = iw[indices[q]];
        if (w >= 0) a[w] -= lik * a[q];
      }
    }
    for (int p = b; p < e; ++p) iw[indices[p]] = -1;
    if (diag[i] < 0 || a[diag[i]] == 0.0) {
      free(iw);
      return 1 + i;
    }
  }
  free(iw);
  return 0;
}

/* x = U^{-1} L^{-1} b  (x may alias b) */
void ilu0_solve(int n, const int *indptr, const int *indices, const double *a, const int *diag,
                const double *b, double *x) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int p = indptr[i]; p < diag[i]; ++p) s -= a[p] * x[indices[p]];
    x[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int p = diag[i] + 1; p < indptr[i + 1]; ++p) s -= a[p] * x[indices[p]];
    x[i] = s / a[diag[i]];
  }
}
