// Vector operations used by the eigenpair driver (library-internal).
#pragma once

#include <cstdint>

#include "kep_internal.h"

namespace kep {

struct VecOps {
  int64_t n = 0;
  int num_blocks = 1;          // blocks of the row-parallel kernels
  double* partial = nullptr;   // num_blocks * max columns (device)
  cudaStream_t stream = nullptr;
  Timer* timer = nullptr;
  // out_dev[c] = V(:, c) . w for c < ncol (column-major V, leading dimension ld)
  void dots(const double* V, int64_t ld, int32_t ncol, const double* w, double* out_dev);
  // y = beta * y + alpha * V(:, 0:ncol) coef
  void combine(const double* V, int64_t ld, int32_t ncol, const double* coef_dev, double alpha, double beta,
               double* y);
  // y = a x + b y
  void axpby(double a, const double* x, double b, double* y);
  // partial[2b] = sum |u - lam v|^2, partial[2b+1] = sum |x|^2 over block b
  void resid_partials(const double* u, const double* v, double lam, const double* x);
};

// Eigenvalues (ascending, in d) and orthonormal eigenvectors (columns of z, ld = m) of the symmetric
// tridiagonal matrix with diagonal d[0..m) and off-diagonal e[0..m-1).  Returns false if the
// iteration does not converge.
bool tridiag_eigen(int m, const double* d, const double* e, double* w, double* z);

}  // namespace kep
