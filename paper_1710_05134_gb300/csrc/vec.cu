// Vector kernels of the Lanczos processes (Eqs. 2.2 and 2.5): many dot products against the
// columns of a basis, basis-times-coefficients updates, and residual norms.  Reductions are done
// in two fixed passes (per-block partials, then one block over the partials) so every result is
// independent of scheduling.
#include "kep_device.cuh"
#include "kep_vec.h"

namespace kep {
namespace {

constexpr int kVecThreads = 256;

// partial[b * ncol + c] = sum over block b's rows of V(i, c) * w(i)
__global__ void __launch_bounds__(kVecThreads) dots_partial_kernel(int64_t n, const double* __restrict__ V,
                                                                   int64_t ld, int32_t ncol,
                                                                   const double* __restrict__ w,
                                                                   double* __restrict__ partial) {
  __shared__ double red[kVecThreads / 32];
  const int64_t rows_per_block = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * rows_per_block;
  const int64_t r1 = min(n, r0 + rows_per_block);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int32_t c = 0; c < ncol; ++c) {
    const double* col = V + c * ld;
    double s = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) s = fma(col[i], w[i], s);
    s = warp_sum(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < kVecThreads / 32; ++q) t += red[q];
      partial[static_cast<int64_t>(blockIdx.x) * ncol + c] = t;
    }
    __syncthreads();
  }
}

__global__ void dots_final_kernel(int32_t nblocks, int32_t ncol, const double* __restrict__ partial,
                                  double* __restrict__ out) {
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int32_t b = 0; b < nblocks; ++b) s += partial[static_cast<int64_t>(b) * ncol + c];
    out[c] = s;
  }
}

// y(i) = beta * y(i) + alpha * sum_c V(i, c) * coef(c)
__global__ void combine_kernel(int64_t n, const double* __restrict__ V, int64_t ld, int32_t ncol,
                               const double* __restrict__ coef, double alpha, double beta,
                               double* __restrict__ y) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double s = 0.0;
    for (int32_t c = 0; c < ncol; ++c) s = fma(V[c * ld + i], coef[c], s);
    y[i] = (beta == 0.0 ? 0.0 : beta * y[i]) + alpha * s;
  }
}

// y = a * x + b * y
__global__ void axpby_kernel(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

// partial sums of |u - lam * v|^2 and |x|^2
__global__ void __launch_bounds__(kVecThreads) resid_partial_kernel(int64_t n, const double* __restrict__ u,
                                                                    const double* __restrict__ v, double lam,
                                                                    const double* __restrict__ x,
                                                                    double* __restrict__ partial) {
  __shared__ double red[2][kVecThreads / 32];
  double s = 0.0, t = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double r = u[i] - lam * v[i];
    s = fma(r, r, s);
    t = fma(x[i], x[i], t);
  }
  s = warp_sum(s); t = warp_sum(t);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) { red[0][warp] = s; red[1][warp] = t; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < kVecThreads / 32; ++q) { a += red[0][q]; b += red[1][q]; }
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = b;
  }
}

}  // namespace

void VecOps::dots(const double* V, int64_t ld, int32_t ncol, const double* w, double* out_dev) {
  const int nb = num_blocks;
  KEP_LAUNCH(timer, KC_VEC, stream,
             dots_partial_kernel<<<nb, kVecThreads, 0, stream>>>(n, V, ld, ncol, w, partial));
  KEP_LAUNCH(timer, KC_VEC, stream,
             dots_final_kernel<<<(ncol + 127) / 128, 128, 0, stream>>>(nb, ncol, partial, out_dev));
}

void VecOps::combine(const double* V, int64_t ld, int32_t ncol, const double* coef_dev, double alpha,
                     double beta, double* y) {
  KEP_LAUNCH(timer, KC_VEC, stream,
             combine_kernel<<<num_blocks, kVecThreads, 0, stream>>>(n, V, ld, ncol, coef_dev, alpha, beta, y));
}

void VecOps::axpby(double a, const double* x, double b, double* y) {
  KEP_LAUNCH(timer, KC_VEC, stream, axpby_kernel<<<num_blocks, kVecThreads, 0, stream>>>(n, a, x, b, y));
}

void VecOps::resid_partials(const double* u, const double* v, double lam, const double* x) {
  KEP_LAUNCH(timer, KC_VEC, stream,
             resid_partial_kernel<<<num_blocks, kVecThreads, 0, stream>>>(n, u, v, lam, x, partial));
}

}  // namespace kep
