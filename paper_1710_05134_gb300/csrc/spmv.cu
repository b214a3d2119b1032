// Sparse products y = A x and y = B x (the operator applications of the Lanczos decompositions,
// Eqs. 2.2 and 2.5), on the full symmetric CSR in the original numbering.  A and B share the
// pattern (Section 4.1), so one pass over the index arrays produces both products.
#include "kep_device.cuh"

namespace kep {

namespace {

constexpr int kSpmvThreads = 256;

// 8 lanes per row: ~70 nonzeros per row gives ~9 loads per lane.
template <bool WA, bool WB>
__global__ void __launch_bounds__(kSpmvThreads) spmv_ab_kernel(int64_t n, const int64_t* __restrict__ rp,
                                                               const int32_t* __restrict__ ci,
                                                               const double* __restrict__ a,
                                                               const double* __restrict__ b,
                                                               const double* __restrict__ x,
                                                               double* __restrict__ ya,
                                                               double* __restrict__ yb) {
  const int64_t gl = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int sub = threadIdx.x & 7;
  for (int64_t row = gl >> 3; row < n; row += (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 3) {
    double sa = 0.0, sb = 0.0;
    const int64_t e1 = rp[row + 1];
    for (int64_t e = rp[row] + sub; e < e1; e += 8) {
      const double xv = __ldg(x + ci[e]);
      if (WA) sa = fma(a[e], xv, sa);
      if (WB) sb = fma(b[e], xv, sb);
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      if (WA) sa += __shfl_xor_sync(0xffffffffu, sa, o, 8);
      if (WB) sb += __shfl_xor_sync(0xffffffffu, sb, o, 8);
    }
    if (sub == 0) {
      if (WA) ya[row] = sa;
      if (WB) yb[row] = sb;
    }
  }
}

}  // namespace

kep_status run_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* a, const double* b,
                    const double* x, double* ya, double* yb, cudaStream_t st, int num_sms,
                    Timer* timer) {
  const int64_t want = (n * 8 + kSpmvThreads - 1) / kSpmvThreads;
  const int grid = static_cast<int>(want < num_sms * 16 ? want : num_sms * 16);
  if (ya && yb)
    KEP_LAUNCH(timer, KC_SPMV, st, spmv_ab_kernel<true, true><<<grid, kSpmvThreads, 0, st>>>(n, rp, ci, a, b, x, ya, yb));
  else if (ya)
    KEP_LAUNCH(timer, KC_SPMV, st, spmv_ab_kernel<true, false><<<grid, kSpmvThreads, 0, st>>>(n, rp, ci, a, b, x, ya, yb));
  else if (yb)
    KEP_LAUNCH(timer, KC_SPMV, st, spmv_ab_kernel<false, true><<<grid, kSpmvThreads, 0, st>>>(n, rp, ci, a, b, x, ya, yb));
  return cudaGetLastError() == cudaSuccess ? KEP_OK : KEP_ERR_CUDA;
}

}  // namespace kep
