// Derivatives of an eigenvalue of the pencil with respect to the entries of A and B
// (Hellmann-Feynman): for A x = lambda B x with x^T B x = s,
//   d lambda / d A_ij = x_i x_j / s,   d lambda / d B_ij = -lambda x_i x_j / s,
// every stored entry taken as an independent variable; a lower-triangle entry of a
// KEP_PATTERN_LOWER input stands for both (i, j) and (j, i) and receives the sum of the two.
// For a Hermitian pencil (x complex, x^H B x = s): d lambda / d A_ij = x_i conj(x_j) / s and
// d lambda / d B_ij = -lambda x_i conj(x_j) / s, so that d lambda = sum Re(conj(G_ij) dM_ij).
// Also kep_set_values: new values of A and B on the pattern of kep_analyze.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "kep_ctx.h"
#include "kep_device.cuh"

namespace kep {
namespace {

// partial[blk] = sum over the block's rows of x_i (B x)_i
__global__ void __launch_bounds__(256) xbx_kernel(int64_t n, const double* x, const double* bx, double* partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    s = fma(x[i], bx[i], s);
  s = warp_sum(s);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// per caller entry e: its full-CSR position p (row found by bisection of rp), then the two
// derivatives scaled by c = lambda_bar / s
__global__ void __launch_bounds__(256) grad_kernel(int64_t n, int64_t nnz_in, const int64_t* rp, const int32_t* ci,
                                                   const int64_t* in2csr, const double* x, double c, double lambda,
                                                   double* ga, double* gb) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz_in;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t code = in2csr[e];
    const int64_t p = code & ((1ll << 62) - 1);
    const double mult = (code >> 62) & 1 ? 2.0 : 1.0;
    int64_t lo = 0, hi = n - 1;                 // row i: rp[i] <= p < rp[i + 1]
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) / 2;
      if (rp[mid] <= p) lo = mid; else hi = mid - 1;
    }
    const double g = mult * c * x[lo] * x[ci[p]];
    if (ga) ga[e] = g;
    if (gb) gb[e] = -lambda * g;
  }
}

// Hermitian pencil: per caller entry (i, j), G = c x_i conj(x_j) (complex, interleaved), doubled
// for a stored lower off-diagonal entry (it stands for (i, j) and its conjugate (j, i))
__global__ void __launch_bounds__(256) herm_grad_kernel(int64_t nnz, const int32_t* hr, const int32_t* hc, bool lower,
                                                        const double* x, double c, double lambda, double* ga,
                                                        double* gb) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t i = hr[e], j = hc[e];
    const double xr = x[2 * i], xi = x[2 * i + 1], yr = x[2 * j], yi = x[2 * j + 1];
    const double s = (lower && i != j) ? 2.0 * c : c;
    const double gr = s * fma(xr, yr, xi * yi), gi = s * fma(xi, yr, -xr * yi);
    if (ga) { ga[2 * e] = gr; ga[2 * e + 1] = gi; }
    if (gb) { gb[2 * e] = -lambda * gr; gb[2 * e + 1] = -lambda * gi; }
  }
}

}  // namespace

kep_status herm_grad(kep_ctx* c, double lambda, const double* x, double lambda_bar, double* ga_out, double* gb_out,
                     int ptr_kind) {
  const int64_t N = c->plan.n, nnz = c->herm_nnz;
  cudaStream_t st = c->stream;
  const double* xd = x;                            // interleaved complex x on the device
  if (ptr_kind == KEP_HOST) {
    if (cudaMemcpyAsync(c->d_io3, x, N * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) return KEP_ERR_CUDA;
    xd = c->d_io3;
  } else if (reinterpret_cast<uintptr_t>(x) & 15) {
    return KEP_ERR_INVALID;
  }
  // s = x^H B x = w^T B_r w for w = [Re x; Im x]
  KEP_TRY(herm_to_blocked(c, xd, c->d_io0));
  KEP_TRY(ctx_spmv_dev(c, c->d_io0, nullptr, c->d_io2));
  const int nb = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c->num_sms * 4, (N + 255) / 256)));
  double* part = c->d_solve_partial;
  KEP_LAUNCH(&c->timer, KC_VEC, st, xbx_kernel<<<nb, 256, 0, st>>>(N, c->d_io0, c->d_io2, part));
  std::vector<double> hp(nb);
  if (cudaMemcpyAsync(hp.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return KEP_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return KEP_ERR_CUDA;
  double s = 0.0;
  for (double v : hp) s += v;
  if (!(s > 0.0) || !std::isfinite(s)) return KEP_ERR_INVALID;
  double *ga = ga_out, *gb = gb_out, *stage = nullptr;
  if (ptr_kind == KEP_HOST) {
    if (cudaMalloc(&stage, sizeof(double) * std::max<int64_t>(1, 4 * nnz)) != cudaSuccess) return KEP_ERR_NOMEM;
    ga = ga_out ? stage : nullptr;
    gb = gb_out ? stage + 2 * nnz : nullptr;
  }
  const int ng = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c->num_sms * 8, (nnz + 255) / 256)));
  KEP_LAUNCH(&c->timer, KC_VEC, st,
             herm_grad_kernel<<<ng, 256, 0, st>>>(nnz, c->d_hrow, c->d_hcol, c->herm_lower, xd, lambda_bar / s, lambda,
                                                  ga, gb));
  kep_status out = KEP_OK;
  if (ptr_kind == KEP_HOST) {
    if ((ga_out && cudaMemcpyAsync(ga_out, ga, 2 * nnz * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
        (gb_out && cudaMemcpyAsync(gb_out, gb, 2 * nnz * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess))
      out = KEP_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) out = KEP_ERR_CUDA;
  if (stage) cudaFree(stage);
  c->timer.collect();
  if (out == KEP_OK && cudaGetLastError() != cudaSuccess) out = KEP_ERR_CUDA;
  return out;
}

}  // namespace kep

using namespace kep;

extern "C" kep_status kep_grad(kep_ctx* c, double lambda, const double* x, double lambda_bar, double* d_lambda_d_a,
                               double* d_lambda_d_b, int ptr_kind) {
  if (!c || !x || (!d_lambda_d_a && !d_lambda_d_b)) return KEP_ERR_INVALID;
  if (ptr_kind != KEP_HOST && ptr_kind != KEP_DEVICE) return KEP_ERR_INVALID;
  if (c->herm_n) return herm_grad(c, lambda, x, lambda_bar, d_lambda_d_a, d_lambda_d_b, ptr_kind);
  const int64_t n = c->plan.n, nnz = c->nnz_in;
  cudaStream_t st = c->stream;
  const double* xd = x;
  if (ptr_kind == KEP_HOST) {
    if (cudaMemcpyAsync(c->d_io0, x, n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) return KEP_ERR_CUDA;
    xd = c->d_io0;
  }
  // s = x^T B x
  kep_status rs = ctx_spmv_dev(c, xd, nullptr, c->d_io2);
  if (rs != KEP_OK) return rs;
  const int nb = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c->num_sms * 4, (n + 255) / 256)));
  double* part = c->d_solve_partial;             // num_sms * 4 * (kSolveBlk + 1) doubles, free here
  KEP_LAUNCH(&c->timer, KC_VEC, st, xbx_kernel<<<nb, 256, 0, st>>>(n, xd, c->d_io2, part));
  std::vector<double> hp(nb);
  if (cudaMemcpyAsync(hp.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return KEP_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return KEP_ERR_CUDA;
  double s = 0.0;
  for (double v : hp) s += v;
  if (!(s > 0.0) || !std::isfinite(s)) return KEP_ERR_INVALID;   // x = 0, or B not positive definite on x
  // outputs (device buffers, or staging for host ones)
  double *ga = d_lambda_d_a, *gb = d_lambda_d_b;
  double* stage = nullptr;
  if (ptr_kind == KEP_HOST) {
    if (cudaMalloc(&stage, sizeof(double) * nnz * 2) != cudaSuccess) return KEP_ERR_NOMEM;
    ga = d_lambda_d_a ? stage : nullptr;
    gb = d_lambda_d_b ? stage + nnz : nullptr;
  }
  const int ng = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c->num_sms * 8, (nnz + 255) / 256)));
  KEP_LAUNCH(&c->timer, KC_VEC, st,
             grad_kernel<<<ng, 256, 0, st>>>(n, nnz, c->d_rp, c->d_ci, c->d_in2csr, xd, lambda_bar / s, lambda, ga, gb));
  kep_status out = KEP_OK;
  if (ptr_kind == KEP_HOST) {
    if ((d_lambda_d_a && cudaMemcpyAsync(d_lambda_d_a, ga, nnz * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
        (d_lambda_d_b && cudaMemcpyAsync(d_lambda_d_b, gb, nnz * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess))
      out = KEP_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) out = KEP_ERR_CUDA;
  if (stage) cudaFree(stage);
  c->timer.collect();
  if (out == KEP_OK && cudaGetLastError() != cudaSuccess) out = KEP_ERR_CUDA;
  return out;
}

extern "C" kep_status kep_set_values(kep_ctx* c, const double* a_val, const double* b_val) {
  if (!c || !a_val || !b_val) return KEP_ERR_INVALID;
  return c->herm_n ? herm_set_values(c, a_val, b_val) : set_values_real(c, a_val, b_val);
}

// the caller's values (kep_analyze layout) into the full CSR, the per-front entry lists and the
// norms; the factors of the old values become invalid
kep_status kep::set_values_real(kep_ctx* c, const double* a_val, const double* b_val) {
  Plan& P = c->plan;
  const int64_t n = P.n, nnz = static_cast<int64_t>(c->csr_src.size());
  std::vector<double> av(nnz), bv(nnz);
  for (int64_t p = 0; p < nnz; ++p) {
    av[p] = a_val[c->csr_src[p]];
    bv[p] = b_val[c->csr_src[p]];
  }
  std::vector<int64_t> rp(n + 1);
  if (cudaMemcpy(rp.data(), c->d_rp, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return KEP_ERR_CUDA;
  double norm = 0.0, norm_b = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double r = 0.0, rb = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) { r += std::fabs(av[p]); rb += std::fabs(bv[p]); }
    norm = std::max(norm, r);
    norm_b = std::max(norm_b, rb);
  }
  const int64_t ne = static_cast<int64_t>(P.ent_src.size());
  for (int64_t o = 0; o < ne; ++o) {
    P.ent_a[o] = av[P.ent_src[o]];
    P.ent_b[o] = bv[P.ent_src[o]];
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemcpy(c->d_a, av.data(), nnz * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_b, bv.data(), nnz * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(const_cast<double*>(c->T.ent_a), P.ent_a.data(), ne * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(const_cast<double*>(c->T.ent_b), P.ent_b.data(), ne * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return KEP_ERR_CUDA;
  P.norm_a_inf = norm;
  c->norm_b_inf = norm_b;
  for (int s = 0; s < 2; ++s) c->slot[s].valid = false;   // factors of the old values are void
  return KEP_OK;
}
