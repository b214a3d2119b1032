// Complex Hermitian pencils (A, B) of order n, B positive definite, through their real symmetric
// embedding of order 2n:
//   A_r = [[Re A, -Im A], [Im A, Re A]],  B_r likewise,  A_r [u; v] = lambda B_r [u; v]
// holds exactly when A (u + i v) = lambda B (u + i v).  The map (u + i v) -> [u; v] and its partner
// (u + i v) -> [-v; u] (the eigenvector times i) span a two-dimensional eigenspace for every
// eigenvalue, so the embedding has the spectrum of (A, B) with every eigenvalue twice, and by
// Sylvester's law of inertia (Section 2.1) nu_sigma(A_r, B_r) = 2 nu_sigma(A, B).  Inertia counts,
// solves, products and the three stages of Algorithm 4 run unchanged on the real pencil; the counts
// reported for a Hermitian context are halved, and complex vectors (interleaved re, im) are mapped
// to and from the embedding's [re; im] layout on the device.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "kep_ctx.h"
#include "kep_device.cuh"

namespace kep {
namespace {

__global__ void to_blocked_kernel(int64_t n, const double* __restrict__ in, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double2 z = reinterpret_cast<const double2*>(in)[i];
    out[i] = z.x;
    out[n + i] = z.y;
  }
}

__global__ void to_interleaved_kernel(int64_t n, const double* __restrict__ in, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    reinterpret_cast<double2*>(out)[i] = make_double2(in[i], in[n + i]);
}

int vec_grid(const kep_ctx* c, int64_t n) {
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c->num_sms * 4, (n + 255) / 256)));
}

}  // namespace

kep_status herm_to_blocked(kep_ctx* c, const double* in, double* out) {
  const int64_t n = c->herm_n;
  KEP_LAUNCH(&c->timer, KC_VEC, c->stream, to_blocked_kernel<<<vec_grid(c, n), 256, 0, c->stream>>>(n, in, out));
  return cudaGetLastError() == cudaSuccess ? KEP_OK : KEP_ERR_CUDA;
}

kep_status herm_to_interleaved(kep_ctx* c, const double* in, double* out) {
  const int64_t n = c->herm_n;
  KEP_LAUNCH(&c->timer, KC_VEC, c->stream, to_interleaved_kernel<<<vec_grid(c, n), 256, 0, c->stream>>>(n, in, out));
  return cudaGetLastError() == cudaSuccess ? KEP_OK : KEP_ERR_CUDA;
}

namespace {
// a complex vector (2 herm_n doubles) from ptr_kind memory into the embedding layout at dst
// (stage: device scratch for host input)
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

kep_status load_complex(kep_ctx* c, const double* src, int ptr_kind, double* stage, double* dst) {
  const int64_t N = c->plan.n;
  if (ptr_kind == KEP_DEVICE && !aligned16(src)) return KEP_ERR_INVALID;   // read as (re, im) pairs
  if (ptr_kind == KEP_HOST) {
    if (cudaMemcpyAsync(stage, src, N * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return KEP_ERR_CUDA;
    src = stage;
  }
  return herm_to_blocked(c, src, dst);
}

// the embedding-layout vector src out to a complex vector in ptr_kind memory (stage: device scratch)
kep_status store_complex(kep_ctx* c, const double* src, int ptr_kind, double* stage, double* dst) {
  const int64_t N = c->plan.n;
  if (ptr_kind == KEP_DEVICE) return aligned16(dst) ? herm_to_interleaved(c, src, dst) : KEP_ERR_INVALID;
  KEP_TRY(herm_to_interleaved(c, src, stage));
  if (cudaMemcpyAsync(dst, stage, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return KEP_ERR_CUDA;
  return KEP_OK;
}

kep_status finish(kep_ctx* c) {
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return KEP_ERR_CUDA;
  c->timer.collect();
  return KEP_OK;
}
}  // namespace

kep_status herm_solve(kep_ctx* c, const double* rhs, double* x, int64_t nrhs, int ptr_kind) {
  if (ptr_kind != KEP_HOST && ptr_kind != KEP_DEVICE) return KEP_ERR_INVALID;
  const int64_t N = c->plan.n;   // doubles per complex vector
  for (int64_t r = 0; r < nrhs; ++r) {
    KEP_TRY(load_complex(c, rhs + r * N, ptr_kind, c->d_io2, c->d_io0));
    KEP_TRY(ctx_solve_dev(c, 0, c->d_io0, c->d_io1));
    KEP_TRY(store_complex(c, c->d_io1, ptr_kind, c->d_io2, x + r * N));
  }
  return finish(c);
}

kep_status herm_spmv(kep_ctx* c, const double* x, double* ax, double* bx, int ptr_kind) {
  if (ptr_kind != KEP_HOST && ptr_kind != KEP_DEVICE) return KEP_ERR_INVALID;
  KEP_TRY(load_complex(c, x, ptr_kind, c->d_io3, c->d_io0));
  KEP_TRY(ctx_spmv_dev(c, c->d_io0, ax ? c->d_io1 : nullptr, bx ? c->d_io2 : nullptr));
  if (ax) KEP_TRY(store_complex(c, c->d_io1, ptr_kind, c->d_io3, ax));
  if (bx) KEP_TRY(store_complex(c, c->d_io2, ptr_kind, c->d_io4, bx));
  return finish(c);
}

kep_status herm_solve_refined(kep_ctx* c, const double* rhs, double* x, int ptr_kind, double tol, int32_t max_iter,
                              int32_t* iters, double* berr) {
  if (ptr_kind != KEP_HOST && ptr_kind != KEP_DEVICE) return KEP_ERR_INVALID;
  // b in d_io0, x in d_io1 (the refinement's scratch is d_io2, d_io3 and its Krylov workspace)
  KEP_TRY(load_complex(c, rhs, ptr_kind, c->d_io4, c->d_io0));
  const kep_status rs = ctx_solve_refined_dev(c, c->d_io0, c->d_io1, tol, max_iter, iters, berr);
  if (rs != KEP_OK && rs != KEP_ERR_NOT_CONVERGED) return rs;
  KEP_TRY(store_complex(c, c->d_io1, ptr_kind, c->d_io4, x));
  KEP_TRY(finish(c));
  return rs;
}

}  // namespace kep

using namespace kep;

extern "C" kep_status kep_analyze_hermitian(int64_t n, const int64_t* rowptr, const int32_t* colind,
                                            const double* a_val, const double* b_val, int flags,
                                            const double* coords, kep_ctx** out) {
  if (!out) return KEP_ERR_INVALID;
  *out = nullptr;
  if (n < 1 || n > (INT32_MAX - 1) / 2 || !rowptr || !colind || !a_val || !b_val) return KEP_ERR_INVALID;
  if (rowptr[0] != 0) return KEP_ERR_INVALID;
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return KEP_ERR_INVALID;
  const bool lower = flags & KEP_PATTERN_LOWER;
  const int64_t nnz_in = rowptr[n];
  // every entry of the full Hermitian matrix: (row, col, a, b); a stored lower off-diagonal entry
  // also gives (col, row) with the conjugate values
  struct Ent { int32_t r, c; double ar, ai, br, bi; int64_t e; bool mir; };
  std::vector<Ent> full;
  full.reserve(static_cast<size_t>(lower ? 2 * nnz_in : nnz_in));
  std::vector<int32_t> hrow(nnz_in), hcol(nnz_in);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int64_t j = colind[e];
      if (j < 0 || j >= n || (lower && j > i)) return KEP_ERR_INVALID;
      const double ar = a_val[2 * e], ai = a_val[2 * e + 1], br = b_val[2 * e], bi = b_val[2 * e + 1];
      if (j == i && (ai != 0.0 || bi != 0.0)) return KEP_ERR_INVALID;   // a Hermitian diagonal is real
      hrow[e] = static_cast<int32_t>(i);
      hcol[e] = static_cast<int32_t>(j);
      full.push_back({static_cast<int32_t>(i), static_cast<int32_t>(j), ar, ai, br, bi, e, false});
      if (lower && j != i)
        full.push_back({static_cast<int32_t>(j), static_cast<int32_t>(i), ar, -ai, br, -bi, e, true});
    }
  // the embedding, row by row (kep_analyze sorts each row and rejects duplicates)
  const int64_t N = 2 * n;
  std::vector<int64_t> cnt(N + 1, 0);
  for (const Ent& t : full) {
    cnt[t.r + 1] += t.r == t.c ? 1 : 2;
    cnt[n + t.r + 1] += t.r == t.c ? 1 : 2;
  }
  for (int64_t i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
  const int64_t nnz = cnt[N];
  std::vector<int32_t> ci(nnz);
  std::vector<double> av(nnz), bv(nnz);
  std::vector<int64_t> emb_src(nnz);
  std::vector<int8_t> emb_part(nnz);
  {
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    // part: which value of the caller's entry lands here (0 Re, +1 Im, -1 -Im)
    auto put = [&](int64_t row, int64_t col, double a, double b, int64_t e, int8_t part) {
      const int64_t o = fill[row]++;
      ci[o] = static_cast<int32_t>(col); av[o] = a; bv[o] = b;
      emb_src[o] = e; emb_part[o] = part;
    };
    for (const Ent& t : full) {
      put(t.r, t.c, t.ar, t.br, t.e, 0);                              // Re block, top left
      put(n + t.r, n + t.c, t.ar, t.br, t.e, 0);                      // Re block, bottom right
      if (t.r != t.c) {
        // (a mirrored entry holds the conjugate: its imaginary part is -Im of the caller's)
        put(t.r, n + t.c, -t.ai, -t.bi, t.e, t.mir ? 1 : -1);         // -Im block, top right
        put(n + t.r, t.c, t.ai, t.bi, t.e, t.mir ? -1 : 1);           // Im block, bottom left
      }
    }
  }
  std::vector<double> co;
  if (coords) {
    co.resize(3 * static_cast<size_t>(N));
    std::copy(coords, coords + 3 * n, co.begin());
    std::copy(coords, coords + 3 * n, co.begin() + 3 * n);
  }
  kep_ctx* c = nullptr;
  const kep_status st = kep_analyze(N, cnt.data(), ci.data(), av.data(), bv.data(),
                                    KEP_PATTERN_FULL | (flags & (KEP_ORDER_GRAPH | KEP_ORDER_REFINED)) | kOrderPairs,
                                    coords ? co.data() : nullptr, &c);
  if (st != KEP_OK) return st;
  c->herm_n = n;
  c->herm_nnz = nnz_in;
  c->herm_lower = lower;
  c->herm_emb_src = std::move(emb_src);
  c->herm_emb_part = std::move(emb_part);
  for (int q = 0; q < 2; ++q) {
    int32_t* d = nullptr;
    const std::vector<int32_t>& h = q == 0 ? hrow : hcol;
    if (cudaMalloc(&d, sizeof(int32_t) * std::max<int64_t>(1, nnz_in)) != cudaSuccess) {
      cudaGetLastError();
      kep_destroy(c);
      return KEP_ERR_NOMEM;
    }
    c->allocs.push_back(d);
    if (nnz_in && cudaMemcpy(d, h.data(), sizeof(int32_t) * nnz_in, cudaMemcpyHostToDevice) != cudaSuccess) {
      kep_destroy(c);
      return KEP_ERR_CUDA;
    }
    (q == 0 ? c->d_hrow : c->d_hcol) = d;
  }
  *out = c;
  return KEP_OK;
}

// New complex values on a Hermitian context: the embedding's values from the map kept at analysis
kep_status kep::herm_set_values(kep_ctx* c, const double* a_val, const double* b_val) {
  std::vector<int32_t> hr(c->herm_nnz), hc(c->herm_nnz);
  if (c->herm_nnz &&
      (cudaMemcpy(hr.data(), c->d_hrow, sizeof(int32_t) * c->herm_nnz, cudaMemcpyDeviceToHost) != cudaSuccess ||
       cudaMemcpy(hc.data(), c->d_hcol, sizeof(int32_t) * c->herm_nnz, cudaMemcpyDeviceToHost) != cudaSuccess))
    return KEP_ERR_CUDA;
  for (int64_t e = 0; e < c->herm_nnz; ++e)
    if (hr[e] == hc[e] && (a_val[2 * e + 1] != 0.0 || b_val[2 * e + 1] != 0.0)) return KEP_ERR_INVALID;
  const size_t m = c->herm_emb_src.size();
  std::vector<double> av(m), bv(m);
  for (size_t o = 0; o < m; ++o) {
    const int64_t e = c->herm_emb_src[o];
    const int8_t part = c->herm_emb_part[o];
    av[o] = part == 0 ? a_val[2 * e] : part * a_val[2 * e + 1];
    bv[o] = part == 0 ? b_val[2 * e] : part * b_val[2 * e + 1];
  }
  return set_values_real(c, av.data(), bv.data());
}
