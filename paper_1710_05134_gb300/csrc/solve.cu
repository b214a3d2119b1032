// Triangular solves with the multifrontal factor: x = Q^T P^T L^{-T} D^{-1} L^{-1} P Q b
// (task (vi) of Section 4.3; the (A - sigma B) y = B v solves of Eq. 2.5 and the B solves of
// Eq. 2.2).
//
// Forward pass, leaves to root: each front gathers its fully-summed right-hand sides, adds its
// children's contribution vectors through the same index maps as the factorization's
// extend-add, applies its pivot permutation and eliminates with its L columns; what is left on
// its contribution rows is passed to the parent.  Backward pass, root to leaves: each front
// reads the solution on its contribution rows (written by its ancestors), applies D^{-1} and
// L^{-T}, and writes its own variables.  No atomics: the result does not depend on scheduling.
#include "kep_device.cuh"

namespace kep {

namespace {

constexpr int kSolveThreads = 256;
constexpr int kBlk = 32;

// block [k0, k0 + kb) of pivots that does not split a 2x2 pair
KEP_D int32_t fwd_block(const int8_t* piv, int32_t k0, int32_t nel) {
  int32_t kb = min(kBlk, nel - k0);
  if (piv[k0 + kb - 1] == 2) kb += 1;
  return kb;
}

__global__ void __launch_bounds__(kSolveThreads) sv_fwd_kernel(FrontTables T, FactorSlot S,
                                                               const int32_t* lf, const double* bnew,
                                                               double* vasm, double* vfac) {
  const int32_t t = lf[blockIdx.x];
  const int32_t d_in = S.d_in[t];
  const int32_t m = T.m_sym[t] + d_in;
  const int32_t nel = S.nelim[t];
  const int32_t psym = T.p_sym[t];
  double* va = vasm + T.vec_off[t];
  double* vf = vfac + T.vec_off[t];
  const int32_t* ap = S.apos + T.vec_off[t];
  const int32_t first = T.first[t];
  for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
    va[i] = (i >= d_in && i < d_in + psym) ? bnew[first + i - d_in] : 0.0;
  __syncthreads();
  int32_t off = 0;
  for (int32_t c = T.child_ptr[t]; c < T.child_ptr[t + 1]; ++c) {
    const int32_t ch = T.child_idx[c];
    const int32_t dout = S.d_out[ch], nelc = S.nelim[ch];
    const int32_t nc = dout + (T.m_sym[ch] - T.p_sym[ch]);
    const double* vc = vfac + T.vec_off[ch] + nelc;
    for (int32_t q = threadIdx.x; q < nc; q += blockDim.x)
      va[parent_pos(T, ch, q, dout, off, d_in)] += vc[q];
    off += dout;
    __syncthreads();
  }
  for (int32_t i = threadIdx.x; i < m; i += blockDim.x) vf[i] = va[ap[i]];
  __syncthreads();
  const double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  const int8_t* piv = S.piv + T.piv_off[t];
  const int32_t warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  int32_t k0 = 0;
  while (k0 < nel) {
    const int32_t kb = fwd_block(piv, k0, nel);
    const int32_t k1 = k0 + kb;
    if (warp == 0) {
      for (int32_t c = k0; c < k1;) {
        if (piv[c] == 2) {
          const double y0 = vf[c], y1 = vf[c + 1];
          for (int32_t a = c + 2 + lane; a < k1; a += 32)
            vf[a] -= L[static_cast<int64_t>(c) * ld + a] * y0 + L[static_cast<int64_t>(c + 1) * ld + a] * y1;
          c += 2;
        } else {
          const double y0 = vf[c];
          for (int32_t a = c + 1 + lane; a < k1; a += 32) vf[a] -= L[static_cast<int64_t>(c) * ld + a] * y0;
          c += 1;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int32_t a = k1 + threadIdx.x; a < m; a += blockDim.x) {
      double s = 0.0;
      for (int32_t c = k0; c < k1; ++c) s += L[static_cast<int64_t>(c) * ld + a] * vf[c];
      vf[a] -= s;
    }
    __syncthreads();
    k0 = k1;
  }
}

__global__ void __launch_bounds__(kSolveThreads) sv_bwd_kernel(FrontTables T, FactorSlot S,
                                                               const int32_t* lf, double* xnew,
                                                               double* vfac) {
  __shared__ double red[kSolveThreads / 32][kBlk + 1];
  __shared__ double part[kBlk + 1];
  const int32_t t = lf[blockIdx.x];
  const int32_t d_in = S.d_in[t];
  const int32_t m = T.m_sym[t] + d_in;
  const int32_t nel = S.nelim[t];
  double* vf = vfac + T.vec_off[t];
  const int32_t* rv = S.rowvar + T.vec_off[t];
  const double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  const int8_t* piv = S.piv + T.piv_off[t];
  const double* Dd = S.Dd + T.piv_off[t];
  const double* De = S.De + T.piv_off[t];
  for (int32_t i = nel + threadIdx.x; i < m; i += blockDim.x) vf[i] = xnew[rv[i]];
  for (int32_t c = threadIdx.x; c < nel; c += blockDim.x) {
    if (piv[c] == 1) {
      vf[c] = vf[c] / Dd[c];
    } else if (piv[c] == 2) {
      const double a = Dd[c], cc = Dd[c + 1], b = De[c];
      const double det = a * cc - b * b;
      const double y0 = vf[c], y1 = vf[c + 1];
      vf[c] = (cc * y0 - b * y1) / det;
      vf[c + 1] = (a * y1 - b * y0) / det;
    }
  }
  __syncthreads();
  const int32_t warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  int32_t k1 = nel;
  while (k1 > 0) {
    int32_t k0 = max(0, k1 - kBlk);
    if (piv[k0] == 0) k0 -= 1;               // keep a 2x2 pair together
    const int32_t kb = k1 - k0;
    double acc[kBlk + 1];
#pragma unroll
    for (int32_t c = 0; c <= kBlk; ++c) acc[c] = 0.0;
    for (int32_t a = k1 + threadIdx.x; a < m; a += blockDim.x) {
      const double xa = vf[a];
#pragma unroll
      for (int32_t c = 0; c <= kBlk; ++c)
        if (c < kb) acc[c] += L[static_cast<int64_t>(k0 + c) * ld + a] * xa;
    }
#pragma unroll
    for (int32_t c = 0; c <= kBlk; ++c) {
      const double v = warp_sum(acc[c]);
      if (lane == 0) red[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < kb) {
      double s = 0.0;
      for (int32_t w = 0; w < kSolveThreads / 32; ++w) s += red[w][threadIdx.x];
      part[threadIdx.x] = s;
    }
    __syncthreads();
    if (warp == 0) {
      for (int32_t c = k1 - 1; c >= k0;) {
        if (piv[c] == 0) {                    // second of a pair at (c-1, c)
          double s0 = 0.0, s1 = 0.0;
          for (int32_t a = c + 1 + lane; a < k1; a += 32) {
            s0 += L[static_cast<int64_t>(c - 1) * ld + a] * vf[a];
            s1 += L[static_cast<int64_t>(c) * ld + a] * vf[a];
          }
          s0 = warp_sum(s0); s1 = warp_sum(s1);
          if (lane == 0) {
            vf[c] -= part[c - k0] + s1;
            vf[c - 1] -= part[c - 1 - k0] + s0;
          }
          c -= 2;
        } else {
          double s0 = 0.0;
          for (int32_t a = c + 1 + lane; a < k1; a += 32) s0 += L[static_cast<int64_t>(c) * ld + a] * vf[a];
          s0 = warp_sum(s0);
          if (lane == 0) vf[c] -= part[c - k0] + s0;
          c -= 1;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    k1 = k0;
  }
  for (int32_t c = threadIdx.x; c < nel; c += blockDim.x) xnew[rv[c]] = vf[c];
}

__global__ void gather_perm_kernel(int64_t n, const int32_t* perm, const double* src, double* dst) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[i] = src[perm[i]];
}

__global__ void scatter_perm_kernel(int64_t n, const int32_t* perm, const double* src, double* dst) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[perm[i]] = src[i];
}

}  // namespace



// x = M^{-1} b for one right-hand side, both on the device (original numbering).
kep_status run_solve(SolveLaunch& L, const double* b, double* x) {
  const Plan& P = *L.plan;
  cudaStream_t st = L.stream;
  const int g = L.num_sms * 4;
  KEP_LAUNCH(L.timer, KC_PERM, st, gather_perm_kernel<<<g, 256, 0, st>>>(P.n, L.d_perm, b, L.bnew));
  for (int32_t l = 0; l < P.nlevels; ++l) {
    const int32_t w = P.level_ptr[l + 1] - P.level_ptr[l];
    KEP_LAUNCH(L.timer, KC_SOLVE_FWD, st,
               sv_fwd_kernel<<<w, kSolveThreads, 0, st>>>(L.T, L.S, L.d_level_fronts + P.level_ptr[l], L.bnew,
                                                          L.vasm, L.vfac));
  }
  for (int32_t l = P.nlevels - 1; l >= 0; --l) {
    const int32_t w = P.level_ptr[l + 1] - P.level_ptr[l];
    KEP_LAUNCH(L.timer, KC_SOLVE_BWD, st,
               sv_bwd_kernel<<<w, kSolveThreads, 0, st>>>(L.T, L.S, L.d_level_fronts + P.level_ptr[l], L.xnew,
                                                          L.vfac));
  }
  KEP_LAUNCH(L.timer, KC_PERM, st, scatter_perm_kernel<<<g, 256, 0, st>>>(P.n, L.d_perm, L.xnew, x));
  return cudaGetLastError() == cudaSuccess ? KEP_OK : KEP_ERR_CUDA;
}

}  // namespace kep
