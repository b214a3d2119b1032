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
#include <algorithm>

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
  __shared__ double Lb[kBlk + 1][kBlk + 2];   // diagonal block, [column][row]
  __shared__ double y[kBlk + 1];
  __shared__ int8_t pb[kBlk + 1];
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
    // the block's triangle, right-hand side and pivot types in shared memory
    for (int32_t e = threadIdx.x; e < kb * kb; e += blockDim.x) {
      const int32_t c = e / kb, a = e % kb;
      Lb[c][a] = L[static_cast<int64_t>(k0 + c) * ld + k0 + a];
    }
    for (int32_t c = threadIdx.x; c < kb; c += blockDim.x) { y[c] = vf[k0 + c]; pb[c] = piv[k0 + c]; }
    __syncthreads();
    if (warp == 0) {
      for (int32_t c = 0; c < kb;) {
        if (pb[c] == 2) {
          const double y0 = y[c], y1 = y[c + 1];
          for (int32_t a = c + 2 + lane; a < kb; a += 32) y[a] -= Lb[c][a] * y0 + Lb[c + 1][a] * y1;
          c += 2;
        } else {
          const double y0 = y[c];
          for (int32_t a = c + 1 + lane; a < kb; a += 32) y[a] -= Lb[c][a] * y0;
          c += 1;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int32_t c = threadIdx.x; c < kb; c += blockDim.x) vf[k0 + c] = y[c];
    for (int32_t a = k1 + threadIdx.x; a < m; a += blockDim.x) {
      double s = 0.0;
      for (int32_t c = 0; c < kb; ++c) s += L[static_cast<int64_t>(k0 + c) * ld + a] * y[c];
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
  __shared__ double Lb[kBlk + 1][kBlk + 2];   // diagonal block, [column][row]
  __shared__ double xb[kBlk + 1];
  __shared__ int8_t pb[kBlk + 1];
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
    for (int32_t e = threadIdx.x; e < kb * kb; e += blockDim.x) {
      const int32_t c = e / kb, a = e % kb;
      Lb[c][a] = L[static_cast<int64_t>(k0 + c) * ld + k0 + a];
    }
    for (int32_t c = threadIdx.x; c < kb; c += blockDim.x) { xb[c] = vf[k0 + c]; pb[c] = piv[k0 + c]; }
    __syncthreads();
    if (warp == 0) {
      for (int32_t c = kb - 1; c >= 0;) {
        if (pb[c] == 0) {                     // second of a pair at (c-1, c)
          double s0 = 0.0, s1 = 0.0;
          for (int32_t a = c + 1 + lane; a < kb; a += 32) {
            s0 += Lb[c - 1][a] * xb[a];
            s1 += Lb[c][a] * xb[a];
          }
          s0 = warp_sum(s0); s1 = warp_sum(s1);
          if (lane == 0) {
            xb[c] -= part[c] + s1;
            xb[c - 1] -= part[c - 1] + s0;
          }
          c -= 2;
        } else {
          double s0 = 0.0;
          for (int32_t a = c + 1 + lane; a < kb; a += 32) s0 += Lb[c][a] * xb[a];
          s0 = warp_sum(s0);
          if (lane == 0) xb[c] -= part[c] + s0;
          c -= 1;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int32_t c = threadIdx.x; c < kb; c += blockDim.x) vf[k0 + c] = xb[c];
    __syncthreads();
    k1 = k0;
  }
  for (int32_t c = threadIdx.x; c < nel; c += blockDim.x) xnew[rv[c]] = vf[c];
}

// ------------------------------------------------------------------------------------------
// multi-block path for the largest fronts: the pivot range is cut into blocks of kSolveBlk
// (boundaries moved by one where they would split a 2x2 pair); every block is one launch whose
// CTAs all reproduce the small diagonal-block solve and then update their own rows.  All such
// fronts of a level share the launches: grid.y = front (fronts[blockIdx.y]), grid.x = the CTAs of
// one front.
// ------------------------------------------------------------------------------------------
KEP_D int32_t blk_start(const int8_t* piv, int32_t b, int32_t nel) {
  if (b <= 0) return 0;
  int32_t s = b * kSolveBlk;
  if (s >= nel) return nel;
  return piv[s] == 0 ? s + 1 : s;
}

// assembly of the front's right-hand side (children in order) and the pivot permutation
__global__ void __launch_bounds__(1024) sv_big_prep_kernel(FrontTables T, FactorSlot S, const int32_t* fronts,
                                                           const double* bnew, double* vasm, double* vfac) {
  const int32_t t = fronts[blockIdx.x];
  const int32_t d_in = S.d_in[t];
  const int32_t m = T.m_sym[t] + d_in;
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
}

// forward block b: y(block) = L11^{-1} f(block) (every CTA), CTA 0 stores it in ysol; rows below
// the block: f(a) -= L(a, block) y(block)
__global__ void __launch_bounds__(256) sv_big_fwd_kernel(FrontTables T, FactorSlot S, const int32_t* fronts,
                                                         int32_t b, double* vfac, double* ysol) {
  __shared__ double y[kSolveBlk + 1];
  __shared__ double Lb[kSolveBlk + 1][kSolveBlk + 2];   // diagonal block, [column][row]
  __shared__ int8_t pb[kSolveBlk + 1];
  const int32_t t = fronts[blockIdx.y];
  const int32_t d_in = S.d_in[t];
  const int32_t m = T.m_sym[t] + d_in;
  const int32_t nel = S.nelim[t];
  const int8_t* piv = S.piv + T.piv_off[t];
  const int32_t k0 = blk_start(piv, b, nel), k1 = blk_start(piv, b + 1, nel);
  if (k0 >= k1) return;
  const double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  double* vf = vfac + T.vec_off[t];
  double* ys = ysol + T.vec_off[t];
  const int32_t kb = k1 - k0;
  for (int32_t e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    const int32_t c = e / kb, a = e % kb;
    Lb[c][a] = L[static_cast<int64_t>(k0 + c) * ld + k0 + a];
  }
  if (threadIdx.x < kb) { y[threadIdx.x] = vf[k0 + threadIdx.x]; pb[threadIdx.x] = piv[k0 + threadIdx.x]; }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int32_t c = 0; c < kb;) {
      if (pb[c] == 2) {
        const double y0 = y[c], y1 = y[c + 1];
        for (int32_t a = c + 2 + lane; a < kb; a += 32) y[a] -= Lb[c][a] * y0 + Lb[c + 1][a] * y1;
        c += 2;
      } else {
        const double y0 = y[c];
        for (int32_t a = c + 1 + lane; a < kb; a += 32) y[a] -= Lb[c][a] * y0;
        c += 1;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x < kb) ys[k0 + threadIdx.x] = y[threadIdx.x];
  for (int32_t a = k1 + blockIdx.x * blockDim.x + threadIdx.x; a < m; a += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int32_t c = 0; c < kb; ++c) s = fma(L[static_cast<int64_t>(k0 + c) * ld + a], y[c], s);
    vf[a] -= s;
  }
}

// backward preparation: solution on the contribution rows, z = D^{-1} y on the pivots
__global__ void sv_big_bwd_prep_kernel(FrontTables T, FactorSlot S, const int32_t* fronts, const double* xnew,
                                       const double* ysol, double* vfac) {
  const int32_t t = fronts[blockIdx.y];
  const int32_t d_in = S.d_in[t];
  const int32_t m = T.m_sym[t] + d_in;
  const int32_t nel = S.nelim[t];
  double* vf = vfac + T.vec_off[t];
  const double* ys = ysol + T.vec_off[t];
  const int32_t* rv = S.rowvar + T.vec_off[t];
  const int8_t* piv = S.piv + T.piv_off[t];
  const double* Dd = S.Dd + T.piv_off[t];
  const double* De = S.De + T.piv_off[t];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    if (i >= nel) { vf[i] = xnew[rv[i]]; continue; }
    if (piv[i] == 1) {
      vf[i] = ys[i] / Dd[i];
    } else if (piv[i] == 2) {
      const double a = Dd[i], cc = Dd[i + 1], bb = De[i];
      const double det = a * cc - bb * bb;
      vf[i] = (cc * ys[i] - bb * ys[i + 1]) / det;
    } else {
      const double a = Dd[i - 1], cc = Dd[i], bb = De[i - 1];
      const double det = a * cc - bb * bb;
      vf[i] = (a * ys[i] - bb * ys[i - 1]) / det;
    }
  }
}

// backward block b, part 1: per-CTA partial sums s_c = sum_{a >= k1} L(a, k0 + c) x(a), stored
// column-major (partial[c * gridDim.x + cta]); warp w owns columns w, w + 8, ..., its lanes stride
// the CTA's rows
__global__ void __launch_bounds__(256) sv_big_bwd_partial_kernel(FrontTables T, FactorSlot S, const int32_t* fronts,
                                                                 int32_t step, const double* vfac, double* partial) {
  constexpr int kCols = (kSolveBlk + 1 + 7) / 8;
  const int32_t t = fronts[blockIdx.y];
  const int32_t d_in = S.d_in[t];
  const int32_t m = T.m_sym[t] + d_in;
  const int32_t nel = S.nelim[t];
  const int32_t b = (nel + kSolveBlk - 1) / kSolveBlk - 1 - step;   // blocks from the last one down
  if (b < 0) return;
  partial += static_cast<int64_t>(blockIdx.y) * (kSolveBlk + 1) * gridDim.x;
  const int8_t* piv = S.piv + T.piv_off[t];
  const int32_t k0 = blk_start(piv, b, nel), k1 = blk_start(piv, b + 1, nel);
  const int32_t kb = k1 - k0;
  const double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  const double* vf = vfac + T.vec_off[t];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  double acc[kCols];
#pragma unroll
  for (int j = 0; j < kCols; ++j) acc[j] = 0.0;
  for (int32_t a = k1 + blockIdx.x * 32 + lane; a < m; a += gridDim.x * 32) {
    const double xa = vf[a];
#pragma unroll
    for (int j = 0; j < kCols; ++j) {
      const int32_t c = warp + 8 * j;
      if (c < kb) acc[j] = fma(L[static_cast<int64_t>(k0 + c) * ld + a], xa, acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < kCols; ++j) {
    const int32_t c = warp + 8 * j;
    const double v = warp_sum(acc[j]);
    if (lane == 0 && c < kb) partial[static_cast<int64_t>(c) * gridDim.x + blockIdx.x] = v;
  }
}

// backward block b, part 2 (one CTA): add the partials, solve the block's unit upper triangle
__global__ void __launch_bounds__(128) sv_big_bwd_block_kernel(FrontTables T, FactorSlot S, const int32_t* fronts,
                                                               int32_t step, int32_t nparts, const double* partial,
                                                               double* vfac) {
  __shared__ double part[kSolveBlk + 1];
  __shared__ double Lb[kSolveBlk + 1][kSolveBlk + 2];   // diagonal block, [column][row]
  __shared__ double xb[kSolveBlk + 1];
  __shared__ int8_t pb[kSolveBlk + 1];
  const int32_t t = fronts[blockIdx.x];
  const int32_t nel = S.nelim[t];
  const int32_t b = (nel + kSolveBlk - 1) / kSolveBlk - 1 - step;
  if (b < 0) return;
  partial += static_cast<int64_t>(blockIdx.x) * (kSolveBlk + 1) * nparts;
  const int8_t* piv = S.piv + T.piv_off[t];
  const int32_t k0 = blk_start(piv, b, nel), k1 = blk_start(piv, b + 1, nel);
  const int32_t kb = k1 - k0;
  const double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  double* vf = vfac + T.vec_off[t];
  for (int32_t e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    const int32_t c = e / kb, a = e % kb;
    Lb[c][a] = L[static_cast<int64_t>(k0 + c) * ld + k0 + a];
  }
  {  // column sums of the partials: warp w takes columns w, w + 4, ..., its lanes the CTAs
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int32_t c = warp; c < kb; c += blockDim.x / 32) {
      double s = 0.0;
      for (int32_t q = lane; q < nparts; q += 32) s += partial[static_cast<int64_t>(c) * nparts + q];
      s = warp_sum(s);
      if (lane == 0) part[c] = s;
    }
  }
  if (threadIdx.x < kb) {
    xb[threadIdx.x] = vf[k0 + threadIdx.x];
    pb[threadIdx.x] = piv[k0 + threadIdx.x];
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int32_t c = kb - 1; c >= 0;) {
      if (pb[c] == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int32_t a = c + 1 + lane; a < kb; a += 32) {
          s0 += Lb[c - 1][a] * xb[a];
          s1 += Lb[c][a] * xb[a];
        }
        s0 = warp_sum(s0); s1 = warp_sum(s1);
        if (lane == 0) { xb[c] -= part[c] + s1; xb[c - 1] -= part[c - 1] + s0; }
        c -= 2;
      } else {
        double s0 = 0.0;
        for (int32_t a = c + 1 + lane; a < kb; a += 32) s0 += Lb[c][a] * xb[a];
        s0 = warp_sum(s0);
        if (lane == 0) xb[c] -= part[c] + s0;
        c -= 1;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (threadIdx.x < kb) vf[k0 + threadIdx.x] = xb[threadIdx.x];
}

__global__ void sv_big_scatter_kernel(FrontTables T, FactorSlot S, const int32_t* fronts, const double* vfac,
                                      double* xnew) {
  const int32_t t = fronts[blockIdx.y];
  const int32_t nel = S.nelim[t];
  const double* vf = vfac + T.vec_off[t];
  const int32_t* rv = S.rowvar + T.vec_off[t];
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nel; c += gridDim.x * blockDim.x) xnew[rv[c]] = vf[c];
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
  // the level's multi-block fronts: their block count and CTAs per front (a uniform grid)
  auto big_shape = [&](int32_t lb, int32_t nbig, int32_t& maxblk, int& gx) {
    int64_t rows = 0;
    maxblk = 0;
    for (int32_t i = 0; i < nbig; ++i) {
      const int32_t t = P.level_fronts[lb + i];
      rows = std::max<int64_t>(rows, P.m_alloc[t]);
      maxblk = std::max(maxblk, (L.h_nelim[t] + kSolveBlk - 1) / kSolveBlk);
    }
    gx = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((rows + 255) / 256 + 1, g / std::max(1, nbig))));
  };
  for (int32_t l = 0; l < P.nlevels; ++l) {
    const int32_t lb = P.level_ptr[l], w = P.level_ptr[l + 1] - lb, nbig = P.level_nbig_solve[l];
    if (nbig > 0) {
      int32_t maxblk;
      int gx;
      big_shape(lb, nbig, maxblk, gx);
      const int32_t* fr = L.d_level_fronts + lb;
      KEP_LAUNCH(L.timer, KC_SOLVE_FWD, st, sv_big_prep_kernel<<<nbig, 1024, 0, st>>>(L.T, L.S, fr, L.bnew, L.vasm, L.vfac));
      for (int32_t bb = 0; bb < maxblk; ++bb)
        KEP_LAUNCH(L.timer, KC_SOLVE_FWD, st,
                   sv_big_fwd_kernel<<<dim3(gx, nbig), 256, 0, st>>>(L.T, L.S, fr, bb, L.vfac, L.vasm));
    }
    if (w > nbig)
      KEP_LAUNCH(L.timer, KC_SOLVE_FWD, st,
                 sv_fwd_kernel<<<w - nbig, kSolveThreads, 0, st>>>(L.T, L.S, L.d_level_fronts + lb + nbig, L.bnew,
                                                                   L.vasm, L.vfac));
  }
  for (int32_t l = P.nlevels - 1; l >= 0; --l) {
    const int32_t lb = P.level_ptr[l], w = P.level_ptr[l + 1] - lb, nbig = P.level_nbig_solve[l];
    if (nbig > 0) {
      int32_t maxblk;
      int gx;
      big_shape(lb, nbig, maxblk, gx);
      const int32_t* fr = L.d_level_fronts + lb;
      KEP_LAUNCH(L.timer, KC_SOLVE_BWD, st,
                 sv_big_bwd_prep_kernel<<<dim3(gx, nbig), 256, 0, st>>>(L.T, L.S, fr, L.xnew, L.vasm, L.vfac));
      for (int32_t step = 0; step < maxblk; ++step) {
        KEP_LAUNCH(L.timer, KC_SOLVE_BWD, st,
                   sv_big_bwd_partial_kernel<<<dim3(gx, nbig), 256, 0, st>>>(L.T, L.S, fr, step, L.vfac, L.partial));
        KEP_LAUNCH(L.timer, KC_SOLVE_BWD, st,
                   sv_big_bwd_block_kernel<<<nbig, 128, 0, st>>>(L.T, L.S, fr, step, gx, L.partial, L.vfac));
      }
      KEP_LAUNCH(L.timer, KC_SOLVE_BWD, st,
                 sv_big_scatter_kernel<<<dim3(gx, nbig), 256, 0, st>>>(L.T, L.S, fr, L.vfac, L.xnew));
    }
    if (w > nbig)
      KEP_LAUNCH(L.timer, KC_SOLVE_BWD, st,
                 sv_bwd_kernel<<<w - nbig, kSolveThreads, 0, st>>>(L.T, L.S, L.d_level_fronts + lb + nbig, L.xnew,
                                                                   L.vfac));
  }
  KEP_LAUNCH(L.timer, KC_PERM, st, scatter_perm_kernel<<<g, 256, 0, st>>>(P.n, L.d_perm, L.xnew, x));
  return cudaGetLastError() == cudaSuccess ? KEP_OK : KEP_ERR_CUDA;
}

}  // namespace kep
