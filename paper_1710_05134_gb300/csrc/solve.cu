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
//
// Fronts of order >= 512 (with at least 32 pivots) are solved by a dataflow kernel instead of one
// CTA per front: their rows are cut into blocks of 64 (pivot blocks never split a 2x2 pair), every
// block is a work item taken from a counter in dependency order, and an item waits only for the
// pivot blocks it needs (forward: the earlier ones; backward: the later ones), which their CTAs
// publish through per-block flags.  Many CTAs then stream one front's L at once, and the chain of
// 64-row diagonal solves is the only serial part.  An item only waits for items taken before it,
// so the waits cannot deadlock whatever the CTA scheduling; every wait is also bounded in time.
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
// dataflow path for the large fronts
// ------------------------------------------------------------------------------------------
constexpr int kDfThreads = 256;

// first pivot of block b (blocks of kSolveBlk, a boundary moved by one where it would split a 2x2
// pair)
KEP_D int32_t blk_start(const int8_t* piv, int32_t b, int32_t nel) {
  if (b <= 0) return 0;
  int32_t s = b * kSolveBlk;
  if (s >= nel) return nel;
  return piv[s] == 0 ? s + 1 : s;
}
constexpr long long kDfWaitNs = 2000000000ll;   // a flag wait gives up after 2 s

KEP_D long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
KEP_D int32_t ld_acquire(const int32_t* p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
KEP_D void st_release(int32_t* p, int32_t v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 waits until *flag == want; false when the time limit passed (err set) or another CTA
// already gave up.
KEP_D bool df_wait(const int32_t* flag, int32_t want, int32_t* err) {
  if (ld_acquire(flag) == want) return true;
  const long long t0 = global_ns();
  unsigned ns = 32;
  while (true) {
    if (ld_acquire(flag) == want) return true;
    if (ld_acquire(err) != 0) return false;
    if (global_ns() - t0 > kDfWaitNs) { atomicExch(err, 1); return false; }
    __nanosleep(ns);
    if (ns < 256) ns *= 2;
  }
}

struct DfArgs {
  const int32_t* fronts;   // the level's dataflow fronts
  const int2* items;       // (front position, round) in the order items are taken
  int32_t nitems;
  int32_t* counter;        // next item (zeroed before the solve)
  int32_t* flags;          // per pivot block: the epoch value once its result is published
  const int32_t* fbase;    // per front: its first flag
  int32_t epoch;
  int32_t* err;            // set when a wait gave up
  // backward only: partial sums of the contribution rows, per front at part_base[front],
  // (pivot block x chunk) x (kSolveBlk + 1) doubles; pcnt counts the finished chunks per block
  double* part;
  const int64_t* part_base;
  int32_t* pcnt;
};

constexpr int kDfChunk = 1024;   // contribution rows per backward partial-sum item

// rows [r0, r1) of work item round r of front t: pivot block r (r < npb), else the r - npb-th
// block of 64 contribution rows
KEP_D void df_rows(const int8_t* piv, int32_t r, int32_t npb, int32_t nel, int32_t m, int32_t& r0, int32_t& r1) {
  if (r < npb) { r0 = blk_start(piv, r, nel); r1 = blk_start(piv, r + 1, nel); }
  else { r0 = nel + (r - npb) * kSolveBlk; r1 = min(m, r0 + kSolveBlk); }
}

// forward: y(block) = L11(block)^{-1} (f(block) - sum_{earlier blocks j} L(block, j) y(j)) for a
// pivot block, f(rows) -= sum_j L(rows, j) y(j) for contribution rows; y is left in vfac
__global__ void __launch_bounds__(kDfThreads) sv_df_fwd_kernel(FrontTables T, FactorSlot S, DfArgs A,
                                                               double* vfac) {
  __shared__ double ys[kSolveBlk + 1];
  __shared__ double red[4][kSolveBlk + 1];
  __shared__ double Lb[kSolveBlk + 1][kSolveBlk + 2];   // diagonal block, [column][row]
  __shared__ int8_t pb[kSolveBlk + 1];
  __shared__ int32_t s_item, s_ok;
  const int32_t tid = threadIdx.x, g = tid / kSolveBlk, rr = tid % kSolveBlk;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(A.counter, 1);
    __syncthreads();
    const int32_t it = s_item;
    __syncthreads();
    if (it >= A.nitems) return;
    const int2 I = A.items[it];
    const int32_t t = A.fronts[I.x];
    const int32_t d_in = S.d_in[t];
    const int32_t m = T.m_sym[t] + d_in;
    const int32_t nel = S.nelim[t];
    const int32_t npb = (nel + kSolveBlk - 1) / kSolveBlk;
    const int8_t* piv = S.piv + T.piv_off[t];
    const double* L = S.F + T.front_off[t];
    const int64_t ld = T.m_alloc[t];
    double* vf = vfac + T.vec_off[t];
    int32_t* fl = A.flags + A.fbase[t];
    int32_t r0, r1;
    df_rows(piv, I.y, npb, nel, m, r0, r1);
    const int32_t nr = r1 - r0;
    const bool pivot = I.y < npb;
    const int32_t ndep = pivot ? I.y : npb;
    const int32_t i0 = r0 + rr;
    const bool v0 = rr < nr, v1 = rr == 0 && nr > kSolveBlk;
    // a pivot item's diagonal block does not depend on the solve: it is staged before the waits,
    // off the chain of diagonal solves (the first barrier of the loop below orders it)
    if (pivot)
      for (int32_t e = tid; e < nr * nr; e += blockDim.x) {
        const int32_t c = e / nr, a = e % nr;
        if (a > c) Lb[c][a] = L[static_cast<int64_t>(r0 + c) * ld + r0 + a];
      }
    double acc0 = 0.0, acc1 = 0.0;
    bool ok = true;
    for (int32_t j = 0; j < ndep && ok; ++j) {
      const int32_t c0 = blk_start(piv, j, nel), c1 = blk_start(piv, j + 1, nel);
      if (tid == 0) s_ok = df_wait(fl + j, A.epoch, A.err) ? 1 : 0;
      __syncthreads();
      ok = s_ok != 0;
      if (ok && tid < c1 - c0) ys[tid] = __ldcg(vf + c0 + tid);
      __syncthreads();
      if (ok) {
#pragma unroll 4
        for (int32_t c = c0 + g; c < c1; c += 4) {
          const double yc = ys[c - c0];
          const double* col = L + static_cast<int64_t>(c) * ld + r0;
          if (v0) acc0 = fma(__ldg(col + rr), yc, acc0);
          if (v1) acc1 = fma(__ldg(col + kSolveBlk), yc, acc1);
        }
      }
      __syncthreads();
    }
    if (!ok) return;
    red[g][rr] = acc0;
    if (rr == 0) red[g][kSolveBlk] = acc1;
    __syncthreads();
    if (!pivot) {
      if (tid < nr) vf[r0 + tid] -= red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid];
      __syncthreads();
      continue;
    }
    if (tid < nr) {
      ys[tid] = vf[r0 + tid] - (red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid]);
      pb[tid] = piv[r0 + tid];
    }
    __syncthreads();
    if (tid < 32) {
      for (int32_t c = 0; c < nr;) {
        if (pb[c] == 2) {
          const double y0 = ys[c], y1 = ys[c + 1];
          for (int32_t a = c + 2 + tid; a < nr; a += 32) ys[a] -= Lb[c][a] * y0 + Lb[c + 1][a] * y1;
          c += 2;
        } else {
          const double y0 = ys[c];
          for (int32_t a = c + 1 + tid; a < nr; a += 32) ys[a] -= Lb[c][a] * y0;
          c += 1;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (tid < nr) vf[r0 + tid] = ys[tid];
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(fl + I.y, A.epoch);
    }
  }
}

// backward preparation: the solution on the contribution rows (written by the ancestors)
__global__ void sv_df_bwd_prep_kernel(FrontTables T, FactorSlot S, const int32_t* fronts, const double* xnew,
                                      double* vfac) {
  const int32_t t = fronts[blockIdx.y];
  const int32_t m = T.m_sym[t] + S.d_in[t];
  const int32_t nel = S.nelim[t];
  double* vf = vfac + T.vec_off[t];
  const int32_t* rv = S.rowvar + T.vec_off[t];
  for (int32_t i = nel + blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    vf[i] = xnew[rv[i]];
}

// backward.  Items with y < 0 (taken first): the partial sums sum_{a in chunk} L(a, block) x(a) of
// pivot block b over one chunk of kDfChunk contribution rows (their x is known), stored for the
// block's item.  Items with y >= 0, pivot block b = npb - 1 - y (from the last block down):
// x(block) = L11(block)^{-T} (D^{-1} y(block) - sum_{rows a below the block} L(a, block) x(a)), the
// contribution rows' part added from the stored partial sums in chunk order, the later pivot
// blocks as they are published
__global__ void __launch_bounds__(kDfThreads) sv_df_bwd_kernel(FrontTables T, FactorSlot S, DfArgs A,
                                                               double* vfac, double* xnew) {
  constexpr int kCols = (kSolveBlk + 1 + 7) / 8;
  __shared__ double xs[kSolveBlk + 1];
  __shared__ double part[kSolveBlk + 1];
  __shared__ double LbT[kSolveBlk + 1][kSolveBlk + 2];  // diagonal block, [row][column]
  __shared__ int8_t pb[kSolveBlk + 1];
  __shared__ int32_t s_item, s_ok;
  const int32_t tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(A.counter, 1);
    __syncthreads();
    const int32_t it = s_item;
    __syncthreads();
    if (it >= A.nitems) return;
    const int2 I = A.items[it];
    const int32_t t = A.fronts[I.x];
    const int32_t d_in = S.d_in[t];
    const int32_t m = T.m_sym[t] + d_in;
    const int32_t nel = S.nelim[t];
    const int32_t npb = (nel + kSolveBlk - 1) / kSolveBlk;
    const int32_t nch = (m - nel + kDfChunk - 1) / kDfChunk;
    const bool partial = I.y < 0;
    const int32_t b = partial ? (-1 - I.y) / max(nch, 1) : npb - 1 - I.y;
    const int8_t* piv = S.piv + T.piv_off[t];
    const double* L = S.F + T.front_off[t];
    const int64_t ld = T.m_alloc[t];
    double* vf = vfac + T.vec_off[t];
    int32_t* fl = A.flags + A.fbase[t];
    const int32_t k0 = blk_start(piv, b, nel), k1 = blk_start(piv, b + 1, nel);
    const int32_t kb = k1 - k0;
    double* pbase = A.part + A.part_base[t] + static_cast<int64_t>(b) * nch * (kSolveBlk + 1);
    double acc[kCols];
#pragma unroll
    for (int j = 0; j < kCols; ++j) acc[j] = 0.0;
    if (partial) {
      const int32_t ch = (-1 - I.y) % nch;
      const int32_t a0 = nel + ch * kDfChunk, a1 = min(m, a0 + kDfChunk);
      for (int32_t a = a0 + lane; a < a1; a += 32) {
        const double xa = __ldcg(vf + a);
#pragma unroll
        for (int j = 0; j < kCols; ++j) {
          const int32_t c = warp + 8 * j;
          if (c < kb) acc[j] = fma(__ldg(L + static_cast<int64_t>(k0 + c) * ld + a), xa, acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kCols; ++j) {
        const int32_t c = warp + 8 * j;
        const double v = warp_sum(acc[j]);
        if (lane == 0 && c < kb) pbase[static_cast<int64_t>(ch) * (kSolveBlk + 1) + c] = v;
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        atomicAdd(A.pcnt + A.fbase[t] + b, 1);
      }
      continue;
    }
    // the diagonal block (transposed) is staged before the waits, off the chain of diagonal
    // solves (the first barrier of the loop below, or the one after the partial sums, orders it)
    for (int32_t e = tid; e < kb * kb; e += blockDim.x) {
      const int32_t c = e / kb, a = e % kb;
      if (a > c) LbT[a][c] = L[static_cast<int64_t>(k0 + c) * ld + k0 + a];
    }
    // later pivot blocks, last first
    bool ok = true;
    for (int32_t bp = npb - 1; bp > b && ok; --bp) {
      const int32_t s0 = blk_start(piv, bp, nel), s1 = blk_start(piv, bp + 1, nel);
      if (tid == 0) s_ok = df_wait(fl + (npb - 1 - bp), A.epoch, A.err) ? 1 : 0;
      __syncthreads();
      ok = s_ok != 0;
      if (ok && tid < s1 - s0) xs[tid] = __ldcg(vf + s0 + tid);
      __syncthreads();
      if (ok) {
        for (int32_t a = s0 + lane; a < s1; a += 32) {
          const double xa = xs[a - s0];
#pragma unroll
          for (int j = 0; j < kCols; ++j) {
            const int32_t c = warp + 8 * j;
            if (c < kb) acc[j] = fma(__ldg(L + static_cast<int64_t>(k0 + c) * ld + a), xa, acc[j]);
          }
        }
      }
      __syncthreads();
    }
    if (!ok) return;
#pragma unroll
    for (int j = 0; j < kCols; ++j) {
      const int32_t c = warp + 8 * j;
      const double v = warp_sum(acc[j]);
      if (lane == 0 && c < kb) part[c] = v;
    }
    // the contribution rows' partial sums, once all chunks of this block are in (chunk order)
    if (nch > 0) {
      if (tid == 0) {
        bool done = false;
        const long long t0 = global_ns();
        unsigned ns = 32;
        while (!done) {
          done = ld_acquire(A.pcnt + A.fbase[t] + b) >= nch;
          if (done) break;
          if (ld_acquire(A.err) != 0) break;
          if (global_ns() - t0 > kDfWaitNs) { atomicExch(A.err, 1); break; }
          __nanosleep(ns);
          if (ns < 256) ns *= 2;
        }
        s_ok = done ? 1 : 0;
      }
      __syncthreads();
      if (!s_ok) return;
      if (tid < kb) {
        double sacc = 0.0;
        for (int32_t ch = 0; ch < nch; ++ch) sacc += __ldcg(pbase + static_cast<int64_t>(ch) * (kSolveBlk + 1) + tid);
        part[tid] += sacc;
      }
    }
    if (tid < kb) pb[tid] = piv[k0 + tid];
    __syncthreads();
    // z = D^{-1} y on the block's rows (a 2x2 pair never straddles blocks)
    if (tid < kb) {
      const int32_t c = k0 + tid;
      const int64_t po = T.piv_off[t];
      const double yc = vf[c];
      double z;
      if (pb[tid] == 1) {
        z = yc / S.Dd[po + c];
      } else if (pb[tid] == 2) {
        const double a = S.Dd[po + c], cc = S.Dd[po + c + 1], bb = S.De[po + c];
        z = (cc * yc - bb * vf[c + 1]) / (a * cc - bb * bb);
      } else {
        const double a = S.Dd[po + c - 1], cc = S.Dd[po + c], bb = S.De[po + c - 1];
        z = (a * yc - bb * vf[c - 1]) / (a * cc - bb * bb);
      }
      xs[tid] = z - part[tid];
    }
    __syncthreads();
    // L11^T x = z - part, last row first in column (axpy) form: once x(c) is final, row c of L11
    // is subtracted from the rows above it (lanes over those rows, no reductions on the chain).
    // The entry (c, c-1) inside a 2x2 pair is not part of the unit triangle and is skipped.
    if (tid < 32) {
      for (int32_t c = kb - 1; c > 0; --c) {
        const double xc = xs[c];
        const int32_t lim = pb[c] == 0 ? c - 1 : c;    // pb 0: second of a pair at (c-1, c)
        for (int32_t a = lane; a < lim; a += 32) xs[a] -= LbT[c][a] * xc;
        __syncwarp();
      }
    }
    __syncthreads();
    if (tid < kb) {
      vf[k0 + tid] = xs[tid];
      xnew[S.rowvar[T.vec_off[t] + k0 + tid]] = xs[tid];
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(fl + I.y, A.epoch);
    }
  }
}

// assembly of the front's right-hand side (children in order) and the pivot permutation
__global__ void __launch_bounds__(1024) sv_df_prep_kernel(FrontTables T, FactorSlot S, const int32_t* fronts,
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
  if (cudaMemsetAsync(L.df_counters, 0, sizeof(int32_t) * (1 + 2 * static_cast<size_t>(P.nlevels)), st) != cudaSuccess ||
      cudaMemsetAsync(L.df_pcnt, 0, sizeof(int32_t) * static_cast<size_t>(L.df_nflags), st) != cudaSuccess)
    return KEP_ERR_CUDA;
  KEP_LAUNCH(L.timer, KC_PERM, st, gather_perm_kernel<<<g, 256, 0, st>>>(P.n, L.d_perm, b, L.bnew));
  auto df_args = [&](int32_t l, bool fwd) {
    DfArgs A;
    A.fronts = L.d_level_fronts + P.level_ptr[l];
    const int32_t* off = fwd ? L.h_df_fwd_off : L.h_df_bwd_off;
    A.items = (fwd ? L.df_fwd_items : L.df_bwd_items) + off[l];
    A.nitems = off[l + 1] - off[l];
    A.counter = L.df_counters + 1 + (fwd ? 0 : P.nlevels) + l;
    A.flags = L.df_flags;
    A.fbase = L.df_fbase;
    A.epoch = fwd ? 2 * L.epoch + 1 : 2 * L.epoch + 2;
    A.err = L.df_counters;
    A.part = L.df_part;
    A.part_base = L.df_part_base;
    A.pcnt = L.df_pcnt;
    return A;
  };
  for (int32_t l = 0; l < P.nlevels; ++l) {
    const int32_t lb = P.level_ptr[l], w = P.level_ptr[l + 1] - lb, nbig = P.level_nbig_solve[l];
    if (nbig > 0) {
      const int32_t* fr = L.d_level_fronts + lb;
      KEP_LAUNCH(L.timer, KC_SOLVE_FWD, st, sv_df_prep_kernel<<<nbig, 1024, 0, st>>>(L.T, L.S, fr, L.bnew, L.vasm, L.vfac));
      const DfArgs A = df_args(l, true);
      if (A.nitems > 0)
        KEP_LAUNCH(L.timer, KC_SOLVE_FWD, st,
                   sv_df_fwd_kernel<<<std::min(A.nitems, g), kDfThreads, 0, st>>>(L.T, L.S, A, L.vfac));
    }
    if (w > nbig)
      KEP_LAUNCH(L.timer, KC_SOLVE_FWD, st,
                 sv_fwd_kernel<<<w - nbig, kSolveThreads, 0, st>>>(L.T, L.S, L.d_level_fronts + lb + nbig, L.bnew,
                                                                   L.vasm, L.vfac));
  }
  for (int32_t l = P.nlevels - 1; l >= 0; --l) {
    const int32_t lb = P.level_ptr[l], w = P.level_ptr[l + 1] - lb, nbig = P.level_nbig_solve[l];
    if (nbig > 0) {
      const int32_t* fr = L.d_level_fronts + lb;
      KEP_LAUNCH(L.timer, KC_SOLVE_BWD, st,
                 sv_df_bwd_prep_kernel<<<dim3(8, nbig), 256, 0, st>>>(L.T, L.S, fr, L.xnew, L.vfac));
      const DfArgs A = df_args(l, false);
      if (A.nitems > 0)
        KEP_LAUNCH(L.timer, KC_SOLVE_BWD, st,
                   sv_df_bwd_kernel<<<std::min(A.nitems, g), kDfThreads, 0, st>>>(L.T, L.S, A, L.vfac, L.xnew));
    }
    if (w > nbig)
      KEP_LAUNCH(L.timer, KC_SOLVE_BWD, st,
                 sv_bwd_kernel<<<w - nbig, kSolveThreads, 0, st>>>(L.T, L.S, L.d_level_fronts + lb + nbig, L.xnew,
                                                                   L.vfac));
  }
  KEP_LAUNCH(L.timer, KC_PERM, st, scatter_perm_kernel<<<g, 256, 0, st>>>(P.n, L.d_perm, L.xnew, x));
  return cudaGetLastError() == cudaSuccess ? KEP_OK : KEP_ERR_CUDA;
}

// Work items of the dataflow solve for one factorization: per level, the leading
// level_nbig_solve[l] fronts; forward rounds r = 0, 1, ... take pivot block r (then contribution
// block r - npb) of every front that has one, backward rounds the pivot blocks from the last.
void build_df_items(const Plan& P, const int32_t* nelim, const int32_t* din, std::vector<int2>& items,
                    std::vector<int32_t>& fwd_off, std::vector<int32_t>& bwd_off, int64_t& bwd_start,
                    std::vector<int64_t>& part_base, int64_t& part_total) {
  items.clear();
  fwd_off.assign(P.nlevels + 1, 0);
  bwd_off.assign(P.nlevels + 1, 0);
  part_base.assign(P.nfronts, 0);
  part_total = 0;
  std::vector<int32_t> npb, nall, nch;
  for (int pass = 0; pass < 2; ++pass) {
    const int64_t base = static_cast<int64_t>(items.size());
    if (pass == 1) bwd_start = base;
    for (int32_t l = 0; l < P.nlevels; ++l) {
      (pass == 0 ? fwd_off : bwd_off)[l] = static_cast<int32_t>(items.size() - base);
      const int32_t lb = P.level_ptr[l], nbig = P.level_nbig_solve[l];
      npb.assign(nbig, 0);
      nall.assign(nbig, 0);
      nch.assign(nbig, 0);
      int32_t rounds = 0;
      for (int32_t q = 0; q < nbig; ++q) {
        const int32_t t = P.level_fronts[lb + q];
        const int32_t nel = nelim[t], m = P.m_sym[t] + din[t];
        npb[q] = (nel + kSolveBlk - 1) / kSolveBlk;
        nch[q] = (m - nel + kDfChunk - 1) / kDfChunk;
        nall[q] = pass == 0 ? npb[q] + (m - nel + kSolveBlk - 1) / kSolveBlk : npb[q];
        rounds = std::max(rounds, nall[q]);
        if (pass == 1) {
          part_base[t] = part_total;
          part_total += static_cast<int64_t>(npb[q]) * nch[q] * (kSolveBlk + 1);
        }
      }
      if (pass == 1)   // the contribution rows' partial sums first: they wait for nothing
        for (int32_t q = 0; q < nbig; ++q)
          for (int32_t v = 0; v < npb[q] * nch[q]; ++v) items.push_back(make_int2(q, -1 - v));
      for (int32_t r = 0; r < rounds; ++r)
        for (int32_t q = 0; q < nbig; ++q)
          if (r < nall[q]) items.push_back(make_int2(q, r));
    }
    (pass == 0 ? fwd_off : bwd_off)[P.nlevels] = static_cast<int32_t>(items.size() - base);
  }
}

// Flag offsets of the dataflow solve: per front, one flag per possible pivot block.
int64_t df_flag_bases(const Plan& P, std::vector<int32_t>& fbase) {
  fbase.assign(P.nfronts, 0);
  int64_t tot = 0;
  for (int32_t t = 0; t < P.nfronts; ++t) {
    fbase[t] = static_cast<int32_t>(tot);
    tot += (P.p_alloc[t] + kSolveBlk - 1) / kSolveBlk + 1;
  }
  return tot;
}

}  // namespace kep
