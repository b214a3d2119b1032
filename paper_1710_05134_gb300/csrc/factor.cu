// Numeric multifrontal LDL^T of ca*A + cb*B on the GPU (Algorithm 1', the factorization and
// inertia steps; task (iv)-(vi) of Section 4.3).
//
// Fronts are processed level by level (leaves first).  All fronts of a level form a batch and
// advance in lock step; every kernel reads its front's dynamic state (delays received, pivots
// eliminated so far) from device memory, so no host synchronisation is needed inside a level.
//
// Per front:
//   assembly   zero the storage, scatter the original entries ca*a + cb*b, extend-add the
//              children's contribution blocks (their delayed columns first);
//   pivoting   a posteriori threshold pivoting on blocks of kPanel fully-summed columns:
//              Bunch-Kaufman (alpha = (1+sqrt 17)/8) inside the diagonal block, then every row
//              below solves against that block and the largest |l| of each column is tested
//              against 1/u; the accepted leading pivots are kept, the rest of the block is
//              restored and retried in the next block; a front whose block fails entirely passes
//              its remaining fully-summed columns to the parent (delayed pivots);
//   update     Schur complement of the trailing matrix with the accepted pivots, FP64 FMA tiles;
//   inertia    the sign rule for 1x1 and 2x2 pivots of D, summed per front.
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "kep_device.cuh"

namespace kep {

namespace {

constexpr int kTile = 64;          // default FP64 Schur-update tile edge (32 or 64, chosen per context)
constexpr int kRowTile = 64;       // rows per CTA in the row-parallel kernels

template <typename X>
struct TypeTag { using type = X; };

KEP_D int32_t children_delays(const FrontTables& T, const FactorSlot& S, int32_t t, bool& bad) {
  int32_t d = 0;
  for (int32_t c = T.child_ptr[t]; c < T.child_ptr[t + 1]; ++c) {
    int32_t ch = T.child_idx[c];
    if (S.d_in[ch] < 0) bad = true;
    d += S.d_out[ch];
  }
  return d;
}

// ------------------------------------------------------------------------------------------
// assembly
// ------------------------------------------------------------------------------------------
__global__ void lf_init_kernel(FrontTables T, SlotSet SS, LargeWork W, Batch B) {
  const int32_t b = B.e0 + blockIdx.y;
  const int32_t t = B.lf[b];
  const int32_t g = entry_shift(B, b);
  const FactorSlot& S = SS.s[g];
  double* const cbpool = SS.cbpool[g];
  bool child_bad = false;
  const int32_t d_in = children_delays(T, S, t, child_bad);
  const bool over = d_in > T.m_alloc[t] - T.m_sym[t];
  const bool bad = child_bad || over;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // a failed front records how many delayed columns it would have had to hold
    S.d_in[t] = bad ? -((over && !child_bad) ? d_in : 0) - 1 : d_in;
    S.nelim[t] = 0;
    S.d_out[t] = 0;
    S.cnt[3 * t] = S.cnt[3 * t + 1] = S.cnt[3 * t + 2] = 0;
    W.k[b] = 0; W.q[b] = 0; W.w[b] = 0; W.fails[b] = 0; W.swap[b] = 0; W.done[b] = bad ? 1 : 0;
    W.ws[b] = 0; W.we[b] = 0; W.kend[b] = 0; W.flush[b] = 0; W.reset[b] = 1; W.finish[b] = 0;
    if (bad) {
      atomicOr(&S.status[0], ST_POOL);
      atomicCAS(&S.status[1], -1, t);
    }
  }
  if (bad) return;
  const FrontView v = front_view(T, S, cbpool, t, d_in);
  for (int32_t j = blockIdx.x; j < v.p; j += gridDim.x) {
    double* col = v.L + static_cast<int64_t>(j) * v.ldL;
    for (int32_t i = j + threadIdx.x; i < v.m; i += blockDim.x) col[i] = 0.0;
  }
  for (int32_t j = blockIdx.x; j < v.c; j += gridDim.x) {
    double* col = v.C + static_cast<int64_t>(j) * v.c;
    for (int32_t i = j + threadIdx.x; i < v.c; i += blockDim.x) col[i] = 0.0;
  }
  int32_t* rv = S.rowvar + T.vec_off[t];
  int32_t* ap = S.apos + T.vec_off[t];
  const int32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int32_t i = gt; i < v.m; i += gs) {
    ap[i] = i;
    if (i >= d_in) rv[i] = T.struct_var[T.struct_ptr[t] + (i - d_in)];
  }
  if (blockIdx.x == 0) {
    int32_t off = 0;
    for (int32_t c = T.child_ptr[t]; c < T.child_ptr[t + 1]; ++c) {
      int32_t ch = T.child_idx[c];
      int32_t dout = S.d_out[ch], nel = S.nelim[ch];
      const int32_t* crv = S.rowvar + T.vec_off[ch];
      for (int32_t q = threadIdx.x; q < dout; q += blockDim.x) rv[off + q] = crv[nel + q];
      off += dout;
    }
  }
}

__global__ void lf_scatter_kernel(FrontTables T, SlotSet SS, Batch B) {
  const int32_t b = B.e0 + blockIdx.y;
  const int32_t t = B.lf[b];
  const int32_t g = entry_shift(B, b);
  const FactorSlot& S = SS.s[g];
  double* const cbpool = SS.cbpool[g];
  const double ca = S.ca, cb = S.cb;
  const int32_t d_in = S.d_in[t];
  if (d_in < 0) return;
  const FrontView v = front_view(T, S, cbpool, t, d_in);
  const int64_t e0 = T.ent_ptr[t], e1 = T.ent_ptr[t + 1];
  for (int64_t e = e0 + blockIdx.x * blockDim.x + threadIdx.x; e < e1;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int32_t r = T.ent_r[e] + d_in, c = T.ent_c[e] + d_in;
    v.L[static_cast<int64_t>(c) * v.ldL + r] = ca * T.ent_a[e] + cb * T.ent_b[e];
  }
}

// Extend-add of the s-th child of every front in the batch (one launch per child slot keeps
// the additions of different children to one parent entry in a fixed order).
__global__ void lf_extend_kernel(FrontTables T, SlotSet SS, Batch B, int32_t s) {
  const int32_t b = B.e0 + blockIdx.y;
  const int32_t t = B.lf[b];
  const int32_t g = entry_shift(B, b);
  const FactorSlot& S = SS.s[g];
  double* const cbpool = SS.cbpool[g];
  const int32_t d_in = S.d_in[t];
  if (d_in < 0) return;
  const int32_t c0 = T.child_ptr[t];
  if (s >= T.child_ptr[t + 1] - c0) return;
  int32_t off = 0;
  for (int32_t u = 0; u < s; ++u) off += S.d_out[T.child_idx[c0 + u]];
  const int32_t ch = T.child_idx[c0 + s];
  const ChildCB cv = child_cb(T, S, cbpool, ch);
  const int32_t nc = cv.size();
  const FrontView v = front_view(T, S, cbpool, t, d_in);
  for (int32_t qj = blockIdx.x; qj < nc; qj += gridDim.x) {
    const int32_t Pj = parent_pos(T, ch, qj, cv.dout, off, d_in);
    for (int32_t qi = qj + threadIdx.x; qi < nc; qi += blockDim.x) {
      const int32_t Pi = parent_pos(T, ch, qi, cv.dout, off, d_in);
      *v.at(Pi, Pj) += cv.get(qi, qj);
    }
  }
}

// ------------------------------------------------------------------------------------------
// move a failed pivot to the end: symmetric interchange of fully-summed positions a < z of the
// front (both < p, so every touched entry lives in the L storage), with its row bookkeeping
// ------------------------------------------------------------------------------------------
KEP_D void sym_swap_front(double* L, int64_t ld, int32_t m, int32_t a, int32_t z, int32_t* rv, int32_t* ap) {
  if (a == z) return;
  if (a > z) { int32_t tmp = a; a = z; z = tmp; }
  for (int32_t c = threadIdx.x; c < a; c += blockDim.x) {        // rows a and z of earlier columns
    double* col = L + static_cast<int64_t>(c) * ld;
    double x = col[a]; col[a] = col[z]; col[z] = x;
  }
  for (int32_t c = a + 1 + threadIdx.x; c < z; c += blockDim.x) { // (c, a) <-> (z, c)
    double* pa = L + static_cast<int64_t>(a) * ld + c;
    double* pz = L + static_cast<int64_t>(c) * ld + z;
    double x = *pa; *pa = *pz; *pz = x;
  }
  for (int32_t r = z + 1 + threadIdx.x; r < m; r += blockDim.x) { // (r, a) <-> (r, z)
    double* pa = L + static_cast<int64_t>(a) * ld + r;
    double* pz = L + static_cast<int64_t>(z) * ld + r;
    double x = *pa; *pa = *pz; *pz = x;
  }
  if (threadIdx.x == 0) {
    double* da = L + static_cast<int64_t>(a) * ld + a;
    double* dz = L + static_cast<int64_t>(z) * ld + z;
    double x = *da; *da = *dz; *dz = x;
    int32_t v = rv[a]; rv[a] = rv[z]; rv[z] = v;
    v = ap[a]; ap[a] = ap[z]; ap[z] = v;
  }
  __syncthreads();
}

// The previous step's bookkeeping, run by the panel kernel before its block: a front that passes
// its remaining columns to the parent finishes (its window flush has run), and a pending move of a
// failed pivot (one or two columns) to the end of the fully-summed range is carried out.
// Returns true when the front has finished.
KEP_D bool pending_swap(const FrontTables& T, const FactorSlot& S, const LargeWork& W, int32_t b, int32_t t) {
  if (W.finish[b]) {
    __syncthreads();
    if (threadIdx.x == 0) { W.done[b] = 1; W.finish[b] = 0; }
    return true;
  }
  const int32_t nf = W.swap[b];
  if (nf == 0) return false;
  const int32_t d_in = S.d_in[t];
  const int32_t m = T.m_sym[t] + d_in, p = T.p_sym[t] + d_in;
  const int32_t k = W.k[b];
  double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  int32_t* rv = S.rowvar + T.vec_off[t];
  int32_t* ap = S.apos + T.vec_off[t];
  const int32_t a0 = k + W.pi[b * kPanel];
  int32_t a1 = nf == 2 ? k + W.pi[b * kPanel + 1] : -1;
  sym_swap_front(L, ld, m, a0, p - 1, rv, ap);
  if (nf == 2) {
    if (a1 == p - 1) a1 = a0;              // the first interchange moved it
    sym_swap_front(L, ld, m, a1, p - 2, rv, ap);
  }
  __syncthreads();
  if (threadIdx.x == 0) W.swap[b] = 0;
  return false;
}

// ------------------------------------------------------------------------------------------
// pivoting panel: Bunch-Kaufman on the w x w diagonal block.  The pivot search runs in warp 0; the
// interchanges, the multipliers and the trailing update of the block use all eight warps (GB300
// issues FP64 arithmetic at a small fraction of its FP32 rate, so the update is spread over every
// scheduler of the SM: lane = row, warp = every eighth column)
// ------------------------------------------------------------------------------------------
constexpr int kPanelThreads = 256;

__global__ void __launch_bounds__(kPanelThreads) lf_panel_kernel(FrontTables T, SlotSet SS, LargeWork W,
                                                                 Batch B) {
  __shared__ double Bk[kPanel][kPanel + 1];
  __shared__ int32_t perm[kPanel];
  __shared__ double dd[kPanel], de[kPanel], lv0[kPanel], lv1[kPanel];
  __shared__ int8_t pt[kPanel];
  __shared__ int32_t s_kind, s_piv;
  const int32_t b = B.e0 + blockIdx.x;
  const int32_t tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  constexpr int32_t kWarps = kPanelThreads / 32;
  if (W.done[b]) return;
  const int32_t t = B.lf[b];
  const FactorSlot& S = SS.s[entry_shift(B, b)];
  if (pending_swap(T, S, W, b, t)) return;
  const int32_t d_in = S.d_in[t];
  const int32_t p = T.p_sym[t] + d_in;
  const int32_t k = W.k[b] + W.q[b];
  int32_t we = W.we[b];
  const bool open = k < p && (k >= we || W.reset[b]);
  if (open) we = min(k + kWindow, p);   // open a new pivot window
  __syncthreads();
  if (tid == 0) {
    W.k[b] = k; W.q[b] = 0; W.flush[b] = 0;
    if (open) { W.ws[b] = k; W.we[b] = we; W.reset[b] = 0; }
  }
  if (k >= p) {
    if (tid == 0) { W.done[b] = 1; S.nelim[t] = k; S.d_out[t] = p - k; W.w[b] = 0; }
    return;
  }
  const int32_t w = min(kPanel, we - k);
  const double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  // the block's lower triangle, mirrored into a full symmetric copy: lane = row, warp = every
  // eighth column (each column one coalesced load)
  for (int32_t c = warp; c < w; c += kWarps) {
    if (lane >= c && lane < w) {
      const double val = L[static_cast<int64_t>(k + c) * ld + k + lane];
      Bk[lane][c] = val;
      Bk[c][lane] = val;
    }
  }
  if (tid < kPanel) perm[tid] = tid;
  __syncthreads();
  int32_t kk = 0;
  while (kk < w) {
    // Bunch-Kaufman choice for column kk (warp 0; every other thread reads the result)
    if (warp == 0) {
      double v = (lane > kk && lane < w) ? fabs(Bk[lane][kk]) : -1.0;
      double lam = warp_max(v);
      const unsigned ball = __ballot_sync(0xffffffffu, v == lam && lane > kk && lane < w);
      const int32_t r = ball ? __ffs(ball) - 1 : -1;
      if (lam < 0) lam = 0.0;
      const double akk = fabs(Bk[kk][kk]);
      int32_t kind = 1, piv = kk;          // kind 1: 1x1 at piv; kind 2: 2x2 (kk, piv)
      if (!(lam == 0.0 || akk >= kBKAlpha * lam) && r >= 0) {   // (r < 0 only for NaN entries)
        double vr = (lane >= kk && lane < w && lane != r) ? fabs(Bk[lane][r]) : -1.0;
        double sig = warp_max(vr);
        if (sig < 0) sig = 0.0;
        if (akk * sig >= kBKAlpha * lam * lam) { kind = 1; piv = kk; }
        else if (fabs(Bk[r][r]) >= kBKAlpha * sig) { kind = 1; piv = r; }
        else { kind = 2; piv = r; }
      }
      if (lane == 0) { s_kind = kind; s_piv = piv; }
    }
    __syncthreads();
    const int32_t kind = s_kind, piv = s_piv;
    const int32_t dst = kind == 1 ? kk : kk + 1;
    if (piv != dst) {   // symmetric interchange of dst and piv in the full block copy
      if (tid < w) { const double tmp = Bk[tid][dst]; Bk[tid][dst] = Bk[tid][piv]; Bk[tid][piv] = tmp; }
      __syncthreads();
      if (tid < w) { const double tmp = Bk[dst][tid]; Bk[dst][tid] = Bk[piv][tid]; Bk[piv][tid] = tmp; }
      if (tid == 0) { const int32_t tp = perm[dst]; perm[dst] = perm[piv]; perm[piv] = tp; }
      __syncthreads();
    }
    const int32_t c0 = kk + kind;         // first column of the trailing block
    if (kind == 1) {
      const double d = Bk[kk][kk];
      if (tid >= c0 && tid < w) lv0[tid] = d != 0.0 ? Bk[tid][kk] / d : 0.0;
    } else {
      const double a = Bk[kk][kk], bb = Bk[kk + 1][kk], c2 = Bk[kk + 1][kk + 1];
      const double det = a * c2 - bb * bb;
      if (tid >= c0 && tid < w) {
        const double w0 = Bk[tid][kk], w1 = Bk[tid][kk + 1];
        lv0[tid] = (c2 * w0 - bb * w1) / det;
        lv1[tid] = (a * w1 - bb * w0) / det;
      }
    }
    __syncthreads();
    // trailing update of the block, rows and columns [c0, w)
    if (lane >= c0 && lane < w) {
      if (kind == 1) {
        const double l0 = lv0[lane];
        for (int32_t c = c0 + warp; c < w; c += kWarps) Bk[lane][c] -= l0 * Bk[c][kk];
      } else {
        const double l0 = lv0[lane], l1 = lv1[lane];
        for (int32_t c = c0 + warp; c < w; c += kWarps) Bk[lane][c] -= l0 * Bk[c][kk] + l1 * Bk[c][kk + 1];
      }
    }
    __syncthreads();
    if (kind == 1) {
      if (tid >= c0 && tid < w) { Bk[tid][kk] = lv0[tid]; Bk[kk][tid] = lv0[tid]; }
      if (tid == 0) { dd[kk] = Bk[kk][kk]; de[kk] = 0.0; pt[kk] = 1; }
    } else {
      if (tid >= c0 && tid < w) {
        Bk[tid][kk] = lv0[tid]; Bk[kk][tid] = lv0[tid];
        Bk[tid][kk + 1] = lv1[tid]; Bk[kk + 1][tid] = lv1[tid];
      }
      if (tid == 0) {
        dd[kk] = Bk[kk][kk]; dd[kk + 1] = Bk[kk + 1][kk + 1]; de[kk] = Bk[kk + 1][kk]; de[kk + 1] = 0.0;
        pt[kk] = 2; pt[kk + 1] = 0;
      }
    }
    __syncthreads();
    kk += kind;
  }
  double* L11 = W.L11 + static_cast<int64_t>(b) * kPanel * kPanel;
  for (int32_t e = tid; e < w * kPanel; e += kPanelThreads) {
    const int32_t c = e / kPanel, r = e % kPanel;
    if (r < w) {
      const double val = (r > c) ? ((pt[c] == 2 && r == c + 1) ? 0.0 : Bk[r][c]) : (r == c ? 1.0 : 0.0);
      L11[c * kPanel + r] = val;
    }
  }
  if (tid < w) {
    W.Dblk[b * 2 * kPanel + tid] = dd[tid];
    W.Dblk[b * 2 * kPanel + kPanel + tid] = de[tid];
    W.pt[b * kPanel + tid] = pt[tid];
    W.pi[b * kPanel + tid] = perm[tid];
    W.colmax[b * kPanel + tid] = 0ull;
  }
  if (tid == 0) W.w[b] = w;
}

// ------------------------------------------------------------------------------------------
// L21 rows and column maxima: row i solves y L11^T = f (f: row i of the permuted block columns),
// then l = y D^{-1}
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kRowTile) lf_l21_kernel(FrontTables T, SlotSet SS, LargeWork W,
                                                          Batch B) {
  __shared__ double L11s[kPanel][kPanel + 1];
  __shared__ double dd[kPanel], r0[kPanel], r1[kPanel], r2[kPanel];
  __shared__ int8_t pt[kPanel];
  __shared__ int32_t pi[kPanel];
  __shared__ double red[kRowTile / 32][kPanel];
  const int32_t b = B.e0 + blockIdx.y;
  if (W.done[b]) return;
  const int32_t t = B.lf[b];
  const int32_t g = entry_shift(B, b);
  const FactorSlot& S = SS.s[g];
  const int32_t d_in = S.d_in[t];
  const int32_t m = T.m_sym[t] + d_in;
  const int32_t k = W.k[b], w = W.w[b];
  const int32_t rows = m - k - w;
  const int32_t ntile = (rows + kRowTile - 1) / kRowTile;
  if (blockIdx.x >= ntile) return;
  const double* L11 = W.L11 + static_cast<int64_t>(b) * kPanel * kPanel;
  for (int32_t e = threadIdx.x; e < kPanel * kPanel; e += blockDim.x)
    L11s[e % kPanel][e / kPanel] = L11[e];
  if (threadIdx.x < kPanel) {
    // D^{-1} of the block once per CTA: 1/d for a 1x1 pivot, the three entries of the inverse
    // [c2 -b; -b a] / det for a 2x2 pivot (kept at its first index)
    const int32_t c = threadIdx.x;
    const double d0 = W.Dblk[b * 2 * kPanel + c];
    dd[c] = d0;
    pt[c] = W.pt[b * kPanel + c];
    pi[c] = W.pi[b * kPanel + c];
    r0[c] = r1[c] = r2[c] = 0.0;
    if (pt[c] == 1) {
      r0[c] = d0 != 0.0 ? 1.0 / d0 : 0.0;
    } else if (pt[c] == 2 && c + 1 < kPanel) {
      const double a = d0, c2 = W.Dblk[b * 2 * kPanel + c + 1], bb = W.Dblk[b * 2 * kPanel + kPanel + c];
      const double inv = 1.0 / (a * c2 - bb * bb);
      r0[c] = c2 * inv;
      r1[c] = -bb * inv;
      r2[c] = a * inv;
    }
  }
  __syncthreads();
  const double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  double* P21 = SS.P21[g] + W.p21_off[t];
  const int64_t ldp = T.m_alloc[t];
  double cm[kPanel];
#pragma unroll
  for (int32_t c = 0; c < kPanel; ++c) cm[c] = 0.0;
  for (int32_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int32_t ii = tile * kRowTile + threadIdx.x;     // row index below the block
    const bool valid = ii < rows;
    const int32_t i = k + w + ii;
    double f[kPanel];
#pragma unroll
    for (int32_t c = 0; c < kPanel; ++c)
      f[c] = (valid && c < w) ? L[static_cast<int64_t>(k + pi[c]) * ld + i] : 0.0;
    // forward substitution with the unit lower L11 (y L11^T = f)
#pragma unroll
    for (int32_t c = 0; c < kPanel; ++c) {
#pragma unroll
      for (int32_t a = c + 1; a < kPanel; ++a) f[a] -= f[c] * L11s[a][c];
    }
    // l = y D^{-1}
#pragma unroll
    for (int32_t c = 0; c < kPanel; ++c) {
      if (c < w) {
        if (pt[c] == 1) {
          f[c] = dd[c] != 0.0 ? f[c] * r0[c] : (f[c] == 0.0 ? 0.0 : INFINITY);
        } else if (pt[c] == 2 && c + 1 < kPanel) {
          const double y0 = f[c], y1 = f[c + 1];
          f[c] = fma(y0, r0[c], y1 * r1[c]);
          f[c + 1] = fma(y1, r2[c], y0 * r1[c]);
        }
      }
    }
    if (valid) {
#pragma unroll
      for (int32_t c = 0; c < kPanel; ++c)
        if (c < w) {
          P21[ii + c * ldp] = f[c];
          double af = fabs(f[c]);
          if (!(af <= cm[c])) cm[c] = af;   // NaN propagates as "larger"
        }
    }
  }
  // reduce column maxima over the CTA, then atomically into the batch entry
  const int32_t warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
  for (int32_t c = 0; c < kPanel; ++c) {
    double v = cm[c];
    for (int o = 16; o > 0; o >>= 1) {
      double u = __shfl_xor_sync(0xffffffffu, v, o);
      if (!(u <= v)) v = u;
    }
    if (lane == 0) red[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < w) {
    double v = 0.0;
    for (int32_t q = 0; q < kRowTile / 32; ++q) {
      double u = red[q][threadIdx.x];
      if (!(u <= v)) v = u;
    }
    if (v != v) v = INFINITY;
    atomicMax(&W.colmax[b * kPanel + threadIdx.x], static_cast<unsigned long long>(__double_as_longlong(v)));
  }
}

// Number of leading pivots of the block whose L columns pass |l| <= 1/u.
KEP_D int32_t accepted_count(const LargeWork& W, int32_t b, int32_t w) {
  const double lim = 1.0 / kThresholdU;
  int32_t c = 0, q = 0;
  while (c < w) {
    const int8_t pt = W.pt[b * kPanel + c];
    const double m0 = __longlong_as_double(static_cast<long long>(W.colmax[b * kPanel + c]));
    if (pt == 2) {
      const double m1 = __longlong_as_double(static_cast<long long>(W.colmax[b * kPanel + c + 1]));
      if (m0 <= lim && m1 <= lim) { c += 2; q = c; } else break;
    } else {
      if (m0 <= lim) { c += 1; q = c; } else break;
    }
  }
  return q;
}

// ------------------------------------------------------------------------------------------
// apply: permute the block, write accepted L columns and D, restore rejected columns
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) lf_apply_kernel(FrontTables T, SlotSet SS, LargeWork W,
                                                       Batch B) {
  __shared__ double Bo[kPanel][kPanel + 1];
  __shared__ double Fo[kPanel][kRowTile + 1];
  __shared__ int32_t pi[kPanel];
  __shared__ int32_t rvo[kPanel], apo[kPanel];
  const int32_t b = B.e0 + blockIdx.y;
  if (W.done[b]) return;
  const int32_t t = B.lf[b];
  const int32_t g = entry_shift(B, b);
  const FactorSlot& S = SS.s[g];
  const int32_t d_in = S.d_in[t];
  const int32_t m = T.m_sym[t] + d_in, p = T.p_sym[t] + d_in;
  const int32_t k = W.k[b], w = W.w[b];
  int32_t q = accepted_count(W, b, w);
  if (q == 0 && T.parent[t] < 0) {
    // a root has no parent to pass columns to: take the block's Bunch-Kaufman pivots as they are
    q = w;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&S.status[0], ST_ROOT_FORCED);
  }
  if (q == 0) {
    // the block's first pivot fails the threshold: move that pivot's column(s) to the end of the
    // fully-summed range and retry with the others; once every remaining column has failed in
    // turn without progress, the remaining columns go to the parent (delayed pivots)
    // (the window's accepted pivots are first applied to everything right of the window, so the
    // column swapped in from the end of the range is up to date)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const int32_t nf = W.pt[b * kPanel] == 2 ? 2 : 1;
      const int32_t f = W.fails[b] + 1;
      W.fails[b] = f;
      W.kend[b] = k;
      W.flush[b] = k > W.ws[b] ? 1 : 0;
      W.reset[b] = 1;
      if (f > p - k || p - k <= nf) {
        W.finish[b] = 1;
        S.nelim[t] = k;
        S.d_out[t] = p - k;
        W.swap[b] = 0;
      } else {
        W.swap[b] = nf;
      }
    }
    return;
  }
  if (threadIdx.x < kPanel) pi[threadIdx.x] = W.pi[b * kPanel + threadIdx.x];
  __syncthreads();
  double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  const int32_t nA = (k + 31) / 32;
  const int32_t rows = m - k - w;
  const int32_t nB = (rows + kRowTile - 1) / kRowTile;
  const double* L11 = W.L11 + static_cast<int64_t>(b) * kPanel * kPanel;
  const double* P21 = SS.P21[g] + W.p21_off[t];
  const int64_t ldp = T.m_alloc[t];
  for (int32_t item = blockIdx.x; item < 1 + nA + nB; item += gridDim.x) {
    if (item == 0) {
      // the diagonal block
      for (int32_t e = threadIdx.x; e < w * w; e += blockDim.x) {
        int32_t a = e % w, c = e / w;
        if (a >= c) {
          double val = L[static_cast<int64_t>(k + c) * ld + k + a];
          Bo[a][c] = val; Bo[c][a] = val;
        }
      }
      int32_t* rv = S.rowvar + T.vec_off[t];
      int32_t* ap = S.apos + T.vec_off[t];
      if (threadIdx.x < w) { rvo[threadIdx.x] = rv[k + threadIdx.x]; apo[threadIdx.x] = ap[k + threadIdx.x]; }
      __syncthreads();
      for (int32_t e = threadIdx.x; e < w * w; e += blockDim.x) {
        int32_t a = e % w, c = e / w;
        if (a < c) continue;
        double val;
        if (c < q) {
          const int8_t ptc = W.pt[b * kPanel + c];
          if (a == c) val = W.Dblk[b * 2 * kPanel + c];
          else if (ptc == 2 && a == c + 1) val = W.Dblk[b * 2 * kPanel + kPanel + c];
          else val = L11[c * kPanel + a];
        } else {
          val = Bo[pi[a]][pi[c]];
        }
        L[static_cast<int64_t>(k + c) * ld + k + a] = val;
      }
      if (threadIdx.x < w) { rv[k + threadIdx.x] = rvo[pi[threadIdx.x]]; ap[k + threadIdx.x] = apo[pi[threadIdx.x]]; }
      const int64_t po = T.piv_off[t];
      if (threadIdx.x < q) {
        S.Dd[po + k + threadIdx.x] = W.Dblk[b * 2 * kPanel + threadIdx.x];
        S.De[po + k + threadIdx.x] = W.Dblk[b * 2 * kPanel + kPanel + threadIdx.x];
        S.piv[po + k + threadIdx.x] = W.pt[b * kPanel + threadIdx.x];
      }
      if (threadIdx.x == 0) {
        int32_t neg = 0, zero = 0, pos = 0;
        bool finite = true;
        for (int32_t c = 0; c < q;) {
          const double a = W.Dblk[b * 2 * kPanel + c];
          if (W.pt[b * kPanel + c] == 2) {
            const double c2 = W.Dblk[b * 2 * kPanel + c + 1], bb = W.Dblk[b * 2 * kPanel + kPanel + c];
            finite = finite && isfinite(a) && isfinite(c2) && isfinite(bb);
            count_pivot2(a, bb, c2, neg, zero, pos);
            c += 2;
          } else {
            finite = finite && isfinite(a);
            count_pivot1(a, neg, zero, pos);
            c += 1;
          }
        }
        S.cnt[3 * t] += neg; S.cnt[3 * t + 1] += zero; S.cnt[3 * t + 2] += pos;
        if (!finite) { atomicOr(&S.status[0], ST_NONFINITE); atomicCAS(&S.status[1], -1, t); }
        W.q[b] = q;
        W.fails[b] = 0;
        if (k + q >= W.we[b]) { W.kend[b] = k + q; W.flush[b] = 1; }   // window complete
      }
      __syncthreads();
    } else if (item <= nA) {
      // rows k .. k+w of the earlier L columns follow the block permutation
      const int32_t warp = threadIdx.x / 32, lane = threadIdx.x % 32;
      const int32_t j0 = (item - 1) * 32;
      for (int32_t j = j0 + warp; j < min(k, j0 + 32); j += blockDim.x / 32) {
        double* col = L + static_cast<int64_t>(j) * ld + k;
        double val = lane < w ? col[pi[lane]] : 0.0;
        __syncwarp();
        if (lane < w) col[lane] = val;
      }
    } else {
      // rows below the block: accepted columns take L21, rejected ones their permuted originals
      const int32_t ii = (item - 1 - nA) * kRowTile + (threadIdx.x % kRowTile);
      const int32_t half = threadIdx.x / kRowTile;        // two threads per row: column halves
      const bool active = ii < rows;
      const int64_t i = k + w + ii;
      for (int32_t c = half; c < w; c += 2)
        if (active) Fo[c][threadIdx.x % kRowTile] = L[static_cast<int64_t>(k + c) * ld + i];
      __syncthreads();
      for (int32_t c = half; c < w; c += 2)
        if (active)
          L[static_cast<int64_t>(k + c) * ld + i] =
              c < q ? P21[ii + c * ldp] : Fo[pi[c]][threadIdx.x % kRowTile];
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------------------------------
// Schur update of the trailing matrix: C(i, j) -= sum_c L(i, c) (L D)(j, c) over the q accepted
// pivots, for s = k + q <= j <= i < m.  64 x 64 tiles, 256 threads with 4 x 4 register tiles.
// ------------------------------------------------------------------------------------------
// Block partition of a trailing region that starts at s: blocks of TS rows/columns, split at p
// (the boundary between L storage and the contribution block), up to m.
template <int TS>
struct Part {
  int32_t s, p, m, nL, base2, nR;
  KEP_D void init(int32_t s_, int32_t p_, int32_t m_) {
    s = s_; p = p_; m = m_;
    nL = s < p ? (p - s + TS - 1) / TS : 0;
    base2 = s > p ? s : p;
    nR = nL + (m > base2 ? (m - base2 + TS - 1) / TS : 0);
  }
  KEP_D int32_t lo(int32_t b) const { return b < nL ? s + b * TS : base2 + (b - nL) * TS; }
  KEP_D int32_t hi(int32_t b) const {
    return b < nL ? min(s + (b + 1) * TS, p) : min(base2 + (b - nL + 1) * TS, m);
  }
};

// Schur update C(i, j) -= sum_{c in [c0, c1)} L(i, c) (L D)(j, c) for s <= j < ce, j <= i < m.
//  WINDOW = true : the rank-q update of the current pivot window's own columns (c0 = k,
//                  c1 = k + q, s = k + q, ce = window end);
//  WINDOW = false: the deferred update of everything right of the window with all pivots the
//                  window accepted (c0 = window start, c1 = its last accepted pivot + 1,
//                  s = ce' = window end, ce = m), issued once per window ("flush").
// TS x TS tiles (TS = 32 or 64, the context's choice), 256 threads with (TS/16) x (TS/16) register
// tiles, the pivot range in chunks of 32.
// R: arithmetic of the tiles (double, or float for the reduced-precision factorization mode)
template <bool WINDOW, typename R, int TS>
__global__ void __launch_bounds__(256) lf_schur_kernel(FrontTables T, SlotSet SS, LargeWork W, Batch B,
                                                       unsigned long long* flops) {
  constexpr int RT = TS / 16;
  __shared__ R Ai[kPanel][TS + 1];
  __shared__ R Wj[kPanel][TS + 1];
  const int32_t b = B.e0 + blockIdx.y;
  int32_t c0, c1, s, ce;
  if (WINDOW) {
    if (W.done[b]) return;
    const int32_t q = W.q[b];
    if (q == 0) return;
    c0 = W.k[b]; c1 = c0 + q; s = c1; ce = W.we[b];
  } else {
    if (W.done[b] || !W.flush[b]) return;
    c0 = W.ws[b]; c1 = W.kend[b]; s = W.we[b];
  }
  const int32_t t = B.lf[b];
  const int32_t g = entry_shift(B, b);
  const FactorSlot& S = SS.s[g];
  const int32_t d_in = S.d_in[t];
  const FrontView v = front_view(T, S, SS.cbpool[g], t, d_in);
  if (!WINDOW) ce = v.m;
  if (c1 <= c0 || s >= ce) return;
  Part<TS> P;
  P.init(s, v.p, v.m);
  int32_t nJ = 0;
  while (nJ < P.nR && P.lo(nJ) < ce) ++nJ;
  // tiles (bi, bj), bj < nJ, bi >= bj; tiles of column block bj start at bj*nR - bj*(bj-1)/2
  const int64_t ntiles = static_cast<int64_t>(nJ) * P.nR - static_cast<int64_t>(nJ) * (nJ - 1) / 2;
  if (blockIdx.x >= ntiles) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {   // algorithmic flops: 2 * rank per updated entry
    const int64_t w = ce - s, h = v.m - s;
    atomicAdd(flops, static_cast<unsigned long long>(2 * static_cast<int64_t>(c1 - c0) * (w * h - w * (w - 1) / 2)));
  }
  const int64_t po = T.piv_off[t];
  const double* Dd = S.Dd + po;
  const double* De = S.De + po;
  const int8_t* pv = S.piv + po;
  const double* Lb = v.L;
  const int64_t ld = v.ldL;
  const int32_t tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int32_t lo = 0, hi = nJ - 1;            // largest bj with start(bj) <= tile
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) / 2;
      const int64_t st = static_cast<int64_t>(mid) * P.nR - static_cast<int64_t>(mid) * (mid - 1) / 2;
      if (st <= tile) lo = mid; else hi = mid - 1;
    }
    const int32_t bj = lo;
    const int64_t stj = static_cast<int64_t>(bj) * P.nR - static_cast<int64_t>(bj) * (bj - 1) / 2;
    const int32_t bi = bj + static_cast<int32_t>(tile - stj);
    const int32_t I0 = P.lo(bi), I1 = P.hi(bi);
    const int32_t J0 = P.lo(bj), J1 = min(P.hi(bj), ce);
    R acc[RT][RT];
#pragma unroll
    for (int32_t x = 0; x < RT; ++x)
#pragma unroll
      for (int32_t y = 0; y < RT; ++y) acc[x][y] = R(0);
    for (int32_t k0 = c0; k0 < c1; k0 += kPanel) {
      const int32_t kn = min(kPanel, c1 - k0);
      __syncthreads();
      // A_I = L(I, chunk) and W_J = L(J, chunk) D (a 2x2 block mixes its two columns)
      for (int32_t e = threadIdx.x; e < kPanel * TS; e += blockDim.x) {
        const int32_t r = e % TS, cc = e / TS;
        double ai = 0.0, wj = 0.0;
        if (cc < kn) {
          const int32_t c = k0 + cc;
          if (I0 + r < I1) ai = Lb[static_cast<int64_t>(c) * ld + I0 + r];
          if (J0 + r < J1) {
            const double x = Lb[static_cast<int64_t>(c) * ld + J0 + r];
            const int8_t ptc = pv[c];
            if (ptc == 1) {
              wj = x * Dd[c];
            } else if (ptc == 2) {
              const double y = Lb[static_cast<int64_t>(c + 1) * ld + J0 + r];
              wj = x * Dd[c] + y * De[c];
            } else {
              const double y = Lb[static_cast<int64_t>(c - 1) * ld + J0 + r];
              wj = y * De[c - 1] + x * Dd[c];
            }
          }
        }
        Ai[cc][r] = static_cast<R>(ai);
        Wj[cc][r] = static_cast<R>(wj);
      }
      __syncthreads();
      for (int32_t cc = 0; cc < kn; ++cc) {
        R a[RT], wv[RT];
#pragma unroll
        for (int32_t x = 0; x < RT; ++x) a[x] = Ai[cc][ty + 16 * x];
#pragma unroll
        for (int32_t y = 0; y < RT; ++y) wv[y] = Wj[cc][tx + 16 * y];
#pragma unroll
        for (int32_t x = 0; x < RT; ++x)
#pragma unroll
          for (int32_t y = 0; y < RT; ++y) acc[x][y] = fma(a[x], wv[y], acc[x][y]);
      }
    }
#pragma unroll
    for (int32_t y = 0; y < RT; ++y) {
      const int32_t j = J0 + tx + 16 * y;
      if (j >= J1) continue;
#pragma unroll
      for (int32_t x = 0; x < RT; ++x) {
        const int32_t i = I0 + ty + 16 * x;
        if (i < I1 && i >= j) *v.at(i, j) -= static_cast<double>(acc[x][y]);
      }
    }
  }
}

__global__ void reduce_inertia_kernel(SlotSet SS, int32_t nfronts, long long* out) {
  const FactorSlot& S = SS.s[blockIdx.x];
  out += 6 * blockIdx.x;
  // out: neg, zero, pos, delayed (sum of d_out over roots is 0; delayed = sum of all d_out)
  long long a = 0, z = 0, c = 0, d = 0;
  for (int32_t t = threadIdx.x; t < nfronts; t += blockDim.x) {
    a += S.cnt[3 * t]; z += S.cnt[3 * t + 1]; c += S.cnt[3 * t + 2]; d += S.d_out[t];
  }
  __shared__ long long red[4][32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o); z += __shfl_xor_sync(0xffffffffu, z, o);
    c += __shfl_xor_sync(0xffffffffu, c, o); d += __shfl_xor_sync(0xffffffffu, d, o);
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) { red[0][warp] = a; red[1][warp] = z; red[2][warp] = c; red[3][warp] = d; }
  __syncthreads();
  if (threadIdx.x < 4) {
    long long s = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[threadIdx.x][w];
    out[threadIdx.x] = s;
  }
  if (threadIdx.x == 0) { out[4] = S.status[0]; out[5] = S.status[1]; }
}

}  // namespace

// ------------------------------------------------------------------------------------------
// host orchestration
// ------------------------------------------------------------------------------------------


static int grid_cap(int64_t want, int64_t cap) {
  if (want < 1) want = 1;
  return static_cast<int>(want < cap ? want : cap);
}

kep_status run_factor(FactorLaunch& F, const double* ca, const double* cb, kep_inertia* out, int* status_bits) {
  const Plan& P = *F.plan;
  cudaStream_t st = F.stream;
  const int G = F.G;
  if (F.emul_min > 0) emul_init();
  for (int g = 0; g < G; ++g) {
    const int32_t init_status[2] = {0, -1};
    if (cudaMemcpyAsync(F.SS.s[g].status, init_status, sizeof(init_status), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return KEP_ERR_CUDA;
    F.SS.s[g].ca = ca[g];
    F.SS.s[g].cb = cb[g];
  }
  const int target = F.num_sms * 8;
  for (int32_t l = 0; l < P.nlevels; ++l) {
    // the level's entries: its fronts in decreasing order, each G times (one per shift)
    const int32_t lb = P.level_ptr[l] * G;
    const int32_t width = (P.level_ptr[l + 1] - P.level_ptr[l]) * G;
    const int32_t* lfh = F.h_ent_front + lb;
    // batches: the tensor-core fronts in groups, each front of a large order alone (with its
    // shifts), the rest together (chunks of 65535)
    int32_t e = 0;
    while (e < width) {
      const int32_t t0 = lfh[e];
      int32_t e1;
      const bool emul = F.emul_min > 0 && P.m_alloc[t0] >= F.emul_min;
      if (emul) {
        e1 = F.h_emul_end[lb + e];   // the level's entries on the tensor-core path, batched
      } else if (P.m_alloc[t0] > 4096) {
        e1 = std::min(e + G, width);
      } else {
        e1 = e + 1;                  // the rest of the level (sorted by size), stopping at an
        while (e1 < width && e1 - e < 65535 &&   // entry that must go alone
               !(F.emul_min > 0 && P.m_alloc[lfh[e1]] >= F.emul_min))
          ++e1;
      }
      const int32_t nb = e1 - e;
      Batch B{F.d_ent_front + lb, F.d_ent_shift ? F.d_ent_shift + lb : nullptr, e};
      int64_t max_m = 0, max_p = 0, max_c = 0, max_ent = 0;
      int32_t maxch = 0;
      for (int32_t i = e; i < e1; ++i) {
        const int32_t t = lfh[i];
        max_m = std::max<int64_t>(max_m, P.m_alloc[t]);
        max_p = std::max<int64_t>(max_p, P.p_alloc[t]);
        max_c = std::max<int64_t>(max_c, P.m_sym[t] - P.p_sym[t]);
        max_ent = std::max<int64_t>(max_ent, P.ent_ptr[t + 1] - P.ent_ptr[t]);
        maxch = std::max(maxch, P.child_ptr[t + 1] - P.child_ptr[t]);
      }
      const int gx_cols = grid_cap(std::max(max_p, max_c), std::max<int64_t>(1, (target + nb - 1) / nb));
      KEP_LAUNCH(F.timer, KC_ASSEMBLE, st, lf_init_kernel<<<dim3(gx_cols, nb), 256, 0, st>>>(F.T, F.SS, F.W, B));
      KEP_LAUNCH(F.timer, KC_ASSEMBLE, st,
                 lf_scatter_kernel<<<dim3(grid_cap((max_ent + 255) / 256, std::max<int64_t>(1, (target + nb - 1) / nb)), nb), 256, 0, st>>>(
                     F.T, F.SS, B));
      for (int32_t s = 0; s < maxch; ++s)
        KEP_LAUNCH(F.timer, KC_ASSEMBLE, st,
                   lf_extend_kernel<<<dim3(grid_cap(max_m, std::max<int64_t>(1, (target + nb - 1) / nb)), nb), 128, 0, st>>>(
                       F.T, F.SS, B, s));
      const int64_t rowtiles = (max_m + kRowTile - 1) / kRowTile;
      // CTAs per front: enough for the largest front of the batch (fronts of one level differ in
      // size by up to ~10x; CTAs beyond a front's own work return at once)
      const int64_t per_front = std::max<int64_t>((target + nb - 1) / nb, F.num_sms);
      const int gx_rows = grid_cap(rowtiles, per_front);
      const int gx_apply = grid_cap(rowtiles + max_p / 32 + 2, per_front);
      const int TS = F.schur_tile == 32 ? 32 : kTile;
      const int64_t tb = (max_m + TS - 1) / TS + 1;
      const int64_t per_front_upd = std::max<int64_t>((F.num_sms * 4 + nb - 1) / nb, 2 * F.num_sms);
      const int gx_upd = grid_cap(tb * (tb + 1) / 2, per_front_upd);
      const int gx_win = grid_cap(tb * (kWindow / TS + 1), per_front_upd);
      int64_t steps = (max_p + kPanel - 1) / kPanel + 1;
      // a guard, not a tuning knob: every step eliminates or moves on from a block, and a column
      // that fails the threshold is retried at most once per pass over the remaining columns
      // before it is delayed, so a level takes at most about (blocks)^2 steps
      const int64_t blocks = (max_p + kPanel - 1) / kPanel + 2;
      const int64_t step_cap = 64 + 2 * blocks * blocks;
      int64_t steps_done = 0;
      // one pass: `steps` pivot steps (panel, L21 rows, apply, in-window and trailing updates),
      // then one more panel call that finalises fronts whose last block was accepted
      auto issue_pass = [&](cudaStream_t sx, int64_t nsteps) {
        for (int64_t it = 0; it < nsteps; ++it) {
          KEP_LAUNCH(F.timer, KC_PANEL, sx, lf_panel_kernel<<<nb, kPanelThreads, 0, sx>>>(F.T, F.SS, F.W, B));
          KEP_LAUNCH(F.timer, KC_L21, sx, lf_l21_kernel<<<dim3(gx_rows, nb), kRowTile, 0, sx>>>(F.T, F.SS, F.W, B));
          KEP_LAUNCH(F.timer, KC_APPLY, sx, lf_apply_kernel<<<dim3(gx_apply, nb), 128, 0, sx>>>(F.T, F.SS, F.W, B));
          if (emul) {
            // in-window and trailing updates on the tensor cores (FP64-accurate splitting)
            launch_emul_update(true, F.fp32_schur, F.T, F.SS, F.W, B, nb, F.emul_ws, F.d_emul_off + lb + e, max_m, sx,
                               F.num_sms, F.timer, F.flops);
            launch_emul_update(false, F.fp32_schur, F.T, F.SS, F.W, B, nb, F.emul_ws, F.d_emul_off + lb + e, max_m, sx,
                               F.num_sms, F.timer, F.flops);
          } else {
            // FP64 (or, for the reduced-precision factor, FP32) tiles of the context's edge
            auto upd = [&](auto win, auto real, auto edge) {
              constexpr bool W_ = decltype(win)::value;
              using R_ = typename decltype(real)::type;
              constexpr int T_ = decltype(edge)::value;
              KEP_LAUNCH(F.timer, KC_UPDATE, sx,
                         (lf_schur_kernel<W_, R_, T_><<<dim3(W_ ? gx_win : gx_upd, nb), 256, 0, sx>>>(
                             F.T, F.SS, F.W, B, F.flops + KC_UPDATE)));
            };
            auto both = [&](auto real, auto edge) {
              upd(std::true_type{}, real, edge);
              upd(std::false_type{}, real, edge);
            };
            using E32 = std::integral_constant<int, 32>;
            using E64 = std::integral_constant<int, kTile>;
            if (F.fp32_schur) {
              if (TS == 32) both(TypeTag<float>{}, E32{}); else both(TypeTag<float>{}, E64{});
            } else {
              if (TS == 32) both(TypeTag<double>{}, E32{}); else both(TypeTag<double>{}, E64{});
            }
          }
        }
        KEP_LAUNCH(F.timer, KC_PANEL, sx, lf_panel_kernel<<<nb, kPanelThreads, 0, sx>>>(F.T, F.SS, F.W, B));
      };
      while (true) {
        if (steps_done > step_cap) return KEP_ERR_NOT_CONVERGED;
        steps_done += steps;
        if (F.graphs && F.graphs->enabled && F.capture_stream && !F.timer->enabled) {
          // the pass as a CUDA graph: captured once per batch, pass length and storage, replayed
          const std::vector<uint64_t> key = {
              static_cast<uint64_t>(l), static_cast<uint64_t>(e), static_cast<uint64_t>(nb),
              static_cast<uint64_t>(steps), static_cast<uint64_t>(G), static_cast<uint64_t>(F.emul_min),
              static_cast<uint64_t>(TS),
              (emul ? 1ull : 0ull) | (F.fp32_schur ? 2ull : 0ull),
              reinterpret_cast<uint64_t>(F.SS.s[0].F), reinterpret_cast<uint64_t>(F.SS.s[G - 1].F),
              reinterpret_cast<uint64_t>(F.W.done), reinterpret_cast<uint64_t>(F.emul_ws),
              reinterpret_cast<uint64_t>(F.d_emul_off), reinterpret_cast<uint64_t>(F.SS.P21[0])};
          GraphEntry* ge = F.graphs->find(key);
          if (!ge) {
            GraphEntry ne;
            int64_t before[KC_COUNT];
            for (int c = 0; c < KC_COUNT; ++c) before[c] = F.timer->launches[c];
            // captured on the context's own capture stream (the legacy default stream, which a
            // caller may use, cannot be captured); the graph is then launched on st
            cudaStream_t cs = F.capture_stream;
            if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return KEP_ERR_CUDA;
            issue_pass(cs, steps);
            cudaGraph_t graph = nullptr;
            if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) return KEP_ERR_CUDA;
            const cudaError_t ie = cudaGraphInstantiate(&ne.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) return KEP_ERR_CUDA;
            for (int c = 0; c < KC_COUNT; ++c) {
              ne.launches[c] = F.timer->launches[c] - before[c];
              F.timer->launches[c] = before[c];
            }
            F.graphs->entries.emplace_back(key, ne);
            ge = &F.graphs->entries.back().second;
          }
          if (cudaGraphLaunch(ge->exec, st) != cudaSuccess) return KEP_ERR_CUDA;
          for (int c = 0; c < KC_COUNT; ++c) F.timer->launches[c] += ge->launches[c];
        } else {
          issue_pass(st, steps);
        }
        if (cudaMemcpyAsync(F.h_done, F.W.done + e, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, st) != cudaSuccess)
          return KEP_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return KEP_ERR_CUDA;
        F.timer->collect();
        bool all = true;
        for (int32_t i = 0; i < nb; ++i) all = all && F.h_done[i];
        if (all) break;
        steps = 8;   // partially accepted blocks need extra steps
      }
      e = e1;
    }
  }
  KEP_LAUNCH(F.timer, KC_REDUCE, st, reduce_inertia_kernel<<<G, 1024, 0, st>>>(F.SS, P.nfronts, F.d_red));
  if (cudaMemcpyAsync(F.h_red, F.d_red, 6 * G * sizeof(long long), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return KEP_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return KEP_ERR_CUDA;
  F.timer->collect();
  if (cudaGetLastError() != cudaSuccess) return KEP_ERR_CUDA;
  for (int g = 0; g < G; ++g) {
    const long long* r = F.h_red + 6 * g;
    out[g].neg = r[0];
    out[g].zero = r[1];
    out[g].pos = r[2];
    out[g].delayed = r[3];
    status_bits[g] = static_cast<int>(r[4]);
  }
  return KEP_OK;
}

}  // namespace kep
