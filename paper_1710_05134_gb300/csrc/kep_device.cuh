// Device-side helpers shared by the library's kernels.
#pragma once

#include <cstdint>

#include "kep_internal.h"

namespace kep {

#define KEP_HD __host__ __device__ __forceinline__
#define KEP_D __device__ __forceinline__

// shift of batch entry b (entries of a multisection step carry one; a single factorization: 0)
KEP_D int32_t entry_shift(const Batch& B, int32_t b) { return B.sh ? B.sh[b] : 0; }

// Element (i, j), i >= j, of a front stored as L storage (columns < p, ld = ldL) plus a
// contribution block (columns >= p, c x c).
struct FrontView {
  double* L;
  double* C;
  int64_t ldL;
  int32_t p, m, c;
  KEP_D double* at(int32_t i, int32_t j) const {
    return j < p ? L + static_cast<int64_t>(j) * ldL + i
                 : C + static_cast<int64_t>(j - p) * c + (i - p);
  }
};

KEP_D FrontView front_view(const FrontTables& T, const FactorSlot& S, double* cbpool, int32_t t,
                           int32_t d_in) {
  FrontView v;
  v.L = S.F + T.front_off[t];
  v.c = T.m_sym[t] - T.p_sym[t];
  v.C = T.cb_off[t] >= 0 ? cbpool + T.cb_off[t] : nullptr;
  v.ldL = T.m_alloc[t];
  v.p = T.p_sym[t] + d_in;
  v.m = T.m_sym[t] + d_in;
  return v;
}

// Contribution block of a factored child, read as a (dout + csym)-order lower triangle:
// index q < dout are the child's delayed columns (still in its L storage), q >= dout its
// symbolic contribution rows (in the pool).
struct ChildCB {
  const double* L;
  const double* C;
  int64_t ldL;
  int32_t nel, dout, csym;
  KEP_D double get(int32_t qi, int32_t qj) const {   // qi >= qj
    return qj < dout ? L[static_cast<int64_t>(nel + qj) * ldL + nel + qi]
                     : C[static_cast<int64_t>(qj - dout) * csym + (qi - dout)];
  }
  KEP_D int32_t size() const { return dout + csym; }
};

KEP_D ChildCB child_cb(const FrontTables& T, const FactorSlot& S, const double* cbpool, int32_t ch) {
  ChildCB v;
  v.L = S.F + T.front_off[ch];
  v.C = T.cb_off[ch] >= 0 ? cbpool + T.cb_off[ch] : nullptr;
  v.ldL = T.m_alloc[ch];
  v.nel = S.nelim[ch];
  v.dout = S.d_out[ch];
  v.csym = T.m_sym[ch] - T.p_sym[ch];
  return v;
}

// Parent assembly position of a child's contribution index q.
KEP_D int32_t parent_pos(const FrontTables& T, int32_t ch, int32_t q, int32_t dout, int32_t off_c,
                         int32_t d_in_parent) {
  return q < dout ? off_c + q : d_in_parent + T.relmap[T.relmap_ptr[ch] + (q - dout)];
}

KEP_D double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

KEP_D double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Inertia of one pivot: 1x1 d, or 2x2 [a b; b c] by the sign of det and trace.
KEP_D void count_pivot1(double d, int32_t& neg, int32_t& zero, int32_t& pos) {
  if (d < 0) ++neg; else if (d > 0) ++pos; else ++zero;
}
KEP_D void count_pivot2(double a, double b, double c, int32_t& neg, int32_t& zero, int32_t& pos) {
  double det = a * c - b * b, tr = a + c;
  if (det < 0) { ++neg; ++pos; return; }
  if (det > 0) { if (tr < 0) neg += 2; else pos += 2; return; }
  if (tr < 0) { ++neg; ++zero; } else if (tr > 0) { ++pos; ++zero; } else zero += 2;
}

}  // namespace kep
